// Device-side helpers shared by the library's kernels: lattice geometry,
// levels, the DD4 predictor (Sec. 2.4) and the collocation stencils (Sec. 2.5).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace wrc {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 152 * 8;   // grid-stride cap: 8 resident blocks per SM
constexpr int kMaxKeys = 16;          // compaction buckets (active + ghosts per level)
constexpr int kTileRounds = 16;       // compaction: points per thread (16, one 16-byte load per mask)
constexpr int kTile = kThreads * kTileRounds;

// Finest-lattice geometry.  NJ is a power of two; p = k*NJ + i.
struct Geom {
    int NJ;      // points per direction
    int L;       // log2(NJ)
    int J;       // number of refinement levels
    int mask;    // NJ - 1
    double h;    // h_J = 2 pi / NJ
};

// Level of lattice point (i, k): 0 when both are multiples of 2^J, else the
// level at which the point is first inserted, J - min(tz(i), tz(k), J).
__host__ __device__ __forceinline__ int level_of(int i, int k, int J) {
#ifdef __CUDA_ARCH__
    return J - (__ffs((unsigned)(i | k) | (1u << J)) - 1);
#else
    unsigned v = (unsigned)(i | k) | (1u << J);
    int t = 0;
    while (!(v & 1u)) { v >>= 1; ++t; }
    return J - t;
#endif
}

// Arithmetic with explicit IEEE rounding (no FMA contraction), so that the
// predictor and the details are bit-identical to a plain evaluation of
// (9*(a+b) - (c+d)) * 0.0625.
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double rsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }

// CG = true: an L2-only load (L1 is not coherent across SMs), for data that
// other blocks of a running kernel may write without an acquire ordering it;
// the Krylov kernel uses plain loads, ordered by its grid barrier's acquire.
template <typename T, bool CG>
__device__ __forceinline__ T ldv(const T* p) {
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

// DD order-4 predictor from the neighbours at -1, +1 (a, b) and -3, +3 (c, d):
// the cubic through them evaluated at 0, weights (-1, 9, 9, -1)/16.
template <typename T>
__device__ __forceinline__ T dd4(T a, T b, T c, T d) {
    return rmul(rsub(rmul(T(9), radd(a, b)), radd(c, d)), T(0.0625));
}

// DD prediction at lattice point (i, k) of level j >= 1 from the coarser
// points of field F: along x for points odd in x only, along y for points odd
// in y only, tensor product (x prediction of four rows, then y) otherwise.
template <typename T, bool CG = false>
__device__ __forceinline__ T predict(const T* __restrict__ F, int i, int k, int j, const Geom& g) {
    const int sh = g.J - j;
    const int s = 1 << sh;
    const int m = g.mask;
    const bool oi = (i >> sh) & 1;
    const bool ok = (k >> sh) & 1;
    if (oi && !ok) {
        const T* row = F + ((size_t)k << g.L);
        return dd4<T>(ldv<T, CG>(row + ((i - s) & m)), ldv<T, CG>(row + ((i + s) & m)),
                      ldv<T, CG>(row + ((i - 3 * s) & m)), ldv<T, CG>(row + ((i + 3 * s) & m)));
    }
    if (!oi && ok) {
        return dd4<T>(ldv<T, CG>(F + ((size_t)((k - s) & m) << g.L) + i), ldv<T, CG>(F + ((size_t)((k + s) & m) << g.L) + i),
                      ldv<T, CG>(F + ((size_t)((k - 3 * s) & m) << g.L) + i),
                      ldv<T, CG>(F + ((size_t)((k + 3 * s) & m) << g.L) + i));
    }
    T r[4];
    const int ks[4] = {k - s, k + s, k - 3 * s, k + 3 * s};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const T* row = F + ((size_t)(ks[q] & m) << g.L);
        r[q] = dd4<T>(ldv<T, CG>(row + ((i - s) & m)), ldv<T, CG>(row + ((i + s) & m)),
                      ldv<T, CG>(row + ((i - 3 * s) & m)), ldv<T, CG>(row + ((i + 3 * s) & m)));
    }
    return dd4<T>(r[0], r[1], r[2], r[3]);
}

// Number of level-j points (j >= 1): the stride-2^(J-j) sublattice minus the
// stride-2^(J-j+1) one.
__host__ __device__ __forceinline__ long long level_count(int j, const Geom& g) {
    const long long n = g.NJ >> (g.J - j);
    return n * n - (n / 2) * (n / 2);
}

// t-th level-j point: first the odd sublattice rows (all columns), then the
// even rows (odd columns), each in row-major order.
// (n = NJ / 2^(J-j) is a power of two, so the divisions are shifts; t < NJ^2 < 2^24.)
__device__ __forceinline__ void level_point(long long t, int j, const Geom& g, int& i, int& k) {
    const int sh = g.J - j;
    const int ln = g.L - sh;                 // log2 n
    const int n = 1 << ln;
    const int tt = (int)t;
    const int half = n << (ln - 1);          // n * n/2
    int ic, kr;
    if (tt < half) {
        kr = 2 * (tt >> ln) + 1;
        ic = tt & (n - 1);
    } else {
        const int u = tt - half;
        kr = 2 * (u >> (ln - 1));
        ic = 2 * (u & ((n >> 1) - 1)) + 1;
    }
    i = ic << sh;
    k = kr << sh;
}

// Packed per-active-point word: lattice index (24 bits) and the stencil
// levels j*_x, j*_y (4 bits each).
__host__ __device__ __forceinline__ uint32_t pack_meta(int p, int jx, int jy) {
    return (uint32_t)p | ((uint32_t)jx << 24) | ((uint32_t)jy << 28);
}
__host__ __device__ __forceinline__ int meta_pos(uint32_t m) { return (int)(m & 0xFFFFFFu); }
__host__ __device__ __forceinline__ int meta_jx(uint32_t m) { return (int)((m >> 24) & 15u); }
__host__ __device__ __forceinline__ int meta_jy(uint32_t m) { return (int)(m >> 28); }

// Effective item count of a launch: from device memory when dn is given (the
// launch then covers a capacity n >= *dn with a grid-stride loop, so it can
// be captured in a CUDA graph), else n.
__device__ __forceinline__ long long eff_n(const int* dn, long long n) { return dn ? (long long)*dn : n; }

// Process-wide count of kernel launches made by the library (host side).
void note_launch();
long long launches_total();

// Programmatic dependent launch.  The grid, flow and Poisson kernels are
// launched with launch_pdl, so that a kernel's blocks can be scheduled while
// its predecessor in the stream drains; each such kernel calls pdl_wait()
// before touching global memory (it returns once the predecessor has
// completed and its writes are visible; without the launch attribute it
// returns at once) and pdl_trigger() after its work, which lets the
// successor's launch begin.  Measured ~1 us saved per kernel boundary.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, (KArgs)args...);
}

inline int blocks_for(long long n, int threads = kThreads) {
    long long b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > kMaxBlocks) b = kMaxBlocks;
    return (int)b;
}

}  // namespace wrc
