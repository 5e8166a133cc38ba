// Device-side helpers shared by the library's kernels: lattice geometry,
// levels, the DD predictors of order 2P (Sec. 2.4) and the collocation
// stencils' weights (Sec. 2.5).
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
    int P;       // DD order 2P (Sec. 2.4): P = 2, 3 or 4
};

constexpr int kMaxP = 4;   // highest DD half-order (2p = 8)

// ---- DD order-2P tables (Sec. 2.4 predictor, Sec. 2.5 derivatives) --------
// Predictor: the polynomial of degree 2P - 1 through the coarser neighbours
// at +-1, +-3, .., +-(2P - 1) evaluated at 0; weight of the pair at
// +-(2k + 1) = dd_pred(P, k) * 2^-dd_shift(P):
//   2p = 4: (9, -1) / 2^4;  2p = 6: (150, -25, 3) / 2^8;
//   2p = 8: (1225, -245, 49, -5) / 2^11.
// First derivative (Sec. 2.5): the derivative of the DD interpolant at a
// collocation point, D u = sum_j -phi'(j) (u_j - u_-j) / h with phi'(j) the
// scaling function's derivative at the integers,
//   2p = 4: phi'(1..2) = -2/3, 1/12              -> (8, -1) / 12
//   2p = 6: phi'(1..4) = -272/365, 53/365, -16/1095, -1/2920
//                                                 -> (6528, -1272, 128, 3) / 8760
//   2p = 8: phi'(1..6) = -39296/49553, 76113/396424, -1664/49553,
//           2645/1189272, 128/743295, -1/1189272
//           -> (4715520, -1141695, 199680, -13225, -1024, 5) / 5946360
// (numerator j = dd_d1(P, j), j = 1 .. 2P - 2, denominator dd_d1den(P)).
// Second derivative: the central stencil of order 2P on 2P + 1 points,
// (n_0 u + sum_j n_j (u_j + u_-j)) / (d h^2):
//   2p = 4: (-30; 16, -1) / 12;  2p = 6: (-490; 270, -27, 2) / 180;
//   2p = 8: (-14350; 8064, -1008, 128, -9) / 5040
// (n_j = dd_d2(P, j), j = 0 .. P, denominator dd_d2den(P)).
// The integers are exact in FP32 and FP64.
__host__ __device__ constexpr double dd_pred(int P, int k) {
    return P == 2 ? (k == 0 ? 9.0 : -1.0)
         : P == 3 ? (k == 0 ? 150.0 : k == 1 ? -25.0 : 3.0)
                  : (k == 0 ? 1225.0 : k == 1 ? -245.0 : k == 2 ? 49.0 : -5.0);
}
__host__ __device__ constexpr int dd_shift(int P) { return P == 2 ? 4 : P == 3 ? 8 : 11; }
__host__ __device__ constexpr int dd_reach1(int P) { return 2 * P - 2; }
__host__ __device__ constexpr int dd_reach(int P) { return 2 * P - 2 > P ? 2 * P - 2 : P; }
__host__ __device__ constexpr double dd_d1(int P, int j) {
    return P == 2 ? (j == 1 ? 8.0 : -1.0)
         : P == 3 ? (j == 1 ? 6528.0 : j == 2 ? -1272.0 : j == 3 ? 128.0 : 3.0)
                  : (j == 1 ? 4715520.0 : j == 2 ? -1141695.0 : j == 3 ? 199680.0 : j == 4 ? -13225.0
                     : j == 5 ? -1024.0 : 5.0);
}
__host__ __device__ constexpr double dd_d1den(int P) { return P == 2 ? 12.0 : P == 3 ? 8760.0 : 5946360.0; }
__host__ __device__ constexpr double dd_d2(int P, int j) {
    return P == 2 ? (j == 0 ? -30.0 : j == 1 ? 16.0 : -1.0)
         : P == 3 ? (j == 0 ? -490.0 : j == 1 ? 270.0 : j == 2 ? -27.0 : 2.0)
                  : (j == 0 ? -14350.0 : j == 1 ? 8064.0 : j == 2 ? -1008.0 : j == 3 ? 128.0 : -9.0);
}
__host__ __device__ constexpr double dd_d2den(int P) { return P == 2 ? 12.0 : P == 3 ? 180.0 : 5040.0; }
// Longest ghost interpolation row over the active points (per DD order).
__host__ __device__ constexpr int dd_row_max(int P) { return P == 2 ? 64 : P == 3 ? 128 : 256; }

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

// DD order-2P predictor from the neighbours at -+(2k + 1) (lo[k], hi[k]),
// k = 0 .. P - 1, with integer numerators: s = c_0 (lo_0 + hi_0), then
// s = s + c_k (lo_k + hi_k), then s 2^-shift, every operation rounded.  For
// P = 2 it is dd4 (c_1 = -1 makes the addition a subtraction).
template <typename T, int P>
__device__ __forceinline__ T ddp(const T (&lo)[P], const T (&hi)[P]) {
    if constexpr (P == 2) {
        return dd4<T>(lo[0], hi[0], lo[1], hi[1]);
    } else {
        T acc = rmul(T(dd_pred(P, 0)), radd(lo[0], hi[0]));
#pragma unroll
        for (int k = 1; k < P; ++k) acc = radd(acc, rmul(T(dd_pred(P, k)), radd(lo[k], hi[k])));
        return rmul(acc, T(1.0 / (double)(1 << dd_shift(P))));
    }
}

// 1-D DD prediction of order 2P along x (alongx) or y at (i, k), coarse
// neighbours at odd multiples of s.
template <typename T, int P, bool CG>
__device__ __forceinline__ T predict_line(const T* __restrict__ F, int i, int k, int s, bool alongx,
                                          const Geom& g) {
    T lo[P], hi[P];
    const int m = g.mask;
#pragma unroll
    for (int q = 0; q < P; ++q) {
        const int o = (2 * q + 1) * s;
        if (alongx) {
            const T* row = F + ((size_t)k << g.L);
            lo[q] = ldv<T, CG>(row + ((i - o) & m));
            hi[q] = ldv<T, CG>(row + ((i + o) & m));
        } else {
            lo[q] = ldv<T, CG>(F + ((size_t)((k - o) & m) << g.L) + i);
            hi[q] = ldv<T, CG>(F + ((size_t)((k + o) & m) << g.L) + i);
        }
    }
    return ddp<T, P>(lo, hi);
}

// Order-2P DD prediction at (i, k) of level j (as predict, below).
template <typename T, int P, bool CG>
__device__ __forceinline__ T predict_p(const T* __restrict__ F, int i, int k, int j, const Geom& g) {
    const int sh = g.J - j;
    const int s = 1 << sh;
    const bool oi = (i >> sh) & 1;
    const bool ok = (k >> sh) & 1;
    if (oi && !ok) return predict_line<T, P, CG>(F, i, k, s, true, g);
    if (!oi && ok) return predict_line<T, P, CG>(F, i, k, s, false, g);
    T lo[P], hi[P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
        const int o = (2 * q + 1) * s;
        lo[q] = predict_line<T, P, CG>(F, i, (k - o) & g.mask, s, true, g);
        hi[q] = predict_line<T, P, CG>(F, i, (k + o) & g.mask, s, true, g);
    }
    return ddp<T, P>(lo, hi);
}

// DD order-4 prediction at lattice point (i, k) of level j >= 1 from the
// coarser points of field F: along x for points odd in x only, along y for
// points odd in y only, tensor product (x prediction of four rows, then y)
// otherwise.
template <typename T, bool CG = false>
__device__ __forceinline__ T predict_dd4(const T* __restrict__ F, int i, int k, int j, const Geom& g) {
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

// DD prediction of order 2 g.P at (i, k) of level j >= 1 (the tensor product
// for points odd in both directions: x predictions of the 2P rows, then y).
template <typename T, bool CG = false>
__device__ __forceinline__ T predict(const T* __restrict__ F, int i, int k, int j, const Geom& g) {
    if (g.P == 3) return predict_p<T, 3, CG>(F, i, k, j, g);
    if (g.P == 4) return predict_p<T, 4, CG>(F, i, k, j, g);
    return predict_dd4<T, CG>(F, i, k, j, g);
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
