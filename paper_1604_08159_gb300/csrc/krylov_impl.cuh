#pragma once
// Device code of the Krylov projection of the time step (Sec. 2.1: the discrete system projected
// onto a Krylov subspace): one persistent cooperative kernel per step,
//   b = A_n omega + g,  beta = |b|,  v_0 = b / beta,
//   Arnoldi with classical Gram-Schmidt applied twice, the second pass
//   delayed by one step (FP64 inner products, deterministic reductions; the
//   norm after the second pass from |u|^2 - |s|^2), happy breakdown when
//   h_{j+1,j} <= tol |A v_j|, then, in the same launch, y = phi_1(dt H_k) e_1
//   from the exponential of the augmented Hessenberg matrix (block 0), one
//   more grid barrier, and omega <- omega + dt beta V_k y (every block, its
//   own points).
// Ghost values of each new basis vector come from exact interpolation rows
// over the active points.  One Arnoldi step takes two phases: the operator
// and all dots of the step | the scalars, the new vectors and their ghost
// values.  Phases are separated by a grid barrier with a bounded wait; every
// block reduces the per-block partial sums itself, in the same order, so all
// blocks hold identical coefficients and take identical breakdown decisions.
// On this part one warp issues at most one FP64 instruction per ~64 cycles
// (about one per 19 cycles per SM), so the kernel is organised around the
// count of FP64 instructions each warp issues and the latency of dependent
// steps, not around bytes.
#include <cooperative_groups.h>

#include <cstdlib>

#include <type_traits>

#include "kernels.h"
#include "operator.cuh"

namespace wrc {

namespace {

constexpr int kPT = 128;      // threads per block of the single-run kernel
constexpr int kNV = 32;       // accumulator slots: basis vectors per pass (<= m + 1 <= 32)
constexpr int kOutP = 66;     // partial sums per block: two sets of (kNV dots + one product)
constexpr int kGhostLanes = 8;   // lanes per ghost value (ghost_values, ghost_step)
constexpr int kGatherLane = 8;   // row terms per lane fetched ahead of their additions
static_assert(kGhostLanes * kGatherLane == kGhostRowMax, "one gather pass covers a whole interpolation row");
constexpr int kCacheGroups = 16; // ghosts per block whose interpolation rows are kept in shared memory

// Shared-memory copy of the interpolation rows of a block's first
// kCacheGroups ghosts (ghost bid + nb q in slot q).
struct RowCache {
    int* len;
    int* idx;      // kCacheGroups x kGhostRowMax
    double* w;
};

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Calls f(std::integral_constant<int, t>) for t = n-1, n-2, ..., 0 (0 <= n <= N
// <= 32): one jump into an unrolled sequence, so that the calls with t >= n
// issue no instructions at all.  (A loop "if (t < n)" over all N unrolled
// iterations becomes predicated instructions, and a predicated-off FP64
// instruction still takes its ~64 issue cycles on this part; a "break" in the
// loop keeps it from being unrolled, sending indexed accumulators to local
// memory.)
template <int N, typename F>
__device__ __forceinline__ void down_from(int n, F&& f) {
    static_assert(N >= 1 && N <= 32, "down_from covers at most 32 calls");
    switch (n) {
#define WRC_DOWN(t)                                            \
    case (t) + 1:                                              \
        if constexpr ((t) < N) f(std::integral_constant<int, (t)>{}); \
        [[fallthrough]];
        WRC_DOWN(31) WRC_DOWN(30) WRC_DOWN(29) WRC_DOWN(28) WRC_DOWN(27) WRC_DOWN(26) WRC_DOWN(25) WRC_DOWN(24)
        WRC_DOWN(23) WRC_DOWN(22) WRC_DOWN(21) WRC_DOWN(20) WRC_DOWN(19) WRC_DOWN(18) WRC_DOWN(17) WRC_DOWN(16)
        WRC_DOWN(15) WRC_DOWN(14) WRC_DOWN(13) WRC_DOWN(12) WRC_DOWN(11) WRC_DOWN(10) WRC_DOWN(9) WRC_DOWN(8)
        WRC_DOWN(7) WRC_DOWN(6) WRC_DOWN(5) WRC_DOWN(4) WRC_DOWN(3) WRC_DOWN(2) WRC_DOWN(1) WRC_DOWN(0)
#undef WRC_DOWN
        default:
            break;
    }
}

// Sum of x over the 32 lanes of a warp, returned to every lane, through 40
// doubles of shared memory ws in a fixed order: lane l < 8 adds lanes
// 4l..4l+3 pairwise, then every lane adds the eight sums pairwise.  Inside
// this kernel a shuffle tree on FP64 values was measured at ~600 cycles per
// level on this part; this takes 4 dependent FP64 additions and shared
// memory round trips.
__device__ __forceinline__ double warp_sum(double x, double* ws) {
    const int l = threadIdx.x & 31;
    ws[l] = x;
    __syncwarp();
    if (l < 8) ws[32 + l] = (ws[4 * l] + ws[4 * l + 1]) + (ws[4 * l + 2] + ws[4 * l + 3]);
    __syncwarp();
    const double* p = ws + 32;
    const double r = ((p[0] + p[1]) + (p[2] + p[3])) + ((p[4] + p[5]) + (p[6] + p[7]));
    __syncwarp();
    return r;
}

// Sums over each group of kGhostLanes (= 8) consecutive lanes of the NV
// values v[] of every lane, through NV * 32 doubles of shared memory ws: lane
// gl < NV of a group adds quantity gl of its group pairwise (7 FP64 additions
// for all quantities at once), and lane 0 of the group receives the sums in
// v[].  Same order in every block.
template <int NV>
__device__ __forceinline__ void group_sums(double (&v)[NV], double* ws) {
    static_assert(kGhostLanes == 8 && NV <= 8, "groups of eight lanes");
    const int lane = threadIdx.x & 31, gl = lane & 7, g8 = lane - gl;
#pragma unroll
    for (int q = 0; q < NV; ++q) ws[q * 32 + lane] = v[q];
    __syncwarp();
    double sum = 0.0;
    if (gl < NV) {
        const double* p = ws + gl * 32 + g8;
        sum = ((p[0] + p[1]) + (p[2] + p[3])) + ((p[4] + p[5]) + (p[6] + p[7]));
    }
    __syncwarp();
    if (gl < NV) ws[gl * 32 + g8] = sum;
    __syncwarp();
    if (gl == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) v[q] = ws[q * 32 + lane];
    __syncwarp();
}

// Grid-wide barrier for a cooperative launch: one atomic per block on a
// counter whose top bit flips when the last block arrives (block 0 adds
// 2^31 - (G - 1), the others 1, so each barrier adds exactly 2^31).  The
// arrival is a release atomic and the wait polls with acquire loads (GPU
// scope; the barrier's __syncthreads extend both to the whole block), so the
// plain loads of the next phase see every block's writes; this measured
// ~0.2 us faster per barrier than __threadfence around a relaxed atomic.
// The wait of each block is bounded by limit_ns; a block that runs out sets
// bit 1 of *err, and every waiter leaves as soon as one of the stopping bits
// (kErrStop) of *err is set, so the kernel always returns.  Bit 4 (16) only
// reports an unclustered run of a clustered launch and stops nothing.
// The barrier spans the nb blocks of one problem (bid = block index within it).
// With a trace buffer, the arrival of each block and the release of block 0
// are stamped (phase index `ph`, counted by the caller).
constexpr int kErrStop = 2 | 4;   // a barrier wait ran out; a ghost row exceeded its capacity

__device__ bool grid_sync(unsigned* bar, int* err, unsigned long long limit_ns, int bid, int nb,
                          unsigned long long* trace = nullptr, int ph = 0) {
    __syncthreads();
    if (threadIdx.x == 0) {
        if (trace && ph < kTracePhases) trace[1 + (size_t)ph * (nb + 1) + bid] = gtimer();
        const unsigned inc = bid == 0 ? 0x80000000u - (unsigned)(nb - 1) : 1u;
        unsigned old;
        asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(bar), "r"(inc) : "memory");
        volatile int* verr = err;
        const unsigned long long t0 = gtimer();
        while (true) {
            unsigned cur;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(bar) : "memory");
            if ((old ^ cur) & 0x80000000u) break;
            if (*verr & kErrStop) break;
            if (gtimer() - t0 > limit_ns) {
                atomicOr(err, 2);
                break;
            }
        }
        if (trace && ph < kTracePhases && bid == 0) trace[1 + (size_t)ph * (nb + 1) + nb] = gtimer();
    }
    __syncthreads();
    return (*(volatile int*)err & kErrStop) == 0;
}

// Per-block sums of acc[0..ndots) into dst[0..ndots) and, with NORM, of
// acc[kNV] (a squared norm) into dst[ndots].  The first NS dot accumulators
// (NS = ndots rounded up to a power of two) are reduced across the warp by a
// reduce-scatter (NS - 1 exchanges; afterwards lane l holds the warp sum of
// accumulator l mod NS), the norm by a shuffle tree.  Every FP64 addition
// costs a warp ~64 cycles of issue on this part, so only the NS accumulators
// in use take part.
template <int PT, bool NORM>
__device__ __forceinline__ void block_partials(double (&acc)[kNV + 1], int ndots, double* dst,
                                               double (*s_red)[kNV + 1]) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (ndots > 0) {
        int ns = 1;
        while (ns < ndots) ns <<= 1;
#pragma unroll
        for (int s = 16; s >= 1; s >>= 1) {
            if (2 * s > ns) continue;
            const bool up = (lane & s) != 0;
#pragma unroll
            for (int i = 0; i < s; ++i) {
                const double send = up ? acc[i] : acc[i + s];
                const double keep = up ? acc[i + s] : acc[i];
                acc[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
            }
        }
        for (int s = ns; s < 32; s <<= 1) acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], s);
        if (lane < ns) s_red[wid][lane] = acc[0];
    }
    if (NORM) {
        double v = acc[kNV];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) s_red[wid][kNV] = v;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < ndots + (NORM ? 1 : 0); t += blockDim.x) {
        const int src = t < ndots ? t : kNV;
        double sum = 0.0;
        for (int q = 0; q < PT / 32; ++q) sum += s_red[q][src];
        dst[t] = sum;
    }
}

// Sum over all blocks of part[b * kOutP + t], t < nout (<= 64), into s_out.
// Up to 32 outputs, the lanes of a warp are split into L = 32 / ns groups
// (ns = nout rounded up to a power of two, so L > 1 only for 16 outputs or
// fewer): lane g ns + t of
// warp w adds output t of blocks w + 4 (g + L u), u = 0, 1, ... (for 4 warps),
// in order; the groups are then combined by shuffles and the warps' sums
// added in warp order.  Same order in every block.  A lane's loads go out
// kReduceBatch at a time ahead of their ordered additions, so one L2 round
// trip covers up to kReduceBatch partials per lane; the additions of a
// partial batch are entered by one jump (down_from: last partial first).  The partials were written by
// other blocks before the grid barrier, whose fences make plain loads see
// them (L1 is invalidated there).
constexpr int kReduceBatch = 24;

template <int PT>
__device__ __forceinline__ void reduce_all(const double* part, int nout, double* s_out,
                                           double (*s_red)[kNV + 1], int nb) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    constexpr int kW = PT / 32;
    if (nout > 32) {
        // two chunks: lane t adds outputs t and 32 + t (if any) of blocks
        // w, w + 4, ..., the loads of both going out together
        constexpr int kB = kReduceBatch / 2;
        const int t2 = 32 + lane;
        const bool has2 = t2 < nout;
        double v1 = 0.0, v2 = 0.0;
        const double* p = part + lane;
        int b = wid;
        for (; b + (kB - 1) * kW < nb; b += kB * kW) {
            double x1[kB], x2[kB];
#pragma unroll
            for (int u = 0; u < kB; ++u) {
                x1[u] = p[(size_t)(b + u * kW) * kOutP];
                x2[u] = has2 ? p[32 + (size_t)(b + u * kW) * kOutP] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < kB; ++u) {
                v1 += x1[u];
                v2 += x2[u];
            }
        }
        const int rest = b < nb ? (nb - 1 - b) / kW + 1 : 0;   // < kB
        double x1[kB], x2[kB];
#pragma unroll
        for (int u = 0; u < kB; ++u)
            if (u < rest) {
                x1[u] = p[(size_t)(b + u * kW) * kOutP];
                x2[u] = has2 ? p[32 + (size_t)(b + u * kW) * kOutP] : 0.0;
            }
        down_from<kB>(rest, [&](auto uc) {
            constexpr int u = decltype(uc)::value;
            v1 += x1[u];
            v2 += x2[u];
        });
        s_red[wid][lane] = v1;
        __syncthreads();
        for (int q = threadIdx.x; q < 32; q += blockDim.x) {
            double sum = 0.0;
            for (int w = 0; w < kW; ++w) sum += s_red[w][q];
            s_out[q] = sum;
        }
        __syncthreads();
        s_red[wid][lane] = v2;
        __syncthreads();
        for (int q = threadIdx.x; q < nout - 32; q += blockDim.x) {
            double sum = 0.0;
            for (int w = 0; w < kW; ++w) sum += s_red[w][q];
            s_out[32 + q] = sum;
        }
        __syncthreads();
        return;
    }
    int ns = 1;
    while (ns < nout) ns <<= 1;
    const int L = 32 / ns;
    const int t = lane & (ns - 1), g = lane / ns;
    const int bstep = kW * L;
    double v = 0.0;
    if (t < nout) {
        const double* p = part + t;
        int b = wid + kW * g;
        for (; b + (kReduceBatch - 1) * bstep < nb; b += kReduceBatch * bstep) {
            double x[kReduceBatch];
#pragma unroll
            for (int u = 0; u < kReduceBatch; ++u) x[u] = p[(size_t)(b + u * bstep) * kOutP];
#pragma unroll
            for (int u = 0; u < kReduceBatch; ++u) v += x[u];
        }
        const int rest = b < nb ? (nb - 1 - b) / bstep + 1 : 0;   // < kReduceBatch
        double x[kReduceBatch];
#pragma unroll
        for (int u = 0; u < kReduceBatch; ++u)
            if (u < rest) x[u] = p[(size_t)(b + u * bstep) * kOutP];
        down_from<kReduceBatch>(rest, [&](auto uc) { v += x[decltype(uc)::value]; });
    }
    // the L groups, added in group order by the lanes of group 0 (shared
    // memory rather than a shuffle tree: see warp_sum)
    s_red[wid][lane] = v;
    __syncwarp();
    if (L > 1) {
        double c = v;
        if (g == 0 && t < nout)
            for (int q = 1; q < L; ++q) c += s_red[wid][q * ns + t];
        __syncwarp();
        if (g == 0 && t < nout) s_red[wid][t] = c;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nout; q += blockDim.x) {
        double sum = 0.0;
        for (int w = 0; w < kW; ++w) sum += s_red[w][q];
        s_out[q] = sum;
    }
    __syncthreads();
}

// ---- phi_1 from the exponential of the augmented matrix ------------------
// y = phi_1(dt H_k) e_1 is the upper part of the last column of exp(M),
// M = [[dt H_k, e_1], [0, 0]] ((k+1) x (k+1)).  That column, exp(M) e_k, is
// computed as the action of the exponential by scaling and the truncated
// Taylor series: B = M / s, x <- sum_{i<=m} B^i x / i!  applied s times.
// With theta = |M|_inf / s (max row sum; the bound only needs a
// sub-multiplicative norm) the dropped tail is at most
// sum_{i>m} theta^i / i! of |x|, and (theta, m) is taken from
//   (1/4, 12), (1/2, 15), (1, 18), (2, 24), (4, 32),
// each pair keeping that tail below 1e-17, as the one with the fewest
// matrix-vector products s m (s = max(1, ceil(|M|_inf / theta))).  exp(B)
// shrinks no vector by more than e^-theta, so the relative truncation error
// is below 6e-16 per sub-step.  Each product is 32 x 32 in FP64 on one SM,
// so their count matters.  One warp, lane r holds row r.
constexpr int kPhiChoices = 5;
__constant__ double c_phi_theta[kPhiChoices] = {0.25, 0.5, 1.0, 2.0, 4.0};
__constant__ int c_phi_terms[kPhiChoices] = {12, 15, 18, 24, 32};
constexpr int kTaylorMax = 32;
__constant__ double c_inv[kTaylorMax + 1] = {
    0.0,       1.0 / 1,  1.0 / 2,  1.0 / 3,  1.0 / 4,  1.0 / 5,  1.0 / 6,  1.0 / 7,  1.0 / 8,
    1.0 / 9,   1.0 / 10, 1.0 / 11, 1.0 / 12, 1.0 / 13, 1.0 / 14, 1.0 / 15, 1.0 / 16, 1.0 / 17,
    1.0 / 18,  1.0 / 19, 1.0 / 20, 1.0 / 21, 1.0 / 22, 1.0 / 23, 1.0 / 24, 1.0 / 25, 1.0 / 26,
    1.0 / 27,  1.0 / 28, 1.0 / 29, 1.0 / 30, 1.0 / 31, 1.0 / 32};

// Largest norm of the Taylor evaluation: a step with |dt H| above it (or not
// finite) has blown up; phi_1 is then not evaluated, y is set to NaN and the
// non-finite flag is raised, so that the step fails cleanly instead of
// looping over an unbounded number of sub-steps.
constexpr double kMaxPhiScale = 4096.0;

// phi_1 by one block of PT threads: lane r of warp w holds row r of M over
// the column group w (32 / (PT/32) columns); each product B x is summed per
// group, then over the groups by warp 0, which keeps x and the partial sum of
// the series (the four FP64 sub-pipes of the SM share the products).
// s_part: [PT/32][>= 32], s_x: [>= 32], s_int: [3]; y (m entries) in global memory.
template <int PT>
__device__ __forceinline__ void phi1_block(const double* __restrict__ H, int k, int m, double dt,
                                           double* __restrict__ y, int* __restrict__ flags,
                                           double (*s_part)[kNV + 1], double* s_x, int* s_int) {
    constexpr int G = PT / 32;
    constexpr int CPG = 32 / G;
    const int r = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int c0 = w * CPG;
    double row[CPG];
    double rs = 0.0;
#pragma unroll
    for (int cc = 0; cc < CPG; ++cc) {
        const int c = c0 + cc;
        double v = 0.0;
        if (r < k && c < k) v = dt * H[(size_t)r * m + c];
        if (r == 0 && c == k) v = 1.0;
        row[cc] = v;
        rs += fabs(v);
    }
    s_part[w][r] = rs;
    __syncthreads();
    if (w == 0) {
        double t = 0.0;   // |row r|_1
        for (int q = 0; q < G; ++q) t += s_part[q][r];
        double nrm = t;   // |M|_inf
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nrm = fmax(nrm, __shfl_xor_sync(0xffffffffu, nrm, o));
        const bool blown = __any_sync(0xffffffffu, !(t == t)) || !(nrm <= kMaxPhiScale);
        if (r == 0) {
            int sb = 1, mb = kTaylorMax;
            if (!blown) {
                long best = 1L << 40;
                for (int q = 0; q < kPhiChoices; ++q) {
                    const int sq = nrm > c_phi_theta[q] ? (int)ceil(nrm / c_phi_theta[q]) : 1;
                    const long cost = (long)sq * c_phi_terms[q];
                    if (cost < best) {
                        best = cost;
                        sb = sq;
                        mb = c_phi_terms[q];
                    }
                }
            }
            s_int[0] = blown ? 1 : 0;
            s_int[1] = sb;
            s_int[2] = mb;
        }
    }
    __syncthreads();
    const int blown = s_int[0], s = s_int[1], mt = s_int[2];
    if (blown) {
        if (threadIdx.x == 0) atomicOr(flags, 1);
        for (int t = threadIdx.x; t < m; t += PT) y[t] = t < k ? __longlong_as_double(0x7ff8000000000000ll) : 0.0;
        return;
    }
    if (s > 1) {
        const double inv_s = 1.0 / s;
#pragma unroll
        for (int cc = 0; cc < CPG; ++cc) row[cc] *= inv_s;
    }
    double x = (w == 0 && r == k) ? 1.0 : 0.0;   // meaningful in warp 0
    for (int q = 0; q < s; ++q) {
        double acc = x;
        if (w == 0) s_x[r] = x;
        __syncthreads();
        for (int i = 1; i <= mt; ++i) {
            double pr = 0.0;
#pragma unroll
            for (int cc = 0; cc < CPG; ++cc) pr += row[cc] * s_x[c0 + cc];
            s_part[w][r] = pr;
            __syncthreads();
            if (w == 0) {
                double t = s_part[0][r];
                for (int g = 1; g < G; ++g) t += s_part[g][r];
                t *= c_inv[i];
                acc += t;
                s_x[r] = t;
            }
            __syncthreads();
        }
        x = acc;
    }
    if (w == 0 && r < m) y[r] = r < k ? x : 0.0;
}

// True for a finite double (exponent field not all ones), by integer
// operations on its high word (an FP64 comparison would take a warp's FP64
// issue slot for ~64 cycles).
__device__ __forceinline__ bool finite_bits(double x) { return ((__double2hiint(x) >> 20) & 0x7ff) != 0x7ff; }

// Exact float -> double by integer operations on the bits (sign, exponent
// rebiased by 1023 - 127, mantissa shifted by 29; infinities and NaNs keep
// the all-ones exponent): the conversion instruction runs on the FP64 pipe,
// the scarce one on this part, at two to three FP64 operations' cost.  A
// float subnormal (never met in practice) takes the conversion instruction.
__device__ __forceinline__ double f2d_exact(float x) {
    const unsigned f = __float_as_uint(x);
    const unsigned e8 = (f >> 23) & 0xffu;
    const unsigned m = f & 0x7fffffu;
    if (e8 == 0u && m != 0u) return (double)x;
    const unsigned e11 = e8 == 0xffu ? 0x7ffu : (e8 == 0u ? 0u : e8 + (1023u - 127u));
    const unsigned hi = (f & 0x80000000u) | (e11 << 20) | (m >> 3);
    return __hiloint2double((int)hi, (int)(m << 29));
}
__device__ __forceinline__ double dbl(double x) { return x; }
__device__ __forceinline__ double dbl(float x) { return f2d_exact(x); }

// sqrt(q) and 1/sqrt(q) in FP64 for the normalisation of a new basis vector:
// an FP32 reciprocal square root as the seed, then two Newton-Raphson steps
// y <- y (3/2 - (q/2) y^2) in FP64 (each doubles the correct bits: ~22 -> ~44
// -> full precision), sqrt(q) = q y; three dependent FP64 operations per
// step.  FP64 division and square root are long instruction sequences on
// this part.  q outside [2^-99, 2^99] (or negative, or not finite) takes the
// library's sqrt and division; the range test is integer work on the
// exponent.
__device__ __forceinline__ void sqrt_and_rsqrt(double q, double& s, double& r) {
    const int hi = __double2hiint(q);
    const int e = (hi >> 20) & 0x7ff;
    if (hi >= 0 && e > 1023 - 99 && e < 1023 + 99) {
        const double hq = 0.5 * q;
        double y = (double)rsqrtf((float)q);
        y = y * fma(-hq, y * y, 1.5);
        y = y * fma(-hq, y * y, 1.5);
        r = y;
        s = q * y;
    } else {
        s = sqrt(q);
        r = 1.0 / s;
    }
}

// x - sum_{t < nv} c_t v_t for the basis values v_t = basis[t ld] of one
// point, in the bulk type: four interleaved partial sums of the projections
// (short dependency chains; FP64 issues one warp instruction per 16 cycles
// per SM on this part), then subtracted at once.
template <typename T>
__device__ __forceinline__ T project_out(T x, const T* __restrict__ col, long long ld, const double* c, int nv) {
    T p[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
    for (int t = 0; t < kNV; ++t)
        if (t < nv) p[t & 3] += col[(size_t)t * ld] * (T)c[t];
    return x - ((p[0] + p[1]) + (p[2] + p[3]));
}

// Ghost values of one Krylov vector.  The ghosts of a problem are dealt out
// round-robin over its blocks (ghost t to block t mod nb); inside a block
// each ghost goes to a group of kGhostLanes consecutive lanes, which split
// its interpolation row (row_idx/row_w over the active values x) and the
// correction sum_{q<nc} c_q Gb[q][t], fetch their terms kGatherLane at a time
// ahead of the additions, and combine the lane sums by shuffles.  Returns,
// for lane 0 of each group with a ghost, the value in *out and its index in
// *tg (-1 otherwise).  Called by every thread of the block (warp-uniform loop).

template <typename T, int PT, typename F>
__device__ __forceinline__ void ghost_values(const KrylovStepArgs& A, const T* __restrict__ x,
                                             const T* __restrict__ Gb, long long ldg, const double* c, int nc,
                                             int bid, int nb, double* ws, F&& emit) {
    constexpr int kGroups = PT / kGhostLanes;                 // ghosts per block per pass
    constexpr int kPerWarp = 32 / kGhostLanes;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int gl = lane % kGhostLanes;
    for (int q0 = wid * kPerWarp; bid + (long long)nb * q0 < A.ng; q0 += kGroups) {
        const long long tl = bid + (long long)nb * (q0 + lane / kGhostLanes);
        const bool valid = tl < A.ng;
        const int t = valid ? (int)tl : 0;
        const int rl = valid ? A.row_len[t] : 0;
        const size_t base = (size_t)t * A.rmax;
        double part = 0.0;
        for (int e0 = 0; e0 < A.rmax; e0 += kGhostLanes * kGatherLane) {
            if (!__any_sync(0xffffffffu, e0 < rl)) break;
            int id[kGatherLane];
            double wt[kGatherLane], xv[kGatherLane];
#pragma unroll
            for (int u = 0; u < kGatherLane; ++u) {
                const int e = e0 + gl + kGhostLanes * u;
                if (e < rl) {
                    id[u] = A.row_idx[base + e];
                    wt[u] = A.row_w[base + e];
                }
            }
#pragma unroll
            for (int u = 0; u < kGatherLane; ++u)
                if (e0 + gl + kGhostLanes * u < rl) xv[u] = dbl(x[id[u]]);
#pragma unroll
            for (int u = 0; u < kGatherLane; ++u)
                if (e0 + gl + kGhostLanes * u < rl) part += wt[u] * xv[u];
        }
        if (valid)
            for (int q = gl; q < nc; q += kGhostLanes) part -= c[q] * dbl(Gb[(size_t)q * ldg + t]);
        double pv[1] = {part};
        group_sums<1>(pv, ws);
        if (valid && gl == 0) emit(t, pv[0]);
    }
}

// Ghost values of step j of the delayed scheme (groups of kGhostLanes lanes
// per ghost, as ghost_values): q_j at ghost g, Gb_j = (Gu - sum_{q<j} s_q Gb_q) / h,
// then the next u there, Gu <- (rows . z - sum_{q<j} t_q Gb_q - qz Gb_j) / h
// (with the new Gb_j), also written into the lattice vector Lq.  The
// interpolation rows of the block's first kCacheGroups ghosts come from the
// shared-memory copy rc (made at the start of the launch: the rows do not
// change during it), the others from global memory.  The ghost's earlier
// values Gb_q are loaded first, and the FP64 products of both sums run for
// the warp's longest row and for q < j only (down_from), not as predicated
// instructions.
template <typename T, int PT, bool CACHE>
__device__ __forceinline__ void ghost_step(const KrylovStepArgs& A, const T* __restrict__ z, T* __restrict__ Gb,
                                           long long ldg, T* __restrict__ Gu, const double* s, const double* tv,
                                           double qz, int j, double hinv, T* __restrict__ Lq, int bid, int nb,
                                           double* ws, const RowCache& rc) {
    constexpr int kGroups = PT / kGhostLanes;
    constexpr int kPerWarp = 32 / kGhostLanes;
    constexpr int kHist = kNV / kGhostLanes;          // earlier values per lane
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int gl = lane % kGhostLanes;
    const int nh = (j + kGhostLanes - 1) / kGhostLanes;
    for (int q0 = wid * kPerWarp; bid + (long long)nb * q0 < A.ng; q0 += kGroups) {
        const int qg = q0 + lane / kGhostLanes;       // the ghost's slot in the block
        const long long tl = bid + (long long)nb * qg;
        const bool valid = tl < A.ng;
        const int t = valid ? (int)tl : 0;
        double gq[kHist];
#pragma unroll
        for (int u = 0; u < kHist; ++u) {
            const int q = gl + kGhostLanes * u;
            gq[u] = (valid && q < j) ? dbl(Gb[(size_t)q * ldg + t]) : 0.0;
        }
        double part = 0.0;   // rows . z, this lane's share
        if (CACHE && q0 < kCacheGroups) {   // warp-uniform
            const int rl = valid ? rc.len[qg] : 0;
            const int* ri = rc.idx + qg * kGhostRowMax;
            const double* rw = rc.w + qg * kGhostRowMax;
            int id[kGatherLane];
            double wt[kGatherLane], xv[kGatherLane];
#pragma unroll
            for (int u = 0; u < kGatherLane; ++u) {
                const int e = gl + kGhostLanes * u;
                id[u] = e < rl ? ri[e] : -1;
                wt[u] = e < rl ? rw[e] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < kGatherLane; ++u) xv[u] = id[u] >= 0 ? dbl(z[id[u]]) : 0.0;
            const int nu = __reduce_max_sync(0xffffffffu, (unsigned)((rl + kGhostLanes - 1) / kGhostLanes));
            down_from<kGatherLane>(nu, [&](auto uc) {
                constexpr int u = decltype(uc)::value;
                part += wt[u] * xv[u];
            });
        } else {
            const int rl = valid ? A.row_len[t] : 0;
            const size_t base = (size_t)t * A.rmax;
            for (int e0 = 0; e0 < A.rmax; e0 += kGhostLanes * kGatherLane) {
                if (!__any_sync(0xffffffffu, e0 < rl)) break;
                int id[kGatherLane];
                double wt[kGatherLane], xv[kGatherLane];
#pragma unroll
                for (int u = 0; u < kGatherLane; ++u) {
                    const int e = e0 + gl + kGhostLanes * u;
                    if (e < rl) {
                        id[u] = A.row_idx[base + e];
                        wt[u] = A.row_w[base + e];
                    }
                }
#pragma unroll
                for (int u = 0; u < kGatherLane; ++u)
                    if (e0 + gl + kGhostLanes * u < rl) xv[u] = dbl(z[id[u]]);
#pragma unroll
                for (int u = 0; u < kGatherLane; ++u)
                    if (e0 + gl + kGhostLanes * u < rl) part += wt[u] * xv[u];
            }
        }
        double ss = 0.0, cs = 0.0;
        down_from<kHist>(nh, [&](auto uc) {
            constexpr int u = decltype(uc)::value;
            const int q = gl + kGhostLanes * u;
            const double sq = q < j ? s[q] : 0.0, tq = q < j ? tv[q] : 0.0;
            ss += sq * gq[u];
            cs += tq * gq[u];
        });
        double pv[3] = {part, ss, cs};
        group_sums<3>(pv, ws);
        if (valid && gl == 0) {
            const T gbj = (T)((dbl(Gu[t]) - pv[1]) * hinv);
            const T gu = (T)((pv[0] - pv[2] - qz * dbl(gbj)) * hinv);
            Gb[(size_t)j * ldg + t] = gbj;
            Gu[t] = gu;
            Lq[A.glist[t]] = gu;
        }
    }
}

// The dots of Arnoldi step j >= 1 over the block's own points, with z = A u
// applied at each point first (with_z; z goes to zb), as block partial sums
// in dst: [q_0.u .. q_{j-1}.u, |u|^2] at 0..j and [q_0.z .. q_{j-1}.z, u.z]
// at j+1..2j+1 (the first j+1 only without z).  Transposed: the threads stage
// u and z of their points in shared memory, and each lane forms whole dot
// products over its warp's 32 points (x row r = q_r for r < j, u for r = j,
// loaded 16 bytes at a time), so the sum over the warp's points is part of
// the product loop and no reduction across lanes is needed: 32 (j < 16, u
// and z on separate half-warps) or 64 FP64 operations per lane and point
// batch, against j or 2j products plus ~31 additions per reduce-scatter
// with one product per point and lane.  The warps' sums are added in warp
// order.  With thread-block clusters of CL > 1 blocks, the blocks of a
// cluster leave their sums in shared memory (s_bp) and the cluster's block
// 0 adds them in rank order through distributed shared memory and writes
// the cluster's sums to dst: the grid-wide reduction then reads nb / CL
// partial sums instead of nb.  A clustered kernel whose launch did not form
// its clusters (formed false) writes each block's sums, as the unclustered
// kernel does.
template <typename T, int PT, int CL, int P>
__device__ __forceinline__ void step_dots(const KrylovStepArgs& A, int j, bool with_z, int bid, int nb, double* dst,
                                          double (*s_dot)[2 * kNV], double (*s_uz)[2][33], double* s_bp,
                                          bool formed) {
    const T* __restrict__ Ua = (const T*)A.Ua;
    const T* __restrict__ Va = (const T*)A.Va;
    const T* __restrict__ Lq = (const T*)A.Lq;
    const T* __restrict__ basis = (const T*)A.basis;
    const T* __restrict__ w = (const T*)A.w;
    T* __restrict__ zb = (T*)A.basis + (size_t)A.m * A.ld;
    const T nu = (T)A.nu, r = (T)A.r, c1J = (T)A.c1J, c2J = (T)A.c2J;
    const int n = A.n, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const bool split = j < 16;                         // rows 0..j fit a half-warp
    const int row = split ? (lane & 15) : lane;
    const bool zlane = split && lane >= 16;
    const bool act = row <= j && (with_z || !zlane);
    const T* __restrict__ xbase = row < j ? basis + (size_t)row * A.ld : w;
    constexpr int kV = 16 / sizeof(T);                 // values per 16-byte load
    using V = typename std::conditional<sizeof(T) == 8, double2, float4>::type;
    double accA = 0.0, accB = 0.0;
    for (int wb = bid * PT + wid * 32; wb < n; wb += nb * PT) {
        const int a = wb + lane;
        T u = T(0), z = T(0);
        if (a < n) {
            u = w[a];
            if (with_z) {
                z = apply_point<T, false, P>(Lq, A.meta[a], Ua[a], Va[a], nu, r, A.g, c1J, c2J);
                zb[a] = z;
            }
        }
        s_uz[wid][0][lane] = dbl(u);
        s_uz[wid][1][lane] = dbl(z);
        __syncwarp();
        if (act) {
            const int nv = n - wb;   // valid points of the batch (>= 1; all 32 when >= 32)
            const V* xr = reinterpret_cast<const V*>(xbase + wb);   // 16-byte aligned: ld and wb are multiples of 32
            const double* yA = s_uz[wid][zlane ? 1 : 0];
            const double* yB = s_uz[wid][1];
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                V xv[16 / kV];
#pragma unroll
                for (int q = 0; q < 16 / kV; ++q) xv[q] = xr[hh * (16 / kV) + q];
#pragma unroll
                for (int q = 0; q < 16 / kV; ++q) {
                    const T* xs = reinterpret_cast<const T*>(&xv[q]);
#pragma unroll
                    for (int e = 0; e < kV; ++e) {
                        const int p = hh * 16 + q * kV + e;
                        const double x = p < nv ? dbl(xs[e]) : 0.0;
                        accA += x * yA[p];
                        if (!split && with_z) accB += x * yB[p];
                    }
                }
            }
        }
        __syncwarp();
    }
    if (act) {
        if (split) s_dot[wid][zlane ? j + 1 + row : row] = accA;
        else {
            s_dot[wid][row] = accA;
            if (with_z) s_dot[wid][j + 1 + row] = accB;
        }
    }
    __syncthreads();
    const int nout = with_z ? 2 * j + 2 : j + 1;
    if (CL == 1 || !formed) {
        for (int t = threadIdx.x; t < nout; t += PT) {
            double sum = 0.0;
            for (int q = 0; q < PT / 32; ++q) sum += s_dot[q][t];
            dst[t] = sum;
        }
    } else {
        // Two cluster barriers per call.  The first (arrive and wait) makes
        // the blocks' sums visible to the cluster's block 0; the second is
        // arrived at once block 0 has read its peers (the peers arrive at
        // once) and waited for at the next call or at the kernel's end, so
        // that no block rewrites its s_bp, or exits, while block 0 may still
        // read it.  Every block of a cluster takes part in the same 2m
        // barriers whatever path it takes (cluster_finish).
        if (j > 1) __cluster_barrier_wait();
        for (int t = threadIdx.x; t < nout; t += PT) {
            double sum = 0.0;
            for (int q = 0; q < PT / 32; ++q) sum += s_dot[q][t];
            s_bp[t] = sum;
        }
        cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
        __cluster_barrier_arrive();
        __cluster_barrier_wait();
        if (cl.block_rank() == 0)
            for (int t = threadIdx.x; t < nout; t += PT) {
                double sum = s_bp[t];
#pragma unroll
                for (int r = 1; r < CL; ++r) sum += cl.map_shared_rank(s_bp, r)[t];
                dst[t] = sum;
            }
        __cluster_barrier_arrive();
    }
}

// End of a clustered launch: wait for the second barrier of the last
// step_dots call (if there was one), then take part in the cluster barriers
// of the calls this block did not make (a breakdown, a failed grid barrier,
// a refusal), so that every block of a cluster passes exactly 2m cluster
// barriers and none exits while a peer may still read its shared memory.
// (Only for a launch that formed its clusters.)
// Each of these waits ends: every block of the cluster reaches its own
// remaining barriers, all its grid-barrier waits being bounded.
__device__ __forceinline__ void cluster_finish(int calls, int m) {
    if (calls > 0) __cluster_barrier_wait();
    for (int c = calls; c < m; ++c) {
        __cluster_barrier_arrive();
        __cluster_barrier_wait();
        __cluster_barrier_arrive();
        __cluster_barrier_wait();
    }
}

// The Krylov step of one problem, run by its nb blocks (bid = this block's
// index among them; with clusters of CL blocks that the launch formed, nb is
// a multiple of CL and the cluster of block bid is bid / CL; a clustered
// kernel whose launch did not form them -- formed false -- runs as the
// unclustered one).  Returns the number of step_dots calls made (Arnoldi
// steps j >= 1 entered), for cluster_finish.
template <typename T, int PT, int CL, int P>
__device__ __forceinline__ int krylov_body(const KrylovStepArgs& A, const int bid, const int nb,
                                           const bool formed = CL > 1) {
    const int pgroups = (CL > 1 && formed) ? CL : 1;   // blocks per partial-sum row
    const T* __restrict__ Ua = (const T*)A.Ua;
    const T* __restrict__ Va = (const T*)A.Va;
    const T* __restrict__ ga = (const T*)A.ga;
    const T* __restrict__ Lb = (const T*)A.L;
    T* __restrict__ Lq = (T*)A.Lq;
    T* __restrict__ basis = (T*)A.basis;
    T* __restrict__ w = (T*)A.w;
    T* __restrict__ Gb = (T*)A.Gb;
    __shared__ double s_red[PT / 32][kNV + 1];
    __shared__ double s_ws[PT / 32][96];   // warp_sum and group_sums scratch
    __shared__ double s_h[kOutP];
    __shared__ double s_c[kNV];
    __shared__ double s_sc[4];   // beta, 1/beta, h_{j+1,j}, 1/h_{j+1,j}
    __shared__ int s_int[3];     // phi_1: blown up, sub-steps, Taylor terms; Arnoldi: sums finite
    __shared__ double sH[kNV][kNV + 1];   // H, held by every block
    __shared__ double s_tmp[4];           // h^2, breakdown threshold on h^2, h qz of a step
    __shared__ double s_dot[PT / 32][2 * kNV];   // the warps' dot sums of a step
    __shared__ double s_uz[PT / 32][2][33];      // u and z of a warp's points
    __shared__ double s_bp[CL > 1 ? kOutP : 1];  // the block's dot sums (clusters)
    __shared__ T s_hT[kOutP];                    // s and t of a step in the bulk type
    __shared__ int s_glen[kCacheGroups];
    __shared__ int s_gidx[kCacheGroups * kGhostRowMax];
    __shared__ double s_gwt[kCacheGroups * kGhostRowMax];
    const RowCache rc{s_glen, s_gidx, s_gwt};
    const int n = A.n;
    const int stride = nb * PT;
    const int a0 = bid * PT + threadIdx.x;
    const bool lead = bid == 0 && threadIdx.x == 0;
    double* P0 = A.part;
    const T nu = (T)A.nu, r = (T)A.r, c1J = (T)A.c1J, c2J = (T)A.c2J;
    const int m = A.m;
    const long long ld = A.ld, ldg = A.ldg;
    double acc[kNV + 1];
    int ph = 0;   // grid barriers passed (phase trace)
    if (lead && A.trace) A.trace[0] = gtimer();
    int calls = 0;   // step_dots calls made
    if (*(volatile const int*)A.row_overflow) {
        if (lead) atomicOr(A.err, 4);
        return calls;
    }
    if (bid == 0)   // H is written by this block only
        for (int t = threadIdx.x; t < (m + 1) * m; t += blockDim.x) A.H[t] = 0.0;
    // the interpolation rows of the block's first kCacheGroups ghosts (order
    // 2P = 4 only, whose rows hold at most kGhostRowMax terms; A.rmax is then
    // kGhostRowMax; read at the first use after the barrier below)
    for (int e = threadIdx.x; P == 2 && e < kCacheGroups * kGhostRowMax; e += PT) {
        const int q = e / kGhostRowMax, i = e - q * kGhostRowMax;
        const long long t = bid + (long long)nb * q;
        const int rl = t < A.ng ? A.row_len[t] : 0;
        if (i == 0) s_glen[q] = rl;
        if (i < rl) {
            s_gidx[e] = A.row_idx[(size_t)t * A.rmax + i];
            s_gwt[e] = A.row_w[(size_t)t * A.rmax + i];
        }
    }
    for (int t = threadIdx.x; t < kNV * (kNV + 1); t += blockDim.x) (&sH[0][0])[t] = 0.0;

    // b = A_n omega + g  (L holds R(omega), ghosts included)
#pragma unroll
    for (int t = 0; t <= kNV; ++t) acc[t] = 0.0;
    for (int a = a0; a < n; a += stride) {
        T v = apply_point<T, false, P>(Lb, A.meta[a], Ua[a], Va[a], nu, r, A.g, c1J, c2J);
        if (ga) v += ga[a];
        w[a] = v;
        acc[kNV] += dbl(v) * dbl(v);
    }
    block_partials<PT, true>(acc, 0, P0 + (size_t)bid * kOutP, s_red);
    if (!grid_sync(A.bar, A.err, A.limit_ns, bid, nb, A.trace, ph++)) return calls;
    reduce_all<PT>(P0, 1, s_h, s_red, nb);
    // scalars of the step, once per block (FP64 division and square root
    // are long instruction sequences on this part)
    if (threadIdx.x == 0) {
        double bt, ib;
        sqrt_and_rsqrt(s_h[0], bt, ib);
        s_sc[0] = bt;
        s_sc[1] = ib;
    }
    __syncthreads();
    const double beta = s_sc[0];
    int k = m;
    if (!(beta > 0.0) || !isfinite(beta)) {
        k = 0;
        if (lead && !isfinite(beta)) atomicOr(A.flags, 1);
    }
    if (lead) *A.beta = beta;

    if (k > 0) {
        // v_0 = b / beta at the active points and, through the interpolation
        // rows, at the ghosts
        const double inv = s_sc[1];
        for (int a = a0; a < n; a += stride) {
            const T v = (T)(dbl(w[a]) * inv);
            basis[a] = v;
            Lq[meta_pos(A.meta[a])] = v;
        }
        ghost_values<T, PT>(A, w, Gb, ldg, s_c, 0, bid, nb, s_ws[threadIdx.x >> 5], [&](int t, double gv) {
            const T g = (T)(gv * inv);
            Gb[t] = g;
            Lq[A.glist[t]] = g;
        });
        if (!grid_sync(A.bar, A.err, A.limit_ns, bid, nb, A.trace, ph++)) return calls;

        // Arnoldi with CGS2 whose second pass is delayed by one step: step j
        // applies A to u, the vector of step j-1 after its first projection,
        // and one reduction gives s = Q^T u, |u|^2, t = Q^T z and u.z
        // (z = A u).  Then q_j = (u - Q s) / h with h^2 = |u|^2 - |s|^2 (the
        // second pass; column j-1 of H gets + s, H[j][j-1] = h), and, by the
        // Arnoldi relation A Q_{j-1} = Q_j H, A q_j = (z - Q_j g) / h with
        // g = H s: its first projection is h1 = ([t; qz] - g) / h, where
        // qz = q_j.z = (u.z - s.t) / h, and the next u = A q_j - Q_j h1
        // = (z - Q_j [t; qz]) / h (g cancels), without a second operator
        // application.  One reduction and one barrier per step; g only
        // enters column j of H, off the path to the next vectors.
        T* __restrict__ zb = basis + (size_t)m * ld;   // z, in the spare basis row
        T* __restrict__ Gu = Gb + (size_t)m * ldg;     // ghost values of u
        // step 0: z = A q_0 and its first projection
#pragma unroll
        for (int t = 0; t <= kNV; ++t) acc[t] = 0.0;
        for (int a = a0; a < n; a += stride) {
            const T z = apply_point<T, false, P>(Lq, A.meta[a], Ua[a], Va[a], nu, r, A.g, c1J, c2J);
            zb[a] = z;
            acc[0] += dbl(basis[a]) * dbl(z);
        }
        block_partials<PT, false>(acc, 1, P0 + (size_t)bid * kOutP, s_red);
        if (!grid_sync(A.bar, A.err, A.limit_ns, bid, nb, A.trace, ph++)) return calls;
        reduce_all<PT>(P0, 1, s_h, s_red, nb);
        if (threadIdx.x == 0) {
            sH[0][0] = s_h[0];
            s_c[0] = s_h[0];
        }
        __syncthreads();
        for (int a = a0; a < n; a += stride) {
            const T u = project_out<T>(zb[a], basis + a, ld, s_c, 1);
            w[a] = u;
            Lq[meta_pos(A.meta[a])] = u;
        }
        ghost_values<T, PT>(A, zb, Gb, ldg, s_c, 1, bid, nb, s_ws[threadIdx.x >> 5], [&](int t, double gv) {
            const T g = (T)gv;
            Gu[t] = g;
            Lq[A.glist[t]] = g;
        });
        if (!grid_sync(A.bar, A.err, A.limit_ns, bid, nb, A.trace, ph++)) return calls;

        for (int j = 1; j <= m; ++j) {
            const bool last = j == m;   // only the second pass of u is left
            // z = A u and the dots of u and z with q_0 .. q_{j-1}: the values
            // [s, |u|^2, t, u.z] (the last step: [s, |u|^2])
            step_dots<T, PT, CL, P>(A, j, !last, bid, nb, P0 + (size_t)(bid / pgroups) * kOutP, s_dot, s_uz, s_bp,
                                    formed);
            calls = j;
            if (!grid_sync(A.bar, A.err, A.limit_ns, bid, nb, A.trace, ph++)) return calls;
            reduce_all<PT>(P0, last ? j + 1 : 2 * j + 2, s_h, s_red, nb / pgroups);
            // scalars (every block the same; s_h holds s at 0..j-1, |u|^2 at j,
            // t at j+1..2j and u.z at 2j+1).  One warp's FP64 instruction
            // occupies its SM sub-partition for about 64 cycles on this part,
            // so only |s|^2 -> h^2 -> 1/h runs on the path to the next vectors
            // (warp 0); warp 1 forms s.t, warp g0 the first-pass norm
            // |H[:, j-1]|^2 (the breakdown threshold), and warps g0.. the
            // partial sums of g = H s, which only enter column j of H, written
            // after the new vectors.
            constexpr int kW = PT / 32;
            static_assert(kW >= 2, "the scalar phase splits the work over at least two warps");
            constexpr int g0 = kW == 2 ? 1 : 2;          // first warp of the g partial sums
            const int li = threadIdx.x & 31, wid = threadIdx.x >> 5;
            const double si = li < j ? s_h[li] : 0.0;
            double hp = 0.0;
            // s and t in the bulk type for the new vectors (one conversion per
            // value, not per product)
            for (int t = threadIdx.x; t < 2 * j + 2; t += PT) s_hT[t] = (T)s_h[t];
            if (wid == 0) {
                const double v = warp_sum(si * si, s_ws[wid]);
                // h_{j,j-1}^2, clamped at +0 by its sign bit (an FP64 max or
                // compare takes two to three FP64 issue slots); a NaN here
                // comes from |u|^2 or s, which the flags below catch
                double q2 = s_h[j] - v;
                if (__double_as_longlong(q2) < 0) q2 = 0.0;
                double h, hinv;
                sqrt_and_rsqrt(q2, h, hinv);
                if (li == 0) {
                    s_sc[2] = h;
                    s_sc[3] = hinv;
                    s_tmp[0] = q2;
                }
            } else {
                hp = li < j ? sH[li][j - 1] : 0.0;   // first pass of column j-1
                if (wid == 1) {
                    const double ti = (!last && li < j) ? s_h[j + 1 + li] : 0.0;
                    const double st = warp_sum(si * ti, s_ws[wid]);
                    if (li == 0) {
                        const double uu = s_h[j], uz = last ? 0.0 : s_h[2 * j + 1];
                        s_tmp[2] = uz - st;   // h qz, qz = q_j.z
                        // a non-finite s or t shows in s.t
                        s_int[0] = finite_bits(st) && finite_bits(uu) && finite_bits(uz);
                    }
                }
                if (wid == g0) {
                    const double hh = warp_sum(hp * hp, s_ws[wid]);
                    if (li == 0) {
                        // breakdown: h <= tol |A q_{j-1}|, |A q_{j-1}|^2 = |H[:, j-1]|^2 + |u|^2
                        s_tmp[1] = A.tol * A.tol * (hh + s_h[j]);
                        s_int[1] = finite_bits(hh);
                    }
                }
                if (!last && wid >= g0) {
                    // rows i < j of g: columns c < j-1 of H, and column j-1
                    // with its second pass (hp + s), dealt over warps g0..kW-1
                    constexpr int ng = kW - g0;
                    const int c0 = wid - g0;
                    const double hs = hp + si;
                    double gp[2] = {0.0, 0.0};
                    if (li < j)
                        down_from<(kNV + ng - 1) / ng>((j - c0 + ng - 1) / ng, [&](auto cc) {
                            constexpr int q = decltype(cc)::value;
                            const int c = q * ng + c0;
                            gp[q & 1] += (c == j - 1 ? hs : sH[li][c]) * s_h[c];
                        });
                    s_red[wid][li] = gp[0] + gp[1];
                }
            }
            __syncthreads();
            const double q2 = s_tmp[0];
            // q2 and the threshold are non-negative: compared as integers
            const int stop = !(s_int[0] && s_int[1] && finite_bits(q2))
                                 ? 2
                                 : (__double_as_longlong(q2) <= __double_as_longlong(s_tmp[1]) ? 1 : 0);
            if (wid == 1) {   // column j-1 of H after its second pass; h_{j,j-1}
                if (li < j) sH[li][j - 1] = hp + si;
                if (li == 0) sH[j][j - 1] = s_sc[2];
            }
            if (stop == 2) {
                if (lead) atomicOr(A.flags, 1);
                k = j;
                break;
            }
            if (stop == 1 || last) {
                k = j;
                break;
            }
            // q_j = (u - Q s) / h and the next u = (z - Q t - q_j qz) / h at
            // the own points; at the ghosts by linearity
            const double hinv = s_sc[3];
            const double qz = s_tmp[2] * hinv;
            for (int a = a0; a < n; a += stride) {
                const T wa = w[a], za = zb[a];
                T ps[4] = {T(0), T(0), T(0), T(0)}, pc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    T qv[kNV / 2];
#pragma unroll
                    for (int t = 0; t < kNV / 2; ++t)
                        if (hh * (kNV / 2) + t < j) qv[t] = basis[(size_t)(hh * (kNV / 2) + t) * ld + a];
                    down_from<kNV / 2>(min(j - hh * (kNV / 2), kNV / 2), [&](auto tc) {
                        constexpr int t = decltype(tc)::value;
                        ps[t & 3] += qv[t] * s_hT[hh * (kNV / 2) + t];
                        pc[t & 3] += qv[t] * s_hT[j + 1 + hh * (kNV / 2) + t];
                    });
                }
                const T qj = (T)(dbl(wa - ((ps[0] + ps[1]) + (ps[2] + ps[3]))) * hinv);
                basis[(size_t)j * ld + a] = qj;
                const T un = (T)((dbl(za) - dbl((pc[0] + pc[1]) + (pc[2] + pc[3])) - dbl(qj) * qz) * hinv);
                w[a] = un;
                Lq[meta_pos(A.meta[a])] = un;
            }
            if (wid == 0) {
                // column j of H: h1 = ([t; qz] - g) / h, g from the warps' partial
                // sums (g_j = h s_{j-1})
                if (li < j) {
                    double gi = 0.0;
                    for (int q = g0; q < kW; ++q) gi += s_red[q][li];
                    sH[li][j] = (s_h[j + 1 + li] - gi) * hinv;
                } else if (li == j) {
                    sH[j][j] = (qz - s_sc[2] * s_h[j - 1]) * hinv;
                }
            }
            ghost_step<T, PT, P == 2>(A, zb, Gb, ldg, Gu, s_h, s_h + j + 1, qz, j, hinv, Lq, bid, nb, s_ws[wid], rc);
            if (!grid_sync(A.bar, A.err, A.limit_ns, bid, nb, A.trace, ph++)) return calls;
        }
        // H (every block holds it) to global memory, by block 0
        __syncthreads();
        if (bid == 0) {
            for (int e = threadIdx.x; e < (k + 1) * k; e += PT) {
                const int i = e / k, c = e - i * k;
                if (i <= c + 1) A.H[(size_t)i * m + c] = sH[i][c];
            }
            __syncthreads();
        }
    }
    // y = phi_1(dt H_k) e_1 by block 0 (which wrote H), then every block:
    // omega <- omega + dt beta V_k y at its points (accumulated in FP64), also
    // written into the lattice array L
    if (k == 0) {
        if (bid == 0)
            for (int t = threadIdx.x; t < m; t += PT) A.y[t] = 0.0;
        if (lead) *A.kstop = 0;
        return calls;
    }
    if (bid == 0) phi1_block<PT>(A.H, k, m, A.dt, A.y, A.flags, s_red, s_h, s_int);
    if (!grid_sync(A.bar, A.err, A.limit_ns, bid, nb, A.trace, ph++)) return calls;
    for (int t = threadIdx.x; t < k; t += PT) s_c[t] = A.dt * beta * A.y[t];
    __syncthreads();
    T* __restrict__ om = (T*)A.omega;
    T* __restrict__ Lo = (T*)A.L;
    for (int a = a0; a < n; a += stride) {
        double inc = 0.0;
        for (int t = 0; t < k; ++t) inc += s_c[t] * dbl(basis[(size_t)t * ld + a]);
        const T x = (T)(dbl(om[a]) + inc);
        om[a] = x;
        Lo[meta_pos(A.meta[a])] = x;
    }
    if (lead) *A.kstop = k;
    return calls;
}

template <typename T, int PT, int CL, int P>
__global__ void __launch_bounds__(PT, 1) k_krylov_step(KrylovStepArgs A) {
    bool formed = false;
    if constexpr (CL > 1) {
        // the cluster pre-sums read peers' shared memory: a launch that did
        // not form the clusters (some profilers replay cooperative launches
        // without them; the test switch A.refuse acts as one) runs as the
        // unclustered kernel -- no peer access, no cluster barrier, one
        // partial-sum row per block -- and says so in bit 4 (16) of *err
        formed = cooperative_groups::this_cluster().num_blocks() == (unsigned)CL && !A.refuse;
        if (!formed && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(A.err, 16);
    }
    const int calls = krylov_body<T, PT, CL, P>(A, blockIdx.x, gridDim.x, formed);
    if constexpr (CL > 1) {
        if (formed) cluster_finish(calls, A.m);
    }
    (void)calls;
}

// Batched form: several problems in one cooperative launch; block b works on
// problem blk2mem[b], whose blocks are mem_b0[q] .. mem_b0[q + 1] - 1.  The
// ensemble's members have few blocks each, which walk many points, so that
// form is bound by the latency of those walks and is compiled for MB =
// batch_min_blocks(PT) resident blocks per SM at the price of register
// spills (measured faster than one or two spill-free blocks per SM); the two
// problems of one run (omega and the passive scalar) spread over all SMs
// and use the spill-free form (MB = 1).
__host__ __device__ constexpr int batch_min_blocks(int pt) { return pt == 64 ? 8 : (pt == 128 ? 4 : 4); }
template <typename T, int PT, int P, int MB>
__global__ void __launch_bounds__(PT, MB) k_krylov_batch(const KrylovStepArgs* __restrict__ args,
                                                        const int* __restrict__ blk2mem,
                                                        const int* __restrict__ mem_b0) {
    const int q = blk2mem[blockIdx.x];
    const int b0 = mem_b0[q];
    (void)krylov_body<T, PT, 1, P>(args[q], blockIdx.x - b0, mem_b0[q + 1] - b0);
}

}  // namespace

// ---- host side of one (bulk type, DD order): occupancy and launches --------

template <typename T, int P>
cudaError_t KrylovKernels<T, P>::occupancy(int* per) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per, k_krylov_step<T, kPT, 1, P>, kPT, 0);
}

template <typename T, int P>
int KrylovKernels<T, P>::cluster_capacity(int CL) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeCooperative;
    at[1].val.cooperative = 1;
    cfg.gridDim = dim3(CL);
    cfg.blockDim = dim3(kPT);
    cfg.attrs = at;
    cfg.numAttrs = 2;
    int nc = 0;
    const cudaError_t e = CL == 4 ? cudaOccupancyMaxActiveClusters(&nc, k_krylov_step<T, kPT, 4, P>, &cfg)
                                  : cudaOccupancyMaxActiveClusters(&nc, k_krylov_step<T, kPT, 2, P>, &cfg);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nc * CL;
}

template <typename T, int P>
cudaError_t KrylovKernels<T, P>::launch(const KrylovStepArgs& args, int blocks, int cl, cudaStream_t s) {
    if (cl == 1) {
        KrylovStepArgs a = args;
        void* params[] = {&a};
        return cudaLaunchCooperativeKernel((const void*)k_krylov_step<T, kPT, 1, P>, dim3(blocks), dim3(kPT), params,
                                           0, s);
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    at[1].id = cudaLaunchAttributeClusterDimension;
    at[1].val.clusterDim.x = cl;
    at[1].val.clusterDim.y = 1;
    at[1].val.clusterDim.z = 1;
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(kPT);
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    return cl == 4 ? cudaLaunchKernelEx(&cfg, k_krylov_step<T, kPT, 4, P>, args)
                   : cudaLaunchKernelEx(&cfg, k_krylov_step<T, kPT, 2, P>, args);
}

template <typename T, int P>
const void* KrylovKernels<T, P>::batch_kernel(int pt, bool pair) {
    if (pair) return pt == 128 ? (const void*)k_krylov_batch<T, 128, P, 1> : nullptr;
    switch (pt) {
        case 64: return (const void*)k_krylov_batch<T, 64, P, batch_min_blocks(64)>;
        case 128: return (const void*)k_krylov_batch<T, 128, P, batch_min_blocks(128)>;
        case 256: return (const void*)k_krylov_batch<T, 256, P, batch_min_blocks(256)>;
        default: return nullptr;
    }
}


}  // namespace wrc
