// Krylov projection of the time step (Sec. 2.1: the discrete system projected
// onto a Krylov subspace): one persistent cooperative kernel per step,
//   b = A_n omega + g,  beta = |b|,  v_0 = b / beta,
//   Arnoldi with classical Gram-Schmidt applied twice (FP64 inner products,
//   deterministic reductions; the norm after the second pass from
//   |w''|^2 = |w'|^2 - |h2|^2), happy breakdown when h_{j+1,j} <= tol |A v_j|,
//   then, in the same launch, y = phi_1(dt H_k) e_1 from the exponential of
//   the augmented Hessenberg matrix (block 0), one more grid barrier, and
//   omega <- omega + dt beta V_k y (every block, its own points).
// Ghost values of each new basis vector come from exact interpolation rows
// over the active points, so one Arnoldi step takes three phases: operator and
// first dots | first update and second dots | second update, normalisation
// and ghosts.  Phases are separated by a grid barrier with a bounded wait; every block
// reduces the per-block partial sums itself, in the same order, so all blocks
// hold identical coefficients and take identical breakdown decisions.
#include "kernels.h"
#include "operator.cuh"

namespace wrc {

namespace {

constexpr int kPT = 128;      // threads per block of the single-run kernel
constexpr int kNV = 32;       // accumulator slots: basis vectors per pass (<= m + 1 <= 32)
constexpr int kOutP = 66;     // partial sums per block: two sets of (kNV dots + one product)

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier for a cooperative launch: one atomic per block on a
// counter whose top bit flips when the last block arrives (block 0 adds
// 2^31 - (G - 1), the others 1, so each barrier adds exactly 2^31).  The wait
// of each block is bounded by limit_ns; a block that runs out sets bit 1 of
// *err, and every waiter leaves as soon as *err is non-zero, so the kernel
// always returns.
// The barrier spans the nb blocks of one problem (bid = block index within it).
// With a trace buffer, the arrival of each block and the release of block 0
// are stamped (phase index `ph`, counted by the caller).
__device__ bool grid_sync(unsigned* bar, int* err, unsigned long long limit_ns, int bid, int nb,
                          unsigned long long* trace = nullptr, int ph = 0) {
    __syncthreads();
    if (threadIdx.x == 0) {
        if (trace && ph < kTracePhases) trace[1 + (size_t)ph * (nb + 1) + bid] = gtimer();
        const unsigned inc = bid == 0 ? 0x80000000u - (unsigned)(nb - 1) : 1u;
        __threadfence();
        const unsigned old = atomicAdd(bar, inc);
        volatile unsigned* vbar = bar;
        volatile int* verr = err;
        const unsigned long long t0 = gtimer();
        while (((old ^ *vbar) & 0x80000000u) == 0u) {
            if (*verr) break;
            if (gtimer() - t0 > limit_ns) {
                atomicOr(err, 2);
                break;
            }
        }
        __threadfence();
        if (trace && ph < kTracePhases && bid == 0) trace[1 + (size_t)ph * (nb + 1) + nb] = gtimer();
    }
    __syncthreads();
    return *(volatile int*)err == 0;
}

// Per-block sums of acc[0..ndots) and of acc[kNV] (a squared norm) into
// dst[0..ndots] (the norm at index ndots).  The first NS dot accumulators
// (NS = ndots rounded up to a power of two) are reduced across the warp by a
// reduce-scatter (NS - 1 exchanges; afterwards lane l holds the warp sum of
// accumulator l mod NS), the norm by a shuffle tree.
template <int PT>
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
    double v = acc[kNV];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) s_red[wid][kNV] = v;
    __syncthreads();
    for (int t = threadIdx.x; t <= ndots; t += blockDim.x) {
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
// trip covers up to kReduceBatch partials per lane.
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
                x1[u] = __ldcg(p + (size_t)(b + u * kW) * kOutP);
                x2[u] = has2 ? __ldcg(p + 32 + (size_t)(b + u * kW) * kOutP) : 0.0;
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
                x1[u] = __ldcg(p + (size_t)(b + u * kW) * kOutP);
                x2[u] = has2 ? __ldcg(p + 32 + (size_t)(b + u * kW) * kOutP) : 0.0;
            }
#pragma unroll
        for (int u = 0; u < kB; ++u)
            if (u < rest) {
                v1 += x1[u];
                v2 += x2[u];
            }
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
            for (int u = 0; u < kReduceBatch; ++u) x[u] = __ldcg(p + (size_t)(b + u * bstep) * kOutP);
#pragma unroll
            for (int u = 0; u < kReduceBatch; ++u) v += x[u];
        }
        const int rest = b < nb ? (nb - 1 - b) / bstep + 1 : 0;   // < kReduceBatch
        double x[kReduceBatch];
#pragma unroll
        for (int u = 0; u < kReduceBatch; ++u)
            if (u < rest) x[u] = __ldcg(p + (size_t)(b + u * bstep) * kOutP);
#pragma unroll
        for (int u = 0; u < kReduceBatch; ++u)
            if (u < rest) v += x[u];
    }
    for (int o = ns; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);   // the L groups
    if (g == 0 && t < nout) s_red[wid][t] = v;
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

// sqrt(q) and 1/sqrt(q) in FP64 for the normalisation of a new basis vector:
// an FP32 reciprocal square root as the seed, then two Newton-Raphson steps
// y <- y (3 - q y^2) / 2 in FP64 (each doubles the correct bits: ~22 -> ~44
// -> full precision), sqrt(q) = q y.  FP64 division and square root are long
// instruction sequences on this part; this is a handful of FMAs.  Values
// outside the FP32 range take the library's sqrt and division.
__device__ __forceinline__ void sqrt_and_rsqrt(double q, double& s, double& r) {
    if (q > 1e-30 && q < 1e30) {
        double y = (double)rsqrtf((float)q);
        y = y * (1.5 - 0.5 * q * y * y);
        y = y * (1.5 - 0.5 * q * y * y);
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
constexpr int kGhostLanes = 8;
constexpr int kGatherLane = 8;

template <typename T, int PT, typename F>
__device__ __forceinline__ void ghost_values(const KrylovStepArgs& A, const T* __restrict__ x,
                                             const T* __restrict__ Gb, long long ldg, const double* c, int nc,
                                             int bid, int nb, F&& emit) {
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
                if (e0 + gl + kGhostLanes * u < rl) xv[u] = (double)__ldcg(x + id[u]);
#pragma unroll
            for (int u = 0; u < kGatherLane; ++u)
                if (e0 + gl + kGhostLanes * u < rl) part += wt[u] * xv[u];
        }
        if (valid)
            for (int q = gl; q < nc; q += kGhostLanes) part -= c[q] * (double)Gb[(size_t)q * ldg + t];
#pragma unroll
        for (int o = 1; o < kGhostLanes; o <<= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (valid && gl == 0) emit(t, part);
    }
}

// Ghost values of step j of the delayed scheme (groups of kGhostLanes lanes
// per ghost, as ghost_values): q_j at ghost t, Gb_j = (Gu - sum_{q<j} s_q Gb_q) / h,
// then the next u there, Gu <- (rows . z) / h - sum_{q<=j} c_q Gb_q (with the
// new Gb_j), also written into the lattice vector Lq.
template <typename T, int PT>
__device__ __forceinline__ void ghost_step(const KrylovStepArgs& A, const T* __restrict__ z, T* __restrict__ Gb,
                                           long long ldg, T* __restrict__ Gu, const double* s, const double* c,
                                           int j, double hinv, T* __restrict__ Lq, int bid, int nb) {
    constexpr int kGroups = PT / kGhostLanes;
    constexpr int kPerWarp = 32 / kGhostLanes;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int gl = lane % kGhostLanes;
    for (int q0 = wid * kPerWarp; bid + (long long)nb * q0 < A.ng; q0 += kGroups) {
        const long long tl = bid + (long long)nb * (q0 + lane / kGhostLanes);
        const bool valid = tl < A.ng;
        const int t = valid ? (int)tl : 0;
        const int rl = valid ? A.row_len[t] : 0;
        const size_t base = (size_t)t * A.rmax;
        double part = 0.0;   // rows . z, this lane's share
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
                if (e0 + gl + kGhostLanes * u < rl) xv[u] = (double)__ldcg(z + id[u]);
#pragma unroll
            for (int u = 0; u < kGatherLane; ++u)
                if (e0 + gl + kGhostLanes * u < rl) part += wt[u] * xv[u];
        }
        double ss = 0.0, cs = 0.0;
        if (valid)
            for (int q = gl; q < j; q += kGhostLanes) {
                const double gq = (double)Gb[(size_t)q * ldg + t];
                ss += s[q] * gq;
                cs += c[q] * gq;
            }
#pragma unroll
        for (int o = 1; o < kGhostLanes; o <<= 1) {
            part += __shfl_xor_sync(0xffffffffu, part, o);
            ss += __shfl_xor_sync(0xffffffffu, ss, o);
            cs += __shfl_xor_sync(0xffffffffu, cs, o);
        }
        if (valid && gl == 0) {
            const T gbj = (T)(((double)Gu[t] - ss) * hinv);
            const T gu = (T)(part * hinv - (cs + c[j] * (double)gbj));
            Gb[(size_t)j * ldg + t] = gbj;
            Gu[t] = gu;
            Lq[A.glist[t]] = gu;
        }
    }
}

// The Krylov step of one problem, run by its nb blocks (bid = this block's
// index among them).
template <typename T, int PT>
__device__ __forceinline__ void krylov_body(const KrylovStepArgs& A, const int bid, const int nb) {
    const T* __restrict__ Ua = (const T*)A.Ua;
    const T* __restrict__ Va = (const T*)A.Va;
    const T* __restrict__ ga = (const T*)A.ga;
    const T* __restrict__ Lb = (const T*)A.L;
    T* __restrict__ Lq = (T*)A.Lq;
    T* __restrict__ basis = (T*)A.basis;
    T* __restrict__ w = (T*)A.w;
    T* __restrict__ Gb = (T*)A.Gb;
    __shared__ double s_red[PT / 32][kNV + 1];
    __shared__ double s_h[kOutP];
    __shared__ double s_c[kNV];
    __shared__ double s_sc[4];   // beta, 1/beta, h_{j+1,j}, 1/h_{j+1,j}
    __shared__ int s_stop;       // 0 go on, 1 happy breakdown, 2 non-finite
    __shared__ int s_int[3];     // phi_1: blown up, sub-steps, Taylor terms
    __shared__ double sH[kNV][kNV + 1];   // H, held by every block
    __shared__ double s_cc[kNV + 1];      // coefficients of the next u
    __shared__ double s_tmp[4];           // |s|^2, |h1|^2, s.t of a step
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
    if (*(volatile const int*)A.row_overflow) {
        if (lead) atomicOr(A.err, 4);
        return;
    }
    if (bid == 0)   // H is written by this block only
        for (int t = threadIdx.x; t < (m + 1) * m; t += blockDim.x) A.H[t] = 0.0;
    for (int t = threadIdx.x; t < kNV * (kNV + 1); t += blockDim.x) (&sH[0][0])[t] = 0.0;

    // b = A_n omega + g  (L holds R(omega), ghosts included)
#pragma unroll
    for (int t = 0; t <= kNV; ++t) acc[t] = 0.0;
    for (int a = a0; a < n; a += stride) {
        T v = apply_point<T, false>(Lb, A.meta[a], Ua[a], Va[a], nu, r, A.g, c1J, c2J);
        if (ga) v += ga[a];
        w[a] = v;
        acc[kNV] += (double)v * (double)v;
    }
    block_partials<PT>(acc, 0, P0 + (size_t)bid * kOutP, s_red);
    if (!grid_sync(A.bar, A.err, A.limit_ns, bid, nb, A.trace, ph++)) return;
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
            const T v = (T)((double)w[a] * inv);
            basis[a] = v;
            Lq[meta_pos(A.meta[a])] = v;
        }
        ghost_values<T, PT>(A, w, Gb, ldg, s_c, 0, bid, nb, [&](int t, double gv) {
            const T g = (T)(gv * inv);
            Gb[t] = g;
            Lq[A.glist[t]] = g;
        });
        if (!grid_sync(A.bar, A.err, A.limit_ns, bid, nb, A.trace, ph++)) return;

        // Arnoldi with CGS2 whose second pass is delayed by one step: step j
        // applies A to u, the vector of step j-1 after its first projection,
        // and one reduction gives s = Q^T u, |u|^2, t = Q^T z and u.z
        // (z = A u).  Then q_j = (u - Q s) / h with h^2 = |u|^2 - |s|^2 (the
        // second pass; column j-1 of H gets + s, H[j][j-1] = h), and, by the
        // Arnoldi relation A Q_{j-1} = Q_j H, A q_j = (z - Q_j g) / h with
        // g = H s: its first projection h1 = ([t; (u.z - s.t)/h] - g) / h
        // and the next u = z / h - Q_j (g / h + h1), without a second operator
        // application.  One reduction and one barrier per step.
        T* __restrict__ zb = basis + (size_t)m * ld;   // z, in the spare basis row
        T* __restrict__ Gu = Gb + (size_t)m * ldg;     // ghost values of u
        // step 0: z = A q_0 and its first projection
#pragma unroll
        for (int t = 0; t <= kNV; ++t) acc[t] = 0.0;
        for (int a = a0; a < n; a += stride) {
            const T z = apply_point<T, true>(Lq, A.meta[a], Ua[a], Va[a], nu, r, A.g, c1J, c2J);
            zb[a] = z;
            const double zd = (double)z;
            acc[0] += (double)basis[a] * zd;
            acc[kNV] += zd * zd;
        }
        block_partials<PT>(acc, 1, P0 + (size_t)bid * kOutP, s_red);
        if (!grid_sync(A.bar, A.err, A.limit_ns, bid, nb, A.trace, ph++)) return;
        reduce_all<PT>(P0, 2, s_h, s_red, nb);
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
        ghost_values<T, PT>(A, zb, Gb, ldg, s_c, 1, bid, nb, [&](int t, double gv) {
            const T g = (T)gv;
            Gu[t] = g;
            Lq[A.glist[t]] = g;
        });
        if (!grid_sync(A.bar, A.err, A.limit_ns, bid, nb, A.trace, ph++)) return;

        for (int j = 1; j <= m; ++j) {
            const bool last = j == m;   // only the second pass of u is left
            // z = A u; dots of u and of z with q_0 .. q_{j-1}.  While both sets
            // fit the accumulators (j <= 15), one pass and one block reduction,
            // interleaved: acc[2t] = q_t.u, acc[2t+1] = q_t.z, acc[30] = |u|^2,
            // acc[31] = u.z; otherwise two passes, acc[t] = q_t.u then q_t.z
            // (layout in the partials: s, |u|^2, t, u.z)
            const bool inter = !last && 2 * j <= kNV - 2;
            if (inter) {
#pragma unroll
                for (int t = 0; t <= kNV; ++t) acc[t] = 0.0;
                for (int a = a0; a < n; a += stride) {
                    const T z = apply_point<T, true>(Lq, A.meta[a], Ua[a], Va[a], nu, r, A.g, c1J, c2J);
                    zb[a] = z;
                    const double zd = (double)z, ud = (double)w[a];
#pragma unroll
                    for (int t = 0; t < kNV / 2 - 1; ++t)
                        if (t < j) {
                            const double q = (double)basis[(size_t)t * ld + a];
                            acc[2 * t] += q * ud;
                            acc[2 * t + 1] += q * zd;
                        }
                    acc[kNV - 2] += ud * ud;
                    acc[kNV - 1] += ud * zd;
                }
                block_partials<PT>(acc, kNV, P0 + (size_t)bid * kOutP, s_red);
            } else {
#pragma unroll
            for (int t = 0; t <= kNV; ++t) acc[t] = 0.0;
            for (int a = a0; a < n; a += stride) {
                const double ud = (double)w[a];
#pragma unroll
                for (int t = 0; t < kNV; ++t)
                    if (t < j) acc[t] += (double)basis[(size_t)t * ld + a] * ud;
                acc[kNV] += ud * ud;
            }
            block_partials<PT>(acc, j, P0 + (size_t)bid * kOutP, s_red);
            if (!last) {
                __syncthreads();   // s_red is reused
#pragma unroll
                for (int t = 0; t <= kNV; ++t) acc[t] = 0.0;
                for (int a = a0; a < n; a += stride) {
                    const T z = apply_point<T, true>(Lq, A.meta[a], Ua[a], Va[a], nu, r, A.g, c1J, c2J);
                    zb[a] = z;
                    const double zd = (double)z;
#pragma unroll
                    for (int t = 0; t < kNV; ++t)
                        if (t < j) acc[t] += (double)basis[(size_t)t * ld + a] * zd;
                    acc[kNV] += (double)w[a] * zd;
                }
                block_partials<PT>(acc, j, P0 + (size_t)bid * kOutP + (j + 1), s_red);
            }
            }
            if (!grid_sync(A.bar, A.err, A.limit_ns, bid, nb, A.trace, ph++)) return;
            reduce_all<PT>(P0, inter ? kNV : (last ? j + 1 : 2 * j + 2), s_h, s_red, nb);
            // scalars (every block the same): the second pass of u, the
            // breakdown tests, and the coefficients of q_j and the next u.  The
            // FP64 work is spread over the warps: one warp's FP64 instruction
            // occupies its SM sub-partition for about 64 cycles on this part.
            {
                constexpr int kW = PT / 32;
                const int i = threadIdx.x & 31, wid = threadIdx.x >> 5;
                const double si = i < j ? s_h[inter ? 2 * i : i] : 0.0;
                const double hp = i < j ? sH[i][j - 1] : 0.0;   // first pass of column j-1
                const double ti = (!last && i < j) ? s_h[inter ? 2 * i + 1 : j + 1 + i] : 0.0;
                const double uu = s_h[inter ? kNV - 2 : j];
                const double uz = last ? 0.0 : s_h[inter ? kNV - 1 : 2 * j + 1];
                // |s|^2, |h1|^2 and s.t, each summed by one warp
#pragma unroll
                for (int q = 0; q < 3; ++q)
                    if (q % kW == wid) {
                        double v = q == 0 ? si * si : (q == 1 ? hp * hp : si * ti);
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                        if (i == 0) s_tmp[q] = v;
                    }
                __syncthreads();
                if (wid == 0) {
                    const bool bad = __any_sync(0xffffffffu, !isfinite(hp + si) || !isfinite(ti)) || !isfinite(uu) ||
                                     !isfinite(uz);
                    if (i < j) {
                        sH[i][j - 1] = hp + si;
                        s_c[i] = si;
                    }
                    if (i == 0) {
                        const double q2 = fmax(uu - s_tmp[0], 0.0);   // h_{j,j-1}^2
                        double h, hinv;
                        sqrt_and_rsqrt(q2, h, hinv);
                        sH[j][j - 1] = h;
                        s_sc[2] = h;
                        s_sc[3] = hinv;
                        // breakdown: h <= tol |A q_{j-1}|, |A q_{j-1}|^2 = |h1|^2 + |u|^2
                        s_stop = (bad || !isfinite(q2)) ? 2 : (q2 <= A.tol * A.tol * (s_tmp[1] + uu) ? 1 : 0);
                    }
                }
                __syncthreads();
                if (s_stop == 0 && !last) {
                    // g = H s (rows 0 .. j): column groups c = w (mod kW) per warp
                    double gp = 0.0;
                    if (i <= j)
#pragma unroll
                        for (int cc = 0; cc < kNV / kW; ++cc) {
                            const int c = cc * kW + wid;
                            if (c < j) gp += sH[i][c] * s_c[c];
                        }
                    s_red[wid][i] = gp;
                    __syncthreads();
                    if (wid == 0 && i <= j) {
                        double gi = s_red[0][i];
                        for (int w = 1; w < kW; ++w) gi += s_red[w][i];
                        const double hinv = s_sc[3];
                        const double qz = (uz - s_tmp[2]) * hinv;
                        const double h1 = i < j ? (ti - gi) * hinv : (qz - gi) * hinv;
                        s_cc[i] = gi * hinv + h1;
                        sH[i][j] = h1;
                    }
                }
            }
            __syncthreads();
            const int stop = s_stop;
            if (stop == 2) {
                if (lead) atomicOr(A.flags, 1);
                k = j;
                break;
            }
            if (stop == 1 || last) {
                k = j;
                break;
            }
            // q_j = (u - Q s) / h and the next u = z / h - Q_j c at the own
            // points; at the ghosts by linearity
            const double hinv = s_sc[3];
            for (int a = a0; a < n; a += stride) {
                T ps[4] = {T(0), T(0), T(0), T(0)}, pc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
                for (int t = 0; t < kNV; ++t)
                    if (t < j) {
                        const T q = basis[(size_t)t * ld + a];
                        ps[t & 3] += q * (T)s_c[t];
                        pc[t & 3] += q * (T)s_cc[t];
                    }
                const T qj = (T)((double)(w[a] - ((ps[0] + ps[1]) + (ps[2] + ps[3]))) * hinv);
                basis[(size_t)j * ld + a] = qj;
                const T un = (T)((double)zb[a] * hinv) - (((pc[0] + pc[1]) + (pc[2] + pc[3])) + qj * (T)s_cc[j]);
                w[a] = un;
                Lq[meta_pos(A.meta[a])] = un;
            }
            ghost_step<T, PT>(A, zb, Gb, ldg, Gu, s_c, s_cc, j, hinv, Lq, bid, nb);
            if (!grid_sync(A.bar, A.err, A.limit_ns, bid, nb, A.trace, ph++)) return;
        }
        // H (every block holds it) to global memory, by block 0
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
        return;
    }
    if (bid == 0) phi1_block<PT>(A.H, k, m, A.dt, A.y, A.flags, s_red, s_h, s_int);
    if (!grid_sync(A.bar, A.err, A.limit_ns, bid, nb, A.trace, ph++)) return;
    for (int t = threadIdx.x; t < k; t += PT) s_c[t] = A.dt * beta * __ldcg(A.y + t);
    __syncthreads();
    T* __restrict__ om = (T*)A.omega;
    T* __restrict__ Lo = (T*)A.L;
    for (int a = a0; a < n; a += stride) {
        double inc = 0.0;
        for (int t = 0; t < k; ++t) inc += s_c[t] * (double)basis[(size_t)t * ld + a];
        const T x = (T)((double)om[a] + inc);
        om[a] = x;
        Lo[meta_pos(A.meta[a])] = x;
    }
    if (lead) *A.kstop = k;
}

template <typename T, int PT>
__global__ void __launch_bounds__(PT, 1) k_krylov_step(KrylovStepArgs A) {
    krylov_body<T, PT>(A, blockIdx.x, gridDim.x);
}

// Batched form: several problems in one cooperative launch; block b works on
// problem blk2mem[b], whose blocks are mem_b0[q] .. mem_b0[q + 1] - 1.
template <typename T, int PT>
__global__ void __launch_bounds__(PT, 1) k_krylov_batch(const KrylovStepArgs* __restrict__ args,
                                                        const int* __restrict__ blk2mem,
                                                        const int* __restrict__ mem_b0) {
    const int q = blk2mem[blockIdx.x];
    const int b0 = mem_b0[q];
    krylov_body<T, PT>(args[q], blockIdx.x - b0, mem_b0[q + 1] - b0);
}

}  // namespace

int krylov_step_init(bool fp32, int* max_blocks) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const cudaError_t e = fp32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_krylov_step<float, kPT>, kPT, 0)
                               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_krylov_step<double, kPT>, kPT, 0);
    if (e != cudaSuccess || per < 1) return -2;
    *max_blocks = sms * per;
    return 0;
}

int krylov_step_blocks(long long n, int max_blocks) {
    long long b = (n + kPT - 1) / kPT;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (int)b;
}

template <typename T>
cudaError_t launch_krylov_step(const KrylovStepArgs& args, int blocks, cudaStream_t s) {
    KrylovStepArgs a = args;
    void* params[] = {&a};
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_krylov_step<T, kPT>, dim3(blocks), dim3(kPT), params, 0, s);
    if (e != cudaSuccess) return e;
    note_launch();
    return cudaGetLastError();
}

template cudaError_t launch_krylov_step<double>(const KrylovStepArgs&, int, cudaStream_t);
template cudaError_t launch_krylov_step<float>(const KrylovStepArgs&, int, cudaStream_t);

size_t krylov_partials_doubles(int max_blocks) { return (size_t)3 * max_blocks * kOutP; }

namespace {
template <typename T, int PT>
const void* batch_kernel() { return (const void*)k_krylov_batch<T, PT>; }
}  // namespace

int krylov_batch_max_blocks(bool fp32, int pt) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const void* k = nullptr;
    switch (pt) {
        case 64: k = fp32 ? batch_kernel<float, 64>() : batch_kernel<double, 64>(); break;
        case 128: k = fp32 ? batch_kernel<float, 128>() : batch_kernel<double, 128>(); break;
        case 256: k = fp32 ? batch_kernel<float, 256>() : batch_kernel<double, 256>(); break;
        default: return -1;
    }
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, pt, 0) != cudaSuccess || per < 1) return -2;
    return sms * per;
}

template <typename T>
cudaError_t launch_krylov_batch(const KrylovStepArgs* d_args, const int* d_blk2mem, const int* d_mem_b0,
                                int members, int blocks, int pt, int max_n, cudaStream_t s) {
    void* params[] = {(void*)&d_args, (void*)&d_blk2mem, (void*)&d_mem_b0};
    const void* k = pt == 64 ? batch_kernel<T, 64>() : pt == 256 ? batch_kernel<T, 256>() : batch_kernel<T, 128>();
    cudaError_t e = cudaLaunchCooperativeKernel(k, dim3(blocks), dim3(pt), params, 0, s);
    if (e != cudaSuccess) return e;
    note_launch();
    (void)members;
    (void)max_n;
    return cudaGetLastError();
}

template cudaError_t launch_krylov_batch<double>(const KrylovStepArgs*, const int*, const int*, int, int, int, int,
                                                 cudaStream_t);
template cudaError_t launch_krylov_batch<float>(const KrylovStepArgs*, const int*, const int*, int, int, int, int,
                                                cudaStream_t);

}  // namespace wrc
