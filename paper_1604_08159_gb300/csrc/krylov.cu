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
constexpr int kOutP = 33;     // partial sums per block: kNV dots + a squared norm

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

// Sum over all blocks of part[b * kOutP + t], t < nout, into s_out.  The
// lanes of a warp are split into L = 32 / ns groups (ns = nout rounded up to
// a power of two, at most 32, so L > 1 only when nout <= 16): lane g ns + t of
// warp w adds output t of blocks w + 4 (g + L u), u = 0, 1, ... (for 4 warps),
// in order; the groups are then combined by shuffles and the warps' sums
// added in warp order.  Same order in every block.  A lane's loads go out
// kReduceBatch at a time ahead of their ordered additions, so one L2 round
// trip covers up to kReduceBatch partials per lane.
constexpr int kReduceBatch = 16;

template <int PT>
__device__ __forceinline__ void reduce_all(const double* part, int nout, double* s_out,
                                           double (*s_red)[kNV + 1], int nb) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    constexpr int kW = PT / 32;
    if (nout > 32) nout = 32;   // (never: nout <= m + 1 <= 32)
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
        double s = 0.0;
        for (int w = 0; w < kW; ++w) s += s_red[w][q];
        s_out[q] = s;
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
constexpr int kGhostLanes = 4;
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
    const int n = A.n;
    const int stride = nb * PT;
    const int a0 = bid * PT + threadIdx.x;
    const bool lead = bid == 0 && threadIdx.x == 0;
    double* P0 = A.part;
    double* P1 = P0 + (size_t)nb * kOutP;
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
        for (int j = 0; j < m; ++j) {
            const int nv = j + 1;
            // phase 1: w = A v_j and the first Gram-Schmidt dots
#pragma unroll
            for (int t = 0; t <= kNV; ++t) acc[t] = 0.0;
            for (int a = a0; a < n; a += stride) {
                const T v = apply_point<T, true>(Lq, A.meta[a], Ua[a], Va[a], nu, r, A.g, c1J, c2J);
                w[a] = v;
                const double vd = (double)v;
#pragma unroll
                for (int t = 0; t < kNV; ++t)
                    if (t < nv) acc[t] += (double)basis[(size_t)t * ld + a] * vd;
                acc[kNV] += vd * vd;
            }
            block_partials<PT>(acc, nv, P0 + (size_t)bid * kOutP, s_red);
            if (!grid_sync(A.bar, A.err, A.limit_ns, bid, nb, A.trace, ph++)) return;
            reduce_all<PT>(P0, nv + 1, s_h, s_red, nb);
            const double wn2 = s_h[nv];
            for (int t = threadIdx.x; t < nv; t += blockDim.x) s_c[t] = s_h[t];
            __syncthreads();
            // phase 2: w' = w - V h1 (stored), second dots and |w'|^2
#pragma unroll
            for (int t = 0; t <= kNV; ++t) acc[t] = 0.0;
            for (int a = a0; a < n; a += stride) {
                const T x = project_out<T>(w[a], basis + a, ld, s_c, nv);
                w[a] = x;
                const double xd = (double)x;
#pragma unroll
                for (int t = 0; t < kNV; ++t)
                    if (t < nv) acc[t] += (double)basis[(size_t)t * ld + a] * xd;
                acc[kNV] += xd * xd;
            }
            block_partials<PT>(acc, nv, P1 + (size_t)bid * kOutP, s_red);
            if (!grid_sync(A.bar, A.err, A.limit_ns, bid, nb, A.trace, ph++)) return;
            reduce_all<PT>(P1, nv + 1, s_h, s_red, nb);
            // h_{:,j} = h1 + h2; |w''|^2 = |w'|^2 - |h2|^2 (V orthonormal,
            // h2 = V^T w'), the breakdown tests and 1/h_{j+1,j}: warp 0, once
            if (threadIdx.x < 32) {
                const int t = threadIdx.x;
                double h2 = 0.0;
                bool bad = false;
                if (t < nv) {
                    h2 = s_h[t] * s_h[t];
                    bad = !isfinite(s_c[t] + s_h[t]);
                    if (bid == 0) A.H[(size_t)t * m + j] = s_c[t] + s_h[t];
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) h2 += __shfl_xor_sync(0xffffffffu, h2, o);
                bad = __any_sync(0xffffffffu, bad);
                if (t == 0) {
                    const double q = fmax(s_h[nv] - h2, 0.0);   // h_{j+1,j}^2
                    double hn, inv;
                    sqrt_and_rsqrt(q, hn, inv);
                    s_sc[2] = hn;
                    s_sc[3] = inv;
                    // breakdown: h <= tol |A v_j|, compared squared
                    s_stop = (bad || !isfinite(q)) ? 2 : (q <= A.tol * A.tol * wn2 ? 1 : 0);
                    if (bid == 0) A.H[(size_t)(j + 1) * m + j] = hn;
                }
            }
            __syncthreads();
            for (int t = threadIdx.x; t < nv; t += blockDim.x) s_c[t] = s_h[t];
            const int stop = s_stop;
            __syncthreads();
            if (stop == 2) {
                if (lead) atomicOr(A.flags, 1);
                k = j + 1;
                break;
            }
            if (stop == 1) {
                k = j + 1;
                break;
            }
            if (j + 1 == m) break;
            // phase 3: v_{j+1} = (w' - V h2) / hn at the active points; at the
            // ghosts by linearity from w' and the ghost values of v_0..v_j
            const double inv2 = s_sc[3];
            for (int a = a0; a < n; a += stride) {
                const T x = project_out<T>(w[a], basis + a, ld, s_c, nv);
                const T v = (T)((double)x * inv2);
                basis[(size_t)(j + 1) * ld + a] = v;
                Lq[meta_pos(A.meta[a])] = v;
            }
            ghost_values<T, PT>(A, w, Gb, ldg, s_c, nv, bid, nb, [&](int t, double gv) {
                const T g = (T)(gv * inv2);
                Gb[(size_t)(j + 1) * ldg + t] = g;
                Lq[A.glist[t]] = g;
            });
            if (!grid_sync(A.bar, A.err, A.limit_ns, bid, nb, A.trace, ph++)) return;
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
