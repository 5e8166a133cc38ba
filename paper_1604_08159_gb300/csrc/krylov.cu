// Krylov projection of the time step (Sec. 2.1: the discrete system projected
// onto a Krylov subspace): one persistent cooperative kernel per step,
//   b = A_n omega + g,  beta = |b|,  v_0 = b / beta,
//   Arnoldi with classical Gram-Schmidt applied twice (FP64 inner products,
//   deterministic reductions; the norm after the second pass from
//   |w''|^2 = |w'|^2 - |h2|^2), happy breakdown when h_{j+1,j} <= tol |A v_j|,
//   then (two small kernels) y = phi_1(dt H_k) e_1 from the exponential of the
//   augmented Hessenberg matrix and omega <- omega + dt beta V_k y.
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
constexpr int kTaylor = 20;   // Taylor terms per scaling sub-step of exp(M) e_k

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

// Sum over all blocks of part[b * kOutP + t], t < nout, into s_out: lane t
// of warp w adds blocks w, w + nwarps, ... in order (one output per lane), the
// warps' sums are then added in warp order.  Same order in every block.  The
// loads go out kReduceBatch at a time ahead of their (ordered) additions, so
// a block pays one L2 round trip per batch rather than one per partial.
constexpr int kReduceBatch = 16;

template <int PT>
__device__ __forceinline__ void reduce_all(const double* part, int nout, double* s_out,
                                           double (*s_red)[kNV + 1], int nb) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    constexpr int kW = PT / 32;
    for (int t0 = 0; t0 < nout; t0 += 32) {
        const int t = t0 + lane;
        double v = 0.0;
        if (t < nout) {
            const double* p = part + t;
            int b = wid;
            for (; b + (kReduceBatch - 1) * kW < nb; b += kReduceBatch * kW) {
                double x[kReduceBatch];
#pragma unroll
                for (int u = 0; u < kReduceBatch; ++u) x[u] = __ldcg(p + (size_t)(b + u * kW) * kOutP);
#pragma unroll
                for (int u = 0; u < kReduceBatch; ++u) v += x[u];
            }
            const int rest = b < nb ? (nb - 1 - b) / kW + 1 : 0;   // < kReduceBatch
            double x[kReduceBatch];
#pragma unroll
            for (int u = 0; u < kReduceBatch; ++u)
                if (u < rest) x[u] = __ldcg(p + (size_t)(b + u * kW) * kOutP);
#pragma unroll
            for (int u = 0; u < kReduceBatch; ++u)
                if (u < rest) v += x[u];
        }
        if (t < nout) s_red[wid][t] = v;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nout; t += blockDim.x) {
        double v = 0.0;
        for (int q = 0; q < kW; ++q) v += s_red[q][t];
        s_out[t] = v;
    }
    __syncthreads();
}

// ---- phi_1 from the exponential of the augmented matrix ------------------
// y = phi_1(dt H_k) e_1 is the upper part of the last column of exp(M),
// M = [[dt H_k, e_1], [0, 0]] ((k+1) x (k+1)).  That column, exp(M) e_k, is
// computed as the action of the exponential by scaling and the truncated
// Taylor series: with s = max(1, ceil(|M|_1)), B = M / s has |B|_1 <= 1,
// x <- sum_{i<=20} B^i x / i!  applied s times; the dropped tail is at most
// sum_{i>20} 1/i! < 2e-20 of |x| per sub-step.  One warp, lane r holds row r.
// Largest scaling count of the Taylor evaluation: a step with |dt H|_1 above
// it (or not finite) has blown up; phi_1 is then not evaluated, y is set to
// NaN and the non-finite flag is raised, so that the step fails cleanly
// instead of looping ceil(|dt H|_1) times.
constexpr double kMaxPhiScale = 4096.0;

__device__ __forceinline__ void phi1_warp(const double* __restrict__ H, const int* __restrict__ kstop, int m,
                                          double dt, double* __restrict__ y, int* __restrict__ flags) {
    const int lane = threadIdx.x;
    const int k = *kstop;
    if (k <= 0) {
        for (int t = lane; t < m; t += 32) y[t] = 0.0;
        return;
    }
    double row[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) {
        double v = 0.0;
        if (lane < k && c < k) v = dt * H[(size_t)lane * m + c];
        if (lane == 0 && c == k) v = 1.0;
        row[c] = v;
    }
    double nrm = 0.0;   // |M|_1 = max column sum
#pragma unroll
    for (int c = 0; c < 32; ++c) {
        double cs = fabs(row[c]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cs += __shfl_xor_sync(0xffffffffu, cs, o);
        nrm = fmax(nrm, cs);
    }
    if (!(nrm <= kMaxPhiScale)) {
        if (lane == 0) atomicOr(flags, 1);
        if (lane < m) y[lane] = lane < k ? __longlong_as_double(0x7ff8000000000000ll) : 0.0;
        return;
    }
    const int s = nrm > 1.0 ? (int)ceil(nrm) : 1;
    const double inv_s = 1.0 / s;
    double x = lane == k ? 1.0 : 0.0;
    for (int q = 0; q < s; ++q) {
        double acc = x, term = x;
        for (int i = 1; i <= kTaylor; ++i) {
            double nt[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
            for (int c = 0; c < 32; ++c) nt[c & 3] += row[c] * __shfl_sync(0xffffffffu, term, c);
            term = ((nt[0] + nt[1]) + (nt[2] + nt[3])) * (inv_s / i);
            acc += term;
        }
        x = acc;
    }
    if (lane < m) y[lane] = lane < k ? x : 0.0;
}

__global__ void __launch_bounds__(32) k_phi1(const double* __restrict__ H, const int* __restrict__ kstop, int m,
                                             double dt, double* __restrict__ y, int* __restrict__ flags) {
    phi1_warp(H, kstop, m, dt, y, flags);
}

// omega <- omega + dt beta V_k y (accumulated in FP64), also written into the
// lattice array L.
template <typename T>
__device__ __forceinline__ void update_body(const T* __restrict__ basis, long long ld, const double* __restrict__ y,
                                            const double* __restrict__ beta, const int* __restrict__ kstop,
                                            double dt, const uint32_t* __restrict__ meta, int n,
                                            T* __restrict__ omega, T* __restrict__ L, int bx, int gx) {
    __shared__ double s_c[kNV];
    const int k = *kstop;
    for (int t = threadIdx.x; t < k; t += blockDim.x) s_c[t] = dt * beta[0] * y[t];
    __syncthreads();
    for (int a = bx * blockDim.x + threadIdx.x; a < n; a += gx * blockDim.x) {
        double inc = 0.0;
        for (int t = 0; t < k; ++t) inc += s_c[t] * (double)basis[(size_t)t * ld + a];
        const T x = (T)((double)omega[a] + inc);
        omega[a] = x;
        L[meta_pos(meta[a])] = x;
    }
}

template <typename T>
__global__ void k_update(const T* __restrict__ basis, long long ld, const double* __restrict__ y,
                         const double* __restrict__ beta, const int* __restrict__ kstop, double dt,
                         const uint32_t* __restrict__ meta, int n, T* __restrict__ omega, T* __restrict__ L) {
    update_body<T>(basis, ld, y, beta, kstop, dt, meta, n, omega, L, blockIdx.x, gridDim.x);
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
        const double bt = sqrt(s_h[0]);
        s_sc[0] = bt;
        s_sc[1] = 1.0 / bt;
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
                    const double hn = sqrt(fmax(s_h[nv] - h2, 0.0));
                    s_sc[2] = hn;
                    s_sc[3] = 1.0 / hn;
                    s_stop = (bad || !isfinite(hn)) ? 2 : (hn <= A.tol * sqrt(wn2) ? 1 : 0);
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

// phi_1 for problem blockIdx.x of a batch (one warp each).
__global__ void __launch_bounds__(32) k_phi1_batch(const KrylovStepArgs* __restrict__ args) {
    const KrylovStepArgs& A = args[blockIdx.x];
    phi1_warp(A.H, A.kstop, A.m, A.dt, A.y, A.flags);
}

// Update of problem blockIdx.y of a batch.
template <typename T>
__global__ void k_update_batch(const KrylovStepArgs* __restrict__ args) {
    const KrylovStepArgs& A = args[blockIdx.y];
    update_body<T>((const T*)A.basis, A.ld, A.y, A.beta, A.kstop, A.dt, A.meta, A.n, (T*)A.omega, (T*)A.L,
                   blockIdx.x, gridDim.x);
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
    k_phi1<<<1, 32, 0, s>>>(args.H, args.kstop, args.m, args.dt, args.y, args.flags);
    note_launch();
    k_update<T><<<blocks_for(args.n), kThreads, 0, s>>>((const T*)args.basis, args.ld, args.y, args.beta, args.kstop,
                                                        args.dt, args.meta, args.n, (T*)args.omega, (T*)args.L);
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
    k_phi1_batch<<<members, 32, 0, s>>>(d_args);
    note_launch();
    k_update_batch<T><<<dim3(blocks_for(max_n) < 64 ? blocks_for(max_n) : 64, members), kThreads, 0, s>>>(d_args);
    note_launch();
    return cudaGetLastError();
}

template cudaError_t launch_krylov_batch<double>(const KrylovStepArgs*, const int*, const int*, int, int, int, int,
                                                 cudaStream_t);
template cudaError_t launch_krylov_batch<float>(const KrylovStepArgs*, const int*, const int*, int, int, int, int,
                                                cudaStream_t);

}  // namespace wrc
