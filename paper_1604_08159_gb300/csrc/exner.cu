// Kernels of the compressible velocity-Exner form of the model (Eqs. 1-2,
// the f-plane Coriolis term and Rayleigh friction for Eq. 4):
//   pi_t = -(u pi_x + v pi_y) - pi (u_x + v_y)
//   u_t  = -(u u_x + v u_y) - C pi_x + f (v - G_y) - r u + nu lap u
//   v_t  = -(u v_x + v v_y) - C pi_y - f (u - G_x) - r v + nu lap v
// on the adaptive collocation grid, derivatives of Sec. 2.5 at each point's
// stencil levels.  The Krylov projection of the step (Sec. 2.1) runs on the
// stacked vector [u; v; pi] of the active points in one persistent
// cooperative kernel: per Krylov vector its three lattices (values at the
// active points, the ghosts through the interpolation rows), the operator
// and classical Gram-Schmidt twice.  No Poisson solve.
#include "krylov_impl.cuh"
#include "wrc.h"

namespace wrc {

namespace {

constexpr int kExThreads = 256;
static_assert(kOutP == kExPartWidth, "partial-sum rows of the velocity-Exner Krylov kernel");

int ex_blocks(long long n) {
    long long b = (n + kExThreads - 1) / kExThreads;
    if (b < 1) b = 1;
    if (b > 8192) b = 8192;
    return (int)b;
}

template <typename F>
void ex_by_order(int P, F&& f) {
    if (P == 3) f(std::integral_constant<int, 3>{});
    else if (P == 4) f(std::integral_constant<int, 4>{});
    else f(std::integral_constant<int, 2>{});
}

// Items t < n: the active point t of each field into its lattice; items
// n <= t < n + ng: ghost t - n of each field from its interpolation row over
// the active values (Eq. 6 evaluated as a fixed linear combination).
__global__ void k_ex_fields(const uint32_t* __restrict__ meta, int n, const int* __restrict__ glist, int ng,
                            const int* __restrict__ row_len, const int* __restrict__ row_idx,
                            const double* __restrict__ row_w, int rmax, const double* __restrict__ s0,
                            const double* __restrict__ s1, const double* __restrict__ s2, double* __restrict__ d0,
                            double* __restrict__ d1, double* __restrict__ d2, const int* __restrict__ kstop, int j) {
    if (kstop && j >= *kstop) return;
    const long long total = (long long)n + ng;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        if (t < n) {
            const int p = meta_pos(meta[t]);
            d0[p] = s0[t];
            d1[p] = s1[t];
            d2[p] = s2[t];
        } else {
            const long long e = t - n;
            const int rl = row_len[e];
            const int* ri = row_idx + e * rmax;
            const double* rw = row_w + e * rmax;
            double a0 = 0.0, a1 = 0.0, a2 = 0.0;
            for (int r0 = 0; r0 < rl; r0 += kGatherLane) {
                int id[kGatherLane];
                double wt[kGatherLane];
#pragma unroll
                for (int u = 0; u < kGatherLane; ++u) {
                    id[u] = r0 + u < rl ? ri[r0 + u] : -1;
                    wt[u] = r0 + u < rl ? rw[r0 + u] : 0.0;
                }
#pragma unroll
                for (int u = 0; u < kGatherLane; ++u)
                    if (id[u] >= 0) {
                        a0 += wt[u] * s0[id[u]];
                        a1 += wt[u] * s1[id[u]];
                        a2 += wt[u] * s2[id[u]];
                    }
            }
            const int p = glist[e];
            d0[p] = a0;
            d1[p] = a1;
            d2[p] = a2;
        }
    }
}

template <int P>
__global__ void k_ex_base(ExArgs a, double* __restrict__ w) {
    const int n = a.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t mw = a.meta[i];
        double ux, uy, lu, vx, vy, lv, px, py, lp;
        point_derivs<double, P>(a.Lb[0], mw, a.g, a.c1J, a.c2J, ux, uy, lu);
        point_derivs<double, P>(a.Lb[1], mw, a.g, a.c1J, a.c2J, vx, vy, lv);
        point_derivs<double, P>(a.Lb[2], mw, a.g, a.c1J, a.c2J, px, py, lp);
        const double u = a.f[0][i], v = a.f[1][i], p = a.f[2][i];
        double* d = a.d;
        const long long ld = a.ld;
        d[i] = ux;
        d[ld + i] = uy;
        d[2 * ld + i] = vx;
        d[3 * ld + i] = vy;
        d[4 * ld + i] = px;
        d[5 * ld + i] = py;
        d[6 * ld + i] = lu;
        d[7 * ld + i] = lv;
        w[i] = -(u * ux + v * uy) - a.C * px + a.fc * (v - a.gy) - a.r * u + a.nu * lu;
        w[n + i] = -(u * vx + v * vy) - a.C * py - a.fc * (u - a.gx) - a.r * v + a.nu * lv;
        w[2 * n + i] = -(u * px + v * py) - p * (ux + vy);
    }
}

// M q at the active points: the frozen-coefficient operator (advection by
// the state's velocity, pressure gradient, pi times the divergence,
// Coriolis, friction, viscosity) plus, for the exact Jacobian, the terms of
// the state's gradients.
// Entry e of M q (e = f n + i: field f at active point i; M the exact
// Jacobian with full, else the frozen-coefficient operator): the own field's
// collocation derivatives at the point's stencil levels and the cross terms
// of the other fields (the lattices a.Lq hold q with its ghost values).
template <int P>
__device__ __forceinline__ double ex_entry(const ExArgs& a, const double* __restrict__ q, int f, int i) {
    const int n = a.n;
    const long long ld = a.ld;
    const uint32_t mw = a.meta[i];
    const double* d = a.d;
    const double u = a.f[0][i], v = a.f[1][i];
    const double du = q[i], dv = q[n + i];
    if (f == 0) {
        double dx, dy, lap;
        point_derivs<double, P>(a.Lq[0], mw, a.g, a.c1J, a.c2J, dx, dy, lap);
        const double dpx = point_d1<double, P>(a.Lq[2], mw, a.g, a.c1J, 0);
        double J = -(u * dx + v * dy) - a.C * dpx + a.fc * dv - a.r * du + a.nu * lap;
        if (a.full) J -= du * d[i] + dv * d[ld + i];
        return J;
    }
    if (f == 1) {
        double dx, dy, lap;
        point_derivs<double, P>(a.Lq[1], mw, a.g, a.c1J, a.c2J, dx, dy, lap);
        const double dpy = point_d1<double, P>(a.Lq[2], mw, a.g, a.c1J, 1);
        double J = -(u * dx + v * dy) - a.C * dpy - a.fc * du - a.r * dv + a.nu * lap;
        if (a.full) J -= du * d[2 * ld + i] + dv * d[3 * ld + i];
        return J;
    }
    const double dpx = point_d1<double, P>(a.Lq[2], mw, a.g, a.c1J, 0);
    const double dpy = point_d1<double, P>(a.Lq[2], mw, a.g, a.c1J, 1);
    const double dux = point_d1<double, P>(a.Lq[0], mw, a.g, a.c1J, 0);
    const double dvy = point_d1<double, P>(a.Lq[1], mw, a.g, a.c1J, 1);
    double J = -(u * dpx + v * dpy) - a.f[2][i] * (dux + dvy);
    if (a.full) J -= (du * d[4 * ld + i] + dv * d[5 * ld + i]) + q[2 * n + i] * (d[i] + d[3 * ld + i]);
    return J;
}

// Field and point of a stacked entry.
__device__ __forceinline__ void ex_split(long long e, int n, int& f, int& i) {
    f = e >= 2LL * n ? 2 : (e >= n ? 1 : 0);
    i = (int)(e - (long long)f * n);
}

// Basis vector q_c = w * scale at the block's own stacked entries, their
// lattices at the active points, and the block's share of the ghost values
// (items f ng + g: field f at ghost g) from the interpolation rows over w
// (whose entries are final for every point when this runs).
__device__ __forceinline__ void ex_new_vector(const ExArgs& a, const ExKrylov& K, int c, double scale, long long e0,
                                              long long stride, double* ws) {
    const int n = a.n;
    const long long N3 = 3LL * n;
    double* q = K.basis + (size_t)c * K.ld3;
    const double* w = K.w;
    for (long long e = e0; e < N3; e += stride) {
        int f, i;
        ex_split(e, n, f, i);
        const double x = w[e] * scale;
        q[e] = x;
        a.Lq[f][meta_pos(a.meta[i])] = x;
    }
    // ghosts: eight lanes per ghost, each gathering up to kGatherLane row
    // terms of the three fields with all its loads in flight, then the
    // group's sums in a fixed order (group_sums); the loop is uniform over
    // the warp
    const int lane = threadIdx.x & 31, gl = lane & (kGhostLanes - 1);
    const long long gstride = stride / kGhostLanes;
    for (long long base = (e0 - lane) / kGhostLanes; base < a.ng; base += gstride) {
        const long long t = base + lane / kGhostLanes;
        const bool valid = t < a.ng;
        const int gi = valid ? (int)t : 0;
        const int rl = valid ? a.row_len[gi] : 0;
        const int* ri = a.row_idx + (size_t)gi * a.rmax;
        const double* rw = a.row_w + (size_t)gi * a.rmax;
        double pv[3] = {0.0, 0.0, 0.0};
        for (int r0 = 0; r0 < rl; r0 += kGhostLanes * kGatherLane) {
            int id[kGatherLane];
            double wt[kGatherLane];
#pragma unroll
            for (int u = 0; u < kGatherLane; ++u) {
                const int r = r0 + gl + kGhostLanes * u;
                id[u] = r < rl ? ri[r] : -1;
                wt[u] = r < rl ? rw[r] : 0.0;
            }
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                double xv[kGatherLane];
#pragma unroll
                for (int u = 0; u < kGatherLane; ++u) xv[u] = id[u] >= 0 ? w[(size_t)f * n + id[u]] : 0.0;
#pragma unroll
                for (int u = 0; u < kGatherLane; ++u) pv[f] += wt[u] * xv[u];
            }
        }
        group_sums<3>(pv, ws);
        if (valid && gl == 0) {
            const int p = a.glist[gi];
            a.Lq[0][p] = pv[0] * scale;
            a.Lq[1][p] = pv[1] * scale;
            a.Lq[2][p] = pv[2] * scale;
        }
    }
}

// Lanes per basis row in the warp dots: 32 / L rows fit, L a power of two.
__device__ __forceinline__ int ex_lanes_per_row(int nv) {
    int L = 32;
    while (L > 1 && L * nv > 32) L >>= 1;
    return L;
}

// After a warp has staged the values x of its 32 consecutive stacked
// entries wb .. wb + 31 in s_x, lane l adds its share of q_t . x for row
// t = l / L (t < nv), entries l mod L, l mod L + L, ... (one FP64 operation
// per entry and lane instead of nv per entry and thread).
__device__ __forceinline__ double ex_warp_dots(const ExKrylov& K, long long N3, int nv, int L, long long wb,
                                               const double* s_x, double acc) {
    const int lane = threadIdx.x & 31;
    const int t = lane / L, sub = lane - t * L;
    if (t < nv) {
        const double* qt = K.basis + (size_t)t * K.ld3 + wb;
        const int np = (int)min(32LL, N3 - wb);
        for (int p = sub; p < np; p += L) acc += qt[p] * s_x[p];
    }
    return acc;
}

// The block's partial sums of the rows (the lanes' shares, the warps in
// order) into prow[0..nv).
__device__ __forceinline__ void ex_dots_finish(double acc, int nv, int L, double* prow, double (*s_dot)[96]) {
    constexpr int PT = kExKrylovThreads;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    s_dot[wid][lane] = acc;
    __syncthreads();
    for (int r = threadIdx.x; r < nv; r += PT) {
        double sum = 0.0;
        for (int w = 0; w < PT / 32; ++w)
            for (int s2 = 0; s2 < L; ++s2) sum += s_dot[w][r * L + s2];
        prow[r] = sum;
    }
    __syncthreads();
}

// Sum over the nb blocks' rows part[b * kOutP + t], t < nout <= 32, into
// s_out, in the same order in every block: lane l of warp w adds output
// l mod ns (ns = nout rounded up to a power of two) of blocks w + kW (g + L u),
// g = l / ns, L = 32 / ns, sixteen loads ahead of their additions; then the
// groups and the warps in order.
__device__ __forceinline__ void ex_reduce(const double* part, int nout, double* s_out, double (*s_red)[kNV + 1],
                                          int nb) {
    constexpr int PT = kExKrylovThreads, kW = PT / 32, kB = 16;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int ns = 1;
    while (ns < nout) ns <<= 1;
    const int L = 32 / ns, t = lane & (ns - 1), g = lane / ns, bstep = kW * L;
    double v = 0.0;
    if (t < nout) {
        const double* p = part + t;
        int b = wid + kW * g;
        // batches of kB loads in flight; the last one padded with zeros,
        // which leave the ordered sum unchanged
        for (; b < nb; b += kB * bstep) {
            double x[kB];
#pragma unroll
            for (int u = 0; u < kB; ++u) x[u] = b + u * bstep < nb ? p[(size_t)(b + u * bstep) * kOutP] : 0.0;
#pragma unroll
            for (int u = 0; u < kB; ++u) v += x[u];
        }
    }
    s_red[wid][lane] = v;
    __syncthreads();
    for (int q = threadIdx.x; q < nout; q += PT) {
        double sum = 0.0;
        for (int w = 0; w < kW; ++w)
            for (int gg = 0; gg < L; ++gg) sum += s_red[w][gg * ns + q];
        s_out[q] = sum;
    }
    __syncthreads();
}

// Block partial sum of v over the block's threads into *dst (warp sums
// through shared memory, then the warps in order).
__device__ __forceinline__ void ex_block_sum(double v, double* dst, double (*s_dot)[96]) {
    constexpr int PT = kExKrylovThreads;
    const int wid = threadIdx.x >> 5;
    const double ws = warp_sum(v, s_dot[wid]);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_dot[wid][0] = ws;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int w = 0; w < PT / 32; ++w) sum += s_dot[w][0];
        *dst = sum;
    }
    __syncthreads();
}

// The Krylov projection of one velocity-Exner step by every block of a
// cooperative launch over the 3 n stacked entries (block bid owns entries
// bid * PT + t, stride nb * PT).  Per Arnoldi step j: w = M q_j entry by
// entry, the first Gram-Schmidt dots (warp-transposed) and |w|^2 | w -= Q c
// and the second dots | w -= Q c' and |w|^2 | h, breakdown test, q_{j+1}
// and its lattices; each | a grid barrier.  Every block reduces the partial
// sums itself, in the same order, so all take the same decisions; block 0
// writes H and evaluates phi_1.
template <int P>
__global__ void __launch_bounds__(kExKrylovThreads, 1) k_ex_krylov(ExArgs a, ExKrylov K) {
    constexpr int PT = kExKrylovThreads;
    __shared__ double s_red[PT / 32][kNV + 1];
    __shared__ double s_h[kOutP];
    __shared__ double s_c[kNV + 1];
    __shared__ double s_x[PT / 32][32];
    __shared__ double s_dot[PT / 32][96];
    __shared__ int s_int[3];
    const int bid = blockIdx.x, nb = gridDim.x, n = a.n, m = K.m, wid = threadIdx.x >> 5;
    const long long N3 = 3LL * n;
    const long long e0 = (long long)bid * PT + threadIdx.x, stride = (long long)nb * PT;
    const long long wb0 = (long long)bid * PT + wid * 32;
    const bool lead = bid == 0 && threadIdx.x == 0;
    double* __restrict__ w = K.w;
    double* prow = K.part + (size_t)bid * kOutP;
    double nrm = 0.0;
    for (long long e = e0; e < N3; e += stride) nrm += w[e] * w[e];
    ex_block_sum(nrm, prow, s_dot);
    if (!grid_sync(K.bar, K.err, K.limit_ns, bid, nb)) return;
    ex_reduce(K.part, 1, s_h, s_red, nb);
    const double beta = sqrt(s_h[0]);
    int k = m;
    if (!(beta > 0.0) || !isfinite(beta)) {
        k = 0;
        if (lead && !isfinite(beta)) atomicOr(K.flags, 1);
    }
    if (lead) *K.beta = beta;
    if (k > 0) {
        ex_new_vector(a, K, 0, 1.0 / beta, e0, stride, s_dot[wid]);
        if (!grid_sync(K.bar, K.err, K.limit_ns, bid, nb)) return;
        for (int j = 0; j < m; ++j) {
            const double* qj = K.basis + (size_t)j * K.ld3;
            const int nv = j + 1, L = ex_lanes_per_row(nv);
            // w = M q_j; c = Q^T w and |w|^2
            nrm = 0.0;
            double acc = 0.0;
            for (long long wb = wb0; wb < N3; wb += stride) {
                const long long e = wb + (threadIdx.x & 31);
                double x = 0.0;
                if (e < N3) {
                    int f, i;
                    ex_split(e, n, f, i);
                    x = ex_entry<P>(a, qj, f, i);
                    w[e] = x;
                    nrm += x * x;
                }
                s_x[wid][threadIdx.x & 31] = x;
                __syncwarp();
                acc = ex_warp_dots(K, N3, nv, L, wb, s_x[wid], acc);
                __syncwarp();
            }
            ex_dots_finish(acc, nv, L, prow, s_dot);
            ex_block_sum(nrm, prow + nv, s_dot);
            if (!grid_sync(K.bar, K.err, K.limit_ns, bid, nb)) return;
            ex_reduce(K.part, nv + 1, s_h, s_red, nb);
            const double wn2 = s_h[nv];
            for (int t = threadIdx.x; t < nv; t += PT) {
                s_c[t] = s_h[t];
                if (bid == 0) K.H[(size_t)t * m + j] = s_h[t];
            }
            __syncthreads();
            // w -= Q c; c' = Q^T w
            acc = 0.0;
            for (long long wb = wb0; wb < N3; wb += stride) {
                const long long e = wb + (threadIdx.x & 31);
                double x = 0.0;
                if (e < N3) {
                    x = w[e];
                    for (int t = 0; t < nv; ++t) x -= s_c[t] * K.basis[(size_t)t * K.ld3 + e];
                    w[e] = x;
                }
                s_x[wid][threadIdx.x & 31] = x;
                __syncwarp();
                acc = ex_warp_dots(K, N3, nv, L, wb, s_x[wid], acc);
                __syncwarp();
            }
            ex_dots_finish(acc, nv, L, prow, s_dot);
            if (!grid_sync(K.bar, K.err, K.limit_ns, bid, nb)) return;
            ex_reduce(K.part, nv, s_h, s_red, nb);
            for (int t = threadIdx.x; t < nv; t += PT) {
                s_c[t] = s_h[t];
                if (bid == 0) K.H[(size_t)t * m + j] += s_h[t];
            }
            __syncthreads();
            // w -= Q c'; |w|^2
            nrm = 0.0;
            for (long long e = e0; e < N3; e += stride) {
                double x = w[e];
                for (int t = 0; t < nv; ++t) x -= s_c[t] * K.basis[(size_t)t * K.ld3 + e];
                w[e] = x;
                nrm += x * x;
            }
            ex_block_sum(nrm, prow, s_dot);
            if (!grid_sync(K.bar, K.err, K.limit_ns, bid, nb)) return;
            ex_reduce(K.part, 1, s_h, s_red, nb);
            const double h = sqrt(s_h[0]);
            if (lead) K.H[(size_t)(j + 1) * m + j] = h;
            const bool bad = !isfinite(h) || !isfinite(wn2);
            if (bad || h <= K.tol * sqrt(wn2)) {
                if (bad && lead) atomicOr(K.flags, 1);
                k = j + 1;
                break;
            }
            if (j + 1 == m) break;
            ex_new_vector(a, K, j + 1, 1.0 / h, e0, stride, s_dot[wid]);
            if (!grid_sync(K.bar, K.err, K.limit_ns, bid, nb)) return;
        }
    }
    if (lead) *K.kstop = k;
    if (k == 0) {
        if (bid == 0)
            for (int t = threadIdx.x; t < m; t += PT) K.y[t] = 0.0;
        return;
    }
    // y = phi_1(dt H_k) e_1 by block 0 (H written by it), then the update
    __syncthreads();
    if (bid == 0) phi1_block<PT>(K.H, k, m, K.dt, K.y, K.flags, s_red, s_c, s_int);
    if (!grid_sync(K.bar, K.err, K.limit_ns, bid, nb)) return;
    for (int t = threadIdx.x; t < k; t += PT) s_c[t] = K.dt * beta * K.y[t];
    __syncthreads();
    for (long long e = e0; e < N3; e += stride) {
        int f, i;
        ex_split(e, n, f, i);
        double inc = 0.0;
        for (int t = 0; t < k; ++t) inc += s_c[t] * K.basis[(size_t)t * K.ld3 + e];
        const double x = a.f_out[f][i] + inc;
        a.f_out[f][i] = x;
        a.Lb[f][meta_pos(a.meta[i])] = x;
    }
}

__global__ void k_ex_fill(double* __restrict__ F, long long n, double value) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        F[i] = value;
}

}  // namespace

cudaError_t ex_scatter_fields(const ExArgs& a, const double* const src[3], double* const dst[3], const int* kstop,
                              int j, cudaStream_t s) {
    k_ex_fields<<<ex_blocks((long long)a.n + a.ng), kExThreads, 0, s>>>(a.meta, a.n, a.glist, a.ng, a.row_len,
                                                                        a.row_idx, a.row_w, a.rmax, src[0], src[1],
                                                                        src[2], dst[0], dst[1], dst[2], kstop, j);
    note_launch();
    return cudaGetLastError();
}

cudaError_t ex_base(const ExArgs& a, double* w, cudaStream_t s) {
    ex_by_order(a.g.P, [&](auto PC) {
        constexpr int P = decltype(PC)::value;
        k_ex_base<P><<<ex_blocks(a.n), kExThreads, 0, s>>>(a, w);
    });
    note_launch();
    return cudaGetLastError();
}

int ex_krylov_max_blocks(int P) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaSuccess;
    ex_by_order(P, [&](auto PC) {
        constexpr int PP = decltype(PC)::value;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_ex_krylov<PP>, kExKrylovThreads, 0);
    });
    if (e != cudaSuccess || per < 1) return -1;
    return sms * per;
}

cudaError_t ex_krylov(const ExArgs& a, const ExKrylov& K, int blocks, cudaStream_t s) {
    ExArgs aa = a;
    ExKrylov kk = K;
    void* params[] = {&aa, &kk};
    cudaError_t e = cudaSuccess;
    ex_by_order(a.g.P, [&](auto PC) {
        constexpr int PP = decltype(PC)::value;
        e = cudaLaunchCooperativeKernel((const void*)k_ex_krylov<PP>, dim3(blocks), dim3(kExKrylovThreads), params,
                                        0, s);
    });
    if (e != cudaSuccess) return e;
    note_launch();
    return cudaGetLastError();
}

cudaError_t ex_fill(double* F, long long n, double value, cudaStream_t s) {
    k_ex_fill<<<ex_blocks(n), kExThreads, 0, s>>>(F, n, value);
    note_launch();
    return cudaGetLastError();
}

}  // namespace wrc
