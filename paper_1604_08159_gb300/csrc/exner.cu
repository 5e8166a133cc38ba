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
            for (int i = 0; i < rl; ++i) {
                const int q = ri[i];
                const double wt = rw[i];
                a0 += wt * s0[q];
                a1 += wt * s1[q];
                a2 += wt * s2[q];
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
template <int P>
__device__ __forceinline__ void ex_point(const ExArgs& a, const double* __restrict__ q, int i, double (&J)[3]) {
    const int n = a.n;
    const long long ld = a.ld;
    const uint32_t mw = a.meta[i];
    double dux, duy, dlu, dvx, dvy, dlv, dpx, dpy, dlp;
    point_derivs<double, P>(a.Lq[0], mw, a.g, a.c1J, a.c2J, dux, duy, dlu);
    point_derivs<double, P>(a.Lq[1], mw, a.g, a.c1J, a.c2J, dvx, dvy, dlv);
    point_derivs<double, P>(a.Lq[2], mw, a.g, a.c1J, a.c2J, dpx, dpy, dlp);
    const double du = q[i], dv = q[n + i], dp = q[2 * n + i];
    const double u = a.f[0][i], v = a.f[1][i], p = a.f[2][i];
    double Ju = -(u * dux + v * duy) - a.C * dpx + a.fc * dv - a.r * du + a.nu * dlu;
    double Jv = -(u * dvx + v * dvy) - a.C * dpy - a.fc * du - a.r * dv + a.nu * dlv;
    double Jp = -(u * dpx + v * dpy) - p * (dux + dvy);
    if (a.full) {
        const double* d = a.d;
        const double ux = d[i], uy = d[ld + i], vx = d[2 * ld + i], vy = d[3 * ld + i];
        const double px = d[4 * ld + i], py = d[5 * ld + i];
        Ju -= du * ux + dv * uy;
        Jv -= du * vx + dv * vy;
        Jp -= (du * px + dv * py) + dp * (ux + vy);
    }
    J[0] = Ju;
    J[1] = Jv;
    J[2] = Jp;
}

// Basis vector q_c = w * scale at the block's own points (stacked entries),
// its lattices at the own active points, and at the block's share of the
// ghosts (ghost bid + nb * t ...) from the interpolation rows over w (whose
// entries are final for every point when this runs).
__device__ __forceinline__ void ex_new_vector(const ExArgs& a, const ExKrylov& K, int c, double scale, int bid,
                                              int nb) {
    const int n = a.n;
    double* q = K.basis + (size_t)c * K.ld3;
    const double* w = K.w;
    for (int i = bid * kExKrylovThreads + threadIdx.x; i < n; i += nb * kExKrylovThreads) {
        const int p = meta_pos(a.meta[i]);
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            const double x = w[(size_t)f * n + i] * scale;
            q[(size_t)f * n + i] = x;
            a.Lq[f][p] = x;
        }
    }
    for (int t = bid * kExKrylovThreads + threadIdx.x; t < a.ng; t += nb * kExKrylovThreads) {
        const int rl = a.row_len[t];
        const int* ri = a.row_idx + (size_t)t * a.rmax;
        const double* rw = a.row_w + (size_t)t * a.rmax;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        for (int e = 0; e < rl; ++e) {
            const int q0 = ri[e];
            const double wt = rw[e];
            s0 += wt * w[q0];
            s1 += wt * w[n + q0];
            s2 += wt * w[2 * n + q0];
        }
        const int p = a.glist[t];
        a.Lq[0][p] = s0 * scale;
        a.Lq[1][p] = s1 * scale;
        a.Lq[2][p] = s2 * scale;
    }
}

// Block partial sums of q_t . x for t < nv (x stacked, the block's own
// points) into prow[0..nv): each warp stages its 32 points' three entries in
// shared memory and lane l forms whole dot products over them (row l mod nv
// and field l / nv when 3 nv <= 32, else row l over all three fields), so
// that no per-thread accumulator array is needed; the warps' sums are added
// in warp order.  1 <= nv <= 31.
__device__ __forceinline__ void ex_dots(const ExKrylov& K, int n, int nv, const double* __restrict__ x,
                                        double* prow, double (*s_x)[96], double (*s_dot)[40], int bid, int nb) {
    constexpr int PT = kExKrylovThreads;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const bool split = 3 * nv <= 32;
    const int t = split ? lane % nv : lane;
    const int f0 = split ? lane / nv : 0, f1 = split ? f0 + 1 : 3;
    const bool act = split ? lane < 3 * nv : lane < nv;
    const double* qt = K.basis + (size_t)(act ? t : 0) * K.ld3;
    double acc = 0.0;
    for (int wb = bid * PT + wid * 32; wb < n; wb += nb * PT) {
        const int i = wb + lane;
#pragma unroll
        for (int f = 0; f < 3; ++f) s_x[wid][f * 32 + lane] = i < n ? x[(size_t)f * n + i] : 0.0;
        __syncwarp();
        if (act) {
            const int np = min(32, n - wb);
            for (int f = f0; f < f1; ++f) {
                const double* qf = qt + (size_t)f * n + wb;
                const double* xf = s_x[wid] + f * 32;
                for (int q = 0; q < np; ++q) acc += qf[q] * xf[q];
            }
        }
        __syncwarp();
    }
    s_dot[wid][lane] = act ? acc : 0.0;
    __syncthreads();
    for (int r = threadIdx.x; r < nv; r += PT) {
        double sum = 0.0;
        for (int w = 0; w < PT / 32; ++w) {
            if (split) sum += (s_dot[w][r] + s_dot[w][nv + r]) + s_dot[w][2 * nv + r];
            else sum += s_dot[w][r];
        }
        prow[r] = sum;
    }
    __syncthreads();
}

// Block partial sum of v over the block's threads into *dst (warp sums
// through shared memory, then the warps in order).
__device__ __forceinline__ void ex_block_sum(double v, double* dst, double (*s_dot)[40]) {
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
// cooperative launch; block bid owns points bid * PT + t, stride nb * PT, and
// their three stacked entries.  Per Arnoldi step j: w = M q_j, the first
// Gram-Schmidt dots and |w|^2 | w -= Q c and the second dots | w -= Q c' and
// |w|^2 | h, breakdown test, q_{j+1} and its lattices; each | a grid
// barrier.  Every block reduces the partial sums itself, in the same order,
// so all take the same decisions; block 0 writes H and evaluates phi_1.
template <int P>
__global__ void __launch_bounds__(kExKrylovThreads, 1) k_ex_krylov(ExArgs a, ExKrylov K) {
    constexpr int PT = kExKrylovThreads;
    __shared__ double s_red[PT / 32][kNV + 1];
    __shared__ double s_h[kOutP];
    __shared__ double s_c[kNV + 1];
    __shared__ double s_x[PT / 32][96];
    __shared__ double s_dot[PT / 32][40];
    __shared__ int s_int[3];
    const int bid = blockIdx.x, nb = gridDim.x, n = a.n, m = K.m;
    const int a0 = bid * PT + threadIdx.x, stride = nb * PT;
    const bool lead = bid == 0 && threadIdx.x == 0;
    double* __restrict__ w = K.w;
    double* prow = K.part + (size_t)bid * kOutP;
    double nrm = 0.0;
    for (int i = a0; i < n; i += stride)
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            const double x = w[(size_t)f * n + i];
            nrm += x * x;
        }
    ex_block_sum(nrm, prow, s_dot);
    if (!grid_sync(K.bar, K.err, K.limit_ns, bid, nb)) return;
    reduce_all<PT>(K.part, 1, s_h, s_red, nb);
    const double beta = sqrt(s_h[0]);
    int k = m;
    if (!(beta > 0.0) || !isfinite(beta)) {
        k = 0;
        if (lead && !isfinite(beta)) atomicOr(K.flags, 1);
    }
    if (lead) *K.beta = beta;
    if (k > 0) {
        ex_new_vector(a, K, 0, 1.0 / beta, bid, nb);
        if (!grid_sync(K.bar, K.err, K.limit_ns, bid, nb)) return;
        for (int j = 0; j < m; ++j) {
            const double* qj = K.basis + (size_t)j * K.ld3;
            // w = M q_j; c = Q^T w and |w|^2
            nrm = 0.0;
            for (int i = a0; i < n; i += stride) {
                double J[3];
                ex_point<P>(a, qj, i, J);
#pragma unroll
                for (int f = 0; f < 3; ++f) w[(size_t)f * n + i] = J[f];
                nrm += (J[0] * J[0] + J[1] * J[1]) + J[2] * J[2];
            }
            __syncthreads();
            ex_dots(K, n, j + 1, w, prow, s_x, s_dot, bid, nb);
            ex_block_sum(nrm, prow + j + 1, s_dot);
            if (!grid_sync(K.bar, K.err, K.limit_ns, bid, nb)) return;
            reduce_all<PT>(K.part, j + 2, s_h, s_red, nb);
            const double wn2 = s_h[j + 1];
            for (int t = threadIdx.x; t <= j; t += PT) {
                s_c[t] = s_h[t];
                if (bid == 0) K.H[(size_t)t * m + j] = s_h[t];
            }
            __syncthreads();
            // w -= Q c; c' = Q^T w
            for (int i = a0; i < n; i += stride) {
                double x[3] = {w[i], w[n + i], w[2 * n + i]};
                for (int t = 0; t <= j; ++t) {
                    const double* qt = K.basis + (size_t)t * K.ld3;
                    const double ct = s_c[t];
                    x[0] -= ct * qt[i];
                    x[1] -= ct * qt[n + i];
                    x[2] -= ct * qt[2 * n + i];
                }
#pragma unroll
                for (int f = 0; f < 3; ++f) w[(size_t)f * n + i] = x[f];
            }
            __syncthreads();
            ex_dots(K, n, j + 1, w, prow, s_x, s_dot, bid, nb);
            if (!grid_sync(K.bar, K.err, K.limit_ns, bid, nb)) return;
            reduce_all<PT>(K.part, j + 1, s_h, s_red, nb);
            for (int t = threadIdx.x; t <= j; t += PT) {
                s_c[t] = s_h[t];
                if (bid == 0) K.H[(size_t)t * m + j] += s_h[t];
            }
            __syncthreads();
            // w -= Q c'; |w|^2
            nrm = 0.0;
            for (int i = a0; i < n; i += stride) {
                double x[3] = {w[i], w[n + i], w[2 * n + i]};
                for (int t = 0; t <= j; ++t) {
                    const double* qt = K.basis + (size_t)t * K.ld3;
                    const double ct = s_c[t];
                    x[0] -= ct * qt[i];
                    x[1] -= ct * qt[n + i];
                    x[2] -= ct * qt[2 * n + i];
                }
#pragma unroll
                for (int f = 0; f < 3; ++f) w[(size_t)f * n + i] = x[f];
                nrm += (x[0] * x[0] + x[1] * x[1]) + x[2] * x[2];
            }
            ex_block_sum(nrm, prow, s_dot);
            if (!grid_sync(K.bar, K.err, K.limit_ns, bid, nb)) return;
            reduce_all<PT>(K.part, 1, s_h, s_red, nb);
            const double h = sqrt(s_h[0]);
            if (lead) K.H[(size_t)(j + 1) * m + j] = h;
            const bool bad = !isfinite(h) || !isfinite(wn2);
            if (bad || h <= K.tol * sqrt(wn2)) {
                if (bad && lead) atomicOr(K.flags, 1);
                k = j + 1;
                break;
            }
            if (j + 1 == m) break;
            ex_new_vector(a, K, j + 1, 1.0 / h, bid, nb);
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
    for (int i = a0; i < n; i += stride) {
        const int p = meta_pos(a.meta[i]);
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            double inc = 0.0;
            for (int t = 0; t < k; ++t) inc += s_c[t] * K.basis[(size_t)t * K.ld3 + (size_t)f * n + i];
            const double x = a.f_out[f][i] + inc;
            a.f_out[f][i] = x;
            a.Lb[f][p] = x;
        }
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
