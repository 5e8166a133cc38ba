// Kernels of the compressible velocity-Exner form of the model (Eqs. 1-2,
// the f-plane Coriolis term and Rayleigh friction for Eq. 4):
//   pi_t = -(u pi_x + v pi_y) - pi (u_x + v_y)
//   u_t  = -(u u_x + v u_y) - C pi_x + f (v - G_y) - r u + nu lap u
//   v_t  = -(u v_x + v v_y) - C pi_y - f (u - G_x) - r v + nu lap v
// on the adaptive collocation grid, derivatives of Sec. 2.5 at each point's
// stencil levels.  The Krylov projection of the step (Sec. 2.1) runs on the
// stacked vector [u; v; pi] of the active points as launches queued by the
// host (api.cu, with the reductions of rosenbrock.cu): per Krylov vector its
// three lattices (values at the active points, the ghosts through the
// interpolation rows) and one operator launch.  No Poisson solve.
#include "kernels.h"
#include "operator.cuh"
#include "wrc.h"

namespace wrc {

namespace {

constexpr int kExThreads = 256;
constexpr int kExMaxK = WRC_MAX_M + 1;   // Krylov dimension bound of the combination

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
__global__ void k_ex_apply(ExArgs a, const double* __restrict__ q, double* __restrict__ w,
                           const int* __restrict__ kstop, int j) {
    if (j >= *kstop) return;
    const int n = a.n;
    const long long ld = a.ld;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
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
        w[i] = Ju;
        w[n + i] = Jv;
        w[2 * n + i] = Jp;
    }
}

// U^{n+1} = U^n + dt beta V_k y (accumulated in FP64) into the compact
// arrays and the state lattices.
__global__ void k_ex_combine(ExArgs a, const double* __restrict__ basis, long long ld3, const double* __restrict__ y,
                             const double* __restrict__ beta, double dt, const int* __restrict__ kstop) {
    __shared__ double s_c[kExMaxK];
    const int k = *kstop;
    for (int t = threadIdx.x; t < k; t += blockDim.x) s_c[t] = dt * (*beta) * y[t];
    __syncthreads();
    const int n = a.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int p = meta_pos(a.meta[i]);
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            const long long e = (long long)f * n + i;
            double inc = 0.0;
            for (int t = 0; t < k; ++t) inc += s_c[t] * basis[(size_t)t * ld3 + e];
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

cudaError_t ex_apply(const ExArgs& a, const double* q, double* w, const int* kstop, int j, cudaStream_t s) {
    ex_by_order(a.g.P, [&](auto PC) {
        constexpr int P = decltype(PC)::value;
        k_ex_apply<P><<<ex_blocks(a.n), kExThreads, 0, s>>>(a, q, w, kstop, j);
    });
    note_launch();
    return cudaGetLastError();
}

cudaError_t ex_combine(const ExArgs& a, const double* basis, long long ld3, const double* y, const double* beta,
                       double dt, const int* kstop, cudaStream_t s) {
    k_ex_combine<<<ex_blocks(a.n), kExThreads, 0, s>>>(a, basis, ld3, y, beta, dt, kstop);
    note_launch();
    return cudaGetLastError();
}

cudaError_t ex_fill(double* F, long long n, double value, cudaStream_t s) {
    k_ex_fill<<<ex_blocks(n), kExThreads, 0, s>>>(F, n, value);
    note_launch();
    return cudaGetLastError();
}

}  // namespace wrc
