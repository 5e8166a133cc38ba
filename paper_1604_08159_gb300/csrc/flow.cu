// Velocity from the streamfunction, the Smagorinsky forcing of Eq. 5, the
// frozen linear operator A_n of the Krylov step (Sec. 2.5 collocation
// derivatives at each point's stencil level), and lattice diagnostics.
#include <algorithm>
#include <type_traits>

#include "kernels.h"
#include "operator.cuh"

namespace wrc {

namespace {

template <typename T>
__device__ __forceinline__ T at(const T* __restrict__ F, int i, int k, const Geom& g) {
    return F[((size_t)(k & g.mask) << g.L) + (i & g.mask)];
}

// First and second derivatives of order 2P on the finest lattice, scaled by
// c1 = 1/(d1 h), c2 = 1/(d2 h^2) with the stencils' denominators (common.cuh;
// for 2P = 4: 1/(12 h), 1/(12 h^2) and the stencils written out).
template <typename T, int P>
__device__ __forceinline__ T dx1(const T* F, int i, int k, const Geom& g, T c1) {
    if constexpr (P == 2) {
        return (T(8) * (at(F, i + 1, k, g) - at(F, i - 1, k, g)) - (at(F, i + 2, k, g) - at(F, i - 2, k, g))) * c1;
    } else {
        T acc = T(dd_d1(P, 1)) * (at(F, i + 1, k, g) - at(F, i - 1, k, g));
#pragma unroll
        for (int o = 2; o <= dd_reach1(P); ++o) acc += T(dd_d1(P, o)) * (at(F, i + o, k, g) - at(F, i - o, k, g));
        return acc * c1;
    }
}
template <typename T, int P>
__device__ __forceinline__ T dy1(const T* F, int i, int k, const Geom& g, T c1) {
    if constexpr (P == 2) {
        return (T(8) * (at(F, i, k + 1, g) - at(F, i, k - 1, g)) - (at(F, i, k + 2, g) - at(F, i, k - 2, g))) * c1;
    } else {
        T acc = T(dd_d1(P, 1)) * (at(F, i, k + 1, g) - at(F, i, k - 1, g));
#pragma unroll
        for (int o = 2; o <= dd_reach1(P); ++o) acc += T(dd_d1(P, o)) * (at(F, i, k + o, g) - at(F, i, k - o, g));
        return acc * c1;
    }
}
template <typename T, int P>
__device__ __forceinline__ T dx2(const T* F, int i, int k, const Geom& g, T c2) {
    if constexpr (P == 2) {
        return (-(at(F, i + 2, k, g) + at(F, i - 2, k, g)) + T(16) * (at(F, i + 1, k, g) + at(F, i - 1, k, g)) -
                T(30) * at(F, i, k, g)) * c2;
    } else {
        T acc = T(dd_d2(P, P)) * (at(F, i + P, k, g) + at(F, i - P, k, g));
#pragma unroll
        for (int o = P - 1; o >= 1; --o) acc += T(dd_d2(P, o)) * (at(F, i + o, k, g) + at(F, i - o, k, g));
        return (acc + T(dd_d2(P, 0)) * at(F, i, k, g)) * c2;
    }
}
template <typename T, int P>
__device__ __forceinline__ T dy2(const T* F, int i, int k, const Geom& g, T c2) {
    if constexpr (P == 2) {
        return (-(at(F, i, k + 2, g) + at(F, i, k - 2, g)) + T(16) * (at(F, i, k + 1, g) + at(F, i, k - 1, g)) -
                T(30) * at(F, i, k, g)) * c2;
    } else {
        T acc = T(dd_d2(P, P)) * (at(F, i, k + P, g) + at(F, i, k - P, g));
#pragma unroll
        for (int o = P - 1; o >= 1; --o) acc += T(dd_d2(P, o)) * (at(F, i, k + o, g) + at(F, i, k - o, g));
        return (acc + T(dd_d2(P, 0)) * at(F, i, k, g)) * c2;
    }
}

// The stencil scales of order 2P for spacing h: 1/(d1 h), 1/(d2 h^2).
template <typename T, int P>
T c1_of(double h) { return T(1.0 / (dd_d1den(P) * h)); }
template <typename T, int P>
T c2_of(double h) { return T(1.0 / (dd_d2den(P) * h * h)); }

// Calls f(std::integral_constant<int, P>) for the DD half-order g.P.
template <typename F>
void by_order(const Geom& g, F&& f) {
    if (g.P == 3) f(std::integral_constant<int, 3>{});
    else if (g.P == 4) f(std::integral_constant<int, 4>{});
    else f(std::integral_constant<int, 2>{});
}

template <typename T, int P>
__global__ void k_velocity_active(const T* __restrict__ psi, const uint32_t* __restrict__ meta, long long n,
                                  T* __restrict__ Ua, T* __restrict__ Va, Geom g, T c1, const int* __restrict__ dn) {
    pdl_wait();
    n = eff_n(dn, n);
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x) {
        const int p = meta_pos(meta[a]);
        const int i = p & g.mask, k = p >> g.L;
        Ua[a] = dy1<T, P>(psi, i, k, g, c1);
        Va[a] = -dx1<T, P>(psi, i, k, g, c1);
    }
    pdl_trigger();
}

// nu_t = (C_s h)^2 * 2 sqrt(S11^2 + S12^2) (Eq. 5); a = 2 nu_t S12, c = nu_t S11
// (nut and c may be null).
// Lattice passes over the rows of listed row pairs only (rows: the flags,
// count and list of launch_scatter; NJ = 2^lg): the number of points, and
// the lattice index of the e-th (nullptr: every point, in order).
__device__ __forceinline__ long long listed_points(const int* rows, long long N, int lg) {
    return rows ? (2LL * rows[1 << (lg - 1)]) << lg : N;
}
__device__ __forceinline__ long long listed_point(const int* rows, long long e, int lg) {
    if (!rows) return e;
    const long long slot = e >> lg;   // row slot: pair slot / 2, row of the pair slot & 1
    const int row = 2 * rows[(1 << (lg - 1)) + 1 + (int)(slot >> 1)] + (int)(slot & 1);
    return ((long long)row << lg) + (e & ((1LL << lg) - 1));
}

template <typename T>
__global__ void k_strain_nut(const T* __restrict__ S11, const T* __restrict__ S12, T* __restrict__ nut,
                             T* __restrict__ a, T* __restrict__ c, long long N, T csh2, const int* __restrict__ rows,
                             int lg) {
    pdl_wait();
    const long long tot = listed_points(rows, N, lg);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const long long p = listed_point(rows, e, lg);
        const T s11 = S11[p], s12 = S12[p];
        const T nt = csh2 * (T(2) * sqrt(s11 * s11 + s12 * s12));
        if (nut) nut[p] = nt;
        if (a) a[p] = T(2) * nt * s12;
        if (c) c[p] = nt * s11;
    }
    pdl_trigger();
}

template <typename T>
__global__ void k_velocity_gather(const T* __restrict__ Ulat, const T* __restrict__ Vlat,
                                  const uint32_t* __restrict__ meta, long long n, T* __restrict__ Ua,
                                  T* __restrict__ Va, const int* __restrict__ dn) {
    pdl_wait();
    n = eff_n(dn, n);
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x) {
        const int p = meta_pos(meta[a]);
        Ua[a] = Ulat[p];
        Va[a] = Vlat[p];
    }
    pdl_trigger();
}

// Pass 3: t0 = d(t3)/dy.
template <typename T, int P>
__global__ void k_sgs3(const T* __restrict__ t3, T* __restrict__ t0, Geom g, T c1, const int* __restrict__ rows) {
    pdl_wait();
    const long long tot = listed_points(rows, (long long)g.NJ * g.NJ, g.L);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const long long p = listed_point(rows, e, g.L);
        const int i = (int)(p & g.mask), k = (int)(p >> g.L);
        t0[p] = dy1<T, P>(t3, i, k, g, c1);
    }
    pdl_trigger();
}

// Pass 4 at the active points: g = Dxx(t2) - Dyy(t2) - 4 Dx(t0).
template <typename T, int P>
__global__ void k_sgs4(const T* __restrict__ t2, const T* __restrict__ t0, const uint32_t* __restrict__ meta,
                       long long n, T* __restrict__ ga, Geom g, T c1, T c2, const int* __restrict__ dn) {
    pdl_wait();
    n = eff_n(dn, n);
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x) {
        const int p = meta_pos(meta[a]);
        const int i = p & g.mask, k = p >> g.L;
        ga[a] = dx2<T, P>(t2, i, k, g, c2) - dy2<T, P>(t2, i, k, g, c2) - T(4) * dx1<T, P>(t0, i, k, g, c1);
    }
    pdl_trigger();
}

// Smagorinsky forcing restricted to where it is read (FP64 path).  g at an
// active point reads 2 nu_t S12 on its cross of radius P and D_y(nu_t S11) on
// its x-neighbours at distance <= 2P - 2, i.e. nu_t S12 and nu_t S11 inside
// the box of radius R = max(2P - 2, P) around it (5 x 5 for 2P = 4); those products are formed only at the lattice points
// of the union of these boxes (the halo), from psi with the same stencils in
// the same order as a full lattice pass would use.  The first visit of a
// halo point (an atomic OR on the 32-bit word holding its mask byte) appends
// it to the list hlist[1..], count in hlist[0], so the products run over the
// halo only; the list order varies, the value at each point does not.  The
// appends of a warp share one atomic addition on the count: each lane keeps
// the points it visited first as bits, the warp scans their counts, lane 0
// reserves the warp's total.  The loop runs warp-uniformly (a lane past n
// takes part with no points), so the warp's shuffles see all 32 lanes.
template <int P>
__global__ void k_sgs_halo_mark(const uint32_t* __restrict__ meta, long long n, uint8_t* __restrict__ halo,
                                int* __restrict__ hlist, Geom g, const int* __restrict__ dn) {
    pdl_wait();
    constexpr int R = dd_reach(P);
    constexpr int W = 2 * R + 1, NB = W * W, NW = (NB + 31) / 32;
    n = eff_n(dn, n);
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long a0 = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); a0 < n; a0 += stride) {
        const long long a = a0 + lane;
        unsigned fresh[NW];
#pragma unroll
        for (int w = 0; w < NW; ++w) fresh[w] = 0u;
        int i = 0, k = 0;
        if (a < n) {
            const int p = meta_pos(meta[a]);
            i = p & g.mask;
            k = p >> g.L;
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const int dk = b / W - R, di = b % W - R;
                const size_t q = ((size_t)((k + dk) & g.mask) << g.L) + ((i + di) & g.mask);
                const unsigned bit = 1u << (8 * (q & 3));
                const unsigned old = atomicOr(reinterpret_cast<unsigned*>(halo + (q & ~(size_t)3)), bit);
                if (!(old & bit)) fresh[b >> 5] |= 1u << (b & 31);
            }
        }
        int c = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) c += __popc(fresh[w]);
        int x = c;   // inclusive scan over the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        const int total = __shfl_sync(0xffffffffu, x, 31);
        int base = 0;
        if (lane == 0 && total > 0) base = atomicAdd(hlist, total);
        int off = __shfl_sync(0xffffffffu, base, 0) + x - c;
#pragma unroll
        for (int b = 0; b < NB; ++b)
            if ((fresh[b >> 5] >> (b & 31)) & 1u) {
                const int dk = b / W - R, di = b % W - R;
                hlist[1 + off++] = (int)(((size_t)((k + dk) & g.mask) << g.L) + ((i + di) & g.mask));
            }
    }
    pdl_trigger();
}

// At halo points: S11 = D_x(D_y psi), S12 = (psi_yy - psi_xx)/2,
// nu_t = (C_s h)^2 2 sqrt(S11^2 + S12^2) (Eq. 5); t2 = 2 nu_t S12, t3 = nu_t S11.
template <typename T, int P>
__global__ void k_sgs_halo_products(const T* __restrict__ psi, const int* __restrict__ hlist,
                                    T* __restrict__ t2, T* __restrict__ t3, Geom g, T c1, T c2, T csh2) {
    pdl_wait();
    const int nh = hlist[0];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nh; e += gridDim.x * blockDim.x) {
        const int p = hlist[1 + e];
        const int i = p & g.mask, k = p >> g.L;
        T s11;
        if constexpr (P == 2) {
            const T up1 = dy1<T, P>(psi, i + 1, k, g, c1), um1 = dy1<T, P>(psi, i - 1, k, g, c1);
            const T up2 = dy1<T, P>(psi, i + 2, k, g, c1), um2 = dy1<T, P>(psi, i - 2, k, g, c1);
            s11 = (T(8) * (up1 - um1) - (up2 - um2)) * c1;
        } else {
            T acc = T(dd_d1(P, 1)) * (dy1<T, P>(psi, i + 1, k, g, c1) - dy1<T, P>(psi, i - 1, k, g, c1));
#pragma unroll
            for (int o = 2; o <= dd_reach1(P); ++o)
                acc += T(dd_d1(P, o)) * (dy1<T, P>(psi, i + o, k, g, c1) - dy1<T, P>(psi, i - o, k, g, c1));
            s11 = acc * c1;
        }
        const T s12 = T(0.5) * (dy2<T, P>(psi, i, k, g, c2) - dx2<T, P>(psi, i, k, g, c2));
        const T nut = csh2 * (T(2) * sqrt(s11 * s11 + s12 * s12));
        t2[p] = T(2) * nut * s12;
        t3[p] = nut * s11;
    }
    pdl_trigger();
}

// At the active points: g = Dxx(t2) - Dyy(t2) - 4 D_x(D_y t3).
template <typename T, int P>
__global__ void k_sgs_halo_forcing(const T* __restrict__ t2, const T* __restrict__ t3,
                                   const uint32_t* __restrict__ meta, long long n, T* __restrict__ ga, Geom g, T c1,
                                   T c2, const int* __restrict__ dn) {
    pdl_wait();
    n = eff_n(dn, n);
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x) {
        const int p = meta_pos(meta[a]);
        const int i = p & g.mask, k = p >> g.L;
        T dxdy;
        if constexpr (P == 2) {
            const T vp1 = dy1<T, P>(t3, i + 1, k, g, c1), vm1 = dy1<T, P>(t3, i - 1, k, g, c1);
            const T vp2 = dy1<T, P>(t3, i + 2, k, g, c1), vm2 = dy1<T, P>(t3, i - 2, k, g, c1);
            dxdy = (T(8) * (vp1 - vm1) - (vp2 - vm2)) * c1;
        } else {
            T acc = T(dd_d1(P, 1)) * (dy1<T, P>(t3, i + 1, k, g, c1) - dy1<T, P>(t3, i - 1, k, g, c1));
#pragma unroll
            for (int o = 2; o <= dd_reach1(P); ++o)
                acc += T(dd_d1(P, o)) * (dy1<T, P>(t3, i + o, k, g, c1) - dy1<T, P>(t3, i - o, k, g, c1));
            dxdy = acc * c1;
        }
        ga[a] = dx2<T, P>(t2, i, k, g, c2) - dy2<T, P>(t2, i, k, g, c2) - T(4) * dxdy;
    }
    pdl_trigger();
}

template <typename T, int P>
__global__ void k_lattice_uv(const T* __restrict__ psi, T* __restrict__ U, T* __restrict__ V, Geom g, T c1) {
    pdl_wait();
    const long long N = (long long)g.NJ * g.NJ;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N;
         p += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(p & g.mask), k = (int)(p >> g.L);
        U[p] = dy1<T, P>(psi, i, k, g, c1);
        V[p] = -dx1<T, P>(psi, i, k, g, c1);
    }
    pdl_trigger();
}

template <typename T, int P>
__global__ void k_lattice_nut(const T* __restrict__ psi, const T* __restrict__ U, T* __restrict__ nut, Geom g,
                              T c1, T c2, T csh2) {
    pdl_wait();
    const long long N = (long long)g.NJ * g.NJ;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N;
         p += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(p & g.mask), k = (int)(p >> g.L);
        const T s11 = dx1<T, P>(U, i, k, g, c1);
        const T s12 = T(0.5) * (dy2<T, P>(psi, i, k, g, c2) - dx2<T, P>(psi, i, k, g, c2));
        nut[p] = csh2 * (T(2) * sqrt(s11 * s11 + s12 * s12));
    }
    pdl_trigger();
}

// w = A_n q at the active points: -U Dx q - V Dy q + nu (Dxx + Dyy) q - r q (+ g),
// each derivative along its axis at the point's stencil level j*, i.e. with
// lattice offsets +-s, +-2s, s = 2^(J-j*), and spacing h_{j*} = s h_J.
template <typename T, int P>
__global__ void __launch_bounds__(kThreads) k_matvec(const T* __restrict__ F, const uint32_t* __restrict__ meta,
                                                     long long n, const T* __restrict__ Ua,
                                                     const T* __restrict__ Va, const T* __restrict__ ga, T nu,
                                                     T r, T* __restrict__ w, Geom g, T c1J, T c2J,
                                                     const int* __restrict__ kstop, int jstep) {
    pdl_wait();
    if (kstop && jstep >= *kstop) return;
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x) {
        T v = apply_point<T, false, P>(F, meta[a], Ua[a], Va[a], nu, r, g, c1J, c2J);
        if (ga) v += ga[a];
        w[a] = v;
    }
    pdl_trigger();
}

// Lattice sums of R, R^2, U^2 + V^2 and |grad R|^2 (deterministic two-stage
// reduction: per-block partials, then the last block sums them in order).
template <typename T, int P>
__global__ void __launch_bounds__(kThreads) k_diag(const T* __restrict__ R, const T* __restrict__ psi,
                                                   double* __restrict__ partials, unsigned* __restrict__ counter,
                                                   double* __restrict__ out, Geom g, T c1) {
    pdl_wait();
    __shared__ double s_red[kThreads / 32][4];
    __shared__ bool s_last;
    const long long N = (long long)g.NJ * g.NJ;
    double acc[4] = {0, 0, 0, 0};
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N;
         p += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(p & g.mask), k = (int)(p >> g.L);
        const double r = (double)R[p];
        const double U = (double)dy1<T, P>(psi, i, k, g, c1), V = -(double)dx1<T, P>(psi, i, k, g, c1);
        const double gx = (double)dx1<T, P>(R, i, k, g, c1), gy = (double)dy1<T, P>(R, i, k, g, c1);
        acc[0] += r;
        acc[1] += r * r;
        acc[2] += U * U + V * V;
        acc[3] += gx * gx + gy * gy;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        double v = acc[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) s_red[wid][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double v = 0;
        for (int w = 0; w < kThreads / 32; ++w) v += s_red[w][threadIdx.x];
        partials[(size_t)blockIdx.x * 4 + threadIdx.x] = v;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (s_last) {
        __threadfence();
        if (threadIdx.x < 4) {
            double v = 0;
            for (unsigned b = 0; b < gridDim.x; ++b) v += __ldcg(&partials[(size_t)b * 4 + threadIdx.x]);
            out[threadIdx.x] = v;
        }
        if (threadIdx.x == 0) *counter = 0;
    }
    pdl_trigger();
}

}  // namespace

template <typename T>
void launch_velocity_active(const T* psi, const uint32_t* meta, long long n, T* Ua, T* Va, const Geom& g,
                            cudaStream_t s, const int* dn) {
    if (n <= 0) return;
    by_order(g, [&](auto PC) {
        constexpr int P = decltype(PC)::value;
        launch_pdl(k_velocity_active<T, P>, blocks_for(n), kThreads, 0, s, psi, meta, n, Ua, Va, g, c1_of<T, P>(g.h),
                   dn);
    });
    note_launch();
}

template <typename T>
void launch_sgs_halo(const T* psi, const uint32_t* meta, long long n, double cs, T* ga, T* t2, T* t3, uint8_t* halo,
                     int* hlist, const Geom& g, cudaStream_t s, const int* dn) {
    const long long N = (long long)g.NJ * g.NJ;
    const T csh2 = T((cs * g.h) * (cs * g.h));
    cudaMemsetAsync(halo, 0, (size_t)N, s);
    cudaMemsetAsync(hlist, 0, sizeof(int), s);
    by_order(g, [&](auto PC) {
        constexpr int P = decltype(PC)::value;
        const T c1 = c1_of<T, P>(g.h), c2 = c2_of<T, P>(g.h);
        if (n > 0) { launch_pdl(k_sgs_halo_mark<P>, blocks_for(n), kThreads, 0, s, meta, n, halo, hlist, g, dn); note_launch(); }
        // grid-stride over the halo count on the device (capturable); 8 blocks per SM of 152
        { launch_pdl(k_sgs_halo_products<T, P>, (int)std::min<long long>(blocks_for(N), 1216), kThreads, 0, s, psi,
                     (const int*)hlist, t2, t3, g, c1, c2, csh2); note_launch(); }
        if (n > 0) { launch_pdl(k_sgs_halo_forcing<T, P>, blocks_for(n), kThreads, 0, s, t2, t3, meta, n, ga, g, c1, c2, dn); note_launch(); }
    });
}

template <typename T>
void launch_sgs_from_strain(const T* S11, const T* S12, const uint32_t* meta, long long n, double cs, T* ga, T* ta,
                            T* tc, T* tdyc, const Geom& g, cudaStream_t s, const int* dn, const int* rows) {
    const long long N = (long long)g.NJ * g.NJ;
    const T csh2 = T((cs * g.h) * (cs * g.h));
    { launch_pdl(k_strain_nut<T>, blocks_for(N), kThreads, 0, s, S11, S12, nullptr, ta, tc, N, csh2, rows, g.L); note_launch(); }
    by_order(g, [&](auto PC) {
        constexpr int P = decltype(PC)::value;
        const T c1 = c1_of<T, P>(g.h), c2 = c2_of<T, P>(g.h);
        { launch_pdl(k_sgs3<T, P>, blocks_for(N), kThreads, 0, s, tc, tdyc, g, c1, rows); note_launch(); }
        if (n > 0) { launch_pdl(k_sgs4<T, P>, blocks_for(n), kThreads, 0, s, ta, tdyc, meta, n, ga, g, c1, c2, dn); note_launch(); }
    });
}

template <typename T>
void launch_nut_from_strain(const T* S11, const T* S12, T* nut, double cs, const Geom& g, cudaStream_t s) {
    const long long N = (long long)g.NJ * g.NJ;
    { launch_pdl(k_strain_nut<T>, blocks_for(N), kThreads, 0, s, S11, S12, nut, nullptr, nullptr, N,
                                                          T((cs * g.h) * (cs * g.h)), (const int*)nullptr, g.L); note_launch(); }
}

template <typename T>
void launch_velocity_gather(const T* Ulat, const T* Vlat, const uint32_t* meta, long long n, T* Ua, T* Va,
                            cudaStream_t s, const int* dn) {
    if (n > 0) { launch_pdl(k_velocity_gather<T>, blocks_for(n), kThreads, 0, s, Ulat, Vlat, meta, n, Ua, Va, dn); note_launch(); }
}

template <typename T>
void launch_lattice_uv_nut(const T* psi, T* U, T* V, T* nut, double cs, T* tmp, const Geom& g, cudaStream_t s,
                           bool uv_given) {
    const long long N = (long long)g.NJ * g.NJ;
    T* Uw = U ? U : tmp;
    by_order(g, [&](auto PC) {
        constexpr int P = decltype(PC)::value;
        const T c1 = c1_of<T, P>(g.h), c2 = c2_of<T, P>(g.h);
        if (!uv_given) { launch_pdl(k_lattice_uv<T, P>, blocks_for(N), kThreads, 0, s, psi, Uw, V ? V : tmp + N, g, c1); note_launch(); }
        if (nut)
            { launch_pdl(k_lattice_nut<T, P>, blocks_for(N), kThreads, 0, s, psi, Uw, nut, g, c1, c2, T((cs * g.h) * (cs * g.h))); note_launch(); }
    });
}

template <typename T>
void launch_matvec(const T* F, const uint32_t* meta, long long n, const T* Ua, const T* Va, const T* ga, double nu,
                   double r, T* w, const Geom& g, const int* kstop, int jstep, cudaStream_t s) {
    if (n <= 0) return;
    by_order(g, [&](auto PC) {
        constexpr int P = decltype(PC)::value;
        launch_pdl(k_matvec<T, P>, blocks_for(n), kThreads, 0, s, F, meta, n, Ua, Va, ga, T(nu), T(r), w, g,
                   c1_of<T, P>(g.h), c2_of<T, P>(g.h), kstop, jstep);
    });
    note_launch();
}

template <typename T>
cudaError_t launch_diag(const T* R, const T* psi, double* partials, unsigned* counter, double* out, const Geom& g,
                        cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    by_order(g, [&](auto PC) {
        constexpr int P = decltype(PC)::value;
        e = launch_pdl(k_diag<T, P>, blocks_for((long long)g.NJ * g.NJ), kThreads, 0, s, R, psi, partials, counter,
                       out, g, c1_of<T, P>(g.h));
    });
    if (e == cudaSuccess) note_launch();
    return e;
}

template <typename A, typename B>
__global__ void k_convert(const A* __restrict__ in, B* __restrict__ out, long long n) {
    pdl_wait();
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        out[t] = (B)in[t];
    pdl_trigger();
}

template <typename A, typename B>
void launch_convert(const A* in, B* out, long long n, cudaStream_t s) {
    if (n > 0) { launch_pdl(k_convert<A, B>, blocks_for(n), kThreads, 0, s, in, out, n); note_launch(); }
}
template void launch_convert<double, float>(const double*, float*, long long, cudaStream_t);
template void launch_convert<float, double>(const float*, double*, long long, cudaStream_t);

#define WRC_INST(T)                                                                                          \
    template void launch_velocity_active<T>(const T*, const uint32_t*, long long, T*, T*, const Geom&,      \
                                            cudaStream_t, const int*);                                      \
    template void launch_sgs_halo<T>(const T*, const uint32_t*, long long, double, T*, T*, T*, uint8_t*,    \
                                     int*, const Geom&, cudaStream_t, const int*);                          \
    template void launch_velocity_gather<T>(const T*, const T*, const uint32_t*, long long, T*, T*,         \
                                            cudaStream_t, const int*);                                      \
    template void launch_sgs_from_strain<T>(const T*, const T*, const uint32_t*, long long, double, T*, T*, \
                                            T*, T*, const Geom&, cudaStream_t, const int*, const int*);     \
    template void launch_nut_from_strain<T>(const T*, const T*, T*, double, const Geom&, cudaStream_t);     \
    template void launch_lattice_uv_nut<T>(const T*, T*, T*, T*, double, T*, const Geom&, cudaStream_t,     \
                                           bool);                                                           \
    template void launch_matvec<T>(const T*, const uint32_t*, long long, const T*, const T*, const T*,      \
                                   double, double, T*, const Geom&, const int*, int, cudaStream_t);        \
    template cudaError_t launch_diag<T>(const T*, const T*, double*, unsigned*, double*, const Geom&, cudaStream_t);
WRC_INST(double)
WRC_INST(float)
#undef WRC_INST

}  // namespace wrc
