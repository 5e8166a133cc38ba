// The frozen linear operator A_n at one active point (Sec. 2.5 collocation
// derivatives at the point's stencil level j*), shared by the stand-alone
// operator kernel and the persistent Krylov kernel.
#pragma once

#include "common.cuh"

namespace wrc {

// -U Dx q - V Dy q + nu (Dxx + Dyy) q - r q at the active point described by
// the packed word mw; q is read from the lattice array F (active and ghost
// values), derivatives (order 2P = 4) with offsets +-s, +-2s (s = 2^(J-j*))
// and spacing h_{j*} = s h_J, so 1/(12 h_j) = c1J 2^-sh and
// 1/(12 h_j^2) = c2J 4^-sh; higher orders in apply_point_wide.
// x 2^-k for a positive normal x whose scaled value stays normal (here
// 1/(12 h_J) and 1/(12 h_J^2) scaled by at most 2^-2J): the exponent field
// lowered by k, which is exact and equal to ldexp(x, -k), in integer
// instructions (ldexp takes FP64 ones, the scarce pipe on this part).
__device__ __forceinline__ double pow2_down(double x, int k) {
    return __longlong_as_double(__double_as_longlong(x) - ((long long)k << 52));
}
__device__ __forceinline__ float pow2_down(float x, int k) { return __int_as_float(__float_as_int(x) - (k << 23)); }

// Order 2P > 4: the stencils of common.cuh (first derivative with reach
// 2P - 2, second derivative with reach P) at the point's stencil levels;
// c1J = 1/(d1 h_J), c2J = 1/(d2 h_J^2) with the stencils' denominators.
template <typename T, bool CG, int P>
__device__ __forceinline__ T apply_point_wide(const T* __restrict__ F, uint32_t mw, T U, T V, T nu, T r,
                                              const Geom& g, T c1J, T c2J) {
    constexpr int R1 = dd_reach1(P);
    const int p = meta_pos(mw);
    const int i = p & g.mask, k = p >> g.L;
    const int shx = g.J - meta_jx(mw), shy = g.J - meta_jy(mw);
    const int sx = 1 << shx, sy = 1 << shy;
    const T* row = F + ((size_t)k << g.L);
    const T q0 = ldv<T, CG>(row + i);
    T xp[R1], xm[R1], yp[R1], ym[R1];
#pragma unroll
    for (int o = 0; o < R1; ++o) {
        xp[o] = ldv<T, CG>(row + ((i + (o + 1) * sx) & g.mask));
        xm[o] = ldv<T, CG>(row + ((i - (o + 1) * sx) & g.mask));
        yp[o] = ldv<T, CG>(F + ((size_t)((k + (o + 1) * sy) & g.mask) << g.L) + i);
        ym[o] = ldv<T, CG>(F + ((size_t)((k - (o + 1) * sy) & g.mask) << g.L) + i);
    }
    const T c1x = pow2_down(c1J, shx), c1y = pow2_down(c1J, shy);
    const T c2x = pow2_down(c2J, 2 * shx), c2y = pow2_down(c2J, 2 * shy);
    T dx = T(dd_d1(P, 1)) * (xp[0] - xm[0]), dy = T(dd_d1(P, 1)) * (yp[0] - ym[0]);
#pragma unroll
    for (int o = 1; o < R1; ++o) {
        dx += T(dd_d1(P, o + 1)) * (xp[o] - xm[o]);
        dy += T(dd_d1(P, o + 1)) * (yp[o] - ym[o]);
    }
    T dxx = T(dd_d2(P, P)) * (xp[P - 1] + xm[P - 1]), dyy = T(dd_d2(P, P)) * (yp[P - 1] + ym[P - 1]);
#pragma unroll
    for (int o = P - 2; o >= 0; --o) {
        dxx += T(dd_d2(P, o + 1)) * (xp[o] + xm[o]);
        dyy += T(dd_d2(P, o + 1)) * (yp[o] + ym[o]);
    }
    dxx += T(dd_d2(P, 0)) * q0;
    dyy += T(dd_d2(P, 0)) * q0;
    return -U * (dx * c1x) - V * (dy * c1y) + nu * (dxx * c2x + dyy * c2y) - r * q0;
}

template <typename T, bool CG, int P = 2>
__device__ __forceinline__ T apply_point(const T* __restrict__ F, uint32_t mw, T U, T V, T nu, T r, const Geom& g,
                                         T c1J, T c2J) {
    if constexpr (P != 2) return apply_point_wide<T, CG, P>(F, mw, U, V, nu, r, g, c1J, c2J);
    const int p = meta_pos(mw);
    const int i = p & g.mask, k = p >> g.L;
    const int shx = g.J - meta_jx(mw), shy = g.J - meta_jy(mw);
    const int sx = 1 << shx, sy = 1 << shy;
    const T* row = F + ((size_t)k << g.L);
    const T q0 = ldv<T, CG>(row + i);
    const T xp1 = ldv<T, CG>(row + ((i + sx) & g.mask)), xm1 = ldv<T, CG>(row + ((i - sx) & g.mask));
    const T xp2 = ldv<T, CG>(row + ((i + 2 * sx) & g.mask)), xm2 = ldv<T, CG>(row + ((i - 2 * sx) & g.mask));
    const T yp1 = ldv<T, CG>(F + ((size_t)((k + sy) & g.mask) << g.L) + i);
    const T ym1 = ldv<T, CG>(F + ((size_t)((k - sy) & g.mask) << g.L) + i);
    const T yp2 = ldv<T, CG>(F + ((size_t)((k + 2 * sy) & g.mask) << g.L) + i);
    const T ym2 = ldv<T, CG>(F + ((size_t)((k - 2 * sy) & g.mask) << g.L) + i);
    const T c1x = pow2_down(c1J, shx), c1y = pow2_down(c1J, shy);
    const T c2x = pow2_down(c2J, 2 * shx), c2y = pow2_down(c2J, 2 * shy);
    const T Dx = (T(8) * (xp1 - xm1) - (xp2 - xm2)) * c1x;
    const T Dy = (T(8) * (yp1 - ym1) - (yp2 - ym2)) * c1y;
    const T Dxx = (-(xp2 + xm2) + T(16) * (xp1 + xm1) - T(30) * q0) * c2x;
    const T Dyy = (-(yp2 + ym2) + T(16) * (yp1 + ym1) - T(30) * q0) * c2y;
    return -U * Dx - V * Dy + nu * (Dxx + Dyy) - r * q0;
}

// The collocation derivatives of a lattice field F at the active point mw
// (Sec. 2.5, each axis at its own stencil level j*, ghost values in F):
// Dx, Dy and the Laplacian Dxx + Dyy, for the operators of the
// velocity-Exner form.
template <typename T, int P>
__device__ __forceinline__ void point_derivs(const T* __restrict__ F, uint32_t mw, const Geom& g, T c1J, T c2J,
                                             T& Dx, T& Dy, T& Lap) {
    constexpr int R1 = P == 2 ? 2 : dd_reach1(P);
    const int p = meta_pos(mw);
    const int i = p & g.mask, k = p >> g.L;
    const int shx = g.J - meta_jx(mw), shy = g.J - meta_jy(mw);
    const int sx = 1 << shx, sy = 1 << shy;
    const T* row = F + ((size_t)k << g.L);
    const T q0 = row[i];
    T xp[R1], xm[R1], yp[R1], ym[R1];
#pragma unroll
    for (int o = 0; o < R1; ++o) {
        xp[o] = row[(i + (o + 1) * sx) & g.mask];
        xm[o] = row[(i - (o + 1) * sx) & g.mask];
        yp[o] = F[((size_t)((k + (o + 1) * sy) & g.mask) << g.L) + i];
        ym[o] = F[((size_t)((k - (o + 1) * sy) & g.mask) << g.L) + i];
    }
    const T c1x = pow2_down(c1J, shx), c1y = pow2_down(c1J, shy);
    const T c2x = pow2_down(c2J, 2 * shx), c2y = pow2_down(c2J, 2 * shy);
    if constexpr (P == 2) {
        Dx = (T(8) * (xp[0] - xm[0]) - (xp[1] - xm[1])) * c1x;
        Dy = (T(8) * (yp[0] - ym[0]) - (yp[1] - ym[1])) * c1y;
        Lap = (-(xp[1] + xm[1]) + T(16) * (xp[0] + xm[0]) - T(30) * q0) * c2x +
              (-(yp[1] + ym[1]) + T(16) * (yp[0] + ym[0]) - T(30) * q0) * c2y;
    } else {
        T dx = T(dd_d1(P, 1)) * (xp[0] - xm[0]), dy = T(dd_d1(P, 1)) * (yp[0] - ym[0]);
#pragma unroll
        for (int o = 1; o < R1; ++o) {
            dx += T(dd_d1(P, o + 1)) * (xp[o] - xm[o]);
            dy += T(dd_d1(P, o + 1)) * (yp[o] - ym[o]);
        }
        T dxx = T(dd_d2(P, P)) * (xp[P - 1] + xm[P - 1]), dyy = T(dd_d2(P, P)) * (yp[P - 1] + ym[P - 1]);
#pragma unroll
        for (int o = P - 2; o >= 0; --o) {
            dxx += T(dd_d2(P, o + 1)) * (xp[o] + xm[o]);
            dyy += T(dd_d2(P, o + 1)) * (yp[o] + ym[o]);
        }
        dxx += T(dd_d2(P, 0)) * q0;
        dyy += T(dd_d2(P, 0)) * q0;
        Dx = dx * c1x;
        Dy = dy * c1y;
        Lap = dxx * c2x + dyy * c2y;
    }
}

// One collocation first derivative of a lattice field F at the active point
// mw along x (axis 0) or y (axis 1), at that axis's stencil level (Sec. 2.5).
template <typename T, int P>
__device__ __forceinline__ T point_d1(const T* __restrict__ F, uint32_t mw, const Geom& g, T c1J, int axis) {
    constexpr int R1 = dd_reach1(P);
    const int p = meta_pos(mw);
    const int i = p & g.mask, k = p >> g.L;
    const int sh = g.J - (axis == 0 ? meta_jx(mw) : meta_jy(mw));
    const int st = 1 << sh;
    T fp[R1], fm[R1];
#pragma unroll
    for (int o = 0; o < R1; ++o) {
        if (axis == 0) {
            fp[o] = F[((size_t)k << g.L) + ((i + (o + 1) * st) & g.mask)];
            fm[o] = F[((size_t)k << g.L) + ((i - (o + 1) * st) & g.mask)];
        } else {
            fp[o] = F[((size_t)((k + (o + 1) * st) & g.mask) << g.L) + i];
            fm[o] = F[((size_t)((k - (o + 1) * st) & g.mask) << g.L) + i];
        }
    }
    const T c1 = pow2_down(c1J, sh);
    if constexpr (P == 2) {
        return (T(8) * (fp[0] - fm[0]) - (fp[1] - fm[1])) * c1;
    } else {
        T d = T(dd_d1(P, 1)) * (fp[0] - fm[0]);
#pragma unroll
        for (int o = 1; o < R1; ++o) d += T(dd_d1(P, o + 1)) * (fp[o] - fm[o]);
        return d * c1;
    }
}

}  // namespace wrc
