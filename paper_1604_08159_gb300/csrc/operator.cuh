// The frozen linear operator A_n at one active point (Sec. 2.5 collocation
// derivatives at the point's stencil level j*), shared by the stand-alone
// operator kernel and the persistent Krylov kernel.
#pragma once

#include "common.cuh"

namespace wrc {

// -U Dx q - V Dy q + nu (Dxx + Dyy) q - r q at the active point described by
// the packed word mw; q is read from the lattice array F (active and ghost
// values), derivatives with offsets +-s, +-2s (s = 2^(J-j*)) and spacing
// h_{j*} = s h_J, so 1/(12 h_j) = c1J 2^-sh and 1/(12 h_j^2) = c2J 4^-sh.
// x 2^-k for a positive normal x whose scaled value stays normal (here
// 1/(12 h_J) and 1/(12 h_J^2) scaled by at most 2^-2J): the exponent field
// lowered by k, which is exact and equal to ldexp(x, -k), in integer
// instructions (ldexp takes FP64 ones, the scarce pipe on this part).
__device__ __forceinline__ double pow2_down(double x, int k) {
    return __longlong_as_double(__double_as_longlong(x) - ((long long)k << 52));
}
__device__ __forceinline__ float pow2_down(float x, int k) { return __int_as_float(__float_as_int(x) - (k << 23)); }

template <typename T, bool CG>
__device__ __forceinline__ T apply_point(const T* __restrict__ F, uint32_t mw, T U, T V, T nu, T r, const Geom& g,
                                         T c1J, T c2J) {
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

}  // namespace wrc
