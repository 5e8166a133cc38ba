// Streamfunction solve on the periodic finest lattice: psi = L_h^{-1}(-(R - mean R))
// with L_h the 4th-order collocation Laplacian (the Sec. 2.5 stencil at h_J),
// diagonalised by the 2-D DFT.
//
// The lattice field is real, so two rows share one complex FFT along x and
// only the kx = 0 .. n/2 half of each row's spectrum is kept, kx = n/2 packed
// into the imaginary part of the kx = 0 bin (both bins are real):
//   1. rows (2q, 2q+1) -> half spectra            (n/2 transforms along x)
//   2. transpose n x n/2 -> n/2 x n
//   3. per column kx: FFT along y, divide by the symbol, inverse FFT along y
//      (n/2 transforms; optionally also the full spectra of U + i V and of
//      S11 + i S12, two columns kx and n - kx from each half column)
//   4. transpose back, 5. inverse FFT along x of two real rows at a time.
// Each FFT runs radix-16 Stockham passes (a radix-2/4/8 pass first when log2 n
// is not a multiple of 4) on 16 values per thread held in registers, and
// exchanges them through padded shared memory between passes (two exchanges
// for n = 4096); no bit reversal.
#include <type_traits>

#include <cstdlib>

#include "kernels.h"

namespace wrc {

namespace {

template <typename T> struct Cx;
template <> struct Cx<double> { using type = double2; };
template <> struct Cx<float> { using type = float2; };
template <typename T> using cx_t = typename Cx<T>::type;

template <typename C>
__device__ __forceinline__ C mk(decltype(C{}.x) a, decltype(C{}.x) b) { C c; c.x = a; c.y = b; return c; }
template <typename C>
__device__ __forceinline__ C cadd(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <typename C>
__device__ __forceinline__ C csub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
template <typename C>
__device__ __forceinline__ C cmul(C a, C b) { return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename C>
__device__ __forceinline__ C cconj(C a) { return mk<C>(a.x, -a.y); }
template <typename C>
__device__ __forceinline__ C cscale(C a, decltype(C{}.x) s) { return mk<C>(a.x * s, a.y * s); }
// a * (-i) for the forward transform, a * (+i) for the inverse
template <bool INV, typename C>
__device__ __forceinline__ C mul_mi(C a) { return INV ? mk<C>(-a.y, a.x) : mk<C>(a.y, -a.x); }
// a * w (forward) or a * conj(w) (inverse), w = exp(-2 pi i m / N) given by (c, s) = (cos, sin)
template <bool INV, typename C>
__device__ __forceinline__ C rot(C a, double c, double s) {
    using R = decltype(C{}.x);
    const R cr = (R)c, sr = INV ? (R)s : (R)(-s);   // w = c + i sr
    return mk<C>(a.x * cr - a.y * sr, a.x * sr + a.y * cr);
}

// cos and sin of pi/8 and pi/4
constexpr double kC8 = 0.92387953251128675613;
constexpr double kS8 = 0.38268343236508977173;
constexpr double kR2 = 0.70710678118654752440;

// ---- DFTs of 2, 4, 8 and 16 points in registers (natural order in and out) --
template <bool INV, typename C>
__device__ __forceinline__ void dft2(C& a, C& b) {
    const C t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

template <bool INV, typename C>
__device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
    const C s0 = cadd(a0, a2), d0 = csub(a0, a2);
    const C s1 = cadd(a1, a3), d1 = mul_mi<INV>(csub(a1, a3));
    a0 = cadd(s0, s1);
    a2 = csub(s0, s1);
    a1 = cadd(d0, d1);
    a3 = csub(d0, d1);
}

// 8 points: two 4-point DFTs of the even and odd samples, then the radix-2
// combination with w8^k.
template <bool INV, typename C>
__device__ __forceinline__ void dft8(C (&a)[8]) {
    C e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
    C o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
    dft4<INV>(e0, e1, e2, e3);
    dft4<INV>(o0, o1, o2, o3);
    o1 = rot<INV>(o1, kR2, kR2);
    o2 = mul_mi<INV>(o2);
    o3 = rot<INV>(o3, -kR2, kR2);
    a[0] = cadd(e0, o0);
    a[4] = csub(e0, o0);
    a[1] = cadd(e1, o1);
    a[5] = csub(e1, o1);
    a[2] = cadd(e2, o2);
    a[6] = csub(e2, o2);
    a[3] = cadd(e3, o3);
    a[7] = csub(e3, o3);
}

// 16 points as 4 x 4: index n = 4 n1 + n2, k = k1 + 4 k2.  DFT over n1 for
// each n2, twiddle w16^(n2 k1), DFT over n2 for each k1; slot 4 k1 + k2 then
// holds X[k1 + 4 k2].
template <bool INV, typename C>
__device__ __forceinline__ void dft16(C (&a)[16]) {
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4<INV>(a[n2], a[4 + n2], a[8 + n2], a[12 + n2]);
    // slot 4 k1 + n2 holds b[n2][k1]; w16^m = (cos, sin)(2 pi m / 16)
    a[5] = rot<INV>(a[5], kC8, kS8);        // k1 = 1, n2 = 1: m = 1
    a[6] = rot<INV>(a[6], kR2, kR2);        // k1 = 1, n2 = 2: m = 2
    a[7] = rot<INV>(a[7], kS8, kC8);        // k1 = 1, n2 = 3: m = 3
    a[9] = rot<INV>(a[9], kR2, kR2);        // k1 = 2, n2 = 1: m = 2
    a[10] = mul_mi<INV>(a[10]);             // k1 = 2, n2 = 2: m = 4
    a[11] = rot<INV>(a[11], -kR2, kR2);     // k1 = 2, n2 = 3: m = 6
    a[13] = rot<INV>(a[13], kS8, kC8);      // k1 = 3, n2 = 1: m = 3
    a[14] = rot<INV>(a[14], -kR2, kR2);     // k1 = 3, n2 = 2: m = 6
    a[15] = rot<INV>(a[15], -kC8, -kS8);    // k1 = 3, n2 = 3: m = 9
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4<INV>(a[4 * k1], a[4 * k1 + 1], a[4 * k1 + 2], a[4 * k1 + 3]);
    C t[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) t[k1 + 4 * k2] = a[4 * k1 + k2];
#pragma unroll
    for (int q = 0; q < 16; ++q) a[q] = t[q];
}

template <int R, bool INV, typename C>
__device__ __forceinline__ void dft(C (&u)[R]) {
    if constexpr (R == 2) dft2<INV>(u[0], u[1]);
    else if constexpr (R == 4) dft4<INV>(u[0], u[1], u[2], u[3]);
    else if constexpr (R == 8) dft8<INV>(u);
    else dft16<INV>(u);
}

// Shared-memory index with one pad slot per 16 (spreads the strided writes
// of the early passes over the banks).
__device__ __forceinline__ int pad(int x) { return x + (x >> 4); }

template <int N> struct Log2;
template <> struct Log2<2> { static constexpr int v = 1; };
template <> struct Log2<4> { static constexpr int v = 2; };
template <> struct Log2<8> { static constexpr int v = 3; };
template <> struct Log2<16> { static constexpr int v = 4; };

// One Stockham pass of radix R over a length-n sequence whose current values
// sit in the registers of the nt = n/E threads of this transform, v[e] being
// element i + e nt.  Butterfly b (thread i takes b = i + nt g, g < E/R) reads
// elements b + r n/R, multiplies them by w_{R p}^{r k} (k = b mod p, p the
// length of the sub-transforms done so far), takes their R-point DFT and
// writes element r to (b - k) R + k + r p.  After the last pass (p = n/R)
// that position is b + r n/R, so the outputs stay in the same registers;
// otherwise they go through shared memory and come back strided.
// The twiddles of a pass come from its own table ptw[r p + k] = w_{R p}^{r k}
// (r < R, k < p): the lanes of a warp hold consecutive k, so each load of a
// warp reads consecutive entries.
template <int E, int R, bool INV, typename C>
__device__ __forceinline__ void radix_pass(C (&v)[E], C* sm, int i, int nt, int p, const C* __restrict__ ptw,
                                           bool last) {
    constexpr int G = E / R;
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const int b = i + nt * g;
        const int k = b & (p - 1);
        C u[R];
#pragma unroll
        for (int r = 0; r < R; ++r) u[r] = v[g + r * G];
        if (p > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                C w = __ldg(ptw + r * p + k);
                if (INV) w.y = -w.y;
                u[r] = cmul(u[r], w);
            }
        }
        dft<R, INV>(u);
        if (last) {
#pragma unroll
            for (int r = 0; r < R; ++r) v[g + r * G] = u[r];
        } else {
            const int base = (b - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) sm[pad(base + r * p)] = u[r];
        }
    }
    if (!last) {
        __syncthreads();
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = sm[pad(i + e * nt)];
        __syncthreads();
    }
}

// Length-n FFT (n = 2^logn) of the strided register vector v (v[e] = element
// i + e n/E on entry and on exit): a radix-R0 pass first when R0 > 1, then
// radix-E passes.  Unnormalised; INV uses exp(+2 pi i ...).  Every thread of
// the block must call it (it synchronises the block).
// tw: the per-pass twiddle tables, one after the other for the passes with
// p > 1 (R p entries each), as built by k_fft_pass_tables.
template <int E, int R0, bool INV, typename C>
__device__ __forceinline__ void fft_reg(C (&v)[E], C* sm, int i, int n, int logn, const C* __restrict__ tw) {
    const int nt = n / E;
    int p = 1, logp = 0;
    const C* ptw = tw;
    if constexpr (R0 > 1) {
        radix_pass<E, R0, INV>(v, sm, i, nt, p, ptw, false);   // p = 1: no twiddles
        p *= R0;
        logp += Log2<R0>::v;
    }
    const int npass = (logn - logp) / Log2<E>::v;
    for (int q = 0; q < npass; ++q) {
        radix_pass<E, E, INV>(v, sm, i, nt, p, ptw, q == npass - 1);
        if (p > 1) ptw += E * p;
        p *= E;
        logp += Log2<E>::v;
    }
}

// The per-pass tables of fft_reg from tw[t] = exp(-2 pi i t / n): for each
// pass with sub-length p > 1 and radix R, entries w_{R p}^{r k} = tw[(r k) n / (R p)]
// at [r p + k] (copies, so the transforms are those of the single table).
template <typename C>
__global__ void k_fft_pass_tables(const C* __restrict__ tw, C* __restrict__ ptw, int n, int logn, int E, int R0) {
    pdl_wait();
    int p = 1, logp = 0, off = 0;
    auto table = [&](int R, int logR) {
        if (p > 1)
            for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < R * p; idx += gridDim.x * blockDim.x) {
                const int r = idx / p, k = idx - r * p;
                ptw[off + idx] = tw[(r * k) << (logn - logp - logR)];
            }
        if (p > 1) off += R * p;
        p *= R;
        logp += logR;
    };
    int logE = 0;
    while ((1 << logE) < E) ++logE;
    if (R0 > 1) {
        int logR0 = 0;
        while ((1 << logR0) < R0) ++logR0;
        table(R0, logR0);
    }
    while (logp < logn) table(E, logE);
    pdl_trigger();
}

// ---- kernels ------------------------------------------------------------------
// Launch shape: transforms of nt = n/E threads each, F = max(1, 128/nt) of
// them per block, each with its own padded shared buffer of smlen values.
__host__ __device__ constexpr int smlen_of(int n) { return n + n / 16 + 1; }

// Step 1: rows 2q and 2q+1 of the real field R as z = R[2q] + i R[2q+1];
// their spectra from Z = FFT(z): X_a[k] = (Z[k] + conj Z[n-k]) / 2,
// X_b[k] = -i (Z[k] - conj Z[n-k]) / 2, kept for k < n/2 in S (n x n/2), with
// S[y][0] = X_y[0] + i X_y[n/2].
template <typename T, int E, int R0>
__global__ void __launch_bounds__(256) k_px_fwd(const T* __restrict__ Rf, cx_t<T>* __restrict__ S, int n, int logn,
                                                const cx_t<T>* __restrict__ tw) {
    pdl_wait();
    using C = cx_t<T>;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nt = n / E, F = blockDim.x / nt;
    const int f = threadIdx.x / nt, i = threadIdx.x - f * nt;
    const int h = n / 2;
    const int q = blockIdx.x * F + f;
    const bool on = q < h;
    C* sm = (C*)smraw + (size_t)f * smlen_of(n);
    C v[E];
    const T* r0 = Rf + (size_t)(2 * q) * n;
    const T* r1 = r0 + n;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int x = i + e * nt;
        v[e] = on ? mk<C>(r0[x], r1[x]) : mk<C>(T(0), T(0));
    }
    fft_reg<E, R0, false>(v, sm, i, n, logn, tw);
#pragma unroll
    for (int e = 0; e < E; ++e) sm[pad(i + e * nt)] = v[e];
    __syncthreads();
    C* sa = S + (size_t)(2 * q) * h;
    C* sb = sa + h;
#pragma unroll
    for (int e = 0; e < E / 2; ++e) {
        const int x = i + e * nt;   // < n/2
        if (!on) continue;
        const C z = v[e];
        if (x == 0) {
            const C zh = sm[pad(h)];
            sa[0] = mk<C>(z.x, zh.x);
            sb[0] = mk<C>(z.y, zh.y);
        } else {
            const C zm = cconj(sm[pad(n - x)]);
            const C s = cadd(z, zm), d = csub(z, zm);
            sa[x] = cscale(s, T(0.5));
            sb[x] = mk<C>(T(0.5) * d.y, T(-0.5) * d.x);
        }
    }
    pdl_trigger();
}

// Step 3: column kx of the transposed half spectrum (row kx of ST, length n):
// FFT along y, then per ky the two values X1, X2 --
//   kx > 0: X1 = F(ky) f(kx, ky), X2 = conj F(n-ky) f(kx, ky)  (= conj psi_hat(kx, n-ky)),
//   kx = 0: the packed column holds kx = 0 and kx = n/2:
//           C0 = (F + conj Fm)/2, CN = -i (F - conj Fm)/2 (Fm = F(n-ky)),
//           X1 = C0 f(0, ky) (0 at ky = 0), X2 = CN f(n/2, ky),
// with f = scale / (sigma(kx) + sigma(ky)).  psi: inverse FFT of X1 (kx > 0)
// or X1 + i X2 (kx = 0), written back into ST.  With QT, columns c1 = kx and
// c2 = n - kx (kx = 0: c2 = n/2) of the full spectrum of U + i V,
// (d(kx) + i d(ky)) X1 and (-d(kx) + i d(ky)) X2 (d the first-derivative
// symbol, odd, 0 at 0 and n/2); with WT those of S11 + i S12,
// (-d(kx) d(ky) + i (sigma(kx) - sigma(ky))/2) X1 and
// (d(kx) d(ky) + i (sigma(c2) - sigma(ky))/2) X2.  Each is inverse-transformed
// along y into row c of QT / WT (n x n).
template <typename T, int E, int R0, bool QW>
__global__ void __launch_bounds__(256) k_py_solve(cx_t<T>* __restrict__ ST, cx_t<T>* __restrict__ QT,
                                                  cx_t<T>* __restrict__ WT, int n, int logn,
                                                  const cx_t<T>* __restrict__ tw, const T* __restrict__ sigma,
                                                  const T* __restrict__ dsym, T scale, int want_psi) {
    pdl_wait();
    using C = cx_t<T>;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nt = n / E, F = blockDim.x / nt;
    const int f = threadIdx.x / nt, i = threadIdx.x - f * nt;
    const int h = n / 2;
    const int kx = blockIdx.x * F + f;
    const bool on = kx < h;
    const int kxs = on ? kx : 0;
    // exchange buffer of the FFT passes; with QW the forward spectrum keeps a
    // buffer of its own (F(ky) in natural order), from which every output
    // recomputes its values instead of holding them in registers
    C* sm = (C*)smraw + (size_t)f * (QW ? 2 : 1) * smlen_of(n);
    C* fb = QW ? sm + smlen_of(n) : sm;
    C* row = ST + (size_t)kxs * n;
    C v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = on ? row[i + e * nt] : mk<C>(T(0), T(0));
    fft_reg<E, R0, false>(v, sm, i, n, logn, tw);
#pragma unroll
    for (int e = 0; e < E; ++e) fb[pad(i + e * nt)] = v[e];
    __syncthreads();
    const T sx = sigma[kxs], sh = sigma[h];
    // X1, X2 at ky from the forward spectrum (see above)
    auto x12 = [&](int ky, C& a, C& b) {
        const C fk = fb[pad(ky)];
        const C fm = cconj(fb[pad((n - ky) & (n - 1))]);
        const T sy = sigma[ky];
        if (kxs == 0) {
            const C s = cadd(fk, fm), d = csub(fk, fm);
            const T f0 = ky == 0 ? T(0) : scale / (sx + sy);
            const T fn = scale / (sh + sy);
            a = cscale(s, T(0.5) * f0);
            b = mk<C>(T(0.5) * fn * d.y, T(-0.5) * fn * d.x);
        } else {
            const T fc = scale / (sx + sy);
            a = cscale(fk, fc);
            b = cscale(fm, fc);
        }
    };
    // psi: X1 (kx > 0) or X1 + i X2 (packed kx = 0, n/2); a step of the FP32
    // form (want_psi 0, uniform over the grid) reads U and V, not psi
    if (!QW || want_psi) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            C a, b;
            x12(i + e * nt, a, b);
            v[e] = kxs == 0 ? mk<C>(a.x - b.y, a.y + b.x) : a;
        }
        if constexpr (!QW) __syncthreads();   // fb is the exchange buffer
        fft_reg<E, R0, true>(v, sm, i, n, logn, tw);
        if (on)
#pragma unroll
            for (int e = 0; e < E; ++e) row[i + e * nt] = v[e];
    }
    if constexpr (QW) {
        const int c2 = kxs == 0 ? h : n - kxs;
        const T dx = dsym[kxs], sc2 = sigma[c2];
        // U + i V, columns c1 = kx and c2
#pragma unroll
        for (int e = 0; e < E; ++e) {
            C a, b;
            x12(i + e * nt, a, b);
            v[e] = cmul(a, mk<C>(dx, dsym[i + e * nt]));
        }
        fft_reg<E, R0, true>(v, sm, i, n, logn, tw);
        if (on)
#pragma unroll
            for (int e = 0; e < E; ++e) QT[(size_t)kxs * n + i + e * nt] = v[e];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            C a, b;
            x12(i + e * nt, a, b);
            v[e] = cmul(b, mk<C>(-dx, dsym[i + e * nt]));
        }
        fft_reg<E, R0, true>(v, sm, i, n, logn, tw);
        if (on)
#pragma unroll
            for (int e = 0; e < E; ++e) QT[(size_t)c2 * n + i + e * nt] = v[e];
        if (WT) {
            // S11 + i S12
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int ky = i + e * nt;
                C a, b;
                x12(ky, a, b);
                v[e] = cmul(a, mk<C>(-dx * dsym[ky], T(0.5) * (sx - sigma[ky])));
            }
            fft_reg<E, R0, true>(v, sm, i, n, logn, tw);
            if (on)
#pragma unroll
                for (int e = 0; e < E; ++e) WT[(size_t)kxs * n + i + e * nt] = v[e];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int ky = i + e * nt;
                C a, b;
                x12(ky, a, b);
                v[e] = cmul(b, mk<C>(dx * dsym[ky], T(0.5) * (sc2 - sigma[ky])));
            }
            fft_reg<E, R0, true>(v, sm, i, n, logn, tw);
            if (on)
#pragma unroll
                for (int e = 0; e < E; ++e) WT[(size_t)c2 * n + i + e * nt] = v[e];
        }
    }
    pdl_trigger();
}

// Step 5 for psi: rows 2q, 2q+1 from their half spectra (Hermitian extension
// X[n-k] = conj X[k]; X[0], X[n/2] from the packed bin): Z = X_a + i X_b,
// inverse FFT, real part to row 2q, imaginary part to row 2q+1.  With rows
// (the list of the pairs wanted: count at rows[h], pairs from rows[h + 1]),
// block b transforms the listed pairs b F .. b F + F - 1 and the blocks past
// the list return at once; a pair is transformed independently of the
// others, so the rows computed are the same.
template <typename T, int E, int R0>
__global__ void __launch_bounds__(256) k_px_inv_real(const cx_t<T>* __restrict__ S, T* __restrict__ out, int n,
                                                     int logn, const cx_t<T>* __restrict__ tw,
                                                     const int* __restrict__ rows) {
    pdl_wait();
    using C = cx_t<T>;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nt = n / E, F = blockDim.x / nt;
    const int f = threadIdx.x / nt, i = threadIdx.x - f * nt;
    const int h = n / 2;
    int q = blockIdx.x * F + f;
    if (rows) {
        const int cnt = rows[h];
        if ((int)blockIdx.x * F >= cnt) {
            pdl_trigger();
            return;
        }
        q = q < cnt ? rows[h + 1 + q] : h;   // h: no pair
    }
    const bool on = q < h;
    C* sm = (C*)smraw + (size_t)f * smlen_of(n);
    const C* sa = S + (size_t)(2 * (on ? q : 0)) * h;
    const C* sb = sa + h;
    C v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int x = i + e * nt;
        C a, b;
        if (x == 0) {
            a = mk<C>(sa[0].x, T(0));
            b = mk<C>(sb[0].x, T(0));
        } else if (x == h) {
            a = mk<C>(sa[0].y, T(0));
            b = mk<C>(sb[0].y, T(0));
        } else if (x < h) {
            a = sa[x];
            b = sb[x];
        } else {
            a = cconj(sa[n - x]);
            b = cconj(sb[n - x]);
        }
        v[e] = mk<C>(a.x - b.y, a.y + b.x);
    }
    fft_reg<E, R0, true>(v, sm, i, n, logn, tw);
    if (!on) return;
    T* o0 = out + (size_t)(2 * q) * n;
    T* o1 = o0 + n;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        o0[i + e * nt] = v[e].x;
        o1[i + e * nt] = v[e].y;
    }
    pdl_trigger();
}

// Step 5 for a full complex spectrum (U + i V, S11 + i S12): row y, inverse
// FFT, real part to A, imaginary part to B.  With rows (the list of row
// pairs wanted, as for k_px_inv_real), block b transforms the rows of the
// listed pairs b F / 2 ..., and the blocks past them return at once.
template <typename T, int E, int R0>
__global__ void __launch_bounds__(256) k_px_inv_pair(const cx_t<T>* __restrict__ Q, T* __restrict__ A,
                                                     T* __restrict__ B, int n, int logn,
                                                     const cx_t<T>* __restrict__ tw, const int* __restrict__ rows) {
    pdl_wait();
    using C = cx_t<T>;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nt = n / E, F = blockDim.x / nt;
    const int f = threadIdx.x / nt, i = threadIdx.x - f * nt;
    int y = blockIdx.x * F + f;
    if (rows) {
        const int h = n / 2, cnt = 2 * rows[h];   // rows of the listed pairs
        if ((int)blockIdx.x * F >= cnt) {
            pdl_trigger();
            return;
        }
        y = y < cnt ? 2 * rows[h + 1 + y / 2] + (y & 1) : n;   // n: no row
    }
    const bool on = y < n;
    C* sm = (C*)smraw + (size_t)f * smlen_of(n);
    const C* row = Q + (size_t)(on ? y : 0) * n;
    C v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = row[i + e * nt];
    fft_reg<E, R0, true>(v, sm, i, n, logn, tw);
    if (!on) return;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        A[(size_t)y * n + i + e * nt] = v[e].x;
        B[(size_t)y * n + i + e * nt] = v[e].y;
    }
    pdl_trigger();
}

// Test switch WRC_TEST_POISON_ROWS: the rows of the pairs not listed (flag
// rows[q] clear) of up to two lattices set to NaN after the inverse passes,
// so that a step that read one would show it.
template <typename T>
__global__ void k_poison_rows(T* __restrict__ a, T* __restrict__ b, const int* __restrict__ rows, int n) {
    pdl_wait();
    const long long N = (long long)n * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N;
         e += (long long)gridDim.x * blockDim.x) {
        if (rows[(int)(e / n) >> 1]) continue;
        a[e] = T(NAN);
        if (b) b[e] = T(NAN);
    }
    pdl_trigger();
}

// out[c][r] = in[r][c] for a rows x cols complex matrix, 32 x 32 tiles.
template <typename C>
__global__ void k_transpose(const C* __restrict__ in, C* __restrict__ out, int rows, int cols) {
    pdl_wait();
    __shared__ C tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int gr = r0 + r, gc = c0 + threadIdx.x;
        if (gr < rows && gc < cols) tile[r][threadIdx.x] = in[(size_t)gr * cols + gc];
    }
    __syncthreads();
    for (int c = threadIdx.y; c < 32; c += blockDim.y) {
        const int gc = c0 + c, gr = r0 + threadIdx.x;
        if (gr < rows && gc < cols) out[(size_t)gc * rows + gr] = tile[threadIdx.x][c];
    }
    pdl_trigger();
}

// Twiddles exp(-2 pi i t/n) (t < n) and the symbols, theta = 2 pi t/n, of the
// stencils of order 2P (all evaluated in FP64 and stored as T):
//   2P = 4: sigma(theta) = (30 - 32 cos theta + 2 cos 2 theta)/(12 h^2)
//           = 4 s^2 (3 + s^2)/(3 h^2), s = sin(theta/2), of the second
//           difference, and d(theta) = (8 sin theta - sin 2 theta)/(6 h) of the
//           first difference (its symbol is i d);
//   2P > 4: with the second-derivative stencil (n_0; n_1..n_P)/(d2 h^2) and
//           n_0 = -2 sum n_j, sigma = 4 sum_j n_j sin^2(j theta/2)/(d2 h^2)
//           (no cancellation at small theta), and with the first-derivative
//           stencil (n_1..n_R)/(d1 h), d = 2 sum_j n_j sin(j theta)/(d1 h).
template <typename T>
__global__ void k_fft_init(cx_t<T>* tw, T* sigma, T* dsym, int n, double h, int P) {
    pdl_wait();
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        double sn, cs;
        sincospi(2.0 * t / n, &sn, &cs);
        tw[t] = mk<cx_t<T>>((T)cs, (T)(-sn));
        if (P == 3 || P == 4) {
            double sg = 0.0, ds = 0.0;
            for (int j = 1; j <= P; ++j) {
                const double sj = sinpi((double)j * t / n);
                sg += dd_d2(P, j) * sj * sj;
            }
            for (int j = 1; j <= dd_reach1(P); ++j) ds += dd_d1(P, j) * sinpi(2.0 * j * t / n);
            sigma[t] = (T)(4.0 * sg / (dd_d2den(P) * h * h));
            dsym[t] = (T)(2.0 * ds / (dd_d1den(P) * h));
        } else {
            const double s = sinpi((double)t / n);
            const double s2 = s * s;
            sigma[t] = (T)(4.0 * s2 * (3.0 + s2) * (1.0 / (3.0 * h * h)));
            dsym[t] = (T)((8.0 * sinpi(2.0 * t / n) - sinpi(4.0 * t / n)) * (1.0 / (6.0 * h)));
        }
    }
    pdl_trigger();
}

constexpr int kMaxLattice = 4096;   // WRC_MAX_NJ
constexpr int kMaxSmem = (int)sizeof(double2) * smlen_of(kMaxLattice);

// The kernels of one (E, R0) shape; dynamic shared memory limits are
// process-wide per kernel, so they are set once for the largest lattice.
bool poison_rows() {
    const char* v = std::getenv("WRC_TEST_POISON_ROWS");
    return v && std::atoi(v) != 0;
}

template <typename T, int E, int R0>
struct Shape {
    static int setup() {
        int bad = 0;
        bad |= cudaFuncSetAttribute(k_px_fwd<T, E, R0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
        bad |= cudaFuncSetAttribute(k_py_solve<T, E, R0, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    kMaxSmem);
        bad |= cudaFuncSetAttribute(k_px_inv_real<T, E, R0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
        if constexpr (std::is_same<T, float>::value) {
            bad |= cudaFuncSetAttribute(k_py_solve<T, E, R0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        kMaxSmem);
            bad |= cudaFuncSetAttribute(k_px_inv_pair<T, E, R0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        kMaxSmem);
        }
        return bad;
    }

    static void run(const PoissonPlan& p, const T* Rf, T* psi, cx_t<T>* C1, cx_t<T>* C2, cudaStream_t s, T* U, T* V,
                    cx_t<T>* C3, T* S11, T* S12, cx_t<T>* C4, const int* rows) {
        using C = cx_t<T>;
        const int n = p.n, logn = p.logn, h = n / 2;
        const int nt = n / E, F = nt >= 128 ? 1 : 128 / nt;
        const int thr = F * nt;
        const size_t smem = sizeof(C) * (size_t)F * smlen_of(n);
        const C* tw = (const C*)p.ptw;   // per-pass tables
        const dim3 tb(32, 8);
        const dim3 g_nh((h + 31) / 32, (n + 31) / 32);   // n x h  -> h x n
        const dim3 g_hn((n + 31) / 32, (h + 31) / 32);   // h x n  -> n x h
        const dim3 g_nn((n + 31) / 32, (n + 31) / 32);
        const int b_half = (h + F - 1) / F, b_full = (n + F - 1) / F;
        C* S = C1;         // n x h half spectra
        C* ST = C1 + (size_t)n * h;   // h x n, transposed
        const bool uv = U && V && C3;
        const bool st = uv && S11 && S12 && C4;
        { launch_pdl(k_px_fwd<T, E, R0>, b_half, thr, smem, s, Rf, S, n, logn, tw); note_launch(); }
        { launch_pdl(k_transpose<C>, g_nh, tb, 0, s, S, ST, n, h); note_launch(); }
        const T scale = T(1.0 / ((double)n * (double)n));
        if constexpr (std::is_same<T, float>::value) {
            if (uv) {
                C* QT = C2;                    // n x n
                C* WT = st ? C3 : nullptr;     // n x n
                { launch_pdl(k_py_solve<T, E, R0, true>, b_half, thr, 2 * smem, s, ST, QT, WT, n, logn, tw,
                                                                        (const T*)p.sigma, (const T*)p.dsym,
                                                                        scale, rows ? 0 : 1); note_launch(); }
                // psi: a step (rows given) reads U and V, not psi
                if (!rows) {
                    { launch_pdl(k_transpose<C>, g_hn, tb, 0, s, ST, S, h, n); note_launch(); }
                    { launch_pdl(k_px_inv_real<T, E, R0>, b_half, thr, smem, s, S, psi, n, logn, tw,
                                 (const int*)nullptr); note_launch(); }
                }
                // U + i V: QT (C2) -> a buffer that V (the caller's, possibly in C1) does not overlap
                C* Q = st ? C4 : C3;
                { launch_pdl(k_transpose<C>, g_nn, tb, 0, s, QT, Q, n, n); note_launch(); }
                { launch_pdl(k_px_inv_pair<T, E, R0>, b_full, thr, smem, s, Q, U, V, n, logn, tw, rows); note_launch(); }
                if (rows && poison_rows()) { launch_pdl(k_poison_rows<T>, 1216, 256, 0, s, U, V, rows, n); note_launch(); }
                if (st) {
                    { launch_pdl(k_transpose<C>, g_nn, tb, 0, s, WT, C4, n, n); note_launch(); }
                    { launch_pdl(k_px_inv_pair<T, E, R0>, b_full, thr, smem, s, C4, S11, S12, n, logn, tw, rows); note_launch(); }
                    if (rows && poison_rows()) { launch_pdl(k_poison_rows<T>, 1216, 256, 0, s, S11, S12, rows, n); note_launch(); }
                }
                return;
            }
        }
        { launch_pdl(k_py_solve<T, E, R0, false>, b_half, thr, smem, s, ST, nullptr, nullptr, n, logn, tw,
                                                                 (const T*)p.sigma, (const T*)p.dsym,
                                                                 scale, 1); note_launch(); }
        { launch_pdl(k_transpose<C>, g_hn, tb, 0, s, ST, S, h, n); note_launch(); }
        { launch_pdl(k_px_inv_real<T, E, R0>, b_half, thr, smem, s, S, psi, n, logn, tw, rows); note_launch(); }
        if (rows && poison_rows()) { launch_pdl(k_poison_rows<T>, 1216, 256, 0, s, psi, (T*)nullptr, rows, n); note_launch(); }
        (void)C2;
    }
};

template <typename T>
int setup_all() {
    return Shape<T, 8, 1>::setup() | Shape<T, 16, 1>::setup() | Shape<T, 16, 2>::setup() |
           Shape<T, 16, 4>::setup() | Shape<T, 16, 8>::setup();
}

template <typename T>
int plan_init_t(PoissonPlan& p, const Geom& g, cudaStream_t s) {
    if (cudaMalloc(&p.tw, sizeof(cx_t<T>) * p.n) != cudaSuccess) return -1;
    if (cudaMalloc(&p.ptw, sizeof(cx_t<T>) * 2 * p.n) != cudaSuccess) return -1;
    if (cudaMalloc(&p.sigma, sizeof(T) * p.n) != cudaSuccess) return -1;
    if (cudaMalloc(&p.dsym, sizeof(T) * p.n) != cudaSuccess) return -1;
    if (setup_all<T>() != 0) return -2;
    { launch_pdl(k_fft_init<T>, (p.n + 255) / 256, 256, 0, s, (cx_t<T>*)p.tw, (T*)p.sigma, (T*)p.dsym, p.n,
                                                       g.h, g.P); note_launch(); }
    const int E = p.logn < 4 ? 8 : 16;
    const int R0 = p.logn < 4 ? 1 : 1 << (p.logn % 4);
    { k_fft_pass_tables<cx_t<T>><<<(p.n + 255) / 256, 256, 0, s>>>((const cx_t<T>*)p.tw, (cx_t<T>*)p.ptw, p.n,
                                                                    p.logn, E, R0); note_launch(); }
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace

int poisson_plan_init(PoissonPlan& p, const Geom& g, bool fp32, cudaStream_t s) {
    p.n = g.NJ;
    p.logn = g.L;
    p.fp32 = fp32;
    if (p.n < 8 || p.n > kMaxLattice || (p.n & (p.n - 1))) return -4;
    return fp32 ? plan_init_t<float>(p, g, s) : plan_init_t<double>(p, g, s);
}

void poisson_plan_free(PoissonPlan& p) {
    if (p.tw) cudaFree(p.tw);
    if (p.ptw) cudaFree(p.ptw);
    p.ptw = nullptr;
    if (p.sigma) cudaFree(p.sigma);
    if (p.dsym) cudaFree(p.dsym);
    p.tw = nullptr;
    p.sigma = nullptr;
    p.dsym = nullptr;
}

template <typename T>
void launch_poisson(const PoissonPlan& p, const T* R, T* psi, void* C1v, void* C2v, const Geom& g, cudaStream_t s,
                    T* U, T* V, void* C3v, T* S11, T* S12, void* C4v, const int* rows) {
    using C = cx_t<T>;
    C* C1 = (C*)C1v;
    C* C2 = (C*)C2v;
    C* C3 = (C*)C3v;
    C* C4 = (C*)C4v;
    const int logn = p.logn;
    if (logn < 4) Shape<T, 8, 1>::run(p, R, psi, C1, C2, s, U, V, C3, S11, S12, C4, rows);
    else if (logn % 4 == 0) Shape<T, 16, 1>::run(p, R, psi, C1, C2, s, U, V, C3, S11, S12, C4, rows);
    else if (logn % 4 == 1) Shape<T, 16, 2>::run(p, R, psi, C1, C2, s, U, V, C3, S11, S12, C4, rows);
    else if (logn % 4 == 2) Shape<T, 16, 4>::run(p, R, psi, C1, C2, s, U, V, C3, S11, S12, C4, rows);
    else Shape<T, 16, 8>::run(p, R, psi, C1, C2, s, U, V, C3, S11, S12, C4, rows);
    (void)g;
}

template void launch_poisson<double>(const PoissonPlan&, const double*, double*, void*, void*, const Geom&,
                                     cudaStream_t, double*, double*, void*, double*, double*, void*, const int*);
template void launch_poisson<float>(const PoissonPlan&, const float*, float*, void*, void*, const Geom&, cudaStream_t,
                                    float*, float*, void*, float*, float*, void*, const int*);

}  // namespace wrc
