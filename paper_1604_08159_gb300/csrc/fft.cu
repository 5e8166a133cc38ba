// Streamfunction solve on the periodic finest lattice: psi = L_h^{-1}(-(R - mean R))
// with L_h the 4th-order collocation Laplacian, diagonalised by the 2-D DFT.
// Five passes: real rows -> FFT along x, transpose, FFT along y / divide by the
// symbol / inverse FFT along y (one CTA per row, all in shared memory),
// transpose back, inverse FFT along x -> real part.  Radix-2 FFTs run in
// shared memory, one CTA per row of up to 4096 complex values.
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
__device__ __forceinline__ C cmul(C a, C b) {
    return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ int bitrev(int t, int logn) { return (int)(__brev((unsigned)t) >> (32 - logn)); }

// In-place radix-2 decimation-in-time FFT in shared memory: input in
// bit-reversed order, output in natural order.  tw[t] = exp(-2 pi i t/n).
template <typename C>
__device__ void fft_smem(C* sm, int n, int logn, const C* __restrict__ tw, bool inverse) {
    for (int st = 1; st <= logn; ++st) {
        const int half = 1 << (st - 1);
        const int tstride = n >> st;
        for (int b = threadIdx.x; b < (n >> 1); b += blockDim.x) {
            const int pos = b & (half - 1);
            const int i0 = ((b >> (st - 1)) << st) + pos;
            const int i1 = i0 + half;
            C w = tw[pos * tstride];
            if (inverse) w.y = -w.y;
            const C u = sm[i0];
            const C v = cmul(sm[i1], w);
            sm[i0] = mk<C>(u.x + v.x, u.y + v.y);
            sm[i1] = mk<C>(u.x - v.x, u.y - v.y);
        }
        __syncthreads();
    }
}

// Twiddles exp(-2 pi i t/n) and the symbol
// sigma(theta) = (30 - 32 cos theta + 2 cos 2 theta)/(12 h^2) = 4 s^2 (3 + s^2)/(3 h^2),
// s = sin(theta/2), theta = 2 pi t/n, both evaluated in FP64 and stored as T.
template <typename T>
__global__ void k_fft_init(cx_t<T>* tw, T* sigma, T* dsym, int n, double inv3h2, double inv6h) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        double sn, cs;
        if (t < n / 2) {
            sincospi(2.0 * t / n, &sn, &cs);
            tw[t] = mk<cx_t<T>>((T)cs, (T)(-sn));
        }
        const double s = sinpi((double)t / n);
        const double s2 = s * s;
        sigma[t] = (T)(4.0 * s2 * (3.0 + s2) * inv3h2);
        // symbol of the 4th-order first derivative: i (8 sin theta - sin 2 theta) / (6 h)
        dsym[t] = (T)((8.0 * sinpi(2.0 * t / n) - sinpi(4.0 * t / n)) * inv6h);
    }
}

// Pass 1: each CTA transforms one real row along x.
template <typename T>
__global__ void k_fft_x_fwd_real(const T* __restrict__ R, cx_t<T>* __restrict__ C, int n, int logn,
                                 const cx_t<T>* __restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smraw[];
    cx_t<T>* sm = (cx_t<T>*)smraw;
    const T* row = R + (size_t)blockIdx.x * n;
    for (int t = threadIdx.x; t < n; t += blockDim.x) sm[bitrev(t, logn)] = mk<cx_t<T>>(row[t], T(0));
    __syncthreads();
    fft_smem(sm, n, logn, tw, false);
    cx_t<T>* out = C + (size_t)blockIdx.x * n;
    for (int t = threadIdx.x; t < n; t += blockDim.x) out[t] = sm[t];
}

// Pass 3: row kx of the transposed spectrum: FFT along y, divide by the
// symbol (mode (0,0) set to 0, 1/n^2 normalisation folded in), inverse FFT.
// With Q given, also the spectrum of U + i V, U = D_y psi, V = -D_x psi
// (D the 4th-order first-derivative stencil, symbol i d(theta)):
// (d(theta_x) + i d(theta_y)) psi_hat, inverse-transformed along y into Q.
// With W given, also the spectrum of S11 + i S12, S11 = D_x D_y psi and
// S12 = (D_yy - D_xx) psi / 2: (-d_x d_y + i (sigma_x - sigma_y) / 2) psi_hat.
template <typename T>
__global__ void k_fft_y_solve(cx_t<T>* __restrict__ C, cx_t<T>* __restrict__ Q, cx_t<T>* __restrict__ W, int n,
                              int logn, const cx_t<T>* __restrict__ tw, const T* __restrict__ sigma,
                              const T* __restrict__ dsym, T scale) {
    extern __shared__ __align__(16) unsigned char smraw[];
    cx_t<T>* sm = (cx_t<T>*)smraw;
    cx_t<T>* sq = sm + n;
    cx_t<T>* sw = sq + n;
    cx_t<T>* row = C + (size_t)blockIdx.x * n;
    for (int t = threadIdx.x; t < n; t += blockDim.x) sm[bitrev(t, logn)] = row[t];
    __syncthreads();
    fft_smem(sm, n, logn, tw, false);
    const T sx = sigma[blockIdx.x];
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const T den = sx + sigma[t];
        const T f = (blockIdx.x == 0 && t == 0) ? T(0) : scale / den;
        sm[t] = mk<cx_t<T>>(sm[t].x * f, sm[t].y * f);
        if (Q) sq[t] = cmul(sm[t], mk<cx_t<T>>(dsym[blockIdx.x], dsym[t]));
        if (W) sw[t] = cmul(sm[t], mk<cx_t<T>>(-dsym[blockIdx.x] * dsym[t], T(0.5) * (sx - sigma[t])));
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int r = bitrev(t, logn);
        if (t < r) {
            const cx_t<T> a = sm[t];
            sm[t] = sm[r];
            sm[r] = a;
            if (Q) {
                const cx_t<T> b = sq[t];
                sq[t] = sq[r];
                sq[r] = b;
            }
            if (W) {
                const cx_t<T> c = sw[t];
                sw[t] = sw[r];
                sw[r] = c;
            }
        }
    }
    __syncthreads();
    fft_smem(sm, n, logn, tw, true);
    for (int t = threadIdx.x; t < n; t += blockDim.x) row[t] = sm[t];
    if (Q) {
        fft_smem(sq, n, logn, tw, true);
        cx_t<T>* qrow = Q + (size_t)blockIdx.x * n;
        for (int t = threadIdx.x; t < n; t += blockDim.x) qrow[t] = sq[t];
    }
    if (W) {
        fft_smem(sw, n, logn, tw, true);
        cx_t<T>* wrow = W + (size_t)blockIdx.x * n;
        for (int t = threadIdx.x; t < n; t += blockDim.x) wrow[t] = sw[t];
    }
}

// Pass 5: inverse FFT along x, real part.
template <typename T>
__global__ void k_fft_x_inv_real(const cx_t<T>* __restrict__ C, T* __restrict__ psi, int n, int logn,
                                 const cx_t<T>* __restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smraw[];
    cx_t<T>* sm = (cx_t<T>*)smraw;
    const cx_t<T>* row = C + (size_t)blockIdx.x * n;
    for (int t = threadIdx.x; t < n; t += blockDim.x) sm[bitrev(t, logn)] = row[t];
    __syncthreads();
    fft_smem(sm, n, logn, tw, true);
    T* out = psi + (size_t)blockIdx.x * n;
    for (int t = threadIdx.x; t < n; t += blockDim.x) out[t] = sm[t].x;
}

// Pass 5 for U + i V: inverse FFT along x, real part to U, imaginary to V.
template <typename T>
__global__ void k_fft_x_inv_pair(const cx_t<T>* __restrict__ C, T* __restrict__ U, T* __restrict__ V, int n,
                                 int logn, const cx_t<T>* __restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smraw[];
    cx_t<T>* sm = (cx_t<T>*)smraw;
    const cx_t<T>* row = C + (size_t)blockIdx.x * n;
    for (int t = threadIdx.x; t < n; t += blockDim.x) sm[bitrev(t, logn)] = row[t];
    __syncthreads();
    fft_smem(sm, n, logn, tw, true);
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        U[(size_t)blockIdx.x * n + t] = sm[t].x;
        V[(size_t)blockIdx.x * n + t] = sm[t].y;
    }
}

// out[c][r] = in[r][c] for an n x n complex matrix, 32 x 32 tiles.
template <typename C>
__global__ void k_transpose(const C* __restrict__ in, C* __restrict__ out, int n) {
    __shared__ C tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int gy = by + r, gx = bx + threadIdx.x;
        if (gy < n && gx < n) tile[r][threadIdx.x] = in[(size_t)gy * n + gx];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int gy = bx + r, gx = by + threadIdx.x;
        if (gy < n && gx < n) out[(size_t)gy * n + gx] = tile[threadIdx.x][r];
    }
}

constexpr int kMaxLattice = 4096;   // WRC_MAX_NJ

template <typename T>
int plan_init_t(PoissonPlan& p, const Geom& g, cudaStream_t s) {
    if (cudaMalloc(&p.tw, sizeof(cx_t<T>) * (p.n / 2 > 0 ? p.n / 2 : 1)) != cudaSuccess) return -1;
    if (cudaMalloc(&p.sigma, sizeof(T) * p.n) != cudaSuccess) return -1;
    if (cudaMalloc(&p.dsym, sizeof(T) * p.n) != cudaSuccess) return -1;
    // The dynamic shared-memory limit is a per-kernel, process-wide attribute:
    // set it for the largest lattice, so runs of different sizes coexist.
    const int smem = (int)(sizeof(cx_t<T>) * kMaxLattice);
    if (cudaFuncSetAttribute(k_fft_x_fwd_real<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
        cudaFuncSetAttribute(k_fft_y_solve<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 3 * smem) != cudaSuccess ||
        cudaFuncSetAttribute(k_fft_x_inv_real<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
        cudaFuncSetAttribute(k_fft_x_inv_pair<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return -2;
    { k_fft_init<T><<<(p.n + 255) / 256, 256, 0, s>>>((cx_t<T>*)p.tw, (T*)p.sigma, (T*)p.dsym, p.n,
                                                       1.0 / (3.0 * g.h * g.h), 1.0 / (6.0 * g.h)); note_launch(); }
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace

int poisson_plan_init(PoissonPlan& p, const Geom& g, bool fp32, cudaStream_t s) {
    p.n = g.NJ;
    p.logn = g.L;
    p.fp32 = fp32;
    return fp32 ? plan_init_t<float>(p, g, s) : plan_init_t<double>(p, g, s);
}

void poisson_plan_free(PoissonPlan& p) {
    if (p.tw) cudaFree(p.tw);
    if (p.sigma) cudaFree(p.sigma);
    if (p.dsym) cudaFree(p.dsym);
    p.tw = nullptr;
    p.sigma = nullptr;
    p.dsym = nullptr;
}

template <typename T>
void launch_poisson(const PoissonPlan& p, const T* R, T* psi, void* C1v, void* C2v, const Geom& g, cudaStream_t s,
                    T* U, T* V, void* C3v, T* S11, T* S12, void* C4v) {
    using C = cx_t<T>;
    C* C1 = (C*)C1v;
    C* C2 = (C*)C2v;
    C* C3 = (C*)C3v;
    C* C4 = (C*)C4v;
    const bool uv = U && V && C3;
    const bool st = uv && S11 && S12 && C4;
    const int n = p.n;
    const size_t smem = sizeof(C) * n;
    const int thr = n >= 512 ? 256 : (n / 2 >= 32 ? n / 2 : 32);
    const dim3 tgrid((n + 31) / 32, (n + 31) / 32), tblk(32, 8);
    const C* tw = (const C*)p.tw;
    { k_fft_x_fwd_real<T><<<n, thr, smem, s>>>(R, C1, n, p.logn, tw); note_launch(); }
    { k_transpose<C><<<tgrid, tblk, 0, s>>>(C1, C2, n); note_launch(); }
    { k_fft_y_solve<T><<<n, thr, (1 + (uv ? 1 : 0) + (st ? 1 : 0)) * smem, s>>>(
          C2, uv ? C1 : nullptr, st ? C4 : nullptr, n, p.logn, tw, (const T*)p.sigma, (const T*)p.dsym,
          T(1.0 / ((double)n * (double)n))); note_launch(); }
    if (uv) {
        { k_transpose<C><<<tgrid, tblk, 0, s>>>(C2, C3, n); note_launch(); }
        { k_fft_x_inv_real<T><<<n, thr, smem, s>>>(C3, psi, n, p.logn, tw); note_launch(); }
        { k_transpose<C><<<tgrid, tblk, 0, s>>>(C1, C2, n); note_launch(); }
        { k_fft_x_inv_pair<T><<<n, thr, smem, s>>>(C2, U, V, n, p.logn, tw); note_launch(); }
        if (st) {
            { k_transpose<C><<<tgrid, tblk, 0, s>>>(C4, C3, n); note_launch(); }
            { k_fft_x_inv_pair<T><<<n, thr, smem, s>>>(C3, S11, S12, n, p.logn, tw); note_launch(); }
        }
    } else {
        { k_transpose<C><<<tgrid, tblk, 0, s>>>(C2, C1, n); note_launch(); }
        { k_fft_x_inv_real<T><<<n, thr, smem, s>>>(C1, psi, n, p.logn, tw); note_launch(); }
    }
    (void)g;
}

template void launch_poisson<double>(const PoissonPlan&, const double*, double*, void*, void*, const Geom&,
                                     cudaStream_t, double*, double*, void*, double*, double*, void*);
template void launch_poisson<float>(const PoissonPlan&, const float*, float*, void*, void*, const Geom&, cudaStream_t,
                                    float*, float*, void*, float*, float*, void*);

}  // namespace wrc
