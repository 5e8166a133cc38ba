// Streamfunction solve on the periodic finest lattice: psi = L_h^{-1}(-(R - mean R))
// with L_h the 4th-order collocation Laplacian, diagonalised by the 2-D DFT.
// Five passes: real rows -> FFT along x, transpose, FFT along y / divide by the
// symbol / inverse FFT along y (one CTA per row, all in shared memory),
// transpose back, inverse FFT along x -> real part.  Radix-2 FFTs run in
// shared memory, one CTA per row of up to 4096 complex values.
#include "kernels.h"

namespace wrc {

namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ int bitrev(int t, int logn) { return (int)(__brev((unsigned)t) >> (32 - logn)); }

// In-place radix-2 decimation-in-time FFT in shared memory: input in
// bit-reversed order, output in natural order.  tw[t] = exp(-2 pi i t/n).
__device__ void fft_smem(double2* sm, int n, int logn, const double2* __restrict__ tw, bool inverse) {
    for (int st = 1; st <= logn; ++st) {
        const int half = 1 << (st - 1);
        const int tstride = n >> st;
        for (int b = threadIdx.x; b < (n >> 1); b += blockDim.x) {
            const int pos = b & (half - 1);
            const int i0 = ((b >> (st - 1)) << st) + pos;
            const int i1 = i0 + half;
            double2 w = __ldg(&tw[pos * tstride]);
            if (inverse) w.y = -w.y;
            const double2 u = sm[i0];
            const double2 v = cmul(sm[i1], w);
            sm[i0] = make_double2(u.x + v.x, u.y + v.y);
            sm[i1] = make_double2(u.x - v.x, u.y - v.y);
        }
        __syncthreads();
    }
}

__global__ void k_fft_init(double2* tw, double* sigma, int n, double inv3h2) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        double sn, cs;
        if (t < n / 2) {
            sincospi(2.0 * t / n, &sn, &cs);
            tw[t] = make_double2(cs, -sn);
        }
        // sigma(theta) = (30 - 32 cos theta + 2 cos 2 theta)/(12 h^2)
        //             = 4 s^2 (3 + s^2) / (3 h^2),  s = sin(theta/2), theta = 2 pi t/n
        const double s = sinpi((double)t / n);
        const double s2 = s * s;
        sigma[t] = 4.0 * s2 * (3.0 + s2) * inv3h2;
    }
}

// Pass 1: each CTA transforms one real row along x.
__global__ void k_fft_x_fwd_real(const double* __restrict__ R, double2* __restrict__ C, int n, int logn,
                                 const double2* __restrict__ tw) {
    extern __shared__ double2 sm[];
    const double* row = R + (size_t)blockIdx.x * n;
    for (int t = threadIdx.x; t < n; t += blockDim.x) sm[bitrev(t, logn)] = make_double2(row[t], 0.0);
    __syncthreads();
    fft_smem(sm, n, logn, tw, false);
    double2* out = C + (size_t)blockIdx.x * n;
    for (int t = threadIdx.x; t < n; t += blockDim.x) out[t] = sm[t];
}

// Pass 3: row kx of the transposed spectrum: FFT along y, divide by the
// symbol (mode (0,0) set to 0, 1/n^2 normalisation folded in), inverse FFT.
__global__ void k_fft_y_solve(double2* __restrict__ C, int n, int logn, const double2* __restrict__ tw,
                              const double* __restrict__ sigma, double scale) {
    extern __shared__ double2 sm[];
    double2* row = C + (size_t)blockIdx.x * n;
    for (int t = threadIdx.x; t < n; t += blockDim.x) sm[bitrev(t, logn)] = row[t];
    __syncthreads();
    fft_smem(sm, n, logn, tw, false);
    const double sx = sigma[blockIdx.x];
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const double den = sx + sigma[t];
        const double f = (blockIdx.x == 0 && t == 0) ? 0.0 : scale / den;
        sm[t] = make_double2(sm[t].x * f, sm[t].y * f);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int r = bitrev(t, logn);
        if (t < r) {
            const double2 a = sm[t];
            sm[t] = sm[r];
            sm[r] = a;
        }
    }
    __syncthreads();
    fft_smem(sm, n, logn, tw, true);
    for (int t = threadIdx.x; t < n; t += blockDim.x) row[t] = sm[t];
}

// Pass 5: inverse FFT along x, real part.
__global__ void k_fft_x_inv_real(const double2* __restrict__ C, double* __restrict__ psi, int n, int logn,
                                 const double2* __restrict__ tw) {
    extern __shared__ double2 sm[];
    const double2* row = C + (size_t)blockIdx.x * n;
    for (int t = threadIdx.x; t < n; t += blockDim.x) sm[bitrev(t, logn)] = row[t];
    __syncthreads();
    fft_smem(sm, n, logn, tw, true);
    double* out = psi + (size_t)blockIdx.x * n;
    for (int t = threadIdx.x; t < n; t += blockDim.x) out[t] = sm[t].x;
}

// out[c][r] = in[r][c] for an n x n complex matrix, 32 x 32 tiles.
__global__ void k_transpose(const double2* __restrict__ in, double2* __restrict__ out, int n) {
    __shared__ double2 tile[32][33];
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

}  // namespace

int poisson_plan_init(PoissonPlan& p, const Geom& g, cudaStream_t s) {
    p.n = g.NJ;
    p.logn = g.L;
    if (cudaMalloc(&p.tw, sizeof(double2) * (p.n / 2 > 0 ? p.n / 2 : 1)) != cudaSuccess) return -1;
    if (cudaMalloc(&p.sigma, sizeof(double) * p.n) != cudaSuccess) return -1;
    const size_t smem = sizeof(double2) * p.n;
    if (cudaFuncSetAttribute(k_fft_x_fwd_real, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaFuncSetAttribute(k_fft_y_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaFuncSetAttribute(k_fft_x_inv_real, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return -2;
    { k_fft_init<<<(p.n + 255) / 256, 256, 0, s>>>(p.tw, p.sigma, p.n, 1.0 / (3.0 * g.h * g.h)); note_launch(); }
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

void poisson_plan_free(PoissonPlan& p) {
    if (p.tw) cudaFree(p.tw);
    if (p.sigma) cudaFree(p.sigma);
    p.tw = nullptr;
    p.sigma = nullptr;
}

void launch_poisson(const PoissonPlan& p, const double* R, double* psi, double2* C1, double2* C2, const Geom& g,
                    cudaStream_t s) {
    const int n = p.n;
    const size_t smem = sizeof(double2) * n;
    const int thr = n >= 512 ? 256 : (n / 2 >= 32 ? n / 2 : 32);
    const dim3 tgrid((n + 31) / 32, (n + 31) / 32), tblk(32, 8);
    { k_fft_x_fwd_real<<<n, thr, smem, s>>>(R, C1, n, p.logn, p.tw); note_launch(); }
    { k_transpose<<<tgrid, tblk, 0, s>>>(C1, C2, n); note_launch(); }
    { k_fft_y_solve<<<n, thr, smem, s>>>(C2, n, p.logn, p.tw, p.sigma, 1.0 / ((double)n * (double)n)); note_launch(); }
    { k_transpose<<<tgrid, tblk, 0, s>>>(C2, C1, n); note_launch(); }
    { k_fft_x_inv_real<<<n, thr, smem, s>>>(C1, psi, n, p.logn, p.tw); note_launch(); }
    (void)g;
}

}  // namespace wrc
