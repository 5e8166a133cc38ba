// Krylov projection of the time step (Sec. 2.1: the discrete system projected
// onto a Krylov subspace): Arnoldi with classical Gram-Schmidt applied twice,
// FP64 inner products with deterministic two-stage reductions, the exponential
// of the small augmented Hessenberg matrix, and the update
// omega += dt * beta * V_k phi_1(dt H_k) e_1.
#include "kernels.h"

namespace wrc {

namespace {

constexpr int kOut = 33;   // reduction outputs per pass: up to 32 dots + a squared norm

// One pass over the n active entries of w with the first nv basis vectors:
//   if coef:   w <- w - sum_i coef[i] v_i           (written back)
//   out[t] = <v_t, w> for t < ndots, out[ndots] = <w, w>    (FP64 sums)
// Each block writes its partial sums; the last block to finish adds them in
// block order, so the result does not depend on scheduling.
template <typename T, int NV>
__global__ void __launch_bounds__(kThreads) k_gs_pass(const T* __restrict__ basis, long long ld, long long n, int nv,
                                                      int ndots, T* __restrict__ w, const double* __restrict__ coef,
                                                      double* __restrict__ out, double* __restrict__ partials,
                                                      unsigned* __restrict__ counter, const int* __restrict__ kstop,
                                                      int jstep) {
    if (kstop && jstep >= *kstop) return;
    __shared__ double s_coef[NV];
    __shared__ double s_red[kThreads / 32][NV + 1];
    __shared__ bool s_last;
    if (coef)
        for (int t = threadIdx.x; t < nv; t += blockDim.x) s_coef[t] = coef[t];
    __syncthreads();
    double acc[NV + 1];
#pragma unroll
    for (int t = 0; t <= NV; ++t) acc[t] = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        double x = (double)w[e];
        if (coef) {
#pragma unroll
            for (int t = 0; t < NV; ++t)
                if (t < nv) x -= (double)basis[t * ld + e] * s_coef[t];
            w[e] = (T)x;
        }
#pragma unroll
        for (int t = 0; t < NV; ++t)
            if (t < ndots) acc[t] += (double)basis[t * ld + e] * x;
        acc[NV] += x * x;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int t = 0; t <= NV; ++t) {
        if (t < ndots || t == NV) {
            double v = acc[t];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) s_red[wid][t] = v;
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t <= ndots; t += blockDim.x) {
        const int src = t < ndots ? t : NV;
        double v = 0.0;
        for (int q = 0; q < kThreads / 32; ++q) v += s_red[q][src];
        partials[(size_t)blockIdx.x * kOut + t] = v;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (s_last) {
        __threadfence();
        for (int t = threadIdx.x; t <= ndots; t += blockDim.x) {
            double v = 0.0;
            for (unsigned b = 0; b < gridDim.x; ++b) v += __ldcg(&partials[(size_t)b * kOut + t]);
            out[t] = v;
        }
        if (threadIdx.x == 0) *counter = 0;
    }
}

// beta = |b| from the preceding norm pass (out[0] = <b, b>); the Krylov
// dimension is m unless b vanishes or is not finite.
__global__ void k_krylov_start(KrylovDev K, int m) {
    const double nb = K.o1[0];
    const double beta = sqrt(nb);
    K.beta[0] = beta;
    if (!isfinite(beta)) {
        K.flags[0] |= 1;
        K.kstop[0] = 0;
    } else {
        K.kstop[0] = beta > 0.0 ? m : 0;
    }
}

// Column j of H from the two Gram-Schmidt passes (o1: first-pass dots and
// |A v_j|^2; o2: second-pass dots; o3: |w|^2 after both).  Happy breakdown
// when h_{j+1,j} <= tol |A v_j|.
__global__ void k_arnoldi_col(KrylovDev K, int j, int m, double tol) {
    if (j >= K.kstop[0]) return;
    bool bad = false;
    for (int i = 0; i <= j; ++i) {
        const double hij = K.o1[i] + K.o2[i];
        K.H[(size_t)i * m + j] = hij;
        bad |= !isfinite(hij);
    }
    const double wn = sqrt(K.o1[j + 1]);
    const double hn = sqrt(K.o3[0]);
    K.H[(size_t)(j + 1) * m + j] = hn;
    if (bad || !isfinite(hn)) {
        K.flags[0] |= 1;
        K.kstop[0] = j + 1;
    } else if (hn <= tol * wn) {
        K.kstop[0] = j + 1;
    }
}

// v_j = w / h_{j,j-1} (v_0 = b / beta) into the basis and into the lattice
// array read by the next operator application.
template <typename T>
__global__ void k_normalize_scatter(KrylovDev K, const uint32_t* __restrict__ meta, long long n, int j, int m,
                                    T* __restrict__ Fq) {
    if (j >= K.kstop[0]) return;
    const double inv = 1.0 / (j == 0 ? K.beta[0] : K.H[(size_t)j * m + (j - 1)]);
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x) {
        const T v = (T)((double)((const T*)K.w)[a] * inv);
        ((T*)K.basis)[(size_t)j * K.ld + a] = v;
        Fq[meta_pos(meta[a])] = v;
    }
}

// ---- exponential of the (k+1) x (k+1) augmented matrix ----------------------
// Pade [13/13] approximant with scaling and squaring (Higham, SIAM J. Matrix
// Anal. Appl. 26 (2005) 1179-1193): theta_13 from that paper; the Pade
// coefficients are generated from their closed form
// c_j = (2m - j)! m! / ((2m)! j! (m - j)!), m = 13, normalised to c_0 = 1.

constexpr int kE = 32;           // padded matrix dimension (k + 1 <= 32)
constexpr int kES = kE * kE;

__device__ void mm(const double* A, const double* B, double* C, int N) {
    for (int t = threadIdx.x; t < N * N; t += blockDim.x) {
        const int r = t / N, c = t % N;
        double s = 0.0;
        for (int q = 0; q < N; ++q) s += A[r * kE + q] * B[q * kE + c];
        C[r * kE + c] = s;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(256) k_phi1(KrylovDev K, int m, double dt) {
    extern __shared__ double sm[];
    double* A = sm;
    double* A2 = A + kES;
    double* A4 = A2 + kES;
    double* A6 = A4 + kES;
    double* U = A6 + kES;
    double* V = U + kES;
    double* T1 = V + kES;
    __shared__ double c[14];
    __shared__ int s_s;
    __shared__ int s_piv;
    const int k = K.kstop[0];
    if (k <= 0) {
        for (int t = threadIdx.x; t < m; t += blockDim.x) K.y[t] = 0.0;
        return;
    }
    const int N = k + 1;
    for (int t = threadIdx.x; t < kES; t += blockDim.x) {
        const int r = t / kE, q = t % kE;
        double v = 0.0;
        if (r < k && q < k) v = dt * K.H[(size_t)r * m + q];
        if (r == 0 && q == k) v = 1.0;
        A[t] = v;
    }
    if (threadIdx.x == 0) {
        c[0] = 1.0;
        for (int j = 1; j <= 13; ++j) c[j] = c[j - 1] * (double)(13 - j + 1) / ((double)j * (double)(26 - j + 1));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double nrm = 0.0;
        for (int q = 0; q < N; ++q) {
            double s = 0.0;
            for (int r = 0; r < N; ++r) s += fabs(A[r * kE + q]);
            nrm = fmax(nrm, s);
        }
        const double theta13 = 5.371920351148152;
        int s = 0;
        if (nrm > theta13) s = (int)ceil(log2(nrm / theta13));
        s_s = s;
    }
    __syncthreads();
    const int s = s_s;
    if (s > 0) {
        const double f = ldexp(1.0, -s);
        for (int t = threadIdx.x; t < kES; t += blockDim.x) A[t] *= f;
        __syncthreads();
    }
    mm(A, A, A2, N);
    mm(A2, A2, A4, N);
    mm(A4, A2, A6, N);
    // U = A [A6 (c13 A6 + c11 A4 + c9 A2) + c7 A6 + c5 A4 + c3 A2 + c1 I]
    // V =    A6 (c12 A6 + c10 A4 + c8 A2) + c6 A6 + c4 A4 + c2 A2 + c0 I
    for (int t = threadIdx.x; t < kES; t += blockDim.x)
        T1[t] = c[13] * A6[t] + c[11] * A4[t] + c[9] * A2[t];
    __syncthreads();
    mm(A6, T1, U, N);
    for (int t = threadIdx.x; t < kES; t += blockDim.x) {
        const int r = t / kE, q = t % kE;
        U[t] += c[7] * A6[t] + c[5] * A4[t] + c[3] * A2[t] + (r == q ? c[1] : 0.0);
        T1[t] = c[12] * A6[t] + c[10] * A4[t] + c[8] * A2[t];
    }
    __syncthreads();
    mm(A6, T1, V, N);
    for (int t = threadIdx.x; t < kES; t += blockDim.x) {
        const int r = t / kE, q = t % kE;
        V[t] += c[6] * A6[t] + c[4] * A4[t] + c[2] * A2[t] + (r == q ? c[0] : 0.0);
    }
    __syncthreads();
    mm(A, U, T1, N);            // T1 = U
    // P = V + U (right-hand sides, into A2), Q = V - U (matrix, into A4)
    for (int t = threadIdx.x; t < kES; t += blockDim.x) {
        A2[t] = V[t] + T1[t];
        A4[t] = V[t] - T1[t];
    }
    __syncthreads();
    // Gaussian elimination with partial pivoting: Q X = P, X into A2.
    for (int col = 0; col < N; ++col) {
        if (threadIdx.x == 0) {
            int piv = col;
            double best = fabs(A4[col * kE + col]);
            for (int r = col + 1; r < N; ++r) {
                const double v = fabs(A4[r * kE + col]);
                if (v > best) { best = v; piv = r; }
            }
            s_piv = piv;
        }
        __syncthreads();
        const int piv = s_piv;
        if (piv != col) {
            for (int q = threadIdx.x; q < N; q += blockDim.x) {
                double a = A4[col * kE + q]; A4[col * kE + q] = A4[piv * kE + q]; A4[piv * kE + q] = a;
                double b = A2[col * kE + q]; A2[col * kE + q] = A2[piv * kE + q]; A2[piv * kE + q] = b;
            }
        }
        __syncthreads();
        const double d = A4[col * kE + col];
        for (int t = threadIdx.x; t < (N - col - 1) * N; t += blockDim.x) {
            const int r = col + 1 + t / N, q = t % N;
            const double f = A4[r * kE + col] / d;
            A2[r * kE + q] -= f * A2[col * kE + q];
            if (q > col) A4[r * kE + q] -= f * A4[col * kE + q];
        }
        __syncthreads();
        for (int r = col + 1 + threadIdx.x; r < N; r += blockDim.x) A4[r * kE + col] = 0.0;
        __syncthreads();
    }
    for (int col = N - 1; col >= 0; --col) {
        for (int q = threadIdx.x; q < N; q += blockDim.x) A2[col * kE + q] /= A4[col * kE + col];
        __syncthreads();
        for (int t = threadIdx.x; t < col * N; t += blockDim.x) {
            const int r = t / N, q = t % N;
            A2[r * kE + q] -= A4[r * kE + col] * A2[col * kE + q];
        }
        __syncthreads();
    }
    // squaring
    double* X = A2;
    double* Y = T1;
    for (int q = 0; q < s; ++q) {
        mm(X, X, Y, N);
        double* tmp = X; X = Y; Y = tmp;
    }
    for (int t = threadIdx.x; t < m; t += blockDim.x) K.y[t] = t < k ? X[t * kE + k] : 0.0;
}

// omega += dt beta sum_i y_i v_i, also written into the lattice array L.
template <typename T>
__global__ void k_update(KrylovDev K, const uint32_t* __restrict__ meta, long long n, double dt, T* __restrict__ omega,
                         T* __restrict__ L) {
    __shared__ double s_c[kE];
    const int k = K.kstop[0];
    for (int t = threadIdx.x; t < k; t += blockDim.x) s_c[t] = dt * K.beta[0] * K.y[t];
    __syncthreads();
    const T* basis = (const T*)K.basis;
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x) {
        double inc = 0.0;
        for (int t = 0; t < k; ++t) inc += s_c[t] * (double)basis[(size_t)t * K.ld + a];
        const T x = (T)((double)omega[a] + inc);
        omega[a] = x;
        L[meta_pos(meta[a])] = x;
    }
}

int gs_blocks(long long n) {
    long long b = (n + kThreads - 1) / kThreads;
    if (b < 1) b = 1;
    if (b > 152 * 4) b = 152 * 4;
    return (int)b;
}

}  // namespace

template <typename T>
void launch_gs_pass(const KrylovDev& K, long long n, int nv, int ndots, const double* coef, double* out,
                    const int* kstop, int jstep, cudaStream_t s) {
    const int nb = gs_blocks(n);
    const T* basis = (const T*)K.basis;
    T* w = (T*)K.w;
    const int need = nv > ndots ? nv : ndots;
    if (need <= 8)
        { k_gs_pass<T, 8><<<nb, kThreads, 0, s>>>(basis, K.ld, n, nv, ndots, w, coef, out, K.partials, K.counter, kstop, jstep); note_launch(); }
    else if (need <= 16)
        { k_gs_pass<T, 16><<<nb, kThreads, 0, s>>>(basis, K.ld, n, nv, ndots, w, coef, out, K.partials, K.counter, kstop, jstep); note_launch(); }
    else
        { k_gs_pass<T, 32><<<nb, kThreads, 0, s>>>(basis, K.ld, n, nv, ndots, w, coef, out, K.partials, K.counter, kstop, jstep); note_launch(); }
}

void launch_krylov_start(const KrylovDev& K, int m, cudaStream_t s) { { k_krylov_start<<<1, 1, 0, s>>>(K, m); note_launch(); } }

void launch_arnoldi_col(const KrylovDev& K, int j, int m, double tol, cudaStream_t s) {
    { k_arnoldi_col<<<1, 1, 0, s>>>(K, j, m, tol); note_launch(); }
}

template <typename T>
void launch_normalize_scatter(const KrylovDev& K, const uint32_t* meta, long long n, int j, int m, T* Fq,
                              cudaStream_t s) {
    if (n > 0) { k_normalize_scatter<T><<<blocks_for(n), kThreads, 0, s>>>(K, meta, n, j, m, Fq); note_launch(); }
}

int phi1_init() {
    return cudaFuncSetAttribute(k_phi1, cudaFuncAttributeMaxDynamicSharedMemorySize, 7 * kES * (int)sizeof(double)) ==
                   cudaSuccess ? 0 : -1;
}

void launch_phi1(const KrylovDev& K, int m, double dt, cudaStream_t s) {
    { k_phi1<<<1, 256, 7 * kES * sizeof(double), s>>>(K, m, dt); note_launch(); }
}

template <typename T>
void launch_update(const KrylovDev& K, const uint32_t* meta, long long n, double dt, T* omega, T* L, cudaStream_t s) {
    if (n > 0) { k_update<T><<<blocks_for(n), kThreads, 0, s>>>(K, meta, n, dt, omega, L); note_launch(); }
}

#define WRC_INST(T)                                                                                          \
    template void launch_gs_pass<T>(const KrylovDev&, long long, int, int, const double*, double*,          \
                                    const int*, int, cudaStream_t);                                        \
    template void launch_normalize_scatter<T>(const KrylovDev&, const uint32_t*, long long, int, int, T*,   \
                                              cudaStream_t);                                               \
    template void launch_update<T>(const KrylovDev&, const uint32_t*, long long, double, T*, T*, cudaStream_t);
WRC_INST(double)
WRC_INST(float)
#undef WRC_INST

}  // namespace wrc
