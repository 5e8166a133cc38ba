// Krylov projection of the time step (Sec. 2.1: the discrete system projected
// onto a Krylov subspace), as one persistent cooperative kernel per step:
//   b = A_n omega + g,  beta = |b|,  v_0 = b / beta,
//   Arnoldi with classical Gram-Schmidt applied twice (FP64 inner products,
//   deterministic reductions), happy breakdown when h_{j+1,j} <= tol |A v_j|,
//   y = phi_1(dt H_k) e_1 from the exponential of the augmented Hessenberg
//   matrix, omega <- omega + dt beta V_k y.
// Phases are separated by a grid barrier with a bounded wait; every block
// reduces the per-block partial sums itself, in the same order, so all blocks
// hold identical coefficients and take identical breakdown decisions.
#include "kernels.h"
#include "operator.cuh"

namespace wrc {

namespace {

constexpr int kPT = 512;      // threads per block
constexpr int kNV = 32;       // accumulator slots: basis vectors per pass (<= m + 1 <= 32)
constexpr int kOutP = 33;     // partial sums per block: kNV dots + a squared norm
constexpr int kE = 32;        // padded dimension of the augmented matrix (k + 1 <= 32)
constexpr int kES = kE * kE;
constexpr int kExpmSmem = 7 * kES * (int)sizeof(double);

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier for a cooperative launch.  The wait of each block is
// bounded by limit_ns; a block that runs out sets bit 1 of *err, and every
// waiter leaves as soon as *err is non-zero, so the kernel always returns.
__device__ bool grid_sync(unsigned* bar, int* err, unsigned long long limit_ns) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* vgen = bar + 1;
        volatile int* verr = err;
        const unsigned gen = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u) + 1u;
        if (arrived == gridDim.x) {
            *(volatile unsigned*)bar = 0u;
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const unsigned long long t0 = gtimer();
            while (*vgen == gen) {
                if (*verr) break;
                if (gtimer() - t0 > limit_ns) {
                    atomicOr(err, 2);
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *(volatile int*)err == 0;
}

// Per-block sums of acc[0..ndots) and of acc[kNV] (a squared norm) into
// dst[0..ndots] (the norm at index ndots).
__device__ __forceinline__ void block_partials(double (&acc)[kNV + 1], int ndots, double* dst,
                                               double (*s_red)[kNV + 1]) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int t = 0; t <= kNV; ++t) {
        if (t < ndots || t == kNV) {
            double v = acc[t];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) s_red[wid][t] = v;
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t <= ndots; t += blockDim.x) {
        const int src = t < ndots ? t : kNV;
        double v = 0.0;
        for (int q = 0; q < kPT / 32; ++q) v += s_red[q][src];
        dst[t] = v;
    }
}

// Sum over all blocks of part[b * kOutP + t], t < nout, into s_out: warp w
// handles outputs w, w + 16, ...; lane l adds blocks l, l + 32, ... in order,
// then a fixed shuffle tree.  Same order in every block.
__device__ __forceinline__ void reduce_all(const double* part, int nout, double* s_out) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int t = wid; t < nout; t += kPT / 32) {
        double v = 0.0;
        for (unsigned b = lane; b < gridDim.x; b += 32) v += __ldcg(part + (size_t)b * kOutP + t);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) s_out[t] = v;
    }
    __syncthreads();
}

// ---- exponential of the augmented matrix, by one block ---------------------
// Pade [13/13] approximant with scaling and squaring (Higham, SIAM J. Matrix
// Anal. Appl. 26 (2005) 1179-1193); theta_13 is that paper's bound, the Pade
// coefficients come from their closed form
// c_j = (2m - j)! m! / ((2m)! j! (m - j)!), m = 13, normalised to c_0 = 1.

__device__ void mm_blk(const double* A, const double* B, double* C, int N) {
    for (int t = threadIdx.x; t < N * N; t += blockDim.x) {
        const int r = t / N, c = t % N;
        double s = 0.0;
        for (int q = 0; q < N; ++q) s += A[r * kE + q] * B[q * kE + c];
        C[r * kE + c] = s;
    }
    __syncthreads();
}

// y[0..m) = phi_1(dt H_k) e_1 (zeros beyond k) from E = exp([[dt H_k, e_1], [0, 0]]).
__device__ void phi1_block(const double* __restrict__ H, int k, int m, double dt, double* __restrict__ y, double* sm) {
    __shared__ double c[14];
    __shared__ double colsum[kE];
    __shared__ int s_s;
    __shared__ double s_f[kE];
    if (k <= 0) {
        for (int t = threadIdx.x; t < m; t += blockDim.x) y[t] = 0.0;
        return;
    }
    double* A = sm;
    double* A2 = A + kES;
    double* A4 = A2 + kES;
    double* A6 = A4 + kES;
    double* U = A6 + kES;
    double* V = U + kES;
    double* T1 = V + kES;
    const int N = k + 1;
    for (int t = threadIdx.x; t < kES; t += blockDim.x) {
        const int r = t / kE, q = t % kE;
        double v = 0.0;
        if (r < k && q < k) v = dt * H[(size_t)r * m + q];
        if (r == 0 && q == k) v = 1.0;
        A[t] = v;
    }
    if (threadIdx.x == 0) {
        c[0] = 1.0;
        for (int j = 1; j <= 13; ++j) c[j] = c[j - 1] * (double)(13 - j + 1) / ((double)j * (double)(26 - j + 1));
    }
    __syncthreads();
    if (threadIdx.x < N) {
        double s = 0.0;
        for (int r = 0; r < N; ++r) s += fabs(A[r * kE + threadIdx.x]);
        colsum[threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double nrm = 0.0;
        for (int q = 0; q < N; ++q) nrm = fmax(nrm, colsum[q]);
        const double theta13 = 5.371920351148152;
        s_s = nrm > theta13 ? (int)ceil(log2(nrm / theta13)) : 0;
    }
    __syncthreads();
    const int s = s_s;
    if (s > 0) {
        const double f = ldexp(1.0, -s);
        for (int t = threadIdx.x; t < kES; t += blockDim.x) A[t] *= f;
        __syncthreads();
    }
    mm_blk(A, A, A2, N);
    mm_blk(A2, A2, A4, N);
    mm_blk(A4, A2, A6, N);
    // U = A [A6 (c13 A6 + c11 A4 + c9 A2) + c7 A6 + c5 A4 + c3 A2 + c1 I]
    // V =    A6 (c12 A6 + c10 A4 + c8 A2) + c6 A6 + c4 A4 + c2 A2 + c0 I
    for (int t = threadIdx.x; t < kES; t += blockDim.x) T1[t] = c[13] * A6[t] + c[11] * A4[t] + c[9] * A2[t];
    __syncthreads();
    mm_blk(A6, T1, U, N);
    for (int t = threadIdx.x; t < kES; t += blockDim.x) {
        const int r = t / kE, q = t % kE;
        U[t] += c[7] * A6[t] + c[5] * A4[t] + c[3] * A2[t] + (r == q ? c[1] : 0.0);
        T1[t] = c[12] * A6[t] + c[10] * A4[t] + c[8] * A2[t];
    }
    __syncthreads();
    mm_blk(A6, T1, V, N);
    for (int t = threadIdx.x; t < kES; t += blockDim.x) {
        const int r = t / kE, q = t % kE;
        V[t] += c[6] * A6[t] + c[4] * A4[t] + c[2] * A2[t] + (r == q ? c[0] : 0.0);
    }
    __syncthreads();
    mm_blk(A, U, T1, N);    // T1 = U
    // solve (V - U) X = (V + U): matrix in A4, right-hand sides (then X) in A2
    for (int t = threadIdx.x; t < kES; t += blockDim.x) {
        A2[t] = V[t] + T1[t];
        A4[t] = V[t] - T1[t];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int col = 0; col < N; ++col) {
        if (threadIdx.x < 32) {   // warp 0: partial pivoting, row swap, multipliers
            double best = lane >= col && lane < N ? fabs(A4[lane * kE + col]) : -1.0;
            int piv = lane;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int op = __shfl_xor_sync(0xffffffffu, piv, o);
                if (ob > best || (ob == best && op < piv)) {
                    best = ob;
                    piv = op;
                }
            }
            if (piv != col && lane < N) {
                const double a = A4[col * kE + lane];
                A4[col * kE + lane] = A4[piv * kE + lane];
                A4[piv * kE + lane] = a;
                const double b = A2[col * kE + lane];
                A2[col * kE + lane] = A2[piv * kE + lane];
                A2[piv * kE + lane] = b;
            }
            __syncwarp();
            if (lane > col && lane < N) s_f[lane] = A4[lane * kE + col] / A4[col * kE + col];
        }
        __syncthreads();
        for (int t = threadIdx.x; t < (N - col - 1) * N; t += blockDim.x) {
            const int r = col + 1 + t / N, q = t % N;
            const double f = s_f[r];
            A2[r * kE + q] -= f * A2[col * kE + q];
            if (q > col) A4[r * kE + q] -= f * A4[col * kE + q];
        }
        __syncthreads();
    }
    // back substitution, one right-hand-side column per thread
    if (threadIdx.x < N) {
        const int q = threadIdx.x;
        for (int row = N - 1; row >= 0; --row) {
            double v = A2[row * kE + q];
            for (int cc = row + 1; cc < N; ++cc) v -= A4[row * kE + cc] * A2[cc * kE + q];
            A2[row * kE + q] = v / A4[row * kE + row];
        }
    }
    __syncthreads();
    double* X = A2;
    double* Y = T1;
    for (int q = 0; q < s; ++q) {
        mm_blk(X, X, Y, N);
        double* tmp = X;
        X = Y;
        Y = tmp;
    }
    for (int t = threadIdx.x; t < m; t += blockDim.x) y[t] = t < k ? X[t * kE + k] : 0.0;
}

__global__ void __launch_bounds__(kPT, 1) k_krylov_step(KrylovStepArgs A) {
    extern __shared__ double dsm[];
    __shared__ double s_red[kPT / 32][kNV + 1];
    __shared__ double s_h[kOutP];
    __shared__ double s_c[kNV];
    const int n = A.n;
    const int stride = gridDim.x * blockDim.x;
    const int a0 = blockIdx.x * blockDim.x + threadIdx.x;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    double* P0 = A.part;
    double* P1 = P0 + (size_t)gridDim.x * kOutP;
    double* P2 = P1 + (size_t)gridDim.x * kOutP;
    const double nu = A.nu, r = A.r;
    const int m = A.m;
    double acc[kNV + 1];

    // b = A_n omega + g  (L holds R(omega), ghosts included)
#pragma unroll
    for (int t = 0; t <= kNV; ++t) acc[t] = 0.0;
    for (int a = a0; a < n; a += stride) {
        double v = apply_point<double, false>(A.L, A.meta[a], A.Ua[a], A.Va[a], nu, r, A.g, A.c1J, A.c2J);
        if (A.ga) v += A.ga[a];
        A.w[a] = v;
        acc[kNV] += v * v;
    }
    block_partials(acc, 0, P0 + (size_t)blockIdx.x * kOutP, s_red);
    if (!grid_sync(A.bar, A.err, A.limit_ns)) return;
    reduce_all(P0, 1, s_h);
    const double beta = sqrt(s_h[0]);
    int k = m;
    if (!(beta > 0.0) || !isfinite(beta)) {
        k = 0;
        if (lead && !isfinite(beta)) atomicOr(A.flags, 1);
    }
    if (lead) *A.beta = beta;

    if (k > 0) {
        const double inv = 1.0 / beta;
        for (int a = a0; a < n; a += stride) {
            const double v = A.w[a] * inv;
            A.basis[a] = v;
            A.Lq[meta_pos(A.meta[a])] = v;
        }
        if (!grid_sync(A.bar, A.err, A.limit_ns)) return;
        for (int j = 0; j < m; ++j) {
            const int nv = j + 1;
            // ghost values of v_j, coarse to fine
            for (int l = 1; l <= A.g.J; ++l) {
                const int cnt = A.gcnt[l];
                if (cnt == 0) continue;
                const int* gl = A.glist + A.gbeg[l];
                for (int t = a0; t < cnt; t += stride) {
                    const int p = gl[t];
                    A.Lq[p] = predict<double, true>(A.Lq, p & A.g.mask, p >> A.g.L, l, A.g);
                }
                if (!grid_sync(A.bar, A.err, A.limit_ns)) return;
            }
            // w = A v_j and the first Gram-Schmidt dots
#pragma unroll
            for (int t = 0; t <= kNV; ++t) acc[t] = 0.0;
            for (int a = a0; a < n; a += stride) {
                const double v = apply_point<double, true>(A.Lq, A.meta[a], A.Ua[a], A.Va[a], nu, r, A.g, A.c1J, A.c2J);
                A.w[a] = v;
#pragma unroll
                for (int t = 0; t < kNV; ++t)
                    if (t < nv) acc[t] += A.basis[(size_t)t * A.ld + a] * v;
                acc[kNV] += v * v;
            }
            block_partials(acc, nv, P0 + (size_t)blockIdx.x * kOutP, s_red);
            if (!grid_sync(A.bar, A.err, A.limit_ns)) return;
            reduce_all(P0, nv + 1, s_h);
            const double wn2 = s_h[nv];
            for (int t = threadIdx.x; t < nv; t += blockDim.x) s_c[t] = s_h[t];
            __syncthreads();
            // second pass: w -= V h1, dots again
#pragma unroll
            for (int t = 0; t <= kNV; ++t) acc[t] = 0.0;
            for (int a = a0; a < n; a += stride) {
                double x = A.w[a];
#pragma unroll
                for (int t = 0; t < kNV; ++t)
                    if (t < nv) x -= A.basis[(size_t)t * A.ld + a] * s_c[t];
                A.w[a] = x;
#pragma unroll
                for (int t = 0; t < kNV; ++t)
                    if (t < nv) acc[t] += A.basis[(size_t)t * A.ld + a] * x;
                acc[kNV] += x * x;
            }
            block_partials(acc, nv, P1 + (size_t)blockIdx.x * kOutP, s_red);
            if (!grid_sync(A.bar, A.err, A.limit_ns)) return;
            reduce_all(P1, nv + 1, s_h);
            bool bad = false;
            for (int t = 0; t < nv; ++t) bad |= !isfinite(s_c[t] + s_h[t]);
            if (blockIdx.x == 0)
                for (int t = threadIdx.x; t < nv; t += blockDim.x) A.H[(size_t)t * m + j] = s_c[t] + s_h[t];
            __syncthreads();
            for (int t = threadIdx.x; t < nv; t += blockDim.x) s_c[t] = s_h[t];
            __syncthreads();
            // third pass: w -= V h2, |w|^2
            acc[kNV] = 0.0;
            for (int a = a0; a < n; a += stride) {
                double x = A.w[a];
#pragma unroll
                for (int t = 0; t < kNV; ++t)
                    if (t < nv) x -= A.basis[(size_t)t * A.ld + a] * s_c[t];
                A.w[a] = x;
                acc[kNV] += x * x;
            }
            block_partials(acc, 0, P2 + (size_t)blockIdx.x * kOutP, s_red);
            if (!grid_sync(A.bar, A.err, A.limit_ns)) return;
            reduce_all(P2, 1, s_h);
            const double hn = sqrt(s_h[0]);
            if (lead) A.H[(size_t)(j + 1) * m + j] = hn;
            if (bad || !isfinite(hn)) {
                if (lead) atomicOr(A.flags, 1);
                k = j + 1;
                break;
            }
            if (hn <= A.tol * sqrt(wn2)) {
                k = j + 1;
                break;
            }
            if (j + 1 < m) {
                const double inv2 = 1.0 / hn;
                for (int a = a0; a < n; a += stride) {
                    const double v = A.w[a] * inv2;
                    A.basis[(size_t)(j + 1) * A.ld + a] = v;
                    A.Lq[meta_pos(A.meta[a])] = v;
                }
                if (!grid_sync(A.bar, A.err, A.limit_ns)) return;
            }
        }
    }
    if (blockIdx.x == 0) {
        if (threadIdx.x == 0) *A.kstop = k;
        __syncthreads();
        phi1_block(A.H, k, m, A.dt, A.y, dsm);
    }
    if (!grid_sync(A.bar, A.err, A.limit_ns)) return;
    // omega <- omega + dt beta V_k y, also into the lattice array L
    for (int t = threadIdx.x; t < k; t += blockDim.x) s_c[t] = A.dt * beta * __ldcg(A.y + t);
    __syncthreads();
    for (int a = a0; a < n; a += stride) {
        double inc = 0.0;
        for (int t = 0; t < k; ++t) inc += s_c[t] * A.basis[(size_t)t * A.ld + a];
        const double x = A.omega[a] + inc;
        A.omega[a] = x;
        A.L[meta_pos(A.meta[a])] = x;
    }
}

}  // namespace

int krylov_step_init(int* max_blocks) {
    if (cudaFuncSetAttribute(k_krylov_step, cudaFuncAttributeMaxDynamicSharedMemorySize, kExpmSmem) != cudaSuccess)
        return -1;
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_krylov_step, kPT, kExpmSmem) != cudaSuccess || per < 1)
        return -2;
    *max_blocks = sms * per;
    return 0;
}

int krylov_step_blocks(long long n, int max_blocks) {
    long long b = (n + kPT - 1) / kPT;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (int)b;
}

cudaError_t launch_krylov_step(const KrylovStepArgs& args, int blocks, cudaStream_t s) {
    KrylovStepArgs a = args;
    void* params[] = {&a};
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_krylov_step, dim3(blocks), dim3(kPT), params,
                                                kExpmSmem, s);
    if (e == cudaSuccess) note_launch();
    return e;
}

size_t krylov_partials_doubles(int max_blocks) { return (size_t)3 * max_blocks * kOutP; }

}  // namespace wrc
