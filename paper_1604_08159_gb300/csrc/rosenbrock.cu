// Kernels of the exponential Rosenbrock-Euler step (Sec. 1 and 2.1: the
// Krylov projection with the Jacobian of the discrete right-hand side,
//   omega^{n+1} = omega^n + dt phi_1(dt J_n) F(omega^n),
//   J_n q = A_n q - U[q] D_x omega^n - V[q] D_y omega^n,
// U[q], V[q] the velocity of q's own streamfunction: a reconstruction and a
// Poisson solve per Krylov vector, so the Arnoldi process runs as a sequence
// of launches driven by the host (api.cu) rather than inside the persistent
// kernel.  Gram-Schmidt is applied twice (classical), with FP64 inner
// products accumulated per block and added in a fixed order; the Krylov
// dimension used (a happy breakdown stops it) lives on the device, and every
// kernel of a later Arnoldi step returns at once.  phi_1 and the update as in
// the persistent kernel.
#include "krylov_impl.cuh"

namespace wrc {

namespace {

constexpr int kRbThreads = 256;
constexpr int kRbMaxVec = kNV + 1;   // basis vectors of a pass, and w itself
static_assert(kRbMaxVec == kRbPartWidth, "partial-sum rows");

// D_x omega, D_y omega at the active points (the operator's first
// derivatives at the stencil levels, ghost values from the lattice F).
template <typename T, int P>
__global__ void k_rb_grad(const T* __restrict__ F, const uint32_t* __restrict__ meta, int n, T* __restrict__ dwx,
                          T* __restrict__ dwy, Geom g, T c1J, T c2J) {
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < n; a += gridDim.x * blockDim.x) {
        // -U Dx - V Dy with (U, V) = (-1, 0) and (0, -1), no diffusion or damping
        dwx[a] = apply_point<T, false, P>(F, meta[a], T(-1), T(0), T(0), T(0), g, c1J, c2J);
        dwy[a] = apply_point<T, false, P>(F, meta[a], T(0), T(-1), T(0), T(0), g, c1J, c2J);
    }
}

// w = A_n q - U[q] D_x omega - V[q] D_y omega (F holds R(q) with its ghosts).
template <typename T, int P>
__global__ void k_rb_apply(const T* __restrict__ F, const uint32_t* __restrict__ meta, int n,
                           const T* __restrict__ Ua, const T* __restrict__ Va, T nu, T r,
                           const T* __restrict__ Uq, const T* __restrict__ Vq, const T* __restrict__ dwx,
                           const T* __restrict__ dwy, T* __restrict__ w, Geom g, T c1J, T c2J,
                           const int* __restrict__ kstop, int j) {
    if (j >= *kstop) return;
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < n; a += gridDim.x * blockDim.x)
        w[a] = apply_point<T, false, P>(F, meta[a], Ua[a], Va[a], nu, r, g, c1J, c2J) - Uq[a] * dwx[a] -
               Vq[a] * dwy[a];
}

// Per-block FP64 partial sums: part[b * kRbMaxVec + v] = sum over the block's
// points of basis_v . w for v < nv, and (self) |w|^2 at v = nv.
template <typename T>
__global__ void __launch_bounds__(kRbThreads) k_rb_dots(const T* __restrict__ basis, long long ld, int nv,
                                                        const T* __restrict__ w, int n, bool self,
                                                        double* __restrict__ part, const int* __restrict__ kstop,
                                                        int j) {
    if (j >= *kstop) return;
    __shared__ double s_red[kRbThreads / 32][kRbMaxVec];
    double acc[kRbMaxVec];
#pragma unroll
    for (int v = 0; v < kRbMaxVec; ++v) acc[v] = 0.0;
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < n; a += gridDim.x * blockDim.x) {
        const double x = (double)w[a];
#pragma unroll
        for (int v = 0; v < kRbMaxVec - 1; ++v)
            if (v < nv) acc[v] += (double)basis[(size_t)v * ld + a] * x;
        if (self) acc[kRbMaxVec - 1] += x * x;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < kRbMaxVec; ++v) {
        double s = acc[v];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) s_red[wid][v] = s;
    }
    __syncthreads();
    for (int v = threadIdx.x; v < kRbMaxVec; v += blockDim.x) {
        double s = 0.0;
        for (int q = 0; q < kRbThreads / 32; ++q) s += s_red[q][v];
        part[(size_t)blockIdx.x * kRbMaxVec + v] = s;
    }
}

// Coefficient bookkeeping of one reduction (one block of 64 threads; the
// partial sums of nblk blocks added in block order):
//   mode 0 (first pass of step j): c = Q^T w -> H[:, j] = c, coef = c, and
//          |A q_j|^2 = |w|^2 kept for the breakdown test;
//   mode 1 (second pass): c = Q^T w -> H[:, j] += c, coef = c;
//   mode 2 (norm after step j): h = |w|, H[j + 1][j] = h; a happy breakdown
//          (h <= tol |A q_j|) or a non-finite h stops the process at
//          k = j + 1 (non-finite also raises flags bit 0), else scale = 1/h;
//   mode 3 (beta): beta = |w| (b); beta = 0 stops it at k = 0, else scale = 1/beta.
// sc: [0] scale, [1] |A q_j|^2.
__global__ void k_rb_sum(const double* __restrict__ part, int nblk, int nv, int mode, int j, int m, double tol,
                         double* __restrict__ H, double* __restrict__ coef, double* __restrict__ sc,
                         double* __restrict__ beta, int* __restrict__ kstop, int* __restrict__ flags) {
    if (mode != 3 && j >= *kstop) return;
    __shared__ double s_out[kRbMaxVec];
    const int nout = (mode == 2 || mode == 3) ? 1 : nv + (mode == 0 ? 1 : 0);
    for (int t = threadIdx.x; t < nout; t += blockDim.x) {
        const int v = (mode == 2 || mode == 3 || t == nv) ? kRbMaxVec - 1 : t;
        double s = 0.0;
        for (int b = 0; b < nblk; ++b) s += part[(size_t)b * kRbMaxVec + v];
        s_out[t] = s;
    }
    __syncthreads();
    if (mode == 0 || mode == 1) {
        for (int t = threadIdx.x; t < nv; t += blockDim.x) {
            const double c = s_out[t];
            coef[t] = c;
            H[(size_t)t * m + j] = mode == 0 ? c : H[(size_t)t * m + j] + c;
        }
        if (mode == 0 && threadIdx.x == 0) sc[1] = s_out[nv];
        return;
    }
    if (threadIdx.x != 0) return;
    const double q = s_out[0];
    const double h = sqrt(q);
    if (mode == 3) {
        *beta = h;
        if (!(h > 0.0) || !isfinite(h)) {
            if (!isfinite(h)) atomicOr(flags, 1);
            *kstop = 0;
            sc[0] = 0.0;
        } else {
            *kstop = m;
            sc[0] = 1.0 / h;
        }
        return;
    }
    H[(size_t)(j + 1) * m + j] = h;
    const bool bad = !isfinite(h) || !isfinite(sc[1]);
    if (bad) atomicOr(flags, 1);
    if (bad || h <= tol * sqrt(sc[1])) *kstop = j + 1;
    else sc[0] = 1.0 / h;
}

// w -= sum_{v < nv} coef_v basis_v (in the bulk type).
template <typename T>
__global__ void k_rb_axpy(const T* __restrict__ basis, long long ld, int nv, const double* __restrict__ coef,
                          T* __restrict__ w, int n, const int* __restrict__ kstop, int j) {
    if (j >= *kstop) return;
    __shared__ T s_c[kNV];
    for (int t = threadIdx.x; t < nv; t += blockDim.x) s_c[t] = (T)coef[t];
    __syncthreads();
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < n; a += gridDim.x * blockDim.x) {
        T p[4] = {T(0), T(0), T(0), T(0)};
        for (int v = 0; v < nv; ++v) p[v & 3] += basis[(size_t)v * ld + a] * s_c[v];
        w[a] -= (p[0] + p[1]) + (p[2] + p[3]);
    }
}

// basis_{j + 1} = w * scale, unless the process stopped at step j.
template <typename T>
__global__ void k_rb_scale(T* __restrict__ basis, long long ld, const T* __restrict__ w, int n,
                           const double* __restrict__ sc, const int* __restrict__ kstop, int j) {
    if (j >= 0 && *kstop <= j + 1) return;   // stopped at or before step j
    const double s = sc[0];
    T* dst = basis + (size_t)(j + 1) * ld;
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < n; a += gridDim.x * blockDim.x)
        dst[a] = (T)((double)w[a] * s);
}

// y = phi_1(dt H_k) e_1 (k = *kstop; zero for k = 0), by one block.
__global__ void __launch_bounds__(kPT) k_rb_phi1(const double* __restrict__ H, const int* __restrict__ kstop, int m,
                                                 double dt, double* __restrict__ y, int* __restrict__ flags) {
    __shared__ double s_part[kPT / 32][kNV + 1];
    __shared__ double s_x[kNV + 1];
    __shared__ int s_int[3];
    const int k = *kstop;
    if (k == 0) {
        for (int t = threadIdx.x; t < m; t += kPT) y[t] = 0.0;
        return;
    }
    phi1_block<kPT>(H, k, m, dt, y, flags, s_part, s_x, s_int);
}

// omega <- omega + dt beta V_k y at the active points (accumulated in FP64),
// also written into the lattice array L.
template <typename T>
__global__ void k_rb_combine(const T* __restrict__ basis, long long ld, const double* __restrict__ y,
                             const double* __restrict__ beta, double dt, const int* __restrict__ kstop,
                             T* __restrict__ omega, T* __restrict__ L, const uint32_t* __restrict__ meta, int n) {
    __shared__ double s_c[kNV];
    const int k = *kstop;
    for (int t = threadIdx.x; t < k; t += blockDim.x) s_c[t] = dt * (*beta) * y[t];
    __syncthreads();
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < n; a += gridDim.x * blockDim.x) {
        double inc = 0.0;
        for (int t = 0; t < k; ++t) inc += s_c[t] * (double)basis[(size_t)t * ld + a];
        const T x = (T)((double)omega[a] + inc);
        omega[a] = x;
        L[meta_pos(meta[a])] = x;
    }
}

int rb_blocks(long long n) {
    long long b = (n + kRbThreads - 1) / kRbThreads;
    if (b < 1) b = 1;
    if (b > kRbPartBlocks) b = kRbPartBlocks;
    return (int)b;
}

template <typename F>
void rb_by_order(int P, F&& f) {
    if (P == 3) f(std::integral_constant<int, 3>{});
    else if (P == 4) f(std::integral_constant<int, 4>{});
    else f(std::integral_constant<int, 2>{});
}

}  // namespace

template <typename T>
cudaError_t rb_gradient(const RbArgs& a, cudaStream_t s) {
    rb_by_order(a.g.P, [&](auto PC) {
        constexpr int P = decltype(PC)::value;
        k_rb_grad<T, P><<<rb_blocks(a.n), kRbThreads, 0, s>>>((const T*)a.L, a.meta, a.n, (T*)a.dwx, (T*)a.dwy, a.g,
                                                               (T)a.c1J, (T)a.c2J);
    });
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t rb_apply(const RbArgs& a, int j, cudaStream_t s) {
    rb_by_order(a.g.P, [&](auto PC) {
        constexpr int P = decltype(PC)::value;
        k_rb_apply<T, P><<<rb_blocks(a.n), kRbThreads, 0, s>>>(
            (const T*)a.Lq, a.meta, a.n, (const T*)a.Ua, (const T*)a.Va, (T)a.nu, (T)a.r, (const T*)a.Uq,
            (const T*)a.Vq, (const T*)a.dwx, (const T*)a.dwy, (T*)a.w, a.g, (T)a.c1J, (T)a.c2J, a.kstop, j);
    });
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t rb_reduce(const RbArgs& a, int nv, bool self, int mode, int j, cudaStream_t s) {
    const int nb = rb_blocks(a.n);
    k_rb_dots<T><<<nb, kRbThreads, 0, s>>>((const T*)a.basis, a.ld, nv, (const T*)a.w, a.n, self, a.part, a.kstop,
                                           mode == 3 ? -1 : j);
    note_launch();
    k_rb_sum<<<1, 64, 0, s>>>(a.part, nb, nv, mode, j, a.m, a.tol, a.H, a.coef, a.sc, a.beta, a.kstop, a.flags);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t rb_axpy(const RbArgs& a, int nv, int j, cudaStream_t s) {
    k_rb_axpy<T><<<rb_blocks(a.n), kRbThreads, 0, s>>>((const T*)a.basis, a.ld, nv, a.coef, (T*)a.w, a.n, a.kstop,
                                                       j);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t rb_scale(const RbArgs& a, int j, cudaStream_t s) {
    k_rb_scale<T><<<rb_blocks(a.n), kRbThreads, 0, s>>>((T*)a.basis, a.ld, (const T*)a.w, a.n, a.sc, a.kstop, j);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t rb_finish(const RbArgs& a, cudaStream_t s) {
    k_rb_phi1<<<1, kPT, 0, s>>>(a.H, a.kstop, a.m, a.dt, a.y, a.flags);
    note_launch();
    k_rb_combine<T><<<rb_blocks(a.n), kRbThreads, 0, s>>>((const T*)a.basis, a.ld, a.y, a.beta, a.dt, a.kstop,
                                                          (T*)a.omega, (T*)a.L, a.meta, a.n);
    note_launch();
    return cudaGetLastError();
}

#define WRC_INST(T)                                                                   \
    template cudaError_t rb_gradient<T>(const RbArgs&, cudaStream_t);                 \
    template cudaError_t rb_apply<T>(const RbArgs&, int, cudaStream_t);               \
    template cudaError_t rb_reduce<T>(const RbArgs&, int, bool, int, int, cudaStream_t); \
    template cudaError_t rb_axpy<T>(const RbArgs&, int, int, cudaStream_t);           \
    template cudaError_t rb_scale<T>(const RbArgs&, int, cudaStream_t);               \
    template cudaError_t rb_finish<T>(const RbArgs&, cudaStream_t);
WRC_INST(double)
WRC_INST(float)
#undef WRC_INST

}  // namespace wrc
