// Host-side launchers of the library's CUDA kernels (internal interface).
#pragma once

#include "common.cuh"

namespace wrc {

// ---- grid.cu: lattice, transform, thresholding, index sets -----------------
template <typename T>
void launch_init_vortices(T* L, const double* params, int n, const Geom& g, cudaStream_t s);
// Launchers taking `dn` read the item count from device memory when it is
// given (n is then the capacity the grid covers; capturable in a CUDA graph).
// With rows (NJ + 1 ints, zero before: h = NJ/2 flags, one per pair of
// rows 2q, 2q+1, then a count and a list), also flags the pairs holding a
// row within `margin` rows of a grid point and lists them (in any order).
template <typename T>
void launch_scatter(const uint32_t* meta, const T* vals, long long n, T* L, cudaStream_t s, const int* dn = nullptr,
                    int* rows = nullptr, int margin = 0, const Geom* g = nullptr);
// L <- R(u): the values at the grid points of act stay, every other lattice
// point gets its coarse-to-fine DD prediction (Eq. 6, detail zero).  One
// tiled launch (or, where its shared-memory arrays do not fit, two launches
// per level).
template <typename T>
void launch_reconstruct(T* L, const uint8_t* act, const Geom& g, cudaStream_t s);
// Values at the points of the new grid nxt that are not in act, by DD
// prediction from the values of act (one launch per level, coarse to fine).
template <typename T>
void launch_recon_new(T* L, const uint8_t* act, const uint8_t* nxt, const Geom& g, cudaStream_t s);
template <typename T>
void launch_details_adj(const uint32_t* meta, long long n, const T* L, double eps, T* det,
                        uint8_t* sig, uint8_t* nxt, const Geom& g, cudaStream_t s, const int* dn = nullptr);
void launch_closure_level(uint8_t* mask, const uint8_t* excl, int j, const Geom& g, cudaStream_t s);
void launch_stencil_ghost(const uint8_t* act, uint8_t* gho, uint8_t* JJ, const Geom& g, cudaStream_t s);
void launch_validate_grid(const uint8_t* act, int* flag, const Geom& g, cudaStream_t s);
void launch_compact(const uint8_t* act, const uint8_t* gho, const Geom& g, int nkeys, int* blk_counts,
                    int* blk_off, int* counts, int* list, cudaStream_t s);
template <typename T>
void launch_finalize(const int* list, long long n, const uint8_t* JJ, const T* L, uint32_t* meta, T* omega,
                     cudaStream_t s, const int* dn = nullptr);
template <typename T>
void launch_ghost_fill(T* F, const int* glist, long long n, int j, const Geom& g, const int* kstop,
                       int jstep, cudaStream_t s);
void launch_level_counts(const uint32_t* meta, long long n, unsigned long long* counts, const Geom& g,
                         cudaStream_t s);
void launch_meta_to_mask(const uint32_t* meta, long long n, uint8_t* mask, cudaStream_t s);
void launch_list_to_mask(const int* list, long long n, uint8_t* mask, cudaStream_t s);
void launch_meta_unpack(const uint32_t* meta, long long n, int* idx, uint8_t* jx, uint8_t* jy,
                        cudaStream_t s);
// Interpolation rows of all ghosts (the list holds the active points, then
// the ghosts of levels 1..J) over the active points, and the combined index
// map.  dcounts: the compaction's per-key counts on the device (all sizes
// are read there; the grids cover cap_a + cap_g items).  One launch for all
// levels: ready (cap_g + 1 ints, cleared here) holds the ghosts' ready flags
// and the counter that hands out ghosts in list order; a wait for a coarser
// ghost's row longer than limit_ns sets bit 1 of *err.
constexpr int kGhostRowMax = 64;
void launch_ghost_rows(const int* list, int J, int* lat2idx, int* row_len, int* row_idx, double* row_w, int rmax,
                       const Geom& g, int* overflow, int* ready, int* err, unsigned long long limit_ns,
                       cudaStream_t s, const int* dcounts, long long cap_a, long long cap_g);

// ---- fft.cu: streamfunction -------------------------------------------------
struct PoissonPlan {
    int n = 0, logn = 0;
    bool fp32 = false;
    void* tw = nullptr;      // exp(-2 pi i t/n), t < n (complex of the run's bulk type)
    void* ptw = nullptr;     // the same twiddles as per-pass tables (see fft.cu)
    void* sigma = nullptr;   // symbol of the 4th-order second-derivative stencil
    void* dsym = nullptr;    // symbol of the 4th-order first-derivative stencil (imaginary part)
};
int poisson_plan_init(PoissonPlan& p, const Geom& g, bool fp32, cudaStream_t s);
void poisson_plan_free(PoissonPlan& p);
// psi = L_h^{-1}(-(R - mean R)), mean(psi) = 0; C1, C2 are NJ*NJ complex work
// arrays.  With U, V and a third work array C3, also U = D_y psi and
// V = -D_x psi on the lattice, evaluated in the Fourier domain (no cancellation);
// with S11, S12 and a fourth work array C4, also the strain S11 = D_x D_y psi and
// S12 = (D_yy - D_xx) psi / 2.  S11 and S12 may not alias C1, C2 or C3.
// With rows (the flags and list launch_scatter makes), the inverse row
// passes take the listed row pairs only, a few per block, so that the blocks
// with work are the first ones and spread over the SMs: psi alone is written
// only on those rows; with U and V (a step's FP32 form), U, V and the strain
// are written only there and psi, which such a step does not read, not at all.
template <typename T>
void launch_poisson(const PoissonPlan& p, const T* R, T* psi, void* C1, void* C2, const Geom& g, cudaStream_t s,
                    T* U = nullptr, T* V = nullptr, void* C3 = nullptr, T* S11 = nullptr, T* S12 = nullptr,
                    void* C4 = nullptr, const int* rows = nullptr);

// ---- flow.cu: velocity, Smagorinsky forcing, operator, diagnostics ----------
template <typename T>
void launch_velocity_active(const T* psi, const uint32_t* meta, long long n, T* Ua, T* Va,
                            const Geom& g, cudaStream_t s, const int* dn = nullptr);
// Smagorinsky forcing at the active points from the lattice psi, with the
// products nu_t S formed only in the 5 x 5 boxes around the active points
// (halo: an NJ*NJ byte mask, 4-byte aligned; hlist: NJ*NJ + 1 ints of work
// space for the halo list; t2, t3: lattice work arrays).
template <typename T>
void launch_sgs_halo(const T* psi, const uint32_t* meta, long long n, double cs, T* ga, T* t2, T* t3,
                     uint8_t* halo, int* hlist, const Geom& g, cudaStream_t s, const int* dn = nullptr);
// Smagorinsky forcing from the lattice strain (S11, S12): nu_t, then
// a = 2 nu_t S12 and c = nu_t S11 into ta, tc, D_y c into tdyc, g at the active points.
// With rows (the row-pair list of launch_scatter, margin 2 dd_reach(P)), the
// lattice passes run on the listed rows only, which hold what g reads.
template <typename T>
void launch_sgs_from_strain(const T* S11, const T* S12, const uint32_t* meta, long long n, double cs, T* ga, T* ta,
                            T* tc, T* tdyc, const Geom& g, cudaStream_t s, const int* dn = nullptr,
                            const int* rows = nullptr);
template <typename T>
void launch_nut_from_strain(const T* S11, const T* S12, T* nut, double cs, const Geom& g, cudaStream_t s);
template <typename T>
void launch_velocity_gather(const T* Ulat, const T* Vlat, const uint32_t* meta, long long n, T* Ua, T* Va,
                            cudaStream_t s, const int* dn = nullptr);
template <typename T>
void launch_lattice_uv_nut(const T* psi, T* U, T* V, T* nut, double cs, T* tmp, const Geom& g,
                           cudaStream_t s, bool uv_given = false);
template <typename T>
void launch_matvec(const T* F, const uint32_t* meta, long long n, const T* Ua, const T* Va,
                   const T* ga, double nu, double r, T* w, const Geom& g, const int* kstop, int jstep,
                   cudaStream_t s);
// sums over the lattice of R, R^2, U^2 + V^2, |grad R|^2 -> out[0..3] (FP64 sums);
// returns the launch status
template <typename T>
cudaError_t launch_diag(const T* R, const T* psi, double* partials, unsigned* counter, double* out, const Geom& g,
                 cudaStream_t s);
template <typename A, typename B>
void launch_convert(const A* in, B* out, long long n, cudaStream_t s);

// ---- rosenbrock.cu: the exponential Rosenbrock-Euler step (full Jacobian) ---
// Arguments of its launches (bulk type T behind the void pointers).
struct RbArgs {
    Geom g;
    const uint32_t* meta;   // active points
    int n;                  // active count
    const void* L;          // R(omega) on the lattice (in); omega^{n+1} at the active points (out)
    void* Lq;               // R(q) of the current Krylov vector on the lattice
    const void *Ua, *Va;    // frozen velocity at the active points
    void *Uq, *Vq;          // velocity of the current Krylov vector at the active points
    void *dwx, *dwy;        // D_x omega^n, D_y omega^n at the active points
    void* w;                // work vector
    void* basis;            // (m + 1) x ld
    long long ld;
    void* omega;            // compact omega, updated in place
    double* part;           // kRbPartBlocks x (kNV + 1) partial sums
    double* coef;           // Gram-Schmidt coefficients of a pass
    double* sc;             // [0] normalisation, [1] |A q_j|^2
    double* H;              // (m + 1) x m row-major
    double* y;
    double* beta;
    int* kstop;             // Krylov dimension used (set on the device)
    int* flags;             // bit 0: non-finite value met
    int m;
    double dt, tol, nu, r, c1J, c2J;
};
constexpr int kRbPartBlocks = 1024;   // blocks of a reduction (partial-sum rows)
constexpr int kRbPartWidth = 33;      // partial sums per block
template <typename T> cudaError_t rb_gradient(const RbArgs& a, cudaStream_t s);
template <typename T> cudaError_t rb_apply(const RbArgs& a, int j, cudaStream_t s);
// Dot products of w with basis vectors 0..nv-1 (and |w|^2 with self), reduced,
// then the bookkeeping of `mode` (0: first Gram-Schmidt pass of step j, 1:
// second pass, 2: norm and breakdown test of step j, 3: beta).
template <typename T> cudaError_t rb_reduce(const RbArgs& a, int nv, bool self, int mode, int j, cudaStream_t s);
template <typename T> cudaError_t rb_axpy(const RbArgs& a, int nv, int j, cudaStream_t s);
template <typename T> cudaError_t rb_scale(const RbArgs& a, int j, cudaStream_t s);
// phi_1 of the projected matrix and the update of omega (and L).
template <typename T> cudaError_t rb_finish(const RbArgs& a, cudaStream_t s);

// ---- exner.cu: the compressible velocity-Exner form (Eqs. 1-2) -------------
// Arguments of its launches (FP64).  Vectors of the Krylov process stack the
// three fields of the active points: [u (n) | v (n) | pi (n)].
struct ExArgs {
    Geom g;
    const uint32_t* meta;   // active points
    int n;                  // active count
    const int* glist;       // lattice positions of the ghosts
    int ng;
    const int* row_len;     // ghost interpolation rows over the active points
    const int* row_idx;
    const double* row_w;
    int rmax;
    double* Lb[3];          // lattices of u, v, pi at t^n (active and ghost values)
    double* Lq[3];          // lattices of the current Krylov vector's three parts
    const double* f[3];     // compact u, v, pi at t^n
    double* f_out[3];       // compact u, v, pi updated in place
    double* d;              // 8 x ld: u_x, u_y, v_x, v_y, pi_x, pi_y, lap u, lap v
    long long ld;           // leading dimension of d (>= n)
    double C, fc, gx, gy, r, nu, c1J, c2J;
    int full;               // 1: the exact Jacobian; 0: the frozen-coefficient operator
};
// Lattices of the three fields from their compact values (active points and,
// through the interpolation rows, the ghosts).
cudaError_t ex_scatter_fields(const ExArgs& a, const double* const src[3], double* const dst[3], const int* kstop,
                              int j, cudaStream_t s);
// First derivatives and Laplacians of the state at the active points (into
// a.d) and the right-hand side F(U^n) stacked into w (3 n).
cudaError_t ex_base(const ExArgs& a, double* w, cudaStream_t s);
// Fill a lattice with a constant.
cudaError_t ex_fill(double* F, long long n, double value, cudaStream_t s);
// The whole Krylov projection of a velocity-Exner step in one persistent
// cooperative launch (b = F(U^n) in w on entry): classical Gram-Schmidt
// twice on the stacked vectors, four grid barriers per Arnoldi step (bounded
// waits: bit 1 of *err on expiry), phi_1 by block 0, the update.
struct ExKrylov {
    double* basis;          // (m + 1) x ld3
    long long ld3;
    double* w;              // 3 n: b on entry, the work vector
    double* part;           // blocks x kExPartWidth partial sums
    double* H;              // (m + 1) x m, zero on entry
    double* y;
    double* beta;
    int* kstop;
    int* flags;             // bit 0: non-finite value met
    unsigned* bar;          // grid barrier words
    int* err;
    unsigned long long limit_ns;
    int m;
    double dt, tol;
};
int ex_krylov_max_blocks(int P);
cudaError_t ex_krylov(const ExArgs& a, const ExKrylov& K, int blocks, cudaStream_t s);
constexpr int kExKrylovThreads = 128;
constexpr int kExPartWidth = 66;

// ---- krylov.cu: the Krylov-projected step as one cooperative kernel ---------
struct KrylovStepArgs {
    Geom g;
    const uint32_t* meta;   // active points (packed lattice index + stencil levels)
    int n;                  // active count
    const int* glist;       // ghost lattice indices (all levels), ng of them
    int ng;
    const int* row_len;     // ghost interpolation rows over the active points
    const int* row_idx;
    const double* row_w;
    int rmax;
    const int* row_overflow; // non-zero: some row exceeded rmax (the kernel refuses to run)
    void* Gb;               // ghost values of the basis vectors, (m+1) x ldg
    long long ldg;
    // arrays of the run's bulk type (double, or float for the mixed mode)
    const void* Ua;
    const void* Va;
    const void* ga;         // SGS forcing at the active points or nullptr
    double nu, r, c1J, c2J; // nu_eff, Rayleigh r, 1/(12 h_J), 1/(12 h_J^2)
    void* L;                // R(omega) on the lattice (in), omega^{n+1} at the active points (out)
    void* Lq;               // lattice array of the current Krylov vector and its ghost values
    void* omega;            // compact omega, updated in place
    void* basis;            // (m+1) x ld
    long long ld;
    void* w;
    double* H;              // (m+1) x m row-major
    double* y;              // m
    double* beta;           // [1]
    int* kstop;             // [1] Krylov dimension used
    int* flags;             // [1] bit 0: non-finite value met
    double* part;           // 3 x blocks x 33 partial sums
    unsigned* bar;          // grid barrier: {count, generation}
    int* err;               // bit 1: a barrier wait ran out; bit 2 (4): row overflow; bit 4 (16): a clustered
                            // launch did not form its clusters and ran unclustered (not an error)
    int m;
    double dt, tol;
    unsigned long long limit_ns;
    int refuse;             // test switch: a clustered launch runs as if its clusters were not formed
    // phase trace (profiling; nullptr when off): trace[0] the start of block
    // 0, then per grid barrier p the arrival time of each block b at
    // trace[1 + p (nb + 1) + b] and block 0's release at trace[1 + p (nb + 1) + nb]
    // (globaltimer ns), for at most kTracePhases barriers
    unsigned long long* trace;
};
constexpr int kTracePhases = 3 + 3 * 31;
// Co-resident capacity of the single-run Krylov kernel on device dev (also
// for clusters of 2 and 4 blocks, kept per device and precision for
// krylov_step_blocks and the launch; a cluster size whose clusters a probe
// launch does not see formed is not used).
int krylov_step_init(int dev, bool fp32, int P, int* max_blocks);
// Largest cluster size a run created now may use: 4, or the cap set by the
// environment variable WRC_KRYLOV_CLUSTER (1 or 2), read when called.
int krylov_cluster_max();
// A clustered Krylov launch on device dev ran unclustered (its clusters were
// not formed): later launches on the device are planned without clusters.
void krylov_clusters_unformed(int dev);
// Blocks for n active points: one thread per point, capped at max_blocks,
// padded to a whole number of 4- or 2-block clusters (at most cmax) where
// that fits.
int krylov_step_blocks(long long n, int max_blocks, bool fp32, int P, int dev, int cmax);
// Cluster size (1, 2 or 4) of the launch krylov_step_blocks plans for n points.
int krylov_step_cluster(long long n, int max_blocks, bool fp32, int P, int dev, int cmax);
// Cooperative launch on device dev (current); clusters of 4 or 2 (<= cmax) blocks when
// `blocks` is a multiple within their capacity (their blocks pre-add the dot
// sums in distributed shared memory).  The first clustered launch per device
// and precision synchronises `s` and, if the clusters were not formed,
// switches them off for the device and launches again without them.
template <typename T>
cudaError_t launch_krylov_step(const KrylovStepArgs& args, int blocks, cudaStream_t s, int dev, int cmax);
size_t krylov_partials_doubles(int max_blocks);
// Batched Krylov step: `members` problems (device array of arguments) in one
// cooperative launch of `blocks` blocks of pt (64, 128 or 256) threads; block
// b works on problem blk2mem[b], whose blocks are mem_b0[q] .. mem_b0[q+1]-1.
// pair: the spill-free form for the two problems of one run (pt = 128).
int krylov_batch_max_blocks(bool fp32, int P, int pt, bool pair = false);
template <typename T>
cudaError_t launch_krylov_batch(const KrylovStepArgs* d_args, const int* d_blk2mem, const int* d_mem_b0,
                                int members, int blocks, int pt, int P, cudaStream_t s, bool pair = false);

// The kernels of one bulk type T and DD half-order P (2, 3, 4), compiled per
// order in krylov_pP.cu: occupancy of the single-run kernel, co-resident
// capacity for clusters of CL = 2 or 4 blocks, the single-run launch with
// clusters of cl blocks (1: plain cooperative launch), and the batched
// kernel for pt threads per block (64, 128, 256; nullptr otherwise; with
// pair, its spill-free form, pt = 128 only).
template <typename T, int P>
struct KrylovKernels {
    cudaError_t occupancy(int* per);
    int cluster_capacity(int CL);
    cudaError_t launch(const KrylovStepArgs& args, int blocks, int cl, cudaStream_t s);
    const void* batch_kernel(int pt, bool pair = false);
};
extern template struct KrylovKernels<double, 2>;
extern template struct KrylovKernels<float, 2>;
extern template struct KrylovKernels<double, 3>;
extern template struct KrylovKernels<float, 3>;
extern template struct KrylovKernels<double, 4>;
extern template struct KrylovKernels<float, 4>;

}  // namespace wrc
