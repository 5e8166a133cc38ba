// C ABI (include/wrc.h): run state on the device and the orchestration of one
// time step -- reconstruction, streamfunction, velocity and Smagorinsky
// forcing, Krylov projection with the phi_1 update, grid adaptation.
#include <algorithm>
#include <chrono>
#include <thread>
#include <atomic>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <cstdio>
#include <vector>
#include <cstring>
#include <string>
#include <type_traits>
#include <utility>

#include "../../include/wrc.h"
#include "batch.h"
#include "kernels.h"

using namespace wrc;

namespace {
std::atomic<long long> g_launches{0};
// While a CUDA graph is being captured on this thread, launches are only
// counted into the graph (and booked each time the graph is launched).
thread_local bool g_capturing = false;
thread_local long long g_captured = 0;
}

void wrc::note_launch() {
    if (g_capturing) ++g_captured;
    else g_launches.fetch_add(1, std::memory_order_relaxed);
}
long long wrc::launches_total() { return g_launches.load(std::memory_order_relaxed); }

namespace {

// Happy breakdown of the Arnoldi process: h_{j+1,j} <= tol |A v_j|.
constexpr double kBreakdownTol = 1e-12;

thread_local std::string g_create_error;

// Growable device buffer.  Plain cudaMalloc/cudaFree (not the stream-ordered
// allocator, whose reuse of memory freed on another run's stream can put a
// hidden inter-stream dependency in front of a graph capture); growth is
// rare, and the free waits for the buffer's stream first.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    cudaError_t grow(size_t need, size_t keep, cudaStream_t s) {
        if (need <= bytes) return cudaSuccess;
        void* q = nullptr;
        cudaError_t e = cudaMalloc(&q, need);
        if (e != cudaSuccess) return e;
        if (p && keep) {
            e = cudaMemcpyAsync(q, p, keep, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return e;
        }
        if (p) {
            e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return e;
            cudaFree(p);
        }
        p = q;
        bytes = need;
        return cudaSuccess;
    }
    void release(cudaStream_t s) {
        if (p) {
            cudaStreamSynchronize(s);
            cudaFree(p);
        }
        p = nullptr;
        bytes = 0;
    }
    template <typename T>
    T* as() const { return (T*)p; }
};

}  // namespace

struct wrc_run {
    wrc_config cfg{};
    Geom g{};
    cudaStream_t st = nullptr;
    int device = 0;
    std::string err;
    long long N = 0;   // NJ * NJ

    // bulk precision: double, or float for the mixed mode (FP64 stays in the
    // Krylov inner products, the Hessenberg matrix and phi_1)
    bool fp32 = false;
    size_t es = sizeof(double);

    // lattice arrays (bulk type)
    void* L = nullptr;       // omega on the grid / its reconstruction
    void* Lq = nullptr;      // Krylov vector on the grid + ghost values
    void* psi = nullptr;
    void* C1 = nullptr;      // FFT work arrays (complex) / Smagorinsky temporaries
    void* C2 = nullptr;
    DevBuf lat64;            // NJ*NJ doubles for conversions of lattice fields (mixed mode)
    uint8_t *act = nullptr, *nxt = nullptr, *gho = nullptr, *sig = nullptr, *JJ = nullptr;
    uint8_t* halo = nullptr;   // Smagorinsky halo mask (FP64 dynamic mode)
    int* list = nullptr;     // active points, then ghosts by level
    int* lat2idx = nullptr;  // lattice -> combined active/ghost number
    int *blk_counts = nullptr, *blk_off = nullptr, *counts_dev = nullptr;
    int* counts_host = nullptr;   // pinned
    int* flag_dev = nullptr;
    unsigned long long* lvl_dev = nullptr;
    double* vort_dev = nullptr;
    double* diag_dev = nullptr;
    PoissonPlan plan;

    // compact arrays (one entry per active point)
    DevBuf meta[2], omega[2], Ua, Va, ga, det, w, basis, tmp;
    int cur = 0;
    long long cap = 0;
    // ghost interpolation rows and the ghost values of the basis vectors
    DevBuf row_len, row_idx, row_w, Gb;
    DevBuf row_ready;   // cap_g + 1 ints: ready flags of the rows, the ghost counter
    DevBuf rows;        // NJ + 1 ints: flags of the row pairs of psi a step reads, their count and list
    bool rows_psi = false;   // psi of the last freeze holds only those rows
    long long cap_g = 0;

    // Krylov small arrays and cooperative-kernel scratch
    struct {
        double* H = nullptr;      // (m+1) x m
        double* beta = nullptr;   // [1]
        double* y = nullptr;      // [32]
        int* kstop = nullptr;     // ints: kstop, flags, err, pad, bar[2], counter, pad
        int* flags = nullptr;
        int* err = nullptr;
        int* overflow = nullptr;
        unsigned* bar = nullptr;
        unsigned* counter = nullptr;
        double* part = nullptr;   // partial sums of the cooperative kernel / diagnostics
    } K;
    int max_blocks = 1;

    // event timing of the Gram-Schmidt passes (wrc_profile)
    bool profiling = false;
    bool tracing = false;    // phase trace of the Krylov kernel (wrc_profile mode 2)
    DevBuf trace;
    int trace_nb = 0;        // blocks of the traced launch
    std::vector<cudaEvent_t> ev_pool;
    // CUDA graphs of the step phases, per phase and ping-pong parity; rebuilt
    // when a buffer they use is reallocated (layout) or eps changes
    struct Phase {
        cudaGraphExec_t exec = nullptr;
        long long layout = -1;
        long long kernels = 0;
    } graphs[3][2];
    long long layout = 0;
    bool use_graphs = false;
    struct ProfRec { int ev; double bytes, flops; };
    std::vector<ProfRec> ev_used;   // start-event index, algorithmic bytes and flops per launch
    // stage timing (wrc_profile mode 3): an event at each stage boundary of a
    // step, st_ids[i] the stage that starts at event i (kStageEnd closes the
    // step); folded into st_ms at the end of a step once many are pending
    bool stage_timing = false;
    bool in_step = false;
    std::vector<cudaEvent_t> st_pool;
    std::vector<int> st_ids;
    double st_ms[WRC_STAGE_COUNT] = {0};
    long long st_steps = 0;
    long long host_syncs = 0;

    // state
    long long n_active = 0, n_ghost = 0, det_count = 0;
    long long pend_na = 0, pend_ng = 0;   // counts of the grid being rebuilt
    long long gcount[16] = {0}, goff[16] = {0};
    double t = 0.0;
    long long nstep = 0;
    double updates = 0.0;   // sum of the active count over the steps taken
    bool nonfinite = false; // a step met a non-finite Arnoldi coefficient (seen at its grid rebuild)
    bool init = false, frozen = false;
    // bound of every device-side wait of the run's kernels (grid barriers of
    // the Krylov kernel), wrc_set_wait_limit
    unsigned long long wait_limit_ns = 2000000000ull;
    int cluster_max = 4;   // largest thread-block cluster of the Krylov launch (WRC_KRYLOV_CLUSTER at creation)
    int rmax = kGhostRowMax;   // longest ghost interpolation row (per DD order)
    cudaEvent_t sync_ev = nullptr;   // wrc_sync with a time limit

    // passive scalar (the vapour mixing ratio with diffusion only), enabled by
    // wrc_scalar_init: compact values on the grid, its reconstruction on the
    // lattice, and the small arrays of its Krylov step (H, beta, y; kstop)
    bool scalar = false;
    double kappa = 0.0;
    DevBuf rv[2], Lr, kr;
    // the scalar's Krylov problem runs beside omega's in one cooperative
    // launch: its own basis, work vector, ghost values, lattice vector,
    // partial sums and barrier words, and the launch's argument array and
    // block map (device, with a pinned host copy)
    DevBuf sbasis, sw, sGb, sLq, spart, sbar, sdev;
    void* shost = nullptr;
    size_t shost_bytes = 0;

    // exponential Rosenbrock step (wrc_config.scheme): U[q], V[q], D_x omega,
    // D_y omega at the active points (4 x cap, bulk type), the reductions'
    // partial sums, and coefficients / scales
    DevBuf jac, rbpart, rbsmall;

    // compressible velocity-Exner form (wrc_config.model = WRC_MODEL_EXNER):
    // u lives in the first field's slots (omega, L), v in the second's (rv,
    // Lr, as the passive scalar), pi in pe and Lp; the Krylov vectors stack
    // the three fields (xbasis (m + 1) x 3 cap, xw 3 cap); Lqx holds the
    // lattices of a Krylov vector's v and pi parts (Lq its u part), xd the
    // state's derivatives at the active points (8 x cap)
    bool exner = false;
    DevBuf pe[2], Lp, Lqx, xd, xbasis, xw;
};

namespace {

wrc_status fail(wrc_run* R, wrc_status s, const std::string& msg) {
    if (R) R->err = msg;
    return s;
}

#define CK(call)                                                                                \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return fail(R, e_ == cudaErrorMemoryAllocation ? WRC_ERR_OOM : WRC_ERR_CUDA,        \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                    \
    } while (0)

#define CKL(what)                                                                               \
    do {                                                                                        \
        cudaError_t e_ = cudaGetLastError();                                                    \
        if (e_ != cudaSuccess)                                                                  \
            return fail(R, WRC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e_));     \
    } while (0)

#define TRY(expr)                                                                               \
    do {                                                                                        \
        wrc_status s_ = (expr);                                                                 \
        if (s_ != WRC_OK) return s_;                                                            \
    } while (0)

// Run the internal function template fn for the run's bulk type.
#define DISPATCH(R, fn, ...) ((R)->fp32 ? fn<float>(__VA_ARGS__) : fn<double>(__VA_ARGS__))

double nu_eff(const wrc_run* R) {
    double nu = 1.0 / R->cfg.re;
    if (R->cfg.sgs == WRC_SGS_APRIORI) nu += (R->cfg.cs * R->g.h) * (R->cfg.cs * R->g.h) * R->cfg.s_apriori;
    return nu;
}

// 2 NJ*NJ doubles of device scratch: lattice conversions, and in the mixed mode the
// third and fourth FFT work arrays.
double* lattice_scratch(wrc_run* R) {
    if (R->lat64.grow(2 * sizeof(double) * R->N, 0, R->st) != cudaSuccess) return nullptr;
    return R->lat64.as<double>();
}

wrc_status ensure_capacity(wrc_run* R, long long n) {
    if (n <= R->cap) return WRC_OK;
    long long c = n + n / 4 + 1024;
    c = (c + 255) / 256 * 256;
    const int m = R->cfg.krylov_m;
    const cudaStream_t s = R->st;
    const size_t be = R->es * (size_t)c;
    // meta/omega of the current grid and the details keep their contents
    CK(R->meta[R->cur].grow(sizeof(uint32_t) * c, sizeof(uint32_t) * R->n_active, s));
    CK(R->meta[1 - R->cur].grow(sizeof(uint32_t) * c, 0, s));
    CK(R->omega[R->cur].grow(be, R->es * R->n_active, s));
    CK(R->omega[1 - R->cur].grow(be, 0, s));
    if (R->scalar || R->exner) {
        CK(R->rv[R->cur].grow(be, R->es * R->n_active, s));
        CK(R->rv[1 - R->cur].grow(be, 0, s));
    }
    if (R->exner) {
        CK(R->pe[R->cur].grow(be, R->es * R->n_active, s));
        CK(R->pe[1 - R->cur].grow(be, 0, s));
        CK(R->xd.grow(8 * be, 0, s));
        CK(R->xw.grow(3 * be, 0, s));
        R->xbasis.release(s);
        CK(R->xbasis.grow(3 * be * (size_t)(m + 1), 0, s));
    }
    CK(R->det.grow(be, R->es * R->det_count, s));
    CK(R->Ua.grow(be, 0, s));
    CK(R->Va.grow(be, 0, s));
    CK(R->ga.grow(be, 0, s));
    CK(R->w.grow(be, 0, s));
    CK(R->tmp.grow(sizeof(double) * (size_t)c, 0, s));   // doubles: conversions and queries
    if (R->cfg.scheme == WRC_SCHEME_ROSENBROCK) CK(R->jac.grow(4 * be, 0, s));
    // the basis is rebuilt every step; its leading dimension changes with c
    R->basis.release(s);
    CK(R->basis.grow(be * (size_t)(m + 1), 0, s));
    R->cap = c;
    R->layout += 1;
    return WRC_OK;
}

wrc_status ensure_ghost_capacity(wrc_run* R, long long ng) {
    if (ng <= R->cap_g && R->row_ready.p) return WRC_OK;   // the ready flags exist even for a grid without ghosts
    long long c = ng + ng / 4 + 1024;
    c = (c + 255) / 256 * 256;
    const cudaStream_t s = R->st;
    const int m = R->cfg.krylov_m;
    CK(R->row_len.grow(sizeof(int) * c, 0, s));
    CK(R->row_ready.grow(sizeof(int) * (c + 1), 0, s));
    CK(R->row_idx.grow(sizeof(int) * c * R->rmax, 0, s));
    CK(R->row_w.grow(sizeof(double) * c * R->rmax, 0, s));
    R->Gb.release(s);
    CK(R->Gb.grow(R->es * c * (m + 1), 0, s));
    R->cap_g = c;
    R->layout += 1;
    return WRC_OK;
}

// A grid rebuild in three parts.  Part 1 (device, capturable): the new grid
// is in `nxt` and its values in L; stencil levels, ghosts, compaction into
// the index list; the per-key counts and the error word go to pinned memory.
wrc_status rebuild_part1(wrc_run* R) {
    const Geom& g = R->g;
    const cudaStream_t s = R->st;
    CK(cudaMemsetAsync(R->gho, 0, R->N, s));
    launch_stencil_ghost(R->nxt, R->gho, R->JJ, g, s);
    for (int j = g.J; j >= 1; --j) launch_closure_level(R->gho, R->nxt, j, g, s);
    const int nkeys = g.J + 1;
    launch_compact(R->nxt, R->gho, g, nkeys, R->blk_counts, R->blk_off, R->counts_dev, R->list, s);
    CK(cudaMemcpyAsync(R->counts_host, R->counts_dev, sizeof(int) * nkeys, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(R->counts_host + kMaxKeys, R->K.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(R->counts_host + kMaxKeys + 1, R->K.flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    CKL("compaction");
    return WRC_OK;
}

// Host part: wait for the counts, report a Krylov-kernel error, grow buffers.
wrc_status rebuild_host(wrc_run* R) {
    const Geom& g = R->g;
    const cudaStream_t s = R->st;
    CK(cudaStreamSynchronize(s));
    R->host_syncs += 1;
    if (R->counts_host[kMaxKeys + 1] & 1) R->nonfinite = true;
    if (R->counts_host[kMaxKeys] != 0) {
        const int ev = R->counts_host[kMaxKeys];
        // bit 4: a clustered launch ran unclustered (its clusters were not
        // formed): plan the device's later launches without clusters
        if (ev & 16) krylov_clusters_unformed(R->device);
        if (ev == 16) {
            CK(cudaMemsetAsync(R->K.err, 0, sizeof(int), s));
        } else {
            CK(cudaMemsetAsync(R->K.err, 0, sizeof(int) * 4, s));   // err and the barrier words
            if (R->sbar.p) CK(cudaMemsetAsync(R->sbar.p, 0, R->sbar.bytes, s));   // the scalar problem's barrier
            if (ev & 4) return fail(R, WRC_ERR_STATE, "a ghost interpolation row exceeded its capacity of " +
                                                          std::to_string(R->rmax) + " terms");
            return fail(R, WRC_ERR_TIMEOUT,
                        "a bounded wait ran out (a grid barrier of the Krylov kernel, or a ghost's wait for a "
                        "coarser ghost's interpolation row); the run's state is undefined until it is "
                        "re-initialised (wrc_init_vortices, wrc_init_field, wrc_set_grid)");
        }
    }
    const long long na = R->counts_host[0];
    long long off = na, ng = 0;
    for (int j = 1; j <= g.J; ++j) {
        R->gcount[j] = R->counts_host[j];
        R->goff[j] = off;
        off += R->gcount[j];
        ng += R->gcount[j];
    }
    TRY(ensure_capacity(R, na));
    TRY(ensure_ghost_capacity(R, ng));
    R->pend_na = na;
    R->pend_ng = ng;
    return WRC_OK;
}

// Part 2 (device, capturable): compact arrays of the new grid and the ghost
// interpolation rows, all sizes read from the counts on the device.
template <typename T>
wrc_status rebuild_part2(wrc_run* R) {
    const cudaStream_t s = R->st;
    const int nc = 1 - R->cur;
    launch_finalize<T>(R->list, R->cap, R->JJ, (const T*)R->L, R->meta[nc].as<uint32_t>(), R->omega[nc].as<T>(), s,
                       R->counts_dev);
    if (R->scalar || R->exner)   // r_v (v) at the new grid from its lattice (meta is rewritten identically)
        launch_finalize<T>(R->list, R->cap, R->JJ, R->Lr.as<T>(), R->meta[nc].as<uint32_t>(), R->rv[nc].as<T>(), s,
                           R->counts_dev);
    if (R->exner)
        launch_finalize<T>(R->list, R->cap, R->JJ, R->Lp.as<T>(), R->meta[nc].as<uint32_t>(), R->pe[nc].as<T>(), s,
                           R->counts_dev);
    CK(cudaMemsetAsync(R->K.overflow, 0, sizeof(int), s));
    launch_ghost_rows(R->list, R->g.J, R->lat2idx, R->row_len.as<int>(), R->row_idx.as<int>(), R->row_w.as<double>(),
                      R->rmax, R->g, R->K.overflow, R->row_ready.as<int>(), R->K.err, R->wait_limit_ns, s,
                      R->counts_dev, R->cap, R->cap_g);
    CKL("finalize");
    return WRC_OK;
}

void rebuild_commit(wrc_run* R) {
    std::swap(R->act, R->nxt);
    R->cur = 1 - R->cur;
    R->n_active = R->pend_na;
    R->n_ghost = R->pend_ng;
    R->frozen = false;
}

// Run a phase: replay its CUDA graph for the current parity, capturing it
// first when missing or stale; without graphs (legacy default stream) issue
// the launches directly.
template <typename F>
wrc_status run_phase(wrc_run* R, int phase, F&& body) {
    if (!R->use_graphs || R->stage_timing) return body();
    auto& G = R->graphs[phase][R->cur];
    if (!G.exec || G.layout != R->layout) {
        if (G.exec) {
            CK(cudaStreamSynchronize(R->st));   // the stale graph may still be running
            cudaGraphExecDestroy(G.exec);
            G.exec = nullptr;
        }
        const cudaError_t pending = cudaGetLastError();
        if (pending != cudaSuccess)
            return fail(R, WRC_ERR_CUDA, std::string("error pending before capture of phase ") +
                                             std::to_string(phase) + ": " + cudaGetErrorString(pending));
        CK(cudaStreamBeginCapture(R->st, cudaStreamCaptureModeRelaxed));
        g_capturing = true;
        g_captured = 0;
        const wrc_status st = body();
        g_capturing = false;
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(R->st, &graph);
        if (st != WRC_OK) {
            if (graph) cudaGraphDestroy(graph);
            R->err = "capture of phase " + std::to_string(phase) + " (parity " + std::to_string(R->cur) +
                     "): " + R->err + " / end capture: " + cudaGetErrorString(ec);
            return st;
        }
        CK(ec);
        const cudaError_t ei = cudaGraphInstantiate(&G.exec, graph, 0);
        cudaGraphDestroy(graph);
        CK(ei);
        G.layout = R->layout;
        G.kernels = g_captured;
    }
    CK(cudaGraphLaunch(G.exec, R->st));
    g_launches.fetch_add(G.kernels, std::memory_order_relaxed);
    return WRC_OK;
}

constexpr int kStageEnd = WRC_STAGE_COUNT;

// Stage timing: record the start of stage `id` (kStageEnd: the step's end) on
// the run's stream.  A no-op unless wrc_profile mode 3 is on and a step is
// being taken (the step's phases then run as direct launches).
wrc_status stage_mark(wrc_run* R, int id) {
    if (!R->stage_timing || !R->in_step) return WRC_OK;
    const size_t i = R->st_ids.size();
    while (R->st_pool.size() <= i) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        R->st_pool.push_back(e);
    }
    CK(cudaEventRecord(R->st_pool[i], R->st));
    R->st_ids.push_back(id);
    return WRC_OK;
}

// Add the recorded intervals to the per-stage totals (synchronises): the
// interval from event i to event i + 1 belongs to stage st_ids[i], except
// after a step's end.
wrc_status stage_fold(wrc_run* R) {
    if (R->st_ids.empty()) return WRC_OK;
    CK(cudaStreamSynchronize(R->st));
    for (size_t i = 0; i < R->st_ids.size(); ++i) {
        if (R->st_ids[i] == kStageEnd) {
            R->st_steps += 1;
            continue;
        }
        if (i + 1 == R->st_ids.size()) break;
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, R->st_pool[i], R->st_pool[i + 1]));
        R->st_ms[R->st_ids[i]] += t;
    }
    R->st_ids.clear();
    return WRC_OK;
}

// Thresholding with eps: details of the values in L on the current grid (or
// on every lattice point for a freshly sampled field), significance and
// adjacent zone into nxt, closure.  The details read only the grid's values
// (its predictor points are in the closed grid).
template <typename T>
wrc_status threshold_marks(wrc_run* R, double eps, bool whole_lattice) {
    const Geom& g = R->g;
    const cudaStream_t s = R->st;
    CK(cudaMemsetAsync(R->sig, 0, R->N, s));
    CK(cudaMemsetAsync(R->nxt, 0, R->N, s));
    if (whole_lattice)
        launch_details_adj<T>(nullptr, R->N, (const T*)R->L, eps, nullptr, R->sig, R->nxt, g, s);
    else
        launch_details_adj<T>(R->meta[R->cur].as<uint32_t>(), R->cap, (const T*)R->L, eps, R->det.as<T>(), R->sig,
                              R->nxt, g, s, R->counts_dev);
    if (R->scalar && !whole_lattice)   // the grid adapts to r_v as well: union of the significant sets
        launch_details_adj<T>(R->meta[R->cur].as<uint32_t>(), R->cap, R->Lr.as<T>(), eps, nullptr, R->sig, R->nxt, g,
                              s, R->counts_dev);
    if (R->exner) {   // the grid adapts to u (L), v (Lr) and pi (Lp): union of the significant sets
        for (T* F : {R->Lr.as<T>(), R->Lp.as<T>()}) {
            if (whole_lattice) launch_details_adj<T>(nullptr, R->N, F, eps, nullptr, R->sig, R->nxt, g, s);
            else
                launch_details_adj<T>(R->meta[R->cur].as<uint32_t>(), R->cap, F, eps, nullptr, R->sig, R->nxt, g, s,
                                      R->counts_dev);
        }
    }
    for (int j = g.J; j >= 1; --j) launch_closure_level(R->nxt, nullptr, j, g, s);
    CKL("threshold");
    return WRC_OK;
}

// Thresholding and the first part of the rebuild (L holds the values on the
// whole lattice, or at least at every point of the new grid).
template <typename T>
wrc_status threshold_body(wrc_run* R, double eps, bool whole_lattice) {
    TRY(threshold_marks<T>(R, eps, whole_lattice));
    return rebuild_part1(R);
}

// Adaptation after a step (Eq. 6), first part: L (and Lr with the passive
// scalar) holds the new values at the current grid's points.  Details,
// threshold, adjacent zone and closure give the new grid in nxt; the values
// at its new points come from the reconstruction on the current grid,
// evaluated only there (coarse to fine); then the rebuild's first part.
template <typename T>
wrc_status adapt_part1(wrc_run* R) {
    TRY(stage_mark(R, WRC_STAGE_ADAPT));
    TRY(threshold_marks<T>(R, R->cfg.eps, false));
    TRY(stage_mark(R, WRC_STAGE_RECONSTRUCT));
    launch_recon_new<T>((T*)R->L, R->act, R->nxt, R->g, R->st);
    if (R->scalar || R->exner) launch_recon_new<T>(R->Lr.as<T>(), R->act, R->nxt, R->g, R->st);
    if (R->exner) launch_recon_new<T>(R->Lp.as<T>(), R->act, R->nxt, R->g, R->st);
    CKL("new values");
    TRY(stage_mark(R, WRC_STAGE_ADAPT));
    return rebuild_part1(R);
}

template <typename T>
wrc_status rebuild_from_mask(wrc_run* R) {
    TRY(rebuild_part1(R));
    TRY(rebuild_host(R));
    TRY(rebuild_part2<T>(R));
    rebuild_commit(R);
    return WRC_OK;
}

template <typename T>
wrc_status threshold_current(wrc_run* R, double eps, bool whole_lattice) {
    TRY(threshold_body<T>(R, eps, whole_lattice));
    R->det_count = whole_lattice ? 0 : R->n_active;
    TRY(rebuild_host(R));
    TRY(rebuild_part2<T>(R));
    rebuild_commit(R);
    return WRC_OK;
}

// L <- R(omega): the grid values, then coarse-to-fine prediction elsewhere.
// With rows, the flags R->rows of the row pairs within 2 dd_reach(P) rows of
// a grid point are set as well: the rows of psi a step reads (the velocity
// stencils at the grid points, and the SGS halo, dd_reach(P) around them,
// with its own stencils).
template <typename T>
wrc_status reconstruct(wrc_run* R, bool rows = false) {
    if (rows) CK(cudaMemsetAsync(R->rows.p, 0, R->rows.bytes, R->st));
    launch_scatter<T>(R->meta[R->cur].as<uint32_t>(), R->omega[R->cur].as<T>(), R->cap, (T*)R->L, R->st,
                      R->counts_dev, rows ? R->rows.as<int>() : nullptr, 2 * dd_reach(R->g.P), &R->g);
    CKL("reconstruct/scatter");
    launch_reconstruct<T>((T*)R->L, R->act, R->g, R->st);
    CKL("reconstruct");
    return WRC_OK;
}

// Lr <- R(r_v), as reconstruct does for omega.
template <typename T>
wrc_status reconstruct_scalar(wrc_run* R) {
    launch_scatter<T>(R->meta[R->cur].as<uint32_t>(), R->rv[R->cur].as<T>(), R->cap, R->Lr.as<T>(), R->st,
                      R->counts_dev);
    launch_reconstruct<T>(R->Lr.as<T>(), R->act, R->g, R->st);
    CKL("reconstruct scalar");
    return WRC_OK;
}

// Linearisation at the current state: R(omega), psi, U, V and the SGS forcing
// (and R(r_v) when the passive scalar is on).  In a step the inverse row
// passes of the Poisson solve run only on the rows the step reads
// (rows_psi): psi there (FP64), or U, V and the strain (FP32 bulk); the
// field queries want all of it.
template <typename T>
wrc_status freeze(wrc_run* R, bool in_step = false) {
    TRY(stage_mark(R, WRC_STAGE_RECONSTRUCT));
    R->rows_psi = in_step;
    TRY(reconstruct<T>(R, R->rows_psi));
    CKL("freeze/reconstruct");
    if (R->scalar) TRY(reconstruct_scalar<T>(R));
    TRY(stage_mark(R, WRC_STAGE_POISSON));
    const cudaStream_t s = R->st;
    const uint32_t* meta = R->meta[R->cur].as<uint32_t>();
    T* t0 = (T*)R->C1;
    T* t1 = t0 + R->N;
    T* t2 = (T*)R->C2;
    T* t3 = t2 + R->N;
    if (R->fp32) {
        // FP32 bulk: U = D_y psi, V = -D_x psi and the strain S11, S12 come
        // from the spectrum, because finest-lattice stencils on an FP32 psi
        // cancel 2 (first derivatives) to 5 (second derivatives) digits away.
        double* scr = lattice_scratch(R);
        if (!scr) return fail(R, WRC_ERR_OOM, "lattice scratch");
        const bool dyn = R->cfg.sgs == WRC_SGS_DYNAMIC;
        T* S11 = t2;
        T* S12 = t3;
        launch_poisson<T>(R->plan, (const T*)R->L, (T*)R->psi, R->C1, R->C2, R->g, s, (T*)R->Lq, t0, scr,
                          dyn ? S11 : nullptr, dyn ? S12 : nullptr, dyn ? (void*)(scr + R->N) : nullptr,
                          R->rows_psi ? R->rows.as<int>() : nullptr);
        CKL("freeze/poisson");
        TRY(stage_mark(R, WRC_STAGE_VELOCITY));
        launch_velocity_gather<T>((const T*)R->Lq, t0, meta, R->cap, R->Ua.as<T>(), R->Va.as<T>(), s, R->counts_dev);
        CKL("freeze/velocity");
        TRY(stage_mark(R, WRC_STAGE_SGS));
        if (dyn)
            launch_sgs_from_strain<T>(S11, S12, meta, R->cap, R->cfg.cs, R->ga.as<T>(), t1, t0, (T*)scr, R->g, s,
                                      R->counts_dev, R->rows_psi ? R->rows.as<int>() : nullptr);
        CKL("freeze");
        R->frozen = true;
        return WRC_OK;
    } else {
        launch_poisson<T>(R->plan, (const T*)R->L, (T*)R->psi, R->C1, R->C2, R->g, s, nullptr, nullptr, nullptr,
                          nullptr, nullptr, nullptr, R->rows_psi ? R->rows.as<int>() : nullptr);
        TRY(stage_mark(R, WRC_STAGE_VELOCITY));
        launch_velocity_active<T>((const T*)R->psi, meta, R->cap, R->Ua.as<T>(), R->Va.as<T>(), R->g, s,
                                  R->counts_dev);
    }
    TRY(stage_mark(R, WRC_STAGE_SGS));
    if (R->cfg.sgs == WRC_SGS_DYNAMIC)
        // t0, t1 (the first work array, free after the Poisson solve here) hold the halo list
        launch_sgs_halo<T>((const T*)R->psi, meta, R->cap, R->cfg.cs, R->ga.as<T>(), t2, t3, R->halo, (int*)t0, R->g,
                           s, R->counts_dev);
    CKL("freeze");
    R->frozen = true;
    return WRC_OK;
}

template <typename T>
void ghost_fill(wrc_run* R, T* F, const int* kstop, int jstep) {
    for (int j = 1; j <= R->g.J; ++j)
        launch_ghost_fill<T>(F, R->list + R->goff[j], R->gcount[j], j, R->g, kstop, jstep, R->st);
}

// Algorithmic bytes of one Krylov step over n active points with Krylov
// dimension k (FP64 words): k + 1 operator applications reading q, U, V and
// writing w; at Arnoldi step j a fused single Gram-Schmidt pass reading j + 1
// basis vectors and w twice and writing w; the combination reading k vectors
// and omega and writing omega.
double krylov_algorithmic_bytes(long long n, int k) {
    double words = 4.0 * (k + 1) + (double)k + 2.0;
    for (int j = 0; j < k; ++j) words += 2.0 * (j + 1) + 3.0;
    return 8.0 * words * (double)n;
}

// Algorithmic FP64 operations of the same step per active point: 30 per
// operator application (k + 1 of them), at Arnoldi step j two Gram-Schmidt
// passes of dots and updates, 8 (j + 1), plus 4 for the norms, one division
// per normalised entry, and 2 k for the combination.
double krylov_algorithmic_flops(long long n, int k) {
    double f = 30.0 * (k + 1) + 3.0 * k;
    for (int j = 0; j < k; ++j) f += 8.0 * (j + 1) + 4.0;
    return f * (double)n;
}

// Arguments of the Krylov step of run R (its current grid and buffers).
KrylovStepArgs krylov_args(wrc_run* R) {
    const long long n = R->n_active;
    const int m = R->cfg.krylov_m;
    KrylovStepArgs A{};
    A.g = R->g;
    A.meta = R->meta[R->cur].as<uint32_t>();
    A.n = (int)n;
    A.glist = R->list + n;
    A.ng = (int)R->n_ghost;
    A.row_len = R->row_len.as<int>();
    A.row_idx = R->row_idx.as<int>();
    A.row_w = R->row_w.as<double>();
    A.rmax = R->rmax;
    A.row_overflow = R->K.overflow;
    A.Gb = R->Gb.p;
    A.ldg = R->cap_g;
    A.Ua = R->Ua.p;
    A.Va = R->Va.p;
    A.ga = R->cfg.sgs == WRC_SGS_DYNAMIC ? R->ga.p : nullptr;
    A.nu = nu_eff(R);
    A.r = R->cfg.rayleigh_r;
    A.c1J = 1.0 / (dd_d1den(R->g.P) * R->g.h);
    A.c2J = 1.0 / (dd_d2den(R->g.P) * R->g.h * R->g.h);
    A.L = R->L;
    A.Lq = R->Lq;
    A.omega = R->omega[R->cur].p;
    A.basis = R->basis.p;
    A.ld = R->cap;
    A.w = R->w.p;
    A.H = R->K.H;
    A.y = R->K.y;
    A.beta = R->K.beta;
    A.kstop = R->K.kstop;
    A.flags = R->K.flags;
    A.part = R->K.part;
    A.bar = R->K.bar;
    A.err = R->K.err;
    A.m = m;
    A.dt = R->cfg.dt;
    A.tol = kBreakdownTol;
    A.limit_ns = R->wait_limit_ns;
    A.trace = R->tracing ? R->trace.as<unsigned long long>() : nullptr;
    return A;
}

// Arguments of the Krylov step of the passive scalar: the same grid,
// velocity and workspace, the operator -U Dx - V Dy + kappa (Dxx + Dyy) (no
// Rayleigh friction, no subgrid forcing), its values and lattice, and its own
// small arrays (the vorticity step's H, beta, y and k stay queryable).
KrylovStepArgs krylov_args_scalar(wrc_run* R) {
    KrylovStepArgs A = krylov_args(R);
    const int m = R->cfg.krylov_m;
    double* d = R->kr.as<double>();
    A.ga = nullptr;
    A.nu = R->kappa;
    A.r = 0.0;
    A.L = R->Lr.p;
    A.omega = R->rv[R->cur].p;
    A.H = d;
    A.beta = d + (size_t)(m + 1) * m;
    A.y = A.beta + 1;
    A.kstop = (int*)(A.y + 32);
    A.trace = nullptr;
    return A;
}

// The Krylov steps of omega and of the passive scalar as two problems of one
// cooperative launch of the batched kernel (each with half of the co-resident
// blocks, its own grid barrier and workspace), so that the latency-bound
// phases of one overlap the FP64 work of the other.  The scalar's workspace
// grows with the grid here.
template <typename T>
wrc_status krylov_pair(wrc_run* R, const KrylovStepArgs& A) {
    const cudaStream_t s = R->st;
    const int m = R->cfg.krylov_m;
    constexpr int kPairPT = 128;   // threads per block of the batched kernel
    const int maxb = krylov_batch_max_blocks(R->fp32, R->g.P, kPairPT, true);
    if (maxb < 2) return fail(R, WRC_ERR_CUDA, "batched Krylov kernel occupancy query failed");
    CK(R->sbasis.grow(R->es * (size_t)R->cap * (m + 1), 0, s));
    CK(R->sw.grow(R->es * (size_t)R->cap, 0, s));
    CK(R->sGb.grow(R->es * (size_t)(R->cap_g > 0 ? R->cap_g : 1) * (m + 1), 0, s));
    CK(R->sLq.grow(R->es * (size_t)R->N, 0, s));
    CK(R->spart.grow(sizeof(double) * krylov_partials_doubles(maxb), 0, s));
    if (!R->sbar.p) {
        CK(R->sbar.grow(sizeof(unsigned) * 4, 0, s));
        CK(cudaMemsetAsync(R->sbar.p, 0, R->sbar.bytes, s));
    }
    KrylovStepArgs B = krylov_args_scalar(R);
    B.basis = R->sbasis.p;
    B.w = R->sw.p;
    B.Gb = R->sGb.p;
    B.Lq = R->sLq.p;
    B.part = R->spart.as<double>();
    B.bar = R->sbar.as<unsigned>();
    const long long need = (R->n_active + kPairPT - 1) / kPairPT;
    const int each = (int)std::max(1LL, std::min(need, (long long)(maxb / 2)));
    const int total = 2 * each;
    const size_t bytes = 2 * sizeof(KrylovStepArgs) + sizeof(int) * (total + 3);
    CK(R->sdev.grow(bytes, 0, s));
    if (R->shost_bytes < bytes) {
        CK(cudaStreamSynchronize(s));   // the last copy from the old staging buffer
        if (R->shost) cudaFreeHost(R->shost);
        R->shost = nullptr;
        R->shost_bytes = 0;
        CK(cudaMallocHost(&R->shost, bytes));
        R->shost_bytes = bytes;
    }
    KrylovStepArgs* ha = (KrylovStepArgs*)R->shost;
    ha[0] = A;
    ha[1] = B;
    int* blk = (int*)(ha + 2);
    for (int b = 0; b < total; ++b) blk[b] = b < each ? 0 : 1;
    blk[total] = 0;
    blk[total + 1] = each;
    blk[total + 2] = total;
    if (R->tracing) R->trace_nb = each;
    CK(cudaMemcpyAsync(R->sdev.p, R->shost, bytes, cudaMemcpyHostToDevice, s));
    const KrylovStepArgs* da = (const KrylovStepArgs*)R->sdev.p;
    const int* dblk = (const int*)(da + 2);
    CK(launch_krylov_batch<T>(da, dblk, dblk + total, 2, total, kPairPT, R->g.P, s, true));
    return WRC_OK;
}

// Clear the phase trace before a traced launch (on the run's stream).
wrc_status trace_reset(wrc_run* R, int nb) {
    if (!R->tracing) return WRC_OK;
    R->trace_nb = nb;
    CK(cudaMemsetAsync(R->trace.p, 0, R->trace.bytes, R->st));
    return WRC_OK;
}

template <typename T>
wrc_status krylov_rosenbrock(wrc_run* R);

// Arnoldi + phi_1 + update for the frozen linearisation (L holds R(omega)),
// one cooperative launch.
template <typename T>
wrc_status krylov(wrc_run* R) {
    const cudaStream_t s = R->st;
    const long long n = R->n_active;
    const int m = R->cfg.krylov_m;
    const KrylovStepArgs A = krylov_args(R);
    const int blocks = krylov_step_blocks(n, R->max_blocks, R->fp32, R->g.P, R->device, R->cluster_max);
    TRY(trace_reset(R, blocks));
    int e0 = -1;
    if (R->profiling) {
        while (R->ev_pool.size() < R->ev_used.size() * 2 + 2) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e));
            R->ev_pool.push_back(e);
        }
        e0 = (int)R->ev_used.size() * 2;
        CK(cudaEventRecord(R->ev_pool[e0], s));
    }
    const bool pair = R->scalar && R->cfg.scheme != WRC_SCHEME_ROSENBROCK;
    if (R->cfg.scheme == WRC_SCHEME_ROSENBROCK) TRY(krylov_rosenbrock<T>(R));
    else if (pair) TRY(krylov_pair<T>(R, A));
    else CK(launch_krylov_step<T>(A, blocks, s, R->device, R->cluster_max));
    if (R->profiling) {
        CK(cudaEventRecord(R->ev_pool[e0 + 1], s));
        const double f = pair ? 2.0 : 1.0;
        R->ev_used.push_back({e0, f * krylov_algorithmic_bytes(n, m), f * krylov_algorithmic_flops(n, m)});
    }
    if (R->scalar && !pair) CK(launch_krylov_step<T>(krylov_args_scalar(R), blocks, s, R->device, R->cluster_max));
    return WRC_OK;
}

// The exponential Rosenbrock-Euler step (WRC_SCHEME_ROSENBROCK; Sec. 1 and
// 2.1 with the full Jacobian of the advection): after the freeze (L holds
// R(omega), U, V and g at the active points), D omega at the active points,
// b = A_n omega + g, then m Arnoldi steps, each applying J_n to q_j -- R(q_j)
// on the lattice by the inverse transform, psi[q_j] by the Poisson solve,
// U[q_j], V[q_j] at the active points -- followed by classical Gram-Schmidt
// twice with FP64 inner products; phi_1 and the update.  Launches only (no
// host synchronisation); a breakdown is decided on the device.
template <typename T>
wrc_status krylov_rosenbrock(wrc_run* R) {
    const cudaStream_t s = R->st;
    const long long n = R->n_active;
    const int m = R->cfg.krylov_m;
    const Geom& g = R->g;
    const uint32_t* meta = R->meta[R->cur].as<uint32_t>();
    CK(R->jac.grow(4 * R->es * (size_t)R->cap, 0, s));
    CK(R->rbpart.grow(sizeof(double) * kRbPartBlocks * kRbPartWidth, 0, s));
    CK(R->rbsmall.grow(sizeof(double) * 64, 0, s));
    T* jb = R->jac.as<T>();
    RbArgs a{};
    a.g = g;
    a.meta = meta;
    a.n = (int)n;
    a.L = R->L;
    a.Lq = R->Lq;
    a.Ua = R->Ua.p;
    a.Va = R->Va.p;
    a.Uq = jb;
    a.Vq = jb + R->cap;
    a.dwx = jb + 2 * R->cap;
    a.dwy = jb + 3 * R->cap;
    a.w = R->w.p;
    a.basis = R->basis.p;
    a.ld = R->cap;
    a.omega = R->omega[R->cur].p;
    a.part = R->rbpart.as<double>();
    a.coef = R->rbsmall.as<double>();
    a.sc = a.coef + 32;
    a.H = R->K.H;
    a.y = R->K.y;
    a.beta = R->K.beta;
    a.kstop = R->K.kstop;
    a.flags = R->K.flags;
    a.m = m;
    a.dt = R->cfg.dt;
    a.tol = kBreakdownTol;
    a.nu = nu_eff(R);
    a.r = R->cfg.rayleigh_r;
    a.c1J = 1.0 / (dd_d1den(g.P) * g.h);
    a.c2J = 1.0 / (dd_d2den(g.P) * g.h * g.h);
    T* Lq = (T*)R->Lq;
    T* Uq = (T*)a.Uq;
    T* Vq = (T*)a.Vq;
    double* scr = R->fp32 ? lattice_scratch(R) : nullptr;
    if (R->fp32 && !scr) return fail(R, WRC_ERR_OOM, "lattice scratch");
    CK(cudaMemsetAsync(R->K.H, 0, sizeof(double) * (m + 1) * m, s));
    CK(rb_gradient<T>(a, s));
    // b = A_n omega + g = F(omega^n), then beta and v_0
    launch_matvec<T>((const T*)R->L, meta, n, R->Ua.as<T>(), R->Va.as<T>(),
                     R->cfg.sgs == WRC_SGS_DYNAMIC ? R->ga.as<T>() : nullptr, a.nu, a.r, (T*)a.w, g, nullptr, 0, s);
    CKL("rosenbrock b");
    CK(rb_reduce<T>(a, 0, true, 3, -1, s));
    CK(rb_scale<T>(a, -1, s));
    for (int j = 0; j < m; ++j) {
        // R(q_j) on the lattice (its ghost values included), psi[q_j], U[q_j], V[q_j]
        launch_scatter<T>(meta, R->basis.as<T>() + (size_t)j * R->cap, n, Lq, s);
        launch_reconstruct<T>(Lq, R->act, g, s);
        if (R->fp32) {
            // spectral U, V (as in the freeze): U into the second half of the
            // scratch (the first holds the third FFT work array), V into C1
            T* Ulat = (T*)(scr + R->N);
            launch_poisson<T>(R->plan, Lq, (T*)R->psi, R->C1, R->C2, g, s, Ulat, (T*)R->C1, scr, nullptr, nullptr,
                              nullptr, R->rows_psi ? R->rows.as<int>() : nullptr);
            launch_velocity_gather<T>(Ulat, (const T*)R->C1, meta, n, Uq, Vq, s);
        } else {
            // psi[q_j] at the rows the velocity stencils read (flagged by the freeze)
            launch_poisson<T>(R->plan, Lq, (T*)R->psi, R->C1, R->C2, g, s, nullptr, nullptr, nullptr, nullptr,
                              nullptr, nullptr, R->rows_psi ? R->rows.as<int>() : nullptr);
            launch_velocity_active<T>((const T*)R->psi, meta, n, Uq, Vq, g, s);
        }
        CKL("rosenbrock jacobian");
        CK(rb_apply<T>(a, j, s));
        CK(rb_reduce<T>(a, j + 1, true, 0, j, s));
        CK(rb_axpy<T>(a, j + 1, j, s));
        CK(rb_reduce<T>(a, j + 1, false, 1, j, s));
        CK(rb_axpy<T>(a, j + 1, j, s));
        CK(rb_reduce<T>(a, 0, true, 2, j, s));
        CK(rb_scale<T>(a, j, s));
    }
    CK(rb_finish<T>(a, s));
    return WRC_OK;
}

// Arguments of the velocity-Exner launches on the run's current grid.
ExArgs exner_args(wrc_run* R) {
    ExArgs a{};
    a.g = R->g;
    a.meta = R->meta[R->cur].as<uint32_t>();
    a.n = (int)R->n_active;
    a.glist = R->list + R->n_active;
    a.ng = (int)R->n_ghost;
    a.row_len = R->row_len.as<int>();
    a.row_idx = R->row_idx.as<int>();
    a.row_w = R->row_w.as<double>();
    a.rmax = R->rmax;
    a.Lb[0] = (double*)R->L;
    a.Lb[1] = R->Lr.as<double>();
    a.Lb[2] = R->Lp.as<double>();
    a.Lq[0] = (double*)R->Lq;
    a.Lq[1] = R->Lqx.as<double>();
    a.Lq[2] = R->Lqx.as<double>() + R->N;
    a.f[0] = a.f_out[0] = R->omega[R->cur].as<double>();
    a.f[1] = a.f_out[1] = R->rv[R->cur].as<double>();
    a.f[2] = a.f_out[2] = R->pe[R->cur].as<double>();
    a.d = R->xd.as<double>();
    a.ld = R->cap;
    a.C = R->cfg.cpt;
    a.fc = R->cfg.coriolis;
    a.gx = R->cfg.gx;
    a.gy = R->cfg.gy;
    a.r = R->cfg.rayleigh_r;
    a.nu = nu_eff(R);
    a.c1J = 1.0 / (dd_d1den(R->g.P) * R->g.h);
    a.c2J = 1.0 / (dd_d2den(R->g.P) * R->g.h * R->g.h);
    a.full = R->cfg.scheme == WRC_SCHEME_ROSENBROCK;
    return a;
}

// The Krylov part of a velocity-Exner step (Eqs. 1-2): the state's lattices
// (active and ghost values) and derivatives and b = F(U^n), then the Arnoldi
// process on the stacked vectors [u; v; pi] (classical Gram-Schmidt twice,
// FP64 partial sums added in a fixed order, breakdown on the device), phi_1
// and the update in one persistent cooperative launch.  FP64 only.
wrc_status exner_krylov(wrc_run* R) {
    const cudaStream_t s = R->st;
    const long long n = R->n_active;
    const int m = R->cfg.krylov_m;
    const int maxb = ex_krylov_max_blocks(R->g.P);
    if (maxb < 1) return fail(R, WRC_ERR_CUDA, "velocity-Exner Krylov kernel occupancy query failed");
    const int blocks =
        (int)std::max(1LL, std::min((long long)maxb, (3 * n + kExKrylovThreads - 1) / kExKrylovThreads));
    CK(R->rbpart.grow(sizeof(double) * (size_t)maxb * kExPartWidth, 0, s));
    const ExArgs a = exner_args(R);
    ExKrylov K{};
    K.basis = R->xbasis.as<double>();
    K.ld3 = 3 * R->cap;
    K.w = R->xw.as<double>();
    K.part = R->rbpart.as<double>();
    K.H = R->K.H;
    K.y = R->K.y;
    K.beta = R->K.beta;
    K.kstop = R->K.kstop;
    K.flags = R->K.flags;
    K.bar = R->K.bar;
    K.err = R->K.err;
    K.limit_ns = R->wait_limit_ns;
    K.m = m;
    K.dt = R->cfg.dt;
    K.tol = kBreakdownTol;
    double* const Lb[3] = {a.Lb[0], a.Lb[1], a.Lb[2]};
    const double* const fs[3] = {a.f[0], a.f[1], a.f[2]};
    CK(cudaMemsetAsync(R->K.H, 0, sizeof(double) * (m + 1) * m, s));
    CK(ex_scatter_fields(a, fs, Lb, nullptr, 0, s));
    CK(ex_base(a, K.w, s));
    CK(ex_krylov(a, K, blocks, s));
    return WRC_OK;
}

enum { kPhaseFreeze = 0, kPhaseAdapt1 = 1, kPhaseAdapt2 = 2 };

// One time step: [freeze] -> Krylov launch -> [adapt part 1] -> host sync for
// the new grid's sizes -> [adapt part 2]; bracketed phases run as CUDA graphs.
template <typename T>
wrc_status step_phases(wrc_run* R) {
    if (R->exner) {
        TRY(stage_mark(R, WRC_STAGE_KRYLOV));
        TRY(exner_krylov(R));
    } else {
        TRY(run_phase(R, kPhaseFreeze, [&] { return freeze<T>(R, true); }));
        R->frozen = true;
        TRY(stage_mark(R, WRC_STAGE_KRYLOV));
        TRY(krylov<T>(R));
    }
    // L holds omega^{n+1} at the grid points (Lr r_v^{n+1}); threshold, then
    // the values at the new grid's new points
    TRY(run_phase(R, kPhaseAdapt1, [&] { return adapt_part1<T>(R); }));
    R->det_count = R->n_active;
    TRY(stage_mark(R, WRC_STAGE_HOST));
    TRY(rebuild_host(R));
    TRY(stage_mark(R, WRC_STAGE_ADAPT));
    TRY(run_phase(R, kPhaseAdapt2, [&] { return rebuild_part2<T>(R); }));
    TRY(stage_mark(R, kStageEnd));
    rebuild_commit(R);
    return WRC_OK;
}

template <typename T>
wrc_status step_once(wrc_run* R) {
    const long long na0 = R->n_active;
    const size_t m0 = R->st_ids.size();
    R->in_step = true;
    const wrc_status st = step_phases<T>(R);
    R->in_step = false;
    if (st != WRC_OK) {
        R->st_ids.resize(m0);   // a step that failed leaves no stage intervals
        return st;
    }
    if (R->st_ids.size() >= 1024) TRY(stage_fold(R));
    R->t += R->cfg.dt;
    R->nstep += 1;
    R->updates += (double)na0;
    return WRC_OK;
}

wrc_status check_ready(wrc_run* R) {
    if (!R) return WRC_ERR_ARG;
    if (!R->init) return fail(R, WRC_ERR_STATE, "run has no initial condition");
    return WRC_OK;
}

// Calls of the vorticity form only.
wrc_status vorticity_only(wrc_run* R, const char* fn) {
    if (R && R->exner) return fail(R, WRC_ERR_STATE, std::string(fn) + " does not apply to a velocity-Exner run");
    return WRC_OK;
}

wrc_status copy_out(wrc_run* R, void* dst, const void* src, size_t bytes, int device_ptr) {
    if (!bytes) return WRC_OK;
    CK(cudaMemcpyAsync(dst, src, bytes, device_ptr ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, R->st));
    return WRC_OK;
}

wrc_status copy_in(wrc_run* R, void* dst, const void* src, size_t bytes, int device_ptr) {
    if (!bytes) return WRC_OK;
    CK(cudaMemcpyAsync(dst, src, bytes, device_ptr ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, R->st));
    return WRC_OK;
}

// n values of the bulk type (device) out to doubles (host or device); FP32
// values are widened in `scratch` (device, >= n doubles) first.
template <typename T>
wrc_status out_as_double(wrc_run* R, double* dst, const T* src, long long n, int device_ptr, double* scratch) {
    if constexpr (std::is_same<T, double>::value) {
        (void)scratch;
        return copy_out(R, dst, src, sizeof(double) * n, device_ptr);
    } else {
        launch_convert<float, double>(src, scratch, n, R->st);
        CKL("convert");
        return copy_out(R, dst, scratch, sizeof(double) * n, device_ptr);
    }
}

// n doubles (host or device) into the bulk type on the device.
template <typename T>
wrc_status in_from_double(wrc_run* R, T* dst, const double* src, long long n, int device_ptr, double* scratch) {
    if constexpr (std::is_same<T, double>::value) {
        (void)scratch;
        return copy_in(R, dst, src, sizeof(double) * n, device_ptr);
    } else {
        TRY(copy_in(R, scratch, src, sizeof(double) * n, device_ptr));
        launch_convert<double, float>(scratch, dst, n, R->st);
        CKL("convert");
        return WRC_OK;
    }
}

template <typename T>
wrc_status init_field_t(wrc_run* R, const double* omega_lattice, int device_ptr) {
    double* scr = R->fp32 ? lattice_scratch(R) : nullptr;
    if (R->fp32 && !scr) return fail(R, WRC_ERR_OOM, "lattice scratch");
    TRY(in_from_double<T>(R, (T*)R->L, omega_lattice, R->N, device_ptr, scr));
    CK(cudaMemsetAsync(R->act, 1, R->N, R->st));
    R->n_active = 0;
    return threshold_current<T>(R, R->cfg.eps, true);
}

// Velocity-Exner initial condition: u, v, pi on the whole lattice in L, Lr,
// Lp; the joint thresholding of their full-lattice transforms.
wrc_status exner_threshold_whole(wrc_run* R) {
    CK(cudaMemsetAsync(R->act, 1, R->N, R->st));
    R->n_active = 0;
    return threshold_current<double>(R, R->cfg.eps, true);
}

template <typename T>
wrc_status set_grid_t(wrc_run* R, const uint8_t* active, const double* omega_lattice, int device_ptr) {
    double* scr = R->fp32 ? lattice_scratch(R) : nullptr;
    if (R->fp32 && !scr) return fail(R, WRC_ERR_OOM, "lattice scratch");
    TRY(copy_in(R, R->nxt, active, R->N, device_ptr));
    TRY(in_from_double<T>(R, (T*)R->L, omega_lattice, R->N, device_ptr, scr));
    CK(cudaMemsetAsync(R->flag_dev, 0, sizeof(int), R->st));
    launch_validate_grid(R->nxt, R->flag_dev, R->g, R->st);
    CKL("validate");
    int flag = 0;
    CK(cudaMemcpyAsync(&flag, R->flag_dev, sizeof(int), cudaMemcpyDeviceToHost, R->st));
    CK(cudaStreamSynchronize(R->st));
    if (flag & 1) return fail(R, WRC_ERR_ARG, "grid misses a level-0 point");
    if (flag & 2) return fail(R, WRC_ERR_ARG, "grid is not closed under DD prediction");
    CK(cudaMemsetAsync(R->sig, 0, R->N, R->st));
    R->det_count = 0;
    return rebuild_from_mask<T>(R);
}

template <typename T>
wrc_status threshold_t(wrc_run* R, double eps) {
    TRY(reconstruct<T>(R));
    if (R->scalar) TRY(reconstruct_scalar<T>(R));
    return threshold_current<T>(R, eps, false);
}

template <typename T>
wrc_status query_field_t(wrc_run* R, int which, double* out, int device_ptr) {
    double* scr = R->fp32 ? lattice_scratch(R) : nullptr;
    if (R->fp32 && !scr) return fail(R, WRC_ERR_OOM, "lattice scratch");
    if (which == WRC_FIELD_OMEGA) {
        TRY(reconstruct<T>(R));
        return out_as_double<T>(R, out, (const T*)R->L, R->N, device_ptr, scr);
    }
    TRY(freeze<T>(R));
    if (which == WRC_FIELD_PSI) return out_as_double<T>(R, out, (const T*)R->psi, R->N, device_ptr, scr);
    T* t0 = (T*)R->C1;   // U
    T* t1 = t0 + R->N;   // V
    T* t2 = (T*)R->C2;   // nu_t
    if (R->fp32) {
        // spectral U, V (into Lq and C1) and strain (into C2), as in freeze
        T* S11 = (T*)R->C2;
        T* S12 = S11 + R->N;
        launch_poisson<T>(R->plan, (const T*)R->L, (T*)R->psi, R->C1, R->C2, R->g, R->st, (T*)R->Lq, (T*)R->C1,
                          scr, S11, S12, (void*)(scr + R->N));
        T* nut = (T*)R->C1 + R->N;
        if (which == WRC_FIELD_NUT) launch_nut_from_strain<T>(S11, S12, nut, R->cfg.cs, R->g, R->st);
        CKL("lattice fields");
        const T* src = which == WRC_FIELD_U ? (const T*)R->Lq : which == WRC_FIELD_V ? (const T*)R->C1 : nut;
        // convert through the second half of the scratch (its first half was an FFT work array)
        return out_as_double<T>(R, out, src, R->N, device_ptr, scr + R->N);
    }
    launch_lattice_uv_nut<T>((const T*)R->psi, t0, t1, which == WRC_FIELD_NUT ? t2 : nullptr, R->cfg.cs, t0, R->g,
                             R->st);
    CKL("lattice fields");
    const T* src = which == WRC_FIELD_U ? t0 : which == WRC_FIELD_V ? t1 : t2;
    return out_as_double<T>(R, out, src, R->N, device_ptr, scr);
}

template <typename T>
wrc_status apply_operator_t(wrc_run* R, const double* q, double* w, double* g_out, int device_ptr) {
    const long long n = R->n_active;
    const uint32_t* meta = R->meta[R->cur].as<uint32_t>();
    double* scr = R->tmp.as<double>();
    T* qb = R->w.as<T>();
    TRY(in_from_double<T>(R, qb, q, n, device_ptr, scr));
    launch_scatter<T>(meta, qb, n, (T*)R->Lq, R->st);
    ghost_fill<T>(R, (T*)R->Lq, nullptr, 0);
    launch_matvec<T>((const T*)R->Lq, meta, n, R->Ua.as<T>(), R->Va.as<T>(), nullptr, nu_eff(R), R->cfg.rayleigh_r,
                     qb, R->g, nullptr, 0, R->st);
    CKL("apply_operator");
    TRY(out_as_double<T>(R, w, qb, n, device_ptr, scr));
    if (g_out) {
        if (R->cfg.sgs == WRC_SGS_DYNAMIC) {
            TRY(out_as_double<T>(R, g_out, R->ga.as<T>(), n, device_ptr, scr));
        } else if (device_ptr) {
            CK(cudaMemsetAsync(g_out, 0, sizeof(double) * n, R->st));
        } else {
            CK(cudaStreamSynchronize(R->st));
            std::memset(g_out, 0, sizeof(double) * n);
        }
    }
    return WRC_OK;
}

template <typename T>
wrc_status diagnostics_t(wrc_run* R) {
    TRY(reconstruct<T>(R));
    launch_poisson<T>(R->plan, (const T*)R->L, (T*)R->psi, R->C1, R->C2, R->g, R->st);
    CK(launch_diag<T>((const T*)R->L, (const T*)R->psi, R->K.part, R->K.counter, R->diag_dev, R->g, R->st));
    CKL("diagnostics");
    return WRC_OK;
}

// Passive scalar from a lattice field: buffers, Lr <- the field, L <- R(omega)
// on the current grid, one joint thresholding (omega's details on its grid,
// the field's on every lattice point), and the rebuild, which samples r_v at
// the new grid from the field.
template <typename T>
wrc_status scalar_init_t(wrc_run* R, double kappa, const double* field, int device_ptr) {
    const cudaStream_t s = R->st;
    const Geom& g = R->g;
    const int m = R->cfg.krylov_m;
    double* scr = R->fp32 ? lattice_scratch(R) : nullptr;
    if (R->fp32 && !scr) return fail(R, WRC_ERR_OOM, "lattice scratch");
    CK(R->Lr.grow(R->es * (size_t)R->N, 0, s));
    CK(R->rv[0].grow(R->es * (size_t)R->cap, 0, s));
    CK(R->rv[1].grow(R->es * (size_t)R->cap, 0, s));
    CK(R->kr.grow(sizeof(double) * ((size_t)(m + 1) * m + 1 + 32) + sizeof(int) * 4, 0, s));
    CK(cudaMemsetAsync(R->kr.p, 0, R->kr.bytes, s));
    TRY(in_from_double<T>(R, R->Lr.as<T>(), field, R->N, device_ptr, scr));
    TRY(reconstruct<T>(R));
    CK(cudaMemsetAsync(R->sig, 0, R->N, s));
    CK(cudaMemsetAsync(R->nxt, 0, R->N, s));
    launch_details_adj<T>(R->meta[R->cur].as<uint32_t>(), R->cap, (const T*)R->L, R->cfg.eps, R->det.as<T>(), R->sig,
                          R->nxt, g, s, R->counts_dev);
    launch_details_adj<T>(nullptr, R->N, R->Lr.as<T>(), R->cfg.eps, nullptr, R->sig, R->nxt, g, s);
    for (int j = g.J; j >= 1; --j) launch_closure_level(R->nxt, nullptr, j, g, s);
    CKL("scalar threshold");
    R->scalar = true;
    R->kappa = kappa;
    R->layout += 1;   // the captured phases change
    R->det_count = R->n_active;
    TRY(rebuild_part1(R));
    TRY(rebuild_host(R));
    TRY(rebuild_part2<T>(R));
    rebuild_commit(R);
    return WRC_OK;
}

void free_run(wrc_run* R) {
    if (!R) return;
    cudaStream_t s = R->st;
    cudaStreamSynchronize(s);
    for (auto* b : {&R->meta[0], &R->meta[1], &R->omega[0], &R->omega[1], &R->Ua, &R->Va, &R->ga, &R->det, &R->w,
                    &R->basis, &R->tmp, &R->row_len, &R->row_ready, &R->row_idx, &R->row_w, &R->Gb, &R->lat64,
                    &R->trace, &R->rows, &R->rv[0],
                    &R->rv[1], &R->Lr, &R->kr, &R->jac, &R->rbpart, &R->rbsmall, &R->pe[0], &R->pe[1], &R->Lp, &R->Lqx,
                    &R->xd, &R->xbasis, &R->xw, &R->sbasis, &R->sw, &R->sGb, &R->sLq, &R->spart, &R->sbar, &R->sdev})
        b->release(s);
    cudaStreamSynchronize(s);
    void* ptrs[] = {R->L, R->Lq, R->psi, R->C1, R->C2, R->act, R->nxt, R->gho, R->sig, R->JJ, R->halo, R->list, R->lat2idx,
                    R->blk_counts, R->blk_off, R->counts_dev, R->flag_dev, R->lvl_dev, R->vort_dev, R->diag_dev,
                    R->K.H, R->K.kstop, R->K.part};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (R->counts_host) cudaFreeHost(R->counts_host);
    if (R->shost) cudaFreeHost(R->shost);
    for (cudaEvent_t e : R->ev_pool) cudaEventDestroy(e);
    if (R->sync_ev) cudaEventDestroy(R->sync_ev);
    for (cudaEvent_t e : R->st_pool) cudaEventDestroy(e);
    for (auto& ph : R->graphs)
        for (auto& G : ph)
            if (G.exec) cudaGraphExecDestroy(G.exec);
    poisson_plan_free(R->plan);
    delete R;
}

bool valid_config(const wrc_config* c, std::string& why) {
    if (!c) { why = "cfg is NULL"; return false; }
    if (c->n0 < 4 || (c->n0 & (c->n0 - 1))) { why = "n0 must be a power of two >= 4"; return false; }
    if (c->J < 1 || c->J > 10) { why = "J must be in 1..10"; return false; }
    if ((long long)c->n0 << c->J > WRC_MAX_NJ) { why = "n0 * 2^J exceeds WRC_MAX_NJ"; return false; }
    if (c->krylov_m < 1 || c->krylov_m > WRC_MAX_M) { why = "krylov_m must be in 1..WRC_MAX_M"; return false; }
    if (c->sgs < 0 || c->sgs > 2) { why = "unknown sgs mode"; return false; }
    if (c->prec != WRC_FP64 && c->prec != WRC_MIXED) { why = "unknown precision"; return false; }
    if (c->p != 0 && (c->p < 2 || c->p > kMaxP)) { why = "p (half the DD order) must be 2, 3 or 4 (0: 2)"; return false; }
    if (c->scheme != WRC_SCHEME_FROZEN && c->scheme != WRC_SCHEME_ROSENBROCK) { why = "unknown scheme"; return false; }
    if (c->model != WRC_MODEL_VORTICITY && c->model != WRC_MODEL_EXNER) { why = "unknown model"; return false; }
    if (c->model == WRC_MODEL_EXNER) {
        if (c->prec != WRC_FP64) { why = "the velocity-Exner form runs in FP64 only"; return false; }
        if (c->sgs == WRC_SGS_DYNAMIC) { why = "the velocity-Exner form takes the a-priori subgrid model only"; return false; }
        if (!(c->cpt >= 0) || !std::isfinite(c->cpt) || !std::isfinite(c->coriolis) || !std::isfinite(c->gx) ||
            !std::isfinite(c->gy)) {
            why = "cpt must be finite and >= 0; coriolis, gx, gy finite";
            return false;
        }
    }
    if (!(c->eps >= 0) || !(c->re > 0) || !(c->dt > 0) || !(c->rayleigh_r >= 0) || !(c->cs >= 0) ||
        !(c->s_apriori >= 0)) {
        why = "eps, re, dt, rayleigh_r, cs, s_apriori out of range";
        return false;
    }
    return true;
}

}  // namespace

bool wrc::valid_run_config(const wrc_config* c, std::string& why) { return valid_config(c, why); }

extern "C" {

wrc_status wrc_create(const wrc_config* cfg, void* cuda_stream, wrc_run** out) {
    if (!out) return WRC_ERR_ARG;
    *out = nullptr;
    std::string why;
    if (!valid_config(cfg, why)) {
        g_create_error = why;
        return WRC_ERR_ARG;
    }
    wrc_run* R = new wrc_run();
    R->cfg = *cfg;
    R->fp32 = cfg->prec == WRC_MIXED;
    R->es = R->fp32 ? sizeof(float) : sizeof(double);
    R->st = (cudaStream_t)cuda_stream;
    cudaGetDevice(&R->device);
    const int NJ = cfg->n0 << cfg->J;
    int Lg = 0;
    while ((1 << Lg) < NJ) ++Lg;
    R->g.NJ = NJ;
    R->g.L = Lg;
    R->g.J = cfg->J;
    R->g.mask = NJ - 1;
    R->g.h = 2.0 * 3.141592653589793238462643383279502884 / NJ;
    R->g.P = cfg->p == 0 ? 2 : cfg->p;
    R->rmax = dd_row_max(R->g.P);
    R->N = (long long)NJ * NJ;
    R->exner = cfg->model == WRC_MODEL_EXNER;
    const long long N = R->N;
    const int m = cfg->krylov_m;
    const int nblk = (int)((N + kTile - 1) / kTile);
    auto alloc = [&](void** p, size_t bytes) { return cudaMalloc(p, bytes); };
    cudaError_t e = cudaSuccess;
    void** lp[] = {(void**)&R->L, (void**)&R->Lq, (void**)&R->psi};
    for (auto p : lp)
        if (e == cudaSuccess) e = alloc(p, R->es * N);
    if (e == cudaSuccess) e = alloc(&R->C1, 2 * R->es * N);
    if (e == cudaSuccess) e = alloc(&R->C2, 2 * R->es * N);
    uint8_t** mp[] = {&R->act, &R->nxt, &R->gho, &R->sig, &R->JJ, &R->halo};
    for (auto p : mp)
        if (e == cudaSuccess) e = alloc((void**)p, N);
    if (e == cudaSuccess) e = alloc((void**)&R->list, sizeof(int) * N);
    if (e == cudaSuccess) e = alloc((void**)&R->lat2idx, sizeof(int) * N);
    if (e == cudaSuccess) e = alloc((void**)&R->blk_counts, sizeof(int) * nblk * kMaxKeys);
    if (e == cudaSuccess) e = alloc((void**)&R->blk_off, sizeof(int) * nblk * kMaxKeys);
    if (e == cudaSuccess) e = alloc((void**)&R->counts_dev, sizeof(int) * kMaxKeys);
    if (e == cudaSuccess) e = alloc((void**)&R->flag_dev, sizeof(int) * 4);
    if (e == cudaSuccess) e = alloc((void**)&R->lvl_dev, sizeof(unsigned long long) * 16);
    if (e == cudaSuccess) e = alloc((void**)&R->vort_dev, sizeof(double) * 4 * WRC_MAX_VORTICES);
    if (e == cudaSuccess) e = alloc((void**)&R->diag_dev, sizeof(double) * 8);
    if (e == cudaSuccess) e = R->rows.grow(sizeof(int) * ((size_t)NJ + 1), 0, R->st);
    // Krylov small arrays: H, then o1/o2/o3/beta/y in one block, partials, ints
    R->cluster_max = krylov_cluster_max();
    if (krylov_step_init(R->device, R->fp32, R->g.P, &R->max_blocks) != 0) {
        g_create_error = "cooperative Krylov kernel set-up failed";
        free_run(R);
        return WRC_ERR_CUDA;
    }
    if (e == cudaSuccess) e = alloc((void**)&R->K.H, sizeof(double) * ((m + 1) * m + 1 + 32));
    if (e == cudaSuccess) e = alloc((void**)&R->K.kstop, sizeof(int) * 8);
    const size_t npart = krylov_partials_doubles(R->max_blocks) > (size_t)kMaxBlocks * 4
                             ? krylov_partials_doubles(R->max_blocks) : (size_t)kMaxBlocks * 4;
    if (e == cudaSuccess) e = alloc((void**)&R->K.part, sizeof(double) * npart);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&R->counts_host, sizeof(int) * (kMaxKeys + 4));
    if (e != cudaSuccess) {
        g_create_error = std::string("allocation failed: ") + cudaGetErrorString(e);
        free_run(R);
        return e == cudaErrorMemoryAllocation ? WRC_ERR_OOM : WRC_ERR_CUDA;
    }
    R->K.beta = R->K.H + (m + 1) * m;
    R->K.y = R->K.beta + 1;
    R->K.flags = R->K.kstop + 1;
    R->K.err = R->K.kstop + 2;
    R->K.overflow = R->K.kstop + 3;
    R->K.bar = (unsigned*)(R->K.kstop + 4);
    R->K.counter = (unsigned*)(R->K.kstop + 6);
    cudaMemsetAsync(R->K.kstop, 0, sizeof(int) * 8, R->st);
    cudaMemsetAsync(R->flag_dev, 0, sizeof(int) * 4, R->st);
    R->use_graphs = R->st != nullptr;   // stream capture needs a non-legacy stream
    if (R->fp32 && !lattice_scratch(R)) {
        g_create_error = "lattice scratch allocation failed";
        free_run(R);
        return WRC_ERR_OOM;
    }
    if (R->exner) {   // lattices of v and pi, and of a Krylov vector's v and pi parts
        cudaError_t ex = R->Lr.grow(sizeof(double) * N, 0, R->st);
        if (ex == cudaSuccess) ex = R->Lp.grow(sizeof(double) * N, 0, R->st);
        if (ex == cudaSuccess) ex = R->Lqx.grow(2 * sizeof(double) * N, 0, R->st);
        if (ex != cudaSuccess) {
            g_create_error = std::string("allocation failed: ") + cudaGetErrorString(ex);
            free_run(R);
            return ex == cudaErrorMemoryAllocation ? WRC_ERR_OOM : WRC_ERR_CUDA;
        }
    }
    if (poisson_plan_init(R->plan, R->g, R->fp32, R->st) != 0) {
        g_create_error = "FFT/expm kernel set-up failed";
        free_run(R);
        return WRC_ERR_CUDA;
    }
    if (cudaStreamSynchronize(R->st) != cudaSuccess) {
        g_create_error = std::string("set-up: ") + cudaGetErrorString(cudaGetLastError());
        free_run(R);
        return WRC_ERR_CUDA;
    }
    *out = R;
    return WRC_OK;
}

wrc_status wrc_init_vortices(wrc_run* R, int32_t n, const double* xc, const double* yc, const double* gamma,
                             const double* s) {
    if (!R) return WRC_ERR_ARG;
    TRY(vorticity_only(R, "wrc_init_vortices"));
    if (n < 1 || n > WRC_MAX_VORTICES || !xc || !yc || !gamma || !s)
        return fail(R, WRC_ERR_ARG, "need 1..WRC_MAX_VORTICES vortices and four host arrays");
    double prm[4 * WRC_MAX_VORTICES];
    for (int v = 0; v < n; ++v) {
        if (!(s[v] > 0) || !std::isfinite(xc[v]) || !std::isfinite(yc[v]) || !std::isfinite(gamma[v]))
            return fail(R, WRC_ERR_ARG, "vortex parameters must be finite with s > 0");
        prm[v] = xc[v];
        prm[n + v] = yc[v];
        prm[2 * n + v] = gamma[v];
        prm[3 * n + v] = s[v];
    }
    CK(cudaMemcpyAsync(R->vort_dev, prm, sizeof(double) * 4 * n, cudaMemcpyHostToDevice, R->st));
    if (R->fp32) launch_init_vortices<float>((float*)R->L, R->vort_dev, n, R->g, R->st);
    else launch_init_vortices<double>((double*)R->L, R->vort_dev, n, R->g, R->st);
    CKL("init_vortices");
    CK(cudaStreamSynchronize(R->st));   // prm is a stack array
    CK(cudaMemsetAsync(R->act, 1, R->N, R->st));
    R->n_active = 0;
    if (R->scalar) R->layout += 1;
    R->scalar = false;   // a new initial condition drops the passive scalar
    TRY(DISPATCH(R, threshold_current, R, R->cfg.eps, true));
    R->init = true;
    R->t = 0.0;
    R->nstep = 0;
    return WRC_OK;
}

wrc_status wrc_init_field(wrc_run* R, const double* omega_lattice, int32_t device_ptr) {
    if (!R) return WRC_ERR_ARG;
    TRY(vorticity_only(R, "wrc_init_field"));
    if (!omega_lattice) return fail(R, WRC_ERR_ARG, "omega_lattice is NULL");
    if (R->scalar) R->layout += 1;
    R->scalar = false;
    TRY(DISPATCH(R, init_field_t, R, omega_lattice, device_ptr));
    R->init = true;
    R->t = 0.0;
    R->nstep = 0;
    return WRC_OK;
}

wrc_status wrc_set_grid(wrc_run* R, const uint8_t* active, const double* omega_lattice, int32_t device_ptr) {
    if (!R) return WRC_ERR_ARG;
    TRY(vorticity_only(R, "wrc_set_grid"));
    if (!active || !omega_lattice) return fail(R, WRC_ERR_ARG, "NULL input");
    if (R->scalar) R->layout += 1;
    R->scalar = false;
    TRY(DISPATCH(R, set_grid_t, R, active, omega_lattice, device_ptr));
    R->init = true;
    return WRC_OK;
}

wrc_status wrc_threshold(wrc_run* R, double eps) {
    TRY(check_ready(R));
    TRY(vorticity_only(R, "wrc_threshold"));
    if (!(eps >= 0)) return fail(R, WRC_ERR_ARG, "eps must be >= 0");
    R->cfg.eps = eps;
    R->layout += 1;   // eps is baked into the captured thresholding phase
    return DISPATCH(R, threshold_t, R, eps);
}

wrc_status wrc_step(wrc_run* R, int32_t nsteps) {
    TRY(check_ready(R));
    if (nsteps < 0) return fail(R, WRC_ERR_ARG, "nsteps < 0");
    for (int q = 0; q < nsteps; ++q) TRY(DISPATCH(R, step_once, R));
    return WRC_OK;
}

wrc_status wrc_sync(wrc_run* R, int32_t timeout_ms) {
    if (!R) return WRC_ERR_ARG;
    if (timeout_ms < 0) {
        CK(cudaStreamSynchronize(R->st));
    } else {
        // poll an event recorded behind the queued work; on expiry the work
        // stays queued and a later wrc_sync can wait for it again
        if (!R->sync_ev) CK(cudaEventCreateWithFlags(&R->sync_ev, cudaEventDisableTiming));
        CK(cudaEventRecord(R->sync_ev, R->st));
        const auto t0 = std::chrono::steady_clock::now();
        while (true) {
            const cudaError_t q = cudaEventQuery(R->sync_ev);
            if (q == cudaSuccess) break;
            if (q != cudaErrorNotReady) CK(q);
            const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            if (ms >= (double)timeout_ms) return fail(R, WRC_ERR_TIMEOUT, "wrc_sync: the run's stream is still busy");
            std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
    }
    int flags = 0;
    CK(cudaMemcpy(&flags, R->K.flags, sizeof(int), cudaMemcpyDeviceToHost));
    if (flags & 1) {
        CK(cudaMemset(R->K.flags, 0, sizeof(int)));
        return fail(R, WRC_ERR_BREAKDOWN_NAN, "non-finite value in the Arnoldi process");
    }
    return WRC_OK;
}

wrc_status wrc_query_counts(wrc_run* R, int64_t* n_active, int64_t* n_ghost, int64_t* per_level) {
    TRY(check_ready(R));
    if (n_active) *n_active = R->n_active;
    if (n_ghost) *n_ghost = R->n_ghost;
    if (per_level) {
        CK(cudaMemsetAsync(R->lvl_dev, 0, sizeof(unsigned long long) * 16, R->st));
        launch_level_counts(R->meta[R->cur].as<uint32_t>(), R->n_active, R->lvl_dev, R->g, R->st);
        CKL("level counts");
        unsigned long long h[16];
        CK(cudaMemcpyAsync(h, R->lvl_dev, sizeof(h), cudaMemcpyDeviceToHost, R->st));
        CK(cudaStreamSynchronize(R->st));
        for (int j = 0; j <= R->g.J; ++j) per_level[j] = (int64_t)h[j];
    }
    return WRC_OK;
}

wrc_status wrc_query_active(wrc_run* R, int32_t* idx_out, double* omega_out, int64_t cap, int32_t device_ptr) {
    TRY(check_ready(R));
    if (cap < R->n_active) return fail(R, WRC_ERR_ARG, "cap smaller than the active count");
    if (omega_out) TRY(vorticity_only(R, "wrc_query_active with omega_out"));
    const long long n = R->n_active;
    if (omega_out) {
        if (R->fp32) TRY(out_as_double<float>(R, omega_out, R->omega[R->cur].as<float>(), n, device_ptr, R->tmp.as<double>()));
        else TRY(copy_out(R, omega_out, R->omega[R->cur].p, sizeof(double) * n, device_ptr));
        CK(cudaStreamSynchronize(R->st));
    }
    if (idx_out) {
        int* tmpi = R->tmp.as<int>();   // tmp holds >= n doubles, i.e. >= 2n ints
        launch_meta_unpack(R->meta[R->cur].as<uint32_t>(), n, tmpi, nullptr, nullptr, R->st);
        CKL("unpack");
        TRY(copy_out(R, idx_out, tmpi, sizeof(int) * n, device_ptr));
    }
    CK(cudaStreamSynchronize(R->st));
    return WRC_OK;
}

wrc_status wrc_scalar_init(wrc_run* R, double kappa, const double* field, int32_t device_ptr) {
    TRY(check_ready(R));
    TRY(vorticity_only(R, "wrc_scalar_init"));
    if (!field) return fail(R, WRC_ERR_ARG, "field is NULL");
    if (!(kappa >= 0) || !std::isfinite(kappa)) return fail(R, WRC_ERR_ARG, "kappa must be finite and >= 0");
    const bool was = R->scalar;
    const wrc_status st = DISPATCH(R, scalar_init_t, R, kappa, field, device_ptr);
    if (st != WRC_OK && !was) R->scalar = false;
    return st;
}

wrc_status wrc_query_scalar(wrc_run* R, int32_t* idx_out, double* r_out, int64_t cap, int32_t device_ptr) {
    TRY(check_ready(R));
    if (!R->scalar) return fail(R, WRC_ERR_STATE, "the passive scalar is not enabled (wrc_scalar_init)");
    if (cap < R->n_active) return fail(R, WRC_ERR_ARG, "cap smaller than the active count");
    const long long n = R->n_active;
    if (r_out) {
        if (R->fp32) TRY(out_as_double<float>(R, r_out, R->rv[R->cur].as<float>(), n, device_ptr, R->tmp.as<double>()));
        else TRY(copy_out(R, r_out, R->rv[R->cur].p, sizeof(double) * n, device_ptr));
        CK(cudaStreamSynchronize(R->st));
    }
    if (idx_out) {
        int* tmpi = R->tmp.as<int>();
        launch_meta_unpack(R->meta[R->cur].as<uint32_t>(), n, tmpi, nullptr, nullptr, R->st);
        CKL("unpack");
        TRY(copy_out(R, idx_out, tmpi, sizeof(int) * n, device_ptr));
    }
    CK(cudaStreamSynchronize(R->st));
    return WRC_OK;
}

wrc_status wrc_exner_init(wrc_run* R, const double* u, const double* v, const double* pi, int32_t device_ptr) {
    if (!R) return WRC_ERR_ARG;
    if (!R->exner) return fail(R, WRC_ERR_STATE, "wrc_exner_init needs a run of model WRC_MODEL_EXNER");
    if (!u || !v || !pi) return fail(R, WRC_ERR_ARG, "NULL field");
    R->init = false;
    TRY(copy_in(R, R->L, u, sizeof(double) * R->N, device_ptr));
    TRY(copy_in(R, R->Lr.p, v, sizeof(double) * R->N, device_ptr));
    TRY(copy_in(R, R->Lp.p, pi, sizeof(double) * R->N, device_ptr));
    TRY(exner_threshold_whole(R));
    R->init = true;
    R->t = 0.0;
    R->nstep = 0;
    return WRC_OK;
}

wrc_status wrc_exner_init_vortices(wrc_run* R, int32_t n, const double* xc, const double* yc, const double* gamma,
                                   const double* s, double pi0) {
    if (!R) return WRC_ERR_ARG;
    if (!R->exner) return fail(R, WRC_ERR_STATE, "wrc_exner_init_vortices needs a run of model WRC_MODEL_EXNER");
    if (n < 1 || n > WRC_MAX_VORTICES || !xc || !yc || !gamma || !s)
        return fail(R, WRC_ERR_ARG, "need 1..WRC_MAX_VORTICES vortices and four host arrays");
    if (!(pi0 > 0) || !std::isfinite(pi0)) return fail(R, WRC_ERR_ARG, "pi0 must be finite and > 0");
    double prm[4 * WRC_MAX_VORTICES];
    for (int q = 0; q < n; ++q) {
        if (!(s[q] > 0) || !std::isfinite(xc[q]) || !std::isfinite(yc[q]) || !std::isfinite(gamma[q]))
            return fail(R, WRC_ERR_ARG, "vortex parameters must be finite with s > 0");
        prm[q] = xc[q];
        prm[n + q] = yc[q];
        prm[2 * n + q] = gamma[q];
        prm[3 * n + q] = s[q];
    }
    R->init = false;
    const cudaStream_t st = R->st;
    CK(cudaMemcpyAsync(R->vort_dev, prm, sizeof(double) * 4 * n, cudaMemcpyHostToDevice, st));
    // omega on the lattice (in Lq), psi, then u = D_y psi into L and v = -D_x psi into Lr
    launch_init_vortices<double>((double*)R->Lq, R->vort_dev, n, R->g, st);
    launch_poisson<double>(R->plan, (const double*)R->Lq, (double*)R->psi, R->C1, R->C2, R->g, st);
    launch_lattice_uv_nut<double>((const double*)R->psi, (double*)R->L, R->Lr.as<double>(), nullptr, 0.0,
                                  (double*)R->C1, R->g, st);
    CKL("exner vortices");
    CK(ex_fill(R->Lp.as<double>(), R->N, pi0, st));
    CK(cudaStreamSynchronize(st));   // prm is a stack array
    TRY(exner_threshold_whole(R));
    R->init = true;
    R->t = 0.0;
    R->nstep = 0;
    return WRC_OK;
}

wrc_status wrc_query_exner(wrc_run* R, int32_t* idx_out, double* u_out, double* v_out, double* pi_out, int64_t cap,
                           int32_t device_ptr) {
    TRY(check_ready(R));
    if (!R->exner) return fail(R, WRC_ERR_STATE, "wrc_query_exner needs a run of model WRC_MODEL_EXNER");
    if (cap < R->n_active) return fail(R, WRC_ERR_ARG, "cap smaller than the active count");
    const long long n = R->n_active;
    if (u_out) TRY(copy_out(R, u_out, R->omega[R->cur].p, sizeof(double) * n, device_ptr));
    if (v_out) TRY(copy_out(R, v_out, R->rv[R->cur].p, sizeof(double) * n, device_ptr));
    if (pi_out) TRY(copy_out(R, pi_out, R->pe[R->cur].p, sizeof(double) * n, device_ptr));
    if (idx_out) {
        int* tmpi = R->tmp.as<int>();
        launch_meta_unpack(R->meta[R->cur].as<uint32_t>(), n, tmpi, nullptr, nullptr, R->st);
        CKL("unpack");
        TRY(copy_out(R, idx_out, tmpi, sizeof(int) * n, device_ptr));
    }
    CK(cudaStreamSynchronize(R->st));
    return WRC_OK;
}

wrc_status wrc_query_masks(wrc_run* R, uint8_t* active, uint8_t* ghost, uint8_t* significant, int32_t device_ptr) {
    TRY(check_ready(R));
    if (active) TRY(copy_out(R, active, R->act, R->N, device_ptr));
    if (ghost) TRY(copy_out(R, ghost, R->gho, R->N, device_ptr));
    if (significant) TRY(copy_out(R, significant, R->sig, R->N, device_ptr));
    CK(cudaStreamSynchronize(R->st));
    return WRC_OK;
}

wrc_status wrc_query_details(wrc_run* R, double* d_out, int64_t cap, int32_t device_ptr) {
    TRY(vorticity_only(R, "wrc_query_details"));
    TRY(check_ready(R));
    if (!d_out) return fail(R, WRC_ERR_ARG, "NULL output");
    if (cap < R->det_count) return fail(R, WRC_ERR_ARG, "cap smaller than the detail count");
    if (R->fp32) TRY(out_as_double<float>(R, d_out, R->det.as<float>(), R->det_count, device_ptr, R->tmp.as<double>()));
    else TRY(copy_out(R, d_out, R->det.p, sizeof(double) * R->det_count, device_ptr));
    CK(cudaStreamSynchronize(R->st));
    return WRC_OK;
}

wrc_status wrc_query_stencil_levels(wrc_run* R, uint8_t* jx_out, uint8_t* jy_out, int64_t cap, int32_t device_ptr) {
    TRY(check_ready(R));
    if (cap < R->n_active) return fail(R, WRC_ERR_ARG, "cap smaller than the active count");
    const long long n = R->n_active;
    uint8_t* jx = R->tmp.as<uint8_t>();
    uint8_t* jy = jx + n;
    launch_meta_unpack(R->meta[R->cur].as<uint32_t>(), n, nullptr, jx, jy, R->st);
    CKL("unpack");
    if (jx_out) TRY(copy_out(R, jx_out, jx, n, device_ptr));
    if (jy_out) TRY(copy_out(R, jy_out, jy, n, device_ptr));
    CK(cudaStreamSynchronize(R->st));
    return WRC_OK;
}

wrc_status wrc_query_field(wrc_run* R, int32_t which, double* out, int32_t device_ptr) {
    TRY(check_ready(R));
    TRY(vorticity_only(R, "wrc_query_field"));
    if (!out || which < 0 || which > 4) return fail(R, WRC_ERR_ARG, "bad field or NULL output");
    TRY(DISPATCH(R, query_field_t, R, which, out, device_ptr));
    CK(cudaStreamSynchronize(R->st));
    return WRC_OK;
}

wrc_status wrc_freeze(wrc_run* R) {
    TRY(check_ready(R));
    TRY(vorticity_only(R, "wrc_freeze"));
    TRY(DISPATCH(R, freeze, R));
    CK(cudaStreamSynchronize(R->st));
    return WRC_OK;
}

wrc_status wrc_apply_operator(wrc_run* R, const double* q, double* w, double* g_out, int32_t device_ptr) {
    TRY(check_ready(R));
    TRY(vorticity_only(R, "wrc_apply_operator"));
    if (!R->frozen) return fail(R, WRC_ERR_STATE, "call wrc_freeze after the last grid change");
    if (!q || !w) return fail(R, WRC_ERR_ARG, "NULL input or output");
    TRY(DISPATCH(R, apply_operator_t, R, q, w, g_out, device_ptr));
    CK(cudaStreamSynchronize(R->st));
    return WRC_OK;
}

wrc_status wrc_query_krylov(wrc_run* R, double* beta, int32_t* k, double* h_last, double* H, double* y) {
    TRY(check_ready(R));
    const int m = R->cfg.krylov_m;
    double hb[(WRC_MAX_M + 1) * WRC_MAX_M];
    double bb = 0, yb[WRC_MAX_M + 1];
    int kk = 0;
    CK(cudaMemcpyAsync(hb, R->K.H, sizeof(double) * (m + 1) * m, cudaMemcpyDeviceToHost, R->st));
    CK(cudaMemcpyAsync(&bb, R->K.beta, sizeof(double), cudaMemcpyDeviceToHost, R->st));
    CK(cudaMemcpyAsync(yb, R->K.y, sizeof(double) * m, cudaMemcpyDeviceToHost, R->st));
    CK(cudaMemcpyAsync(&kk, R->K.kstop, sizeof(int), cudaMemcpyDeviceToHost, R->st));
    CK(cudaStreamSynchronize(R->st));
    if (beta) *beta = bb;
    if (k) *k = kk;
    if (h_last) *h_last = kk > 0 ? hb[(size_t)kk * m + (kk - 1)] : 0.0;
    if (H) std::memcpy(H, hb, sizeof(double) * (m + 1) * m);
    if (y) std::memcpy(y, yb, sizeof(double) * m);
    return WRC_OK;
}

wrc_status wrc_diagnostics(wrc_run* R, double out[9]) {
    TRY(check_ready(R));
    TRY(vorticity_only(R, "wrc_diagnostics"));
    if (!out) return fail(R, WRC_ERR_ARG, "NULL output");
    TRY(DISPATCH(R, diagnostics_t, R));
    double s[4];
    CK(cudaMemcpyAsync(s, R->diag_dev, sizeof(s), cudaMemcpyDeviceToHost, R->st));
    CK(cudaStreamSynchronize(R->st));
    const double w = R->g.h * R->g.h;
    out[0] = 0.5 * w * s[2];
    out[1] = 0.5 * w * s[1];
    out[2] = 0.5 * w * s[3];
    out[3] = w * s[0];
    out[4] = R->t;
    out[5] = (double)R->nstep;
    out[6] = (double)R->n_active;
    out[7] = (double)R->n_ghost;
    out[8] = 0.0;
    if (R->nstep > 0) {
        double beta = 0.0, hl = 0.0, y[WRC_MAX_M];
        int32_t k = 0;
        TRY(wrc_query_krylov(R, &beta, &k, &hl, nullptr, y));
        if (k > 0) out[8] = R->cfg.dt * beta * hl * std::fabs(y[k - 1]);
    }
    return WRC_OK;
}

wrc_status wrc_query_stats(wrc_run* R, int64_t out[4]) {
    if (!R || !out) return WRC_ERR_ARG;
    out[0] = launches_total();
    out[1] = R->nstep;
    out[2] = R->host_syncs;
    out[3] = R->n_active;
    return WRC_OK;
}

wrc_status wrc_profile(wrc_run* R, int32_t enable) {
    if (!R) return WRC_ERR_ARG;
    if (enable < 0 || enable > 3) return fail(R, WRC_ERR_ARG, "enable must be 0, 1, 2 or 3");
    if (enable == 2) TRY(vorticity_only(R, "the phase trace of wrc_profile"));
    CK(cudaStreamSynchronize(R->st));
    R->profiling = enable == 1 || enable == 2;
    R->tracing = enable == 2;
    R->stage_timing = enable == 3;
    R->st_ids.clear();
    std::fill(R->st_ms, R->st_ms + WRC_STAGE_COUNT, 0.0);
    R->st_steps = 0;
    if (R->tracing) {
        const size_t words = 1 + (size_t)kTracePhases * (kMaxBlocks + 1);
        CK(R->trace.grow(sizeof(unsigned long long) * words, 0, R->st));
    }
    R->ev_used.clear();
    return WRC_OK;
}

wrc_status wrc_query_krylov_form(wrc_run* R, int32_t* cluster_size) {
    if (!R || !cluster_size) return WRC_ERR_ARG;
    *cluster_size = krylov_step_cluster(R->n_active, R->max_blocks, R->fp32, R->g.P, R->device, R->cluster_max);
    return WRC_OK;
}

wrc_status wrc_set_wait_limit(wrc_run* R, double seconds) {
    if (!R) return WRC_ERR_ARG;
    if (!(seconds > 0) || !(seconds <= 60.0)) return fail(R, WRC_ERR_ARG, "the wait limit must be in (0, 60] s");
    double ns = std::ceil(seconds * 1e9);
    R->wait_limit_ns = (unsigned long long)(ns < 1.0 ? 1.0 : ns);
    R->layout += 1;   // the captured rebuild phase holds the limit in its ghost-row launch
    return WRC_OK;
}

wrc_status wrc_query_phase_trace(wrc_run* R, double* out, int32_t cap, int32_t* nphases) {
    if (!R || !out || !nphases) return WRC_ERR_ARG;
    if (!R->tracing || !R->trace_nb) return fail(R, WRC_ERR_STATE, "no traced Krylov launch (wrc_profile(run, 2))");
    CK(cudaStreamSynchronize(R->st));
    const int nb = R->trace_nb;
    std::vector<unsigned long long> h(1 + (size_t)kTracePhases * (nb + 1));
    CK(cudaMemcpy(h.data(), R->trace.p, sizeof(unsigned long long) * h.size(), cudaMemcpyDeviceToHost));
    const unsigned long long t0 = h[0];
    int np = 0;
    for (int p = 0; p < kTracePhases; ++p) {
        const unsigned long long* row = h.data() + 1 + (size_t)p * (nb + 1);
        if (row[nb] == 0) break;   // block 0 never left barrier p
        if (4 * (p + 1) > cap) return fail(R, WRC_ERR_ARG, "cap too small for the traced phases");
        unsigned long long lo = ~0ull, hi = 0;
        int who = 0;
        for (int b = 0; b < nb; ++b) {
            lo = std::min(lo, row[b]);
            if (row[b] > hi) {
                hi = row[b];
                who = b;
            }
        }
        out[4 * p + 0] = 1e-3 * (double)(lo - t0);
        out[4 * p + 1] = 1e-3 * (double)(hi - t0);
        out[4 * p + 2] = (double)who;
        out[4 * p + 3] = 1e-3 * (double)(row[nb] - t0);
        np = p + 1;
    }
    *nphases = np;
    return WRC_OK;
}

wrc_status wrc_query_stages(wrc_run* R, double* out, int32_t cap) {
    if (!R || !out) return WRC_ERR_ARG;
    if (cap < 1 + WRC_STAGE_COUNT) return fail(R, WRC_ERR_ARG, "cap must be at least 1 + WRC_STAGE_COUNT");
    if (!R->stage_timing) return fail(R, WRC_ERR_STATE, "stage timing is off (wrc_profile(run, 3))");
    TRY(stage_fold(R));
    out[0] = (double)R->st_steps;
    for (int s = 0; s < WRC_STAGE_COUNT; ++s) out[1 + s] = R->st_ms[s];
    return WRC_OK;
}

wrc_status wrc_query_profile(wrc_run* R, double out[4]) {
    if (!R || !out) return WRC_ERR_ARG;
    CK(cudaStreamSynchronize(R->st));
    double ms = 0.0, bytes = 0.0, flops = 0.0;
    for (const auto& u : R->ev_used) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, R->ev_pool[u.ev], R->ev_pool[u.ev + 1]));
        ms += t;
        bytes += u.bytes;
        flops += u.flops;
    }
    out[0] = (double)R->ev_used.size();
    out[1] = ms;
    out[2] = bytes;
    out[3] = flops;
    return WRC_OK;
}

const char* wrc_last_error(const wrc_run* R) { return R ? R->err.c_str() : g_create_error.c_str(); }

void wrc_destroy(wrc_run* R) { free_run(R); }

}  // extern "C"

// ============================================================================
// Batched stepping of several runs (ensemble and server)
// ============================================================================

namespace {

constexpr int kBatchStreams = 8;

wrc_status cfail(BatchCtx& C, wrc_status s, const std::string& msg) {
    C.err = msg;
    return s;
}

#define BCK(call)                                                                               \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return cfail(C, e_ == cudaErrorMemoryAllocation ? WRC_ERR_OOM : WRC_ERR_CUDA,       \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                   \
    } while (0)

// Block plan: run i gets ceil(n_i / (pt * ept)) blocks, clamped to
// [1, its partial-sum capacity]; if the total exceeds what can be co-resident,
// every run's share is scaled down (keeping at least one block each).
wrc_status plan_batch(BatchCtx& C, const std::vector<wrc_run*>& runs, int max_coresident, int& total) {
    const size_t M = runs.size();
    std::vector<int> nb(M);
    long long sum = 0;
    for (size_t i = 0; i < M; ++i) {
        const wrc_run* R = runs[i];
        long long b = (R->n_active + (long long)C.pt * C.ept - 1) / ((long long)C.pt * C.ept);
        b = b < 1 ? 1 : b;
        b = b > R->max_blocks ? R->max_blocks : b;
        nb[i] = (int)b;
        sum += b;
    }
    if ((long long)M > max_coresident)
        return cfail(C, WRC_ERR_ARG, "more runs than co-resident blocks of the batched kernel");
    if (sum > max_coresident) {
        const double f = (double)(max_coresident - (long long)M) / (double)(sum - (long long)M);
        sum = 0;
        for (size_t i = 0; i < M; ++i) {
            nb[i] = 1 + (int)std::floor((nb[i] - 1) * f);
            sum += nb[i];
        }
    }
    total = (int)sum;
    if (total + (int)M + 1 > C.blk_cap) {
        BCK(cudaStreamSynchronize(C.main));   // the old tables may still be read
        if (C.h_blk) cudaFreeHost(C.h_blk);
        if (C.d_blk) cudaFree(C.d_blk);
        C.h_blk = nullptr;
        C.d_blk = nullptr;
        C.blk_cap = total + (int)M + 1 + 1024;
        BCK(cudaMallocHost((void**)&C.h_blk, sizeof(int) * C.blk_cap));
        BCK(cudaMalloc((void**)&C.d_blk, sizeof(int) * C.blk_cap));
    }
    if ((int)M > C.args_cap) {
        BCK(cudaStreamSynchronize(C.main));
        if (C.h_args) cudaFreeHost(C.h_args);
        if (C.d_args) cudaFree(C.d_args);
        C.h_args = nullptr;
        C.d_args = nullptr;
        C.args_cap = (int)M + 64;
        BCK(cudaMallocHost((void**)&C.h_args, sizeof(KrylovStepArgs) * C.args_cap));
        BCK(cudaMalloc((void**)&C.d_args, sizeof(KrylovStepArgs) * C.args_cap));
    }
    int* blk2mem = C.h_blk;
    int* b0 = C.h_blk + total;
    int off = 0;
    for (size_t i = 0; i < M; ++i) {
        b0[i] = off;
        for (int b = 0; b < nb[i]; ++b) blk2mem[off + b] = (int)i;
        off += nb[i];
    }
    b0[M] = off;
    return WRC_OK;
}

// The batched launch and the stream joins around it, for the runs `live`.
template <typename T>
wrc_status batch_krylov(BatchCtx& C, const std::vector<wrc_run*>& live) {
    for (size_t q = 0; q < C.streams.size(); ++q) {
        BCK(cudaEventRecord(C.ev_streams[q], C.streams[q]));
        BCK(cudaStreamWaitEvent(C.main, C.ev_streams[q], 0));
    }
    const int maxb = krylov_batch_max_blocks(C.fp32, C.P, C.pt);
    if (maxb <= 0) return cfail(C, WRC_ERR_CUDA, "batched Krylov kernel occupancy query failed");
    int total = 0;
    TRY(plan_batch(C, live, maxb, total));
    const size_t M = live.size();
    int max_n = 1;
    for (size_t i = 0; i < M; ++i) {
        C.h_args[i] = krylov_args(live[i]);
        max_n = std::max(max_n, (int)live[i]->n_active);
        if (live[i]->tracing) {
            const int nbi = C.h_blk[total + i + 1] - C.h_blk[total + i];
            wrc_run* R = live[i];
            R->trace_nb = nbi;
            BCK(cudaMemsetAsync(R->trace.p, 0, R->trace.bytes, C.main));
        }
    }
    BCK(cudaMemcpyAsync(C.d_args, C.h_args, sizeof(KrylovStepArgs) * M, cudaMemcpyHostToDevice, C.main));
    BCK(cudaMemcpyAsync(C.d_blk, C.h_blk, sizeof(int) * (total + M + 1), cudaMemcpyHostToDevice, C.main));
    cudaEvent_t pa = nullptr, pb = nullptr;
    if (C.profiling) {
        BCK(cudaEventCreate(&pa));
        BCK(cudaEventCreate(&pb));
        BCK(cudaEventRecord(pa, C.main));
    }
    (void)max_n;
    BCK(launch_krylov_batch<T>(C.d_args, C.d_blk, C.d_blk + total, (int)M, total, C.pt, C.P, C.main));
    if (C.profiling) {
        BCK(cudaEventRecord(pb, C.main));
        C.prof.push_back({pa, pb});
    }
    C.last_blocks = total;
    BCK(cudaEventRecord(C.ev_main, C.main));
    for (size_t q = 0; q < C.streams.size(); ++q) BCK(cudaStreamWaitEvent(C.streams[q], C.ev_main, 0));
    return WRC_OK;
}

// One step of every run: freeze phases on the runs' streams, one batched
// Krylov launch, adaptation part 1, one wait for all streams, then the host
// part and adaptation part 2 of each run.
template <typename T>
wrc_status batch_step_t(BatchCtx& C, const std::vector<wrc_run*>& runs, std::vector<wrc_status>& rs) {
    const size_t M = runs.size();
    rs.assign(M, WRC_OK);
    if (!M) return WRC_OK;
    wrc_status first = WRC_OK;
    std::string first_msg;
    auto mark = [&](size_t i, wrc_status st) {
        rs[i] = st;
        if (first == WRC_OK) {
            first = st;
            first_msg = "run " + std::to_string(i) + ": " + runs[i]->err;
        }
    };
    // a failure that is not one run's fails every run still going
    auto fail_all = [&](wrc_status st) {
        for (size_t i = 0; i < M; ++i)
            if (rs[i] == WRC_OK) {
                rs[i] = st;
                runs[i]->err = "batched step: " + C.err;
            }
        return st;
    };
    std::vector<long long> na0(M);
    for (size_t i = 0; i < M; ++i)
        if (runs[i]->scalar) {
            runs[i]->err = "the passive scalar is advanced by wrc_step only";
            mark(i, WRC_ERR_ARG);
        } else if (runs[i]->cfg.scheme == WRC_SCHEME_ROSENBROCK) {
            runs[i]->err = "the exponential Rosenbrock scheme is advanced by wrc_step only";
            mark(i, WRC_ERR_ARG);
        }
    for (size_t i = 0; i < M; ++i) {
        wrc_run* R = runs[i];
        na0[i] = R->n_active;
        if (rs[i] != WRC_OK) continue;
        const wrc_status st = run_phase(R, kPhaseFreeze, [&] { return freeze<T>(R, true); });
        if (st != WRC_OK) mark(i, st);
        else R->frozen = true;
    }
    std::vector<wrc_run*> live;
    std::vector<size_t> live_i;
    for (size_t i = 0; i < M; ++i)
        if (rs[i] == WRC_OK) {
            live.push_back(runs[i]);
            live_i.push_back(i);
        }
    if (!live.empty()) {
        const wrc_status st = batch_krylov<T>(C, live);
        if (st != WRC_OK) return fail_all(st);
    }
    for (size_t i : live_i) {
        wrc_run* R = runs[i];
        const wrc_status st = run_phase(R, kPhaseAdapt1, [&] { return adapt_part1<T>(R); });
        if (st != WRC_OK) mark(i, st);
        else R->det_count = R->n_active;
    }
    for (cudaStream_t st : C.streams) {
        const cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return fail_all(cfail(C, WRC_ERR_CUDA, std::string("stream wait: ") + cudaGetErrorString(e)));
    }
    for (size_t i : live_i) {
        if (rs[i] != WRC_OK) continue;
        wrc_run* R = runs[i];
        wrc_status st = rebuild_host(R);
        if (st == WRC_OK) st = run_phase(R, kPhaseAdapt2, [&] { return rebuild_part2<T>(R); });
        if (st != WRC_OK) {
            mark(i, st);
            continue;
        }
        rebuild_commit(R);
        R->t += R->cfg.dt;
        R->nstep += 1;
        R->updates += (double)na0[i];
    }
    // the run streams must not run ahead of the next batched launch's reads
    for (size_t q = 0; q < C.streams.size(); ++q) {
        const cudaError_t e1 = cudaEventRecord(C.ev_streams[q], C.streams[q]);
        const cudaError_t e2 = e1 == cudaSuccess ? cudaStreamWaitEvent(C.main, C.ev_streams[q], 0) : e1;
        if (e2 != cudaSuccess) return fail_all(cfail(C, WRC_ERR_CUDA, std::string("stream join: ") + cudaGetErrorString(e2)));
    }
    if (first != WRC_OK) C.err = first_msg;
    return first;
}

// Autotuner cache: best (threads per block, points per thread) per precision,
// run-count bucket and total-active-points bucket, for this process.
struct TuneKey {
    bool fp32;
    int mb, nb;
    bool operator<(const TuneKey& o) const { return std::tie(fp32, mb, nb) < std::tie(o.fp32, o.mb, o.nb); }
};
std::map<TuneKey, std::pair<int, int>> g_tune_cache;
std::mutex g_tune_mutex;

int log2_bucket(long long v) {
    int b = 0;
    while (v > 1) {
        v >>= 1;
        ++b;
    }
    return b;
}

// Capacity a compact array is grown to for n entries (as ensure_capacity).
long long grown_capacity(long long n) {
    long long c = n + n / 4 + 1024;
    return (c + 255) / 256 * 256;
}

}  // namespace

wrc_status wrc::batch_init(BatchCtx& C, cudaStream_t main, int nstreams, bool fp32, int P) {
    C.fp32 = fp32;
    C.P = P;
    C.main = main;
    if (!C.main) {   // keep the batched launches off the legacy default stream
        BCK(cudaStreamCreateWithFlags(&C.main, cudaStreamNonBlocking));
        C.own_main = true;
    }
    for (int q = 0; q < nstreams; ++q) {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        BCK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        C.streams.push_back(st);
        BCK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        C.ev_streams.push_back(ev);
    }
    BCK(cudaEventCreateWithFlags(&C.ev_main, cudaEventDisableTiming));
    return WRC_OK;
}

void wrc::batch_free(BatchCtx& C) {
    if (C.main) cudaStreamSynchronize(C.main);
    for (cudaStream_t st : C.streams) cudaStreamSynchronize(st);
    for (auto& pe : C.prof) {
        cudaEventDestroy(pe.first);
        cudaEventDestroy(pe.second);
    }
    C.prof.clear();
    for (cudaEvent_t ev : C.ev_streams) cudaEventDestroy(ev);
    if (C.ev_main) cudaEventDestroy(C.ev_main);
    for (cudaStream_t st : C.streams) cudaStreamDestroy(st);
    if (C.own_main && C.main) cudaStreamDestroy(C.main);
    if (C.h_args) cudaFreeHost(C.h_args);
    if (C.d_args) cudaFree(C.d_args);
    if (C.h_blk) cudaFreeHost(C.h_blk);
    if (C.d_blk) cudaFree(C.d_blk);
    C = BatchCtx();
}

wrc_status wrc::batch_step(BatchCtx& C, const std::vector<wrc_run*>& runs, std::vector<wrc_status>* per_run) {
    std::vector<wrc_status> local;
    std::vector<wrc_status>& rs = per_run ? *per_run : local;
    return C.fp32 ? batch_step_t<float>(C, runs, rs) : batch_step_t<double>(C, runs, rs);
}

double wrc::batch_take_profile(BatchCtx& C) {
    if (C.main) cudaStreamSynchronize(C.main);
    double ms = 0.0;
    for (auto& pe : C.prof) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, pe.first, pe.second) == cudaSuccess) ms += t;
        cudaEventDestroy(pe.first);
        cudaEventDestroy(pe.second);
    }
    C.prof.clear();
    return ms;
}

bool wrc::tuned_shape(bool fp32, long long runs, long long active, int& pt, int& ept) {
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    auto it = g_tune_cache.find({fp32, log2_bucket(runs), log2_bucket(active)});
    if (it == g_tune_cache.end()) return false;
    pt = it->second.first;
    ept = it->second.second;
    return true;
}

void wrc::store_tuned_shape(bool fp32, long long runs, long long active, int pt, int ept) {
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    g_tune_cache[{fp32, log2_bucket(runs), log2_bucket(active)}] = {pt, ept};
}

double wrc::run_bytes_for(const wrc_config& cfg, long long na, long long ng) {
    const double N = (double)((long long)cfg.n0 << cfg.J) * (double)((long long)cfg.n0 << cfg.J);
    const double es = cfg.prec == WRC_MIXED ? 4.0 : 8.0;
    const double m1 = cfg.krylov_m + 1;
    const double nblk = std::ceil(N / kTile);
    // L, Lq, psi; complex C1, C2; six byte masks; list and lat2idx; block
    // counts and offsets; the 2N-double scratch (mixed mode always, FP64 on
    // the first query that converts a lattice field)
    double b = 7.0 * es * N + 6.0 * N + 8.0 * N + 8.0 * nblk * kMaxKeys + 16.0 * N;
    // FFT tables: twiddles, symbols
    b += 4.0 * es * std::sqrt(N) + 16.0 * std::sqrt(N);
    // Krylov small arrays and partial sums (at most kMaxBlocks blocks)
    b += 8.0 * (m1 * cfg.krylov_m + 33) +
         8.0 * (double)std::max(krylov_partials_doubles(kMaxBlocks), (size_t)kMaxBlocks * 4);
    const double c = (double)grown_capacity(na), cg = (double)grown_capacity(ng);
    // meta x2, omega x2, details, U, V, g, w, basis (m+1), doubles scratch
    b += c * (8.0 + 2.0 * es + 5.0 * es + es * m1 + 8.0);
    // ghost rows: length, ready flag, dd_row_max(p) indices and weights; ghost basis values
    b += cg * (8.0 + (4.0 + 8.0) * dd_row_max(cfg.p == 0 ? 2 : cfg.p) + es * m1) + 4.0;
    return b;
}

double wrc::run_device_bytes(const wrc_run* R) {
    const wrc_config& cfg = R->cfg;
    const double N = (double)R->N;
    const double es = (double)R->es;
    const double m1 = cfg.krylov_m + 1;
    const double nblk = std::ceil(N / kTile);
    double b = 7.0 * es * N + 6.0 * N + 8.0 * N + 8.0 * nblk * kMaxKeys + (double)R->lat64.bytes;
    b += 4.0 * es * R->g.NJ + 16.0 * R->g.NJ;
    b += 8.0 * (m1 * cfg.krylov_m + 33) +
         8.0 * (double)std::max(krylov_partials_doubles(R->max_blocks), (size_t)kMaxBlocks * 4);
    const DevBuf* bufs[] = {&R->meta[0], &R->meta[1], &R->omega[0], &R->omega[1], &R->Ua, &R->Va, &R->ga,
                            &R->det, &R->w, &R->basis, &R->tmp, &R->row_len, &R->row_ready, &R->row_idx, &R->row_w,
                            &R->Gb, &R->rows};
    for (const DevBuf* d : bufs) b += (double)d->bytes;
    return b;
}

double wrc::run_updates(const wrc_run* R) { return R->updates; }

bool wrc::run_nonfinite(const wrc_run* R) { return R->nonfinite; }

// ============================================================================
// Batched ensemble
// ============================================================================

struct wrc_ensemble {
    BatchCtx C;
    std::vector<wrc_run*> members;
    long long nstep = 0;
    std::string err;
};

namespace {

thread_local std::string g_ens_create_error;

wrc_status efail(wrc_ensemble* E, wrc_status s, const std::string& msg) {
    if (E) E->err = msg;
    return s;
}

long long ensemble_active(const wrc_ensemble* E) {
    long long tot = 0;
    for (const wrc_run* R : E->members) tot += R->n_active;
    return tot;
}

}  // namespace

extern "C" {

wrc_status wrc_ensemble_create(int32_t n, const wrc_config* cfgs, void* cuda_stream, wrc_ensemble** out) {
    if (!out) return WRC_ERR_ARG;
    *out = nullptr;
    if (n < 1 || !cfgs) {
        g_ens_create_error = "need at least one member configuration";
        return WRC_ERR_ARG;
    }
    for (int i = 0; i < n; ++i)
        if (cfgs[i].model != WRC_MODEL_VORTICITY) {
            g_ens_create_error = "the batched ensemble runs the vorticity form only";
            return WRC_ERR_ARG;
        }
    for (int i = 1; i < n; ++i)
        if (cfgs[i].prec != cfgs[0].prec || (cfgs[i].p == 0 ? 2 : cfgs[i].p) != (cfgs[0].p == 0 ? 2 : cfgs[0].p)) {
            g_ens_create_error = "all members of an ensemble share one precision and one DD order";
            return WRC_ERR_ARG;
        }
    wrc_ensemble* E = new wrc_ensemble();
    auto cleanup = [&](wrc_status st, const std::string& msg) {
        g_ens_create_error = msg;
        wrc_ensemble_destroy(E);
        return st;
    };
    if (batch_init(E->C, (cudaStream_t)cuda_stream, std::min(kBatchStreams, (int)n), cfgs[0].prec == WRC_MIXED,
                   cfgs[0].p == 0 ? 2 : cfgs[0].p) !=
        WRC_OK)
        return cleanup(WRC_ERR_CUDA, E->C.err);
    const int S = (int)E->C.streams.size();
    for (int i = 0; i < n; ++i) {
        wrc_run* R = nullptr;
        const wrc_status st = wrc_create(&cfgs[i], E->C.streams[i % S], &R);
        if (st != WRC_OK) return cleanup(st, "member " + std::to_string(i) + ": " + g_create_error);
        E->members.push_back(R);
    }
    *out = E;
    return WRC_OK;
}

wrc_status wrc_ensemble_member(wrc_ensemble* E, int32_t member, wrc_run** run) {
    if (!E || !run) return WRC_ERR_ARG;
    if (member < 0 || member >= (int)E->members.size()) return efail(E, WRC_ERR_ARG, "member index out of range");
    *run = E->members[member];
    return WRC_OK;
}

wrc_status wrc_ensemble_step(wrc_ensemble* E, int32_t nsteps) {
    if (!E) return WRC_ERR_ARG;
    if (nsteps < 0) return efail(E, WRC_ERR_ARG, "nsteps < 0");
    for (size_t i = 0; i < E->members.size(); ++i)
        if (!E->members[i]->init)
            return efail(E, WRC_ERR_STATE, "member " + std::to_string(i) + " has no initial condition");
    for (int q = 0; q < nsteps; ++q) {
        const wrc_status st = batch_step(E->C, E->members, nullptr);
        if (st != WRC_OK) return efail(E, st, E->C.err);
        E->nstep += 1;
    }
    return WRC_OK;
}

wrc_status wrc_ensemble_set_shape(wrc_ensemble* E, int32_t threads_per_block, int32_t points_per_thread) {
    if (!E) return WRC_ERR_ARG;
    if ((threads_per_block != 64 && threads_per_block != 128 && threads_per_block != 256) || points_per_thread < 1 ||
        points_per_thread > 64)
        return efail(E, WRC_ERR_ARG, "threads_per_block must be 64, 128 or 256; points_per_thread 1..64");
    E->C.pt = threads_per_block;
    E->C.ept = points_per_thread;
    return WRC_OK;
}

wrc_status wrc_ensemble_tune(wrc_ensemble* E, int32_t steps_per_candidate, int32_t out_shape[2]) {
    if (!E) return WRC_ERR_ARG;
    if (steps_per_candidate < 1) return efail(E, WRC_ERR_ARG, "steps_per_candidate < 1");
    const long long nmem = (long long)E->members.size(), nact = ensemble_active(E);
    int cpt = 0, cept = 0;
    if (tuned_shape(E->C.fp32, nmem, nact, cpt, cept)) {
        E->C.pt = cpt;
        E->C.ept = cept;
        if (out_shape) {
            out_shape[0] = cpt;
            out_shape[1] = cept;
        }
        return WRC_OK;
    }
    const int pts[3] = {64, 128, 256};
    const int epts[3] = {1, 2, 4};
    double best = 1e300;
    int bpt = E->C.pt, bept = E->C.ept;
    batch_take_profile(E->C);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            // a shape needs one co-resident block per member at least
            if (krylov_batch_max_blocks(E->C.fp32, E->C.P, pts[a]) < (int)E->members.size()) continue;
            E->C.pt = pts[a];
            E->C.ept = epts[b];
            E->C.profiling = true;
            TRY(wrc_ensemble_step(E, steps_per_candidate));
            const double ms = batch_take_profile(E->C);
            E->C.profiling = false;
            if (ms < best) {
                best = ms;
                bpt = pts[a];
                bept = epts[b];
            }
        }
    E->C.pt = bpt;
    E->C.ept = bept;
    store_tuned_shape(E->C.fp32, nmem, nact, bpt, bept);
    if (out_shape) {
        out_shape[0] = bpt;
        out_shape[1] = bept;
    }
    return WRC_OK;
}

wrc_status wrc_ensemble_stats(wrc_ensemble* E, int64_t out[6]) {
    if (!E || !out) return WRC_ERR_ARG;
    out[0] = (int64_t)E->members.size();
    out[1] = ensemble_active(E);
    out[2] = E->nstep;
    out[3] = E->C.last_blocks;
    out[4] = E->C.pt;
    out[5] = E->C.ept;
    return WRC_OK;
}

wrc_status wrc_ensemble_profile(wrc_ensemble* E, int32_t enable, double* ms_out) {
    if (!E) return WRC_ERR_ARG;
    const double ms = batch_take_profile(E->C);
    if (ms_out) *ms_out = ms;
    E->C.profiling = enable != 0;
    return WRC_OK;
}

const char* wrc_ensemble_last_error(const wrc_ensemble* E) { return E ? E->err.c_str() : g_ens_create_error.c_str(); }

void wrc_ensemble_destroy(wrc_ensemble* E) {
    if (!E) return;
    if (E->C.main) cudaStreamSynchronize(E->C.main);
    for (cudaStream_t st : E->C.streams) cudaStreamSynchronize(st);
    for (wrc_run* R : E->members) wrc_destroy(R);
    batch_free(E->C);
    delete E;
}

}  // extern "C"
