// Request server (the wrc_server_* calls of include/wrc.h): runs of any
// lattice and parameters arrive over time; a worker thread admits them in
// arrival order within a slot count and an HBM budget, keeps each admitted
// run's adaptive-grid state on the device, and advances all resident runs
// one step per iteration -- the runs of each bulk precision in one batched
// step, so that runs join and leave the batch between steps (continuous
// batching).  The plain per-run form (one run at a time, wrc_step) is the
// FIFO policy.  Clients only touch host data under the server's mutex; every
// CUDA call is made by the worker thread.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/wrc.h"
#include "batch.h"

using namespace wrc;

namespace {

using Clock = std::chrono::steady_clock;

constexpr int kServerStreams = 8;
constexpr int kMaxSlots = 1024;

struct Request {
    int64_t id = 0;
    wrc_config cfg{};
    std::vector<double> xc, yc, gamma, s;
    int64_t nsteps = 0;
    double estimate = 0.0;
    wrc_request_info info{};
    std::string err;
    std::vector<int32_t> idx;     // final active set (DONE)
    std::vector<double> omega;
    wrc_run* run = nullptr;       // worker thread only
    bool failed = false;          // worker thread only: retire as failed
    wrc_status fail_status = WRC_OK;
    std::string fail_msg;
};

thread_local std::string g_srv_create_error;

// Active-count bound of the admission estimate: all level-0 points and the
// adjacent zones of a few vortices fit in 8192 points up to NJ = 128; beyond,
// a sixteenth of the lattice (the Gaussian-vortex grids at eps = 1e-4 hold
// under 2% of a 1024^2 and 0.2% of a 4096^2 lattice).
double na_bound(const wrc_config& c) {
    const double NJ = (double)((long long)c.n0 << c.J);
    return std::min(NJ * NJ, 8192.0 + NJ * NJ / 16.0);
}

double estimate_bytes(const wrc_config& c) {
    const long long na = (long long)na_bound(c);
    return run_bytes_for(c, na, na / 2);
}

}  // namespace

struct wrc_server {
    wrc_server_config cfg{};
    int device = 0;
    Clock::time_point t0;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    bool fatal = false;
    std::string err;
    int64_t next_id = 0;
    std::map<int64_t, std::unique_ptr<Request>> reqs;
    std::deque<Request*> queue;   // not admitted yet, by (arrival, id)
    double charged = 0.0, peak_charged = 0.0;
    int64_t resident = 0, peak_resident = 0;
    int64_t n_submitted = 0, n_done = 0, n_failed = 0;
    int64_t iterations = 0;
    double updates = 0.0;
    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

void finish(wrc_server* S, Request* q, bool ok, wrc_status st, const std::string& msg) {
    std::lock_guard<std::mutex> lk(S->mu);
    if (q->info.state == WRC_REQ_RUNNING) {
        S->resident -= 1;
        S->charged -= q->info.charged_bytes;
        if (S->resident == 0) S->charged = 0.0;   // no rounding drift across runs
    }
    q->info.state = ok ? WRC_REQ_DONE : WRC_REQ_FAILED;
    q->info.status = ok ? WRC_OK : st;
    q->info.t_done = S->now();
    q->err = msg;
    if (ok) S->n_done += 1;
    else S->n_failed += 1;
    S->cv_done.notify_all();
}

// A resident run leaves: on success its status, diagnostics and active set
// are read back; then its device memory is freed.
void retire(wrc_server* S, Request* q) {
    wrc_run* R = q->run;
    wrc_status st = q->failed ? q->fail_status : WRC_OK;
    std::string msg = q->fail_msg;
    double d[9] = {0};
    int64_t na = 0, ng = 0;
    std::vector<int32_t> idx;
    std::vector<double> om;
    if (st == WRC_OK) st = wrc_sync(R, -1);
    if (st == WRC_OK) st = wrc_diagnostics(R, d);
    if (st == WRC_OK) st = wrc_query_counts(R, &na, &ng, nullptr);
    if (st == WRC_OK) {
        idx.resize((size_t)na);
        om.resize((size_t)na);
        st = wrc_query_active(R, idx.data(), om.data(), na, 0);
    }
    if (st != WRC_OK && msg.empty()) msg = wrc_last_error(R);
    const double upd = run_updates(R);
    int64_t stats[4] = {0};
    wrc_query_stats(R, stats);
    wrc_destroy(R);
    q->run = nullptr;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        q->info.steps = stats[1];
        q->info.updates = upd;
        if (st == WRC_OK) {
            q->info.n_active = na;
            q->info.n_ghost = ng;
            for (int k = 0; k < 4; ++k) q->info.diag[k] = d[k];
            q->info.time = d[4];
            q->idx.swap(idx);
            q->omega.swap(om);
        }
    }
    finish(S, q, st == WRC_OK, st, msg);
}

int64_t run_steps(wrc_run* R) {
    int64_t stats[4] = {0};
    wrc_query_stats(R, stats);
    return stats[1];
}

// Block shape of one batched step of `runs`: the server's, else the
// autotuned one for this precision and size, else 128 x 1; 64 threads when
// more runs than co-resident blocks of the chosen shape.
void pick_shape(const wrc_server* S, BatchCtx& C, const std::vector<wrc_run*>& runs) {
    int pt = 128, ept = 1;
    if (S->cfg.threads_per_block > 0) {
        pt = S->cfg.threads_per_block;
        ept = S->cfg.points_per_thread;
    } else {
        long long act = 0;
        int64_t st[4];
        for (wrc_run* R : runs) {
            wrc_query_stats(R, st);
            act += st[3];
        }
        int tpt = 0, tept = 0;
        if (tuned_shape(C.fp32, (long long)runs.size(), act, tpt, tept)) {
            pt = tpt;
            ept = tept;
        }
    }
    if ((int)runs.size() > krylov_batch_max_blocks(C.fp32, C.P, pt)) pt = 64;
    C.pt = pt;
    C.ept = ept;
}

void serve(wrc_server* S) {
    cudaSetDevice(S->device);
    // one batch context per (precision, DD order): group g = 3 fp32 + (p - 2)
    constexpr int kGroups = 6;
    BatchCtx ctx[kGroups];
    bool ctx_ok[kGroups] = {false, false, false, false, false, false};
    auto group_of = [](const wrc_config& c) { return 3 * (c.prec == WRC_MIXED ? 1 : 0) + ((c.p == 0 ? 2 : c.p) - 2); };
    std::vector<Request*> res;   // resident runs, in admission order
    bool hold = false;           // device out of memory: admit nothing until a run leaves
    unsigned rr = 0;
    const bool fifo = S->cfg.policy == WRC_SERVE_FIFO;
    const size_t slots = fifo ? 1 : (size_t)S->cfg.max_slots;
    for (;;) {
        std::vector<Request*> admit;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            for (;;) {
                if (S->stop) break;
                if (res.empty()) hold = false;
                const double now = S->now();
                while (!hold && !S->queue.empty() && res.size() + admit.size() < slots) {
                    Request* q = S->queue.front();
                    if (q->info.t_arrival > now) break;
                    if (S->charged + q->estimate > S->cfg.hbm_budget_bytes) break;
                    S->queue.pop_front();
                    S->charged += q->estimate;
                    q->info.charged_bytes = q->estimate;
                    q->info.state = WRC_REQ_RUNNING;
                    q->info.t_admit = now;
                    S->resident += 1;
                    admit.push_back(q);
                }
                S->peak_charged = std::max(S->peak_charged, S->charged);
                S->peak_resident = std::max(S->peak_resident, S->resident);
                if (!res.empty() || !admit.empty()) break;
                if (S->queue.empty()) {
                    S->cv_work.wait(lk);
                } else {
                    const double wait = std::max(1e-4, S->queue.front()->info.t_arrival - now);
                    S->cv_work.wait_for(lk, std::chrono::duration<double>(wait));
                }
            }
            if (S->stop) break;   // (nothing was admitted in this pass)
        }
        // create and initialise the admitted runs
        for (size_t a = 0; a < admit.size(); ++a) {
            Request* q = admit[a];
            const int g = group_of(q->cfg);
            wrc_status st = WRC_OK;
            std::string msg;
            if (!ctx_ok[g]) {
                st = batch_init(ctx[g], nullptr, kServerStreams, g >= 3, 2 + g % 3);
                if (st == WRC_OK) ctx_ok[g] = true;
                else msg = ctx[g].err;
            }
            wrc_run* R = nullptr;
            if (st == WRC_OK) {
                st = wrc_create(&q->cfg, ctx[g].streams[rr++ % kServerStreams], &R);
                if (st != WRC_OK) msg = wrc_last_error(nullptr);
            }
            if (st == WRC_OK) {
                st = wrc_init_vortices(R, (int32_t)q->xc.size(), q->xc.data(), q->yc.data(), q->gamma.data(),
                                       q->s.data());
                if (st != WRC_OK) {
                    msg = wrc_last_error(R);
                    wrc_destroy(R);
                    R = nullptr;
                }
            }
            if (st == WRC_ERR_OOM && !res.empty()) {
                // wait for a resident run to leave: this and the later ones go back
                std::lock_guard<std::mutex> lk(S->mu);
                for (size_t b = admit.size(); b-- > a;) {
                    Request* r = admit[b];
                    S->resident -= 1;
                    S->charged -= r->info.charged_bytes;
                    r->info.state = WRC_REQ_QUEUED;
                    r->info.t_admit = -1.0;
                    S->queue.push_front(r);
                }
                hold = true;
                break;
            }
            if (st != WRC_OK) {
                finish(S, q, false, st, "admission: " + msg);
                continue;
            }
            q->run = R;
            {
                std::lock_guard<std::mutex> lk(S->mu);
                const double held = run_device_bytes(R);
                if (held > q->info.charged_bytes) {
                    S->charged += held - q->info.charged_bytes;
                    q->info.charged_bytes = held;
                }
                S->peak_charged = std::max(S->peak_charged, S->charged);
            }
            res.push_back(q);
        }
        if (res.empty()) continue;
        // one step of every resident run that has steps left
        double upd0 = 0.0;
        for (Request* q : res) upd0 += run_updates(q->run);
        bool stepped = false;
        if (fifo) {
            Request* q = res.front();
            if (run_steps(q->run) < q->nsteps) {
                const wrc_status st = wrc_step(q->run, 1);
                if (st != WRC_OK) {
                    q->failed = true;
                    q->fail_status = st;
                    q->fail_msg = wrc_last_error(q->run);
                }
                stepped = true;
            }
        } else {
            for (int g = 0; g < kGroups; ++g) {
                std::vector<wrc_run*> runs;
                std::vector<Request*> who;
                for (Request* q : res)
                    if (group_of(q->cfg) == g && run_steps(q->run) < q->nsteps) {
                        runs.push_back(q->run);
                        who.push_back(q);
                    }
                if (runs.empty()) continue;
                pick_shape(S, ctx[g], runs);
                std::vector<wrc_status> rs;
                batch_step(ctx[g], runs, &rs);
                for (size_t i = 0; i < runs.size(); ++i)
                    if (rs[i] != WRC_OK) {
                        who[i]->failed = true;
                        who[i]->fail_status = rs[i];
                        who[i]->fail_msg = wrc_last_error(runs[i]);
                    }
                stepped = true;
            }
        }
        for (Request* q : res)
            if (!q->failed && run_nonfinite(q->run)) {
                q->failed = true;
                q->fail_status = WRC_ERR_BREAKDOWN_NAN;
                q->fail_msg = "non-finite value in the Arnoldi process";
            }
        // retire finished and failed runs; charge growth of the others
        double upd1 = 0.0;
        bool device_error = false;
        std::vector<Request*> keep;
        for (Request* q : res) {
            upd1 += run_updates(q->run);
            if (q->failed || run_steps(q->run) >= q->nsteps) {
                device_error = device_error || (q->failed && q->fail_status == WRC_ERR_CUDA);
                retire(S, q);
                hold = false;   // memory was freed
            } else {
                keep.push_back(q);
                std::lock_guard<std::mutex> lk(S->mu);
                const double held = run_device_bytes(q->run);
                if (held > q->info.charged_bytes) {
                    S->charged += held - q->info.charged_bytes;
                    q->info.charged_bytes = held;
                    S->peak_charged = std::max(S->peak_charged, S->charged);
                }
                q->info.steps = run_steps(q->run);
            }
        }
        res.swap(keep);
        // after a CUDA failure: a sticky device error (the context is lost)
        // ends the server; any other is cleared and serving goes on
        cudaError_t sticky = cudaSuccess;
        if (device_error) {
            cudaGetLastError();
            sticky = cudaDeviceSynchronize();
        }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            if (stepped) S->iterations += 1;
            S->updates += upd1 - upd0;
            if (sticky != cudaSuccess) {
                S->fatal = true;
                S->err = std::string("device error: ") + cudaGetErrorString(sticky);
            }
            if (S->fatal) break;
        }
    }
    // stop: fail what is left
    for (Request* q : res) {
        if (q->run) wrc_destroy(q->run);
        q->run = nullptr;
        finish(S, q, false, WRC_ERR_STATE, "server stopped");
    }
    std::deque<Request*> left;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        left.swap(S->queue);
    }
    for (Request* q : left) finish(S, q, false, WRC_ERR_STATE, "server stopped");
    for (int g = 0; g < kGroups; ++g)
        if (ctx_ok[g]) batch_free(ctx[g]);
}

Request* find_req(wrc_server* S, int64_t id) {
    auto it = S->reqs.find(id);
    return it == S->reqs.end() ? nullptr : it->second.get();
}

}  // namespace

extern "C" {

wrc_status wrc_server_estimate(const wrc_config* cfg, double* bytes) {
    std::string why;
    if (!bytes || !valid_run_config(cfg, why)) return WRC_ERR_ARG;
    *bytes = estimate_bytes(*cfg);
    return WRC_OK;
}

wrc_status wrc_server_create(const wrc_server_config* cfg, wrc_server** out) {
    if (!out) return WRC_ERR_ARG;
    *out = nullptr;
    auto bad = [](const char* why) {
        g_srv_create_error = why;
        return WRC_ERR_ARG;
    };
    if (!cfg) return bad("cfg is NULL");
    if (cfg->policy != WRC_SERVE_BATCHED && cfg->policy != WRC_SERVE_FIFO) return bad("unknown policy");
    if (cfg->max_slots < 1 || cfg->max_slots > kMaxSlots) return bad("max_slots must be in 1..1024");
    const int tpb = cfg->threads_per_block, ppt = cfg->points_per_thread;
    if (!((tpb == 0 && ppt == 0) || ((tpb == 64 || tpb == 128 || tpb == 256) && ppt >= 1 && ppt <= 64)))
        return bad("threads_per_block 64/128/256 with points_per_thread 1..64, or both 0");
    if (!(cfg->hbm_budget_bytes > 0) || !std::isfinite(cfg->hbm_budget_bytes)) return bad("hbm_budget_bytes must be > 0");
    if (cfg->policy == WRC_SERVE_BATCHED) {
        // every resident run needs one block of the batched launch at least
        for (int f = 0; f < 2 * 3; ++f) {
            const int lim = krylov_batch_max_blocks(f >= 3, 2 + f % 3, 64);
            if (lim <= 0) {
                g_srv_create_error = "batched Krylov kernel occupancy query failed";
                return WRC_ERR_CUDA;
            }
            if (cfg->max_slots > lim) return bad("max_slots exceeds the co-resident blocks of the batched kernel");
        }
    }
    wrc_server* S = new wrc_server();
    S->cfg = *cfg;
    cudaGetDevice(&S->device);
    S->t0 = Clock::now();
    try {
        S->worker = std::thread(serve, S);
    } catch (...) {
        delete S;
        g_srv_create_error = "could not start the worker thread";
        return WRC_ERR_STATE;
    }
    *out = S;
    return WRC_OK;
}

wrc_status wrc_server_submit(wrc_server* S, const wrc_config* cfg, int32_t nv, const double* xc, const double* yc,
                             const double* gamma, const double* s, int64_t nsteps, double arrival_s, int64_t* id) {
    if (!S || !id) return WRC_ERR_ARG;
    std::string why;
    if (!valid_run_config(cfg, why) || cfg->model != WRC_MODEL_VORTICITY) {
        std::lock_guard<std::mutex> lk(S->mu);
        S->err = "submit: " + (why.empty() ? std::string("the server runs the vorticity form only") : why);
        return WRC_ERR_ARG;
    }
    if (nv < 1 || nv > WRC_MAX_VORTICES || !xc || !yc || !gamma || !s || nsteps < 0 || !std::isfinite(arrival_s)) {
        std::lock_guard<std::mutex> lk(S->mu);
        S->err = "submit: need 1..WRC_MAX_VORTICES vortices, four host arrays, nsteps >= 0";
        return WRC_ERR_ARG;
    }
    for (int v = 0; v < nv; ++v)
        if (!(s[v] > 0) || !std::isfinite(xc[v]) || !std::isfinite(yc[v]) || !std::isfinite(gamma[v])) {
            std::lock_guard<std::mutex> lk(S->mu);
            S->err = "submit: vortex parameters must be finite with s > 0";
            return WRC_ERR_ARG;
        }
    auto q = std::make_unique<Request>();
    q->cfg = *cfg;
    q->xc.assign(xc, xc + nv);
    q->yc.assign(yc, yc + nv);
    q->gamma.assign(gamma, gamma + nv);
    q->s.assign(s, s + nv);
    q->nsteps = nsteps;
    q->estimate = estimate_bytes(*cfg);
    q->info.state = WRC_REQ_QUEUED;
    q->info.t_admit = -1.0;
    q->info.t_done = -1.0;
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->fatal || S->stop) {
        S->err = "submit: the server has stopped";
        return WRC_ERR_STATE;
    }
    if (q->estimate > S->cfg.hbm_budget_bytes) {
        S->err = "submit: the run's estimate exceeds the whole HBM budget";
        return WRC_ERR_BUSY;
    }
    q->id = S->next_id++;
    q->info.t_arrival = std::max(arrival_s, S->now());
    Request* r = q.get();
    S->reqs[r->id] = std::move(q);
    auto pos = S->queue.end();
    while (pos != S->queue.begin() && (*(pos - 1))->info.t_arrival > r->info.t_arrival) --pos;
    S->queue.insert(pos, r);
    S->n_submitted += 1;
    *id = r->id;
    S->cv_work.notify_all();
    return WRC_OK;
}

wrc_status wrc_server_query(wrc_server* S, int64_t id, wrc_request_info* out) {
    if (!S || !out) return WRC_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    Request* q = find_req(S, id);
    if (!q) return WRC_ERR_ARG;
    *out = q->info;
    return WRC_OK;
}

wrc_status wrc_server_result_active(wrc_server* S, int64_t id, int32_t* idx_out, double* omega_out, int64_t cap) {
    if (!S) return WRC_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    Request* q = find_req(S, id);
    if (!q) return WRC_ERR_ARG;
    if (q->info.state != WRC_REQ_DONE) return WRC_ERR_STATE;
    const int64_t n = (int64_t)q->idx.size();
    if (cap < n) return WRC_ERR_ARG;
    if (idx_out && n) std::memcpy(idx_out, q->idx.data(), sizeof(int32_t) * n);
    if (omega_out && n) std::memcpy(omega_out, q->omega.data(), sizeof(double) * n);
    return WRC_OK;
}

wrc_status wrc_server_request_error(wrc_server* S, int64_t id, char* buf, int64_t cap) {
    if (!S || !buf || cap < 1) return WRC_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    Request* q = find_req(S, id);
    if (!q) return WRC_ERR_ARG;
    const size_t n = std::min((size_t)(cap - 1), q->err.size());
    std::memcpy(buf, q->err.data(), n);
    buf[n] = 0;
    return WRC_OK;
}

wrc_status wrc_server_wait(wrc_server* S, int64_t id, double timeout_s) {
    if (!S || !(timeout_s >= 0)) return WRC_ERR_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    if (id != -1 && !find_req(S, id)) return WRC_ERR_ARG;
    auto done = [&] {
        if (id == -1) return S->n_done + S->n_failed >= S->n_submitted;
        const Request* q = find_req(S, id);
        return !q || q->info.state >= WRC_REQ_DONE;
    };
    const double t = std::min(timeout_s, 1e7);
    if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(t), done)) return WRC_ERR_TIMEOUT;
    return WRC_OK;
}

wrc_status wrc_server_release(wrc_server* S, int64_t id) {
    if (!S) return WRC_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    Request* q = find_req(S, id);
    if (!q) return WRC_ERR_ARG;
    if (q->info.state < WRC_REQ_DONE) return WRC_ERR_STATE;
    S->reqs.erase(id);
    return WRC_OK;
}

wrc_status wrc_server_stats(wrc_server* S, double out[12]) {
    if (!S || !out) return WRC_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    out[0] = (double)S->n_submitted;
    out[1] = (double)S->n_done;
    out[2] = (double)S->n_failed;
    out[3] = (double)S->queue.size();
    out[4] = (double)S->resident;
    out[5] = (double)S->peak_resident;
    out[6] = S->charged;
    out[7] = S->peak_charged;
    out[8] = (double)S->iterations;
    out[9] = S->updates;
    out[10] = S->now();
    out[11] = S->fatal ? 1.0 : 0.0;
    return WRC_OK;
}

const char* wrc_server_last_error(const wrc_server* S) { return S ? S->err.c_str() : g_srv_create_error.c_str(); }

void wrc_server_destroy(wrc_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    delete S;
}

}  // extern "C"
