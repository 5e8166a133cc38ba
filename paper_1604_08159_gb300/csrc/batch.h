// Stepping several runs together, shared by the batched ensemble and the
// request server: each run's freeze and adaptation phases replay as its own
// CUDA graphs on one of a few shared streams, and the Krylov part of all the
// runs of one bulk precision and DD order goes into ONE cooperative launch whose blocks
// are shared out in proportion to their active counts.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/wrc.h"
#include "kernels.h"

namespace wrc {

struct BatchCtx {
    cudaStream_t main = nullptr;             // the batched Krylov launch
    bool own_main = false;
    std::vector<cudaStream_t> streams;       // run streams (owned)
    std::vector<cudaEvent_t> ev_streams;
    cudaEvent_t ev_main = nullptr;
    bool fp32 = false;
    int P = 2;                               // DD half-order of the runs (2p = 4, 6, 8)
    int pt = 128;                            // threads per block of the batched kernel
    int ept = 1;                             // target active points per thread
    KrylovStepArgs* h_args = nullptr;        // pinned
    KrylovStepArgs* d_args = nullptr;
    int args_cap = 0;
    int* h_blk = nullptr;                    // pinned: block -> run, then run block offsets
    int* d_blk = nullptr;
    int blk_cap = 0;
    int last_blocks = 0;
    bool profiling = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof;
    std::string err;
};

// Streams (nstreams run streams, and `main`, created when NULL) and events,
// for runs of bulk precision fp32 and DD half-order P.
wrc_status batch_init(BatchCtx& C, cudaStream_t main, int nstreams, bool fp32, int P);
void batch_free(BatchCtx& C);

// One step of every run in `runs` (all of C's bulk precision and DD order, each created on
// one of C.streams and initialised).  per_run (may be NULL) receives each
// run's status: a run whose phase fails is left out of the later phases of
// this step and the others carry on; a failure that is not one run's (the
// batched launch, a stream wait) fails every run.  Returns the first failure,
// explained in C.err.
wrc_status batch_step(BatchCtx& C, const std::vector<wrc_run*>& runs, std::vector<wrc_status>* per_run);

// Device time of the batched launches recorded while C.profiling, since the
// last call (synchronises C.main); clears the record.
double batch_take_profile(BatchCtx& C);

// Autotuned block shape for (precision, run count, total active points), as
// stored by the ensemble autotuner in this process; false when none is.
bool tuned_shape(bool fp32, long long runs, long long active, int& pt, int& ept);
void store_tuned_shape(bool fp32, long long runs, long long active, int pt, int ept);

// The checks wrc_create makes on a configuration (why explains a failure).
bool valid_run_config(const wrc_config* cfg, std::string& why);

// Device bytes of a run of configuration cfg holding grids of up to na active
// and ng ghost points (the allocations wrc_create makes plus the compact and
// ghost arrays at the capacity the run would grow them to).
double run_bytes_for(const wrc_config& cfg, long long na, long long ng);
// Device bytes the run holds now.
double run_device_bytes(const wrc_run* R);
// Sum of the active count over the run's steps so far (active-point updates).
double run_updates(const wrc_run* R);
// True once a step of the run met a non-finite Arnoldi coefficient (known at
// the host synchronisation of that step's grid rebuild).
bool run_nonfinite(const wrc_run* R);

}  // namespace wrc
