// The library context (opaque to callers of pf.h).
#pragma once
#include <cstdarg>
#include <cstdint>
#include <mutex>
#include <string>

#include <cuda_runtime.h>

#include "pf.h"
#include "pf_internal.cuh"
#include "pf_kernels.h"

namespace pf {

struct Scratch {
    int64_t *order, *idx, *n_idx, *tiles, *bin_start;
    unsigned long long *work, *hist, *cursor;
    int *ident;
    uint8_t *need;   // pairs left to verify (see FilterArgs::need)
};

struct ServeState;

constexpr int kSideStreams = 4;

int pf_default_cfg(int E);

}  // namespace pf

struct pf_ctx {
    int device = 0;
    int sms = 0;
    cudaStream_t stream = nullptr;
    size_t hbm_budget = 0;

    unsigned *d_err = nullptr;   // device error bits
    unsigned *h_err = nullptr;   // pinned copy read by pf_sync

    std::mutex mu;
    pf_status sticky = PF_OK;
    std::string msg, last_msg;

    void *scratch = nullptr;
    size_t scratch_bytes = 0;

    // tuned kernel per decider set and threshold
    int tune_cfg[4][PF_MAX_E + 1];
    bool tune_plain[4][PF_MAX_E + 1] = {};  // pf_tune found the plain kernel fastest
    int tune_chunk[4][PF_MAX_E + 1];
    // batches of fewer pairs take one plain launch (no binning, no per-bin
    // launches); 0 sends every batch through the batched scheduler
    int64_t small_batch = int64_t(1) << 20;
    bool resolve_bounds = true;  // skip verifying pairs whose count bounds agree
    // what pf_last_verified_count reads: 0 nothing, 1 the count at the start
    // of scratch, 2 zero (the last pf_filter_verify had no pairs)
    int verified_state = 0;
    int grid_cache[4][pf::kNumBatchCfgs] = {};
    // the last run_filter grouped its pairs: the scratch's order (unless
    // *ident) lists them by configuration and length class
    bool binned = false;

    cudaStream_t side_streams[pf::kSideStreams] = {};
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_join[pf::kSideStreams] = {};

    pf::ServeState *serve = nullptr;

    pf_status fail(pf_status s, const char *fmt, ...);
    pf_status cuda(cudaError_t e, const char *what);
    pf_status ensure_scratch(size_t bytes);
    pf_status scratch_layout(int64_t n, pf::Scratch *s);
    int grid_for(int dec, int cfg);
    void reset_tuning();
    pf_status run_batched(unsigned dec, const pf::FilterArgs &a, const pf::Scratch &s);
    // run_batched, or one plain launch for a batch below small_batch
    pf_status run_filter(unsigned dec, const pf::FilterArgs &a, const pf::Scratch &s);
};

void pf_serve_teardown(pf_ctx *ctx);
