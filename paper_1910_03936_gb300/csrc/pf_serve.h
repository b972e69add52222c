// Serving (a8): types shared by the two modes of the request loop.
// pf_serve.cu holds the device-resident loop and the public calls,
// pf_serve_batch.cu the batched mode.  Contracts: pf.h.
#pragma once
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "pf_ctx.h"

namespace pf {

// Per-slot request descriptor, in device memory (uploaded with the request).
struct ServeDesc {
    const uint8_t *reads, *refs;
    const int64_t *byte_off;   // the caller's offsets (not rebased)
    int64_t *word_off;         // filled by the loop, chunk by chunk
    const int16_t *E;
    uint32_t *rlo, *rhi, *rnm, *flo, *fhi, *fnm;
    uint8_t *accept;
    int16_t *count;
    int32_t *dist;
    unsigned *err;
    int64_t n;
    int chunk, nchunks;
    unsigned deciders;
    unsigned epoch;
};

struct ServeDevice {
    const ServeDesc *desc;            // [max_requests], device
    unsigned *done;                   // [max_requests], device: chunks finished
    unsigned long long *head;         // device: next item to claim
    const unsigned long long *items;  // mapped host ring
    const unsigned long long *tail;   // mapped host: items published
    const unsigned *stop;             // mapped host
    unsigned *complete;               // mapped host [max_requests]: epoch of the finished request
    unsigned long long *last_claim;   // device: globaltimer of the latest claim, any block
    unsigned long long *dev_tail;     // device: mirror of *tail
    unsigned long long *last_poll;    // device: globaltimer of the latest mirror refresh
    unsigned *dev_exit;               // device: set by a block that finds the loop idle or stopped
    unsigned long long idle_ns;
};

struct BatchPool;  // batched mode (pf_serve_batch.cu)


struct ServeReq {
    uint64_t ticket = 0;
    pf_request req{};
    int slot = -1;
    size_t off = 0, bytes = 0;     // device arena
    size_t hoff = 0, hbytes = 0;   // pinned staging arena
    int64_t total_bytes = 0, total_words = 0;
    int nchunks = 0;
    unsigned epoch = 0;
    enum State { PENDING, STAGING, RUNNING, DRAINING, DONE } state = PENDING;
    cudaEvent_t ev = nullptr;
    using tp = std::chrono::steady_clock::time_point;
    tp t_submit, t_admit, t_pub, t_seen, t_done;
    pf_status status = PF_OK;
    // pinned staging pieces
    int64_t *h_boff = nullptr;
    int16_t *h_E = nullptr;
    uint8_t *h_acc = nullptr;
    int16_t *h_cnt = nullptr;
    int32_t *h_dist = nullptr;
    unsigned *h_err = nullptr;
    // batched mode: the request is placed into device batches in parts
    int64_t next = 0;              // pairs placed so far
    int parts = 0, parts_done = 0;
    unsigned dev_err = 0;          // device error bits of its finished parts
    int E_max = 0;                 // the largest threshold of its pairs
    int64_t longest = 0;           // its longest pair, bytes
    bool admitted = false;
    // device-visible views: page-locked inputs read in place (else copied
    // into the batch slot), outputs written in place (else pinned staging)
    const int64_t *d_boff = nullptr;
    const int16_t *d_E = nullptr;
    uint8_t *d_acc = nullptr;
    int16_t *d_cnt = nullptr;
    int32_t *d_dist = nullptr;
    bool in_mapped = false, out_mapped = false;
};

// First-fit allocator over [0, size) for the two arenas.
struct Arena {
    std::map<size_t, size_t> free_list;  // offset -> size
    void reset(size_t size) {
        free_list.clear();
        if (size) free_list[0] = size;
    }
    bool alloc(size_t bytes, size_t *off) {
        for (auto it = free_list.begin(); it != free_list.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t o = it->first + bytes;
                free_list.erase(it);
                if (rest) free_list[o] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        auto it = free_list.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_list.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_list.erase(nx);
        }
        if (it != free_list.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_list.erase(it);
            }
        }
    }
};

struct ServeState {
    pf_serve_config cfg{};
    pf_ctx *ctx = nullptr;         // the serving context (for its tuning table)
    BatchPool *bp = nullptr;       // batched mode
    int device = 0;
    size_t budget = 0, stage_budget = 0;
    char *arena = nullptr;         // device
    char *stage_mem = nullptr;     // pinned host
    Arena dev_arena, host_arena;
    ServeDesc *d_desc = nullptr;
    ServeDesc *h_desc = nullptr;   // pinned staging, one per slot
    unsigned *d_done = nullptr;
    unsigned long long *d_head = nullptr, *d_last = nullptr, *d_tail = nullptr, *d_poll = nullptr;
    unsigned *d_exit = nullptr;
    unsigned long long *h_items = nullptr, *h_tail = nullptr;
    unsigned *h_stop = nullptr, *h_complete = nullptr;
    ServeDevice dev{};
    cudaStream_t s_copy = nullptr, s_loop = nullptr;
    cudaEvent_t ev_loop = nullptr;
    bool loop_running = false;
    std::atomic<bool> paused{false};
    uint64_t published = 0;        // items published (host copy of *h_tail)
    uint64_t inflight_items = 0;

    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_idle;
    bool quit = false;
    int waiters = 0;               // threads inside pf_wait
    std::thread th;
    uint64_t next_ticket = 1;
    std::deque<std::shared_ptr<ServeReq>> pending;
    std::vector<std::shared_ptr<ServeReq>> active;      // admitted, not done
    std::map<uint64_t, std::shared_ptr<ServeReq>> reqs; // every unreleased ticket
    std::vector<int> free_slots;
    std::vector<unsigned> slot_epoch;
    pf_serve_stats stats{};
    std::string fatal;
};

inline size_t up256(size_t x) { return (x + 255) & ~size_t(255); }
inline int slots_of(unsigned deciders) { return deciders == 3u ? 2 : 1; }
inline double secs(ServeReq::tp a, ServeReq::tp b) {
    return std::chrono::duration<double>(b - a).count();
}

// Batched mode, pf_serve_batch.cu.  batch_start allocates the pool (PF_OK or
// a failure status recorded on ctx); batch_prepare sizes a submitted request
// (PF_ENOMEM if it could never be staged); batch_scheduler is the scheduler
// thread's body; batch_stop releases everything after the thread has ended
// (unfinished requests end cancelled).
pf_status batch_start(pf_ctx *ctx, ServeState *S);
pf_status batch_prepare(pf_ctx *ctx, ServeState *S, ServeReq *q);
void batch_scheduler(ServeState *S);
void batch_stop(ServeState *S);
pf_status batch_trace(ServeState *S, double *records, int cap, int *count);

}  // namespace pf
