// a8: serving.  A persistent device loop takes work items (chunks of
// admitted requests) from a ring in mapped host memory; a host scheduler
// thread admits requests by slots, device memory and ring room, stages
// them, publishes their items and returns results.  Contracts: pf.h.
//
// Every device wait is bounded: a block that finds no item sleeps in
// short steps and leaves after idle_exit_us (globaltimer) or when the stop
// flag is set; the scheduler relaunches the loop when new items appear.
// Items are claimed by compare-and-swap on a device head counter only
// after the block has seen them published, so an exiting block never
// drops an item.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#if defined(__linux__)
#include <sys/prctl.h>
#endif

#include "pf_serve.h"
#include "pf_filter.cuh"
#include "pf_pack.cuh"
#include "pf_verify.cuh"

namespace pf {

constexpr int kServeThreads = 256;
constexpr int kServeMaxChunk = 1024;
constexpr int kServeTpp = 8;      // lanes per pair in the loop's filter
constexpr int kServeDpt = 8;      // slots per lane: E <= 31
constexpr uint64_t kRingSize = 1u << 16;


__device__ __forceinline__ unsigned long long ld_acquire_sys(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned ld_relaxed_sys(const unsigned *p) {
    unsigned v;
    asm volatile("ld.relaxed.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_sys64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_sys(unsigned *p, unsigned v) {
    asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned long long *p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// The descriptor of a slot, read through L2: the copy engine rewrites it for
// every request admitted to the slot while the loop runs.
__device__ __forceinline__ ServeDesc load_desc(const ServeDesc *p) {
    static_assert(sizeof(ServeDesc) % 8 == 0, "descriptor is read in 8-byte words");
    ServeDesc d;
    const unsigned long long *src = reinterpret_cast<const unsigned long long *>(p);
    unsigned long long *dst = reinterpret_cast<unsigned long long *>(&d);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(ServeDesc) / 8); ++i) dst[i] = __ldcg(src + i);
    return d;
}

template <int DEC>
__device__ __forceinline__ void serve_filter_chunk(const ServeDesc &d, const PairsView &pv,
                                                   int64_t c0, int64_t c1) {
    const int lane = threadIdx.x & 31;
    const int g = lane & (kServeTpp - 1);
    const unsigned gmask = ((1u << kServeTpp) - 1u) << (lane & ~(kServeTpp - 1));
    const int group = threadIdx.x / kServeTpp;
    constexpr int groups = kServeThreads / kServeTpp;
    FilterArgs a;
    a.pairs = pv;
    a.accept = d.accept;
    a.count = d.count;
    a.n = d.n;
    for (int64_t p = c0 + group; p < c1; p += groups) {
        const int64_t b0 = __ldcg(d.byte_off + p);
        const int m = (int)(__ldcg(d.byte_off + p + 1) - b0);
        const int E = __ldcg(d.E + p);
        if (m < 0 || E < 0 || E > PF_MAX_E) {
            if (g == 0) {
                a.count[p] = -1;
                a.accept[p] = 0;
                if (DEC == 3) {
                    a.count[a.n + p] = -1;
                    a.accept[a.n + p] = 0;
                }
                atomicOr(d.err, ERR_PAIR_ARGS);
            }
            continue;
        }
        PairFilter<kServeTpp, kServeDpt, DEC, -1, LdCG> st;
        st.init(pv, p, m, E);
        st.run(pv, g, gmask);
        int ssc = 0, gkc = 0;
        st.finish(g, gmask, &ssc, &gkc);
        if (g == 0) write_outputs<DEC>(a, p, E, ssc, gkc, st.h);
    }
}

// Before each launch: the idle clock starts now, the exit flag is clear.
__global__ void serve_stamp_kernel(unsigned long long *last_claim, unsigned *dev_exit,
                                   unsigned long long *last_poll) {
    *last_claim = globaltimer_ns();
    *dev_exit = 0u;
    *last_poll = 0ull;
}

// Claiming work.  No block ever waits for another one: every block may
// refresh the device-side mirror of the ring tail from host memory (at most
// one refresh per 2 microseconds across the grid, arbitrated by a
// compare-and-swap on the time of the last refresh), and every block
// decides on its own that the loop is idle: no claim by any block for
// idle_ns and nothing published beyond the head in host memory.  A block
// that finds the loop idle or stopped raises dev_exit so the others leave
// at their next poll.  Returns 1 with *item set, or 0 to leave.
__device__ int serve_claim(const ServeDevice &sd, unsigned long long *item) {
    unsigned nap = 500;
    for (unsigned polls = 0; polls < (1u << 22); ++polls) {
        const unsigned long long t = ld_acquire_gpu(sd.dev_tail);
        const unsigned long long h = *(volatile unsigned long long *)sd.head;
        if (h < t) {
            if (atomicCAS(sd.head, h, h + 1) == h) {
                *item = ld_relaxed_sys64(sd.items + (h % kRingSize));
                atomicMax(sd.last_claim, globaltimer_ns());
                return 1;
            }
            continue;  // another block took it: look again at once
        }
        if (*(volatile unsigned *)sd.dev_exit) return 0;
        const unsigned long long now = globaltimer_ns();
        const unsigned long long lp = *(volatile unsigned long long *)sd.last_poll;
        const unsigned long long last = *(volatile unsigned long long *)sd.last_claim;
        const bool idle = now > last && now - last > sd.idle_ns;
        if (idle || (now > lp + 2000 && atomicCAS(sd.last_poll, lp, now) == lp)) {
            if (ld_relaxed_sys(sd.stop)) {
                atomicExch(sd.dev_exit, 1u);
                return 0;
            }
            const unsigned long long ht = ld_acquire_sys(sd.tail);
            if (ht > t) {
                __threadfence();  // the items the host wrote before ht, then the mirror
                atomicMax(sd.dev_tail, ht);
                nap = 500;
                continue;
            }
            if (idle) {
                atomicExch(sd.dev_exit, 1u);
                return 0;
            }
        }
        __nanosleep(nap);
        nap = nap < 16000 ? nap * 2 : 16000;
    }
    return 0;
}

__global__ void __launch_bounds__(kServeThreads) serve_loop_kernel(ServeDevice sd) {
    __shared__ unsigned long long s_item;
    __shared__ int s_cmd;
    __shared__ int64_t s_woff[kServeMaxChunk + 1];
    __shared__ int64_t s_boff[kServeMaxChunk + 1];
    for (;;) {
        if (threadIdx.x == 0) {
            unsigned long long it = 0;
            s_cmd = serve_claim(sd, &it);
            s_item = it;
        }
        __syncthreads();
        if (s_cmd == 0) return;
        const unsigned long long item = s_item;
        const int slot = (int)(item >> 32);
        const int ci = (int)(item & 0xffffffffu);
        const ServeDesc d = load_desc(sd.desc + slot);  // uploaded before the item was published
        const int64_t c0 = (int64_t)ci * d.chunk;
        const int64_t c1 = min(d.n, c0 + (int64_t)d.chunk);
        const int np = (int)(c1 - c0);

        // ---- pack the chunk's reads and references (a1).  Sequence s of the
        // request starts at word floor(b_s / 32) + s, b_s its byte offset from
        // the request's first byte: never overlapping (floor((b+L)/32) + 1 >=
        // floor(b/32) + ceil(L/32)), computable per chunk without a scan.
        const int64_t b00 = __ldcg(d.byte_off);
        for (int i = threadIdx.x; i <= np; i += blockDim.x) {
            const int64_t b = __ldcg(d.byte_off + c0 + i) - b00;
            s_boff[i] = b;
            s_woff[i] = (b >> 5) + c0 + i;
            if (i < np) d.word_off[c0 + i] = s_woff[i];
        }
        __syncthreads();
        const int64_t wbase = s_woff[0];
        const int wtot = (int)(s_woff[np] - wbase);
        const int64_t btot = __ldcg(d.byte_off + d.n) - b00;  // the request's bytes
        for (int j = threadIdx.x; j < wtot; j += blockDim.x) {
            const int64_t gw = wbase + j;
            int l = 0, r = np - 1;
            while (l < r) {
                const int mid = (l + r + 1) >> 1;
                if (s_woff[mid] <= gw) l = mid; else r = mid - 1;
            }
            const int w = (int)(gw - s_woff[l]);
            const int len = (int)(s_boff[l + 1] - s_boff[l]);
            if (w >= (len + 31) / 32) continue;  // gap word between sequences
            pack_word<LdCG>(d.reads + s_boff[l], len, w, d.rlo + gw, d.rhi + gw, d.rnm + gw, d.err,
                            d.reads + btot);
            pack_word<LdCG>(d.refs + s_boff[l], len, w, d.flo + gw, d.fhi + gw, d.fnm + gw, d.err,
                            d.refs + btot);
        }
        __syncthreads();

        // ---- filter (a2-a4)
        PairsView pv;
        pv.read = SeqView{d.rlo, d.rhi, d.rnm, d.word_off, 0};
        pv.ref = SeqView{d.flo, d.fhi, d.fnm, d.word_off, 0};
        if (d.deciders == 1u) serve_filter_chunk<1>(d, pv, c0, c1);
        else if (d.deciders == 2u) serve_filter_chunk<2>(d, pv, c0, c1);
        else serve_filter_chunk<3>(d, pv, c0, c1);
        __syncthreads();

        // ---- verify the accepted pairs (a5-a6); the first selected
        // decider's flags are slot 0
        for (int64_t p = c0 + threadIdx.x; p < c1; p += blockDim.x) {
            const int E = __ldcg(d.E + p);
            const int m = (int)(s_boff[p - c0 + 1] - s_boff[p - c0]);  // byte offsets
            int32_t v;
            if (m < 0 || E < 0 || E > PF_MAX_E) v = -1;
            else if (__ldcg(d.accept + p)) v = verify_pair<uint64_t, LdCG>(pv, p, m, E);
            else v = E + 1;
            d.dist[p] = v;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned prev = atomicAdd(sd.done + slot, 1u);
            if (prev + 1 == (unsigned)d.nchunks) {
                __threadfence_system();
                st_release_sys(sd.complete + slot, d.epoch);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// host side

namespace {


// Device bytes a request needs in the arena.
size_t request_bytes(const pf_request &r, int64_t total_bytes, int64_t total_words) {
    const size_t n = (size_t)r.n, sl = (size_t)slots_of(r.deciders);
    return up256((size_t)total_bytes) * 2 + up256((n + 1) * 8) * 2 + up256(n * 2) +
           up256((size_t)total_words * 4) * 6 + up256(sl * n) + up256(sl * n * 2) +
           up256(n * 4) + 256;
}

// Pinned staging bytes: offsets and thresholds in, results out.
size_t staging_bytes(const pf_request &r) {
    const size_t n = (size_t)r.n, sl = (size_t)slots_of(r.deciders);
    return up256((n + 1) * 8) + up256(n * 2) + up256(sl * n) + up256(sl * n * 2) +
           up256(n * 4) + 256;
}

void stage(ServeState &S, ServeReq &q) {
    const pf_request &r = q.req;
    const size_t n = (size_t)r.n, sl = (size_t)slots_of(r.deciders);
    char *b = S.arena + q.off;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        char *p = b + o;
        o += up256(bytes);
        return p;
    };
    ServeDesc &d = S.h_desc[q.slot];
    d.reads = reinterpret_cast<uint8_t *>(take((size_t)q.total_bytes));
    d.refs = reinterpret_cast<uint8_t *>(take((size_t)q.total_bytes));
    int64_t *boff = reinterpret_cast<int64_t *>(take((n + 1) * 8));
    d.byte_off = boff;
    d.word_off = reinterpret_cast<int64_t *>(take((n + 1) * 8));
    d.E = reinterpret_cast<int16_t *>(take(n * 2));
    uint32_t *pl[6];
    for (auto &x : pl) x = reinterpret_cast<uint32_t *>(take((size_t)q.total_words * 4));
    d.rlo = pl[0]; d.rhi = pl[1]; d.rnm = pl[2];
    d.flo = pl[3]; d.fhi = pl[4]; d.fnm = pl[5];
    d.accept = reinterpret_cast<uint8_t *>(take(sl * n));
    d.count = reinterpret_cast<int16_t *>(take(sl * n * 2));
    d.dist = reinterpret_cast<int32_t *>(take(n * 4));
    d.err = reinterpret_cast<unsigned *>(take(4));
    d.n = r.n;
    d.chunk = S.cfg.chunk_pairs;
    d.nchunks = q.nchunks;
    d.deciders = r.deciders;
    d.epoch = q.epoch;

    // pinned staging pieces
    char *h = S.stage_mem + q.hoff;
    size_t ho = 0;
    auto htake = [&](size_t bytes) {
        char *p = h + ho;
        ho += up256(bytes);
        return p;
    };
    q.h_boff = reinterpret_cast<int64_t *>(htake((n + 1) * 8));
    q.h_E = reinterpret_cast<int16_t *>(htake(n * 2));
    q.h_acc = reinterpret_cast<uint8_t *>(htake(sl * n));
    q.h_cnt = reinterpret_cast<int16_t *>(htake(sl * n * 2));
    q.h_dist = reinterpret_cast<int32_t *>(htake(n * 4));
    q.h_err = reinterpret_cast<unsigned *>(htake(4));
    std::memcpy(q.h_boff, r.byte_off, (n + 1) * 8);
    if (n) std::memcpy(q.h_E, r.E, n * 2);

    cudaStream_t st = S.s_copy;
    if (q.total_bytes) {
        // page-locked inputs go straight to the copy engine; pageable ones are
        // staged by the driver (the call returns once they are read)
        cudaMemcpyAsync((void *)d.reads, r.reads + r.byte_off[0], (size_t)q.total_bytes,
                        cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync((void *)d.refs, r.refs + r.byte_off[0], (size_t)q.total_bytes,
                        cudaMemcpyHostToDevice, st);
    }
    cudaMemcpyAsync(boff, q.h_boff, (n + 1) * 8, cudaMemcpyHostToDevice, st);
    if (n) cudaMemcpyAsync((void *)d.E, q.h_E, n * 2, cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(d.err, 0, 4, st);
    cudaMemsetAsync(S.d_done + q.slot, 0, sizeof(unsigned), st);
    cudaMemcpyAsync(S.d_desc + q.slot, &d, sizeof(ServeDesc), cudaMemcpyHostToDevice, st);
    cudaEventRecord(q.ev, st);
}

void drain(ServeState &S, ServeReq &q) {
    const pf_request &r = q.req;
    const ServeDesc &d = S.h_desc[q.slot];
    const size_t n = (size_t)r.n, sl = (size_t)slots_of(r.deciders);
    cudaStream_t st = S.s_copy;
    if (n) {
        cudaMemcpyAsync(q.h_acc, d.accept, sl * n, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(q.h_cnt, d.count, sl * n * 2, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(q.h_dist, d.dist, n * 4, cudaMemcpyDeviceToHost, st);
    }
    cudaMemcpyAsync(q.h_err, d.err, 4, cudaMemcpyDeviceToHost, st);
    cudaEventRecord(q.ev, st);
}

// Results to the caller's buffers, resources back to the pools (scheduler
// thread, or pf_serve_stop after the thread has ended).
void finish_req(ServeState &S, ServeReq &q, pf_status st, bool copy_out) {
    const pf_request &r = q.req;
    const size_t n = (size_t)r.n, sl = (size_t)slots_of(r.deciders);
    if (copy_out && n) {
        std::memcpy(r.accept, q.h_acc, sl * n);
        std::memcpy(r.count, q.h_cnt, sl * n * 2);
        std::memcpy(r.dist, q.h_dist, n * 4);
    }
    q.status = st;
    q.t_done = std::chrono::steady_clock::now();
    if (q.slot >= 0) {
        S.free_slots.push_back(q.slot);
        S.dev_arena.release(q.off, q.bytes);
        S.host_arena.release(q.hoff, q.hbytes);
        S.inflight_items -= (uint64_t)q.nchunks;
        q.slot = -1;
    }
}

// The scheduler thread owns the admission queue, the active list, the
// arenas, the slots and the ring; the mutex guards only the hand-offs with
// callers (new submissions in, finished requests out), so submitting and
// waiting never stall behind copies or polling.
void scheduler(ServeState *Sp) {
    ServeState &S = *Sp;
    cudaSetDevice(S.device);
#if defined(__linux__)
    prctl(PR_SET_TIMERSLACK, 1000UL, 0UL, 0UL, 0UL);  // short polling sleeps stay short
#endif
    std::deque<std::shared_ptr<ServeReq>> queue;      // admission order
    std::vector<std::shared_ptr<ServeReq>> finished;  // to hand back under the lock
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(S.mu);
            for (auto &q : finished) {
                q->state = ServeReq::DONE;
                if (q->status == PF_OK) {
                    S.stats.completed++;
                    S.stats.pairs_completed += (uint64_t)q->req.n;
                    const double tq = secs(q->t_submit, q->t_admit);
                    const double ts = secs(q->t_admit, q->t_pub);
                    const double td = secs(q->t_pub, q->t_seen);
                    const double tr = secs(q->t_seen, q->t_done);
                    S.stats.queue_s += tq;
                    S.stats.stage_s += ts;
                    S.stats.device_s += td;
                    S.stats.drain_s += tr;
                    S.stats.queue_max_s = std::max(S.stats.queue_max_s, tq);
                    S.stats.stage_max_s = std::max(S.stats.stage_max_s, ts);
                    S.stats.device_max_s = std::max(S.stats.device_max_s, td);
                    S.stats.drain_max_s = std::max(S.stats.drain_max_s, tr);
                } else {
                    S.stats.failed++;
                }
            }
            if (!finished.empty()) S.cv_done.notify_all();
            finished.clear();
            if (S.quit) break;
            if (queue.empty() && S.active.empty() && S.pending.empty())
                S.cv_work.wait_for(lk, std::chrono::milliseconds(20));
            while (!S.pending.empty()) {
                queue.push_back(S.pending.front());
                S.pending.pop_front();
            }
        }
        bool progress = false;
        // admission: FIFO, as slots, device memory, staging memory and ring room allow
        while (!queue.empty() && !S.free_slots.empty()) {
            auto q = queue.front();
            if (S.inflight_items + (uint64_t)q->nchunks > kRingSize) break;
            size_t off = 0, hoff = 0;
            if (!S.dev_arena.alloc(q->bytes, &off)) break;
            if (!S.host_arena.alloc(q->hbytes, &hoff)) {
                S.dev_arena.release(off, q->bytes);
                break;
            }
            queue.pop_front();
            q->off = off;
            q->hoff = hoff;
            q->slot = S.free_slots.back();
            S.free_slots.pop_back();
            q->epoch = ++S.slot_epoch[q->slot];
            S.inflight_items += (uint64_t)q->nchunks;
            q->state = ServeReq::STAGING;
            q->t_admit = std::chrono::steady_clock::now();
            stage(S, *q);
            S.active.push_back(q);
            progress = true;
        }
        bool running = false;
        for (size_t i = 0; i < S.active.size();) {
            ServeReq &q = *S.active[i];
            if (q.state == ServeReq::STAGING && cudaEventQuery(q.ev) == cudaSuccess) {
                // publish the request's items, then the new tail
                for (int c = 0; c < q.nchunks; ++c)
                    S.h_items[(S.published + c) % kRingSize] =
                        ((unsigned long long)q.slot << 32) | (unsigned)c;
                S.published += (uint64_t)q.nchunks;
                std::atomic_thread_fence(std::memory_order_release);
                *(volatile unsigned long long *)S.h_tail = S.published;
                q.state = ServeReq::RUNNING;
                q.t_pub = std::chrono::steady_clock::now();
                if (q.nchunks == 0) {
                    q.t_seen = q.t_pub;
                    q.state = ServeReq::DRAINING;
                    drain(S, q);
                }
                progress = true;
            } else if (q.state == ServeReq::RUNNING &&
                       *(volatile unsigned *)(S.h_complete + q.slot) == q.epoch) {
                std::atomic_thread_fence(std::memory_order_acquire);
                q.t_seen = std::chrono::steady_clock::now();
                q.state = ServeReq::DRAINING;
                drain(S, q);
                progress = true;
            } else if (q.state == ServeReq::DRAINING && cudaEventQuery(q.ev) == cudaSuccess) {
                const unsigned e = *q.h_err;
                finish_req(S, q,
                           (e & ERR_PAIR_ARGS) ? PF_EINVAL : (e & ERR_BYTES) ? PF_EDATA : PF_OK,
                           true);
                finished.push_back(S.active[i]);
                S.active[i] = S.active.back();
                S.active.pop_back();
                progress = true;
                continue;
            }
            running |= q.state == ServeReq::RUNNING;
            ++i;
        }
        // the device loop: (re)start it while published items wait
        if (S.loop_running && cudaEventQuery(S.ev_loop) == cudaSuccess) S.loop_running = false;
        if (running && !S.loop_running && !S.paused.load()) {
            // the idle clock starts at the launch
            serve_stamp_kernel<<<1, 1, 0, S.s_loop>>>(S.d_last, S.d_exit, S.d_poll);
            serve_loop_kernel<<<S.cfg.workers, kServeThreads, 0, S.s_loop>>>(S.dev);
            if (cudaGetLastError() != cudaSuccess) {
                S.fatal = "serve loop launch failed";
            } else {
                cudaEventRecord(S.ev_loop, S.s_loop);
                S.loop_running = true;
                S.stats.loop_launches++;
            }
        }
        if (!progress && finished.empty() && (!queue.empty() || !S.active.empty()))
            std::this_thread::sleep_for(std::chrono::microseconds(5));
    }
    // requests the thread still owns end cancelled; pf_serve_stop reports them
    for (auto &q : queue) {
        std::lock_guard<std::mutex> lk(S.mu);
        S.pending.push_front(q);
    }
}

}  // namespace

}  // namespace pf

using namespace pf;

void pf_serve_teardown(pf_ctx *ctx) {
    if (ctx && ctx->serve) pf_serve_stop(ctx);
}

extern "C" {

pf_status pf_serve_start(pf_ctx *ctx, const pf_serve_config *cfg) {
    if (!ctx) return PF_EINVAL;
    if (ctx->serve) return ctx->fail(PF_EBUSY, "already serving");
    if (!cfg) return ctx->fail(PF_EINVAL, "null config");
    pf_serve_config c = *cfg;
    if (c.mode != PF_SERVE_BATCHED && c.mode != PF_SERVE_DEVICE_LOOP)
        return ctx->fail(PF_EINVAL, "serve mode must be PF_SERVE_BATCHED or PF_SERVE_DEVICE_LOOP");
    if (c.batch_pairs < 0 || c.overlap_pairs < 0)
        return ctx->fail(PF_EINVAL, "batch_pairs or overlap_pairs < 0");
    if (c.max_requests == 0) c.max_requests = 256;
    if (c.chunk_pairs == 0) c.chunk_pairs = kServeMaxChunk;
    if (c.idle_exit_us == 0) c.idle_exit_us = 500;
    if (c.max_requests < 1 || c.max_requests > 4096 || c.chunk_pairs < 32 ||
        c.chunk_pairs > kServeMaxChunk || c.idle_exit_us < 50 || c.idle_exit_us > 1000000 ||
        c.workers < 0)
        return ctx->fail(PF_EINVAL, "serve config out of range");
    cudaSetDevice(ctx->device);
    if (c.workers == 0) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, serve_loop_kernel, kServeThreads, 0);
        c.workers = std::max(1, std::min(per_sm, 2)) * ctx->sms;
    }
    size_t budget = c.hbm_budget ? c.hbm_budget : ctx->hbm_budget;
    if (!budget) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        budget = fr / 4;
    }
    budget &= ~size_t(255);
    auto S = new ServeState();
    S->cfg = c;
    S->ctx = ctx;
    S->device = ctx->device;
    S->budget = budget;
    // pinned staging: ~20 B per pair against ~370 B per pair on the device
    S->stage_budget = std::max<size_t>(budget / 16, size_t(64) << 20) & ~size_t(255);
    S->paused = c.start_paused != 0;
    if (c.mode == PF_SERVE_BATCHED) {
        bool ok = cudaHostAlloc(&S->stage_mem, S->stage_budget, cudaHostAllocMapped) == cudaSuccess;
        pf_status st = ok ? batch_start(ctx, S) : ctx->fail(PF_ENOMEM, "serve staging allocation");
        if (st != PF_OK) {
            cudaGetLastError();
            ctx->serve = S;
            pf_serve_stop(ctx);
            return st;
        }
        S->host_arena.reset(S->stage_budget);
        ctx->serve = S;
        S->th = std::thread(batch_scheduler, S);
        return PF_OK;
    }
    bool ok = cudaMalloc(&S->arena, budget) == cudaSuccess &&
              cudaMalloc(&S->d_desc, sizeof(ServeDesc) * c.max_requests) == cudaSuccess &&
              cudaMalloc(&S->d_done, sizeof(unsigned) * c.max_requests) == cudaSuccess &&
              cudaMalloc(&S->d_head, sizeof(unsigned long long)) == cudaSuccess &&
              cudaMalloc(&S->d_last, sizeof(unsigned long long)) == cudaSuccess &&
              cudaMalloc(&S->d_tail, sizeof(unsigned long long)) == cudaSuccess &&
              cudaMemset(S->d_tail, 0, sizeof(unsigned long long)) == cudaSuccess &&
              cudaMalloc(&S->d_exit, sizeof(unsigned)) == cudaSuccess &&
              cudaMalloc(&S->d_poll, sizeof(unsigned long long)) == cudaSuccess &&
              cudaMemset(S->d_head, 0, sizeof(unsigned long long)) == cudaSuccess &&
              cudaHostAlloc(&S->h_desc, sizeof(ServeDesc) * c.max_requests, 0) == cudaSuccess &&
              cudaHostAlloc(&S->h_items, sizeof(unsigned long long) * kRingSize,
                            cudaHostAllocMapped) == cudaSuccess &&
              cudaHostAlloc(&S->h_tail, sizeof(unsigned long long), cudaHostAllocMapped) ==
                  cudaSuccess &&
              cudaHostAlloc(&S->h_stop, sizeof(unsigned), cudaHostAllocMapped) == cudaSuccess &&
              cudaHostAlloc(&S->h_complete, sizeof(unsigned) * c.max_requests,
                            cudaHostAllocMapped) == cudaSuccess &&
              cudaHostAlloc(&S->stage_mem, S->stage_budget, 0) == cudaSuccess &&
              cudaStreamCreateWithFlags(&S->s_copy, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&S->s_loop, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&S->ev_loop, cudaEventDisableTiming) == cudaSuccess;
    if (ok) {
        *S->h_tail = 0;
        *S->h_stop = 0;
        std::memset(S->h_complete, 0, sizeof(unsigned) * c.max_requests);
        void *p = nullptr;
        S->dev.desc = S->d_desc;
        S->dev.done = S->d_done;
        S->dev.head = S->d_head;
        S->dev.last_claim = S->d_last;
        S->dev.dev_tail = S->d_tail;
        S->dev.dev_exit = S->d_exit;
        S->dev.last_poll = S->d_poll;
        ok = cudaHostGetDevicePointer(&p, S->h_items, 0) == cudaSuccess;
        S->dev.items = static_cast<const unsigned long long *>(p);
        ok = ok && cudaHostGetDevicePointer(&p, S->h_tail, 0) == cudaSuccess;
        S->dev.tail = static_cast<const unsigned long long *>(p);
        ok = ok && cudaHostGetDevicePointer(&p, S->h_stop, 0) == cudaSuccess;
        S->dev.stop = static_cast<const unsigned *>(p);
        ok = ok && cudaHostGetDevicePointer(&p, S->h_complete, 0) == cudaSuccess;
        S->dev.complete = static_cast<unsigned *>(p);
        S->dev.idle_ns = (unsigned long long)c.idle_exit_us * 1000ull;
    }
    if (!ok) {
        cudaGetLastError();
        ctx->serve = S;
        pf_serve_stop(ctx);
        return ctx->fail(PF_ENOMEM, "serve allocation failed");
    }
    S->dev_arena.reset(budget);
    S->host_arena.reset(S->stage_budget);
    S->slot_epoch.assign(c.max_requests, 0);
    for (int i = c.max_requests - 1; i >= 0; --i) S->free_slots.push_back(i);
    ctx->serve = S;
    S->th = std::thread(scheduler, S);
    return PF_OK;
}

pf_status pf_serve_resume(pf_ctx *ctx) {
    if (!ctx || !ctx->serve) return PF_EBUSY;
    ctx->serve->paused = false;
    ctx->serve->cv_work.notify_all();
    return PF_OK;
}

pf_status pf_submit(pf_ctx *ctx, const pf_request *req, uint64_t *ticket) {
    if (!ctx) return PF_EINVAL;
    ServeState *S = ctx->serve;
    if (!S) return ctx->fail(PF_EBUSY, "not serving");
    if (!req || !ticket || req->n < 0 || (req->deciders & 3u) == 0 || (req->deciders & ~3u))
        return ctx->fail(PF_EINVAL, "malformed request");
    if (!req->byte_off || (req->n > 0 && (!req->reads || !req->refs || !req->E ||
                                          !req->accept || !req->count || !req->dist)))
        return ctx->fail(PF_EINVAL, "malformed request: null pointer");
    bool bad_off = false, bad_E = false;
    int64_t longest = 0;
    int emax = 0;
    for (int64_t p = 0; p < req->n; ++p) {
        const int64_t len = req->byte_off[p + 1] - req->byte_off[p];
        const int e = req->E[p];
        bad_off |= len < 0;
        bad_E |= (e < 0) | (e > PF_MAX_E);
        longest = std::max(longest, len);
        emax = std::max(emax, e);
    }
    if (bad_off) return ctx->fail(PF_EINVAL, "malformed request: offsets decrease");
    if (bad_E) return ctx->fail(PF_EINVAL, "malformed request: E outside [0, %d]", PF_MAX_E);
    const int64_t tb = req->n ? req->byte_off[req->n] - req->byte_off[0] : 0;
    const int64_t words = (tb >> 5) + req->n + 1;
    auto q = std::make_shared<ServeReq>();
    q->req = *req;
    q->E_max = emax;
    q->longest = longest;
    if (S->bp) {  // batched mode: requests stream through the batch buffers
        const pf_status st = batch_prepare(ctx, S, q.get());
        if (st != PF_OK) return st;
        q->t_submit = std::chrono::steady_clock::now();
        {
            std::lock_guard<std::mutex> lk(S->mu);
            q->ticket = S->next_ticket++;
            S->pending.push_back(q);
            S->reqs[q->ticket] = q;
            S->stats.submitted++;
        }
        S->cv_work.notify_all();
        *ticket = q->ticket;
        return PF_OK;
    }
    q->total_bytes = req->n ? req->byte_off[req->n] - req->byte_off[0] : 0;
    q->total_words = words;
    q->nchunks = (int)((req->n + S->cfg.chunk_pairs - 1) / S->cfg.chunk_pairs);
    q->bytes = request_bytes(*req, q->total_bytes, words);
    q->hbytes = staging_bytes(*req);
    if (q->bytes > S->budget || q->hbytes > S->stage_budget || (uint64_t)q->nchunks > kRingSize)
        return ctx->fail(PF_ENOMEM, "request needs %zu device bytes, budget %zu", q->bytes,
                         S->budget);
    if (cudaEventCreateWithFlags(&q->ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return ctx->fail(PF_ECUDA, "event creation failed");
    }
    q->t_submit = std::chrono::steady_clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        q->ticket = S->next_ticket++;
        S->pending.push_back(q);
        S->reqs[q->ticket] = q;
        S->stats.submitted++;
    }
    S->cv_work.notify_all();
    *ticket = q->ticket;
    return PF_OK;
}

pf_status pf_poll(pf_ctx *ctx, uint64_t ticket, int *done) {
    if (!ctx || !done) return PF_EINVAL;
    ServeState *S = ctx->serve;
    if (!S) return PF_EBUSY;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return PF_EINVAL;
    *done = it->second->state == ServeReq::DONE;
    return PF_OK;
}

pf_status pf_wait(pf_ctx *ctx, uint64_t ticket, int timeout_ms, double *latency_ms) {
    if (!ctx) return PF_EINVAL;
    ServeState *S = ctx->serve;
    if (!S) return PF_EBUSY;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return PF_EINVAL;
    auto q = it->second;
    auto ready = [&] { return q->state == ServeReq::DONE; };
    S->waiters++;
    bool ok = true;
    if (timeout_ms < 0) S->cv_done.wait(lk, ready);
    else ok = S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
    S->waiters--;
    S->cv_idle.notify_all();
    if (!ok) return PF_ETIMEOUT;
    if (latency_ms)
        *latency_ms =
            std::chrono::duration<double, std::milli>(q->t_done - q->t_submit).count();
    if (q->ev) cudaEventDestroy(q->ev);
    q->ev = nullptr;
    S->reqs.erase(ticket);
    return q->status;
}

pf_status pf_serve_stats_get(pf_ctx *ctx, pf_serve_stats *out) {
    if (!ctx || !out) return PF_EINVAL;
    ServeState *S = ctx->serve;
    if (!S) return PF_EBUSY;
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->stats;
    return PF_OK;
}

pf_status pf_serve_replay(pf_ctx *ctx, const pf_request *pool, int npool,
                          const double *arrival_s, int count, double *latency_ms,
                          double *elapsed_s) {
    if (!ctx) return PF_EINVAL;
    if (!ctx->serve) return ctx->fail(PF_EBUSY, "not serving");
    if (!pool || npool <= 0 || !arrival_s || count < 0 || (count > 0 && !latency_ms))
        return ctx->fail(PF_EINVAL, "pf_serve_replay: bad arguments");
    for (int i = 1; i < count; ++i)
        if (arrival_s[i] < arrival_s[i - 1])
            return ctx->fail(PF_EINVAL, "pf_serve_replay: arrival times decrease");
    using clk = std::chrono::steady_clock;
    std::vector<uint64_t> tickets((size_t)count, 0);
#if defined(__linux__)
    // arrivals are paced by short sleeps: tighten the calling thread's timer
    // slack for the replay, and give it back afterwards
    const int slack = prctl(PR_GET_TIMERSLACK, 0UL, 0UL, 0UL, 0UL);
    prctl(PR_SET_TIMERSLACK, 1000UL, 0UL, 0UL, 0UL);
#endif
    const auto t0 = clk::now();
    pf_status first = PF_OK;
    for (int i = 0; i < count; ++i) {
        const auto due = t0 + std::chrono::duration_cast<clk::duration>(
                                  std::chrono::duration<double>(arrival_s[i]));
        while (clk::now() + std::chrono::microseconds(200) < due)
            std::this_thread::sleep_for(std::chrono::microseconds(100));
        while (clk::now() < due) std::this_thread::yield();
        const pf_status st = pf_submit(ctx, &pool[i % npool], &tickets[(size_t)i]);
        if (st != PF_OK) {
            if (first == PF_OK) first = st;
            tickets[(size_t)i] = 0;
        }
    }
    for (int i = 0; i < count; ++i) {
        latency_ms[i] = -1.0;
        if (!tickets[(size_t)i]) continue;
        const pf_status st = pf_wait(ctx, tickets[(size_t)i], -1, &latency_ms[i]);
        if (st != PF_OK && first == PF_OK) first = st;
    }
    if (elapsed_s) *elapsed_s = std::chrono::duration<double>(clk::now() - t0).count();
#if defined(__linux__)
    if (slack > 0) prctl(PR_SET_TIMERSLACK, (unsigned long)slack, 0UL, 0UL, 0UL);
#endif
    return first;
}

pf_status pf_serve_trace(pf_ctx *ctx, double *records, int cap, int *count) {
    if (!ctx) return PF_EINVAL;
    ServeState *S = ctx->serve;
    if (!S || !S->bp) return ctx->fail(PF_EBUSY, "not serving in the batched mode");
    if (!count || cap < 0 || (cap > 0 && !records))
        return ctx->fail(PF_EINVAL, "pf_serve_trace: bad arguments");
    return batch_trace(S, records, cap, count);
}

pf_status pf_serve_stop(pf_ctx *ctx) {
    if (!ctx) return PF_EINVAL;
    ServeState *S = ctx->serve;
    if (!S) return PF_EBUSY;
    cudaSetDevice(ctx->device);
    if (S->h_stop) *(volatile unsigned *)S->h_stop = 1;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->quit = true;
    }
    S->cv_work.notify_all();
    if (S->th.joinable()) S->th.join();
    if (S->bp) batch_stop(S);
    if (S->s_loop) cudaStreamSynchronize(S->s_loop);
    if (S->s_copy) cudaStreamSynchronize(S->s_copy);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        for (auto &kv : S->reqs) {
            ServeReq &q = *kv.second;
            if (q.state == ServeReq::DONE) continue;
            finish_req(*S, q, PF_ECANCELLED, false);
            q.state = ServeReq::DONE;
            S->stats.failed++;
        }
        S->pending.clear();
        S->active.clear();
    }
    S->cv_done.notify_all();
    {   // let every thread inside pf_wait leave before S goes away
        std::unique_lock<std::mutex> lk(S->mu);
        S->cv_idle.wait(lk, [&] { return S->waiters == 0; });
    }
    for (auto &kv : S->reqs)
        if (kv.second->ev) cudaEventDestroy(kv.second->ev);
    if (S->arena) cudaFree(S->arena);
    if (S->d_desc) cudaFree(S->d_desc);
    if (S->d_done) cudaFree(S->d_done);
    if (S->d_head) cudaFree(S->d_head);
    if (S->d_last) cudaFree(S->d_last);
    if (S->d_tail) cudaFree(S->d_tail);
    if (S->d_exit) cudaFree(S->d_exit);
    if (S->d_poll) cudaFree(S->d_poll);
    if (S->h_desc) cudaFreeHost(S->h_desc);
    if (S->h_items) cudaFreeHost(S->h_items);
    if (S->h_tail) cudaFreeHost(S->h_tail);
    if (S->h_stop) cudaFreeHost(S->h_stop);
    if (S->h_complete) cudaFreeHost(S->h_complete);
    if (S->stage_mem) cudaFreeHost(S->stage_mem);
    if (S->s_copy) cudaStreamDestroy(S->s_copy);
    if (S->s_loop) cudaStreamDestroy(S->s_loop);
    if (S->ev_loop) cudaEventDestroy(S->ev_loop);
    ctx->serve = nullptr;
    delete S;
    return PF_OK;
}

}  // extern "C"
