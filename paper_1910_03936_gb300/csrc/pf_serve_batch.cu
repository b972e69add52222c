// a8, batched mode: continuous batching of admitted requests into device
// batches that run the tuned path.  Contracts: pf.h (PF_SERVE_BATCHED).
//
// Batch slots.  A slot is one batch: a device byte area for reads and one
// for references, and a segment table (one entry per request part).  The
// scheduler thread places admitted requests, in arrival order, into the
// open slot and starts their uploads on the copy stream at once; a request
// larger than the room left is split and its rest placed into the next
// slot.  A slot is launched when fewer than two batches are on the GPU.
//
// Per-pair arrays (offsets, planes, outputs, scheduler scratch) live once,
// in a compute area that every batch uses in turn: batches run one after
// the other on the serving context's stream, so a batch's epilogue has read
// its outputs before the next batch's offsets kernel overwrites them.
//
// A batch on the GPU: wait for its uploads (every part's bytes, the segment
// table, and the byte offsets and thresholds of pageable requests: all on
// the copy stream, since a copy issued on the compute stream would queue in
// the copy engine behind later batches' uploads); the offsets kernel turns
// the parts' byte offsets (page-locked ones read in place, which spares the
// copy engine two small transfers per part) into the batch's byte and word
// offsets, lengths and thresholds; both planes are packed; the scheduler's binned filter,
// compaction and verification run as in pf_filter_verify; the epilogue
// writes every pair's results into its request's buffers in the request's
// own output layout (directly when they are page-locked: 10 bytes per pair
// of posted writes).
#include <algorithm>
#include <cstring>
#if defined(__linux__)
#include <sys/prctl.h>
#endif

#include "pf_serve.h"

namespace pf {

namespace {

constexpr int kMaxSegs = 1024;          // request parts per batch
constexpr int kBatchSlots = 4;          // two batches on the GPU, up to two filling
// Batches of up to 2^20 pairs: larger ones raise a burst's throughput
// little (the uploads bind) and lengthen the latency of every request they
// hold (measured: p99 at 73% of the host-link bound 14 ms with 2^20, 31 ms
// with 2^22).
constexpr int64_t kDefaultBatchPairs = int64_t(1) << 20;
constexpr int64_t kBytesPerPairCap = 200;  // byte area per pair of capacity, per side
constexpr unsigned kErrLaunch = 1u << 30;   // a batch whose launch failed
// Default of overlap_pairs: a second batch joins the one on the GPU only
// once it holds this many pairs; smaller batches wait for the GPU to drain
// and grow meanwhile (a batch costs about 0.2 ms of fixed latency, its
// chain of launches).
constexpr int64_t kOverlapPairs = int64_t(1) << 18;
constexpr uint64_t kTraceCap = 65536;   // batches kept by the trace
constexpr int kOffsetsIlp = 4;          // positions per thread and round, offsets kernel

// One request part in a batch: pairs [a, a + n) of the request are batch
// positions [p0, p0 + n); their bytes start at bbase in the slot's areas.
struct SegDesc {
    int64_t p0, n, a, bbase, req_n;
    const int64_t *boff;   // the part's n + 1 byte offsets (device-visible)
    const int16_t *E;      // the part's n thresholds (device-visible)
    uint8_t *acc;          // request outputs (device-visible)
    int16_t *cnt;
    int32_t *dist;
    uint32_t dec, pad;
};

// Batch position i -> its segment (the last whose p0 <= i), by binary
// search over the table's p0 column staged in shared memory.
__device__ __forceinline__ int seg_of_pos(const int64_t *sp0, int nseg, int64_t i) {
    int l = 0, r = nseg - 1;
    while (l < r) {
        const int mid = (l + r + 1) >> 1;
        if (sp0[mid] <= i) l = mid; else r = mid - 1;
    }
    return l;
}

// Byte offsets relative to the slot's areas (the parts are adjacent there),
// word offsets floor(b / 32) + i (disjoint without a scan: sequence i ends
// before floor(b_{i+1} / 32) + i + 1), lengths, thresholds and segment ids;
// block 0 also clears the parts' error words for the packer.
__global__ void __launch_bounds__(256)
batch_offsets_kernel(const SegDesc *segs, int nseg, int64_t P, int64_t *boff, int64_t *woff,
                     int32_t *lens, int16_t *E, int32_t *seg_of, unsigned *seg_err) {
    __shared__ int64_t sp0[kMaxSegs];
    for (int k = threadIdx.x; k < nseg; k += blockDim.x) {
        sp0[k] = segs[k].p0;
        if (blockIdx.x == 0) seg_err[k] = 0u;
    }
    __syncthreads();
    // kOffsetsIlp positions per thread and round, all their loads issued
    // before any is used: the offsets and thresholds of page-locked requests
    // come over the host link, whose round trips a thread would otherwise
    // wait out one by one
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < P;
         i0 += stride * kOffsetsIlp) {
        int sg[kOffsetsIlp];
        int64_t r0[kOffsetsIlp], xb[kOffsetsIlp], xe[kOffsetsIlp], base[kOffsetsIlp];
        int16_t th[kOffsetsIlp];
#pragma unroll
        for (int u = 0; u < kOffsetsIlp; ++u) {
            const int64_t i = i0 + u * stride;
            if (i >= P) continue;
            sg[u] = seg_of_pos(sp0, nseg, i);
            const SegDesc &d = segs[sg[u]];
            const int64_t j = i - d.p0;
            base[u] = d.bbase;
            r0[u] = d.boff[0];
            xb[u] = d.boff[j];
            xe[u] = d.boff[j + 1];
            th[u] = d.E[j];
        }
#pragma unroll
        for (int u = 0; u < kOffsetsIlp; ++u) {
            const int64_t i = i0 + u * stride;
            if (i >= P) continue;
            const int64_t b = xb[u] - r0[u] + base[u];
            const int64_t e = xe[u] - r0[u] + base[u];
            boff[i] = b;
            woff[i] = (b >> 5) + i;
            lens[i] = (int32_t)(e - b);
            E[i] = th[u];
            seg_of[i] = sg[u];
            if (i == P - 1) {
                boff[P] = e;
                woff[P] = (e >> 5) + P;
            }
        }
    }
}

// Results of batch position i into its request's layout.  bdec is the
// decider set the batch ran (the union of its requests'): slot 0 of the
// batch outputs is SneakySnake unless bdec == 2.  A request that asked for
// GateKeeper alone in a batch that also ran SneakySnake gets dist = E + 1
// where GateKeeper rejects; where GateKeeper accepts, the batch's distance
// (verified when SneakySnake accepts, E + 1 otherwise) is already its own:
// a pair SneakySnake rejects is beyond E (its count never exceeds the edit
// distance).  Also copies the parts' device error bits to host memory.
__global__ void __launch_bounds__(256)
batch_epilogue_kernel(const SegDesc *segs, int nseg, int64_t P, unsigned bdec,
                      const int32_t *seg_of, const uint8_t *acc, const int16_t *cnt,
                      const int32_t *dist, const int16_t *E, const unsigned *seg_err,
                      unsigned *seg_err_host) {
    if (blockIdx.x == 0)
        for (int k = threadIdx.x; k < nseg; k += blockDim.x) seg_err_host[k] = seg_err[k];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P;
         i += (int64_t)gridDim.x * blockDim.x) {
        const SegDesc &d = segs[seg_of[i]];
        const int64_t p = d.a + (i - d.p0);
        const int32_t dv = dist[i];
        if (d.dec == 3u) {
            d.acc[p] = acc[i];
            d.acc[d.req_n + p] = acc[P + i];
            d.cnt[p] = cnt[i];
            d.cnt[d.req_n + p] = cnt[P + i];
            d.dist[p] = dv;
        } else if (d.dec == 1u) {
            d.acc[p] = acc[i];
            d.cnt[p] = cnt[i];
            d.dist[p] = dv;
        } else {
            const int64_t g = (bdec == 3u) ? P + i : i;
            const uint8_t ga = acc[g];
            d.acc[p] = ga;
            d.cnt[p] = cnt[g];
            d.dist[p] = (bdec == 3u && !ga) ? (int32_t)E[i] + 1 : dv;
        }
    }
}

struct BatchSlot {
    uint8_t *reads = nullptr, *refs = nullptr;  // device byte areas
    int64_t *raw_off = nullptr;                  // parts' byte offsets, P + kMaxSegs
    int16_t *raw_E = nullptr;                    // parts' thresholds, P
    SegDesc *h_segs = nullptr;                   // pinned
    SegDesc *d_segs = nullptr;                   // device
    unsigned *h_err = nullptr;                   // pinned, mapped: per-part error bits
    unsigned *d_err_map = nullptr;               // its device address
    std::vector<std::shared_ptr<ServeReq>> reqs; // per part
    int nseg = 0;
    int64_t pairs = 0, bytes = 0;
    unsigned dec = 0;
    int E_max = 0;
    bool full = false;
    bool closed = false;  // its uploads end here: segment table sent, ev_copied recorded
    bool failed = false;  // its launch failed: nothing it holds is valid
    cudaEvent_t ev_copied = nullptr, ev_enq = nullptr, ev_start = nullptr, ev_done = nullptr;
    cudaEvent_t ev_phase[4] = {};       // after offsets, pack, filter, verification
    double t_launch = 0, host_ms = 0;   // trace: scheduler clock, enqueue time

    void reset() {
        reqs.clear();
        nseg = 0;
        pairs = bytes = 0;
        dec = 0;
        E_max = 0;
        full = false;
        closed = false;
        failed = false;
    }
};

}  // namespace

struct BatchPool {
    pf_ctx *sub = nullptr;          // the serving thread's context
    cudaStream_t s_compute = nullptr, s_copy = nullptr;
    int64_t P = 0, B = 0, W = 0;    // pairs, bytes per side, words per plane of a batch
    char *mem = nullptr;            // device: compute area and slot byte areas
    int64_t *boff = nullptr, *woff = nullptr;
    int32_t *lens = nullptr, *seg_of = nullptr;
    int16_t *E = nullptr;
    uint32_t *pl[6] = {};
    uint8_t *acc = nullptr;
    int16_t *cnt = nullptr;
    int32_t *dist = nullptr;
    unsigned *seg_err = nullptr;
    Scratch scr{};
    BatchSlot slots[kBatchSlots];
    std::deque<int> inflight;       // launched slots, in launch order
    std::deque<int> ready;          // full slots waiting for the GPU, in order
    std::vector<int> free_slots;
    int open = -1;
    int admitted = 0;               // requests admitted and not finished
    int64_t overlap = kOverlapPairs;
    // trace of the most recent batches (pf_serve_trace), a ring
    std::mutex trace_mu;
    std::vector<double> trace;      // kTraceCap records of PF_SERVE_TRACE_FIELDS
    uint64_t trace_n = 0;           // records written so far
    std::chrono::steady_clock::time_point t0;
};

namespace {

// Device-visible address of host memory, or null if it is not page-locked
// (pageable memory has none).
template <typename T>
T *mapped(const T *p) {
    if (!p) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    return static_cast<T *>(a.devicePointer);
}

// Pinned staging bytes a request needs: its outputs, when they are
// pageable (the GPU writes page-locked ones in place).
size_t staging_need(const ServeReq &q) {
    const size_t n = (size_t)q.req.n, sl = (size_t)slots_of(q.req.deciders);
    return q.out_mapped ? 0 : up256(sl * n) + up256(sl * n * 2) + up256(n * 4);
}

// First placement of a request: staging (if any), device-visible views.
bool admit(ServeState &S, ServeReq &q) {
    BatchPool &B = *S.bp;
    if (B.admitted >= S.cfg.max_requests) return false;
    q.hbytes = staging_need(q);
    if (q.hbytes) {
        size_t hoff = 0;
        if (!S.host_arena.alloc(q.hbytes, &hoff)) return false;
        q.hoff = hoff;
        const size_t n = (size_t)q.req.n, sl = (size_t)slots_of(q.req.deciders);
        char *h = S.stage_mem + hoff;
        size_t o = 0;
        auto take = [&](size_t bytes) {
            char *p = h + o;
            o += up256(bytes);
            return p;
        };
        if (!q.out_mapped) {
            q.h_acc = reinterpret_cast<uint8_t *>(take(sl * n));
            q.h_cnt = reinterpret_cast<int16_t *>(take(sl * n * 2));
            q.h_dist = reinterpret_cast<int32_t *>(take(n * 4));
            q.d_acc = mapped(q.h_acc);
            q.d_cnt = mapped(q.h_cnt);
            q.d_dist = mapped(q.h_dist);
        }
    }
    q.admitted = true;
    B.admitted++;
    q.state = ServeReq::STAGING;
    q.t_admit = std::chrono::steady_clock::now();
    return true;
}

// Pairs of q (from q.next on) that fit the slot's room.
int64_t fit(const BatchPool &B, const BatchSlot &b, const ServeReq &q) {
    if (b.nseg >= kMaxSegs) return 0;
    const int64_t *off = q.req.byte_off;
    int64_t k = std::min(q.req.n - q.next, B.P - b.pairs);
    const int64_t room = B.B - b.bytes;
    if (off[q.next + k] - off[q.next] <= room) return k;
    int64_t lo = 0, hi = k;  // largest k with bytes <= room
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) / 2;
        if (off[q.next + mid] - off[q.next] <= room) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Place k pairs of q into slot b and start their uploads: bytes, byte
// offsets (k + 1, at raw_off + p0 + the part's index, so that every part
// keeps its closing offset) and thresholds.
void place(ServeState &S, BatchSlot &b, const std::shared_ptr<ServeReq> &qp, int64_t k) {
    BatchPool &B = *S.bp;
    ServeReq &q = *qp;
    const int64_t x0 = q.req.byte_off[q.next], x1 = q.req.byte_off[q.next + k];
    SegDesc &d = b.h_segs[b.nseg];
    d.p0 = b.pairs;
    d.n = k;
    d.a = q.next;
    d.bbase = b.bytes;
    d.req_n = q.req.n;
    if (q.in_mapped) {  // page-locked: the offsets kernel reads them in place
        d.boff = q.d_boff + q.next;
        d.E = q.d_E + q.next;
    } else {
        int64_t *off = b.raw_off + b.pairs + b.nseg;
        int16_t *thr = b.raw_E + b.pairs;
        d.boff = off;
        d.E = thr;
        cudaMemcpyAsync(off, q.req.byte_off + q.next, (size_t)(k + 1) * sizeof(int64_t),
                        cudaMemcpyHostToDevice, B.s_copy);
        cudaMemcpyAsync(thr, q.req.E + q.next, (size_t)k * sizeof(int16_t),
                        cudaMemcpyHostToDevice, B.s_copy);
    }
    d.acc = q.d_acc;
    d.cnt = q.d_cnt;
    d.dist = q.d_dist;
    d.dec = q.req.deciders;
    d.pad = 0;
    if (x1 > x0) {
        cudaMemcpyAsync(b.reads + b.bytes, q.req.reads + x0, (size_t)(x1 - x0),
                        cudaMemcpyHostToDevice, B.s_copy);
        cudaMemcpyAsync(b.refs + b.bytes, q.req.refs + x0, (size_t)(x1 - x0),
                        cudaMemcpyHostToDevice, B.s_copy);
    }
    b.reqs.push_back(qp);
    b.nseg++;
    b.pairs += k;
    b.bytes += x1 - x0;
    b.dec |= q.req.deciders;
    b.E_max = std::max(b.E_max, q.E_max);
    q.next += k;
    q.parts++;
    if (b.pairs >= B.P || b.nseg >= kMaxSegs) b.full = true;
}

// The batch takes no more placements: its segment table joins its uploads
// on the copy stream (a copy issued on the compute stream would queue in the
// copy engine behind the uploads of later batches), and ev_copied marks the
// end of its uploads there, before any of the next batch's.  Recorded when
// the batch fills up, so that its launch does not also wait for the uploads
// placed into the next batch in the meantime.
void close_uploads(BatchPool &B, BatchSlot &b) {
    if (b.closed) return;
    cudaMemcpyAsync(b.d_segs, b.h_segs, sizeof(SegDesc) * (size_t)b.nseg, cudaMemcpyHostToDevice,
                    B.s_copy);
    cudaEventRecord(b.ev_copied, B.s_copy);
    b.closed = true;
}

// The batch's device work on the compute stream.
pf_status launch(ServeState &S, BatchSlot &b) {
    BatchPool &B = *S.bp;
    pf_ctx *sub = B.sub;
    cudaStream_t st = B.s_compute;
    const int64_t P = b.pairs;
    const int ns = b.nseg;
    close_uploads(B, b);
    cudaEventRecord(b.ev_enq, st);
    cudaStreamWaitEvent(st, b.ev_copied, 0);
    cudaEventRecord(b.ev_start, st);
    const unsigned grid =
        (unsigned)std::max<int64_t>(1, std::min<int64_t>((P + 255) / 256, (int64_t)sub->sms * 8));
    batch_offsets_kernel<<<grid, 256, 0, st>>>(b.d_segs, ns, P, B.boff, B.woff, B.lens, B.E,
                                               B.seg_of, B.seg_err);
    cudaEventRecord(b.ev_phase[0], st);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = launch_pack_ragged(b.reads, B.boff, B.woff, P, B.pl[0], B.pl[1], B.pl[2], sub->d_err,
                               st, B.seg_of, B.seg_err);
    if (e == cudaSuccess)
        e = launch_pack_ragged(b.refs, B.boff, B.woff, P, B.pl[3], B.pl[4], B.pl[5], sub->d_err,
                               st, B.seg_of, B.seg_err);
    if (e != cudaSuccess) return sub->cuda(e, "serve batch pack");
    cudaEventRecord(b.ev_phase[1], st);
    PairsView pv;
    pv.read = SeqView{B.pl[0], B.pl[1], B.pl[2], B.woff, 0};
    pv.ref = SeqView{B.pl[3], B.pl[4], B.pl[5], B.woff, 0};
    FilterArgs a;
    a.pairs = pv;
    a.lens = B.lens;
    a.E = B.E;
    a.E_max = b.E_max;
    a.accept = B.acc;
    a.count = B.cnt;
    a.n = P;
    a.err = sub->d_err;
    a.dist = B.dist;  // E + 1 for the pairs the filter rejects
    if (sub->resolve_bounds && (b.dec & 1u)) a.need = B.scr.need;
    sub->stream = st;
    pf_status s = sub->run_filter(b.dec, a, B.scr);
    if (s != PF_OK) return s;
    cudaEventRecord(b.ev_phase[2], st);
    e = launch_compact(a.need ? a.need : B.acc, P, B.scr.idx, B.scr.n_idx, B.scr.tiles, st,
                       sub->binned ? B.scr.order : nullptr, B.scr.ident);
    if (e == cudaSuccess)
        e = launch_verify(pv, B.lens, B.E, b.E_max, B.scr.idx, B.scr.n_idx, P, B.dist, sub->d_err,
                          sub->sms, st, B.scr.work + kNumBatchCfgs, sub->binned);
    cudaEventRecord(b.ev_phase[3], st);
    if (e == cudaSuccess) {
        batch_epilogue_kernel<<<grid, 256, 0, st>>>(b.d_segs, ns, P, b.dec, B.seg_of, B.acc,
                                                    B.cnt, B.dist, B.E, B.seg_err, b.d_err_map);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(b.ev_done, st);
    return sub->cuda(e, "serve batch launch");
}

// Results to the caller (pageable outputs), staging back to the pool.
void finish(ServeState &S, ServeReq &q, pf_status st, bool copy_out) {
    BatchPool &B = *S.bp;
    const size_t n = (size_t)q.req.n, sl = (size_t)slots_of(q.req.deciders);
    if (copy_out && n && !q.out_mapped) {
        std::memcpy(q.req.accept, q.h_acc, sl * n);
        std::memcpy(q.req.count, q.h_cnt, sl * n * 2);
        std::memcpy(q.req.dist, q.h_dist, n * 4);
    }
    q.status = st;
    q.t_done = std::chrono::steady_clock::now();
    if (q.admitted) {
        if (q.hbytes) S.host_arena.release(q.hoff, q.hbytes);
        q.hbytes = 0;
        B.admitted--;
        q.admitted = false;
    }
}

// A finished batch: account its parts, finish the requests it completes.
void complete(ServeState &S, BatchSlot &b, std::vector<std::shared_ptr<ServeReq>> &finished) {
    const auto now = std::chrono::steady_clock::now();
    for (int k = 0; k < b.nseg; ++k) {
        ServeReq &q = *b.reqs[(size_t)k];
        q.dev_err |= b.failed ? kErrLaunch : b.h_err[k];
        q.parts_done++;
        if (q.next == q.req.n && q.parts_done == q.parts) {
            q.t_seen = now;
            const pf_status st = (q.dev_err & kErrLaunch)    ? PF_ECUDA
                                 : (q.dev_err & ERR_PAIR_ARGS) ? PF_EINVAL
                                 : (q.dev_err & ERR_BYTES)     ? PF_EDATA
                                                               : PF_OK;
            finish(S, q, st, true);
            finished.push_back(b.reqs[(size_t)k]);
        }
    }
    b.reset();
}

}  // namespace

pf_status batch_start(pf_ctx *ctx, ServeState *Sp) {
    ServeState &S = *Sp;
    auto *Bp = new BatchPool();
    S.bp = Bp;
    BatchPool &B = *Bp;
    // capacity: compute area per pair (offsets, lengths, thresholds, segment
    // ids, outputs, scheduler scratch, planes) and the slots' byte areas
    const int64_t words_per_pair = kBytesPerPairCap / 32 + 2;
    const int64_t per_pair = 8 + 8 + 4 + 2 + 4 + 2 + 4 + 4 + 8 + 8 + 1 + 6 * 4 * words_per_pair +
                             kBatchSlots * (2 * kBytesPerPairCap + 8 + 2);
    int64_t P = S.cfg.batch_pairs ? S.cfg.batch_pairs : kDefaultBatchPairs;
    P = std::min<int64_t>(P, (int64_t)(S.budget / (size_t)per_pair));
    if (P < 1) return ctx->fail(PF_ENOMEM, "serve budget too small for one batch pair");
    B.P = P;
    B.B = P * kBytesPerPairCap;
    if (S.cfg.overlap_pairs) B.overlap = S.cfg.overlap_pairs;
    B.W = B.B / 32 + P + 1;
    size_t o = 0;
    auto add = [&](size_t bytes) {
        const size_t at = o;
        o += up256(bytes);
        return at;
    };
    const size_t nn = (size_t)P;
    const size_t o_boff = add((nn + 1) * 8), o_woff = add((nn + 1) * 8), o_lens = add(nn * 4),
                 o_E = add(nn * 2), o_seg = add(nn * 4), o_acc = add(2 * nn),
                 o_cnt = add(2 * nn * 2), o_dist = add(nn * 4), o_serr = add(kMaxSegs * 4);
    size_t o_pl[6];
    for (auto &x : o_pl) x = add((size_t)B.W * 4);
    const size_t o_ord = add(nn * 8), o_idx = add(nn * 8), o_nidx = add(8),
                 o_tiles = add((size_t)compact_tiles(P) * 8),
                 o_bins = add((kNumBatchCfgs + 1) * 8), o_work = add(kWorkCounters * 8),
                 o_hist = add(kNumBinKeys * 8), o_cur = add(kNumBinKeys * 8),
                 o_ident = add(4), o_need = add(nn);
    size_t o_rd[kBatchSlots], o_rf[kBatchSlots], o_sg[kBatchSlots], o_ro[kBatchSlots],
        o_re[kBatchSlots];
    for (int i = 0; i < kBatchSlots; ++i) {
        o_rd[i] = add((size_t)B.B);
        o_rf[i] = add((size_t)B.B);
        o_sg[i] = add(sizeof(SegDesc) * kMaxSegs);
        o_ro[i] = add((nn + kMaxSegs) * 8);
        o_re[i] = add(nn * 2);
    }
    if (cudaMalloc(&B.mem, o) != cudaSuccess) {
        cudaGetLastError();
        return ctx->fail(PF_ENOMEM, "serve batch buffers (%zu bytes)", o);
    }
    char *m = B.mem;
    B.boff = reinterpret_cast<int64_t *>(m + o_boff);
    B.woff = reinterpret_cast<int64_t *>(m + o_woff);
    B.lens = reinterpret_cast<int32_t *>(m + o_lens);
    B.E = reinterpret_cast<int16_t *>(m + o_E);
    B.seg_of = reinterpret_cast<int32_t *>(m + o_seg);
    B.acc = reinterpret_cast<uint8_t *>(m + o_acc);
    B.cnt = reinterpret_cast<int16_t *>(m + o_cnt);
    B.dist = reinterpret_cast<int32_t *>(m + o_dist);
    B.seg_err = reinterpret_cast<unsigned *>(m + o_serr);
    for (int i = 0; i < 6; ++i) B.pl[i] = reinterpret_cast<uint32_t *>(m + o_pl[i]);
    B.scr.order = reinterpret_cast<int64_t *>(m + o_ord);
    B.scr.idx = reinterpret_cast<int64_t *>(m + o_idx);
    B.scr.n_idx = reinterpret_cast<int64_t *>(m + o_nidx);
    B.scr.tiles = reinterpret_cast<int64_t *>(m + o_tiles);
    B.scr.bin_start = reinterpret_cast<int64_t *>(m + o_bins);
    B.scr.work = reinterpret_cast<unsigned long long *>(m + o_work);
    B.scr.hist = reinterpret_cast<unsigned long long *>(m + o_hist);
    B.scr.cursor = reinterpret_cast<unsigned long long *>(m + o_cur);
    B.scr.ident = reinterpret_cast<int *>(m + o_ident);
    B.scr.need = reinterpret_cast<uint8_t *>(m + o_need);
    bool ok = cudaStreamCreateWithFlags(&B.s_compute, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&B.s_copy, cudaStreamNonBlocking) == cudaSuccess;
    for (int i = 0; ok && i < kBatchSlots; ++i) {
        BatchSlot &b = B.slots[i];
        b.reads = reinterpret_cast<uint8_t *>(m + o_rd[i]);
        b.refs = reinterpret_cast<uint8_t *>(m + o_rf[i]);
        b.d_segs = reinterpret_cast<SegDesc *>(m + o_sg[i]);
        b.raw_off = reinterpret_cast<int64_t *>(m + o_ro[i]);
        b.raw_E = reinterpret_cast<int16_t *>(m + o_re[i]);
        void *dp = nullptr;
        ok = cudaHostAlloc(&b.h_segs, sizeof(SegDesc) * kMaxSegs, 0) == cudaSuccess &&
             cudaHostAlloc(&b.h_err, sizeof(unsigned) * kMaxSegs, cudaHostAllocMapped) ==
                 cudaSuccess &&
             cudaHostGetDevicePointer(&dp, b.h_err, 0) == cudaSuccess &&
             cudaEventCreateWithFlags(&b.ev_copied, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreate(&b.ev_enq) == cudaSuccess &&
             cudaEventCreate(&b.ev_phase[0]) == cudaSuccess &&
             cudaEventCreate(&b.ev_phase[1]) == cudaSuccess &&
             cudaEventCreate(&b.ev_phase[2]) == cudaSuccess &&
             cudaEventCreate(&b.ev_phase[3]) == cudaSuccess &&
             cudaEventCreate(&b.ev_start) == cudaSuccess &&
             cudaEventCreate(&b.ev_done) == cudaSuccess;
        b.d_err_map = static_cast<unsigned *>(dp);
        B.free_slots.push_back(kBatchSlots - 1 - i);
    }
    // the serving thread's own context: its stream, side streams and
    // tuning table (copied from ctx), so that calls on ctx may run beside it
    pf_config sc{ctx->device, B.s_compute, 0, 0u};
    ok = ok && pf_create(&B.sub, &sc) == PF_OK;
    if (!ok) {
        cudaGetLastError();
        return ctx->fail(PF_ENOMEM, "serve batch set-up failed");
    }
    std::memcpy(B.sub->tune_cfg, ctx->tune_cfg, sizeof(ctx->tune_cfg));
    std::memcpy(B.sub->tune_plain, ctx->tune_plain, sizeof(ctx->tune_plain));
    std::memcpy(B.sub->tune_chunk, ctx->tune_chunk, sizeof(ctx->tune_chunk));
    B.sub->small_batch = ctx->small_batch;
    B.sub->resolve_bounds = ctx->resolve_bounds;
    // occupancy queries before the first batch
    for (int d = 1; d <= 3; ++d)
        for (int c = 0; c < kNumBatchCfgs; ++c) B.sub->grid_for(d, c);
    B.trace.assign(kTraceCap * PF_SERVE_TRACE_FIELDS, 0.0);
    B.t0 = std::chrono::steady_clock::now();
    return PF_OK;
}

pf_status batch_trace(ServeState *Sp, double *records, int cap, int *count) {
    BatchPool &B = *Sp->bp;
    std::lock_guard<std::mutex> tl(B.trace_mu);
    const uint64_t have = std::min<uint64_t>(B.trace_n, kTraceCap);
    const uint64_t k = std::min<uint64_t>(have, (uint64_t)cap);
    const uint64_t first = B.trace_n - k;   // the k most recent, oldest first
    for (uint64_t i = 0; i < k; ++i)
        std::memcpy(records + i * PF_SERVE_TRACE_FIELDS,
                    &B.trace[((first + i) % kTraceCap) * PF_SERVE_TRACE_FIELDS],
                    sizeof(double) * PF_SERVE_TRACE_FIELDS);
    *count = (int)k;
    return PF_OK;
}

pf_status batch_prepare(pf_ctx *ctx, ServeState *Sp, ServeReq *q) {
    ServeState &S = *Sp;
    const pf_request &r = q->req;
    if (q->longest > S.bp->B)
        return ctx->fail(PF_ENOMEM, "a pair of %lld bytes exceeds the batch area of %lld",
                         (long long)q->longest, (long long)S.bp->B);
    q->d_boff = mapped(r.byte_off);
    q->d_E = mapped(r.E);
    q->in_mapped = q->d_boff && q->d_E;
    q->d_acc = mapped(r.accept);
    q->d_cnt = mapped(r.count);
    q->d_dist = mapped(r.dist);
    q->out_mapped = q->d_acc && q->d_cnt && q->d_dist;
    q->hbytes = staging_need(*q);
    if (q->hbytes > S.stage_budget)
        return ctx->fail(PF_ENOMEM, "request needs %zu pinned staging bytes, pool %zu",
                         q->hbytes, S.stage_budget);
    q->hbytes = 0;
    return PF_OK;
}

void batch_scheduler(ServeState *Sp) {
    ServeState &S = *Sp;
    BatchPool &B = *S.bp;
    cudaSetDevice(S.device);
#if defined(__linux__)
    // short polling sleeps must stay short: the default timer slack of a
    // thread stretches a 5 us sleep to about 55 us
    prctl(PR_SET_TIMERSLACK, 1000UL, 0UL, 0UL, 0UL);
#endif
    using clk = std::chrono::steady_clock;
    double place_s = 0, launch_s = 0, gpu_s = 0;
    uint64_t pairs_sum = 0, pairs_max = 0;
    std::deque<std::shared_ptr<ServeReq>> queue;      // arrival order, not fully placed
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
            S.stats.batch_pairs = pairs_sum;
            S.stats.batch_pairs_max = pairs_max;
            S.stats.batch_gpu_s = gpu_s;
            S.stats.place_host_s = place_s;
            S.stats.launch_host_s = launch_s;
            if (S.quit) break;
            if (queue.empty() && S.pending.empty() && B.inflight.empty())
                S.cv_work.wait_for(lk, std::chrono::milliseconds(20));
            while (!S.pending.empty()) {
                queue.push_back(S.pending.front());
                S.pending.pop_front();
            }
        }
        bool progress = false;
        // finished batches, in launch order
        while (!B.inflight.empty()) {
            BatchSlot &b = B.slots[B.inflight.front()];
            const cudaError_t e = b.failed ? cudaSuccess : cudaEventQuery(b.ev_done);
            if (e == cudaErrorNotReady) break;
            if (e != cudaSuccess) {
                cudaGetLastError();
                S.fatal = "serve batch failed on the device";
                b.failed = true;
            }
            float ms = 0.f, wait_ms = 0.f;
            if (!b.failed && cudaEventElapsedTime(&ms, b.ev_start, b.ev_done) == cudaSuccess)
                gpu_s += ms * 1e-3;
            if (b.failed || cudaEventElapsedTime(&wait_ms, b.ev_enq, b.ev_start) != cudaSuccess)
                wait_ms = -1.f;
            {
                std::lock_guard<std::mutex> tl(B.trace_mu);
                double *r = &B.trace[(B.trace_n % kTraceCap) * PF_SERVE_TRACE_FIELDS];
                r[0] = b.t_launch;
                r[1] = std::chrono::duration<double>(clk::now() - B.t0).count();
                r[2] = (double)b.pairs;
                r[3] = (double)b.nseg;
                r[4] = wait_ms;
                r[5] = ms;
                r[6] = b.host_ms;
                r[7] = (double)b.dec;
                cudaEvent_t marks[6] = {b.ev_start, b.ev_phase[0], b.ev_phase[1], b.ev_phase[2],
                                        b.ev_phase[3], b.ev_done};
                for (int k = 0; k < 5; ++k) {
                    float pm = -1.f;
                    if (b.failed || cudaEventElapsedTime(&pm, marks[k], marks[k + 1]) != cudaSuccess)
                        pm = -1.f;
                    r[8 + k] = pm;
                }
                B.trace_n++;
            }
            complete(S, b, finished);
            B.free_slots.push_back(B.inflight.front());
            B.inflight.pop_front();
            progress = true;
        }
        // place arrivals into the open batch
        const auto t_place = clk::now();
        while (!queue.empty()) {
            const std::shared_ptr<ServeReq> qp = queue.front();
            ServeReq &q = *qp;
            if (!q.admitted && !admit(S, q)) break;  // slots or staging memory
            if (q.req.n == 0) {
                q.t_pub = q.t_seen = std::chrono::steady_clock::now();
                finish(S, q, PF_OK, false);
                finished.push_back(qp);
                queue.pop_front();
                progress = true;
                continue;
            }
            if (B.open < 0) {
                if (B.free_slots.empty()) break;
                B.open = B.free_slots.back();
                B.free_slots.pop_back();
                B.slots[B.open].reset();
            }
            BatchSlot &b = B.slots[B.open];
            const int64_t k = b.full ? 0 : fit(B, b, q);
            if (k == 0 && b.nseg == 0) {  // not even one pair fits an empty batch
                finish(S, q, PF_ENOMEM, false);
                finished.push_back(qp);
                queue.pop_front();
                continue;
            }
            if (k == 0) b.full = true;  // no room left: the rest goes to the next batch
            else {
                place(S, b, qp, k);
                progress = true;
                if (q.next == q.req.n) queue.pop_front();
            }
            if (b.full) {  // waits for the GPU; the next slot opens
                close_uploads(B, b);
                B.ready.push_back(B.open);
                B.open = -1;
            }
        }
        place_s += std::chrono::duration<double>(clk::now() - t_place).count();
        // launch the oldest full batch, else the open one, when the GPU has
        // no batch, or as the second one once it is large (full, or
        // overlap_pairs)
        int next = -1;
        if (!B.ready.empty()) next = B.ready.front();
        else if (B.open >= 0 && B.slots[B.open].nseg > 0) next = B.open;
        if (!S.paused.load() && next >= 0 &&
            (B.inflight.empty() ||
             (B.inflight.size() == 1 &&
              (B.slots[next].full || B.slots[next].pairs >= B.overlap)))) {
            if (next == B.open) B.open = -1;
            else B.ready.pop_front();
            BatchSlot &b = B.slots[next];
            const auto t_launch = clk::now();
            b.t_launch = std::chrono::duration<double>(t_launch - B.t0).count();
            const pf_status st = launch(S, b);
            b.host_ms = std::chrono::duration<double, std::milli>(clk::now() - t_launch).count();
            launch_s += b.host_ms * 1e-3;
            pairs_sum += (uint64_t)b.pairs;
            pairs_max = std::max(pairs_max, (uint64_t)b.pairs);
            const auto now = std::chrono::steady_clock::now();
            for (auto &q : b.reqs) {
                q->t_pub = now;
                if (q->state == ServeReq::STAGING && q->next == q->req.n)
                    q->state = ServeReq::RUNNING;
            }
            if (st != PF_OK) {
                S.fatal = "serve batch launch failed";
                b.failed = true;
            }
            B.inflight.push_back(next);
            S.stats.loop_launches++;
            progress = true;
        }
        if (!progress && finished.empty())
            std::this_thread::sleep_for(std::chrono::microseconds(2));
    }
    // requests the thread still holds end cancelled; pf_serve_stop reports them
    std::lock_guard<std::mutex> lk(S.mu);
    for (auto it = queue.rbegin(); it != queue.rend(); ++it) S.pending.push_front(*it);
}

void batch_stop(ServeState *Sp) {
    ServeState &S = *Sp;
    BatchPool *Bp = S.bp;
    if (!Bp) return;
    BatchPool &B = *Bp;
    if (B.s_copy) cudaStreamSynchronize(B.s_copy);
    if (B.s_compute) cudaStreamSynchronize(B.s_compute);
    {
        std::lock_guard<std::mutex> lk(S.mu);
        for (auto &kv : S.reqs) {
            ServeReq &q = *kv.second;
            if (q.state == ServeReq::DONE) continue;
            finish(S, q, PF_ECANCELLED, false);
            q.state = ServeReq::DONE;
            S.stats.failed++;
        }
        S.pending.clear();
    }
    for (auto &b : B.slots) {
        b.reqs.clear();
        if (b.h_segs) cudaFreeHost(b.h_segs);
        if (b.h_err) cudaFreeHost(b.h_err);
        if (b.ev_copied) cudaEventDestroy(b.ev_copied);
        if (b.ev_start) cudaEventDestroy(b.ev_start);
        if (b.ev_enq) cudaEventDestroy(b.ev_enq);
        for (auto &x : b.ev_phase)
            if (x) cudaEventDestroy(x);
        if (b.ev_done) cudaEventDestroy(b.ev_done);
    }
    if (B.sub) pf_destroy(B.sub);
    if (B.mem) cudaFree(B.mem);
    if (B.s_copy) cudaStreamDestroy(B.s_copy);
    if (B.s_compute) cudaStreamDestroy(B.s_compute);
    delete Bp;
    S.bp = nullptr;
}

}  // namespace pf
