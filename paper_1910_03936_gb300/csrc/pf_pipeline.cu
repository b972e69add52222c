// a7: the whole path on host buffers, in chunks, replayed as CUDA graphs.
// Contract: pf_run_host in pf.h.
//
// Two slots alternate.  A slot owns device buffers for one chunk (ASCII,
// offsets, planes, outputs, scheduler scratch) and a stream.  Its device
// work for a chunk -- offsets and lengths, pack of reads and references,
// the batched filter, compaction, the fill of rejected distances and the
// verification -- is captured once per chunk size as a CUDA graph and then
// launched for every chunk, so a chunk costs one graph launch plus its
// copies.  Chunk c uploads on slot c % 2 while chunk c-1 runs on the other.
#include <algorithm>
#include <cstring>
#include <vector>

#include "pf_ctx.h"
#include "pf_kernels.h"

namespace pf {

namespace {

// Ragged chunk: byte offsets relative to the chunk's first byte, word
// offsets floor(b / 32) + s (disjoint, no scan needed) and lengths.
__global__ void chunk_offsets_kernel(const int64_t *boff_abs, int64_t nc, int64_t *boff,
                                     int64_t *woff, int32_t *lens) {
    const int64_t b0 = boff_abs[0];
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s <= nc;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = boff_abs[s] - b0;
        boff[s] = b;
        woff[s] = (b >> 5) + s;
        if (s < nc) lens[s] = (int32_t)(boff_abs[s + 1] - boff_abs[s]);
    }
}

__global__ void fill_lens_kernel(int32_t *lens, int64_t n, int len) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x)
        lens[s] = len;
}

inline size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t ev_done = nullptr;
    char *mem = nullptr;
    uint8_t *reads = nullptr, *refs = nullptr;
    int64_t *boff_abs = nullptr, *boff = nullptr, *woff = nullptr;
    int32_t *lens = nullptr;
    int16_t *E = nullptr;
    uint32_t *pl[6] = {};
    uint8_t *acc = nullptr;
    int16_t *cnt = nullptr;
    int32_t *dist = nullptr;
    Scratch scr{};
    cudaGraphExec_t exec_full = nullptr, exec_tail = nullptr;
    int64_t c0 = -1, nc = 0;   // chunk in flight
};

struct Job {
    pf_ctx *ctx;
    unsigned dec;
    const uint8_t *reads, *refs;
    const int64_t *byte_off;
    int len;
    const int16_t *E;
    int E_max;
    uint8_t *accept;
    int16_t *count;
    int32_t *dist;
    int64_t n, C;
    int slots;
    size_t bytes_max, words_max;
};

pf_status alloc_slot(Job &J, Slot &s) {
    const size_t C = (size_t)J.C, sl = (size_t)J.slots;
    size_t o = 0;
    auto add = [&](size_t b) {
        const size_t at = o;
        o += up256(b);
        return at;
    };
    const size_t o_r = add(J.bytes_max), o_f = add(J.bytes_max), o_ba = add((C + 1) * 8),
                 o_b = add((C + 1) * 8), o_w = add((C + 1) * 8), o_l = add(C * 4),
                 o_e = add(C * 2);
    size_t o_p[6];
    for (auto &x : o_p) x = add(J.words_max * 4);
    const size_t o_acc = add(sl * C), o_cnt = add(sl * C * 2), o_dist = add(C * 4);
    const size_t o_ord = add(C * 8), o_idx = add(C * 8), o_nidx = add(8),
                 o_tiles = add((size_t)compact_tiles((int64_t)C) * 8),
                 o_bins = add((kNumBatchCfgs + 1) * 8), o_work = add(kWorkCounters * 8),
                 o_hist = add(kNumBinKeys * 8), o_cur = add(kNumBinKeys * 8),
                 o_ident = add(4), o_need = add(C);
    if (cudaMalloc(&s.mem, o) != cudaSuccess) {
        cudaGetLastError();
        return J.ctx->fail(PF_ENOMEM, "pf_run_host: %zu device bytes per slot", o);
    }
    char *m = s.mem;
    s.reads = reinterpret_cast<uint8_t *>(m + o_r);
    s.refs = reinterpret_cast<uint8_t *>(m + o_f);
    s.boff_abs = reinterpret_cast<int64_t *>(m + o_ba);
    s.boff = reinterpret_cast<int64_t *>(m + o_b);
    s.woff = reinterpret_cast<int64_t *>(m + o_w);
    s.lens = reinterpret_cast<int32_t *>(m + o_l);
    s.E = reinterpret_cast<int16_t *>(m + o_e);
    for (int i = 0; i < 6; ++i) s.pl[i] = reinterpret_cast<uint32_t *>(m + o_p[i]);
    s.acc = reinterpret_cast<uint8_t *>(m + o_acc);
    s.cnt = reinterpret_cast<int16_t *>(m + o_cnt);
    s.dist = reinterpret_cast<int32_t *>(m + o_dist);
    s.scr.order = reinterpret_cast<int64_t *>(m + o_ord);
    s.scr.idx = reinterpret_cast<int64_t *>(m + o_idx);
    s.scr.n_idx = reinterpret_cast<int64_t *>(m + o_nidx);
    s.scr.tiles = reinterpret_cast<int64_t *>(m + o_tiles);
    s.scr.bin_start = reinterpret_cast<int64_t *>(m + o_bins);
    s.scr.work = reinterpret_cast<unsigned long long *>(m + o_work);
    s.scr.hist = reinterpret_cast<unsigned long long *>(m + o_hist);
    s.scr.cursor = reinterpret_cast<unsigned long long *>(m + o_cur);
    s.scr.ident = reinterpret_cast<int *>(m + o_ident);
    s.scr.need = reinterpret_cast<uint8_t *>(m + o_need);
    if (cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s.ev_done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return J.ctx->fail(PF_ECUDA, "pf_run_host: stream/event creation failed");
    }
    if (!J.byte_off) {
        fill_lens_kernel<<<std::max<int64_t>(1, std::min<int64_t>((J.C + 255) / 256, 1024)), 256,
                           0, s.st>>>(s.lens, J.C, J.len);
        if (cudaGetLastError() != cudaSuccess) return J.ctx->fail(PF_ECUDA, "fill launch");
    }
    return PF_OK;
}

// The device work of one chunk of nc pairs on slot s, on s.st.
pf_status enqueue_chunk(Job &J, Slot &s, int64_t nc) {
    pf_ctx *ctx = J.ctx;
    PairsView pv;
    pv.read = SeqView{s.pl[0], s.pl[1], s.pl[2], nullptr, 0};
    pv.ref = SeqView{s.pl[3], s.pl[4], s.pl[5], nullptr, 0};
    cudaError_t e = cudaSuccess;
    if (J.byte_off) {
        const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((nc + 256) / 256, 4096));
        chunk_offsets_kernel<<<blocks, 256, 0, s.st>>>(s.boff_abs, nc, s.boff, s.woff, s.lens);
        e = cudaGetLastError();
        if (e == cudaSuccess)
            e = launch_pack_ragged(s.reads, s.boff, s.woff, nc, s.pl[0], s.pl[1], s.pl[2],
                                   ctx->d_err, s.st);
        if (e == cudaSuccess)
            e = launch_pack_ragged(s.refs, s.boff, s.woff, nc, s.pl[3], s.pl[4], s.pl[5],
                                   ctx->d_err, s.st);
        pv.read.off = s.woff;
        pv.ref.off = s.woff;
    } else {
        const int W = (J.len + 31) / 32;
        e = launch_pack_fixed(s.reads, nc, J.len, s.pl[0], s.pl[1], s.pl[2], ctx->d_err, ctx->sms,
                              s.st);
        if (e == cudaSuccess)
            e = launch_pack_fixed(s.refs, nc, J.len, s.pl[3], s.pl[4], s.pl[5], ctx->d_err,
                                  ctx->sms, s.st);
        pv.read.stride = W;
        pv.ref.stride = W;
    }
    if (e != cudaSuccess) return ctx->cuda(e, "pf_run_host pack");
    FilterArgs a;
    a.pairs = pv;
    a.lens = s.lens;
    a.E = J.E ? s.E : nullptr;
    a.E_max = J.E_max;
    a.accept = s.acc;
    a.count = s.cnt;
    a.n = nc;
    a.err = ctx->d_err;
    a.dist = s.dist;  // E + 1 for the pairs the filter rejects
    if (ctx->resolve_bounds && (J.dec & 1u)) a.need = s.scr.need;
    cudaStream_t saved = ctx->stream;
    ctx->stream = s.st;
    pf_status st = ctx->run_filter(J.dec, a, s.scr);
    ctx->stream = saved;
    if (st != PF_OK) return st;
    e = launch_compact(a.need ? a.need : s.acc, nc, s.scr.idx, s.scr.n_idx, s.scr.tiles, s.st,
                       ctx->binned ? s.scr.order : nullptr, s.scr.ident);
    if (e == cudaSuccess)
        e = launch_verify(pv, s.lens, a.E, J.E_max, s.scr.idx, s.scr.n_idx, nc, s.dist,
                          ctx->d_err, ctx->sms, s.st, s.scr.work + kNumBatchCfgs, ctx->binned);
    return ctx->cuda(e, "pf_run_host launch");
}

pf_status capture(Job &J, Slot &s, int64_t nc, cudaGraphExec_t *exec) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s.st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return J.ctx->cuda(e, "pf_run_host capture");
    pf_status st = enqueue_chunk(J, s, nc);
    e = cudaStreamEndCapture(s.st, &g);
    if (st != PF_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return J.ctx->cuda(e, "pf_run_host end capture");
    e = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    return J.ctx->cuda(e, "pf_run_host instantiate");
}

void free_slot(Slot &s) {
    if (s.st) cudaStreamSynchronize(s.st);
    if (s.exec_full) cudaGraphExecDestroy(s.exec_full);
    if (s.exec_tail) cudaGraphExecDestroy(s.exec_tail);
    if (s.mem) cudaFree(s.mem);
    if (s.ev_done) cudaEventDestroy(s.ev_done);
    if (s.st) cudaStreamDestroy(s.st);
}

// Results of the chunk on slot s into the caller's buffers.
void copy_out(Job &J, Slot &s) {
    const size_t nc = (size_t)s.nc, c0 = (size_t)s.c0, n = (size_t)J.n;
    for (int k = 0; k < J.slots; ++k) {
        cudaMemcpyAsync(J.accept + k * n + c0, s.acc + k * nc, nc, cudaMemcpyDeviceToHost, s.st);
        cudaMemcpyAsync(J.count + k * n + c0, s.cnt + k * nc, nc * 2, cudaMemcpyDeviceToHost,
                        s.st);
    }
    cudaMemcpyAsync(J.dist + c0, s.dist, nc * 4, cudaMemcpyDeviceToHost, s.st);
}

}  // namespace

}  // namespace pf

using namespace pf;

extern "C" pf_status pf_run_host(pf_ctx *ctx, unsigned deciders, const uint8_t *reads,
                                 const uint8_t *refs, const int64_t *byte_off, int len,
                                 const int16_t *E, int E_max, uint8_t *accept, int16_t *count,
                                 int32_t *dist, int64_t n, int64_t chunk_pairs) {
    if (!ctx) return PF_EINVAL;
    if (n < 0 || chunk_pairs < 0 || (deciders & 3u) == 0 || (deciders & ~3u) || E_max < 0 ||
        E_max > PF_MAX_E || (!byte_off && len < 0))
        return ctx->fail(PF_EINVAL, "pf_run_host: bad arguments");
    if (n == 0) return PF_OK;
    if (!reads || !refs || !accept || !count || !dist)
        return ctx->fail(PF_EINVAL, "pf_run_host: null pointer argument");
    cudaSetDevice(ctx->device);
    Job J{ctx, deciders, reads, refs, byte_off, len, E, E_max, accept, count, dist, n,
          chunk_pairs ? chunk_pairs : (int64_t)1 << 20, deciders == 3u ? 2 : 1, 0, 0};
    J.C = std::min(J.C, n);
    const int64_t nchunks = (n + J.C - 1) / J.C;
    // the largest chunk in bytes and words
    if (byte_off) {
        int64_t bmax = 0;
        for (int64_t c = 0; c < nchunks; ++c) {
            const int64_t a = c * J.C, b = std::min(n, a + J.C);
            if (byte_off[b] < byte_off[a]) return ctx->fail(PF_EINVAL, "offsets decrease");
            bmax = std::max(bmax, byte_off[b] - byte_off[a]);
        }
        J.bytes_max = (size_t)bmax;
        J.words_max = (size_t)(bmax >> 5) + (size_t)J.C + 1;
    } else {
        J.bytes_max = (size_t)J.C * (size_t)len;
        J.words_max = (size_t)J.C * (size_t)((len + 31) / 32);
    }
    // occupancy queries before any capture
    for (int c = 0; c < kNumBatchCfgs; ++c) ctx->grid_for((int)deciders, c);

    Slot slots[2];
    pf_status st = PF_OK;
    const int64_t tail = n - (nchunks - 1) * J.C;
    for (int i = 0; i < 2 && st == PF_OK; ++i) {
        st = alloc_slot(J, slots[i]);
        if (st == PF_OK) st = capture(J, slots[i], J.C, &slots[i].exec_full);
        if (st == PF_OK && tail != J.C) st = capture(J, slots[i], tail, &slots[i].exec_tail);
    }
    for (int64_t c = 0; c < nchunks && st == PF_OK; ++c) {
        Slot &s = slots[c & 1];
        const int64_t c0 = c * J.C, nc = std::min(J.C, n - c0);
        // the slot's previous chunk: results are in host memory once its
        // copies (queued on the same stream) are done
        s.c0 = c0;
        s.nc = nc;
        const int64_t b0 = byte_off ? byte_off[c0] : c0 * (int64_t)len;
        const int64_t nb = byte_off ? byte_off[c0 + nc] - b0 : nc * (int64_t)len;
        if (nb) {
            cudaMemcpyAsync(s.reads, reads + b0, (size_t)nb, cudaMemcpyHostToDevice, s.st);
            cudaMemcpyAsync(s.refs, refs + b0, (size_t)nb, cudaMemcpyHostToDevice, s.st);
        }
        if (byte_off)
            cudaMemcpyAsync(s.boff_abs, byte_off + c0, (size_t)(nc + 1) * 8, cudaMemcpyHostToDevice,
                            s.st);
        if (E) cudaMemcpyAsync(s.E, E + c0, (size_t)nc * 2, cudaMemcpyHostToDevice, s.st);
        st = ctx->cuda(cudaGraphLaunch(nc == J.C ? s.exec_full : s.exec_tail, s.st),
                       "pf_run_host graph launch");
        if (st != PF_OK) break;
        copy_out(J, s);
        cudaEventRecord(s.ev_done, s.st);
    }
    for (auto &s : slots) free_slot(s);
    if (st != PF_OK) return st;
    st = ctx->cuda(cudaGetLastError(), "pf_run_host");
    if (st != PF_OK) return st;
    return pf_sync(ctx);
}
