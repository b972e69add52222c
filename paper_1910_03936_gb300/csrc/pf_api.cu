// C-ABI of the library: context, argument checks, the batch scheduler
// (binning by threshold, tuned kernel per bin, concurrent persistent
// launches) and the whole-path call.  Declarations and contracts: pf.h.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "pf_ctx.h"
#include "pf_kernels.h"

using namespace pf;

namespace pf {

// ---------------------------------------------------------------------------
// binning kernels: group pair indices by the configuration of their E

struct BinTable {
    int cfg_of_E[PF_MAX_E + 1];
};

__global__ void bin_init_kernel(int64_t *bin_start, unsigned long long *work,
                                unsigned long long *hist, int nb, int single_cfg, int64_t n) {
    for (int i = threadIdx.x; i <= nb; i += blockDim.x) {
        bin_start[i] = (single_cfg >= 0) ? (i <= single_cfg ? 0 : n) : 0;
        if (i < nb) work[i] = 0ull;
    }
    for (int i = threadIdx.x; i < kNumBinKeys; i += blockDim.x) hist[i] = 0ull;
}

// Key of pair p: its threshold's configuration, then its length class.
// Inside a configuration the pairs of one length run together (a warp does
// not wait on its longest pair), and in a layout grouped by threshold and
// length (pf_pack_layout_grouped) they lie together in the planes.
__device__ __forceinline__ int len_class(int len) {
    const int wc = len <= 0 ? 0 : ((len - 1) >> 5) + 1;
    return wc < kLenClasses - 1 ? wc : kLenClasses - 1;
}

// tab[e] = the first key of E = e's configuration, staged in shared memory
// by each block (indexing the kernel parameter by a run-time threshold
// costs far more).
__device__ __forceinline__ void stage_keys(const BinTable &t, int *tab) {
    if (threadIdx.x <= PF_MAX_E) tab[threadIdx.x] = t.cfg_of_E[threadIdx.x] * kLenClasses;
}

__device__ __forceinline__ int key_of(int e, int len, int E_max, const int *tab) {
    e = e < 0 ? 0 : (e > E_max ? E_max : e);
    return tab[e] + len_class(len);
}

// Each thread counts 8 consecutive pairs per round (one 16-byte load of
// thresholds, two of lengths), adding a run of equal keys to its counter
// at once.  The threshold -> key table is staged in shared memory.
constexpr int kHistPer = 8;

__global__ void __launch_bounds__(256)
bin_hist_kernel(const int16_t *E, const int32_t *lens, int64_t n, int E_max, BinTable t,
                unsigned long long *hist) {
    __shared__ unsigned cnt[kNumBinKeys];
    __shared__ int tab[PF_MAX_E + 1];
    for (int i = threadIdx.x; i < kNumBinKeys; i += blockDim.x) cnt[i] = 0;
    stage_keys(t, tab);
    __syncthreads();
    const bool vec = ((reinterpret_cast<uintptr_t>(E) | reinterpret_cast<uintptr_t>(lens)) & 15u) == 0;
    int cur = -1;
    unsigned run = 0;
    auto add = [&](int e, int len) {
        const int key = key_of(e, len, E_max, tab);
        if (key != cur) {
            if (run) atomicAdd(&cnt[cur], run);
            cur = key;
            run = 0;
        }
        ++run;
    };
    for (int64_t p0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * kHistPer; p0 < n;
         p0 += (int64_t)gridDim.x * blockDim.x * kHistPer) {
        if (vec && p0 + kHistPer <= n) {
            const int4 ev = __ldg(reinterpret_cast<const int4 *>(E + p0));
            const int4 la = __ldg(reinterpret_cast<const int4 *>(lens + p0));
            const int4 lb = __ldg(reinterpret_cast<const int4 *>(lens + p0 + 4));
            add((int16_t)(ev.x & 0xffff), la.x);
            add((int16_t)((unsigned)ev.x >> 16), la.y);
            add((int16_t)(ev.y & 0xffff), la.z);
            add((int16_t)((unsigned)ev.y >> 16), la.w);
            add((int16_t)(ev.z & 0xffff), lb.x);
            add((int16_t)((unsigned)ev.z >> 16), lb.y);
            add((int16_t)(ev.w & 0xffff), lb.z);
            add((int16_t)((unsigned)ev.w >> 16), lb.w);
        } else {
            for (int64_t p = p0; p < n && p < p0 + kHistPer; ++p) add(__ldg(E + p), __ldg(lens + p));
        }
    }
    if (run) atomicAdd(&cnt[cur], run);
    __syncthreads();
    for (int i = threadIdx.x; i < kNumBinKeys; i += blockDim.x)
        if (cnt[i]) atomicAdd(&hist[i], (unsigned long long)cnt[i]);
}

// One warp: exclusive scan of the key counts into the scatter's cursors; a
// configuration's bin starts at its first key.  When every pair falls in
// one configuration the grouping is the identity: `ident` tells the
// scatter to skip and the filter to index pairs directly (pair order is
// kept; the length classes are not separated).
__global__ void bin_scan_kernel(const unsigned long long *hist, int64_t *bin_start,
                                unsigned long long *cursor, int *ident) {
    constexpr int kPer = (kNumBinKeys + 31) / 32;
    __shared__ unsigned long long h[kNumBinKeys];
    const int lane = threadIdx.x;
    if (lane >= 32) return;
    for (int i = lane; i < kNumBinKeys; i += 32) h[i] = hist[i];  // independent loads
    __syncwarp();
    int64_t sum = 0;
    for (int k = 0; k < kPer; ++k) {
        const int i = lane * kPer + k;
        if (i < kNumBinKeys) sum += (int64_t)h[i];
    }
    int64_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    int64_t run = inc - sum;
    for (int k = 0; k < kPer; ++k) {
        const int i = lane * kPer + k;
        if (i >= kNumBinKeys) break;
        cursor[i] = (unsigned long long)run;
        if (i % kLenClasses == 0) bin_start[i / kLenClasses] = run;
        run += (int64_t)h[i];
    }
    if (lane == 31) bin_start[kNumBatchCfgs] = inc;
    int used = 0;
    for (int c0 = 0; c0 < kNumBatchCfgs; c0 += 32) {
        const int c = c0 + lane;
        bool any = false;
        if (c < kNumBatchCfgs)
            for (int j = 0; j < kLenClasses; ++j) any |= h[c * kLenClasses + j] != 0ull;
        used += __popc(__ballot_sync(0xffffffffu, any));
    }
    if (lane == 0) *ident = (used <= 1);
}

// Each block takes tiles of 2,048 pairs, 8 rounds of 256 consecutive pairs
// (one per thread), ranks them per key in shared memory and claims room for
// the tile's pairs per key with one global atomic per key.  Large tiles
// keep the contended global cursors (one per key, a few dozen in use) to a
// few atomics per 2,048 pairs.  Order inside a tile's share follows the
// order in which the warps' atomics land: a warp's pairs of one key keep
// their order, so a bin's pairs stay in runs of consecutive pairs (which a
// layout grouped by threshold and length keeps side by side in memory).
// Results do not depend on it: every pair keeps its own index.
constexpr int kScatterPer = 8;

__global__ void __launch_bounds__(256)
bin_scatter_kernel(const int16_t *E, const int32_t *lens, int64_t n, int E_max, BinTable t,
                   unsigned long long *cursor, int64_t *order, const int *ident) {
    __shared__ unsigned cnt[kNumBinKeys];
    __shared__ unsigned long long base[kNumBinKeys];
    __shared__ int tab[PF_MAX_E + 1];
    if (*ident) return;
    stage_keys(t, tab);
    constexpr int64_t kTile = 256 * kScatterPer;
    for (int64_t t0 = (int64_t)blockIdx.x * kTile; t0 < n; t0 += (int64_t)gridDim.x * kTile) {
        for (int i = threadIdx.x; i < kNumBinKeys; i += blockDim.x) cnt[i] = 0;
        __syncthreads();  // tab staged; cnt zeroed
        const int64_t p0 = t0 + threadIdx.x;
        int key[kScatterPer];
        unsigned rank[kScatterPer];
#pragma unroll
        for (int k = 0; k < kScatterPer; ++k) {
            const int64_t p = p0 + k * 256;
            key[k] = p < n ? key_of(__ldg(E + p), __ldg(lens + p), E_max, tab) : -1;
            rank[k] = key[k] >= 0 ? atomicAdd(&cnt[key[k]], 1u) : 0u;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kNumBinKeys; i += blockDim.x)
            base[i] = cnt[i] ? atomicAdd(&cursor[i], (unsigned long long)cnt[i]) : 0ull;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kScatterPer; ++k)
            if (key[k] >= 0) order[base[key[k]] + rank[k]] = p0 + k * 256;
        __syncthreads();  // cnt and base are reused by the next tile
    }
}

}  // namespace pf

// ---------------------------------------------------------------------------
// context helpers

static thread_local std::string g_tls_msg;

pf_status pf_ctx::fail(pf_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    std::lock_guard<std::mutex> lk(mu);
    if (sticky == PF_OK) {
        sticky = s;
        msg = buf;
    }
    return s;
}

pf_status pf_ctx::cuda(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return PF_OK;
    return fail(PF_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

pf_status pf_ctx::ensure_scratch(size_t bytes) {
    if (bytes <= scratch_bytes) return PF_OK;
    verified_state = 0;
    if (scratch) {
        cudaStreamSynchronize(stream);
        cudaFree(scratch);
        scratch = nullptr;
        scratch_bytes = 0;
    }
    size_t want = std::max(bytes, scratch_bytes * 3 / 2);
    if (cudaMalloc(&scratch, want) != cudaSuccess) {
        cudaGetLastError();
        if (cudaMalloc(&scratch, bytes) != cudaSuccess) {
            cudaGetLastError();
            scratch = nullptr;
            return fail(PF_ENOMEM, "scratch allocation of %zu bytes failed", bytes);
        }
        want = bytes;
    }
    scratch_bytes = want;
    return PF_OK;
}

// Carve the scratch block: returns pointers for n pairs.
pf_status pf_ctx::scratch_layout(int64_t n, Scratch *s) {
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t nn = (size_t)std::max<int64_t>(n, 1);
    size_t off = 0;
    const size_t o_nidx = off;  off += up(sizeof(int64_t));  // first: pf_last_verified_count
    const size_t o_order = off; off += up(nn * sizeof(int64_t));
    const size_t o_idx = off;   off += up(nn * sizeof(int64_t));
    const size_t o_tiles = off; off += up((size_t)compact_tiles((int64_t)nn) * sizeof(int64_t));
    const size_t o_bins = off;  off += up((kNumBatchCfgs + 1) * sizeof(int64_t));
    const size_t o_work = off;  off += up(kWorkCounters * sizeof(unsigned long long));
    const size_t o_hist = off;  off += up(kNumBinKeys * sizeof(unsigned long long));
    const size_t o_cur = off;   off += up(kNumBinKeys * sizeof(unsigned long long));
    const size_t o_ident = off; off += up(sizeof(int));
    const size_t o_need = off;  off += up(nn);
    pf_status st = ensure_scratch(off);
    if (st != PF_OK) return st;
    char *b = static_cast<char *>(scratch);
    s->order = reinterpret_cast<int64_t *>(b + o_order);
    s->idx = reinterpret_cast<int64_t *>(b + o_idx);
    s->n_idx = reinterpret_cast<int64_t *>(b + o_nidx);
    s->tiles = reinterpret_cast<int64_t *>(b + o_tiles);
    s->bin_start = reinterpret_cast<int64_t *>(b + o_bins);
    s->work = reinterpret_cast<unsigned long long *>(b + o_work);
    s->hist = reinterpret_cast<unsigned long long *>(b + o_hist);
    s->cursor = reinterpret_cast<unsigned long long *>(b + o_cur);
    s->ident = reinterpret_cast<int *>(b + o_ident);
    s->need = reinterpret_cast<uint8_t *>(b + o_need);
    return PF_OK;
}

int pf_ctx::grid_for(int dec, int cfg) {
    int &g = grid_cache[dec][cfg];
    if (g == 0) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, filter_batched_fn(dec, cfg),
                                                      cfg_threads(kBatchCfgs[cfg], dec),
                                                      cfg_smem(kBatchCfgs[cfg], dec));
        g = std::max(1, per_sm) * sms;
    }
    return g;
}

// Default configuration for threshold E before any tuning: the
// exact-threshold one-thread kernel up to E = 15 (its two-phase form for
// E = 1..7, with shared arrays that hold pairs up to 256 bases), eight
// lanes per pair above (the two-phase lane-group form: at 250 bp, E = 25 it
// takes 3.26 ms per 2M pairs with both deciders against 3.74 for the fused
// loop).
int pf::pf_default_cfg(int E) {
    if (E >= 1 && E <= 7)
        for (int c = 0; c < kNumBatchCfgs; ++c)
            if (kBatchCfgs[c].xe == E && kBatchCfgs[c].words >= 8) return c;
    if (E <= 15) return kFirstExactCfg + E;
    // the two-phase form with two or four lanes per pair and the fewest
    // slots that hold the 2E+1 diagonals (four lanes on a tie)
    int best = -1;
    for (int c = 0; c < kNumBatchCfgs; ++c) {
        const KernelCfg &k = kBatchCfgs[c];
        if ((k.tpp != 2 && k.tpp != 4) || k.xe >= 0 || k.ecap < E || k.words < 8) continue;
        if (best < 0 || k.ecap < kBatchCfgs[best].ecap ||
            (k.ecap == kBatchCfgs[best].ecap && k.tpp > kBatchCfgs[best].tpp))
            best = c;
    }
    return best;
}

// E = 0 compares one diagonal and is bound by memory: the plain kernel
// (full occupancy, no shared work counter) is the default there.
static bool default_plain(int E) { return E == 0; }

void pf_ctx::reset_tuning() {
    for (int d = 0; d < 4; ++d)
        for (int e = 0; e <= PF_MAX_E; ++e) {
            tune_cfg[d][e] = pf_default_cfg(e);
            tune_chunk[d][e] = 256;
            tune_plain[d][e] = default_plain(e);
        }
}

// ---------------------------------------------------------------------------
// argument checks

static bool seqs_ok(const pf_seqs &s) {
    return s.lo && s.hi && s.nmask && (s.word_off || s.stride_words >= 0);
}

static PairsView to_view(const pf_pairs *p) {
    PairsView v;
    v.read = SeqView{p->read.lo, p->read.hi, p->read.nmask, p->read.word_off, p->read.stride_words};
    v.ref = SeqView{p->ref.lo, p->ref.hi, p->ref.nmask, p->ref.word_off, p->ref.stride_words};
    return v;
}

static pf_status check_filter_args(pf_ctx *ctx, unsigned deciders, const pf_pairs *pairs,
                                   const int32_t *lens, int E_max, uint8_t *accept,
                                   int16_t *count, int64_t n) {
    if (!ctx) return PF_EINVAL;
    if (n < 0) return ctx->fail(PF_EINVAL, "n = %lld < 0", (long long)n);
    if ((deciders & 3u) == 0 || (deciders & ~3u))
        return ctx->fail(PF_EINVAL, "deciders must be PF_SNEAKYSNAKE, PF_GATEKEEPER or both");
    if (E_max < 0 || E_max > PF_MAX_E)
        return ctx->fail(PF_EINVAL, "E_max = %d outside [0, %d]", E_max, PF_MAX_E);
    if (n == 0) return PF_OK;
    if (!pairs || !seqs_ok(pairs->read) || !seqs_ok(pairs->ref) || !lens || !accept || !count)
        return ctx->fail(PF_EINVAL, "null pointer argument");
    return PF_OK;
}

static FilterArgs make_filter_args(pf_ctx *ctx, const pf_pairs *pairs, const int32_t *lens,
                                   const int16_t *E, int E_max, uint8_t *accept, int16_t *count,
                                   int64_t n) {
    FilterArgs a;
    a.pairs = to_view(pairs);
    a.lens = lens;
    a.E = E;
    a.E_max = E_max;
    a.accept = accept;
    a.count = count;
    a.n = n;
    a.err = ctx->d_err;
    return a;
}

// ---------------------------------------------------------------------------
// scheduler

pf_status pf_ctx::run_batched(unsigned dec, const FilterArgs &a, const Scratch &s) {
    BatchArgs b;
    b.f = a;
    b.bin_start = s.bin_start;
    b.bin_cfg = nullptr;
    b.nbins = kNumBatchCfgs;
    b.work = s.work;
    b.chunk_start = nullptr;
    std::vector<int> used;
    int single = -1;
    if (!a.E) {
        single = tune_cfg[dec][a.E_max];
        used.push_back(single);
        b.order = nullptr;
    } else {
        b.order = s.order;
        for (int e = 0; e <= a.E_max; ++e) {
            const int c = tune_cfg[dec][e];
            if (std::find(used.begin(), used.end(), c) == used.end()) used.push_back(c);
        }
        if (used.size() == 1) {
            single = used[0];
            b.order = nullptr;
        }
    }
    b.ident = (single < 0) ? s.ident : nullptr;
    binned = single < 0;
    bin_init_kernel<<<1, 32, 0, stream>>>(s.bin_start, s.work, s.hist, kNumBatchCfgs, single,
                                          a.n);
    if (single < 0) {
        BinTable t;
        for (int e = 0; e <= PF_MAX_E; ++e) t.cfg_of_E[e] = tune_cfg[dec][std::min(e, a.E_max)];
        const int64_t hh = std::min<int64_t>((a.n + 256 * kHistPer - 1) / (256 * kHistPer),
                                             (int64_t)sms * 8);
        bin_hist_kernel<<<(unsigned)std::max<int64_t>(hh, 1), 256, 0, stream>>>(
            a.E, a.lens, a.n, a.E_max, t, s.hist);
        bin_scan_kernel<<<1, 32, 0, stream>>>(s.hist, s.bin_start, s.cursor, s.ident);
        bin_scatter_kernel<<<(unsigned)std::max<int64_t>(hh, 1), 256, 0, stream>>>(
            a.E, a.lens, a.n, a.E_max, t, s.cursor, s.order, s.ident);
    }
    pf_status st = cuda(cudaGetLastError(), "binning launch");
    if (st != PF_OK) return st;

    if (used.size() == 1) {
        const int c = used[0];
        b.chunk = tune_chunk[dec][a.E_max];
        // enough warps for each to take one step of pairs at once (the
        // kernels shrink their work items to spread a short batch over the
        // grid), at most one resident wave
        const int64_t steps = (a.n + cfg_step(kBatchCfgs[c], (int)dec) - 1) /
                              cfg_step(kBatchCfgs[c], (int)dec);
        const int wpb = cfg_threads(kBatchCfgs[c], (int)dec) / 32;  // warps per block
        const int grid = (int)std::min<int64_t>(grid_for(dec, c),
                                                std::max<int64_t>(1, (steps + wpb - 1) / wpb));
        return cuda(launch_filter_batched(dec, c, grid, b, c, stream), "filter launch");
    }
    // several configurations: one persistent launch each, concurrently
    cudaEventRecord(ev_fork, stream);
    for (size_t i = 0; i < used.size(); ++i) {
        cudaStream_t side = side_streams[i % kSideStreams];
        cudaStreamWaitEvent(side, ev_fork, 0);
        const int c = used[i];
        BatchArgs bi = b;
        bi.chunk = 256;
        for (int e = 0; e <= a.E_max; ++e)
            if (tune_cfg[dec][e] == c) bi.chunk = tune_chunk[dec][e];
        const int grid = grid_for(dec, c);
        st = cuda(launch_filter_batched(dec, c, grid, bi, c, side), "filter launch");
        if (st != PF_OK) return st;
    }
    for (int i = 0; i < kSideStreams && i < (int)used.size(); ++i) {
        cudaEventRecord(ev_join[i], side_streams[i]);
        cudaStreamWaitEvent(stream, ev_join[i], 0);
    }
    return cuda(cudaGetLastError(), "filter launch");
}

// ---------------------------------------------------------------------------
// C ABI

extern "C" {

const char *pf_status_string(pf_status s) {
    switch (s) {
        case PF_OK: return "PF_OK";
        case PF_EINVAL: return "PF_EINVAL";
        case PF_ENOMEM: return "PF_ENOMEM";
        case PF_ECUDA: return "PF_ECUDA";
        case PF_ETIMEOUT: return "PF_ETIMEOUT";
        case PF_EBUSY: return "PF_EBUSY";
        case PF_ECANCELLED: return "PF_ECANCELLED";
        case PF_EDATA: return "PF_EDATA";
    }
    return "PF_?";
}

pf_status pf_create(pf_ctx **out, const pf_config *cfg) {
    if (!out || !cfg || cfg->flags != 0) return PF_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) {
        cudaGetLastError();
        g_tls_msg = "no such CUDA device";
        return PF_ECUDA;
    }
    if (cudaSetDevice(cfg->device) != cudaSuccess) return PF_ECUDA;
    pf_ctx *c = new pf_ctx();
    c->device = cfg->device;
    c->stream = static_cast<cudaStream_t>(cfg->stream);
    if (!c->stream) c->stream = cudaStreamPerThread;
    c->hbm_budget = cfg->hbm_budget;
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, cfg->device);
    bool ok = cudaMalloc(&c->d_err, sizeof(unsigned)) == cudaSuccess &&
              cudaMemset(c->d_err, 0, sizeof(unsigned)) == cudaSuccess &&
              cudaMallocHost(&c->h_err, sizeof(unsigned)) == cudaSuccess &&
              cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; ok && i < kSideStreams; ++i)
        ok = cudaStreamCreateWithFlags(&c->side_streams[i], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&c->ev_join[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        pf_destroy(c);
        return PF_ECUDA;
    }
    *c->h_err = 0;
    c->reset_tuning();
    *out = c;
    return PF_OK;
}

pf_status pf_destroy(pf_ctx *ctx) {
    if (!ctx) return PF_EINVAL;
    cudaSetDevice(ctx->device);
    pf_serve_teardown(ctx);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    if (ctx->scratch) cudaFree(ctx->scratch);
    if (ctx->d_err) cudaFree(ctx->d_err);
    if (ctx->h_err) cudaFreeHost(ctx->h_err);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    for (int i = 0; i < kSideStreams; ++i) {
        if (ctx->side_streams[i]) cudaStreamDestroy(ctx->side_streams[i]);
        if (ctx->ev_join[i]) cudaEventDestroy(ctx->ev_join[i]);
    }
    delete ctx;
    return PF_OK;
}

pf_status pf_set_stream(pf_ctx *ctx, void *stream) {
    if (!ctx) return PF_EINVAL;
    ctx->stream = stream ? static_cast<cudaStream_t>(stream) : cudaStreamPerThread;
    return PF_OK;
}

pf_status pf_set_resolve_by_bounds(pf_ctx *ctx, int enable) {
    if (!ctx) return PF_EINVAL;
    ctx->resolve_bounds = enable != 0;
    return PF_OK;
}

pf_status pf_sync(pf_ctx *ctx) {
    if (!ctx) return PF_EINVAL;
    cudaSetDevice(ctx->device);
    pf_status st = ctx->cuda(cudaMemcpyAsync(ctx->h_err, ctx->d_err, sizeof(unsigned),
                                             cudaMemcpyDeviceToHost, ctx->stream),
                             "error word copy");
    if (st == PF_OK) st = ctx->cuda(cudaStreamSynchronize(ctx->stream), "stream sync");
    if (st == PF_OK && *ctx->h_err) {
        const unsigned e = *ctx->h_err;
        *ctx->h_err = 0;
        cudaMemsetAsync(ctx->d_err, 0, sizeof(unsigned), ctx->stream);
        cudaStreamSynchronize(ctx->stream);
        if (e & ERR_PAIR_ARGS)
            ctx->fail(PF_EINVAL, "a pair had a negative length or E outside [0, E_max]");
        else if (e & ERR_TIMEOUT)
            ctx->fail(PF_ETIMEOUT, "a bounded device wait ran out");
        else if (e & ERR_BYTES)
            ctx->fail(PF_EDATA, "input bytes other than A/C/G/T/N were packed as N");
    }
    std::lock_guard<std::mutex> lk(ctx->mu);
    return ctx->sticky;
}

const char *pf_last_error(pf_ctx *ctx) {
    if (!ctx) return g_tls_msg.empty() ? "no context" : g_tls_msg.c_str();
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->last_msg = ctx->sticky == PF_OK ? std::string("no error") : ctx->msg;
    ctx->sticky = PF_OK;
    ctx->msg.clear();
    return ctx->last_msg.c_str();
}

pf_status pf_pack_layout(const int64_t *byte_off_host, int64_t nseq, int64_t *word_off_host,
                         int64_t *total_words) {
    if (!byte_off_host || nseq < 0 || !total_words) return PF_EINVAL;
    int64_t acc = 0;
    for (int64_t s = 0; s < nseq; ++s) {
        const int64_t len = byte_off_host[s + 1] - byte_off_host[s];
        if (len < 0) return PF_EINVAL;
        if (word_off_host) word_off_host[s] = acc;
        acc += (len + 31) / 32;
    }
    if (word_off_host) word_off_host[nseq] = acc;
    *total_words = acc;
    return PF_OK;
}

pf_status pf_pack_layout_grouped(const int64_t *byte_off_host, const int16_t *E_host,
                                 int64_t nseq, int64_t *word_start_host, int64_t *total_words) {
    if (!byte_off_host || nseq < 0 || !total_words) return PF_EINVAL;
    // classes (E, W) with W = ceil(len/32) capped at kWCap: a counting sort
    constexpr int kWCap = 64;
    constexpr int kW = kWCap + 1;
    std::vector<int64_t> start((size_t)(PF_MAX_E + 1) * kW, 0);
    auto cls = [&](int64_t s, int64_t W) {
        const int e = E_host ? E_host[s] : 0;
        return (size_t)e * kW + (size_t)std::min<int64_t>(W, kWCap);
    };
    for (int64_t s = 0; s < nseq; ++s) {
        const int64_t len = byte_off_host[s + 1] - byte_off_host[s];
        if (len < 0) return PF_EINVAL;
        if (E_host && (E_host[s] < 0 || E_host[s] > PF_MAX_E)) return PF_EINVAL;
        start[cls(s, (len + 31) / 32)] += (len + 31) / 32;
    }
    int64_t acc = 0;
    for (auto &x : start) {
        const int64_t t = x;
        x = acc;
        acc += t;
    }
    if (word_start_host)
        for (int64_t s = 0; s < nseq; ++s) {
            const int64_t W = (byte_off_host[s + 1] - byte_off_host[s] + 31) / 32;
            int64_t &c = start[cls(s, W)];
            word_start_host[s] = c;
            c += W;
        }
    *total_words = acc;
    return PF_OK;
}

pf_status pf_pack_starts(pf_ctx *ctx, const uint8_t *ascii, const int64_t *byte_off,
                         const int64_t *word_start, int64_t nseq, uint32_t *lo, uint32_t *hi,
                         uint32_t *nmask) {
    if (!ctx) return PF_EINVAL;
    if (nseq < 0) return ctx->fail(PF_EINVAL, "nseq < 0");
    if (nseq == 0) return PF_OK;
    if (!ascii || !byte_off || !word_start || !lo || !hi || !nmask)
        return ctx->fail(PF_EINVAL, "null pointer argument");
    cudaSetDevice(ctx->device);
    return ctx->cuda(launch_pack_starts(ascii, byte_off, word_start, nseq, lo, hi, nmask,
                                        ctx->d_err, ctx->stream),
                     "pack launch");
}

pf_status pf_pack(pf_ctx *ctx, const uint8_t *ascii, const int64_t *byte_off,
                  const int64_t *word_off, int64_t nseq, uint32_t *lo, uint32_t *hi,
                  uint32_t *nmask) {
    if (!ctx) return PF_EINVAL;
    if (nseq < 0) return ctx->fail(PF_EINVAL, "nseq < 0");
    if (nseq == 0) return PF_OK;
    if (!ascii || !byte_off || !word_off || !lo || !hi || !nmask)
        return ctx->fail(PF_EINVAL, "null pointer argument");
    cudaSetDevice(ctx->device);
    return ctx->cuda(launch_pack_ragged(ascii, byte_off, word_off, nseq, lo, hi, nmask,
                                        ctx->d_err, ctx->stream),
                     "pack launch");
}

pf_status pf_pack_fixed(pf_ctx *ctx, const uint8_t *ascii, int64_t nseq, int len, uint32_t *lo,
                        uint32_t *hi, uint32_t *nmask) {
    if (!ctx) return PF_EINVAL;
    if (nseq < 0 || len < 0) return ctx->fail(PF_EINVAL, "nseq or len < 0");
    if (nseq == 0 || len == 0) return PF_OK;
    if (!ascii || !lo || !hi || !nmask) return ctx->fail(PF_EINVAL, "null pointer argument");
    cudaSetDevice(ctx->device);
    return ctx->cuda(launch_pack_fixed(ascii, nseq, len, lo, hi, nmask, ctx->d_err, ctx->sms,
                                       ctx->stream),
                     "pack launch");
}

// The plain kernel serving E_max: the first with DPT - 1 >= E_max.
static int plain_index(int E_max) {
    int pi = 0;
    while (pi < kNumPlain && kPlainDpt[pi] - 1 < E_max) ++pi;
    return pi;
}

pf_status pf_ctx::run_filter(unsigned dec, const FilterArgs &a, const Scratch &s) {
    // small batches: fixed costs of binning and per-bin launches dominate;
    // otherwise the plain kernel where pf_tune found it fastest for every
    // threshold the batch can hold
    binned = false;
    bool plain = a.n < small_batch;
    if (!plain) {
        plain = true;
        for (int e = a.E ? 0 : a.E_max; e <= a.E_max && plain; ++e) plain = tune_plain[dec][e];
    }
    if (plain) {
        // one threshold for the whole batch: the plain kernel with it fixed
        // at compile time (every shift and liveness test a constant)
        if (!a.E && a.E_max <= kPlainExactMaxE)
            return cuda(launch_filter_plain_exact((int)dec, a.E_max, a, stream), "filter launch");
        return cuda(launch_filter_plain((int)dec, plain_index(a.E_max), a, stream),
                    "filter launch");
    }
    return run_batched(dec, a, s);
}

pf_status pf_filter_plain(pf_ctx *ctx, unsigned deciders, const pf_pairs *pairs,
                          const int32_t *lens, const int16_t *E, int E_max, uint8_t *accept,
                          int16_t *count, int64_t n) {
    pf_status st = check_filter_args(ctx, deciders, pairs, lens, E_max, accept, count, n);
    if (st != PF_OK || n == 0) return st;
    cudaSetDevice(ctx->device);
    const FilterArgs a = make_filter_args(ctx, pairs, lens, E, E_max, accept, count, n);
    return ctx->cuda(launch_filter_plain((int)deciders, plain_index(E_max), a, ctx->stream),
                     "filter launch");
}

pf_status pf_filter_plain_exact(pf_ctx *ctx, unsigned deciders, const pf_pairs *pairs,
                                const int32_t *lens, int E, uint8_t *accept, int16_t *count,
                                int64_t n) {
    pf_status st = check_filter_args(ctx, deciders, pairs, lens, E, accept, count, n);
    if (st != PF_OK || n == 0) return st;
    if (E > kPlainExactMaxE)
        return ctx->fail(PF_EINVAL, "pf_filter_plain_exact: E = %d above %d", E, kPlainExactMaxE);
    cudaSetDevice(ctx->device);
    const FilterArgs a = make_filter_args(ctx, pairs, lens, nullptr, E, accept, count, n);
    return ctx->cuda(launch_filter_plain_exact((int)deciders, E, a, ctx->stream), "filter launch");
}

pf_status pf_filter(pf_ctx *ctx, unsigned deciders, const pf_pairs *pairs, const int32_t *lens,
                    const int16_t *E, int E_max, uint8_t *accept, int16_t *count, int64_t n) {
    pf_status st = check_filter_args(ctx, deciders, pairs, lens, E_max, accept, count, n);
    if (st != PF_OK || n == 0) return st;
    cudaSetDevice(ctx->device);
    Scratch s;
    st = ctx->scratch_layout(n, &s);
    if (st != PF_OK) return st;
    const FilterArgs a = make_filter_args(ctx, pairs, lens, E, E_max, accept, count, n);
    return ctx->run_filter(deciders, a, s);
}

pf_status pf_compact(pf_ctx *ctx, const uint8_t *flags, int64_t n, int64_t *idx,
                     int64_t *n_out) {
    if (!ctx) return PF_EINVAL;
    if (n < 0) return ctx->fail(PF_EINVAL, "n < 0");
    if (!n_out || (n > 0 && (!flags || !idx))) return ctx->fail(PF_EINVAL, "null pointer argument");
    cudaSetDevice(ctx->device);
    Scratch s;
    pf_status st = ctx->scratch_layout(n, &s);
    if (st != PF_OK) return st;
    return ctx->cuda(launch_compact(flags, n, idx, n_out, s.tiles, ctx->stream), "compact launch");
}

pf_status pf_verify(pf_ctx *ctx, const pf_pairs *pairs, const int32_t *lens, const int16_t *E,
                    int E_max, const int64_t *idx, const int64_t *n_idx, int64_t n,
                    int32_t *dist) {
    if (!ctx) return PF_EINVAL;
    if (n < 0) return ctx->fail(PF_EINVAL, "n < 0");
    if (E_max < 0 || E_max > PF_MAX_E)
        return ctx->fail(PF_EINVAL, "E_max = %d outside [0, %d]", E_max, PF_MAX_E);
    if (n == 0) return PF_OK;
    if (!pairs || !seqs_ok(pairs->read) || !seqs_ok(pairs->ref) || !lens || !dist ||
        (idx && !n_idx))
        return ctx->fail(PF_EINVAL, "null pointer argument");
    cudaSetDevice(ctx->device);
    return ctx->cuda(launch_verify(to_view(pairs), lens, E, E_max, idx, n_idx, n, dist,
                                   ctx->d_err, ctx->sms, ctx->stream),
                     "verify launch");
}

pf_status pf_filter_verify(pf_ctx *ctx, unsigned deciders, const pf_pairs *pairs,
                           const int32_t *lens, const int16_t *E, int E_max, uint8_t *accept,
                           int16_t *count, int32_t *dist, int64_t n) {
    pf_status st = check_filter_args(ctx, deciders, pairs, lens, E_max, accept, count, n);
    if (st != PF_OK) return st;
    ctx->verified_state = 0;
    if (n == 0) {
        ctx->verified_state = 2;
        return PF_OK;
    }
    if (!dist) return ctx->fail(PF_EINVAL, "null pointer argument");
    cudaSetDevice(ctx->device);
    Scratch s;
    st = ctx->scratch_layout(n, &s);
    if (st != PF_OK) return st;
    FilterArgs a = make_filter_args(ctx, pairs, lens, E, E_max, accept, count, n);
    a.dist = dist;  // the filter writes E + 1 for the pairs it rejects
    // with SneakySnake selected the filter also resolves the pairs whose
    // obstacle count equals their Hamming distance
    if (ctx->resolve_bounds && (deciders & 1u)) a.need = s.need;
    st = ctx->run_filter(deciders, a, s);
    if (st != PF_OK) return st;
    // the first selected decider's accept flags (less the resolved pairs)
    // choose the pairs to verify
    // (in the scheduler's grouping, when it grouped them)
    st = ctx->cuda(launch_compact(a.need ? a.need : accept, n, s.idx, s.n_idx, s.tiles,
                                  ctx->stream, ctx->binned ? s.order : nullptr, s.ident),
                   "compact launch");
    if (st != PF_OK) return st;
    st = ctx->cuda(launch_verify(to_view(pairs), lens, E, E_max, s.idx, s.n_idx, n, dist,
                                 ctx->d_err, ctx->sms, ctx->stream, s.work + kNumBatchCfgs,
                                 ctx->binned),
                   "verify launch");
    ctx->verified_state = (st == PF_OK) ? 1 : 0;
    return st;
}

pf_status pf_last_verified_count(pf_ctx *ctx, int64_t *n_verified) {
    if (!ctx) return PF_EINVAL;
    if (!n_verified) return ctx->fail(PF_EINVAL, "null pointer argument");
    if (ctx->verified_state == 2) {
        *n_verified = 0;
        return PF_OK;
    }
    if (ctx->verified_state != 1 || !ctx->scratch)
        return ctx->fail(PF_EINVAL, "no pf_filter_verify result on this context");
    cudaSetDevice(ctx->device);
    pf_status st = ctx->cuda(cudaMemcpyAsync(n_verified, ctx->scratch, sizeof(int64_t),
                                             cudaMemcpyDeviceToHost, ctx->stream),
                             "count copy");
    if (st == PF_OK) st = ctx->cuda(cudaStreamSynchronize(ctx->stream), "stream sync");
    return st;
}

pf_status pf_kernel_configs(int *tpp, int *dpt, int *ecap, int *exact_e, int *words, int cap,
                            int *count) {
    if (!count || cap < 0) return PF_EINVAL;
    for (int c = 0; c < kNumBatchCfgs && c < cap; ++c) {
        if (tpp) tpp[c] = kBatchCfgs[c].tpp;
        if (dpt) dpt[c] = kBatchCfgs[c].dpt;
        if (ecap) ecap[c] = kBatchCfgs[c].ecap;
        if (exact_e) exact_e[c] = kBatchCfgs[c].xe;
        if (words) words[c] = kBatchCfgs[c].words;
    }
    *count = kNumBatchCfgs;
    return PF_OK;
}

pf_status pf_tune_batch(pf_ctx *ctx, unsigned deciders, const pf_pairs *pairs,
                        const int32_t *lens, const int16_t *E, int E_max, int64_t n,
                        int64_t sample, int reps) {
    if (!ctx) return PF_EINVAL;
    if (n <= 0 || reps <= 0 || sample < 0 || !E)
        return ctx->fail(PF_EINVAL, "pf_tune_batch: bad n/reps/sample or no per-pair E");
    pf_status st = check_filter_args(ctx, deciders, pairs, lens, E_max,
                                     reinterpret_cast<uint8_t *>(1),
                                     reinterpret_cast<int16_t *>(2), n);
    if (st != PF_OK) return st;
    if (sample == 0) sample = int64_t(1) << 20;
    cudaSetDevice(ctx->device);
    Scratch s;
    st = ctx->scratch_layout(n, &s);
    if (st != PF_OK) return st;
    // group the pairs by threshold: bin e holds the pairs with E = e
    BinTable t;
    for (int e = 0; e <= PF_MAX_E; ++e) t.cfg_of_E[e] = e;
    bin_init_kernel<<<1, 32, 0, ctx->stream>>>(s.bin_start, s.work, s.hist, kNumBatchCfgs, -1, n);
    const int64_t hh = std::max<int64_t>(
        1, std::min<int64_t>((n + 256 * kHistPer - 1) / (256 * kHistPer), (int64_t)ctx->sms * 8));
    bin_hist_kernel<<<(unsigned)hh, 256, 0, ctx->stream>>>(E, lens, n, E_max, t, s.hist);
    bin_scan_kernel<<<1, 32, 0, ctx->stream>>>(s.hist, s.bin_start, s.cursor, s.ident);
    bin_scatter_kernel<<<(unsigned)hh, 256, 0, ctx->stream>>>(E, lens, n, E_max, t, s.cursor,
                                                               s.order, s.ident);
    int64_t starts[PF_MAX_E + 2];
    std::vector<unsigned long long> keys(kNumBinKeys);
    int ident = 0;
    st = ctx->cuda(cudaMemcpyAsync(starts, s.bin_start, sizeof(starts), cudaMemcpyDeviceToHost,
                                   ctx->stream),
                   "pf_tune_batch bins");
    if (st == PF_OK)
        st = ctx->cuda(cudaMemcpyAsync(keys.data(), s.hist, kNumBinKeys * sizeof(keys[0]),
                                       cudaMemcpyDeviceToHost, ctx->stream),
                       "pf_tune_batch bins");
    if (st == PF_OK)
        st = ctx->cuda(cudaMemcpyAsync(&ident, s.ident, sizeof(int), cudaMemcpyDeviceToHost,
                                       ctx->stream),
                       "pf_tune_batch bins");
    if (st == PF_OK) st = ctx->cuda(cudaStreamSynchronize(ctx->stream), "pf_tune_batch sync");
    if (st != PF_OK) return st;
    const int slots = (deciders == 3u) ? 2 : 1;
    uint8_t *acc = nullptr;
    int16_t *cnt = nullptr;
    int64_t *range = nullptr;  // [2] positions timed, then the work counter
    int64_t *sample_order = nullptr;
    if (cudaMalloc(&acc, (size_t)slots * n) != cudaSuccess ||
        cudaMalloc(&cnt, (size_t)slots * n * sizeof(int16_t)) != cudaSuccess ||
        cudaMalloc(&range, 4 * sizeof(int64_t)) != cudaSuccess ||
        cudaMalloc(&sample_order, (size_t)std::min<int64_t>(sample, n) * sizeof(int64_t)) !=
            cudaSuccess) {
        cudaGetLastError();
        if (acc) cudaFree(acc);
        if (cnt) cudaFree(cnt);
        if (range) cudaFree(range);
        return ctx->fail(PF_ENOMEM, "pf_tune_batch: buffers");
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    static const int chunks[] = {64, 256, 1024};
    for (int e = 0; e <= E_max && st == PF_OK; ++e) {
        const int64_t bin = starts[e + 1] - starts[e];
        const int64_t m = std::min(bin, sample);
        if (m < 1024) continue;  // too few pairs at this threshold to time
        // The sample: the same share of each length class of the threshold,
        // each share a contiguous run of the class (the pairs a launch takes
        // together), so that the configurations are timed on the batch's
        // mix of lengths.
        int64_t r[2] = {0, m};
        const int64_t *ord = s.order;
        if (ident) {  // one threshold: pair order
            r[0] = starts[e];
            r[1] = starts[e] + m;
        } else {
            int64_t at = 0, k0 = starts[e];
            for (int j = 0; j < kLenClasses && st == PF_OK; ++j) {
                const int64_t cls = (int64_t)keys[e * kLenClasses + j];
                int64_t take = (j == kLenClasses - 1) ? m - at : (cls * m) / bin;
                take = std::min(take, cls);
                if (take > 0)
                    st = ctx->cuda(cudaMemcpyAsync(sample_order + at, s.order + k0,
                                                   take * sizeof(int64_t),
                                                   cudaMemcpyDeviceToDevice, ctx->stream),
                                   "pf_tune_batch sample");
                at += take;
                k0 += cls;
            }
            r[1] = at;
            ord = sample_order;
        }
        if (st != PF_OK) break;
        cudaMemcpyAsync(range, r, sizeof(r), cudaMemcpyHostToDevice, ctx->stream);
        cudaStreamSynchronize(ctx->stream);
        BatchArgs b;
        b.f = make_filter_args(ctx, pairs, lens, E, E_max, acc, cnt, n);
        b.order = ident ? nullptr : ord;
        b.bin_start = range;
        b.bin_cfg = nullptr;
        b.nbins = 1;
        b.work = reinterpret_cast<unsigned long long *>(range + 2);
        b.chunk_start = nullptr;
        b.ident = nullptr;
        int bc = ctx->tune_cfg[deciders][e], bk = ctx->tune_chunk[deciders][e];
        float bms = 1e30f;
        for (int c = 0; st == PF_OK && c < kNumBatchCfgs; ++c) {
            if (!cfg_serves(kBatchCfgs[c], e)) continue;
            for (int k : chunks) {
                b.chunk = k;
                const int wpb = cfg_threads(kBatchCfgs[c], (int)deciders) / 32;
                const int step = cfg_step(kBatchCfgs[c], (int)deciders);
                const int64_t steps = (r[1] - r[0] + step - 1) / step;
                const int grid = (int)std::min<int64_t>(ctx->grid_for((int)deciders, c),
                                                        std::max<int64_t>(1, (steps + wpb - 1) / wpb));
                float best = 1e30f;
                for (int rep = 0; rep <= reps && st == PF_OK; ++rep) {  // the first run warms up
                    cudaMemsetAsync(b.work, 0, sizeof(unsigned long long), ctx->stream);
                    cudaEventRecord(e0, ctx->stream);
                    st = ctx->cuda(launch_filter_batched((int)deciders, c, grid, b, 0, ctx->stream),
                                   "pf_tune_batch launch");
                    cudaEventRecord(e1, ctx->stream);
                    if (st == PF_OK) st = ctx->cuda(cudaEventSynchronize(e1), "pf_tune_batch sync");
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (rep > 0 && ms < best) best = ms;
                }
                if (best < bms) {
                    bms = best;
                    bc = c;
                    bk = k;
                }
            }
        }
        if (st == PF_OK) {
            ctx->tune_cfg[deciders][e] = bc;
            ctx->tune_chunk[deciders][e] = bk;
            ctx->tune_plain[deciders][e] = false;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(acc);
    cudaFree(cnt);
    cudaFree(range);
    cudaFree(sample_order);
    return st;
}

pf_status pf_set_small_batch(pf_ctx *ctx, int64_t pairs) {
    if (!ctx) return PF_EINVAL;
    if (pairs < 0) return ctx->fail(PF_EINVAL, "pf_set_small_batch: pairs < 0");
    ctx->small_batch = pairs;
    return PF_OK;
}

pf_status pf_tune_set(pf_ctx *ctx, unsigned deciders, int E, int cfg, int chunk) {
    if (!ctx) return PF_EINVAL;
    if ((deciders & 3u) == 0 || (deciders & ~3u) || E < 0 || E > PF_MAX_E || cfg < -1 ||
        cfg >= kNumBatchCfgs || (cfg >= 0 && !cfg_serves(kBatchCfgs[cfg], E)) || chunk < 1 ||
        chunk > 65536)
        return ctx->fail(PF_EINVAL, "pf_tune_set: bad deciders/E/cfg/chunk");
    ctx->tune_plain[deciders][E] = cfg == -1;  // -1: the plain kernel
    if (cfg >= 0) ctx->tune_cfg[deciders][E] = cfg;
    ctx->tune_chunk[deciders][E] = chunk;
    return PF_OK;
}

pf_status pf_tune_get(pf_ctx *ctx, unsigned deciders, int E, int *cfg, int *chunk) {
    if (!ctx) return PF_EINVAL;
    if ((deciders & 3u) == 0 || (deciders & ~3u) || E < 0 || E > PF_MAX_E)
        return ctx->fail(PF_EINVAL, "pf_tune_get: bad deciders/E");
    if (cfg) *cfg = ctx->tune_plain[deciders][E] ? -1 : ctx->tune_cfg[deciders][E];
    if (chunk) *chunk = ctx->tune_chunk[deciders][E];
    return PF_OK;
}

pf_status pf_tune(pf_ctx *ctx, unsigned deciders, const pf_pairs *pairs, const int32_t *lens,
                  int E, int64_t n, int reps, int *best_cfg, int *best_chunk, float *best_ms) {
    if (!ctx) return PF_EINVAL;
    if (n <= 0 || reps <= 0 || E < 0 || E > PF_MAX_E)
        return ctx->fail(PF_EINVAL, "pf_tune: bad n/reps/E");
    pf_status st = check_filter_args(ctx, deciders, pairs, lens, E, reinterpret_cast<uint8_t *>(1),
                                     reinterpret_cast<int16_t *>(2), n);
    if (st != PF_OK) return st;
    cudaSetDevice(ctx->device);
    const int slots = (deciders == 3u) ? 2 : 1;
    uint8_t *acc = nullptr;
    int16_t *cnt = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMalloc(&acc, (size_t)slots * n) != cudaSuccess ||
        cudaMalloc(&cnt, (size_t)slots * n * sizeof(int16_t)) != cudaSuccess) {
        cudaGetLastError();
        if (acc) cudaFree(acc);
        return ctx->fail(PF_ENOMEM, "pf_tune: output buffers");
    }
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    Scratch s;
    st = ctx->scratch_layout(n, &s);
    const int keep_cfg = ctx->tune_cfg[deciders][E], keep_chunk = ctx->tune_chunk[deciders][E];
    int bc = keep_cfg, bk = keep_chunk;
    float bms = 1e30f;
    static const int chunks[] = {64, 256, 1024};
    for (int c = 0; st == PF_OK && c < kNumBatchCfgs; ++c) {
        if (!cfg_serves(kBatchCfgs[c], E)) continue;
        for (int k : chunks) {
            ctx->tune_cfg[deciders][E] = c;
            ctx->tune_chunk[deciders][E] = k;
            const FilterArgs a = make_filter_args(ctx, pairs, lens, nullptr, E, acc, cnt, n);
            float best = 1e30f;
            for (int r = 0; r <= reps && st == PF_OK; ++r) {  // first run warms up
                cudaEventRecord(e0, ctx->stream);
                st = ctx->run_batched(deciders, a, s);
                cudaEventRecord(e1, ctx->stream);
                if (st == PF_OK) st = ctx->cuda(cudaEventSynchronize(e1), "tune sync");
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (r > 0 && ms < best) best = ms;
            }
            if (best < bms) {
                bms = best;
                bc = c;
                bk = k;
            }
        }
    }
    // the plain one-thread-per-pair kernel over the same pairs
    bool plain_best = false;
    if (st == PF_OK) {
        const FilterArgs a = make_filter_args(ctx, pairs, lens, nullptr, E, acc, cnt, n);
        float best = 1e30f;
        for (int r = 0; r <= reps && st == PF_OK; ++r) {  // first run warms up
            cudaEventRecord(e0, ctx->stream);
            st = ctx->cuda(launch_filter_plain((int)deciders, plain_index(E), a, ctx->stream),
                           "tune launch");
            cudaEventRecord(e1, ctx->stream);
            if (st == PF_OK) st = ctx->cuda(cudaEventSynchronize(e1), "tune sync");
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (r > 0 && ms < best) best = ms;
        }
        // a change from the default by a clear margin only: a tuning sample
        // weighs the scheduler's fixed cost (one more launch) more than the
        // large batches it serves, and keeps part of its input in L2
        const float margin = default_plain(E) ? 1.1f : 0.9f;
        if (st == PF_OK && best < margin * bms) {
            bms = best;
            plain_best = true;
        }
    }
    ctx->tune_cfg[deciders][E] = (st == PF_OK) ? bc : keep_cfg;
    ctx->tune_chunk[deciders][E] = (st == PF_OK) ? bk : keep_chunk;
    if (st == PF_OK) ctx->tune_plain[deciders][E] = plain_best;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(acc);
    cudaFree(cnt);
    if (st != PF_OK) return st;
    if (best_cfg) *best_cfg = plain_best ? -1 : bc;
    if (best_chunk) *best_chunk = bk;
    if (best_ms) *best_ms = bms;
    return PF_OK;
}

}  // extern "C"
