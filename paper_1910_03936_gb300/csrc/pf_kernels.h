// Host-side table of the filter kernel configurations and the launchers of
// every kernel in the library.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "pf_internal.cuh"

namespace pf {

// One batched-filter configuration: TPP lanes per pair, DPT diagonal slots
// per lane; it serves thresholds E <= ecap.  xe >= 0 marks the
// exact-threshold form (one thread per pair, serves E == xe only).  words
// > 0 marks its two-phase form: the mask words of pairs up to `words`
// 32-column words are kept in shared memory and SneakySnake runs as a
// per-lane step loop over them (longer pairs take the fused loop).
struct KernelCfg {
    int tpp, dpt, ecap, xe, words;
};

constexpr KernelCfg kBatchCfgs[] = {
    {1, 4, 3, -1},   {2, 4, 3, -1},   {4, 2, 3, -1},   {8, 1, 3, -1},
    {1, 8, 7, -1},   {2, 8, 7, -1},   {4, 4, 7, -1},   {8, 2, 7, -1},  {16, 1, 7, -1},
    {1, 16, 15, -1}, {2, 16, 15, -1}, {4, 8, 15, -1},  {8, 4, 15, -1}, {16, 2, 15, -1},
    {32, 1, 15, -1},
    {2, 32, 31, -1}, {4, 16, 31, -1}, {8, 8, 31, -1},  {16, 4, 31, -1}, {32, 2, 31, -1},
    {1, 1, 0, 0},    {1, 2, 1, 1},    {1, 3, 2, 2},    {1, 4, 3, 3},   {1, 5, 4, 4},
    {1, 6, 5, 5},    {1, 7, 6, 6},    {1, 8, 7, 7},    {1, 9, 8, 8},   {1, 10, 9, 9},
    {1, 11, 10, 10}, {1, 12, 11, 11}, {1, 13, 12, 12}, {1, 14, 13, 13}, {1, 15, 14, 14},
    {1, 16, 15, 15},
    // two-phase forms, E = 1..12: as many words as keep a 4-warp block's
    // arrays within about 56 KB (four blocks per SM)
    {1, 2, 1, 1, 8},     {1, 3, 2, 2, 8},     {1, 4, 3, 3, 8},     {1, 5, 4, 4, 8},
    {1, 6, 5, 5, 8},     {1, 7, 6, 6, 8},     {1, 8, 7, 7, 7},     {1, 9, 8, 8, 6},
    {1, 10, 9, 9, 5},    {1, 11, 10, 10, 5},  {1, 12, 11, 11, 4},  {1, 13, 12, 12, 4},
    // and with 5-word arrays (pairs up to 160 bases) for E = 1..7: smaller
    // blocks, more of them per SM,
    {1, 2, 1, 1, 5},     {1, 3, 2, 2, 5},     {1, 4, 3, 3, 5},     {1, 5, 4, 4, 5},
    {1, 6, 5, 5, 5},     {1, 7, 6, 6, 5},     {1, 8, 7, 7, 5},
    // and for E = 11..15 (up to 79 KB per block, two or three per SM)
    {1, 12, 11, 11, 5},  {1, 13, 12, 12, 5},  {1, 14, 13, 13, 5},  {1, 15, 14, 14, 5},
    {1, 16, 15, 15, 5},
    // two-phase forms with a lane group per pair (pairs up to 256 bases): for
    // thresholds whose masks do not fit one thread
    {4, 4, 7, -1, 8},    {4, 8, 15, -1, 8},   {8, 4, 15, -1, 8},   {4, 16, 31, -1, 8},
    {8, 8, 31, -1, 8},   {16, 4, 31, -1, 8},
    // fewer slots per lane, fewer dead ones: 56 slots for E <= 27, 48 for
    // E <= 23, 40 for E <= 19
    {8, 7, 27, -1, 8},   {8, 6, 23, -1, 8},   {8, 5, 19, -1, 8},
    // one thread per pair with 8-word arrays (pairs up to 256 bases) for
    // E = 8..13: 68 KB (three blocks per SM) to 108 KB (two) per block
    {1, 9, 8, 8, 8},     {1, 10, 9, 9, 8},    {1, 11, 10, 10, 8},  {1, 12, 11, 11, 8},
    {1, 13, 12, 12, 8},  {1, 14, 13, 13, 8},
    // lane groups of two and four (fewer shuffles per step, the walk's
    // control repeated by fewer lanes): the fastest at E = 16..31
    {2, 17, 16, -1, 8},  {4, 11, 21, -1, 8},  {4, 13, 25, -1, 8},  {2, 26, 25, -1, 8},
};

// The two-phase form applies where SneakySnake runs (deciders 1 and 3);
// GateKeeper alone runs a two-phase configuration as the fused loop.
constexpr bool cfg_split(const KernelCfg &c, int dec) { return c.words > 0 && dec != 2; }
// Diagonal slots one lane stores per word in the two-phase form.
constexpr int cfg_slots(const KernelCfg &c) { return c.xe >= 0 ? 2 * c.xe + 1 : c.dpt; }
// Block size and dynamic shared memory of a configuration's kernel.
constexpr int cfg_threads(const KernelCfg &c, int dec) {
    return cfg_split(c, dec) ? kSplitWarps * 32 : 256;
}
constexpr size_t cfg_smem(const KernelCfg &c, int dec) {
    return cfg_split(c, dec)
               ? (size_t)kSplitWarps * c.words * cfg_slots(c) * 32 * sizeof(uint32_t)
               : 0;
}

// Pairs one warp of a configuration's kernel takes at once: one per lane in
// the two-phase form, one per lane group in the fused loop.
constexpr int cfg_step(const KernelCfg &c, int dec) { return 32 / c.tpp; }

// a configuration serves threshold E
constexpr bool cfg_serves(const KernelCfg &c, int E) {
    return c.xe >= 0 ? c.xe == E : c.ecap >= E;
}
constexpr int kNumBatchCfgs = sizeof(kBatchCfgs) / sizeof(kBatchCfgs[0]);
// Inside a configuration's bin the scheduler groups pairs by length class
// (ceil(len/32) words, the last class holding 8 words and more): keys of
// the binning counting sort.
constexpr int kLenClasses = 9;
constexpr int kNumBinKeys = kNumBatchCfgs * kLenClasses;
// Work counters in the scheduler's scratch: one per configuration's bin,
// then the verifier's.
constexpr int kWorkCounters = kNumBatchCfgs + 1;
constexpr int kFirstExactCfg = 20;  // kBatchCfgs[20 + E] serves exactly E

// Plain kernel (one thread per pair): DPT = kPlainDpt[i] serves E <= DPT - 1.
constexpr int kPlainDpt[] = {1, 2, 4, 8, 16, 32};
constexpr int kNumPlain = sizeof(kPlainDpt) / sizeof(kPlainDpt[0]);

// The plain kernel with the threshold fixed at compile time: E = 0..15.
constexpr int kPlainExactMaxE = 15;

// dec in {1, 2, 3}
cudaError_t launch_filter_plain(int dec, int plain_idx, const FilterArgs &a, cudaStream_t st);
cudaError_t launch_filter_plain_exact(int dec, int E, const FilterArgs &a, cudaStream_t st);
cudaError_t launch_filter_batched(int dec, int cfg, int grid, const BatchArgs &b, int bin,
                                  cudaStream_t st);
const void *filter_batched_fn(int dec, int cfg);

cudaError_t launch_pack_ragged(const uint8_t *ascii, const int64_t *byte_off,
                               const int64_t *word_off, int64_t nseq, uint32_t *lo,
                               uint32_t *hi, uint32_t *nm, unsigned *err, cudaStream_t st,
                               const int32_t *seg_of = nullptr, unsigned *seg_err = nullptr);
cudaError_t launch_pack_starts(const uint8_t *ascii, const int64_t *byte_off,
                               const int64_t *word_start, int64_t nseq, uint32_t *lo,
                               uint32_t *hi, uint32_t *nm, unsigned *err, cudaStream_t st);
cudaError_t launch_pack_fixed(const uint8_t *ascii, int64_t nseq, int len, uint32_t *lo,
                              uint32_t *hi, uint32_t *nm, unsigned *err, int sms,
                              cudaStream_t st);
int64_t compact_tiles(int64_t n);
// order (may be null; used unless *ident): position q stands for pair
// order[q], and the indices come out in that order.
cudaError_t launch_compact(const uint8_t *flags, int64_t n, int64_t *idx, int64_t *n_out,
                           int64_t *tile_scratch, cudaStream_t st,
                           const int64_t *order = nullptr, const int *ident = nullptr);
cudaError_t launch_verify(const PairsView &pv, const int32_t *lens, const int16_t *E, int E_max,
                          const int64_t *idx, const int64_t *n_idx, int64_t n, int32_t *dist,
                          unsigned *err, int sms, cudaStream_t st,
                          unsigned long long *work = nullptr, bool grouped = false);

}  // namespace pf
