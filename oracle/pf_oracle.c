/*
 * CPU oracle for the pre-alignment filtering hot path (Alser, "Accelerating
 * the Understanding of Life's Code through Better Algorithms and Hardware
 * Design", 2018/2019).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check of the
 * package entry module and the CPU-baseline leg of the benchmark may load
 * this library.  The product path never calls it and shares no code,
 * header, table or helper with it.
 *
 * Everything here is deliberately plain: sequences stay as ASCII bytes,
 * the neighbourhood map is a byte matrix, every loop follows the text of
 * the thesis step by step.  No bit tricks, no blocking, no early exits
 * beyond the ones the method itself defines.
 *
 * Readings of the thesis that this file fixes (the text is silent or
 * ambiguous on each):
 *   R1  accept <=> count <= E for both deciders (correct mapping = at most
 *       E edits, Ch. 3 "Pre-alignment Filter Performance Metrics").
 *   R2  out-of-range ("vacant") cells of the neighbourhood map are 1
 *       (mismatch), as Shouji fills the bits vacated by shifting with ones
 *       (Ch. 6, Discussion); used for both deciders.
 *   R3  the advancing grid column is the REFERENCE position i; the
 *       diagonal offset d indexes the read: cell (i, d) compares F[i]
 *       with R[i+d], |d| <= E.  Eq. 8.2 indexes the column by the
 *       reference A[i] with j in [i-E, i+E] on the read, the masks of
 *       GateKeeper and Shouji shift the read against the reference
 *       (§5.2.2, Ch. 6 Discussion), and only this orientation walks the
 *       three pipes GGTG, AGAG, T named for the example of Fig. 8.1/8.2.
 *   R4  'N' (either case) never matches anything, not even another N.
 *   R5  the SneakySnake count saturates at E+1: the walk stops once its
 *       tries are spent (§8.4.2).
 *   R6  after a pipe ends, the obstacle is counted and the snake moves one
 *       column ahead, also when the longest pipe has length 0 (§8.2,
 *       §8.4.2).
 *   R7  GateKeeper amends every bit 1..m-2 of the ORIGINAL mask in
 *       parallel (no cascading), neighbours beyond the ends read as 0,
 *       bits 0 and m-1 are copied (§5.2.2).
 *   R8  GateKeeper's count is the Hamming popcount when the fast path of
 *       §5.2.1 accepts, otherwise the popcount of the AND of the amended
 *       masks; both saturate at E+1 like R5.
 *   R9  base codes A=00, C=01, G=10, T=11 (only A=00 and T=11 are printed
 *       in §5.2.3); N packs as code 00 with its N bit set; bases past the
 *       end of a sequence in its last 32-bit word pack as N.
 *   R15 partitioned SneakySnake (§8.5): sub-matrix s covers columns
 *       [s*t, min((s+1)*t, m)); its pipes end at its own last column (a
 *       pipe that reaches it leaves the sub-matrix, no obstacle), so the
 *       last, narrower sub-matrix holds only real columns; it contributes
 *       min(y, t_s - sum of the y pipe depths), which equals the obstacles
 *       its y replications pass.  The total saturates at E+1 like R5.
 *   R16 Shouji (Ch. 6): window c covers columns c..c+3 for every c in
 *       [0, m); window cells past column m-1 read as 1 and the bit-vector
 *       has no bits there; the bit-vector starts all 1; a diagonal's 4-bit
 *       vector wins with more zeros, on a tie the first one (in row order
 *       d = -E .. E) whose first bit is 0, else the first one; it replaces
 *       the bit-vector's bits c..c+3 only with strictly more zeros than
 *       they hold.  The count saturates at E+1 like R5.  Parity partly
 *       unpinned: the 4-column window, the example of Fig. 6.1 and zero
 *       false rejects are pinned, but the tie order, the strict
 *       replacement and the value of window cells past the end are
 *       readings that change the count of some pairs and that no printed
 *       example fixes.
 *   R17 SHD-style GateKeeper (Ch. 3): "vacant zero" fills the out-of-range
 *       cells of the masks with 0 (SHD's arithmetic shifts) instead of R2's
 *       1; the "streak" counter charges each maximal run of L ones in the
 *       final bit-vector ceil(L/3) edits, the counting that charges three
 *       consecutive ones as a single edit (Ch. 3, Conservative Counting).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

/* ------------------------------------------------------------------ */
/* Bases                                                               */
/* ------------------------------------------------------------------ */

/* Code of one ASCII base: 0..3 for A,C,G,T (either case), 4 for N,
 * -1 for any other byte.  Encoding per R9 (§5.2.3). */
int or_base_code(uint8_t b)
{
    switch (b) {
    case 'A': case 'a': return 0;
    case 'C': case 'c': return 1;
    case 'G': case 'g': return 2;
    case 'T': case 't': return 3;
    case 'N': case 'n': return 4;
    default: return -1;
    }
}

/* Pairwise match of two bases (R4): equal codes and neither is N. */
static int or_match(uint8_t x, uint8_t y)
{
    int cx = or_base_code(x), cy = or_base_code(y);
    if (cx < 0 || cy < 0 || cx == 4 || cy == 4) return 0;
    return cx == cy;
}

/* ------------------------------------------------------------------ */
/* Packing (§5.2.3, R9)                                                */
/* ------------------------------------------------------------------ */

/* Pack one ASCII sequence of length len into three bit-planes of
 * ceil(len/32) 32-bit words each: base i sets bit (i % 32) of word i/32 in
 * `lo` (low code bit), `hi` (high code bit) and `nmask` (1 for N).  Bits
 * past the end of the sequence in the last word are N.  Returns the number
 * of bytes that were neither ACGT nor N (they pack as N). */
int or_pack(const uint8_t *s, int len, uint32_t *lo, uint32_t *hi, uint32_t *nmask)
{
    int words = (len + 31) / 32, bad = 0;
    for (int w = 0; w < words; ++w) { lo[w] = 0; hi[w] = 0; nmask[w] = 0; }
    for (int i = 0; i < words * 32; ++i) {
        int code;
        if (i < len) {
            code = or_base_code(s[i]);
            if (code < 0) { bad++; code = 4; }
        } else {
            code = 4;
        }
        uint32_t bit = 1u << (i % 32);
        if (code == 4) {
            nmask[i / 32] |= bit;
        } else {
            if (code & 1) lo[i / 32] |= bit;
            if (code & 2) hi[i / 32] |= bit;
        }
    }
    return bad;
}

/* ------------------------------------------------------------------ */
/* Neighbourhood map (Eq. 6.1, R2, R3)                                 */
/* ------------------------------------------------------------------ */

/* Fill map[(d+E)*m + i] for d in [-E, E], i in [0, m): 0 where the
 * reference base F[i] matches the read base R[i+d], 1 where it does not or
 * where i+d falls outside the read (R3). */
void or_neighborhood_map(const uint8_t *R, const uint8_t *F, int m, int E, uint8_t *map)
{
    for (int d = -E; d <= E; ++d) {
        for (int i = 0; i < m; ++i) {
            int j = i + d;
            uint8_t v;
            if (j < 0 || j >= m) v = 1;
            else v = or_match(F[i], R[j]) ? 0 : 1;
            map[(size_t)(d + E) * m + i] = v;
        }
    }
}

/* ------------------------------------------------------------------ */
/* SneakySnake, unweighted neighbourhood maze (Ch. 8)                  */
/* ------------------------------------------------------------------ */

/* Depth of the pipe that starts at column c on diagonal d: the number of
 * consecutive available cells (§8.4.1, Eq. 8.2) before the first blocked
 * cell or the end of the grid. */
static int or_pipe_depth(const uint8_t *map, int m, int E, int d, int c)
{
    int r = 0;
    while (c + r < m && map[(size_t)(d + E) * m + c + r] == 0) r++;
    return r;
}

/* Greedy walk of §8.4.2 with a limit on the obstacles it may pass:
 * from the current checkpoint, search every diagonal for the deepest pipe
 * (the depth-first probe of the text), travel it, and if the grid is not
 * yet left, count the obstacle at its end and step one column past it.
 * Stops when the snake exits the grid or when more than `limit` obstacles
 * were counted; returns the obstacles counted. */
static int or_snake_walk(const uint8_t *map, int m, int E, int limit)
{
    int c = 0, k = 0;
    for (;;) {
        int best = 0;
        for (int d = -E; d <= E; ++d) {
            int r = or_pipe_depth(map, m, E, d, c);
            if (r > best) best = r;
        }
        c += best;
        if (c >= m) return k;
        k += 1;          /* the obstacle that ends the chosen pipe (R6) */
        c += 1;          /* travel across it, one column ahead */
        if (c >= m) return k;
        if (k > limit) return k;
    }
}

/* SneakySnake count with saturation R5: min(obstacles, E+1). */
int or_sneakysnake(const uint8_t *R, const uint8_t *F, int m, int E)
{
    if (m <= 0) return 0;
    uint8_t *map = (uint8_t *)malloc((size_t)(2 * E + 1) * m);
    or_neighborhood_map(R, F, m, E, map);
    int k = or_snake_walk(map, m, E, E);
    free(map);
    return k > E + 1 ? E + 1 : k;
}

/* Same walk with no limit on obstacles (used only by tests: the
 * unsaturated count is non-increasing in E). */
int or_sneakysnake_full(const uint8_t *R, const uint8_t *F, int m, int E)
{
    if (m <= 0) return 0;
    uint8_t *map = (uint8_t *)malloc((size_t)(2 * E + 1) * m);
    or_neighborhood_map(R, F, m, E, map);
    int k = or_snake_walk(map, m, E, 1 << 30);
    free(map);
    return k;
}

/* The pipes the walk travels (no obstacle limit): start column and
 * length of each, up to max_pipes; returns the number of pipes written.
 * Used by tests to pin the orientation reading R3 against Fig. 8.1/8.2. */
int or_sneakysnake_trace(const uint8_t *R, const uint8_t *F, int m, int E,
                         int *starts, int *lengths, int max_pipes)
{
    if (m <= 0) return 0;
    uint8_t *map = (uint8_t *)malloc((size_t)(2 * E + 1) * m);
    or_neighborhood_map(R, F, m, E, map);
    int c = 0, np = 0;
    while (c < m) {
        int best = 0;
        for (int d = -E; d <= E; ++d) {
            int r = or_pipe_depth(map, m, E, d, c);
            if (r > best) best = r;
        }
        if (best > 0 && np < max_pipes) { starts[np] = c; lengths[np] = best; np++; }
        c += best + 1;
    }
    free(map);
    return np;
}

/* Second, independent formulation of the Sneaky Snake Problem (§8.2):
 * the minimum number of obstacles over all snake paths, by dynamic
 * programming over checkpoints.  best[c] = fewest obstacles with which the
 * snake can stand at column c free to pick any pipe.  From there it may
 * ride any pipe for up to its depth and pay one obstacle at any column it
 * reaches, landing one column further.  Returns min(result, E+1). */
int or_sneakysnake_dp(const uint8_t *R, const uint8_t *F, int m, int E)
{
    if (m <= 0) return 0;
    uint8_t *map = (uint8_t *)malloc((size_t)(2 * E + 1) * m);
    or_neighborhood_map(R, F, m, E, map);
    int inf = 1 << 30;
    int *best = (int *)malloc(sizeof(int) * (size_t)(m + 2));
    for (int c = 0; c <= m + 1; ++c) best[c] = inf;
    best[0] = 0;
    int answer = inf;
    for (int c = 0; c < m; ++c) {
        if (best[c] == inf) continue;
        int reach = 0;
        for (int d = -E; d <= E; ++d) {
            int r = or_pipe_depth(map, m, E, d, c);
            if (r > reach) reach = r;
        }
        if (c + reach >= m) {
            if (best[c] < answer) answer = best[c];
        }
        for (int stop = c; stop <= c + reach && stop < m; ++stop) {
            int land = stop + 1;
            int cost = best[c] + 1;
            if (land >= m) {
                if (cost < answer) answer = cost;
            } else if (cost < best[land]) {
                best[land] = cost;
            }
        }
    }
    free(best);
    free(map);
    return answer > E + 1 ? E + 1 : answer;
}

/* ------------------------------------------------------------------ */
/* GateKeeper (Ch. 5)                                                  */
/* ------------------------------------------------------------------ */

/* Hamming mask popcount of §5.2.1: mismatches on the main diagonal. */
int or_hamming(const uint8_t *R, const uint8_t *F, int m)
{
    int h = 0;
    for (int i = 0; i < m; ++i) h += or_match(R[i], F[i]) ? 0 : 1;
    return h;
}

/* Amending of §5.2.2 (R7): a 0 whose two left and two right neighbours
 * make it part of a "101" or "1001" pattern becomes 1.  Written as the
 * per-bit rule that one 5-input look-up table evaluates. */
void or_amend(const uint8_t *H, int m, uint8_t *A)
{
    for (int i = 0; i < m; ++i) {
        if (i == 0 || i == m - 1) { A[i] = H[i]; continue; }
        int l1 = (i - 1 >= 0) ? H[i - 1] : 0;
        int l2 = (i - 2 >= 0) ? H[i - 2] : 0;
        int r1 = (i + 1 < m) ? H[i + 1] : 0;
        int r2 = (i + 2 < m) ? H[i + 2] : 0;
        int v = H[i];
        if (!v) {
            if (l1 && r1) v = 1;          /* 1 0 1            */
            if (l1 && !r1 && r2) v = 1;   /* 1 0 0 1, first 0 */
            if (!l1 && l2 && r1) v = 1;   /* 1 0 0 1, second 0 */
        }
        A[i] = (uint8_t)v;
    }
}

/* GateKeeper count per R8: the fast Hamming check of §5.2.1, then the
 * 2E+1 masks of §5.2.2 (vacant bits 1, R2), amended, ANDed, popcounted. */
int or_gatekeeper(const uint8_t *R, const uint8_t *F, int m, int E)
{
    if (m <= 0) return 0;
    int h = or_hamming(R, F, m);
    if (h <= E) return h;
    uint8_t *map = (uint8_t *)malloc((size_t)(2 * E + 1) * m);
    uint8_t *amended = (uint8_t *)malloc((size_t)m);
    uint8_t *final_mask = (uint8_t *)malloc((size_t)m);
    or_neighborhood_map(R, F, m, E, map);
    for (int i = 0; i < m; ++i) final_mask[i] = 1;
    for (int d = -E; d <= E; ++d) {
        or_amend(map + (size_t)(d + E) * m, m, amended);
        for (int i = 0; i < m; ++i) final_mask[i] = final_mask[i] & amended[i];
    }
    int count = 0;
    for (int i = 0; i < m; ++i) count += final_mask[i];
    free(final_mask);
    free(amended);
    free(map);
    return count > E + 1 ? E + 1 : count;
}

/* ------------------------------------------------------------------ */
/* Work the method needs per pair (a measurement aid, not a result)    */
/* ------------------------------------------------------------------ */

/* How much of the map each decider needs before its answer is known, for
 * the "needed work" roofline of a word-parallel implementation that stops
 * a pair once both deciders are decided.  Changes no result.
 *   out[0]  SneakySnake: 32-column words spanned by its deepest-pipe
 *           searches, summed over the searches the walk of §8.4.2 makes
 *           with the limit of R5 (a search from column c whose deepest
 *           pipe ends at column e (its obstacle, or the last column) spans
 *           the words of columns c..e);
 *   out[1]  SneakySnake: leading columns it reads (through the last
 *           obstacle it meets, or all m);
 *   out[2]  GateKeeper: leading columns the Hamming count of §5.2.1 needs
 *           (all m when it is at most E; else through the column where it
 *           first exceeds E);
 *   out[3]  GateKeeper: leading columns the amended-mask AND of §5.2.2-
 *           §5.2.3 needs (0 when the Hamming check accepts; through the
 *           column where the AND's popcount first exceeds E, plus the two
 *           columns an amended bit looks ahead, when it rejects; else m). */
void or_work_counts(const uint8_t *R, const uint8_t *F, int m, int E, int *out)
{
    out[0] = out[1] = out[2] = out[3] = 0;
    if (m <= 0) return;
    uint8_t *map = (uint8_t *)malloc((size_t)(2 * E + 1) * m);
    or_neighborhood_map(R, F, m, E, map);
    /* the walk of or_snake_walk, counting what it reads */
    int c = 0, k = 0, words = 0, cols = 0;
    for (;;) {
        int best = 0;
        for (int d = -E; d <= E; ++d) {
            int r = or_pipe_depth(map, m, E, d, c);
            if (r > best) best = r;
        }
        int end = c + best < m ? c + best : m - 1;   /* last column this search reads */
        words += end / 32 - c / 32 + 1;
        if (end + 1 > cols) cols = end + 1;
        c += best;
        if (c >= m) break;
        k += 1;
        c += 1;
        if (c >= m) break;
        if (k > E) break;
    }
    out[0] = words;
    out[1] = cols;
    /* GateKeeper's prefix counts */
    int h = or_hamming(R, F, m);
    if (h <= E) {
        out[2] = m;
        out[3] = 0;
    } else {
        int run = 0, i = 0;
        for (; i < m; ++i) {
            run += or_match(R[i], F[i]) ? 0 : 1;
            if (run > E) break;
        }
        out[2] = i + 1;
        uint8_t *amended = (uint8_t *)malloc((size_t)m);
        uint8_t *fin = (uint8_t *)malloc((size_t)m);
        for (int x = 0; x < m; ++x) fin[x] = 1;
        for (int d = -E; d <= E; ++d) {
            or_amend(map + (size_t)(d + E) * m, m, amended);
            for (int x = 0; x < m; ++x) fin[x] = fin[x] & amended[x];
        }
        int cnt = 0, x = 0;
        for (; x < m; ++x) {
            cnt += fin[x];
            if (cnt > E) break;
        }
        out[3] = (x < m) ? (x + 3 < m ? x + 3 : m) : m;
        free(fin);
        free(amended);
    }
    free(map);
}

/* ------------------------------------------------------------------ */
/* SneakySnake on sub-matrices of t columns (§8.5, R15)                */
/* ------------------------------------------------------------------ */

/* Obstacles that y replications of the search pass in the sub-matrix
 * [b, b+ts) of the map: each replication finds the largest number of
 * leading zeros x over the 2E+1 rows from the current column (a run stops
 * at the sub-matrix's last column: reaching it leaves the sub-matrix
 * without an obstacle), then every row shifts by x+1.  Returns
 * min(y, ts - sum x). */
static int or_submatrix_obstacles(const uint8_t *map, int m, int E, int b, int ts, int y)
{
    int c = 0, sum_x = 0;
    for (int o = 0; o < y; ++o) {
        int x = 0;
        for (int d = -E; d <= E; ++d) {
            int r = 0;
            while (c + r < ts && map[(size_t)(d + E) * m + b + c + r] == 0) r++;
            if (r > x) x = r;
        }
        sum_x += x;
        c += x + 1;
        if (c > ts) c = ts;  /* past the end every row reads as leading ones */
    }
    int k = ts - sum_x;
    return k < y ? k : y;
}

/* Partitioned SneakySnake count min(sum over sub-matrices, E+1). */
int or_sneakysnake_partitioned(const uint8_t *R, const uint8_t *F, int m, int E, int t, int y)
{
    if (m <= 0) return 0;
    uint8_t *map = (uint8_t *)malloc((size_t)(2 * E + 1) * m);
    or_neighborhood_map(R, F, m, E, map);
    int total = 0;
    for (int b = 0; b < m; b += t) {
        int ts = (m - b < t) ? m - b : t;
        total += or_submatrix_obstacles(map, m, E, b, ts, y);
    }
    free(map);
    return total > E + 1 ? E + 1 : total;
}

/* ------------------------------------------------------------------ */
/* Shouji (Ch. 6, R16)                                                 */
/* ------------------------------------------------------------------ */

/* Runs Methods 1-2 of Ch. 6 and leaves the Shouji bit-vector in sbv[m];
 * returns its number of ones (unsaturated). */
int or_shouji_vector(const uint8_t *R, const uint8_t *F, int m, int E, uint8_t *sbv)
{
    if (m <= 0) return 0;
    uint8_t *map = (uint8_t *)malloc((size_t)(2 * E + 1) * m);
    or_neighborhood_map(R, F, m, E, map);
    for (int i = 0; i < m; ++i) sbv[i] = 1;
    for (int c = 0; c < m; ++c) {
        /* Step 1: the 4-bit diagonal vector of window c with the most zeros */
        int best = 0, best_z = -1, best_lead = 0;
        for (int d = -E; d <= E; ++d) {
            int z = 0;
            for (int q = 0; q < 4; ++q) {
                int col = c + q;
                int bit = (col < m) ? map[(size_t)(d + E) * m + col] : 1;
                z += bit ? 0 : 1;
            }
            int lead = map[(size_t)(d + E) * m + c] == 0;
            if (z > best_z || (z == best_z && lead && !best_lead)) {
                best = d;
                best_z = z;
                best_lead = lead;
            }
        }
        /* Step 2: keep it if it has more zeros than the bit-vector there */
        int cur_z = 0;
        for (int q = 0; q < 4 && c + q < m; ++q) cur_z += sbv[c + q] ? 0 : 1;
        if (best_z > cur_z)
            for (int q = 0; q < 4 && c + q < m; ++q)
                sbv[c + q] = map[(size_t)(best + E) * m + c + q];
    }
    free(map);
    /* Method 3: the edits are the ones of the bit-vector */
    int ones = 0;
    for (int i = 0; i < m; ++i) ones += sbv[i];
    return ones;
}

/* Shouji count min(ones of the bit-vector, E+1). */
int or_shouji(const uint8_t *R, const uint8_t *F, int m, int E)
{
    if (m <= 0) return 0;
    uint8_t *sbv = (uint8_t *)malloc((size_t)m);
    int ones = or_shouji_vector(R, F, m, E, sbv);
    free(sbv);
    return ones > E + 1 ? E + 1 : ones;
}

/* ------------------------------------------------------------------ */
/* GateKeeper with SHD's conventions (Ch. 3, R17)                      */
/* ------------------------------------------------------------------ */

/* GateKeeper with two switches: vacant_zero fills out-of-range mask cells
 * with 0 instead of 1, streak charges each run of L ones ceil(L/3) edits
 * instead of L.  Both off: or_gatekeeper.  Returns min(count, E+1). */
int or_gatekeeper_shd(const uint8_t *R, const uint8_t *F, int m, int E, int vacant_zero,
                      int streak)
{
    if (m <= 0) return 0;
    int h = or_hamming(R, F, m);
    if (h <= E) return h;
    uint8_t *map = (uint8_t *)malloc((size_t)(2 * E + 1) * m);
    uint8_t *amended = (uint8_t *)malloc((size_t)m);
    uint8_t *final_mask = (uint8_t *)malloc((size_t)m);
    or_neighborhood_map(R, F, m, E, map);
    if (vacant_zero)
        for (int d = -E; d <= E; ++d)
            for (int i = 0; i < m; ++i)
                if (i + d < 0 || i + d >= m) map[(size_t)(d + E) * m + i] = 0;
    for (int i = 0; i < m; ++i) final_mask[i] = 1;
    for (int d = -E; d <= E; ++d) {
        or_amend(map + (size_t)(d + E) * m, m, amended);
        for (int i = 0; i < m; ++i) final_mask[i] = final_mask[i] & amended[i];
    }
    int count = 0;
    if (streak) {
        int run = 0;
        for (int i = 0; i <= m; ++i) {
            if (i < m && final_mask[i]) { run++; continue; }
            count += (run + 2) / 3;
            run = 0;
        }
    } else {
        for (int i = 0; i < m; ++i) count += final_mask[i];
    }
    free(final_mask);
    free(amended);
    free(map);
    return count > E + 1 ? E + 1 : count;
}

/* ------------------------------------------------------------------ */
/* Edit distance (Ch. 2 "Accelerating Read Alignment"; Ch. 3 metrics)  */
/* ------------------------------------------------------------------ */

/* Wagner-Fischer global Levenshtein distance with unit costs, full
 * (la+1) x (lb+1) table; matching per R4. */
int or_wf(const uint8_t *a, int la, const uint8_t *b, int lb)
{
    int *prev = (int *)malloc(sizeof(int) * (size_t)(lb + 1));
    int *cur = (int *)malloc(sizeof(int) * (size_t)(lb + 1));
    for (int j = 0; j <= lb; ++j) prev[j] = j;
    for (int i = 1; i <= la; ++i) {
        cur[0] = i;
        for (int j = 1; j <= lb; ++j) {
            int sub = prev[j - 1] + (or_match(a[i - 1], b[j - 1]) ? 0 : 1);
            int del = prev[j] + 1;
            int ins = cur[j - 1] + 1;
            int v = sub < del ? sub : del;
            cur[j] = v < ins ? v : ins;
        }
        int *t = prev; prev = cur; cur = t;
    }
    int d = prev[lb];
    free(prev);
    free(cur);
    return d;
}

/* Ukkonen's banded Levenshtein distance for two sequences of length m:
 * only cells with |i-j| <= E are computed, cells outside the band count
 * as unreachable; returns min(distance, E+1). */
int or_wf_banded(const uint8_t *R, const uint8_t *F, int m, int E)
{
    const int inf = 1 << 29;
    int *prev = (int *)malloc(sizeof(int) * (size_t)(m + 1));
    int *cur = (int *)malloc(sizeof(int) * (size_t)(m + 1));
    for (int j = 0; j <= m; ++j) prev[j] = (j <= E) ? j : inf;
    for (int i = 1; i <= m; ++i) {
        for (int j = 0; j <= m; ++j) {
            int diff = i - j;
            if (diff < 0) diff = -diff;
            if (diff > E) { cur[j] = inf; continue; }
            if (j == 0) { cur[j] = i; continue; }
            int v = prev[j - 1] + (or_match(R[i - 1], F[j - 1]) ? 0 : 1);
            if (prev[j] + 1 < v) v = prev[j] + 1;
            if (cur[j - 1] + 1 < v) v = cur[j - 1] + 1;
            cur[j] = v;
        }
        int *t = prev; prev = cur; cur = t;
    }
    int d = prev[m];
    free(prev);
    free(cur);
    return d > E + 1 ? E + 1 : d;
}

/* ------------------------------------------------------------------ */
/* Batch drivers over ASCII pairs (plain loops, spread over threads)   */
/* ------------------------------------------------------------------ */

typedef struct {
    const uint8_t *reads, *refs;
    const int64_t *read_off, *ref_off;
    const int32_t *lens;
    const int16_t *E;
    int E_stride;
    unsigned deciders;
    uint8_t *accept;
    int16_t *count;
    int32_t *dist;
    int64_t n, begin, end;
    int kind; /* 0 filter, 1 verify, 2 full WF, 3 SS dp, 4 SS full, 5 hamming,
                 6 partitioned SS (p0 = t, p1 = y), 7 Shouji,
                 8 SHD-style GateKeeper (p0 = vacant zero, p1 = streak),
                 9 work counts (four ints per pair) */
    int p0, p1;
} or_job;

static void *or_run_job(void *arg)
{
    or_job *j = (or_job *)arg;
    for (int64_t p = j->begin; p < j->end; ++p) {
        const uint8_t *R = j->reads + j->read_off[p];
        const uint8_t *F = j->refs + j->ref_off[p];
        int m = j->lens[p];
        int E = j->E[j->E_stride ? p : 0];
        switch (j->kind) {
        case 0: {
            int slot = 0;
            if (j->deciders & 1) {
                int c = or_sneakysnake(R, F, m, E);
                j->count[slot * j->n + p] = (int16_t)c;
                j->accept[slot * j->n + p] = (uint8_t)(c <= E);
                slot++;
            }
            if (j->deciders & 2) {
                int c = or_gatekeeper(R, F, m, E);
                j->count[slot * j->n + p] = (int16_t)c;
                j->accept[slot * j->n + p] = (uint8_t)(c <= E);
            }
            break;
        }
        case 1: j->dist[p] = or_wf_banded(R, F, m, E); break;
        case 2: j->dist[p] = or_wf(R, m, F, m); break;
        case 3: j->dist[p] = or_sneakysnake_dp(R, F, m, E); break;
        case 4: j->dist[p] = or_sneakysnake_full(R, F, m, E); break;
        case 5: j->dist[p] = or_hamming(R, F, m); break;
        case 6: j->dist[p] = or_sneakysnake_partitioned(R, F, m, E, j->p0, j->p1); break;
        case 7: j->dist[p] = or_shouji(R, F, m, E); break;
        case 8: j->dist[p] = or_gatekeeper_shd(R, F, m, E, j->p0, j->p1); break;
        case 9: or_work_counts(R, F, m, E, j->dist + 4 * p); break;
        }
    }
    return NULL;
}

static void or_run(or_job proto, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 512) nthreads = 512;
    if (proto.n < nthreads) nthreads = proto.n > 0 ? (int)proto.n : 1;
    pthread_t tid[512];
    or_job jobs[512];
    int64_t per = (proto.n + nthreads - 1) / nthreads;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = proto;
        jobs[t].begin = per * t < proto.n ? per * t : proto.n;
        jobs[t].end = per * (t + 1) < proto.n ? per * (t + 1) : proto.n;
        if (nthreads == 1) or_run_job(&jobs[t]);
        else pthread_create(&tid[t], NULL, or_run_job, &jobs[t]);
    }
    if (nthreads > 1)
        for (int t = 0; t < nthreads; ++t) pthread_join(tid[t], NULL);
}

/* Filter n pairs.  Pair p is reads[read_off[p] .. +lens[p]) against
 * refs[ref_off[p] .. +lens[p]) with threshold E[E_stride ? p : 0].
 * deciders: bit 0 SneakySnake, bit 1 GateKeeper; with both, slot 0 of
 * accept/count holds SneakySnake and slot 1 (offset n) GateKeeper. */
void or_filter_batch(const uint8_t *reads, const int64_t *read_off,
                     const uint8_t *refs, const int64_t *ref_off,
                     const int32_t *lens, const int16_t *E, int E_stride,
                     unsigned deciders, uint8_t *accept, int16_t *count,
                     int64_t n, int nthreads)
{
    or_job j;
    memset(&j, 0, sizeof j);
    j.reads = reads; j.refs = refs; j.read_off = read_off; j.ref_off = ref_off;
    j.lens = lens; j.E = E; j.E_stride = E_stride; j.deciders = deciders;
    j.accept = accept; j.count = count; j.n = n; j.kind = 0;
    or_run(j, nthreads);
}

/* Per-pair integer results: kind 1 banded WF min(ED, E+1), 2 full WF,
 * 3 SneakySnake DP formulation, 4 unsaturated SneakySnake, 5 Hamming,
 * 6 partitioned SneakySnake (p0 = t, p1 = y), 7 Shouji, 8 SHD-style
 * GateKeeper (p0 = vacant zero, p1 = streak counting), 9 the work counts
 * of or_work_counts (out holds 4 n ints). */
void or_int_batch(int kind, const uint8_t *reads, const int64_t *read_off,
                  const uint8_t *refs, const int64_t *ref_off,
                  const int32_t *lens, const int16_t *E, int E_stride,
                  int32_t *out, int64_t n, int nthreads, int p0, int p1)
{
    or_job j;
    memset(&j, 0, sizeof j);
    j.reads = reads; j.refs = refs; j.read_off = read_off; j.ref_off = ref_off;
    j.lens = lens; j.E = E; j.E_stride = E_stride;
    j.dist = out; j.n = n; j.kind = kind; j.p0 = p0; j.p1 = p1;
    or_run(j, nthreads);
}

/* Pack nseq sequences (byte ranges [byte_off[s], byte_off[s+1])) into
 * bit-planes at word offsets word_off[s]; returns the count of bytes that
 * were neither ACGT nor N. */
int64_t or_pack_batch(const uint8_t *ascii, const int64_t *byte_off, int64_t nseq,
                      const int64_t *word_off, uint32_t *lo, uint32_t *hi, uint32_t *nmask)
{
    int64_t bad = 0;
    for (int64_t s = 0; s < nseq; ++s) {
        int len = (int)(byte_off[s + 1] - byte_off[s]);
        bad += or_pack(ascii + byte_off[s], len, lo + word_off[s], hi + word_off[s],
                       nmask + word_off[s]);
    }
    return bad;
}
