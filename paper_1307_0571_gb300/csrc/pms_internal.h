// Internal declarations shared by the CUDA translation units of libpms.
//
// Device data of one batch (one launch sequence):
//   seqs     all instances' sequences, byte-concatenated (instance i at InstDesc.seq_off)
//   maps     256-byte letter -> code table per instance (0xFF = not in the alphabet)
//   lmers    every l-mer of every string as bit planes: plane b holds bit b of each
//            letter's code, bit p = position p (Section 2.1 "Compress l-mers", planar form)
//   items    (instance, x, branch row, u) subproblems that passed the 2d filter
//   keys     verified motifs as 128-bit sortable keys (instance id in the top bits)
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pms {

constexpr int kTMax = 8;        // deepest stack (threshold) supported
constexpr int kRMax = 64;       // most strings per instance (row bitmasks are 64-bit)
constexpr int kCandBuf = 64;    // leaf buffer per warp
constexpr int kInstBits = 16;   // instance id bits in the output key

// One instance of a batch, as the kernels see it.
struct InstDesc {
    uint64_t seq_off;     // byte offset of the instance's strings in the batch buffer
    uint64_t lmer_off;    // offset (in l-mers) of its l-mer table
    uint64_t x_off;       // offset of its first x in the batch's x enumeration
    int n, m, l, d;
    int L;                // m - l + 1
    int k;                // alphabet size
    int kbits;            // bits per letter in the output key
    int t;                // threshold stack size
    int x_begin, x_end;   // subproblem range of S_1
};

// One (x, u) subproblem: x = S_1[x..], u = S_b[u..] with Hd(x,u) <= 2d and b the
// smallest row of the 2d filter (Section 2.1 "Sort rows by size").  b = 0xFFFF marks a
// single-string instance (no u).  [lo, hi) restricts the subproblem to those positions
// of the level-2 branch row (the stack's third l-mer; for threshold 3 the tuples of the
// enumeration): a subproblem that runs past its time budget hands the rest of its range
// to other warps as items with narrower ranges.  hi = 0xFFFF means the whole row.
//   With threshold 4 an item can also stand for one level-2 position p2 = lo (hi = lo+1)
// and the tuples [lo3, hi3) of the branch row below it; hi3 = 0xFFFF means "not so".
struct Item {
    uint32_t inst;
    uint16_t x;
    uint16_t u;
    uint16_t b;
    uint16_t lo;
    uint16_t hi;
    uint16_t lo3;
    uint16_t hi3;
    uint16_t pad;
};
constexpr uint16_t kAllRange = 0xFFFF;

// Per-item profile record (written only when tracing is on; see PMS_ITEM_TRACE).
struct ItemTrace {
    Item item;
    unsigned long long cycles, nodes, leaves, tuples;
};

// Counters the kernels accumulate (one struct in device memory per solve).
struct DevStats {
    unsigned long long items;
    unsigned long long tuples;
    unsigned long long hd_compares;
    unsigned long long enum_nodes;
    unsigned long long leaves;
    unsigned long long raw_motifs;
    unsigned long long cyc_filter;   // SM cycles summed over warps, per search phase
    unsigned long long cyc_enum;
    unsigned long long cyc_verify;
    unsigned long long search_ops;   // algorithmic integer ops of the search kernel
    unsigned long long busy_max;     // largest per-warp busy time (cycles)
    unsigned long long busy_sum;     // per-warp busy time summed over warps
    unsigned long long warps;        // warps of the search launch
    unsigned long long item_max;     // most cycles one item took
    unsigned long long bad_site;     // PMS_BOUNDS_CHECK builds: first failing check's line
    unsigned long long bad_value;    // ... and the index it saw
};

// Algorithmic integer-op counts per unit of work, for NB planes of 32-bit words (64-bit
// words cost twice).  A diff (positions where two l-mers differ) is NB three-input
// logic ops; Hd is diff + popcount + compare.
//   Hd test                           NB + 2
//   Theorem 1 triple, given D(s,top)  NB + 6  (diff, or, popc, and3, popc, add, compare)
//   level-2 test (x, u, v)            2 NB + 10
//   filter test at stack size k       NB + 2 + k (NB + 6)
//   Lemma 1 for four l-mers (filter)  14      (3 masks of 2-3 logic ops, 3 popc, adds)
//   frontier child (packed budgets)   29 + 2 NB (letter mismatch bytes, 3 byte permutes,
//                                     3 adds, 4 byte-wise compares, the budget sum and its
//                                     compare, set the letter)
//   per-lane walk node, tuple of tk   tk (NB + 3) + 5 C(tk,2) + 9 C(tk,3)
__host__ __device__ inline unsigned long long op_hd(int nb) { return nb + 2; }
__host__ __device__ inline unsigned long long op_level2(int nb) { return 2 * nb + 10; }
__host__ __device__ inline unsigned long long op_filter(int nb, int k)
{
    return nb + 2 + (unsigned long long)k * (nb + 6);
}
__host__ __device__ inline unsigned long long op_lemma4() { return 14; }
__host__ __device__ inline unsigned long long op_child(int nb) { return 29 + 2 * nb; }
__host__ __device__ inline unsigned long long op_walk(int nb, int tk)
{
    return (unsigned long long)tk * (nb + 3) + 5ull * tk * (tk - 1) / 2 +
           9ull * tk * (tk - 1) * (tk - 2) / 6;
}

// Status bits a kernel raises.
enum : int {
    kErrAlphabet = 1,
    kErrItemsOverflow = 2,
    kErrKeysOverflow = 4,
    kErrListOverflow = 8,
    kErrTuneCapped = 16,      // an autotuning pass stopped an item at its cycle cap
    kErrBounds = 32,          // PMS_BOUNDS_CHECK builds: an index failed its check
};

// Plane layout classes: bits per letter (2 for |alphabet| <= 4, else 5) and word width.
enum class Layout { DNA32, DNA64, P5_32, P5_64 };

// ---- kernels (pms_kernels.cu) ----
struct LaunchCfg {
    int warps_per_block;
    int blocks;           // search grid size
};

// Pack every string of the batch into planar l-mers; flags bytes outside the alphabet.
cudaError_t launch_pack(Layout lay, const InstDesc *d_inst, const uint64_t *d_lmer_prefix,
                        int ninst, uint64_t total_lmers, const uint8_t *d_seqs,
                        const uint8_t *d_maps, void *d_lmers, int *d_status,
                        cudaStream_t s);

// The 2d filter of every x (Section 2): picks the smallest row and emits the items.
cudaError_t launch_items(Layout lay, const InstDesc *d_inst, const uint64_t *d_x_prefix,
                         int ninst, uint64_t total_x, const void *d_lmers, Item *d_items,
                         unsigned long long *d_item_count, uint64_t item_cap,
                         int *d_status, DevStats *d_stats, cudaStream_t s);

// Arguments of one search launch.
struct SearchArgs {
    const InstDesc *inst;
    const void *lmers;
    const Item *items;
    const unsigned long long *item_count;
    uint64_t item_cap;
    unsigned long long *item_next;
    uint32_t *lists;          // scratch: search_levels(t) lists of list_cap entries per warp
    uint64_t list_cap;
    uint64_t *keys;
    unsigned long long *key_count;
    uint64_t key_cap;
    int *status;
    DevStats *stats;
    int key_shift;
    int multi;
    LaunchCfg cfg;
    unsigned char *fscr;      // scratch: frontier-enumeration tables and levels per warp
    uint64_t fscr_stride;     // bytes per warp (search_frontier_bytes(lay, lmax))
    int lmax;                 // longest l in the batch
    int item_stride;          // search items 0, s, 2s, ... only (autotuner samples); 1 = all
    Item *donate;             // items handed on by subproblems past their budget
    unsigned long long *donate_count;
    uint64_t donate_cap;
    long long budget;         // cycles an item runs before it hands on the rest of its range
    ItemTrace *trace;         // per-item records of the first pass, or null
    void *planes;             // scratch: the l-mers of the list entries (same shape as lists)
    long long tune_cap;       // autotuning: stop any item still running after this many
                              // cycles (0: no cap)
};

// Lists each search warp keeps for threshold t (levels 2..t-1, at least one).  Every list
// entry is 4 bytes of (string, position) in `lists` plus the l-mer itself in `planes`.
inline int search_levels(int t) { return t > 2 ? t - 2 : 1; }

// The stack search + enumeration + verification (Algorithm 2 with Algorithm 1),
// persistent over the item list, for plane layout `lay` and threshold t (2..kTMax).
cudaError_t launch_search(Layout lay, int t, const SearchArgs &a, cudaStream_t s);

// Resident search blocks per SM for a block of `warps_per_block` warps.
int search_max_blocks(Layout lay, int t, int warps_per_block);

// Frontier-enumeration scratch bytes per warp for l-mers up to lmax letters.
size_t search_frontier_bytes(Layout lay, int lmax);

// ---- sort / unique / decode (pms_sort.cu) ----
struct SortScratch {
    uint64_t *keys_alt;         // second key buffer (2 words per key)
    unsigned int *hist;         // digit histograms
    unsigned int *flags;        // per-tile counts for compaction
    size_t cap_keys;
    size_t cap_tiles;
};

constexpr int kSortTile = 1024;

// Sort n 128-bit keys (pairs of u64: [2i] = high word, [2i+1] = low word) ascending on
// their low `bits` bits (high word first) and remove duplicates.  Returns the number of
// unique keys, left in `keys`.  Synchronises the stream once to read the count back.
cudaError_t sort_unique_keys(uint64_t *keys, size_t n, int bits, SortScratch &scr,
                             unsigned long long *d_total, size_t *n_unique, cudaStream_t s);

// Per-instance index ranges [first, last] of sorted unique keys (-1 when empty).
cudaError_t launch_ranges(const uint64_t *d_keys, size_t n, int key_shift, int multi,
                          int ninst, long long *d_first, long long *d_last, cudaStream_t s);

// Decode sorted keys into letters: key i of instance j goes to
// out + byte_off[j] + (i - first[j]) * l_j.  `alpha` holds 32 letters per instance.
cudaError_t launch_decode(const uint64_t *d_keys, size_t n, int key_shift, int multi,
                          const InstDesc *d_inst, const uint8_t *d_alpha, char *d_out,
                          const uint64_t *d_byte_off, const long long *d_first,
                          cudaStream_t s);

}  // namespace pms
