// The stack search of PMS8 (Algorithm 2) with neighbourhood enumeration (Algorithm 1)
// and verification, as one persistent kernel per plane layout and threshold T.
//
// Method: Section 2 (stack, filtering, threshold), Section 2.1 (sort rows by size,
// in-place R update), Section 2.3 (subproblems), Section 2.4 (two-l-mer condition,
// consensus distance Cd, Lemma 1, Theorem 1), Algorithms 1 and 2.
//
// Mapping:
//  * A warp owns one (x, u) item at a time (x from S_1, u from the smallest row of the 2d
//    filter) and takes the next from a global counter, so cheap and expensive items
//    balance across the GPU.
//  * Level k (stack size k) keeps, for each string not on the stack, the list of its
//    surviving l-mers: one flat list per level in the warp's scratch, rows in string
//    order, entries (string << 16 | position) with the l-mer's planes inline.  Filtering
//    is lane-parallel over that flat list with warp-ballot compaction; a row's lanes form
//    a segment of each 32-element chunk, whose last lane adds the row's survivors.
//  * The threshold T is the stack size of the pattern-driven part.  The stack is filtered
//    up to size T-1; then every l-mer u' of the smallest remaining row closes one tuple
//    (stack, u') whose common neighbourhood is enumerated directly, and its leaves are
//    verified against the level-(T-1) lists.  The last filter level is skipped because it
//    rarely empties a row and would cost more than the enumeration it saves; the result
//    is the same, since a neighbour's witness in every row survives all necessary filters.
//  * Enumeration, up to four l-mers per tuple (T <= 4): a frontier of nodes with packed
//    byte budgets, expanded a chunk at a time from the deepest level, one child per lane,
//    against per-tuple limit tables.  Larger tuples: the tuples times the subtrees below
//    a P-letter prefix form units that lanes take round-robin and walk depth first.  In
//    both, leaves go to a shared buffer verified 32 at a time.
#pragma once

#include "pms_device.cuh"

namespace pms {
namespace search {

using namespace dev;

// With PMS_BOUNDS_CHECK defined (always for the 64-bit-plane layouts, see their
// translation units) list, l-mer, item and buffer indices are checked before use: a
// failing check records its line and index, raises kErrBounds and skips the access.
#ifdef PMS_BOUNDS_CHECK
#define PMS_OK_IDX(C, idx, lim)                                                         \
    (((unsigned long long)(idx) < (unsigned long long)(lim))                            \
         ? true                                                                         \
         : (pms::search::bad_index((C).stats_dbg, (C).status, __LINE__,                 \
                                   (unsigned long long)(idx)),                          \
            false))
#else
#define PMS_OK_IDX(C, idx, lim) true
#endif
// Debug builds with PMS_DEBUG_DEADLINE stop every warp ~40 s (SM cycles at 2 GHz) into
// a launch, so that a checked run of a long case ends by itself.
#ifdef PMS_DEBUG_DEADLINE
#define PMS_DEADLINE_CYCLES 80000000000ll
#define PMS_PAST_DEADLINE(C) (clock64() - (C).launch_t0 > PMS_DEADLINE_CYCLES)
#else
#define PMS_PAST_DEADLINE(C) false
#endif

#ifndef PMS_SEARCH_MIN_BLOCKS
#define PMS_SEARCH_MIN_BLOCKS 8
#endif
// Resident 4-warp blocks per SM the register allocation must allow.  The search is bound
// by dependent integer ops, so more resident warps beat the spills they cost: 8 blocks
// (64 registers, 32 warps per SM) ran (17,6) 10% faster than 5 (96 registers); 10 and 12
// spilled too much.
constexpr int kSearchMinBlocks = PMS_SEARCH_MIN_BLOCKS;

template <int NB, typename W, int T>
struct WarpSm {
    Lm<NB, W> stk[T];
    Lm<NB, W> cand[kCandBuf];
    uint64_t live[T + 1];
    int len[T + 1];
    int brow[T + 1];
    int bpos[T + 1];
    int start[T + 1][kRMax];
    int cnt[T + 1][kRMax];
    int stop;                 // autotuning: the item ran past its cap
};

struct WarpCounters {
    unsigned long long tuples = 0, compares = 0, nodes = 0, leaves = 0, motifs = 0, ops = 0;
    long long cyc_filter = 0, cyc_enum = 0, cyc_verify = 0;
};

template <typename W>
__device__ __forceinline__ unsigned long long wscale() { return sizeof(W) / 4; }

static __device__ __noinline__ void bad_index(DevStats *st, int *status, int line,
                                       unsigned long long idx)
{
    if (atomicCAS(&st->bad_site, 0ull, (unsigned long long)line) == 0ull)
        st->bad_value = idx;
    atomicOr(status, kErrBounds);
}

template <int NB, typename W>
struct SearchCtx {
    const InstDesc *I;
    int inst;
    const Lm<NB, W> *lm;      // this instance's l-mer table
    uint32_t *lists;          // this warp's lists; level k at (k-2)*list_cap
    Lm<NB, W> *planes;        // the l-mers of those list entries, same indexing
    uint64_t list_cap;
    unsigned char *fscr;      // this warp's frontier-enumeration scratch
    int lmax;                 // longest l of the batch (sizes fscr's table)
    uint64_t *keys;
    unsigned long long *key_count;
    uint64_t key_cap;
    int *status;
    int key_shift;
    int multi;
    Item item;                // the item being searched
    long long t0;             // its start (clock64, lane 0's)
    Item *donate;
    unsigned long long *donate_count;
    uint64_t donate_cap;
    long long budget;
    const unsigned long long *item_next;   // the pass's item counter
    unsigned long long nitems;             // items of this pass
    long long tune_cap;                    // autotuning: items stop after this many cycles
    DevStats *stats_dbg;                   // where index checks record a failure
    long long launch_t0;                   // launch start (checked builds' deadline)
    uint64_t levels;                       // lists per warp
    uint64_t nlm;                          // l-mers of this instance (n * L)
};

// Autotuning only: true (for the whole warp) once the launch has run past the tuning
// cap, here or in another warp; the item then stops, and the pass is reported as capped.
template <int NB, typename W, int T>
__device__ __forceinline__ bool tune_capped(WarpSm<NB, W, T> &S, const SearchCtx<NB, W> &C,
                                            int lane)
{
    if (!C.tune_cap)
        return false;
    if (lane == 0 && !S.stop) {
        if (clock64() - C.launch_t0 > C.tune_cap) {
            S.stop = 1;
            atomicOr(C.status, kErrTuneCapped);
        } else if (*(volatile const int *)C.status & kErrTuneCapped) {
            S.stop = 1;
        }
    }
    __syncwarp();
    return S.stop != 0;
}

// Work splitting: an item that has run longer than the budget hands the positions
// [pos, end) of its range to other warps as up to 64 items with narrower ranges (the
// receiving warp rebuilds the same lists, which are deterministic).  With p2 < 0 the
// range is the item's level-2 range (for threshold 3, its tuples); with p2 >= 0 it is the
// tuples of the level-3 branch row under level-2 position p2 (threshold 4).  Returns true
// when the rest was handed on (the caller stops), false to keep going.
template <int NB, typename W>
__device__ bool maybe_donate(const SearchCtx<NB, W> &C, int pos, int end, int lane,
                             int p2 = -1)
{
    if (!C.donate || end - pos < 2)
        return false;
    long long now = clock64();
    now = __shfl_sync(kFull, now, 0);
    if (now - C.t0 < C.budget)
        return false;
    // only once every item of the pass has been taken: until then idle warps have other
    // work, and splitting would only repeat list building
    unsigned long long taken = 0;
    if (lane == 0)
        taken = *(volatile const unsigned long long *)C.item_next;
    if (__shfl_sync(kFull, taken, 0) < C.nitems)
        return false;
    const int R = end - pos;
    const int chunk = (R + 63) / 64;
    const int nsub = (R + chunk - 1) / chunk;
    // reserve nsub slots only if they all fit, so the list never holds unwritten slots
    unsigned long long base = ~0ull;
    if (lane == 0) {
        unsigned long long cur = *(volatile unsigned long long *)C.donate_count;
        while (cur + nsub <= C.donate_cap) {
            const unsigned long long seen = atomicCAS(C.donate_count, cur, cur + nsub);
            if (seen == cur) {
                base = cur;
                break;
            }
            cur = seen;
        }
    }
    base = __shfl_sync(kFull, base, 0);
    if (base == ~0ull)
        return false;   // no room: keep searching here
    for (int i = lane; i < nsub; i += 32) {
        Item sub = C.item;
        const uint16_t a = (uint16_t)(pos + i * chunk);
        const uint16_t b = (uint16_t)(pos + i * chunk + chunk < end ? pos + i * chunk + chunk : end);
        if (p2 < 0) {
            sub.lo = a;
            sub.hi = b;
            sub.lo3 = 0;
            sub.hi3 = kAllRange;
        } else {
            sub.lo = (uint16_t)p2;
            sub.hi = (uint16_t)(p2 + 1);
            sub.lo3 = a;
            sub.hi3 = b;
        }
        C.donate[base + i] = sub;
    }
    return true;
}

// Row with the fewest survivors at level k (Section 2.1 "Sort rows by size": the next
// stack element comes from the smallest row).  Ties go to the lower string index.
template <int NB, typename W, int T>
__device__ __forceinline__ int choose_branch(const WarpSm<NB, W, T> &S, int k, int lane)
{
    const uint64_t live = S.live[k];
    unsigned a = ((live >> lane) & 1) ? ((unsigned)S.cnt[k][lane] << 6 | lane) : 0xFFFFFFFFu;
    unsigned b = ((live >> (lane + 32)) & 1) ? ((unsigned)S.cnt[k][lane + 32] << 6 | (lane + 32))
                                             : 0xFFFFFFFFu;
    unsigned m = __reduce_min_sync(kFull, a < b ? a : b);
    return (int)(m & 63);
}

// Segment starts of level k from its per-row counts (rows keep string order).
template <int NB, typename W, int T>
__device__ __forceinline__ void row_starts(WarpSm<NB, W, T> &S, int k, int lane)
{
    const uint64_t live = S.live[k];
    int c0 = ((live >> lane) & 1) ? S.cnt[k][lane] : 0;
    int c1 = ((live >> (lane + 32)) & 1) ? S.cnt[k][lane + 32] : 0;
    int s0 = c0, s1 = c1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t0 = __shfl_up_sync(kFull, s0, o);
        int t1 = __shfl_up_sync(kFull, s1, o);
        if (lane >= o) {
            s0 += t0;
            s1 += t1;
        }
    }
    int tot0 = __shfl_sync(kFull, s0, 31);
    S.start[k][lane] = s0 - c0;
    S.start[k][lane + 32] = tot0 + s1 - c1;
    __syncwarp();
}

// Level 2 straight from the strings: stack (x, u); v of string r survives when
// Hd(x,v) <= 2d, Hd(u,v) <= 2d and Cd(x,u,v) <= 3d (Theorem 1 with budgets d,d,d;
// Hd(x,u) <= 2d holds for every item).  Returns false when a row empties.
template <int NB, typename W, int T>
__device__ bool build_level2(WarpSm<NB, W, T> &S, const SearchCtx<NB, W> &C, int b, int lane,
                             WarpCounters &wc)
{
    const InstDesc &I = *C.I;
    const Lm<NB, W> x = S.stk[0], u = S.stk[1];
    const W dxu = diff(x, u);
    const int two_d = 2 * I.d, three_d = 3 * I.d;
    uint32_t *out = C.lists;
    Lm<NB, W> *out_lm = C.planes;
    int len = 0;
    uint64_t live = 0;
    // the l-mers of the next chunk are loaded before the current chunk is tested
    int r_next = b == 1 ? 2 : 1;
    Lm<NB, W> v_next;
#pragma unroll
    for (int b2 = 0; b2 < NB; b2++)
        v_next.p[b2] = 0;
    if (r_next < I.n && lane < I.L)
        v_next = C.lm[(size_t)r_next * I.L + lane];
    for (int r = 1; r < I.n; r++) {
        if (r == b)
            continue;
        const int s0 = len;
        for (int j0 = 0; j0 < I.L; j0 += 32) {
            const int j = j0 + lane;
            bool ok = false;
            const Lm<NB, W> v = v_next;
            {
                int rn = r, jn = j0 + 32;
                if (jn >= I.L) {
                    rn = r + 1 == b ? r + 2 : r + 1;
                    jn = 0;
                }
                if (rn < I.n && jn + lane < I.L)
                    v_next = C.lm[(size_t)rn * I.L + jn + lane];
            }
            if (j < I.L) {
                const W dxv = diff(x, v), duv = diff(u, v);
                ok = popc(dxv) <= two_d && popc(duv) <= two_d &&
                     popc(dxu | dxv) + popc(dxu & dxv & duv) <= three_d;
            }
            const unsigned bal = __ballot_sync(kFull, ok);
            if (ok) {
                const int at = len + __popc(bal & lanemask_lt());
                if (PMS_OK_IDX(C, at, C.list_cap)) {
                    out[at] = ((uint32_t)r << 16) | (uint32_t)j;
                    out_lm[at] = v;
                }
            }
            len += __popc(bal);
        }
        wc.compares += 3ull * I.L;
        wc.ops += (unsigned long long)I.L * op_level2(NB) * wscale<W>();
        if (lane == 0)
            S.cnt[2][r] = len - s0;
        if (len == s0)
            return false;
        live |= 1ull << r;
    }
    if (lane == 0) {
        S.len[2] = len;
        S.live[2] = live;
    }
    __syncwarp();
    row_starts(S, 2, lane);
    return true;
}

// Push stk[k] (stack size becomes k+1) and filter the rows of level k other than the
// branch row into level k+1: v survives when Hd(top,v) <= 2d and, for every earlier stack
// l-mer s, Cd(s, top, v) <= 3d (Theorem 1 with budgets d,d,d; the pair conditions with
// earlier l-mers hold from earlier levels).  With two l-mers below the top, v must also
// meet Lemma 1 for all four: Cd(x, u, top, v) <= 4d.  Returns false as soon as a row
// empties (Section 2: an empty row ends this stack and the search moves on).
template <int NB, typename W, int T>
__device__ bool filter_level(WarpSm<NB, W, T> &S, const SearchCtx<NB, W> &C, int k, int lane,
                             WarpCounters &wc)
{
    const InstDesc &I = *C.I;
    const int two_d = 2 * I.d, three_d = 3 * I.d;
    const Lm<NB, W> top = S.stk[k];
    Lm<NB, W> st[T];
    W dst[T];
#pragma unroll
    for (int i = 0; i < T; i++) {
        if (i < k) {
            st[i] = S.stk[i];
            dst[i] = diff(st[i], top);
        }
    }
    // constants of the four-l-mer condition (stack x, u plus top), used when k == 2
    const W lmask = low_mask<W>(I.l);
    const W dxu = k >= 2 ? diff(st[0], st[1]) : W(0);
    const W c4_none = k >= 2 ? dxu & dst[0] & dst[1] : W(0);   // x,u,top pairwise differ
    const W c4_xuxt = k >= 2 ? dxu | dst[0] : W(0);             // x differs from u or top
    const uint32_t *in = C.lists + (size_t)(k - 2) * C.list_cap;
    uint32_t *out = C.lists + (size_t)(k - 1) * C.list_cap;
    const Lm<NB, W> *in_lm = C.planes + (size_t)(k - 2) * C.list_cap;
    Lm<NB, W> *out_lm = C.planes + (size_t)(k - 1) * C.list_cap;
    const int br = S.brow[k];
    const int bs = S.start[k][br], bc = S.cnt[k][br];
    const int total = S.len[k] - bc;
    const uint64_t live1 = S.live[k] & ~(1ull << br);
    S.cnt[k + 1][lane] = 0;
    S.cnt[k + 1][lane + 32] = 0;
    __syncwarp();
    int len = 0;
    // element vi of the input: the level-k list without the branch row; the entries of a
    // row are contiguous, so a row ends where the next element's row differs
    uint32_t e_next = 0;
    Lm<NB, W> v_next;
#pragma unroll
    for (int b2 = 0; b2 < NB; b2++)
        v_next.p[b2] = 0;
    {
        const int idx = lane < bs ? lane : lane + bc;
        if (lane < total && PMS_OK_IDX(C, idx, C.list_cap)) {
            e_next = in[idx];
            v_next = in_lm[idx];
        }
    }
    for (int c0 = 0; c0 < total; c0 += 32) {
        const int vi = c0 + lane;
        const bool valid = vi < total;
        const uint32_t e = e_next;
        const Lm<NB, W> v = v_next;
        // load the next chunk before working on this one
        {
            const int vn = vi + 32;
            const int idx = vn < bs ? vn : vn + bc;
            if (vn < total && PMS_OK_IDX(C, idx, C.list_cap)) {
                e_next = in[idx];
                v_next = in_lm[idx];
            }
        }
        int row = valid ? (int)(e >> 16) : -1;
        if (valid && !PMS_OK_IDX(C, row, kRMax))
            row = 0;
        bool ok = false;
        if (valid) {
            const W dtv = diff(top, v);
            ok = popc(dtv) <= two_d;
            W div[T];
#pragma unroll
            for (int i = 0; i < T; i++) {
                if (i < k) {
                    div[i] = diff(st[i], v);
                    ok = ok && (popc(dst[i] | div[i]) + popc(dst[i] & div[i] & dtv) <= three_d);
                }
            }
            if (T >= 4 && k == 2) {
                // Lemma 1 for the four l-mers x, u, top, v: per column Cd contributes
                // 3 - [some pair equal] - [some three equal] - [all four equal].
                const W dxv = div[0], duv = div[1];
                const W has2 = ~(c4_none & dxv & duv & dtv) & lmask;
                const W has3 = ~(c4_xuxt & (dxu | dxv) & (dst[0] | dxv) & (dst[1] | duv)) & lmask;
                const W all4 = ~(c4_xuxt | dxv) & lmask;
                ok = ok && 3 * I.l - popc(has2) - popc(has3) - popc(all4) <= 4 * I.d;
            }
        }
        const unsigned bal = __ballot_sync(kFull, ok);
        if (ok) {
            const int at = len + __popc(bal & lanemask_lt());
            if (PMS_OK_IDX(C, at, C.list_cap)) {
                out[at] = e;
                out_lm[at] = v;
            }
        }
        len += __popc(bal);
        // survivors per row: the lanes of one row form a segment of the chunk; its last
        // lane adds the segment's count and, when the row ends there, checks it
        const int first_next = __shfl_sync(kFull, c0 + 32 < total ? (int)(e_next >> 16) : -1, 0);
        const int prow = __shfl_up_sync(kFull, row, 1);
        int nrow = __shfl_down_sync(kFull, row, 1);
        if (lane == 31)
            nrow = first_next;
        const unsigned starts = __ballot_sync(kFull, valid && (lane == 0 || prow != row));
        const bool row_end = valid && (nrow != row || vi + 1 == total);
        bool empty = false;
        if (row_end || (valid && lane == 31)) {
            const unsigned le = (lanemask_lt() << 1) | 1u;
            const int s0 = 31 - __clz(starts & le);
            const int add = __popc(bal & le & ~((1u << s0) - 1u));
            const int tot = S.cnt[k + 1][row] + add;
            S.cnt[k + 1][row] = tot;
            empty = row_end && tot == 0;
        }
        __syncwarp();
        if (__any_sync(kFull, empty)) {
            const int done = c0 + 32 < total ? c0 + 32 : total;
            wc.compares += (unsigned long long)done * (k + 1);
            wc.ops += (unsigned long long)done * (op_filter(NB, k) + (T >= 4 && k == 2 ? op_lemma4() : 0)) * wscale<W>();
            return false;
        }
    }
    wc.compares += (unsigned long long)total * (k + 1);
    wc.ops += (unsigned long long)total * (op_filter(NB, k) + (T >= 4 && k == 2 ? op_lemma4() : 0)) * wscale<W>();
    if (lane == 0) {
        S.len[k + 1] = len;
        S.live[k + 1] = live1;
    }
    __syncwarp();
    row_starts(S, k + 1, lane);
    return true;
}

// prune(T, r) of Algorithm 1 for a prefix of length q (positions [0, q) fixed in M), for
// the tuple st[0..tk-1]: every budget r_i = d - Hd(M[0..q), st_i[0..q)) stays >= 0, every
// pair keeps Hd(st_i[q..], st_j[q..]) <= r_i + r_j (two-l-mer condition, Section 2.4),
// and every triple keeps Cd(st_i[q..], st_j[q..], st_h[q..]) <= r_i + r_j + r_h (Lemma 1;
// with the pair conditions this is Theorem 1, exact for three l-mers).
template <int NB, typename W, int T>
__device__ __forceinline__ bool node_ok(const Lm<NB, W> &M, int q, int tk, int d, W lmask,
                                        const Lm<NB, W> (&st)[T], const W (&dp)[T][T])
{
    const W pre = low_mask<W>(q);
    const W suf = lmask & ~pre;
    int e[T];
    bool ok = true;
#pragma unroll
    for (int i = 0; i < T; i++) {
        if (i < tk) {
            e[i] = popc(diff(M, st[i]) & pre);
            ok = ok && e[i] <= d;
        }
    }
#pragma unroll
    for (int i = 0; i < T; i++) {
#pragma unroll
        for (int j = i + 1; j < T; j++) {
            if (j < tk)
                ok = ok && (e[i] + e[j] + popc(dp[i][j] & suf) <= 2 * d);
        }
    }
#pragma unroll
    for (int i = 0; i < T; i++) {
#pragma unroll
        for (int j = i + 1; j < T; j++) {
#pragma unroll
            for (int h = j + 1; h < T; h++) {
                if (h < tk) {
                    const W a = dp[i][j], b = dp[i][h], c = dp[j][h];
                    const int cd = popc((a | b) & suf) + popc(a & b & c & suf);
                    ok = ok && (e[i] + e[j] + e[h] + cd <= 3 * d);
                }
            }
        }
    }
    return ok;
}

// The 128-bit output key of motif M: letter codes most significant first in the low
// l*kbits bits, the instance id above bit `key_shift` for batches.
template <int NB, typename W>
__device__ __forceinline__ void motif_key(const Lm<NB, W> &M, int l, int kbits, uint64_t inst,
                                          int key_shift, int multi, uint64_t &hi, uint64_t &lo)
{
    hi = 0;
    lo = 0;
    for (int p = 0; p < l; p++) {
        const uint64_t c = (uint64_t)get_letter(M, p);
        hi = (hi << kbits) | (lo >> (64 - kbits));
        lo = (lo << kbits) | c;
    }
    if (multi) {
        if (key_shift >= 64)
            hi |= inst << (key_shift - 64);
        else {
            lo |= inst << key_shift;
            if (key_shift > 64 - kInstBits)
                hi |= inst >> (64 - key_shift);
        }
    }
}

// isMotif(M, R') of Algorithm 2 for up to 32 buffered leaves (one per lane): every row in
// `rows` must hold an l-mer of the level-k list within d of M.  Rows of the tuple are
// satisfied by construction, and an l-mer within d of a common neighbour of the stack
// survives every necessary filter, so scanning the lists equals scanning whole strings.
template <int NB, typename W, int T>
__device__ void verify_and_emit(const WarpSm<NB, W, T> &S, const SearchCtx<NB, W> &C, int k,
                                uint64_t rows, int ncand, int lane, WarpCounters &wc)
{
    const long long c_start = clock64();
    const InstDesc &I = *C.I;
    const Lm<NB, W> M = S.cand[lane < ncand ? lane : 0];
    bool alive = lane < ncand;
    const Lm<NB, W> *list_lm = k >= 2 ? C.planes + (size_t)(k - 2) * C.list_cap : C.planes;
    while (rows && __any_sync(kFull, alive)) {
        // next, the row with the fewest l-mers left: the cheapest to scan and the one
        // most likely to have no neighbour of a candidate
        const unsigned k0 = ((rows >> lane) & 1)
                                ? ((unsigned)min(S.cnt[k][lane], (1 << 25) - 1) << 6) | lane
                                : ~0u;
        const unsigned k1 = ((rows >> (lane + 32)) & 1)
                                ? ((unsigned)min(S.cnt[k][lane + 32], (1 << 25) - 1) << 6) |
                                      (lane + 32)
                                : ~0u;
        const int r = (int)(__reduce_min_sync(kFull, k0 < k1 ? k0 : k1) & 63u);
        rows &= ~(1ull << r);
        const int s0 = S.start[k][r], c = S.cnt[k][r];
        bool hit = false;
        const int nalive = __popc(__ballot_sync(kFull, alive));
        for (int j0 = 0; j0 < c; j0 += 32) {
            const int vi = s0 + (j0 + lane < c ? j0 + lane : 0);
            const Lm<NB, W> vj = PMS_OK_IDX(C, vi, C.list_cap) ? list_lm[vi] : list_lm[0];
            const int jn = c - j0 < 32 ? c - j0 : 32;
            for (int jj = 0; jj < jn; jj++) {
                const Lm<NB, W> v = shfl_lm(vj, jj);
                hit = hit || popc(diff(M, v)) <= I.d;
            }
            wc.compares += (unsigned long long)jn * nalive;
            wc.ops += (unsigned long long)jn * nalive * op_hd(NB) * wscale<W>();
            if (__all_sync(kFull, hit || !alive))
                break;
        }
        alive = alive && hit;
    }
    const unsigned bal = __ballot_sync(kFull, alive);
    if (bal) {
        unsigned long long base = 0;
        if (lane == 0)
            base = atomicAdd(C.key_count, (unsigned long long)__popc(bal));
        base = __shfl_sync(kFull, base, 0);
        wc.motifs += __popc(bal);
        if (alive) {
            const unsigned long long pos = base + __popc(bal & lanemask_lt());
            if (pos < C.key_cap) {
                uint64_t hi, lo;
                motif_key(M, I.l, I.kbits, (uint64_t)C.inst, C.key_shift, C.multi, hi, lo);
                C.keys[2 * pos] = hi;
                C.keys[2 * pos + 1] = lo;
            } else {
                atomicOr(C.status, kErrKeysOverflow);
            }
        }
    }
    wc.cyc_verify += clock64() - c_start;
}

// GenerateNeighborhood (Algorithm 1) followed by isMotif on every leaf.
//  br < 0:  one tuple, the stack stk[0..k-1]; verify against the live rows of level k.
//  br >= 0: k == T-1 and every l-mer u' in the branch row br of level k closes the tuple
//           (stk[0..k-1], u'); verify against the live rows of level k except br.
template <int NB, typename W, int T>
__device__ void enumerate(WarpSm<NB, W, T> &S, const SearchCtx<NB, W> &C, int k, int br,
                          int lane, WarpCounters &wc)
{
    const long long c_start = clock64();
    const long long v_before = wc.cyc_verify;
    const InstDesc &I = *C.I;
    const int l = I.l, d = I.d, K = I.k;
    const W lmask = low_mask<W>(l);
    const bool branch = br >= 0;
    const int tk = branch ? k + 1 : k;
    const uint64_t rows = branch ? (S.live[k] & ~(1ull << br)) : S.live[k];
    Lm<NB, W> st[T];
    W dp[T][T];
#pragma unroll
    for (int i = 0; i < T; i++)
        if (i < k)
            st[i] = S.stk[i];
#pragma unroll
    for (int i = 0; i < T; i++)
#pragma unroll
        for (int j = i + 1; j < T; j++)
            if (j < k)
                dp[i][j] = diff(st[i], st[j]);

    const int B = branch ? S.cnt[k][br] : 1;
    const Lm<NB, W> *blist_lm =
        branch ? C.planes + (size_t)(k - 2) * C.list_cap + S.start[k][br] : C.planes;
    int P = 0, U = 1;
    while (P < l && B * U < 64) {
        P++;
        U *= K;
    }
    const int nunits = B * U;
    wc.tuples += B;

    int ncand = 0;
    int unit = lane - 32;
    bool have = false;
    int q = 0, a = 0;
    Lm<NB, W> M;
#pragma unroll
    for (int b = 0; b < NB; b++)
        M.p[b] = 0;
    unsigned long long nodes = 0;
    unsigned walk_steps = 0;
    for (;;) {
        if ((++walk_steps & 63) == 0 && (tune_capped(S, C, lane) ||
                                          __any_sync(kFull, PMS_PAST_DEADLINE(C))))
            break;
        // Pick this lane's next node: the next sibling, after backtracking as far as
        // needed, or the root of the next unit.  Every lane then tests one node.
        if (have) {
            while (a == K) {
                q--;
                if (q < P) {
                    have = false;
                    break;
                }
                a = get_letter(M, q) + 1;
            }
        }
        bool fresh = false;
        if (!have) {
            unit += 32;
            if (unit < nunits) {
                const int tb = unit / U;
                int code = unit - tb * U;
                if (branch) {
                    st[T - 1] = PMS_OK_IDX(C, S.start[k][br] + tb, C.list_cap) ? blist_lm[tb]
                                                                               : blist_lm[0];
#pragma unroll
                    for (int i = 0; i < T - 1; i++)
                        dp[i][T - 1] = diff(st[i], st[T - 1]);
                }
                for (int p = P - 1; p >= 0; p--) {
                    set_letter(M, p, code % K);
                    code /= K;
                }
                fresh = true;
            }
        } else {
            set_letter(M, q, a);
            a++;
        }
        const bool active = have || fresh;
        const int qt = fresh ? P : q + 1;
        bool leaf = false;
        if (active) {
            nodes++;
            if (node_ok<NB, W, T>(M, qt, tk, d, lmask, st, dp)) {
                if (qt == l)
                    leaf = true;
                else {
                    have = true;
                    q = qt;
                    a = 0;
                }
            }
        }
        const unsigned lb = __ballot_sync(kFull, leaf);
        if (leaf && PMS_OK_IDX(C, ncand + __popc(lb & lanemask_lt()), kCandBuf))
            S.cand[ncand + __popc(lb & lanemask_lt())] = M;
        ncand += __popc(lb);
        wc.leaves += __popc(lb);
        __syncwarp();
        if (ncand >= 32) {
            verify_and_emit(S, C, k, rows, 32, lane, wc);
            __syncwarp();
            const Lm<NB, W> rest = S.cand[32 + (lane < ncand - 32 ? lane : 0)];
            __syncwarp();
            if (lane < ncand - 32)
                S.cand[lane] = rest;
            ncand -= 32;
            __syncwarp();
        }
        if (!__any_sync(kFull, have || unit + 32 < nunits))
            break;
    }
    if (ncand > 0)
        verify_and_emit(S, C, k, rows, ncand, lane, wc);
    __syncwarp();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        nodes += __shfl_xor_sync(kFull, nodes, o);
    wc.nodes += nodes;
    wc.ops += nodes * op_walk(NB, tk) * wscale<W>();
    wc.cyc_enum += (clock64() - c_start) - (wc.cyc_verify - v_before);
}

// ---------------------------------------------------------------------------------
// Frontier form of Algorithm 1 for tuples of at most four l-mers (T <= 4, d <= 41).
//
// Budgets travel with each tree node as packed bytes e (byte i = mismatches so far with
// tuple l-mer i).  With rotations of e inside the tuple, one 32-bit add forms every pair
// sum (bytes e_i + e_{i+1}, e_i + e_{i+2}) and every triple sum (e_i + e_{i+1} + e_{i+2}),
// and a borrow-free byte compare tests them all against per-position limits at once:
//   e_i <= d,   e_i + e_j <= 2d - Hd(T_i[q..], T_j[q..]),
//   e_i + e_j + e_h <= 3d - Cd(T_i[q..], T_j[q..], T_h[q..])
//   e_0 + e_1 + e_2 + e_3 <= 4d - Cd(T_0[q..], .., T_3[q..])        (four l-mers)
// which is prune(T, r) of Algorithm 1 with r_i = d - e_i: the two-l-mer condition and
// Lemma 1 on the suffix (Theorem 1 for three l-mers, Section 2.4).  The limits depend
// only on the tuple and the prefix length q, so they are tabulated once per tuple.
//
// Nodes are expanded a chunk at a time from the deepest non-empty level (so the level
// below is always empty and each level holds at most kFrontCap nodes); every lane tests
// one (node, letter) child.

constexpr int kTupleRound = 32;   // tuples enumerated together
constexpr int kFrontCap = 32;     // nodes per frontier level

template <int NB, typename W>
struct FNode {
    Lm<NB, W> M;                  // prefix (positions below the node's level)
    uint32_t e;                   // packed mismatch counts
    uint32_t b;                   // tuple index within the round
};

template <int NB, typename W>
__host__ __device__ constexpr size_t frontier_scratch_bytes(int lmax)
{
    return (size_t)kTupleRound * (lmax + 1) * sizeof(uint4) +
           (size_t)lmax * kFrontCap * sizeof(FNode<NB, W>);
}

// Any byte of s greater than the same byte of lim (all bytes below 128).
__device__ __forceinline__ bool bytes_gt(uint32_t s, uint32_t lim)
{
    return (((lim | 0x80808080u) - s) & 0x80808080u) != 0x80808080u;
}

// Byte-permute selectors rotating the first tk bytes by one and by two places (other
// bytes read as zero).
__device__ __forceinline__ void rot_selectors(int tk, uint32_t &r1, uint32_t &r2)
{
    r1 = tk == 4 ? 0x0321u : tk == 3 ? 0x4021u : tk == 2 ? 0x4401u : 0x4444u;
    r2 = tk == 4 ? 0x1032u : tk == 3 ? 0x4102u : 0x4444u;
}

// Limit tables of one round of tuples, built by all lanes at once.  Entry b * (l + 1) + q,
// for tuple b and prefix length q, is {letters of the tuple's l-mers at position q-1,
// pair limits (i,i+1), pair limits (i,i+2), triple limits (i,i+1,i+2)}, so testing a
// child at position p reads the single entry for q = p+1.  Every limit needs only a
// count over the suffix from position q: one popcount of a difference mask restricted to
// positions q.., so the entries are independent.  Returns the mask of tuples whose root
// already fails the pair or triple condition (no common d-neighbour, Theorem 1).
template <int NB, typename W, int T>
__device__ uint32_t build_tables(const SearchCtx<NB, W> &C, const Lm<NB, W> (&stack)[T],
                                 const W (&dps)[T][T], int k, const Lm<NB, W> *blist,
                                 uint64_t bpos, int nb, int tk, int l, int d, W lmask,
                                 uint4 *tbl, int lane)
{
    uint32_t bad = 0;
    const int E = nb * (l + 1);
    for (int idx = lane; idx < E; idx += 32) {
        const int b = idx / (l + 1);
        const int q = idx - b * (l + 1);
        Lm<NB, W> st[T];
        W dp[T][T];
#pragma unroll
        for (int i = 0; i < T; i++) {
            st[i] = stack[i];
#pragma unroll
            for (int j = 0; j < T; j++)
                dp[i][j] = dps[i][j];
        }
        if (tk > k) {   // the tuple's last l-mer comes from the branch row
            st[T - 1] = PMS_OK_IDX(C, bpos + b, C.list_cap) ? blist[b] : blist[0];
#pragma unroll
            for (int i = 0; i < T - 1; i++)
                dp[i][T - 1] = diff(st[i], st[T - 1]);
        }
        const W sfx = lmask & ~low_mask<W>(q);
        bool ok = true;
        uint32_t lim1 = 0x7F7F7F7Fu, lim2 = 0xFF7F7F7Fu, lim3 = 0x7F7F7F7Fu, codes = 0;
#pragma unroll
        for (int i = 0; i < T; i++) {
            if (i < tk) {
                const int sh = 8 * i;
                if (tk >= 2) {
                    const int j = (i + 1) % tk;
                    const W dij = i < j ? dp[i][j] : dp[j][i];
                    const int v = 2 * d - popc(dij & sfx);
                    ok = ok && v >= 0;
                    lim1 = (lim1 & ~(0xFFu << sh)) | ((uint32_t)(v < 0 ? 0 : v) << sh);
                }
                if (tk == 4) {
                    const int j = (i + 2) % 4;
                    const W dij = i < j ? dp[i][j] : dp[j][i];
                    const int v = 2 * d - popc(dij & sfx);
                    ok = ok && v >= 0;
                    lim2 = (lim2 & ~(0xFFu << sh)) | ((uint32_t)(v < 0 ? 0 : v) << sh);
                }
                if (tk >= 3) {
                    int a = i, b2 = (i + 1) % tk, c = (i + 2) % tk;
                    if (a > b2) { int t0 = a; a = b2; b2 = t0; }
                    if (b2 > c) { int t0 = b2; b2 = c; c = t0; }
                    if (a > b2) { int t0 = a; a = b2; b2 = t0; }
                    const W x = dp[a][b2], y = dp[a][c], z = dp[b2][c];
                    const int v = 3 * d - popc((x | y) & sfx) - popc(x & y & z & sfx);
                    ok = ok && v >= 0;
                    lim3 = (lim3 & ~(0xFFu << sh)) | ((uint32_t)(v < 0 ? 0 : v) << sh);
                }
                if (q > 0)
                    codes |= (uint32_t)get_letter(st[i], q - 1) << sh;
            }
        }
        if (T >= 4 && tk == 4) {
            // Cd of four l-mers over positions q.. (Lemma 1): per column 4 minus the
            // largest number of equal letters
            const W d01 = dp[0][1], d02 = dp[0][2], d03 = dp[0][3];
            const W d12 = dp[1][2], d13 = dp[1][3], d23 = dp[2][3];
            const W has2 = ~(d01 & d02 & d03 & d12 & d13 & d23);
            const W has3 = ~((d01 | d02) & (d01 | d03) & (d02 | d03) & (d12 | d13));
            const W all4 = ~(d01 | d02 | d03);
            const int cs4 = 3 * (l - q) - popc(has2 & sfx) - popc(has3 & sfx) - popc(all4 & sfx);
            const int v = 4 * d - cs4;
            ok = ok && v >= 0;
            lim2 = (lim2 & 0x00FFFFFFu) | ((uint32_t)(v < 0 ? 0 : v) << 24);
        }
        tbl[idx] = make_uint4(codes, lim1, lim2, lim3);
        if (q == 0 && !ok)
            bad |= 1u << b;
    }
    return __reduce_or_sync(kFull, bad);
}

// Algorithm 1 + isMotif for up to four l-mers per tuple; arguments as in enumerate().
template <int NB, typename W, int T>
__device__ void enumerate_frontier(WarpSm<NB, W, T> &S, const SearchCtx<NB, W> &C, int k,
                                   int br, int lane, WarpCounters &wc, int t_lo = 0,
                                   int t_hi = 1 << 30, bool may_split = false, int p2 = -1)
{
    static_assert(T <= 4, "the packed-byte frontier holds at most four budgets");
    const long long c_start = clock64();
    const long long v_before = wc.cyc_verify;
    const InstDesc &I = *C.I;
    const int l = I.l, d = I.d, K = I.k;
    const bool branch = br >= 0;
    const int tk = branch ? k + 1 : k;
    const uint64_t rows = branch ? (S.live[k] & ~(1ull << br)) : S.live[k];
    uint4 *const tbl_all = reinterpret_cast<uint4 *>(C.fscr);
    FNode<NB, W> *const front = reinterpret_cast<FNode<NB, W> *>(
        C.fscr + (size_t)kTupleRound * (C.lmax + 1) * sizeof(uint4));
    const int B = branch ? S.cnt[k][br] : 1;
    const Lm<NB, W> *blist_lm =
        branch ? C.planes + (size_t)(k - 2) * C.list_cap + S.start[k][br] : C.planes;

    const W lmask = low_mask<W>(l);
    Lm<NB, W> stack[T];
    W dps[T][T];
#pragma unroll
    for (int i = 0; i < T; i++) {
        if (i < k)
            stack[i] = S.stk[i];
        else
#pragma unroll
            for (int b2 = 0; b2 < NB; b2++)
                stack[i].p[b2] = 0;
    }
#pragma unroll
    for (int i = 0; i < T; i++)
#pragma unroll
        for (int j = 0; j < T; j++)
            dps[i][j] = (i < j && j < k) ? diff(stack[i], stack[j]) : W(0);

    uint32_t r1, r2;
    rot_selectors(tk, r1, r2);
    uint32_t lim0 = 0x7F7F7F7Fu, used = 0;
    for (int i = 0; i < tk; i++) {
        lim0 = (lim0 & ~(0xFFu << (8 * i))) | ((uint32_t)d << (8 * i));
        used |= 1u << (8 * i);
    }
    const int chunk = K >= 32 ? 1 : 32 / K;   // nodes expanded per step
    const int my_node = lane / K, my_alpha = lane - (lane / K) * K;
    const uint32_t alpha_rep = (uint32_t)my_alpha * 0x01010101u;
    wc.tuples += (t_hi < B ? t_hi : B) > t_lo ? (t_hi < B ? t_hi : B) - t_lo : 0;
    unsigned long long nodes = 0;
    int ncand = 0;

    const int t_end = t_hi < B ? t_hi : B;
    unsigned steps = 0;
    for (int base = t_lo; base < t_end; base += kTupleRound) {
        if (may_split && base > t_lo && maybe_donate(C, base, t_end, lane, p2))
            break;
        if (tune_capped(S, C, lane))
            break;
        const int nb = t_end - base < kTupleRound ? t_end - base : kTupleRound;
        __syncwarp();   // the previous round's nodes are all read
        const uint32_t bad = build_tables<NB, W, T>(
            C, stack, dps, k, blist_lm + base, branch ? (uint64_t)S.start[k][br] + base : 0, nb,
            tk, l, d, lmask, tbl_all, lane);
        const bool root_ok = lane < nb && !((bad >> lane) & 1);
        __syncwarp();
        // roots: empty prefix, no mismatches
        unsigned bal = __ballot_sync(kFull, root_ok);
        if (root_ok) {
            FNode<NB, W> nd;
#pragma unroll
            for (int b2 = 0; b2 < NB; b2++)
                nd.M.p[b2] = 0;
            nd.e = 0;
            nd.b = (uint32_t)lane;
            front[__popc(bal & lanemask_lt())] = nd;
        }
        // lane i keeps the node counts of levels i and i + 32
        int cnt_lo = lane == 0 ? __popc(bal) : 0, cnt_hi = 0;
        // the deepest non-empty level and its node count (warp-uniform)
        int deepest = __popc(bal) ? 0 : -1, have = __popc(bal);
        __syncwarp();
        while (deepest >= 0) {
            if ((++steps & 63) == 0 && (tune_capped(S, C, lane) ||
                                        __any_sync(kFull, PMS_PAST_DEADLINE(C))))
                break;
            const int p = deepest;
            const int c = have < chunk ? have : chunk;
            const int first = have - c;
            if (lane == (p & 31)) {
                if (p < 32)
                    cnt_lo = first;
                else
                    cnt_hi = first;
            }
            bool ok = false;
            FNode<NB, W> child;
            if (my_node < c) {
                const FNode<NB, W> nd = front[(unsigned)p * kFrontCap + first + my_node];
                const uint4 lim = tbl_all[nd.b * (unsigned)(l + 1) + (unsigned)(p + 1)];
                const uint32_t x = lim.x ^ alpha_rep;
                const uint32_t inc =
                    (((((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x) & 0x80808080u) >> 7) & used;
                const uint32_t e = nd.e + inc;
                const uint32_t s1 = e + __byte_perm(e, 0, r1);
                const uint32_t s2 = e + __byte_perm(e, 0, r2);
                const uint32_t s3 = s1 + __byte_perm(e, 0, r2);
                // byte 3 of lim.z bounds the sum of all budgets used (Lemma 1, four l-mers)
                ok = !(bytes_gt(e, lim0) | bytes_gt(s1, lim.y) |
                       bytes_gt(s2 & 0x00FFFFFFu, lim.z | 0x7F000000u) | bytes_gt(s3, lim.w) |
                       (((e * 0x01010101u) >> 24) > (lim.z >> 24)));
                child.M = nd.M;
                set_letter(child.M, p, my_alpha);
                child.e = e;
                child.b = nd.b;
                nodes++;
            }
            const unsigned okb = __ballot_sync(kFull, ok);
            if (p + 1 == l) {
                if (ok && PMS_OK_IDX(C, ncand + __popc(okb & lanemask_lt()), kCandBuf))
                    S.cand[ncand + __popc(okb & lanemask_lt())] = child.M;
                ncand += __popc(okb);
                wc.leaves += __popc(okb);
                __syncwarp();
                if (ncand >= 32) {
                    verify_and_emit(S, C, k, rows, 32, lane, wc);
                    __syncwarp();
                    const Lm<NB, W> rest = S.cand[32 + (lane < ncand - 32 ? lane : 0)];
                    __syncwarp();
                    if (lane < ncand - 32)
                        S.cand[lane] = rest;
                    ncand -= 32;
                    __syncwarp();
                }
            } else if (okb) {
                // the level below is empty: its nodes start at 0
                if (ok)
                    front[(unsigned)(p + 1) * kFrontCap + __popc(okb & lanemask_lt())] = child;
                if (lane == ((p + 1) & 31)) {
                    if (p + 1 < 32)
                        cnt_lo = __popc(okb);
                    else
                        cnt_hi = __popc(okb);
                }
                __syncwarp();
            }
            if (p + 1 < l && okb) {
                deepest = p + 1;
                have = __popc(okb);
            } else if (first > 0) {
                have = first;
            } else {
                // level p is used up: the next is the highest lane whose count is non-zero
                const unsigned hi = __ballot_sync(kFull, cnt_hi > 0);
                const unsigned lo = __ballot_sync(kFull, cnt_lo > 0);
                deepest = hi ? 63 - __clz(hi) : lo ? 31 - __clz(lo) : -1;
                have = deepest < 0 ? 0
                                   : __shfl_sync(kFull, deepest < 32 ? cnt_lo : cnt_hi,
                                                 deepest & 31);
            }
        }
    }
    if (ncand > 0)
        verify_and_emit(S, C, k, rows, ncand, lane, wc);
    __syncwarp();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        nodes += __shfl_xor_sync(kFull, nodes, o);
    wc.nodes += nodes;
    wc.ops += nodes * (op_child(NB) - 2ull * NB + 2ull * NB * wscale<W>());
    wc.cyc_enum += (clock64() - c_start) - (wc.cyc_verify - v_before);
}

// Enumeration entry: the frontier form for T <= 4 (the host sends instances with
// d > 41 to T >= 5), the per-lane walk otherwise.
template <int NB, typename W, int T>
__device__ __forceinline__ void enumerate_any(WarpSm<NB, W, T> &S, const SearchCtx<NB, W> &C,
                                              int k, int br, int lane, WarpCounters &wc)
{
    if constexpr (T <= 4)
        enumerate_frontier(S, C, k, br, lane, wc);
    else
        enumerate(S, C, k, br, lane, wc);
}

// One (x, u) item: Algorithm 2 from stack size 2, with an explicit stack of levels.
template <int NB, typename W, int T>
__device__ void run_item(WarpSm<NB, W, T> &S, SearchCtx<NB, W> &C, const Item &it, int lane,
                         WarpCounters &wc)
{
    const InstDesc &I = *C.I;
    if (lane == 0) {
        S.stk[0] = PMS_OK_IDX(C, it.x, C.nlm) ? C.lm[it.x] : C.lm[0];
        S.stop = 0;
    }
    if (it.b == 0xFFFF) {  // one string: the d-neighbourhood of x is the answer
        if (lane == 0)
            S.live[1] = 0;
        __syncwarp();
        enumerate_any(S, C, 1, -1, lane, wc);
        return;
    }
    if (lane == 0)
        S.stk[1] = PMS_OK_IDX(C, (uint64_t)it.b * I.L + it.u, C.nlm)
                       ? C.lm[(size_t)it.b * I.L + it.u]
                       : C.lm[0];
    __syncwarp();
    long long c0 = clock64();
    const bool alive = build_level2(S, C, it.b, lane, wc);
    wc.cyc_filter += clock64() - c0;
    if (!alive)
        return;
    if (T == 2 || S.live[2] == 0) {
        enumerate_any(S, C, 2, -1, lane, wc);
        return;
    }
    if constexpr (T == 3) {
        enumerate_frontier(S, C, 2, choose_branch(S, 2, lane), lane, wc, it.lo,
                           it.hi == kAllRange ? 1 << 30 : it.hi, true);
        return;
    }
    int k = 2;
    const int b2 = choose_branch(S, 2, lane);
    const int end2 = it.hi == kAllRange ? S.cnt[2][b2] : (it.hi < S.cnt[2][b2] ? it.hi : S.cnt[2][b2]);
    if (lane == 0) {
        S.brow[2] = b2;
        S.bpos[2] = it.lo;
    }
    __syncwarp();
    if constexpr (T == 4) {
        if (it.hi3 != kAllRange) {
            // one level-2 position and a range of the tuples below it
            if (it.lo >= end2)
                return;
            const Lm<NB, W> e = C.planes[S.start[2][b2] + it.lo];
            __syncwarp();
            if (lane == 0) {
                S.bpos[2] = it.lo + 1;
                S.stk[2] = e;
            }
            __syncwarp();
            if (!filter_level(S, C, 2, lane, wc) || S.live[3] == 0)
                return;
            enumerate_frontier(S, C, 3, choose_branch(S, 3, lane), lane, wc, it.lo3, it.hi3,
                               true, it.lo);
            return;
        }
    }
    for (;;) {
        // invariant: k < T-1 and the branch row of level k is chosen
        const int br = S.brow[k];
        const int pos = S.bpos[k];
        if (pos >= (k == 2 ? end2 : S.cnt[k][br])) {
            if (k == 2)
                return;
            k--;
            continue;
        }
        if (k == 2 && pos > it.lo && maybe_donate(C, pos, end2, lane))
            return;
        if (tune_capped(S, C, lane))
            return;
        const uint64_t pidx = (uint64_t)(k - 2) * C.list_cap + S.start[k][br] + pos;
        const Lm<NB, W> e = PMS_OK_IDX(C, pidx, C.levels * C.list_cap) ? C.planes[pidx]
                                                                          : C.planes[0];
        __syncwarp();
        if (lane == 0) {
            S.bpos[k] = pos + 1;
            S.stk[k] = e;
        }
        __syncwarp();
        c0 = clock64();
        const bool ok = filter_level(S, C, k, lane, wc);
        wc.cyc_filter += clock64() - c0;
        if (!ok)
            continue;
        const int k1 = k + 1;
        if (S.live[k1] == 0) {
            enumerate_any(S, C, k1, -1, lane, wc);
        } else if (k1 == T - 1) {
            if constexpr (T == 4)
                enumerate_frontier(S, C, k1, choose_branch(S, k1, lane), lane, wc, 0, 1 << 30,
                                   true, pos);
            else
                enumerate_any(S, C, k1, choose_branch(S, k1, lane), lane, wc);
        } else {
            k = k1;
            const int nb = choose_branch(S, k, lane);
            if (lane == 0) {
                S.brow[k] = nb;
                S.bpos[k] = 0;
            }
            __syncwarp();
        }
    }
}

template <int NB, typename W, int T>
__global__ void __launch_bounds__(128, kSearchMinBlocks) search_kernel(
    const InstDesc *__restrict__ inst, const Lm<NB, W> *__restrict__ lmers,
    const Item *__restrict__ items, const unsigned long long *item_count, uint64_t item_cap,
    unsigned long long *item_next, uint32_t *lists, uint64_t list_cap, uint64_t *keys,
    unsigned long long *key_count, uint64_t key_cap, int *status, DevStats *stats,
    int key_shift, int multi, unsigned char *fscr, uint64_t fscr_stride, int lmax,
    int item_stride, Item *donate, unsigned long long *donate_count, uint64_t donate_cap,
    long long budget, ItemTrace *trace, void *planes, long long tune_cap)
{
    extern __shared__ unsigned char smem_raw[];
    WarpSm<NB, W, T> &S = reinterpret_cast<WarpSm<NB, W, T> *>(smem_raw)[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    constexpr int levels = T > 2 ? T - 2 : 1;
    SearchCtx<NB, W> C;
    C.lists = lists + gw * (uint64_t)levels * list_cap;
    C.planes = static_cast<Lm<NB, W> *>(planes) + gw * (uint64_t)levels * list_cap;
    C.list_cap = list_cap;
    C.fscr = fscr + gw * fscr_stride;
    C.lmax = lmax;
    C.keys = keys;
    C.key_count = key_count;
    C.key_cap = key_cap;
    C.status = status;
    C.key_shift = key_shift;
    C.multi = multi;
    C.donate = donate;
    C.donate_count = donate_count;
    C.donate_cap = donate_cap;
    C.budget = budget;
    WarpCounters wc;
    unsigned long long done = 0, item_max = 0;
    const long long busy0 = clock64();
    const unsigned long long nall = *item_count < item_cap ? *item_count : item_cap;
    const unsigned long long nitems = (nall + item_stride - 1) / item_stride;
    C.item_next = item_next;
    C.nitems = nitems;
    C.tune_cap = tune_cap;
    C.stats_dbg = stats;
    C.levels = levels;
    C.launch_t0 = clock64();
    for (;;) {
        unsigned long long it = 0;
        if (lane == 0)
            it = (tune_cap && (*(volatile const int *)status & kErrTuneCapped))
                     ? nitems   // a tuning pass already capped: nothing more to learn
                     : atomicAdd(item_next, 1ull);
        it = __shfl_sync(kFull, it, 0);
        if (it >= nitems)
            break;
        if (!PMS_OK_IDX(C, it * item_stride, item_cap))
            break;
        if (PMS_PAST_DEADLINE(C)) {
            if (lane == 0)
                bad_index(stats, status, 1000000 + __LINE__, it);
            break;
        }
        const Item item = items[it * item_stride];
        C.I = inst + item.inst;
        C.inst = (int)item.inst;
        C.lm = lmers + C.I->lmer_off;
        C.nlm = (uint64_t)C.I->n * C.I->L;
        const long long it0 = __shfl_sync(kFull, clock64(), 0);
        C.item = item;
        C.t0 = it0;
        const unsigned long long n0 = wc.nodes, l0 = wc.leaves, t0 = wc.tuples;
        run_item(S, C, item, lane, wc);
        const unsigned long long dt = (unsigned long long)(clock64() - it0);
        if (trace && lane == 0)
            trace[it] = ItemTrace{item, dt, wc.nodes - n0, wc.leaves - l0, wc.tuples - t0};
        item_max = dt > item_max ? dt : item_max;
        done++;
        __syncwarp();
    }
    if (lane == 0) {
        atomicAdd(&stats->items, done);
        atomicAdd(&stats->tuples, wc.tuples);
        atomicAdd(&stats->hd_compares, wc.compares);
        atomicAdd(&stats->enum_nodes, wc.nodes);
        atomicAdd(&stats->leaves, wc.leaves);
        atomicAdd(&stats->raw_motifs, wc.motifs);
        atomicAdd(&stats->cyc_filter, (unsigned long long)wc.cyc_filter);
        atomicAdd(&stats->cyc_enum, (unsigned long long)wc.cyc_enum);
        atomicAdd(&stats->cyc_verify, (unsigned long long)wc.cyc_verify);
        atomicAdd(&stats->search_ops, wc.ops);
        const unsigned long long busy = (unsigned long long)(clock64() - busy0);
        atomicMax(&stats->busy_max, busy);
        atomicAdd(&stats->busy_sum, busy);
        atomicAdd(&stats->warps, 1ull);
        atomicMax(&stats->item_max, item_max);
    }
}

template <int NB, typename W, int T>
size_t smem_bytes(int wpb)
{
    return sizeof(WarpSm<NB, W, T>) * (size_t)wpb;
}

template <int NB, typename W, int T>
cudaError_t launch(const SearchArgs &a, cudaStream_t s)
{
    const size_t smem = smem_bytes<NB, W, T>(a.cfg.warps_per_block);
    cudaError_t e = cudaFuncSetAttribute(search_kernel<NB, W, T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    search_kernel<NB, W, T><<<a.cfg.blocks, a.cfg.warps_per_block * 32, smem, s>>>(
        a.inst, static_cast<const Lm<NB, W> *>(a.lmers), a.items, a.item_count, a.item_cap,
        a.item_next, a.lists, a.list_cap, a.keys, a.key_count, a.key_cap, a.status, a.stats,
        a.key_shift, a.multi, a.fscr, a.fscr_stride, a.lmax, a.item_stride > 0 ? a.item_stride : 1,
        a.donate, a.donate_count, a.donate_cap, a.budget, a.trace, a.planes, a.tune_cap);
    return cudaGetLastError();
}

template <int NB, typename W, int T>
int max_blocks(int wpb)
{
    int nb = 0;
    const size_t smem = smem_bytes<NB, W, T>(wpb);
    cudaFuncSetAttribute(search_kernel<NB, W, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, search_kernel<NB, W, T>, wpb * 32,
                                                      smem) != cudaSuccess)
        return 0;
    return nb;
}

// Dispatch over the thresholds 2..kTMax for one plane layout.
template <int NB, typename W>
cudaError_t launch_layout(int t, const SearchArgs &a, cudaStream_t s)
{
    switch (t) {
    case 2: return launch<NB, W, 2>(a, s);
    case 3: return launch<NB, W, 3>(a, s);
    case 4: return launch<NB, W, 4>(a, s);
    case 5: return launch<NB, W, 5>(a, s);
    case 6: return launch<NB, W, 6>(a, s);
    case 7: return launch<NB, W, 7>(a, s);
    case 8: return launch<NB, W, 8>(a, s);
    }
    return cudaErrorInvalidValue;
}

template <int NB, typename W>
int max_blocks_layout(int t, int wpb)
{
    switch (t) {
    case 2: return max_blocks<NB, W, 2>(wpb);
    case 3: return max_blocks<NB, W, 3>(wpb);
    case 4: return max_blocks<NB, W, 4>(wpb);
    case 5: return max_blocks<NB, W, 5>(wpb);
    case 6: return max_blocks<NB, W, 6>(wpb);
    case 7: return max_blocks<NB, W, 7>(wpb);
    case 8: return max_blocks<NB, W, 8>(wpb);
    }
    return 0;
}

template <int NB, typename W>
size_t fscr_layout(int lmax)
{
    return frontier_scratch_bytes<NB, W>(lmax);
}

}  // namespace search
}  // namespace pms
