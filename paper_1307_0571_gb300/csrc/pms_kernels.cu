// Search kernels of libpms: packing, the 2d filter of every x, and the persistent
// stack search with neighbourhood enumeration and verification.
//
// Method (Nicolae & Rajasekaran, PMS8): Section 2 (matrix R, stack, filtering, threshold),
// Section 2.1 (sort rows by size, compressed l-mers, in-place R update), Section 2.3 (one
// subproblem per l-mer of S_1), Section 2.4 (two-l-mer condition, consensus distance,
// Lemma 1, Theorem 1), Algorithm 1 (GenerateNeighborhood) and Algorithm 2 (PMS8).
//
// GPU mapping:
//  * l-mers are stored as bit planes (plane b = bit b of every letter code), so the set of
//    positions where two l-mers differ is OR_b(a_b ^ b_b) and Hd is one popcount per word
//    (replaces the paper's 2^16-entry lookup table of Section 2.1).
//  * One warp owns one (x, u) subproblem at a time and pulls the next one from a global
//    counter.  Filtering is lane-parallel over the surviving l-mers of all rows with
//    warp-ballot stream compaction into per-warp lists (the in-place R update of
//    Section 2.1 becomes a stack of compacted lists, one per stack size).
//  * The pattern-driven part runs one depth-first walk per lane over a slice of the
//    Algorithm 1 tree; leaves are buffered in shared memory and verified 32 at a time.
#include <climits>
#include <cstdint>

#include "pms_internal.h"

namespace pms {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

template <typename W>
__device__ __forceinline__ int popc(W x);
template <>
__device__ __forceinline__ int popc<uint32_t>(uint32_t x) { return __popc(x); }
template <>
__device__ __forceinline__ int popc<uint64_t>(uint64_t x) { return __popcll(x); }

// Bits [0, q) set; q in [0, 8*sizeof(W)].
template <typename W>
__device__ __forceinline__ W low_mask(int q)
{
    return q >= (int)(8 * sizeof(W)) ? ~W(0) : ((W(1) << q) - W(1));
}

// A packed l-mer: NB bit planes of one word each.
template <int NB, typename W>
struct alignas(NB == 2 ? 2 * sizeof(W) : sizeof(W)) Lm {
    W p[NB];
};

// Positions where a and b differ (the XOR of the compressed l-mers, Section 2.1).
template <int NB, typename W>
__device__ __forceinline__ W diff(const Lm<NB, W> &a, const Lm<NB, W> &b)
{
    W x = a.p[0] ^ b.p[0];
#pragma unroll
    for (int i = 1; i < NB; i++)
        x |= a.p[i] ^ b.p[i];
    return x;
}

template <int NB, typename W>
__device__ __forceinline__ void set_letter(Lm<NB, W> &M, int pos, int code)
{
#pragma unroll
    for (int b = 0; b < NB; b++) {
        W bit = W(1) << pos;
        M.p[b] = (M.p[b] & ~bit) | (((code >> b) & 1) ? bit : W(0));
    }
}

template <int NB, typename W>
__device__ __forceinline__ int get_letter(const Lm<NB, W> &M, int pos)
{
    int c = 0;
#pragma unroll
    for (int b = 0; b < NB; b++)
        c |= (int)((M.p[b] >> pos) & 1) << b;
    return c;
}

template <int NB, typename W>
__device__ __forceinline__ Lm<NB, W> shfl_lm(const Lm<NB, W> &v, int src)
{
    Lm<NB, W> o;
#pragma unroll
    for (int b = 0; b < NB; b++)
        o.p[b] = __shfl_sync(kFull, v.p[b], src);
    return o;
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Index of the instance owning global element g, given ascending per-instance offsets.
template <typename F>
__device__ __forceinline__ int find_inst(int ninst, uint64_t g, F off)
{
    int lo = 0, hi = ninst - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off(mid) <= g)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// ------------------------------------------------------------------------------- pack

template <int NB, typename W>
__global__ void pack_kernel(const InstDesc *__restrict__ inst, int ninst, uint64_t total,
                            const uint8_t *__restrict__ seqs, const uint8_t *__restrict__ maps,
                            Lm<NB, W> *__restrict__ out, int *status)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += stride) {
        int ii = find_inst(ninst, g, [&](int i) { return inst[i].lmer_off; });
        const InstDesc I = inst[ii];
        uint64_t loc = g - I.lmer_off;
        int r = (int)(loc / (uint64_t)I.L);
        int j = (int)(loc % (uint64_t)I.L);
        const uint8_t *s = seqs + I.seq_off + (uint64_t)r * I.m + j;
        const uint8_t *map = maps + 256 * (size_t)ii;
        Lm<NB, W> v;
#pragma unroll
        for (int b = 0; b < NB; b++)
            v.p[b] = 0;
        int bad = 0;
        for (int p = 0; p < I.l; p++) {
            int c = map[s[p]];
            bad |= (c == 0xFF);
#pragma unroll
            for (int b = 0; b < NB; b++)
                v.p[b] |= (W)((c >> b) & 1) << p;
        }
        if (bad)
            atomicOr(status, kErrAlphabet);
        out[g] = v;
    }
}

// ------------------------------------------------------------------------------ items

// One warp per x of S_1: count, for every other string, the l-mers within 2d of x
// (Section 2, first filter); if none is empty, the smallest row (Section 2.1) becomes
// the branch row b and every compatible u of it becomes an item (x, b, u).
template <int NB, typename W>
__global__ void items_kernel(const InstDesc *__restrict__ inst, int ninst, uint64_t total_x,
                             const Lm<NB, W> *__restrict__ lmers, Item *__restrict__ items,
                             unsigned long long *item_count, uint64_t item_cap, int *status,
                             DevStats *stats)
{
    const int lane = threadIdx.x & 31;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long compares = 0;
    for (uint64_t g = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < total_x;
         g += nwarps) {
        int ii = find_inst(ninst, g, [&](int i) { return inst[i].x_off; });
        const InstDesc I = inst[ii];
        const int x = I.x_begin + (int)(g - I.x_off);
        const Lm<NB, W> *lm = lmers + I.lmer_off;
        const Lm<NB, W> xv = lm[x];
        if (I.n == 1) {
            if (lane == 0) {
                unsigned long long pos = atomicAdd(item_count, 1ull);
                if (pos < item_cap)
                    items[pos] = Item{(uint32_t)ii, (uint16_t)x, 0, 0xFFFF, 0};
                else
                    atomicOr(status, kErrItemsOverflow);
            }
            continue;
        }
        const int two_d = 2 * I.d;
        int best = INT_MAX, brow = -1;
        bool dead = false;
        for (int r = 1; r < I.n && !dead; r++) {
            int c = 0;
            for (int j0 = 0; j0 < I.L; j0 += 32) {
                int j = j0 + lane;
                bool ok = j < I.L && popc(diff(xv, lm[(size_t)r * I.L + j])) <= two_d;
                c += __popc(__ballot_sync(kFull, ok));
            }
            compares += I.L;
            if (c == 0)
                dead = true;
            else if (c < best) {
                best = c;
                brow = r;
            }
        }
        if (dead)
            continue;
        for (int j0 = 0; j0 < I.L; j0 += 32) {
            int j = j0 + lane;
            bool ok = j < I.L && popc(diff(xv, lm[(size_t)brow * I.L + j])) <= two_d;
            unsigned bal = __ballot_sync(kFull, ok);
            if (!bal)
                continue;
            unsigned long long base = 0;
            if (lane == 0)
                base = atomicAdd(item_count, (unsigned long long)__popc(bal));
            base = __shfl_sync(kFull, base, 0);
            if (ok) {
                unsigned long long pos = base + __popc(bal & lanemask_lt());
                if (pos < item_cap)
                    items[pos] = Item{(uint32_t)ii, (uint16_t)x, (uint16_t)j, (uint16_t)brow, 0};
                else
                    atomicOr(status, kErrItemsOverflow);
            }
        }
    }
    if (lane == 0 && compares)
        atomicAdd(&stats->hd_compares, compares);
}

// ----------------------------------------------------------------------------- search

// Per-warp shared state of the stack search.  Level k = stack size k: the rows not yet
// on the stack, each a segment [start, start+cnt) of the level's compacted list of
// entries (row << 16 | position).
template <int NB, typename W>
struct WarpSm {
    Lm<NB, W> stk[kTMax];
    Lm<NB, W> cand[kCandBuf];
    uint64_t live[kTMax + 1];
    int len[kTMax + 1];
    int brow[kTMax + 1];
    int bpos[kTMax + 1];
    int start[kTMax + 1][kRMax];
    int cnt[kTMax + 1][kRMax];
};

struct WarpCounters {
    unsigned long long tuples = 0, compares = 0, nodes = 0, leaves = 0, motifs = 0;
};

template <int NB, typename W>
struct SearchCtx {
    const InstDesc *I;
    int inst;
    const Lm<NB, W> *lm;      // this instance's l-mer table
    uint32_t *lists;          // this warp's lists, level k at (k-2)*list_cap
    uint64_t list_cap;
    uint64_t *keys;
    unsigned long long *key_count;
    uint64_t key_cap;
    int *status;
    int key_shift;            // bit position of the instance id in the key
    int multi;                // batch holds more than one instance
};

// Row with the fewest survivors at level k (Section 2.1 "Sort rows by size": the next
// stack element comes from the smallest row).  Ties go to the lower string index.
template <int NB, typename W>
__device__ __forceinline__ int choose_branch(WarpSm<NB, W> &S, int k, int lane)
{
    uint64_t live = S.live[k];
    unsigned a = ((live >> lane) & 1) ? ((unsigned)S.cnt[k][lane] << 6 | lane) : 0xFFFFFFFFu;
    unsigned b = ((live >> (lane + 32)) & 1) ? ((unsigned)S.cnt[k][lane + 32] << 6 | (lane + 32))
                                             : 0xFFFFFFFFu;
    unsigned m = __reduce_min_sync(kFull, a < b ? a : b);
    return (int)(m & 63);
}

// Segment starts of level k from its per-row counts (rows keep ascending string order).
template <int NB, typename W>
__device__ __forceinline__ void row_starts(WarpSm<NB, W> &S, int k, int lane)
{
    uint64_t live = S.live[k];
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
template <int NB, typename W>
__device__ bool build_level2(WarpSm<NB, W> &S, const SearchCtx<NB, W> &C, int b, int lane,
                             WarpCounters &wc)
{
    const InstDesc &I = *C.I;
    const Lm<NB, W> x = S.stk[0], u = S.stk[1];
    const W dxu = diff(x, u);
    const int two_d = 2 * I.d, three_d = 3 * I.d;
    uint32_t *out = C.lists;
    int len = 0;
    uint64_t live = 0;
    for (int r = 1; r < I.n; r++) {
        if (r == b)
            continue;
        const int s0 = len;
        const Lm<NB, W> *row = C.lm + (size_t)r * I.L;
        for (int j0 = 0; j0 < I.L; j0 += 32) {
            int j = j0 + lane;
            bool ok = false;
            if (j < I.L) {
                Lm<NB, W> v = row[j];
                W dxv = diff(x, v), duv = diff(u, v);
                ok = popc(dxv) <= two_d && popc(duv) <= two_d &&
                     popc(dxu | dxv) + popc(dxu & dxv & duv) <= three_d;
            }
            unsigned bal = __ballot_sync(kFull, ok);
            if (ok)
                out[len + __popc(bal & lanemask_lt())] = ((uint32_t)r << 16) | (uint32_t)j;
            len += __popc(bal);
        }
        wc.compares += 3ull * I.L;
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

// Push the l-mer stk[k] (stack size becomes k+1) and filter the rows of level k other
// than the branch row into level k+1: v survives when Hd(top,v) <= 2d and, for every
// earlier stack l-mer s, Cd(s, top, v) <= 3d (Theorem 1 with budgets d,d,d; the pair
// conditions with earlier l-mers hold from earlier levels).  Returns false as soon as a
// row empties (Section 2: "If any row becomes empty ... try a different l-mer").
template <int NB, typename W>
__device__ bool filter_level(WarpSm<NB, W> &S, const SearchCtx<NB, W> &C, int k, int lane,
                             WarpCounters &wc)
{
    const InstDesc &I = *C.I;
    const int two_d = 2 * I.d, three_d = 3 * I.d;
    const Lm<NB, W> top = S.stk[k];
    Lm<NB, W> st[kTMax];
    W dst[kTMax];
#pragma unroll
    for (int i = 0; i < kTMax; i++) {
        if (i < k) {
            st[i] = S.stk[i];
            dst[i] = diff(st[i], top);
        }
    }
    const uint32_t *in = C.lists + (size_t)(k - 2) * C.list_cap;
    uint32_t *out = C.lists + (size_t)(k - 1) * C.list_cap;
    const int br = S.brow[k];
    const int bs = S.start[k][br], bc = S.cnt[k][br];
    const int total = S.len[k] - bc;
    const uint64_t live1 = S.live[k] & ~(1ull << br);
    S.cnt[k + 1][lane] = 0;
    S.cnt[k + 1][lane + 32] = 0;
    __syncwarp();
    int len = 0;
    for (int c0 = 0; c0 < total; c0 += 32) {
        const int vi = c0 + lane;
        const bool valid = vi < total;
        const int idx = vi < bs ? vi : vi + bc;
        bool ok = false;
        int row = -1;
        uint32_t e = 0;
        if (valid) {
            e = in[idx];
            row = (int)(e >> 16);
            Lm<NB, W> v = C.lm[(size_t)row * I.L + (e & 0xFFFF)];
            W dtv = diff(top, v);
            ok = popc(dtv) <= two_d;
#pragma unroll
            for (int i = 0; i < kTMax; i++) {
                if (i < k) {
                    W div = diff(st[i], v);
                    ok = ok && (popc(dst[i] | div) + popc(dst[i] & div & dtv) <= three_d);
                }
            }
        }
        unsigned bal = __ballot_sync(kFull, ok);
        if (ok)
            out[len + __popc(bal & lanemask_lt())] = e;
        len += __popc(bal);
        unsigned grp = __match_any_sync(kFull, row);
        if (valid && lane == __ffs(grp) - 1)
            S.cnt[k + 1][row] += __popc(grp & bal);
        __syncwarp();
        bool last = valid && idx == S.start[k][row] + S.cnt[k][row] - 1;
        if (__any_sync(kFull, last && S.cnt[k + 1][row] == 0)) {
            wc.compares += (unsigned long long)(c0 + 32) * (k + 1);
            return false;
        }
    }
    wc.compares += (unsigned long long)total * (k + 1);
    if (lane == 0) {
        S.len[k + 1] = len;
        S.live[k + 1] = live1;
    }
    __syncwarp();
    row_starts(S, k + 1, lane);
    return true;
}

// prune(T, r) of Algorithm 1 for a prefix of length q (positions [0, q) fixed in M):
// every budget r_i = d - Hd(M[0..q), T_i[0..q)) stays >= 0, every pair keeps
// Hd(T_i[q..], T_j[q..]) <= r_i + r_j (two-l-mer condition, Section 2.4), and every
// triple keeps Cd(T_i[q..], T_j[q..], T_h[q..]) <= r_i + r_j + r_h (Lemma 1; with the
// pair conditions this is Theorem 1, exact for three l-mers).
template <int NB, typename W>
__device__ __forceinline__ bool node_ok(const Lm<NB, W> &M, int q, int k, int d, W lmask,
                                        const Lm<NB, W> (&st)[kTMax],
                                        const W (&dp)[kTMax][kTMax])
{
    const W pre = low_mask<W>(q);
    const W suf = lmask & ~pre;
    int e[kTMax];
    bool ok = true;
#pragma unroll
    for (int i = 0; i < kTMax; i++) {
        if (i < k) {
            e[i] = popc(diff(M, st[i]) & pre);
            ok = ok && e[i] <= d;
        }
    }
    if (!ok)
        return false;
#pragma unroll
    for (int i = 0; i < kTMax; i++) {
#pragma unroll
        for (int j = i + 1; j < kTMax; j++) {
            if (j < k)
                ok = ok && (e[i] + e[j] + popc(dp[i][j] & suf) <= 2 * d);
        }
    }
    if (!ok)
        return false;
#pragma unroll
    for (int i = 0; i < kTMax; i++) {
#pragma unroll
        for (int j = i + 1; j < kTMax; j++) {
#pragma unroll
            for (int h = j + 1; h < kTMax; h++) {
                if (h < k) {
                    W a = dp[i][j], b = dp[i][h], c = dp[j][h];
                    int cd = popc((a | b) & suf) + popc(a & b & c & suf);
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
        uint64_t c = (uint64_t)get_letter(M, p);
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

// isMotif(M, R') of Algorithm 2 for up to 32 buffered leaves (one per lane): every row
// still on level k must hold an l-mer within d of M.  Rows on the stack are satisfied by
// construction, and an l-mer within d of a common neighbour of the stack survives every
// necessary filter, so scanning the level-k lists equals scanning the whole strings.
template <int NB, typename W>
__device__ void verify_and_emit(WarpSm<NB, W> &S, const SearchCtx<NB, W> &C, int k, int ncand,
                                int lane, WarpCounters &wc)
{
    const InstDesc &I = *C.I;
    Lm<NB, W> M = S.cand[lane < ncand ? lane : 0];
    bool alive = lane < ncand;
    const uint32_t *list = k >= 2 ? C.lists + (size_t)(k - 2) * C.list_cap : C.lists;
    uint64_t rows = S.live[k];
    while (rows && __any_sync(kFull, alive)) {
        const int r = __ffsll((long long)rows) - 1;
        rows &= rows - 1;
        const int s0 = S.start[k][r], c = S.cnt[k][r];
        const Lm<NB, W> *row = C.lm + (size_t)r * I.L;
        bool hit = false;
        const int nalive = __popc(__ballot_sync(kFull, alive));
        for (int j0 = 0; j0 < c; j0 += 32) {
            Lm<NB, W> vj;
            if (j0 + lane < c)
                vj = row[list[s0 + j0 + lane] & 0xFFFF];
            else
                vj = row[0];
            const int jn = c - j0 < 32 ? c - j0 : 32;
            for (int jj = 0; jj < jn; jj++) {
                Lm<NB, W> v = shfl_lm(vj, jj);
                hit = hit || popc(diff(M, v)) <= I.d;
            }
            wc.compares += (unsigned long long)jn * nalive;
            if (__all_sync(kFull, hit || !alive))
                break;
        }
        alive = alive && hit;
    }
    unsigned bal = __ballot_sync(kFull, alive);
    if (!bal)
        return;
    unsigned long long base = 0;
    if (lane == 0)
        base = atomicAdd(C.key_count, (unsigned long long)__popc(bal));
    base = __shfl_sync(kFull, base, 0);
    wc.motifs += __popc(bal);
    if (alive) {
        unsigned long long pos = base + __popc(bal & lanemask_lt());
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

// GenerateNeighborhood (Algorithm 1) for the k l-mers on the stack, followed by isMotif
// on every leaf.  The tree is cut into K^P subtrees by the letters of the first P
// positions (K^P >= 32 when l allows); lanes take subtrees round-robin and walk each
// depth first, testing one child per step.
template <int NB, typename W>
__device__ void enumerate_stack(WarpSm<NB, W> &S, const SearchCtx<NB, W> &C, int k, int lane,
                                WarpCounters &wc)
{
    const InstDesc &I = *C.I;
    const int l = I.l, d = I.d, K = I.k;
    const W lmask = low_mask<W>(l);
    Lm<NB, W> st[kTMax];
    W dp[kTMax][kTMax];
#pragma unroll
    for (int i = 0; i < kTMax; i++)
        if (i < k)
            st[i] = S.stk[i];
#pragma unroll
    for (int i = 0; i < kTMax; i++)
#pragma unroll
        for (int j = i + 1; j < kTMax; j++)
            if (j < k)
                dp[i][j] = diff(st[i], st[j]);

    int P = 0, U = 1;
    while (P < l && U < 32) {
        P++;
        U *= K;
    }
    wc.tuples++;
    int ncand = 0;
    int unit = lane - 32;
    bool have = false;
    int q = 0, a = 0;
    Lm<NB, W> M;
#pragma unroll
    for (int b = 0; b < NB; b++)
        M.p[b] = 0;
    unsigned long long nodes = 0;
    for (;;) {
        bool leaf = false;
        if (!have) {
            unit += 32;
            if (unit < U) {
                int code = unit;
                for (int p = P - 1; p >= 0; p--) {
                    set_letter(M, p, code % K);
                    code /= K;
                }
                nodes++;
                if (node_ok(M, P, k, d, lmask, st, dp)) {
                    if (P == l)
                        leaf = true;
                    else {
                        have = true;
                        q = P;
                        a = 0;
                    }
                }
            }
        } else if (a < K) {
            set_letter(M, q, a);
            a++;
            nodes++;
            if (node_ok(M, q + 1, k, d, lmask, st, dp)) {
                if (q + 1 == l)
                    leaf = true;
                else {
                    q++;
                    a = 0;
                }
            }
        } else {
            q--;
            if (q < P)
                have = false;
            else
                a = get_letter(M, q) + 1;
        }
        unsigned lb = __ballot_sync(kFull, leaf);
        if (leaf)
            S.cand[ncand + __popc(lb & lanemask_lt())] = M;
        ncand += __popc(lb);
        wc.leaves += __popc(lb);
        __syncwarp();
        if (ncand >= 32) {
            verify_and_emit(S, C, k, 32, lane, wc);
            __syncwarp();
            Lm<NB, W> rest = S.cand[32 + (lane < ncand - 32 ? lane : 0)];
            __syncwarp();
            if (lane < ncand - 32)
                S.cand[lane] = rest;
            ncand -= 32;
            __syncwarp();
        }
        if (!__any_sync(kFull, have || unit + 32 < U))
            break;
    }
    if (ncand > 0)
        verify_and_emit(S, C, k, ncand, lane, wc);
    __syncwarp();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        nodes += __shfl_xor_sync(kFull, nodes, o);
    wc.nodes += nodes;
}

// One (x, u) subproblem: Algorithm 2 from stack size 2 with an explicit stack of levels.
template <int NB, typename W>
__device__ void run_item(WarpSm<NB, W> &S, SearchCtx<NB, W> &C, const Item &it, int lane,
                         WarpCounters &wc)
{
    const InstDesc &I = *C.I;
    const int t = I.t;
    if (lane == 0)
        S.stk[0] = C.lm[it.x];
    if (it.b == 0xFFFF) {  // a single string: the d-neighbourhood of x is the answer
        if (lane == 0)
            S.live[1] = 0;
        __syncwarp();
        enumerate_stack(S, C, 1, lane, wc);
        return;
    }
    if (lane == 0)
        S.stk[1] = C.lm[(size_t)it.b * I.L + it.u];
    __syncwarp();
    if (!build_level2(S, C, it.b, lane, wc))
        return;
    int k = 2;
    if (k < t && S.live[2] != 0) {
        int br = choose_branch(S, 2, lane);
        if (lane == 0) {
            S.brow[2] = br;
            S.bpos[2] = 0;
        }
        __syncwarp();
    }
    for (;;) {
        if (k >= t || S.live[k] == 0) {
            enumerate_stack(S, C, k, lane, wc);
            if (k == 2)
                return;
            k--;
            continue;
        }
        const int br = S.brow[k];
        const int pos = S.bpos[k];
        if (pos >= S.cnt[k][br]) {
            if (k == 2)
                return;
            k--;
            continue;
        }
        const uint32_t *in = C.lists + (size_t)(k - 2) * C.list_cap;
        const uint32_t e = in[S.start[k][br] + pos];
        __syncwarp();
        if (lane == 0) {
            S.bpos[k] = pos + 1;
            S.stk[k] = C.lm[(size_t)(e >> 16) * I.L + (e & 0xFFFF)];
        }
        __syncwarp();
        if (!filter_level(S, C, k, lane, wc))
            continue;
        k++;
        if (k < t && S.live[k] != 0) {
            int nb = choose_branch(S, k, lane);
            if (lane == 0) {
                S.brow[k] = nb;
                S.bpos[k] = 0;
            }
        }
        __syncwarp();
    }
}

template <int NB, typename W>
__global__ void __launch_bounds__(128) search_kernel(
    const InstDesc *__restrict__ inst, const Lm<NB, W> *__restrict__ lmers,
    const Item *__restrict__ items, const unsigned long long *item_count, uint64_t item_cap,
    unsigned long long *item_next, uint32_t *lists, uint64_t list_cap, uint64_t *keys,
    unsigned long long *key_count, uint64_t key_cap, int *status, DevStats *stats,
    int key_shift, int multi, int levels)
{
    extern __shared__ unsigned char smem_raw[];
    WarpSm<NB, W> &S = reinterpret_cast<WarpSm<NB, W> *>(smem_raw)[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    SearchCtx<NB, W> C;
    C.lists = lists + gw * (uint64_t)levels * list_cap;
    C.list_cap = list_cap;
    C.keys = keys;
    C.key_count = key_count;
    C.key_cap = key_cap;
    C.status = status;
    C.key_shift = key_shift;
    C.multi = multi;
    WarpCounters wc;
    unsigned long long done = 0;
    const unsigned long long nitems = *item_count < item_cap ? *item_count : item_cap;
    for (;;) {
        unsigned long long it = 0;
        if (lane == 0)
            it = atomicAdd(item_next, 1ull);
        it = __shfl_sync(kFull, it, 0);
        if (it >= nitems)
            break;
        const Item item = items[it];
        C.I = inst + item.inst;
        C.inst = (int)item.inst;
        C.lm = lmers + C.I->lmer_off;
        run_item(S, C, item, lane, wc);
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
    }
}

template <int NB, typename W>
cudaError_t pack_t(const InstDesc *d_inst, int ninst, uint64_t total, const uint8_t *d_seqs,
                   const uint8_t *d_maps, void *d_lmers, int *d_status, cudaStream_t s)
{
    if (total == 0)
        return cudaSuccess;
    uint64_t blocks = (total + 255) / 256;
    if (blocks > 65535ull * 16)
        blocks = 65535ull * 16;
    pack_kernel<NB, W><<<(unsigned)blocks, 256, 0, s>>>(
        d_inst, ninst, total, d_seqs, d_maps, static_cast<Lm<NB, W> *>(d_lmers), d_status);
    return cudaGetLastError();
}

template <int NB, typename W>
cudaError_t items_t(const InstDesc *d_inst, int ninst, uint64_t total_x, const void *d_lmers,
                    Item *d_items, unsigned long long *d_item_count, uint64_t item_cap,
                    int *d_status, DevStats *d_stats, cudaStream_t s)
{
    if (total_x == 0)
        return cudaSuccess;
    uint64_t warps = total_x;
    uint64_t blocks = (warps + 7) / 8;
    if (blocks > 65535ull * 16)
        blocks = 65535ull * 16;
    items_kernel<NB, W><<<(unsigned)blocks, 256, 0, s>>>(
        d_inst, ninst, total_x, static_cast<const Lm<NB, W> *>(d_lmers), d_items, d_item_count,
        item_cap, d_status, d_stats);
    return cudaGetLastError();
}

template <int NB, typename W>
size_t smem_t(int wpb)
{
    return sizeof(WarpSm<NB, W>) * (size_t)wpb;
}

template <int NB, typename W>
cudaError_t search_t(const InstDesc *d_inst, const void *d_lmers, const Item *d_items,
                     const unsigned long long *d_item_count, uint64_t item_cap,
                     unsigned long long *d_item_next,
                     uint32_t *d_lists, uint64_t list_cap, uint64_t *d_keys,
                     unsigned long long *d_key_count, uint64_t key_cap, int *d_status,
                     DevStats *d_stats, const LaunchCfg &cfg, int key_shift, int multi,
                     int levels, cudaStream_t s)
{
    size_t smem = smem_t<NB, W>(cfg.warps_per_block);
    cudaError_t e = cudaFuncSetAttribute(search_kernel<NB, W>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    search_kernel<NB, W><<<cfg.blocks, cfg.warps_per_block * 32, smem, s>>>(
        d_inst, static_cast<const Lm<NB, W> *>(d_lmers), d_items, d_item_count, item_cap,
        d_item_next, d_lists, list_cap, d_keys, d_key_count, key_cap, d_status, d_stats, key_shift, multi,
        levels);
    return cudaGetLastError();
}

template <int NB, typename W>
int max_blocks_t(int wpb)
{
    int nb = 0;
    size_t smem = smem_t<NB, W>(wpb);
    cudaFuncSetAttribute(search_kernel<NB, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, search_kernel<NB, W>, wpb * 32,
                                                      smem) != cudaSuccess)
        return 0;
    return nb;
}

}  // namespace

#define PMS_DISPATCH(lay, CALL)                                  \
    switch (lay) {                                               \
    case Layout::DNA32: { constexpr int NB = 2; using W = uint32_t; return CALL; } \
    case Layout::DNA64: { constexpr int NB = 2; using W = uint64_t; return CALL; } \
    case Layout::P5_32: { constexpr int NB = 5; using W = uint32_t; return CALL; } \
    case Layout::P5_64: { constexpr int NB = 5; using W = uint64_t; return CALL; } \
    }

cudaError_t launch_pack(Layout lay, const InstDesc *d_inst, const uint64_t *, int ninst,
                        uint64_t total_lmers, const uint8_t *d_seqs, const uint8_t *d_maps,
                        void *d_lmers, int *d_status, cudaStream_t s)
{
    PMS_DISPATCH(lay, (pack_t<NB, W>(d_inst, ninst, total_lmers, d_seqs, d_maps, d_lmers,
                                     d_status, s)));
    return cudaErrorInvalidValue;
}

cudaError_t launch_items(Layout lay, const InstDesc *d_inst, const uint64_t *, int ninst,
                         uint64_t total_x, const void *d_lmers, Item *d_items,
                         unsigned long long *d_item_count, uint64_t item_cap, int *d_status,
                         DevStats *d_stats, cudaStream_t s)
{
    PMS_DISPATCH(lay, (items_t<NB, W>(d_inst, ninst, total_x, d_lmers, d_items, d_item_count,
                                      item_cap, d_status, d_stats, s)));
    return cudaErrorInvalidValue;
}

cudaError_t launch_search(Layout lay, const InstDesc *d_inst, const void *d_lmers,
                          const Item *d_items, const unsigned long long *d_item_count,
                          uint64_t item_cap, unsigned long long *d_item_next, uint32_t *d_lists,
                          uint64_t list_cap,
                          uint64_t *d_keys, unsigned long long *d_key_count, uint64_t key_cap,
                          int *d_status, DevStats *d_stats, const LaunchCfg &cfg,
                          int key_shift, int multi, int levels, cudaStream_t s)
{
    PMS_DISPATCH(lay, (search_t<NB, W>(d_inst, d_lmers, d_items, d_item_count, item_cap,
                                       d_item_next,
                                       d_lists, list_cap, d_keys, d_key_count, key_cap,
                                       d_status, d_stats, cfg, key_shift, multi, levels, s)));
    return cudaErrorInvalidValue;
}

int search_max_blocks(Layout lay, int warps_per_block)
{
    PMS_DISPATCH(lay, (max_blocks_t<NB, W>(warps_per_block)));
    return 0;
}

size_t search_smem_bytes(Layout lay, int warps_per_block)
{
    PMS_DISPATCH(lay, (smem_t<NB, W>(warps_per_block)));
    return 0;
}

}  // namespace pms
