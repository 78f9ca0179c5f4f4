// Device helpers shared by the CUDA translation units of libpms: packed l-mers as bit
// planes and their distance primitives, warp utilities.
//
// Packing (Section 2.1, compressed l-mers): plane b of an l-mer holds bit b of every
// letter's code, bit p for position p.  The positions where two l-mers differ are
// OR_b(a_b XOR b_b), so Hd is one popcount per word; this replaces the paper's table of
// 2^16 precomputed group counts.
#pragma once

#include <climits>
#include <cstdint>

#include "pms_internal.h"

namespace pms {
namespace dev {

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

}  // namespace dev
}  // namespace pms
