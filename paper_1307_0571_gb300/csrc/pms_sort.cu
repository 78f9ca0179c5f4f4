// Collection of the motif set: LSD radix sort of 128-bit motif keys, duplicate removal,
// per-instance ranges and decoding to letters.
//
// A motif is found once for every subproblem and every stack whose common neighbourhood
// holds it; Algorithm 2 outputs each find, and the set (sorted, each motif once) is the
// union over all subproblems (Section 2.3: the scheduler gathers every worker's motifs).
//
// Sort: 8-bit digits over only the key bits in use, one tile of kSortTile keys per block.
// Each pass is histogram -> exclusive scan (digit-major over tiles) -> stable scatter; the
// scatter ranks equal digits inside a warp with __match_any_sync and orders warps by a
// per-warp digit count, so every pass is stable.
#include <cstdint>

#include "pms_internal.h"

namespace pms {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kPerWarp = kSortTile / kWarps;   // 128 consecutive keys per warp

__device__ __forceinline__ unsigned digit_of(uint64_t hi, uint64_t lo, int shift)
{
    return shift < 64 ? (unsigned)((lo >> shift) & 0xFF) : (unsigned)((hi >> (shift - 64)) & 0xFF);
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// hist[digit * ntiles + tile] = number of keys of the tile with that digit.
__global__ void hist_kernel(const uint64_t *__restrict__ keys, size_t n, int shift,
                            unsigned *__restrict__ hist, unsigned ntiles)
{
    __shared__ unsigned h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        h[i] = 0;
    __syncthreads();
    size_t base = (size_t)blockIdx.x * kSortTile;
    for (int i = threadIdx.x; i < kSortTile; i += blockDim.x) {
        size_t g = base + i;
        if (g < n)
            atomicAdd(&h[digit_of(keys[2 * g], keys[2 * g + 1], shift)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        hist[(size_t)i * ntiles + blockIdx.x] = h[i];
}

// In-place exclusive scan of n values by one block; the grand total goes to *total.
__global__ void scan_kernel(unsigned *data, size_t n, unsigned long long *total)
{
    __shared__ unsigned long long warp_sums[32];
    __shared__ unsigned long long carry;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    if (threadIdx.x == 0)
        carry = 0;
    __syncthreads();
    for (size_t base = 0; base < n; base += blockDim.x) {
        size_t i = base + threadIdx.x;
        unsigned long long v = i < n ? data[i] : 0;
        unsigned long long s = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long t = __shfl_up_sync(kFull, s, o);
            if (lane >= o)
                s += t;
        }
        if (lane == 31)
            warp_sums[w] = s;
        __syncthreads();
        if (w == 0) {
            unsigned long long ws = lane < nw ? warp_sums[lane] : 0;
            unsigned long long wsum = ws;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                unsigned long long t = __shfl_up_sync(kFull, wsum, o);
                if (lane >= o)
                    wsum += t;
            }
            if (lane < nw)
                warp_sums[lane] = wsum - ws;
        }
        __syncthreads();
        unsigned long long excl = carry + warp_sums[w] + s - v;
        if (i < n)
            data[i] = (unsigned)excl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1)
            carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total)
        *total = carry;
}

// Stable scatter of one tile by digit.
__global__ void scatter_kernel(const uint64_t *__restrict__ src, uint64_t *__restrict__ dst,
                               size_t n, int shift, const unsigned *__restrict__ offs,
                               unsigned ntiles)
{
    __shared__ unsigned wcnt[kWarps][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kWarps * 256; i += blockDim.x)
        (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const size_t wbase = (size_t)blockIdx.x * kSortTile + (size_t)w * kPerWarp;
    for (int c = 0; c < kPerWarp; c += 32) {
        size_t g = wbase + c + lane;
        bool valid = g < n;
        unsigned dg = valid ? digit_of(src[2 * g], src[2 * g + 1], shift) : 256u + lane;
        unsigned peers = __match_any_sync(kFull, dg);
        if (valid && lane == __ffs(peers) - 1)
            wcnt[w][dg] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit: base of each warp = global offset + counts of earlier warps
    for (int dg = threadIdx.x; dg < 256; dg += blockDim.x) {
        unsigned run = offs[(size_t)dg * ntiles + blockIdx.x];
        for (int ww = 0; ww < kWarps; ww++) {
            unsigned c = wcnt[ww][dg];
            wcnt[ww][dg] = run;
            run += c;
        }
    }
    __syncthreads();
    for (int c = 0; c < kPerWarp; c += 32) {
        size_t g = wbase + c + lane;
        bool valid = g < n;
        uint64_t hi = 0, lo = 0;
        unsigned dg = 256u + lane;
        if (valid) {
            hi = src[2 * g];
            lo = src[2 * g + 1];
            dg = digit_of(hi, lo, shift);
        }
        unsigned peers = __match_any_sync(kFull, dg);
        if (valid) {
            unsigned pos = wcnt[w][dg] + __popc(peers & lanemask_lt());
            dst[2 * (size_t)pos] = hi;
            dst[2 * (size_t)pos + 1] = lo;
        }
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1)
            wcnt[w][dg] += __popc(peers);
        __syncwarp();
    }
}

__device__ __forceinline__ bool is_head(const uint64_t *k, size_t g)
{
    return g == 0 || k[2 * g] != k[2 * g - 2] || k[2 * g + 1] != k[2 * g - 1];
}

// counts[tile] = number of first-of-a-run keys in the tile.
__global__ void head_count_kernel(const uint64_t *__restrict__ keys, size_t n,
                                  unsigned *__restrict__ counts)
{
    __shared__ unsigned c;
    if (threadIdx.x == 0)
        c = 0;
    __syncthreads();
    size_t base = (size_t)blockIdx.x * kSortTile;
    unsigned mine = 0;
    for (int i = threadIdx.x; i < kSortTile; i += blockDim.x) {
        size_t g = base + i;
        if (g < n && is_head(keys, g))
            mine++;
    }
    atomicAdd(&c, mine);
    __syncthreads();
    if (threadIdx.x == 0)
        counts[blockIdx.x] = c;
}

// Stable compaction of the run heads.
__global__ void head_compact_kernel(const uint64_t *__restrict__ src, uint64_t *__restrict__ dst,
                                    size_t n, const unsigned *__restrict__ offs)
{
    __shared__ unsigned wc[kWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const size_t wbase = (size_t)blockIdx.x * kSortTile + (size_t)w * kPerWarp;
    unsigned mine = 0;
    for (int c = 0; c < kPerWarp; c += 32) {
        size_t g = wbase + c + lane;
        mine += __popc(__ballot_sync(kFull, g < n && is_head(src, g)));
    }
    if (lane == 0)
        wc[w] = mine;
    __syncthreads();
    unsigned run = offs[blockIdx.x];
    for (int ww = 0; ww < w; ww++)
        run += wc[ww];
    for (int c = 0; c < kPerWarp; c += 32) {
        size_t g = wbase + c + lane;
        bool h = g < n && is_head(src, g);
        unsigned bal = __ballot_sync(kFull, h);
        if (h) {
            size_t pos = run + __popc(bal & lanemask_lt());
            dst[2 * pos] = src[2 * g];
            dst[2 * pos + 1] = src[2 * g + 1];
        }
        run += __popc(bal);
    }
}

__device__ __forceinline__ unsigned key_inst(const uint64_t *k, size_t g, int key_shift, int multi)
{
    if (!multi)
        return 0;
    uint64_t hi = k[2 * g], lo = k[2 * g + 1];
    if (key_shift >= 64)
        return (unsigned)((hi >> (key_shift - 64)) & 0xFFFF);
    uint64_t v = lo >> key_shift;
    if (key_shift > 64 - kInstBits)
        v |= hi << (64 - key_shift);
    return (unsigned)(v & 0xFFFF);
}

__global__ void ranges_kernel(const uint64_t *__restrict__ keys, size_t n, int key_shift,
                              int multi, long long *first, long long *last)
{
    for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < n;
         g += (size_t)gridDim.x * blockDim.x) {
        unsigned ii = key_inst(keys, g, key_shift, multi);
        if (g == 0 || key_inst(keys, g - 1, key_shift, multi) != ii)
            first[ii] = (long long)g;
        if (g == n - 1 || key_inst(keys, g + 1, key_shift, multi) != ii)
            last[ii] = (long long)g;
    }
}

__global__ void decode_kernel(const uint64_t *__restrict__ keys, size_t n, int key_shift,
                              int multi, const InstDesc *__restrict__ inst,
                              const uint8_t *__restrict__ alpha, char *__restrict__ out,
                              const uint64_t *__restrict__ byte_off,
                              const long long *__restrict__ first)
{
    for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < n;
         g += (size_t)gridDim.x * blockDim.x) {
        unsigned ii = key_inst(keys, g, key_shift, multi);
        const int l = inst[ii].l, kb = inst[ii].kbits;
        const uint64_t hi = keys[2 * g], lo = keys[2 * g + 1];
        char *dst = out + byte_off[ii] + (uint64_t)(g - first[ii]) * l;
        const uint64_t cm = (1ull << kb) - 1;
        for (int p = 0; p < l; p++) {
            int sh = (l - 1 - p) * kb;
            uint64_t c = sh >= 64 ? (hi >> (sh - 64)) : ((lo >> sh) | (sh ? hi << (64 - sh) : 0));
            dst[p] = (char)alpha[32 * (size_t)ii + (c & cm)];
        }
    }
}

unsigned grid_for(size_t n, int threads)
{
    size_t b = (n + threads - 1) / threads;
    if (b > 65535u * 8)
        b = 65535u * 8;
    return (unsigned)(b ? b : 1);
}

}  // namespace

cudaError_t sort_unique_keys(uint64_t *keys, size_t n, int bits, SortScratch &scr,
                             unsigned long long *d_total, size_t *n_unique, cudaStream_t s)
{
    *n_unique = 0;
    if (n == 0)
        return cudaSuccess;
    const unsigned ntiles = (unsigned)((n + kSortTile - 1) / kSortTile);
    if (n > scr.cap_keys || ntiles > scr.cap_tiles)
        return cudaErrorInvalidValue;
    uint64_t *src = keys, *dst = scr.keys_alt;
    const int passes = (bits + 7) / 8;
    cudaError_t e;
    for (int p = 0; p < passes; p++) {
        const int shift = 8 * p;
        hist_kernel<<<ntiles, kThreads, 0, s>>>(src, n, shift, scr.hist, ntiles);
        scan_kernel<<<1, 1024, 0, s>>>(scr.hist, (size_t)256 * ntiles, nullptr);
        scatter_kernel<<<ntiles, kThreads, 0, s>>>(src, dst, n, shift, scr.hist, ntiles);
        if ((e = cudaGetLastError()) != cudaSuccess)
            return e;
        uint64_t *t = src;
        src = dst;
        dst = t;
    }
    head_count_kernel<<<ntiles, kThreads, 0, s>>>(src, n, scr.flags);
    scan_kernel<<<1, 1024, 0, s>>>(scr.flags, ntiles, d_total);
    head_compact_kernel<<<ntiles, kThreads, 0, s>>>(src, dst, n, scr.flags);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    unsigned long long total = 0;
    if ((e = cudaMemcpyAsync(&total, d_total, sizeof total, cudaMemcpyDeviceToHost, s)) !=
        cudaSuccess)
        return e;
    if (dst != keys &&
        (e = cudaMemcpyAsync(keys, dst, (size_t)total * 16, cudaMemcpyDeviceToDevice, s)) !=
            cudaSuccess)
        return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess)
        return e;
    *n_unique = (size_t)total;
    return cudaSuccess;
}

cudaError_t launch_ranges(const uint64_t *d_keys, size_t n, int key_shift, int multi, int,
                          long long *d_first, long long *d_last, cudaStream_t s)
{
    if (n == 0)
        return cudaSuccess;
    ranges_kernel<<<grid_for(n, 256), 256, 0, s>>>(d_keys, n, key_shift, multi, d_first, d_last);
    return cudaGetLastError();
}

cudaError_t launch_decode(const uint64_t *d_keys, size_t n, int key_shift, int multi,
                          const InstDesc *d_inst, const uint8_t *d_alpha, char *d_out,
                          const uint64_t *d_byte_off, const long long *d_first, cudaStream_t s)
{
    if (n == 0)
        return cudaSuccess;
    decode_kernel<<<grid_for(n, 256), 256, 0, s>>>(d_keys, n, key_shift, multi, d_inst, d_alpha,
                                                   d_out, d_byte_off, d_first);
    return cudaGetLastError();
}

}  // namespace pms
