// Packing and the 2d filter of every l-mer of S_1 (the first filter of Section 2), for
// every plane layout.  The items these kernels emit feed the search kernels.
#include "pms_device.cuh"

namespace pms {
namespace {

using namespace dev;

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
                    items[pos] = Item{(uint32_t)ii, (uint16_t)x, 0, 0xFFFF, 0, kAllRange, 0, kAllRange, 0};
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
                    items[pos] = Item{(uint32_t)ii, (uint16_t)x, (uint16_t)j, (uint16_t)brow, 0,
                                      kAllRange, 0, kAllRange, 0};
                else
                    atomicOr(status, kErrItemsOverflow);
            }
        }
    }
    if (lane == 0 && compares)
        atomicAdd(&stats->hd_compares, compares);
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

}  // namespace

#define PMS_DISPATCH(lay, CALL)                                                        \
    switch (lay) {                                                                     \
    case Layout::DNA32: { constexpr int NB = 2; using W = uint32_t; return CALL; }     \
    case Layout::DNA64: { constexpr int NB = 2; using W = uint64_t; return CALL; }     \
    case Layout::P5_32: { constexpr int NB = 5; using W = uint32_t; return CALL; }     \
    case Layout::P5_64: { constexpr int NB = 5; using W = uint64_t; return CALL; }     \
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

}  // namespace pms

namespace pms {

cudaError_t launch_search_dna32(int t, const SearchArgs &a, cudaStream_t s);
cudaError_t launch_search_dna64(int t, const SearchArgs &a, cudaStream_t s);
cudaError_t launch_search_p5_32(int t, const SearchArgs &a, cudaStream_t s);
int max_blocks_dna32(int t, int wpb);
size_t fscr_dna32(int lmax);
size_t fscr_dna64(int lmax);
size_t fscr_p5_32(int lmax);
int max_blocks_dna64(int t, int wpb);
int max_blocks_p5_32(int t, int wpb);

cudaError_t launch_search(Layout lay, int t, const SearchArgs &a, cudaStream_t s)
{
    switch (lay) {
    case Layout::DNA32: return launch_search_dna32(t, a, s);
    case Layout::DNA64: return launch_search_dna64(t, a, s);
    case Layout::P5_32: return launch_search_p5_32(t, a, s);
    case Layout::P5_64: break;   // 5-bit letters fit 128-bit keys only up to l = 25
    }
    return cudaErrorInvalidValue;
}

size_t search_frontier_bytes(Layout lay, int lmax)
{
    switch (lay) {
    case Layout::DNA32: return fscr_dna32(lmax);
    case Layout::DNA64: return fscr_dna64(lmax);
    case Layout::P5_32: return fscr_p5_32(lmax);
    case Layout::P5_64: break;
    }
    return 0;
}

int search_max_blocks(Layout lay, int t, int wpb)
{
    switch (lay) {
    case Layout::DNA32: return max_blocks_dna32(t, wpb);
    case Layout::DNA64: return max_blocks_dna64(t, wpb);
    case Layout::P5_32: return max_blocks_p5_32(t, wpb);
    case Layout::P5_64: break;
    }
    return 0;
}

}  // namespace pms
