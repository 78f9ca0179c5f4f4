// pms_solve_device_noalloc: the device-resident solve without any device allocation.
//
// Some callers cannot allocate device memory once they are running: a service that
// reserves all of its device memory in its own pool at start-up (so a later cudaMalloc
// either fails or breaks its budget), or a real-time pipeline where cudaMalloc/cudaFree
// would stall the device and fragment memory in the middle of a frame.  This entry point
// gives them the same solve as pms_solve_device using only a fixed scratch array that
// lives in this library's device image (it is created when the library is loaded on a
// device and stays until the process exits).  The caller still provides the input
// strings and the output buffer in device memory.
//
// The kernels are the same ones the other entry points launch; only the places their
// working memory comes from differ.  No context, stream, event or buffer is created.
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>

#include "pms.h"
#include "pms_internal.h"

using namespace pms;

namespace {

// Size of the fixed scratch array (bytes).
constexpr size_t kNoAllocScratch = 64ull << 20;
// Largest raw (not yet de-duplicated) motif list the scratch holds.
constexpr uint64_t kNoAllocRawKeys = 1ull << 18;

// The scratch: every call of the entry point on a device shares it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratch];

std::mutex g_noalloc_mu;
void *g_noalloc_addr[256];   // device address of the array, per device ordinal

// The array's name in host code is only a stand-in for the symbol; kernels need its device
// address, which is looked up once per device (with that device current).
int noalloc_scratch(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= 256)
        return PMS_E_CUDA;
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return PMS_E_CUDA;
        }
        g_noalloc_addr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_noalloc_addr[dev]);
    return PMS_OK;
}

size_t na_lmer_bytes(Layout lay)
{
    switch (lay) {
    case Layout::DNA32: return 8;
    case Layout::DNA64: return 16;
    case Layout::P5_32: return 20;
    case Layout::P5_64: return 40;
    }
    return 40;
}

double na_nbhd(int l, int d, int k)
{
    double s = 0, c = 1;
    for (int i = 0; i <= (d < l ? d : l); i++) {
        s += c * std::pow((double)(k - 1), i);
        c = c * (l - i) / (i + 1);
    }
    return s;
}

// The threshold of the Appendix D cost model (the autotuner's starting point).
int na_model_threshold(int n, int m, int l, int d, int k)
{
    const double L = m - l + 1;
    const double nd = na_nbhd(l, d, k), n2d = na_nbhd(l, 2 * d, k);
    const double p = std::fmin(1.0, n2d / std::pow((double)k, l));
    const double q = std::fmin(1.0, nd / std::fmax(n2d, 1.0));
    int best = 2;
    double best_cost = INFINITY;
    for (int t = 2; t <= (n < kTMax ? n : kTMax); t++) {
        double ts = 0;
        for (int j = 1; j <= t; j++)
            ts += std::pow(L, j) * std::pow(p, j * (j - 1) / 2.0);
        ts *= (double)n * l;
        const double tp =
            std::pow(L, t) * std::pow(p, t * (t - 1) / 2.0) * nd * std::pow(q, t - 1) * l;
        if (ts + tp < best_cost) {
            best_cost = ts + tp;
            best = t;
        }
    }
    return best;
}

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

#define NA_CU(call)                                \
    do {                                           \
        if ((call) != cudaSuccess) {               \
            cudaGetLastError();                    \
            return PMS_E_CUDA;                     \
        }                                          \
    } while (0)

struct NaCounters {
    unsigned long long item_count;
    unsigned long long item_next;
    unsigned long long key_count;
    unsigned long long uniq_total;
    int status;
    int pad;
    DevStats stats;
};

int solve_noalloc(const char *d_seqs, int n, int m, const char *alphabet, int l, int d,
                  int threshold, char *d_motifs, uint64_t cap, uint64_t *count, void *stream)
{
    if (!d_seqs || !alphabet || !count || (!d_motifs && cap))
        return PMS_E_INVAL;
    const size_t k = strnlen(alphabet, 64);
    if (k < 2 || k > 32)
        return PMS_E_INVAL;
    bool seen[256] = {false};
    for (size_t i = 0; i < k; i++) {
        if (seen[(unsigned char)alphabet[i]])
            return PMS_E_INVAL;
        seen[(unsigned char)alphabet[i]] = true;
    }
    if (n < 1 || n > kRMax || l < 1 || m < l || d < 0 || l > 64 || m - l + 1 > 65535)
        return PMS_E_INVAL;
    const int kbits = k <= 4 ? 2 : 5;
    if (l * kbits > 128 || (threshold && (threshold < 2 || threshold > kTMax)))
        return PMS_E_INVAL;
    const int L = m - l + 1;
    const Layout lay = kbits == 2 ? (l <= 32 ? Layout::DNA32 : Layout::DNA64)
                                  : (l <= 32 ? Layout::P5_32 : Layout::P5_64);
    int t = threshold ? threshold : na_model_threshold(n, m, l, d, (int)k);
    if (d > 41 && t < 5)
        t = 5;   // thresholds 2..4 keep budgets in bytes

    int dev = 0;
    NA_CU(cudaGetDevice(&dev));
    int sms = 0;
    NA_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    std::lock_guard<std::mutex> guard(g_noalloc_mu);
    unsigned char *base = nullptr;
    int rc = noalloc_scratch(dev, &base);
    if (rc != PMS_OK)
        return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    // carve the array: fixed regions first, then per-warp search scratch
    const uint64_t nlmers = (uint64_t)n * L;
    const uint64_t item_cap = (uint64_t)L * (n > 1 ? (uint64_t)L : 1);
    const uint64_t list_cap = (uint64_t)(n > 1 ? n - 1 : 1) * L;
    const uint64_t ntiles_max = (kNoAllocRawKeys + kSortTile - 1) / kSortTile;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off += up256(bytes);
        return at;
    };
    const size_t o_cnt = take(sizeof(NaCounters));
    const size_t o_inst = take(sizeof(InstDesc));
    const size_t o_maps = take(256);
    const size_t o_alpha = take(32);
    const size_t o_first = take(8), o_last = take(8), o_boff = take(8);
    const size_t o_lmers = take(na_lmer_bytes(lay) * nlmers);
    const size_t o_items = take(sizeof(Item) * item_cap);
    const size_t o_keys = take(16 * kNoAllocRawKeys);
    const size_t o_alt = take(16 * kNoAllocRawKeys);
    const size_t o_hist = take(4 * 256 * ntiles_max);
    const size_t o_flags = take(4 * ntiles_max);
    if (off + 1024 >= kNoAllocScratch)
        return PMS_E_NOMEM;
    const uint64_t fstride = up256(search_frontier_bytes(lay, l));
    const uint64_t per_warp = (4ull + na_lmer_bytes(lay)) * search_levels(t) * list_cap + fstride;
    const int wpb = 4;
    int per_sm = search_max_blocks(lay, t, wpb);
    if (per_sm <= 0)
        return PMS_E_CUDA;
    // leave room for the 256-byte rounding of the three regions below
    uint64_t blocks = (kNoAllocScratch - off - 1024) / (per_warp * wpb);
    if (blocks > (uint64_t)per_sm * sms)
        blocks = (uint64_t)per_sm * sms;
    if (blocks < 8)
        return PMS_E_NOMEM;   // too little scratch left for a useful search grid
    const uint64_t nwarps = blocks * wpb;
    const size_t o_lists = take(4ull * nwarps * search_levels(t) * list_cap);
    const size_t o_planes = take(na_lmer_bytes(lay) * nwarps * search_levels(t) * list_cap);
    const size_t o_fscr = take(fstride * nwarps);
    if (off > kNoAllocScratch)
        return PMS_E_NOMEM;

    NaCounters *dc = reinterpret_cast<NaCounters *>(base + o_cnt);
    InstDesc desc{};
    desc.n = n;
    desc.m = m;
    desc.l = l;
    desc.d = d;
    desc.L = L;
    desc.k = (int)k;
    desc.kbits = kbits;
    desc.t = t;
    desc.x_begin = 0;
    desc.x_end = L;
    unsigned char maps[256], alpha[32] = {0};
    memset(maps, 0xFF, sizeof maps);
    for (size_t a = 0; a < k; a++) {
        maps[(unsigned char)alphabet[a]] = (unsigned char)a;
        alpha[a] = (unsigned char)alphabet[a];
    }
    // every call starts from cleared counters and ranges (the array keeps the last call's
    // contents)
    NA_CU(cudaMemsetAsync(dc, 0, sizeof(NaCounters), s));
    NA_CU(cudaMemcpyAsync(base + o_inst, &desc, sizeof desc, cudaMemcpyHostToDevice, s));
    NA_CU(cudaMemcpyAsync(base + o_maps, maps, sizeof maps, cudaMemcpyHostToDevice, s));
    NA_CU(cudaMemcpyAsync(base + o_alpha, alpha, sizeof alpha, cudaMemcpyHostToDevice, s));
    NA_CU(cudaMemsetAsync(base + o_first, 0xFF, 8, s));
    NA_CU(cudaMemsetAsync(base + o_last, 0xFF, 8, s));
    const InstDesc *d_inst = reinterpret_cast<const InstDesc *>(base + o_inst);
    NA_CU(launch_pack(lay, d_inst, nullptr, 1, nlmers, reinterpret_cast<const uint8_t *>(d_seqs),
                      base + o_maps, base + o_lmers, &dc->status, s));
    NA_CU(launch_items(lay, d_inst, nullptr, 1, (uint64_t)L, base + o_lmers,
                       reinterpret_cast<Item *>(base + o_items), &dc->item_count, item_cap,
                       &dc->status, &dc->stats, s));
    SearchArgs sa{d_inst, base + o_lmers, reinterpret_cast<Item *>(base + o_items),
                  &dc->item_count, item_cap, &dc->item_next,
                  reinterpret_cast<uint32_t *>(base + o_lists), list_cap,
                  reinterpret_cast<uint64_t *>(base + o_keys), &dc->key_count, kNoAllocRawKeys,
                  &dc->status, &dc->stats, l * kbits, 0,
                  LaunchCfg{wpb, (int)blocks}, base + o_fscr, fstride, l, 1, nullptr, nullptr,
                  0, 0, nullptr, base + o_planes, 0};
    NA_CU(launch_search(lay, t, sa, s));
    NaCounters hc;
    NA_CU(cudaMemcpyAsync(&hc, dc, sizeof hc, cudaMemcpyDeviceToHost, s));
    NA_CU(cudaStreamSynchronize(s));
    if (hc.status & kErrAlphabet)
        return PMS_E_ALPHABET;
    if (hc.status & kErrItemsOverflow)
        return PMS_E_CUDA;
    if (hc.status & kErrKeysOverflow)
        return PMS_E_OVERFLOW;   // more raw motifs than the fixed scratch holds

    SortScratch scr{reinterpret_cast<uint64_t *>(base + o_alt),
                    reinterpret_cast<unsigned *>(base + o_hist),
                    reinterpret_cast<unsigned *>(base + o_flags), kNoAllocRawKeys, ntiles_max};
    size_t nuniq = 0;
    uint64_t *keys = reinterpret_cast<uint64_t *>(base + o_keys);
    NA_CU(sort_unique_keys(keys, hc.key_count, l * kbits, scr, &dc->uniq_total, &nuniq, s));
    *count = nuniq;
    if (nuniq > cap)
        return PMS_E_OVERFLOW;
    if (nuniq) {
        long long *first = reinterpret_cast<long long *>(base + o_first);
        NA_CU(launch_ranges(keys, nuniq, l * kbits, 0, 1, first,
                            reinterpret_cast<long long *>(base + o_last), s));
        NA_CU(cudaMemsetAsync(base + o_boff, 0, 8, s));
        NA_CU(launch_decode(keys, nuniq, l * kbits, 0, d_inst, base + o_alpha, d_motifs,
                            reinterpret_cast<const uint64_t *>(base + o_boff), first, s));
    }
    NA_CU(cudaStreamSynchronize(s));
    return PMS_OK;
}

}  // namespace

extern "C" int pms_solve_device_noalloc(const char *d_seqs, int n, int m, const char *alphabet,
                                        int l, int d, int threshold, char *d_motifs,
                                        uint64_t cap, uint64_t *count, void *stream)
{
    return solve_noalloc(d_seqs, n, m, alphabet, l, d, threshold, d_motifs, cap, count, stream);
}
