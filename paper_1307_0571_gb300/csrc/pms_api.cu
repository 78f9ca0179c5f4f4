// C ABI of libpms (include/pms.h): contexts, device workspaces, the batch pipeline
// (pack -> 2d filter/items -> search -> sort/unique -> decode), the threshold model and
// autotuner, and the continuous-batching serving loop behind pms_submit/pms_poll.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "pms.h"
#include "pms_internal.h"

using namespace pms;

namespace {

// ------------------------------------------------------------------ device buffers

// A device buffer that grows in stream order from the context's memory pool, so growing
// one serving slot's buffers never synchronises the device under the other slots.
struct DBuf {
    void *p = nullptr;
    size_t cap = 0;
    cudaMemPool_t pool = nullptr;
    ~DBuf() { release(); }
    void release()
    {
        if (p)
            cudaFree(p);
        p = nullptr;
        cap = 0;
    }
    // Grow to at least `bytes` on stream s (contents are not kept).
    int ensure(size_t bytes, std::atomic<size_t> &held, cudaStream_t s)
    {
        if (bytes <= cap)
            return PMS_OK;
        size_t want = std::max(bytes, cap + cap / 2);
        want = (want + 255) & ~size_t(255);
        release_counted(held, s);
        if (cudaMallocFromPoolAsync(&p, want, pool, s) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            if (cudaMallocFromPoolAsync(&p, bytes, pool, s) != cudaSuccess) {
                cudaGetLastError();
                p = nullptr;
                return PMS_E_NOMEM;
            }
            want = bytes;
        }
        cap = want;
        held += cap;
        return PMS_OK;
    }
    void release_counted(std::atomic<size_t> &held, cudaStream_t s)
    {
        if (p) {
            held -= cap;
            cudaFreeAsync(p, s);
            p = nullptr;
            cap = 0;
        }
    }
    template <typename T>
    T *as() const { return static_cast<T *>(p); }
};

struct Counters {           // one device block of small counters
    unsigned long long item_count;
    unsigned long long item_next;
    unsigned long long key_count;
    unsigned long long uniq_total;
    int status;
    int pad;
    DevStats stats;
    unsigned long long donate_count[2];
};

// Items handed on per search pass (ping-pong buffers), and the time an item runs before
// it hands on the rest of its range (cycles; ~2 ms at 2 GHz).  Splitting happens only
// once a pass has handed out all its items, so it trims the tail that the heaviest items
// (100x the median) would otherwise set, without repeating work earlier in the pass.
constexpr uint64_t kDonateCap = 1u << 20;
constexpr long long kItemBudget = 4000000;
// Autotuning: an item running longer than this (cycles, ~10 ms) stops and marks the
// candidate threshold as capped.
// Cycles a tuning launch may run for the first candidate (~10 s).  Later candidates are
// capped at the best time so far; a cap below a legitimate pass (large instances such as
// (21,8), whose sample passes take seconds) would reject every candidate.
constexpr long long kTuneItemCap = 20000000000LL;
constexpr unsigned long long kTuneItemsPerWarp = 8;   // tuning sample size per search warp
constexpr double kMaxCyclesPerMs = 2.1e6;             // SM cycles per ms at the highest clock

// Everything one pipeline run needs on the device; a context owns one for blocking calls
// and one per serving slot, so slots run concurrently on their own streams.
struct Workspace {
    cudaStream_t stream = nullptr;
    int share = 1;   // the search grid takes 1/share of the GPU's resident blocks
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    DBuf seqs, maps, inst, alpha, lmers, items, lists, fscr, keys, keys_alt, hist, flags,
        out_chars, byte_off, first, last, counters, don0, don1, trace, planes;
    std::vector<DBuf *> all()
    {
        return {&seqs, &maps, &inst, &alpha, &lmers, &items, &lists, &fscr, &keys, &keys_alt,
                &hist, &flags, &out_chars, &byte_off, &first, &last, &counters, &don0, &don1,
                &trace, &planes};
    }
};

// PMS_DEBUG set in the environment: diagnostics go to stderr.
bool debug_on()
{
    static const bool on = std::getenv("PMS_DEBUG") != nullptr;
    return on;
}

// A failing CUDA call returns PMS_E_CUDA; with PMS_DEBUG set the call, its place and
// CUDA's error string also go to stderr.
void report_cuda(cudaError_t e, const char *what, int line)
{
    if (debug_on())
        std::fprintf(stderr, "libpms: %s failed at pms_api.cu:%d: %s (%d)\n", what, line,
                     cudaGetErrorString(e), (int)e);
}

#define PMS_CU(call)                               \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) {                   \
            report_cuda(e_, #call, __LINE__);      \
            cudaGetLastError();                    \
            return PMS_E_CUDA;                     \
        }                                          \
    } while (0)
#define PMS_TRY(call)                              \
    do {                                           \
        int r_ = (call);                           \
        if (r_ != PMS_OK)                          \
            return r_;                             \
    } while (0)

// ---------------------------------------------------------------- instance checks

struct Prep {
    const char *seqs = nullptr;   // host or device (see on_device)
    bool on_device = false;
    int n = 0, m = 0, l = 0, d = 0, L = 0, k = 0, kbits = 0, t = 0, xb = 0, xe = 0;
    std::string alphabet;
    Layout lay = Layout::DNA32;
};

int prepare(const char *seqs, int n, int m, const char *alphabet, int l, int d,
            const pms_opts &o, Prep &p)
{
    if (!seqs || !alphabet)
        return PMS_E_INVAL;
    size_t k = strnlen(alphabet, 64);
    if (k < 2 || k > 32)
        return PMS_E_INVAL;
    bool seen[256] = {false};
    for (size_t i = 0; i < k; i++) {
        unsigned char c = (unsigned char)alphabet[i];
        if (seen[c])
            return PMS_E_INVAL;
        seen[c] = true;
    }
    if (n < 1 || n > kRMax || l < 1 || m < l || d < 0 || l > 64 || m - l + 1 > 65535)
        return PMS_E_INVAL;
    int kbits = k <= 4 ? 2 : 5;
    if (l * kbits > 128)
        return PMS_E_INVAL;
    p.seqs = seqs;
    p.n = n;
    p.m = m;
    p.l = l;
    p.d = d;
    p.L = m - l + 1;
    p.k = (int)k;
    p.kbits = kbits;
    p.alphabet.assign(alphabet, k);
    p.lay = kbits == 2 ? (l <= 32 ? Layout::DNA32 : Layout::DNA64)
                       : (l <= 32 ? Layout::P5_32 : Layout::P5_64);
    p.xb = 0;
    p.xe = p.L;
    if (o.x_begin || o.x_end) {
        p.xb = std::max(0, std::min(o.x_begin, p.L));
        p.xe = std::max(p.xb, std::min(o.x_end, p.L));
    }
    return PMS_OK;
}

size_t lmer_bytes(Layout lay)
{
    switch (lay) {
    case Layout::DNA32: return 8;
    case Layout::DNA64: return 16;
    case Layout::P5_32: return 20;
    case Layout::P5_64: return 40;
    }
    return 40;
}

// ----------------------------------------------------- threshold model (Appendix D)

double nbhd(int l, int d, int k)
{
    double s = 0, c = 1;   // c = C(l, i)
    for (int i = 0; i <= std::min(d, l); i++) {
        s += c * std::pow((double)(k - 1), i);
        c = c * (l - i) / (i + 1);
    }
    return s;
}

// Appendix D: with p = N_2d/|S|^l (chance that an l-mer survives the 2d filter of the
// stack top) and q = N_d/N_2d, the sample-driven part costs
// Time_s(t) = n l sum_{j<=t} L^j p^{j(j-1)/2} and the pattern-driven part
// Time_p(t) = L^t p^{t(t-1)/2} N_d q^{t-1} l.
double model_cost(int n, int m, int l, int d, int k, int t)
{
    const double L = m - l + 1;
    const double nd = nbhd(l, d, k), n2d = nbhd(l, 2 * d, k);
    const double total = std::pow((double)k, l);
    const double p = std::min(1.0, n2d / total), q = std::min(1.0, nd / std::max(n2d, 1.0));
    double ts = 0;
    for (int j = 1; j <= t; j++)
        ts += std::pow(L, j) * std::pow(p, j * (j - 1) / 2.0);
    ts *= (double)n * l;
    const double tp =
        std::pow(L, t) * std::pow(p, t * (t - 1) / 2.0) * nd * std::pow(q, t - 1) * l;
    return ts + tp;
}

// The t in 2..min(n, 8) that minimises the Appendix D cost.
int model_threshold(int n, int m, int l, int d, int k)
{
    int best = 2;
    double best_cost = INFINITY;
    for (int t = 2; t <= std::min(n, kTMax); t++) {
        const double cost = model_cost(n, m, l, d, k, t);
        if (cost < best_cost) {
            best_cost = cost;
            best = t;
        }
    }
    return best;
}

}  // namespace

// ------------------------------------------------------------------------- context

struct Request {
    uint64_t ticket;
    std::string seqs, alphabet;
    int n, m, l, d;
    int x_begin, x_end;
    std::chrono::steady_clock::time_point arrival;
};

struct Finished {
    int rc;
    pms_result res;
};

struct pms_ctx {
    int device = 0;
    int sm_count = 0;
    pms_opts opts{};
    std::atomic<size_t> held{0};
    size_t budget = 0;
    cudaMemPool_t pool = nullptr;   // device memory of all workspaces (kept, not returned)
    Workspace main;
    std::mutex solve_mu;
    // threshold autotuner cache: tune_key -> t
    std::mutex tune_mu;
    std::map<std::tuple<int, int, int, int, int>, int> tune;
    // serving
    std::mutex q_mu;
    std::condition_variable q_cv;      // workers: requests pending or stop
    std::condition_variable done_cv;   // pms_wait: a batch finished or stop
    std::deque<Request> pending;
    std::unordered_map<uint64_t, Finished> finished;
    std::unordered_map<uint64_t, int> in_flight;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::vector<std::unique_ptr<Workspace>> slots;
    std::vector<std::thread> workers;
    std::once_flag serve_once;
};

namespace {

int ws_init(pms_ctx *c, Workspace &w)
{
    PMS_CU(cudaSetDevice(c->device));
    PMS_CU(cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking));
    for (DBuf *b : w.all())
        b->pool = c->pool;
    for (auto &e : w.ev)
        PMS_CU(cudaEventCreate(&e));
    return PMS_OK;
}

void ws_free(pms_ctx *c, Workspace &w)
{
    cudaSetDevice(c->device);
    for (DBuf *b : w.all())
        b->release_counted(c->held, w.stream);
    if (w.stream)
        cudaStreamSynchronize(w.stream);
    for (auto &e : w.ev)
        if (e)
            cudaEventDestroy(e);
    if (w.stream)
        cudaStreamDestroy(w.stream);
    w.stream = nullptr;
}

// Autotuner classes: (l, d, alphabet size) and n, m rounded to the nearest power of two
// (their effect on the best threshold is smooth; see Appendix D's cost model).
std::tuple<int, int, int, int, int> tune_key(const Prep &p)
{
    return std::make_tuple(p.l, p.d, p.k, (int)std::lround(std::log2((double)p.n)),
                           (int)std::lround(std::log2((double)p.m)));
}

// Thresholds 2..4 enumerate with packed byte budgets, which hold d <= 41.
int threshold_for_raw(pms_ctx *c, const Prep &p);

int threshold_for(pms_ctx *c, const Prep &p)
{
    int t = threshold_for_raw(c, p);
    if (p.d > 41 && t < 5)
        t = std::min(5, kTMax);
    return t;
}

int threshold_for_raw(pms_ctx *c, const Prep &p)
{
    if (c->opts.threshold)
        return std::max(2, std::min(c->opts.threshold, kTMax));
    std::lock_guard<std::mutex> g(c->tune_mu);
    auto it = c->tune.find(tune_key(p));
    if (it != c->tune.end())
        return it->second;
    return model_threshold(p.n, p.m, p.l, p.d, p.k);
}

struct BatchOut {
    // host path: per-instance results; device path: user buffer
    std::vector<pms_result> *host = nullptr;
    char *dev_motifs = nullptr;
    uint64_t dev_cap = 0;
    uint64_t *dev_count = nullptr;
    std::vector<int> rc;
};

// The whole pipeline for instances that share one plane layout.
// With `tune` set, run only packing, the 2d filter and the search on a strided sample of
// the items for every threshold in tune->cand, and report the fastest in tune->best.
struct Tune {
    std::vector<int> cand;
    int best = 0;
    std::vector<float> ms;   // device time of each candidate's sample (infinite: capped)
};

int run_group(pms_ctx *c, Workspace &w, std::vector<Prep> &ins, BatchOut &bo,
              const std::vector<int> &idx, pms_stats *stats_out, Tune *tune = nullptr)
{
    uint64_t h2d = 0, d2h = 0;
    auto copy = [&](void *dst, const void *src, size_t bytes, cudaMemcpyKind kind,
                    cudaStream_t st) {
        if (kind == cudaMemcpyHostToDevice)
            h2d += bytes;
        else if (kind == cudaMemcpyDeviceToHost)
            d2h += bytes;
        return cudaMemcpyAsync(dst, src, bytes, kind, st);
    };
    const int ninst = (int)ins.size();
    cudaStream_t s = w.stream;
    const Layout lay = ins[0].lay;
    std::vector<InstDesc> desc(ninst);
    uint64_t seq_total = 0, lmer_total = 0, x_total = 0, item_cap = 0, list_cap = 0;
    int key_bits = 0, lmax = 1;
    const int t = ins[0].t;   // every instance of a group shares the threshold
    for (int i = 0; i < ninst; i++) {
        Prep &p = ins[i];
        InstDesc &D = desc[i];
        D.seq_off = seq_total;
        D.lmer_off = lmer_total;
        D.x_off = x_total;
        D.n = p.n;
        D.m = p.m;
        D.l = p.l;
        D.d = p.d;
        D.L = p.L;
        D.k = p.k;
        D.kbits = p.kbits;
        D.t = p.t;
        D.x_begin = p.xb;
        D.x_end = p.xe;
        seq_total += (uint64_t)p.n * p.m;
        lmer_total += (uint64_t)p.n * p.L;
        x_total += (uint64_t)(p.xe - p.xb);
        item_cap += (uint64_t)(p.xe - p.xb) * (p.n > 1 ? (uint64_t)p.L : 1);
        list_cap = std::max<uint64_t>(list_cap, (uint64_t)std::max(1, p.n - 1) * p.L);
        key_bits = std::max(key_bits, p.l * p.kbits);
        lmax = std::max(lmax, p.l);
    }
    const int multi = ninst > 1;
    const int sort_bits = key_bits + (multi ? kInstBits : 0);
    const int levels = search_levels(t);

    // search launch shape for threshold tt
    int wpb = c->opts.warps_per_block ? std::max(1, std::min(c->opts.warps_per_block, 4)) : 4;
    auto shape = [&](int tt, LaunchCfg &cfg) {
        int per_sm = search_max_blocks(lay, tt, wpb);
        if (per_sm <= 0)
            return PMS_E_CUDA;
        if (c->opts.blocks_per_sm)
            per_sm = std::min(per_sm, c->opts.blocks_per_sm);
        cfg = LaunchCfg{wpb, std::max(c->sm_count, per_sm * c->sm_count / std::max(1, w.share))};
        return PMS_OK;
    };
    LaunchCfg cfg{};
    PMS_TRY(shape(t, cfg));
    (void)levels;

    // buffers; the raw motif list is sized from the expected number of motifs of random
    // strings (Appendix C: |S|^l q^n, q = 1 - (1 - N_d/|S|^l)^(m-l+1)) times the number of
    // finds per motif seen in practice (2.5-5), so reruns after an overflow are rare
    double expect = 0;
    for (const Prep &p : ins) {
        const double nd = nbhd(p.l, p.d, p.k), total = std::pow((double)p.k, p.l);
        const double q = 1.0 - std::pow(1.0 - std::min(1.0, nd / total), (double)p.L);
        expect += std::min(total, total * std::pow(q, p.n)) + 1.0;
    }
    const double want_keys = std::min(6.0 * expect + 65536.0,
                                      (double)std::max<uint64_t>(c->opts.max_motifs, 1) * 8.0);
    uint64_t key_cap = std::max<uint64_t>((uint64_t)want_keys, w.keys.cap / 16);
    PMS_TRY(w.seqs.ensure(seq_total, c->held, s));
    PMS_TRY(w.maps.ensure(256 * (size_t)ninst, c->held, s));
    PMS_TRY(w.alpha.ensure(32 * (size_t)ninst, c->held, s));
    PMS_TRY(w.inst.ensure(sizeof(InstDesc) * ninst, c->held, s));
    PMS_TRY(w.lmers.ensure(lmer_bytes(lay) * lmer_total, c->held, s));
    PMS_TRY(w.items.ensure(sizeof(Item) * std::max<uint64_t>(item_cap, 1), c->held, s));
    const uint64_t fstride = (search_frontier_bytes(lay, lmax) + 255) & ~uint64_t(255);
    // per-warp scratch of a search launch with threshold tt
    auto scratch = [&](int tt, const LaunchCfg &cf) {
        const uint64_t nw = (uint64_t)cf.blocks * cf.warps_per_block;
        int rc = w.lists.ensure(4ull * nw * search_levels(tt) * list_cap, c->held, s);
        if (rc == PMS_OK)
            rc = w.planes.ensure(lmer_bytes(lay) * nw * search_levels(tt) * list_cap, c->held,
                                 s);
        if (rc == PMS_OK)
            rc = w.fscr.ensure(fstride * nw, c->held, s);
        return rc;
    };
    PMS_TRY(scratch(t, cfg));
    PMS_TRY(w.keys.ensure(16 * key_cap, c->held, s));
    PMS_TRY(w.counters.ensure(sizeof(Counters), c->held, s));
    PMS_TRY(w.don0.ensure(sizeof(Item) * kDonateCap, c->held, s));
    PMS_TRY(w.don1.ensure(sizeof(Item) * kDonateCap, c->held, s));
    PMS_TRY(w.first.ensure(8 * (size_t)ninst, c->held, s));
    PMS_TRY(w.last.ensure(8 * (size_t)ninst, c->held, s));
    PMS_TRY(w.byte_off.ensure(8 * (size_t)ninst, c->held, s));
    if (c->budget && c->held > c->budget)
        return PMS_E_NOMEM;

    // inputs
    std::vector<uint8_t> maps(256 * (size_t)ninst, 0xFF), alpha(32 * (size_t)ninst, 0);
    for (int i = 0; i < ninst; i++) {
        for (int a = 0; a < ins[i].k; a++) {
            maps[256 * (size_t)i + (uint8_t)ins[i].alphabet[a]] = (uint8_t)a;
            alpha[32 * (size_t)i + a] = (uint8_t)ins[i].alphabet[a];
        }
        uint8_t *dst = w.seqs.as<uint8_t>() + desc[i].seq_off;
        size_t bytes = (size_t)ins[i].n * ins[i].m;
        PMS_CU(copy(dst, ins[i].seqs, bytes,
                               ins[i].on_device ? cudaMemcpyDeviceToDevice
                                                : cudaMemcpyHostToDevice,
                               s));
    }
    PMS_CU(cudaEventRecord(w.ev[0], s));
    PMS_CU(copy(w.maps.p, maps.data(), maps.size(), cudaMemcpyHostToDevice, s));
    PMS_CU(copy(w.alpha.p, alpha.data(), alpha.size(), cudaMemcpyHostToDevice, s));
    PMS_CU(copy(w.inst.p, desc.data(), sizeof(InstDesc) * ninst,
                           cudaMemcpyHostToDevice, s));
    Counters *dc = w.counters.as<Counters>();
    PMS_CU(cudaMemsetAsync(dc, 0, sizeof(Counters), s));

    PMS_CU(launch_pack(lay, w.inst.as<InstDesc>(), nullptr, ninst, lmer_total,
                       w.seqs.as<uint8_t>(), w.maps.as<uint8_t>(), w.lmers.p, &dc->status, s));
    PMS_CU(launch_items(lay, w.inst.as<InstDesc>(), nullptr, ninst, x_total, w.lmers.p,
                        w.items.as<Item>(), &dc->item_count, item_cap, &dc->status, &dc->stats,
                        s));
    uint64_t launches = (lmer_total ? 1 : 0) + (x_total ? 1 : 0);
    // Optional per-item profile (env PMS_ITEM_TRACE = output file, binary ItemTrace records
    // of the first pass): a profiling aid, off by default.
    const char *trace_path = std::getenv("PMS_ITEM_TRACE");
    ItemTrace *trace = nullptr;
    if (trace_path && *trace_path && !tune) {
        PMS_TRY(w.trace.ensure(sizeof(ItemTrace) * std::max<uint64_t>(item_cap, 1), c->held, s));
        trace = w.trace.as<ItemTrace>();
    }
    // The search: pass 0 over the items, then passes over the items handed on by
    // subproblems that ran past their budget, until none are.
    auto search = [&](int tt, const LaunchCfg &cf, int stride, long long cap = 0) -> int {
        Item *don[2] = {w.don0.as<Item>(), w.don1.as<Item>()};
        for (int pass = 0;; pass++) {
            const bool first_pass = pass == 0;
            const int out = pass & 1;
            unsigned long long zero = 0;
            PMS_CU(cudaMemcpyAsync(&dc->item_next, &zero, 8, cudaMemcpyHostToDevice, s));
            PMS_CU(cudaMemcpyAsync(&dc->donate_count[out], &zero, 8, cudaMemcpyHostToDevice,
                                   s));
            SearchArgs sa{w.inst.as<InstDesc>(), w.lmers.p,
                          first_pass ? w.items.as<Item>() : don[out ^ 1],
                          first_pass ? &dc->item_count : &dc->donate_count[out ^ 1],
                          first_pass ? item_cap : kDonateCap, &dc->item_next,
                          w.lists.as<uint32_t>(), list_cap, w.keys.as<uint64_t>(),
                          &dc->key_count, key_cap, &dc->status, &dc->stats, key_bits, multi,
                          cf, w.fscr.as<unsigned char>(), fstride, lmax,
                          first_pass ? stride : 1, don[out], &dc->donate_count[out],
                          kDonateCap, kItemBudget, first_pass ? trace : nullptr, w.planes.p,
                          cap};
            PMS_CU(launch_search(lay, tt, sa, s));
            launches++;
            unsigned long long handed = 0;
            PMS_CU(cudaMemcpyAsync(&handed, &dc->donate_count[out], 8, cudaMemcpyDeviceToHost,
                                   s));
            PMS_CU(cudaStreamSynchronize(s));
            if (handed == 0)
                return PMS_OK;
        }
    };
    Counters hc{};
    if (tune) {
        // Section 2.2 picks the threshold by trying the search on a sample of the work.
        unsigned long long nitems = 0;
        PMS_CU(copy(&nitems, &dc->item_count, sizeof nitems, cudaMemcpyDeviceToHost, s));
        PMS_CU(cudaStreamSynchronize(s));
        // A candidate's cost is the device time of the search over every stride-th item,
        // with work splitting as in a full run.  The sample holds at least kTuneItemsPerWarp
        // items per search warp, so the passes run at the occupancy of a full run (at low
        // occupancy, latency that a full run hides would count against the list filter).
        // The first candidate's launches run under a generous safety cap; each later one's
        // are capped at the best time so far in cycles at the highest SM clock, so a
        // capped candidate (out) has a single launch slower than the best whole sample.
        double best_ms = INFINITY;
        tune->ms.clear();
        for (int tt : tune->cand) {
            LaunchCfg cf{};
            PMS_TRY(shape(tt, cf));
            PMS_TRY(scratch(tt, cf));
            const unsigned long long warps = (unsigned long long)cf.blocks * cf.warps_per_block;
            const int stride = (int)std::max<unsigned long long>(
                1, nitems / std::max<unsigned long long>(1024, kTuneItemsPerWarp * warps));
            const long long cap =
                tune->best ? std::min<long long>(kTuneItemCap, (long long)(best_ms * kMaxCyclesPerMs))
                           : kTuneItemCap;
            PMS_CU(cudaMemsetAsync(&dc->status, 0, sizeof(int), s));
            PMS_CU(cudaMemsetAsync(&dc->stats, 0, sizeof(DevStats), s));
            PMS_CU(cudaEventRecord(w.ev[1], s));
            PMS_TRY(search(tt, cf, stride, cap));
            PMS_CU(cudaEventRecord(w.ev[2], s));
            Counters tc{};
            PMS_CU(cudaMemcpyAsync(&tc, dc, sizeof tc, cudaMemcpyDeviceToHost, s));
            PMS_CU(cudaStreamSynchronize(s));
            float ms = 0;
            cudaEventElapsedTime(&ms, w.ev[1], w.ev[2]);
            const bool capped = (tc.status & kErrTuneCapped) != 0;
            tune->ms.push_back(capped ? INFINITY : ms);
            if (debug_on())
                std::fprintf(stderr, "pms autotune: l=%d d=%d n=%d m=%d t=%d stride=%d ms=%.3f%s\n",
                             ins[0].l, ins[0].d, ins[0].n, ins[0].m, tt, stride, ms,
                             capped ? " (capped)" : "");
            if (!capped && ms < best_ms) {
                best_ms = ms;
                tune->best = tt;
            }
        }
        return PMS_OK;
    }
    for (int attempt = 0;; attempt++) {
        PMS_CU(cudaEventRecord(w.ev[1], s));
        PMS_TRY(search(t, cfg, 1));
        PMS_CU(cudaEventRecord(w.ev[2], s));
        PMS_CU(copy(&hc, dc, sizeof hc, cudaMemcpyDeviceToHost, s));
        PMS_CU(cudaStreamSynchronize(s));
        if (hc.status & kErrAlphabet)
            return PMS_E_ALPHABET;
        if (hc.status & kErrItemsOverflow) {
            report_cuda(cudaErrorUnknown, "item list overflow", __LINE__);
            return PMS_E_CUDA;
        }
        if (hc.status & kErrBounds) {
            report_cuda(cudaErrorUnknown, "search index check", (int)hc.stats.bad_site);
            return PMS_E_CUDA;
        }
        if (!(hc.status & kErrKeysOverflow))
            break;
        // the raw (not yet unique) motif list outgrew its buffer: grow and search again
        uint64_t want = hc.key_count + hc.key_count / 4 + 1024;
        uint64_t limit = std::max<uint64_t>(c->opts.max_motifs, 1) * 64;
        if (want > limit || attempt > 4)
            return PMS_E_OVERFLOW;
        PMS_TRY(w.keys.ensure(16 * want, c->held, s));
        key_cap = w.keys.cap / 16;
        if (c->budget && c->held > c->budget)
            return PMS_E_NOMEM;
        unsigned long long zero[2] = {0, 0};
        PMS_CU(copy(&dc->item_next, zero, 16, cudaMemcpyHostToDevice, s));
        PMS_CU(cudaMemsetAsync(&dc->status, 0, sizeof(int), s));
        PMS_CU(cudaMemsetAsync(&dc->stats, 0, sizeof(DevStats), s));
    }

    if (trace) {
        const uint64_t n = std::min<uint64_t>(hc.item_count, item_cap);
        std::vector<ItemTrace> recs(n);
        PMS_CU(cudaMemcpy(recs.data(), trace, sizeof(ItemTrace) * n, cudaMemcpyDeviceToHost));
        if (FILE *f = std::fopen(trace_path, "wb")) {
            std::fwrite(recs.data(), sizeof(ItemTrace), n, f);
            std::fclose(f);
        }
    }

    // collect: sort, unique, per-instance ranges
    const size_t nkeys = hc.key_count;
    const size_t ntiles = (nkeys + kSortTile - 1) / kSortTile;
    PMS_TRY(w.keys_alt.ensure(16 * std::max<size_t>(nkeys, 1), c->held, s));
    PMS_TRY(w.hist.ensure(4 * 256 * std::max<size_t>(ntiles, 1), c->held, s));
    PMS_TRY(w.flags.ensure(4 * std::max<size_t>(ntiles, 1), c->held, s));
    SortScratch scr{w.keys_alt.as<uint64_t>(), w.hist.as<unsigned>(), w.flags.as<unsigned>(),
                    w.keys_alt.cap / 16, w.flags.cap / 4};
    size_t nuniq = 0;
    PMS_CU(sort_unique_keys(w.keys.as<uint64_t>(), nkeys, sort_bits, scr, &dc->uniq_total,
                            &nuniq, s));
    if (nkeys) {
        launches += 3ull * ((sort_bits + 7) / 8) + 3 + (nuniq ? 1 : 0);
        d2h += sizeof(unsigned long long);   // the unique count read back by the sort
    }
    PMS_CU(cudaMemsetAsync(w.first.p, 0xFF, 8 * (size_t)ninst, s));
    PMS_CU(cudaMemsetAsync(w.last.p, 0xFF, 8 * (size_t)ninst, s));
    PMS_CU(launch_ranges(w.keys.as<uint64_t>(), nuniq, key_bits, multi, ninst,
                         w.first.as<long long>(), w.last.as<long long>(), s));
    std::vector<long long> first(ninst), last(ninst);
    PMS_CU(copy(first.data(), w.first.p, 8 * (size_t)ninst, cudaMemcpyDeviceToHost, s));
    PMS_CU(copy(last.data(), w.last.p, 8 * (size_t)ninst, cudaMemcpyDeviceToHost, s));
    PMS_CU(cudaStreamSynchronize(s));
    std::vector<uint64_t> counts(ninst), byte_off(ninst);
    uint64_t bytes = 0;
    for (int i = 0; i < ninst; i++) {
        counts[i] = first[i] < 0 ? 0 : (uint64_t)(last[i] - first[i] + 1);
        byte_off[i] = bytes;
        bytes += counts[i] * (uint64_t)ins[i].l;
    }
    char *out_dev = nullptr;
    if (bo.host) {
        PMS_TRY(w.out_chars.ensure(std::max<uint64_t>(bytes, 1), c->held, s));
        out_dev = w.out_chars.as<char>();
    } else {
        out_dev = bo.dev_motifs;
        if (counts[0] > bo.dev_cap)
            bytes = 0;   // decode nothing past the caller's capacity
    }
    PMS_CU(copy(w.byte_off.p, byte_off.data(), 8 * (size_t)ninst,
                           cudaMemcpyHostToDevice, s));
    launches += bytes ? 1 : 0;
    if (bytes)
        PMS_CU(launch_decode(w.keys.as<uint64_t>(), nuniq, key_bits, multi, w.inst.as<InstDesc>(),
                             w.alpha.as<uint8_t>(), out_dev, w.byte_off.as<uint64_t>(),
                             w.first.as<long long>(), s));
    PMS_CU(cudaEventRecord(w.ev[3], s));
    PMS_CU(cudaStreamSynchronize(s));

    float total_ms = 0, search_ms = 0;
    cudaEventElapsedTime(&total_ms, w.ev[0], w.ev[3]);
    cudaEventElapsedTime(&search_ms, w.ev[1], w.ev[2]);
    pms_stats st{};
    st.items = hc.stats.items;
    st.tuples = hc.stats.tuples;
    st.hd_compares = hc.stats.hd_compares;
    st.enum_nodes = hc.stats.enum_nodes;
    st.leaves = hc.stats.leaves;
    st.raw_motifs = hc.stats.raw_motifs;
    st.cyc_filter = hc.stats.cyc_filter;
    st.cyc_enum = hc.stats.cyc_enum;
    st.cyc_verify = hc.stats.cyc_verify;
    st.search_ops = hc.stats.search_ops;
    st.launches = launches;
    st.busy_max = hc.stats.busy_max;
    st.busy_mean = hc.stats.warps ? hc.stats.busy_sum / hc.stats.warps : 0;
    st.item_max = hc.stats.item_max;
    st.h2d_bytes = h2d;
    st.d2h_bytes = d2h;
    st.kernel_ms = total_ms;
    st.search_ms = search_ms;
    st.threshold = ins[0].t;
    if (stats_out)
        *stats_out = st;

    const uint64_t maxm = c->opts.max_motifs;
    if (bo.host) {
        for (int i = 0; i < ninst; i++) {
            pms_result &r = (*bo.host)[idx[i]];
            r.count = 0;
            r.l = ins[i].l;
            r.motifs = nullptr;
            r.stats = st;
            r.stats.threshold = ins[i].t;
            if (counts[i] > maxm) {
                bo.rc[idx[i]] = PMS_E_OVERFLOW;
                continue;
            }
            size_t nb = counts[i] * (size_t)ins[i].l;
            if (nb) {
                r.motifs = static_cast<char *>(std::malloc(nb));
                if (!r.motifs) {
                    bo.rc[idx[i]] = PMS_E_NOMEM;
                    continue;
                }
                d2h += nb;
                PMS_CU(cudaMemcpy(r.motifs, out_dev + byte_off[i], nb, cudaMemcpyDeviceToHost));
            }
            r.count = counts[i];
            bo.rc[idx[i]] = PMS_OK;
        }
    } else {
        *bo.dev_count = counts[0];
        bo.rc[0] = counts[0] > bo.dev_cap || counts[0] > maxm ? PMS_E_OVERFLOW : PMS_OK;
    }
    return PMS_OK;
}

// Autotuner: the first time an instance class (tune_key) is seen, time the search on a
// sample of its items for the thresholds around the Appendix D model and cache the
// fastest.  The motif set does not depend on the threshold.
void autotune(pms_ctx *c, Workspace &w, const Prep &p)
{
    const auto key = tune_key(p);
    {
        std::lock_guard<std::mutex> g(c->tune_mu);
        if (c->tune.count(key))
            return;
    }
    const int model = model_threshold(p.n, p.m, p.l, p.d, p.k);
    const int hi = std::min(p.n, kTMax);
    Tune tu;
    // candidates: thresholds around the model's, the most often best one (4) first (tuning
    // passes stop any item that runs past a cycle cap, so a candidate whose
    // neighbourhoods explode costs little)
    std::vector<int> around;
    for (int t = std::max(2, std::min(model - 1, 3)); t <= std::min(hi, std::max(model + 1, 5));
         t++)
        if (!(p.d > 41 && t < 5))
            around.push_back(t);
    for (int t : around)
        if (t == 4)
            tu.cand.push_back(t);
    for (int t : around)
        if (t != 4)
            tu.cand.push_back(t);
    int chosen = model;
    if (tu.cand.size() > 1 && p.n >= 3) {
        std::vector<Prep> one{p};
        one[0].t = tu.cand[0];
        one[0].xb = 0;
        one[0].xe = p.L;
        BatchOut bo;
        std::vector<pms_result> dummy(1);
        bo.host = &dummy;
        bo.rc.assign(1, PMS_OK);
        std::vector<int> idx{0};
        if (run_group(c, w, one, bo, idx, nullptr, &tu) == PMS_OK && tu.best)
            chosen = tu.best;
    }
    std::lock_guard<std::mutex> g(c->tune_mu);
    c->tune[key] = chosen;
}

// Split a batch into groups that can share one launch sequence (same plane layout, key
// room for the instance id) and run each.
int run_batch(pms_ctx *c, Workspace &w, std::vector<Prep> &ins, BatchOut &bo, pms_stats *agg)
{
    if (!c->opts.threshold)
        for (auto &p : ins)
            autotune(c, w, p);
    std::map<int, std::vector<int>> groups;
    for (int i = 0; i < (int)ins.size(); i++) {
        ins[i].t = threshold_for(c, ins[i]);
        int key = (int)ins[i].lay * 16 + ins[i].t;
        if (ins[i].l * ins[i].kbits + kInstBits > 128)
            key = 1000 + i;   // no room for the instance id: runs alone
        groups[key].push_back(i);
    }
    pms_stats total{};
    for (auto &g : groups) {
        for (size_t off = 0; off < g.second.size(); off += 60000) {
            std::vector<int> idx(g.second.begin() + off,
                                 g.second.begin() + std::min(g.second.size(), off + 60000));
            std::vector<Prep> part;
            for (int i : idx)
                part.push_back(ins[i]);
            pms_stats st{};
            int rc = run_group(c, w, part, bo, idx, &st);
            if (rc != PMS_OK) {
                for (int i : idx)
                    bo.rc[i] = rc;
                if (!bo.host)
                    return rc;
                continue;
            }
            total.items += st.items;
            total.tuples += st.tuples;
            total.hd_compares += st.hd_compares;
            total.enum_nodes += st.enum_nodes;
            total.leaves += st.leaves;
            total.raw_motifs += st.raw_motifs;
            total.cyc_filter += st.cyc_filter;
            total.cyc_enum += st.cyc_enum;
            total.cyc_verify += st.cyc_verify;
            total.search_ops += st.search_ops;
            total.launches += st.launches;
            total.busy_max = std::max(total.busy_max, st.busy_max);
            total.busy_mean = std::max(total.busy_mean, st.busy_mean);
            total.item_max = std::max(total.item_max, st.item_max);
            total.h2d_bytes += st.h2d_bytes;
            total.d2h_bytes += st.d2h_bytes;
            total.kernel_ms += st.kernel_ms;
            total.search_ms += st.search_ms;
            total.threshold = st.threshold;
        }
    }
    if (agg)
        *agg = total;
    return PMS_OK;
}

// --------------------------------------------------------------------- serving loop

// One serving slot: waits for requests, admits as many as fit (count and memory budget),
// runs them as one batch on its own stream and publishes the results.  Several slots run
// at once, so requests that arrive while a batch is on the GPU start on another slot.
void serve_worker(pms_ctx *c, Workspace *w)
{
    cudaSetDevice(c->device);
    const int max_batch = c->opts.serve_max_batch;
    for (;;) {
        std::vector<Request> batch;
        {
            std::unique_lock<std::mutex> lk(c->q_mu);
            c->q_cv.wait(lk, [&] { return c->stop || !c->pending.empty(); });
            if (c->stop && c->pending.empty())
                return;
            // Admission: the cheapest pending request first (Appendix D cost estimate), then
            // others no more than 8x costlier, within the batch size and the memory still
            // free under the budget (strings, l-mers, items, raw motifs), so light requests
            // are not held behind heavy ones.
            const size_t room = c->budget > c->held ? c->budget - c->held : 0;
            auto cost = [](const Request &r) {
                const int k = (int)r.alphabet.size();
                return model_cost(r.n, r.m, r.l, r.d, k,
                                  model_threshold(r.n, r.m, r.l, r.d, k));
            };
            auto bytes = [](const Request &r) {
                const size_t L = (size_t)(r.m - r.l + 1);
                return (size_t)r.n * r.m * 2 + (size_t)r.n * L * 40 + L * L * 8;
            };
            std::vector<std::pair<double, size_t>> order;
            for (size_t i = 0; i < c->pending.size(); i++)
                order.emplace_back(cost(c->pending[i]), i);
            std::sort(order.begin(), order.end());
            std::vector<size_t> take;
            size_t est_total = 0;
            for (auto &oc : order) {
                if ((int)take.size() >= max_batch)
                    break;
                if (!take.empty() && oc.first > 8.0 * order[0].first)
                    break;
                const size_t est = bytes(c->pending[oc.second]);
                if (!take.empty() && est_total + est > room)
                    break;
                est_total += est;
                take.push_back(oc.second);
            }
            std::sort(take.begin(), take.end());
            for (size_t j = take.size(); j-- > 0;) {
                batch.push_back(std::move(c->pending[take[j]]));
                c->pending.erase(c->pending.begin() + (long)take[j]);
            }
            for (auto &r : batch)
                c->in_flight[r.ticket] = 1;
        }
        std::vector<Prep> ins(batch.size());
        std::vector<pms_result> res(batch.size());
        BatchOut bo;
        bo.host = &res;
        bo.rc.assign(batch.size(), PMS_OK);
        std::vector<int> pre_rc(batch.size(), PMS_OK);
        std::vector<Prep> ok_ins;
        std::vector<int> ok_idx;
        for (size_t i = 0; i < batch.size(); i++) {
            pms_opts o = c->opts;
            if (batch[i].x_begin || batch[i].x_end) {
                o.x_begin = batch[i].x_begin;
                o.x_end = batch[i].x_end;
            }
            pre_rc[i] = prepare(batch[i].seqs.data(), batch[i].n, batch[i].m,
                                batch[i].alphabet.c_str(), batch[i].l, batch[i].d, o, ins[i]);
            if (pre_rc[i] == PMS_OK) {
                ok_ins.push_back(ins[i]);
                ok_idx.push_back((int)i);
            }
        }
        if (!ok_ins.empty()) {
            std::vector<pms_result> ok_res(ok_ins.size());
            BatchOut ob;
            ob.host = &ok_res;
            ob.rc.assign(ok_ins.size(), PMS_OK);
            run_batch(c, *w, ok_ins, ob, nullptr);
            for (size_t j = 0; j < ok_idx.size(); j++) {
                res[ok_idx[j]] = ok_res[j];
                pre_rc[ok_idx[j]] = ob.rc[j];
            }
        }
        {
            std::lock_guard<std::mutex> lk(c->q_mu);
            for (size_t i = 0; i < batch.size(); i++) {
                c->in_flight.erase(batch[i].ticket);
                c->finished[batch[i].ticket] = Finished{pre_rc[i], res[i]};
            }
        }
        c->done_cv.notify_all();
    }
}

int start_serving(pms_ctx *c)
{
    int rc = PMS_OK;
    std::call_once(c->serve_once, [&] {
        for (int i = 0; i < c->opts.serve_slots; i++) {
            auto w = std::make_unique<Workspace>();
            if (ws_init(c, *w) != PMS_OK) {
                rc = PMS_E_CUDA;
                return;
            }
            c->slots.push_back(std::move(w));
        }
        for (auto &w : c->slots)
            c->workers.emplace_back(serve_worker, c, w.get());
    });
    return rc;
}

}  // namespace

// ---------------------------------------------------------------------------- C ABI

extern "C" {

const char *pms_strerror(int code)
{
    switch (code) {
    case PMS_OK: return "ok";
    case PMS_E_INVAL: return "invalid argument";
    case PMS_E_ALPHABET: return "sequence byte not in the alphabet";
    case PMS_E_NOMEM: return "out of memory or over the memory budget";
    case PMS_E_OVERFLOW: return "motif set larger than max_motifs";
    case PMS_E_TIMEOUT: return "timed out";
    case PMS_E_CUDA: return "CUDA error or no usable sm_103a device";
    case PMS_E_BUSY: return "busy";
    case PMS_E_NOTFOUND: return "unknown ticket";
    }
    return "unknown error";
}

int pms_create(pms_ctx **out, int device, const pms_opts *opts)
{
    if (!out)
        return PMS_E_INVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return PMS_E_CUDA;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess)
        return PMS_E_CUDA;
    if (prop.major != 10 || prop.minor != 3)
        return PMS_E_CUDA;   // the kernels are built for sm_103a only
    auto *c = new (std::nothrow) pms_ctx();
    if (!c)
        return PMS_E_NOMEM;
    c->device = device;
    c->sm_count = prop.multiProcessorCount;
    if (opts)
        c->opts = *opts;
    if (!c->opts.max_motifs)
        c->opts.max_motifs = 1ull << 26;
    if (!c->opts.serve_slots)
        c->opts.serve_slots = 2;
    if (!c->opts.serve_max_batch)
        c->opts.serve_max_batch = 16;
    if (c->opts.threshold && (c->opts.threshold < 2 || c->opts.threshold > kTMax)) {
        delete c;
        return PMS_E_INVAL;
    }
    if (cudaSetDevice(device) != cudaSuccess) {
        delete c;
        return PMS_E_CUDA;
    }
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    c->budget = c->opts.mem_budget ? c->opts.mem_budget : free_b / 4 * 3;
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    if (cudaMemPoolCreate(&c->pool, &props) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return PMS_E_CUDA;
    }
    uint64_t keep = UINT64_MAX;   // freed blocks stay in the pool for the next solve
    cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (ws_init(c, c->main) != PMS_OK) {
        ws_free(c, c->main);
        cudaMemPoolDestroy(c->pool);
        delete c;
        return PMS_E_CUDA;
    }
    *out = c;
    return PMS_OK;
}

void pms_destroy(pms_ctx *c)
{
    if (!c)
        return;
    {
        std::lock_guard<std::mutex> lk(c->q_mu);
        c->stop = true;
    }
    c->q_cv.notify_all();
    c->done_cv.notify_all();
    for (auto &t : c->workers)
        t.join();
    for (auto &w : c->slots)
        ws_free(c, *w);
    for (auto &f : c->finished)
        std::free(f.second.res.motifs);
    ws_free(c, c->main);
    if (c->pool)
        cudaMemPoolDestroy(c->pool);
    delete c;
}

int pms_solve(pms_ctx *c, const char *seqs, int n, int m, const char *alphabet, int l, int d,
              pms_result *out)
{
    if (!c || !out)
        return PMS_E_INVAL;
    pms_instance in{seqs, n, m, alphabet, l, d, 0, 0};
    return pms_solve_batch(c, &in, 1, out);
}

int pms_solve_batch(pms_ctx *c, const pms_instance *inst, int count, pms_result *outs)
{
    if (!c || (!inst && count) || (!outs && count) || count < 0)
        return PMS_E_INVAL;
    std::vector<Prep> ins(count);
    for (int i = 0; i < count; i++) {
        outs[i] = pms_result{};
        pms_opts o = c->opts;
        if (inst[i].x_begin || inst[i].x_end) {
            o.x_begin = inst[i].x_begin;
            o.x_end = inst[i].x_end;
        }
        int rc = prepare(inst[i].seqs, inst[i].n, inst[i].m, inst[i].alphabet, inst[i].l,
                         inst[i].d, o, ins[i]);
        if (rc != PMS_OK)
            return rc;
    }
    if (!count)
        return PMS_OK;
    std::lock_guard<std::mutex> g(c->solve_mu);
    if (cudaSetDevice(c->device) != cudaSuccess)
        return PMS_E_CUDA;
    std::vector<pms_result> res(count);
    BatchOut bo;
    bo.host = &res;
    bo.rc.assign(count, PMS_OK);
    int rc = run_batch(c, c->main, ins, bo, nullptr);
    int first_err = rc;
    for (int i = 0; i < count; i++) {
        outs[i] = res[i];
        if (first_err == PMS_OK && bo.rc[i] != PMS_OK)
            first_err = bo.rc[i];
    }
    if (first_err != PMS_OK)
        for (int i = 0; i < count; i++)
            pms_result_free(&outs[i]);
    return first_err;
}

int pms_solve_device(pms_ctx *c, const char *d_seqs, int n, int m, const char *alphabet, int l,
                     int d, char *d_motifs, uint64_t cap, uint64_t *count, void *stream,
                     pms_stats *stats)
{
    if (!c || !count || (!d_motifs && cap))
        return PMS_E_INVAL;
    std::vector<Prep> ins(1);
    int rc = prepare(d_seqs, n, m, alphabet, l, d, c->opts, ins[0]);
    if (rc != PMS_OK)
        return rc;
    ins[0].on_device = true;
    std::lock_guard<std::mutex> g(c->solve_mu);
    if (cudaSetDevice(c->device) != cudaSuccess)
        return PMS_E_CUDA;
    cudaStream_t saved = c->main.stream;
    if (stream)
        c->main.stream = static_cast<cudaStream_t>(stream);
    if (!c->opts.threshold)
        autotune(c, c->main, ins[0]);
    ins[0].t = threshold_for(c, ins[0]);
    BatchOut bo;
    bo.dev_motifs = d_motifs;
    bo.dev_cap = cap;
    bo.dev_count = count;
    bo.rc.assign(1, PMS_OK);
    std::vector<int> idx{0};
    pms_stats st{};
    rc = run_group(c, c->main, ins, bo, idx, &st);
    c->main.stream = saved;
    if (stats)
        *stats = st;
    return rc != PMS_OK ? rc : bo.rc[0];
}

int pms_submit(pms_ctx *c, const pms_instance *inst, uint64_t *ticket)
{
    if (!c || !inst || !ticket || !inst->seqs || !inst->alphabet || inst->n < 1 || inst->m < 1)
        return PMS_E_INVAL;
    int rc = start_serving(c);
    if (rc != PMS_OK)
        return rc;
    Request r;
    r.seqs.assign(inst->seqs, (size_t)inst->n * inst->m);
    r.alphabet.assign(inst->alphabet, strnlen(inst->alphabet, 64));
    r.n = inst->n;
    r.m = inst->m;
    r.l = inst->l;
    r.d = inst->d;
    r.x_begin = inst->x_begin;
    r.x_end = inst->x_end;
    r.arrival = std::chrono::steady_clock::now();
    {
        std::lock_guard<std::mutex> lk(c->q_mu);
        if (c->pending.size() >= 1000000)
            return PMS_E_BUSY;
        r.ticket = c->next_ticket++;
        *ticket = r.ticket;
        c->pending.push_back(std::move(r));
    }
    c->q_cv.notify_one();
    return PMS_OK;
}

int pms_poll(pms_ctx *c, uint64_t ticket, pms_result *out, int *done)
{
    if (!c || !out || !done)
        return PMS_E_INVAL;
    *done = 0;
    std::lock_guard<std::mutex> lk(c->q_mu);
    auto it = c->finished.find(ticket);
    if (it == c->finished.end()) {
        if (c->in_flight.count(ticket))
            return PMS_OK;
        for (auto &r : c->pending)
            if (r.ticket == ticket)
                return PMS_OK;
        return PMS_E_NOTFOUND;
    }
    *out = it->second.res;
    int rc = it->second.rc;
    c->finished.erase(it);
    *done = 1;
    return rc;
}

int pms_wait(pms_ctx *c, uint64_t ticket, pms_result *out, int timeout_ms)
{
    if (!c || !out)
        return PMS_E_INVAL;
    std::unique_lock<std::mutex> lk(c->q_mu);
    auto known = [&] {
        if (c->finished.count(ticket) || c->in_flight.count(ticket))
            return true;
        for (auto &r : c->pending)
            if (r.ticket == ticket)
                return true;
        return false;
    };
    if (!known())
        return PMS_E_NOTFOUND;
    auto ready = [&] { return c->stop || c->finished.count(ticket) > 0; };
    if (timeout_ms < 0)
        c->done_cv.wait(lk, ready);
    else if (!c->done_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
        return PMS_E_TIMEOUT;
    auto it = c->finished.find(ticket);
    if (it == c->finished.end())
        return PMS_E_NOTFOUND;   // the context is being destroyed
    *out = it->second.res;
    const int rc = it->second.rc;
    c->finished.erase(it);
    return rc;
}

void pms_result_free(pms_result *res)
{
    if (!res)
        return;
    std::free(res->motifs);
    res->motifs = nullptr;
    res->count = 0;
}

int pms_autotune_entries(pms_ctx *c)
{
    if (!c)
        return 0;
    std::lock_guard<std::mutex> g(c->tune_mu);
    return (int)c->tune.size();
}

void pms_autotune_reset(pms_ctx *c)
{
    if (!c)
        return;
    std::lock_guard<std::mutex> g(c->tune_mu);
    c->tune.clear();
}

}  // extern "C"
