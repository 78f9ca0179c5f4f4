/*
 * pms.h - C ABI of the GB300 planted motif search library (libpms.so).
 *
 * The library solves the (l,d) planted motif search problem exactly (Nicolae & Rajasekaran,
 * "Efficient Sequential and Parallel Algorithms for Planted Motif Search", Section 1):
 * given n strings S_1..S_n of length m over an alphabet and integers l, d, it returns every
 * l-mer M such that each S_i holds an l-mer within Hamming distance d of M.
 *
 * The search follows the paper's method (PMS8, Section 2 and Algorithms 1-2): one
 * subproblem per l-mer x of S_1 (Section 2.3), a 2d compatibility filter (Section 2), a
 * stack of l-mers filtered with the three-l-mer condition (Theorem 1, Section 2.4), and
 * enumeration of the common d-neighbourhood of the stack (Algorithm 1) with every
 * candidate verified against all strings.  All of it runs in CUDA kernels built for
 * sm_103a; there is no CPU fallback: without a usable GPU every call fails with
 * PMS_E_CUDA.
 *
 * Conventions for every call:
 *  - Return value: PMS_OK (0) or a negative PMS_E_* code; pms_strerror names it.
 *  - Sequences: n*m bytes, row-major (string i is bytes [i*m, (i+1)*m)), no terminators.
 *  - Alphabet: NUL-terminated string of 2..32 distinct bytes.  Its order defines the
 *    letter codes and therefore the output order.  A sequence byte outside the alphabet
 *    gives PMS_E_ALPHABET.
 *  - Limits: 1 <= n <= 64, 1 <= l <= m, m - l + 1 <= 65535, 0 <= d, l <= 64, and
 *    l * ceil(log2 |alphabet|) <= 128 (l <= 64 for DNA, l <= 25 for 20 amino acids);
 *    anything else gives PMS_E_INVAL.  d >= l is legal (every l-mer is a motif) but
 *    usually overflows max_motifs.
 *  - Output: the motif set, sorted ascending in the alphabet's order, duplicates removed,
 *    as count*l bytes (no separators, no terminators).  Results the library allocates are
 *    released with pms_result_free.
 *  - Inputs are borrowed for the duration of the call (pms_submit copies them).
 *  - A context is used by one thread at a time, except pms_submit/pms_poll, which may be
 *    called from any thread.
 */
#ifndef PMS_H
#define PMS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    PMS_OK = 0,
    PMS_E_INVAL = -1,     /* bad argument or size outside the limits above */
    PMS_E_ALPHABET = -2,  /* a sequence byte is not in the alphabet */
    PMS_E_NOMEM = -3,     /* device or host allocation failed, or memory budget exceeded */
    PMS_E_OVERFLOW = -4,  /* the motif set is larger than opts.max_motifs */
    PMS_E_TIMEOUT = -5,   /* a bounded wait expired (pms_wait) */
    PMS_E_CUDA = -6,      /* CUDA error, or no usable sm_103a device */
    PMS_E_BUSY = -7,      /* serving queue full */
    PMS_E_NOTFOUND = -8   /* unknown ticket */
};

typedef struct pms_ctx pms_ctx;

/* Tuning and resource options.  Zero in any field selects the default. */
typedef struct pms_opts {
    int threshold;            /* stack size t at which the search switches from filtering to
                                 neighbourhood enumeration (Section 2.2 "threshold",
                                 Algorithm 2 ThresholdCondition); 0 = autotuned.  The motif
                                 set does not depend on it.  Range 2..8. */
    int warps_per_block;      /* search kernel block size in warps (default 4) */
    int blocks_per_sm;        /* resident search blocks per SM (default: occupancy limit) */
    uint64_t max_motifs;      /* upper bound on the result size before PMS_E_OVERFLOW
                                 (default 1<<26) */
    size_t mem_budget;        /* device bytes the context may hold (default: 3/4 of free) */
    int x_begin, x_end;       /* restrict the subproblems to the l-mers x_begin..x_end-1 of
                                 S_1 (Section 2.3); both 0 = all.  Disjoint ranges merged
                                 give the whole set (multi-device sharding by replicas). */
    int serve_slots;          /* concurrent batches in the serving loop (default 2) */
    int serve_max_batch;      /* instances per serving batch (default 16) */
} pms_opts;

/* One problem instance (Section 1). */
typedef struct pms_instance {
    const char *seqs;         /* n*m bytes, row-major */
    int n, m;
    const char *alphabet;     /* NUL-terminated */
    int l, d;
    int x_begin, x_end;       /* subproblems of the l-mers x_begin..x_end-1 of S_1 only
                                 (Section 2.3); both 0 = the context's range (all) */
} pms_instance;

/* Counters of one solve, summed over the kernels that ran. */
typedef struct pms_stats {
    uint64_t items;           /* (x, u) subproblems searched */
    uint64_t tuples;          /* stacks that reached the enumeration */
    uint64_t hd_compares;     /* l-mer distance evaluations (Hd or Theorem 1 triple) */
    uint64_t enum_nodes;      /* Algorithm 1 tree nodes tested */
    uint64_t leaves;          /* common neighbours produced (before verification) */
    uint64_t raw_motifs;      /* verified motifs before duplicate removal */
    uint64_t cyc_filter;      /* search-kernel SM cycles in filtering, summed over warps */
    uint64_t cyc_enum;        /* ... in neighbourhood enumeration (Algorithm 1) */
    uint64_t cyc_verify;      /* ... in verification (isMotif) */
    uint64_t search_ops;      /* algorithmic integer ops of the search kernel (unit costs in
                                 the library's documentation of the roofline) */
    uint64_t launches;        /* kernels launched by the solve */
    uint64_t busy_max;        /* search kernel: largest per-warp busy time (SM cycles) */
    uint64_t busy_mean;       /* search kernel: mean per-warp busy time (SM cycles) */
    uint64_t item_max;        /* search kernel: most cycles a single (x, u) item took */
    uint64_t h2d_bytes;       /* bytes copied host -> device by the solve */
    uint64_t d2h_bytes;       /* bytes copied device -> host by the solve */
    double kernel_ms;         /* device time of the whole solve (CUDA events) */
    double search_ms;         /* device time of the search kernel alone */
    int threshold;            /* threshold used */
} pms_stats;

/* A solved motif set. */
typedef struct pms_result {
    uint64_t count;           /* number of motifs */
    int l;                    /* motif length */
    char *motifs;             /* count*l bytes, sorted, library-allocated (may be NULL if 0) */
    pms_stats stats;
} pms_result;

/* Create a context on CUDA device `device` (opts may be NULL).  Fails with PMS_E_CUDA
 * when the device is missing or is not compute capability 10.3. */
int pms_create(pms_ctx **out, int device, const pms_opts *opts);
void pms_destroy(pms_ctx *ctx);

/* Solve one instance from host memory (Section 1 problem statement).  Blocking. */
int pms_solve(pms_ctx *ctx, const char *seqs, int n, int m, const char *alphabet, int l,
              int d, pms_result *out);

/* Solve `count` instances in one batched launch sequence; outs[i] receives instance i.
 * The motif sets equal those of `count` separate pms_solve calls.  Blocking. */
int pms_solve_batch(pms_ctx *ctx, const pms_instance *inst, int count, pms_result *outs);

/*
 * Solve one instance whose sequences are already in device memory, leaving the result
 * in device memory; for callers that keep data resident on the GPU.
 *   d_seqs       device pointer, n*m bytes
 *   d_motifs     device pointer, room for cap*l bytes; receives the sorted motif set
 *   cap          capacity of d_motifs in motifs
 *   count        host pointer; receives the motif count (even when > cap, in which case
 *                PMS_E_OVERFLOW is returned and d_motifs holds the first cap motifs)
 *   stream       cudaStream_t to run on (NULL = the context's stream); the call returns
 *                after the work on it has finished.
 */
int pms_solve_device(pms_ctx *ctx, const char *d_seqs, int n, int m, const char *alphabet,
                     int l, int d, char *d_motifs, uint64_t cap, uint64_t *count,
                     void *stream, pms_stats *stats);

/*
 * The device-resident solve of pms_solve_device for callers that must not allocate device
 * memory once running: a service that reserves its device memory in its own pool at
 * start-up, so a later cudaMalloc would fail or break its budget, or a real-time pipeline
 * in which cudaMalloc/cudaFree would stall the device and fragment memory.  It needs no
 * context and creates no stream, event or buffer.  (The paper has no counterpart; this is
 * a deployment interface.)
 *
 * All working memory is one fixed 64 MiB array inside the library's device image, which
 * every device that loads the library holds until the process exits.  The caller passes
 * the strings (d_seqs, device, n*m bytes) and the output buffer (d_motifs, device, room
 * for cap*l bytes); *count (host) receives the number of motifs.  Arguments as in
 * pms_solve_device, plus threshold (2..8, or 0 for the Appendix D cost model; no
 * autotuning, which would allocate).  Runs on the current device and on `stream` (NULL =
 * the default stream) and returns after the work on it has finished.
 *
 * Limits: the request must fit the fixed array: the l-mer table, one item per compatible
 * (x, u) pair of up to (m-l+1)^2, at most 262144 raw motif finds, and per-warp search
 * lists of (n-1)*(m-l+1) entries for at least 32 warps.  A request that does not fit
 * returns PMS_E_NOMEM (nothing runs); more raw finds than fit returns PMS_E_OVERFLOW.
 * With the default threshold, DNA instances up to n=20, m=1000 fit.
 *
 * The first call on each device looks up the array's device address; make that first call
 * before any stream capture.  Every call reuses the same array (each call clears what it
 * needs), so calls must not overlap on the GPU: calls from several host threads are
 * serialised inside the library, but two processes or overlapping streams sharing a
 * device must not call it at the same time.
 */
int pms_solve_device_noalloc(const char *d_seqs, int n, int m, const char *alphabet, int l,
                             int d, int threshold, char *d_motifs, uint64_t cap,
                             uint64_t *count, void *stream);

/* Serving: queue an instance (inputs are copied before return) and get a ticket. */
int pms_submit(pms_ctx *ctx, const pms_instance *inst, uint64_t *ticket);

/* Serving: non-blocking check of a ticket.  *done = 1 and *out filled (ownership passes
 * to the caller; the ticket is retired) when finished; *done = 0 otherwise.  The return
 * value is the solve's own status once done. */
int pms_poll(pms_ctx *ctx, uint64_t ticket, pms_result *out, int *done);

/* Serving: block until a ticket finishes, for at most timeout_ms milliseconds (negative:
 * no limit).  When it finishes, *out is filled (ownership passes to the caller; the
 * ticket is retired) and the return value is the solve's own status.  PMS_E_TIMEOUT: the
 * wait expired, nothing changed and the ticket stays valid.  PMS_E_NOTFOUND: unknown or
 * retired ticket, or the context is being destroyed.  Any thread may wait; each ticket's
 * result goes to one caller.  (A serving convenience; the paper has no counterpart.) */
int pms_wait(pms_ctx *ctx, uint64_t ticket, pms_result *out, int timeout_ms);

/* Release the motif buffer of a result (safe on zeroed results). */
void pms_result_free(pms_result *res);

/* Static description of an error code. */
const char *pms_strerror(int code);

/* Number of instance classes (l, d, alphabet size, and n and m rounded to powers of two)
 * whose threshold the autotuner has cached, and a reset of that cache. */
int pms_autotune_entries(pms_ctx *ctx);
void pms_autotune_reset(pms_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* PMS_H */
