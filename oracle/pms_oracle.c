/*
 * Plain CPU oracle for exact planted (l,d) motif search.
 *
 * TEST INFRASTRUCTURE.  This library exists to check the CUDA path.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it; the product path never
 * calls it, and it shares no code, header, table or helper with the CUDA path.
 *
 * Everything works on letter codes 0..k-1 (one byte per letter, no packing) and on
 * character-by-character loops, so each function can be checked against the paper by eye.
 *
 *   oracle_hd            Hamming distance (Section 1).
 *   oracle_cd            Consensus total distance Cd(T) (Definition 1, Section 2.4).
 *   oracle_theorem1      The three-l-mer condition of Theorem 1 (Section 2.4).
 *   oracle_theorem1_witness  A common neighbour built as in the proof of Theorem 1.
 *   oracle_neighborhood  Algorithm 1 (Appendix A), common d-neighbourhood of a tuple.
 *   oracle_is_motif      The motif predicate of Section 1 for one l-mer.
 *   oracle_motifs_def    The motif set straight from the definition (Section 1): every motif
 *                        is within d of some l-mer of S_1, so the candidates are the
 *                        d-neighbourhoods of the l-mers of S_1, each tested directly against
 *                        every string.
 *   oracle_motifs_pms8   Algorithm 2 (Appendix B) with the filters of Section 2 (2d filter,
 *                        Theorem 1 for triples), rows sorted by size (Section 2.1), and
 *                        Algorithm 1 for the pattern-driven part.  A second, faster oracle for
 *                        sizes where the definition is too slow; pinned to the definition.
 *
 * Motif sets come back sorted ascending by code (the alphabet's order) with duplicates
 * removed, as count*l code bytes in a buffer the caller frees with oracle_free.
 */
#define _GNU_SOURCE
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

/* ---------------------------------------------------------------- basics (Section 1) */

/* Hd(u,v): the number of positions where the two l-mers differ (Section 1). */
int oracle_hd(const uint8_t *u, const uint8_t *v, int l)
{
    int c = 0;
    for (int i = 0; i < l; i++)
        if (u[i] != v[i])
            c++;
    return c;
}

/* Hd(u,v) <= d, stopping at the first position that makes it false. */
static int within(const uint8_t *u, const uint8_t *v, int l, int d)
{
    int c = 0;
    for (int i = 0; i < l; i++)
        if (u[i] != v[i] && ++c > d)
            return 0;
    return 1;
}

/*
 * Consensus total distance (Definition 1, Section 2.4): for k l-mers T_1..T_k, column i
 * contributes k - m_i where m_i is the highest frequency of any letter in that column.
 * `tuple` holds the k l-mers back to back (k*l bytes).  Letters are codes below 256.
 */
int oracle_cd(const uint8_t *tuple, int k, int l)
{
    int total = 0;
    for (int i = 0; i < l; i++) {
        int freq[256];
        memset(freq, 0, sizeof freq);
        int best = 0;
        for (int j = 0; j < k; j++) {
            int f = ++freq[tuple[j * l + i]];
            if (f > best)
                best = f;
        }
        total += k - best;
    }
    return total;
}

/* Cd of three l-mers given by pointers (same definition as oracle_cd). */
static int cd3(const uint8_t *a, const uint8_t *b, const uint8_t *c, int len)
{
    int total = 0;
    for (int i = 0; i < len; i++) {
        int best = 1;
        if (a[i] == b[i] || a[i] == c[i] || b[i] == c[i])
            best = 2;
        if (a[i] == b[i] && b[i] == c[i])
            best = 3;
        total += 3 - best;
    }
    return total;
}

/*
 * Theorem 1 (Section 2.4): three l-mers a, b, c have a common neighbour M with
 * Hd(M,a) <= da, Hd(M,b) <= db, Hd(M,c) <= dc if and only if
 *   (i)  Cd(a,b) <= da+db, Cd(a,c) <= da+dc, Cd(b,c) <= db+dc   (Cd of two l-mers is Hd), and
 *   (ii) Cd(a,b,c) <= da+db+dc.
 * Negative budgets admit no neighbour.
 */
int oracle_theorem1(const uint8_t *a, const uint8_t *b, const uint8_t *c, int l,
                    int da, int db, int dc)
{
    if (da < 0 || db < 0 || dc < 0)
        return 0;
    if (oracle_hd(a, b, l) > da + db)
        return 0;
    if (oracle_hd(a, c, l) > da + dc)
        return 0;
    if (oracle_hd(b, c, l) > db + dc)
        return 0;
    return cd3(a, b, c, l) <= da + db + dc;
}

/*
 * The "if" half of Theorem 1 made constructive, following its proof (Section 2.4).  Columns
 * are typed by which l-mer is the odd one out: N0 all equal, N_i only T_i differs (the
 * other two agree), N4 all three distinct; n_i counts them.
 *   Case 1, some n_i >= d_i: M copies T_i except in d_i columns of type N_i, where it takes
 *     the letter the other two share.  Then Hd(M,T_i) = d_i and, M lying on a shortest
 *     path from T_i to T_j, Hd(M,T_j) = Hd(T_i,T_j) - d_i <= d_j.
 *   Case 2, every n_i < d_i: M takes the majority letter in every column of type N0..N3,
 *     so Hd(M,T_i) = n_i plus its mismatches in N4 columns; then for each i it copies T_i
 *     in max(0, n_i + n4 - d_i) of the N4 columns not yet used.  The conditions of the
 *     theorem are exactly what makes these choices fit in the n4 columns.
 * Writes M (l codes) and returns 1 when the conditions of Theorem 1 hold; returns 0 and
 * leaves M untouched otherwise.
 */
int oracle_theorem1_witness(const uint8_t *a, const uint8_t *b, const uint8_t *c, int l,
                            int da, int db, int dc, uint8_t *M)
{
    const uint8_t *T[3] = {a, b, c};
    const int dd[3] = {da, db, dc};
    int type_n[5] = {0, 0, 0, 0, 0};
    if (!oracle_theorem1(a, b, c, l, da, db, dc))
        return 0;
    for (int k = 0; k < l; k++) {
        const int e12 = a[k] == b[k], e13 = a[k] == c[k], e23 = b[k] == c[k];
        type_n[e12 && e13 ? 0 : e23 ? 1 : e13 ? 2 : e12 ? 3 : 4]++;
    }
    for (int i = 0; i < 3; i++) {
        if (type_n[i + 1] >= dd[i]) {   /* case 1 with T_i */
            const int j = (i + 1) % 3;
            int left = dd[i];
            for (int k = 0; k < l; k++) {
                const int e12 = a[k] == b[k], e13 = a[k] == c[k], e23 = b[k] == c[k];
                const int ty = e12 && e13 ? 0 : e23 ? 1 : e13 ? 2 : e12 ? 3 : 4;
                if (ty == i + 1 && left > 0) {
                    M[k] = T[j][k];
                    left--;
                } else {
                    M[k] = T[i][k];
                }
            }
            return 1;
        }
    }
    /* case 2 */
    int want[3];
    for (int i = 0; i < 3; i++) {
        want[i] = type_n[i + 1] + type_n[4] - dd[i];
        if (want[i] < 0)
            want[i] = 0;
    }
    for (int k = 0; k < l; k++) {
        const int e12 = a[k] == b[k], e13 = a[k] == c[k], e23 = b[k] == c[k];
        const int ty = e12 && e13 ? 0 : e23 ? 1 : e13 ? 2 : e12 ? 3 : 4;
        if (ty == 1) {
            M[k] = b[k];
        } else if (ty != 4) {
            M[k] = a[k];
        } else {
            int pick = 0;
            while (pick < 3 && want[pick] == 0)
                pick++;
            if (pick < 3) {
                M[k] = T[pick][k];
                want[pick]--;
            } else {
                M[k] = a[k];
            }
        }
    }
    return 1;
}

/* ------------------------------------------------------------ growable motif list */

typedef struct {
    uint8_t *buf;
    size_t count, cap;
    int l;
    int oom;
} mlist;

static void ml_push(mlist *ml, const uint8_t *M)
{
    if (ml->oom)
        return;
    if (ml->count == ml->cap) {
        size_t nc = ml->cap ? ml->cap * 2 : 1024;
        uint8_t *nb = realloc(ml->buf, nc * (size_t)ml->l);
        if (!nb) {
            ml->oom = 1;
            return;
        }
        ml->buf = nb;
        ml->cap = nc;
    }
    memcpy(ml->buf + ml->count * (size_t)ml->l, M, (size_t)ml->l);
    ml->count++;
}

static int cmp_lmer(const void *x, const void *y, void *arg)
{
    return memcmp(x, y, (size_t)(intptr_t)arg);
}

/* Sort ascending by code and drop duplicates, in place. */
static void ml_sort_unique(mlist *ml)
{
    if (ml->count == 0)
        return;
    qsort_r(ml->buf, ml->count, (size_t)ml->l, cmp_lmer, (void *)(intptr_t)ml->l);
    size_t w = 1;
    for (size_t r = 1; r < ml->count; r++) {
        const uint8_t *cur = ml->buf + r * (size_t)ml->l;
        const uint8_t *last = ml->buf + (w - 1) * (size_t)ml->l;
        if (memcmp(cur, last, (size_t)ml->l) != 0) {
            if (w != r)
                memmove(ml->buf + w * (size_t)ml->l, cur, (size_t)ml->l);
            w++;
        }
    }
    ml->count = w;
}

void oracle_free(void *p)
{
    free(p);
}

/* ------------------------------------------------------ Algorithm 1 (Appendix A) */

/*
 * GenerateNeighborhood(T, d) of Appendix A: a depth-first walk over positions p = 0..l-1.
 * Every l-mer T_i carries a budget r_i, initially d.  Choosing letter alpha at position p
 * lowers r_i by one for every T_i whose letter there differs from alpha.  A node is cut by
 * prune(T, r), which the paper leaves undefined; any condition that holds whenever a
 * completion exists is correct.  This one cuts when
 *   - some r_i < 0,
 *   - some pair has Hd(T_i[p..], T_j[p..]) > r_i + r_j        (two-l-mer condition, §2.4),
 *   - some triple has Cd(T_i[p..], T_j[p..], T_k[p..]) > r_i + r_j + r_k   (Lemma 1 and
 *     Theorem 1 on the remaining columns).
 * At p = l the l-mer is reported when every r_i >= 0.
 */
typedef struct {
    const uint8_t *const *T;
    int t, l, k;
    uint8_t *M;
    int *r;     /* (l+1) levels of t budgets */
    mlist *out;
    long long nodes;
} nb_walk;

static int prune(const nb_walk *w, const int *r, int p)
{
    int rem = w->l - p;
    for (int i = 0; i < w->t; i++)
        if (r[i] < 0)
            return 1;
    for (int i = 0; i < w->t; i++)
        for (int j = i + 1; j < w->t; j++)
            if (oracle_hd(w->T[i] + p, w->T[j] + p, rem) > r[i] + r[j])
                return 1;
    for (int i = 0; i < w->t; i++)
        for (int j = i + 1; j < w->t; j++)
            for (int q = j + 1; q < w->t; q++)
                if (cd3(w->T[i] + p, w->T[j] + p, w->T[q] + p, rem) > r[i] + r[j] + r[q])
                    return 1;
    return 0;
}

static void nb_rec(nb_walk *w, int p)
{
    const int *r = w->r + (size_t)p * w->t;
    w->nodes++;
    if (p == w->l) {
        for (int i = 0; i < w->t; i++)
            if (r[i] < 0)
                return;
        ml_push(w->out, w->M);
        return;
    }
    if (prune(w, r, p))
        return;
    int *rn = w->r + (size_t)(p + 1) * w->t;
    for (int alpha = 0; alpha < w->k; alpha++) {
        w->M[p] = (uint8_t)alpha;
        for (int i = 0; i < w->t; i++)
            rn[i] = r[i] - (w->T[i][p] != alpha);
        nb_rec(w, p + 1);
    }
}

static int neighborhood(const uint8_t *const *T, int t, int l, int k, int d, mlist *out)
{
    nb_walk w;
    w.T = T;
    w.t = t;
    w.l = l;
    w.k = k;
    w.out = out;
    w.nodes = 0;
    w.M = malloc((size_t)l);
    w.r = malloc(sizeof(int) * (size_t)(l + 1) * (size_t)(t > 0 ? t : 1));
    if (!w.M || !w.r) {
        free(w.M);
        free(w.r);
        return -1;
    }
    for (int i = 0; i < t; i++)
        w.r[i] = d;
    nb_rec(&w, 0);
    free(w.M);
    free(w.r);
    return 0;
}

/*
 * Common d-neighbourhood of the t l-mers in `tuple` (t*l code bytes), by Algorithm 1.
 * Returns the number of l-mers (sorted, unique) and stores them in *out (caller frees
 * with oracle_free), or -1 on allocation failure.
 */
long long oracle_neighborhood(const uint8_t *tuple, int t, int l, int k, int d,
                              uint8_t **out)
{
    const uint8_t **T = malloc(sizeof(*T) * (size_t)(t > 0 ? t : 1));
    if (!T)
        return -1;
    for (int i = 0; i < t; i++)
        T[i] = tuple + (size_t)i * l;
    mlist ml = {0};
    ml.l = l;
    int rc = neighborhood(T, t, l, k, d, &ml);
    free(T);
    if (rc != 0 || ml.oom) {
        free(ml.buf);
        return -1;
    }
    ml_sort_unique(&ml);
    *out = ml.buf;
    return (long long)ml.count;
}

/* ------------------------------------------------------------- motif predicate */

/*
 * Section 1: M is a motif iff for every string S_i some l-mer S_i[j..j+l-1],
 * 0 <= j <= m-l, has Hd(M, S_i[j..j+l-1]) <= d.  `S` is n*m codes, row-major.
 */
int oracle_is_motif(const uint8_t *M, const uint8_t *S, int n, int m, int l, int d)
{
    for (int i = 0; i < n; i++) {
        int found = 0;
        for (int j = 0; j + l <= m && !found; j++)
            found = within(M, S + (size_t)i * m + j, l, d);
        if (!found)
            return 0;
    }
    return 1;
}

/* ----------------------------------------------------------- threaded drivers */

typedef struct job job;
typedef void (*x_fn)(job *jb, mlist *out, int x, void *scratch);

struct job {
    const uint8_t *S;
    int n, m, k, l, d, t;
    int x_begin, x_end;
    int next;                 /* next x to hand out */
    pthread_mutex_t lock;
    x_fn fn;
    size_t scratch_bytes;
    int failed;
};

typedef struct {
    job *jb;
    mlist out;
} worker;

static void *worker_main(void *arg)
{
    worker *wk = arg;
    job *jb = wk->jb;
    void *scratch = jb->scratch_bytes ? malloc(jb->scratch_bytes) : NULL;
    if (jb->scratch_bytes && !scratch) {
        pthread_mutex_lock(&jb->lock);
        jb->failed = 1;
        pthread_mutex_unlock(&jb->lock);
        return NULL;
    }
    for (;;) {
        pthread_mutex_lock(&jb->lock);
        int x = jb->next < jb->x_end ? jb->next++ : -1;
        pthread_mutex_unlock(&jb->lock);
        if (x < 0)
            break;
        jb->fn(jb, &wk->out, x, scratch);
    }
    free(scratch);
    return NULL;
}

/* Run fn over x in [x_begin, x_end) on `threads` threads, merge, sort and dedupe. */
static long long run_job(job *jb, int threads, uint8_t **out)
{
    if (threads <= 0) {
        long c = sysconf(_SC_NPROCESSORS_ONLN);
        threads = c > 0 ? (int)c : 1;
    }
    worker *wk = calloc((size_t)threads, sizeof(worker));
    pthread_t *th = calloc((size_t)threads, sizeof(pthread_t));
    if (!wk || !th) {
        free(wk);
        free(th);
        return -1;
    }
    pthread_mutex_init(&jb->lock, NULL);
    jb->next = jb->x_begin;
    jb->failed = 0;
    int started = 0;
    for (int i = 0; i < threads; i++) {
        wk[i].jb = jb;
        wk[i].out.l = jb->l;
        if (pthread_create(&th[i], NULL, worker_main, &wk[i]) == 0)
            started++;
        else
            break;
    }
    if (started == 0)
        worker_main(&wk[0]);
    for (int i = 0; i < started; i++)
        pthread_join(th[i], NULL);
    pthread_mutex_destroy(&jb->lock);

    mlist all = {0};
    all.l = jb->l;
    int bad = jb->failed;
    for (int i = 0; i < threads; i++) {
        if (wk[i].out.oom)
            bad = 1;
        for (size_t c = 0; c < wk[i].out.count && !bad; c++)
            ml_push(&all, wk[i].out.buf + c * (size_t)jb->l);
        free(wk[i].out.buf);
    }
    free(wk);
    free(th);
    if (bad || all.oom) {
        free(all.buf);
        return -1;
    }
    ml_sort_unique(&all);
    *out = all.buf;
    return (long long)all.count;
}

static int check_args(const uint8_t *S, int n, int m, int k, int l, int d, int xb, int xe)
{
    if (!S || n < 1 || l < 1 || m < l || k < 2 || k > 256 || d < 0)
        return -1;
    if (xb < 0 || xe < xb || xe > m - l + 1)
        return -1;
    for (size_t i = 0; i < (size_t)n * m; i++)
        if (S[i] >= k)
            return -1;
    return 0;
}

/* ----------------------------------------------- the definition (Section 1) */

/*
 * Candidates for subproblem x: the d-neighbourhood of x = S_1[x..x+l-1] (every motif is
 * within d of the l-mer where it occurs in S_1).  The neighbourhood is walked position by
 * position with one budget (Algorithm 1 with a single l-mer and only the r < 0 cut), and
 * every neighbour is tested against all n strings by the Section 1 predicate.
 */
typedef struct {
    job *jb;
    const uint8_t *x;
    uint8_t *M;
    mlist *out;
} def_walk;

static void def_rec(def_walk *w, int p, int budget)
{
    const job *jb = w->jb;
    if (p == jb->l) {
        if (oracle_is_motif(w->M, jb->S, jb->n, jb->m, jb->l, jb->d))
            ml_push(w->out, w->M);
        return;
    }
    w->M[p] = w->x[p];
    def_rec(w, p + 1, budget);
    if (budget == 0)
        return;
    for (int alpha = 0; alpha < jb->k; alpha++) {
        if (alpha == w->x[p])
            continue;
        w->M[p] = (uint8_t)alpha;
        def_rec(w, p + 1, budget - 1);
    }
}

static void def_x(job *jb, mlist *out, int x, void *scratch)
{
    def_walk w;
    w.jb = jb;
    w.x = jb->S + x;          /* row 0 is S_1 */
    w.M = scratch;
    w.out = out;
    def_rec(&w, 0, jb->d);
}

/*
 * The motif set by definition, from the candidates of the l-mers x_begin..x_end-1 of S_1
 * (the whole set when the range is [0, m-l+1)).  Returns the count, or -1 on bad
 * arguments or allocation failure.
 */
long long oracle_motifs_def(const uint8_t *S, int n, int m, int k, int l, int d,
                            int x_begin, int x_end, int threads, uint8_t **out)
{
    if (check_args(S, n, m, k, l, d, x_begin, x_end) != 0)
        return -1;
    job jb = {0};
    jb.S = S;
    jb.n = n;
    jb.m = m;
    jb.k = k;
    jb.l = l;
    jb.d = d;
    jb.x_begin = x_begin;
    jb.x_end = x_end;
    jb.fn = def_x;
    jb.scratch_bytes = (size_t)l;
    return run_job(&jb, threads, out);
}

/* ------------------------------------------- Algorithm 2 (Appendix B), plainly */

/*
 * Work space of one thread for Algorithm 2.  Level `lev` (the stack size) keeps, for each
 * string not yet on the stack, the list of surviving l-mer start offsets (into S) and its
 * length.  Every level owns its own copy: a plain restatement, not the in-place update of
 * Section 2.1.
 */
typedef struct {
    int *off;         /* (n+1) levels * n rows * L offsets */
    int *cnt;         /* (n+1) levels * n counts */
    int *row;         /* (n+1) levels * n row ids, in the order rows are kept */
    int *nrows;       /* (n+1) row counts per level */
    const uint8_t **stack;
} pms8_ws;

static size_t pms8_scratch_bytes(int n, int L)
{
    size_t lv = (size_t)n + 1;
    return lv * n * L * sizeof(int) + 3 * lv * n * sizeof(int) + lv * sizeof(int) +
           ((size_t)n + 1) * sizeof(uint8_t *) + 64;
}

static pms8_ws ws_view(void *scratch, int n, int L)
{
    pms8_ws w;
    size_t lv = (size_t)n + 1;
    char *p = scratch;
    w.off = (int *)p;
    p += lv * n * L * sizeof(int);
    w.cnt = (int *)p;
    p += lv * n * sizeof(int);
    w.row = (int *)p;
    p += lv * n * sizeof(int);
    w.nrows = (int *)p;
    p += lv * sizeof(int);
    p += (8 - ((uintptr_t)p & 7)) & 7;
    w.stack = (const uint8_t **)p;
    return w;
}

/*
 * The leaf of Algorithm 2: generate the common d-neighbourhood of the stack with
 * Algorithm 1 and output every neighbour M that isMotif(M, R') accepts, i.e. every M such
 * that each remaining row of R' holds an l-mer u with Hd(M,u) <= d.  Checking R' instead
 * of the whole string loses nothing: an l-mer within d of a common neighbour of the stack
 * passes every necessary filter, so it is still in R'.
 */
static void pms8_leaf(job *jb, pms8_ws *w, int lev, mlist *out)
{
    int L = jb->m - jb->l + 1;
    mlist nb = {0};
    nb.l = jb->l;
    if (neighborhood(w->stack, lev, jb->l, jb->k, jb->d, &nb) != 0 || nb.oom) {
        free(nb.buf);
        out->oom = 1;
        return;
    }
    int nr = w->nrows[lev];
    const int *off = w->off + (size_t)lev * jb->n * L;
    const int *cnt = w->cnt + (size_t)lev * jb->n;
    for (size_t c = 0; c < nb.count; c++) {
        const uint8_t *M = nb.buf + c * (size_t)jb->l;
        int ok = 1;
        for (int r = 0; r < nr && ok; r++) {
            int found = 0;
            for (int j = 0; j < cnt[r] && !found; j++)
                found = within(M, jb->S + off[(size_t)r * L + j], jb->l, jb->d);
            ok = found;
        }
        if (ok)
            ml_push(out, M);
    }
    free(nb.buf);
}

/*
 * GenerateMotifs of Algorithm 2 at stack size `lev`: the rows of level `lev` are already
 * filtered against the stack and none is empty.  When the threshold is reached (stack
 * size t) or no row is left, the pattern-driven part runs; otherwise the rows are sorted
 * by size (Section 2.1), every l-mer u of the smallest row is pushed in turn, and the other
 * rows are filtered: v survives when Hd(u,v) <= 2d and, for every l-mer s already on the
 * stack, s, u and v meet Theorem 1 with budgets (d,d,d).  When a row empties, u is
 * abandoned (Section 2).
 */
static void pms8_rec(job *jb, pms8_ws *w, int lev, mlist *out)
{
    int n = jb->n, l = jb->l, d = jb->d;
    int L = jb->m - l + 1;
    int nr = w->nrows[lev];
    if (lev >= jb->t || nr == 0) {
        pms8_leaf(jb, w, lev, out);
        return;
    }
    int *off = w->off + (size_t)lev * n * L;
    int *cnt = w->cnt + (size_t)lev * n;
    int *row = w->row + (size_t)lev * n;
    /* sort rows by size, ascending (insertion sort: stable, ties keep string order) */
    for (int a = 1; a < nr; a++) {
        for (int b = a; b > 0 && cnt[b] < cnt[b - 1]; b--) {
            int tc = cnt[b];
            cnt[b] = cnt[b - 1];
            cnt[b - 1] = tc;
            int tr = row[b];
            row[b] = row[b - 1];
            row[b - 1] = tr;
            int span = cnt[b] > cnt[b - 1] ? cnt[b] : cnt[b - 1];
            for (int j = 0; j < span; j++) {
                int to = off[(size_t)b * L + j];
                off[(size_t)b * L + j] = off[(size_t)(b - 1) * L + j];
                off[(size_t)(b - 1) * L + j] = to;
            }
        }
    }
    int *noff = w->off + (size_t)(lev + 1) * n * L;
    int *ncnt = w->cnt + (size_t)(lev + 1) * n;
    int *nrow = w->row + (size_t)(lev + 1) * n;
    for (int c = 0; c < cnt[0]; c++) {
        const uint8_t *u = jb->S + off[c];
        w->stack[lev] = u;
        int alive = 1;
        for (int r = 1; r < nr && alive; r++) {
            int kept = 0;
            for (int j = 0; j < cnt[r]; j++) {
                const uint8_t *v = jb->S + off[(size_t)r * L + j];
                int ok = oracle_hd(u, v, l) <= 2 * d;
                for (int s = 0; s < lev && ok; s++)
                    ok = oracle_theorem1(w->stack[s], u, v, l, d, d, d);
                if (ok)
                    noff[(size_t)(r - 1) * L + kept++] = off[(size_t)r * L + j];
            }
            ncnt[r - 1] = kept;
            nrow[r - 1] = row[r];
            alive = kept > 0;
        }
        if (!alive)
            continue;
        w->nrows[lev + 1] = nr - 1;
        pms8_rec(jb, w, lev + 1, out);
    }
}

/*
 * One subproblem of Section 2.3: row 1 of R is the single l-mer x = S_1[x..x+l-1].
 * x goes on the stack and every other row keeps the l-mers within 2d of it (Section 2).
 */
static void pms8_x(job *jb, mlist *out, int x, void *scratch)
{
    int n = jb->n, m = jb->m, l = jb->l, d = jb->d;
    int L = m - l + 1;
    pms8_ws w = ws_view(scratch, n, L);
    const uint8_t *xs = jb->S + x;
    w.stack[0] = xs;
    int *off = w.off + (size_t)1 * n * L;
    int *cnt = w.cnt + (size_t)1 * n;
    int *row = w.row + (size_t)1 * n;
    for (int i = 1; i < n; i++) {
        int kept = 0;
        for (int j = 0; j < L; j++) {
            const uint8_t *u = jb->S + (size_t)i * m + j;
            if (oracle_hd(xs, u, l) <= 2 * d)
                off[(size_t)(i - 1) * L + kept++] = i * m + j;
        }
        if (kept == 0)
            return;
        cnt[i - 1] = kept;
        row[i - 1] = i;
    }
    w.nrows[1] = n - 1;
    pms8_rec(jb, &w, 1, out);
}

/*
 * The motif set by Algorithm 2 over the subproblems x_begin..x_end-1, switching to the
 * pattern-driven part at stack size t (t >= 1; the set does not depend on t).
 */
long long oracle_motifs_pms8(const uint8_t *S, int n, int m, int k, int l, int d, int t,
                             int x_begin, int x_end, int threads, uint8_t **out)
{
    if (check_args(S, n, m, k, l, d, x_begin, x_end) != 0 || t < 1)
        return -1;
    job jb = {0};
    jb.S = S;
    jb.n = n;
    jb.m = m;
    jb.k = k;
    jb.l = l;
    jb.d = d;
    jb.t = t;
    jb.x_begin = x_begin;
    jb.x_end = x_end;
    jb.fn = pms8_x;
    jb.scratch_bytes = pms8_scratch_bytes(n, m - l + 1);
    return run_job(&jb, threads, out);
}
