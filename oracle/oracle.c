/*
 * CPU oracle for exhaustive dense-QUBO minimisation.
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the CPU-baseline leg of the
 * benchmark load this library; the product (the CUDA library and its Python binding) never
 * does, and shares no code with it.
 *
 * What is computed (Sec. 1, the objective E(x) = sum_{i,j} Q_ij x_i x_j, x in {0,1}^n):
 *   - E_min, the exact minimum over every state of the (sub)cube;
 *   - the tie set {x : E(x) = E_min}: its exact size, and its `cap` smallest codes ascending;
 *   - the K lowest states ordered by (E, code) ascending (the "k lowest energies" list of
 *     Sec. 6.2, counted with multiplicity).
 * A state code holds variable i in bit i.  A sub-cube fixes the top `fix_bits` bits of the
 * code to `fix_value` (the fixed-prefix split of Sec. 3.3.1).
 *
 * Q may be any square matrix; the objective sums every entry, so Q is first folded into the
 * upper-triangular U with U_ii = Q_ii and U_ij = Q_ij + Q_ji for i < j (Sec. 2.1 works with
 * an upper-triangular Q; the fold gives the same E for every x).
 *
 * Two evaluators, neither of which uses the prefix/suffix tables of Sec. 2-3:
 *   direct: the O(n^2)-per-state evaluation (the naive brute force of Sec. 1.4), in one
 *           fixed order: i ascending, then j ascending over the upper triangle.  For floats
 *           this order defines the reference FP64 energy.
 *   gray:   the O(n)-per-state method of Sec. 1.4: states are visited in reflected Gray
 *           order (Sec. 3.2, Fig. "3-bit Gray code"), so consecutive states differ in one
 *           bit k, and E changes by (U_kk + h_k) with the sign of the flip, where
 *           h_k = sum_{j != k} U_{min(j,k),max(j,k)} x_j is kept up to date in O(n) per flip.
 *           Integers are exact.  For floats the walk only pre-selects candidates within a
 *           rigorous error bound of the running K-th best; every candidate is re-evaluated
 *           by the direct evaluator, and those values decide the answer.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------ */
/* Fold and direct energies.                                                             */
/* ------------------------------------------------------------------------------------ */

void oracle_fold_i64(const int64_t *Q, int n, int64_t *U)
{
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            if (i == j)
                U[i * n + j] = Q[i * n + i];
            else if (i < j)
                U[i * n + j] = Q[i * n + j] + Q[j * n + i];
            else
                U[i * n + j] = 0;
        }
}

void oracle_fold_f64(const double *Q, int n, double *U)
{
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            if (i == j)
                U[i * n + j] = Q[i * n + i];
            else if (i < j)
                U[i * n + j] = Q[i * n + j] + Q[j * n + i];
            else
                U[i * n + j] = 0.0;
        }
}

/* E(x) = sum_i U_ii x_i + sum_{i<j} U_ij x_i x_j, accumulated i ascending then j ascending. */
int64_t oracle_energy_i64(const int64_t *U, int n, uint64_t x)
{
    int64_t acc = 0;
    for (int i = 0; i < n; i++) {
        if (!((x >> i) & 1u))
            continue;
        acc += U[i * n + i];
        for (int j = i + 1; j < n; j++)
            if ((x >> j) & 1u)
                acc += U[i * n + j];
    }
    return acc;
}

double oracle_energy_f64(const double *U, int n, uint64_t x)
{
    double acc = 0.0;
    for (int i = 0; i < n; i++) {
        if (!((x >> i) & 1u))
            continue;
        acc += U[i * n + i];
        for (int j = i + 1; j < n; j++)
            if ((x >> j) & 1u)
                acc += U[i * n + j];
    }
    return acc;
}

/* Reflected binary Gray code: the i-th state of the walk (Sec. 3.2). */
uint64_t oracle_gray_code(uint64_t i) { return i ^ (i >> 1); }

/* Energies along a full Gray walk of all 2^n states, by the O(n) field update; out[i] is the
 * energy of state oracle_gray_code(i).  Used to pin the walk against the direct evaluator. */
void oracle_gray_walk_i64(const int64_t *U, int n, int64_t *out)
{
    int64_t h[64];
    uint64_t x = 0;
    int64_t E = 0;
    for (int j = 0; j < n; j++)
        h[j] = 0;
    out[0] = 0;
    uint64_t total = 1ull << n;
    for (uint64_t t = 0; t + 1 < total; t++) {
        int k = __builtin_ctzll(t + 1);
        x ^= 1ull << k;
        int up = (int)((x >> k) & 1u);
        int64_t d = U[k * n + k] + h[k];
        E += up ? d : -d;
        for (int j = 0; j < n; j++) {
            if (j == k)
                continue;
            int64_t w = j < k ? U[j * n + k] : U[k * n + j];
            h[j] += up ? w : -w;
        }
        out[t + 1] = E;
    }
}

/* ------------------------------------------------------------------------------------ */
/* Result collector: minimum, tie set (exact count, `cap` smallest codes), K lowest states. */
/* ------------------------------------------------------------------------------------ */

#define ORACLE_MAX_K 4096

typedef struct {
    int K;
    uint64_t cap;
    int has;
    double emin;      /* energies are held as double for floats, as int64 for integers */
    int64_t emin_i;
    uint64_t nties;
    uint64_t *heap;   /* max-heap of the smallest tie codes, size <= cap */
    uint64_t nheap;
    int nk;
    double *topE;
    int64_t *topE_i;
    uint64_t *topC;
} coll_t;

static int coll_init(coll_t *c, int K, uint64_t cap)
{
    memset(c, 0, sizeof(*c));
    c->K = K;
    c->cap = cap;
    c->heap = (uint64_t *)malloc(sizeof(uint64_t) * (cap ? cap : 1));
    c->topE = (double *)malloc(sizeof(double) * (K ? K : 1));
    c->topE_i = (int64_t *)malloc(sizeof(int64_t) * (K ? K : 1));
    c->topC = (uint64_t *)malloc(sizeof(uint64_t) * (K ? K : 1));
    return (c->heap && c->topE && c->topE_i && c->topC) ? 0 : -1;
}

static void coll_free(coll_t *c)
{
    free(c->heap);
    free(c->topE);
    free(c->topE_i);
    free(c->topC);
}

static void heap_clear(coll_t *c) { c->nheap = 0; }

/* Keep the `cap` smallest codes: a max-heap whose root is the largest kept code. */
static void heap_offer(coll_t *c, uint64_t code)
{
    if (c->cap == 0)
        return;
    if (c->nheap < c->cap) {
        uint64_t i = c->nheap++;
        c->heap[i] = code;
        while (i > 0) {
            uint64_t p = (i - 1) / 2;
            if (c->heap[p] >= c->heap[i])
                break;
            uint64_t t = c->heap[p];
            c->heap[p] = c->heap[i];
            c->heap[i] = t;
            i = p;
        }
        return;
    }
    if (code >= c->heap[0])
        return;
    c->heap[0] = code;
    uint64_t i = 0;
    for (;;) {
        uint64_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < c->nheap && c->heap[l] > c->heap[m])
            m = l;
        if (r < c->nheap && c->heap[r] > c->heap[m])
            m = r;
        if (m == i)
            break;
        uint64_t t = c->heap[m];
        c->heap[m] = c->heap[i];
        c->heap[i] = t;
        i = m;
    }
}

/* (E, code) ordering; `isint` selects which energy field is meaningful. */
static int less_ec(int isint, double ea, int64_t eai, uint64_t ca, double eb, int64_t ebi, uint64_t cb)
{
    if (isint) {
        if (eai != ebi)
            return eai < ebi;
    } else {
        if (ea != eb)
            return ea < eb;
    }
    return ca < cb;
}

static void topk_offer(coll_t *c, int isint, double E, int64_t Ei, uint64_t code)
{
    if (c->K == 0)
        return;
    if (c->nk == c->K &&
        !less_ec(isint, E, Ei, code, c->topE[c->nk - 1], c->topE_i[c->nk - 1], c->topC[c->nk - 1]))
        return;
    int pos = c->nk < c->K ? c->nk : c->K - 1;
    while (pos > 0 && less_ec(isint, E, Ei, code, c->topE[pos - 1], c->topE_i[pos - 1], c->topC[pos - 1])) {
        c->topE[pos] = c->topE[pos - 1];
        c->topE_i[pos] = c->topE_i[pos - 1];
        c->topC[pos] = c->topC[pos - 1];
        pos--;
    }
    c->topE[pos] = E;
    c->topE_i[pos] = Ei;
    c->topC[pos] = code;
    if (c->nk < c->K)
        c->nk++;
}

static void coll_feed_i64(coll_t *c, int64_t E, uint64_t code)
{
    if (!c->has || E < c->emin_i) {
        c->has = 1;
        c->emin_i = E;
        c->nties = 1;
        heap_clear(c);
        heap_offer(c, code);
    } else if (E == c->emin_i) {
        c->nties++;
        heap_offer(c, code);
    }
    topk_offer(c, 1, 0.0, E, code);
}

static void coll_feed_f64(coll_t *c, double E, uint64_t code)
{
    if (!c->has || E < c->emin) {
        c->has = 1;
        c->emin = E;
        c->nties = 1;
        heap_clear(c);
        heap_offer(c, code);
    } else if (E == c->emin) {
        c->nties++;
        heap_offer(c, code);
    }
    topk_offer(c, 0, E, 0, code);
}

/* The largest energy that can still change the collector's result (ints). */
static int coll_needs_i64(const coll_t *c, int64_t E)
{
    if (!c->has)
        return 1;
    if (E <= c->emin_i)
        return 1;
    return c->K > 0 && (c->nk < c->K || E <= c->topE_i[c->nk - 1]);
}

static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : x > y;
}

/* Merge per-thread collectors and write the outputs. */
static void coll_merge_out(coll_t *cs, int nc, int isint, int K, uint64_t cap, void *out_min,
                           uint64_t *out_nties, uint64_t *out_ties, uint64_t *out_nwritten,
                           uint64_t *out_topk, void *out_topkE, int *out_nk)
{
    int have = 0;
    double gmin = 0.0;
    int64_t gmin_i = 0;
    for (int t = 0; t < nc; t++) {
        if (!cs[t].has)
            continue;
        if (!have || (isint ? cs[t].emin_i < gmin_i : cs[t].emin < gmin)) {
            gmin = cs[t].emin;
            gmin_i = cs[t].emin_i;
        }
        have = 1;
    }
    uint64_t nties = 0, ntot = 0;
    for (int t = 0; t < nc; t++) {
        if (!cs[t].has)
            continue;
        if (isint ? cs[t].emin_i == gmin_i : cs[t].emin == gmin) {
            nties += cs[t].nties;
            ntot += cs[t].nheap;
        }
    }
    uint64_t *all = (uint64_t *)malloc(sizeof(uint64_t) * (ntot ? ntot : 1));
    uint64_t w = 0;
    for (int t = 0; t < nc; t++) {
        if (!cs[t].has)
            continue;
        if (isint ? cs[t].emin_i == gmin_i : cs[t].emin == gmin)
            for (uint64_t q = 0; q < cs[t].nheap; q++)
                all[w++] = cs[t].heap[q];
    }
    qsort(all, w, sizeof(uint64_t), cmp_u64);
    uint64_t nw = w < cap ? w : cap;
    for (uint64_t q = 0; q < nw; q++)
        out_ties[q] = all[q];
    free(all);
    if (isint)
        *(int64_t *)out_min = gmin_i;
    else
        *(double *)out_min = gmin;
    *out_nties = nties;
    *out_nwritten = nw;

    /* K lowest: merge every thread's list through one more collector. */
    coll_t m;
    coll_init(&m, K, 0);
    for (int t = 0; t < nc; t++)
        for (int q = 0; q < cs[t].nk; q++)
            topk_offer(&m, isint, cs[t].topE[q], cs[t].topE_i[q], cs[t].topC[q]);
    for (int q = 0; q < m.nk; q++) {
        out_topk[q] = m.topC[q];
        if (isint)
            ((int64_t *)out_topkE)[q] = m.topE_i[q];
        else
            ((double *)out_topkE)[q] = m.topE[q];
    }
    *out_nk = m.nk;
    coll_free(&m);
}

/* ------------------------------------------------------------------------------------ */
/* Solvers.                                                                               */
/* ------------------------------------------------------------------------------------ */

enum { ORACLE_DIRECT = 0, ORACLE_GRAY = 1 };

static int check_args(int n, int fix_bits, int K, int nthreads)
{
    if (n < 1 || n > 64 || fix_bits < 0 || fix_bits > n || n - fix_bits > 46)
        return -1;
    if (K < 0 || K > ORACLE_MAX_K || nthreads < 0)
        return -1;
    return 0;
}

/* Walk length between direct re-evaluations in the float Gray walk. */
#define ORACLE_F64_ANCHOR 1024

/*
 * Integer solve.  Q: n x n row-major int64.  Restricted to codes whose top `fix_bits` bits
 * equal fix_value.  Outputs: *out_min, *out_nties (exact), out_ties[0..*out_nwritten) the
 * smallest tie codes ascending (at most cap), out_topk / out_topkE the min(K, states) lowest
 * states by (E, code).  Returns 0, or -1 for bad arguments, -2 for allocation failure.
 */
int oracle_solve_i64(const int64_t *Q, int n, int method, int fix_bits, uint64_t fix_value, int K,
                     uint64_t cap, int nthreads, int64_t *out_min, uint64_t *out_nties,
                     uint64_t *out_ties, uint64_t *out_nwritten, uint64_t *out_topk,
                     int64_t *out_topkE, int *out_nk)
{
    if (check_args(n, fix_bits, K, nthreads))
        return -1;
    int64_t *U = (int64_t *)malloc(sizeof(int64_t) * n * n);
    if (!U)
        return -2;
    oracle_fold_i64(Q, n, U);
    int free_bits = n - fix_bits;
    uint64_t base = fix_bits ? (fix_value << free_bits) : 0;
    if (fix_bits == 64)
        base = fix_value;
    uint64_t states = 1ull << free_bits;
    int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
    coll_t *cs = (coll_t *)calloc(nt, sizeof(coll_t));
    for (int t = 0; t < nt; t++)
        coll_init(&cs[t], K, cap);

    if (method == ORACLE_DIRECT) {
#pragma omp parallel for num_threads(nt) schedule(dynamic, 4096)
        for (uint64_t s = 0; s < states; s++) {
            coll_t *c = &cs[omp_get_thread_num()];
            uint64_t code = base | s;
            int64_t E = oracle_energy_i64(U, n, code);
            if (coll_needs_i64(c, E))
                coll_feed_i64(c, E, code);
        }
    } else {
        /* Chunks of 2^m states share their high bits; each chunk is one Gray walk over its
         * low m bits, started from a direct evaluation. */
        int m = free_bits < 16 ? free_bits : 16;
        uint64_t nchunks = states >> m;
        int64_t *W = (int64_t *)calloc((size_t)n * n, sizeof(int64_t));
        for (int a = 0; a < n; a++)
            for (int b = 0; b < n; b++)
                if (a != b)
                    W[a * n + b] = a < b ? U[a * n + b] : U[b * n + a];
#pragma omp parallel for num_threads(nt) schedule(dynamic, 1)
        for (uint64_t ch = 0; ch < nchunks; ch++) {
            coll_t *c = &cs[omp_get_thread_num()];
            uint64_t x = base | (ch << m);
            int64_t h[64];
            for (int j = 0; j < n; j++) {
                int64_t acc = 0;
                for (int i = 0; i < n; i++)
                    if ((x >> i) & 1u)
                        acc += W[i * n + j];
                h[j] = acc;
            }
            int64_t E = oracle_energy_i64(U, n, x);
            if (coll_needs_i64(c, E))
                coll_feed_i64(c, E, x);
            uint64_t len = 1ull << m;
            for (uint64_t t = 0; t + 1 < len; t++) {
                int k = __builtin_ctzll(t + 1);
                x ^= 1ull << k;
                const int64_t *Wk = W + (size_t)k * n;
                if ((x >> k) & 1u) {
                    E += U[k * n + k] + h[k];
                    for (int j = 0; j < n; j++)
                        h[j] += Wk[j];
                } else {
                    E -= U[k * n + k] + h[k];
                    for (int j = 0; j < n; j++)
                        h[j] -= Wk[j];
                }
                if (coll_needs_i64(c, E))
                    coll_feed_i64(c, E, x);
            }
        }
        free(W);
    }
    coll_merge_out(cs, nt, 1, K, cap, out_min, out_nties, out_ties, out_nwritten, out_topk, out_topkE,
                   out_nk);
    for (int t = 0; t < nt; t++)
        coll_free(&cs[t]);
    free(cs);
    free(U);
    return 0;
}

/* Growable candidate list used by the float Gray walk. */
typedef struct {
    uint64_t *v;
    uint64_t n, cap;
} clist_t;

static int clist_push(clist_t *l, uint64_t code)
{
    if (l->n == l->cap) {
        uint64_t nc = l->cap ? 2 * l->cap : 1024;
        uint64_t *nv = (uint64_t *)realloc(l->v, nc * sizeof(uint64_t));
        if (!nv)
            return -1;
        l->v = nv;
        l->cap = nc;
    }
    l->v[l->n++] = code;
    return 0;
}

/* Running K-th smallest of the values offered so far (K >= 1), counted with multiplicity. */
typedef struct {
    int K, n;
    double *v;
} kth_t;

static void kth_offer(kth_t *q, double E)
{
    if (q->n == q->K && E >= q->v[q->n - 1])
        return;
    int pos = q->n < q->K ? q->n : q->K - 1;
    while (pos > 0 && E < q->v[pos - 1]) {
        q->v[pos] = q->v[pos - 1];
        pos--;
    }
    q->v[pos] = E;
    if (q->n < q->K)
        q->n++;
}

static double kth_bound(const kth_t *q) { return q->n < q->K ? INFINITY : q->v[q->n - 1]; }

/*
 * Float solve.  Q: n x n row-major double (FP32 inputs widened exactly).  Results are defined
 * by the direct FP64 evaluator.  Extra output *out_ncand: how many states the Gray pre-pass
 * forwarded to the direct evaluator (the direct method forwards every state).
 */
int oracle_solve_f64(const double *Q, int n, int method, int fix_bits, uint64_t fix_value, int K,
                     uint64_t cap, int nthreads, double *out_min, uint64_t *out_nties, uint64_t *out_ties,
                     uint64_t *out_nwritten, uint64_t *out_topk, double *out_topkE, int *out_nk,
                     uint64_t *out_ncand)
{
    if (check_args(n, fix_bits, K, nthreads))
        return -1;
    double *U = (double *)malloc(sizeof(double) * n * n);
    if (!U)
        return -2;
    oracle_fold_f64(Q, n, U);
    int free_bits = n - fix_bits;
    uint64_t base = fix_bits ? (fix_value << free_bits) : 0;
    if (fix_bits == 64)
        base = fix_value;
    uint64_t states = 1ull << free_bits;
    int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
    coll_t *cs = (coll_t *)calloc(nt, sizeof(coll_t));
    for (int t = 0; t < nt; t++)
        coll_init(&cs[t], K, cap);
    uint64_t ncand = 0;

    if (method == ORACLE_DIRECT) {
#pragma omp parallel for num_threads(nt) schedule(dynamic, 4096)
        for (uint64_t s = 0; s < states; s++) {
            coll_t *c = &cs[omp_get_thread_num()];
            uint64_t code = base | s;
            coll_feed_f64(c, oracle_energy_f64(U, n, code), code);
        }
        ncand = states;
    } else {
        /* Rigorous bound on |E_walk - E_direct|: every partial sum is at most S = sum |U_ij| in
         * magnitude and each rounding costs at most 2^-53 of it.  The direct value takes at most
         * n(n+1)/2 roundings; a walk re-evaluated every A steps carries at most
         * n(n+1)/2 + A(n+2) + A^2/2 of them (each step adds one rounding to E plus the error
         * of the field h_k, which itself gains one rounding per step).  Doubled for margin. */
        double S = 0.0;
        for (int i = 0; i < n; i++)
            for (int j = i; j < n; j++)
                S += fabs(U[i * n + j]);
        double A = ORACLE_F64_ANCHOR;
        double tol = 2.0 * ((double)n * (n + 1) + A * (n + 2) + A * A) * ldexp(1.0, -53) * S;
        int Kq = K > 0 ? K : 1;
        int m = free_bits < 16 ? free_bits : 16;
        uint64_t nchunks = states >> m;
        double *W = (double *)calloc((size_t)n * n, sizeof(double));
        for (int a = 0; a < n; a++)
            for (int b = 0; b < n; b++)
                if (a != b)
                    W[a * n + b] = a < b ? U[a * n + b] : U[b * n + a];
        clist_t *cl = (clist_t *)calloc(nt, sizeof(clist_t));
        kth_t *kq = (kth_t *)calloc(nt, sizeof(kth_t));
        for (int t = 0; t < nt; t++) {
            kq[t].K = Kq;
            kq[t].v = (double *)malloc(sizeof(double) * Kq);
        }
        int fail = 0;
#pragma omp parallel for num_threads(nt) schedule(dynamic, 1)
        for (uint64_t ch = 0; ch < nchunks; ch++) {
            int tid = omp_get_thread_num();
            uint64_t x = base | (ch << m);
            double h[64];
            double E = 0.0;
            uint64_t len = 1ull << m;
            for (uint64_t t = 0; t < len; t++) {
                if (t % ORACLE_F64_ANCHOR == 0) {
                    /* (re-)anchor: direct energy and fields of the current state */
                    for (int j = 0; j < n; j++) {
                        double acc = 0.0;
                        for (int i = 0; i < n; i++)
                            if ((x >> i) & 1u)
                                acc += W[i * n + j];
                        h[j] = acc;
                    }
                    E = oracle_energy_f64(U, n, x);
                }
                kth_offer(&kq[tid], E);
                if (E <= kth_bound(&kq[tid]) + 2.0 * tol)
                    if (clist_push(&cl[tid], x))
                        fail = 1;
                if (t + 1 == len)
                    break;
                int k = __builtin_ctzll(t + 1);
                x ^= 1ull << k;
                const double *Wk = W + (size_t)k * n;
                if ((x >> k) & 1u) {
                    E += U[k * n + k] + h[k];
                    for (int j = 0; j < n; j++)
                        h[j] += Wk[j];
                } else {
                    E -= U[k * n + k] + h[k];
                    for (int j = 0; j < n; j++)
                        h[j] -= Wk[j];
                }
            }
        }
        /* Direct re-evaluation of every forwarded candidate decides the result. */
        for (int t = 0; t < nt; t++) {
            for (uint64_t q = 0; q < cl[t].n; q++)
                coll_feed_f64(&cs[t], oracle_energy_f64(U, n, cl[t].v[q]), cl[t].v[q]);
            ncand += cl[t].n;
            free(cl[t].v);
            free(kq[t].v);
        }
        free(cl);
        free(kq);
        free(W);
        if (fail) {
            for (int t = 0; t < nt; t++)
                coll_free(&cs[t]);
            free(cs);
            free(U);
            return -2;
        }
    }
    coll_merge_out(cs, nt, 0, K, cap, out_min, out_nties, out_ties, out_nwritten, out_topk, out_topkE,
                   out_nk);
    if (out_ncand)
        *out_ncand = ncand;
    for (int t = 0; t < nt; t++)
        coll_free(&cs[t]);
    free(cs);
    free(U);
    return 0;
}

/* Number of threads OpenMP would use by default (the host cores the oracle runs on). */
/* ------------------------------------------------------------------------------------ */
/* Sub-problem with fixed variables (Sec. 3.3.1, x = (x_r, x_f); Sec. 4.3 applies it to    */
/* instances wider than one scan).                                                        */
/* ------------------------------------------------------------------------------------ */

/*
 * Variables m..n-1 are fixed to xf[0..n-m-1] (one byte per variable, 0 or 1); n may exceed 64.
 * Splitting the folded objective sum_{i<=j} U_ij x_i x_j by where i and j lie:
 *   both free (i <= j < m)        -> R_ij = U_ij, kept as a QUBO over x_0..x_{m-1};
 *   i free, j fixed (i < m <= j)  -> x_i * U_ij * xf_j: linear in x_i, so R_ii gains U_ij xf_j;
 *   both fixed (m <= i <= j)      -> U_ij xf_i xf_j, summed into the constant c.
 * Then E(x) = sum_{i<=j<m} R_ij x_i x_j + c for every x whose fixed part is xf.
 * U is the folded n x n matrix; R is m x m (upper-triangular, zeros below the diagonal).
 */
void oracle_reduce_i64(const int64_t *U, int n, int m, const uint8_t *xf, int64_t *R, int64_t *c)
{
    int64_t cc = 0;
    memset(R, 0, sizeof(int64_t) * (size_t)m * m);
    for (int i = 0; i < n; ++i)
        for (int j = i; j < n; ++j) {
            const int64_t u = U[(size_t)i * n + j];
            if (j < m)
                R[(size_t)i * m + j] += u;
            else if (i < m)
                R[(size_t)i * m + i] += xf[j - m] ? u : 0;
            else
                cc += (xf[i - m] && xf[j - m]) ? u : 0;
        }
    *c = cc;
}

void oracle_reduce_f64(const double *U, int n, int m, const uint8_t *xf, double *R, double *c)
{
    double cc = 0.0;
    memset(R, 0, sizeof(double) * (size_t)m * m);
    for (int i = 0; i < n; ++i)
        for (int j = i; j < n; ++j) {
            const double u = U[(size_t)i * n + j];
            if (j < m)
                R[(size_t)i * m + j] += u;
            else if (i < m)
                R[(size_t)i * m + i] += xf[j - m] ? u : 0.0;
            else
                cc += (xf[i - m] && xf[j - m]) ? u : 0.0;
        }
    *c = cc;
}

int oracle_max_threads(void) { return omp_get_max_threads(); }
