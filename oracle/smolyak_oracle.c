/*
 * Smolyak operator action -- CPU ORACLE (test infrastructure only).
 *
 * This file is the plain, slow, obviously-correct FP64 statement of what the
 * Smolyak action H|psi> computes.  It is used by the test-suite, the smoke
 * check and the benchmark's CPU-baseline leg, and by nothing else.  It shares
 * no code, header, table or constant generator with the CUDA library.
 *
 * Definitions followed (arXiv 2111.13655):
 *   - Smolyak representation S_L = sum_{R(l)} D_l  S^1_{l_1} x ... x S^n_{l_n},
 *     restriction R(l): L-n+1 <= |l| <= L, D_l = (-1)^{L-|l|} C(n-1, L-|l|)
 *     (Sec. 2, Eq. (8));  level -> size rule N_l = A + B*l (Sec. 2).
 *   - Term order, in-term order and compact order as printed in Table 2
 *     (Sec. 3): terms with l_1 varying fastest; inside a term k_1 fastest;
 *     compact basis lexicographic with the first mode slowest.
 *   - The operator, Eq. (16): y = sum_l D_l P_l^T A_l P_l x, P_l the
 *     restriction of the compact basis to term l (the mapping M^B of Table 2),
 *     A_l = (x_i B_i^T W_i) O_l (x_i B_i): the transfer to the term's
 *     direct-product grid (Eq. (15)), the operator on that grid, and the
 *     transfer back (Eq. (14)).
 *   - The operator on the grid (Sec. 3, "conventional" action on the grid):
 *     the potential multiplied point by point; the kinetic part
 *     -omega_j/2 d^2/dq_j^2 through the second derivatives of the basis
 *     functions at the nodes.
 *
 * Readings where the paper is silent (listed with the design notes):
 *   - primitive basis "Hm": orthonormal Hermite functions
 *       b_k(Q) = sqrt(s) h_k(s (Q - Q0)),  h_k(x) = (2^k k! sqrt(pi))^-1/2 H_k(x) e^{-x^2/2};
 *   - grid: Gauss-Hermite nodes x_u (Golub-Welsch + Newton), Q_u = Q0 + x_u / s, with
 *     weights w_u = w^GH_u e^{x_u^2} / s (the classical weight times e^{x^2}) so that sum_u w_u b_k b_k' = delta_kk'
 *     whenever nq >= nb (the w_i of Eq. (6));
 *   - second derivative: b_k''(Q) = s^2 (x^2 - (2k+1)) b_k(Q) (Hermite ODE).
 *
 * No blocking, fusion or reordering: every term is taken through the full
 * direct-product grid of all its modes, including modes at level 0.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2

/* ------------------------------------------------------------------------ */
/* Symmetric eigenproblem by cyclic Jacobi rotations (used for Golub-Welsch). */
/* A: n x n row-major symmetric, destroyed (diagonal -> eigenvalues).         */
/* V: n x n row-major, columns -> orthonormal eigenvectors.                   */
/* ------------------------------------------------------------------------ */
static void jacobi_eigen(int n, double *A, double *V)
{
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) V[i * n + j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 100; sweep++) {
        double off = 0.0, diag = 0.0;
        for (int i = 0; i < n; i++)
            for (int j = 0; j < n; j++) {
                if (i != j) off += A[i * n + j] * A[i * n + j];
                else diag += A[i * n + j] * A[i * n + j];
            }
        if (off <= 1e-32 * (diag + 1e-300)) break;
        for (int p = 0; p < n - 1; p++)
            for (int q = p + 1; q < n; q++) {
                double apq = A[p * n + q];
                if (apq == 0.0) continue;
                /* rotation J in the (p,q) plane that zeroes A'_pq of J^T A J */
                double theta = (A[p * n + p] - A[q * n + q]) / (2.0 * apq);
                double sg = (theta >= 0.0) ? 1.0 : -1.0;
                double t = -sg / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; k++) { /* columns: A J */
                    double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * akq;
                    A[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; k++) { /* rows: J^T (A J) */
                    double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * aqk;
                    A[q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; k++) { /* eigenvectors: V J */
                    double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - s * vkq;
                    V[k * n + q] = s * vkp + c * vkq;
                }
            }
    }
}

/* Orthonormal Hermite functions h_0..h_{nb-1} at x, by the normalised
 * three-term recurrence. */
static void hermite_functions(int nb, double x, double *h)
{
    h[0] = pow(M_PI, -0.25) * exp(-0.5 * x * x);
    if (nb > 1) h[1] = sqrt(2.0) * x * h[0];
    for (int k = 1; k + 1 < nb; k++)
        h[k + 1] = sqrt(2.0 / (k + 1)) * x * h[k] - sqrt((double)k / (k + 1)) * h[k - 1];
}

/* Gauss-Hermite rule of n points.  Nodes: Golub-Welsch -- the eigenvalues of
 * the symmetric tridiagonal Jacobi matrix of the Hermite recurrence
 * (off-diagonal sqrt(k/2)) -- polished by two Newton steps on h_n, using
 * h_n' = sqrt(2n) h_{n-1} - x h_n.  Weights in the Hermite-function
 * normalisation, wf_u = w_u e^{x_u^2} = 1 / (n h_{n-1}(x_u)^2): the classical
 * Gauss-Hermite weight formula written with orthonormal Hermite functions (it
 * never multiplies a tiny weight by a huge e^{x^2}).
 * x: nodes, ascending; w: classical weights (weight function e^{-x^2});
 * wf: function-normalised weights (may be NULL). */
static int gauss_hermite_rule(int n, double *x, double *w, double *wf)
{
    if (n < 1 || n > 200) return ORC_EINVAL;
    double *A = (double *)calloc((size_t)n * n, sizeof(double));
    double *V = (double *)calloc((size_t)n * n, sizeof(double));
    double *h = (double *)calloc((size_t)n + 1, sizeof(double));
    if (!A || !V || !h) { free(A); free(V); free(h); return ORC_ENOMEM; }
    for (int k = 1; k < n; k++) {
        A[(k - 1) * n + k] = sqrt(0.5 * k);
        A[k * n + (k - 1)] = sqrt(0.5 * k);
    }
    jacobi_eigen(n, A, V);
    for (int u = 0; u < n; u++) x[u] = A[u * n + u];
    /* insertion sort by node */
    for (int i = 1; i < n; i++) {
        double xi = x[i];
        int j = i - 1;
        while (j >= 0 && x[j] > xi) { x[j + 1] = x[j]; j--; }
        x[j + 1] = xi;
    }
    for (int u = 0; u < n; u++) {
        double xu = x[u];
        for (int it = 0; it < 2; it++) {
            hermite_functions(n + 1, xu, h);
            double d = sqrt(2.0 * n) * h[n - 1] - xu * h[n];
            if (d != 0.0) xu -= h[n] / d;
        }
        x[u] = xu;
        hermite_functions(n, xu, h);
        double f = 1.0 / (n * h[n - 1] * h[n - 1]);
        if (wf) wf[u] = f;
        w[u] = f * exp(-xu * xu);
    }
    free(A); free(V); free(h);
    return ORC_OK;
}

int orc_gauss_hermite(int n, double *x, double *w)
{
    return gauss_hermite_rule(n, x, w, NULL);
}

/* 1D tables of one mode at one level (Sec. 2, Eqs. (6),(7)):
 *   B[u*nb+k]  = b_k(Q_u)          (basis -> grid, Eq. (15))
 *   D2[u*nb+k] = b_k''(Q_u)        (kinetic on the grid)
 *   W[u]       = w_u               (grid -> basis uses w_u b_k(Q_u), Eq. (14))
 *   Q[u]       = Q_u               (grid coordinates for the potential)      */
int orc_mode_tables(int nb, int nq, double q0, double scale,
                    double *B, double *D2, double *W, double *Q)
{
    if (nb < 1 || nq < 1 || nb > 200 || nq > 200 || !(scale > 0)) return ORC_EINVAL;
    double *x = (double *)malloc(sizeof(double) * nq);
    double *wg = (double *)malloc(sizeof(double) * nq);
    double *wf = (double *)malloc(sizeof(double) * nq);
    double *h = (double *)malloc(sizeof(double) * nb);
    if (!x || !wg || !wf || !h) { free(x); free(wg); free(wf); free(h); return ORC_ENOMEM; }
    int rc = gauss_hermite_rule(nq, x, wg, wf);
    if (rc == ORC_OK) {
        for (int u = 0; u < nq; u++) {
            hermite_functions(nb, x[u], h);
            for (int k = 0; k < nb; k++) {
                double b = sqrt(scale) * h[k];
                B[u * nb + k] = b;
                D2[u * nb + k] = scale * scale * (x[u] * x[u] - (2.0 * k + 1.0)) * b;
            }
            W[u] = wf[u] / scale;
            Q[u] = q0 + x[u] / scale;
        }
    }
    free(x); free(wg); free(wf); free(h);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Sizes, terms and the compact basis                                       */
/* ------------------------------------------------------------------------ */
static inline int nsize(int A, int B, int l) { return A + B * l; }

/* smallest level whose basis contains function index k (k 0-based) */
static inline int lmin_of(int A, int B, int k)
{
    int l = 0;
    while (nsize(A, B, l) <= k) l++;
    return l;
}

static int64_t binom_i64(int n, int k)
{
    if (k < 0 || n < 0 || k > n) return 0;
    int64_t r = 1;
    for (int i = 1; i <= k; i++) r = r * (n - k + i) / i;
    return r;
}

/* Combination coefficient D_l = (-1)^{L-|l|} C(n-1, L-|l|) of Eq. (8). */
int64_t orc_combination_coefficient(int D, int L, int sum_l)
{
    int r = L - sum_l;
    if (r < 0 || r > D - 1) return 0;
    int64_t c = binom_i64(D - 1, r);
    return (r % 2) ? -c : c;
}

/* Enumerate the terms of R(l) in the order of Table 2 (l_1 fastest).
 * levels: out, n_terms x D (may be NULL to count only); coef: out (may be NULL). */
int64_t orc_enumerate_terms(int D, int L, int *levels, int64_t *coef)
{
    if (D < 1 || L < 0) return -1;
    int *l = (int *)calloc(D, sizeof(int));
    if (!l) return -1;
    int64_t n = 0;
    int sum = 0;
    int lo = L - D + 1;
    for (;;) {
        if (sum >= lo && sum <= L) {
            if (levels) memcpy(levels + n * D, l, sizeof(int) * D);
            if (coef) coef[n] = orc_combination_coefficient(D, L, sum);
            n++;
        }
        int i = 0;
        while (i < D) {
            l[i]++; sum++;
            if (sum <= L) break;
            sum -= l[i]; l[i] = 0; i++;
        }
        if (i == D) break;
    }
    free(l);
    return n;
}

/* Enumerate the compact basis (union of all term boxes) in lexicographic
 * order with the first mode slowest (Table 2, bottom).  A multi-index k is in
 * the union iff sum_i lmin_i(k_i) <= L.  kout: n x D (may be NULL). */
int64_t orc_enumerate_compact(int D, int L, const int *nbA, const int *nbB, int *kout)
{
    if (D < 1 || L < 0) return -1;
    int *k = (int *)calloc(D, sizeof(int));
    int *cost = (int *)calloc(D, sizeof(int));
    if (!k || !cost) { free(k); free(cost); return -1; }
    int64_t n = 0;
    int sum = 0; /* sum_i lmin_i(k_i) */
    for (;;) {
        if (kout) memcpy(kout + n * D, k, sizeof(int) * D);
        n++;
        int i = D - 1;
        while (i >= 0) {
            k[i]++;
            int c = lmin_of(nbA[i], nbB[i], k[i]);
            sum += c - cost[i]; cost[i] = c;
            if (sum <= L) break;
            sum -= cost[i]; cost[i] = 0; k[i] = 0; i--;
        }
        if (i < 0) break;
    }
    free(k); free(cost);
    return n;
}

/* Counts of Table 1 by generating functions (no enumeration):
 *   n_terms = #R(l), N_s = sum_{R(l)} prod_i nb_i(l_i), N_cs = #compact.
 * Uses the per-mode polynomials sum_l x^l, sum_l nb_i(l) x^l and
 * sum_k x^{lmin_i(k)}, multiplied and truncated at degree L. */
int orc_counts(int D, int L, const int *nbA, const int *nbB,
               int64_t *n_terms, int64_t *n_s, int64_t *n_cs)
{
    if (D < 1 || L < 0) return ORC_EINVAL;
    int64_t *pt = (int64_t *)calloc(L + 1, sizeof(int64_t));
    int64_t *ps = (int64_t *)calloc(L + 1, sizeof(int64_t));
    int64_t *pc = (int64_t *)calloc(L + 1, sizeof(int64_t));
    int64_t *t = (int64_t *)calloc(L + 1, sizeof(int64_t));
    int64_t *f = (int64_t *)calloc(L + 1, sizeof(int64_t));
    if (!pt || !ps || !pc || !t || !f) { free(pt); free(ps); free(pc); free(t); free(f); return ORC_ENOMEM; }
    pt[0] = ps[0] = pc[0] = 1;
    for (int i = 0; i < D; i++) {
        /* terms: factor sum_l x^l */
        for (int s = 0; s <= L; s++) { t[s] = 0; for (int a = 0; a <= s; a++) t[s] += pt[s - a]; }
        memcpy(pt, t, sizeof(int64_t) * (L + 1));
        /* N_s: factor sum_l nb(l) x^l */
        for (int s = 0; s <= L; s++) { t[s] = 0; for (int a = 0; a <= s; a++) t[s] += ps[s - a] * nsize(nbA[i], nbB[i], a); }
        memcpy(ps, t, sizeof(int64_t) * (L + 1));
        /* N_cs: factor sum_k x^{lmin(k)} = sum_l (#k with lmin(k)=l) x^l */
        for (int a = 0; a <= L; a++) f[a] = nsize(nbA[i], nbB[i], a) - (a ? nsize(nbA[i], nbB[i], a - 1) : 0);
        for (int s = 0; s <= L; s++) { t[s] = 0; for (int a = 0; a <= s; a++) t[s] += pc[s - a] * f[a]; }
        memcpy(pc, t, sizeof(int64_t) * (L + 1));
    }
    int64_t nt = 0, ns = 0, nc = 0;
    for (int s = 0; s <= L; s++) {
        if (s >= L - D + 1) { nt += pt[s]; ns += ps[s]; }
        nc += pc[s];
    }
    *n_terms = nt; *n_s = ns; *n_cs = nc;
    free(pt); free(ps); free(pc); free(t); free(f);
    return ORC_OK;
}

/* position of k in the lexicographically sorted compact list (binary search) */
static int64_t compact_find(const int *kc, int64_t ncs, int D, const int *k)
{
    int64_t lo = 0, hi = ncs - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        const int *km = kc + mid * D;
        int cmp = 0;
        for (int i = 0; i < D && !cmp; i++) cmp = (km[i] < k[i]) ? -1 : (km[i] > k[i]) ? 1 : 0;
        if (cmp == 0) return mid;
        if (cmp < 0) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* Mapping table M^B of Table 2: for each term (Table 2 order) the compact
 * index of each of its basis functions (k_1 fastest), 0-based.
 * term_offsets: n_terms+1 (out); cs_index: N_s (out). */
int orc_term_map(int D, int L, const int *nbA, const int *nbB,
                 int64_t *term_offsets, int64_t *cs_index)
{
    int64_t nt = orc_enumerate_terms(D, L, NULL, NULL);
    int64_t ncs = orc_enumerate_compact(D, L, nbA, nbB, NULL);
    if (nt < 0 || ncs < 0) return ORC_EINVAL;
    int *lv = (int *)malloc(sizeof(int) * nt * D);
    int *kc = (int *)malloc(sizeof(int) * ncs * D);
    int *k = (int *)calloc(D, sizeof(int));
    if (!lv || !kc || !k) { free(lv); free(kc); free(k); return ORC_ENOMEM; }
    orc_enumerate_terms(D, L, lv, NULL);
    orc_enumerate_compact(D, L, nbA, nbB, kc);
    int64_t pos = 0;
    for (int64_t t = 0; t < nt; t++) {
        term_offsets[t] = pos;
        const int *l = lv + t * D;
        memset(k, 0, sizeof(int) * D);
        for (;;) {
            cs_index[pos++] = compact_find(kc, ncs, D, k);
            int i = 0;
            while (i < D) {
                k[i]++;
                if (k[i] < nsize(nbA[i], nbB[i], l[i])) break;
                k[i] = 0; i++;
            }
            if (i == D) break;
        }
    }
    term_offsets[nt] = pos;
    free(lv); free(kc); free(k);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Operator action                                                          */
/* ------------------------------------------------------------------------ */

/* out = M x_mode in : contract mode `mode` of a tensor (mode 0 fastest) with
 * the rows x cols matrix M (row-major), cols = dims[mode]. */
static void contract_mode(const double *in, double *out, int D, const int *dims,
                          int mode, const double *M, int rows, int cols)
{
    int64_t left = 1, right = 1;
    for (int i = 0; i < mode; i++) left *= dims[i];
    for (int i = mode + 1; i < D; i++) right *= dims[i];
    for (int64_t b = 0; b < right; b++)
        for (int r = 0; r < rows; r++)
            for (int64_t a = 0; a < left; a++) {
                double s = 0.0;
                for (int c = 0; c < cols; c++)
                    s += M[r * cols + c] * in[a + left * (c + (int64_t)cols * b)];
                out[a + left * (r + (int64_t)rows * b)] = s;
            }
}

typedef struct {
    int nb, nq;
    double *B, *D2, *W, *Q, *BW; /* BW[k*nq+u] = w_u b_k(Q_u) */
} mode_level_tables;

/*
 * y = H_S x for nvec vectors (column-major, N_cs each, compact order).
 * Terms processed: all (term_subset == NULL) or the listed term indices.
 * Vectors of the potential: monomial m = coef[m] * prod over its nfac[m]
 * factors of Q_{fmode}^{fpow}, factors stored back to back.
 * nthreads <= 0: OpenMP default.  Per-thread partial results are summed in
 * thread order, so the result is deterministic for a fixed thread count.
 */
int orc_apply(int D, int L,
              const int *nbA, const int *nbB, const int *nqA, const int *nqB,
              const double *q0, const double *scale, const double *omega,
              int nmono, const double *coef, const int *nfac, const int *fmode, const int *fpow,
              const double *x, double *y, int nvec,
              const int64_t *term_subset, int64_t nsub, int nthreads)
{
    if (D < 1 || L < 0 || nvec < 1) return ORC_EINVAL;
    for (int i = 0; i < D; i++)
        if (nbA[i] < 1 || nbB[i] < 0 || nqA[i] < nbA[i] || nqB[i] < nbB[i]) return ORC_EINVAL;
    int64_t nt = orc_enumerate_terms(D, L, NULL, NULL);
    int64_t ncs = orc_enumerate_compact(D, L, nbA, nbB, NULL);
    int *lv = (int *)malloc(sizeof(int) * nt * D);
    int64_t *cl = (int64_t *)malloc(sizeof(int64_t) * nt);
    int *kc = (int *)malloc(sizeof(int) * ncs * D);
    mode_level_tables *tab = (mode_level_tables *)calloc((size_t)D * (L + 1), sizeof(mode_level_tables));
    int *foff = (int *)malloc(sizeof(int) * (nmono + 1));
    if (!lv || !cl || !kc || !tab || !foff) return ORC_ENOMEM;
    orc_enumerate_terms(D, L, lv, cl);
    orc_enumerate_compact(D, L, nbA, nbB, kc);
    foff[0] = 0;
    for (int m = 0; m < nmono; m++) foff[m + 1] = foff[m] + nfac[m];

    for (int i = 0; i < D; i++)
        for (int l = 0; l <= L; l++) {
            mode_level_tables *t = &tab[i * (L + 1) + l];
            t->nb = nsize(nbA[i], nbB[i], l);
            t->nq = nsize(nqA[i], nqB[i], l);
            t->B = (double *)malloc(sizeof(double) * t->nb * t->nq);
            t->D2 = (double *)malloc(sizeof(double) * t->nb * t->nq);
            t->BW = (double *)malloc(sizeof(double) * t->nb * t->nq);
            t->W = (double *)malloc(sizeof(double) * t->nq);
            t->Q = (double *)malloc(sizeof(double) * t->nq);
            orc_mode_tables(t->nb, t->nq, q0[i], scale[i], t->B, t->D2, t->W, t->Q);
            for (int k = 0; k < t->nb; k++)
                for (int u = 0; u < t->nq; u++) t->BW[k * t->nq + u] = t->W[u] * t->B[u * t->nb + k];
        }

    int64_t nwork = term_subset ? nsub : nt;
    /* largest term grid / basis */
    int64_t maxg = 1, maxb = 1;
    for (int64_t w = 0; w < nwork; w++) {
        int64_t t = term_subset ? term_subset[w] : w;
        int64_t g = 1, b = 1;
        for (int i = 0; i < D; i++) {
            g *= tab[i * (L + 1) + lv[t * D + i]].nq;
            b *= tab[i * (L + 1) + lv[t * D + i]].nb;
        }
        if (g > maxg) maxg = g;
        if (b > maxb) maxb = b;
    }
    int64_t big = maxg > maxb ? maxg : maxb;

    int nth = 1;
#ifdef _OPENMP
    nth = (nthreads > 0) ? nthreads : omp_get_max_threads();
#endif
    double *ypart = (double *)calloc((size_t)nth * ncs * nvec, sizeof(double));
    if (!ypart) return ORC_ENOMEM;
    int fail = 0;

#ifdef _OPENMP
#pragma omp parallel num_threads(nth)
#endif
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *yp = ypart + (size_t)tid * ncs * nvec;
        double *X = (double *)malloc(sizeof(double) * big);
        double *T1 = (double *)malloc(sizeof(double) * big);
        double *T2 = (double *)malloc(sizeof(double) * big);
        double *G = (double *)malloc(sizeof(double) * big);   /* psi on the grid          */
        double *Yg = (double *)malloc(sizeof(double) * big);  /* O psi on the grid        */
        int64_t *rank = (int64_t *)malloc(sizeof(int64_t) * maxb);
        int *dims = (int *)malloc(sizeof(int) * D);
        int *k = (int *)malloc(sizeof(int) * D);
        int *u = (int *)malloc(sizeof(int) * D);
        const mode_level_tables **mt = (const mode_level_tables **)malloc(sizeof(void *) * D);
        if (!X || !T1 || !T2 || !G || !Yg || !rank || !dims || !k || !u || !mt) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            fail = 1;
        } else {
#ifdef _OPENMP
#pragma omp for schedule(static, 1)
#endif
            for (int64_t w = 0; w < nwork; w++) {
                int64_t t = term_subset ? term_subset[w] : w;
                const int *l = lv + t * D;                     /* {l_1..l_n} <- i^st      */
                double c = (double)cl[t];                      /* D_l of Eq. (8)          */
                int64_t nbt = 1, nqt = 1;
                for (int i = 0; i < D; i++) {
                    mt[i] = &tab[i * (L + 1) + l[i]];
                    nbt *= mt[i]->nb; nqt *= mt[i]->nq;
                }
                /* M^B: compact index of every basis function of the term (k_1 fastest) */
                memset(k, 0, sizeof(int) * D);
                for (int64_t s = 0; s < nbt; s++) {
                    rank[s] = compact_find(kc, ncs, D, k);
                    for (int i = 0; i < D; i++) { if (++k[i] < mt[i]->nb) break; k[i] = 0; }
                }
                for (int v = 0; v < nvec; v++) {
                    const double *xv = x + (size_t)v * ncs;
                    /* P_l x: the term's coefficients, looked up in the compact basis (M^B, Table 2) */
                    for (int64_t s = 0; s < nbt; s++) X[s] = xv[rank[s]];
                    /* (x_i B_i) P_l x: the term's function on its direct-product grid (Eq. (15)) */
                    for (int i = 0; i < D; i++) dims[i] = mt[i]->nb;
                    memcpy(T1, X, sizeof(double) * nbt);
                    for (int i = 0; i < D; i++) {
                        contract_mode(T1, T2, D, dims, i, mt[i]->B, mt[i]->nq, mt[i]->nb);
                        dims[i] = mt[i]->nq;
                        double *sw = T1; T1 = T2; T2 = sw;
                    }
                    memcpy(G, T1, sizeof(double) * nqt);
                    /* V(Q) times the grid values, point by point */
                    memset(u, 0, sizeof(int) * D);
                    for (int64_t g = 0; g < nqt; g++) {
                        double V = 0.0;
                        for (int m = 0; m < nmono; m++) {
                            double p = coef[m];
                            for (int f = foff[m]; f < foff[m + 1]; f++) {
                                double qv = mt[fmode[f]]->Q[u[fmode[f]]];
                                for (int e = 0; e < fpow[f]; e++) p *= qv;
                            }
                            V += p;
                        }
                        Yg[g] = V * G[g];
                        for (int i = 0; i < D; i++) { if (++u[i] < mt[i]->nq) break; u[i] = 0; }
                    }
                    /* plus the kinetic part -omega_j/2 d^2/dq_j^2 on the grid: the
                     * transfer of Eq. (15) with b'' in place of b for mode j */
                    for (int j = 0; j < D; j++) {
                        if (omega[j] == 0.0) continue;
                        for (int i = 0; i < D; i++) dims[i] = mt[i]->nb;
                        memcpy(T1, X, sizeof(double) * nbt);
                        for (int i = 0; i < D; i++) {
                            contract_mode(T1, T2, D, dims, i, (i == j) ? mt[i]->D2 : mt[i]->B,
                                          mt[i]->nq, mt[i]->nb);
                            dims[i] = mt[i]->nq;
                            double *sw = T1; T1 = T2; T2 = sw;
                        }
                        for (int64_t g = 0; g < nqt; g++) Yg[g] += -0.5 * omega[j] * T1[g];
                    }
                    /* (x_i B_i^T W_i): back to the term's basis (Eq. (14)) */
                    for (int i = 0; i < D; i++) dims[i] = mt[i]->nq;
                    memcpy(T1, Yg, sizeof(double) * nqt);
                    for (int i = 0; i < D; i++) {
                        contract_mode(T1, T2, D, dims, i, mt[i]->BW, mt[i]->nb, mt[i]->nq);
                        dims[i] = mt[i]->nb;
                        double *sw = T1; T1 = T2; T2 = sw;
                    }
                    /* y += D_l P_l^T (...): the term's share of Eq. (16), D_l of Eq. (8) */
                    double *yv = yp + (size_t)v * ncs;
                    for (int64_t s = 0; s < nbt; s++) yv[rank[s]] += c * T1[s];
                }
            }
        }
        free(X); free(T1); free(T2); free(G); free(Yg); free(rank); free(dims); free(k); free(u); free(mt);
    }
    if (!fail) {
        memset(y, 0, sizeof(double) * ncs * nvec);
        for (int t = 0; t < nth; t++) {
            const double *yp = ypart + (size_t)t * ncs * nvec;
            for (int64_t i = 0; i < ncs * nvec; i++) y[i] += yp[i];
        }
    }
    free(ypart);
    for (int i = 0; i < D * (L + 1); i++) {
        free(tab[i].B); free(tab[i].D2); free(tab[i].W); free(tab[i].Q); free(tab[i].BW);
    }
    free(tab); free(lv); free(cl); free(kc); free(foff);
    return fail ? ORC_ENOMEM : ORC_OK;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
