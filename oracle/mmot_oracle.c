/*
 * Plain FP64 CPU oracle for multi-marginal Sinkhorn with pairwise L1 cost
 * (arXiv 2405.19246).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark load this library.  It shares no code,
 * header, table or helper with the CUDA path, and nothing in the product
 * path calls it.
 *
 * Everything is FP64 and deliberately simple: no blocking, no fusion, no
 * reordering beyond what each cited definition or algorithm states.
 *
 * Notation (Section 2 and Section 4.2 of the paper):
 *   l marginals, marginal k has N_k sorted support points x_k and weights mu_k.
 *   Pairwise L1 cost  c(y_1..y_l) = sum_{p<q} |y_p - y_q|        (Sec. 4.2)
 *   Gibbs kernel      K = exp(-c/eps)                            (Sec. 4.2)
 *   Plan              t = prod_k phi_k(i_k) K                    (Eq. k-marginal T value)
 *   Marginal product  M_j(i) = sum over the other marginals' points of
 *                     prod_{m != j} phi_m K                       (Eq. Jk k margin)
 *   Potentials        g_k = eps ln phi_k   (so phi = exp(g/eps))
 *   The paper's dual variable is alpha_k = -g_k - eps/l           (Sec. 2, phi definition)
 *
 * Functions:
 *   mo_merge            total order of all points by (x, marginal, index);
 *                       reproduces the tie rules of the order classes D_p (Eq. D_p)
 *   mo_marginal_classes ln M_j by the paper's l! order-class chains
 *                       (Sec. 4.2: classes D_1..D_{l!}, nested prefix recursion
 *                       of J^{(l)}_{i_l,1}; the other classes "similar")
 *   mo_marginal_subset  ln M_j by the subset-state form of the same chains
 *                       (orderings that put the same set left of a point share
 *                       one running sum); validated against brute force and
 *                       the class chains by the tests
 *   mo_allpass          all l marginals of the plan, total mass Z and the
 *                       transport cost W = <C, T> (Eq. k-mmot distance)
 *   mo_ftvp1            Algorithm 2 (FTVP-1), l = 3, uniform grid
 *   mo_ftvp2            Algorithm 3 (FTVP-2), l = 3, uniform grid, with the
 *                       two initial values R_{N,5}, R_{N,6} carrying the factor N
 *                       that Eq. RkSk implies (the printed initialisation omits it)
 *   mo_fs3              Algorithm 4 (fast Sinkhorn, l = 3), returning W with a
 *                       single factor h (FTVP-2 already multiplies by h)
 *   mo_sinkhorn         Gauss-Seidel Sinkhorn for general l (Sec. 4.2 update
 *                       formulas; Algorithm 1 loop structure) in the log domain
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define MO_MAXL 8

/* log(exp(a) + exp(b)) */
static double lae(double a, double b)
{
    if (a == -INFINITY) return b;
    if (b == -INFINITY) return a;
    if (a >= b) return a + log1p(exp(b - a));
    return b + log1p(exp(a - b));
}

static int popcount_u(unsigned v)
{
    int c = 0;
    while (v) { c += (int)(v & 1u); v >>= 1; }
    return c;
}

/* Decay rate of the running sum of a tuple part with s of the l points
 * placed: while s points lie left of z, s(l-s) pairs straddle z, so the cost
 * integral grows at rate s(l-s) (every |y_p - y_q| is the length of the
 * interval between the two points). */
static double rate(int l, int s) { return (double)s * (double)(l - s); }

/* ------------------------------------------------------------------ */
/* Merged order.                                                        */
/* ------------------------------------------------------------------ */

/* Merge the l sorted supports into one total order by the key (x, k, i).
 * mid_out[t] = marginal of the t-th point, loc_out[t] = its index within the
 * marginal.  Ties between marginals are broken by the marginal index, which
 * is the tie rule of the classes D_p (Eq. D_p: i <= j <= k puts the earlier
 * marginal first on equal coordinates).  Returns 0, or -1 if a support is not
 * sorted. */
int mo_merge(int l, const int64_t *N, const double *const *x, int *mid_out, int64_t *loc_out)
{
    int64_t head[MO_MAXL];
    int64_t T = 0;
    for (int k = 0; k < l; ++k) {
        head[k] = 0;
        T += N[k];
        for (int64_t i = 1; i < N[k]; ++i)
            if (x[k][i] < x[k][i - 1]) return -1;
    }
    for (int64_t t = 0; t < T; ++t) {
        int best = -1;
        for (int k = 0; k < l; ++k) {
            if (head[k] >= N[k]) continue;
            if (best < 0 || x[k][head[k]] < x[best][head[best]]) best = k;
        }
        mid_out[t] = best;
        loc_out[t] = head[best];
        head[best] += 1;
    }
    return 0;
}

static int merged_alloc(int l, const int64_t *N, const double *const *x,
                        int **mid, int64_t **loc, double **xm, int64_t *T)
{
    int64_t tot = 0;
    for (int k = 0; k < l; ++k) tot += N[k];
    *T = tot;
    *mid = (int *)malloc(sizeof(int) * (size_t)(tot ? tot : 1));
    *loc = (int64_t *)malloc(sizeof(int64_t) * (size_t)(tot ? tot : 1));
    *xm = (double *)malloc(sizeof(double) * (size_t)(tot ? tot : 1));
    if (!*mid || !*loc || !*xm) return -2;
    if (mo_merge(l, N, x, *mid, *loc) != 0) return -1;
    for (int64_t t = 0; t < tot; ++t) (*xm)[t] = x[(*mid)[t]][(*loc)[t]];
    return 0;
}

static void merged_free(int *mid, int64_t *loc, double *xm)
{
    free(mid);
    free(loc);
    free(xm);
}

/* ------------------------------------------------------------------ */
/* Order-class chains (the paper's l! classes, Sec. 4.2).               */
/* ------------------------------------------------------------------ */

/* Next permutation in lexicographic order; returns 0 after the last one. */
static int next_perm(int *a, int n)
{
    int i = n - 2;
    while (i >= 0 && a[i] >= a[i + 1]) --i;
    if (i < 0) return 0;
    int j = n - 1;
    while (a[j] <= a[i]) --j;
    int tmp = a[i]; a[i] = a[j]; a[j] = tmp;
    for (int p = i + 1, q = n - 1; p < q; ++p, --q) { tmp = a[p]; a[p] = a[q]; a[q] = tmp; }
    return 1;
}

/* ln M_j(i) for every point i of marginal j by summing, over all l! order
 * classes (the orderings of the l marginals' points along the line), the
 * class sum evaluated as two nested running sums: the chain of marginals left
 * of the j-point (a prefix recursion, like J^{(l)}_{i_l,1} of Sec. 4.2) times
 * the chain right of it (the mirrored suffix recursion, like J_{k,5}, J_{k,6}
 * of Eq. recurrence formula Jk).  Within a class the L1 cost has no absolute
 * values (Eq. form of K), so each level of a chain is a first-order recurrence
 * whose multiplier is exp(-s(l-s) dx/eps) when s points are placed.
 * Complexity O(l! * l * T); meant for l <= 6 and modest T. */
int mo_marginal_classes(int l, const int64_t *N, const double *const *x,
                        const double *const *g, double eps, int j, double *lnM_out)
{
    int *mid; int64_t *loc; double *xm; int64_t T;
    int rc = merged_alloc(l, N, x, &mid, &loc, &xm, &T);
    if (rc) { merged_free(mid, loc, xm); return rc; }
    double *left = (double *)malloc(sizeof(double) * (size_t)(N[j] ? N[j] : 1));
    double *right = (double *)malloc(sizeof(double) * (size_t)(N[j] ? N[j] : 1));
    for (int64_t i = 0; i < N[j]; ++i) lnM_out[i] = -INFINITY;

    int sigma[MO_MAXL];
    for (int k = 0; k < l; ++k) sigma[k] = k;
    do {
        int r = 0;                      /* position of j in sigma */
        while (sigma[r] != j) ++r;
        /* left chain: sigma[0], ..., sigma[r-1] */
        double run[MO_MAXL + 1];
        run[0] = 0.0;
        for (int q = 1; q <= r; ++q) run[q] = -INFINITY;
        for (int64_t t = 0; t < T; ++t) {
            if (t > 0) {
                double dx = (xm[t] - xm[t - 1]) / eps;
                for (int q = 1; q <= r; ++q) run[q] -= rate(l, q) * dx;
            }
            int m = mid[t];
            if (m == j) { left[loc[t]] = run[r]; continue; }
            for (int q = 1; q <= r; ++q)
                if (sigma[q - 1] == m) run[q] = lae(run[q], g[m][loc[t]] / eps + run[q - 1]);
        }
        /* right chain: from the right end, the q-th placed marginal is sigma[l-q] */
        int nr = l - 1 - r;
        run[0] = 0.0;
        for (int q = 1; q <= nr; ++q) run[q] = -INFINITY;
        for (int64_t t = T - 1; t >= 0; --t) {
            if (t < T - 1) {
                double dx = (xm[t + 1] - xm[t]) / eps;
                for (int q = 1; q <= nr; ++q) run[q] -= rate(l, q) * dx;
            }
            int m = mid[t];
            if (m == j) { right[loc[t]] = run[nr]; continue; }
            for (int q = 1; q <= nr; ++q)
                if (sigma[l - q] == m) run[q] = lae(run[q], g[m][loc[t]] / eps + run[q - 1]);
        }
        for (int64_t i = 0; i < N[j]; ++i) lnM_out[i] = lae(lnM_out[i], left[i] + right[i]);
    } while (next_perm(sigma, l));

    free(left);
    free(right);
    merged_free(mid, loc, xm);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Subset-state form.                                                   */
/* ------------------------------------------------------------------ */

/* Forward running sums over subsets S of the marginals in `bits` (a list of
 * nb marginals): L[S] = ln of the sum over placements of one point of each
 * marginal in S, all strictly before the current position, of
 * prod phi * exp(-cost integral up to the current position).  Orderings that
 * place the same set S share L[S]; L[empty] = 0.  The update at a point of
 * marginal m adds phi_m times L[S without m] to every S containing m; the
 * decay between points is exp(-|S|(l-|S|) dx/eps).
 *
 * The backward sums are the same with the order reversed.
 *
 * For target j (bits = all marginals but j) the marginal product at a j-point
 * is  M_j = sum_S F_S(before) * G_{R\S}(after)  over S subset of R. */

/* ln M_j at all j-points (want == NULL) or at the sorted list of j-point
 * indices want[0..nwant-1] (results in lnM_out[0..nwant-1]). */
int mo_marginal_subset_sel(int l, const int64_t *N, const double *const *x,
                           const double *const *g, double eps, int j,
                           int64_t nwant, const int64_t *want, double *lnM_out)
{
    int *mid; int64_t *loc; double *xm; int64_t T;
    int rc = merged_alloc(l, N, x, &mid, &loc, &xm, &T);
    if (rc) { merged_free(mid, loc, xm); return rc; }

    int nb = 0, bitof[MO_MAXL];
    for (int k = 0; k < l; ++k) bitof[k] = (k == j) ? -1 : nb++;
    const unsigned NS = 1u << nb;
    const unsigned FULL = NS - 1u;
    int64_t nout = want ? nwant : N[j];
    /* slot of each j-point in the output (or -1) */
    int64_t *slot = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N[j] ? N[j] : 1));
    for (int64_t i = 0; i < N[j]; ++i) slot[i] = want ? -1 : i;
    if (want)
        for (int64_t w = 0; w < nwant; ++w) slot[want[w]] = w;
    double *Gst = (double *)malloc(sizeof(double) * (size_t)(nout ? nout : 1) * NS);
    double *L = (double *)malloc(sizeof(double) * NS);
    int *lev = (int *)malloc(sizeof(int) * NS);
    for (unsigned S = 0; S < NS; ++S) lev[S] = popcount_u(S);

    /* backward sweep: store G at requested j-points */
    for (unsigned S = 0; S < NS; ++S) L[S] = (S == 0) ? 0.0 : -INFINITY;
    for (int64_t t = T - 1; t >= 0; --t) {
        if (t < T - 1) {
            double dx = (xm[t + 1] - xm[t]) / eps;
            for (unsigned S = 1; S < NS; ++S) L[S] -= rate(l, lev[S]) * dx;
        }
        int m = mid[t];
        if (m == j) {
            int64_t s = slot[loc[t]];
            if (s >= 0) memcpy(Gst + (size_t)s * NS, L, sizeof(double) * NS);
            continue;
        }
        unsigned b = 1u << bitof[m];
        double lg = g[m][loc[t]] / eps;
        for (unsigned S = 0; S < NS; ++S)
            if (S & b) L[S] = lae(L[S], lg + L[S ^ b]);
    }
    /* forward sweep: combine */
    for (unsigned S = 0; S < NS; ++S) L[S] = (S == 0) ? 0.0 : -INFINITY;
    for (int64_t t = 0; t < T; ++t) {
        if (t > 0) {
            double dx = (xm[t] - xm[t - 1]) / eps;
            for (unsigned S = 1; S < NS; ++S) L[S] -= rate(l, lev[S]) * dx;
        }
        int m = mid[t];
        if (m == j) {
            int64_t s = slot[loc[t]];
            if (s >= 0) {
                double acc = -INFINITY;
                for (unsigned S = 0; S < NS; ++S)
                    acc = lae(acc, L[S] + Gst[(size_t)s * NS + (FULL ^ S)]);
                lnM_out[s] = acc;
            }
            continue;
        }
        unsigned b = 1u << bitof[m];
        double lg = g[m][loc[t]] / eps;
        for (unsigned S = 0; S < NS; ++S)
            if (S & b) L[S] = lae(L[S], lg + L[S ^ b]);
    }
    free(slot); free(Gst); free(L); free(lev);
    merged_free(mid, loc, xm);
    return 0;
}

int mo_marginal_subset(int l, const int64_t *N, const double *const *x,
                       const double *const *g, double eps, int j, double *lnM_out)
{
    return mo_marginal_subset_sel(l, N, x, g, eps, j, 0, NULL, lnM_out);
}

/* All marginals of the plan and the objective terms in one forward and one
 * backward sweep over all 2^l subsets of the l marginals.
 *   lnM_out[k][i] = ln M_k(i)              (may be NULL)
 *   *lnZ          = ln of the total mass sum_t t
 *   *W            = <C, T> = sum over tuples of c * t     (Eq. k-mmot distance)
 * The cost term uses that, between consecutive merged points, a tuple with the
 * set S left of the gap pays |S|(l-|S|) per unit length, so
 *   W = sum_t dx_t * sum_S |S|(l-|S|) F_S(x_t^-) G_{S^c}(x_t, incl. t)
 * where F excludes point t and G includes it. */
int mo_allpass(int l, const int64_t *N, const double *const *x, const double *const *g,
               double eps, double *const *lnM_out, double *lnZ, double *W)
{
    int *mid; int64_t *loc; double *xm; int64_t T;
    int rc = merged_alloc(l, N, x, &mid, &loc, &xm, &T);
    if (rc) { merged_free(mid, loc, xm); return rc; }
    const unsigned NS = 1u << l;
    const unsigned FULL = NS - 1u;
    int *lev = (int *)malloc(sizeof(int) * NS);
    for (unsigned S = 0; S < NS; ++S) lev[S] = popcount_u(S);
    /* G after processing point t (inclusive), stored for every point */
    double *Gi = (double *)malloc(sizeof(double) * (size_t)(T ? T : 1) * NS);
    double *L = (double *)malloc(sizeof(double) * NS);
    if (!Gi || !L) { free(lev); free(Gi); free(L); merged_free(mid, loc, xm); return -2; }

    for (unsigned S = 0; S < NS; ++S) L[S] = (S == 0) ? 0.0 : -INFINITY;
    for (int64_t t = T - 1; t >= 0; --t) {
        if (t < T - 1) {
            double dx = (xm[t + 1] - xm[t]) / eps;
            for (unsigned S = 1; S < NS; ++S) L[S] -= rate(l, lev[S]) * dx;
        }
        int m = mid[t];
        unsigned b = 1u << m;
        double lg = g[m][loc[t]] / eps;
        for (unsigned S = 0; S < NS; ++S)
            if (S & b) L[S] = lae(L[S], lg + L[S ^ b]);
        /* inclusive values: the sets that reach point t or beyond */
        memcpy(Gi + (size_t)t * NS, L, sizeof(double) * NS);
    }
    /* Forward sweep.  At point t (marginal m), with F = values before t:
     *   M_m(i) = sum over S without m of F_S * Gexcl_{(all\m)\S}
     * Gexcl at t equals Gincl at t for every set that does not contain m, and
     * (all\m)\S never contains m, so Gincl can be used directly. */
    for (unsigned S = 0; S < NS; ++S) L[S] = (S == 0) ? 0.0 : -INFINITY;
    double lnW = -INFINITY;
    for (int64_t t = 0; t < T; ++t) {
        double dx = 0.0;
        if (t > 0) {
            dx = (xm[t] - xm[t - 1]) / eps;
            for (unsigned S = 1; S < NS; ++S) L[S] -= rate(l, lev[S]) * dx;
        }
        const double *G = Gi + (size_t)t * NS;
        if (t > 0 && dx > 0.0) {
            /* cost across the gap (x_{t-1}, x_t): sum_S w_S F_S(x_t^-) G_{S^c}(incl) */
            double acc = -INFINITY;
            for (unsigned S = 1; S < FULL; ++S)
                acc = lae(acc, log(rate(l, lev[S])) + L[S] + G[FULL ^ S]);
            lnW = lae(lnW, log(dx * eps) + acc);
        }
        int m = mid[t];
        unsigned b = 1u << m;
        if (lnM_out && lnM_out[m]) {
            unsigned rest = FULL ^ b;
            double acc = -INFINITY;
            for (unsigned S = 0; S < NS; ++S)
                if (!(S & b)) acc = lae(acc, L[S] + G[rest ^ S]);
            lnM_out[m][loc[t]] = acc;
        }
        double lg = g[m][loc[t]] / eps;
        for (unsigned S = 0; S < NS; ++S)
            if (S & b) L[S] = lae(L[S], lg + L[S ^ b]);
    }
    if (lnZ) *lnZ = L[FULL];
    if (W) *W = exp(lnW);
    free(lev); free(Gi); free(L);
    merged_free(mid, loc, xm);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Literal l = 3 uniform-grid algorithms (Sec. 3).                      */
/* ------------------------------------------------------------------ */

/* Algorithm 2 (FTVP-1): out_k = sum_{i,j} K_{ijk} phi_i psi_j on a uniform
 * grid, K_{ijk} = lam^{|i-j|+|i-k|+|j-k|}.  The six class sums J_{k,p}
 * (Eq. Jk) are evaluated by the recurrences of Eq. recurrence formula Jk with
 * the prefix/suffix sums P_{k,p}, Q_{k,p} of Eq. recurrence formula PkQk; on
 * the classes the exponent coefficients are (a_p, b_p, c_p) of Eq. a_p b_p c_p,
 * so every multiplier is lam^2.  Arrays are 0-based here: index k here is the
 * paper's k+1. */
void mo_ftvp1(int64_t N, const double *phi, const double *psi, double lam, double *out)
{
    if (N <= 0) return;
    double l2 = lam * lam, l4 = l2 * l2;
    double *P1 = calloc(N, sizeof(double)), *P2 = calloc(N, sizeof(double));
    double *P3 = calloc(N, sizeof(double)), *P4 = calloc(N, sizeof(double));
    double *P5 = calloc(N, sizeof(double)), *P6 = calloc(N, sizeof(double));
    double *Q3 = calloc(N, sizeof(double)), *Q4 = calloc(N, sizeof(double));
    double *J1 = calloc(N, sizeof(double)), *J2 = calloc(N, sizeof(double));
    double *J3 = calloc(N, sizeof(double)), *J4 = calloc(N, sizeof(double));
    double *J5 = calloc(N, sizeof(double)), *J6 = calloc(N, sizeof(double));
    /* initial values */
    J1[0] = phi[0] * psi[0];
    P1[0] = phi[0];
    P2[0] = l2 * psi[0];
    P3[0] = phi[0];
    Q3[N - 1] = l2 * psi[N - 1];
    P4[0] = psi[0];
    Q4[N - 1] = l2 * phi[N - 1];
    P5[N - 1] = l2 * psi[N - 1];
    P6[N - 1] = l4 * phi[N - 1];
    /* prefix and suffix sums */
    for (int64_t k = 0; k + 1 < N; ++k) {
        int64_t r = N - 2 - k;          /* the paper's N-k, 0-based */
        P1[k + 1] = l2 * P1[k] + phi[k + 1];
        P2[k + 1] = l2 * P2[k] + l2 * psi[k + 1];
        P3[k + 1] = l2 * P3[k] + phi[k + 1];
        Q3[r] = l2 * Q3[r + 1] + l2 * psi[r];
        P4[k + 1] = l2 * P4[k] + psi[k + 1];
        Q4[r] = l2 * Q4[r + 1] + l2 * phi[r];
        P5[r] = l2 * P5[r + 1] + l2 * psi[r];
        P6[r] = l2 * P6[r + 1] + l4 * phi[r];
    }
    /* forward class sums and the two product classes */
    for (int64_t k = 0; k + 1 < N; ++k) {
        J1[k + 1] = l2 * J1[k] + psi[k + 1] * P1[k + 1];
        J2[k + 1] = l2 * J2[k] + phi[k + 1] * P2[k];
        J3[k] = P3[k] * Q3[k + 1];
        J4[k] = P4[k] * Q4[k + 1];
    }
    /* backward class sums */
    for (int64_t k = N - 1; k >= 1; --k) J5[k - 1] = l2 * J5[k] + phi[k] * P5[k];
    for (int64_t k = N - 2; k >= 1; --k) J6[k - 1] = l2 * J6[k] + psi[k] * P6[k + 1];
    for (int64_t k = 0; k < N; ++k) out[k] = J1[k] + J2[k] + J3[k] + J4[k] + J5[k] + J6[k];
    free(P1); free(P2); free(P3); free(P4); free(P5); free(P6); free(Q3); free(Q4);
    free(J1); free(J2); free(J3); free(J4); free(J5); free(J6);
}

/* Algorithm 3 (FTVP-2): out_k = sum_{i,j} c_{ijk} K_{ijk} phi_i psi_j with
 * c_{ijk} = (|i-j|+|i-k|+|j-k|) h.  First-moment class sums hat J_{k,p}
 * (Eq. hat Jk) by Eq. recurrence formula hat Jk, with the moment sums R, S of
 * Eq. RkSk / recurrence formula RkSk.  By Eq. RkSk the backward starting
 * values are R_{N,5} = b_5 N psi_N lam^{a_5 N + b_5 N + c_5 (N-1)} = 2N lam^2 psi_N
 * and R_{N,6} = a_6 N phi_N lam^{...} = 2N lam^4 phi_N; both carry the factor N. */
void mo_ftvp2(int64_t N, const double *phi, const double *psi, double lam, double h, double *out)
{
    if (N <= 0) return;
    double l2 = lam * lam, l4 = l2 * l2;
    double *P1 = calloc(N, sizeof(double)), *P2 = calloc(N, sizeof(double));
    double *P3 = calloc(N, sizeof(double)), *P4 = calloc(N, sizeof(double));
    double *P5 = calloc(N, sizeof(double)), *P6 = calloc(N, sizeof(double));
    double *Q3 = calloc(N, sizeof(double)), *Q4 = calloc(N, sizeof(double));
    double *J1 = calloc(N, sizeof(double)), *J2 = calloc(N, sizeof(double));
    double *J5 = calloc(N, sizeof(double)), *J6 = calloc(N, sizeof(double));
    double *R1 = calloc(N, sizeof(double)), *R2 = calloc(N, sizeof(double));
    double *R3 = calloc(N, sizeof(double)), *R4 = calloc(N, sizeof(double));
    double *R5 = calloc(N, sizeof(double)), *R6 = calloc(N, sizeof(double));
    double *S3 = calloc(N, sizeof(double)), *S4 = calloc(N, sizeof(double));
    double *H1 = calloc(N, sizeof(double)), *H2 = calloc(N, sizeof(double));
    double *H3 = calloc(N, sizeof(double)), *H4 = calloc(N, sizeof(double));
    double *H5 = calloc(N, sizeof(double)), *H6 = calloc(N, sizeof(double));
    /* zeroth-moment sums as in Algorithm 2 */
    J1[0] = phi[0] * psi[0];
    P1[0] = phi[0]; P2[0] = l2 * psi[0]; P3[0] = phi[0]; Q3[N - 1] = l2 * psi[N - 1];
    P4[0] = psi[0]; Q4[N - 1] = l2 * phi[N - 1]; P5[N - 1] = l2 * psi[N - 1]; P6[N - 1] = l4 * phi[N - 1];
    for (int64_t k = 0; k + 1 < N; ++k) {
        int64_t r = N - 2 - k;
        P1[k + 1] = l2 * P1[k] + phi[k + 1];
        P2[k + 1] = l2 * P2[k] + l2 * psi[k + 1];
        P3[k + 1] = l2 * P3[k] + phi[k + 1];
        Q3[r] = l2 * Q3[r + 1] + l2 * psi[r];
        P4[k + 1] = l2 * P4[k] + psi[k + 1];
        Q4[r] = l2 * Q4[r + 1] + l2 * phi[r];
        P5[r] = l2 * P5[r + 1] + l2 * psi[r];
        P6[r] = l2 * P6[r + 1] + l4 * phi[r];
    }
    for (int64_t k = 0; k + 1 < N; ++k) {
        J1[k + 1] = l2 * J1[k] + psi[k + 1] * P1[k + 1];
        J2[k + 1] = l2 * J2[k] + phi[k + 1] * P2[k];
    }
    for (int64_t k = N - 1; k >= 1; --k) J5[k - 1] = l2 * J5[k] + phi[k] * P5[k];
    for (int64_t k = N - 2; k >= 1; --k) J6[k - 1] = l2 * J6[k] + psi[k] * P6[k + 1];

    /* first-moment sums; the paper's index k+1 is 0-based k, so the paper's
     * multiplier (k+1) for 0-based position k is (double)(k + 1) */
    double Nd = (double)N;
    R1[0] = -2.0 * phi[0];
    R2[0] = -2.0 * l2 * psi[0];
    R3[0] = -2.0 * phi[0];
    S3[N - 1] = 2.0 * Nd * l2 * psi[N - 1];
    R4[0] = -2.0 * psi[0];
    S4[N - 1] = 2.0 * Nd * l2 * phi[N - 1];
    R5[N - 1] = 2.0 * Nd * l2 * psi[N - 1];
    R6[N - 1] = 2.0 * Nd * l4 * phi[N - 1];
    for (int64_t k = 0; k + 1 < N; ++k) {
        int64_t r = N - 2 - k;          /* 0-based index of the paper's N-k */
        double kp1 = (double)(k + 2);   /* paper's k+1 for 1-based k = k+1 */
        double nk = (double)(r + 1);    /* paper's N-k */
        R1[k + 1] = l2 * R1[k] - 2.0 * kp1 * phi[k + 1];
        R2[k + 1] = l2 * R2[k] - 2.0 * kp1 * l2 * psi[k + 1];
        R3[k + 1] = l2 * R3[k] - 2.0 * kp1 * phi[k + 1];
        S3[r] = l2 * S3[r + 1] + 2.0 * nk * l2 * psi[r];
        R4[k + 1] = l2 * R4[k] - 2.0 * kp1 * psi[k + 1];
        S4[r] = l2 * S4[r + 1] + 2.0 * nk * l2 * phi[r];
        R5[r] = l2 * R5[r + 1] + 2.0 * nk * l2 * psi[r];
        R6[r] = l2 * R6[r + 1] + 2.0 * nk * l4 * phi[r];
    }
    /* hat J */
    H1[0] = 0.0;   /* (a_1+b_1+c_1) phi_1 psi_1 lam^0 = 0 */
    for (int64_t k = 0; k + 1 < N; ++k) {
        double kp1 = (double)(k + 2);
        H1[k + 1] = l2 * H1[k] + 2.0 * l2 * J1[k] + psi[k + 1] * R1[k + 1] + 2.0 * kp1 * psi[k + 1] * P1[k + 1];
        H2[k + 1] = l2 * H2[k] + 2.0 * l2 * J2[k] + phi[k + 1] * R2[k] + 2.0 * kp1 * phi[k + 1] * P2[k];
        H3[k] = R3[k] * Q3[k + 1] + P3[k] * S3[k + 1];
        H4[k] = R4[k] * Q4[k + 1] + P4[k] * S4[k + 1];
    }
    for (int64_t k = N - 1; k >= 1; --k) {
        double km1 = (double)k;         /* paper's k-1 for 1-based k = k+1 */
        H5[k - 1] = l2 * H5[k] + 2.0 * l2 * J5[k] + phi[k] * R5[k] - 2.0 * km1 * phi[k] * P5[k];
    }
    for (int64_t k = N - 2; k >= 1; --k) {
        double km1 = (double)k;
        H6[k - 1] = l2 * H6[k] + 2.0 * l2 * J6[k] + psi[k] * R6[k + 1] - 2.0 * km1 * psi[k] * P6[k + 1];
    }
    for (int64_t k = 0; k < N; ++k) out[k] = h * (H1[k] + H2[k] + H3[k] + H4[k] + H5[k] + H6[k]);
    free(P1); free(P2); free(P3); free(P4); free(P5); free(P6); free(Q3); free(Q4);
    free(J1); free(J2); free(J5); free(J6);
    free(R1); free(R2); free(R3); free(R4); free(R5); free(R6); free(S3); free(S4);
    free(H1); free(H2); free(H3); free(H4); free(H5); free(H6);
}

/* Algorithm 4 (fast Sinkhorn for l = 3 on a uniform grid with spacing h).
 * Scalings start at 1/N; each iteration updates phi, psi, varphi in turn with
 * FTVP-1 products (the kernel is symmetric in its three indices, which is the
 * index-permutation argument of Sec. 3.3), then Res sums the L1 errors of the
 * first two marginals.  Returns W = <varphi, FTVP-2(phi, psi)>; FTVP-2 already
 * carries the factor h of Eq. tensor-vector-product-2, so no second h. */
int mo_fs3(int64_t N, const double *u, const double *v, const double *w, double h, double eps,
           double tol, int itr_max, double *phi, double *psi, double *vphi,
           double *W, int *iters, double *res)
{
    double lam = exp(-h / eps);
    double *tmp = (double *)malloc(sizeof(double) * (size_t)N);
    double *tmp2 = (double *)malloc(sizeof(double) * (size_t)N);
    for (int64_t i = 0; i < N; ++i) { phi[i] = psi[i] = vphi[i] = 1.0 / (double)N; }
    int t = 0;
    double Res = INFINITY;
    while (t < itr_max && Res > tol) {
        t += 1;
        mo_ftvp1(N, psi, vphi, lam, tmp);
        for (int64_t i = 0; i < N; ++i) phi[i] = u[i] / tmp[i];
        mo_ftvp1(N, phi, vphi, lam, tmp);
        for (int64_t i = 0; i < N; ++i) psi[i] = v[i] / tmp[i];
        mo_ftvp1(N, phi, psi, lam, tmp);
        for (int64_t i = 0; i < N; ++i) vphi[i] = w[i] / tmp[i];
        mo_ftvp1(N, psi, vphi, lam, tmp);
        mo_ftvp1(N, phi, vphi, lam, tmp2);
        Res = 0.0;
        for (int64_t i = 0; i < N; ++i)
            Res += fabs(phi[i] * tmp[i] - u[i]) + fabs(psi[i] * tmp2[i] - v[i]);
    }
    mo_ftvp2(N, phi, psi, lam, h, tmp);
    double acc = 0.0;
    for (int64_t i = 0; i < N; ++i) acc += vphi[i] * tmp[i];
    *W = acc;
    *iters = t;
    *res = Res;
    free(tmp);
    free(tmp2);
    return 0;
}

/* ------------------------------------------------------------------ */
/* General-l Sinkhorn in the log domain.                                */
/* ------------------------------------------------------------------ */

/* Sum over marginals k < kend of ||phi_k . M_k - mu_k||_1, from ln M_k.  The
 * stopping test of Algorithm 1 sums marginals 1..l-1 (kend = l - 1): the last
 * marginal is exact right after its update. */
static double residual_from(int kend, const int64_t *N, const double *const *mu,
                            double *const *g, double eps, double *const *lnM)
{
    double res = 0.0;
    for (int k = 0; k < kend; ++k)
        for (int64_t i = 0; i < N[k]; ++i) {
            double a = g[k][i] / eps + lnM[k][i];
            double marg = (a == -INFINITY) ? 0.0 : exp(a);
            res += fabs(marg - mu[k][i]);
        }
    return res;
}

/* Potential update of marginal j (Sec. 4.2 update formulas, phi_j = mu_j / M_j,
 * written for g_j = eps ln phi_j).  A zero weight gives g = -inf. */
static void update_potential(int64_t n, const double *mu, const double *lnM, double eps, double *g)
{
    for (int64_t i = 0; i < n; ++i)
        g[i] = (mu[i] > 0.0) ? eps * (log(mu[i]) - lnM[i]) : -INFINITY;
}

/* Gauss-Seidel Sinkhorn.  g[k] must hold the starting potentials (the paper
 * starts from phi = 1/N, i.e. g = -eps ln N_k) and receives the final ones.
 * Each iteration updates j = 1..l in order; then Res is the summed L1 marginal
 * error of marginals 1..l-1 at the end of the iteration (the stopping test of
 * Algorithm 1; marginal l is exact after its update); the loop runs while
 * t < itr_max and Res > tol (Algorithm 1 loop).  With tol <= 0 the residual is
 * evaluated only once, after the last iteration (the loop cannot stop early).
 * Outputs: iterations, residual, W = <C,T>, primal sum_k <g_k, marg_k>,
 * dual sum_k <g_k, mu_k> + eps - eps Z, and the mass Z. */
int mo_sinkhorn(int l, const int64_t *N, const double *const *x, const double *const *mu,
                double eps, double tol, int itr_max, double *const *g,
                int *iters, double *res, double *W, double *primal, double *dual, double *mass)
{
    double *lnM[MO_MAXL];
    int64_t maxN = 1;
    for (int k = 0; k < l; ++k) if (N[k] > maxN) maxN = N[k];
    for (int k = 0; k < l; ++k) lnM[k] = (double *)malloc(sizeof(double) * (size_t)(N[k] ? N[k] : 1));
    double *tmp = (double *)malloc(sizeof(double) * (size_t)maxN);
    int t = 0;
    double Res = INFINITY;
    int rc = 0;
    while (t < itr_max && Res > tol) {
        t += 1;
        for (int j = 0; j < l; ++j) {
            rc = mo_marginal_subset(l, N, x, (const double *const *)g, eps, j, tmp);
            if (rc) goto done;
            update_potential(N[j], mu[j], tmp, eps, g[j]);
        }
        if (tol > 0.0 || t == itr_max) {
            double lnZ, Wv;
            rc = mo_allpass(l, N, x, (const double *const *)g, eps, lnM, &lnZ, &Wv);
            if (rc) goto done;
            Res = residual_from(l - 1, N, mu, g, eps, lnM);
        }
    }
    {
        double lnZ, Wv;
        rc = mo_allpass(l, N, x, (const double *const *)g, eps, lnM, &lnZ, &Wv);
        if (rc) goto done;
        if (t == 0) Res = residual_from(l - 1, N, mu, g, eps, lnM);
        double P = 0.0, D = 0.0;
        for (int k = 0; k < l; ++k)
            for (int64_t i = 0; i < N[k]; ++i) {
                if (g[k][i] == -INFINITY) continue;
                double marg = exp(g[k][i] / eps + lnM[k][i]);
                P += g[k][i] * marg;
                D += g[k][i] * mu[k][i];
            }
        double Z = exp(lnZ);
        D += eps - eps * Z;
        *iters = t; *res = Res; *W = Wv; *primal = P; *dual = D; *mass = Z;
    }
done:
    for (int k = 0; k < l; ++k) free(lnM[k]);
    free(tmp);
    return rc;
}
