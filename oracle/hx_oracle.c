/*
 * ORACLE — test infrastructure only (see hx_oracle.h).  Plain FP64 C99, no
 * blocking, fusion or reordering beyond what the paper's definitions state.
 * Section / equation references are to Brumm, arXiv:1403.3511.
 */
#include "hx_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Index sets (Sec. 1.2)                                                      */
/* ------------------------------------------------------------------------- */

/* Number of k in N^n with prod_l (1 + k_l) <= budget: the hyperbolic cross of
 * Sec. 1.2 with K + 1 = budget.  Counted leaf by leaf, which is slow but plain. */
static int64_t hc_count_rec(int n, int64_t budget)
{
    if (n == 0) return 1;
    int64_t total = 0;
    for (int64_t k = 0; 1 + k <= budget; ++k) total += hc_count_rec(n - 1, budget / (1 + k));
    return total;
}

int64_t ho_hc_count(int N, int64_t B)
{
    if (N < 1 || B < 1) return 0;
    return hc_count_rec(N, B);
}

/* Writes the hyperbolic cross in lexicographic order, last coordinate fastest:
 * coordinate d runs over 0 .. budget_d - 1 where budget_d = floor(B / prod_{i<d}(1+k_i)). */
static void hc_fill_rec(int N, int d, int64_t budget, int32_t *prefix, int32_t *out, int64_t *pos)
{
    if (d == N) {
        memcpy(out + (*pos) * N, prefix, sizeof(int32_t) * (size_t)N);
        ++*pos;
        return;
    }
    for (int64_t k = 0; 1 + k <= budget; ++k) {
        prefix[d] = (int32_t)k;
        hc_fill_rec(N, d + 1, budget / (1 + k), prefix, out, pos);
    }
}

static ho_set *set_alloc(int N, int64_t size)
{
    ho_set *s = (ho_set *)calloc(1, sizeof(ho_set));
    if (!s) return NULL;
    s->N = N;
    s->size = size;
    s->k = (int32_t *)malloc(sizeof(int32_t) * (size_t)(size > 0 ? size : 1) * (size_t)N);
    if (!s->k) { free(s); return NULL; }
    return s;
}

ho_set *ho_hc_create(int N, int64_t B)
{
    if (N < 1 || B < 1) return NULL;
    int64_t size = ho_hc_count(N, B);
    ho_set *s = set_alloc(N, size);
    if (!s) return NULL;
    int32_t *prefix = (int32_t *)calloc((size_t)N, sizeof(int32_t));
    int64_t pos = 0;
    hc_fill_rec(N, 0, B, prefix, s->k, &pos);
    free(prefix);
    return s;
}

static int lex_cmp(const int32_t *a, const int32_t *b, int N)
{
    for (int l = 0; l < N; ++l) {
        if (a[l] < b[l]) return -1;
        if (a[l] > b[l]) return 1;
    }
    return 0;
}

/* Any finite index set given as a strictly increasing list (Sec. 1.2 allows
 * any downward-closed set; the oracle accepts any set at all). */
ho_set *ho_list_create(int N, int64_t size, const int32_t *k)
{
    if (N < 1 || size < 0) return NULL;
    for (int64_t i = 1; i < size; ++i)
        if (lex_cmp(k + (i - 1) * N, k + i * N, N) >= 0) return NULL;
    ho_set *s = set_alloc(N, size);
    if (!s) return NULL;
    if (size > 0) memcpy(s->k, k, sizeof(int32_t) * (size_t)size * (size_t)N);
    return s;
}

void ho_set_free(ho_set *s)
{
    if (!s) return;
    free(s->k);
    free(s->up);
    free(s->dn);
    free(s);
}

int32_t *ho_set_k(ho_set *s) { return s->k; }
int64_t ho_set_size(const ho_set *s) { return s->size; }

/* Position of k in the sorted list, or -1: plain binary search. */
int64_t ho_rank(const ho_set *s, const int32_t *k)
{
    int64_t lo = 0, hi = s->size - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        int c = lex_cmp(s->k + mid * s->N, k, s->N);
        if (c == 0) return mid;
        if (c < 0) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

int ho_neighbors_build(ho_set *s)
{
    if (s->up) return 0;
    int N = s->N;
    s->up = (int32_t *)malloc(sizeof(int32_t) * (size_t)N * (size_t)(s->size ? s->size : 1));
    s->dn = (int32_t *)malloc(sizeof(int32_t) * (size_t)N * (size_t)(s->size ? s->size : 1));
    if (!s->up || !s->dn) { free(s->up); free(s->dn); s->up = s->dn = NULL; return -1; }
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    for (int64_t j = 0; j < s->size; ++j) {
        for (int l = 0; l < N; ++l) {
            memcpy(tmp, s->k + j * N, sizeof(int32_t) * (size_t)N);
            tmp[l] += 1;
            s->up[(int64_t)l * s->size + j] = (int32_t)ho_rank(s, tmp);
            tmp[l] -= 2;
            s->dn[(int64_t)l * s->size + j] = tmp[l] >= 0 ? (int32_t)ho_rank(s, tmp) : -1;
        }
    }
    free(tmp);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Coordinate matrices and the fast algorithm (Sec. 3)                        */
/* ------------------------------------------------------------------------- */

/* (X^{(l)} v)_j = sqrt(j_l/2) v_{j-e_l} + sqrt((j_l+1)/2) v_{j+e_l}, Eq. (DirectOperationWithX);
 * a term whose index lies outside the set is absent (the set is truncated there). */
void ho_direct_op(ho_set *s, int l, const ho_z *v, ho_z *out)
{
    ho_neighbors_build(s);
    const int32_t *up = s->up + (int64_t)l * s->size;
    const int32_t *dn = s->dn + (int64_t)l * s->size;
    for (int64_t j = 0; j < s->size; ++j) {
        double jl = (double)s->k[j * s->N + l];
        ho_z acc = 0.0;
        if (dn[j] >= 0) acc += sqrt(jl / 2.0) * v[dn[j]];
        if (up[j] >= 0) acc += sqrt((jl + 1.0) / 2.0) * v[up[j]];
        out[j] = acc;
    }
}

/* out = T_r(X^{(l)}/L) v using T_0 = 1, T_1(x) = x, T_{n+1} = 2x T_n - T_{n-1},
 * Eq. (ChebyshevRecurrence), with x replaced by the coordinate matrix over L. */
void ho_cheb_apply(ho_set *s, int l, int r, double L, const ho_z *v, ho_z *out)
{
    int64_t n = s->size;
    if (r == 0) { memcpy(out, v, sizeof(ho_z) * (size_t)n); return; }
    ho_z *t_prev = (ho_z *)malloc(sizeof(ho_z) * (size_t)(n ? n : 1)); /* T_{m-1} v */
    ho_z *t_cur = (ho_z *)malloc(sizeof(ho_z) * (size_t)(n ? n : 1));  /* T_m v */
    ho_z *x_t = (ho_z *)malloc(sizeof(ho_z) * (size_t)(n ? n : 1));
    memcpy(t_prev, v, sizeof(ho_z) * (size_t)n);
    ho_direct_op(s, l, v, t_cur);
    for (int64_t j = 0; j < n; ++j) t_cur[j] /= L;
    for (int m = 1; m < r; ++m) {
        ho_direct_op(s, l, t_cur, x_t);
        for (int64_t j = 0; j < n; ++j) {
            ho_z next = 2.0 * x_t[j] / L - t_prev[j];
            t_prev[j] = t_cur[j];
            t_cur[j] = next;
        }
    }
    memcpy(out, t_cur, sizeof(ho_z) * (size_t)n);
    free(t_prev); free(t_cur); free(x_t);
}

/* One Chebyshev product prod_l T_{r_l}(X^{(l)}/L) applied to v in the given
 * axis order.  Each term starts again from the input vector. */
static void product_apply(ho_set *s, const int32_t *r, double L, int ascending, const ho_z *v, ho_z *out, ho_z *tmp)
{
    int N = s->N;
    memcpy(out, v, sizeof(ho_z) * (size_t)s->size);
    for (int i = 0; i < N; ++i) {
        int l = ascending ? i : N - 1 - i;
        if (r[l] == 0) continue;
        ho_cheb_apply(s, l, r[l], L, out, tmp);
        memcpy(out, tmp, sizeof(ho_z) * (size_t)s->size);
    }
}

/* res = W^pol(X_K) v = sum_r alpha_r prod_l T_{r_l}(X^{(l)}/L) v, Eq. (Horner), term by term
 * as in Algorithm fast_algorithm.  order selects the factor order (hx_oracle.h). */
int ho_fast_algorithm(ho_set *s, int nterms, const int32_t *r, const double *alpha, double L,
                      int order, const ho_z *v, ho_z *res)
{
    int64_t n = s->size;
    int N = s->N;
    if (ho_neighbors_build(s)) return -1;
    ho_z *a = (ho_z *)malloc(sizeof(ho_z) * (size_t)(n ? n : 1));
    ho_z *b = (ho_z *)malloc(sizeof(ho_z) * (size_t)(n ? n : 1));
    ho_z *tmp = (ho_z *)malloc(sizeof(ho_z) * (size_t)(n ? n : 1));
    if (!a || !b || !tmp) { free(a); free(b); free(tmp); return -1; }
    for (int64_t j = 0; j < n; ++j) res[j] = 0.0;
    for (int t = 0; t < nterms; ++t) {
        const int32_t *rt = r + (int64_t)t * N;
        int active = 0;
        for (int l = 0; l < N; ++l) active += rt[l] > 0;
        if (order == HO_ORDER_ALG || order == HO_ORDER_EQ || active <= 1) {
            product_apply(s, rt, L, order == HO_ORDER_ALG, v, a, tmp);
            for (int64_t j = 0; j < n; ++j) res[j] += alpha[t] * a[j];
        } else {
            product_apply(s, rt, L, 0, v, a, tmp);
            product_apply(s, rt, L, 1, v, b, tmp);
            for (int64_t j = 0; j < n; ++j) res[j] += alpha[t] * 0.5 * (a[j] + b[j]);
        }
    }
    free(a); free(b); free(tmp);
    return 0;
}

/* (D_K v)_j = sum_l (j_l + 1/2) v_j, the harmonic-oscillator diagonal of Sec. 1.2. */
void ho_diag_apply(const ho_set *s, const ho_z *v, ho_z *out)
{
    for (int64_t j = 0; j < s->size; ++j) {
        double d = 0.0;
        for (int l = 0; l < s->N; ++l) d += (double)s->k[j * s->N + l] + 0.5;
        out[j] = d * v[j];
    }
}

/* y = A(t) v = D_K v + W^pol(X_K, t) v, the right-hand side of Eq. (ODECoefficientsPol). */
int ho_apply(ho_set *s, int nterms, const int32_t *r, const double *alpha, double L, int order,
             const ho_z *v, ho_z *y)
{
    int64_t n = s->size;
    ho_z *w = (ho_z *)malloc(sizeof(ho_z) * (size_t)(n ? n : 1));
    if (!w) return -1;
    if (ho_fast_algorithm(s, nterms, r, alpha, L, order, v, w)) { free(w); return -1; }
    ho_diag_apply(s, v, y);
    for (int64_t j = 0; j < n; ++j) y[j] += w[j];
    free(w);
    return 0;
}

/* Selected entries y_j of y = A(t) c on a large set, one row at a time.
 *
 * Row j of a Chebyshev product only involves index paths that start at j and
 * take at most r_l steps along each axis l, and only axes with r_l > 0 move.
 * So the product evaluated on a window
 *     W_j = { k in K : k_l = j_l off the term's axes,  |k_l - j_l| <= rad_l on them }
 * with rad_l >= r_l (and c restricted to W_j) gives the same value at j as on all
 * of K: every path from j stays inside W_j and sees the same set membership.
 * Terms are grouped by their set of active axes; each group is evaluated by the
 * same fast algorithm as ho_fast_algorithm on one window whose radius on each
 * axis is the largest degree of the group. */
int ho_apply_rows_local(ho_set *full, int64_t B, int nterms, const int32_t *r, const double *alpha,
                        double L, int order, const ho_z *c, int64_t nrows, const int64_t *rows, ho_z *out)
{
    (void)B;
    int N = full->N;
    int32_t *pt = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int32_t *lo = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int32_t *hi = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int32_t *rad = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int *group = (int *)malloc(sizeof(int) * (size_t)(nterms > 0 ? nterms : 1));
    int32_t *gr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nterms > 0 ? nterms : 1) * (size_t)N);
    double *ga = (double *)malloc(sizeof(double) * (size_t)(nterms > 0 ? nterms : 1));
    /* group id = first term with the same support */
    for (int t = 0; t < nterms; ++t) {
        group[t] = t;
        for (int u = 0; u < t; ++u) {
            int same = 1;
            for (int l = 0; l < N; ++l) same &= (r[(int64_t)t * N + l] > 0) == (r[(int64_t)u * N + l] > 0);
            if (same) { group[t] = group[u]; break; }
        }
    }
    for (int64_t q = 0; q < nrows; ++q) {
        int64_t j = rows[q];
        if (j < 0 || j >= full->size) {
            free(pt); free(lo); free(hi); free(rad); free(group); free(gr); free(ga);
            return -1;
        }
        const int32_t *kj = full->k + j * N;
        double dj = 0.0;
        for (int l = 0; l < N; ++l) dj += (double)kj[l] + 0.5;
        ho_z acc = dj * c[j];
        for (int g = 0; g < nterms; ++g) {
            if (group[g] != g) continue;
            int ng = 0;
            for (int l = 0; l < N; ++l) rad[l] = 0;
            for (int t = g; t < nterms; ++t) {
                if (group[t] != g) continue;
                memcpy(gr + (int64_t)ng * N, r + (int64_t)t * N, sizeof(int32_t) * (size_t)N);
                ga[ng++] = alpha[t];
                for (int l = 0; l < N; ++l)
                    if (r[(int64_t)t * N + l] > rad[l]) rad[l] = r[(int64_t)t * N + l];
            }
            int64_t box = 1;
            for (int l = 0; l < N; ++l) {
                lo[l] = kj[l] - rad[l] < 0 ? 0 : kj[l] - rad[l];
                hi[l] = kj[l] + rad[l];
                box *= (int64_t)(hi[l] - lo[l] + 1);
            }
            /* enumerate the box in lexicographic order, keep members of K */
            int32_t *wk = (int32_t *)malloc(sizeof(int32_t) * (size_t)box * (size_t)N);
            int64_t *widx = (int64_t *)malloc(sizeof(int64_t) * (size_t)box);
            int64_t wn = 0, center = -1;
            memcpy(pt, lo, sizeof(int32_t) * (size_t)N);
            for (int64_t b = 0; b < box; ++b) {
                int64_t idx = ho_rank(full, pt);
                if (idx >= 0) {
                    memcpy(wk + wn * N, pt, sizeof(int32_t) * (size_t)N);
                    widx[wn] = idx;
                    if (idx == j) center = wn;
                    ++wn;
                }
                for (int l = N - 1; l >= 0; --l) { /* odometer, last coordinate fastest */
                    if (pt[l] < hi[l]) { ++pt[l]; break; }
                    pt[l] = lo[l];
                }
            }
            ho_set *win = ho_list_create(N, wn, wk);
            ho_z *cw = (ho_z *)malloc(sizeof(ho_z) * (size_t)wn);
            ho_z *yw = (ho_z *)malloc(sizeof(ho_z) * (size_t)wn);
            for (int64_t i = 0; i < wn; ++i) cw[i] = c[widx[i]];
            ho_fast_algorithm(win, ng, gr, ga, L, order, cw, yw);
            acc += yw[center];
            ho_set_free(win);
            free(cw); free(yw); free(wk); free(widx);
        }
        out[q] = acc;
    }
    free(pt); free(lo); free(hi); free(rad); free(group); free(gr); free(ga);
    return 0;
}
