/*
 * ORACLE — test infrastructure only.
 *
 * A plain, slow, FP64 CPU restatement of the matrix-free Galerkin operator of
 * Brumm, "A fast matrix-free algorithm for spectral approximations to the
 * Schroedinger equation" (arXiv:1403.3511).  It exists to check the CUDA
 * library, shares no code with it, and must never be linked into, imported by
 * or called from the product path.  Only tests/, __graft_entry__.smoke() and
 * the cpu_baseline / reference legs of bench.py may use it.
 *
 * Conventions
 *   - An index set is a list of multi-indices k in N^N stored row-major
 *     (size x N, int32), sorted lexicographically with the LAST coordinate
 *     varying fastest.  Rank = position in that list.
 *   - Vectors are complex128 (C99 double _Complex, i.e. interleaved re/im).
 *   - A Chebyshev term is a multi-index r in N^N plus a real weight alpha_r,
 *     standing for alpha_r * prod_l T_{r_l}(x_l / L)  (Sec. 1.3).
 */
#ifndef HX_ORACLE_H
#define HX_ORACLE_H

#include <complex.h>
#include <stdint.h>

typedef double _Complex ho_z;

typedef struct {
    int N;
    int64_t size;
    int32_t *k;   /* size x N */
    int32_t *up;  /* N x size: rank of k+e_l, -1 if absent (built on demand) */
    int32_t *dn;  /* N x size: rank of k-e_l, -1 if absent (built on demand) */
} ho_set;

/* Factor order inside one Chebyshev product (Sec. 3.2 / 3.3):
 *   HO_ORDER_EQ  : T_{r_1}(X1/L)( ... (T_{r_N}(XN/L) v)) as written in Eq. (Horner):
 *                  axis N is applied to v first.
 *   HO_ORDER_ALG : axes applied to v in the order l = 1, 2, ..., N, as in the
 *                  loop of Algorithm fast_algorithm.
 *   HO_ORDER_SYM : the mean of the two, which is symmetric for real alpha. */
enum { HO_ORDER_SYM = 0, HO_ORDER_EQ = 1, HO_ORDER_ALG = 2 };

int64_t ho_hc_count(int N, int64_t B);
ho_set *ho_hc_create(int N, int64_t B);
ho_set *ho_list_create(int N, int64_t size, const int32_t *k);
void ho_set_free(ho_set *s);
int32_t *ho_set_k(ho_set *s);
int64_t ho_set_size(const ho_set *s);
int64_t ho_rank(const ho_set *s, const int32_t *k);
int ho_neighbors_build(ho_set *s);

void ho_direct_op(ho_set *s, int l, const ho_z *v, ho_z *out);
void ho_cheb_apply(ho_set *s, int l, int r, double L, const ho_z *v, ho_z *out);
int ho_fast_algorithm(ho_set *s, int nterms, const int32_t *r, const double *alpha,
                      double L, int order, const ho_z *v, ho_z *res);
void ho_diag_apply(const ho_set *s, const ho_z *v, ho_z *out);
int ho_apply(ho_set *s, int nterms, const int32_t *r, const double *alpha, double L,
             int order, const ho_z *v, ho_z *y);
int ho_apply_rows_local(ho_set *full, int64_t B, int nterms, const int32_t *r,
                        const double *alpha, double L, int order, const ho_z *c,
                        int64_t nrows, const int64_t *rows, ho_z *out);

#endif
