// Internal declarations of libhx (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/hx.h"

namespace hx {

constexpr int kMaxN = 16;
constexpr int kMaxOps = 48;
constexpr int kMaxDelta = 255;                 // distinct row offsets of one problem (both stages)
constexpr int kMaxDidx = 4096;                 // footprint -> offset map entries of one operator set
constexpr int kMaxDeg = HX_MAX_DEG;
constexpr int kSpan = 2 * kMaxDeg + 1;         // offsets -deg..deg
constexpr int kMaxKrylov = 32;
constexpr int kApplyThreads = 256;

void set_error(const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);

// ---------------------------------------------------------------------------------------
// Index set on the device.
//
// Canonical order is lexicographic, last coordinate fastest.  A row is the set of elements
// sharing one prefix p = (k_0, ..., k_{N-2}); it holds k_{N-1} = 0 .. floor(B / q(p)) - 1,
// q(p) = prod (1 + p_l), stored contiguously, and the rows follow each other in the
// lexicographic order of their prefixes.  For N = 1 there is one row.
//
// Rank tables: for level m >= 1 and prefix product q (1 <= q <= B),
//   Q_m(q, k) = sum_{i<k} |K_m(floor(B / (q (1 + i))))|,   0 <= k <= floor(B / q),
// stored at Q[(m - 1) * qtotal + qoff[q] + k].  Then
//   rank(k) = sum_{d<N-1} Q_{N-1-d}(q_d, k_d) + k_{N-1},   q_d = prod_{l<d} (1 + k_l).
// ---------------------------------------------------------------------------------------
struct DevSet {
    int N, B, size, nrow, qtotal;
    const int4 *row_info;             // nrow: {start rank, q(p), sum_l p_l, length}
    const uint16_t *row_k;            // nrow x (N - 1) prefixes
    const int4 *elem;                 // size: per element {row, prod_l (1 + k_l), sum_l k_l, k_{N-1} | row length << 16}
    const int *qoff;                  // B + 2
    const int *Q;                     // (N - 1) x qtotal
    const int *nt;                    // nt[x] = floor(B / x), x = 1..B (nt[0] unused)
};

struct IndexSetHost {
    int N;
    int B;
    int64_t size;
    int nrow;
    int qtotal;
    std::vector<int> qoff;            // B + 2
    std::vector<int> Q;               // (N - 1) x qtotal
    std::vector<int4> row_info;       // nrow
    std::vector<uint16_t> row_k;      // nrow x (N - 1)
};

// ---------------------------------------------------------------------------------------
// Compiled potential.  Each op contributes w(t) * (op matrix) * (input) to A c:
//   kind 0: identity;  kind 1: P(X_a) (line);  kind 2: Sym/ordered P(X_a) Q(X_b) (plane, a < b).
// The input is c (src = -1) or a channel vector written by a first stage.  A plane op whose
// footprint is large is evaluated in two stages: stage 1 writes the channels Q(X_b) c and
// P(X_a) c (line ops with dst >= 0), stage 2 applies P(X_a) and Q(X_b) to them as line ops.
// Row tables: for a univariate polynomial P of degree p, entry
//   tab[base + ((i * (p + 1) + d) * (2p + 1)) + (s + p)] = [P(J_n / L)]_{i, i+s},  n = i + 1 + d,
// where J_n is the n x n truncated Jacobi matrix of the Hermite recurrence (Eq. (Recurrence1D)):
// row i of a fibre whose top is d steps above i (d = p stands for "p or more").
// Packed row tables (a polynomial of pure parity and degree p <= 3, whose row has p + 1 entries
// that can be nonzero, at s = -p, -p + 2, ..., p):
//   tab[pbase + (i * (p + 1) + d) * 4 + j] = [P(J_n / L)]_{i, i-p+2j},  j <= p, zero for j > p,
// one 16-byte (FP32) or 32-byte (FP64) load per row.
// ---------------------------------------------------------------------------------------
// op classes with compile-time stencils (pure parity: P has only terms of the parity of its degree)
enum { CLS_ID = 0, CLS_LINE = 1, CLS_PLANE = 10, CLS_GENERIC = 30 };
// axis roles: an axis of the row prefix (moving along it changes the row) or the last axis
enum { ROLE_ROW = 0, ROLE_LAST = 1, ROLE_NONE = 2 };

struct Op {
    int kind;
    int cls;                  // CLS_ID, CLS_LINE + p, CLS_PLANE + 3 (p-1) + (q-1) (pure parity, p, q <= 3), CLS_GENERIC
    int ra, rb;               // axis roles: ROLE_ROW (< N-1), ROLE_LAST (N-1), ROLE_NONE
    int a, b;                 // axes (b = -1 for a line op)
    int p, q;                 // degrees on a and b
    int pmask, qmask;         // bit (s + p) set when the rows can be nonzero at offset s
    int tabP, tabQ;           // row table bases
    int ptabP, ptabQ;         // packed row table bases (pure parity, degree <= 3; 0 otherwise)
    int dbase;                // base into didx (footprint position -> row offset index)
    int src, dst;             // input channel (-1 = c), output channel (stage 1 only)
    int mergeB;               // plane ops: index of a line op on axis b evaluated inside this op (-1: none)
    int merged;               // line ops: 1 when evaluated inside a plane op (skipped on its own)
    int mod;                  // hx_mod_kind
    double amp, omega, phase;
    int pw_off, pw_n;         // into the pw value array
    double pw_t0, pw_t1;
};

struct OpSet {
    int nops;
    double wAB, wBA;          // factor-order weights for plane ops
    int ndidx;
    Op op[kMaxOps];
    uint8_t didx[kMaxDidx];   // footprint position -> column of the row-offset table
};

// Row offsets used by a problem's operators: axis0, step0, axis1, step1 (axis -1 = none), over
// the prefix axes 0..N-2; offset 0 is the zero offset.  The row-offset table holds, for
// offset d and row r, the start rank of row r + offset d, or -1 when that prefix is not in K:
//   rnb[d * nrow + r].
struct RowOffsets {
    int n;
    int8_t d[kMaxDelta][4];
};

struct ApplyArgsBase {
    DevSet S;
    const int *rnb;           // row-offset table, nd x nrow
    const double *t_ptr;      // device time
    double t_shift;           // A is evaluated at *t_ptr + t_shift
    const double *pw_values;  // device
    const void *tab;          // row tables (float or double)
};

struct Problem;

struct IndexSetObj {
    IndexSetHost h;
    DevSet d;
    int device;
    void *dmem;               // one device allocation for all tables
};

// per-launch options of the apply kernel used by the Krylov step
struct ApplyFuse {
    const double *in_scale;   // multiply A v by *in_scale (nullptr = 1)
    int ndot;                 // fused dots <v_i, y> for i < ndot (0 = none)
    const void *const *vecs;  // device array of ndot vector pointers (problem dtype)
    const double *vscale;     // device array of ndot scales
    double *partials;         // gridDim.x x (2 * ndot) doubles
    unsigned *counter;        // zero-initialised; reset by the last block
    double *result;           // 2 * ndot doubles: sum_i scale_i * <v_i, y> (re, im)
};

struct Problem {
    const IndexSetObj *set;
    hx_config cfg;
    cudaStream_t stream;
    int device;
    int num_sms;
    double t_host;
    // compiled potential
    bool have_pot;
    int generation;           // incremented by every hx_potential_set (cached batch graphs check it)
    OpSet ops;                // main stage (accumulates y)
    OpSet ops1;               // first stage (writes channels), nops = 0 if unused
    int nch;                  // channel vectors
    void *chan;
    size_t chan_ld;           // elements between channels
    RowOffsets roff;          // row offsets of ops and ops1
    int *rnb;                 // row-offset table (device), roff.n x nrow
    bool skip_diag;           // internal: omit D_K (gradient direction operators)
    void *tab;                // device row tables
    size_t tab_bytes;
    double *pw_values;
    double *dscal;            // device scalars (time, etc.), see hx_krylov.cu
    // Krylov workspace
    void *krylov;
    size_t krylov_bytes;
    void *graph_exec;
    double graph_dt;
    int graph_nsteps;
    std::vector<void *> extra;   // further device allocations owned by the problem
};

// launchers (hx_apply.cu)
int launch_apply(Problem *p, const void *cin, void *cout, const double *t_ptr, double t_shift,
                 const ApplyFuse *fuse, cudaStream_t st);
int launch_export(const IndexSetObj *s, int32_t *k_dev, cudaStream_t st);
int launch_elem_info(const IndexSetObj *s);
int launch_rowtab(const DevSet &S, const RowOffsets &ro, int *rnb, cudaStream_t st);
int launch_norm(Problem *p, const void *c, int is_c128, double *partials, unsigned *counter, double *result,
                cudaStream_t st);
int apply_grid(const Problem *p);
int apply_launches(const Problem *p);   // kernels per product (1, or 2 with a channel stage)

// Lanczos workspaces outside the step graph (hx_krylov.cu), used by the adjoint gradient
struct LanczosWS {
    void *sc;          // device scalars
    void *V;           // (m + 1) complex128 vectors
    double *partials;
    size_t vec_bytes;
    int m;
};
int lanczos_alloc(Problem *p, int m, LanczosWS *L);
void lanczos_free(LanczosWS *L);
int lanczos_enqueue(Problem *p, LanczosWS *L, const double2 *c, const double *t_ptr, double t_shift, cudaStream_t st);
int lanczos_exp(Problem *p, LanczosWS *L, double h, double2 *out, cudaStream_t st);
int lanczos_project(Problem *p, LanczosWS *L, const double2 *w, double *Mcol, cudaStream_t st);
int lanczos_apply_basis(Problem *px, LanczosWS *L, int r, double2 *out, const double *t_ptr, cudaStream_t st);
int adjoint_term(LanczosWS *Lp, LanczosWS *Ll, const double *M, double dt, double *gacc, cudaStream_t st);

// Batches of independent problems stepped by one graph (hx_krylov.cu)
struct Batch {
    std::vector<Problem *> probs;
    std::vector<void *> cptr;
    std::vector<int> gen;     // member generations the graph was captured with
    cudaGraphExec_t exec = nullptr;
    double dt = 0.0;
    cudaStream_t stream = nullptr;
};
int batch_step(Batch *b, void *const *c, double dt, int nsteps);
void batch_free(Batch *b);

// Krylov stepping (hx_krylov.cu)
int krylov_step(Problem *p, void *c, double dt, int nsteps);
int krylov_info(Problem *p, int *m_used, double *alpha, double *beta, double *norm);
void *krylov_host_state(Problem *p);
void krylov_free(Problem *p);

}  // namespace hx
