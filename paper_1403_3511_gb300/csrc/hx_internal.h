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
constexpr int kMaxDelta = 160;                 // distinct outer-axis offsets of one operator set
constexpr int kMaxDidx = 4096;                 // footprint -> offset map entries of one operator set
constexpr int kMaxDeg = HX_MAX_DEG;
constexpr int kSpan = 2 * kMaxDeg + 1;         // offsets -deg..deg
constexpr int kMaxKrylov = 32;
constexpr int kItemElems = 1024;               // elements per work item (tile)
constexpr int kApplyThreads = 256;

void set_error(const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);

// ---------------------------------------------------------------------------------------
// Index set on the device.
//
// Canonical order is lexicographic, last coordinate fastest.  The first N-2 axes are the
// "outer" axes; a slab is the set of elements sharing one outer prefix p, and it is the
// 2-D hyperbolic cross {(i, j) : (1+i)(1+j) <= floor(B / q(p))}, q(p) = prod (1 + p_l),
// stored contiguously (row i, then j).  For N <= 2 there is one slab.
//
// Rank tables: for level m >= 1 and prefix product q (1 <= q <= B),
//   Q_m(q, k) = sum_{i<k} |K_m(floor(B / (q (1 + i))))|,   0 <= k <= floor(B / q),
// stored at Q[(m - 1) * qtotal + qoff[q] + k].  Then
//   rank(k) = sum_{d<N-1} Q_{N-1-d}(q_d, k_d) + k_{N-1},   q_d = prod_{l<d} (1 + k_l),
// the start of a slab with prefix p is the same sum over the outer axes, and the position
// of (i, j) inside a slab with prefix product q is Q_1(q, i) + j.
// ---------------------------------------------------------------------------------------
struct DevSet {
    int N, B, size, nslab, qtotal;
    const int *slab_start;            // nslab + 1
    const uint16_t *slab_k;           // nslab x (N - 2) outer prefixes
    const int *qoff;                  // B + 1
    const int *Q;                     // (N - 1) x qtotal
    const int *nt;                    // nt[x] = floor(B / x), x = 1..B (nt[0] unused)
};

struct IndexSetHost {
    int N;
    int B;
    int64_t size;
    int nslab;
    int qtotal;
    std::vector<int> qoff;            // B + 1
    std::vector<int> Q;               // (N - 1) x qtotal
    std::vector<int> slab_start;      // nslab + 1
    std::vector<uint16_t> slab_k;     // nslab x (N - 2)
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
// ---------------------------------------------------------------------------------------
// op classes with compile-time stencils (pure parity: P has only terms of the parity of its degree)
enum { CLS_ID = 0, CLS_LINE = 1, CLS_PLANE = 10, CLS_GENERIC = 30 };
enum { ROLE_OUT = 0, ROLE_I1 = 1, ROLE_I2 = 2, ROLE_NONE = 3 };

struct Op {
    int kind;
    int cls;                  // CLS_ID, CLS_LINE + p (p <= 3, pure), CLS_PLANE + 3 (p-1) + (q-1) (pure), CLS_GENERIC
    int ra, rb;               // axis roles: ROLE_OUT (< N-2), ROLE_I1 (N-2), ROLE_I2 (N-1), ROLE_NONE
    int a, b;                 // axes (b = -1 for a line op)
    int p, q;                 // degrees on a and b
    int pmask, qmask;         // bit (s + p) set when the rows can be nonzero at offset s
    int tabP, tabQ;           // row table bases
    int dbase;                // base into didx (footprint position -> outer offset index)
    int src, dst;             // input channel (-1 = c), output channel (stage 1 only)
    int mod;                  // hx_mod_kind
    double amp, omega, phase;
    int pw_off, pw_n;         // into the pw value array
    double pw_t0, pw_t1;
};

struct OpSet {
    int nops;
    int ndelta;
    double wAB, wBA;          // factor-order weights for plane ops
    int ndidx;
    Op op[kMaxOps];
    int8_t delta[kMaxDelta][4];       // outer offset: axis0, step0, axis1, step1 (axis -1 = none)
    uint8_t didx[kMaxDidx];
};

struct ApplyArgsBase {
    DevSet S;
    const int4 *items;        // {slab_first, slab_last, e0, e1}
    int nitems;
    int slabs_per_item;
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
    OpSet ops;                // main stage (accumulates y)
    OpSet ops1;               // first stage (writes channels), nops = 0 if unused
    int nch;                  // channel vectors
    void *chan;
    size_t chan_ld;           // elements between channels
    std::vector<int4> items_h;
    int4 *items;
    int nitems;
    int slabs_per_item;
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
int launch_norm(Problem *p, const void *c, int is_c128, double *partials, unsigned *counter, double *result,
                cudaStream_t st);
int apply_grid(const Problem *p);
int apply_launches(const Problem *p);   // kernels per product (1, or 2 with a channel stage)

// Krylov stepping (hx_krylov.cu)
int krylov_step(Problem *p, void *c, double dt, int nsteps);
int krylov_info(Problem *p, int *m_used, double *alpha, double *beta, double *norm);
void *krylov_host_state(Problem *p);
void krylov_free(Problem *p);

}  // namespace hx
