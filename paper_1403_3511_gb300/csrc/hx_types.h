// Device-side types and constants of libhx shared by the CUDA sources and by the kernels that
// hx_potential_set compiles at run time for one potential's operator structure.  Plain C++ with
// CUDA vector types only (no standard-library headers), so that the run-time compiler can read it.
#pragma once

namespace hx {

constexpr int kMaxN = 16;
constexpr int kMaxOps = 48;
constexpr int kMaxDelta = 255;                 // distinct row offsets of one problem (both stages)
constexpr int kMaxDidx = 4096;                 // footprint -> offset map entries of one operator set
constexpr int kMaxDeg = 8;                     // HX_MAX_DEG
constexpr int kSpan = 2 * kMaxDeg + 1;         // offsets -deg..deg
constexpr int kMaxKrylov = 32;
constexpr int kApplyThreads = 256;
constexpr int kNtSpan = 16;          // the floor(B / x) table covers x <= kNtSpan B (products of shifted points)
constexpr int kTopWords = 4;        // 32-bit words of precomputed fibre tops per element (at most)
constexpr int kMaxFusedDots = 8;     // projections one product launch can compute (Krylov steps m <= 8)

// time modulations (values of hx_mod_kind)
enum { MOD_CONST = 0, MOD_COS = 1, MOD_SIN2 = 2, MOD_PWCONST = 3 };

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
// A group is the set of rows sharing k_0, ..., k_{N-3} (one group when N <= 2); its rows are
// consecutive, row k_{N-2} of the group being row gfirst[g] + k_{N-2}.  The row index of a prefix is
//   row(p) = sum_{d<N-2} Q_{N-2-d}(q_d, p_d) + p_{N-2}
// (the same tables one level up: Q_m counts the rows below a subtree as |K_m|).
// ---------------------------------------------------------------------------------------
struct DevSet {
    int N, B, size, nrow, qtotal, ngroup;
    int general;                      // 1: a general downward-closed set (membership from the tables)
    const int4 *row_info;             // nrow: {start rank, q(p), sum_l p_l, length}
    const unsigned short *row_k;            // nrow x (N - 1) prefixes
    const int4 *elem;                 // size: per element {row, group, prod_l (1 + k_l) | sum_l k_l << 16,
                                      //                    k_{N-1} | row length << 16}
    const int *rstart;                // nrow + 1: start rank of each row, rstart[nrow] = size
    const int *rgrp;                  // nrow: group of each row
    const int *gfirst;                // ngroup + 1: first row of each group, gfirst[ngroup] = nrow
    const int *qoff;                  // B + 2
    const int *Q;                     // (N - 1) x qtotal
    const int *nt;                    // nt[x] = floor(B / x) for 0 < x <= kNtSpan B, nt[0] = 0
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
// Packed row tables (a polynomial of pure parity and degree p <= 8, whose row has p + 1 entries
// that can be nonzero, at s = -p, -p + 2, ..., p), W = packed_width(p) = 4 ceil((p + 1) / 4) entries
// per row:
//   tab[pbase + (i * (p + 1) + d) * W + j] = [P(J_n / L)]_{i, i-p+2j},  j <= p, zero for j > p,
// W / 4 16-byte loads (FP32) or W / 2 (FP64) per row.
// ---------------------------------------------------------------------------------------
__host__ __device__ constexpr int packed_width(int p) { return 4 * ((p + 4) / 4); }

// op classes with compile-time stencils (pure parity: P has only terms of the parity of its degree)
enum { CLS_ID = 0, CLS_LINE = 1, CLS_PLANE = 10, CLS_GENERIC = 30 };
// axis roles: an axis of the row prefix (moving along it changes the row) or the last axis
enum { ROLE_ROW = 0, ROLE_LAST = 1, ROLE_NONE = 2 };

struct Op {
    int kind;
    int cls;                  // CLS_ID, CLS_LINE + p (p <= 8), CLS_PLANE + 3 (p-1) + (q-1) (p, q <= 3), CLS_GENERIC (pure parity)
    int ra, rb;               // axis roles: ROLE_ROW (< N-1), ROLE_LAST (N-1), ROLE_NONE
    int a, b;                 // axes (b = -1 for a line op)
    int p, q;                 // degrees on a and b
    int pmask, qmask;         // bit (s + p) set when the rows can be nonzero at offset s
    int tabP, tabQ;           // row table bases
    int ptabP, ptabQ;         // packed row table bases (pure parity, line degree <= 8, plane degrees <= 3; 0 otherwise);
                              // a plane operator's degree-1 second factor has its two rows per coordinate side by side
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
    float wAB32, wBA32;       // the same in FP32 (read by the FP32 kernels)
    int ndidx;
    Op op[kMaxOps];
    unsigned char didx[kMaxDidx];   // footprint position -> column of the row-offset table
};

// Row offsets used by a problem's operators: axis0, step0, axis1, step1 (axis -1 = none), over
// the prefix axes 0..N-2; offset 0 is the zero offset.  Each offset is split into its move on the
// group axes 0..N-3 (an "outer move", om >= 0, or none, om = -1) and its step s4 on axis N-2.  The
// group-neighbour table holds, for group g and outer move om, the first row of the group reached,
// or -1 when that group is not in K:  gnb[g * gstride + om].  The row of a prefix p moved by
// offset d is then gnb[g(p) * gstride + om(d)] + p_{N-2} + s4(d) (om(d) >= 0) or row(p) + s4(d).
struct RowMove {
    short om;                 // outer move (-1: none)
    short s4;                 // step on axis N-2
};

struct RowOffsets {
    int n;
    signed char d[kMaxDelta][4];
    RowMove mv[kMaxDelta];    // decomposition of each offset
    int nom;                  // outer moves
    signed char om[kMaxDelta][4];   // axis0, step0, axis1, step1 of each outer move (axes < N-2)
};

// Work queue of a batched product launch (device memory, zero before the first launch): the next
// tile, the blocks that have left (the last resets both), and a flag set by a block whose clock64
// budget ran out.
struct BatchQueue {
    unsigned next;
    unsigned done;
    int timeout;
    int pad;
};

struct ApplyArgsBase {
    DevSet S;
    const int *gnb;           // group-neighbour table, ngroup x gstride
    const int *gnbn;          // general sets: rows of each neighbour group (0: none), same layout
    int gstride;
    double dscale;            // S^2: factor of D_K for the basis phi_k(S x)
    float dscale32;           // the same in FP32 (read by the FP32 kernels)
    const double *t_ptr;      // device time
    double t_shift;           // A is evaluated at *t_ptr + t_shift
    const double *pw_values;  // device
    const void *tab;          // row tables (float or double)
    RowMove mv[kMaxDelta];    // per row-offset column: outer move and step on axis N-2
    // kernels compiled per potential: each element's fibre-top distances packed in tops_words
    // 32-bit words, word w of element e at tops[w * S.size + e] (tops_words = 0: none); tops_out:
    // where the kernel that packs them writes
    const unsigned *tops;
    int tops_words;
    unsigned *tops_out;
};

}  // namespace hx
