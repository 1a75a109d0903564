// Internal declarations of libhx (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/hx.h"
#include "hx_types.h"

namespace hx {

static_assert(kMaxDeg == HX_MAX_DEG, "hx_types.h and hx.h disagree on the maximal degree");
static_assert((int)MOD_COS == (int)HX_MOD_COS && (int)MOD_SIN2 == (int)HX_MOD_SIN2 &&
                  (int)MOD_PWCONST == (int)HX_MOD_PWCONST,
              "hx_types.h and hx.h disagree on the modulation kinds");

void set_error(const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);

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
    int ngroup;
    std::vector<int> rgrp;            // nrow: group of each row (rows sharing k_0..k_{N-3})
    std::vector<int> gfirst;          // ngroup: first row of each group
    // a general downward-closed set (hx_indexset_create_list): B is 1 + the largest coordinate,
    // and ranks come from the sorted list instead of the rank tables
    bool general = false;
    std::vector<int32_t> list;        // size x N, lexicographic order
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
    // projections h_i = s_i <v_i, y> (i <= dk, skipped when dk >= *m_used) computed by the product
    // launch itself; only when apply_fuses_dots(p) (dvec == nullptr: none)
    const void *dvec;         // v_0 in the problem dtype; v_i at dvec + i * dld elements
    size_t dld;
    int dk;                   // < kMaxFusedDots
    const int *m_used;
    const double *s;          // s_i
    double *h;                // 2 (dk + 1) doubles: h_i (re, im)
    double *partials;         // apply_grid(p) x 2 (dk + 1) doubles
    unsigned *counter;        // zero-initialised; reset by the last block
    // rq: instead of the projections, s[0] <c_in, y> (the input's Rayleigh quotient) into h[0..1]
    // (partials: apply_grid(p) x 2 doubles); only when apply_fuses_dots(p)
    bool rq;
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
    void *jit;                // kernel compiled for the operator structure (hx_jit.cu), or null
    std::string jit_reason;   // why jit is (or is not) set
    RowOffsets roff;          // row offsets of ops and ops1 (and their outer moves)
    int *gnb;                 // group-neighbour table (device), ngroup x gstride
    int *gnbn;                // general sets: rows of each neighbour group (0: none), same layout
    // the specialised kernel's fibre-top fields per element (jit_fill_tops), and the kernel they were
    // packed for
    unsigned *tops;
    size_t tops_bytes;
    const void *tops_src;
    int gstride;
    double scale;             // basis scaling S (phi_k(S x)); D_K is multiplied by S^2
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
    void *proj_ws = nullptr;     // hx_apply_project scalars and partial sums (one of extra)
};

// launchers (hx_apply.cu)
int launch_apply(Problem *p, const void *cin, void *cout, const double *t_ptr, double t_shift,
                 const ApplyFuse *fuse, cudaStream_t st);
int launch_export(const IndexSetObj *s, int32_t *k_dev, cudaStream_t st);
int launch_elem_info(const IndexSetObj *s);
int launch_groupnb(const DevSet &S, const RowOffsets &ro, int gstride, int *gnb, cudaStream_t st);
int launch_norm(Problem *p, const void *c, int is_c128, double *partials, unsigned *counter, double *result,
                cudaStream_t st);
int apply_grid(const Problem *p);
int apply_launches(const Problem *p);     // kernels per product (1, or 2 with a channel stage)
bool apply_fuses_dots(const Problem *p);  // the product kernel can compute ApplyFuse projections
bool apply_dual(const Problem *p);        // one launch can give the products at two times
// cout = A(t + t_shift) cin and cout2 = A(t + t_shift2) cin, in one launch when apply_dual(p)
int launch_apply_dual(Problem *p, const void *cin, void *cout, void *cout2, const double *t_ptr, double t_shift,
                      double t_shift2, const ApplyFuse *fuse, cudaStream_t st);
// cout = A(t + t_shift) cin and cout2 = A(t + t_shift2) cin2, in one launch when apply_dual(p);
// then, with mag_out, that launch writes only (cin + cin2)/2 - i mag_g (cout - cout2) to mag_out
// (the 2-stage Magnus combination) and apply_dual(p) tells the caller it did
int launch_apply_pair(Problem *p, const void *cin, void *cout, double t_shift, const void *cin2, void *cout2,
                      double t_shift2, const double *t_ptr, cudaStream_t st, void *mag_out = nullptr,
                      double mag_g = 0.0);

// batched products (hx_apply.cu): launch arguments of one member's Lanczos product, their size, and
// one persistent launch over the tiles of all members of one precision and degree class
int batch_member_args(Problem *p, const void *cin, void *cout, const double *t_ptr, double t_shift,
                      const double *in_scale, void *out);
size_t apply_args_size();
int launch_batch_apply(bool c64, int md, const void *margs, const int2 *tiles, int ntiles, int tile, long long budget,
                       void *queue, int num_sms, cudaStream_t st);
int max_degree(const Problem *p);

// hx_apply_project after the argument checks (hx_krylov.cu)
int apply_project_dispatch(Problem *p, const void *c, void *y, const void *basis, size_t ld, int k, double *h);
int apply_rayleigh_dispatch(Problem *p, const void *c, void *y, double *r);

extern thread_local bool g_batch_capture;   // hx_krylov.cu: a batch graph is being captured

// kernels compiled at run time for one potential's operator structure (hx_jit.cu)
void jit_prepare(Problem *p);
int jit_launch(const Problem *p, const void *args, int blocks, cudaStream_t st);
bool jit_has_stage1(const Problem *p);   // the compiled kernels include the first (channel) stage
int jit_tops_words(const Problem *p);   // 32-bit words of fibre-top fields the compiled kernels read
int jit_fill_tops(Problem *p);          // after jit_prepare: packs those fields for the problem's set

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
constexpr int kSchedMembers = 0, kSchedBatched = 1, kSchedHybrid = 2, kSchedSerial = 3, kNumSched = 4;
struct Batch {
    std::vector<Problem *> probs;
    std::vector<void *> cptr;
    std::vector<int> gen;     // member generations the graphs were captured with
    double dt = 0.0;
    cudaStream_t stream = nullptr;
    // schedules (kSched*): one graph each among the candidates, the fastest step kept
    std::vector<int> cand;               // candidate schedules of the captured graphs
    cudaGraphExec_t exec[kNumSched] = {};
    int kern[kNumSched] = {};            // kernel launches of one replay of each graph
    float sched_ms[kNumSched] = {-1.f, -1.f, -1.f, -1.f};   // one timed step of each candidate
    int schedule = -1;                   // the chosen one (-1 while candidates are timed)
    int tile = 0;             // elements per tile of the batched launches (autotuned at first use)
    long long budget = -1;    // clock64 budget of each block of a batched product (< 0: none)
    double budget_s = -1.0;
    std::vector<double> tune_ms;   // tile autotuner: product time per candidate tile size
    std::vector<int> tune_tiles;
    void *dmem[kNumSched] = {};    // device: launch arguments, tile lists and queues per schedule
    size_t dmem_bytes[kNumSched] = {};
    cudaStream_t cap = nullptr;    // capture stream of the batched graphs
    std::vector<cudaEvent_t> ev;   // fork/join events (one per member, one for the fork)
};
int batch_step(Batch *b, void *const *c, double dt, int nsteps);
int batch_timed_out(Batch *b);     // 1 when a batched product's budget ran out since the last call
void batch_free(Batch *b);
void batch_drop_graphs(Batch *b);

// Krylov stepping (hx_krylov.cu)
int krylov_step(Problem *p, void *c, double dt, int nsteps);
int krylov_info(Problem *p, int *m_used, double *alpha, double *beta, double *norm);
int krylov_substeps(Problem *p, int *last, long long *total, double *err_max);

// binds the allocation-free norm's scratch on device dev (hx_noalloc.cu)
int noalloc_bind(int dev);
void *krylov_host_state(Problem *p);
void krylov_free(Problem *p);
void krylov_invalidate(Problem *p);   // drops the captured step graph, keeps the workspace

}  // namespace hx
