// Device code of the matrix-free product shared by the generic apply kernel (hx_apply.cu) and by the
// kernels that hx_potential_set compiles at run time for one potential's operator structure
// (hx_jit.cu): the launch arguments, operator weights, the per-element view, the specialised
// line and plane stencils and the element loop.  See hx_apply.cu for the method.
#pragma once

#include "hx_types.h"

namespace hx {

template <typename R> struct Vec2;
template <> struct Vec2<float> { using T = float2; };
template <> struct Vec2<double> { using T = double2; };

struct ApplyArgs : ApplyArgsBase {
    OpSet ops;
    int nrow;                  // row-offset table stride
    const void *cin;
    void *cout;
    const double *out_scale;   // nullptr = 1
    void *chan;                // channel vectors (read by the main stage, written by stage 1)
    size_t chan_ld;
    int stage1;                // 1: write each op's result to its channel instead of y
    int skip_diag;             // 1: omit D_K
    // projections h_i = s_i <v_i, y>, i <= dk, computed with the product (kernels compiled per
    // potential only; dvec == nullptr: none; skipped when dk >= *dm_used)
    const void *dvec;          // v_0 (problem dtype); v_i at dvec + i * dld elements
    size_t dld;
    int dk;
    const int *dm_used;
    const double *ds;          // s_i
    double *dh;                // h (re, im per vector)
    double *dpartials;         // gridDim.x x 2 (dk + 1)
    unsigned *dcounter;        // zero; reset by the last block
    // a second product at another time, A(*t_ptr + t_shift2) cin2 into cout2, cin2 == nullptr
    // meaning cin (kernels compiled per potential only; cout2 == nullptr: none)
    void *cout2;
    const void *cin2;
    double t_shift2;
    // with cin2: instead of the two products y, y2 write the 2-stage Magnus combination
    // (cin + cin2)/2 - i mag_g (y - y2) to cout (0: off)
    double mag_g;
};

// Block and grid stages of the reductions: wsum[w][j] (shared, filled by the caller, followed by a
// barrier) holds warp w's sum of value j < nval.  Writes the nval per-block sums to
// partials[blockIdx.x * nval + j].  In the last block to arrive, thread t adds value
// j = t mod nval over the blocks c, c + nc, ... (c = t div nval, nc = blockDim / nval) and the nc
// chunk sums are added in chunk order, so the totals land in tot[0..nval) (shared) in an order
// that does not depend on block timing.  Returns true in every thread of that last block.
// Needs blockDim.x <= 256 and nval <= NMAX.
template <int NMAX>
static __device__ bool reduce_warp_sums(double (*wsum)[NMAX], int nval, double *partials, unsigned *counter,
                                        double *tot)
{
    __shared__ double csum[256];
    __shared__ bool last;
    const int nw = blockDim.x >> 5;
    if ((int)threadIdx.x < nval) {
        double s = 0.0;
        for (int i = 0; i < nw; ++i) s += wsum[i][threadIdx.x];
        partials[blockIdx.x * nval + threadIdx.x] = s;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return false;
    __threadfence();
    const int nc = blockDim.x / nval, j = threadIdx.x % nval, c = threadIdx.x / nval;
    double s = 0.0;
    if (c < nc)
        // L2-coherent loads (the other blocks' partials are visible after their fence and the counter);
        // unlike volatile loads they can all be in flight at once
        for (int blk = c; blk < (int)gridDim.x; blk += nc) s += __ldcg(partials + blk * nval + j);
    csum[threadIdx.x] = s;
    __syncthreads();
    if ((int)threadIdx.x < nval) {
        double t = 0.0;
        for (int i = 0; i < nc; ++i) t += csum[i * nval + threadIdx.x];
        tot[threadIdx.x] = t;
    }
    __syncthreads();
    return true;
}

// The reduction of nval FP64 values per thread (vals[0..nval)): warp sums by FP64 shuffles, then
// reduce_warp_sums.  (Each shuffle round is an FP64 add per value and thread; the kernels that
// reduce many values from FP32 accumulators fill the warp sums themselves.)
constexpr int kRedMax = 2 * (kMaxKrylov + 1);
template <int NMAX = kRedMax>   // nval <= NMAX (sizes the shared warp sums)
static __device__ bool reduce_partials(const double *vals, int nval, double *partials, unsigned *counter, double *tot)
{
    __shared__ double wsum[8][NMAX];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int j = 0; j < nval; ++j) {
        double v = vals[j];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) wsum[wid][j] = v;
    }
    __syncthreads();
    return reduce_warp_sums<NMAX>(wsum, nval, partials, counter, tot);
}

// amp * f(t) in the stencil precision R (the interval index of a piecewise-constant modulation is
// always found in FP64 so that both precisions switch intervals at the same t).
template <typename R>
__device__ __forceinline__ R op_weight(const Op &op, double t, const double *pw)
{
    R f = (R)1;
    switch (op.mod) {
        case MOD_COS: f = cos((R)(op.omega * t + op.phase)); break;
        case MOD_SIN2: { R s = sin((R)(op.omega * t)); f = s * s; } break;
        case MOD_PWCONST: {
            double x = floor((t - op.pw_t0) / (op.pw_t1 - op.pw_t0) * op.pw_n);
            int qi = x < 0.0 ? 0 : (x >= op.pw_n ? op.pw_n - 1 : (int)x);
            f = (R)pw[op.pw_off + qi];
        } break;
        default: break;
    }
    return (R)op.amp * f;
}

// Exact a / b when b divides a, 1 <= b <= a < 2^16: __fdividef is within 2 ulp of a / b, so the
// computed quotient (an integer below 2^16) is off by less than 2^-6 and rounds to itself.
__device__ __forceinline__ int exact_div(int a, int b) { return __float2int_rn(__fdividef((float)a, (float)b)); }

// Error-free sum of two floats (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

template <typename R> struct Acc;
template <> struct Acc<double> {
    double x = 0.0, y = 0.0;
    __device__ void add(double a, double b) { x += a; y += b; }
    __device__ double2 get() const { return make_double2(x, y); }
};
template <> struct Acc<float> {   // compensated accumulation of the operator contributions
    float x = 0.f, y = 0.f, ex = 0.f, ey = 0.f;
    __device__ void add(float a, float b)
    {
        float s, e;
        two_sum(x, a, s, e); x = s; ex += e;
        two_sum(y, b, s, e); y = s; ey += e;
    }
    __device__ float2 get() const { return make_float2(x + ex, y + ey); }
};

// Per-thread view of one output element.
struct Elem {
    int e;                  // rank
    int k2;                 // last coordinate k_{N-1}
    int qall;               // prod_l (1 + k_l)
    int rlen;               // length of the own row
    const int *nb;          // row-offset table at the own row (column d at nb[d * nrow])
    const unsigned short *kr;     // prefix k_0..k_{N-2} of the own row
};

struct Ctx {
    const DevSet *S;
    int nrow;
    __device__ int k(const Elem &el, int l) const { return l == S->N - 1 ? el.k2 : (int)__ldg(el.kr + l); }
    // start rank of the row reached by row offset d (d > 0; the point must lie in K)
    __device__ int row(const Elem &el, int d) const { return __ldg(el.nb + (size_t)d * nrow); }
};

// floor(B / x) for x >= 1 from the table (0 when x > B: no element has those coordinates).
__device__ __forceinline__ int nt_of(const DevSet &S, int x) { return x <= S.B ? __ldg(S.nt + x) : 0; }

// One packed row (4 entries, see the packed row tables): a 16-byte load for FP32, two for FP64.
template <typename R> struct Row4 { R v[4]; };
__device__ __forceinline__ Row4<float> load_row4(const float *p)
{
    const float4 q = __ldg(reinterpret_cast<const float4 *>(p));
    return {{q.x, q.y, q.z, q.w}};
}
__device__ __forceinline__ Row4<double> load_row4(const double *p)
{
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p)), b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    return {{a.x, a.y, b.x, b.y}};
}

// The specialised stencils below issue every load of an operator unconditionally: a footprint
// point outside K reads the row-offset table at its (always valid) slot and gathers the output
// element itself, and gets weight 0.  Without branches around them, all loads of an operator are
// in flight together instead of one dependent pair (table, gather) after another.  This pays for
// degrees <= 3; at degree 8 on short fibres most points lie outside K and the loads they would
// waste cost more than the overlap gains, so those operators keep the branching generic loop.

// Line operator P(X_a), P of pure parity and degree P (offsets -P, -P+2, ..., P), axis role RA,
// applied to NSRC inputs at once (the addresses and weights are shared): sx[s], sy[s] get the sum
// for srcs[s].
template <typename R, int P, int RA, int NSRC>
__device__ __forceinline__ void line_role_n(const Ctx &c, const Elem &el, const OpSet &O, const Op &op, const R *tab,
                                            const typename Vec2<R>::T *const (&srcs)[NSRC], R (&sx)[NSRC],
                                            R (&sy)[NSRC])
{
    using V = typename Vec2<R>::T;
    const DevSet &S = *c.S;
    const int ka = RA == ROLE_LAST ? el.k2 : c.k(el, op.a);
    // steps to the top of the a-fibre (>= 0: the element itself is in K)
    const int top = RA == ROLE_LAST ? el.rlen - 1 - el.k2 : nt_of(S, exact_div(el.qall, 1 + ka)) - 1 - ka;
    const Row4<R> row = load_row4(tab + op.ptabP + (ka * (P + 1) + min(P, top)) * 4);   // entries at s = -P + 2j
    constexpr int NP = P + 1;
    int addr[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        const int s = -P + 2 * j;
        const bool ok = ka + s >= 0 && s <= top;
        int a;
        if (RA == ROLE_LAST) a = el.e + s;
        else a = s == 0 ? el.e : c.row(el, O.didx[op.dbase + s + P]) + el.k2;
        addr[j] = ok ? a : el.e;
    }
    V v[NSRC][NP];
#pragma unroll
    for (int q = 0; q < NSRC; ++q)
#pragma unroll
        for (int j = 0; j < NP; ++j) v[q][j] = srcs[q][addr[j]];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        const int s = -P + 2 * j;
        const R w = (ka + s >= 0 && s <= top) ? row.v[j] : (R)0;
#pragma unroll
        for (int q = 0; q < NSRC; ++q) {
            sx[q] += w * v[q][j].x;
            sy[q] += w * v[q][j].y;
        }
    }
}

template <typename R, int P, int RA>
__device__ __forceinline__ void line_role(const Ctx &c, const Elem &el, const OpSet &O, const Op &op, const R *tab,
                                          const typename Vec2<R>::T *src, R &sx, R &sy)
{
    const typename Vec2<R>::T *srcs[1] = {src};
    R x[1] = {sx}, y[1] = {sy};
    line_role_n<R, P, RA, 1>(c, el, O, op, tab, srcs, x, y);
    sx = x[0];
    sy = y[0];
}

// Plane operator wAB P(X_a) Q(X_b) + wBA Q(X_b) P(X_a), pure parities, degrees P, Q; a is a prefix
// axis, b has role RB.  A footprint point k + s e_a + s2 e_b carries [P]_{k, k+s e_a}
// [Q]_{k+s e_a, k+s e_a+s2 e_b} (path through k + s e_a) and [Q]_{k, k+s2 e_b} [P]_{k+s2 e_b,
// k+s2 e_b+s e_a} (path through k + s2 e_b); a path exists only if its intermediate point is in K.
// Rows of P(J_n / L) and Q(J_n / L) come from the tables, indexed by the coordinate and the
// distance to the fibre top.
// SB > 0: a line operator S(X_b) of degree SB (parity of Q, SB = Q or Q + 2) merged into this op
// (P is even, so the points s = 0 are footprint points); its sum goes to (lx, ly), which the
// caller weights with the line operator's own weight.  NSRC inputs at once (addresses, fibre tops
// and weights shared): the sums for srcs[q] go to sx[q], sy[q], lx[q], ly[q].
template <typename R, int P, int Q, int RB, int SB, int NSRC>
__device__ __forceinline__ void plane_role_n(const Ctx &c, const Elem &el, const OpSet &O, const Op &op, const R *tab,
                                             const typename Vec2<R>::T *const (&srcs)[NSRC], R (&sx)[NSRC],
                                             R (&sy)[NSRC], R (&lx)[NSRC], R (&ly)[NSRC])
{
    using V = typename Vec2<R>::T;
    const DevSet &S = *c.S;
    const int ka = c.k(el, op.a);
    const int kb = RB == ROLE_LAST ? el.k2 : c.k(el, op.b);
    const int rab = exact_div(el.qall, (1 + ka) * (1 + kb));
    const R wAB = (R)O.wAB, wBA = (R)O.wBA;
    const R *tP = tab + op.ptabP, *tQ = tab + op.ptabQ;   // packed rows: entry i at offset -P + 2i
    constexpr int NS = P + 1, NS2 = Q + 1;         // offsets s = -P + 2i, s2 = -Q + 2j
    // a-fibre tops at k + s2 e_b (-1: that point is not in K), b-fibre tops at k + s e_a
    int topA[NS2], topB[NS];
#pragma unroll
    for (int j = 0; j < NS2; ++j) {
        const int s2 = -Q + 2 * j;
        topA[j] = kb + s2 >= 0 ? nt_of(S, rab * (1 + kb + s2)) - 1 - ka : -1;
    }
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        const int s = -P + 2 * i;
        topB[i] = ka + s >= 0 ? nt_of(S, rab * (1 + ka + s)) - 1 - kb : -1;
    }
    // fibre tops at k itself (s = 0 or s2 = 0 need not be footprint offsets)
    const int topA0 = (Q & 1) ? nt_of(S, rab * (1 + kb)) - 1 - ka : topA[Q / 2];
    const int topB0 = RB == ROLE_LAST ? el.rlen - 1 - el.k2 : ((P & 1) ? nt_of(S, rab * (1 + ka)) - 1 - kb : topB[P / 2]);
    const Row4<R> rowP0 = load_row4(tP + (ka * (P + 1) + min(P, topA0)) * 4);   // P row at k
    const Row4<R> rowQ0 = load_row4(tQ + (kb * (Q + 1) + min(Q, topB0)) * 4);   // Q row at k
    // addresses of the footprint points (own element when the point is not in K)
    int addr[NS][NS2];
    const int own = el.e - el.k2;                       // start of the own row
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        const int s = -P + 2 * i;
        int base_s = own;                               // RB = LAST: start of the row of k + s e_a
        if (RB == ROLE_LAST && s != 0) base_s = c.row(el, O.didx[op.dbase + (s + P) * (2 * Q + 1) + Q]);
#pragma unroll
        for (int j = 0; j < NS2; ++j) {
            const int s2 = -Q + 2 * j;
            const bool ok = ka + s >= 0 && kb + s2 >= 0 && s <= topA[j];
            int a;
            if (RB == ROLE_LAST) a = base_s + el.k2 + s2;
            else if (s == 0 && s2 == 0) a = el.e;
            else a = c.row(el, O.didx[op.dbase + (s + P) * (2 * Q + 1) + (s2 + Q)]) + el.k2;
            addr[i][j] = ok ? a : el.e;
        }
    }
    constexpr int NX = SB > Q ? 2 : 0;                  // merged line points +-SB outside the plane footprint
    int xaddr[NX > 0 ? NX : 1];
#pragma unroll
    for (int j = 0; j < NX; ++j) {
        const int s2 = j == 0 ? -SB : SB;
        const bool ok = kb + s2 >= 0 && s2 <= topB0;
        int a;
        if (RB == ROLE_LAST) {
            a = el.e + s2;
        } else {
            const Op &ls = O.op[op.mergeB];
            a = c.row(el, O.didx[ls.dbase + s2 + SB]) + el.k2;
        }
        xaddr[j] = ok ? a : el.e;
    }
    V v[NSRC][NS][NS2];
#pragma unroll
    for (int q = 0; q < NSRC; ++q)
#pragma unroll
        for (int i = 0; i < NS; ++i)
#pragma unroll
            for (int j = 0; j < NS2; ++j) v[q][i][j] = srcs[q][addr[i][j]];
    V xv[NSRC][NX > 0 ? NX : 1];
#pragma unroll
    for (int q = 0; q < NSRC; ++q)
#pragma unroll
        for (int j = 0; j < NX; ++j) xv[q][j] = srcs[q][xaddr[j]];
    // weights
    Row4<R> rowS0 = {};
    if (SB > 0) {
        const Op &ls = O.op[op.mergeB];
        rowS0 = load_row4(tab + ls.ptabP + (kb * (SB + 1) + min(SB, topB0)) * 4);   // entry at s2: (s2 + SB) / 2
    }
    Row4<R> rowPs[NS2];                                 // P rows at k + s2 e_b
#pragma unroll
    for (int j = 0; j < NS2; ++j) rowPs[j] = load_row4(tP + (ka * (P + 1) + max(0, min(P, topA[j]))) * 4);
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        const int s = -P + 2 * i;
        const bool inA = ka + s >= 0 && s <= topA0;             // k + s e_a in K
        const R pj = inA ? rowP0.v[i] : (R)0;
        const Row4<R> rowQs = load_row4(tQ + (kb * (Q + 1) + max(0, min(Q, topB[i]))) * 4);   // Q row at k + s e_a
#pragma unroll
        for (int j = 0; j < NS2; ++j) {
            const int s2 = -Q + 2 * j;
            const bool ok = ka + s >= 0 && kb + s2 >= 0 && s <= topA[j];
            const R cab = inA ? pj * rowQs.v[j] : (R)0;                                   // path via k + s e_a
            const R cba = (kb + s2 >= 0 && s2 <= topB0) ? rowQ0.v[j] * rowPs[j].v[i] : (R)0;   // path via k + s2 e_b
            const R w = ok ? wAB * cab + wBA * cba : (R)0;
#pragma unroll
            for (int q = 0; q < NSRC; ++q) {
                sx[q] += w * v[q][i][j].x;
                sy[q] += w * v[q][i][j].y;
            }
            if (SB > 0 && s == 0) {                     // k + s2 e_b is also a point of the merged line op
                const R ws = ok ? rowS0.v[(s2 + SB) / 2] : (R)0;
#pragma unroll
                for (int q = 0; q < NSRC; ++q) {
                    lx[q] += ws * v[q][i][j].x;
                    ly[q] += ws * v[q][i][j].y;
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < NX; ++j) {
        const int s2 = j == 0 ? -SB : SB;
        const R ws = (kb + s2 >= 0 && s2 <= topB0) ? rowS0.v[(s2 + SB) / 2] : (R)0;
#pragma unroll
        for (int q = 0; q < NSRC; ++q) {
            lx[q] += ws * xv[q][j].x;
            ly[q] += ws * xv[q][j].y;
        }
    }
}

template <typename R, int P, int Q, int RB, int SB>
__device__ __forceinline__ void plane_role(const Ctx &c, const Elem &el, const OpSet &O, const Op &op, const R *tab,
                                           const typename Vec2<R>::T *src, R &sx, R &sy, R &lx, R &ly)
{
    const typename Vec2<R>::T *srcs[1] = {src};
    R x[1] = {sx}, y[1] = {sy}, u[1] = {lx}, w[1] = {ly};
    plane_role_n<R, P, Q, RB, SB, 1>(c, el, O, op, tab, srcs, x, y, u, w);
    sx = x[0];
    sy = y[0];
    lx = u[0];
    ly = w[0];
}


// Warp sums of NV per-lane values (NV a power of two <= 32) by a butterfly reduce-scatter: in
// each of the first log2 NV exchange rounds a lane keeps one half of its values, sends the other
// half to its partner and adds the partner's copy of the kept half; the remaining rounds add up
// the one value left.  Lane l then holds the warp sum of value l >> (5 - log2 NV) (NV - 1 + 5 -
// log2 NV shuffles instead of 5 NV for separate reductions).
template <int NV>
__device__ __forceinline__ float warp_reduce_scatter(float (&v)[NV])
{
    const int lane = threadIdx.x & 31;
    int o = 16;
#pragma unroll
    for (int half = NV / 2; half >= 1; half >>= 1, o >>= 1) {
        const bool hi = (lane & o) != 0;
#pragma unroll
        for (int j = 0; j < half; ++j) {
            const float keep = hi ? v[j + half] : v[j], send = hi ? v[j] : v[j + half];
            v[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    float r = v[0];
#pragma unroll
    for (; o >= 1; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    return r;
}

// log2 of the exchange width for nd projections (2 nd values rounded up to a power of two)
__device__ __forceinline__ int dot_width_log2(int nd) { return nd <= 1 ? 1 : nd <= 2 ? 2 : nd <= 4 ? 3 : 4; }

// Adds this element's conj(v_i) y, i < nd, to the lane's compensated sum (hs, hc) of the warp
// sums of value lane >> (5 - log2 NV).
template <int NV>
__device__ __forceinline__ void add_projections(const ApplyArgs &args, int nd, int e, bool valid, float2 y, float &hs,
                                                float &hc)
{
    const float2 *dv = (const float2 *)args.dvec;
    float v[NV];
#pragma unroll
    for (int i = 0; i < NV / 2; ++i) {
        float2 x = make_float2(0.f, 0.f);
        if (i < nd && valid) x = dv[(size_t)i * args.dld + e];
        v[2 * i] = fmaf(x.x, y.x, x.y * y.y);        // Re conj(v_i) y
        v[2 * i + 1] = fmaf(x.x, y.y, -x.y * y.x);   // Im conj(v_i) y
    }
    const float r = warp_reduce_scatter<NV>(v);
    const float t = hs + r, bb = t - hs;            // TwoSum
    hc += (hs - (t - bb)) + (r - bb);
    hs = t;
}

// The per-thread view of element e from its record er = {row, prod (1 + k_l), sum k_l,
// k_{N-1} | row length << 16}.
__device__ __forceinline__ Elem make_elem(const ApplyArgs &args, int e, int4 er)
{
    Elem el;
    el.e = e;
    el.k2 = er.w & 0xffff;
    el.qall = er.y;
    el.rlen = (int)((unsigned)er.w >> 16);
    el.nb = args.rnb + er.x;
    el.kr = args.S.row_k + (size_t)er.x * (args.S.N - 1);
    return el;
}

// One element: D_K on the diagonal, body(ctx, el, acc, sm_w, cin, tab) adds the operators'
// contributions, and y = out_scale * acc is written unless the launch only writes channel vectors
// (stage 1); returns y.
template <typename R, typename Body>
__device__ __forceinline__ typename Vec2<R>::T apply_element(const ApplyArgs &args, const Ctx &ctx, int e, int4 er,
                                                             R oscale, const R *sm_w, Body &body)
{
    using V = typename Vec2<R>::T;
    const DevSet &S = args.S;
    const V *cin = (const V *)args.cin;
    const Elem el = make_elem(args, e, er);
    Acc<R> acc;
    if (!args.stage1 && !args.skip_diag) {
        const V ce = cin[e];
        const R dj = (R)er.z + (R)0.5 * (R)S.N;   // (D_K)_jj = sum_l (j_l + 1/2)
        acc.add(dj * ce.x, dj * ce.y);
    }
    body(ctx, el, acc, sm_w, cin, (const R *)args.tab);
    V y = acc.get();
    if (!args.stage1) {
        y.x *= oscale;
        y.y *= oscale;
        ((V *)args.cout)[e] = y;
    }
    return y;
}

// The element loop: one thread per output element (grid-stride).  With DOTS (complex64 only) the
// launch also computes the projections h_i = s_i <v_i, y>, i <= dk, of the launch arguments from
// the stored y: per element the products conj(v_i) y go through warp_reduce_scatter, each lane
// adds its warp sum to one compensated FP32 sum (TwoSum), and the sums are reduced over the grid
// at the end.  The loop then runs warp-uniformly (whole warps per trip) so that every lane takes
// part in the exchanges.
template <typename R, bool DOTS = false, typename Body>
__device__ __forceinline__ void apply_elements(const ApplyArgs &args, Body body)
{
    __shared__ R sm_w[kMaxOps];
    const DevSet &S = args.S;
    const OpSet &O = args.ops;
    if ((int)threadIdx.x < O.nops) sm_w[threadIdx.x] = op_weight<R>(O.op[threadIdx.x], *args.t_ptr + args.t_shift, args.pw_values);
    const R oscale = args.out_scale ? (R)(*args.out_scale) : (R)1;
    __syncthreads();
    Ctx ctx;
    ctx.S = &S;
    ctx.nrow = args.nrow;
    const int stride = gridDim.x * blockDim.x;
    if constexpr (!DOTS) {
        for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < S.size; e += stride)
            apply_element<R>(args, ctx, e, __ldg(S.elem + e), oscale, sm_w, body);
    } else {
        // the element records stream from DRAM: each trip loads the next trip's record before it
        // works on its own, so that the load's latency overlaps a whole element's stencil (measured
        // faster in this loop and slower in the plain loop above)
        auto record = [&](int e) { return e < S.size ? __ldg(S.elem + e) : make_int4(0, 0, 0, 0); };
        static_assert(sizeof(R) == 4, "fused projections are implemented for complex64 vectors");
        const int nd = args.dvec && !args.stage1 && args.dk < *args.dm_used ? args.dk + 1 : 0;
        const int lane = threadIdx.x & 31;
        const int wl = dot_width_log2(nd);
        float hs = 0.f, hc = 0.f;              // this lane's TwoSum of value lane >> (5 - wl)
        int4 er = record(blockIdx.x * blockDim.x + threadIdx.x);
        for (int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < S.size; base += stride) {
            const int e = base + lane;
            const int4 next = record(e + stride);
            float2 y = make_float2(0.f, 0.f);
            if (e < S.size) y = apply_element<R>(args, ctx, e, er, oscale, sm_w, body);
            er = next;
            if (nd) {
                const bool valid = e < S.size;
                if (wl == 4) add_projections<16>(args, nd, e, valid, y, hs, hc);
                else if (wl == 3) add_projections<8>(args, nd, e, valid, y, hs, hc);
                else if (wl == 2) add_projections<4>(args, nd, e, valid, y, hs, hc);
                else add_projections<2>(args, nd, e, valid, y, hs, hc);
            }
        }
        if (nd) {
            // the lanes already hold warp sums (lane l: value l >> (5 - wl)): one write per value and warp
            __shared__ double wsum[8][2 * kMaxFusedDots];
            const int sh = 5 - wl, j = lane >> sh;
            if ((lane & ((1 << sh) - 1)) == 0 && j < 2 * nd) wsum[threadIdx.x >> 5][j] = (double)hs + (double)hc;
            __syncthreads();
            __shared__ double tot[2 * kMaxFusedDots];
            if (reduce_warp_sums<2 * kMaxFusedDots>(wsum, 2 * nd, args.dpartials, args.dcounter, tot) && threadIdx.x == 0) {
                for (int i = 0; i < nd; ++i) {
                    args.dh[2 * i] = args.ds[i] * tot[2 * i];
                    args.dh[2 * i + 1] = args.ds[i] * tot[2 * i + 1];
                }
                *args.dcounter = 0;
            }
        }
    }
}

// Two products in one pass: y = A(*t_ptr + t_shift) c into cout and y2 = A(*t_ptr + t_shift2) c2
// into cout2, c2 = c unless cin2 is given (the products of the 2-stage Magnus method).  The stencil
// coefficients do not depend on the time, only the operator weights do, so all index work and the
// weights are shared, and for c2 = c every gather too; body(ctx, el, acc, acc2, sm_w, sm_w2, cin,
// cin2, tab) adds each operator's sum with its weight at either time.
template <typename R, typename Body>
__device__ __forceinline__ void apply_elements_dual(const ApplyArgs &args, Body body)
{
    using V = typename Vec2<R>::T;
    __shared__ R sm_w[kMaxOps], sm_w2[kMaxOps];
    const DevSet &S = args.S;
    const OpSet &O = args.ops;
    if ((int)threadIdx.x < O.nops) {
        sm_w[threadIdx.x] = op_weight<R>(O.op[threadIdx.x], *args.t_ptr + args.t_shift, args.pw_values);
        sm_w2[threadIdx.x] = op_weight<R>(O.op[threadIdx.x], *args.t_ptr + args.t_shift2, args.pw_values);
    }
    const R oscale = args.out_scale ? (R)(*args.out_scale) : (R)1;
    __syncthreads();
    Ctx ctx;
    ctx.S = &S;
    ctx.nrow = args.nrow;
    const V *cin = (const V *)args.cin;
    const V *cin2 = args.cin2 ? (const V *)args.cin2 : cin;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < S.size; e += gridDim.x * blockDim.x) {
        const int4 er = __ldg(S.elem + e);
        const Elem el = make_elem(args, e, er);
        Acc<R> acc, acc2;
        if (!args.skip_diag) {
            const V ce = cin[e], ce2 = cin2[e];
            const R dj = (R)er.z + (R)0.5 * (R)S.N;
            acc.add(dj * ce.x, dj * ce.y);
            acc2.add(dj * ce2.x, dj * ce2.y);
        }
        body(ctx, el, acc, acc2, (const R *)sm_w, (const R *)sm_w2, cin, cin2, (const R *)args.tab);
        V y = acc.get(), y2 = acc2.get();
        y.x *= oscale;
        y.y *= oscale;
        y2.x *= oscale;
        y2.y *= oscale;
        if (args.mag_g != 0.0) {
            const V a = cin[e], b = cin2[e];
            const R g = (R)args.mag_g, half = (R)0.5;
            V r;
            r.x = half * (a.x + b.x) + g * (y.y - y2.y);        // -i g z = g (z.y, -z.x)
            r.y = half * (a.y + b.y) - g * (y.x - y2.x);
            ((V *)args.cout)[e] = r;
        } else {
            ((V *)args.cout)[e] = y;
            ((V *)args.cout2)[e] = y2;
        }
    }
}

}  // namespace hx
