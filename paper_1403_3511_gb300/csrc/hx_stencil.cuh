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
    // drq = 1: instead, the one projection ds[0] <cin, y> of the input (the Rayleigh quotient of a
    // Lanczos step) into dh[0..1], with dpartials (gridDim.x x 2) and dcounter (kernels compiled per
    // potential only)
    int drq;
    // a second product at another time, A(*t_ptr + t_shift2) cin2 into cout2, cin2 == nullptr
    // meaning cin (kernels compiled per potential only; cout2 == nullptr: none)
    void *cout2;
    const void *cin2;
    double t_shift2;
    // with cin2: instead of the two products y, y2 write the 2-stage Magnus combination
    // (cin + cin2)/2 - i mag_g (y - y2) to cout (0: off)
    double mag_g;
    float mag_g32;             // mag_g in FP32 (read by the FP32 kernels)
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

// Packed pairs of FP32 values: one instruction applies the IEEE round-to-nearest operation to both
// halves (the complex64 re/im pair), so a complex-times-real multiply-add or a complex TwoSum step
// costs one instruction instead of two.
union F2Bits {
    float2 f;
    unsigned long long u;
};
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c)
{
    F2Bits x, y, z, r;
    x.f = a;
    y.f = b;
    z.f = c;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.u) : "l"(x.u), "l"(y.u), "l"(z.u));
    return r.f;
}
__device__ __forceinline__ float2 f2_add(float2 a, float2 b)
{
    F2Bits x, y, r;
    x.f = a;
    y.f = b;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.u) : "l"(x.u), "l"(y.u));
    return r.f;
}
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b)
{
    F2Bits x, y, r;
    x.f = a;
    y.f = b;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.u) : "l"(x.u), "l"(y.u));
    return r.f;
}
__device__ __forceinline__ float2 f2_mul(float2 a, float2 b)
{
    F2Bits x, y, r;
    x.f = a;
    y.f = b;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.u) : "l"(x.u), "l"(y.u));
    return r.f;
}

// acc + w v for a complex v and a real weight w
__device__ __forceinline__ float2 cmad(float w, float2 v, float2 acc) { return f2_fma(make_float2(w, w), v, acc); }
__device__ __forceinline__ double2 cmad(double w, double2 v, double2 acc)
{
    return make_double2(fma(w, v.x, acc.x), fma(w, v.y, acc.y));
}
__device__ __forceinline__ float2 cscale(float w, float2 v) { return f2_mul(make_float2(w, w), v); }
__device__ __forceinline__ double2 cscale(double w, double2 v) { return make_double2(w * v.x, w * v.y); }
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return f2_add(a, b); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

// A launch constant in the stencil precision: the FP32 kernels read the FP32 copy the host stores
// beside the FP64 field (a conversion of the FP64 field, which the compiler may repeat at every use
// under register pressure, runs on the FP64 pipe, a small fraction of the FP32 rate on GB300).
template <typename R>
__device__ __forceinline__ R rconst(double d, float f)
{
    if constexpr (sizeof(R) == 4) return f;
    else return (R)d;
}
template <typename V> __device__ __forceinline__ V czero();
template <> __device__ __forceinline__ float2 czero<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }

template <typename R> struct Acc;
template <> struct Acc<double> {
    double2 s = {0.0, 0.0};
    __device__ void add(double2 a) { s.x += a.x; s.y += a.y; }
    __device__ void add(double a, double b) { s.x += a; s.y += b; }
    __device__ double2 get() const { return s; }
};
template <> struct Acc<float> {   // compensated accumulation of the operator contributions
    float2 s = {0.f, 0.f}, e = {0.f, 0.f};
    // TwoSum on both halves at once: s + err == s_old + a exactly, err summed separately
    __device__ void add(float2 a)
    {
        const float2 t = f2_add(s, a), bb = f2_sub(t, s);
        const float2 err = f2_add(f2_sub(s, f2_sub(t, bb)), f2_sub(a, bb));
        s = t;
        e = f2_add(e, err);
    }
    __device__ void add(float a, float b) { add(make_float2(a, b)); }
    __device__ float2 get() const { return f2_add(s, e); }
};

// Per-thread view of one output element.
struct Elem {
    int e;                  // rank
    int j;                  // last coordinate k_{N-1}
    int qall;               // prod_l (1 + k_l)
    int ksum;               // sum_l k_l
    int rlen;               // length of the own row
    int r;                  // own row
    int k4;                 // k_{N-2} (0 for N = 1)
    const unsigned short *kr;     // prefix k_0..k_{N-2} of the own row
    const int *gn;                // group-neighbour table row of the own group
    // general sets only: rows of the own group, and the row counts of the neighbour groups
    int grows;
    const int *gnn;
    unsigned tw[kTopWords];       // precomputed fibre-top distances (kernels compiled per potential)
};

// Field of width w at bit off of an element's top words (off and w compile-time after unrolling),
// and the packing counterpart.
__device__ __forceinline__ int top_field(const Elem &el, int off, int w)
{
    return (int)((el.tw[off >> 5] >> (off & 31)) & ((1u << w) - 1u));
}
__device__ __forceinline__ void put_top_field(unsigned *tw, int off, int x) { tw[off >> 5] |= (unsigned)x << (off & 31); }

struct Ctx {
    const DevSet *S;
    const RowMove *mv;
    __device__ int k(const Elem &el, int l) const
    {
        return l == S->N - 1 ? el.j : (l == S->N - 2 ? el.k4 : (int)__ldg(el.kr + l));
    }
    // Start rank of the row reached from the own row by the row move (om, s4) when ok (the point
    // lies in K, so that row exists); the start of the own row otherwise.
    __device__ __forceinline__ int start_mv(const Elem &el, int om, int s4, bool ok) const
    {
        int st = el.e - el.j;
        if (ok) {   // a predicated pair of loads: lanes whose point lies outside K read nothing
            const int row = om >= 0 ? __ldg(el.gn + om) + el.k4 + s4 : el.r + s4;
            st = __ldg(S->rstart + row);
        }
        return st;
    }
    // the same for a row already known (the group-neighbour entry read by the caller)
    __device__ __forceinline__ int start_row(const Elem &el, int row, bool ok) const
    {
        int st = el.e - el.j;
        if (ok) st = __ldg(S->rstart + row);
        return st;
    }
    // the same for row-offset column d
    __device__ __forceinline__ int start(const Elem &el, int d, bool ok) const
    {
        const RowMove m = mv[d];
        return start_mv(el, m.om, m.s4, ok);
    }
    // General sets (no product test): whether the point reached by row-offset column d and a shift
    // sh of the last coordinate lies in K, and the start rank of its row (the own row's when not).
    // The row exists when its group does and its coordinate k_{N-2} is below the group's row
    // count; the point, when its last coordinate is below that row's length.
    __device__ __forceinline__ bool member(const Elem &el, int d, int sh, int &start) const
    {
        const RowMove m = mv[d];
        const int i4 = el.k4 + m.s4;
        int rows = el.grows, row = el.r + m.s4;
        if (m.om >= 0) {
            rows = __ldg(el.gnn + m.om);
            row = __ldg(el.gn + m.om) + i4;
        }
        bool ok = i4 >= 0 && i4 < rows;
        row = ok ? row : el.r;
        const int st = __ldg(S->rstart + row), len = __ldg(S->rstart + row + 1) - st;
        const int jj = el.j + sh;
        ok = ok && jj >= 0 && jj < len;
        start = ok ? st : el.e - el.j;
        return ok;
    }
};

// Coordinate k_l of the element on axis l: l compile-time (CM::kA, CM::kB >= 0 with N = CM::kN, the
// kernels compiled per potential: equal reads of two operators are one load) or read from the
// operator at run time.
template <int L, int N>
__device__ __forceinline__ int coord_ct(const Elem &el)
{
    return L == N - 1 ? el.j : (L == N - 2 ? el.k4 : (int)__ldg(el.kr + L));
}
template <typename CM>
__device__ __forceinline__ int coord_a(const Ctx &c, const Elem &el, const Op &op)
{
    if constexpr (CM::kA >= 0) return coord_ct<CM::kA, CM::kN>(el);
    else return c.k(el, op.a);
}
template <typename CM>
__device__ __forceinline__ int coord_b(const Ctx &c, const Elem &el, const Op &op)
{
    if constexpr (CM::kB >= 0) return coord_ct<CM::kB, CM::kN>(el);
    else return c.k(el, op.b);
}

// Row moves of an operator's footprint points, read at run time from the operator list (the
// generic kernel); the kernels compiled per potential use generated types with the same two
// functions whose moves are compile-time constants.  pos: footprint position of the point
// ((s + p) (2 q + 1) + (s2 + q)); startx: the merged line op's points s2 = -SB, SB.
struct ColsRuntime {
    static constexpr bool kTopsBits = false;     // fibre tops computed in the kernel
    static constexpr int kA = -1, kB = -1, kN = 0;   // the operator's axes and N read at run time
    struct Gn {};                                // group-neighbour entries read per point
    __device__ static __forceinline__ Gn gn_load(const Elem &) { return {}; }
    __device__ static __forceinline__ int start(const Ctx &c, const Elem &el, const OpSet &O, const Op &op, const Gn &,
                                                int pos, bool ok)
    {
        return c.start(el, O.didx[op.dbase + pos], ok);
    }
    __device__ static __forceinline__ int startx(const Ctx &c, const Elem &el, const OpSet &O, const Op &op, const Gn &,
                                                 int j, int sb, bool ok)
    {
        const Op &ls = O.op[op.mergeB];
        return c.start(el, O.didx[ls.dbase + (j == 0 ? 0 : 2 * sb)], ok);
    }
};

// floor(B / x) for x >= 1 from the table (0 when x > B: no element has those coordinates).
__device__ __forceinline__ int nt_of(const DevSet &S, int x) { return x <= S.B ? __ldg(S.nt + x) : 0; }

// One packed row (4 entries, see the packed row tables): a 16-byte load for FP32, two for FP64.
template <typename R> struct Row4 { R v[4]; };
// A packed row of W entries (a multiple of 4): W / 4 16-byte loads for FP32, W / 2 for FP64.
template <typename R, int W> struct RowW { R v[W]; };
template <int W> __device__ __forceinline__ RowW<float, W> load_roww(const float *p)
{
    RowW<float, W> r;
#pragma unroll
    for (int i = 0; i < W / 4; ++i) {
        const float4 q = __ldg(reinterpret_cast<const float4 *>(p) + i);
        r.v[4 * i] = q.x;
        r.v[4 * i + 1] = q.y;
        r.v[4 * i + 2] = q.z;
        r.v[4 * i + 3] = q.w;
    }
    return r;
}
template <int W> __device__ __forceinline__ RowW<double, W> load_roww(const double *p)
{
    RowW<double, W> r;
#pragma unroll
    for (int i = 0; i < W / 2; ++i) {
        const double2 q = __ldg(reinterpret_cast<const double2 *>(p) + i);
        r.v[2 * i] = q.x;
        r.v[2 * i + 1] = q.y;
    }
    return r;
}
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

// The specialised stencils below issue the loads of an operator without branches: every footprint
// point's row start and gather are predicated on its membership in K (a lane whose point lies
// outside K reads nothing and contributes zero; the tabulated rows of P(J_n / L) are zero at the
// columns outside the fibre as well), so all loads of an operator are in flight together instead
// of one dependent pair (table, gather) after another.  This pays for degrees <= 3; at degree 8 on
// short fibres most points lie outside K, so those operators keep the branching generic loop.
//
// Membership and fibre tops come from integer products only: with r = prod over the other axes
// of (1 + k_l), the point k + u e_a + v e_b lies in K iff its coordinates are >= 0 and
// r (1 + k_a + u)(1 + k_b + v) <= B (no overflow: the product is at most 16 B for |u|, |v| <= 3).

// Steps from k to the top of its fibre along a prefix axis with coordinate ka, capped at P.
template <int P>
__device__ __forceinline__ int line_top(const Ctx &c, const Elem &el, int ka)
{
    const int other = exact_div(el.qall, 1 + ka), slack = c.S->B - el.qall;
    int top = 0;
#pragma unroll
    for (int t = 1; t <= P; ++t) top += other * t <= slack ? 1 : 0;
    return top;
}

// Membership and fibre-top distances around k for a plane operator on axes a, b: with
// r = prod over the other axes of (1 + k_l), k + u e_a + v e_b lies in K iff its coordinates are >= 0
// and r (1 + k_a + u)(1 + k_b + v) <= B (u, v compile-time after unrolling; a point with no positive
// step is in K once its coordinates are, K being downward closed).  topA(v): steps to the a-fibre
// top at k + v e_b, capped at P; topB(u, cap): steps to the b-fibre top at k + u e_a, capped at
// min(cap, TB) (0 when that point is not in K: no step from it stays in K).
template <int P, int TB>
struct PlaneTops {
    int ka, kb, rab, B;
    __device__ __forceinline__ bool in_k(int u, int v) const
    {
        bool r = true;
        if (u < 0) r = r && ka + u >= 0;
        if (v < 0) r = r && kb + v >= 0;
        if (u > 0 || v > 0) r = r && rab * (1 + ka + u) * (1 + kb + v) <= B;
        return r;
    }
    __device__ __forceinline__ int topA(int v) const
    {
        int d = 0;
#pragma unroll
        for (int t = 1; t <= P; ++t) d += in_k(t, v) ? 1 : 0;
        return d;
    }
    __device__ __forceinline__ int topB(int u, int cap) const
    {
        int d = 0;
#pragma unroll
        for (int t = 1; t <= TB; ++t) d += (t <= cap && in_k(u, t)) ? 1 : 0;
        return d;
    }
};

// Line operator P(X_a), P of pure parity and degree P (offsets -P, -P+2, ..., P), axis role RA,
// applied to NSRC inputs at once (the addresses and weights are shared): out[q] = P(X_a) srcs[q]
// at the element.
template <typename R, int P, int RA, int NSRC, typename CM = ColsRuntime>
__device__ __forceinline__ void line_role_n(const Ctx &c, const Elem &el, const OpSet &O, const Op &op, const R *tab,
                                            const typename Vec2<R>::T *const (&srcs)[NSRC],
                                            typename Vec2<R>::T (&out)[NSRC])
{
    using V = typename Vec2<R>::T;
    const int ka = RA == ROLE_LAST ? el.j : coord_a<CM>(c, el, op);
    // steps from k to the top of its a-fibre, capped at P
    int top;
    if (RA == ROLE_LAST) {
        top = min(P, el.rlen - 1 - el.j);
    } else if constexpr (CM::kTopsBits) {
        top = CM::lineTop(el);
    } else {
        top = line_top<P>(c, el, ka);
    }
    constexpr int W = packed_width(P);
    const RowW<R, W> row = load_roww<W>(tab + op.ptabP + (ka * (P + 1) + top) * W);   // entries at s = -P + 2j
    constexpr int NP = P + 1;
    const auto gn = CM::gn_load(el);
    int addr[NP];
    bool okj[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        const int s = -P + 2 * j;
        const bool ok = ka + s >= 0 && s <= top;
        okj[j] = ok;
        if (RA == ROLE_LAST) addr[j] = el.e + s;
        else addr[j] = s == 0 ? el.e : CM::start(c, el, O, op, gn, s + P, ok) + el.j;
    }
    // gathers predicated on membership (a point outside K contributes nothing)
    V v[NSRC][NP];
#pragma unroll
    for (int q = 0; q < NSRC; ++q)
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            v[q][j] = czero<V>();
            if (okj[j]) v[q][j] = srcs[q][addr[j]];
        }
#pragma unroll
    for (int q = 0; q < NSRC; ++q) {
        V acc = czero<V>();
#pragma unroll
        for (int j = 0; j < NP; ++j) acc = cmad(row.v[j], v[q][j], acc);
        out[q] = acc;
    }
}

template <typename R, int P, int RA, typename CM = ColsRuntime>
__device__ __forceinline__ typename Vec2<R>::T line_role(const Ctx &c, const Elem &el, const OpSet &O, const Op &op,
                                                         const R *tab, const typename Vec2<R>::T *src)
{
    const typename Vec2<R>::T *srcs[1] = {src};
    typename Vec2<R>::T out[1];
    line_role_n<R, P, RA, 1, CM>(c, el, O, op, tab, srcs, out);
    return out[0];
}

// Plane operator wAB P(X_a) Q(X_b) + wBA Q(X_b) P(X_a), pure parities, degrees P, Q <= 2; a is a
// prefix axis, b has role RB.  Evaluated factor by factor:
//   AB: sum_s [P]_{k, k+s e_a} sum_s2 [Q]_{k+s e_a, k+s e_a+s2 e_b} c(k + s e_a + s2 e_b),
//   BA: sum_s2 [Q]_{k, k+s2 e_b} sum_s [P]_{k+s2 e_b, k+s2 e_b+s e_a} c(k + s e_a + s2 e_b),
// with the rows of P(J_n / L) and Q(J_n / L) taken from the tables by coordinate and distance to
// the fibre top (a path through an intermediate point outside K meets a zero entry).  ORD = 0:
// both orders with the weights wAB, wBA of O; 1: AB only (weight 1); 2: BA only (weight 1); 3: both
// orders with weight 1/2 each, (AB + BA) / 2 (the same rounding: halving is exact).
// SB > 0: a line operator S(X_b) of degree SB (parity of Q, SB = Q or Q + 2) merged into this op
// (P is even, so the points s = 0 are footprint points); its sum goes to lout.  NSRC inputs at once
// (addresses, fibre tops and weights shared): the sums for srcs[q] go to out[q] and lout[q].
template <typename R, int P, int Q, int RB, int SB, int NSRC, int ORD = 0, typename CM = ColsRuntime>
__device__ __forceinline__ void plane_role_n(const Ctx &c, const Elem &el, const OpSet &O, const Op &op, const R *tab,
                                             const typename Vec2<R>::T *const (&srcs)[NSRC],
                                             typename Vec2<R>::T (&out)[NSRC], typename Vec2<R>::T (&lout)[NSRC])
{
    using V = typename Vec2<R>::T;
    const int B = c.S->B;
    const int ka = coord_a<CM>(c, el, op);
    const int kb = RB == ROLE_LAST ? el.j : coord_b<CM>(c, el, op);
    const R *tP = tab + op.ptabP, *tQ = tab + op.ptabQ;   // packed rows: entry i at offset -P + 2i
    constexpr int NS = P + 1, NS2 = Q + 1;         // offsets s = -P + 2i, s2 = -Q + 2j
    constexpr int TB = SB > Q ? SB : Q;            // b-distances needed at k
    // membership and fibre-top distances: computed here (PlaneTops), or read from the element's
    // top words, which plane_tops filled with the same PlaneTops (kernels compiled per potential)
    const PlaneTops<P, TB> G{ka, kb, CM::kTopsBits ? 0 : exact_div(el.qall, (1 + ka) * (1 + kb)), B};
    auto topA = [&](int s2) {
        if constexpr (CM::kTopsBits) return CM::topA(el, s2);
        else return G.topA(s2);
    };
    auto topB = [&](int s, int cap) {
        if constexpr (CM::kTopsBits) return CM::topB(el, s);   // stored with cap TB at s = 0, Q elsewhere
        else return G.topB(s, cap);
    };
    // k + u e_a + v e_b in K (with the top words: a point with a positive step along a is in K iff
    // that many steps stay below the a-fibre top at k + v e_b, one with only a positive step along b
    // iff they stay below the b-fibre top at k + u e_a)
    auto in_k = [&](int u, int v) {
        if constexpr (!CM::kTopsBits) {
            return G.in_k(u, v);
        } else {
            bool r = true;
            if (u < 0) r = r && ka + u >= 0;
            if (v < 0) r = r && kb + v >= 0;
            if (u > 0) r = r && topA(v) >= u;
            else if (v > 0) r = r && topB(u, v) >= v;
            return r;
        }
    };
    // RB = LAST: the row of k + s e_a exists (with the top words: it holds a footprint point in K,
    // which is all the addresses need)
    auto row_in_k = [&](int s) {
        if constexpr (!CM::kTopsBits) {
            return s < 0 ? ka + s >= 0 : (s == 0 || G.rab * (1 + ka + s) <= B);
        } else {
            bool r = s == 0;
#pragma unroll
            for (int j = 0; j < NS2; ++j) r = r || in_k(s, -Q + 2 * j);
            return r;
        }
    };
    // addresses of the footprint points and their membership; the gathers are predicated on it (a
    // point outside K contributes nothing)
    const auto gn = CM::gn_load(el);
    int addr[NS][NS2];
    bool okp[NS][NS2];
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        const int s = -P + 2 * i;
        int base_s = el.e - el.j;                       // RB = LAST: start of the row of k + s e_a
        if (RB == ROLE_LAST && s != 0)
            base_s = CM::start(c, el, O, op, gn, (s + P) * (2 * Q + 1) + Q, row_in_k(s));
#pragma unroll
        for (int j = 0; j < NS2; ++j) {
            const int s2 = -Q + 2 * j;
            const bool ok = in_k(s, s2);
            okp[i][j] = ok;
            int a;
            if (RB == ROLE_LAST) a = base_s + el.j + s2;
            else if (s == 0 && s2 == 0) a = el.e;
            else a = CM::start(c, el, O, op, gn, (s + P) * (2 * Q + 1) + (s2 + Q), ok) + el.j;
            addr[i][j] = a;
        }
    }
    constexpr int NX = SB > Q ? 2 : 0;                  // merged line points +-SB outside the plane footprint
    int xaddr[NX > 0 ? NX : 1];
    bool okx[NX > 0 ? NX : 1];
#pragma unroll
    for (int j = 0; j < NX; ++j) {
        const int s2 = j == 0 ? -SB : SB;
        const bool ok = in_k(0, s2);
        okx[j] = ok;
        int a;
        if (RB == ROLE_LAST) {
            a = el.e + s2;
        } else {
            a = CM::startx(c, el, O, op, gn, j, SB, ok) + el.j;
        }
        xaddr[j] = a;
    }
    V v[NSRC][NS][NS2];
#pragma unroll
    for (int q = 0; q < NSRC; ++q)
#pragma unroll
        for (int i = 0; i < NS; ++i)
#pragma unroll
            for (int j = 0; j < NS2; ++j) {
                v[q][i][j] = czero<V>();
                if (okp[i][j]) v[q][i][j] = srcs[q][addr[i][j]];
            }
    V xv[NSRC][NX > 0 ? NX : 1];
#pragma unroll
    for (int q = 0; q < NSRC; ++q)
#pragma unroll
        for (int j = 0; j < NX; ++j) {
            xv[q][j] = czero<V>();
            if (okx[j]) xv[q][j] = srcs[q][xaddr[j]];
        }
    const int dB0 = topB(0, TB);                        // b-distance at k, capped at max(Q, SB)
    // rows of Q(J_n / L) at k_b for distance d to the b-fibre top: for degree 1 both distances come
    // from one 4-entry load (the rows are stored side by side)
    [[maybe_unused]] Row4<R> qpair;
    if constexpr (Q == 1) qpair = load_row4(tQ + kb * 4);
    auto rowQ = [&](int d) {
        if constexpr (Q == 1) {
            Row4<R> r;
            r.v[0] = d ? qpair.v[2] : qpair.v[0];
            r.v[1] = d ? qpair.v[3] : qpair.v[1];
            r.v[2] = r.v[3] = (R)0;
            return r;
        } else {
            return load_row4(tQ + (kb * (Q + 1) + d) * 4);
        }
    };
#pragma unroll
    for (int q = 0; q < NSRC; ++q) out[q] = czero<V>();
    if constexpr (sizeof(R) == 8 && NSRC == 1 && (ORD == 0 || ORD == 3)) {
        // FP64, one input, both orders: one real weight per footprint point,
        //   w_ij = wAB [P]_{k, k+s e_a} [Q]_{k+s e_a, k+s e_a+s2 e_b} + wBA [Q]_{k, k+s2 e_b} [P]_{k+s2 e_b, k+s e_a+s2 e_b},
        // then one complex multiply-add per point: 2 NS NS2 + NS + NS2 operations for the weights and
        // 4 NS NS2 for the sums, instead of 8 NS NS2 + 4 for the two nested sums (the FP64 kernels are
        // bound by their FP64 arithmetic); the same rows and the same exact-zero entries outside K.
        // The FP32 kernels keep the nested sums: at their 64-register limit the weights spilled.
        const R wab = ORD == 3 ? (R)0.5 : (R)O.wAB, wba = ORD == 3 ? (R)0.5 : (R)O.wBA;
        const Row4<R> rowP0 = load_row4(tP + (ka * (P + 1) + topA(0)) * 4);
        const Row4<R> rowQ0 = rowQ(min(Q, dB0));
        R hp[NS], hq[NS2];
#pragma unroll
        for (int i = 0; i < NS; ++i) hp[i] = wab * rowP0.v[i];
#pragma unroll
        for (int j = 0; j < NS2; ++j) hq[j] = wba * rowQ0.v[j];
        R w[NS][NS2];
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            const int s = -P + 2 * i;
            const Row4<R> rq = rowQ(s == 0 ? min(Q, dB0) : topB(s, Q));
#pragma unroll
            for (int j = 0; j < NS2; ++j) w[i][j] = hp[i] * rq.v[j];
        }
#pragma unroll
        for (int j = 0; j < NS2; ++j) {
            const Row4<R> rp = load_row4(tP + (ka * (P + 1) + topA(-Q + 2 * j)) * 4);
#pragma unroll
            for (int i = 0; i < NS; ++i) w[i][j] = fma(hq[j], rp.v[i], w[i][j]);
        }
#pragma unroll
        for (int q = 0; q < NSRC; ++q) {
            V o = czero<V>();
#pragma unroll
            for (int i = 0; i < NS; ++i)
#pragma unroll
                for (int j = 0; j < NS2; ++j) o = cmad(w[i][j], v[q][i][j], o);
            out[q] = o;
        }
    } else {
    if (ORD != 2) {   // P(X_a) (Q(X_b) c)
        const Row4<R> rowP0 = load_row4(tP + (ka * (P + 1) + topA(0)) * 4);
        Row4<R> rowQs[NS];
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            const int s = -P + 2 * i;
            const int d = s == 0 ? min(Q, dB0) : topB(s, Q);
            rowQs[i] = rowQ(d);
        }
#pragma unroll
        for (int q = 0; q < NSRC; ++q) {
            V ab = czero<V>();
#pragma unroll
            for (int i = 0; i < NS; ++i) {
                V u = czero<V>();
#pragma unroll
                for (int j = 0; j < NS2; ++j) u = cmad(rowQs[i].v[j], v[q][i][j], u);
                ab = cmad(rowP0.v[i], u, ab);
            }
            out[q] = ORD == 0 ? cscale(rconst<R>(O.wAB, O.wAB32), ab) : ab;
        }
    }
    if (ORD != 1) {   // Q(X_b) (P(X_a) c)
        const Row4<R> rowQ0 = rowQ(min(Q, dB0));
        Row4<R> rowPs[NS2];
#pragma unroll
        for (int j = 0; j < NS2; ++j) rowPs[j] = load_row4(tP + (ka * (P + 1) + topA(-Q + 2 * j)) * 4);
#pragma unroll
        for (int q = 0; q < NSRC; ++q) {
            V ba = czero<V>();
#pragma unroll
            for (int j = 0; j < NS2; ++j) {
                V w = czero<V>();
#pragma unroll
                for (int i = 0; i < NS; ++i) w = cmad(rowPs[j].v[i], v[q][i][j], w);
                ba = cmad(rowQ0.v[j], w, ba);
            }
            out[q] = ORD == 0 ? cmad(rconst<R>(O.wBA, O.wBA32), ba, out[q])
                   : ORD == 3 ? cscale((R)0.5, cadd(out[q], ba)) : ba;
        }
    }
    }
    if (SB > 0) {   // the merged line op: points k + s2 e_b, s2 = -SB, -SB + 2, ..., SB
        const Op &ls = O.op[op.mergeB];
        const Row4<R> rowS0 = load_row4(tab + ls.ptabP + (kb * (SB + 1) + min(SB, dB0)) * 4);   // entry (s2 + SB) / 2
#pragma unroll
        for (int q = 0; q < NSRC; ++q) {
            V l = czero<V>();
#pragma unroll
            for (int j = 0; j < NS2; ++j) {
                const int s2 = -Q + 2 * j;
                l = cmad(rowS0.v[(s2 + SB) / 2], v[q][P / 2][j], l);   // s = 0 is column P / 2
            }
#pragma unroll
            for (int j = 0; j < NX; ++j) l = cmad(rowS0.v[j == 0 ? 0 : SB], xv[q][j], l);
            lout[q] = l;
        }
    } else {
#pragma unroll
        for (int q = 0; q < NSRC; ++q) lout[q] = czero<V>();
    }
}

// The fibre-top distances plane_role_n reads from the top words (CM::kTopsBits), computed and
// packed at the offsets of CM: topA at v = 0 and at the footprint's steps along b, topB at the
// footprint's steps along a (cap TB at 0, Q elsewhere).
template <int P, int Q, int RB, int SB, typename CM>
__device__ __forceinline__ void plane_tops(const Ctx &c, const Elem &el, const Op &op, unsigned *tw)
{
    constexpr int TB = SB > Q ? SB : Q;
    const int ka = coord_a<CM>(c, el, op);
    const int kb = RB == ROLE_LAST ? el.j : coord_b<CM>(c, el, op);
    const PlaneTops<P, TB> G{ka, kb, exact_div(el.qall, (1 + ka) * (1 + kb)), c.S->B};
    put_top_field(tw, CM::offA(0), G.topA(0));
#pragma unroll
    for (int j = 0; j <= Q; ++j)
        if (-Q + 2 * j != 0) put_top_field(tw, CM::offA(-Q + 2 * j), G.topA(-Q + 2 * j));
#pragma unroll
    for (int i = 0; i <= P; ++i) {
        const int s = -P + 2 * i;
        put_top_field(tw, CM::offB(s), G.topB(s, s == 0 ? TB : Q));
    }
}

// The same for a line operator along a prefix axis (line_role_n with the top words).
template <int P, typename CM>
__device__ __forceinline__ void line_tops(const Ctx &c, const Elem &el, const Op &op, unsigned *tw)
{
    put_top_field(tw, CM::offT, line_top<P>(c, el, coord_a<CM>(c, el, op)));
}

template <typename R, int P, int Q, int RB, int SB, int ORD = 0, typename CM = ColsRuntime>
__device__ __forceinline__ void plane_role(const Ctx &c, const Elem &el, const OpSet &O, const Op &op, const R *tab,
                                           const typename Vec2<R>::T *src, typename Vec2<R>::T &out,
                                           typename Vec2<R>::T &lout)
{
    const typename Vec2<R>::T *srcs[1] = {src};
    typename Vec2<R>::T o[1], l[1];
    plane_role_n<R, P, Q, RB, SB, 1, ORD, CM>(c, el, O, op, tab, srcs, o, l);
    out = o[0];
    lout = l[0];
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

// The per-thread view of element e from its record er = {row, group, prod (1 + k_l) | sum k_l << 16,
// k_{N-1} | row length << 16}.
__device__ __forceinline__ Elem make_elem(const ApplyArgs &args, int e, int4 er)
{
    Elem el;
    const int N = args.S.N;
    el.e = e;
    el.j = er.w & 0xffff;
    el.rlen = (int)((unsigned)er.w >> 16);
    el.qall = er.z & 0xffff;
    el.ksum = (int)((unsigned)er.z >> 16);
    el.r = er.x;
    el.kr = args.S.row_k + (size_t)er.x * (N - 1);
    el.k4 = N >= 2 ? (int)__ldg(el.kr + N - 2) : 0;
    el.gn = args.gnb + (size_t)er.y * args.gstride;
#pragma unroll
    for (int w = 0; w < kTopWords; ++w)
        el.tw[w] = w < args.tops_words ? __ldg(args.tops + (size_t)w * args.S.size + e) : 0u;
    el.grows = 0;
    el.gnn = nullptr;
    if (args.S.general) {
        el.grows = __ldg(args.S.gfirst + er.y + 1) - __ldg(args.S.gfirst + er.y);
        el.gnn = args.gnbn + (size_t)er.y * args.gstride;
    }
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
        const R dj = rconst<R>(args.dscale, args.dscale32) * ((R)el.ksum + (R)0.5 * (R)S.N);   // (D_K)_jj = sum_l (j_l + 1/2), times S^2
        acc.add(cscale(dj, cin[e]));
    }
    body(ctx, el, acc, sm_w, cin, (const R *)args.tab);
    V y = acc.get();
    if (!args.stage1) {
        y = cscale(oscale, y);
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
template <typename R, int DOTS = 0, typename Body>
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
    ctx.mv = args.mv;
    const int stride = gridDim.x * blockDim.x;
    if constexpr (DOTS == 0) {
        for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < S.size; e += stride)
            apply_element<R>(args, ctx, e, __ldg(S.elem + e), oscale, sm_w, body);
    } else if constexpr (DOTS == 2) {
        // the Rayleigh quotient ds[0] <cin, y>: each thread keeps a TwoSum-compensated FP32 sum of
        // conj(cin_e) y_e (cin_e is in L1 from the diagonal term), warps add the pairs by shuffles,
        // blocks by reduce_warp_sums
        static_assert(sizeof(R) == 4, "the fused Rayleigh quotient is implemented for complex64 vectors");
        const float2 *cin = (const float2 *)args.cin;
        float rs = 0.f, rc = 0.f, is = 0.f, ic = 0.f;
        auto add = [](float &sum, float &comp, float x) {
            const float t = sum + x, bb = t - sum;
            comp += (sum - (t - bb)) + (x - bb);
            sum = t;
        };
        for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < S.size; e += stride) {
            const float2 y = apply_element<R>(args, ctx, e, __ldg(S.elem + e), oscale, sm_w, body);
            const float2 x = cin[e];
            add(rs, rc, fmaf(x.x, y.x, x.y * y.y));
            add(is, ic, fmaf(x.x, y.y, -x.y * y.x));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ors = __shfl_xor_sync(0xffffffffu, rs, o), orc = __shfl_xor_sync(0xffffffffu, rc, o);
            const float ois = __shfl_xor_sync(0xffffffffu, is, o), oic = __shfl_xor_sync(0xffffffffu, ic, o);
            rc += orc;
            add(rs, rc, ors);
            ic += oic;
            add(is, ic, ois);
        }
        __shared__ double wsum[8][2];
        if ((threadIdx.x & 31) == 0) {
            wsum[threadIdx.x >> 5][0] = (double)rs + (double)rc;
            wsum[threadIdx.x >> 5][1] = (double)is + (double)ic;
        }
        __syncthreads();
        __shared__ double tot[2];
        if (reduce_warp_sums<2>(wsum, 2, args.dpartials, args.dcounter, tot) && threadIdx.x == 0) {
            args.dh[0] = args.ds[0] * tot[0];
            args.dh[1] = args.ds[0] * tot[1];
            *args.dcounter = 0;
        }
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
    ctx.mv = args.mv;
    const V *cin = (const V *)args.cin;
    const V *cin2 = args.cin2 ? (const V *)args.cin2 : cin;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < S.size; e += gridDim.x * blockDim.x) {
        const int4 er = __ldg(S.elem + e);
        const Elem el = make_elem(args, e, er);
        Acc<R> acc, acc2;
        if (!args.skip_diag) {
            const R dj = rconst<R>(args.dscale, args.dscale32) * ((R)el.ksum + (R)0.5 * (R)S.N);
            acc.add(cscale(dj, cin[e]));
            acc2.add(cscale(dj, cin2[e]));
        }
        body(ctx, el, acc, acc2, (const R *)sm_w, (const R *)sm_w2, cin, cin2, (const R *)args.tab);
        const V y = cscale(oscale, acc.get()), y2 = cscale(oscale, acc2.get());
        if (args.mag_g != 0.0) {
            const V a = cin[e], b = cin2[e];
            const R g = rconst<R>(args.mag_g, args.mag_g32), half = (R)0.5;
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
