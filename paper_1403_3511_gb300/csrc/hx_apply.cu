// The matrix-free product y = A(t) c = D_K c + W^pol(X_K, t) c on the hyperbolic cross
// (Sec. 3 of Brumm, arXiv:1403.3511), as one fused kernel per launch.
//
// W^pol is compiled on the host (hx_capi.cu) into operators of three kinds: the identity,
// line operators P(X_a) and plane operators P(X_a) Q(X_b) (a < b, in the configured factor
// order).  X_K^{(a)} is block-diagonal over the fibres of K along axis a, and on a fibre of
// length n it is the truncated Jacobi matrix J_n of the recurrence Eq. (Recurrence1D); so
// P(X_a) is banded with half-width deg P and its rows are the rows of P(J_n / L), read from
// precomputed row tables.  Each output coefficient is computed once, by gathering the input
// coefficients in its stencil footprint: the paper's term-by-term sweep (Algorithm
// fast_algorithm) is reordered into a single pass over the output.
//
// Tiling.  A work item is a run of consecutive slabs (elements sharing the outer prefix
// k_0..k_{N-3}), at most kItemElems elements.  Phase A computes, for each slab of the item
// and each outer offset delta the operators need, the start of slab "prefix + delta" and its
// prefix product (shared memory).  Phase B assigns one thread per output element.
#include <math.h>

#include "hx_internal.h"

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
};

// amp * f(t) in the stencil precision R (the interval index of a piecewise-constant modulation is
// always found in FP64 so that both precisions switch intervals at the same t).
template <typename R>
__device__ __forceinline__ R op_weight(const Op &op, double t, const double *pw)
{
    R f = (R)1;
    switch (op.mod) {
        case HX_MOD_COS: f = cos((R)(op.omega * t + op.phase)); break;
        case HX_MOD_SIN2: { R s = sin((R)(op.omega * t)); f = s * s; } break;
        case HX_MOD_PWCONST: {
            double x = floor((t - op.pw_t0) / (op.pw_t1 - op.pw_t0) * op.pw_n);
            int qi = x < 0.0 ? 0 : (x >= op.pw_n ? op.pw_n - 1 : (int)x);
            f = (R)pw[op.pw_off + qi];
        } break;
        default: break;
    }
    return (R)op.amp * f;
}

// Exact a / b when b divides a (both < 2^24): the correctly rounded float quotient is the integer.
__device__ __forceinline__ int exact_div(int a, int b) { return __float2int_rn(__fdiv_rn((float)a, (float)b)); }

// floor(B / x) for integers B, x >= 1 with B + x < 2^24: the rounding error of the correctly rounded
// float quotient, at most 2^-24 (B / x + 1), is smaller than the distance 1/x to the next integer.
__device__ __forceinline__ int floor_div(int B, int x) { return __float2int_rz(__fdiv_rn((float)B, (float)x)); }

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
    int e;          // rank
    int start;      // start of own slab
    int qoff;       // qoff[q] of own slab
    int sl;         // slab index inside the item
    int qall;       // prod_l (1 + k_l)
    int k1, k2;     // coordinates on the inner axes N-2, N-1 (k1 = 0 when N == 1)
};

struct Ctx {
    const DevSet *S;
    const int2 *nb;           // item neighbour table (shared): slab start, qoff
    int nd;
    const uint16_t *kk;       // shared multi-indices, [l * blockDim + tid]
    int tid, nthr;
    __device__ int k(int l) const { return kk[l * nthr + tid]; }
};

// Address of element k + s e_a + s2 e_b (footprint position pos of the operator).
__device__ __forceinline__ int point_addr(const Ctx &c, const Elem &el, const OpSet &O, const Op &op, int pos,
                                          int a, int s, int b, int s2)
{
    const DevSet &S = *c.S;
    int N = S.N;
    int di = O.didx[op.dbase + pos];
    int start = el.start, qoff = el.qoff;
    if (di != 0) {
        int2 nb = c.nb[el.sl * c.nd + di];
        start = nb.x;
        qoff = nb.y;
    }
    int i2 = el.k2 + (a == N - 1 ? s : 0) + (b == N - 1 ? s2 : 0);
    if (N == 1) return start + i2;
    int i1 = el.k1 + (a == N - 2 ? s : 0) + (b == N - 2 ? s2 : 0);
    return start + S.Q[qoff + i1] + i2;
}

// Number of steps (capped at p) from coordinate i to the top of its fibre, given the product
// `other` of (1 + k_l) over the remaining axes: steps t with (1 + i + t) * other <= B.
__device__ __forceinline__ int top_dist(int i, int other, int p, int B)
{
    int d = 0;
#pragma unroll 8
    for (int t = 1; t <= kMaxDeg; ++t)
        if (t <= p && (1 + i + t) * other <= B) d = t;
    return d;
}

template <typename R, int MP, bool UNROLL>
__device__ __forceinline__ void line_op(const Ctx &c, const Elem &el, const OpSet &O, const Op &op, const R *tab,
                                        const typename Vec2<R>::T *cin, R &sx, R &sy)
{
    const int B = c.S->B;
    const int a = op.a, p = op.p;
    const int ka = c.k(a);
    const int other = __float2int_rn(__fdiv_rn((float)el.qall, (float)(1 + ka)));
    const int d = top_dist(ka, other, p, B);
    const R *row = tab + op.tabP + ((size_t)ka * (p + 1) + d) * (2 * p + 1) + p;
#pragma unroll(UNROLL ? 2 * MP + 1 : 1)
    for (int s = -MP; s <= MP; ++s) {
        if (s < -p || s > p || !((op.pmask >> (s + p)) & 1)) continue;
        if (ka + s < 0 || s > d) continue;
        int addr = point_addr(c, el, O, op, (s + p), a, s, -1, 0);
        typename Vec2<R>::T v = cin[addr];
        R w = row[s];
        sx += w * v.x;
        sy += w * v.y;
    }
}

template <typename R, int MP, int MQ, bool UNROLL>
__device__ __forceinline__ void plane_op(const Ctx &c, const Elem &el, const OpSet &O, const Op &op, const R *tab,
                                         const typename Vec2<R>::T *cin, R &sx, R &sy)
{
    const int B = c.S->B;
    const int a = op.a, b = op.b, p = op.p, q = op.q;
    const int ka = c.k(a), kb = c.k(b);
    const int rab = __float2int_rn(__fdiv_rn((float)el.qall, (float)((1 + ka) * (1 + kb))));
    const R wAB = (R)O.wAB, wBA = (R)O.wBA;
    // fibre-top distances: along a at k + s2 e_b, along b at k + s e_a
    int dA[2 * MQ + 1], dB[2 * MP + 1];
#pragma unroll(UNROLL ? 2 * MQ + 1 : 1)
    for (int s2 = -MQ; s2 <= MQ; ++s2) dA[s2 + MQ] = top_dist(ka, rab * (1 + kb + s2), p, B);
#pragma unroll(UNROLL ? 2 * MP + 1 : 1)
    for (int s = -MP; s <= MP; ++s) dB[s + MP] = top_dist(kb, rab * (1 + ka + s), q, B);
    const int dA0 = dA[MQ], dB0 = dB[MP];
    const R *rowP0 = tab + op.tabP + ((size_t)ka * (p + 1) + dA0) * (2 * p + 1) + p;
    const R *rowQ0 = tab + op.tabQ + ((size_t)kb * (q + 1) + dB0) * (2 * q + 1) + q;
#pragma unroll(UNROLL ? 2 * MP + 1 : 1)
    for (int s = -MP; s <= MP; ++s) {
        if (s < -p || s > p || !((op.pmask >> (s + p)) & 1) || ka + s < 0) continue;
        const bool inA = s <= dA0;                      // k + s e_a in K
        const R pj = inA ? rowP0[s] : (R)0;
        const R *rowQs = tab + op.tabQ + ((size_t)kb * (q + 1) + dB[s + MP]) * (2 * q + 1) + q;
#pragma unroll(UNROLL ? 2 * MQ + 1 : 1)
        for (int s2 = -MQ; s2 <= MQ; ++s2) {
            if (s2 < -q || s2 > q || !((op.qmask >> (s2 + q)) & 1) || kb + s2 < 0) continue;
            if (rab * (1 + ka + s) * (1 + kb + s2) > B) continue;   // footprint point not in K
            R cab = inA ? pj * rowQs[s2] : (R)0;                     // P(X_a) (Q(X_b) c)
            R cba = (R)0;                                            // Q(X_b) (P(X_a) c)
            if (s2 <= dB0) {
                const R *rowPs = tab + op.tabP + ((size_t)ka * (p + 1) + dA[s2 + MQ]) * (2 * p + 1) + p;
                cba = rowQ0[s2] * rowPs[s];
            }
            R w = wAB * cab + wBA * cba;
            int addr = point_addr(c, el, O, op, (s + p) * (2 * q + 1) + (s2 + q), a, s, b, s2);
            typename Vec2<R>::T v = cin[addr];
            sx += w * v.x;
            sy += w * v.y;
        }
    }
}

// floor(B / x) for x >= 1 from the table (0 when x > B: no element has those coordinates).
__device__ __forceinline__ int nt_of(const DevSet &S, int x) { return x <= S.B ? __ldg(S.nt + x) : 0; }

// Row start (global rank of local row i) inside the slab described by (start, qoff); N >= 2.
__device__ __forceinline__ int row_start(const DevSet &S, int start, int qoff, int i) { return start + __ldg(S.Q + qoff + i); }

// Base rank of the point that moves by s along an axis of role RA (k + s e_a), before adding the
// last coordinate: own slab for inner roles, neighbour slab for an outer axis.
template <int RA>
__device__ __forceinline__ int2 slab_of(const Ctx &c, const Elem &el, const OpSet &O, int didx_pos)
{
    if (RA == ROLE_OUT) {
        const int di = O.didx[didx_pos];
        return c.nb[el.sl * c.nd + di];
    }
    return make_int2(el.start, el.qoff);
}

// Line operator P(X_a), P of pure parity and degree P (offsets -P, -P+2, ..., P), axis role RA.
template <typename R, int P, int RA>
__device__ __forceinline__ void line_role(const Ctx &c, const Elem &el, const OpSet &O, const Op &op, const R *tab,
                                          const typename Vec2<R>::T *src, R &sx, R &sy)
{
    const DevSet &S = *c.S;
    const int ka = RA == ROLE_I2 ? el.k2 : (RA == ROLE_I1 ? el.k1 : c.k(op.a));
    const int top = nt_of(S, exact_div(el.qall, 1 + ka)) - 1 - ka;      // steps to the top of the a-fibre
    const R *row = tab + op.tabP + (ka * (P + 1) + min(P, top)) * (2 * P + 1) + P;
    const int own_row = RA == ROLE_I2 ? (S.N >= 2 ? row_start(S, el.start, el.qoff, el.k1) : el.start) : 0;
#pragma unroll
    for (int s = -P; s <= P; s += 2) {
        if (ka + s < 0 || s > top) continue;
        int addr;
        if (RA == ROLE_I2) {
            addr = own_row + el.k2 + s;
        } else if (RA == ROLE_I1) {
            addr = row_start(S, el.start, el.qoff, el.k1 + s) + el.k2;
        } else {
            const int2 nb = slab_of<ROLE_OUT>(c, el, O, op.dbase + s + P);
            addr = (S.N >= 2 ? row_start(S, nb.x, nb.y, el.k1) : nb.x) + el.k2;
        }
        const typename Vec2<R>::T v = src[addr];
        const R w = row[s];
        sx += w * v.x;
        sy += w * v.y;
    }
}

// Plane operator wAB P(X_a) Q(X_b) + wBA Q(X_b) P(X_a), pure parities, degrees P, Q, roles RA < RB.
// A footprint point k + s e_a + s2 e_b carries [P]_{k, k+s e_a} [Q]_{k+s e_a, k+s e_a+s2 e_b} (path
// through k + s e_a) and [Q]_{k, k+s2 e_b} [P]_{k+s2 e_b, k+s2 e_b+s e_a} (path through k + s2 e_b);
// a path exists only if its intermediate point is in K.  Rows of P(J_n / L) and Q(J_n / L) come
// from the tables, indexed by the coordinate and the distance to the fibre top.
template <typename R, int P, int Q, int RA, int RB>
__device__ __forceinline__ void plane_role(const Ctx &c, const Elem &el, const OpSet &O, const Op &op, const R *tab,
                                           const typename Vec2<R>::T *src, R &sx, R &sy)
{
    const DevSet &S = *c.S;
    const int ka = RA == ROLE_I1 ? el.k1 : c.k(op.a);
    const int kb = RB == ROLE_I2 ? el.k2 : (RB == ROLE_I1 ? el.k1 : c.k(op.b));
    const int rab = exact_div(el.qall, (1 + ka) * (1 + kb));
    const R wAB = (R)O.wAB, wBA = (R)O.wBA;
    const R *tP = tab + op.tabP, *tQ = tab + op.tabQ;
    // a-fibre tops at k + s2 e_b, b-fibre tops at k + s e_a
    int topA[2 * Q + 1], topB[2 * P + 1];
    const R *rowP[2 * Q + 1];   // P row at k + s2 e_b (valid when that point is in K)
    const R *rowQ[2 * P + 1];   // Q row at k + s e_a
    topA[Q] = nt_of(S, rab * (1 + kb)) - 1 - ka;
    topB[P] = nt_of(S, rab * (1 + ka)) - 1 - kb;
#pragma unroll
    for (int s2 = -Q; s2 <= Q; s2 += 2)
        if (s2 != 0) topA[s2 + Q] = kb + s2 >= 0 ? nt_of(S, rab * (1 + kb + s2)) - 1 - ka : -1;
#pragma unroll
    for (int s = -P; s <= P; s += 2)
        if (s != 0) topB[s + P] = ka + s >= 0 ? nt_of(S, rab * (1 + ka + s)) - 1 - kb : -1;
#pragma unroll
    for (int s2 = -Q; s2 <= Q; ++s2)
        if (s2 == 0 || ((s2 - Q) & 1) == 0) rowP[s2 + Q] = tP + (ka * (P + 1) + max(0, min(P, topA[s2 + Q]))) * (2 * P + 1) + P;
#pragma unroll
    for (int s = -P; s <= P; ++s)
        if (s == 0 || ((s - P) & 1) == 0) rowQ[s + P] = tQ + (kb * (Q + 1) + max(0, min(Q, topB[s + P]))) * (2 * Q + 1) + Q;
    const int topA0 = topA[Q], topB0 = topB[P];
    int own_row = 0;
    if (RB == ROLE_I2 && RA == ROLE_I1) own_row = 0;   // rows vary with s below
#pragma unroll
    for (int s = -P; s <= P; s += 2) {
        if (ka + s < 0) continue;
        const bool inA = s <= topA0;                    // k + s e_a in K
        const R pj = inA ? rowP[Q][s] : (R)0;
        int base_s = 0;                                 // rank of row containing k + s e_a (+ s2 e_b for RB = I2)
        int2 nb_s = make_int2(el.start, el.qoff);
        if (RA == ROLE_OUT && RB != ROLE_OUT) nb_s = slab_of<ROLE_OUT>(c, el, O, op.dbase + (s + P) * (2 * Q + 1) + Q);
        if (RB == ROLE_I2) base_s = (RA == ROLE_I1) ? row_start(S, el.start, el.qoff, el.k1 + s) : row_start(S, nb_s.x, nb_s.y, el.k1);
#pragma unroll
        for (int s2 = -Q; s2 <= Q; s2 += 2) {
            if (kb + s2 < 0 || s > topA[s2 + Q]) continue;     // footprint point not in K
            const R cab = inA ? pj * rowQ[s + P][s2] : (R)0;
            const R cba = s2 <= topB0 ? rowQ[P][s2] * rowP[s2 + Q][s] : (R)0;   // k + s2 e_b in K
            const R w = wAB * cab + wBA * cba;
            int addr;
            if (RB == ROLE_I2) {
                addr = base_s + el.k2 + s2;
            } else if (RB == ROLE_I1) {                 // RA outer: neighbour slab by s, row k1 + s2
                addr = row_start(S, nb_s.x, nb_s.y, el.k1 + s2) + el.k2;
            } else {                                    // both outer: neighbour slab by (s, s2)
                const int2 nb = slab_of<ROLE_OUT>(c, el, O, op.dbase + (s + P) * (2 * Q + 1) + (s2 + Q));
                addr = row_start(S, nb.x, nb.y, el.k1) + el.k2;
            }
            const typename Vec2<R>::T v = src[addr];
            sx += w * v.x;
            sy += w * v.y;
        }
    }
    (void)own_row;
}

template <typename R, int P, int Q>
__device__ __forceinline__ void plane_dispatch(int key, const Ctx &c, const Elem &el, const OpSet &O, const Op &op,
                                               const R *tab, const typename Vec2<R>::T *src, R &sx, R &sy)
{
    if (key == ROLE_OUT * 4 + ROLE_OUT) plane_role<R, P, Q, ROLE_OUT, ROLE_OUT>(c, el, O, op, tab, src, sx, sy);
    else if (key == ROLE_OUT * 4 + ROLE_I1) plane_role<R, P, Q, ROLE_OUT, ROLE_I1>(c, el, O, op, tab, src, sx, sy);
    else if (key == ROLE_OUT * 4 + ROLE_I2) plane_role<R, P, Q, ROLE_OUT, ROLE_I2>(c, el, O, op, tab, src, sx, sy);
    else plane_role<R, P, Q, ROLE_I1, ROLE_I2>(c, el, O, op, tab, src, sx, sy);
}

template <typename R, int P>
__device__ __forceinline__ void line_dispatch(int ra, const Ctx &c, const Elem &el, const OpSet &O, const Op &op,
                                              const R *tab, const typename Vec2<R>::T *src, R &sx, R &sy)
{
    if (ra == ROLE_OUT) line_role<R, P, ROLE_OUT>(c, el, O, op, tab, src, sx, sy);
    else if (ra == ROLE_I1) line_role<R, P, ROLE_I1>(c, el, O, op, tab, src, sx, sy);
    else line_role<R, P, ROLE_I2>(c, el, O, op, tab, src, sx, sy);
}

// MD: largest polynomial degree of the compiled potential (3: unrolled stencils; kMaxDeg: rolled loops).
template <typename R, int MD>
__global__ void __launch_bounds__(kApplyThreads, MD <= 3 ? 3 : 1) apply_kernel(const __grid_constant__ ApplyArgs args)
{
    using V = typename Vec2<R>::T;
    extern __shared__ int2 sm_nb[];
    __shared__ int sm_start[65];
    __shared__ int sm_q[64];
    __shared__ uint16_t sm_pre[64 * kMaxN];
    __shared__ uint16_t sm_k[kMaxN * kApplyThreads];
    __shared__ R sm_w[kMaxOps];
    __shared__ int8_t sm_delta[kMaxDelta * 4];

    const DevSet &S = args.S;
    const OpSet &O = args.ops;
    const int N = S.N, nout = N > 2 ? N - 2 : 0, nd = O.ndelta;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const V *cin = (const V *)args.cin;
    V *cout = (V *)args.cout;
    const R *tab = (const R *)args.tab;
    const int *Q1 = S.Q;     // level m = 1

    if (tid < O.nops) sm_w[tid] = op_weight<R>(O.op[tid], *args.t_ptr + args.t_shift, args.pw_values);
    for (int x = tid; x < O.ndelta * 4; x += blockDim.x) sm_delta[x] = O.delta[x >> 2][x & 3];
    const R oscale = args.out_scale ? (R)(*args.out_scale) : (R)1;

    Ctx ctx;
    ctx.S = &S;
    ctx.nb = sm_nb;
    ctx.nd = nd;
    ctx.kk = sm_k;
    ctx.tid = tid;
    ctx.nthr = nthr;

    for (int item = blockIdx.x; item < args.nitems; item += gridDim.x) {
        const int4 it = args.items[item];
        const int s0 = it.x, ns = it.y - it.x + 1, e0 = it.z, e1 = it.w;
        __syncthreads();
        // ---- phase A: own slabs, then the neighbour slabs of every outer offset
        for (int x = tid; x < ns; x += nthr) {
            sm_start[x] = S.slab_start[s0 + x];
            int q = 1;
            for (int l = 0; l < nout; ++l) {
                int pl = S.slab_k[(size_t)(s0 + x) * nout + l];
                sm_pre[x * kMaxN + l] = (uint16_t)pl;
                q *= 1 + pl;
            }
            sm_q[x] = q;
        }
        __syncthreads();
        for (int x = tid; x < ns * nd; x += nthr) {
            const int sl = x / nd, di = x - sl * nd;
            int2 res = make_int2(-1, 0);
            int pre[kMaxN];
            bool ok = true;
            for (int l = 0; l < nout; ++l) pre[l] = sm_pre[sl * kMaxN + l];
            for (int j = 0; j < 2; ++j) {
                int ax = sm_delta[di * 4 + 2 * j];
                if (ax >= 0) pre[ax] += sm_delta[di * 4 + 2 * j + 1];
            }
            long long q = 1;
            for (int l = 0; l < nout; ++l) {
                if (pre[l] < 0) ok = false;
                q *= 1 + pre[l];
            }
            if (ok && q <= S.B) {
                int start = 0, qd = 1;
                for (int d = 0; d < nout; ++d) {
                    int m = N - 1 - d;
                    start += S.Q[(size_t)(m - 1) * S.qtotal + S.qoff[qd] + pre[d]];
                    qd *= 1 + pre[d];
                }
                res = make_int2(start, (int)S.qoff[qd]);
            }
            sm_nb[x] = res;
        }
        __syncthreads();
        // ---- phase B: one thread per output element
        for (int e = e0 + tid; e < e1; e += nthr) {
            int lo = 0, hi = ns - 1;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (sm_start[mid] <= e) lo = mid; else hi = mid - 1;
            }
            Elem el;
            el.e = e;
            el.sl = lo;
            el.start = sm_start[lo];
            const int q = sm_q[lo];
            el.qoff = S.qoff[q];
            const int local = e - el.start;
            if (N >= 2) {
                int b = S.B / q;                // rows i = 0 .. b-1 of the slab
                int l2 = 0, h2 = b - 1;
                while (l2 < h2) {
                    int mid = (l2 + h2 + 1) >> 1;
                    if (Q1[el.qoff + mid] <= local) l2 = mid; else h2 = mid - 1;
                }
                el.k1 = l2;
                el.k2 = local - Q1[el.qoff + l2];
            } else {
                el.k1 = 0;
                el.k2 = local;
            }
            int qall = q;
            R dsum = (R)0;
            for (int l = 0; l < nout; ++l) {
                int kl = sm_pre[lo * kMaxN + l];
                sm_k[l * nthr + tid] = (uint16_t)kl;
                dsum += (R)kl;
            }
            if (N >= 2) {
                sm_k[(N - 2) * nthr + tid] = (uint16_t)el.k1;
                qall *= 1 + el.k1;
                dsum += (R)el.k1;
            }
            sm_k[(N - 1) * nthr + tid] = (uint16_t)el.k2;
            qall *= 1 + el.k2;
            dsum += (R)el.k2;
            el.qall = qall;
            const V ce = cin[e];
            Acc<R> acc;
            const R dj = dsum + (R)0.5 * (R)N;   // (D_K)_jj = sum_l (j_l + 1/2)
            if (!args.stage1) acc.add(dj * ce.x, dj * ce.y);
            for (int o = 0; o < O.nops; ++o) {
                const Op &op = O.op[o];
                const V *src = op.src < 0 ? cin : (const V *)args.chan + (size_t)op.src * args.chan_ld;
                R sx = (R)0, sy = (R)0;
                if (op.kind == 0) {
                    const V cs = src[e];
                    sx = cs.x;
                    sy = cs.y;
                } else if (MD <= 3) {
                    const int key = op.ra * 4 + op.rb;
                    switch (op.cls) {
                        case CLS_LINE + 1: line_dispatch<R, 1>(op.ra, ctx, el, O, op, tab, src, sx, sy); break;
                        case CLS_LINE + 2: line_dispatch<R, 2>(op.ra, ctx, el, O, op, tab, src, sx, sy); break;
                        case CLS_LINE + 3: line_dispatch<R, 3>(op.ra, ctx, el, O, op, tab, src, sx, sy); break;
                        case CLS_PLANE + 0: plane_dispatch<R, 1, 1>(key, ctx, el, O, op, tab, src, sx, sy); break;
                        case CLS_PLANE + 3: plane_dispatch<R, 2, 1>(key, ctx, el, O, op, tab, src, sx, sy); break;
                        case CLS_PLANE + 1: plane_dispatch<R, 1, 2>(key, ctx, el, O, op, tab, src, sx, sy); break;
                        case CLS_PLANE + 4: plane_dispatch<R, 2, 2>(key, ctx, el, O, op, tab, src, sx, sy); break;
                        default:
                            if (op.kind == 1) line_op<R, 3, true>(ctx, el, O, op, tab, src, sx, sy);
                            else plane_op<R, 3, 3, true>(ctx, el, O, op, tab, src, sx, sy);
                    }
                } else {
                    if (op.kind == 1) line_op<R, kMaxDeg, false>(ctx, el, O, op, tab, src, sx, sy);
                    else plane_op<R, kMaxDeg, kMaxDeg, false>(ctx, el, O, op, tab, src, sx, sy);
                }
                const R w = sm_w[o];
                if (args.stage1) {
                    V ch;
                    ch.x = w * sx;
                    ch.y = w * sy;
                    ((V *)args.chan)[(size_t)op.dst * args.chan_ld + e] = ch;
                } else {
                    acc.add(w * sx, w * sy);
                }
            }
            if (!args.stage1) {
                V y = acc.get();
                y.x *= oscale;
                y.y *= oscale;
                cout[e] = y;
            }
        }
    }
}

int apply_grid(const Problem *p)
{
    int per_sm = 4;
    int g = p->num_sms * per_sm;
    return p->nitems < g ? (p->nitems > 0 ? p->nitems : 1) : g;
}

template <typename R, int MD>
static int launch_apply_t(Problem *p, const OpSet &ops, int stage1, const void *cin, void *cout,
                          const double *t_ptr, double t_shift, const double *out_scale, cudaStream_t st)
{
    ApplyArgs a;
    memset(&a, 0, sizeof(a));
    a.S = p->set->d;
    a.items = p->items;
    a.nitems = p->nitems;
    a.slabs_per_item = p->slabs_per_item;
    a.t_ptr = t_ptr;
    a.t_shift = t_shift;
    a.pw_values = p->pw_values;
    a.tab = p->tab;
    a.ops = ops;
    a.cin = cin;
    a.cout = cout;
    a.out_scale = out_scale;
    a.chan = p->chan;
    a.chan_ld = p->chan_ld;
    a.stage1 = stage1;
    size_t smem = (size_t)p->slabs_per_item * ops.ndelta * sizeof(int2);
    apply_kernel<R, MD><<<apply_grid(p), kApplyThreads, smem, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "apply kernel launch");
    return HX_OK;
}

static int launch_stage(Problem *p, const OpSet &ops, int stage1, const void *cin, void *cout, const double *t_ptr,
                        double t_shift, const double *scale, cudaStream_t st)
{
    int md = 0;
    for (int i = 0; i < ops.nops; ++i) md = max(md, max(ops.op[i].p, ops.op[i].q));
    if (p->cfg.dtype == HX_C64)
        return md <= 3 ? launch_apply_t<float, 3>(p, ops, stage1, cin, cout, t_ptr, t_shift, scale, st)
                       : launch_apply_t<float, kMaxDeg>(p, ops, stage1, cin, cout, t_ptr, t_shift, scale, st);
    return md <= 3 ? launch_apply_t<double, 3>(p, ops, stage1, cin, cout, t_ptr, t_shift, scale, st)
                   : launch_apply_t<double, kMaxDeg>(p, ops, stage1, cin, cout, t_ptr, t_shift, scale, st);
}

int apply_launches(const Problem *p) { return p->ops1.nops > 0 ? 2 : 1; }

int launch_apply(Problem *p, const void *cin, void *cout, const double *t_ptr, double t_shift, const ApplyFuse *fuse,
                 cudaStream_t st)
{
    const double *scale = fuse ? fuse->in_scale : nullptr;
    if (p->ops1.nops > 0) {
        int rc = launch_stage(p, p->ops1, 1, cin, nullptr, t_ptr, t_shift, nullptr, st);
        if (rc) return rc;
    }
    return launch_stage(p, p->ops, 0, cin, cout, t_ptr, t_shift, scale, st);
}

// ---------------------------------------------------------------------------------------
// export of all multi-indices (unrank on the device: slab by binary search, then the
// position inside the slab)
// ---------------------------------------------------------------------------------------
__global__ void export_kernel(DevSet S, int32_t *k)
{
    const int N = S.N, nout = N > 2 ? N - 2 : 0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < S.size; e += gridDim.x * blockDim.x) {
        int lo = 0, hi = S.nslab - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (S.slab_start[mid] <= e) lo = mid; else hi = mid - 1;
        }
        int q = 1;
        for (int l = 0; l < nout; ++l) {
            int pl = S.slab_k[(size_t)lo * nout + l];
            k[(size_t)e * N + l] = pl;
            q *= 1 + pl;
        }
        int local = e - S.slab_start[lo];
        if (N >= 2) {
            const int *row = S.Q + S.qoff[q];
            int l2 = 0, h2 = S.B / q - 1;
            while (l2 < h2) {
                int mid = (l2 + h2 + 1) >> 1;
                if (row[mid] <= local) l2 = mid; else h2 = mid - 1;
            }
            k[(size_t)e * N + N - 2] = l2;
            k[(size_t)e * N + N - 1] = local - row[l2];
        } else {
            k[e] = local;
        }
    }
}

int launch_export(const IndexSetObj *s, int32_t *k_dev, cudaStream_t st)
{
    int blocks = (int)((s->h.size + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    export_kernel<<<blocks, 256, 0, st>>>(s->d, k_dev);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "export kernel");
    return HX_OK;
}

// ---------------------------------------------------------------------------------------
// ||c||^2 in FP64 with a deterministic two-level reduction (per-block partials, summed in
// block order by the last block to finish)
// ---------------------------------------------------------------------------------------
__device__ double block_sum(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    return s;   // valid in thread 0
}

template <typename V>
__global__ void norm2_kernel(const V *c, int n, double *partials, unsigned *counter, double *result)
{
    __shared__ double red[32];
    __shared__ bool last;
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        V v = c[i];
        acc += (double)v.x * (double)v.x + (double)v.y * (double)v.y;
    }
    double s = block_sum(acc, red);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = s;
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double t = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b) t += ((volatile double *)partials)[b];
        *result = t;
        *counter = 0;
    }
}

int launch_norm(Problem *p, const void *c, int is_c128, double *partials, unsigned *counter, double *result,
                cudaStream_t st)
{
    int G = apply_grid(p);
    int n = p->set->d.size;
    if (is_c128) norm2_kernel<double2><<<G, 256, 0, st>>>((const double2 *)c, n, partials, counter, result);
    else norm2_kernel<float2><<<G, 256, 0, st>>>((const float2 *)c, n, partials, counter, result);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "norm kernel launch");
    return HX_OK;
}

}  // namespace hx
