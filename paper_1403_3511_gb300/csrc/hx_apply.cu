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
// Addressing.  One thread per output element.  The element lies in a row (fixed prefix
// k_0..k_{N-2}, contiguous in k_{N-1}); a footprint point that moves along prefix axes lies in
// row "r + offset", whose start rank comes from the row-offset table built once per potential
// (index structure only; the matrix is never formed).  Whether a point lies in K, and the fibre
// tops that select the row-table entries, follow from products of (1 + k_l) and floor(B / x).
#include <math.h>

#include <algorithm>

#include "hx_internal.h"
#include "hx_stencil.cuh"

namespace hx {

// Address of element k + s e_a + s2 e_b (footprint position pos of the operator); the point lies in K.
__device__ __forceinline__ int point_addr(const Ctx &c, const Elem &el, const OpSet &O, const Op &op, int pos,
                                          int a, int s, int b, int s2)
{
    const int N = c.S->N;
    const int di = O.didx[op.dbase + pos];
    const int shift = (a == N - 1 ? s : 0) + (b == N - 1 ? s2 : 0);
    return (di ? c.start(el, di, true) : el.e - el.j) + el.j + shift;
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
    const int ka = c.k(el, a);
    const int other = exact_div(el.qall, 1 + ka);
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
    const int ka = c.k(el, a), kb = c.k(el, b);
    const int rab = exact_div(el.qall, (1 + ka) * (1 + kb));
    const R wAB = rconst<R>(O.wAB, O.wAB32), wBA = rconst<R>(O.wBA, O.wBA32);
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

// ---- general downward-closed sets: membership and fibre tops from the row tables ----------
//
// A footprint point's row is reached through its row-offset column (every position of the
// operator's (2p+1)(2q+1) grid has one for a general set) and Ctx::member decides whether the point
// lies in K; the distance to a fibre top along axis a is the number of t = 1..p for which the point
// moved by t along a still lies in K.

// whether the point at grid position (u, v) of op lies in K (u along a, v along b; b = -1 for a
// line op), and its address (the own element when not)
__device__ __forceinline__ bool point_g(const Ctx &c, const Elem &el, const OpSet &O, const Op &op, int u, int v,
                                        int &addr)
{
    const int N = c.S->N;
    const int q = op.kind == 2 ? op.q : 0;
    const int d = O.didx[op.dbase + (u + op.p) * (2 * q + 1) + (v + q)];
    const int sh = (op.a == N - 1 ? u : 0) + (op.kind == 2 && op.b == N - 1 ? v : 0);
    int start;
    const bool ok = c.member(el, d, sh, start);
    addr = ok ? start + el.j + sh : el.e;
    return ok;
}

template <typename R, int MP, bool UNROLL>
__device__ __forceinline__ void line_op_g(const Ctx &c, const Elem &el, const OpSet &O, const Op &op, const R *tab,
                                          const typename Vec2<R>::T *cin, R &sx, R &sy)
{
    const int p = op.p;
    const int ka = c.k(el, op.a);
    int d = 0, addr;
#pragma unroll(UNROLL ? MP : 1)
    for (int t = 1; t <= MP; ++t)
        if (t <= p && point_g(c, el, O, op, t, 0, addr)) d = t;
    const R *row = tab + op.tabP + ((size_t)ka * (p + 1) + d) * (2 * p + 1) + p;
#pragma unroll(UNROLL ? 2 * MP + 1 : 1)
    for (int s = -MP; s <= MP; ++s) {
        if (s < -p || s > p || !((op.pmask >> (s + p)) & 1)) continue;
        if (!point_g(c, el, O, op, s, 0, addr)) continue;
        const typename Vec2<R>::T v = cin[addr];
        const R w = row[s];
        sx += w * v.x;
        sy += w * v.y;
    }
}

template <typename R, int MP, int MQ, bool UNROLL>
__device__ __forceinline__ void plane_op_g(const Ctx &c, const Elem &el, const OpSet &O, const Op &op, const R *tab,
                                           const typename Vec2<R>::T *cin, R &sx, R &sy)
{
    const int p = op.p, q = op.q;
    const int ka = c.k(el, op.a), kb = c.k(el, op.b);
    const R wAB = rconst<R>(O.wAB, O.wAB32), wBA = rconst<R>(O.wBA, O.wBA32);
    int addr;
    // fibre-top distances: along a at k + s2 e_b, along b at k + s e_a (0 when that point is not in K)
    int dA[2 * MQ + 1], dB[2 * MP + 1];
#pragma unroll(UNROLL ? 2 * MQ + 1 : 1)
    for (int s2 = -MQ; s2 <= MQ; ++s2) {
        int d = 0;
        if (s2 >= -q && s2 <= q)
            for (int t = 1; t <= p; ++t)
                if (point_g(c, el, O, op, t, s2, addr)) d = t;
        dA[s2 + MQ] = d;
    }
#pragma unroll(UNROLL ? 2 * MP + 1 : 1)
    for (int s = -MP; s <= MP; ++s) {
        int d = 0;
        if (s >= -p && s <= p)
            for (int t = 1; t <= q; ++t)
                if (point_g(c, el, O, op, s, t, addr)) d = t;
        dB[s + MP] = d;
    }
    const int dA0 = dA[MQ], dB0 = dB[MP];
    const R *rowP0 = tab + op.tabP + ((size_t)ka * (p + 1) + dA0) * (2 * p + 1) + p;
    const R *rowQ0 = tab + op.tabQ + ((size_t)kb * (q + 1) + dB0) * (2 * q + 1) + q;
#pragma unroll(UNROLL ? 2 * MP + 1 : 1)
    for (int s = -MP; s <= MP; ++s) {
        if (s < -p || s > p || !((op.pmask >> (s + p)) & 1) || ka + s < 0) continue;
        const bool inA = s == 0 || point_g(c, el, O, op, s, 0, addr);   // k + s e_a in K
        const R pj = inA ? rowP0[s] : (R)0;
        const R *rowQs = tab + op.tabQ + ((size_t)kb * (q + 1) + dB[s + MP]) * (2 * q + 1) + q;
#pragma unroll(UNROLL ? 2 * MQ + 1 : 1)
        for (int s2 = -MQ; s2 <= MQ; ++s2) {
            if (s2 < -q || s2 > q || !((op.qmask >> (s2 + q)) & 1) || kb + s2 < 0) continue;
            if (!point_g(c, el, O, op, s, s2, addr)) continue;              // footprint point not in K
            const R cab = inA ? pj * rowQs[s2] : (R)0;                      // P(X_a) (Q(X_b) c)
            R cba = (R)0;                                                   // Q(X_b) (P(X_a) c)
            if (s2 <= dB0) {
                const R *rowPs = tab + op.tabP + ((size_t)ka * (p + 1) + dA[s2 + MQ]) * (2 * p + 1) + p;
                cba = rowQ0[s2] * rowPs[s];
            }
            const R w = wAB * cab + wBA * cba;
            const typename Vec2<R>::T v = cin[addr];
            sx += w * v.x;
            sy += w * v.y;
        }
    }
}

template <typename R, int P, int Q, int SB>
__device__ __forceinline__ void plane_dispatch_sb(int rb, const Ctx &c, const Elem &el, const OpSet &O, const Op &op,
                                                  const R *tab, const typename Vec2<R>::T *src, typename Vec2<R>::T &s,
                                                  typename Vec2<R>::T &l)
{
    if (rb == ROLE_LAST) plane_role<R, P, Q, ROLE_LAST, SB>(c, el, O, op, tab, src, s, l);
    else plane_role<R, P, Q, ROLE_ROW, SB>(c, el, O, op, tab, src, s, l);
}

// sb: degree of the merged line op (0: none); only sb in {0, Q, Q + 2 <= 3} occurs.
template <typename R, int P, int Q>
__device__ __forceinline__ void plane_dispatch(int rb, int sb, const Ctx &c, const Elem &el, const OpSet &O, const Op &op,
                                               const R *tab, const typename Vec2<R>::T *src, typename Vec2<R>::T &s,
                                               typename Vec2<R>::T &l)
{
    if (sb == 0) plane_dispatch_sb<R, P, Q, 0>(rb, c, el, O, op, tab, src, s, l);
    else if (sb == Q) plane_dispatch_sb<R, P, Q, Q>(rb, c, el, O, op, tab, src, s, l);
    else if (Q + 2 <= 3) plane_dispatch_sb<R, P, Q, (Q + 2 <= 3 ? Q + 2 : Q)>(rb, c, el, O, op, tab, src, s, l);
}

template <typename R, int P>
__device__ __forceinline__ typename Vec2<R>::T line_dispatch(int ra, const Ctx &c, const Elem &el, const OpSet &O,
                                                             const Op &op, const R *tab, const typename Vec2<R>::T *src)
{
    if (ra == ROLE_LAST) return line_role<R, P, ROLE_LAST>(c, el, O, op, tab, src);
    return line_role<R, P, ROLE_ROW>(c, el, O, op, tab, src);
}

// MD: largest polynomial degree of the compiled potential (3: unrolled stencils; kMaxDeg: rolled loops).
// The operator list is read from the launch arguments and dispatched per operator; the kernels
// compiled at run time for one potential (hx_jit.cu) replace this loop by the fixed sequence.
// The operator list of args at one element, dispatched per operator (the kernels compiled for one
// potential replace this loop by the fixed sequence).  MD: largest polynomial degree (3: unrolled
// stencils; kMaxDeg: rolled loops); GENERAL: a general index set (membership from the row tables).
template <typename R, int MD, bool GENERAL>
__device__ __forceinline__ void generic_ops(const ApplyArgs &args, const Ctx &ctx, const Elem &el, Acc<R> &acc,
                                            const R *sm_w, const typename Vec2<R>::T *cin, const R *tab)
{
    using V = typename Vec2<R>::T;
    const OpSet &O = args.ops;
    const int e = el.e;
    for (int o = 0; o < O.nops; ++o) {
        const Op &op = O.op[o];
        if (op.merged) continue;
        R lx = (R)0, ly = (R)0;     // sum of a line op merged into a plane op
        const V *src = op.src < 0 ? cin : (const V *)args.chan + (size_t)op.src * args.chan_ld;
        R sx = (R)0, sy = (R)0;
        if (op.kind == 0) {
            const V cs = src[e];
            sx = cs.x;
            sy = cs.y;
        } else if (GENERAL) {
            if (op.kind == 1) line_op_g<R, (MD <= 3 ? 3 : kMaxDeg), (MD <= 3)>(ctx, el, O, op, tab, src, sx, sy);
            else plane_op_g<R, (MD <= 3 ? 3 : kMaxDeg), (MD <= 3 ? 3 : kMaxDeg), (MD <= 3)>(ctx, el, O, op, tab, src, sx, sy);
        } else if (MD <= 3) {
            const int sb = op.mergeB >= 0 ? O.op[op.mergeB].p : 0;
            V o = czero<V>(), l = czero<V>();
            switch (op.cls) {
                case CLS_LINE + 1: o = line_dispatch<R, 1>(op.ra, ctx, el, O, op, tab, src); break;
                case CLS_LINE + 2: o = line_dispatch<R, 2>(op.ra, ctx, el, O, op, tab, src); break;
                case CLS_LINE + 3: o = line_dispatch<R, 3>(op.ra, ctx, el, O, op, tab, src); break;
                case CLS_PLANE + 0: plane_dispatch<R, 1, 1>(op.rb, sb, ctx, el, O, op, tab, src, o, l); break;
                case CLS_PLANE + 3: plane_dispatch<R, 2, 1>(op.rb, sb, ctx, el, O, op, tab, src, o, l); break;
                case CLS_PLANE + 1: plane_dispatch<R, 1, 2>(op.rb, sb, ctx, el, O, op, tab, src, o, l); break;
                case CLS_PLANE + 4: plane_dispatch<R, 2, 2>(op.rb, sb, ctx, el, O, op, tab, src, o, l); break;
                default:
                    if (op.kind == 1) line_op<R, 3, true>(ctx, el, O, op, tab, src, sx, sy);
                    else plane_op<R, 3, 3, true>(ctx, el, O, op, tab, src, sx, sy);
                    o = V{sx, sy};
            }
            sx = o.x;
            sy = o.y;
            lx = l.x;
            ly = l.y;
        } else {
            if (op.kind == 1) line_op<R, kMaxDeg, false>(ctx, el, O, op, tab, src, sx, sy);
            else plane_op<R, kMaxDeg, kMaxDeg, false>(ctx, el, O, op, tab, src, sx, sy);
        }
        const R w = sm_w[o];
        if (op.mergeB >= 0) {
            const R wl = sm_w[op.mergeB];
            acc.add(w * sx + wl * lx, w * sy + wl * ly);
            continue;
        }
        if (args.stage1) {
            V ch;
            ch.x = w * sx;
            ch.y = w * sy;
            ((V *)args.chan)[(size_t)op.dst * args.chan_ld + e] = ch;
        } else {
            acc.add(w * sx, w * sy);
        }
    }
}

template <typename R, int MD, bool GENERAL>
__global__ void __launch_bounds__(kApplyThreads, MD <= 3 ? 3 : 1) apply_kernel(const __grid_constant__ ApplyArgs args)
{
    using V = typename Vec2<R>::T;
    apply_elements<R>(args, [&](const Ctx &ctx, const Elem &el, Acc<R> &acc, const R *sm_w, const V *cin, const R *tab) {
        generic_ops<R, MD, GENERAL>(args, ctx, el, acc, sm_w, cin, tab);
    });
}

// ---------------------------------------------------------------------------------------
// One product launch for a batch of independent problems (the Lanczos products of a batch step):
// persistent blocks take tiles of consecutive elements of any member from one queue, largest
// members first, and evaluate them with the member's launch arguments (kept in device memory) and
// the generic operator loop.  A block stops taking tiles once its clock64 budget is spent (budget
// < 0: none) and then flags the queue; nothing waits on anything, so an exhausted budget leaves an
// incomplete product and a flag, never a stalled kernel.  The last block to leave resets the queue.
// ---------------------------------------------------------------------------------------
template <typename R, int MD>
__global__ void __launch_bounds__(kApplyThreads, MD <= 3 ? 3 : 1)
batch_apply_kernel(const ApplyArgs *margs, const int2 *tiles, int ntiles, int tile, long long budget, BatchQueue *q)
{
    using V = typename Vec2<R>::T;
    __shared__ int sh_tile;
    __shared__ R sm_w[kMaxOps];
    const long long t0 = clock64();
    for (;;) {
        if (threadIdx.x == 0) {
            int t = -1;
            if (budget >= 0 && clock64() - t0 >= budget) q->timeout = 1;
            else t = (int)atomicAdd(&q->next, 1u);
            sh_tile = t;
        }
        __syncthreads();
        const int t = sh_tile;
        if (t < 0 || t >= ntiles) break;
        const int2 tl = tiles[t];
        const ApplyArgs &args = margs[tl.x];
        if ((int)threadIdx.x < args.ops.nops)
            sm_w[threadIdx.x] = op_weight<R>(args.ops.op[threadIdx.x], *args.t_ptr + args.t_shift, args.pw_values);
        __syncthreads();
        Ctx ctx;
        ctx.S = &args.S;
        ctx.mv = args.mv;
        const R oscale = args.out_scale ? (R)(*args.out_scale) : (R)1;
        const int end = min(tl.y + tile, args.S.size);
        auto body = [&](const Ctx &c, const Elem &el, Acc<R> &acc, const R *w, const V *cin, const R *tab) {
            generic_ops<R, MD, false>(args, c, el, acc, w, cin, tab);
        };
        for (int e = tl.y + (int)threadIdx.x; e < end; e += blockDim.x)
            apply_element<R>(args, ctx, e, __ldg(args.S.elem + e), oscale, sm_w, body);
        __syncthreads();                     // sm_w is rewritten for the next tile
    }
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&q->done, 1u) == gridDim.x - 1) {
            q->next = 0;
            q->done = 0;
            __threadfence();
        }
    }
}

template <typename R, int MD>
static int batch_launch_t(const void *margs, const int2 *tiles, int ntiles, int tile, long long budget, void *queue,
                          int num_sms, cudaStream_t st)
{
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_apply_kernel<R, MD>, kApplyThreads, 0);
    const int grid = std::max(1, std::min(num_sms * std::max(per_sm, 1), ntiles));
    batch_apply_kernel<R, MD><<<grid, kApplyThreads, 0, st>>>((const ApplyArgs *)margs, tiles, ntiles, tile, budget,
                                                               (BatchQueue *)queue);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "batch product kernel launch");
    return HX_OK;
}

int launch_batch_apply(bool c64, int md, const void *margs, const int2 *tiles, int ntiles, int tile, long long budget,
                       void *queue, int num_sms, cudaStream_t st)
{
    if (c64) return md <= 3 ? batch_launch_t<float, 3>(margs, tiles, ntiles, tile, budget, queue, num_sms, st)
                            : batch_launch_t<float, kMaxDeg>(margs, tiles, ntiles, tile, budget, queue, num_sms, st);
    return md <= 3 ? batch_launch_t<double, 3>(margs, tiles, ntiles, tile, budget, queue, num_sms, st)
                   : batch_launch_t<double, kMaxDeg>(margs, tiles, ntiles, tile, budget, queue, num_sms, st);
}

int apply_grid(const Problem *p)
{
    const int per_sm = 4;
    const int blocks = (p->set->d.size + kApplyThreads - 1) / kApplyThreads;
    const int g = p->num_sms * per_sm;
    return blocks < g ? (blocks > 0 ? blocks : 1) : g;
}

// Launch arguments of a batch member's Lanczos product: y = *in_scale * A(*t_ptr + t_shift) cin into
// cout, main stage, no fused projections.
int batch_member_args(Problem *p, const void *cin, void *cout, const double *t_ptr, double t_shift,
                      const double *in_scale, void *out)
{
    ApplyArgs &a = *(ApplyArgs *)out;
    memset(&a, 0, sizeof(a));
    a.S = p->set->d;
    a.gnb = p->gnb;
    a.gnbn = p->gnbn;
    a.gstride = p->gstride;
    a.dscale = p->scale * p->scale;
    a.dscale32 = (float)a.dscale;
    memcpy(a.mv, p->roff.mv, sizeof(a.mv));
    a.t_ptr = t_ptr;
    a.t_shift = t_shift;
    a.pw_values = p->pw_values;
    a.tab = p->tab;
    a.ops = p->ops;
    a.cin = cin;
    a.cout = cout;
    a.out_scale = in_scale;
    a.chan = p->chan;
    a.chan_ld = p->chan_ld;
    a.skip_diag = p->skip_diag;
    return HX_OK;
}

size_t apply_args_size() { return sizeof(ApplyArgs); }

template <typename R, int MD>
static int launch_apply_t(Problem *p, const OpSet &ops, int stage1, const void *cin, void *cout,
                          const double *t_ptr, double t_shift, const ApplyFuse *fuse, cudaStream_t st,
                          void *cout2 = nullptr, double t_shift2 = 0.0, const void *cin2 = nullptr,
                          double mag_g = 0.0)
{
    ApplyArgs a;
    memset(&a, 0, sizeof(a));
    a.S = p->set->d;
    a.gnb = p->gnb;
    a.gnbn = p->gnbn;
    a.gstride = p->gstride;
    a.dscale = p->scale * p->scale;
    a.dscale32 = (float)a.dscale;
    memcpy(a.mv, p->roff.mv, sizeof(a.mv));
    a.t_ptr = t_ptr;
    a.t_shift = t_shift;
    a.pw_values = p->pw_values;
    a.tab = p->tab;
    a.ops = ops;
    a.cin = cin;
    a.cout = cout;
    a.out_scale = fuse ? fuse->in_scale : nullptr;
    if (fuse && fuse->dvec) {
        if (stage1 || !apply_fuses_dots(p) || fuse->dk < 0 || fuse->dk >= kMaxFusedDots) {
            set_error("projections requested from a product kernel that cannot compute them");
            return HX_EUNSUPPORTED;
        }
        a.dvec = fuse->dvec;
        a.dld = fuse->dld;
        a.dk = fuse->dk;
        a.dm_used = fuse->m_used;
        a.ds = fuse->s;
        a.dh = fuse->h;
        a.dpartials = fuse->partials;
        a.dcounter = fuse->counter;
    } else if (fuse && fuse->rq) {
        if (stage1 || !apply_fuses_dots(p)) {
            set_error("a Rayleigh quotient requested from a product kernel that cannot compute it");
            return HX_EUNSUPPORTED;
        }
        a.drq = 1;
        a.ds = fuse->s;
        a.dh = fuse->h;
        a.dpartials = fuse->partials;
        a.dcounter = fuse->counter;
    }
    a.chan = p->chan;
    a.chan_ld = p->chan_ld;
    a.stage1 = stage1;
    a.skip_diag = p->skip_diag;
    a.cout2 = cout2;
    a.cin2 = cin2;
    a.t_shift2 = t_shift2;
    a.mag_g = mag_g;
    a.mag_g32 = (float)mag_g;
    const int blocks = (p->set->d.size + kApplyThreads - 1) / kApplyThreads;
    if (p->jit && !g_batch_capture && (!stage1 || jit_has_stage1(p))) {   // the potential's specialised kernel
        a.tops = p->tops;
        a.tops_words = p->tops ? jit_tops_words(p) : 0;
        return jit_launch(p, &a, blocks, st);
    }
    if (cout2) {
        set_error("internal: a two-time product needs the specialised kernel");
        return HX_EUNSUPPORTED;
    }
    int per_sm = 1;
    const bool general = p->set->d.general != 0;
    if (general) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, apply_kernel<R, MD, true>, kApplyThreads, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, apply_kernel<R, MD, false>, kApplyThreads, 0);
    int grid = p->num_sms * (per_sm > 0 ? per_sm : 1);     // one wave of resident CTAs
    if (grid > blocks) grid = blocks > 0 ? blocks : 1;
    if (general) apply_kernel<R, MD, true><<<grid, kApplyThreads, 0, st>>>(a);
    else apply_kernel<R, MD, false><<<grid, kApplyThreads, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "apply kernel launch");
    return HX_OK;
}

static int launch_stage(Problem *p, const OpSet &ops, int stage1, const void *cin, void *cout, const double *t_ptr,
                        double t_shift, const ApplyFuse *scale, cudaStream_t st)
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

int max_degree(const Problem *p)
{
    int md = 0;
    for (int i = 0; i < p->ops.nops; ++i) md = max(md, max(p->ops.op[i].p, p->ops.op[i].q));
    return md;
}

bool apply_dual(const Problem *p) { return p->jit && !g_batch_capture && p->ops1.nops == 0; }

int launch_apply_dual(Problem *p, const void *cin, void *cout, void *cout2, const double *t_ptr, double t_shift,
                      double t_shift2, const ApplyFuse *fuse, cudaStream_t st)
{
    if (!apply_dual(p)) {
        int rc = launch_apply(p, cin, cout, t_ptr, t_shift, fuse, st);
        return rc ? rc : launch_apply(p, cin, cout2, t_ptr, t_shift2, fuse, st);
    }
    return p->cfg.dtype == HX_C64
               ? launch_apply_t<float, 3>(p, p->ops, 0, cin, cout, t_ptr, t_shift, fuse, st, cout2, t_shift2)
               : launch_apply_t<double, 3>(p, p->ops, 0, cin, cout, t_ptr, t_shift, fuse, st, cout2, t_shift2);
}

int launch_apply_pair(Problem *p, const void *cin, void *cout, double t_shift, const void *cin2, void *cout2,
                      double t_shift2, const double *t_ptr, cudaStream_t st, void *mag_out, double mag_g)
{
    if (!apply_dual(p)) {
        int rc = launch_apply(p, cin, cout, t_ptr, t_shift, nullptr, st);
        return rc ? rc : launch_apply(p, cin2, cout2, t_ptr, t_shift2, nullptr, st);
    }
    // with mag_out: the kernel writes the Magnus combination there and neither product
    void *o1 = mag_out ? mag_out : cout;
    const double g = mag_out ? mag_g : 0.0;
    return p->cfg.dtype == HX_C64
               ? launch_apply_t<float, 3>(p, p->ops, 0, cin, o1, t_ptr, t_shift, nullptr, st, cout2, t_shift2, cin2, g)
               : launch_apply_t<double, 3>(p, p->ops, 0, cin, o1, t_ptr, t_shift, nullptr, st, cout2, t_shift2, cin2, g);
}

bool apply_fuses_dots(const Problem *p)
{
    return p->jit && !g_batch_capture && p->ops1.nops == 0 && p->cfg.dtype == HX_C64;
}

int launch_apply(Problem *p, const void *cin, void *cout, const double *t_ptr, double t_shift, const ApplyFuse *fuse,
                 cudaStream_t st)
{
    if (p->ops1.nops > 0) {
        int rc = launch_stage(p, p->ops1, 1, cin, nullptr, t_ptr, t_shift, nullptr, st);
        if (rc) return rc;
    }
    return launch_stage(p, p->ops, 0, cin, cout, t_ptr, t_shift, fuse, st);
}

// ---------------------------------------------------------------------------------------
// Row structure on the device
// ---------------------------------------------------------------------------------------

// Per-element record: the row holding rank e (largest r with start(r) <= e), its group, the
// product of (1 + k_l) with the coordinate sum above it, and k_{N-1} with the row length above it
// (all four below 2^16 since B < 2^16).
__global__ void elem_info_kernel(DevSet S, int4 *elem)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < S.size; e += gridDim.x * blockDim.x) {
        int lo = 0, hi = S.nrow - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (S.rstart[mid] <= e) lo = mid; else hi = mid - 1;
        }
        const int4 ri = S.row_info[lo];
        const int k2 = e - ri.x;
        const unsigned qall = (unsigned)(ri.y * (1 + k2)), ksum = (unsigned)(ri.z + k2);
        elem[e] = make_int4(lo, S.rgrp[lo], (int)(qall | (ksum << 16)), (int)((unsigned)k2 | ((unsigned)ri.w << 16)));
    }
}

int launch_elem_info(const IndexSetObj *s)
{
    int blocks = (int)std::min<int64_t>((s->h.size + 255) / 256, 8192);
    elem_info_kernel<<<std::max(blocks, 1), 256>>>(s->d, const_cast<int4 *>(s->d.elem));
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "element record kernel");
    return HX_OK;
}

// gnb[g * gstride + m] = first row of the group whose prefix (k_0..k_{N-3}) is that of group g
// moved by outer move m, or -1 when a coordinate turns negative or the prefix product exceeds B.
// The first row of a group is the row of the prefix (k_0..k_{N-3}, 0), whose index is
// sum_{d<N-2} Q_{N-2-d}(q_d, k_d) (the rank tables one level up).
__global__ void groupnb_kernel(DevSet S, RowOffsets ro, int gstride, int *gnb)
{
    const int npre = S.N - 1, nouter = S.N - 2;
    const int64_t total = (int64_t)S.ngroup * ro.nom;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x) {
        const int g = (int)(x / ro.nom), m = (int)(x - (int64_t)g * ro.nom);
        const int a0 = ro.om[m][0], s0 = ro.om[m][1], a1 = ro.om[m][2], s1 = ro.om[m][3];
        const int r0 = S.gfirst[g];
        int q = 1, row = 0;
        bool ok = true;
        for (int l = 0; l < nouter; ++l) {
            const int kl = (int)S.row_k[(size_t)r0 * npre + l] + (l == a0 ? s0 : 0) + (l == a1 ? s1 : 0);
            if (kl < 0 || (int64_t)q * (1 + kl) > S.B) { ok = false; break; }
            row += S.Q[(size_t)(nouter - 1 - l) * S.qtotal + S.qoff[q] + kl];   // level m = N-2-l
            q *= 1 + kl;
        }
        gnb[(size_t)g * gstride + m] = ok ? row : -1;
    }
}

int launch_groupnb(const DevSet &S, const RowOffsets &ro, int gstride, int *gnb, cudaStream_t st)
{
    const int64_t total = (int64_t)ro.nom * S.ngroup;
    if (total == 0) return HX_OK;
    int blocks = (int)std::min<int64_t>((total + 255) / 256, 16384);
    groupnb_kernel<<<std::max(blocks, 1), 256, 0, st>>>(S, ro, gstride, gnb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "group-neighbour table kernel");
    return HX_OK;
}

// ---------------------------------------------------------------------------------------
// export of all multi-indices (row prefix, then the position in the row)
// ---------------------------------------------------------------------------------------
__global__ void export_kernel(DevSet S, int32_t *k)
{
    const int N = S.N, npre = N - 1;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < S.size; e += gridDim.x * blockDim.x) {
        const int r = S.elem[e].x;
        for (int l = 0; l < npre; ++l) k[(size_t)e * N + l] = S.row_k[(size_t)r * npre + l];
        k[(size_t)e * N + N - 1] = e - S.row_info[r].x;
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
        for (int b = 0; b < (int)gridDim.x; ++b) t += __ldcg(partials + b);   // L2-coherent, batched
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
