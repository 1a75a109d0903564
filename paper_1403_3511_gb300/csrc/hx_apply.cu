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
};

__device__ __forceinline__ double op_weight(const Op &op, double t, const double *pw)
{
    double f = 1.0;
    switch (op.mod) {
        case HX_MOD_COS: f = cos(op.omega * t + op.phase); break;
        case HX_MOD_SIN2: { double s = sin(op.omega * t); f = s * s; } break;
        case HX_MOD_PWCONST: {
            double x = floor((t - op.pw_t0) / (op.pw_t1 - op.pw_t0) * op.pw_n);
            int qi = x < 0.0 ? 0 : (x >= op.pw_n ? op.pw_n - 1 : (int)x);
            f = pw[op.pw_off + qi];
        } break;
        default: break;
    }
    return op.amp * f;
}

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
    const int4 *nb;           // item neighbour table (shared)
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
        int4 nb = c.nb[el.sl * c.nd + di];
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

// MD: largest polynomial degree of the compiled potential (3: unrolled stencils; kMaxDeg: rolled loops).
template <typename R, int MD>
__global__ void __launch_bounds__(kApplyThreads, MD <= 3 ? 2 : 1) apply_kernel(const __grid_constant__ ApplyArgs args)
{
    using V = typename Vec2<R>::T;
    extern __shared__ int4 sm_nb[];
    __shared__ int sm_start[65];
    __shared__ int sm_q[64];
    __shared__ uint16_t sm_pre[64 * kMaxN];
    __shared__ uint16_t sm_k[kMaxN * kApplyThreads];
    __shared__ R sm_w[kMaxOps];

    const DevSet &S = args.S;
    const OpSet &O = args.ops;
    const int N = S.N, nout = N > 2 ? N - 2 : 0, nd = O.ndelta;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const V *cin = (const V *)args.cin;
    V *cout = (V *)args.cout;
    const R *tab = (const R *)args.tab;
    const int *Q1 = S.Q;     // level m = 1

    if (tid < O.nops) sm_w[tid] = (R)op_weight(O.op[tid], *args.t_ptr + args.t_shift, args.pw_values);
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
            int4 res = make_int4(-1, 0, 0, 0);
            int pre[kMaxN];
            bool ok = true;
            for (int l = 0; l < nout; ++l) pre[l] = sm_pre[sl * kMaxN + l];
            for (int j = 0; j < 2; ++j) {
                int ax = O.delta[di][2 * j];
                if (ax >= 0) pre[ax] += O.delta[di][2 * j + 1];
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
                res = make_int4(start, (int)S.qoff[qd], qd, 0);
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
            acc.add(dj * ce.x, dj * ce.y);
            for (int o = 0; o < O.nops; ++o) {
                const Op &op = O.op[o];
                R sx = (R)0, sy = (R)0;
                if (op.kind == 0) {
                    sx = ce.x;
                    sy = ce.y;
                } else if (MD <= 3) {
                    if (op.kind == 1) {
                        if (op.p <= 1) line_op<R, 1, true>(ctx, el, O, op, tab, cin, sx, sy);
                        else line_op<R, 3, true>(ctx, el, O, op, tab, cin, sx, sy);
                    } else {
                        if (op.p <= 2 && op.q <= 1) plane_op<R, 2, 1, true>(ctx, el, O, op, tab, cin, sx, sy);
                        else if (op.p <= 2 && op.q <= 2) plane_op<R, 2, 2, true>(ctx, el, O, op, tab, cin, sx, sy);
                        else plane_op<R, 3, 3, true>(ctx, el, O, op, tab, cin, sx, sy);
                    }
                } else {
                    if (op.kind == 1) line_op<R, kMaxDeg, false>(ctx, el, O, op, tab, cin, sx, sy);
                    else plane_op<R, kMaxDeg, kMaxDeg, false>(ctx, el, O, op, tab, cin, sx, sy);
                }
                const R w = sm_w[o];
                acc.add(w * sx, w * sy);
            }
            V y = acc.get();
            y.x *= oscale;
            y.y *= oscale;
            cout[e] = y;
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
static int launch_apply_t(Problem *p, const void *cin, void *cout, const double *t_ptr, double t_shift,
                          const double *out_scale, cudaStream_t st)
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
    a.ops = p->ops;
    a.cin = cin;
    a.cout = cout;
    a.out_scale = out_scale;
    size_t smem = (size_t)p->slabs_per_item * p->ops.ndelta * sizeof(int4);
    apply_kernel<R, MD><<<apply_grid(p), kApplyThreads, smem, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "apply kernel launch");
    return HX_OK;
}

int launch_apply(Problem *p, const void *cin, void *cout, const double *t_ptr, double t_shift, const ApplyFuse *fuse,
                 cudaStream_t st)
{
    const double *scale = fuse ? fuse->in_scale : nullptr;
    int md = 0;
    for (int i = 0; i < p->ops.nops; ++i) md = max(md, max(p->ops.op[i].p, p->ops.op[i].q));
    if (p->cfg.dtype == HX_C64)
        return md <= 3 ? launch_apply_t<float, 3>(p, cin, cout, t_ptr, t_shift, scale, st)
                       : launch_apply_t<float, kMaxDeg>(p, cin, cout, t_ptr, t_shift, scale, st);
    return md <= 3 ? launch_apply_t<double, 3>(p, cin, cout, t_ptr, t_shift, scale, st)
                   : launch_apply_t<double, kMaxDeg>(p, cin, cout, t_ptr, t_shift, scale, st);
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
