// Kernel source generated by the library (csrc/hx_jit.cu) for the complex64 N=6, B=4096 Hénon-Heiles
// chain with a cos(t)-modulated dipole (the bench workload hh6_b4096), written by setting
// HX_JIT_SOURCE_DUMP=<file> for `python bench.py --no-fp64 --no-cpu-baseline` on a machine with a
// GB300.  The two-time kernels' launch bounds were then set to the
// 3 blocks per SM that the generator now writes.  tests/test_jit_source.py compiles it against the
// current csrc/hx_stencil.cuh and checks registers and spills.
#include "hx_stencil.cuh"
namespace hx {
struct ColsK0 {
    static constexpr int kA = 0, kB = 1, kN = 6;
    __device__ static constexpr int om(int x) { return x == 0 ? 0 : x == 1 ? -1 : x == 2 ? 1 : x == 3 ? -1 : x == 4 ? -1 : x == 5 ? -1 : x == 6 ? 2 : x == 7 ? -1 : x == 8 ? 3 : x == 9 ? -1 : x == 10 ? -1 : x == 11 ? -1 : x == 12 ? 4 : x == 13 ? -1 : x == 14 ? 5 : 0; }
    __device__ static constexpr int s4(int x) { return x == 0 ? 0 : x == 1 ? 0 : x == 2 ? 0 : x == 3 ? 0 : x == 4 ? 0 : x == 5 ? 0 : x == 6 ? 0 : x == 7 ? 0 : x == 8 ? 0 : x == 9 ? 0 : x == 10 ? 0 : x == 11 ? 0 : x == 12 ? 0 : x == 13 ? 0 : x == 14 ? 0 : 0; }
    __device__ static constexpr int omx(int x) { return x == 0 ? 6 : x == 1 ? 7 : 0; }
    __device__ static constexpr int s4x(int x) { return x == 0 ? 0 : x == 1 ? 0 : 0; }
    static constexpr int kGnLo = 0, kGnN = 2;
    struct Gn { int4 q[kGnN > 0 ? kGnN : 1]; };
    __device__ static __forceinline__ Gn gn_load(const Elem &el)
    {
        Gn g;
#pragma unroll
        for (int i = 0; i < kGnN; ++i) g.q[i] = __ldg(reinterpret_cast<const int4 *>(el.gn) + kGnLo + i);
        return g;
    }
    __device__ static __forceinline__ int gnv(const Gn &g, int m)
    {
        const int k = m - 4 * kGnLo;
        const int4 q = g.q[k >> 2];
        return (k & 3) == 0 ? q.x : (k & 3) == 1 ? q.y : (k & 3) == 2 ? q.z : q.w;
    }
    __device__ static __forceinline__ int start(const Ctx &c, const Elem &el, const OpSet &, const Op &, const Gn &g, int pos, bool ok)
    { return c.start_row(el, om(pos) >= 0 ? gnv(g, om(pos)) + el.k4 + s4(pos) : el.r + s4(pos), ok); }
    __device__ static __forceinline__ int startx(const Ctx &c, const Elem &el, const OpSet &, const Op &, const Gn &g, int j, int, bool ok)
    { return c.start_row(el, omx(j) >= 0 ? gnv(g, omx(j)) + el.k4 + s4x(j) : el.r + s4x(j), ok); }
    static constexpr bool kTopsBits = true;
    __device__ static constexpr int offA(int v) { return v == -1 ? 2 : v == 0 ? 0 : v == 1 ? 4 : 0; }
    __device__ static constexpr int offB(int v) { return v == -2 ? 6 : v == 0 ? 7 : v == 2 ? 9 : 0; }
    __device__ static constexpr int wB(int v) { return v == -2 ? 1 : v == 0 ? 2 : v == 2 ? 1 : 0; }
    static constexpr int wA = 2;
    __device__ static __forceinline__ int topA(const Elem &el, int v) { return top_field(el, offA(v), wA); }
    __device__ static __forceinline__ int topB(const Elem &el, int s) { return top_field(el, offB(s), wB(s)); }
};
struct ColsK2 {
    static constexpr int kA = 1, kB = 2, kN = 6;
    __device__ static constexpr int om(int x) { return x == 0 ? 8 : x == 1 ? -1 : x == 2 ? 9 : x == 3 ? -1 : x == 4 ? -1 : x == 5 ? -1 : x == 6 ? 10 : x == 7 ? -1 : x == 8 ? 11 : x == 9 ? -1 : x == 10 ? -1 : x == 11 ? -1 : x == 12 ? 12 : x == 13 ? -1 : x == 14 ? 13 : 0; }
    __device__ static constexpr int s4(int x) { return x == 0 ? 0 : x == 1 ? 0 : x == 2 ? 0 : x == 3 ? 0 : x == 4 ? 0 : x == 5 ? 0 : x == 6 ? 0 : x == 7 ? 0 : x == 8 ? 0 : x == 9 ? 0 : x == 10 ? 0 : x == 11 ? 0 : x == 12 ? 0 : x == 13 ? 0 : x == 14 ? 0 : 0; }
    __device__ static constexpr int omx(int x) { return x == 0 ? 14 : x == 1 ? 15 : 0; }
    __device__ static constexpr int s4x(int x) { return x == 0 ? 0 : x == 1 ? 0 : 0; }
    static constexpr int kGnLo = 2, kGnN = 2;
    struct Gn { int4 q[kGnN > 0 ? kGnN : 1]; };
    __device__ static __forceinline__ Gn gn_load(const Elem &el)
    {
        Gn g;
#pragma unroll
        for (int i = 0; i < kGnN; ++i) g.q[i] = __ldg(reinterpret_cast<const int4 *>(el.gn) + kGnLo + i);
        return g;
    }
    __device__ static __forceinline__ int gnv(const Gn &g, int m)
    {
        const int k = m - 4 * kGnLo;
        const int4 q = g.q[k >> 2];
        return (k & 3) == 0 ? q.x : (k & 3) == 1 ? q.y : (k & 3) == 2 ? q.z : q.w;
    }
    __device__ static __forceinline__ int start(const Ctx &c, const Elem &el, const OpSet &, const Op &, const Gn &g, int pos, bool ok)
    { return c.start_row(el, om(pos) >= 0 ? gnv(g, om(pos)) + el.k4 + s4(pos) : el.r + s4(pos), ok); }
    __device__ static __forceinline__ int startx(const Ctx &c, const Elem &el, const OpSet &, const Op &, const Gn &g, int j, int, bool ok)
    { return c.start_row(el, omx(j) >= 0 ? gnv(g, omx(j)) + el.k4 + s4x(j) : el.r + s4x(j), ok); }
    static constexpr bool kTopsBits = true;
    __device__ static constexpr int offA(int v) { return v == -1 ? 12 : v == 0 ? 10 : v == 1 ? 14 : 0; }
    __device__ static constexpr int offB(int v) { return v == -2 ? 16 : v == 0 ? 17 : v == 2 ? 19 : 0; }
    __device__ static constexpr int wB(int v) { return v == -2 ? 1 : v == 0 ? 2 : v == 2 ? 1 : 0; }
    static constexpr int wA = 2;
    __device__ static __forceinline__ int topA(const Elem &el, int v) { return top_field(el, offA(v), wA); }
    __device__ static __forceinline__ int topB(const Elem &el, int s) { return top_field(el, offB(s), wB(s)); }
};
struct ColsK4 {
    static constexpr int kA = 2, kB = 3, kN = 6;
    __device__ static constexpr int om(int x) { return x == 0 ? 16 : x == 1 ? -1 : x == 2 ? 17 : x == 3 ? -1 : x == 4 ? -1 : x == 5 ? -1 : x == 6 ? 18 : x == 7 ? -1 : x == 8 ? 19 : x == 9 ? -1 : x == 10 ? -1 : x == 11 ? -1 : x == 12 ? 20 : x == 13 ? -1 : x == 14 ? 21 : 0; }
    __device__ static constexpr int s4(int x) { return x == 0 ? 0 : x == 1 ? 0 : x == 2 ? 0 : x == 3 ? 0 : x == 4 ? 0 : x == 5 ? 0 : x == 6 ? 0 : x == 7 ? 0 : x == 8 ? 0 : x == 9 ? 0 : x == 10 ? 0 : x == 11 ? 0 : x == 12 ? 0 : x == 13 ? 0 : x == 14 ? 0 : 0; }
    __device__ static constexpr int omx(int x) { return x == 0 ? 22 : x == 1 ? 23 : 0; }
    __device__ static constexpr int s4x(int x) { return x == 0 ? 0 : x == 1 ? 0 : 0; }
    static constexpr int kGnLo = 4, kGnN = 2;
    struct Gn { int4 q[kGnN > 0 ? kGnN : 1]; };
    __device__ static __forceinline__ Gn gn_load(const Elem &el)
    {
        Gn g;
#pragma unroll
        for (int i = 0; i < kGnN; ++i) g.q[i] = __ldg(reinterpret_cast<const int4 *>(el.gn) + kGnLo + i);
        return g;
    }
    __device__ static __forceinline__ int gnv(const Gn &g, int m)
    {
        const int k = m - 4 * kGnLo;
        const int4 q = g.q[k >> 2];
        return (k & 3) == 0 ? q.x : (k & 3) == 1 ? q.y : (k & 3) == 2 ? q.z : q.w;
    }
    __device__ static __forceinline__ int start(const Ctx &c, const Elem &el, const OpSet &, const Op &, const Gn &g, int pos, bool ok)
    { return c.start_row(el, om(pos) >= 0 ? gnv(g, om(pos)) + el.k4 + s4(pos) : el.r + s4(pos), ok); }
    __device__ static __forceinline__ int startx(const Ctx &c, const Elem &el, const OpSet &, const Op &, const Gn &g, int j, int, bool ok)
    { return c.start_row(el, omx(j) >= 0 ? gnv(g, omx(j)) + el.k4 + s4x(j) : el.r + s4x(j), ok); }
    static constexpr bool kTopsBits = true;
    __device__ static constexpr int offA(int v) { return v == -1 ? 22 : v == 0 ? 20 : v == 1 ? 24 : 0; }
    __device__ static constexpr int offB(int v) { return v == -2 ? 26 : v == 0 ? 27 : v == 2 ? 29 : 0; }
    __device__ static constexpr int wB(int v) { return v == -2 ? 1 : v == 0 ? 2 : v == 2 ? 1 : 0; }
    static constexpr int wA = 2;
    __device__ static __forceinline__ int topA(const Elem &el, int v) { return top_field(el, offA(v), wA); }
    __device__ static __forceinline__ int topB(const Elem &el, int s) { return top_field(el, offB(s), wB(s)); }
};
struct ColsK6 {
    static constexpr int kA = 3, kB = 4, kN = 6;
    __device__ static constexpr int om(int x) { return x == 0 ? 24 : x == 1 ? -1 : x == 2 ? 24 : x == 3 ? -1 : x == 4 ? -1 : x == 5 ? -1 : x == 6 ? -1 : x == 7 ? -1 : x == 8 ? -1 : x == 9 ? -1 : x == 10 ? -1 : x == 11 ? -1 : x == 12 ? 25 : x == 13 ? -1 : x == 14 ? 25 : 0; }
    __device__ static constexpr int s4(int x) { return x == 0 ? -1 : x == 1 ? 0 : x == 2 ? 1 : x == 3 ? 0 : x == 4 ? 0 : x == 5 ? 0 : x == 6 ? -1 : x == 7 ? 0 : x == 8 ? 1 : x == 9 ? 0 : x == 10 ? 0 : x == 11 ? 0 : x == 12 ? -1 : x == 13 ? 0 : x == 14 ? 1 : 0; }
    __device__ static constexpr int omx(int x) { return x == 0 ? -1 : x == 1 ? -1 : 0; }
    __device__ static constexpr int s4x(int x) { return x == 0 ? -3 : x == 1 ? 3 : 0; }
    static constexpr int kGnLo = 6, kGnN = 1;
    struct Gn { int4 q[kGnN > 0 ? kGnN : 1]; };
    __device__ static __forceinline__ Gn gn_load(const Elem &el)
    {
        Gn g;
#pragma unroll
        for (int i = 0; i < kGnN; ++i) g.q[i] = __ldg(reinterpret_cast<const int4 *>(el.gn) + kGnLo + i);
        return g;
    }
    __device__ static __forceinline__ int gnv(const Gn &g, int m)
    {
        const int k = m - 4 * kGnLo;
        const int4 q = g.q[k >> 2];
        return (k & 3) == 0 ? q.x : (k & 3) == 1 ? q.y : (k & 3) == 2 ? q.z : q.w;
    }
    __device__ static __forceinline__ int start(const Ctx &c, const Elem &el, const OpSet &, const Op &, const Gn &g, int pos, bool ok)
    { return c.start_row(el, om(pos) >= 0 ? gnv(g, om(pos)) + el.k4 + s4(pos) : el.r + s4(pos), ok); }
    __device__ static __forceinline__ int startx(const Ctx &c, const Elem &el, const OpSet &, const Op &, const Gn &g, int j, int, bool ok)
    { return c.start_row(el, omx(j) >= 0 ? gnv(g, omx(j)) + el.k4 + s4x(j) : el.r + s4x(j), ok); }
    static constexpr bool kTopsBits = true;
    __device__ static constexpr int offA(int v) { return v == -1 ? 32 : v == 0 ? 30 : v == 1 ? 34 : 0; }
    __device__ static constexpr int offB(int v) { return v == -2 ? 36 : v == 0 ? 37 : v == 2 ? 39 : 0; }
    __device__ static constexpr int wB(int v) { return v == -2 ? 1 : v == 0 ? 2 : v == 2 ? 1 : 0; }
    static constexpr int wA = 2;
    __device__ static __forceinline__ int topA(const Elem &el, int v) { return top_field(el, offA(v), wA); }
    __device__ static __forceinline__ int topB(const Elem &el, int s) { return top_field(el, offB(s), wB(s)); }
};
struct ColsK8 {
    static constexpr int kA = 4, kB = 5, kN = 6;
    __device__ static constexpr int om(int x) { return x == 0 ? -1 : x == 1 ? -1 : x == 2 ? -1 : x == 3 ? -1 : x == 4 ? -1 : x == 5 ? -1 : x == 6 ? -1 : x == 7 ? -1 : x == 8 ? -1 : x == 9 ? -1 : x == 10 ? -1 : x == 11 ? -1 : x == 12 ? -1 : x == 13 ? -1 : x == 14 ? -1 : 0; }
    __device__ static constexpr int s4(int x) { return x == 0 ? -2 : x == 1 ? -2 : x == 2 ? -2 : x == 3 ? 0 : x == 4 ? 0 : x == 5 ? 0 : x == 6 ? 0 : x == 7 ? 0 : x == 8 ? 0 : x == 9 ? 0 : x == 10 ? 0 : x == 11 ? 0 : x == 12 ? 2 : x == 13 ? 2 : x == 14 ? 2 : 0; }
    __device__ static constexpr int omx(int x) { return x == 0 ? -1 : x == 1 ? -1 : 0; }
    __device__ static constexpr int s4x(int x) { return x == 0 ? 0 : x == 1 ? 0 : 0; }
    static constexpr int kGnLo = 0, kGnN = 0;
    struct Gn { int4 q[kGnN > 0 ? kGnN : 1]; };
    __device__ static __forceinline__ Gn gn_load(const Elem &el)
    {
        Gn g;
#pragma unroll
        for (int i = 0; i < kGnN; ++i) g.q[i] = __ldg(reinterpret_cast<const int4 *>(el.gn) + kGnLo + i);
        return g;
    }
    __device__ static __forceinline__ int gnv(const Gn &g, int m)
    {
        const int k = m - 4 * kGnLo;
        const int4 q = g.q[k >> 2];
        return (k & 3) == 0 ? q.x : (k & 3) == 1 ? q.y : (k & 3) == 2 ? q.z : q.w;
    }
    __device__ static __forceinline__ int start(const Ctx &c, const Elem &el, const OpSet &, const Op &, const Gn &g, int pos, bool ok)
    { return c.start_row(el, om(pos) >= 0 ? gnv(g, om(pos)) + el.k4 + s4(pos) : el.r + s4(pos), ok); }
    __device__ static __forceinline__ int startx(const Ctx &c, const Elem &el, const OpSet &, const Op &, const Gn &g, int j, int, bool ok)
    { return c.start_row(el, omx(j) >= 0 ? gnv(g, omx(j)) + el.k4 + s4x(j) : el.r + s4x(j), ok); }
    static constexpr bool kTopsBits = true;
    __device__ static constexpr int offA(int v) { return v == -1 ? 42 : v == 0 ? 40 : v == 1 ? 44 : 0; }
    __device__ static constexpr int offB(int v) { return v == -2 ? 46 : v == 0 ? 47 : v == 2 ? 49 : 0; }
    __device__ static constexpr int wB(int v) { return v == -2 ? 1 : v == 0 ? 2 : v == 2 ? 1 : 0; }
    static constexpr int wA = 2;
    __device__ static __forceinline__ int topA(const Elem &el, int v) { return top_field(el, offA(v), wA); }
    __device__ static __forceinline__ int topB(const Elem &el, int s) { return top_field(el, offB(s), wB(s)); }
};
struct ColsK10 {
    static constexpr int kA = 0, kB = -1, kN = 6;
    __device__ static constexpr int om(int x) { return x == 0 ? 26 : x == 1 ? -1 : x == 2 ? 27 : 0; }
    __device__ static constexpr int s4(int x) { return x == 0 ? 0 : x == 1 ? 0 : x == 2 ? 0 : 0; }
    __device__ static constexpr int omx(int) { return -1; }
    __device__ static constexpr int s4x(int) { return 0; }
    static constexpr int kGnLo = 6, kGnN = 1;
    struct Gn { int4 q[kGnN > 0 ? kGnN : 1]; };
    __device__ static __forceinline__ Gn gn_load(const Elem &el)
    {
        Gn g;
#pragma unroll
        for (int i = 0; i < kGnN; ++i) g.q[i] = __ldg(reinterpret_cast<const int4 *>(el.gn) + kGnLo + i);
        return g;
    }
    __device__ static __forceinline__ int gnv(const Gn &g, int m)
    {
        const int k = m - 4 * kGnLo;
        const int4 q = g.q[k >> 2];
        return (k & 3) == 0 ? q.x : (k & 3) == 1 ? q.y : (k & 3) == 2 ? q.z : q.w;
    }
    __device__ static __forceinline__ int start(const Ctx &c, const Elem &el, const OpSet &, const Op &, const Gn &g, int pos, bool ok)
    { return c.start_row(el, om(pos) >= 0 ? gnv(g, om(pos)) + el.k4 + s4(pos) : el.r + s4(pos), ok); }
    __device__ static __forceinline__ int startx(const Ctx &c, const Elem &el, const OpSet &, const Op &, const Gn &g, int j, int, bool ok)
    { return c.start_row(el, omx(j) >= 0 ? gnv(g, omx(j)) + el.k4 + s4x(j) : el.r + s4x(j), ok); }
    static constexpr bool kTopsBits = true;
    static constexpr int offT = 50, wT = 1;
    __device__ static __forceinline__ int lineTop(const Elem &el) { return top_field(el, offT, wT); }
};
using R = float;
using V = Vec2<R>::T;
__device__ __forceinline__ void ops(const ApplyArgs &args, const Ctx &ctx, const Elem &el, Acc<R> &acc,
                                    const R *sm_w, const V *cin, const R *tab)
{
    const OpSet &O = args.ops;
    { V o, l;
      plane_role<R, 2, 1, ROLE_ROW, 3, 3, ColsK0>(ctx, el, O, O.op[0], tab, cin, o, l);
      acc.add(cmad(sm_w[1], l, cscale(sm_w[0], o))); }
    { V o, l;
      plane_role<R, 2, 1, ROLE_ROW, 3, 3, ColsK2>(ctx, el, O, O.op[2], tab, cin, o, l);
      acc.add(cmad(sm_w[3], l, cscale(sm_w[2], o))); }
    { V o, l;
      plane_role<R, 2, 1, ROLE_ROW, 3, 3, ColsK4>(ctx, el, O, O.op[4], tab, cin, o, l);
      acc.add(cmad(sm_w[5], l, cscale(sm_w[4], o))); }
    { V o, l;
      plane_role<R, 2, 1, ROLE_ROW, 3, 3, ColsK6>(ctx, el, O, O.op[6], tab, cin, o, l);
      acc.add(cmad(sm_w[7], l, cscale(sm_w[6], o))); }
    { V o, l;
      plane_role<R, 2, 1, ROLE_LAST, 3, 3, ColsK8>(ctx, el, O, O.op[8], tab, cin, o, l);
      acc.add(cmad(sm_w[9], l, cscale(sm_w[8], o))); }
    { const V o = line_role<R, 1, ROLE_ROW, ColsK10>(ctx, el, O, O.op[10], tab, cin);
      acc.add(cscale(sm_w[10], o)); }
}
__device__ __forceinline__ void ops_dual(const ApplyArgs &args, const Ctx &ctx, const Elem &el, Acc<R> &acc,
                                         Acc<R> &acc2, const R *sm_w, const R *sm_w2, const V *cin, const R *tab)
{
    const OpSet &O = args.ops;
    { V o, l;
      plane_role<R, 2, 1, ROLE_ROW, 3, 3, ColsK0>(ctx, el, O, O.op[0], tab, cin, o, l);
      acc.add(cmad(sm_w[1], l, cscale(sm_w[0], o)));
      acc2.add(cmad(sm_w2[1], l, cscale(sm_w2[0], o))); }
    { V o, l;
      plane_role<R, 2, 1, ROLE_ROW, 3, 3, ColsK2>(ctx, el, O, O.op[2], tab, cin, o, l);
      acc.add(cmad(sm_w[3], l, cscale(sm_w[2], o)));
      acc2.add(cmad(sm_w2[3], l, cscale(sm_w2[2], o))); }
    { V o, l;
      plane_role<R, 2, 1, ROLE_ROW, 3, 3, ColsK4>(ctx, el, O, O.op[4], tab, cin, o, l);
      acc.add(cmad(sm_w[5], l, cscale(sm_w[4], o)));
      acc2.add(cmad(sm_w2[5], l, cscale(sm_w2[4], o))); }
    { V o, l;
      plane_role<R, 2, 1, ROLE_ROW, 3, 3, ColsK6>(ctx, el, O, O.op[6], tab, cin, o, l);
      acc.add(cmad(sm_w[7], l, cscale(sm_w[6], o)));
      acc2.add(cmad(sm_w2[7], l, cscale(sm_w2[6], o))); }
    { V o, l;
      plane_role<R, 2, 1, ROLE_LAST, 3, 3, ColsK8>(ctx, el, O, O.op[8], tab, cin, o, l);
      acc.add(cmad(sm_w[9], l, cscale(sm_w[8], o)));
      acc2.add(cmad(sm_w2[9], l, cscale(sm_w2[8], o))); }
    { const V o = line_role<R, 1, ROLE_ROW, ColsK10>(ctx, el, O, O.op[10], tab, cin);
      acc.add(cscale(sm_w[10], o)); acc2.add(cscale(sm_w2[10], o)); }
}
__device__ __forceinline__ void ops_pair(const ApplyArgs &args, const Ctx &ctx, const Elem &el, Acc<R> &acc,
                                         Acc<R> &acc2, const R *sm_w, const R *sm_w2, const V *cin,
                                         const V *cin2, const R *tab)
{
    const OpSet &O = args.ops;
    { const V *sr[2] = {cin, cin2}; V o[2], l[2];
      plane_role_n<R, 2, 1, ROLE_ROW, 3, 2, 3, ColsK0>(ctx, el, O, O.op[0], tab, sr, o, l);
      acc.add(cmad(sm_w[1], l[0], cscale(sm_w[0], o[0])));
      acc2.add(cmad(sm_w2[1], l[1], cscale(sm_w2[0], o[1]))); }
    { const V *sr[2] = {cin, cin2}; V o[2], l[2];
      plane_role_n<R, 2, 1, ROLE_ROW, 3, 2, 3, ColsK2>(ctx, el, O, O.op[2], tab, sr, o, l);
      acc.add(cmad(sm_w[3], l[0], cscale(sm_w[2], o[0])));
      acc2.add(cmad(sm_w2[3], l[1], cscale(sm_w2[2], o[1]))); }
    { const V *sr[2] = {cin, cin2}; V o[2], l[2];
      plane_role_n<R, 2, 1, ROLE_ROW, 3, 2, 3, ColsK4>(ctx, el, O, O.op[4], tab, sr, o, l);
      acc.add(cmad(sm_w[5], l[0], cscale(sm_w[4], o[0])));
      acc2.add(cmad(sm_w2[5], l[1], cscale(sm_w2[4], o[1]))); }
    { const V *sr[2] = {cin, cin2}; V o[2], l[2];
      plane_role_n<R, 2, 1, ROLE_ROW, 3, 2, 3, ColsK6>(ctx, el, O, O.op[6], tab, sr, o, l);
      acc.add(cmad(sm_w[7], l[0], cscale(sm_w[6], o[0])));
      acc2.add(cmad(sm_w2[7], l[1], cscale(sm_w2[6], o[1]))); }
    { const V *sr[2] = {cin, cin2}; V o[2], l[2];
      plane_role_n<R, 2, 1, ROLE_LAST, 3, 2, 3, ColsK8>(ctx, el, O, O.op[8], tab, sr, o, l);
      acc.add(cmad(sm_w[9], l[0], cscale(sm_w[8], o[0])));
      acc2.add(cmad(sm_w2[9], l[1], cscale(sm_w2[8], o[1]))); }
    { const V *sr[2] = {cin, cin2}; V o[2];
      line_role_n<R, 1, ROLE_ROW, 2, ColsK10>(ctx, el, O, O.op[10], tab, sr, o);
      acc.add(cscale(sm_w[10], o[0])); acc2.add(cscale(sm_w2[10], o[1])); }
}
}  // namespace hx
extern "C" __global__ void __launch_bounds__(hx::kApplyThreads, 4)
hx_apply_specialised(const __grid_constant__ hx::ApplyArgs args)
{
    hx::apply_elements<hx::R>(args, [&](const hx::Ctx &ctx, const hx::Elem &el, hx::Acc<hx::R> &acc,
                                        const hx::R *sm_w, const hx::V *cin, const hx::R *tab) {
        hx::ops(args, ctx, el, acc, sm_w, cin, tab);
    });
}
extern "C" __global__ void __launch_bounds__(hx::kApplyThreads, 3)
hx_apply_specialised_dual(const __grid_constant__ hx::ApplyArgs args)
{
    hx::apply_elements_dual<hx::R>(args, [&](const hx::Ctx &ctx, const hx::Elem &el, hx::Acc<hx::R> &acc,
                                             hx::Acc<hx::R> &acc2, const hx::R *sm_w, const hx::R *sm_w2,
                                             const hx::V *cin, const hx::V *, const hx::R *tab) {
        hx::ops_dual(args, ctx, el, acc, acc2, sm_w, sm_w2, cin, tab);
    });
}
extern "C" __global__ void __launch_bounds__(hx::kApplyThreads, 3)
hx_apply_specialised_pair(const __grid_constant__ hx::ApplyArgs args)
{
    hx::apply_elements_dual<hx::R>(args, [&](const hx::Ctx &ctx, const hx::Elem &el, hx::Acc<hx::R> &acc,
                                             hx::Acc<hx::R> &acc2, const hx::R *sm_w, const hx::R *sm_w2,
                                             const hx::V *cin, const hx::V *cin2, const hx::R *tab) {
        hx::ops_pair(args, ctx, el, acc, acc2, sm_w, sm_w2, cin, cin2, tab);
    });
}
extern "C" __global__ void __launch_bounds__(hx::kApplyThreads)
hx_apply_tops(const __grid_constant__ hx::ApplyArgs args)
{
    using namespace hx;
    Ctx ctx;
    ctx.S = &args.S;
    ctx.mv = args.mv;
    const OpSet &O = args.ops;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < args.S.size; e += gridDim.x * blockDim.x) {
        const Elem el = make_elem(args, e, __ldg(args.S.elem + e));
        unsigned tw[kTopWords] = {};
        plane_tops<2, 1, ROLE_ROW, 3, ColsK0>(ctx, el, O.op[0], tw);
        plane_tops<2, 1, ROLE_ROW, 3, ColsK2>(ctx, el, O.op[2], tw);
        plane_tops<2, 1, ROLE_ROW, 3, ColsK4>(ctx, el, O.op[4], tw);
        plane_tops<2, 1, ROLE_ROW, 3, ColsK6>(ctx, el, O.op[6], tw);
        plane_tops<2, 1, ROLE_LAST, 3, ColsK8>(ctx, el, O.op[8], tw);
        line_tops<1, ColsK10>(ctx, el, O.op[10], tw);
        for (int w = 0; w < 2; ++w) args.tops_out[(size_t)w * args.S.size + e] = tw[w];
    }
}
extern "C" __global__ void __launch_bounds__(hx::kApplyThreads, 4)
hx_apply_specialised_dots(const __grid_constant__ hx::ApplyArgs args)
{
    hx::apply_elements<hx::R, 1>(args, [&](const hx::Ctx &ctx, const hx::Elem &el, hx::Acc<hx::R> &acc,
                                           const hx::R *sm_w, const hx::V *cin, const hx::R *tab) {
        hx::ops(args, ctx, el, acc, sm_w, cin, tab);
    });
}
extern "C" __global__ void __launch_bounds__(hx::kApplyThreads, 4)
hx_apply_specialised_rq(const __grid_constant__ hx::ApplyArgs args)
{
    hx::apply_elements<hx::R, 2>(args, [&](const hx::Ctx &ctx, const hx::Elem &el, hx::Acc<hx::R> &acc,
                                           const hx::R *sm_w, const hx::V *cin, const hx::R *tab) {
        hx::ops(args, ctx, el, acc, sm_w, cin, tab);
    });
}
