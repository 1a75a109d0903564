// Kernels compiled at run time for one potential's operator structure.
//
// The generic apply kernel (hx_apply.cu) reads the compiled operator list from its launch
// arguments and dispatches every operator of every element through a switch.  When all operators
// of a potential have specialised stencils (identity, pure-parity line operators of degree <= 3,
// plane operators with both degrees <= 2, no channel stage), hx_potential_set writes the operator
// sequence out as CUDA source: the same element loop and stencil functions (hx_stencil.cuh), but
// with every operator's class, axis roles and merged line fixed at compile time, so the compiler
// sees one straight sequence of loads and arithmetic instead of a loop over a switch.  The source
// is compiled with NVRTC for sm_103a and loaded through the driver API; kernels are cached per
// device, precision and structure (potentials that differ only in coefficients, time modulation or
// tables share one kernel).  Operator data (table offsets, degrees' rows, weights) still come from
// the launch arguments.  When compilation or loading fails the generic kernel is used.  For
// complex64 the module holds a second kernel that also computes the Lanczos projections
// h_i = s_i <v_i, A v_k> from the values it stores (ApplyFuse), which saves the time step one pass
// over the new vector per Krylov step.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <nvrtc.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>

#include <map>
#include <mutex>
#include <string>

#include "hx_internal.h"
#include "hx_stencil.cuh"
#include "hx_jit_sources.inc"   // kJitTypesSource, kJitStencilSource (generated by build.py)

namespace hx {

struct JitKernel {
    CUfunction fn = nullptr;
    CUfunction fn_dots = nullptr;   // complex64 only: the product with fused projections
    CUfunction fn_rq = nullptr;     // complex64 only: the product with the Rayleigh quotient <c, y>
    CUfunction fn_dual = nullptr;   // two times at once
    CUfunction fn_pair = nullptr;   // two inputs at two times
    CUfunction fn_stage1 = nullptr; // the first stage of a two-stage potential (channel vectors)
    CUfunction fn_tops = nullptr;   // packs each element's fibre-top fields (tops_words > 0)
    int tops_words = 0;
    int per_sm = 1, per_sm_dots = 1, per_sm_rq = 1, per_sm_dual = 1, per_sm_pair = 1, per_sm_stage1 = 1;
};

// Driver functions, looked up through the runtime (the library does not link the driver library,
// so that it also loads on machines without a GPU driver).
struct Driver {
    PFN_cuModuleLoadData_v2000 moduleLoadData = nullptr;
    PFN_cuModuleGetFunction_v2000 moduleGetFunction = nullptr;
    PFN_cuLaunchKernel_v4000 launchKernel = nullptr;
    PFN_cuOccupancyMaxActiveBlocksPerMultiprocessor_v6050 occupancy = nullptr;
    PFN_cuGetErrorString_v6000 errorString = nullptr;
    bool ok = false;
};

static const Driver &driver()
{
    static Driver d;
    static std::once_flag once;
    std::call_once(once, [] {
        auto get = [](const char *name, void **fn) {
            cudaDriverEntryPointQueryResult q;
            return cudaGetDriverEntryPointByVersion(name, fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
                   q == cudaDriverEntryPointSuccess && *fn;
        };
        d.ok = get("cuModuleLoadData", (void **)&d.moduleLoadData) &&
               get("cuModuleGetFunction", (void **)&d.moduleGetFunction) &&
               get("cuLaunchKernel", (void **)&d.launchKernel) &&
               get("cuOccupancyMaxActiveBlocksPerMultiprocessor", (void **)&d.occupancy) &&
               get("cuGetErrorString", (void **)&d.errorString);
    });
    return d;
}

static std::mutex g_jit_mu;
static std::map<std::string, JitKernel> g_jit_cache;

static bool specialised_plane(const Op &op, int sb)
{
    const bool cls = op.cls == CLS_PLANE + 0 || op.cls == CLS_PLANE + 3 || op.cls == CLS_PLANE + 1 || op.cls == CLS_PLANE + 4;
    return cls && (sb == 0 || sb == op.q || (sb == op.q + 2 && sb <= 3));
}

// Factor-order template argument of the plane stencils: 0 both orders with the runtime weights,
// 1 P(X_a) Q(X_b) alone, 2 Q(X_b) P(X_a) alone (the literal orders, weight 1), 3 both with weight
// 1/2 (the symmetric order).
static int plane_order(const OpSet &O)
{
    if (O.wAB == 1.0 && O.wBA == 0.0) return 1;
    if (O.wAB == 0.0 && O.wBA == 1.0) return 2;
    if (O.wAB == 0.5 && O.wBA == 0.5) return 3;
    return 0;
}

static const char *role_name(int r) { return r == ROLE_LAST ? "ROLE_LAST" : "ROLE_ROW"; }

// Weight expression of the line op merged into plane op i ("" when none); w = "sm_w" or "sm_w2".
static std::string merged_weight(const OpSet &O, const Op &op, const char *w)
{
    if (op.mergeB < 0) return "";
    return std::string(w) + "[" + std::to_string(op.mergeB) + "]";
}

// Fields of the precomputed fibre-top distances (the element's top words): per plane operator
// topA at v = 0 and at the footprint's steps v along b (width for 0..P), topB at the footprint's
// steps s along a (width for 0..TB at s = 0, 0..Q elsewhere); per line operator along a prefix axis
// its top (0..P).  No field straddles a 32-bit word.  on = false when they need more than
// kTopWords words (the kernels then compute the tops themselves).
struct TopLayout {
    bool on = false;
    int words = 0;
    std::map<int, std::map<int, int>> offA, offB;   // op -> step -> bit offset
    std::map<int, int> offT, wA;
    std::map<int, std::map<int, int>> wB;
};

static int field_bits(int maxval)
{
    int b = 1;
    while ((1 << b) <= maxval) ++b;
    return b;
}

static TopLayout top_layout(const OpSet &O)
{
    TopLayout L;
    int cur = 0;
    auto place = [&](int w) {
        if ((cur & 31) + w > 32) cur = (cur + 31) & ~31;
        const int off = cur;
        cur += w;
        return off;
    };
    for (int i = 0; i < O.nops; ++i) {
        const Op &op = O.op[i];
        if (op.merged) continue;
        if (op.kind == 2) {
            const int P = op.p, Q = op.q, SB = op.mergeB >= 0 ? O.op[op.mergeB].p : 0, TB = SB > Q ? SB : Q;
            L.wA[i] = field_bits(P);
            L.offA[i][0] = place(L.wA[i]);
            for (int j = 0; j <= Q; ++j)
                if (-Q + 2 * j != 0) L.offA[i][-Q + 2 * j] = place(L.wA[i]);
            for (int k = 0; k <= P; ++k) {
                const int st = -P + 2 * k, w = field_bits(st == 0 ? TB : Q);
                L.wB[i][st] = w;
                L.offB[i][st] = place(w);
            }
        } else if (op.kind == 1 && op.ra == ROLE_ROW) {
            L.wA[i] = field_bits(op.p);
            L.offT[i] = place(L.wA[i]);
        }
    }
    L.words = (cur + 31) / 32;
    L.on = L.words > 0 && L.words <= kTopWords;
    return L;
}

// Compile-time row moves of operator i's footprint points (a type with the start / startx
// functions of ColsRuntime): move (om, s4) of the column that didx gives each position; with a top
// layout also the offsets of its fibre-top fields and their readers.
static std::string cols_type(const OpSet &O, const RowOffsets &ro, int i, const char *prefix, int N,
                             const TopLayout *L = nullptr)
{
    const Op &op = O.op[i];
    const int span = (2 * op.p + 1) * (2 * op.q + 1);
    auto chain = [&](const char *name, int n, auto value) {
        std::string f = "    __device__ static constexpr int " + std::string(name) + "(int x) { return ";
        for (int x = 0; x < n; ++x) f += "x == " + std::to_string(x) + " ? " + std::to_string(value(x)) + " : ";
        f += "0; }\n";
        return f;
    };
    auto col = [&](int dbase, int x) { return (int)O.didx[dbase + x]; };
    std::string t = "struct " + std::string(prefix) + std::to_string(i) + " {\n";
    t += "    static constexpr int kA = " + std::to_string(op.a) + ", kB = " + std::to_string(op.kind == 2 ? op.b : -1) +
         ", kN = " + std::to_string(N) + ";\n";
    t += chain("om", span, [&](int x) { return (int)ro.mv[col(op.dbase, x)].om; });
    t += chain("s4", span, [&](int x) { return (int)ro.mv[col(op.dbase, x)].s4; });
    if (op.kind == 2 && op.mergeB >= 0) {
        const Op &ls = O.op[op.mergeB];
        const int sb = ls.p;
        t += chain("omx", 2, [&](int j) { return (int)ro.mv[col(ls.dbase, j == 0 ? 0 : 2 * sb)].om; });
        t += chain("s4x", 2, [&](int j) { return (int)ro.mv[col(ls.dbase, j == 0 ? 0 : 2 * sb)].s4; });
    } else {
        t += "    __device__ static constexpr int omx(int) { return -1; }\n";
        t += "    __device__ static constexpr int s4x(int) { return 0; }\n";
    }
    // the outer moves this operator's points take: their group-neighbour entries are read with
    // 16-byte loads of the group's row (gstride is a multiple of 4) when they span at most 4 of them
    int mlo = 1 << 30, mhi = -1;
    for (int x = 0; x < span; ++x) {
        const int m = ro.mv[col(op.dbase, x)].om;
        if (m >= 0) { mlo = std::min(mlo, m); mhi = std::max(mhi, m); }
    }
    if (op.kind == 2 && op.mergeB >= 0) {
        const Op &ls = O.op[op.mergeB];
        for (int j = 0; j < 2; ++j) {
            const int m = ro.mv[col(ls.dbase, j == 0 ? 0 : 2 * ls.p)].om;
            if (m >= 0) { mlo = std::min(mlo, m); mhi = std::max(mhi, m); }
        }
    }
    const int qlo = mhi >= 0 ? mlo / 4 : 0, nq = mhi >= 0 ? mhi / 4 - mlo / 4 + 1 : 0;
    if (nq > 4) {
        t += "    struct Gn {};\n"
             "    __device__ static __forceinline__ Gn gn_load(const Elem &) { return {}; }\n"
             "    __device__ static __forceinline__ int start(const Ctx &c, const Elem &el, const OpSet &, const Op &, const Gn &, int pos, bool ok)\n"
             "    { return c.start_mv(el, om(pos), s4(pos), ok); }\n"
             "    __device__ static __forceinline__ int startx(const Ctx &c, const Elem &el, const OpSet &, const Op &, const Gn &, int j, int, bool ok)\n"
             "    { return c.start_mv(el, omx(j), s4x(j), ok); }\n";
    } else {
        t += "    static constexpr int kGnLo = " + std::to_string(qlo) + ", kGnN = " + std::to_string(nq) + ";\n"
             "    struct Gn { int4 q[kGnN > 0 ? kGnN : 1]; };\n"
             "    __device__ static __forceinline__ Gn gn_load(const Elem &el)\n"
             "    {\n"
             "        Gn g;\n"
             "#pragma unroll\n"
             "        for (int i = 0; i < kGnN; ++i) g.q[i] = __ldg(reinterpret_cast<const int4 *>(el.gn) + kGnLo + i);\n"
             "        return g;\n"
             "    }\n"
             "    __device__ static __forceinline__ int gnv(const Gn &g, int m)\n"
             "    {\n"
             "        const int k = m - 4 * kGnLo;\n"
             "        const int4 q = g.q[k >> 2];\n"
             "        return (k & 3) == 0 ? q.x : (k & 3) == 1 ? q.y : (k & 3) == 2 ? q.z : q.w;\n"
             "    }\n"
             "    __device__ static __forceinline__ int start(const Ctx &c, const Elem &el, const OpSet &, const Op &, const Gn &g, int pos, bool ok)\n"
             "    { return c.start_row(el, om(pos) >= 0 ? gnv(g, om(pos)) + el.k4 + s4(pos) : el.r + s4(pos), ok); }\n"
             "    __device__ static __forceinline__ int startx(const Ctx &c, const Elem &el, const OpSet &, const Op &, const Gn &g, int j, int, bool ok)\n"
             "    { return c.start_row(el, omx(j) >= 0 ? gnv(g, omx(j)) + el.k4 + s4x(j) : el.r + s4x(j), ok); }\n";
    }
    const bool bits = L && L->on && (L->offA.count(i) || L->offT.count(i));
    t += std::string("    static constexpr bool kTopsBits = ") + (bits ? "true" : "false") + ";\n";
    if (bits) {
        auto steps = [](const std::map<int, int> &m, const char *name) {
            std::string f = "    __device__ static constexpr int " + std::string(name) + "(int v) { return ";
            for (const auto &kv : m) f += "v == " + std::to_string(kv.first) + " ? " + std::to_string(kv.second) + " : ";
            f += "0; }\n";
            return f;
        };
        if (L->offA.count(i)) {
            t += steps(L->offA.at(i), "offA");
            t += steps(L->offB.at(i), "offB");
            t += steps(L->wB.at(i), "wB");
            t += "    static constexpr int wA = " + std::to_string(L->wA.at(i)) + ";\n";
            t += "    __device__ static __forceinline__ int topA(const Elem &el, int v) { return top_field(el, offA(v), wA); }\n"
                 "    __device__ static __forceinline__ int topB(const Elem &el, int s) { return top_field(el, offB(s), wB(s)); }\n";
        } else {
            t += "    static constexpr int offT = " + std::to_string(L->offT.at(i)) + ", wT = " + std::to_string(L->wA.at(i)) + ";\n";
            t += "    __device__ static __forceinline__ int lineTop(const Elem &el) { return top_field(el, offT, wT); }\n";
        }
    }
    t += "};\n";
    return t;
}

static std::string jit_types(const OpSet &O, const RowOffsets &ro, int N, const char *prefix = "ColsK",
                             const TopLayout *L = nullptr)
{
    std::string t;
    for (int i = 0; i < O.nops; ++i)
        if (O.op[i].kind >= 1 && !O.op[i].merged) t += cols_type(O, ro, i, prefix, N, L);
    return t;
}

// The packing of the top fields, one call per operator with fields (the top-word kernel's body).
static std::string jit_body_tops(const OpSet &O, const TopLayout &L)
{
    std::string b;
    char line[512];
    for (int i = 0; i < O.nops; ++i) {
        const Op &op = O.op[i];
        if (op.merged) continue;
        if (L.offA.count(i)) {
            const int sb = op.mergeB >= 0 ? O.op[op.mergeB].p : 0;
            snprintf(line, sizeof(line), "        plane_tops<%d, %d, %s, %d, ColsK%d>(ctx, el, O.op[%d], tw);\n", op.p,
                     op.q, role_name(op.rb), sb, i, i);
            b += line;
        } else if (L.offT.count(i)) {
            snprintf(line, sizeof(line), "        line_tops<%d, ColsK%d>(ctx, el, O.op[%d], tw);\n", op.p, i, i);
            b += line;
        }
    }
    return b;
}

static bool specialised_line(const Op &op) { return op.cls >= CLS_LINE + 1 && op.cls <= CLS_LINE + kMaxDeg; }

// Input vector of op i in the generated code: c, or the channel a first stage wrote.
static std::string src_expr(const Op &op)
{
    if (op.src < 0) return "cin";
    return "((const V *)args.chan + (size_t)" + std::to_string(op.src) + " * args.chan_ld)";
}

// The first stage of a two-stage potential (line operators writing the channel vectors
// P(X_a) c), or "" when some operator needs the generic loop.
static std::string jit_body_stage1(const OpSet &O)
{
    std::string b;
    char line[768];
    for (int i = 0; i < O.nops; ++i) {
        const Op &op = O.op[i];
        if (op.kind != 1 || !specialised_line(op) || op.src >= 0 || op.dst < 0) return "";
        snprintf(line, sizeof(line),
                 "    { const V o = line_role<R, %d, %s, ColsS%d>(ctx, el, O, O.op[%d], tab, cin);\n"
                 "      ((V *)args.chan)[(size_t)%d * args.chan_ld + el.e] = cscale(sm_w[%d], o); }\n",
                 op.p, op.ra == ROLE_LAST ? "ROLE_LAST" : "ROLE_ROW", i, i, op.dst, i);
        b += line;
    }
    return b;
}

// The specialised sequence for O, or "" when some operator needs the generic loop.  dual: each
// operator's sum also goes to acc2 with its weight at the second time (sm_w2).
static std::string jit_body(const OpSet &O, bool dual = false)
{
    std::string b;
    char line[1024];
    const int ord = plane_order(O);
    for (int i = 0; i < O.nops; ++i) {
        const Op &op = O.op[i];
        if (op.merged) continue;
        if (op.dst >= 0 || (op.src >= 0 && op.kind != 1)) return "";
        std::string add2;
        if (op.kind == 0) {
            if (dual) add2 = " acc2.add(cscale(sm_w2[" + std::to_string(i) + "], cs));";
            snprintf(line, sizeof(line), "    { const V cs = cin[el.e]; acc.add(cscale(sm_w[%d], cs));%s }\n", i,
                     add2.c_str());
        } else if (op.kind == 1) {
            if (!specialised_line(op) || op.mergeB >= 0) return "";
            if (dual) add2 = " acc2.add(cscale(sm_w2[" + std::to_string(i) + "], o));";
            snprintf(line, sizeof(line),
                     "    { const V o = line_role<R, %d, %s, ColsK%d>(ctx, el, O, O.op[%d], tab, %s);\n"
                     "      acc.add(cscale(sm_w[%d], o));%s }\n",
                     op.p, role_name(op.ra), i, i, src_expr(op).c_str(), i, add2.c_str());
        } else {
            const int sb = op.mergeB >= 0 ? O.op[op.mergeB].p : 0;
            if (!specialised_plane(op, sb)) return "";
            const std::string wl = merged_weight(O, op, "sm_w"), wl2 = merged_weight(O, op, "sm_w2");
            const std::string v1 = wl.empty() ? "cscale(sm_w[" + std::to_string(i) + "], o)"
                                              : "cmad(" + wl + ", l, cscale(sm_w[" + std::to_string(i) + "], o))";
            const std::string v2 = wl2.empty() ? "cscale(sm_w2[" + std::to_string(i) + "], o)"
                                               : "cmad(" + wl2 + ", l, cscale(sm_w2[" + std::to_string(i) + "], o))";
            if (dual) add2 = "\n      acc2.add(" + v2 + ");";
            snprintf(line, sizeof(line),
                     "    { V o, l;\n"
                     "      plane_role<R, %d, %d, %s, %d, %d, ColsK%d>(ctx, el, O, O.op[%d], tab, cin, o, l);\n"
                     "      acc.add(%s);%s }\n",
                     op.p, op.q, role_name(op.rb), sb, ord, i, i, v1.c_str(), add2.c_str());
        }
        b += line;
    }
    return b;
}

// The sequence for two inputs (cin into acc at the first time, cin2 into acc2 at the second):
// each stencil's addresses and weights serve both inputs.  Called only for an O that jit_body
// accepts.
static std::string jit_body_pair(const OpSet &O)
{
    std::string b;
    char line[1280];
    const int ord = plane_order(O);
    for (int i = 0; i < O.nops; ++i) {
        const Op &op = O.op[i];
        if (op.merged) continue;
        if (op.kind == 0) {
            snprintf(line, sizeof(line),
                     "    { acc.add(cscale(sm_w[%d], cin[el.e])); acc2.add(cscale(sm_w2[%d], cin2[el.e])); }\n", i, i);
        } else if (op.kind == 1) {
            snprintf(line, sizeof(line),
                     "    { const V *sr[2] = {cin, cin2}; V o[2];\n"
                     "      line_role_n<R, %d, %s, 2, ColsK%d>(ctx, el, O, O.op[%d], tab, sr, o);\n"
                     "      acc.add(cscale(sm_w[%d], o[0])); acc2.add(cscale(sm_w2[%d], o[1])); }\n",
                     op.p, role_name(op.ra), i, i, i, i);
        } else {
            const int sb = op.mergeB >= 0 ? O.op[op.mergeB].p : 0;
            const std::string wl = merged_weight(O, op, "sm_w"), wl2 = merged_weight(O, op, "sm_w2");
            const std::string is = std::to_string(i);
            const std::string v1 = wl.empty() ? "cscale(sm_w[" + is + "], o[0])" : "cmad(" + wl + ", l[0], cscale(sm_w[" + is + "], o[0]))";
            const std::string v2 = wl2.empty() ? "cscale(sm_w2[" + is + "], o[1])" : "cmad(" + wl2 + ", l[1], cscale(sm_w2[" + is + "], o[1]))";
            snprintf(line, sizeof(line),
                     "    { const V *sr[2] = {cin, cin2}; V o[2], l[2];\n"
                     "      plane_role_n<R, %d, %d, %s, %d, 2, %d, ColsK%d>(ctx, el, O, O.op[%d], tab, sr, o, l);\n"
                     "      acc.add(%s);\n"
                     "      acc2.add(%s); }\n",
                     op.p, op.q, role_name(op.rb), sb, ord, i, i, v1.c_str(), v2.c_str());
        }
        b += line;
    }
    return b;
}

static std::string jit_source(bool f32, const std::string &types, const std::string &body, const std::string &body2,
                              const std::string &body3, const std::string &body_s1 = "",
                              const std::string &body_tops = "", int tops_words = 0)
{
    std::string s;
    s += "#include \"hx_stencil.cuh\"\n";
    s += "namespace hx {\n";
    s += types;
    s += "using R = ";
    s += f32 ? "float" : "double";
    s += ";\nusing V = Vec2<R>::T;\n";
    s += "__device__ __forceinline__ void ops(const ApplyArgs &args, const Ctx &ctx, const Elem &el, Acc<R> &acc,\n"
         "                                    const R *sm_w, const V *cin, const R *tab)\n{\n"
         "    const OpSet &O = args.ops;\n";
    s += body;
    s += "}\n";
    s += "__device__ __forceinline__ void ops_dual(const ApplyArgs &args, const Ctx &ctx, const Elem &el, Acc<R> &acc,\n"
         "                                         Acc<R> &acc2, const R *sm_w, const R *sm_w2, const V *cin, const R *tab)\n{\n"
         "    const OpSet &O = args.ops;\n";
    s += body2;
    s += "}\n";
    s += "__device__ __forceinline__ void ops_pair(const ApplyArgs &args, const Ctx &ctx, const Elem &el, Acc<R> &acc,\n"
         "                                         Acc<R> &acc2, const R *sm_w, const R *sm_w2, const V *cin,\n"
         "                                         const V *cin2, const R *tab)\n{\n"
         "    const OpSet &O = args.ops;\n";
    s += body3;
    s += "}\n";
    if (!body_s1.empty()) {
        s += "__device__ __forceinline__ void ops_stage1(const ApplyArgs &args, const Ctx &ctx, const Elem &el, Acc<R> &acc,\n"
             "                                           const R *sm_w, const V *cin, const R *tab)\n{\n"
             "    const OpSet &O = args.ops;\n";
        s += body_s1;
        s += "}\n";
    }
    s += "}  // namespace hx\n";
    if (!body_s1.empty()) {   // the first stage of a two-stage potential: writes the channel vectors
        s += f32 ? "extern \"C\" __global__ void __launch_bounds__(hx::kApplyThreads, 4)\n"
                 : "extern \"C\" __global__ void __launch_bounds__(hx::kApplyThreads, 3)\n";
        s += "hx_apply_specialised_stage1(const __grid_constant__ hx::ApplyArgs args)\n{\n"
             "    hx::apply_elements<hx::R>(args, [&](const hx::Ctx &ctx, const hx::Elem &el, hx::Acc<hx::R> &acc,\n"
             "                                        const hx::R *sm_w, const hx::V *cin, const hx::R *tab) {\n"
             "        hx::ops_stage1(args, ctx, el, acc, sm_w, cin, tab);\n"
             "    });\n}\n";
    }
    // 4 blocks of 256 per SM fit the FP32 kernels in 64 registers without spills (more warps to hide
    // the load latency); the FP64 kernels would spill there and keep 3 blocks (80 registers)
    s += f32 ? "extern \"C\" __global__ void __launch_bounds__(hx::kApplyThreads, 4)\n"
             : "extern \"C\" __global__ void __launch_bounds__(hx::kApplyThreads, 3)\n";
    s += "hx_apply_specialised(const __grid_constant__ hx::ApplyArgs args)\n{\n"
         "    hx::apply_elements<hx::R>(args, [&](const hx::Ctx &ctx, const hx::Elem &el, hx::Acc<hx::R> &acc,\n"
         "                                        const hx::R *sm_w, const hx::V *cin, const hx::R *tab) {\n"
         "        hx::ops(args, ctx, el, acc, sm_w, cin, tab);\n"
         "    });\n}\n";
    // two times at once (the 2-stage Magnus method's A_1 v and A_2 v).  The two-time kernels keep 3
    // blocks of 256 per SM in both precisions: at 4 (64 registers) the complex64 ones spilled (the
    // Hénon-Heiles chain at N=6: 112 and 588 bytes) and ran the Magnus step 24 % slower
    s += "extern \"C\" __global__ void __launch_bounds__(hx::kApplyThreads, 3)\n";
    s += "hx_apply_specialised_dual(const __grid_constant__ hx::ApplyArgs args)\n{\n"
         "    hx::apply_elements_dual<hx::R>(args, [&](const hx::Ctx &ctx, const hx::Elem &el, hx::Acc<hx::R> &acc,\n"
         "                                             hx::Acc<hx::R> &acc2, const hx::R *sm_w, const hx::R *sm_w2,\n"
         "                                             const hx::V *cin, const hx::V *, const hx::R *tab) {\n"
         "        hx::ops_dual(args, ctx, el, acc, acc2, sm_w, sm_w2, cin, tab);\n"
         "    });\n}\n";
    // two inputs at two times (the Magnus method's A_2 (A_1 v) and A_1 (A_2 v))
    s += "extern \"C\" __global__ void __launch_bounds__(hx::kApplyThreads, 3)\n";
    s += "hx_apply_specialised_pair(const __grid_constant__ hx::ApplyArgs args)\n{\n"
         "    hx::apply_elements_dual<hx::R>(args, [&](const hx::Ctx &ctx, const hx::Elem &el, hx::Acc<hx::R> &acc,\n"
         "                                             hx::Acc<hx::R> &acc2, const hx::R *sm_w, const hx::R *sm_w2,\n"
         "                                             const hx::V *cin, const hx::V *cin2, const hx::R *tab) {\n"
         "        hx::ops_pair(args, ctx, el, acc, acc2, sm_w, sm_w2, cin, cin2, tab);\n"
         "    });\n}\n";
    if (!body_tops.empty()) {   // each element's fibre-top fields, packed once per potential and index set
        s += "extern \"C\" __global__ void __launch_bounds__(hx::kApplyThreads)\n"
             "hx_apply_tops(const __grid_constant__ hx::ApplyArgs args)\n{\n"
             "    using namespace hx;\n"
             "    Ctx ctx;\n"
             "    ctx.S = &args.S;\n"
             "    ctx.mv = args.mv;\n"
             "    const OpSet &O = args.ops;\n"
             "    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < args.S.size; e += gridDim.x * blockDim.x) {\n"
             "        const Elem el = make_elem(args, e, __ldg(args.S.elem + e));\n"
             "        unsigned tw[kTopWords] = {};\n";
        s += body_tops;
        s += "        for (int w = 0; w < " + std::to_string(tops_words) + "; ++w) args.tops_out[(size_t)w * args.S.size + e] = tw[w];\n"
             "    }\n}\n";
    }
    if (f32) {   // the same product that also computes the Lanczos projections (ApplyFuse)
        s += "extern \"C\" __global__ void __launch_bounds__(hx::kApplyThreads, 4)\n"
             "hx_apply_specialised_dots(const __grid_constant__ hx::ApplyArgs args)\n{\n"
             "    hx::apply_elements<hx::R, 1>(args, [&](const hx::Ctx &ctx, const hx::Elem &el, hx::Acc<hx::R> &acc,\n"
             "                                           const hx::R *sm_w, const hx::V *cin, const hx::R *tab) {\n"
             "        hx::ops(args, ctx, el, acc, sm_w, cin, tab);\n"
             "    });\n}\n";
        // the same product with the Rayleigh quotient <c, y> of its input (the Lanczos step's sweep)
        s += "extern \"C\" __global__ void __launch_bounds__(hx::kApplyThreads, 4)\n"
             "hx_apply_specialised_rq(const __grid_constant__ hx::ApplyArgs args)\n{\n"
             "    hx::apply_elements<hx::R, 2>(args, [&](const hx::Ctx &ctx, const hx::Elem &el, hx::Acc<hx::R> &acc,\n"
             "                                           const hx::R *sm_w, const hx::V *cin, const hx::R *tab) {\n"
             "        hx::ops(args, ctx, el, acc, sm_w, cin, tab);\n"
             "    });\n}\n";
    }
    return s;
}

static bool compile_and_load(const std::string &src, int dev, JitKernel *out, std::string &reason)
{
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major != 10 || minor != 3) {
        reason = "run-time compiled kernels target sm_103a only";
        return false;
    }
    const Driver &drv = driver();
    if (!drv.ok) {
        reason = "driver entry points for module loading are unavailable";
        return false;
    }
    nvrtcProgram prog;
    const char *headers[] = {kJitTypesSource, kJitStencilSource};
    const char *names[] = {"hx_types.h", "hx_stencil.cuh"};
    if (nvrtcCreateProgram(&prog, src.c_str(), "hx_apply_specialised.cu", 2, headers, names) != NVRTC_SUCCESS) {
        reason = "nvrtcCreateProgram failed";
        return false;
    }
    const char *opts[] = {"--gpu-architecture=sm_103a", "--std=c++17", "-lineinfo"};
    nvrtcResult rc = nvrtcCompileProgram(prog, 3, opts);
    if (rc != NVRTC_SUCCESS) {
        size_t n = 0;
        nvrtcGetProgramLogSize(prog, &n);
        std::string log(n, '\0');
        if (n) nvrtcGetProgramLog(prog, &log[0]);
        reason = std::string("nvrtc: ") + nvrtcGetErrorString(rc) + ": " + log.substr(0, 400);
        nvrtcDestroyProgram(&prog);
        return false;
    }
    size_t nbin = 0;
    nvrtcGetCUBINSize(prog, &nbin);
    std::string cubin(nbin, '\0');
    nvrtcGetCUBIN(prog, &cubin[0]);
    nvrtcDestroyProgram(&prog);
    CUmodule mod;
    CUfunction fn;
    if (drv.moduleLoadData(&mod, cubin.data()) != CUDA_SUCCESS ||
        drv.moduleGetFunction(&fn, mod, "hx_apply_specialised") != CUDA_SUCCESS) {
        reason = "loading the compiled kernel failed";
        return false;
    }
    CUfunction fn_dots = nullptr, fn_dual = nullptr, fn_pair = nullptr, fn_stage1 = nullptr, fn_tops = nullptr;
    if (src.find("hx_apply_tops") != std::string::npos &&
        drv.moduleGetFunction(&fn_tops, mod, "hx_apply_tops") != CUDA_SUCCESS) {
        reason = "loading the compiled kernel failed";
        return false;
    }
    if (src.find("hx_apply_specialised_stage1") != std::string::npos &&
        drv.moduleGetFunction(&fn_stage1, mod, "hx_apply_specialised_stage1") != CUDA_SUCCESS) {
        reason = "loading the compiled kernel failed";
        return false;
    }
    CUfunction fn_rq = nullptr;
    if ((src.find("hx_apply_specialised_dots") != std::string::npos &&
         drv.moduleGetFunction(&fn_dots, mod, "hx_apply_specialised_dots") != CUDA_SUCCESS) ||
        (src.find("hx_apply_specialised_rq") != std::string::npos &&
         drv.moduleGetFunction(&fn_rq, mod, "hx_apply_specialised_rq") != CUDA_SUCCESS) ||
        drv.moduleGetFunction(&fn_dual, mod, "hx_apply_specialised_dual") != CUDA_SUCCESS ||
        drv.moduleGetFunction(&fn_pair, mod, "hx_apply_specialised_pair") != CUDA_SUCCESS) {
        reason = "loading the compiled kernel failed";
        return false;
    }
    auto occ = [&](CUfunction f) {
        int per_sm = 1;
        if (!f || drv.occupancy(&per_sm, f, kApplyThreads, 0) != CUDA_SUCCESS || per_sm < 1) per_sm = 1;
        return per_sm;
    };
    out->fn = fn;
    out->fn_dots = fn_dots;
    out->fn_rq = fn_rq;
    out->fn_dual = fn_dual;
    out->fn_pair = fn_pair;
    out->fn_stage1 = fn_stage1;
    out->fn_tops = fn_tops;
    out->per_sm_stage1 = occ(fn_stage1);
    out->per_sm = occ(fn);
    out->per_sm_dots = occ(fn_dots);
    out->per_sm_rq = occ(fn_rq);
    out->per_sm_dual = occ(fn_dual);
    out->per_sm_pair = occ(fn_pair);
    return true;
}

// Prepares the specialised kernel of p's main-stage operators (after compile_potential); p->jit is
// left null when the generic kernel must be used.  Never fails the caller.
void jit_prepare(Problem *p)
{
    p->jit = nullptr;
    std::string &reason = p->jit_reason;
    const char *env = getenv("HX_APPLY_SPECIALISE");
    if (env && env[0] == '0') {
        reason = "disabled by HX_APPLY_SPECIALISE=0";
        return;
    }
    if (p->set->h.general) {
        reason = "a general index set: the generic kernel decides membership from the row tables";
        return;
    }
    const std::string body = jit_body(p->ops);
    if (body.empty()) {
        reason = "an operator has no specialised stencil";
        return;
    }
    std::string body_s1;
    if (p->ops1.nops > 0) {
        body_s1 = jit_body_stage1(p->ops1);
        if (body_s1.empty()) {
            reason = "a first-stage operator has no specialised stencil";
            return;
        }
    }
    const bool f32 = p->cfg.dtype == HX_C64;
    const TopLayout L = top_layout(p->ops);
    const std::string body_tops = L.on ? jit_body_tops(p->ops, L) : "";
    const int tops_words = body_tops.empty() ? 0 : L.words;
    const int N = p->set->h.N;
    const std::string types = jit_types(p->ops, p->roff, N, "ColsK", body_tops.empty() ? nullptr : &L) +
                              jit_types(p->ops1, p->roff, N, "ColsS");
    const std::string key = std::to_string(p->device) + (f32 ? "|f|" : "|d|") + types + body + body_s1;
    // the two-time kernels run only for single-stage potentials (apply_dual)
    const std::string body_dual = p->ops1.nops ? "" : jit_body(p->ops, true);
    const std::string body_pair = p->ops1.nops ? "" : jit_body_pair(p->ops);
    std::lock_guard<std::mutex> lock(g_jit_mu);
    auto it = g_jit_cache.find(key);
    if (it == g_jit_cache.end()) {
        JitKernel k;
        // HX_JIT_SOURCE_DUMP=<file>: the generated source is appended there before it is compiled
        // (one source per kernel set the process compiles)
        if (const char *dump = getenv("HX_JIT_SOURCE_DUMP")) {
            if (FILE *f = fopen(dump, "a")) {
                fprintf(f, "// ---- kernel set %s, N = %d\n", f32 ? "complex64" : "complex128", N);
                const std::string src = jit_source(f32, types, body, body_dual, body_pair, body_s1, body_tops, tops_words);
                fwrite(src.data(), 1, src.size(), f);
                fclose(f);
            }
        }
        if (!compile_and_load(jit_source(f32, types, body, body_dual, body_pair, body_s1, body_tops, tops_words), p->device,
                              &k, reason))
            return;
        k.tops_words = k.fn_tops ? tops_words : 0;
        it = g_jit_cache.emplace(key, k).first;
    }
    p->jit = &it->second;
    reason = "specialised kernel in use";
}

// Launches the specialised kernel with the generic kernel's arguments.
int jit_launch(const Problem *p, const void *args, int blocks, cudaStream_t st)
{
    const JitKernel *k = (const JitKernel *)p->jit;
    const ApplyArgs *a = (const ApplyArgs *)args;
    const bool dots = a->dvec != nullptr, rq = a->drq != 0, dual = a->cout2 != nullptr, pair = dual && a->cin2 != nullptr;
    if (a->stage1) {
        if (!k->fn_stage1) {
            set_error("internal: no compiled first-stage kernel");
            return HX_EUNSUPPORTED;
        }
        const int grid = std::max(1, std::min({p->num_sms * k->per_sm_stage1, apply_grid(p), blocks}));
        void *params[] = {const_cast<void *>(args)};
        CUresult r = driver().launchKernel(k->fn_stage1, grid, 1, 1, kApplyThreads, 1, 1, 0, (CUstream)st, params, nullptr);
        if (r != CUDA_SUCCESS) {
            const char *msg = nullptr;
            driver().errorString(r, &msg);
            set_error("specialised first-stage kernel launch: %s", msg ? msg : "unknown error");
            return HX_ECUDA;
        }
        return HX_OK;
    }
    if ((dots && !k->fn_dots) || (rq && !k->fn_rq) || ((dots || rq) && dual) || (dots && rq)) {
        set_error("the specialised kernel has no fused projections here (complex64 single products only)");
        return HX_EUNSUPPORTED;
    }
    CUfunction fn = pair ? k->fn_pair : dual ? k->fn_dual : dots ? k->fn_dots : rq ? k->fn_rq : k->fn;
    const int per_sm = pair ? k->per_sm_pair : dual ? k->per_sm_dual : dots ? k->per_sm_dots : rq ? k->per_sm_rq : k->per_sm;
    // apply_grid(p) blocks at most: the size of the partial-sum buffers
    int grid = std::min(p->num_sms * per_sm, apply_grid(p));
    if (grid > blocks) grid = blocks > 0 ? blocks : 1;
    void *params[] = {const_cast<void *>(args)};
    const Driver &drv = driver();
    CUresult r = drv.launchKernel(fn, grid, 1, 1, kApplyThreads, 1, 1, 0, (CUstream)st, params, nullptr);
    if (r != CUDA_SUCCESS) {
        const char *msg = nullptr;
        drv.errorString(r, &msg);
        set_error("specialised apply kernel launch: %s", msg ? msg : "unknown error");
        return HX_ECUDA;
    }
    return HX_OK;
}

}  // namespace hx

namespace hx {
bool jit_has_stage1(const Problem *p) { return p->jit && ((const JitKernel *)p->jit)->fn_stage1 != nullptr; }

int jit_tops_words(const Problem *p) { return p->jit ? ((const JitKernel *)p->jit)->tops_words : 0; }

// Packs the fibre-top fields of every element for the specialised kernel (once per kernel and index
// set: kept while both stay the same).
int jit_fill_tops(Problem *p)
{
    const JitKernel *k = (const JitKernel *)p->jit;
    if (!k || k->tops_words == 0) return HX_OK;
    const size_t n = (size_t)p->set->d.size, bytes = n * k->tops_words * sizeof(unsigned);
    if (p->tops && p->tops_src == (const void *)k && p->tops_bytes == bytes) return HX_OK;
    if (p->tops_bytes != bytes) {
        cudaFree(p->tops);
        p->tops = nullptr;
        p->tops_bytes = 0;
        cudaError_t e = cudaMalloc((void **)&p->tops, std::max<size_t>(bytes, 4));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(fibre-top fields)");
        p->tops_bytes = bytes;
    }
    p->tops_src = nullptr;
    ApplyArgs a;
    memset(&a, 0, sizeof(a));
    a.S = p->set->d;
    memcpy(a.mv, p->roff.mv, sizeof(a.mv));
    a.ops = p->ops;
    a.tops_out = p->tops;
    const int blocks = (int)std::min<size_t>((n + kApplyThreads - 1) / kApplyThreads, (size_t)p->num_sms * 8);
    void *params[] = {&a};
    const Driver &drv = driver();
    CUresult r = drv.launchKernel(k->fn_tops, std::max(blocks, 1), 1, 1, kApplyThreads, 1, 1, 0, (CUstream)p->stream, params,
                                  nullptr);
    if (r != CUDA_SUCCESS) {
        const char *msg = nullptr;
        drv.errorString(r, &msg);
        set_error("fibre-top kernel launch: %s", msg ? msg : "unknown error");
        return HX_ECUDA;
    }
    cudaError_t e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "fibre-top kernel");
    p->tops_src = k;
    return HX_OK;
}
}  // namespace hx
