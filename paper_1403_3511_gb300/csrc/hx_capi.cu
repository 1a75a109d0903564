// C ABI of libhx: argument checking, index-set and potential set-up on the host, and
// dispatch to the kernels in hx_apply.cu / hx_krylov.cu.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <new>

#include "hx_internal.h"

namespace hx {

// plane operators with more footprint points than this go through two stages
constexpr int kDirectFootprint = 36;

static thread_local char g_err[512] = "no error";

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int cuda_fail(cudaError_t e, const char *what)
{
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? HX_ENOMEM : HX_ECUDA;
}

#define HX_CUDA(call, what)                        \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// ---------------------------------------------------------------------------------------
// index set tables (host)
// ---------------------------------------------------------------------------------------

// |K_m(b)| for every b in the quotient set {floor(B/q)} of B, by
// |K_m(b)| = sum_{k=0}^{b-1} |K_{m-1}(floor(b/(1+k)))|, |K_0(b)| = 1 for b >= 1.
// floor(floor(B/q)/j) = floor(B/(qj)), so only quotient values are ever needed.
static bool counts_by_quotient(int N, int B, std::vector<std::vector<int64_t>> &C)
{
    std::vector<int> quot;
    for (int q = 1; q <= B;) {
        int v = B / q;
        quot.push_back(v);
        q = B / v + 1;
    }
    std::sort(quot.begin(), quot.end());
    C.assign(N + 1, std::vector<int64_t>(B + 1, 0));
    for (int v : quot) C[0][v] = 1;
    const int64_t cap = (int64_t)1 << 40;
    for (int m = 1; m <= N; ++m) {
        for (int v : quot) {
            int64_t s = 0;
            for (int k = 0; k < v; ++k) {
                s += C[m - 1][v / (1 + k)];
                if (s > cap) s = cap;
            }
            C[m][v] = s;
        }
    }
    return true;
}

// Rows in lexicographic order of their prefixes (axes 0..N-2): start rank, prefix product,
// coordinate sum and length floor(B / q) of each.
static void enum_rows(int depth, int npre, int q, int ksum, int B, uint16_t *prefix, IndexSetHost &h, int64_t &pos)
{
    if (depth == npre) {
        if (npre == 0 || prefix[npre - 1] == 0) {   // first row of a new group (k_{N-2} = 0)
            h.gfirst.push_back((int)h.row_info.size());
            h.ngroup = (int)h.gfirst.size();
        }
        h.rgrp.push_back(h.ngroup - 1);
        h.row_k.insert(h.row_k.end(), prefix, prefix + npre);
        int len = B / q;
        h.row_info.push_back(make_int4((int)pos, q, ksum, len));
        pos += len;
        return;
    }
    for (int k = 0; (int64_t)q * (1 + k) <= B; ++k) {
        prefix[depth] = (uint16_t)k;
        enum_rows(depth + 1, npre, q * (1 + k), ksum + k, B, prefix, h, pos);
    }
}

static int build_host_tables(int N, int B, IndexSetHost &h)
{
    std::vector<std::vector<int64_t>> C;
    counts_by_quotient(N, B, C);
    int64_t size = C[N][B];
    if (size >= ((int64_t)1 << 31) - 1) {
        set_error("index set too large: |K| = %lld needs 64-bit ranks", (long long)size);
        return HX_EUNSUPPORTED;
    }
    h.N = N;
    h.B = B;
    h.size = size;
    h.qoff.assign(B + 2, 0);
    int64_t tot = 0;
    for (int q = 1; q <= B; ++q) {
        h.qoff[q] = (int)tot;
        tot += B / q + 1;
    }
    h.qoff[B + 1] = (int)tot;
    h.qtotal = (int)tot;
    int levels = N - 1;
    h.Q.assign((size_t)std::max(levels, 0) * tot, 0);
    for (int m = 1; m <= levels; ++m) {
        int *Qm = h.Q.data() + (size_t)(m - 1) * tot;
        for (int q = 1; q <= B; ++q) {
            int bq = B / q;
            int64_t acc = 0;
            int *row = Qm + h.qoff[q];
            for (int k = 0; k <= bq; ++k) {
                row[k] = (int)acc;
                if (k < bq) acc += C[m][B / (q * (1 + k))];
            }
        }
    }
    uint16_t prefix[kMaxN];
    int64_t pos = 0;
    h.row_info.clear();
    h.row_k.clear();
    h.rgrp.clear();
    h.gfirst.clear();
    h.ngroup = 0;
    enum_rows(0, N - 1, 1, 0, B, prefix, h, pos);
    h.nrow = (int)h.row_info.size();
    if (pos != size) {
        set_error("internal: row lengths sum to %lld != |K| %lld", (long long)pos, (long long)size);
        return HX_ECUDA;
    }
    return HX_OK;
}

// Tables of a general downward-closed set given as a list of multi-indices (any order): the list
// sorted lexicographically (last coordinate fastest), checked for duplicates, negative coordinates
// and downward closure, and its rows and groups as for the hyperbolic cross.  B becomes 1 + the
// largest coordinate (the row tables of the potential cover the coordinates 0..B-1).
static bool lex_less(const int32_t *a, const int32_t *b, int N)
{
    for (int l = 0; l < N; ++l)
        if (a[l] != b[l]) return a[l] < b[l];
    return false;
}

static int64_t list_find(const IndexSetHost &h, const int32_t *k)
{
    int64_t lo = 0, hi = h.size - 1;
    const int N = h.N;
    while (lo <= hi) {
        const int64_t mid = (lo + hi) / 2;
        const int32_t *x = h.list.data() + (size_t)mid * N;
        if (lex_less(x, k, N)) lo = mid + 1;
        else if (lex_less(k, x, N)) hi = mid - 1;
        else return mid;
    }
    return -1;
}

static int build_list_tables(int N, int64_t count, const int32_t *k, IndexSetHost &h)
{
    if (count < 1 || count >= ((int64_t)1 << 31) - 1) {
        set_error("hx_indexset_create_list: need 1 <= count < 2^31 - 1 (got %lld)", (long long)count);
        return count < 1 ? HX_EINVAL : HX_EUNSUPPORTED;
    }
    std::vector<int64_t> idx(count);
    for (int64_t i = 0; i < count; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) { return lex_less(k + a * N, k + b * N, N); });
    h.N = N;
    h.general = true;
    h.size = count;
    h.list.resize((size_t)count * N);
    int maxc = 0;
    for (int64_t i = 0; i < count; ++i) {
        const int32_t *x = k + idx[i] * N;
        int ksum = 0;
        for (int l = 0; l < N; ++l) {
            if (x[l] < 0 || x[l] > 65534) {
                set_error("hx_indexset_create_list: coordinate %d outside 0..65534", x[l]);
                return HX_EINVAL;
            }
            maxc = std::max(maxc, (int)x[l]);
            ksum += x[l];
        }
        if (ksum > 65535) {
            set_error("hx_indexset_create_list: a coordinate sum above 65535 is not supported");
            return HX_EUNSUPPORTED;
        }
        memcpy(h.list.data() + (size_t)i * N, x, N * sizeof(int32_t));
        if (i > 0 && !lex_less(h.list.data() + (size_t)(i - 1) * N, x, N)) {
            set_error("hx_indexset_create_list: duplicate multi-index");
            return HX_EINVAL;
        }
    }
    std::vector<int32_t> y(N);
    for (int64_t i = 0; i < count; ++i) {            // downward closure: k - e_l in K for k_l > 0
        const int32_t *x = h.list.data() + (size_t)i * N;
        for (int l = 0; l < N; ++l) {
            if (x[l] == 0) continue;
            memcpy(y.data(), x, N * sizeof(int32_t));
            y[l] -= 1;
            if (list_find(h, y.data()) < 0) {
                set_error("hx_indexset_create_list: the set is not downward closed (multi-index %lld lacks its "
                          "neighbour below it along axis %d)", (long long)i, l);
                return HX_EINVAL;
            }
        }
    }
    h.B = maxc + 1;
    h.qtotal = 0;
    h.qoff.assign(h.B + 2, 0);
    h.Q.clear();
    h.row_info.clear();
    h.row_k.clear();
    h.rgrp.clear();
    h.gfirst.clear();
    h.ngroup = 0;
    const int npre = N - 1;
    for (int64_t i = 0; i < count;) {                // rows: runs of a common prefix k_0..k_{N-2}
        const int32_t *x = h.list.data() + (size_t)i * N;
        int64_t j = i + 1;
        while (j < count && !memcmp(h.list.data() + (size_t)j * N, x, npre * sizeof(int32_t))) ++j;
        const int len = (int)(j - i);
        if (len > 65535 || h.list[(size_t)(j - 1) * N + N - 1] != len - 1) {
            set_error("hx_indexset_create_list: a row longer than 65535 or not contiguous");
            return len > 65535 ? HX_EUNSUPPORTED : HX_EINVAL;
        }
        if (npre == 0 || x[npre - 1] == 0) {
            h.gfirst.push_back((int)h.row_info.size());
            h.ngroup = (int)h.gfirst.size();
        }
        h.rgrp.push_back(h.ngroup - 1);
        int ksum = 0;
        for (int l = 0; l < npre; ++l) {
            h.row_k.push_back((uint16_t)x[l]);
            ksum += x[l];
        }
        h.row_info.push_back(make_int4((int)i, 0, ksum, len));
        i = j;
    }
    h.nrow = (int)h.row_info.size();
    return HX_OK;
}

static int64_t host_rank(const IndexSetHost &h, const int32_t *k)
{
    if (h.general) {
        for (int l = 0; l < h.N; ++l)
            if (k[l] < 0) return -1;
        return list_find(h, k);
    }
    int64_t q = 1;
    for (int l = 0; l < h.N; ++l) {
        if (k[l] < 0) return -1;
        q *= (1 + (int64_t)k[l]);
        if (q > h.B) return -1;
    }
    int64_t r = 0;
    q = 1;
    for (int d = 0; d < h.N - 1; ++d) {
        int m = h.N - 1 - d;
        r += h.Q[(size_t)(m - 1) * h.qtotal + h.qoff[q] + k[d]];
        q *= (1 + k[d]);
    }
    return r + k[h.N - 1];
}

static int host_unrank(const IndexSetHost &h, int64_t rank, int32_t *k)
{
    if (rank < 0 || rank >= h.size) return HX_EINVAL;
    if (h.general) {
        memcpy(k, h.list.data() + (size_t)rank * h.N, h.N * sizeof(int32_t));
        return HX_OK;
    }
    int64_t q = 1, rem = rank;
    for (int d = 0; d < h.N - 1; ++d) {
        int m = h.N - 1 - d;
        const int *row = h.Q.data() + (size_t)(m - 1) * h.qtotal + h.qoff[q];
        int bq = (int)(h.B / q);
        // largest i < bq with row[i] <= rem (row is nondecreasing, row[0] = 0)
        int lo = 0, hi = bq - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) / 2;
            if (row[mid] <= rem) lo = mid; else hi = mid - 1;
        }
        k[d] = lo;
        rem -= row[lo];
        q *= (1 + lo);
    }
    k[h.N - 1] = (int32_t)rem;
    return HX_OK;
}

// ---------------------------------------------------------------------------------------
// potential compilation (host)
// ---------------------------------------------------------------------------------------

// Row i of P(J_n / L) for P = sum_r a_r T_r, via the Chebyshev recurrence on row vectors
// rho_{r+1} = 2 rho_r (J_n / L) - rho_{r-1}, rho_0 = e_i (Eq. (ChebyshevRecurrence)); J_n is the
// truncated Jacobi matrix with J_{k,k+1} = J_{k+1,k} = sqrt((k+1)/2) (Eq. (Recurrence1D)).
static void poly_row(const std::vector<double> &a, double L, int i, int n, double *out /* 2p+1 */)
{
    int p = (int)a.size() - 1;
    int W = 2 * p + 3;  // window i-p-1 .. i+p+1 keeps the recurrence in range
    std::vector<double> r0(W, 0.0), r1(W, 0.0), r2(W, 0.0), row(W, 0.0);
    auto idx = [&](int m) { return m - (i - p - 1); };
    auto valid = [&](int m) { return m >= 0 && m < n && m >= i - p - 1 && m <= i + p + 1; };
    r0[idx(i)] = 1.0;
    auto times_J = [&](const std::vector<double> &x, std::vector<double> &y) {
        for (int m = i - p - 1; m <= i + p + 1; ++m) {
            double v = 0.0;
            if (valid(m)) {
                if (valid(m - 1)) v += x[idx(m - 1)] * sqrt(m / 2.0);
                if (valid(m + 1)) v += x[idx(m + 1)] * sqrt((m + 1) / 2.0);
            }
            y[idx(m)] = v;
        }
    };
    for (int m = 0; m < W; ++m) row[m] = a[0] * r0[m];
    if (p >= 1) {
        times_J(r0, r1);
        for (int m = 0; m < W; ++m) {
            r1[m] /= L;
            row[m] += a[1] * r1[m];
        }
    }
    for (int r = 2; r <= p; ++r) {
        times_J(r1, r2);
        for (int m = 0; m < W; ++m) {
            r2[m] = 2.0 * r2[m] / L - r0[m];
            row[m] += a[r] * r2[m];
        }
        r0.swap(r1);
        r1.swap(r2);
    }
    for (int s = -p; s <= p; ++s) out[s + p] = row[idx(i + s)];
}

static int parity_mask(const std::vector<double> &a)
{
    // T_r(J/L) has nonzero row entries only at offsets of the parity of r
    int p = (int)a.size() - 1;
    bool even = false, odd = false;
    for (int r = 0; r <= p; ++r)
        if (a[r] != 0.0) (r % 2 ? odd : even) = true;
    int mask = 0;
    for (int s = -p; s <= p; ++s) {
        bool sodd = (s % 2) != 0;
        if ((sodd && odd) || (!sodd && even)) mask |= 1 << (s + p);
    }
    return mask;
}

// Coefficients below 1e-15 of the largest one are round-off of exact zeros (interpolation of an
// even or odd function, elimination residue); they are set to zero, then trailing zeros dropped.
static void trim(std::vector<double> &a)
{
    double big = 0.0;
    for (double x : a) big = std::max(big, fabs(x));
    for (double &x : a)
        if (fabs(x) <= 1e-15 * big) x = 0.0;
    while (a.size() > 1 && a.back() == 0.0) a.pop_back();
}

struct PolyKey {
    std::vector<double> a;
    bool operator<(const PolyKey &o) const { return a < o.a; }
};

struct Compiler {
    const IndexSetObj *set;
    double L;
    std::map<PolyKey, int> poly_base;    // polynomial -> row-table base
    std::map<PolyKey, int> packed_base;  // polynomial -> packed row-table base
    std::vector<double> tab;             // all row tables (double)
    OpSet ops;                           // main stage
    OpSet ops1;                          // first stage (channel writers)
    std::vector<std::pair<int, std::vector<double>>> chans;   // (axis, normalised polynomial)
    std::vector<double> pw;

    int poly(const std::vector<double> &a)
    {
        auto it = poly_base.find(PolyKey{a});
        if (it != poly_base.end()) return it->second;
        int p = (int)a.size() - 1;
        int B = set->h.B;
        int base = (int)tab.size();
        tab.resize(tab.size() + (size_t)B * (p + 1) * (2 * p + 1));
        for (int i = 0; i < B; ++i)
            for (int d = 0; d <= p; ++d)
                poly_row(a, L, i, i + 1 + d, &tab[base + ((size_t)i * (p + 1) + d) * (2 * p + 1)]);
        poly_base[PolyKey{a}] = base;
        return base;
    }

    // Packed rows of a pure-parity polynomial of degree <= 8 (packed_width(p) entries per row,
    // 4-aligned base).
    int packed(const std::vector<double> &a)
    {
        auto it = packed_base.find(PolyKey{a});
        if (it != packed_base.end()) return it->second;
        int p = (int)a.size() - 1;
        int B = set->h.B;
        const int W = packed_width(p);
        tab.resize((tab.size() + 3) & ~(size_t)3, 0.0);
        int base = (int)tab.size();
        tab.resize(tab.size() + (size_t)B * (p + 1) * W, 0.0);
        double row[2 * kMaxDeg + 1];
        for (int i = 0; i < B; ++i)
            for (int d = 0; d <= p; ++d) {
                poly_row(a, L, i, i + 1 + d, row);
                for (int j = 0; j <= p; ++j) tab[base + ((size_t)i * (p + 1) + d) * W + j] = row[2 * j];
            }
        packed_base[PolyKey{a}] = base;
        return base;
    }

    // The second factor of a plane operator when it has degree 1: the rows of both fibre-top
    // distances side by side, tab[base + 4 i + 2 d + j] = [Q(J_n / L)]_{i, i-1+2j}, n = i + 1 + d,
    // so that one 4-entry load gives both (4-aligned base).
    std::map<PolyKey, int> pair_base;
    int packed_pairs(const std::vector<double> &a)
    {
        auto it = pair_base.find(PolyKey{a});
        if (it != pair_base.end()) return it->second;
        const int B = set->h.B;
        tab.resize((tab.size() + 3) & ~(size_t)3, 0.0);
        const int base = (int)tab.size();
        tab.resize(tab.size() + (size_t)B * 4, 0.0);
        double row[3];
        for (int i = 0; i < B; ++i)
            for (int d = 0; d <= 1; ++d) {
                poly_row(a, L, i, i + 1 + d, row);
                for (int j = 0; j <= 1; ++j) tab[base + (size_t)i * 4 + 2 * d + j] = row[2 * j];
            }
        pair_base[PolyKey{a}] = base;
        return base;
    }

    RowOffsets roff;                     // row offsets of both stages (0: zero offset)

    // Column of the row-offset table for the point k + s0 e_a0 + s1 e_a1 (moves along the last
    // axis stay in the row and need no column), or -1 when the table is full.
    int delta_index(int a0, int s0, int a1, int s1)
    {
        int N = set->h.N;
        int8_t e[4] = {-1, 0, -1, 0};
        int n = 0;
        if (a0 >= 0 && a0 < N - 1 && s0 != 0) { e[0] = (int8_t)a0; e[1] = (int8_t)s0; n = 1; }
        if (a1 >= 0 && a1 < N - 1 && s1 != 0) { e[2 * n] = (int8_t)a1; e[2 * n + 1] = (int8_t)s1; }
        if (e[0] < 0 && e[2] < 0) return 0;
        for (int i = 1; i < roff.n; ++i)
            if (!memcmp(roff.d[i], e, 4)) return i;
        if (roff.n >= kMaxDelta) return -1;
        memcpy(roff.d[roff.n], e, 4);
        return roff.n++;
    }

    // Appends an operator to S.  scale multiplies the term amplitude.
    int add_op(OpSet &S, int kind, int a, int b, const std::vector<double> &P, const std::vector<double> &Q,
               const hx_term &t, double scale, int src = -1, int dst = -1)
    {
        if (S.nops >= kMaxOps) {
            set_error("potential compiles to more than %d operators", kMaxOps);
            return HX_EUNSUPPORTED;
        }
        Op &o = S.op[S.nops];
        memset(&o, 0, sizeof(o));
        o.kind = kind;
        o.a = a;
        o.b = b;
        o.p = kind >= 1 ? (int)P.size() - 1 : 0;
        o.q = kind == 2 ? (int)Q.size() - 1 : 0;
        o.pmask = kind >= 1 ? parity_mask(P) : 1;
        o.qmask = kind == 2 ? parity_mask(Q) : 1;
        o.tabP = kind >= 1 ? poly(P) : 0;
        o.tabQ = kind == 2 ? poly(Q) : 0;
        o.src = src;
        o.dst = dst;
        o.mergeB = -1;
        o.merged = 0;
        {
            const int N = set->h.N;
            auto role = [N](int ax) { return ax < 0 ? ROLE_NONE : (ax == N - 1 ? ROLE_LAST : ROLE_ROW); };
            o.ra = role(kind >= 1 ? a : -1);
            o.rb = role(kind == 2 ? b : -1);
        }
        {
            auto pure = [](int mask, int deg) {   // only offsets of the parity of deg
                int want = 0;
                for (int s = -deg; s <= deg; s += 2) want |= 1 << (s + deg);
                return mask == want;
            };
            if (kind == 0) o.cls = CLS_ID;
            else if (kind == 1 && o.p <= kMaxDeg && pure(o.pmask, o.p)) o.cls = CLS_LINE + o.p;
            else if (kind == 2 && o.p <= 3 && o.q <= 3 && pure(o.pmask, o.p) && pure(o.qmask, o.q))
                o.cls = CLS_PLANE + 3 * (o.p - 1) + (o.q - 1);
            else o.cls = CLS_GENERIC;
            o.ptabP = o.ptabQ = 0;
            if (o.cls != CLS_ID && o.cls != CLS_GENERIC) {
                o.ptabP = packed(P);
                if (kind == 2) o.ptabQ = o.q == 1 ? packed_pairs(Q) : packed(Q);
            }
        }
        o.mod = t.mod_kind;
        o.amp = t.amp * scale;
        o.omega = t.omega;
        o.phase = t.phase;
        o.pw_off = (int)pw.size();
        o.pw_n = t.mod_kind == HX_MOD_PWCONST ? t.pw_n : 0;
        o.pw_t0 = t.pw_t0;
        o.pw_t1 = t.pw_t1;
        if (t.mod_kind == HX_MOD_PWCONST) pw.insert(pw.end(), t.pw_values, t.pw_values + t.pw_n);
        o.dbase = S.ndidx;
        if (kind >= 1) {
            int span = (2 * o.p + 1) * (2 * o.q + 1);
            if (S.ndidx + span > kMaxDidx) {
                set_error("potential footprint exceeds %d entries", kMaxDidx);
                return HX_EUNSUPPORTED;
            }
            for (int s = -o.p; s <= o.p; ++s)
                for (int s2 = -o.q; s2 <= o.q; ++s2) {
                    // only footprint points whose rows can be nonzero get a table column; a plane op
                    // on the last axis also looks up (s, 0), the row of k + s e_a
                    bool used = ((o.pmask >> (s + o.p)) & 1) &&
                                (((o.qmask >> (s2 + o.q)) & 1) || (s2 == 0 && o.rb == ROLE_LAST));
                    // a general set decides membership and fibre tops point by point: all positions
                    used = used || set->h.general;
                    if (!used) {
                        S.didx[o.dbase + (s + o.p) * (2 * o.q + 1) + (s2 + o.q)] = 0;
                        continue;
                    }
                    int di = delta_index(a, s, kind == 2 ? b : -1, s2);
                    if (di < 0) {
                        set_error("potential needs more than %d distinct neighbour offsets", kMaxDelta);
                        return HX_EUNSUPPORTED;
                    }
                    S.didx[o.dbase + (s + o.p) * (2 * o.q + 1) + (s2 + o.q)] = (uint8_t)di;
                }
            S.ndidx += span;
        }
        S.nops++;
        return HX_OK;
    }

    // Channel holding Pn(X_axis) c for a normalised polynomial Pn (created in stage 1 on first use).
    int channel(int axis, const std::vector<double> &Pn)
    {
        for (size_t i = 0; i < chans.size(); ++i) {
            if (chans[i].first != axis || chans[i].second.size() != Pn.size()) continue;
            bool same = true;
            for (size_t r = 0; r < Pn.size(); ++r) same &= fabs(chans[i].second[r] - Pn[r]) <= 1e-14;
            if (same) return (int)i;
        }
        hx_term unit;
        memset(&unit, 0, sizeof(unit));
        unit.mod_kind = HX_MOD_CONST;
        unit.amp = 1.0;
        int ch = (int)chans.size();
        if (add_op(ops1, 1, axis, -1, Pn, Pn, unit, 1.0, -1, ch)) return -1;
        chans.push_back({axis, Pn});
        return ch;
    }
};

// P = scale * Pn with the largest |coefficient| of Pn equal to 1.
static double normalise(const std::vector<double> &P, std::vector<double> &Pn)
{
    double big = 0.0;
    for (double x : P)
        if (fabs(x) > fabs(big)) big = x;
    Pn = P;
    for (double &x : Pn) x /= big;
    return big;
}

// C = sum_k u_k v_k^T by Gaussian elimination with complete pivoting; once the largest remaining
// entry is below 1e-13 * max|C| the rest is dropped (an exactly low-rank C, e.g. the interpolant of
// a product or a sum of products of univariate functions, leaves only round-off there).
static void rank_one_pieces(std::vector<double> C, int n0, int n1, std::vector<std::vector<double>> &U,
                            std::vector<std::vector<double>> &V)
{
    double cmax = 0.0;
    for (double x : C) cmax = std::max(cmax, fabs(x));
    if (cmax == 0.0) return;
    for (int it = 0; it < std::min(n0, n1); ++it) {
        int bi = -1, bj = -1;
        double best = 0.0;
        for (int i = 0; i < n0; ++i)
            for (int j = 0; j < n1; ++j)
                if (fabs(C[i * n1 + j]) > best) { best = fabs(C[i * n1 + j]); bi = i; bj = j; }
        if (best <= 1e-13 * cmax) break;
        std::vector<double> u(n0), v(n1);
        double piv = C[bi * n1 + bj];
        for (int i = 0; i < n0; ++i) u[i] = C[i * n1 + bj];
        for (int j = 0; j < n1; ++j) v[j] = C[bi * n1 + j] / piv;
        for (int i = 0; i < n0; ++i)
            for (int j = 0; j < n1; ++j) C[i * n1 + j] -= u[i] * v[j];
        U.push_back(u);
        V.push_back(v);
    }
}

// Lexicographic comparison of two coordinate prefixes of length n (<0, 0, >0).
static int memcmp_u16(const uint16_t *a, const uint16_t *b, int n)
{
    for (int i = 0; i < n; ++i)
        if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
    return 0;
}

static int compile_potential(Problem *pr, const hx_potential *pot)
{
    const IndexSetObj *set = pr->set;
    int N = set->h.N;
    if (!pot || !(pot->L > 0.0) || pot->n_terms < 0 || (pot->n_terms > 0 && !pot->terms)) {
        set_error("hx_potential_set: need L > 0 and a term array");
        return HX_EINVAL;
    }
    Compiler cp;
    cp.set = set;
    // basis phi_k(S x): with y = S x, A = S^2 D_K + (1/S^2 - S^2)/2 sum_l Y_l^2 + W(Y / S); W's
    // Chebyshev expansion in x / L is one in y / (S L), so the terms keep their coefficients on
    // [-S L, S L], and the quadratic term is a degree-2 line operator on every axis
    const double S = pr->scale;
    cp.L = pot->L * S;
    memset(&cp.ops, 0, sizeof(cp.ops));
    memset(&cp.ops1, 0, sizeof(cp.ops1));
    memset(&cp.roff, 0, sizeof(cp.roff));
    cp.roff.n = 1;   // column 0: zero offset
    cp.roff.d[0][0] = cp.roff.d[0][2] = -1;
    int order = pr->cfg.order;
    cp.ops.wAB = order == HX_ORDER_SYM ? 0.5 : (order == HX_ORDER_EQ ? 1.0 : 0.0);
    cp.ops.wBA = order == HX_ORDER_SYM ? 0.5 : (order == HX_ORDER_ALG ? 1.0 : 0.0);
    cp.ops.wAB32 = (float)cp.ops.wAB;
    cp.ops.wBA32 = (float)cp.ops.wBA;
    for (int ti = 0; ti < pot->n_terms; ++ti) {
        const hx_term &t = pot->terms[ti];
        if (t.n_axes < 1 || t.n_axes > 2) {
            set_error("term %d: n_axes = %d (this build supports 1 or 2)", ti, t.n_axes);
            return t.n_axes > 2 ? HX_EUNSUPPORTED : HX_EINVAL;
        }
        if (!t.coef || t.mod_kind < 0 || t.mod_kind > HX_MOD_PWCONST ||
            (t.mod_kind == HX_MOD_PWCONST && (!t.pw_values || t.pw_n < 1 || !(t.pw_t1 > t.pw_t0)))) {
            set_error("term %d: bad coefficient pointer or modulation", ti);
            return HX_EINVAL;
        }
        for (int i = 0; i < t.n_axes; ++i)
            if (t.axes[i] < 0 || t.axes[i] >= N || t.deg[i] < 0 || t.deg[i] > kMaxDeg ||
                (i == 1 && t.axes[1] <= t.axes[0])) {
                set_error("term %d: bad axes or degrees", ti);
                return HX_EINVAL;
            }
        int rc;
        if (t.n_axes == 1) {
            std::vector<double> a(t.coef, t.coef + t.deg[0] + 1);
            trim(a);
            if (a.size() == 1) {
                if (a[0] != 0.0 && (rc = cp.add_op(cp.ops, 0, -1, -1, a, a, t, a[0]))) return rc;
            } else if ((rc = cp.add_op(cp.ops, 1, t.axes[0], -1, a, a, t, 1.0))) return rc;
        } else {
            int n0 = t.deg[0] + 1, n1 = t.deg[1] + 1;
            std::vector<double> C(t.coef, t.coef + n0 * n1);
            std::vector<std::vector<double>> U, V;
            // Split by parity first: T_i T_j with i and j of fixed parities form four blocks, and each
            // block's rank-one pieces are polynomials of pure parity, which have specialised stencils
            // with half the footprint (e.g. the interpolant of cos(x_a - x_b) splits exactly into the
            // cos (x) cos and sin (x) sin pieces).  Blocks at round-off level are dropped.
            double cmax = 0.0;
            for (double x : C) cmax = std::max(cmax, fabs(x));
            for (int pi = 0; pi < 2; ++pi)
                for (int pj = 0; pj < 2; ++pj) {
                    std::vector<double> Cb(C.size(), 0.0);
                    double bmax = 0.0;
                    for (int i = pi; i < n0; i += 2)
                        for (int j = pj; j < n1; j += 2) {
                            Cb[i * n1 + j] = C[i * n1 + j];
                            bmax = std::max(bmax, fabs(C[i * n1 + j]));
                        }
                    if (bmax > 1e-14 * cmax) rank_one_pieces(Cb, n0, n1, U, V);
                }
            for (size_t k = 0; k < U.size(); ++k) {
                std::vector<double> P = U[k], Qp = V[k];
                trim(P);
                trim(Qp);
                if (P.size() == 1 && Qp.size() == 1) {
                    if ((rc = cp.add_op(cp.ops, 0, -1, -1, P, P, t, P[0] * Qp[0]))) return rc;
                } else if (P.size() == 1) {
                    for (double &x : Qp) x *= P[0];
                    if ((rc = cp.add_op(cp.ops, 1, t.axes[1], -1, Qp, Qp, t, 1.0))) return rc;
                } else if (Qp.size() == 1) {
                    for (double &x : P) x *= Qp[0];
                    if ((rc = cp.add_op(cp.ops, 1, t.axes[0], -1, P, P, t, 1.0))) return rc;
                } else {
                    int foot = __builtin_popcount(parity_mask(P)) * __builtin_popcount(parity_mask(Qp));
                    if (foot <= kDirectFootprint) {
                        if ((rc = cp.add_op(cp.ops, 2, t.axes[0], t.axes[1], P, Qp, t, 1.0))) return rc;
                    } else {   // two stages: P(X_a) (Q(X_b) c) and Q(X_b) (P(X_a) c) through channels
                        std::vector<double> Pn, Qn;
                        double sp = normalise(P, Pn), sq = normalise(Qp, Qn);
                        int chQ = cp.channel(t.axes[1], Qn), chP = cp.channel(t.axes[0], Pn);
                        if (chQ < 0 || chP < 0) return HX_EUNSUPPORTED;
                        if (cp.ops.wAB != 0.0 &&
                            (rc = cp.add_op(cp.ops, 1, t.axes[0], -1, P, P, t, sq * cp.ops.wAB, chQ))) return rc;
                        if (cp.ops.wBA != 0.0 &&
                            (rc = cp.add_op(cp.ops, 1, t.axes[1], -1, Qp, Qp, t, sp * cp.ops.wBA, chP))) return rc;
                    }
                }
            }
        }
    }
    if (S != 1.0) {
        const double c = 0.5 * (1.0 / (S * S) - S * S), L2 = cp.L * cp.L;
        const std::vector<double> quad = {0.5 * c * L2, 0.0, 0.5 * c * L2};   // c y^2 = c L^2 (T_0 + T_2) / 2
        hx_term unit;
        memset(&unit, 0, sizeof(unit));
        unit.mod_kind = HX_MOD_CONST;
        unit.amp = 1.0;
        for (int l = 0; l < N; ++l) {
            int rc = cp.add_op(cp.ops, 1, l, -1, quad, quad, unit, 1.0);
            if (rc) return rc;
        }
    }
    // A pure line op on the second axis of a pure plane op, with the parity of the plane op's second
    // polynomial and a degree of q or q + 2, shares the plane op's points k + s2 e_b: evaluate it
    // inside the plane op (one gather per shared point); it keeps its own weight.
    // (only when every op has degree <= 3: the kernel for higher degrees has no merged path; only
    // into plane ops with both degrees <= 2, the classes with a specialised plane stencil; and only
    // when the plane op's first degree is even, so that its stencil visits the points s = 0)
    int maxdeg = 0;
    for (int i = 0; i < cp.ops.nops; ++i) maxdeg = std::max(maxdeg, std::max(cp.ops.op[i].p, cp.ops.op[i].q));
    for (int i = 0; i < cp.ops.nops && maxdeg <= 3 && !set->h.general; ++i) {
        Op &o = cp.ops.op[i];
        if (o.kind != 2 || o.cls < CLS_PLANE || o.cls >= CLS_GENERIC || o.src >= 0) continue;
        if (o.p > 2 || o.q > 2 || o.p % 2) continue;
        for (int j = 0; j < cp.ops.nops; ++j) {
            Op &l = cp.ops.op[j];
            if (l.kind != 1 || l.merged || l.src >= 0 || l.a != o.b || l.cls != CLS_LINE + l.p) continue;
            if (!(l.p == o.q || (l.p == o.q + 2 && l.p <= 3))) continue;
            o.mergeB = j;
            l.merged = 1;
            break;
        }
    }
    // upload
    size_t es = pr->cfg.dtype == HX_C64 ? sizeof(float) : sizeof(double);
    size_t tab_bytes = std::max<size_t>(cp.tab.size(), 1) * es;
    if (tab_bytes > ((size_t)1 << 30)) {
        set_error("coefficient row tables need %zu bytes", tab_bytes);
        return HX_EUNSUPPORTED;
    }
    std::vector<char> stage(tab_bytes);
    if (pr->cfg.dtype == HX_C64) {
        float *f = (float *)stage.data();
        for (size_t i = 0; i < cp.tab.size(); ++i) f[i] = (float)cp.tab[i];
    } else if (!cp.tab.empty()) {
        memcpy(stage.data(), cp.tab.data(), cp.tab.size() * sizeof(double));
    }
    if (pr->tab) cudaFree(pr->tab);
    if (pr->pw_values) cudaFree(pr->pw_values);
    pr->tab = nullptr;
    pr->pw_values = nullptr;
    HX_CUDA(cudaMalloc(&pr->tab, tab_bytes), "cudaMalloc(row tables)");
    HX_CUDA(cudaMemcpy(pr->tab, stage.data(), tab_bytes, cudaMemcpyHostToDevice), "upload row tables");
    size_t pwb = std::max<size_t>(cp.pw.size(), 1) * sizeof(double);
    HX_CUDA(cudaMalloc((void **)&pr->pw_values, pwb), "cudaMalloc(pw)");
    if (!cp.pw.empty())
        HX_CUDA(cudaMemcpy(pr->pw_values, cp.pw.data(), cp.pw.size() * sizeof(double), cudaMemcpyHostToDevice),
                "upload pw");
    pr->tab_bytes = tab_bytes;
    pr->ops = cp.ops;
    pr->ops1 = cp.ops1;
    // channel vectors of the first stage
    if (pr->chan) cudaFree(pr->chan);
    pr->chan = nullptr;
    pr->nch = (int)cp.chans.size();
    {
        size_t es2 = pr->cfg.dtype == HX_C64 ? 8 : 16;
        size_t ld = (((size_t)set->h.size * es2 + 255) / 256) * 256 / es2;
        pr->chan_ld = ld;
        if (pr->nch) HX_CUDA(cudaMalloc(&pr->chan, ld * es2 * pr->nch), "cudaMalloc(channels)");
    }
    // split every row offset into its move on the group axes 0..N-3 and its step on axis N-2
    {
        RowOffsets &ro = cp.roff;
        ro.nom = 0;
        for (int d = 0; d < ro.n; ++d) {
            signed char om[4] = {-1, 0, -1, 0};
            int n = 0, s4 = 0;
            for (int i = 0; i < 2; ++i) {
                const int ax = ro.d[d][2 * i], st = ro.d[d][2 * i + 1];
                if (ax < 0) continue;
                if (ax == N - 2) s4 = st;
                else { om[2 * n] = (signed char)ax; om[2 * n + 1] = (signed char)st; ++n; }
            }
            int m = -1;
            if (n > 0) {
                for (int i = 0; i < ro.nom && m < 0; ++i)
                    if (!memcmp(ro.om[i], om, 4)) m = i;
                if (m < 0) { memcpy(ro.om[ro.nom], om, 4); m = ro.nom++; }
            }
            ro.mv[d].om = (short)m;
            ro.mv[d].s4 = (short)s4;
        }
    }
    // group-neighbour table: kept when the outer moves are those of the previous potential
    const IndexSetHost &h = set->h;
    bool same = pr->gnb && pr->roff.nom == cp.roff.nom && !memcmp(pr->roff.om, cp.roff.om, sizeof(cp.roff.om[0]) * cp.roff.nom);
    pr->roff = cp.roff;
    if (!same) {
        if (pr->gnb) cudaFree(pr->gnb);
        if (pr->gnbn) cudaFree(pr->gnbn);
        pr->gnb = pr->gnbn = nullptr;
        pr->gstride = (std::max(cp.roff.nom, 1) + 3) & ~3;   // 16-byte rows (the compiled kernels read them so)
        size_t bytes = (size_t)pr->gstride * std::max(h.ngroup, 1) * sizeof(int);
        HX_CUDA(cudaMalloc((void **)&pr->gnb, bytes), "cudaMalloc(group-neighbour table)");
        if (!h.general) {
            HX_CUDA(cudaMemsetAsync(pr->gnb, 0xff, bytes, pr->stream), "clear group-neighbour table");
            int rc = launch_groupnb(set->d, pr->roff, pr->gstride, pr->gnb, pr->stream);
            if (rc) return rc;
            HX_CUDA(cudaStreamSynchronize(pr->stream), "group-neighbour table");
        } else {
            // general set: the neighbour group of every group and outer move, found by binary search
            // over the groups' prefixes (k_0..k_{N-3}, in lexicographic order), with its row count
            HX_CUDA(cudaMalloc((void **)&pr->gnbn, bytes), "cudaMalloc(group row counts)");
            const int npre = N - 1, nout = std::max(N - 2, 0), G = h.ngroup;
            std::vector<int> first(bytes / sizeof(int), -1), rows(bytes / sizeof(int), 0);
            auto gprefix = [&](int g) { return h.row_k.data() + (size_t)h.gfirst[g] * npre; };
            std::vector<uint16_t> key(std::max(nout, 1));
            for (int g = 0; g < G; ++g) {
                for (int m = 0; m < cp.roff.nom; ++m) {
                    bool ok = true;
                    for (int l = 0; l < nout; ++l) {
                        int kl = gprefix(g)[l];
                        if (cp.roff.om[m][0] == l) kl += cp.roff.om[m][1];
                        if (cp.roff.om[m][2] == l) kl += cp.roff.om[m][3];
                        if (kl < 0 || kl > 65534) ok = false;
                        key[l] = (uint16_t)std::max(kl, 0);
                    }
                    if (!ok) continue;
                    int lo = 0, hi = G - 1, found = -1;
                    while (lo <= hi) {
                        const int mid = (lo + hi) / 2;
                        const int c = memcmp_u16(gprefix(mid), key.data(), nout);
                        if (c < 0) lo = mid + 1;
                        else if (c > 0) hi = mid - 1;
                        else { found = mid; break; }
                    }
                    if (found < 0) continue;
                    first[(size_t)g * pr->gstride + m] = h.gfirst[found];
                    rows[(size_t)g * pr->gstride + m] =
                        (found + 1 < G ? h.gfirst[found + 1] : h.nrow) - h.gfirst[found];
                }
            }
            HX_CUDA(cudaMemcpy(pr->gnb, first.data(), bytes, cudaMemcpyHostToDevice), "upload group-neighbour table");
            HX_CUDA(cudaMemcpy(pr->gnbn, rows.data(), bytes, cudaMemcpyHostToDevice), "upload group row counts");
        }
    }
    jit_prepare(pr);
    if (int rc = jit_fill_tops(pr)) return rc;
    pr->have_pot = true;
    pr->generation++;
    return HX_OK;
}

// Device copies of the index tables of s (one allocation), then the per-element records.
static int upload_set(IndexSetObj *s)
{
    const IndexSetHost &h = s->h;
    size_t b_info = (size_t)std::max(h.nrow, 1) * sizeof(int4);
    size_t b_k = std::max<size_t>(h.row_k.size(), 1) * sizeof(uint16_t);
    size_t b_of = (size_t)std::max<int64_t>(h.size, 1) * sizeof(int4);
    size_t b_qoff = (size_t)(h.B + 2) * sizeof(int);
    size_t b_Q = std::max<size_t>(h.Q.size(), 1) * sizeof(int);
    size_t b_nt = (size_t)(kNtSpan * h.B + 1) * sizeof(int);
    size_t b_rs = (size_t)(h.nrow + 1) * sizeof(int);
    size_t b_rg = (size_t)std::max(h.nrow, 1) * sizeof(int);
    size_t b_gf = (size_t)(h.ngroup + 1) * sizeof(int);
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t total = al(b_info) + al(b_k) + al(b_of) + al(b_qoff) + al(b_Q) + al(b_nt) + al(b_rs) + al(b_rg) + al(b_gf);
    cudaGetDevice(&s->device);
    cudaError_t e = cudaMalloc(&s->dmem, total);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(index tables)");
    char *base = (char *)s->dmem;
    int4 *d_info = (int4 *)base;
    base += al(b_info);
    uint16_t *d_k = (uint16_t *)base;
    base += al(b_k);
    int4 *d_of = (int4 *)base;
    base += al(b_of);
    int *d_qoff = (int *)base;
    base += al(b_qoff);
    int *d_Q = (int *)base;
    base += al(b_Q);
    int *d_nt = (int *)base;
    base += al(b_nt);
    int *d_rs = (int *)base;
    base += al(b_rs);
    int *d_rg = (int *)base;
    base += al(b_rg);
    int *d_gf = (int *)base;
    {
        std::vector<int> nt((size_t)kNtSpan * h.B + 1, 0);
        for (int x = 1; x <= h.B; ++x) nt[x] = h.B / x;
        e = cudaMemcpy(d_nt, nt.data(), b_nt, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemcpy(d_info, h.row_info.data(), (size_t)h.nrow * sizeof(int4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !h.row_k.empty())
        e = cudaMemcpy(d_k, h.row_k.data(), h.row_k.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_qoff, h.qoff.data(), b_qoff, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        std::vector<int> rs(h.nrow + 1);
        for (int r = 0; r < h.nrow; ++r) rs[r] = h.row_info[r].x;
        rs[h.nrow] = (int)h.size;
        e = cudaMemcpy(d_rs, rs.data(), b_rs, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemcpy(d_rg, h.rgrp.data(), (size_t)h.nrow * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        std::vector<int> gf(h.gfirst);
        gf.push_back(h.nrow);
        e = cudaMemcpy(d_gf, gf.data(), b_gf, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess && !h.Q.empty()) e = cudaMemcpy(d_Q, h.Q.data(), h.Q.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess || (e = cudaGetLastError()) != cudaSuccess) {
        cudaFree(s->dmem);
        s->dmem = nullptr;
        return cuda_fail(e, "upload index tables");
    }
    s->d.N = h.N;
    s->d.B = h.B;
    s->d.size = (int)h.size;
    s->d.nrow = h.nrow;
    s->d.qtotal = h.qtotal;
    s->d.row_info = d_info;
    s->d.row_k = d_k;
    s->d.elem = d_of;
    s->d.qoff = d_qoff;
    s->d.Q = d_Q;
    s->d.nt = d_nt;
    s->d.rstart = d_rs;
    s->d.rgrp = d_rg;
    s->d.gfirst = d_gf;
    s->d.ngroup = h.ngroup;
    s->d.general = h.general ? 1 : 0;
    int rc = launch_elem_info(s);
    if (rc) {
        cudaFree(s->dmem);
        s->dmem = nullptr;
        return rc;
    }
    // the host copies of the row tables are no longer needed (rank/unrank use Q and qoff, or the
    // sorted list); a general set keeps its row prefixes and groups for its group-neighbour tables
    std::vector<int4>().swap(s->h.row_info);
    std::vector<int>().swap(s->h.rgrp);
    if (!h.general) {
        std::vector<uint16_t>().swap(s->h.row_k);
        std::vector<int>().swap(s->h.gfirst);
    }
    return HX_OK;
}


}  // namespace hx

using namespace hx;

struct hx_indexset : IndexSetObj {};
struct hx_problem : Problem {};
struct hx_batch : Batch {};

extern "C" {

const char *hx_last_error(void) { return g_err; }

int hx_indexset_create(int N, int64_t B, hx_indexset **out)
{
    if (!out || N < 1 || N > kMaxN || B < 1) {
        set_error("hx_indexset_create: need 1 <= N <= %d, B >= 1, out != NULL", kMaxN);
        return HX_EINVAL;
    }
    *out = nullptr;
    if (B > 65535) {
        set_error("hx_indexset_create: B = %lld > 65535 is not supported", (long long)B);
        return HX_EUNSUPPORTED;
    }
    hx_indexset *s = new (std::nothrow) hx_indexset();
    if (!s) { set_error("out of host memory"); return HX_ENOMEM; }
    int rc = build_host_tables(N, (int)B, s->h);
    if (rc) { delete s; return rc; }
    int rc2 = upload_set(s);
    if (rc2) { delete s; return rc2; }
    *out = s;
    return HX_OK;
}

int hx_indexset_create_list(int N, int64_t count, const int32_t *k, hx_indexset **out)
{
    if (!out || N < 1 || N > kMaxN || !k) {
        set_error("hx_indexset_create_list: need 1 <= N <= %d, a list and out != NULL", kMaxN);
        return HX_EINVAL;
    }
    *out = nullptr;
    hx_indexset *s = new (std::nothrow) hx_indexset();
    if (!s) { set_error("out of host memory"); return HX_ENOMEM; }
    int rc = build_list_tables(N, count, k, s->h);
    if (!rc) rc = upload_set(s);
    if (rc) { delete s; return rc; }
    *out = s;
    return HX_OK;
}

int64_t hx_indexset_size(const hx_indexset *s) { return s ? s->h.size : -1; }

int hx_indexset_unrank(const hx_indexset *s, int64_t rank, int32_t *k_out)
{
    if (!s || !k_out) { set_error("hx_indexset_unrank: NULL argument"); return HX_EINVAL; }
    int rc = host_unrank(s->h, rank, k_out);
    if (rc) set_error("hx_indexset_unrank: rank %lld out of range", (long long)rank);
    return rc;
}

int64_t hx_indexset_rank(const hx_indexset *s, const int32_t *k)
{
    if (!s || !k) return -1;
    return host_rank(s->h, k);
}

int hx_indexset_export(const hx_indexset *s, int32_t *k_out)
{
    if (!s || !k_out) { set_error("hx_indexset_export: NULL argument"); return HX_EINVAL; }
    size_t bytes = (size_t)s->h.size * s->h.N * sizeof(int32_t);
    int32_t *d = nullptr;
    HX_CUDA(cudaMalloc((void **)&d, std::max<size_t>(bytes, 4)), "cudaMalloc(export)");
    int rc = launch_export(s, d, 0);
    if (!rc) {
        cudaError_t e = cudaMemcpy(k_out, d, bytes, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) rc = cuda_fail(e, "export copy");
    }
    cudaFree(d);
    return rc;
}

void hx_indexset_destroy(hx_indexset *s)
{
    if (!s) return;
    cudaFree(s->dmem);
    delete s;
}

int hx_problem_create(const hx_indexset *s, const hx_config *cfg, hx_problem **out)
{
    if (!s || !out) { set_error("hx_problem_create: NULL argument"); return HX_EINVAL; }
    *out = nullptr;
    hx_config c = {HX_C128, HX_ORDER_SYM, 7, nullptr, HX_SCHEME_EXPMPR, 0.0, 0.0};
    if (cfg) c = *cfg;
    if (!(c.scale == 0.0 || (c.scale >= 1e-3 && c.scale <= 1e3))) {
        set_error("hx_problem_create: scale S must be 0 (meaning 1) or in [1e-3, 1e3]");
        return HX_EINVAL;
    }
    if ((c.dtype != HX_C128 && c.dtype != HX_C64) || c.order < 0 || c.order > 2 || c.m < 1 || c.m > kMaxKrylov ||
        (c.scheme != HX_SCHEME_EXPMPR && c.scheme != HX_SCHEME_MAGNUS4) || !(c.tol >= 0.0 && c.tol <= 1.0)) {
        set_error("hx_problem_create: bad dtype, order, m (1..%d), scheme or tol (0..1)", kMaxKrylov);
        return HX_EINVAL;
    }
    hx_problem *p = new (std::nothrow) hx_problem();
    if (!p) { set_error("out of host memory"); return HX_ENOMEM; }
    p->set = s;
    p->cfg = c;
    p->scale = c.scale > 0.0 ? c.scale : 1.0;
    p->stream = (cudaStream_t)c.stream;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) { delete p; return cuda_fail(e, "hx_problem_create: no CUDA device"); }
    int rc = noalloc_bind(p->device);   // hx_norm_noalloc's scratch: bound here, where allocation is expected
    if (rc) { delete p; return rc; }
    e = cudaMalloc((void **)&p->dscal, 64 * sizeof(double));
    if (e != cudaSuccess) { delete p; return cuda_fail(e, "cudaMalloc(scalars)"); }
    if ((e = cudaMemset(p->dscal, 0, 64 * sizeof(double))) != cudaSuccess) {
        cudaFree(p->dscal);
        delete p;
        return cuda_fail(e, "hx_problem_create: clear scalars");
    }
    *out = p;
    return HX_OK;
}

void hx_problem_destroy(hx_problem *p)
{
    if (!p) return;
    if (p->stream) cudaStreamSynchronize(p->stream); else cudaDeviceSynchronize();
    krylov_free(p);
    cudaFree(p->tab);
    cudaFree(p->pw_values);
    cudaFree(p->gnb);
    cudaFree(p->gnbn);
    cudaFree(p->tops);
    cudaFree(p->chan);
    cudaFree(p->dscal);
    for (void *x : p->extra) cudaFree(x);
    delete p;
}

int hx_set_time(hx_problem *p, double t)
{
    if (!p) { set_error("hx_set_time: NULL problem"); return HX_EINVAL; }
    p->t_host = t;
    HX_CUDA(cudaMemcpyAsync(p->dscal, &t, sizeof(double), cudaMemcpyHostToDevice, p->stream), "set time");
    HX_CUDA(cudaStreamSynchronize(p->stream), "set time");
    return HX_OK;
}

int hx_get_time(const hx_problem *p, double *t)
{
    if (!p || !t) { set_error("hx_get_time: NULL argument"); return HX_EINVAL; }
    *t = p->t_host;
    return HX_OK;
}

int hx_potential_set(hx_problem *p, const hx_potential *pot, double t)
{
    if (!p) { set_error("hx_potential_set: NULL problem"); return HX_EINVAL; }
    if (p->stream) cudaStreamSynchronize(p->stream); else cudaDeviceSynchronize();
    int rc = compile_potential(p, pot);
    if (rc) return rc;
    krylov_free(p);   // cached graphs refer to the old potential
    return hx_set_time(p, t);
}

// Device vectors must be aligned to their element size (8 bytes for HX_C64, 16 for HX_C128).
static bool elem_aligned(const Problem *p, const void *x)
{
    return (uintptr_t)x % (p->cfg.dtype == HX_C64 ? 8 : 16) == 0;
}

// Whether the byte ranges [a, a + na) and [b, b + nb) share a byte.
static bool ranges_overlap(const void *a, size_t na, const void *b, size_t nb)
{
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return na > 0 && nb > 0 && x < y + nb && y < x + na;
}

static size_t vec_bytes(const Problem *p) { return (size_t)p->set->h.size * (p->cfg.dtype == HX_C64 ? 8 : 16); }

int hx_apply(hx_problem *p, const void *c_in, void *c_out)
{
    if (!p || !c_in || !c_out) { set_error("hx_apply: NULL argument"); return HX_EINVAL; }
    if (!p->have_pot) { set_error("hx_apply: call hx_potential_set first"); return HX_EINVAL; }
    if (c_in == c_out || ranges_overlap(c_in, vec_bytes(p), c_out, vec_bytes(p))) {
        set_error("hx_apply: c_in and c_out must not overlap");
        return HX_EINVAL;
    }
    if (!elem_aligned(p, c_in) || !elem_aligned(p, c_out)) {
        set_error("hx_apply: vectors must be aligned to the element size");
        return HX_EINVAL;
    }
    return launch_apply(p, c_in, c_out, p->dscal, 0.0, nullptr, p->stream);
}

int hx_apply_project(hx_problem *p, const void *c, void *y, const void *basis, size_t ld, int k, double *h)
{
    if (!p || !c || !y || !basis || !h) { set_error("hx_apply_project: NULL argument"); return HX_EINVAL; }
    if (!p->have_pot) { set_error("hx_apply_project: call hx_potential_set first"); return HX_EINVAL; }
    if (c == y) { set_error("hx_apply_project: c and y must not overlap"); return HX_EINVAL; }
    if (k < 0 || k >= kMaxFusedDots) { set_error("hx_apply_project: k must be in [0, %d)", kMaxFusedDots); return HX_EINVAL; }
    if (ld < (size_t)p->set->h.size) { set_error("hx_apply_project: ld below the vector length"); return HX_EINVAL; }
    {
        const size_t vb = vec_bytes(p), es = p->cfg.dtype == HX_C64 ? 8 : 16;
        const size_t bb = (size_t)k * ld * es + vb;   // vectors 0..k of the basis
        if (ranges_overlap(c, vb, y, vb) || ranges_overlap(y, vb, basis, bb)) {
            set_error("hx_apply_project: y must overlap neither c nor the basis");
            return HX_EINVAL;
        }
    }
    if (!elem_aligned(p, c) || !elem_aligned(p, y) || !elem_aligned(p, basis) || (uintptr_t)h % 8) {
        set_error("hx_apply_project: vectors must be aligned to the element size");
        return HX_EINVAL;
    }
    return apply_project_dispatch(p, c, y, basis, ld, k, h);
}

int hx_apply_host(hx_problem *p, const void *c_in_host, void *c_out_host)
{
    if (!p || !c_in_host || !c_out_host) { set_error("hx_apply_host: NULL argument"); return HX_EINVAL; }
    size_t es = p->cfg.dtype == HX_C64 ? 8 : 16;
    size_t bytes = (size_t)p->set->h.size * es;
    void *d = nullptr;
    HX_CUDA(cudaMallocAsync(&d, 2 * std::max<size_t>(bytes, 16), p->stream), "cudaMallocAsync(apply_host)");
    char *din = (char *)d, *dout = (char *)d + std::max<size_t>(bytes, 16);
    int rc = HX_OK;
    cudaError_t e = cudaMemcpyAsync(din, c_in_host, bytes, cudaMemcpyHostToDevice, p->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "apply_host copy in");
    if (!rc) rc = hx_apply(p, din, dout);
    if (!rc && (e = cudaMemcpyAsync(c_out_host, dout, bytes, cudaMemcpyDeviceToHost, p->stream)) != cudaSuccess)
        rc = cuda_fail(e, "apply_host copy out");
    cudaFreeAsync(d, p->stream);
    if ((e = cudaStreamSynchronize(p->stream)) != cudaSuccess && !rc) rc = cuda_fail(e, "apply_host sync");
    return rc;
}

int hx_energy(hx_problem *p, const void *c, double *out)
{
    if (!p || !c || !out) { set_error("hx_energy: NULL argument"); return HX_EINVAL; }
    if (!p->have_pot) { set_error("hx_energy: call hx_potential_set first"); return HX_EINVAL; }
    if (!elem_aligned(p, c)) { set_error("hx_energy: vector must be aligned to the element size"); return HX_EINVAL; }
    const size_t es = p->cfg.dtype == HX_C64 ? 8 : 16;
    const size_t bytes = std::max<size_t>((size_t)p->set->h.size * es, 16);
    char *buf = nullptr;   // y = A c, then h_0 = <c, y> (two doubles)
    const size_t hoff = ((bytes + 255) / 256) * 256;
    HX_CUDA(cudaMallocAsync((void **)&buf, hoff + 256, p->stream), "cudaMallocAsync(energy)");
    double *h = (double *)(buf + hoff);
    int rc = apply_rayleigh_dispatch(p, c, buf, h);
    double hv[2] = {0.0, 0.0};
    if (!rc) {
        cudaError_t e = cudaMemcpyAsync(hv, h, sizeof(hv), cudaMemcpyDeviceToHost, p->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "hx_energy");
    }
    cudaFreeAsync(buf, p->stream);
    cudaStreamSynchronize(p->stream);
    *out = hv[0];
    return rc;
}

int hx_apply_rayleigh(hx_problem *p, const void *c, void *y, double *r)
{
    if (!p || !c || !y || !r) { set_error("hx_apply_rayleigh: NULL argument"); return HX_EINVAL; }
    if (!p->have_pot) { set_error("hx_apply_rayleigh: call hx_potential_set first"); return HX_EINVAL; }
    if (!elem_aligned(p, c) || !elem_aligned(p, y) || (uintptr_t)r % 8) {
        set_error("hx_apply_rayleigh: vectors must be aligned to the element size and r to 8 bytes");
        return HX_EINVAL;
    }
    const size_t bytes = (size_t)p->set->h.size * (p->cfg.dtype == HX_C64 ? 8 : 16);
    if (ranges_overlap(c, bytes, y, bytes) || ranges_overlap(c, bytes, r, 16) || ranges_overlap(y, bytes, r, 16)) {
        set_error("hx_apply_rayleigh: c, y and r must not overlap");
        return HX_EINVAL;
    }
    return apply_rayleigh_dispatch(p, c, y, r);
}

int hx_norm(hx_problem *p, const void *c, double *out)
{
    if (!p || !c || !out) { set_error("hx_norm: NULL argument"); return HX_EINVAL; }
    if (!elem_aligned(p, c)) { set_error("hx_norm: vector must be aligned to the element size"); return HX_EINVAL; }
    int G = apply_grid(p);
    double *buf = nullptr;
    HX_CUDA(cudaMallocAsync((void **)&buf, (G + 2) * sizeof(double) + 64, p->stream), "cudaMallocAsync(norm)");
    unsigned *cnt = (unsigned *)(buf + G + 1);
    cudaMemsetAsync(cnt, 0, sizeof(unsigned), p->stream);
    int rc = launch_norm(p, c, p->cfg.dtype == HX_C128, buf, cnt, buf + G, p->stream);
    double r = 0.0;
    if (!rc) {
        cudaError_t e = cudaMemcpyAsync(&r, buf + G, sizeof(double), cudaMemcpyDeviceToHost, p->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "hx_norm");
    }
    cudaFreeAsync(buf, p->stream);
    cudaStreamSynchronize(p->stream);
    *out = sqrt(r);
    if (!rc && !isfinite(*out)) {
        set_error("hx_norm: the norm is not finite (the vector holds a NaN or an infinity, or overflows)");
        rc = HX_ENONFINITE;
    }
    return rc;
}

int hx_step(hx_problem *p, void *c, double dt, int nsteps)
{
    if (!p || !c || nsteps < 0 || !(dt == dt)) { set_error("hx_step: bad argument"); return HX_EINVAL; }
    if (!p->have_pot) { set_error("hx_step: call hx_potential_set first"); return HX_EINVAL; }
    if ((uintptr_t)c % 16) { set_error("hx_step: the complex128 state must be 16-byte aligned"); return HX_EINVAL; }
    if (nsteps == 0) return HX_OK;
    return krylov_step(p, c, dt, nsteps);
}

int hx_step_host(hx_problem *p, void *c_host, double dt, int nsteps)
{
    if (!p || !c_host) { set_error("hx_step_host: NULL argument"); return HX_EINVAL; }
    if (!p->have_pot) { set_error("hx_step_host: call hx_potential_set first"); return HX_EINVAL; }
    size_t bytes = (size_t)p->set->h.size * 16;
    void *d = krylov_host_state(p);
    if (!d) { set_error("hx_step_host: cannot allocate the device state"); return HX_ENOMEM; }
    int rc = HX_OK;
    cudaError_t e = cudaMemcpyAsync(d, c_host, bytes, cudaMemcpyHostToDevice, p->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "step_host copy in");
    if (!rc) rc = hx_step(p, d, dt, nsteps);
    if (!rc && (e = cudaMemcpyAsync(c_host, d, bytes, cudaMemcpyDeviceToHost, p->stream)) != cudaSuccess)
        rc = cuda_fail(e, "step_host copy out");
    if ((e = cudaStreamSynchronize(p->stream)) != cudaSuccess && !rc) rc = cuda_fail(e, "step_host sync");
    return rc;
}

// One step with potentials re-interpolated for it (the time-propagation algorithm, step (1)):
// the potential at the integrator's evaluation times replaces the problem's, then one hx_step.
static int reinterp_one_step(hx_problem *p, void *c, double dt, hx_potential_fn fn, void *user)
{
    HX_CUDA(cudaStreamSynchronize(p->stream), "hx_step_reinterp");   // no kernel reads the old tables
    const double t = p->t_host;
    int rc;
    if (p->cfg.scheme == HX_SCHEME_MAGNUS4 && dt != 0.0) {
        // A(t + c1 dt) from the first potential, A(t + c2 dt) from the second: each term is switched
        // on over its half of the step interval by a two-interval piecewise-constant modulation (the
        // Gauss-Legendre points c1 < 1/2 < c2 lie inside the two halves; for dt < 0 the first point
        // lies in the upper half of [t + dt, t))
        const double c1 = 0.5 - sqrt(3.0) / 6.0, c2 = 0.5 + sqrt(3.0) / 6.0;
        const bool fwd = dt > 0.0;
        static const double first[2] = {1.0, 0.0}, second[2] = {0.0, 1.0};
        std::vector<hx_term> terms;
        std::vector<std::vector<double>> coefs;   // copies: the first potential may not outlive the next call
        double L = 0.0;
        for (int g = 0; g < 2; ++g) {
            const hx_potential *pot = fn(t + (g ? c2 : c1) * dt, user);
            if (!pot || (pot->n_terms > 0 && !pot->terms) || pot->n_terms < 0) {
                set_error("hx_step_reinterp: the potential callback returned no potential at t = %g", t);
                return HX_EINVAL;
            }
            if (g == 0) L = pot->L;
            else if (pot->L != L) {
                set_error("hx_step_reinterp: the two Gauss-point potentials have different L");
                return HX_EINVAL;
            }
            for (int i = 0; i < pot->n_terms; ++i) {
                hx_term tm = pot->terms[i];
                if (tm.mod_kind != HX_MOD_CONST) {
                    set_error("hx_step_reinterp: with HX_SCHEME_MAGNUS4 every term must be HX_MOD_CONST (term %d)", i);
                    return HX_EINVAL;
                }
                if (!tm.coef || tm.n_axes < 1 || tm.n_axes > 2 || tm.deg[0] < 0 || tm.deg[0] > kMaxDeg ||
                    (tm.n_axes == 2 && (tm.deg[1] < 0 || tm.deg[1] > kMaxDeg))) {
                    set_error("hx_step_reinterp: term %d: bad coefficients, axes or degrees", i);
                    return HX_EINVAL;
                }
                const int nc = (tm.deg[0] + 1) * (tm.n_axes == 2 ? tm.deg[1] + 1 : 1);
                coefs.emplace_back(tm.coef, tm.coef + nc);
                tm.mod_kind = HX_MOD_PWCONST;
                tm.pw_values = (g == 0) == fwd ? first : second;
                tm.pw_n = 2;
                tm.pw_t0 = fwd ? t : t + dt;
                tm.pw_t1 = fwd ? t + dt : t;
                terms.push_back(tm);
            }
        }
        for (size_t i = 0; i < terms.size(); ++i) terms[i].coef = coefs[i].data();
        hx_potential both = {L, (int)terms.size(), terms.data()};
        rc = compile_potential(p, &both);
    } else {   // the exponential midpoint rule (and a Magnus step of length 0: both points at t)
        const hx_potential *pot = fn(t + 0.5 * dt, user);
        if (!pot) {
            set_error("hx_step_reinterp: the potential callback returned no potential at t = %g", t);
            return HX_EINVAL;
        }
        rc = compile_potential(p, pot);
    }
    if (rc) return rc;
    krylov_invalidate(p);   // the captured step refers to the previous tables
    return hx_step(p, c, dt, 1);
}

int hx_step_reinterp(hx_problem *p, void *c, double dt, int nsteps, hx_potential_fn fn, void *user)
{
    if (!p || !c || !fn || nsteps < 0 || !(dt == dt)) { set_error("hx_step_reinterp: bad argument"); return HX_EINVAL; }
    if ((uintptr_t)c % 16) { set_error("hx_step_reinterp: the complex128 state must be 16-byte aligned"); return HX_EINVAL; }
    for (int n = 0; n < nsteps; ++n) {
        int rc = reinterp_one_step(p, c, dt, fn, user);
        if (rc) return rc;
    }
    return HX_OK;
}

int hx_batch_create(hx_problem *const *probs, int n, hx_batch **out)
{
    if (!probs || n < 1 || !out) { set_error("hx_batch_create: need n >= 1 problems and out != NULL"); return HX_EINVAL; }
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        if (!probs[i] || !probs[i]->have_pot) {
            set_error("hx_batch_create: problem %d is NULL or has no potential", i);
            return HX_EINVAL;
        }
        for (int j = 0; j < i; ++j)
            if (probs[j] == probs[i]) { set_error("hx_batch_create: problem %d appears twice", i); return HX_EINVAL; }
    }
    hx_batch *b = new (std::nothrow) hx_batch();
    if (!b) { set_error("out of host memory"); return HX_ENOMEM; }
    b->probs.assign(probs, probs + n);
    b->stream = probs[0]->stream;
    *out = b;
    return HX_OK;
}

int hx_batch_step(hx_batch *b, void *const *c, double dt, int nsteps)
{
    if (!b || !c || nsteps < 0 || !(dt == dt)) { set_error("hx_batch_step: bad argument"); return HX_EINVAL; }
    const size_t np = b->probs.size();
    for (size_t i = 0; i < np; ++i)
        if (!c[i] || (uintptr_t)c[i] % 16) { set_error("hx_batch_step: state %zu is NULL or not 16-byte aligned", i); return HX_EINVAL; }
    // the members run concurrently: no two may step the same memory
    std::vector<std::pair<uintptr_t, uintptr_t>> span(np);
    for (size_t i = 0; i < np; ++i)
        span[i] = {(uintptr_t)c[i], (uintptr_t)c[i] + (uintptr_t)b->probs[i]->set->h.size * 16};
    std::vector<size_t> ord(np);
    for (size_t i = 0; i < np; ++i) ord[i] = i;
    std::sort(ord.begin(), ord.end(), [&](size_t x, size_t y) { return span[x].first < span[y].first; });
    for (size_t j = 1; j < np; ++j)
        if (span[ord[j]].first < span[ord[j - 1]].second) {
            set_error("hx_batch_step: the states of problems %zu and %zu overlap", ord[j - 1], ord[j]);
            return HX_EINVAL;
        }
    if (nsteps == 0) return HX_OK;
    int rc = batch_step(b, c, dt, nsteps);
    if (rc || b->budget < 0) return rc;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "hx_batch_step");
    if (batch_timed_out(b)) {
        set_error("hx_batch_step: a batched product ran out of its budget; the states are incomplete");
        return HX_ETIMEOUT;
    }
    return HX_OK;
}

int hx_batch_set_budget(hx_batch *b, double seconds)
{
    if (!b || !(seconds == seconds)) { set_error("hx_batch_set_budget: bad argument"); return HX_EINVAL; }
    long long cycles = -1;
    if (seconds >= 0.0) {
        int dev = 0, khz = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
        if (e != cudaSuccess) return cuda_fail(e, "hx_batch_set_budget");
        const double c = seconds * 1e3 * (double)khz;        // the SM clock counts clock64 ticks
        cycles = c > 9.0e18 ? (long long)9.0e18 : (long long)c;
    }
    if (cycles != b->budget) {
        if (b->stream) cudaStreamSynchronize(b->stream);
        batch_drop_graphs(b);                              // the budget is a launch argument
    }
    b->budget = cycles;
    b->budget_s = seconds >= 0.0 ? seconds : -1.0;
    return HX_OK;
}

int hx_batch_info(const hx_batch *b, hx_batch_stats *out)
{
    if (!b || !out) { set_error("hx_batch_info: NULL argument"); return HX_EINVAL; }
    memset(out, 0, sizeof(*out));
    out->schedule = b->schedule;
    out->tile = b->tile;
    out->launches = b->schedule >= 0 ? b->kern[b->schedule] : 0;
    const int n = std::min((int)b->tune_tiles.size(), 8);
    out->ntiles = n;
    for (int i = 0; i < n; ++i) {
        out->tiles[i] = b->tune_tiles[i];
        out->tile_ms[i] = (float)b->tune_ms[i];
    }
    for (int s = 0; s < kNumSched; ++s) out->step_ms[s] = b->sched_ms[s];
    return HX_OK;
}

void hx_batch_destroy(hx_batch *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream); else cudaDeviceSynchronize();
    batch_free(b);
    delete b;
}

int hx_apply_specialised(const hx_problem *p)
{
    if (!p) { set_error("hx_apply_specialised: NULL problem"); return HX_EINVAL; }
    if (!p->have_pot) { set_error("hx_apply_specialised: call hx_potential_set first"); return HX_EINVAL; }
    set_error("%s", p->jit_reason.c_str());
    return p->jit ? 1 : 0;
}

int hx_step_launches(const hx_problem *p, int *per_apply, int *per_step)
{
    if (!p) { set_error("hx_step_launches: NULL problem"); return HX_EINVAL; }
    if (!p->have_pot) { set_error("hx_step_launches: call hx_potential_set first"); return HX_EINVAL; }
    const int a = apply_launches(p);
    if (per_apply) *per_apply = a;
    const int m = p->cfg.m;
    // expMPR: the product kernel computes the projections itself when it is specialised (m <= 8)
    const int dots = m <= kMaxFusedDots && apply_fuses_dots(p) ? 0 : 1;
    // Gram-Schmidt per Lanczos vector: one sweep for m <= 8, else two passes (the second pass of the
    // last vector only with an error tolerance); then the start vector, the exponential and the
    // recombination, and with a tolerance the error estimate
    const bool sweep = m <= kMaxFusedDots;
    const int gs = sweep ? 1 : 2;
    const int fixed = sweep ? 3 : 2;
    const int est = p->cfg.tol > 0.0 ? (sweep ? 1 : 2) : 0;
    // 2-stage Magnus: A_1 v and A_2 v in one launch, A_2 A_1 v and A_1 A_2 v in another, with the
    // specialised kernel (the second launch also forms H v), else four products and a combination;
    // then the projections and the Gram-Schmidt launches
    const int mag = (apply_dual(p) ? 2 * a : 4 * a + 1) + 1 + gs;
    if (per_step) *per_step = (p->cfg.scheme == HX_SCHEME_MAGNUS4 ? m * mag : m * (a + gs + dots)) + fixed + est;
    return HX_OK;
}

int hx_step_info(hx_problem *p, int *m_used, double *alpha, double *beta, double *norm)
{
    if (!p) { set_error("hx_step_info: NULL problem"); return HX_EINVAL; }
    return krylov_info(p, m_used, alpha, beta, norm);
}

int hx_step_substeps(hx_problem *p, int *last, int64_t *total, double *err_max)
{
    if (!p) { set_error("hx_step_substeps: NULL problem"); return HX_EINVAL; }
    long long tot = 0;
    int rc = krylov_substeps(p, last, &tot, err_max);
    if (!rc && total) *total = tot;
    return rc;
}

int hx_cheb_nodes(int R, double *u_out)
{
    if (R < 0 || !u_out) { set_error("hx_cheb_nodes: bad argument"); return HX_EINVAL; }
    for (int i = 0; i <= R; ++i) u_out[i] = cos(M_PI * (2 * i + 1) / (2.0 * R + 2.0));
    return HX_OK;
}

// a_r = (2 - delta_{r0}) / (R + 1) sum_i f(u_i) cos(r theta_i), theta_i = pi (2i + 1) / (2R + 2):
// discrete orthogonality of T_r at the first-kind nodes (Sec. 1.3).
int hx_cheb_coeffs(int R, int dims, const double *values, double *coef_out)
{
    if (R < 0 || (dims != 1 && dims != 2) || !values || !coef_out) {
        set_error("hx_cheb_coeffs: bad argument");
        return HX_EINVAL;
    }
    int n = R + 1;
    std::vector<double> Cm((size_t)n * n);
    for (int r = 0; r < n; ++r)
        for (int i = 0; i < n; ++i)
            Cm[(size_t)r * n + i] = (r == 0 ? 1.0 : 2.0) / n * cos(r * M_PI * (2 * i + 1) / (2.0 * n));
    if (dims == 1) {
        for (int r = 0; r < n; ++r) {
            double s = 0.0;
            for (int i = 0; i < n; ++i) s += Cm[(size_t)r * n + i] * values[i];
            coef_out[r] = s;
        }
        return HX_OK;
    }
    std::vector<double> tmp((size_t)n * n, 0.0);
    for (int r = 0; r < n; ++r)
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int i = 0; i < n; ++i) s += Cm[(size_t)r * n + i] * values[(size_t)i * n + j];
            tmp[(size_t)r * n + j] = s;
        }
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) {
            double s = 0.0;
            for (int j = 0; j < n; ++j) s += tmp[(size_t)r * n + j] * Cm[(size_t)c * n + j];
            coef_out[(size_t)r * n + c] = s;
        }
    return HX_OK;
}

// x^p on [-L, L]: (L u)^p with u^p = 2^{1-p} sum_{j <= p/2} binom(p, j) T_{p-2j}(u), the j = p/2 term halved.
int hx_cheb_monomial(int p, double L, double *coef_out)
{
    if (p < 0 || p > 60 || !coef_out) { set_error("hx_cheb_monomial: bad argument"); return HX_EINVAL; }
    for (int r = 0; r <= p; ++r) coef_out[r] = 0.0;
    double binom = 1.0;
    for (int j = 0; 2 * j <= p; ++j) {
        double c = binom * ldexp(1.0, 1 - p);
        if (2 * j == p) c *= 0.5;
        coef_out[p - 2 * j] += c * pow(L, p);
        binom = binom * (p - j) / (j + 1);
    }
    return HX_OK;
}

}  // extern "C"
