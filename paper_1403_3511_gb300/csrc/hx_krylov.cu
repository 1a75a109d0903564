// Time stepping: the exponential midpoint rule c^{n+1} = exp(-i h A(t^n + h/2)) c^n (Eq. (expMPR),
// Sec. 2.1) with the exponential approximated by an m-step Hermitian Lanczos process,
// c^{n+1} = ||c^n|| V_m exp(-i h T_m) e_1 (Sec. 2.2), entirely on the device.
//
// One step is a fixed sequence of kernels (captured once into a CUDA graph and replayed):
//   init      v_0 = c (in the Krylov dtype), beta_0 = ||c|| (FP64)
//   for k = 0 .. m-1:
//     apply   w = A(t + h/2) v_k                              (hx_apply.cu)
//     dot     h_i = <v_i, w>, i <= k                            (FP64; done by the apply kernel
//                                                                when it is specialised, m <= 8)
//     update  w -= sum_i h_i v_i;  h'_i = <v_i, w>               (FP64)
//     update  w -= sum_i h'_i v_i; beta_k = ||w||, v_{k+1} = w / beta_k   (k < m-1)
//     alpha_k = Re(h_k + h'_k)
//   eig       T_m = Q diag(lambda) Q^T (cyclic Jacobi, FP64), y = beta_0 Q exp(-i h lambda) Q^T e_1
//   combine   c = sum_i y_i v_i  (complex128 accumulation)
// Classical Gram-Schmidt applied twice keeps V_m orthonormal to working precision.  Vectors are
// stored unnormalised with a device scale s_k (v_k = s_k * stored_k) so no pass is spent on
// normalisation.  All scalars live in device memory, so the step has no host round trip.
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <type_traits>

#include "hx_internal.h"
#include "hx_convert.h"
#include "hx_stencil.cuh"   // reduce_partials, kMaxFusedDots

namespace hx {

struct Scal {                       // device scalars of one problem
    double t;                       // problem time (shared with hx_apply)
    double beta0;
    double s[kMaxKrylov + 1];       // vector scales
    double alpha[kMaxKrylov];
    double beta[kMaxKrylov];
    double h[2 * (kMaxKrylov + 1)];
    double h2[2 * (kMaxKrylov + 1)];
    double y[2 * kMaxKrylov];
    double Q[kMaxKrylov * kMaxKrylov];   // eigenvectors of T_m (row-major, m_used x m_used)
    double lam[kMaxKrylov];              // eigenvalues of T_m
    double scale;                   // running max_i(|alpha_i| + beta_{i-1}) for the breakdown test
    double norm_out;
    double err_max;                 // largest a-posteriori error estimate since it was last cleared
    double t_save;                  // problem time at the start of an adaptive step (restored on retry)
    // one-sweep Gram-Schmidt (m <= 8): p_j = <v_j, u_k> of the next vector's first-pass direction
    // u_k = s_k V_k against the finished v_j, and nu = ||u_k - sum_j p_j v_j|| (see sweep_k_kernel)
    double p[2 * kMaxFusedDots];
    double nu;
    int m_used;
    int flags;                      // bit 0: breakdown seen, bit 1: non-finite, bit 2: eigensolver stalled
    unsigned counter;
};

struct Work {
    Scal *sc;
    void *V;                        // (m + 1) x n vectors of the Krylov dtype
    double2 *state;                 // complex128 state the captured graph reads and writes
    double2 *host_state;            // device buffer used by hx_step_host
    double *partials;               // G x 2 (m + 2)
    void *mag;                      // HX_SCHEME_MAGNUS4: 4 vectors of the Krylov dtype (A_1 v, A_2 v, A_2 A_1 v, A_1 A_2 v)
    size_t vec_bytes;
    cudaGraphExec_t exec;
    cudaStream_t cap_stream;
    double dt;
    // automatic sub-steps (hx_config.tol > 0)
    double2 *backup;                // state at the start of the step being attempted
    double *err_host;               // page-locked copy of err_max
    int sub;                        // sub-steps per step for the next step
    int sub_last;                   // sub-steps of the last accepted step
    long long sub_total;            // sub-steps of the last hx_step call
    double err_last;                // largest estimate of the last hx_step call
    int steps_last;                 // steps of the last hx_step call
};

static Work *work_of(Problem *p) { return (Work *)p->krylov; }

// Set while a batch graph is captured.  Batch members run the generic apply kernel: one 32-problem
// batch with the kernels specialised per potential stopped with cudaErrorInvalidAddressSpace, which
// bounds-checked copies of the same kernels did not reproduce; until the cause is known, batch graphs
// keep the kernel they were validated with.
thread_local bool g_batch_capture = false;

// Grid of a streaming kernel: one wave of resident blocks (a second, partial wave would run at a
// fraction of the occupancy and take as long as the first), at most apply_grid(p) blocks (the
// size of the partial-sum buffers).
template <typename K>
static int resident_grid(const Problem *p, K kernel, int threads)
{
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1) per_sm = 1;
    return std::max(1, std::min(apply_grid(p), p->num_sms * per_sm));
}



// Error-free transformations (Knuth's TwoSum, and TwoProd with a fused multiply-add) and the
// compensated dot product built from them (Ogita, Rump and Oishi, "Accurate sum and dot product",
// 2005, Algorithm Dot2): the float result is as accurate as if accumulated in twice the precision.
struct F2 {
    float s = 0.f, c = 0.f;
    __device__ void add_prod(float a, float b)
    {
        float p = a * b;
        float e = fmaf(a, b, -p);
        float t = s + p;
        float bb = t - s;
        float q = (s - (t - bb)) + (p - bb);
        s = t;
        c += q + e;
    }
    __device__ double value() const { return (double)s + (double)c; }
};

// sum x^2 over FP64 values x without FP64 arithmetic for the usual magnitudes: x = hi + lo split
// into binary32 parts with integer operations (hx_convert.h), hi^2 + 2 hi lo accumulated as a
// compensated FP32 pair (relative error of order 2^-44).  Magnitudes in [2^-174, 2^-74) go to a
// second pair scaled by 2^200 (x by 2^100), the rest (tinier, or 2^100 and above) to FP64.
struct NormAcc {
    F2 a, b;
    double rest = 0.0;
    // adds x^2 and returns x rounded to binary32 (to nearest, ties to even)
    __device__ float add(double x)
    {
        float h, l;
        if (d2f_split(x, h, l)) {
            a.add_prod(h, h);
            a.c = fmaf(2.f * h, l, a.c);
            return h;
        }
        const uint64_t bx = conv_bits64(x);
        const uint32_t e = (uint32_t)(bx >> 52) & 0x7ffu;
        if (e - (1023u - 174u) < 100u && d2f_split(conv_from_bits64(bx + (100ull << 52)), h, l)) {
            b.add_prod(h, h);
            b.c = fmaf(2.f * h, l, b.c);
        } else {
            rest = fma(x, x, rest);
        }
        return d2f_rn(x);
    }
    __device__ double value() const { return a.value() + 0x1p-200 * b.value() + rest; }
};

// v_0 = c in the Krylov dtype; beta_0 = ||c||, s_0 = 1 / beta_0.  For complex64 vectors the
// rounding to binary32 and the norm use integer and FP32 operations only (NormAcc).
template <typename V>
__global__ void init_kernel(const double2 *c, V *v0, int n, double *partials, Scal *sc, int m)
{
    double acc = 0.0;
    if constexpr (std::is_same<V, float2>::value) {
        NormAcc na;   // two elements per thread and iteration: 32 bytes in, one 16-byte store out
        const int gid = blockIdx.x * blockDim.x + threadIdx.x, gstride = gridDim.x * blockDim.x;
        for (int q = gid; q < (n >> 1); q += gstride) {
            const double2 x = c[2 * q], y = c[2 * q + 1];
            const float xr = na.add(x.x), xi = na.add(x.y), yr = na.add(y.x), yi = na.add(y.y);
            *reinterpret_cast<float4 *>(v0 + 2 * q) = make_float4(xr, xi, yr, yi);
        }
        if ((n & 1) && gid == 0) {
            const double2 x = c[n - 1];
            const float xr = na.add(x.x), xi = na.add(x.y);
            v0[n - 1] = make_float2(xr, xi);
        }
        acc = na.value();
    } else {
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
            const double2 x = c[i];
            v0[i] = x;
            acc += x.x * x.x + x.y * x.y;
        }
    }
    __shared__ double tot[1];
    if (reduce_partials(&acc, 1, partials, &sc->counter, tot) && threadIdx.x == 0) {
        double b0 = sqrt(tot[0]);
        sc->beta0 = b0;
        sc->s[0] = b0 > 0.0 ? 1.0 / b0 : 0.0;
        sc->m_used = b0 > 0.0 ? m : 0;
        sc->scale = 0.0;
        if (!isfinite(b0)) sc->flags |= 2;
        sc->counter = 0;
    }
}

// Per-thread accumulator of Re/Im conj(v) w: compensated FP32 (Dot2) for complex64 vectors, FP64 for
// complex128 vectors.
template <typename V> struct CAcc;
template <> struct CAcc<float2> {
    F2 re, im;
    __device__ void add(float2 v, float2 w)
    {
        re.add_prod(v.x, w.x);
        re.add_prod(v.y, w.y);
        im.add_prod(v.x, w.y);
        im.add_prod(-v.y, w.x);
    }
    __device__ double r() const { return re.value(); }
    __device__ double i() const { return im.value(); }
};
template <> struct CAcc<double2> {
    double re = 0.0, im = 0.0;
    __device__ void add(double2 v, double2 w)
    {
        re = fma(v.x, w.x, fma(v.y, w.y, re));
        im = fma(v.x, w.y, fma(-v.y, w.x, im));
    }
    __device__ double r() const { return re; }
    __device__ double i() const { return im; }
};

// Accumulator of Re/Im conj(v) w over pairs of elements: the four products of a pair are summed
// with fused multiply-adds (a few ulp of their magnitudes) and the pair sums are accumulated
// with TwoSum compensation, so the rounding does not grow with the number of elements; about a
// third of the work of Dot2 on every product.  Used by the paired loops for complex64 vectors.
struct TwoSumAcc {
    float s = 0.f, c = 0.f;
    __device__ void add(float p)
    {
        const float t = s + p, bb = t - s;
        c += (s - (t - bb)) + (p - bb);
        s = t;
    }
    __device__ double value() const { return (double)s + (double)c; }
};
struct PairAcc {
    TwoSumAcc re, im;
    __device__ void add(float2 va, float2 wa, float2 vb, float2 wb)
    {
        re.add(fmaf(va.x, wa.x, fmaf(va.y, wa.y, fmaf(vb.x, wb.x, vb.y * wb.y))));
        im.add(fmaf(va.x, wa.y, fmaf(-va.y, wa.x, fmaf(vb.x, wb.y, -vb.y * wb.x))));
    }
    __device__ void add(float2 v, float2 w) { add(v, w, make_float2(0.f, 0.f), make_float2(0.f, 0.f)); }
    __device__ double r() const { return re.value(); }
    __device__ double i() const { return im.value(); }
};
// complex128 vectors keep FP64 accumulation
template <typename V> struct PairAccOf { using T = PairAcc; };
template <> struct PairAccOf<double2> { using T = CAcc<double2>; };
template <typename A, typename V>
__device__ __forceinline__ void add_pair(A &acc, const V &va, const V &wa, const V &vb, const V &wb)
{
    if constexpr (std::is_same<A, PairAcc>::value) acc.add(va, wa, vb, wb);
    else { acc.add(va, wa); acc.add(vb, wb); }
}

template <typename V> struct Real;
template <> struct Real<float2> { using T = float; };
template <> struct Real<double2> { using T = double; };

// Elements e and e + 1 of a vector (e even; vectors start on 256-byte boundaries): one 16-byte
// access for complex64, two for complex128.  Two elements per thread and iteration keep twice as
// many bytes in flight per thread as one.
template <typename V> struct Pair { V a, b; };
__device__ __forceinline__ Pair<float2> load_pair(const float2 *p, int e)
{
    const float4 q = *reinterpret_cast<const float4 *>(p + e);
    return {make_float2(q.x, q.y), make_float2(q.z, q.w)};
}
__device__ __forceinline__ Pair<double2> load_pair(const double2 *p, int e) { return {p[e], p[e + 1]}; }
__device__ __forceinline__ void store_pair(float2 *p, int e, const Pair<float2> &x)
{
    *reinterpret_cast<float4 *>(p + e) = make_float4(x.a.x, x.a.y, x.b.x, x.b.y);
}
__device__ __forceinline__ void store_pair(double2 *p, int e, const Pair<double2> &x)
{
    p[e] = x.a;
    p[e + 1] = x.b;
}

// x -= (cr + i ci) v in the vector precision
template <typename V, typename R>
__device__ __forceinline__ void sub_scaled(V &x, R cr, R ci, const V &v)
{
    x.x -= cr * v.x - ci * v.y;
    x.y -= cr * v.y + ci * v.x;
}

__host__ __device__ constexpr int pow2_at_least(int x) { return x <= 1 ? 1 : 2 * pow2_at_least((x + 1) / 2); }
__host__ __device__ constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x / 2); }

// Warp sums of NV compensated FP32 values s_j + c_j (NV a power of two, at most 32) by a butterfly
// reduce-scatter in FP32 pairs: in each of the first log2 NV rounds a lane keeps half of its
// values and adds its partner's copy of them with TwoSum, the remaining rounds add up the one
// value left; lane l then holds value l >> (5 - log2 NV).  One lane per value and warp writes it
// as FP64 to wsum[warp][j] (j < nval).  On this GPU an FP64 add costs about as much as 64 FP32
// operations, so this replaces 5 FP64 shuffle-adds per value and thread.
template <int NV, int NMAX>
__device__ __forceinline__ void warp_pair_sums(float (&s)[NV], float (&c)[NV], int nval, double (*wsum)[NMAX])
{
    const int lane = threadIdx.x & 31;
    int o = 16;
#pragma unroll
    for (int half = NV / 2; half >= 1; half >>= 1, o >>= 1) {
        const bool hi = (lane & o) != 0;
#pragma unroll
        for (int j = 0; j < half; ++j) {
            const float ks = hi ? s[j + half] : s[j], kc = hi ? c[j + half] : c[j];
            const float xs = hi ? s[j] : s[j + half], xc = hi ? c[j] : c[j + half];
            const float rs = __shfl_xor_sync(0xffffffffu, xs, o), rc = __shfl_xor_sync(0xffffffffu, xc, o);
            const float t = ks + rs, bb = t - ks;
            c[j] = kc + rc + ((ks - (t - bb)) + (rs - bb));
            s[j] = t;
        }
    }
#pragma unroll
    for (; o >= 1; o >>= 1) {
        const float rs = __shfl_xor_sync(0xffffffffu, s[0], o), rc = __shfl_xor_sync(0xffffffffu, c[0], o);
        const float t = s[0] + rs, bb = t - s[0];
        c[0] = c[0] + rc + ((s[0] - (t - bb)) + (rs - bb));
        s[0] = t;
    }
    constexpr int sh = 5 - ilog2(NV);
    const int j = lane >> sh;
    if ((lane & ((1 << sh) - 1)) == 0 && j < nval) wsum[threadIdx.x >> 5][j] = (double)s[0] + (double)c[0];
}

// h_i = s_i <v_i, w> for i <= k.
// proj = 1 (projection onto a finished basis): k is clipped to the vectors actually built.
template <typename V, int NV>
__global__ void __launch_bounds__(256) dot_kernel(const V *w, const V *Vb, size_t ld, int n, int k, double *partials, Scal *sc,
                                                  int proj = 0)
{
    __shared__ double tot[2 * NV];
    if (proj) k = min(k, sc->m_used - 1);
    if (k < 0 || k >= sc->m_used) return;
    using A = typename std::conditional<(NV <= 8), typename PairAccOf<V>::T, CAcc<V>>::type;
    A acc[NV];
    const int gid = blockIdx.x * blockDim.x + threadIdx.x, gstride = gridDim.x * blockDim.x;
    if constexpr (NV <= 8) {
        for (int q = gid; q < (n >> 1); q += gstride) {
            const int e = 2 * q;
            const Pair<V> x = load_pair(w, e);
            Pair<V> v[NV];
#pragma unroll
            for (int i = 0; i < NV; ++i)
                if (i <= k) v[i] = load_pair(Vb + i * ld, e);
#pragma unroll
            for (int i = 0; i < NV; ++i)
                if (i <= k) add_pair(acc[i], v[i].a, x.a, v[i].b, x.b);
        }
        if ((n & 1) && gid == 0) {                          // odd length: the last element
            const V x = w[n - 1];
#pragma unroll
            for (int i = 0; i < NV; ++i)
                if (i <= k) acc[i].add(Vb[i * ld + n - 1], x);
        }
    } else {
        for (int e = gid; e < n; e += gstride) {
            const V x = w[e];
            for (int i = 0; i < NV; ++i)
                if (i <= k) acc[i].add(Vb[i * ld + e], x);
        }
    }
    const int nval = 2 * (k + 1);
    bool done;
    if constexpr (std::is_same<V, float2>::value && NV <= 8) {   // warp sums in FP32 pairs
        float ps[2 * NV], pc[2 * NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            ps[2 * i] = acc[i].re.s;
            pc[2 * i] = acc[i].re.c;
            ps[2 * i + 1] = acc[i].im.s;
            pc[2 * i + 1] = acc[i].im.c;
        }
        __shared__ double wsum[8][2 * NV];
        warp_pair_sums<2 * NV>(ps, pc, nval, wsum);
        __syncthreads();
        done = reduce_warp_sums<2 * NV>(wsum, nval, partials, &sc->counter, tot);
    } else {
        double vals[2 * NV];
#pragma unroll(NV <= 8 ? NV : 1)
        for (int i = 0; i < NV; ++i) {
            vals[2 * i] = acc[i].r();
            vals[2 * i + 1] = acc[i].i();
        }
        done = reduce_partials(vals, nval, partials, &sc->counter, tot);
    }
    if (done && threadIdx.x == 0) {
        for (int i = 0; i <= k; ++i) {
            sc->h[2 * i] = sc->s[i] * tot[2 * i];
            sc->h[2 * i + 1] = sc->s[i] * tot[2 * i + 1];
        }
        sc->counter = 0;
    }
}

// After the grid reduction of an update pass (last block, thread 0): pass 0 stores h'_i and
// alpha_k = Re(h_k + h'_k) and tracks the scale of T; pass 1 stores beta_k = ||w|| and
// s_{k+1} = 1 / beta_k, or stops the process at an invariant subspace.
template <int pass>
__device__ void update_scalars(Scal *sc, int k, const double *tot)
{
    if (pass == 0) {
        for (int i = 0; i <= k; ++i) {
            sc->h2[2 * i] = sc->s[i] * tot[2 * i];
            sc->h2[2 * i + 1] = sc->s[i] * tot[2 * i + 1];
        }
        double a = sc->h[2 * k] + sc->h2[2 * k];
        sc->alpha[k] = a;
        double sc_k = fabs(a) + (k > 0 ? sc->beta[k - 1] : 0.0);
        if (sc_k > sc->scale) sc->scale = sc_k;
    } else {
        double b = sqrt(tot[0]);
        if (!isfinite(b)) sc->flags |= 2;
        if (b <= 1e-13 * sc->scale) {       // invariant subspace: stop with k + 1 vectors
            if (k + 1 < sc->m_used) {
                sc->m_used = k + 1;
                sc->flags |= 1;
            } else {                        // the pass after the last vector (error estimate): exact
                sc->beta[k] = 0.0;
            }
        } else {
            sc->beta[k] = b;
            sc->s[k + 1] = 1.0 / b;
        }
    }
    sc->counter = 0;
}

// pass 0: w -= sum_i h_i s_i v_i, then h'_i = s_i <v_i, w>, alpha_k = Re(h_k + h'_k).
// pass 1: w -= sum_i h'_i s_i v_i, then beta_k = ||w||, s_{k+1} = 1 / beta_k, breakdown test.
// The update runs in the vector precision; the inner products and the norm as in dot_kernel.
// Every v_i is read once per element (the values are kept for the inner products).
template <typename V, int NV, int pass>
__global__ void __launch_bounds__(256, (sizeof(V) == 8 && NV <= 8) ? 3 : 1) update_kernel(V *w, const V *Vb, size_t ld, int n, int k, double *partials, Scal *sc)
{
    using R = typename Real<V>::T;
    __shared__ double tot[2 * NV];
    if (k >= sc->m_used) return;
    const double *coef = pass == 0 ? sc->h : sc->h2;
    R cr[NV], ci[NV];
#pragma unroll(NV <= 8 ? NV : 1)
    for (int i = 0; i < NV; ++i) {
        cr[i] = i <= k ? (R)(coef[2 * i] * sc->s[i]) : (R)0;
        ci[i] = i <= k ? (R)(coef[2 * i + 1] * sc->s[i]) : (R)0;
    }
    using A = typename std::conditional<(NV <= 8), typename PairAccOf<V>::T, CAcc<V>>::type;
    A acc[NV];
    A nrm;
    const int gid = blockIdx.x * blockDim.x + threadIdx.x, gstride = gridDim.x * blockDim.x;
    if constexpr (NV <= 8) {
        for (int q = gid; q < (n >> 1); q += gstride) {
            const int e = 2 * q;
            Pair<V> x = load_pair(w, e);
            Pair<V> v[NV];
#pragma unroll
            for (int i = 0; i < NV; ++i)
                if (i <= k) v[i] = load_pair(Vb + i * ld, e);
#pragma unroll
            for (int i = 0; i < NV; ++i)
                if (i <= k) {
                    sub_scaled(x.a, cr[i], ci[i], v[i].a);
                    sub_scaled(x.b, cr[i], ci[i], v[i].b);
                }
            store_pair(w, e, x);
            if constexpr (pass == 0) {
#pragma unroll
                for (int i = 0; i < NV; ++i)
                    if (i <= k) add_pair(acc[i], v[i].a, x.a, v[i].b, x.b);
            } else {
                add_pair(nrm, x.a, x.a, x.b, x.b);
            }
        }
        if ((n & 1) && gid == 0) {                          // odd length: the last element
            const int e = n - 1;
            V x = w[e];
            V v[NV];
#pragma unroll
            for (int i = 0; i < NV; ++i)
                if (i <= k) {
                    v[i] = Vb[i * ld + e];
                    sub_scaled(x, cr[i], ci[i], v[i]);
                }
            w[e] = x;
            if constexpr (pass == 0) {
#pragma unroll
                for (int i = 0; i < NV; ++i)
                    if (i <= k) acc[i].add(v[i], x);
            } else {
                nrm.add(x, x);
            }
        }
    } else {
        for (int e = gid; e < n; e += gstride) {
            V x = w[e];
            for (int i = 0; i < NV; ++i)
                if (i <= k) sub_scaled(x, cr[i], ci[i], Vb[i * ld + e]);
            w[e] = x;
            if constexpr (pass == 0) {
                for (int i = 0; i <= k && i < NV; ++i) acc[i].add(Vb[i * ld + e], x);
            } else {
                nrm.add(x, x);
            }
        }
    }
    double vals[2 * NV];
    int nval;
    if (pass == 0) {
#pragma unroll(NV <= 8 ? NV : 1)
        for (int i = 0; i < NV; ++i) {
            vals[2 * i] = acc[i].r();
            vals[2 * i + 1] = acc[i].i();
        }
        nval = 2 * (k + 1);
    } else {
        vals[0] = nrm.r();
        nval = 1;
    }
    if (reduce_partials(vals, nval, partials, &sc->counter, tot) && threadIdx.x == 0) update_scalars<pass>(sc, k, tot);
}

// out = *scale <u, z> (re, im), skipped when k >= *m_used (m_used may be null): the Rayleigh quotient
// of a Lanczos step whose product launch does not compute it (u = V_k, z = A u_k, scale = s_k), and
// of hx_apply_rayleigh.  paired: u and z 16-byte aligned (two elements per 16-byte load).
template <typename V>
__global__ void __launch_bounds__(256) rayleigh_kernel(const V *u, const V *z, int n, bool paired, const double *scale,
                                                      const int *m_used, int k, double *out, double *partials,
                                                      unsigned *counter)
{
    __shared__ double tot[2];
    if (m_used && k >= *m_used) return;
    typename PairAccOf<V>::T acc;
    const int gid = blockIdx.x * blockDim.x + threadIdx.x, gstride = gridDim.x * blockDim.x;
    if (paired) {
        for (int q = gid; q < (n >> 1); q += gstride) {
            const Pair<V> a = load_pair(u, 2 * q), x = load_pair(z, 2 * q);
            add_pair(acc, a.a, x.a, a.b, x.b);
        }
        if ((n & 1) && gid == 0) acc.add(u[n - 1], z[n - 1]);
    } else {
        for (int e = gid; e < n; e += gstride) acc.add(u[e], z[e]);
    }
    const double vals[2] = {acc.r(), acc.i()};
    if (reduce_partials<2>(vals, 2, partials, counter, tot) && threadIdx.x == 0) {
        out[0] = *scale * tot[0];
        out[1] = *scale * tot[1];
        *counter = 0;
    }
}

// Lanczos index K < 8 in one sweep over the vectors: classical Gram-Schmidt in which the second
// pass of each vector is done by the sweep of the next index.  On entry slot K holds V_K with
// u_K = s_K V_K, the first-pass direction of the K-th vector (unit norm), the finished v_j = V_j
// (j < K, s_j = 1), sc->p_j = <v_j, u_K> and sc->nu = ||u_K - sum_j p_j v_j|| from the sweep of
// index K - 1, and slot K + 1 holds z = A u_K with r = sc->h_0 = <u_K, z> from the product launch
// (or rayleigh_kernel).  The sweep writes
//   v_K = (u_K - sum_{j<K} p_j v_j) / nu                                 (second pass of v_K)
//   w   = (z - sum_{j<K} q_j v_j) / nu - c_K v_K,  c_K = (r - sum_j conj(p_j) q_j) / nu^2,
// which is A v_K - sum_{j<=K} <v_j, A v_K> v_j (first pass of the next vector): A v_K = (z - sum_j
// p_j A v_j) / nu, and the Krylov relation A v_j = beta_{j-1} v_{j-1} + alpha_j v_j + beta_j v_{j+1}
// (A Hermitian) gives both <v_K, A v_{K-1}> = beta_{K-1} and q_j = <v_j, z> = <A v_j, u_K> =
// beta_{j-1} p_{j-1} + alpha_j p_j + beta_j p_{j+1} (p_K read as nu), so the coefficients collapse
// to those above and z's only measured projection is r.  The terms the three-term relation drops
// are of the size of the rounding; what they leave in w, like the rounding itself, is removed by the
// measured second pass.  The sweep also sums d_l = <v_l, w> (l <= K) and ||w||^2.  Then
// h_K = <v_K, A v_K> = c_K - p_{K-1} beta_{K-1} / nu and, as with two passes per vector,
// alpha_K = Re(h_K + d_K); the next direction is u_{K+1} = w / ||w|| with p'_l = d_l / ||w||,
// nu' = sqrt(1 - sum |p'_l|^2) and beta_K = ||w|| nu'.  In exact arithmetic alpha, beta and the v's
// are those of two full passes per vector; each basis vector is read once per Lanczos index instead
// of three times (the projections of z and two update passes).
template <typename V, int K>
constexpr int sweep_k_blocks()   // resident blocks per SM that keep the kernel free of spills
{
    return sizeof(V) == 8 ? (K < 5 ? 3 : 2) : (K < 3 ? 2 : 1);
}

constexpr int kSweepVals = 2 * kMaxFusedDots + 2;   // d_l (re, im), l < 8, and ||w||^2

template <typename V, int K>
__global__ void __launch_bounds__(256, sweep_k_blocks<V, K>()) sweep_k_kernel(V *Vb, size_t ld, int n, double *partials,
                                                                                 Scal *sc)
{
    constexpr int NK = K + 1, NVAL = 2 * NK + 1;
    constexpr int U = K + 3 >= 5 ? 1 : (K + 3 >= 3 ? 2 : 4);
    using R = typename Real<V>::T;
    __shared__ double tot[kSweepVals];
    __shared__ double cf[4 * NK + 2];   // b_j (j < K), c_i (i <= K) as re, im pairs; a; 1 / nu
    if (K >= sc->m_used) return;
    if (threadIdx.x == 0) {
        const double nu = K == 0 ? 1.0 : sc->nu, inv = 1.0 / nu;
        double cr = sc->h[0], ci = sc->h[1];                        // r - sum_j conj(p_j) q_j
        for (int j = 0; j < K; ++j) {
            const double pr = sc->p[2 * j], pi = sc->p[2 * j + 1];
            // q_j = beta_{j-1} p_{j-1} + alpha_j p_j + beta_j p_{j+1}, p_K = nu
            double qr = sc->alpha[j] * pr, qi = sc->alpha[j] * pi;
            if (j > 0) {
                qr += sc->beta[j - 1] * sc->p[2 * (j - 1)];
                qi += sc->beta[j - 1] * sc->p[2 * (j - 1) + 1];
            }
            if (j + 1 < K) {
                qr += sc->beta[j] * sc->p[2 * (j + 1)];
                qi += sc->beta[j] * sc->p[2 * (j + 1) + 1];
            } else {
                qr += sc->beta[j] * nu;
            }
            cf[2 * j] = pr * inv;
            cf[2 * j + 1] = pi * inv;
            cf[2 * K + 2 * j] = qr * inv;
            cf[2 * K + 2 * j + 1] = qi * inv;
            cr -= pr * qr + pi * qi;
            ci -= pr * qi - pi * qr;
        }
        cf[4 * K] = cr * inv * inv;
        cf[4 * K + 1] = ci * inv * inv;
        cf[4 * K + 2] = sc->s[K] * inv;
        cf[4 * K + 3] = inv;
    }
    __syncthreads();
    R br[K > 0 ? K : 1], bi[K > 0 ? K : 1], cr[NK], ci[NK];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        br[j] = (R)cf[2 * j];
        bi[j] = (R)cf[2 * j + 1];
    }
#pragma unroll
    for (int i = 0; i < NK; ++i) {
        cr[i] = (R)cf[2 * K + 2 * i];
        ci[i] = (R)cf[2 * K + 2 * i + 1];
    }
    const R a = (R)cf[4 * K + 2], inv = (R)cf[4 * K + 3];
    V *const uk = Vb + (size_t)K * ld, *const zk = Vb + (size_t)(K + 1) * ld;
    using A = typename PairAccOf<V>::T;
    A acc[NK];
    A nrm;
    const int npair = n >> 1;
    const int gid = blockIdx.x * blockDim.x + threadIdx.x, gstride = gridDim.x * blockDim.x;
    auto element = [&](V u, V z, const V *v, V &vk, V &w) {
        vk.x = a * u.x;
        vk.y = a * u.y;
#pragma unroll
        for (int j = 0; j < K; ++j) sub_scaled(vk, br[j], bi[j], v[j]);
        w.x = inv * z.x;
        w.y = inv * z.y;
#pragma unroll
        for (int j = 0; j < K; ++j) sub_scaled(w, cr[j], ci[j], v[j]);
        sub_scaled(w, cr[K], ci[K], vk);
    };
    for (int q0 = gid; q0 < npair; q0 += U * gstride) {
        Pair<V> x[U], y[U], v[U][K > 0 ? K : 1];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int q = q0 + u * gstride;
            if (q < npair) {
                x[u] = load_pair(uk, 2 * q);
                y[u] = load_pair(zk, 2 * q);
#pragma unroll
                for (int j = 0; j < K; ++j) v[u][j] = load_pair(Vb + j * ld, 2 * q);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int q = q0 + u * gstride;
            if (q < npair) {
                V va[K > 0 ? K : 1], vb[K > 0 ? K : 1];
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    va[j] = v[u][j].a;
                    vb[j] = v[u][j].b;
                }
                Pair<V> vk, w;
                element(x[u].a, y[u].a, va, vk.a, w.a);
                element(x[u].b, y[u].b, vb, vk.b, w.b);
                store_pair(uk, 2 * q, vk);
                store_pair(zk, 2 * q, w);
#pragma unroll
                for (int j = 0; j < K; ++j) add_pair(acc[j], va[j], w.a, vb[j], w.b);
                add_pair(acc[K], vk.a, w.a, vk.b, w.b);
                add_pair(nrm, w.a, w.a, w.b, w.b);
            }
        }
    }
    if ((n & 1) && gid == 0) {                              // odd length: the last element
        const int e = n - 1;
        V v[K > 0 ? K : 1];
#pragma unroll
        for (int j = 0; j < K; ++j) v[j] = Vb[j * ld + e];
        V vk, w;
        element(uk[e], zk[e], v, vk, w);
        uk[e] = vk;
        zk[e] = w;
#pragma unroll
        for (int j = 0; j < K; ++j) acc[j].add(v[j], w);
        acc[K].add(vk, w);
        nrm.add(w, w);
    }
    bool last;
    if constexpr (std::is_same<V, float2>::value) {
        // the 2 (K + 1) projections and the norm: warp sums in FP32 pairs, one FP64 value per warp
        constexpr int NV = pow2_at_least(NVAL);
        float ps[NV], pc[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            ps[i] = 0.f;
            pc[i] = 0.f;
        }
#pragma unroll
        for (int i = 0; i < NK; ++i) {
            ps[2 * i] = acc[i].re.s;
            pc[2 * i] = acc[i].re.c;
            ps[2 * i + 1] = acc[i].im.s;
            pc[2 * i + 1] = acc[i].im.c;
        }
        ps[2 * NK] = nrm.re.s;
        pc[2 * NK] = nrm.re.c;
        __shared__ double wsum[8][kSweepVals];
        warp_pair_sums<NV>(ps, pc, NVAL, wsum);
        __syncthreads();
        last = reduce_warp_sums<kSweepVals>(wsum, NVAL, partials, &sc->counter, tot);
    } else {
        double vals[NVAL];
#pragma unroll
        for (int i = 0; i < NK; ++i) {
            vals[2 * i] = acc[i].r();
            vals[2 * i + 1] = acc[i].i();
        }
        vals[2 * NK] = nrm.r();
        last = reduce_partials<kSweepVals>(vals, NVAL, partials, &sc->counter, tot);
    }
    if (last && threadIdx.x == 0) {
        const double nu = K == 0 ? 1.0 : sc->nu;
        const double nw = sqrt(tot[2 * NK]);
        // h_K = c_K - p_{K-1} beta_{K-1} / nu (real part), alpha_K = Re(h_K + d_K)
        double hk = cf[4 * K];
        if (K > 0) hk -= sc->p[2 * (K - 1)] * sc->beta[K - 1] / nu;
        const double a_k = hk + tot[2 * K];
        sc->alpha[K] = a_k;
        const double sc_k = fabs(a_k) + (K > 0 ? sc->beta[K - 1] : 0.0);
        if (sc_k > sc->scale) sc->scale = sc_k;
        sc->s[K] = 1.0;                                      // v_K is stored normalised
        double pp = 0.0;
        for (int l = 0; l < NK; ++l) {
            const double pr = tot[2 * l] / nw, pi = tot[2 * l + 1] / nw;
            sc->p[2 * l] = pr;
            sc->p[2 * l + 1] = pi;
            pp += pr * pr + pi * pi;
        }
        const double nu1 = sqrt(fmax(1.0 - pp, 0.0)), b = nw * nu1;
        if (!isfinite(b)) sc->flags |= 2;
        if (b <= 1e-13 * sc->scale) {                        // invariant subspace: stop with K + 1 vectors
            if (K + 1 < sc->m_used) {
                sc->m_used = K + 1;
                sc->flags |= 1;
            } else {                                         // after the last vector (error estimate): exact
                sc->beta[K] = 0.0;
            }
        } else {
            sc->beta[K] = b;
            sc->s[K + 1] = 1.0 / nw;
            sc->nu = nu1;
        }
        sc->counter = 0;
    }
}

// T_m = Q diag(lambda) Q^T by the implicit-shift QL iteration for symmetric tridiagonal matrices
// (Bowdler, Martin, Reinsch and Wilkinson, "The QR and QL algorithms for symmetric matrices",
// Numer. Math. 11, 1968): a shift from the leading 2 x 2 block, then a chase of plane rotations
// from the bottom of the unreduced block up; an off-diagonal entry is zero once it is below
// 2^-53 (|d_i| + |d_{i+1}|).  One warp: every lane runs the same scalar recurrence (so all lanes
// agree on every rotation) and applies each rotation to its own row of Q.
// y = beta_0 Q exp(-i h lambda) Q^T e_1, stored as y_i * s_i for the combination pass; also
// advances the problem time by h.
__device__ void eig_warp(Scal *sc, double h)
{
    const int lane = threadIdx.x;
    const int m = sc->m_used;
    double d[kMaxKrylov], e[kMaxKrylov], z[kMaxKrylov];   // diagonal, off-diagonal (i, i+1), row `lane` of Q
    for (int i = 0; i < m; ++i) {
        d[i] = sc->alpha[i];
        e[i] = i + 1 < m ? sc->beta[i] : 0.0;
        z[i] = i == lane ? 1.0 : 0.0;
    }
    const double tiny = 0x1p-53;
    for (int l = 0; l < m; ++l) {
        for (int iter = 0;; ++iter) {
            int u = l;                                  // end of the unreduced block starting at l
            while (u < m - 1 && fabs(e[u]) > tiny * (fabs(d[u]) + fabs(d[u + 1]))) ++u;
            if (u == l) break;
            if (iter == 60) {                           // no convergence: report, keep what we have
                if (lane == 0) sc->flags |= 4;
                break;
            }
            // shift: the eigenvalue of the leading 2 x 2 block closer to d_l
            double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
            double r = hypot(g, 1.0);
            g = d[u] - d[l] + e[l] / (g + copysign(r, g));
            double sn = 1.0, cs = 1.0, p = 0.0;
            bool restart = false;
            for (int i = u - 1; i >= l; --i) {
                const double f = sn * e[i], b = cs * e[i];
                r = hypot(f, g);
                e[i + 1] = r;
                if (r == 0.0) {                         // the block splits: deflate and start again
                    d[i + 1] -= p;
                    e[u] = 0.0;
                    restart = true;
                    break;
                }
                sn = f / r;
                cs = g / r;
                g = d[i + 1] - p;
                r = (d[i] - g) * sn + 2.0 * cs * b;
                p = sn * r;
                d[i + 1] = g + p;
                g = cs * r - b;
                const double zi = z[i], zi1 = z[i + 1];   // Q <- Q G(i, i+1)
                z[i + 1] = sn * zi + cs * zi1;
                z[i] = cs * zi - sn * zi1;
            }
            if (restart) continue;
            d[l] -= p;
            e[l] = g;
            e[u] = 0.0;
        }
    }
    double yr = 0.0, yi = 0.0;
    for (int j = 0; j < m; ++j) {
        const double q0 = __shfl_sync(0xffffffffu, z[j], 0);   // Q_{0 j}
        const double ph = -h * d[j];
        const double w = z[j] * q0;
        yr += w * cos(ph);
        yi += w * sin(ph);
        if (lane < m) sc->Q[lane * m + j] = z[j];
    }
    if (lane < m) {
        sc->lam[lane] = d[lane];
        sc->y[2 * lane] = sc->beta0 * yr * sc->s[lane];
        sc->y[2 * lane + 1] = sc->beta0 * yi * sc->s[lane];
    }
    if (lane == 0) sc->t += h;
}

__global__ void __launch_bounds__(32) eig_kernel(Scal *sc, double h) { eig_warp(sc, h); }

// The same iteration for m <= 8 with T and the rows of Q in registers: every loop over indices is
// unrolled and the block bounds l and u become predicates, so that no array is indexed at run time
// (in eig_kernel d, e and z live in local memory).  A rotation takes sqrt(f^2 + g^2) and one
// reciprocal (the magnitudes here are far from the FP64 range limits; a result below 2^-500 falls
// back to hypot).  Eight lanes: lane i holds row i of Q; lane j computes the phase of eigenvalue j.
constexpr int kEigSmall = 8;
__device__ void eig_small_warp(Scal *sc, double h)   // run by lanes 0 .. 7 of a warp
{
    constexpr int M = kEigSmall;
    constexpr unsigned mask = (1u << M) - 1;
    const int lane = threadIdx.x;
    const int m = sc->m_used;
    double d[M], e[M], z[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
        d[i] = i < m ? sc->alpha[i] : 0.0;
        e[i] = i + 1 < m ? sc->beta[i] : 0.0;
        z[i] = i == lane ? 1.0 : 0.0;
    }
    const double tiny = 0x1p-53;
    auto rot_norm = [](double f, double g) {
        double r = sqrt(fma(f, f, g * g));
        return r < 0x1p-500 ? hypot(f, g) : r;
    };
#pragma unroll
    for (int l = 0; l < M - 1; ++l) {        // l = M - 1 is a 1 x 1 block
        if (l >= m) break;
        for (int iter = 0;; ++iter) {
            int u = m - 1;                      // end of the unreduced block starting at l
            bool open = true;
#pragma unroll
            for (int j = l; j < M - 1; ++j)
                if (open && (j >= m - 1 || !(fabs(e[j]) > tiny * (fabs(d[j]) + fabs(d[j + 1]))))) {
                    u = j;
                    open = false;
                }
            if (u == l) break;
            if (iter == 60) {                   // no convergence: report, keep what we have
                if (lane == 0) sc->flags |= 4;
                break;
            }
            double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
            double r = rot_norm(g, 1.0);
            double du = d[M - 1];
#pragma unroll
            for (int j = l + 1; j < M - 1; ++j)
                if (j == u) du = d[j];
            g = du - d[l] + e[l] / (g + copysign(r, g));
            double sn = 1.0, cs = 1.0, p = 0.0;
            bool restart = false, live = true;
#pragma unroll
            for (int i = M - 2; i >= l; --i) {
                if (live && i < u) {
                    const double f = sn * e[i], b = cs * e[i];
                    r = rot_norm(f, g);
                    e[i + 1] = r;
                    if (r == 0.0) {                 // the block splits: deflate and start again
                        d[i + 1] -= p;
#pragma unroll
                        for (int j = l + 1; j < M; ++j)
                            if (j == u) e[j] = 0.0;
                        restart = true;
                        live = false;
                    } else {
                        const double inv = 1.0 / r;
                        sn = f * inv;
                        cs = g * inv;
                        g = d[i + 1] - p;
                        r = (d[i] - g) * sn + 2.0 * cs * b;
                        p = sn * r;
                        d[i + 1] = g + p;
                        g = cs * r - b;
                        const double zi = z[i], zi1 = z[i + 1];   // Q <- Q G(i, i+1)
                        z[i + 1] = sn * zi + cs * zi1;
                        z[i] = cs * zi - sn * zi1;
                    }
                }
            }
            if (restart) continue;
            d[l] -= p;
            e[l] = g;
#pragma unroll
            for (int j = l + 1; j < M; ++j)
                if (j == u) e[j] = 0.0;
        }
    }
    double dl = d[0];
#pragma unroll
    for (int j = 1; j < M; ++j)
        if (j == lane) dl = d[j];
    double sph = 0.0, cph = 1.0;
    if (lane < m) sincos(-h * dl, &sph, &cph);
    double yr = 0.0, yi = 0.0;
#pragma unroll
    for (int j = 0; j < M; ++j) {
        const double q0 = __shfl_sync(mask, z[j], 0);   // Q_{0 j}
        const double cj = __shfl_sync(mask, cph, j), sj = __shfl_sync(mask, sph, j);
        if (j < m) {
            const double w = z[j] * q0;
            yr += w * cj;
            yi += w * sj;
            if (lane < m) sc->Q[lane * m + j] = z[j];
        }
    }
    if (lane < m) {
        sc->lam[lane] = dl;
        sc->y[2 * lane] = sc->beta0 * yr * sc->s[lane];
        sc->y[2 * lane + 1] = sc->beta0 * yi * sc->s[lane];
    }
    if (lane == 0) sc->t += h;
}

__global__ void __launch_bounds__(kEigSmall) eig_small_kernel(Scal *sc, double h) { eig_small_warp(sc, h); }

// y = beta_0 Q exp(-i h Lambda) Q^T e_1 for m <= 8 with few FP64 instructions (each costs about 64
// FP32 ones for a single warp here), one eigenpair per lane j < m:
//   1. lambda_j (the (j+1)-th smallest) by bisection on [lo, hi] in FP32 with Sturm counts (the signs
//      of the pivots of T - x I = L D L^T);
//   2. three Newton steps in FP64 on det(T - x I) and its derivative (three-term recurrences);
//   3. the eigenvector by inverse iteration: T - lambda_j I = L D L^T in FP64 (pivots below
//      1e-14 (hi - lo) replaced by that), two solves from the vector of ones, normalised.
// When two eigenvalues lie closer than 1 % of hi - lo (the eigenvectors of inverse iteration then
// lose orthogonality in proportion to eps (hi - lo) / gap), or a Newton step fails, it returns false
// without writing anything and the caller runs the QL solver.  Warp-uniform; 32 lanes call it.
__device__ bool eig_fast_warp(Scal *sc, double h, double lo, double hi)
{
    constexpr int M = kEigSmall;
    const int lane = threadIdx.x & 31;
    const int mu = sc->m_used;
    double a[M], b[M];                                  // b[i] = T_{i, i+1}
    float af[M], b2f[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
        a[i] = i < mu ? sc->alpha[i] : 0.0;
        b[i] = i + 1 < mu ? sc->beta[i] : 0.0;
        af[i] = (float)a[i];
        b2f[i] = (float)(b[i] * b[i]);
    }
    const double span = hi - lo;
    // 1. bisection (FP32): lane j keeps [lf, uf] with count(lf) <= j < count(uf)
    float lf = (float)(lo - 1e-6 * span) - 1e-30f, uf = (float)(hi + 1e-6 * span) + 1e-30f;
    for (int it = 0; it < 32; ++it) {
        const float x = 0.5f * (lf + uf);
        int cnt = 0;
        float q = 1.f;
#pragma unroll
        for (int i = 0; i < M; ++i)
            if (i < mu) {
                q = (af[i] - x) - (i > 0 ? __fdividef(b2f[i - 1], q) : 0.f);
                if (fabsf(q) < 1e-30f) q = -1e-30f;
                cnt += q < 0.f;
            }
        if (cnt > lane) uf = x;
        else lf = x;
    }
    // 2. Newton (FP64)
    const double xb = 0.5 * ((double)lf + (double)uf);
    double x = xb;
    bool ok = true;
    for (int it = 0; it < 3; ++it) {
        double p0 = 1.0, p1 = a[0] - x, d0 = 0.0, d1 = -1.0;
#pragma unroll
        for (int i = 1; i < M; ++i)
            if (i < mu) {
                const double bb = b[i - 1] * b[i - 1];
                const double p2 = (a[i] - x) * p1 - bb * p0, d2 = (a[i] - x) * d1 - p1 - bb * d0;
                p0 = p1;
                p1 = p2;
                d0 = d1;
                d1 = d2;
            }
        const double step = p1 / d1;
        if (isfinite(step)) x -= step;
        else if (p1 != 0.0) ok = false;
    }
    ok = ok && isfinite(x) && fabs(x - xb) <= 4.0 * ((double)uf - (double)lf) + 1e-12 * span;
    // gaps between consecutive eigenvalues (lane j: lambda_{j+1} - lambda_j)
    const double xn = __shfl_down_sync(0xffffffffu, x, 1);
    if (lane + 1 < mu) ok = ok && xn - x > 1e-2 * span;
    if (!__all_sync(0xffffffffu, ok || lane >= mu) || !(span > 0.0)) return false;
    // 3. inverse iteration (FP64)
    const double tiny = 1e-14 * span;
    double inv_d[M], l[M], z[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
        if (i < mu) {
            l[i] = i > 0 ? b[i - 1] * inv_d[i - 1] : 0.0;
            double d = a[i] - x - (i > 0 ? l[i] * b[i - 1] : 0.0);
            if (fabs(d) < tiny) d = tiny;
            inv_d[i] = 1.0 / d;
        } else {
            l[i] = 0.0;
            inv_d[i] = 0.0;
        }
        z[i] = i < mu ? 1.0 : 0.0;
    }
    for (int pass = 0; pass < 2; ++pass) {
#pragma unroll
        for (int i = 1; i < M; ++i) z[i] -= l[i] * z[i - 1];          // L y = r
#pragma unroll
        for (int i = M - 1; i >= 0; --i) z[i] = z[i] * inv_d[i] - (i + 1 < M ? l[i + 1] * z[i + 1] : 0.0);   // D L^T z = y
        double nr = 0.0;
#pragma unroll
        for (int i = 0; i < M; ++i) nr = fma(z[i], z[i], nr);
        const double inv = rsqrt(nr);
#pragma unroll
        for (int i = 0; i < M; ++i) z[i] *= inv;
    }
    // y_i = beta_0 sum_j z_j[i] z_j[0] e^{-i h lambda_j}
    __shared__ double Zs[M][M];
    double ps, pc;
    sincos(-h * x, &ps, &pc);
    const double wr = lane < mu ? z[0] * pc : 0.0, wi = lane < mu ? z[0] * ps : 0.0;
    if (lane < mu) {
#pragma unroll
        for (int i = 0; i < M; ++i) Zs[lane][i] = z[i];
    }
    __syncwarp();
    double yr = 0.0, yi = 0.0;
#pragma unroll
    for (int j = 0; j < M; ++j) {
        const double wrj = __shfl_sync(0xffffffffu, wr, j), wij = __shfl_sync(0xffffffffu, wi, j);
        if (j < mu && lane < M) {
            const double q = Zs[j][lane];
            yr = fma(q, wrj, yr);
            yi = fma(q, wij, yi);
        }
    }
    if (lane < mu) {
        sc->y[2 * lane] = sc->beta0 * yr * sc->s[lane];
        sc->y[2 * lane + 1] = sc->beta0 * yi * sc->s[lane];
    }
    if (lane == 0) sc->t += h;
    return true;
}

// y = beta_0 exp(-i h T_m) e_1 for the time step, which needs no eigenvectors.  With c, r from the
// Gershgorin bounds of T_m, T_m = c I + r X with the spectrum of X in [-1, 1], and by the
// Jacobi-Anger expansion exp(-i h T_m) = e^{-i h c} sum_k eps_k (-i sgn h)^k J_k(|h| r) T_k(X)
// (eps_0 = 1, eps_k = 2), truncated where the Bessel terms fall below 1e-17 (at index about
// z + 10 z^(1/3) + 12 for z = |h| r).  The J_k come from Miller's backward recurrence
// J_{n-1} = (2n/z) J_n - J_{n+1}, started 10 indices further out and normalised by
// J_0 + 2 sum_k J_2k = 1.  When |h| r exceeds 32 the step is split into s equal parts and the
// series applied s times.  On this GPU a single warp's FP64 instruction costs about as much as
// 64 FP32 ones: the QL iteration takes a few thousand of them whatever |h| r, the series about
// 6 (real vector) to 14 (complex) per term, so the series runs for |h| r <= 96 (at most three
// applications) and the QL eigensolver otherwise (and for a non-finite T).
// One warp: lane j holds component j of the Chebyshev vectors (T_m is tridiagonal, so X t
// takes the neighbours by shuffles).
constexpr int kChebZ = 32;         // largest |h| r per series application
constexpr int kChebN = 96;         // Bessel values kept (truncation index for z = 32 is 76)
constexpr int kChebMaxSub = 3;     // beyond 3 applications the QL eigendecomposition is cheaper

__device__ __forceinline__ int cheb_terms(double z) { return z < 1e-20 ? 0 : (int)ceil(z + 10.0 * cbrt(z) + 12.0); }

template <bool SMALL>   // SMALL: m <= 8, so that the QL fallback is eig_small_warp
__global__ void __launch_bounds__(32) expv_kernel(Scal *sc, double h)
{
    const int j = threadIdx.x;
    const int mu = sc->m_used;
    if (mu <= 0) {
        if (j == 0) sc->t += h;
        return;
    }
    __shared__ double J[kChebN];
    const double aj = j < mu ? sc->alpha[j] : 0.0;
    const double bj = j + 1 < mu ? sc->beta[j] : 0.0;              // T_{j, j+1}
    double bjm = __shfl_up_sync(0xffffffffu, bj, 1);
    if (j == 0) bjm = 0.0;
    double lo = j < mu ? aj - fabs(bjm) - fabs(bj) : INFINITY, hi = j < mu ? aj + fabs(bjm) + fabs(bj) : -INFINITY;
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    const double c = 0.5 * (lo + hi);
    double r = 0.5 * (hi - lo);
    if (!(r >= 1e-290)) r = 1e-290;                                // T = c I (or non-finite: propagates)
    const double sgn = h < 0.0 ? -1.0 : 1.0;
    const double z_all = fabs(h) * r;
    if (!(z_all <= kChebZ * kChebMaxSub)) {      // large |h| ||T|| or non-finite T: eigenpairs instead
        if (!SMALL) eig_warp(sc, h);
        else if (!eig_fast_warp(sc, h, lo, hi) && j < kEigSmall) eig_small_warp(sc, h);
        return;
    }
    const int nsub = z_all > kChebZ ? (int)ceil(z_all / kChebZ) : 1;
    const double z = z_all / nsub;
    const int K = cheb_terms(z);
    if (j == 0) {                                                   // Miller's recurrence (lane 0)
        if (K == 0) {
            J[0] = 1.0;
        } else {
            int n0 = K + 10;
            n0 += n0 & 1;
            const double tz = 2.0 / z;
            double jp1 = 0.0, jn = 1e-280, norm = 0.0;
            for (int n = n0; n >= 1; --n) {
                if (n <= K) J[n] = jn;
                if (!(n & 1)) norm += 2.0 * jn;
                const double jm1 = (tz * n) * jn - jp1;
                jp1 = jn;
                jn = jm1;
                if (fabs(jn) > 1e250) {                             // rescale (only for small z)
                    for (int k = n; k <= K; ++k) J[k] *= 1e-250;
                    norm *= 1e-250;
                    jp1 *= 1e-250;
                    jn *= 1e-250;
                }
            }
            J[0] = jn;
            norm += jn;
            const double inv = 1.0 / norm;
            for (int k = 0; k <= K; ++k) J[k] *= inv;
        }
    }
    __syncwarp();
    const double ax = j < mu ? (aj - c) / r : 0.0, bx = bj / r, bxm = bjm / r;   // row j of X
    double ps, pc;
    sincos(-h * c / nsub, &ps, &pc);                                // e^{-i h c / s}
    double vr = j == 0 ? 1.0 : 0.0, vi = 0.0;
    for (int sub = 0; sub < nsub; ++sub) {
        // y = sum_k eps_k (-i sgn)^k J_k T_k(X) v by the three-term recurrence of T_k
        double t0r = vr, t0i = vi;
        double yr = J[0] * t0r, yi = J[0] * t0i;
        if (K >= 1) {
            const bool real = sub == 0;                             // v = e_1: T_k(X) v stays real
            double t1r = ax * t0r + bxm * __shfl_up_sync(0xffffffffu, t0r, 1) + bx * __shfl_down_sync(0xffffffffu, t0r, 1);
            double t1i = real ? 0.0 : ax * t0i + bxm * __shfl_up_sync(0xffffffffu, t0i, 1) + bx * __shfl_down_sync(0xffffffffu, t0i, 1);
            double pr = 0.0, pi = -sgn;                             // (-i sgn)^1
            double cr = 2.0 * J[1] * pr, ci = 2.0 * J[1] * pi;
            yr += cr * t1r - ci * t1i;
            yi += cr * t1i + ci * t1r;
            for (int k = 2; k <= K; ++k) {
                const double npr = sgn * pi, npi = -sgn * pr;       // times (-i sgn)
                pr = npr;
                pi = npi;
                const double ur = __shfl_up_sync(0xffffffffu, t1r, 1), dr = __shfl_down_sync(0xffffffffu, t1r, 1);
                const double t2r = 2.0 * (ax * t1r + bxm * ur + bx * dr) - t0r;
                double t2i = 0.0;
                if (!real) {
                    const double ui = __shfl_up_sync(0xffffffffu, t1i, 1), di = __shfl_down_sync(0xffffffffu, t1i, 1);
                    t2i = 2.0 * (ax * t1i + bxm * ui + bx * di) - t0i;
                }
                const double w = 2.0 * J[k];
                cr = w * pr;
                ci = w * pi;
                yr += cr * t2r - ci * t2i;
                yi += cr * t2i + ci * t2r;
                t0r = t1r;
                t0i = t1i;
                t1r = t2r;
                t1i = t2i;
            }
        }
        vr = pc * yr - ps * yi;
        vi = pc * yi + ps * yr;
    }
    if (j < mu) {
        sc->y[2 * j] = sc->beta0 * vr * sc->s[j];
        sc->y[2 * j + 1] = sc->beta0 * vi * sc->s[j];
    }
    if (j == 0) sc->t += h;
}

// Eigen-decomposition and the Krylov coefficients of the step for m_used <= m.
static void launch_eig(Scal *sc, int m, double h, cudaStream_t st)
{
    if (m <= kEigSmall) eig_small_kernel<<<1, kEigSmall, 0, st>>>(sc, h);
    else eig_kernel<<<1, 32, 0, st>>>(sc, h);
}

// c = sum_i y_i v_i, and ||c||^2 for hx_step_info.  Complex128 vectors accumulate in FP64; for
// complex64 vectors each y_i is split into float parts hi + lo and the sum is accumulated with
// the compensated products of F2 (Dot2), which keeps it as accurate as FP64 accumulation (relative
// error of order 2^-48 of sum |y_i v_i|); per element the only FP64 operations are the two adds
// that round the pair sums to the complex128 state (the norm goes through NormAcc).
template <typename V, int NV>
__global__ void combine_kernel(double2 *c, const V *Vb, size_t ld, int n, double *partials, Scal *sc)
{
    const int m = sc->m_used;
    double acc = 0.0;
    if constexpr (std::is_same<V, float2>::value) {
        float yrh[NV], yrl[NV], yih[NV], yil[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            const double yr = i < m ? sc->y[2 * i] : 0.0, yi = i < m ? sc->y[2 * i + 1] : 0.0;
            yrh[i] = (float)yr;
            yrl[i] = (float)(yr - (double)yrh[i]);
            yih[i] = (float)yi;
            yil[i] = (float)(yi - (double)yih[i]);
        }
        NormAcc na;
        for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
            F2 xr, xi;
#pragma unroll(NV <= 8 ? NV : 1)
            for (int i = 0; i < NV; ++i)
                if (i < m) {
                    const float2 v = Vb[i * ld + e];
                    xr.add_prod(yrh[i], v.x);
                    xr.add_prod(-yih[i], v.y);
                    xr.c = fmaf(yrl[i], v.x, fmaf(-yil[i], v.y, xr.c));
                    xi.add_prod(yrh[i], v.y);
                    xi.add_prod(yih[i], v.x);
                    xi.c = fmaf(yrl[i], v.y, fmaf(yil[i], v.x, xi.c));
                }
            // the pair sums as FP64 (exact binary32 -> binary64 conversions, one FP64 add each)
            const double2 x = make_double2(f2d_exact(xr.s) + f2d_exact(xr.c), f2d_exact(xi.s) + f2d_exact(xi.c));
            c[e] = x;
            na.add(x.x);
            na.add(x.y);
        }
        acc = na.value();
    } else {
        double yr[NV], yi[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            yr[i] = i < m ? sc->y[2 * i] : 0.0;
            yi[i] = i < m ? sc->y[2 * i + 1] : 0.0;
        }
        for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
            double xr = 0.0, xi = 0.0;
#pragma unroll(NV <= 8 ? NV : 1)
            for (int i = 0; i < NV; ++i)
                if (i < m) {
                    const V v = Vb[i * ld + e];
                    xr += yr[i] * v.x - yi[i] * v.y;
                    xi += yr[i] * v.y + yi[i] * v.x;
                }
            c[e] = make_double2(xr, xi);
            acc += xr * xr + xi * xi;
        }
    }
    __shared__ double tot[1];
    if (reduce_partials(&acc, 1, partials, &sc->counter, tot) && threadIdx.x == 0) {
        double nr = sqrt(tot[0]);
        sc->norm_out = nr;
        if (!isfinite(nr)) sc->flags |= 2;
        sc->counter = 0;
    }
}

// One term y_i v of the complex64 recombination into the compensated pairs (xr, xi), with
// y_i = (yr_hi + yr_lo) + i (yi_hi + yi_lo) packed in y as (yr_hi, yr_lo, yi_hi, yi_lo).
__device__ __forceinline__ void combine_term(F2 &xr, F2 &xi, float4 y, float2 v)
{
    xr.add_prod(y.x, v.x);
    xr.add_prod(-y.z, v.y);
    xr.c = fmaf(y.y, v.x, fmaf(-y.w, v.y, xr.c));
    xi.add_prod(y.x, v.y);
    xi.add_prod(y.z, v.x);
    xi.c = fmaf(y.y, v.y, fmaf(y.w, v.x, xi.c));
}

// The same compensated accumulation for the real and imaginary parts at once, in packed FP32x2
// instructions (each lane the IEEE operation of F2::add_prod, in the same order).
struct F2x2 {
    float2 s = {0.f, 0.f}, c = {0.f, 0.f};
    __device__ __forceinline__ void add_prod(float2 a, float2 b)
    {
        const float2 p = f2_mul(a, b);
        const float2 e = f2_fma(a, b, make_float2(-p.x, -p.y));
        const float2 t = f2_add(s, p), bb = f2_sub(t, s);
        const float2 q = f2_add(f2_sub(s, f2_sub(t, bb)), f2_sub(p, bb));
        s = t;
        c = f2_add(c, f2_add(q, e));
    }
};

// combine_term on both parts: (re, im) += (yr + i yi) (vx + i vy) with y = (yr_hi, yr_lo, yi_hi, yi_lo)
__device__ __forceinline__ void combine_term2(F2x2 &x, float4 y, float2 v)
{
    const float2 vs = make_float2(v.y, v.x);
    x.add_prod(make_float2(y.x, y.x), v);            // yr_hi (vx, vy)
    x.add_prod(make_float2(-y.z, y.z), vs);          // yi_hi (-vy, vx)
    x.c = f2_fma(make_float2(y.y, y.y), v, f2_fma(make_float2(-y.w, y.w), vs, x.c));
}

// The complex64 recombination for m = M <= 8 known at compile time: two elements per thread and
// iteration (16-byte loads of every basis vector, all issued before the arithmetic), the split
// coefficients in shared memory.  Same arithmetic per element as combine_kernel, in packed FP32x2
// instructions.
template <int M>
__global__ void __launch_bounds__(256) combine_m_kernel(double2 *c, const float2 *Vb, size_t ld, int n,
                                                        double *partials, Scal *sc)
{
    __shared__ float4 ys[M];
    const int mu = sc->m_used;
    if ((int)threadIdx.x < M) {
        const int i = threadIdx.x;
        const double yr = i < mu ? sc->y[2 * i] : 0.0, yi = i < mu ? sc->y[2 * i + 1] : 0.0;
        const float yrh = (float)yr, yih = (float)yi;
        ys[i] = make_float4(yrh, (float)(yr - (double)yrh), yih, (float)(yi - (double)yih));
    }
    __syncthreads();
    NormAcc na;
    const int npair = n >> 1;
    const int gid = blockIdx.x * blockDim.x + threadIdx.x, gstride = gridDim.x * blockDim.x;
    for (int q = gid; q < npair; q += gstride) {
        const int e = 2 * q;
        Pair<float2> v[M];
#pragma unroll
        for (int i = 0; i < M; ++i)
            if (i < mu) v[i] = load_pair(Vb + i * ld, e);
        F2x2 pa, pb;
#pragma unroll
        for (int i = 0; i < M; ++i)
            if (i < mu) {
                const float4 y = ys[i];
                combine_term2(pa, y, v[i].a);
                combine_term2(pb, y, v[i].b);
            }
        const double2 xa = make_double2(f2d_exact(pa.s.x) + f2d_exact(pa.c.x), f2d_exact(pa.s.y) + f2d_exact(pa.c.y));
        const double2 xb = make_double2(f2d_exact(pb.s.x) + f2d_exact(pb.c.x), f2d_exact(pb.s.y) + f2d_exact(pb.c.y));
        c[e] = xa;
        c[e + 1] = xb;
        na.add(xa.x);
        na.add(xa.y);
        na.add(xb.x);
        na.add(xb.y);
    }
    if ((n & 1) && gid == 0) {                              // odd length: the last element
        const int e = n - 1;
        F2 ar, ai;
#pragma unroll
        for (int i = 0; i < M; ++i)
            if (i < mu) combine_term(ar, ai, ys[i], Vb[i * ld + e]);
        const double2 xa = make_double2(f2d_exact(ar.s) + f2d_exact(ar.c), f2d_exact(ai.s) + f2d_exact(ai.c));
        c[e] = xa;
        na.add(xa.x);
        na.add(xa.y);
    }
    double acc = na.value();
    __shared__ double tot[1];
    if (reduce_partials(&acc, 1, partials, &sc->counter, tot) && threadIdx.x == 0) {
        double nr = sqrt(tot[0]);
        sc->norm_out = nr;
        if (!isfinite(nr)) sc->flags |= 2;
        sc->counter = 0;
    }
}

template <int M>
static void launch_combine_m(const Problem *p, double2 *c, const float2 *Vb, size_t ld, int n, double *partials, Scal *sc,
                             cudaStream_t st)
{
    combine_m_kernel<M><<<resident_grid(p, combine_m_kernel<M>, 256), 256, 0, st>>>(c, Vb, ld, n, partials, sc);
}

// H v for the 2-stage Magnus exponent, Eq. (2stageMagnus) written as Omega = -i h H:
// H v = (A_1 v + A_2 v) / 2 - i g (A_2 A_1 v - A_1 A_2 v), g = sqrt(3) h / 12.
template <typename V>
__global__ void magnus_combine_kernel(V *out, const V *a1v, const V *a2v, const V *a2a1v, const V *a1a2v, int n,
                                      double g_)
{
    using R = typename Real<V>::T;
    const R g = (R)g_, half = (R)0.5;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const V x1 = a1v[e], x2 = a2v[e], y1 = a2a1v[e], y2 = a1a2v[e];
        V r;
        r.x = half * (x1.x + x2.x) + g * (y1.y - y2.y);   // -i g z = g (z.y, -z.x)
        r.y = half * (x1.y + x2.y) - g * (y1.x - y2.x);
        out[e] = r;
    }
}

template <typename V, int K>
static void launch_sweep_k_t(const Problem *p, V *Vb, size_t ld, int n, double *partials, Scal *sc, cudaStream_t st)
{
    const int G = resident_grid(p, sweep_k_kernel<V, K>, 256);
    sweep_k_kernel<V, K><<<G, 256, 0, st>>>(Vb, ld, n, partials, sc);
}

// The Gram-Schmidt sweep of Lanczos index k < 8 with the kernel specialised for k.
template <typename V>
static int launch_sweep_k(const Problem *p, V *Vb, size_t ld, int n, int k, double *partials, Scal *sc,
                          cudaStream_t st)
{
#define HX_SWEEP_K(K)                                               \
    case K:                                                         \
        launch_sweep_k_t<V, K>(p, Vb, ld, n, partials, sc, st);     \
        return HX_OK;
    switch (k) {
        HX_SWEEP_K(0) HX_SWEEP_K(1) HX_SWEEP_K(2) HX_SWEEP_K(3)
        HX_SWEEP_K(4) HX_SWEEP_K(5) HX_SWEEP_K(6) HX_SWEEP_K(7)
    }
#undef HX_SWEEP_K
    set_error("internal: Gram-Schmidt sweep kernel for k = %d", k);
    return HX_EUNSUPPORTED;
}

// A-posteriori estimate of the relative error of the Lanczos exponential (Sec. 2.2), from the
// residual of the Krylov relation A V_m = V_m T_m + beta_m v_{m+1} e_m^T:
//   ||exp(-ihA) c - ||c|| V_m exp(-ihT_m) e_1|| / ||c||  ~  |h| beta_m |e_m^T exp(-ihT_m) e_1|,
// with beta_m from the pass after the last vector and the last component of exp(-ihT_m) e_1 from
// the stored combination weights (y_i = beta_0 s_i [exp(-ihT_m) e_1]_i).  Zero after a breakdown
// (the Krylov space is invariant).  err_max keeps the largest value since it was cleared.
__global__ void err_est_kernel(Scal *sc, double h, int m)
{
    const int mu = sc->m_used;
    double est = 0.0;
    if (mu == m && mu > 0 && sc->beta0 > 0.0) {
        const int i = mu - 1;
        const double ur = sc->y[2 * i] / (sc->beta0 * sc->s[i]), ui = sc->y[2 * i + 1] / (sc->beta0 * sc->s[i]);
        est = fabs(h) * sc->beta[i] * sqrt(ur * ur + ui * ui);
    }
    if (!(est <= sc->err_max)) sc->err_max = est;   // NaN propagates
}

// Parts of a step for batch graphs that take the Lanczos products from a batched launch: the whole
// step (kPhaseAll), the start vector (kPhaseInit), the work after product k (phase k: projections
// and Gram-Schmidt passes, the product itself skipped), or the end (phase m: the exponential and the
// recombination).
constexpr int kPhaseAll = -2, kPhaseInit = -1;

template <typename V, int NV>
static int enqueue_step(Problem *p, Work *w, double2 *state, cudaStream_t st, double dt, int phase = kPhaseAll)
{
    const int n = p->set->d.size;
    const int m = p->cfg.m;
    const int G = apply_grid(p);
    const int T = 256;
    V *Vb = (V *)w->V;
    const size_t ld = w->vec_bytes / sizeof(V);
    Scal *sc = w->sc;
    const int Gd = resident_grid(p, dot_kernel<V, NV>, T), Gr = resident_grid(p, rayleigh_kernel<V>, T);
    const bool all = phase == kPhaseAll;
    // the exponential midpoint step takes the projections from the product kernel when it can
    const bool fused = all && p->cfg.scheme == HX_SCHEME_EXPMPR && NV <= kMaxFusedDots && apply_fuses_dots(p);
    if (all || phase == kPhaseInit) init_kernel<V><<<G, T, 0, st>>>(state, Vb, n, w->partials, sc, m);
    for (int k = 0; k < m; ++k) {
        if (!all && phase != k) continue;
        ApplyFuse f;
        memset(&f, 0, sizeof(f));
        f.in_scale = &sc->s[k];
        int rc;
        if (!all) {
            // the product was done by a batched launch
        } else if (p->cfg.scheme == HX_SCHEME_MAGNUS4) {   // Eq. (2stageMagnus): nodes 1/2 -+ sqrt(3)/6
            const double c1 = 0.5 - sqrt(3.0) / 6.0, c2 = 0.5 + sqrt(3.0) / 6.0;
            V *a1v = (V *)w->mag, *a2v = a1v + ld, *a2a1v = a2v + ld, *a1a2v = a2a1v + ld;
            const double g = sqrt(3.0) * dt / 12.0;
            V *hv = Vb + (size_t)(k + 1) * ld;
            if ((rc = launch_apply_dual(p, Vb + (size_t)k * ld, a1v, a2v, &sc->t, c1 * dt, c2 * dt, &f, st)) ||
                (rc = launch_apply_pair(p, a1v, a2a1v, c2 * dt, a2v, a1a2v, c1 * dt, &sc->t, st, hv, g)))
                return rc;
            if (!apply_dual(p))   // the specialised kernel wrote the combination itself
                magnus_combine_kernel<V><<<G, T, 0, st>>>(hv, a1v, a2v, a2a1v, a1a2v, n, g);
        } else {
            if (fused) {     // r = s_k <V_k, y> from the product kernel's own values (one sweep, m <= 8)
                f.rq = true;
                f.s = &sc->s[k];
                f.h = sc->h;
                f.partials = w->partials;
                f.counter = &sc->counter;
            }
            rc = launch_apply(p, Vb + (size_t)k * ld, Vb + (size_t)(k + 1) * ld, &sc->t, 0.5 * dt, &f, st);
            if (rc) return rc;
        }
        V *wv = Vb + (size_t)(k + 1) * ld;
        if constexpr (NV <= 8) {   // one sweep per vector (the second pass of v_k and the first of v_{k+1})
            if (!f.rq)
                rayleigh_kernel<V><<<Gr, T, 0, st>>>(Vb + (size_t)k * ld, wv, n, true, &sc->s[k], &sc->m_used, k, sc->h,
                                                     w->partials, &sc->counter);
            if ((rc = launch_sweep_k<V>(p, Vb, ld, n, k, w->partials, sc, st))) return rc;
        } else {
            if (!f.dvec) dot_kernel<V, NV><<<Gd, T, 0, st>>>(wv, Vb, ld, n, k, w->partials, sc);
            // two passes; the second also runs after the last vector when the step estimates its
            // error (beta_m)
            const bool pass1 = k < m - 1 || p->cfg.tol > 0.0;
            const int Gu0 = resident_grid(p, update_kernel<V, NV, 0>, T), Gu1 = resident_grid(p, update_kernel<V, NV, 1>, T);
            update_kernel<V, NV, 0><<<Gu0, T, 0, st>>>(wv, Vb, ld, n, k, w->partials, sc);
            if (pass1) update_kernel<V, NV, 1><<<Gu1, T, 0, st>>>(wv, Vb, ld, n, k, w->partials, sc);
        }
    }
    if (!all && phase != m) {
        cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? HX_OK : cuda_fail(e, "step kernel launch");
    }
    if (m <= kEigSmall) expv_kernel<true><<<1, 32, 0, st>>>(sc, dt);
    else expv_kernel<false><<<1, 32, 0, st>>>(sc, dt);
    if (p->cfg.tol > 0.0) err_est_kernel<<<1, 1, 0, st>>>(sc, dt, m);
    if constexpr (std::is_same<V, float2>::value) {
        switch (m) {
        case 1: launch_combine_m<1>(p, state, Vb, ld, n, w->partials, sc, st); break;
        case 2: launch_combine_m<2>(p, state, Vb, ld, n, w->partials, sc, st); break;
        case 3: launch_combine_m<3>(p, state, Vb, ld, n, w->partials, sc, st); break;
        case 4: launch_combine_m<4>(p, state, Vb, ld, n, w->partials, sc, st); break;
        case 5: launch_combine_m<5>(p, state, Vb, ld, n, w->partials, sc, st); break;
        case 6: launch_combine_m<6>(p, state, Vb, ld, n, w->partials, sc, st); break;
        case 7: launch_combine_m<7>(p, state, Vb, ld, n, w->partials, sc, st); break;
        case 8: launch_combine_m<8>(p, state, Vb, ld, n, w->partials, sc, st); break;
        default:
            combine_kernel<V, NV><<<resident_grid(p, combine_kernel<V, NV>, T), T, 0, st>>>(state, Vb, ld, n, w->partials, sc);
        }
    } else {
        combine_kernel<V, NV><<<resident_grid(p, combine_kernel<V, NV>, T), T, 0, st>>>(state, Vb, ld, n, w->partials, sc);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "step kernel launch");
    return HX_OK;
}

// ---------------------------------------------------------------------------------------
// hx_apply_project: the product with the first projections of a Lanczos step, outside the graph
// ---------------------------------------------------------------------------------------

struct ProjWS {
    Scal sc;                        // m_used = kMaxFusedDots, s_i = 1, counter, h
    double partials[1];             // apply_grid(p) x 2 kMaxFusedDots
};

static ProjWS *proj_ws(Problem *p)
{
    if (p->proj_ws) return (ProjWS *)p->proj_ws;
    const size_t bytes = sizeof(ProjWS) + (size_t)apply_grid(p) * 2 * kMaxFusedDots * sizeof(double);
    void *d = nullptr;
    cudaError_t e = cudaMalloc(&d, bytes);
    if (e != cudaSuccess) { cuda_fail(e, "cudaMalloc(projection workspace)"); return nullptr; }
    Scal h;
    memset(&h, 0, sizeof(h));
    h.m_used = kMaxFusedDots;
    for (int i = 0; i < kMaxFusedDots; ++i) h.s[i] = 1.0;
    if ((e = cudaMemcpy(d, &h, sizeof(h), cudaMemcpyHostToDevice)) != cudaSuccess) {
        cudaFree(d);
        cuda_fail(e, "projection workspace init");
        return nullptr;
    }
    p->extra.push_back(d);
    p->proj_ws = d;
    return (ProjWS *)d;
}

template <typename V>
static int apply_project(Problem *p, const void *c, void *y, const void *basis, size_t ld, int k, double *h)
{
    ProjWS *ws = proj_ws(p);
    if (!ws) return HX_ECUDA;
    const int n = p->set->d.size;
    cudaStream_t st = p->stream;
    if (apply_fuses_dots(p)) {
        ApplyFuse f;
        memset(&f, 0, sizeof(f));
        f.dvec = basis;
        f.dld = ld;
        f.dk = k;
        f.m_used = &ws->sc.m_used;
        f.s = ws->sc.s;
        f.h = h;
        f.partials = ws->partials;
        f.counter = &ws->sc.counter;
        return launch_apply(p, c, y, p->dscal, 0.0, &f, st);
    }
    int rc = launch_apply(p, c, y, p->dscal, 0.0, nullptr, st);
    if (rc) return rc;
    // the paired variant reads two complex64 values per 16-byte load: y, the basis and its row
    // stride must be 16-byte aligned for it; otherwise the element-wise variant runs
    const bool paired = (uintptr_t)y % 16 == 0 && (uintptr_t)basis % 16 == 0 && (ld * sizeof(V)) % 16 == 0;
    if (paired) {
        const int G = resident_grid(p, dot_kernel<V, kMaxFusedDots>, 256);
        dot_kernel<V, kMaxFusedDots><<<G, 256, 0, st>>>((const V *)y, (const V *)basis, ld, n, k, ws->partials, &ws->sc);
    } else {
        const int G = resident_grid(p, dot_kernel<V, kMaxKrylov>, 256);
        dot_kernel<V, kMaxKrylov><<<G, 256, 0, st>>>((const V *)y, (const V *)basis, ld, n, k, ws->partials, &ws->sc);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, ws->sc.h, 2 * (k + 1) * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "projection kernel");
    return HX_OK;
}

int apply_project_dispatch(Problem *p, const void *c, void *y, const void *basis, size_t ld, int k, double *h)
{
    return p->cfg.dtype == HX_C64 ? apply_project<float2>(p, c, y, basis, ld, k, h)
                                  : apply_project<double2>(p, c, y, basis, ld, k, h);
}

// y = A c and r = <c, y>: one launch of the specialised complex64 kernel, else the product and
// rayleigh_kernel.  The projection workspace supplies the unit scale, partial sums and counter.
template <typename V>
static int apply_rayleigh(Problem *p, const void *c, void *y, double *r)
{
    ProjWS *ws = proj_ws(p);
    if (!ws) return HX_ECUDA;
    cudaStream_t st = p->stream;
    if (apply_fuses_dots(p)) {
        ApplyFuse f;
        memset(&f, 0, sizeof(f));
        f.rq = true;
        f.s = ws->sc.s;
        f.h = r;
        f.partials = ws->partials;
        f.counter = &ws->sc.counter;
        return launch_apply(p, c, y, p->dscal, 0.0, &f, st);
    }
    int rc = launch_apply(p, c, y, p->dscal, 0.0, nullptr, st);
    if (rc) return rc;
    const bool paired = (uintptr_t)c % 16 == 0 && (uintptr_t)y % 16 == 0;
    const int G = resident_grid(p, rayleigh_kernel<V>, 256);
    rayleigh_kernel<V><<<G, 256, 0, st>>>((const V *)c, (const V *)y, p->set->d.size, paired, ws->sc.s, nullptr, 0, r,
                                          ws->partials, &ws->sc.counter);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "Rayleigh quotient kernel");
    return HX_OK;
}

int apply_rayleigh_dispatch(Problem *p, const void *c, void *y, double *r)
{
    return p->cfg.dtype == HX_C64 ? apply_rayleigh<float2>(p, c, y, r) : apply_rayleigh<double2>(p, c, y, r);
}

static int enqueue(Problem *p, Work *w, double2 *state, cudaStream_t st, double dt, int phase = kPhaseAll)
{
    const bool c64 = p->cfg.dtype == HX_C64;
    if (p->cfg.m <= 8)
        return c64 ? enqueue_step<float2, 8>(p, w, state, st, dt, phase)
                   : enqueue_step<double2, 8>(p, w, state, st, dt, phase);
    return c64 ? enqueue_step<float2, kMaxKrylov>(p, w, state, st, dt, phase)
               : enqueue_step<double2, kMaxKrylov>(p, w, state, st, dt, phase);
}

static int ensure_work(Problem *p)
{
    if (p->krylov) return HX_OK;
    Work *w = new Work();
    memset(w, 0, sizeof(*w));
    const size_t n = (size_t)p->set->h.size;
    const size_t es = p->cfg.dtype == HX_C64 ? 8 : 16;
    w->vec_bytes = ((n * es + 255) / 256) * 256;
    const int G = apply_grid(p);
    cudaError_t e;
    const bool mag = p->cfg.scheme == HX_SCHEME_MAGNUS4;
    if ((e = cudaMalloc(&w->V, w->vec_bytes * (p->cfg.m + 1))) != cudaSuccess ||
        (e = cudaMalloc((void **)&w->partials, (size_t)G * 2 * (kMaxKrylov + 2) * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc((void **)&w->sc, sizeof(Scal))) != cudaSuccess ||
        (mag && (e = cudaMalloc(&w->mag, w->vec_bytes * 4)) != cudaSuccess)) {
        cudaFree(w->V); cudaFree(w->partials); cudaFree(w->sc); cudaFree(w->mag);
        delete w;
        return cuda_fail(e, "cudaMalloc(Krylov workspace)");
    }
    cudaMemset(w->sc, 0, sizeof(Scal));
    // the time lives in the problem's scalar block; copy it in
    cudaMemcpy(&w->sc->t, p->dscal, sizeof(double), cudaMemcpyDeviceToDevice);
    if ((e = cudaStreamCreateWithFlags(&w->cap_stream, cudaStreamNonBlocking)) != cudaSuccess) {
        cudaFree(w->V); cudaFree(w->partials); cudaFree(w->sc); cudaFree(w->mag);
        delete w;
        return cuda_fail(e, "cudaStreamCreate");
    }
    p->krylov = w;
    return HX_OK;
}

// The workspace (Krylov vectors, partial sums, scalars) does not depend on the potential; the
// captured step does (operator parameters and table pointers are kernel arguments).
void krylov_invalidate(Problem *p)
{
    Work *w = work_of(p);
    if (w && w->exec) {
        cudaGraphExecDestroy(w->exec);
        w->exec = nullptr;
    }
}

void krylov_free(Problem *p)
{
    Work *w = work_of(p);
    if (!w) return;
    if (w->exec) cudaGraphExecDestroy(w->exec);
    if (w->cap_stream) cudaStreamDestroy(w->cap_stream);
    cudaFree(w->V);
    cudaFree(w->host_state);
    cudaFree(w->partials);
    cudaFree(w->sc);
    cudaFree(w->mag);
    cudaFree(w->backup);
    cudaFreeHost(w->err_host);
    delete w;
    p->krylov = nullptr;
}

// The step graph is captured for one (state pointer, step size) pair and replayed; a call with
// another vector or step size captures a new graph (a few hundred microseconds).
static int ensure_graph(Problem *p, Work *w, void *c, double h)
{
    if (w->exec && w->dt == h && w->state == (double2 *)c) return HX_OK;
    if (w->exec) { cudaGraphExecDestroy(w->exec); w->exec = nullptr; }
    w->state = (double2 *)c;
    cudaGraph_t g;
    cudaError_t e;
    if ((e = cudaStreamBeginCapture(w->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return cuda_fail(e, "begin capture");
    int rc = enqueue(p, w, w->state, w->cap_stream, h);
    e = cudaStreamEndCapture(w->cap_stream, &g);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    e = cudaGraphInstantiate(&w->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { w->exec = nullptr; return cuda_fail(e, "graph instantiate"); }
    w->dt = h;
    return HX_OK;
}

// Steps with automatic sub-steps: each step of size dt is taken as s sub-steps of size dt / s; if
// the largest a-posteriori estimate over them exceeds tol the step is taken again from the saved
// state with 2 s sub-steps (at most kMaxSub), and after a step whose estimate is far below tol
// (by 2^(m+1), about what halving the step changes it by when the Lanczos process has converged)
// the next step tries s / 2.  One host synchronisation per attempted step.
static int adaptive_steps(Problem *p, Work *w, void *c, double dt, int nsteps)
{
    constexpr int kMaxSub = 1 << 16;
    cudaStream_t st = p->stream;
    const size_t bytes = (size_t)p->set->h.size * sizeof(double2);
    cudaError_t e;
    if (!w->backup && (e = cudaMalloc((void **)&w->backup, std::max<size_t>(bytes, 16))) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc(step backup)");
    if (!w->err_host && (e = cudaMallocHost((void **)&w->err_host, sizeof(double))) != cudaSuccess)
        return cuda_fail(e, "cudaMallocHost(error estimate)");
    if (w->sub < 1) w->sub = 1;
    const double tol = p->cfg.tol;
    w->sub_total = 0;
    w->err_last = 0.0;
    for (int n = 0; n < nsteps; ++n) {
        for (;;) {
            const int s = w->sub;
            int rc = ensure_graph(p, w, c, dt / s);
            if (rc) return rc;
            if ((e = cudaMemcpyAsync(w->backup, c, bytes, cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
                (e = cudaMemcpyAsync(&w->sc->t_save, &w->sc->t, sizeof(double), cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
                (e = cudaMemsetAsync(&w->sc->err_max, 0, sizeof(double), st)) != cudaSuccess)
                return cuda_fail(e, "adaptive step set-up");
            for (int i = 0; i < s; ++i)
                if ((e = cudaGraphLaunch(w->exec, st)) != cudaSuccess) return cuda_fail(e, "graph launch");
            if ((e = cudaMemcpyAsync(w->err_host, &w->sc->err_max, sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
                (e = cudaStreamSynchronize(st)) != cudaSuccess)
                return cuda_fail(e, "error estimate");
            const double err = *w->err_host;
            if (err > tol && s < kMaxSub) {        // reject: restore the state and the time
                if ((e = cudaMemcpyAsync(c, w->backup, bytes, cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
                    (e = cudaMemcpyAsync(&w->sc->t, &w->sc->t_save, sizeof(double), cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
                    return cuda_fail(e, "adaptive step restore");
                w->sub = std::min(2 * s, kMaxSub);
                continue;
            }
            w->sub_last = s;
            w->sub_total += s;
            if (!(err <= w->err_last)) w->err_last = err;
            if (s > 1 && err * ldexp(1.0, p->cfg.m + 1) < tol) w->sub = s / 2;
            break;
        }
    }
    w->steps_last = nsteps;
    return HX_OK;
}

int krylov_step(Problem *p, void *c, double dt, int nsteps)
{
    int rc = ensure_work(p);
    if (rc) return rc;
    Work *w = work_of(p);
    cudaStream_t st = p->stream;
    cudaError_t e;
    // the problem time is authoritative in p->dscal[0]; the step graph advances sc->t
    if ((e = cudaMemcpyAsync(&w->sc->t, p->dscal, sizeof(double), cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(&w->sc->flags, 0, sizeof(int), st)) != cudaSuccess)
        return cuda_fail(e, "step set-up");
    if (p->cfg.tol > 0.0) {
        if ((rc = adaptive_steps(p, w, c, dt, nsteps))) return rc;
    } else {
        if ((rc = ensure_graph(p, w, c, dt))) return rc;
        for (int s = 0; s < nsteps; ++s)
            if ((e = cudaGraphLaunch(w->exec, st)) != cudaSuccess) return cuda_fail(e, "graph launch");
        w->sub_last = 1;
        w->sub_total = nsteps;
        w->steps_last = nsteps;
        w->err_last = 0.0;
    }
    if ((e = cudaMemcpyAsync(p->dscal, &w->sc->t, sizeof(double), cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return cuda_fail(e, "step copy-out");
    p->t_host += dt * nsteps;
    return HX_OK;
}

int krylov_substeps(Problem *p, int *last, long long *total, double *err_max)
{
    Work *w = work_of(p);
    if (!w) { set_error("hx_step_substeps: no step has run"); return HX_EINVAL; }
    if (last) *last = w->sub_last;
    if (total) *total = w->sub_total;
    if (err_max) *err_max = w->err_last;
    return HX_OK;
}

// Device buffer for hx_step_host (kept, so the captured graph stays valid between calls).
void *krylov_host_state(Problem *p)
{
    if (ensure_work(p)) return nullptr;
    Work *w = work_of(p);
    if (!w->host_state && cudaMalloc((void **)&w->host_state, std::max<size_t>(p->set->h.size, 1) * 16) != cudaSuccess)
        return nullptr;
    return w->host_state;
}

int krylov_info(Problem *p, int *m_used, double *alpha, double *beta, double *norm)
{
    Work *w = work_of(p);
    if (!w) { set_error("hx_step_info: no step has run"); return HX_EINVAL; }
    Scal sc;
    cudaError_t e = cudaStreamSynchronize(p->stream);
    if (e == cudaSuccess) e = cudaMemcpy(&sc, w->sc, sizeof(Scal), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "hx_step_info");
    if (m_used) *m_used = sc.m_used;
    for (int i = 0; i < sc.m_used; ++i) {
        if (alpha) alpha[i] = sc.alpha[i];
        if (beta && i + 1 < sc.m_used) beta[i] = sc.beta[i];
    }
    if (norm) *norm = sc.norm_out;
    if (sc.flags & 2) { set_error("non-finite norm in a time step"); return HX_ENONFINITE; }
    if (sc.flags & 4) { set_error("tridiagonal eigensolver did not converge in 60 iterations"); return HX_ENONFINITE; }
    if (sc.flags & 1) { set_error("Lanczos breakdown: fewer than m vectors were used"); return HX_EBREAKDOWN; }
    return HX_OK;
}


// ---------------------------------------------------------------------------------------
// Batches.  Three schedules of the same kernels (each member's arithmetic is the same in all
// three, so they give the same bits):
//   kSchedMembers  one graph per step with every member's step as an independent child graph;
//   kSchedBatched  per Lanczos index one persistent product launch per (precision, degree) class
//                  over all members (batch_apply_kernel: tiles of any member from one queue,
//                  largest members first), the members' projections, Gram-Schmidt passes,
//                  exponentials and recombinations forked from and joined to those launches;
//   kSchedHybrid   members that fill the GPU alone (|K| of at least one wave of product blocks)
//                  run their whole step on their own stream, the others as in kSchedBatched;
//   kSchedSerial   members with a kernel specialised to their potential and at least four waves
//                  of product blocks run their own step graph's kernels (specialised product,
//                  fused projections) one member after another, nothing else running beside
//                  them, then the others as in kSchedBatched.
// The first three give the same bits; kSchedSerial gives the single-problem step's bits for its
// large members.  The first steps of a call time each candidate graph once and keep the fastest;
// the tile size of the batched launches is chosen before that by timing the candidate sizes.
// ---------------------------------------------------------------------------------------
// Kernel nodes of a graph, child graphs included: the launches of one replay.
static int count_kernel_nodes(cudaGraph_t g)
{
    size_t n = 0;
    if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess) return -1;
    std::vector<cudaGraphNode_t> nodes(n);
    if (n && cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return -1;
    int k = 0;
    for (cudaGraphNode_t x : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(x, &t) != cudaSuccess) return -1;
        if (t == cudaGraphNodeTypeKernel) ++k;
        else if (t == cudaGraphNodeTypeGraph) {
            cudaGraph_t child;
            if (cudaGraphChildGraphNodeGetGraph(x, &child) != cudaSuccess) return -1;
            const int c = count_kernel_nodes(child);
            if (c < 0) return -1;
            k += c;
        }
    }
    return k;
}

static int batch_instantiate(Batch *b, int sched, cudaGraph_t g)
{
    b->kern[sched] = count_kernel_nodes(g);
    cudaError_t e = cudaGraphInstantiate(&b->exec[sched], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { b->exec[sched] = nullptr; return cuda_fail(e, "batch instantiate"); }
    if ((e = cudaGraphUpload(b->exec[sched], b->stream)) != cudaSuccess) return cuda_fail(e, "batch graph upload");
    return HX_OK;
}

static int batch_capture_members(Batch *b, void *const *c, double dt)
{
    const int np = (int)b->probs.size();
    cudaError_t e;
    cudaGraph_t g;
    if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) return cuda_fail(e, "batch graph");
    for (int i = 0; i < np; ++i) {
        Problem *p = b->probs[i];
        Work *w = work_of(p);
        cudaGraph_t child;
        if ((e = cudaStreamBeginCapture(w->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
            cudaGraphDestroy(g);
            return cuda_fail(e, "batch capture");
        }
        g_batch_capture = true;             // batch members run the generic apply kernel
        int rc = enqueue(p, w, (double2 *)c[i], w->cap_stream, dt);
        g_batch_capture = false;
        e = cudaStreamEndCapture(w->cap_stream, &child);
        if (rc || e != cudaSuccess) {
            if (e == cudaSuccess) cudaGraphDestroy(child);
            cudaGraphDestroy(g);
            return rc ? rc : cuda_fail(e, "batch capture");
        }
        cudaGraphNode_t node;
        e = cudaGraphAddChildGraphNode(&node, g, nullptr, 0, child);
        cudaGraphDestroy(child);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            return cuda_fail(e, "batch child node");
        }
    }
    return batch_instantiate(b, kSchedMembers, g);
}

namespace {
struct BatchGroup {
    bool c64;
    int md;
    std::vector<int> members;       // batch indices, largest first
    size_t args_off;                // device offset of mmax x count launch arguments (k-major)
    std::vector<size_t> tiles_off;  // per Lanczos index: the tile list (members with m > k)
    std::vector<int> ntiles;
    size_t queue_off;
};
}  // namespace

static int batch_mmax(const Batch *b)
{
    int m = 0;
    for (const Problem *p : b->probs) m = std::max(m, p->cfg.m);
    return m;
}

static bool batch_allows_batched(const Batch *b)
{
    for (const Problem *p : b->probs)
        if (p->cfg.scheme != HX_SCHEME_EXPMPR || p->ops1.nops > 0 || p->set->d.general || p->cfg.tol > 0.0)
            return false;
    return true;
}

// Members that take part in the batched product launches of a schedule.
static bool batch_in_launch(const Batch *b, int sched, int i)
{
    if (sched == kSchedBatched) return true;
    const Problem *p = b->probs[i];
    const int64_t wave = (int64_t)p->num_sms * 4 * kApplyThreads;    // one wave of product blocks
    if (sched == kSchedSerial) return !(p->jit && (int64_t)p->set->h.size >= 4 * wave);
    return (int64_t)p->set->h.size < wave;
}

static std::vector<BatchGroup> batch_groups(const Batch *b, int sched, int tile, size_t &bytes)
{
    std::vector<BatchGroup> gs;
    for (int i = 0; i < (int)b->probs.size(); ++i) {
        if (!batch_in_launch(b, sched, i)) continue;
        const Problem *p = b->probs[i];
        const bool c64 = p->cfg.dtype == HX_C64;
        const int md = max_degree(p) <= 3 ? 3 : kMaxDeg;
        BatchGroup *g = nullptr;
        for (auto &x : gs)
            if (x.c64 == c64 && x.md == md) g = &x;
        if (!g) { gs.push_back(BatchGroup{c64, md, {}, 0, {}, {}, 0}); g = &gs.back(); }
        g->members.push_back(i);
    }
    const int mmax = batch_mmax(b);
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    bytes = 0;
    for (auto &g : gs) {
        std::stable_sort(g.members.begin(), g.members.end(),
                         [&](int x, int y) { return b->probs[x]->set->h.size > b->probs[y]->set->h.size; });
        g.args_off = bytes;
        bytes = al(bytes + (size_t)mmax * g.members.size() * apply_args_size());
        g.tiles_off.assign(mmax, 0);
        g.ntiles.assign(mmax, 0);
        for (int k = 0; k < mmax; ++k) {
            for (int i : g.members)
                if (b->probs[i]->cfg.m > k) g.ntiles[k] += (int)((b->probs[i]->set->h.size + tile - 1) / tile);
            g.tiles_off[k] = bytes;
            bytes = al(bytes + (size_t)g.ntiles[k] * sizeof(int2));
        }
        g.queue_off = bytes;
        bytes = al(bytes + sizeof(BatchQueue));
    }
    return gs;
}

// Device copies of the groups' launch arguments and tile lists (the queues are cleared).
static int batch_upload(Batch *b, int sched, const std::vector<BatchGroup> &gs, size_t bytes, double dt, int tile)
{
    if (bytes > b->dmem_bytes[sched]) {
        cudaFree(b->dmem[sched]);
        b->dmem[sched] = nullptr;
        b->dmem_bytes[sched] = 0;
        cudaError_t e = cudaMalloc(&b->dmem[sched], bytes);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(batch tables)");
        b->dmem_bytes[sched] = bytes;
    }
    if (bytes == 0) return HX_OK;
    std::vector<char> host(bytes, 0);
    const int mmax = batch_mmax(b);
    for (const auto &g : gs) {
        for (int k = 0; k < mmax; ++k) {
            int2 *tl = (int2 *)(host.data() + g.tiles_off[k]);
            int t = 0;
            for (size_t j = 0; j < g.members.size(); ++j) {
                Problem *p = b->probs[g.members[j]];
                if (p->cfg.m <= k) continue;
                Work *w = work_of(p);
                const size_t es = p->cfg.dtype == HX_C64 ? 8 : 16, ld = w->vec_bytes / es;
                char *V = (char *)w->V;
                batch_member_args(p, V + (size_t)k * ld * es, V + (size_t)(k + 1) * ld * es, &w->sc->t, 0.5 * dt,
                                  &w->sc->s[k],
                                  host.data() + g.args_off + ((size_t)k * g.members.size() + j) * apply_args_size());
                const int n = (int)p->set->h.size;
                for (int s = 0; s < n; s += tile) tl[t++] = make_int2((int)j, s);
            }
        }
    }
    cudaError_t e = cudaMemcpy(b->dmem[sched], host.data(), bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "upload batch tables");
    return HX_OK;
}

static int batch_products(Batch *b, int sched, const std::vector<BatchGroup> &gs, int k, int tile, long long budget,
                          cudaStream_t st)
{
    const Problem *p0 = b->probs[0];
    for (const auto &g : gs) {
        if (g.ntiles[k] == 0) continue;
        const char *base = (const char *)b->dmem[sched];
        int rc = launch_batch_apply(g.c64, g.md, base + g.args_off + (size_t)k * g.members.size() * apply_args_size(),
                                    (const int2 *)(base + g.tiles_off[k]), g.ntiles[k], tile, budget,
                                    (void *)(base + g.queue_off), p0->num_sms, st);
        if (rc) return rc;
    }
    return HX_OK;
}

// The tile size: each candidate's batched products (all members) for the first Lanczos index,
// timed on the batch's capture stream after a warm-up launch (the workspace's contents do not
// matter for the time; the next step overwrites them), the fastest kept.
static int batch_autotune(Batch *b, double dt)
{
    const int cand[] = {256, 512, 1024, 2048, 4096};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(e, "batch autotune events");
    }
    b->tune_tiles.clear();
    b->tune_ms.clear();
    double best = 1e300;
    int best_tile = 1024, rc = HX_OK;
    for (int tile : cand) {
        size_t bytes;
        auto gs = batch_groups(b, kSchedBatched, tile, bytes);
        if ((rc = batch_upload(b, kSchedBatched, gs, bytes, dt, tile)) ||
            (rc = batch_products(b, kSchedBatched, gs, 0, tile, -1, b->cap)))      // warm-up
            break;
        cudaEventRecord(e0, b->cap);
        rc = batch_products(b, kSchedBatched, gs, 0, tile, -1, b->cap);
        cudaEventRecord(e1, b->cap);
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess && !rc) rc = cuda_fail(e, "batch autotune");
        if (rc) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        b->tune_tiles.push_back(tile);
        b->tune_ms.push_back(ms);
        if (ms < best) { best = ms; best_tile = tile; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!rc) b->tile = best_tile;
    return rc;
}

static int batch_capture_batched(Batch *b, int sched, void *const *c, double dt)
{
    const int np = (int)b->probs.size();
    const int m = batch_mmax(b);
    size_t bytes;
    auto gs = batch_groups(b, sched, b->tile, bytes);
    int rc = batch_upload(b, sched, gs, bytes, dt, b->tile);
    if (rc) return rc;
    cudaError_t e;
    cudaGraph_t g;
    if ((e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return cuda_fail(e, "batch capture");
    auto fork = [&](int i) {
        Work *w = work_of(b->probs[i]);
        if ((e = cudaEventRecord(b->ev[np], b->cap)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(w->cap_stream, b->ev[np], 0)) != cudaSuccess)
            return cuda_fail(e, "batch fork");
        return (int)HX_OK;
    };
    auto join = [&](int i) {
        Work *w = work_of(b->probs[i]);
        if ((e = cudaEventRecord(b->ev[i], w->cap_stream)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(b->cap, b->ev[i], 0)) != cudaSuccess)
            return cuda_fail(e, "batch join");
        return (int)HX_OK;
    };
    // members outside the batched launches: their whole step, on their own stream (hybrid) or one
    // after another on the batch stream with their own kernels (serial)
    for (int i = 0; i < np && !rc; ++i) {
        if (batch_in_launch(b, sched, i)) continue;
        Problem *p = b->probs[i];
        if (sched == kSchedSerial) {
            rc = enqueue(p, work_of(p), (double2 *)c[i], b->cap, dt);
            continue;
        }
        if ((rc = fork(i))) break;
        g_batch_capture = true;
        rc = enqueue(p, work_of(p), (double2 *)c[i], work_of(p)->cap_stream, dt);
        g_batch_capture = false;
    }
    // phase: -1 start vectors, 0..m-1 work after product k, m the end
    for (int phase = kPhaseInit; phase <= m && !rc; ++phase) {
        if (phase >= 0 && phase < m && (rc = batch_products(b, sched, gs, phase, b->tile, b->budget, b->cap))) break;
        for (int i = 0; i < np && !rc; ++i) {
            Problem *p = b->probs[i];
            if (!batch_in_launch(b, sched, i) || phase > p->cfg.m) continue;   // own stream, or its step ended
            if (!(rc = fork(i)) && !(rc = enqueue(p, work_of(p), (double2 *)c[i], work_of(p)->cap_stream, dt, phase)))
                rc = join(i);
        }
    }
    for (int i = 0; i < np && !rc && sched != kSchedSerial; ++i)
        if (!batch_in_launch(b, sched, i)) rc = join(i);
    e = cudaStreamEndCapture(b->cap, &g);
    if (rc) {
        if (e == cudaSuccess) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "batch capture");
    return batch_instantiate(b, sched, g);
}

int batch_timed_out(Batch *b)
{
    if (b->schedule <= kSchedMembers) return 0;
    int out = 0;
    for (int sched : {kSchedBatched, kSchedHybrid, kSchedSerial}) {
        if (!b->dmem[sched] || !b->exec[sched]) continue;
        size_t bytes;
        auto gs = batch_groups(b, sched, b->tile, bytes);
        for (const auto &g : gs) {
            BatchQueue q;
            BatchQueue *dq = (BatchQueue *)((char *)b->dmem[sched] + g.queue_off);
            if (cudaMemcpy(&q, dq, sizeof(q), cudaMemcpyDeviceToHost) != cudaSuccess) return 0;
            if (q.timeout) {
                out = 1;
                cudaMemset(&dq->timeout, 0, sizeof(int));
            }
        }
    }
    return out;
}

void batch_drop_graphs(Batch *b)
{
    for (int s = 0; s < kNumSched; ++s) {
        if (b->exec[s]) cudaGraphExecDestroy(b->exec[s]);
        b->exec[s] = nullptr;
        b->kern[s] = 0;
    }
}

// Candidate schedules: forced by HX_BATCH_BATCHED (0 member graphs, 1 batched, 2 hybrid, 3 serial),
// else every schedule that the members allow and that differs from the others.
static std::vector<int> batch_candidates(const Batch *b)
{
    const char *env = getenv("HX_BATCH_BATCHED");
    const bool ok = batch_allows_batched(b);
    if (env && env[0] == '0') return {kSchedMembers};
    if (!ok) return {kSchedMembers};
    if (env && env[0] >= '1' && env[0] <= '3') return {env[0] - '0'};
    const int np = (int)b->probs.size();
    int small = 0, rest = 0;
    for (int i = 0; i < np; ++i) {
        small += batch_in_launch(b, kSchedHybrid, i);
        rest += batch_in_launch(b, kSchedSerial, i);
    }
    std::vector<int> c = {kSchedMembers, kSchedBatched};
    if (small > 0 && small < np) c.push_back(kSchedHybrid);
    if (rest < np) c.push_back(kSchedSerial);
    return c;
}

int batch_step(Batch *b, void *const *c, double dt, int nsteps)
{
    const int np = (int)b->probs.size();
    for (Problem *p : b->probs) {
        int rc = ensure_work(p);
        if (rc) return rc;
    }
    const std::vector<int> cand = batch_candidates(b);
    bool same = b->dt == dt && b->cand == cand;
    for (int i = 0; same && i < np; ++i) same = b->cptr[i] == c[i] && b->gen[i] == b->probs[i]->generation;
    for (int s : cand) same = same && b->exec[s];
    cudaError_t e;
    if (!same) {
        // the tables below are read by a graph of this batch that may still run, and the tile
        // autotuner writes into the members' workspaces: wait for the batch and member streams
        if ((e = cudaStreamSynchronize(b->stream)) != cudaSuccess) return cuda_fail(e, "batch sync");
        for (Problem *p : b->probs)
            if ((e = cudaStreamSynchronize(p->stream)) != cudaSuccess) return cuda_fail(e, "batch sync");
        batch_drop_graphs(b);
        b->schedule = cand.size() == 1 ? cand[0] : -1;
        for (int s = 0; s < kNumSched; ++s) b->sched_ms[s] = -1.f;
        if (!b->cap && (e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(e, "cudaStreamCreate(batch)");
        for (int i = (int)b->ev.size(); i < np + 1; ++i) {
            cudaEvent_t ev;
            if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
                return cuda_fail(e, "cudaEventCreate(batch)");
            b->ev.push_back(ev);
        }
        for (int s : cand) {
            int rc;
            if (s != kSchedMembers && b->tile == 0 && (rc = batch_autotune(b, dt))) return rc;
            rc = s == kSchedMembers ? batch_capture_members(b, c, dt) : batch_capture_batched(b, s, c, dt);
            if (rc) { batch_drop_graphs(b); return rc; }
        }
        b->cand = cand;
        b->cptr.assign(c, c + np);
        b->gen.resize(np);
        for (int i = 0; i < np; ++i) b->gen[i] = b->probs[i]->generation;
        b->dt = dt;
    }
    cudaStream_t st = b->stream;
    for (Problem *p : b->probs) {
        Work *w = work_of(p);
        if ((e = cudaMemcpyAsync(&w->sc->t, p->dscal, sizeof(double), cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
            (e = cudaMemsetAsync(&w->sc->flags, 0, sizeof(int), st)) != cudaSuccess)
            return cuda_fail(e, "batch set-up");
    }
    int s = 0;
    // schedule choice: the next untimed candidate runs one step between two events
    while (b->schedule < 0 && s < nsteps) {
        int next = -1;
        for (int x : b->cand)
            if (b->sched_ms[x] < 0.f) { next = x; break; }
        cudaEvent_t e0, e1;
        if ((e = cudaEventCreate(&e0)) != cudaSuccess) return cuda_fail(e, "batch timing");
        if ((e = cudaEventCreate(&e1)) != cudaSuccess) { cudaEventDestroy(e0); return cuda_fail(e, "batch timing"); }
        cudaEventRecord(e0, st);
        e = cudaGraphLaunch(b->exec[next], st);
        cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (e != cudaSuccess) return cuda_fail(e, "batch graph launch");
        b->sched_ms[next] = ms;
        ++s;
        bool all = true;
        for (int x : b->cand) all = all && b->sched_ms[x] >= 0.f;
        if (all) {
            int best = b->cand[0];
            for (int x : b->cand)
                if (b->sched_ms[x] < b->sched_ms[best]) best = x;
            b->schedule = best;
        }
    }
    const int run = b->schedule >= 0 ? b->schedule : b->cand[0];
    for (; s < nsteps; ++s)
        if ((e = cudaGraphLaunch(b->exec[run], st)) != cudaSuccess) return cuda_fail(e, "batch graph launch");
    for (Problem *p : b->probs) {
        Work *w = work_of(p);
        if ((e = cudaMemcpyAsync(p->dscal, &w->sc->t, sizeof(double), cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
            return cuda_fail(e, "batch copy-out");
        p->t_host += dt * nsteps;
    }
    return HX_OK;
}

void batch_free(Batch *b)
{
    batch_drop_graphs(b);
    for (int s = 0; s < kNumSched; ++s) {
        cudaFree(b->dmem[s]);
        b->dmem[s] = nullptr;
        b->dmem_bytes[s] = 0;
    }
    for (cudaEvent_t ev : b->ev) cudaEventDestroy(ev);
    b->ev.clear();
    if (b->cap) cudaStreamDestroy(b->cap);
    b->cap = nullptr;
}

// ---------------------------------------------------------------------------------------
// Lanczos workspaces outside the step graph (used by the adjoint gradient): the same kernels,
// complex128 vectors, launched directly.
// ---------------------------------------------------------------------------------------
int lanczos_alloc(Problem *p, int m, LanczosWS *L)
{
    memset(L, 0, sizeof(*L));
    const size_t n = (size_t)p->set->h.size;
    L->vec_bytes = ((n * 16 + 255) / 256) * 256;
    L->m = m;
    const int G = apply_grid(p);
    cudaError_t e;
    if ((e = cudaMalloc(&L->V, L->vec_bytes * (m + 1))) != cudaSuccess ||
        (e = cudaMalloc((void **)&L->partials, (size_t)G * 2 * (kMaxKrylov + 2) * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&L->sc, sizeof(Scal))) != cudaSuccess) {
        lanczos_free(L);
        return cuda_fail(e, "cudaMalloc(Lanczos workspace)");
    }
    cudaMemset(L->sc, 0, sizeof(Scal));
    return HX_OK;
}

void lanczos_free(LanczosWS *L)
{
    cudaFree(L->V);
    cudaFree(L->partials);
    cudaFree(L->sc);
    memset(L, 0, sizeof(*L));
}

template <int NV>
static int lanczos_enqueue_t(Problem *p, LanczosWS *L, const double2 *c, const double *t_ptr, double t_shift,
                             cudaStream_t st)
{
    const int n = p->set->d.size, m = L->m, G = apply_grid(p), T = 256;
    double2 *Vb = (double2 *)L->V;
    const size_t ld = L->vec_bytes / sizeof(double2);
    Scal *sc = (Scal *)L->sc;
    init_kernel<double2><<<G, T, 0, st>>>(c, Vb, n, L->partials, sc, m);
    for (int k = 0; k < m; ++k) {
        ApplyFuse f;
        memset(&f, 0, sizeof(f));
        f.in_scale = &sc->s[k];
        int rc = launch_apply(p, Vb + (size_t)k * ld, Vb + (size_t)(k + 1) * ld, t_ptr, t_shift, &f, st);
        if (rc) return rc;
        double2 *wv = Vb + (size_t)(k + 1) * ld;
        dot_kernel<double2, NV><<<resident_grid(p, dot_kernel<double2, NV>, T), T, 0, st>>>(wv, Vb, ld, n, k, L->partials, sc);
        update_kernel<double2, NV, 0><<<resident_grid(p, update_kernel<double2, NV, 0>, T), T, 0, st>>>(wv, Vb, ld, n, k,
                                                                                                       L->partials, sc);
        if (k < m - 1)
            update_kernel<double2, NV, 1><<<resident_grid(p, update_kernel<double2, NV, 1>, T), T, 0, st>>>(wv, Vb, ld, n, k,
                                                                                                          L->partials, sc);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HX_OK : cuda_fail(e, "Lanczos kernel launch");
}

int lanczos_enqueue(Problem *p, LanczosWS *L, const double2 *c, const double *t_ptr, double t_shift, cudaStream_t st)
{
    return L->m <= 8 ? lanczos_enqueue_t<8>(p, L, c, t_ptr, t_shift, st)
                     : lanczos_enqueue_t<kMaxKrylov>(p, L, c, t_ptr, t_shift, st);
}

// Eigen-decomposition of T (kept in the workspace) and, when out != nullptr,
// out = beta_0 V Q exp(-i h Lambda) Q^T e_1.
int lanczos_exp(Problem *p, LanczosWS *L, double h, double2 *out, cudaStream_t st)
{
    const int n = p->set->d.size, G = apply_grid(p);
    Scal *sc = (Scal *)L->sc;
    launch_eig(sc, L->m, h, st);
    if (out) {
        const size_t ld = L->vec_bytes / sizeof(double2);
        if (L->m <= 8) combine_kernel<double2, 8><<<G, 256, 0, st>>>(out, (const double2 *)L->V, ld, n, L->partials, sc);
        else combine_kernel<double2, kMaxKrylov><<<G, 256, 0, st>>>(out, (const double2 *)L->V, ld, n, L->partials, sc);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HX_OK : cuda_fail(e, "Lanczos exp launch");
}

// out = (operator of px) v_r for the orthonormal Lanczos vector v_r of L.
int lanczos_apply_basis(Problem *px, LanczosWS *L, int r, double2 *out, const double *t_ptr, cudaStream_t st)
{
    Scal *sc = (Scal *)L->sc;
    ApplyFuse f;
    memset(&f, 0, sizeof(f));
    f.in_scale = &sc->s[r];
    const size_t ld = L->vec_bytes / sizeof(double2);
    return launch_apply(px, (const double2 *)L->V + (size_t)r * ld, out, t_ptr, 0.0, &f, st);
}

// Mcol[2 i .. 2 i + 1] = <v_i, w> for the orthonormal Lanczos vectors v_i, i < m_used.
__global__ void copy_h_kernel(const Scal *sc, double *Mcol, int m)
{
    for (int i = threadIdx.x; i < 2 * m; i += blockDim.x) Mcol[i] = i < 2 * sc->m_used ? sc->h[i] : 0.0;
}

int lanczos_project(Problem *p, LanczosWS *L, const double2 *w, double *Mcol, cudaStream_t st)
{
    const int n = p->set->d.size, G = apply_grid(p);
    Scal *sc = (Scal *)L->sc;
    const size_t ld = L->vec_bytes / sizeof(double2);
    // dot_kernel with k = m - 1 projects on every stored vector (vectors beyond m_used are skipped)
    if (L->m <= 8) dot_kernel<double2, 8><<<G, 256, 0, st>>>(w, (const double2 *)L->V, ld, n, L->m - 1, L->partials, sc, 1);
    else dot_kernel<double2, kMaxKrylov><<<G, 256, 0, st>>>(w, (const double2 *)L->V, ld, n, L->m - 1, L->partials, sc, 1);
    copy_h_kernel<<<1, 64, 0, st>>>(sc, Mcol, L->m);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HX_OK : cuda_fail(e, "projection launch");
}

// (e^z - 1) / z for z = i theta, theta real.
__device__ double2 phi1_imag(double theta)
{
    if (fabs(theta) < 1e-4) {
        const double t2 = theta * theta;
        return make_double2(1.0 - t2 / 6.0 + t2 * t2 / 120.0, theta / 2.0 - theta * t2 / 24.0);
    }
    return make_double2(sin(theta) / theta, (1.0 - cos(theta)) / theta);
}

// Adds to *gacc (complex) the sub-step term of d<phi, psi_M>/du,
//   -i dt integral_0^1 (e^{i(1-s) dt A} lambda_n)^H X (e^{-i s dt A} psi_{n-1}) ds,
// with both exponentials in their Krylov spaces (Lanczos of psi_{n-1} in Lp, of lambda_n in Ll,
// eigen-decompositions already stored): with T_psi = Q_p diag(mu) Q_p^T, T_lam = Q_l diag(lam) Q_l^T,
// a = Q_l^T e_1, b = Q_p^T e_1 and M_pr = <v^l_p, X v^p_r>, the term is
//   -i dt beta_l beta_p sum_{p,r} M_pr sum_{j,k} Q_l[p,j] Q_p[r,k] a_j b_k e^{-i dt lam_j} phi_1(-i dt (mu_k - lam_j)),
// phi_1(z) = (e^z - 1)/z, because integral_0^1 e^{-i dt ((1-s) lam_j + s mu_k)} ds = e^{-i dt lam_j} phi_1(...).
__global__ void __launch_bounds__(32) adjoint_term_kernel(const Scal *Sp, const Scal *Sl, const double *M, int mmax,
                                                          double dt, double *gacc)
{
    __shared__ double Fr[kMaxKrylov * kMaxKrylov], Fi[kMaxKrylov * kMaxKrylov];
    __shared__ double Gr[kMaxKrylov * kMaxKrylov], Gi[kMaxKrylov * kMaxKrylov];
    const int lane = threadIdx.x;
    const int mp = Sp->m_used, ml = Sl->m_used;
    // F_jk = a_j b_k e^{-i dt lam_j} phi_1(-i dt (mu_k - lam_j))
    for (int idx = lane; idx < ml * mp; idx += 32) {
        const int j = idx / mp, k = idx % mp;
        const double aj = Sl->Q[0 * ml + j], bk = Sp->Q[0 * mp + k];
        const double2 ph = phi1_imag(-dt * (Sp->lam[k] - Sl->lam[j]));
        const double c = cos(dt * Sl->lam[j]), s = -sin(dt * Sl->lam[j]);
        Fr[idx] = aj * bk * (c * ph.x - s * ph.y);
        Fi[idx] = aj * bk * (c * ph.y + s * ph.x);
    }
    __syncwarp();
    // H = F Q_p^T, then G = Q_l H
    for (int idx = lane; idx < ml * mp; idx += 32) {
        const int j = idx / mp, r = idx % mp;
        double hr = 0.0, hi = 0.0;
        for (int k = 0; k < mp; ++k) {
            const double q = Sp->Q[r * mp + k];
            hr += Fr[j * mp + k] * q;
            hi += Fi[j * mp + k] * q;
        }
        Gr[idx] = hr;
        Gi[idx] = hi;
    }
    __syncwarp();
    double gr_loc[kMaxKrylov], gi_loc[kMaxKrylov];   // this lane's entries of G, written after all reads
    int cnt = 0;
    for (int idx = lane; idx < ml * mp; idx += 32, ++cnt) {
        const int pp = idx / mp, r = idx % mp;
        double gr = 0.0, gi = 0.0;
        for (int j = 0; j < ml; ++j) {
            const double ql = Sl->Q[pp * ml + j];
            gr += ql * Gr[j * mp + r];
            gi += ql * Gi[j * mp + r];
        }
        gr_loc[cnt] = gr;
        gi_loc[cnt] = gi;
    }
    __syncwarp();
    cnt = 0;
    for (int idx = lane; idx < ml * mp; idx += 32, ++cnt) {
        Gr[idx] = gr_loc[cnt];
        Gi[idx] = gi_loc[cnt];
    }
    __syncwarp();
    // sum_{p,r} M_pr G_pr, M stored by columns: M[(r * mmax + p) * 2 + {0,1}] = <v^l_p, X v^p_r>
    double sr = 0.0, si = 0.0;
    for (int idx = lane; idx < ml * mp; idx += 32) {
        const int pp = idx / mp, r = idx % mp;
        const double mr = M[(r * mmax + pp) * 2], mi = M[(r * mmax + pp) * 2 + 1];
        sr += mr * Gr[idx] - mi * Gi[idx];
        si += mr * Gi[idx] + mi * Gr[idx];
    }
    for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    if (lane == 0) {
        const double scale = dt * Sl->beta0 * Sp->beta0;   // times -i
        gacc[0] += scale * si;
        gacc[1] += -scale * sr;
    }
}

int adjoint_term(LanczosWS *Lp, LanczosWS *Ll, const double *M, double dt, double *gacc, cudaStream_t st)
{
    adjoint_term_kernel<<<1, 32, 0, st>>>((const Scal *)Lp->sc, (const Scal *)Ll->sc, M, Ll->m, dt, gacc);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HX_OK : cuda_fail(e, "adjoint term launch");
}

}  // namespace hx
