// Time stepping: the exponential midpoint rule c^{n+1} = exp(-i h A(t^n + h/2)) c^n (Eq. (expMPR),
// Sec. 2.1) with the exponential approximated by an m-step Hermitian Lanczos process,
// c^{n+1} = ||c^n|| V_m exp(-i h T_m) e_1 (Sec. 2.2), entirely on the device.
//
// One step is a fixed sequence of kernels (captured once into a CUDA graph and replayed):
//   init      v_0 = c (in the Krylov dtype), beta_0 = ||c|| (FP64)
//   for k = 0 .. m-1:
//     apply   w = A(t + h/2) v_k                              (hx_apply.cu)
//     dot     h_i = <v_i, w>, i <= k                            (FP64)
//     update  w -= sum_i h_i v_i;  h'_i = <v_i, w>               (FP64)
//     update  w -= sum_i h'_i v_i; beta_k = ||w||, v_{k+1} = w / beta_k   (k < m-1)
//     alpha_k = Re(h_k + h'_k)
//   eig       T_m = Q diag(lambda) Q^T (cyclic Jacobi, FP64), y = beta_0 Q exp(-i h lambda) Q^T e_1
//   combine   c = sum_i y_i v_i  (complex128 accumulation)
// Classical Gram-Schmidt applied twice keeps V_m orthonormal to working precision.  Vectors are
// stored unnormalised with a device scale s_k (v_k = s_k * stored_k) so no pass is spent on
// normalisation.  All scalars live in device memory, so the step has no host round trip.
#include <math.h>

#include "hx_internal.h"

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
    double scale;                   // running max_i(|alpha_i| + beta_{i-1}) for the breakdown test
    double norm_out;
    int m_used;
    int flags;                      // bit 0: breakdown seen, bit 1: non-finite
    unsigned counter;
};

struct Work {
    Scal *sc;
    void *V;                        // (m + 1) x n vectors of the Krylov dtype
    double2 *state;                 // complex128 state the captured graph reads and writes
    double2 *host_state;            // device buffer used by hx_step_host
    double *partials;               // G x 2 (m + 2)
    size_t vec_bytes;
    cudaGraphExec_t exec;
    cudaStream_t cap_stream;
    double dt;
};

static Work *work_of(Problem *p) { return (Work *)p->krylov; }

__device__ double block_reduce(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    __syncthreads();
    return s;   // thread 0
}

// Writes nval per-block sums to partials[blockIdx.x * nval + j].  In the last block to arrive, all
// threads then add the partials up (each thread a fixed strided subset, then a fixed tree), so the
// totals land in tot[0..nval) (shared) in an order that does not depend on block timing.  Returns
// true in every thread of that last block.
__device__ bool reduce_partials(const double *vals, int nval, double *partials, unsigned *counter, double *red,
                                double *tot)
{
    __shared__ bool last;
    for (int j = 0; j < nval; ++j) {
        double s = block_reduce(vals[j], red);
        if (threadIdx.x == 0) partials[blockIdx.x * nval + j] = s;
    }
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    for (int j = 0; j < nval; ++j) {
        double t = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t += ((volatile const double *)partials)[b * nval + j];
        t = block_reduce(t, red);
        if (threadIdx.x == 0) tot[j] = t;
    }
    __syncthreads();
    return true;
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

template <typename V>
__device__ __forceinline__ V to_vec(double2 x);
template <> __device__ __forceinline__ float2 to_vec<float2>(double2 x) { return make_float2((float)x.x, (float)x.y); }
template <> __device__ __forceinline__ double2 to_vec<double2>(double2 x) { return x; }

// v_0 = c in the Krylov dtype; beta_0 = ||c||, s_0 = 1 / beta_0.
template <typename V>
__global__ void init_kernel(const double2 *c, V *v0, int n, double *partials, Scal *sc, int m)
{
    __shared__ double red[32];
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double2 x = c[i];
        v0[i] = to_vec<V>(x);
        acc += x.x * x.x + x.y * x.y;
    }
    __shared__ double tot[1];
    if (reduce_partials(&acc, 1, partials, &sc->counter, red, tot) && threadIdx.x == 0) {
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

template <typename V> struct Real;
template <> struct Real<float2> { using T = float; };
template <> struct Real<double2> { using T = double; };

// h_i = s_i <v_i, w> for i <= k.
template <typename V, int NV>
__global__ void __launch_bounds__(256) dot_kernel(const V *w, const V *Vb, size_t ld, int n, int k, double *partials, Scal *sc)
{
    __shared__ double red[32];
    __shared__ double tot[2 * NV];
    if (k >= sc->m_used) return;
    CAcc<V> acc[NV];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        V x = w[e];
#pragma unroll(NV <= 8 ? NV : 1)
        for (int i = 0; i < NV; ++i)
            if (i <= k) acc[i].add(Vb[i * ld + e], x);
    }
    double vals[2 * NV];
#pragma unroll(NV <= 8 ? NV : 1)
    for (int i = 0; i < NV; ++i) {
        vals[2 * i] = acc[i].r();
        vals[2 * i + 1] = acc[i].i();
    }
    const int nval = 2 * (k + 1);
    if (reduce_partials(vals, nval, partials, &sc->counter, red, tot) && threadIdx.x == 0) {
        for (int i = 0; i <= k; ++i) {
            sc->h[2 * i] = sc->s[i] * tot[2 * i];
            sc->h[2 * i + 1] = sc->s[i] * tot[2 * i + 1];
        }
        sc->counter = 0;
    }
}

// pass 0: w -= sum_i h_i s_i v_i, then h'_i = s_i <v_i, w>, alpha_k = Re(h_k + h'_k).
// pass 1: w -= sum_i h'_i s_i v_i, then beta_k = ||w||, s_{k+1} = 1 / beta_k, breakdown test.
// The update runs in the vector precision; the inner products and the norm as in dot_kernel.
template <typename V, int NV>
__global__ void __launch_bounds__(256) update_kernel(V *w, const V *Vb, size_t ld, int n, int k, int pass, double *partials, Scal *sc)
{
    using R = typename Real<V>::T;
    __shared__ double red[32];
    __shared__ double tot[2 * NV];
    if (k >= sc->m_used) return;
    const double *coef = pass == 0 ? sc->h : sc->h2;
    R cr[NV], ci[NV];
#pragma unroll(NV <= 8 ? NV : 1)
    for (int i = 0; i < NV; ++i) {
        cr[i] = i <= k ? (R)(coef[2 * i] * sc->s[i]) : (R)0;
        ci[i] = i <= k ? (R)(coef[2 * i + 1] * sc->s[i]) : (R)0;
    }
    CAcc<V> acc[NV];
    CAcc<V> nrm;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        V x = w[e];
#pragma unroll(NV <= 8 ? NV : 1)
        for (int i = 0; i < NV; ++i)
            if (i <= k) {
                V v = Vb[i * ld + e];
                x.x -= cr[i] * v.x - ci[i] * v.y;
                x.y -= cr[i] * v.y + ci[i] * v.x;
            }
        w[e] = x;
        if (pass == 0) {
#pragma unroll(NV <= 8 ? NV : 1)
            for (int i = 0; i < NV; ++i)
                if (i <= k) acc[i].add(Vb[i * ld + e], x);
        } else {
            nrm.add(x, x);
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
    if (reduce_partials(vals, nval, partials, &sc->counter, red, tot) && threadIdx.x == 0) {
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
                sc->m_used = k + 1;
                sc->flags |= 1;
            } else {
                sc->beta[k] = b;
                sc->s[k + 1] = 1.0 / b;
            }
        }
        sc->counter = 0;
    }
}

// T_m = Q diag(lambda) Q^T by cyclic Jacobi rotations (Jacobi's method, Golub & Van Loan Sec. 8.5),
// y = beta_0 Q exp(-i h lambda) Q^T e_1; stored as y_i * s_i for the combination pass.  One warp:
// the rotation angle is computed by every lane, the rows and columns it touches are updated one
// lane per index.  Also advances the problem time by h.
__global__ void __launch_bounds__(32) eig_kernel(Scal *sc, double h)
{
    __shared__ double A[kMaxKrylov * kMaxKrylov], Qm[kMaxKrylov * kMaxKrylov];
    __shared__ double cph[kMaxKrylov], sph[kMaxKrylov];
    const int lane = threadIdx.x;
    const int m = sc->m_used;
    for (int i = 0; i < m; ++i)
        if (lane < m) {
            const int j = lane;
            A[i * m + j] = i == j ? sc->alpha[i] : ((j == i + 1 || i == j + 1) ? sc->beta[i < j ? i : j] : 0.0);
            Qm[i * m + j] = i == j ? 1.0 : 0.0;
        }
    __syncwarp();
    double nr = 0.0;
    for (int i = 0; i < m; ++i) nr += A[i * m + i] * A[i * m + i] + (i + 1 < m ? 2.0 * A[i * m + i + 1] * A[i * m + i + 1] : 0.0);
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        if (lane < m)
            for (int j = lane + 1; j < m; ++j) off += A[lane * m + j] * A[lane * m + j];
        for (int o = 16; o > 0; o >>= 1) off += __shfl_xor_sync(0xffffffffu, off, o);
        if (off <= 1e-34 * nr) break;
        for (int p = 0; p < m; ++p)
            for (int q = p + 1; q < m; ++q) {
                const double apq = A[p * m + q];
                if (apq == 0.0) continue;
                const double theta = (A[q * m + q] - A[p * m + p]) / (2.0 * apq);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                __syncwarp();
                if (lane < m) {                      // A <- A J (columns p, q)
                    const double arp = A[lane * m + p], arq = A[lane * m + q];
                    A[lane * m + p] = c * arp - s * arq;
                    A[lane * m + q] = s * arp + c * arq;
                }
                __syncwarp();
                if (lane < m) {                      // A <- J^T A (rows p, q)
                    const double apr = A[p * m + lane], aqr = A[q * m + lane];
                    A[p * m + lane] = c * apr - s * aqr;
                    A[q * m + lane] = s * apr + c * aqr;
                    const double qrp = Qm[lane * m + p], qrq = Qm[lane * m + q];   // Q <- Q J
                    Qm[lane * m + p] = c * qrp - s * qrq;
                    Qm[lane * m + q] = s * qrp + c * qrq;
                }
                __syncwarp();
            }
    }
    if (lane < m) {
        const double ph = -h * A[lane * m + lane];
        cph[lane] = cos(ph);
        sph[lane] = sin(ph);
    }
    __syncwarp();
    if (lane < m) {
        double yr = 0.0, yi = 0.0;
        for (int j = 0; j < m; ++j) {
            const double w = Qm[lane * m + j] * Qm[0 * m + j];
            yr += w * cph[j];
            yi += w * sph[j];
        }
        sc->y[2 * lane] = sc->beta0 * yr * sc->s[lane];
        sc->y[2 * lane + 1] = sc->beta0 * yi * sc->s[lane];
    }
    if (lane == 0) sc->t += h;
}

// c = sum_i y_i v_i (complex128 accumulation), and ||c||^2 for hx_step_info.
template <typename V, int NV>
__global__ void combine_kernel(double2 *c, const V *Vb, size_t ld, int n, double *partials, Scal *sc)
{
    __shared__ double red[32];
    const int m = sc->m_used;
    double yr[NV], yi[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        yr[i] = i < m ? sc->y[2 * i] : 0.0;
        yi[i] = i < m ? sc->y[2 * i + 1] : 0.0;
    }
    double acc = 0.0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        double xr = 0.0, xi = 0.0;
#pragma unroll(NV <= 8 ? NV : 1)
        for (int i = 0; i < NV; ++i)
            if (i < m) {
                V v = Vb[i * ld + e];
                xr += yr[i] * v.x - yi[i] * v.y;
                xi += yr[i] * v.y + yi[i] * v.x;
            }
        c[e] = make_double2(xr, xi);
        acc += xr * xr + xi * xi;
    }
    __shared__ double tot[1];
    if (reduce_partials(&acc, 1, partials, &sc->counter, red, tot) && threadIdx.x == 0) {
        double nr = sqrt(tot[0]);
        sc->norm_out = nr;
        if (!isfinite(nr)) sc->flags |= 2;
        sc->counter = 0;
    }
}

template <typename V, int NV>
static int enqueue_step(Problem *p, Work *w, cudaStream_t st, double dt)
{
    const int n = p->set->d.size;
    const int m = p->cfg.m;
    const int G = apply_grid(p);
    const int T = 256;
    V *Vb = (V *)w->V;
    const size_t ld = w->vec_bytes / sizeof(V);
    Scal *sc = w->sc;
    init_kernel<V><<<G, T, 0, st>>>(w->state, Vb, n, w->partials, sc, m);
    for (int k = 0; k < m; ++k) {
        ApplyFuse f;
        memset(&f, 0, sizeof(f));
        f.in_scale = &sc->s[k];
        int rc = launch_apply(p, Vb + (size_t)k * ld, Vb + (size_t)(k + 1) * ld, &sc->t, 0.5 * dt, &f, st);
        if (rc) return rc;
        V *wv = Vb + (size_t)(k + 1) * ld;
        dot_kernel<V, NV><<<G, T, 0, st>>>(wv, Vb, ld, n, k, w->partials, sc);
        update_kernel<V, NV><<<G, T, 0, st>>>(wv, Vb, ld, n, k, 0, w->partials, sc);
        if (k < m - 1) update_kernel<V, NV><<<G, T, 0, st>>>(wv, Vb, ld, n, k, 1, w->partials, sc);
    }
    eig_kernel<<<1, 32, 0, st>>>(sc, dt);
    combine_kernel<V, NV><<<G, T, 0, st>>>(w->state, Vb, ld, n, w->partials, sc);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "step kernel launch");
    return HX_OK;
}

static int enqueue(Problem *p, Work *w, cudaStream_t st, double dt)
{
    const bool c64 = p->cfg.dtype == HX_C64;
    if (p->cfg.m <= 8)
        return c64 ? enqueue_step<float2, 8>(p, w, st, dt) : enqueue_step<double2, 8>(p, w, st, dt);
    return c64 ? enqueue_step<float2, kMaxKrylov>(p, w, st, dt) : enqueue_step<double2, kMaxKrylov>(p, w, st, dt);
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
    if ((e = cudaMalloc(&w->V, w->vec_bytes * (p->cfg.m + 1))) != cudaSuccess ||
        (e = cudaMalloc((void **)&w->partials, (size_t)G * 2 * (kMaxKrylov + 2) * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc((void **)&w->sc, sizeof(Scal))) != cudaSuccess) {
        cudaFree(w->V); cudaFree(w->partials); cudaFree(w->sc);
        delete w;
        return cuda_fail(e, "cudaMalloc(Krylov workspace)");
    }
    cudaMemset(w->sc, 0, sizeof(Scal));
    // the time lives in the problem's scalar block; copy it in
    cudaMemcpy(&w->sc->t, p->dscal, sizeof(double), cudaMemcpyDeviceToDevice);
    if ((e = cudaStreamCreateWithFlags(&w->cap_stream, cudaStreamNonBlocking)) != cudaSuccess) {
        cudaFree(w->V); cudaFree(w->partials); cudaFree(w->sc);
        delete w;
        return cuda_fail(e, "cudaStreamCreate");
    }
    p->krylov = w;
    return HX_OK;
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
    delete w;
    p->krylov = nullptr;
}

// The step graph is captured for one (state pointer, dt) pair and replayed; a call with another
// vector or step size captures a new graph (a few hundred microseconds).
int krylov_step(Problem *p, void *c, double dt, int nsteps)
{
    int rc = ensure_work(p);
    if (rc) return rc;
    Work *w = work_of(p);
    cudaStream_t st = p->stream;
    cudaError_t e;
    if (!w->exec || w->dt != dt || w->state != (double2 *)c) {
        if (w->exec) { cudaGraphExecDestroy(w->exec); w->exec = nullptr; }
        w->state = (double2 *)c;
        cudaGraph_t g;
        if ((e = cudaStreamBeginCapture(w->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return cuda_fail(e, "begin capture");
        rc = enqueue(p, w, w->cap_stream, dt);
        e = cudaStreamEndCapture(w->cap_stream, &g);
        if (rc) return rc;
        if (e != cudaSuccess) return cuda_fail(e, "end capture");
        e = cudaGraphInstantiate(&w->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { w->exec = nullptr; return cuda_fail(e, "graph instantiate"); }
        w->dt = dt;
    }
    // the problem time is authoritative in p->dscal[0]; the step graph advances sc->t
    if ((e = cudaMemcpyAsync(&w->sc->t, p->dscal, sizeof(double), cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(&w->sc->flags, 0, sizeof(int), st)) != cudaSuccess)
        return cuda_fail(e, "step set-up");
    for (int s = 0; s < nsteps; ++s)
        if ((e = cudaGraphLaunch(w->exec, st)) != cudaSuccess) return cuda_fail(e, "graph launch");
    if ((e = cudaMemcpyAsync(p->dscal, &w->sc->t, sizeof(double), cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return cuda_fail(e, "step copy-out");
    p->t_host += dt * nsteps;
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
    if (sc.flags & 1) { set_error("Lanczos breakdown: fewer than m vectors were used"); return HX_EBREAKDOWN; }
    return HX_OK;
}

}  // namespace hx
