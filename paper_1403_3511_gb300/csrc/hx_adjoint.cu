// Gradient of J = |<phi, psi(T)>|^2 with respect to a piecewise-constant control u(t) that enters
// the potential as u(t) x_axis (hx_adjoint_grad in include/hx.h).
//
// The state is propagated by the exponential midpoint rule, psi_n = U_n psi_{n-1},
// U_n = exp(-i dt A(t_{n-1} + dt/2)) (Eq. (expMPR)), each exponential by Lanczos (Sec. 2.2).
// With a = <phi, psi_M>, lambda_M = phi and lambda_{n-1} = U_n^H lambda_n,
//   dJ/du_q = 2 Re( conj(a) sum_{n in interval q} lambda_n^H (dU_n/du) psi_{n-1} ),
// dU_n/du being the Frechet derivative of exp at -i dt A_n in the direction -i dt X_axis.  Each
// such term is evaluated from the Lanczos bases of psi_{n-1} and lambda_n (adjoint_term in
// hx_krylov.cu), and the same basis of lambda_n gives lambda_{n-1}.  States at the start of every
// control interval are kept (checkpoints); inside an interval they are recomputed forwards.
#include <math.h>
#include <string.h>

#include <vector>

#include "hx_internal.h"

namespace hx {

struct AdjBuffers {
    double2 *ckpt = nullptr;      // n_intervals x n
    double2 *states = nullptr;    // (substeps + 1) x n
    double2 *cur = nullptr;       // stepping buffer
    double2 *lam = nullptr;       // adjoint state
    double2 *tmp = nullptr;       // X v
    double *M = nullptr;          // m x m complex projections (by columns)
    double *gacc = nullptr;       // 2 x n_intervals
    double *tmid = nullptr;       // device time for the Lanczos runs
    double *dots = nullptr;       // partials + counter + result for <phi, psi>
    ~AdjBuffers()
    {
        cudaFree(ckpt); cudaFree(states); cudaFree(cur); cudaFree(lam); cudaFree(tmp);
        cudaFree(M); cudaFree(gacc); cudaFree(tmid); cudaFree(dots);
    }
};

// <x, y> = sum conj(x) y in FP64 (one block per 256 x 4 elements, partials summed on the host in order)
__global__ void cdot_kernel(const double2 *x, const double2 *y, int n, double *partials)
{
    __shared__ double sr[256], si[256];
    double ar = 0.0, ai = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double2 a = x[i], b = y[i];
        ar += a.x * b.x + a.y * b.y;
        ai += a.x * b.y - a.y * b.x;
    }
    sr[threadIdx.x] = ar;
    si[threadIdx.x] = ai;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            sr[threadIdx.x] += sr[threadIdx.x + o];
            si[threadIdx.x] += si[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = sr[0];
        partials[2 * blockIdx.x + 1] = si[0];
    }
}

static int cdot(const double2 *x, const double2 *y, int n, double *partials, cudaStream_t st, double &re, double &im)
{
    const int G = 64;
    cdot_kernel<<<G, 256, 0, st>>>(x, y, n, partials);
    std::vector<double> h(2 * G);
    cudaError_t e = cudaMemcpyAsync(h.data(), partials, 2 * G * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint inner product");
    re = im = 0.0;
    for (int b = 0; b < G; ++b) {
        re += h[2 * b];
        im += h[2 * b + 1];
    }
    return HX_OK;
}

}  // namespace hx

using namespace hx;

struct hx_indexset : IndexSetObj {};
struct hx_problem : Problem {};

#define ADJ_CUDA(call, what)                                   \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) { rc = cuda_fail(e_, what); goto done; } \
    } while (0)
#define ADJ_RC(call)                                           \
    do {                                                       \
        rc = (call);                                           \
        if (rc) goto done;                                     \
    } while (0)

extern "C" HX_API int hx_adjoint_grad(const hx_indexset *s, const hx_config *cfg, const hx_potential *fixed,
                                      const hx_control *ctl, const void *c0, const void *phi, double *grad_out,
                                      double *J_out)
{
    if (!s || !fixed || !ctl || !c0 || !phi || !J_out || !ctl->u) {
        set_error("hx_adjoint_grad: NULL argument");
        return HX_EINVAL;
    }
    if (ctl->n_intervals < 1 || ctl->substeps < 1 || !(ctl->t1 > ctl->t0) || ctl->axis < 0 || ctl->axis >= s->h.N) {
        set_error("hx_adjoint_grad: need n_intervals >= 1, substeps >= 1, t1 > t0 and a valid axis");
        return HX_EINVAL;
    }
    const int n = (int)s->h.size;
    const int NI = ctl->n_intervals, S = ctl->substeps;
    const double dt = (ctl->t1 - ctl->t0) / ((double)NI * S);
    hx_config c = {HX_C128, HX_ORDER_SYM, 7, nullptr, HX_SCHEME_EXPMPR, 0.0, 0.0};
    if (cfg) c = *cfg;
    if (c.scheme != HX_SCHEME_EXPMPR) {
        set_error("hx_adjoint_grad: the gradient is that of the exponential midpoint rule (scheme HX_SCHEME_EXPMPR)");
        return HX_EUNSUPPORTED;
    }
    if (!(c.scale == 0.0 || c.scale == 1.0)) {
        set_error("hx_adjoint_grad: the unscaled basis only (scale 0 or 1)");
        return HX_EUNSUPPORTED;
    }
    c.tol = 0.0;                            // fixed Lanczos exponentials (their count sets the sub-steps)
    c.dtype = HX_C128;                      // the gradient is an FP64 computation
    cudaStream_t st = (cudaStream_t)c.stream;
    hx_problem *Pf = nullptr, *Px = nullptr;
    AdjBuffers b;
    LanczosWS Lp, Ll;
    memset(&Lp, 0, sizeof(Lp));
    memset(&Ll, 0, sizeof(Ll));
    int rc = HX_OK;
    double a_re = 0.0, a_im = 0.0;
    const size_t vb = (size_t)n * sizeof(double2);
    // the full potential: the fixed terms plus u(t) x_axis
    std::vector<hx_term> terms(fixed->terms, fixed->terms + fixed->n_terms);
    double xcoef[2];
    hx_cheb_monomial(1, fixed->L, xcoef);
    hx_term ct;
    memset(&ct, 0, sizeof(ct));
    ct.n_axes = 1;
    ct.axes[0] = ctl->axis;
    ct.deg[0] = 1;
    ct.coef = xcoef;
    ct.mod_kind = HX_MOD_PWCONST;
    ct.amp = 1.0;
    ct.pw_values = ctl->u;
    ct.pw_n = NI;
    ct.pw_t0 = ctl->t0;
    ct.pw_t1 = ctl->t1;
    terms.push_back(ct);
    hx_potential full = {fixed->L, (int)terms.size(), terms.data()};
    hx_term xt;
    memset(&xt, 0, sizeof(xt));
    xt.n_axes = 1;
    xt.axes[0] = ctl->axis;
    xt.deg[0] = 1;
    xt.coef = xcoef;
    xt.mod_kind = HX_MOD_CONST;
    xt.amp = 1.0;
    hx_potential xpot = {fixed->L, 1, &xt};
    hx_config cx = c;
    cx.m = 1;

    ADJ_RC(hx_problem_create(s, &c, &Pf));
    ADJ_RC(hx_potential_set(Pf, &full, ctl->t0));
    ADJ_RC(hx_problem_create(s, &cx, &Px));
    ADJ_RC(hx_potential_set(Px, &xpot, ctl->t0));
    Px->skip_diag = true;
    ADJ_CUDA(cudaMalloc((void **)&b.cur, vb), "cudaMalloc(adjoint)");
    ADJ_CUDA(cudaMalloc((void **)&b.dots, 4096 * sizeof(double)), "cudaMalloc(adjoint)");
    ADJ_CUDA(cudaMalloc((void **)&b.ckpt, vb * NI), "cudaMalloc(adjoint checkpoints)");

    // forward pass, keeping the state at the start of every interval
    ADJ_CUDA(cudaMemcpyAsync(b.cur, c0, vb, cudaMemcpyDeviceToDevice, st), "adjoint copy");
    ADJ_RC(hx_set_time(Pf, ctl->t0));
    for (int q = 0; q < NI; ++q) {
        ADJ_CUDA(cudaMemcpyAsync(b.ckpt + (size_t)q * n, b.cur, vb, cudaMemcpyDeviceToDevice, st), "checkpoint");
        ADJ_RC(hx_step(Pf, b.cur, dt, S));
    }
    ADJ_RC(cdot((const double2 *)phi, b.cur, n, b.dots, st, a_re, a_im));
    *J_out = a_re * a_re + a_im * a_im;
    if (!grad_out) goto done;

    // backward pass
    {
        const int m = c.m;
        ADJ_CUDA(cudaMalloc((void **)&b.states, vb * (S + 1)), "cudaMalloc(adjoint)");
        ADJ_CUDA(cudaMalloc((void **)&b.lam, vb), "cudaMalloc(adjoint)");
        ADJ_CUDA(cudaMalloc((void **)&b.tmp, vb), "cudaMalloc(adjoint)");
        ADJ_CUDA(cudaMalloc((void **)&b.M, (size_t)2 * m * m * sizeof(double)), "cudaMalloc(adjoint)");
        ADJ_CUDA(cudaMalloc((void **)&b.gacc, (size_t)2 * NI * sizeof(double)), "cudaMalloc(adjoint)");
        ADJ_CUDA(cudaMalloc((void **)&b.tmid, sizeof(double)), "cudaMalloc(adjoint)");
        ADJ_CUDA(cudaMemsetAsync(b.gacc, 0, (size_t)2 * NI * sizeof(double), st), "adjoint clear");
        ADJ_RC(lanczos_alloc(Pf, m, &Lp));
        ADJ_RC(lanczos_alloc(Pf, m, &Ll));
        ADJ_CUDA(cudaMemcpyAsync(b.lam, phi, vb, cudaMemcpyDeviceToDevice, st), "adjoint copy");
        for (int q = NI - 1; q >= 0; --q) {
            // states inside interval q, recomputed from its checkpoint
            const double tq = ctl->t0 + (double)q * S * dt;
            ADJ_CUDA(cudaMemcpyAsync(b.states, b.ckpt + (size_t)q * n, vb, cudaMemcpyDeviceToDevice, st), "recompute");
            ADJ_CUDA(cudaMemcpyAsync(b.cur, b.states, vb, cudaMemcpyDeviceToDevice, st), "recompute");
            ADJ_RC(hx_set_time(Pf, tq));
            for (int i = 1; i <= S; ++i) {
                ADJ_RC(hx_step(Pf, b.cur, dt, 1));
                ADJ_CUDA(cudaMemcpyAsync(b.states + (size_t)i * n, b.cur, vb, cudaMemcpyDeviceToDevice, st), "recompute");
            }
            for (int i = S; i >= 1; --i) {
                const double tm = tq + (i - 0.5) * dt;     // midpoint of sub-step i of interval q
                ADJ_CUDA(cudaMemcpyAsync(b.tmid, &tm, sizeof(double), cudaMemcpyHostToDevice, st), "adjoint time");
                // Lanczos bases of psi_{n-1} and lambda_n for A at the midpoint
                ADJ_RC(lanczos_enqueue(Pf, &Lp, b.states + (size_t)(i - 1) * n, b.tmid, 0.0, st));
                ADJ_RC(lanczos_exp(Pf, &Lp, dt, nullptr, st));
                ADJ_RC(lanczos_enqueue(Pf, &Ll, b.lam, b.tmid, 0.0, st));
                // M[:, r] = V_lambda^H X v^psi_r
                for (int r = 0; r < m; ++r) {
                    ADJ_RC(lanczos_apply_basis(Px, &Lp, r, b.tmp, b.tmid, st));
                    ADJ_RC(lanczos_project(Pf, &Ll, b.tmp, b.M + (size_t)2 * m * r, st));
                }
                ADJ_RC(lanczos_exp(Pf, &Ll, -dt, b.lam, st));   // lambda_{n-1} = exp(+i dt A) lambda_n
                ADJ_RC(adjoint_term(&Lp, &Ll, b.M, dt, b.gacc + 2 * q, st));
            }
        }
        std::vector<double> g(2 * NI);
        ADJ_CUDA(cudaMemcpyAsync(g.data(), b.gacc, g.size() * sizeof(double), cudaMemcpyDeviceToHost, st), "adjoint read");
        ADJ_CUDA(cudaStreamSynchronize(st), "adjoint sync");
        for (int q = 0; q < NI; ++q)   // 2 Re(conj(a) g_q)
            grad_out[q] = 2.0 * (a_re * g[2 * q] + a_im * g[2 * q + 1]);
    }
done:
    if (Lp.V) lanczos_free(&Lp);
    if (Ll.V) lanczos_free(&Ll);
    if (st) cudaStreamSynchronize(st); else cudaDeviceSynchronize();
    hx_problem_destroy(Px);
    hx_problem_destroy(Pf);
    return rc;
}
