"""Python binding of libhx (include/hx.h): argument marshalling only.

Every function has the name of the C entry point it calls.  Device vectors are torch CUDA
tensors (complex128 or complex64, contiguous, canonical order); host vectors are numpy
arrays.  All arithmetic happens in libhx.so; importing this module raises if the library
has not been built, and a failing call raises HxError with the library's message.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhx.so")

HX_C128, HX_C64 = 0, 1
HX_ORDER_SYM, HX_ORDER_EQ, HX_ORDER_ALG = 0, 1, 2
HX_SCHEME_EXPMPR, HX_SCHEME_MAGNUS4 = 0, 1
HX_SCHED_MEMBERS, HX_SCHED_BATCHED, HX_SCHED_HYBRID, HX_SCHED_SERIAL = 0, 1, 2, 3
HX_MOD_CONST, HX_MOD_COS, HX_MOD_SIN2, HX_MOD_PWCONST = 0, 1, 2, 3
HX_EINVAL, HX_ENOMEM, HX_ECUDA, HX_ENONFINITE, HX_EBREAKDOWN, HX_ETIMEOUT, HX_EUNSUPPORTED = -1, -2, -3, -4, -5, -6, -7
ORDERS = {"sym": HX_ORDER_SYM, "eq": HX_ORDER_EQ, "alg": HX_ORDER_ALG}
MODS = {"const": HX_MOD_CONST, "cos": HX_MOD_COS, "sin2": HX_MOD_SIN2, "pwconst": HX_MOD_PWCONST}


class HxError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"hx status {status}: {msg}")
        self.status = status


class hx_term(ctypes.Structure):
    _fields_ = [("n_axes", ctypes.c_int), ("axes", ctypes.c_int * 2), ("deg", ctypes.c_int * 2),
                ("coef", ctypes.POINTER(ctypes.c_double)), ("mod_kind", ctypes.c_int),
                ("amp", ctypes.c_double), ("omega", ctypes.c_double), ("phase", ctypes.c_double),
                ("pw_values", ctypes.POINTER(ctypes.c_double)), ("pw_n", ctypes.c_int),
                ("pw_t0", ctypes.c_double), ("pw_t1", ctypes.c_double)]


class hx_potential(ctypes.Structure):
    _fields_ = [("L", ctypes.c_double), ("n_terms", ctypes.c_int), ("terms", ctypes.POINTER(hx_term))]


class hx_control(ctypes.Structure):
    _fields_ = [("axis", ctypes.c_int), ("n_intervals", ctypes.c_int), ("substeps", ctypes.c_int),
                ("t0", ctypes.c_double), ("t1", ctypes.c_double), ("u", ctypes.POINTER(ctypes.c_double))]


class hx_config(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int), ("order", ctypes.c_int), ("m", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("scheme", ctypes.c_int), ("tol", ctypes.c_double), ("scale", ctypes.c_double)]


class BatchStats(ctypes.Structure):
    """hx_batch_stats."""
    _fields_ = [("schedule", ctypes.c_int), ("tile", ctypes.c_int), ("launches", ctypes.c_int),
                ("ntiles", ctypes.c_int), ("tiles", ctypes.c_int * 8), ("tile_ms", ctypes.c_float * 8),
                ("step_ms", ctypes.c_float * 4)]


# const hx_potential *(*)(double t, void *user)
POTENTIAL_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p)


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_1403_3511_gb300.build.build() "
                          "(there is no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    P, i64, i32p = ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32)
    dp = ctypes.POINTER(ctypes.c_double)
    sig = {
        "hx_indexset_create": (ctypes.c_int, [ctypes.c_int, i64, ctypes.POINTER(P)]),
        "hx_indexset_create_list": (ctypes.c_int, [ctypes.c_int, i64, i32p, ctypes.POINTER(P)]),
        "hx_indexset_size": (i64, [P]),
        "hx_indexset_unrank": (ctypes.c_int, [P, i64, i32p]),
        "hx_indexset_rank": (i64, [P, i32p]),
        "hx_indexset_export": (ctypes.c_int, [P, i32p]),
        "hx_indexset_destroy": (None, [P]),
        "hx_problem_create": (ctypes.c_int, [P, ctypes.POINTER(hx_config), ctypes.POINTER(P)]),
        "hx_problem_destroy": (None, [P]),
        "hx_potential_set": (ctypes.c_int, [P, ctypes.POINTER(hx_potential), ctypes.c_double]),
        "hx_get_time": (ctypes.c_int, [P, dp]),
        "hx_set_time": (ctypes.c_int, [P, ctypes.c_double]),
        "hx_apply": (ctypes.c_int, [P, P, P]),
        "hx_apply_host": (ctypes.c_int, [P, P, P]),
        "hx_apply_project": (ctypes.c_int, [P, P, P, P, ctypes.c_size_t, ctypes.c_int, P]),
        "hx_step": (ctypes.c_int, [P, P, ctypes.c_double, ctypes.c_int]),
        "hx_step_host": (ctypes.c_int, [P, P, ctypes.c_double, ctypes.c_int]),
        "hx_step_reinterp": (ctypes.c_int, [P, P, ctypes.c_double, ctypes.c_int, POTENTIAL_FN, P]),
        "hx_step_info": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int), dp, dp, dp]),
        "hx_step_substeps": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64), dp]),
        "hx_step_launches": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
        "hx_apply_specialised": (ctypes.c_int, [P]),
        "hx_norm": (ctypes.c_int, [P, P, dp]),
        "hx_energy": (ctypes.c_int, [P, P, dp]),
        "hx_apply_rayleigh": (ctypes.c_int, [P, P, P, P]),
        "hx_batch_create": (ctypes.c_int, [ctypes.POINTER(P), ctypes.c_int, ctypes.POINTER(P)]),
        "hx_batch_step": (ctypes.c_int, [P, ctypes.POINTER(P), ctypes.c_double, ctypes.c_int]),
        "hx_batch_destroy": (None, [P]),
        "hx_batch_set_budget": (ctypes.c_int, [P, ctypes.c_double]),
        "hx_batch_info": (ctypes.c_int, [P, ctypes.POINTER(BatchStats)]),
        "hx_adjoint_grad": (ctypes.c_int, [P, ctypes.POINTER(hx_config), ctypes.POINTER(hx_potential),
                                           ctypes.POINTER(hx_control), P, P, dp, dp]),
        "hx_norm_noalloc": (ctypes.c_int, [P, P, dp]),
        "hx_cheb_nodes": (ctypes.c_int, [ctypes.c_int, dp]),
        "hx_cheb_coeffs": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, dp, dp]),
        "hx_cheb_monomial": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, dp]),
        "hx_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


lib = _load()


def hx_last_error() -> str:
    return lib.hx_last_error().decode()


def _check(status: int, allow=()):
    if status != 0 and status not in allow:
        raise HxError(status, hx_last_error())
    return status


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _tptr(t) -> int:
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


# element type and |K| of every problem handle this module created, so that a device vector of the
# wrong type or length is refused here instead of being read past its end by the library
_PROBLEMS = {}


def _handle(p) -> int:
    return p.value if isinstance(p, ctypes.c_void_p) else int(p)


def _vec(p, t, state: bool = False) -> int:
    """Device pointer of t after checking it against problem p: complex128 for a time-step state
    (state=True), else the problem dtype; at least |K| elements."""
    ptr = _tptr(t)
    info = _PROBLEMS.get(_handle(p))
    if info is not None:
        dtype, size = info
        want = "torch.complex128" if (state or dtype == HX_C128) else "torch.complex64"
        if str(t.dtype) != want:
            raise ValueError(f"expected a {want} tensor for this problem, got {t.dtype}")
        if t.numel() < size:
            raise ValueError(f"expected at least |K| = {size} elements, got {t.numel()}")
    return ptr


# ---- index set ---------------------------------------------------------------------------

def hx_indexset_create(N: int, B: int):
    h = ctypes.c_void_p()
    _check(lib.hx_indexset_create(N, B, ctypes.byref(h)))
    return h


def hx_indexset_create_list(ks) -> ctypes.c_void_p:
    """A general downward-closed set from an array of multi-indices, shape (count, N), any order."""
    kk = np.ascontiguousarray(ks, dtype=np.int32)
    if kk.ndim != 2:
        raise ValueError("expected an array of shape (count, N)")
    h = ctypes.c_void_p()
    _check(lib.hx_indexset_create_list(kk.shape[1], kk.shape[0], kk.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                       ctypes.byref(h)))
    return h


def hx_indexset_size(s) -> int:
    return int(lib.hx_indexset_size(s))


def hx_indexset_unrank(s, rank: int, N: int) -> np.ndarray:
    k = np.zeros(N, dtype=np.int32)
    _check(lib.hx_indexset_unrank(s, rank, k.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
    return k


def hx_indexset_rank(s, k) -> int:
    kk = np.ascontiguousarray(k, dtype=np.int32)
    return int(lib.hx_indexset_rank(s, kk.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))


def hx_indexset_export(s, N: int) -> np.ndarray:
    n = hx_indexset_size(s)
    k = np.zeros((n, N), dtype=np.int32)
    _check(lib.hx_indexset_export(s, k.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
    return k


def hx_indexset_destroy(s):
    lib.hx_indexset_destroy(s)


# ---- problem -----------------------------------------------------------------------------

def hx_problem_create(s, dtype: int = HX_C128, order: int = HX_ORDER_SYM, m: int = 7, stream: int = 0,
                      scheme: int = HX_SCHEME_EXPMPR, tol: float = 0.0, scale: float = 0.0):
    cfg = hx_config(dtype, order, m, ctypes.c_void_p(stream), scheme, tol, scale)
    h = ctypes.c_void_p()
    _check(lib.hx_problem_create(s, ctypes.byref(cfg), ctypes.byref(h)))
    _PROBLEMS[h.value] = (dtype, hx_indexset_size(s))
    return h


def hx_problem_destroy(p):
    _PROBLEMS.pop(_handle(p) if p is not None else None, None)
    lib.hx_problem_destroy(p)


def _potential(L: float, terms: list):
    keep = []
    arr = (hx_term * max(len(terms), 1))()
    for i, t_ in enumerate(terms):
        coef = np.ascontiguousarray(t_["coef"], dtype=np.float64)
        keep.append(coef)
        axes = list(t_["axes"])
        tm = arr[i]
        tm.n_axes = len(axes)
        for j, a in enumerate(axes[:2]):     # more than two axes: the library reports it
            tm.axes[j] = a
            tm.deg[j] = coef.shape[j] - 1
        tm.coef = _dptr(coef)
        tm.mod_kind = t_.get("mod", HX_MOD_CONST)
        tm.amp = t_.get("amp", 1.0)
        tm.omega = t_.get("omega", 0.0)
        tm.phase = t_.get("phase", 0.0)
        if tm.mod_kind == HX_MOD_PWCONST:
            pw = np.ascontiguousarray(t_["pw_values"], dtype=np.float64)
            keep.append(pw)
            tm.pw_values = _dptr(pw)
            tm.pw_n = len(pw)
            tm.pw_t0 = t_["pw_t0"]
            tm.pw_t1 = t_["pw_t1"]
    return hx_potential(L, len(terms), arr), (keep, arr)


def hx_potential_set(p, L: float, terms: list, t: float = 0.0):
    """terms: list of dicts {axes: [a] or [a, b], coef: ndarray (deg+1,) or (deg_a+1, deg_b+1),
    mod: hx_mod_kind, amp, omega, phase, pw_values, pw_t0, pw_t1}."""
    pot, _keep = _potential(L, terms)
    _check(lib.hx_potential_set(p, ctypes.byref(pot), t))


def hx_get_time(p) -> float:
    t = ctypes.c_double()
    _check(lib.hx_get_time(p, ctypes.byref(t)))
    return t.value


def hx_set_time(p, t: float):
    _check(lib.hx_set_time(p, t))


def hx_apply(p, c_in, c_out):
    _check(lib.hx_apply(p, ctypes.c_void_p(_vec(p, c_in)), ctypes.c_void_p(_vec(p, c_out))))


def hx_apply_project(p, c, y, basis, k: int, h):
    """y = A(t) c and h_i = <basis[i], y> for i <= k.  basis: CUDA tensor of at least k + 1 rows of
    |K| elements (row stride = ld), h: CUDA float64 tensor of 2 (k + 1) values (re, im)."""
    if not (basis.is_cuda and basis.dim() == 2 and basis.stride(1) == 1):
        raise ValueError("basis must be a CUDA tensor of rows with unit element stride")
    if not (h.is_cuda and str(h.dtype) == "torch.float64" and h.is_contiguous()):
        raise ValueError("h must be a contiguous CUDA float64 tensor")
    _check(lib.hx_apply_project(p, ctypes.c_void_p(_vec(p, c)), ctypes.c_void_p(_vec(p, y)),
                                ctypes.c_void_p(basis.data_ptr()), basis.stride(0), k, ctypes.c_void_p(h.data_ptr())))


def hx_apply_rayleigh(p, c, y, r):
    """y = A(t) c and r = <c, y> (r: CUDA float64 tensor of 2 values, re and im); see include/hx.h."""
    if not (r.is_cuda and str(r.dtype) == "torch.float64" and r.is_contiguous() and r.numel() >= 2):
        raise ValueError("r must be a contiguous CUDA float64 tensor of at least 2 values")
    _check(lib.hx_apply_rayleigh(p, ctypes.c_void_p(_vec(p, c)), ctypes.c_void_p(_vec(p, y)),
                                 ctypes.c_void_p(r.data_ptr())))


def _host_vec(a: np.ndarray, dtypes) -> ctypes.c_void_p:
    if not (isinstance(a, np.ndarray) and a.dtype in dtypes and a.flags.c_contiguous):
        raise ValueError(f"expected a contiguous numpy array of {' or '.join(str(np.dtype(d)) for d in dtypes)}")
    return a.ctypes.data_as(ctypes.c_void_p)


def hx_apply_host(p, c_in: np.ndarray, c_out: np.ndarray):
    """c_in, c_out: |K| elements of the problem dtype (complex128 or complex64)."""
    if c_in.dtype != c_out.dtype or not c_out.flags.writeable:
        raise ValueError("c_in and c_out must have the same dtype and c_out must be writeable")
    _check(lib.hx_apply_host(p, _host_vec(c_in, (np.complex128, np.complex64)),
                             _host_vec(c_out, (np.complex128, np.complex64))))


def hx_step(p, c, dt: float, nsteps: int) -> int:
    return _check(lib.hx_step(p, ctypes.c_void_p(_vec(p, c, state=True)), dt, nsteps), allow=(HX_EBREAKDOWN,))


def hx_step_host(p, c: np.ndarray, dt: float, nsteps: int) -> int:
    """c: the complex128 state (|K| elements), stepped in place."""
    if not c.flags.writeable:
        raise ValueError("the state must be writeable")
    return _check(lib.hx_step_host(p, _host_vec(c, (np.complex128,)), dt, nsteps), allow=(HX_EBREAKDOWN,))


def hx_step_reinterp(p, c, dt: float, nsteps: int, fn) -> int:
    """nsteps steps with the potential re-interpolated for every step: fn(t) -> (L, terms), terms
    as for hx_potential_set, is called at the times the problem's scheme evaluates A (t + dt/2, or
    the two Gauss-Legendre points of the 2-stage Magnus method)."""
    held = []

    def cb(t, _user):
        L, terms = fn(t)
        pot, keep = _potential(L, terms)
        held.append((pot, keep))
        del held[:-2]                       # the library holds at most the last two potentials
        return ctypes.addressof(pot)

    cfn = POTENTIAL_FN(cb)
    return _check(lib.hx_step_reinterp(p, ctypes.c_void_p(_vec(p, c, state=True)), dt, nsteps, cfn, None),
                  allow=(HX_EBREAKDOWN,))


def hx_step_info(p, m: int = 32) -> dict:
    mu = ctypes.c_int()
    a = np.zeros(m)
    b = np.zeros(m)
    nr = ctypes.c_double()
    st = _check(lib.hx_step_info(p, ctypes.byref(mu), _dptr(a), _dptr(b), ctypes.byref(nr)), allow=(HX_EBREAKDOWN,))
    return {"m_used": mu.value, "alpha": a[: mu.value], "beta": b[: max(mu.value - 1, 0)], "norm": nr.value,
            "breakdown": st == HX_EBREAKDOWN}


def hx_step_substeps(p) -> dict:
    """Sub-steps of the last hx_step (last step, total) and the largest a-posteriori estimate."""
    last, total, err = ctypes.c_int(), ctypes.c_int64(), ctypes.c_double()
    _check(lib.hx_step_substeps(p, ctypes.byref(last), ctypes.byref(total), ctypes.byref(err)))
    return {"last": last.value, "total": total.value, "err_max": err.value}


def hx_apply_specialised(p) -> int:
    """1 when the product runs the kernel compiled for this potential's operator structure, 0 when it
    runs the generic kernel (hx_last_error() says why)."""
    r = lib.hx_apply_specialised(p)
    if r < 0:
        raise HxError(r, hx_last_error())
    return r


def hx_step_launches(p) -> tuple:
    """(kernels per product, kernels per time step)."""
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(lib.hx_step_launches(p, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def hx_batch_create(problems: list):
    arr = (ctypes.c_void_p * len(problems))(*[p.value if isinstance(p, ctypes.c_void_p) else p for p in problems])
    h = ctypes.c_void_p()
    _check(lib.hx_batch_create(arr, len(problems), ctypes.byref(h)))
    return h


def hx_batch_step(b, states: list, dt: float, nsteps: int):
    arr = (ctypes.c_void_p * len(states))(*[_tptr(c) for c in states])
    _check(lib.hx_batch_step(b, arr, dt, nsteps))


def hx_batch_destroy(b):
    lib.hx_batch_destroy(b)


def hx_batch_set_budget(b, seconds: float):
    _check(lib.hx_batch_set_budget(b, float(seconds)))


def hx_batch_info(b) -> dict:
    """The batch's schedule state after its last step: {'schedule': HX_SCHED_* or -1, 'batched':
    a batched schedule in use, 'tile', 'launches' (kernels per step), 'candidates': [(tile, ms)],
    'step_ms': {schedule: ms of its timed step}}."""
    st = BatchStats()
    _check(lib.hx_batch_info(b, ctypes.byref(st)))
    return {"schedule": st.schedule, "batched": st.schedule > HX_SCHED_MEMBERS,
            "tile": st.tile, "launches": st.launches,
            "candidates": [(st.tiles[i], st.tile_ms[i]) for i in range(st.ntiles)],
            "step_ms": {i: st.step_ms[i] for i in range(4) if st.step_ms[i] >= 0}}


def hx_norm(p, c) -> float:
    out = ctypes.c_double()
    _check(lib.hx_norm(p, ctypes.c_void_p(_vec(p, c)), ctypes.byref(out)))
    return out.value


def hx_energy(p, c) -> float:
    """<c, A(t) c> (see include/hx.h)."""
    out = ctypes.c_double()
    _check(lib.hx_energy(p, ctypes.c_void_p(_vec(p, c)), ctypes.byref(out)))
    return out.value


def hx_norm_noalloc(p, c) -> float:
    """hx_norm without any device allocation (fixed scratch inside the library); see include/hx.h."""
    out = ctypes.c_double()
    _check(lib.hx_norm_noalloc(p, ctypes.c_void_p(_vec(p, c)), ctypes.byref(out)))
    return out.value


def hx_adjoint_grad(s, L: float, fixed_terms: list, axis: int, u, t0: float, t1: float, substeps: int, c0, phi,
                    m: int = 20, order: int = HX_ORDER_SYM, stream: int = 0, gradient: bool = True):
    """(J, dJ/du) for J = |<phi, psi(t1)>|^2 with the control u(t) x_axis (see include/hx.h).
    c0, phi: complex128 CUDA tensors; u: host values, one per interval."""
    pot, _keep = _potential(L, fixed_terms)
    uu = np.ascontiguousarray(u, dtype=np.float64)
    ctl = hx_control(axis, len(uu), substeps, t0, t1, _dptr(uu))
    cfg = hx_config(HX_C128, order, m, ctypes.c_void_p(stream), HX_SCHEME_EXPMPR, 0.0, 0.0)
    grad = np.zeros(len(uu))
    J = ctypes.c_double()
    _check(lib.hx_adjoint_grad(s, ctypes.byref(cfg), ctypes.byref(pot), ctypes.byref(ctl),
                               ctypes.c_void_p(_tptr(c0)), ctypes.c_void_p(_tptr(phi)),
                               _dptr(grad) if gradient else None, ctypes.byref(J)))
    return J.value, (grad if gradient else None)


def control_objective(s, L: float, fixed_terms: list, axis: int, t0: float, t1: float, substeps: int, c0, phi,
                      m: int = 20):
    """A torch.autograd.Function J(u): forward and gradient both from hx_adjoint_grad."""
    import torch

    class _ControlObjective(torch.autograd.Function):
        @staticmethod
        def forward(ctx, u):
            J, g = hx_adjoint_grad(s, L, fixed_terms, axis, u.detach().cpu().numpy(), t0, t1, substeps, c0, phi, m)
            ctx.save_for_backward(torch.as_tensor(g, dtype=u.dtype, device=u.device))
            return torch.tensor(J, dtype=u.dtype, device=u.device)

        @staticmethod
        def backward(ctx, gout):
            (g,) = ctx.saved_tensors
            return gout * g

    return _ControlObjective.apply


# ---- Chebyshev helpers -------------------------------------------------------------------

def hx_cheb_nodes(R: int) -> np.ndarray:
    u = np.zeros(R + 1)
    _check(lib.hx_cheb_nodes(R, _dptr(u)))
    return u


def hx_cheb_coeffs(R: int, values: np.ndarray) -> np.ndarray:
    v = np.ascontiguousarray(values, dtype=np.float64)
    out = np.zeros_like(v)
    _check(lib.hx_cheb_coeffs(R, v.ndim, _dptr(v), _dptr(out)))
    return out


def hx_cheb_monomial(p: int, L: float) -> np.ndarray:
    out = np.zeros(p + 1)
    _check(lib.hx_cheb_monomial(p, L, _dptr(out)))
    return out


def terms_from_spec(spec: dict, t: float = 0.0) -> list:
    """hx_term dictionaries for a workload's potential (see paper_1403_3511_gb300.inputs): monomials
    through hx_cheb_monomial, smooth functions through their values at hx_cheb_nodes and
    hx_cheb_coeffs (a function that itself depends on time, "omega" != 0, at time t).  Evaluating
    the user's function at the nodes is the only arithmetic here."""
    L = spec["L"]
    tt = t
    out = []
    for comp in spec["potential"]:
        mod = comp.get("mod", {"kind": "const"})
        t = {"mod": MODS[mod["kind"]], "amp": comp["coef"], "omega": mod.get("omega", 0.0),
             "phase": mod.get("phase", 0.0)}
        if mod["kind"] == "pwconst":
            t.update(pw_values=mod["values"], pw_t0=mod["t0"], pw_t1=mod["t1"])
        if "powers" in comp and not comp["powers"]:     # a constant: degree 0 on axis 0 (the diagonal)
            t["axes"] = [0]
            t["coef"] = np.ones(1)
        elif "powers" in comp:
            axes = sorted(comp["powers"])
            if len(axes) > 2:
                raise ValueError("terms on more than two axes are not supported")
            cs = [hx_cheb_monomial(comp["powers"][a], L) for a in axes]
            t["axes"] = axes
            t["coef"] = cs[0] if len(cs) == 1 else np.outer(cs[0], cs[1])
        elif comp["func"] == "cos_diff":
            R = comp["R"]
            u = hx_cheb_nodes(R)
            t["axes"] = list(comp["axes"])
            t["coef"] = hx_cheb_coeffs(R, np.cos(L * u[:, None] - L * u[None, :] + comp.get("omega", 0.0) * tt))
        elif comp["func"] == "cos_scaled":
            R = comp["R"]
            u = hx_cheb_nodes(R)
            t["axes"] = list(comp["axes"])
            t["coef"] = hx_cheb_coeffs(R, np.cos(comp["scale"] * L * u + comp.get("omega", 0.0) * tt))
        else:
            raise KeyError(comp["func"])
        out.append(t)
    return out


class Problem:
    """Convenience owner of an index set and a problem (frees both)."""

    def __init__(self, N: int, B: int, dtype: int = HX_C128, order: str = "sym", m: int = 7, stream: int = 0,
                 indexset=None, scheme: int = HX_SCHEME_EXPMPR, tol: float = 0.0, scale: float = 0.0):
        self._own_set = indexset is None
        self.set = hx_indexset_create(N, B) if indexset is None else indexset
        self.N, self.B = N, B
        self.size = hx_indexset_size(self.set)
        self.dtype = dtype
        self.p = hx_problem_create(self.set, dtype, ORDERS[order] if isinstance(order, str) else order, m, stream,
                                   scheme, tol, scale)

    def set_potential(self, spec: dict, t: float = 0.0):
        hx_potential_set(self.p, spec["L"], terms_from_spec(spec, t), t)

    def step_reinterp(self, spec: dict, c, dt: float, nsteps: int) -> int:
        """hx_step_reinterp with the workload's potential interpolated at every time the scheme asks for."""
        return hx_step_reinterp(self.p, c, dt, nsteps, lambda t: (spec["L"], terms_from_spec(spec, t)))

    def close(self):
        if getattr(self, "p", None) is not None:
            hx_problem_destroy(self.p)
            self.p = None
        if getattr(self, "set", None) is not None and self._own_set:
            hx_indexset_destroy(self.set)
            self.set = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
