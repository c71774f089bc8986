"""ctypes binding of libga_gb300.so: the C ABI of include/ga.h and include/ga_ops.h.

Argument marshalling only. Arrays may be torch tensors (CUDA tensors are passed as device
pointers, CPU tensors as host pointers) or NumPy arrays (host pointers); they must be C-contiguous
and of the context's element type (float64 for GA_PREC_FP64, float32 for GA_PREC_MIXED). Every
compute call runs in the CUDA library; there is no Python or CPU fallback, and a missing library
raises GaError.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

GA_MODEL_ADVECTION, GA_MODEL_CONTINUITY, GA_MODEL_INCOMPRESSIBLE = 0, 1, 2
GA_PREC_FP64, GA_PREC_MIXED = 0, 1
GA_MEM_HOST, GA_MEM_DEVICE = 0, 1
GA_METHOD_GA_NGMRES, GA_METHOD_RPGD, GA_METHOD_GA_AA = 0, 1, 2
STATUS = {0: "GA_OK", 1: "GA_ERR_ARG", 2: "GA_ERR_CUDA", 3: "GA_ERR_NOMEM", 4: "GA_ERR_NAN",
          5: "GA_ERR_LINESEARCH", 6: "GA_ERR_NOT_CONVERGED", 7: "GA_ERR_TIMEOUT"}
MODELS = {"advection": GA_MODEL_ADVECTION, "continuity": GA_MODEL_CONTINUITY,
          "incompressible": GA_MODEL_INCOMPRESSIBLE}

_c_int, _c_double, _vp = ctypes.c_int, ctypes.c_double, ctypes.c_void_p


class ProblemDesc(ctypes.Structure):
    _fields_ = [("dim", _c_int), ("n", _c_int * 3), ("nt", _c_int), ("model", _c_int),
                ("reg_order", _c_int), ("alpha", _c_double), ("prec", _c_int), ("ckpt_every", _c_int)]


class SolverOpts(ctypes.Structure):
    _fields_ = [("window", _c_int), ("sigma", _c_int), ("tau", _c_int), ("max_iter", _c_int),
                ("rel_tol", _c_double), ("armijo_c", _c_double), ("max_backtracks", _c_int),
                ("variant", _c_int), ("method", _c_int), ("graphs", _c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("iters", _c_int), ("grad_evals", _c_int), ("obj_evals", _c_int), ("pde_solves", _c_int),
                ("ls_trials", _c_int), ("last_branch", _c_int), ("converged", _c_int),
                ("obj", _c_double), ("mismatch", _c_double), ("rel_grad_inf", _c_double),
                ("grad_inf0", _c_double), ("rho_mem", _c_double), ("last_rho", _c_double),
                ("t_grad_ms", _c_double), ("t_obj_ms", _c_double), ("t_total_ms", _c_double)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class GaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def library_path():
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "libga_gb300.so")


_LIB = None

_SIGS = {
    "ga_workspace_bytes": ([ctypes.POINTER(ProblemDesc), ctypes.POINTER(SolverOpts), ctypes.POINTER(ctypes.c_size_t)],
                           _c_int),
    "ga_setup": ([ctypes.POINTER(ProblemDesc), ctypes.POINTER(SolverOpts), _vp, _vp, _c_int, _vp,
                  ctypes.POINTER(_vp)], _c_int),
    "ga_objective": ([_vp, _vp, _c_int, ctypes.POINTER(_c_double)], _c_int),
    "ga_gradient": ([_vp, _vp, _vp, _c_int, ctypes.POINTER(_c_double)], _c_int),
    "ga_deformation": ([_vp, _vp, _vp, _vp, _c_int], _c_int),
    "ga_precond": ([_vp, _vp, _vp, _c_int], _c_int),
    "ga_step": ([_vp, _vp, _c_int, ctypes.POINTER(Stats)], _c_int),
    "ga_solve": ([_vp, _vp, _c_int, ctypes.POINTER(Stats)], _c_int),
    "ga_reset": ([_vp], _c_int),
    "ga_solve_batch": ([_c_int, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _c_int, ctypes.POINTER(Stats)], _c_int),
    "ga_get_stats": ([_vp, ctypes.POINTER(Stats)], _c_int),
    "ga_destroy": ([_vp], None),
    "ga_status_str": ([_c_int], ctypes.c_char_p),
    "ga_last_error": ([_vp], ctypes.c_char_p),
    "ga_op_departure": ([_vp, _vp, _vp, _vp], _c_int),
    "ga_op_forward": ([_vp, _vp, _vp], _c_int),
    "ga_op_adjoint": ([_vp, _vp, _vp, _vp], _c_int),
    "ga_op_body_force": ([_vp, _vp, _vp, _vp], _c_int),
    "ga_op_deriv": ([_vp, _vp, _c_int, _vp], _c_int),
    "ga_op_div": ([_vp, _vp, _vp], _c_int),
    "ga_op_get_tiles": ([_vp, ctypes.POINTER(_c_int)], _c_int),
    "ga_op_set_tiles": ([_vp, ctypes.POINTER(_c_int)], _c_int),
    "ga_op_get_sl_depth": ([_vp, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int)], _c_int),
    "ga_op_set_sl_depth": ([_vp, _c_int, _c_int], _c_int),
    "ga_op_fft_r2c": ([_vp, _vp, _vp], _c_int),
    "ga_op_fft_c2r": ([_vp, _vp, _vp], _c_int),
    "ga_op_apply_L": ([_vp, _vp, _vp], _c_int),
    "ga_op_leray": ([_vp, _vp, _vp], _c_int),
    "ga_op_dots": ([_vp, _vp, ctypes.POINTER(_vp), _c_int, ctypes.c_size_t, ctypes.POINTER(_c_double)], _c_int),
    "ga_op_lsq": ([_vp, _c_int, _c_double, ctypes.POINTER(_c_double), ctypes.POINTER(_c_double),
                   ctypes.POINTER(_c_double)], _c_int),
    "ga_transport": ([_vp, _vp, _vp, _c_int], _c_int),
    "ga_transport_vjp": ([_vp, _vp, _vp, _vp, _c_int], _c_int),
    "ga_transport_vjp_exact": ([_vp, _vp, _vp, _vp, _c_int], _c_int),
    "ga_gradient_dto": ([_vp, _vp, _vp, _c_int, ctypes.POINTER(_c_double)], _c_int),
    "ga_prof_start": ([_vp, _c_int], _c_int),
    "ga_prof_stop": ([_vp, ctypes.POINTER(_c_double), ctypes.POINTER(ctypes.c_longlong)], _c_int),
    "ga_kernel_launches": ([], ctypes.c_longlong),
    "ga_dots_noalloc": ([_c_int, _vp, ctypes.POINTER(_vp), _c_int, ctypes.c_size_t, _vp, _vp], _c_int),
}


def lib():
    """The loaded CUDA library (raises GaError if it has not been built)."""
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            raise GaError(2, f"CUDA library {path} is missing; build it with "
                             "`python -m paper_2510_08782_gb300.build`")
        L = ctypes.CDLL(path)
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _LIB = L
    return _LIB


def ga_status_str(status):
    return lib().ga_status_str(int(status)).decode()


def ga_last_error(ctx=None):
    return lib().ga_last_error(ctx).decode()


def _check(status, ctx=None, ok=(0,)):
    if status not in ok:
        raise GaError(status, ga_last_error(ctx))
    return status


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype):
    """(address, mem kind) of a C-contiguous array of element type dtype."""
    if _is_torch(x):
        import torch

        want = torch.float64 if dtype == np.float64 else torch.float32
        if x.dtype != want or not x.is_contiguous():
            raise GaError(1, f"tensor must be contiguous {want}, got {x.dtype}")
        return x.data_ptr(), (GA_MEM_DEVICE if x.is_cuda else GA_MEM_HOST)
    if isinstance(x, np.ndarray):
        if x.dtype != dtype or not x.flags["C_CONTIGUOUS"]:
            raise GaError(1, f"array must be C-contiguous {np.dtype(dtype).name}, got {x.dtype}")
        return x.ctypes.data, GA_MEM_HOST
    raise GaError(1, f"unsupported array type {type(x)}")


def _ptrs(dtype, *arrays):
    out = [_ptr(a, dtype) for a in arrays]
    kinds = {k for _, k in out}
    if len(kinds) != 1:
        raise GaError(1, "all arrays of one call must live in the same memory (host or device)")
    return [p for p, _ in out], kinds.pop()


# Grid of every live context created through this module (handle -> (dim, shape, nt, device index)).
# The C calls take plain pointers and read as many elements as the context's grid implies, so the
# wrappers check element counts and devices here: a short array would otherwise be read or written
# past its end.
_CTX_INFO = {}


def _numel(x):
    return int(x.numel()) if _is_torch(x) else int(np.asarray(x).size)


def _device_of(x):
    return x.device.index if (_is_torch(x) and x.is_cuda) else None


def _check_device(arrays, want=None):
    """All CUDA tensors of one call on one device, which must be the current device (and the
    context's device when `want` is given)."""
    devs = {_device_of(a) for a in arrays} - {None}
    if not devs:
        return
    if len(devs) != 1:
        raise GaError(1, f"all CUDA tensors of one call must be on one device, got {sorted(devs)}")
    import torch

    dev = devs.pop()
    if dev != torch.cuda.current_device():
        raise GaError(1, f"tensors are on cuda:{dev} but the current device is cuda:{torch.cuda.current_device()}")
    if want is not None and dev != want:
        raise GaError(1, f"tensors are on cuda:{dev} but the context lives on cuda:{want}")


def _sizes(ctx, **kinds):
    """Check each array against the context's grid. kinds: name=(array, kind) with kind one of
    'scalar' (prod n), 'vec' (dim prod n), 'states' ((n_t+1) prod n) or 'half' (2 x the half
    spectrum: interleaved re, im)."""
    info = _CTX_INFO.get(ctx)
    if info is None:
        return
    dim, shape, nt, dev = info
    n = int(np.prod(shape))
    half = int(np.prod(shape[:-1])) * (shape[-1] // 2 + 1) * 2
    want = {"scalar": n, "vec": dim * n, "states": (nt + 1) * n, "half": half}
    for name, (arr, kind) in kinds.items():
        got = _numel(arr)
        if got != want[kind]:
            raise GaError(1, f"{name}: expected {want[kind]} elements for grid {shape} ({kind}), got {got}")
    _check_device([a for a, _ in kinds.values()], dev)


def _current_stream():
    try:
        import torch

        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:  # torch absent: the legacy default stream
        pass
    return None


# ---- raw C calls with the C names ------------------------------------------------------------------

def ga_setup(desc, opts, m0, m1, stream=None):
    """Create a context; returns (handle, element dtype)."""
    dtype = np.float64 if desc.prec == GA_PREC_FP64 else np.float32
    (p0, p1), mem = _ptrs(dtype, m0, m1)
    shape = tuple(int(desc.n[i]) for i in range(desc.dim))
    n = int(np.prod(shape)) if desc.dim > 0 else 0
    if _numel(m0) != n or _numel(m1) != n:
        raise GaError(1, f"m0, m1: expected {n} elements for grid {shape}, got {_numel(m0)}, {_numel(m1)}")
    _check_device([m0, m1])
    h = _vp()
    st = lib().ga_setup(ctypes.byref(desc), ctypes.byref(opts), p0, p1, mem,
                        _vp(stream if stream is not None else _current_stream()), ctypes.byref(h))
    _check(st, None)
    dev = None
    try:
        import torch

        if torch.cuda.is_available():
            dev = torch.cuda.current_device()
    except Exception:
        pass
    _CTX_INFO[h.value] = (int(desc.dim), shape, int(desc.nt), dev)
    return h.value


def ga_workspace_bytes(desc, opts):
    """Device bytes ga_setup allocates for this descriptor and these options (host arithmetic)."""
    out = ctypes.c_size_t()
    _check(lib().ga_workspace_bytes(ctypes.byref(desc), ctypes.byref(opts), ctypes.byref(out)), None)
    return int(out.value)


def ga_destroy(ctx):
    _CTX_INFO.pop(ctx, None)
    lib().ga_destroy(ctx)


def ga_objective(ctx, dtype, v):
    _sizes(ctx, v=(v, 'vec'))
    (pv,), mem = _ptrs(dtype, v)
    out = _c_double()
    _check(lib().ga_objective(ctx, pv, mem, ctypes.byref(out)), ctx)
    return out.value


def ga_gradient(ctx, dtype, v, g):
    _sizes(ctx, v=(v, 'vec'), g=(g, 'vec'))
    (pv, pg), mem = _ptrs(dtype, v, g)
    out = _c_double()
    _check(lib().ga_gradient(ctx, pv, pg, mem, ctypes.byref(out)), ctx)
    return out.value


def ga_deformation(ctx, dtype, v, u, detj):
    _sizes(ctx, v=(v, 'vec'), u=(u, 'vec'), detj=(detj, 'scalar'))
    (pv, pu, pj), mem = _ptrs(dtype, v, u, detj)
    _check(lib().ga_deformation(ctx, pv, pu, pj, mem), ctx)


def ga_precond(ctx, dtype, g, s):
    _sizes(ctx, g=(g, 'vec'), s=(s, 'vec'))
    (pg, ps), mem = _ptrs(dtype, g, s)
    _check(lib().ga_precond(ctx, pg, ps, mem), ctx)


def ga_step(ctx, dtype, v):
    _sizes(ctx, v=(v, 'vec'))
    (pv,), mem = _ptrs(dtype, v)
    stt = Stats()
    st = lib().ga_step(ctx, pv, mem, ctypes.byref(stt))
    _check(st, ctx)
    return stt


def ga_get_stats(ctx):
    stt = Stats()
    _check(lib().ga_get_stats(ctx, ctypes.byref(stt)), ctx)
    return stt


def ga_solve(ctx, dtype, v):
    _sizes(ctx, v=(v, 'vec'))
    (pv,), mem = _ptrs(dtype, v)
    stt = Stats()
    st = lib().ga_solve(ctx, pv, mem, ctypes.byref(stt))
    _check(st, ctx, ok=(0, 6))
    return stt, st


def ga_solve_batch(ctxs, dtype, vs):
    if len(ctxs) != len(vs):
        raise GaError(1, f"{len(ctxs)} contexts but {len(vs)} velocity arrays")
    for c, v in zip(ctxs, vs):
        _sizes(c, v=(v, 'vec'))
    ptrs, mem = _ptrs(dtype, *vs)
    n = len(ctxs)
    carr = (_vp * n)(*ctxs)
    varr = (_vp * n)(*ptrs)
    stats = (Stats * n)()
    st = lib().ga_solve_batch(n, carr, varr, mem, stats)
    _check(st, None, ok=(0, 6))
    return list(stats), st


def ga_reset(ctx):
    _check(lib().ga_reset(ctx), ctx)


def ga_transport(ctx, dtype, v, m1_out):
    _sizes(ctx, v=(v, 'vec'), m1_out=(m1_out, 'scalar'))
    (pv, pm), mem = _ptrs(dtype, v, m1_out)
    _check(lib().ga_transport(ctx, pv, pm, mem), ctx)


def ga_transport_vjp(ctx, dtype, v, gamma, grad_v):
    _sizes(ctx, v=(v, 'vec'), gamma=(gamma, 'scalar'), grad_v=(grad_v, 'vec'))
    (pv, pgam, pg), mem = _ptrs(dtype, v, gamma, grad_v)
    _check(lib().ga_transport_vjp(ctx, pv, pgam, pg, mem), ctx)


def ga_transport_vjp_exact(ctx, dtype, v, gamma, grad_v):
    _sizes(ctx, v=(v, 'vec'), gamma=(gamma, 'scalar'), grad_v=(grad_v, 'vec'))
    (pv, pgam, pg), mem = _ptrs(dtype, v, gamma, grad_v)
    _check(lib().ga_transport_vjp_exact(ctx, pv, pgam, pg, mem), ctx)


def ga_gradient_dto(ctx, dtype, v, g):
    _sizes(ctx, v=(v, 'vec'), g=(g, 'vec'))
    (pv, pg), mem = _ptrs(dtype, v, g)
    out = _c_double()
    _check(lib().ga_gradient_dto(ctx, pv, pg, mem, ctypes.byref(out)), ctx)
    return out.value


def _dev(dtype, *arrays):
    ptrs, mem = _ptrs(dtype, *arrays)
    if mem != GA_MEM_DEVICE:
        raise GaError(1, "operator-level calls take CUDA tensors")
    return ptrs


def ga_op_departure(ctx, dtype, v, xm, xp):
    _sizes(ctx, v=(v, 'vec'), xm=(xm, 'vec'), xp=(xp, 'vec'))
    _check(lib().ga_op_departure(ctx, *_dev(dtype, v, xm, xp)), ctx)


def ga_op_forward(ctx, dtype, v, states):
    _sizes(ctx, v=(v, 'vec'), states=(states, 'states'))
    _check(lib().ga_op_forward(ctx, *_dev(dtype, v, states)), ctx)


def ga_op_adjoint(ctx, dtype, v, lam1, lams):
    _sizes(ctx, v=(v, 'vec'), lam1=(lam1, 'scalar'), lams=(lams, 'states'))
    _check(lib().ga_op_adjoint(ctx, *_dev(dtype, v, lam1, lams)), ctx)


def ga_op_body_force(ctx, dtype, v, lam1, b):
    _sizes(ctx, v=(v, 'vec'), lam1=(lam1, 'scalar'), b=(b, 'vec'))
    _check(lib().ga_op_body_force(ctx, *_dev(dtype, v, lam1, b)), ctx)


def ga_op_deriv(ctx, dtype, f, axis, df):
    _sizes(ctx, f=(f, 'scalar'), df=(df, 'scalar'))
    pf, pd = _dev(dtype, f, df)
    _check(lib().ga_op_deriv(ctx, pf, int(axis), pd), ctx)


def ga_op_get_tiles(ctx, dim):
    """Complex pencils per CTA of the FFT-derivative passes, chosen by the autotuner: dim values for the
    one-field passes along each axis, then dim values for the body force's two-time-step passes."""
    arr = (_c_int * (2 * dim))()
    _check(lib().ga_op_get_tiles(ctx, arr), ctx)
    return list(arr)


def ga_op_get_sl_depth(ctx):
    """Brick depths (z voxels per thread) of the FP32 3D state and adjoint steps chosen by the autotuner:
    (state_depth, adjoint_depth)."""
    a, b = _c_int(), _c_int()
    _check(lib().ga_op_get_sl_depth(ctx, ctypes.byref(a), ctypes.byref(b)), ctx)
    return a.value, b.value


def ga_op_set_sl_depth(ctx, state_depth, adjoint_depth=None):
    """Set both depths (adjoint_depth defaults to state_depth); 0 restores 8."""
    b = state_depth if adjoint_depth is None else adjoint_depth
    _check(lib().ga_op_set_sl_depth(ctx, int(state_depth), int(b)), ctx)


def ga_op_set_tiles(ctx, pencils):
    arr = (_c_int * len(pencils))(*[int(p) for p in pencils])
    _check(lib().ga_op_set_tiles(ctx, arr), ctx)


def ga_op_div(ctx, dtype, v, mu):
    _sizes(ctx, v=(v, 'vec'), mu=(mu, 'scalar'))
    _check(lib().ga_op_div(ctx, *_dev(dtype, v, mu)), ctx)


def ga_op_fft_r2c(ctx, dtype, f, fhat):
    _sizes(ctx, f=(f, 'scalar'), fhat=(fhat, 'half'))
    _check(lib().ga_op_fft_r2c(ctx, *_dev(dtype, f, fhat)), ctx)


def ga_op_fft_c2r(ctx, dtype, fhat, f):
    _sizes(ctx, fhat=(fhat, 'half'), f=(f, 'scalar'))
    _check(lib().ga_op_fft_c2r(ctx, *_dev(dtype, fhat, f)), ctx)


def ga_op_apply_L(ctx, dtype, v, Lv):
    _sizes(ctx, v=(v, 'vec'), Lv=(Lv, 'vec'))
    _check(lib().ga_op_apply_L(ctx, *_dev(dtype, v, Lv)), ctx)


def ga_op_leray(ctx, dtype, v, pv):
    _sizes(ctx, v=(v, 'vec'), pv=(pv, 'vec'))
    _check(lib().ga_op_leray(ctx, *_dev(dtype, v, pv)), ctx)


def _dots_args(a, bs):
    if len(bs) < 1:
        raise GaError(1, "at least one vector b_i")
    na = _numel(a)
    for i, b in enumerate(bs):
        if _numel(b) != na:
            raise GaError(1, f"b[{i}] has {_numel(b)} elements, a has {na}")


def ga_op_dots(ctx, dtype, a, bs):
    _dots_args(a, bs)
    _check_device([a, *bs], (_CTX_INFO.get(ctx) or (None,) * 4)[3])
    ptrs = _dev(dtype, a, *bs)
    n = len(bs)
    arr = (_vp * n)(*ptrs[1:])
    out = (_c_double * n)()
    _check(lib().ga_op_dots(ctx, ptrs[0], arr, n, int(np.prod(tuple(a.shape))), out), ctx)
    return np.array(out[:])


def ga_op_lsq(ctx, c, a, M):
    a = np.ascontiguousarray(a, dtype=np.float64)
    M = np.ascontiguousarray(M, dtype=np.float64)
    m = a.shape[0]
    beta = np.zeros(m)
    dp = ctypes.POINTER(_c_double)
    _check(lib().ga_op_lsq(ctx, m, float(c), a.ctypes.data_as(dp), M.ctypes.data_as(dp),
                           beta.ctypes.data_as(dp)), ctx)
    return beta


def ga_dots_noalloc(dtype, a, bs, out, stream=None):
    """FP64-accurate inner products <a, b_i> into the device array `out` (float64, len(bs)) without
    any device allocation; see include/ga_ops.h for who needs this and its limits (at most 32 vectors,
    calls that overlap on the GPU race)."""
    _dots_args(a, bs)
    ptrs = _dev(dtype, a, *bs)
    (pout,) = _dev(np.float64, out)
    n = len(bs)
    if _numel(out) < n:
        raise GaError(1, f"out holds {_numel(out)} doubles, {n} are written")
    _check_device([a, *bs, out])
    arr = (_vp * n)(*ptrs[1:])
    prec = GA_PREC_FP64 if dtype == np.float64 else GA_PREC_MIXED
    st = lib().ga_dots_noalloc(prec, ptrs[0], arr, n, _numel(a), pout,
                               _vp(stream if stream is not None else _current_stream()))
    _check(st, None)


def ga_prof_start(ctx, kernel_class):
    _check(lib().ga_prof_start(ctx, int(kernel_class)), ctx)


def ga_kernel_launches():
    """Kernels launched by the library in this process so far."""
    return int(lib().ga_kernel_launches())


def ga_prof_stop(ctx):
    ms, n = _c_double(), ctypes.c_longlong()
    _check(lib().ga_prof_stop(ctx, ctypes.byref(ms), ctypes.byref(n)), ctx)
    return ms.value, n.value


# ---- convenience object --------------------------------------------------------------------------

class Problem:
    """One problem context: m0, m1 on a periodic grid, model, regulariser and solver options.

    m0, m1: arrays of shape n (2D or 3D). prec: 'fp64' or 'mixed'. Arrays passed to the methods
    follow the binding rules above; vector fields have shape (dim, *n).
    """

    def __init__(self, m0, m1, nt, model="advection", reg_order=2, alpha=1e-3, prec="fp64",
                 ckpt_every=0, window=5, sigma=4, tau=2, max_iter=200, rel_tol=1e-2, armijo_c=1e-4,
                 max_backtracks=20, variant=1, method="ga-ngmres", stream=None, graphs=False):
        shape = tuple(int(s) for s in m0.shape)
        self.shape = shape
        self.dim = len(shape)
        self.dtype = np.float64 if prec == "fp64" else np.float32
        d = ProblemDesc()
        d.dim = self.dim
        for i, s in enumerate(shape):
            d.n[i] = s
        d.nt = int(nt)
        d.model = MODELS[model]
        d.reg_order = int(reg_order)
        d.alpha = float(alpha)
        d.prec = GA_PREC_FP64 if prec == "fp64" else GA_PREC_MIXED
        d.ckpt_every = int(ckpt_every)
        o = SolverOpts()
        o.window, o.sigma, o.tau, o.max_iter = int(window), int(sigma), int(tau), int(max_iter)
        o.rel_tol, o.armijo_c, o.max_backtracks = float(rel_tol), float(armijo_c), int(max_backtracks)
        o.variant = int(variant)
        methods = {"ga-ngmres": GA_METHOD_GA_NGMRES, "rpgd": GA_METHOD_RPGD, "ga-aa": GA_METHOD_GA_AA}
        if method not in methods:
            raise ValueError(f"method must be one of {sorted(methods)}")
        o.method = methods[method]
        # graphs: False/0 kernel by kernel; True/1 evaluations replayed from CUDA graphs; "device"/2 the
        # whole solve as one graph, its line search and step decisions taken on the device
        graph_modes = {False: 0, True: 1, 0: 0, 1: 1, 2: 2, "device": 2}
        if graphs not in graph_modes:
            raise ValueError("graphs must be False, True or 'device'")
        o.graphs = graph_modes[graphs]
        self.desc, self.opts = d, o
        self.ctx = ga_setup(d, o, m0, m1, stream)

    def close(self):
        if getattr(self, "ctx", None):
            ga_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def vshape(self):
        return (self.dim,) + self.shape

    def objective(self, v):
        return ga_objective(self.ctx, self.dtype, v)

    def gradient(self, v, g):
        return ga_gradient(self.ctx, self.dtype, v, g)

    def precond(self, g, s):
        ga_precond(self.ctx, self.dtype, g, s)

    def deformation(self, v, u, detj):
        """Displacement u (grid units) of the map y = x + h u and det grad y for the velocity v."""
        ga_deformation(self.ctx, self.dtype, v, u, detj)

    def step(self, v):
        return ga_step(self.ctx, self.dtype, v)

    def solve(self, v):
        return ga_solve(self.ctx, self.dtype, v)

    def reset(self):
        ga_reset(self.ctx)

    def stats(self):
        """Counters and last-iterate metrics of the context (also after a failed call)."""
        return ga_get_stats(self.ctx)

    def transport(self, v, m1_out):
        ga_transport(self.ctx, self.dtype, v, m1_out)

    def transport_vjp(self, v, gamma, grad_v, exact=False):
        (ga_transport_vjp_exact if exact else ga_transport_vjp)(self.ctx, self.dtype, v, gamma, grad_v)

    def gradient_dto(self, v, g):
        """Gradient of the discrete objective (discretise-then-optimise); returns obj(v)."""
        return ga_gradient_dto(self.ctx, self.dtype, v, g)
