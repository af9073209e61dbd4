"""GB300-native ensemble ODE solver (the method of arXiv 2011.01740).

Thin Python binding of the C ABI declared in ``include/ens.h``: every function
below has the C name, marshals its arguments (numpy arrays, torch tensors on
the host or the GPU, streams) into plain pointers and sizes, and raises
``EnsError`` with ``ens_last_error`` when the call fails.  All numerical work
runs in the CUDA kernels of ``libens.so``; there is no CPU fallback, and a
missing library is an error.

PyTorch is used for device memory and streams only: pass CUDA tensors as
inputs / destinations and a ``torch.cuda.Stream`` (or a raw ``cudaStream_t``
integer) as ``stream``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import workloads  # noqa: F401  (input generators, no method arithmetic)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libens.so")

# enums of ens.h
ENS_OK, ENS_EINVAL, ENS_ENOMEM, ENS_ECUDA, ENS_ETIMEOUT, ENS_ESYSTEM, ENS_ENOTSUP = range(7)
ENS_SYS_TOY_X2P, ENS_SYS_LORENZ, ENS_SYS_KELLER_MIKSIS, ENS_SYS_RELIEF_VALVE, ENS_SYS_KELLER_MIKSIS_TANGENT = range(5)
ENS_RK4, ENS_RKCK45, ENS_DOPRI5 = 0, 1, 2
ENS_FP64, ENS_FP32_COMP, ENS_FP64_STRICT, ENS_FP32X2 = 0, 1, 2, 3
ENS_SYS_DT_UNDERFLOW, ENS_SYS_MAX_STEPS, ENS_SYS_NONFINITE = 1, 2, 4
ENS_SYS_EVENT_NO_CONVERGE, ENS_SYS_TIMEOUT = 8, 16
ENS_STATE, ENS_ACC, ENS_STATUS, ENS_NSTEPS, ENS_NREJ, ENS_NRHS, ENS_TIME, ENS_DT = range(8)
ENS_LAUNCH_PLAIN, ENS_LAUNCH_PERSISTENT = 0, 1

DIM = {ENS_SYS_TOY_X2P: 1, ENS_SYS_LORENZ: 3, ENS_SYS_KELLER_MIKSIS: 2, ENS_SYS_RELIEF_VALVE: 3,
       ENS_SYS_KELLER_MIKSIS_TANGENT: 4}
NPAR = {ENS_SYS_TOY_X2P: 1, ENS_SYS_LORENZ: 3, ENS_SYS_KELLER_MIKSIS: 13, ENS_SYS_RELIEF_VALVE: 5,
        ENS_SYS_KELLER_MIKSIS_TANGENT: 13}

_STATUS_NAMES = {0: "ENS_OK", 1: "ENS_EINVAL", 2: "ENS_ENOMEM", 3: "ENS_ECUDA", 4: "ENS_ETIMEOUT",
                 5: "ENS_ESYSTEM", 6: "ENS_ENOTSUP"}


class EnsError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class EnsTol(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("atol", ctypes.c_double), ("dt0", ctypes.c_double),
                ("dt_min", ctypes.c_double), ("dt_max", ctypes.c_double),
                ("event_tol", ctypes.c_double), ("max_steps", ctypes.c_int64),
                ("n_steps", ctypes.c_int64), ("n_phases", ctypes.c_int32),
                ("prec", ctypes.c_int32), ("phase_len", ctypes.c_double),
                ("acc_t_start", ctypes.c_double), ("timeout_s", ctypes.c_double),
                ("n_transient", ctypes.c_int32)]


class EnsLaunch(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("block", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("cost_order", ctypes.c_int32), ("systems_per_thread", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2)]

    def as_dict(self):
        return dict(mode=self.mode, block=self.block, blocks_per_sm=self.blocks_per_sm,
                    use_graph=self.use_graph, cost_order=self.cost_order,
                    systems_per_thread=max(1, self.systems_per_thread))


class EnsTuneRow(ctypes.Structure):
    _fields_ = [("launch", EnsLaunch), ("ms", ctypes.c_double), ("horizon_frac", ctypes.c_double)]


class EnsLiquid(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("rho", "c", "mu", "sigma", "pv", "pinf", "gamma")]


_lock = threading.Lock()
_lib = None


def lib() -> ctypes.CDLL:
    """Load libens.so (building it with nvcc first if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        from . import build as _build
        if not _build.up_to_date():
            _build.build()
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: the CUDA library must be built")
        L = ctypes.CDLL(LIB_PATH)
        vp, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
        st = ctypes.c_int
        L.ens_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int64, vp, vp,
                                 ctypes.c_double * 2, ctypes.c_int, ctypes.POINTER(EnsTol)]
        L.ens_create.restype = st
        L.ens_set_inputs.argtypes = [vp, vp, vp, vp]
        L.ens_set_inputs.restype = st
        L.ens_set_launch.argtypes = [vp, ctypes.POINTER(EnsLaunch)]
        L.ens_set_launch.restype = st
        L.ens_get_launch.argtypes = [vp, ctypes.POINTER(EnsLaunch)]
        L.ens_get_launch.restype = st
        L.ens_solve.argtypes = [vp, vp]
        L.ens_solve.restype = st
        L.ens_sync.argtypes = [vp]
        L.ens_sync.restype = st
        L.ens_kernel_ms.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
        L.ens_kernel_ms.restype = st
        L.ens_read.argtypes = [vp, ctypes.c_int, vp, ctypes.c_size_t]
        L.ens_read.restype = st
        L.ens_acc_rows.argtypes = [vp]
        L.ens_acc_rows.restype = ctypes.c_int64
        L.ens_size.argtypes = [vp]
        L.ens_size.restype = ctypes.c_int64
        L.ens_dim.argtypes = [vp]
        L.ens_dim.restype = ctypes.c_int32
        L.ens_npar.argtypes = [vp]
        L.ens_npar.restype = ctypes.c_int32
        L.ens_autotune.argtypes = [vp, vp, ctypes.POINTER(EnsLaunch)]
        L.ens_autotune.restype = st
        L.ens_last_error.argtypes = [vp]
        L.ens_last_error.restype = ctypes.c_char_p
        L.ens_destroy.argtypes = [vp]
        L.ens_destroy.restype = None
        L.ens_km_coefficients.argtypes = [ctypes.c_int64, vp, vp, vp, vp, vp, vp,
                                          ctypes.POINTER(EnsLiquid), vp, vp]
        L.ens_km_coefficients.restype = st
        L.ens_version.restype = ctypes.c_char_p
        _lib = L
        return L


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------

def _ptr(x, keep: list):
    """Raw address of a float64 / int array (numpy or torch, host or device)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):                  # torch tensor
        if not x.is_contiguous():
            x = x.contiguous()
        keep.append(x)
        return x.data_ptr()
    a = np.ascontiguousarray(x)
    keep.append(a)
    return a.ctypes.data


def _as_f64(x):
    if hasattr(x, "data_ptr"):
        import torch
        return x.to(torch.float64).contiguous()
    return np.ascontiguousarray(x, dtype=np.float64)


def _stream(stream, keep=None):
    """The raw stream handle.  With `keep` (the arrays of a call), every CUDA
    tensor among them is marked as used by that stream (record_stream), so
    that PyTorch's caching allocator does not hand its memory to another
    tensor while the asynchronous work queued here may still read or write
    it -- also when the caller drops its last reference right after the call
    (a temporary argument)."""
    if keep and stream is not None:
        try:
            import torch
            ts = stream if isinstance(stream, torch.cuda.Stream) else torch.cuda.ExternalStream(int(stream))
            for t in keep:
                if isinstance(t, torch.Tensor) and t.is_cuda:
                    t.record_stream(ts)
        except ImportError:
            pass
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return 0
    if hasattr(stream, "cuda_stream"):
        return int(stream.cuda_stream)
    return int(stream)


def _check(status: int, ctx=None):
    if status != ENS_OK:
        msg = lib().ens_last_error(ctx).decode(errors="replace")
        raise EnsError(status, msg)


def make_tol(rtol=1e-10, atol=1e-10, dt0=1e-2, dt_min=1e-14, dt_max=1e-1, event_tol=1e-6,
             max_steps=2_000_000_000, n_steps=0, n_phases=0, prec=ENS_FP64, phase_len=1.0,
             acc_t_start=0.0, timeout_s=600.0, n_transient=0) -> EnsTol:
    return EnsTol(rtol, atol, dt0, dt_min, dt_max, event_tol, int(max_steps), int(n_steps),
                  int(n_phases), int(prec), phase_len, acc_t_start, timeout_s, int(n_transient))


def make_launch(mode=ENS_LAUNCH_PERSISTENT, block=128, blocks_per_sm=2, use_graph=0,
                cost_order=0, systems_per_thread=1) -> EnsLaunch:
    return EnsLaunch(mode, block, blocks_per_sm, use_graph, cost_order, systems_per_thread)


# ---------------------------------------------------------------------------
# the C ABI, one Python function per entry point
# ---------------------------------------------------------------------------

def ens_version() -> str:
    return lib().ens_version().decode()


def ens_create(sys: int, n: int, params, y0, t_span, solver: int, tol: EnsTol) -> int:
    """Returns the context handle (an int); inputs are copied by the library."""
    keep = []
    params = _as_f64(params)
    y0 = _as_f64(y0)
    ctx = ctypes.c_void_p()
    ts = (ctypes.c_double * 2)(float(t_span[0]), float(t_span[1]))
    st = lib().ens_create(ctypes.byref(ctx), int(sys), int(n), _ptr(params, keep), _ptr(y0, keep),
                          ts, int(solver), ctypes.byref(tol))
    _check(st, None)
    return ctx.value


def ens_set_inputs(ctx: int, params=None, y0=None, stream=None):
    keep = []
    params = None if params is None else _as_f64(params)
    y0 = None if y0 is None else _as_f64(y0)
    _check(lib().ens_set_inputs(ctx, _ptr(params, keep), _ptr(y0, keep), _stream(stream, keep)), ctx)


def ens_set_launch(ctx: int, cfg: EnsLaunch | None):
    _check(lib().ens_set_launch(ctx, ctypes.byref(cfg) if cfg is not None else None), ctx)


def ens_get_launch(ctx: int) -> EnsLaunch:
    cfg = EnsLaunch()
    _check(lib().ens_get_launch(ctx, ctypes.byref(cfg)), ctx)
    return cfg


def ens_solve(ctx: int, stream=None):
    _check(lib().ens_solve(ctx, _stream(stream)), ctx)


def ens_sync(ctx: int, raise_on_system: bool = False) -> int:
    """Wait for the last solve; returns ENS_OK / ENS_ETIMEOUT / ENS_ESYSTEM
    (raises for call failures, and for the latter two if asked)."""
    st = lib().ens_sync(ctx)
    if st in (ENS_ETIMEOUT, ENS_ESYSTEM) and not raise_on_system:
        return st
    _check(st, ctx)
    return st


def ens_kernel_ms(ctx: int) -> float:
    """Device milliseconds of the last solve's main kernel (after ens_sync)."""
    ms = ctypes.c_double(0.0)
    _check(lib().ens_kernel_ms(ctx, ctypes.byref(ms)), ctx)
    return ms.value


_READ_DTYPE = {ENS_STATE: np.float64, ENS_ACC: np.float64, ENS_STATUS: np.int32,
               ENS_NSTEPS: np.int64, ENS_NREJ: np.int64, ENS_NRHS: np.int64,
               ENS_TIME: np.float64, ENS_DT: np.float64}


def ens_read(ctx: int, which: int, dst=None):
    """Copy one output into dst (numpy / torch, host or device); with dst=None
    a numpy array of the selector's shape is returned."""
    L = lib()
    n = L.ens_size(ctx)
    if dst is None:
        rows = {ENS_STATE: L.ens_dim(ctx), ENS_ACC: L.ens_acc_rows(ctx)}.get(which, 1)
        dst = np.empty((rows, n) if which in (ENS_STATE, ENS_ACC) else (n,), dtype=_READ_DTYPE[which])
    keep = []
    p = _ptr(dst, keep)
    nbytes = dst.element_size() * dst.numel() if hasattr(dst, "element_size") else dst.nbytes
    _check(L.ens_read(ctx, int(which), p, nbytes), ctx)
    return dst


def ens_acc_rows(ctx: int) -> int:
    return int(lib().ens_acc_rows(ctx))


def ens_size(ctx: int) -> int:
    return int(lib().ens_size(ctx))


def ens_dim(ctx: int) -> int:
    return int(lib().ens_dim(ctx))


def ens_npar(ctx: int) -> int:
    return int(lib().ens_npar(ctx))


def ens_autotune(ctx: int, stream=None) -> EnsLaunch:
    best = EnsLaunch()
    _check(lib().ens_autotune(ctx, _stream(stream), ctypes.byref(best)), ctx)
    return best


def ens_autotune_table(ctx: int) -> list:
    """Candidates of the context's last ens_autotune: a list of dicts with the
    launch, the main-kernel milliseconds and the horizon fraction timed."""
    L = lib()
    if not getattr(L, "_tune_bound", False):
        L.ens_autotune_table.argtypes = [ctypes.c_void_p, ctypes.POINTER(EnsTuneRow), ctypes.c_int32]
        L.ens_autotune_table.restype = ctypes.c_int32
        L._tune_bound = True
    n = int(L.ens_autotune_table(ctx, None, 0))
    rows = (EnsTuneRow * max(n, 1))()
    n = int(L.ens_autotune_table(ctx, rows, n))
    return [dict(launch=r.launch.as_dict(), ms=r.ms, horizon_frac=r.horizon_frac) for r in rows[:n]]


def ens_eval_rhs(sys: int, n: int, params, t, y, dy, stream=None):
    """dy = f(t, y; params) on the device (all arrays torch CUDA tensors)."""
    L = lib()
    if not getattr(L, "_rhs_bound", False):
        vp = ctypes.c_void_p
        L.ens_eval_rhs.argtypes = [ctypes.c_int, ctypes.c_int64, vp, vp, vp, vp, vp]
        L.ens_eval_rhs.restype = ctypes.c_int
        L._rhs_bound = True
    keep = []
    _check(L.ens_eval_rhs(int(sys), int(n), _ptr(params, keep), _ptr(t, keep), _ptr(y, keep), _ptr(dy, keep),
                          _stream(stream, keep)), None)
    return dy


def ens_solve_noalloc(sys: int, n: int, params, y0, t_span, tol: EnsTol, y, t_out, dt_out, acc, status,
                      nacc, nrej, nrhs, cost_order: int = 1, stream=None):
    """Allocation-free solve on caller-owned device buffers (torch CUDA
    tensors); see ens.h.  For callers that cannot allocate device memory."""
    L = lib()
    if not getattr(L, "_noalloc_bound", False):
        vp = ctypes.c_void_p
        L.ens_solve_noalloc.argtypes = [ctypes.c_int, ctypes.c_int64, vp, vp, ctypes.c_double * 2,
                                        ctypes.POINTER(EnsTol)] + [vp] * 8 + [ctypes.c_int32, vp]
        L.ens_solve_noalloc.restype = ctypes.c_int
        L._noalloc_bound = True
    keep = []
    ts = (ctypes.c_double * 2)(float(t_span[0]), float(t_span[1]))
    ptrs = [_ptr(a, keep) for a in (params, y0)]
    outs = [_ptr(a, keep) for a in (y, t_out, dt_out, acc, status, nacc, nrej, nrhs)]
    _check(L.ens_solve_noalloc(int(sys), int(n), *ptrs, ts, ctypes.byref(tol), *outs, int(cost_order),
                               _stream(stream, keep)), None)


def ens_last_error(ctx: int | None = None) -> str:
    return lib().ens_last_error(ctx).decode(errors="replace")


def ens_destroy(ctx: int):
    if ctx:
        lib().ens_destroy(ctx)


def ens_km_coefficients(pA1, f1, pA2, f2, theta, RE, liquid: dict, out=None, stream=None):
    """C0..C12 (13, n) from SI parameters; all arrays host (numpy) or all
    device (torch CUDA tensors)."""
    arrs = [_as_f64(a) for a in (pA1, f1, pA2, f2, theta, RE)]
    n = int(arrs[0].numel() if hasattr(arrs[0], "numel") else arrs[0].size)
    if out is None:
        if hasattr(arrs[0], "data_ptr") and arrs[0].is_cuda:
            import torch
            out = torch.empty((13, n), dtype=torch.float64, device=arrs[0].device)
        else:
            out = np.empty((13, n), dtype=np.float64)
    keep = []
    liq = EnsLiquid(*[float(liquid[k]) for k in ("rho", "c", "mu", "sigma", "pv", "pinf", "gamma")])
    st = lib().ens_km_coefficients(n, *[_ptr(a, keep) for a in arrs], ctypes.byref(liq),
                                   _ptr(out, keep), _stream(stream, keep))
    _check(st, None)
    return out


# ---------------------------------------------------------------------------
# surrogate network (device arrays: torch CUDA tensors)
# ---------------------------------------------------------------------------

class EnsTrainCfg(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int32), ("batch", ctypes.c_int32), ("lr", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
                ("seed", ctypes.c_uint64), ("lr_final", ctypes.c_float)]


def make_train_cfg(epochs=50, batch=1024, lr=2e-3, beta1=0.9, beta2=0.999, eps=1e-8, seed=20201103,
                   lr_final=0.0):
    return EnsTrainCfg(int(epochs), int(batch), lr, beta1, beta2, eps, int(seed), lr_final)


_mlp_bound = False


def _mlp_lib():
    global _mlp_bound
    L = lib()
    if not _mlp_bound:
        vp = ctypes.c_void_p
        st = ctypes.c_int
        L.ens_mlp_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int32, ctypes.c_uint64]
        L.ens_mlp_create.restype = st
        L.ens_mlp_param_count.restype = ctypes.c_int64
        L.ens_mlp_set_params.argtypes = [vp, vp, ctypes.c_size_t]
        L.ens_mlp_set_params.restype = st
        L.ens_mlp_get_params.argtypes = [vp, vp, ctypes.c_size_t]
        L.ens_mlp_get_params.restype = st
        L.ens_mlp_forward.argtypes = [vp, ctypes.c_int64, vp, vp, vp]
        L.ens_mlp_forward.restype = st
        L.ens_mlp_loss_grad.argtypes = [vp, ctypes.c_int64, vp, vp, vp, vp, vp]
        L.ens_mlp_loss_grad.restype = st
        L.ens_mlp_train.argtypes = [vp, ctypes.c_int64, vp, vp, ctypes.POINTER(EnsTrainCfg), vp, vp]
        L.ens_mlp_train.restype = st
        L.ens_mlp_screen.argtypes = [vp, ctypes.c_int64, vp, vp, vp, vp, vp]
        L.ens_mlp_screen.restype = st
        L.ens_mlp_last_error.argtypes = [vp]
        L.ens_mlp_last_error.restype = ctypes.c_char_p
        L.ens_mlp_destroy.argtypes = [vp]
        L.ens_mlp_destroy.restype = None
        L.ens_km_features.argtypes = [ctypes.c_int64, vp, vp, ctypes.c_double * 4, vp, vp]
        L.ens_km_features.restype = st
        L.ens_km_labels.argtypes = [ctypes.c_int64, vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, vp, vp]
        L.ens_km_labels.restype = st
        L.ens_select_above.argtypes = [ctypes.c_int64, vp, ctypes.c_float, vp, ctypes.POINTER(ctypes.c_int64), vp]
        L.ens_select_above.restype = st
        L.ens_select_gate.argtypes = [ctypes.c_int64, vp, ctypes.c_float, vp, ctypes.c_float, vp,
                                      ctypes.POINTER(ctypes.c_int64), vp]
        L.ens_select_gate.restype = st
        L.ens_grid_gradient.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, vp, ctypes.c_float,
                                        ctypes.c_float, vp, vp]
        L.ens_grid_gradient.restype = st
        L.ens_feature_stencil.argtypes = [ctypes.c_int64, vp, ctypes.c_float, ctypes.c_float, vp, vp]
        L.ens_feature_stencil.restype = st
        L.ens_stencil_gradient.argtypes = [ctypes.c_int64, vp, ctypes.c_float, ctypes.c_float, vp, vp]
        L.ens_stencil_gradient.restype = st
        L.ens_gather_f64.argtypes = [ctypes.c_int64, vp, vp, vp, vp]
        L.ens_gather_f64.restype = st
        L.ens_scatter_labels.argtypes = [ctypes.c_int64, vp, vp, vp, vp]
        L.ens_scatter_labels.restype = st
        _mlp_bound = True
    return L


def _mcheck(status: int, m=None):
    if status != ENS_OK:
        raise EnsError(status, _mlp_lib().ens_mlp_last_error(m).decode(errors="replace"))


def _nbytes(a):
    return a.element_size() * a.numel() if hasattr(a, "element_size") else a.nbytes


def ens_mlp_create(members: int = 4, seed: int = 20201103) -> int:
    m = ctypes.c_void_p()
    _mcheck(_mlp_lib().ens_mlp_create(ctypes.byref(m), int(members), int(seed)))
    return m.value


def ens_mlp_param_count() -> int:
    return int(_mlp_lib().ens_mlp_param_count())


def ens_mlp_set_params(m: int, params):
    keep = []
    _mcheck(_mlp_lib().ens_mlp_set_params(m, _ptr(params, keep), _nbytes(params)), m)


def ens_mlp_get_params(m: int, params):
    keep = []
    _mcheck(_mlp_lib().ens_mlp_get_params(m, _ptr(params, keep), _nbytes(params)), m)
    return params


def ens_mlp_forward(m: int, n: int, x, out, stream=None):
    keep = []
    _mcheck(_mlp_lib().ens_mlp_forward(m, int(n), _ptr(x, keep), _ptr(out, keep), _stream(stream, keep)), m)
    return out


def ens_mlp_loss_grad(m: int, n: int, x, y, members: int, grad, stream=None):
    keep = []
    loss = (ctypes.c_float * members)()
    _mcheck(_mlp_lib().ens_mlp_loss_grad(m, int(n), _ptr(x, keep), _ptr(y, keep), ctypes.cast(loss, ctypes.c_void_p),
                                         _ptr(grad, keep), _stream(stream, keep)), m)
    return np.array(list(loss), dtype=np.float32)


def ens_mlp_train(m: int, n: int, x, y, cfg: EnsTrainCfg, members: int, stream=None):
    keep = []
    hist = np.zeros((max(cfg.epochs, 1), members), dtype=np.float32)
    _mcheck(_mlp_lib().ens_mlp_train(m, int(n), _ptr(x, keep), _ptr(y, keep), ctypes.byref(cfg),
                                     hist.ctypes.data, _stream(stream, keep)), m)
    return hist[: cfg.epochs]


def ens_mlp_screen(m: int, n: int, x, mean, stdv, p1, stream=None):
    keep = []
    _mcheck(_mlp_lib().ens_mlp_screen(m, int(n), _ptr(x, keep), _ptr(mean, keep), _ptr(stdv, keep), _ptr(p1, keep),
                                      _stream(stream, keep)), m)


def ens_mlp_set_screen_impl(m: int, impl: int) -> int:
    """Select the screening kernel (1 tcgen05, 0 mma.sync); returns 1 if a
    tcgen05 launch since the last call gave up waiting for its tensor cores."""
    L = _mlp_lib()
    if not getattr(L, "_impl_bound", False):
        L.ens_mlp_set_screen_impl.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
        L.ens_mlp_set_screen_impl.restype = ctypes.c_int
        L._impl_bound = True
    flag = ctypes.c_int32(0)
    _mcheck(L.ens_mlp_set_screen_impl(m, int(impl), ctypes.byref(flag)), m)
    return int(flag.value)


def ens_mlp_set_train_impl(m: int, impl: int) -> int:
    """Select the training kernels (1 tcgen05, 0 mma.sync); returns 1 if a
    tcgen05 training launch gave up waiting for its tensor cores since the
    flag was last cleared."""
    L = _mlp_lib()
    if not getattr(L, "_train_impl_bound", False):
        L.ens_mlp_set_train_impl.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
        L.ens_mlp_set_train_impl.restype = ctypes.c_int
        L._train_impl_bound = True
    flag = ctypes.c_int32(0)
    _mcheck(L.ens_mlp_set_train_impl(m, int(impl), ctypes.byref(flag)), m)
    return int(flag.value)


def ens_mlp_last_error(m: int | None = None) -> str:
    return _mlp_lib().ens_mlp_last_error(m).decode(errors="replace")


def ens_mlp_destroy(m: int):
    if m:
        _mlp_lib().ens_mlp_destroy(m)


def ens_km_features(n: int, pA, f, rng, x, stream=None):
    keep = []
    r = (ctypes.c_double * 4)(*[float(v) for v in rng])
    _mcheck(_mlp_lib().ens_km_features(int(n), _ptr(pA, keep), _ptr(f, keep), r, _ptr(x, keep), _stream(stream, keep)))
    return x


def ens_km_labels(n: int, acc, n_phases: int, first_phase: int, spread_tol: float, y, stream=None):
    keep = []
    _mcheck(_mlp_lib().ens_km_labels(int(n), _ptr(acc, keep), int(n_phases), int(first_phase), float(spread_tol),
                                     _ptr(y, keep), _stream(stream, keep)))
    return y


def ens_select_gate(n: int, v, thr: float, w, thr_w: float, idx, stream=None) -> int:
    """Indices with v > thr or w > thr_w (w may be None) into idx; returns the count."""
    keep = []
    cnt = ctypes.c_int64(0)
    _mcheck(_mlp_lib().ens_select_gate(int(n), _ptr(v, keep), float(thr), _ptr(w, keep), float(thr_w),
                                       _ptr(idx, keep), ctypes.byref(cnt), _stream(stream, keep)))
    return int(cnt.value)


def ens_grid_gradient(rows: int, cols: int, stride: int, v, d_row: float, d_col: float, g, stream=None):
    keep = []
    _mcheck(_mlp_lib().ens_grid_gradient(int(rows), int(cols), int(stride), _ptr(v, keep), float(d_row),
                                         float(d_col), _ptr(g, keep), _stream(stream, keep)))
    return g


def ens_feature_stencil(n: int, x, d0: float, d1: float, out, stream=None):
    keep = []
    _mcheck(_mlp_lib().ens_feature_stencil(int(n), _ptr(x, keep), float(d0), float(d1), _ptr(out, keep),
                                           _stream(stream, keep)))
    return out


def ens_stencil_gradient(n: int, v, d0: float, d1: float, g, stream=None):
    keep = []
    _mcheck(_mlp_lib().ens_stencil_gradient(int(n), _ptr(v, keep), float(d0), float(d1), _ptr(g, keep),
                                            _stream(stream, keep)))
    return g


def ens_select_above(n: int, v, thr: float, idx, stream=None) -> int:
    keep = []
    cnt = ctypes.c_int64(0)
    _mcheck(_mlp_lib().ens_select_above(int(n), _ptr(v, keep), float(thr), _ptr(idx, keep), ctypes.byref(cnt),
                                        _stream(stream, keep)))
    return int(cnt.value)


def ens_gather_f64(k: int, idx, src, dst, stream=None):
    keep = []
    _mcheck(_mlp_lib().ens_gather_f64(int(k), _ptr(idx, keep), _ptr(src, keep), _ptr(dst, keep), _stream(stream, keep)))
    return dst


def ens_scatter_labels(k: int, idx, y, dst, stream=None):
    keep = []
    _mcheck(_mlp_lib().ens_scatter_labels(int(k), _ptr(idx, keep), _ptr(y, keep), _ptr(dst, keep), _stream(stream, keep)))
    return dst
