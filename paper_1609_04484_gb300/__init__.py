"""GB300 double-layer Stokes solver: Python binding of libstokes.so.

The functions below have the names of the C ABI in include/stokes.h and do
argument marshalling only: every step of the computation runs in the CUDA
library. Arrays may be numpy arrays (host memory) or torch tensors (host or
CUDA); they must be C-contiguous float64 (offsets/centres: host). Importing
this package raises if the compiled library is missing: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import pathlib

import numpy as np

__all__ = [
    "STOKES_OK", "STOKES_EINVAL", "STOKES_ENOMEM", "STOKES_ECUDA", "STOKES_ENOTCONV",
    "STOKES_EBREAKDOWN", "STOKES_ESTATE", "STOKES_FP64", "STOKES_FP32", "STOKES_DF64",
    "STOKES_MIXED_IR", "STOKES_PC_NONE", "STOKES_PC_BLOCKDIAG", "STOKES_PC_RIGHT", "STOKES_PC_LEFT",
    "StokesError", "lib", "library_path", "stokes_geometry_create", "stokes_geometry_destroy",
    "stokes_geometry_num_nodes", "stokes_matvec", "stokes_precond_setup", "stokes_precond_apply",
    "stokes_precond_apply_prec", "stokes_precond_setup_twogrid", "STOKES_PC_TWOGRID",
    "stokes_gmres_solve", "stokes_eval_velocity", "stokes_last_error", "Geometry",
    "stokes_profile_enable", "stokes_profile_read", "STOKES_PROF_PAIRS_FP64", "STOKES_PROF_PAIRS_FP32",
    "STOKES_PROF_PAIRS_DF64", "STOKES_PROF_EPILOGUE", "STOKES_PROF_BD_APPLY", "STOKES_PROF_ARNOLDI",
    "STOKES_PROF_BD_SETUP", "STOKES_PROF_LU_GEMM", "STOKES_PROF_LU_PANEL", "STOKES_PROF_COARSE_SOLVE",
    "stokes_kernel_launches", "stokes_matvec_noalloc",
    "stokes_pair_shape_count", "stokes_pair_shape_info", "stokes_set_pair_shape", "stokes_get_pair_shape",
    "stokes_autotune", "stokes_tune_cache_insert", "stokes_tune_cache_lookup", "stokes_tune_cache_clear",
    "stokes_tune_cache_save", "stokes_tune_cache_load", "stokes_batch_matvec", "stokes_batch_solve",
    "stokes_precond_setup_twogrid_ex", "stokes_rcp_f64", "STOKES_PC_BD_LEARNED", "STOKES_PC_BD_COARSE",
    "stokes_coarse_model_num_params", "stokes_coarse_model_create", "stokes_coarse_model_destroy",
    "stokes_coarse_model_add_geometry", "stokes_coarse_model_num_samples", "stokes_coarse_model_train",
    "stokes_coarse_model_save", "stokes_coarse_model_load", "stokes_coarse_model_forward",
    "stokes_coarse_model_loss_grad", "stokes_coarse_model_adam_step", "stokes_coarse_features",
    "stokes_coarse_operator", "STOKES_TG_COARSE_AUTO", "STOKES_TG_COARSE_INVERSE", "STOKES_TG_COARSE_LU",
]

STOKES_OK, STOKES_EINVAL, STOKES_ENOMEM, STOKES_ECUDA = 0, -1, -2, -3
STOKES_ENOTCONV, STOKES_EBREAKDOWN, STOKES_ESTATE = -4, -5, -6
STOKES_FP64, STOKES_FP32, STOKES_DF64, STOKES_MIXED_IR = 0, 1, 2, 3
STOKES_PC_NONE, STOKES_PC_BLOCKDIAG, STOKES_PC_TWOGRID, STOKES_PC_BD_LEARNED, STOKES_PC_BD_COARSE = 0, 1, 2, 3, 4
STOKES_PC_RIGHT, STOKES_PC_LEFT = 0, 1
STOKES_TG_COARSE_AUTO, STOKES_TG_COARSE_INVERSE, STOKES_TG_COARSE_LU = 0, 1, 2
(STOKES_PROF_PAIRS_FP64, STOKES_PROF_PAIRS_FP32, STOKES_PROF_PAIRS_DF64, STOKES_PROF_EPILOGUE,
 STOKES_PROF_BD_APPLY, STOKES_PROF_ARNOLDI, STOKES_PROF_BD_SETUP, STOKES_PROF_LU_GEMM, STOKES_PROF_LU_PANEL,
 STOKES_PROF_COARSE_SOLVE) = range(10)

_PKG = pathlib.Path(__file__).resolve().parent
library_path = _PKG / "lib" / "libstokes.so"


class StokesError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


def _load():
    if not library_path.exists():
        raise ImportError(f"libstokes.so not built ({library_path}); run __graft_entry__.build()")
    L = ctypes.CDLL(str(library_path))
    P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    sig = {
        "stokes_geometry_create": (I, [P, P, P, P, P, I, I, P, P, ctypes.POINTER(P)]),
        "stokes_geometry_destroy": (I, [P]),
        "stokes_geometry_num_nodes": (I64, [P]),
        "stokes_matvec": (I, [P, P, P, I]),
        "stokes_precond_setup": (I, [P, I, P]),
        "stokes_coarse_model_num_params": (I64, []),
        "stokes_coarse_model_create": (I, [P, I64, P, ctypes.POINTER(P)]),
        "stokes_coarse_model_destroy": (I, [P]),
        "stokes_coarse_model_add_geometry": (I, [P, P]),
        "stokes_coarse_model_num_samples": (I64, [P]),
        "stokes_coarse_model_train": (I, [P, I, D, ctypes.POINTER(D)]),
        "stokes_coarse_model_save": (I, [P, P, P]),
        "stokes_coarse_model_load": (I, [P, P, P]),
        "stokes_coarse_model_forward": (I, [P, P, I64, P]),
        "stokes_coarse_model_loss_grad": (I, [P, P, P, P, I64, ctypes.POINTER(D), P]),
        "stokes_coarse_model_adam_step": (I, [P, P, D]),
        "stokes_coarse_features": (I, [P, P, P]),
        "stokes_coarse_operator": (I, [P, P, P]),
        "stokes_precond_setup_twogrid": (I, [P, I]),
        "stokes_precond_setup_twogrid_ex": (I, [P, I, I]),
        "stokes_precond_apply": (I, [P, P, P]),
        "stokes_precond_apply_prec": (I, [P, P, P, I]),
        "stokes_gmres_solve": (I, [P, P, D, I, I, I, I, P, ctypes.POINTER(I), ctypes.POINTER(D),
                                   ctypes.POINTER(D)]),
        "stokes_eval_velocity": (I, [P, P, P, I64, P, I]),
        "stokes_last_error": (ctypes.c_char_p, []),
        "stokes_profile_enable": (I, [P, I]),
        "stokes_kernel_launches": (I64, []),
        "stokes_matvec_noalloc": (I, [P, P, P, P, P, I, I, P, P, P, P]),
        "stokes_profile_read": (I, [P, I, ctypes.POINTER(I64), ctypes.POINTER(D), ctypes.POINTER(D)]),
        "stokes_pair_shape_count": (I, [I]),
        "stokes_pair_shape_info": (I, [I, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)]),
        "stokes_set_pair_shape": (I, [P, I, I, I]),
        "stokes_get_pair_shape": (I, [P, I, I64, ctypes.POINTER(I), ctypes.POINTER(I)]),
        "stokes_autotune": (I, [P, I, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(D)]),
        "stokes_tune_cache_insert": (I, [I, I64, I64, I, I, D]),
        "stokes_tune_cache_lookup": (I, [I, I64, I64, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(D)]),
        "stokes_tune_cache_clear": (I, []),
        "stokes_tune_cache_save": (I, [ctypes.c_char_p]),
        "stokes_tune_cache_load": (I, [ctypes.c_char_p, ctypes.POINTER(I)]),
        "stokes_batch_matvec": (I, [P, I, I, P, P, I]),
        "stokes_batch_solve": (I, [P, I, I, P, D, I, I, I, P, P, P, P]),
        "stokes_rcp_f64": (I, [P, P, I64, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    return L


lib = _load()


def stokes_last_error() -> str:
    return lib.stokes_last_error().decode()


def _check(code, allow=()):
    if code != STOKES_OK and code not in allow:
        raise StokesError(code, stokes_last_error())
    return code


def _ptr(a, dtype=np.float64, count=None):
    """Address of a C-contiguous numpy array or torch tensor (host or CUDA)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):  # torch.Tensor
        import torch
        want = {np.float64: torch.float64, np.int64: torch.int64}[dtype]
        if a.dtype != want or not a.is_contiguous():
            raise TypeError(f"tensor must be contiguous {want}")
        if count is not None and a.numel() != count:
            raise ValueError(f"expected {count} elements, got {a.numel()}")
        return ctypes.c_void_p(a.data_ptr())
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
        raise TypeError(f"array must be a C-contiguous {np.dtype(dtype).name} numpy array or tensor")
    if count is not None and a.size != count:
        raise ValueError(f"expected {count} elements, got {a.size}")
    return ctypes.c_void_p(a.ctypes.data)


def stokes_geometry_create(nodes, normals, weights, curvature, offsets, n_comp, outer_comp,
                           centres=None, stream=None):
    """Returns an opaque handle (int). See include/stokes.h."""
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    N = int(off[-1])
    cen = None if centres is None else np.ascontiguousarray(centres, dtype=np.float64)
    h = ctypes.c_void_p()
    st = None if stream is None else ctypes.c_void_p(int(stream))
    _check(lib.stokes_geometry_create(_ptr(nodes, count=2 * N), _ptr(normals, count=2 * N),
                                      _ptr(weights, count=N), _ptr(curvature, count=N),
                                      _ptr(off, np.int64), int(n_comp), int(outer_comp),
                                      _ptr(cen), st, ctypes.byref(h)))
    return h.value


def stokes_geometry_destroy(handle):
    _check(lib.stokes_geometry_destroy(ctypes.c_void_p(handle)))


def stokes_geometry_num_nodes(handle) -> int:
    return int(lib.stokes_geometry_num_nodes(ctypes.c_void_p(handle)))


def stokes_matvec(handle, sigma, y, precision=STOKES_FP64):
    n2 = 2 * stokes_geometry_num_nodes(handle)
    _check(lib.stokes_matvec(ctypes.c_void_p(handle), _ptr(sigma, count=n2), _ptr(y, count=n2), int(precision)))


def stokes_precond_setup(handle, pc_kind=STOKES_PC_BLOCKDIAG, model=None):
    _check(lib.stokes_precond_setup(ctypes.c_void_p(handle), int(pc_kind),
                                    None if model is None else ctypes.c_void_p(model)))


def stokes_precond_setup_twogrid(handle, coarsen=8):
    _check(lib.stokes_precond_setup_twogrid(ctypes.c_void_p(handle), int(coarsen)))


def stokes_precond_setup_twogrid_ex(handle, coarsen=8, coarse_mode=STOKES_TG_COARSE_AUTO):
    _check(lib.stokes_precond_setup_twogrid_ex(ctypes.c_void_p(handle), int(coarsen), int(coarse_mode)))


def stokes_precond_apply(handle, v, z):
    n2 = 2 * stokes_geometry_num_nodes(handle)
    _check(lib.stokes_precond_apply(ctypes.c_void_p(handle), _ptr(v, count=n2), _ptr(z, count=n2)))


def stokes_precond_apply_prec(handle, v, z, precision=STOKES_FP64):
    n2 = 2 * stokes_geometry_num_nodes(handle)
    _check(lib.stokes_precond_apply_prec(ctypes.c_void_p(handle), _ptr(v, count=n2), _ptr(z, count=n2),
                                         int(precision)))


def stokes_gmres_solve(handle, f, sigma, tol=1e-8, restart=50, max_iter=2000,
                       precision=STOKES_FP64, pc_side=STOKES_PC_RIGHT):
    """Solves in place into `sigma` (its content is the initial guess).
    Returns (status, iters, true_relres, pc_relres); status is STOKES_OK or
    STOKES_ENOTCONV, other failures raise."""
    n2 = 2 * stokes_geometry_num_nodes(handle)
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    pr = ctypes.c_double(0.0)
    code = lib.stokes_gmres_solve(ctypes.c_void_p(handle), _ptr(f, count=n2), float(tol), int(restart),
                                  int(max_iter), int(precision), int(pc_side), _ptr(sigma, count=n2),
                                  ctypes.byref(it), ctypes.byref(rr), ctypes.byref(pr))
    _check(code, allow=(STOKES_ENOTCONV,))
    return code, it.value, rr.value, pr.value


def stokes_eval_velocity(handle, sigma, targets, u, precision=STOKES_FP64):
    n2 = 2 * stokes_geometry_num_nodes(handle)
    T = (targets.numel() if hasattr(targets, "numel") else targets.size) // 2
    _check(lib.stokes_eval_velocity(ctypes.c_void_p(handle), _ptr(sigma, count=n2), _ptr(targets, count=2 * T),
                                    ctypes.c_int64(T), _ptr(u, count=2 * T), int(precision)))


def stokes_kernel_launches() -> int:
    return int(lib.stokes_kernel_launches())


def stokes_profile_enable(handle, on=True):
    _check(lib.stokes_profile_enable(ctypes.c_void_p(handle), int(bool(on))))


def stokes_profile_read(handle, kind):
    """Returns (launches, total_ms, total_units) for one kernel class."""
    n = ctypes.c_int64(0)
    ms = ctypes.c_double(0.0)
    u = ctypes.c_double(0.0)
    _check(lib.stokes_profile_read(ctypes.c_void_p(handle), int(kind), ctypes.byref(n), ctypes.byref(ms),
                                   ctypes.byref(u)))
    return n.value, ms.value, u.value


def stokes_matvec_noalloc(nodes, normals, weights, curvature, offsets, n_comp, outer_comp, centres, sigma, y,
                          stream=None):
    """y = A sigma in FP64 without a handle and without allocating GPU memory
    (for callers that cannot allocate). nodes, normals, weights, curvature,
    sigma and y must be device arrays (torch CUDA tensors) of the current
    device; offsets (n_comp + 1 entries) and centres (2 n_comp) are host
    arrays. Returns the status code (STOKES_EINVAL for host arrays or a
    problem beyond the fixed scratch size)."""
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    cen = np.ascontiguousarray(centres, dtype=np.float64)
    if off.ndim != 1 or off.size != int(n_comp) + 1:
        raise ValueError(f"offsets must have n_comp + 1 = {int(n_comp) + 1} entries, got {off.size}")
    if cen.size < 2 * int(n_comp):
        raise ValueError(f"centres must have 2 n_comp = {2 * int(n_comp)} entries, got {cen.size}")
    N = int(off[int(n_comp)])
    st = None if stream is None else ctypes.c_void_p(int(stream))
    return int(lib.stokes_matvec_noalloc(_ptr(nodes, count=2 * N), _ptr(normals, count=2 * N),
                                         _ptr(weights, count=N), _ptr(curvature, count=N),
                                         _ptr(off, np.int64), int(n_comp), int(outer_comp), _ptr(cen),
                                         _ptr(sigma, count=2 * N), _ptr(y, count=2 * N), st))


def stokes_pair_shape_count(precision) -> int:
    n = int(lib.stokes_pair_shape_count(int(precision)))
    if n < 0:
        raise StokesError(n, "unknown precision")
    return n


def stokes_pair_shape_info(precision, variant):
    """Returns (threads, targets_per_thread, tile) of a compiled variant."""
    th, tpt, tile = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    _check(lib.stokes_pair_shape_info(int(precision), int(variant), ctypes.byref(th), ctypes.byref(tpt),
                                      ctypes.byref(tile)))
    return th.value, tpt.value, tile.value


def stokes_set_pair_shape(handle, precision, variant, ctas_per_sm=4):
    _check(lib.stokes_set_pair_shape(ctypes.c_void_p(handle), int(precision), int(variant), int(ctas_per_sm)))


def stokes_get_pair_shape(handle, precision, n_targets):
    """Returns (variant, ctas_per_sm) the handle uses for n_targets targets."""
    v, c = ctypes.c_int(0), ctypes.c_int(0)
    _check(lib.stokes_get_pair_shape(ctypes.c_void_p(handle), int(precision), ctypes.c_int64(n_targets),
                                     ctypes.byref(v), ctypes.byref(c)))
    return v.value, c.value


def stokes_autotune(handle, precision, reps=2):
    """Times every shape of the pair kernel; returns (variant, ctas_per_sm, ms)."""
    v, c, ms = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0.0)
    _check(lib.stokes_autotune(ctypes.c_void_p(handle), int(precision), int(reps), ctypes.byref(v),
                               ctypes.byref(c), ctypes.byref(ms)))
    return v.value, c.value, ms.value


def stokes_tune_cache_insert(precision, n_sources, n_targets, variant, ctas_per_sm, ms=0.0):
    _check(lib.stokes_tune_cache_insert(int(precision), ctypes.c_int64(n_sources), ctypes.c_int64(n_targets),
                                        int(variant), int(ctas_per_sm), float(ms)))


def stokes_tune_cache_lookup(precision, n_sources, n_targets):
    """Returns (variant, ctas_per_sm, ms); variant -1 when absent."""
    v, c, ms = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0.0)
    _check(lib.stokes_tune_cache_lookup(int(precision), ctypes.c_int64(n_sources), ctypes.c_int64(n_targets),
                                        ctypes.byref(v), ctypes.byref(c), ctypes.byref(ms)))
    return v.value, c.value, ms.value


def stokes_tune_cache_clear():
    _check(lib.stokes_tune_cache_clear())


def stokes_tune_cache_save(path):
    _check(lib.stokes_tune_cache_save(str(path).encode()))


def stokes_tune_cache_load(path) -> int:
    n = ctypes.c_int(0)
    _check(lib.stokes_tune_cache_load(str(path).encode(), ctypes.byref(n)))
    return n.value


def _ptr_array(handles_or_arrays, counts=None):
    """A C array of pointers (void*[]) to handles or device arrays."""
    vals = []
    for k, a in enumerate(handles_or_arrays):
        if isinstance(a, int):
            vals.append(a)
        else:
            vals.append(_ptr(a, count=None if counts is None else counts[k]).value)
    return (ctypes.c_void_p * len(vals))(*vals)


def stokes_batch_matvec(handles, n_rhs, sigma, y, precision=STOKES_FP32):
    """y[k * n_rhs + r] = A_k sigma[k * n_rhs + r] for every geometry k and
    right-hand side r (device tensors), one persistent pair launch."""
    ns = [2 * stokes_geometry_num_nodes(h) for h in handles for _ in range(n_rhs)]
    _check(lib.stokes_batch_matvec(_ptr_array(handles), len(handles), int(n_rhs), _ptr_array(sigma, ns),
                                   _ptr_array(y, ns), int(precision)))


def stokes_batch_solve(handles, n_rhs, f, sigma, tol=1e-8, restart=50, max_iter=2000,
                       precision=STOKES_MIXED_IR):
    """Lockstep flexible GMRES of all (geometry, right-hand side) systems;
    solves in place into the device tensors `sigma` (initial guesses).
    Returns (iters, relres, status) lists per system."""
    S = len(handles) * n_rhs
    ns = [2 * stokes_geometry_num_nodes(h) for h in handles for _ in range(n_rhs)]
    it = (ctypes.c_int * S)()
    rr = (ctypes.c_double * S)()
    st = (ctypes.c_int * S)()
    _check(lib.stokes_batch_solve(_ptr_array(handles), len(handles), int(n_rhs), _ptr_array(f, ns), float(tol),
                                  int(restart), int(max_iter), int(precision), _ptr_array(sigma, ns), it, rr, st))
    return list(it), list(rr), list(st)


def _fptr(a, count):
    """Address of a C-contiguous float32 (or int32) numpy array or torch tensor."""
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous() or a.element_size() != 4 or a.numel() != count:
            raise TypeError(f"expected a contiguous 4-byte tensor of {count} elements")
        return ctypes.c_void_p(a.data_ptr())
    if not isinstance(a, np.ndarray) or a.dtype not in (np.float32, np.int32) or not a.flags["C_CONTIGUOUS"]:
        raise TypeError("expected a C-contiguous float32 or int32 array")
    if a.size != count:
        raise ValueError(f"expected {count} elements, got {a.size}")
    return ctypes.c_void_p(a.ctypes.data)


COARSE_FEATURES, COARSE_OUTPUTS, COARSE_NEIGHBOURS = 35, 153, 16
COARSE_STATS = 2 * COARSE_FEATURES + 2 * COARSE_OUTPUTS


def stokes_coarse_model_num_params() -> int:
    return int(lib.stokes_coarse_model_num_params())


def stokes_coarse_model_create(params, stream=None):
    """A coarse model from initial float32 parameters; returns its handle."""
    n = stokes_coarse_model_num_params()
    h = ctypes.c_void_p()
    st = None if stream is None else ctypes.c_void_p(int(stream))
    _check(lib.stokes_coarse_model_create(_fptr(params, n), ctypes.c_int64(n), st, ctypes.byref(h)))
    return h.value


def stokes_coarse_model_destroy(model):
    _check(lib.stokes_coarse_model_destroy(ctypes.c_void_p(model)))


def stokes_coarse_model_add_geometry(model, handle):
    _check(lib.stokes_coarse_model_add_geometry(ctypes.c_void_p(model), ctypes.c_void_p(handle)))


def stokes_coarse_model_num_samples(model) -> int:
    return int(lib.stokes_coarse_model_num_samples(ctypes.c_void_p(model)))


def stokes_coarse_model_train(model, steps, lr):
    """Returns the loss of the last step."""
    loss = ctypes.c_double(0.0)
    _check(lib.stokes_coarse_model_train(ctypes.c_void_p(model), int(steps), float(lr), ctypes.byref(loss)))
    return loss.value


def stokes_coarse_model_save(model, params, stats=None):
    _check(lib.stokes_coarse_model_save(ctypes.c_void_p(model), _fptr(params, stokes_coarse_model_num_params()),
                                        None if stats is None else _fptr(stats, COARSE_STATS)))


def stokes_coarse_model_load(model, params, stats):
    _check(lib.stokes_coarse_model_load(ctypes.c_void_p(model), _fptr(params, stokes_coarse_model_num_params()),
                                        _fptr(stats, COARSE_STATS)))


def stokes_coarse_model_forward(model, x, y):
    rows = (x.numel() if hasattr(x, "numel") else x.size) // COARSE_FEATURES
    _check(lib.stokes_coarse_model_forward(ctypes.c_void_p(model), _fptr(x, rows * COARSE_FEATURES),
                                           ctypes.c_int64(rows), _fptr(y, rows * COARSE_OUTPUTS)))


def stokes_coarse_model_loss_grad(model, x, t, mask, grad):
    """Returns the loss; the gradient is written into `grad`."""
    rows = (x.numel() if hasattr(x, "numel") else x.size) // COARSE_FEATURES
    loss = ctypes.c_double(0.0)
    _check(lib.stokes_coarse_model_loss_grad(ctypes.c_void_p(model), _fptr(x, rows * COARSE_FEATURES),
                                             _fptr(t, rows * COARSE_OUTPUTS), _fptr(mask, rows * COARSE_OUTPUTS),
                                             ctypes.c_int64(rows), ctypes.byref(loss),
                                             _fptr(grad, stokes_coarse_model_num_params())))
    return loss.value


def stokes_coarse_model_adam_step(model, grad, lr):
    _check(lib.stokes_coarse_model_adam_step(ctypes.c_void_p(model), _fptr(grad, stokes_coarse_model_num_params()),
                                             float(lr)))


def stokes_coarse_features(handle, n_pores):
    """Returns (features float32 [M x 35], neighbours int32 [M x 16])."""
    x = np.zeros((n_pores, COARSE_FEATURES), dtype=np.float32)
    nb = np.zeros((n_pores, COARSE_NEIGHBOURS), dtype=np.int32)
    _check(lib.stokes_coarse_features(ctypes.c_void_p(handle), _fptr(x, x.size), _fptr(nb, nb.size)))
    return x, nb


def stokes_coarse_operator(handle, n_pores):
    """Returns (Y = A Z [2N x 3M], E = Z^T W Y [3M x 3M]) as float64 arrays."""
    n2 = 2 * stokes_geometry_num_nodes(handle)
    m = 3 * n_pores
    y = np.zeros(n2 * m)
    e = np.zeros(m * m)
    _check(lib.stokes_coarse_operator(ctypes.c_void_p(handle), _ptr(y, count=n2 * m), _ptr(e, count=m * m)))
    return y.reshape(m, n2).T, e.reshape(m, m)


def stokes_rcp_f64(x, y, stream=None):
    """y = 1 / x by the FP64 pair kernel's Newton reciprocal (device tensors)."""
    n = x.numel() if hasattr(x, "numel") else x.size
    st = None if stream is None else ctypes.c_void_p(int(stream))
    _check(lib.stokes_rcp_f64(_ptr(x, count=n), _ptr(y, count=n), ctypes.c_int64(n), st))


class Geometry:
    """Owning wrapper of a handle built from a stokes_inputs.Geometry-like
    object (nodes, normals, weights, curvature, offsets, outer_comp, centres)."""

    def __init__(self, geom, stream=None, centres=True):
        arr = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        self.N = int(geom.offsets[-1])
        self.handle = stokes_geometry_create(
            arr(geom.nodes).reshape(-1), arr(geom.normals).reshape(-1), arr(geom.weights),
            arr(geom.curvature), geom.offsets, len(geom.offsets) - 1, geom.outer_comp,
            arr(geom.centres).reshape(-1) if centres else None, stream)

    def close(self):
        if self.handle:
            stokes_geometry_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
