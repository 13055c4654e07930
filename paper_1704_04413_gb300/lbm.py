"""Thin ctypes binding of liblbm (include/lbm.h): same names, argument marshalling only.

Every computation runs in the library's CUDA kernels.  Arrays may be numpy
float64 arrays (host) or CUDA torch tensors of dtype float64 (device; passed by
data_ptr with on_device=1).  Importing this module loads the in-tree
liblbm.so and raises if it is missing: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm.so")

D2Q9, D2V17, D2V37 = 0, 1, 2
BGK, PR, RR = 0, 1, 2
PERIODIC, ZERO_GRADIENT = 0, 1
A1_PROJECTION, A1_FINITE_DIFFERENCE = 0, 1
A1_SOURCES = {"projection": A1_PROJECTION, "fd": A1_FINITE_DIFFERENCE}
F64, F32, F16_SHIFT, BF16_SHIFT, I16_SHIFT = 0, 1, 2, 3, 4
OK, EINVAL, ENOMEM, ECUDA, EUNSTABLE, ETIMEOUT, EIO = 0, -1, -2, -3, -4, -5, -6

LATTICES = {"D2Q9": D2Q9, "D2V17": D2V17, "D2V37": D2V37}
COLLISIONS = {"bgk": BGK, "pr": PR, "rr": RR}
STORAGES = {"f64": F64, "f32": F32, "f16": F16_SHIFT, "bf16": BF16_SHIFT, "i16": I16_SHIFT}
EXPORTED = ["lbm_lattice_info", "lbm_create", "lbm_destroy", "lbm_init", "lbm_step", "lbm_moments",
            "lbm_conservation", "lbm_diagnostics", "lbm_get_populations", "lbm_set_populations",
            "lbm_step_count", "lbm_tau", "lbm_save", "lbm_load", "lbm_strerror", "lbm_last_error",
            "lbm_test_inject_copy_fault",
            "lbm_conservation_noalloc", "lbm_batch_create", "lbm_batch_destroy", "lbm_batch_context",
            "lbm_batch_step", "lbm_batch_set_launch", "lbm_batch_get_launch", "lbm_batch_autotune",
            "lbm_closure_create", "lbm_closure_destroy", "lbm_closure_set_weights", "lbm_closure_get_weights",
            "lbm_closure_forward", "lbm_closure_train_step", "lbm_closure_gradients", "lbm_closure_features",
            "lbm_closure_coarsen", "lbm_step_closure", "lbm_closure_apply"]


class lbm_params(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_int), ("hermite_order", ctypes.c_int), ("reg_order", ctypes.c_int),
                ("collision", ctypes.c_int), ("thermal", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nu", ctypes.c_double), ("tau", ctypes.c_double), ("bc_x", ctypes.c_int), ("bc_y", ctypes.c_int),
                ("storage", ctypes.c_int), ("compute", ctypes.c_int), ("rho0", ctypes.c_double),
                ("store_scale", ctypes.c_double), ("stream", ctypes.c_void_p), ("tau3", ctypes.c_double),
                ("tau4", ctypes.c_double), ("a1_source", ctypes.c_int)]


class LbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (msg, code, lbm_strerror(code)))
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load liblbm.so (raises OSError when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError("liblbm.so not built at %s (run paper_1704_04413_gb300/build.py)" % path)
    lib = ctypes.CDLL(path)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    sig = {
        "lbm_lattice_info": (ctypes.c_int, [ctypes.c_int, ip, ip, ip, dp, dp]),
        "lbm_create": (ctypes.c_int, [ctypes.POINTER(lbm_params), ctypes.POINTER(vp)]),
        "lbm_destroy": (None, [vp]),
        "lbm_init": (ctypes.c_int, [vp, vp, vp, vp, vp, vp, ctypes.c_int]),
        "lbm_step": (ctypes.c_int, [vp, ctypes.c_int]),
        "lbm_moments": (ctypes.c_int, [vp, vp, vp, vp, vp, ctypes.c_int]),
        "lbm_conservation": (ctypes.c_int, [vp, dp]),
        "lbm_diagnostics": (ctypes.c_int, [vp, dp]),
        "lbm_get_populations": (ctypes.c_int, [vp, vp, ctypes.c_int]),
        "lbm_set_populations": (ctypes.c_int, [vp, vp, ctypes.c_int]),
        "lbm_step_count": (ctypes.c_longlong, [vp]),
        "lbm_test_inject_copy_fault": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_double]),
        "lbm_tau": (ctypes.c_double, [vp]),
        "lbm_save": (ctypes.c_int, [vp, ctypes.c_char_p]),
        "lbm_load": (ctypes.c_int, [vp, ctypes.c_char_p]),
        "lbm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "lbm_last_error": (ctypes.c_char_p, [vp]),
        "lbm_conservation_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int,
                                                    ctypes.c_int, ctypes.c_double, ctypes.c_double, vp, vp]),
        "lbm_batch_create": (ctypes.c_int, [ctypes.POINTER(lbm_params), ctypes.c_int, ctypes.POINTER(vp)]),
        "lbm_batch_destroy": (None, [vp]),
        "lbm_batch_context": (vp, [vp, ctypes.c_int]),
        "lbm_batch_step": (ctypes.c_int, [vp, ctypes.c_int]),
        "lbm_batch_set_launch": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
        "lbm_batch_get_launch": (ctypes.c_int, [vp, ip, ip, ip]),
        "lbm_batch_autotune": (ctypes.c_int, [vp, ctypes.c_int, dp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a):
    """(address, on_device) of a numpy array or a torch tensor (None -> NULL)."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("arrays must be C-contiguous float64")
        return a.ctypes.data, 0
    if hasattr(a, "data_ptr"):
        if str(a.dtype) != "torch.float64" or not a.is_contiguous():
            raise TypeError("tensors must be contiguous float64")
        return a.data_ptr(), 1 if a.is_cuda else 0
    raise TypeError("unsupported array type %r" % type(a))


def _check(rc, ctx=None, what="liblbm"):
    if rc != OK:
        detail = load().lbm_last_error(ctx).decode() if ctx else ""
        raise LbmError(rc, "%s: %s" % (what, detail) if detail else what)
    return rc


def lbm_strerror(code: int) -> str:
    return load().lbm_strerror(code).decode()


def lbm_last_error(ctx) -> str:
    return load().lbm_last_error(ctx).decode()


def lbm_lattice_info(lattice):
    lat = LATTICES.get(lattice, lattice)
    V = ctypes.c_int()
    cx = (ctypes.c_int * 64)()
    cy = (ctypes.c_int * 64)()
    w = (ctypes.c_double * 64)()
    cs2 = ctypes.c_double()
    _check(load().lbm_lattice_info(lat, ctypes.byref(V), cx, cy, w, ctypes.byref(cs2)), what="lbm_lattice_info")
    n = V.value
    return n, np.array(cx[:n]), np.array(cy[:n]), np.array(w[:n]), cs2.value


def make_params(lattice="D2Q9", nx=64, ny=64, tau=0.0, nu=0.0, collision="rr", hermite_order=2, reg_order=0,
                thermal=False, bc_x=PERIODIC, bc_y=PERIODIC, storage="f32", rho0=0.0, store_scale=0.0,
                stream=None, tau3=0.0, tau4=0.0, a1_source=0) -> lbm_params:
    st = STORAGES.get(storage, storage)
    compute = F64 if st == F64 else F32
    return lbm_params(LATTICES.get(lattice, lattice), hermite_order, reg_order,
                      COLLISIONS.get(collision, collision), int(thermal), nx, ny, float(nu), float(tau), bc_x, bc_y,
                      st, compute, float(rho0), float(store_scale), stream, float(tau3), float(tau4),
                      A1_SOURCES.get(a1_source, a1_source))


def lbm_create(params: lbm_params):
    ctx = ctypes.c_void_p()
    _check(load().lbm_create(ctypes.byref(params), ctypes.byref(ctx)), what="lbm_create")
    return ctx


def lbm_destroy(ctx) -> None:
    load().lbm_destroy(ctx)


def lbm_init(ctx, rho, ux, uy, theta=None, grad_u=None):
    ptrs = [_ptr(a) for a in (rho, ux, uy, theta, grad_u)]
    flags = {p[1] for p in ptrs if p[1] is not None}
    if len(flags) != 1:
        raise TypeError("mix of host and device arrays")
    return _check(load().lbm_init(ctx, *[p[0] for p in ptrs], flags.pop()), ctx, "lbm_init")


def lbm_step(ctx, n: int = 1):
    return _check(load().lbm_step(ctx, int(n)), ctx, "lbm_step")


def lbm_moments(ctx, rho=None, ux=None, uy=None, theta=None):
    ptrs = [_ptr(a) for a in (rho, ux, uy, theta)]
    flags = {p[1] for p in ptrs if p[1] is not None}
    if len(flags) != 1:
        raise TypeError("mix of host and device arrays")
    return _check(load().lbm_moments(ctx, *[p[0] for p in ptrs], flags.pop()), ctx, "lbm_moments")


def lbm_conservation(ctx, raise_unstable=True) -> np.ndarray:
    out = np.zeros(4)
    rc = load().lbm_conservation(ctx, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != EUNSTABLE or raise_unstable:
        _check(rc, ctx, "lbm_conservation")
    return out


def lbm_diagnostics(ctx, raise_unstable=True) -> np.ndarray:
    out = np.zeros(4)
    rc = load().lbm_diagnostics(ctx, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != EUNSTABLE or raise_unstable:
        _check(rc, ctx, "lbm_diagnostics")
    return out


def lbm_get_populations(ctx, f):
    p, dev = _ptr(f)
    return _check(load().lbm_get_populations(ctx, p, dev), ctx, "lbm_get_populations")


def lbm_set_populations(ctx, f):
    p, dev = _ptr(f)
    return _check(load().lbm_set_populations(ctx, p, dev), ctx, "lbm_set_populations")


def lbm_step_count(ctx) -> int:
    return load().lbm_step_count(ctx)


def lbm_test_inject_copy_fault(ctx, block: int, wait_seconds: float):
    """Testing hook of the staged step kernels' failure path (lbm.h): block >= 0 makes that block's last
    copies never issue, so its bounded wait runs out after wait_seconds; -1 turns it off."""
    return _check(load().lbm_test_inject_copy_fault(ctx, int(block), float(wait_seconds)), ctx,
                  "lbm_test_inject_copy_fault")


def lbm_tau(ctx) -> float:
    return load().lbm_tau(ctx)


def lbm_save(ctx, path: str):
    return _check(load().lbm_save(ctx, path.encode()), ctx, "lbm_save")


def lbm_load(ctx, path: str):
    return _check(load().lbm_load(ctx, path.encode()), ctx, "lbm_load")


_STORAGE_BYTES = {F64: 8, F32: 4, F16_SHIFT: 2, BF16_SHIFT: 2, I16_SHIFT: 2}


def lbm_conservation_noalloc(lattice, storage, f, nx, ny, pitch, out4, rho0=0.0, store_scale=0.0, stream=None):
    """Allocation-free conservation sums: f and out4 are device buffers the caller owns, written on `stream`.

    Torch tensors are checked before the call: both on the current CUDA device and contiguous, f with the
    element size of `storage` and at least V * ny * pitch elements, out4 float64 with at least 4.  Raw
    integer device addresses are passed through unchecked (the library still refuses host addresses)."""
    lat = LATTICES.get(lattice, lattice)
    st = STORAGES.get(storage, storage)
    if st not in _STORAGE_BYTES:
        raise ValueError("unknown storage %r" % (storage,))
    if hasattr(f, "data_ptr") or hasattr(out4, "data_ptr"):
        if not (hasattr(f, "data_ptr") and hasattr(out4, "data_ptr")):
            raise TypeError("f and out4 must both be tensors or both be device addresses")
        import torch
        dev = torch.cuda.current_device()
        for name, t in (("f", f), ("out4", out4)):
            if not t.is_cuda or t.device.index != dev:
                raise TypeError("%s must be a CUDA tensor on the current device (cuda:%d)" % (name, dev))
            if not t.is_contiguous():
                raise TypeError("%s must be contiguous" % name)
        if f.element_size() != _STORAGE_BYTES[st]:
            raise TypeError("f has %d-byte elements; storage %r stores %d" % (f.element_size(), storage,
                                                                            _STORAGE_BYTES[st]))
        V = lbm_lattice_info(lat)[0]
        if nx < 1 or ny < 1 or pitch < nx or f.numel() < V * ny * pitch:
            raise ValueError("f holds %d elements; V * ny * pitch = %d" % (f.numel(), V * ny * pitch))
        if out4.dtype != torch.float64 or out4.numel() < 4:
            raise TypeError("out4 must be a float64 tensor of at least 4 elements")
        fp, op = f.data_ptr(), out4.data_ptr()
    else:
        fp, op = int(f), int(out4)
    rc = load().lbm_conservation_noalloc(lat, st, fp, nx, ny, pitch, rho0, store_scale, op, stream)
    return _check(rc, None, "lbm_conservation_noalloc")


def lbm_batch_create(params_list):
    arr = (lbm_params * len(params_list))(*params_list)
    b = ctypes.c_void_p()
    _check(load().lbm_batch_create(arr, len(params_list), ctypes.byref(b)), what="lbm_batch_create")
    return b


def lbm_batch_destroy(b) -> None:
    load().lbm_batch_destroy(b)


def lbm_batch_context(b, i: int):
    p = load().lbm_batch_context(b, int(i))
    if not p:
        raise LbmError(EINVAL, "lbm_batch_context: index out of range")
    return ctypes.c_void_p(p)


def lbm_batch_step(b, n: int = 1):
    return _check(load().lbm_batch_step(b, int(n)), what="lbm_batch_step")


def lbm_batch_set_launch(b, threads: int, rows: int, blocks_per_sm: int):
    return _check(load().lbm_batch_set_launch(b, threads, rows, blocks_per_sm), what="lbm_batch_set_launch")


def lbm_batch_get_launch(b):
    t, r, q = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().lbm_batch_get_launch(b, ctypes.byref(t), ctypes.byref(r), ctypes.byref(q)), what="lbm_batch_get_launch")
    return t.value, r.value, q.value


def lbm_batch_autotune(b, steps: int = 3) -> float:
    ms = ctypes.c_double()
    _check(load().lbm_batch_autotune(b, int(steps), ctypes.byref(ms)), what="lbm_batch_autotune")
    return ms.value


# ---------------------------------------------------------------------------
# Learned closure
# ---------------------------------------------------------------------------
CLOSURE_IN, CLOSURE_HID, CLOSURE_OUT, CLOSURE_NPARAM = 32, 64, 8, 10952


def _dptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_cuda or not a.is_contiguous():
            raise TypeError("closure arrays must be contiguous CUDA tensors")
        return a.data_ptr()
    return int(a)


def _closure_sigs(lib):
    vp, fp, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_float), ctypes.c_double
    sig = {
        "lbm_closure_create": (ctypes.c_int, [ctypes.POINTER(vp)]),
        "lbm_closure_destroy": (None, [vp]),
        "lbm_closure_set_weights": (ctypes.c_int, [vp, fp, ctypes.c_int]),
        "lbm_closure_get_weights": (ctypes.c_int, [vp, fp, ctypes.c_int]),
        "lbm_closure_forward": (ctypes.c_int, [vp, vp, ctypes.c_int, vp, vp]),
        "lbm_closure_train_step": (ctypes.c_int, [vp, vp, vp, ctypes.c_int, ctypes.c_float, fp, vp]),
        "lbm_closure_gradients": (ctypes.c_int, [vp, vp, vp, ctypes.c_int, fp, fp]),
        "lbm_closure_features": (ctypes.c_int, [vp, vp, vp, ctypes.c_int, ctypes.c_int, dp, vp, vp]),
        "lbm_closure_coarsen": (ctypes.c_int, [vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, vp, vp, vp,
                                               vp, vp]),
        "lbm_step_closure": (ctypes.c_int, [vp, vp, dp, ctypes.c_int]),
        "lbm_closure_apply": (ctypes.c_int, [vp, vp, dp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args


_closure_ready = False


def _cl():
    global _closure_ready
    lib = load()
    if not _closure_ready:
        _closure_sigs(lib)
        _closure_ready = True
    return lib


def _fptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def lbm_closure_create():
    c = ctypes.c_void_p()
    _check(_cl().lbm_closure_create(ctypes.byref(c)), what="lbm_closure_create")
    return c


def lbm_closure_destroy(cl) -> None:
    _cl().lbm_closure_destroy(cl)


def lbm_closure_set_weights(cl, w):
    w = np.ascontiguousarray(w, dtype=np.float32)
    return _check(_cl().lbm_closure_set_weights(cl, _fptr(w), w.size), what="lbm_closure_set_weights")


def lbm_closure_get_weights(cl) -> np.ndarray:
    w = np.empty(CLOSURE_NPARAM, dtype=np.float32)
    _check(_cl().lbm_closure_get_weights(cl, _fptr(w), w.size), what="lbm_closure_get_weights")
    return w


def lbm_closure_forward(cl, x, n, y, stream=None):
    return _check(_cl().lbm_closure_forward(cl, _dptr(x), int(n), _dptr(y), stream), what="lbm_closure_forward")


def lbm_closure_train_step(cl, x, y, n, lr, stream=None) -> float:
    loss = np.zeros(1, dtype=np.float32)
    _check(_cl().lbm_closure_train_step(cl, _dptr(x), _dptr(y), int(n), float(lr), _fptr(loss), stream),
           what="lbm_closure_train_step")
    return float(loss[0])


def lbm_closure_gradients(cl, x, y, n):
    g = np.empty(CLOSURE_NPARAM, dtype=np.float32)
    loss = np.zeros(1, dtype=np.float32)
    _check(_cl().lbm_closure_gradients(cl, _dptr(x), _dptr(y), int(n), _fptr(g), _fptr(loss)),
           what="lbm_closure_gradients")
    return g, float(loss[0])


def lbm_closure_features(rho, ux, uy, nx, ny, u0, x, stream=None):
    return _check(_cl().lbm_closure_features(_dptr(rho), _dptr(ux), _dptr(uy), nx, ny, float(u0), _dptr(x), stream),
                  what="lbm_closure_features")


def lbm_closure_coarsen(rho, ux, uy, nx, ny, factor, u0, rho_c, ux_c, uy_c, y, stream=None):
    return _check(_cl().lbm_closure_coarsen(_dptr(rho), _dptr(ux), _dptr(uy), nx, ny, int(factor), float(u0),
                                            _dptr(rho_c), _dptr(ux_c), _dptr(uy_c), _dptr(y), stream),
                  what="lbm_closure_coarsen")


def lbm_step_closure(ctx, cl, u0, n=1):
    return _check(_cl().lbm_step_closure(ctx, cl, float(u0), int(n)), ctx, "lbm_step_closure")


def lbm_closure_apply(ctx, y, u0):
    return _check(_cl().lbm_closure_apply(ctx, _dptr(y), float(u0)), ctx, "lbm_closure_apply")


# ---------------------------------------------------------------------------
# Three-dimensional lattices (include/lbm3.h)
# ---------------------------------------------------------------------------
D3Q19, D3Q27, D3V39, D3Q103 = 10, 11, 12, 13
LATTICES3 = {"D3Q19": D3Q19, "D3Q27": D3Q27, "D3V39": D3V39, "D3Q103": D3Q103}
EXPORTED3 = ["lbm3_lattice_info", "lbm3_create", "lbm3_destroy", "lbm3_init", "lbm3_step", "lbm3_moments",
             "lbm3_conservation", "lbm3_get_populations", "lbm3_set_populations", "lbm3_tau",
             "lbm3_test_inject_copy_fault"]


class lbm3_params(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_int), ("hermite_order", ctypes.c_int), ("reg_order", ctypes.c_int),
                ("collision", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("nu", ctypes.c_double), ("tau", ctypes.c_double), ("bc_x", ctypes.c_int), ("bc_y", ctypes.c_int),
                ("bc_z", ctypes.c_int), ("storage", ctypes.c_int), ("compute", ctypes.c_int),
                ("rho0", ctypes.c_double), ("store_scale", ctypes.c_double), ("stream", ctypes.c_void_p)]


_lbm3_ready = False


def _l3():
    global _lbm3_ready
    lib = load()
    if not _lbm3_ready:
        vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
        sig = {
            "lbm3_lattice_info": (ctypes.c_int, [ctypes.c_int, ip, ip, ip, ip, dp, dp]),
            "lbm3_create": (ctypes.c_int, [ctypes.POINTER(lbm3_params), ctypes.POINTER(vp)]),
            "lbm3_destroy": (None, [vp]),
            "lbm3_init": (ctypes.c_int, [vp, vp, vp, vp, ctypes.c_int]),
            "lbm3_step": (ctypes.c_int, [vp, ctypes.c_int]),
            "lbm3_moments": (ctypes.c_int, [vp, vp, vp, ctypes.c_int]),
            "lbm3_conservation": (ctypes.c_int, [vp, dp]),
            "lbm3_get_populations": (ctypes.c_int, [vp, vp, ctypes.c_int]),
            "lbm3_set_populations": (ctypes.c_int, [vp, vp, ctypes.c_int]),
            "lbm3_tau": (ctypes.c_double, [vp]),
            "lbm3_test_inject_copy_fault": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_double]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lbm3_ready = True
    return lib


def lbm3_lattice_info(lattice):
    """(V, cx, cy, cz, w, cs2) of a 3D lattice, in the library's velocity order."""
    V = ctypes.c_int()
    cx, cy, cz = (np.zeros(128, dtype=np.int32) for _ in range(3))
    w = np.zeros(128)
    cs2 = ctypes.c_double()
    ip = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    _check(_l3().lbm3_lattice_info(LATTICES3.get(lattice, lattice), ctypes.byref(V), ip(cx), ip(cy), ip(cz),
                                   w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(cs2)),
           what="lbm3_lattice_info")
    n = V.value
    return n, cx[:n].copy(), cy[:n].copy(), cz[:n].copy(), w[:n].copy(), cs2.value


def make_params3(lattice="D3Q19", nx=16, ny=16, nz=16, tau=0.0, nu=0.0, collision="rr", hermite_order=2,
                 reg_order=0, bc=(PERIODIC, PERIODIC, PERIODIC), storage="f32", rho0=0.0, store_scale=0.0,
                 stream=None) -> lbm3_params:
    st = STORAGES.get(storage, storage)
    compute = F64 if st == F64 else F32
    return lbm3_params(LATTICES3.get(lattice, lattice), hermite_order, reg_order,
                       COLLISIONS.get(collision, collision), nx, ny, nz, float(nu), float(tau), bc[0], bc[1], bc[2],
                       st, compute, float(rho0), float(store_scale), stream)


def lbm3_create(p: lbm3_params):
    c = ctypes.c_void_p()
    _check(_l3().lbm3_create(ctypes.byref(p), ctypes.byref(c)), what="lbm3_create")
    return c


def lbm3_destroy(ctx) -> None:
    _l3().lbm3_destroy(ctx)


def _ptrs(*arrays):
    ptrs = [_ptr(a) for a in arrays]
    flags = {p[1] for p in ptrs if p[1] is not None}
    if len(flags) != 1:
        raise TypeError("mix of host and device arrays")
    return [p[0] for p in ptrs], flags.pop()


def lbm3_init(ctx, rho, u, grad=None):
    """rho [nz][ny][nx], u [3][nz][ny][nx], grad [9][nz][ny][nx] (component 3a + b = d u_a / d x_b) or None."""
    (pr, pu, pg), dev = _ptrs(rho, u, grad)
    return _check(_l3().lbm3_init(ctx, pr, pu, pg, dev), what="lbm3_init")


def lbm3_step(ctx, n=1):
    return _check(_l3().lbm3_step(ctx, int(n)), what="lbm3_step")


def lbm3_moments(ctx, rho=None, u=None):
    (pr, pu), dev = _ptrs(rho, u)
    return _check(_l3().lbm3_moments(ctx, pr, pu, dev), what="lbm3_moments")


def lbm3_conservation(ctx, raise_unstable=True) -> np.ndarray:
    out = np.zeros(4)
    rc = _l3().lbm3_conservation(ctx, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != EUNSTABLE or raise_unstable:
        _check(rc, what="lbm3_conservation")
    return out


def lbm3_get_populations(ctx, f):
    (p,), dev = _ptrs(f)
    return _check(_l3().lbm3_get_populations(ctx, p, dev), what="lbm3_get_populations")


def lbm3_set_populations(ctx, f):
    (p,), dev = _ptrs(f)
    return _check(_l3().lbm3_set_populations(ctx, p, dev), what="lbm3_set_populations")


def lbm3_tau(ctx) -> float:
    return _l3().lbm3_tau(ctx)


def lbm3_test_inject_copy_fault(ctx, block: int, wait_seconds: float):
    """Testing hook of the staged 3D kernel's failure path (lbm3.h)."""
    return _check(_l3().lbm3_test_inject_copy_fault(ctx, int(block), float(wait_seconds)),
                  what="lbm3_test_inject_copy_fault")
