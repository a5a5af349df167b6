"""ctypes binding of liblbm_gb300.so (include/lbm.h), argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of its own: it converts Python / numpy / torch arguments into
pointers and sizes, calls the library, and raises ``LbmError`` on a negative
status.  Device memory and streams come from PyTorch: torch tensors are passed
by ``data_ptr()`` on their device, the stream defaults to
``torch.cuda.current_stream()``, and the library's own allocations go through
PyTorch's caching allocator (``lbm_set_allocator``).

There is no CPU fallback: if the shared library is missing, importing this
module raises ImportError.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm_gb300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("liblbm_gb300.so is not built (run paper_1303_4624_gb300.build.build()); "
                      "the LBM library has no CPU fallback")
_lib = ctypes.CDLL(LIB_PATH)

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_ESTATE, LBM_EDEVICE, LBM_EIO = \
    0, -1, -2, -3, -4, -5, -6, -7
VARIANT_AUTO, VARIANT_DIRECT, VARIANT_TMA, VARIANT_SPLIT, VARIANT_PAIR = 0, 1, 2, 3, 4
LBM_D2Q33, LBM_D3Q95 = 0, 1
LBM_FP64, LBM_FP32, LBM_FP16DEV, LBM_BF16DEV = 0, 1, 2, 3
LBM_HOST, LBM_DEVICE = 0, 1

MODELS = {"D2Q33": LBM_D2Q33, "D3Q95": LBM_D3Q95}
STORAGES = {"fp64": LBM_FP64, "fp32": LBM_FP32, "fp16": LBM_FP16DEV, "bf16": LBM_BF16DEV}
STORAGE_DTYPE = {LBM_FP64: np.float64, LBM_FP32: np.float32, LBM_FP16DEV: np.float16,
                 LBM_BF16DEV: np.uint16}
ADJ_DTYPE = {LBM_FP64: np.float64, LBM_FP32: np.float32, LBM_FP16DEV: np.float32,
             LBM_BF16DEV: np.float32}

# exported symbols of include/lbm.h
SYMBOLS = ("lbm_model_info", "lbm_set_allocator", "lbm_create", "lbm_destroy", "lbm_set_omega",
           "lbm_set_variant", "lbm_set_graph_steps", "lbm_set_fixed_ends", "lbm_set_stream",
           "lbm_init", "lbm_step", "lbm_steps_done", "lbm_set_audit_every", "lbm_save", "lbm_load",
           "lbm_moments", "lbm_audit",
           "lbm_get_populations", "lbm_set_populations", "lbm_get_raw", "lbm_set_raw",
           "lbm_record", "lbm_record_bounded", "lbm_backward", "lbm_release_record", "lbm_synchronize",
           "lbm_launch_count", "lbm_test_stall", "lbm_create_slab", "lbm_halo_info",
           "lbm_halo_pack", "lbm_halo_unpack", "lbm_halo_plan", "lbm_audit_noalloc", "lbm_equation_count", "lbm_generate_model",
           "lbm_strerror", "lbm_last_error")

_vp, _i, _i64, _d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)

_sig = {
    "lbm_model_info": (_i, [_i, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "lbm_set_allocator": (_i, [_ALLOC_FN, _FREE_FN, _vp]),
    "lbm_create": (_i, [ctypes.POINTER(_vp), _i, ctypes.POINTER(_i64), _d, _i, _vp]),
    "lbm_destroy": (_i, [_vp]),
    "lbm_set_omega": (_i, [_vp, _d]),
    "lbm_set_variant": (_i, [_vp, _i]),
    "lbm_set_graph_steps": (_i, [_vp, _i]),
    "lbm_set_fixed_ends": (_i, [_vp, _i, _i, _vp, _vp]),
    "lbm_set_stream": (_i, [_vp, _vp]),
    "lbm_init": (_i, [_vp, _vp, _vp, _vp, _i]),
    "lbm_step": (_i, [_vp, _i64]),
    "lbm_steps_done": (_i64, [_vp]),
    "lbm_set_audit_every": (_i, [_vp, _i64]),
    "lbm_save": (_i, [_vp, ctypes.c_char_p]),
    "lbm_load": (_i, [_vp, ctypes.c_char_p]),
    "lbm_moments": (_i, [_vp, _vp, _vp, _vp, _i]),
    "lbm_audit": (_i, [_vp, _vp]),
    "lbm_get_populations": (_i, [_vp, _vp, _i]),
    "lbm_set_populations": (_i, [_vp, _vp, _i]),
    "lbm_get_raw": (_i, [_vp, _vp, ctypes.c_size_t, _i]),
    "lbm_set_raw": (_i, [_vp, _vp, ctypes.c_size_t, _i]),
    "lbm_record": (_i, [_vp, _i64, _i64]),
    "lbm_record_bounded": (_i, [_vp, _i64, _i64]),
    "lbm_backward": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _i]),
    "lbm_release_record": (_i, [_vp]),
    "lbm_synchronize": (_i, [_vp]),
    "lbm_launch_count": (_i64, [_vp]),
    "lbm_test_stall": (_i, [_vp, _i64, _i64]),
    "lbm_create_slab": (_i, [ctypes.POINTER(_vp), _i, ctypes.POINTER(_i64), _d, _i, _vp]),
    "lbm_halo_info": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i64), ctypes.POINTER(_i),
                           ctypes.POINTER(ctypes.c_size_t)]),
    "lbm_halo_pack": (_i, [_vp, _i, _vp]),
    "lbm_halo_unpack": (_i, [_vp, _i, _vp]),
    "lbm_halo_plan": (_i, [_i, _i64, _i, _i, _vp, ctypes.POINTER(_i)]),
    "lbm_audit_noalloc": (_i, [_i, _i, ctypes.POINTER(_i64), _vp, ctypes.c_size_t, _vp, _vp]),
    "lbm_equation_count": (_i, [_i, _i, ctypes.POINTER(_i64)]),
    "lbm_generate_model": (_i, [_i, _i, _i, _vp, _i, _i, ctypes.POINTER(_i), _vp, _vp,
                                ctypes.POINTER(_d), ctypes.POINTER(_d), ctypes.POINTER(_i)]),
    "lbm_strerror": (ctypes.c_char_p, [_i]),
    "lbm_last_error": (ctypes.c_char_p, []),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class LbmError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = _lib.lbm_last_error().decode() or _lib.lbm_strerror(code).decode()
        super().__init__("%s failed (%d, %s): %s" % (where, code, _lib.lbm_strerror(code).decode(), msg))


def _check(rc, where):
    if rc != LBM_OK:
        raise LbmError(rc, where)
    return rc


def _ptr(a):
    """(pointer, where) of a numpy array (host) or torch tensor (host or device)."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data, LBM_HOST
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr(), (LBM_DEVICE if a.is_cuda else LBM_HOST)
    raise TypeError("expected a numpy array or a torch tensor, got %r" % type(a))


def _where(*arrays):
    ws = {w for _, w in (_ptr(a) for a in arrays if a is not None)}
    if len(ws) > 1:
        raise ValueError("mixing host and device buffers in one call")
    return ws.pop() if ws else LBM_HOST


# ------------------------------------------------------------------ allocator (PyTorch)
_alloc_refs = None


def _install_torch_allocator():
    """Route the library's device allocations through torch's caching allocator."""
    global _alloc_refs
    if _alloc_refs is not None:
        return
    import torch

    @_ALLOC_FN
    def _alloc(nbytes, stream, user):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), stream=stream or None))
        except Exception:  # out of memory -> NULL -> LBM_ENOMEM
            return None

    @_FREE_FN
    def _free(ptr, stream, user):
        torch.cuda.caching_allocator_delete(int(ptr))

    _check(_lib.lbm_set_allocator(_alloc, _free, None), "lbm_set_allocator")
    _alloc_refs = (_alloc, _free)


# ------------------------------------------------------------------ entry points
def lbm_model_info(model):
    """dict(Q, D, reach, e [Q, D] int32, w [Q], c, T0) of a model."""
    m = MODELS.get(model, model)
    Q, D, R = _i(), _i(), _i()
    _check(_lib.lbm_model_info(m, ctypes.byref(Q), ctypes.byref(D), ctypes.byref(R), None, None,
                               None, None), "lbm_model_info")
    e = np.zeros((Q.value, D.value), dtype=np.int32)
    w = np.zeros(Q.value)
    c, T0 = _d(), _d()
    _check(_lib.lbm_model_info(m, None, None, None, e.ctypes.data, w.ctypes.data, ctypes.byref(c),
                               ctypes.byref(T0)), "lbm_model_info")
    return {"Q": Q.value, "D": D.value, "reach": R.value, "e": e, "w": w, "c": c.value,
            "T0": T0.value}


def lbm_equation_count(m, D):
    """Omega(m, D): the number of moment equations of Formula 5 up to n_max = 2m (Table 1)."""
    out = _i64()
    _check(_lib.lbm_equation_count(int(m), int(D), ctypes.byref(out)), "lbm_equation_count")
    return out.value


def lbm_generate_model(D, m, reps, which=0):
    """Velocity set of order m in D dimensions from one representative per symmetry
    group (Formulas 5, 9, 10): dict(Q, e [Q, D] int32, w [Q], c, residual, nsolutions).
    Runs on the host; needs no GPU."""
    reps = np.ascontiguousarray(np.asarray(reps, dtype=np.int32).reshape(-1, int(D)))
    Q, c, res, nsol = _i(), _d(), _d(), _i()
    rc = _lib.lbm_generate_model(int(D), int(m), reps.shape[0], reps.ctypes.data, int(which), 0,
                                 ctypes.byref(Q), None, None, ctypes.byref(c), ctypes.byref(res),
                                 ctypes.byref(nsol))
    if rc != LBM_OK and Q.value == 0:
        raise LbmError(rc, "lbm_generate_model")
    e = np.zeros((Q.value, int(D)), dtype=np.int32)
    w = np.zeros(Q.value)
    _check(_lib.lbm_generate_model(int(D), int(m), reps.shape[0], reps.ctypes.data, int(which),
                                   Q.value, ctypes.byref(Q), e.ctypes.data, w.ctypes.data,
                                   ctypes.byref(c), ctypes.byref(res), ctypes.byref(nsol)),
           "lbm_generate_model")
    return {"Q": Q.value, "e": e, "w": w, "c": c.value, "residual": res.value,
            "nsolutions": nsol.value}


def lbm_create(model, dims, omega, storage, stream=None, torch_allocator=True):
    """Create a context; returns its handle (int).  stream: torch.cuda.Stream, raw handle or None
    (torch's current stream)."""
    import torch
    if torch_allocator:
        _install_torch_allocator()
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    elif hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    h = _vp()
    d = (_i64 * 3)(*[int(x) for x in dims])
    _check(_lib.lbm_create(ctypes.byref(h), MODELS.get(model, model), d, float(omega),
                           STORAGES.get(storage, storage), stream), "lbm_create")
    return h.value


def lbm_create_slab(model, dims, omega, storage, stream=None, torch_allocator=True):
    """Create the context of one slab of a grid split along its slowest axis; dims are
    the slab's interior extents (see include/lbm.h).  Returns its handle."""
    import torch
    if torch_allocator:
        _install_torch_allocator()
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    elif hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    h = _vp()
    d = (_i64 * 3)(*[int(x) for x in dims])
    _check(_lib.lbm_create_slab(ctypes.byref(h), MODELS.get(model, model), d, float(omega),
                                STORAGES.get(storage, storage), stream), "lbm_create_slab")
    return h.value


def lbm_halo_info(ctx):
    """dict(ghost, interior, segments, face_bytes) of a slab context."""
    g, n, sg, b = _i(), _i64(), _i(), ctypes.c_size_t()
    _check(_lib.lbm_halo_info(ctx, ctypes.byref(g), ctypes.byref(n), ctypes.byref(sg), ctypes.byref(b)),
           "lbm_halo_info")
    return {"ghost": g.value, "interior": n.value, "segments": sg.value, "face_bytes": b.value}


def lbm_halo_pack(ctx, face, buf):
    p, w = _ptr(buf)
    if w != LBM_DEVICE:
        raise ValueError("halo messages live in device memory")
    _check(_lib.lbm_halo_pack(ctx, int(face), p), "lbm_halo_pack")


def lbm_halo_unpack(ctx, face, buf):
    p, w = _ptr(buf)
    if w != LBM_DEVICE:
        raise ValueError("halo messages live in device memory")
    _check(_lib.lbm_halo_unpack(ctx, int(face), p), "lbm_halo_unpack")


def lbm_halo_plan(model, interior, face, send):
    """[count, 2] int32 array of (direction, local plane) segments, in message order
    (host only, needs no GPU)."""
    m = MODELS.get(model, model)
    n = _i(0)
    _check(_lib.lbm_halo_plan(m, int(interior), int(face), int(bool(send)), None, ctypes.byref(n)),
           "lbm_halo_plan")
    out = np.zeros((n.value, 2), dtype=np.int32)
    _check(_lib.lbm_halo_plan(m, int(interior), int(face), int(bool(send)), out.ctypes.data,
                              ctypes.byref(n)), "lbm_halo_plan")
    return out


def lbm_destroy(ctx):
    _check(_lib.lbm_destroy(ctx), "lbm_destroy")


def lbm_set_omega(ctx, omega):
    _check(_lib.lbm_set_omega(ctx, float(omega)), "lbm_set_omega")


def lbm_set_variant(ctx, variant):
    _check(_lib.lbm_set_variant(ctx, int(variant)), "lbm_set_variant")


def lbm_set_audit_every(ctx, k):
    """lbm_step audits every k steps and stops with LBM_EUNSTABLE on non-finite values."""
    _check(_lib.lbm_set_audit_every(ctx, int(k)), "lbm_set_audit_every")


def lbm_save(ctx, path):
    _check(_lib.lbm_save(ctx, os.fsencode(path)), "lbm_save")


def lbm_load(ctx, path):
    _check(_lib.lbm_load(ctx, os.fsencode(path)), "lbm_load")


def lbm_set_graph_steps(ctx, steps):
    """Steps per CUDA-graph replay in lbm_step (0: direct launches; default 32)."""
    _check(_lib.lbm_set_graph_steps(ctx, int(steps)), "lbm_set_graph_steps")


def lbm_set_fixed_ends(ctx, axis, width, lo=None, hi=None):
    """Hold the first / last ``width`` planes along ``axis`` at the equilibrium of the
    states lo, hi = (rho, U_1..U_D, T) (lattice units); width 0 switches them off."""
    if width == 0:
        _check(_lib.lbm_set_fixed_ends(ctx, int(axis), 0, None, None), "lbm_set_fixed_ends")
        return
    a = np.ascontiguousarray(lo, dtype=np.float64)
    b = np.ascontiguousarray(hi, dtype=np.float64)
    _check(_lib.lbm_set_fixed_ends(ctx, int(axis), int(width), a.ctypes.data, b.ctypes.data),
           "lbm_set_fixed_ends")


def lbm_set_stream(ctx, stream):
    if hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    _check(_lib.lbm_set_stream(ctx, stream), "lbm_set_stream")


def lbm_init(ctx, rho, U, T):
    w = _where(rho, U, T)
    _check(_lib.lbm_init(ctx, _ptr(rho)[0], _ptr(U)[0], _ptr(T)[0], w), "lbm_init")


def lbm_step(ctx, n=1):
    _check(_lib.lbm_step(ctx, int(n)), "lbm_step")


def lbm_steps_done(ctx):
    return int(_lib.lbm_steps_done(ctx))


def lbm_moments(ctx, rho=None, U=None, T=None):
    w = _where(rho, U, T)
    _check(_lib.lbm_moments(ctx, _ptr(rho)[0], _ptr(U)[0], _ptr(T)[0], w), "lbm_moments")


def lbm_audit(ctx, check=False):
    """dict of the conservation audit; raises on non-finite populations only if check."""
    out = np.zeros(8)
    rc = _lib.lbm_audit(ctx, out.ctypes.data)
    if rc != LBM_OK and (check or rc != LBM_EUNSTABLE):
        raise LbmError(rc, "lbm_audit")
    return {"mass": out[0], "momentum": out[1:4].copy(), "energy": out[4],
            "min_f_over_w": out[5], "nonfinite": int(out[6]), "cells": int(out[7]),
            "status": rc}


def lbm_get_populations(ctx, f):
    p, w = _ptr(f)
    _check(_lib.lbm_get_populations(ctx, p, w), "lbm_get_populations")


def lbm_set_populations(ctx, f):
    p, w = _ptr(f)
    _check(_lib.lbm_set_populations(ctx, p, w), "lbm_set_populations")


def _nbytes(a):
    return a.nbytes if isinstance(a, np.ndarray) else a.numel() * a.element_size()


def lbm_get_raw(ctx, h):
    p, w = _ptr(h)
    _check(_lib.lbm_get_raw(ctx, p, _nbytes(h), w), "lbm_get_raw")


def lbm_set_raw(ctx, h):
    p, w = _ptr(h)
    _check(_lib.lbm_set_raw(ctx, p, _nbytes(h), w), "lbm_set_raw")


def lbm_record(ctx, nsteps, ckpt_every):
    _check(_lib.lbm_record(ctx, int(nsteps), int(ckpt_every)), "lbm_record")


def lbm_record_bounded(ctx, nsteps, max_states):
    _check(_lib.lbm_record_bounded(ctx, int(nsteps), int(max_states)), "lbm_record_bounded")


def lbm_backward(ctx, dL_drhoN, dL_drho0=None, dL_dU0=None, dL_dT0=None):
    """Reverse sweep; fills the given gradient buffers and returns dL/domega."""
    w = _where(dL_drhoN, dL_drho0, dL_dU0, dL_dT0)
    dom = _d()
    _check(_lib.lbm_backward(ctx, _ptr(dL_drhoN)[0], _ptr(dL_drho0)[0], _ptr(dL_dU0)[0],
                             _ptr(dL_dT0)[0], ctypes.byref(dom), w), "lbm_backward")
    return dom.value


def lbm_release_record(ctx):
    _check(_lib.lbm_release_record(ctx), "lbm_release_record")


def lbm_synchronize(ctx):
    _check(_lib.lbm_synchronize(ctx), "lbm_synchronize")


def lbm_launch_count(ctx):
    return int(_lib.lbm_launch_count(ctx))


def lbm_test_stall(ctx, chunk, limit_ns):
    """Test hook: the next TMA launch skips one chunk's copies; its bounded wait runs out."""
    _check(_lib.lbm_test_stall(ctx, int(chunk), int(limit_ns)), "lbm_test_stall")


def lbm_audit_noalloc(model, storage, dims, h, out, stream=None):
    """Audit of a caller-owned device population array into a caller-owned device
    buffer of 8 doubles, without any device allocation (see include/lbm.h).

    h and out are torch tensors; the library itself refuses host memory, another
    device's memory and an h smaller than the grid's populations (LBM_EINVAL)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    elif hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    if out.dtype != torch.float64 or out.numel() < 8:
        raise ValueError("out must be a float64 tensor of at least 8 elements")
    d = (_i64 * 3)(*[int(x) for x in dims])
    _check(_lib.lbm_audit_noalloc(MODELS.get(model, model), STORAGES.get(storage, storage), d,
                                  _ptr(h)[0], _nbytes(h), _ptr(out)[0], stream),
           "lbm_audit_noalloc")


def lbm_strerror(code):
    return _lib.lbm_strerror(code).decode()


def lbm_last_error():
    return _lib.lbm_last_error().decode()


# ------------------------------------------------------------------ convenience wrapper
class Lattice:
    """Owns one context; thin object form of the entry points above."""

    def __init__(self, model, dims, omega, storage="fp32", stream=None):
        self.info = lbm_model_info(model)
        self.model, self.storage = model, STORAGES.get(storage, storage)
        self.dims = tuple(int(x) for x in dims)
        self.cells = self.dims[0] * self.dims[1] * self.dims[2]
        self.omega = omega
        self.ctx = lbm_create(model, dims, omega, storage, stream)

    def close(self):
        if self.ctx:
            lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        nx, ny, nz = self.dims
        return (nz, ny, nx)

    def init(self, rho, U, T):
        lbm_init(self.ctx, rho, U, T)

    def step(self, n=1):
        lbm_step(self.ctx, n)

    def moments(self):
        D = self.info["D"]
        rho = np.zeros(self.shape)
        U = np.zeros((D,) + self.shape)
        T = np.zeros(self.shape)
        lbm_moments(self.ctx, rho, U, T)
        return rho, U, T

    def populations(self):
        f = np.zeros((self.info["Q"],) + self.shape)
        lbm_get_populations(self.ctx, f)
        return f

    def set_populations(self, f):
        lbm_set_populations(self.ctx, np.ascontiguousarray(f, dtype=np.float64))

    def raw(self):
        h = np.zeros((self.info["Q"],) + self.shape, dtype=STORAGE_DTYPE[self.storage])
        lbm_get_raw(self.ctx, h)
        return h

    def set_raw(self, h):
        lbm_set_raw(self.ctx, np.ascontiguousarray(h))

    def audit(self):
        return lbm_audit(self.ctx)

    def save(self, path):
        lbm_save(self.ctx, path)

    def load(self, path):
        lbm_load(self.ctx, path)

    def synchronize(self):
        lbm_synchronize(self.ctx)
