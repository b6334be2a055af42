"""Python binding of libovl.so, the GB300 library for x = sign(H_W(mu)) b.

Thin ctypes marshalling over the C ABI declared in include/ovl.h: every function here has
the C name, converts arguments (numpy arrays for host buffers, torch CUDA tensors for
device buffers) and raises OvlError on a failing status. All arithmetic runs in the
library's CUDA kernels; there is no Python or CPU fallback. Importing this package fails
loudly when libovl.so has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libovl.so")

# status codes (include/ovl.h)
OVL_OK, OVL_PENDING = 0, 1
OVL_EINVAL, OVL_ENOMEM, OVL_ECUDA, OVL_EBREAKDOWN = -1, -2, -3, -4
OVL_ENOCONV, OVL_ETIMEOUT, OVL_EBUSY, OVL_EILLPOSED, OVL_ENOTFOUND = -5, -6, -7, -8, -9
STATUS_NAMES = {0: "OK", 1: "PENDING", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "EBREAKDOWN",
                -5: "ENOCONV", -6: "ETIMEOUT", -7: "EBUSY", -8: "EILLPOSED", -9: "ENOTFOUND"}
OVL_F64, OVL_F32, OVL_F16R12 = 1, 2, 4
OVL_C128, OVL_C64 = 0, 1
OVL_DAGGER, OVL_GAMMA5, OVL_NATIVE, OVL_LINKS_F32, OVL_LINKS_F16R12 = 1, 2, 4, 8, 16
OVL_DIRECT_2SL, OVL_MULTISHIFT_BICG, OVL_FOM_RESTARTED = 0, 1, 2
OVL_PREC_F64, OVL_PREC_F32, OVL_PREC_F32_F16LINKS = 0, 1, 2
OVL_RAT_NEUBERGER, OVL_RAT_ZOLOTAREV, OVL_RAT_CUSTOM = 0, 1, 2


class OvlError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (%d): %s" % (STATUS_NAMES.get(status, "?"), status, msg))
        self.status = status


class ovl_sign_params(ctypes.Structure):
    _fields_ = [
        ("method", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("m_W", ctypes.c_double), ("mu", ctypes.c_double), ("tol", ctypes.c_double),
        ("k_max", ctypes.c_int32), ("check_every", ctypes.c_int32), ("use_deflation", ctypes.c_int32),
        ("rational_kind", ctypes.c_int32), ("s", ctypes.c_int32),
        ("spec_lo", ctypes.c_double), ("spec_hi", ctypes.c_double),
        ("omega", ctypes.POINTER(ctypes.c_double)), ("sigma", ctypes.POINTER(ctypes.c_double)),
        ("host_io", ctypes.c_int32), ("use_graphs", ctypes.c_int32), ("fixed_k", ctypes.c_int32),
        ("priority", ctypes.c_int32), ("restart_k", ctypes.c_int32), ("two_pass", ctypes.c_int32),
    ]


class ovl_sign_info(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32), ("iterations", ctypes.c_int32), ("matvecs", ctypes.c_int32),
        ("poles", ctypes.c_int32), ("est_error", ctypes.c_double), ("t_total_ms", ctypes.c_double),
        ("t_small_ms", ctypes.c_double), ("residual", ctypes.c_double), ("t_kernel_ms", ctypes.c_double),
        ("t_update_ms", ctypes.c_double), ("kernel_samples", ctypes.c_int32), ("kernel_launches", ctypes.c_int32),
        ("evaluations", ctypes.c_int32), ("ritz_evaluations", ctypes.c_int32), ("t_finish_ms", ctypes.c_double),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ovl_server_cfg(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_int64), ("max_slots", ctypes.c_int32), ("streams", ctypes.c_int32)]


class ovl_request(ctypes.Structure):
    _fields_ = [
        ("field_id", ctypes.c_int32), ("nrhs", ctypes.c_int32), ("mu", ctypes.c_double), ("m_W", ctypes.c_double),
        ("tol", ctypes.c_double), ("k_max", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("b", ctypes.c_void_p), ("method", ctypes.c_int32), ("use_deflation", ctypes.c_int32),
        ("rational_kind", ctypes.c_int32), ("s", ctypes.c_int32), ("spec_lo", ctypes.c_double),
        ("spec_hi", ctypes.c_double), ("two_pass", ctypes.c_int32),
    ]


_P = ctypes.c_void_p
_I = ctypes.c_int32
_D = ctypes.c_double
_PROTOS = {
    "ovl_ctx_create": (_I, [_I, ctypes.POINTER(_P)]),
    "ovl_ctx_destroy": (_I, [_P]),
    "ovl_last_error": (ctypes.c_char_p, []),
    "ovl_version": (ctypes.c_char_p, []),
    "ovl_create_lattice": (_I, [_P, ctypes.POINTER(_I), _I, ctypes.POINTER(_P)]),
    "ovl_destroy_lattice": (_I, [_P]),
    "ovl_lattice_n": (ctypes.c_int64, [_P]),
    "ovl_set_links": (_I, [_P, _P, _I, ctypes.c_uint32]),
    "ovl_set_deflation": (_I, [_P, _D, _D, _I, _P, _P, _P, _I]),
    "ovl_to_native": (_I, [_P, _I, _I, _P, _P, _P]),
    "ovl_from_native": (_I, [_P, _I, _I, _P, _P, _P]),
    "ovl_apply_DW": (_I, [_P, _D, _D, ctypes.c_uint32, _I, _I, _P, _P, _P]),
    "ovl_sign_params_default": (None, [ctypes.POINTER(ovl_sign_params)]),
    "ovl_apply_sign": (_I, [_P, ctypes.POINTER(ovl_sign_params), _I, _P, _P, ctypes.POINTER(ovl_sign_info), _P]),
    "ovl_apply_sign_noalloc": (_I, [_P, ctypes.POINTER(ovl_sign_params), _I, _P, _P,
                                    ctypes.POINTER(ovl_sign_info), _P]),
    "ovl_set_pair_variant": (_I, [ctypes.c_int64, _I, _I]),
    "ovl_get_pair_variant": (_I, [ctypes.c_int64, _I]),
    "ovl_get_tridiag": (_I, [_P, _I, _I, ctypes.POINTER(_I), _P, _P, _P]),
    "ovl_small_sign": (_I, [_I, _P, _P, _P, _P, _I]),
    "ovl_rational_coeffs": (_I, [_I, _I, _D, _D, _D, _I, _P, _P, ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "ovl_server_create": (_I, [_P, ctypes.POINTER(ovl_server_cfg), ctypes.POINTER(_P)]),
    "ovl_server_add_field": (_I, [_P, _P, ctypes.POINTER(_I)]),
    "ovl_submit": (_I, [_P, ctypes.POINTER(ovl_request), ctypes.POINTER(ctypes.c_uint64)]),
    "ovl_poll": (_I, [_P, ctypes.c_uint64, ctypes.POINTER(ovl_sign_info), _P]),
    "ovl_server_destroy": (_I, [_P]),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libovl.so is not built (%s): run `python -c 'import __graft_entry__ as g; g.build()'`"
                          % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _PROTOS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def _err(status):
    return OvlError(status, lib.ovl_last_error().decode())


def _check(status):
    if status < 0:
        raise _err(status)
    return status


def _ptr(a):
    """Address of a numpy array or torch tensor (contiguous)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError("expected a numpy array or torch tensor, got %r" % type(a))


def _on_device(a):
    return hasattr(a, "is_cuda") and a.is_cuda


def _stream(stream, *tensors):
    if stream is not None:
        return stream
    if any(_on_device(t) for t in tensors):
        import torch
        return torch.cuda.current_stream().cuda_stream
    return None


def _dtype_code(a):
    name = str(a.dtype)
    if name.endswith("complex128"):
        return OVL_C128
    if name.endswith("complex64"):
        return OVL_C64
    raise TypeError("spinor buffers must be complex128 or complex64, got %s" % name)


# ------------------------------------------------------------------ context, lattice
def ovl_version() -> str:
    return lib.ovl_version().decode()


_CTX_DEVICE: dict = {}  # context handle -> CUDA device ordinal
_LAT_DEVICE: dict = {}  # lattice handle -> CUDA device ordinal


def ovl_ctx_create(device: int = 0):
    h = _P()
    _check(lib.ovl_ctx_create(device, ctypes.byref(h)))
    _CTX_DEVICE[h.value] = int(device)
    return h


def ovl_ctx_destroy(ctx):
    _check(lib.ovl_ctx_destroy(ctx))
    _CTX_DEVICE.pop(ctx.value, None)


def ovl_create_lattice(ctx, dims, t_bc: int = -1):
    arr = (_I * 4)(*[int(d) for d in dims])
    h = _P()
    _check(lib.ovl_create_lattice(ctx, arr, int(t_bc), ctypes.byref(h)))
    if ctx.value in _CTX_DEVICE:
        _LAT_DEVICE[h.value] = _CTX_DEVICE[ctx.value]
    return h


def ovl_destroy_lattice(lat):
    _check(lib.ovl_destroy_lattice(lat))
    _LAT_DEVICE.pop(lat.value, None)


def ovl_lattice_n(lat) -> int:
    return int(lib.ovl_lattice_n(lat))


def _host_or_device_c128(a, count, where, nm):
    """A complex128 input of `count` elements: a numpy array (made contiguous complex128 here) or
    a contiguous complex128 tensor (CUDA, or CPU). Returns (buffer, on_device)."""
    if isinstance(a, np.ndarray):
        a = np.ascontiguousarray(a, dtype=np.complex128)
        size, dev = a.size, False
    elif hasattr(a, "data_ptr"):
        if str(a.dtype) != "torch.complex128" or not a.is_contiguous():
            raise TypeError("%s: %s must be a contiguous complex128 tensor" % (where, nm))
        size, dev = a.numel(), _on_device(a)
    else:
        raise TypeError("%s: %s must be a numpy array or a torch tensor, got %r" % (where, nm, type(a)))
    if size != count:
        raise ValueError("%s: %s holds %d complex entries, %d expected" % (where, nm, size, count))
    return a, dev


def ovl_set_links(lat, U, formats: int = OVL_F64):
    """U: the canonical [4][Lt][Lz][Ly][Lx][3][3] complex128 links (36 V entries), host or device."""
    U, dev = _host_or_device_c128(U, 3 * ovl_lattice_n(lat), "ovl_set_links", "U")
    _check(lib.ovl_set_links(lat, _ptr(U), 1 if dev else 0, formats))


def ovl_set_deflation(lat, m_W, mu, R, L, lam):
    """R, L: [m][n] complex128 (canonical), lam: [m] complex128; all on the host or all on the device."""
    if R is None or len(R) == 0:
        _check(lib.ovl_set_deflation(lat, m_W, mu, 0, None, None, None, 0))
        return
    m, n = int(R.shape[0]), ovl_lattice_n(lat)
    R, dev = _host_or_device_c128(R, m * n, "ovl_set_deflation", "R")
    L, dev_l = _host_or_device_c128(L, m * n, "ovl_set_deflation", "L")
    lam, dev_lam = _host_or_device_c128(lam, m, "ovl_set_deflation", "lam")
    if not dev == dev_l == dev_lam:
        raise TypeError("ovl_set_deflation: R, L and lam must all be host or all be device buffers")
    _check(lib.ovl_set_deflation(lat, m_W, mu, m, _ptr(R), _ptr(L), _ptr(lam), 1 if dev else 0))


def _spinor_pair(lat, inp, out, where):
    """Validate the in / out pair of a stream-ordered spinor call before any pointer reaches the
    library: contiguous CUDA tensors on the lattice's device, the same complex dtype, a whole
    number of spinors each. Returns nrhs."""
    n = ovl_lattice_n(lat)
    for nm, a in (("in", inp), ("out", out)):
        if not _on_device(a):
            raise TypeError("%s: %s must be a CUDA tensor" % (where, nm))
        if not a.is_contiguous():
            raise TypeError("%s: %s must be contiguous" % (where, nm))
        dev = _LAT_DEVICE.get(lat.value)
        if dev is not None and a.device.index != dev:
            raise ValueError("%s: %s is on cuda:%s, the lattice on cuda:%d" % (where, nm, a.device.index, dev))
    _dtype_code(inp)
    if out.dtype != inp.dtype:
        raise TypeError("%s: in and out must have the same dtype" % where)
    if inp.numel() == 0 or inp.numel() % n != 0 or out.numel() != inp.numel():
        raise ValueError("%s: in/out must hold nrhs * n elements (n = %d), got %d and %d"
                         % (where, n, inp.numel(), out.numel()))
    return inp.numel() // n


def ovl_to_native(lat, inp, out, stream=None):
    nrhs = _spinor_pair(lat, inp, out, "ovl_to_native")
    _check(lib.ovl_to_native(lat, _dtype_code(inp), nrhs, _ptr(inp), _ptr(out), _stream(stream, inp)))


def ovl_from_native(lat, inp, out, stream=None):
    nrhs = _spinor_pair(lat, inp, out, "ovl_from_native")
    _check(lib.ovl_from_native(lat, _dtype_code(inp), nrhs, _ptr(inp), _ptr(out), _stream(stream, inp)))


def ovl_apply_DW(lat, m_W, mu, flags, inp, out, stream=None):
    """out = D_W(mu) inp (flags OVL_DAGGER / OVL_GAMMA5 / OVL_NATIVE / OVL_LINKS_*); device tensors."""
    nrhs = _spinor_pair(lat, inp, out, "ovl_apply_DW")
    _check(lib.ovl_apply_DW(lat, m_W, mu, flags, _dtype_code(inp), nrhs, _ptr(inp), _ptr(out),
                            _stream(stream, inp, out)))


# ------------------------------------------------------------------ sign
def ovl_sign_params_default(**kw) -> ovl_sign_params:
    p = ovl_sign_params()
    lib.ovl_sign_params_default(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def _sign_buffers(lat, b, x, where):
    """Validate the b / x pair of a sign solve before any pointer reaches the library (a short or
    mistyped x would otherwise be written out of bounds by the kernels). Returns (nrhs, host)."""
    n = ovl_lattice_n(lat)
    host = isinstance(b, np.ndarray)
    if host != isinstance(x, np.ndarray):
        raise TypeError("%s: b and x must both be host (numpy) or both device (torch) buffers" % where)
    if host:
        for nm, a in (("b", b), ("x", x)):
            if a.dtype != np.complex128 or not a.flags["C_CONTIGUOUS"]:
                raise TypeError("%s: %s must be a C-contiguous complex128 array" % (where, nm))
        size_b, size_x = b.size, x.size
    else:
        for nm, a in (("b", b), ("x", x)):
            if not _on_device(a):
                raise TypeError("%s: %s must be a CUDA tensor (or both numpy arrays)" % (where, nm))
            if str(a.dtype) != "torch.complex128" or not a.is_contiguous():
                raise TypeError("%s: %s must be a contiguous complex128 tensor" % (where, nm))
            dev = _LAT_DEVICE.get(lat.value)
            if dev is not None and a.device.index != dev:
                raise ValueError("%s: %s is on cuda:%s, the lattice on cuda:%d" % (where, nm, a.device.index, dev))
        size_b, size_x = b.numel(), x.numel()
    if size_b == 0 or size_b % n != 0:
        raise ValueError("%s: b holds %d elements, not a whole number of spinors of n = %d" % (where, size_b, n))
    if size_x != size_b:
        raise ValueError("%s: x holds %d elements, b %d" % (where, size_x, size_b))
    return size_b // n, host


def ovl_apply_sign(lat, params: ovl_sign_params, b, x, stream=None, raise_on_error=False):
    """x = sign(H_W(mu)) b. b, x: complex128 [nrhs][...] as torch CUDA tensors, or numpy arrays
    (then params.host_io is set). Returns (status, [info dict per rhs]); raises OvlError for
    argument/CUDA/memory errors (and for every error if raise_on_error)."""
    nrhs, host = _sign_buffers(lat, b, x, "ovl_apply_sign")
    params.host_io = 1 if host else 0
    infos = (ovl_sign_info * nrhs)()
    st = lib.ovl_apply_sign(lat, ctypes.byref(params), nrhs, _ptr(b), _ptr(x), infos, _stream(stream, b, x))
    if st in (OVL_EINVAL, OVL_ENOMEM, OVL_ECUDA) or (raise_on_error and st < 0):
        raise _err(st)
    return st, [i.as_dict() for i in infos]


def ovl_apply_sign_noalloc(lat, params: ovl_sign_params, b, x, stream=None):
    """ovl_apply_sign's direct method without any device allocation (scratch in a static
    64 MiB device array): for callers that cannot allocate device memory. b, x are torch CUDA
    tensors. Returns (status, [info dict per rhs]); raises OvlError for argument/CUDA errors."""
    nrhs, host = _sign_buffers(lat, b, x, "ovl_apply_sign_noalloc")
    if host:
        raise TypeError("ovl_apply_sign_noalloc: b and x must be CUDA tensors")
    infos = (ovl_sign_info * nrhs)()
    st = lib.ovl_apply_sign_noalloc(lat, ctypes.byref(params), nrhs, _ptr(b), _ptr(x), infos, _stream(stream, b, x))
    if st in (OVL_EINVAL, OVL_ENOMEM, OVL_ECUDA):
        raise _err(st)
    return st, [i.as_dict() for i in infos]


def ovl_set_pair_variant(volume: int, precision: int, variant: int):
    """Pin (variant >= 0) or clear (-1) the pair-stencil shape for (volume, precision)."""
    st = lib.ovl_set_pair_variant(volume, precision, variant)
    if st != OVL_OK:
        raise _err(st)


def ovl_get_pair_variant(volume: int, precision: int) -> int:
    return int(lib.ovl_get_pair_variant(volume, precision))


def ovl_get_tridiag(lat, rhs: int = 0, k_cap: int = 100000):
    k = _I()
    st = lib.ovl_get_tridiag(lat, rhs, 0, ctypes.byref(k), None, None, None)
    if st not in (OVL_OK, OVL_EINVAL):
        raise _err(st)
    kk = k.value
    a = np.zeros(kk, np.complex128)
    b = np.zeros(max(kk - 1, 0), np.complex128)
    d = np.zeros(max(kk - 1, 0), np.complex128)
    _check(lib.ovl_get_tridiag(lat, rhs, kk, ctypes.byref(k), _ptr(a), _ptr(b) if kk > 1 else None,
                               _ptr(d) if kk > 1 else None))
    return a, b, d


# ------------------------------------------------------------------ host-side pieces
def ovl_small_sign(alpha, beta, delta, method: int = 0):
    """(status, y) with y = sign(T) e_1 for the tridiagonal (alpha, beta super, delta sub)."""
    a = np.ascontiguousarray(alpha, dtype=np.complex128)
    b = np.ascontiguousarray(beta, dtype=np.complex128)
    d = np.ascontiguousarray(delta, dtype=np.complex128)
    y = np.zeros(len(a), np.complex128)
    st = lib.ovl_small_sign(len(a), _ptr(a), _ptr(b) if len(b) else None, _ptr(d) if len(d) else None, _ptr(y),
                            method)
    if st == OVL_EINVAL:
        raise _err(st)
    return st, y


def ovl_rational_coeffs(kind, s, lo, hi, eps=0.0, s_cap=512):
    om = np.zeros(s_cap)
    sg = np.zeros(s_cap)
    so = _I()
    err = _D()
    _check(lib.ovl_rational_coeffs(kind, s, lo, hi, eps, s_cap, _ptr(om), _ptr(sg), ctypes.byref(so),
                                   ctypes.byref(err)))
    return om[:so.value].copy(), sg[:so.value].copy(), err.value


# ------------------------------------------------------------------ serving
def ovl_server_create(ctx, mem_budget_bytes: int, max_slots: int = 8, streams: int = 4):
    cfg = ovl_server_cfg(mem_budget_bytes, max_slots, streams)
    h = _P()
    _check(lib.ovl_server_create(ctx, ctypes.byref(cfg), ctypes.byref(h)))
    return h


def ovl_server_add_field(srv, lat) -> int:
    fid = _I()
    _check(lib.ovl_server_add_field(srv, lat, ctypes.byref(fid)))
    return fid.value


def _nrhs_of(b: np.ndarray, nrhs):
    """Right-hand sides in a canonical spinor array: [Lt][Lz][Ly][Lx][4][3] is one,
    [nrhs][Lt][Lz][Ly][Lx][4][3] is a batch; a flat array needs nrhs given."""
    if nrhs is not None:
        return int(nrhs)
    if b.ndim == 7:
        return int(b.shape[0])
    if b.ndim == 6:
        return 1
    raise ValueError("pass nrhs for a spinor array of shape %r" % (b.shape,))


def ovl_submit(srv, field_id, b: np.ndarray, mu, tol, m_W=-2.0, k_max=600, precision=OVL_PREC_F64, nrhs=None,
               method=OVL_DIRECT_2SL, use_deflation=0, rational_kind=OVL_RAT_NEUBERGER, s=0, spec_lo=0.0,
               spec_hi=0.0, two_pass=0):
    """Queue x = sign(H_W(mu)) b on a registered field; b is copied before the call returns.
    method OVL_MULTISHIFT_BICG needs spec_lo < spec_hi (and s > 0 for Zolotarev)."""
    b = np.ascontiguousarray(b, dtype=np.complex128)
    nr = _nrhs_of(b, nrhs)
    if b.size % (12 * nr) != 0:
        raise ValueError("b does not hold nrhs whole spinors")
    req = ovl_request(field_id, nr, mu, m_W, tol, k_max, precision, b.ctypes.data, method, use_deflation,
                      rational_kind, s, spec_lo, spec_hi, two_pass)
    t = ctypes.c_uint64()
    _check(lib.ovl_submit(srv, ctypes.byref(req), ctypes.byref(t)))
    return t.value


def ovl_poll(srv, ticket, nrhs, x_out: np.ndarray | None = None):
    """Returns (status, infos); status OVL_PENDING while running. x_out (complex128) must hold
    the request's nrhs spinors; it is written once, when the request is done."""
    if x_out is not None and (x_out.dtype != np.complex128 or not x_out.flags["C_CONTIGUOUS"]):
        raise TypeError("x_out must be a C-contiguous complex128 array")
    infos = (ovl_sign_info * max(nrhs, 1))()
    st = lib.ovl_poll(srv, ticket, infos, _ptr(x_out) if x_out is not None else None)
    if st in (OVL_EINVAL, OVL_ENOTFOUND, OVL_ECUDA, OVL_ENOMEM):
        raise _err(st)
    return st, [i.as_dict() for i in infos]


def ovl_server_destroy(srv):
    _check(lib.ovl_server_destroy(srv))
