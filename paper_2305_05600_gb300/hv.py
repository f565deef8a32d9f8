"""Thin ctypes binding of libhv (include/hv.h), same names as the C ABI.

Argument marshalling only: every step of the method runs in the CUDA
kernels of libhv.  PyTorch supplies device memory (through the allocation
hook) and streams.  There is no fallback: if libhv cannot be built or
loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

HV_OK, HV_EINVAL, HV_ENOMEM, HV_ECUDA, HV_ECFL, HV_ENAN, HV_ETIMEOUT, HV_ESTATE = range(8)
STATUS_NAMES = ["HV_OK", "HV_EINVAL", "HV_ENOMEM", "HV_ECUDA", "HV_ECFL", "HV_ENAN",
                "HV_ETIMEOUT", "HV_ESTATE"]
SHAPES = {"ngp": 0, "qs": 1, "cic": 2}


class HVError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {message}")


class Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("nsub", ctypes.c_int32), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("dz", ctypes.c_double), ("dt", ctypes.c_double), ("Te", ctypes.c_double),
                ("gamma_e", ctypes.c_double), ("eta", ctypes.c_double),
                ("eta_h", ctypes.c_double), ("n_floor", ctypes.c_double),
                ("shape", ctypes.c_int32), ("smooth_passes", ctypes.c_int32),
                ("sort_every", ctypes.c_int32), ("field_smooth_passes", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("pe_eq", ctypes.c_int32),
                ("ohm_model", ctypes.c_int32), ("kappa", ctypes.c_double),
                ("relativistic", ctypes.c_int32), ("open_faces", ctypes.c_int32),
                ("c_light", ctypes.c_double)]


class Diag(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("t", ctypes.c_double), ("W_K", ctypes.c_double),
                ("P", ctypes.c_double * 3), ("charge", ctypes.c_double),
                ("W_B", ctypes.c_double), ("max_divB", ctypes.c_double),
                ("err_word", ctypes.c_int32), ("pad", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {"step": self.step, "t": self.t, "W_K": self.W_K, "P": list(self.P),
                "charge": self.charge, "W_B": self.W_B, "max_divB": self.max_divB,
                "err_word": self.err_word}


class Prof(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("ms_sort", "ms_push", "ms_moments", "ms_field", "ms_ohm", "ms_diag")] + \
               [(n, ctypes.c_int64) for n in
                ("n_sort", "n_push", "n_moments", "n_field", "n_ohm", "n_diag", "steps",
                 "launches")]

    def as_dict(self) -> dict:
        return {f[0]: getattr(self, f[0]) for f in self._fields_}


class Info(ctypes.Structure):
    _fields_ = [("ncell", ctypes.c_int64), ("tile", ctypes.c_int32 * 3),
                ("ntiles", ctypes.c_int32), ("nspecies", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("n", ctypes.c_int64 * 8), ("step", ctypes.c_int64)]


assert ctypes.sizeof(Params) == 144, ctypes.sizeof(Params)

_lib = None
_lock = threading.Lock()
_hooks = []  # keep ctypes callbacks alive

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                           ctypes.c_void_p)

EXPORTS = ["hv_set_allocator", "hv_init_grid", "hv_load_ions", "hv_step", "hv_moments",
           "hv_diag", "hv_diag_async", "hv_diag_wait", "hv_get_ions", "hv_query", "hv_profile", "hv_profile_read", "hv_destroy",
           "hv_sort_keys", "hv_sort_keys_noalloc", "hv_set_filter", "hv_filter_moments",
           "hv_filter_train_init", "hv_filter_grad", "hv_filter_train_step",
           "hv_filter_get_params", "hv_electron_pressure", "hv_get_tile_offsets",
           "hv_inject_error", "hv_error_status", "hv_set_external_field", "hv_reserve_ions", "hv_set_injection",
           "hv_last_error"]


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libhv, building it in-tree first if its sources are newer."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        # HV_LIB selects a prebuilt copy of libhv (e.g. a tuning variant)
        path = os.environ.get("HV_LIB") or _build.build()
        L = ctypes.CDLL(path)
        P, I32, I64, V = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
        L.hv_set_allocator.argtypes = [ALLOC_FN, FREE_FN, P]
        L.hv_init_grid.argtypes = [ctypes.POINTER(Params), P, P, ctypes.POINTER(P)]
        L.hv_load_ions.argtypes = [P, I32, ctypes.c_double, ctypes.c_double, I64, P, P, P, P,
                                   ctypes.c_int]
        L.hv_step.argtypes = [P, I32]
        L.hv_moments.argtypes = [P, P, P, P, P, ctypes.c_int]
        L.hv_diag.argtypes = [P, ctypes.POINTER(Diag)]
        L.hv_diag_async.argtypes = [P]
        L.hv_diag_wait.argtypes = [P, ctypes.POINTER(Diag)]
        L.hv_electron_pressure.argtypes = [P, P, ctypes.c_int]
        L.hv_get_ions.argtypes = [P, I32, ctypes.POINTER(I64), P, P, P, P, ctypes.c_int]
        L.hv_query.argtypes = [P, ctypes.POINTER(Info)]
        L.hv_get_tile_offsets.argtypes = [P, I32, P]
        L.hv_inject_error.argtypes = [P, I32]
        L.hv_error_status.argtypes = [I32]
        L.hv_set_external_field.argtypes = [P, P]
        L.hv_reserve_ions.argtypes = [P, I32, I64]
        L.hv_set_injection.argtypes = [P, I32, I32, ctypes.c_double, P, ctypes.c_double,
                                       ctypes.c_double]
        L.hv_set_filter.argtypes = [P, P, P, ctypes.c_double, ctypes.c_double]
        L.hv_filter_moments.argtypes = [P, P, P, ctypes.c_int]
        L.hv_filter_train_init.argtypes = [P, P, P]
        L.hv_filter_grad.argtypes = [P, P, P, I32, P, ctypes.POINTER(ctypes.c_double),
                                     ctypes.c_int]
        L.hv_filter_train_step.argtypes = [P, P, P, I32, ctypes.c_double,
                                           ctypes.POINTER(ctypes.c_double), ctypes.c_int]
        L.hv_filter_get_params.argtypes = [P, P]
        L.hv_profile.argtypes = [P, ctypes.c_int]
        L.hv_profile_read.argtypes = [P, ctypes.POINTER(Prof)]
        L.hv_destroy.argtypes = [P]
        L.hv_destroy.restype = None
        L.hv_sort_keys.argtypes = [P, I64, I32, P, P, P]
        L.hv_sort_keys_noalloc.argtypes = [P, I64, I32, P, P, P]
        L.hv_last_error.restype = ctypes.c_char_p
        for nm in EXPORTS:
            if nm != "hv_destroy" and nm != "hv_last_error":
                getattr(L, nm).restype = ctypes.c_int
        _lib = L
        return _lib


def _check(rc: int):
    if rc != HV_OK:
        raise HVError(rc, lib().hv_last_error().decode())


def hv_last_error() -> str:
    return lib().hv_last_error().decode()


def hv_set_allocator(use_torch: bool = True):
    """Route every library allocation through PyTorch's caching allocator
    (use_torch=True) or back to cudaMallocAsync (False)."""
    L = lib()
    if not use_torch:
        _check(L.hv_set_allocator(ALLOC_FN(0), FREE_FN(0), None))
        return
    import torch

    def _alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                      int(stream or 0))
        except Exception:  # out of memory: report NULL to the library
            return None

    def _free(ptr, nbytes, stream, user):
        torch.cuda.caching_allocator_delete(int(ptr))

    a, f = ALLOC_FN(_alloc), FREE_FN(_free)
    _hooks[:] = [a, f]
    _check(L.hv_set_allocator(a, f, None))


def params_from(d: dict) -> Params:
    shape = d.get("shape", "qs")
    shape = SHAPES[shape] if isinstance(shape, str) else int(shape)
    return Params(int(d["nx"]), int(d["ny"]), int(d["nz"]), int(d.get("nsub", 1)),
                  float(d["dx"]), float(d.get("dy", 1.0)), float(d["dz"]), float(d["dt"]),
                  float(d.get("Te", 0.0)), float(d.get("gamma_e", 1.0)), float(d.get("eta", 0.0)),
                  float(d.get("eta_h", 0.0)), float(d.get("n_floor", 0.05)), shape,
                  int(d.get("smooth_passes", 0)), int(d.get("sort_every", 0)),
                  int(d.get("field_smooth_passes", 0)),
                  int(d.get("seed", 0)), int(d.get("pe_eq", 0)), int(d.get("ohm_model", 0)),
                  float(d.get("kappa", 0.0)), int(d.get("relativistic", 0)),
                  int(d.get("open_faces", 0)), float(d.get("c_light", 0.0)))


def _ptr(a):
    """(pointer, on_device) of a numpy array or torch tensor (contiguous)."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data, 0
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), int(a.is_cuda)
    raise TypeError(type(a))


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


class Ctx:
    """Owning handle of an hv_ctx."""

    def __init__(self, handle: int, params: Params):
        self.handle = ctypes.c_void_p(handle)
        self.params = params

    @property
    def ncell(self) -> int:
        return self.params.nx * self.params.ny * self.params.nz

    def close(self):
        if self.handle:
            lib().hv_destroy(self.handle)
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hv_init_grid(params, B0=None, stream=None) -> Ctx:
    p = params if isinstance(params, Params) else params_from(params)
    b = None
    if B0 is not None:
        b = np.ascontiguousarray(np.asarray(B0, dtype=np.float32).reshape(-1))
        if b.size != 3 * p.nx * p.ny * p.nz:
            raise ValueError("B0 must have 3*nx*ny*nz values")
    out = ctypes.c_void_p()
    _check(lib().hv_init_grid(ctypes.byref(p), b.ctypes.data if b is not None else None,
                              _stream_handle(stream), ctypes.byref(out)))
    return Ctx(out.value, p)


def hv_set_external_field(ctx: Ctx, B0ext):
    """Fixed external field B0 [3][nz][ny][nx] of the B = B0 + B1 split."""
    p = ctx.params
    b = np.ascontiguousarray(np.asarray(B0ext, dtype=np.float32).reshape(-1))
    if b.size != 3 * p.nx * p.ny * p.nz:
        raise ValueError("the external field must have 3*nx*ny*nz values")
    _check(lib().hv_set_external_field(ctx.handle, b.ctypes.data))


def hv_reserve_ions(ctx: Ctx, species: int, capacity: int):
    """Particle slots for ions injected through open faces."""
    _check(lib().hv_reserve_ions(ctx.handle, int(species), int(capacity)))


def hv_set_injection(ctx: Ctx, species: int, face: int, n: float, u, T: float, w: float):
    """Drifting Maxwellian injected through an open face every step."""
    uu = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(3))
    _check(lib().hv_set_injection(ctx.handle, int(species), int(face), float(n),
                                  uu.ctypes.data, float(T), float(w)))


def hv_load_ions(ctx: Ctx, species: int, q: float, m: float, cell, off3, v3, w):
    n = int(cell.shape[0])
    pc, d0 = _ptr(cell)
    po, d1 = _ptr(off3)
    pv, d2 = _ptr(v3)
    pw, d3 = _ptr(w)
    if len({d0, d1, d2, d3}) != 1:
        raise ValueError("particle arrays must all be on the host or all on the device")
    _check(lib().hv_load_ions(ctx.handle, species, float(q), float(m), n, pc, po, pv, pw, d0))


def hv_step(ctx: Ctx, nsteps: int = 1):
    _check(lib().hv_step(ctx.handle, int(nsteps)))


def hv_moments(ctx: Ctx, n_out=None, J_out=None, E_out=None, B_out=None, host: bool = True):
    """Copy n, J (last half-step moments), E, B out.  With host=True and no
    outputs given, returns numpy arrays [nz,ny,nx] / [3,nz,ny,nx]."""
    p = ctx.params
    shp = (p.nz, p.ny, p.nx)
    if host and n_out is None and J_out is None and E_out is None and B_out is None:
        n_out = np.zeros(shp, np.float32)
        J_out = np.zeros((3,) + shp, np.float32)
        E_out = np.zeros((3,) + shp, np.float32)
        B_out = np.zeros((3,) + shp, np.float32)
    ptrs, devs = zip(*[_ptr(a) for a in (n_out, J_out, E_out, B_out)])
    on_dev = max(devs)
    _check(lib().hv_moments(ctx.handle, *ptrs, on_dev))
    return {"n": n_out, "J": J_out, "E": E_out, "B": B_out}


def hv_electron_pressure(ctx: Ctx, pe_out=None, host: bool = True):
    """Copy the electron pressure field p_e [nz,ny,nx] out (contexts created
    with pe_eq = 1).  With host=True and no output given, returns a numpy
    array."""
    p = ctx.params
    if host and pe_out is None:
        pe_out = np.zeros((p.nz, p.ny, p.nx), np.float32)
    ptr, dev = _ptr(pe_out)
    _check(lib().hv_electron_pressure(ctx.handle, ptr, dev))
    return pe_out


def hv_diag(ctx: Ctx, check: bool = True) -> dict:
    d = Diag()
    rc = lib().hv_diag(ctx.handle, ctypes.byref(d))
    if check:
        _check(rc)
    out = d.as_dict()
    out["status"] = rc
    return out


def hv_diag_async(ctx: Ctx):
    """Enqueue the diagnostics of the state after the last step (up to 4
    pending); hv_diag_wait collects them oldest first."""
    _check(lib().hv_diag_async(ctx.handle))


def hv_diag_wait(ctx: Ctx, check: bool = True) -> dict:
    d = Diag()
    rc = lib().hv_diag_wait(ctx.handle, ctypes.byref(d))
    if check:
        _check(rc)
    out = d.as_dict()
    out["status"] = rc
    return out


def hv_get_ions(ctx: Ctx, species: int = 0) -> dict:
    n = ctypes.c_int64()
    _check(lib().hv_get_ions(ctx.handle, species, ctypes.byref(n), None, None, None, None, 0))
    nn = n.value
    cell = np.zeros(nn, np.int32)
    off = np.zeros((3, nn), np.float32)
    v = np.zeros((3, nn), np.float32)
    w = np.zeros(nn, np.float32)
    _check(lib().hv_get_ions(ctx.handle, species, ctypes.byref(n), cell.ctypes.data,
                             off.ctypes.data, v.ctypes.data, w.ctypes.data, 0))
    return {"cell": cell, "off": off, "v": v, "w": w}


FILTER_NPARAM = 3492


def hv_set_filter(ctx: Ctx, params=None, scale=(1.0, 1.0, 1.0, 1.0), gate_nmin=0.0,
                  gate_rmax=1.0):
    """Install the learned moment filter (params: 3492 floats) or remove it
    (params=None)."""
    if params is None:
        _check(lib().hv_set_filter(ctx.handle, None, None, 0.0, 0.0))
        return
    P = np.ascontiguousarray(np.asarray(params, dtype=np.float32).reshape(-1))
    if P.size != FILTER_NPARAM:
        raise ValueError(f"filter needs {FILTER_NPARAM} parameters")
    S = np.ascontiguousarray(np.asarray(scale, dtype=np.float32).reshape(4))
    _check(lib().hv_set_filter(ctx.handle, P.ctypes.data, S.ctypes.data, float(gate_nmin),
                               float(gate_rmax)))


def hv_filter_moments(ctx: Ctx, m4) -> np.ndarray:
    m = np.ascontiguousarray(np.asarray(m4, dtype=np.float32))
    y = np.zeros_like(m)
    _check(lib().hv_filter_moments(ctx.handle, m.ctypes.data, y.ctypes.data, 0))
    return y


def hv_filter_train_init(ctx: Ctx, params, scale=(1.0, 1.0, 1.0, 1.0)):
    P = np.ascontiguousarray(np.asarray(params, dtype=np.float32).reshape(-1))
    S = np.ascontiguousarray(np.asarray(scale, dtype=np.float32).reshape(4))
    _check(lib().hv_filter_train_init(ctx.handle, P.ctypes.data, S.ctypes.data))


def _pairs(m, t):
    m = np.ascontiguousarray(np.asarray(m, dtype=np.float32))
    t = np.ascontiguousarray(np.asarray(t, dtype=np.float32))
    if m.shape != t.shape:
        raise ValueError("input and target batches differ in shape")
    nb = m.shape[0] if m.ndim > 2 else 1
    return m, t, nb


def hv_filter_grad(ctx: Ctx, m, t):
    """(loss, gradient[3492]) of a batch of pairs [nb][4][...] at the current
    parameters."""
    m, t, nb = _pairs(m, t)
    g = np.zeros(FILTER_NPARAM, np.float32)
    loss = ctypes.c_double()
    _check(lib().hv_filter_grad(ctx.handle, m.ctypes.data, t.ctypes.data, nb, g.ctypes.data,
                                ctypes.byref(loss), 0))
    return loss.value, g


def hv_filter_train_step(ctx: Ctx, m, t, lr: float) -> float:
    m, t, nb = _pairs(m, t)
    loss = ctypes.c_double()
    _check(lib().hv_filter_train_step(ctx.handle, m.ctypes.data, t.ctypes.data, nb, float(lr),
                                      ctypes.byref(loss), 0))
    return loss.value


def hv_filter_get_params(ctx: Ctx) -> np.ndarray:
    P = np.zeros(FILTER_NPARAM, np.float32)
    _check(lib().hv_filter_get_params(ctx.handle, P.ctypes.data))
    return P


def hv_query(ctx: Ctx) -> dict:
    info = Info()
    _check(lib().hv_query(ctx.handle, ctypes.byref(info)))
    return {"ncell": info.ncell, "tile": tuple(info.tile), "ntiles": info.ntiles,
            "nspecies": info.nspecies, "n": list(info.n)[:info.nspecies], "step": info.step}


def hv_get_tile_offsets(ctx: Ctx, species: int = 0) -> np.ndarray:
    """Ion range of every supercell tile of a species (ntiles + 1 offsets)."""
    nt = hv_query(ctx)["ntiles"]
    out = np.zeros(nt + 1, np.int32)
    _check(lib().hv_get_tile_offsets(ctx.handle, int(species), out.ctypes.data))
    return out


def hv_inject_error(ctx: Ctx, bits: int):
    """OR error bits into the context's device error word (failure-path
    testing); the next synchronising call reports them."""
    _check(lib().hv_inject_error(ctx.handle, int(bits)))


def hv_error_status(err_word: int) -> int:
    """Status code a synchronising call returns for a device error word."""
    return int(lib().hv_error_status(int(err_word)))


def hv_profile(ctx: Ctx, enable: bool = True):
    _check(lib().hv_profile(ctx.handle, int(bool(enable))))


def hv_profile_read(ctx: Ctx) -> dict:
    pr = Prof()
    _check(lib().hv_profile_read(ctx.handle, ctypes.byref(pr)))
    return pr.as_dict()


def hv_destroy(ctx: Ctx):
    ctx.close()


def hv_sort_keys(keys, nkeys: int, stream=None):
    """Stable sort permutation and key counts of an int32 CUDA tensor."""
    import torch
    if keys.dtype != torch.int32 or not keys.is_cuda:
        raise TypeError("keys must be an int32 CUDA tensor")
    keys = keys.contiguous()
    n = keys.numel()
    perm = torch.empty(n, dtype=torch.int32, device=keys.device)
    counts = torch.empty(int(nkeys), dtype=torch.int32, device=keys.device)
    _check(lib().hv_sort_keys(keys.data_ptr(), n, int(nkeys), perm.data_ptr(),
                              counts.data_ptr(), _stream_handle(stream)))
    return perm, counts


def hv_sort_keys_noalloc(keys, nkeys: int, perm, counts=None, stream=None):
    """The allocation-free key sort: the caller supplies the output tensors
    (int32 CUDA perm [n] and optional counts [nkeys]); the library uses only
    its static device scratch (n <= 1,048,576).  The C side cannot check
    buffer sizes, so every tensor is checked here: contiguous int32 on one
    CUDA device, perm with at least n and counts with at least nkeys
    elements.  The call runs with that device current."""
    import torch
    named = [("keys", keys), ("perm", perm)] + ([("counts", counts)] if counts is not None else [])
    for name, t in named:
        if not isinstance(t, torch.Tensor) or t.dtype != torch.int32 or not t.is_cuda:
            raise TypeError(f"{name} must be an int32 CUDA tensor")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    if len({t.device for _, t in named}) != 1:
        raise ValueError("keys, perm and counts must be on one device")
    n = keys.numel()
    if int(nkeys) < 1:
        raise ValueError("nkeys must be >= 1")
    if perm.numel() < n:
        raise ValueError(f"perm has {perm.numel()} elements, fewer than the {n} keys")
    if counts is not None and counts.numel() < int(nkeys):
        raise ValueError(f"counts has {counts.numel()} elements, fewer than nkeys = {nkeys}")
    with torch.cuda.device(keys.device):
        _check(lib().hv_sort_keys_noalloc(keys.data_ptr(), n, int(nkeys), perm.data_ptr(),
                                          counts.data_ptr() if counts is not None else None,
                                          _stream_handle(stream)))
    return perm, counts


def load_workload(wl, stream=None, **override) -> Ctx:
    """Create a context for a seeded workload (see ``inputs``) and load its
    ions from host memory."""
    p = dict(wl.params)
    p.update(override)
    ctx = hv_init_grid(p, wl.B0, stream)
    for s_idx, s in enumerate(wl.species):
        hv_load_ions(ctx, s_idx, s.q, s.m, s.cell, s.off, s.v, s.w)
        if getattr(wl, "reserve", 0.0) > 0.0:
            hv_reserve_ions(ctx, s_idx, int(wl.reserve * s.n) + 1024)
    for s_idx, face, n, u, T, w in getattr(wl, "inject", []):
        hv_set_injection(ctx, s_idx, face, n, u, T, w)
    return ctx
