"""Plain FP64 CPU oracle of the hybrid PIC ion loop (arXiv 2305.05600).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the CPU
baseline leg of the benchmark, never by the library.  It shares no code with
the CUDA path.  The arithmetic lives in ``hvo.c`` (plain loops, paper order);
this module only compiles it with gcc and marshals numpy arrays.

Grids are component-major ``[ncomp][ncell]`` float64 arrays with the linear
cell index ``c = i + nx*(j + ny*k)`` (x fastest).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hvo.c")
_LIB = os.path.join(_HERE, "_build", "libhvo.so")
_lock = threading.Lock()
_lib = None

SHAPES = {"ngp": 0, "qs": 1, "cic": 2}


def build(force: bool = False) -> str:
    """Compile hvo.c into a shared library with gcc (no FMA contraction, so
    x86 and Arm hosts round identically), with OpenMP where gcc has it (the
    all-core baseline; one thread unless set_threads is called)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        base = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared",
                "-o", tmp, _SRC, "-lm"]
        r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
        if r.returncode != 0:
            subprocess.run(base, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("dt", ctypes.c_double), ("nsub", ctypes.c_int64),
                ("Te", ctypes.c_double), ("gamma_e", ctypes.c_double),
                ("eta", ctypes.c_double), ("eta_h", ctypes.c_double),
                ("n_floor", ctypes.c_double), ("shape", ctypes.c_int64),
                ("smooth_passes", ctypes.c_int64), ("field_smooth_passes", ctypes.c_int64),
                ("pe_eq", ctypes.c_int64), ("kappa", ctypes.c_double),
                ("ohm_model", ctypes.c_int64), ("relativistic", ctypes.c_int64),
                ("c_light", ctypes.c_double), ("open", ctypes.c_int64 * 3),
                ("B0", ctypes.c_void_p)]


class _Species(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("q", ctypes.c_double), ("m", ctypes.c_double),
                ("cell", ctypes.c_void_p), ("ox", ctypes.c_void_p), ("oy", ctypes.c_void_p),
                ("oz", ctypes.c_void_p), ("vx", ctypes.c_void_p), ("vy", ctypes.c_void_p),
                ("vz", ctypes.c_void_p), ("w", ctypes.c_void_p)]


class Diag(ctypes.Structure):
    _fields_ = [("W_K", ctypes.c_double), ("P", ctypes.c_double * 3),
                ("charge", ctypes.c_double), ("W_B", ctypes.c_double),
                ("max_divB", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {"W_K": self.W_K, "P": list(self.P), "charge": self.charge,
                "W_B": self.W_B, "max_divB": self.max_divB}


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            D = ctypes.c_double
            L.hvo_shape.argtypes = [I64, D, D, D, P, P, P, P]
            L.hvo_shape.restype = ctypes.c_int
            L.hvo_gather.argtypes = [P, P, I64, I64, D, D, D, P]
            L.hvo_boris.argtypes = [D, P, P, P]
            L.hvo_boris_rel.argtypes = [D, D, P, P, P]
            L.hvo_move.argtypes = [P, P, P, P, D]
            L.hvo_deposit.argtypes = [P, P, I64, P, P]
            L.hvo_push_deposit.argtypes = [P, P, I64, P, P, P, P, P]
            for nm in ("hvo_curl", "hvo_grad", "hvo_div"):
                getattr(L, nm).argtypes = [P, P, P]
            L.hvo_lap.argtypes = [P, P, I64, P]
            L.hvo_ohm.argtypes = [P, P, P, P, P]
            L.hvo_field_advance.argtypes = [P, P, P, P]
            L.hvo_ohm_pe.argtypes = [P, P, P, P, P, P]
            L.hvo_dpdt.argtypes = [P, P, P, P, P, P]
            L.hvo_field_advance_pe.argtypes = [P, P, P, P, P]
            L.hvo_init_pe.argtypes = [P, P, I64, P, P, P, P, P]
            L.hvo_step_pe.argtypes = [P, P, I64, P, P, P, P, P, P, P, P]
            L.hvo_smooth.argtypes = [P, P, I64, I64]
            L.hvo_extrapolate.argtypes = [I64, P, P, P]
            L.hvo_diag_grid.argtypes = [P, P, P, P, P, P]
            L.hvo_init.argtypes = [P, P, I64, P, P, P, P]
            L.hvo_step.argtypes = [P, P, I64, P, P, P, P, P, P, P]
            L.hvo_sort_stable.argtypes = [P, I64, I64, P, P, P]
            L.hvo_sort_stable.restype = ctypes.c_int
            L.hvo_filter_net.argtypes = [P, P, P, ctypes.c_int, P, P, P]
            L.hvo_filter_apply.argtypes = [P, P, P, D, D, ctypes.c_int, P, P]
            L.hvo_filter_loss_grad.argtypes = [P, P, P, ctypes.c_int, P, P, P]
            L.hvo_filter_loss_grad.restype = D
            L.hvo_ohm_open.argtypes = [P, P, P, P, P]
            L.hvo_field_advance_open.argtypes = [P, P, P, P]
            L.hvo_push_deposit_open.argtypes = [P, P, I64, P, P, P, P, P]
            L.hvo_init_open.argtypes = [P, P, I64, P, P, P, P]
            L.hvo_step_open.argtypes = [P, P, I64, P, P, P, P, P, P, P]
            L.hvo_philox4x32_10.argtypes = [P, P, P]
            L.hvo_inject_nfix.argtypes = [P, D, P]
            L.hvo_inject_nfix.restype = ctypes.c_uint64
            L.hvo_inject.argtypes = [P, I64, D, P, ctypes.c_uint64, I64, P, P, P, I64]
            L.hvo_inject.restype = I64
            L.hvo_max_div.argtypes = [P, P]
            L.hvo_max_div.restype = D
            L.hvo_xcount.argtypes = [P]
            L.hvo_xcount.restype = I64
            L.hvo_set_threads.argtypes = [ctypes.c_int]
            L.hvo_get_threads.restype = ctypes.c_int
            L.hvo_max_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def set_threads(n: int) -> None:
    """Threads of the particle and cell loops (1, the default, for parity)."""
    lib().hvo_set_threads(int(n))


def get_threads() -> int:
    return int(lib().hvo_get_threads())


def max_threads() -> int:
    """Threads OpenMP can use on this host (1 without OpenMP)."""
    return int(lib().hvo_max_threads())


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def make_grid(nx, ny, nz, dx, dy, dz, dt, nsub=1, Te=0.0, gamma_e=1.0, eta=0.0,
              eta_h=0.0, n_floor=0.0, shape="qs", smooth_passes=0,
              field_smooth_passes=0, pe_eq=0, kappa=0.0, ohm_model=0, relativistic=0,
              c_light=0.0, open_axes=(0, 0, 0), B0ext=None) -> Grid:
    """Grid and physics parameters.  open_axes: 1 per axis with open faces
    (Sec. 2.3).  B0ext: a fixed external field [3][ncell] (the B0 of the
    B = B0 + B1 split, Sec. 2.3) or None; the grid keeps a reference."""
    s = SHAPES[shape] if isinstance(shape, str) else int(shape)
    g = Grid(nx, ny, nz, dx, dy, dz, dt, nsub, Te, gamma_e, eta, eta_h, n_floor, s,
             smooth_passes, field_smooth_passes, int(pe_eq), float(kappa), int(ohm_model),
             int(relativistic), float(c_light), (ctypes.c_int64 * 3)(*[int(a) for a in open_axes]),
             None)
    if B0ext is not None:
        b0 = np.ascontiguousarray(np.asarray(B0ext, dtype=np.float64).reshape(3, -1))
        if b0.shape[1] != nx * ny * nz:
            raise ValueError("B0ext must have 3 * ncell values")
        g._b0_keep = b0
        g.B0 = b0.ctypes.data
    return g


def ncell(g: Grid) -> int:
    return g.nx * g.ny * g.nz


@dataclass
class Species:
    """One ion species as FP64 arrays (cell int64; offsets and v [3][n])."""
    q: float
    m: float
    cell: np.ndarray
    off: np.ndarray
    v: np.ndarray
    w: np.ndarray
    _keep: list = field(default_factory=list, repr=False)

    def __post_init__(self):
        self.cell = np.ascontiguousarray(self.cell, dtype=np.int64)
        self.off = _f64(self.off).reshape(3, -1).copy()
        self.v = _f64(self.v).reshape(3, -1).copy()
        self.w = _f64(self.w).copy()

    @property
    def n(self) -> int:
        return int(self.cell.shape[0])

    def struct(self) -> _Species:
        return _Species(self.n, self.q, self.m, self.cell.ctypes.data,
                        self.off[0].ctypes.data, self.off[1].ctypes.data,
                        self.off[2].ctypes.data, self.v[0].ctypes.data,
                        self.v[1].ctypes.data, self.v[2].ctypes.data, self.w.ctypes.data)

    def copy(self) -> "Species":
        return Species(self.q, self.m, self.cell.copy(), self.off.copy(), self.v.copy(),
                       self.w.copy())


def _species_array(sp):
    arr = (_Species * len(sp))(*[s.struct() for s in sp])
    return arr


# ----------------------------------------------------------------------------
# thin wrappers, one per oracle routine
# ----------------------------------------------------------------------------

def shape_weights(shape, d):
    si = np.zeros(8, np.int32)
    sj = np.zeros(8, np.int32)
    sk = np.zeros(8, np.int32)
    wt = np.zeros(8, np.float64)
    s = SHAPES[shape] if isinstance(shape, str) else int(shape)
    nt = lib().hvo_shape(s, float(d[0]), float(d[1]), float(d[2]), _p(si), _p(sj), _p(sk),
                         _p(wt))
    return np.stack([si[:nt], sj[:nt], sk[:nt]], axis=1), wt[:nt].copy()


def gather(g: Grid, F: np.ndarray, cell: int, d) -> np.ndarray:
    F = _f64(F).reshape(-1, ncell(g))
    out = np.zeros(F.shape[0])
    lib().hvo_gather(ctypes.byref(g), _p(F), F.shape[0], int(cell), float(d[0]), float(d[1]),
                     float(d[2]), _p(out))
    return out


def boris(qmdt: float, E, B, v) -> np.ndarray:
    E = _f64(E)
    B = _f64(B)
    v = _f64(v).copy()
    lib().hvo_boris(float(qmdt), _p(E), _p(B), _p(v))
    return v


def boris_rel(qmdt: float, c: float, E, B, u) -> np.ndarray:
    E = _f64(E)
    B = _f64(B)
    u = _f64(u).copy()
    lib().hvo_boris_rel(float(qmdt), float(c), _p(E), _p(B), _p(u))
    return u


def move(g: Grid, cell: int, d, v, frac: float = 1.0):
    c = np.array([cell], np.int64)
    d = _f64(d).copy()
    v = _f64(v)
    lib().hvo_move(ctypes.byref(g), _p(c), _p(d), _p(v), float(frac))
    return int(c[0]), d


def deposit(g: Grid, species) -> tuple[np.ndarray, np.ndarray]:
    n = np.zeros(ncell(g))
    J = np.zeros(3 * ncell(g))
    arr = _species_array(species)
    lib().hvo_deposit(ctypes.byref(g), arr, len(species), _p(n), _p(J))
    return n, J.reshape(3, -1)


def push_deposit(g: Grid, species, E, B):
    E = _f64(E).reshape(3, -1)
    B = _f64(B).reshape(3, -1)
    n = np.zeros(ncell(g))
    J = np.zeros(3 * ncell(g))
    kin = np.zeros(4)
    arr = _species_array(species)
    lib().hvo_push_deposit(ctypes.byref(g), arr, len(species), _p(E), _p(B), _p(n), _p(J),
                           _p(kin))
    return n, J.reshape(3, -1), kin


def _vec_op(name, g, A, ncomp_out):
    A = _f64(A)
    out = np.zeros(ncomp_out * ncell(g))
    getattr(lib(), name)(ctypes.byref(g), _p(A), _p(out))
    return out.reshape(ncomp_out, -1) if ncomp_out > 1 else out


def curl(g, A):
    return _vec_op("hvo_curl", g, _f64(A).reshape(3, -1), 3)


def grad(g, f):
    return _vec_op("hvo_grad", g, _f64(f).reshape(-1), 3)


def div(g, A):
    return _vec_op("hvo_div", g, _f64(A).reshape(3, -1), 1)


def lap(g, A, nc):
    A = _f64(A).reshape(nc, -1)
    out = np.zeros(nc * ncell(g))
    lib().hvo_lap(ctypes.byref(g), _p(A), nc, _p(out))
    return out.reshape(nc, -1)


def ohm(g, B, n, Ji):
    B = _f64(B).reshape(3, -1)
    n = _f64(n).reshape(-1)
    Ji = _f64(Ji).reshape(3, -1)
    E = np.zeros(3 * ncell(g))
    lib().hvo_ohm(ctypes.byref(g), _p(B), _p(n), _p(Ji), _p(E))
    return E.reshape(3, -1)


def field_advance(g, B, n, Ji):
    B = _f64(B).reshape(3, -1).copy()
    n = _f64(n).reshape(-1)
    Ji = _f64(Ji).reshape(3, -1)
    lib().hvo_field_advance(ctypes.byref(g), _p(B), _p(n), _p(Ji))
    return B


def ohm_pe(g, B, n, Ji, pe):
    B = _f64(B).reshape(3, -1)
    n = _f64(n).reshape(-1)
    Ji = _f64(Ji).reshape(3, -1)
    pe = _f64(pe).reshape(-1)
    E = np.zeros(3 * ncell(g))
    lib().hvo_ohm_pe(ctypes.byref(g), _p(B), _p(n), _p(Ji), _p(pe), _p(E))
    return E.reshape(3, -1)


def dpdt(g, B, pe, n, Ji):
    B = _f64(B).reshape(3, -1)
    pe = _f64(pe).reshape(-1)
    n = _f64(n).reshape(-1)
    Ji = _f64(Ji).reshape(3, -1)
    out = np.zeros(ncell(g))
    lib().hvo_dpdt(ctypes.byref(g), _p(B), _p(pe), _p(n), _p(Ji), _p(out))
    return out


def field_advance_pe(g, B, pe, n, Ji):
    B = _f64(B).reshape(3, -1).copy()
    pe = _f64(pe).reshape(-1).copy()
    n = _f64(n).reshape(-1)
    Ji = _f64(Ji).reshape(3, -1)
    lib().hvo_field_advance_pe(ctypes.byref(g), _p(B), _p(pe), _p(n), _p(Ji))
    return B, pe


def smooth(g, q, passes):
    q = _f64(q).copy()
    nc = q.size // ncell(g)
    lib().hvo_smooth(ctypes.byref(g), _p(q), nc, int(passes))
    return q


def extrapolate(half, prev):
    half = _f64(half)
    prev = _f64(prev)
    out = np.zeros_like(half)
    lib().hvo_extrapolate(half.size, _p(half), _p(prev), _p(out))
    return out


def diag_grid(g, B, n):
    B = _f64(B).reshape(3, -1)
    n = _f64(n).reshape(-1)
    wb = np.zeros(1)
    ch = np.zeros(1)
    md = np.zeros(1)
    lib().hvo_diag_grid(ctypes.byref(g), _p(B), _p(n), _p(wb), _p(ch), _p(md))
    return float(wb[0]), float(ch[0]), float(md[0])


def sort_stable(keys, nkeys):
    keys = np.ascontiguousarray(keys, dtype=np.int64)
    n = keys.shape[0]
    perm = np.zeros(n, np.int64)
    counts = np.zeros(nkeys, np.int64)
    offsets = np.zeros(nkeys + 1, np.int64)
    rc = lib().hvo_sort_stable(_p(keys), n, int(nkeys), _p(perm), _p(counts), _p(offsets))
    if rc != 0:
        raise ValueError("key out of range")
    return perm, counts, offsets


def sort_pred_coeffs(params):
    """The library's key-cell prediction coefficients per axis (FP32):
    1.375 * sort_every * dt / Delta, 0 on single-cell axes, with open faces
    and without sorting (``include/hv.h``, sort_every)."""
    p = params
    on = p.get("sort_every", 0) > 0 and not p.get("open_faces", 0)
    return tuple(np.float32(1.375 * p["sort_every"] * p["dt"] / p[d]) if on and p[n] > 1
                 else np.float32(0.0)
                 for n, d in (("nx", "dx"), ("ny", "dy"), ("nz", "dz")))


def supercell_keys(cell, nx, ny, nz, tile, off=None, v=None, pc=None):
    """Keys of the library's documented ion order (``include/hv.h``,
    hv_query / hv_get_tile_offsets), restated here so that the oracle side
    never calls the product: for linear cell c = i + nx (j + ny k) and tile
    extents (tx, ty, tz), key = tile index * (tx ty tz) + the cell's linear
    index inside its tile, both x fastest.  With off, v [3][n] (FP32 state)
    and pc (sort_pred_coeffs) the key is that of the predicted cell: the
    cell moved by one along each axis where off + v * pc (FP32, product and
    sum rounded separately) is >= 1 or < -1, periodically.  The paper
    prescribes no ion order; sorting only permutes the oracle's FP64
    summation order."""
    c = np.asarray(cell, dtype=np.int64)
    tx, ty, tz = (int(t) for t in tile)
    i, j, k = c % nx, (c // nx) % ny, c // (nx * ny)
    if off is not None:
        o = np.asarray(off, dtype=np.float32)
        w = np.asarray(v, dtype=np.float32)
        sh = []
        for a in range(3):
            q = o[a] + w[a] * np.float32(pc[a])
            sh.append((q >= np.float32(1.0)).astype(np.int64) - (q < np.float32(-1.0)))
        i, j, k = (i + sh[0]) % nx, (j + sh[1]) % ny, (k + sh[2]) % nz
    ntx, nty = -(-nx // tx), -(-ny // ty)
    t = (i // tx) + ntx * ((j // ty) + nty * (k // tz))
    return t * (tx * ty * tz) + (i % tx) + tx * ((j % ty) + ty * (k % tz))


def supercell_nkeys(nx, ny, nz, tile) -> int:
    tx, ty, tz = (int(t) for t in tile)
    return (-(-nx // tx)) * (-(-ny // ty)) * (-(-nz // tz)) * tx * ty * tz


FILTER_NPARAM = 3492


def bf16(a) -> np.ndarray:
    """Round to bfloat16 (nearest even) and return as float64."""
    f = np.asarray(a, dtype=np.float32).copy()
    u = f.view(np.uint32)
    lsb = (u >> 16) & 1
    r = ((u.astype(np.uint64) + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    special = (u & 0x7F800000) == 0x7F800000
    r[special] = u[special]
    return r.view(np.float32).astype(np.float64)


def filter_net(g, params, x, round_bf16=True):
    """Network output f for normalised moments x [4][ncell]; also h1, h2."""
    P = _f64(params)
    x = _f64(x).reshape(4, -1)
    nce = ncell(g)
    f = np.zeros(4 * nce)
    h1 = np.zeros(16 * nce)
    h2 = np.zeros(16 * nce)
    lib().hvo_filter_net(ctypes.byref(g), _p(P), _p(x), int(round_bf16), _p(f), _p(h1), _p(h2))
    return f.reshape(4, -1), h1.reshape(16, -1), h2.reshape(16, -1)


def filter_apply(g, params, scale, nmin, rmax, m, round_bf16=True):
    P = _f64(params)
    s = _f64(scale)
    m = _f64(m).reshape(4, -1)
    y = np.zeros_like(m)
    lib().hvo_filter_apply(ctypes.byref(g), _p(P), _p(s), float(nmin), float(rmax),
                           int(round_bf16), _p(m), _p(y))
    return y


def filter_loss_grad(g, params, scale, m, target, round_bf16=True):
    P = _f64(params)
    s = _f64(scale)
    m = _f64(m).reshape(4, -1)
    t = _f64(target).reshape(4, -1)
    grad = np.zeros(FILTER_NPARAM)
    loss = lib().hvo_filter_loss_grad(ctypes.byref(g), _p(P), _p(s), int(round_bf16), _p(m),
                                      _p(t), _p(grad))
    return loss, grad


def xcount(g: Grid) -> int:
    """Cells of the grid extended by one ghost cell beyond every open face."""
    return int(lib().hvo_xcount(ctypes.byref(g)))


def xshape(g: Grid):
    """(Nz, Ny, Nx) of the extended grid."""
    o = [int(a) for a in g.open]
    return (g.nz + 2 * o[2], g.ny + 2 * o[1], g.nx + 2 * o[0])


def ohm_open(g, B1, n, Ji):
    """E on the extended grid (open faces) from interior B1, n, Ji."""
    B1 = _f64(B1).reshape(3, -1)
    n = _f64(n).reshape(-1)
    Ji = _f64(Ji).reshape(3, -1)
    E = np.zeros(3 * xcount(g))
    lib().hvo_ohm_open(ctypes.byref(g), _p(B1), _p(n), _p(Ji), _p(E))
    return E.reshape(3, -1)


def max_div(g, B) -> float:
    """max |div B| over the interior (open faces: ghost copies)."""
    B = _f64(B).reshape(3, -1)
    return float(lib().hvo_max_div(ctypes.byref(g), _p(B)))


def field_advance_open(g, B1, n, Ji):
    B1 = _f64(B1).reshape(3, -1).copy()
    lib().hvo_field_advance_open(ctypes.byref(g), _p(B1), _p(_f64(n).reshape(-1)),
                                 _p(_f64(Ji).reshape(3, -1)))
    return B1


def extended_interior(g, F):
    """Interior cells [nc][ncell] of an extended field [nc][next]."""
    F = np.asarray(F)
    nc = F.shape[0]
    Nz, Ny, Nx = xshape(g)
    o = [int(a) for a in g.open]
    G = F.reshape(nc, Nz, Ny, Nx)[:, o[2]:o[2] + g.nz, o[1]:o[1] + g.ny, o[0]:o[0] + g.nx]
    return np.ascontiguousarray(G).reshape(nc, -1)


class InjectFace(ctypes.Structure):
    """Drifting Maxwellian injected through an open face (face 0 -x, 1 +x,
    2 -y, 3 +y, 4 -z, 5 +z): density n, flow u, temperature T, weight w."""
    _fields_ = [("face", ctypes.c_int64), ("n", ctypes.c_double), ("u", ctypes.c_double * 3),
                ("T", ctypes.c_double), ("w", ctypes.c_double)]


def inject_face(face, n, u, T, w) -> InjectFace:
    return InjectFace(int(face), float(n), (ctypes.c_double * 3)(*[float(a) for a in u]),
                      float(T), float(w))


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().hvo_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def inject_nfix(g, m, f: InjectFace) -> int:
    return int(lib().hvo_inject_nfix(ctypes.byref(g), float(m), ctypes.byref(f)))


def inject(g, s_idx, m, f: InjectFace, seed, step):
    """Ions injected through one face at one step: (cell, off [3][k], v [3][k])."""
    L = lib()
    k = int(L.hvo_inject(ctypes.byref(g), int(s_idx), float(m), ctypes.byref(f),
                         int(seed), int(step), None, None, None, 0))
    cell = np.zeros(k, np.int64)
    off = np.zeros((3, k))
    v = np.zeros((3, k))
    if k:
        L.hvo_inject(ctypes.byref(g), int(s_idx), float(m), ctypes.byref(f), int(seed),
                     int(step), _p(cell), _p(off), _p(v), k)
    return cell, off, v


class Sim:
    """Whole-state oracle simulation: species plus B, E and the previous
    (half-step) moments, advanced by ``hvo_step``.  B0 is the initial
    (total) magnetic field; with an external field on the grid (B0ext of
    make_grid) the advanced state ``B`` is B1 = B0 - B0ext and
    ``B_total()`` adds the external part back."""

    def __init__(self, g: Grid, species, B0, inject=None, seed=0):
        """inject: list of (species index, InjectFace) for open faces; seed
        keys the injection's random numbers."""
        self.g = g
        self.inject = list(inject or [])
        self.seed = int(seed)
        self.species = [s.copy() for s in species]
        nce = ncell(g)
        self.B = _f64(B0).reshape(3, nce).copy()
        ext = getattr(g, "_b0_keep", None)
        if ext is not None:
            self.B -= ext
        self.E = np.zeros((3, nce))
        self.n_prev = np.zeros(nce)
        self.J_prev = np.zeros((3, nce))
        self.n_ext = np.zeros(nce)
        self.J_ext = np.zeros((3, nce))
        self.step_count = 0
        self.diags: list[dict] = []
        arr = _species_array(self.species)
        self.pe = np.zeros(nce) if g.pe_eq else None
        self.open = any(int(a) for a in g.open)
        if self.open:
            # E lives on the grid extended by the ghost cells of open faces
            self.Ex = np.zeros((3, xcount(g)))
            lib().hvo_init_open(ctypes.byref(g), arr, len(self.species), _p(self.B),
                                _p(self.Ex), _p(self.n_prev), _p(self.J_prev))
            self.E = extended_interior(g, self.Ex)
        elif g.pe_eq:
            lib().hvo_init_pe(ctypes.byref(g), arr, len(self.species), _p(self.B), _p(self.E),
                              _p(self.pe), _p(self.n_prev), _p(self.J_prev))
        else:
            lib().hvo_init(ctypes.byref(g), arr, len(self.species), _p(self.B), _p(self.E),
                           _p(self.n_prev), _p(self.J_prev))

    def B_total(self) -> np.ndarray:
        ext = getattr(self.g, "_b0_keep", None)
        return self.B + ext if ext is not None else self.B

    def sort(self, key_fn=None):
        """Apply the stable counting sort to every species, by cell or by
        key_fn(cell) (integer keys >= 0)."""
        for s in self.species:
            keys = s.cell if key_fn is None else np.asarray(key_fn(s.cell), dtype=np.int64)
            nk = int(keys.max()) + 1 if keys.size else 1
            perm, _, _ = sort_stable(keys, max(nk, ncell(self.g)))
            s.cell = np.ascontiguousarray(s.cell[perm])
            s.off = np.ascontiguousarray(s.off[:, perm])
            s.v = np.ascontiguousarray(s.v[:, perm])
            s.w = np.ascontiguousarray(s.w[perm])

    def step(self, nsteps: int = 1, sort_every: int = 0, key_fn=None):
        for _ in range(nsteps):
            if sort_every > 0 and self.step_count % sort_every == 0:
                self.sort(key_fn)
            arr = _species_array(self.species)
            d = Diag()
            if self.open:
                lib().hvo_step_open(ctypes.byref(self.g), arr, len(self.species), _p(self.B),
                                    _p(self.Ex), _p(self.n_prev), _p(self.J_prev),
                                    _p(self.n_ext), _p(self.J_ext), ctypes.byref(d))
                self.E = extended_interior(self.g, self.Ex)
                for k, s in enumerate(self.species):  # absorbed ions were compacted out
                    m = int(arr[k].n)
                    s.cell, s.w = s.cell[:m].copy(), s.w[:m].copy()
                    s.off, s.v = s.off[:, :m].copy(), s.v[:, :m].copy()
                # injected ions appended after the push, species by species,
                # faces in the order given (they deposit from the next step)
                for s_idx, f in self.inject:
                    sp = self.species[s_idx]
                    c, o, vv = inject(self.g, s_idx, sp.m, f, self.seed, self.step_count)
                    sp.cell = np.concatenate([sp.cell, c])
                    sp.off = np.ascontiguousarray(np.concatenate([sp.off, o], axis=1))
                    sp.v = np.ascontiguousarray(np.concatenate([sp.v, vv], axis=1))
                    sp.w = np.concatenate([sp.w, np.full(c.shape[0], f.w)])
            elif self.pe is not None:
                lib().hvo_step_pe(ctypes.byref(self.g), arr, len(self.species), _p(self.B),
                                  _p(self.E), _p(self.pe), _p(self.n_prev), _p(self.J_prev),
                                  _p(self.n_ext), _p(self.J_ext), ctypes.byref(d))
            else:
                lib().hvo_step(ctypes.byref(self.g), arr, len(self.species), _p(self.B),
                               _p(self.E), _p(self.n_prev), _p(self.J_prev), _p(self.n_ext),
                               _p(self.J_ext), ctypes.byref(d))
            self.step_count += 1
            self.diags.append(d.as_dict())
        return self.diags[-1] if self.diags else None
