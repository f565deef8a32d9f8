"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports
every function include/hv.h declares, its structs have the declared layout,
and host-side argument checks reject bad input before touching a GPU."""
import ctypes
import math
import os
import re

import pytest

from paper_2305_05600_gb300 import hv

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hv.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(hv_[a-z_]+)\s*\(", src)
    return sorted(set(n for n in names if not n.endswith("_fn")))


def test_library_exports_every_declared_function():
    L = hv.lib()
    names = declared_functions()
    assert "hv_step" in names and "hv_init_grid" in names
    for n in names:
        assert hasattr(L, n), n
    assert set(names) <= set(hv.EXPORTS)


def test_struct_layouts():
    assert ctypes.sizeof(hv.Params) == 144
    assert ctypes.sizeof(hv.Diag) == 8 * 9 + 8
    assert ctypes.sizeof(hv.Prof) == 8 * 14


def _params(**kw):
    d = dict(nx=16, ny=1, nz=8, dx=0.5, dy=1.0, dz=0.5, dt=0.01, nsub=10, Te=0.1,
             n_floor=0.05, shape="qs")
    d.update(kw)
    return hv.params_from(d)


def _init_status(p):
    out = ctypes.c_void_p()
    rc = hv.lib().hv_init_grid(ctypes.byref(p), None, None, ctypes.byref(out))
    return rc, out.value


@pytest.mark.parametrize("bad", [dict(nx=0), dict(nsub=0), dict(dx=-1.0), dict(dt=math.nan),
                                 dict(shape=5), dict(n_floor=0.0), dict(smooth_passes=-1),
                                 dict(Te=-1.0), dict(eta=-1e-3), dict(field_smooth_passes=-1),
                                 dict(field_smooth_passes=65), dict(pe_eq=2),
                                 dict(pe_eq=1, kappa=-1.0), dict(kappa=math.inf),
                                 dict(ohm_model=3), dict(relativistic=1),
                                 dict(relativistic=1, c_light=-1.0)])
def test_init_rejects_bad_parameters_on_host(bad):
    rc, h = _init_status(_params(**bad))
    assert rc == hv.HV_EINVAL and not h
    assert len(hv.hv_last_error()) > 0


def test_init_rejects_heat_conduction_limit_violation():
    # h (gamma-1) kappa / n_floor * (4/dx^2 + 4/dz^2) = 0.001 * 2/3 * 10 / 0.05 * 32 = 4.3 > 2
    rc, h = _init_status(_params(pe_eq=1, kappa=10.0, gamma_e=5.0 / 3.0))
    assert rc == hv.HV_ECFL and not h
    assert "heat" in hv.hv_last_error()


def test_init_rejects_whistler_limit_violation():
    # dt/nsub = 0.1 >= dx^2/pi = 0.0796 (Sec. 2.1)
    rc, h = _init_status(_params(dt=1.0, nsub=10))
    assert rc == hv.HV_ECFL and not h
    assert "whistler" in hv.hv_last_error()


def test_sort_keys_rejects_bad_sizes_on_host():
    L = hv.lib()
    assert L.hv_sort_keys(None, -1, 4, None, None, None) == hv.HV_EINVAL
    assert L.hv_sort_keys(None, 4, 0, None, None, None) == hv.HV_EINVAL


def test_allocator_hooks_must_come_in_pairs():
    L = hv.lib()
    a = hv.ALLOC_FN(lambda n, s, u: None)
    assert L.hv_set_allocator(a, hv.FREE_FN(0), None) == hv.HV_EINVAL
    assert L.hv_set_allocator(hv.ALLOC_FN(0), hv.FREE_FN(0), None) == hv.HV_OK


def test_error_word_maps_to_status_without_a_gpu():
    """The device error word -> status mapping every synchronising call
    uses (the failure-detection codes of include/hv.h), checked on the
    host: each bit alone and the precedence when several are set."""
    st = hv.hv_error_status
    assert st(0) == hv.HV_OK
    assert st(1) == hv.HV_ECFL
    assert st(2) == hv.HV_ENAN
    assert st(4) == hv.HV_ECUDA
    assert st(8) == hv.HV_ETIMEOUT
    assert "bounded device wait" in hv.hv_last_error()
    assert st(8 | 1) == hv.HV_ECFL
    assert st(8 | 2 | 1) == hv.HV_ENAN
    assert st(8 | 4) == hv.HV_ECUDA


def test_context_calls_reject_null_on_host():
    L = hv.lib()
    assert L.hv_inject_error(None, 8) == hv.HV_EINVAL
    assert L.hv_get_tile_offsets(None, 0, None) == hv.HV_EINVAL
    assert L.hv_diag_async(None) == hv.HV_EINVAL
    assert L.hv_diag_wait(None, None) == hv.HV_EINVAL


def test_noalloc_binding_rejects_host_tensors():
    torch = pytest.importorskip("torch")
    keys = torch.zeros(8, dtype=torch.int32)
    perm = torch.zeros(8, dtype=torch.int32)
    with pytest.raises(TypeError):
        hv.hv_sort_keys_noalloc(keys, 4, perm)


@pytest.mark.parametrize("bad", [dict(open_faces=8), dict(open_faces=2),
                                 dict(open_faces=1, pe_eq=1), dict(open_faces=1, smooth_passes=1),
                                 dict(open_faces=4, ohm_model=1),
                                 dict(open_faces=1, relativistic=1, c_light=10.0)])
def test_open_faces_rejected_outside_their_scope(bad):
    """Open faces (Sec. 2.3): bits 1, 2, 4 only, an open axis needs more than
    one cell (the 2D layout's y axis has one), hybrid Ohm's law with the
    equation of state, no smoothing, no relativistic push."""
    rc, h = _init_status(_params(**bad))
    assert rc == hv.HV_EINVAL and not h


def test_capacity_error_bit_maps_to_enomem():
    assert hv.hv_error_status(16) == hv.HV_ENOMEM
    assert "slot" in hv.hv_last_error()
    assert hv.hv_error_status(16 | 8) == hv.HV_ETIMEOUT
