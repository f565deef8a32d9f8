"""Host-side checks of the expanding-cloud workload and of the front analysis
used by the shape / smoothing comparison (Sec. 3.2).  CPU only."""
import math

import numpy as np

from paper_2305_05600_gb300 import explosion as X
from paper_2305_05600_gb300 import inputs as I


def test_workload_debris_mass_and_radial_speed():
    wl = I.explosion2d(nx=64, nz=48, length=125.0, ppc=4, n_debris=20000, r_m=20.0, mach=15.0,
                       seed=1)
    p = wl.params
    s = wl.species[0]
    assert p["field_smooth_passes"] == p["smooth_passes"] == 0
    assert s.off.min() >= -1.0 and s.off.max() < 1.0 and np.all(s.off[1] == 0)
    w = s.w.astype(np.float64)
    nb = 64 * 48 * 4
    # the background weights add up to n0 times the box area; the debris to
    # a disc of radius r_m of the background
    bg = np.isclose(w, p["dx"] * p["dz"] / 4, rtol=1e-6)
    assert bg.sum() == nb
    assert abs(w[bg].sum() - 64 * 48 * p["dx"] * p["dz"]) < 1e-3 * w[bg].sum()
    assert abs(w[~bg].sum() - math.pi * 20.0 ** 2) < 1e-3 * math.pi * 20.0 ** 2
    # debris: in-plane velocity radial from the centre at about mach v_A
    x, _, z = I.positions(p, s.cell[~bg].astype(np.int64), s.off[:, ~bg].astype(np.float64))
    rx, rz = x - 0.5 * 64 * p["dx"], z - 0.5 * 48 * p["dz"]
    r = np.hypot(rx, rz)
    vr = (s.v[0, ~bg] * rx + s.v[2, ~bg] * rz) / r
    assert abs(np.median(vr) - 15.0) < 0.1
    assert np.mean(r) < 0.2 * 20.0 * 1.5  # Gaussian of width r_m / 10


def rings(nx, dx, radii, width=2.0):
    """Density 1 with concentric rings of density 3 at the given radii
    (cells within `width` cells of the radius) about the box centre."""
    c = (np.arange(nx) + 0.5) * dx
    Xc, Zc = np.meshgrid(c, c)
    r = np.hypot(Xc - 0.5 * nx * dx, Zc - 0.5 * nx * dx)
    n = np.ones_like(r)
    for rad in radii:
        n[np.abs(r - rad) < width * dx] = 3.0
    return n


def test_layer_count_uses_hysteresis():
    assert X.layer_count(np.array([1.0, 1.6, 1.3, 1.7, 1.0])) == 1  # dip not below 1.2
    assert X.layer_count(np.array([1.0, 1.6, 1.1, 1.7, 1.0])) == 2
    assert X.layer_count(np.array([2.0, 1.0, 1.0, 1.9, 1.0, 1.6])) == 3
    assert X.layer_count(np.ones(10)) == 0


def test_one_shell_is_one_layer_at_its_radius():
    dx = 2.0
    n = rings(256, dx, [150.0])
    for ang in X.SECTORS.values():
        m = X.sector_metrics(n, dx, ang)
        assert m["layers"] == 1.0 and m["multi"] == 0.0
        assert abs(m["r_lead"] - 154.0) < dx  # outer edge of the shell
        assert abs(m["r_peak"] - 150.0) < 3 * dx
        assert abs(m["n_max"] - 3.0) < 0.1


def test_split_shell_counts_two_layers_and_the_leading_edge():
    dx = 2.0
    n = rings(256, dx, [120.0, 170.0])
    m = X.sector_metrics(n, dx, X.SECTORS["across_B0"])
    assert m["layers"] == 2.0 and m["multi"] == 1.0
    assert abs(m["r_lead"] - 174.0) < dx


def test_sectors_see_only_their_directions():
    """A shell split only along x (the B0 direction) shows in the along-B0
    sector and not across B0."""
    dx = 2.0
    n = rings(256, dx, [120.0])
    c = (np.arange(256) + 0.5) * dx
    Xc, Zc = np.meshgrid(c, c)
    r = np.hypot(Xc - 256.0, Zc - 256.0)
    along = np.abs(Zc - 256.0) < 0.2 * np.abs(Xc - 256.0)
    n[along & (np.abs(r - 180.0) < 2 * dx)] = 3.0
    ma = X.sector_metrics(n, dx, X.SECTORS["along_B0"], half_width=0.15)
    mc = X.sector_metrics(n, dx, X.SECTORS["across_B0"])
    assert ma["layers"] == 2.0 and mc["layers"] == 1.0


def test_hose_channel_measures_kink_and_width():
    from paper_2305_05600_gb300 import hose as H
    nz, nx, dz = 64, 32, 0.25
    z = (np.arange(nz) + 0.5) * dz
    x = np.arange(nx)
    # a Gaussian channel of width 1 whose centre moves as 0.5 sin(2 pi x / nx)
    zc = 8.0 + 0.5 * np.sin(2 * np.pi * x / nx)
    n = -np.exp(-0.5 * (z[:, None] - zc[None, :]) ** 2)  # electrons: negative density
    kink, width = H.channel(n, dz)
    assert abs(kink - 0.5 / np.sqrt(2)) < 0.01
    assert abs(width - 1.0) < 0.02
    kink0, _ = H.channel(-np.exp(-0.5 * (z[:, None] - 8.0) ** 2) * np.ones((1, nx)), dz)
    assert kink0 < 1e-12
