"""Whole-method pin of the oracle: the parallel Alfven/whistler dispersion of
the hybrid model (Sec. 2.1: cold ions, massless electrons, Hall term).

For parallel propagation with cold ions the two circularly polarised branches
obey omega = k v_A (+- k d_i / 2 + sqrt(1 + (k d_i / 2)^2)), + for the
right-hand (whistler) branch and - for the left-hand (ion-cyclotron) branch.
A linearly polarised dB_y = a sin(k x) splits into both; the complex Fourier
amplitude b(t) = sum_x (B_y + i B_z) exp(-i k x) is then a sum of two
exponentials exp(+i w_R t) + exp(-i w_L t), fitted here by second-order
linear prediction (Prony).  CPU only; about 15 s."""
import numpy as np
import pytest

from paper_2305_05600_gb300 import inputs as I
from tests.helpers import oracle_sim


def prony2(b, T):
    """Two complex frequencies of samples b_n ~ sum_j c_j exp(-i w_j n T)."""
    A = np.stack([b[0:-2], b[1:-1]], axis=1)
    coef, *_ = np.linalg.lstsq(A, b[2:], rcond=None)
    z = np.roots([1.0, -coef[1], -coef[0]])
    return 1j * np.log(z) / T


@pytest.mark.slow
def test_hybrid_parallel_dispersion_within_one_percent():
    wl = I.whistler1d(ppc=128, steps=2000, dt=0.05, nsub=5)
    sim = oracle_sim(wl)
    p = wl.params
    nx = p["nx"]
    x = (np.arange(nx) + 0.5) * p["dx"]
    k = 2 * np.pi / (nx * p["dx"])
    ph = np.exp(-1j * k * x)
    every = 2
    samples = []
    for s in range(wl.steps):
        if s % every == 0:
            samples.append(((sim.B[1] + 1j * sim.B[2]) * ph).sum() / nx)
        sim.step(1)
    om = prony2(np.array(samples), p["dt"] * every)
    w_R = k * (k / 2 + np.sqrt(1 + k * k / 4))
    w_L = k * (-k / 2 + np.sqrt(1 + k * k / 4))
    re = np.sort(om.real)
    # right-hand branch rotates as exp(+i w t) in this convention
    assert abs(-re[0] - w_R) < 0.01 * w_R, (om, w_R)
    assert abs(re[1] - w_L) < 0.01 * w_L, (om, w_L)
    # weakly damped, not growing
    assert np.all(np.abs(om.imag) < 0.01 * w_R)
