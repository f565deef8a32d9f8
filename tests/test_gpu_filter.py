"""GPU parity of the learned moment filter (tensor-core bf16 convolutions,
gate, binomial fallback) against the oracle with the same bf16 parameters
and rounding points.

Tolerance: both sides round the input and the two hidden layers to bf16; the
GPU accumulates in FP32, the oracle in FP64, so an activation whose FP32 and
FP64 pre-activations straddle a bf16 rounding boundary differs by one bf16
ulp (2^-8 relative) on the two sides.  Such flips are rare and perturb f by
about |W| 2^-8 |h|; the test bounds the relative L2 error of the filtered
moments by 1e-3 and the element-wise error by 2^-6 of the channel's range.
Cells whose gate decision lies within 1e-3 of its threshold are excluded
from the element-wise check (the decision may legitimately differ)."""
import numpy as np
import pytest

import oracle as O
from paper_2305_05600_gb300 import inputs as I
from tests.helpers import oracle_grid

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hvmod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_05600_gb300 import hv
    hv.lib()
    hv.hv_set_allocator(True)
    return hv


def random_params(rng, scale=0.15):
    P = rng.normal(size=O.FILTER_NPARAM) * scale
    return O.bf16(P)


def test_filter_matches_oracle(hvmod):
    rng = np.random.default_rng(99)
    wl = I.harris(nx=40, nz=24, ppc=4, dx=0.25, seed=3)
    p = wl.params
    ctx = hvmod.hv_init_grid(p, wl.B0)
    nc = p["nx"] * p["nz"]
    m = np.zeros((4, nc))
    m[0] = rng.uniform(0.02, 1.5, nc)
    m[1:] = rng.normal(size=(3, nc)) * 0.3
    m = m.astype(np.float32).astype(np.float64)
    P = random_params(rng)
    scale = np.array([1.0, 0.5, 0.5, 0.5])
    nmin, rmax = 0.1, 0.5
    hvmod.hv_set_filter(ctx, P, scale, nmin, rmax)
    y = hvmod.hv_filter_moments(ctx, m.reshape(4, p["nz"], 1, p["nx"])).reshape(4, -1)
    g = oracle_grid(p)
    yo = O.filter_apply(g, P, scale, nmin, rmax, m, round_bf16=True)
    # gate margins (oracle): exclude cells near the residual threshold
    x = m / scale[:, None]
    f, _, _ = O.filter_net(g, P, x, round_bf16=True)
    ref = np.maximum(m[0], p["n_floor"])
    margin = np.abs(np.abs(scale[0] * f[0]) - rmax * ref) / (rmax * ref)
    keep = margin > 1e-3
    assert keep.mean() > 0.95
    fell_back = (m[0] < nmin) | (np.abs(scale[0] * f[0]) > rmax * ref)
    assert 0.05 < fell_back.mean() < 0.95  # both branches exercised
    err = np.linalg.norm((y - yo)[:, keep]) / np.linalg.norm(yo[:, keep])
    assert err < 1e-3, err
    rng_ch = yo.max(axis=1) - yo.min(axis=1)
    assert (np.abs(y - yo)[:, keep] <= 2 ** -6 * rng_ch[:, None]).all()
    ctx.close()


def test_zero_filter_is_identity_on_gpu(hvmod):
    wl = I.harris(nx=32, nz=16, ppc=4, dx=0.25, seed=4)
    p = wl.params
    ctx = hvmod.hv_init_grid(p, wl.B0)
    nc = p["nx"] * p["nz"]
    rng = np.random.default_rng(5)
    m = rng.uniform(0.2, 1.0, (4, nc)).astype(np.float32)
    hvmod.hv_set_filter(ctx, np.zeros(O.FILTER_NPARAM), (1, 1, 1, 1), 0.0, 1e9)
    y = hvmod.hv_filter_moments(ctx, m.reshape(4, p["nz"], 1, p["nx"])).reshape(4, -1)
    assert np.array_equal(y, m)
    ctx.close()


def test_step_with_filter_matches_oracle_composition(hvmod):
    """Two steps with the filter in place of the smoothing, against the
    oracle's step composed from its routines (push + deposit, filter,
    extrapolation, subcycled field advance, Ohm)."""
    rng = np.random.default_rng(11)
    wl = I.harris(nx=48, nz=32, ppc=16, dx=0.25, seed=12, sort_every=0)
    p = wl.params
    P = random_params(rng, 0.05)
    scale = np.array([1.0, 0.5, 0.5, 0.5])
    nmin, rmax = 0.1, 0.3
    ctx = hvmod.load_workload(wl)
    hvmod.hv_set_filter(ctx, P, scale, nmin, rmax)
    hvmod.hv_step(ctx, 2)
    mg = hvmod.hv_moments(ctx)
    g = oracle_grid(p)
    from tests.helpers import oracle_species
    sp = oracle_species(wl)
    B = wl.B0.astype(np.float64).reshape(3, -1)
    n0, J0 = O.deposit(g, sp)
    prev = O.filter_apply(g, P, scale, nmin, rmax, np.vstack([n0[None], J0]))
    E = O.ohm(g, B, prev[0], prev[1:])
    for _ in range(2):
        n, J, _ = O.push_deposit(g, sp, E, B)
        half = O.filter_apply(g, P, scale, nmin, rmax, np.vstack([n[None], J]))
        ext = O.extrapolate(half, prev)
        B = O.field_advance(g, B, half[0], half[1:])
        E = O.ohm(g, B, ext[0], ext[1:])
        prev = half
    err_n = np.linalg.norm(mg["n"].reshape(-1) - prev[0]) / np.linalg.norm(prev[0])
    err_B = np.linalg.norm(mg["B"].reshape(3, -1) - B) / np.linalg.norm(B)
    assert err_n < 1e-3, err_n
    assert err_B < 1e-6, err_B
    ctx.close()


def test_training_gradient_matches_oracle(hvmod):
    """Loss and gradient of a batch of two pairs against the oracle (FP64
    backward through the same bf16-rounded forward).  The GPU rounds the
    back-propagated signals to bf16 for the tensor-core convolutions
    (relative 2^-9 per value), so the gradient is compared by relative L2
    (<= 3e-2) and direction (cosine >= 0.999); the loss to 1e-3."""
    rng = np.random.default_rng(21)
    p = I.base_params(32, 1, 32, 0.25, 1.0, 0.25, 0.02, 10, Te=0.1)
    ctx = hvmod.hv_init_grid(p, None)
    nc = 32 * 32
    P = random_params(rng, 0.2)
    scale = np.array([1.0, 0.5, 0.5, 0.5])
    hvmod.hv_filter_train_init(ctx, P, scale)
    ms, ts = [], []
    for b in range(2):
        t = np.zeros((4, nc))
        t[0] = 1.0 + 0.3 * rng.normal(size=nc)
        t[1:] = 0.2 * rng.normal(size=(3, nc))
        m = t + 0.1 * rng.normal(size=t.shape)
        ms.append(m.astype(np.float32))
        ts.append(t.astype(np.float32))
    m = np.stack(ms).reshape(2, 4, 32, 1, 32)
    t = np.stack(ts).reshape(2, 4, 32, 1, 32)
    loss, grad = hvmod.hv_filter_grad(ctx, m, t)
    g = oracle_grid(p)
    lo, go = 0.0, np.zeros(O.FILTER_NPARAM)
    for b in range(2):
        l_b, g_b = O.filter_loss_grad(g, P, scale, ms[b].astype(np.float64),
                                      ts[b].astype(np.float64), round_bf16=True)
        lo += l_b / 2
        go += g_b / 2
    assert abs(loss - lo) < 1e-3 * lo, (loss, lo)
    rel = np.linalg.norm(grad - go) / np.linalg.norm(go)
    cos = grad.dot(go) / (np.linalg.norm(grad) * np.linalg.norm(go))
    assert rel < 3e-2 and cos > 0.999, (rel, cos)
    ctx.close()


def test_training_reduces_denoising_loss(hvmod):
    """Adam steps on noisy/clean pairs lower the loss and the trained
    parameters move the filtered moments toward the clean ones."""
    rng = np.random.default_rng(22)
    p = I.base_params(64, 1, 32, 0.25, 1.0, 0.25, 0.02, 10, Te=0.1)
    ctx = hvmod.hv_init_grid(p, None)
    x = (np.arange(64) + 0.5) / 64
    z = (np.arange(32) + 0.5) / 32
    X, Z = np.meshgrid(x, z)
    clean = np.zeros((4, 32, 64))
    clean[0] = 1.0 + 0.3 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Z)
    clean[1] = 0.2 * np.cos(2 * np.pi * Z)
    clean[2] = 0.1 * np.sin(4 * np.pi * X)
    noisy = [clean + 0.15 * rng.normal(size=clean.shape) for _ in range(4)]
    m = np.stack(noisy).reshape(4, 4, 32, 1, 64).astype(np.float32)
    t = np.stack([clean] * 4).reshape(4, 4, 32, 1, 64).astype(np.float32)
    hvmod.hv_filter_train_init(ctx, np.zeros(O.FILTER_NPARAM) + 0.01 * rng.normal(size=O.FILTER_NPARAM))
    first = hvmod.hv_filter_train_step(ctx, m, t, 3e-3)
    for _ in range(150):
        last = hvmod.hv_filter_train_step(ctx, m, t, 3e-3)
    assert last < 0.5 * first, (first, last)
    P = hvmod.hv_filter_get_params(ctx)
    assert np.isfinite(P).all()
    ctx.close()
