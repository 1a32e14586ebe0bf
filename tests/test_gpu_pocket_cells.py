"""Pocket packing on the device (lg_pocket_load): the per-node cells of
trilinear coefficients that every lookup reads (the grids stay on the GPU,
Sec. 3.2).  The device kernel and the host packing give the same bits, the
cells follow their definition, and each cell's polynomial reproduces the grid
values at its corners."""
import dataclasses

import numpy as np
import pytest

from paper_2110_11644_gb300 import lg, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = lg.Context(0)
    yield c
    c.close()


def _cells(ctx, pocket, host):
    ctx.set_option("pocket_pack_host", 1 if host else 0)
    try:
        pid = ctx.load_pocket(pocket)
    finally:
        ctx.set_option("pocket_pack_host", 0)
    try:
        return lg.lg_diag_pocket_cells(ctx.h, pid, pocket.n)
    finally:
        ctx.unload_pocket(pid)


def _definition(g):
    """Cells from their definition: corners of the cell at each node (indices
    clamped to the last layer), coefficients as FP64 differences, in FP32."""
    n = g.shape[0]
    v = g.astype(np.float64)
    nx = np.minimum(np.arange(n) + 1, n - 1)

    def c(di, dj, dk):  # v[k + dk, j + dj, i + di], arrays indexed [k, j, i]
        a = v
        if dk:
            a = a[nx, :, :]
        if dj:
            a = a[:, nx, :]
        if di:
            a = a[:, :, nx]
        return a

    v000, v100, v010, v110 = c(0, 0, 0), c(1, 0, 0), c(0, 1, 0), c(1, 1, 0)
    v001, v101, v011, v111 = c(0, 0, 1), c(1, 0, 1), c(0, 1, 1), c(1, 1, 1)
    out = np.stack([v000, v100 - v000, v010 - v000, v001 - v000,
                    v110 - v100 - v010 + v000, v101 - v100 - v001 + v000, v011 - v010 - v001 + v000,
                    v111 - v110 - v101 - v011 + v100 + v010 + v001 - v000], axis=-1)
    return out.astype(np.float32).reshape(n ** 3, 8)


def _random_pocket(n, seed):
    """A pocket of n^3 random grid values spanning many binades (and zeros)."""
    base = synth.config_pocket(1)
    rng = np.random.default_rng(seed)

    def grid():
        g = rng.standard_normal((n, n, n)) * np.exp2(rng.integers(-30, 30, (n, n, n)))
        g[rng.random((n, n, n)) < 0.05] = 0.0
        return g.astype(np.float32)

    pp = np.zeros((1, 3), np.int32)
    return dataclasses.replace(base, n=n, phi_o=grid(), phi_v=grid(), phi_e=grid(), pocket_points=pp)


@pytest.mark.parametrize("which", ["config1", "config2", "random2", "random7"])
def test_device_packing_equals_host_packing_and_the_definition(ctx, which):
    pocket = {"config1": lambda: synth.config_pocket(1), "config2": lambda: synth.config_pocket(2),
              "random2": lambda: _random_pocket(2, 1), "random7": lambda: _random_pocket(7, 2)}[which]()
    o_dev, ve_dev = _cells(ctx, pocket, host=False)
    o_host, ve_host = _cells(ctx, pocket, host=True)
    assert np.array_equal(o_dev.view(np.uint32), o_host.view(np.uint32))
    assert np.array_equal(ve_dev.view(np.uint32), ve_host.view(np.uint32))
    assert np.array_equal(o_dev, _definition(pocket.phi_o))
    assert np.array_equal(ve_dev[:, :8], _definition(pocket.phi_v))
    assert np.array_equal(ve_dev[:, 8:], _definition(pocket.phi_e))


def test_cell_polynomial_reproduces_the_corner_values(ctx):
    # the trilinear polynomial of node (i, j, k)'s cell at local corner
    # (a, b, c) in {0, 1}^3 equals the grid at (i + a, j + b, k + c), clamped
    pocket = synth.config_pocket(2)
    o, _ = _cells(ctx, pocket, host=False)
    n = pocket.n
    rng = np.random.default_rng(5)
    g = pocket.phi_o.astype(np.float64)
    for t in rng.integers(0, n ** 3, 400):
        i, j, k = t % n, (t // n) % n, t // (n * n)
        c = o[t].astype(np.float64)
        for a in (0, 1):
            for b in (0, 1):
                for cc in (0, 1):
                    p = (c[0] + a * c[1] + b * c[2] + cc * c[3] + a * b * c[4] + a * cc * c[5] + b * cc * c[6]
                         + a * b * cc * c[7])
                    want = g[min(k + cc, n - 1), min(j + b, n - 1), min(i + a, n - 1)]
                    assert abs(p - want) <= 4e-6 * max(1.0, np.abs(g).max()), (i, j, k, a, b, cc)


def test_fp32_peak_microbenchmark_is_near_the_derived_peak(ctx):
    # the FMA microbenchmark that cross-checks the roofline's derived FP32
    # peak (SMs x 128 lanes x 2 FLOP x clock) lands near it
    import torch
    t, sec = lg.lg_diag_fp32_peak(ctx.h, 3)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    derived = sms * 128 * 2 * 2.07e9 / 1e12
    assert 0.5 * derived < t < 1.05 * derived, (t, derived)
    assert sec > 0
    with pytest.raises(lg.LgError):
        lg.lg_diag_fp32_peak(ctx.h, 0)
