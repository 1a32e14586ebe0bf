"""GPU ligand flattening (lg_flatten_batch, Sec. 3.1 step 1) against the FP64
oracle, checked in replay: the oracle follows every step the GPU applied and
each step that differs from the oracle's own choice must be a near-tie (sum of
distances within 1e-5 relative, or a clash distance within 1e-5 of d_clash^2);
the flattened coordinates then agree to 1e-3 A RMSD and the final sum of
distances to 1e-5 relative."""
import numpy as np
import pytest

import oracle
from paper_2110_11644_gb300 import lg, synth

from _parity import near_tie_ok

pytestmark = pytest.mark.gpu

A = 36
TOL_RMSD = 1e-3
TOL_D = 1e-5


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = lg.Context(0)
    yield c
    c.close()


def check_flatten(batch, passes, gpu, d_clash=2.0):
    dc2 = float(np.float32(d_clash)) ** 2
    rep = oracle.flatten(batch, passes, d_clash, replay=gpu["tors"], trace=True)
    assert np.array_equal(rep["status"] == 0, gpu["status"] == 0)
    n_dev = 0
    for k in range(len(gpu["tors"])):
        g, o = int(gpu["tors"][k]), int(rep["own"][k])
        if g != o:
            n_dev += 1
            s = rep["trace_D"][k * A:(k + 1) * A]
            d2 = rep["trace_d2"][k * A:(k + 1) * A]
            assert near_tie_ok(s, d2, g, o, dc2), f"decision {k}: GPU step {g} vs oracle {o}"
    worst = 0.0
    for l in range(batch.L):
        if gpu["status"][l] != 0:
            continue
        a0, a1 = int(batch.atom_off[l]), int(batch.atom_off[l + 1])
        Xg = gpu["xyz"][3 * a0:3 * a1].reshape(-1, 3).astype(np.float64)
        Xo = rep["xyz"][3 * a0:3 * a1].reshape(-1, 3)
        rmsd = float(np.sqrt(((Xg - Xo) ** 2).sum(1).mean()))
        worst = max(worst, rmsd)
        assert rmsd <= TOL_RMSD, f"ligand {l}: RMSD {rmsd}"
        assert abs(gpu["dsum"][l] - rep["D"][l]) <= TOL_D * rep["D"][l], f"ligand {l}: distance sum"
    return dict(decisions=len(gpu["tors"]), deviations=n_dev, worst_rmsd=worst)


@pytest.mark.parametrize("cfg,L,passes", [(1, 256, 2), (2, 600, 3), (3, 300, 3)])
def test_flatten_matches_oracle(ctx, cfg, L, passes):
    batch = synth.config_ligands(cfg, L)
    gpu = ctx.flatten(batch, passes)
    assert np.all(gpu["status"] == 0)
    rep = check_flatten(batch, passes, gpu)
    assert rep["deviations"] <= 0.01 * rep["decisions"] + 2, rep


def test_flatten_at_maximum_sizes(ctx):
    # 128 atoms and 32 torsional bonds, next to small ligands
    batch = synth.make_ligands(77, np.array([lg.LG_MAX_ATOMS, 12, 100]), np.array([lg.LG_MAX_ROT, 2, 20]))
    gpu = ctx.flatten(batch, 2)
    assert np.all(gpu["status"] == 0)
    rep = check_flatten(batch, 2, gpu)
    assert rep["deviations"] <= 0.01 * rep["decisions"] + 2, rep


def test_flatten_device_io_equals_host(ctx):
    batch = synth.config_ligands(2, 200)
    a = ctx.flatten(batch, 2)
    b = ctx.flatten(batch, 2, device_io=True)
    for k in ("xyz", "tors", "dsum", "status"):
        assert np.array_equal(a[k], b[k]), k


def test_flatten_edge_cases(ctx):
    batch = synth.config_ligands(1, 8)
    # empty batch
    assert len(ctx.flatten(batch.subset([]), 2)["status"]) == 0
    # zero passes and rigid ligands keep their coordinates (to FP32 rounding of the centroid frame)
    out = ctx.flatten(batch, 0)
    x0 = np.stack([batch.x, batch.y, batch.z], 1).reshape(-1)
    assert np.allclose(out["xyz"], x0, atol=1e-5, rtol=0)
    # a malformed ligand next to valid ones: only it is rejected, its coordinates pass through
    bad_parent = batch.parent.copy()
    a0 = int(batch.atom_off[1])
    bad_parent[a0 + 2] = 5  # parent after the child
    bad = synth.LigandBatch(batch.atom_off, batch.x, batch.y, batch.z, batch.q, batch.type, bad_parent,
                            batch.rot_off, batch.rot_child, batch.uid)
    out = ctx.flatten(bad, 2)
    assert out["status"][1] == lg.LG_EINVAL and np.all(out["status"][[0, 2, 3]] == 0)
    a1 = int(batch.atom_off[2])
    assert np.array_equal(out["xyz"][3 * a0:3 * a1], x0[3 * a0:3 * a1].astype(np.float32))
    assert np.isnan(out["dsum"][1])
    good = ctx.flatten(batch, 2)
    keep = [0, 2, 3]
    assert np.array_equal(out["dsum"][keep], good["dsum"][keep])


def test_flattened_ligands_dock(ctx, cfg1):
    pocket, full, params = cfg1
    batch = full.subset(range(32))
    f = ctx.flatten(batch, 2)
    X = f["xyz"].reshape(-1, 3)
    flat = synth.LigandBatch(batch.atom_off, X[:, 0].copy(), X[:, 1].copy(), X[:, 2].copy(), batch.q, batch.type,
                             batch.parent, batch.rot_off, batch.rot_child, batch.uid)
    pid = ctx.load_pocket(pocket)
    out = ctx.dock(pid, flat, params)
    assert np.all(out["status"] == 0) and np.all(np.isfinite(out["score"]))
    ctx.unload_pocket(pid)
