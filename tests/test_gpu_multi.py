"""Several pockets in one launch (lg_dock_multi): bit-identical to one
lg_dock_batch call per pocket in both visiting orders, parity with the FP64
oracle on a pocket of the 15-pocket set, per-ligand status on every pocket,
pose ranking, and argument errors."""
import dataclasses

import numpy as np
import pytest

from paper_2110_11644_gb300 import lg, synth

from _parity import check

pytestmark = pytest.mark.gpu

KEYS = ("score", "best_restart", "status", "tors_idx", "pose", "restart_score", "restart_tors")


@pytest.fixture(scope="module")
def multi():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = lg.Context(0)
    pockets = [synth.config_pocket(1), synth.config_pocket(4, 0), synth.config_pocket(4, 3)]
    pids = [ctx.load_pocket(p) for p in pockets]
    yield ctx, pockets, pids
    ctx.close()


def _params():
    return synth.DockParams(restarts=16, passes=2)


def _one_bad(uid):
    # atom 3 hangs under atom 1 after atom 2: subtrees are not contiguous
    rng = np.random.default_rng(uid)
    parent = [-1, 0, 0, 1]
    pos = np.zeros((4, 3))
    for i in range(1, 4):
        d = rng.normal(size=3)
        pos[i] = pos[parent[i]] + 1.5 * d / np.linalg.norm(d)
    return synth.LigandBatch(np.array([0, 4], np.int32), pos[:, 0].astype(np.float32), pos[:, 1].astype(np.float32),
                             pos[:, 2].astype(np.float32), np.zeros(4, np.float32), np.zeros(4, np.uint8),
                             np.array(parent, np.int16), np.array([0, 0], np.int32), np.zeros(0, np.int16),
                             np.array([uid], np.uint64))


@pytest.mark.parametrize("order", [0, 1])
def test_multi_equals_one_call_per_pocket(multi, order):
    ctx, _, pids = multi
    batch = synth.config_ligands(2, 96)
    params = _params()
    ctx.set_option("multi_order", order)
    try:
        got = ctx.dock_multi(pids, batch, params, restart_score=True, restart_tors=True)
    finally:
        ctx.set_option("multi_order", 0)
    for pid, g in zip(pids, got):
        want = ctx.dock(pid, batch, params, restart_score=True, restart_tors=True)
        for k in KEYS:
            assert np.array_equal(g[k], want[k]), (pid, k)


def test_multi_device_io_equals_host(multi):
    ctx, _, pids = multi
    batch = synth.config_ligands(2, 40)
    params = _params()
    a = ctx.dock_multi(pids, batch, params)
    b = ctx.dock_multi(pids, batch, params, device_io=True)
    for x, y in zip(a, b):
        for k in ("score", "best_restart", "status", "tors_idx", "pose"):
            assert np.array_equal(x[k], y[k]), k


def test_multi_matches_oracle(multi):
    ctx, pockets, pids = multi
    batch = synth.config_ligands(2, 48)
    params = _params()
    got = ctx.dock_multi(pids, batch, params, restart_score=True, restart_tors=True)
    for pocket, g in zip(pockets[1:], got[1:]):  # the 40^3 and 64^3 pockets of the 15-pocket set
        rep = check(pocket, batch, params, g)
        assert rep["worst_rmsd"] <= 1e-3


def test_multi_status_on_every_pocket(multi):
    ctx, _, pids = multi
    good = synth.config_ligands(2, 3)
    mix = synth.LigandBatch.concat([good.subset([0]), _one_bad(77), good.subset([1, 2])])
    got = ctx.dock_multi(pids, mix, _params())
    for g in got:
        assert list(g["status"]) == [0, lg.LG_EINVAL, 0, 0]
        assert np.isnan(g["score"][1]) and g["best_restart"][1] == -1
        assert np.all(np.isfinite(g["score"][[0, 2, 3]]))


def test_multi_with_ranking(multi):
    ctx, _, pids = multi
    batch = synth.config_ligands(2, 32)
    params = dataclasses.replace(_params(), cluster_rmsd=3.0, rescore_top=5)
    got = ctx.dock_multi(pids, batch, params)
    for pid, g in zip(pids, got):
        want = ctx.dock(pid, batch, params)
        for k in ("score", "best_restart", "rank", "leader", "restart_geo", "pose"):
            assert np.array_equal(g[k], want[k]), (pid, k)


def test_multi_heavy_tailed_with_ranking_both_orders(multi):
    # ligands up to 100 atoms (no size classes across pockets) with pose
    # ranking, in both visiting orders: each pocket's results equal its own call
    import dataclasses
    ctx, _, pids = multi
    batch = synth.config_ligands(3, 300)
    assert batch.n_atoms().max() > 64
    params = dataclasses.replace(synth.config_params(3), restarts=12, passes=2, cluster_rmsd=3.0, rescore_top=4)
    want = [ctx.dock(pid, batch, params) for pid in pids]
    try:
        for order in (0, 1):
            ctx.set_option("multi_order", order)
            got = ctx.dock_multi(pids, batch, params)
            for w, g in zip(want, got):
                for k in ("score", "best_restart", "status", "rank", "leader", "restart_geo", "pose"):
                    assert np.array_equal(g[k], w[k]), (order, k)
    finally:
        ctx.set_option("multi_order", 0)


def test_multi_bad_arguments(multi):
    ctx, _, pids = multi
    batch = synth.config_ligands(2, 4)
    with pytest.raises(lg.LgError):
        ctx.dock_multi([pids[0], 999], batch, _params())
    arrs = lg.host_batch_arrays(batch)
    b = lg.make_batch_struct(arrs, batch.L)
    p = lg.make_params(16, 2, 1, mode=lg.LG_MODE_PLAIN)
    r, _ = lg.alloc_result(batch.L, int(batch.atom_off[-1]), int(batch.rot_off[-1]), 16, 2)
    with pytest.raises(lg.LgError):
        lg.lg_dock_multi(ctx.h, pids, b, p, [r] * len(pids))
    with pytest.raises(lg.LgError):
        lg.lg_dock_multi(ctx.h, [], b, lg.make_params(16, 2, 1), [])
    # decision ranks: per-pocket launches only (pocket-major); ligand-major refuses
    pm = ctx.dock_multi(pids, batch, _params(), restart_tors=True, decision_rank=True)
    for pid, g in zip(pids, pm):
        want = ctx.dock(pid, batch, _params(), restart_tors=True, decision_rank=True)
        assert np.array_equal(g["decision_rank"], want["decision_rank"])
    ctx.set_option("multi_order", 1)
    try:
        with pytest.raises(lg.LgError):
            ctx.dock_multi(pids, batch, _params(), decision_rank=True)
    finally:
        ctx.set_option("multi_order", 0)
    # the context stays usable
    assert all(np.all(g["status"] == 0) for g in ctx.dock_multi(pids, batch, _params()))
