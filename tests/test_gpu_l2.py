"""L2 residency of the pockets (the paper keeps the binding site resident in
the GPU's texture memory, Sec. 3.2): lg_pocket_load reserves a persisting L2
set-aside sized for the largest loaded pocket's overlap cells, and every
docking launch against one pocket marks that pocket's cells persisting with an
access-policy window.  The window changes where lines live in L2, never a
result: docking with and without it is bit-identical, for one pocket and for
several pockets in both visiting orders."""
import numpy as np
import pytest

from paper_2110_11644_gb300 import lg, synth

pytestmark = pytest.mark.gpu

KEYS = ("score", "best_restart", "status", "tors_idx", "pose", "restart_score", "restart_tors")


@pytest.fixture(scope="module")
def ctx_pockets():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = lg.Context(0)
    pockets = [synth.config_pocket(4, 0), synth.config_pocket(4, 14), synth.config_pocket(2)]
    pids = [ctx.load_pocket(p) for p in pockets]
    yield ctx, pockets, pids
    ctx.close()


def test_pocket_load_sets_the_window(ctx_pockets):
    import torch
    ctx, pockets, pids = ctx_pockets
    prop = torch.cuda.get_device_properties(0)
    batch = synth.config_ligands(2, 64)
    params = synth.DockParams(restarts=8, passes=2)
    ctx.dock(pids[2], batch, params)
    st = ctx.stats()
    largest = max(p.n ** 3 * 32 for p in pockets)
    persist_max = getattr(prop, "persisting_l2_cache_max_size", None)
    if persist_max is not None:
        assert st.l2_persist_bytes == min(largest, persist_max)
    assert st.l2_persist_bytes > 0
    assert 0 < st.l2_window_bytes <= pockets[2].n ** 3 * 32
    ctx.set_option("l2_window", 0)
    try:
        ctx.dock(pids[2], batch, params)
        assert ctx.stats().l2_window_bytes == 0
    finally:
        ctx.set_option("l2_window", 1)


def test_window_never_changes_a_result(ctx_pockets):
    ctx, _, pids = ctx_pockets
    batch = synth.config_ligands(2, 300)
    params = synth.DockParams(restarts=16, passes=2)
    on = [ctx.dock(pid, batch, params, restart_score=True, restart_tors=True) for pid in pids]
    multi_on = {o: None for o in (0, 1)}
    for order in (0, 1):
        ctx.set_option("multi_order", order)
        multi_on[order] = ctx.dock_multi(pids, batch, params, restart_score=True, restart_tors=True)
    ctx.set_option("multi_order", 0)
    ctx.set_option("l2_window", 0)
    try:
        off = [ctx.dock(pid, batch, params, restart_score=True, restart_tors=True) for pid in pids]
        multi_off = ctx.dock_multi(pids, batch, params, restart_score=True, restart_tors=True)
    finally:
        ctx.set_option("l2_window", 1)
    for a, b in zip(on, off):
        for k in KEYS:
            assert np.array_equal(a[k], b[k], equal_nan=True), k
    for order in (0, 1):
        for a, b in zip(multi_on[order], multi_off):
            for k in KEYS:
                assert np.array_equal(a[k], b[k], equal_nan=True), (order, k)


def test_unload_shrinks_the_set_aside():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = lg.Context(0)
    try:
        small, big = synth.config_pocket(4, 0), synth.config_pocket(4, 14)
        p_small = ctx.load_pocket(small)
        batch = synth.config_ligands(2, 16)
        params = synth.DockParams(restarts=8, passes=1)
        ctx.dock(p_small, batch, params)
        s1 = ctx.stats().l2_persist_bytes
        p_big = ctx.load_pocket(big)
        ctx.dock(p_small, batch, params)
        s2 = ctx.stats().l2_persist_bytes
        ctx.unload_pocket(p_big)
        ctx.dock(p_small, batch, params)
        s3 = ctx.stats().l2_persist_bytes
        assert 0 < s1 <= small.n ** 3 * 32
        assert s2 >= s1 and s3 == s1
    finally:
        ctx.close()
