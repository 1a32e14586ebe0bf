"""Size classes, restart tiles and the autotuner of the batched kernels: a
batch whose atom maximum exceeds 64 is docked by one persistent launch per
size class, each with shared memory for its own maximum; the restart tile
(lanes per restart) and warps per CTA of each class are chosen by timing on
the first call.  Results never depend on any of them."""
import dataclasses

import numpy as np
import pytest

from paper_2110_11644_gb300 import lg, synth

from _parity import check

pytestmark = pytest.mark.gpu

KEYS = ("score", "best_restart", "status", "tors_idx", "pose", "restart_score", "restart_tors")


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = lg.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def heavy():
    """Heavy-tailed ligands spanning all three size classes."""
    b = synth.config_ligands(3, 3000)
    n = b.n_atoms()
    assert n.max() > 64 and n.min() <= 32
    return b


def _dock(ctx, pid, batch, params, **kw):
    return ctx.dock(pid, batch, params, restart_score=True, restart_tors=True, **kw)


def test_results_do_not_depend_on_warps_or_tuning(ctx, cfg2_pocket, heavy):
    pid = ctx.load_pocket(cfg2_pocket)
    params = synth.config_params(3)
    sub = heavy.subset(range(1200))
    ref = None
    try:
        for opt in (0, 1, 2, 4):
            ctx.set_option("warps_per_cta", opt)
            for tune in (1, 0):
                ctx.set_option("autotune", tune)
                out = _dock(ctx, pid, sub, params)
                if ref is None:
                    ref = out
                for k in KEYS:
                    assert np.array_equal(out[k], ref[k]), (opt, tune, k)
        # device batch with no declared maxima: all three classes launched
        out = _dock(ctx, pid, sub, params, device_io=True)
        for k in KEYS:
            assert np.array_equal(out[k], ref[k]), k
    finally:
        ctx.set_option("warps_per_cta", 0)
        ctx.set_option("autotune", 1)
        ctx.unload_pocket(pid)


# every (lanes per restart, warps per CTA) the batched kernel comes with
TILES = ((4, 1), (4, 2), (4, 4), (2, 1), (2, 2), (2, 4), (8, 1), (8, 2), (8, 4), (8, 8),
         (16, 1), (16, 2), (16, 4), (16, 8), (16, 16))


@pytest.mark.parametrize("rigid", [0, 2])
def test_every_restart_tile_gives_the_same_bits(ctx, cfg2_pocket, heavy, rigid):
    """2, 4, 8 and 16 lanes per restart (16, 8, 4 and 2 restart slots per warp;
    ragged step rounds at 8 and 16) at every warp count their launch bounds
    allow, with and without rigid moves, on ligands of all three size
    classes: every output equals the 4-lane tile's, bit for bit."""
    pid = ctx.load_pocket(cfg2_pocket)
    n = heavy.n_atoms()
    idx = np.concatenate([np.nonzero(n > 64)[0][:60], np.nonzero(n <= 32)[0][:60], np.nonzero((n > 32) & (n <= 64))[0][:60]])
    sub = heavy.subset(np.sort(idx))
    params = dataclasses.replace(synth.config_params(3), rigid_steps=rigid, restarts=30 if rigid == 0 else 20)
    ref = None
    try:
        ctx.set_option("autotune", 0)
        for lanes, warps in TILES:
            ctx.set_option("restart_lanes", lanes)
            ctx.set_option("warps_per_cta", warps)
            out = _dock(ctx, pid, sub, params, restart_rigid=rigid > 0, decision_rank=False)
            st = ctx.stats()
            assert (st.restart_lanes, st.warps_per_cta) == (lanes, warps)
            if ref is None:
                ref = out
                # at 4 lanes the outputs match the oracle within the near-tie rule
                rep = check(cfg2_pocket, sub, params, out)
                assert rep["deviations"] <= 0.002 * rep["decisions"] + 2, rep
            for k in KEYS + (("restart_rigid",) if rigid else ()):
                assert np.array_equal(out[k], ref[k]), (lanes, warps, k)
    finally:
        ctx.set_option("restart_lanes", 0)
        ctx.set_option("warps_per_cta", 0)
        ctx.set_option("autotune", 1)
        ctx.unload_pocket(pid)


def test_tiles_the_ranking_and_trace_forms_lack_fall_back_to_four_lanes(ctx, cfg1):
    pocket, full, params = cfg1
    pid = ctx.load_pocket(pocket)
    sub = full.subset(range(200))
    ranked = dataclasses.replace(params, cluster_rmsd=2.0, rescore_top=4)
    try:
        ctx.set_option("restart_lanes", 0)
        ref_r = _dock(ctx, pid, sub, ranked)
        ref_t = _dock(ctx, pid, sub, params, decision_rank=True)
        ctx.set_option("restart_lanes", 16)
        got_r = _dock(ctx, pid, sub, ranked)
        assert ctx.stats().restart_lanes == 4
        got_t = _dock(ctx, pid, sub, params, decision_rank=True)
        assert ctx.stats().restart_lanes == 4
        _dock(ctx, pid, sub, params)
        assert ctx.stats().restart_lanes == 16
        for k in ref_r:
            if ref_r[k] is not None:
                assert np.array_equal(got_r[k], ref_r[k]), k
        assert np.array_equal(got_t["decision_rank"], ref_t["decision_rank"])
        with pytest.raises(lg.LgError):
            ctx.set_option("restart_lanes", 3)
    finally:
        ctx.set_option("restart_lanes", 0)
        ctx.unload_pocket(pid)


def test_autotuner_caches_its_choice(ctx, cfg2_pocket, heavy):
    pid = ctx.load_pocket(cfg2_pocket)
    params = synth.config_params(3)
    ctx.set_option("autotune", 1)  # clears the cache
    _dock(ctx, pid, heavy, params)   # 3,000 ligands: more than one wave of 2-warp CTAs
    first = ctx.stats().launches
    _dock(ctx, pid, heavy, params)
    second = ctx.stats().launches
    ctx.unload_pocket(pid)
    # prep + sort (3) + one launch per class (3); the first call adds the timing trials
    assert second == 6
    assert first > second


def test_tuning_carries_to_another_context(ctx, cfg2_pocket, heavy):
    # the tuned choices exported as JSON and imported by a fresh context: its
    # first call runs no timing trials and docks identically
    import json
    pid = ctx.load_pocket(cfg2_pocket)
    params = synth.config_params(3)
    ctx.set_option("autotune", 1)  # clears the cache
    assert json.loads(ctx.tune_export())["entries"] == []
    ref = _dock(ctx, pid, heavy, params)
    text = ctx.tune_export()
    doc = json.loads(text)
    assert doc["sms"] > 0 and len(doc["entries"]) == 3
    assert all(len(e) == 10 and (e[8], e[9]) in TILES for e in doc["entries"]), doc["entries"]
    ctx.unload_pocket(pid)
    c2 = lg.Context(0)
    try:
        p2 = c2.load_pocket(cfg2_pocket)
        c2.tune_import(text)
        got = _dock(c2, p2, heavy, params)
        assert c2.stats().launches == 6  # prep + sort (3) + one launch per class (3): no trials
        for k in KEYS:
            assert np.array_equal(got[k], ref[k]), k
        assert json.loads(c2.tune_export())["entries"] == doc["entries"]
        # another device, or text that does not parse: refused, cache unchanged
        other = dict(doc, device=doc["device"] + " X")
        for bad in (json.dumps(other), json.dumps(dict(doc, sms=doc["sms"] + 1)), text.replace("]]", "]"),
                    text.replace("[[", "[[99, ") if doc["entries"] else text + "x", "not json"):
            with pytest.raises(lg.LgError):
                c2.tune_import(bad)
        assert json.loads(c2.tune_export())["entries"] == doc["entries"]
    finally:
        c2.close()


def test_small_batches_take_a_latency_tile_untuned(ctx, cfg1, cfg2_pocket):
    # a batch that fits in one wave runs at one CTA per ligand with all its
    # restarts in flight over 16 lanes each, without tuning; results as at
    # any tile and width
    pocket, full, params = cfg1
    pid = ctx.load_pocket(pocket)
    ctx.set_option("autotune", 1)
    small = full.subset(range(64))
    out = _dock(ctx, pid, small, params)
    st = ctx.stats()
    # 16 restarts at 2 per warp: 8 warps; prep + sort (2) + one launch
    assert (st.restart_lanes, st.warps_per_cta, st.launches) == (16, 8, 4)
    ctx.set_option("warps_per_cta", 1)
    try:
        ref = _dock(ctx, pid, small, params)
    finally:
        ctx.set_option("warps_per_cta", 0)
    for k in KEYS:
        assert np.array_equal(out[k], ref[k]), k
    ctx.unload_pocket(pid)
    pid = ctx.load_pocket(cfg2_pocket)
    _dock(ctx, pid, synth.config_ligands(2, 64), synth.config_params(2))
    st = ctx.stats()
    assert (st.restart_lanes, st.warps_per_cta) == (16, 15)  # 30 restarts at 2 per warp
    ctx.unload_pocket(pid)


def test_heavy_tailed_split_matches_oracle(ctx, cfg2_pocket, heavy):
    pid = ctx.load_pocket(cfg2_pocket)
    params = synth.config_params(3)
    idx = np.concatenate([np.nonzero(heavy.n_atoms() > 64)[0][:40], np.nonzero(heavy.n_atoms() <= 32)[0][:40],
                          np.nonzero((heavy.n_atoms() > 32) & (heavy.n_atoms() <= 64))[0][:40]])
    sub = heavy.subset(np.sort(idx))
    out = _dock(ctx, pid, sub, params)
    ctx.unload_pocket(pid)
    rep = check(cfg2_pocket, sub, params, out)
    assert rep["deviations"] <= 0.002 * rep["decisions"] + 2, rep


def test_graph_capture_and_replay(ctx, cfg1):
    import torch
    pocket, full, params = cfg1
    pid = ctx.load_pocket(pocket)
    batch = full.subset(range(64))
    L, A, R = batch.L, int(batch.atom_off[-1]), int(batch.rot_off[-1])
    darr = lg.device_batch_arrays(batch)
    b = lg.make_batch_struct(darr, L)
    p = lg.make_params(params.restarts, params.passes, params.seed, params.d_clash)
    side = torch.cuda.Stream()

    def run(r):
        lg.lg_dock_batch(ctx.h, pid, b, p, r, side.cuda_stream)
        side.synchronize()
        return ctx.stats().graph

    r0, o0 = lg.alloc_result(L, A, R, params.restarts, params.passes, device=True)
    run(r0)  # eager reference (graphs off)
    ref = {k: v.cpu().numpy() for k, v in o0.items() if v is not None}
    ctx.set_option("graphs", 1)
    try:
        r1, o1 = lg.alloc_result(L, A, R, params.restarts, params.passes, device=True)
        modes = [run(r1) for _ in range(3)]
        assert modes[-2:] == [2, 1] or modes == [2, 1, 1], modes   # captured once, then replayed
        for k, v in o1.items():
            if v is not None:
                assert np.array_equal(v.cpu().numpy(), ref[k]), k
        # other output buffers: a new graph; the default stream: no graph
        r2, o2 = lg.alloc_result(L, A, R, params.restarts, params.passes, device=True)
        assert run(r2) == 2 and np.array_equal(o2["score"].cpu().numpy(), ref["score"])
        lg.lg_dock_batch(ctx.h, pid, b, p, r2, None)
        torch.cuda.synchronize()
        assert ctx.stats().graph == 0
    finally:
        ctx.set_option("graphs", 2)
        ctx.unload_pocket(pid)


def test_graphs_by_default_when_arguments_recur(ctx, cfg1):
    # the default (graphs = 2): a call whose arguments were not seen before
    # runs directly, the second call with the same arguments is captured,
    # later ones replay; new arguments start over; results never change
    import torch
    pocket, full, params = cfg1
    pid = ctx.load_pocket(pocket)
    batch = full.subset(range(96))
    L, A, R = batch.L, int(batch.atom_off[-1]), int(batch.rot_off[-1])
    darr = lg.device_batch_arrays(batch)
    b = lg.make_batch_struct(darr, L)
    p = lg.make_params(params.restarts, params.passes, params.seed, params.d_clash)
    side = torch.cuda.Stream()
    try:
        ctx.set_option("graphs", 2)

        def run(r):
            lg.lg_dock_batch(ctx.h, pid, b, p, r, side.cuda_stream)
            side.synchronize()
            return ctx.stats().graph

        r1, o1 = lg.alloc_result(L, A, R, params.restarts, params.passes, device=True)
        modes = [run(r1)]
        ref = {k: v.cpu().numpy() for k, v in o1.items() if v is not None}
        for _ in range(3):
            modes.append(run(r1))
            for k, v in o1.items():
                if v is not None:
                    assert np.array_equal(v.cpu().numpy(), ref[k]), k
        assert modes == [0, 2, 1, 1], modes
        r2, o2 = lg.alloc_result(L, A, R, params.restarts, params.passes, device=True)
        assert [run(r2), run(r2)] == [0, 2]
        assert np.array_equal(o2["score"].cpu().numpy(), ref["score"])
    finally:
        ctx.set_option("graphs", 2)
        ctx.unload_pocket(pid)


def test_graph_replay_with_ranking_over_size_classes(ctx, cfg2_pocket, heavy):
    # a captured call that launches one kernel per size class with pose
    # ranking replays to the eager call's results
    import dataclasses
    import torch
    pid = ctx.load_pocket(cfg2_pocket)
    sub = heavy.subset(range(700))
    prm = dataclasses.replace(synth.config_params(3), restarts=12, passes=2, cluster_rmsd=3.0, rescore_top=4)
    L, A, R = sub.L, int(sub.atom_off[-1]), int(sub.rot_off[-1])
    darr = lg.device_batch_arrays(sub)
    b = lg.make_batch_struct(darr, L)
    p = lg.make_params(prm.restarts, prm.passes, prm.seed, prm.d_clash, cluster_rmsd=prm.cluster_rmsd,
                       rescore_top=prm.rescore_top)
    side = torch.cuda.Stream()
    r0, o0 = lg.alloc_result(L, A, R, prm.restarts, prm.passes, device=True, ranking=True)
    lg.lg_dock_batch(ctx.h, pid, b, p, r0, side.cuda_stream)  # eager (tunes)
    side.synchronize()
    ref = {k: v.cpu().numpy() for k, v in o0.items() if v is not None}
    ctx.set_option("graphs", 1)
    try:
        r1, o1 = lg.alloc_result(L, A, R, prm.restarts, prm.passes, device=True, ranking=True)
        modes = []
        for _ in range(3):
            lg.lg_dock_batch(ctx.h, pid, b, p, r1, side.cuda_stream)
            side.synchronize()
            modes.append(ctx.stats().graph)
            for k, v in o1.items():
                if v is not None:
                    assert np.array_equal(v.cpu().numpy(), ref[k]), k
        assert modes[-1] == 1, modes
    finally:
        ctx.set_option("graphs", 2)
        ctx.unload_pocket(pid)


def test_async_calls_on_two_streams_share_scratch_safely(ctx, cfg1):
    # two device-memory calls issued back to back on different streams use the
    # same context scratch; the library orders them on the device
    import torch
    pocket, full, params = cfg1
    pid = ctx.load_pocket(pocket)
    a_b, b_b = full.subset(range(0, 128)), full.subset(range(128, 256))
    res = []
    for batch in (a_b, b_b):
        L, A, R = batch.L, int(batch.atom_off[-1]), int(batch.rot_off[-1])
        darr = lg.device_batch_arrays(batch)
        res.append((batch, darr, lg.make_batch_struct(darr, L),
                    lg.alloc_result(L, A, R, params.restarts, params.passes, device=True)))
    p = lg.make_params(params.restarts, params.passes, params.seed, params.d_clash)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    for (batch, _, b, (r, _)), s in zip(res, (s1, s2)):
        lg.lg_dock_batch(ctx.h, pid, b, p, r, s.cuda_stream)
    torch.cuda.synchronize()
    for batch, _, _, (_, outs) in res:
        ref = ctx.dock(pid, batch, params)
        assert np.array_equal(outs["score"][:batch.L].cpu().numpy(), ref["score"])
        assert np.array_equal(outs["best_restart"][:batch.L].cpu().numpy(), ref["best_restart"])
    ctx.unload_pocket(pid)
