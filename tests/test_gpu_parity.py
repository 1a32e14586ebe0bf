"""GPU parity: the CUDA path through the C-ABI against the FP64 oracle."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2110_11644_gb300 import lg, synth

from _parity import check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = lg.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def pocket1(ctx, cfg1):
    return ctx.load_pocket(cfg1[0])


def _dock(ctx, pid, batch, params, **kw):
    return ctx.dock(pid, batch, params, restart_score=True, restart_tors=True, **kw)


# ----------------------------------------------------------------------------- primitives
def test_philox_matches_oracle_and_curand(ctx):
    import torch
    n = 1 << 20
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    dc = torch.from_numpy(ctr.view(np.int32)).cuda()
    dk = torch.from_numpy(key.view(np.int32)).cuda()
    out_own = torch.zeros(n * 4, dtype=torch.int32, device="cuda")
    out_cur = torch.zeros(n * 4, dtype=torch.int32, device="cuda")
    lg.lg_diag_philox(ctx.h, n, dc.data_ptr(), dk.data_ptr(), out_own.data_ptr(), 0)
    lg.lg_diag_philox(ctx.h, n, dc.data_ptr(), dk.data_ptr(), out_cur.data_ptr(), 1)
    a = out_own.cpu().numpy().view(np.uint32).reshape(n, 4)
    b = out_cur.cpu().numpy().view(np.uint32).reshape(n, 4)
    assert np.array_equal(a, b)
    for i in rng.integers(0, n, size=2000):
        assert np.array_equal(a[i], oracle.philox4x32_10(ctr[i], key[i]))


def test_score_poses_matches_oracle(ctx, cfg1, pocket1):
    pocket, batch, _ = cfg1
    rng = np.random.default_rng(1)
    lo, hi = pocket.origin - 3.0, pocket.origin + pocket.h * (pocket.n - 1) + 3.0
    xyz = rng.uniform(lo, hi, size=(len(batch.x), 3)).astype(np.float32)
    E_g = ctx.score_poses(pocket1, batch.atom_off, xyz, batch.q, batch.type)
    E_o, Eabs = oracle.score_poses(pocket, batch.atom_off, xyz.astype(np.float64), batch.q, batch.type)
    err = np.abs(E_g - E_o) / np.maximum(np.abs(E_o), Eabs)
    assert err.max() <= 1e-5, err.max()


def test_score_poses_at_nodes_equals_direct_sum(ctx, cfg1, pocket1):
    pocket = cfg1[0]
    rng = np.random.default_rng(2)
    ijk = rng.integers(0, pocket.n, size=(500, 3))
    xyz = pocket.node_xyz(ijk)
    v, e = synth.direct_potentials(pocket, xyz)
    q = rng.normal(0, 0.3, size=500).astype(np.float32)
    t = rng.integers(0, 5, size=500).astype(np.uint8)
    E_g = ctx.score_poses(pocket1, np.arange(501, dtype=np.int32), xyz.astype(np.float32), q, t)
    want = pocket.type_w[t].astype(np.float64) * v + q * e
    assert np.all(np.abs(E_g - want) <= 1e-5 * (np.abs(pocket.type_w[t] * v) + np.abs(q * e) + 1e-3))


# ----------------------------------------------------------------------------- docking parity
def test_dock_config1_matches_oracle(ctx, cfg1, pocket1):
    pocket, batch, params = cfg1
    gpu = _dock(ctx, pocket1, batch, params)
    rep = {}
    check(pocket, batch, params, gpu, rep)
    print("config-1 parity:", rep)
    assert rep["decisions"] > 1000
    assert rep["deviations"] <= 0.01 * rep["decisions"]


def test_plain_and_batched_forms_agree_bitwise(ctx, cfg1, pocket1):
    _, batch, params = cfg1
    sub = batch.subset(range(64))
    a = _dock(ctx, pocket1, sub, params, mode=lg.LG_MODE_BATCHED)
    b = _dock(ctx, pocket1, sub, params, mode=lg.LG_MODE_PLAIN, plain_streams=4)
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def _oracle_rank_bounds(trace_s, choice):
    """Per decision, the least and largest 1 + (steps ranked before the
    chosen one by overlap score, ties to the lower step) over orderings that
    may swap scores within the 1e-5 near-tie tolerance."""
    s = trace_s.reshape(-1, 36)
    c = choice.astype(int)
    sc = s[np.arange(len(c)), c]
    tol = 1e-5 * np.maximum(np.abs(s).max(1), 1e-30)
    other = np.arange(36)[None, :] != c[:, None]
    exact = 1 + ((s > sc[:, None]) | ((s == sc[:, None]) & (np.arange(36)[None, :] < c[:, None]))).sum(1)
    lo = 1 + ((s > (sc + tol)[:, None]) & other).sum(1)
    hi = 1 + ((s >= (sc - tol)[:, None]) & other).sum(1)
    return exact, lo, hi


def test_decision_ranks_match_oracle_and_both_forms(ctx, cfg1, pocket1, cfg2_pocket):
    # decision_rank: 1 + the steps ranked before the chosen one; the oracle
    # replays the GPU's choices and ranks the same steps in FP64
    pocket, batch, params = cfg1
    sub = batch.subset(range(96))
    a = _dock(ctx, pocket1, sub, params, decision_rank=True)
    b = _dock(ctx, pocket1, sub, params, decision_rank=True, mode=lg.LG_MODE_PLAIN, plain_streams=4)
    c = _dock(ctx, pocket1, sub, params, decision_rank=True, device_io=True)
    assert np.array_equal(a["decision_rank"], b["decision_rank"])
    assert np.array_equal(a["decision_rank"], c["decision_rank"])
    plain = _dock(ctx, pocket1, sub, params)
    for k in plain:  # asking for the ranks changes nothing else
        if plain[k] is not None:
            assert np.array_equal(plain[k], a[k]), k
    rep = oracle.dock(pocket, sub, params, replay=a["restart_tors"], trace=True)
    exact, lo, hi = _oracle_rank_bounds(rep["trace_s"], a["restart_tors"])
    g = a["decision_rank"].astype(int) & 0x7F  # bit 7 marks a skipped decision
    assert np.all((g >= lo) & (g <= hi))
    assert np.mean(g == exact) > 0.99
    assert g.min() >= 1 and g.max() <= 36 and g.mean() > 1.0
    _check_skip_marks(sub, params, a)
    # throughput ligands, whose convergence stops skip decisions: the skipped
    # ones repeat the bond's previous rank, as the oracle's full sweep finds
    pid = ctx.load_pocket(cfg2_pocket)
    prm2 = synth.config_params(2)
    lig2 = synth.config_ligands(2, 48)
    d = _dock(ctx, pid, lig2, prm2, decision_rank=True)
    ctx.unload_pocket(pid)
    rep = oracle.dock(cfg2_pocket, lig2, prm2, replay=d["restart_tors"], trace=True)
    exact, lo, hi = _oracle_rank_bounds(rep["trace_s"], d["restart_tors"])
    g = d["decision_rank"].astype(int) & 0x7F
    assert np.all((g >= lo) & (g <= hi))
    assert np.mean(g == exact) > 0.99
    assert _check_skip_marks(lig2, prm2, d) > 0


def _check_skip_marks(batch, params, res):
    """Bit 7 of decision_rank marks exactly the decisions after a restart's
    exact stop: R decisions in a row without a move, every later decision
    repeating one of them.  Returns how many are marked."""
    S, P = params.restarts, params.passes
    dr = res["decision_rank"].astype(int)
    tors = res["restart_tors"].astype(int)
    marked = 0
    for l in range(batch.L):
        r0, R = int(batch.rot_off[l]), int(batch.rot_off[l + 1] - batch.rot_off[l])
        for r in range(S):
            d0 = S * P * r0 + r * P * R
            zrun, stopped = 0, False
            for q in range(P * R):
                want = stopped
                assert bool(dr[d0 + q] & 0x80) == want, (l, r, q)
                marked += want
                if not stopped:
                    zrun = 0 if tors[d0 + q] else zrun + 1
                    stopped = zrun >= R
                else:
                    assert tors[d0 + q] == 0
    return marked


def test_host_and_device_io_agree_and_runs_repeat(ctx, cfg1, pocket1):
    _, batch, params = cfg1
    a = _dock(ctx, pocket1, batch, params)
    b = _dock(ctx, pocket1, batch, params, device_io=True)
    c = _dock(ctx, pocket1, batch, params)
    for k in a:
        assert np.array_equal(a[k], b[k]), k
        assert np.array_equal(a[k], c[k]), k


def test_result_independent_of_batch_mix(ctx, cfg1, pocket1):
    _, batch, params = cfg1
    full = _dock(ctx, pocket1, batch, params)
    perm = np.random.default_rng(3).permutation(batch.L)[:77]
    mixed = _dock(ctx, pocket1, batch.subset(perm), params)
    assert np.array_equal(full["score"][perm], mixed["score"])
    assert np.array_equal(full["best_restart"][perm], mixed["best_restart"])
    alone = _dock(ctx, pocket1, batch.subset([int(perm[5])]), params)
    assert alone["score"][0] == full["score"][perm[5]]


def test_dock_config2_sample_matches_oracle(ctx, cfg2_pocket):
    pid = ctx.load_pocket(cfg2_pocket)
    params = synth.config_params(2)
    batch = synth.config_ligands(2, 96)
    gpu = _dock(ctx, pid, batch, params)
    rep = {}
    check(cfg2_pocket, batch, params, gpu, rep)
    print("config-2 sample parity:", rep)
    assert rep["deviations"] <= 0.01 * rep["decisions"]
    ctx.unload_pocket(pid)


def test_dock_heavy_tailed_sample_matches_oracle(ctx, cfg2_pocket):
    pid = ctx.load_pocket(cfg2_pocket)
    params = synth.config_params(3)
    full = synth.config_ligands(3, 4000)
    order = np.argsort(-full.n_atoms(), kind="stable")
    idx = np.concatenate([order[:24], order[-24:], order[1000:1024]])   # largest, smallest, middle
    batch = full.subset(idx)
    gpu = _dock(ctx, pid, batch, params)
    rep = {}
    check(cfg2_pocket, batch, params, gpu, rep)
    print("heavy-tailed sample parity:", rep)
    ctx.unload_pocket(pid)


# ----------------------------------------------------------------------------- edge cases
def _one(N, parent, rot, uid=5, seed=11):
    rng = np.random.default_rng(seed)
    # a chain-like layout with ~1.5 A bonds so distances are realistic
    pos = np.zeros((N, 3))
    for i in range(1, N):
        d = rng.normal(size=3); d /= np.linalg.norm(d)
        pos[i] = pos[parent[i]] + 1.5 * d
    return synth.LigandBatch(np.array([0, N], np.int32), pos[:, 0].astype(np.float32), pos[:, 1].astype(np.float32),
                             pos[:, 2].astype(np.float32), rng.normal(0, 0.2, N).astype(np.float32),
                             rng.integers(0, 5, N).astype(np.uint8), np.array(parent, np.int16),
                             np.array([0, len(rot)], np.int32), np.array(rot, np.int16), np.array([uid], np.uint64))


def test_edge_cases(ctx, cfg1, pocket1):
    pocket, batch, params = cfg1
    # empty batch
    empty = batch.subset([])
    out = ctx.dock(pocket1, empty, params)
    assert len(out["score"]) == 0
    # single atom, rigid ligand, S = 1, P = 0
    single = _one(1, [-1], [])
    p1 = synth.DockParams(restarts=1, passes=0, seed=params.seed)
    g = _dock(ctx, pocket1, single, p1)
    check(pocket, single, p1, g)
    # invalid topology next to valid ligands: only it fails
    bad = _one(4, [-1, 0, 0, 1], [])
    mix = synth.LigandBatch.concat([batch.subset([0]), bad, batch.subset([1])])
    g = ctx.dock(pocket1, mix, params)
    assert list(g["status"]) == [0, lg.LG_EINVAL, 0]
    assert np.isnan(g["score"][1]) and g["best_restart"][1] == -1
    ref = ctx.dock(pocket1, batch.subset([0, 1]), params)
    assert np.array_equal(g["score"][[0, 2]], ref["score"])
    # non-ascending torsion list is rejected
    nonasc = _one(6, [-1, 0, 1, 2, 3, 4], [3, 2])
    assert ctx.dock(pocket1, nonasc, params)["status"][0] == lg.LG_EINVAL


def test_maximum_sizes(ctx, cfg1, pocket1):
    pocket, _, params = cfg1
    big = synth.make_ligands(123, np.array([lg.LG_MAX_ATOMS, 100, 2]), np.array([lg.LG_MAX_ROT, 20, 0]))
    assert big.n_rot()[0] >= 20
    p = synth.DockParams(restarts=3, passes=2, seed=params.seed)
    g = _dock(ctx, pocket1, big, p)
    check(pocket, big, p, g)
    # the plain form takes at most 32 warps; more restarts tile over them
    p40 = synth.DockParams(restarts=40, passes=1, seed=params.seed)
    sub = big.subset([1, 2])
    a = _dock(ctx, pocket1, sub, p40, mode=lg.LG_MODE_PLAIN)
    b = _dock(ctx, pocket1, sub, p40)
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    check(pocket, sub, p40, b)


def test_declared_maxima_reject_larger_ligands(ctx, cfg1, pocket1):
    _, batch, params = cfg1
    n = batch.n_atoms()
    g = ctx.dock(pocket1, batch.subset(range(40)), params, max_atoms=20)
    want = np.where(n[:40] <= 20, 0, lg.LG_EINVAL)
    assert np.array_equal(g["status"], want)
    ref = ctx.dock(pocket1, batch.subset(range(40)), params)
    ok = want == 0
    assert np.array_equal(g["score"][ok], ref["score"][ok])


def test_bad_arguments_raise(ctx, cfg1, pocket1):
    _, batch, params = cfg1
    with pytest.raises(lg.LgError) as e:
        ctx.dock(pocket1 + 99, batch.subset([0]), params)
    assert e.value.code == lg.LG_ENOPOCKET
    with pytest.raises(lg.LgError) as e:
        ctx.dock(pocket1, batch.subset([0]), synth.DockParams(restarts=0, passes=1))
    assert e.value.code == lg.LG_EINVAL


# ----------------------------------------------------------------------------- rigid refinement
def test_rigid_refinement_matches_oracle(ctx, cfg1, pocket1):
    import dataclasses
    pocket, batch, params = cfg1
    prm = dataclasses.replace(params, rigid_steps=2)
    sub = batch.subset(range(96))
    g = ctx.dock(pocket1, sub, prm, restart_score=True, restart_tors=True, restart_rigid=True)
    assert np.all(g["status"] == 0)
    rep = check(pocket, sub, prm, g)
    assert rep["rigid_decisions"] == sub.L * prm.restarts * prm.passes * prm.rigid_steps
    assert rep["rigid_deviations"] <= 0.01 * rep["rigid_decisions"] + 2, rep
    # rigid moves are taken, and the result differs from the torsion-only method
    assert np.any(g["restart_rigid"] != 0)
    base = ctx.dock(pocket1, sub, params)
    assert not np.array_equal(base["score"], g["score"])


def test_rigid_refinement_plain_equals_batched(ctx, cfg1, pocket1):
    import dataclasses
    _, batch, params = cfg1
    prm = dataclasses.replace(params, rigid_steps=3, rigid_shift=0.5)
    sub = batch.subset(range(40))
    a = ctx.dock(pocket1, sub, prm, restart_score=True, restart_tors=True, restart_rigid=True)
    b = ctx.dock(pocket1, sub, prm, restart_score=True, restart_tors=True, restart_rigid=True,
                 mode=lg.LG_MODE_PLAIN)
    for k in ("score", "best_restart", "tors_idx", "pose", "restart_score", "restart_tors", "restart_rigid"):
        assert np.array_equal(a[k], b[k]), k


def test_all_stages_together_on_heavy_tailed_ligands(ctx, cfg2_pocket):
    # ranking, rigid moves and decision ranks at once on ligands of all three
    # size classes: the two forms agree bit for bit, at every width; the
    # oracle replaying the GPU's torsion and rigid choices (ranking off: it
    # changes only which restart is reported) finds only near-ties
    import dataclasses
    pid = ctx.load_pocket(cfg2_pocket)
    heavy = synth.config_ligands(3, 3000)
    n = heavy.n_atoms()
    idx = np.sort(np.concatenate([np.nonzero(n > 64)[0][:6], np.nonzero(n <= 32)[0][:6],
                                  np.nonzero((n > 32) & (n <= 64))[0][:6]]))
    sub = heavy.subset(idx)
    prm = dataclasses.replace(synth.config_params(3), restarts=12, passes=2, cluster_rmsd=3.0, rescore_top=4,
                              rigid_steps=2)
    kw = dict(restart_score=True, restart_tors=True, restart_rigid=True, decision_rank=True)
    keys = ("score", "best_restart", "status", "tors_idx", "pose", "restart_score", "restart_tors", "restart_rigid",
            "decision_rank", "rank", "leader", "restart_geo")
    ref = ctx.dock(pid, sub, prm, mode=lg.LG_MODE_PLAIN, **kw)
    try:
        for w in (1, 2, 4):
            ctx.set_option("warps_per_cta", w)
            got = ctx.dock(pid, sub, prm, **kw)
            for k in keys:
                assert np.array_equal(got[k], ref[k]), (w, k)
    finally:
        ctx.set_option("warps_per_cta", 0)
    prm_r = dataclasses.replace(prm, cluster_rmsd=0.0, rescore_top=0)
    g = ctx.dock(pid, sub, prm_r, **kw)
    ctx.unload_pocket(pid)
    for k in ("restart_score", "restart_tors", "restart_rigid", "decision_rank"):
        assert np.array_equal(g[k], ref[k]), k  # ranking leaves every restart as it was
    rep = check(cfg2_pocket, sub, prm_r, g)
    assert rep["deviations"] <= 0.01 * rep["decisions"] + 2, rep
    assert rep["rigid_deviations"] <= 0.01 * rep["rigid_decisions"] + 2, rep


def test_small_split_batches_take_wide_ctas(ctx, cfg2_pocket):
    # a heavy-tailed batch small enough for one wave of 8-lane, 8-warp CTAs
    # (but not of 16-lane, 15-warp ones): every size class runs with all 30
    # restarts of a ligand in flight, untuned, with the results of 1 warp
    pid = ctx.load_pocket(cfg2_pocket)
    heavy = synth.config_ligands(3, 3000)
    n = heavy.n_atoms()
    sub = heavy.subset(np.sort(np.concatenate([np.nonzero(n > 64)[0][:30], np.nonzero(n <= 64)[0][:170]])))
    prm = synth.config_params(3)
    ctx.set_option("autotune", 1)
    a = _dock(ctx, pid, sub, prm)
    st = ctx.stats()
    # prep + sort (3) + one launch per class, no trials
    assert (st.restart_lanes, st.warps_per_cta, st.launches) == (8, 8, 6)
    ctx.set_option("warps_per_cta", 1)
    try:
        b = _dock(ctx, pid, sub, prm)
    finally:
        ctx.set_option("warps_per_cta", 0)
    ctx.unload_pocket(pid)
    for k in a:
        if a[k] is not None:
            assert np.array_equal(a[k], b[k]), k


def test_rigid_refinement_throughput_ligands(ctx, cfg2_pocket):
    import dataclasses
    sub = synth.config_ligands(2, 48)
    prm = dataclasses.replace(synth.config_params(2), rigid_steps=1)
    pid = ctx.load_pocket(cfg2_pocket)
    g = ctx.dock(pid, sub, prm, restart_score=True, restart_tors=True, restart_rigid=True)
    ctx.unload_pocket(pid)
    rep = check(cfg2_pocket, sub, prm, g)
    assert rep["rigid_deviations"] <= 0.01 * rep["rigid_decisions"] + 2, rep


# ----------------------------------------------------------------------------- full sizes
def _slice_outputs(batch, gpu, idx, S, P):
    """The outputs of ligands idx of a docked batch, laid out as for batch.subset(idx)."""
    aoff, roff = batch.atom_off, batch.rot_off
    out = {k: [] for k in ("score", "best_restart", "status", "tors_idx", "pose", "restart_score", "restart_tors")}
    for l in idx:
        a0, a1, r0, r1 = int(aoff[l]), int(aoff[l + 1]), int(roff[l]), int(roff[l + 1])
        out["score"].append(gpu["score"][l:l + 1])
        out["best_restart"].append(gpu["best_restart"][l:l + 1])
        out["status"].append(gpu["status"][l:l + 1])
        out["tors_idx"].append(gpu["tors_idx"][P * r0:P * r1])
        out["pose"].append(gpu["pose"][3 * a0:3 * a1])
        out["restart_score"].append(gpu["restart_score"][S * l:S * (l + 1)])
        out["restart_tors"].append(gpu["restart_tors"][S * P * r0:S * P * r1])
    return {k: np.concatenate(v) for k, v in out.items()}


@pytest.mark.parametrize("cfg,L", [(2, 100_000), (3, 1_000_000)])
def test_full_size_launch_sampled_against_oracle(ctx, cfg2_pocket, cfg, L):
    # the throughput (100,000 ligands) and heavy-tailed (1,000,000 ligands)
    # workloads in the bench's launch configuration: device-resident batch,
    # declared maxima, one persistent launch (per size class); sampled ligands
    # are replayed in the oracle
    pid = ctx.load_pocket(cfg2_pocket)
    params = synth.config_params(cfg)
    batch = synth.config_ligands(cfg, L)
    S, P = params.restarts, params.passes
    gpu = ctx.dock(pid, batch, params, device_io=True, restart_score=True, restart_tors=True,
                   max_atoms=int(batch.n_atoms().max()), max_rot=max(1, int(batch.n_rot().max())))
    ctx.unload_pocket(pid)
    assert np.all(gpu["status"] == 0)
    rng = np.random.default_rng(cfg)
    idx = np.sort(rng.choice(L, size=48, replace=False))
    idx = np.concatenate([idx, [int(np.argmax(batch.n_atoms()))]])  # and the largest ligand
    sub = batch.subset(idx)
    rep = check(cfg2_pocket, sub, params, _slice_outputs(batch, gpu, idx, S, P))
    assert rep["deviations"] <= 0.01 * rep["decisions"] + 2, rep


# ----------------------------------------------------------------------------- invariants of GPU poses
def _bond_distance(parent):
    N = len(parent)
    adj = [[] for _ in range(N)]
    for i in range(1, N):
        adj[i].append(int(parent[i]))
        adj[int(parent[i])].append(i)
    D = np.full((N, N), 10 ** 6)
    for s in range(N):
        D[s, s] = 0
        front = [s]
        while front:
            nxt = []
            for v in front:
                for w in adj[v]:
                    if D[s, w] > D[s, v] + 1:
                        D[s, w] = D[s, v] + 1
                        nxt.append(w)
            front = nxt
    return D


def test_gpu_poses_keep_geometry_and_are_clash_free(ctx, cfg2_pocket):
    # the GPU's best poses: every bond length equals the input's to 1e-5 A
    # (measured: 3e-6 A after 3 passes of FP32 moves), and no pair three or
    # more bonds apart is closer than d_clash (up to the near-tie margin)
    pid = ctx.load_pocket(cfg2_pocket)
    params = synth.config_params(2)
    batch = synth.config_ligands(2, 200)
    g = ctx.dock(pid, batch, params)
    ctx.unload_pocket(pid)
    worst_bond = 0.0
    dc2 = float(np.float32(params.d_clash)) ** 2
    for l in range(batch.L):
        a0, a1 = int(batch.atom_off[l]), int(batch.atom_off[l + 1])
        par = batch.parent[a0:a1].astype(int)
        X0 = np.stack([batch.x[a0:a1], batch.y[a0:a1], batch.z[a0:a1]], 1).astype(np.float64)
        X = g["pose"][3 * a0:3 * a1].reshape(-1, 3).astype(np.float64)
        b0 = np.linalg.norm(X0[1:] - X0[par[1:]], axis=1)
        b1 = np.linalg.norm(X[1:] - X[par[1:]], axis=1)
        worst_bond = max(worst_bond, float(np.abs(b1 - b0).max(initial=0.0)))
        D = _bond_distance(par)
        i, j = np.nonzero(np.triu(D >= 3))
        d2 = ((X[i] - X[j]) ** 2).sum(1)
        assert np.all(d2 >= dc2 * (1 - 1e-4)), (l, float(d2.min()))
    assert worst_bond <= 1e-5, worst_bond
    print("worst bond-length change (A):", worst_bond)
