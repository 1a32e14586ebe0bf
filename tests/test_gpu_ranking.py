"""GPU pose ranking (Sec. 3.1, steps 3-4) through the C-ABI against the FP64
oracle: geometric scores, geometric order, greedy leader clustering, the
ranked list and the rescored best pose.

The GPU's restarts are replayed in the oracle (as in the docking parity
check), so both sides rank the same poses.  What is unique is compared
exactly; where FP32 rounding can decide (two geometric scores within
TOL_G, an RMSD within TOL_RMSD2 of the threshold, two scores within
TOL_SCORE) the GPU's choice is checked to be one of the valid ones."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2110_11644_gb300 import lg, synth

pytestmark = pytest.mark.gpu

TOL_G = 1e-5        # relative, on the geometric score
TOL_RMSD2 = 1e-4    # relative, on RMSD^2 against the threshold^2 (FP32 sum over 3N terms)
TOL_SCORE = 1e-5    # relative, on the pose score


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


def _ranked(params, thr, K, restarts=None):
    kw = dict(cluster_rmsd=thr, rescore_top=K)
    if restarts is not None:
        kw["restarts"] = restarts
    return dataclasses.replace(params, **kw)


def _dock(ctx, pid, batch, params, **kw):
    return ctx.dock(pid, batch, params, restart_score=True, restart_tors=True, **kw)


def check_ranking(pocket, batch, params, gpu):
    """Validate the GPU ranking outputs against the oracle replay of the GPU's
    decisions; returns counts of exact agreement."""
    S, thr = params.restarts, float(params.cluster_rmsd)
    K = params.rescore_top if 0 < params.rescore_top <= S else S
    rep = oracle.dock(pocket, batch, params, replay=gpu["restart_tors"], poses=True)
    aoff = batch.atom_off
    same_order = same_leader = 0
    for l in range(batch.L):
        N = int(aoff[l + 1] - aoff[l])
        a0 = int(aoff[l])
        X = rep["poses"][3 * S * a0:3 * S * (a0 + N)].reshape(S, N, 3)
        E_o = rep["restart_E"][l]
        scale = np.maximum(np.abs(E_o), rep["restart_Eabs"][l])
        E_g = gpu["restart_score"][l * S:(l + 1) * S]
        assert np.all(np.abs(E_g - E_o) <= TOL_SCORE * scale), f"ligand {l}: restart scores"
        G_o = rep["geo"][l]
        G_g = gpu["restart_geo"][l * S:(l + 1) * S]
        tolG = TOL_G * np.maximum(np.abs(G_o), 1.0)
        assert np.all(np.abs(G_g - G_o) <= tolG), f"ligand {l}: geometric scores"
        rank = gpu["rank"][l * S:(l + 1) * S]
        lead = gpu["leader"][l * S:(l + 1) * S]
        assert sorted(rank.tolist()) == list(range(S)), f"ligand {l}: rank is not a permutation"
        # geometric order implied by the GPU's own G (exact: same values, same rule)
        geo = sorted(range(S), key=lambda r: (-G_g[r], r))
        # the oracle's order may differ only by swapping near-tied neighbours
        for p in range(S - 1):
            a, b = geo[p], geo[p + 1]
            if G_o[a] < G_o[b]:
                assert G_o[b] - G_o[a] <= tolG[a] + tolG[b], f"ligand {l}: geometric order"
        # leaders: first earlier leader within thr (FP64 RMSD^2 of the replayed poses)
        D2 = ((X[:, None] - X[None]) ** 2).sum(-1).mean(-1) if thr > 0 else np.full((S, S), np.inf)
        leaders = []
        for r in geo:
            ls = np.array(leaders, dtype=np.int64)
            d2 = D2[r, ls]
            near = np.abs(d2 - thr * thr) <= TOL_RMSD2 * thr * thr
            within = d2 <= thr * thr
            if lead[r] == r:
                assert not np.any(within & ~near), f"ligand {l}: restart {r} leads but is within thr of a leader"
                leaders.append(r)
                continue
            hit = np.nonzero(ls == lead[r])[0]
            assert hit.size == 1, f"ligand {l}: restart {r} has leader {lead[r]} that is no earlier leader"
            j = int(hit[0])
            assert within[j] or near[j], f"ligand {l}: restart {r} joined leader {lead[r]} at RMSD^2 {d2[j]}"
            assert not np.any(within[:j] & ~near[:j]), f"ligand {l}: restart {r} skipped an earlier leader"
        want = [r for r in geo if lead[r] == r] + [r for r in geo if lead[r] != r]
        assert rank.tolist() == want, f"ligand {l}: ranking is not leaders-then-members in geometric order"
        # rescoring: the GPU's best is the lowest replayed E among its first K
        top = rank[:K]
        ro = int(top[np.argmin(E_o[top])])
        rg = int(gpu["best_restart"][l])
        assert rg in top.tolist(), f"ligand {l}: best restart outside the first K"
        assert abs(E_o[rg] - E_o[ro]) <= TOL_SCORE * max(scale[rg], scale[ro]), f"ligand {l}: rescored best"
        assert gpu["score"][l] == gpu["restart_score"][l * S + rg]
        same_order += int(np.array_equal(rank, rep["order"][l]))
        same_leader += int(np.array_equal(lead, rep["leader"][l]))
    return dict(same_order=same_order, same_leader=same_leader, L=batch.L)


@pytest.mark.parametrize("thr,K", [(9.0, 4), (3.0, 0), (9.0, 0), (0.0, 3), (1.5, 1)])
def test_ranking_matches_oracle(ctx, cfg1, pocket1, thr, K):
    pocket, full, params = cfg1
    batch = full.subset(range(96))
    prm = _ranked(params, thr, K)
    gpu = _dock(ctx, pocket1, batch, prm)
    assert np.all(gpu["status"] == 0)
    res = check_ranking(pocket, batch, prm, gpu)
    # rounding decides only rarely: most ligands agree with the oracle outright
    assert res["same_order"] >= 0.9 * res["L"] and res["same_leader"] >= 0.9 * res["L"], res


def test_ranking_ragged_restarts(ctx, cfg1, pocket1):
    pocket, full, params = cfg1
    batch = full.subset(range(40))
    for S in (13, 40, 97):  # ragged restart tiles and bit-matrix rows
        prm = _ranked(params, 9.0, 5, restarts=S)
        gpu = _dock(ctx, pocket1, batch, prm)
        assert np.all(gpu["status"] == 0)
        res = check_ranking(pocket, batch, prm, gpu)
        assert res["same_order"] >= 0.9 * res["L"], res


def test_ranking_paper_setting(ctx, cfg1, pocket1):
    # 256 restarts, 3 A, the top 30 rescored (the paper's experiment)
    pocket, full, params = cfg1
    batch = full.subset(range(24))
    prm = _ranked(params, 3.0, 30, restarts=256)
    gpu = _dock(ctx, pocket1, batch, prm)
    assert np.all(gpu["status"] == 0)
    res = check_ranking(pocket, batch, prm, gpu)
    assert res["same_order"] >= 0.9 * res["L"], res


def test_ranking_max_restarts_runs(ctx, cfg1, pocket1):
    # the largest restart count: the ranking is a permutation led by the leaders,
    # and plain and batched forms agree bitwise
    _, full, params = cfg1
    batch = full.subset(range(6))
    S = 1024
    prm = _ranked(params, 6.0, 30, restarts=S)
    a = _dock(ctx, pocket1, batch, prm)
    b = _dock(ctx, pocket1, batch, prm, mode=lg.LG_MODE_PLAIN)
    for k in ("score", "best_restart", "rank", "leader", "restart_geo"):
        assert np.array_equal(a[k], b[k]), k
    for l in range(batch.L):
        rank, lead = a["rank"][l * S:(l + 1) * S], a["leader"][l * S:(l + 1) * S]
        assert sorted(rank.tolist()) == list(range(S))
        n_lead = int(np.sum(lead == np.arange(S)))
        assert np.all(lead[rank[:n_lead]] == rank[:n_lead]) and np.all(lead[rank[n_lead:]] != rank[n_lead:])


def test_ranking_at_maximum_sizes(ctx, cfg1, pocket1):
    # the largest ligand (128 atoms, 32 torsional bonds) with 1,024 ranked
    # restarts and rigid moves: plain and batched forms agree bitwise
    _, _, params = cfg1
    big = synth.make_ligands(321, np.array([lg.LG_MAX_ATOMS, 70]), np.array([lg.LG_MAX_ROT, 10]))
    S = 1024
    prm = dataclasses.replace(_ranked(params, 6.0, 30, restarts=S), passes=1, rigid_steps=1)
    a = ctx.dock(pocket1, big, prm, restart_score=True, restart_tors=True, restart_rigid=True, decision_rank=True)
    b = ctx.dock(pocket1, big, prm, restart_score=True, restart_tors=True, restart_rigid=True, decision_rank=True,
                 mode=lg.LG_MODE_PLAIN)
    for k in ("score", "best_restart", "status", "rank", "leader", "restart_geo", "restart_score", "restart_tors",
              "restart_rigid", "decision_rank", "pose"):
        assert np.array_equal(a[k], b[k]), k
    assert np.all(a["status"] == 0)


def test_ranking_plain_equals_batched(ctx, cfg1, pocket1):
    _, full, params = cfg1
    batch = full.subset(range(48))
    prm = _ranked(params, 9.0, 4)
    a = _dock(ctx, pocket1, batch, prm)
    b = _dock(ctx, pocket1, batch, prm, mode=lg.LG_MODE_PLAIN)
    for k in ("score", "best_restart", "status", "tors_idx", "pose", "restart_score", "restart_tors", "rank",
              "leader", "restart_geo"):
        assert np.array_equal(a[k], b[k]), k


def test_ranking_device_io_equals_host(ctx, cfg1, pocket1):
    _, full, params = cfg1
    batch = full.subset(range(48))
    prm = _ranked(params, 3.0, 6)
    a = _dock(ctx, pocket1, batch, prm)
    b = _dock(ctx, pocket1, batch, prm, device_io=True)
    for k in ("score", "best_restart", "rank", "leader", "restart_geo", "pose"):
        assert np.array_equal(a[k], b[k]), k


def test_rescore_all_without_clustering_is_plain_best(ctx, cfg1, pocket1):
    # K >= S and no clustering: ranking is off and the result is the lowest score
    _, full, params = cfg1
    batch = full.subset(range(32))
    a = _dock(ctx, pocket1, batch, params)
    b = _dock(ctx, pocket1, batch, _ranked(params, 0.0, params.restarts))
    assert b["rank"] is None
    assert np.array_equal(a["score"], b["score"]) and np.array_equal(a["best_restart"], b["best_restart"])
    # clustering at a threshold no two poses meet, rescoring all: same best pose
    c = _dock(ctx, pocket1, batch, _ranked(params, 1e-6, 0))
    assert np.array_equal(a["score"], c["score"]) and np.array_equal(a["best_restart"], c["best_restart"])
    S = params.restarts
    assert np.array_equal(c["leader"].reshape(-1, S), np.tile(np.arange(S, dtype=np.int32), (batch.L, 1)))


def test_ranking_bad_parameters_rejected(ctx, cfg1, pocket1):
    _, full, params = cfg1
    batch = full.subset(range(4))
    for thr, K in ((-1.0, 0), (float("nan"), 0), (float("inf"), 0), (3.0, -2)):
        with pytest.raises(lg.LgError):
            _dock(ctx, pocket1, batch, _ranked(params, thr, K))
    # the context stays usable
    assert np.all(_dock(ctx, pocket1, batch, params)["status"] == 0)


def test_ranking_served_equals_direct(ctx, cfg1, pocket1):
    _, full, params = cfg1
    prm = _ranked(params, 9.0, 4)
    subs = [full.subset(range(s, s + n)) for s, n in ((0, 5), (5, 30), (35, 12))]
    reqs, tickets = [], []
    for sub in subs:
        arrs = lg.host_batch_arrays(sub)
        b = lg.make_batch_struct(arrs, sub.L)
        p = lg.make_params(prm.restarts, prm.passes, prm.seed, prm.d_clash, cluster_rmsd=prm.cluster_rmsd,
                           rescore_top=prm.rescore_top)
        r, outs = lg.alloc_result(sub.L, int(sub.atom_off[-1]), int(sub.rot_off[-1]), prm.restarts, prm.passes,
                                  ranking=True)
        reqs.append((sub, arrs, b, p, r, outs))
        tickets.append(lg.lg_stream_submit(ctx.h, pocket1, b, p, r))
    for t in tickets:
        assert lg.lg_stream_wait(ctx.h, t, 60000) == lg.LG_OK
    S = prm.restarts
    for sub, _, _, _, _, outs in reqs:
        d = ctx.dock(pocket1, sub, prm)
        for k in ("score", "best_restart", "rank", "leader", "restart_geo"):
            n = sub.L * (S if k in ("rank", "leader", "restart_geo") else 1)
            assert np.array_equal(outs[k][:n], d[k][:n]), k
