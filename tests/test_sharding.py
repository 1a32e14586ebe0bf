"""Ligand sharding over ranks (host logic), world_size 2 on CPU with gloo.

Each rank docks its cost-balanced shard -- with the FP64 oracle standing in
for the rank's GPU -- and the global ranking gathered on rank 0 equals the
ranking of the whole library docked in one process.
"""
import os
import socket

import numpy as np
import pytest

from paper_2110_11644_gb300 import shard, synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import torch.distributed as dist

    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pocket = synth.config_pocket(1)
        batch = synth.config_ligands(1, 96)
        params = synth.config_params(1)
        parts = shard.partition(shard.ligand_flops(batch, params.restarts, params.passes), world)
        mine = batch.subset(parts[rank])
        out = oracle.dock(pocket, mine, params, nthreads=2)
        top = shard.gather_ranking(mine.uid, out["best_E"], k=20)
        if rank == 0:
            q.put((top[0].tolist(), top[1].tolist()))
    finally:
        dist.destroy_process_group()


def test_partition_balances_and_covers():
    rng = np.random.default_rng(0)
    costs = rng.lognormal(0, 1, size=1000)
    parts = shard.partition(costs, 4)
    allidx = np.sort(np.concatenate(parts))
    assert np.array_equal(allidx, np.arange(1000))
    loads = np.array([costs[p].sum() for p in parts])
    assert loads.max() / loads.mean() < 1.01
    # equal-size slabs of a heavy-tailed library are far less balanced
    slabs = np.array_split(np.arange(1000), 4)
    slab_loads = np.array([costs[s].sum() for s in slabs])
    assert slab_loads.max() / slab_loads.mean() > loads.max() / loads.mean()


# uids above 2^53 (not exact in FP64) and at or above 2^63 (negative as int64)
_BIG_UIDS = np.array([2 ** 53 + 1, 2 ** 53 + 3, 2 ** 63 - 1, 2 ** 63, 2 ** 63 + 5, 2 ** 64 - 1, 7, 2 ** 53 + 2],
                     np.uint64)
_BIG_SCORES = np.array([-3.0, -3.0, 1.5, -3.0, 0.25, -3.0, np.nan, 1.5])


def _gather_big(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = np.arange(rank, len(_BIG_UIDS), world)
        top = shard.gather_ranking(_BIG_UIDS[mine], _BIG_SCORES[mine], k=6)
        if rank == 0:
            q.put(([int(v) for v in top[0]], top[1].tolist(), str(top[0].dtype)))
    finally:
        dist.destroy_process_group()


def test_gather_keeps_full_64_bit_uids():
    # the gathered uids are the exact uint64 values, ordered by score, then uid
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gather_big, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    uids, scores, dtype = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert dtype == "uint64"
    ok = np.isfinite(_BIG_SCORES)
    want = sorted(zip(_BIG_SCORES[ok].tolist(), [int(u) for u in _BIG_UIDS[ok]]))[:6]
    assert uids == [u for _, u in want]
    assert scores == [s for s, _ in want]
    assert uids[:4] == [2 ** 53 + 1, 2 ** 53 + 3, 2 ** 63, 2 ** 64 - 1]


def test_ligand_flops_matches_moving_atoms():
    import oracle
    b = synth.config_ligands(2, 50)
    m = shard.moving_atoms_per_ligand(b)
    for l in range(b.L):
        lig = b.ligand(l)
        end = oracle.subtree_end(lig["parent"])
        assert m[l] == sum(int(end[c]) - int(c) - 1 for c in lig["rot_child"])


def test_two_rank_gather_equals_single_process():
    import multiprocessing as mp

    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    pocket = synth.config_pocket(1)
    batch = synth.config_ligands(1, 96)
    params = synth.config_params(1)
    out = oracle.dock(pocket, batch, params)
    order = np.lexsort((batch.uid, out["best_E"]))[:20]
    assert got[0] == batch.uid[order].tolist()
    assert np.allclose(got[1], out["best_E"][order], rtol=0, atol=0)


def test_cost_model_counts_match_brute_force():
    # moving atoms and clash pairs per ligand against breadth-first topological
    # distances on the bond tree
    from collections import deque
    batch = synth.config_ligands(2, 60)
    m_got = shard.moving_atoms_per_ligand(batch)
    p_got = shard.clash_pairs_per_ligand(batch)
    for l in range(batch.L):
        a0, a1 = int(batch.atom_off[l]), int(batch.atom_off[l + 1])
        N = a1 - a0
        par = batch.parent[a0:a1].astype(int)
        adj = [[] for _ in range(N)]
        for i in range(1, N):
            adj[i].append(par[i])
            adj[par[i]].append(i)
        dist = np.zeros((N, N), int)
        for s in range(N):
            d = [-1] * N
            d[s] = 0
            dq = deque([s])
            while dq:
                u = dq.popleft()
                for v in adj[u]:
                    if d[v] < 0:
                        d[v] = d[u] + 1
                        dq.append(v)
            dist[s] = d
        m_want = p_want = 0
        for k in range(int(batch.rot_off[l]), int(batch.rot_off[l + 1])):
            b = int(batch.rot_child[k])
            sub = {b}
            for i in range(b + 1, N):       # preorder: a subtree is contiguous
                if par[i] in sub:
                    sub.add(i)
                else:
                    break
            moving = sorted(sub - {b})
            fixed = [j for j in range(N) if j not in sub]
            m_want += len(moving)
            p_want += sum(1 for i in moving for j in fixed if dist[i, j] >= 3)
        assert m_got[l] == m_want and p_got[l] == p_want, l
    F = shard.ligand_flops(batch, 30, 3)
    N = np.diff(batch.atom_off)
    want = 30 * (21 * N + 40 + 3 * (36 * 51 * m_got + 8 * p_got) + 64 * N)
    assert np.allclose(F, want, rtol=0, atol=1e-6)


def test_ranked_flops_credit_each_decision():
    # j* from the oracle's own decisions (1 + steps ranked before the chosen
    # one); all ones give the lower bound; otherwise the pair term counts
    # j* * Pi_k * 8 decision by decision
    import oracle
    pocket = synth.config_pocket(1)
    batch = synth.config_ligands(1, 24)
    params = synth.config_params(1)
    S, P = params.restarts, params.passes
    out = oracle.dock(pocket, batch, params, trace=True)
    s = out["trace_s"].reshape(-1, 36)
    ch = out["choice"].astype(int)
    sc = s[np.arange(len(ch)), ch]
    jstar = 1 + ((s > sc[:, None]) | ((s == sc[:, None]) & (np.arange(36)[None, :] < ch[:, None]))).sum(1)
    assert jstar.max() > 1
    ones = shard.ligand_flops_ranked(batch, S, P, np.ones(len(ch)))
    assert np.allclose(ones, shard.ligand_flops(batch, S, P), rtol=0, atol=1e-6)
    got = shard.ligand_flops_ranked(batch, S, P, jstar)
    m, pairs, rl, _ = shard._bond_counts(batch)
    for l in range(batch.L):
        N = int(batch.atom_off[l + 1] - batch.atom_off[l])
        r0, R = int(batch.rot_off[l]), int(batch.rot_off[l + 1] - batch.rot_off[l])
        want = S * (21 * N + 40 + 64 * N)
        for r in range(S):
            for ps in range(P):
                for k in range(R):
                    d = S * P * r0 + (r * P + ps) * R + k
                    want += 36 * 51 * m[r0 + k] + 8 * pairs[r0 + k] * jstar[d]
        assert abs(got[l] - want) <= 1e-9 * want, l


def test_resume_after_a_failed_rank_docks_only_the_missing_uids():
    # a rank fails after its first chunk; the resumed run docks the pending
    # uids only and the union equals one uninterrupted run bit for bit
    import oracle
    pocket = synth.config_pocket(1)
    batch = synth.config_ligands(1, 64)
    params = synth.config_params(1)
    whole = oracle.dock(pocket, batch, params, nthreads=2)
    parts = shard.partition(shard.ligand_flops(batch, params.restarts, params.passes), 2)
    done_uid, done_E, done_r = [], [], []
    for rank, idx in enumerate(parts):
        chunks = np.array_split(idx, 3)
        for c, chunk in enumerate(chunks):
            if rank == 1 and c == 1:
                break  # rank 1 fails here; its first chunk's results were kept
            out = oracle.dock(pocket, batch.subset(chunk), params, nthreads=2)
            done_uid += list(batch.uid[chunk]); done_E += list(out["best_E"]); done_r += list(out["best_r"])
    todo = shard.pending(batch.uid, done_uid)
    assert 0 < len(todo) < batch.L and not np.isin(batch.uid[todo], done_uid).any()
    out = oracle.dock(pocket, batch.subset(todo), params, nthreads=2)
    done_uid += list(batch.uid[todo]); done_E += list(out["best_E"]); done_r += list(out["best_r"])
    order = np.argsort(np.asarray(done_uid, np.uint64))
    want = np.argsort(batch.uid)
    assert np.array_equal(np.asarray(done_uid, np.uint64)[order], batch.uid[want])
    assert np.array_equal(np.asarray(done_E)[order], whole["best_E"][want])
    assert np.array_equal(np.asarray(done_r)[order], whole["best_r"][want])
    assert len(shard.pending(batch.uid, done_uid)) == 0


def test_pending_edge_cases():
    uid = np.array([5, 3, 9, 1], np.uint64)
    assert np.array_equal(shard.pending(uid, []), np.arange(4))
    assert len(shard.pending(uid, uid)) == 0
    assert np.array_equal(shard.pending(uid, np.array([9, 7], np.uint64)), np.array([0, 1, 3]))
    assert len(shard.pending(np.zeros(0, np.uint64), uid)) == 0


def test_needed_flops_credit_only_decisions_before_the_exact_stop():
    # The oracle sweeps every decision.  After R decisions in a row without a
    # move, the state repeats a full round of bonds, so every later decision
    # of the oracle is step 0 too: the stop the kernels take is exact.  The
    # needed count credits the decisions up to the stop (j* from the
    # oracle's traces), and with no decision marked it equals the ranked count.
    import oracle
    pocket = synth.config_pocket(1)
    batch = synth.config_ligands(1, 24)
    params = synth.config_params(1)
    S, P = params.restarts, params.passes
    out = oracle.dock(pocket, batch, params, trace=True)
    s = out["trace_s"].reshape(-1, 36)
    ch = out["own"].astype(int)
    sc = s[np.arange(len(ch)), ch]
    jstar = 1 + ((s > sc[:, None]) | ((s == sc[:, None]) & (np.arange(36)[None, :] < ch[:, None]))).sum(1)
    coded = jstar.copy()
    m, pairs, _, _ = shard._bond_counts(batch)
    n_skipped = 0
    for l in range(batch.L):
        N = int(batch.atom_off[l + 1] - batch.atom_off[l])
        r0, R = int(batch.rot_off[l]), int(batch.rot_off[l + 1] - batch.rot_off[l])
        want = S * (21 * N + 40 + 64 * N)
        for r in range(S):
            zrun, stopped = 0, False
            for q in range(P * R):
                d = S * P * r0 + r * P * R + q
                if stopped:
                    assert ch[d] == 0  # the oracle repeats step 0 after the stop
                    coded[d] |= 0x80
                    n_skipped += 1
                    continue
                want += 36 * 51 * m[r0 + q % R] + 8 * pairs[r0 + q % R] * jstar[d]
                zrun = 0 if ch[d] else zrun + 1
                stopped = zrun >= R
        got = shard.ligand_flops_needed(batch, S, P, coded)[l]
        assert abs(got - want) <= 1e-9 * want, l
    assert n_skipped > 0
    ranked = shard.ligand_flops_ranked(batch, S, P, jstar)
    assert np.allclose(shard.ligand_flops_needed(batch, S, P, jstar), ranked, rtol=1e-12)
    # the marked ranks keep their j* for the ranked count
    assert np.allclose(shard.ligand_flops_ranked(batch, S, P, coded), ranked, rtol=1e-12)
