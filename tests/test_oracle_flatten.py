"""Pins of the FP64 flattening oracle (Sec. 3.1, step 1: turn the torsional
bonds to maximise the sum of all pairwise atom distances; no pocket).

Each pin restates what the definition fixes with independent tools (scipy
rotations and pdist, breadth-first bond distances, a closed-form dihedral),
so a dropped pair, a wrong moving set, a flipped rotation sense or a wrong
tie rule in the oracle fails one of them."""
import itertools

import numpy as np
import pytest
from scipy.spatial.distance import pdist
from scipy.spatial.transform import Rotation

import oracle
from paper_2110_11644_gb300 import synth

A = 36
D_CLASH = 2.0


def _subtree(parent, b):
    out = []
    for i in range(len(parent)):
        v = i
        while v != -1 and v != b:
            v = parent[v]
        if v == b:
            out.append(i)
    return np.array(out, np.int64)


def _topo_dist(parent):
    N = len(parent)
    adj = [[] for _ in range(N)]
    for i in range(1, N):
        adj[i].append(parent[i])
        adj[parent[i]].append(i)
    D = np.full((N, N), 10 ** 6, np.int64)
    for s in range(N):
        D[s, s] = 0
        frontier = [s]
        while frontier:
            nxt = []
            for v in frontier:
                for w in adj[v]:
                    if D[s, w] > D[s, v] + 1:
                        D[s, w] = D[s, v] + 1
                        nxt.append(w)
            frontier = nxt
    return D


def _turn(X, a, b, moving, theta):
    u = X[b] - X[a]
    u = u / np.linalg.norm(u)
    Y = X.copy()
    Y[moving] = Rotation.from_rotvec(theta * u).apply(X[moving] - X[b]) + X[b]
    return Y


def _xyz(lig):
    return np.stack([lig.x, lig.y, lig.z], 1).astype(np.float64)


def _chain(dihedral_deg, bond=1.5, angle_deg=109.5):
    """4-atom chain 0-1-2-3 with the given dihedral, torsional bond (1, 2)."""
    th = np.radians(180.0 - angle_deg)
    p0 = np.array([0.0, 0.0, 0.0])
    p1 = p0 + [bond, 0.0, 0.0]
    p2 = p1 + bond * np.array([np.cos(th), np.sin(th), 0.0])
    # atom 3: bond angle at 2, dihedral about 1->2
    b2 = (p2 - p1) / np.linalg.norm(p2 - p1)
    n = np.cross(p1 - p0, b2)
    n /= np.linalg.norm(n)
    m = np.cross(n, b2)
    phi = np.radians(dihedral_deg)
    d = np.array([-np.cos(np.radians(angle_deg)), np.sin(np.radians(angle_deg)) * np.cos(phi),
                  np.sin(np.radians(angle_deg)) * np.sin(phi)])
    p3 = p2 + bond * (d[0] * b2 + d[1] * m + d[2] * n)
    X = np.stack([p0, p1, p2, p3]).astype(np.float32)
    return synth.LigandBatch(np.array([0, 4], np.int32), X[:, 0].copy(), X[:, 1].copy(), X[:, 2].copy(),
                             np.zeros(4, np.float32), np.zeros(4, np.uint8), np.array([-1, 0, 1, 2], np.int16),
                             np.array([0, 1], np.int32), np.array([2], np.int16), np.array([5], np.uint64))


def _dihedral(p0, p1, p2, p3):
    b0, b1, b2 = p0 - p1, p2 - p1, p3 - p2
    b1 = b1 / np.linalg.norm(b1)
    v = b0 - np.dot(b0, b1) * b1
    w = b2 - np.dot(b2, b1) * b1
    return np.degrees(np.arctan2(np.dot(np.cross(b1, v), w), np.dot(v, w)))


def test_chain_turns_to_anti():
    # closed form: in a 4-atom chain only |x3 - x0| changes with the torsion and
    # it is largest at the anti conformation (dihedral 180 deg), which the 10 deg
    # grid reaches from a 60 deg start
    lig = _chain(60.0)
    assert abs(abs(_dihedral(*_xyz(lig))) - 60.0) < 1e-4
    out = oracle.flatten(lig, passes=1)
    X = out["xyz"].reshape(4, 3)
    assert abs(abs(_dihedral(*X)) - 180.0) < 1e-4
    assert out["own"][0] in (12, 24)
    D_in = pdist(_xyz(lig)).sum()
    assert out["D"][0] > D_in


def test_single_bond_step_equals_brute_force():
    batch = synth.config_ligands(1, 256)
    done = 0
    for l in range(batch.L):
        if batch.n_rot()[l] != 1:
            continue
        lig = batch.subset([l])
        par = lig.parent.astype(np.int64)
        b = int(lig.rot_child[0])
        a = int(par[b])
        sub = _subtree(par, b)
        moving = sub[sub != b]
        fixed = np.setdiff1d(np.arange(len(par)), sub)
        T = _topo_dist(par)
        X = _xyz(lig)
        Dt = np.empty(A)
        adm = np.zeros(A, bool)
        for t in range(A):
            Y = _turn(X, a, b, moving, 2 * np.pi * t / A)
            Dt[t] = pdist(Y).sum()
            pairs = [(i, j) for i in moving for j in fixed if T[i, j] >= 3]
            adm[t] = t == 0 or all(np.sum((Y[i] - Y[j]) ** 2) >= D_CLASH ** 2 for i, j in pairs)
        want = int(np.flatnonzero(adm & (Dt == Dt[adm].max()))[0])
        out = oracle.flatten(lig, passes=1, trace=True)
        assert out["own"][0] == want
        np.testing.assert_allclose(out["trace_D"][:A], Dt, rtol=1e-12)
        Yw = _turn(X, a, b, moving, 2 * np.pi * want / A)
        np.testing.assert_allclose(out["xyz"].reshape(-1, 3), Yw, atol=1e-9)
        done += 1
        if done == 12:
            break
    assert done >= 6


def test_flatten_invariants_and_monotone():
    for cfg, L in ((1, 64), (2, 24)):
        batch = synth.config_ligands(cfg, L)
        out = oracle.flatten(batch, passes=3, trace=True)
        assert np.all(out["status"] == 0)
        for l in range(batch.L):
            a0, a1 = int(batch.atom_off[l]), int(batch.atom_off[l + 1])
            r0, r1 = int(batch.rot_off[l]), int(batch.rot_off[l + 1])
            N, R = a1 - a0, r1 - r0
            par = batch.parent[a0:a1].astype(np.int64)
            X0 = np.stack([batch.x[a0:a1], batch.y[a0:a1], batch.z[a0:a1]], 1).astype(np.float64)
            X = out["xyz"][3 * a0:3 * a1].reshape(N, 3)
            # bonds and the never-moving atoms
            for i in range(1, N):
                assert abs(np.linalg.norm(X[i] - X[par[i]]) - np.linalg.norm(X0[i] - X0[par[i]])) < 1e-9
            movers = set()
            for k in range(r0, r1):
                b = int(batch.rot_child[k])
                movers |= set(int(i) for i in _subtree(par, b) if i != b)
            still = [i for i in range(N) if i not in movers]
            assert np.array_equal(X[still], X0[still])
            # the sum of distances never decreases, step by step and overall
            tr = out["trace_D"][A * 3 * r0:A * 3 * r1].reshape(3 * R, A)
            ch = out["choice"][3 * r0:3 * r1]
            for d in range(3 * R):
                assert tr[d, ch[d]] >= tr[d, 0]
            assert out["D"][l] >= pdist(X0).sum() - 1e-9
            np.testing.assert_allclose(out["D"][l], pdist(X).sum(), rtol=1e-12)
            # still clash-free (the generator's inputs are)
            T = _topo_dist(par)
            for i, j in zip(*np.nonzero(T >= 3)):
                assert np.sum((X[i] - X[j]) ** 2) >= D_CLASH ** 2 - 1e-9


def test_greedy_bounded_by_exhaustive_search():
    batch = synth.config_ligands(1, 256)
    tested = 0
    for l in range(batch.L):
        if batch.n_rot()[l] != 2 or batch.n_atoms()[l] > 16:
            continue
        lig = batch.subset([l])
        par = lig.parent.astype(np.int64)
        X = _xyz(lig)
        b1, b2 = (int(v) for v in lig.rot_child)
        best = -np.inf
        for t1, t2 in itertools.product(range(A), range(A)):
            Y = _turn(X, int(par[b1]), b1, [i for i in _subtree(par, b1) if i != b1], 2 * np.pi * t1 / A)
            Y = _turn(Y, int(par[b2]), b2, [i for i in _subtree(par, b2) if i != b2], 2 * np.pi * t2 / A)
            best = max(best, pdist(Y).sum())
        out = oracle.flatten(lig, passes=2)
        assert out["D"][0] <= best + 1e-9
        tested += 1
        if tested == 3:
            break
    assert tested >= 1


def test_replay_of_own_choices_is_identity():
    batch = synth.config_ligands(2, 16)
    a = oracle.flatten(batch, passes=2)
    b = oracle.flatten(batch, passes=2, replay=a["choice"])
    assert np.array_equal(a["xyz"], b["xyz"]) and np.array_equal(a["own"], b["own"])
    # planting another step changes the result and the oracle still reports its own choice
    rep = a["choice"].copy()
    k = int(np.flatnonzero(rep != 0)[0])
    rep[k] = (rep[k] + 1) % A
    c = oracle.flatten(batch, passes=2, replay=rep)
    assert not np.array_equal(c["xyz"], a["xyz"])
    assert c["own"][k] == a["own"][k]


def test_invalid_ligand_status():
    lig = _chain(60.0)
    bad = synth.LigandBatch(lig.atom_off, lig.x, lig.y, lig.z, lig.q, lig.type,
                            np.array([-1, 0, 0, 1], np.int16), lig.rot_off, lig.rot_child, lig.uid)
    assert oracle.flatten(bad, passes=1)["status"][0] != 0
