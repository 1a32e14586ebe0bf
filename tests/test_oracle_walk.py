"""Pins of the oracle's greedy torsion walk across bonds and passes (the
docking sweep and the flattening sweep, Sec. 3.1: torsional bonds handled one
after the other, greedy passes).

The other sweep pins fix one decision at a time (a single bond by brute
force), bound the result (exhaustive search), or use ligands whose decisions
do not depend on their order (separable stars).  None of them would notice a
walk that visits the bonds in another order, applies only its first pass, or
takes a later bond's axis from coordinates before an earlier move.  Here the
whole walk is restated from its starting conformation with independent tools:
for every pass and every torsional bond in ascending child order, the 36 steps
are scored at the CURRENT coordinates (scipy trilinear interpolation for
docking, scipy pdist sums for flattening), the clash pairs come from
breadth-first bond distances, the best admissible step (lowest on ties) is
applied with a scipy rotation about the axis of the moved coordinates, and
the walk goes on.  Every traced score and clash distance, every choice and
the final conformation must agree with the oracle's.
"""
import dataclasses

import numpy as np
from scipy.ndimage import map_coordinates
from scipy.spatial.distance import pdist
from scipy.spatial.transform import Rotation

import oracle
from paper_2110_11644_gb300 import synth

A = 36


# ----------------------------------------------------------------------------- helpers
def _subtree(parent, b):
    """Atoms whose ancestor chain reaches b (no use of the preorder ranges)."""
    out = []
    for i in range(len(parent)):
        v = i
        while v != -1 and v != b:
            v = parent[v]
        if v == b:
            out.append(i)
    return np.array(out, np.int64)


def _bond_distances(parent):
    """Topological (bond-count) distances by breadth-first search."""
    N = len(parent)
    adj = [[] for _ in range(N)]
    for i in range(1, N):
        adj[i].append(int(parent[i]))
        adj[int(parent[i])].append(i)
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


def _turned(X, a, b, moving, theta):
    """Moving atoms turned by theta about the axis X[a] -> X[b] through X[b]."""
    u = X[b] - X[a]
    u = u / np.linalg.norm(u)
    return Rotation.from_rotvec(theta * u).apply(X[moving] - X[b]) + X[b]


def _interp(pocket, pts):
    """Overlap grid at the points, trilinear with edge clamping (scipy)."""
    g = (np.atleast_2d(pts) - pocket.origin[None, :]) / pocket.h
    coords = np.stack([g[:, 2], g[:, 1], g[:, 0]])  # the array is indexed [k, j, i]
    return map_coordinates(pocket.phi_o.astype(np.float64), coords, order=1, mode="nearest", prefilter=False)


def _xyz(batch, l):
    a0, a1 = int(batch.atom_off[l]), int(batch.atom_off[l + 1])
    return np.stack([batch.x[a0:a1], batch.y[a0:a1], batch.z[a0:a1]], 1).astype(np.float64)


def _bond_sets(parent, b, D):
    """Moving set M (subtree of b without b), fixed set F (outside the subtree)
    and the (M, F) pairs three or more bonds apart."""
    sub = _subtree(parent, b)
    M = sub[sub != b]
    F = np.setdiff1d(np.arange(len(parent)), sub)
    far = D[np.ix_(M, F)] >= 3
    return M, F, far


def _min_d2(TM, XF, far):
    if TM.size == 0 or XF.size == 0 or not far.any():
        return np.inf
    d2 = ((TM[:, None, :] - XF[None, :, :]) ** 2).sum(-1)
    return float(d2[far].min())


def _walk(score_steps, X, parent, rot, passes, d_clash, trace_s, trace_d2, own, rel=1e-12):
    """Greedy walk from X; checks the oracle's traces and choices decision by
    decision (decision index ps * R + k) and returns the final coordinates and
    the number of decisions that moved."""
    D = _bond_distances(parent)
    dc2 = d_clash * d_clash
    order = sorted(int(b) for b in rot)  # ascending child order, whatever order rot is given in
    R = len(order)
    moves = 0
    for ps in range(passes):
        for k, b in enumerate(order):
            a = int(parent[b])
            M, F, far = _bond_sets(parent, b, D)
            dec = ps * R + k
            s = np.empty(A)
            d2 = np.empty(A)
            for t in range(A):
                TM = X[M] if t == 0 else _turned(X, a, b, M, 2 * np.pi * t / A)
                s[t] = score_steps(X, M, TM)
                d2[t] = _min_d2(TM, X[F], far)
            got_s = trace_s[dec * A:(dec + 1) * A]
            np.testing.assert_allclose(got_s, s, rtol=rel, atol=1e-12, err_msg=f"scores, decision {dec}")
            got_d2 = trace_d2[dec * A:(dec + 1) * A]
            fin = np.isfinite(d2)
            assert np.array_equal(np.isfinite(got_d2), fin), f"clash pairs, decision {dec}"
            np.testing.assert_allclose(got_d2[fin], d2[fin], rtol=1e-12, atol=1e-12)
            ok = (np.arange(A) == 0) | (d2 >= dc2)
            # the lowest admissible step with the highest score; scores equal
            # to rounding (flat stretches of the grid give exact ties in the
            # oracle's arithmetic) count as ties
            smax = s[ok].max()
            want = int(np.flatnonzero(ok & (s >= smax - 1e-11 * max(abs(smax), 1.0)))[0])
            got = int(own[dec])
            assert got == want, f"decision {dec}: oracle chose step {got}, restatement {want}"
            if want:
                X = X.copy()
                X[M] = _turned(X, a, b, M, 2 * np.pi * want / A)
                moves += 1
    return X, moves


def _batch_with(batch, ids):
    return batch.subset(list(ids))


# ----------------------------------------------------------------------------- docking
def _check_docking_walk(pocket, sub, params):
    out = oracle.dock(pocket, sub, params, trace=True, poses=True)
    assert np.all(out["status"] == 0)
    S, P = params.restarts, params.passes
    moves = 0
    for l in range(sub.L):
        a0, a1 = int(sub.atom_off[l]), int(sub.atom_off[l + 1])
        r0, r1 = int(sub.rot_off[l]), int(sub.rot_off[l + 1])
        N, R = a1 - a0, r1 - r0
        par = sub.parent[a0:a1].astype(np.int64)
        rot = sub.rot_child[r0:r1]
        X0 = _xyz(sub, l)
        for r in range(S):
            Rm, p, _ = oracle.restart_pose(pocket, params, int(sub.uid[l]), r)
            X = (X0 - X0.mean(0)) @ Rm.T + p
            d0 = S * P * r0 + r * P * R  # the ligand's decisions, restart r
            X, mv = _walk(lambda X, M, TM: float(_interp(pocket, TM).sum()) if len(M) else 0.0,
                          X, par, rot, P, float(np.float32(params.d_clash)),
                          out["trace_s"][d0 * A:(d0 + P * R) * A], out["trace_d2"][d0 * A:(d0 + P * R) * A],
                          out["own"][d0:d0 + P * R])
            moves += mv
            assert np.array_equal(out["choice"][d0:d0 + P * R], out["own"][d0:d0 + P * R])
            got = out["poses"][3 * (S * a0 + r * N):3 * (S * a0 + (r + 1) * N)].reshape(N, 3)
            np.testing.assert_allclose(got, X, atol=1e-9)
    return moves


def test_docking_walk_small_ligands_three_passes(cfg1):
    """Ligands of 12-30 atoms with 3 or 4 torsional bonds, 3 passes."""
    pocket, batch, prm = cfg1
    ids = [l for l in range(batch.L) if batch.n_rot()[l] >= 3][:6]
    assert len(ids) >= 4
    params = dataclasses.replace(prm, restarts=4, passes=3)
    moves = _check_docking_walk(pocket, _batch_with(batch, ids), params)
    assert moves > 0


def test_docking_walk_many_bonds(cfg2_pocket):
    """Throughput-workload ligands with 8 or more torsional bonds, 3 passes:
    long chains of dependent decisions, later passes that still move."""
    batch = synth.config_ligands(2, 400)
    ids = [l for l in range(batch.L) if batch.n_rot()[l] >= 8 and batch.n_atoms()[l] <= 40][:3]
    assert len(ids) == 3
    params = synth.DockParams(restarts=2, passes=3)
    sub = _batch_with(batch, ids)
    moves = _check_docking_walk(cfg2_pocket, sub, params)
    assert moves > 0
    # the walk is not a repetition of its first pass: some decision after the
    # first pass moves (else a first-pass-only walk would pass unnoticed)
    out = oracle.dock(cfg2_pocket, sub, params)
    later = 0
    for l in range(sub.L):
        r0, R = int(sub.rot_off[l]), int(sub.n_rot()[l])
        for r in range(params.restarts):
            d0 = params.restarts * params.passes * r0 + r * params.passes * R
            later += int(np.count_nonzero(out["own"][d0 + R:d0 + params.passes * R]))
    assert later > 0


# ----------------------------------------------------------------------------- flattening
def test_flattening_walk_across_bonds_and_passes():
    """The flattening sweep (sum of all pairwise distances) from the input
    conformation, several bonds, 3 passes."""
    batch = synth.config_ligands(2, 400)
    ids = [l for l in range(batch.L) if batch.n_rot()[l] >= 6 and batch.n_atoms()[l] <= 36][:4]
    assert len(ids) == 4
    sub = _batch_with(batch, ids)
    passes, dc = 3, 2.0
    out = oracle.flatten(sub, passes, dc, trace=True)
    assert np.all(out["status"] == 0)
    moves = later = 0
    for l in range(sub.L):
        a0, a1 = int(sub.atom_off[l]), int(sub.atom_off[l + 1])
        r0, r1 = int(sub.rot_off[l]), int(sub.rot_off[l + 1])
        N, R = a1 - a0, r1 - r0
        par = sub.parent[a0:a1].astype(np.int64)
        X = _xyz(sub, l)

        def dsum(X, M, TM):
            Y = X.copy()
            Y[M] = TM
            return float(pdist(Y).sum())

        d0 = passes * r0
        X, mv = _walk(dsum, X, par, sub.rot_child[r0:r1], passes, float(np.float32(dc)),
                      out["trace_D"][d0 * A:(d0 + passes * R) * A], out["trace_d2"][d0 * A:(d0 + passes * R) * A],
                      out["own"][d0:d0 + passes * R])
        moves += mv
        later += int(np.count_nonzero(out["own"][d0 + R:d0 + passes * R]))
        np.testing.assert_allclose(out["xyz"][3 * a0:3 * a1].reshape(N, 3), X, atol=1e-9)
        np.testing.assert_allclose(out["D"][l], pdist(X).sum(), rtol=1e-12)
    assert moves > 0 and later > 0
