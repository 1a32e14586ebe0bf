"""Pins of the oracle's rigid greedy refinement: after each torsion pass,
rigid_steps moves of the whole ligand, each the best of 13 candidates (stay,
+-shift along x, y, z, +-10 deg about x, y, z through the centroid) by the
geometric score G = sum over all atoms of the overlap grid.

Restated independently: candidates with scipy rotations about the centroid,
G with scipy's trilinear interpolation (edge-clamped), the greedy walk
re-run step by step from the restart pose."""
import dataclasses

import numpy as np
from scipy.ndimage import map_coordinates
from scipy.spatial.transform import Rotation

import oracle
from paper_2110_11644_gb300 import synth

A = 36


def _scipy_G(pocket, X):
    g = (np.atleast_2d(X) - pocket.origin[None, :]) / pocket.h
    coords = np.stack([g[:, 2], g[:, 1], g[:, 0]])
    return float(map_coordinates(pocket.phi_o.astype(np.float64), coords, order=1, mode="nearest",
                                 prefilter=False).sum())


def _candidate(X, cand, shift, angle):
    c = X.mean(0)
    if cand == 0:
        return X.copy()
    if cand <= 6:
        v = np.zeros(3)
        v[(cand - 1) // 2] = shift if cand % 2 == 1 else -shift
        return X + v
    axis = np.zeros(3)
    axis[(cand - 7) // 2] = 1.0
    th = angle if cand % 2 == 1 else -angle
    return Rotation.from_rotvec(th * axis).apply(X - c) + c


def _rigid_only(batch):
    """The same ligands without torsional bonds."""
    return synth.LigandBatch(batch.atom_off, batch.x, batch.y, batch.z, batch.q, batch.type, batch.parent,
                             np.zeros(batch.L + 1, np.int32), np.zeros(0, np.int16), batch.uid)


def test_candidates_match_scipy():
    rng = np.random.default_rng(3)
    X = rng.normal(0, 3, size=(11, 3)) + 7.0
    for cand in range(13):
        got = oracle.rigid_candidate(X, cand, 0.375, 2 * np.pi / A)
        np.testing.assert_allclose(got, _candidate(X, cand, 0.375, 2 * np.pi / A), atol=1e-12)
        # rigid: every pairwise distance kept
        d0 = np.linalg.norm(X[:, None] - X[None], axis=-1)
        d1 = np.linalg.norm(got[:, None] - got[None], axis=-1)
        np.testing.assert_allclose(d1, d0, atol=1e-12)


def test_greedy_walk_equals_step_by_step_restatement(cfg1):
    pocket, batch, prm = cfg1
    sub = _rigid_only(batch.subset(range(6)))
    params = dataclasses.replace(prm, restarts=3, passes=2, rigid_steps=3)
    out = oracle.dock(pocket, sub, params, trace=True, poses=True)
    S, P, Rs = params.restarts, params.passes, params.rigid_steps
    shift = float(np.float32(params.rigid_shift))
    for l in range(sub.L):
        a0, a1 = int(sub.atom_off[l]), int(sub.atom_off[l + 1])
        N = a1 - a0
        X0 = np.stack([sub.x[a0:a1], sub.y[a0:a1], sub.z[a0:a1]], 1).astype(np.float64)
        for r in range(S):
            Rm, p, _ = oracle.restart_pose(pocket, params, int(sub.uid[l]), r)
            X = (X0 - X0.mean(0)) @ Rm.T + p
            for d in range(P * Rs):
                dec = (S * P * Rs) * l + r * P * Rs + d
                G = np.array([_scipy_G(pocket, _candidate(X, c, shift, 2 * np.pi / A)) for c in range(13)])
                np.testing.assert_allclose(out["trace_G"][13 * dec:13 * dec + 13], G, rtol=1e-10, atol=1e-12)
                want = int(np.flatnonzero(G == G.max())[0])
                own = int(out["own_rigid"][dec])
                assert own == want or abs(G[own] - G[want]) <= 1e-10 * abs(G[want])
                assert G[own] >= G[0] - 1e-12          # never worse than staying
                X = _candidate(X, own, shift, 2 * np.pi / A)
            got = out["poses"][3 * (S * a0 + r * N):3 * (S * a0 + (r + 1) * N)].reshape(N, 3)
            np.testing.assert_allclose(got, X, atol=1e-9)


def test_rigid_moves_interleave_with_torsions_and_keep_geometry(cfg1):
    pocket, batch, prm = cfg1
    sub = batch.subset(range(12))
    params = dataclasses.replace(prm, rigid_steps=2)
    out = oracle.dock(pocket, sub, params, trace=True, poses=True)
    S = params.restarts
    # G never drops across a rigid decision; torsion decisions are still made
    tg = out["trace_G"].reshape(-1, 13)
    ch = out["choice_rigid"]
    assert np.all(tg[np.arange(len(ch)), ch] >= tg[:, 0])
    assert np.any(ch != 0)
    # bond lengths of the final poses equal the input's
    for l in range(sub.L):
        a0, a1 = int(sub.atom_off[l]), int(sub.atom_off[l + 1])
        N = a1 - a0
        par = sub.parent[a0:a1]
        X0 = np.stack([sub.x[a0:a1], sub.y[a0:a1], sub.z[a0:a1]], 1).astype(np.float64)
        b0 = np.linalg.norm(X0[1:] - X0[par[1:]], axis=1)
        for r in range(S):
            X = out["poses"][3 * (S * a0 + r * N):3 * (S * a0 + (r + 1) * N)].reshape(N, 3)
            np.testing.assert_allclose(np.linalg.norm(X[1:] - X[par[1:]], axis=1), b0, atol=1e-9)


def test_rigid_off_is_the_plain_method(cfg1):
    pocket, batch, prm = cfg1
    sub = batch.subset(range(8))
    a = oracle.dock(pocket, sub, prm)
    b = oracle.dock(pocket, sub, dataclasses.replace(prm, rigid_steps=0, rigid_shift=1.0))
    assert np.array_equal(a["restart_E"], b["restart_E"]) and np.array_equal(a["choice"], b["choice"])
    # and rigid moves change the result
    c = oracle.dock(pocket, sub, dataclasses.replace(prm, rigid_steps=2))
    assert not np.array_equal(a["restart_E"], c["restart_E"])
