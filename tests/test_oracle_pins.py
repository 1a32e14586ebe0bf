"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test pins one step of the dock-and-score method (Sec. 3.1 of the paper,
read as stated in oracle/oracle.c) to a published value, a closed form, a
mathematical invariant, an independent library routine (scipy) or a brute-force
search, chosen so that a dropped term, a wrong sign or index, or a transposed
operand in the oracle fails at least one of them.
"""
import itertools
import os

import numpy as np
import pytest
from scipy.ndimage import map_coordinates
from scipy.spatial.transform import Rotation

import oracle
from paper_2110_11644_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
A = 36


# ----------------------------------------------------------------------------- helpers
def _subtree(parent, b):
    """Atoms whose ancestor chain reaches b (independent of the oracle's range logic)."""
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
        adj[i].append(parent[i]); adj[parent[i]].append(i)
    D = np.full((N, N), 10 ** 6, np.int64)
    for s in range(N):
        D[s, s] = 0
        frontier = [s]
        while frontier:
            nxt = []
            for v in frontier:
                for w in adj[v]:
                    if D[s, w] > D[s, v] + 1:
                        D[s, w] = D[s, v] + 1; nxt.append(w)
            frontier = nxt
    return D


def _scipy_trilinear(pocket, grid, pts):
    """Trilinear interpolation with edge clamping by scipy (order=1, mode='nearest')."""
    g = (np.atleast_2d(pts) - pocket.origin[None, :]) / pocket.h
    coords = np.stack([g[:, 2], g[:, 1], g[:, 0]])       # array is indexed [k, j, i]
    return map_coordinates(grid.astype(np.float64), coords, order=1, mode="nearest", prefilter=False)


def _rot(axis_from, axis_to, theta, pts):
    u = axis_to - axis_from
    u = u / np.linalg.norm(u)
    return Rotation.from_rotvec(theta * u).apply(pts - axis_to) + axis_to


def _ligand_xyz(lig):
    return np.stack([lig["x"], lig["y"], lig["z"]], 1).astype(np.float64)


def _single(batch, l):
    return batch.subset([l])


# ----------------------------------------------------------------------------- Philox
def test_philox_known_answer_vectors():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert [int(o) for o in out] == v[6:10]


def test_philox_counter_sensitivity():
    # every counter and key word changes every output word (avalanche sanity)
    base = oracle.philox4x32_10([1, 2, 3, 4], [5, 6])
    for w in range(6):
        c = [1, 2, 3, 4, 5, 6]; c[w] ^= 1
        out = oracle.philox4x32_10(c[0:4], c[4:6])
        assert np.all(out != base)


# ----------------------------------------------------------------------------- rotations
def test_shoemake_is_a_rotation():
    rng = np.random.default_rng(1)
    for u in rng.random((500, 3)):
        R = oracle.shoemake(*u)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(R) - 1.0) < 1e-14


def test_shoemake_haar_moments():
    # For the Haar measure on SO(3): E[R] = 0, E[tr R] = 0, E[(tr R)^2] = 1,
    # and R e is uniform on the sphere: E[(Re)(Re)^T] = I/3.
    rng = np.random.default_rng(2)
    Rs = np.array([oracle.shoemake(*u) for u in rng.random((20000, 3))])
    tol = 5 * np.sqrt(1.0 / 3.0 / len(Rs))
    assert np.abs(Rs.mean(0)).max() < tol
    tr = np.trace(Rs, axis1=1, axis2=2)
    assert abs(tr.mean()) < 5 * tr.std() / np.sqrt(len(tr))
    assert abs((tr ** 2).mean() - 1.0) < 0.05
    v = Rs[:, :, 2]
    assert np.abs(v.T @ v / len(v) - np.eye(3) / 3).max() < 0.02


def test_restart_pose_wiring(cfg1):
    # Philox -> 24-bit uniforms -> Shoemake -> pocket point: rotations are Haar
    # distributed across restarts and the pocket point index is uniform.
    pocket, _, prm = cfg1
    Rs, idx = [], []
    for r in range(6000):
        R, p, i = oracle.restart_pose(pocket, prm, 12345, r)
        Rs.append(R); idx.append(i)
        if r < 50:
            assert np.allclose(p, pocket.origin + pocket.h * pocket.pocket_points[i])
    Rs = np.array(Rs)
    assert np.abs(Rs.mean(0)).max() < 5 * np.sqrt(1 / 3 / len(Rs))
    npp = len(pocket.pocket_points)
    hist = np.bincount(np.array(idx) * 20 // npp, minlength=20)
    chi2 = ((hist - len(idx) / 20) ** 2 / (len(idx) / 20)).sum()
    assert chi2 < 60  # 19 dof; p ~ 1e-6
    # different uids and seeds give different poses
    R0, _, _ = oracle.restart_pose(pocket, prm, 12345, 0)
    R1, _, _ = oracle.restart_pose(pocket, prm, 12346, 0)
    assert not np.allclose(R0, R1)


def test_rotate_about_matches_scipy_rotvec():
    rng = np.random.default_rng(3)
    for _ in range(200):
        xa, xb, x = rng.normal(size=(3, 3)) * 3
        th = rng.uniform(0, 2 * np.pi)
        got = oracle.rotate_about(xa, xb, np.cos(th), np.sin(th), x)
        want = _rot(xa, xb, th, x[None])[0]
        assert np.allclose(got, want, atol=1e-12)


# ----------------------------------------------------------------------------- trilinear
def test_trilinear_exact_on_trilinear_field():
    # f(i,j,k) = integer trilinear polynomial: node values are exact in FP32 and the
    # interpolant equals the polynomial everywhere inside the box (closed form).
    n, h = 12, 0.375
    origin = np.array([-1.5, 2.25, 0.125])
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    c = [3, -2, 5, 1, 2, -1, 3, -1]
    f = lambda i, j, k: (c[0] + c[1] * i + c[2] * j + c[3] * k + c[4] * i * j + c[5] * i * k + c[6] * j * k
                         + c[7] * i * j * k)
    grid = f(i, j, k).astype(np.float32)
    assert np.all(grid.astype(np.float64) == f(i, j, k))

    class P:  # minimal pocket
        pass
    P.n, P.h, P.origin = n, h, origin
    P.phi_o = P.phi_v = P.phi_e = grid
    P.pocket_points = np.zeros((1, 3), np.int32)
    P.type_w = np.ones(5, np.float32); P.k_out = 0.0
    rng = np.random.default_rng(4)
    g = rng.uniform(0, n - 1, size=(400, 3))
    pts = origin + h * g
    got = oracle.trilinear(P, "o", pts)
    want = f(g[:, 0], g[:, 1], g[:, 2])
    assert np.allclose(got, want, rtol=1e-12, atol=1e-9)
    # node values are reproduced exactly
    nodes = rng.integers(0, n, size=(100, 3))
    got = oracle.trilinear(P, "o", origin + h * nodes)
    assert np.array_equal(got, f(nodes[:, 0], nodes[:, 1], nodes[:, 2]).astype(np.float64))


def test_trilinear_matches_scipy_inside_and_outside(cfg1):
    pocket = cfg1[0]
    rng = np.random.default_rng(5)
    lo, hi = pocket.origin, pocket.origin + pocket.h * (pocket.n - 1)
    pts = rng.uniform(lo - 4.0, hi + 4.0, size=(3000, 3))     # includes clamped points
    for which, grid in (("o", pocket.phi_o), ("v", pocket.phi_v), ("e", pocket.phi_e)):
        got = oracle.trilinear(pocket, which, pts)
        want = _scipy_trilinear(pocket, grid, pts)
        assert np.allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(grid).max())


def test_trilinear_continuous_across_cells(cfg1):
    pocket = cfg1[0]
    rng = np.random.default_rng(6)
    for _ in range(200):
        node = rng.integers(1, pocket.n - 1, size=3)
        x = pocket.origin + pocket.h * node
        d = rng.normal(size=3); d /= np.linalg.norm(d)
        a = oracle.trilinear(pocket, "v", [x - 1e-9 * d])[0]
        b = oracle.trilinear(pocket, "v", [x + 1e-9 * d])[0]
        assert abs(a - b) < 1e-6 * max(1.0, abs(a))


# ----------------------------------------------------------------------------- pose energy
def test_energy_at_nodes_equals_direct_pairwise_sum(cfg1):
    pocket = cfg1[0]
    rng = np.random.default_rng(7)
    ijk = rng.integers(0, pocket.n, size=(300, 3))
    xyz = pocket.node_xyz(ijk)
    v, e = synth.direct_potentials(pocket, xyz)
    for t in range(5):
        q = rng.normal(0, 0.3, size=len(xyz)).astype(np.float32)
        types = np.full(len(xyz), t, np.uint8)
        aoff = np.arange(len(xyz) + 1, dtype=np.int32)
        E, _ = oracle.score_poses(pocket, aoff, xyz, q, types)
        want = pocket.type_w[t].astype(np.float64) * v + q.astype(np.float64) * e
        scale = np.abs(pocket.type_w[t] * v) + np.abs(q * e) + 1e-3
        assert np.all(np.abs(E - want) <= 2e-6 * scale)


def test_interpolation_error_within_second_derivative_bound(cfg1):
    # off the nodes, the oracle's trilinear lookup of the generator's grids
    # equals the direct pairwise sum up to the textbook interpolation bound
    # (h^2/8) * sum_i max |d^2 f / dx_i^2| over the cell.  Atoms whose cutoff
    # sphere crosses the cell make the field jump there; their terms enter the
    # reference as the trilinear interpolation of their values at the 8 nodes.
    # (Caught by it: transposed or shifted grids, a wrong interpolation order.)
    from paper_2110_11644_gb300.synth import (COULOMB_CUT, COULOMB_K, COULOMB_RMIN, LJ_CAP, LJ_CUT, LJ_EPS,
                                              LJ_R0, LJ_RMIN)
    pocket = cfg1[0]
    h, n = float(pocket.h), pocket.n
    atoms, qa = pocket.atoms_xyz, pocket.atoms_q
    rng = np.random.default_rng(21)
    g = rng.uniform(1, n - 2, size=(4000, 3))
    pts = pocket.origin + h * g
    dmin = np.linalg.norm(pts[:, None] - atoms[None], axis=-1).min(1)
    pts, g = pts[dmin > 3.5][:300], g[dmin > 3.5][:300]
    assert len(pts) >= 100
    e_int = oracle.trilinear(pocket, "e", pts)
    v_int = oracle.trilinear(pocket, "v", pts)
    corner = np.array([[c, b, a] for a in (0, 1) for b in (0, 1) for c in (0, 1)], np.float64)  # x fastest

    def coul(d):
        r = np.maximum(d, COULOMB_RMIN)
        return np.where(d < COULOMB_CUT, COULOMB_K / (4 * r * r), 0.0)

    def lj(d):
        x = LJ_R0 / np.maximum(d, LJ_RMIN)
        return np.where(d < LJ_CUT, LJ_EPS * (x ** 12 - 2 * x ** 6), 0.0)

    checked_v = 0
    for k in range(len(pts)):
        f = g[k] - np.floor(g[k])
        cxyz = pocket.origin + h * (np.floor(g[k]) + corner)
        w = np.prod(np.where(corner == 1, f, 1 - f), axis=1)           # trilinear weights of the nodes
        dc = np.linalg.norm(cxyz[:, None] - atoms[None], axis=-1)     # [8, na]
        dp = np.linalg.norm(pts[k] - atoms, axis=-1)
        r_lo = np.maximum(dc.min(0) - h * np.sqrt(3.0), 1e-3)          # lower bound of r over the cell
        r_hi = dc.max(0)
        # electrostatics: f = K q / (4 r^2), sum_i |f_ii| <= 18 K |q| / (4 r^4)
        cross = (r_lo < COULOMB_CUT) & (r_hi >= COULOMB_CUT)
        smooth = (r_hi < COULOMB_CUT) & ~cross
        ref = np.sum(qa[smooth] * coul(dp[smooth])) + np.sum(qa[cross] * (w @ coul(dc[:, cross])))
        bound = (h * h / 8) * np.sum(18 * COULOMB_K * np.abs(qa[smooth]) / (4 * r_lo[smooth] ** 4))
        assert abs(e_int[k] - ref) <= bound + 1e-6 * (abs(ref) + 1), (k, e_int[k], ref, bound)
        # vdW-like: |f''| + 2 |f'| / r bounds sum_i |f_ii|; only where the cap is not reached
        if (lj(dc).sum(1) >= LJ_CAP).any() or lj(dp).sum() >= LJ_CAP:
            continue
        cross = (r_lo < LJ_CUT) & (r_hi >= LJ_CUT)
        smooth = (r_hi < LJ_CUT) & ~cross
        r = r_lo[smooth]
        f1 = LJ_EPS * (12 * LJ_R0 ** 12 / r ** 13 + 12 * LJ_R0 ** 6 / r ** 7)
        f2 = LJ_EPS * (156 * LJ_R0 ** 12 / r ** 14 + 84 * LJ_R0 ** 6 / r ** 8)
        ref = np.sum(lj(dp[smooth])) + np.sum(w @ lj(dc[:, cross]))
        bound = (h * h / 8) * np.sum(f2 + 2 * f1 / r)
        assert abs(v_int[k] - ref) <= bound + 1e-6 * (abs(ref) + 1), (k, v_int[k], ref, bound)
        checked_v += 1
    assert checked_v >= 100


def test_energy_outside_box_adds_linear_penalty(cfg1):
    pocket = cfg1[0]
    hi = pocket.origin + pocket.h * (pocket.n - 1)
    edge = np.array([hi[0], pocket.origin[1] + 5 * pocket.h, pocket.origin[2] + 7 * pocket.h])
    q = np.array([0.3], np.float32); t = np.array([2], np.uint8)
    E0, _ = oracle.pose_energy(pocket, edge, q, t)
    for D in (0.5, 2.0, 7.25):
        out = edge + np.array([D, 0, 0])
        E, _ = oracle.pose_energy(pocket, out, q, t)
        assert abs(E - (E0 + pocket.k_out * D)) < 1e-9 * max(1, abs(E))
    # diagonal exit: Euclidean distance to the clamped point
    out = hi + np.array([3.0, 4.0, 0.0])
    E, _ = oracle.pose_energy(pocket, out, q, t)
    Ec, _ = oracle.pose_energy(pocket, hi, q, t)
    assert abs(E - (Ec + pocket.k_out * 5.0)) < 1e-9 * max(1, abs(E))


def test_score_poses_sums_atoms(cfg1):
    pocket, batch, _ = cfg1
    xyz = np.stack([batch.x, batch.y, batch.z], 1).astype(np.float64) * 0.2 + pocket.center
    E, A_ = oracle.score_poses(pocket, batch.atom_off, xyz, batch.q, batch.type)
    aoff = np.arange(len(batch.x) + 1, dtype=np.int32)
    e1, a1 = oracle.score_poses(pocket, aoff, xyz, batch.q, batch.type)
    assert np.allclose(E, np.add.reduceat(e1, batch.atom_off[:-1]), rtol=1e-12, atol=1e-9)
    assert np.allclose(A_, np.add.reduceat(np.abs(e1), batch.atom_off[:-1]), rtol=1e-12)


# ----------------------------------------------------------------------------- topology
def test_topology_validation():
    assert oracle.subtree_end([-1, 0, 1, 1, 0]) is not None
    assert list(oracle.subtree_end([-1, 0, 1, 1, 0])) == [5, 4, 3, 4, 5]
    assert oracle.subtree_end([-1, 0, 0, 1]) is None      # subtree(1) = {1, 3} not contiguous
    assert oracle.subtree_end([0, 0]) is None             # root must have parent -1
    assert oracle.subtree_end([-1, 2, 0]) is None         # parent after child
    rng = np.random.default_rng(8)
    b = synth.make_ligands(9, rng.integers(2, 60, size=50), rng.integers(0, 10, size=50))
    for l in range(b.L):
        par = b.ligand(l)["parent"]
        end = oracle.subtree_end(par)
        for v in range(len(par)):
            assert np.array_equal(_subtree(par, v), np.arange(v, end[v]))


# ----------------------------------------------------------------------------- rigid and torsion moves
def test_rigid_pose_preserves_distances_and_centres(cfg1):
    pocket, batch, prm = cfg1
    p0 = synth.DockParams(restarts=5, passes=0, seed=prm.seed)
    sub = batch.subset(range(20))
    out = oracle.dock(pocket, sub, p0, poses=True)
    for l in range(sub.L):
        lig = sub.ligand(l)
        X = _ligand_xyz(lig)
        N = len(X)
        D0 = np.linalg.norm(X[:, None] - X[None], axis=2)
        a0 = sub.atom_off[l]
        for r in range(5):
            Y = out["poses"][3 * 5 * a0 + 3 * N * r: 3 * 5 * a0 + 3 * N * (r + 1)].reshape(N, 3)
            D1 = np.linalg.norm(Y[:, None] - Y[None], axis=2)
            assert np.allclose(D0, D1, atol=1e-11)
            R, p, _ = oracle.restart_pose(pocket, p0, int(lig["uid"]), r)
            assert np.allclose(Y.mean(0), p, atol=1e-11)
            # the map is a proper rotation (no reflection): compare with scipy's fit
            rot, _ = Rotation.align_vectors(Y - Y.mean(0), X - X.mean(0))
            assert np.allclose(rot.as_matrix(), R, atol=1e-9)


def test_torsion_moves_keep_bonds_and_rigid_fragments(cfg1):
    pocket, batch, prm = cfg1
    sub = batch.subset([l for l in range(batch.L) if batch.n_rot()[l] >= 3][:15])
    p0 = synth.DockParams(restarts=3, passes=0, seed=prm.seed)
    p2 = synth.DockParams(restarts=3, passes=2, seed=prm.seed)
    before = oracle.dock(pocket, sub, p0, poses=True)["poses"]
    after = oracle.dock(pocket, sub, p2, poses=True)
    assert (after["choice"] != 0).any()
    for l in range(sub.L):
        lig = sub.ligand(l)
        par = lig["parent"].astype(np.int64)
        N = len(par)
        rot = set(int(b) for b in lig["rot_child"])
        # rigid fragments: components of the tree without the rotatable bonds
        frag = np.arange(N)
        for i in range(1, N):
            if i not in rot:
                frag[i] = frag[par[i]]
        a0 = sub.atom_off[l]
        for r in range(3):
            sl = slice(3 * 3 * a0 + 3 * N * r, 3 * 3 * a0 + 3 * N * (r + 1))
            X, Y = before[sl].reshape(N, 3), after["poses"][sl].reshape(N, 3)
            bl0 = np.linalg.norm(X[1:] - X[par[1:]], axis=1)
            bl1 = np.linalg.norm(Y[1:] - Y[par[1:]], axis=1)
            assert np.allclose(bl0, bl1, atol=1e-11)
            for f in np.unique(frag):
                m = np.where(frag == f)[0]
                # a fragment plus the atom it hangs from stays rigid
                if m[0] > 0:
                    m = np.append(m, par[m[0]])
                D0 = np.linalg.norm(X[m][:, None] - X[m][None], axis=2)
                D1 = np.linalg.norm(Y[m][:, None] - Y[m][None], axis=2)
                assert np.allclose(D0, D1, atol=1e-10)
            # atoms before the first rotatable child never move
            first = min(rot) if rot else N
            assert np.array_equal(X[:first + 1], Y[:first + 1])


def _initial_pose(pocket, prm, sub, r, N):
    p0 = synth.DockParams(restarts=prm.restarts, passes=0, seed=prm.seed, d_clash=prm.d_clash)
    X = oracle.dock(pocket, sub, p0, poses=True)["poses"]
    return X[3 * N * r: 3 * N * (r + 1)].reshape(N, 3)


def _brute_step(pocket, X, parent, b, d_clash, D):
    """Scores and admissibility of the 36 steps of bond (parent[b], b) by brute force."""
    a = parent[b]
    M = _subtree(parent, b); M = M[M != b]
    F = np.setdiff1d(np.arange(len(X)), _subtree(parent, b))
    s, ok = np.zeros(A), np.zeros(A, bool)
    for t in range(A):
        T = X[M] if t == 0 else _rot(X[a], X[b], 2 * np.pi * t / A, X[M])
        s[t] = _scipy_trilinear(pocket, pocket.phi_o, T).sum() if len(M) else 0.0
        d = np.linalg.norm(T[:, None] - X[F][None], axis=2) if len(M) and len(F) else np.zeros((0, 0))
        far = D[np.ix_(M, F)] >= 3 if d.size else np.zeros((0, 0), bool)
        ok[t] = (t == 0) or not (d[far] < d_clash).any()
    return s, ok, M


def test_single_bond_sweep_equals_brute_force(cfg1):
    pocket, batch, prm = cfg1
    ids = [l for l in range(batch.L) if batch.n_rot()[l] == 1][:25]
    assert len(ids) >= 10
    p1 = synth.DockParams(restarts=4, passes=1, seed=prm.seed, d_clash=prm.d_clash)
    n_nonzero = 0
    for l in ids:
        sub = _single(batch, l)
        lig = sub.ligand(0)
        par = lig["parent"].astype(np.int64)
        N, b = len(par), int(lig["rot_child"][0])
        D = _topo_dist(par)
        out = oracle.dock(pocket, sub, p1, trace=True)
        for r in range(p1.restarts):
            X = _initial_pose(pocket, p1, sub, r, N)
            s, ok, _ = _brute_step(pocket, X, par, b, p1.d_clash, D)
            assert np.allclose(out["trace_s"][A * r: A * (r + 1)], s, rtol=1e-12, atol=1e-12)
            best = max(np.where(ok)[0], key=lambda t: (s[t], -t))
            assert out["choice"][r] == best
            n_nonzero += best != 0
    assert n_nonzero > 0


def _total_overlap(pocket, X):
    return _scipy_trilinear(pocket, pocket.phi_o, X).sum()


def _clash_free(X, D, d_clash):
    d = np.linalg.norm(X[:, None] - X[None], axis=2)
    return not (d[D >= 3] < d_clash).any()


def _exhaustive(pocket, X, par, rot, D, d_clash):
    """Best clash-free total overlap over all 36^R torsion combinations."""
    best = -np.inf
    for combo in itertools.product(range(A), repeat=len(rot)):
        Y = X.copy()
        for b, t in zip(rot, combo):
            if t:
                M = _subtree(par, b); M = M[M != b]
                Y[M] = _rot(Y[par[b]], Y[b], 2 * np.pi * t / A, Y[M])
        if _clash_free(Y, D, d_clash):
            best = max(best, _total_overlap(pocket, Y))
    return best


@pytest.mark.slow
def test_greedy_bounded_by_exhaustive_search(cfg1):
    pocket, batch, prm = cfg1
    ids = [l for l in range(batch.L) if batch.n_rot()[l] == 2 and batch.n_atoms()[l] <= 18][:4]
    assert ids
    p = synth.DockParams(restarts=2, passes=2, seed=prm.seed, d_clash=prm.d_clash)
    for l in ids:
        sub = _single(batch, l)
        lig = sub.ligand(0)
        par = lig["parent"].astype(np.int64)
        N, rot = len(par), [int(b) for b in lig["rot_child"]]
        D = _topo_dist(par)
        out = oracle.dock(pocket, sub, p, poses=True)
        for r in range(p.restarts):
            X = _initial_pose(pocket, p, sub, r, N)
            Y = out["poses"][3 * N * r: 3 * N * (r + 1)].reshape(N, 3)
            g = _total_overlap(pocket, Y)
            assert _clash_free(Y, D, p.d_clash)
            assert g >= _total_overlap(pocket, X) - 1e-12       # greedy never loses overlap
            assert g <= _exhaustive(pocket, X, par, rot, D, p.d_clash) + 1e-9


def _star_ligand(rng):
    """Root with three arms root-a1-a2-a3(-a4); rotatable bond (a1, a2) on each
    arm, so the moving sets {a3, a4} are disjoint and far apart: the total
    overlap is a sum of one term per bond (separable)."""
    dirs = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], float) / np.sqrt(3)
    pos, par = [np.zeros(3)], [-1]
    for arm in range(3):
        d = dirs[arm]
        perp = np.cross(d, rng.normal(size=3)); perp /= np.linalg.norm(perp)
        prev = 0
        pts = [d * 1.5, d * 2.6 + perp * 1.0, d * 3.9 + perp * 0.3, d * 5.0 + perp * 1.3]
        for k, p in enumerate(pts):
            pos.append(p); par.append(prev); prev = len(pos) - 1
    pos = np.array(pos)
    # preorder already (arms appended depth first); rotatable children are the a2 atoms
    rot = [1 + 4 * arm + 1 for arm in range(3)]
    return pos, np.array(par, np.int16), rot


def test_greedy_equals_exhaustive_when_separable(cfg1):
    pocket, _, prm = cfg1
    rng = np.random.default_rng(10)
    checked = 0
    for trial in range(6):
        pos, par, rot = _star_ligand(rng)
        N = len(par)
        Rm = Rotation.random(random_state=trial).as_matrix()
        pos = pos @ Rm.T
        b = synth.LigandBatch(np.array([0, N], np.int32), pos[:, 0].astype(np.float32),
                              pos[:, 1].astype(np.float32), pos[:, 2].astype(np.float32),
                              np.zeros(N, np.float32), np.zeros(N, np.uint8), par,
                              np.array([0, 3], np.int32), np.array(rot, np.int16),
                              np.array([trial], np.uint64))
        p = synth.DockParams(restarts=3, passes=1, seed=prm.seed, d_clash=prm.d_clash)
        out = oracle.dock(pocket, b, p, poses=True)
        D = _topo_dist(par.astype(np.int64))
        for r in range(p.restarts):
            X = _initial_pose(pocket, p, b, r, N)
            Y = out["poses"][3 * N * r: 3 * N * (r + 1)].reshape(N, 3)
            # separable objective: best per bond independently
            tot = _total_overlap(pocket, X)
            for bb in rot:
                s, ok, M = _brute_step(pocket, X, par.astype(np.int64), bb, p.d_clash, D)
                assert ok.all()
                tot += s.max() - s[0]
            assert abs(_total_overlap(pocket, Y) - tot) < 1e-9
            checked += 1
    assert checked == 18


# ----------------------------------------------------------------------------- whole-method invariants
def test_docked_poses_are_clash_free_and_best_restart_is_min(cfg1):
    pocket, batch, prm = cfg1
    sub = batch.subset(range(60))
    out = oracle.dock(pocket, sub, prm, poses=True)
    S = prm.restarts
    for l in range(sub.L):
        lig = sub.ligand(l)
        par = lig["parent"].astype(np.int64)
        N = len(par)
        D = _topo_dist(par)
        a0 = sub.atom_off[l]
        E = out["restart_E"][l]
        assert out["best_r"][l] == int(np.argmin(E))           # argmin takes the first minimum
        assert out["best_E"][l] == E.min()
        for r in range(S):
            Y = out["poses"][3 * S * a0 + 3 * N * r: 3 * S * a0 + 3 * N * (r + 1)].reshape(N, 3)
            assert _clash_free(Y, D, prm.d_clash)
            e, _ = oracle.pose_energy(pocket, Y, lig["q"], lig["type"])
            assert e == E[r]
        assert np.array_equal(out["best_pose"][3 * a0: 3 * (a0 + N)],
                              out["poses"][3 * S * a0 + 3 * N * out["best_r"][l]:
                                           3 * S * a0 + 3 * N * (out["best_r"][l] + 1)])


def test_choice_maximises_admissible_overlap(cfg1):
    pocket, batch, prm = cfg1
    sub = batch.subset(range(80))
    out = oracle.dock(pocket, sub, prm, trace=True)
    s = out["trace_s"].reshape(-1, A)
    d2 = out["trace_d2"].reshape(-1, A)
    ch = out["choice"][: len(s)]
    ok = d2 >= np.float32(prm.d_clash) ** 2
    ok[:, 0] = True
    for t in range(len(s)):
        cand = np.where(ok[t])[0]
        best = cand[np.argmax(s[t, cand])]                         # first maximum = lowest step
        assert ch[t] == best
        assert s[t, ch[t]] >= s[t, 0]
    assert (ch != 0).mean() > 0.2 and (~ok).any()               # moves and clashes both occur


def test_replay_of_own_choices_is_identity(cfg1):
    pocket, batch, prm = cfg1
    sub = batch.subset(range(40))
    a = oracle.dock(pocket, sub, prm)
    b = oracle.dock(pocket, sub, prm, replay=a["choice"])
    assert np.array_equal(a["restart_E"], b["restart_E"])
    assert np.array_equal(a["own"], b["own"])


def test_results_independent_of_batch_mix_and_threads(cfg1):
    pocket, batch, prm = cfg1
    full = oracle.dock(pocket, batch.subset(range(32)), prm, nthreads=4)
    perm = np.random.default_rng(11).permutation(32)
    mixed = oracle.dock(pocket, batch.subset(perm), prm, nthreads=1)
    assert np.array_equal(full["best_E"][perm], mixed["best_E"])
    assert np.array_equal(full["best_r"][perm], mixed["best_r"])
    alone = oracle.dock(pocket, batch.subset([int(perm[3])]), prm)
    assert alone["best_E"][0] == full["best_E"][perm[3]]


def test_degenerate_ligands(cfg1):
    pocket, _, prm = cfg1
    one = synth.LigandBatch(np.array([0, 1], np.int32), np.array([1.0], np.float32), np.array([2.0], np.float32),
                            np.array([3.0], np.float32), np.array([0.1], np.float32), np.array([3], np.uint8),
                            np.array([-1], np.int16), np.array([0, 0], np.int32), np.zeros(0, np.int16),
                            np.array([77], np.uint64))
    out = oracle.dock(pocket, one, prm, poses=True)
    assert out["status"][0] == 0
    R, p, _ = oracle.restart_pose(pocket, prm, 77, int(out["best_r"][0]))
    assert np.allclose(out["best_pose"][:3], p)                 # single atom lands on its pocket point
    bad = synth.LigandBatch(np.array([0, 3], np.int32), np.zeros(3, np.float32), np.zeros(3, np.float32),
                            np.zeros(3, np.float32), np.zeros(3, np.float32), np.zeros(3, np.uint8),
                            np.array([-1, 0, 3], np.int16), np.array([0, 0], np.int32), np.zeros(0, np.int16),
                            np.array([1], np.uint64))
    assert oracle.dock(pocket, bad, prm)["status"][0] != 0


# ----------------------------------------------------------------------------- ranking (clustering + rescoring)
def _check_ranking(pocket, poses, E, G, order, leader, thr, K, best_r, best_E):
    S, N = poses.shape[0], poses.shape[1]
    # G is the total overlap of the final pose (scipy interpolation)
    for r in range(S):
        assert abs(G[r] - _scipy_trilinear(pocket, pocket.phi_o, poses[r]).sum()) < 1e-9 * max(1.0, abs(G[r]))
    geo = sorted(range(S), key=lambda r: (-G[r], r))
    rmsd = lambda a, b: np.sqrt(((poses[a] - poses[b]) ** 2).sum(1).mean())
    leaders = [r for r in geo if leader[r] == r]
    for i, a in enumerate(leaders):                       # leaders are mutually farther than thr
        for b in leaders[i + 1:]:
            assert rmsd(a, b) > thr
    pos = {r: i for i, r in enumerate(geo)}
    for r in range(S):
        if leader[r] != r:
            q = leader[r]
            assert leader[q] == q and pos[q] < pos[r] and rmsd(q, r) <= thr
            earlier = [l for l in leaders if pos[l] < pos[q]]
            assert all(rmsd(l, r) > thr for l in earlier)   # it joined the first leader within thr
        else:
            assert all(rmsd(l, r) > thr for l in leaders if pos[l] < pos[r])
    assert list(order) == leaders + [r for r in geo if leader[r] != r]
    k = S if K <= 0 or K > S else K
    top = list(order[:k])
    want = min(top, key=lambda r: (E[r], r))
    assert best_r == want and best_E == E[want]


def test_ranking_clusters_and_rescores(cfg1):
    pocket, batch, prm = cfg1
    sub = batch.subset(range(24))
    grouped = {}
    for thr, K in ((3.0, 5), (1.5, 3), (9.0, 16), (9.0, 4), (3.0, 0)):
        p = synth.DockParams(restarts=16, passes=2, seed=prm.seed, cluster_rmsd=thr, rescore_top=K)
        out = oracle.dock(pocket, sub, p, poses=True)
        n_clusters = []
        for l in range(sub.L):
            N = int(sub.n_atoms()[l])
            a0 = int(sub.atom_off[l])
            poses = out["poses"][3 * 16 * a0: 3 * 16 * (a0 + N)].reshape(16, N, 3)
            _check_ranking(pocket, poses, out["restart_E"][l], out["geo"][l], out["order"][l], out["leader"][l],
                           thr, K, int(out["best_r"][l]), out["best_E"][l])
            n_clusters.append(int((out["leader"][l] == np.arange(16)).sum()))
        grouped[thr] = np.mean(n_clusters)
    assert grouped[9.0] < 12 < grouped[3.0]          # the larger threshold actually groups poses


def test_ranking_limits():
    # threshold 0: every pose leads its own cluster -> pure geometric order;
    # a huge threshold: one cluster -> geometric order as well; K = all -> min E
    rng = np.random.default_rng(12)
    from paper_2110_11644_gb300 import synth as sy
    pocket = sy.config_pocket(1)
    poses = pocket.center + rng.normal(0, 4, size=(10, 7, 3))
    E = rng.normal(size=10)
    for thr in (0.0, 1e6):
        G, order, leader, br, be = oracle.rank_poses(pocket, poses, E, thr, 0)
        geo = sorted(range(10), key=lambda r: (-G[r], r))
        assert list(order) == geo
        assert br == int(np.argmin(E)) and be == E.min()
    G, order, leader, br, be = oracle.rank_poses(pocket, poses, E, 1e6, 0)
    assert (leader == geo[0]).all()
    # rescoring only the first K ranked poses
    G, order, leader, br, be = oracle.rank_poses(pocket, poses, E, 0.0, 3)
    assert br == min(order[:3], key=lambda r: (E[r], r))
