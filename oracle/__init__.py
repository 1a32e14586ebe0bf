"""FP64 CPU oracle of the dock-and-score hot path (ctypes wrapper of oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use it.  The library never imports it and it
imports nothing from the library: pockets and ligand batches are passed in as
plain objects with the attributes listed in ``_pocket_struct`` and ``dock``.

Every function follows oracle.c, whose header states the readings of the
paper's dock-and-score step (Sec. 3.1) that it implements.

Parity pins: every function here is pinned by a ``-m "not gpu"`` test in
tests/test_oracle_pins.py (Philox known-answer vectors, rotation-group
properties, exactness of trilinear interpolation on trilinear fields and
against scipy's map_coordinates, grid energies against direct pairwise sums
at nodes, torsion/rigid-move invariants, brute-force and exhaustive torsion
searches on small ligands), and the greedy walk across bonds and passes is
restated step by step with scipy in tests/test_oracle_walk.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile liboracle.so (gcc, FP64, OpenMP over ligands, no fused multiply-add
    contraction so x86 and Arm hosts round alike)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Pocket(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("h", ctypes.c_double), ("origin", ctypes.c_double * 3),
                ("phi_o", ctypes.c_void_p), ("phi_v", ctypes.c_void_p), ("phi_e", ctypes.c_void_p),
                ("n_pp", ctypes.c_int32), ("pp", ctypes.c_void_p), ("type_w", ctypes.c_double * 5),
                ("k_out", ctypes.c_double)]


class _Params(ctypes.Structure):
    _fields_ = [("restarts", ctypes.c_int32), ("passes", ctypes.c_int32), ("angle_steps", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("d_clash", ctypes.c_double), ("cluster_rmsd", ctypes.c_double),
                ("rescore_top", ctypes.c_int32), ("rigid_steps", ctypes.c_int32), ("rigid_shift", ctypes.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P, i32, d, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double, ctypes.c_uint64
            lib.or_philox4x32_10.argtypes = [P, P, P]
            lib.or_shoemake.argtypes = [d, d, d, P]
            lib.or_restart_pose.argtypes = [P, P, u64, i32, P, P, P]
            lib.or_trilinear.argtypes = [P, P, P]
            lib.or_trilinear.restype = d
            lib.or_rotate_about.argtypes = [P, P, d, d, P, P]
            lib.or_pose_energy.argtypes = [P, i32, P, P, P, P]
            lib.or_pose_energy.restype = d
            lib.or_topology.argtypes = [i32, P, P]
            lib.or_topology.restype = ctypes.c_int
            lib.or_dock_ligand.restype = ctypes.c_int
            lib.or_dock_batch.argtypes = [P, P, i32] + [P] * 10 + [P] * 11 + [P, P, P] + [P] * 4 + [i32]
            lib.or_rank_poses.argtypes = [P, i32, i32, P, P, d, i32, P, P, P, P, P]
            lib.or_dock_batch.restype = ctypes.c_int
            lib.or_score_poses.argtypes = [P, i32, P, P, P, P, P, P]
            lib.or_rigid_candidate.argtypes = [i32, P, i32, d, d, P]
            lib.or_rigid_candidate.restype = None
            lib.or_flatten_batch.argtypes = [i32, P, P, P, P, P, P, P, P, i32, i32, d] + [P] * 8 + [i32]
            lib.or_flatten_batch.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"], "arrays passed to the oracle must be C-contiguous"
    return a.ctypes.data_as(ctypes.c_void_p)


class OraclePocket:
    """Holds the ctypes pocket struct and keeps its arrays alive."""

    def __init__(self, pocket):
        self.src = pocket
        self.phi_o = np.ascontiguousarray(pocket.phi_o, np.float32).reshape(-1)
        self.phi_v = np.ascontiguousarray(pocket.phi_v, np.float32).reshape(-1)
        self.phi_e = np.ascontiguousarray(pocket.phi_e, np.float32).reshape(-1)
        self.pp = np.ascontiguousarray(pocket.pocket_points, np.int32).reshape(-1)
        s = _Pocket()
        s.n = int(pocket.n)
        s.h = float(np.float32(pocket.h))
        for c in range(3):
            s.origin[c] = float(np.float32(pocket.origin[c]))
        s.phi_o, s.phi_v, s.phi_e = _ptr(self.phi_o), _ptr(self.phi_v), _ptr(self.phi_e)
        s.n_pp = len(self.pp) // 3
        s.pp = _ptr(self.pp)
        for t in range(5):
            s.type_w[t] = float(np.float32(pocket.type_w[t]))
        s.k_out = float(np.float32(pocket.k_out))
        self.struct = s
        self.ref = ctypes.byref(s)


def _as_oracle_pocket(pocket):
    return pocket if isinstance(pocket, OraclePocket) else OraclePocket(pocket)


def _params(params):
    s = _Params()
    s.restarts, s.passes, s.angle_steps = int(params.restarts), int(params.passes), int(params.angle_steps)
    s.seed = int(params.seed)
    s.d_clash = float(np.float32(params.d_clash))
    s.cluster_rmsd = float(np.float32(getattr(params, "cluster_rmsd", 0.0)))
    s.rescore_top = int(getattr(params, "rescore_top", 0))
    s.rigid_steps = int(getattr(params, "rigid_steps", 0))
    s.rigid_shift = float(np.float32(getattr(params, "rigid_shift", 0.0)))
    return s


# ------------------------------------------------------------------ primitives
def philox4x32_10(ctr, key) -> np.ndarray:
    lib = _load()
    c = np.ascontiguousarray(ctr, np.uint32); k = np.ascontiguousarray(key, np.uint32)
    out = np.empty(4, np.uint32)
    lib.or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def shoemake(u0: float, u1: float, u2: float) -> np.ndarray:
    lib = _load()
    R = np.empty(9)
    lib.or_shoemake(u0, u1, u2, _ptr(R))
    return R.reshape(3, 3)


def restart_pose(pocket, params, uid: int, r: int):
    lib = _load()
    op = _as_oracle_pocket(pocket)
    pr = _params(params)
    R = np.empty(9); p = np.empty(3); idx = ctypes.c_int32()
    lib.or_restart_pose(op.ref, ctypes.byref(pr), uid, r, _ptr(R), _ptr(p), ctypes.byref(idx))
    return R.reshape(3, 3), p, idx.value


def trilinear(pocket, which: str, pts) -> np.ndarray:
    lib = _load()
    op = _as_oracle_pocket(pocket)
    grid = {"o": op.phi_o, "v": op.phi_v, "e": op.phi_e}[which]
    pts = np.ascontiguousarray(np.atleast_2d(pts), np.float64)
    return np.array([lib.or_trilinear(op.ref, _ptr(grid), _ptr(np.ascontiguousarray(p))) for p in pts])


def rotate_about(xa, xb, c: float, s: float, x) -> np.ndarray:
    lib = _load()
    xa = np.ascontiguousarray(xa, np.float64); xb = np.ascontiguousarray(xb, np.float64)
    x = np.ascontiguousarray(x, np.float64)
    out = np.empty(3)
    lib.or_rotate_about(_ptr(xa), _ptr(xb), c, s, _ptr(x), _ptr(out))
    return out


def rigid_candidate(xyz, cand: int, shift: float, angle: float) -> np.ndarray:
    """Candidate `cand` (0..12) of a rigid move applied to the atoms xyz[N][3]."""
    lib = _load()
    X = np.ascontiguousarray(xyz, np.float64)
    out = np.empty_like(X)
    lib.or_rigid_candidate(len(X), _ptr(X), int(cand), float(shift), float(angle), _ptr(out))
    return out


def pose_energy(pocket, xyz, q, type_):
    lib = _load()
    op = _as_oracle_pocket(pocket)
    xyz = np.ascontiguousarray(xyz, np.float64).reshape(-1)
    q = np.ascontiguousarray(q, np.float32); t = np.ascontiguousarray(type_, np.uint8)
    eabs = ctypes.c_double()
    E = lib.or_pose_energy(op.ref, len(q), _ptr(xyz), _ptr(q), _ptr(t), ctypes.byref(eabs))
    return E, eabs.value


def subtree_end(parent) -> np.ndarray | None:
    lib = _load()
    par = np.ascontiguousarray(parent, np.int16)
    end = np.empty(len(par), np.int32)
    rc = lib.or_topology(len(par), _ptr(par), _ptr(end))
    return end if rc == 0 else None


def score_poses(pocket, atom_off, xyz, q, type_):
    lib = _load()
    op = _as_oracle_pocket(pocket)
    atom_off = np.ascontiguousarray(atom_off, np.int32)
    L = len(atom_off) - 1
    xyz = np.ascontiguousarray(xyz, np.float64).reshape(-1)
    q = np.ascontiguousarray(q, np.float32); t = np.ascontiguousarray(type_, np.uint8)
    E = np.empty(L); A = np.empty(L)
    lib.or_score_poses(op.ref, L, _ptr(atom_off), _ptr(xyz), _ptr(q), _ptr(t), _ptr(E), _ptr(A))
    return E, A


# ------------------------------------------------------------------ docking
def dock(pocket, batch, params, *, replay=None, replay_rigid=None, trace=False, poses=False, nthreads=None) -> dict:
    """Dock every ligand of a CSR batch (attributes atom_off, x, y, z, q, type,
    parent, rot_off, rot_child, uid).  Returns a dict of numpy arrays:
      best_E[L], best_r[L], status[L], restart_E[L,S], restart_Eabs[L,S],
      choice / own (flat, S*P*rot_off[l] per ligand), best_pose (flat xyz, 3*atom_off),
      and with trace=True trace_s / trace_d2 (flat, A*S*P*rot_off[l]),
      with poses=True poses (flat, 3*S*atom_off[l]); with rigid moves
      choice_rigid / own_rigid (flat, S*P*rigid_steps*l) and with trace=True
      trace_G (13 per rigid decision)."""
    lib = _load()
    op = _as_oracle_pocket(pocket)
    pr = _params(params)
    S, PS, A = pr.restarts, pr.passes, pr.angle_steps
    aoff = np.ascontiguousarray(batch.atom_off, np.int32)
    roff = np.ascontiguousarray(batch.rot_off, np.int32)
    L = len(aoff) - 1
    natoms, nrot = int(aoff[-1]), int(roff[-1])
    arr = {k: np.ascontiguousarray(getattr(batch, k)) for k in ("x", "y", "z", "q")}
    t = np.ascontiguousarray(batch.type, np.uint8)
    par = np.ascontiguousarray(batch.parent, np.int16)
    rc = np.ascontiguousarray(batch.rot_child, np.int16)
    uid = np.ascontiguousarray(batch.uid, np.uint64)
    ndec = S * PS * nrot
    out = dict(restart_E=np.full(L * S, np.nan), restart_Eabs=np.full(L * S, np.nan),
               choice=np.zeros(max(ndec, 1), np.uint8), own=np.zeros(max(ndec, 1), np.uint8),
               best_pose=np.zeros(max(3 * natoms, 1)), best_r=np.full(L, -1, np.int32),
               best_E=np.full(L, np.nan), status=np.zeros(L, np.int32))
    if trace:
        out["trace_s"] = np.zeros(max(ndec * A, 1)); out["trace_d2"] = np.zeros(max(ndec * A, 1))
    if poses:
        out["poses"] = np.zeros(max(3 * S * natoms, 1))
    ranking = pr.cluster_rmsd > 0 or 0 < pr.rescore_top < S
    if ranking:
        out["rank"] = np.zeros(max(2 * S * L, 1), np.int32)
        out["geo"] = np.zeros(max(S * L, 1))
    nrig = S * PS * pr.rigid_steps * L
    if pr.rigid_steps > 0:
        out["choice_rigid"] = np.zeros(max(nrig, 1), np.uint8)
        out["own_rigid"] = np.zeros(max(nrig, 1), np.uint8)
        if trace:
            out["trace_G"] = np.zeros(max(13 * nrig, 1))
    rep_rigid = None
    if replay_rigid is not None:
        rep_rigid = np.ascontiguousarray(replay_rigid, np.uint8)
        assert rep_rigid.size >= nrig
    rep = None
    if replay is not None:
        rep = np.ascontiguousarray(replay, np.uint8)
        assert rep.size >= ndec
    if nthreads is None:
        nthreads = len(os.sched_getaffinity(0))
    lib.or_dock_batch(op.ref, ctypes.byref(pr), L, _ptr(aoff), _ptr(arr["x"]), _ptr(arr["y"]), _ptr(arr["z"]),
                      _ptr(arr["q"]), _ptr(t), _ptr(par), _ptr(roff), _ptr(rc), _ptr(uid), _ptr(rep),
                      _ptr(out["restart_E"]), _ptr(out["restart_Eabs"]), _ptr(out["choice"]), _ptr(out["own"]),
                      _ptr(out.get("trace_s")), _ptr(out.get("trace_d2")), _ptr(out.get("poses")),
                      _ptr(out["best_pose"]), _ptr(out["best_r"]), _ptr(out["best_E"]), _ptr(out["status"]),
                      _ptr(out.get("rank")), _ptr(out.get("geo")), _ptr(rep_rigid), _ptr(out.get("choice_rigid")),
                      _ptr(out.get("own_rigid")), _ptr(out.get("trace_G")), int(nthreads))
    out["restart_E"] = out["restart_E"].reshape(L, S)
    out["restart_Eabs"] = out["restart_Eabs"].reshape(L, S)
    if ranking:
        rk = out.pop("rank")[: 2 * S * L].reshape(L, 2, S)
        out["order"], out["leader"] = rk[:, 0, :].copy(), rk[:, 1, :].copy()
        out["geo"] = out["geo"][: S * L].reshape(L, S)
    return out


def rank_poses(pocket, poses, E, thr, K):
    """Ranking of one ligand's S final poses (poses[S][N][3], E[S]): returns
    (G, order, leader, best_r, best_E)."""
    lib = _load()
    op = _as_oracle_pocket(pocket)
    poses = np.ascontiguousarray(poses, np.float64)
    S, N = poses.shape[0], poses.shape[1]
    E = np.ascontiguousarray(E, np.float64)
    G = np.empty(S); order = np.empty(S, np.int32); leader = np.empty(S, np.int32)
    br = ctypes.c_int32(); be = ctypes.c_double()
    lib.or_rank_poses(op.ref, S, N, _ptr(poses), _ptr(E), float(thr), int(K), _ptr(G), _ptr(order), _ptr(leader),
                      ctypes.byref(br), ctypes.byref(be))
    return G, order, leader, br.value, be.value


# ------------------------------------------------------------------ flattening
def flatten(batch, passes: int, d_clash: float = 2.0, *, angle_steps: int = 36, replay=None, trace=False,
            nthreads=None) -> dict:
    """Flatten every ligand of a CSR batch (Sec. 3.1, step 1): returns xyz
    (flat, 3*atom_off), D[L] (sum of all pairwise distances of the result),
    choice / own (flat, passes*rot_off[l] per ligand), status[L], and with
    trace=True trace_D / trace_d2 (flat, A*passes*rot_off[l])."""
    lib = _load()
    aoff = np.ascontiguousarray(batch.atom_off, np.int32)
    roff = np.ascontiguousarray(batch.rot_off, np.int32)
    L = len(aoff) - 1
    natoms, nrot = int(aoff[-1]), int(roff[-1])
    arr = {k: np.ascontiguousarray(getattr(batch, k), np.float32) for k in ("x", "y", "z")}
    t = np.ascontiguousarray(batch.type, np.uint8)
    par = np.ascontiguousarray(batch.parent, np.int16)
    rc = np.ascontiguousarray(batch.rot_child, np.int16)
    ndec = passes * nrot
    out = dict(xyz=np.zeros(max(3 * natoms, 1)), D=np.full(L, np.nan), choice=np.zeros(max(ndec, 1), np.uint8),
               own=np.zeros(max(ndec, 1), np.uint8), status=np.zeros(L, np.int32))
    if trace:
        out["trace_D"] = np.zeros(max(ndec * angle_steps, 1))
        out["trace_d2"] = np.zeros(max(ndec * angle_steps, 1))
    rep = None
    if replay is not None:
        rep = np.ascontiguousarray(replay, np.uint8)
        assert rep.size >= ndec
    if nthreads is None:
        nthreads = len(os.sched_getaffinity(0))
    lib.or_flatten_batch(L, _ptr(aoff), _ptr(arr["x"]), _ptr(arr["y"]), _ptr(arr["z"]), _ptr(t), _ptr(par),
                         _ptr(roff), _ptr(rc), int(passes), int(angle_steps), float(d_clash), _ptr(rep),
                         _ptr(out["xyz"]), _ptr(out["choice"]), _ptr(out["own"]), _ptr(out.get("trace_D")),
                         _ptr(out.get("trace_d2")), _ptr(out["D"]), _ptr(out["status"]), int(nthreads))
    out["xyz"] = out["xyz"][:3 * natoms]
    out["choice"] = out["choice"][:ndec]
    out["own"] = out["own"][:ndec]
    return out
