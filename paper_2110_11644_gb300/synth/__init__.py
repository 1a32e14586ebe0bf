"""Seeded synthetic docking workloads (inputs only).

This module is the one piece of code that both the FP64 oracle (``oracle/``)
and the CUDA path are fed from.  It builds ligand batches and pocket grids and
holds none of the docking arithmetic: no pose sampling, torsion sweep,
interpolation or scoring.  Random numbers that the docking method itself draws
(restart poses) are NOT made here: each side implements Philox4x32-10 itself.

The paper's inputs (MEDIATE chemical libraries, SARS-CoV-2 binding sites of
Table 1) are not available; these synthetic workloads stand in for them with
the shape cues the paper gives: ligands of tens of atoms with up to tens of
torsional bonds (Sec. 3.1), a rigid binding site read once per run (Sec. 3.2),
ligands described by atom positions, types and bonds (Sec. 4.1).

Workloads (the ``config`` function):
  1  tiny     : sphere cavity r=8 A, 2,000 shell atoms in r in [8,16] A, 48^3 grid,
               256 ligands of U{12..30} atoms, U{0..4} rotatable bonds, 16 restarts, 2 passes.
  2  plain    : ellipsoid cavity (6,8,12) A, 4,000 atoms in an 8 A shell, 64^3 grid,
               ligands of U{15..60} atoms, U{0..12} rotatable bonds, 30 restarts, 3 passes.
  3  batched  : the workload-2 pocket; atoms clip(round(lognormal(ln 28, 0.45)), 10, 100),
               rotatable bonds clip(round(0.2 N + N(0, 1.5)), 0, 20), 30 restarts, 3 passes.
  4  multi    : 15 pockets, cavity radii U(5,14) A, 2,000-6,000 shell atoms, 40^3..96^3
               grids, workload-2 ligands.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB_PATH = os.path.join(_HERE, "libsynth.so")
_lib = None
_lock = threading.Lock()

# Grid-potential constants (input recipe; see the module docstring of synth.c).
H_DEFAULT = 0.375           # grid spacing, A
POCKET_CLEARANCE = 3.0      # pocket points keep this distance from protein atoms, A
OVERLAP_SIGMA = 1.0         # Gaussian width of the pocket-overlap field, A
OVERLAP_CUT = 3.0           # truncation radius of each Gaussian, A
LJ_EPS, LJ_R0, LJ_CUT, LJ_CAP, LJ_RMIN = 0.15, 3.6, 8.0, 10.0, 0.5
COULOMB_K, COULOMB_CUT, COULOMB_RMIN = 332.0636, 12.0, 1.0
TYPE_WEIGHTS = (1.00, 0.90, 0.85, 1.20, 1.10)   # C N O S Cl multipliers of the vdW grid
K_OUT = 10.0                # out-of-box penalty slope, (kcal/mol)/A
LIGAND_MIN_SEP = 2.2        # generator's minimum separation of non-bonded atoms, A
LIGAND_OFFSET = 30.0        # ligands are translated by U(-30, 30) A per axis


def build(force: bool = False) -> str:
    """Compile libsynth.so next to its source (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            d, i, u64 = ctypes.c_double, ctypes.c_int, ctypes.c_uint64
            lib.synth_ligands.argtypes = [i, P, P, P, d, d, P, P, P, P, P, P, P, P]
            lib.synth_ligands.restype = i
            lib.synth_pocket_points.argtypes = [i, d, P, i, P, P, P, d, P]
            lib.synth_pocket_points.restype = i
            lib.synth_overlap_grid.argtypes = [i, d, i, P, d, d, P]
            lib.synth_direct_potentials.argtypes = [i, P, i, P, P] + [d] * 8 + [P, P]
            lib.synth_potential_grids.argtypes = [i, d, P, i, P, P] + [d] * 8 + [P, P]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------- pockets
@dataclass
class Pocket:
    n: int
    h: float
    origin: np.ndarray          # float64[3]; world position of node (0,0,0); exact in float32
    center: np.ndarray          # float64[3]; cavity centre
    phi_o: np.ndarray           # float32[n,n,n] indexed [k,j,i] (x fastest in memory)
    phi_v: np.ndarray
    phi_e: np.ndarray
    pocket_points: np.ndarray   # int32[n_pp,3] node indices (i,j,k)
    atoms_xyz: np.ndarray       # float64[na,3] protein atoms (for direct-sum checks)
    atoms_q: np.ndarray         # float64[na]
    type_w: np.ndarray = field(default_factory=lambda: np.array(TYPE_WEIGHTS, np.float32))
    k_out: float = K_OUT

    def node_xyz(self, ijk: np.ndarray) -> np.ndarray:
        return self.origin[None, :] + self.h * np.asarray(ijk, np.float64)


def direct_potentials(pocket: Pocket, pts: np.ndarray):
    """vdW-like and electrostatic potentials at points, summed directly over the
    pocket's protein atoms with the same formulas the grids were built with."""
    lib = _load()
    pts = np.ascontiguousarray(pts, np.float64)
    v = np.empty(len(pts)); e = np.empty(len(pts))
    xyz = np.ascontiguousarray(pocket.atoms_xyz); q = np.ascontiguousarray(pocket.atoms_q)
    lib.synth_direct_potentials(len(pts), _p(pts), len(xyz), _p(xyz), _p(q), LJ_EPS, LJ_R0, LJ_CUT,
                                LJ_CAP, LJ_RMIN, COULOMB_K, COULOMB_CUT, COULOMB_RMIN, _p(v), _p(e))
    return v, e


def _shell_atoms(rng: np.random.Generator, n_atoms: int, radii, thickness: float):
    """Protein atoms uniform in volume in a shell of the given thickness outside
    the cavity ellipsoid, measured along each radial direction."""
    d = rng.normal(size=(n_atoms, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r_e = 1.0 / np.sqrt(((d / np.asarray(radii, np.float64)) ** 2).sum(1))
    u = rng.random(n_atoms)
    r = np.cbrt(r_e ** 3 + u * ((r_e + thickness) ** 3 - r_e ** 3))
    return d * r[:, None]


def make_pocket(seed: int, *, radii, n_atoms: int, thickness: float, n: int, h: float = H_DEFAULT,
                center=None) -> Pocket:
    """Synthetic rigid binding site: protein atoms in a shell around a cavity
    ellipsoid (a sphere when the three radii agree), the pocket points that fill
    the cavity on the grid, and three FP32 grids (overlap, vdW-like, electrostatic)."""
    lib = _load()
    rng = np.random.default_rng(seed)
    if center is None:
        center = rng.integers(-80, 81, size=3) / 8.0     # dyadic: origin exact in float32
    center = np.asarray(center, np.float64)
    half = h * (n - 1) / 2.0
    origin = center - half
    assert np.all(origin.astype(np.float32).astype(np.float64) == origin)
    xyz = center[None, :] + _shell_atoms(rng, n_atoms, radii, thickness)
    xyz = np.ascontiguousarray(xyz)
    q = rng.normal(0.0, 0.2, size=n_atoms)
    q -= q.mean()
    q = np.ascontiguousarray(q)
    org = np.ascontiguousarray(origin)
    cav_c = np.ascontiguousarray(center)
    cav_r = np.ascontiguousarray(np.asarray(radii, np.float64))
    pp = np.empty((n * n * n, 3), np.int32)
    npp = lib.synth_pocket_points(n, h, _p(org), n_atoms, _p(xyz), _p(cav_c), _p(cav_r),
                                  POCKET_CLEARANCE, _p(pp))
    pp = np.ascontiguousarray(pp[:npp])
    phi_o = np.empty(n ** 3); phi_v = np.empty(n ** 3); phi_e = np.empty(n ** 3)
    lib.synth_overlap_grid(n, h, npp, _p(pp), OVERLAP_SIGMA, OVERLAP_CUT, _p(phi_o))
    lib.synth_potential_grids(n, h, _p(org), n_atoms, _p(xyz), _p(q), LJ_EPS, LJ_R0, LJ_CUT, LJ_CAP,
                              LJ_RMIN, COULOMB_K, COULOMB_CUT, COULOMB_RMIN, _p(phi_v), _p(phi_e))
    f32 = lambda a: np.ascontiguousarray(a.astype(np.float32).reshape(n, n, n))
    return Pocket(n=n, h=h, origin=origin, center=center, phi_o=f32(phi_o), phi_v=f32(phi_v),
                  phi_e=f32(phi_e), pocket_points=pp, atoms_xyz=xyz, atoms_q=q)


# --------------------------------------------------------------------------- ligands
@dataclass
class LigandBatch:
    """Ligands in CSR structure-of-arrays layout.

    Atoms of ligand l are atom_off[l] .. atom_off[l+1]-1, in depth-first preorder
    (parent[i] < i, parent[0] = -1, every subtree a contiguous index range; parent
    indices are local to the ligand).  Rotatable bond k of ligand l is identified
    by its child atom rot_child[rot_off[l] + k] (ascending, local index); the bond
    is (parent[child], child).  Types 0..4 = C, N, O, S, Cl.
    """
    atom_off: np.ndarray   # int32[L+1]
    x: np.ndarray          # float32[A]
    y: np.ndarray
    z: np.ndarray
    q: np.ndarray
    type: np.ndarray       # uint8[A]
    parent: np.ndarray     # int16[A]
    rot_off: np.ndarray    # int32[L+1]
    rot_child: np.ndarray  # int16[Rtot]
    uid: np.ndarray        # uint64[L]

    @property
    def L(self) -> int:
        return len(self.atom_off) - 1

    def n_atoms(self) -> np.ndarray:
        return np.diff(self.atom_off)

    def n_rot(self) -> np.ndarray:
        return np.diff(self.rot_off)

    def ligand(self, l: int) -> dict:
        a0, a1 = int(self.atom_off[l]), int(self.atom_off[l + 1])
        r0, r1 = int(self.rot_off[l]), int(self.rot_off[l + 1])
        return dict(x=self.x[a0:a1], y=self.y[a0:a1], z=self.z[a0:a1], q=self.q[a0:a1],
                    type=self.type[a0:a1], parent=self.parent[a0:a1],
                    rot_child=self.rot_child[r0:r1], uid=int(self.uid[l]))

    def subset(self, idx) -> "LigandBatch":
        idx = np.asarray(idx, np.int64)
        na, nr = self.n_atoms()[idx], self.n_rot()[idx]
        aoff = np.zeros(len(idx) + 1, np.int32); aoff[1:] = np.cumsum(na)
        roff = np.zeros(len(idx) + 1, np.int32); roff[1:] = np.cumsum(nr)
        asel = np.concatenate([np.arange(self.atom_off[l], self.atom_off[l + 1]) for l in idx]) \
            if len(idx) else np.zeros(0, np.int64)
        rsel = np.concatenate([np.arange(self.rot_off[l], self.rot_off[l + 1]) for l in idx]) \
            if len(idx) else np.zeros(0, np.int64)
        asel = asel.astype(np.int64); rsel = rsel.astype(np.int64)
        return LigandBatch(aoff, self.x[asel].copy(), self.y[asel].copy(), self.z[asel].copy(),
                           self.q[asel].copy(), self.type[asel].copy(), self.parent[asel].copy(),
                           roff, self.rot_child[rsel].copy(), self.uid[idx].copy())

    @staticmethod
    def concat(batches) -> "LigandBatch":
        batches = list(batches)
        na = np.concatenate([b.n_atoms() for b in batches])
        nr = np.concatenate([b.n_rot() for b in batches])
        aoff = np.zeros(len(na) + 1, np.int32); aoff[1:] = np.cumsum(na)
        roff = np.zeros(len(nr) + 1, np.int32); roff[1:] = np.cumsum(nr)
        cat = lambda f: np.concatenate([getattr(b, f) for b in batches])
        return LigandBatch(aoff, cat("x"), cat("y"), cat("z"), cat("q"), cat("type"), cat("parent"),
                           roff, cat("rot_child"), cat("uid"))


def make_ligands(seed: int, n_atoms: np.ndarray, r_target: np.ndarray, uid_base: int = 0,
                 offset: float = LIGAND_OFFSET) -> LigandBatch:
    """Acyclic heavy-atom trees of the given sizes (see synth.c for the recipe)."""
    lib = _load()
    n_atoms = np.ascontiguousarray(n_atoms, np.int32)
    r_target = np.ascontiguousarray(r_target, np.int32)
    L = len(n_atoms)
    assert np.all(n_atoms >= 1) and np.all(n_atoms <= 256)
    seeds = np.random.default_rng(seed).integers(0, 2 ** 63, size=L, dtype=np.uint64)
    seeds = np.ascontiguousarray(seeds)
    aoff = np.zeros(L + 1, np.int32); aoff[1:] = np.cumsum(n_atoms)
    A = int(aoff[-1])
    x = np.empty(A, np.float32); y = np.empty(A, np.float32); z = np.empty(A, np.float32)
    q = np.empty(A, np.float32); t = np.empty(A, np.uint8); par = np.empty(A, np.int16)
    rtmp = np.empty(max(A, 1), np.int16); rout = np.empty(L, np.int32)
    bad = lib.synth_ligands(L, _p(seeds), _p(r_target), _p(aoff), offset, LIGAND_MIN_SEP, _p(x), _p(y),
                            _p(z), _p(q), _p(t), _p(par), _p(rtmp), _p(rout))
    if bad:
        raise RuntimeError(f"ligand generator failed on {bad} ligands")
    roff = np.zeros(L + 1, np.int32); roff[1:] = np.cumsum(rout)
    if L:
        starts = np.repeat(aoff[:-1], rout)
        within = np.arange(int(roff[-1])) - np.repeat(roff[:-1], rout)
        rot = rtmp[(starts + within).astype(np.int64)].copy()
    else:
        rot = np.zeros(0, np.int16)
    uid = np.arange(L, dtype=np.uint64) + np.uint64(uid_base)
    return LigandBatch(aoff, x, y, z, q, t, par, roff, rot.astype(np.int16), uid)


# --------------------------------------------------------------------------- workloads
@dataclass
class DockParams:
    restarts: int
    passes: int
    angle_steps: int = 36
    seed: int = 0x2110116440000000
    d_clash: float = 2.0
    cluster_rmsd: float = 0.0   # 0: no clustering
    rescore_top: int = 0        # 0: rescore every pose
    rigid_steps: int = 0        # rigid greedy moves after each torsion pass (0: none)
    rigid_shift: float = 0.375  # translation step of a rigid move (A)


CONFIG_SEEDS = {1: 0, 2: 2, 3: 3, 4: 4, 5: 5}
_pocket_cache: dict = {}


def _seeds(cfg: int, k: int):
    ss = np.random.SeedSequence(CONFIG_SEEDS[cfg]).spawn(k)
    return [int(s.generate_state(1, np.uint64)[0]) for s in ss]


def config_pocket(cfg: int, which: int = 0) -> Pocket:
    """The pocket of a workload (cached per process)."""
    key = (cfg, which)
    if key in _pocket_cache:
        return _pocket_cache[key]
    if cfg == 1:
        s = _seeds(1, 3)[0]
        p = make_pocket(s, radii=(8.0, 8.0, 8.0), n_atoms=2000, thickness=8.0, n=48)
    elif cfg in (2, 3):
        s = _seeds(2, 3)[0]
        p = make_pocket(s, radii=(6.0, 8.0, 12.0), n_atoms=4000, thickness=8.0, n=64)
    elif cfg in (4, 5):
        specs = multi_pocket_specs()
        sp = specs[which]
        p = make_pocket(sp["seed"], radii=sp["radii"], n_atoms=sp["n_atoms"], thickness=8.0, n=sp["n"])
    else:
        raise ValueError(cfg)
    _pocket_cache[key] = p
    return p


def multi_pocket_specs():
    """15 pockets: cavity radii U(5,14) A, 2,000-6,000 shell atoms, grid size
    n = clamp(8*ceil((2*max_radius + 6)/(8h)), 40, 96), pocket 0 forced to 40^3 and
    pocket 14 to 96^3 so the set spans the stated range."""
    rng = np.random.default_rng(_seeds(4, 3)[0])
    specs = []
    for p in range(15):
        radii = tuple(float(v) for v in rng.uniform(5.0, 14.0, size=3))
        na = int(rng.integers(2000, 6001))
        n = int(np.clip(8 * np.ceil((2 * max(radii) + 6) / (8 * H_DEFAULT)), 40, 96))
        if p == 0:
            n = 40
        if p == 14:
            n = 96
        specs.append(dict(seed=int(rng.integers(0, 2 ** 62)), radii=radii, n_atoms=na, n=n))
    return specs


def config_ligands(cfg: int, L: int | None = None, uid_base: int = 0) -> LigandBatch:
    """The ligands of a workload.  The first L ligands of a workload are the same
    whatever L is asked for (sizes and per-ligand seeds are drawn in order)."""
    if cfg == 1:
        L = 256 if L is None else L
        s_sz, s_lig = _seeds(1, 3)[1:]
        rng = np.random.default_rng(s_sz)
        n = rng.integers(12, 31, size=max(L, 256))[:L]
        r = rng.integers(0, 5, size=max(L, 256))[:L]
    elif cfg in (2, 4, 5):
        L = 100_000 if L is None else L
        s_sz, s_lig = _seeds(2, 3)[1:]
        n, r = _sizes_uniform(s_sz, L, 15, 60, 0, 12)
    elif cfg == 3:
        L = 1_000_000 if L is None else L
        s_sz, s_lig = _seeds(3, 3)[1:]
        n, r = _sizes_lognormal(s_sz, L)
    else:
        raise ValueError(cfg)
    return make_ligands(s_lig, n, r, uid_base=uid_base)


def _sizes_uniform(seed, L, n_lo, n_hi, r_lo, r_hi, chunk=1 << 16):
    # drawn in fixed chunks so that any prefix of the workload is stable
    rng = np.random.default_rng(seed)
    ns, rs, got = [], [], 0
    while got < L:
        ns.append(rng.integers(n_lo, n_hi + 1, size=chunk))
        rs.append(rng.integers(r_lo, r_hi + 1, size=chunk))
        got += chunk
    return np.concatenate(ns)[:L], np.concatenate(rs)[:L]


def _sizes_lognormal(seed, L, chunk=1 << 16):
    rng = np.random.default_rng(seed)
    ns, rs, got = [], [], 0
    while got < L:
        n = np.clip(np.round(rng.lognormal(np.log(28.0), 0.45, size=chunk)), 10, 100).astype(np.int64)
        r = np.clip(np.round(0.2 * n + rng.normal(0.0, 1.5, size=chunk)), 0, 20).astype(np.int64)
        ns.append(n); rs.append(r); got += chunk
    return np.concatenate(ns)[:L], np.concatenate(rs)[:L]


def config_params(cfg: int) -> DockParams:
    if cfg == 1:
        return DockParams(restarts=16, passes=2)
    return DockParams(restarts=30, passes=3)
