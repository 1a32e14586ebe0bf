"""Sharding a ligand library over GPUs (host logic).

Every (ligand, pocket) evaluation is independent (paper Sec. 3.2: a ligand's
description is all a dock needs), so a screening run splits the library over
ranks and needs no exchange while docking; only the final ranking is gathered.
The paper splits its input file into equal-size slabs per MPI rank and notes
that this static split cannot balance ligands of very different cost
(Sec. 3.2-3.3); here shards are balanced by the estimated docking cost instead.

Cost model (also the bench's algorithmic FLOP count per ligand), the
rotate-then-interpolate accounting of the method with an FMA counted as 2:
  restarts * (21 N + 40 + passes * sum_k (36 m_k (21 + 30) + 8 Pi_k) + 64 N)
with N the atoms, m_k the atoms torsional bond k moves and Pi_k the clash
pairs of bond k (moving atom, atom outside the child's subtree, three or more
bonds apart).  Per step and moving atom: 21 to rotate it about the bond,
30 for a trilinear lookup; per restart 21 N + 40 for the rigid pose and 64 per
atom for the final score.  A clash pair costs 8 and is credited j* times per
decision, j* = 1 + the number of steps ranked before the chosen one by overlap
score: a method must clash-check those steps (each was rejected) and the
chosen one, and no others.  ligand_flops takes j* = 1, a lower bound;
ligand_flops_ranked takes each decision's j* from the docking run's own
decisions (lg_dock_result.decision_rank).  ligand_flops_needed credits only
the decisions the run did not skip by its exact convergence stops (the work
the result needed); ligand_flops_circle counts the lower figure of the circle
form the kernels evaluate.
"""
from __future__ import annotations

import heapq

import numpy as np

C_ROT, C_TRI, C_PAIR, C_FIN, C_POSE_ATOM, C_RESTART = 21, 30, 8, 64, 21, 40
# circle form: 12 (point on the circle) + 3 (cell fractions) + 14 (polynomial)
# + 1 (sum) per moving atom and step; 30 per moving atom and decision for its
# circle and the move; 21 + 44 per atom and restart
C_LOOKUP_CIRCLE, C_BOND_CIRCLE, C_FINAL_CIRCLE = 30, 30, 44
# decision_rank: j* in the low 7 bits; bit 7 marks a decision skipped by an
# exact convergence stop (its rank repeats the bond's previous one)
RANK_MASK, RANK_SKIPPED = 0x7F, 0x80


def _bond_counts(batch):
    """Per torsional bond (CSR order): atoms moved m_k, clash pairs Pi_k, and
    the ligand index of the bond."""
    aoff = batch.atom_off.astype(np.int64)
    A = int(aoff[-1])
    L = len(aoff) - 1
    lig = np.repeat(np.arange(L), np.diff(aoff))
    par = batch.parent.astype(np.int64)
    gpar = np.where(par >= 0, par + aoff[lig], -1)
    depth = np.zeros(A, np.int64)
    nonroot = gpar >= 0
    for _ in range(int(np.diff(aoff).max(initial=1))):
        nd = np.where(nonroot, depth[np.maximum(gpar, 0)] + 1, 0)
        if np.array_equal(nd, depth):
            break
        depth = nd
    size = np.ones(A, np.int64)
    for d in range(int(depth.max(initial=0)), 0, -1):
        idx = np.where(depth == d)[0]
        np.add.at(size, gpar[idx], size[idx])
    nchild = np.zeros(A, np.int64)
    np.add.at(nchild, gpar[nonroot], 1)
    roff = batch.rot_off.astype(np.int64)
    rl = np.repeat(np.arange(L), np.diff(roff))
    child = batch.rot_child.astype(np.int64) + aoff[rl]
    m = size[child] - 1
    N = np.diff(aoff)[rl]
    # moving atom i, fixed atom j: the path runs i .. child - parent .. j, so
    # only (child of the bond's child, the bond's parent) is closer than 3 bonds
    pairs = m * (N - m - 1) - nchild[child]
    return m, pairs, rl, L


def moving_atoms_per_ligand(batch) -> np.ndarray:
    """Sum over each ligand's torsional bonds of the atoms the bond moves
    (subtree size of the bond's child minus one)."""
    m, _, rl, L = _bond_counts(batch)
    out = np.zeros(L, np.int64)
    np.add.at(out, rl, m)
    return out


def clash_pairs_per_ligand(batch) -> np.ndarray:
    """Sum over each ligand's torsional bonds of the clash pairs Pi_k."""
    _, pairs, rl, L = _bond_counts(batch)
    out = np.zeros(L, np.int64)
    np.add.at(out, rl, pairs)
    return out


def ligand_flops(batch, restarts: int, passes: int, rigid_steps: int = 0) -> np.ndarray:
    """Algorithmic FLOPs of docking each ligand (see the module docstring);
    rigid refinement adds, per pass and rigid move, 13 candidates of N rotated
    atoms and lookups."""
    N = np.diff(batch.atom_off).astype(np.float64)
    m, pairs, rl, L = _bond_counts(batch)
    per_bond = 36.0 * m * (C_ROT + C_TRI) + C_PAIR * pairs.astype(np.float64)
    sweep = np.zeros(L)
    np.add.at(sweep, rl, per_bond)
    rigid = rigid_steps * 13.0 * N * (C_ROT + C_TRI)
    return restarts * (C_POSE_ATOM * N + C_RESTART + passes * (sweep + rigid) + C_FIN * N)


def ligand_flops_ranked(batch, restarts: int, passes: int, decision_rank, rigid_steps: int = 0) -> np.ndarray:
    """ligand_flops with each decision's clash pairs credited j* times:
    decision_rank holds j* for every decision of every restart in the layout
    of lg_dock_result.restart_tors (restarts*passes*rot_off[l] + (r*passes +
    pass)*R_l + k)."""
    _, pairs, rl, L = _bond_counts(batch)
    roff = batch.rot_off.astype(np.int64)
    nrot = np.diff(roff)
    per = restarts * passes * nrot                      # decisions per ligand
    ranks = (np.asarray(decision_rank)[: int(per.sum())].astype(np.int64) & RANK_MASK).astype(np.float64)
    lig = np.repeat(np.arange(L), per)
    local = np.arange(ranks.size) - np.repeat(np.cumsum(per) - per, per)
    bond = roff[lig] + local % np.maximum(nrot[lig], 1)
    jsum = np.bincount(bond, weights=ranks, minlength=int(roff[-1]))  # sum of j* per bond
    extra = np.zeros(L)
    np.add.at(extra, rl, C_PAIR * (jsum - restarts * passes) * pairs)
    return ligand_flops(batch, restarts, passes, rigid_steps) + extra


def ligand_flops_needed(batch, restarts: int, passes: int, decision_rank) -> np.ndarray:
    """The work a docking run needed: ligand_flops_ranked without the
    decisions its exact convergence stops skipped (bit 7 of decision_rank:
    after R decisions in a row without a move every later decision repeats
    one of them, so neither its lookups nor its clash pairs are needed).  Per
    restart the rigid pose and the final score stay."""
    m, pairs, rl, L = _bond_counts(batch)
    roff = batch.rot_off.astype(np.int64)
    nrot = np.diff(roff)
    per = restarts * passes * nrot
    raw = np.asarray(decision_rank)[: int(per.sum())].astype(np.int64)
    run = (raw & RANK_SKIPPED) == 0
    jstar = (raw & RANK_MASK).astype(np.float64)
    lig = np.repeat(np.arange(L), per)
    local = np.arange(raw.size) - np.repeat(np.cumsum(per) - per, per)
    bond = roff[lig] + local % np.maximum(nrot[lig], 1)
    work = np.where(run, 36.0 * m[bond] * (C_ROT + C_TRI) + C_PAIR * jstar * pairs[bond], 0.0)
    N = np.diff(batch.atom_off).astype(np.float64)
    out = restarts * (C_POSE_ATOM * N + C_RESTART + C_FIN * N)
    np.add.at(out, lig, work)
    return out


def ligand_flops_circle(batch, restarts: int, passes: int) -> np.ndarray:
    """FLOPs of the circle form the kernels evaluate (no clash pairs)."""
    N = np.diff(batch.atom_off).astype(np.float64)
    msum = moving_atoms_per_ligand(batch).astype(np.float64)
    return restarts * (passes * msum * (36 * C_LOOKUP_CIRCLE + C_BOND_CIRCLE) +
                       N * (C_POSE_ATOM + C_FINAL_CIRCLE) + C_RESTART)


def partition(costs, world: int):
    """Split ligands over `world` ranks with balanced total cost (longest
    processing time first: each ligand, in descending cost, goes to the least
    loaded rank).  Returns one sorted index array per rank."""
    costs = np.asarray(costs, np.float64)
    heap = [(0.0, r) for r in range(world)]
    parts = [[] for _ in range(world)]
    for l in np.argsort(-costs, kind="stable"):
        load, r = heapq.heappop(heap)
        parts[r].append(int(l))
        heapq.heappush(heap, (load + float(costs[l]), r))
    return [np.array(sorted(p), np.int64) for p in parts]


def pending(uid, done_uid) -> np.ndarray:
    """Indices of the ligands whose uid has no result yet: a screen resumed
    after a failure docks only these (results are keyed by uid and a re-run
    of a uid is bit-identical, so nothing else needs saving)."""
    return np.nonzero(~np.isin(np.asarray(uid, np.uint64), np.asarray(done_uid, np.uint64)))[0]


def gather_ranking(uid, score, k: int, group=None):
    """Global k best (lowest score, then lowest uid) over all ranks of the
    default process group: each rank sends its own k best, rank 0 merges.
    Returns (uid as uint64, score) arrays on rank 0 and None elsewhere.

    uids are full 64-bit values (both halves feed the restart counters), so
    they travel as their own int64 tensor holding the uint64 bits, never
    through a floating-point column; the tie rule compares them as uint64."""
    import torch
    import torch.distributed as dist

    uid = np.asarray(uid, np.uint64)
    score = np.asarray(score, np.float64)
    ok = np.isfinite(score)
    uid, score = uid[ok], score[ok]
    order = np.lexsort((uid, score))[:k]
    world = dist.get_world_size(group)
    n = torch.tensor([len(order)], dtype=torch.int64)
    counts = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(counts, n, group=group)
    kmax = int(max(c.item() for c in counts))
    u_pad = torch.zeros(kmax, dtype=torch.int64)
    s_pad = torch.full((kmax,), float("nan"), dtype=torch.float64)
    u_pad[: len(order)] = torch.from_numpy(np.ascontiguousarray(uid[order]).view(np.int64))
    s_pad[: len(order)] = torch.from_numpy(np.ascontiguousarray(score[order]))
    u_bufs = [torch.empty(kmax, dtype=torch.int64) for _ in range(world)]
    s_bufs = [torch.empty(kmax, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(u_bufs, u_pad, group=group)
    dist.all_gather(s_bufs, s_pad, group=group)
    if dist.get_rank(group) != 0:
        return None
    u = np.concatenate([b[: int(c.item())].numpy() for b, c in zip(u_bufs, counts)]).view(np.uint64)
    s = np.concatenate([b[: int(c.item())].numpy() for b, c in zip(s_bufs, counts)])
    order = np.lexsort((u, s))[:k]
    return u[order], s[order]
