"""GPU-vs-oracle parity check with the near-tie rule.

The GPU computes in FP32 and the oracle in FP64, so a torsion decision may
legitimately differ where two candidate steps score within rounding of each
other, or where a clash distance sits within rounding of d_clash.  The check
therefore REPLAYS the GPU's decisions in the oracle: the oracle follows every
step the GPU applied (for every restart), records at each decision what it
would have chosen itself, its FP64 scores and clash distances, and then:

  1. every decision where the GPU's step differs from the oracle's own choice
     must be a near-tie: the GPU's step is admissible in FP64 or its clash
     margin is within TOL_CLASH, and every step the oracle ranks above it is
     within TOL_TIE of its score or has a clash margin within TOL_CLASH;
  2. every restart's score matches the replayed FP64 score to TOL_SCORE
     relative to max(|E|, sum |e_i|);
  3. the best restart is the oracle's argmin, or within TOL_SCORE of it;
  4. the best pose matches the replayed FP64 pose to RMSD <= TOL_RMSD A;
  5. tors_idx equals the best restart's decisions;
  6. with rigid refinement, every rigid move the GPU took that differs from
     the oracle's own choice scores within TOL_TIE of the oracle's best.

Tolerances (from the accuracy target): score gap 1e-5 relative, clash margin
1e-5 relative to d_clash^2, scores 1e-5 relative, pose RMSD 1e-3 A.
"""
import numpy as np

import oracle

TOL_TIE = 1e-5
TOL_CLASH = 1e-5
TOL_SCORE = 1e-5
TOL_RMSD = 1e-3
A = 36


def near_tie_ok(s, d2, g, o, dc2):
    """Is the GPU's step g acceptable where the oracle chose o (FP64 scores s and
    clash distances d2 of the 36 steps)?"""
    if g == o:
        return True
    tol_s = TOL_TIE * max(abs(s[o]), 1e-30)
    tol_c = TOL_CLASH * dc2
    adm = d2 >= dc2
    adm[0] = True
    if not adm[g] and abs(d2[g] - dc2) > tol_c:
        return False
    for t in range(A):
        if t == g or not adm[t]:
            continue
        beats = s[t] > s[g] or (s[t] == s[g] and t < g)
        if not beats:
            continue
        if s[t] - s[g] <= tol_s:
            continue
        if t != 0 and abs(d2[t] - dc2) <= tol_c:
            continue
        return False
    return True


def check(pocket, batch, params, gpu, report=None):
    """gpu: dict with score, best_restart, status, tors_idx, pose, restart_score,
    restart_tors (flat numpy arrays as the C-ABI lays them out)."""
    S, P = params.restarts, params.passes
    dc2 = float(np.float32(params.d_clash)) ** 2
    Rs = int(getattr(params, "rigid_steps", 0))
    rigid = gpu.get("restart_rigid") if Rs > 0 else None
    if Rs > 0:
        assert rigid is not None, "rigid refinement needs the GPU's restart_rigid decisions"
    rep = oracle.dock(pocket, batch, params, replay=gpu["restart_tors"], replay_rigid=rigid, trace=True, poses=True)
    n_rig = n_rig_dev = 0
    if Rs > 0:
        tg = rep["trace_G"].reshape(-1, 13)
        for d in range(len(rigid)):
            g, o = int(rigid[d]), int(rep["own_rigid"][d])
            n_rig += 1
            if g != o:
                n_rig_dev += 1
                assert tg[d, g] >= tg[d, o] - TOL_TIE * max(abs(tg[d, o]), 1e-30), \
                    f"rigid decision {d}: GPU candidate {g} vs oracle {o}, G={tg[d, [g, o]]}"

    L = batch.L
    aoff, roff = batch.atom_off, batch.rot_off
    n_dec = n_dev = 0
    worst_score = worst_rmsd = 0.0
    best_r_near = 0
    for l in range(L):
        assert rep["status"][l] == 0 and gpu["status"][l] == 0, f"ligand {l}: status"
        R = int(roff[l + 1] - roff[l])
        N = int(aoff[l + 1] - aoff[l])
        d0 = S * P * int(roff[l])
        for k in range(S * P * R):
            g = int(gpu["restart_tors"][d0 + k])
            o = int(rep["own"][d0 + k])
            n_dec += 1
            if g != o:
                n_dev += 1
                s = rep["trace_s"][(d0 + k) * A:(d0 + k + 1) * A]
                d2 = rep["trace_d2"][(d0 + k) * A:(d0 + k + 1) * A]
                assert near_tie_ok(s, d2, g, o, dc2), \
                    f"ligand {l} decision {k}: GPU step {g} vs oracle {o}, s={s[[g, o]]}, d2={d2[[g, o]]}"
        E_o = rep["restart_E"][l]
        Eabs = rep["restart_Eabs"][l]
        E_g = gpu["restart_score"][l * S:(l + 1) * S]
        scale = np.maximum(np.abs(E_o), Eabs)
        err = np.abs(E_g - E_o) / np.maximum(scale, 1e-30)
        worst_score = max(worst_score, float(err.max()))
        assert np.all(err <= TOL_SCORE), f"ligand {l}: restart scores rel err {err.max():.3g}"
        rg = int(gpu["best_restart"][l])
        ro = int(np.argmin(E_o))
        assert gpu["score"][l] == E_g[rg]
        if rg != ro:
            best_r_near += 1
            assert abs(E_o[rg] - E_o[ro]) <= TOL_SCORE * max(scale[rg], scale[ro]), f"ligand {l}: best restart"
        R_l = R
        assert np.array_equal(gpu["tors_idx"][P * int(roff[l]):P * int(roff[l]) + P * R_l],
                              gpu["restart_tors"][d0 + rg * P * R_l:d0 + (rg + 1) * P * R_l])
        a0 = int(aoff[l])
        Xo = rep["poses"][3 * S * a0 + 3 * N * rg:3 * S * a0 + 3 * N * (rg + 1)].reshape(N, 3)
        Xg = gpu["pose"][3 * a0:3 * (a0 + N)].reshape(N, 3).astype(np.float64)
        rmsd = float(np.sqrt(((Xo - Xg) ** 2).sum(1).mean()))
        worst_rmsd = max(worst_rmsd, rmsd)
        assert rmsd <= TOL_RMSD, f"ligand {l}: pose RMSD {rmsd:.3g}"
    out = dict(decisions=n_dec, deviations=n_dev, worst_score_rel=worst_score, worst_rmsd=worst_rmsd,
               best_restart_near_ties=best_r_near, rigid_decisions=n_rig, rigid_deviations=n_rig_dev)
    if report is not None:
        report.update(out)
    return out
