"""The GPU-vs-oracle parity checker itself, exercised on CPU with results made
by the oracle (a perfect 'GPU') and with planted mistakes it must catch."""
import numpy as np
import pytest

import oracle
from _parity import check, near_tie_ok


def _as_abi(batch, params, out):
    """Oracle outputs laid out like the C-ABI results."""
    S, P = params.restarts, params.passes
    L = batch.L
    tors = np.zeros(max(P * int(batch.rot_off[-1]), 1), np.uint8)
    for l in range(L):
        R = int(batch.rot_off[l + 1] - batch.rot_off[l])
        d0 = S * P * int(batch.rot_off[l])
        r = int(out["best_r"][l])
        tors[P * int(batch.rot_off[l]):P * int(batch.rot_off[l]) + P * R] = out["choice"][d0 + r * P * R:d0 + (r + 1) * P * R]
    return dict(score=out["best_E"].copy(), best_restart=out["best_r"].copy(), status=out["status"].copy(),
                tors_idx=tors, pose=out["best_pose"].astype(np.float32), restart_score=out["restart_E"].reshape(-1).copy(),
                restart_tors=out["choice"].copy())


def test_checker_accepts_the_oracle(cfg1):
    pocket, batch, params = cfg1
    sub = batch.subset(range(48))
    gpu = _as_abi(sub, params, oracle.dock(pocket, sub, params))
    rep = check(pocket, sub, params, gpu)
    assert rep["deviations"] == 0 and rep["decisions"] > 100


def test_checker_rejects_a_wrong_decision(cfg1):
    pocket, batch, params = cfg1
    sub = batch.subset(range(48))
    out = oracle.dock(pocket, sub, params, trace=True)
    gpu = _as_abi(sub, params, out)
    s = out["trace_s"].reshape(-1, 36)
    # a decision where the best step beats the runner-up clearly
    k = next(i for i in range(len(s)) if np.sort(s[i])[-1] - np.sort(s[i])[-2] > 1e-3 * abs(s[i].max()))
    bad = dict(gpu)
    bad["restart_tors"] = gpu["restart_tors"].copy()
    bad["restart_tors"][k] = (int(gpu["restart_tors"][k]) + 18) % 36
    with pytest.raises(AssertionError):
        check(pocket, sub, params, bad)


def test_checker_rejects_score_and_pose_errors(cfg1):
    pocket, batch, params = cfg1
    sub = batch.subset(range(16))
    gpu = _as_abi(sub, params, oracle.dock(pocket, sub, params))
    bad = dict(gpu); bad["restart_score"] = gpu["restart_score"] * (1 + 1e-4)
    bad["score"] = bad["restart_score"].reshape(sub.L, -1)[np.arange(sub.L), gpu["best_restart"]]
    with pytest.raises(AssertionError):
        check(pocket, sub, params, bad)
    bad = dict(gpu); bad["pose"] = gpu["pose"] + np.float32(0.01)
    with pytest.raises(AssertionError):
        check(pocket, sub, params, bad)


def test_near_tie_rule():
    s = np.zeros(36); d2 = np.full(36, 10.0)
    s[5] = 1.0; s[7] = 1.0 - 1e-7; s[9] = 0.9
    assert near_tie_ok(s, d2, 7, 5, 4.0)          # within 1e-5 of the winner
    assert not near_tie_ok(s, d2, 9, 5, 4.0)      # clearly worse
    d2[5] = 4.0 + 1e-6                            # winner admissible only by a hair:
    assert near_tie_ok(s, d2, 7, 5, 4.0)          # the GPU may see it clash and take 7,
    assert not near_tie_ok(s, d2, 9, 5, 4.0)      # but never skip 7 as well
    d2[7] = 4.0 - 1e-6
    assert near_tie_ok(s, d2, 9, 5, 4.0)          # unless 7 is a clash near-tie too
    d2[9] = 3.0                                   # GPU picked a clearly clashing step
    assert not near_tie_ok(s, d2, 9, 0, 4.0)
