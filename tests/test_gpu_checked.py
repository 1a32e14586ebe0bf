"""The debug build with device-side bounds checks (-DLG_CHECKS): every grid
cell, near-atom list entry, clash-pair pool entry and decision record index
of the docking kernels, and every ranking scratch slot, is checked, and a
failure turns into an error of the call.  The checked library docks the
parity cases (best restart, ranking, rigid moves, heavy-tailed size classes
at every width and with ranking, several pockets, flattening, the
allocation-free entry point, the serving loop) without a
failure and with results equal to the product build's bit for bit."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2110_11644_gb300 import build, lg, synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RUN = r"""
import dataclasses, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2110_11644_gb300 import lg, synth
out = {}
ctx = lg.Context(0)
p1, b1, prm1 = synth.config_pocket(1), synth.config_ligands(1), synth.config_params(1)
pid = ctx.load_pocket(p1)
for name, prm in (("best", prm1), ("ranking", dataclasses.replace(prm1, cluster_rmsd=3.0, rescore_top=4)),
                  ("rigid", dataclasses.replace(prm1, rigid_steps=2))):
    r = ctx.dock(pid, b1, prm, restart_score=True, restart_tors=True, decision_rank=True)
    for k, v in r.items():
        if v is not None:
            out[name + "/" + k] = v
p2 = synth.config_pocket(2)
pid2 = ctx.load_pocket(p2)
heavy, prm3 = synth.config_ligands(3, 900), synth.config_params(3)
for w in (1, 2, 4):
    ctx.set_option("warps_per_cta", w)
    r = ctx.dock(pid2, heavy, prm3, restart_score=True, restart_tors=True)
    for k, v in r.items():
        if v is not None:
            out["heavy%d/%s" % (w, k)] = v
ctx.set_option("warps_per_cta", 0)
# ranking over size classes: every class's launch uses the scratch slots
prm3r = dataclasses.replace(prm3, restarts=12, cluster_rmsd=3.0, rescore_top=4, rigid_steps=1)
r = ctx.dock(pid2, heavy, prm3r, restart_score=True, restart_tors=True, restart_rigid=True)
for k, v in r.items():
    if v is not None:
        out["heavyrank/" + k] = v
multi = ctx.dock_multi([pid, pid2], b1.subset(range(64)), prm1)
for j, r in enumerate(multi):
    out["multi%d/score" % j] = r["score"]
f = ctx.flatten(synth.config_ligands(2, 300), 3)
for k in ("xyz", "tors", "dsum"):
    out["flatten/" + k] = f[k]
# the allocation-free entry point collects its own bounds-check record
import torch
L, A, R = b1.L, int(b1.atom_off[-1]), int(b1.rot_off[-1])
dev = lg.device_batch_arrays(b1)
r, outs = lg.alloc_result(L, A, R, prm1.restarts, prm1.passes, device=True, pose=True, tors=True,
                          restart_tors=True)
st = torch.cuda.current_stream()
lg.lg_dock_batch_noalloc(ctx.h, pid, lg.make_batch_struct(dev, L),
                         lg.make_params(prm1.restarts, prm1.passes, prm1.seed, prm1.d_clash), r, st.cuda_stream)
st.synchronize()
for k, v in outs.items():
    if v is not None:
        out["noalloc/" + k] = v.cpu().numpy()
# the device-resident serving loop (descriptor ring and per-CTA slots checked)
keep = []
for j in range(3):
    sub = b1.subset(range(50 * j, 50 * j + 50))
    arrs = lg.host_batch_arrays(sub)
    bs = lg.make_batch_struct(arrs, sub.L)
    ps = lg.make_params(prm1.restarts, prm1.passes, prm1.seed, prm1.d_clash)
    rr, oo = lg.alloc_result(sub.L, int(sub.atom_off[-1]), int(sub.rot_off[-1]), prm1.restarts, prm1.passes)
    keep.append((arrs, bs, ps, rr, oo, lg.lg_stream_submit(ctx.h, pid if j != 1 else pid2, bs, ps, rr)))
for j, (_, _, _, _, oo, t) in enumerate(keep):
    lg.lg_stream_wait(ctx.h, t, 120000)
    for k in ("score", "best_restart", "status", "tors_idx", "pose"):
        out["loop%d/%s" % (j, k)] = oo[k]
ctx.close()
np.savez(sys.argv[2], **out)
"""


def _run(tmp_path, variant):
    path = str(tmp_path / f"res_{variant or 'product'}.npz")
    env = dict(os.environ, LG_LIBRARY_VARIANT=variant)
    subprocess.run([sys.executable, "-c", RUN, ROOT, path], check=True, env=env, timeout=900)
    return np.load(path)


def test_checked_build_docks_without_bounds_failures_and_equal_results(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build(variant="checked")
    got = _run(tmp_path, "checked")  # a bounds failure would raise in the child
    want = _run(tmp_path, "")
    assert set(got.files) == set(want.files)
    for k in want.files:
        assert np.array_equal(got[k], want[k]), k
