"""Host helpers of bench.py: the kernel-source hash that keys the committed
DRAM-traffic record ignores comments and layout but not code, and the FLOP
counts it reports are the cost model's."""
import importlib.util
import os

import numpy as np

from paper_2110_11644_gb300 import shard, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_kernel_hash_ignores_comments_but_not_code(tmp_path, monkeypatch):
    bench = _bench()
    src = tmp_path / "paper_2110_11644_gb300" / "csrc"
    src.mkdir(parents=True)
    for f in bench.KERNEL_SOURCES:
        (src / f).write_text("int a = 1; // note\n/* block\n comment */ int b = 2;\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_sha()
    for f in bench.KERNEL_SOURCES:
        (src / f).write_text("int a = 1;   // another note\n\n int b = 2; /* x */\n")
    assert bench.kernel_source_sha() == h0
    (src / bench.KERNEL_SOURCES[0]).write_text("int a = 2; int b = 2;\n")
    assert bench.kernel_source_sha() != h0


def test_traffic_record_is_well_formed():
    # the committed DRAM-traffic record: per-launch bytes of one capture, keyed
    # by the kernels' code (the bench reports null when the key is stale)
    import json
    rec = json.load(open(os.path.join(ROOT, "profiles", "dock_batched_traffic.json")))
    assert rec["passes"] == 1 and len(rec["kernel_source_sha"]) == 16
    assert rec["dram_bytes_per_launch"] == rec["dram_bytes_read_per_launch"] + rec["dram_bytes_write_per_launch"] > 0


def test_algorithmic_flops_are_the_cost_model():
    bench = _bench()
    b = synth.config_ligands(2, 40)
    assert bench.algorithmic_flops(b, 30, 3) == float(shard.ligand_flops(b, 30, 3).sum())
    assert bench.circle_form_flops(b, 30, 3) < bench.algorithmic_flops(b, 30, 3)
    ones = np.ones(int(30 * 3 * b.rot_off[-1]))
    assert np.isclose(shard.ligand_flops_ranked(b, 30, 3, ones).sum(), bench.algorithmic_flops(b, 30, 3))
