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


class _FakeQueue:
    """Stand-in for the library's serving calls: at most `cap` requests in
    flight (a full queue answers LG_EAGAIN), each poll finishes the oldest."""

    def __init__(self, lg, cap, fail_at=None):
        self.lg, self.cap, self.fail_at = lg, cap, fail_at
        self.next, self.flight, self.done, self.waited, self.eagain = 0, [], set(), [], 0

    def submit(self, h, pid, b, p, r):
        if self.fail_at is not None and self.next == self.fail_at:
            raise self.lg.LgError(self.lg.LG_EINVAL, "bad request")
        if len(self.flight) >= self.cap:
            self.eagain += 1
            raise self.lg.LgError(self.lg.LG_EAGAIN, "serving queue full")
        t = self.next
        self.next += 1
        self.flight.append(t)
        return t

    def poll(self, h, t):
        if self.flight:
            self.done.add(self.flight.pop(0))
        return (self.lg.LG_REQ_DONE, 1e-3) if t in self.done else (self.lg.LG_REQ_RUNNING, 0.0)

    def wait(self, h, t, timeout_ms):
        self.waited.append(t)
        if t in self.flight:
            self.flight.remove(t)
        self.done.add(t)


def _fake_serving(monkeypatch, q):
    from paper_2110_11644_gb300 import lg

    class Ctx:
        h = None

        def set_option(self, k, v):
            pass

        def stats(self):
            return type("S", (), {"serve_loop_launches": 1, "serve_loop_switches": 0})()

    monkeypatch.setattr(lg, "lg_stream_submit", q.submit)
    monkeypatch.setattr(lg, "lg_stream_poll", q.poll)
    monkeypatch.setattr(lg, "lg_stream_wait", q.wait)
    monkeypatch.setattr(lg, "make_params", lambda *a, **k: None)
    monkeypatch.setattr(lg, "make_batch_struct", lambda *a, **k: None)
    monkeypatch.setattr(lg, "alloc_result", lambda *a, **k: (None, {}))
    return Ctx()


def test_serving_client_waits_on_a_full_queue(monkeypatch):
    # a full host queue pushes back: the request is resubmitted once earlier
    # ones finish, and every request of the leg completes
    from paper_2110_11644_gb300 import lg
    bench = _bench()
    q = _FakeQueue(lg, cap=2)
    ctx = _fake_serving(monkeypatch, q)
    pool = synth.config_ligands(2, 64)
    r = bench.serving_leg(ctx, [0], pool, synth.config_params(2), 1000.0, 1.0, 0.2, max_size=8)
    assert q.eagain > 0
    assert r["requests"] == q.next and not q.flight and len(q.done) == q.next
    assert r["ligands"] > 0 and r["p99_latency_s"] == 1e-3


def test_serving_client_keeps_buffers_until_requests_finish(monkeypatch):
    # an error of one submission leaves the leg only after every request
    # already in flight has finished (the library writes into their buffers)
    from paper_2110_11644_gb300 import lg
    bench = _bench()
    q = _FakeQueue(lg, cap=1 << 20, fail_at=6)
    q.poll = lambda h, t: (lg.LG_REQ_RUNNING, 0.0)  # nothing finishes on its own
    ctx = _fake_serving(monkeypatch, q)
    pool = synth.config_ligands(2, 64)
    try:
        bench.serving_leg(ctx, [0], pool, synth.config_params(2), 1000.0, 1.0, 0.5, max_size=8)
        raise AssertionError("the failed submission was not reported")
    except lg.LgError as e:
        assert e.code == lg.LG_EINVAL
    assert q.waited == list(range(6)) and not q.flight


def test_serving_leg_reports_latency_by_request_size(monkeypatch):
    from paper_2110_11644_gb300 import lg
    bench = _bench()
    q = _FakeQueue(lg, cap=4)
    ctx = _fake_serving(monkeypatch, q)
    pool = synth.config_ligands(2, 600)
    r = bench.serving_leg(ctx, [0], pool, synth.config_params(2), 2e5, 1.0, 0.2, max_size=512)
    groups = r["by_request_size"]
    assert sum(g["requests"] for g in groups.values()) == r["requests"]
    assert set(groups) <= {"1-63", "64-511", "512-2047"}
    assert r["p999_latency_s"] >= r["p99_latency_s"] >= r["p50_latency_s"]
