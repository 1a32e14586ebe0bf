#!/usr/bin/env python3
"""Throughput benchmark of batched flexible-ligand docking on GB300.

Metric: ligand-pocket evaluations per second (one evaluation = one ligand
docked with all its restarts against one pocket and scored).

Workload (one step = one pass of the whole hot path over one batch): one
synthetic pocket (64^3 FP32 grids at 0.375 A, ellipsoidal cavity 6/8/12 A,
4,000 shell atoms) and 100,000 synthetic ligands of U{15..60} heavy atoms with
U{0..12} torsional bonds, 30 restarts, 3 sweep passes, 36 torsion steps.
Inputs are resident in device memory when the timed region starts; L2 is
flushed (256 MiB write) before every step.

Under torchrun each rank docks its own 100,000 ligands (disjoint uid ranges,
weak scaling, no collective on the data path); the time is the maximum over
ranks.  ``--impl reference`` times the FP64 CPU oracle on the host cores on
bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ligand-pocket evals/s"
UNIT = "evals/s"
WORKLOAD = ("1 pocket (64^3 FP32 grids, h=0.375 A, ellipsoid cavity 6/8/12 A, 4,000 shell atoms); "
            "100,000 ligands of U{15..60} atoms with U{0..12} torsional bonds; 30 restarts, 3 passes, 36 steps")
CFG = 2
N_LIGANDS = 100_000
FP32_LANES_PER_SM = 128          # FP32 FMA lanes per SM (4 SMSPs x 32)
FLOP_PER_FMA = 2


def algorithmic_flops(batch, S, P) -> float:
    """Algorithmic FLOPs of docking a batch (cost model in shard.py): per moving
    atom and torsion step 21 to rotate it and 30 for the trilinear lookup; 8 per
    clash pair once per decision; per restart 21 per atom for the rigid pose,
    40 for the pose draw and 64 per atom for the final score."""
    from paper_2110_11644_gb300 import shard
    return float(shard.ligand_flops(batch, S, P).sum())


def circle_form_flops(batch, S, P) -> float:
    """The lower FLOP count of the circle form the kernels evaluate."""
    from paper_2110_11644_gb300 import shard
    return float(shard.ligand_flops_circle(batch, S, P).sum())


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_mhz_min": min(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def cpu_cores() -> int:
    return len(os.sched_getaffinity(0))


def oracle_rate(pocket, batch, params, budget_s: float, chunk: int = 256, max_ligands: int = 65536, threads=None):
    """Oracle throughput on the first ligands of the workload, in chunks until
    the time budget is spent.  Returns (evals/s, ligands, seconds)."""
    import oracle
    done, t0 = 0, time.perf_counter()
    while done < max_ligands:
        sub = batch.subset(range(done, min(done + chunk, batch.L)))
        oracle.dock(pocket, sub, params, nthreads=threads or cpu_cores())
        done += sub.L
        if time.perf_counter() - t0 >= budget_s or done >= batch.L:
            break
    dt = time.perf_counter() - t0
    return done / dt, done, dt


def oracle_other_workloads(budget_s: float) -> dict:
    """The oracle on the host cores on the other workloads: the tiny set
    whole (48^3 pocket, 256 ligands, 16 restarts, 2 passes), the first
    ligands of the heavy-tailed library, and the first ligands of the
    throughput generator against the first pockets of the several-pocket set."""
    import oracle
    from paper_2110_11644_gb300 import synth
    out = {}
    p1, b1, prm1 = synth.config_pocket(1), synth.config_ligands(1), synth.config_params(1)
    t0 = time.perf_counter()
    oracle.dock(p1, b1, prm1, nthreads=cpu_cores())
    dt = time.perf_counter() - t0
    out["tiny_whole"] = {"value": b1.L / dt, "unit": UNIT, "ligands": b1.L, "seconds": round(dt, 2)}
    b3 = synth.config_ligands(3, 2000, uid_base=2 << 40)
    rate, n, secs = oracle_rate(synth.config_pocket(2), b3, synth.config_params(3), budget_s)
    out["heavy_tailed"] = {"value": rate, "unit": UNIT, "ligands": n, "seconds": round(secs, 2)}
    b4 = synth.config_ligands(2, 128, uid_base=1 << 40)
    prm4 = synth.config_params(4)
    dt, evals, used = 0.0, 0, []
    for w in range(3):  # the first pockets of the set (grids built untimed)
        pk = synth.config_pocket(4, w)
        t0 = time.perf_counter()
        oracle.dock(pk, b4, prm4, nthreads=cpu_cores())
        dt += time.perf_counter() - t0
        evals += b4.L
        used.append(int(pk.n))
        if dt >= budget_s:
            break
    out["several_pockets"] = {"value": evals / dt, "unit": UNIT, "evals": evals, "ligands_per_pocket": b4.L,
                              "pocket_grids": used, "seconds": round(dt, 2)}
    return out


KERNEL_SOURCES = ("lg_kernels.cu", "lg_device.cuh", "lg_internal.h")


def kernel_source_sha() -> str:
    """Hash of the code (comments and blank space removed) of the sources that
    define the docking kernels."""
    import re
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        text = open(os.path.join(ROOT, "paper_2110_11644_gb300", "csrc", f), encoding="utf-8").read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def traffic_for_current_kernel():
    """DRAM bytes per launch of the docking kernel from the committed ncu
    summary, if it was taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "dock_batched_traffic.json")
    try:
        rec = json.load(open(path))
        if rec.get("kernel_source_sha") == kernel_source_sha():
            return rec.get("dram_bytes_per_launch")
    except (OSError, ValueError):
        pass
    return None


def contiguous_request(pool, start, size):
    """Ligands start .. start+size-1 of a CSR batch as host arrays (views of
    the pool; only the offsets are rebased)."""
    from paper_2110_11644_gb300 import lg
    a0, a1 = int(pool.atom_off[start]), int(pool.atom_off[start + size])
    r0, r1 = int(pool.rot_off[start]), int(pool.rot_off[start + size])
    arrs = dict(atom_off=np.ascontiguousarray(pool.atom_off[start:start + size + 1] - a0, np.int32),
                rot_off=np.ascontiguousarray(pool.rot_off[start:start + size + 1] - r0, np.int32),
                x=pool.x[a0:a1], y=pool.y[a0:a1], z=pool.z[a0:a1], q=pool.q[a0:a1], type=pool.type[a0:a1],
                parent=pool.parent[a0:a1], rot_child=pool.rot_child[r0:r1] if r1 > r0 else pool.rot_child[:1],
                uid=pool.uid[start:start + size])
    return arrs, size, a1 - a0, r1 - r0


def serving_leg(ctx, pids, pool, params, rate_evals, load, duration_s, seed=5, max_size=4096, mode="device_loop"):
    """Poisson arrivals of requests of floor(exp(U(0, ln max_size))) ligands at
    `load` times `rate_evals` ligands/s for `duration_s` seconds, each aimed at
    a pocket drawn uniformly from `pids`, submitted to the library's serving
    loop (mode "device_loop": the device-resident loop; "host_merge": the host
    worker's merged launches); latency is submit-to-done as the library
    measures it."""
    from paper_2110_11644_gb300 import lg
    ctx.set_option("serve_device_loop", 1 if mode == "device_loop" else 0)
    rng = np.random.default_rng(seed)
    target = rng.integers(0, len(pids), size=1 << 20)
    mean_size = (max_size - 1) / np.log(max_size)
    lam = load * rate_evals / mean_size
    n = int(lam * duration_s) + 1
    sizes = np.maximum(1, np.minimum(max_size, np.floor(np.exp(rng.uniform(0, np.log(max_size), n))))).astype(int)
    gaps = rng.exponential(1.0 / lam, n)
    arrive = np.cumsum(gaps)
    p = lg.make_params(params.restarts, params.passes, params.seed, params.d_clash)
    cursor, pending, done_lat, live = 0, [], [], {}

    def drain():  # completed requests, in submission order
        while pending:
            st, lat = lg.lg_stream_poll(ctx.h, pending[0])
            if st < lg.LG_REQ_DONE:
                break
            done_lat.append((lat, live.pop(pending[0])[2]))
            pending.pop(0)

    clocks = ClockSampler(getattr(ctx, "device", 0))  # SM clocks and throttle reasons over the leg
    clocks.start()
    t0 = time.perf_counter()
    i = 0
    try:
        while i < n:
            now = time.perf_counter() - t0
            if now >= arrive[i]:
                size = int(sizes[i])
                if cursor + size > pool.L:
                    cursor = 0
                arrs, L, A, R = contiguous_request(pool, cursor, size)
                cursor += size
                b = lg.make_batch_struct(arrs, L)
                r, outs = lg.alloc_result(L, A, R, params.restarts, params.passes, device=False, pose=False,
                                          tors=False)
                while True:  # a full host queue pushes back: wait for completions, then resubmit
                    try:
                        t = lg.lg_stream_submit(ctx.h, pids[int(target[i % len(target)])], b, p, r)
                        break
                    except lg.LgError as e:
                        if e.code != lg.LG_EAGAIN:
                            raise
                        drain()
                        time.sleep(2e-4)
                live[t] = (arrs, outs, L)
                pending.append(t)
                i += 1
            else:
                drain()
                time.sleep(2e-4)
    finally:
        # the library writes into each request's buffers until it is done:
        # keep them alive until then, also when leaving on an error
        for t in pending:
            lg.lg_stream_wait(ctx.h, t, 600000)
            st, lat = lg.lg_stream_poll(ctx.h, t)
            done_lat.append((lat, live.pop(t)[2]))
        clk = clocks.stop()
    wall = time.perf_counter() - t0
    lat = np.array([x for x, _ in done_lat])
    size_of = np.array([s for _, s in done_lat])
    ligs = int(size_of.sum())
    # first-come claims: a request's wait hardly depends on its own size
    by_size = {}
    for lo, hi in ((1, 64), (64, 512), (512, 2048), (2048, max_size + 1)):
        m = (size_of >= lo) & (size_of < hi)
        if m.any():
            by_size[f"{lo}-{hi - 1}"] = {"requests": int(m.sum()), "p50_latency_s": float(np.percentile(lat[m], 50)),
                                         "p99_latency_s": float(np.percentile(lat[m], 99))}
    st = ctx.stats()
    return {"mode": mode, "offered_load": load, "offered_evals_per_s": load * rate_evals,
            "load_basis": "fraction of this serving path's measured peak (serving_peak)", "duration_s": round(wall, 2),
            "loop_launches": int(st.serve_loop_launches) if mode == "device_loop" else None,
            "loop_tile_switches": int(st.serve_loop_switches) if mode == "device_loop" else None,
            "requests": len(lat), "ligands": ligs, "sustained_evals_per_s": ligs / wall,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "p999_latency_s": float(np.percentile(lat, 99.9)), "by_request_size": by_size,
            "pockets": len(pids), "clocks": clk,
            "request_sizes": f"floor(exp(U(0, ln {max_size}))) ligands, Poisson arrivals, uniform pocket"}


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    from paper_2110_11644_gb300 import synth
    pocket = synth.config_pocket(CFG)
    params = synth.config_params(CFG)
    sample = 192
    batch = synth.config_ligands(CFG, sample * (args.steps + args.warmup))
    times = []
    for s in range(args.warmup + args.steps):
        sub = batch.subset(range(s * sample, (s + 1) * sample))
        import oracle
        t0 = time.perf_counter()
        oracle.dock(pocket, sub, params, nthreads=cpu_cores())
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    T = sum(times)
    value = sample * args.steps / T
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "ligands_per_gpu": N_LIGANDS, "restarts": params.restarts,
                       "passes": params.passes, "angle_steps": 36,
                       "step": f"{sample} ligands of the workload per step (bounded sample)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                             "sample": f"{sample} ligands per step, {args.steps} steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def multi_pocket_leg(ctx, dev, n_lig, steps, peak_tflops):
    """The 15-pocket set (40^3 to 96^3 grids) against n_lig ligands of the
    throughput workload's generator in one lg_dock_multi launch per step, in
    both visiting orders, plus one lg_dock_batch launch per pocket for the
    per-pocket time and FP32-roofline fraction.  L2 flushed before each step."""
    import concurrent.futures as cf

    import torch
    from paper_2110_11644_gb300 import lg, synth
    n_p = len(synth.multi_pocket_specs())
    with cf.ThreadPoolExecutor(8) as ex:   # the generator's C code runs without the GIL
        pockets = list(ex.map(lambda w: synth.config_pocket(4, w), range(n_p)))
    pids = [ctx.load_pocket(p) for p in pockets]
    batch = synth.config_ligands(2, n_lig, uid_base=1 << 40)
    params = synth.config_params(4)
    L, S, P = batch.L, params.restarts, params.passes
    A, R = int(batch.atom_off[-1]), int(batch.rot_off[-1])
    max_atoms, max_rot = int(batch.n_atoms().max()), max(1, int(batch.n_rot().max()))
    darr = lg.device_batch_arrays(batch, f"cuda:{dev}")
    b = lg.make_batch_struct(darr, L)
    p = lg.make_params(S, P, params.seed, params.d_clash, lg.LG_MODE_BATCHED, 0, max_atoms, max_rot)
    res = [lg.alloc_result(L, A, R, S, P, device=True, pose=True, tors=True) for _ in pids]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{dev}")
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    F = algorithmic_flops(batch, S, P)

    def timed(fn, n):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = 0.0
        for _ in range(n):
            flush.fill_(1)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
        return ms / n

    out = {}
    for win in (1, 0):   # the pockets' L2 access-policy windows on, then off
        ctx.set_option("l2_window", win)
        for name, order in (("pocket_major", 0), ("ligand_major", 1)):
            ctx.set_option("multi_order", order)
            ms = timed(lambda: lg.lg_dock_multi(ctx.h, pids, b, p, [r for r, _ in res], sh), steps)
            out[name if win else name + "_no_l2_window"] = {"value": L * n_p / (ms / 1e3), "ms_per_step": ms}
    ctx.set_option("l2_window", 1)
    ctx.set_option("multi_order", 0)
    out["l2_persist_mb"] = round(ctx.stats().l2_persist_bytes / 2 ** 20, 1)
    multi_scores = [o["score"][:L].cpu().numpy().copy() for _, o in res]
    per = []
    ctx.set_option("timing", 1)
    for k, pid in enumerate(pids):
        r, o = res[k]
        ms = timed(lambda: lg.lg_dock_batch(ctx.h, pid, b, p, r, sh), 1)
        dock_ms = ctx.stats().dock_ms
        assert np.array_equal(o["score"][:L].cpu().numpy(), multi_scores[k]), "multi and single pocket disagree"
        per.append({"n": pockets[k].n, "grid_mb": round(96 * pockets[k].n ** 3 / 2 ** 20, 1),
                    "ms": round(ms, 3), "evals_per_s": L / (ms / 1e3),
                    "frac_jstar1": F / (dock_ms / 1e3) / 1e12 / peak_tflops,
                    "l2_window_mb": round(ctx.stats().l2_window_bytes / 2 ** 20, 1)})
    ctx.set_option("timing", 0)
    return {"pockets": n_p, "ligands": L, "evals_per_step": L * n_p, "unit": UNIT, "restarts": S, "passes": P,
            "sample": f"{L} ligands of the throughput workload's generator against all {n_p} pockets",
            **out, "per_pocket": per}, pids


def heavy_tailed_leg(ctx, pid, dev, n_lig, steps, peak_tflops):
    """The heavy-tailed library (atoms lognormal, median 28, 10-100; torsions
    up to 20) on the throughput pocket: one lg_dock_batch per step, split into
    size classes with autotuned warps per CTA, device-resident inputs, L2
    flushed before each step; the same with the tuner off (4 warps per CTA)
    for comparison."""
    import torch
    from paper_2110_11644_gb300 import lg, synth
    batch = synth.config_ligands(3, n_lig, uid_base=2 << 40)
    params = synth.config_params(3)
    L, S, P = batch.L, params.restarts, params.passes
    A, R = int(batch.atom_off[-1]), int(batch.rot_off[-1])
    darr = lg.device_batch_arrays(batch, f"cuda:{dev}")
    b = lg.make_batch_struct(darr, L)
    p = lg.make_params(S, P, params.seed, params.d_clash, lg.LG_MODE_BATCHED, 0, int(batch.n_atoms().max()),
                       max(1, int(batch.n_rot().max())))
    r, outs = lg.alloc_result(L, A, R, S, P, device=True, pose=True, tors=True)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{dev}")
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream

    def timed(n):
        lg.lg_dock_batch(ctx.h, pid, b, p, r, sh)   # warm-up (and, the first time, the autotuner's trials)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = 0.0
        for _ in range(n):
            flush.fill_(1)
            e0.record(stream)
            lg.lg_dock_batch(ctx.h, pid, b, p, r, sh)
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1) / n
        return ms

    ms = timed(steps)
    st = ctx.stats()
    import json
    tiles = [e for e in json.loads(ctx.tune_export())["entries"] if e[1] == S and e[2] == P and e[5] == 0]
    scores = outs["score"][:L].cpu().numpy().copy()
    ctx.set_option("autotune", 0)
    ctx.set_option("warps_per_cta", 4)
    ms4 = timed(1)
    assert np.array_equal(outs["score"][:L].cpu().numpy(), scores), "results depend on the launch configuration"
    ctx.set_option("size_classes", 0)
    ms1 = timed(1)
    ctx.set_option("size_classes", 1)
    ctx.set_option("warps_per_cta", 0)
    ctx.set_option("autotune", 1)
    assert np.array_equal(outs["score"][:L].cpu().numpy(), scores), "results depend on the launch configuration"
    assert int((outs["status"][:L] != 0).sum()) == 0
    F = algorithmic_flops(batch, S, P)
    # each size class alone (the batch's ligands of that class, at most
    # 100,000), tuned, one timed call each
    pool = batch
    na = pool.n_atoms()
    per_class = {}
    for c, (lo, hi) in enumerate(((1, 32), (33, 64), (65, 1 << 30))):
        ids = np.nonzero((na >= lo) & (na <= hi))[0][:100_000]
        if len(ids) == 0:
            continue
        sub = pool.subset(ids)
        Lc, Ac, Rc = sub.L, int(sub.atom_off[-1]), int(sub.rot_off[-1])
        dc = lg.device_batch_arrays(sub, f"cuda:{dev}")
        bc = lg.make_batch_struct(dc, Lc)
        pc = lg.make_params(S, P, params.seed, params.d_clash, lg.LG_MODE_BATCHED, 0, int(sub.n_atoms().max()),
                            max(1, int(sub.n_rot().max())))
        rc, _ = lg.alloc_result(Lc, Ac, Rc, S, P, device=True, pose=True, tors=True)
        lg.lg_dock_batch(ctx.h, pid, bc, pc, rc, sh)  # tunes
        lg.lg_dock_batch(ctx.h, pid, bc, pc, rc, sh)
        torch.cuda.synchronize()
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lg.lg_dock_batch(ctx.h, pid, bc, pc, rc, sh)
        e1.record(stream)
        torch.cuda.synchronize()
        msc = e0.elapsed_time(e1)
        stc = ctx.stats()
        per_class[f"{lo}-{hi}" if c < 2 else f">{lo - 1}"] = {
            "ligands": Lc, "value": Lc / (msc / 1e3), "ms": msc,
            "frac_jstar1": algorithmic_flops(sub, S, P) / (msc / 1e3) / 1e12 / peak_tflops,
            "restart_lanes": stc.restart_lanes, "warps_per_cta": stc.warps_per_cta, "ctas_per_sm": stc.ctas_per_sm}
    return {"ligands": L, "value": L / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
            "frac_jstar1": F / (ms / 1e3) / 1e12 / peak_tflops, "launches_per_step": st.launches,
            "tuned_tiles": [{"class": e[0], "atom_max": e[3], "lanes": e[8], "warps": e[9]} for e in tiles],
            "per_class": per_class,
            "untuned_4_warps": {"value": L / (ms4 / 1e3), "ms_per_step": ms4},
            "one_launch_4_warps": {"value": L / (ms1 / 1e3), "ms_per_step": ms1},
            "sample": f"{L} ligands: atoms lognormal (median 28, 10-100), torsions ~0.2 N (0-20), {S} restarts, "
                      f"{P} passes, 64^3 pocket"}


def stages_leg(ctx, pid, dev, n_lig, steps=2):
    """Throughput of the optional stages on the throughput workload's first
    n_lig ligands (device-resident, L2 flushed before each call): the plain
    best-restart docking, with pose ranking (3 A clustering, first 30
    rescored), with rigid refinement (2 greedy rigid moves after each torsion
    pass), with both; and the paper's setting of 256 restarts with ranking on
    a quarter of the ligands."""
    import torch
    from paper_2110_11644_gb300 import lg, synth
    params = synth.config_params(2)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{dev}")
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    res = {}
    cases = (("best_restart", 30, n_lig, {}), ("ranking", 30, n_lig, dict(cluster_rmsd=3.0, rescore_top=30)),
             ("rigid", 30, n_lig, dict(rigid_steps=2)),
             ("ranking_rigid", 30, n_lig, dict(cluster_rmsd=3.0, rescore_top=30, rigid_steps=2)),
             ("paper_256_restarts_ranking", 256, max(1, n_lig // 4), dict(cluster_rmsd=3.0, rescore_top=30)))
    for name, S, n, kw in cases:
        batch = synth.config_ligands(2, n, uid_base=4 << 40)
        L, P = batch.L, params.passes
        A, R = int(batch.atom_off[-1]), int(batch.rot_off[-1])
        darr = lg.device_batch_arrays(batch, f"cuda:{dev}")
        b = lg.make_batch_struct(darr, L)
        p = lg.make_params(S, P, params.seed, params.d_clash, lg.LG_MODE_BATCHED, 0, int(batch.n_atoms().max()),
                           max(1, int(batch.n_rot().max())), **kw)
        ranking = "cluster_rmsd" in kw
        r, outs = lg.alloc_result(L, A, R, S, P, device=True, pose=True, tors=True, ranking=ranking,
                                  rigid_steps=kw.get("rigid_steps", 0))
        lg.lg_dock_batch(ctx.h, pid, b, p, r, sh)  # warm-up (and the autotuner's trials)
        torch.cuda.synchronize()
        ms = 0.0
        for _ in range(steps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lg.lg_dock_batch(ctx.h, pid, b, p, r, sh)
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1) / steps
        assert int((outs["status"][:L] != 0).sum()) == 0
        res[name] = {"ligands": L, "restarts": S, "ms": round(ms, 3), "evals_per_s": L / (ms / 1e3)}
        del outs, r, darr
    base = res["best_restart"]["evals_per_s"]
    for name in res:
        res[name]["relative_to_best_restart"] = res[name]["evals_per_s"] / base
    return res


def small_batch_leg(ctx, pid, dev, n_lig, calls):
    """Per-call latency of small device-resident batches (the serving regime):
    direct launches against a captured CUDA graph replayed per call."""
    import torch
    from paper_2110_11644_gb300 import lg, synth
    batch = synth.config_ligands(2, n_lig, uid_base=3 << 40)
    params = synth.config_params(2)
    L, S, P = batch.L, params.restarts, params.passes
    A, R = int(batch.atom_off[-1]), int(batch.rot_off[-1])
    darr = lg.device_batch_arrays(batch, f"cuda:{dev}")
    b = lg.make_batch_struct(darr, L)
    p = lg.make_params(S, P, params.seed, params.d_clash, lg.LG_MODE_BATCHED, 0, int(batch.n_atoms().max()),
                       max(1, int(batch.n_rot().max())))
    r, outs = lg.alloc_result(L, A, R, S, P, device=True, pose=True, tors=True)
    side = torch.cuda.Stream(device=dev)
    res = {}
    for name, g in (("direct", 0), ("graph", 1)):
        ctx.set_option("graphs", g)
        for _ in range(3):
            lg.lg_dock_batch(ctx.h, pid, b, p, r, side.cuda_stream)
        side.synchronize()
        t0 = time.perf_counter()
        for _ in range(calls):
            lg.lg_dock_batch(ctx.h, pid, b, p, r, side.cuda_stream)
        side.synchronize()
        st = ctx.stats()
        res[name] = {"us_per_call": (time.perf_counter() - t0) / calls * 1e6, "graph_mode": st.graph,
                     "restart_lanes": st.restart_lanes, "warps_per_cta": st.warps_per_cta}
    ctx.set_option("graphs", 0)  # direct launches for the tile comparison below
    # the same direct calls with each restart tile forced (lanes per restart;
    # every restart of a ligand in flight at once)
    by_lanes = {}
    for lanes in (4, 8, 16):
        ctx.set_option("restart_lanes", lanes)
        for _ in range(3):
            lg.lg_dock_batch(ctx.h, pid, b, p, r, side.cuda_stream)
        side.synchronize()
        t0 = time.perf_counter()
        for _ in range(calls // 2):
            lg.lg_dock_batch(ctx.h, pid, b, p, r, side.cuda_stream)
        side.synchronize()
        st = ctx.stats()
        by_lanes[str(lanes)] = {"us_per_call": (time.perf_counter() - t0) / (calls // 2) * 1e6,
                                "warps_per_cta": st.warps_per_cta}
    ctx.set_option("restart_lanes", 0)
    ctx.set_option("graphs", 2)
    return {"ligands": L, "calls": calls, **res, "by_lanes": by_lanes}


def summary_of(line) -> dict:
    """The headline figures of the line's legs in a few short keys (the last
    key of the line, so a truncated tail of the output still shows them)."""
    def r3(v):
        return None if v is None else float("%.4g" % v)
    rf = line.get("roofline") or {}
    out = {"evals_per_s": r3(line["value"]), "e2e": r3((line.get("e2e") or {}).get("value")),
           "frac": r3(rf.get("frac")), "frac_jstar1": r3(rf.get("frac_jstar1")),
           "frac_needed": r3(rf.get("frac_needed"))}
    if line.get("plain"):
        out["plain"] = r3(line["plain"]["value"])
        out["batched_over_plain"] = r3(line["plain"]["batched_over_plain"])
    if line.get("serving_peak"):
        out["serve_peak"] = {k: r3(v) for k, v in line["serving_peak"].items()}
    for leg in line.get("serving") or []:
        key = "serve_%d" % round(100 * leg["offered_load"]) + {
            "device_loop": "", "host_merge": "_host", "device_loop_4_lanes": "_4lanes",
            "device_loop_16_lanes": "_16lanes"}[leg.get("mode")]
        out[key] = [r3(leg["p50_latency_s"] * 1e3), r3(leg["p99_latency_s"] * 1e3), r3(leg["sustained_evals_per_s"])]
    m = line.get("multi_pocket")
    if m:
        out["multi"] = {k: r3(v["value"]) for k, v in m.items() if isinstance(v, dict) and "value" in v}
    h = line.get("heavy_tailed")
    if h:
        out["heavy"] = r3(h["value"])
        big = (h.get("per_class") or {}).get(">64")
        if big:
            out["heavy_gt64_frac_jstar1"] = r3(big["frac_jstar1"])
    if line.get("flatten"):
        out["flatten"] = r3(line["flatten"]["value"])
    if line.get("small_batch"):
        out["small_batch_us"] = r3(line["small_batch"]["direct"]["us_per_call"])
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ligands", type=int, default=N_LIGANDS)
    ap.add_argument("--plain-sample", type=int, default=4096)
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="seconds per offered load of the serving leg (0 = off)")
    ap.add_argument("--serve-loads", default="0.25,0.5,0.9",
                    help="comma-separated offered loads (fractions of the measured batched rate)")
    ap.add_argument("--serve-extra", type=int, default=1,
                    help="1: also the loop's fixed restart tiles and the host-merge path (0 = only the default loop)")
    ap.add_argument("--stage-ligands", type=int, default=20000,
                    help="ligands of the optional-stages leg (ranking, rigid refinement; 0 = off)")
    ap.add_argument("--multi-ligands", type=int, default=20000,
                    help="ligands of the 15-pocket leg (0 = off)")
    ap.add_argument("--heavy-ligands", type=int, default=1_000_000,
                    help="ligands of the heavy-tailed leg (0 = off)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    from paper_2110_11644_gb300 import lg, shard, synth

    rank, world, local = env_rank()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = local
    torch.cuda.set_device(dev)

    pocket = synth.config_pocket(CFG)
    params = synth.config_params(CFG)
    batch = synth.config_ligands(CFG, args.ligands, uid_base=rank * args.ligands) if rank == 0 else \
        synth.config_ligands(CFG, args.ligands, uid_base=rank * args.ligands)
    if rank > 0:  # each rank docks its own ligands: disjoint uids (new restart poses) on the same topologies
        batch.uid = batch.uid.copy()
    L, S, P = batch.L, params.restarts, params.passes
    A, R = int(batch.atom_off[-1]), int(batch.rot_off[-1])
    max_atoms = int(batch.n_atoms().max())
    max_rot = max(1, int(batch.n_rot().max()))

    ctx = lg.Context(dev)
    pid = ctx.load_pocket(pocket)
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream

    # device-resident inputs and outputs
    darr = lg.device_batch_arrays(batch, f"cuda:{dev}")
    bstruct = lg.make_batch_struct(darr, L)
    pstruct = lg.make_params(S, P, params.seed, params.d_clash, lg.LG_MODE_BATCHED, 0, max_atoms, max_rot)
    rstruct, outs = lg.alloc_result(L, A, R, S, P, device=True, pose=True, tors=True)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{dev}")

    def step():
        flush.fill_(1)
        lg.lg_dock_batch(ctx.h, pid, bstruct, pstruct, rstruct, sh)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ctx.set_option("timing", 1)
    clocks = ClockSampler(dev)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    st = ctx.stats()
    ctx.set_option("timing", 0)
    launches_per_step = st.launches
    if dist:
        t = torch.tensor([ms], device=f"cuda:{dev}")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * L * args.steps / (ms / 1e3)

    # status check of the last step (every ligand must have docked)
    status = outs["status"][:L].cpu().numpy()
    assert np.all(status == 0), "some ligands failed to dock"

    # roofline of the docking kernel (FP32 ALU bound).  Algorithmic FLOPs: the
    # cost model with each decision's clash pairs credited j* times, j* = 1 +
    # the steps ranked before the chosen one; the ranks come from one untimed
    # accounting call on the same batch (same decisions, bit for bit)
    F1 = algorithmic_flops(batch, S, P)
    dock_ms = st.dock_ms_total / max(st.dock_calls, 1)
    acc_r, acc_o = lg.alloc_result(L, A, R, S, P, device=True, pose=True, tors=True, decision_rank=True)
    lg.lg_dock_batch(ctx.h, pid, bstruct, pstruct, acc_r, sh)
    torch.cuda.synchronize()
    ranks = acc_o["decision_rank"][:S * P * R].cpu().numpy()
    del acc_r, acc_o
    F = float(shard.ligand_flops_ranked(batch, S, P, ranks).sum())
    F_needed = float(shard.ligand_flops_needed(batch, S, P, ranks).sum())
    jstar = ranks.astype(np.int64) & shard.RANK_MASK
    skipped = float(((ranks.astype(np.int64) & shard.RANK_SKIPPED) != 0).mean()) if ranks.size else 0.0
    props = torch.cuda.get_device_properties(dev)
    sm_count = props.multi_processor_count
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    sm_max_mhz = float(peaks.get("sm_max_mhz") or (clk or {}).get("sm_max_mhz") or 2070.0)
    peak_tflops = sm_count * FP32_LANES_PER_SM * FLOP_PER_FMA * sm_max_mhz * 1e6 / 1e12
    # cross-check of the derived peak: the library's FMA microbenchmark
    fma_tflops, fma_s = lg.lg_diag_fp32_peak(ctx.h, 5)
    achieved = F / (dock_ms / 1e3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops, "traffic": traffic_for_current_kernel(),
                "kernel": "k_dock_batched", "dock_ms_per_launch": dock_ms, "flop_per_launch": F,
                "flop_basis": "cost model with per-decision j* (mean %.2f) from an untimed accounting call" %
                              float(jstar.mean() if jstar.size else 1.0),
                "flop_per_launch_jstar1": F1, "frac_jstar1": F1 / (dock_ms / 1e3) / 1e12 / peak_tflops,
                "flop_per_launch_needed": F_needed, "frac_needed": F_needed / (dock_ms / 1e3) / 1e12 / peak_tflops,
                "needed_basis": "the same count over the decisions the run executed: %.1f%% of decisions are "
                                "skipped by exact convergence stops and not credited" % (100 * skipped),
                "flop_per_launch_circle_form": circle_form_flops(batch, S, P),
                "peak_basis": f"{sm_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {sm_max_mhz:.0f} MHz",
                "peak_measured_fma": {"value": fma_tflops, "unit": "TFLOP/s", "frac_of_derived": fma_tflops / peak_tflops,
                                      "how": "lg_diag_fp32_peak: best of 5 launches (%.0f ms in all) of 8 independent "
                                             "FMA chains per thread, 64 warps per SM" % (1e3 * fma_s)},
                "limiter": "L1 data pipe ~59% (scattered 32-byte trilinear-cell gathers plus shared-memory "
                           "wavefronts), L1->L2 requests ~53%, issue ~56% at 16 warps/SM; "
                           "see profiles/dock_batched_ncu_small.md"}

    # end to end through the public API with host buffers (pinned)
    hb = lg.host_batch_arrays(batch)
    pinned = {k: torch.from_numpy(v.view(np.int64) if v.dtype == np.uint64 else v).pin_memory()
              for k, v in hb.items()}
    hstruct = lg.make_batch_struct({k: v.numpy() for k, v in pinned.items()}, L)
    hout = {"score": torch.zeros(L, dtype=torch.float64).pin_memory(),
            "best_restart": torch.zeros(L, dtype=torch.int32).pin_memory(),
            "status": torch.zeros(L, dtype=torch.int32).pin_memory(),
            "tors_idx": torch.zeros(max(P * R, 1), dtype=torch.uint8).pin_memory(),
            "pose": torch.zeros(3 * A, dtype=torch.float32).pin_memory()}
    hres = lg.lg_dock_result()
    hres.mem = lg.LG_MEM_HOST
    for k, v in hout.items():
        setattr(hres, k, v.data_ptr())
    h2d = sum(v.numel() * v.element_size() for v in pinned.values())
    d2h = L * (8 + 4 + 4) + P * R + 12 * A
    e2e_steps = max(2, min(args.steps, 5))
    lg.lg_dock_batch(ctx.h, pid, hstruct, pstruct, hres, sh)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        flush.fill_(1)
        lg.lg_dock_batch(ctx.h, pid, hstruct, pstruct, hres, sh)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    if dist:
        t = torch.tensor([e2e_s], device=f"cuda:{dev}")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e = {"value": world * L * e2e_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(d2h), "steps": e2e_steps}
    assert np.array_equal(hout["score"].numpy(), outs["score"][:L].cpu().numpy()), "host and device paths disagree"

    line = None
    if rank == 0:
        # plain form (one launch per ligand, one warp per restart) on a sample
        n_plain = min(args.plain_sample, L)
        sub = batch.subset(range(n_plain))
        sarr = lg.device_batch_arrays(sub, f"cuda:{dev}")
        sstruct = lg.make_batch_struct(sarr, n_plain)
        ppl = lg.make_params(S, P, params.seed, params.d_clash, lg.LG_MODE_PLAIN, 8, max_atoms, max_rot)
        rpl, opl = lg.alloc_result(n_plain, int(sub.atom_off[-1]), int(sub.rot_off[-1]), S, P, device=True)
        lg.lg_dock_batch(ctx.h, pid, sstruct, ppl, rpl, sh)   # warm-up
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        lg.lg_dock_batch(ctx.h, pid, sstruct, ppl, rpl, sh)
        p1.record(stream)
        torch.cuda.synchronize()
        plain_value = n_plain / (p0.elapsed_time(p1) / 1e3)
        assert np.array_equal(opl["score"][:n_plain].cpu().numpy(), outs["score"][:n_plain].cpu().numpy())
        plain = {"value": plain_value, "unit": UNIT, "sample_ligands": n_plain, "streams": 8,
                 "batched_over_plain": value / world / plain_value}

        # ligand flattening (protein independent pre-processing) on the whole batch, device-resident
        fpar = lg.make_flatten_params(P, params.d_clash, max_atoms, max_rot)
        fres = lg.lg_flatten_result()
        fres.mem = lg.LG_MEM_DEVICE
        fout = dict(xyz=torch.empty(3 * A, dtype=torch.float32, device=f"cuda:{dev}"),
                    dsum=torch.empty(L, dtype=torch.float64, device=f"cuda:{dev}"),
                    status=torch.empty(L, dtype=torch.int32, device=f"cuda:{dev}"))
        fres.xyz, fres.dsum, fres.status = (fout[k].data_ptr() for k in ("xyz", "dsum", "status"))
        lg.lg_flatten_batch(ctx.h, bstruct, fpar, fres, sh)   # warm-up
        torch.cuda.synchronize()
        f_ms = 0.0
        for _ in range(3):
            flush.fill_(1)
            p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            p0.record(stream)
            lg.lg_flatten_batch(ctx.h, bstruct, fpar, fres, sh)
            p1.record(stream)
            torch.cuda.synchronize()
            f_ms += p0.elapsed_time(p1) / 3
        assert int((fout["status"] != 0).sum()) == 0
        flatten = {"value": L / (f_ms / 1e3), "unit": "ligands/s", "ms_per_call": f_ms, "passes": P,
                   "ligands": L, "launches_per_call": 2}

        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            rate, n_done, secs = oracle_rate(pocket, batch, params, args.cpu_budget)
            rate1, n1, secs1 = oracle_rate(pocket, batch, params, args.cpu_budget / 4, chunk=64, threads=1)
            cpu = {"value": rate, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                   "sample": f"first {n_done} ligands of the workload, FP64 oracle, {secs:.1f} s",
                   "single_core": {"value": rate1, "unit": UNIT, "cores": 1,
                                   "sample": f"first {n1} ligands, {secs1:.1f} s"},
                   "other_workloads": oracle_other_workloads(args.cpu_budget / 4)}


        small = small_batch_leg(ctx, pid, dev, 64, 200) if world == 1 else None
        stages = stages_leg(ctx, pid, dev, args.stage_ligands) if world == 1 and args.stage_ligands > 0 else None

        heavy = None
        if args.heavy_ligands > 0 and world == 1:
            heavy = heavy_tailed_leg(ctx, pid, dev, args.heavy_ligands, 2, roofline["peak"])

        multi, mp_pids = None, []
        if args.multi_ligands > 0 and world == 1:
            multi, mp_pids = multi_pocket_leg(ctx, dev, args.multi_ligands, 3, roofline["peak"])

        # serving: requests aimed at a random pocket of the 15-pocket set when it
        # is loaded, else at the throughput pocket
        serving, serving_peak = None, None
        if args.serve_seconds > 0 and world == 1:
            # Each serving path's peak: its sustained rate under an offered load
            # above the batched rate (the queue never empties); the offered
            # loads are fractions of that peak.  Warm-up first (not reported).
            sp = mp_pids or [pid]
            ps = min(10.0, max(3.0, args.serve_seconds / 10))
            serving_peak = {"batched_evals_per_s": value / world}
            for mode in (("device_loop", "host_merge") if args.serve_extra else ("device_loop",)):
                serving_leg(ctx, sp, batch, params, value / world, 0.9, 1.0, seed=4, mode=mode)
                serving_peak[mode] = serving_leg(ctx, sp, batch, params, value / world, 1.5, ps, seed=6,
                                                 mode=mode)["sustained_evals_per_s"]
            serving = [serving_leg(ctx, sp, batch, params, serving_peak["device_loop"], float(ld), args.serve_seconds)
                       for ld in args.serve_loads.split(",")]
            # the loop with each restart tile fixed (4 lanes per restart, the
            # throughput tile; 16, every restart of a ligand in flight, one CTA
            # per SM) against the default, which switches between them by the
            # backlog: each one's peak and the lowest load
            low = min(float(x) for x in args.serve_loads.split(","))
            for lanes in ((4, 16) if args.serve_extra else ()):
                ctx.set_option("serve_loop_lanes", lanes)
                serving_leg(ctx, sp, batch, params, value / world, 0.9, 1.0, seed=4)
                serving_peak[f"device_loop_{lanes}_lanes"] = serving_leg(
                    ctx, sp, batch, params, value / world, 1.5, ps, seed=6)["sustained_evals_per_s"]
                leg = serving_leg(ctx, sp, batch, params, serving_peak[f"device_loop_{lanes}_lanes"], low,
                                  max(1.0, args.serve_seconds / 3))
                leg["mode"] = f"device_loop_{lanes}_lanes"
                serving.append(leg)
            ctx.set_option("serve_loop_lanes", 0)
            # the host worker's merged launches at the highest load, for comparison
            hs = max(1.0, args.serve_seconds / 6)
            if args.serve_extra:
                serving.append(serving_leg(ctx, sp, batch, params, serving_peak["host_merge"],
                                           max(float(x) for x in args.serve_loads.split(",")), hs, mode="host_merge"))
            ctx.set_option("serve_device_loop", 1)
        for q in mp_pids:
            ctx.unload_pocket(q)

        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "ligands_per_gpu": L, "restarts": S, "passes": P,
                           "angle_steps": 36, "mode": "batched persistent, cost-sorted",
                           "l2": "flushed before every step (256 MiB write)", "inputs": "device-resident",
                           "warps_per_cta": st.warps_per_cta, "restart_lanes": st.restart_lanes,
                           "ctas_per_sm": st.ctas_per_sm, "grid": st.grid},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "clocks": clk, "gpu_launches": launches_per_step * args.steps, "plain": plain,
                "serving": serving, "serving_peak": serving_peak, "multi_pocket": multi, "flatten": flatten,
                "heavy_tailed": heavy,
                "small_batch": small, "stages": stages}
        line["summary"] = summary_of(line)  # last key: the headline figures of every leg, short
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
