"""Serving (lg_stream_submit / poll / wait) on the GPU: continuous batching
of requests of uneven size, results identical to docking each request alone,
bounded waits, admission under a tight free-memory reserve -- through the
device-resident loop (the default) and, where marked, the host worker that
merges requests into ordinary launches."""
import time

import numpy as np
import pytest

from paper_2110_11644_gb300 import lg, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def served():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = lg.Context(0)
    pocket = synth.config_pocket(1)
    pid = ctx.load_pocket(pocket)
    yield ctx, pid
    ctx.close()


def _request(batch, params):
    """Host arrays + structs of one request (kept alive by the caller)."""
    arrs = lg.host_batch_arrays(batch)
    b = lg.make_batch_struct(arrs, batch.L)
    p = lg.make_params(params.restarts, params.passes, params.seed, params.d_clash)
    r, outs = lg.alloc_result(batch.L, int(batch.atom_off[-1]), int(batch.rot_off[-1]), params.restarts,
                              params.passes, device=False, pose=True, tors=True)
    return dict(arrs=arrs, b=b, p=p, r=r, outs=outs, L=batch.L, A=int(batch.atom_off[-1]),
                R=int(batch.rot_off[-1]))


def _trim(req, P):
    n = dict(score=req["L"], best_restart=req["L"], status=req["L"], tors_idx=P * req["R"], pose=3 * req["A"])
    return {k: v[:n[k]] for k, v in req["outs"].items() if k in n}


def test_results_same_alone_and_in_the_mix(served):
    ctx, pid = served
    params = synth.config_params(1)
    full = synth.config_ligands(1)
    rng = np.random.default_rng(0)
    sizes = [1, 7, 40, 3, 64, 17, 100, 24]
    starts = np.cumsum([0] + sizes)
    reqs, tickets = [], []
    for k, s in enumerate(sizes):  # submitted back to back: they are merged and overlap on the device
        sub = full.subset(range(starts[k], starts[k] + s))
        req = _request(sub, params)
        reqs.append((sub, req))
        tickets.append(lg.lg_stream_submit(ctx.h, pid, req["b"], req["p"], req["r"]))
    for t in tickets:
        assert lg.lg_stream_wait(ctx.h, t, 60000) == lg.LG_OK
        st, lat = lg.lg_stream_poll(ctx.h, t)
        assert st == lg.LG_REQ_DONE and lat >= 0.0
    for sub, req in reqs:
        alone = ctx.dock(pid, sub, params)
        got = _trim(req, params.passes)
        for k in got:
            assert np.array_equal(got[k], alone[k][:len(got[k])]), k
    # and equal to the same ligands docked inside the whole batch
    whole = ctx.dock(pid, full.subset(range(int(starts[-1]))), params)
    mixed = np.concatenate([_trim(req, params.passes)["score"] for _, req in reqs])
    assert np.array_equal(mixed, whole["score"])


def test_bounded_wait_and_unknown_ticket(served):
    ctx, pid = served
    params = synth.DockParams(restarts=16, passes=2)
    batch = synth.config_ligands(1, 200)
    req = _request(batch, params)
    t = lg.lg_stream_submit(ctx.h, pid, req["b"], req["p"], req["r"])
    try:
        lg.lg_stream_wait(ctx.h, t, 0)
    except lg.LgError as e:
        assert e.code == lg.LG_ETIMEOUT
    assert lg.lg_stream_wait(ctx.h, t, 60000) == lg.LG_OK
    with pytest.raises(lg.LgError) as e:
        lg.lg_stream_poll(ctx.h, 10 ** 12)
    assert e.value.code == lg.LG_EINVAL
    with pytest.raises(lg.LgError) as e:
        lg.lg_stream_wait(ctx.h, 10 ** 12, 10)
    assert e.value.code == lg.LG_EINVAL


@pytest.mark.parametrize("device_loop", [1, 0])
def test_admission_under_tight_memory_still_completes(device_loop):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = lg.Context(0)
    try:
        ctx.set_option("serve_device_loop", device_loop)
        # a reserve larger than the device: every request beyond the first in
        # flight waits for memory, but an idle device always admits one
        ctx.set_option("serve_mem_reserve_mb", 1 << 30)
        ctx.set_option("serve_max_inflight", 4)
        pid = ctx.load_pocket(synth.config_pocket(1))
        params = synth.config_params(1)
        full = synth.config_ligands(1)
        reqs, tickets = [], []
        for k in range(6):
            sub = full.subset(range(40 * k, 40 * k + 40))
            req = _request(sub, params)
            reqs.append((sub, req))
            tickets.append(lg.lg_stream_submit(ctx.h, pid, req["b"], req["p"], req["r"]))
        for t in tickets:
            assert lg.lg_stream_wait(ctx.h, t, 60000) == lg.LG_OK
        ref = ctx.dock(pid, full.subset(range(240)), params)
        got = np.concatenate([_trim(req, params.passes)["score"] for _, req in reqs])
        assert np.array_equal(got, ref["score"])
    finally:
        ctx.close()


def test_many_small_requests_latency_recorded(served):
    ctx, pid = served
    params = synth.config_params(1)
    full = synth.config_ligands(1)
    reqs, tickets = [], []
    t0 = time.perf_counter()
    for k in range(64):
        sub = full.subset([k % full.L])
        req = _request(sub, params)
        reqs.append(req)
        tickets.append(lg.lg_stream_submit(ctx.h, pid, req["b"], req["p"], req["r"]))
    for t in tickets:
        lg.lg_stream_wait(ctx.h, t, 60000)
    lats = [lg.lg_stream_poll(ctx.h, t)[1] for t in tickets]
    assert all(0.0 <= x <= time.perf_counter() - t0 + 1e-3 for x in lats)


def test_requests_with_rigid_moves_and_ranking(served):
    # requests with rigid refinement and pose ranking are merged only with
    # requests of the same kind; each result equals the direct call
    import dataclasses
    ctx, pid = served
    base = synth.config_params(1)
    kinds = [base, dataclasses.replace(base, rigid_steps=1),
             dataclasses.replace(base, rigid_steps=2, cluster_rmsd=3.0, rescore_top=4)]
    full = synth.config_ligands(1)
    reqs, tickets = [], []
    for k in range(9):
        prm = kinds[k % 3]
        sub = full.subset(range(20 * k, 20 * k + 20))
        arrs = lg.host_batch_arrays(sub)
        b = lg.make_batch_struct(arrs, sub.L)
        p = lg.make_params(prm.restarts, prm.passes, prm.seed, prm.d_clash, cluster_rmsd=prm.cluster_rmsd,
                           rescore_top=prm.rescore_top, rigid_steps=prm.rigid_steps, rigid_shift=prm.rigid_shift)
        ranking = prm.cluster_rmsd > 0
        r, outs = lg.alloc_result(sub.L, int(sub.atom_off[-1]), int(sub.rot_off[-1]), prm.restarts, prm.passes,
                                  restart_tors=True, ranking=ranking, rigid_steps=prm.rigid_steps)
        reqs.append((sub, prm, arrs, b, p, r, outs))
        tickets.append(lg.lg_stream_submit(ctx.h, pid, b, p, r))
    for t in tickets:
        assert lg.lg_stream_wait(ctx.h, t, 60000) == lg.LG_OK
    for sub, prm, _, _, _, _, outs in reqs:
        d = ctx.dock(pid, sub, prm, restart_tors=True, restart_rigid=True)
        S, P, R = prm.restarts, prm.passes, int(sub.rot_off[-1])
        n = dict(score=sub.L, best_restart=sub.L, pose=3 * int(sub.atom_off[-1]), restart_tors=S * P * R,
                 restart_rigid=sub.L * S * P * prm.rigid_steps, rank=sub.L * S, leader=sub.L * S)
        for k, m in n.items():
            if outs.get(k) is not None and m:
                assert np.array_equal(outs[k][:m], d[k][:m]), (prm, k)


def test_heavy_tailed_ranking_requests_equal_direct_calls(served):
    # merged requests of heavy-tailed ligands (atoms up to 100: one launch
    # per size class) with pose ranking: each result equals the direct call
    import dataclasses
    ctx, pid = served
    prm = dataclasses.replace(synth.config_params(3), restarts=12, passes=2, cluster_rmsd=3.0, rescore_top=4)
    heavy = synth.config_ligands(3, 600)
    assert heavy.n_atoms().max() > 64
    reqs, tickets = [], []
    for k in range(12):
        sub = heavy.subset(range(50 * k, 50 * k + 50))
        arrs = lg.host_batch_arrays(sub)
        b = lg.make_batch_struct(arrs, sub.L)
        p = lg.make_params(prm.restarts, prm.passes, prm.seed, prm.d_clash, cluster_rmsd=prm.cluster_rmsd,
                           rescore_top=prm.rescore_top)
        r, outs = lg.alloc_result(sub.L, int(sub.atom_off[-1]), int(sub.rot_off[-1]), prm.restarts, prm.passes,
                                  restart_tors=True, ranking=True)
        reqs.append((sub, arrs, b, p, r, outs))
        tickets.append(lg.lg_stream_submit(ctx.h, pid, b, p, r))
    for t in tickets:
        assert lg.lg_stream_wait(ctx.h, t, 60000) == lg.LG_OK
    for sub, _, _, _, _, outs in reqs:
        d = ctx.dock(pid, sub, prm, restart_tors=True)
        S, P, R = prm.restarts, prm.passes, int(sub.rot_off[-1])
        n = dict(score=sub.L, best_restart=sub.L, status=sub.L, pose=3 * int(sub.atom_off[-1]),
                 restart_tors=S * P * R, rank=sub.L * S, leader=sub.L * S, restart_geo=sub.L * S)
        for k, m in n.items():
            assert np.array_equal(outs[k][:m], d[k][:m]), k


@pytest.mark.parametrize("device_loop", [1, 0])
def test_requests_for_different_pockets_share_launches(device_loop):
    # requests aimed at three pockets share one launch (the loop always; the
    # host worker with serve_cross_pocket, one pocket per ligand); every result
    # equals docking the request alone against its pocket
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = lg.Context(0)
    try:
        ctx.set_option("serve_device_loop", device_loop)
        ctx.set_option("serve_max_inflight", 1)  # one slot: everything queued is merged
        ctx.set_option("serve_cross_pocket", 1)
        pockets = [synth.config_pocket(1), synth.config_pocket(4, 0), synth.config_pocket(4, 3)]
        pids = [ctx.load_pocket(p) for p in pockets]
        params = synth.config_params(1)
        full = synth.config_ligands(2, 400)
        reqs, tickets = [], []
        for k in range(18):
            sub = full.subset(range(20 * k, 20 * k + 20))
            req = _request(sub, params)
            pid = pids[k % 3]
            reqs.append((sub, pid, req))
            tickets.append(lg.lg_stream_submit(ctx.h, pid, req["b"], req["p"], req["r"]))
        for t in tickets:
            assert lg.lg_stream_wait(ctx.h, t, 60000) == lg.LG_OK
        for sub, pid, req in reqs:
            alone = ctx.dock(pid, sub, params)
            got = _trim(req, params.passes)
            for k in got:
                assert np.array_equal(got[k], alone[k][:len(got[k])]), k
    finally:
        ctx.close()


def test_admission_holds_back_a_ranked_request_while_a_slot_is_busy():
    # A ranked request needs pose slots in device scratch (12 B per atom,
    # restart and slot) on top of its inputs and outputs.  With free memory
    # minus the reserve below that need, it waits in the queue while another
    # batch runs, and is admitted once the device is idle.
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import dataclasses
    ctx = lg.Context(0)
    try:
        ctx.set_option("serve_device_loop", 0)  # the host worker's merged launches
        ctx.set_option("serve_max_inflight", 2)
        ctx.set_option("serve_mem_reserve_mb", 0)
        pid = ctx.load_pocket(synth.config_pocket(2))
        lig = synth.config_ligands(2, 62_000)
        busy_prm = dataclasses.replace(synth.config_params(2), restarts=64)
        busy = _request(lig.subset(range(60_000)), busy_prm)
        ranked_prm = dataclasses.replace(synth.config_params(2), restarts=256, cluster_rmsd=3.0, rescore_top=30)
        sub = lig.subset(range(60_000, 62_000))
        arrs = lg.host_batch_arrays(sub)
        b = lg.make_batch_struct(arrs, sub.L)
        p = lg.make_params(ranked_prm.restarts, ranked_prm.passes, ranked_prm.seed, ranked_prm.d_clash,
                           cluster_rmsd=ranked_prm.cluster_rmsd, rescore_top=ranked_prm.rescore_top)
        r, outs = lg.alloc_result(sub.L, int(sub.atom_off[-1]), int(sub.rot_off[-1]), ranked_prm.restarts,
                                  ranked_prm.passes, ranking=True)
        # pose slots of the ranked request: about 2,000 ligands x 256 restarts x
        # 60 atoms x 12 B = 370 MB; its inputs and outputs alone need ~10 MB
        t_busy = lg.lg_stream_submit(ctx.h, pid, busy["b"], busy["p"], busy["r"])
        while lg.lg_stream_poll(ctx.h, t_busy)[0] == lg.LG_REQ_QUEUED:
            time.sleep(1e-4)
        free, _ = torch.cuda.mem_get_info()
        ctx.set_option("serve_mem_reserve_mb", max(0, free // (1 << 20) - 100))
        t_rank = lg.lg_stream_submit(ctx.h, pid, b, p, r)
        held = 0
        while True:
            s_rank = lg.lg_stream_poll(ctx.h, t_rank)[0]  # the ranked request first: see below
            s_busy = lg.lg_stream_poll(ctx.h, t_busy)[0]
            # admitted only once the busy batch is done (its state is set
            # before the idle device admits the next batch)
            assert not (s_rank >= lg.LG_REQ_RUNNING and s_busy < lg.LG_REQ_DONE)
            held += s_rank == lg.LG_REQ_QUEUED and s_busy == lg.LG_REQ_RUNNING
            if s_busy >= lg.LG_REQ_DONE:
                break
            time.sleep(2e-4)
        assert held > 0
        assert lg.lg_stream_wait(ctx.h, t_busy, 120000) == lg.LG_OK
        assert lg.lg_stream_wait(ctx.h, t_rank, 120000) == lg.LG_OK
        d = ctx.dock(pid, sub, ranked_prm)
        for k in ("score", "best_restart", "status"):
            assert np.array_equal(outs[k][:sub.L], d[k][:sub.L]), k
    finally:
        ctx.close()


def _loop_ctx(idle_ms=None):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = lg.Context(0)
    if idle_ms is not None:
        ctx.set_option("serve_loop_idle_ms", idle_ms)
    return ctx


@pytest.mark.parametrize("lanes", [0, 16, 4])
def test_loop_requests_arriving_while_others_run(lanes):
    # requests of uneven size aimed at three pockets arrive one by one while
    # earlier ones are on the device: each result equals the request docked
    # alone, and the loop docked every ligand -- with the loop's restart tile
    # chosen by the backlog (the default) or fixed at 16 or 4 lanes
    ctx = _loop_ctx()
    try:
        ctx.set_option("serve_loop_lanes", lanes)
        pockets = [synth.config_pocket(2), synth.config_pocket(4, 0), synth.config_pocket(4, 5)]
        pids = [ctx.load_pocket(p) for p in pockets]
        params = synth.DockParams(restarts=64, passes=3)
        pool = synth.config_ligands(2, 12000)
        rng = np.random.default_rng(11)
        sizes = [int(v) for v in np.floor(np.exp(rng.uniform(0, np.log(2000), 14)))]
        starts = np.cumsum([0] + sizes)
        reqs, tickets = [], []
        for k, n in enumerate(sizes):
            sub = pool.subset(range(starts[k], starts[k] + n))
            req = _request(sub, params)
            pid = pids[k % 3]
            reqs.append((sub, pid, req))
            tickets.append(lg.lg_stream_submit(ctx.h, pid, req["b"], req["p"], req["r"]))
            time.sleep(2e-4)
        states = [lg.lg_stream_poll(ctx.h, t)[0] for t in tickets]
        for t in tickets:
            assert lg.lg_stream_wait(ctx.h, t, 120000) == lg.LG_OK
        st = ctx.stats()
        assert st.serve_loop_launches >= 1 and st.serve_loop_items == sum(sizes)
        for sub, pid, req in reqs:
            alone = ctx.dock(pid, sub, params)
            got = _trim(req, params.passes)
            for k in got:
                assert np.array_equal(got[k], alone[k][:len(got[k])]), k
        assert any(s < lg.LG_REQ_DONE for s in states)  # some were still running when the last arrived
    finally:
        ctx.close()


def test_loop_idle_limit_ends_the_launch_and_work_relaunches_it():
    # every wait of the loop is bounded: with no ligand to claim for the idle
    # limit its CTAs leave and the launch ends with LG_ETIMEOUT; a later
    # request launches it again
    ctx = _loop_ctx(idle_ms=5)
    try:
        pid = ctx.load_pocket(synth.config_pocket(1))
        params = synth.config_params(1)
        full = synth.config_ligands(1)
        first = _request(full.subset(range(0, 40)), params)
        t = lg.lg_stream_submit(ctx.h, pid, first["b"], first["p"], first["r"])
        assert lg.lg_stream_wait(ctx.h, t, 60000) == lg.LG_OK
        deadline = time.time() + 10.0
        while ctx.stats().serve_loop_status != lg.LG_ETIMEOUT and time.time() < deadline:
            time.sleep(0.01)
        st = ctx.stats()
        assert st.serve_loop_status == lg.LG_ETIMEOUT and st.serve_loop_launches == 1
        second = _request(full.subset(range(40, 100)), params)
        t = lg.lg_stream_submit(ctx.h, pid, second["b"], second["p"], second["r"])
        assert lg.lg_stream_wait(ctx.h, t, 60000) == lg.LG_OK
        assert ctx.stats().serve_loop_launches == 2
        for req, rng in ((first, range(0, 40)), (second, range(40, 100))):
            alone = ctx.dock(pid, full.subset(rng), params)
            got = _trim(req, params.passes)
            for k in got:
                assert np.array_equal(got[k], alone[k][:len(got[k])]), k
    finally:
        ctx.close()


def test_loop_closes_with_requests_in_flight():
    # closing the context stops the loop after the ligands on the device: the
    # call returns, and every request is either done or failed
    ctx = _loop_ctx()
    pid = ctx.load_pocket(synth.config_pocket(2))
    params = synth.config_params(2)
    pool = synth.config_ligands(2, 3000)
    reqs, tickets = [], []
    for k in range(6):
        req = _request(pool.subset(range(500 * k, 500 * k + 500)), params)
        reqs.append(req)
        tickets.append(lg.lg_stream_submit(ctx.h, pid, req["b"], req["p"], req["r"]))
    t0 = time.time()
    ctx.close()
    assert time.time() - t0 < 60.0


def test_loop_switches_restart_tiles_by_backlog():
    # the default tile choice: small requests run at 16 lanes per restart; a
    # request of 4,000 ligands lifts the backlog above eight waves of that
    # loop, which is stopped and relaunched at 4 lanes with the ligands its
    # CTAs had claimed carried over; after a quiet spell a small request
    # brings the 16-lane tile back.  Every result equals the request docked
    # alone.
    ctx = _loop_ctx()
    try:
        ctx.set_option("serve_loop_lanes", 0)
        pid = ctx.load_pocket(synth.config_pocket(2))
        params = synth.config_params(2)
        pool = synth.config_ligands(2, 4100)
        parts = [(0, 24), (24, 4024), (4024, 4040), (4040, 4060)]
        done = []
        for k, (a, b) in enumerate(parts):
            sub = pool.subset(range(a, b))
            req = _request(sub, params)
            t = lg.lg_stream_submit(ctx.h, pid, req["b"], req["p"], req["r"])
            assert lg.lg_stream_wait(ctx.h, t, 120000) == lg.LG_OK
            done.append((sub, req))
            sw = ctx.stats().serve_loop_switches
            if k == 0:
                assert sw == 0
            elif k == 1:
                assert sw == 1  # to 4 lanes for the large request
            elif k == 2:
                time.sleep(0.05)  # the backlog stays low
        assert ctx.stats().serve_loop_switches == 2  # back to 16 lanes for the last request
        assert ctx.stats().serve_loop_items == 4060
        for sub, req in done:
            alone = ctx.dock(pid, sub, params)
            got = _trim(req, params.passes)
            for k in got:
                assert np.array_equal(got[k], alone[k][:len(got[k])]), k
    finally:
        ctx.close()
