"""lg_dock_batch_noalloc: docking for callers that cannot let the library
allocate device memory (applications whose device memory is owned by their own
pool allocator, and latency-critical callers that cannot take the device-wide
synchronisation of cudaMalloc / cudaFree).  Its scratch is a fixed device array
inside the library.

The file name sorts last so that, when it fails, a run that stops at the first
failure has already run every other test.  It builds its own context, so it
also passes alone in a fresh process.
"""
import numpy as np
import pytest

from paper_2110_11644_gb300 import lg, synth

pytestmark = pytest.mark.gpu


def _run(fn, ctx, pid, dev, L, A, R, params, stream):
    r, outs = lg.alloc_result(L, A, R, params.restarts, params.passes, device=True, pose=True, tors=True,
                              restart_score=True, restart_tors=True, decision_rank=True)
    b = lg.make_batch_struct(dev, L)
    p = lg.make_params(params.restarts, params.passes, params.seed, params.d_clash)
    fn(ctx.h, pid, b, p, r, stream.cuda_stream)
    stream.synchronize()
    n = dict(score=L, best_restart=L, status=L, tors_idx=params.passes * R, pose=3 * A,
             restart_score=L * params.restarts, restart_tors=params.restarts * params.passes * R,
             decision_rank=params.restarts * params.passes * R)
    return {k: v.cpu().numpy()[:n[k]] for k, v in outs.items() if v is not None}


def test_noalloc_matches_dock_batch_twice_in_a_row():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pocket = synth.config_pocket(1)
    batch = synth.config_ligands(1)
    params = synth.config_params(1)
    ctx = lg.Context(0)
    try:
        pid = ctx.load_pocket(pocket)
        L, A, R = batch.L, int(batch.atom_off[-1]), int(batch.rot_off[-1])
        dev = lg.device_batch_arrays(batch)
        stream = torch.cuda.current_stream()
        ref = _run(lg.lg_dock_batch, ctx, pid, dev, L, A, R, params, stream)
        assert np.all(ref["status"] == 0)
        first = _run(lg.lg_dock_batch_noalloc, ctx, pid, dev, L, A, R, params, stream)
        second = _run(lg.lg_dock_batch_noalloc, ctx, pid, dev, L, A, R, params, stream)
        for k in ref:
            # the same kernels run on the same inputs: results agree exactly,
            # which is within every tolerance the parity tests use
            assert np.array_equal(first[k], ref[k], equal_nan=True), k
            assert np.array_equal(second[k], ref[k], equal_nan=True), k

        # host memory would need staging buffers: rejected
        hb = lg.make_batch_struct(lg.host_batch_arrays(batch), L)
        r, _ = lg.alloc_result(L, A, R, params.restarts, params.passes, device=True)
        with pytest.raises(lg.LgError) as e:
            lg.lg_dock_batch_noalloc(ctx.h, pid, hb, lg.make_params(params.restarts, params.passes, params.seed), r,
                                     stream.cuda_stream)
        assert e.value.code == lg.LG_EINVAL
        # a batch beyond the fixed scratch is rejected with a clear error
        big = lg.lg_ligand_batch()
        big.L, big.mem = 1 << 20, lg.LG_MEM_DEVICE
        for f in ("atom_off", "x", "y", "z", "q", "type", "parent", "rot_off", "rot_child", "uid"):
            setattr(big, f, dev["x"].data_ptr())
        with pytest.raises(lg.LgError) as e:
            lg.lg_dock_batch_noalloc(ctx.h, pid, big, lg.make_params(params.restarts, params.passes, params.seed), r,
                                     stream.cuda_stream)
        assert e.value.code == lg.LG_EINVAL and "static scratch" in str(e.value)
    finally:
        ctx.close()
