"""ctypes binding of liblgdock (include/lg.h).

The ``lg_*`` functions here have the C names and take ctypes structs; they do
argument marshalling only -- every docking and scoring step runs in the CUDA
library.  ``Context`` adds numpy / torch conveniences on top (host arrays are
numpy, device arrays are CUDA torch tensors; PyTorch is used only for device
memory and streams).  If the library is missing or fails to load, every call
raises: there is no CPU fallback.
"""
from __future__ import annotations

import atexit
import ctypes
import os
import threading
import weakref

import numpy as np

from . import build as _build

LG_OK, LG_EINVAL, LG_ENOMEM, LG_EAGAIN, LG_ETIMEOUT, LG_ECUDA, LG_ENOPOCKET = range(7)
LG_MEM_HOST, LG_MEM_DEVICE = 0, 1
LG_MODE_BATCHED, LG_MODE_PLAIN = 0, 1
LG_REQ_QUEUED, LG_REQ_RUNNING, LG_REQ_DONE, LG_REQ_FAILED = range(4)
LG_MAX_ATOMS, LG_MAX_ROT, LG_MAX_PASSES, LG_MAX_RESTARTS = 128, 32, 8, 1024
LG_ANGLE_STEPS, LG_NUM_TYPES = 36, 5

_P = ctypes.c_void_p


class lg_pocket_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("h", ctypes.c_float), ("origin", ctypes.c_float * 3),
                ("phi_o", _P), ("phi_v", _P), ("phi_e", _P), ("n_pp", ctypes.c_int32), ("pocket_points", _P),
                ("type_w", ctypes.c_float * LG_NUM_TYPES), ("k_out", ctypes.c_float)]


class lg_ligand_batch(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("mem", ctypes.c_int32), ("atom_off", _P), ("x", _P), ("y", _P), ("z", _P),
                ("q", _P), ("type", _P), ("parent", _P), ("rot_off", _P), ("rot_child", _P), ("uid", _P)]


class lg_dock_params(ctypes.Structure):
    _fields_ = [("restarts", ctypes.c_int32), ("passes", ctypes.c_int32), ("angle_steps", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("d_clash", ctypes.c_float), ("mode", ctypes.c_int32),
                ("plain_streams", ctypes.c_int32), ("max_atoms", ctypes.c_int32), ("max_rot", ctypes.c_int32),
                ("cluster_rmsd", ctypes.c_float), ("rescore_top", ctypes.c_int32),
                ("rigid_steps", ctypes.c_int32), ("rigid_shift", ctypes.c_float)]


class lg_dock_result(ctypes.Structure):
    _fields_ = [("mem", ctypes.c_int32), ("score", _P), ("best_restart", _P), ("tors_idx", _P), ("pose", _P),
                ("status", _P), ("restart_score", _P), ("restart_tors", _P), ("rank", _P), ("leader", _P),
                ("restart_geo", _P), ("restart_rigid", _P), ("decision_rank", _P)]


class lg_flatten_params(ctypes.Structure):
    _fields_ = [("passes", ctypes.c_int32), ("angle_steps", ctypes.c_int32), ("d_clash", ctypes.c_float),
                ("max_atoms", ctypes.c_int32), ("max_rot", ctypes.c_int32)]


class lg_flatten_result(ctypes.Structure):
    _fields_ = [("mem", ctypes.c_int32), ("xyz", _P), ("tors", _P), ("dsum", _P), ("status", _P)]


class lg_pose_batch(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("mem", ctypes.c_int32), ("atom_off", _P), ("xyz", _P), ("q", _P),
                ("type", _P)]


class lg_stats(ctypes.Structure):
    _fields_ = [("dock_ms", ctypes.c_float), ("dock_calls", ctypes.c_int32), ("dock_ms_total", ctypes.c_double),
                ("launches", ctypes.c_int32), ("grid", ctypes.c_int32),
                ("warps_per_cta", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("smem_bytes", ctypes.c_int32),
                ("graph", ctypes.c_int32), ("serve_loop_status", ctypes.c_int32), ("restart_lanes", ctypes.c_int32),
                ("l2_window_bytes", ctypes.c_int64), ("l2_persist_bytes", ctypes.c_int64),
                ("serve_loop_launches", ctypes.c_int64), ("serve_loop_items", ctypes.c_int64),
                ("serve_loop_switches", ctypes.c_int64)]


# Every symbol include/lg.h declares (checked by the ABI test).
EXPORTS = ("lg_create", "lg_destroy", "lg_last_error", "lg_pocket_load", "lg_pocket_unload", "lg_dock_batch",
           "lg_score_poses", "lg_stream_submit", "lg_stream_poll", "lg_stream_wait", "lg_get_stats", "lg_set_option",
           "lg_diag_philox", "lg_diag_pocket_cells", "lg_diag_fp32_peak", "lg_dock_batch_noalloc", "lg_dock_multi", "lg_flatten_batch", "lg_tune_export",
           "lg_tune_import")

_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load():
    """Load liblgdock.so (building it first when missing or stale); the
    environment variable LG_LIBRARY_VARIANT=checked loads the debug build with
    device-side bounds checks instead."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build(variant=os.environ.get("LG_LIBRARY_VARIANT", ""))
            lib = ctypes.CDLL(path)
            c = ctypes
            V = c.c_void_p
            lib.lg_create.argtypes = [c.c_int, c.POINTER(V)]
            lib.lg_destroy.argtypes = [V]
            lib.lg_destroy.restype = None
            lib.lg_last_error.argtypes = [V]
            lib.lg_last_error.restype = c.c_char_p
            lib.lg_pocket_load.argtypes = [V, c.POINTER(lg_pocket_desc), c.POINTER(c.c_int32)]
            lib.lg_pocket_unload.argtypes = [V, c.c_int32]
            lib.lg_dock_batch.argtypes = [V, c.c_int32, c.POINTER(lg_ligand_batch), c.POINTER(lg_dock_params),
                                          c.POINTER(lg_dock_result), V]
            lib.lg_score_poses.argtypes = [V, c.c_int32, c.POINTER(lg_pose_batch), V, V]
            lib.lg_stream_submit.argtypes = [V, c.c_int32, c.POINTER(lg_ligand_batch), c.POINTER(lg_dock_params),
                                             c.POINTER(lg_dock_result), c.POINTER(c.c_uint64)]
            lib.lg_stream_poll.argtypes = [V, c.c_uint64, c.POINTER(c.c_int32), c.POINTER(c.c_double)]
            lib.lg_stream_wait.argtypes = [V, c.c_uint64, c.c_int32]
            lib.lg_get_stats.argtypes = [V, c.POINTER(lg_stats)]
            lib.lg_set_option.argtypes = [V, c.c_char_p, c.c_int64]
            lib.lg_diag_philox.argtypes = [V, c.c_int32, V, V, V, c.c_int32]
            lib.lg_diag_pocket_cells.argtypes = [V, c.c_int32, V, V]
            lib.lg_diag_fp32_peak.argtypes = [V, c.c_int32, c.POINTER(c.c_double), c.POINTER(c.c_double)]
            lib.lg_dock_batch_noalloc.argtypes = [V, c.c_int32, c.POINTER(lg_ligand_batch), c.POINTER(lg_dock_params),
                                                  c.POINTER(lg_dock_result), V]
            lib.lg_dock_multi.argtypes = [V, c.POINTER(c.c_int32), c.c_int32, c.POINTER(lg_ligand_batch),
                                          c.POINTER(lg_dock_params), c.POINTER(lg_dock_result), V]
            lib.lg_flatten_batch.argtypes = [V, c.POINTER(lg_ligand_batch), c.POINTER(lg_flatten_params),
                                             c.POINTER(lg_flatten_result), V]
            lib.lg_tune_export.argtypes = [V, c.c_char_p, c.c_int64, c.POINTER(c.c_int64)]
            lib.lg_tune_import.argtypes = [V, c.c_char_p]
            for name in EXPORTS:
                if name not in ("lg_destroy", "lg_last_error"):
                    getattr(lib, name).restype = c.c_int
            _lib = lib
    return _lib


class LgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"liblgdock error {code}: {msg}")
        self.code = code


def _check(ctx_handle, rc):
    if rc != LG_OK:
        msg = load().lg_last_error(ctx_handle)
        raise LgError(rc, msg.decode() if msg else "")
    return rc


# ----------------------------------------------------------------------------- C-named calls
def lg_create(device: int = 0):
    h = ctypes.c_void_p()
    _check(None, load().lg_create(device, ctypes.byref(h)))
    return h


def lg_destroy(h):
    load().lg_destroy(h)


def lg_last_error(h) -> str:
    return load().lg_last_error(h).decode()


def lg_pocket_load(h, desc: lg_pocket_desc) -> int:
    pid = ctypes.c_int32()
    _check(h, load().lg_pocket_load(h, ctypes.byref(desc), ctypes.byref(pid)))
    return pid.value


def lg_pocket_unload(h, pid: int):
    _check(h, load().lg_pocket_unload(h, pid))


def lg_dock_batch(h, pid, batch: lg_ligand_batch, params: lg_dock_params, out: lg_dock_result, stream=None):
    _check(h, load().lg_dock_batch(h, pid, ctypes.byref(batch), ctypes.byref(params), ctypes.byref(out), stream))


def lg_tune_export(h) -> str:
    """The autotuner's cached choices as JSON text (see lg.h)."""
    n = ctypes.c_int64()
    rc = load().lg_tune_export(h, None, 0, ctypes.byref(n))
    if rc != LG_OK and n.value <= 0:
        _check(h, rc)
    buf = ctypes.create_string_buffer(n.value + 1)
    _check(h, load().lg_tune_export(h, buf, n.value + 1, ctypes.byref(n)))
    return buf.value.decode()


def lg_tune_import(h, text: str):
    _check(h, load().lg_tune_import(h, text.encode()))


def lg_dock_batch_noalloc(h, pid, batch: lg_ligand_batch, params: lg_dock_params, out: lg_dock_result, stream=None):
    """Batched docking of a device-memory batch that allocates no memory (see lg.h)."""
    _check(h, load().lg_dock_batch_noalloc(h, pid, ctypes.byref(batch), ctypes.byref(params), ctypes.byref(out),
                                           stream))


def lg_dock_multi(h, pids, batch: lg_ligand_batch, params: lg_dock_params, outs, stream=None):
    """Dock one batch against several pockets in one launch; outs is a sequence
    of lg_dock_result, one per pocket id."""
    n = len(pids)
    ids = (ctypes.c_int32 * n)(*[int(p) for p in pids])
    res = (lg_dock_result * n)(*outs)
    _check(h, load().lg_dock_multi(h, ids, n, ctypes.byref(batch), ctypes.byref(params), res, stream))


def lg_flatten_batch(h, batch: lg_ligand_batch, params: lg_flatten_params, out: lg_flatten_result, stream=None):
    _check(h, load().lg_flatten_batch(h, ctypes.byref(batch), ctypes.byref(params), ctypes.byref(out), stream))


def make_flatten_params(passes, d_clash=2.0, max_atoms=0, max_rot=0):
    p = lg_flatten_params()
    p.passes, p.angle_steps, p.d_clash = int(passes), LG_ANGLE_STEPS, float(d_clash)
    p.max_atoms, p.max_rot = int(max_atoms), int(max_rot)
    return p


def lg_score_poses(h, pid, poses: lg_pose_batch, energies_ptr, stream=None):
    _check(h, load().lg_score_poses(h, pid, ctypes.byref(poses), energies_ptr, stream))


def lg_stream_submit(h, pid, batch, params, out) -> int:
    t = ctypes.c_uint64()
    _check(h, load().lg_stream_submit(h, pid, ctypes.byref(batch), ctypes.byref(params), ctypes.byref(out),
                                      ctypes.byref(t)))
    return t.value


def lg_stream_poll(h, ticket):
    st = ctypes.c_int32()
    lat = ctypes.c_double()
    _check(h, load().lg_stream_poll(h, ticket, ctypes.byref(st), ctypes.byref(lat)))
    return st.value, lat.value


def lg_stream_wait(h, ticket, timeout_ms: int) -> int:
    """Returns LG_OK, or raises (LG_ETIMEOUT and LG_ECUDA included)."""
    return _check(h, load().lg_stream_wait(h, ticket, timeout_ms))


def lg_get_stats(h) -> lg_stats:
    s = lg_stats()
    _check(h, load().lg_get_stats(h, ctypes.byref(s)))
    return s


def lg_set_option(h, key: str, value: int):
    _check(h, load().lg_set_option(h, key.encode(), int(value)))


def lg_diag_philox(h, n, ctr_ptr, key_ptr, out_ptr, use_curand: int):
    _check(h, load().lg_diag_philox(h, n, ctr_ptr, key_ptr, out_ptr, use_curand))


def lg_diag_fp32_peak(h, reps: int = 5):
    """Measured FP32 FMA throughput (TFLOP/s, best of reps) and the timed seconds."""
    t, sec = ctypes.c_double(), ctypes.c_double()
    _check(h, load().lg_diag_fp32_peak(h, reps, ctypes.byref(t), ctypes.byref(sec)))
    return t.value, sec.value


def lg_diag_pocket_cells(h, pid: int, n: int):
    """The packed cells of a loaded pocket: (cell_o [n^3, 8], cell_ve [n^3, 16]) float32."""
    import numpy as np
    o = np.empty((n ** 3, 8), np.float32)
    ve = np.empty((n ** 3, 16), np.float32)
    _check(h, load().lg_diag_pocket_cells(h, pid, o.ctypes.data, ve.ctypes.data))
    return o, ve


# ----------------------------------------------------------------------------- conveniences
def _ptr(a):
    """Address of a numpy array or torch tensor (None passes NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    assert a.is_contiguous()
    return a.data_ptr()


def _is_device(a) -> bool:
    return not isinstance(a, np.ndarray) and getattr(a, "is_cuda", False)


_BATCH_DTYPES = dict(atom_off=np.int32, x=np.float32, y=np.float32, z=np.float32, q=np.float32, type=np.uint8,
                     parent=np.int16, rot_off=np.int32, rot_child=np.int16, uid=np.uint64)


def host_batch_arrays(batch) -> dict:
    return {k: np.ascontiguousarray(getattr(batch, k), dt) for k, dt in _BATCH_DTYPES.items()}


def device_batch_arrays(batch, device="cuda") -> dict:
    """Copy a CSR batch (numpy attributes) into CUDA torch tensors."""
    import torch
    out = {}
    for k, dt in _BATCH_DTYPES.items():
        a = np.ascontiguousarray(getattr(batch, k), dt)
        if dt == np.uint64:
            a = a.view(np.int64)
        if dt == np.uint8:
            t = torch.from_numpy(a)
        else:
            t = torch.from_numpy(a)
        out[k] = t.to(device)
    return out


def make_batch_struct(arrs: dict, L: int) -> lg_ligand_batch:
    dev = _is_device(arrs["x"])
    b = lg_ligand_batch()
    b.L = L
    b.mem = LG_MEM_DEVICE if dev else LG_MEM_HOST
    for k in _BATCH_DTYPES:
        a = arrs[k]
        setattr(b, k, _ptr(a) if (a is not None and (len(a) if isinstance(a, np.ndarray) else a.numel()) > 0)
                else (_ptr(arrs["x"]) if k == "rot_child" else None))
    return b


def make_params(restarts, passes, seed, d_clash=2.0, mode=LG_MODE_BATCHED, plain_streams=0, max_atoms=0, max_rot=0,
                cluster_rmsd=0.0, rescore_top=0, rigid_steps=0, rigid_shift=0.375):
    p = lg_dock_params()
    p.restarts, p.passes, p.angle_steps = int(restarts), int(passes), LG_ANGLE_STEPS
    p.seed = int(seed)
    p.d_clash = float(d_clash)
    p.mode = int(mode)
    p.plain_streams = int(plain_streams)
    p.max_atoms, p.max_rot = int(max_atoms), int(max_rot)
    p.cluster_rmsd, p.rescore_top = float(cluster_rmsd), int(rescore_top)
    p.rigid_steps, p.rigid_shift = int(rigid_steps), float(rigid_shift)
    return p


def alloc_result(L, A, R, S, P, device=False, pose=True, tors=True, restart_score=False, restart_tors=False,
                 ranking=False, rigid_steps=0, decision_rank=False):
    """Output arrays for a batch: numpy (host) or CUDA torch tensors (device)."""
    if device:
        import torch
        z = lambda n, dt: torch.zeros(max(n, 1), dtype=dt, device="cuda")
        arrs = dict(score=z(L, torch.float64), best_restart=z(L, torch.int32), status=z(L, torch.int32),
                    tors_idx=z(P * R, torch.uint8) if tors else None, pose=z(3 * A, torch.float32) if pose else None,
                    restart_score=z(L * S, torch.float64) if restart_score else None,
                    restart_tors=z(S * P * R, torch.uint8) if restart_tors else None,
                    rank=z(L * S, torch.int32) if ranking else None, leader=z(L * S, torch.int32) if ranking else None,
                    restart_geo=z(L * S, torch.float64) if ranking else None,
                    restart_rigid=z(L * S * P * rigid_steps, torch.uint8) if rigid_steps else None,
                    decision_rank=z(S * P * R, torch.uint8) if decision_rank else None)
    else:
        z = lambda n, dt: np.zeros(max(n, 1), dt)
        arrs = dict(score=z(L, np.float64), best_restart=z(L, np.int32), status=z(L, np.int32),
                    tors_idx=z(P * R, np.uint8) if tors else None, pose=z(3 * A, np.float32) if pose else None,
                    restart_score=z(L * S, np.float64) if restart_score else None,
                    restart_tors=z(S * P * R, np.uint8) if restart_tors else None,
                    rank=z(L * S, np.int32) if ranking else None, leader=z(L * S, np.int32) if ranking else None,
                    restart_geo=z(L * S, np.float64) if ranking else None,
                    restart_rigid=z(L * S * P * rigid_steps, np.uint8) if rigid_steps else None,
                    decision_rank=z(S * P * R, np.uint8) if decision_rank else None)
    r = lg_dock_result()
    r.mem = LG_MEM_DEVICE if device else LG_MEM_HOST
    for k, v in arrs.items():
        setattr(r, k, _ptr(v))
    return r, arrs


def pocket_desc(pocket):
    """lg_pocket_desc for an object with n, h, origin, phi_o/v/e, pocket_points, type_w, k_out
    (the arrays must stay alive for the duration of lg_pocket_load)."""
    keep = dict(phi_o=np.ascontiguousarray(pocket.phi_o, np.float32).reshape(-1),
                phi_v=np.ascontiguousarray(pocket.phi_v, np.float32).reshape(-1),
                phi_e=np.ascontiguousarray(pocket.phi_e, np.float32).reshape(-1),
                pp=np.ascontiguousarray(pocket.pocket_points, np.int32).reshape(-1))
    d = lg_pocket_desc()
    d.n = int(pocket.n)
    d.h = float(pocket.h)
    for c in range(3):
        d.origin[c] = float(pocket.origin[c])
    d.phi_o, d.phi_v, d.phi_e = _ptr(keep["phi_o"]), _ptr(keep["phi_v"]), _ptr(keep["phi_e"])
    d.n_pp = len(keep["pp"]) // 3
    d.pocket_points = _ptr(keep["pp"])
    for t in range(LG_NUM_TYPES):
        d.type_w[t] = float(pocket.type_w[t])
    d.k_out = float(pocket.k_out)
    return d, keep


# Contexts still open when the interpreter exits are destroyed first (at
# exit, before modules and buffers are torn down), so the library's serving
# worker is stopped and joined while the buffers it writes into still exist.
_live_contexts = weakref.WeakSet()


@atexit.register
def _close_live_contexts():
    for c in list(_live_contexts):
        try:
            c.close()
        except Exception:
            pass


class Context:
    """One liblgdock context on a CUDA device."""

    def __init__(self, device: int = 0):
        self.h = lg_create(device)
        self.device = device
        _live_contexts.add(self)

    def close(self):
        if self.h is not None:
            lg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_pocket(self, pocket) -> int:
        d, keep = pocket_desc(pocket)
        return lg_pocket_load(self.h, d)

    def unload_pocket(self, pid):
        lg_pocket_unload(self.h, pid)

    def set_option(self, key, value):
        lg_set_option(self.h, key, value)

    def tune_export(self) -> str:
        return lg_tune_export(self.h)

    def tune_import(self, text: str):
        lg_tune_import(self.h, text)

    def stats(self) -> lg_stats:
        return lg_get_stats(self.h)

    def dock(self, pid, batch, params, *, mode=LG_MODE_BATCHED, device_io=False, pose=True, tors=True,
             restart_score=False, restart_tors=False, restart_rigid=False, stream=None, plain_streams=0, max_atoms=0,
             max_rot=0, decision_rank=False):
        """Dock a CSR batch (numpy attributes).  With device_io=True the batch is
        copied to the GPU first and the results come back from device buffers;
        otherwise the library stages host memory itself.  Returns numpy arrays.
        Pose ranking follows params.cluster_rmsd / params.rescore_top when the
        params object has them; its outputs are then rank, leader, restart_geo."""
        L = len(batch.atom_off) - 1
        A, R = int(batch.atom_off[-1]), int(batch.rot_off[-1])
        S, P = int(params.restarts), int(params.passes)
        arrs = device_batch_arrays(batch) if device_io else host_batch_arrays(batch)
        b = make_batch_struct(arrs, L)
        thr = float(getattr(params, "cluster_rmsd", 0.0))
        K = int(getattr(params, "rescore_top", 0))
        ranking = thr > 0.0 or 0 < K < S
        Rs = int(getattr(params, "rigid_steps", 0))
        p = make_params(S, P, params.seed, params.d_clash, mode, plain_streams, max_atoms, max_rot, thr, K, Rs,
                        float(getattr(params, "rigid_shift", 0.375)))
        r, outs = alloc_result(L, A, R, S, P, device=device_io, pose=pose, tors=tors, restart_score=restart_score,
                               restart_tors=restart_tors, ranking=ranking, rigid_steps=Rs if restart_rigid else 0,
                               decision_rank=decision_rank)
        if device_io:
            import torch
            s = torch.cuda.current_stream()
            lg_dock_batch(self.h, pid, b, p, r, s.cuda_stream if stream is None else stream)
            s.synchronize()
            outs = {k: (v.cpu().numpy() if v is not None else None) for k, v in outs.items()}
        else:
            lg_dock_batch(self.h, pid, b, p, r, stream)
        n = dict(score=L, best_restart=L, status=L, tors_idx=P * R, pose=3 * A, restart_score=L * S,
                 restart_tors=S * P * R, rank=L * S, leader=L * S, restart_geo=L * S, restart_rigid=L * S * P * Rs,
                 decision_rank=S * P * R)
        return {k: (v[:n[k]] if v is not None else None) for k, v in outs.items()}

    def dock_multi(self, pids, batch, params, *, device_io=False, pose=True, tors=True, restart_score=False,
                   restart_tors=False, restart_rigid=False, stream=None, max_atoms=0, max_rot=0, decision_rank=False):
        """Dock a CSR batch against several pockets in one launch; returns one
        dict of numpy arrays per pocket (as dock())."""
        L = len(batch.atom_off) - 1
        A, R = int(batch.atom_off[-1]), int(batch.rot_off[-1])
        S, P = int(params.restarts), int(params.passes)
        thr = float(getattr(params, "cluster_rmsd", 0.0))
        K = int(getattr(params, "rescore_top", 0))
        ranking = thr > 0.0 or 0 < K < S
        Rs = int(getattr(params, "rigid_steps", 0))
        arrs = device_batch_arrays(batch) if device_io else host_batch_arrays(batch)
        b = make_batch_struct(arrs, L)
        p = make_params(S, P, params.seed, params.d_clash, LG_MODE_BATCHED, 0, max_atoms, max_rot, thr, K, Rs,
                        float(getattr(params, "rigid_shift", 0.375)))
        res = [alloc_result(L, A, R, S, P, device=device_io, pose=pose, tors=tors, restart_score=restart_score,
                            restart_tors=restart_tors, ranking=ranking, rigid_steps=Rs if restart_rigid else 0,
                               decision_rank=decision_rank)
               for _ in pids]
        if device_io:
            import torch
            s = torch.cuda.current_stream()
            lg_dock_multi(self.h, pids, b, p, [r for r, _ in res], s.cuda_stream if stream is None else stream)
            s.synchronize()
        else:
            lg_dock_multi(self.h, pids, b, p, [r for r, _ in res], stream)
        n = dict(score=L, best_restart=L, status=L, tors_idx=P * R, pose=3 * A, restart_score=L * S,
                 restart_tors=S * P * R, rank=L * S, leader=L * S, restart_geo=L * S, restart_rigid=L * S * P * Rs,
                 decision_rank=S * P * R)
        out = []
        for _, outs in res:
            if device_io:
                outs = {k: (v.cpu().numpy() if v is not None else None) for k, v in outs.items()}
            out.append({k: (v[:n[k]] if v is not None else None) for k, v in outs.items()})
        return out

    def flatten(self, batch, passes, d_clash=2.0, *, device_io=False, stream=None):
        """Flatten a CSR batch; returns numpy xyz (flat, 3*atom_off), tors,
        dsum and status."""
        L = len(batch.atom_off) - 1
        A, R = int(batch.atom_off[-1]), int(batch.rot_off[-1])
        arrs = device_batch_arrays(batch) if device_io else host_batch_arrays(batch)
        b = make_batch_struct(arrs, L)
        p = make_flatten_params(passes, d_clash)
        if device_io:
            import torch
            z = lambda n, dt: torch.zeros(max(n, 1), dtype=dt, device="cuda")
            outs = dict(xyz=z(3 * A, torch.float32), tors=z(passes * R, torch.uint8), dsum=z(L, torch.float64),
                        status=z(L, torch.int32))
        else:
            z = lambda n, dt: np.zeros(max(n, 1), dt)
            outs = dict(xyz=z(3 * A, np.float32), tors=z(passes * R, np.uint8), dsum=z(L, np.float64),
                        status=z(L, np.int32))
        r = lg_flatten_result()
        r.mem = LG_MEM_DEVICE if device_io else LG_MEM_HOST
        for k, v in outs.items():
            setattr(r, k, _ptr(v))
        if device_io:
            import torch
            s = torch.cuda.current_stream()
            lg_flatten_batch(self.h, b, p, r, s.cuda_stream if stream is None else stream)
            s.synchronize()
            outs = {k: v.cpu().numpy() for k, v in outs.items()}
        else:
            lg_flatten_batch(self.h, b, p, r, stream)
        n = dict(xyz=3 * A, tors=passes * R, dsum=L, status=L)
        return {k: v[:n[k]] for k, v in outs.items()}

    def score_poses(self, pid, atom_off, xyz, q, type_):
        atom_off = np.ascontiguousarray(atom_off, np.int32)
        xyz = np.ascontiguousarray(xyz, np.float32).reshape(-1)
        q = np.ascontiguousarray(q, np.float32)
        t = np.ascontiguousarray(type_, np.uint8)
        L = len(atom_off) - 1
        E = np.zeros(max(L, 1), np.float64)
        pb = lg_pose_batch()
        pb.L, pb.mem = L, LG_MEM_HOST
        pb.atom_off, pb.xyz, pb.q, pb.type = _ptr(atom_off), _ptr(xyz), _ptr(q), _ptr(t)
        lg_score_poses(self.h, pid, pb, _ptr(E), None)
        return E[:L]
