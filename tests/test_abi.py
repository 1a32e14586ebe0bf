"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/lg.h declares (CPU only: no compute call is made)."""
import ctypes
import os
import re

import pytest

from paper_2110_11644_gb300 import build as lgbuild
from paper_2110_11644_gb300 import lg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lg_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_calls():
    names = _declared()
    for must in ("lg_create", "lg_destroy", "lg_pocket_load", "lg_dock_batch", "lg_score_poses",
                 "lg_stream_submit", "lg_stream_poll", "lg_stream_wait"):
        assert must in names
    assert set(names) == set(lg.EXPORTS)


def test_library_builds_and_exports_every_declared_symbol():
    path = lgbuild.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name


def test_struct_layouts_match_header():
    # sizes of the ctypes mirrors against the C layout rules (LP64)
    assert ctypes.sizeof(lg.lg_ligand_batch) == 8 + 10 * 8
    assert ctypes.sizeof(lg.lg_dock_params) == 64
    assert ctypes.sizeof(lg.lg_dock_result) == 8 + 12 * 8
    assert ctypes.sizeof(lg.lg_pose_batch) == 8 + 4 * 8
    assert ctypes.sizeof(lg.lg_stats) == 88
    assert ctypes.sizeof(lg.lg_flatten_params) == 20
    assert ctypes.sizeof(lg.lg_flatten_result) == 8 + 4 * 8


def test_struct_layout_against_compiled_c(tmp_path):
    # compile a tiny C program against include/lg.h and compare sizeof/offsetof
    prog = tmp_path / "lay.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "lg.h"\nint main(){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n",'
                    'sizeof(lg_pocket_desc), sizeof(lg_ligand_batch), sizeof(lg_dock_params), sizeof(lg_dock_result),'
                    'sizeof(lg_pose_batch), sizeof(lg_stats), offsetof(lg_dock_params, seed),'
                    'offsetof(lg_dock_params, rescore_top), offsetof(lg_dock_result, restart_geo),'
                    'sizeof(lg_flatten_params), sizeof(lg_flatten_result));return 0;}\n')
    exe = tmp_path / "lay"
    import subprocess
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(lg.lg_pocket_desc), ctypes.sizeof(lg.lg_ligand_batch), ctypes.sizeof(lg.lg_dock_params),
            ctypes.sizeof(lg.lg_dock_result), ctypes.sizeof(lg.lg_pose_batch), ctypes.sizeof(lg.lg_stats),
            lg.lg_dock_params.seed.offset, lg.lg_dock_params.rescore_top.offset, lg.lg_dock_result.restart_geo.offset,
            ctypes.sizeof(lg.lg_flatten_params), ctypes.sizeof(lg.lg_flatten_result)]
    assert got == want


def test_no_gpu_create_fails_cleanly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib = lg.load()
    h = ctypes.c_void_p()
    rc = lib.lg_create(0, ctypes.byref(h))
    assert rc in (lg.LG_ECUDA, lg.LG_EINVAL)
    assert lib.lg_last_error(None)
