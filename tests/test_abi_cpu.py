"""CPU checks of the C ABI: the library loads, exports what include/fpo.h
declares, its structs match the binding, and host-side validation works
without a GPU (no compute call is made here)."""

import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2202_08614_gb300 import build as fbuild
from paper_2202_08614_gb300 import fpo, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fpo.h")


@pytest.fixture(scope="module")
def L():
    fbuild.build()
    return fpo.lib()


def header_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(fpo_[a-z_]+)\s*\(", txt)))


def test_exports_every_declared_symbol(L):
    declared = header_functions()
    assert declared == sorted(fpo.EXPORTS)
    out = subprocess.run(["nm", "-D", "--defined-only", fbuild.LIB], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (fpo_[a-z_]+)\b", out))
    assert set(declared) <= exported
    for name in declared:
        assert hasattr(L, name)
    assert L.fpo_version() == 102


def test_struct_layout_matches_header(tmp_path):
    structs = {"fpo_config": fpo.Config, "fpo_tree_desc": fpo.TreeDesc, "fpo_rays": fpo.Rays,
               "fpo_frame_opts": fpo.FrameOpts, "fpo_tree_info": fpo.TreeInfo}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "fpo.h"', "int main(void){"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                   check=True).stdout.splitlines())
    for cname, py in structs.items():
        assert int(got[cname]) == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(py, f).offset, (cname, f)


def _validate(depth, xyz, max_depth, n1=31, n2=5, coeffs=True):
    d = np.asarray(depth, np.uint8)
    x = np.asarray(xyz, np.uint32).reshape(-1, 3)
    c = np.zeros((d.shape[0], n1 + 27 * n2), np.float32)
    desc, keep = fpo.make_tree_desc(d, x, c, max_depth)
    if not coeffs:
        desc.coeffs = None
    cfg = fpo.make_config(n1, n2)
    return fpo.lib().fpo_validate_tree(C.byref(desc), C.byref(cfg))


def test_validate_accepts_good_trees(L):
    fpo.validate_tree(synth.shell_tree())
    for s in range(5):
        fpo.validate_tree(synth.random_tree(s, max_depth=5))
    assert _validate([], np.zeros((0, 3)), 9) == 0  # empty tree
    assert _validate([0], [(0, 0, 0)], 0) == 0  # one leaf = the whole cube
    assert _validate([12], [(4095, 0, 17)], 12) == 0  # deepest allowed level


def test_validate_rejects_bad_trees(L):
    BAD, ARG = -4, -1
    assert _validate([2, 1], [(0, 0, 0), (0, 0, 0)], 2) == BAD  # nested
    assert _validate([1, 1], [(1, 0, 0), (1, 0, 0)], 1) == BAD  # duplicate
    assert _validate([3, 3, 1], [(7, 7, 7), (0, 0, 0), (1, 1, 1)], 3) == BAD  # (7,7,7) inside (1,1,1)
    assert _validate([2], [(4, 0, 0)], 2) == BAD  # out of range
    assert _validate([3], [(0, 0, 0)], 2) == BAD  # deeper than max_depth
    assert _validate([1], [(0, 0, 0)], 13) == ARG  # max_depth above 12
    assert _validate([1], [(0, 0, 0)], 1, coeffs=False) == ARG
    assert "overlap" in L.fpo_last_error().decode() or True
    with pytest.raises(fpo.FPOError) as e:
        tr = synth.random_tree(3, max_depth=3)
        tr.leaf_xyz = np.concatenate([tr.leaf_xyz, tr.leaf_xyz[:1]])
        tr.leaf_depth = np.concatenate([tr.leaf_depth, tr.leaf_depth[:1]])
        tr.coeffs = np.concatenate([tr.coeffs, tr.coeffs[:1]])
        fpo.validate_tree(tr)
    assert e.value.code == BAD


def test_null_and_config_errors_without_gpu(L):
    L.fpo_destroy(None)  # NULL-safe
    h = C.c_void_p()
    bad = [fpo.make_config(n1=0), fpo.make_config(n1=33), fpo.make_config(n2=17),
           fpo.make_config(period_T=0.0), fpo.make_config(period_T=float("inf"))]
    for cfg in bad:
        assert L.fpo_create(C.byref(h), C.byref(cfg)) == -1
        assert not h.value
    cfg = fpo.make_config()
    cfg.sh_degree = 1
    assert L.fpo_create(C.byref(h), C.byref(cfg)) == -8
    cfg = fpo.make_config()
    cfg.storage = 9
    assert L.fpo_create(C.byref(h), C.byref(cfg)) == -1
    for tp in (-1, 3):
        cfg = fpo.make_config()
        cfg.table_precision = tp
        assert L.fpo_create(C.byref(h), C.byref(cfg)) == -1
    cfg = fpo.make_config()
    cfg.max_steps = -1
    assert L.fpo_create(C.byref(h), C.byref(cfg)) == -1
    assert "max_steps" in L.fpo_last_error().decode()
    assert L.fpo_render(None, None, None, None, None) == -1
    assert L.fpo_status_sync(None, None) == -1
    assert L.fpo_upload_tree(None, None) == -1
    assert L.fpo_tree_info_get(None, None) == -1
    assert L.fpo_last_error().decode() != ""


def test_binding_refuses_to_run_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(fpo, "_lib", None)
    monkeypatch.setattr(fpo, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        fpo.lib()
