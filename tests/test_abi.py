"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/cg.h declares; the Python binding's struct layouts match the
header. No compute call is made (none needs a GPU here)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2207_04350_gb300 import _build, cg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cg.h")


@pytest.fixture(scope="module")
def libpath():
    return _build.build()


def declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^CG_API\s+[^(]*?\b(cg_\w+)\s*\(", txt, flags=re.M)))


def test_header_declares_the_paper_steps():
    names = declared()
    for n in ("cg_load_graph", "cg_mask_branches", "cg_chains", "cg_emit_contigs"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (cg_\w+)$", out, flags=re.M))
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(libpath)
    for n in declared():
        assert hasattr(lib, n)
    assert set(cg.API) == set(declared())


def test_build_targets_sm103a_only():
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_status_strings(libpath):
    for i, name in enumerate(["CG_OK", "CG_EINVAL", "CG_ENOMEM", "CG_ECUDA", "CG_EGRAPH", "CG_ETIMEOUT", "CG_EBUSY",
                              "CG_EKERNEL"]):
        assert cg.cg_status_str(i) == name


def test_struct_layouts_match_header(tmp_path):
    src = tmp_path / "layout.c"
    fields = [f for f, _ in cg.GraphDesc._fields_]
    body = "\n".join(f'printf("{f} %zu\\n", offsetof(cg_graph_desc, {f}));' for f in fields)
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "cg.h"\nint main(void){\n'
                   f'printf("size %zu\\n", sizeof(cg_graph_desc));\n{body}\n'
                   'printf("stats %zu %zu\\n", sizeof(cg_stats), offsetof(cg_stats, stage_ms));\nreturn 0;}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = dict(l.split(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                         check=True).stdout.strip().splitlines())
    assert int(out["size"]) == ctypes.sizeof(cg.GraphDesc)
    for f in fields:
        assert int(out[f]) == getattr(cg.GraphDesc, f).offset, f
    s, o = out["stats"].split()
    assert ctypes.sizeof(cg.Tuning) == 16
    assert int(s) == ctypes.sizeof(cg.Stats) and int(o) == cg.Stats.stage_ms.offset


def test_no_gpu_here_reports_cuda_error(libpath):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(cg.CgError) as e:
        cg.cg_create(0)
    assert e.value.status == cg.CG_ECUDA


def test_binding_checks_before_the_library():
    """An argument check of the binding that runs before any library call: a
    part assignment must be int32 (numpy or torch)."""
    import numpy as np
    with pytest.raises(ValueError):
        cg.cg_emit_part(None, np.zeros(4, np.int64), 0)
    with pytest.raises(ValueError):
        cg.cg_emit_part(None, np.zeros(4, np.float32), 0)
    try:
        import torch
    except ImportError:
        return
    t = torch.zeros(4, dtype=torch.int64)          # a host tensor of the wrong type
    with pytest.raises(ValueError):
        cg.cg_emit_part(None, t, 0)
