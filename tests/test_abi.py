"""The C-ABI library builds, loads and exports every function include/hlbm.h declares; the
ctypes mirror of lbm_config has the C layout; invalid configurations are rejected with
LBM_ERR_ARG before any CUDA call (no GPU needed)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hlbm.h")


@pytest.fixture(scope="module")
def L():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2207_11567_gb300 import _lib
    return _lib


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L.lib, n), n
    assert set(names) == set(L.EXPORTED)


def test_config_layout_matches_header(L, tmp_path):
    fields = ["dim", "storage", "bc_lo", "thermal", "dx", "nu_ref", "P_ref", "omega_hi", "thicken_F",
              "flame_sensor", "sensor_Ta", "closed_domain", "sp", "rx", "T_in", "Y_in", "stream", "alloc", "alloc_user"]
    src = tmp_path / "probe.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "hlbm.h"\nint main(void){\n'
                   '  printf("size %zu\\n", sizeof(lbm_config));\n'
                   + "".join(f'  printf("{f} %zu\\n", offsetof(lbm_config, {f}));\n' for f in fields)
                   + '  printf("reaction %zu\\n", sizeof(lbm_reaction));\n  return 0;\n}\n')
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines())
    assert int(out["size"]) == C.sizeof(L.Config)
    assert int(out["reaction"]) == C.sizeof(L.Reaction)
    for f in fields:
        assert int(out[f]) == getattr(L.Config, f).offset, f


@pytest.mark.parametrize("mutate,msg", [
    (lambda c: setattr(c, "dim", 4), "dim"),
    (lambda c: setattr(c, "nx", 0), "grid"),
    (lambda c: c.bc_hi.__setitem__(0, 2), "inlet"),
    (lambda c: setattr(c, "dx", -1.0), "dx"),
    (lambda c: setattr(c, "closed_domain", 1), "closed_domain"),
    (lambda c: setattr(c, "storage", 7), "storage"),
])
def test_invalid_configurations_are_rejected(L, mutate, msg):
    import workloads as W
    cfg = L.config_from_dict(W.generate.box(2, 8).cfg)
    mutate(cfg)
    ctx = C.c_void_p()
    st = L.lib.lbm_init(C.byref(cfg), C.byref(ctx))
    assert st == L.LBM_ERR_ARG
    assert msg in L.lib.lbm_last_error(ctx).decode()
    L.lib.lbm_destroy(ctx)


def test_null_arguments(L):
    assert L.lib.lbm_init(None, None) == L.LBM_ERR_ARG
    assert L.lib.lbm_step(None, 1) == L.LBM_ERR_ARG


def test_package_without_the_library_fails_loudly(tmp_path):
    """A copy of the package without libhlbm.so does not import (no CPU path to fall back to)."""
    import shutil
    import sys
    src = os.path.join(ROOT, "paper_2207_11567_gb300")
    dst = tmp_path / "paper_2207_11567_gb300"
    shutil.copytree(src, dst, ignore=shutil.ignore_patterns("*.so", "_build", "__pycache__"))
    r = subprocess.run([sys.executable, "-c", "import paper_2207_11567_gb300"], cwd=tmp_path,
                       capture_output=True, text=True)
    assert r.returncode != 0 and "libhlbm.so is missing" in r.stderr
