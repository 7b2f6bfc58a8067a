"""The C-ABI library loads and exports every entry point include/lqcd.h declares; the ctypes
structures match the C layout (checked by compiling a probe against the header with gcc)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2609_37049_b300 import lqcd

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
HEADER = os.path.join(ROOT, "include", "lqcd.h")


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(lqcd_\w+)\s*\(", text, re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["lqcd_gauge_upload", "lqcd_dirac_apply", "lqcd_solve_full", "lqcd_solve_domain",
              "lqcd_perambulator", "lqcd_loops", "lqcd_disc_correlator"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(os.path.join(ROOT, "paper_2609_37049_b300", "liblqcd.so"))
    for n in declared_functions():
        assert hasattr(lib, n), n
    assert set(declared_functions()) <= set(lqcd.EXPORTED) | {"lqcd_default_params"}


def test_struct_layout_matches_header(tmp_path):
    src = tmp_path / "probe.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "lqcd.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu\\n", sizeof(lqcd_solve_params),'
                   ' sizeof(lqcd_solve_stats), offsetof(lqcd_solve_params, projection),'
                   ' offsetof(lqcd_solve_stats, device_loops)); printf("%zu\\n",'
                   ' offsetof(lqcd_solve_params, residual)); return 0;}\n')
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    assert int(out[0]) == ctypes.sizeof(lqcd.lqcd_solve_params)
    assert int(out[1]) == ctypes.sizeof(lqcd.lqcd_solve_stats)
    assert int(out[2]) == lqcd.lqcd_solve_params.projection.offset
    assert int(out[3]) == lqcd.lqcd_solve_stats.device_loops.offset
    assert int(out[4]) == lqcd.lqcd_solve_params.residual.offset


def test_default_params():
    p = lqcd.default_params()
    assert p.tol == 1e-10 and p.solver == lqcd.LQCD_SOLVER_BICGSTAB64 and p.use_graph == 1


def test_invalid_create_rejected_without_gpu_work():
    h = ctypes.c_void_p()
    L = (ctypes.c_int * 4)(4, 4, 3, 8)  # odd extent
    assert lqcd.lib().lqcd_create(ctypes.byref(h), L, 1, None) == lqcd.LQCD_ERR_INVALID_ARG
    assert b"even" in lqcd.lib().lqcd_last_error(None)
    L = (ctypes.c_int * 4)(4, 4, 4, 512)
    assert lqcd.lib().lqcd_create(ctypes.byref(h), L, 1, None) == lqcd.LQCD_ERR_INVALID_ARG


def test_numpy_marshalling_checks():
    import numpy as np
    with pytest.raises(ValueError):
        lqcd._ptr(np.zeros(4, dtype=np.float64))
    assert lqcd._where(np.zeros(2, dtype=complex)) == lqcd.LQCD_HOST


def test_missing_library_fails_loudly(tmp_path):
    """No CPU fallback: without the built library the binding raises instead of computing."""
    with pytest.raises(ImportError):
        lqcd.load_library(str(tmp_path / "liblqcd.so"))


def test_product_never_imports_the_oracle():
    """The package (binding, autotuner, sharding, build script) has no route to the oracle."""
    pkg = os.path.join(ROOT, "paper_2609_37049_b300")
    for name in os.listdir(pkg):
        if name.endswith(".py"):
            text = open(os.path.join(pkg, name)).read()
            assert not re.search(r"^\s*(from|import)\s+oracle\b", text, re.M), name
