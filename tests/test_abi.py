"""The C ABI: liblpb.so loads and exports every function include/lpb.h declares, and the
ctypes structures of the binding have the header's layout.  No GPU needed."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lpb.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lpb_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no CUDA toolkit")
    from paper_1609_08114_gb300 import build
    return build.build()


def test_every_declared_symbol_is_exported(lib_path):
    names = _declared()
    assert "lpb_solve" in names and "lpb_hyperbox" in names and len(names) >= 10
    lib = ctypes.CDLL(lib_path)
    for name in names:
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (lpb_\w+)", out))
    assert set(names) <= exported


def test_binding_declares_every_symbol():
    from paper_1609_08114_gb300 import _lib
    assert set(_declared()) == set(_lib.SIGNATURES)


def test_host_only_calls(lib_path):
    from paper_1609_08114_gb300 import _lib
    lib = _lib.load()
    assert b"liblpb" in lib.lpb_version()
    assert lib.lpb_strerror(_lib.ENOMEM) == b"workspace too small"
    assert lib.lpb_create(None, 0) == _lib.EINVAL       # NULL handle pointer rejected on the host
    assert lib.lpb_destroy(None) == _lib.EINVAL


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_struct_layouts_match_header(tmp_path):
    from paper_1609_08114_gb300 import _lib
    prog = tmp_path / "layout.c"
    checks = {
        "lpb_batch": (_lib.Batch, ["count", "max_m", "max_n", "dtype", "m", "n", "a_off", "b_off", "c_off", "A", "b", "c",
                                   "min_m", "min_n"]),
        "lpb_result": (_lib.Result, ["status", "iters", "obj", "x", "y", "basis"]),
        "lpb_options": (_lib.Options, ["prec", "max_iter", "eps_p", "eps_d", "feas_tol", "keep_basis_inverse",
                                       "kernel", "threads", "reg_warps", "pivot_rule", "seed"]),
        "lpb_stats": (_lib.Stats, ["resolved_fp64", "deferred", "kernels", "reserved"]),
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lpb.h"', "int main(void){"]
    for cname, (_, fields) in checks.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f in fields:
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0;}")
    prog.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for cname, (cls, fields) in checks.items():
        assert int(got[cname]) == ctypes.sizeof(cls), cname
        for f in fields:
            assert int(got[f"{cname}.{f}"]) == getattr(cls, f).offset, (cname, f)


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_enum_values_match_header(tmp_path):
    """Every constant of the binding equals the header's enumerator of the same name."""
    from paper_1609_08114_gb300 import _lib
    names = ["OPTIMAL", "INFEASIBLE", "UNBOUNDED", "ITER_LIMIT", "NUMERIC", "BAD_SIZE",
             "OK", "EINVAL", "ENOMEM", "ECUDA", "EUNSUPPORTED", "EDEVICE",
             "FP64", "FP32_REFINE", "FP32", "DTYPE_F32", "DTYPE_F64",
             "KERNEL_AUTO", "KERNEL_SMEM", "KERNEL_GMEM", "KERNEL_REG", "KERNEL_PACK", "KERNEL_WARP",
             "PIVOT_LPC", "PIVOT_RPC", "PIVOT_STEEPEST"]
    prog = tmp_path / "enums.c"
    body = "".join(f'printf("{n} %d\\n", (int)LPB_{n});' for n in names)
    prog.write_text('#include <stdio.h>\n#include "lpb.h"\nint main(void){' + body + "return 0;}")
    exe = tmp_path / "enums"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for n in names:
        assert int(got[n]) == getattr(_lib, n), n
    from paper_1609_08114_gb300 import PIVOT_RULES
    assert PIVOT_RULES == {"lpc": _lib.PIVOT_LPC, "rpc": _lib.PIVOT_RPC, "steepest": _lib.PIVOT_STEEPEST}


def test_batch_size_hints():
    """LPBatch carries the host size hints the planner uses (min = max: one size class)."""
    import numpy as np
    import torch
    from paper_1609_08114_gb300 import LPBatch
    m, n = np.array([3, 5, 4]), np.array([2, 2, 6])
    A = np.ones(int((m * n).sum())); b = np.ones(int(m.sum())); c = np.ones(int(n.sum()))
    bt = LPBatch.from_packed(m, n, A, b, c, device="cpu")
    assert (bt.max_m, bt.max_n, bt.min_m, bt.min_n) == (5, 6, 3, 2)
    cs = bt.cstruct()
    assert (cs.max_m, cs.max_n, cs.min_m, cs.min_n) == (5, 6, 3, 2)
    d = LPBatch.from_dense(torch.ones(4, 7, 3, dtype=torch.float64), torch.ones(4, 7, dtype=torch.float64),
                           torch.ones(4, 3, dtype=torch.float64))
    assert (d.max_m, d.max_n, d.min_m, d.min_n) == (7, 3, 7, 3)
