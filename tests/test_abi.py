"""The C-ABI library builds for sm_103a, loads, exports every entry point that
include/copula.h declares, and validates partitions on the host (no GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1609_05530_gb300 as cg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "copula.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(copula_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = cg.lib()
    names = _declared()
    assert "copula_fit" in names and "copula_fit_batch" in names and len(names) >= 12
    for n in names:
        assert hasattr(L, n), n


def test_library_is_built_for_sm103a_only():
    from paper_1609_05530_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.exists(cg.library_path())


def _ws(off, dtype=cg.DTYPE_F32, precision="f32c"):
    off = np.ascontiguousarray(off, dtype=np.int64)
    o = cg.Opts()
    cg.lib().copula_opts_default(ctypes.byref(o))
    o.precision = cg.PRECISIONS[precision]
    nb = ctypes.c_size_t()
    rc = cg.lib().copula_fit_workspace_size(None, dtype, ctypes.byref(o), off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                            off.shape[0] - 1, ctypes.byref(nb))
    return rc, nb.value


def test_partition_validation_on_host():
    assert _ws([0, 1000, 2000])[0] == 0
    assert _ws([0, 1, 2000])[0] == -1           # subset of size 1
    assert _ws([0, 1000, 1000, 2000])[0] == -1  # empty subset
    assert _ws([0, 1500, 1000])[0] == -1        # not increasing
    assert _ws([5, 1000])[0] == -1              # does not start at 0
    assert _ws([0, cg.MAX_SUBSET])[0] == 0
    assert _ws([0, cg.MAX_SUBSET_F64], cg.DTYPE_F64)[0] == 0
    # beyond one thread block: the streaming path, up to its own limit
    r_res, b_res = _ws([0, cg.MAX_SUBSET])
    r_str, b_str = _ws([0, cg.MAX_SUBSET + 1])
    assert r_str == 0 and b_str > b_res
    assert _ws([0, cg.MAX_SUBSET_STREAM])[0] == 0
    assert _ws([0, cg.MAX_SUBSET_STREAM + 1])[0] == -4  # larger than the library fits
    assert _ws([0, cg.MAX_SUBSET_F64 + 1], cg.DTYPE_F64)[0] == 0
    assert _ws([0, cg.MAX_SUBSET_STREAM_F64], cg.DTYPE_F64)[0] == 0
    assert _ws([0, cg.MAX_SUBSET_STREAM_F64 + 1], cg.DTYPE_F64)[0] == -4


def test_header_limits_match_binding():
    hdr = open(os.path.join(ROOT, "include", "copula.h")).read()
    for name in ("MAX_SUBSET", "MAX_SUBSET_F64", "MAX_SUBSET_STREAM", "MAX_SUBSET_STREAM_F64"):
        m = re.search(r"#define COPULA_%s (\d+)" % name, hdr)
        assert m and int(m.group(1)) == getattr(cg, name), name


def test_workspace_grows_with_n_and_precision():
    r1, a = _ws(np.arange(0, 10_001, 1000))
    r2, b = _ws(np.arange(0, 100_001, 1000))
    r3, c = _ws(np.arange(0, 100_001, 10_000), precision="f64")
    assert r1 == r2 == r3 == 0
    assert 0 < a < b and c > 0


def test_product_path_never_touches_the_oracle():
    pkg = os.path.join(ROOT, "paper_1609_05530_gb300")
    for dp, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                txt = open(os.path.join(dp, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "liboracle" not in txt, f
