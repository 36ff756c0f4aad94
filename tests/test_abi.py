"""The C-ABI library builds, loads without a GPU and exports every entry
point that include/rlgl.h declares; the Python binding covers them all.
No compute call is made here."""
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rlgl.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rlgl_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("rlgl_create", "rlgl_step", "rlgl_solve", "rlgl_estimate", "rlgl_destroy"):
        assert s in syms


def test_library_exports_every_declared_symbol():
    from paper_2008_02710_gb300 import _build
    lib = _build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\sT\s(rlgl_[a-z_]+)", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing


def test_binding_signatures_cover_header():
    from paper_2008_02710_gb300 import rlgl
    assert sorted(rlgl.SIGNATURES) == declared_symbols()
    lib = rlgl.load()
    for s in declared_symbols():
        assert hasattr(lib, s)


def test_host_only_entry_points():
    from paper_2008_02710_gb300 import rlgl
    p = rlgl.default_params()
    assert p.theta_scale == 1.0 and p.r == 1 and p.top_frac == 0.01
    lib = rlgl.load()
    assert lib.rlgl_status_string(5) == b"RLGL_EDEGENERATE"
    with pytest.raises(rlgl.RLGLError):
        rlgl._check(lib, None, lib.rlgl_set_params(None, None))


def test_torch_tensor_with_numpy_dtype_is_converted():
    """A torch tensor passed where the C ABI wants float64 is converted with
    the matching torch dtype (host tensor: host memory space)."""
    torch = pytest.importorskip("torch")
    from paper_2008_02710_gb300 import rlgl
    t = torch.arange(4, dtype=torch.float32)
    p, sp, keep = rlgl._ptr(t, np.float64)
    assert sp == rlgl.HOST and keep.dtype == torch.float64 and p == keep.data_ptr()
    assert keep.tolist() == [0.0, 1.0, 2.0, 3.0]


def _struct_fields(name):
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    body = re.search(r"typedef struct \{([^}]*)\}\s*" + name + r"\s*;", text).group(1)
    return re.findall(r"\b(int32_t|int64_t|uint64_t|double|float)\s+(\w+)(\[\d+\])?\s*;", body)


def test_params_struct_matches_header():
    """The binding's rlgl_params has the header's fields in the header's
    order and types (the struct crosses the ABI by value)."""
    import ctypes
    from paper_2008_02710_gb300 import rlgl
    ctype = {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "uint64_t": ctypes.c_uint64,
             "double": ctypes.c_double, "float": ctypes.c_float}
    want = [(n, ctype[t]) for t, n, _ in _struct_fields("rlgl_params")]
    got = [(n, t) for n, t in rlgl.Params._fields_]
    assert got == want
    p = rlgl.default_params()
    assert p.theta_lag == 0 and p.stall_moves == 32 and p.persistent == 1
