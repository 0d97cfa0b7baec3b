"""The C ABI library loads and exports every function include/vpmps.h declares (CPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "vpmps.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = "\n".join(l for l in text.splitlines() if not l.lstrip().startswith("typedef"))
    names = re.findall(r"^[A-Za-z_][\w \*]*?\b(\w+)\s*\(", text, flags=re.M)
    return sorted({n for n in names if not n.startswith(("typedef", "VP_"))} - {"if", "return"})


def test_header_declares_the_entry_points():
    names = declared_functions()
    for required in ("mps_create", "mps_apply_mpo", "mps_compress", "vp_density", "vp_poisson", "vp_step", "vp_run"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2205_11990_gb300 import build as B
    from paper_2205_11990_gb300 import vpmps
    try:
        B.build()
    except RuntimeError as e:  # no nvcc in this environment
        pytest.skip(str(e))
    lib = ctypes.CDLL(vpmps.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(vpmps.EXPORTS) <= set(declared_functions())


def test_binding_fails_loudly_without_a_device():
    import torch
    from paper_2205_11990_gb300 import vpmps
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(vpmps.VpError):
        vpmps.Context()
