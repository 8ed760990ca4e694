"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
function that include/*.h declares (no compute calls here)."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\([^;{]*\)\s*;", text,
                             flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def cudalib():
    from paper_2302_07411_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_headers_declare_the_boundary():
    names = declared_functions()
    for required in ("enc_init", "encrypt_frames", "decrypt_frames", "crypt_frames_host", "enc_save_state",
                     "enc_load_state", "enc_sync_status", "enc_destroy", "vc_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(cudalib):
    missing = [n for n in declared_functions() if not hasattr(cudalib, n)]
    assert not missing, missing


def test_status_strings(cudalib):
    cudalib.vc_strerror.restype = ctypes.c_char_p
    assert cudalib.vc_strerror(0) == b"ok"
    assert b"layout" in cudalib.vc_strerror(3)


def test_argument_validation_without_gpu(cudalib):
    """Null arguments are rejected before any CUDA call."""
    from paper_2302_07411_gb300 import binding as B

    L = B.lib()
    assert L.enc_init(None, None, None) == 1
    assert L.encrypt_frames(None, None, None, 1, None) == 1
    assert L.enc_set_chunk(None, 4) == 1
    assert L.enc_join(None, None) == 1
    assert L.enc_sync_status(None) == 1


def test_binding_refuses_cpu_tensors():
    torch = pytest.importorskip("torch")
    from paper_2302_07411_gb300 import binding as B

    with pytest.raises(ValueError):
        B._dptr(torch.zeros(4, dtype=torch.uint8))


def header_defines():
    out = {}
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            for m in re.finditer(r"^#define\s+(VC_[A-Z0-9_]+)\s+(-?\d+)\b", open(os.path.join(ROOT, "include", h)).read(),
                                 flags=re.M):
                out[m.group(1)] = int(m.group(2))
    return out


def test_binding_constants_match_the_headers():
    """Every VC_* constant the Python binding exposes has the value the C
    headers define (maps, options, batch options, status codes)."""
    from paper_2302_07411_gb300 import binding as B

    defs = header_defines()
    names = [n for n in dir(B) if n.startswith("VC_") and isinstance(getattr(B, n), int)]
    assert {"VC_PLCM", "VC_2DLASM", "VC_LOGISTIC", "VC_OPT_DIFFUSION"} <= set(names)
    for n in names:
        assert n in defs, f"{n} is not defined in include/*.h"
        assert getattr(B, n) == defs[n], (n, getattr(B, n), defs[n])


def test_bench_maps_are_the_library_maps():
    import importlib.util

    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    defs = header_defines()
    assert bench.MAP_KIND == {"plcm": defs["VC_PLCM"], "2dlasm": defs["VC_2DLASM"], "logistic": defs["VC_LOGISTIC"]}
