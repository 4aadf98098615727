"""The C-ABI library: it builds, loads, exports every declared symbol, and
rejects bad arguments on the host before touching the device (CPU only:
no call here launches a kernel or allocates device memory)."""
from __future__ import annotations

import ctypes as C
import glob
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2508_15967_gb300 as gf
from paper_2508_15967_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libgf():
    B.build()
    return gf.lib()


def declared_functions() -> list[str]:
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(gf_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(libgf):
    names = declared_functions()
    assert "gf_trace_rk4" in names and "gf_medium_create" in names
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (gf_[a-z0-9_]+)$", out, flags=re.M))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(libgf, n)


def test_version_and_empty_error(libgf):
    assert libgf.gf_version() >= 100
    assert isinstance(libgf.gf_last_error(), bytes)


def test_medium_create_rejects_bad_descriptions(libgf):
    h = C.c_void_p()
    assert libgf.gf_medium_create(None, C.byref(h)) == gf.GF_ERR_INVALID_ARG
    bad = [
        gf.GfMediumDesc(99, 0, 0, 0, 1.0, 1.5, 2.0, None, None),            # kind
        gf.GfMediumDesc(0, 0, 0, 7, 1.0, 1.5, 2.0, None, None),             # reserved
        gf.GfMediumDesc(0, 0, 0, 0, -1.0, 1.5, 2.0, None, None),            # n_h <= 0
        gf.GfMediumDesc(1, 65, 0, 0, 1.0, 1.5, 2.0, None, None),            # too many blobs
        gf.GfMediumDesc(1, 2, 0, 0, 1.0, 1.5, 2.0, None, None),             # blobs missing
        gf.GfMediumDesc(4, 0, 2, 0, 1.0, 1.5, 2.0, None, None),             # grid missing / small
    ]
    for d in bad:
        assert libgf.gf_medium_create(C.byref(d), C.byref(h)) == gf.GF_ERR_INVALID_ARG
        assert libgf.gf_last_error()
    blobs = np.array([[0.1, 0, 0, 0, 0.0]])                                 # zero width
    d = gf.GfMediumDesc(1, 1, 0, 0, 1.0, 1.5, 2.0, blobs.ctypes.data, None)
    assert libgf.gf_medium_create(C.byref(d), C.byref(h)) == gf.GF_ERR_INVALID_ARG
    assert b"width" in libgf.gf_last_error()


def test_calls_with_null_medium_or_rays_fail_cleanly(libgf):
    rays = gf.GfRays(1, 1, None, None, None, None, None, None)
    assert libgf.gf_trace_rk4(None, gf.GF_F64, C.byref(rays), 1.0, 1e-3, 10, 0.0, 0, None, None) \
        == gf.GF_ERR_INVALID_ARG
    assert b"medium" in libgf.gf_last_error()
    assert libgf.gf_rays_onshell(None, gf.GF_F64, C.byref(rays), None, 1.0, None) == gf.GF_ERR_INVALID_ARG
    assert libgf.gf_medium_set_amplitudes(None, None, None) == gf.GF_ERR_INVALID_ARG
    assert libgf.gf_medium_destroy(None) == gf.GF_OK


def test_binding_raises_with_message(libgf):
    with pytest.raises(gf.GfError, match="unknown kind|n_h"):
        gf.gf_medium_create("homog", n_h=0.0)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(gf, "_lib", None)
    monkeypatch.setattr(gf, "LIB_PATH", str(tmp_path / "libgf.so"))
    with pytest.raises(RuntimeError, match="libgf.so not found"):
        gf.lib()


def test_fault_injection_and_allocation_count_on_the_host(libgf):
    """The failure-testing hooks are host-only: arming and disarming touch no
    device, and a process that has created nothing holds no allocation."""
    assert libgf.gf_fault_inject(C.c_int64(5)) == gf.GF_OK
    assert libgf.gf_fault_inject(C.c_int64(0)) == gf.GF_OK
    assert libgf.gf_fault_inject(C.c_int64(-3)) == gf.GF_OK
    n, nbytes = gf.gf_bench_live_allocations()
    assert n >= 0 and nbytes >= 0
