"""The C-ABI library loads and exports every symbol include/arnold.h declares.

No compute calls: these run without a GPU (argument validation and host
fault injection happen before any CUDA call)."""
import ctypes
import os
import re
import subprocess
import sys

import pytest

from paper_1107_4107_b300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "arnold.h")


@pytest.fixture(scope="module")
def L():
    build.build()
    return _lib.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(arnold_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("arnold_create", "arnold_iterate", "arnold_indicator", "arnold_destroy",
                     "arnold_set_state", "arnold_init_grid", "arnold_stats_compute", "arnold_sync"):
        assert required in names


def test_every_declared_symbol_is_exported(L):
    out = subprocess.check_output(["nm", "-D", "--defined-only", _lib.LIB_PATH]).decode()
    exported = set(re.findall(r"\bT (arnold_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(L, n)


def test_binding_covers_the_header():
    assert set(declared_functions()) <= set(_lib.SIGNATURES)


def test_params_default_and_strerror(L):
    p = _lib.Params()
    L.arnold_params_default(ctypes.byref(p))
    assert p.eps == 1.0 and abs(p.h - 0.02 * 3.141592653589793) < 1e-15
    assert p.scheme == 0 and p.precision == 0 and p.tangent == 1 and p.renorm_every == 100
    assert p.chaos_kappa == 10.0
    assert _lib.strerror(_lib.EINVAL) == "invalid argument"
    assert _lib.strerror(12345) == "unknown status"


def _create(L, p, n=16):
    h = ctypes.c_void_p()
    return L.arnold_create(ctypes.byref(p), n, 0, None, ctypes.byref(h)), h


def test_create_rejects_bad_arguments_before_cuda(L):
    base = _lib.Params()
    L.arnold_params_default(ctypes.byref(base))
    bad = []
    for field, val in (("h", 0.0), ("scheme", 7), ("precision", 4), ("renorm_every", 0), ("window", -1),
                       ("chaos_kappa", 0.0), ("block_size", 48), ("tangent", 2), ("megno", 2),
                       ("reserved", 1)):
        p = _lib.Params.from_buffer_copy(base)
        setattr(p, field, val)
        bad.append(p)
    for p in bad:
        rc, h = _create(L, p)
        assert rc == _lib.EINVAL and not h.value
    rc, _ = _create(L, base, n=0)
    assert rc == _lib.EINVAL
    # MEGNO is a tangent indicator: megno = 1 with the tangent off is rejected
    p = _lib.Params.from_buffer_copy(base)
    p.megno, p.tangent = 1, 0
    rc, h = _create(L, p)
    assert rc == _lib.EINVAL and not h.value


def test_params_struct_matches_the_header():
    """The ctypes mirror has the C layout: 8 + 8 + 4 * 4 + 8 + 8 + 4 * 4 bytes."""
    assert ctypes.sizeof(_lib.Params) == 64
    assert _lib.Params.megno.offset == 56 and _lib.Params.reserved.offset == 60


def test_alloc_fault_injection_on_host():
    """ARNOLD_FAULT=alloc makes create fail with ENOMEM before touching CUDA."""
    code = ("import ctypes; from paper_1107_4107_b300 import _lib; L=_lib.lib(); p=_lib.Params();"
            "L.arnold_params_default(ctypes.byref(p)); h=ctypes.c_void_p();"
            "print(L.arnold_create(ctypes.byref(p), 8, 0, None, ctypes.byref(h)), h.value)")
    env = dict(os.environ, ARNOLD_FAULT="alloc", PYTHONPATH=ROOT)
    out = subprocess.check_output([sys.executable, "-c", code], env=env, cwd=ROOT).decode().split()
    assert int(out[0]) == _lib.ENOMEM and out[1] == "None"


def test_null_handles_are_rejected(L):
    assert L.arnold_iterate(None, 1) == _lib.EINVAL
    assert L.arnold_set_snapshots(None, None, 0) == _lib.EINVAL
    assert L.arnold_sync(None) == _lib.EINVAL
    assert L.arnold_steps_done(None) == -1
    L.arnold_destroy(None)
