"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, exports every function the header declares, and its entry
points fail cleanly (no crash) when called with invalid arguments or
without a device."""
import ctypes
import subprocess
import sys

import pytest

from paper_1608_03984_gb300 import build, fdwave


@pytest.fixture(scope="module")
def L():
    build.build()
    return fdwave.lib()


def test_exports_every_declared_symbol(L):
    names = fdwave.declared_symbols()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    # the binding declares exactly the header's functions
    assert sorted(fdwave._SIGS) == names


def test_version_string(L):
    assert b"sm_103a" in L.fdw_version()


def test_invalid_arguments_fail_cleanly(L):
    h = ctypes.c_void_p()
    # bad order / sizes / storage are rejected before any device call
    assert L.fdw_create(ctypes.byref(h), 10, 10, 10, 10.0, 2, 0, 3, 0, None) == -1
    assert L.fdw_create(ctypes.byref(h), 10, 10, 10, 10.0, 2, 0, 18, 0, None) == -1
    assert L.fdw_create(ctypes.byref(h), 0, 10, 10, 10.0, 2, 0, 4, 0, None) == -1
    assert L.fdw_create(ctypes.byref(h), 10, 10, 10, -1.0, 2, 0, 4, 0, None) == -1
    assert L.fdw_create(ctypes.byref(h), 10, 10, 10, 10.0, 2, 7, 4, 0, None) == -1
    assert L.fdw_create(ctypes.byref(h), 10, 10, 10, 10.0, 2, 0, 4, 9, None) == -1
    assert L.fdw_create(None, 10, 10, 10, 10.0, 2, 0, 4, 0, None) == -1
    assert b"order" in L.fdw_last_error() or b"NULL" in L.fdw_last_error()
    # NULL solver handles
    assert L.fdw_step(None, 1) == -1
    assert L.fdw_set_dt(None, 1e-3) == -1
    assert L.fdw_destroy(None) == 0
    assert L.fdw_max_stable_dt(None) < 0
    assert L.fdw_current_step(None) == -1


def test_no_device_is_an_error_not_a_crash():
    """Run in a subprocess with no visible GPU: create must return an error."""
    code = ("import ctypes,sys; sys.path.insert(0, %r);"
            "from paper_1608_03984_gb300 import fdwave as F; L=F.lib();"
            "h=ctypes.c_void_p(); rc=L.fdw_create(ctypes.byref(h),8,8,8,10.0,2,0,4,0,None);"
            "print(rc)" % fdwave._build.ROOT)
    env = dict(__import__("os").environ, CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                         timeout=300)
    assert out.returncode == 0, out.stderr
    assert int(out.stdout.strip().splitlines()[-1]) in (-3, -4), out.stdout
