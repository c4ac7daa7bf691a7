"""Host-side fault injection without a GPU: the spec parser, arming and
disarming, and the SNSOLVE_FAULT environment variable.  The failures the armed
faults cause are checked on the GPU (tests/test_gpu_fault.py); nothing here
launches a kernel."""
import ctypes as C
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NONE, ALLOC, LAUNCH, TIMEOUT = 0, 1, 2, 3


@pytest.fixture()
def lib():
    from paper_2409_14309_gb300 import abi
    if not os.path.exists(abi.LIB_PATH):
        from paper_2409_14309_gb300 import build
        build.build()
    L = abi.lib()
    yield L
    assert L.snsolve_debug_set_fault(None) == abi.SNS_OK      # leave the process disarmed


def armed(L):
    left = C.c_int64(-1)
    k = L.snsolve_debug_fault_armed(C.byref(left))
    return k, left.value


@pytest.mark.parametrize("spec, want", [
    (b"alloc", (ALLOC, 1)), (b"launch", (LAUNCH, 1)), (b"timeout", (TIMEOUT, 1)),
    (b"launch:7", (LAUNCH, 7)), (b"alloc:1", (ALLOC, 1)), (b"timeout:123456789012", (TIMEOUT, 123456789012)),
])
def test_valid_specs_arm(lib, spec, want):
    from paper_2409_14309_gb300 import abi
    assert lib.snsolve_debug_set_fault(spec) == abi.SNS_OK
    assert armed(lib) == want


@pytest.mark.parametrize("spec", [b"alloc:0", b"launch:-2", b"launch:", b"launch:x", b"launch:3x", b"Alloc",
                                  b"allocx", b"time", b"launch:1:2", b":3", b" alloc"])
def test_invalid_specs_are_rejected_and_change_nothing(lib, spec):
    from paper_2409_14309_gb300 import abi
    assert lib.snsolve_debug_set_fault(b"timeout:4") == abi.SNS_OK
    assert lib.snsolve_debug_set_fault(spec) == abi.SNS_EINVAL
    assert armed(lib) == (TIMEOUT, 4)


@pytest.mark.parametrize("spec", [None, b"", b"none"])
def test_empty_spec_disarms(lib, spec):
    from paper_2409_14309_gb300 import abi
    assert lib.snsolve_debug_set_fault(b"alloc:2") == abi.SNS_OK
    assert lib.snsolve_debug_set_fault(spec) == abi.SNS_OK
    assert armed(lib) == (NONE, 0)


def test_rearming_replaces_the_previous_fault(lib):
    lib.snsolve_debug_set_fault(b"alloc:5")
    lib.snsolve_debug_set_fault(b"launch:2")
    assert armed(lib) == (LAUNCH, 2)


def _armed_in_child(env_value):
    code = ("import ctypes as C, sys; sys.path.insert(0, %r)\n"
            "from paper_2409_14309_gb300 import abi\n"
            "L = abi.lib(); left = C.c_int64(-1)\n"
            "print(L.snsolve_debug_fault_armed(C.byref(left)), left.value)\n") % ROOT
    env = dict(os.environ)
    env.pop("SNSOLVE_FAULT", None)
    if env_value is not None:
        env["SNSOLVE_FAULT"] = env_value
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    k, left = out.stdout.split()
    return int(k), int(left)


def test_environment_variable_arms_at_first_check(lib):
    assert _armed_in_child("launch:3") == (LAUNCH, 3)
    assert _armed_in_child("alloc") == (ALLOC, 1)
    assert _armed_in_child(None) == (NONE, 0)
    assert _armed_in_child("bogus") == (NONE, 0)          # unparsable: nothing armed
