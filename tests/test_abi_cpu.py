"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/rtc.h declares; host-side argument checks fail cleanly without a GPU."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = []
    for hp in HEADERS:
        text = open(hp).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b(rtc_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1805_07254_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["rtc_create", "rtc_destroy", "rtc_load_calib", "rtc_load_cmat",
                     "rtc_process_frame", "rtc_last_error", "rtc_load_subaps"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_1805_07254_gb300.rtc import SIGNATURES
    assert sorted(SIGNATURES) == declared_functions()


def test_exports_are_c_symbols(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(rtc_\w+)\b", out))
    assert set(declared_functions()) <= exported


def test_create_rejects_bad_config_without_device(lib):
    from paper_1805_07254_gb300.rtc import Rtc, RtcError, RTC_EINVAL
    with pytest.raises(RtcError) as e:
        Rtc(nsub=0, npx=10, nact=5)
    assert e.value.code == RTC_EINVAL
    with pytest.raises(RtcError):
        Rtc(nsub=8, npx=8, nact=69, thr_mode=3)
    with pytest.raises(RtcError):
        Rtc(nsub=8, npx=8, nact=69, obs=1.5)


def test_version_string(lib):
    from paper_1805_07254_gb300 import version
    assert "sm_103a" in version()


def test_null_handle_calls_return_einval(lib):
    from paper_1805_07254_gb300.rtc import load_library
    L = load_library()
    assert L.rtc_destroy(None) == 0
    assert L.rtc_set_gain(None, 0.4, 0.99) == -1
    assert L.rtc_process_frame(None, None, None, None) == -1
    assert L.rtc_reset(None) == -1
