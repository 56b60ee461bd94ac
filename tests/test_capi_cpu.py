"""Host-side checks of the C-ABI library (no GPU needed).

The library is compiled here for sm_103a; these tests load it, check that it
exports every entry point include/dns.h declares, and exercise the argument
validation and error reporting that run before any device work.
"""

import ctypes
import os
import re

import pytest

from paper_1602_03638_gb300 import _lib
from paper_1602_03638_gb300 import build as B

HEADER_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")


@pytest.fixture(scope="module")
def L():
    B.build()
    return _lib.lib()


def _declared(header):
    with open(os.path.join(HEADER_DIR, header)) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dns_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared("dns.h")
    for need in ("dns_create", "dns_set_state", "dns_step", "dns_get_state", "dns_diagnostics", "dns_destroy"):
        assert need in names


def test_library_exports_every_declared_symbol(L):
    for header in sorted(os.listdir(HEADER_DIR)):
        if header.endswith(".h"):
            for name in _declared(header):
                assert hasattr(L, name), f"{name} declared in {header} but not exported"


def test_binding_covers_the_header(L):
    assert set(_declared("dns.h")) <= set(_lib.SIGNATURES)


def test_argument_validation_without_device(L):
    h = ctypes.c_void_p()
    assert L.dns_create(10, 0.01, 0.01, 0, ctypes.byref(h)) == _lib.DNS_ERR_ARG
    assert "N = 10" in _lib.last_error()
    assert L.dns_create(32, -1.0, 0.01, 0, ctypes.byref(h)) == _lib.DNS_ERR_ARG
    assert L.dns_create(32, 0.01, 0.0, 0, ctypes.byref(h)) == _lib.DNS_ERR_ARG
    assert L.dns_create(32, 0.01, 0.01, 7, ctypes.byref(h)) == _lib.DNS_ERR_ARG
    assert L.dns_create(32, 0.01, 0.01, 0, None) == _lib.DNS_ERR_ARG
    assert L.dns_step(None, 1) == _lib.DNS_ERR_ARG
    assert L.dns_diagnostics(None, None) == _lib.DNS_ERR_ARG
    assert L.dns_set_option(None, b"nu", 0.1) == _lib.DNS_ERR_ARG
    coef = (ctypes.c_double * 3)(0.0, 1.0, 2.0)
    assert L.dns_set_rk_tableau(None, 1, 3, coef, coef) == _lib.DNS_ERR_ARG
    assert L.dns_destroy(None) == _lib.DNS_OK
    assert L.dns_device_bytes(None) == 0
    assert L.dns_debug_fail_alloc_after(-1) == _lib.DNS_ERR_ARG
    assert L.dns_debug_fail_alloc_after(0) == _lib.DNS_OK
    v = ctypes.c_double()
    assert L.dns_get_option(None, b"nu", ctypes.byref(v)) == _lib.DNS_ERR_ARG
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    assert L.dns_tune_tiles(None, 5, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)) == _lib.DNS_ERR_ARG


def test_create_reports_missing_device_instead_of_crashing(L):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    h = ctypes.c_void_p()
    rc = L.dns_create(32, 0.01, 0.01, 0, ctypes.byref(h))
    assert rc == _lib.DNS_ERR_UNSUPPORTED
    assert h.value is None
    assert _lib.last_error()


def test_product_path_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(B, "library_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="missing"):
        _lib.lib()


def test_supported_sizes_match_the_instances():
    sizes = sorted({n for _, _, n in B.instances()})
    assert sizes == [8, 12, 16, 24, 32, 48, 64, 96, 128, 256, 512, 1024]
    with open(os.path.join(HEADER_DIR, "dns.h")) as f:
        assert "8, 12, 16, 24, 32, 48, 64, 96, 128, 256, 512, 1024" in f.read()


def test_tune_cache_file_lookup(tmp_path, L):
    """The tune cache's text format (dns_set_tune_cache): later entries win, malformed and
    foreign lines are ignored, and an unwritable path is refused. Host only."""
    from paper_1602_03638_gb300 import set_tune_cache, tune_cache_lookup

    path = tmp_path / "tune.txt"
    path.write_text(
        "tiles GB300 32 32 32 f32 8 4 16 5\n"
        "tiles GB300 32 32 32 f32 16 4 8 9\n"     # later line wins
        "tiles GB300 48 48 48 f64 0 0 4 x\n"      # malformed value: ignored
        "tiles GB300 256 256 256 f32 0 0 0 0\n"
        "tiles GB300 64 64 64 f32 4 4\n"          # too few values: ignored
        "tiles Other 32 32 32 f32 4 4 4 1\n"      # another device
        "ensemble GB300 f32 32:2,48:1 0 4\n"
        "garbage\n")
    try:
        set_tune_cache(path)
        assert tune_cache_lookup("GB300", 32, "f32") == {"y_inverse": 16, "y_forward": 4, "z": 8, "plan": 9}
        assert tune_cache_lookup("GB300", 256, "f32") == {"y_inverse": 0, "y_forward": 0, "z": 0, "plan": 0}
        assert tune_cache_lookup("GB300", 64, "f32") is None
        assert tune_cache_lookup("GB300", (32, 32, 32), "f64") is None
        assert tune_cache_lookup("GB300", 48, "f64") is None
        assert tune_cache_lookup("Other", 32, "f32")["plan"] == 1
        set_tune_cache(None)
        assert tune_cache_lookup("GB300", 32, "f32") is None  # cache off
        with pytest.raises(_lib.DnsError):
            set_tune_cache(tmp_path / "no_such_dir" / "tune.txt")
    finally:
        set_tune_cache(None)
    a = ctypes.c_int()
    assert L.dns_tune_cache_lookup(None, 32, 32, 32, 0, ctypes.byref(a), ctypes.byref(a), ctypes.byref(a),
                                   ctypes.byref(a)) == _lib.DNS_ERR_ARG
