"""ctypes binding of libdns_gb300.so (include/dns.h): argument marshalling only.

Every function of the C ABI is exposed under the same name. The library must
have been built (paper_1602_03638_gb300.build.build()); importing this module
never falls back to anything else -- a missing library raises immediately.
"""

from __future__ import annotations

import ctypes
import os

from . import build as _build

DNS_OK = 0
DNS_ERR_ARG = -1
DNS_ERR_OOM = -2
DNS_ERR_CUDA = -3
DNS_ERR_NONFINITE = -4
DNS_ERR_TIMEOUT = -5
DNS_ERR_UNSUPPORTED = -6
DNS_F32 = 0
DNS_F64 = 1

STATUS_NAMES = {
    DNS_OK: "DNS_OK",
    DNS_ERR_ARG: "DNS_ERR_ARG",
    DNS_ERR_OOM: "DNS_ERR_OOM",
    DNS_ERR_CUDA: "DNS_ERR_CUDA",
    DNS_ERR_NONFINITE: "DNS_ERR_NONFINITE",
    DNS_ERR_TIMEOUT: "DNS_ERR_TIMEOUT",
    DNS_ERR_UNSUPPORTED: "DNS_ERR_UNSUPPORTED",
}


class dns_diag(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("t", "energy", "dissipation", "max_div", "helicity", "enstrophy")]


# name -> (restype, argtypes)
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
SIGNATURES = {
    "dns_create": (_I, [_I, _D, _D, _I, ctypes.POINTER(_P)]),
    "dns_create3": (_I, [_I, _I, _I, _D, _D, _I, ctypes.POINTER(_P)]),
    "dns_destroy": (_I, [_P]),
    "dns_set_stream": (_I, [_P, _P]),
    "dns_set_option": (_I, [_P, ctypes.c_char_p, _D]),
    "dns_get_option": (_I, [_P, ctypes.c_char_p, ctypes.POINTER(_D)]),
    "dns_tune_tiles": (_I, [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "dns_set_tune_cache": (_I, [ctypes.c_char_p]),
    "dns_tune_cache_lookup": (_I, [ctypes.c_char_p, _I, _I, _I, _I, ctypes.POINTER(_I), ctypes.POINTER(_I),
                                   ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "dns_set_rk_tableau": (_I, [_P, _I, _I, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "dns_tile_widths": (_I, [_I, _I, _I, ctypes.POINTER(_I), _I]),
    "dns_set_state": (_I, [_P, _P, _I]),
    "dns_set_state_spectral": (_I, [_P, _P, _I]),
    "dns_step": (_I, [_P, _I]),
    "dns_get_state": (_I, [_P, _P, _I]),
    "dns_get_state_spectral": (_I, [_P, _P, _I]),
    "dns_rhs": (_I, [_P, _P, _I]),
    "dns_diagnostics": (_I, [_P, ctypes.POINTER(dns_diag)]),
    "dns_profile_steps": (_I, [_P, _I, ctypes.POINTER(_D), ctypes.POINTER(_I), _I]),
    "dns_device_bytes": (ctypes.c_size_t, [_P]),
    "dns_last_error": (ctypes.c_char_p, [_P]),
    "dns_debug_fail_alloc_after": (_I, [_I]),
    "dns_spectral_sums_noalloc": (_I, [_P, _I, _I, _D, _P, _P]),
    "dns_ensemble_create": (_I, [_I, ctypes.POINTER(_I), ctypes.POINTER(_D), ctypes.POINTER(_D), _I, ctypes.POINTER(_P)]),
    "dns_ensemble_destroy": (_I, [_P]),
    "dns_ensemble_size": (_I, [_P]),
    "dns_ensemble_member": (_I, [_P, _I, ctypes.POINTER(_P)]),
    "dns_ensemble_set_streams": (_I, [_P, _I]),
    "dns_ensemble_streams": (_I, [_P]),
    "dns_ensemble_set_batching": (_I, [_P, _I]),
    "dns_ensemble_batching": (_I, [_P]),
    "dns_ensemble_tune": (_I, [_P, ctypes.POINTER(_I)]),
    "dns_transform_r2c": (_I, [_P, _P, _P]),
    "dns_transform_c2r": (_I, [_P, _P, _P]),
    "dns_set_forcing": (_I, [_P, _P, _I]),
    "dns_spectral_filter": (_I, [_P, _I, _P, _I, _I, _P]),
    "dns_spectral_gradient": (_I, [_P, _I, _P, _I, _P]),
    "dns_stress_force": (_I, [_P, _I, _P, _I, _P]),
    "dns_pointwise_products": (_I, [_P, _I, _P, _I, _P]),
    "dns_subtract_products": (_I, [_P, _P, _I, _I, _P]),
    "dns_mlp_param_count": (_I, []),
    "dns_mlp_create": (_I, [ctypes.POINTER(_P)]),
    "dns_mlp_destroy": (_I, [_P]),
    "dns_mlp_set_params": (_I, [_P, ctypes.POINTER(ctypes.c_float), _I]),
    "dns_mlp_get_params": (_I, [_P, ctypes.POINTER(ctypes.c_float), _I]),
    "dns_mlp_forward": (_I, [_P, _P, _P, _I, _P]),
    "dns_mlp_set_normalisation": (_I, [_P, _P, _P, _I, _P]),
    "dns_set_closure": (_I, [_P, _P, _D]),
    "dns_mlp_loss_grad": (_I, [_P, _P, _P, _I, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float), _P]),
    "dns_mlp_train_step": (_I, [_P, _P, _P, _I, _D, ctypes.POINTER(ctypes.c_float), _P]),
    "dns_ensemble_step": (_I, [_P, _I]),
    "dns_ensemble_synchronize": (_I, [_P]),
    "dns_ensemble_time_steps": (_I, [_P, _I, ctypes.POINTER(_D)]),
    "dns_measure_fp64_peak": (_I, [ctypes.POINTER(_D)]),
}

_lib = None


class DnsError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def lib() -> ctypes.CDLL:
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = _build.library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing: run __graft_entry__.build() first")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def last_error() -> str:
    return lib().dns_last_error(None).decode()


def check(code: int, where: str) -> int:
    if code != DNS_OK:
        raise DnsError(code, where, last_error())
    return code
