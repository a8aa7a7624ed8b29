"""ctypes declarations of the libvipgb C ABI (include/vipgb.h).

Loading fails loudly when the library has not been built: there is no CPU
fallback anywhere in this package.
"""
import ctypes
import os

from . import build as _build

c_int, c_float, c_double, c_size_t, c_uint64 = (ctypes.c_int, ctypes.c_float,
                                                ctypes.c_double, ctypes.c_size_t,
                                                ctypes.c_uint64)
c_void_p = ctypes.c_void_p
c_int_p = ctypes.POINTER(ctypes.c_int)


class FwiGeom(ctypes.Structure):
    _fields_ = [("nz", c_int), ("nx", c_int), ("dx", c_float), ("dt", c_float),
                ("nt", c_int), ("nsponge", c_int), ("sponge_alpha", c_float),
                ("f0", c_float), ("t0", c_float), ("nsrc", c_int),
                ("src_iz", c_int_p), ("src_ix", c_int_p), ("nrec", c_int),
                ("rec_iz", c_int_p), ("rec_ix", c_int_p)]


_SIGS = {
    "vip_strerror": (ctypes.c_char_p, [c_int]),
    "vip_last_error": (ctypes.c_char_p, []),
    "vip_clear_error": (None, []),
    "fwi_create": (c_int, [ctypes.POINTER(FwiGeom), c_size_t, ctypes.POINTER(c_void_p)]),
    "fwi_destroy": (None, [c_void_p]),
    "fwi_set_mode": (c_int, [c_void_p, c_int, c_int]),
    "fwi_set_autotune": (c_int, [c_void_p, c_int]),
    "fwi_set_plan": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_int]),
    "fwi_autotune": (c_int, [c_void_p, c_int, c_int]),
    "fwi_query_plan": (c_int, [c_void_p, c_int, c_int, c_int_p, ctypes.POINTER(c_size_t)]),
    "fwi_forward": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_void_p]),
    "fwi_gradient": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_double, c_void_p,
                             c_void_p, c_int, c_void_p]),
    "fwi_gradient_sources": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_double, c_void_p,
                                     c_int, c_void_p, c_void_p, c_int, c_void_p]),
    "fwi_adjoint": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_int,
                            c_void_p]),
    "fwi_last_status": (c_int, [c_void_p]),
    "fwi_bytes_needed": (c_size_t, [c_void_p]),
    "fwi_set_fill": (c_int, [c_void_p, c_int]),
    "fwi_query_fill": (c_int, [c_void_p, c_int, c_int, c_int_p]),
    "svgd_status": (c_int, [c_void_p, c_void_p]),
    "vip_test_set_wait": (c_int, [ctypes.c_longlong, c_int]),
    "svgd_workspace_size": (c_size_t, [c_int, c_int, c_int, c_int]),
    "svgd_sqdist": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p,
                            c_size_t, c_void_p]),
    "svgd_step": (c_int, [c_void_p, c_void_p, c_float, c_int, c_int, c_float, c_float, c_void_p,
                          c_void_p, c_int, c_void_p, c_size_t, c_void_p, c_void_p]),
    "svgd_step_noalloc": (c_int, [c_void_p, c_void_p, c_float, c_int, c_int, c_float, c_float,
                                  c_void_p, c_void_p, c_int, c_void_p, c_void_p]),
    "ssvgd_step": (c_int, [c_void_p, c_void_p, c_float, c_int, c_int, c_float, c_float, c_void_p,
                           c_void_p, c_int, c_void_p, c_size_t, c_void_p, c_uint64,
                           c_uint64, c_void_p, c_void_p, c_void_p]),
    "svgd_step_q": (c_int, [c_void_p, c_void_p, c_float, c_void_p, c_int, c_int, c_float,
                            c_float, c_void_p, c_void_p, c_int, c_void_p, c_size_t, c_void_p,
                            c_void_p]),
    "ssvgd_step_q": (c_int, [c_void_p, c_void_p, c_float, c_void_p, c_int, c_int, c_float,
                             c_float, c_void_p, c_void_p, c_int, c_void_p, c_size_t, c_void_p,
                             c_uint64, c_uint64, c_void_p, c_void_p, c_void_p]),
    "svgd_inverse_variance": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p]),
    "advi_sample": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int, c_void_p,
                            c_void_p, c_void_p, c_void_p]),
    "advi_step": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_float,
                          c_int, c_int, c_void_p, c_void_p, c_float, c_void_p]),
    "advi_step_opt": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_float,
                              c_int, c_int, c_void_p, c_void_p, c_float, c_int, c_void_p]),
    "vip_to_unconstrained": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int, c_void_p,
                                     c_void_p]),
    "vip_to_model": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int, c_void_p, c_void_p]),
    "vip_unconstrained_gradient": (c_int, [c_void_p, c_void_p, c_float, c_void_p, c_void_p,
                                           c_int, c_int, c_void_p, c_void_p]),
    "advi_lowrank_sample": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p,
                                    c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
    "advi_lowrank_step": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_int,
                                  c_void_p, c_void_p, c_void_p, c_float, c_int, c_int, c_void_p,
                                  c_void_p, c_float, c_void_p]),
    "vip_philox_normal": (c_int, [c_void_p, c_int, c_int, c_uint64, c_uint64, c_void_p]),
    "tomo_create": (c_int, [c_int, c_int, c_double, c_int, c_int_p, ctypes.POINTER(c_void_p)]),
    "tomo_destroy": (c_int, [c_void_p]),
    "tomo_pair_count": (c_int, [c_void_p]),
    "tomo_traveltimes": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_void_p]),
    "tomo_gradient": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p,
                              c_void_p, c_void_p, c_void_p]),
    "tomo_gradient_sources": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p,
                                      c_int, c_void_p, c_void_p, c_void_p]),
    "tomo_last_status": (c_int, [c_void_p]),
}

# Symbols every build exports (checked by the CPU test suite).
EXPORTS = tuple(_SIGS)

_lib = None


def lib_path():
    return _build.LIB


def load():
    """Load libvipgb.so and declare its entry points."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError("libvipgb.so is not built (%s); run "
                           "paper_2310_13325_gb300.build.build() first" % path)
    L = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


class VipError(RuntimeError):
    def __init__(self, code, where):
        L = load()
        msg = L.vip_strerror(code).decode()
        detail = L.vip_last_error().decode()
        L.vip_clear_error()
        super().__init__("%s failed: %s (%d)%s" % (where, msg, code,
                                                   "; " + detail if detail else ""))
        self.code = code


def check(code, where):
    if code != 0:
        raise VipError(code, where)
    return code
