"""ctypes declarations of libgnaosc.so (include/gnaosc.h).  Argument marshalling only."""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgnaosc.so")

c_double = ctypes.c_double
c_int = ctypes.c_int
c_int64 = ctypes.c_int64
c_void_p = ctypes.c_void_p
c_char_p = ctypes.c_char_p

GNA_OK, GNA_EINVAL, GNA_ESHAPE, GNA_ENOMEM, GNA_ECUDA, GNA_ETIMEOUT, GNA_ESTATE = range(7)
GNA_FP64, GNA_MIXED_F64PHASE, GNA_MIXED_FFPHASE = 0, 1, 2
GNA_PEARSON, GNA_POISSON = 0, 1
GNA_PLAN_WITH_PLAIN = 1
GNA_PLAN_FORCE_SPLIT = 2
GNA_PLAN_FORCE_BINS = 4
GNA_PLAN_FORCE_SLICES = 8
GNA_PLAN_GENERAL = 16


class GnaOsc(ctypes.Structure):
    _fields_ = [("s2_12", c_double), ("s2_13", c_double), ("dm2_21", c_double), ("dm2_32", c_double)]


class GnaOscFull(ctypes.Structure):
    _fields_ = [("s2_12", c_double), ("s2_13", c_double), ("s2_23", c_double), ("delta_cp", c_double),
                ("dm2_21", c_double), ("dm2_32", c_double)]


class GnaPlanDesc(ctypes.Structure):
    _fields_ = [
        ("nbins", c_int),
        ("edges", ctypes.POINTER(c_double)),
        ("nodes_per_bin", c_int),
        ("npts", c_int),
        ("node_counts", ctypes.POINTER(ctypes.c_int32)),
        ("nL", c_int),
        ("L", ctypes.POINTER(c_double)),
        ("Lweight", ctypes.POINTER(c_double)),
        ("norm", c_double),
        ("e_scale", c_double),
        ("prec", c_int),
        ("kind", c_int),
        ("max_datasets", c_int),
        ("flags", c_int),
        ("alpha", c_int),
        ("beta", c_int),
        ("anti", c_int),
    ]


class GnaOutputs(ctypes.Structure):
    _fields_ = [("chi2", c_void_p), ("grad", c_void_p), ("grad_eta", c_void_p), ("mu", c_void_p),
                ("spectra", c_void_p)]


# name -> (restype, argtypes), mirroring include/gnaosc.h
SIGNATURES = {
    "gna_strerror": (c_char_p, [c_int]),
    "gna_gl_nodes": (c_int, [c_int, c_void_p, c_void_p, c_void_p]),
    "gna_pmns": (c_int, [ctypes.POINTER(GnaOscFull), ctypes.POINTER(c_double), ctypes.POINTER(c_double)]),
    "gna_oscprob": (c_int, [c_void_p, c_int64, ctypes.POINTER(c_double), c_int, c_int, c_int, c_int,
                            ctypes.POINTER(GnaOscFull), c_int, c_void_p, c_void_p]),
    "gna_poisson_datasets": (c_int, [ctypes.POINTER(c_double), c_int, c_int64, ctypes.c_uint64, c_void_p, c_void_p]),
    "gna_oscprob_ee": (c_int, [c_void_p, c_int64, ctypes.POINTER(c_double), c_int, ctypes.POINTER(GnaOsc), c_int,
                               c_void_p, c_void_p]),
    "gna_oscprob_ee_staged": (c_int, [c_void_p, c_int64, ctypes.POINTER(c_double), c_int, ctypes.POINTER(GnaOsc),
                                      c_int, c_void_p, c_int64, c_void_p]),
    "gna_plan_create": (c_int, [ctypes.POINTER(c_void_p), ctypes.POINTER(GnaPlanDesc), c_void_p]),
    "gna_plan_destroy": (c_int, [c_void_p]),
    "gna_plan_error": (c_char_p, [c_void_p]),
    "gna_plan_status": (c_int, [c_void_p]),
    "gna_plan_info": (c_int, [c_void_p, ctypes.POINTER(c_int64), ctypes.POINTER(c_int64), ctypes.POINTER(c_int64)]),
    "gna_chain_eval": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_void_p, c_int, ctypes.POINTER(GnaOutputs),
                               c_void_p]),
    "gna_chain_eval_general": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_void_p, c_int,
                                       ctypes.POINTER(GnaOutputs), c_void_p]),
    "gna_chain_eval_cached": (c_int, [c_void_p, c_void_p, c_double, c_void_p, c_int, ctypes.POINTER(GnaOutputs),
                                      c_void_p]),
    "gna_chain_eval_host": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_void_p, c_int, c_void_p, c_void_p,
                                    c_void_p, c_void_p]),
    "gna_chain_eval_host_async": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_void_p, c_int, c_int, c_int,
                                          c_void_p, ctypes.POINTER(c_int64)]),
    "gna_chain_eval_host_wait": (c_int, [c_void_p, c_int64, c_void_p, c_void_p, c_void_p]),
    "gna_chain_eval_plain": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_void_p, c_int,
                                     ctypes.POINTER(GnaOutputs), c_void_p]),
    "gna_fit_batch": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_double, c_void_p, c_int, c_void_p]),
    "gna_plan_autotune": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_int, c_void_p]),
    "gna_plan_autotune_general": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_int, c_void_p]),
    "gna_plan_get_tuning": (c_int, [c_void_p, c_char_p, c_int]),
    "gna_plan_set_tuning": (c_int, [c_void_p, c_char_p]),
    "gna_plan_set_graph": (c_int, [c_void_p, c_int]),
    "gna_plan_kernel_launches": (c_int, [c_void_p]),
    "gna_plan_profile": (c_int, [c_void_p, c_int]),
    "gna_plan_profile_read": (c_int, [c_void_p, ctypes.POINTER(c_double), ctypes.POINTER(c_int)]),
    "gna_fp32_probe": (c_int, [c_int, c_int, c_void_p, c_void_p]),
    "gna_grad_scale": (c_int, [c_void_p, ctypes.c_int64, c_void_p, ctypes.c_int64, c_void_p, c_void_p]),
    "gna_chain_eval_general_host": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_void_p, c_int, c_void_p, c_void_p,
                                            c_void_p]),
    "gna_chain_eval_general_host_async": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_void_p, c_int, c_int,
                                                  c_void_p, ctypes.POINTER(ctypes.c_int64)]),
    "gna_fit_batch_general": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_double, c_void_p, c_int, c_void_p]),
    "gna_chain_eval_noalloc": (c_int, [c_int, c_int, c_void_p, c_void_p, ctypes.POINTER(c_double), c_int,
                                       ctypes.POINTER(c_double), c_void_p, c_double, c_int, c_void_p, c_void_p,
                                       c_void_p, c_void_p, c_void_p]),
}

_lock = threading.Lock()
_lib = None


class NativeMissing(RuntimeError):
    pass


def lib():
    """Load libgnaosc.so; raises NativeMissing if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise NativeMissing("libgnaosc.so is not built (%s); run paper_1804_07682_gb300.build.build()" % LIB_PATH)
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


class GnaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (status %d): %s" % (lib().gna_strerror(code).decode(), code, msg))
        self.code = code


def check(code, plan_handle=None, what=""):
    if code != GNA_OK:
        msg = what
        if plan_handle:
            msg += ": " + (lib().gna_plan_error(plan_handle) or b"").decode()
        raise GnaError(code, msg)
