"""ctypes declarations of the C ABI in include/sb.h (argument marshalling only).

The library is loaded on the first call through ``lib`` (importing the package
alone loads nothing, so the numbers-only module ``workloads`` can be imported
without it). Loading builds the in-tree library first if it is missing or
older than its sources; if that fails the call raises: there is no fallback
path. With SB_LIBRARY=checked in the environment the bounds-checked build
(libsbtrack_checked.so, same entry points) is loaded instead.
"""
import ctypes
import os

from . import build as _build

c_int32, c_int64, c_uint64, c_double = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
c_void_p, c_char_p = ctypes.c_void_p, ctypes.c_char_p
P = ctypes.POINTER

(SB_OK, SB_ERR_ARG, SB_ERR_CSR, SB_ERR_CUDA, SB_ERR_OOM, SB_ERR_TIMEOUT, SB_ERR_STATE,
 SB_ERR_BOUNDS) = range(8)
SB_ASB, SB_BSB, SB_DSB = 0, 1, 2
SB_J_FP32, SB_J_BF16 = 0, 1
SB_OPT_GRAPH = 0
SB_OPT_TILED = 1
SB_OPT_STEP_RT = 2
SB_OPT_STEP_RPC = 3
SB_OPT_STEP_UNROLL = 4
SB_OPT_DSB_SIGNS = 5
SB_OPT_REPLICA_GROUPS = 6
SB_OPT_L2_PERSIST = 7
SB_OPT_STREAM = 8
SB_OPT_ROWS_PER_WARP = 9
SB_OPT_HEAVY_FIRST = 10
SB_OPT_R1_LANES = 11
SB_OPT_WAIT_NS = 12
SB_OPT_TEST_SKIP_STAGE = 13
SB_OPT_FACTOR = 14
SB_OPT_TEST_BAD_COL = 15
CHECKED = os.environ.get("SB_LIBRARY", "") == "checked"


class SbEventParams(ctypes.Structure):
    _fields_ = [("n_tracks", c_int32), ("n_layers", c_int32), ("radii", c_double * 16),
                ("noise_frac", c_double), ("bz", c_double), ("inv_pt_min", c_double),
                ("inv_pt_max", c_double), ("eta_max", c_double), ("z0_sigma", c_double),
                ("smear_rphi", c_double), ("smear_z", c_double)]


class SbBuildParams(ctypes.Structure):
    _fields_ = [("dphi_slope", c_double), ("dphi_margin", c_double), ("z0_max", c_double),
                ("kappa_max", c_double), ("dtheta_max", c_double), ("dkappa_max", c_double),
                ("w_q", c_double), ("w_c", c_double), ("five_hit_rule", c_int32),
                ("coupling_mode", c_int32), ("bias_mode", c_int32), ("s_min", c_double),
                ("alpha", c_double), ("beta", c_double), ("gamma", c_double),
                ("lam", c_double)]


class SbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"sb status {code}: {msg}")
        self.code = code


_SIGS = {
    "sb_last_error": (c_char_p, []),
    "sb_version": (c_char_p, []),
    "sb_event_params_default": (None, [P(SbEventParams)]),
    "sb_event_generate": (c_int32, [c_uint64, P(SbEventParams), P(c_void_p)]),
    "sb_event_num_hits": (c_int32, [c_void_p]),
    "sb_event_num_true": (c_int32, [c_void_p]),
    "sb_event_hits": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                c_void_p, c_void_p]),
    "sb_event_destroy": (None, [c_void_p]),
    "sb_build_params_default": (None, [P(SbBuildParams)]),
    "sb_qubo_build": (c_int32, [c_void_p, P(SbBuildParams), P(c_void_p)]),
    "sb_qubo_sizes": (c_int32, [c_void_p, P(c_int32), P(c_int64)]),
    "sb_qubo_arrays": (c_int32, [c_void_p] + [c_void_p] * 9),
    "sb_qubo_destroy": (None, [c_void_p]),
    "sb_qubo_factor": (c_int32, [c_void_p, c_void_p, c_void_p, P(c_double), P(c_int32)]),
    "sb_set_factor": (c_int32, [c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_double]),
    "sb_factor_info": (c_int32, [c_void_p, c_void_p]),
    "sb_qubo_build_device": (c_int32, [c_void_p, P(SbBuildParams), P(c_void_p), P(c_double),
                                       c_void_p]),
    "sb_tracks": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, P(c_int32), c_void_p,
                            c_void_p, c_void_p, c_void_p]),
    "sb_create": (c_int32, [c_int32, c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_int32,
                            P(c_void_p)]),
    "sb_create_batch": (c_int32, [c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                  c_void_p, c_int32, P(c_void_p)]),
    "sb_destroy": (None, [c_void_p]),
    "sb_step_info": (c_int32, [c_void_p, P(c_int32), P(c_int64)]),
    "sb_gather_probe": (c_int32, [c_int64, c_int32, c_int32, c_uint64, P(c_double), c_void_p]),
    "sb_info": (c_int32, [c_void_p, c_int32, P(c_int32), P(c_int64), P(c_double), P(c_double),
                          P(c_double)]),
    "sb_num_events": (c_int32, [c_void_p]),
    "sb_total_rows": (c_int32, [c_void_p]),
    "sb_run": (c_int32, [c_void_p, c_int32, c_double, c_double, c_double, c_int32, c_int32,
                         c_uint64, c_void_p, c_void_p]),
    "sb_advance": (c_int32, [c_void_p, c_int32, c_double, c_double, c_double, c_int32, c_void_p,
                             c_void_p]),
    "sb_set_state": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_int32]),
    "sb_get_state": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32]),
    "sb_energy": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p]),
    "sb_best": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "sb_readout_device": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "sb_set_option": (c_int32, [c_void_p, c_int32, c_int64]),
    "sb_set_weights": (c_int32, [c_void_p, c_void_p, c_void_p, c_double, c_double]),
    "sb_backward": (c_int32, [c_void_p, c_double, c_double, c_double, c_int32, c_int32, c_uint64,
                              c_void_p, c_int32, P(c_double), c_void_p, c_void_p, c_void_p]),
    "sb_autotune": (c_int32, [c_void_p, c_int32, c_int32, c_int32, c_void_p, c_void_p, c_void_p]),
    "sb_energy_noalloc": (c_int32, [c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                    c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_void_p]),
    "sb_checked_build": (c_int32, []),
    "sb_check_bounds": (c_int32, [P(c_uint64)]),
}


def _load():
    path = _build.LIB_CHECKED if CHECKED else _build.LIB
    try:
        _build.build(checked=CHECKED)
    except Exception as exc:  # a missing toolchain with a present library is fine
        if not os.path.exists(path):
            raise ImportError(f"{os.path.basename(path)} is missing and could not be built: "
                              f"{exc}") from exc
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


class _Lib:
    """The loaded library, on first attribute access; each resolved entry
    point is cached on the instance."""

    def __init__(self):
        self._dll = None

    def __getattr__(self, name):
        if name.startswith("__"):
            raise AttributeError(name)
        if self.__dict__.get("_dll") is None:
            self.__dict__["_dll"] = _load()
        fn = getattr(self._dll, name)
        setattr(self, name, fn)
        return fn

    def loaded(self):
        return self.__dict__.get("_dll") is not None


lib = _Lib()
LIB_PATH = _build.LIB_CHECKED if CHECKED else _build.LIB


def check(status):
    if status != SB_OK:
        raise SbError(status, lib.sb_last_error().decode(errors="replace"))
    return status
