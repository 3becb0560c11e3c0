"""GB300 simulated-bifurcation solver for the triplet QUBO of track
reconstruction (Okawa, Zeng, Tao, Yung, arXiv:2402.14718).

Thin Python binding of the C ABI in include/sb.h: the functions keep the C
names and only marshal arguments (numpy arrays for host buffers, torch CUDA
tensors or raw integers for device buffers and streams). Every step of the
solver runs in the library's CUDA kernels; there is no Python or CPU fallback.
"""
import ctypes

import numpy as np

from . import _lib
from ._lib import (SB_ASB, SB_BSB, SB_DSB, SB_J_BF16, SB_J_FP32, SB_OPT_DSB_SIGNS, SB_OPT_GRAPH,
                   SB_OPT_HEAVY_FIRST, SB_OPT_L2_PERSIST, SB_OPT_R1_LANES, SB_OPT_REPLICA_GROUPS,
                   SB_OPT_ROWS_PER_WARP, SB_OPT_STEP_RPC, SB_OPT_STEP_RT, SB_OPT_STEP_UNROLL,
                   SB_OPT_STREAM, SB_OPT_TEST_SKIP_STAGE, SB_OPT_TILED, SB_OPT_WAIT_NS,
                   SB_OPT_FACTOR, SB_OPT_TEST_BAD_COL, SB_ERR_BOUNDS, SbError, check, lib)

__all__ = [
    "SB_ASB", "SB_BSB", "SB_DSB", "SB_J_FP32", "SB_J_BF16", "SB_OPT_GRAPH", "SB_OPT_TILED",
    "SB_OPT_STREAM", "SB_OPT_ROWS_PER_WARP", "SB_OPT_HEAVY_FIRST", "SB_OPT_R1_LANES", "SB_OPT_STEP_RT", "SB_OPT_STEP_RPC",
    "SB_OPT_STEP_UNROLL", "SB_OPT_DSB_SIGNS", "SB_OPT_REPLICA_GROUPS", "SB_OPT_L2_PERSIST",
    "SB_OPT_WAIT_NS", "SB_OPT_TEST_SKIP_STAGE", "SB_OPT_FACTOR", "SB_OPT_TEST_BAD_COL",
    "SB_ERR_BOUNDS", "SbError", "sb_checked_build", "sb_check_bounds", "decode_bounds",
    "event_params", "build_params", "sb_event_generate", "sb_qubo_build", "sb_tracks",
    "sb_qubo_build_device", "sb_qubo_factor", "sb_set_factor", "sb_factor_info",
    "sb_create", "sb_create_batch", "sb_destroy", "sb_info", "sb_step_info", "sb_gather_probe",
    "sb_run", "sb_advance",
    "sb_set_state", "sb_get_state", "sb_energy", "sb_best", "sb_readout_device", "sb_set_option",
    "sb_energy_noalloc", "sb_autotune", "sb_set_weights", "sb_backward", "SBRelaxedEnergy",
    "sb_version", "LIB_PATH",
]

LIB_PATH = _lib.LIB_PATH
VARIANTS = {"asb": SB_ASB, "bsb": SB_BSB, "dsb": SB_DSB}


def _variant(v):
    return VARIANTS[v.lower()] if isinstance(v, str) else int(v)


def _host(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def _dev_ptr(t):
    """Device pointer of a torch CUDA tensor, an int, or None."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def sb_version():
    return lib.sb_version().decode()


# ------------------------------------------------------------------ host side
def event_params(**kw):
    p = _lib.SbEventParams()
    lib.sb_event_params_default(ctypes.byref(p))
    for k, v in kw.items():
        if k == "radii":
            p.n_layers = len(v)
            for i, r in enumerate(v):
                p.radii[i] = r
        else:
            setattr(p, k, v)
    return p


def build_params(**kw):
    p = _lib.SbBuildParams()
    lib.sb_build_params_default(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, int(v) if k in ("five_hit_rule", "coupling_mode", "bias_mode") else v)
    return p


class Event:
    """Owns an sb_event handle; ``arrays()`` copies the hits out."""

    def __init__(self, handle):
        self._h = handle
        self.n_hits = lib.sb_event_num_hits(handle)
        self.n_true = lib.sb_event_num_true(handle)

    @property
    def handle(self):
        return self._h

    def arrays(self):
        n = self.n_hits
        out = {"layer": np.zeros(n, np.int32), "r": np.zeros(n), "phi": np.zeros(n),
               "z": np.zeros(n), "x": np.zeros(n), "y": np.zeros(n),
               "particle": np.zeros(n, np.int32)}
        check(lib.sb_event_hits(self._h, *(out[k].ctypes.data_as(ctypes.c_void_p) for k in
                                           ("layer", "r", "phi", "z", "x", "y", "particle"))))
        return out

    def __del__(self):
        if getattr(self, "_h", None):
            lib.sb_event_destroy(self._h)
            self._h = None


def sb_event_generate(seed, params=None):
    h = ctypes.c_void_p()
    p = params if params is not None else event_params()
    check(lib.sb_event_generate(ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), ctypes.byref(p),
                                ctypes.byref(h)))
    return Event(h.value)


class Qubo:
    """Owns an sb_qubo handle; arrays are copied out at construction."""

    def __init__(self, handle):
        self._h = handle
        n = ctypes.c_int32()
        nnz = ctypes.c_int64()
        check(lib.sb_qubo_sizes(handle, ctypes.byref(n), ctypes.byref(nnz)))
        self.n, self.nnz = n.value, nnz.value
        self.rowptr = np.zeros(self.n + 1, np.int32)
        self.col = np.zeros(self.nnz, np.int32)
        self.val = np.zeros(self.nnz)
        self.lin = np.zeros(self.n)
        self.cls = np.zeros(self.nnz, np.int8)
        self.quality = np.zeros(self.n)
        self.trip = np.zeros((self.n, 3), np.int32)
        self.kappa = np.zeros(self.n)
        self.dtheta = np.zeros(self.n)
        check(lib.sb_qubo_arrays(handle, *(a.ctypes.data_as(ctypes.c_void_p) for a in (
            self.rowptr, self.col, self.val, self.lin, self.cls, self.quality, self.trip,
            self.kappa, self.dtheta))))

    @property
    def handle(self):
        return self._h

    def __del__(self):
        if getattr(self, "_h", None):
            lib.sb_qubo_destroy(self._h)
            self._h = None


def sb_qubo_build(event, params=None):
    h = ctypes.c_void_p()
    p = params if params is not None else build_params()
    check(lib.sb_qubo_build(event.handle, ctypes.byref(p), ctypes.byref(h)))
    return Qubo(h.value)


def sb_qubo_factor(qubo):
    """(member [n, 3] int32, couple [3, 3] uint8, w, n_ids) of the builder's QUBO."""
    member = np.zeros((qubo.n, 3), np.int32)
    couple = np.zeros((3, 3), np.uint8)
    w = ctypes.c_double()
    n_ids = ctypes.c_int32()
    check(lib.sb_qubo_factor(qubo.handle, member.ctypes.data_as(ctypes.c_void_p),
                             couple.ctypes.data_as(ctypes.c_void_p), ctypes.byref(w),
                             ctypes.byref(n_ids)))
    return member, couple, w.value, n_ids.value


def sb_qubo_build_device(event, params=None, stream=None):
    """Build on the GPU; returns (Qubo, device milliseconds)."""
    h = ctypes.c_void_p()
    ms = ctypes.c_double()
    p = params if params is not None else build_params()
    check(lib.sb_qubo_build_device(event.handle, ctypes.byref(p), ctypes.byref(h), ctypes.byref(ms),
                                   _stream(stream)))
    return Qubo(h.value), ms.value


def sb_tracks(event, qubo, T, min_hits=4):
    T, pT = _host(T, np.uint8)
    if T.shape[0] != qubo.n:
        raise ValueError("T must have one entry per triplet")
    nh = event.n_hits
    ntr = ctypes.c_int32()
    ptr = np.zeros(nh + 1, np.int32)
    hits = np.zeros(max(nh, 1), np.int32)
    counts = np.zeros(3, np.int64)
    ep = np.zeros(2)
    check(lib.sb_tracks(event.handle, qubo.handle, pT, int(min_hits), ctypes.byref(ntr),
                        ptr.ctypes.data_as(ctypes.c_void_p), hits.ctypes.data_as(ctypes.c_void_p),
                        counts.ctypes.data_as(ctypes.c_void_p), ep.ctypes.data_as(ctypes.c_void_p)))
    tracks = [hits[ptr[k]:ptr[k + 1]].tolist() for k in range(ntr.value)]
    return {"tracks": tracks, "tp": int(counts[0]), "fp": int(counts[1]), "fn": int(counts[2]),
            "efficiency": float(ep[0]), "purity": float(ep[1])}


# ------------------------------------------------------------------ device side
class Ctx:
    """Owns an sb_ctx handle (device memory is released by sb_destroy / GC)."""

    def __init__(self, handle):
        self._h = handle
        self.n_events = lib.sb_num_events(handle)
        self.n = lib.sb_total_rows(handle)
        self.R = 0

    @property
    def handle(self):
        if not self._h:
            raise ValueError("context destroyed")
        return self._h

    def __del__(self):
        sb_destroy(self)


def sb_create(n, rowptr, col, qval, qlin, prec=SB_J_FP32):
    rp, prp = _host(rowptr, np.int32)
    c, pc = _host(col, np.int32)
    v, pv = _host(qval, np.float64)
    a, pa = _host(qlin, np.float64)
    h = ctypes.c_void_p()
    check(lib.sb_create(int(n), int(c.shape[0]), prp, pc, pv, pa, int(prec), ctypes.byref(h)))
    return Ctx(h.value)


def sb_create_batch(events, prec=SB_J_FP32):
    """``events``: sequence of (rowptr, col, qval, qlin) per event (local indices)."""
    ns = np.array([len(e[3]) for e in events], np.int32)
    zs = np.array([len(e[1]) for e in events], np.int64)
    rp, prp = _host(np.concatenate([np.asarray(e[0], np.int32) for e in events]), np.int32)
    c, pc = _host(np.concatenate([np.asarray(e[1], np.int32) for e in events]), np.int32)
    v, pv = _host(np.concatenate([np.asarray(e[2], np.float64) for e in events]), np.float64)
    a, pa = _host(np.concatenate([np.asarray(e[3], np.float64) for e in events]), np.float64)
    h = ctypes.c_void_p()
    check(lib.sb_create_batch(len(events), ns.ctypes.data_as(ctypes.c_void_p),
                              zs.ctypes.data_as(ctypes.c_void_p), prp, pc, pv, pa, int(prec),
                              ctypes.byref(h)))
    return Ctx(h.value)


def sb_destroy(ctx):
    if getattr(ctx, "_h", None):
        lib.sb_destroy(ctx._h)
        ctx._h = None


def sb_info(ctx, e=0):
    n = ctypes.c_int32()
    nnz = ctypes.c_int64()
    off, sig, c0 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    check(lib.sb_info(ctx.handle, int(e), ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(off),
                      ctypes.byref(sig), ctypes.byref(c0)))
    return {"n": n.value, "nnz": nnz.value, "offset": off.value, "sigma_j": sig.value,
            "c0_auto": c0.value}


def sb_set_factor(ctx, n_ids, member, couple, w):
    """``member`` [n, k] int32 block ids (-1: none), ``couple`` [k, k] 0/1; see include/sb.h.
    ``member=None`` removes the factor."""
    if member is None:
        check(lib.sb_set_factor(ctx.handle, 0, 0, None, None, 0.0))
        return
    m, pm = _host(member, np.int32)
    c, pc = _host(couple, np.uint8)
    k = m.shape[1] if m.ndim == 2 else 1
    check(lib.sb_set_factor(ctx.handle, int(n_ids), int(k), pm, pc, float(w)))


def sb_factor_info(ctx):
    out = np.zeros(7, np.int64)
    check(lib.sb_factor_info(ctx.handle, out.ctypes.data_as(ctypes.c_void_p)))
    keys = ("set", "rows", "residual_nnz", "u_rows", "blocks", "members", "max_count")
    return {k: int(v) for k, v in zip(keys, out)}


def sb_checked_build():
    """True when the loaded library is the bounds-checked build."""
    return bool(lib.sb_checked_build())


BOUNDS_MODULES = {1: "step / energy kernels", 2: "factored kernels", 3: "row-group kernel"}
BOUNDS_SITES = {1: "CSR column", 2: "row-pointer pair", 3: "U row", 4: "group member",
                5: "row-group union column"}


def decode_bounds(word):
    """(module, site, index) of a word from sb_check_bounds (see include/sb.h);
    None for 0."""
    if not word:
        return None
    idx = word & 0xFFFFFFFF
    if idx >= 1 << 31:
        idx -= 1 << 32
    return (BOUNDS_MODULES.get(word >> 48, "?"), BOUNDS_SITES.get((word >> 32) & 0xFFFF, "?"), idx)


def sb_check_bounds():
    """Synchronise and read / clear the recorded out-of-range indices: None if
    none, else (status SB_ERR_BOUNDS, decoded word, message); raises on other
    errors."""
    w = ctypes.c_uint64()
    st = lib.sb_check_bounds(ctypes.byref(w))
    if st == SB_ERR_BOUNDS:
        return st, decode_bounds(w.value), lib.sb_last_error().decode(errors="replace")
    check(st)
    return None


def sb_step_info(ctx):
    """(rows per warp of the row-group tables, 0 if not built; union entries)."""
    rw = ctypes.c_int32()
    ent = ctypes.c_int64()
    check(lib.sb_step_info(ctx.handle, ctypes.byref(rw), ctypes.byref(ent)))
    return rw.value, ent.value


def sb_gather_probe(array_bytes, row_bytes, repeats=5, seed=1, stream=None):
    """Bytes per second of random whole-row reads (see include/sb.h)."""
    out = ctypes.c_double()
    check(lib.sb_gather_probe(int(array_bytes), int(row_bytes), int(repeats),
                              ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), ctypes.byref(out),
                              _stream(stream)))
    return out.value


def sb_run(ctx, variant, a0, c0, dt, steps, replicas, seed, a_sched=None, stream=None):
    check(lib.sb_run(ctx.handle, _variant(variant), float(a0), float(c0), float(dt), int(steps),
                     int(replicas), ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF),
                     _dev_ptr(a_sched), _stream(stream)))
    ctx.R = int(replicas)


def sb_advance(ctx, variant, a0, c0, dt, steps, a_sched, stream=None):
    check(lib.sb_advance(ctx.handle, _variant(variant), float(a0), float(c0), float(dt),
                         int(steps), _dev_ptr(a_sched), _stream(stream)))


def sb_set_state(ctx, x, y):
    """``x``, ``y``: [N, R] float32, numpy (host) or torch CUDA tensors (device)."""
    if isinstance(x, np.ndarray):
        xs, px = _host(x, np.float32)
        ys, py = _host(y, np.float32)
        R = xs.shape[1] if xs.ndim == 2 else 1
        check(lib.sb_set_state(ctx.handle, px, py, R, 0))
    else:
        R = x.shape[1] if x.dim() == 2 else 1
        check(lib.sb_set_state(ctx.handle, _dev_ptr(x), _dev_ptr(y), R, 1))
    ctx.R = int(R)


def sb_get_state(ctx):
    """Current (x, y) as host float32 arrays of shape [N, R]."""
    x = np.zeros((ctx.n, ctx.R), np.float32)
    y = np.zeros((ctx.n, ctx.R), np.float32)
    check(lib.sb_get_state(ctx.handle, x.ctypes.data_as(ctypes.c_void_p),
                           y.ctypes.data_as(ctypes.c_void_p), 0))
    return x, y


def sb_energy(ctx, spins=None, replicas=None):
    """QUBO energies [E, R]; ``spins`` int8 [N, R] (+1 selects) or None for sgn(x)."""
    if spins is not None:
        s, ps = _host(spins, np.int8)
        R = s.shape[1] if s.ndim == 2 else 1
    else:
        ps, R = None, int(replicas or ctx.R)
    out = np.zeros((ctx.n_events, R))
    check(lib.sb_energy(ctx.handle, ps, R, out.ctypes.data_as(ctypes.c_void_p)))
    return out


def sb_best(ctx):
    """(T [N] uint8 of the best replica per event, best energy [E], best replica [E])."""
    T = np.zeros(ctx.n, np.uint8)
    E = np.zeros(ctx.n_events)
    r = np.zeros(ctx.n_events, np.int32)
    check(lib.sb_best(ctx.handle, T.ctypes.data_as(ctypes.c_void_p),
                      E.ctypes.data_as(ctypes.c_void_p), r.ctypes.data_as(ctypes.c_void_p)))
    return T, E, r


def sb_readout_device(ctx, d_E_all=None, d_best_E=None, d_best_r=None, d_T=None, stream=None):
    check(lib.sb_readout_device(ctx.handle, _dev_ptr(d_E_all), _dev_ptr(d_best_E),
                                _dev_ptr(d_best_r), _dev_ptr(d_T), _stream(stream)))


def sb_set_option(ctx, key, value):
    check(lib.sb_set_option(ctx.handle, int(key), int(value)))


def sb_energy_noalloc(n, d_rowptr, d_col, d_qval, d_qlin, d_x, d_spins, replicas, d_E,
                      d_best_E=None, d_best_r=None, stream=None):
    """Readout into caller-owned device buffers with the library's static scratch
    (no device allocation); all array arguments are torch CUDA tensors or ints."""
    check(lib.sb_energy_noalloc(int(n), _dev_ptr(d_rowptr), _dev_ptr(d_col), _dev_ptr(d_qval),
                                _dev_ptr(d_qlin), _dev_ptr(d_x), _dev_ptr(d_spins), int(replicas),
                                _dev_ptr(d_E), _dev_ptr(d_best_E), _dev_ptr(d_best_r),
                                _stream(stream)))


def sb_autotune(ctx, variant, replicas, trial_steps=50, stream=None):
    """Time the step-kernel candidates and keep the fastest; returns
    ({"tiled", "tile", "rows_per_cta", "unroll", "groups", "l2_persist",
    "rows_per_warp", "factor"}, microseconds per step)."""
    cfg = np.zeros(8, np.int32)
    us = ctypes.c_float()
    check(lib.sb_autotune(ctx.handle, _variant(variant), int(replicas), int(trial_steps),
                          cfg.ctypes.data_as(ctypes.c_void_p), ctypes.byref(us), _stream(stream)))
    return {"tiled": int(cfg[0]), "tile": int(cfg[1]), "rows_per_cta": int(cfg[2]),
            "unroll": int(cfg[3]), "groups": int(cfg[4]), "l2_persist": int(cfg[5]),
            "rows_per_warp": int(cfg[6]), "factor": int(cfg[7])}, us.value


def sb_set_weights(ctx, cls, quality, w_q, w_c):
    c, pc = _host(cls, np.int8)
    q, pq = _host(quality, np.float64)
    check(lib.sb_set_weights(ctx.handle, pc, pq, float(w_q), float(w_c)))


def sb_backward(ctx, a0, c0, dt, steps, replicas, seed, a_sched=None, ckpt_every=32,
                d_grad_sched=None, stream=None):
    """Returns (loss, {"dt", "c0", "w_q", "w_c"}); dL/da_k goes to ``d_grad_sched``
    (a float64 CUDA tensor of ``steps`` values) when given."""
    loss = ctypes.c_double()
    g = np.zeros(4)
    check(lib.sb_backward(ctx.handle, float(a0), float(c0), float(dt), int(steps), int(replicas),
                          ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), _dev_ptr(a_sched),
                          int(ckpt_every), ctypes.byref(loss), g.ctypes.data_as(ctypes.c_void_p),
                          _dev_ptr(d_grad_sched), _stream(stream)))
    return loss.value, {"dt": g[0], "c0": g[1], "w_q": g[2], "w_c": g[3]}


def _autograd_function():
    import torch

    class SBRelaxedEnergy(torch.autograd.Function):
        """Mean relaxed Ising energy of a bSB run as a differentiable function of
        (dt, c0, a_sched, w_q, w_c). Forward and gradient both run in the
        library's kernels (sb_set_weights + sb_backward); backward scales the
        stored gradients by the incoming gradient."""

        @staticmethod
        def forward(fctx, dt, c0, a_sched, w_q, w_c, sbctx, cls, quality, replicas, seed,
                    ckpt_every=32):
            sb_set_weights(sbctx, cls, quality, float(w_q), float(w_c))
            sched = a_sched.detach().to(device="cuda", dtype=torch.float32).contiguous()
            g_sched = torch.zeros(sched.numel(), dtype=torch.float64, device="cuda")
            loss, g = sb_backward(sbctx, 1.0, float(c0), float(dt), sched.numel(), replicas, seed,
                                  sched, ckpt_every, g_sched)
            fctx.save_for_backward(g_sched)
            fctx.g = g
            fctx.dtypes = (a_sched.dtype, a_sched.device)
            return torch.tensor(loss, dtype=torch.float64)

        @staticmethod
        def backward(fctx, grad_out):
            (g_sched,) = fctx.saved_tensors
            g = fctx.g
            go = float(grad_out)
            dtype, device = fctx.dtypes
            t = lambda v: torch.tensor(go * v, dtype=torch.float64)
            return (t(g["dt"]), t(g["c0"]), (g_sched * go).to(dtype=dtype, device=device),
                    t(g["w_q"]), t(g["w_c"]), None, None, None, None, None, None)

    return SBRelaxedEnergy


def __getattr__(name):
    if name == "SBRelaxedEnergy":
        fn = _autograd_function()
        globals()[name] = fn
        return fn
    raise AttributeError(name)
