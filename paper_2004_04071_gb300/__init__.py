"""Python binding of libmlkd (include/mlkd.h): argument marshalling only.

Every step of the correlated-pair path runs in the CUDA library; this module
builds ctypes structs, hands over device buffers and streams owned by
PyTorch, and converts the results.  If the library is missing it raises: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# MLKD_CHECKED=1 loads the debug build, the same library with device checks
LIB_PATH = os.path.join(_HERE, "_lib", "libmlkd_checked.so" if os.environ.get("MLKD_CHECKED") == "1"
                        else "libmlkd.so")

MLKD_OK = 0
MLKD_EINVAL = -1
MLKD_ENOMEM = -2
MLKD_ECUDA = -3
MLKD_ETIMEDOUT = -4
MLKD_EBUSY = -5
MLKD_ENOTFOUND = -6
MLKD_EINTERNAL = -7

QOI_X2, QOI_X2_PERIODIC, QOI_DENSITY, QOI_X = 0, 1, 2, 3
INIT_ORIGIN, INIT_COSINE, INIT_POINT = 0, 1, 2
BG_HOMOGENEOUS, BG_B1, BG_B2 = 0, 1, 2
PREC_FP64, PREC_FP32_DY64, PREC_FP32_COMP, PREC_FP64_U24 = 0, 1, 2, 3
MAX_LEVELS = 16
MAX_BINS = 1024
ABI_VERSION = 3

EXPORTED = ["mlkd_status_string", "mlkd_abi_version", "mlkd_workspace_bytes",
            "mlkd_context_create", "mlkd_context_destroy", "mlkd_run_level",
            "mlkd_estimate", "mlkd_debug_pairs", "mlkd_context_set_timing",
            "mlkd_context_get_timing", "mlkd_run_level_noalloc", "mlkd_batch_workspace_bytes",
            "mlkd_estimate_batch", "mlkd_autotune_batch", "mlkd_server_start", "mlkd_submit",
            "mlkd_poll", "mlkd_cancel", "mlkd_server_stats_get", "mlkd_server_stop",
            "mlkd_debug_transforms", "mlkd_level_select", "mlkd_estimate_resumable",
            "mlkd_level_select_opt", "mlkd_level_pilot", "mlkd_level_warmup",
            "mlkd_estimate_sequence", "mlkd_debug_batch_pairs", "mlkd_debug_coarse_draws",
            "mlkd_device_checks", "mlkd_debug_check_selftest", "mlkd_debug_kd_coeffs"]
NOALLOC_MAX_BINS = 256


class MlkdError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__("%s: %s (%d)" % (what, status_string(status), status))


class Problem(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("mu", ctypes.c_double), ("T", ctypes.c_double),
                ("dt0", ctypes.c_double), ("M", ctypes.c_int32), ("L", ctypes.c_int32),
                ("qoi", ctypes.c_int32), ("init", ctypes.c_int32), ("nbins", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("lo", ctypes.c_double), ("hi", ctypes.c_double),
                ("tol", ctypes.c_double), ("n_warmup", ctypes.c_int32),
                ("request", ctypes.c_uint32), ("seed", ctypes.c_uint64),
                ("n_fixed", ctypes.POINTER(ctypes.c_int64)), ("n_set", ctypes.c_int32),
                ("reserved_", ctypes.c_int32), ("level_set", ctypes.POINTER(ctypes.c_int32)),
                ("background", ctypes.c_int32), ("reserved2_", ctypes.c_int32),
                ("bg_a", ctypes.c_double), ("bg_b", ctypes.c_double), ("x0", ctypes.c_double)]


class LevelStats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("sy", ctypes.c_double), ("sy2", ctypes.c_double),
                ("sqf", ctypes.c_double), ("sqf2", ctypes.c_double), ("sqc", ctypes.c_double),
                ("sqc2", ctypes.c_double), ("events_f", ctypes.c_uint64),
                ("events_c", ctypes.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class KernelTiming(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64), ("pair_kernel_ms", ctypes.c_double),
                ("other_launches", ctypes.c_uint64)]


class Result(ctypes.Structure):
    _fields_ = [("estimate", ctypes.c_double), ("variance", ctypes.c_double),
                ("n_levels", ctypes.c_int32), ("rounds", ctypes.c_int32),
                ("lv", LevelStats * MAX_LEVELS), ("var_level", ctypes.c_double * MAX_LEVELS),
                ("cost_level", ctypes.c_double * MAX_LEVELS),
                ("density", ctypes.POINTER(ctypes.c_double)), ("seconds", ctypes.c_double)]


class BatchConfig(ctypes.Structure):
    _fields_ = [("pairs_per_thread", ctypes.c_int32), ("substeps_per_launch", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("max_requests", ctypes.c_int32),
                ("max_nbins", ctypes.c_int32), ("refill_min", ctypes.c_int32),
                ("publish_wait_spins", ctypes.c_int32), ("test_stall_queues", ctypes.c_int32),
                ("warp_pair_min_events", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def batch_config(pairs_per_thread=1, substeps_per_launch=256, use_graph=1, max_requests=64,
                 max_nbins=128, refill_min=0, publish_wait_spins=0, test_stall_queues=0,
                 warp_pair_min_events=0) -> BatchConfig:
    c = BatchConfig()
    c.pairs_per_thread, c.substeps_per_launch, c.use_graph = pairs_per_thread, substeps_per_launch, use_graph
    c.max_requests, c.max_nbins, c.refill_min = max_requests, max_nbins, refill_min
    c.publish_wait_spins, c.test_stall_queues = publish_wait_spins, test_stall_queues
    c.warp_pair_min_events = warp_pair_min_events
    return c


class ServerConfig(ctypes.Structure):
    _fields_ = [("batch", BatchConfig), ("precision", ctypes.c_int32), ("max_pending", ctypes.c_int32),
                ("seed", ctypes.c_uint64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("admitted", ctypes.c_uint64),
                ("completed", ctypes.c_uint64), ("cancelled", ctypes.c_uint64),
                ("rejected", ctypes.c_uint64), ("iterations", ctypes.c_uint64),
                ("busy_seconds", ctypes.c_double), ("events", ctypes.c_uint64),
                ("events_processed", ctypes.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def server_config(batch: BatchConfig, precision=PREC_FP32_DY64, seed=0, max_pending=4096) -> ServerConfig:
    c = ServerConfig()
    c.batch = batch
    c.precision, c.seed, c.max_pending = precision, seed & 0xFFFFFFFFFFFFFFFF, max_pending
    return c


_lib = None


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libmlkd.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER
        vp, u64, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int32
        L.mlkd_status_string.argtypes = [ctypes.c_int]
        L.mlkd_status_string.restype = ctypes.c_char_p
        L.mlkd_abi_version.restype = ctypes.c_int
        if L.mlkd_abi_version() != ABI_VERSION:
            raise RuntimeError("libmlkd.so has ABI version %d, the binding expects %d; rebuild it"
                               % (L.mlkd_abi_version(), ABI_VERSION))
        L.mlkd_device_checks.argtypes = [P(ctypes.c_uint32)]
        L.mlkd_device_checks.restype = ctypes.c_int
        L.mlkd_debug_check_selftest.argtypes = [ctypes.c_int]
        L.mlkd_debug_check_selftest.restype = ctypes.c_int
        L.mlkd_debug_kd_coeffs.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, vp, vp, u64, vp, vp, vp, vp, vp, vp]
        L.mlkd_debug_kd_coeffs.restype = ctypes.c_int
        L.mlkd_workspace_bytes.argtypes = [P(Problem)]
        L.mlkd_workspace_bytes.restype = ctypes.c_size_t
        L.mlkd_context_create.argtypes = [ctypes.c_int, vp, ctypes.c_size_t, P(vp)]
        L.mlkd_context_create.restype = ctypes.c_int
        L.mlkd_context_destroy.argtypes = [vp]
        L.mlkd_context_destroy.restype = None
        L.mlkd_run_level.argtypes = [vp, P(Problem), ctypes.c_int, u64, u64, vp, P(LevelStats),
                                     P(ctypes.c_uint64)]
        L.mlkd_run_level.restype = ctypes.c_int
        L.mlkd_estimate.argtypes = [vp, P(Problem), vp, P(Result)]
        L.mlkd_estimate.restype = ctypes.c_int
        L.mlkd_debug_pairs.argtypes = [vp, P(Problem), ctypes.c_int, u64, u64, vp, vp, vp, vp, vp]
        L.mlkd_debug_pairs.restype = ctypes.c_int
        L.mlkd_context_set_timing.argtypes = [vp, ctypes.c_int]
        L.mlkd_context_set_timing.restype = ctypes.c_int
        L.mlkd_context_get_timing.argtypes = [vp, P(KernelTiming), ctypes.c_int]
        L.mlkd_context_get_timing.restype = ctypes.c_int
        L.mlkd_run_level_noalloc.argtypes = [P(Problem), ctypes.c_int, u64, u64, vp, P(LevelStats),
                                             P(ctypes.c_uint64)]
        L.mlkd_run_level_noalloc.restype = ctypes.c_int
        L.mlkd_batch_workspace_bytes.argtypes = [P(BatchConfig)]
        L.mlkd_batch_workspace_bytes.restype = ctypes.c_size_t
        L.mlkd_estimate_batch.argtypes = [vp, P(Problem), ctypes.c_int, P(BatchConfig), vp, P(Result)]
        L.mlkd_estimate_batch.restype = ctypes.c_int
        L.mlkd_debug_coarse_draws.argtypes = [vp, P(Problem), ctypes.c_int, u64, u64, ctypes.c_int,
                                              vp, vp, vp, vp, vp]
        L.mlkd_debug_coarse_draws.restype = ctypes.c_int
        L.mlkd_debug_batch_pairs.argtypes = [vp, P(Problem), P(BatchConfig), ctypes.c_int, vp,
                                             P(Result), vp, vp, vp, vp]
        L.mlkd_debug_batch_pairs.restype = ctypes.c_int
        L.mlkd_autotune_batch.argtypes = [vp, P(Problem), ctypes.c_int, P(BatchConfig), vp,
                                          P(BatchConfig), P(ctypes.c_double)]
        L.mlkd_autotune_batch.restype = ctypes.c_int
        L.mlkd_server_start.argtypes = [vp, P(ServerConfig)]
        L.mlkd_server_start.restype = ctypes.c_int
        L.mlkd_submit.argtypes = [vp, P(Problem), P(ctypes.c_uint64)]
        L.mlkd_submit.restype = ctypes.c_int
        L.mlkd_poll.argtypes = [vp, ctypes.c_uint64, ctypes.c_int, P(Result)]
        L.mlkd_poll.restype = ctypes.c_int
        L.mlkd_cancel.argtypes = [vp, ctypes.c_uint64]
        L.mlkd_cancel.restype = ctypes.c_int
        L.mlkd_server_stats_get.argtypes = [vp, P(ServerStats)]
        L.mlkd_server_stats_get.restype = ctypes.c_int
        L.mlkd_server_stop.argtypes = [vp]
        L.mlkd_server_stop.restype = ctypes.c_int
        L.mlkd_debug_transforms.argtypes = [vp, u64, vp, vp, vp, vp]
        L.mlkd_debug_transforms.restype = ctypes.c_int
        L.mlkd_level_select.argtypes = [P(ctypes.c_double), P(ctypes.c_double), ctypes.c_int,
                                        P(ctypes.c_int32), P(ctypes.c_int32)]
        L.mlkd_level_select.restype = ctypes.c_int
        L.mlkd_level_select_opt.argtypes = [P(ctypes.c_double), P(ctypes.c_double),
                                            P(ctypes.c_double), ctypes.c_int,
                                            P(ctypes.c_int32), P(ctypes.c_int32)]
        L.mlkd_level_select_opt.restype = ctypes.c_int
        L.mlkd_level_pilot.argtypes = [vp, P(Problem), u64, vp, P(ctypes.c_double),
                                       P(ctypes.c_double), P(ctypes.c_double)]
        L.mlkd_level_pilot.restype = ctypes.c_int
        L.mlkd_estimate_resumable.argtypes = [vp, P(Problem), P(Result), P(ctypes.c_uint64), ctypes.c_int,
                                              vp, P(Result), P(ctypes.c_uint64)]
        L.mlkd_estimate_resumable.restype = ctypes.c_int
        L.mlkd_level_warmup.argtypes = [vp, P(Problem), u64, vp, P(ctypes.c_double),
                                        P(ctypes.c_double), P(ctypes.c_int32)]
        L.mlkd_level_warmup.restype = ctypes.c_int
        L.mlkd_estimate_sequence.argtypes = [vp, P(Problem), ctypes.c_int, P(ctypes.c_double), vp,
                                             P(Result)]
        L.mlkd_estimate_sequence.restype = ctypes.c_int
        _lib = L
    return _lib


def status_string(status: int) -> str:
    try:
        return lib().mlkd_status_string(int(status)).decode()
    except RuntimeError:
        return "status %d" % status


def _check(rc, what):
    if rc != MLKD_OK:
        raise MlkdError(rc, what)


def make_problem(eps, T, dt0, M=2, L=1, qoi=QOI_X2, init=INIT_ORIGIN, nbins=0, lo=-3.0, hi=3.0,
                 tol=0.0, n_warmup=100, precision=PREC_FP64, seed=0, request=0, mu=0.0,
                 n_fixed=None, level_set=None, background=BG_HOMOGENEOUS, bg_a=0.0, bg_b=0.0,
                 x0=0.0) -> Problem:
    p = Problem()
    p.eps, p.mu, p.T, p.dt0 = eps, mu, T, dt0
    p.background, p.bg_a, p.bg_b, p.x0 = background, bg_a, bg_b, x0
    p.M, p.L, p.qoi, p.init, p.nbins, p.precision = M, L, qoi, init, nbins, precision
    p.lo, p.hi, p.tol, p.n_warmup = lo, hi, tol, n_warmup
    p.request, p.seed = request & 0xFFFFFFFF, seed & 0xFFFFFFFFFFFFFFFF
    if n_fixed is not None:
        arr = (ctypes.c_int64 * len(n_fixed))(*[int(v) for v in n_fixed])
        p._n_fixed_keep = arr
        p.n_fixed = ctypes.cast(arr, ctypes.POINTER(ctypes.c_int64))
    if level_set is not None:
        ls = (ctypes.c_int32 * len(level_set))(*[int(v) for v in level_set])
        p._level_set_keep = ls
        p.level_set = ctypes.cast(ls, ctypes.POINTER(ctypes.c_int32))
        p.n_set = len(level_set)
    return p


def debug_transforms(words_dev, log_dev=None, sin_dev=None, cos_dev=None, stream=None):
    """mlkd_debug_transforms on torch device tensors (uint32 words in an int32
    tensor, float32 outputs)."""
    vp = ctypes.c_void_p
    ptr = lambda t: vp(t.data_ptr()) if t is not None else vp(0)
    _check(lib().mlkd_debug_transforms(ptr(words_dev), words_dev.numel(), ptr(log_dev), ptr(sin_dev),
                                       ptr(cos_dev), _stream_handle(stream)), "mlkd_debug_transforms")


def device_checks():
    """mlkd_device_checks: (1 in the debug build with device checks, else 0;
    source line of the last failed check, 0 if none)."""
    line = ctypes.c_uint32()
    on = lib().mlkd_device_checks(ctypes.byref(line))
    return int(on), int(line.value)


def debug_check_selftest(device: int = 0) -> int:
    """mlkd_debug_check_selftest: the status the checks report for a kernel
    whose check fails on purpose (debug build: MLKD_EINTERNAL)."""
    return int(lib().mlkd_debug_check_selftest(device))


def debug_kd_coeffs(precision, R, mu, sigma, theta_dev, dv_dev, stream=None):
    """mlkd_debug_kd_coeffs on torch FP64 device tensors: returns the device
    tensors (a, d, hs, om, beta_hat_sq)."""
    import torch
    n = theta_dev.numel()
    outs = [torch.empty(n, dtype=torch.float64, device=theta_dev.device) for _ in range(5)]
    vp = ctypes.c_void_p
    _check(lib().mlkd_debug_kd_coeffs(precision, R, mu, sigma, vp(theta_dev.data_ptr()),
                                      vp(dv_dev.data_ptr()), n, *[vp(t.data_ptr()) for t in outs],
                                      _stream_handle(stream)), "mlkd_debug_kd_coeffs")
    return tuple(outs)


def level_select(V, Vd):
    """mlkd_level_select (Alg. 3): level set from V_l = Var(F(x_l)) and
    Vd_l = Var(Y_l) (Vd[0] unused)."""
    L = len(V) - 1
    v = (ctypes.c_double * (L + 1))(*[float(x) for x in V])
    vd = (ctypes.c_double * (L + 1))(*[float(x) for x in Vd])
    out = (ctypes.c_int32 * (L + 1))()
    n = ctypes.c_int32()
    _check(lib().mlkd_level_select(v, vd, L, out, ctypes.byref(n)), "mlkd_level_select")
    return [int(out[i]) for i in range(n.value)]


def level_select_opt(V, rho, C):
    """mlkd_level_select_opt (Sec. 4.2): the cost-optimal level set from
    V_i = Var(F(x_i)), C_i (i = 0..L) and rho_i = corr(F(x_L), F(x_i))
    (i = 0..L-1)."""
    L = len(V) - 1
    v = (ctypes.c_double * (L + 1))(*[float(x) for x in V])
    r = (ctypes.c_double * max(L, 1))(*[float(x) for x in rho])
    c = (ctypes.c_double * (L + 1))(*[float(x) for x in C])
    out = (ctypes.c_int32 * (L + 1))()
    n = ctypes.c_int32()
    _check(lib().mlkd_level_select_opt(v, r, c, L, out, ctypes.byref(n)), "mlkd_level_select_opt")
    return [int(out[i]) for i in range(n.value)]


def workspace_bytes(problem: Problem) -> int:
    return int(lib().mlkd_workspace_bytes(ctypes.byref(problem)))


def batch_workspace_bytes(cfg: BatchConfig) -> int:
    return int(lib().mlkd_batch_workspace_bytes(ctypes.byref(cfg)))


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Context:
    """mlkd_context over a device arena owned by a torch uint8 tensor."""

    def __init__(self, device: int = 0, arena_bytes: int = 0):
        import torch
        L = lib()
        self.device = device
        need = int(L.mlkd_workspace_bytes(ctypes.byref(make_problem(1.0, 1.0, 1.0))))
        nbytes = max(int(arena_bytes), need)
        self.arena = torch.empty(nbytes, dtype=torch.uint8, device="cuda:%d" % device)
        h = ctypes.c_void_p()
        _check(L.mlkd_context_create(device, ctypes.c_void_p(self.arena.data_ptr()), nbytes,
                                     ctypes.byref(h)), "mlkd_context_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().mlkd_context_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- mlkd_context_set_timing / mlkd_context_get_timing ------------------
    def set_timing(self, enable: bool = True):
        _check(lib().mlkd_context_set_timing(self.handle, 1 if enable else 0),
               "mlkd_context_set_timing")

    def get_timing(self, reset: bool = False) -> dict:
        t = KernelTiming()
        _check(lib().mlkd_context_get_timing(self.handle, ctypes.byref(t), 1 if reset else 0),
               "mlkd_context_get_timing")
        return {"launches": int(t.launches), "pair_kernel_ms": float(t.pair_kernel_ms),
                "other_launches": int(t.other_launches)}

    # -- mlkd_run_level ----------------------------------------------------
    def level_pilot(self, problem: Problem, n: int, stream=None):
        """mlkd_level_pilot: (V[0..L], rho[0..L-1], C[0..L]) from n pairs per
        coupling of L with each coarser level."""
        L = problem.L
        v = (ctypes.c_double * (L + 1))()
        r = (ctypes.c_double * max(L, 1))()
        c = (ctypes.c_double * (L + 1))()
        _check(lib().mlkd_level_pilot(self.handle, ctypes.byref(problem), n, _stream_handle(stream),
                                      v, r, c), "mlkd_level_pilot")
        return list(v), list(r)[:L], list(c)

    def level_warmup(self, problem: Problem, n_warmup: int = 100, stream=None):
        """mlkd_level_warmup (Sec. 5.3, off-line phase): (V[0..L], Vd[0..L], tau)
        for mlkd_level_select."""
        L = problem.L
        v = (ctypes.c_double * (L + 1))()
        vd = (ctypes.c_double * (L + 1))()
        tau = ctypes.c_int32()
        _check(lib().mlkd_level_warmup(self.handle, ctypes.byref(problem), n_warmup,
                                       _stream_handle(stream), v, vd, ctypes.byref(tau)),
               "mlkd_level_warmup")
        return list(v), list(vd), int(tau.value)

    def estimate_sequence(self, problem: Problem, tols, stream=None):
        """mlkd_estimate_sequence (Sec. 5.3, on-line phase): one estimate
        continued through the tolerances; one EstimateResult per stage."""
        n = len(tols)
        t = (ctypes.c_double * n)(*[float(x) for x in tols])
        res = (Result * n)()
        dens = []
        for r in res:
            d = np.zeros(problem.nbins, np.float64) if problem.nbins > 0 else None
            if d is not None:
                r.density = d.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            dens.append(d)
        _check(lib().mlkd_estimate_sequence(self.handle, ctypes.byref(problem), n, t,
                                            _stream_handle(stream), res), "mlkd_estimate_sequence")
        out = []
        for r, d in zip(res, dens):
            nl = r.n_levels
            out.append(EstimateResult(r.estimate, r.variance, r.rounds,
                                      [r.lv[l].as_dict() for l in range(nl)],
                                      [r.var_level[l] for l in range(nl)],
                                      [r.cost_level[l] for l in range(nl)], d, r.seconds))
        return out

    def run_level(self, problem: Problem, level: int, first_pair: int, n_pairs: int, stream=None):
        st = LevelStats()
        hist = None
        hp = None
        if problem.nbins > 0:
            hist = np.zeros(3 * problem.nbins, np.uint64)
            hp = hist.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
        _check(lib().mlkd_run_level(self.handle, ctypes.byref(problem), level, first_pair, n_pairs,
                                    _stream_handle(stream), ctypes.byref(st), hp),
               "mlkd_run_level")
        out = st.as_dict()
        if hist is not None:
            nb = problem.nbins
            out["hist_f"], out["hist_c"], out["hist_both"] = hist[:nb], hist[nb:2 * nb], hist[2 * nb:]
        return out

    # -- mlkd_debug_pairs --------------------------------------------------
    def debug_pairs(self, problem: Problem, level: int, first_pair: int, n_pairs: int, stream=None):
        import torch
        dev = "cuda:%d" % self.device
        xf = torch.empty(max(n_pairs, 1), dtype=torch.float64, device=dev)
        xc = torch.empty(max(n_pairs, 1), dtype=torch.float64, device=dev)
        kf = torch.empty(max(n_pairs, 1), dtype=torch.int32, device=dev)
        kc = torch.empty(max(n_pairs, 1), dtype=torch.int32, device=dev)
        vp = ctypes.c_void_p
        _check(lib().mlkd_debug_pairs(self.handle, ctypes.byref(problem), level, first_pair,
                                      n_pairs, _stream_handle(stream), vp(xf.data_ptr()),
                                      vp(xc.data_ptr()), vp(kf.data_ptr()), vp(kc.data_ptr())),
               "mlkd_debug_pairs")
        n = n_pairs
        return (xf[:n].cpu().numpy(), xc[:n].cpu().numpy(), kf[:n].cpu().numpy().astype(np.int64),
                kc[:n].cpu().numpy().astype(np.int64))

    def debug_coarse_draws(self, problem: Problem, level: int, first_pair: int, n_pairs: int,
                           per_pair: int = 64, stream=None):
        """mlkd_debug_coarse_draws: (nu~, E~, chi~, pair_of) of every recorded
        coarse step, concatenated in pair order, and each pair's coarse-step
        count (steps past per_pair are counted but not recorded)."""
        import torch
        dev = "cuda:%d" % self.device
        m = max(n_pairs * per_pair, 1)
        nu = torch.empty(m, dtype=torch.float64, device=dev)
        E = torch.empty(m, dtype=torch.float64, device=dev)
        chi = torch.empty(m, dtype=torch.float64, device=dev)
        cnt = torch.empty(max(n_pairs, 1), dtype=torch.int32, device=dev)
        vp = ctypes.c_void_p
        _check(lib().mlkd_debug_coarse_draws(self.handle, ctypes.byref(problem), level, first_pair,
                                             n_pairs, per_pair, _stream_handle(stream),
                                             vp(nu.data_ptr()), vp(E.data_ptr()), vp(chi.data_ptr()),
                                             vp(cnt.data_ptr())), "mlkd_debug_coarse_draws")
        counts = cnt[:n_pairs].cpu().numpy().astype(np.int64)
        rec = np.minimum(counts, per_pair)
        idx = np.concatenate([j * per_pair + np.arange(r) for j, r in enumerate(rec)]) if n_pairs else \
            np.zeros(0, np.int64)
        pair_of = np.repeat(np.arange(n_pairs), rec)
        return (nu.cpu().numpy()[idx], E.cpu().numpy()[idx], chi.cpu().numpy()[idx], pair_of, counts)

    # -- mlkd_estimate_batch / mlkd_autotune_batch ----------------------------
    def estimate_batch(self, problems, cfg: BatchConfig, stream=None):
        n = len(problems)
        arr = (Problem * n)(*problems)
        res = (Result * n)()
        dens = []
        for i, p in enumerate(problems):
            d = None
            if p.nbins > 0:
                d = np.zeros(p.nbins, np.float64)
                res[i].density = d.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            dens.append(d)
        _check(lib().mlkd_estimate_batch(self.handle, arr, n, ctypes.byref(cfg),
                                         _stream_handle(stream), res), "mlkd_estimate_batch")
        out = []
        for i in range(n):
            r = res[i]
            nl = r.n_levels
            out.append(EstimateResult(r.estimate, r.variance, r.rounds,
                                      [r.lv[l].as_dict() for l in range(nl)],
                                      [r.var_level[l] for l in range(nl)],
                                      [r.cost_level[l] for l in range(nl)], dens[i], r.seconds))
        return out

    def debug_batch_pairs(self, problem: Problem, cfg: BatchConfig, level: int, stream=None):
        """mlkd_debug_batch_pairs: (EstimateResult, xf, xc, kf, kc) of a
        fixed-count problem in the batched form, with the per-pair results of
        estimator level `level`."""
        import torch
        dev = "cuda:%d" % self.device
        n = int(problem.n_fixed[level])
        xf = torch.empty(max(n, 1), dtype=torch.float64, device=dev)
        xc = torch.empty(max(n, 1), dtype=torch.float64, device=dev)
        kf = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        kc = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        r = Result()
        d = None
        if problem.nbins > 0:
            d = np.zeros(problem.nbins, np.float64)
            r.density = d.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        vp = ctypes.c_void_p
        _check(lib().mlkd_debug_batch_pairs(self.handle, ctypes.byref(problem), ctypes.byref(cfg), level,
                                            _stream_handle(stream), ctypes.byref(r), vp(xf.data_ptr()),
                                            vp(xc.data_ptr()), vp(kf.data_ptr()), vp(kc.data_ptr())),
               "mlkd_debug_batch_pairs")
        nl = r.n_levels
        er = EstimateResult(r.estimate, r.variance, r.rounds, [r.lv[l].as_dict() for l in range(nl)],
                            [r.var_level[l] for l in range(nl)], [r.cost_level[l] for l in range(nl)],
                            d, r.seconds)
        return (er, xf[:n].cpu().numpy(), xc[:n].cpu().numpy(),
                kf[:n].cpu().numpy().astype(np.int64), kc[:n].cpu().numpy().astype(np.int64))

    def autotune_batch(self, problems, base: BatchConfig, stream=None):
        n = len(problems)
        arr = (Problem * n)(*problems)
        best = BatchConfig()
        secs = (ctypes.c_double * 48)()
        _check(lib().mlkd_autotune_batch(self.handle, arr, n, ctypes.byref(base),
                                         _stream_handle(stream), ctypes.byref(best), secs),
               "mlkd_autotune_batch")
        return best, list(secs)

    # -- serving: mlkd_server_start / submit / poll / cancel / stop ----------
    def server_start(self, cfg: ServerConfig):
        _check(lib().mlkd_server_start(self.handle, ctypes.byref(cfg)), "mlkd_server_start")

    def submit(self, problem: Problem) -> int:
        rid = ctypes.c_uint64()
        _check(lib().mlkd_submit(self.handle, ctypes.byref(problem), ctypes.byref(rid)), "mlkd_submit")
        return int(rid.value)

    def try_submit(self, problem: Problem):
        """mlkd_submit returning (status, id) instead of raising."""
        rid = ctypes.c_uint64()
        rc = lib().mlkd_submit(self.handle, ctypes.byref(problem), ctypes.byref(rid))
        return rc, int(rid.value)

    def poll(self, req_id: int, timeout_ms: int = -1, nbins: int = 0):
        """Returns (status, EstimateResult or None)."""
        r = Result()
        dens = None
        if nbins > 0:
            dens = np.zeros(nbins, np.float64)
            r.density = dens.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        rc = lib().mlkd_poll(self.handle, req_id, timeout_ms, ctypes.byref(r))
        if rc != MLKD_OK:
            return rc, None
        nl = r.n_levels
        return rc, EstimateResult(r.estimate, r.variance, r.rounds,
                                  [r.lv[l].as_dict() for l in range(nl)],
                                  [r.var_level[l] for l in range(nl)],
                                  [r.cost_level[l] for l in range(nl)], dens, r.seconds)

    def cancel(self, req_id: int) -> int:
        return lib().mlkd_cancel(self.handle, req_id)

    def server_stats(self) -> dict:
        st = ServerStats()
        _check(lib().mlkd_server_stats_get(self.handle, ctypes.byref(st)), "mlkd_server_stats_get")
        return st.as_dict()

    def server_stop(self):
        _check(lib().mlkd_server_stop(self.handle), "mlkd_server_stop")

    # -- mlkd_estimate_resumable ----------------------------------------------
    def estimate_resumable(self, problem: Problem, resume=None, hist_in=None, max_rounds=64,
                           stream=None):
        """Returns (EstimateResult, histogram counts [J*3*nbins] or None): a
        checkpoint that resume/hist_in continue exactly."""
        r = Result()
        dens = None
        hist = None
        hp = None
        if problem.nbins > 0:
            dens = np.zeros(problem.nbins, np.float64)
            r.density = dens.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            J = problem.n_set if problem.n_set > 0 else problem.L + 1
            hist = np.zeros(J * 3 * problem.nbins, np.uint64)
            hp = hist.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
        rs = None
        hin = None
        if resume is not None:
            rs = _result_struct(resume)
            if hist_in is not None:
                hin_arr = np.ascontiguousarray(hist_in, np.uint64)
                hin = hin_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
        _check(lib().mlkd_estimate_resumable(self.handle, ctypes.byref(problem),
                                             ctypes.byref(rs) if rs is not None else None, hin,
                                             max_rounds, _stream_handle(stream), ctypes.byref(r), hp),
               "mlkd_estimate_resumable")
        n = r.n_levels
        er = EstimateResult(r.estimate, r.variance, r.rounds, [r.lv[l].as_dict() for l in range(n)],
                            [r.var_level[l] for l in range(n)], [r.cost_level[l] for l in range(n)],
                            dens, r.seconds)
        return er, hist

    # -- mlkd_estimate -----------------------------------------------------
    def estimate(self, problem: Problem, stream=None):
        r = Result()
        dens = None
        if problem.nbins > 0:
            dens = np.zeros(problem.nbins, np.float64)
            r.density = dens.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        _check(lib().mlkd_estimate(self.handle, ctypes.byref(problem), _stream_handle(stream),
                                   ctypes.byref(r)), "mlkd_estimate")
        n = r.n_levels
        return EstimateResult(r.estimate, r.variance, r.rounds,
                              [r.lv[l].as_dict() for l in range(n)],
                              [r.var_level[l] for l in range(n)],
                              [r.cost_level[l] for l in range(n)], dens, r.seconds)


def run_level_noalloc(problem: Problem, level: int, first_pair: int, n_pairs: int, stream=None):
    """mlkd_run_level_noalloc: level sums without a context or arena, for
    callers that cannot allocate device memory (scratch lives in a static
    device array inside the library; overlapping calls race)."""
    st = LevelStats()
    hist = None
    hp = None
    if problem.nbins > 0:
        hist = np.zeros(3 * problem.nbins, np.uint64)
        hp = hist.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
    _check(lib().mlkd_run_level_noalloc(ctypes.byref(problem), level, first_pair, n_pairs,
                                        _stream_handle(stream), ctypes.byref(st), hp),
           "mlkd_run_level_noalloc")
    out = st.as_dict()
    if hist is not None:
        nb = problem.nbins
        out["hist_f"], out["hist_c"], out["hist_both"] = hist[:nb], hist[nb:2 * nb], hist[2 * nb:]
    return out


def _result_struct(er) -> Result:
    """mlkd_result holding the level sums and round count of an EstimateResult."""
    r = Result()
    r.estimate, r.variance = er.estimate, er.variance
    r.n_levels, r.rounds = len(er.levels), er.rounds
    for l, lv in enumerate(er.levels):
        for k, _ in LevelStats._fields_:
            setattr(r.lv[l], k, lv[k])
        r.var_level[l] = er.var_level[l]
        r.cost_level[l] = er.cost_level[l]
    return r


def checkpoint_to_json(er, hist=None) -> str:
    """Text form of a checkpoint (exact: floats round-trip through repr)."""
    import json
    return json.dumps({"rounds": er.rounds, "levels": er.levels,
                       "hist": None if hist is None else [int(v) for v in hist]})


def checkpoint_from_json(text: str):
    """(EstimateResult, hist) from checkpoint_to_json's text."""
    import json
    d = json.loads(text)
    levels = d["levels"]
    n = len(levels)
    er = EstimateResult(0.0, 0.0, d["rounds"], levels, [0.0] * n, [0.0] * n, None, 0.0)
    hist = None if d["hist"] is None else np.array(d["hist"], np.uint64)
    return er, hist


@dataclass
class EstimateResult:
    estimate: float
    variance: float
    rounds: int
    levels: list
    var_level: list
    cost_level: list
    density: np.ndarray
    seconds: float
