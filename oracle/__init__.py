"""CPU oracle for the ML-KDMC correlated-pair path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does.

``mlkd_oracle.c`` restates Alg. 1 (KD path), Alg. 2 (correlated pair) and the
random-number mapping/aggregation of Sec. 3 in FP64 with its own Philox4x32-10.
This module adds, in plain numpy:

* the quantities of interest F(x(T)) and the level difference
  Y_l = F(x_l) - F(x_{l-1}) of eq. mlmc-compact (Sec. 4.1);
* the per-level sums that set the sample counts, and the histogram counts of
  the density estimator;
* the adaptive sample-count rule of eqs. Nopt1/Noptj (Sec. 4.1).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mlkd_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liborc.so")

QOI_X2 = 0            # F(x) = x^2 (free space)
QOI_X2_PERIODIC = 1   # F(x) = (x mod 1)^2 on the periodic unit interval
QOI_DENSITY = 2       # histogram density drives the sample counts
QOI_X = 3             # F(x) = x, the paper's test-case QoI (Sec. 5)
INIT_ORIGIN = 0
INIT_COSINE = 1
INIT_POINT = 2        # every path starts at Problem.x0
RECIPE_24 = 0         # 24-bit uniforms (FP32 form of the stream)
RECIPE_53 = 1         # 53-bit uniforms (FP64 form of the stream)

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FP contraction, no fast-math)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
                           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class LevelDesc(ctypes.Structure):
    _fields_ = [("R", ctypes.c_double), ("mu", ctypes.c_double), ("sigma", ctypes.c_double),
                ("dt", ctypes.c_double), ("n", ctypes.c_int64), ("M", ctypes.c_int32),
                ("level", ctypes.c_int32), ("init", ctypes.c_int32), ("recipe", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("request", ctypes.c_uint32), ("coupled", ctypes.c_int32),
                ("x0", ctypes.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.POINTER
            d, i64, u64, u32 = ctypes.c_double, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32
            L.orc_philox4x32_10.argtypes = [P(u32), P(u32), P(u32)]
            L.orc_philox4x32_10.restype = None
            L.orc_uniform24.argtypes = [u32]
            L.orc_uniform24.restype = d
            L.orc_uniform53.argtypes = [u32, u32]
            L.orc_uniform53.restype = d
            for name in ("orc_fs", "orc_gs", "orc_hs", "orc_cosine_G", "orc_cosine_inverse"):
                getattr(L, name).argtypes = [d]
                getattr(L, name).restype = d
            L.orc_advection.argtypes = [d, d, d, d]
            L.orc_advection.restype = d
            L.orc_diffusion.argtypes = [d, d, d, d, d]
            L.orc_diffusion.restype = d
            L.orc_zeta.argtypes = [d, d]
            L.orc_zeta.restype = d
            L.orc_theta_prime.argtypes = [d, d]
            L.orc_theta_prime.restype = d
            L.orc_beta.argtypes = [d, d, d]
            L.orc_beta.restype = d
            L.orc_pairs.argtypes = [P(LevelDesc), u64, i64, P(d), P(d), P(i64), P(i64)]
            L.orc_pairs.restype = ctypes.c_int
            L.orc_single_paths.argtypes = [P(LevelDesc), u64, i64, P(d), P(i64)]
            L.orc_single_paths.restype = ctypes.c_int
            L.orc_pair_injected.argtypes = [P(LevelDesc), d, P(d), P(d), P(d), i64, P(d), P(d),
                                            P(i64), P(i64), i64, P(i64), P(d), P(d), P(d), P(d),
                                            P(i64)]
            L.orc_pair_injected.restype = ctypes.c_int
            L.orc_coarse_draws.argtypes = [P(LevelDesc), u64, i64, i64, P(d), P(d), P(d), P(i64)]
            L.orc_coarse_draws.restype = i64
            L.orc_stream_draws.argtypes = [P(LevelDesc), u64, i64, P(d), P(d), P(d), P(d)]
            L.orc_stream_draws.restype = None
            L.orc_het_R.argtypes = [P(HetBg), d]
            L.orc_het_R.restype = d
            L.orc_het_depth.argtypes = [P(HetBg), d, d, d, d]
            L.orc_het_depth.restype = d
            L.orc_het_flight.argtypes = [P(HetBg), d, d, d, d]
            L.orc_het_flight.restype = d
            L.orc_het_pairs.argtypes = [P(HetDesc), u64, i64, P(d), P(d), P(i64), P(i64)]
            L.orc_het_pairs.restype = ctypes.c_int
            L.orc_het_coarse_draws.argtypes = [P(HetDesc), u64, i64, i64, P(d), P(d), P(d)]
            L.orc_het_coarse_draws.restype = i64
            _lib = L
    return _lib


class HetBg(ctypes.Structure):
    _fields_ = [("b", ctypes.c_double), ("a_left", ctypes.c_double), ("a_right", ctypes.c_double)]


class HetDesc(ctypes.Structure):
    _fields_ = [("bg", HetBg), ("dt", ctypes.c_double), ("n", ctypes.c_int64), ("M", ctypes.c_int32),
                ("level", ctypes.c_int32), ("recipe", ctypes.c_int32), ("coupled", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("request", ctypes.c_uint32), ("pad_", ctypes.c_int32),
                ("x0", ctypes.c_double)]


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def philox4x32_10(ctr, key):
    """Philox4x32-10 block (SC'11) for a 4-word counter and 2-word key."""
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


# --------------------------------------------------------------------------
# Problem description (the paper's problem statement, Sec. 4.1, in the
# diffusive scaling: R = 1/eps^2, sigma = 1/eps).
# --------------------------------------------------------------------------
@dataclass
class Problem:
    eps: float
    T: float
    dt0: float
    M: int = 2
    L: int = 1
    qoi: int = QOI_X2
    init: int = INIT_ORIGIN
    nbins: int = 0
    lo: float = -3.0
    hi: float = 3.0
    tol: float = 0.0
    n_warmup: int = 100
    recipe: int = RECIPE_53
    seed: int = 0
    request: int = 0
    mu: float = 0.0
    n_fixed: list = field(default_factory=list)
    level_set: list = field(default_factory=list)   # estimator levels (Sec. 4.2); empty: 0..L
    x0: float = 0.0                                 # start of every path for INIT_POINT
    background: int = 0                             # 0 homogeneous; BG_B1 / BG_B2 (Sec. 5)
    a: float = 0.0                                  # B1/B2: R(x) from a, b; mu = 0, sigma = 1
    b: float = 0.0

    @property
    def R(self):
        return self.b if self.background else 1.0 / (self.eps * self.eps)

    @property
    def sigma(self):
        return 1.0 if self.background else 1.0 / self.eps

    def steps0(self) -> int:
        r = self.T / self.dt0
        n0 = int(round(r))
        if n0 < 1 or abs(r - n0) > 1e-12 * max(1.0, r):
            raise ValueError("T/dt0 must be a positive integer")
        return n0

    def dt(self, level: int) -> float:
        return self.dt0 / float(self.M) ** level

    def nsteps(self, level: int) -> int:
        return self.steps0() * self.M ** level

    def estimator_levels(self):
        """(fine level, coarsening to the previous estimator level) per
        estimator level j: level_set[j] with M^(level_set[j] - level_set[j-1])."""
        ls = list(self.level_set) if self.level_set else list(range(self.L + 1))
        return [(l, self.M ** (l - ls[j - 1]) if j else self.M) for j, l in enumerate(ls)]

    def level_desc(self, j: int) -> LevelDesc:
        """Oracle description of estimator level j."""
        level, m = self.estimator_levels()[j]
        d = LevelDesc()
        d.R, d.mu, d.sigma = self.R, self.mu, self.sigma
        d.dt = self.dt(level)
        d.n = self.nsteps(level)
        d.M = m
        d.level = level
        d.coupled = 1 if j > 0 else 0
        d.init = self.init
        d.recipe = self.recipe
        d.seed = self.seed
        d.request = self.request
        d.x0 = self.x0
        return d

    def bin_range(self):
        if self.periodic():
            return 0.0, 1.0
        return self.lo, self.hi

    def periodic(self) -> bool:
        return self.qoi == QOI_X2_PERIODIC or self.init == INIT_COSINE


# --------------------------------------------------------------------------
# Paths and pairs.
# --------------------------------------------------------------------------
def pairs(problem: Problem, level: int, first: int, count: int, threads: int = 1):
    """Final positions (x_l, x_{l-1}) and event counts of pairs
    [first, first+count) of estimator level `level`.  Estimator level 0 is
    Alg. 1 (x_c = 0)."""
    if problem.background:
        fine, coarsening = problem.estimator_levels()[level]
        x0 = problem.x0 if problem.init == INIT_POINT else 0.0
        return het_pairs(problem.background, problem.a, problem.b, problem.T, problem.dt0,
                         problem.M, fine, level > 0, first, count, x0=x0, seed=problem.seed,
                         request=problem.request, recipe=problem.recipe, coarsening=coarsening,
                         threads=threads)
    d = problem.level_desc(level)
    xf = np.zeros(count, np.float64)
    xc = np.zeros(count, np.float64)
    ef = np.zeros(count, np.int64)
    ec = np.zeros(count, np.int64)
    L = lib()
    threads = max(1, min(int(threads), count if count > 0 else 1))
    bounds = np.linspace(0, count, threads + 1).astype(np.int64)

    def work(t):
        a, b = int(bounds[t]), int(bounds[t + 1])
        if b <= a:
            return 0
        dt = ctypes.c_double
        i64 = ctypes.c_int64
        return L.orc_pairs(ctypes.byref(d), first + a, b - a,
                           ctypes.cast(xf.ctypes.data + 8 * a, ctypes.POINTER(dt)),
                           ctypes.cast(xc.ctypes.data + 8 * a, ctypes.POINTER(dt)),
                           ctypes.cast(ef.ctypes.data + 8 * a, ctypes.POINTER(i64)),
                           ctypes.cast(ec.ctypes.data + 8 * a, ctypes.POINTER(i64)))

    if threads == 1:
        rcs = [work(0)]
    else:
        with ThreadPoolExecutor(threads) as ex:
            rcs = list(ex.map(work, range(threads)))
    if any(rc != 0 for rc in rcs):
        raise RuntimeError("oracle pair simulation failed: %r" % rcs)
    return xf, xc, ef, ec


def _fine_desc(problem: Problem, level: int) -> LevelDesc:
    """Single-path description of fine level `level` (any level, not an
    estimator index)."""
    d = LevelDesc()
    d.R, d.mu, d.sigma = problem.R, problem.mu, problem.sigma
    d.dt, d.n, d.M = problem.dt(level), problem.nsteps(level), problem.M
    d.level = level
    d.init, d.recipe, d.seed, d.request, d.coupled = (problem.init, problem.recipe, problem.seed,
                                                      problem.request, 0)
    d.x0 = problem.x0
    return d


def single_paths(problem: Problem, level: int, first: int, count: int, key_level: int = None):
    """Independent single-level (Alg. 1) paths at dt_level, keyed by key_level."""
    d = _fine_desc(problem, level)
    if key_level is not None:
        d.level = key_level
    x = np.zeros(count, np.float64)
    ev = np.zeros(count, np.int64)
    rc = lib().orc_single_paths(ctypes.byref(d), first, count, _ptr(x, ctypes.c_double),
                                _ptr(ev, ctypes.c_int64))
    if rc:
        raise RuntimeError("oracle path simulation failed")
    return x, ev


def pair_injected(R, mu, sigma, dt, n, M, x0, nu, E, chi, level=1):
    """One path (level 0) or pair (level >= 1) on caller-chosen random numbers:
    nu[k], E[k] for k = 0..K and chi[k] for k = 0..K-1 (the paper's y_l)."""
    nu = np.ascontiguousarray(nu, np.float64)
    E = np.ascontiguousarray(E, np.float64)
    chi = np.ascontiguousarray(chi, np.float64)
    assert len(nu) == len(E) and len(chi) >= len(nu) - 1
    d = LevelDesc()
    d.R, d.mu, d.sigma, d.dt, d.n, d.M, d.level = R, mu, sigma, dt, n, M, level
    d.coupled = 1 if level != 0 else 0
    cap = 4096
    kappa = np.zeros(cap, np.int64)
    nu_t, E_t, chi_t, cc = (np.zeros(cap) for _ in range(4))
    xf, xc = ctypes.c_double(), ctypes.c_double()
    ef, ec, nco = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    dd = ctypes.c_double
    rc = lib().orc_pair_injected(ctypes.byref(d), x0, _ptr(nu, dd), _ptr(E, dd), _ptr(chi, dd),
                                 len(nu), ctypes.byref(xf), ctypes.byref(xc), ctypes.byref(ef),
                                 ctypes.byref(ec), cap, _ptr(kappa, ctypes.c_int64),
                                 _ptr(nu_t, dd), _ptr(E_t, dd), _ptr(chi_t, dd), _ptr(cc, dd),
                                 ctypes.byref(nco))
    if rc:
        raise RuntimeError("injected pair ran out of random numbers (rc=%d)" % rc)
    k = nco.value
    return dict(xf=xf.value, xc=xc.value, ev_f=ef.value, ev_c=ec.value,
                kappa=kappa[:k].copy(), nu_t=nu_t[:k].copy(), E_t=E_t[:k].copy(),
                chi_t=chi_t[:k].copy(), coarse_collision=cc[:k].copy())


def coarse_draws(problem: Problem, level: int, first: int, count: int, cap: int):
    """Aggregated coarse random numbers (nu~, E~, chi~) of Philox pairs."""
    d = problem.level_desc(level)
    nu_t, E_t, chi_t = np.zeros(cap), np.zeros(cap), np.zeros(cap)
    pair_of = np.zeros(cap, np.int64)
    dd = ctypes.c_double
    w = lib().orc_coarse_draws(ctypes.byref(d), first, count, cap, _ptr(nu_t, dd), _ptr(E_t, dd),
                               _ptr(chi_t, dd), _ptr(pair_of, ctypes.c_int64))
    if w < 0:
        raise RuntimeError("oracle coarse draws failed")
    return nu_t[:w], E_t[:w], chi_t[:w], pair_of[:w]


def stream_draws(problem: Problem, level: int, pair: int, K: int):
    """(nu_0, E_0, u_x0) and (nu_k, E_k, chi_{k-1}) for k = 1..K of one stream
    (fine level `level`)."""
    d = _fine_desc(problem, level)
    init = np.zeros(3)
    nu, E, chi = np.zeros(K), np.zeros(K), np.zeros(K)
    dd = ctypes.c_double
    lib().orc_stream_draws(ctypes.byref(d), pair, K, _ptr(init, dd), _ptr(nu, dd), _ptr(E, dd),
                           _ptr(chi, dd))
    return init, nu, E, chi


# --------------------------------------------------------------------------
# Quantities of interest and level sums (Sec. 4.1).
# --------------------------------------------------------------------------
def qoi_values(problem: Problem, x: np.ndarray) -> np.ndarray:
    if problem.qoi == QOI_X:
        return np.array(x, np.float64, copy=True)
    if problem.periodic():
        xm = x - np.floor(x)
        return xm * xm
    return x * x


def bin_index(problem: Problem, x: np.ndarray) -> np.ndarray:
    """Histogram bin of each position; -1 when it falls outside [lo, hi)
    (free space).  Periodic problems wrap x into [0, 1) first."""
    lo, hi = problem.bin_range()
    nb = problem.nbins
    if problem.periodic():
        x = x - np.floor(x)
    h = (hi - lo) / nb
    b = np.floor((x - lo) / h).astype(np.int64)
    b[(x < lo) | (x >= hi)] = -1
    b[b >= nb] = nb - 1
    return b


@dataclass
class LevelSums:
    n: int = 0
    sy: float = 0.0
    sy2: float = 0.0
    sqf: float = 0.0
    sqf2: float = 0.0
    sqc: float = 0.0
    sqc2: float = 0.0
    events_f: int = 0
    events_c: int = 0
    hist_f: np.ndarray = None
    hist_c: np.ndarray = None
    hist_both: np.ndarray = None

    def add(self, o: "LevelSums"):
        self.n += o.n
        for k in ("sy", "sy2", "sqf", "sqf2", "sqc", "sqc2"):
            setattr(self, k, getattr(self, k) + getattr(o, k))
        self.events_f += o.events_f
        self.events_c += o.events_c
        if o.hist_f is not None:
            if self.hist_f is None:
                self.hist_f = np.zeros_like(o.hist_f)
                self.hist_c = np.zeros_like(o.hist_c)
                self.hist_both = np.zeros_like(o.hist_both)
            self.hist_f += o.hist_f
            self.hist_c += o.hist_c
            self.hist_both += o.hist_both

    def mean(self):
        return self.sy / self.n if self.n else 0.0

    def var(self):
        if self.n < 2:
            return 0.0
        return max(0.0, (self.sy2 - self.sy * self.sy / self.n) / (self.n - 1))

    def cost(self):
        return (self.events_f + self.events_c) / self.n if self.n else 0.0


def level_sums(problem: Problem, level: int, xf, xc, ef, ec) -> LevelSums:
    qf = qoi_values(problem, xf)
    if level == 0:
        qc = np.zeros_like(qf)
        y = qf
    else:
        qc = qoi_values(problem, xc)
        if problem.periodic() or problem.qoi == QOI_X:
            y = qf - qc
        else:
            y = (xf - xc) * (xf + xc)     # x_f^2 - x_c^2 without cancellation
    s = LevelSums(n=len(xf), sy=float(np.sum(y)), sy2=float(np.sum(y * y)),
                  sqf=float(np.sum(qf)), sqf2=float(np.sum(qf * qf)),
                  sqc=float(np.sum(qc)), sqc2=float(np.sum(qc * qc)),
                  events_f=int(np.sum(ef)), events_c=int(np.sum(ec)))
    if problem.nbins > 0:
        nb = problem.nbins
        bf = bin_index(problem, xf)
        hf = np.bincount(bf[bf >= 0], minlength=nb).astype(np.int64)
        if level == 0:
            hc = np.zeros(nb, np.int64)
            hb = np.zeros(nb, np.int64)
        else:
            bc = bin_index(problem, xc)
            hc = np.bincount(bc[bc >= 0], minlength=nb).astype(np.int64)
            same = (bf == bc) & (bf >= 0)
            hb = np.bincount(bf[same], minlength=nb).astype(np.int64)
        s.hist_f, s.hist_c, s.hist_both = hf, hc, hb
    return s


def run_level(problem: Problem, level: int, first: int, count: int, threads: int = 1) -> LevelSums:
    xf, xc, ef, ec = pairs(problem, level, first, count, threads)
    return level_sums(problem, level, xf, xc, ef, ec)


# --------------------------------------------------------------------------
# Adaptive MLMC (eqs. mse, statistical_contraint, Nopt1, Noptj; Sec. 4.1).
# --------------------------------------------------------------------------
def level_variance(problem: Problem, s: LevelSums) -> float:
    """V_l of the quantity that sets N_l.  For a density QoI: the largest bin
    variance of the per-bin density difference (sup norm over bins)."""
    if problem.qoi == QOI_DENSITY and problem.nbins > 0 and s.n >= 2:
        lo, hi = problem.bin_range()
        h = (hi - lo) / problem.nbins
        sy = (s.hist_f - s.hist_c).astype(np.float64)
        sy2 = (s.hist_f + s.hist_c - 2 * s.hist_both).astype(np.float64)
        v = (sy2 - sy * sy / s.n) / (s.n - 1)
        return float(max(0.0, v.max())) / (h * h)
    return s.var()


def level_select(V, Vd):
    """Heuristic level selection (Alg. 3): the first level l whose
    difference variance Vd[l] = Var(Q_l - Q_{l-1}) is below V[l] = Var(Q_l),
    with the level below it; then each later level whose Vd is below half of
    the last selected one.  The finest level L is always kept (the estimator
    ends there).  Without any such l: the single level L."""
    L = len(V) - 1
    l = 1
    while l <= L and Vd[l] > V[l]:
        l += 1
    if l > L:
        return [L]
    chosen = [l - 1, l]
    vmin = Vd[l]
    for k in range(l + 1, L + 1):
        if Vd[k] < vmin / 2.0:
            chosen.append(k)
            vmin = Vd[k]
    if chosen[-1] != L:
        chosen.append(L)
    return chosen


def v_pair_approx(V_i, V_j, rho_Li, rho_Lj):
    """Sec. 4.2, eq. V_approx: V_{i,j} ~ V_i + V_j - 2 sqrt((rho_{L,i}^2 +
    rho_{L,j}^2 - 1) V_i V_j), rho_{i,j} taken as the geometric mean of its
    bounds.  A negative argument of the root (the bounds admit rho_{i,j} = 0)
    is read as 0: V_{i,j} = V_i + V_j."""
    arg = (rho_Li * rho_Li + rho_Lj * rho_Lj - 1.0) * V_i * V_j
    return V_i + V_j - 2.0 * math.sqrt(max(arg, 0.0))


def level_set_cost(levels, V, rho, C):
    """Cost of eq. level_selection for the level set `levels` (increasing,
    ending at L): sqrt(V_{l1} C_{l1}) + sum_j sqrt(V_{lj,lj-1} C_{lj,lj-1}),
    with V_{i,j} from eq. V_approx (rho_{L,L} = 1) and C_{i,j} = C_i + C_j
    (cost measured in KD events of both paths of a pair)."""
    r = list(rho) + [1.0]
    total = math.sqrt(V[levels[0]] * C[levels[0]])
    for a, b in zip(levels[:-1], levels[1:]):
        total += math.sqrt(max(v_pair_approx(V[b], V[a], r[b], r[a]), 0.0) * (C[a] + C[b]))
    return total


def level_select_opt(V, rho, C):
    """Sec. 4.2: the level set containing L with the smallest cost of eq.
    level_selection, found by trying every subset of 0..L-1 (the plain
    definition; the library solves the same problem as a shortest path)."""
    L = len(V) - 1
    best, best_set = None, None
    for mask in range(1 << L):
        levels = [i for i in range(L) if mask >> i & 1] + [L]
        c = level_set_cost(levels, V, rho, C)
        if best is None or c < best:
            best, best_set = c, levels
    return best_set


def level_pilot(problem: Problem, n: int, threads: int = 1):
    """Pilot statistics of Sec. 4.2 for a scalar QoI: n pairs coupling L
    with each level i < L (level sets {i, L}; the fine path of pair p is the
    same in every coupling).  Returns V[0..L] (variance of F on each level),
    rho[0..L-1] (correlation of F(x_L) with F(x_i)) and C[0..L] (KD events per
    path).  Level i comes from the coarse path of the (i, L) coupling, level L
    from the fine path of the (L-1, L) one."""
    L = problem.L
    V, C, rho = [0.0] * (L + 1), [0.0] * (L + 1), [0.0] * L
    for i in range(L):
        q = Problem(**{**problem.__dict__, "level_set": [i, L], "n_fixed": []})
        xf, xc, ef, ec = pairs(q, 1, 0, n, threads)
        ff, fc = qoi_values(q, xf), qoi_values(q, xc)
        cov = np.cov(ff, fc, ddof=1)
        V[i] = float(cov[1, 1])
        C[i] = float(np.mean(ec))
        rho[i] = float(cov[0, 1] / math.sqrt(cov[0, 0] * cov[1, 1])) if cov[0, 0] * cov[1, 1] > 0 else 0.0
        if i == L - 1:
            V[L] = float(cov[0, 0])
            C[L] = float(np.mean(ef))
    return V, rho, C


def warmup_tau(problem: Problem) -> int:
    """Sec. 5.3: the level tau with dt_tau near 1/R, read as the first level
    l >= 1 whose step is at most 1/R; the finest level L when none is."""
    for l in range(1, problem.L + 1):
        if problem.R * problem.dt(l) <= 1.0:
            return l
    return problem.L


def level_warmup(problem: Problem, n_warmup: int = 100, threads: int = 1):
    """Off-line phase of Sec. 5.3 for a scalar QoI: n_warmup samples on levels
    0..tau give V_l (variance of F(x_l)) and V_{l,l-1} (variance of Y_l); past
    tau, V_{l,l-1} follows the asymptotic O(dt_l^3) decay from its value on
    tau, and V_l keeps its value on tau.  Returns (V, Vd, tau), Vd[0] = 0,
    the input of level_select (Alg. 3)."""
    L = problem.L
    tau = warmup_tau(problem)
    V, Vd = [0.0] * (L + 1), [0.0] * (L + 1)
    for l in range(tau + 1):
        xf, xc, ef, ec = pairs(problem, l, 0, n_warmup, threads)
        qf = qoi_values(problem, xf)
        V[l] = float(np.var(qf, ddof=1))
        if l > 0:
            y = qf - qoi_values(problem, xc)
            Vd[l] = float(np.var(y, ddof=1))
    for l in range(tau + 1, L + 1):
        V[l] = V[tau]
        Vd[l] = Vd[tau] * float(problem.M) ** (-3 * (l - tau))
    return V, Vd, tau


def optimal_counts(V, C, tol):
    """N_j = ceil(2/tol^2 sqrt(V_j/C_j) sum_i sqrt(V_i C_i))  (eqs. Nopt1/Noptj)."""
    total = sum(math.sqrt(v * c) for v, c in zip(V, C))
    out = []
    for v, c in zip(V, C):
        if v <= 0.0 or c <= 0.0:
            out.append(0)
        else:
            out.append(int(math.ceil(2.0 / (tol * tol) * math.sqrt(v / c) * total)))
    return out


@dataclass
class MLMCResult:
    estimate: float
    variance: float
    levels: list
    density: np.ndarray = None


def _result(problem: Problem, sums) -> MLMCResult:
    est = sum(s.mean() for s in sums)
    var = sum(level_variance(problem, s) / s.n for s in sums if s.n > 0)
    dens = None
    if problem.nbins > 0:
        lo, hi = problem.bin_range()
        h = (hi - lo) / problem.nbins
        dens = sum((s.hist_f - s.hist_c) / s.n for s in sums) / h
    return MLMCResult(est, var, sums, dens)


def estimate_sequence(problem: Problem, tols, threads: int = 1, max_rounds: int = 64):
    """On-line phase of Sec. 5.3: one MLMC estimator run for a decreasing
    sequence of RMSE tolerances, keeping its samples from one tolerance to the
    next.  Each stage raises N_l to the optimal counts for its tolerance
    (eqs. Nopt1/Noptj) until no level needs more.  Returns one result per
    tolerance (each with a snapshot of the level sums)."""
    import copy
    J = len(problem.estimator_levels())
    sums = [LevelSums() for _ in range(J)]
    for l in range(J):
        sums[l].add(run_level(problem, l, 0, problem.n_warmup, threads))
    out = []
    for tol in tols:
        for _ in range(max_rounds):
            V = [level_variance(problem, s) for s in sums]
            C = [s.cost() for s in sums]
            target = optimal_counts(V, C, tol)
            grew = False
            for l in range(J):
                if target[l] > sums[l].n:
                    sums[l].add(run_level(problem, l, sums[l].n, target[l] - sums[l].n, threads))
                    grew = True
            if not grew:
                break
        out.append(_result(problem, copy.deepcopy(sums)))
    return out


def estimate(problem: Problem, threads: int = 1, max_rounds: int = 64) -> MLMCResult:
    """Adaptive MLMC on levels 0..L: warm-up, then grow N_l to the optimal
    counts until the statistical constraint holds."""
    J = len(problem.estimator_levels())
    sums = [LevelSums() for _ in range(J)]
    if problem.n_fixed:
        for l in range(J):
            sums[l].add(run_level(problem, l, 0, int(problem.n_fixed[l]), threads))
    else:
        for l in range(J):
            sums[l].add(run_level(problem, l, 0, problem.n_warmup, threads))
        for _ in range(max_rounds):
            V = [level_variance(problem, s) for s in sums]
            C = [s.cost() for s in sums]
            target = optimal_counts(V, C, problem.tol)
            grew = False
            for l in range(J):
                if target[l] > sums[l].n:
                    sums[l].add(run_level(problem, l, sums[l].n, target[l] - sums[l].n, threads))
                    grew = True
            if not grew:
                break
    return _result(problem, sums)


# --------------------------------------------------------------------------
# Heterogeneous backgrounds B1/B2 (Sec. 5): mu = 0, sigma = 1, piecewise-linear
# R(x) = b (1 + a_left max(1 - x, 0) + a_right max(x - 1, 0)); B1 has
# a_left = a_right = a, B2 a_left = 0, a_right = a.  Levels dt_l = dt0 M^-l.
# --------------------------------------------------------------------------
BG_B1, BG_B2 = 1, 2


def het_bg(kind: int, a: float, b: float) -> HetBg:
    return HetBg(b, a if kind == BG_B1 else 0.0, a)


def het_R(bg: HetBg, x: float) -> float:
    return lib().orc_het_R(ctypes.byref(bg), x)


def het_depth(bg: HetBg, x0: float, v: float, dt: float, u: float) -> float:
    """int_0^u R(x0 + v dt w) dt dw (steps u; negative u: the segment behind)."""
    return lib().orc_het_depth(ctypes.byref(bg), x0, v, dt, u)


def het_flight(bg: HetBg, x0: float, v: float, dt: float, E: float) -> float:
    """Flight in steps from x0 at velocity v that collects optical depth E (eq. intinv)."""
    return lib().orc_het_flight(ctypes.byref(bg), x0, v, dt, E)


def _het_desc(kind, a, b, T, dt0, M, level, coupled, x0, seed, request, recipe, coarsening):
    r = T / dt0
    n0 = int(round(r))
    if n0 < 1 or abs(r - n0) > 1e-12 * max(1.0, r):
        raise ValueError("T/dt0 must be a positive integer")
    d = HetDesc()
    d.bg = het_bg(kind, a, b)
    d.dt = dt0 / float(M) ** level
    d.n = n0 * M ** level
    d.M = coarsening if coarsening else M
    d.level, d.recipe, d.coupled = level, recipe, 1 if coupled else 0
    d.seed, d.request, d.x0 = seed, request, x0
    return d


def het_coarse_draws(kind, a, b, T, dt0, M, level, first, count, cap, x0=1.0, seed=0, request=0,
                     coarsening=None):
    """(nu~, E~, chi~) of every coarse step of heterogeneous pairs, in order;
    the coarse step is dt * coarsening (default M)."""
    d = _het_desc(kind, a, b, T, dt0, M, level, True, x0, seed, request, RECIPE_53, coarsening)
    nu, E, chi = np.zeros(cap), np.zeros(cap), np.zeros(cap)
    dd = ctypes.c_double
    w = lib().orc_het_coarse_draws(ctypes.byref(d), first, count, cap, _ptr(nu, dd), _ptr(E, dd),
                                   _ptr(chi, dd))
    if w < 0:
        raise RuntimeError("oracle heterogeneous coarse draws failed")
    return nu[:w], E[:w], chi[:w]


def het_pairs(kind, a, b, T, dt0, M, level, coupled, first, count, x0=1.0, seed=0, request=0,
              recipe=RECIPE_53, coarsening=None, threads=1):
    """Final positions and event counts of pairs [first, first + count) of
    fine level `level` (dt = dt0 M^-level) in background B1/B2; coupled pairs
    couple with the step dt * coarsening (default M)."""
    r = T / dt0
    n0 = int(round(r))
    if n0 < 1 or abs(r - n0) > 1e-12 * max(1.0, r):
        raise ValueError("T/dt0 must be a positive integer")
    d = HetDesc()
    d.bg = het_bg(kind, a, b)
    d.dt = dt0 / float(M) ** level
    d.n = n0 * M ** level
    d.M = coarsening if coarsening else M
    d.level, d.recipe, d.coupled = level, recipe, 1 if coupled else 0
    d.seed, d.request, d.x0 = seed, request, x0
    xf, xc = np.zeros(count), np.zeros(count)
    ef, ec = np.zeros(count, np.int64), np.zeros(count, np.int64)
    L = lib()
    threads = max(1, min(int(threads), count if count > 0 else 1))
    bounds = np.linspace(0, count, threads + 1).astype(np.int64)

    def work(t):
        lo, hi = int(bounds[t]), int(bounds[t + 1])
        if hi <= lo:
            return 0
        dd, i64 = ctypes.c_double, ctypes.c_int64
        return L.orc_het_pairs(ctypes.byref(d), first + lo, hi - lo,
                               ctypes.cast(xf.ctypes.data + 8 * lo, ctypes.POINTER(dd)),
                               ctypes.cast(xc.ctypes.data + 8 * lo, ctypes.POINTER(dd)),
                               ctypes.cast(ef.ctypes.data + 8 * lo, ctypes.POINTER(i64)),
                               ctypes.cast(ec.ctypes.data + 8 * lo, ctypes.POINTER(i64)))

    if threads == 1:
        rcs = [work(0)]
    else:
        with ThreadPoolExecutor(threads) as ex:
            rcs = list(ex.map(work, range(threads)))
    if any(rc != 0 for rc in rcs):
        raise RuntimeError("oracle heterogeneous pair simulation failed: %r" % rcs)
    return xf, xc, ef, ec
