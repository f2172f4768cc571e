"""Plain FP64 CPU oracle for parallel tempering of the 3D Heisenberg spin glass.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the engine in
``paper_1006_4247_gb300`` never does.  It shares no code with the CUDA engine.

The arithmetic lives in ``pt_oracle.c`` (plain C, double precision, one site at
a time, in the order Hasenbusch & Schaefer, arXiv:1006.4247, state it).  This
module only compiles it with gcc and marshals numpy arrays through ctypes.

Parity status of each function (what pins it; see ``tests/test_oracle_*``):
  philox4x32_10      cuRAND's host Philox4_32_10 generator (library run, not read)
  hb_update          exact CDF inversion F(c(r)) = r; Langevin mean; KS test;
                     the paper's printed formula (section III.C) at moderate R
  or_update          involution, conservation of s.S, reflection geometry
  energy / overlap   brute force over all site pairs; rotation invariance
  exchange_plain     crafted energies: acceptance = min(1, e^Delta) exactly
  decimation_lnA     Gauss-Legendre quadrature of I(beta S); beta1 = beta2 => 0
  cool/heat sweeps   inverse property; finite-difference Jacobians (per site and
                     the whole 2N-dimensional map at L = 2); eps = 0 limit
  pt_run             beta = 0 closed forms; high-temperature series of <H>;
                     all three exchanges give the same <H>(beta)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pt_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile pt_oracle.c into oracle/_build/liboracle.so with gcc."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-std=c11",
           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_u64 = C.c_uint64
_u32 = C.c_uint32


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            sig = {
                "orc_philox4x32_10": (None, [_u32p, _u32p, _u32p]),
                "orc_rng_words": (None, [_u64, _u32, _u32, _u32, _u64, _u32, _u32p]),
                "orc_local_field": (None, [C.c_int, _dp, _dp, C.c_int, _dp]),
                "orc_energy": (C.c_double, [C.c_int, _dp, _dp]),
                "orc_overlap": (C.c_double, [C.c_int, _dp, _dp, _dp]),
                "orc_onb": (None, [_dp, _dp, _dp]),
                "orc_hb_t": (C.c_double, [C.c_double, C.c_double]),
                "orc_hb_update": (None, [C.c_double, _dp, _u32, _u32, _dp]),
                "orc_or_update": (None, [_dp, _dp]),
                "orc_hb_halfsweep": (None, [C.c_int, _dp, _dp, C.c_int, C.c_double,
                                            _u64, _u32, _u32, _u64, _u32]),
                "orc_or_halfsweep": (None, [C.c_int, _dp, _dp, C.c_int]),
                "orc_hb_sweep_typewriter": (None, [C.c_int, _dp, _dp, C.c_double,
                                                   _u64, _u32, _u32, _u64]),
                "orc_or_sweep_typewriter": (None, [C.c_int, _dp, _dp]),
                "orc_init_spins": (None, [C.c_int, _dp, C.c_int, _u64, _u32, _u32]),
                "orc_roundtrip_update": (None, [C.c_int, _i32p, _i32p, _i64p]),
                "orc_exchange_plain": (None, [C.c_int, C.c_int, _dp, _dp, _dp, _i32p,
                                              _i32p, _i64p, _i64p, _i64p, _u64, _u32,
                                              _u32, _u64]),
                "orc_ln_sinhc": (C.c_double, [C.c_double]),
                "orc_decimation_lnA": (C.c_double, [C.c_int, _dp, _dp, _dp, C.c_int,
                                                    C.c_double, C.c_double]),
                "orc_exchange_decimation": (None, [C.c_int, _dp, C.c_int, _dp, _dp,
                                                   _dp, _i32p, _i32p, _i64p, _i64p,
                                                   _i64p, _u64, _u32, _u32, _u64]),
                "orc_cool_site": (C.c_double, [C.c_double, _dp, _dp]),
                "orc_heat_site": (C.c_double, [C.c_double, _dp, _dp]),
                "orc_kepler_solve": (C.c_double, [C.c_double, C.c_double]),
                "orc_cool_sweep": (C.c_double, [C.c_int, _dp, _dp, C.c_double]),
                "orc_heat_sweep": (C.c_double, [C.c_int, _dp, _dp, C.c_double]),
                "orc_coolheat_lnA": (C.c_double, [C.c_int, _dp, _dp, _dp, C.c_double,
                                                  C.c_double, C.c_double, C.c_double,
                                                  C.c_double, _dp, _dp,
                                                  C.POINTER(C.c_double),
                                                  C.POINTER(C.c_double)]),
                "orc_test_set_jacobian_variant": (None, [C.c_int]),
                "orc_exchange_coolheat": (None, [C.c_int, _dp, C.c_int, _dp, _dp, _dp,
                                                 _dp, _i32p, _i32p, _i64p, _i64p,
                                                 _i64p, _u64, _u32, _u32, _u64]),
                "orc_pt_run": (None, [C.c_int, _dp, C.c_int, _dp, _dp, C.c_int, _dp,
                                      _dp, _i32p, _i32p, _i64p, _i64p, _i64p, C.c_int,
                                      C.c_int, C.c_int, C.c_int, C.c_int, _u64, _u32,
                                      C.POINTER(C.c_uint64), C.c_void_p, C.c_void_p,
                                      C.c_void_p]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# Random numbers
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    """Philox4x32-10 block: four 32-bit counter words, two key words."""
    out = np.zeros(4, np.uint32)
    _load().orc_philox4x32_10(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def rng_words(seed, sample, c0, c1, step, purpose):
    out = np.zeros(4, np.uint32)
    _load().orc_rng_words(seed, sample, c0, c1, step, purpose, out)
    return out


# --------------------------------------------------------------------------
# Lattice, single-site moves
# --------------------------------------------------------------------------
def local_field(L, J, s, x):
    S = np.zeros(3)
    _load().orc_local_field(L, _d(J).ravel(), _d(s).ravel(), int(x), S)
    return S


def energy(L, J, s):
    """H = -sum_<xy> J_xy s_x.s_y (J as [3, N], s as [N, 3])."""
    return _load().orc_energy(L, _d(J).ravel(), _d(s).ravel())


def overlap(L, s1, s2):
    """Return (Q[3,3], chi) for two configurations."""
    Q = np.zeros(9)
    chi = _load().orc_overlap(L, _d(s1).ravel(), _d(s2).ravel(), Q)
    return Q.reshape(3, 3), chi


def onb(n):
    e1 = np.zeros(3)
    e2 = np.zeros(3)
    _load().orc_onb(_d(n), e1, e2)
    return e1, e2


def hb_t(R, q):
    return _load().orc_hb_t(float(R), float(q))


def hb_update(beta, S, w0, w1):
    out = np.zeros(3)
    _load().orc_hb_update(float(beta), _d(S), int(w0), int(w1), out)
    return out


def or_update(S, s):
    s = _d(s).copy()
    _load().orc_or_update(_d(S), s)
    return s


def hb_halfsweep(L, J, s, color, beta, seed, sample, rep_id, step, purpose=0):
    s = _d(s).copy()
    _load().orc_hb_halfsweep(L, _d(J).ravel(), s.reshape(-1), int(color), float(beta),
                             seed, sample, rep_id, step, purpose)
    return s


def or_halfsweep(L, J, s, color):
    s = _d(s).copy()
    _load().orc_or_halfsweep(L, _d(J).ravel(), s.reshape(-1), int(color))
    return s


def init_spins(L, mode, seed, sample, rep_id):
    s = np.zeros((L ** 3, 3))
    _load().orc_init_spins(L, s.reshape(-1), int(mode), seed, sample, rep_id)
    return s


# --------------------------------------------------------------------------
# Exchanges (one chain)
# --------------------------------------------------------------------------
class Chain:
    """State of one chain (sample, copy): configs by beta index, H, labels,
    round-trip state and per-pair counters, all numpy arrays."""

    def __init__(self, L, J, betas, spins, copy=0, sample=0, seed=0):
        self.L = L
        self.J = _d(J).reshape(3, -1).copy()
        self.betas = _d(betas).copy()
        self.NT = len(betas)
        self.spins = _d(spins).reshape(self.NT, L ** 3, 3).copy()
        self.copy = copy
        self.sample = sample
        self.seed = seed
        self.H = np.array([energy(L, self.J, self.spins[b]) for b in range(self.NT)])
        self.label = np.arange(self.NT, dtype=np.int32)
        self.rt_state = np.zeros(self.NT, np.int32)
        self.rt_state[0] = 1
        self.rt_count = np.zeros(1, np.int64)
        self.prop = np.zeros(self.NT - 1, np.int64)
        self.acc = np.zeros(self.NT - 1, np.int64)

    def exchange(self, mode, step, eps=None):
        lib = _load()
        sp = self.spins.reshape(-1)
        if mode == 0:
            lib.orc_exchange_plain(self.L, self.NT, self.betas, sp, self.H, self.label,
                                   self.rt_state, self.rt_count, self.prop, self.acc,
                                   self.seed, self.sample, self.copy, step)
        elif mode == 1:
            lib.orc_exchange_decimation(self.L, self.J.ravel(), self.NT, self.betas, sp,
                                        self.H, self.label, self.rt_state, self.rt_count,
                                        self.prop, self.acc, self.seed, self.sample,
                                        self.copy, step)
        else:
            e = _d(np.broadcast_to(np.asarray(eps, np.float64), (self.NT - 1,)))
            lib.orc_exchange_coolheat(self.L, self.J.ravel(), self.NT, self.betas, e, sp,
                                      self.H, self.label, self.rt_state, self.rt_count,
                                      self.prop, self.acc, self.seed, self.sample,
                                      self.copy, step)


def roundtrip_update(label, rt_state, rt_count):
    _load().orc_roundtrip_update(len(label), label, rt_state, rt_count)


def ln_sinhc(R):
    return _load().orc_ln_sinhc(float(R))


def decimation_lnA(L, J, s1, s2, d, b1, b2):
    return _load().orc_decimation_lnA(L, _d(J).ravel(), _d(s1).ravel(), _d(s2).ravel(),
                                      int(d), float(b1), float(b2))


def cool_site(eps, S, s):
    s = _d(s).copy()
    lj = _load().orc_cool_site(float(eps), _d(S), s)
    return s, lj


def heat_site(eps, S, s):
    s = _d(s).copy()
    lj = _load().orc_heat_site(float(eps), _d(S), s)
    return s, lj


def kepler_solve(e, thp):
    return _load().orc_kepler_solve(float(e), float(thp))


def cool_sweep(L, J, s, eps):
    s = _d(s).copy()
    lj = _load().orc_cool_sweep(L, _d(J).ravel(), s.reshape(-1), float(eps))
    return s, lj


def heat_sweep(L, J, s, eps):
    s = _d(s).copy()
    lj = _load().orc_heat_sweep(L, _d(J).ravel(), s.reshape(-1), float(eps))
    return s, lj


def coolheat_lnA(L, J, s1, s2, H1, H2, b1, b2, eps):
    N = L ** 3
    t1 = np.zeros(3 * N)
    t2 = np.zeros(3 * N)
    Hc = C.c_double()
    Hh = C.c_double()
    lnA = _load().orc_coolheat_lnA(L, _d(J).ravel(), _d(s1).ravel(), _d(s2).ravel(),
                                   float(H1), float(H2), float(b1), float(b2),
                                   float(eps), t1, t2, C.byref(Hc), C.byref(Hh))
    return lnA, t1.reshape(N, 3), t2.reshape(N, 3), Hc.value, Hh.value


class jacobian_variant:
    """Test hook (context manager): run the cooling/heating acceptance with
    the Jacobian of the heated configuration taken at its pre-image (0, the
    default and the only correct choice), at the heated configuration itself
    (1, the printed formula read literally) or left out (2), so that a test
    can show that the exactness check detects the wrong choices."""

    def __init__(self, v):
        self.v = int(v)

    def __enter__(self):
        _load().orc_test_set_jacobian_variant(self.v)
        return self

    def __exit__(self, *exc):
        _load().orc_test_set_jacobian_variant(0)
        return False


# --------------------------------------------------------------------------
# Whole runs of one sample
# --------------------------------------------------------------------------
class Run:
    """One sample with n_copies chains, advanced by ``cycles``."""

    def __init__(self, L, J, betas, n_copies=2, seed=0, sample=0, start=0,
                 spins=None, eps=None):
        self.L, self.N = L, L ** 3
        self.J = _d(J).reshape(3, -1).copy()
        self.betas = _d(betas).copy()
        self.NT = len(betas)
        self.C = n_copies
        self.seed, self.sample = seed, sample
        if spins is None:
            spins = np.stack([np.stack([init_spins(L, start, seed, sample, c * self.NT + b)
                                        for b in range(self.NT)]) for c in range(n_copies)])
        self.spins = _d(spins).reshape(n_copies, self.NT, self.N, 3).copy()
        self.eps = _d(np.zeros(self.NT - 1) if eps is None else
                      np.broadcast_to(np.asarray(eps, np.float64), (self.NT - 1,)))
        self.H = np.zeros((n_copies, self.NT))
        self.label = np.tile(np.arange(self.NT, dtype=np.int32), (n_copies, 1))
        self.rt_state = np.zeros((n_copies, self.NT), np.int32)
        self.rt_state[:, 0] = 1
        self.rt_count = np.zeros(n_copies, np.int64)
        self.prop = np.zeros((n_copies, self.NT - 1), np.int64)
        self.acc = np.zeros((n_copies, self.NT - 1), np.int64)
        self.step = C.c_uint64(0)

    def cycles(self, n_cycles, n_hb=1, n_or=1, mode=0, order=0, record=True):
        Hs = np.zeros((n_cycles, self.C, self.NT)) if record else None
        chis = np.zeros((n_cycles, self.NT)) if (record and self.C == 2) else None
        Qs = np.zeros((n_cycles, self.NT, 9)) if (record and self.C == 2) else None
        ptr = lambda a: None if a is None else a.ctypes.data_as(C.c_void_p)
        _load().orc_pt_run(self.L, self.J.ravel(), self.NT, self.betas, self.eps, self.C,
                           self.spins.reshape(-1), self.H.reshape(-1),
                           self.label.reshape(-1), self.rt_state.reshape(-1),
                           self.rt_count, self.prop.reshape(-1), self.acc.reshape(-1),
                           int(n_cycles), int(n_hb), int(n_or), int(mode), int(order),
                           self.seed, self.sample, C.byref(self.step),
                           ptr(Hs), ptr(chis), ptr(Qs))
        return Hs, chis, Qs
