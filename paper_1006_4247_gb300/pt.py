"""Python binding of the C ABI in include/pt.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: all of the sweep, exchange and measurement work runs
in the CUDA kernels of libpt.so.  If the library has not been built the first
call raises; there is no fallback.

PyTorch, when present, supplies the CUDA stream (``torch.cuda.current_stream``)
and may own the device memory through the allocator callback
(``use_torch_allocator=True``).
"""
from __future__ import annotations

import ctypes as C
import json
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpt.so")

PT_OK, PT_ERR_ARG, PT_ERR_ODD_L, PT_ERR_EPS, PT_ERR_CUDA, PT_ERR_TIMEOUT, PT_ERR_STATE, PT_ERR_NOMEM = (
    0, -1, -2, -3, -4, -5, -6, -7)
PT_PLAIN, PT_DECIMATION, PT_COOLHEAT = 0, 1, 2
PT_FP32, PT_FP64 = 0, 1
PT_START_RANDOM, PT_START_ORDERED = 0, 1
MODES = {"plain": PT_PLAIN, "decimation": PT_DECIMATION, "coolheat": PT_COOLHEAT}

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

# Entry points declared in include/pt.h (the symbol test checks this list
# against the header).
ENTRY_POINTS = ["pt_options_default", "pt_create", "pt_create_batch", "pt_sweep", "pt_sweep_samples",
                "pt_cycles", "pt_autotune", "pt_get_paths", "pt_set_paths", "pt_exchange",
                "pt_measure", "pt_measure_device", "pt_get_stats", "pt_get_exchange_log", "pt_get_spins",
                "pt_set_spins",
                "pt_set_params", "pt_set_rng_step", "pt_get_rng_step", "pt_save", "pt_load",
                "pt_profile", "pt_profile_read", "pt_set_policy", "pt_set_wait_limit", "pt_energy_noalloc",
                "pt_smem_bandwidth",
                "pt_destroy",
                "pt_last_error", "pt_mlp_create", "pt_mlp_num_params", "pt_mlp_set_params",
                "pt_mlp_get_params", "pt_mlp_forward", "pt_mlp_loss_grad", "pt_mlp_train", "pt_mlp_ladder",
                "pt_mlp_destroy"]
PT_KERNEL_KINDS = 7
KERNEL_KINDS = ["hb", "or", "energy", "exchange", "measure", "other", "resident"]
PT_POLICY_AUTO, PT_POLICY_STREAMING, PT_POLICY_RESIDENT = 0, 1, 2
POLICIES = {"auto": 0, "streaming": 1, "resident": 2}


class PtOptions(C.Structure):
    _fields_ = [("n_samples", C.c_int), ("n_copies", C.c_int), ("precision", C.c_int),
                ("seed", C.c_uint64), ("start", C.c_int), ("stream", C.c_void_p),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", C.c_void_p)]


class PtError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"pt status {status}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None


def load_library(path: str = LIB_PATH):
    """Load libpt.so; raise if it was not built (no fallback exists)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise ImportError(f"{path} not found: build the engine first "
                                  "(python -c 'import __graft_entry__ as g; g.build()')")
            lib = C.CDLL(path)
            vp, ip, dp, fp = C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_float)
            i64p, i32p = C.POINTER(C.c_int64), C.POINTER(C.c_int32)
            sig = {
                "pt_options_default": (None, [C.POINTER(PtOptions)]),
                "pt_create": (ip, [C.POINTER(vp), ip, fp, dp, ip, C.POINTER(PtOptions)]),
                "pt_create_batch": (ip, [C.POINTER(vp), ip, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                         C.POINTER(fp), C.POINTER(dp), C.POINTER(PtOptions)]),
                "pt_sweep": (ip, [vp, ip, ip]),
                "pt_sweep_samples": (ip, [vp, ip, C.POINTER(C.c_int)]),
                "pt_cycles": (ip, [vp, ip, ip, ip, C.POINTER(C.c_int), ip, ip]),
                "pt_autotune": (ip, [vp, ip, ip, C.POINTER(C.c_int), dp]),
                "pt_get_paths": (ip, [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
                "pt_set_paths": (ip, [vp, C.POINTER(C.c_int)]),
                "pt_exchange": (ip, [vp, ip, fp]),
                "pt_measure": (ip, [vp, dp, dp, dp]),
                "pt_measure_device": (ip, [vp, vp, vp, vp]),
                "pt_profile": (ip, [vp, ip]),
                "pt_profile_read": (ip, [vp, dp, i64p]),
                "pt_set_policy": (ip, [vp, ip]),
                "pt_set_wait_limit": (ip, [vp, C.c_ulonglong, ip]),
                "pt_energy_noalloc": (ip, [vp, ip, ip, ip, vp, vp, vp]),
                "pt_smem_bandwidth": (ip, [vp, dp, dp, dp]),
                "pt_get_stats": (ip, [vp, i64p, i64p, i64p, i32p]),
                "pt_get_exchange_log": (ip, [vp, dp, dp]),
                "pt_get_spins": (ip, [vp, ip, ip, ip, dp]),
                "pt_set_spins": (ip, [vp, ip, ip, ip, dp]),
                "pt_set_params": (ip, [vp, dp, fp]),
                "pt_set_rng_step": (ip, [vp, C.c_uint64]),
                "pt_get_rng_step": (ip, [vp, C.POINTER(C.c_uint64)]),
                "pt_save": (ip, [vp, C.c_char_p]),
                "pt_load": (ip, [vp, C.c_char_p]),
                "pt_destroy": (ip, [vp]),
                "pt_last_error": (C.c_char_p, []),
                "pt_mlp_create": (ip, [C.POINTER(vp), ip, C.c_uint64, vp]),
                "pt_mlp_num_params": (ip, [vp]),
                "pt_mlp_set_params": (ip, [vp, fp]),
                "pt_mlp_get_params": (ip, [vp, fp, C.POINTER(C.c_uint16)]),
                "pt_mlp_forward": (ip, [vp, ip, fp, fp]),
                "pt_mlp_loss_grad": (ip, [vp, ip, fp, fp, C.c_float, fp, fp]),
                "pt_mlp_train": (ip, [vp, ip, fp, fp, C.c_float, ip, C.c_float, fp]),
                "pt_mlp_ladder": (ip, [vp, ip, fp, dp, dp, C.POINTER(C.c_int), ip, C.c_float, C.c_double, dp, fp]),
                "pt_mlp_destroy": (ip, [vp]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(st):
    if st != PT_OK:
        raise PtError(st, load_library().pt_last_error().decode(errors="replace"))


def _ptr(a, ctype):
    return None if a is None else a.ctypes.data_as(C.POINTER(ctype))


def pt_last_error() -> str:
    return load_library().pt_last_error().decode(errors="replace")


def pt_options_default() -> PtOptions:
    o = PtOptions()
    load_library().pt_options_default(C.byref(o))
    return o


def pt_create(L, couplings, betas, n_replicas, opt: PtOptions | None = None):
    """couplings float32 [S, 3, L^3]; betas float64 [S, n_replicas]."""
    J = np.ascontiguousarray(couplings, np.float32)
    B = np.ascontiguousarray(betas, np.float64)
    h = C.c_void_p()
    _check(load_library().pt_create(C.byref(h), int(L), _ptr(J, C.c_float), _ptr(B, C.c_double),
                                    int(n_replicas), None if opt is None else C.byref(opt)))
    return h


def pt_create_batch(L, n_replicas, couplings, betas, opt: PtOptions | None = None):
    """Per-sample lists: L[s], n_replicas[s], couplings[s] float32 [3, L^3],
    betas[s] float64 [n_replicas[s]]."""
    S = len(L)
    Ls = (C.c_int * S)(*[int(v) for v in L])
    NTs = (C.c_int * S)(*[int(v) for v in n_replicas])
    Js = [np.ascontiguousarray(j, np.float32) for j in couplings]
    Bs = [np.ascontiguousarray(b, np.float64) for b in betas]
    Jp = (C.POINTER(C.c_float) * S)(*[_ptr(j, C.c_float) for j in Js])
    Bp = (C.POINTER(C.c_double) * S)(*[_ptr(b, C.c_double) for b in Bs])
    h = C.c_void_p()
    _check(load_library().pt_create_batch(C.byref(h), S, Ls, NTs, Jp, Bp,
                                          None if opt is None else C.byref(opt)))
    return h


def pt_sweep(h, n_hb, n_or):
    _check(load_library().pt_sweep(h, int(n_hb), int(n_or)))


def pt_sweep_samples(h, n_hb, n_or):
    a = np.ascontiguousarray(n_or, np.int32)
    _check(load_library().pt_sweep_samples(h, int(n_hb), _ptr(a, C.c_int)))


def pt_cycles(h, n_cycles, n_hb, n_or, mode, measure=False, n_or_samples=None):
    mode = MODES.get(mode, mode) if isinstance(mode, str) else int(mode)
    a = None if n_or_samples is None else np.ascontiguousarray(n_or_samples, np.int32)
    _check(load_library().pt_cycles(h, int(n_cycles), int(n_hb), int(n_or), _ptr(a, C.c_int), mode,
                                    int(bool(measure))))


def pt_autotune(h, n_hb, n_or, n_samples):
    """Return (choice[S], best_ms[S]); choice = sites per thread, +10 if resident."""
    choice = np.zeros(n_samples, np.int32)
    best = np.zeros(n_samples)
    _check(load_library().pt_autotune(h, int(n_hb), int(n_or), _ptr(choice, C.c_int), _ptr(best, C.c_double)))
    return choice, best


def pt_set_paths(h, choice):
    c = np.ascontiguousarray(choice, np.int32)
    _check(load_library().pt_set_paths(h, _ptr(c, C.c_int)))


def autotune_cache_key(L, NT, copies, precision, n_hb, n_or, device_name):
    """Key of an autotuner result: the batch shape, precision, block and GPU."""
    return json.dumps({"L": [int(v) for v in L], "NT": [int(v) for v in NT], "copies": int(copies),
                       "precision": precision, "n_hb": int(n_hb), "n_or": int(n_or), "gpu": device_name},
                      sort_keys=True)


def pt_exchange(h, mode, eps=None):
    mode = MODES.get(mode, mode) if isinstance(mode, str) else int(mode)
    e = None if eps is None else np.ascontiguousarray(eps, np.float32)
    _check(load_library().pt_exchange(h, mode, _ptr(e, C.c_float)))


def pt_measure(h, energy=None, overlap=None, chi=None):
    """Fill the given float64 arrays (any may be None)."""
    _check(load_library().pt_measure(h, _ptr(energy, C.c_double), _ptr(overlap, C.c_double),
                                     _ptr(chi, C.c_double)))


def pt_measure_device(h, d_energy=None, d_overlap=None, d_chi=None):
    """Enqueue the reductions into device buffers (integer device pointers or
    None) without synchronising."""
    _check(load_library().pt_measure_device(h, d_energy, d_overlap, d_chi))


def pt_profile(h, enable):
    _check(load_library().pt_profile(h, int(enable)))


def pt_profile_read(h):
    """Return ({kind: ms}, {kind: launches}) since the last pt_profile call."""
    ms = np.zeros(PT_KERNEL_KINDS)
    n = np.zeros(PT_KERNEL_KINDS, np.int64)
    _check(load_library().pt_profile_read(h, _ptr(ms, C.c_double), _ptr(n, C.c_int64)))
    return dict(zip(KERNEL_KINDS, ms.tolist())), dict(zip(KERNEL_KINDS, n.tolist()))


def pt_set_policy(h, policy):
    policy = POLICIES.get(policy, policy) if isinstance(policy, str) else int(policy)
    _check(load_library().pt_set_policy(h, policy))


def pt_set_wait_limit(h, limit=0, inject=False):
    _check(load_library().pt_set_wait_limit(h, int(limit), 1 if inject else 0))


def pt_energy_noalloc(d_spins, precision, L, n_configs, d_couplings, d_energy, stream=None):
    """Energies of n_configs configurations in caller-owned device memory
    (integer device pointers), without any allocation by the library; see
    include/pt.h for the layout, the scratch limit and the ordering rules."""
    precision = PT_FP64 if precision in ("fp64", PT_FP64) else PT_FP32
    _check(load_library().pt_energy_noalloc(d_spins, precision, int(L), int(n_configs), d_couplings,
                                            d_energy, stream))


def pt_smem_bandwidth(stream=None):
    """(bytes/s over all SMs, bytes per clock per SM, SM MHz) of the measured
    shared-memory load stream on the current device."""
    out = [C.c_double(), C.c_double(), C.c_double()]
    _check(load_library().pt_smem_bandwidth(stream, *[C.byref(o) for o in out]))
    return tuple(o.value for o in out)


def pt_get_stats(h, proposals=None, accepts=None, round_trips=None, perm=None):
    _check(load_library().pt_get_stats(h, _ptr(proposals, C.c_int64), _ptr(accepts, C.c_int64),
                                       _ptr(round_trips, C.c_int64), _ptr(perm, C.c_int32)))


def pt_get_exchange_log(h, lnA=None, lnJ=None):
    _check(load_library().pt_get_exchange_log(h, _ptr(lnA, C.c_double), _ptr(lnJ, C.c_double)))


def pt_get_spins(h, sample, copy, replica, out):
    _check(load_library().pt_get_spins(h, int(sample), int(copy), int(replica), _ptr(out, C.c_double)))


def pt_set_spins(h, sample, copy, replica, xyz):
    a = np.ascontiguousarray(xyz, np.float64)
    _check(load_library().pt_set_spins(h, int(sample), int(copy), int(replica), _ptr(a, C.c_double)))


def pt_set_params(h, betas=None, eps=None):
    b = None if betas is None else np.ascontiguousarray(betas, np.float64)
    e = None if eps is None else np.ascontiguousarray(eps, np.float32)
    _check(load_library().pt_set_params(h, _ptr(b, C.c_double), _ptr(e, C.c_float)))


def pt_set_rng_step(h, step):
    _check(load_library().pt_set_rng_step(h, int(step)))


def pt_get_rng_step(h) -> int:
    v = C.c_uint64()
    _check(load_library().pt_get_rng_step(h, C.byref(v)))
    return int(v.value)


def pt_save(h, path):
    _check(load_library().pt_save(h, os.fsencode(path)))


def pt_load(h, path):
    _check(load_library().pt_load(h, os.fsencode(path)))


def pt_destroy(h):
    _check(load_library().pt_destroy(h))


# --------------------------------------------------------------------------
# Convenience wrapper: shapes, numpy outputs, torch stream / allocator.
# --------------------------------------------------------------------------
def _torch_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


class _TorchAllocator:
    """Device memory from PyTorch's caching allocator."""

    def __init__(self):
        import torch
        self.torch = torch
        self.dev = torch.cuda.current_device()

        def _alloc(n, ctx):
            return int(torch.cuda.caching_allocator_alloc(int(n), self.dev))

        def _free(p, ctx):
            torch.cuda.caching_allocator_delete(int(p))

        self.alloc = ALLOC_FN(_alloc)
        self.free = FREE_FN(_free)


class Engine:
    """A batch of disorder samples with shapes kept on the Python side."""

    def __init__(self, L, couplings, betas, n_copies=2, precision="fp32", seed=0,
                 start="random", stream=None, use_torch_allocator=False):
        uneven = isinstance(L, (list, tuple))
        opt = pt_options_default()
        opt.n_copies = n_copies
        opt.precision = PT_FP64 if precision in ("fp64", PT_FP64) else PT_FP32
        opt.seed = seed & 0xFFFFFFFFFFFFFFFF
        opt.start = PT_START_ORDERED if start in ("ordered", PT_START_ORDERED) else PT_START_RANDOM
        st = _torch_stream() if stream is None else stream
        opt.stream = st
        self.precision = "fp64" if opt.precision == PT_FP64 else "fp32"
        self.seed = int(opt.seed)
        self._alloc = None
        if use_torch_allocator:
            self._alloc = _TorchAllocator()
            opt.alloc = self._alloc.alloc
            opt.free = self._alloc.free
        self.C = n_copies
        if uneven:
            self.L = [int(v) for v in L]
            self.NT = [len(b) for b in betas]
            opt.n_samples = len(self.L)
            self.h = pt_create_batch(self.L, self.NT, couplings, betas, opt)
        else:
            J = np.asarray(couplings, np.float32)
            if J.ndim == 2:
                J = J[None]
            B = np.asarray(betas, np.float64)
            if B.ndim == 1:
                B = np.broadcast_to(B, (J.shape[0], B.size))
            opt.n_samples = J.shape[0]
            self.L = [int(L)] * J.shape[0]
            self.NT = [B.shape[1]] * J.shape[0]
            self.h = pt_create(L, J, B, B.shape[1], opt)
        self.S = len(self.L)
        self.uniform = not uneven
        self.R = sum(self.C * n for n in self.NT)
        self.P = sum(self.C * (n - 1) for n in self.NT)

    # shapes -------------------------------------------------------------
    def _shape(self, per_sample, rect):
        return rect if self.uniform else (per_sample,)

    def sweep(self, n_hb=1, n_or=1):
        pt_sweep(self.h, n_hb, n_or)

    def exchange(self, mode="plain", eps=None):
        pt_exchange(self.h, mode, eps)

    def sweep_samples(self, n_hb, n_or):
        pt_sweep_samples(self.h, n_hb, n_or)

    def cycles(self, n_cycles, n_hb=1, n_or=1, mode="plain", measure=False, n_or_samples=None):
        pt_cycles(self.h, n_cycles, n_hb, n_or, mode, measure, n_or_samples)

    def paths(self):
        """Per-sample sweep path codes (see pt_get_paths) and CTAs per replica."""
        ch = (C.c_int * self.S)()
        ct = (C.c_int * self.S)()
        _check(load_library().pt_get_paths(self.h, ch, ct))
        return np.array(ch[:], np.int32), np.array(ct[:], np.int32)

    def autotune(self, n_hb=1, n_or=1, cache=None):
        """Time the candidate paths (pt_autotune) and return (choice, best_ms).
        With `cache` (a JSON file), a result stored there for the same batch
        shape, precision, block and GPU is applied with pt_set_paths instead
        of timing again, and a new result is stored."""
        key = None
        if cache:
            import torch
            key = autotune_cache_key(self.L, self.NT, self.C, self.precision, n_hb, n_or,
                                     torch.cuda.get_device_name())
            table = {}
            if os.path.exists(cache):
                with open(cache) as fh:
                    table = json.load(fh)
            if key in table:
                choice = np.array(table[key]["choice"], np.int32)
                self.set_paths(choice)
                return choice, np.array(table[key]["best_ms"])
        choice, best = pt_autotune(self.h, n_hb, n_or, self.S)
        if cache:
            table = {}
            if os.path.exists(cache):
                with open(cache) as fh:
                    table = json.load(fh)
            table[key] = {"choice": choice.tolist(), "best_ms": best.tolist()}
            tmp = cache + ".tmp"
            with open(tmp, "w") as fh:
                json.dump(table, fh, indent=1)
            os.replace(tmp, cache)
        return choice, best

    def set_paths(self, choice):
        """Apply per-sample path codes (the encoding of pt_get_paths)."""
        pt_set_paths(self.h, choice)

    def energies(self):
        out = np.zeros(self.R)
        pt_measure(self.h, energy=out)
        return out.reshape(self.S, self.C, self.NT[0]) if self.uniform else out

    def overlap(self):
        n = sum(self.NT)
        Q = np.zeros(n * 9)
        chi = np.zeros(n)
        pt_measure(self.h, overlap=Q, chi=chi)
        if self.uniform:
            return Q.reshape(self.S, self.NT[0], 3, 3), chi.reshape(self.S, self.NT[0])
        return Q.reshape(n, 3, 3), chi

    def measure(self):
        n = sum(self.NT)
        H = np.zeros(self.R)
        Q = np.zeros(n * 9) if self.C == 2 else None
        chi = np.zeros(n) if self.C == 2 else None
        pt_measure(self.h, H, Q, chi)
        return H, Q, chi

    def set_policy(self, policy):
        pt_set_policy(self.h, policy)

    def set_wait_limit(self, limit=0, inject=False):
        """Poll limit of the bounded device-side waits (0: default) and the
        hook that makes one of them run out (see pt_set_wait_limit)."""
        pt_set_wait_limit(self.h, limit, inject)

    def measure_device(self, d_energy=None, d_overlap=None, d_chi=None):
        """Enqueue the reductions; results also go to the given device
        tensors (float64, contiguous, the layouts of pt_measure), if any."""
        ptr = lambda t: None if t is None else int(t.data_ptr())
        pt_measure_device(self.h, ptr(d_energy), ptr(d_overlap), ptr(d_chi))

    def profile(self, enable=True):
        pt_profile(self.h, enable)

    def profile_read(self):
        return pt_profile_read(self.h)

    def stats(self):
        prop = np.zeros(self.P, np.int64)
        acc = np.zeros(self.P, np.int64)
        rt = np.zeros(self.S * self.C, np.int64)
        perm = np.zeros(self.R, np.int32)
        pt_get_stats(self.h, prop, acc, rt, perm)
        if self.uniform:
            NT = self.NT[0]
            return (prop.reshape(self.S, self.C, NT - 1), acc.reshape(self.S, self.C, NT - 1),
                    rt.reshape(self.S, self.C), perm.reshape(self.S, self.C, NT))
        return prop, acc, rt, perm

    def exchange_log(self):
        """(ln A, ln det J terms) of every pair's most recent proposal; shapes
        [S][C][NT-1] and [S][C][NT-1][2] for a uniform batch, flat otherwise."""
        lnA = np.zeros(self.P)
        lnJ = np.zeros(2 * self.P)
        pt_get_exchange_log(self.h, lnA, lnJ)
        if self.uniform:
            NT = self.NT[0]
            return lnA.reshape(self.S, self.C, NT - 1), lnJ.reshape(self.S, self.C, NT - 1, 2)
        return lnA, lnJ.reshape(-1, 2)

    def get_spins(self, sample, copy, replica):
        out = np.zeros((self.L[sample] ** 3, 3))
        pt_get_spins(self.h, sample, copy, replica, out)
        return out

    def set_spins(self, sample, copy, replica, xyz):
        pt_set_spins(self.h, sample, copy, replica, xyz)

    def set_params(self, betas=None, eps=None):
        pt_set_params(self.h, betas, eps)

    @property
    def step(self):
        return pt_get_rng_step(self.h)

    @step.setter
    def step(self, v):
        pt_set_rng_step(self.h, v)

    def save(self, path):
        pt_save(self.h, path)

    def load(self, path):
        pt_load(self.h, path)

    def close(self):
        if getattr(self, "h", None) is not None:
            pt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ---------------------------------------------------------------- learned ladder
MLP_IN, MLP_HIDDEN, MLP_MAX_KNOTS = 4, 64, 64


def mlp_num_params(n_knots: int) -> int:
    """Size of the float parameter vector of a net with n_knots knots."""
    N = 2 * n_knots + 1
    return MLP_HIDDEN * MLP_IN + MLP_HIDDEN + MLP_HIDDEN * MLP_HIDDEN + MLP_HIDDEN + N * MLP_HIDDEN + N


class Mlp:
    """The ladder network behind pt_mlp_* (argument marshalling only)."""

    def __init__(self, n_knots: int, seed: int = 1, stream=None):
        lib = load_library()
        h = C.c_void_p()
        s = None if stream is None else C.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
        _check(lib.pt_mlp_create(C.byref(h), int(n_knots), C.c_uint64(seed), s))
        self.h = h
        self.n_knots = int(n_knots)
        self.n_params = lib.pt_mlp_num_params(h)

    @staticmethod
    def _rows(x):
        x = np.ascontiguousarray(x, np.float32)
        if x.ndim != 2 or x.shape[1] != MLP_IN:
            raise ValueError(f"features must be [batch, {MLP_IN}]")
        return x

    def _targets(self, x, t):
        t = np.ascontiguousarray(t, np.float32)
        if t.shape != (x.shape[0], 2 * self.n_knots + 1):
            raise ValueError(f"targets must be [batch, {2 * self.n_knots + 1}]")
        return t

    def params(self):
        """(master float32 [n], bfloat16 bits uint16 [n])."""
        p = np.zeros(self.n_params, np.float32)
        b = np.zeros(self.n_params, np.uint16)
        _check(load_library().pt_mlp_get_params(self.h, _ptr(p, C.c_float), _ptr(b, C.c_uint16)))
        return p, b

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        if p.shape != (self.n_params,):
            raise ValueError(f"expected {self.n_params} parameters")
        _check(load_library().pt_mlp_set_params(self.h, _ptr(p, C.c_float)))

    def forward(self, x):
        x = self._rows(x)
        z = np.zeros((x.shape[0], 2 * self.n_knots + 1), np.float32)
        _check(load_library().pt_mlp_forward(self.h, x.shape[0], _ptr(x, C.c_float), _ptr(z, C.c_float)))
        return z

    def loss_grad(self, x, t, w_kappa=1.0):
        x = self._rows(x)
        t = self._targets(x, t)
        loss = C.c_float()
        g = np.zeros(self.n_params, np.float32)
        _check(load_library().pt_mlp_loss_grad(self.h, x.shape[0], _ptr(x, C.c_float), _ptr(t, C.c_float),
                                               C.c_float(w_kappa), C.byref(loss), _ptr(g, C.c_float)))
        return float(loss.value), g

    def train(self, x, t, steps, lr=1e-3, w_kappa=1.0, record=False):
        """Full-batch Adam on the device; returns the per-step losses when
        record is set (one synchronisation per step), else None."""
        x = self._rows(x)
        t = self._targets(x, t)
        losses = np.zeros(max(int(steps), 1), np.float32) if record else None
        _check(load_library().pt_mlp_train(self.h, x.shape[0], _ptr(x, C.c_float), _ptr(t, C.c_float),
                                           C.c_float(w_kappa), int(steps), C.c_float(lr),
                                           _ptr(losses, C.c_float)))
        return None if losses is None else losses[:int(steps)]

    def ladder(self, x, beta_min, beta_max, n_temps, kappa_max, sigma_target=0.0, max_temps=512):
        """Per row: (betas float64 [NT], eps float32 [NT - 1]).  n_temps <= 0
        lets the net choose NT for the acceptance of sigma_target (at most
        max_temps)."""
        x = self._rows(x)
        B = x.shape[0]
        bmin = np.ascontiguousarray(np.broadcast_to(beta_min, (B,)), np.float64)
        bmax = np.ascontiguousarray(np.broadcast_to(beta_max, (B,)), np.float64)
        nt = np.array(np.broadcast_to(n_temps, (B,)), np.int32)
        stride = int(max(nt.max(), max_temps if (nt <= 0).any() else 2))
        betas = np.zeros((B, stride), np.float64)
        eps = np.zeros((B, stride - 1), np.float32)
        _check(load_library().pt_mlp_ladder(self.h, B, _ptr(x, C.c_float), _ptr(bmin, C.c_double),
                                            _ptr(bmax, C.c_double), _ptr(nt, C.c_int), stride,
                                            C.c_float(kappa_max), C.c_double(sigma_target),
                                            _ptr(betas, C.c_double), _ptr(eps, C.c_float)))
        return [(betas[r, :nt[r]].copy(), eps[r, :nt[r] - 1].copy()) for r in range(B)]

    def close(self):
        if getattr(self, "h", None) is not None:
            pt_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def pt_mlp_destroy(h):
    _check(load_library().pt_mlp_destroy(h))
