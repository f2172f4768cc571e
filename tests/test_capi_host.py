"""CPU checks of the C-ABI library: it builds for sm_103a, loads without a GPU,
exports every entry point that include/pt.h declares, and rejects invalid
arguments on the host before any device work."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1006_4247_gb300 import _build, pt
    _build.build()
    return pt.load_library()


def _declared():
    src = open(os.path.join(ROOT, "include", "pt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pt_[a-z_]+)\s*\(", src)) - {"pt_alloc_fn", "pt_free_fn"})


def test_header_entry_points_exported(lib):
    from paper_1006_4247_gb300 import pt
    names = _declared()
    assert len(names) >= 19
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(pt.ENTRY_POINTS) == names


def test_options_default_and_struct_layout(lib):
    from paper_1006_4247_gb300 import pt
    o = pt.pt_options_default()
    assert (o.n_samples, o.n_copies, o.precision, o.seed, o.start) == (1, 2, 0, 0, 0)
    assert C.sizeof(pt.PtOptions) == 64


def _create(L, J, B, NT, **kw):
    from paper_1006_4247_gb300 import pt
    o = pt.pt_options_default()
    for k, v in kw.items():
        setattr(o, k, v)
    h = C.c_void_p()
    lib = pt.load_library()
    Jp = J.ctypes.data_as(C.POINTER(C.c_float)) if J is not None else None
    Bp = B.ctypes.data_as(C.POINTER(C.c_double)) if B is not None else None
    return lib.pt_create(C.byref(h), L, Jp, Bp, NT, C.byref(o)), lib.pt_last_error().decode()


@pytest.mark.parametrize("L", [3, 5, 1, 0, -4])
def test_rejects_odd_or_small_L(lib, L):
    from paper_1006_4247_gb300 import pt
    J = np.zeros((3, max(L, 1) ** 3), np.float32)
    B = np.array([1.0, 2.0])
    st, msg = _create(L, J, B, 2)
    assert st == pt.PT_ERR_ODD_L and "even" in msg


def test_rejects_bad_arguments(lib):
    from paper_1006_4247_gb300 import pt
    L = 4
    J = np.random.default_rng(0).standard_normal((3, L ** 3)).astype(np.float32)
    assert _create(L, J, np.array([2.0, 1.0]), 2)[0] == pt.PT_ERR_ARG          # not increasing
    assert _create(L, J, np.array([-1.0, 1.0]), 2)[0] == pt.PT_ERR_ARG         # negative beta
    assert _create(L, J, np.array([1.0]), 1)[0] == pt.PT_ERR_ARG               # one replica
    assert _create(L, J, np.array([1.0, np.nan]), 2)[0] == pt.PT_ERR_ARG
    Jn = J.copy(); Jn[1, 5] = np.inf
    st, msg = _create(L, Jn, np.array([1.0, 2.0]), 2)
    assert st == pt.PT_ERR_ARG and "coupling" in msg
    assert _create(L, J, np.array([1.0, 2.0]), 2, n_copies=3)[0] == pt.PT_ERR_ARG
    assert _create(L, J, np.array([1.0, 2.0]), 2, precision=7)[0] == pt.PT_ERR_ARG
    assert _create(L, None, np.array([1.0, 2.0]), 2)[0] == pt.PT_ERR_ARG
    assert lib.pt_sweep(None, 1, 1) == pt.PT_ERR_ARG
    assert lib.pt_destroy(None) == pt.PT_OK


def test_python_binding_fails_loudly_without_library(tmp_path):
    from paper_1006_4247_gb300 import pt
    with pytest.raises(ImportError):
        # a fresh loader pointed at a missing file must not fall back to anything
        import importlib
        mod = importlib.reload(pt)
        mod._lib = None
        mod.load_library(str(tmp_path / "missing.so"))
    importlib.reload(pt)


def test_handle_calls_reject_null_on_the_host(lib):
    """Every call that takes a handle returns PT_ERR_ARG for a NULL handle
    (or NULL output) without touching a device."""
    from paper_1006_4247_gb300 import pt
    i = C.c_int(0)
    codes = (C.c_int * 2)(14, 4)
    u = C.c_uint64(0)
    assert lib.pt_sweep_samples(None, 1, codes) == pt.PT_ERR_ARG
    assert lib.pt_cycles(None, 1, 1, 1, None, 0, 0) == pt.PT_ERR_ARG
    assert lib.pt_exchange(None, 0, None) == pt.PT_ERR_ARG
    assert lib.pt_measure(None, None, None, None) == pt.PT_ERR_ARG
    assert lib.pt_get_paths(None, codes, None) == pt.PT_ERR_ARG
    assert lib.pt_set_paths(None, codes) == pt.PT_ERR_ARG
    assert lib.pt_set_wait_limit(None, 16, 1) == pt.PT_ERR_ARG
    assert lib.pt_set_policy(None, 0) == pt.PT_ERR_ARG
    assert lib.pt_get_rng_step(None, C.byref(u)) == pt.PT_ERR_ARG
    assert lib.pt_profile(None, 1) == pt.PT_ERR_ARG
    assert lib.pt_save(None, b"x") == pt.PT_ERR_ARG
    assert lib.pt_mlp_destroy(None) in (pt.PT_OK, pt.PT_ERR_ARG)
    assert "NULL" in lib.pt_last_error().decode()
