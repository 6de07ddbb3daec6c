"""Host-side checks of the C-ABI library (no GPU needed): it loads and exports
every function that include/hk.h declares."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hk.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hk_[A-Za-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_0902_0852_gb300 import build, hk
    build.build()
    return hk.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["hk_load_moments", "hk_factor", "hk_smallest_eig", "hk_create", "hk_destroy",
                     "hk_get_R", "hk_strerror", "hk_workspace_bytes", "hk_set_workspace"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_export_list_matches_header():
    from paper_0902_0852_gb300 import hk
    assert sorted(hk.EXPORTS) == declared_functions()


def test_strerror_and_argument_checks_without_gpu(lib):
    assert lib.hk_strerror(0) == b"ok"
    assert b"positive definite" in lib.hk_strerror(2)
    import ctypes
    b = ctypes.c_size_t()
    assert lib.hk_workspace_bytes(0, 64, ctypes.byref(b)) == 1      # N < 1
    assert lib.hk_workspace_bytes(10, 48, ctypes.byref(b)) == 1     # P not a multiple of 32
    assert lib.hk_workspace_bytes(10, 64, ctypes.byref(b)) == 0 and b.value > 0


def test_pack_roundtrip():
    from paper_0902_0852_gb300 import hk, inputs
    vals = inputs.moments(6, (7, 4), 96) + [(0, 0), (-(1 << 95) - 5, -7)]
    assert hk.unpack(*hk.pack(vals, 96)) == vals


def test_every_entry_point_rejects_a_null_context_or_bad_argument(lib):
    """Status codes, never an abort: with no context (or an out-of-range
    operation) every entry point returns HK_ERR_ARG without touching a GPU."""
    ARG = 1
    calls = [
        lambda: lib.hk_create(None, 0, None),
        lambda: lib.hk_set_workspace(None, None, 0),
        lambda: lib.hk_load_moments(None, 4, 1, 1, 64, None),
        lambda: lib.hk_load_moments_flat(None, 4, 1, 1, 64, None, None, None, 0),
        lambda: lib.hk_factor(None, None),
        lambda: lib.hk_get_R(None, None),
        lambda: lib.hk_get_R_flat(None, None, None, None),
        lambda: lib.hk_smallest_eig(None, 1, None, None),
        lambda: lib.hk_get_history_flat(None, 1, None, None, None),
        lambda: lib.hk_get_timings(None, None, 1),
        lambda: lib.hk_get_stats(None, None, 1),
        lambda: lib.hk_set_update_path(None, 0),
        lambda: lib.hk_set_option(None, 0, 0),
        lambda: lib.hk_batch_solve(None, 1, None, None, None, None, None, 0, 1, None, None, None),
        lambda: lib.hk_set_predictor(None, None, None),
        lambda: lib.hk_predict(None, 1, None, None, None),
        lambda: lib.hk_selftest_mp(9, 1, None, 0, 0, None, 0, 0, None, None),
        lambda: lib.hk_mp_op_noalloc(9, 1, None, 0, 0, None, 0, 0, None, None, None),
        lambda: lib.hk_probe_int_peaks(0, None, 0),
        lambda: lib.hk_mlp_forward(None, None, 0, None, None),
        lambda: lib.hk_update_plan(0, -1, None, None, None, None, None, 0, None),
        lambda: lib.hk_selftest_wait(None),
        lambda: lib.hk_ldlt_det(None, None, None, None, None),
        lambda: lib.hk_get_ldlt_flat(None, 0, None, None, None),
        lambda: lib.hk_secant(None, 10, None, None),
        lambda: lib.hk_get_secant_flat(None, 0, None, None, None, None, None, None),
        lambda: lib.hk_secant_verify(None, None, 130, 512, None),
        lambda: lib.hk_time_update_slice(None, 16, None, None),
        lambda: lib.hk_selftest_scalar(9, 1, None, None, None, None),
    ]
    for k, call in enumerate(calls):
        assert call() == ARG, k
