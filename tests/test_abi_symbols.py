"""The C-ABI library builds, loads without a GPU and exports every function the public
header declares; the ctypes table matches the header (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mdpgpu.h")


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"^\s*typedef[^;]*;", "", text, flags=re.M)  # callback types are not entry points
    names = re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(\w+)\s*\(", text, flags=re.M)
    return sorted({n for n in names if n not in ("if", "while", "for", "return", "sizeof")})


@pytest.fixture(scope="module")
def built():
    from paper_2211_04299_gb300 import build
    return build.build()


def test_header_lists_the_expected_entry_points():
    names = header_functions()
    for must in ["mdp_create_dense", "mdp_create_ell", "bellman_apply", "policy_eval_gmres",
                 "ipi_solve", "vi_solve", "pi_solve", "opi_solve", "mdp_destroy"]:
        assert must in names


def test_library_exports_every_header_symbol(built):
    lib = ctypes.CDLL(built)
    missing = [n for n in header_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_ctypes_table_matches_header(built):
    from paper_2211_04299_gb300 import _lib
    assert sorted(_lib.SIGNATURES) == header_functions()
    lib = _lib.load(built)
    assert lib.mdp_version().decode().startswith("mdpgpu")
    o = lib.mdp_opts_default()
    assert o.restart == 30 and abs(o.alpha - 0.1) < 1e-15 and o.precision == 1
    assert o.forcing_c == 0.0 and not o.v0 and o.precond_block == 0


def test_invalid_arguments_fail_before_any_device_work(built):
    """Argument checks happen on the host before the CUDA runtime is touched."""
    from paper_2211_04299_gb300 import _lib
    lib = _lib.load(built)
    h = ctypes.c_void_p()
    assert lib.mdp_create_dense(0, 1, None, 0, None, 0.9, None, ctypes.byref(h)) == _lib.MDP_EINVAL
    assert b"S must be" in lib.mdp_last_error()
    assert lib.mdp_create_ell(4, 1, 9, None, None, 0, None, 0.9, None, ctypes.byref(h)) == _lib.MDP_EINVAL
    assert lib.mdp_create_ell(4, 1, 2, None, None, 0, None, 1.5, None, ctypes.byref(h)) == _lib.MDP_EINVAL
    assert lib.ipi_solve(None, None, None, None, None) == _lib.MDP_EINVAL
    assert lib.mdp_set_geometry(None, 0, 0, 0) == _lib.MDP_EINVAL
    # batches: argument and option checks precede any device work
    b = ctypes.c_void_p()
    assert lib.mdp_batch_create(None, 0, None, ctypes.byref(b)) == _lib.MDP_EINVAL
    one = (ctypes.c_void_p * 1)(None)
    assert lib.mdp_batch_create(one, 1, None, None) == _lib.MDP_EINVAL
    o = lib.mdp_opts_default()
    o.precision = _lib.MDP_PREC_FP64
    assert lib.mdp_batch_create(one, 1, ctypes.byref(o), ctypes.byref(b)) == _lib.MDP_EINVAL
    assert b"MIXED" in lib.mdp_last_error()
    o = lib.mdp_opts_default()
    o.restart = 0
    assert lib.mdp_batch_create(one, 1, ctypes.byref(o), ctypes.byref(b)) == _lib.MDP_EINVAL
    o = lib.mdp_opts_default()
    o.forcing_c = -1.0
    assert lib.mdp_batch_create(one, 1, ctypes.byref(o), ctypes.byref(b)) == _lib.MDP_EINVAL
    assert b"forcing_c" in lib.mdp_last_error()
    o = lib.mdp_opts_default()
    o.precond_block = 256  # the two-level preconditioner is an ipi_solve option
    assert lib.mdp_batch_create(one, 1, ctypes.byref(o), ctypes.byref(b)) == _lib.MDP_EINVAL
    assert b"precond_block" in lib.mdp_last_error()
    assert not b.value
    assert lib.mdp_batch_solve(None, None, None, None) == _lib.MDP_EINVAL
    assert lib.mdp_batch_solve_dev(None, None, None, None) == _lib.MDP_EINVAL
    assert lib.mdp_batch_geometry(None, 0, None, None, None, None, None) == _lib.MDP_EINVAL
    assert lib.mdp_batch_tune(None) == _lib.MDP_EINVAL
    assert lib.mdp_batch_set_stream(None, None) == _lib.MDP_EINVAL
    assert lib.mdp_batch_device_bytes(None) == 0
    assert lib.ipi_solve_batch(None, 0, None, None, None, None) == _lib.MDP_EINVAL
    lib.mdp_batch_destroy(None)
    # servers: option checks precede any device work
    so = lib.mdp_server_opts_default()
    assert so.max_slots == 256 and so.iters_per_launch == 4 and so.hbm_budget_bytes == 120 << 30
    srv = ctypes.c_void_p()
    for field, bad in (("max_slots", 0), ("iters_per_launch", 0), ("hbm_budget_bytes", 0)):
        so = lib.mdp_server_opts_default()
        setattr(so, field, bad)
        assert lib.mdp_server_create(ctypes.byref(so), ctypes.byref(srv)) == _lib.MDP_EINVAL
    so = lib.mdp_server_opts_default()
    so.solver.precision = _lib.MDP_PREC_FP64
    assert lib.mdp_server_create(ctypes.byref(so), ctypes.byref(srv)) == _lib.MDP_EINVAL
    so = lib.mdp_server_opts_default()
    so.solver.precond_block = 256
    assert lib.mdp_server_create(ctypes.byref(so), ctypes.byref(srv)) == _lib.MDP_EINVAL
    assert b"precond_block" in lib.mdp_last_error()
    assert lib.mdp_server_create(None, None) == _lib.MDP_EINVAL
    assert lib.mdp_server_submit(None, 1, 1, 1, None, None, None, 0.9, None, None, None) == _lib.MDP_EINVAL
    assert lib.mdp_server_poll(None, None, None, 0, None) == _lib.MDP_EINVAL
    assert lib.mdp_server_drain(None) == _lib.MDP_EINVAL
    assert lib.mdp_server_info(None, None, None, None, None) == _lib.MDP_EINVAL
    lib.mdp_server_destroy(None)


def test_no_cpu_fallback_when_library_missing(tmp_path):
    from paper_2211_04299_gb300 import _lib
    saved = _lib._LIB
    _lib._LIB = None
    try:
        with pytest.raises(ImportError):
            _lib.load(str(tmp_path / "libmdpgpu.so"))
    finally:
        _lib._LIB = saved
