"""The C ABI library builds, loads and exports every entry point that
include/gbs.h declares (CPU only: no call here touches a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gbs.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gbs_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2011_00715_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["gbs_ctx_create", "gbs_mat_create_aij", "gbs_mat_mult", "gbs_vec_axpy",
                     "gbs_vec_aypx", "gbs_vec_dot", "gbs_vec_norm2", "gbs_pc_jacobi_create",
                     "gbs_pc_apply", "gbs_ksp_solve_cg", "gbs_ksp_solve_cg_batched",
                     "gbs_server_submit"]:
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True)
    exported = set(re.findall(r"\bT (gbs_\w+)", out.stdout))
    assert set(declared_functions()) <= exported


def test_host_only_calls(libpath):
    from paper_2011_00715_gb300 import gbs
    assert "sm_103a" in gbs.gbs_version()
    assert gbs.gbs_status_string(gbs.GBS_ERR_TIMEOUT) == "device-side wait timed out"
    assert gbs.gbs_status_string(12345) == "unknown status"
    o = gbs.gbs_opts_default()
    assert (o.mode, o.algorithm, o.inner_rtol, o.outer_maxit, o.barrier_timeout_ms,
            o.fault_skip_arrival) == (gbs.GBS_MODE_FP64, gbs.GBS_ALG_AUTO, 1e-4, 30, 2000, -1)
    assert gbs.lib().gbs_opts_default(None) == gbs.GBS_ERR_ARG
    # argument checks that never reach the device
    assert gbs.lib().gbs_ctx_create(0, None, None, None) == gbs.GBS_ERR_ARG
    assert gbs.lib().gbs_mat_destroy(None) == gbs.GBS_OK
    assert gbs.lib().gbs_vec_destroy(None) == gbs.GBS_OK
    assert gbs.lib().gbs_ksp_solve_cg(None, None, None, 1e-8, 10, None, None) == gbs.GBS_ERR_ARG


def test_status_codes_match_header():
    from paper_2011_00715_gb300 import gbs
    text = open(HEADER).read()
    for name, val in re.findall(r"\b(GBS_(?:OK|DIVERGED_ITS|ERR_[A-Z]+))\s*=\s*(-?\d+)", text):
        assert getattr(gbs, name) == int(val), name


def test_enums_and_limits_match_header():
    from paper_2011_00715_gb300 import gbs
    text = open(HEADER).read()
    found = re.findall(r"\b(GBS_(?:ALG|MODE|NORM)_[A-Z0-9]+)\s*=\s*(-?\d+)", text)
    found += re.findall(r"#define\s+(GBS_[A-Z_]+_MAX_ROWS)\s+(\d+)", text)
    assert any(n == "GBS_ALG_CLUSTER" for n, _ in found)
    for name, val in found:
        assert getattr(gbs, name) == int(val), name


def test_binding_names_are_the_abi_names():
    from paper_2011_00715_gb300 import gbs
    for n in declared_functions():
        assert callable(getattr(gbs, n, None)), n
