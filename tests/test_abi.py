"""The C-ABI library builds, loads and exports every entry point that include/amg.h declares
(no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "amg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(amg_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2103_10476_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("amg_setup", "amg_solve", "amg_free", "amg_params_default", "amg_level_info", "amg_export",
                 "amg_spgemm", "amg_vcycle"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_params_defaults_and_status_strings(libpath):
    from paper_2103_10476_gb300 import amg
    p = amg.amg_params_default()
    assert (p.theta, p.variants, p.tau, p.cheb_degree, p.cheb_ratio, p.power_iters, p.max_coarse) == \
        (0.0, 0, 1.1, 2, 10.0, 10, 500)
    assert p.sigma == 1.0 / 3.0 and p.precision == amg.AMG_FP64 and p.pt_scaling == amg.AMG_PT_ORTHONORMAL
    assert amg.amg_status_string(amg.AMG_ERR_EIGEN).startswith("eigenvalue")


def test_invalid_arguments_rejected_without_device_work(libpath):
    # argument checks run before any CUDA call
    from paper_2103_10476_gb300 import amg
    p = amg.amg_params_default(theta=2.0)
    A = amg.amg_csr_t(0, 0, None, None, None, 0)
    h, s = amg.amg_setup_status(A, None, p)
    assert h is None and s == amg.AMG_ERR_INVALID_ARG
    A = amg.amg_csr_t(-1, 0, None, None, None, 0)
    h, s = amg.amg_setup_status(A, None, amg.amg_params_default())
    assert s == amg.AMG_ERR_INVALID_ARG
