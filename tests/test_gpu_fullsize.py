"""Parity at the benchmark's full sizes, in the launch configuration bench.py times (matrix,
right-hand side and solution resident on the device, the solve on torch's current stream).

stretched64 (262,144 unknowns, 6.86M entries; the five methods the benchmark steps through),
randcoef128 (2,097,152 unknowns, 55.7M entries; 1Norm + OffLmp, FP64 and mixed) and the
nonsymmetric convdiff64 (262,144 unknowns; GMRES(30), FP64 and mixed) and the elasticity
system (201,720 unknowns, three per node, six rigid-body modes; FP64 and mixed): the whole hierarchy
against the oracle's (integer structures bit-exact, values within VAL_TOL), PCG or GMRES
iterations by the rule of the small-size tests, solutions within SOL_TOL, and the
relative residual ||b - A x|| / ||b|| recomputed here on the host with scipy.
"""
import numpy as np
import pytest

from paper_2103_10476_gb300 import problems as P
from tests.gpu_common import SOL_TOL, compare_hierarchies, gpu_params, iterations_agree

pytestmark = pytest.mark.gpu

TOL = 1e-8


@pytest.fixture(scope="module")
def amg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2103_10476_gb300 import build
    build.build()
    from paper_2103_10476_gb300 import amg as m
    return m


def _device_solve(amg, A, b, **kw):
    import torch
    stream = torch.cuda.current_stream()
    rp, ci, v = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (A.row_ptr, A.col, A.val))
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    p = gpu_params(amg, cuda_stream=stream.cuda_stream, **kw)
    h = amg.amg_setup(amg.csr_arg(A.n, rp, ci, v), None, p)
    info = amg.amg_solve(h, bd, xd, TOL)
    torch.cuda.synchronize()
    return h, info, xd.cpu().numpy()


def _relres(A, x, b):
    S = A.to_scipy()
    return float(np.linalg.norm(b - S @ x) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def stretched64():
    A, b, _ = P.workload_stretched64()
    return A, b


@pytest.mark.parametrize("variants", [0, 1, 2, 4, 8], ids=["traditional", "1norm", "offlmp", "sprsfy", "cnstrnt"])
def test_stretched64_matches_oracle(amg, oracle_lib, stretched64, variants):
    A, b = stretched64
    kw = dict(theta=0.02, variants=variants)
    h, info, x = _device_solve(amg, A, b, **kw)
    oh, ost = oracle_lib.setup(A, **kw)
    assert ost == 0
    bad = compare_hierarchies(h, oh)
    amg.amg_free(h)
    assert not bad, bad[:8]
    xo, oinfo, ostat = oh.solve(b, TOL)
    assert info.status == 0 and ostat == 0
    assert iterations_agree(oracle_lib, A, kw, b, TOL, info.iters, oinfo.iters), (info.iters, oinfo.iters)
    if info.iters == oinfo.iters:
        assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= SOL_TOL
    assert _relres(A, x, b) <= 1.01 * TOL


def test_randcoef128_matches_oracle_fp64_and_mixed(amg, oracle_lib):
    A, b, _ = P.workload_randcoef128()
    kw = dict(theta=0.02, variants=3)
    h, info, x = _device_solve(amg, A, b, **kw)
    oh, ost = oracle_lib.setup(A, **kw)
    assert ost == 0
    bad = compare_hierarchies(h, oh)
    amg.amg_free(h)
    assert not bad, bad[:8]
    xo, oinfo, ostat = oh.solve(b, TOL)
    assert info.status == 0 and ostat == 0
    assert iterations_agree(oracle_lib, A, kw, b, TOL, info.iters, oinfo.iters), (info.iters, oinfo.iters)
    if info.iters == oinfo.iters:
        assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= SOL_TOL
    assert _relres(A, x, b) <= 1.01 * TOL
    # mixed precision: the same stopping test, iterations within one of the FP64 oracle's
    hm, infom, xm = _device_solve(amg, A, b, precision=amg.AMG_MIXED, **kw)
    amg.amg_free(hm)
    assert infom.status == 0 and abs(infom.iters - oinfo.iters) <= 1, (infom.iters, oinfo.iters)
    assert _relres(A, xm, b) <= 1.01 * TOL
    assert np.linalg.norm(xm - xo) / np.linalg.norm(xo) <= 1e-6


def test_convdiff64_gmres_matches_oracle_fp64_and_mixed(amg, oracle_lib):
    # the nonsymmetric line of the benchmark: symmetrised strength, general coarsest inverse,
    # flexible GMRES(30)
    A, b, kw = P.workload_convdiff64()
    h, info, x = _device_solve(amg, A, b, **kw)
    oh, ost = oracle_lib.setup(A, **kw)
    assert ost == 0
    bad = compare_hierarchies(h, oh)
    amg.amg_free(h)
    assert not bad, bad[:8]
    xo, oinfo, ostat = oh.solve(b, TOL)
    assert info.status == 0 and ostat == 0
    assert iterations_agree(oracle_lib, A, kw, b, TOL, info.iters, oinfo.iters), (info.iters, oinfo.iters)
    if info.iters == oinfo.iters:
        assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= SOL_TOL
    assert _relres(A, x, b) <= 1.01 * TOL
    hm, infom, xm = _device_solve(amg, A, b, precision=amg.AMG_MIXED, **kw)
    amg.amg_free(hm)
    assert infom.status == 0 and abs(infom.iters - oinfo.iters) <= 2, (infom.iters, oinfo.iters)
    assert _relres(A, xm, b) <= 1.01 * TOL


def test_elasticity40_matches_oracle_fp64_and_mixed(amg, oracle_lib):
    # the systems line of the benchmark: 3D elasticity, six rigid-body modes
    A, b, kw = P.workload_elasticity()
    B = A.meta["rbm"]
    import torch
    stream = torch.cuda.current_stream()
    rp, ci, v = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (A.row_ptr, A.col, A.val))
    Bd = torch.from_numpy(np.ascontiguousarray(B).reshape(-1)).cuda()
    bd = torch.from_numpy(b).cuda()
    oh, ost = oracle_lib.setup(A, nullspace=B, **kw)
    assert ost == 0
    xo, oinfo, ostat = oh.solve(b, TOL)
    for prec in (amg.AMG_FP64, amg.AMG_MIXED):
        h = amg.amg_setup(amg.csr_arg(A.n, rp, ci, v), Bd,
                          gpu_params(amg, cuda_stream=stream.cuda_stream, precision=prec, **kw))
        if prec == amg.AMG_FP64:
            bad = compare_hierarchies(h, oh)
            assert not bad, bad[:8]
        xd = torch.zeros_like(bd)
        info = amg.amg_solve(h, bd, xd, TOL)
        torch.cuda.synchronize()
        amg.amg_free(h)
        x = xd.cpu().numpy()
        assert info.status == 0 and ostat == 0
        assert abs(info.iters - oinfo.iters) <= (0 if prec == amg.AMG_FP64 else 1), (prec, info.iters, oinfo.iters)
        assert _relres(A, x, b) <= 1.01 * TOL
        assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= (SOL_TOL if prec == amg.AMG_FP64 else 1e-6)
