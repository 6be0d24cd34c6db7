"""Parity of the CUDA path with the oracle for nonsymmetric operators: setup with the
symmetrised strength mask, the general coarsest inverse, and flexible GMRES(m) with one V-cycle
per step (the outer iteration of §3's wind pressure system).

Bars: integer structures bit-exact and values within VAL_TOL (the hierarchy); GMRES
iterations by the rule of the PCG parity tests (identical, or within 2 at a borderline stop);
solutions within SOL_TOL when the counts agree; the true relative residual recomputed here on
the host with scipy.
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


def _arg(amg, A):
    return amg.csr_arg(A.n, np.ascontiguousarray(A.row_ptr, np.int64), np.ascontiguousarray(A.col, np.int32),
                       np.ascontiguousarray(A.val, np.float64))


def _setup(amg, A, **kw):
    return amg.amg_setup_status(_arg(amg, A), None, gpu_params(amg, **kw))


def _relres(A, x, b):
    return float(np.linalg.norm(b - A.to_scipy() @ x) / np.linalg.norm(b))


CASES = [(10, 0.05, 0), (14, 0.02, 0), (14, 0.05, 3), (14, 0.02, 15), (20, 0.05, 3), (20, 0.02, 15)]


@pytest.mark.parametrize("N,theta,variants", CASES, ids=[f"cd{c[0]}-t{c[1]}-v{c[2]}" for c in CASES])
def test_gmres_hierarchy_and_solve_match_oracle(amg, oracle_lib, N, theta, variants):
    A = P.convection_diffusion_box(N)
    b = P.rhs_uniform(A.n, 5)
    kw = dict(theta=theta, variants=variants, krylov=1, max_coarse=40)
    h, st = _setup(amg, A, **kw)
    oh, ost = oracle_lib.setup(A, **kw)
    assert st == ost == 0, (st, ost, amg.amg_last_error())
    bad = compare_hierarchies(h, oh)
    assert not bad, bad[:8]
    x = np.zeros(A.n)
    info = amg.amg_solve(h, b, x, TOL)
    amg.amg_free(h)
    xo, oinfo, ostat = oh.solve(b, TOL)
    assert info.status == 0 and ostat == 0
    assert iterations_agree(oracle_lib, A, kw, b, TOL, info.iters, oinfo.iters), (info.iters, oinfo.iters)
    if info.iters == oinfo.iters:
        assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= SOL_TOL
    assert _relres(A, x, b) <= 1.01 * TOL
    assert abs(info.relres_true - _relres(A, x, b)) <= 1e-3 * TOL


@pytest.mark.parametrize("restart", [1, 2, 5, 7])
def test_gmres_restarted_matches_oracle(amg, oracle_lib, restart):
    # short cycles: restarts (true residual, new v_0) happen many times within one solve
    A = P.convection_diffusion_box(14)
    b = P.rhs_uniform(A.n, 8)
    kw = dict(theta=0.05, variants=3, krylov=1, restart=restart, max_coarse=40, max_iter=400)
    h, st = _setup(amg, A, **kw)
    assert st == 0
    x = np.zeros(A.n)
    info = amg.amg_solve(h, b, x, TOL)
    amg.amg_free(h)
    oh, _ = oracle_lib.setup(A, **kw)
    xo, oinfo, ostat = oh.solve(b, TOL)
    assert info.status == ostat == 0
    assert iterations_agree(oracle_lib, A, kw, b, TOL, info.iters, oinfo.iters), (info.iters, oinfo.iters)
    if info.iters == oinfo.iters:
        assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= SOL_TOL
    assert _relres(A, x, b) <= 1.01 * TOL


def test_gmres_iteration_limit_matches_oracle(amg, oracle_lib):
    # the limit falls inside a cycle: the partial cycle's update is applied, status says so
    A = P.convection_diffusion_box(14)
    b = P.rhs_uniform(A.n, 2)
    kw = dict(theta=0.05, variants=3, krylov=1, restart=6, max_coarse=40, max_iter=9)
    h, _ = _setup(amg, A, **kw)
    x = np.zeros(A.n)
    info = amg.amg_solve(h, b, x, 1e-14)
    amg.amg_free(h)
    oh, _ = oracle_lib.setup(A, **kw)
    xo, oinfo, ostat = oh.solve(b, 1e-14)
    assert info.status == ostat == amg.AMG_ERR_NOT_CONVERGED
    assert info.iters == oinfo.iters == 9
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= 1e-9
    assert info.relres_true == pytest.approx(oinfo.relres_true, rel=1e-6)


def test_gmres_mixed_precision(amg, oracle_lib):
    # FP32 V-cycle inside flexible GMRES: the basis stays FP64, so the count is the FP64
    # oracle's within 2 and the same stopping test holds
    A = P.convection_diffusion_box(20)
    b = P.rhs_uniform(A.n, 4)
    kw = dict(theta=0.05, variants=3, krylov=1, max_coarse=40)
    h, st = _setup(amg, A, precision=amg.AMG_MIXED, **kw)
    assert st == 0
    x = np.zeros(A.n)
    info = amg.amg_solve(h, b, x, TOL)
    amg.amg_free(h)
    oh, _ = oracle_lib.setup(A, **kw)
    xo, oinfo, _ = oh.solve(b, TOL)
    assert info.status == 0 and abs(info.iters - oinfo.iters) <= 2, (info.iters, oinfo.iters)
    assert _relres(A, x, b) <= 1.01 * TOL
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= 1e-6


def test_gmres_on_symmetric_operator_matches_pcg(amg):
    # on a symmetric operator the symmetrised mask is the mask (same hierarchy) and both
    # Krylov methods reach the same solution
    A = P.stretched_box(16, 1.1)
    b = P.rhs_uniform(A.n, 3)
    kw = dict(theta=0.02, variants=3, max_coarse=40)
    hc, _ = _setup(amg, A, **kw)
    hg, st = _setup(amg, A, krylov=amg.AMG_KRYLOV_GMRES, **kw)
    assert st == 0
    for l in range(amg.amg_num_levels(hc) - 1):
        for what in ("strong", "agg", "P.v"):
            assert np.array_equal(amg.amg_export(hc, l, what), amg.amg_export(hg, l, what)), (l, what)
    xc, xg = np.zeros(A.n), np.zeros(A.n)
    ic = amg.amg_solve(hc, b, xc, 1e-10)
    ig = amg.amg_solve(hg, b, xg, 1e-10)
    amg.amg_free(hc)
    amg.amg_free(hg)
    assert ic.status == 0 and ig.status == 0
    assert np.linalg.norm(xg - xc) / np.linalg.norm(xc) <= 1e-8


def test_gmres_device_buffers_and_repeat(amg):
    # device-resident b and x on torch's current stream; a second solve on the same handle
    # reuses the basis and gives the same bits
    import torch
    A = P.convection_diffusion_box(14)
    b = P.rhs_uniform(A.n, 6)
    stream = torch.cuda.current_stream()
    rp, ci, v = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (A.row_ptr, A.col, A.val))
    p = gpu_params(amg, theta=0.05, variants=3, krylov=1, max_coarse=40, cuda_stream=stream.cuda_stream)
    h = amg.amg_setup(amg.csr_arg(A.n, rp, ci, v), None, p)
    bd = torch.from_numpy(b).cuda()
    x1, x2 = torch.zeros_like(bd), torch.zeros_like(bd)
    i1 = amg.amg_solve(h, bd, x1, TOL)
    i2 = amg.amg_solve(h, bd, x2, TOL)
    torch.cuda.synchronize()
    xh = np.zeros(A.n)
    i3 = amg.amg_solve(h, b, xh, TOL)
    amg.amg_free(h)
    assert i1.status == i2.status == i3.status == 0 and i1.iters == i2.iters == i3.iters
    assert torch.equal(x1, x2)
    assert np.array_equal(x1.cpu().numpy(), xh)


def test_gmres_graph_steps_equal_eager_steps(amg):
    # each Arnoldi step is a CUDA graph launched one step ahead; with profiling on, the same
    # steps run eagerly one after another: identical bits, iterations and launch counts
    A = P.convection_diffusion_box(14)
    b = P.rhs_uniform(A.n, 7)
    h, st = _setup(amg, A, theta=0.05, variants=3, krylov=1, restart=8, max_coarse=40)
    assert st == 0
    xg, xe = np.zeros(A.n), np.zeros(A.n)
    amg.amg_solve(h, b, xg, TOL)                 # captures the step graphs
    c0 = amg.amg_launch_count()
    ig = amg.amg_solve(h, b, xg, TOL)
    c1 = amg.amg_launch_count()
    amg.amg_profile_enable(1)
    try:
        ie = amg.amg_solve(h, b, xe, TOL)
        c2 = amg.amg_launch_count()
    finally:
        amg.amg_profile_enable(0)
    amg.amg_free(h)
    assert ig.status == ie.status == 0 and ig.iters == ie.iters
    assert np.array_equal(xg, xe)
    assert c1 - c0 == c2 - c1 > 0


def test_gmres_zero_rhs_and_unsupported_modes(amg):
    A = P.convection_diffusion_box(10)
    h, st = _setup(amg, A, theta=0.05, krylov=1, max_coarse=40)
    assert st == 0
    x = np.ones(A.n)
    info = amg.amg_solve(h, np.zeros(A.n), x, TOL)
    assert info.status == 0 and info.iters == 0 and not x.any()
    # several right-hand sides at once and the batch engine run PCG only
    B = np.stack([P.rhs_uniform(A.n, 1), P.rhs_uniform(A.n, 2)])
    st = amg.lib.amg_solve_multi(h, 2, B.ctypes.data, np.zeros_like(B).ctypes.data, TOL, None)
    assert st == amg.AMG_ERR_UNSUPPORTED and "PCG" in amg.amg_last_error()
    bt = amg.C.c_void_p()
    arr = (amg.C.c_void_p * 1)(h.value)
    st = amg.lib.amg_batch_create(1, arr, None, 0, amg.C.byref(bt))
    assert st == amg.AMG_ERR_UNSUPPORTED and "PCG" in amg.amg_last_error()
    amg.amg_free(h)


def test_gmres_restart_out_of_range_rejected(amg):
    A = P.convection_diffusion_box(6)
    for r in (0, 513):
        h, st = _setup(amg, A, theta=0.05, krylov=1, restart=r)
        assert h is None and st == amg.AMG_ERR_INVALID_ARG
