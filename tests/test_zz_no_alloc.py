"""The allocation-free sparse product (amg_spgemm_noalloc) against the allocating one
(amg_spgemm), through the C ABI.

amg_spgemm_noalloc exists for callers that must not allocate device memory (a process that
gives all GPU memory to its own pool, or a serving loop with a fixed budget); it keeps every
temporary in a fixed array inside the library.  Both entry points sum each entry over the
same ascending inner index with separately rounded products, so the results must agree bit
for bit -- the same bar as the other SpGEMM parity tests -- on two calls in a row (the shared
array keeps the previous call's contents; nothing may leak from one call into the next).
This file is collected last, and passes alone in a fresh process as well as after the rest.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2103_10476_gb300 import build
    build.build()
    from paper_2103_10476_gb300 import amg as m
    return m


def _random_csr(rng, m, k, density):
    import scipy.sparse as sp
    M = sp.random(m, k, density=density, random_state=rng, format="csr")
    M.sort_indices()
    return M.indptr.astype(np.int64), M.indices.astype(np.int32), M.data.astype(np.float64)


def _device(amg, n, rp, ci, v):
    import torch
    t = (torch.from_numpy(rp).cuda(), torch.from_numpy(ci).cuda(), torch.from_numpy(v).cuda())
    return amg.csr_arg(n, *t), t


@pytest.mark.parametrize("seed,m,k,ncol,dens", [(11, 300, 200, 1000, 0.05), (12, 8, 400, 20000, 0.6),
                                                (13, 2000, 2000, 2000, 0.004)])
def test_noalloc_spgemm_matches_allocating_entry_point(amg, seed, m, k, ncol, dens):
    import torch
    rng = np.random.default_rng(seed)
    A = _random_csr(rng, m, k, dens)
    B = _random_csr(rng, k, ncol, dens)
    # reference: the allocating entry point, from host arrays
    ref = amg.amg_spgemm(amg.csr_arg(m, *A), k, amg.csr_arg(k, *B), ncol)
    nnz = len(ref[1])
    Ad, keepA = _device(amg, m, *A)
    Bd, keepB = _device(amg, k, *B)
    for call in range(2):
        crp = torch.full((m + 1,), -7, dtype=torch.int64, device="cuda")
        cci = torch.full((nnz + 5,), -7, dtype=torch.int32, device="cuda")
        cv = torch.full((nnz + 5,), float("nan"), dtype=torch.float64, device="cuda")
        st, got = amg.amg_spgemm_noalloc(Ad, k, Bd, ncol, crp, cci, cv, nnz + 5)
        torch.cuda.synchronize()
        assert st == amg.AMG_OK, (call, st, amg.amg_last_error())
        assert got == nnz
        assert np.array_equal(crp.cpu().numpy(), ref[0]), call
        assert np.array_equal(cci.cpu().numpy()[:nnz], ref[1]), call
        assert np.array_equal(cv.cpu().numpy()[:nnz], ref[2]), call
    del keepA, keepB


def test_noalloc_spgemm_reports_small_output_and_size_limit(amg):
    import torch
    rng = np.random.default_rng(5)
    A = _random_csr(rng, 50, 60, 0.1)
    B = _random_csr(rng, 60, 70, 0.1)
    ref = amg.amg_spgemm(amg.csr_arg(50, *A), 60, amg.csr_arg(60, *B), 70)
    nnz = len(ref[1])
    Ad, keepA = _device(amg, 50, *A)
    Bd, keepB = _device(amg, 60, *B)
    crp = torch.zeros(51, dtype=torch.int64, device="cuda")
    cci = torch.zeros(max(nnz - 1, 1), dtype=torch.int32, device="cuda")
    cv = torch.zeros(max(nnz - 1, 1), dtype=torch.float64, device="cuda")
    st, got = amg.amg_spgemm_noalloc(Ad, 60, Bd, 70, crp, cci, cv, nnz - 1)
    assert st == amg.AMG_ERR_BUDGET and got == nnz
    # then with room: the same result as the allocating product
    cci = torch.zeros(nnz, dtype=torch.int32, device="cuda")
    cv = torch.zeros(nnz, dtype=torch.float64, device="cuda")
    st, got = amg.amg_spgemm_noalloc(Ad, 60, Bd, 70, crp, cci, cv, nnz)
    assert st == amg.AMG_OK and np.array_equal(cv.cpu().numpy(), ref[2])
    # more rows than the documented limit: refused before any device work
    big = amg.amg_csr_t(1_000_001, 0, Ad.row_ptr, Ad.col, Ad.val, 1)
    st, _ = amg.amg_spgemm_noalloc(big, 60, Bd, 70, crp, cci, cv, nnz)
    assert st == amg.AMG_ERR_UNSUPPORTED and "1,000,000" in amg.amg_last_error()
    # host arrays are refused (this entry point only takes device arrays)
    st, _ = amg.amg_spgemm_noalloc(amg.csr_arg(50, *A), 60, Bd, 70, crp, cci, cv, nnz)
    assert st == amg.AMG_ERR_INVALID_ARG
    del keepA, keepB
