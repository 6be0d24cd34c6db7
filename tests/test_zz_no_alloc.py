"""The allocation-free sparse product (amg_spgemm_noalloc) against the allocating one
(amg_spgemm), through the C ABI.

amg_spgemm_noalloc exists for callers that must not allocate device memory (a process that
gives all GPU memory to its own pool, or a serving loop with a fixed budget); it keeps every
temporary in a fixed array inside the library.  Both entry points sum each entry over the
same ascending inner index, each term added by one fused multiply-add, so the results must
agree bit for bit -- the same bar as the other SpGEMM parity tests -- on two calls in a row (the shared
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


def test_noalloc_spgemm_refuses_long_row_tables_beyond_the_scratch(amg):
    # one row of A reaches 8 rows of B with 600,000 entries each over 5,000,000 columns: its
    # hash table (the next power of two above twice 4.8M slots, 4 bytes each) is larger than
    # the 32 MiB array, so the call must refuse before any long-row kernel runs, leave C's
    # column and value arrays untouched, and the next call must be exact again
    import torch
    ncol = 5_000_000
    rng = np.random.default_rng(21)
    per = 600_000
    brp = np.arange(0, 9 * per, per, dtype=np.int64)
    bci = np.concatenate([np.sort(rng.choice(ncol, per, replace=False)) for _ in range(8)]).astype(np.int32)
    bv = rng.uniform(-1, 1, len(bci))
    arp = np.array([0, 8, 9], dtype=np.int64)
    aci = np.array(list(range(8)) + [3], dtype=np.int32)
    av = rng.uniform(-1, 1, 9)
    Ad, keepA = _device(amg, 2, arp, aci, av)
    Bd, keepB = _device(amg, 8, brp, bci, bv)
    crp = torch.full((3,), -7, dtype=torch.int64, device="cuda")
    cap = 16
    cci = torch.full((cap,), -7, dtype=torch.int32, device="cuda")
    cv = torch.full((cap,), 3.5, dtype=torch.float64, device="cuda")
    st, _ = amg.amg_spgemm_noalloc(Ad, 8, Bd, ncol, crp, cci, cv, cap)
    assert st == amg.AMG_ERR_UNSUPPORTED and "do not fit" in amg.amg_last_error()
    assert (cci.cpu().numpy() == -7).all() and (cv.cpu().numpy() == 3.5).all()
    del keepA, keepB
    # a normal product right after: bit for bit the allocating entry point's
    A = _random_csr(rng, 400, 300, 0.03)
    B = _random_csr(rng, 300, 500, 0.03)
    ref = amg.amg_spgemm(amg.csr_arg(400, *A), 300, amg.csr_arg(300, *B), 500)
    nnz = len(ref[1])
    Ad, keepA = _device(amg, 400, *A)
    Bd, keepB = _device(amg, 300, *B)
    crp = torch.zeros(401, dtype=torch.int64, device="cuda")
    cci = torch.zeros(nnz, dtype=torch.int32, device="cuda")
    cv = torch.zeros(nnz, dtype=torch.float64, device="cuda")
    st, got = amg.amg_spgemm_noalloc(Ad, 300, Bd, 500, crp, cci, cv, nnz)
    assert st == amg.AMG_OK and got == nnz
    assert np.array_equal(crp.cpu().numpy(), ref[0]) and np.array_equal(cci.cpu().numpy(), ref[1])
    assert np.array_equal(cv.cpu().numpy(), ref[2])
    del keepA, keepB


def test_noalloc_spgemm_rejects_bad_row_pointers_and_columns(amg):
    # checked before any kernel walks a row: a decreasing row pointer, a last row pointer that
    # is not nnz, and a column index outside B; C is left as it was in each case
    import torch
    rng = np.random.default_rng(9)
    A = _random_csr(rng, 40, 30, 0.2)
    B = _random_csr(rng, 30, 50, 0.2)
    Bd, keepB = _device(amg, 30, *B)
    crp = torch.full((41,), -7, dtype=torch.int64, device="cuda")
    cci = torch.full((2000,), -7, dtype=torch.int32, device="cuda")
    cv = torch.full((2000,), 3.5, dtype=torch.float64, device="cuda")
    bad_rp = A[0].copy()
    bad_rp[5], bad_rp[6] = bad_rp[6], bad_rp[5] - 1        # decreasing at row 5
    bad_end = A[0].copy()
    bad_end[-1] -= 1                                       # ends before nnz
    bad_col = A[1].copy()
    bad_col[len(bad_col) // 2] = 30                        # column 30 of a 30-row B
    for rp, ci in ((bad_rp, A[1]), (bad_end, A[1]), (A[0], bad_col)):
        Ad, keepA = _device(amg, 40, rp, ci, A[2])
        Ad.nnz = len(ci)                                   # the entries the arrays hold
        st, _ = amg.amg_spgemm_noalloc(Ad, 30, Bd, 50, crp, cci, cv, 2000)
        assert st == amg.AMG_ERR_INVALID_ARG, amg.amg_last_error()
        assert (cci.cpu().numpy() == -7).all() and (cv.cpu().numpy() == 3.5).all()
        del keepA
    # NULL column array with entries: refused on the host
    Ad, keepA = _device(amg, 40, *A)
    nullc = amg.amg_csr_t(40, int(A[0][-1]), Ad.row_ptr, None, Ad.val, 1)
    st, _ = amg.amg_spgemm_noalloc(nullc, 30, Bd, 50, crp, cci, cv, 2000)
    assert st == amg.AMG_ERR_INVALID_ARG
    del keepA, keepB
