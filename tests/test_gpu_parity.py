"""Parity of the CUDA path (through the C ABI) with the CPU oracle on seeded inputs."""
import numpy as np
import pytest

from paper_2103_10476_gb300 import problems as P
from tests.gpu_common import SOL_TOL, compare_hierarchies, gpu_setup, iterations_agree, rel_err
from tests.helpers import csr_from_dense

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


def _solve_both(amg, oracle_lib, A, b, tol=1e-8, **kw):
    h, st = gpu_setup(A, **kw)
    oh, ost = oracle_lib.setup(A, **kw)
    assert st == ost, (st, ost, amg.amg_last_error())
    if st != 0:
        return None
    bad = compare_hierarchies(h, oh)
    x = np.zeros(A.n)
    info = amg.amg_solve(h, b, x, tol)
    xo, oinfo, ostat = oh.solve(b, tol)
    amg.amg_free(h)
    return bad, info, x, oinfo, xo, ostat


# ---------------------------------------------------------------- whole method, small and ragged sizes

CASES = [
    ("laplace20", lambda: P.laplace_cube(20), dict(theta=0.0)),
    ("laplace13", lambda: P.laplace_cube(13), dict(theta=0.0, max_coarse=20)),
    ("stretched17", lambda: P.stretched_box(17, 1.1), dict(theta=0.02, max_coarse=40)),
    ("random11", lambda: P.random_coefficient_cube(11, 2), dict(theta=0.02, max_coarse=30)),
]
VARIANTS = [0, 1, 2, 4, 8, 3, 15, 12]


@pytest.mark.parametrize("variants", VARIANTS)
@pytest.mark.parametrize("name,make,kw", CASES, ids=[c[0] for c in CASES])
def test_hierarchy_and_solve_match_oracle(amg, oracle_lib, name, make, kw, variants):
    A = make()
    b = P.rhs_uniform(A.n, 7)
    out = _solve_both(amg, oracle_lib, A, b, variants=variants, **kw)
    if out is None:
        return   # same failure status on both sides (e.g. the traditional method's zero diagonal)
    bad, info, x, oinfo, xo, ostat = out
    assert not bad, bad[:8]
    assert info.status == ostat
    assert iterations_agree(oracle_lib, A, dict(variants=variants, **kw), b, 1e-8, info.iters, oinfo.iters), \
        (info.iters, oinfo.iters)
    if info.iters == oinfo.iters:
        assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= SOL_TOL
    assert info.relres_true <= 1e-8


@pytest.mark.parametrize("pt_unit", [0, 1])
def test_bit_exact_values_when_lambda_is_fixed(amg, oracle_lib, pt_unit):
    # with lambda fixed (1Norm's bound) the whole setup is evaluated in the same order on both
    # sides, so every hierarchy value agrees to the last bit
    A = P.stretched_box(15, 1.15)
    h, st = gpu_setup(A, theta=0.02, variants=3, pt_unit=pt_unit, max_coarse=30)
    oh, ost = oracle_lib.setup(A, theta=0.02, variants=3, pt_unit=pt_unit, max_coarse=30)
    assert st == 0 and ost == 0
    for l in range(amg.amg_num_levels(h) - 1):
        for w in ("Abar.v", "Dsm", "P.v", "R.v"):
            assert np.array_equal(amg.amg_export(h, l, w), oh.get(l, w)), (l, w)
        assert np.array_equal(amg.amg_export(h, l + 1, "A.v"), oh.get(l + 1, "A.v")), l
    amg.amg_free(h)


def test_unit_and_orthonormal_give_same_iterations(amg):
    A = P.random_coefficient_cube(12, 5)
    b = P.rhs_uniform(A.n, 3)
    its = []
    for pt in (0, 1):
        h, st = gpu_setup(A, theta=0.02, variants=1, pt_unit=pt, max_coarse=30)
        x = np.zeros(A.n)
        its.append(amg.amg_solve(h, b, x, 1e-8).iters)
        amg.amg_free(h)
    assert abs(its[0] - its[1]) <= 1


def test_device_pointers_and_host_pointers_agree(amg):
    import torch
    A = P.stretched_box(12, 1.2)
    b = P.rhs_uniform(A.n, 5)
    h, st = gpu_setup(A, theta=0.02, variants=2, max_coarse=30)
    x_host = np.zeros(A.n)
    i1 = amg.amg_solve(h, b, x_host, 1e-8)
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    i2 = amg.amg_solve(h, bd, xd, 1e-8)
    torch.cuda.synchronize()
    assert i1.iters == i2.iters
    assert np.array_equal(xd.cpu().numpy(), x_host)   # deterministic: bitwise identical
    amg.amg_free(h)
    # the matrix itself from device memory
    rp = torch.from_numpy(A.row_ptr).cuda()
    ci = torch.from_numpy(A.col).cuda()
    v = torch.from_numpy(A.val).cuda()
    arg = amg.csr_arg(A.n, rp, ci, v)
    assert arg.on_device == 1
    h2 = amg.amg_setup(arg, None, amg.amg_params_default(theta=0.02, variants=2, max_coarse=30))
    x2 = np.zeros(A.n)
    amg.amg_solve(h2, b, x2, 1e-8)
    assert np.array_equal(x2, x_host)
    amg.amg_free(h2)


def test_runs_are_bitwise_reproducible(amg):
    A = P.random_coefficient_cube(14, 8)
    b = P.rhs_uniform(A.n, 1)
    xs = []
    for _ in range(2):
        h, st = gpu_setup(A, theta=0.02, variants=2, max_coarse=40)
        assert st == 0
        x = np.zeros(A.n)
        amg.amg_solve(h, b, x, 1e-8)
        xs.append(x)
        amg.amg_free(h)
    assert np.array_equal(xs[0], xs[1])


# ---------------------------------------------------------------- SpGEMM on its own

@pytest.mark.parametrize("seed,m,k,ncol,dens", [(0, 1, 1, 1, 1.0), (1, 37, 53, 29, 0.1), (2, 300, 200, 1000, 0.05),
                                                (3, 64, 64, 7000, 0.9), (4, 500, 40, 5, 0.3)])
def test_spgemm_matches_oracle_bitwise(amg, oracle_lib, seed, m, k, ncol, dens):
    import scipy.sparse as sp
    rng = np.random.default_rng(seed)
    Am = sp.random(m, k, density=dens, random_state=rng, format="csr")
    Bm = sp.random(k, ncol, density=dens, random_state=rng, format="csr")
    Am.sort_indices(); Bm.sort_indices()
    from paper_2103_10476_gb300.problems import CSR
    Ac = CSR(m, Am.indptr.astype(np.int64), Am.indices.astype(np.int32), Am.data.astype(np.float64))
    Bc = CSR(k, Bm.indptr.astype(np.int64), Bm.indices.astype(np.int32), Bm.data.astype(np.float64))
    rp, ci, v = amg.amg_spgemm(amg.csr_arg(m, Ac.row_ptr, Ac.col, Ac.val), k,
                               amg.csr_arg(k, Bc.row_ptr, Bc.col, Bc.val), ncol)
    Co = oracle_lib.spgemm(Ac, Bc, ncol)
    assert np.array_equal(rp, Co.row_ptr) and np.array_equal(ci, Co.col)
    assert np.array_equal(v, Co.val)


def test_spgemm_long_rows_use_global_tables(amg, oracle_lib):
    # a dense-ish row block whose products exceed the shared-memory tables
    import scipy.sparse as sp
    rng = np.random.default_rng(9)
    Am = sp.random(8, 400, density=0.9, random_state=rng, format="csr")
    Bm = sp.random(400, 20000, density=0.05, random_state=rng, format="csr")
    from paper_2103_10476_gb300.problems import CSR
    Ac = CSR(8, Am.indptr.astype(np.int64), Am.indices.astype(np.int32), Am.data)
    Bc = CSR(400, Bm.indptr.astype(np.int64), Bm.indices.astype(np.int32), Bm.data)
    rp, ci, v = amg.amg_spgemm(amg.csr_arg(8, Ac.row_ptr, Ac.col, Ac.val), 400,
                               amg.csr_arg(400, Bc.row_ptr, Bc.col, Bc.val), 20000)
    Co = oracle_lib.spgemm(Ac, Bc, 20000)
    assert np.array_equal(ci, Co.col) and np.array_equal(v, Co.val)


@pytest.mark.parametrize("ncol", [20000, 60000], ids=["dense-counters", "hash-tables"])
def test_spgemm_rows_of_thousands_of_entries(amg, oracle_lib, ncol):
    # rows of C with thousands of entries: counted in shared memory per block when B has at most
    # 49,152 columns, in global hash tables beyond; and a short row beside them
    import scipy.sparse as sp
    rng = np.random.default_rng(17)
    Am = sp.random(9, 400, density=0.9, random_state=rng, format="lil")
    Am[8, :] = 0
    Am[8, 3] = 1.5
    Am = Am.tocsr()
    Am.sort_indices()
    Bm = sp.random(400, ncol, density=0.05, random_state=rng, format="csr")
    Bm.sort_indices()
    from paper_2103_10476_gb300.problems import CSR
    Ac = CSR(9, Am.indptr.astype(np.int64), Am.indices.astype(np.int32), Am.data.astype(np.float64))
    Bc = CSR(400, Bm.indptr.astype(np.int64), Bm.indices.astype(np.int32), Bm.data.astype(np.float64))
    rp, ci, v = amg.amg_spgemm(amg.csr_arg(9, Ac.row_ptr, Ac.col, Ac.val), 400,
                               amg.csr_arg(400, Bc.row_ptr, Bc.col, Bc.val), ncol)
    Co = oracle_lib.spgemm(Ac, Bc, ncol)
    assert np.diff(Co.row_ptr).max() > 2048
    assert np.array_equal(rp, Co.row_ptr) and np.array_equal(ci, Co.col)
    assert np.array_equal(v, Co.val)


def _structured_product(rng, m, ncol):
    """A (m rows) and B (3000 rows, ncol columns) whose rows reach every branch of the product on
    at least 32,768 rows: bounds above 1,024 slots that hold more than 512 columns (the second
    symbolic round) and that hold 40 (kept from the first), rows of more than 2,048 products (dense
    counters when B is narrow enough), rows of A of more than 256 entries with one term a k (the
    segment kernels' buckets) and with eight (their per-k sweep), and short rows around them."""
    import scipy.sparse as sp
    from paper_2103_10476_gb300.problems import CSR
    brows = []
    for k in range(3000):
        if k < 2000:
            cols = rng.choice(ncol, 8, replace=False)
        elif k < 2500:
            cols = rng.choice(40, 10, replace=False)
        else:
            cols = rng.choice(ncol, 1, replace=False)
        brows.append(np.sort(cols))
    arows = []
    for i in range(m):
        if i < 50:
            ks = rng.choice(2000, 150, replace=False)
        elif i < 100:
            ks = 2000 + rng.choice(500, 100, replace=False)
        elif i < 110:
            ks = 2500 + rng.choice(500, 400, replace=False)
        elif i < 115:
            ks = rng.choice(2000, 300, replace=False)
        else:
            ks = rng.choice(3000, 3, replace=False)
        arows.append(np.sort(ks))

    def csr(rows, n):
        rp = np.zeros(len(rows) + 1, dtype=np.int64)
        rp[1:] = np.cumsum([len(r) for r in rows])
        ci = np.concatenate(rows).astype(np.int32)
        v = rng.standard_normal(len(ci))
        return CSR(len(rows), rp, ci, v)
    return csr(arows, m), csr(brows, 3000)


@pytest.mark.parametrize("ncol", [40000, 6000], ids=["wide-B", "narrow-B"])
def test_spgemm_capped_tables_and_segments(amg, oracle_lib, ncol):
    # B of 40,000 columns: the capped first round and its retry, dense counters, the segment
    # kernels' binary-search accumulator; B of 6,000: the bitmap order of long rows of C and
    # the segment kernels' dense accumulator -- every result bit-exact against the oracle
    rng = np.random.default_rng(23 + ncol)
    m = 40000
    Ac, Bc = _structured_product(rng, m, ncol)
    rp, ci, v = amg.amg_spgemm(amg.csr_arg(m, Ac.row_ptr, Ac.col, Ac.val), 3000,
                               amg.csr_arg(3000, Bc.row_ptr, Bc.col, Bc.val), ncol)
    Co = oracle_lib.spgemm(Ac, Bc, ncol)
    lens = np.diff(Co.row_ptr)
    assert lens[:50].min() > 512 and lens[50:100].max() <= 40 and lens[110:115].min() > 1024
    assert np.array_equal(rp, Co.row_ptr) and np.array_equal(ci, Co.col)
    assert np.array_equal(v, Co.val)


def test_spgemm_capped_tables_at_their_boundary(amg, oracle_lib):
    # 33,000 rows (capped first tables on): rows whose product bounds ask for 2,048 slots and
    # that hold exactly 512 columns (kept from the first round) or 513 (the second round), empty
    # rows of A between them, and empty rows of B inside the heavy rows' sums
    from paper_2103_10476_gb300.problems import CSR
    rng = np.random.default_rng(41)
    m, k, ncol = 33000, 1100, 30000
    brows = [np.array([], dtype=np.int64) if j % 11 == 0 else np.sort(rng.choice(ncol, 2, replace=False))
             for j in range(k)]
    brows[1] = np.arange(512)            # row 0 of A: 512 columns from B's row 1 ...
    brows[2] = np.arange(513)            # ... row 2 of A: 513 from B's row 2
    arows = []
    for i in range(m):
        if i == 0:
            ks = np.array([1] + list(range(1000, 1100)))          # bound 512 + 100 x 4 = 912
        elif i == 2:
            ks = np.array([2] + list(range(1000, 1100)))
        elif i % 7 == 3:
            ks = np.array([], dtype=np.int64)
        else:
            ks = np.sort(rng.choice(k, 3, replace=False))
        arows.append(ks)
    # rows 0 and 2 take their extra columns only inside 0..511 / 0..512: B's rows 1000-1099
    # point there, so the distinct counts stay 512 and 513
    for j in range(1000, 1100):
        brows[j] = np.sort(rng.choice(512, 4, replace=False))

    def csr(rows, n):
        rp = np.zeros(n + 1, dtype=np.int64)
        rp[1:] = np.cumsum([len(r) for r in rows])
        ci = (np.concatenate(rows) if rp[-1] else np.zeros(0)).astype(np.int32)
        return CSR(n, rp, ci, rng.standard_normal(len(ci)))
    Ac, Bc = csr(arows, m), csr(brows, k)
    rp, ci, v = amg.amg_spgemm(amg.csr_arg(m, Ac.row_ptr, Ac.col, Ac.val), k,
                               amg.csr_arg(k, Bc.row_ptr, Bc.col, Bc.val), ncol)
    Co = oracle_lib.spgemm(Ac, Bc, ncol)
    lens = np.diff(Co.row_ptr)
    assert lens[0] == 512 and lens[2] == 513 and lens[3] == 0
    assert np.array_equal(rp, Co.row_ptr) and np.array_equal(ci, Co.col)
    assert np.array_equal(v, Co.val)


# ---------------------------------------------------------------- degenerate cases

def test_single_level_one_iteration(amg):
    A = P.laplace_cube(6)
    b = P.rhs_uniform(A.n, 0)
    h, st = gpu_setup(A)
    assert st == 0 and amg.amg_num_levels(h) == 1
    x = np.zeros(A.n)
    info = amg.amg_solve(h, b, x, 1e-8)
    assert info.status == 0 and info.iters == 1 and info.relres_true < 1e-12
    amg.amg_free(h)


@pytest.mark.parametrize("decades,N", [(2.0, 8), (12.0, 7)])
def test_coarse_inverse_single_level(amg, decades, N):
    # the whole matrix is the coarsest level: one PCG step with its dense inverse solves the
    # system.  Moderate contrast takes the FP32 factorisation refined by Newton-Schulz in FP64;
    # 10^12 contrast leaves FP32 without a usable factor and takes the direct FP64 path.
    A = P.random_coefficient_cube(N, 5, decades)
    b = P.rhs_uniform(A.n, 1)
    h, st = gpu_setup(A, max_coarse=1000)
    assert st == 0 and amg.amg_num_levels(h) == 1
    x = np.zeros(A.n)
    info = amg.amg_solve(h, b, x, 1e-10)
    amg.amg_free(h)
    assert info.status == 0 and info.relres_true <= 1e-10, (info.status, info.relres_true)
    if decades <= 2.0:
        # well conditioned: the inverse is exact to rounding, one step
        xr = np.linalg.solve(A.to_dense(), b)
        assert info.iters == 1 and np.linalg.norm(x - xr) / np.linalg.norm(xr) <= 1e-13
    else:
        # condition number ~1e14: the explicit inverse leaves a residual of order cond * eps,
        # which the outer PCG removes in a few steps
        assert info.iters <= 6, info.iters


def test_zero_rhs_and_empty_matrix(amg):
    A = P.laplace_cube(10)
    h, st = gpu_setup(A, max_coarse=20)
    x = np.ones(A.n)
    info = amg.amg_solve(h, np.zeros(A.n), x, 1e-8)
    assert info.status == 0 and info.iters == 0 and not x.any()
    amg.amg_free(h)
    E = csr_from_dense(np.zeros((0, 0)))
    h, st = gpu_setup(E)
    assert st == 0
    info = amg.amg_solve(h, np.zeros(1), np.zeros(1), 1e-8)
    assert info.iters == 0
    amg.amg_free(h)


def test_error_statuses_match_oracle(amg, oracle_lib):
    # traditional SA with large coefficient jumps: a row whose off-diagonals are all weak is
    # lumped to its row sum, zero for an interior row (zero filtered diagonal, §1.2)
    A = P.random_coefficient_cube(14, 8)
    h, st = gpu_setup(A, theta=0.02, variants=0, max_coarse=40)
    _, ost = oracle_lib.setup(A, theta=0.02, variants=0, max_coarse=40)
    assert st == ost == 4
    # with no strong connection at all the level is not coarsened: a single (dense) level
    A = P.stretched_box(10, 1.1)
    h, st = gpu_setup(A, theta=0.2, variants=0)
    oh, ost = oracle_lib.setup(A, theta=0.2, variants=0)
    assert st == ost == 0 and amg.amg_num_levels(h) == oh.nlevels == 1
    amg.amg_free(h)
    # indefinite coarse operator
    d = -np.eye(5) * 2.0
    h, st = gpu_setup(csr_from_dense(d))
    assert st == 6
    # unsorted columns
    A = P.laplace_cube(4)
    A.col = A.col.copy()
    A.col[[0, 1]] = A.col[[1, 0]]
    h, st = gpu_setup(A)
    assert st == 1


def test_not_converged_returns_last_iterate(amg):
    A = P.random_coefficient_cube(12, 1)
    b = P.rhs_uniform(A.n, 2)
    h, st = gpu_setup(A, theta=0.02, max_coarse=30, max_iter=3)
    x = np.zeros(A.n)
    info = amg.amg_solve(h, b, x, 1e-12)
    assert info.status == 7 and info.iters == 3 and 0 < info.relres_true < 1
    amg.amg_free(h)


@pytest.mark.parametrize("variants", [0, 1, 2, 4, 8])
def test_mixed_precision_iterations_track_fp64(amg, oracle_lib, variants):
    # FP32 hierarchy and V-cycle inside FP64 flexible PCG: same 1e-8 true residual, iteration
    # count within one of the FP64 oracle's, solution within the accuracy the stop guarantees
    A = P.stretched_box(28, 1.1)
    b = P.rhs_uniform(A.n, 1)
    h, st = gpu_setup(A, theta=0.02, variants=variants, max_coarse=60, precision=1)
    oh, ost = oracle_lib.setup(A, theta=0.02, variants=variants, max_coarse=60)
    assert st == 0 and ost == 0
    x = np.zeros(A.n)
    info = amg.amg_solve(h, b, x, 1e-8)
    xo, oinfo, _ = oh.solve(b, 1e-8)
    amg.amg_free(h)
    assert info.status == 0 and info.relres_true <= 1e-8
    assert abs(info.iters - oinfo.iters) <= 1, (info.iters, oinfo.iters)
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) < 1e-6


def test_mixed_precision_meets_tolerance(amg, oracle_lib):
    A = P.random_coefficient_cube(16, 2)
    b = P.rhs_uniform(A.n, 2)
    h, st = gpu_setup(A, theta=0.02, variants=3, max_coarse=40, precision=1)
    x = np.zeros(A.n)
    info = amg.amg_solve(h, b, x, 1e-8)
    oh, _ = oracle_lib.setup(A, theta=0.02, variants=3, max_coarse=40)
    xo, oinfo, _ = oh.solve(b, 1e-8)
    assert info.status == 0 and info.relres_true <= 1e-8
    assert abs(info.iters - oinfo.iters) <= 1
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) < 1e-6
    amg.amg_free(h)
