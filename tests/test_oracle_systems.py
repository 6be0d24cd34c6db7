"""Pins of the elasticity generator and of the oracle's path for systems of PDEs (several
unknowns per node, a multi-vector near-null space): block strength between nodes, MIS-2
on the node graph, the QR tentative prolongator, and the whole hierarchy.

Each test checks against something other than the code under test: closed-form energies and the
kernel of the Neumann operator, dense brute force on small blocks, exact algebraic identities
of the QR (orthonormal columns, Pt Bc = B), the Galerkin operator annihilating the coarse
near-null space, equality with the scalar path on a decoupled system, and PCG iteration bounds.
"""
import numpy as np
import pytest

from paper_2103_10476_gb300 import problems as P


def _box(nx, ny, nz, clamp=True):
    return P.elasticity_box(np.ones(nx), np.ones(ny), np.ones(nz), clamp=clamp)


# ------------------------------------------------------------------ generator

def test_elasticity_generator_kernel_symmetry_and_energy():
    A = _box(3, 2, 2, clamp=False)
    S = A.to_scipy()
    B = A.meta["rbm"]
    assert abs(S - S.T).max() == 0.0
    assert np.abs(S @ B.T).max() <= 1e-13 * abs(S).max()
    # u = F x with symmetric F: u^T K u = vol (lam tr(F)^2 + 2 mu F:F), exact for trilinear
    # elements and the 2x2x2 rule
    F = np.array([[0.3, 0.1, -0.2], [0.1, -0.5, 0.25], [-0.2, 0.25, 0.7]])
    u = (A.meta["coords"] @ F.T).ravel()
    nu = 0.3
    lam, mu = nu / ((1 + nu) * (1 - 2 * nu)), 1 / (2 * (1 + nu))
    assert u @ (S @ u) == pytest.approx(12.0 * (lam * np.trace(F) ** 2 + 2 * mu * np.sum(F * F)), rel=1e-13)
    # clamped: positive definite
    C = _box(2, 2, 2).to_dense()
    assert np.linalg.eigvalsh(C).min() > 0


# ------------------------------------------------------------------ block strength

def test_block_strength_bs1_is_eq7(oracle_lib):
    A = P.random_coefficient_cube(6, 3, 2.0)
    for theta in (0.0, 0.02, 0.1, 0.3):
        nrp, nci, nF, ns, strong = oracle_lib.node_strength(A, 1, theta)
        assert np.array_equal(nrp, A.row_ptr) and np.array_equal(nci, A.col)
        assert np.array_equal(nF, np.abs(A.val))
        assert np.array_equal(strong, oracle_lib.strength(A, theta))


def test_block_strength_brute_force(oracle_lib):
    A = _box(2, 2, 1, clamp=False)
    D = A.to_dense()
    bs = 3
    nn = A.n // bs
    for theta in (0.0, 0.05, 0.2):
        nrp, nci, nF, ns, strong = oracle_lib.node_strength(A, bs, theta)
        Fd = np.array([np.sqrt(np.sum(D[3 * I:3 * I + 3, 3 * I:3 * I + 3] ** 2)) for I in range(nn)])
        for I in range(nn):
            want = [J for J in range(nn) if np.any(D[3 * I:3 * I + 3, 3 * J:3 * J + 3] != 0)
                    or any(c // 3 == J for r in range(3 * I, 3 * I + 3)
                           for c in A.col[A.row_ptr[r]:A.row_ptr[r + 1]])]
            assert list(nci[nrp[I]:nrp[I + 1]]) == sorted(set(want))
            for t in range(nrp[I], nrp[I + 1]):
                J = nci[t]
                F = np.sqrt(np.sum(D[3 * I:3 * I + 3, 3 * J:3 * J + 3] ** 2))
                assert nF[t] == pytest.approx(F, rel=1e-15, abs=1e-300)
                thr = theta * np.sqrt(Fd[I] * Fd[J])
                if J != I and abs(F - thr) > 1e-12 * F:
                    assert ns[t] == (F >= thr)
                if J == I:
                    assert ns[t] == 0
        # entries inside a node's block are strong, others take their node pair's flag
        rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
        for e in range(A.nnz):
            I, J = rows[e] // 3, A.col[e] // 3
            if I == J:
                assert strong[e] == (A.col[e] != rows[e])
            else:
                t = nrp[I] + list(nci[nrp[I]:nrp[I + 1]]).index(J)
                assert strong[e] == ns[t]


# ------------------------------------------------------------------ QR tentative prolongator

def test_block_tentative_qr_identities(oracle_lib):
    A = _box(4, 3, 3)
    B = A.meta["rbm"]
    bs, k = 3, 6
    nn = A.n // bs
    nagg = 7
    # contiguous runs of ~11 nodes (each spans several grid lines: rank 6), then shuffled labels
    node_agg = np.random.default_rng(1).permutation(nagg)[(np.arange(nn) * nagg) // nn].astype(np.int32)
    Qv, Bc, st = oracle_lib.block_tentative(A.n, bs, k, node_agg, nagg, B)
    assert st == 0
    # Pt Bc = B
    Pt = np.zeros((A.n, nagg * k))
    for i in range(A.n):
        a = node_agg[i // bs]
        Pt[i, a * k:a * k + k] = Qv[i]
    assert np.abs(Pt @ Bc.T - B.T).max() <= 1e-13 * np.abs(B).max()
    # orthonormal columns, R upper triangular with a positive diagonal
    assert np.abs(Pt.T @ Pt - np.eye(nagg * k)).max() <= 1e-13
    for a in range(nagg):
        R = Bc[:, a * k:a * k + k].T
        assert np.all(np.tril(R, -1) == 0) and np.all(np.diag(R) > 0)
    # an aggregate of one node carries 3 unknowns: it cannot hold 6 independent vectors
    node_agg2 = node_agg.copy()
    node_agg2[:] = np.minimum(node_agg2, nagg - 1)
    node_agg2[0] = nagg                                     # a one-node aggregate
    _, _, st2 = oracle_lib.block_tentative(A.n, bs, k, node_agg2, nagg + 1, B)
    assert st2 == oracle_lib.ERR_UNSUPPORTED


# ------------------------------------------------------------------ the whole method

def test_galerkin_annihilates_coarse_nullspace(oracle_lib):
    # theta = 0 on the Neumann operator: Abar = A, A B = 0, so P Bc = B and R A P Bc = 0
    A = _box(4, 4, 3, clamp=False)
    B = A.meta["rbm"]
    h, st = oracle_lib.prolongator_only(A, nullspace=B, theta=0.0, block_size=3, nullspace_dim=6)
    assert st == 0
    l0 = h.level(0)
    Pm = l0["P"]
    import scipy.sparse as sp
    nagg = l0["nagg"]
    Psp = sp.csr_matrix((Pm.val, Pm.col, Pm.row_ptr), shape=(A.n, nagg * 6))
    Bc = None
    # Bc from the QR of the same aggregates
    _, Bc, st2 = oracle_lib.block_tentative(A.n, 3, 6, l0["agg"], nagg, B)
    assert st2 == 0
    S = A.to_scipy()
    PB = Psp @ Bc.T
    assert np.abs(PB - B.T).max() <= 1e-10 * np.abs(B).max()
    Ac = Psp.T @ (S @ Psp)
    assert np.abs(Ac @ Bc.T).max() <= 1e-10 * abs(Ac).max()
    assert abs(Ac - Ac.T).max() <= 1e-13 * abs(Ac).max()


def _interleave(A, copies):
    """copies decoupled copies of scalar A, interleaved (unknown copies v + c)."""
    rows, cols, vals = [], [], []
    r = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    for c in range(copies):
        rows.append(copies * r + c)
        cols.append(copies * A.col.astype(np.int64) + c)
        vals.append(A.val)
    rows, cols, vals = (np.concatenate(x) for x in (rows, cols, vals))
    o = np.lexsort((cols, rows))
    n = copies * A.n
    rp = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rp, rows[o] + 1, 1)
    return P.CSR(n, np.cumsum(rp), cols[o].astype(np.int32), vals[o])


def test_decoupled_system_equals_scalar_hierarchy(oracle_lib):
    # two interleaved copies of a scalar operator with the two component constants: theta = 0
    # (every coupling strong) and a fixed lambda make the block path the scalar one, copy by copy
    A = P.stretched_box(8, 1.1)
    A2 = _interleave(A, 2)
    kw = dict(theta=0.0, lambda_override=1.7)
    hs, st = oracle_lib.setup(A, max_coarse=30, **kw)
    hb, st2 = oracle_lib.setup(A2, block_size=2, nullspace_dim=2, max_coarse=60, **kw)
    assert st == st2 == 0 and hs.nlevels == hb.nlevels
    for l in range(hs.nlevels - 1):
        assert np.array_equal(hs.get(l, "agg"), hb.get(l, "agg"))
        Ps, Pb = hs.level(l)["P"], hb.level(l)["P"]
        Ab, As = hb.get(l + 1, "A.v"), hs.get(l + 1, "A.v")
        # P of the system = P of the scalar operator on each copy
        import scipy.sparse as sp
        na = hs.level(l)["nagg"]
        Psc = sp.csr_matrix((Ps.val, Ps.col, Ps.row_ptr), shape=(Ps.n, na)).toarray()
        Pbl = sp.csr_matrix((Pb.val, Pb.col, Pb.row_ptr), shape=(Pb.n, 2 * na)).toarray()
        # (equal to rounding: the scalar path scales P's columns after smoothing, the QR path
        # smooths the orthonormal Pt)
        for c in range(2):
            assert np.abs(Pbl[c::2, c::2] - Psc).max() <= 1e-13 * np.abs(Psc).max()
            assert not Pbl[c::2, 1 - c::2].any()
        nb = len(hb.get(l + 1, "A.rp")) - 1
        ns_ = len(hs.get(l + 1, "A.rp")) - 1
        Db = sp.csr_matrix((Ab, hb.get(l + 1, "A.ci"), hb.get(l + 1, "A.rp")), shape=(nb, nb)).toarray()
        Ds = sp.csr_matrix((As, hs.get(l + 1, "A.ci"), hs.get(l + 1, "A.rp")), shape=(ns_, ns_)).toarray()
        for c in range(2):
            assert np.abs(Db[c::2, c::2] - Ds).max() <= 1e-12 * np.abs(Ds).max()
            assert not Db[c::2, 1 - c::2].any()


def test_block_path_errors(oracle_lib):
    A = _box(3, 3, 3)
    B = A.meta["rbm"]
    h, st = oracle_lib.setup(A, nullspace=B, block_size=3, nullspace_dim=6, variants=1)
    assert h is None and st == oracle_lib.ERR_UNSUPPORTED
    h, st = oracle_lib.setup(A, block_size=3, nullspace_dim=6)          # no vectors given, k != bs
    assert h is None and st == oracle_lib.ERR_INVALID_ARG
    A2 = P.stretched_box(5, 1.1)                                       # 125 rows: not a multiple of 2
    h, st = oracle_lib.setup(A2, block_size=2, nullspace_dim=2)
    assert h is None and st == oracle_lib.ERR_INVALID_ARG


def test_rigid_body_modes_beat_translations(oracle_lib):
    A = _box(10, 10, 10)
    b = P.rhs_uniform(A.n, 1)
    h6, st = oracle_lib.setup(A, nullspace=A.meta["rbm"], theta=0.02, block_size=3, nullspace_dim=6,
                              max_coarse=100)
    h3, st3 = oracle_lib.setup(A, theta=0.02, block_size=3, nullspace_dim=3, max_coarse=100)
    assert st == st3 == 0
    x6, i6, s6 = h6.solve(b, 1e-8)
    x3, i3, s3 = h3.solve(b, 1e-8)
    _, ip = oracle_lib.pcg_plain(A, b, 1e-8, 5000)
    assert s6 == s3 == 0
    assert i6.iters < i3.iters < ip.iters
    assert np.linalg.norm(b - A.to_scipy() @ x6) / np.linalg.norm(b) <= 1e-8
    # the V-cycle is a symmetric operator
    f, g = P.rhs_uniform(A.n, 2), P.rhs_uniform(A.n, 3)
    Mf, Mg = h6.vcycle(f), h6.vcycle(g)
    assert abs(f @ Mg - g @ Mf) <= 1e-12 * abs(f @ Mg)
