"""Pins of the general-hexahedron generator and of the oracle's distance-Laplacian strength
(§3.1: strength of connection, Eq. 7, evaluated on a Laplacian built from the distances
between the coordinates of coupled rows; coarse coordinates are aggregate centroids).

Each test checks against something other than the code under test: the closed-form Q1
element matrices of a box, exact energy identities of linear functions, closed-form
distances on a uniform grid, exact scaling invariance, brute force on tiny inputs.
"""
import numpy as np
import pytest

from paper_2103_10476_gb300 import problems as P


def _box_nodes(ax, ay, az):
    Z, Y, X = np.meshgrid(az, ay, ax, indexing="ij")
    return X, Y, Z


# ------------------------------------------------------------------ generator

def test_hex_unit_cube_element_matrices_closed_form():
    # one element, all nodes kept: the Q1 Laplacian of the unit cube has 1/3 on the diagonal,
    # 0 between nodes on a common edge, -1/12 across a face diagonal and across the body;
    # the mass matrix is the tensor product of h/6 [2 1; 1 2]
    X, Y, Z = _box_nodes([0.0, 1.0], [0.0, 1.0], [0.0, 1.0])
    K = P.hex_q1_matrix(X, Y, Z, dirichlet=False).to_dense()
    KM = P.hex_q1_matrix(X, Y, Z, coef=np.zeros((1, 1, 1)), reaction=1.0, dirichlet=False).to_dense()
    for a in range(8):
        for b in range(8):
            d = bin(a ^ b).count("1")
            assert K[a, b] == pytest.approx({0: 1 / 3, 1: 0.0, 2: -1 / 12, 3: -1 / 12}[d], abs=1e-15)
            assert KM[a, b] == pytest.approx({0: 8, 1: 4, 2: 2, 3: 1}[d] / 216.0, abs=1e-16)


def test_hex_tensor_mesh_matches_tensor_assembly():
    hx, hy, hz = np.array([0.5, 1.0, 0.7, 1.3]), np.array([1.0, 0.8, 1.2]), np.array([0.9, 1.1, 1.0, 0.6, 1.4])
    A = P.q1_matrix(hx, hy, hz)
    X, Y, Z = _box_nodes(*[np.r_[0.0, np.cumsum(h)] for h in (hx, hy, hz)])
    B = P.hex_q1_matrix(X, Y, Z)
    assert np.array_equal(A.row_ptr, B.row_ptr) and np.array_equal(A.col, B.col)
    assert np.abs(A.val - B.val).max() <= 1e-14 * np.abs(A.val).max()


def test_hex_general_mesh_energy_of_linear_functions():
    # on any mesh of trilinear hexahedra, Q1 reproduces linear u = a . x, whose gradient is a:
    # u^T K u = |a|^2 vol and K 1 = 0 (Neumann), with vol = 1^T M 1 (the 2x2x2 rule is exact
    # for these integrands)
    rng = np.random.default_rng(7)
    n1 = 5
    g = np.arange(n1, dtype=np.float64)
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    X = X + 0.3 * rng.random(X.shape)
    Y = Y + 0.3 * rng.random(Y.shape)
    Z = 2.0 * (Z + 0.3 * rng.random(Z.shape))
    K = P.hex_q1_matrix(X, Y, Z, dirichlet=False)
    M = P.hex_q1_matrix(X, Y, Z, coef=np.zeros((n1 - 1,) * 3), reaction=1.0, dirichlet=False)
    xyz = K.meta["coords"]
    vol = M.to_scipy().sum()
    S = K.to_scipy()
    assert np.abs(S @ np.ones(K.n)).max() < 1e-12
    for a in (np.array([1.0, 0.0, 0.0]), np.array([0.3, -1.2, 0.7])):
        u = xyz @ a
        assert u @ (S @ u) == pytest.approx(float(a @ a) * vol, rel=1e-12)
    St = S - S.T
    assert St.count_nonzero() == 0 or abs(St).max() == 0.0


def test_perturbed_and_graded_cubes_shapes():
    A = P.perturbed_cube(6)
    assert A.n == 5 ** 3 and A.meta["coords"].shape == (A.n, 3)
    zs = A.meta["coords"][:, 2]
    xs = A.meta["coords"][:, 0]
    assert zs.max() - zs.min() > 50 * (xs.max() - xs.min())      # 100:1 in z
    h = P.graded_sizes(10.0)
    assert h[0] == pytest.approx(0.1) and h[-1] == pytest.approx(1.0) and h.sum() == pytest.approx(33.0)
    G = P.graded_cube(1, 5, 10, 1e2, ne=8)
    # the reaction term makes every row sum positive (§3.2)
    assert (np.add.reduceat(G.val, G.row_ptr[:-1]) > 0).all()


# ------------------------------------------------------------------ distance Laplacian

def _uniform(ne, h):
    ax = h * np.arange(ne + 1, dtype=np.float64)
    return P.hex_q1_matrix(*_box_nodes(ax, ax, ax))


def test_distance_laplacian_uniform_grid_closed_form(oracle_lib):
    h = 0.5
    A = _uniform(8, h)
    L, st = oracle_lib.distance_laplacian(A, A.meta["coords"])
    assert st == 0
    nx = A.meta["grid"][0]
    r = 3 + nx * (3 + nx * 3)
    want = {1: -1 / h, 2: -1 / (h * np.sqrt(2)), 3: -1 / (h * np.sqrt(3))}
    diag = 6 / h + 12 / (h * np.sqrt(2)) + 8 / (h * np.sqrt(3))
    for e in range(A.row_ptr[r], A.row_ptr[r + 1]):
        c = int(A.col[e])
        d = (abs(c % nx - r % nx) + abs((c // nx) % nx - (r // nx) % nx) + abs(c // (nx * nx) - r // (nx * nx)))
        assert L[e] == pytest.approx(diag if d == 0 else want[d], rel=1e-14)
    # every row sums to zero
    sums = np.add.reduceat(L, A.row_ptr[:-1])
    diag_all = L[A.col == np.repeat(np.arange(A.n), np.diff(A.row_ptr))]
    assert np.abs(sums).max() <= 1e-14 * diag_all.max()


@pytest.mark.parametrize("theta,count", [(0.025, 26), (0.035, 18), (0.045, 6), (0.06, 0)])
def test_distance_strength_thresholds_on_uniform_grid(oracle_lib, theta, count):
    # interior node with interior neighbours: |L_ij| / L_ii = 1 / 19.104 (faces), 0.0370
    # (edges), 0.0302 (corners), so theta decides class by class (1Norm: keeping only the
    # face entries, which are 0 for this operator, would leave the lumped diagonal 0)
    A = _uniform(8, 0.5)
    h, st = oracle_lib.setup(A, coords=A.meta["coords"], theta=theta, strength=1, max_coarse=10,
                             variants=["1norm"])
    assert st == 0
    s = h.get(0, "strong")
    nx = A.meta["grid"][0]
    r = 3 + nx * (3 + nx * 3)
    assert int(s[A.row_ptr[r]:A.row_ptr[r + 1]].sum()) == count


def test_distance_strength_scale_invariant_and_theta0(oracle_lib):
    A = P.perturbed_cube(8)
    X = A.meta["coords"]
    h1, _ = oracle_lib.setup(A, coords=X, theta=0.025, strength=1, max_coarse=20)
    h2, _ = oracle_lib.setup(A, coords=2.0 * X, theta=0.025, strength=1, max_coarse=20)
    # doubling every coordinate halves every L entry exactly: the same decisions
    assert np.array_equal(h1.get(0, "strong"), h2.get(0, "strong"))
    # and the coarse coordinates (sums and divisions of doubled values) double exactly
    assert np.array_equal(2.0 * h1.get(1, "coords"), h2.get(1, "coords"))
    # theta = 0 keeps every entry whatever the criterion: the matrix criterion's hierarchy
    h3, _ = oracle_lib.setup(A, coords=X, theta=0.0, strength=1, max_coarse=20)
    h4, _ = oracle_lib.setup(A, theta=0.0, max_coarse=20)
    for what in ("strong", "agg", "P.v"):
        assert np.array_equal(h3.get(0, what), h4.get(0, what)), what


def test_distance_strength_errors(oracle_lib):
    A = _uniform(4, 1.0)
    h, st = oracle_lib.setup(A, theta=0.025, strength=1)
    assert h is None and st == oracle_lib.ERR_INVALID_ARG
    X = A.meta["coords"].copy()
    X[1] = X[0]                                 # two coupled rows at one point
    h, st = oracle_lib.setup(A, coords=X, theta=0.025, strength=1, max_coarse=1)
    assert h is None and st == oracle_lib.ERR_INVALID_ARG


def test_coarse_coordinates_brute_force(oracle_lib):
    rng = np.random.default_rng(3)
    n, nagg, dim = 40, 7, 3
    agg = np.r_[np.arange(nagg), rng.integers(0, nagg, n - nagg)].astype(np.int32)
    X = rng.standard_normal((n, dim))
    out = oracle_lib.coarse_coords(agg, nagg, X)
    for a in range(nagg):
        for c in range(dim):
            s = 0.0
            cnt = 0
            for i in range(n):
                if agg[i] == a:
                    s = s + X[i, c]
                    cnt += 1
            assert out[a, c] == s / cnt


def test_distance_aggregates_lie_in_xy_planes(oracle_lib):
    # §3.1: with the z spacing 100x the x and y spacing, the distance criterion gives
    # aggregates oriented along x and y (the matrix criterion does not)
    A = P.perturbed_cube(12)
    nx, ny, nz = A.meta["grid"]
    idx = np.arange(A.n)
    i, j, k = idx % nx, (idx // nx) % ny, idx // (nx * ny)

    def extents(agg):
        na = int(agg.max()) + 1
        return [np.mean([v[agg == a].max() - v[agg == a].min() for a in range(na)]) for v in (i, j, k)]

    hd, _ = oracle_lib.setup(A, coords=A.meta["coords"], theta=0.025, strength=1, max_coarse=50)
    hm, _ = oracle_lib.setup(A, theta=0.025, max_coarse=50)
    ex, ey, ez = extents(hd.get(0, "agg"))
    assert ez < 0.1 * min(ex, ey)
    mx, my, mz = extents(hm.get(0, "agg"))
    assert mz > 0.5 * min(mx, my)
