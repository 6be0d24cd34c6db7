"""Pins of the oracle's sums along long stored rows (the filtered matrix of Eq. 6 and
Algorithm 2, the 1Norm diagonal of Eq. 9-10).

The paper fixes no summation order.  The oracle sums a row of at most 256 stored positions left
to right; a longer row (stalled coarse levels hold rows of thousands) in segments of 256
positions, each left to right from 0, the segment sums then added left to right.  The pins:

* exactness on dyadic values (every partial sum representable, so any order gives the exact
  sum): a term dropped or counted twice at a segment boundary, or a whole segment lost, changes
  the result;
* the error bound of recursive summation on random values, against math.fsum;
* composition: a long row's result from the results of the same oracle on short rows (whose
  left-to-right sums the other filter pins fix), which is what the segment rule states.
"""
import math

import numpy as np
import pytest

from paper_2103_10476_gb300.problems import CSR

SEG = 256


def _one_long_row(vals_off, diag=0.0, tail_rows=True):
    """Row 0 = [diag, vals_off...] on columns 0..m; rows 1..m are 1 x 1 identities (coupled back
    to row 0 only when tail_rows, so that the matrix stays structurally symmetric)."""
    m = len(vals_off)
    n = m + 1
    rp = [0]
    ci = []
    v = []
    ci += list(range(n))
    v += [diag] + list(vals_off)
    rp.append(len(ci))
    for j in range(1, n):
        if tail_rows:
            ci += [0, j]
            v += [vals_off[j - 1], 1.0]
        else:
            ci += [j]
            v += [1.0]
        rp.append(len(ci))
    return CSR(n, np.array(rp, np.int64), np.array(ci, np.int32), np.array(v, np.float64))


def _row0_removed(A, mask_off):
    """removed flags: row 0's off-diagonals where mask_off, nothing else"""
    rem = np.zeros(len(A.col), np.uint8)
    m = len(mask_off)
    rem[1:m + 1] = mask_off.astype(np.uint8)
    return rem


@pytest.mark.parametrize("m", [255, 256, 257, 511, 512, 513, 1000, 3000])
def test_lumped_diagonal_exact_on_dyadic_values(oracle_lib, m):
    # values k / 1024 with small integers k: every partial sum is exact in FP64
    rng = np.random.default_rng(m)
    k = rng.integers(-64, 65, size=m)
    vals = k / 1024.0
    mask = rng.random(m) < 0.5
    # removed entries on both sides of every segment boundary
    for b in range(SEG - 1, m + 1, SEG):
        for t in (b - 2, b - 1, b, b + 1):
            if 0 <= t < m:
                mask[t] = True
    A = _one_long_row(vals, diag=8.0)
    Ab, _ = oracle_lib.filtered(A, _row0_removed(A, mask), offlmp=False)
    exact = 8.0 + int(k[mask].sum()) / 1024.0
    assert Ab.col[0] == 0 and Ab.val[0] == exact
    # kept entries unchanged, in order
    kept = np.nonzero(~mask)[0]
    e = Ab.row_ptr[1]
    assert np.array_equal(Ab.col[1:e], kept + 1) and np.array_equal(Ab.val[1:e], vals[kept])


@pytest.mark.parametrize("m", [300, 1000, 7000])
def test_lumped_diagonal_within_recursive_summation_bound(oracle_lib, m):
    rng = np.random.default_rng(7 + m)
    vals = -np.exp(rng.uniform(-6, 0, m))
    mask = rng.random(m) < 0.7
    A = _one_long_row(vals, diag=0.0)
    Ab, _ = oracle_lib.filtered(A, _row0_removed(A, mask), offlmp=False)
    terms = vals[mask]
    exact = math.fsum(terms)
    # any recursive summation of q terms: |error| <= (q - 1) u sum |terms| (to first order)
    bound = (len(terms) + 1) * 2.0 ** -53 * float(np.abs(terms).sum())
    assert abs(Ab.val[0] - exact) <= bound


def test_long_row_composes_from_short_rows(oracle_lib):
    # A row of 600 positions: the diagonal first (0.0, not a term, so the lumped diagonal is
    # 0 + r_i = r_i exactly), then entries e_0 .. e_598.  Segments are positions 0-255, 256-511
    # and 512-599.  With the first entry of segments 1 and 2 kept (not a term), each segment's
    # terms are exactly those of a short row [0, entries] of at most 256 positions, whose lumped
    # diagonal is their left-to-right sum from 0; the long row's r_i must be those three sums
    # added left to right, bit for bit.
    rng = np.random.default_rng(11)
    m = 599
    vals = rng.normal(size=m)
    mask = rng.random(m) < 0.6
    mask[SEG - 1] = False            # entry at position 256
    mask[2 * SEG - 1] = False        # entry at position 512
    A = _one_long_row(vals, diag=0.0, tail_rows=False)
    Ab, _ = oracle_lib.filtered(A, _row0_removed(A, mask), offlmp=False)
    pieces = [(0, SEG - 1), (SEG, 2 * SEG - 1), (2 * SEG, m)]    # entry ranges of the short rows
    sums = []
    for lo, hi in pieces:
        sub = _one_long_row(vals[lo:hi], diag=0.0, tail_rows=False)
        assert sub.row_ptr[1] <= SEG
        S, _ = oracle_lib.filtered(sub, _row0_removed(sub, mask[lo:hi]), offlmp=False)
        sums.append(S.val[0])
    assert Ab.val[0] == (sums[0] + sums[1]) + sums[2]
    terms = vals[mask]
    assert abs(Ab.val[0] - math.fsum(terms)) <= (len(terms) + 1) * 2.0 ** -53 * np.abs(terms).sum()


def test_offlmp_long_row_diagonal_branch_exact(oracle_lib):
    # Algorithm 2 with r_i >= 0 (every removed entry positive): all of r_i goes to the diagonal;
    # dyadic values make it exact, and kept entries are unchanged
    rng = np.random.default_rng(5)
    m = 1500
    k = rng.integers(1, 33, size=m) * np.where(rng.random(m) < 0.5, 1, -1)
    vals = k / 512.0
    mask = vals > 0
    A = _one_long_row(vals, diag=64.0)
    Ab, flag = oracle_lib.filtered(A, _row0_removed(A, mask), offlmp=True, tau=1.1)
    assert flag[0] == 0                                    # the diagonal branch
    assert Ab.val[0] == 64.0 + int(k[mask].sum()) / 512.0


def test_offlmp_long_row_kplus_branch_preserves_row_sum(oracle_lib):
    # r_i < 0 with |r_i| <= kappa+: K+ absorbs r_i (scaled by 1 + r_i / kappa+), the row sum is
    # preserved to rounding; kappa+ and r_i are sums over 2 000 positions
    rng = np.random.default_rng(9)
    m = 2000
    vals = np.where(rng.random(m) < 0.5, 1.0, -1.0) * rng.uniform(0.1, 1.0, m)
    mask = (vals < 0) & (rng.random(m) < 0.5)
    A = _one_long_row(vals, diag=1.5 * np.abs(vals).sum())
    Ab, flag = oracle_lib.filtered(A, _row0_removed(A, mask), offlmp=True, tau=1.1)
    assert flag[0] == 1                                    # the K+ branch
    e = Ab.row_ptr[1]
    before = math.fsum(A.val[:m + 1])
    after = math.fsum(Ab.val[:e])
    assert abs(after - before) <= 1e-12 * np.abs(vals).sum()


def test_1norm_diagonal_of_long_row_exact_on_dyadic_values(oracle_lib):
    # Eq. (9)-(10) on a long filtered row: Dtilde_00 = max(sum |abar_0j|, 2 sum abar_0j); theta = 0
    # keeps every entry, so Abar = A; dyadic values make both sums exact
    rng = np.random.default_rng(13)
    m = 1200
    k = rng.integers(-40, 41, size=m)
    k[k == 0] = 1
    vals = k / 256.0
    A = _one_long_row(vals, diag=float(np.abs(k).sum()) / 256.0 + 1.0)
    h, st = oracle_lib.setup(A, theta=0.0, variants=1, max_levels=2, max_coarse=1)
    assert st == 0
    L0 = h.level(0)
    row = L0["Abar"].val[L0["Abar"].row_ptr[0]:L0["Abar"].row_ptr[1]]
    d = (float(np.abs(k).sum()) / 256.0 + 1.0) + float(np.abs(k).sum()) / 256.0
    s = (float(np.abs(k).sum()) / 256.0 + 1.0) + float(k.sum()) / 256.0
    assert np.array_equal(row, A.val[:m + 1])
    assert L0["Dsm"][0] == max(d, 2.0 * s)


def test_segment_boundary_closed_form(oracle_lib):
    # r_i over a row whose position 1 holds 1.0 and positions 2 .. 511 hold 2^-53 (all removed):
    # left to right from 0 every 2^-53 is lost against 1.0 (a tie, rounded to even), so segment 0
    # (positions 0-255) sums to exactly 1.0; segment 1 (positions 256-511) sums its 256 terms
    # exactly to 2^-45; r_i = 1 + 2^-45, exactly.  A plain left-to-right sum gives 1.0, and a
    # boundary one position off gives 1 + 129 * 2^-52.
    tiny = 2.0 ** -53
    vals = np.array([1.0] + [tiny] * 510)
    A = _one_long_row(vals, diag=0.0, tail_rows=False)
    Ab, _ = oracle_lib.filtered(A, _row0_removed(A, np.ones(len(vals), bool)), offlmp=False)
    assert Ab.val[0] == 1.0 + 2.0 ** -45


# ------------------------------------------------------------------ Galerkin products, long rows

def _csr_rows(rows, ncol):
    """CSR from a list of rows, each a list of (column, value) with ascending columns"""
    rp = [0]
    ci, v = [], []
    for r in rows:
        for j, x in r:
            ci.append(j)
            v.append(x)
        rp.append(len(ci))
    return CSR(len(rows), np.array(rp, np.int64), np.array(ci, np.int32), np.array(v, np.float64))


def _random_b(rng, nk, ncol, per_row, dyadic):
    rows = []
    for k in range(nk):
        cols = np.sort(rng.choice(ncol, size=per_row, replace=False))
        if dyadic:
            vals = rng.integers(-8, 9, size=per_row) / 16.0
        else:
            vals = rng.normal(size=per_row)
        rows.append(list(zip(cols.tolist(), vals.tolist())))
    return rows


@pytest.mark.parametrize("m", [256, 257, 600, 1500])
def test_spgemm_long_row_exact_on_dyadic_values(oracle_lib, m):
    # products of dyadic numbers of few bits: every partial sum exact, so C = the integer product
    rng = np.random.default_rng(m)
    ncol = 40
    Bl = _random_b(rng, m, ncol, 5, dyadic=True)
    a = rng.integers(-8, 9, size=m) / 8.0
    A = _csr_rows([list(zip(range(m), a.tolist()))], m)
    B = _csr_rows(Bl, ncol)
    C = oracle_lib.spgemm(A, B, ncol)
    dense_b = np.zeros((m, ncol))
    for k, r in enumerate(Bl):
        for j, x in r:
            dense_b[k, j] = x
    ref = (a * 8.0).astype(np.int64) @ (dense_b * 16.0).astype(np.int64)
    got = np.zeros(ncol)
    got[C.col] = C.val
    assert np.array_equal(got, ref / 128.0)
    assert np.array_equal(np.sort(C.col), np.nonzero((dense_b != 0).any(0))[0])


def test_spgemm_long_row_composes_from_short_rows(oracle_lib):
    # row of 700 entries = segments of 256, 256 and 188; each segment's sums are those of the
    # short row holding its entries (the plain rule, pinned against scipy elsewhere); the long
    # row's c_ij are the segment results added in order, bit for bit (a column missing from a
    # segment contributes 0)
    rng = np.random.default_rng(3)
    m, ncol = 700, 30
    Bl = _random_b(rng, m, ncol, 4, dyadic=False)
    a = rng.normal(size=m)
    B = _csr_rows(Bl, ncol)
    C = oracle_lib.spgemm(_csr_rows([list(zip(range(m), a.tolist()))], m), B, ncol)
    parts = []
    for lo, hi in ((0, SEG), (SEG, 2 * SEG), (2 * SEG, m)):
        S = oracle_lib.spgemm(_csr_rows([list(zip(range(lo, hi), a[lo:hi].tolist()))], m), B, ncol)
        d = np.zeros(ncol)
        d[S.col] = S.val
        parts.append(d)
    got = np.zeros(ncol)
    got[C.col] = C.val
    assert np.array_equal(got, (parts[0] + parts[1]) + parts[2])


def test_spgemm_segment_boundary_closed_form(oracle_lib):
    # c_00 = sum_k a_0k b_k0 with a_00 b_00 = 1 and 511 terms 2^-53 after it: segment 0 (terms
    # 0-255) rounds to 1 exactly, segment 1 (terms 256-511) is 256 x 2^-53 = 2^-45 exactly,
    # c_00 = 1 + 2^-45; the plain left-to-right rule would give 1
    tiny = 2.0 ** -53
    m = 512
    a = np.array([1.0] + [tiny] * (m - 1))
    A = _csr_rows([list(zip(range(m), a.tolist()))], m)
    B = _csr_rows([[(0, 1.0)] for _ in range(m)], 1)
    C = oracle_lib.spgemm(A, B, 1)
    assert C.val[0] == 1.0 + 2.0 ** -45
