"""Invariants of the synthetic inputs (they stand in for the MITgcm matrices of Section 7)."""
import numpy as np
import pytest

import m3d_inputs as mi


@pytest.fixture(scope="module", params=["tiny_4x3x3", "tiny_6x4x4", "ndop_64x32x8"])
def prob(request):
    return mi.make_problem(request.param)


def _rows(p):
    return np.repeat(np.arange(p.n), np.diff(p.exp_rowptr))


def test_sizes_of_the_paper_grid():
    # Section 7: 2.8125 degrees, 15 layers, 52749 wet cells per tracer
    p = mi.make_problem("ndop_128x64x15")
    assert p.n == 52749 and p.ncol == 4448 and p.lmax == 15
    nnz_row = np.diff(p.exp_rowptr)
    assert 10 <= nnz_row.mean() <= 20


def test_csr_is_sorted_and_in_range(prob):
    p = prob
    assert p.exp_rowptr[0] == 0 and p.exp_rowptr[-1] == p.nnz
    for i in range(0, p.n, max(1, p.n // 200)):
        cols = p.exp_colidx[p.exp_rowptr[i]:p.exp_rowptr[i + 1]]
        assert np.all(np.diff(cols) > 0) and cols.min() >= 0 and cols.max() < p.n
        assert i in cols


def test_explicit_conserves_mass_and_constants(prob):
    p = prob
    rows = _rows(p)
    for m in range(p.nmonth):
        v = p.exp_val[m]
        rs = np.zeros(p.n)
        np.add.at(rs, rows, v)
        assert np.abs(rs - 1.0).max() < 1e-14                  # A 1 = 1
        cs = np.zeros(p.n)
        np.add.at(cs, p.exp_colidx, p.vol[rows] * v)
        assert np.abs(cs / p.vol - 1.0).max() < 1e-14          # V^T A = V^T
        assert v.min() >= 0.0                                    # nonnegative
        diag = v[rows == p.exp_colidx]
        assert diag.min() >= 0.5


def test_implicit_blocks(prob):
    p = prob
    for c in range(p.ncol):
        L = int(p.nlayer[c])
        o = int(p.blk_off[c])
        assert int(p.blk_off[c + 1]) - o == L * L
        hh = p.h[p.col_start[c]:p.col_start[c + 1]]
        for m in range(p.nmonth):
            B = p.imp_blk[m, o:o + L * L].reshape(L, L)
            assert np.abs(B.sum(axis=1) - 1.0).max() < 1e-14   # A_imp 1 = 1
            assert np.abs(hh @ B / hh - 1.0).max() < 1e-14     # V^T A_imp = V^T (area is per column)
            assert B.min() >= 0.0


def test_seeded_and_deterministic():
    a = mi.make_problem("tiny_6x4x4")
    b = mi.make_problem("tiny_6x4x4")
    assert np.array_equal(a.exp_val, b.exp_val) and np.array_equal(a.imp_blk, b.imp_blk)
