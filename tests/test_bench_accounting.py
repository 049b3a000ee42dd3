"""The benchmark's per-step accounting (host logic, no GPU): the method's algorithmic bytes and
flops, the executed counts of each kernel form, and the ensemble's, against counts taken
directly from a problem's arrays."""
import numpy as np

import bench
import m3d_inputs as mi


def counts(p):
    nnz = int(p.exp_rowptr[-1])
    L = np.diff(p.col_start)
    s_imp = int(np.sum(L.astype(np.int64) ** 2))
    n_eu = int(np.sum(np.minimum(L, 2)))
    return nnz, s_imp, n_eu


def test_method_count_matches_the_arrays():
    p = mi.make_problem("tiny_6x4x4")
    nnz, s_imp, n_eu = counts(p)
    assert nnz == p.nnz and s_imp == p.s_imp
    b, f = bench.method_per_step(p)
    # two months of values (8 B each) and an int32 index per entry, row pointers, two months
    # of dense blocks, two tracers read and written
    assert b == nnz * 20 + 4 * (p.n + 1) + s_imp * 16 + 2 * p.n * 16
    # interpolation plus one FMA per tracer for every explicit and block entry, ~50 flops per
    # euphotic cell and tracer
    assert f == (nnz + s_imp) * 6 + 50 * n_eu * 2


def test_executed_forms_differ_from_the_method_where_they_should():
    p = mi.make_problem("ndop_64x32x8")
    nnz, s_imp, n_eu = counts(p)
    b_m, _ = bench.method_per_step(p)
    b_d, f_d = bench.executed_per_step(p, tridiagonal=False)
    b_t, f_t = bench.executed_per_step(p, tridiagonal=True)
    b_s, f_s = bench.executed_per_step(p, tridiagonal=True, step_operators=True)
    assert b_d == b_m                                   # the dense form moves the method's bytes
    assert b_t == b_d - s_imp * 16 + 2 * 3 * p.n * 8   # Thomas factors instead of dense blocks
    assert f_t == f_d - s_imp * 6 + 13 * 2 * p.n
    assert b_s == b_t - nnz * 8                         # one interpolated matrix per step
    assert f_s == f_t - nnz * 2                         # no interpolation in the kernel
    assert f_s < f_t < f_d


def test_ensemble_counts():
    p = mi.make_problem("tiny_6x4x4")
    nnz, s_imp, _ = counts(p)
    members = mi.make_ensemble(((mi.MODEL_NDOP, 2), (mi.MODEL_NPZD, 1)), seed=2)
    W = sum(m.ntracer for m in members)
    assert W == 2 * 2 + 5
    alg = bench.ensemble_flops_per_step(p, members)
    ex = bench.ensemble_flops_per_step(p, members, executed=True)
    assert alg - ex == s_imp * (2 + 2 * W) - 13 * p.n * W
    # one member of the ensemble's count carries the explicit part once for all its tracers
    one = bench.ensemble_flops_per_step(p, members[:1])
    assert one < alg
