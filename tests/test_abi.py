"""The C ABI library loads and exports every function include/metos3d.h declares (no GPU needed)."""
import ctypes
import os

import numpy as np
import pytest

import paper_1410_0204_gb300 as m3d
from paper_1410_0204_gb300 import build as b


@pytest.fixture(scope="module")
def lib():
    b.build()
    return ctypes.CDLL(b.LIB)


def test_header_declares_the_boundary():
    names = m3d.declared_symbols()
    for required in ("metos3d_init", "metos3d_step", "metos3d_year_map", "metos3d_year_map_host",
                     "metos3d_mass", "metos3d_residual", "metos3d_bgc", "metos3d_free", "metos3d_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in m3d.declared_symbols():
        assert hasattr(lib, name), name


def test_binding_loads(lib):
    L = m3d.load()
    assert L is not None
    assert os.path.exists(m3d.library_path())


def test_init_rejects_bad_grid_without_gpu_work(lib):
    # argument validation happens before any device call
    L = m3d.load()
    ctx = ctypes.c_void_p()
    assert L.metos3d_init(ctypes.byref(ctx), None, None, None, None) == m3d.M3D_ERR_ARG
    assert b"null" in L.metos3d_last_error(None)


def test_ensemble_init_rejects_bad_members_without_gpu_work(lib):
    # member checks happen before any device call
    import types
    import m3d_inputs as mi
    p = mi.make_problem("tiny_4x3x3")
    fake_stream = types.SimpleNamespace(cuda_stream=0)
    with pytest.raises(m3d.Metos3dError) as ei:
        m3d.Ensemble.from_problem(p, [(mi.MODEL_NDOP, mi.default_params(mi.MODEL_NDOP)[:5])], stream=fake_stream)
    assert ei.value.status == m3d.M3D_ERR_ARG and "parameters" in str(ei.value)
    with pytest.raises(m3d.Metos3dError) as ei:
        m3d.Ensemble.from_problem(p, [(4, np.zeros(4))], stream=fake_stream)
    assert ei.value.status == m3d.M3D_ERR_UNSUPPORTED
    with pytest.raises(m3d.Metos3dError) as ei:
        m3d.Ensemble.from_problem(p, [], stream=fake_stream)
    assert ei.value.status == m3d.M3D_ERR_ARG


def test_single_context_model_counts_are_checked_without_gpu_work(lib):
    import types
    import m3d_inputs as mi
    p = mi.make_problem("tiny_4x3x3")
    fake_stream = types.SimpleNamespace(cuda_stream=0)
    with pytest.raises(m3d.Metos3dError) as ei:
        m3d.Context.from_problem(p, model=m3d.MODEL_PHY, ntracer=2, nparam=11, stream=fake_stream)
    assert ei.value.status == m3d.M3D_ERR_ARG and "3 tracers and 11 parameters" in str(ei.value)
    with pytest.raises(m3d.Metos3dError) as ei:
        m3d.Context.from_problem(p, model=4, ntracer=4, nparam=4, stream=fake_stream)
    assert ei.value.status == m3d.M3D_ERR_UNSUPPORTED


def test_every_entry_point_rejects_a_null_handle_without_gpu_work(lib):
    """Each call that takes a context or an ensemble returns M3D_ERR_ARG (or its documented
    sentinel) for a NULL handle, before any device work, and leaves a message behind."""
    L = ctypes.CDLL(b.LIB)
    vp, i, d, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    N = None
    calls = {
        "metos3d_set_stream": (N, N),
        "metos3d_step": (N, i(0), N, N, N),
        "metos3d_year_map": (N, N, N, N),
        "metos3d_year_map_host": (N, N, N, N),
        "metos3d_year_tangent": (N, N, N, N, N, N),
        "metos3d_year_adjoint": (N, N, N, N, N, N, i(240)),
        "metos3d_mass": (N, N, N),
        "metos3d_residual": (N, N, N, N),
        "metos3d_check_finite": (N, N),
        "metos3d_sync": (N,),
        "metos3d_set_option": (N, i(0), ll(0)),
        "metos3d_spinup": (N, N, N, i(1), d(0.0), N, N),
        "metos3d_newton_solve": (N, N, N, N, N),
        "metos3d_periodic_gradient": (N, N, N, N, N, N, N, N),
        "metos3d_info": (N, N, N, N, N),
        "metos3d_ensemble_layout": (N, N, N, N, N, N),
        "metos3d_ensemble_set_stream": (N, N),
        "metos3d_ensemble_set_params": (N, i(0), N),
        "metos3d_ensemble_steps": (N, i(0), i(1), N, N),
        "metos3d_ensemble_year_map": (N, N, N),
        "metos3d_ensemble_set_tiling": (N, i(1), i(4)),
        "metos3d_ensemble_get_tiling": (N, N, N),
        "metos3d_ensemble_autotune": (N, N, i(1), N, N, N),
        "metos3d_ensemble_year_adjoint": (N, N, N, N, N, i(240)),
        "metos3d_ensemble_newton_solve": (N, N, N, N, N, N),
    }
    assert set(calls) | {"metos3d_init", "metos3d_ensemble_init", "metos3d_ensemble_init_tangent", "metos3d_bgc",
                         "metos3d_residual_static", "metos3d_residual_static_error", "metos3d_get_option",
                         "metos3d_newton_default_options", "metos3d_gradient_default_options",
                         "metos3d_ensemble_last_launch_count", "metos3d_ensemble_last_error",
                         "metos3d_ensemble_free", "metos3d_last_launch_count", "metos3d_last_error",
                         "metos3d_free"} == set(m3d.declared_symbols())
    for name, args in calls.items():
        f = getattr(L, name)
        f.restype = ctypes.c_int
        assert f(*args) == m3d.M3D_ERR_ARG, name
    for name in ("metos3d_get_option",):
        f = getattr(L, name)
        f.restype = ll
        assert f(N, i(0)) == -1
    for name in ("metos3d_last_launch_count", "metos3d_ensemble_last_launch_count"):
        f = getattr(L, name)
        f.restype = ll
        assert f(N) == -1, name
    L.metos3d_last_error.restype = ctypes.c_char_p
    L.metos3d_ensemble_last_error.restype = ctypes.c_char_p
    assert L.metos3d_last_error(N) is not None and L.metos3d_ensemble_last_error(N) is not None
    L.metos3d_free(N)
    L.metos3d_ensemble_free(N)


def test_bgc_interface_checks_its_arguments_without_gpu_work(lib):
    """The model interface of Section 5.2 rejects bad sizes and arrays before it touches the
    device: no layers, too many layers, no internal step, the wrong tracer or parameter count
    for PO4-DOP, a missing array; an unknown model is unsupported."""
    L = m3d.load()
    h = np.array([50.0, 70.0, 90.0])
    d = np.cumsum(h) - 0.5 * h
    y = np.full(6, 2.0)
    out = np.zeros(6)
    u = np.ones(7)
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))  # noqa: E731

    def call(model=m3d.MODEL_NDOP, ntr=2, nl=3, nparam=7, nsub=1, hh=h, uu=u):
        return L.metos3d_bgc(model, 0.0, 1.0 / 2880, 0.0, 300.0, 0.5, 0.0, 0.0, ntr, nl,
                             dp(hh) if hh is not None else None, dp(d), None, None, dp(y), dp(out),
                             nparam, dp(uu) if uu is not None else None, nsub)

    assert call(nl=0) == m3d.M3D_ERR_ARG
    assert call(nl=100000) == m3d.M3D_ERR_ARG
    assert call(nsub=0) == m3d.M3D_ERR_ARG
    assert call(ntr=3) == m3d.M3D_ERR_ARG
    assert call(nparam=6) == m3d.M3D_ERR_ARG
    assert call(hh=None) == m3d.M3D_ERR_ARG
    assert call(uu=None) == m3d.M3D_ERR_ARG
    assert call(model=4) == m3d.M3D_ERR_UNSUPPORTED
    assert np.all(out == 0.0)


def test_init_validates_every_input_rule_without_gpu_work(lib):
    """metos3d_init checks the grid and the matrices on the host before it allocates or
    launches anything (the problem statement of Section 3): each malformed input below is
    rejected with M3D_ERR_ARG and a message naming the rule, never read out of bounds."""
    import types
    import m3d_inputs as mi
    p = mi.make_problem("ndop_64x32x8")
    fake_stream = types.SimpleNamespace(cuda_stream=0)
    base = dict(col_start=p.col_start, h=p.h, zc=p.zc, vol=p.vol, lat=p.lat, exp_rowptr=p.exp_rowptr,
                exp_colidx=p.exp_colidx, exp_val=p.exp_val, imp_blk=p.imp_blk)
    rp, ci = np.asarray(p.exp_rowptr), np.asarray(p.exp_colidx)
    r = int(np.argmax(np.diff(rp) >= 3))                 # a row with at least three entries
    a = int(rp[r])

    def changed(key, edit):
        arr = np.array(base[key], copy=True)
        edit(arr)
        return dict(base, **{key: arr})

    def shift(k):
        def edit(cs):
            cs[1] = k
        return edit

    cases = {
        "col_start must run from 0 to n": changed("col_start", lambda cs: cs.__setitem__(0, 1)),
        "layers (1..": changed("col_start", shift(0)),              # column 0 without layers
        "latitude": changed("lat", lambda x: x.__setitem__(3, 91.0)),
        "bad h, zc or vol": changed("h", lambda x: x.__setitem__(7, 0.0)),
        "bad h, zc or vol ": changed("zc", lambda x: x.__setitem__(7, np.inf)),
        "bad h, zc or vol  ": changed("vol", lambda x: x.__setitem__(7, np.nan)),
        "s_imp": dict(base, imp_blk=np.ascontiguousarray(np.asarray(p.imp_blk)[:, :-1])),
        "rowptr must run from 0 to nnz": changed("exp_rowptr", lambda x: x.__setitem__(0, 1)),
        "rowptr decreases": changed("exp_rowptr", lambda x: x.__setitem__(r + 1, x[r] - 1)),
        "rowptr exceeds nnz": changed("exp_rowptr", lambda x: x.__setitem__(1, p.nnz + 100000)),
        "column index out of range": changed("exp_colidx", lambda x: x.__setitem__(a, -1)),
        "column index out of range ": changed("exp_colidx", lambda x: x.__setitem__(a, p.n)),
        "not sorted": changed("exp_colidx", lambda x: x.__setitem__(slice(a, a + 2), x[a:a + 2][::-1].copy())),
        "not sorted ": changed("exp_colidx", lambda x: x.__setitem__(a + 1, x[a])),
        "non-finite values": changed("exp_val", lambda x: x.__setitem__((5, 11), np.nan)),
        "non-finite values ": changed("imp_blk", lambda x: x.__setitem__((11, 2), np.inf)),
    }
    cs = np.asarray(base["col_start"])
    k = int(np.argmax(cs > 64))                               # merge columns 0..k-1 into one deeper than 64
    cases["layers (1..%d allowed)" % 64] = dict(base, col_start=np.concatenate([[0], cs[k:]]).astype(np.int32),
                                                lat=np.asarray(base["lat"])[k - 1:])
    for rule, kw in cases.items():
        with pytest.raises(m3d.Metos3dError) as ei:
            m3d.Context(**kw, stream=fake_stream)
        assert ei.value.status == m3d.M3D_ERR_ARG, rule
        assert rule.strip() in str(ei.value), (rule, str(ei.value))
