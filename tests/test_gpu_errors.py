"""Error behaviour of the C ABI on a GPU: every failure is a status code, the
context stays usable, and nothing faults the device.

Failures are made on the host side of the data (bad sizes, non-finite
material values, iteration caps, an inverted deformation gradient); no test
makes a kernel fault or wait.
"""
import numpy as np
import pytest

from paper_1905_12725_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dbfft():
    from paper_1905_12725_gb300 import dbfft
    return dbfft


def _status(exc):
    from paper_1905_12725_gb300 import dbfft
    return dbfft.STATUS[exc.status]


def test_unsupported_grid_is_refused():
    dbfft = _dbfft()
    for shape in [(12, 16, 16), (16, 16, 6), (512, 8, 8)]:
        with pytest.raises(dbfft.DbfftError) as ei:
            dbfft.Solver(shape, np.zeros(shape, np.uint16), dbfft.iso_phases([1.0], [0.3]), np.zeros((1, 3, 3)))
        assert _status(ei.value) == "DBFFT_E_UNSUPPORTED_GRID"


def test_bad_arguments_are_refused():
    dbfft = _dbfft()
    shape = (8, 8, 8)
    with pytest.raises(dbfft.DbfftError) as ei:  # phase id outside the phase table
        dbfft.Solver(shape, np.full(shape, 3, np.uint16), dbfft.iso_phases([1.0, 2.0], [0.3, 0.3]),
                     np.zeros((1, 3, 3)))
    assert _status(ei.value) == "DBFFT_E_ARG"
    s = dbfft.Solver(shape, np.zeros(shape, np.uint16), dbfft.iso_phases([1.0], [0.3]), np.zeros((1, 3, 3)))
    u = torch.from_numpy(synth.random_spectrum(shape, 3, 1)).cuda()
    st = s.lib.dbfft_apply(s.ctx, 0, u.data_ptr(), None, u.data_ptr(), None)  # out aliases the input
    assert dbfft.STATUS[st] == "DBFFT_E_ARG"
    assert "alias" in s.lib.dbfft_last_error(s.ctx).decode()
    st = s.lib.dbfft_apply(s.ctx, dbfft.DBFFT_APPLY_RESIDUAL | dbfft.DBFFT_APPLY_FP32, u.data_ptr(), None,
                           torch.empty_like(u).data_ptr(), None)  # the residual exists in FP64 only
    assert dbfft.STATUS[st] == "DBFFT_E_ARG"
    assert dbfft.STATUS[s.lib.dbfft_set_precond_refresh(s.ctx, 7)] == "DBFFT_E_ARG"  # unknown policy
    with pytest.raises(dbfft.DbfftError) as ei:  # SVK needs finite kinematics
        dbfft.Solver(shape, np.zeros(shape, np.uint16), dbfft.svk_phases([1.0], [1.5]), np.zeros((1, 3, 3)))
    assert _status(ei.value) == "DBFFT_E_ARG"
    out, _ = s.apply(u)  # the context still works
    assert torch.isfinite(out).all()
    s.close()


def test_non_finite_inputs_are_reported():
    dbfft = _dbfft()
    shape = (8, 8, 16)
    scale = np.ones(shape)
    scale[3, 4, 5] = np.nan
    eps = np.zeros((1, 3, 3))
    eps[0, 0, 0] = 1e-3
    cases = [dict(phases=dbfft.iso_phases([1.0], [0.3]), target=eps, E_scale=scale),
             dict(phases=dbfft.iso_phases([np.inf], [0.3]), target=eps, E_scale=None),
             dict(phases=dbfft.iso_phases([1.0], [0.3]), target=eps * np.nan, E_scale=None)]
    for c in cases:
        with pytest.raises(dbfft.DbfftError) as ei:
            dbfft.Solver(shape, np.zeros(shape, np.uint16), c["phases"], c["target"], E_scale=c["E_scale"])
        assert _status(ei.value) == "DBFFT_E_NONFINITE"


@pytest.mark.parametrize("precision", [0, 1])
def test_iteration_cap_returns_not_converged_with_report(precision):
    dbfft = _dbfft()
    shape = (16, 16, 16)
    g = np.random.default_rng(5)
    phase = (g.random(shape) < 0.4).astype(np.uint16)
    eps = np.zeros((1, 3, 3))
    eps[0, 0, 1] = eps[0, 1, 0] = 1e-3
    s = dbfft.Solver(shape, phase, dbfft.iso_phases([1.0, 1000.0], [0.3, 0.3]), eps, tol=1e-13, max_iter=3,
                     max_newton=2, precision=precision, eta_inner=1e-3)
    rep = s.solve_increment(0, allow_not_converged=True)
    assert rep["status"] == "DBFFT_E_NOT_CONVERGED"
    assert rep["true_rel_res"] > 1e-13 and np.isfinite(rep["true_rel_res"])
    assert np.isfinite(s.homogenized_stress()).all()
    with pytest.raises(dbfft.DbfftError):
        s.solve_increment(0)
    s.close()


def test_inverted_deformation_gradient_is_a_material_failure():
    dbfft = _dbfft()
    shape = (8, 8, 8)
    F = np.diag([-0.5, 1.0, 1.0])  # det F < 0 everywhere
    s = dbfft.Solver(shape, np.zeros(shape, np.uint16), dbfft.neo_hooke_phases([1.0], [1.5]), F[None],
                     kinematics=dbfft.DBFFT_FINITE)
    with pytest.raises(dbfft.DbfftError) as ei:
        s.solve_increment(0)
    assert _status(ei.value) == "DBFFT_E_MATERIAL"
    s.close()
