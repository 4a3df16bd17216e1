"""Degenerate and limiting cases of the method on the GPU, checked against closed
forms (not against the oracle): an empty batch, a homogeneous medium (the
exact answer needs no iteration; the preconditioner is exact, so mixed control
takes one), and a laminate whose effective shear and uniaxial-strain moduli
are the Reuss means of the layers.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dbfft():
    from paper_1905_12725_gb300 import dbfft
    return dbfft


def _lame(E, nu):
    return E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))


def test_empty_batch_is_refused():
    dbfft = _dbfft()
    shape = (8, 8, 8)
    with pytest.raises(dbfft.DbfftError) as ei:
        dbfft.Solver(shape, np.zeros(shape, np.uint16), dbfft.iso_phases([1.0], [0.3]), np.zeros((0, 3, 3)))
    assert dbfft.STATUS[ei.value.status] == "DBFFT_E_ARG"


@pytest.mark.parametrize("precision", [0, 1])
def test_homogeneous_medium_is_exact_without_iterations(precision):
    dbfft = _dbfft()
    shape = (16, 8, 32)
    E, nu = 3.0, 0.27
    eps = np.array([[1e-3, 2e-4, -1e-4], [2e-4, -5e-4, 3e-4], [-1e-4, 3e-4, 2e-4]])
    s = dbfft.Solver(shape, np.zeros(shape, np.uint16), dbfft.iso_phases([E], [nu]), eps[None], tol=1e-12,
                     precision=precision)
    rep = s.solve_increment(0)
    assert rep["cg_iters"] == 0
    lam, mu = _lame(E, nu)
    ref = lam * np.trace(eps) * np.eye(3) + 2 * mu * eps
    assert np.abs(s.homogenized_stress()[0] - ref).max() <= 1e-14 * np.abs(ref).max()
    u, _ = s.get_solution()
    assert float(u.abs().max()) == 0.0
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_homogeneous_uniaxial_stress_gives_youngs_modulus(precision):
    """eps_xx prescribed, every other macro stress zero: sigma_xx = E eps_xx exactly,
    lateral strains -nu eps_xx; the macro-block preconditioner is exact here."""
    dbfft = _dbfft()
    shape = (8, 16, 16)
    E, nu = 2.5, 0.31
    mask = np.ones((3, 3), bool)
    mask[0, 0] = False
    tgt = np.zeros((3, 3))
    tgt[0, 0] = 1e-3
    s = dbfft.Solver(shape, np.zeros(shape, np.uint16), dbfft.iso_phases([E], [nu]), tgt[None],
                     stress_mask=mask.reshape(-1), tol=1e-12 if precision == 0 else 1e-8, precision=precision)
    rep = s.solve_increment(0)
    sig = s.homogenized_stress()[0]
    assert abs(sig[0, 0] - E * 1e-3) <= 1e-10 * E * 1e-3
    assert np.abs(sig - np.diag([sig[0, 0], 0, 0])).max() <= 1e-10 * E * 1e-3
    _, e = s.get_solution()
    assert abs(e[0][1] + nu * 1e-3) <= 1e-10 and abs(e[0][2] + nu * 1e-3) <= 1e-10  # Mandel e22, e33
    assert rep["cg_iters"] <= 2
    s.close()


def test_laminate_reuss_means_on_the_gpu():
    """Layers normal to x1 with even widths: shear eps_12 gives the Reuss mean of mu,
    uniaxial strain eps_11 the Reuss mean of lambda + 2 mu (FP64 solve to 1e-12)."""
    dbfft = _dbfft()
    shape = (32, 8, 8)
    phase = np.zeros(shape, np.uint16)
    phase[12:] = 1  # widths 12 and 20
    f = np.array([12, 20]) / 32
    E, nu = np.array([1.0, 40.0]), np.array([0.3, 0.2])
    lam, mu = _lame(E, nu)
    tgt = np.zeros((2, 3, 3))
    tgt[0, 0, 1] = tgt[0, 1, 0] = 1e-3
    tgt[1, 0, 0] = 1e-3
    s = dbfft.Solver(shape, phase, dbfft.iso_phases(E, nu), tgt, batch=2, tol=1e-12)
    s.solve_increment(0)
    sig = s.homogenized_stress()
    mu_R = 1.0 / np.sum(f / mu)
    m_R = 1.0 / np.sum(f / (lam + 2 * mu))
    assert abs(sig[0, 0, 1] - 2 * mu_R * 1e-3) <= 1e-10 * abs(2 * mu_R * 1e-3)
    assert abs(sig[1, 0, 0] - m_R * 1e-3) <= 1e-10 * abs(m_R * 1e-3)
    s.close()
