"""GPU parity of the nonlinear paths: Neo-Hookean and St. Venant-Kirchhoff finite
strain with strain or mixed control (Sec. 2.4, Sec. 3) and small-strain crystal
plasticity, against the FP64 oracle.

Both sides run Newton to tight tolerances so that the difference is bounded by
the solve error: bar 1e-10 relative on the homogenized stress per increment
for FP64, 1e-6 for the FP32-inner / FP64-outer form.
"""
import math

import numpy as np
import pytest

import oracle.dbfft_oracle as o
from paper_1905_12725_gb300 import synth
from tests.helpers import mask9, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dbfft():
    from paper_1905_12725_gb300 import dbfft
    return dbfft


# ------------------------------------------------------------------ Neo-Hooke
NH_MASK = np.zeros((3, 3), bool)
NH_MASK[0, 1] = NH_MASK[0, 2] = NH_MASK[1, 2] = NH_MASK[1, 1] = NH_MASK[2, 2] = True


def _nh_case(shape, seed=3):
    g = np.random.default_rng(seed)
    phase = (g.random(shape) < 0.3).astype(np.uint16)
    mu = np.array([1.0, 20.0])
    lam = 1.5 * mu
    return phase, mu, lam


def _nh_targets(F11, n):
    out = []
    for k in range(n):
        t = np.eye(3)
        t[0, 0] = 1.0 + (F11 - 1.0) * (k + 1) / n
        t[NH_MASK] = 0.0
        out.append(t)
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_neo_hooke_mixed_control_increments(precision):
    shape = (16, 8, 16)
    phase, mu, lam = _nh_case(shape)
    n_inc, F11 = 3, 1.12
    dbfft = _dbfft()
    tgt = _nh_targets(F11, n_inc)[-1]
    s = dbfft.Solver(shape, phase, dbfft.neo_hooke_phases(mu, lam), tgt[None], kinematics=dbfft.DBFFT_FINITE,
                     precision=precision, stress_mask=NH_MASK.reshape(-1), n_increments=n_inc,
                     newton_tol=1e-11 if precision == 0 else 1e-8, load_tol=1e-12 if precision == 0 else 1e-9,
                     eta_inner=1e-6 if precision == 0 else 1e-3, tol=1e-12)
    prob = o.Problem(shape, "finite", NH_MASK.reshape(-1))
    ref, _ = o.newton_increments(prob, o.neo_hooke_material(mu[phase], lam[phase]), _nh_targets(F11, n_inc),
                                 newton_tol=1e-12, load_tol=1e-13, eta=1e-8)
    for k in range(n_inc):
        rep = s.solve_increment(k)
        P = s.homogenized_stress()[0]
        assert rel_err(P, ref[k]["stress_bar"]) < (1e-10 if precision == 0 else 1e-6), (k, rep)
        assert rep["eps_eq"] <= (1e-11 if precision == 0 else 1e-8)
    if precision == 0:
        u, e = s.get_solution()
        assert rel_err(u.cpu().numpy()[0], ref[-1]["x"][0]) < 1e-9


def test_neo_hooke_tangent_operator_matches_oracle():
    """K(F) applied to random spectra after a residual evaluation at a random F field (FP64)."""
    shape = (8, 16, 8)
    phase, mu, lam = _nh_case(shape, 5)
    dbfft = _dbfft()
    Fbar = np.array([[1.05, 0.02, 0.0], [0.01, 0.97, 0.03], [0.0, -0.02, 1.01]])
    s = dbfft.Solver(shape, phase, dbfft.neo_hooke_phases(mu, lam), Fbar[None], kinematics=dbfft.DBFFT_FINITE)
    prob = o.Problem(shape, "finite")
    x = synth.random_spectrum(shape, 3, 21) * 2e-4
    r, _ = s.apply(torch.from_numpy(x).cuda(), residual=True)  # constitutive update at F(x)
    F = prob.field_from(x[0], np.zeros(0)) + Fbar[:, :, None, None, None]
    Pf, Kf = o.neo_hooke(F, mu[phase], lam[phase])
    qu, _ = prob.adjoint(Pf)
    assert rel_err(r.cpu().numpy()[0], -qu) < 1e-12
    u = synth.random_spectrum(shape, 3, 22)
    out, _ = s.apply(torch.from_numpy(u).cuda())
    ref, _ = prob.apply_K(o.FullTangent(Kf), u[0], np.zeros(0))
    assert rel_err(out.cpu().numpy()[0], ref) < 1e-12


# ------------------------------------------------------------------ St. Venant-Kirchhoff
@pytest.mark.parametrize("fp32", [False, True])
def test_svk_tangent_operator_matches_oracle(fp32):
    """SVK: P(F) by a residual evaluation at a random F field, then K(F) applied to
    random spectra (FP64 tangent, or the FP32 tangent of the mixed solve)."""
    shape = (8, 16, 8)
    c = synth.porous_svk(8, 1, 0.1, seed=11)
    phase = np.resize(c["phase"], shape).astype(np.uint16)
    mu, lam = c["mu"], c["lam"]
    dbfft = _dbfft()
    Fbar = np.array([[1.3, 0.05, 0.0], [0.02, 0.95, 0.04], [0.0, -0.03, 1.02]])
    s = dbfft.Solver(shape, phase, dbfft.svk_phases(mu, lam), Fbar[None], kinematics=dbfft.DBFFT_FINITE,
                     precision=dbfft.DBFFT_MIXED if fp32 else dbfft.DBFFT_FP64)
    prob = o.Problem(shape, "finite")
    x = synth.random_spectrum(shape, 3, 23) * 2e-3
    r, _ = s.apply(torch.from_numpy(x).cuda(), residual=True)  # constitutive update at F(x)
    F = prob.field_from(x[0], np.zeros(0)) + Fbar[:, :, None, None, None]
    Pf, Kf = o.svk(F, mu[phase], lam[phase])
    qu, _ = prob.adjoint(Pf)
    assert rel_err(r.cpu().numpy()[0], -qu) < 1e-12
    u = synth.random_spectrum(shape, 3, 24)
    out, _ = s.apply(torch.from_numpy(u).cuda(), fp32=fp32)
    ref, _ = prob.apply_K(o.FullTangent(Kf), u[0], np.zeros(0))
    assert rel_err(out.cpu().numpy()[0], ref) < (2e-5 if fp32 else 1e-12)
    s.close()


@pytest.mark.parametrize("precision,control", [(0, "strain"), (1, "strain"), (0, "mixed"), (1, "mixed")])
def test_svk_porous_increments(precision, control):
    """Porous SVK matrix (compliant pores, 1/100 stiffness) stretched along x: every
    component of F prescribed, or the lateral and shear stresses held at zero."""
    c = synth.porous_svk(16, 2, 0.15, seed=5)
    phase, mu, lam = c["phase"], c["mu"], c["lam"]
    shape = phase.shape
    n_inc, F11 = 3, 1.3
    mask = NH_MASK if control == "mixed" else np.zeros((3, 3), bool)
    targets = []
    for k in range(n_inc):
        t = np.eye(3)
        t[0, 0] = 1.0 + (F11 - 1.0) * (k + 1) / n_inc
        t[mask] = 0.0
        targets.append(t)
    dbfft = _dbfft()
    s = dbfft.Solver(shape, phase, dbfft.svk_phases(mu, lam), targets[-1][None], kinematics=dbfft.DBFFT_FINITE,
                     precision=precision, stress_mask=mask.reshape(-1) if control == "mixed" else None,
                     n_increments=n_inc, newton_tol=1e-11 if precision == 0 else 1e-8,
                     load_tol=1e-12 if precision == 0 else 1e-9, eta_inner=1e-6 if precision == 0 else 1e-3,
                     tol=1e-12, max_newton=40)
    prob = o.Problem(shape, "finite", mask.reshape(-1) if control == "mixed" else None)
    ref, _ = o.newton_increments(prob, o.svk_material(mu[phase], lam[phase]), targets,
                                 newton_tol=1e-12, load_tol=1e-13, eta=1e-8)
    for k in range(n_inc):
        rep = s.solve_increment(k)
        P = s.homogenized_stress()[0]
        assert rel_err(P, ref[k]["stress_bar"]) < (1e-10 if precision == 0 else 1e-6), (k, rep)
        assert rep["eps_eq"] <= (1e-11 if precision == 0 else 1e-8)
    if precision == 0:
        u, _ = s.get_solution()
        assert rel_err(u.cpu().numpy()[0], ref[-1]["x"][0]) < 1e-9
    s.close()


def test_precond_refresh_policies_give_the_same_solution():
    """The reference stiffness of the preconditioner (initial, per increment, per Newton
    iterate) changes the CG iteration count, not the converged increments."""
    c = synth.porous_svk(16, 2, 0.15, seed=5)
    phase, mu, lam = c["phase"], c["mu"], c["lam"]
    n_inc, F11 = 3, 1.5
    targets = []
    for k in range(n_inc):
        t = np.eye(3)
        t[0, 0] = 1.0 + (F11 - 1.0) * (k + 1) / n_inc
        targets.append(t)
    prob = o.Problem(phase.shape, "finite")
    ref, _ = o.newton_increments(prob, o.svk_material(mu[phase], lam[phase]), targets,
                                 newton_tol=1e-12, load_tol=1e-13, eta=1e-8)
    dbfft = _dbfft()
    its = {}
    for policy in (dbfft.DBFFT_PRECOND_PER_INCREMENT, dbfft.DBFFT_PRECOND_INITIAL, dbfft.DBFFT_PRECOND_PER_NEWTON):
        s = dbfft.Solver(phase.shape, phase, dbfft.svk_phases(mu, lam), targets[-1][None],
                         kinematics=dbfft.DBFFT_FINITE, n_increments=n_inc, newton_tol=1e-11, eta_inner=1e-6,
                         tol=1e-12, max_newton=40)
        s.set_precond_refresh(policy)
        its[policy] = []
        for k in range(n_inc):
            rep = s.solve_increment(k)
            its[policy].append(rep["cg_iters"])
            assert rel_err(s.homogenized_stress()[0], ref[k]["stress_bar"]) < 1e-10, (policy, k)
        s.close()
    assert its[dbfft.DBFFT_PRECOND_INITIAL] != its[dbfft.DBFFT_PRECOND_PER_INCREMENT], its


# ------------------------------------------------------------------ crystal plasticity
CP_MASK = np.ones((3, 3), bool)
CP_MASK[0, 0] = False


def _cp_targets(n, dt, rate=1e-3):
    out = []
    for k in range(n):
        t = np.zeros((3, 3))
        t[0, 0] = rate * dt * (k + 1)
        out.append(t)
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_crystal_plasticity_polycrystal_increments(precision):
    shape = (8, 8, 16)
    rng = synth.Xoshiro256ss(4242)
    grains, _ = synth.periodic_voronoi(8, 5, rng)
    grains = np.concatenate([grains, grains], axis=2)  # 8 x 8 x 16, periodic copy along x3
    quats = synth.uniform_quaternions(5, rng)
    n_inc, dt = 6, 0.5
    dbfft = _dbfft()
    tgt = _cp_targets(n_inc, dt)[-1]
    s = dbfft.Solver(shape, grains, dbfft.cp_phases(quats), tgt[None], stress_mask=CP_MASK.reshape(-1),
                     precision=precision, n_increments=n_inc, total_time=n_inc * dt,
                     newton_tol=1e-11 if precision == 0 else 1e-8, load_tol=1e-12 if precision == 0 else 1e-9,
                     eta_inner=1e-6 if precision == 0 else 1e-3)
    cp = o.CrystalPlasticity(quats)
    prob = o.Problem(shape, "small", CP_MASK.reshape(-1))
    ref, _ = o.newton_increments(prob, o.cp_material(cp, grains, dt), _cp_targets(n_inc, dt),
                                 newton_tol=1e-12, load_tol=1e-13, eta=1e-8)
    for k in range(n_inc):
        rep = s.solve_increment(k)
        sig = s.homogenized_stress()[0]
        assert rel_err(sig, ref[k]["stress_bar"]) < (1e-10 if precision == 0 else 1e-6), (k, rep)


def test_crystal_plasticity_single_crystal_steady_state():
    """Cube-oriented crystal in [100] tension at 1e-3/s: u = 0 and sigma_xx -> sigma_ss."""
    shape = (8, 8, 8)
    dbfft = _dbfft()
    n_inc, dt = 40, 0.5
    tgt = _cp_targets(n_inc, dt)[-1]
    s = dbfft.Solver(shape, np.zeros(shape, np.uint16), dbfft.cp_phases([[1.0, 0, 0, 0]]), tgt[None],
                     stress_mask=CP_MASK.reshape(-1), n_increments=n_inc, total_time=n_inc * dt,
                     newton_tol=1e-10, load_tol=1e-11)
    for k in range(n_inc):
        s.solve_increment(k)
    sig = s.homogenized_stress()[0]
    sig_ss = math.sqrt(6) * 50.0 * (math.sqrt(6) * 1e-3 / (8 * 1e-3)) ** 0.05
    assert abs(sig[0, 0] - sig_ss) < 1e-9 * sig_ss
    u, _ = s.get_solution()
    assert float(u.abs().max()) < 1e-12
