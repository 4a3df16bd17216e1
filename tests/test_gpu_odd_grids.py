"""GPU parity on odd grids (Sec. 2.1's frequency set; the paper's experiments use
63^3): mixed-radix (3, 5, 7) transforms along axes 1 and 2 and the paired
complex transform of pass 3 along an odd axis 3, against the FP64 oracle.

Bars as for the even grids: 1e-12 (FP64 operator) and 2e-5 (FP32 operator);
solves to 1e-12 agree with the oracle's to 1e-10 on sigma_bar (FP64) and 1e-6
(mixed).
"""
import numpy as np
import pytest

import oracle.dbfft_oracle as o
from paper_1905_12725_gb300 import synth
from tests.helpers import e9_to_oracle, e_oracle_to9, iso_tangent, mask9, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPES = [(15, 9, 21), (21, 16, 9), (16, 15, 32), (9, 9, 9), (27, 25, 45),
          (243, 9, 8), (8, 245, 9), (9, 8, 243)]  # the largest compiled odd lengths on each axis


def _dbfft():
    from paper_1905_12725_gb300 import dbfft
    return dbfft


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("fp32", [False, True])
def test_odd_grid_operator_matches_oracle(shape, fp32):
    B = 2
    phase = (np.random.default_rng(5).random(shape) < 0.35).astype(np.uint16)
    E, nu = [1.0, 30.0], [0.3, 0.2]
    dbfft = _dbfft()
    s = dbfft.Solver(shape, phase, dbfft.iso_phases(E, nu), np.zeros((B, 3, 3)), batch=B,
                     precision=dbfft.DBFFT_MIXED if fp32 else dbfft.DBFFT_FP64)
    u = synth.random_spectrum(shape, 3, 13, batch=B)
    out, _ = s.apply(torch.from_numpy(u).cuda(), fp32=fp32)
    out = out.cpu().numpy()
    s.close()
    prob = o.Problem(shape)
    T = iso_tangent(phase, E, nu)
    for b in range(B):
        ref, _ = prob.apply_K(T, u[b], np.zeros(0))
        assert rel_err(out[b], ref) < (2e-5 if fp32 else 1e-12), b


def test_odd_grid_operator_with_macro_unknowns():
    shape = (15, 21, 9)
    mask = mask9([(0, 0), (1, 2), (0, 1)])
    phase = (np.random.default_rng(6).random(shape) < 0.35).astype(np.uint16)
    E, nu = [2.0, 0.5], [0.3, 0.35]
    dbfft = _dbfft()
    s = dbfft.Solver(shape, phase, dbfft.iso_phases(E, nu), np.zeros((1, 3, 3)), stress_mask=mask)
    prob = o.Problem(shape, "small", mask)
    u = synth.random_spectrum(shape, 3, 17)
    e = np.random.default_rng(3).standard_normal(prob.ne)
    out, eo = s.apply(torch.from_numpy(u).cuda(), torch.from_numpy(e_oracle_to9(prob, e)[None]).cuda())
    qu, qe = prob.apply_K(iso_tangent(phase, E, nu), u[0], e)
    s.close()
    assert rel_err(out.cpu().numpy()[0], qu) < 1e-12
    assert rel_err(e9_to_oracle(prob, eo.cpu().numpy()[0]), qe) < 1e-12


def test_odd_axes_1_2_with_finite_strain():
    """Odd n1 and n2 with an even n3: the mixed-radix strided transforms carry the
    nine components of the finite-strain gradient (Neo-Hookean tangent)."""
    shape = (9, 15, 16)
    phase = (np.random.default_rng(7).random(shape) < 0.3).astype(np.uint16)
    mu = np.array([1.0, 20.0])
    lam = 1.5 * mu
    Fbar = np.array([[1.05, 0.02, 0.0], [0.01, 0.97, 0.03], [0.0, -0.02, 1.01]])
    dbfft = _dbfft()
    s = dbfft.Solver(shape, phase, dbfft.neo_hooke_phases(mu, lam), Fbar[None], kinematics=dbfft.DBFFT_FINITE)
    prob = o.Problem(shape, "finite")
    x = synth.random_spectrum(shape, 3, 21) * 2e-4
    r, _ = s.apply(torch.from_numpy(x).cuda(), residual=True)
    F = prob.field_from(x[0], np.zeros(0)) + Fbar[:, :, None, None, None]
    Pf, Kf = o.neo_hooke(F, mu[phase], lam[phase])
    qu, _ = prob.adjoint(Pf)
    assert rel_err(r.cpu().numpy()[0], -qu) < 1e-12
    u = synth.random_spectrum(shape, 3, 22)
    out, _ = s.apply(torch.from_numpy(u).cuda())
    ref, _ = prob.apply_K(o.FullTangent(Kf), u[0], np.zeros(0))
    s.close()
    assert rel_err(out.cpu().numpy()[0], ref) < 1e-12


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("control", ["strain", "stress"])
def test_odd_grid_inclusion_solves(precision, control):
    """21^3 centred inclusion (vf 0.2, contrast 10): uniaxial strain, or uniaxial
    stress with every component stress-controlled (Sec. 3, first and second benchmarks)."""
    c = synth.inclusion(21, contrast=10.0)
    phase, E, nu = c["phase"], c["E"], c["nu"]
    shape = phase.shape
    if control == "strain":
        mask, target = None, np.diag([1e-3, 0.0, 0.0])
    else:
        mask, target = np.ones(9, bool), np.diag([70.0 * 1e-3, 0.0, 0.0])
    dbfft = _dbfft()
    s = dbfft.Solver(shape, phase, dbfft.iso_phases(E, nu), target[None], stress_mask=mask,
                     tol=1e-12 if precision == 0 else 1e-9, precision=precision, eta_inner=1e-3)
    rep = s.solve_increment(0)
    sig = s.homogenized_stress()[0]
    u, e = s.get_solution()
    s.close()
    prob = o.Problem(shape, "small", mask)
    ref = o.solve_linear(prob, iso_tangent(phase, E, nu), target, tol=1e-12)
    assert rel_err(sig, ref["sig_bar"]) < (1e-10 if precision == 0 else 1e-6), rep
    if precision == 0:
        assert rel_err(u.cpu().numpy()[0], ref["u"]) < 1e-9


def test_odd_63_cubed_operator_matches_oracle():
    """The paper's grid: one FP64 and one FP32 application at 63^3."""
    c = synth.inclusion(63, contrast=1e3)
    phase, E, nu = c["phase"], c["E"], c["nu"]
    shape = phase.shape
    u = synth.random_spectrum(shape, 3, 63)
    ref, _ = o.Problem(shape).apply_K(iso_tangent(phase, E, nu), u[0], np.zeros(0))
    dbfft = _dbfft()
    for fp32 in (False, True):
        s = dbfft.Solver(shape, phase, dbfft.iso_phases(E, nu), np.zeros((1, 3, 3)),
                         precision=dbfft.DBFFT_MIXED if fp32 else dbfft.DBFFT_FP64)
        out, _ = s.apply(torch.from_numpy(u).cuda(), fp32=fp32)
        s.close()
        assert rel_err(out.cpu().numpy()[0], ref) < (2e-5 if fp32 else 1e-12), fp32


def test_odd_n3_nonlinear_outside_the_compiled_lengths_is_refused():
    dbfft = _dbfft()
    shape = (8, 8, 25)
    with pytest.raises(dbfft.DbfftError) as ei:
        dbfft.Solver(shape, np.zeros(shape, np.uint16), dbfft.neo_hooke_phases([1.0], [1.5]), np.eye(3)[None],
                     kinematics=dbfft.DBFFT_FINITE)
    assert dbfft.STATUS[ei.value.status] == "DBFFT_E_UNSUPPORTED_GRID"


def test_odd_n3_neo_hooke_and_svk_tangent_operators():
    """Nine gradient components on an odd axis 3 (five component pairs, the last with a
    zero partner): constitutive update (residual) and tangent application, FP64 and FP32."""
    shape = (9, 8, 15)
    phase = (np.random.default_rng(8).random(shape) < 0.3).astype(np.uint16)
    mu = np.array([1.0, 20.0])
    lam = 1.5 * mu
    Fbar = np.array([[1.05, 0.02, 0.0], [0.01, 0.97, 0.03], [0.0, -0.02, 1.01]])
    dbfft = _dbfft()
    prob = o.Problem(shape, "finite")
    for law, phases_fn, oracle_fn in (("nh", dbfft.neo_hooke_phases, o.neo_hooke), ("svk", dbfft.svk_phases, o.svk)):
        for fp32 in (False, True):
            s = dbfft.Solver(shape, phase, phases_fn(mu, lam), Fbar[None], kinematics=dbfft.DBFFT_FINITE,
                             precision=dbfft.DBFFT_MIXED if fp32 else dbfft.DBFFT_FP64)
            x = synth.random_spectrum(shape, 3, 31) * 2e-4
            r, _ = s.apply(torch.from_numpy(x).cuda(), residual=True)
            F = prob.field_from(x[0], np.zeros(0)) + Fbar[:, :, None, None, None]
            Pf, Kf = oracle_fn(F, mu[phase], lam[phase])
            qu, _ = prob.adjoint(Pf)
            assert rel_err(r.cpu().numpy()[0], -qu) < 1e-12, (law, fp32)
            u = synth.random_spectrum(shape, 3, 32)
            out, _ = s.apply(torch.from_numpy(u).cuda(), fp32=fp32)
            ref, _ = prob.apply_K(o.FullTangent(Kf), u[0], np.zeros(0))
            s.close()
            assert rel_err(out.cpu().numpy()[0], ref) < (2e-5 if fp32 else 1e-12), (law, fp32)


@pytest.mark.parametrize("precision", [0, 1])
def test_odd_n3_porous_svk_increments(precision):
    """The porous St. Venant-Kirchhoff stretch on an odd 15^3 grid, strain control."""
    c = synth.porous_svk(15, 2, 0.15, seed=5)
    phase, mu, lam = c["phase"], c["mu"], c["lam"]
    n_inc, F11 = 2, 1.2
    targets = []
    for k in range(n_inc):
        t = np.eye(3)
        t[0, 0] = 1.0 + (F11 - 1.0) * (k + 1) / n_inc
        targets.append(t)
    dbfft = _dbfft()
    s = dbfft.Solver(phase.shape, phase, dbfft.svk_phases(mu, lam), targets[-1][None], kinematics=dbfft.DBFFT_FINITE,
                     precision=precision, n_increments=n_inc, newton_tol=1e-11 if precision == 0 else 1e-8,
                     eta_inner=1e-6 if precision == 0 else 1e-3, tol=1e-12, max_newton=40)
    prob = o.Problem(phase.shape, "finite")
    ref, _ = o.newton_increments(prob, o.svk_material(mu[phase], lam[phase]), targets, newton_tol=1e-12,
                                 load_tol=1e-13, eta=1e-8)
    for k in range(n_inc):
        rep = s.solve_increment(k)
        assert rel_err(s.homogenized_stress()[0], ref[k]["stress_bar"]) < (1e-10 if precision == 0 else 1e-6), (k, rep)
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_odd_n3_crystal_plasticity_increments(precision):
    """Polycrystal on an 8 x 8 x 9 grid (odd axis 3): CP update and tangent on paired lines."""
    shape = (8, 8, 9)
    rng = synth.Xoshiro256ss(777)
    g8, _ = synth.periodic_voronoi(8, 4, rng)
    grains = np.concatenate([g8, g8[:, :, :1]], axis=2).astype(np.uint16)
    quats = synth.uniform_quaternions(4, rng)
    mask = np.ones((3, 3), bool)
    mask[0, 0] = False
    n_inc, dt = 3, 0.5
    targets = []
    for k in range(n_inc):
        t = np.zeros((3, 3))
        t[0, 0] = 1e-3 * dt * (k + 1)
        targets.append(t)
    dbfft = _dbfft()
    s = dbfft.Solver(shape, grains, dbfft.cp_phases(quats), targets[-1][None], stress_mask=mask.reshape(-1),
                     precision=precision, n_increments=n_inc, total_time=n_inc * dt,
                     newton_tol=1e-11 if precision == 0 else 1e-8, load_tol=1e-12 if precision == 0 else 1e-9,
                     eta_inner=1e-6 if precision == 0 else 1e-3)
    cp = o.CrystalPlasticity(quats)
    prob = o.Problem(shape, "small", mask.reshape(-1))
    ref, _ = o.newton_increments(prob, o.cp_material(cp, grains, dt), targets, newton_tol=1e-12, load_tol=1e-13,
                                 eta=1e-8)
    for k in range(n_inc):
        rep = s.solve_increment(k)
        assert rel_err(s.homogenized_stress()[0], ref[k]["stress_bar"]) < (1e-10 if precision == 0 else 1e-6), (k, rep)
    s.close()
