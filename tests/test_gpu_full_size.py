"""Parity at the workloads' full sizes, in the launch shapes the benchmark uses.

The oracle cannot solve these sizes in seconds, but it can evaluate one
operator application or one residual. So each test checks what is fixed at
any size:
  * 256^3 operator: the whole output of one FP64 and one FP32 application
    against the oracle's K u (1e-12 / 2e-5);
  * 64^3 sphere composite, 6 right-hand sides: the oracle's own residual of
    the GPU solutions (FP64 and mixed), C_eff symmetric and inside the Voigt
    and Reuss bounds, mixed within 1e-6 of FP64;
  * 128^3 Neo-Hookean fibres: the oracle's equilibrium and loading residuals
    of the GPU state after two increments, FP64 and mixed P_bar within 1e-6;
  * 256^3 polycrystal: first increment, mixed sigma_bar within 1e-6 of FP64;
  * 32 x 64^3 adjoint: mixed dJ/dE within 1e-6 of FP64, Euler identity and
    sign of the FP64 sensitivities.
"""
import math

import numpy as np
import pytest

import oracle.dbfft_oracle as o
from paper_1905_12725_gb300 import synth
from tests.helpers import e9_to_oracle, iso_tangent, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dbfft():
    from paper_1905_12725_gb300 import dbfft
    return dbfft


def test_operator_256_cubed_matches_oracle(tmp_path):
    n = 256
    shape = (n, n, n)
    phase = (np.random.default_rng(7).random(shape) < 0.3).astype(np.uint16)
    E, nu = [1.0, 100.0], [0.3, 0.3]
    u = synth.random_spectrum(shape, 3, 2561)
    ref, _ = o.Problem(shape).apply_K(iso_tangent(phase, E, nu), u[0], np.zeros(0))
    dbfft = _dbfft()
    for fp32 in (False, True):
        s = dbfft.Solver(shape, phase, dbfft.iso_phases(E, nu), np.zeros((1, 3, 3)),
                         precision=dbfft.DBFFT_MIXED if fp32 else dbfft.DBFFT_FP64)
        s.autotune(str(tmp_path / "tune.txt"))
        out, _ = s.apply(torch.from_numpy(u).cuda(), fp32=fp32)
        out = out.cpu().numpy()[0]
        s.close()
        assert rel_err(out, ref) < (2e-5 if fp32 else 1e-12), fp32


def _voigt_reuss(phase, E, nu):
    """Volume averages of the Mandel stiffness and of the compliance."""
    f1 = float(phase.mean())
    Cs = [o.tensor4_to_mandel(o.iso_stiffness(*o.lame(E[p], nu[p]))) for p in (0, 1)]
    CV = (1 - f1) * Cs[0] + f1 * Cs[1]
    CR = np.linalg.inv((1 - f1) * np.linalg.inv(Cs[0]) + f1 * np.linalg.inv(Cs[1]))
    return CV, CR


def test_sphere_composite_64_cubed_six_rhs():
    c = synth.config2()
    phase, E, nu = c["phase"], c["E"], c["nu"]
    shape = phase.shape
    dbfft = _dbfft()
    res = {}
    for prec, tol in [(dbfft.DBFFT_FP64, 1e-10), (dbfft.DBFFT_MIXED, 1e-6)]:
        s = dbfft.Solver(shape, phase, dbfft.iso_phases(E, nu), np.zeros((6, 3, 3)), batch=6, tol=tol,
                         precision=prec, eta_inner=1e-3)
        Ceff, rep = s.homogenized_tangent()
        u, _ = s.get_solution()
        res[prec] = (Ceff[0], u.cpu().numpy(), tol)
        s.close()
    prob = o.Problem(shape)
    T = iso_tangent(phase, E, nu)
    basis = o.mandel_basis()
    for prec, (Ceff, u, tol) in res.items():
        for m in range(6):  # the oracle's residual of the GPU solution of right-hand side m
            b = o.linear_rhs(prob, T, basis[m])
            r, _, _ = o.residual(prob, T.apply, (u[m], np.zeros(0)), basis[m], np.zeros(0))
            rel = math.sqrt(prob.dot(r, r)) / math.sqrt(prob.dot(b, b))
            assert rel <= 1.5 * tol, (prec, m, rel)
        assert np.abs(Ceff - Ceff.T).max() <= 10 * tol * np.abs(Ceff).max()
    C64, Cmx = res[dbfft.DBFFT_FP64][0], res[dbfft.DBFFT_MIXED][0]
    assert rel_err(Cmx, C64) < 1e-6
    CV, CR = _voigt_reuss(phase, E, nu)
    Cs = 0.5 * (C64 + C64.T)
    assert np.linalg.eigvalsh(CV - Cs).min() >= -1e-9 * np.abs(CV).max()
    assert np.linalg.eigvalsh(Cs - CR).min() >= -1e-9 * np.abs(CV).max()


NH_MASK = np.zeros((3, 3), bool)
NH_MASK[0, 1] = NH_MASK[0, 2] = NH_MASK[1, 2] = NH_MASK[1, 1] = NH_MASK[2, 2] = True


def test_neo_hooke_fibres_128_cubed_first_increments():
    c = synth.config3()
    phase, mu, lam = c["phase"], c["mu"], c["lam"]
    shape = phase.shape
    n_inc, F11, run = 20, 1.2, 2
    tgt_end = np.eye(3)
    tgt_end[0, 0] = F11
    tgt_end[NH_MASK] = 0.0
    dbfft = _dbfft()
    prob = o.Problem(shape, "finite", NH_MASK.reshape(-1))
    Pbar = {}
    for prec in (dbfft.DBFFT_FP64, dbfft.DBFFT_MIXED):
        s = dbfft.Solver(shape, phase, dbfft.neo_hooke_phases(mu, lam), tgt_end[None], kinematics=dbfft.DBFFT_FINITE,
                         precision=prec, stress_mask=NH_MASK.reshape(-1), n_increments=n_inc, newton_tol=1e-8,
                         load_tol=1e-10, eta_inner=1e-4, max_newton=30, max_iter=5000)
        for k in range(run):
            s.solve_increment(k)
        Pbar[prec] = s.homogenized_stress()[0]
        u, e = s.get_solution()
        s.close()
        # the oracle's residual of the GPU state at the end of increment `run`
        t = np.eye(3)
        t[0, 0] = 1.0 + (F11 - 1.0) * run / n_inc
        t[NH_MASK] = 0.0
        fU, sig_f = o.split_load(prob, t)
        x = (u.cpu().numpy()[0], e9_to_oracle(prob, e[0]))
        r, _, P = o.residual(prob, lambda F: o.neo_hooke(F, mu[phase], lam[phase])[0], x, fU, sig_f)
        Pb = P.reshape(3, 3, -1).mean(axis=-1)
        assert rel_err(Pb, Pbar[prec]) < 1e-10
        assert o.equilibrium_residual(prob, r, Pb) <= 1.5e-8
        assert np.abs(r[1]).max() / (prob.N * np.linalg.norm(Pb)) <= 1.5e-10
    assert rel_err(Pbar[dbfft.DBFFT_MIXED], Pbar[dbfft.DBFFT_FP64]) < 1e-6


def test_polycrystal_256_cubed_first_increment():
    c = synth.config4()
    mask = np.ones((3, 3), bool)
    mask[0, 0] = False
    tgt = np.zeros((3, 3))
    tgt[0, 0] = 0.02
    dbfft = _dbfft()
    sig = {}
    for prec in (dbfft.DBFFT_FP64, dbfft.DBFFT_MIXED):
        s = dbfft.Solver(c["phase"].shape, c["phase"], dbfft.cp_phases(c["quat"]), tgt[None], precision=prec,
                         stress_mask=mask.reshape(-1), n_increments=40, total_time=20.0, newton_tol=1e-8,
                         load_tol=1e-10, eta_inner=1e-4, max_newton=40, max_iter=5000)
        rep = s.solve_increment(0)
        assert rep["eps_eq"] <= 1e-8 and rep["load_res"] <= 1e-10
        sig[prec] = s.homogenized_stress()[0]
        s.close()
    assert rel_err(sig[dbfft.DBFFT_MIXED], sig[dbfft.DBFFT_FP64]) < 1e-6
    # uniaxial: the stress-controlled components vanish
    s64 = sig[dbfft.DBFFT_FP64]
    assert np.abs(s64 - np.diag([s64[0, 0], 0, 0])).max() <= 1e-9 * abs(s64[0, 0])


def test_batched_adjoint_32_rves_of_64_cubed():
    c = synth.config5()
    n_rve = c["phase"].shape[0]
    shape = c["phase"].shape[1:]
    E = c["E"][np.arange(n_rve)[:, None, None, None], c["phase"]]
    eps = np.zeros((n_rve, 3, 3))
    eps[:, 0, 0] = 1e-3
    g = np.zeros((n_rve, 9))
    g[:, 0] = 1.0
    dbfft = _dbfft()
    out = {}
    for prec, tol in [(dbfft.DBFFT_FP64, 1e-10), (dbfft.DBFFT_MIXED, 1e-7)]:
        s = dbfft.Solver(shape, np.zeros_like(c["phase"]), dbfft.iso_phases([1.0], [0.3]), eps, E_scale=E,
                         precision=prec, tol=tol, eta_inner=1e-3)
        dJ, _ = s.adjoint(g)
        out[prec] = (dJ.cpu().numpy(), s.homogenized_stress()[:, 0, 0])
        s.close()
    dJ64, J64 = out[dbfft.DBFFT_FP64]
    dJmx, _ = out[dbfft.DBFFT_MIXED]
    assert rel_err(dJmx, dJ64) < 1e-6
    for b in range(n_rve):
        assert abs(np.sum(E[b] * dJ64[b]) - J64[b]) < 1e-9 * abs(J64[b])
        assert dJ64[b].min() >= -1e-12 * dJ64[b].max()
