"""GPU adjoint: dJ/dE(x) of J = g : <sigma> against the oracle's FP64 adjoint,
the Euler identity, central finite differences of GPU solves, and the
torch.autograd.Function built on it.
"""
import numpy as np
import pytest

import oracle.dbfft_oracle as o
from paper_1905_12725_gb300 import synth
from tests.helpers import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dbfft():
    from paper_1905_12725_gb300 import dbfft
    return dbfft


def _case(shape, B, seed=31):
    g = np.random.default_rng(seed)
    E = np.where(g.random((B,) + shape) < 0.3, 25.0, 1.0)
    return E


def test_adjoint_matches_oracle_and_euler_identity():
    shape = (16, 16, 8)
    B = 3
    E = _case(shape, B)
    nu = 0.3
    eps = np.zeros((B, 3, 3))
    eps[:, 0, 0] = 1e-3
    eps[1, 1, 2] = eps[1, 2, 1] = 4e-4
    gJ = np.zeros((B, 3, 3))
    gJ[:, 0, 0] = 1.0
    gJ[2] = [[0.2, 0.1, 0], [0.1, -0.5, 0.3], [0, 0.3, 0.7]]
    dbfft = _dbfft()
    s = dbfft.Solver(shape, np.zeros((B,) + shape, np.uint16), dbfft.iso_phases([1.0], [nu]), eps, E_scale=E,
                     tol=1e-13)
    dJ, rep = s.adjoint(gJ.reshape(B, 9))
    dJ = dJ.cpu().numpy()
    sig = s.homogenized_stress()
    prob = o.Problem(shape)
    for b in range(B):
        ref, J, _ = o.adjoint_dJ_dE(prob, E[b], np.full(shape, nu), eps[b], gJ[b], tol=1e-13)
        assert rel_err(dJ[b], ref) < 1e-10
        Jg = float(np.sum(gJ[b] * sig[b]))
        assert abs(np.sum(E[b] * dJ[b]) - Jg) < 1e-10 * abs(Jg)


def test_adjoint_finite_differences_of_gpu_solves():
    shape = (16, 8, 16)
    E = _case(shape, 1, seed=5)
    nu = 0.3
    eps = np.zeros((1, 3, 3))
    eps[0, 0, 0] = 1e-3
    dbfft = _dbfft()
    ph = np.zeros((1,) + shape, np.uint16)
    s = dbfft.Solver(shape, ph, dbfft.iso_phases([1.0], [nu]), eps, E_scale=E, tol=1e-13)
    gJ = np.zeros((1, 9))
    gJ[0, 0] = 1.0
    dJ, _ = s.adjoint(gJ)
    dJ = dJ.cpu().numpy()[0]
    rng = synth.Xoshiro256ss(77)
    for v in synth.random_voxels(E[0].size, 6, rng):
        idx = np.unravel_index(v, shape)
        d = 1e-3 * E[0][idx]
        Js = []
        for sgn in (+1, -1):
            Ep = E.copy()
            Ep[(0,) + idx] += sgn * d
            sp = dbfft.Solver(shape, ph, dbfft.iso_phases([1.0], [nu]), eps, E_scale=Ep, tol=1e-13)
            sp.solve_increment(0)
            Js.append(sp.homogenized_stress()[0, 0, 0])
            sp.close()
        fd = (Js[0] - Js[1]) / (2 * d)
        assert abs(fd - dJ[idx]) < 1e-4 * abs(dJ[idx])


def test_autograd_function_gradient():
    shape = (8, 16, 16)
    B = 2
    E = torch.from_numpy(_case(shape, B, seed=9)).cuda().requires_grad_(True)
    eps = torch.zeros(B, 3, 3, dtype=torch.float64)
    eps[:, 0, 0] = 1e-3
    fn = _dbfft().homogenized_stress_fn()
    sig = fn.apply(E, 0.3, eps)
    J = sig[:, 0, 0].sum()
    J.backward()
    prob = o.Problem(shape)
    gJ = np.zeros((3, 3))
    gJ[0, 0] = 1.0
    for b in range(B):
        ref, _, _ = o.adjoint_dJ_dE(prob, E.detach().cpu().numpy()[b], np.full(shape, 0.3),
                                    eps[b].numpy(), gJ, tol=1e-12)
        assert rel_err(E.grad.cpu().numpy()[b], ref) < 1e-8


def test_device_resident_maps_give_the_host_results():
    """Phase map and stiffness scale passed as device arrays (dbfft_materials.device_arrays):
    counted, checked and averaged on the GPU; the solution equals the host-map one."""
    shape = (16, 8, 16)
    B = 2
    E = _case(shape, B, seed=13)
    eps = np.zeros((B, 3, 3))
    eps[:, 0, 0] = 1e-3
    eps[1, 0, 1] = eps[1, 1, 0] = 5e-4
    dbfft = _dbfft()
    ph = np.zeros((B,) + shape, np.uint16)
    sh = dbfft.Solver(shape, ph, dbfft.iso_phases([1.0], [0.3]), eps, E_scale=E, tol=1e-13)
    sh.solve_increment(0)
    sd = dbfft.Solver(shape, torch.from_numpy(ph.astype(np.int16)).cuda(), dbfft.iso_phases([1.0], [0.3]), eps,
                      E_scale=torch.from_numpy(E).cuda(), tol=1e-13)
    sd.solve_increment(0)
    assert rel_err(sd.homogenized_stress(), sh.homogenized_stress()) < 1e-11
    sh.close()
    sd.close()
    # the checks run on the device too: an id beyond the phases and a non-finite scale are refused
    bad = torch.zeros((1,) + shape, dtype=torch.int16, device="cuda")
    bad[0, 3, 2, 1] = 1
    with pytest.raises(dbfft.DbfftError):
        dbfft.Solver(shape, bad, dbfft.iso_phases([1.0], [0.3]), eps[:1])
    Eb = torch.ones((1,) + shape, dtype=torch.float64, device="cuda")
    Eb[0, 1, 1, 1] = float("nan")
    with pytest.raises(dbfft.DbfftError):
        dbfft.Solver(shape, torch.zeros((1,) + shape, dtype=torch.int16, device="cuda"), dbfft.iso_phases([1.0], [0.3]),
                     eps[:1], E_scale=Eb)


def test_adjoint_reuses_the_forward_solve():
    """After a converged solve of increment 0 the adjoint runs the adjoint solve only:
    the same dJ/dE with fewer CG iterations than a call that must solve forward first."""
    shape = (16, 16, 8)
    E = _case(shape, 1, seed=17)
    eps = np.zeros((1, 3, 3))
    eps[0, 0, 0] = 1e-3
    gJ = np.zeros((1, 9))
    gJ[0, 0] = 1.0
    dbfft = _dbfft()
    ph = np.zeros((1,) + shape, np.uint16)
    fresh = dbfft.Solver(shape, ph, dbfft.iso_phases([1.0], [0.3]), eps, E_scale=E, tol=1e-13)
    d_fresh, rep_fresh = fresh.adjoint(gJ)
    fresh.close()
    s = dbfft.Solver(shape, ph, dbfft.iso_phases([1.0], [0.3]), eps, E_scale=E, tol=1e-13)
    rep_fwd = s.solve_increment(0)
    d_reuse, rep_reuse = s.adjoint(gJ)
    assert rep_reuse["cg_iters"] + rep_fwd["cg_iters"] == rep_fresh["cg_iters"]
    assert rel_err(d_reuse.cpu().numpy(), d_fresh.cpu().numpy()) < 1e-10
    d_again, rep_again = s.adjoint(gJ)  # the state after an adjoint is the forward solve again
    assert rep_again["cg_iters"] == rep_reuse["cg_iters"]
    assert rel_err(s.homogenized_stress(), fresh_sig(shape, ph, E, eps)) < 1e-10
    s.close()


def fresh_sig(shape, ph, E, eps):
    dbfft = _dbfft()
    t = dbfft.Solver(shape, ph, dbfft.iso_phases([1.0], [0.3]), eps, E_scale=E, tol=1e-13)
    t.solve_increment(0)
    sig = t.homogenized_stress()
    t.close()
    return sig


def test_autograd_backward_runs_one_adjoint_solve():
    """forward + backward of the autograd function: one forward and one adjoint solve
    (the backward's report counts the adjoint solve only), with E kept on the device."""
    shape = (8, 16, 16)
    E = torch.from_numpy(_case(shape, 1, seed=21)).cuda().requires_grad_(True)
    eps = torch.zeros(1, 3, 3, dtype=torch.float64)
    eps[0, 0, 0] = 1e-3
    fn = _dbfft().homogenized_stress_fn()
    sig = fn.apply(E, 0.3, eps)
    sig[:, 0, 0].sum().backward()
    rep = fn.last_adjoint_report
    dbfft = _dbfft()
    s = dbfft.Solver(shape, np.zeros((1,) + shape, np.uint16), dbfft.iso_phases([1.0], [0.3]), eps.numpy(),
                     E_scale=E.detach().cpu().numpy(), tol=1e-10)
    _, rep_both = s.adjoint(np.eye(3).reshape(1, 9) * np.array([1, 0, 0, 0, 0, 0, 0, 0, 0]))
    s.close()
    assert 0 < rep["cg_iters"] < rep_both["cg_iters"]


# ------------------------------------------------------------------ effective-stiffness sensitivity
def test_stiffness_sensitivity_matches_oracle_and_euler_identity():
    """dJ/dE(x) for J = G : C_eff against the oracle (six forward and six adjoint solves
    there; the library reuses the six forward fields), two material maps, 1e-10 in FP64."""
    shape = (16, 8, 16)
    Bm = 2
    g = np.random.default_rng(19)
    E = np.where(g.random((Bm,) + shape) < 0.3, 20.0, 1.0) * (0.8 + 0.4 * g.random((Bm,) + shape))
    G = g.standard_normal((Bm, 6, 6))
    dbfft = _dbfft()
    s = dbfft.Solver(shape, np.zeros((Bm,) + shape, np.uint16), dbfft.iso_phases([1.0], [0.3]),
                     np.zeros((6 * Bm, 3, 3)), batch=6 * Bm, E_scale=E, tol=1e-13)
    dJ, C, rep = s.tangent_sensitivity(G)
    dJ = dJ.cpu().numpy()
    n_first = rep["cg_iters"]
    dJ2, _, rep2 = s.tangent_sensitivity(G)  # reuses the six solves
    assert rep2["cg_iters"] == 0 < n_first
    assert np.array_equal(dJ2.cpu().numpy(), dJ)
    s.close()
    for m in range(Bm):
        ref, J, Cref = o.effective_stiffness_sensitivity(shape, E[m], np.full(shape, 0.3), G[m], tol=1e-13)
        assert rel_err(C[m], Cref) < 1e-10
        assert rel_err(dJ[m], ref) < 1e-10
        Jg = float(np.sum(G[m] * C[m]))
        assert abs(np.sum(E[m] * dJ[m]) - Jg) < 1e-10 * np.abs(G[m] * C[m]).sum()


def test_stiffness_sensitivity_mixed_precision_and_autograd():
    """The FP32-inner solve gives the FP64 sensitivity to 1e-6; the autograd function
    returns it as the gradient of sum(G * C_eff)."""
    shape = (8, 16, 16)
    g = np.random.default_rng(23)
    E = np.where(g.random((1,) + shape) < 0.25, 50.0, 1.0)
    G = np.zeros((1, 6, 6))
    G[0, 0, 0] = 1.0
    G[0, 3, 5] = G[0, 5, 3] = 0.5
    dbfft = _dbfft()
    ref = None
    for prec, bar in ((dbfft.DBFFT_FP64, None), (dbfft.DBFFT_MIXED, 1e-6)):
        s = dbfft.Solver(shape, np.zeros((1,) + shape, np.uint16), dbfft.iso_phases([1.0], [0.3]),
                         np.zeros((6, 3, 3)), batch=6, E_scale=E, tol=1e-12 if bar is None else 1e-9, precision=prec)
        dJ, _, _ = s.tangent_sensitivity(G)
        s.close()
        if bar is None:
            ref = dJ.cpu().numpy()
        else:
            assert rel_err(dJ.cpu().numpy(), ref) < bar
    Et = torch.from_numpy(E).cuda().requires_grad_(True)
    fn = dbfft.effective_stiffness_fn()
    C = fn.apply(Et, 0.3, dbfft.DBFFT_FP64, 1e-12)
    (C * torch.from_numpy(G).cuda()).sum().backward()
    assert fn.last_report["cg_iters"] == 0  # the backward reuses the forward's six solves
    assert rel_err(Et.grad.cpu().numpy(), ref) < 1e-9
