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
