"""GPU adjoint of the crystal-plasticity increments against the FP64 oracle.

A polycrystal (R14 power-law flow rule) is loaded in uniaxial mixed control
(eps_11 prescribed, the other macro stresses zero) through four plastic
increments (Sec. 2.4, Newton per increment). The library keeps each
increment's converged stress as its checkpoint and sweeps back over them
with one FP64 adjoint solve per increment; the oracle runs the same reverse
sweep in numpy (pinned there by central differences of whole Newton runs).
Bar: 1e-9 relative (max norm) on dJ/ds(x), both sides converged to 1e-12.
"""
import numpy as np
import pytest

import oracle.dbfft_oracle as o
from paper_1905_12725_gb300 import synth
from tests.helpers import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CP_MASK = np.ones((3, 3), bool)
CP_MASK[0, 0] = False


def _dbfft():
    from paper_1905_12725_gb300 import dbfft
    return dbfft


def _case():
    shape = (8, 8, 16)
    rng = synth.Xoshiro256ss(4242)
    grains, _ = synth.periodic_voronoi(8, 5, rng)
    grains = np.concatenate([grains, grains], axis=2)
    quats = synth.uniform_quaternions(5, rng)
    return shape, grains, quats


def _targets(n, per_inc):
    out = []
    for k in range(n):
        t = np.zeros((3, 3))
        t[0, 0] = per_inc * (k + 1)
        out.append(t)
    return out


def test_cp_adjoint_over_increments_matches_oracle():
    shape, grains, quats = _case()
    n_inc, dt = 4, 0.5
    targets = _targets(n_inc, 1e-3)
    g = np.array([[1.0, 0.1, 0.0], [0.1, 0.0, 0.0], [0.0, 0.0, 0.2]])
    dbfft = _dbfft()
    s = dbfft.Solver(shape, grains, dbfft.cp_phases(quats), targets[-1][None], stress_mask=CP_MASK.reshape(-1),
                     n_increments=n_inc, total_time=n_inc * dt, newton_tol=1e-12, load_tol=1e-12, eta_inner=1e-8,
                     tol=1e-13)
    s.set_checkpointing(True)
    for k in range(n_inc):
        s.solve_increment(k)
    sig_before = s.homogenized_stress()
    dJ, rep = s.cp_adjoint(g[None])
    assert rep["outer_iters"] == n_inc and rep["cg_iters"] > 0
    assert rel_err(s.homogenized_stress(), sig_before) < 1e-13  # the forward state is restored
    s.close()
    cp = o.CrystalPlasticity(quats)
    prob = o.Problem(shape, "small", CP_MASK.reshape(-1))
    ref, J, recs = o.cp_adjoint_increments(prob, cp, grains, dt, targets, g)
    assert rel_err(sig_before[0], recs[-1]["stress_bar"]) < 1e-10
    assert rel_err(dJ.cpu().numpy()[0], ref) < 1e-9


def test_cp_adjoint_needs_checkpoints_and_fp64():
    shape, grains, quats = _case()
    dbfft = _dbfft()
    tgt = _targets(2, 1e-3)[-1][None]
    s = dbfft.Solver(shape, grains, dbfft.cp_phases(quats), tgt, stress_mask=CP_MASK.reshape(-1), n_increments=2,
                     total_time=1.0)
    s.solve_increment(0)
    with pytest.raises(dbfft.DbfftError):  # no checkpoints recorded
        s.cp_adjoint(np.eye(3)[None])
    with pytest.raises(dbfft.DbfftError):  # too late to start recording
        s.set_checkpointing(True)
    s.close()
    s = dbfft.Solver(shape, grains, dbfft.cp_phases(quats), tgt, stress_mask=CP_MASK.reshape(-1), n_increments=2,
                     total_time=1.0, precision=dbfft.DBFFT_MIXED)
    s.set_checkpointing(True)
    s.solve_increment(0)
    with pytest.raises(dbfft.DbfftError):  # the FP32 tangent of the mixed form is not the adjoint's operator
        s.cp_adjoint(np.eye(3)[None])
    s.close()
