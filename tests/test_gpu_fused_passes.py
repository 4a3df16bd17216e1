"""The fused first and last passes of the FP32 CG iteration.

In the mixed-precision inner CG, the preconditioner, the direction and
iterate updates and the gradient run inside the inverse axis-2 transform,
and the divergence, null mask, residual update and CG reductions inside the
forward axis-2 transform (Sec. 2.2, Eqs. s-hat and d-hat; Sec. 2.5). These
tests solve with that chain on grids whose n2 selects it (32 to 256), with
stress-controlled components (the macro rows read sigma-hat(0) inside the
fused divergence pass) and right-hand sides that stop at different
iterations, and compare the homogenized stress with the FP64 oracle at the
mixed-form bar; the fused and the unfused chain must also agree.
"""
import os

import numpy as np
import pytest

import oracle.dbfft_oracle as o
from tests.helpers import iso_tangent, mask9, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dbfft():
    from paper_1905_12725_gb300 import dbfft
    return dbfft


def _solve(shape, phase, E, nu, tgt, mask, fuse):
    dbfft = _dbfft()
    old = os.environ.get("DBFFT_FUSE_AX2")
    os.environ["DBFFT_FUSE_AX2"] = "1" if fuse else "0"
    try:
        s = dbfft.Solver(shape, phase, dbfft.iso_phases(E, nu), tgt, batch=tgt.shape[0],
                         stress_mask=None if mask is None else mask.reshape(-1), precision=dbfft.DBFFT_MIXED,
                         tol=1e-9, eta_inner=1e-3)
    finally:
        if old is None:
            del os.environ["DBFFT_FUSE_AX2"]
        else:
            os.environ["DBFFT_FUSE_AX2"] = old
    reps = [s.solve_increment(0), s.solve_increment(0)]  # the second inner solves run as a CUDA graph
    sig = s.homogenized_stress()
    s.close()
    return sig, reps


@pytest.mark.parametrize("shape", [(8, 32, 16), (16, 64, 8), (8, 128, 32), (9, 32, 15)])
def test_fused_cg_passes_match_oracle(shape):
    g = np.random.default_rng(sum(shape))
    phase = (g.random(shape) < 0.35).astype(np.uint16)
    E, nu = [1.0, 30.0], [0.3, 0.25]
    mask = mask9([(1, 1), (2, 2), (0, 1)])
    tgt = np.zeros((2, 3, 3))
    tgt[0, 0, 0] = 1e-3
    tgt[1, 0, 2] = tgt[1, 2, 0] = 4e-4
    sig, reps = _solve(shape, phase, E, nu, tgt, mask.reshape(3, 3), fuse=True)
    prob = o.Problem(shape, "small", mask)
    T = iso_tangent(phase, E, nu)
    for b in range(2):
        ref = o.solve_linear(prob, T, tgt[b], tol=1e-12)["sig_bar"]
        assert rel_err(sig[b], ref) < 1e-7, b
    sig0, _ = _solve(shape, phase, E, nu, tgt, mask.reshape(3, 3), fuse=False)
    assert rel_err(sig, sig0) < 1e-7
