"""The line-bulk pass 3 (FP32 CG applications on lines of n3 = 64, 128 or 256 values).

The kernel moves whole tiles by bulk copies and runs each line's half-length
transform as two register stages with one swizzled exchange (Sec. 2.2,
Eq. lineqf: the C2R, the contraction and the R2C of one application). These
tests compare its K u with the FP64 oracle at the FP32 operator bar (2e-5,
max-norm relative): tiles of 2 to 16 lines, several right-hand sides per
material map (line slots that do not fill the last block of 16), per-voxel
scale, the Neo-Hookean tangent after a constitutive update, the stored
crystal-plasticity tangent against the plain kernel on the same tangent,
whole graph-captured PCG solves, and the bounded wait that returns E_TIMEOUT.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle.dbfft_oracle as o
from paper_1905_12725_gb300 import synth
from tests.helpers import iso_tangent, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_OP = 2e-5


def _dbfft():
    from paper_1905_12725_gb300 import dbfft
    return dbfft


CASES = [
    # shape, B, n_materials, lines
    ((8, 8, 256), 1, 1, 8),
    ((16, 8, 256), 2, 1, 2),
    ((8, 8, 256), 3, 3, 16),
    ((8, 16, 128), 1, 1, 16),
    ((8, 8, 128), 2, 2, 4),
    ((16, 8, 128), 3, 1, 8),
    ((8, 8, 64), 1, 1, 16),
    ((16, 8, 64), 6, 1, 4),
    ((8, 8, 64), 6, 6, 2),
]


@pytest.mark.parametrize("shape,B,nmat,lines", CASES)
@pytest.mark.parametrize("scaled", [False, True])
def test_line_bulk_pass3_matches_oracle(shape, B, nmat, lines, scaled):
    dbfft = _dbfft()
    g = np.random.default_rng(sum(shape) + 7 * B + lines)
    phase = (g.random((nmat,) + shape) < 0.4).astype(np.uint16)
    E, nu = [1.0, 25.0], [0.3, 0.2]
    scale = 0.5 + g.random((nmat,) + shape) if scaled else None
    s = dbfft.Solver(shape, phase, dbfft.iso_phases(E, nu), np.zeros((B, 3, 3)), batch=B, E_scale=scale,
                     precision=dbfft.DBFFT_MIXED)
    s.set_pass3_shape(0, 3, 0, lines)
    u = synth.random_spectrum(shape, 3, 300 + lines, batch=B)
    out, _ = s.apply(torch.from_numpy(u).cuda(), fp32=True)
    out = out.cpu().numpy()
    prob = o.Problem(shape)
    Rm = B // nmat
    for b in range(B):
        T = iso_tangent(phase[b // Rm], E, nu, None if scale is None else scale[b // Rm])
        ref, _ = prob.apply_K(T, u[b], np.zeros(0))
        assert rel_err(out[b], ref) < FP32_OP, b
    s.close()


def test_line_bulk_refuses_unsupported_shapes():
    dbfft = _dbfft()
    s = dbfft.Solver((8, 8, 32), np.zeros((8, 8, 32), np.uint16), dbfft.iso_phases([1.0], [0.3]), np.zeros((1, 3, 3)),
                     precision=dbfft.DBFFT_MIXED)
    with pytest.raises(dbfft.DbfftError):  # n3 = 32 has no line-bulk kernel
        s.set_pass3_shape(0, 3, 0, 8)
    s.close()
    s = dbfft.Solver((8, 8, 128), np.zeros((8, 8, 128), np.uint16), dbfft.iso_phases([1.0], [0.3]),
                     np.zeros((1, 3, 3)), precision=dbfft.DBFFT_MIXED)
    for args in [(0, 3, 0, 3), (1, 3, 0, 4), (0, 3, 0, 128)]:  # odd lines, FP64, too much shared memory
        with pytest.raises(dbfft.DbfftError):
            s.set_pass3_shape(*args)
    s.close()


@pytest.mark.parametrize("n3", [128, 64])
def test_line_bulk_neo_hooke_tangent_matches_oracle(n3):
    """Finite strain (nine components): K(F) in FP32 after a constitutive update at a random F."""
    dbfft = _dbfft()
    shape = (8, 8, n3)
    g = np.random.default_rng(5)
    phase = (g.random(shape) < 0.3).astype(np.uint16)
    mu = np.array([1.0, 20.0])
    lam = 1.5 * mu
    Fbar = np.array([[1.05, 0.02, 0.0], [0.01, 0.97, 0.03], [0.0, -0.02, 1.01]])
    s = dbfft.Solver(shape, phase, dbfft.neo_hooke_phases(mu, lam), Fbar[None], kinematics=dbfft.DBFFT_FINITE,
                     precision=dbfft.DBFFT_MIXED)
    s.set_pass3_shape(0, 3, 0, 4)
    prob = o.Problem(shape, "finite")
    x = synth.random_spectrum(shape, 3, 31) * 2e-4
    s.apply(torch.from_numpy(x).cuda(), residual=True)  # constitutive update at F(x): stores the FP32 tangent
    F = prob.field_from(x[0], np.zeros(0)) + Fbar[:, :, None, None, None]
    _, Kf = o.neo_hooke(F, mu[phase], lam[phase])
    u = synth.random_spectrum(shape, 3, 32)
    out, _ = s.apply(torch.from_numpy(u).cuda(), fp32=True)
    ref, _ = prob.apply_K(o.FullTangent(Kf), u[0], np.zeros(0))
    assert rel_err(out.cpu().numpy()[0], ref) < FP32_OP
    s.close()


@pytest.mark.parametrize("n3", [256, 64])
def test_line_bulk_crystal_plasticity_tangent_equals_plain_kernel(n3):
    """Small-strain crystal plasticity: the stored 21-value tangent applied by the
    line-bulk and the plain kernel, after the same constitutive update."""
    dbfft = _dbfft()
    shape = (8, 8, n3)
    rng = synth.Xoshiro256ss(77)
    grains, _ = synth.periodic_voronoi(8, 6, rng)
    grains = np.tile(grains, (1, 1, n3 // 8))
    quats = synth.uniform_quaternions(6, rng)
    tgt = np.zeros((1, 3, 3))
    tgt[0, 0, 0] = 4e-3  # beyond the elastic limit: the tangent differs from grain to grain and in slip
    s = dbfft.Solver(shape, grains, dbfft.cp_phases(quats), tgt, precision=dbfft.DBFFT_MIXED, total_time=1.0)
    x = synth.random_spectrum(shape, 3, 41) * 1e-4
    s.apply(torch.from_numpy(x).cuda(), residual=True)
    u = torch.from_numpy(synth.random_spectrum(shape, 3, 42)).cuda()
    s.set_pass3_shape(0, 0, 8, 8)
    ref, _ = s.apply(u, fp32=True)
    s.set_pass3_shape(0, 3, 0, 8)
    out, _ = s.apply(u, fp32=True)
    assert rel_err(out.cpu().numpy(), ref.cpu().numpy()) < FP32_OP
    s.close()


@pytest.mark.parametrize("shape", [(8, 16, 128), (8, 8, 256), (16, 8, 64)])
def test_pcg_with_line_bulk_pass3_matches_oracle(shape):
    """Mixed-control solves of two right-hand sides (graph-captured inner PCG,
    right-hand sides that stop at different iterations) with the line-bulk pass."""
    dbfft = _dbfft()
    g = np.random.default_rng(43)
    phase = (g.random(shape) < 0.3).astype(np.uint16)
    E, nu = [1.0, 40.0], [0.3, 0.3]
    mask = np.zeros((3, 3), bool)
    mask[1, 1] = mask[2, 2] = True
    tgt = np.zeros((2, 3, 3))
    tgt[0, 0, 0] = 1e-3
    tgt[1, 0, 1] = tgt[1, 1, 0] = 5e-4
    s = dbfft.Solver(shape, phase, dbfft.iso_phases(E, nu), tgt, batch=2, stress_mask=mask.reshape(-1),
                     precision=dbfft.DBFFT_MIXED, tol=1e-9, eta_inner=1e-3)
    s.set_pass3_shape(0, 3, 0, 4)
    s.solve_increment(0)
    s.solve_increment(0)  # the second solve runs the inner PCG as a CUDA graph
    sig = s.homogenized_stress()
    s.close()
    prob = o.Problem(shape, "small", mask.reshape(-1))
    T = iso_tangent(phase, E, nu)
    for b in range(2):
        ref = o.solve_linear(prob, T, tgt[b], tol=1e-12)["sig_bar"]
        assert rel_err(sig[b], ref) < 1e-7


_TIMEOUT_CHILD = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_1905_12725_gb300 import dbfft
shape = (8, 8, 256)
phase = (np.random.default_rng(3).random(shape) < 0.3).astype(np.uint16)
eps = np.zeros((1, 3, 3)); eps[0, 0, 0] = 1e-3
s = dbfft.Solver(shape, phase, dbfft.iso_phases([1.0, 10.0], [0.3, 0.3]), eps, precision=dbfft.DBFFT_MIXED,
                 max_iter=50, max_newton=2)
s.set_pass3_shape(0, 3, 0, 8)
try:
    s.solve_increment(0)
    print("NO_ERROR")
except dbfft.DbfftError as exc:
    print(dbfft.STATUS[exc.status])
s.close()
torch.cuda.synchronize()  # the context is still usable
print("SYNC_OK")
"""


def test_line_bulk_bounded_wait_returns_timeout():
    """A one-poll limit on the first bulk-copy wait runs out before the copies
    land: the kernel records it, waits (with the full limit) for its copies and
    skips its work; the solve returns E_TIMEOUT and the GPU context stays usable."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, DBFFT_WAIT_POLLS="1")
    r = subprocess.run([sys.executable, "-c", _TIMEOUT_CHILD, root], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = r.stdout.split()
    assert "DBFFT_E_TIMEOUT" in lines and "SYNC_OK" in lines, r.stdout


@pytest.mark.parametrize("shape,B,nmat,threads", [((8, 16, 256), 1, 1, -1), ((16, 8, 128), 3, 1, -1),
                                                   ((8, 8, 256), 2, 2, -1), ((16, 16, 256), 1, 1, 192),
                                                   ((8, 16, 128), 2, 1, 192), ((8, 16, 256), 1, 1, -2),
                                                   ((16, 8, 128), 3, 1, -2), ((8, 8, 256), 2, 2, -2),
                                                   ((16, 8, 64), 6, 1, -2), ((8, 16, 64), 2, 1, -1),
                                                   ((8, 8, 64), 3, 3, 192)])
def test_line_bulk_warp_lines_and_thread_caps_match_oracle(shape, B, nmat, threads):
    """The warp-lines forms (every warp takes its own lines through all phases: radix -1 with
    16-line tiles, -2 with two lines per warp) and a 192-thread cap, against the oracle."""
    dbfft = _dbfft()
    g = np.random.default_rng(sum(shape) + B + threads)
    phase = (g.random((nmat,) + shape) < 0.4).astype(np.uint16)
    E, nu = [1.0, 25.0], [0.3, 0.2]
    scale = 0.5 + g.random((nmat,) + shape)
    s = dbfft.Solver(shape, phase, dbfft.iso_phases(E, nu), np.zeros((B, 3, 3)), batch=B, E_scale=scale,
                     precision=dbfft.DBFFT_MIXED)
    lines = (8 if shape[2] == 256 else 4) if threads == -2 else 16
    s.set_pass3_shape(0, 3, threads, lines)
    u = synth.random_spectrum(shape, 3, 700 + B, batch=B)
    out, _ = s.apply(torch.from_numpy(u).cuda(), fp32=True)
    out = out.cpu().numpy()
    prob = o.Problem(shape)
    Rm = B // nmat
    for b in range(B):
        ref, _ = prob.apply_K(iso_tangent(phase[b // Rm], E, nu, scale[b // Rm]), u[b], np.zeros(0))
        assert rel_err(out[b], ref) < FP32_OP, b
    with pytest.raises(dbfft.DbfftError):  # warp lines need 16-line tiles
        s.set_pass3_shape(0, 3, -1, 8)
    s.close()


@pytest.mark.parametrize("rhs,threads,lines", [(1, 0, 4), (2, -2, 4), (3, 192, 2), (6, -1, 16)])
def test_line_bulk_rhs_groups_match_oracle(rhs, threads, lines):
    """Six right-hand sides on one material map, the line-bulk CTAs taking 1, 2, 3 or 6 of them."""
    dbfft = _dbfft()
    shape = (16, 8, 64)
    g = np.random.default_rng(90 + rhs)
    phase = (g.random(shape) < 0.4).astype(np.uint16)
    E, nu = [1.0, 25.0], [0.3, 0.2]
    s = dbfft.Solver(shape, phase, dbfft.iso_phases(E, nu), np.zeros((6, 3, 3)), batch=6, precision=dbfft.DBFFT_MIXED)
    s.set_pass3_rhs_group(rhs)
    s.set_pass3_shape(0, 3, threads, lines)
    u = synth.random_spectrum(shape, 3, 800 + rhs, batch=6)
    out, _ = s.apply(torch.from_numpy(u).cuda(), fp32=True)
    out = out.cpu().numpy()
    prob = o.Problem(shape)
    T = iso_tangent(phase, E, nu)
    for b in range(6):
        ref, _ = prob.apply_K(T, u[b], np.zeros(0))
        assert rel_err(out[b], ref) < FP32_OP, b
    for bad in (4, 9, -1):  # 4 does not divide 6; at most 8
        with pytest.raises(dbfft.DbfftError):
            s.set_pass3_rhs_group(bad)
    s.close()
