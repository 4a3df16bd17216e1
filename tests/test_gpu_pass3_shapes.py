"""Pass 3 launch shapes: every shape of the plain and the pipelined (bulk-copy,
double-buffered) pass gives the oracle's K u, with and without per-voxel
scale, for several right-hand sides per material map, and full PCG solves
agree between the two kernels.

Shapes span several tiles per CTA (persistent loop), both radices, tiles of
2 to 16 lines and grids where n3 is the shortest and the longest axis.
"""
import numpy as np
import pytest

import oracle.dbfft_oracle as o
from paper_1905_12725_gb300 import synth
from tests.helpers import iso_tangent, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dbfft():
    from paper_1905_12725_gb300 import dbfft
    return dbfft


CASES = [
    # shape, B, n_materials, fp64, radix, lines
    ((16, 16, 16), 1, 1, 0, 8, 2),
    ((16, 16, 16), 2, 1, 0, 16, 4),
    ((8, 16, 64), 3, 3, 0, 8, 8),
    ((32, 8, 32), 2, 1, 1, 4, 2),
    ((16, 32, 128), 1, 1, 0, 16, 16),
    ((16, 8, 256), 2, 2, 0, 8, 4),
    ((8, 8, 256), 1, 1, 1, 4, 4),
    ((32, 32, 8), 4, 2, 0, 8, 16),
]


@pytest.mark.parametrize("shape,B,nmat,fp64,radix,lines", CASES)
@pytest.mark.parametrize("scaled", [False, True])
def test_pipelined_pass3_matches_oracle(shape, B, nmat, fp64, radix, lines, scaled):
    dbfft = _dbfft()
    g = np.random.default_rng(sum(shape) + B + lines)
    phase = (g.random((nmat,) + shape) < 0.4).astype(np.uint16)
    E, nu = [1.0, 25.0], [0.3, 0.2]
    scale = 0.5 + g.random((nmat,) + shape) if scaled else None
    s = dbfft.Solver(shape, phase, dbfft.iso_phases(E, nu), np.zeros((B, 3, 3)), batch=B, E_scale=scale,
                     precision=dbfft.DBFFT_FP64 if fp64 else dbfft.DBFFT_MIXED)
    u = synth.random_spectrum(shape, 3, 500 + lines, batch=B)
    prob = o.Problem(shape)
    Rm = B // nmat
    refs = [prob.apply_K(iso_tangent(phase[b // Rm], E, nu, None if scale is None else scale[b // Rm]), u[b],
                         np.zeros(0))[0] for b in range(B)]
    for pipelined in (1, 2):  # two shared-memory stages, one stage
        s.set_pass3_shape(fp64, pipelined, radix, lines)
        out, _ = s.apply(torch.from_numpy(u).cuda(), fp32=not fp64)
        out = out.cpu().numpy()
        for b in range(B):
            assert rel_err(out[b], refs[b]) < (1e-12 if fp64 else 2e-5), (pipelined, b)
    s.close()


def test_invalid_pipelined_shapes_are_refused():
    dbfft = _dbfft()
    shape = (8, 8, 16)
    s = dbfft.Solver(shape, np.zeros(shape, np.uint16), dbfft.iso_phases([1.0], [0.3]), np.zeros((1, 3, 3)))
    for args in [(0, 1, 8, 3), (0, 1, 8, 5), (0, 1, 32, 4), (1, 1, 8, 4), (0, 1, 8, 128), (1, 0, 4, 0), (0, 3, 8, 4)]:
        with pytest.raises(dbfft.DbfftError):
            s.set_pass3_shape(*args)
    s.set_pass3_shape(0, 1, 8, 4)
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_pcg_with_pipelined_pass3_equals_plain(precision):
    """Whole mixed-control solves (graph-captured inner PCG) with either kernel."""
    dbfft = _dbfft()
    shape = (16, 16, 32)
    g = np.random.default_rng(41)
    phase = (g.random(shape) < 0.3).astype(np.uint16)
    E, nu = [1.0, 40.0], [0.3, 0.3]
    mask = np.zeros((3, 3), bool)
    mask[1, 1] = mask[2, 2] = True
    tgt = np.zeros((2, 3, 3))
    tgt[0, 0, 0] = 1e-3
    tgt[1, 0, 1] = tgt[1, 1, 0] = 5e-4
    sig = []
    for pipelined in (0, 1, 2):
        s = dbfft.Solver(shape, phase, dbfft.iso_phases(E, nu), tgt, batch=2, stress_mask=mask.reshape(-1),
                         precision=precision, tol=1e-11 if precision == 0 else 1e-9, eta_inner=1e-3)
        fp64 = 1 if precision == 0 else 0
        s.set_pass3_shape(fp64, pipelined, 4 if fp64 else 8, 4)
        s.solve_increment(0)
        s.solve_increment(0)  # the second solve runs the inner PCG as a CUDA graph
        sig.append(s.homogenized_stress())
        s.close()
    prob = o.Problem(shape, "small", mask.reshape(-1))
    T = iso_tangent(phase, E, nu)
    for b in range(2):
        ref = o.solve_linear(prob, T, tgt[b], tol=1e-12)["sig_bar"]
        for k in range(3):
            assert rel_err(sig[k][b], ref) < (1e-10 if precision == 0 else 1e-7)


@pytest.mark.parametrize("shape,B,nmat,lines,fp64", [((16, 16, 64), 1, 1, 8, 0), ((8, 32, 32), 3, 3, 5, 0),
                                                     ((32, 16, 16), 6, 1, 7, 0), ((16, 8, 8), 2, 2, 3, 0),
                                                     ((8, 8, 128), 2, 1, 4, 0), ((8, 8, 256), 1, 1, 12, 0),
                                                     ((16, 8, 64), 2, 1, 3, 1),
                                                     ((8, 16, 32), 1, 1, 6, 1)])
def test_radix32_pass3_matches_oracle(shape, B, nmat, lines, fp64):
    """Radix 32: one thread holds a whole line (no exchange) for n3 <= 64, or half a
    line (one exchange) for n3 = 128; FP32 and FP64."""
    dbfft = _dbfft()
    g = np.random.default_rng(7 * lines + B)
    phase = (g.random((nmat,) + shape) < 0.4).astype(np.uint16)
    E, nu = [1.0, 25.0], [0.3, 0.2]
    s = dbfft.Solver(shape, phase, dbfft.iso_phases(E, nu), np.zeros((B, 3, 3)), batch=B,
                     precision=dbfft.DBFFT_FP64 if fp64 else dbfft.DBFFT_MIXED)
    s.set_pass3_shape(fp64, 0, 32, lines)
    u = synth.random_spectrum(shape, 3, 900 + lines, batch=B)
    out, _ = s.apply(torch.from_numpy(u).cuda(), fp32=not fp64)
    out = out.cpu().numpy()
    prob = o.Problem(shape)
    Rm = B // nmat
    for b in range(B):
        ref, _ = prob.apply_K(iso_tangent(phase[b // Rm], E, nu), u[b], np.zeros(0))
        assert rel_err(out[b], ref) < (1e-12 if fp64 else 2e-5), b
    s.close()
