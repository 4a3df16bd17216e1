"""GPU parity of one DBFFT operator application against the FP64 oracle.

The CUDA path (called through the C ABI) and the oracle receive the same
seeded Hermitian-consistent spectra. Shapes span several tiles of every pass
and ragged tails (n3/2 + 1 columns, non-cubic grids). Bar: 1e-12 relative
(max-norm) for FP64 applications, 2e-5 for FP32.
"""
import numpy as np
import pytest

import oracle.dbfft_oracle as o
from paper_1905_12725_gb300 import synth
from tests.helpers import e9_to_oracle, e_oracle_to9, iso_tangent, mask9, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPES = [(16, 16, 16), (8, 16, 32), (32, 8, 16), (64, 32, 8), (16, 64, 64)]


def _solver(shape, phase, E, nu, target, **kw):
    from paper_1905_12725_gb300 import dbfft
    return dbfft.Solver(shape, phase, dbfft.iso_phases(E, nu), target, **kw)


def _random_phase(shape, seed, nmat=1):
    g = np.random.default_rng(seed)
    return (g.random((nmat,) + shape) < 0.35).astype(np.uint16)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("fp32", [False, True])
def test_small_strain_operator_matches_oracle(shape, fp32):
    B = 2
    phase = _random_phase(shape, 1)
    E, nu = [1.0, 30.0], [0.3, 0.2]
    s = _solver(shape, phase, E, nu, np.zeros((B, 3, 3)), batch=B)
    u = synth.random_spectrum(shape, 3, 7, batch=B)
    out, _ = s.apply(torch.from_numpy(u).cuda(), fp32=fp32)
    out = out.cpu().numpy()
    prob = o.Problem(shape)
    T = iso_tangent(phase[0], E, nu)
    for b in range(B):
        ref, _ = prob.apply_K(T, u[b], np.zeros(0))
        assert rel_err(out[b], ref) < (2e-5 if fp32 else 1e-12)
    s.close()


def test_batched_materials_and_rhs_sharing_a_map():
    """B = 6 right-hand sides over 3 material maps (2 per map)."""
    shape = (16, 8, 32)
    phase = _random_phase(shape, 3, nmat=3)
    E, nu = [1.0, 12.0], [0.25, 0.3]
    s = _solver(shape, phase, E, nu, np.zeros((6, 3, 3)), batch=6)
    u = synth.random_spectrum(shape, 3, 9, batch=6)
    out, _ = s.apply(torch.from_numpy(u).cuda())
    out = out.cpu().numpy()
    prob = o.Problem(shape)
    for b in range(6):
        ref, _ = prob.apply_K(iso_tangent(phase[b // 2], E, nu), u[b], np.zeros(0))
        assert rel_err(out[b], ref) < 1e-12


def test_operator_with_macro_unknowns_matches_oracle():
    shape = (16, 16, 8)
    mask = mask9([(0, 0), (1, 2), (0, 1)])
    phase = _random_phase(shape, 5)
    E, nu = [2.0, 0.5], [0.3, 0.35]
    s = _solver(shape, phase, E, nu, np.zeros((1, 3, 3)), stress_mask=mask)
    prob = o.Problem(shape, "small", mask)
    u = synth.random_spectrum(shape, 3, 11)
    e = np.random.default_rng(2).standard_normal(prob.ne)
    e9 = e_oracle_to9(prob, e)
    out, eo = s.apply(torch.from_numpy(u).cuda(), torch.from_numpy(e9[None]).cuda())
    qu, qe = prob.apply_K(iso_tangent(phase[0], E, nu), u[0], e)
    assert rel_err(out.cpu().numpy()[0], qu) < 1e-12
    assert rel_err(e9_to_oracle(prob, eo.cpu().numpy()[0]), qe) < 1e-12


@pytest.mark.parametrize("fp32", [False, True])
def test_preconditioner_matches_oracle(fp32):
    shape = (32, 16, 16)
    mask = mask9([(1, 1), (0, 2)])
    phase = _random_phase(shape, 6)
    E, nu = [1.0, 8.0], [0.3, 0.3]
    s = _solver(shape, phase, E, nu, np.zeros((1, 3, 3)), stress_mask=mask)
    prob = o.Problem(shape, "small", mask)
    T = iso_tangent(phase[0], E, nu)
    M = prob.make_preconditioner(T.mean())
    u = synth.random_spectrum(shape, 3, 12)
    e = np.random.default_rng(3).standard_normal(prob.ne)
    out, eo = s.apply(torch.from_numpy(u).cuda(), torch.from_numpy(e_oracle_to9(prob, e)[None]).cuda(),
                      fp32=fp32, precond=True)
    zu, ze = M((u[0], e))
    assert rel_err(out.cpu().numpy()[0], zu) < (2e-5 if fp32 else 1e-12)
    assert rel_err(e9_to_oracle(prob, eo.cpu().numpy()[0]), ze) < 1e-12


def test_residual_chain_matches_oracle():
    """b - K u with the macro load (FP64), mixed control."""
    shape = (16, 32, 16)
    mask = mask9([(1, 1), (2, 2)])
    phase = _random_phase(shape, 8)
    E, nu = [1.0, 20.0], [0.3, 0.3]
    target = np.array([[1e-3, 2e-4, 0.0], [2e-4, 0.5, 0.0], [0.0, 0.0, -0.2]])
    s = _solver(shape, phase, E, nu, target[None], stress_mask=mask)
    prob = o.Problem(shape, "small", mask)
    u = synth.random_spectrum(shape, 3, 13) * 1e-6
    e = np.random.default_rng(4).standard_normal(prob.ne) * 1e-3
    out, eo = s.apply(torch.from_numpy(u).cuda(), torch.from_numpy(e_oracle_to9(prob, e)[None]).cuda(),
                      residual=True)
    T = iso_tangent(phase[0], E, nu)
    epsU, sig_f = o.split_load(prob, target)
    r, _, _ = o.residual(prob, T.apply, (u[0], e), epsU, sig_f)
    assert rel_err(out.cpu().numpy()[0], r[0]) < 1e-12
    assert rel_err(e9_to_oracle(prob, eo.cpu().numpy()[0]), r[1]) < 1e-12


@pytest.mark.parametrize("precision", [0, 1])
def test_autotuned_launch_shapes_keep_results(precision, tmp_path):
    """dbfft_autotune picks launch shapes by timing; the operator is unchanged."""
    from paper_1905_12725_gb300 import dbfft
    shape = (32, 16, 64)
    B = 3
    phase = _random_phase(shape, 31)
    E, nu = [1.0, 30.0], [0.3, 0.2]
    s = _solver(shape, phase, E, nu, np.zeros((B, 3, 3)), batch=B, precision=precision)
    u = synth.random_spectrum(shape, 3, 33, batch=B)
    fp32 = precision == 1
    before, _ = s.apply(torch.from_numpy(u).cuda(), fp32=fp32)
    cache = str(tmp_path / "tune.txt")
    note = s.autotune(cache)
    assert "pass3" in note
    after, _ = s.apply(torch.from_numpy(u).cuda(), fp32=fp32)
    assert rel_err(after.cpu().numpy(), before.cpu().numpy()) < (2e-6 if fp32 else 1e-13)
    # a second context reads the cache instead of timing
    s2 = _solver(shape, phase, E, nu, np.zeros((B, 3, 3)), batch=B, precision=precision)
    assert s2.autotune(cache).startswith("from cache:")
    prob = o.Problem(shape)
    ref, _ = prob.apply_K(iso_tangent(phase[0], E, nu), u[0], np.zeros(0))
    assert rel_err(after.cpu().numpy()[0], ref) < (2e-5 if fp32 else 1e-12)
