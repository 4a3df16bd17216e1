"""GPU parity of full linear solves (FP64 and FP32-inner / FP64-outer) against the oracle.

Parity runs solve both sides to 1e-12 (FP64) so that the difference is the
solve error, not a CG rounding path: bar 1e-10 relative on fields and
homogenized stress for FP64, 1e-6 on the homogenized stress for MIXED.
"""
import numpy as np
import pytest

import oracle.dbfft_oracle as o
from paper_1905_12725_gb300 import synth
from tests.helpers import iso_tangent, mask9, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dbfft():
    from paper_1905_12725_gb300 import dbfft
    return dbfft


def test_config1_fp64_parity():
    """Centred sphere, 16^3, E 1 / 10, nu 0.3, eps_xx = 1e-3."""
    c = synth.config1()
    dbfft = _dbfft()
    s = dbfft.Solver((16, 16, 16), c["phase"], dbfft.iso_phases(c["E"], c["nu"]), c["eps_bar"][None],
                     tol=1e-12)
    rep = s.solve_increment(0)
    sig = s.homogenized_stress()[0]
    u, _ = s.get_solution()
    prob = o.Problem((16, 16, 16))
    ref = o.solve_linear(prob, iso_tangent(c["phase"], c["E"], c["nu"]), c["eps_bar"], tol=1e-12)
    assert rep["true_rel_res"] <= 1e-12
    assert rel_err(sig, ref["sig_bar"]) < 1e-10
    assert rel_err(u.cpu().numpy()[0], ref["u"]) < 1e-10
    # the configuration's own tolerance: PCG to 1e-8
    s2 = dbfft.Solver((16, 16, 16), c["phase"], dbfft.iso_phases(c["E"], c["nu"]), c["eps_bar"][None], tol=1e-8)
    rep2 = s2.solve_increment(0)
    assert rep2["true_rel_res"] <= 1e-8
    assert rel_err(s2.homogenized_stress()[0], ref["sig_bar"]) < 1e-7


@pytest.mark.parametrize("precision", [0, 1])
def test_mixed_control_solve_parity(precision):
    shape = (16, 16, 32)
    g = np.random.default_rng(17)
    phase = (g.random(shape) < 0.3).astype(np.uint16)
    E, nu = [1.0, 50.0], [0.3, 0.25]
    mask = mask9([(1, 1), (2, 2), (1, 2)])
    target = np.array([[1e-3, 1e-4, 0], [1e-4, 0.0, 0.0], [0, 0.0, 0.0]])
    dbfft = _dbfft()
    s = dbfft.Solver(shape, phase, dbfft.iso_phases(E, nu), target[None], stress_mask=mask, tol=1e-12 if precision == 0 else 1e-9,
                     precision=precision, eta_inner=1e-3)
    s.solve_increment(0)
    sig = s.homogenized_stress()[0]
    prob = o.Problem(shape, "small", mask)
    ref = o.solve_linear(prob, iso_tangent(phase, E, nu), target, tol=1e-12)
    assert rel_err(sig, ref["sig_bar"]) < (1e-10 if precision == 0 else 1e-6)
    u, e = s.get_solution()
    if precision == 0:
        assert rel_err(u.cpu().numpy()[0], ref["u"]) < 1e-9
        assert np.abs(e[0][[1, 2, 3]] - ref["e"]).max() < 1e-10 * np.abs(ref["e"]).max()


@pytest.mark.parametrize("precision", [0, 1])
def test_homogenized_tangent_six_rhs_batched(precision):
    """Six unit Mandel strains solved as one batch of right-hand sides sharing one map."""
    shape = (16, 16, 16)
    rng = synth.Xoshiro256ss(99)
    phase, _ = synth.rsa_spheres(16, 2.5, 0.2, rng)
    E, nu = [1.0, 100.0], [0.3, 0.3]
    dbfft = _dbfft()
    s = dbfft.Solver(shape, phase, dbfft.iso_phases(E, nu), np.zeros((6, 3, 3)), batch=6,
                     tol=1e-12 if precision == 0 else 1e-7, precision=precision, eta_inner=1e-3)
    Ceff, rep = s.homogenized_tangent()
    Ceff = Ceff[0]
    Cref, _ = o.homogenized_tangent(shape, iso_tangent(phase, E, nu), tol=1e-12)
    assert rel_err(Ceff, Cref) < (1e-10 if precision == 0 else 1e-6)
    assert np.abs(Ceff - Ceff.T).max() < (1e-10 if precision == 0 else 1e-6) * np.abs(Ceff).max()


@pytest.mark.parametrize("precision", [0, 1])
def test_centred_inclusion_64_cubed_gives_a_cubic_stiffness(precision):
    """A property that holds at any size: one centred sphere on an equal-sided even grid is
    unchanged by the cube's symmetries, and so is the discrete operator, so C_eff is cubic
    (C11 = C22 = C33, C12 = C13 = C23, C44 = C55 = C66, no other coupling). Axis 3 runs through
    other kernels (the real-to-complex pass) than axes 1-2, so an axis-specific slip there
    breaks it. C_eff also lies between the Reuss and Voigt bounds."""
    n = 64
    phase = synth.centred_sphere(n, 16)
    E, nu = [1.0, 10.0], [0.3, 0.3]
    dbfft = _dbfft()
    s = dbfft.Solver((n, n, n), phase, dbfft.iso_phases(E, nu), np.zeros((6, 3, 3)), batch=6,
                     tol=1e-12 if precision == 0 else 1e-7, precision=precision, eta_inner=1e-3)
    C, _ = s.homogenized_tangent()
    C = C[0]
    bar = (1e-9 if precision == 0 else 1e-6) * np.abs(C).max()
    d = np.diag(C)
    assert np.ptp(d[:3]) < bar and np.ptp(d[3:]) < bar
    assert np.ptp([C[0, 1], C[0, 2], C[1, 2], C[1, 0], C[2, 0], C[2, 1]]) < bar
    assert np.abs(C[:3, 3:]).max() < bar and np.abs(C[3:, :3]).max() < bar
    assert np.abs(C[3:, 3:] - np.diag(d[3:])).max() < bar
    vf = phase.mean()
    Cm = [o.tensor4_to_mandel(o.iso_stiffness(*o.lame(e, v))) for e, v in zip(E, nu)]
    Cv = (1 - vf) * Cm[0] + vf * Cm[1]
    Cr = np.linalg.inv((1 - vf) * np.linalg.inv(Cm[0]) + vf * np.linalg.inv(Cm[1]))
    assert np.linalg.eigvalsh(Cv - C).min() > -bar
    assert np.linalg.eigvalsh(C - Cr).min() > -bar


def test_zero_load_returns_zero_without_iterations():
    shape = (8, 8, 8)
    dbfft = _dbfft()
    s = dbfft.Solver(shape, np.zeros(shape, np.uint16), dbfft.iso_phases([1.0], [0.3]), np.zeros((1, 3, 3)))
    rep = s.solve_increment(0)
    assert rep["cg_iters"] == 0
    assert np.abs(s.homogenized_stress()).max() == 0.0


def test_graph_and_launch_by_launch_inner_solves_agree():
    """The inner PCG runs as one CUDA graph (WHILE node) after a warm solve; with
    profiling on it is launched kernel by kernel. Both give the same iterates."""
    shape = (16, 16, 32)
    g = np.random.default_rng(23)
    phase = (g.random(shape) < 0.3).astype(np.uint16)
    E, nu = [1.0, 30.0], [0.3, 0.3]
    tgt = np.zeros((2, 3, 3))
    tgt[0, 0, 0] = 1e-3
    tgt[1, 0, 1] = tgt[1, 1, 0] = 5e-4
    dbfft = _dbfft()
    s = dbfft.Solver(shape, phase, dbfft.iso_phases(E, nu), tgt, batch=2, tol=1e-10, precision=1, eta_inner=1e-3)
    r0 = s.solve_increment(0)           # first inner solve launch by launch, later ones as graphs
    sig_graph = s.homogenized_stress()
    n0 = s.launch_count()
    s.profile(True)                      # profiling forces launch-by-launch execution
    r1 = s.solve_increment(0)
    sig_plain = s.homogenized_stress()
    s.profile(False)
    assert r0["cg_iters"] == r1["cg_iters"]
    assert np.abs(sig_graph - sig_plain).max() <= 1e-14 * np.abs(sig_plain).max()
    assert s.launch_count() > n0


_PDL_CHILD = r"""
import sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_1905_12725_gb300 import dbfft
shape = (16, 16, 32)
g = np.random.default_rng(23)
phase = (g.random(shape) < 0.3).astype(np.uint16)
tgt = np.zeros((2, 3, 3)); tgt[0, 0, 0] = 1e-3; tgt[1, 0, 1] = tgt[1, 1, 0] = 5e-4
s = dbfft.Solver(shape, phase, dbfft.iso_phases([1.0, 30.0], [0.3, 0.3]), tgt, batch=2, tol=1e-10, precision=1,
                 eta_inner=1e-3)
s.solve_increment(0)
r = s.solve_increment(0)  # graph-captured inner solves
np.save(sys.argv[2], np.concatenate([s.homogenized_stress().ravel(), [r["cg_iters"]]]))
"""


def test_programmatic_dependent_launch_gives_the_same_solve(tmp_path):
    """The CG graph with programmatic dependencies between its kernels (DBFFT_PDL=1, off by
    default) and without them reach the same iterates."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = {}
    for flag in ("0", "1"):
        f = str(tmp_path / f"pdl{flag}.npy")
        r = subprocess.run([sys.executable, "-c", _PDL_CHILD, root, f], env=dict(os.environ, DBFFT_PDL=flag),
                           capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stderr[-2000:]
        out[flag] = np.load(f)
    assert out["0"][-1] == out["1"][-1]  # CG iterations
    assert np.abs(out["0"][:-1] - out["1"][:-1]).max() <= 1e-14 * np.abs(out["0"][:-1]).max()
