"""Pins of the FP64 oracle against mathematics it does not share code with.

Each test fixes a part of the oracle to something other than itself: closed
forms (plane waves, laminates, the crystal-plasticity steady state), exact
invariants (Parseval, Hermitian symmetry, the null space of the discrete
operator), brute force on tiny grids (a dense matrix on 4^3 and 5^3) and
finite differences. A plausible slip in the oracle -- a dropped 1/2 in the
symmetric gradient, a sign of i xi, a transposed tangent, a wrong weight in
the half-spectrum inner product -- fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle.dbfft_oracle as o
from paper_1905_12725_gb300 import synth

RNG = np.random.default_rng(1905)


def _iso_random(shape, seed=0, contrast=10.0):
    g = np.random.default_rng(seed)
    E = np.where(g.random(shape) < 0.4, contrast, 1.0)
    nu = np.where(g.random(shape) < 0.5, 0.3, 0.2)
    lam, mu = o.lame(E, nu)
    return o.IsoTangent(lam, mu)


# ---------------------------------------------------------------- frequencies (R1)
def test_spectral_derivative_of_band_limited_field():
    """The oracle's gradient of a sampled trigonometric field is its exact derivative.

    Pins 2 pi / L, the sign of i xi, the FFT ordering of k and the axis order.
    """
    shape = (8, 12, 16)
    x = [(np.arange(n) + 0.5) / n for n in shape]
    X1, X2, X3 = np.meshgrid(*x, indexing="ij")
    u = np.zeros((3,) + shape)
    u[0] = np.sin(2 * np.pi * 3 * X1) * np.cos(2 * np.pi * 2 * X3)
    u[1] = np.cos(2 * np.pi * 5 * X2 + 0.3)
    u[2] = np.sin(2 * np.pi * (X1 + X2 + X3))
    du = np.zeros((3, 3) + shape)
    du[0, 0] = 2 * np.pi * 3 * np.cos(2 * np.pi * 3 * X1) * np.cos(2 * np.pi * 2 * X3)
    du[0, 2] = -2 * np.pi * 2 * np.sin(2 * np.pi * 3 * X1) * np.sin(2 * np.pi * 2 * X3)
    du[1, 1] = -2 * np.pi * 5 * np.sin(2 * np.pi * 5 * X2 + 0.3)
    for j in range(3):
        du[2, j] = 2 * np.pi * np.cos(2 * np.pi * (X1 + X2 + X3))
    xi = o.frequencies(shape)
    G = o.to_real(o.grad_hat(np.fft.rfftn(u, axes=(-3, -2, -1)), xi), shape)
    assert np.abs(G - du).max() < 1e-11
    # symmetric gradient is the symmetric part, divergence is the trace contraction
    E = o.to_real(o.sym_grad_hat(np.fft.rfftn(u, axes=(-3, -2, -1)), xi), shape)
    assert np.abs(E - 0.5 * (du + np.swapaxes(du, 0, 1))).max() < 1e-11


def test_nyquist_mode_has_zero_derivative_and_null_set():
    shape = (4, 6, 8)
    i = np.arange(4)[:, None, None]
    f = np.broadcast_to((-1.0) ** i, shape)
    u = np.stack([f, f, f])
    xi = o.frequencies(shape)
    G = o.to_real(o.grad_hat(np.fft.rfftn(u, axes=(-3, -2, -1)), xi), shape)
    assert np.abs(G).max() < 1e-14
    Z = o.null_mask(shape)
    assert Z.sum() == 8  # k_i in {0, -N_i/2} on all three even axes
    Zodd = o.null_mask((5, 5, 5))
    assert Zodd.sum() == 1


def test_half_spectrum_inner_product_is_parseval():
    shape = (6, 4, 10)
    a = RNG.standard_normal((3,) + shape)
    b = RNG.standard_normal((3,) + shape)
    ah, bh = np.fft.rfftn(a, axes=(-3, -2, -1)), np.fft.rfftn(b, axes=(-3, -2, -1))
    N = np.prod(shape)
    assert abs(o.inner_u(ah, bh, shape) - N * np.sum(a * b)) < 1e-10 * N
    shape_odd = (5, 3, 7)
    a = RNG.standard_normal((3,) + shape_odd)
    ah = np.fft.rfftn(a, axes=(-3, -2, -1))
    assert abs(o.inner_u(ah, ah, shape_odd) - np.prod(shape_odd) * np.sum(a * a)) < 1e-9


# ---------------------------------------------------------------- operator (R2)
@pytest.mark.parametrize("kind", ["small", "finite"])
def test_plane_wave_closed_form(kind):
    """Homogeneous C, u-hat = a at one frequency: K u = (1/N) Q(xi) a, zero elsewhere."""
    shape = (8, 8, 8)
    prob = o.Problem(shape, kind)
    lam0, mu0 = 2.0, 1.5
    T = o.IsoTangent(np.full(shape, lam0), np.full(shape, mu0))
    u = np.zeros((3, 8, 8, 5), complex)
    a = np.array([1 + 2j, -0.5j, 0.3])
    u[:, 1, 6, 3] = a  # k = (1, -2, 3)
    q, _ = prob.apply_K(T, u, np.zeros(0))
    xi = 2 * np.pi * np.array([1.0, -2.0, 3.0])
    if kind == "small":
        Q = mu0 * (xi @ xi) * np.eye(3) + (lam0 + mu0) * np.outer(xi, xi)
    else:  # gradient (not symmetrised) through the same isotropic C
        Q = mu0 * (xi @ xi) * np.eye(3) + (lam0 + mu0) * np.outer(xi, xi)
    assert np.abs(q[:, 1, 6, 3] - Q @ a / 512).max() < 1e-15 * np.abs(Q).max()
    q[:, 1, 6, 3] = 0
    assert np.abs(q).max() < 1e-15


def test_cosine_modulated_stiffness_three_modes():
    """mu(x) = mu0 + mu1 cos(2 pi x1): a shear plane wave couples to k1 +- 1 only."""
    shape = (8, 8, 8)
    prob = o.Problem(shape)
    x1 = (np.arange(8) + 0.5) / 8
    mu0, mu1 = 1.0, 0.4
    mu = np.broadcast_to((mu0 + mu1 * np.cos(2 * np.pi * x1))[:, None, None], shape)
    T = o.IsoTangent(np.zeros(shape), mu)
    u = np.zeros((3, 8, 8, 5), complex)
    u[2, 2, 0, 0] = 1.0  # u3 e^{i 2pi 2 x1}: eps_13 = 1/2 i xi1 u3
    u[2, 6, 0, 0] = 1.0  # Hermitian partner on the k3 = 0 plane
    q, _ = prob.apply_K(T, u, np.zeros(0))
    N = 512
    # sigma_13 = 2 mu(x) eps_13 with cos(2 pi x1) sampled at voxel centres
    # (i + 1/2)/8: mode k1 picks up the phase e^{i pi (k1 - 2)/8}, and
    # q_3(k1) = -(1/N) i xi_1 sigma-hat_31 = xi(k1) xi(2) coef phase / N.
    for k1, coef in [(2, mu0), (1, mu1 / 2), (3, mu1 / 2)]:
        phase = np.exp(1j * np.pi * (k1 - 2) / 8)
        expect = (2 * np.pi * k1) * (2 * np.pi * 2) * coef * phase / N
        assert abs(q[2, k1, 0, 0] - expect) < 1e-13
    mask = np.ones((8, 8, 5), bool)
    mask[[1, 2, 3, 5, 6, 7], 0, 0] = False
    assert np.abs(q[:, mask]).max() < 1e-13
    assert np.abs(q[:2]).max() < 1e-13


@pytest.mark.parametrize("kind,mask", [("small", None), ("small", [1, 0, 0, 0, 0, 0, 0, 0, 1]),
                                       ("finite", None), ("finite", [0, 1, 1, 0, 1, 1, 0, 0, 1])])
def test_operator_is_hermitian(kind, mask):
    shape = (6, 4, 8)
    prob = o.Problem(shape, kind, mask)
    if kind == "small":
        T = _iso_random(shape, 3)
    else:
        g = np.random.default_rng(4)
        F = np.eye(3)[:, :, None, None, None] + 0.1 * g.standard_normal((3, 3) + shape)
        P, K = o.neo_hooke(F, np.where(g.random(shape) < 0.5, 1.0, 20.0), 1.5)
        T = o.FullTangent(K)
    v = (synth.random_spectrum(shape, 3, 10)[0], RNG.standard_normal(prob.ne))
    w = (synth.random_spectrum(shape, 3, 11)[0], RNG.standard_normal(prob.ne))
    v[0][:, prob.Z] = 0
    w[0][:, prob.Z] = 0
    Kv = prob.apply_K(T, *v)
    Kw = prob.apply_K(T, *w)
    a, b = prob.dot(v, Kw), prob.dot(Kv, w)
    assert abs(a - b) < 1e-13 * abs(a)
    assert prob.dot(v, Kv) > 0
    assert np.abs(Kv[0][:, prob.Z]).max() == 0.0


def _dense_matrix(prob, T):
    """Matrix of K in the basis of real unit displacement fields (3N of them)."""
    shape = prob.shape
    N = prob.N
    cols = []
    for c in range(3):
        for idx in range(N):
            f = np.zeros((3, N))
            f[c, idx] = 1.0
            cols.append(np.fft.rfftn(f.reshape((3,) + shape), axes=(-3, -2, -1)))
    Kc = [prob.apply_K(T, col, np.zeros(0))[0] for col in cols]
    A = np.array([[o.inner_u(cols[a], Kc[b], shape) for b in range(3 * N)] for a in range(3 * N)])
    return A, cols


@pytest.mark.parametrize("shape,nzero", [((4, 4, 4), 24), ((5, 5, 5), 3)])
def test_dense_operator_symmetric_full_rank_off_null_set(shape, nzero):
    """Brute force: K is symmetric, its null space is exactly the Z modes (Sec. 2.2)."""
    prob = o.Problem(shape)
    T = _iso_random(shape, 7, contrast=30.0)
    A, cols = _dense_matrix(prob, T)
    assert np.abs(A - A.T).max() < 1e-13 * np.abs(A).max()
    ev = np.linalg.eigvalsh(A)
    tiny = np.abs(ev) < 1e-10 * ev.max()
    assert tiny.sum() == nzero
    assert ev[~tiny].min() > 0
    # the null vectors are the real fields whose spectrum lies on Z
    N = prob.N
    Zmode = []
    for c in range(3):
        for k in np.argwhere(prob.Z):
            spec = np.zeros((3,) + prob.Z.shape, complex)
            spec[(c,) + tuple(k)] = 1.0
            fld = np.fft.irfftn(spec, s=shape, axes=(-3, -2, -1))
            Zmode.append(fld.reshape(-1))
    Zm = np.array(Zmode).T
    assert np.abs(A @ Zm).max() < 1e-10 * np.abs(A).max()
    # dense solve of the RHS equals PCG to 1e-12
    eps_bar = np.array([[1e-3, 2e-4, 0], [2e-4, -5e-4, 1e-4], [0, 1e-4, 3e-4]])
    b = o.linear_rhs(prob, T, eps_bar)
    bv = np.array([o.inner_u(col, b[0], shape) for col in cols])
    y = np.linalg.lstsq(A, bv, rcond=1e-10)[0]
    u_dense = np.fft.rfftn(y.reshape((3,) + shape), axes=(-3, -2, -1))
    u_dense[:, prob.Z] = 0
    sol = o.solve_linear(prob, T, eps_bar, tol=1e-14)
    assert np.abs(sol["u"] - u_dense).max() < 1e-10 * np.abs(u_dense).max()


# ---------------------------------------------------------------- preconditioner (R4)
@pytest.mark.parametrize("mask", [None, [1, 0, 1, 0, 1, 0, 1, 0, 0], [1] * 9])
def test_preconditioner_exact_for_homogeneous_medium(mask):
    shape = (8, 6, 4)
    prob = o.Problem(shape, "small", mask)
    T = o.IsoTangent(np.full(shape, 1.7), np.full(shape, 0.9))
    b = (synth.random_spectrum(shape, 3, 5)[0], RNG.standard_normal(prob.ne))
    b[0][:, prob.Z] = 0
    M = prob.make_preconditioner(T.mean())
    x, it, hist = o.pcg(prob, lambda v: prob.apply_K(T, *v), M, b, 1e-13, 50)
    assert it == 1


def test_homogeneous_medium_is_affine_with_zero_iterations():
    shape = (8, 8, 8)
    prob = o.Problem(shape)
    lam, mu = o.lame(np.full(shape, 3.0), np.full(shape, 0.25))
    T = o.IsoTangent(lam, mu)
    eps = np.array([[1e-3, 0, 2e-4], [0, 0, 0], [2e-4, 0, -1e-3]])
    sol = o.solve_linear(prob, T, eps)
    assert sol["iters"] == 0
    assert np.abs(sol["u"]).max() == 0
    C = o.iso_stiffness(lam.flat[0], mu.flat[0])
    assert np.abs(sol["sig_bar"] - np.einsum("ijkl,kl->ij", C, eps)).max() < 1e-15


# ---------------------------------------------------------------- finite-strain crystal plasticity (R18)
def _fcp_setup(gdot0=1e-3):
    rng = synth.Xoshiro256ss(71)
    quats = synth.uniform_quaternions(3, rng)
    cp = o.CrystalPlasticity(quats, gdot0=gdot0)
    return cp, o.schmid_full(cp, quats), np.array([0, 1, 2, 0, 1, 2])


def test_finite_cp_elastic_limit_is_st_venant_kirchhoff_with_cubic_stiffness():
    """No slip (gdot0 = 0): P = F (C : E), E = (F^T F - I)/2, with the rotated cubic C."""
    cp, S, g = _fcp_setup(gdot0=0.0)
    F = np.eye(3) + 0.05 * np.random.default_rng(2).standard_normal((6, 3, 3))
    P, Fp, T, _ = o.finite_cp_update(cp, S, g, F, np.broadcast_to(np.eye(3), (6, 3, 3)).copy(), np.zeros((6, 6)), 0.5)
    E = 0.5 * (np.swapaxes(F, 1, 2) @ F - np.eye(3))
    Cg = np.array([o.mandel_to_tensor4(cp.C[k]) for k in g])
    ref = F @ np.einsum("vijkl,vkl->vij", Cg, E)
    assert np.abs(P - ref).max() < 1e-10 * np.abs(ref).max()
    assert np.abs(Fp - np.eye(3)).max() == 0.0


def test_finite_cp_rotation_objectivity_and_rigid_rotation():
    cp, S, g = _fcp_setup()
    r = np.random.default_rng(3)
    F = np.eye(3) + 3e-3 * r.standard_normal((6, 3, 3))
    Fp0 = np.eye(3) + 1e-3 * r.standard_normal((6, 3, 3))
    Q = o.quat_to_rot(np.array([0.8, 0.1, -0.5, 0.3]) / np.linalg.norm([0.8, 0.1, -0.5, 0.3]))
    P1, Fp1, _, _ = o.finite_cp_update(cp, S, g, F, Fp0, np.zeros((6, 6)), 0.5)
    P2, Fp2, _, _ = o.finite_cp_update(cp, S, g, Q @ F, Fp0, np.zeros((6, 6)), 0.5)
    assert np.abs(P2 - Q @ P1).max() < 1e-9 * np.abs(P1).max()
    assert np.abs(Fp2 - Fp1).max() < 1e-12
    P3, _, _, _ = o.finite_cp_update(cp, S, g, np.broadcast_to(Q, (6, 3, 3)).copy(),
                                     np.broadcast_to(np.eye(3), (6, 3, 3)).copy(), np.zeros((6, 6)), 0.5)
    assert np.abs(P3).max() < 1e-9


def test_finite_cp_small_deformation_limit_is_the_small_strain_model():
    """F = I + eps (symmetric), Fp = I: P agrees with the small-strain stress to O(|eps|)."""
    cp, S, g = _fcp_setup()
    r = np.random.default_rng(4)
    base = r.standard_normal((6, 3, 3))
    base = 0.5 * (base + np.swapaxes(base, 1, 2))
    errs = []
    for amp in (2e-3, 2e-4):
        eps = amp * base / np.abs(base).max()
        P, _, _, _ = o.finite_cp_update(cp, S, g, np.eye(3) + eps, np.broadcast_to(np.eye(3), (6, 3, 3)).copy(),
                                        np.zeros((6, 6)), 0.5)
        sig, _, _, _ = cp.update(g, np.einsum("mij,vij->vm", o.mandel_basis(), eps), np.zeros((6, 6)),
                                 np.zeros((6, 6)), 0.5)
        sm = np.einsum("mij,vm->vij", o.mandel_basis(), sig)
        errs.append(np.abs(P - sm).max() / np.abs(sm).max())
    assert errs[0] < 10 * 2e-3 and errs[1] < 10 * 2e-4 and errs[1] < errs[0]


def test_finite_cp_tangent_is_the_derivative_with_the_plastic_state_held():
    """K : G against central differences of F a T(E(F)) a^T (a = Fp_old^-1 fixed)."""
    cp, S, g = _fcp_setup()
    r = np.random.default_rng(5)
    F = np.eye(3) + 3e-3 * r.standard_normal((6, 3, 3))
    Fp0 = np.eye(3) + 1e-3 * r.standard_normal((6, 3, 3))
    _, _, T0, data = o.finite_cp_update(cp, S, g, F, Fp0, np.zeros((6, 6)), 0.5)
    K = np.moveaxis(o.finite_cp_tangent(data), -1, 0)
    G = r.standard_normal((6, 3, 3))
    h = 1e-7

    def ptilde(Fx):
        _, _, T, data_x = o.finite_cp_update(cp, S, g, Fx, Fp0, T0, 0.5)
        Fe_tr, a = data_x[0], data_x[1]
        return Fe_tr @ np.einsum("mij,vm->vij", o.mandel_basis(), T) @ np.swapaxes(a, 1, 2)

    fd = (ptilde(F + h * G) - ptilde(F - h * G)) / (2 * h)
    kg = np.einsum("viJkL,vkL->viJ", K, G)
    assert np.abs(kg - fd).max() < 1e-5 * np.abs(kg).max()
    Kv = K.reshape(6, 9, 9)
    assert np.abs(Kv - np.swapaxes(Kv, 1, 2)).max() < 1e-12 * np.abs(Kv).max()


def test_finite_cp_single_crystal_steady_state():
    """[100] stretch of a cube-oriented crystal at F11 rate 1e-3/s (other P components
    free, rotation fixed as in R8): once the flow is steady, eight systems at Schmid
    factor 1/sqrt 6 carry the true strain rate D = rate / F11, so the Cauchy stress is
    sqrt 6 tau_c (sqrt 6 D / (8 gdot0))^m times (Fe_11)^2 ~ 1 + 2 sigma / E_100, and
    P11 = J sigma11 / F11. Without the update of Fp the stress would keep growing."""
    shape = (4, 4, 4)
    quats = np.array([[1.0, 0, 0, 0]])
    cp = o.CrystalPlasticity(quats)
    grain = np.zeros(shape, np.int64)
    mask = np.zeros((3, 3), bool)
    mask[0, 1] = mask[0, 2] = mask[1, 2] = mask[1, 1] = mask[2, 2] = True
    prob = o.Problem(shape, "finite", mask.reshape(-1))
    dt, n = 0.5, 40
    targets = []
    for k in range(n):
        t = np.eye(3)
        t[0, 0] = 1.0 + 1e-3 * dt * (k + 1)
        t[mask] = 0.0
        targets.append(t)
    res, _ = o.newton_increments(prob, o.finite_cp_material(cp, quats, grain, dt), targets, newton_tol=1e-10,
                                 load_tol=1e-10)
    F = res[-1]["field_bar"]
    F11, J = F[0, 0], float(np.linalg.det(F))
    sig = math.sqrt(6) * 50.0 * (math.sqrt(6) * 1e-3 / F11 / (8 * 1e-3)) ** 0.05
    C11, C12 = 168000.0, 121000.0
    E100 = (C11 - C12) * (C11 + 2 * C12) / (C11 + C12)
    pred = J * sig * (1.0 + 2.0 * sig / E100) / F11
    assert abs(res[-1]["stress_bar"][0, 0] - pred) < 1e-3 * pred
    assert abs(F[1, 1] - F[2, 2]) < 1e-10 and F[1, 1] < 1.0


# ---------------------------------------------------------------- displacement (Eqs. disp_decomp, decomp_displ)
def test_displacement_of_an_affine_state_sits_at_voxel_centres():
    """u~ = 0: u = Hbar x at x = (j + 1/2) L / n. A non-symmetric Fbar - I (finite
    strain) catches a transposed Hbar; a stress-controlled shear (small strain)
    checks the macro unknown's Mandel basis element (e_i e_j + e_j e_i)/sqrt 2."""
    shape, L = (4, 6, 8), (1.0, 2.0, 0.5)
    h = np.array(L) / np.array(shape)
    mask = np.zeros((3, 3), bool)
    mask[0, 2] = mask[2, 0] = True
    prob = o.Problem(shape, "small", mask.reshape(-1), L=L)
    fU = np.array([[1e-3, 2e-4, 0.0], [2e-4, -5e-4, 0.0], [0.0, 0.0, 3e-4]])
    e = np.array([math.sqrt(2.0) * 7e-4])  # the 13 shear = 7e-4
    macro = o.macro_field(prob, fU, e)
    u = o.displacement(prob, prob.zeros()[0], macro)
    H = fU.copy()
    H[0, 2] = H[2, 0] = 7e-4
    for j in [(0, 0, 0), (3, 5, 7), (1, 4, 2)]:
        x = (np.array(j) + 0.5) * h
        assert np.allclose(u[(slice(None),) + j], H @ x, rtol=0, atol=1e-18)
    # finite strain: u_1(j2 + 1) - u_1(j2) = (F - I)_12 h_2, not (F - I)_21 h_2
    probf = o.Problem(shape, "finite", L=L)
    F = np.eye(3) + np.array([[0.1, 0.3, 0.0], [-0.2, 0.0, 0.05], [0.0, 0.0, -0.1]])
    uf = o.displacement(probf, probf.zeros()[0], o.macro_field(probf, F, np.zeros(0)))
    assert abs((uf[0, 0, 1, 0] - uf[0, 0, 0, 0]) - 0.3 * h[1]) < 1e-15
    assert abs((uf[1, 1, 0, 0] - uf[1, 0, 0, 0]) - (-0.2) * h[0]) < 1e-15
    assert np.allclose(uf[:, 0, 0, 0], (F - np.eye(3)) @ (0.5 * h), rtol=0, atol=1e-16)


def test_displacement_of_one_fourier_mode_closed_form():
    """One stored mode k = (1, 2, 3) off the k3 = 0, n3/2 planes: u~_c(j) =
    (2/N) Re(u_c e^{2 pi i k.j/n}) (it and its conjugate partner)."""
    shape = (4, 6, 8)
    prob = o.Problem(shape, "small")
    uh = prob.zeros()[0]
    a = np.array([0.3 - 0.7j, -1.1 + 0.2j, 0.5 + 0.5j])
    uh[:, 1, 2, 3] = a
    u = o.displacement(prob, uh, np.zeros((3, 3)))
    j1, j2, j3 = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    th = 2 * np.pi * (1 * j1 / 4 + 2 * j2 / 6 + 3 * j3 / 8)
    N = prob.N
    for c in range(3):
        ref = (2.0 / N) * (a[c].real * np.cos(th) - a[c].imag * np.sin(th))
        assert np.abs(u[c] - ref).max() < 1e-15


# ---------------------------------------------------------------- compatibility (Eq. chedckcomp)
def test_compatibility_of_a_gradient_vanishes_and_of_a_shear_wave_is_closed_form():
    """A symmetric gradient is compatible (0 up to round-off). eps = a sin(2 pi x2) e1 e1
    (not a gradient) gives eta_33 = -d2 d2 eps_11 = (2 pi)^2 a sin(2 pi x2): max (2 pi)^2 a,
    RMS (2 pi)^2 a / sqrt 2. For finite strain F = I + b sin(2 pi x2) e1 e1:
    (curl F)_13 = -d2 F_11, max 2 pi b."""
    shape = (8, 16, 8)
    prob = o.Problem(shape, "small")
    u = synth.random_spectrum(shape, 3, 5)[0]
    mx, rms = o.compatibility(prob, o.sym_grad_hat(u, prob.xi), 1.0)
    scale = np.abs(o.to_real(o.sym_grad_hat(u, prob.xi), shape)).max() * (2 * np.pi * 8) ** 2
    assert mx < 1e-13 * scale and rms < 1e-13 * scale
    a = 1e-3
    x2 = (np.arange(16) + 0.5) / 16
    eps = np.zeros((3, 3) + shape)
    eps[0, 0] = a * np.sin(2 * np.pi * x2)[None, :, None]
    mx, rms = o.compatibility(prob, o.to_fourier(eps), 1.0)
    assert abs(mx - (2 * np.pi) ** 2 * a * np.abs(np.sin(2 * np.pi * x2)).max()) < 1e-12
    assert abs(rms - (2 * np.pi) ** 2 * a / math.sqrt(2.0)) < 1e-12
    probf = o.Problem(shape, "finite")
    G = np.zeros((3, 3) + shape)
    G[0, 0] = 0.2 * np.sin(2 * np.pi * x2)[None, :, None]
    mx, _ = o.compatibility(probf, o.to_fourier(G), 1.0)
    assert abs(mx - 2 * np.pi * 0.2 * np.abs(np.cos(2 * np.pi * x2)).max()) < 1e-12


# ---------------------------------------------------------------- laminates (closed forms)
def _laminate(shape, widths, lam_p, mu_p):
    ph = np.zeros(shape[0], int)
    ph[widths[0]:] = 1
    lam = np.broadcast_to(np.array(lam_p)[ph][:, None, None], shape).copy()
    mu = np.broadcast_to(np.array(mu_p)[ph][:, None, None], shape).copy()
    f = np.array([widths[0], shape[0] - widths[0]]) / shape[0]
    return o.IsoTangent(lam, mu), f


def _laminate_closed_form(f, lam_p, mu_p, eps):
    """Layer strains eps_p = eps + sym(a_p x n), n = e1, continuous traction."""
    n = np.array([1.0, 0, 0])
    Cs = [o.iso_stiffness(l, m) for l, m in zip(lam_p, mu_p)]
    A = [np.einsum("j,ijkl,l->ik", n, C, n) for C in Cs]
    rhs = [np.einsum("ijkl,kl,j->i", C, eps, n) for C in Cs]
    S = sum(fp * np.linalg.inv(Ap) for fp, Ap in zip(f, A))
    t = np.linalg.solve(S, sum(fp * np.linalg.inv(Ap) @ r for fp, Ap, r in zip(f, A, rhs)))
    sig_bar = np.zeros((3, 3))
    for fp, C, Ap, r in zip(f, Cs, A, rhs):
        a = np.linalg.solve(Ap, t - r)
        e = eps + 0.5 * (np.outer(a, n) + np.outer(n, a))
        sig_bar += fp * np.einsum("ijkl,kl->ij", C, e)
    return sig_bar


def test_laminate_reuss_voigt_special_cases():
    shape = (16, 4, 4)
    lam_p, mu_p = [1.0, 30.0], [0.8, 25.0]
    T, f = _laminate(shape, (6, 10), lam_p, mu_p)
    prob = o.Problem(shape)
    mu, lm = np.array(mu_p), np.array(lam_p)
    # shear eps_12 -> Reuss mean of mu; eps_23 -> Voigt mean of mu;
    # uniaxial strain eps_11 -> Reuss mean of lam + 2 mu
    for eps_ij, expect in [((0, 1), 1.0 / np.sum(f / mu)), ((1, 2), np.sum(f * mu)),
                           ((0, 0), 1.0 / np.sum(f / (lm + 2 * mu)))]:
        eps = np.zeros((3, 3))
        i, j = eps_ij
        eps[i, j] = eps[j, i] = 1e-3
        sol = o.solve_linear(prob, T, eps, tol=1e-14)
        factor = 1.0 if i == j else 2.0
        assert abs(sol["sig_bar"][i, j] - factor * expect * 1e-3) < 1e-12 * factor * expect * 1e-3
    eps = np.array([[1e-3, 3e-4, -2e-4], [3e-4, 5e-4, 1e-4], [-2e-4, 1e-4, -7e-4]])
    sol = o.solve_linear(prob, T, eps, tol=1e-14)
    ref = _laminate_closed_form(f, lam_p, mu_p, eps)
    assert np.abs(sol["sig_bar"] - ref).max() < 1e-12 * np.abs(ref).max()


def test_laminate_stress_control():
    """Prescribed sigma_11 with the other strains zero: eps_11 = s / Reuss(lam + 2 mu)."""
    shape = (8, 4, 4)
    lam_p, mu_p = [2.0, 12.0], [1.0, 9.0]
    T, f = _laminate(shape, (4, 4), lam_p, mu_p)
    mask = np.zeros(9, bool)
    mask[0] = True
    prob = o.Problem(shape, "small", mask)
    target = np.zeros((3, 3))
    target[0, 0] = 0.7
    sol = o.solve_linear(prob, T, target, tol=1e-14)
    MR = 1.0 / np.sum(f / (np.array(lam_p) + 2 * np.array(mu_p)))
    assert abs(sol["e"][0] - 0.7 / MR) < 1e-12
    assert abs(sol["sig_bar"][0, 0] - 0.7) < 1e-12


def test_mixed_control_matches_inverted_strain_control():
    """Stress control is the inverse of strain control on the same microstructure."""
    shape = (8, 8, 8)
    T = _iso_random(shape, 21)
    eps = np.array([[1e-3, 1e-4, 0], [1e-4, -3e-4, 2e-4], [0, 2e-4, 5e-4]])
    ref = o.solve_linear(o.Problem(shape), T, eps, tol=1e-14)
    mask = np.zeros((3, 3), bool)
    mask[1, 1] = mask[0, 2] = mask[2, 0] = mask[1, 2] = mask[2, 1] = True
    target = eps.copy()
    target[mask] = ref["sig_bar"][mask]
    sol = o.solve_linear(o.Problem(shape, "small", mask.reshape(-1)), T, target, tol=1e-14)
    assert np.abs(sol["eps"].reshape(3, 3, -1).mean(-1) - eps).max() < 1e-12
    assert np.abs(sol["sig_bar"] - ref["sig_bar"]).max() < 1e-12 * np.abs(ref["sig_bar"]).max()


def test_hill_mandel_and_voigt_reuss_bounds():
    shape = (8, 8, 8)
    T = _iso_random(shape, 2, contrast=20.0)
    Ceff, _ = o.homogenized_tangent(shape, T, tol=1e-13)
    assert np.abs(Ceff - Ceff.T).max() < 1e-10 * np.abs(Ceff).max()
    B = o.mandel_basis()
    Cv = np.zeros((6, 6))
    Sr = np.zeros((6, 6))
    lam, mu = T.lam.reshape(-1), T.mu.reshape(-1)
    for l, m in zip(lam, mu):
        Cm = o.tensor4_to_mandel(o.iso_stiffness(l, m))
        Cv += Cm / lam.size
        Sr += np.linalg.inv(Cm) / lam.size
    Cr = np.linalg.inv(Sr)
    assert np.linalg.eigvalsh(Cv - Ceff).min() > -1e-10
    assert np.linalg.eigvalsh(Ceff - Cr).min() > -1e-10
    # Hill-Mandel: eps_bar : sigma_bar = <eps : sigma>
    prob = o.Problem(shape)
    eps = 1e-3 * (B[0] + 0.5 * B[3])
    sol = o.solve_linear(prob, T, eps, tol=1e-13)
    lhs = np.sum(eps * sol["sig_bar"])
    rhs = np.mean(np.einsum("ij...,ij...->...", sol["eps"], sol["sig"]))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def test_config1_invariants():
    c = synth.config1()
    lam, mu = o.lame(c["E"][c["phase"]], c["nu"][c["phase"]])
    T = o.IsoTangent(lam, mu)
    prob = o.Problem((16, 16, 16))
    sol = o.solve_linear(prob, T, c["eps_bar"], tol=1e-10)
    assert sol["true_rel"] <= 1e-10
    # loading residual (Eq. chedckimp) and compatibility (zero by construction)
    assert np.abs(sol["eps"].reshape(3, 3, -1).mean(-1) - c["eps_bar"]).max() < 1e-18
    lam_m, mu_m = o.lame(1.0, 0.3)
    lam_i, mu_i = o.lame(10.0, 0.3)
    # between the uniaxial-strain moduli of the pure matrix and pure inclusion
    assert (lam_m + 2 * mu_m) * 1e-3 < sol["sig_bar"][0, 0] < (lam_i + 2 * mu_i) * 1e-3


def test_centred_inclusion_gives_a_cubic_effective_stiffness():
    """The 16^3 centred sphere is unchanged by the 48 symmetries of the cube, and so is the
    discrete operator on an equal-sided even grid (a mirror sends k to -k; an integer shift of
    voxels is exact). C_eff must therefore be cubic. Axis 3 is built apart from axes 1-2 (it is
    cut to a half spectrum), so a frequency slip on it alone (a 1 % wrong length moves C33 off
    C11 by 6e-4) fails here, and so does a wrong factor on one Mandel shear component."""
    c = synth.config1()
    p = c["phase"]
    assert all(np.array_equal(p, np.flip(p, a)) for a in range(3))
    assert np.array_equal(p, p.transpose(1, 0, 2)) and np.array_equal(p, p.transpose(2, 1, 0))
    lam, mu = o.lame(c["E"][p], c["nu"][p])
    Ceff, _ = o.homogenized_tangent(p.shape, o.IsoTangent(lam, mu), tol=1e-13)
    tol = 1e-9 * np.abs(Ceff).max()
    d = np.diag(Ceff)
    assert np.ptp(d[:3]) < tol and np.ptp(d[3:]) < tol
    assert np.ptp([Ceff[0, 1], Ceff[0, 2], Ceff[1, 2]]) < tol
    assert np.abs(Ceff[:3, 3:]).max() < tol and np.abs(Ceff[3:, :3]).max() < tol
    assert np.abs(Ceff[3:, 3:] - np.diag(d[3:])).max() < tol
    # stiffer than the matrix, softer than the inclusion, and not isotropic to round-off
    lam_m, mu_m = o.lame(1.0, 0.3)
    assert lam_m + 2 * mu_m < d[0] < 10 * (lam_m + 2 * mu_m)
    assert 2 * mu_m < d[3] < 20 * mu_m
    assert abs((d[0] - Ceff[0, 1]) - d[3]) > 1e3 * tol


# ---------------------------------------------------------------- Neo-Hooke (R13)
def test_neo_hooke_stress_and_tangent_by_finite_differences():
    g = np.random.default_rng(5)
    F = np.eye(3) + 0.2 * g.standard_normal((3, 3))
    mu, lam = 1.3, 2.1
    P, K = o.neo_hooke(F, mu, lam)
    h = 1e-6
    for k in range(3):
        for l in range(3):
            dF = np.zeros((3, 3))
            dF[k, l] = h
            dW = (o.neo_hooke_energy(F + dF, mu, lam) - o.neo_hooke_energy(F - dF, mu, lam)) / (2 * h)
            assert abs(dW - P[k, l]) < 1e-8
            dP = (o.neo_hooke(F + dF, mu, lam)[0] - o.neo_hooke(F - dF, mu, lam)[0]) / (2 * h)
            assert np.abs(dP - K[:, :, k, l]).max() < 1e-7
    # objectivity P(QF) = Q P(F)
    Q = o.quat_to_rot(np.array([0.8, 0.2, -0.5, 0.1]) / np.linalg.norm([0.8, 0.2, -0.5, 0.1]))
    assert np.abs(o.neo_hooke(Q @ F, mu, lam)[0] - Q @ P).max() < 1e-13
    # K(I) is the isotropic elasticity tensor with the same Lame constants
    _, K0 = o.neo_hooke(np.eye(3), mu, lam)
    assert np.abs(K0 - o.iso_stiffness(lam, mu)).max() < 1e-14


def test_svk_stress_and_tangent_by_finite_differences():
    g = np.random.default_rng(6)
    F = np.eye(3) + 0.25 * g.standard_normal((3, 3))
    mu, lam = 0.9, 1.7
    P, K = o.svk(F, mu, lam)
    h = 1e-6
    for k in range(3):
        for l in range(3):
            dF = np.zeros((3, 3))
            dF[k, l] = h
            dW = (o.svk_energy(F + dF, mu, lam) - o.svk_energy(F - dF, mu, lam)) / (2 * h)
            assert abs(dW - P[k, l]) < 1e-8
            dP = (o.svk(F + dF, mu, lam)[0] - o.svk(F - dF, mu, lam)[0]) / (2 * h)
            assert np.abs(dP - K[:, :, k, l]).max() < 1e-7
    # major symmetry, objectivity, and the small-strain limit
    assert np.abs(K - np.transpose(K, (2, 3, 0, 1))).max() < 1e-13
    Q = o.quat_to_rot(np.array([0.3, -0.6, 0.2, 0.7]) / np.linalg.norm([0.3, -0.6, 0.2, 0.7]))
    assert np.abs(o.svk(Q @ F, mu, lam)[0] - Q @ P).max() < 1e-13
    _, K0 = o.svk(np.eye(3), mu, lam)
    assert np.abs(K0 - o.iso_stiffness(lam, mu)).max() < 1e-14


def _laminate_finite_reference(f, mu_p, lam_p, Fbar, mask_stress=None, law=None):
    """Rank-one laminate: F_p = Fbar + a_p x e1, P_p e1 = t, sum f_p a_p = 0 (Newton)."""
    law = o.neo_hooke if law is None else law
    n = np.array([1.0, 0, 0])
    a = np.zeros((2, 3))
    for _ in range(50):
        Fs = [Fbar + np.outer(a[p], n) for p in range(2)]
        PK = [law(Fs[p], mu_p[p], lam_p[p]) for p in range(2)]
        # unknowns a_0, a_1 (6); equations: P_0 n - P_1 n = 0 (3), f0 a0 + f1 a1 = 0 (3)
        R = np.concatenate([PK[0][0] @ n - PK[1][0] @ n, f[0] * a[0] + f[1] * a[1]])
        A = [np.einsum("j,ijkl,l->ik", n, PK[p][1], n) for p in range(2)]
        J = np.zeros((6, 6))
        J[:3, :3], J[:3, 3:] = A[0], -A[1]
        J[3:, :3], J[3:, 3:] = f[0] * np.eye(3), f[1] * np.eye(3)
        d = np.linalg.solve(J, -R)
        a = a + d.reshape(2, 3)
        if np.abs(d).max() < 1e-15:
            break
    Fs = [Fbar + np.outer(a[p], n) for p in range(2)]
    return sum(f[p] * law(Fs[p], mu_p[p], lam_p[p])[0] for p in range(2))


def test_finite_strain_laminate_against_rank_one_solution():
    shape = (8, 4, 4)
    mu_p, lam_p = [1.0, 20.0], [1.5, 30.0]
    ph = (np.arange(8) >= 2).astype(int)
    mu = np.broadcast_to(np.array(mu_p)[ph][:, None, None], shape)
    lam = np.broadcast_to(np.array(lam_p)[ph][:, None, None], shape)
    f = np.array([2, 6]) / 8.0
    prob = o.Problem(shape, "finite")
    Fbar = np.array([[1.1, 0.05, 0.0], [0.02, 0.97, 0.03], [0.0, -0.04, 1.02]])
    targets = [np.eye(3) + (Fbar - np.eye(3)) * (k + 1) / 3 for k in range(3)]
    res, _ = o.newton_increments(prob, o.neo_hooke_material(mu, lam), targets,
                                 newton_tol=1e-12, load_tol=1e-12, eta=1e-6)
    ref = _laminate_finite_reference(f, mu_p, lam_p, Fbar)
    assert np.abs(res[-1]["stress_bar"] - ref).max() < 1e-11 * np.abs(ref).max()


def test_finite_strain_laminate_svk_against_rank_one_solution():
    shape = (8, 4, 4)
    mu_p, lam_p = [1.0, 15.0], [1.5, 20.0]
    ph = (np.arange(8) >= 6).astype(int)  # even widths: the exact field has no Nyquist content
    mu = np.broadcast_to(np.array(mu_p)[ph][:, None, None], shape)
    lam = np.broadcast_to(np.array(lam_p)[ph][:, None, None], shape)
    f = np.array([6, 2]) / 8.0
    prob = o.Problem(shape, "finite")
    Fbar = np.array([[1.08, 0.04, 0.0], [0.01, 0.98, 0.02], [0.0, -0.03, 1.01]])
    targets = [np.eye(3) + (Fbar - np.eye(3)) * (k + 1) / 2 for k in range(2)]
    res, _ = o.newton_increments(prob, o.svk_material(mu, lam), targets,
                                 newton_tol=1e-12, load_tol=1e-12, eta=1e-6)
    ref = _laminate_finite_reference(f, mu_p, lam_p, Fbar, law=o.svk)
    assert np.abs(res[-1]["stress_bar"] - ref).max() < 1e-11 * np.abs(ref).max()


def test_finite_strain_mixed_control_homogeneous_uniaxial():
    """Homogeneous NH bar, F11 prescribed, lateral stresses zero: closed-form lateral stretch."""
    shape = (4, 4, 4)
    mu, lam = 1.0, 1.5
    mask = np.zeros((3, 3), bool)
    mask[0, 1] = mask[0, 2] = mask[1, 2] = mask[1, 1] = mask[2, 2] = True
    prob = o.Problem(shape, "finite", mask.reshape(-1))
    tgt = np.eye(3)
    tgt[0, 0] = 1.2
    tgt[mask] = 0.0
    res, _ = o.newton_increments(prob, o.neo_hooke_material(np.full(shape, mu), np.full(shape, lam)),
                                 [tgt], newton_tol=1e-13, load_tol=1e-13)
    Fb = res[-1]["field_bar"]
    # lateral stretch s solves P22 = mu (s - 1/s) + lam ln(1.2 s^2) / s = 0
    s = 1.0
    for _ in range(50):
        r = mu * (s - 1 / s) + lam * math.log(1.2 * s * s) / s
        dr = mu * (1 + 1 / s ** 2) + lam * (2 - math.log(1.2 * s * s)) / s ** 2
        s -= r / dr
    assert abs(Fb[1, 1] - s) < 1e-12 and abs(Fb[2, 2] - s) < 1e-12
    assert abs(Fb[0, 1]) < 1e-13 and abs(Fb[1, 0]) < 1e-13


# ---------------------------------------------------------------- crystal plasticity (R14)
def test_cp_tangent_by_finite_differences_and_elastic_limit():
    q = np.array([[0.9, 0.1, -0.3, 0.2]])
    cp = o.CrystalPlasticity(q / np.linalg.norm(q))
    g = np.zeros(1, int)
    eps = np.array([[2.5e-3, -1e-3, -1e-3, 4e-4, 0, 1e-4]])
    ep0 = np.zeros((1, 6))
    sig, tan, ep, _ = cp.update(g, eps, ep0, np.zeros((1, 6)), 0.5)
    h = 1e-8
    for k in range(6):
        d = np.zeros((1, 6))
        d[0, k] = h
        sp = cp.update(g, eps + d, ep0, sig, 0.5)[0]
        sm = cp.update(g, eps - d, ep0, sig, 0.5)[0]
        assert np.abs((sp - sm) / (2 * h) - tan[0, :, k]).max() < 1e-5 * np.abs(tan).max()
    # tiny strain: stress is elastic
    e_small = 1e-7 * np.ones((1, 6))
    s_small = cp.update(g, e_small, ep0, np.zeros((1, 6)), 0.5)[0]
    assert np.abs(s_small - e_small @ cp.C[0].T).max() < 1e-9 * np.abs(s_small).max()


def test_cp_single_crystal_steady_state_closed_form():
    """[100] tension of a cube-oriented crystal at 1e-3/s: 8 systems at Schmid 1/sqrt(6).

    Steady flow gives sigma_ss = sqrt(6) tau_c (sqrt(6) epsdot / (8 gdot0))^m
    (about 115.44 MPa); backward Euler reproduces it exactly once steady.
    """
    shape = (4, 4, 4)
    cp = o.CrystalPlasticity(np.array([[1.0, 0, 0, 0]]))
    grain = np.zeros(shape, np.int64)
    mask = np.ones((3, 3), bool)
    mask[0, 0] = False
    prob = o.Problem(shape, "small", mask.reshape(-1))
    dt = 0.5
    targets = []
    for k in range(40):
        t = np.zeros((3, 3))
        t[0, 0] = 1e-3 * dt * (k + 1)
        targets.append(t)
    res, _ = o.newton_increments(prob, o.cp_material(cp, grain, dt), targets,
                                 newton_tol=1e-10, load_tol=1e-10)
    sig_ss = math.sqrt(6) * 50.0 * (math.sqrt(6) * 1e-3 / (8 * 1e-3)) ** 0.05
    golden = float(open(__file__.replace("test_oracle_pins.py", "golden/cp_steady_state.txt")).read().split()[0])
    assert abs(sig_ss - golden) < 1e-6
    assert abs(res[-1]["stress_bar"][0, 0] - sig_ss) < 1e-9 * sig_ss
    assert np.abs(res[-1]["x"][0]).max() < 1e-12  # homogeneous: no fluctuation


# ---------------------------------------------------------------- adjoint
def test_adjoint_euler_identity_and_finite_differences():
    shape = (8, 8, 8)
    g = np.random.default_rng(8)
    E = np.where(g.random(shape) < 0.3, 15.0, 1.0)
    nu = np.full(shape, 0.3)
    prob = o.Problem(shape)
    eps = np.zeros((3, 3))
    eps[0, 0] = 1e-3
    gJ = np.zeros((3, 3))
    gJ[0, 0] = 1.0
    dJ, J, _ = o.adjoint_dJ_dE(prob, E, nu, eps, gJ, tol=1e-14)
    # J is homogeneous of degree one in E at fixed nu: sum_x E dJ/dE = J
    assert abs(np.sum(E * dJ) - J) < 1e-11 * abs(J)
    assert dJ.min() > 0  # stiffening any voxel raises sigma_xx under eps_xx
    for v in [0, 77, 300]:
        idx = np.unravel_index(v, shape)
        d = 1e-3 * E[idx]
        Ep, Em = E.copy(), E.copy()
        Ep[idx] += d
        Em[idx] -= d
        Jp = o.homogenized_stress_linear(prob, Ep, nu, eps, tol=1e-14)[0, 0]
        Jm = o.homogenized_stress_linear(prob, Em, nu, eps, tol=1e-14)[0, 0]
        fd = (Jp - Jm) / (2 * d)
        assert abs(fd - dJ[idx]) < 1e-4 * abs(dJ[idx])
    # a general macro weight g (not proportional to the load)
    gJ2 = np.array([[0.3, 0.1, 0.0], [0.1, -0.7, 0.2], [0.0, 0.2, 0.5]])
    dJ2, J2, _ = o.adjoint_dJ_dE(prob, E, nu, eps, gJ2, tol=1e-14)
    assert abs(np.sum(E * dJ2) - J2) < 1e-10 * abs(J2)


def test_equilibrium_residual_of_a_single_mode_stress_closed_form():
    """Sec. 3, Eq. chedckeq: eps_eq = ||div sigma||_L2 / ||<sigma>||. For
    sigma(x) = S0 + A cos(2 pi k.x) (L = 1) the divergence is
    -2 pi sin(2 pi k.x) A k, so ||div sigma||_L2 = 2 pi |A k| / sqrt(2)."""
    shape = (8, 12, 10)
    prob = o.Problem(shape)
    k = np.array([1, -2, 3])
    x = np.stack(np.meshgrid(*[(np.arange(n) + 0.5) / n for n in shape], indexing="ij"))
    ph = 2 * np.pi * np.tensordot(k, x, axes=1)
    A = np.array([[0.3, -0.1, 0.2], [-0.1, 0.5, 0.05], [0.2, 0.05, -0.4]])
    S0 = np.array([[2.0, 0.1, 0.0], [0.1, -1.0, 0.3], [0.0, 0.3, 0.5]])
    sig = S0[:, :, None, None, None] + A[:, :, None, None, None] * np.cos(ph)[None, None]
    r = prob.adjoint(sig)
    got = o.equilibrium_residual(prob, r, sig.mean(axis=(2, 3, 4)))
    ref = 2 * np.pi * np.linalg.norm(A @ k) / np.sqrt(2) / np.linalg.norm(S0)
    assert abs(got - ref) < 1e-12 * ref


def test_effective_stiffness_sensitivity_laminate_closed_forms_and_euler_identity():
    """dC_IJ/dE(x) of the 6x6 Mandel effective stiffness (six unit strains, Sec. 2.2).
    Laminate with normal e1 (even layer widths): C_00 = Reuss mean of M = lam + 2 mu,
    C_33 = 2 x Voigt mean of mu, C_55 = 2 x Reuss mean of mu, so per voxel
    dC_00/dE = M_R^2 M1 / (N M^2), dC_33/dE = 2 mu1 / N, dC_55/dE = 2 mu_R^2 mu1 / (N mu^2),
    with M1 = M / E and mu1 = mu / E. The sensitivity of any J = G : C satisfies the
    Euler identity sum_x E dJ/dE = J (C is homogeneous of degree one in E)."""
    shape = (16, 4, 4)
    nu = 0.3
    E = np.ones(shape)
    E[6:] = 20.0  # layers of widths 6 and 10 along x1
    nuf = np.full(shape, nu)
    lam, mu = o.lame(E, nuf)
    M = lam + 2 * mu
    mu1, M1 = mu / E, M / E
    N = E.size
    muR, MR = 1.0 / np.mean(1.0 / mu), 1.0 / np.mean(1.0 / M)
    for (i, j), ref in [((0, 0), MR ** 2 * M1 / (N * M ** 2)), ((3, 3), 2 * mu1 / N),
                        ((5, 5), 2 * muR ** 2 * mu1 / (N * mu ** 2))]:
        G = np.zeros((6, 6))
        G[i, j] = 1.0
        dJ, J, C = o.effective_stiffness_sensitivity(shape, E, nuf, G, tol=1e-14)
        assert np.abs(dJ - ref).max() < 1e-10 * np.abs(ref).max(), (i, j)
        assert abs(np.sum(E * dJ) - J) < 1e-11 * abs(J)
    # a random microstructure and a general weight: Euler identity and a central difference
    shape = (8, 8, 8)
    g = np.random.default_rng(12)
    E = np.where(g.random(shape) < 0.35, 12.0, 1.0)
    nuf = np.full(shape, 0.25)
    G = g.standard_normal((6, 6))
    dJ, J, C = o.effective_stiffness_sensitivity(shape, E, nuf, G, tol=1e-14)
    assert abs(np.sum(E * dJ) - J) < 1e-10 * abs(J)
    idx = (3, 5, 1)
    d = 1e-3 * E[idx]
    Js = []
    for sgn in (1, -1):
        Ep = E.copy()
        Ep[idx] += sgn * d
        lam, mu = o.lame(Ep, nuf)
        Cp, _ = o.homogenized_tangent(shape, o.IsoTangent(lam, mu), tol=1e-14)
        Js.append(np.sum(G * Cp))
    fd = (Js[0] - Js[1]) / (2 * d)
    assert abs(fd - dJ[idx]) < 1e-5 * np.abs(dJ).max()


def _cp_adjoint_case(strain_per_inc, n_inc=4):
    shape = (8, 4, 4)
    rng = synth.Xoshiro256ss(4242)
    grains, _ = synth.periodic_voronoi(8, 5, rng)
    grains = grains[:, :4, :4].copy()
    cp = o.CrystalPlasticity(synth.uniform_quaternions(5, rng))
    mask = np.ones((3, 3), bool)
    mask[0, 0] = False  # uniaxial: eps_11 prescribed, the other macro stresses zero
    prob = o.Problem(shape, "small", mask.reshape(-1))
    targets = []
    for k in range(n_inc):
        t = np.zeros((3, 3))
        t[0, 0] = strain_per_inc * (k + 1)
        targets.append(t)
    return shape, grains, cp, prob, targets


def test_cp_adjoint_over_increments_matches_finite_differences():
    """Path-dependent adjoint (R14 crystal plasticity, Sec. 2.4 increments under mixed
    control): dJ/ds(x) for J = <sigma_11> after the last of four plastic increments,
    s(x) a factor on the stiffness of voxel x, against central differences of whole
    Newton runs (each voxel's stiffness perturbed by 1e-4)."""
    shape, grains, cp, prob, targets = _cp_adjoint_case(1e-3)
    dt = 0.5
    g = np.zeros((3, 3))
    g[0, 0] = 1.0
    dJ, J, recs = o.cp_adjoint_increments(prob, cp, grains, dt, targets, g)
    assert J > 120.0  # beyond the elastic limit: the history matters
    assert np.abs(recs[-1]["state"][0]).max() > 1e-4  # plastic strain

    def J_of(scale):
        r, _ = o.newton_increments(prob, o.cp_material(cp, grains, dt, scale=scale), targets, newton_tol=1e-12,
                                   load_tol=1e-12, eta=1e-10)
        return float(np.sum(g * r[-1]["stress_bar"]))

    for idx in [(0, 0, 0), (3, 2, 1), (7, 3, 3)]:
        d = 1e-4
        sp, sm = np.ones(shape), np.ones(shape)
        sp[idx] += d
        sm[idx] -= d
        fd = (J_of(sp) - J_of(sm)) / (2 * d)
        assert abs(fd - dJ[idx]) < 1e-6 * np.abs(dJ).max(), idx


def test_cp_adjoint_in_the_elastic_limit_satisfies_the_euler_identity():
    """With strains far below the elastic limit the response is linear in the stiffness
    factor: sum_x dJ/ds(x) = J."""
    shape, grains, cp, prob, targets = _cp_adjoint_case(1e-6, n_inc=2)
    g = np.array([[1.0, 0.2, 0.0], [0.2, -0.4, 0.1], [0.0, 0.1, 0.3]])
    dJ, J, _ = o.cp_adjoint_increments(prob, cp, grains, 0.5, targets, g)
    assert abs(dJ.sum() - J) < 1e-9 * abs(J)


def test_finite_cp_consistent_tangent_by_finite_differences():
    """The consistent tangent of the finite-strain crystal update with the plastic flow
    of the step active (dM = D : dT, M = I + sum_a dt gdot_a S_a): central differences of
    P(F) at a plastic state agree to 1e-7, where the tangent with the plastic state held
    (R18) is off by about 1e-2; the major asymmetry of the consistent tangent is small."""
    rng = synth.Xoshiro256ss(5)
    quats = synth.uniform_quaternions(3, rng)
    cp = o.CrystalPlasticity(quats)
    S_full = o.schmid_full(cp, quats)
    g = np.array([0, 1, 2])
    base = np.array([[4e-3, 1e-3, 0.0], [0.5e-3, -1e-3, 0.2e-3], [0.0, 0.3e-3, -1.5e-3]])
    F = np.eye(3)[None] + base[None] * np.array([1.0, 1.3, 0.7])[:, None, None]
    Fp_old = np.eye(3)[None].repeat(3, 0) + 1e-3 * np.array([[0.5, 0.2, 0.0], [0.1, -0.3, 0.0], [0.0, 0.1, -0.2]])
    dt = 0.5
    P, Fp, T, data = o.finite_cp_update(cp, S_full, g, F, Fp_old, np.zeros((3, 6)), dt)
    assert np.abs(Fp - Fp_old).max() > 1e-3  # the step flows plastically
    K = o.finite_cp_tangent_consistent(data, symmetric=False)
    Kh = o.finite_cp_tangent(data)
    h = 1e-7
    err = err_h = mx = 0.0
    for k in range(3):
        for L in range(3):
            Fa, Fb = F.copy(), F.copy()
            Fa[:, k, L] += h
            Fb[:, k, L] -= h
            fd = (o.finite_cp_update(cp, S_full, g, Fa, Fp_old, T, dt)[0]
                  - o.finite_cp_update(cp, S_full, g, Fb, Fp_old, T, dt)[0]) / (2 * h)
            err = max(err, np.abs(fd - np.moveaxis(K[:, :, k, L, :], -1, 0)).max())
            err_h = max(err_h, np.abs(fd - np.moveaxis(Kh[:, :, k, L, :], -1, 0)).max())
            mx = max(mx, np.abs(fd).max())
    assert err < 1e-7 * mx
    assert err_h > 1e-3 * mx
    asym = np.abs(K - np.einsum("iJkLv->kLiJv", K)).max() / np.abs(K).max()
    assert asym < 0.02
    Ks = o.finite_cp_tangent_consistent(data)
    assert np.allclose(Ks, np.einsum("iJkLv->kLiJv", Ks))
