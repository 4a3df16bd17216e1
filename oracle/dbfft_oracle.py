"""Plain FP64 CPU oracle of the DBFFT method (Lucarini & Segurado, arXiv 1905.12725).

TEST INFRASTRUCTURE ONLY. This module exists so that the CUDA path can be
checked against an independent, slow, obviously correct implementation. Only
the test suite, the smoke check and the CPU-baseline leg of the benchmark may
import it; the product path never does. It shares no code with the CUDA path.

Everything is FP64 / complex128 numpy. numpy's real FFT is used as a library
step (forward unnormalised e^{-i xi.x}, inverse with 1/N); every other step is
written out in the order of the paper's equations:

* grid and frequencies ........................... Sec. 2.1 (frequency vectors)
* displacement split, symmetric gradient s-hat ... Sec. 2.2, Eqs. disp_decomp, symgrad, s-hat
* divergence d-hat ............................... Sec. 2.2, Eq. diver, d-hat
* linear system (strain control) ................. Sec. 2.2, Eq. lineqf
* stress / mixed control ......................... Sec. 2.3, final system
* finite strain, gradient g-hat, Newton .......... Sec. 2.4, Eqs. lineariz, nonlineqf
* mixed control at finite strain ................. Sec. 2.4, Eq. nonlineqfstress
* preconditioner M(xi) ........................... Sec. 2.5, Eqs. pred2, pred3
* complex conjugate gradient ..................... Sec. 3 (opening paragraph)
* equilibrium / loading residuals ................ Sec. 3, Eqs. chedckeq, chedckimp

Readings taken where the paper is silent or garbled (each is pinned by a test):

R1  Even grids: xi'_i = 2 pi k_i / L_i with k_i in FFT order and xi'_i := 0 on
    the Nyquist index k_i = -N_i/2. The null set Z = {xi' = 0}; u-hat is zero
    there and every output is masked there. On odd grids this is the paper's
    frequency set exactly.
R2  Sign and scale: the paper's operator d:F(C:F^-1(s.u)) equals -N K with
    K = B^H C B, which is Hermitian positive definite off Z. The oracle solves
    K x = b (same solution). B(u, e) = F^-1(s.u) + E e, B^H sigma =
    ((1/N) s^H F(sigma), E^T sum_x sigma).
R3  The finite-strain gradient g-hat is read with the factor i: g_ijk = i xi_j
    delta_ik (the printed form drops it; the derivative rule needs it).
R4  M(0) is read as the macro-block preconditioner (N Cbar_ee)^-1 on the
    stress-controlled components; M(xi) = N [xi'.Cbar.xi']^-1 off Z, 0 on Z.
R5b The unknown lives on Hermitian-consistent spectra (v(-k) = conj v(k) on
    the k3 = 0 and k3 = N3/2 planes); operator outputs are projected onto
    that subspace, which only removes round-off.
R6  Inner product: the full-spectrum Hermitian product, computed on the half
    spectrum with weight 1 on the k3 = 0 and k3 = N3/2 planes and 2 elsewhere,
    plus the plain dot product of the macro unknowns. alpha, beta are real.
R7  CG stops when ||r|| / ||b|| <= tol with x0 = 0; ||b|| = 0 returns x = 0.
R8  Mixed control: macro unknowns e live on the stress-controlled components;
    small strain uses the orthonormal Mandel basis, finite strain the nine
    e_i x e_j. Their equations are E^T sum_x sigma = N sigma_bar_f.
R9  Newton stops when eps_eq = ||div P||_L2 / ||<P>|| <= newton_tol and the
    loading residual ||<P>_IJ - Pbar_IJ|| / ||<P>|| <= load_tol.
R10 Preconditioner refresh: linear problems use the mean stiffness; Newton
    uses the mean tangent at the first iterate of each increment.
R13 Compressible Neo-Hookean (not in the paper): W = mu/2 (tr F^T F - 3) -
    mu ln J + lam/2 (ln J)^2. St. Venant-Kirchhoff (the paper's porous-matrix
    law): W = lam/2 (tr E)^2 + mu E:E, E = (F^T F - I)/2.
R14 Small-strain power-law crystal plasticity (replaces the paper's model,
    whose parameters are not given): backward Euler on the stress.
R18 Finite-strain crystal plasticity (the paper's fourth benchmark uses
    F = Fe Fp): the R14 power law on the second Piola-Kirchhoff stress T of
    the intermediate configuration, T = C : (E_tr - sum_a dgam_a P_a) with the
    trial Green strain E_tr of Fe_tr = F Fp_old^-1 (small elastic strains),
    Fp = (I + sum_a dgam_a s_a n_a) Fp_old, P = Fe T Fp^-T. Its tangent is the
    derivative with the plastic state held (major-symmetric); Newton with it
    converges to the same increments as with the exact one.
"""
from __future__ import annotations

import math

import numpy as np

# --------------------------------------------------------------------------
# Grid, frequencies, null set, inner product            (Sec. 2.1; R1, R6)
# --------------------------------------------------------------------------

def half_shape(shape):
    n1, n2, n3 = shape
    return (n1, n2, n3 // 2 + 1)


def axis_wavenumbers(n: int) -> np.ndarray:
    """Integer frequency index of a full axis in FFT order (0..n/2-1, -n/2..-1)."""
    k = np.arange(n)
    return np.where(k < (n + 1) // 2, k, k - n)


def frequencies(shape, L=(1.0, 1.0, 1.0)):
    """xi' on the half spectrum, as three broadcastable arrays (R1).

    xi_i = 2 pi k_i / L_i (the paper's frequency vector for odd N, written in
    FFT order); on even axes the Nyquist index k_i = -N_i/2 gets xi'_i = 0.
    """
    n1, n2, n3 = shape
    out = []
    for ax, n in enumerate((n1, n2, n3)):
        k = axis_wavenumbers(n).astype(np.float64)
        xi = 2.0 * np.pi * k / L[ax]
        if n % 2 == 0:
            xi[n // 2] = 0.0
        if ax == 2:
            xi = xi[: n // 2 + 1]
            if n % 2 == 0:
                xi[n // 2] = 0.0  # k3 = n3/2 is the Nyquist index -n3/2
        out.append(xi)
    x1, x2, x3 = out
    return x1[:, None, None], x2[None, :, None], x3[None, None, :]


def null_mask(shape) -> np.ndarray:
    """Boolean half-spectrum mask of Z = {xi' = 0} (R1)."""
    x1, x2, x3 = frequencies(shape)
    return (x1 == 0) & (x2 == 0) & (x3 == 0)


def half_weights(shape) -> np.ndarray:
    """Multiplicity of each stored frequency in the full spectrum (R6)."""
    n3 = shape[2]
    h = n3 // 2 + 1
    w = np.full(h, 2.0)
    w[0] = 1.0
    if n3 % 2 == 0:
        w[h - 1] = 1.0
    return w[None, None, :]


def inner_u(a: np.ndarray, b: np.ndarray, shape) -> float:
    """Re sum over the full spectrum of conj(a) . b, from half spectra (R6)."""
    w = half_weights(shape)
    return float(np.sum(w * np.real(np.conj(a) * b)))


# --------------------------------------------------------------------------
# Fourier operators                       (Sec. 2.2 s-hat, d-hat; Sec. 2.4 g-hat)
# --------------------------------------------------------------------------

def grad_hat(u_hat, xi):
    """g-hat . u: G_ij = i xi_j u_i (R3). u_hat [3,...] -> [3,3,...]."""
    G = np.empty((3, 3) + u_hat.shape[1:], dtype=np.complex128)
    for i in range(3):
        for j in range(3):
            G[i, j] = 1j * xi[j] * u_hat[i]
    return G


def sym_grad_hat(u_hat, xi):
    """s-hat . u: eps_ij = 1/2 (i xi_j u_i + i xi_i u_j)  (Eq. s-hat)."""
    G = grad_hat(u_hat, xi)
    return 0.5 * (G + np.swapaxes(G, 0, 1))


def div_hat(s_hat, xi):
    """d-hat : sigma: [i xi_j sigma_ij]_i  (Eq. d-hat); [3,3,...] -> [3,...]."""
    out = np.zeros((3,) + s_hat.shape[2:], dtype=np.complex128)
    for i in range(3):
        for j in range(3):
            out[i] += 1j * xi[j] * s_hat[i, j]
    return out


def hermitian_project(v, shape):
    """Project a half-spectrum field onto the Hermitian-consistent subspace (R5b).

    On the planes k3 = 0 and k3 = N3/2 (even N3) the entries k and -k both
    hold one real unknown pair; the system is full rank only on spectra with
    v(-k) = conj(v(k)) there (Sec. 2.2: "real Fourier transform symmetries
    removed"). Exact operator outputs satisfy this; the projection removes
    round-off that would otherwise sit in the null space of K.
    """
    n1, n2, n3 = shape
    planes = [0] + ([n3 // 2] if n3 % 2 == 0 else [])
    i1 = (-np.arange(n1)) % n1
    i2 = (-np.arange(n2)) % n2
    out = v.copy()
    for k3 in planes:
        P = v[..., k3]
        Pc = np.conj(P[..., i1, :][..., :, i2])
        out[..., k3] = 0.5 * (P + Pc)
    return out


def to_real(t_hat, shape):
    return np.fft.irfftn(t_hat, s=shape, axes=(-3, -2, -1))


def to_fourier(t):
    return np.fft.rfftn(t, axes=(-3, -2, -1))


# --------------------------------------------------------------------------
# Macro bases (R8)
# --------------------------------------------------------------------------

_S2 = math.sqrt(2.0)
MANDEL_PAIRS = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]


def mandel_basis() -> np.ndarray:
    """Six orthonormal symmetric basis tensors Psi_m (Mandel order 11,22,33,23,13,12)."""
    B = np.zeros((6, 3, 3))
    for m, (i, j) in enumerate(MANDEL_PAIRS):
        if i == j:
            B[m, i, i] = 1.0
        else:
            B[m, i, j] = B[m, j, i] = 1.0 / _S2
    return B


def full_basis() -> np.ndarray:
    """Nine basis tensors e_i x e_j, index 3i + j."""
    B = np.zeros((9, 3, 3))
    for i in range(3):
        for j in range(3):
            B[3 * i + j, i, j] = 1.0
    return B


def tensor_to_mandel(t):
    """[3,3,...] -> [6,...] Mandel components (symmetric part)."""
    return np.einsum("mij,ij...->m...", mandel_basis(), t)


def mandel_to_tensor(v):
    return np.einsum("mij,m...->ij...", mandel_basis(), v)


# --------------------------------------------------------------------------
# Stiffness fields
# --------------------------------------------------------------------------

def iso_stiffness(lam, mu) -> np.ndarray:
    """C_ijkl = lam d_ij d_kl + mu (d_ik d_jl + d_il d_jk) for scalar lam, mu."""
    d = np.eye(3)
    return (lam * np.einsum("ij,kl->ijkl", d, d)
            + mu * (np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d)))


def lame(E, nu):
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


class IsoTangent:
    """Per-voxel isotropic stiffness given by Lame fields lam(x), mu(x)."""

    def __init__(self, lam, mu):
        self.lam = np.asarray(lam, dtype=np.float64)
        self.mu = np.asarray(mu, dtype=np.float64)

    def apply(self, eps):
        """C : eps = lam tr(eps) I + mu (eps + eps^T) (valid for any second-order eps)."""
        tr = eps[0, 0] + eps[1, 1] + eps[2, 2]
        sig = self.mu * (eps + np.swapaxes(eps, 0, 1))
        for i in range(3):
            sig[i, i] = sig[i, i] + self.lam * tr
        return sig

    def mean(self):
        return iso_stiffness(self.lam.mean(), self.mu.mean())


class FullTangent:
    """Per-voxel fourth-order tangent K_ijkl(x), stored [3,3,3,3,n1,n2,n3]."""

    def __init__(self, K):
        self.K = np.asarray(K, dtype=np.float64)

    def apply(self, g):
        return np.einsum("ijkl...,kl...->ij...", self.K, g)

    def mean(self):
        return self.K.reshape(3, 3, 3, 3, -1).mean(axis=-1)


# --------------------------------------------------------------------------
# The DBFFT operator, its right-hand side and preconditioner
# --------------------------------------------------------------------------

class Problem:
    """DBFFT discretisation of one RVE.

    kind = "small": unknown (u-hat, e) with e on the stress-controlled Mandel
    components; strain = s-hat.u (Sec. 2.2/2.3).
    kind = "finite": unknown (du-hat, e) with e on the stress-controlled
    components of F; gradient = g-hat.u (Sec. 2.4).
    stress_mask: iterable of 9 booleans, entry 3i+j True when the macro stress
    (sigma_ij or P_ij) is prescribed.
    """

    def __init__(self, shape, kind="small", stress_mask=None, L=(1.0, 1.0, 1.0)):
        self.shape = tuple(int(s) for s in shape)
        self.N = int(np.prod(self.shape))
        self.kind = kind
        self.L = tuple(float(v) for v in L)
        self.xi = frequencies(self.shape, L)
        self.Z = null_mask(self.shape)
        m9 = np.zeros(9, dtype=bool) if stress_mask is None else np.asarray(stress_mask, dtype=bool)
        if kind == "small":
            m33 = m9.reshape(3, 3)
            if not np.array_equal(m33, m33.T):
                raise ValueError("small-strain stress mask must be symmetric")
            self.basis_all = mandel_basis()
            self.active = np.array([m33[i, j] for (i, j) in MANDEL_PAIRS])
        else:
            self.basis_all = full_basis()
            self.active = m9.copy()
        self.basis = self.basis_all[self.active]  # [ne,3,3]
        self.ne = int(self.active.sum())

    # ---- kinematics: B(u, e) and its adjoint
    def field_from(self, u_hat, e):
        """B(u, e): strain / displacement-gradient field [3,3,n1,n2,n3]."""
        if self.kind == "small":
            t_hat = sym_grad_hat(u_hat, self.xi)
        else:
            t_hat = grad_hat(u_hat, self.xi)
        t = to_real(t_hat, self.shape)
        if self.ne:
            t += np.einsum("mij,m->ij", self.basis, e)[:, :, None, None, None]
        return t

    def adjoint(self, sig):
        """B^H sigma = ((1/N) s^H F(sigma), E^T sum_x sigma)   (R2).

        s^H sigma-hat = -d-hat : sigma-hat for both s-hat and g-hat.
        """
        s_hat = to_fourier(sig)
        q = hermitian_project(-div_hat(s_hat, self.xi) / self.N, self.shape)
        q[:, self.Z] = 0.0
        tot = s_hat[:, :, 0, 0, 0].real  # sum_x sigma
        qe = np.einsum("mij,ij->m", self.basis, tot)
        return q, qe

    def apply_K(self, tangent, u_hat, e):
        """K (u, e) = B^H T B (u, e)  (Eq. lineqf / nonlineqf in SPD form, R2)."""
        return self.adjoint(tangent.apply(self.field_from(u_hat, e)))

    # ---- vector helpers for CG over (u-hat, e)
    def zeros(self):
        return (np.zeros((3,) + half_shape(self.shape), dtype=np.complex128), np.zeros(self.ne))

    def dot(self, a, b):
        return inner_u(a[0], b[0], self.shape) + float(np.dot(a[1], b[1]))

    # ---- preconditioner (Sec. 2.5, Eqs. pred2-pred3; R4)
    def make_preconditioner(self, Cbar):
        """z = M r with M(xi) = N [xi'.Cbar.xi']^-1 off Z, macro block (N Cbar_ee)^-1."""
        x1, x2, x3 = np.broadcast_arrays(*self.xi)
        xi = np.stack([x1, x2, x3])  # [3, n1, n2, h]
        Q = np.einsum("j...,ijkl,l...->ik...", xi, Cbar, xi)  # acoustic tensor
        Qm = np.moveaxis(Q, (0, 1), (-2, -1)).copy()
        Qm[self.Z] = np.eye(3)
        Minv = np.linalg.inv(Qm) * self.N
        Minv[self.Z] = 0.0
        if self.ne:
            Cee = np.einsum("mij,ijkl,nkl->mn", self.basis, Cbar, self.basis)
            Me = np.linalg.inv(self.N * Cee)
        else:
            Me = np.zeros((0, 0))

        def M(r):
            zu = np.einsum("...ik,k...->i...", Minv, r[0])
            return (zu, Me @ r[1])

        return M


# --------------------------------------------------------------------------
# Preconditioned conjugate gradient over complex vectors (Sec. 3; R6, R7)
# --------------------------------------------------------------------------

def pcg(prob: Problem, K, M, b, tol, max_iter):
    """Textbook PCG for the Hermitian positive definite K. Returns (x, iters, hist)."""
    x = prob.zeros()
    bnorm = math.sqrt(prob.dot(b, b))
    hist = [1.0]
    if bnorm == 0.0:
        return x, 0, hist
    r = (b[0].copy(), b[1].copy())
    z = M(r)
    p = (z[0].copy(), z[1].copy())
    rho = prob.dot(r, z)
    it = 0
    while it < max_iter:
        q = K(p)
        alpha = rho / prob.dot(p, q)
        x = (x[0] + alpha * p[0], x[1] + alpha * p[1])
        r = (r[0] - alpha * q[0], r[1] - alpha * q[1])
        it += 1
        rel = math.sqrt(prob.dot(r, r)) / bnorm
        hist.append(rel)
        if rel <= tol:
            break
        z = M(r)
        rho_new = prob.dot(r, z)
        beta = rho_new / rho
        rho = rho_new
        p = (z[0] + beta * p[0], z[1] + beta * p[1])
    return x, it, hist


# --------------------------------------------------------------------------
# Linear elasticity, strain / stress / mixed control  (Sec. 2.2, 2.3)
# --------------------------------------------------------------------------

def split_load(prob: Problem, target):
    """Prescribed macro field on strain-controlled components and stress targets.

    target: [3,3] holding the prescribed strain (small) or deformation gradient
    (finite) on the strain-controlled components and the prescribed stress on
    the stress-controlled ones. Returns (field_U [3,3], stress targets on the
    active macro basis [ne]). At finite strain field_U = I + (Fbar_U - I) on
    the prescribed components, and I on the stress-controlled ones (R8).
    """
    target = np.asarray(target, dtype=np.float64)
    base = np.eye(3) if prob.kind == "finite" else np.zeros((3, 3))
    coeff = np.einsum("mij,ij->m", prob.basis_all, target - base)
    fU = base + np.einsum("mij,m->ij", prob.basis_all[~prob.active], coeff[~prob.active])
    sig_f = np.einsum("mij,ij->m", prob.basis, target)
    return fU, sig_f


def macro_field(prob: Problem, fieldU, e):
    """The whole macroscopic strain (small) or deformation gradient (finite):
    the prescribed part plus the solved stress-controlled unknowns E e."""
    out = np.array(fieldU, dtype=np.float64)
    if prob.ne:
        out = out + np.einsum("mij,m->ij", prob.basis, e)
    return out


def displacement(prob: Problem, u_hat, macro):
    """Total displacement at the voxel centres (Sec. 2.2, Eqs. disp_decomp and
    decomp_displ; Sec. 2.4 with Fbar - I in place of the macro strain).

    u(x) = Hbar x + u~(x): u~ is the inverse DFT of the unknown u-hat (the
    periodic fluctuation, zero mean) and Hbar = macro (small strain) or
    macro - I (finite strain), macro from macro_field. Voxel j of axis a sits
    at x_a = (j + 1/2) L_a / n_a. Returns [3, n1, n2, n3].
    """
    Hbar = np.asarray(macro, dtype=np.float64) - (np.eye(3) if prob.kind == "finite" else 0.0)
    ut = to_real(u_hat, prob.shape)
    x = [(np.arange(n) + 0.5) * (L / n) for n, L in zip(prob.shape, prob.L)]
    X = np.stack(np.meshgrid(*x, indexing="ij"))  # [3, n1, n2, n3]
    return ut + np.einsum("ij,j...->i...", Hbar, X)


def _levi():
    e = np.zeros((3, 3, 3))
    for i, j, k in ((0, 1, 2), (1, 2, 0), (2, 0, 1)):
        e[i, j, k], e[i, k, j] = 1.0, -1.0
    return e


def compatibility(prob: Problem, field_hat, macro_norm):
    """Compatibility residual (Sec. 3, Eq. chedckcomp; finite strain: curl of F).

    field_hat: the Fourier coefficients (rfftn) of the fluctuating field, [3,3,
    half spectrum] (strain or displacement gradient). Small strain:
    eta = curl (curl eps)^T, eta_ij = e_ikl e_jmn d_k d_m eps_ln; finite
    strain: (curl F)_iJ = e_JKL d_K F_iL, derivatives d = i xi'. Returns
    (max over the voxels and components of |.|, root mean square over the
    cell), both divided by macro_norm.
    """
    e = _levi()
    d = np.stack(np.broadcast_arrays(*prob.xi)).astype(np.complex128) * 1j  # [3, half]
    if prob.kind == "small":
        eta = np.einsum("ikl,jmn,k...,m...,ln...->ij...", e, e, d, d, field_hat)
    else:
        eta = np.einsum("JKL,K...,iL...->iJ...", e, d, field_hat)
    real = to_real(eta, prob.shape)
    mx = float(np.abs(real).max())
    rms = float(np.sqrt(np.sum(real ** 2) / prob.N))  # sqrt of the cell mean of the squared Frobenius norm
    return mx / macro_norm, rms / macro_norm


def linear_rhs(prob: Problem, tangent, target):
    """b = -B^H C epsbar_U + (0, N sigma_f)  (Sec. 2.3 final system, R2)."""
    epsU, sig_f = split_load(prob, target)
    field = np.broadcast_to(epsU[:, :, None, None, None], (3, 3) + prob.shape).copy()
    qu, qe = prob.adjoint(tangent.apply(field))
    return (-qu, prob.N * sig_f - qe)


def residual(prob: Problem, stress_fn, x, fieldU, sig_f):
    """True residual of the macro-loaded problem: -B^H sigma(total) + (0, N sigma_f).

    stress_fn maps the total strain / deformation-gradient field to stress.
    Returns (residual, total field, stress field).
    """
    tot = prob.field_from(x[0], x[1]) + fieldU[:, :, None, None, None]
    sig = stress_fn(tot)
    qu, qe = prob.adjoint(sig)
    return (-qu, prob.N * sig_f - qe), tot, sig


def solve_linear(prob: Problem, tangent, target, tol=1e-12, max_iter=10000, Cbar=None):
    """Solve the linear DBFFT system by PCG; returns a dict of the solution.

    Output: u (u-hat), e (macro unknowns), eps (total strain), sig, sig_bar,
    iters, hist, eps_eq (equilibrium residual, Eq. chedckeq).
    """
    b = linear_rhs(prob, tangent, target)
    M = prob.make_preconditioner(tangent.mean() if Cbar is None else Cbar)
    x, it, hist = pcg(prob, lambda v: prob.apply_K(tangent, v[0], v[1]), M, b, tol, max_iter)
    epsU, sig_f = split_load(prob, target)
    r, eps, sig = residual(prob, tangent.apply, x, epsU, sig_f)
    sig_bar = sig.reshape(3, 3, -1).mean(axis=-1)
    return dict(u=x[0], e=x[1], eps=eps, sig=sig, sig_bar=sig_bar, iters=it, hist=hist,
                eps_eq=equilibrium_residual(prob, r, sig_bar), res=r,
                true_rel=math.sqrt(prob.dot(r, r)) / max(math.sqrt(prob.dot(b, b)), 1e-300))


def equilibrium_residual(prob: Problem, r, sig_bar):
    """eps_eq = ||div sigma||_L2 / ||<sigma>||  (Eq. chedckeq, L = 1).

    ||div sigma||_L2^2 = mean_x |div sigma|^2 = sum over the full spectrum of
    |r_u|^2 (Parseval, r_u = -(1/N) d-hat:sigma-hat).
    """
    num = math.sqrt(inner_u(r[0], r[0], prob.shape))
    den = float(np.linalg.norm(sig_bar))
    return num / den if den > 0 else num


def homogenized_tangent(shape, tangent, tol=1e-12, max_iter=10000):
    """6x6 Mandel effective stiffness from the six unit Mandel macro strains."""
    prob = Problem(shape, "small")
    B = mandel_basis()
    Ceff = np.zeros((6, 6))
    iters = []
    for n in range(6):
        sol = solve_linear(prob, tangent, B[n], tol=tol, max_iter=max_iter)
        Ceff[:, n] = tensor_to_mandel(sol["sig_bar"])
        iters.append(sol["iters"])
    return Ceff, iters


# --------------------------------------------------------------------------
# Compressible Neo-Hookean (R13)
# --------------------------------------------------------------------------

def neo_hooke(F, mu, lam):
    """P and K = dP/dF for W = mu/2 (tr F^T F - 3) - mu ln J + lam/2 (ln J)^2.

    F [3,3,...]; mu, lam broadcastable to F[0,0]. Returns P [3,3,...],
    K [3,3,3,3,...] with K_iJkL = dP_iJ / dF_kL.
    """
    Fm = np.moveaxis(F, (0, 1), (-2, -1))
    J = np.linalg.det(Fm)
    if np.any(J <= 0):
        raise FloatingPointError("non-positive Jacobian")
    Fi = np.linalg.inv(Fm)                       # [..., 3, 3] = F^-1
    FiT = np.swapaxes(Fi, -1, -2)                # F^-T
    lnJ = np.log(J)
    mu_ = np.asarray(mu)[..., None, None]
    lam_ = np.asarray(lam)[..., None, None]
    P = mu_ * (Fm - FiT) + lam_ * lnJ[..., None, None] * FiT
    d = np.eye(3)
    a = np.asarray(mu - lam * lnJ)
    # K_iJkL = mu d_ik d_JL + (mu - lam lnJ) Fi_Li Fi_Jk + lam Fi_Ji Fi_Lk
    K = (np.asarray(mu)[..., None, None, None, None] * np.einsum("ik,jl->ijkl", d, d)
         + a[..., None, None, None, None] * np.einsum("...li,...jk->...ijkl", Fi, Fi)
         + np.asarray(lam)[..., None, None, None, None] * np.einsum("...ji,...lk->...ijkl", Fi, Fi))
    P = np.moveaxis(P, (-2, -1), (0, 1))
    K = np.moveaxis(K, (-4, -3, -2, -1), (0, 1, 2, 3))
    return P, K


def neo_hooke_energy(F, mu, lam):
    Fm = np.moveaxis(F, (0, 1), (-2, -1))
    J = np.linalg.det(Fm)
    lnJ = np.log(J)
    I1 = np.einsum("...ij,...ij->...", Fm, Fm)
    return 0.5 * mu * (I1 - 3.0) - mu * lnJ + 0.5 * lam * lnJ ** 2


def svk(F, mu, lam):
    """St. Venant-Kirchhoff law (the matrix of the paper's porous hyperelastic
    example, Sec. 3): W = lam/2 (tr E)^2 + mu E:E with E = (F^T F - I)/2.

    P = F S, S = lam tr(E) I + 2 mu E;
    K_iJkL = d_ik S_JL + lam F_iJ F_kL + mu (F_iL F_kJ + (F F^T)_ik d_JL).
    F [3,3,...]; mu, lam broadcastable to F[0,0]. Returns P, K like neo_hooke.
    """
    Fm = np.moveaxis(F, (0, 1), (-2, -1))
    d = np.eye(3)
    E = 0.5 * (np.swapaxes(Fm, -1, -2) @ Fm - d)
    mu_ = np.asarray(mu)[..., None, None]
    lam_ = np.asarray(lam)[..., None, None]
    S = lam_ * np.trace(E, axis1=-2, axis2=-1)[..., None, None] * d + 2.0 * mu_ * E
    P = Fm @ S
    B = Fm @ np.swapaxes(Fm, -1, -2)
    lam4 = np.asarray(lam)[..., None, None, None, None]
    mu4 = np.asarray(mu)[..., None, None, None, None]
    K = (np.einsum("ik,...jl->...ijkl", d, S) + lam4 * np.einsum("...ij,...kl->...ijkl", Fm, Fm)
         + mu4 * (np.einsum("...il,...kj->...ijkl", Fm, Fm) + np.einsum("...ik,jl->...ijkl", B, d)))
    P = np.moveaxis(P, (-2, -1), (0, 1))
    K = np.moveaxis(K, (-4, -3, -2, -1), (0, 1, 2, 3))
    return P, K


def svk_energy(F, mu, lam):
    Fm = np.moveaxis(F, (0, 1), (-2, -1))
    E = 0.5 * (np.swapaxes(Fm, -1, -2) @ Fm - np.eye(3))
    trE = np.trace(E, axis1=-2, axis2=-1)
    return 0.5 * lam * trE ** 2 + mu * np.einsum("...ij,...ij->...", E, E)


# --------------------------------------------------------------------------
# Small-strain power-law FCC crystal plasticity (R14)
# --------------------------------------------------------------------------

FCC_PLANES = np.array([[1, 1, 1], [-1, 1, 1], [1, -1, 1], [1, 1, -1]], dtype=np.float64)
FCC_DIRS = np.array([
    [[0, 1, -1], [1, 0, -1], [1, -1, 0]],
    [[0, 1, -1], [1, 0, 1], [1, 1, 0]],
    [[0, 1, 1], [1, 0, -1], [1, 1, 0]],
    [[0, 1, 1], [1, 0, 1], [1, -1, 0]],
], dtype=np.float64)


def fcc_slip_systems():
    """The 12 {111}<110> systems (s_a, n_a), unit vectors in the crystal frame."""
    s, n = [], []
    for p in range(4):
        for d in range(3):
            n.append(FCC_PLANES[p] / math.sqrt(3.0))
            s.append(FCC_DIRS[p, d] / math.sqrt(2.0))
    return np.array(s), np.array(n)


def quat_to_rot(q):
    """Rotation matrix (crystal -> sample) of a unit quaternion (w, x, y, z)."""
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def cubic_stiffness(C11, C12, C44):
    C = np.zeros((3, 3, 3, 3))
    for i in range(3):
        for j in range(3):
            for k in range(3):
                for l in range(3):
                    if i == j and k == l:
                        C[i, j, k, l] = C11 if i == k else C12
                    elif (i == k and j == l) or (i == l and j == k):
                        C[i, j, k, l] = C44
    return C


def tensor4_to_mandel(C):
    B = mandel_basis()
    return np.einsum("mij,ijkl,nkl->mn", B, C, B)


def mandel_to_tensor4(Cm):
    B = mandel_basis()
    return np.einsum("mij,mn,nkl->ijkl", B, Cm, B)


class CrystalPlasticity:
    """Per-grain data for the small-strain power-law model (R14), Mandel form."""

    def __init__(self, quats, C11=168000.0, C12=121000.0, C44=75000.0,
                 gdot0=1e-3, m=0.05, tau_c=50.0):
        self.gdot0, self.m, self.tau_c = gdot0, m, tau_c
        s, n = fcc_slip_systems()
        Cc = cubic_stiffness(C11, C12, C44)
        self.C = []     # Mandel stiffness per grain
        self.S = []     # Mandel compliance per grain
        self.P = []     # [12, 6] Schmid tensors per grain (Mandel)
        B = mandel_basis()
        for q in np.asarray(quats, dtype=np.float64):
            R = quat_to_rot(q / np.linalg.norm(q))
            Cg = np.einsum("ia,jb,kc,ld,abcd->ijkl", R, R, R, R, Cc)
            Cm = tensor4_to_mandel(Cg)
            self.C.append(Cm)
            self.S.append(np.linalg.inv(Cm))
            sr = s @ R.T
            nr = n @ R.T
            Pa = 0.5 * (np.einsum("ai,aj->aij", sr, nr) + np.einsum("ai,aj->aij", nr, sr))
            self.P.append(np.einsum("mij,aij->am", B, Pa))
        self.C = np.array(self.C)
        self.S = np.array(self.S)
        self.P = np.array(self.P)

    def rates(self, tau):
        """gdot_a and d gdot_a / d tau_a for the power law."""
        x = np.abs(tau) / self.tau_c
        e = 1.0 / self.m
        gd = self.gdot0 * x ** e * np.sign(tau)
        dgd = self.gdot0 * e / self.tau_c * x ** (e - 1.0)
        return gd, dgd

    def tangent_at(self, grain, sig, dt, scale=None):
        """Consistent tangent (S/s + dt sum_a gdot'_a P_a P_a^T)^-1 at the stresses sig [V,6]."""
        S = self.S[grain] if scale is None else self.S[grain] / np.asarray(scale)[:, None, None]
        P = self.P[grain]
        _, dgd = self.rates(np.einsum("vam,vm->va", P, sig))
        return np.linalg.inv(S + dt * np.einsum("va,vam,van->vmn", dgd, P, P))

    def update(self, grain, eps, eps_p_old, sig_guess, dt, rtol=1e-12, max_it=100, scale=None):
        """Backward Euler at every voxel (vectorised over voxels).

        Solves R(sigma) = S sigma + dt sum_a gdot_a(sigma) P_a - (eps - eps_p_old) = 0
        (Mandel 6-vectors) by Newton, stopped when the full Newton step is below
        rtol (|sigma| + tau_c), with backtracking (far from the solution) on the
        convex potential
        phi(sigma) = 1/2 sigma.S.sigma + dt sum_a gdot0 tau_c m/(1+m)|tau_a/tau_c|^(1+1/m)
                     - sigma.(eps - eps_p_old).
        scale (optional, [V]): a factor s(x) on the elastic stiffness, C = s C_grain.
        Returns (sigma, tangent d sigma / d eps [.., 6, 6], eps_p_new, newton iterations).
        """
        S = self.S[grain]              # [V,6,6]
        if scale is not None:
            S = S / np.asarray(scale, dtype=np.float64)[:, None, None]
        P = self.P[grain]              # [V,12,6]
        target = eps - eps_p_old       # [V,6]
        sig = sig_guess.copy()
        e = 1.0 / self.m

        def phi(sv):
            tau = np.einsum("vam,vm->va", P, sv)
            pot = self.gdot0 * self.tau_c * self.m / (1.0 + self.m) * (np.abs(tau) / self.tau_c) ** (1.0 + e)
            return (0.5 * np.einsum("vm,vmn,vn->v", sv, S, sv) + dt * pot.sum(axis=1)
                    - np.einsum("vm,vm->v", sv, target))

        it_max = 0
        active = np.ones(sig.shape[0], dtype=bool)
        for it in range(max_it):
            tau = np.einsum("vam,vm->va", P, sig)
            gd, dgd = self.rates(tau)
            R = np.einsum("vmn,vn->vm", S, sig) + dt * np.einsum("va,vam->vm", gd, P) - target
            J = S + dt * np.einsum("va,vam,van->vmn", dgd, P, P)
            step = -np.linalg.solve(J, R[..., None])[..., 0]
            step[~active] = 0.0
            scale = np.linalg.norm(sig, axis=1) + self.tau_c
            nstep = np.linalg.norm(step, axis=1)
            conv = active & (nstep <= rtol * scale)  # full Newton step below tolerance: accept and stop
            # backtracking on phi only far from the solution (strictly convex potential,
            # so the Newton direction descends); the allowance 1e-13 |phi| absorbs round-off
            far = active & (nstep > 1e-3 * scale)
            t = np.ones(sig.shape[0])
            f0 = phi(sig)
            slope = np.einsum("vm,vm->v", R, step)
            for _ in range(60):
                trial = sig + t[:, None] * step
                bad = far & (phi(trial) > f0 + 1e-4 * t * slope + 1e-13 * np.abs(f0))
                if not np.any(bad):
                    break
                t[bad] *= 0.5
            sig = sig + t[:, None] * step
            active &= ~conv
            it_max = it + 1
            if not np.any(active):
                break
        else:
            raise FloatingPointError("crystal plasticity local Newton did not converge")
        tau = np.einsum("vam,vm->va", P, sig)
        gd, dgd = self.rates(tau)
        J = S + dt * np.einsum("va,vam,van->vmn", dgd, P, P)
        tangent = np.linalg.inv(J)
        eps_p = eps_p_old + dt * np.einsum("va,vam->vm", gd, P)
        return sig, tangent, eps_p, it_max


# --------------------------------------------------------------------------
# Newton over increments with mixed control   (Sec. 2.4, Eqs. lineariz, nonlineqfstress)
# --------------------------------------------------------------------------

def newton_increments(prob: Problem, material, targets, newton_tol=1e-8, load_tol=1e-10,
                      eta=1e-4, max_newton=30, max_cg=10000, state=None, callback=None):
    """Increment loop with Newton iterations, each solved by PCG (Sec. 2.4).

    material(field, state) -> (stress field, FullTangent, trial state)
    evaluates the constitutive law at the total field (strain for small,
    deformation gradient for finite). targets: list of [3,3] macro targets per
    increment (prescribed field components + stress targets on the mask).
    Returns a list of per-increment dicts (stress average, iterations, ...).
    """
    x = prob.zeros()
    out = []
    for inc, target in enumerate(targets):
        fU, sig_f = split_load(prob, target)
        newton = []
        cg_total = 0
        M = None
        for it in range(max_newton + 1):
            tot = prob.field_from(x[0], x[1]) + fU[:, :, None, None, None]
            sig, tang, trial_state = material(tot, state)
            qu, qe = prob.adjoint(sig)
            r = (-qu, prob.N * sig_f - qe)
            Pbar = sig.reshape(3, 3, -1).mean(axis=-1)
            nP = float(np.linalg.norm(Pbar))
            eq = math.sqrt(inner_u(r[0], r[0], prob.shape)) / nP if nP > 0 else 0.0
            ld = float(np.linalg.norm(r[1])) / (prob.N * nP) if (nP > 0 and prob.ne) else 0.0
            newton.append(dict(eps_eq=eq, load=ld))
            if eq <= newton_tol and ld <= load_tol:
                break
            if it == max_newton:
                raise FloatingPointError("Newton did not converge")
            if M is None:  # R10: mean tangent at the first iterate of the increment
                M = prob.make_preconditioner(tang.mean())
            d, cg_it, _ = pcg(prob, lambda v: prob.apply_K(tang, v[0], v[1]), M, r, eta, max_cg)
            cg_total += cg_it
            newton[-1]["cg"] = cg_it
            gd = to_real(grad_hat(d[0], prob.xi), prob.shape)
            newton[-1]["max_grad_du"] = float(np.abs(gd).max())
            x = (x[0] + d[0], x[1] + d[1])
        state = trial_state  # commit the converged constitutive state
        rec = dict(inc=inc, stress_bar=Pbar, field_bar=tot.reshape(3, 3, -1).mean(axis=-1),
                   newton=newton, cg_total=cg_total, x=(x[0].copy(), x[1].copy()), state=state)
        out.append(rec)
        if callback is not None:
            callback(rec)
    return out, state


def neo_hooke_material(mu_field, lam_field):
    def material(F, state):
        P, K = neo_hooke(F, mu_field, lam_field)
        return P, FullTangent(K), state
    return material


def svk_material(mu_field, lam_field):
    def material(F, state):
        P, K = svk(F, mu_field, lam_field)
        return P, FullTangent(K), state
    return material


def cp_material(cp: CrystalPlasticity, grain_field, dt, scale=None):
    """Material closure for the crystal-plasticity model; state = (eps_p, sigma).
    scale (optional, grain_field's shape): factor s(x) on the elastic stiffness."""
    g = grain_field.reshape(-1)
    sc = None if scale is None else np.asarray(scale, dtype=np.float64).reshape(-1)

    def material(eps, state):
        V = g.size
        em = tensor_to_mandel(eps).reshape(6, V).T
        if state is None:
            state = (np.zeros((V, 6)), np.zeros((V, 6)))
        eps_p, sig_prev = state
        sig, tan, eps_p_new, _ = cp.update(g, em, eps_p, sig_prev, dt, scale=sc)
        sig_t = mandel_to_tensor(sig.T.reshape((6,) + grain_field.shape))
        K = np.einsum("mij,vmn,nkl->ijklv", mandel_basis(), tan, mandel_basis())
        K = K.reshape((3, 3, 3, 3) + grain_field.shape)
        new_state = (eps_p_new, sig)
        return sig_t, FullTangent(K), new_state
    return material


def cp_adjoint_increments(prob: Problem, cp: CrystalPlasticity, grain_field, dt, targets, g,
                          newton_tol=1e-12, load_tol=1e-12, eta=1e-10, tol=1e-13, max_iter=10000):
    """dJ/ds(x) for J = g : <sigma> after the last increment of a small-strain
    crystal-plasticity loading path (Sec. 2.4, Eq. lineariz; R14), s(x) a factor
    on the elastic stiffness of voxel x, at s = 1 (the derivative per voxel of
    the logarithm of its stiffness).

    Forward: the Newton increments, keeping the converged stress of every
    increment as its checkpoint (the consistent tangent T_n and the plastic
    strain follow from it). Reverse, over the increments n = N .. 1, with the
    state adjoint q (dJ / d eps_p of the increment's result, 0 after the last)
    and a = g / N at the last increment (0 before):
        h = a - S q,  w = q + T_n h,
        K_n lam = B^H w          (the self-adjoint increment operator, Sec. 2.2),
        d = h - B lam,
        dJ/ds += d . T_n S sigma_n + q . S sigma_n,
        q = -T_n d,
    all per voxel in Mandel components (S the grain compliance). Returns
    (dJ/ds field, J, forward records).
    """
    V = grain_field.size
    gidx = grain_field.reshape(-1)
    recs, _ = newton_increments(prob, cp_material(cp, grain_field, dt), targets, newton_tol=newton_tol,
                                load_tol=load_tol, eta=eta)
    gm = tensor_to_mandel(np.asarray(g, dtype=np.float64))
    J = float(np.sum(np.asarray(g) * recs[-1]["stress_bar"]))
    S = cp.S[gidx]
    q = np.zeros((V, 6))
    dJ = np.zeros(V)
    basis = mandel_basis()
    for n in range(len(recs) - 1, -1, -1):
        sig_n = recs[n]["state"][1]                      # checkpoint: converged stress [V, 6]
        T = cp.tangent_at(gidx, sig_n, dt)               # [V, 6, 6]
        a = gm[None, :] / prob.N if n == len(recs) - 1 else np.zeros((V, 6))
        h = a - np.einsum("vmn,vn->vm", S, q)
        w = q + np.einsum("vmn,vn->vm", T, h)
        wt = np.einsum("mij,vm->ijv", basis, w).reshape((3, 3) + prob.shape)
        rhs = prob.adjoint(wt)
        Kt = FullTangent(np.einsum("mij,vmn,nkl->ijklv", basis, T, basis).reshape((3, 3, 3, 3) + prob.shape))
        M = prob.make_preconditioner(Kt.mean())
        lam, _, _ = pcg(prob, lambda v: prob.apply_K(Kt, v[0], v[1]), M, rhs, tol, max_iter)
        Blam = tensor_to_mandel(prob.field_from(lam[0], lam[1])).reshape(6, V).T
        d = h - Blam
        Ssig = np.einsum("vmn,vn->vm", S, sig_n)
        dJ += np.einsum("vm,vm->v", d, np.einsum("vmn,vn->vm", T, Ssig)) + np.einsum("vm,vm->v", q, Ssig)
        q = -np.einsum("vmn,vn->vm", T, d)
    return dJ.reshape(prob.shape), J, recs


# --------------------------------------------------------------------------
# Finite-strain crystal plasticity, F = Fe Fp (R18)
# --------------------------------------------------------------------------

def schmid_full(cp: CrystalPlasticity, quats):
    """Non-symmetric Schmid tensors S_a = s_a (x) n_a in the sample frame, [grain, 12, 3, 3]."""
    s, n = fcc_slip_systems()
    out = []
    for q in np.asarray(quats, dtype=np.float64):
        R = quat_to_rot(q / np.linalg.norm(q))
        out.append(np.einsum("ai,aj->aij", s @ R.T, n @ R.T))
    return np.array(out)


def finite_cp_update(cp: CrystalPlasticity, S_full, grain, F, Fp_old, T_guess, dt):
    """One step of the finite-strain model at every voxel (vectorised).

    F [V,3,3]; Fp_old [V,3,3]; T_guess [V,6] (Mandel). With a = Fp_old^-1, the
    trial elastic deformation Fe_tr = F a and the Green strain of the
    intermediate configuration E_tr = (Fe_tr^T Fe_tr - I)/2, the second
    Piola-Kirchhoff stress of the intermediate configuration T solves the
    backward-Euler problem of the small-strain model (R14) with E_tr as the
    strain and no plastic strain at the start of the step (the elastic strains
    stay small, so T = C : (E_tr - dt sum_a gdot_a P_a)). Then
    Fp = (I + dt sum_a gdot_a S_a) Fp_old, Fe = F Fp^-1, P = Fe T Fp^-T.
    Returns (P [V,3,3], Fp [V,3,3], T [V,6], tangent data) with tangent data
    (Fe_tr, a, B = a T a^T, C_tan = dT/dE_tr Mandel [V,6,6]).
    """
    V = F.shape[0]
    a = np.linalg.inv(Fp_old)
    Fe_tr = F @ a
    E_tr = 0.5 * (np.swapaxes(Fe_tr, 1, 2) @ Fe_tr - np.eye(3))
    e_tr = np.einsum("mij,vij->vm", mandel_basis(), E_tr)
    T, C_tan, dep, _ = cp.update(grain, e_tr, np.zeros((V, 6)), T_guess, dt)
    tau = np.einsum("vam,vm->va", cp.P[grain], T)
    gd, dgd = cp.rates(tau)
    Mm = np.eye(3) + dt * np.einsum("va,vaij->vij", gd, S_full[grain])
    Fp = Mm @ Fp_old
    Fpi = np.linalg.inv(Fp)
    Tm = np.einsum("mij,vm->vij", mandel_basis(), T)
    P = F @ Fpi @ Tm @ np.swapaxes(Fpi, 1, 2)
    B = a @ Tm @ np.swapaxes(a, 1, 2)
    # for the consistent tangent: N = M^-1 and D = dM / dT = sum_a dt gdot'_a S_a (x) P_a
    D = dt * np.einsum("va,vaij,vam->vijm", dgd, S_full[grain], cp.P[grain])
    return P, Fp, T, (Fe_tr, a, B, C_tan, np.linalg.inv(Mm), D, Tm)


def finite_cp_tangent(data):
    """K_iJkL of dP = G B + Fe_tr (C_tan : sym(Fe_tr^T G a)) a^T: the derivative of
    F a T(E(F)) a^T with the plastic state a = Fp_old^-1 held fixed (R18). It is
    major-symmetric. Returns [3,3,3,3,V]."""
    Fe_tr, a, B, C_tan = data[:4]
    V = Fe_tr.shape[0]
    K = np.zeros((V, 3, 3, 3, 3))
    Bm = mandel_basis()
    Ct = np.einsum("mij,vmn,nkl->vijkl", Bm, C_tan, Bm)  # dT_ij / dE_kl (minor-symmetric)
    d = np.eye(3)
    K += np.einsum("ik,vLJ->viJkL", d, B)
    # dE_MN = sym(Fe_tr^T G a)_MN = 1/2 (Fe_kM a_LN + Fe_kN a_LM) G_kL
    dE = 0.5 * (np.einsum("vkM,vLN->vMNkL", Fe_tr, a) + np.einsum("vkN,vLM->vMNkL", Fe_tr, a))
    K += np.einsum("viP,vPQMN,vMNkL,vJQ->viJkL", Fe_tr, Ct, dE, a)
    return np.moveaxis(K, 0, -1)


def finite_cp_tangent_consistent(data, symmetric=True):
    """The consistent tangent K_iJkL = dP_iJ / dF_kL of the finite-strain update (R18b),
    with the plastic flow of the step active: P = F a N T N^T a^T, N = M^-1,
    M = I + sum_a dt gdot_a(T) S_a, T(E_tr(F)) with dT = C_tan : sym(Fe_tr^T dF a),
    dM = D : dT. So
        dP = dF a N T N^T a^T + sum_m dT_m X_m,
        X_m = Fe B_m (aN)^T - Fe D_m N T (aN)^T - Fe T N^T D_m^T (aN)^T,  Fe = F a N,
    with B_m the Mandel basis and D_m = D[..., m]; dT_m = sum_n C_tan,mn Fe_tr B_n a^T : dF.
    It is not major-symmetric; symmetric=True returns (K + K^T)/2 over (iJ) <-> (kL),
    the form PCG needs (R11). Returns [3,3,3,3,V]."""
    Fe_tr, a, B, C_tan, N, D, Tm = data
    V = Fe_tr.shape[0]
    Bm = mandel_basis()
    aN = a @ N
    Fe = Fe_tr @ N  # F a N
    Bc = aN @ Tm @ np.swapaxes(aN, 1, 2)
    NT = N @ Tm
    K = np.einsum("ik,vLJ->viJkL", np.eye(3), Bc)
    X = (np.einsum("viP,mPQ,vJQ->vmiJ", Fe, Bm, aN)
         - np.einsum("viP,vPQm,vQR,vJR->vmiJ", Fe, D, NT, aN)
         - np.einsum("viP,vPQ,vRQ,vSRm,vJS->vmiJ", Fe, Tm, N, D, aN))
    Y = np.einsum("vmn,vkP,nPQ,vLQ->vmkL", C_tan, Fe_tr, Bm, a)
    K += np.einsum("vmiJ,vmkL->viJkL", X, Y)
    if symmetric:
        K = 0.5 * (K + np.einsum("viJkL->vkLiJ", K))
    return np.moveaxis(K, 0, -1)


def finite_cp_material(cp: CrystalPlasticity, quats, grain_field, dt, tangent="held"):
    """Material closure of the finite-strain model; state = (Fp [V,3,3], T [V,6]).
    tangent: "held" (R18, the plastic state held; the library's tangent) or
    "consistent" (the symmetrised consistent tangent, finite_cp_tangent_consistent)."""
    g = grain_field.reshape(-1)
    S_full = schmid_full(cp, quats)

    def material(F, state):
        V = g.size
        Fv = np.moveaxis(F.reshape(3, 3, V), -1, 0)
        if state is None:
            state = (np.broadcast_to(np.eye(3), (V, 3, 3)).copy(), np.zeros((V, 6)))
        Fp_old, T_old = state
        P, Fp, T, data = finite_cp_update(cp, S_full, g, Fv, Fp_old, T_old, dt)
        Pf = np.moveaxis(P, 0, -1).reshape((3, 3) + grain_field.shape)
        Kv = finite_cp_tangent_consistent(data) if tangent == "consistent" else finite_cp_tangent(data)
        K = Kv.reshape((3, 3, 3, 3) + grain_field.shape)
        return Pf, FullTangent(K), (Fp, T)
    return material


# --------------------------------------------------------------------------
# Adjoint sensitivity of g : sigma_bar w.r.t. the per-voxel Young's modulus
# --------------------------------------------------------------------------

def adjoint_dJ_dE(prob: Problem, E_field, nu_field, eps_bar, g, tol=1e-12, max_iter=10000):
    """dJ/dE(x) for J = g : sigma_bar, linear isotropic C(x) = E(x) C1(nu(x)), strain control.

    Steps: forward solve K u = b(E); adjoint solve K lam = dJ/du, with
    dJ/du = (1/N) B^H C g (K is self-adjoint, Eq. lineqf's Hermitian form);
    then dJ/dE(x) = (1/N) g : C1 : eps(x) - (B lam)(x) : C1 : eps(x), the
    explicit dependence of J on E(x) minus lam^H d(K u - b)/dE(x).
    Returns (dJ/dE field, J).
    """
    if prob.ne:
        raise ValueError("adjoint is written for full strain control")
    lam1, mu1 = lame(np.ones_like(E_field), nu_field)
    C1 = IsoTangent(lam1, mu1)
    lam, mu = lame(E_field, nu_field)
    C = IsoTangent(lam, mu)
    fwd = solve_linear(prob, C, eps_bar, tol=tol, max_iter=max_iter)
    eps = fwd["eps"]
    J = float(np.sum(np.asarray(g) * fwd["sig_bar"]))
    gfield = np.broadcast_to(np.asarray(g, dtype=np.float64)[:, :, None, None, None], (3, 3) + prob.shape)
    qu, _ = prob.adjoint(C.apply(gfield.copy()))
    rhs = (qu / prob.N, np.zeros(0))
    M = prob.make_preconditioner(C.mean())
    lam_v, _, _ = pcg(prob, lambda v: prob.apply_K(C, v[0], v[1]), M, rhs, tol, max_iter)
    Blam = prob.field_from(lam_v[0], lam_v[1])
    c1eps = C1.apply(eps.copy())
    dJ = (np.einsum("ij,ij...->...", np.asarray(g), c1eps) / prob.N
          - np.einsum("ij...,ij...->...", Blam, c1eps))
    return dJ, J, fwd


def effective_stiffness_sensitivity(shape, E_field, nu_field, G, tol=1e-12, max_iter=10000):
    """dJ/dE(x) for J = sum_IJ G_IJ C_IJ, C the 6x6 Mandel effective stiffness
    of a linear isotropic C(x) = E(x) C1(nu(x)) (Sec. 2.2, the six unit strains).

    C_IJ = e_I : sigma_bar(e_J), so J = sum_J g_J : sigma_bar(e_J) with the
    tensor g_J = sum_I G_IJ e_I, and dJ/dE is the sum over J of the adjoint
    sensitivities of the six strain-controlled problems (adjoint_dJ_dE: a
    forward and an adjoint solve each). Returns (dJ/dE field, J, C).
    """
    prob = Problem(shape, "small")
    basis = mandel_basis()
    G = np.asarray(G, dtype=np.float64)
    dJ = np.zeros(prob.shape)
    Ceff = np.zeros((6, 6))
    for j in range(6):
        gj = np.einsum("i,ikl->kl", G[:, j], basis)
        dj, _, fwd = adjoint_dJ_dE(prob, E_field, nu_field, basis[j], gj, tol=tol, max_iter=max_iter)
        dJ += dj
        Ceff[:, j] = tensor_to_mandel(fwd["sig_bar"])
    return dJ, float(np.sum(G * Ceff)), Ceff


def homogenized_stress_linear(prob, E_field, nu_field, eps_bar, tol=1e-12):
    lam, mu = lame(E_field, nu_field)
    return solve_linear(prob, IsoTangent(lam, mu), eps_bar, tol=tol)["sig_bar"]
