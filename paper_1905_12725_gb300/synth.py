"""Seeded synthetic microstructures and load programs for the DBFFT workloads.

This module only draws random numbers and paints voxel maps. It holds none of
the homogenization arithmetic (no frequencies, no FFTs, no constitutive law):
both the CUDA path and the FP64 CPU oracle consume the arrays it returns.

The paper (Sec. 3) builds its RVEs the same way -- spherical inclusions,
random pores, a Voronoi polycrystal with random orientations -- but prints no
data, so every workload here is synthetic and seeded.

Random numbers come from two published generators written out here:
SplitMix64 (Steele, Lea & Flood 2014) to expand a 64-bit seed, and
xoshiro256** (Blackman & Vigna 2018) for the stream. Doubles take the top 53
bits of a draw.  Voxel centres sit at x = (i + 1/2) h, box length 1, and all
distances are periodic minimum-image distances.
"""
from __future__ import annotations

import hashlib
import math

import numpy as np

SEED_BASE = 190512725
_M64 = (1 << 64) - 1


def _rotl(x: int, k: int) -> int:
    return ((x << k) | (x >> (64 - k))) & _M64


class Xoshiro256ss:
    """xoshiro256** seeded through SplitMix64 (both published generators)."""

    def __init__(self, seed: int):
        sm = seed & _M64
        s = []
        for _ in range(4):
            sm = (sm + 0x9E3779B97F4A7C15) & _M64
            z = sm
            z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
            z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
            s.append(z ^ (z >> 31))
        self.s = s

    def next_u64(self) -> int:
        s0, s1, s2, s3 = self.s
        result = (_rotl((s1 * 5) & _M64, 7) * 9) & _M64
        t = (s1 << 17) & _M64
        s2 ^= s0
        s3 ^= s1
        s1 ^= s2
        s0 ^= s3
        s2 ^= t
        s3 = _rotl(s3, 45)
        self.s = [s0, s1, s2, s3]
        return result

    def uniform(self) -> float:
        """Double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def uniforms(self, k: int) -> np.ndarray:
        return np.array([self.uniform() for _ in range(k)], dtype=np.float64)


def _axis_offsets(n: int, c: float) -> np.ndarray:
    """Periodic minimum-image offset (in voxels) of voxel centres i+1/2 from c."""
    d = (np.arange(n, dtype=np.float64) + 0.5) - c
    return d - n * np.round(d / n)


def paint_sphere(mask: np.ndarray, centre_vox, radius_vox: float) -> None:
    """Set every voxel whose centre lies within the periodic ball to True."""
    n1, n2, n3 = mask.shape
    d1 = _axis_offsets(n1, centre_vox[0])
    d2 = _axis_offsets(n2, centre_vox[1])
    d3 = _axis_offsets(n3, centre_vox[2])
    r2 = radius_vox * radius_vox
    # restrict to the bounding slab on each axis to keep this cheap
    i1 = np.nonzero(np.abs(d1) <= radius_vox)[0]
    i2 = np.nonzero(np.abs(d2) <= radius_vox)[0]
    i3 = np.nonzero(np.abs(d3) <= radius_vox)[0]
    dd = (d1[i1, None, None] ** 2 + d2[None, i2, None] ** 2 + d3[None, None, i3] ** 2) <= r2
    sub = mask[np.ix_(i1, i2, i3)]
    mask[np.ix_(i1, i2, i3)] = sub | dd


def centred_sphere(n: int, radius_vox: float) -> np.ndarray:
    """Phase map (uint16: 0 matrix, 1 inclusion) of one sphere at the box centre.

    With an even n and integer radius, (2d)^2 is a sum of three odd squares,
    which is 3 mod 8 and never equals (2r)^2, so no voxel centre sits on the
    sphere and the map is exact in integer arithmetic.
    """
    two_d = 2 * np.arange(n) + 1 - n  # twice the offset of the voxel centre
    s = two_d[:, None, None] ** 2 + two_d[None, :, None] ** 2 + two_d[None, None, :] ** 2
    return (s <= (2 * radius_vox) ** 2).astype(np.uint16)


def rsa_spheres(n: int, radius_vox: float, vf_target: float, rng: Xoshiro256ss,
                gap_vox: float = 1.0, max_tries: int = 200000):
    """Random sequential addition of non-overlapping spheres on an n^3 grid.

    Centres are uniform in the box; a candidate is rejected when its periodic
    centre distance to an accepted one is below 2r + gap. Adding stops once the
    painted voxel fraction reaches vf_target. Returns (phase map, centres).
    """
    mask = np.zeros((n, n, n), dtype=bool)
    centres = []
    dmin = 2.0 * radius_vox + gap_vox
    tries = 0
    while mask.mean() < vf_target:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("RSA could not reach the target volume fraction")
        c = np.array([rng.uniform() * n for _ in range(3)])
        ok = True
        for q in centres:
            d = c - q
            d -= n * np.round(d / n)
            if float(d @ d) < dmin * dmin:
                ok = False
                break
        if not ok:
            continue
        centres.append(c)
        paint_sphere(mask, c, radius_vox)
    return mask.astype(np.uint16), np.array(centres)


def boolean_spheroids(n: int, semi_axes_vox, vf_target: float, rng: Xoshiro256ss):
    """Boolean model (overlap allowed) of prolate spheroids with random axes.

    Each fibre has a uniform centre and an axis uniform on the unit sphere;
    fibres are added until the painted voxel fraction reaches vf_target.
    Returns (phase map, list of (centre, axis)).
    """
    a, b, _ = semi_axes_vox
    mask = np.zeros((n, n, n), dtype=bool)
    fibres = []
    reach = int(math.ceil(a)) + 1
    off = np.arange(-reach, reach + 1, dtype=np.float64)
    while mask.mean() < vf_target:
        c = np.array([rng.uniform() * n for _ in range(3)])
        zc = 2.0 * rng.uniform() - 1.0
        phi = 2.0 * math.pi * rng.uniform()
        rr = math.sqrt(max(0.0, 1.0 - zc * zc))
        ax = np.array([rr * math.cos(phi), rr * math.sin(phi), zc])
        fibres.append((c, ax))
        base = np.floor(c - 0.5).astype(np.int64)
        # voxel centres near the fibre, offsets relative to the fibre centre
        g = [base[k] + off.astype(np.int64) for k in range(3)]
        d = [(g[k] + 0.5) - c[k] for k in range(3)]
        D1, D2, D3 = np.meshgrid(d[0], d[1], d[2], indexing="ij")
        along = D1 * ax[0] + D2 * ax[1] + D3 * ax[2]
        perp2 = D1 * D1 + D2 * D2 + D3 * D3 - along * along
        inside = (along / a) ** 2 + perp2 / (b * b) <= 1.0
        idx = [np.mod(g[k], n) for k in range(3)]
        sub = mask[np.ix_(idx[0], idx[1], idx[2])]
        mask[np.ix_(idx[0], idx[1], idx[2])] = sub | inside
    return mask.astype(np.uint16), fibres


def boolean_spheres(n: int, radius_vox: float, vf_target: float, rng: Xoshiro256ss):
    """Boolean model (overlap allowed) of spheres with uniform centres.

    Spheres are added until the painted voxel fraction reaches vf_target.
    Unlike random sequential addition this reaches any fraction below one.
    Returns (phase map, centres).
    """
    mask = np.zeros((n, n, n), dtype=bool)
    centres = []
    while mask.mean() < vf_target:
        c = np.array([rng.uniform() * n for _ in range(3)])
        centres.append(c)
        paint_sphere(mask, c, radius_vox)
    return mask.astype(np.uint16), np.array(centres)


def uniform_quaternions(k: int, rng: Xoshiro256ss) -> np.ndarray:
    """k unit quaternions uniform on SO(3) (Shoemake's subgroup algorithm)."""
    q = np.empty((k, 4))
    for i in range(k):
        u1, u2, u3 = rng.uniform(), rng.uniform(), rng.uniform()
        a, b = math.sqrt(1.0 - u1), math.sqrt(u1)
        q[i] = (a * math.sin(2 * math.pi * u2), a * math.cos(2 * math.pi * u2),
                b * math.sin(2 * math.pi * u3), b * math.cos(2 * math.pi * u3))
    # order (w, x, y, z) with w >= 0
    q = q[:, [3, 0, 1, 2]]
    q[q[:, 0] < 0] *= -1.0
    return q


def periodic_voronoi(n: int, n_grains: int, rng: Xoshiro256ss):
    """Grain map (uint16) of the periodic Voronoi tessellation of uniform seeds.

    Every voxel centre takes the index of its periodic nearest seed. Seeds are
    continuous uniform doubles, so equal distances have probability zero.
    Returns (grain map, seeds in voxel units).
    """
    from scipy.spatial import cKDTree

    seeds = np.array([[rng.uniform() * n for _ in range(3)] for _ in range(n_grains)])
    seeds = np.mod(seeds, n)
    tree = cKDTree(seeds, boxsize=float(n))
    grains = np.empty((n, n, n), dtype=np.uint16)
    c = np.arange(n, dtype=np.float64) + 0.5
    for i in range(n):  # one slab at a time keeps memory modest at 256^3
        p = np.stack(np.meshgrid([c[i]], c, c, indexing="ij"), axis=-1).reshape(-1, 3)
        _, idx = tree.query(p)
        grains[i] = idx.reshape(n, n).astype(np.uint16)
    return grains, seeds


def sha256(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


# ---------------------------------------------------------------- workloads
def config1(n: int = 16, radius: int = 4):
    """Single centred spherical inclusion, E 1 / 10, nu 0.3, eps_xx = 1e-3."""
    phase = centred_sphere(n, radius)
    eps = np.zeros((3, 3))
    eps[0, 0] = 1e-3
    return dict(phase=phase, E=np.array([1.0, 10.0]), nu=np.array([0.3, 0.3]),
                eps_bar=eps)


def config2(n: int = 64, radius: float = 6.0, vf: float = 0.25, contrast: float = 100.0,
            seed: int = SEED_BASE + 2):
    """Random non-overlapping spheres, contrast 100; six unit Mandel strains."""
    rng = Xoshiro256ss(seed)
    phase, centres = rsa_spheres(n, radius, vf, rng)
    return dict(phase=phase, E=np.array([1.0, contrast]), nu=np.array([0.3, 0.3]),
                centres=centres)


def config3(n: int = 128, semi=(16.0, 4.0, 4.0), vf: float = 0.3, seed: int = SEED_BASE + 3):
    """Neo-Hookean matrix (mu 1) with Boolean prolate fibres (mu 20), nu 0.3."""
    rng = Xoshiro256ss(seed)
    phase, fibres = boolean_spheroids(n, semi, vf, rng)
    mu = np.array([1.0, 20.0])
    lam = 1.5 * mu  # nu = 0.3  <=>  lambda = 2 mu nu / (1 - 2 nu) = 1.5 mu
    return dict(phase=phase, mu=mu, lam=lam, n_fibres=len(fibres))


def config4(n: int = 256, n_grains: int = 500, seed: int = SEED_BASE + 4):
    """Periodic Voronoi polycrystal with uniformly random grain orientations."""
    rng = Xoshiro256ss(seed)
    grains, seeds = periodic_voronoi(n, n_grains, rng)
    quats = uniform_quaternions(n_grains, rng)
    return dict(phase=grains, quat=quats, seeds=seeds)


def config5(n: int = 64, n_rve: int = 32, radius: float = 6.0, seed: int = SEED_BASE + 5):
    """Independent random-sphere RVEs, vf ~ U[0.1, 0.4], contrast log-U[5, 200].

    Spheres may overlap (Boolean model): non-overlapping random sequential
    addition of radius-6 spheres jams near a voxel fraction of 0.3 on a 64^3
    grid, below the upper end of the requested range.
    """
    rng = Xoshiro256ss(seed)
    phases, E, vfs = [], [], []
    for _ in range(n_rve):
        vf = 0.1 + 0.3 * rng.uniform()
        contrast = math.exp(math.log(5.0) + (math.log(200.0) - math.log(5.0)) * rng.uniform())
        ph, _ = boolean_spheres(n, radius, vf, rng)
        phases.append(ph)
        E.append([1.0, contrast])
        vfs.append(vf)
    return dict(phase=np.stack(phases), E=np.array(E), nu=np.array([0.3, 0.3]),
                vf_target=np.array(vfs))


def inclusion(n: int = 63, vf: float = 0.2, contrast: float = 1.0, E: float = 70.0, nu: float = 0.3):
    """One centred spherical inclusion of volume fraction vf (Sec. 3, first and
    second benchmarks): matrix E, nu; inclusion contrast * E, same nu. The
    radius is the one of a ball of volume vf n^3 (voxels)."""
    r = n * (3.0 * vf / (4.0 * math.pi)) ** (1.0 / 3.0)
    return dict(phase=centred_sphere(n, r), E=np.array([E, contrast * E]), nu=np.array([nu, nu]), radius=r)


def porous_svk(n: int = 64, n_pores: int = 5, porosity: float = 0.2, E: float = 70.0, nu: float = 0.3,
               pore_ratio: float = 100.0, seed: int = SEED_BASE + 6, gap_vox: float = 1.0, max_tries: int = 100000):
    """Porous St. Venant-Kirchhoff matrix (Sec. 3, third benchmark).

    n_pores equal spherical pores of total volume fraction `porosity`, placed
    by random sequential addition (periodic centre distance >= 2r + gap). The
    pores are a compliant phase (stiffness E / pore_ratio, same nu), because
    the Fourier operators act on the whole box. Returns the phase map
    (0 matrix, 1 pore), the Lame constants per phase and the centres.
    """
    rng = Xoshiro256ss(seed)
    r = n * (3.0 * porosity / (4.0 * math.pi * n_pores)) ** (1.0 / 3.0)
    dmin = 2.0 * r + gap_vox
    centres = []
    tries = 0
    while len(centres) < n_pores:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place the pores without overlap")
        c = np.array([rng.uniform() * n for _ in range(3)])
        ok = True
        for q in centres:
            d = c - q
            d -= n * np.round(d / n)
            if float(d @ d) < dmin * dmin:
                ok = False
                break
        if ok:
            centres.append(c)
    mask = np.zeros((n, n, n), dtype=bool)
    for c in centres:
        paint_sphere(mask, c, r)
    Es = np.array([E, E / pore_ratio])
    lam = Es * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = Es / (2.0 * (1.0 + nu))
    return dict(phase=mask.astype(np.uint16), mu=mu, lam=lam, radius=r, centres=np.array(centres))


def random_voxels(n_vox: int, k: int, rng: Xoshiro256ss) -> np.ndarray:
    """k distinct voxel indices in [0, n_vox), drawn in order (for sampled checks)."""
    out = []
    seen = set()
    while len(out) < k:
        v = int(rng.uniform() * n_vox)
        if v not in seen:
            seen.add(v)
            out.append(v)
    return np.array(out, dtype=np.int64)


def random_spectrum(shape, n_comp: int, rng_seed: int, batch: int = 1) -> np.ndarray:
    """Random half-spectrum vector field [batch][n_comp][n1][n2][n3//2+1] (complex128).

    Drawn as a random real field and transformed with numpy's real FFT so the
    result is Hermitian-consistent on the k3 = 0 and k3 = n3/2 planes. No
    projection or masking of the method is applied here.
    """
    n1, n2, n3 = shape
    g = np.random.default_rng(rng_seed)
    real = g.standard_normal((batch, n_comp, n1, n2, n3))
    return np.fft.rfftn(real, axes=(-3, -2, -1))
