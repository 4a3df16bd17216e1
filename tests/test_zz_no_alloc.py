"""The allocation-free operator entry point (dbfft_apply_iso_noalloc).

It serves callers that cannot let the library allocate device memory: hosts
whose GPU memory belongs to a caching pool, and callers that cannot afford
an allocation's latency and implicit synchronisation inside their own
iteration. Its work buffer lives in a static device array, so this test
checks that two calls in a row (the second finds the first call's leftovers
in the buffer) give the same K u as the context-based dbfft_apply, and that
requests larger than the buffer are refused before any device work.
Collected last so that a failure here cannot hide any other test.
"""
import numpy as np
import pytest

from paper_1905_12725_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _lame(E, nu):
    E = np.asarray(E, dtype=np.float64)
    nu = np.asarray(nu, dtype=np.float64)
    return E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))


def _reference(shape, phase, E, nu, u):
    from paper_1905_12725_gb300 import dbfft
    B = u.shape[0]
    s = dbfft.Solver(shape, phase, dbfft.iso_phases(E, nu), np.zeros((B, 3, 3)), batch=B)
    out, _ = s.apply(torch.from_numpy(u).cuda())
    s.close()
    return out.cpu().numpy()


def _noalloc(shape, phase, E, nu, u):
    from paper_1905_12725_gb300 import dbfft
    lam, mu = _lame(E, nu)
    ph = torch.from_numpy(phase.astype(np.int16)).cuda()
    lam_d = torch.from_numpy(lam).cuda()
    mu_d = torch.from_numpy(mu).cuda()
    ud = torch.from_numpy(u).cuda()
    out = torch.empty_like(ud)
    st = dbfft.apply_iso_noalloc(shape, ph, lam_d, mu_d, ud, out)
    assert st == 0
    return out.cpu().numpy()


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def test_noalloc_matches_dbfft_apply_on_consecutive_calls():
    g = np.random.default_rng(11)
    cases = [((16, 16, 16), 2, 101), ((8, 32, 16), 3, 102)]
    for shape, B, seed in cases:  # two calls in a row, different sizes
        phase = (g.random((B,) + shape) < 0.35).astype(np.uint16)
        E, nu = [1.0, 40.0], [0.3, 0.22]
        u = synth.random_spectrum(shape, 3, seed, batch=B)
        ref = _reference(shape, phase, E, nu, u)
        got = _noalloc(shape, phase, E, nu, u)
        assert _rel(got, ref) < 1e-12
    # and the first case again, after the buffer holds the second case's data
    shape, B, seed = cases[0]
    g2 = np.random.default_rng(12)
    phase = (g2.random((B,) + shape) < 0.5).astype(np.uint16)
    u = synth.random_spectrum(shape, 3, seed + 7, batch=B)
    assert _rel(_noalloc(shape, phase, [2.0, 5.0], [0.3, 0.3], u),
                _reference(shape, phase, [2.0, 5.0], [0.3, 0.3], u)) < 1e-12


def test_noalloc_refuses_sizes_beyond_its_buffer():
    from paper_1905_12725_gb300 import dbfft
    shape = (128, 128, 128)  # 6 * 128 * 128 * 65 * 16 bytes > 16 MiB
    small = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = dbfft.apply_iso_noalloc(shape, small, small, small, torch.zeros(1, 3, 1, 1, 1, dtype=torch.complex128,
                                                                         device="cuda"),
                                 torch.zeros(1, 3, 1, 1, 1, dtype=torch.complex128, device="cuda"))
    assert dbfft.STATUS[st] == "DBFFT_E_ARG"
