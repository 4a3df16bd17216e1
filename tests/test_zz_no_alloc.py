"""The allocation-free operator entry point (dbfft_apply_iso_noalloc).

It serves callers that cannot let the library allocate device memory: hosts
whose GPU memory belongs to a caching pool (a framework that has reserved
most of the GPU), and callers that cannot afford an allocation's latency and
implicit synchronisation inside their own iteration. Its work buffer lives in
a static device array that every call shares, so these tests make two calls
in a row (the second finds the first call's leftovers in the buffer) and
check each against the FP64 oracle's K u (Sec. 2.2, Eq. lineqf in SPD form)
at the operator bar of 1e-12, and against the context-based dbfft_apply.
They also check that a call allocates no device memory, that a non-unit box
is honoured, that oversized requests and out-of-range phase ids are refused
with a message, and that the binding rejects tensors that do not match the
grid. Collected last so that a failure here cannot hide any other test.
"""
import numpy as np
import pytest

import oracle.dbfft_oracle as o
from paper_1905_12725_gb300 import synth
from tests.helpers import iso_tangent, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OP_TOL = 1e-12  # FP64 operator application against the oracle (max-norm relative)


def _lame(E, nu):
    E = np.asarray(E, dtype=np.float64)
    nu = np.asarray(nu, dtype=np.float64)
    return E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))


def _oracle(shape, phase, E, nu, u, L=(1.0, 1.0, 1.0)):
    prob = o.Problem(shape, L=L)
    return np.stack([prob.apply_K(iso_tangent(phase[b], E, nu), u[b], np.zeros(0))[0] for b in range(u.shape[0])])


def _context_apply(shape, phase, E, nu, u):
    from paper_1905_12725_gb300 import dbfft
    B = u.shape[0]
    s = dbfft.Solver(shape, phase, dbfft.iso_phases(E, nu), np.zeros((B, 3, 3)), batch=B)
    out, _ = s.apply(torch.from_numpy(u).cuda())
    s.close()
    return out.cpu().numpy()


def _device_inputs(phase, E, nu, u):
    lam, mu = _lame(E, nu)
    return (torch.from_numpy(phase.astype(np.int16)).cuda(), torch.from_numpy(lam).cuda(),
            torch.from_numpy(mu).cuda(), torch.from_numpy(u).cuda())


def _noalloc(shape, phase, E, nu, u, L=None):
    from paper_1905_12725_gb300 import dbfft
    ph, lam_d, mu_d, ud = _device_inputs(phase, E, nu, u)
    out = torch.empty_like(ud)
    st = dbfft.apply_iso_noalloc(shape, ph, lam_d, mu_d, ud, out, L=L)
    assert st == 0, dbfft.noalloc_last_error()
    return out.cpu().numpy()


def test_noalloc_matches_the_oracle_on_consecutive_calls():
    g = np.random.default_rng(11)
    cases = [((16, 16, 16), 2, 101), ((8, 32, 16), 3, 102)]
    for shape, B, seed in cases:  # two calls in a row, different sizes
        phase = (g.random((B,) + shape) < 0.35).astype(np.uint16)
        E, nu = [1.0, 40.0], [0.3, 0.22]
        u = synth.random_spectrum(shape, 3, seed, batch=B)
        got = _noalloc(shape, phase, E, nu, u)
        assert rel_err(got, _oracle(shape, phase, E, nu, u)) < OP_TOL
        assert rel_err(got, _context_apply(shape, phase, E, nu, u)) < OP_TOL
    # the first case again, after the buffer holds the second case's data
    shape, B, seed = cases[0]
    phase = (np.random.default_rng(12).random((B,) + shape) < 0.5).astype(np.uint16)
    u = synth.random_spectrum(shape, 3, seed + 7, batch=B)
    got = _noalloc(shape, phase, [2.0, 5.0], [0.3, 0.3], u)
    assert rel_err(got, _oracle(shape, phase, [2.0, 5.0], [0.3, 0.3], u)) < OP_TOL


def test_noalloc_honours_a_non_unit_box():
    shape, B = (16, 8, 32), 2
    L = (2.0, 1.0, 0.5)
    phase = (np.random.default_rng(13).random((B,) + shape) < 0.4).astype(np.uint16)
    E, nu = [1.0, 25.0], [0.3, 0.25]
    u = synth.random_spectrum(shape, 3, 103, batch=B)
    for _ in range(2):  # the second call reuses the uploaded tables of this box
        assert rel_err(_noalloc(shape, phase, E, nu, u, L=L), _oracle(shape, phase, E, nu, u, L=L)) < OP_TOL
    # and back to the unit box: the tables must be replaced
    assert rel_err(_noalloc(shape, phase, E, nu, u), _oracle(shape, phase, E, nu, u)) < OP_TOL


def test_noalloc_call_allocates_no_device_memory():
    from paper_1905_12725_gb300 import dbfft
    shape, B = (16, 16, 16), 2
    phase = (np.random.default_rng(14).random((B,) + shape) < 0.3).astype(np.uint16)
    ph, lam_d, mu_d, ud = _device_inputs(phase, [1.0, 9.0], [0.3, 0.3], synth.random_spectrum(shape, 3, 104, batch=B))
    out = torch.empty_like(ud)
    assert dbfft.apply_iso_noalloc(shape, ph, lam_d, mu_d, ud, out) == 0  # warm-up
    torch.cuda.synchronize()
    a0, r0 = torch.cuda.memory_allocated(), torch.cuda.memory_reserved()
    free0 = torch.cuda.mem_get_info()[0]
    assert dbfft.apply_iso_noalloc(shape, ph, lam_d, mu_d, ud, out) == 0
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == a0 and torch.cuda.memory_reserved() == r0
    assert torch.cuda.mem_get_info()[0] == free0  # no driver allocation either


def test_noalloc_refuses_sizes_beyond_its_buffer():
    from paper_1905_12725_gb300 import dbfft
    shape = (128, 128, 128)  # 6 * 128 * 128 * 65 * 16 bytes > 16 MiB
    lib = dbfft.load_library()
    import ctypes as C
    n = (C.c_int * 3)(*shape)
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")
    p = C.c_void_p(dummy.data_ptr())
    st = lib.dbfft_apply_iso_noalloc(n, None, 1, p, 1, p, p, p, C.c_void_p(dummy.data_ptr() + 16), None)
    assert dbfft.STATUS[st] == "DBFFT_E_ARG"
    assert "exceeds the static work buffer" in dbfft.noalloc_last_error()


def test_noalloc_reports_a_phase_id_beyond_n_phases():
    from paper_1905_12725_gb300 import dbfft
    shape, B = (8, 8, 8), 1
    phase = np.zeros((B,) + shape, np.uint16)
    phase[0, 3, 4, 5] = 2  # two phases given: id 2 is out of range
    ph, lam_d, mu_d, ud = _device_inputs(phase, [1.0, 3.0], [0.3, 0.3], synth.random_spectrum(shape, 3, 105, batch=B))
    out = torch.empty_like(ud)
    st = dbfft.apply_iso_noalloc(shape, ph, lam_d, mu_d, ud, out)
    assert dbfft.STATUS[st] == "DBFFT_E_ARG"
    assert "n_phases" in dbfft.noalloc_last_error()
    # the next valid call succeeds and clears the message
    phase[0, 3, 4, 5] = 1
    u = synth.random_spectrum(shape, 3, 106, batch=B)
    assert rel_err(_noalloc(shape, phase, [1.0, 3.0], [0.3, 0.3], u),
                   _oracle(shape, phase, [1.0, 3.0], [0.3, 0.3], u)) < OP_TOL
    assert dbfft.noalloc_last_error() == ""


def test_noalloc_binding_rejects_mismatched_tensors():
    from paper_1905_12725_gb300 import dbfft
    shape, B = (8, 8, 8), 1
    phase = np.zeros((B,) + shape, np.uint16)
    ph, lam_d, mu_d, ud = _device_inputs(phase, [1.0], [0.3], synth.random_spectrum(shape, 3, 107, batch=B))
    out = torch.empty_like(ud)
    with pytest.raises(ValueError):  # wrong grid for these tensors
        dbfft.apply_iso_noalloc((8, 8, 16), ph, lam_d, mu_d, ud, out)
    with pytest.raises(ValueError):  # non-contiguous output
        dbfft.apply_iso_noalloc(shape, ph, lam_d, mu_d, ud, torch.empty_like(ud).transpose(1, 2))
    with pytest.raises(ValueError):  # phase ids of the wrong width
        dbfft.apply_iso_noalloc(shape, ph.to(torch.int32), lam_d, mu_d, ud, out)
    with pytest.raises(ValueError):  # lam / mu of different lengths
        dbfft.apply_iso_noalloc(shape, ph, torch.cat([lam_d, lam_d]), mu_d, ud, out)
