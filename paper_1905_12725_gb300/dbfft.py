"""ctypes binding of libdbfft (include/dbfft.h): argument marshalling only.

Every step of the DBFFT path runs in the CUDA library; this module converts
torch tensors and numpy arrays into the plain pointers and sizes of the C ABI.
PyTorch supplies device memory (through the allocator callbacks) and the
stream. There is no CPU fallback: if the library cannot be built or loaded,
the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

# ---------------------------------------------------------------- ABI mirror
DBFFT_OK = 0
STATUS = {0: "DBFFT_OK", 1: "DBFFT_E_ARG", 2: "DBFFT_E_UNSUPPORTED_GRID", 3: "DBFFT_E_NOMEM",
          4: "DBFFT_E_CUDA", 5: "DBFFT_E_NOT_CONVERGED", 6: "DBFFT_E_NONFINITE", 7: "DBFFT_E_TIMEOUT",
          8: "DBFFT_E_MATERIAL", 9: "DBFFT_E_STATE"}
DBFFT_SMALL, DBFFT_FINITE = 0, 1
DBFFT_FP64, DBFFT_MIXED = 0, 1
DBFFT_ISO_ELASTIC, DBFFT_NEO_HOOKE, DBFFT_CP_FCC_POWERLAW, DBFFT_SVK, DBFFT_CP_FCC_FINITE = 0, 1, 2, 3, 4
DBFFT_PRECOND_PER_INCREMENT, DBFFT_PRECOND_INITIAL, DBFFT_PRECOND_PER_NEWTON = 0, 1, 2
DBFFT_APPLY_FP32, DBFFT_APPLY_PRECOND, DBFFT_APPLY_RESIDUAL = 1, 2, 4


class dbfft_grid(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("L", C.c_double * 3), ("batch", C.c_int), ("n_materials", C.c_int),
                ("kinematics", C.c_int), ("precision", C.c_int), ("tol", C.c_double), ("max_iter", C.c_int),
                ("newton_tol", C.c_double), ("load_tol", C.c_double), ("eta_inner", C.c_double),
                ("max_newton", C.c_int)]


class dbfft_phase(C.Structure):
    _fields_ = [("model", C.c_int), ("E", C.c_double), ("nu", C.c_double), ("mu", C.c_double),
                ("lambda_", C.c_double), ("C11", C.c_double), ("C12", C.c_double), ("C44", C.c_double),
                ("gdot0", C.c_double), ("m", C.c_double), ("tau_c", C.c_double), ("quat", C.c_double * 4)]


class dbfft_materials(C.Structure):
    _fields_ = [("phase_id", C.POINTER(C.c_uint16)), ("E_scale", C.POINTER(C.c_double)),
                ("n_phases", C.c_int), ("phases", C.POINTER(dbfft_phase)), ("device_arrays", C.c_int)]


class dbfft_load(C.Structure):
    _fields_ = [("stress_mask", C.c_uint), ("target", C.POINTER(C.c_double)), ("n_increments", C.c_int),
                ("total_time", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class dbfft_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


class dbfft_report(C.Structure):
    _fields_ = [("newton_iters", C.c_int), ("outer_iters", C.c_int), ("cg_iters", C.c_longlong),
                ("cg_iters_max", C.c_int), ("eps_eq", C.c_double), ("load_res", C.c_double),
                ("true_rel_res", C.c_double), ("wall_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class dbfft_profile_entry(C.Structure):
    _fields_ = [("name", C.c_char * 40), ("launches", C.c_longlong), ("ms", C.c_double), ("bytes", C.c_double)]


EXPORTS = ["dbfft_create", "dbfft_apply", "dbfft_solve_increment", "dbfft_homogenized_stress",
           "dbfft_homogenized_tangent", "dbfft_adjoint", "dbfft_get_solution", "dbfft_device_bytes",
           "dbfft_destroy", "dbfft_last_error", "dbfft_status_string", "dbfft_profile",
           "dbfft_profile_read", "dbfft_launch_count", "dbfft_apply_iso_noalloc", "dbfft_autotune",
           "dbfft_tuning", "dbfft_set_pass3_shape", "dbfft_set_pass3_rhs_group", "dbfft_set_precond_refresh",
           "dbfft_displacement", "dbfft_compatibility",
           "dbfft_tangent_sensitivity", "dbfft_set_checkpointing", "dbfft_cp_adjoint",
           "dbfft_fp64_fma_rate", "dbfft_l2_copy_rate"]

_LIB = None


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Load libdbfft.so (building it with nvcc when absent). Raises if impossible."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"libdbfft.so not built ({path}); run __graft_entry__.build()")
        path = _build.build()
    lib = C.CDLL(path)
    vp, ip, dp = C.c_void_p, C.c_int, C.POINTER(C.c_double)
    lib.dbfft_create.argtypes = [C.POINTER(dbfft_grid), C.POINTER(dbfft_materials), C.POINTER(dbfft_load),
                                 C.POINTER(dbfft_allocator), vp, C.POINTER(vp)]
    lib.dbfft_create.restype = ip
    lib.dbfft_apply.argtypes = [vp, ip, vp, vp, vp, vp]
    lib.dbfft_apply.restype = ip
    lib.dbfft_solve_increment.argtypes = [vp, ip, C.POINTER(dbfft_report)]
    lib.dbfft_solve_increment.restype = ip
    lib.dbfft_homogenized_stress.argtypes = [vp, dp]
    lib.dbfft_homogenized_stress.restype = ip
    lib.dbfft_homogenized_tangent.argtypes = [vp, dp, C.POINTER(dbfft_report)]
    lib.dbfft_homogenized_tangent.restype = ip
    lib.dbfft_adjoint.argtypes = [vp, dp, vp, C.POINTER(dbfft_report)]
    lib.dbfft_adjoint.restype = ip
    lib.dbfft_get_solution.argtypes = [vp, vp, dp]
    lib.dbfft_get_solution.restype = ip
    lib.dbfft_device_bytes.argtypes = [vp]
    lib.dbfft_device_bytes.restype = C.c_size_t
    lib.dbfft_destroy.argtypes = [vp]
    lib.dbfft_destroy.restype = None
    lib.dbfft_last_error.argtypes = [vp]
    lib.dbfft_last_error.restype = C.c_char_p
    lib.dbfft_status_string.argtypes = [ip]
    lib.dbfft_status_string.restype = C.c_char_p
    lib.dbfft_profile.argtypes = [vp, ip]
    lib.dbfft_profile.restype = ip
    lib.dbfft_profile_read.argtypes = [vp, C.POINTER(dbfft_profile_entry), ip]
    lib.dbfft_profile_read.restype = ip
    lib.dbfft_launch_count.argtypes = [vp]
    lib.dbfft_launch_count.restype = C.c_longlong
    lib.dbfft_apply_iso_noalloc.argtypes = [C.POINTER(C.c_int), dp, ip, vp, ip, vp, vp, vp, vp, vp]
    lib.dbfft_apply_iso_noalloc.restype = ip
    lib.dbfft_autotune.argtypes = [vp, C.c_char_p]
    lib.dbfft_autotune.restype = ip
    lib.dbfft_tuning.argtypes = [vp]
    lib.dbfft_tuning.restype = C.c_char_p
    lib.dbfft_set_pass3_shape.argtypes = [vp, ip, ip, ip, ip]
    lib.dbfft_set_pass3_shape.restype = ip
    lib.dbfft_set_pass3_rhs_group.argtypes = [vp, ip]
    lib.dbfft_set_pass3_rhs_group.restype = ip
    lib.dbfft_set_precond_refresh.argtypes = [vp, ip]
    lib.dbfft_set_precond_refresh.restype = ip
    lib.dbfft_displacement.argtypes = [vp, vp]
    lib.dbfft_displacement.restype = ip
    lib.dbfft_compatibility.argtypes = [vp, dp]
    lib.dbfft_compatibility.restype = ip
    lib.dbfft_tangent_sensitivity.argtypes = [vp, dp, vp, dp, C.POINTER(dbfft_report)]
    lib.dbfft_tangent_sensitivity.restype = ip
    lib.dbfft_set_checkpointing.argtypes = [vp, ip]
    lib.dbfft_set_checkpointing.restype = ip
    lib.dbfft_cp_adjoint.argtypes = [vp, dp, vp, C.POINTER(dbfft_report)]
    lib.dbfft_cp_adjoint.restype = ip
    lib.dbfft_fp64_fma_rate.argtypes = [dp, vp]
    lib.dbfft_fp64_fma_rate.restype = ip
    lib.dbfft_l2_copy_rate.argtypes = [dp, vp]
    lib.dbfft_l2_copy_rate.restype = ip
    _LIB = lib
    return lib


class DbfftError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


# ---------------------------------------------------------------- materials
def iso_phases(E, nu):
    out = (dbfft_phase * len(E))()
    for i, (e, n) in enumerate(zip(E, nu)):
        out[i].model = DBFFT_ISO_ELASTIC
        out[i].E = float(e)
        out[i].nu = float(n)
    return out


def neo_hooke_phases(mu, lam):
    out = (dbfft_phase * len(mu))()
    for i, (m, l) in enumerate(zip(mu, lam)):
        out[i].model = DBFFT_NEO_HOOKE
        out[i].mu = float(m)
        out[i].lambda_ = float(l)
    return out


def svk_phases(mu, lam):
    """St. Venant-Kirchhoff phases from Lame constants (finite strain)."""
    out = (dbfft_phase * len(mu))()
    for i, (m, l) in enumerate(zip(mu, lam)):
        out[i].model = DBFFT_SVK
        out[i].mu = float(m)
        out[i].lambda_ = float(l)
    return out


def cp_phases(quats, C11=168000.0, C12=121000.0, C44=75000.0, gdot0=1e-3, m=0.05, tau_c=50.0,
              finite=False):
    """One FCC grain per quaternion; finite=True selects the finite-strain
    form (F = Fe Fp, FINITE kinematics) of the same crystal."""
    out = (dbfft_phase * len(quats))()
    for i, q in enumerate(quats):
        out[i].model = DBFFT_CP_FCC_FINITE if finite else DBFFT_CP_FCC_POWERLAW
        out[i].C11, out[i].C12, out[i].C44 = C11, C12, C44
        out[i].gdot0, out[i].m, out[i].tau_c = gdot0, m, tau_c
        for k in range(4):
            out[i].quat[k] = float(q[k])
    return out


def stress_mask_bits(mask) -> int:
    """9 booleans (index 3i+j) -> bit mask."""
    bits = 0
    for k, v in enumerate(np.asarray(mask, dtype=bool).reshape(-1)):
        if v:
            bits |= 1 << k
    return bits


# ---------------------------------------------------------------- context
class Solver:
    """One dbfft context on the current CUDA device and torch stream.

    phase: uint16 array [n_materials, n1, n2, n3] (or [n1, n2, n3]);
    phases: ctypes array from iso_phases / neo_hooke_phases / svk_phases / cp_phases
    (cp_phases(..., finite=True) for the finite-strain crystal);
    target: [batch, 3, 3] end-of-ramp macro targets; stress_mask: 9 booleans.
    """

    def __init__(self, shape, phase, phases, target, *, batch=None, kinematics=DBFFT_SMALL,
                 precision=DBFFT_FP64, stress_mask=None, n_increments=1, total_time=1.0, tol=1e-8,
                 max_iter=10000, newton_tol=1e-8, load_tol=1e-10, eta_inner=1e-4, max_newton=50,
                 E_scale=None, L=(1.0, 1.0, 1.0), stream=None, device=None):
        import torch

        self.torch = torch
        self.lib = load_library()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.shape = tuple(int(s) for s in shape)
        self.L = tuple(float(v) for v in L)
        # maps on the device (torch CUDA tensors) are handed over as device
        # pointers: the library copies them on the GPU, nothing crosses to the host
        dev_maps = isinstance(phase, torch.Tensor) and phase.is_cuda
        if dev_maps:
            ph = phase.contiguous()
            if ph.element_size() != 2 or ph.is_floating_point():
                raise ValueError("a device phase map must hold 2-byte integers")
            if ph.dim() == 3:
                ph = ph.unsqueeze(0)
        else:
            ph = np.ascontiguousarray(phase, dtype=np.uint16)
            if ph.ndim == 3:
                ph = ph[None]
        self.n_materials = ph.shape[0]
        tgt = np.ascontiguousarray(np.asarray(target, dtype=np.float64).reshape(-1, 9))
        self.batch = int(batch if batch is not None else tgt.shape[0])
        if tgt.shape[0] != self.batch:
            raise ValueError("target must hold one 3x3 tensor per right-hand side")
        g = dbfft_grid()
        for k in range(3):
            g.n[k] = self.shape[k]
            g.L[k] = float(L[k])
        g.batch, g.n_materials = self.batch, self.n_materials
        g.kinematics, g.precision = kinematics, precision
        g.tol, g.max_iter, g.newton_tol, g.load_tol = tol, max_iter, newton_tol, load_tol
        g.eta_inner, g.max_newton = eta_inner, max_newton
        self.kinematics, self.precision = kinematics, precision
        self._keep = [ph, tgt, phases]
        mat = dbfft_materials()
        if dev_maps:
            mat.device_arrays = 1
            mat.phase_id = C.cast(C.c_void_p(ph.data_ptr()), C.POINTER(C.c_uint16))
            if E_scale is not None:
                es = torch.as_tensor(E_scale, dtype=torch.float64, device=ph.device).reshape(tuple(ph.shape))
                es = es.contiguous()
                self._keep.append(es)
                mat.E_scale = C.cast(C.c_void_p(es.data_ptr()), C.POINTER(C.c_double))
        else:
            mat.phase_id = ph.ctypes.data_as(C.POINTER(C.c_uint16))
            if E_scale is not None:
                if isinstance(E_scale, torch.Tensor):
                    E_scale = E_scale.detach().cpu().numpy()
                es = np.ascontiguousarray(E_scale, dtype=np.float64).reshape(ph.shape)
                self._keep.append(es)
                mat.E_scale = _dptr(es)
        mat.n_phases = len(phases)
        mat.phases = C.cast(phases, C.POINTER(dbfft_phase))
        ld = dbfft_load()
        ld.stress_mask = stress_mask_bits(stress_mask) if stress_mask is not None else 0
        ld.target = _dptr(tgt)
        ld.n_increments = n_increments
        ld.total_time = total_time
        # device memory from torch's caching allocator
        self._blocks = {}
        dev = self.device

        def _alloc(nbytes, user):
            t = torch.empty(int(nbytes), dtype=torch.uint8, device=dev)
            self._blocks[t.data_ptr()] = t
            return t.data_ptr()

        def _free(ptr, user):
            self._blocks.pop(ptr, None)

        self._alloc_cb = ALLOC_FN(_alloc)
        self._free_cb = FREE_FN(_free)
        al = dbfft_allocator(self._alloc_cb, self._free_cb, None)
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        ctx = C.c_void_p()
        st = self.lib.dbfft_create(C.byref(g), C.byref(mat), C.byref(ld), C.byref(al),
                                   C.c_void_p(self.stream.cuda_stream), C.byref(ctx))
        if st != DBFFT_OK:
            raise DbfftError(st, "dbfft_create failed (see stderr)")
        self.ctx = ctx
        n1, n2, n3 = self.shape
        self.half = (n1, n2, n3 // 2 + 1)

    # -- helpers
    def _check(self, st):
        if st != DBFFT_OK:
            raise DbfftError(st, self.lib.dbfft_last_error(self.ctx).decode())

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.dbfft_destroy(self.ctx)
            self.ctx = None
            self._blocks.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def device_bytes(self) -> int:
        return int(self.lib.dbfft_device_bytes(self.ctx))

    def autotune(self, cache_path=None):
        """Pick launch shapes by timing them (dbfft_autotune); returns the choice as text."""
        if cache_path is None:
            cache_path = os.environ.get("DBFFT_TUNE_CACHE")
        p = cache_path.encode() if cache_path else None
        self._check(self.lib.dbfft_autotune(self.ctx, p))
        return self.lib.dbfft_tuning(self.ctx).decode()

    def set_pass3_shape(self, fp64, pipelined, radix, lines):
        """Fix pass 3's launch shape for one inner precision (dbfft_set_pass3_shape)."""
        self._check(self.lib.dbfft_set_pass3_shape(self.ctx, int(fp64), int(pipelined), int(radix), int(lines)))

    def set_pass3_rhs_group(self, rhs):
        """Right-hand sides per CTA of the line-bulk pass 3 (dbfft_set_pass3_rhs_group); 0 = default."""
        self._check(self.lib.dbfft_set_pass3_rhs_group(self.ctx, int(rhs)))

    def set_precond_refresh(self, policy):
        """Preconditioner refresh policy of the nonlinear models (dbfft_set_precond_refresh)."""
        self._check(self.lib.dbfft_set_precond_refresh(self.ctx, int(policy)))

    def launch_count(self) -> int:
        return int(self.lib.dbfft_launch_count(self.ctx))

    def profile(self, enable=True):
        self._check(self.lib.dbfft_profile(self.ctx, 1 if enable else 0))

    def profile_read(self):
        rows = (dbfft_profile_entry * 64)()
        n = self.lib.dbfft_profile_read(self.ctx, rows, 64)
        return {rows[i].name.decode(): dict(launches=rows[i].launches, ms=rows[i].ms, bytes=rows[i].bytes)
                for i in range(min(n, 64))}

    # -- entry points
    def apply(self, u_hat, e=None, *, fp32=False, precond=False, residual=False):
        """out = K u (or M u, or b - K u); u_hat torch complex [B,3,n1,n2,h] on the device."""
        torch = self.torch
        flags = (DBFFT_APPLY_FP32 if fp32 else 0) | (DBFFT_APPLY_PRECOND if precond else 0) | \
                (DBFFT_APPLY_RESIDUAL if residual else 0)
        dt = torch.complex64 if fp32 else torch.complex128
        u = u_hat.to(device=self.device, dtype=dt).contiguous()
        out = torch.empty_like(u)
        e_in = None if e is None else e.to(device=self.device, dtype=torch.float64).contiguous()
        e_out = torch.zeros(self.batch, 9, dtype=torch.float64, device=self.device)
        st = self.lib.dbfft_apply(self.ctx, flags, C.c_void_p(u.data_ptr()),
                                  C.c_void_p(e_in.data_ptr()) if e_in is not None else None,
                                  C.c_void_p(out.data_ptr()), C.c_void_p(e_out.data_ptr()))
        self._check(st)
        return out, e_out

    def solve_increment(self, inc=0, allow_not_converged=False):
        rep = dbfft_report()
        st = self.lib.dbfft_solve_increment(self.ctx, int(inc), C.byref(rep))
        if not (allow_not_converged and st == 5):
            self._check(st)
        d = rep.as_dict()
        d["status"] = STATUS.get(st, st)
        return d

    def homogenized_stress(self):
        out = np.zeros((self.batch, 9))
        self._check(self.lib.dbfft_homogenized_stress(self.ctx, _dptr(out)))
        return out.reshape(self.batch, 3, 3)

    def homogenized_tangent(self):
        out = np.zeros((self.n_materials, 6, 6))
        rep = dbfft_report()
        self._check(self.lib.dbfft_homogenized_tangent(self.ctx, _dptr(out), C.byref(rep)))
        return out, rep.as_dict()

    def adjoint(self, dJ_dsigma):
        torch = self.torch
        g = np.ascontiguousarray(np.asarray(dJ_dsigma, dtype=np.float64).reshape(self.batch, 9))
        out = torch.empty((self.batch,) + self.shape, dtype=torch.float64, device=self.device)
        rep = dbfft_report()
        self._check(self.lib.dbfft_adjoint(self.ctx, _dptr(g), C.c_void_p(out.data_ptr()), C.byref(rep)))
        return out, rep.as_dict()

    def tangent_sensitivity(self, G):
        """dJ/dE(x) for J = sum_IJ G_IJ C_IJ per material map (dbfft_tangent_sensitivity).

        G: [n_materials, 6, 6] Mandel weights. Returns (dJ/dE device tensor
        [n_materials, n1, n2, n3], C_eff [n_materials, 6, 6], report)."""
        torch = self.torch
        g = np.ascontiguousarray(np.asarray(G, dtype=np.float64).reshape(self.n_materials, 6, 6))
        out = torch.empty((self.n_materials,) + self.shape, dtype=torch.float64, device=self.device)
        C_eff = np.zeros((self.n_materials, 6, 6))
        rep = dbfft_report()
        self._check(self.lib.dbfft_tangent_sensitivity(self.ctx, _dptr(g), C.c_void_p(out.data_ptr()), _dptr(C_eff),
                                                       C.byref(rep)))
        return out, C_eff, rep.as_dict()

    def set_checkpointing(self, enable=True):
        """Keep every converged crystal-plasticity increment (dbfft_set_checkpointing)."""
        self._check(self.lib.dbfft_set_checkpointing(self.ctx, 1 if enable else 0))

    def cp_adjoint(self, dJ_dsigma):
        """dJ/ds(x) over the solved increments (dbfft_cp_adjoint); dJ_dsigma [batch, 3, 3]."""
        torch = self.torch
        g = np.ascontiguousarray(np.asarray(dJ_dsigma, dtype=np.float64).reshape(self.batch, 9))
        out = torch.empty((self.batch,) + self.shape, dtype=torch.float64, device=self.device)
        rep = dbfft_report()
        self._check(self.lib.dbfft_cp_adjoint(self.ctx, _dptr(g), C.c_void_p(out.data_ptr()), C.byref(rep)))
        return out, rep.as_dict()

    def get_solution(self):
        torch = self.torch
        u = torch.empty((self.batch, 3) + self.half, dtype=torch.complex128, device=self.device)
        e = np.zeros((self.batch, 9))
        self._check(self.lib.dbfft_get_solution(self.ctx, C.c_void_p(u.data_ptr()), _dptr(e)))
        return u, e

    def compatibility(self):
        """Compatibility residual per right-hand side (dbfft_compatibility), numpy [B]."""
        out = np.zeros(self.batch)
        self._check(self.lib.dbfft_compatibility(self.ctx, _dptr(out)))
        return out

    def save_deformed_shape(self, path, scale=1.0, rhs=0):
        """Write the deformed voxel-centre positions x + scale * u(x) of one right-hand side
        as a raw little-endian float64 array [3, n1, n2, n3] (C order) at `path`, with a
        JSON sidecar `path + '.json'` giving shape, dtype, box lengths and scale. u comes from
        dbfft_displacement; the positions are formed on the host for the file."""
        import json
        u = self.displacement()[rhs].cpu().numpy()
        x = [(np.arange(n) + 0.5) * (Lk / n) for n, Lk in zip(self.shape, self.L)]
        X = np.stack(np.meshgrid(*x, indexing="ij"))
        pos = np.ascontiguousarray(X + scale * u, dtype="<f8")
        pos.tofile(path)
        with open(str(path) + ".json", "w") as f:
            json.dump({"shape": [3] + list(self.shape), "dtype": "float64", "order": "C",
                       "box": list(self.L), "scale": float(scale), "rhs": int(rhs),
                       "content": "x + scale * u at the voxel centres x = (i + 1/2) L / n"}, f)
        return pos.shape

    def displacement(self):
        """Total displacement at the voxel centres, device float64 [B, 3, n1, n2, n3]."""
        torch = self.torch
        out = torch.empty((self.batch, 3) + tuple(self.shape), dtype=torch.float64, device=self.device)
        self._check(self.lib.dbfft_displacement(self.ctx, C.c_void_p(out.data_ptr())))
        return out


def apply_iso_noalloc(shape, phase_id, lam, mu, u_hat, out, L=None, stream=None):
    """out = K u_hat through dbfft_apply_iso_noalloc (no device allocation in the call).

    phase_id: contiguous 2-byte CUDA tensor [B, n1, n2, n3] (uint16 values; an
    int16 view is fine); lam, mu: contiguous float64 CUDA tensors [n_phases];
    u_hat, out: contiguous complex128 CUDA tensors [B, 3, n1, n2, n3//2 + 1].
    Every tensor is checked against `shape` before the call (ValueError
    otherwise), because the C entry point only sees raw device addresses.
    Returns the status code (0 on success; DBFFT_E_ARG for a phase id at or
    beyond n_phases, found by the library on the device).
    """
    import torch

    shape = tuple(int(v) for v in shape)
    if len(shape) != 3:
        raise ValueError("shape must have three entries")
    B = int(u_hat.shape[0]) if u_hat.dim() > 0 else 0
    half = (B, 3, shape[0], shape[1], shape[2] // 2 + 1)

    def need(cond, what):
        if not cond:
            raise ValueError(f"apply_iso_noalloc: {what}")

    for name, t in (("u_hat", u_hat), ("out", out)):
        need(t.is_cuda and t.dtype == torch.complex128 and t.is_contiguous(),
             f"{name} must be a contiguous complex128 CUDA tensor")
        need(tuple(t.shape) == half, f"{name} must have shape {half}")
    need(phase_id.is_cuda and phase_id.element_size() == 2 and phase_id.is_contiguous() and
         not phase_id.is_floating_point(), "phase_id must be a contiguous 2-byte integer CUDA tensor")
    need(phase_id.numel() == B * shape[0] * shape[1] * shape[2], "phase_id must hold B * n1 * n2 * n3 ids")
    for name, t in (("lam", lam), ("mu", mu)):
        need(t.is_cuda and t.dtype == torch.float64 and t.is_contiguous(),
             f"{name} must be a contiguous float64 CUDA tensor")
    need(lam.numel() == mu.numel() and lam.numel() >= 1, "lam and mu must have the same, non-zero length")
    need(len({t.device for t in (u_hat, out, phase_id, lam, mu)}) == 1, "all tensors must be on one device")

    lib = load_library()
    n = (C.c_int * 3)(*shape)
    Lh = None
    if L is not None:
        Larr = np.ascontiguousarray(L, dtype=np.float64)
        need(Larr.shape == (3,), "L must have three entries")
        Lh = _dptr(Larr)
    st = stream if stream is not None else torch.cuda.current_stream()
    return lib.dbfft_apply_iso_noalloc(n, Lh, B, C.c_void_p(phase_id.data_ptr()), int(lam.numel()),
                                       C.c_void_p(lam.data_ptr()), C.c_void_p(mu.data_ptr()),
                                       C.c_void_p(u_hat.data_ptr()), C.c_void_p(out.data_ptr()),
                                       C.c_void_p(st.cuda_stream))


def fp64_fma_rate(stream=None) -> float:
    """Measured FP64 FMA rate of the current GPU in TFLOP/s (dbfft_fp64_fma_rate)."""
    import torch

    v = C.c_double(0.0)
    st = stream if stream is not None else torch.cuda.current_stream()
    rc = load_library().dbfft_fp64_fma_rate(C.byref(v), C.c_void_p(st.cuda_stream))
    if rc != DBFFT_OK:
        raise DbfftError(rc, "dbfft_fp64_fma_rate failed")
    return v.value


def l2_copy_rate(stream=None) -> float:
    """Measured L2 copy bandwidth of the current GPU in GB/s (dbfft_l2_copy_rate)."""
    import torch

    v = C.c_double(0.0)
    st = stream if stream is not None else torch.cuda.current_stream()
    rc = load_library().dbfft_l2_copy_rate(C.byref(v), C.c_void_p(st.cuda_stream))
    if rc != DBFFT_OK:
        raise DbfftError(rc, "dbfft_l2_copy_rate failed")
    return v.value


def noalloc_last_error() -> str:
    """Message of the calling thread's last failed dbfft_apply_iso_noalloc call."""
    return load_library().dbfft_last_error(None).decode()


# ---------------------------------------------------------------- autograd
def homogenized_stress_fn():
    """torch.autograd.Function: <sigma>(E(x)) for linear isotropic RVEs, backward by the adjoint.

    forward(E_field [B, n1, n2, n3] float64, nu, eps_bar [B,3,3]) -> sigma_bar [B,3,3];
    backward returns dJ/dE(x) from dbfft_adjoint with dJ/dsigma = grad_output.
    """
    import torch

    class HomogenizedStress(torch.autograd.Function):
        last_adjoint_report = None  # report of the latest backward's dbfft_adjoint call

        @staticmethod
        def forward(ctx, E_field, nu, eps_bar, precision=DBFFT_FP64, tol=1e-10):
            B = E_field.shape[0]
            shape = tuple(E_field.shape[1:])
            # the field stays on the device: one phase (E = 1) scaled voxel by voxel by E(x)
            phase = torch.zeros((B,) + shape, dtype=torch.int16, device=E_field.device)
            s = Solver(shape, phase, iso_phases([1.0], [float(nu)]), eps_bar.detach().cpu().numpy().reshape(B, 9),
                       precision=precision, tol=tol, E_scale=E_field.detach().double().contiguous())
            s.solve_increment(0)
            sig = torch.as_tensor(s.homogenized_stress(), device=E_field.device)
            ctx.solver = s
            return sig

        @staticmethod
        def backward(ctx, grad_out):
            s = ctx.solver
            # the adjoint reuses the forward solution of this context (no second forward solve)
            dJ, rep = s.adjoint(grad_out.detach().cpu().numpy().reshape(s.batch, 9))
            HomogenizedStress.last_adjoint_report = rep
            s.close()
            return dJ.to(grad_out.device), None, None, None, None

    return HomogenizedStress


def effective_stiffness_fn():
    """torch.autograd.Function: C_eff(E(x)) for linear isotropic RVEs, backward by the
    stiffness sensitivity (the six unit-strain solves of the forward pass are reused).

    forward(E_field [Bm, n1, n2, n3] float64, nu) -> C_eff [Bm, 6, 6] (Mandel);
    backward returns dJ/dE(x) from dbfft_tangent_sensitivity with G = grad_output.
    """
    import torch

    class EffectiveStiffness(torch.autograd.Function):
        last_report = None  # report of the latest backward's sensitivity call

        @staticmethod
        def forward(ctx, E_field, nu, precision=DBFFT_FP64, tol=1e-10):
            Bm = E_field.shape[0]
            shape = tuple(E_field.shape[1:])
            phase = torch.zeros((Bm,) + shape, dtype=torch.int16, device=E_field.device)
            s = Solver(shape, phase, iso_phases([1.0], [float(nu)]), np.zeros((6 * Bm, 3, 3)), batch=6 * Bm,
                       precision=precision, tol=tol, E_scale=E_field.detach().double().contiguous())
            C_eff, _ = s.homogenized_tangent()
            ctx.solver = s
            return torch.as_tensor(C_eff, device=E_field.device)

        @staticmethod
        def backward(ctx, grad_out):
            s = ctx.solver
            dJ, _, rep = s.tangent_sensitivity(grad_out.detach().cpu().numpy())
            EffectiveStiffness.last_report = rep
            s.close()
            return dJ.to(grad_out.device), None, None, None

    return EffectiveStiffness
