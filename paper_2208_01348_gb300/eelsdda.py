"""Python binding of libeelsdda (ctypes).  Argument marshalling only: every
step of the computation runs in the CUDA library.  Function names follow
the C ABI in include/eelsdda.h.

Importing this module loads the in-tree shared library and raises if it is
missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libeelsdda.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"libeelsdda.so not built ({_LIB_PATH}); run __graft_entry__.build() or "
                      "python -m paper_2208_01348_gb300.build")
_lib = C.CDLL(_LIB_PATH)

EELS_OK = 0
EELS_E_INVALID_ARG = -1
EELS_E_BEAM_INSIDE = -2
EELS_E_THRESHOLD = -3
EELS_E_NOT_CONVERGED = -4
EELS_E_OOM = -5
EELS_E_CUDA = -6
EELS_E_TIMEOUT = -7
EELS_E_NO_GRID = -8
EELS_E_UNSUPPORTED = -9
EELS_FP64 = 0
EELS_MIXED = 1
EELS_QMR = 0
EELS_BICGSTAB = 1
EELS_QMR2 = 2
EELS_INT_POINT = 0
EELS_INT_IGT_SO = 1
EELS_POL_CM = 0
EELS_POL_IGT_SO = 1


class eels_c128(C.Structure):
    _fields_ = [("re", C.c_double), ("im", C.c_double)]


class eels_grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("d_nm", C.c_double),
                ("occ", C.POINTER(C.c_uint8)), ("origin_nm", C.c_double * 3)]


class eels_beam(C.Structure):
    _fields_ = [("x0_nm", C.c_double), ("y0_nm", C.c_double)]


class eels_opts(C.Structure):
    _fields_ = [("ekin_keV", C.c_double), ("precision", C.c_int), ("solver", C.c_int),
                ("eps_it", C.c_double), ("eps_inner", C.c_double), ("max_iter", C.c_int),
                ("n_dir", C.c_int), ("max_batch", C.c_int), ("inner_max_iter", C.c_int),
                ("beam_dir", C.c_double * 3), ("interaction", C.c_int), ("polarizability", C.c_int),
                ("device_loop", C.c_int)]


class eels_point_stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("refinements", C.c_int), ("residual", C.c_double), ("converged", C.c_int)]


class eels_server_opts(C.Structure):
    _fields_ = [("device", C.c_int), ("hbm_budget", C.c_size_t), ("max_concurrent", C.c_int), ("flags", C.c_int)]


class eels_job_info(C.Structure):
    _fields_ = [("state", C.c_int), ("code", C.c_int), ("t_submit", C.c_double), ("t_start", C.c_double),
                ("t_end", C.c_double), ("footprint", C.c_size_t), ("n_points", C.c_int)]


class eels_vacuum_map(C.Structure):
    _fields_ = [("ekin_keV", C.c_double), ("energy_eV", C.c_double), ("length_scale", C.c_double),
                ("eps_p_scale", C.c_double), ("p_scale", C.c_double)]


EELS_JOB_QUEUED, EELS_JOB_RUNNING, EELS_JOB_DONE, EELS_JOB_FAILED = 0, 1, 2, 3
EELS_SERVER_DRYRUN = 1

_P = C.c_void_p
_dp = C.POINTER(C.c_double)
_cp = C.POINTER(eels_c128)
_sig = {
    "eels_default_opts": (None, [C.POINTER(eels_opts)]),
    "eels_create": (C.c_int, [C.POINTER(_P), C.c_int, _P]),
    "eels_destroy": (None, [_P]),
    "eels_last_error": (C.c_char_p, [_P]),
    "eels_set_grid": (C.c_int, [_P, C.POINTER(eels_grid)]),
    "eels_num_dipoles": (C.c_int, [_P]),
    "eels_padded_dims": (C.c_int, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "eels_solve": (C.c_int, [_P, C.POINTER(eels_opts), C.c_int, _dp, C.c_int, _cp, _cp, C.c_int,
                             C.POINTER(eels_beam), _dp, _dp, _dp, _dp, _cp, C.POINTER(eels_point_stats)]),
    "eels_solve_async": (C.c_int, [_P, C.POINTER(eels_opts), C.c_int, _dp, C.c_int, _cp, _cp, C.c_int,
                                   C.POINTER(eels_beam), _dp, _dp, _dp, _dp, _cp, C.POINTER(eels_point_stats),
                                   C.POINTER(_P)]),
    "eels_job_poll": (C.c_int, [_P, C.POINTER(C.c_int)]),
    "eels_job_wait": (C.c_int, [_P]),
    "eels_query_footprint": (C.c_int, [C.POINTER(eels_grid), C.POINTER(eels_opts), C.c_int, C.POINTER(C.c_size_t)]),
    "eels_bessel_k01_dev": (C.c_int, [_P, _P, _P, C.c_int, _P]),
    "eels_incident_field": (C.c_int, [_P, C.c_double, C.c_double, eels_c128, eels_beam, _cp, _cp]),
    "eels_incident_field_dir": (C.c_int, [_P, C.c_double, C.c_double, eels_c128, eels_beam, _dp, _cp, _cp]),
    "eels_apply_matrix": (C.c_int, [_P, C.c_int, C.c_double, C.c_int, _cp, eels_c128, C.c_int, _cp, _cp]),
    "eels_directions": (C.c_int, [C.c_int, _dp, _dp]),
    "eels_prepare_operator": (C.c_int, [_P, C.c_int, _dp, C.c_int, _cp, _cp]),
    "eels_set_interaction": (C.c_int, [_P, C.c_int, C.c_int]),
    "eels_matvec_dev": (C.c_int, [_P, C.c_int, _P, _P, C.c_int, _P]),
    "eels_kernel_launches": (C.c_longlong, []),
    "eels_cl_total": (C.c_int, [C.c_int, _dp, _dp, _dp, _dp]),
    "eels_frank_tamm": (C.c_int, [C.c_double, eels_c128, _dp]),
    "eels_extrapolate": (C.c_int, [C.c_int, _dp, _dp, _dp, _dp]),
    "eels_vacuum_equivalent": (C.c_int, [C.c_int, C.c_double, C.c_double, C.c_double, C.POINTER(eels_vacuum_map)]),
    "eels_tile_widths": (C.c_int, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "eels_tuned_xpass": (C.c_int, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "eels_xpass_timings": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                     C.POINTER(C.c_float)]),
    "eels_matvec_dev_noalloc": (C.c_int, [_P, C.c_int, _P, _P, C.c_int, _P]),
    "eels_krylov_solve_dev": (C.c_int, [_P, C.c_int, C.c_int, _P, _P, C.c_int, C.c_double, C.c_int,
                                        C.POINTER(C.c_int), C.POINTER(C.c_int), _P]),
    "eels_solve_dev": (C.c_int, [_P, C.POINTER(eels_opts), C.c_int, _P, C.c_int, _P, _P, C.c_int, _P,
                                 _P, _P, _P, _P, _P, _P, _P]),
    "eels_server_create": (C.c_int, [C.POINTER(_P), C.POINTER(eels_server_opts)]),
    "eels_server_submit": (C.c_int, [_P, C.POINTER(eels_grid), C.POINTER(eels_opts), C.c_int, _dp, C.c_int, _cp, _cp,
                                     C.c_int, C.POINTER(eels_beam), C.POINTER(C.c_longlong)]),
    "eels_server_poll": (C.c_int, [_P, C.c_longlong, C.POINTER(eels_job_info)]),
    "eels_server_wait": (C.c_int, [_P, C.c_longlong, _dp, _dp, _dp, _dp, C.POINTER(eels_point_stats),
                                   C.POINTER(eels_job_info)]),
    "eels_server_stats": (C.c_int, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_size_t)]),
    "eels_server_destroy": (None, [_P]),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_sig)


class EelsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"eelsdda error {code}: {msg}")
        self.code = code


def _check(code: int, ctx=None):
    if code != EELS_OK:
        msg = _lib.eels_last_error(ctx).decode() if ctx else ""
        raise EelsError(code, msg)


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


def _cptr(a: np.ndarray):
    return a.ctypes.data_as(_cp)


def _dptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(_dp)


def eels_default_opts(**kw) -> eels_opts:
    o = eels_opts()
    _lib.eels_default_opts(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        if k == "beam_dir":
            v = (C.c_double * 3)(*[float(c) for c in v])
        setattr(o, k, v)
    return o


def eels_create(device: int = 0, stream: int = 0):
    h = _P()
    _check(_lib.eels_create(C.byref(h), device, _P(stream) if stream else None))
    return h


def eels_destroy(ctx) -> None:
    _lib.eels_destroy(ctx)


def eels_last_error(ctx) -> str:
    return _lib.eels_last_error(ctx).decode()


def _grid(occ: np.ndarray, d_nm: float, origin_nm=(0.0, 0.0, 0.0)):
    occ = np.ascontiguousarray(occ, dtype=np.uint8)
    nz, ny, nx = occ.shape
    g = eels_grid(nx, ny, nz, float(d_nm), occ.ctypes.data_as(C.POINTER(C.c_uint8)),
                  (C.c_double * 3)(*[float(v) for v in origin_nm]))
    return g, occ


def eels_set_grid(ctx, occ: np.ndarray, d_nm: float, origin_nm=(0.0, 0.0, 0.0)) -> None:
    """occ [nz][ny][nx] material indices; origin_nm: lattice centre in the beams' frame."""
    g, keep = _grid(occ, d_nm, origin_nm)
    _check(_lib.eels_set_grid(ctx, C.byref(g)), ctx)


def eels_num_dipoles(ctx) -> int:
    return _lib.eels_num_dipoles(ctx)


def eels_padded_dims(ctx):
    a, b, c = C.c_int(), C.c_int(), C.c_int()
    _check(_lib.eels_padded_dims(ctx, C.byref(a), C.byref(b), C.byref(c)), ctx)
    return a.value, b.value, c.value


@dataclass
class SolveResult:
    p_eels: np.ndarray
    p_cl: Optional[np.ndarray]
    p_ext: Optional[np.ndarray]
    p_abs: Optional[np.ndarray]
    p: Optional[np.ndarray]
    iters: np.ndarray
    refinements: np.ndarray
    residual: np.ndarray
    converged: np.ndarray
    code: int

    @property
    def p_cl_tot(self) -> Optional[np.ndarray]:
        """P_CL^tot (Eq. 41) when P_ext and P_CL were requested."""
        if self.p_ext is None or self.p_cl is None:
            return None
        return eels_cl_total(self.p_eels, self.p_ext, self.p_cl)


class _SolveCall:
    """Marshalled arguments and output buffers of one eels_solve call."""

    def __init__(self, ctx, opts, energies_eV, eps_p, eps_h, beams_nm, want_cl, want_ext, want_abs, want_p):
        self.e = np.ascontiguousarray(energies_eV, dtype=np.float64).ravel()
        ne = len(self.e)
        self.ep = _c128(eps_p).reshape(ne, -1)
        self.eh = _c128(eps_h).ravel()
        bm = np.ascontiguousarray(beams_nm, dtype=np.float64).reshape(-1, 2)
        nb = len(bm)
        self.beams = (eels_beam * nb)(*[eels_beam(float(x), float(y)) for x, y in bm])
        self.out = {k: np.zeros((ne, nb)) for k in ("eels", "cl", "ext", "abs")}
        self.want = (want_cl, want_ext, want_abs, want_p)
        n = eels_num_dipoles(ctx)
        self.p = np.zeros((ne, nb, n, 3), dtype=np.complex128) if want_p else None
        self.st = (eels_point_stats * (ne * nb))()
        self.shape = (ne, nb)
        self.opts = opts

    def args(self, ctx):
        o, (wc, we, wa, wp) = self.out, self.want
        return (ctx, C.byref(self.opts), self.shape[0], self.e.ctypes.data_as(_dp), self.ep.shape[1], _cptr(self.ep),
                _cptr(self.eh), self.shape[1], self.beams, _dptr(o["eels"]), _dptr(o["cl"]) if wc else None,
                _dptr(o["ext"]) if we else None, _dptr(o["abs"]) if wa else None, _cptr(self.p) if wp else None,
                self.st)

    def result(self, code, ctx, raise_not_converged):
        if code != EELS_OK and not (code == EELS_E_NOT_CONVERGED and not raise_not_converged):
            _check(code, ctx)
        ne, nb = self.shape
        wc, we, wa, _ = self.want
        sa = np.array([(s.iters, s.refinements, s.residual, s.converged) for s in self.st]).reshape(ne, nb, 4)
        o = self.out
        return SolveResult(o["eels"], o["cl"] if wc else None, o["ext"] if we else None, o["abs"] if wa else None,
                           self.p, sa[..., 0].astype(int), sa[..., 1].astype(int), sa[..., 2],
                           sa[..., 3].astype(bool), code)


def eels_solve(ctx, opts: eels_opts, energies_eV, eps_p, eps_h, beams_nm, want_cl=True, want_ext=True,
               want_abs=True, want_p=False, raise_not_converged=True) -> SolveResult:
    """energies [E]; eps_p [E][n_mat]; eps_h [E]; beams [B][2] -> arrays [E][B]."""
    call = _SolveCall(ctx, opts, energies_eV, eps_p, eps_h, beams_nm, want_cl, want_ext, want_abs, want_p)
    return call.result(_lib.eels_solve(*call.args(ctx)), ctx, raise_not_converged)


class SolveJob:
    """A running eels_solve_async; its buffers live until wait() returns."""

    def __init__(self, ctx, call: _SolveCall, handle):
        self._ctx, self._call, self._h = ctx, call, handle

    def poll(self) -> bool:
        d = C.c_int()
        _check(_lib.eels_job_poll(self._h, C.byref(d)))
        return bool(d.value)

    def wait(self, raise_not_converged=True) -> SolveResult:
        if self._h is None:
            raise RuntimeError("job already waited")
        code = _lib.eels_job_wait(self._h)
        self._h = None
        return self._call.result(code, self._ctx, raise_not_converged)


def eels_solve_async(ctx, opts: eels_opts, energies_eV, eps_p, eps_h, beams_nm, want_cl=True, want_ext=True,
                     want_abs=True, want_p=False) -> SolveJob:
    """Start eels_solve on a library thread; SolveJob.wait() returns its SolveResult."""
    call = _SolveCall(ctx, opts, energies_eV, eps_p, eps_h, beams_nm, want_cl, want_ext, want_abs, want_p)
    h = _P()
    _check(_lib.eels_solve_async(*call.args(ctx), C.byref(h)), ctx)
    return SolveJob(ctx, call, h)


def eels_query_footprint(occ: np.ndarray, d_nm: float, opts: eels_opts, n_systems: int) -> int:
    g, keep = _grid(occ, d_nm)
    b = C.c_size_t()
    _check(_lib.eels_query_footprint(C.byref(g), C.byref(opts), n_systems, C.byref(b)))
    return b.value


def eels_bessel_k01_dev(z_ptr: int, k0_ptr: int, k1_ptr: int, n: int, stream: int = 0) -> None:
    _check(_lib.eels_bessel_k01_dev(_P(z_ptr), _P(k0_ptr), _P(k1_ptr), n, _P(stream) if stream else None))


def eels_incident_field(ctx, ekin_keV: float, energy_eV: float, eps_h: complex, beam_nm, beam_dir=None):
    """E_inc and E_a at the dipoles (SI); beam_dir None: electron along +z."""
    n = eels_num_dipoles(ctx)
    e = np.zeros((n, 3), dtype=np.complex128)
    ea = np.zeros((n, 3), dtype=np.complex128)
    eh = complex(eps_h)
    bm = eels_beam(float(beam_nm[0]), float(beam_nm[1]))
    if beam_dir is None:
        code = _lib.eels_incident_field(ctx, ekin_keV, energy_eV, eels_c128(eh.real, eh.imag), bm, _cptr(e), _cptr(ea))
    else:
        dv = np.ascontiguousarray(beam_dir, dtype=np.float64)
        code = _lib.eels_incident_field_dir(ctx, ekin_keV, energy_eV, eels_c128(eh.real, eh.imag), bm, _dptr(dv),
                                            _cptr(e), _cptr(ea))
    _check(code, ctx)
    return e, ea


def eels_apply_matrix(ctx, precision: int, energy_eV: float, eps_p, eps_h: complex, x: np.ndarray) -> np.ndarray:
    """x [n_vec][N][3] (or [N][3]) -> A x in SI (m^-3 times the units of x)."""
    x = _c128(x)
    single = x.ndim == 2
    if single:
        x = x[None]
    y = np.zeros_like(x)
    ep = _c128(eps_p).ravel()
    eh = complex(eps_h)
    _check(_lib.eels_apply_matrix(ctx, precision, energy_eV, len(ep), _cptr(ep), eels_c128(eh.real, eh.imag),
                                  x.shape[0], _cptr(x), _cptr(y)), ctx)
    return y[0] if single else y


def eels_set_interaction(ctx, interaction: int = EELS_INT_POINT, polarizability: int = EELS_POL_CM) -> None:
    """Interaction term and polarizability of eels_apply_matrix / eels_prepare_operator."""
    _check(_lib.eels_set_interaction(ctx, int(interaction), int(polarizability)), ctx)


def eels_prepare_operator(ctx, energies_eV, eps_p, eps_h) -> None:
    e = np.ascontiguousarray(energies_eV, dtype=np.float64).ravel()
    ep = _c128(eps_p).reshape(len(e), -1)
    eh = _c128(eps_h).ravel()
    _check(_lib.eels_prepare_operator(ctx, len(e), e.ctypes.data_as(_dp), ep.shape[1], _cptr(ep), _cptr(eh)), ctx)


def eels_matvec_dev(ctx, precision: int, x_ptr: int, y_ptr: int, n_sys: int, stream: int = 0) -> None:
    _check(_lib.eels_matvec_dev(ctx, precision, _P(x_ptr), _P(y_ptr), n_sys, _P(stream) if stream else None), ctx)


def eels_krylov_solve_dev(ctx, precision: int, solver: int, b_ptr: int, x_ptr: int, n_sys: int, eps: float,
                          max_iter: int, stream: int = 0):
    """Krylov solve A' x = b on the prepared operator (device vectors [n_sys][3][N]);
    returns (status, iters) arrays [n_sys] (1 converged, 2 iteration limit, 3 breakdown)."""
    st = (C.c_int * n_sys)()
    it = (C.c_int * n_sys)()
    _check(_lib.eels_krylov_solve_dev(ctx, precision, solver, _P(b_ptr), _P(x_ptr), n_sys, float(eps), int(max_iter),
                                      st, it, _P(stream) if stream else None), ctx)
    return np.array(st[:], dtype=int), np.array(it[:], dtype=int)


def eels_solve_dev(ctx, opts: eels_opts, energies, eps_p, eps_h, beams, p_eels, p_cl=None, p_ext=None, p_abs=None,
                   p_out=None, stats=None, stream: int = 0) -> int:
    """eels_solve on device buffers: every array argument is a torch CUDA
    tensor (energies float64 [E]; eps_p complex128 [E][n_mat]; eps_h complex128
    [E]; beams float64 [B][2]; outputs float64 [E][B], p_out complex128
    [E][B][N][3], stats: a uint8 tensor of E*B*sizeof(eels_point_stats) bytes).
    Returns the eels_solve code (EELS_OK or EELS_E_NOT_CONVERGED); raises on
    other errors."""
    def ptr(t):
        if t is None:
            return None
        if not t.is_contiguous():
            raise ValueError("eels_solve_dev: tensors must be contiguous")
        return _P(t.data_ptr())
    ne = int(energies.numel())
    n_mat = int(eps_p.numel()) // ne
    nb = int(beams.numel()) // 2
    code = _lib.eels_solve_dev(ctx, C.byref(opts), ne, ptr(energies), n_mat, ptr(eps_p), ptr(eps_h), nb, ptr(beams),
                               ptr(p_eels), ptr(p_cl), ptr(p_ext), ptr(p_abs), ptr(p_out), ptr(stats),
                               _P(stream) if stream else None)
    if code not in (EELS_OK, EELS_E_NOT_CONVERGED):
        _check(code, ctx)
    return code


EELS_NOALLOC_SCRATCH_BYTES = 64 << 20


def eels_matvec_dev_noalloc(ctx, precision: int, x_ptr: int, y_ptr: int, n_sys: int, stream: int = 0) -> None:
    """eels_matvec_dev without any device allocation: the FFT scratch is a
    fixed 64 MiB array inside the library, shared by every call on a device
    (serialise overlapping calls; make the first call on a device before any
    stream capture)."""
    _check(_lib.eels_matvec_dev_noalloc(ctx, precision, _P(x_ptr), _P(y_ptr), n_sys, _P(stream) if stream else None),
           ctx)


def eels_cl_total(p_eels, p_ext, p_cl) -> np.ndarray:
    """P_CL^tot (Eq. 41) from the three probabilities (same shapes)."""
    a, b, c = (np.ascontiguousarray(v, dtype=np.float64) for v in (p_eels, p_ext, p_cl))
    out = np.empty_like(a)
    _check(_lib.eels_cl_total(a.size, _dptr(a), _dptr(b), _dptr(c), _dptr(out)))
    return out


def eels_frank_tamm(ekin_keV: float, eps_h: complex) -> float:
    """Host-only loss per unit path length, eV^-1 m^-1 (Eq. 29; 0 below threshold)."""
    r = C.c_double()
    _check(_lib.eels_frank_tamm(float(ekin_keV), eels_c128(complex(eps_h).real, complex(eps_h).imag), C.byref(r)))
    return r.value


def eels_extrapolate(d, values):
    """(value at d = 0, 95 % half-width) from results at dipole sizes d (Sec. 3.2)."""
    dd_ = np.ascontiguousarray(d, dtype=np.float64)
    vv = np.ascontiguousarray(values, dtype=np.float64)
    v0, ci = C.c_double(), C.c_double()
    _check(_lib.eels_extrapolate(len(dd_), _dptr(dd_), _dptr(vv), C.byref(v0), C.byref(ci)))
    return v0.value, ci.value


EELS_SCALE_ENERGY, EELS_SCALE_LENGTH, EELS_SCALE_ULTRAREL = 0, 1, 2


def eels_vacuum_equivalent(ekin_keV: float, eps_h: float, energy_eV: float, rule: int = EELS_SCALE_ENERGY) -> dict:
    """Vacuum problem equivalent to a particle in the real host eps_h (Sec. 2.7:
    Eq. 45 / 46, or with EELS_SCALE_ULTRAREL the approximate Eq. S16 above the
    threshold).  Keys: ekin_keV (inf for v = c), energy_eV, length_scale,
    eps_p_scale (applied to eps_p at the original energy), p_scale
    (P_host = p_scale * P_vacuum)."""
    m = eels_vacuum_map()
    _check(_lib.eels_vacuum_equivalent(int(rule), float(ekin_keV), float(eps_h), float(energy_eV), C.byref(m)))
    return {f: getattr(m, f) for f, _ in eels_vacuum_map._fields_}


def eels_tile_widths(ctx):
    """(FP32, FP64) x-pass tile widths timed on the first solve of the grid (0: not yet)."""
    a, b = C.c_int(), C.c_int()
    _check(_lib.eels_tile_widths(ctx, C.byref(a), C.byref(b)), ctx)
    return a.value, b.value


def eels_tuned_xpass(ctx):
    """(mode, beams per block) timed for the register x pass (0, 0: not yet / not used)."""
    a, b = C.c_int(), C.c_int()
    _check(_lib.eels_tuned_xpass(ctx, C.byref(a), C.byref(b)), ctx)
    return a.value, b.value


def eels_xpass_timings(ctx):
    """[(mode, beams per block, ms)] of every register x-pass candidate timed for the grid shape."""
    n = C.c_int()
    _check(_lib.eels_xpass_timings(ctx, 0, C.byref(n), None, None, None), ctx)
    k = n.value
    if k == 0:
        return []
    m, b, t = (C.c_int * k)(), (C.c_int * k)(), (C.c_float * k)()
    _check(_lib.eels_xpass_timings(ctx, k, C.byref(n), m, b, t), ctx)
    return [(m[i], b[i], float(t[i])) for i in range(min(k, n.value))]


def eels_kernel_launches() -> int:
    return int(_lib.eels_kernel_launches())


def eels_directions(n_dir: int = 2562):
    d = np.zeros((n_dir, 3))
    w = np.zeros(n_dir)
    _check(_lib.eels_directions(n_dir, _dptr(d), _dptr(w)))
    return d, w


class Context:
    """Owns one eels_ctx (RAII convenience over the functions above)."""

    def __init__(self, device: int = 0, stream: int = 0):
        self.h = eels_create(device, stream)

    def close(self):
        if self.h:
            eels_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- serving loop
def eels_server_create(device: int = 0, hbm_budget: int = 0, max_concurrent: int = 4, flags: int = 0):
    h = _P()
    o = eels_server_opts(device, hbm_budget, max_concurrent, flags)
    _check(_lib.eels_server_create(C.byref(h), C.byref(o)))
    return h


def eels_server_submit(srv, occ: np.ndarray, d_nm: float, opts: eels_opts, energies_eV, eps_p, eps_h, beams_nm,
                       origin_nm=(0.0, 0.0, 0.0)) -> int:
    g, keep = _grid(occ, d_nm, origin_nm)
    e = np.ascontiguousarray(energies_eV, dtype=np.float64).ravel()
    ep = _c128(eps_p).reshape(len(e), -1)
    eh = _c128(eps_h).ravel()
    bm = np.ascontiguousarray(beams_nm, dtype=np.float64).reshape(-1, 2)
    beams = (eels_beam * len(bm))(*[eels_beam(float(x), float(y)) for x, y in bm])
    jid = C.c_longlong()
    _check(_lib.eels_server_submit(srv, C.byref(g), C.byref(opts), len(e), e.ctypes.data_as(_dp), ep.shape[1],
                                   _cptr(ep), _cptr(eh), len(bm), beams, C.byref(jid)))
    return jid.value


def _info_dict(i: eels_job_info) -> dict:
    return dict(state=i.state, code=i.code, t_submit=i.t_submit, t_start=i.t_start, t_end=i.t_end,
                footprint=i.footprint, n_points=i.n_points)


def eels_server_poll(srv, job: int) -> dict:
    i = eels_job_info()
    _check(_lib.eels_server_poll(srv, job, C.byref(i)))
    return _info_dict(i)


def eels_server_wait(srv, job: int, n_energy: int, n_beam: int, want_cl: bool = True):
    out = {k: np.zeros((n_energy, n_beam)) for k in ("eels", "cl", "ext", "abs")}
    st = (eels_point_stats * (n_energy * n_beam))()
    i = eels_job_info()
    code = _lib.eels_server_wait(srv, job, _dptr(out["eels"]), _dptr(out["cl"]) if want_cl else None,
                                 _dptr(out["ext"]), _dptr(out["abs"]), st, C.byref(i))
    return code, out, _info_dict(i)


def eels_server_stats(srv):
    a, b, c = C.c_int(), C.c_int(), C.c_size_t()
    _check(_lib.eels_server_stats(srv, C.byref(a), C.byref(b), C.byref(c)))
    return dict(running_max=a.value, completed=b.value, in_use=c.value)


def eels_server_destroy(srv) -> None:
    _lib.eels_server_destroy(srv)
