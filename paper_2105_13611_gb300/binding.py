"""ctypes binding of the C ABI in include/mpsa.h (argument marshalling only).

Host arrays are numpy arrays; device buffers are torch CUDA tensors whose data
pointers are passed through.  Every call runs in the CUDA library; a missing
library raises instead of falling back to any CPU code.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("MPSA_LIBRARY") or os.path.join(HERE, "_lib", "libmpsa.so")

MPSA_OK, MPSA_EINVAL, MPSA_ENOMEM, MPSA_ECUDA, MPSA_ESTATE, MPSA_ETIMEOUT = 0, -1, -2, -3, -4, -5
PREC_FP32_COMPENSATED, PREC_FP32_NAIVE, PREC_FP64, PREC_FP32_POP32 = 0, 1, 2, 3
MEAN_ARITH, MEAN_GEOM = 0, 1

EXPORTED = ["mpsa_create", "mpsa_destroy", "mpsa_last_error", "mpsa_version", "mpsa_grid_size",
            "load_linelist", "set_atmosphere_grid", "synth_opacity", "build_odf", "synth_spectrum",
            "mpsa_profile_enable", "mpsa_profile_read", "build_odf_noalloc",
            "mpsa_server_create", "mpsa_server_submit", "mpsa_server_wait", "mpsa_server_get_stats",
            "mpsa_server_destroy", "mpsa_server_cancel_queued",
            "mpsa_batch_create", "mpsa_batch_run", "mpsa_batch_get_info", "mpsa_batch_destroy", "mpsa_voigt",
            "odf_intensity", "set_atmosphere_grid_eos", "mpsa_get_populations", "synth_continuum"]
REQ_SPECTRUM, REQ_ODF = 1, 2
KERNEL_PROFILE, KERNEL_ODF, KERNEL_BINS, KERNEL_CONTINUUM = 0, 1, 2, 3
CONT_ELEC, CONT_HBF, CONT_HFF, CONT_HRAY, CONT_ALL = 1, 2, 4, 8, 15

_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)
_ip = C.POINTER(C.c_int32)


class Elements(C.Structure):
    _fields_ = [("n_elements", C.c_int32), ("mass_amu", _dp), ("chi_eV", _dp), ("U1", _dp), ("U2", _dp),
                ("log_eps", _dp)]


class Eos(C.Structure):
    _fields_ = [("n_elements", C.c_int32), ("mass_amu", _dp), ("log_eps", _dp), ("n_stages", _ip), ("chi_eV", _dp),
                ("lnU", _dp)]


class Lines(C.Structure):
    _fields_ = [("n_lines", C.c_int64), ("lambda_nm", _dp), ("log_gf", _fp), ("E_eV", _fp), ("species", _ip),
                ("log_gR", _fp), ("log_gS", _fp), ("log_gW", _fp)]


class LGrid(C.Structure):
    _fields_ = [("lambda0_nm", C.c_double), ("lambda1_nm", C.c_double), ("R", C.c_double)]


class SynthOpts(C.Structure):
    _fields_ = [("cut", C.c_double), ("kc_factor", C.c_double), ("precision", C.c_int32), ("tile", C.c_int32),
                ("continuum", C.c_int32), ("reserved", C.c_int32)]


class Atmos(C.Structure):
    _fields_ = [("n_depth", C.c_int32), ("m", _dp), ("T", _dp), ("P", _dp), ("comp", C.c_int32)]


class Request(C.Structure):
    _fields_ = [("kind", C.c_int32), ("atm", Atmos), ("win", LGrid), ("n_mu", C.c_int32), ("mu", _dp),
                ("I_out", _fp), ("n_sel", C.c_int32), ("sel", _ip), ("grid", LGrid), ("K", C.c_int32),
                ("bounds", C.POINTER(C.c_int64)), ("n_steps", C.c_int32), ("widths", _dp), ("odf_out", _dp),
                ("kappa_c_out", _fp), ("mean_kind", C.c_int32)]


class BatchGroup(C.Structure):
    _fields_ = [("grid", LGrid), ("n_sel", C.c_int32), ("sel", _ip), ("kappa_out", C.c_void_p),
                ("kappa_c_out", C.c_void_p), ("evals_out", C.c_void_p), ("K", C.c_int32),
                ("bounds", C.POINTER(C.c_int64)), ("n_steps", C.c_int32), ("widths", _dp), ("odf_out", C.c_void_p),
                ("mean_kind", C.c_int32)]


class OdfTable(C.Structure):
    _fields_ = [("nT", C.c_int32), ("nP", C.c_int32), ("log10_T", _dp), ("log10_P", _dp), ("K", C.c_int32),
                ("n_steps", C.c_int32), ("odf", C.c_void_p), ("kappa_c", C.c_void_p), ("lam_c_nm", _dp),
                ("widths", _dp)]


class BatchInfo(C.Structure):
    _fields_ = [("pts_per_thread", C.c_int32), ("threads", C.c_int32), ("min_blocks", C.c_int32),
                ("n_rows", C.c_int32), ("n_units", C.c_int64), ("n_tuned", C.c_int32),
                ("tune_ms_per_mpoint", C.c_double * 8)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64), ("running", C.c_int64),
                ("queued", C.c_int64), ("bytes_in_use", C.c_size_t), ("bytes_peak", C.c_size_t)]


class MpsaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"mpsa error {code}: {msg}")
        self.code = code


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libmpsa.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing: run paper_2105_13611_gb300/build.py (no CPU fallback)")
    lib = C.CDLL(path)
    vp = C.c_void_p
    lib.mpsa_create.argtypes = [C.POINTER(vp), C.c_int]
    lib.mpsa_destroy.argtypes = [vp]
    lib.mpsa_destroy.restype = None
    lib.mpsa_last_error.restype = C.c_char_p
    lib.mpsa_version.restype = C.c_char_p
    lib.set_atmosphere_grid_eos.argtypes = [vp, C.POINTER(Eos), C.c_int32, _dp, _dp, C.c_int32, _dp, C.c_double]
    lib.set_atmosphere_grid_eos.restype = C.c_int
    lib.mpsa_get_populations.argtypes = [vp, C.c_int32, C.c_int32, _dp, _ip]
    lib.mpsa_get_populations.restype = C.c_int
    lib.synth_continuum.argtypes = [vp, C.POINTER(LGrid), C.c_int32, _ip, C.c_int32, vp, vp]
    lib.synth_continuum.restype = C.c_int
    lib.mpsa_grid_size.argtypes = [C.POINTER(LGrid)]
    lib.mpsa_grid_size.restype = C.c_int64
    lib.load_linelist.argtypes = [vp, C.c_int32, _ip, _ip, C.POINTER(Lines)]
    lib.set_atmosphere_grid.argtypes = [vp, C.POINTER(Elements), C.c_int32, _dp, _dp, C.c_int32, _dp, C.c_double]
    lib.synth_opacity.argtypes = [vp, C.POINTER(LGrid), C.c_int32, _ip, vp, vp, vp, C.POINTER(SynthOpts), vp]
    lib.build_odf.argtypes = [vp, vp, C.c_int32, C.c_int64, C.c_int32, C.POINTER(C.c_int64), C.c_int32, _dp,
                              C.c_int32, vp, vp]
    lib.synth_spectrum.argtypes = [vp, C.POINTER(Atmos), C.POINTER(LGrid), C.c_int32, _dp, vp,
                                   C.POINTER(SynthOpts), vp]
    lib.odf_intensity.argtypes = [vp, C.POINTER(OdfTable), C.c_int32, C.c_int32, vp, vp, vp, C.c_int32, _dp, vp, vp,
                                  vp]
    lib.odf_intensity.restype = C.c_int
    lib.build_odf_noalloc.argtypes = [C.c_int32, vp, C.c_int32, C.c_int64, C.c_int32, C.POINTER(C.c_int64), C.c_int32,
                                      _dp, C.c_int32, vp, vp]
    lib.build_odf_noalloc.restype = C.c_int
    lib.mpsa_server_create.argtypes = [C.POINTER(vp), vp, C.c_size_t, C.c_int32, C.c_int32]
    lib.mpsa_server_submit.argtypes = [vp, C.POINTER(Request), C.POINTER(C.c_int64)]
    lib.mpsa_server_wait.argtypes = [vp, C.c_int64, C.c_int32, C.POINTER(C.c_double)]
    lib.mpsa_server_get_stats.argtypes = [vp, C.POINTER(ServerStats)]
    lib.mpsa_server_cancel_queued.argtypes = [vp, C.POINTER(C.c_int64)]
    lib.mpsa_server_cancel_queued.restype = C.c_int
    lib.mpsa_server_destroy.argtypes = [vp]
    lib.mpsa_server_destroy.restype = None
    for f in ("mpsa_server_create", "mpsa_server_submit", "mpsa_server_wait", "mpsa_server_get_stats"):
        getattr(lib, f).restype = C.c_int
    lib.mpsa_batch_create.argtypes = [vp, C.c_int32, C.POINTER(BatchGroup), C.POINTER(SynthOpts), C.c_int32, vp,
                                      C.POINTER(vp)]
    lib.mpsa_batch_run.argtypes = [vp, vp]
    lib.mpsa_batch_get_info.argtypes = [vp, C.POINTER(BatchInfo)]
    lib.mpsa_batch_destroy.argtypes = [vp]
    lib.mpsa_batch_destroy.restype = None
    for f in ("mpsa_batch_create", "mpsa_batch_run", "mpsa_batch_get_info"):
        getattr(lib, f).restype = C.c_int
    lib.mpsa_voigt.argtypes = [vp, vp, vp, C.c_int64, C.c_int32, vp, vp]
    lib.mpsa_voigt.restype = C.c_int
    lib.mpsa_profile_enable.argtypes = [vp, C.c_int]
    lib.mpsa_profile_read.argtypes = [vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int64)]
    for f in ("mpsa_create", "load_linelist", "set_atmosphere_grid", "synth_opacity", "build_odf", "synth_spectrum",
              "mpsa_profile_enable", "mpsa_profile_read"):
        getattr(lib, f).restype = C.c_int
    _lib = lib
    return lib


def _check(rc):
    if rc != MPSA_OK:
        raise MpsaError(rc, _lib.mpsa_last_error().decode())


def _arr(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def _dev(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("device buffers must be contiguous CUDA tensors")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def grid_size(lam0_nm, lam1_nm, R) -> int:
    lib = load_library()
    return int(lib.mpsa_grid_size(C.byref(LGrid(lam0_nm, lam1_nm, R))))


def make_opts(cut=1e-3, kc_factor=1e-2, precision=PREC_FP32_COMPENSATED, continuum=0):
    return SynthOpts(cut, kc_factor, precision, 0, continuum, 0)


def _odf_args(kappa, bounds, widths, odf_out, device):
    """Host arrays of an ODF call after checking the device buffers against them: kappa a
    float32 [n_rows][N] and odf_out a float64 [n_rows][K][n_steps] CUDA tensor, both on
    `device` (a mismatch would let the kernel read or write outside the buffers)."""
    import torch
    b = _arr(bounds, np.int64)
    w = _arr(widths, np.float64)
    if kappa.dtype != torch.float32 or kappa.dim() != 2:
        raise ValueError(f"kappa must be a float32 [n_rows][N] tensor, got {kappa.dtype} {tuple(kappa.shape)}")
    if odf_out.dtype != torch.float64:
        raise ValueError(f"odf_out must be float64, got {odf_out.dtype}")
    n_rows, N = kappa.shape
    if tuple(odf_out.shape) != (n_rows, len(b) - 1, len(w)):
        raise ValueError(f"odf_out has shape {tuple(odf_out.shape)}, expected {(n_rows, len(b) - 1, len(w))}")
    for name, t in (("kappa", kappa), ("odf_out", odf_out)):
        if not t.is_cuda or t.device.index != int(device):
            raise ValueError(f"{name} is on {t.device}, expected cuda:{int(device)}")
    return b, w, n_rows, N


def build_odf_noalloc(device, kappa, bounds, widths, odf_out, mean_kind=MEAN_ARITH, stream=None):
    """build_odf without device allocation (fixed library-owned staging array; see include/mpsa.h)."""
    lib = load_library()
    b, w, n_rows, N = _odf_args(kappa, bounds, widths, odf_out, device)
    rc = lib.build_odf_noalloc(int(device), _dev(kappa), n_rows, N, len(b) - 1, _ptr(b, C.c_int64), len(w),
                               _ptr(w, C.c_double), mean_kind, _dev(odf_out), _stream(stream))
    _check(rc)


class Context:
    """One mpsa_ctx on one CUDA device: resident line list and population table."""

    def __init__(self, device: int = 0):
        self.lib = load_library()
        h = C.c_void_p()
        _check(self.lib.mpsa_create(C.byref(h), int(device)))
        self.h = h
        self.device = device
        self._keep = []

    def close(self):
        if self.h:
            self.lib.mpsa_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def profile_enable(self, on=True):
        _check(self.lib.mpsa_profile_enable(self.h, 1 if on else 0))

    def profile_read(self, kernel):
        """(total device ms, launches) of KERNEL_PROFILE, KERNEL_ODF or KERNEL_BINS since the last read."""
        ms = C.c_double()
        n = C.c_int64()
        _check(self.lib.mpsa_profile_read(self.h, kernel, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def load_linelist(self, lines, species_element, species_stage):
        """lines: workloads.LineList (or any object with the same fields)."""
        se = _arr(species_element, np.int32)
        ss = _arr(species_stage, np.int32)
        f = dict(lam=_arr(lines.lam_nm, np.float64), gf=_arr(lines.log_gf, np.float32), E=_arr(lines.E_eV, np.float32),
                 sp=_arr(lines.species, np.int32), R=_arr(lines.log_gR, np.float32), S=_arr(lines.log_gS, np.float32),
                 W=_arr(lines.log_gW, np.float32))
        L = Lines(len(f["lam"]), _ptr(f["lam"], C.c_double), _ptr(f["gf"], C.c_float), _ptr(f["E"], C.c_float),
                  _ptr(f["sp"], C.c_int32), _ptr(f["R"], C.c_float), _ptr(f["S"], C.c_float), _ptr(f["W"], C.c_float))
        _check(self.lib.load_linelist(self.h, len(se), _ptr(se, C.c_int32), _ptr(ss, C.c_int32), C.byref(L)))

    def set_atmosphere_grid(self, el, T, P, abund_scale=None, vturb=0.0):
        """el: workloads.Elements; T, P: arrays of the atmosphere points; abund_scale [n_comp][n_el] or None."""
        arrs = [_arr(el.mass_amu, np.float64), _arr(el.chi_eV, np.float64), _arr(el.U1, np.float64),
                _arr(el.U2, np.float64), _arr(el.log_eps, np.float64)]
        E = Elements(len(arrs[0]), *[_ptr(a, C.c_double) for a in arrs])
        T = _arr(T, np.float64)
        P = _arr(P, np.float64)
        if abund_scale is None:
            n_comp, ab = 1, None
        else:
            ab = _arr(abund_scale, np.float64)
            n_comp = ab.shape[0]
        _check(self.lib.set_atmosphere_grid(self.h, C.byref(E), len(T), _ptr(T, C.c_double), _ptr(P, C.c_double),
                                            n_comp, _ptr(ab, C.c_double) if ab is not None else None, float(vturb)))
        self.n_points = len(T)

    def set_atmosphere_grid_eos(self, eos, T, P, abund_scale=None, vturb=0.0):
        """eos: workloads.EosTable (multi-stage table); T, P, abund_scale as for set_atmosphere_grid."""
        n = eos.n
        arrs = [_arr(eos.mass_amu, np.float64), _arr(eos.log_eps, np.float64)]
        ns = _arr(eos.n_stages, np.int32)
        chi = _arr(np.asarray(eos.chi_eV).reshape(n, 4), np.float64)
        lnU = _arr(np.asarray(eos.lnU).reshape(n, 5, 3), np.float64)
        E = Eos(n, _ptr(arrs[0], C.c_double), _ptr(arrs[1], C.c_double), _ptr(ns, C.c_int32), _ptr(chi, C.c_double),
                _ptr(lnU, C.c_double))
        T = _arr(T, np.float64)
        P = _arr(P, np.float64)
        if abund_scale is None:
            n_comp, ab = 1, None
        else:
            ab = _arr(abund_scale, np.float64)
            n_comp = ab.shape[0]
        _check(self.lib.set_atmosphere_grid_eos(self.h, C.byref(E), len(T), _ptr(T, C.c_double), _ptr(P, C.c_double),
                                                n_comp, _ptr(ab, C.c_double) if ab is not None else None, float(vturb)))
        self.n_points = len(T)

    def get_populations(self, row0, n_rows):
        """Rows of the FP64 population table as a numpy array [n_rows][5 + 5 n_elements]: T, P, n_e,
        n_HI, rho, then N/U of stages I..V of every element."""
        st = C.c_int32()
        _check(self.lib.mpsa_get_populations(self.h, int(row0), 0, None, C.byref(st)))
        out = np.empty((int(n_rows), st.value), dtype=np.float64)
        _check(self.lib.mpsa_get_populations(self.h, int(row0), int(n_rows), _ptr(out, C.c_double), C.byref(st)))
        return out

    def synth_opacity(self, grid, sel, kappa_out, kappa_c_out=None, evals_out=None, opts=None, stream=None):
        s = _arr(sel, np.int32)
        g = LGrid(grid.lam0_nm, grid.lam1_nm, grid.R)
        o = opts if opts is not None else make_opts()
        _check(self.lib.synth_opacity(self.h, C.byref(g), len(s), _ptr(s, C.c_int32), _dev(kappa_out),
                                      _dev(kappa_c_out), _dev(evals_out), C.byref(o), _stream(stream)))

    def build_odf(self, kappa, bounds, widths, odf_out, mean_kind=MEAN_ARITH, stream=None):
        b, w, n_rows, N = _odf_args(kappa, bounds, widths, odf_out, self.device)
        _check(self.lib.build_odf(self.h, _dev(kappa), n_rows, N, len(b) - 1, _ptr(b, C.c_int64), len(w),
                                  _ptr(w, C.c_double), mean_kind, _dev(odf_out), _stream(stream)))

    def synth_continuum(self, grid, sel, kappa_out, sources=CONT_ALL, stream=None):
        """Closed-form continuum (synth_continuum in include/mpsa.h) of rows sel on grid into the
        float32 CUDA tensor kappa_out [len(sel)][N]."""
        s_ = _arr(sel, np.int32)
        g = LGrid(grid.lam0_nm, grid.lam1_nm, grid.R)
        _check(self.lib.synth_continuum(self.h, C.byref(g), len(s_), _ptr(s_, C.c_int32), int(sources),
                                        _dev(kappa_out), _stream(stream)))

    def voigt(self, v, a, out, precision=0, stream=None):
        """H(v, a) on the device as the kernels evaluate it; v, a, out: device float64 tensors."""
        _check(self.lib.mpsa_voigt(self.h, _dev(v), _dev(a), int(v.numel()), int(precision), _dev(out),
                                   _stream(stream)))

    def synth_spectrum(self, m, T, P, win, mus, I_out, comp=0, opts=None, stream=None):
        m = _arr(m, np.float64)
        T = _arr(T, np.float64)
        P = _arr(P, np.float64)
        mu = _arr(mus, np.float64)
        a = Atmos(len(m), _ptr(m, C.c_double), _ptr(T, C.c_double), _ptr(P, C.c_double), int(comp))
        g = LGrid(win.lam0_nm, win.lam1_nm, win.R)
        o = opts if opts is not None else make_opts()
        _check(self.lib.synth_spectrum(self.h, C.byref(a), C.byref(g), len(mu), _ptr(mu, C.c_double), _dev(I_out),
                                       C.byref(o), _stream(stream)))


    def odf_intensity(self, log10_T, log10_P, odf, kappa_c, lam_c_nm, widths, m, T, P, mus, I_out,
                      ray_status=None, stream=None):
        """Bin intensities of many rays from an ODF table (odf_intensity in include/mpsa.h).

        log10_T [nT], log10_P [nP], lam_c_nm [K], widths [n_steps], mus: host arrays;
        odf (float64 [nT*nP][K][n_steps]), kappa_c (float32 [nT*nP]), m, T, P (float64
        [n_rays][n_depth]), I_out (float32 [n_rays][n_mu][K]) and ray_status (int32 [n_rays]
        or None): CUDA tensors."""
        lt = _arr(log10_T, np.float64)
        lp = _arr(log10_P, np.float64)
        lam = _arr(lam_c_nm, np.float64)
        w = _arr(widths, np.float64)
        mu = _arr(mus, np.float64)
        K, ns = int(odf.shape[-2]), int(odf.shape[-1])
        tab = OdfTable(len(lt), len(lp), _ptr(lt, C.c_double), _ptr(lp, C.c_double), K, ns, _dev(odf),
                       _dev(kappa_c), _ptr(lam, C.c_double), _ptr(w, C.c_double))
        n_rays, n_depth = int(m.shape[0]), int(m.shape[1])
        _check(self.lib.odf_intensity(self.h, C.byref(tab), n_rays, n_depth, _dev(m), _dev(T), _dev(P), len(mu),
                                      _ptr(mu, C.c_double), _dev(I_out), _dev(ray_status), _stream(stream)))


class Server:
    """Continuous-batching request server on a Context (see mpsa_server_* in include/mpsa.h).

    submit_spectrum / submit_odf copy their inputs and return a ticket; wait(ticket) returns
    the result (numpy array(s)) and the latency in ms.  The context must not be used
    directly while the server exists.
    """

    def __init__(self, ctx: Context, hbm_budget_bytes: int, max_inflight: int = 4, rows_per_chunk: int = 8):
        self.lib = ctx.lib
        self.ctx = ctx
        h = C.c_void_p()
        _check(self.lib.mpsa_server_create(C.byref(h), ctx.h, int(hbm_budget_bytes), int(max_inflight),
                                           int(rows_per_chunk)))
        self.h = h
        self._pending = {}

    def submit_spectrum(self, m, T, P, win, mus, comp=0):
        m = _arr(m, np.float64); T = _arr(T, np.float64); P = _arr(P, np.float64); mu = _arr(mus, np.float64)
        N = grid_size(win.lam0_nm, win.lam1_nm, win.R)
        out = np.empty((len(mu), N), dtype=np.float32)
        q = Request()
        q.kind = REQ_SPECTRUM
        q.atm = Atmos(len(m), _ptr(m, C.c_double), _ptr(T, C.c_double), _ptr(P, C.c_double), int(comp))
        q.win = LGrid(win.lam0_nm, win.lam1_nm, win.R)
        q.n_mu = len(mu)
        q.mu = _ptr(mu, C.c_double)
        q.I_out = _ptr(out, C.c_float)
        t = C.c_int64()
        _check(self.lib.mpsa_server_submit(self.h, C.byref(q), C.byref(t)))
        self._pending[t.value] = (out,)
        return t.value

    def submit_odf(self, sel, grid, bounds, widths, mean_kind=MEAN_ARITH):
        s = _arr(sel, np.int32); b = _arr(bounds, np.int64); w = _arr(widths, np.float64)
        out = np.empty((len(s), len(b) - 1, len(w)), dtype=np.float64)
        kc = np.empty(len(s), dtype=np.float32)
        q = Request()
        q.kind = REQ_ODF
        q.n_sel = len(s)
        q.sel = _ptr(s, C.c_int32)
        q.grid = LGrid(grid.lam0_nm, grid.lam1_nm, grid.R)
        q.K = len(b) - 1
        q.bounds = _ptr(b, C.c_int64)
        q.n_steps = len(w)
        q.widths = _ptr(w, C.c_double)
        q.odf_out = _ptr(out, C.c_double)
        q.kappa_c_out = _ptr(kc, C.c_float)
        q.mean_kind = mean_kind
        t = C.c_int64()
        _check(self.lib.mpsa_server_submit(self.h, C.byref(q), C.byref(t)))
        self._pending[t.value] = (out, kc)
        return t.value

    def wait(self, ticket, timeout_ms=600_000):
        lat = C.c_double()
        _check(self.lib.mpsa_server_wait(self.h, int(ticket), int(timeout_ms), C.byref(lat)))
        res = self._pending.pop(ticket)
        return (res[0] if len(res) == 1 else res), lat.value

    def cancel_queued(self):
        n = C.c_int64()
        _check(self.lib.mpsa_server_cancel_queued(self.h, C.byref(n)))
        return n.value

    def stats(self):
        st = ServerStats()
        _check(self.lib.mpsa_server_get_stats(self.h, C.byref(st)))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self):
        if self.h:
            self.lib.mpsa_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Persistent, graph-captured batch of row groups (see mpsa_batch_* in include/mpsa.h).

    groups: list of dicts with keys grid, sel, kappa (CUDA tensor [n_sel][N]) and optionally
    kappa_c, evals (CUDA tensors), bounds, widths, odf (CUDA tensor [n_sel][K][n_steps])."""

    def __init__(self, ctx: Context, groups, opts=None, autotune=True, stream=None):
        self.lib = ctx.lib
        self._keep = []
        arr = (BatchGroup * len(groups))()
        for i, g in enumerate(groups):
            sel = _arr(g["sel"], np.int32)
            self._keep.append(sel)
            q = arr[i]
            q.grid = LGrid(g["grid"].lam0_nm, g["grid"].lam1_nm, g["grid"].R)
            q.n_sel = len(sel)
            q.sel = _ptr(sel, C.c_int32)
            q.kappa_out = _dev(g["kappa"])
            q.kappa_c_out = _dev(g.get("kappa_c"))
            q.evals_out = _dev(g.get("evals"))
            if g.get("odf") is not None:
                b = _arr(g["bounds"], np.int64)
                w = _arr(g["widths"], np.float64)
                self._keep += [b, w]
                q.K = len(b) - 1
                q.bounds = _ptr(b, C.c_int64)
                q.n_steps = len(w)
                q.widths = _ptr(w, C.c_double)
                q.odf_out = _dev(g["odf"])
                q.mean_kind = g.get("mean_kind", MEAN_ARITH)
            else:
                q.K = 0
        o = opts if opts is not None else make_opts()
        h = C.c_void_p()
        _check(self.lib.mpsa_batch_create(ctx.h, len(groups), arr, C.byref(o), 1 if autotune else 0, _stream(stream),
                                          C.byref(h)))
        self.h = h

    def run(self, stream=None):
        _check(self.lib.mpsa_batch_run(self.h, _stream(stream)))

    def info(self):
        i = BatchInfo()
        _check(self.lib.mpsa_batch_get_info(self.h, C.byref(i)))
        return {"pts_per_thread": i.pts_per_thread, "threads": i.threads, "min_blocks": i.min_blocks,
                "n_rows": i.n_rows, "n_units": i.n_units,
                "tune_ms_per_mpoint": [i.tune_ms_per_mpoint[k] for k in range(i.n_tuned)]}

    def close(self):
        if self.h:
            self.lib.mpsa_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
