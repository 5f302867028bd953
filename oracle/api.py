"""numpy wrappers around the FP64 oracle's ``extern "C"`` entry points.

Test infrastructure: see the package docstring. Grids are [chan][tranche][bin];
templates are SoA ``theta[8, n_tpl]`` in the order (M_c [M_sun], eta, f_0 [Hz],
phi_0, lambda, beta, psi, iota).
"""
import ctypes

import numpy as np

from .build import load_library

_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_U8 = ctypes.POINTER(ctypes.c_uint8)

PN_NEWTONIAN = 0
PN_1PN = 1
RESP_NONE = 0
RESP_LW = 1
RESP_TDI = 2
FRESNEL_PAPER = 0
FRESNEL_EXACT = 1


def _lib():
    lib = load_library()
    if not getattr(lib, "_typed", False):
        lib.oracle_statistic.restype = ctypes.c_int
        lib.oracle_statistic.argtypes = [
            ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
            _D, _D, _D, _U8, ctypes.c_int, ctypes.c_int, ctypes.c_int,
            _D, ctypes.c_int64, ctypes.c_int, _D, _I32, _I32, _I32, ctypes.c_int]
        lib.oracle_gradient.restype = ctypes.c_int
        lib.oracle_gradient.argtypes = [
            ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
            _D, _D, _D, _U8, ctypes.c_int, ctypes.c_int, ctypes.c_int,
            _D, ctypes.c_int64, ctypes.c_int, _D, _D, ctypes.c_int]
        lib.oracle_gradient_scale.restype = ctypes.c_int
        lib.oracle_gradient_scale.argtypes = lib.oracle_gradient.argtypes[:-3] + [
            _D, ctypes.c_int, ctypes.c_int]
        lib.oracle_segments.restype = ctypes.c_int
        lib.oracle_segments.argtypes = [
            ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
            _D, _D, _D, _U8, ctypes.c_int, ctypes.c_int, ctypes.c_int,
            _D, ctypes.c_int, _D, _D, _D, _D]
        lib.oracle_statistic_harm.restype = ctypes.c_int
        lib.oracle_statistic_harm.argtypes = [
            ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
            _D, _D, _D, _U8, ctypes.c_int, ctypes.c_int, ctypes.c_int,
            ctypes.c_int, _D, _D, _D,
            _D, ctypes.c_int64, ctypes.c_int, _D, _I32, _I32, _I32, ctypes.c_int]
        lib.oracle_segments_harm.restype = ctypes.c_int
        lib.oracle_segments_harm.argtypes = [
            ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
            _D, _D, _D, _U8, ctypes.c_int, ctypes.c_int, ctypes.c_int,
            ctypes.c_int, _D, _D, _D,
            _D, ctypes.c_int, _D, _D, _D, _D]
        lib.oracle_fresnel.restype = None
        lib.oracle_fresnel.argtypes = [ctypes.c_int, _D, ctypes.c_int64, _D, _D]
        lib.oracle_tranche_ft.restype = None
        lib.oracle_tranche_ft.argtypes = [
            ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
            ctypes.c_int64, ctypes.c_int64, ctypes.c_int, _D, _D]
        lib.oracle_source.restype = None
        lib.oracle_source.argtypes = [_D, ctypes.c_int, _D]
        lib.oracle_track.restype = None
        lib.oracle_track.argtypes = [_D, ctypes.c_int, ctypes.c_int, _D, ctypes.c_int64,
                                     ctypes.c_double, _D, _D, _D, _D, _D, _U8]
        lib.oracle_response.restype = None
        lib.oracle_response.argtypes = [_D, _D, ctypes.c_int64, ctypes.c_int, _D, _D]
        lib.oracle_response_tdi.restype = None
        lib.oracle_response_tdi.argtypes = [_D, _D, _D, ctypes.c_int64, ctypes.c_int, _D, _D]
        lib.oracle_spacecraft_offsets.restype = None
        lib.oracle_spacecraft_offsets.argtypes = [ctypes.c_double, _D]
        lib.oracle_detector_tensors.restype = None
        lib.oracle_detector_tensors.argtypes = [ctypes.c_double, _D, _D]
        lib.oracle_polarisation.restype = None
        lib.oracle_polarisation.argtypes = [_D, _D, _D]
        lib.oracle_max_threads.restype = ctypes.c_int
        lib.oracle_max_threads.argtypes = []
        lib._typed = True
    return lib


def _p(a, t=_D):
    return a.ctypes.data_as(t) if a is not None else None


def _grid(d, w, mask):
    d = np.asarray(d)
    if d.ndim == 2:
        d = d[None]
    w = np.asarray(w, dtype=np.float64)
    if w.ndim == 2:
        w = w[None]
    d_re = np.ascontiguousarray(d.real, dtype=np.float64)
    d_im = np.ascontiguousarray(d.imag, dtype=np.float64)
    w = np.ascontiguousarray(w)
    if w.shape != d_re.shape:
        raise ValueError("data and weights must have the same [chan][tranche][bin] shape")
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    if m is not None and m.shape != (d_re.shape[1],):
        raise ValueError("mask must have one entry per tranche")
    return d_re, d_im, w, m


def max_threads():
    return _lib().oracle_max_threads()


def statistic(d, w, mask, theta, n_seg, dT, t0=0.0, pn_order=PN_NEWTONIAN, response=RESP_NONE,
              fresnel_mode=FRESNEL_PAPER, n_threads=0):
    """Upsilon_{N_seg} (Eq. Upsilon-seg) per template.

    Returns (stat[n], n_eff[n], n_active[n], n_noncompact[n]).
    """
    d_re, d_im, w, m = _grid(d, w, mask)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    if th.ndim != 2 or th.shape[0] != 8:
        raise ValueError("theta must be SoA [8, n_tpl]")
    n = th.shape[1]
    out = np.zeros(n)
    neff = np.zeros(n, np.int32)
    nact = np.zeros(n, np.int32)
    nnc = np.zeros(n, np.int32)
    rc = _lib().oracle_statistic(
        d_re.shape[0], d_re.shape[1], d_re.shape[2], float(dT), float(t0),
        _p(d_re), _p(d_im), _p(w), _p(m, _U8), int(pn_order), int(response), int(fresnel_mode),
        _p(th), n, int(n_seg), _p(out), _p(neff, _I32), _p(nact, _I32), _p(nnc, _I32),
        int(n_threads))
    if rc != 0:
        raise ValueError(f"oracle_statistic failed with code {rc}")
    return out, neff, nact, nnc


def gradient(d, w, mask, theta, n_seg, dT, t0=0.0, pn_order=PN_NEWTONIAN, response=RESP_NONE,
             fresnel_mode=FRESNEL_PAPER, n_threads=0):
    """Upsilon_{N_seg} and d Upsilon/d theta (SoA [8, n]) by forward-mode dual numbers."""
    d_re, d_im, w, m = _grid(d, w, mask)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    n = th.shape[1]
    out = np.zeros(n)
    grad = np.zeros((8, n))
    rc = _lib().oracle_gradient(
        d_re.shape[0], d_re.shape[1], d_re.shape[2], float(dT), float(t0),
        _p(d_re), _p(d_im), _p(w), _p(m, _U8), int(pn_order), int(response), int(fresnel_mode),
        _p(th), n, int(n_seg), _p(out), _p(grad), int(n_threads))
    if rc != 0:
        raise ValueError(f"oracle_gradient failed with code {rc}")
    return out, grad


def gradient_scale(d, w, mask, theta, n_seg, dT, t0=0.0, pn_order=PN_NEWTONIAN,
                   response=RESP_NONE, fresnel_mode=FRESNEL_PAPER, tranche_level=False,
                   n_threads=0):
    """Term scale [8, n] of each gradient component, whose signed sum of terms is
    dUpsilon/dtheta_p (Eq. Upsilon-seg differentiated): the sum over segments of the
    absolute values of 8 Re(conj(Z_n) dZ_n)/N_n and 4 |Z_n|^2 dN_n/N_n^2, or with
    tranche_level=True the sum over every (segment, tranche) of
    |8 Re(conj(Z_n) dz_m)/N_n - 4 |Z_n|^2 dn_m/N_n^2| with z_m, n_m the tranche's shares.
    An evaluation that forms those terms with unit roundoff u resolves a component only
    to about u times its scale."""
    d_re, d_im, w, m = _grid(d, w, mask)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    n = th.shape[1]
    out = np.zeros((8, n))
    rc = _lib().oracle_gradient_scale(
        d_re.shape[0], d_re.shape[1], d_re.shape[2], float(dT), float(t0),
        _p(d_re), _p(d_im), _p(w), _p(m, _U8), int(pn_order), int(response), int(fresnel_mode),
        _p(th), n, int(n_seg), _p(out), int(bool(tranche_level)), int(n_threads))
    if rc != 0:
        raise ValueError(f"oracle_gradient_scale failed with code {rc}")
    return out


def segments(d, w, mask, theta8, n_seg, dT, t0=0.0, pn_order=PN_NEWTONIAN,
             response=RESP_NONE, fresnel_mode=FRESNEL_PAPER):
    """Per-segment Z_n (complex) and N_n of one template, and Upsilon."""
    d_re, d_im, w, m = _grid(d, w, mask)
    th = np.ascontiguousarray(theta8, dtype=np.float64).ravel()
    zr = np.zeros(n_seg)
    zi = np.zeros(n_seg)
    nn = np.zeros(n_seg)
    ups = np.zeros(1)
    rc = _lib().oracle_segments(
        d_re.shape[0], d_re.shape[1], d_re.shape[2], float(dT), float(t0),
        _p(d_re), _p(d_im), _p(w), _p(m, _U8), int(pn_order), int(response), int(fresnel_mode),
        _p(th), int(n_seg), _p(zr), _p(zi), _p(nn), _p(ups))
    if rc != 0:
        raise ValueError(f"oracle_segments failed with code {rc}")
    return zr + 1j * zi, nn, float(ups[0])


def _harmonics(nu, c):
    nu = np.ascontiguousarray(np.atleast_1d(nu), dtype=np.float64)
    c = np.atleast_1d(np.asarray(c, dtype=np.complex128))
    if nu.ndim != 1 or c.shape != nu.shape or nu.size < 1:
        raise ValueError("nu and c must be 1-D of the same length >= 1")
    return nu, np.ascontiguousarray(c.real), np.ascontiguousarray(c.imag)


def statistic_harm(d, w, mask, theta, n_seg, dT, nu, c, t0=0.0, pn_order=PN_NEWTONIAN,
                   response=RESP_NONE, fresnel_mode=FRESNEL_PAPER, n_threads=0):
    """Upsilon_{N_seg} of multi-harmonic templates: harmonic h has phase nu[h] Phi,
    frequency nu[h] f, derivative nu[h] fdot and amplitude c[h] A.

    Returns (stat[n], n_eff[n], n_active[n], n_noncompact[n]).
    """
    d_re, d_im, w, m = _grid(d, w, mask)
    nu, cr, ci = _harmonics(nu, c)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    if th.ndim != 2 or th.shape[0] != 8:
        raise ValueError("theta must be SoA [8, n_tpl]")
    n = th.shape[1]
    out = np.zeros(n)
    neff = np.zeros(n, np.int32)
    nact = np.zeros(n, np.int32)
    nnc = np.zeros(n, np.int32)
    rc = _lib().oracle_statistic_harm(
        d_re.shape[0], d_re.shape[1], d_re.shape[2], float(dT), float(t0),
        _p(d_re), _p(d_im), _p(w), _p(m, _U8), int(pn_order), int(response), int(fresnel_mode),
        nu.size, _p(nu), _p(cr), _p(ci),
        _p(th), n, int(n_seg), _p(out), _p(neff, _I32), _p(nact, _I32), _p(nnc, _I32),
        int(n_threads))
    if rc != 0:
        raise ValueError(f"oracle_statistic_harm failed with code {rc}")
    return out, neff, nact, nnc


def segments_harm(d, w, mask, theta8, n_seg, dT, nu, c, t0=0.0, pn_order=PN_NEWTONIAN,
                  response=RESP_NONE, fresnel_mode=FRESNEL_PAPER):
    """Per-segment Z_n (complex) and N_n of one multi-harmonic template, and Upsilon."""
    d_re, d_im, w, m = _grid(d, w, mask)
    nu, cr, ci = _harmonics(nu, c)
    th = np.ascontiguousarray(theta8, dtype=np.float64).ravel()
    zr = np.zeros(n_seg)
    zi = np.zeros(n_seg)
    nn = np.zeros(n_seg)
    ups = np.zeros(1)
    rc = _lib().oracle_segments_harm(
        d_re.shape[0], d_re.shape[1], d_re.shape[2], float(dT), float(t0),
        _p(d_re), _p(d_im), _p(w), _p(m, _U8), int(pn_order), int(response), int(fresnel_mode),
        nu.size, _p(nu), _p(cr), _p(ci), _p(th), int(n_seg), _p(zr), _p(zi), _p(nn), _p(ups))
    if rc != 0:
        raise ValueError(f"oracle_segments_harm failed with code {rc}")
    return zr + 1j * zi, nn, float(ups[0])


def fresnel(z, mode=FRESNEL_PAPER):
    z = np.ascontiguousarray(z, dtype=np.float64).ravel()
    C = np.empty_like(z)
    S = np.empty_like(z)
    _lib().oracle_fresnel(int(mode), _p(z), z.size, _p(C), _p(S))
    return C, S


def tranche_ft(amp, phi, fm, fdot, dT, k0, nk, fresnel_mode=FRESNEL_PAPER):
    """h~(k delta f) for k = k0 .. k0+nk-1 (Eq. fresnel-ft), complex array."""
    re = np.empty(nk)
    im = np.empty(nk)
    _lib().oracle_tranche_ft(float(amp), float(phi), float(fm), float(fdot), float(dT),
                             int(k0), int(nk), int(fresnel_mode), _p(re), _p(im))
    return re + 1j * im


def source_constants(theta8, pn_order=PN_NEWTONIAN):
    """(t_c, F0, C2, P5, P3) of one template."""
    th = np.ascontiguousarray(theta8, dtype=np.float64)
    out = np.empty(5)
    _lib().oracle_source(_p(th), int(pn_order), _p(out))
    return out


def track(theta8, t, t_anchor=0.0, pn_order=PN_NEWTONIAN, response=RESP_NONE):
    """Track at detector times t: dict of f, fdot, amp, dphi (since t_anchor), tprime, alive."""
    th = np.ascontiguousarray(theta8, dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.float64).ravel()
    n = t.size
    out = {k: np.empty(n) for k in ("f", "fdot", "amp", "dphi", "tprime")}
    alive = np.empty(n, np.uint8)
    _lib().oracle_track(_p(th), int(pn_order), int(response), _p(t), n, float(t_anchor),
                        _p(out["f"]), _p(out["fdot"]), _p(out["amp"]), _p(out["dphi"]),
                        _p(out["tprime"]), _p(alive, _U8))
    out["alive"] = alive.astype(bool)
    return out


def response(theta8, t, n_chan=2):
    """T_alpha(t) = F+ A+ - i Fx Ax, complex [n_chan, n]."""
    th = np.ascontiguousarray(theta8, dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.float64).ravel()
    re = np.empty((n_chan, t.size))
    im = np.empty((n_chan, t.size))
    _lib().oracle_response(_p(th), _p(t), t.size, int(n_chan), _p(re), _p(im))
    return re + 1j * im


def response_tdi(theta8, t, f, n_chan=2):
    """TDI-1.5 transfer T_alpha(t, f) of the A/E channels, complex [n_chan, n]."""
    th = np.ascontiguousarray(theta8, dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.float64).ravel()
    f = np.ascontiguousarray(np.broadcast_to(f, t.shape), dtype=np.float64)
    re = np.empty((n_chan, t.size))
    im = np.empty((n_chan, t.size))
    _lib().oracle_response_tdi(_p(th), _p(t), _p(f), t.size, int(n_chan), _p(re), _p(im))
    return re + 1j * im


def spacecraft_offsets(t):
    """Spacecraft positions relative to the guiding centre [light-s], [3, 3]."""
    p = np.empty(9)
    _lib().oracle_spacecraft_offsets(float(t), _p(p))
    return p.reshape(3, 3)


def detector_tensors(t):
    DA = np.empty(9)
    DE = np.empty(9)
    _lib().oracle_detector_tensors(float(t), _p(DA), _p(DE))
    return DA.reshape(3, 3), DE.reshape(3, 3)


def polarisation(theta8):
    th = np.ascontiguousarray(theta8, dtype=np.float64)
    ep = np.empty(9)
    ex = np.empty(9)
    _lib().oracle_polarisation(_p(th), _p(ep), _p(ex))
    return ep.reshape(3, 3), ex.reshape(3, 3)
