"""Python binding of libtfs (include/tfs.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts numpy arrays and
torch tensors to pointers, allocates outputs, and raises on error codes. Arrays on
the context's GPU are passed as device pointers (the call is then asynchronous on the
current torch stream); host arrays are passed as host pointers (the call returns
after the results are copied back).

If the shared library is missing and cannot be built, importing the binding fails:
there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

from . import build as _build

PATH_FP64, PATH_PLAIN, PATH_MIXED = 0, 1, 2
PIX_F32, PIX_F16, PIX_BF16, PIX_F16_ALL, PIX_BF16_ALL = 0, 1, 2, 3, 4
_PIX_NAMES = {"f32": PIX_F32, "f16": PIX_F16, "bf16": PIX_BF16, "f16all": PIX_F16_ALL,
              "bf16all": PIX_BF16_ALL}
_PATH_NAMES = {"fp64": PATH_FP64, "plain": PATH_PLAIN, "mixed": PATH_MIXED}

_ERRORS = {
    -1: "TFS_ERR_ARG", -2: "TFS_ERR_STATE", -3: "TFS_ERR_NSEG", -4: "TFS_ERR_OOM",
    -5: "TFS_ERR_CUDA", -6: "TFS_ERR_TIMEOUT", -7: "TFS_ERR_DEVICE_CHECK",
}


class TFSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRORS.get(code, code)}: {msg}")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int), ("pixel", ctypes.c_int), ("pn_order", ctypes.c_int),
                ("response", ctypes.c_int), ("checked", ctypes.c_int), ("sort", ctypes.c_int),
                ("warps_per_cta", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("profile", ctypes.c_int), ("tile_variant", ctypes.c_int),
                ("max_device_bytes", ctypes.c_int64)]


class Swarm(ctypes.Structure):
    """tfs_swarm (include/tfs.h)."""
    _fields_ = [("n_swarm", ctypes.c_int), ("n_part", ctypes.c_int),
                ("lo", ctypes.c_void_p), ("hi", ctypes.c_void_p),
                ("inertia", ctypes.c_double), ("c1", ctypes.c_double), ("c2", ctypes.c_double),
                ("seed", ctypes.c_uint64),
                ("x", ctypes.c_void_p), ("v", ctypes.c_void_p), ("pbest", ctypes.c_void_p),
                ("pval", ctypes.c_void_p), ("gbest", ctypes.c_void_p), ("gval", ctypes.c_void_p)]


class Refine(ctypes.Structure):
    """tfs_refine (include/tfs.h)."""
    _fields_ = [("n", ctypes.c_int64),
                ("theta", ctypes.c_void_p), ("best_theta", ctypes.c_void_p),
                ("best_grad", ctypes.c_void_p), ("best_stat", ctypes.c_void_p),
                ("eta", ctypes.c_void_p), ("sigma", ctypes.c_void_p),
                ("lo", ctypes.c_double * 8), ("hi", ctypes.c_double * 8),
                ("eta_up", ctypes.c_double), ("eta_down", ctypes.c_double)]


_lib = None


def library_path():
    return _build.LIB


def load_library(build_if_missing=True):
    """Load libtfs.so (building it with nvcc if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        try:
            _build.build()
        except Exception as e:  # noqa: BLE001
            if not os.path.exists(_build.LIB):
                raise ImportError(f"libtfs.so is not built and could not be built: {e}") from e
    if not os.path.exists(_build.LIB):
        raise ImportError(f"libtfs.so not found at {_build.LIB}")
    lib = ctypes.CDLL(_build.LIB)
    P = ctypes.c_void_p
    i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
    sig = {
        "tfs_version": (i32, []),
        "tfs_default_options": (None, [ctypes.POINTER(Options)]),
        "tfs_create": (i32, [ctypes.POINTER(P), i32, ctypes.POINTER(Options)]),
        "tfs_destroy": (i32, [P]),
        "tfs_set_options": (i32, [P, ctypes.POINTER(Options)]),
        "tfs_get_options": (i32, [P, ctypes.POINTER(Options)]),
        "tfs_load_tf_data": (i32, [P, i32, i32, i32, dbl, dbl, dbl, P, P]),
        "tfs_set_noise_weights": (i32, [P, P, P]),
        "tfs_set_harmonics": (i32, [P, i32, P, P, P]),
        "tfs_noise_realisation": (i32, [P, ctypes.c_uint64]),
        "tfs_eval_statistic": (i32, [P, P, i64, P, i32, i32, P, P, P, P]),
        "tfs_grad_statistic": (i32, [P, P, i64, ctypes.c_int32, P, P, P]),
        "tfs_select_top": (i32, [P, P, i64, i64, P, P]),
        "tfs_ascent_step": (i32, [P, P, P, i64, P, P, P, P]),
        "tfs_pso_init": (i32, [P, ctypes.POINTER(Swarm), P]),
        "tfs_pso_step": (i32, [P, ctypes.POINTER(Swarm), P, i64, i32, P, P]),
        "tfs_refine_step": (i32, [P, ctypes.POINTER(Refine), P, P, P, P]),
        "tfs_last_profile": (i32, [P, ctypes.POINTER(ctypes.c_double)]),
        "tfs_last_launch_count": (i64, [P]),
        "tfs_last_launch_shape": (i32, [P, P]),
        "tfs_last_error": (ctypes.c_char_p, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    """Names of the tfs_* entry points the loaded library exports."""
    lib = load_library()
    return sorted(n for n in dir(lib) if n.startswith("tfs_"))


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """(pointer, keepalive) of a contiguous numpy array or torch tensor, or (None, None)."""
    if x is None:
        return None, None
    if _is_torch(x):
        x = x.contiguous()
        return ctypes.c_void_p(x.data_ptr()), x
    x = np.ascontiguousarray(x)
    return ctypes.c_void_p(x.ctypes.data), x


class TFS:
    """A libtfs context on one CUDA device.

    Options (keyword arguments): path ('mixed' | 'plain' | 'fp64'), pixel ('f16' | 'bf16'
    | 'f32' | 'f16all' | 'bf16all'), pn_order (0 | 1), response (0 | 1 | 2), sort,
    warps_per_cta, tile_variant, use_graph, profile, checked, max_device_bytes.
    """

    def __init__(self, device=0, **opts):
        self.lib = load_library()
        self.device = device
        o = Options()
        self.lib.tfs_default_options(ctypes.byref(o))
        self._apply(o, opts)
        h = ctypes.c_void_p()
        rc = self.lib.tfs_create(ctypes.byref(h), int(device), ctypes.byref(o))
        if rc != 0:
            raise TFSError(rc, "tfs_create failed (no CUDA device?)")
        self.h = h
        self.shape = None

    @staticmethod
    def _apply(o, opts):
        for k, v in opts.items():
            if k == "path" and isinstance(v, str):
                v = _PATH_NAMES[v]
            if k == "pixel" and isinstance(v, str):
                v = _PIX_NAMES[v]
            if not hasattr(o, k):
                raise TypeError(f"unknown option {k}")
            setattr(o, k, int(v))

    def close(self):
        if getattr(self, "h", None):
            self.lib.tfs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def _check(self, rc):
        if rc != 0:
            raise TFSError(rc, self.lib.tfs_last_error(self.h).decode())

    @property
    def options(self):
        o = Options()
        self._check(self.lib.tfs_get_options(self.h, ctypes.byref(o)))
        return {f: getattr(o, f) for f, _ in Options._fields_}

    def set_options(self, **opts):
        o = Options()
        self._check(self.lib.tfs_get_options(self.h, ctypes.byref(o)))
        self._apply(o, opts)
        self._check(self.lib.tfs_set_options(self.h, ctypes.byref(o)))

    def _stream(self, *arrays):
        for a in arrays:
            if a is not None and _is_torch(a) and a.is_cuda:
                import torch
                return ctypes.c_void_p(torch.cuda.current_stream(a.device).cuda_stream)
        return ctypes.c_void_p(0)

    # -- data ---------------------------------------------------------------------------
    def load_tf_data(self, d, dt, dT, t0=0.0):
        """d: complex [n_chan][n_tranche][n_bins] (numpy or torch, host or device)."""
        if _is_torch(d):
            re, im = d.real.double().contiguous(), d.imag.double().contiguous()
            shape = tuple(d.shape)
        else:
            d = np.asarray(d)
            re = np.ascontiguousarray(d.real, dtype=np.float64)
            im = np.ascontiguousarray(d.imag, dtype=np.float64)
            shape = d.shape
        if len(shape) == 2:
            shape = (1,) + tuple(shape)
        pr, kr = _ptr(re)
        pi, ki = _ptr(im)
        self._check(self.lib.tfs_load_tf_data(self.h, shape[0], shape[1], shape[2], float(dt),
                                              float(dT), float(t0), pr, pi))
        self.shape = shape

    def set_noise_weights(self, inv_psd, mask=None):
        """inv_psd: float64 [n_chan][n_tranche][n_bins] = 1/S; mask: uint8 [n_tranche] or None."""
        if _is_torch(inv_psd):
            inv_psd = inv_psd.double()
        else:
            inv_psd = np.ascontiguousarray(inv_psd, dtype=np.float64)
        if mask is not None:
            mask = mask.to(dtype=__import__("torch").uint8) if _is_torch(mask) else \
                np.ascontiguousarray(mask, dtype=np.uint8)
        pw, kw = _ptr(inv_psd)
        pm, km = _ptr(mask)
        self._check(self.lib.tfs_set_noise_weights(self.h, pw, pm))

    def noise_realisation(self, seed):
        """Replace the data by a noise-only realisation drawn from the current weights
        (tfs_noise_realisation)."""
        self._check(self.lib.tfs_noise_realisation(self.h, int(seed) & 0xFFFFFFFFFFFFFFFF))

    # -- statistic ----------------------------------------------------------------------
    def eval_statistic(self, theta, n_seg, per_template=False, diag=False, out=None):
        """Upsilon_{N_seg} for theta [8, n] (SoA).

        n_seg: int or list of up to 4 ints (all evaluated in one pass), or with
        per_template=True an int32 array [n]. Returns (stat, n_eff, diag_or_None) with
        stat [levels, n] (levels squeezed when n_seg is a scalar or per-template).
        Outputs live where theta lives (device tensors -> asynchronous call).
        """
        dev = _is_torch(theta) and theta.is_cuda
        if _is_torch(theta):
            theta = theta.double().contiguous()
        else:
            theta = np.ascontiguousarray(theta, dtype=np.float64)
        n = theta.shape[1]
        scalar = np.isscalar(n_seg) and not per_template
        if per_template:
            ns = n_seg.to(dtype=__import__("torch").int32).contiguous() if _is_torch(n_seg) else \
                np.ascontiguousarray(n_seg, dtype=np.int32)
            L = 1
        else:
            ns = np.atleast_1d(np.asarray(n_seg, dtype=np.int32))
            L = ns.size
        if dev:
            import torch
            stat = out if out is not None else torch.empty((L, n), dtype=torch.float64, device=theta.device)
            neff = torch.empty((L, n), dtype=torch.int32, device=theta.device)
            dg = torch.empty((2, n), dtype=torch.int32, device=theta.device) if diag else None
        else:
            stat = out if out is not None else np.empty((L, n))
            neff = np.empty((L, n), np.int32)
            dg = np.empty((2, n), np.int32) if diag else None
        pt, kt = _ptr(theta)
        pn, kn = _ptr(ns)
        ps, _ = _ptr(stat)
        pe, _ = _ptr(neff)
        pd, _ = _ptr(dg)
        self._check(self.lib.tfs_eval_statistic(self.h, pt, n, pn, int(L), int(bool(per_template)),
                                                ps, pe, pd, self._stream(theta)))
        if scalar or per_template:
            return stat[0], neff[0], dg
        return stat, neff, dg

    def set_harmonics(self, nu=(), c=()):
        """Harmonic content of the templates: harmonic h has phase nu[h] Phi, frequency
        nu[h] f, derivative nu[h] fdot and complex amplitude c[h] (relative to the
        dominant mode's A). Empty (the default) = the dominant mode alone."""
        nu = np.ascontiguousarray(np.atleast_1d(np.asarray(nu, dtype=np.float64)))
        c = np.atleast_1d(np.asarray(c, dtype=np.complex128))
        if nu.shape != c.shape or nu.ndim != 1:
            raise ValueError("nu and c must be 1-D of the same length")
        cr = np.ascontiguousarray(c.real)
        ci = np.ascontiguousarray(c.imag)
        if nu.size == 0:
            self._check(self.lib.tfs_set_harmonics(self.h, 0, None, None, None))
        else:
            self._check(self.lib.tfs_set_harmonics(
                self.h, int(nu.size), nu.ctypes.data_as(ctypes.c_void_p),
                cr.ctypes.data_as(ctypes.c_void_p), ci.ctypes.data_as(ctypes.c_void_p)))

    def grad_statistic(self, theta, n_seg, out=None):
        """(Upsilon [n], d Upsilon / d theta [8, n]) at one N_seg. out: optional
        (stat [n], grad [8, n]) float64 arrays to write into (contiguous; CUDA tensors
        for a device theta)."""
        dev = _is_torch(theta) and theta.is_cuda
        if _is_torch(theta):
            theta = theta.double().contiguous()
        else:
            theta = np.ascontiguousarray(theta, dtype=np.float64)
        n = theta.shape[1]
        if out is not None:
            stat, grad = out
            for a, shape in ((stat, (n,)), (grad, (8, n))):
                if tuple(a.shape) != shape or str(a.dtype).split(".")[-1] != "float64" or \
                        not (a.is_contiguous() if _is_torch(a) else a.flags.c_contiguous):
                    raise ValueError("out must be contiguous float64 arrays of shapes [n], [8, n]")
        elif dev:
            import torch
            stat = torch.empty(n, dtype=torch.float64, device=theta.device)
            grad = torch.empty((8, n), dtype=torch.float64, device=theta.device)
        else:
            stat = np.empty(n)
            grad = np.empty((8, n))
        pt, kt = _ptr(theta)
        ps, _ = _ptr(stat)
        pg, _ = _ptr(grad)
        self._check(self.lib.tfs_grad_statistic(self.h, pt, n, int(n_seg), ps, pg,
                                                self._stream(theta)))
        return stat, grad

    def select_top(self, stat, k):
        """Indices [k] of the k largest values, decreasing (ties: lower index first)."""
        dev = _is_torch(stat) and stat.is_cuda
        if _is_torch(stat):
            stat = stat.double().contiguous()
        else:
            stat = np.ascontiguousarray(stat, dtype=np.float64)
        n = stat.shape[0]
        if dev:
            import torch
            idx = torch.empty(k, dtype=torch.int64, device=stat.device)
        else:
            idx = np.empty(k, np.int64)
        ps, ks = _ptr(stat)
        pi, _ = _ptr(idx)
        self._check(self.lib.tfs_select_top(self.h, ps, n, int(k), pi, self._stream(stat)))
        return idx

    def ascent_step(self, theta, grad, step, lo, hi):
        """In-place projected ascent step theta += step * grad (see include/tfs.h)."""
        n = theta.shape[1]
        pt, kt = _ptr(theta)
        pg, kg = _ptr(grad)
        s = np.ascontiguousarray(step, dtype=np.float64)
        lo_ = np.ascontiguousarray(lo, dtype=np.float64)
        hi_ = np.ascontiguousarray(hi, dtype=np.float64)
        if not _is_torch(theta) and kt is not theta:
            raise ValueError("theta must be a contiguous float64 array (updated in place)")
        self._check(self.lib.tfs_ascent_step(self.h, pt, pg, n, _ptr(s)[0], _ptr(lo_)[0],
                                             _ptr(hi_)[0], self._stream(theta)))
        return theta

    # -- search steps (device state only) -------------------------------------------------
    def pso_init(self, sw, stream_of):
        """tfs_pso_init on a Swarm whose arrays live on this context's device."""
        self._check(self.lib.tfs_pso_init(self.h, ctypes.byref(sw), self._stream(stream_of)))

    def pso_step(self, sw, f, it, move, history=None):
        """tfs_pso_step with the objective f [S*P] (device tensor) at the positions."""
        ph, _ = _ptr(history)
        self._check(self.lib.tfs_pso_step(self.h, ctypes.byref(sw), _ptr(f)[0], int(it),
                                          int(bool(move)), ph, self._stream(f)))

    def refine_step(self, rf, stat, grad, mean_out=None):
        """tfs_refine_step from stat [n] and grad [8, n] (device tensors)."""
        pm, _ = _ptr(mean_out)
        self._check(self.lib.tfs_refine_step(self.h, ctypes.byref(rf), _ptr(stat)[0],
                                             _ptr(grad)[0], pm, self._stream(stat)))

    # -- accounting -----------------------------------------------------------------------
    def last_profile(self):
        ms = (ctypes.c_double * 4)()
        self._check(self.lib.tfs_last_profile(self.h, ms))
        return {"setup": ms[0], "sort": ms[1], "statistic": ms[2], "output": ms[3]}

    def last_launch_count(self):
        return int(self.lib.tfs_last_launch_count(self.h))

    def last_launch_shape(self):
        """Shape of the last statistic launch (see tfs_last_launch_shape)."""
        out = np.zeros(6, np.int32)
        self._check(self.lib.tfs_last_launch_shape(self.h, out.ctypes.data_as(ctypes.c_void_p)))
        keys = ("variant", "threads_per_cta", "ctas", "ctas_per_sm", "sms", "tune_trials")
        return dict(zip(keys, (int(x) for x in out)))
