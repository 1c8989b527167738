"""ctypes binding of libkpm.so (argument marshalling only).

Every function has the name of the C entry point it calls (include/kpm.h) and
passes raw pointers: torch CUDA tensors for device buffers, numpy arrays or
torch CPU tensors where the C ABI accepts host buffers.  All arithmetic runs
in the library's CUDA kernels; if the library is missing or fails to load,
`load()` raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libkpm.so")

KPM_OK = 0
KPM_EINVAL = -1
KPM_ENOMEM = -2
KPM_ECUDA = -3
KPM_ENONFINITE = -4
KPM_ETIMEDOUT = -5
KPM_ENOTCONV = -6
KPM_FP64 = 0
KPM_FP32 = 1
KPM_DF64 = 2
KPM_FLAG_DOUBLE_STEP = 1
KPM_FLAG_PH_HALF = 2
KPM_FLAG_KEEP_TAIL = 4
KPM_REGENERATE = -1


class kpm_model(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("flux", ctypes.c_int32),
                ("gutzwiller", ctypes.c_int32), ("t", ctypes.c_double), ("tp", ctypes.c_double),
                ("J", ctypes.c_double)]


class kpm_opts(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int32), ("precision", ctypes.c_int32), ("block_width", ctypes.c_int32),
                ("cols_per_block", ctypes.c_int32), ("margin", ctypes.c_double), ("temperature", ctypes.c_double),
                ("flags", ctypes.c_int32),
                ("probe_p", ctypes.c_int32), ("probe_seed", ctypes.c_int32), ("site_begin", ctypes.c_int32),
                ("site_end", ctypes.c_int32), ("band_rows", ctypes.c_int32)]


class kpm_rmft_opts(ctypes.Structure):
    _fields_ = [("n_target", ctypes.c_double), ("alpha", ctypes.c_double), ("alpha_n", ctypes.c_double),
                ("eta", ctypes.c_double), ("tol", ctypes.c_double), ("paramagnetic", ctypes.c_int32),
                ("strict", ctypes.c_int32), ("anderson", ctypes.c_int32), ("sync_every", ctypes.c_int32)]


class kpm_rmft_stats(ctypes.Structure):
    _fields_ = [("residual", ctypes.c_double), ("density_error", ctypes.c_double), ("mu", ctypes.c_double),
                ("omega", ctypes.c_double), ("a", ctypes.c_double), ("b", ctypes.c_double),
                ("recursion_ms", ctypes.c_double), ("recursion_bytes", ctypes.c_double),
                ("iterations", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("kernel_launches", ctypes.c_int32), ("recursion_launches", ctypes.c_int32)]


_P = ctypes.c_void_p
_SIGNATURES = {
    "kpm_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int]),
    "kpm_destroy": (ctypes.c_int, [_P]),
    "kpm_set_scratch_budget": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "kpm_sync_status": (ctypes.c_int, [_P, _P]),
    "kpm_inject_lost_copy": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double]),
    "kpm_measure_peaks": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double), _P]),
    "rmft_prepare": (ctypes.c_int, [_P, ctypes.POINTER(kpm_model), ctypes.POINTER(kpm_opts), _P, _P, _P, _P, _P, _P,
                                    _P]),
    "rmft_update": (ctypes.c_int, [_P, ctypes.POINTER(kpm_model), ctypes.POINTER(kpm_rmft_opts), _P, _P, _P, _P, _P]),
    "kpm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "kpm_last_error": (ctypes.c_char_p, [_P]),
    "kpm_peierls_phases": (ctypes.c_int, [_P, ctypes.POINTER(kpm_model), _P, _P]),
    "kpm_build_H": (ctypes.c_int, [_P, ctypes.POINTER(kpm_model), _P, _P, ctypes.c_double, _P, _P, _P]),
    "kpm_bounds": (ctypes.c_int, [_P, ctypes.POINTER(kpm_model), _P, ctypes.c_double, _P, _P]),
    "kpm_observables": (ctypes.c_int, [_P, ctypes.POINTER(kpm_model), ctypes.POINTER(kpm_opts), _P, _P, _P, _P, _P]),
    "rmft_iterate": (ctypes.c_int, [_P, ctypes.POINTER(kpm_model), ctypes.POINTER(kpm_opts),
                                    ctypes.POINTER(kpm_rmft_opts), _P, _P, _P, ctypes.c_int,
                                    ctypes.POINTER(kpm_rmft_stats), _P]),
    "kpm_order_parameters": (ctypes.c_int, [_P, ctypes.POINTER(kpm_model), _P, _P, _P, _P, _P]),
    "kpm_ldos": (ctypes.c_int, [_P, ctypes.POINTER(kpm_model), ctypes.POINTER(kpm_opts), _P, _P, _P, ctypes.c_int,
                                _P, ctypes.c_double, ctypes.c_double, _P, _P]),
    "kpm_observables_noalloc": (ctypes.c_int, [ctypes.POINTER(kpm_model), ctypes.POINTER(kpm_opts), _P, _P, _P,
                                               _P, _P]),
    "kpm_autotune": (ctypes.c_int, [_P, ctypes.POINTER(kpm_model), ctypes.POINTER(kpm_opts), _P, _P,
                                    ctypes.POINTER(kpm_opts), ctypes.POINTER(ctypes.c_double), _P]),
    "rmft_iterate_batched": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(kpm_model), ctypes.POINTER(kpm_opts),
                                            ctypes.POINTER(kpm_rmft_opts), ctypes.POINTER(ctypes.c_void_p),
                                            ctypes.POINTER(ctypes.c_void_p), _P, ctypes.c_int,
                                            ctypes.POINTER(kpm_rmft_stats), _P]),
    "kpm_backward": (ctypes.c_int, [_P, ctypes.POINTER(kpm_model), ctypes.POINTER(kpm_opts), _P, _P, _P,
                                    ctypes.c_double, _P, _P, _P, _P, ctypes.c_int, _P]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libkpm.so once; raise if it is not built (no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class KPMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def _ptr(x):
    """Raw pointer of a torch tensor or numpy array (contiguous, float64)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr())
    if hasattr(x, "ctypes"):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(x.ctypes.data)
    raise TypeError(f"unsupported buffer type {type(x)}")


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def make_model(nx, ny, t=1.0, tp=-0.3, J=0.3, flux=1, gutzwiller=True):
    return kpm_model(nx, ny, flux, 1 if gutzwiller else 0, t, tp, J)


def make_opts(M, precision=KPM_FP32, block_width=0, cols_per_block=0, margin=0.01, flags=0, probe_p=0,
              probe_seed=0, temperature=0.0, site_begin=0, site_end=0, band_rows=0):
    return kpm_opts(M, precision, block_width, cols_per_block, margin, temperature, flags, probe_p, probe_seed,
                    site_begin, site_end, band_rows)


def make_rmft_opts(n_target, alpha=0.5, alpha_n=0.05, eta=0.5, tol=1e-7, paramagnetic=True, strict=False,
                   anderson=0, sync_every=0):
    return kpm_rmft_opts(n_target, alpha, alpha_n, eta, tol, 1 if paramagnetic else 0, 1 if strict else 0,
                         int(anderson), int(sync_every))


class Context:
    """Owns one kpm_ctx (scratch memory of the library on one GPU)."""

    def __init__(self, device: int = 0):
        lib = load()
        h = ctypes.c_void_p()
        st = lib.kpm_create(ctypes.byref(h), device)
        if st != KPM_OK:
            raise KPMError(st, f"kpm_create: {lib.kpm_strerror(st).decode()}")
        self.handle = h
        self.lib = lib

    def check(self, st, what):
        if st != KPM_OK:
            msg = self.lib.kpm_last_error(self.handle).decode()
            raise KPMError(st, f"{what}: {self.lib.kpm_strerror(st).decode()}: {msg}")
        return st

    def close(self):
        if self.handle:
            self.lib.kpm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kpm_create(device: int = 0) -> Context:
    return Context(device)


def kpm_destroy(ctx: Context):
    ctx.close()


def kpm_set_scratch_budget(ctx: Context, nbytes: int):
    return ctx.check(ctx.lib.kpm_set_scratch_budget(ctx.handle, int(nbytes)), "kpm_set_scratch_budget")


def kpm_sync_status(ctx: Context, stream=None):
    return ctx.check(ctx.lib.kpm_sync_status(ctx.handle, _stream(stream)), "kpm_sync_status")


def kpm_inject_lost_copy(ctx: Context, count, wait_limit_s=0.0):
    return ctx.check(ctx.lib.kpm_inject_lost_copy(ctx.handle, int(count), float(wait_limit_s)),
                     "kpm_inject_lost_copy")


def kpm_measure_peaks(ctx: Context, stream=None):
    """(FP64 TFLOP/s, FP32 TFLOP/s, packed f32x2 TFLOP/s, median SM MHz)."""
    out = (ctypes.c_double * 4)()
    ctx.check(ctx.lib.kpm_measure_peaks(ctx.handle, out, _stream(stream)), "kpm_measure_peaks")
    return tuple(out)


def rmft_prepare(ctx: Context, model, opts, phi, params, mu_eff, fields, ab, mu_out, stream=None):
    return ctx.check(ctx.lib.rmft_prepare(ctx.handle, ctypes.byref(model), ctypes.byref(opts), _ptr(phi),
                                          _ptr(params), _ptr(mu_eff), _ptr(fields), _ptr(ab), _ptr(mu_out),
                                          _stream(stream)), "rmft_prepare")


def rmft_update(ctx: Context, model, ropts, params, obs, mu_eff, stats_out, stream=None):
    return ctx.check(ctx.lib.rmft_update(ctx.handle, ctypes.byref(model), ctypes.byref(ropts), _ptr(params),
                                         _ptr(obs), _ptr(mu_eff), _ptr(stats_out), _stream(stream)), "rmft_update")


def kpm_peierls_phases(ctx: Context, model, phi, stream=None):
    return ctx.check(ctx.lib.kpm_peierls_phases(ctx.handle, ctypes.byref(model), _ptr(phi), _stream(stream)),
                     "kpm_peierls_phases")


def kpm_build_H(ctx: Context, model, phi, params, mu, fields, w_out=None, stream=None):
    return ctx.check(ctx.lib.kpm_build_H(ctx.handle, ctypes.byref(model), _ptr(phi), _ptr(params), float(mu),
                                         _ptr(fields), _ptr(w_out), _stream(stream)), "kpm_build_H")


def kpm_bounds(ctx: Context, model, fields, margin, ab, stream=None):
    return ctx.check(ctx.lib.kpm_bounds(ctx.handle, ctypes.byref(model), _ptr(fields), float(margin), _ptr(ab),
                                        _stream(stream)), "kpm_bounds")


def kpm_observables(ctx: Context, model, opts, fields, ab, obs, omega=None, stream=None):
    return ctx.check(ctx.lib.kpm_observables(ctx.handle, ctypes.byref(model), ctypes.byref(opts), _ptr(fields),
                                             _ptr(ab), _ptr(obs), _ptr(omega), _stream(stream)), "kpm_observables")


def rmft_iterate(ctx: Context, model, opts, ropts, phi, params, mu_eff, n_iter, stream=None, check=True):
    """Returns (status, kpm_rmft_stats)."""
    stats = kpm_rmft_stats()
    st = ctx.lib.rmft_iterate(ctx.handle, ctypes.byref(model), ctypes.byref(opts), ctypes.byref(ropts),
                              _ptr(phi), _ptr(params), _ptr(mu_eff), int(n_iter), ctypes.byref(stats),
                              _stream(stream))
    if check:
        ctx.check(st, "rmft_iterate")
    return st, stats


def kpm_autotune(ctx: Context, model, opts, fields, ab, stream=None):
    """Returns (best kpm_opts, ms per recursion step or -1 when cached)."""
    best = kpm_opts()
    ms = ctypes.c_double()
    ctx.check(ctx.lib.kpm_autotune(ctx.handle, ctypes.byref(model), ctypes.byref(opts), _ptr(fields), _ptr(ab),
                                   ctypes.byref(best), ctypes.byref(ms), _stream(stream)), "kpm_autotune")
    return best, ms.value


def rmft_iterate_batched(ctx: Context, models, opts, ropts, phis, params, mu_eff, n_iter, stream=None, check=True):
    """Batched iterations of independent cells; models/ropts: lists of structs,
    phis/params: lists of CUDA tensors, mu_eff: CUDA tensor of len(models).
    Returns (status, list of kpm_rmft_stats)."""
    n = len(models)
    M_arr = (kpm_model * n)(*models)
    R_arr = (kpm_rmft_opts * n)(*ropts)
    P_arr = (ctypes.c_void_p * n)(*[x.data_ptr() for x in phis])
    Q_arr = (ctypes.c_void_p * n)(*[x.data_ptr() for x in params])
    S_arr = (kpm_rmft_stats * n)()
    st = ctx.lib.rmft_iterate_batched(ctx.handle, n, M_arr, ctypes.byref(opts), R_arr, P_arr, Q_arr, _ptr(mu_eff),
                                      int(n_iter), S_arr, _stream(stream))
    if check:
        ctx.check(st, "rmft_iterate_batched")
    return st, list(S_arr)


def kpm_backward(ctx: Context, model, opts, fields, ab, grad_obs, grad_omega, grad_fields, phi=None, params=None,
                 grad_phi=None, ckpt_every=0, stream=None):
    return ctx.check(ctx.lib.kpm_backward(ctx.handle, ctypes.byref(model), ctypes.byref(opts), _ptr(fields), _ptr(ab),
                                          _ptr(grad_obs), float(grad_omega), _ptr(grad_fields), _ptr(phi),
                                          _ptr(params), _ptr(grad_phi), int(ckpt_every), _stream(stream)),
                     "kpm_backward")


def kpm_observables_noalloc(model, opts, fields, ab, obs, omega=None, stream=None):
    """kpm_observables without a context or any device allocation (for
    callers whose device memory is owned by another allocator, or who cannot
    afford cudaMalloc's synchronisation).  Uses the library's fixed 48 MiB
    per-device scratch array; calls that overlap on the GPU race, so
    serialise them.  Returns the C status (0 on success)."""
    lib = load()
    return lib.kpm_observables_noalloc(ctypes.byref(model), ctypes.byref(opts), _ptr(fields), _ptr(ab),
                                       _ptr(obs), _ptr(omega), _stream(stream))


def kpm_ldos(ctx: Context, model, opts, fields, ab, params, omega, ldos, gamma_alpha=0.25, gamma0=3e-4, stream=None):
    """Local density of states [2][len(omega)][N] into `ldos` (device); omega a
    float64 numpy array or CUDA tensor; params a CUDA tensor or None."""
    import numpy as np
    if not hasattr(omega, "data_ptr"):
        omega = np.ascontiguousarray(omega, dtype=np.float64)
    return ctx.check(ctx.lib.kpm_ldos(ctx.handle, ctypes.byref(model), ctypes.byref(opts), _ptr(fields), _ptr(ab),
                                      _ptr(params), int(len(omega)), _ptr(omega), float(gamma_alpha), float(gamma0),
                                      _ptr(ldos), _stream(stream)), "kpm_ldos")


def kpm_order_parameters(ctx: Context, model, phi, params, delta_out, mag_out, stream=None):
    """Physical pairing Delta_i (2N doubles: re, im) and staggered magnetisation M_i (N)."""
    return ctx.check(ctx.lib.kpm_order_parameters(ctx.handle, ctypes.byref(model), _ptr(phi), _ptr(params),
                                                  _ptr(delta_out), _ptr(mag_out), _stream(stream)),
                     "kpm_order_parameters")
