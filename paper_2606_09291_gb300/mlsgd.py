"""Thin ctypes binding of libmlsgd (include/mlsgd.h): argument marshalling only.

Every function keeps the C name and forwards device pointers (torch CUDA
tensors) and the current torch stream to the library; all computation runs in
the library's CUDA kernels.  There is no CPU fallback: if the library cannot
be loaded, every call raises.
"""
import ctypes
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmlsgd.so")

MLSGD_FP64, MLSGD_MIXED = 0, 1
S_COUNT, S_SHIFT, S_MEAN_DY, S_S2_DY, S_S2_DX, S_PHI_MAX, S_ITERS, S_NOCONV = range(8)
NSCALARS = 8
STATUS = {0: "ok", 1: "EINVAL", 2: "ENOMEM", 3: "ENOCONV", 4: "ENONFINITE", 5: "ECUDA", 6: "ENOTIMPL"}


class Config(ctypes.Structure):
    _fields_ = [("n_levels", ctypes.c_int), ("n0", ctypes.c_int), ("ctrl_level", ctypes.c_int),
                ("n_modes", ctypes.c_int), ("corr_len", ctypes.c_double), ("sigma", ctypes.c_double),
                ("theta", ctypes.c_double), ("alpha", ctypes.c_double), ("rtol", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("precision", ctypes.c_int), ("inner_iters", ctypes.c_int),
                ("max_batch", ctypes.c_int), ("field_tc", ctypes.c_int), ("ir_steps", ctypes.c_int),
                ("field_model", ctypes.c_int), ("target_freq", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("stencil", ctypes.c_int), ("z_chunks", ctypes.c_int), ("omega", ctypes.c_double),
                ("inner_iters_next", ctypes.c_int)]


class LevelStats(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int), ("field_dev", ctypes.c_void_p), ("scalars_dev", ctypes.c_void_p)]


class StepReport(ctypes.Structure):
    _fields_ = [("grad_norm", ctypes.c_double), ("risk", ctypes.c_double), ("ey", ctypes.c_double),
                ("shift", ctypes.c_double), ("truncated", ctypes.c_int), ("err_sam", ctypes.c_double),
                ("err_num", ctypes.c_double), ("alpha_hat", ctypes.c_double), ("eps2", ctypes.c_double),
                ("next_levels", ctypes.c_int), ("next_counts", ctypes.c_int64 * 16),
                ("ex_norm2", ctypes.c_double), ("c_hat", ctypes.c_double),
                ("mean_dx_norm2", ctypes.c_double * 16), ("v2", ctypes.c_double * 16),
                ("tau", ctypes.c_double), ("l_hat", ctypes.c_double), ("tau_fallback", ctypes.c_int),
                ("m2_dx", ctypes.c_double * 16), ("m2_dy", ctypes.c_double * 16),
                ("mean_dx_norm", ctypes.c_double * 16), ("mean_dy_abs", ctypes.c_double * 16),
                ("beta_x", ctypes.c_double), ("beta_y", ctypes.c_double), ("alpha_x", ctypes.c_double),
                ("alpha_y", ctypes.c_double), ("z_norm", ctypes.c_double), ("objective", ctypes.c_double)]

_PER_LEVEL = ("mean_dx_norm2", "v2", "m2_dx", "m2_dy", "mean_dx_norm", "mean_dy_abs")


class ProfileEntry(ctypes.Structure):
    _fields_ = [("cls", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("flops", ctypes.c_double)]


EXPORTS = ["mlsgd_create", "mlsgd_destroy", "mlsgd_last_error", "mlsgd_status_string", "mlsgd_n_ctrl_cells",
           "mlsgd_workspace_bytes", "mlsgd_mode_table", "mlsgd_sample_field", "mlsgd_solve_state_adjoint",
           "mlsgd_level_gradient", "mlsgd_stats_reset", "mlsgd_stats_merge", "mlsgd_step",
           "mlsgd_launch_count", "mlsgd_profile_start", "mlsgd_profile_stop", "mlsgd_solve_state_adjoint_noalloc",
           "mlsgd_sample_field_tc", "mlsgd_step_adaptive", "mlsgd_set_workspace"]

_lib = None


def load(path=LIB_PATH):
    """Load the library (once).  Raises OSError if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError("libmlsgd.so not built (run __graft_entry__.build()): " + path)
    L = ctypes.CDLL(path)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    L.mlsgd_create.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(vp)]
    L.mlsgd_destroy.argtypes = [vp]
    L.mlsgd_destroy.restype = None
    L.mlsgd_last_error.argtypes = [vp]
    L.mlsgd_last_error.restype = ctypes.c_char_p
    L.mlsgd_status_string.argtypes = [i32]
    L.mlsgd_status_string.restype = ctypes.c_char_p
    L.mlsgd_n_ctrl_cells.argtypes = [vp]
    L.mlsgd_n_ctrl_cells.restype = i64
    L.mlsgd_workspace_bytes.argtypes = [vp, i32, i32]
    L.mlsgd_workspace_bytes.restype = ctypes.c_size_t
    L.mlsgd_mode_table.argtypes = [vp, vp, vp]
    L.mlsgd_sample_field.argtypes = [vp, i32, i32, i32, i64, i32, vp, vp, vp]
    L.mlsgd_solve_state_adjoint.argtypes = [vp, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp]
    L.mlsgd_level_gradient.argtypes = [vp, i32, i32, i64, i32, vp, ctypes.POINTER(LevelStats), vp]
    L.mlsgd_stats_reset.argtypes = [vp, ctypes.POINTER(LevelStats), vp]
    L.mlsgd_stats_merge.argtypes = [vp, ctypes.POINTER(LevelStats), ctypes.POINTER(LevelStats), vp]
    L.mlsgd_step.argtypes = [vp, ctypes.POINTER(LevelStats), i32, dbl, dbl, i32, vp, vp, ctypes.POINTER(StepReport), vp]
    L.mlsgd_step_adaptive.argtypes = [vp, ctypes.POINTER(LevelStats), i32, dbl, dbl, dbl, i32, vp, vp,
                                      ctypes.POINTER(StepReport), vp]
    L.mlsgd_sample_field_tc.argtypes = [vp, i32, i32, i32, i64, i32, vp, vp, vp]
    L.mlsgd_set_workspace.argtypes = [vp, vp, ctypes.c_size_t]
    L.mlsgd_solve_state_adjoint_noalloc.argtypes = [vp, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp]
    L.mlsgd_launch_count.argtypes = []
    L.mlsgd_launch_count.restype = i64
    L.mlsgd_profile_start.argtypes = [ctypes.c_char_p]
    L.mlsgd_profile_stop.argtypes = [ctypes.POINTER(ProfileEntry), i32]
    for name in EXPORTS:
        if name not in ("mlsgd_destroy", "mlsgd_last_error", "mlsgd_status_string", "mlsgd_n_ctrl_cells",
                        "mlsgd_workspace_bytes", "mlsgd_mode_table", "mlsgd_launch_count"):
            getattr(L, name).restype = i32
    L.mlsgd_mode_table.restype = i32
    _lib = L
    return L


def mlsgd_launch_count():
    return int(load().mlsgd_launch_count())


def mlsgd_profile_start(kernel_class):
    load().mlsgd_profile_start(None if kernel_class is None else kernel_class.encode())


def mlsgd_profile_stop(max_entries=128):
    """Returns {class: dict(launches, total_ms, bytes, flops)}."""
    arr = (ProfileEntry * max_entries)()
    n = load().mlsgd_profile_stop(arr, max_entries)
    if n < 0:
        raise RuntimeError("mlsgd_profile_stop: CUDA error")
    return {arr[i].cls.decode(): dict(launches=arr[i].launches, total_ms=arr[i].total_ms, bytes=arr[i].bytes,
                                      flops=arr[i].flops) for i in range(min(n, max_entries))}


class MlsgdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


def _ptr(t):
    if t is None:
        return None
    assert isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Context:
    """Owns one mlsgd_ctx; methods mirror the C entry points."""

    def __init__(self, **cfg):
        L = load()
        c = Config()
        defaults = dict(n_levels=3, n0=8, ctrl_level=None, n_modes=64, corr_len=0.3, sigma=1.0, theta=1.0,
                        alpha=1e-4, rtol=1e-8, max_iter=200, precision=MLSGD_FP64, inner_iters=0,
                        max_batch=256, field_tc=0, ir_steps=0, field_model=0,
                        target_freq=1, seed=0, stencil=0, z_chunks=0, omega=0.0, inner_iters_next=0)
        defaults.update(cfg)
        if defaults["ctrl_level"] is None:
            defaults["ctrl_level"] = defaults["n_levels"] - 1
        if isinstance(defaults["precision"], str):
            defaults["precision"] = {"fp64": MLSGD_FP64, "mixed": MLSGD_MIXED}[defaults["precision"]]
        for k, v in defaults.items():
            setattr(c, k, v)
        self.cfg = defaults
        self._c = c
        h = ctypes.c_void_p()
        st = L.mlsgd_create(ctypes.byref(c), ctypes.byref(h))
        if st != 0:
            raise MlsgdError(st, "mlsgd_create failed")
        self.h = h
        self.L = L
        self.n_ctrl = int(L.mlsgd_n_ctrl_cells(h))

    def close(self):
        if getattr(self, "h", None):
            self.L.mlsgd_destroy(self.h)
            self.h = None

    __del__ = close

    def _check(self, st):
        if st != 0:
            raise MlsgdError(st, self.L.mlsgd_last_error(self.h).decode())

    def N(self, level):
        return self.cfg["n0"] << level

    # --- C entry points -------------------------------------------------
    def mlsgd_workspace_bytes(self, level, n_samples):
        return int(self.L.mlsgd_workspace_bytes(self.h, level, n_samples))

    def mlsgd_set_workspace(self, ptr, nbytes):
        """Use [ptr, ptr + nbytes) of caller-owned device memory as scratch (ptr an int
        device address, 0 with nbytes 0 to return to the context's own scratch)."""
        self._check(self.L.mlsgd_set_workspace(self.h, ctypes.c_void_p(ptr) if ptr else None, nbytes))

    def mlsgd_mode_table(self):
        K = self.cfg["n_modes"]
        idx = (ctypes.c_int * (3 * K))()
        lam = (ctypes.c_double * K)()
        n1d = self.L.mlsgd_mode_table(self.h, idx, lam)
        return [tuple(idx[3 * k:3 * k + 3]) for k in range(K)], list(lam), n1d

    def mlsgd_sample_field(self, it, level, grid, first, n, xi=None, log_a=None, stream=None):
        self._check(self.L.mlsgd_sample_field(self.h, it, level, grid, first, n, _ptr(xi), _ptr(log_a),
                                              _stream(stream)))

    def mlsgd_sample_field_tc(self, it, level, grid, first, n, log_a_f32=None, a_bf16=None, stream=None):
        self._check(self.L.mlsgd_sample_field_tc(self.h, it, level, grid, first, n, _ptr(log_a_f32), _ptr(a_bf16),
                                                 _stream(stream)))

    def mlsgd_solve_state_adjoint(self, grid, n, log_a, z, y, q, phi, iters, status, stream=None):
        return self.L.mlsgd_solve_state_adjoint(self.h, grid, n, _ptr(log_a), _ptr(z), _ptr(y), _ptr(q), _ptr(phi),
                                                _ptr(iters), _ptr(status), _stream(stream))

    def mlsgd_solve_state_adjoint_noalloc(self, grid, n, log_a, z, y, q, phi, iters, status, stream=None):
        """Same as mlsgd_solve_state_adjoint with scratch from the library's static
        device array (no device allocation); returns the C status."""
        return self.L.mlsgd_solve_state_adjoint_noalloc(self.h, grid, n, _ptr(log_a), _ptr(z), _ptr(y), _ptr(q),
                                                        _ptr(phi), _ptr(iters), _ptr(status), _stream(stream))

    def mlsgd_level_gradient(self, it, level, first, n, z, stats, stream=None):
        self._check(self.L.mlsgd_level_gradient(self.h, it, level, first, n, _ptr(z), ctypes.byref(stats.c),
                                                _stream(stream)))

    def mlsgd_stats_reset(self, stats, stream=None):
        self._check(self.L.mlsgd_stats_reset(self.h, ctypes.byref(stats.c), _stream(stream)))

    def mlsgd_stats_merge(self, dst, src, stream=None):
        self._check(self.L.mlsgd_stats_merge(self.h, ctypes.byref(dst.c), ctypes.byref(src.c), _stream(stream)))

    def mlsgd_step(self, stats_list, tau, z, eta=0.9, max_levels=None, grad=None, stream=None):
        n = len(stats_list)
        arr = (LevelStats * n)(*[s.c for s in stats_list])
        rep = StepReport()
        ml = self.cfg["n_levels"] if max_levels is None else max_levels
        self._check(self.L.mlsgd_step(self.h, arr, n, tau, eta, ml, _ptr(z), _ptr(grad), ctypes.byref(rep),
                                      _stream(stream)))
        return _report(rep, n)

    def mlsgd_step_adaptive(self, stats_list, tau0, tau_prev, z, grad_prev, eta=0.9, max_levels=None, stream=None):
        n = len(stats_list)
        arr = (LevelStats * n)(*[s.c for s in stats_list])
        rep = StepReport()
        ml = self.cfg["n_levels"] if max_levels is None else max_levels
        self._check(self.L.mlsgd_step_adaptive(self.h, arr, n, tau0, tau_prev, eta, ml, _ptr(z), _ptr(grad_prev),
                                               ctypes.byref(rep), _stream(stream)))
        return _report(rep, n)

    # --- helpers (allocation only) --------------------------------------
    def new_stats(self, level, device="cuda"):
        s = Stats(level, self.n_ctrl, device)
        self.mlsgd_stats_reset(s)
        return s


def _report(rep, n):
    out = {k: getattr(rep, k) for k, _ in StepReport._fields_ if k != "next_counts" and k not in _PER_LEVEL}
    out["next_counts"] = [int(rep.next_counts[l]) for l in range(rep.next_levels)]
    for k in _PER_LEVEL:
        out[k] = [getattr(rep, k)[l] for l in range(n)]
    return out


class Stats:
    """Device-resident mlsgd_level_stats: field [n_ctrl] and scalars [8], FP64."""

    def __init__(self, level, n_ctrl, device="cuda"):
        self.field = torch.zeros(n_ctrl, dtype=torch.float64, device=device)
        self.scalars = torch.zeros(NSCALARS, dtype=torch.float64, device=device)
        self.c = LevelStats(level, self.field.data_ptr(), self.scalars.data_ptr())
        self.level = level

    def host(self):
        s = self.scalars.cpu().tolist()
        return dict(count=s[S_COUNT], shift=s[S_SHIFT], mean_dy=s[S_MEAN_DY], s2_dy=s[S_S2_DY], s2_dx=s[S_S2_DX],
                    phi_max=s[S_PHI_MAX], iters=s[S_ITERS], noconv=s[S_NOCONV])
