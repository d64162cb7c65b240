"""ctypes binding of libaimx (argument marshalling only; every step runs in the library).

The library must have been built (``paper_2009_02281_gb300.build.build()``);
there is no fallback: a missing library raises ``AimxError``.
"""

import ctypes
import os

import numpy as np

from . import build as _build

EFIE = 0
PMCHWT = 1
CFIE = 2
F32 = 0
F64 = 1

_STATUS = {0: "ok", -1: "invalid argument", -2: "invalid mesh", -3: "stencil outside the grid",
           -4: "out of memory", -5: "CUDA error", -6: "bounded device wait expired",
           -7: "call not valid for this context", -8: "static-data file error",
           1: "solver did not reach the tolerance"}


class AimxError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__("aimx status %d (%s)%s" % (code, _STATUS.get(code, "?"), (": " + msg) if msg else ""))
        self.code = code


class _Mesh(ctypes.Structure):
    _fields_ = [("nv", ctypes.c_int32), ("nt", ctypes.c_int32),
                ("xyz", ctypes.POINTER(ctypes.c_double)), ("tri", ctypes.POINTER(ctypes.c_int32))]


class _Material(ctypes.Structure):
    _fields_ = [("formulation", ctypes.c_int32), ("eps_out", ctypes.c_double), ("mu_out", ctypes.c_double),
                ("eps_in", ctypes.c_double), ("mu_in", ctypes.c_double), ("sigma", ctypes.c_double),
                ("cfie_alpha", ctypes.c_double)]


class Schedule(ctypes.Structure):
    """Product schedule (aimx_schedule): variant 0 fused/register, 1 fused/shared memory, 2 generic."""
    _fields_ = [("variant", ctypes.c_int32), ("pass_", ctypes.c_int32), ("ms", ctypes.c_double)]

    def as_dict(self):
        return {"variant": int(self.variant), "pass": int(self.pass_), "ms": float(self.ms)}


class Port(ctypes.Structure):
    """Delta-gap port: plane (point, normal) restricted to the box [box_lo, box_hi] (aimx_port)."""
    _fields_ = [("point", ctypes.c_double * 3), ("normal", ctypes.c_double * 3), ("box_lo", ctypes.c_double * 3),
                ("box_hi", ctypes.c_double * 3)]

    @classmethod
    def make(cls, point, normal, box_lo, box_hi):
        p = cls()
        for a in range(3):
            p.point[a], p.normal[a] = float(point[a]), float(normal[a])
            p.box_lo[a], p.box_hi[a] = float(box_lo[a]), float(box_hi[a])
        return p


class _Grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32 * 3), ("h", ctypes.c_double * 3), ("origin", ctypes.c_double * 3),
                ("near_radius", ctypes.c_int32), ("pad", ctypes.c_int32 * 3)]


class _Info(ctypes.Structure):
    _fields_ = [("n_basis", ctypes.c_int32), ("n_unknowns", ctypes.c_int32), ("near_nnz", ctypes.c_int64),
                ("grid_n", ctypes.c_int32 * 3), ("pad", ctypes.c_int32 * 3), ("grid_h", ctypes.c_double * 3),
                ("grid_origin", ctypes.c_double * 3), ("order", ctypes.c_int32),
                ("formulation", ctypes.c_int32), ("device_bytes", ctypes.c_int64)]


_lib = None

# (name, restype, argtypes) of every exported entry point
_SIGS = [
    ("aimx_setup", ctypes.c_int, [ctypes.POINTER(_Mesh), ctypes.POINTER(_Material), ctypes.POINTER(_Grid),
                                  ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    ("aimx_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("aimx_info", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(_Info)]),
    ("aimx_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("aimx_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
    ("aimx_matvec", ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    ("aimx_matvec_host", ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    ("aimx_export_setup", ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_void_p] * 7),
    ("aimx_set_path", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("aimx_set_linear_term", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("aimx_export_linear_term", ctypes.c_int, [ctypes.c_void_p] * 6),
    ("aimx_set_conventional_aim", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("aimx_set_schedule", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("aimx_get_schedule", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("aimx_wait_timeouts", ctypes.c_int, [ctypes.c_void_p]),
    ("aimx_set_wait_limit", ctypes.c_int, [ctypes.c_int64]),
    ("aimx_set_plane_cap", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("aimx_autotune", ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_char_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    ("aimx_export_aim_near", ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p]),
    ("aimx_set_charge_form", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("aimx_export_charge", ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_void_p] * 7),
    ("aimx_matvec_path", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("aimx_profile", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("aimx_profile_read", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("aimx_profile_stage_name", ctypes.c_char_p, [ctypes.c_int]),
    ("aimx_measure_fp32_peak", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    ("aimx_matvec_noalloc", ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p]),
    ("aimx_solve", ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("aimx_rhs_planewave", ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("aimx_farfield", ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("aimx_sweep", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                  ctypes.c_void_p]),
    ("aimx_sweep_batched", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("aimx_precond_apply", ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("aimx_batch_solve", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("aimx_batch_create", ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_void_p)]),
    ("aimx_batch_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("aimx_batch_matvec", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p]),
    ("aimx_batch_graph_nodes", ctypes.c_int64, [ctypes.c_void_p]),
    ("aimx_batch_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
    ("aimx_port_vectors", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p]),
    ("aimx_rhs_ports", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p]),
    ("aimx_port_currents", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("aimx_sweep_ports", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p]),
    ("aimx_save_static", ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p]),
    ("aimx_load_static", ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(ctypes.c_void_p)]),
    ("aimx_gnn_create", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    ("aimx_gnn_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("aimx_gnn_num_params", ctypes.c_int64, [ctypes.c_void_p]),
    ("aimx_gnn_set_params", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]),
    ("aimx_gnn_get_params", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]),
    ("aimx_gnn_loss_grad", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_int,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                          ctypes.c_void_p, ctypes.c_void_p]),
    ("aimx_gnn_train_step", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_int,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    ("aimx_gnn_attach", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("aimx_gnn_features", ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("aimx_gnn_outputs", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p,
                                        ctypes.c_void_p]),
]

PRECOND_DIAG = 0
PRECOND_NONE = 1
PRECOND_BLOCK = 2
PRECOND_LEARNED = 3


class _AdamOpts(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_double), ("clip", ctypes.c_double)]


class _SolveOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("restart", ctypes.c_int32), ("max_iter", ctypes.c_int32),
                ("max_refine", ctypes.c_int32), ("inner_precision", ctypes.c_int32), ("precond", ctypes.c_int32),
                ("use_x0", ctypes.c_int32), ("learned_trial", ctypes.c_int32)]


class _SolveStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("refinements", ctypes.c_int32), ("rel_residual", ctypes.c_double),
                ("status", ctypes.c_int32), ("precond_used", ctypes.c_int32)]


def _opts(tol, restart, max_iter, inner_precision, precond, use_x0=0, max_refine=0, learned_trial=0):
    return _SolveOpts(float(tol), int(restart), int(max_iter), int(max_refine), int(inner_precision), int(precond),
                      int(use_x0), int(learned_trial))


def _stats_list(arr):
    return [dict(iterations=s.iterations, refinements=s.refinements, rel_residual=s.rel_residual, status=s.status,
                 precond_used=s.precond_used) for s in arr]


def lib_path():
    return _build.LIB


def load(build_if_missing=False):
    """Load libaimx.so (optionally building it first); raises AimxError if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise AimxError(-5, "libaimx.so not built at %s; run paper_2009_02281_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    for name, res, args in _SIGS:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def wait_timeouts():
    """Bounded device waits that ran out since the last call (0 normally); resets the count."""
    n = ctypes.c_int(0)
    rc = load().aimx_wait_timeouts(ctypes.byref(n))
    if rc != 0:
        raise AimxError(rc)
    return n.value


def set_wait_limit(cycles):
    """Test hook (aimx_set_wait_limit): per-tile copy-wait limit of the TMA z-pass; <= 0 restores the default."""
    rc = load().aimx_set_wait_limit(int(cycles))
    if rc != 0:
        raise AimxError(rc)


def measure_fp32_peak(packed=False):
    """FP32 TFLOP/s of the current device (aimx_measure_fp32_peak): scalar or packed two-lane FMAs."""
    t = ctypes.c_double(0.0)
    rc = load().aimx_measure_fp32_peak(1 if packed else 0, ctypes.byref(t))
    if rc != 0:
        raise AimxError(rc)
    return t.value


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


class Context:
    """An AIMx problem on the current CUDA device (wraps aimx_setup / aimx_destroy)."""

    def __init__(self, xyz, tri, grid_n, order=2, formulation=EFIE, eps_out=1.0, mu_out=1.0,
                 eps_in=1.0, mu_in=1.0, h=None, origin=None, near_radius=3, pad=None, sigma=0.0, cfie_alpha=0.0):
        self._lib = load()
        self._xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        self._tri = np.ascontiguousarray(tri, dtype=np.int32)
        mesh = _Mesh(len(self._xyz), len(self._tri),
                     self._xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                     self._tri.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        mat = _Material(formulation, eps_out, mu_out, eps_in, mu_in, sigma, cfie_alpha)
        g = _Grid()
        for a in range(3):
            g.n[a] = int(grid_n[a])
            g.h[a] = 0.0 if h is None else float(h[a])
            g.origin[a] = 0.0 if origin is None else float(origin[a])
            g.pad[a] = 0 if pad is None else int(pad[a])
        g.near_radius = int(near_radius)
        out = ctypes.c_void_p()
        rc = self._lib.aimx_setup(ctypes.byref(mesh), ctypes.byref(mat), ctypes.byref(g), int(order),
                                  ctypes.byref(out))
        if rc != 0:
            raise AimxError(rc)
        self._ctx = out
        self.info = self._info()
        self.N = self.info["n_basis"]
        self.nunk = self.info["n_unknowns"]
        self.formulation = formulation

    @classmethod
    def load_static(cls, path):
        """A context restored from a file written by save_static (aimx_load_static)."""
        self = cls.__new__(cls)
        self._lib = load()
        out = ctypes.c_void_p()
        rc = self._lib.aimx_load_static(os.fsencode(path), ctypes.byref(out))
        if rc != 0:
            raise AimxError(rc, str(path))
        self._ctx = out
        self.info = self._info()
        self.N = self.info["n_basis"]
        self.nunk = self.info["n_unknowns"]
        self.formulation = self.info["formulation"]
        return self

    def save_static(self, path):
        """Write the frequency-independent setup products to a file (aimx_save_static)."""
        self._check(self._lib.aimx_save_static(self._ctx, os.fsencode(path)))

    def _check(self, rc):
        if rc < 0:
            msg = self._lib.aimx_last_error(self._ctx)
            raise AimxError(rc, msg.decode() if msg else "")
        return rc

    def _info(self):
        inf = _Info()
        self._check(self._lib.aimx_info(self._ctx, ctypes.byref(inf)))
        return dict(n_basis=inf.n_basis, n_unknowns=inf.n_unknowns, near_nnz=inf.near_nnz,
                    grid_n=tuple(inf.grid_n), pad=tuple(inf.pad), grid_h=tuple(inf.grid_h),
                    grid_origin=tuple(inf.grid_origin), order=inf.order, formulation=inf.formulation,
                    device_bytes=inf.device_bytes)

    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.aimx_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- hot path
    def matvec(self, freq, x, y=None, stream=None):
        """y = A(k) x for a CUDA tensor x [nrhs, nunk] (complex64 -> FP32, complex128 -> FP64)."""
        import torch
        if not x.is_cuda or not x.is_contiguous():
            raise AimxError(-1, "x must be a contiguous CUDA tensor")
        if x.dim() == 1:
            x = x.unsqueeze(0)
        prec = {torch.complex64: F32, torch.complex128: F64}.get(x.dtype)
        if prec is None or x.shape[-1] != self.nunk:
            raise AimxError(-1, "x must be complex64/complex128 with last dim = %d" % self.nunk)
        if y is None:
            y = torch.empty_like(x)
        self._check(self._lib.aimx_matvec(self._ctx, float(freq), x.shape[0], ctypes.c_void_p(x.data_ptr()),
                                          ctypes.c_void_p(y.data_ptr()), prec, _stream_handle(stream)))
        return y

    def matvec_host(self, freq, x, stream=None):
        """Same product on host numpy arrays (copies in and out inside the library)."""
        x = np.ascontiguousarray(np.atleast_2d(x))
        prec = F64 if x.dtype == np.complex128 else F32
        x = x.astype(np.complex128 if prec == F64 else np.complex64, copy=False)
        y = np.empty_like(x)
        self._check(self._lib.aimx_matvec_host(self._ctx, float(freq), x.shape[0], _ptr(x), _ptr(y), prec,
                                               _stream_handle(stream)))
        return y

    def matvec_host_ptr(self, freq, nrhs, x_ptr, y_ptr, precision=F32, stream=None):
        """aimx_matvec_host on raw host addresses (e.g. pinned torch tensors)."""
        self._check(self._lib.aimx_matvec_host(self._ctx, float(freq), int(nrhs), ctypes.c_void_p(x_ptr),
                                               ctypes.c_void_p(y_ptr), int(precision), _stream_handle(stream)))

    # ---------------------------------------------------------------- solve / sweep / excitation
    def rhs_planewave(self, freq, dirs, pols, stream=None):
        """Plane-wave right-hand sides as a CUDA complex128 tensor [nwave, nunk]."""
        import torch
        d = np.ascontiguousarray(np.atleast_2d(dirs), dtype=np.float64)
        p = np.ascontiguousarray(np.atleast_2d(pols), dtype=np.float64)
        b = torch.empty((len(d), self.nunk), dtype=torch.complex128, device="cuda")
        self._check(self._lib.aimx_rhs_planewave(self._ctx, float(freq), len(d), _ptr(d), _ptr(p),
                                                 ctypes.c_void_p(b.data_ptr()), _stream_handle(stream)))
        return b

    def solve(self, freq, b, x0=None, tol=1e-6, restart=50, max_iter=1000, inner_precision=F32,
              precond=PRECOND_DIAG, max_refine=0, learned_trial=0, stream=None):
        """Solve A x = b for CUDA complex128 b [nrhs, nunk]; returns (x, stats, status)."""
        import torch
        if b.dim() == 1:
            b = b.unsqueeze(0)
        b = b.contiguous()
        x = x0.clone().contiguous() if x0 is not None else torch.empty_like(b)
        st = (_SolveStats * b.shape[0])()
        o = _opts(tol, restart, max_iter, inner_precision, precond, 1 if x0 is not None else 0, max_refine,
                  learned_trial)
        rc = self._check(self._lib.aimx_solve(self._ctx, float(freq), b.shape[0], ctypes.c_void_p(b.data_ptr()),
                                              ctypes.c_void_p(x.data_ptr()), ctypes.byref(o), st,
                                              _stream_handle(stream)))
        return x, _stats_list(st), rc

    def precond_apply(self, freq, v, precond=PRECOND_BLOCK, stream=None):
        """z = M v for CUDA complex128 v [nrhs, nunk]."""
        import torch
        if v.dim() == 1:
            v = v.unsqueeze(0)
        v = v.contiguous()
        z = torch.empty_like(v)
        self._check(self._lib.aimx_precond_apply(self._ctx, float(freq), int(precond), v.shape[0],
                                                 ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(z.data_ptr()),
                                                 _stream_handle(stream)))
        return z

    def farfield(self, freq, x, dirs, stream=None):
        """Far-zone E (r e^{jkr} E) [nrhs, ndir, 3] for CUDA complex128 currents x [nrhs, nunk]."""
        if x.dim() == 1:
            x = x.unsqueeze(0)
        x = x.contiguous()
        d = np.ascontiguousarray(np.atleast_2d(dirs), dtype=np.float64)
        E = np.zeros((x.shape[0], len(d), 3), dtype=np.complex128)
        self._check(self._lib.aimx_farfield(self._ctx, float(freq), x.shape[0], ctypes.c_void_p(x.data_ptr()), len(d),
                                            _ptr(d), _ptr(E), _stream_handle(stream)))
        return E

    def sweep(self, freqs, dirs, pols, tol=1e-6, restart=50, max_iter=1000, inner_precision=F32,
              precond=PRECOND_DIAG, warm_start=True, stream=None):
        """Solve the plane-wave problems at every frequency; returns (X [nf, nwave, nunk], stats, status)."""
        import torch
        f = np.ascontiguousarray(freqs, dtype=np.float64)
        d = np.ascontiguousarray(np.atleast_2d(dirs), dtype=np.float64)
        p = np.ascontiguousarray(np.atleast_2d(pols), dtype=np.float64)
        X = torch.empty((len(f), len(d), self.nunk), dtype=torch.complex128, device="cuda")
        st = (_SolveStats * (len(f) * len(d)))()
        o = _opts(tol, restart, max_iter, inner_precision, precond)
        rc = self._check(self._lib.aimx_sweep(self._ctx, len(f), _ptr(f), len(d), _ptr(d), _ptr(p),
                                              ctypes.c_void_p(X.data_ptr()), ctypes.byref(o), 1 if warm_start else 0,
                                              st, _stream_handle(stream)))
        return X, _stats_list(st), rc

    def sweep_batched(self, freqs, B, tol=1e-6, restart=50, max_iter=1000, inner_precision=F32,
                      precond=PRECOND_DIAG, max_batch=0, warm_start=False, x0=None, stream=None):
        """Solve A(k_f) x = b for every frequency f and RHS at once (aimx_sweep_batched).

        B: CUDA complex128 [nf, nrhs, nunk].  Returns (X, stats [nf][nrhs], rc, counters) with
        counters = (cycles, graphs captured, batched products)."""
        import torch
        freqs = np.ascontiguousarray(freqs, dtype=np.float64)
        B = B.contiguous()
        nf, nrhs = int(B.shape[0]), int(B.shape[1])
        X = x0.clone().contiguous() if x0 is not None else torch.empty_like(B)
        st = (_SolveStats * (nf * nrhs))()
        cnt = np.zeros(3, dtype=np.int64)
        o = _opts(tol, restart, max_iter, inner_precision, precond, 1 if x0 is not None else 0, 0, 0)
        rc = self._check(self._lib.aimx_sweep_batched(self._ctx, nf, _ptr(freqs), nrhs, ctypes.c_void_p(B.data_ptr()),
                                                      ctypes.c_void_p(X.data_ptr()), ctypes.byref(o), int(max_batch),
                                                      1 if warm_start else 0, st, _ptr(cnt), _stream_handle(stream)))
        stats = _stats_list(st)
        return X, [stats[f * nrhs:(f + 1) * nrhs] for f in range(nf)], rc, tuple(int(v) for v in cnt)

    def set_path(self, path):
        """0 = automatic (plane-fused FP32 path when supported), 1 = generic path, 2 = generic with cuFFT."""
        self._check(self._lib.aimx_set_path(self._ctx, int(path)))

    def matvec_path(self, precision=F32):
        return self._check(self._lib.aimx_matvec_path(self._ctx, int(precision)))

    def set_linear_term(self, enable=True):
        """Linear-term modification of Sec. III-A-3 on overlapping pairs (built on the first enable)."""
        self._check(self._lib.aimx_set_linear_term(self._ctx, 1 if enable else 0))

    def set_plane_cap(self, cap):
        """Test hook (aimx_set_plane_cap): bases per grid plane kept in shared memory by the
        register inverse-xy kernel; <= 0 restores the default."""
        self._check(self._lib.aimx_set_plane_cap(self._ctx, int(cap)))

    def set_schedule(self, variant, pass_=0):
        """Product schedule: variant 0 fused/register, 1 fused/shared memory, 2 generic; RHS per pass (0 = all)."""
        sch = Schedule(int(variant), int(pass_), 0.0)
        self._check(self._lib.aimx_set_schedule(self._ctx, ctypes.byref(sch)))

    def get_schedule(self):
        sch = Schedule()
        self._check(self._lib.aimx_get_schedule(self._ctx, ctypes.byref(sch)))
        return sch.as_dict()

    def autotune(self, freq, nrhs, cache_path=None, stream=None):
        """Time the candidate schedules of an FP32 product of nrhs RHS and keep the fastest.

        Returns {"best": schedule, "tried": [schedules with ms]} ("tried" is empty on a cache hit)."""
        best = Schedule()
        tried = (Schedule * 32)()
        n = ctypes.c_int(0)
        path = None if cache_path is None else str(cache_path).encode()
        self._check(self._lib.aimx_autotune(self._ctx, float(freq), int(nrhs), path, ctypes.byref(best), tried, 32,
                                            ctypes.byref(n), _stream_handle(stream)))
        return {"best": best.as_dict(), "tried": [tried[i].as_dict() for i in range(n.value)]}

    def set_conventional_aim(self, enable=True):
        """Conventional-AIM comparison mode (Sec. II-B): near entries refilled at every new frequency."""
        self._check(self._lib.aimx_set_conventional_aim(self._ctx, 1 if enable else 0))

    def set_charge_form(self, enable=True):
        """Charge-form scalar potential L^Phi = D^T Pt D (EFIE); builds the triangle data on the first enable."""
        self._check(self._lib.aimx_set_charge_form(self._ctx, 1 if enable else 0))

    def export_charge(self):
        """Charge-form setup in caller triangle numbering: anchors, near pairs, N_Pt values, pulse weights."""
        n = ctypes.c_int64(0)
        ntc = ctypes.c_int32(0)
        self._check(self._lib.aimx_export_charge(self._ctx, ctypes.byref(ntc), ctypes.byref(n), None, None, None,
                                                 None, None))
        nt = int(ntc.value)
        U = (self.info["order"] + 1) ** 3
        tanc = np.zeros((nt, 3), dtype=np.int32)
        rows = np.zeros(n.value, dtype=np.int32)
        cols = np.zeros(n.value, dtype=np.int32)
        npt = np.zeros(n.value)
        lp = np.zeros((nt, U))
        self._check(self._lib.aimx_export_charge(self._ctx, None, None, _ptr(tanc), _ptr(rows), _ptr(cols),
                                                 _ptr(npt), _ptr(lp)))
        return dict(tanc=tanc, rows=rows, cols=cols, npt=npt, lp=lp)

    def export_aim_near(self, freq):
        """Conventional-AIM near entries at freq, complex [nnz], in export_setup's near order."""
        z = np.zeros((self.info["near_nnz"], 2))
        self._check(self._lib.aimx_export_aim_near(self._ctx, float(freq), _ptr(z)))
        return z[:, 0] + 1j * z[:, 1]

    def export_linear_term(self):
        """{row_ptr, cols, NA, NP}: N^A_lin, N^Phi_lin on the overlapping pairs, caller numbering."""
        nl = np.zeros(1, dtype=np.int64)
        self._check(self._lib.aimx_export_linear_term(self._ctx, _ptr(nl), None, None, None, None))
        n = int(nl[0])
        rp = np.zeros(self.N + 1, dtype=np.int64)
        cols = np.zeros(n, dtype=np.int32)
        na, nphi = np.zeros(n), np.zeros(n)
        self._check(self._lib.aimx_export_linear_term(self._ctx, None, _ptr(rp), _ptr(cols), _ptr(na), _ptr(nphi)))
        return dict(row_ptr=rp, cols=cols, NA=na, NP=nphi)

    # ---------------------------------------------------------------- profiling
    def profile(self, enable=True):
        self._check(self._lib.aimx_profile(self._ctx, 1 if enable else 0))

    def profile_read(self):
        """{stage name: (milliseconds, launches)} since the last read (synchronises)."""
        ms = np.zeros(32)
        cnt = np.zeros(32, dtype=np.int64)
        n = self._check(self._lib.aimx_profile_read(self._ctx, _ptr(ms), _ptr(cnt), 32))
        out = {}
        for k in range(n):
            if cnt[k]:
                out[self._lib.aimx_profile_stage_name(k).decode()] = (float(ms[k]), int(cnt[k]))
        return out

    # ---------------------------------------------------------------- export
    def export_setup(self):
        N, U = self.N, (self.info["order"] + 1) ** 3
        nnz = self.info["near_nnz"]
        anc = np.zeros((N, 3), dtype=np.int32)
        w = np.zeros((N, U, 4))
        rp = np.zeros(N + 1, dtype=np.int64)
        cols = np.zeros(nnz, dtype=np.int32)
        na, nphi, nk = np.zeros(nnz), np.zeros(nnz), np.zeros(nnz)
        self._check(self._lib.aimx_export_setup(self._ctx, _ptr(anc), _ptr(w), _ptr(rp), _ptr(cols), _ptr(na),
                                                _ptr(nphi), _ptr(nk)))
        return dict(anchors=anc, weights=w, row_ptr=rp, cols=cols, NA=na, NP=nphi, NK=nk)

    # ---------------------------------------------------------------- delta-gap ports
    @staticmethod
    def _ports(ports):
        return (Port * len(ports))(*ports)

    def port_vectors(self, ports):
        """(c [nport, N] float64 port vectors, gap-edge counts [nport])."""
        c = np.zeros((len(ports), self.N))
        ne = np.zeros(len(ports), dtype=np.int32)
        self._check(self._lib.aimx_port_vectors(self._ctx, len(ports), self._ports(ports), _ptr(c), _ptr(ne)))
        return c, ne

    def rhs_ports(self, ports, stream=None):
        """Unit-voltage excitations as a CUDA complex128 tensor [nport, nunk]."""
        import torch
        b = torch.empty((len(ports), self.nunk), dtype=torch.complex128, device="cuda")
        self._check(self._lib.aimx_rhs_ports(self._ctx, len(ports), self._ports(ports),
                                             ctypes.c_void_p(b.data_ptr()), _stream_handle(stream)))
        return b

    def port_currents(self, ports, x, stream=None):
        """Port currents [nrhs, nport] (complex128) of CUDA complex128 coefficients x [nrhs, nunk]."""
        if x.dim() == 1:
            x = x.unsqueeze(0)
        x = x.contiguous()
        out = np.zeros((x.shape[0], len(ports)), dtype=np.complex128)
        self._check(self._lib.aimx_port_currents(self._ctx, len(ports), self._ports(ports), x.shape[0],
                                                 ctypes.c_void_p(x.data_ptr()), _ptr(out), _stream_handle(stream)))
        return out

    def sweep_ports(self, freqs, ports, tol=1e-6, restart=50, max_iter=1000, inner_precision=F32,
                    precond=PRECOND_DIAG, stream=None):
        """Y-parameters [nf, nport, nport] over a frequency sweep; returns (Y, stats, status)."""
        f = np.ascontiguousarray(freqs, dtype=np.float64)
        P = len(ports)
        Y = np.zeros((len(f), P, P), dtype=np.complex128)
        st = (_SolveStats * (len(f) * P))()
        o = _opts(tol, restart, max_iter, inner_precision, precond)
        rc = self._check(self._lib.aimx_sweep_ports(self._ctx, len(f), _ptr(f), P, self._ports(ports), _ptr(Y),
                                                    ctypes.byref(o), st, _stream_handle(stream)))
        return Y, _stats_list(st), rc

    # ---------------------------------------------------------------- learned preconditioner
    def gnn_attach(self, net):
        """Copy ``net``'s parameters into this context for PRECOND_LEARNED (None detaches)."""
        self._check(self._lib.aimx_gnn_attach(self._ctx, net._net if net is not None else None))

    def gnn_features(self, freq):
        """(node [N,8] by basis, edge [nnz,16], basis [nnz,8], rows, cols) of the network inputs at freq."""
        nnz = self.info["near_nnz"]
        node = np.zeros((self.N, 8), dtype=np.float32)
        edge = np.zeros((nnz, 16), dtype=np.float32)
        basis = np.zeros((nnz, 8), dtype=np.float32)
        rows = np.zeros(nnz, dtype=np.int32)
        cols = np.zeros(nnz, dtype=np.int32)
        self._check(self._lib.aimx_gnn_features(self._ctx, float(freq), _ptr(node), _ptr(edge), _ptr(basis),
                                                _ptr(rows), _ptr(cols)))
        return node, edge, basis, rows, cols

    def gnn_outputs(self, net, freq):
        """Network outputs (o [nnz,K] in gnn_features' edge order, g [N,K]) with ``net``'s parameters."""
        K = net.K
        o = np.zeros((self.info["near_nnz"], K), dtype=np.float32)
        g = np.zeros((self.N, K), dtype=np.float32)
        self._check(self._lib.aimx_gnn_outputs(self._ctx, net._net, float(freq), _ptr(o), _ptr(g)))
        return o, g


class Gnn:
    """The learned near-field preconditioner network (see include/aimx.h)."""

    def __init__(self, formulation=EFIE, layers=4):
        self._lib = load()
        h = ctypes.c_void_p()
        rc = self._lib.aimx_gnn_create(int(formulation), int(layers), ctypes.byref(h))
        if rc != 0:
            raise AimxError(rc, "aimx_gnn_create")
        self._net = h
        self.K = 2 if formulation == EFIE else 8
        self.layers = layers
        self.n_params = int(self._lib.aimx_gnn_num_params(h))

    def close(self):
        if getattr(self, "_net", None):
            self._lib.aimx_gnn_destroy(self._net)
            self._net = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, ctx=None):
        if rc != 0:
            msg = self._lib.aimx_last_error(ctx._ctx).decode() if ctx is not None else ""
            raise AimxError(rc, msg)

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        self._check(self._lib.aimx_gnn_set_params(self._net, _ptr(p), p.size))

    def params(self):
        p = np.zeros(self.n_params, dtype=np.float32)
        self._check(self._lib.aimx_gnn_get_params(self._net, _ptr(p), p.size))
        return p

    def loss_grad(self, ctx, freq, Z, Y, want_grad=True, stream=None):
        """Probe loss (and gradient) for device complex64 tensors Z, Y [P, n_unknowns]."""
        loss = ctypes.c_double()
        g = np.zeros(self.n_params, dtype=np.float32) if want_grad else None
        self._check(self._lib.aimx_gnn_loss_grad(self._net, ctx._ctx, float(freq), Z.shape[0],
                                                 ctypes.c_void_p(Z.data_ptr()), ctypes.c_void_p(Y.data_ptr()),
                                                 ctypes.byref(loss), _ptr(g), _stream_handle(stream)), ctx)
        return loss.value, g

    def train_step(self, ctx, freq, Z, Y, lr=1e-3, clip=0.0, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        loss = ctypes.c_double()
        o = _AdamOpts(float(lr), float(beta1), float(beta2), float(eps), float(clip))
        self._check(self._lib.aimx_gnn_train_step(self._net, ctx._ctx, float(freq), Z.shape[0],
                                                  ctypes.c_void_p(Z.data_ptr()), ctypes.c_void_p(Y.data_ptr()),
                                                  ctypes.byref(o), ctypes.byref(loss), _stream_handle(stream)), ctx)
        return loss.value

    def init_params(self, seed=0):
        """He-initialised hidden layers, zero E, f, G, g (C = 0: the diagonal preconditioner)."""
        rng = np.random.default_rng(seed)
        p = np.zeros(self.n_params, dtype=np.float32)
        off = 0

        def take(rows, cols, he):
            nonlocal off
            n = rows * cols
            if he:
                p[off:off + n] = (rng.standard_normal(n) * np.sqrt(2.0 / cols)).astype(np.float32)
            off += n

        take(64, 8, True)            # A0
        take(64, 1, False)           # a0
        for _ in range(self.layers):
            take(64, 64, True)       # B
            take(64, 16, True)       # C
            take(64, 1, False)       # c
            take(64, 64, True)       # D
            take(64, 1, False)       # d
        take(64, 64, True)           # Ua
        take(64, 64, True)           # Ub
        take(64, 16, True)           # Uc
        take(64, 1, False)           # u
        assert off + self.K * (8 * 64 + 8 + 64 + 1) == self.n_params
        self.set_params(p)
        return p

    def fit(self, samples, steps, nprobe=8, lr=1e-3, clip=1.0, seed=0, log=None, cosine=True):
        """Adam on the probe loss, cycling over ``samples`` = [(Context, freq), ...].

        Each step draws nprobe seeded complex Gaussian probes z on the device,
        forms y = A z with the context's FP32 product, and takes one step; with
        ``cosine`` the step size decays as lr (0.05 + 0.95 (1 + cos(pi t / steps)) / 2)."""
        import math
        import torch
        gen = torch.Generator(device="cuda")
        gen.manual_seed(int(seed))
        losses = []
        steps = int(steps)
        for it in range(steps):
            ctx, freq = samples[it % len(samples)]
            n = ctx.nunk
            Z = torch.randn(nprobe, n, 2, device="cuda", generator=gen, dtype=torch.float32)
            Z = torch.view_as_complex(Z).contiguous()
            Y = ctx.matvec(freq, Z)
            lr_t = lr * (0.05 + 0.475 * (1.0 + math.cos(math.pi * it / steps))) if cosine else lr
            losses.append(self.train_step(ctx, freq, Z, Y, lr=lr_t, clip=clip))
            if log is not None:
                log(it, losses[-1])
        return losses


class Batch:
    """FP32 products of several contexts as one captured CUDA graph (aimx_batch_*).

    The contexts are borrowed: keep them open while the batch is used."""

    def __init__(self, contexts, nstreams=0):
        self._lib = load()
        self.contexts = list(contexts)
        arr = (ctypes.c_void_p * len(self.contexts))(*[c._ctx for c in self.contexts])
        h = ctypes.c_void_p()
        rc = self._lib.aimx_batch_create(len(self.contexts), arr, int(nstreams), ctypes.byref(h))
        if rc != 0:
            raise AimxError(rc, "aimx_batch_create")
        self._b = h

    def close(self):
        if getattr(self, "_b", None):
            self._lib.aimx_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def matvec(self, freqs, xs, ys, stream=None):
        """ys[i] = A_i(freqs[i]) xs[i] for complex64 CUDA tensors [nrhs_i, n_unknowns_i]."""
        n = len(self.contexts)
        f = (ctypes.c_double * n)(*[float(v) for v in freqs])
        nr = (ctypes.c_int * n)(*[int(x.shape[0]) for x in xs])
        xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
        yp = (ctypes.c_void_p * n)(*[y.data_ptr() for y in ys])
        rc = self._lib.aimx_batch_matvec(self._b, f, nr, xp, yp, _stream_handle(stream))
        if rc != 0:
            raise AimxError(rc, (self._lib.aimx_batch_last_error(self._b) or b"").decode())
        return ys

    def solve(self, freqs, bs, tol=1e-6, restart=50, max_iter=1000, inner_precision=F32, precond=PRECOND_DIAG,
              stream=None):
        """Solve every member (aimx_batch_solve): bs[i] complex128 CUDA [nrhs_i, n_unknowns_i].
        Returns (xs, stats per member, status)."""
        import torch
        n = len(self.contexts)
        bs = [b.contiguous() for b in bs]
        xs = [torch.empty_like(b) for b in bs]
        f = (ctypes.c_double * n)(*[float(v) for v in freqs])
        nr = (ctypes.c_int * n)(*[int(b.shape[0]) for b in bs])
        bp = (ctypes.c_void_p * n)(*[b.data_ptr() for b in bs])
        xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
        st = [(_SolveStats * int(b.shape[0]))() for b in bs]
        sp = (ctypes.c_void_p * n)(*[ctypes.addressof(a) for a in st])
        o = _opts(tol, restart, max_iter, inner_precision, precond)
        rc = self._lib.aimx_batch_solve(self._b, f, nr, bp, xp, ctypes.byref(o), sp, _stream_handle(stream))
        if rc < 0:
            raise AimxError(rc, (self._lib.aimx_batch_last_error(self._b) or b"").decode())
        return xs, [_stats_list(a) for a in st], rc

    @property
    def graph_nodes(self):
        return int(self._lib.aimx_batch_graph_nodes(self._b))
