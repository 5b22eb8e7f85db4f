"""Thin ctypes binding of the C ABI in include/dwf.h (argument marshalling only).

Every computation runs in the CUDA library ``_lib/libdwf.so``; this module
only turns torch tensors into device pointers and the current CUDA stream
into a ``cudaStream_t``.  If the library is missing the calls fail loudly:
there is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "_lib", "libdwf.so")

STANDARD, NEFF = 0, 1
F64, F32, F16 = 0, 1, 2
OP_FULL5D, OP_EO_PREC = 0, 1
PREC = {"f64": F64, "f32": F32, "f16": F16, F64: F64, F32: F32, F16: F16}
FORM = {"standard": STANDARD, "neff": NEFF, STANDARD: STANDARD, NEFF: NEFF}
OP_EO5_PREC = 2
OPS = {"full": OP_FULL5D, "full5d": OP_FULL5D, "eo": OP_EO_PREC, "eo_prec": OP_EO_PREC, "eo5": OP_EO5_PREC,
       OP_FULL5D: OP_FULL5D, OP_EO_PREC: OP_EO_PREC, OP_EO5_PREC: OP_EO5_PREC}

STATUS = {0: "DWF_OK", 1: "DWF_EINVAL", 2: "DWF_ENOMEM", 3: "DWF_ECUDA", 4: "DWF_ENOTCONV",
          5: "DWF_ENONFINITE", 6: "DWF_ETIMEOUT", 7: "DWF_EBREAKDOWN", 8: "DWF_ENOGAUGE"}

EXPORTED = ["dwf_create", "dwf_create_s", "dwf_destroy", "dwf_strerror", "dwf_last_error", "dwf_set_gauge",
            "dwf_apply", "dwf_apply_dag", "dwf_solve_eo5", "dwf_wait_probe", "dwf_source_5d", "dwf_project_4d",
            "dwf_solve_params_default", "dwf_solve", "dwf_propagator_host", "dwf_solve_batch",
            "dwf_fifth_matrix", "dwf_fifth_matrix_host", "dwf_device_bytes", "dwf_time_hop", "dwf_time_iteration", "dwf_spectrum_bounds", "dwf_launch_count",
            "dwf_set_hop_config", "dwf_get_hop_config", "dwf_set_sweep", "dwf_get_sweep",
            "dwf_create_slab", "dwf_slab_apply_eo", "dwf_slab_faces", "dwf_slab_exchange_ring",
            "dwf_slab_cgnr_ring", "dwf_autotune", "dwf_device_status",
            "dwf_set_mix_mode", "dwf_get_mix_mode", "dwf_apply_eo_noalloc",
            "dwf_train_params_default", "dwf_precond_init", "dwf_precond_set_weights", "dwf_precond_get_weights",
            "dwf_precond_apply", "dwf_precond_loss_grad", "dwf_precond_train", "dwf_precond_adam_step",
            "dwf_precond_save", "dwf_precond_load", "dwf_alu_peaks", "dwf_precond_fcg", "dwf_time_mix"]


class SolveParams(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("inner_prec", ctypes.c_int),
                ("delta", ctypes.c_double), ("check_every", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("precond", ctypes.c_int), ("use_initial_guess", ctypes.c_int), ("verbose", ctypes.c_int),
                ("batch_wave", ctypes.c_int), ("eo_form", ctypes.c_int)]


class SolveStats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iterations", ctypes.c_int), ("reliable_updates", ctypes.c_int),
                ("d_applications", ctypes.c_int), ("true_residual", ctypes.c_double),
                ("eo_residual", ctypes.c_double), ("seconds", ctypes.c_double),
                ("history", ctypes.c_double * 64), ("n_history", ctypes.c_int),
                ("kernel_launches", ctypes.c_longlong), ("waves", ctypes.c_int),
                ("precond_applications", ctypes.c_int), ("fallbacks", ctypes.c_int)]

    def as_dict(self):
        return dict(status=STATUS.get(self.status, self.status), iterations=self.iterations,
                    reliable_updates=self.reliable_updates, d_applications=self.d_applications,
                    true_residual=self.true_residual, eo_residual=self.eo_residual, seconds=self.seconds,
                    history=list(self.history[:self.n_history]), kernel_launches=self.kernel_launches,
                    waves=self.waves, precond_applications=self.precond_applications,
                    fallbacks=self.fallbacks)


class TrainParams(ctypes.Structure):
    _fields_ = [("layers", ctypes.c_int), ("epochs", ctypes.c_int), ("batch", ctypes.c_int),
                ("lr", ctypes.c_double), ("solve_inner_prec", ctypes.c_int), ("solve_tol", ctypes.c_double),
                ("seed", ctypes.c_ulonglong), ("noise", ctypes.c_double), ("verbose", ctypes.c_int),
                ("random_pairs", ctypes.c_int)]


class TrainStats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("pairs", ctypes.c_int), ("epochs", ctypes.c_int),
                ("steps", ctypes.c_int), ("loss_first", ctypes.c_double), ("loss_last", ctypes.c_double),
                ("loss_history", ctypes.c_double * 64), ("n_history", ctypes.c_int),
                ("seconds", ctypes.c_double), ("solve_seconds", ctypes.c_double)]

    def as_dict(self):
        return dict(status=STATUS.get(self.status, self.status), pairs=self.pairs, epochs=self.epochs,
                    steps=self.steps, loss_first=self.loss_first, loss_last=self.loss_last,
                    loss_history=list(self.loss_history[:self.n_history]), seconds=self.seconds,
                    solve_seconds=self.solve_seconds)


class DwfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


_lib = None


def lib():
    """Load the CUDA library (built by paper_2602_14454_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError("CUDA library %s is missing; build it with "
                           "paper_2602_14454_gb300.build.build()" % _LIB_PATH)
    L = ctypes.CDLL(_LIB_PATH)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    ip = ctypes.POINTER(ctypes.c_int)
    L.dwf_create.argtypes = [ip, i, d, d, d, d, i, d, ip, ctypes.POINTER(vp)]
    L.dwf_create_s.argtypes = [ip, i, d, d, ctypes.POINTER(d), ctypes.POINTER(d), ip, ctypes.POINTER(vp)]
    L.dwf_destroy.argtypes = [vp]
    L.dwf_strerror.restype = ctypes.c_char_p
    L.dwf_strerror.argtypes = [i]
    L.dwf_last_error.restype = ctypes.c_char_p
    L.dwf_last_error.argtypes = []
    L.dwf_set_gauge.argtypes = [vp, vp, vp]
    L.dwf_apply.argtypes = [vp, i, i, vp, vp, vp]
    L.dwf_create_slab.argtypes = [ctypes.POINTER(ctypes.c_int), i, i, i, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, i, ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                                  ctypes.POINTER(vp)]
    L.dwf_slab_apply_eo.argtypes = [vp, i, i, i, vp, vp, vp]
    L.dwf_slab_faces.argtypes = [vp, i, i, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                 ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_size_t)]
    L.dwf_slab_exchange_ring.argtypes = [ctypes.POINTER(vp), i, i, i, vp]
    L.dwf_slab_cgnr_ring.argtypes = [ctypes.POINTER(vp), i, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.c_double,
                                     i, ctypes.POINTER(i), ctypes.POINTER(ctypes.c_double), vp]
    L.dwf_apply_dag.argtypes = [vp, i, i, vp, vp, vp]
    L.dwf_solve_eo5.argtypes = [vp, vp, vp, d, i, ip, ctypes.POINTER(d), vp]
    L.dwf_wait_probe.argtypes = [vp, ctypes.c_longlong, vp]
    L.dwf_source_5d.argtypes = [vp, vp, vp, vp]
    L.dwf_project_4d.argtypes = [vp, vp, vp, vp]
    L.dwf_solve_params_default.argtypes = [ctypes.POINTER(SolveParams)]
    L.dwf_solve_params_default.restype = None
    L.dwf_solve.argtypes = [vp, vp, vp, ctypes.POINTER(SolveParams), ctypes.POINTER(SolveStats), vp]
    L.dwf_propagator_host.argtypes = [vp, vp, vp, ctypes.POINTER(SolveParams), ctypes.POINTER(SolveStats), vp]
    L.dwf_solve_batch.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), i,
                                  ctypes.POINTER(SolveParams), ctypes.POINTER(SolveStats), vp]
    L.dwf_fifth_matrix.argtypes = [vp, i, i, ctypes.POINTER(ctypes.c_double)]
    L.dwf_fifth_matrix_host.argtypes = [i, d, d, ctypes.POINTER(d), ctypes.POINTER(d), i, d, i, i,
                                        ctypes.POINTER(ctypes.c_double), ip]
    L.dwf_device_bytes.argtypes = [vp]
    L.dwf_device_bytes.restype = ctypes.c_size_t
    L.dwf_time_hop.argtypes = [vp, i, i, i, ctypes.POINTER(d), ctypes.POINTER(d), vp]
    L.dwf_time_iteration.argtypes = [vp, i, i, i, ctypes.POINTER(d), ctypes.POINTER(d), vp]
    L.dwf_time_mix.argtypes = [vp, i, i, i, i, ctypes.POINTER(d), ctypes.POINTER(d), vp]
    L.dwf_spectrum_bounds.argtypes = [vp, i, i, d, ctypes.c_ulonglong, ctypes.POINTER(d), ctypes.POINTER(d), ip, vp]
    L.dwf_set_hop_config.argtypes = [vp, i, i, i, i]
    L.dwf_get_hop_config.argtypes = [vp, i, ip, ip, ip]
    L.dwf_set_sweep.argtypes = [vp, i, i]
    L.dwf_get_sweep.argtypes = [vp, i, ip]
    L.dwf_device_status.argtypes = [vp, vp]
    L.dwf_set_mix_mode.argtypes = [vp, i, i]
    L.dwf_get_mix_mode.argtypes = [vp, i, ip]
    L.dwf_apply_eo_noalloc.argtypes = [vp, i, i, vp, vp, vp]
    L.dwf_autotune.argtypes = [vp, i, ctypes.c_char_p, vp]
    L.dwf_launch_count.argtypes = [vp]
    L.dwf_launch_count.restype = ctypes.c_longlong
    L.dwf_alu_peaks.argtypes = [ctypes.POINTER(d), vp]
    dp = ctypes.POINTER(ctypes.c_double)
    L.dwf_train_params_default.argtypes = [ctypes.POINTER(TrainParams)]
    L.dwf_train_params_default.restype = None
    L.dwf_precond_init.argtypes = [vp, i, ctypes.c_ulonglong, d]
    L.dwf_precond_set_weights.argtypes = [vp, i, dp]
    L.dwf_precond_get_weights.argtypes = [vp, i, i, dp]
    L.dwf_precond_apply.argtypes = [vp, i, vp, vp, vp]
    L.dwf_precond_loss_grad.argtypes = [vp, i, ctypes.POINTER(vp), ctypes.POINTER(vp), dp, dp, vp]
    L.dwf_precond_adam_step.argtypes = [vp, i, dp, d, vp]
    L.dwf_precond_fcg.argtypes = [vp, vp, vp, d, i, i, dp, ip, vp]
    L.dwf_precond_save.argtypes = [vp, ctypes.c_char_p]
    L.dwf_precond_load.argtypes = [vp, ctypes.c_char_p]
    L.dwf_precond_train.argtypes = [vp, i, ctypes.POINTER(vp), ctypes.POINTER(TrainParams),
                                    ctypes.POINTER(TrainStats), vp]
    _lib = L
    return L


def check(rc):
    if rc != 0:
        raise DwfError(rc, lib().dwf_last_error().decode())
    return rc


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t, dtype=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if t.dtype != torch.complex128:
        raise TypeError("fields and links are complex128")
    return ctypes.c_void_p(t.data_ptr())


def default_params(**kw) -> SolveParams:
    p = SolveParams()
    lib().dwf_solve_params_default(ctypes.byref(p))
    for k, v in kw.items():
        if k == "inner_prec":
            v = PREC[v]
        setattr(p, k, v)
    return p


def _coeffs(v, Ls):
    """(C array of Ls doubles, scalar or None): a number gives Ls copies."""
    a = np.broadcast_to(np.asarray(v, dtype=np.float64), (Ls,))
    return (ctypes.c_double * Ls)(*a), (float(a[0]) if np.ndim(v) == 0 else None)


class Operator:
    """One lattice, one 5D operator (standard or Neff form), one gauge field.
    b and c are numbers, or (standard form) sequences of Ls coefficients b_s, c_s."""

    def __init__(self, dims, Ls, M0, mf, b, c, form="standard", alpha=1.0, bc=None):
        self.dims = tuple(int(x) for x in dims)
        self.Ls = int(Ls)
        h = ctypes.c_void_p()
        d = (ctypes.c_int * 4)(*self.dims)
        bcp = (ctypes.c_int * 4)(*bc) if bc is not None else None
        if np.ndim(b) == 0 and np.ndim(c) == 0:
            check(lib().dwf_create(d, self.Ls, float(M0), float(mf), float(b), float(c), FORM[form],
                                   float(alpha), bcp, ctypes.byref(h)))
            self.b, self.c = float(b), float(c)
        else:
            if FORM[form] != STANDARD:
                raise ValueError("s-dependent coefficients need the standard form")
            ba, _ = _coeffs(b, self.Ls)
            ca, _ = _coeffs(c, self.Ls)
            check(lib().dwf_create_s(d, self.Ls, float(M0), float(mf), ba, ca, bcp, ctypes.byref(h)))
            self.b, self.c = np.array(ba), np.array(ca)
        self._h = h
        self.M0, self.mf = float(M0), float(mf)
        self.form, self.alpha = form, float(alpha)
        Lx, Ly, Lz, Lt = self.dims
        self.site_shape = (Lt, Lz, Ly, Lx)
        self.V = Lx * Ly * Lz * Lt

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            lib().dwf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_gauge(self, U):
        self._U = U
        check(lib().dwf_set_gauge(self._h, _ptr(U), _stream()))

    def _new(self, shape):
        import torch
        return torch.empty(shape, dtype=torch.complex128, device="cuda")

    def shape5(self):
        return (self.Ls,) + self.site_shape + (4, 3)

    def shape_eo(self):
        return (self.Ls, self.V // 2, 4, 3)

    def apply(self, x, op="full", prec="f64", dag=False, out=None):
        o = OPS[op]
        if out is None:
            out = self._new(x.shape)
        fn = lib().dwf_apply_dag if dag else lib().dwf_apply
        check(fn(self._h, o, PREC[prec], _ptr(x), _ptr(out), _stream()))
        return out

    def wait_probe(self, limit_ns):
        """A bounded device wait that runs out (failure-detection probe, dwf_wait_probe)."""
        check(lib().dwf_wait_probe(self._h, int(limit_ns), _stream()))

    def solve_eo5(self, b5, tol=1e-10, max_iter=20000):
        """FP64 CGNR through the 5D even-odd split (dwf_solve_eo5): x5 and the residual history."""
        x5 = self._new(self.shape5())
        its = ctypes.c_int()
        hist = (ctypes.c_double * (max_iter + 1))()
        check(lib().dwf_solve_eo5(self._h, _ptr(b5), _ptr(x5), float(tol), int(max_iter), ctypes.byref(its), hist,
                                  _stream()))
        return x5, list(hist[:its.value + 1])

    def source_5d(self, b4, out=None):
        if out is None:
            out = self._new(self.shape5())
        check(lib().dwf_source_5d(self._h, _ptr(b4), _ptr(out), _stream()))
        return out

    def project_4d(self, x5, out=None):
        if out is None:
            out = self._new(self.site_shape + (4, 3))
        check(lib().dwf_project_4d(self._h, _ptr(x5), _ptr(out), _stream()))
        return out

    def solve(self, b5, x5=None, allow_notconv=False, **kw):
        if x5 is None:
            x5 = self._new(self.shape5())
        p = default_params(**kw)
        st = SolveStats()
        rc = lib().dwf_solve(self._h, _ptr(b5), _ptr(x5), ctypes.byref(p), ctypes.byref(st), _stream())
        if rc != 0 and not (allow_notconv and rc == 4):
            check(rc)
        return x5, st.as_dict()

    def propagator_host(self, b4: np.ndarray, **kw):
        b4 = np.ascontiguousarray(b4, dtype=np.complex128)
        x4 = np.empty_like(b4)
        p = default_params(**kw)
        st = SolveStats()
        rc = lib().dwf_propagator_host(self._h, b4.ctypes.data_as(ctypes.c_void_p),
                                       x4.ctypes.data_as(ctypes.c_void_p), ctypes.byref(p),
                                       ctypes.byref(st), _stream())
        check(rc)
        return x4, st.as_dict()

    def fifth_matrix(self, which, chirality):
        out = (ctypes.c_double * (self.Ls * self.Ls))()
        check(lib().dwf_fifth_matrix(self._h, int(which), int(chirality), out))
        return np.array(out, dtype=np.float64).reshape(self.Ls, self.Ls)

    def set_hop_config(self, prec, variant, ns, sb):
        check(lib().dwf_set_hop_config(self._h, PREC[prec], int(variant), int(ns), int(sb)))

    def hop_config(self, prec):
        var, ns, sb = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(lib().dwf_get_hop_config(self._h, PREC[prec], ctypes.byref(var), ctypes.byref(ns),
                                       ctypes.byref(sb)))
        return var.value, ns.value, sb.value

    def set_sweep(self, prec, zblock):
        check(lib().dwf_set_sweep(self._h, PREC[prec], int(zblock)))

    def sweep(self, prec):
        zb = ctypes.c_int()
        check(lib().dwf_get_sweep(self._h, PREC[prec], ctypes.byref(zb)))
        return zb.value

    def set_mix_mode(self, prec, mode):
        check(lib().dwf_set_mix_mode(self._h, PREC[prec], int(mode)))

    def mix_mode(self, prec):
        m = ctypes.c_int()
        check(lib().dwf_get_mix_mode(self._h, PREC[prec], ctypes.byref(m)))
        return m.value

    def device_status(self):
        """DWF_OK, or raises DwfError(DWF_ETIMEOUT) if a bounded device wait gave up."""
        return check(lib().dwf_device_status(self._h, _stream()))

    def autotune(self, prec, cache_path=None):
        cp = cache_path.encode() if cache_path else None
        check(lib().dwf_autotune(self._h, PREC[prec], cp, _stream()))
        return self.hop_config(prec)

    def launch_count(self):
        return int(lib().dwf_launch_count(self._h))

    def device_bytes(self):
        return int(lib().dwf_device_bytes(self._h))

    # ------------------------------------------------ learned preconditioner
    def _wshape(self, layers):
        return (int(layers), 9, 2, self.Ls, self.Ls)

    def precond_init(self, layers=3, seed=7, noise=1e-3):
        check(lib().dwf_precond_init(self._h, int(layers), int(seed), float(noise)))

    def precond_set_weights(self, w):
        w = np.ascontiguousarray(w, dtype=np.complex128)
        check(lib().dwf_precond_set_weights(self._h, int(w.shape[0]),
                                            w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))

    def precond_get_weights(self, layers=3, compute_copy=True):
        w = np.empty(self._wshape(layers), dtype=np.complex128)
        check(lib().dwf_precond_get_weights(self._h, int(layers), int(bool(compute_copy)),
                                            w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return w

    def precond_apply(self, r, out=None, which="N"):
        """which: "N" the network, "Ndag" its adjoint, "M" = N N^dag."""
        if out is None:
            out = self._new(r.shape)
        check(lib().dwf_precond_apply(self._h, {"N": 0, "Ndag": 1, "M": 2}[which], _ptr(r), _ptr(out), _stream()))
        return out

    def precond_loss_grad(self, bs, xs, layers=3):
        n = len(bs)
        B = (ctypes.c_void_p * n)(*[_ptr(b).value for b in bs])
        X = (ctypes.c_void_p * n)(*[_ptr(x).value for x in xs])
        loss = ctypes.c_double()
        g = np.empty(self._wshape(layers), dtype=np.complex128)
        check(lib().dwf_precond_loss_grad(self._h, n, B, X, ctypes.byref(loss),
                                          g.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _stream()))
        return loss.value, g

    def precond_train(self, b4s, **kw):
        p = TrainParams()
        lib().dwf_train_params_default(ctypes.byref(p))
        for k, v in kw.items():
            if k == "solve_inner_prec":
                v = PREC[v]
            setattr(p, k, v)
        n = len(b4s)
        B = (ctypes.c_void_p * n)(*[_ptr(b).value for b in b4s])
        st = TrainStats()
        check(lib().dwf_precond_train(self._h, n, B, ctypes.byref(p), ctypes.byref(st), _stream()))
        return st.as_dict()

    def precond_adam_step(self, grad, lr, layers=3):
        """One Adam step of the network from a host gradient (weight layout)."""
        g = np.ascontiguousarray(np.asarray(grad, dtype=np.complex128))
        check(lib().dwf_precond_adam_step(self._h, int(layers), g.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                          float(lr), _stream()))

    def precond_fcg(self, b, tol=1e-6, max_iter=200, plain=False, out=None):
        """FP32 flexible CG on D^dag D x = b (EO fields) preconditioned by N N^dag
        (or by 1 when plain); returns (x, residual history)."""
        x = out if out is not None else self._new(self.shape_eo())
        hist = np.zeros(int(max_iter) + 1)
        n = ctypes.c_int()
        check(lib().dwf_precond_fcg(self._h, _ptr(b), _ptr(x), float(tol), int(max_iter), int(bool(plain)),
                                    hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(n),
                                    _stream()))
        return x, hist[: n.value + 1]

    def precond_save(self, path):
        check(lib().dwf_precond_save(self._h, os.fsencode(path)))

    def precond_load(self, path):
        check(lib().dwf_precond_load(self._h, os.fsencode(path)))

    def time_hop(self, prec="f32", reps=20, flush_l2=True):
        us = ctypes.c_double()
        by = ctypes.c_double()
        check(lib().dwf_time_hop(self._h, PREC[prec], int(reps), int(bool(flush_l2)), ctypes.byref(us),
                                 ctypes.byref(by), _stream()))
        return us.value, by.value

    def time_mix(self, prec="f32", mode=2, reps=20, flush_l2=True):
        """(us per launch, algorithmic bytes) of one stand-alone mixing launch."""
        us = ctypes.c_double()
        by = ctypes.c_double()
        check(lib().dwf_time_mix(self._h, PREC[prec], int(mode), int(reps), int(bool(flush_l2)), ctypes.byref(us),
                                 ctypes.byref(by), _stream()))
        return us.value, by.value

    def spectrum_bounds(self, max_steps=2000, rtol=1e-8, seed=1, eo_form=0):
        """(lambda_min, lambda_max, steps) of D^dag D, D the even-odd matrix (FP64 Lanczos);
        eo_form 1: the second even-odd form 1 - D_eo D_oo^-1 D_oe D_ee^-1."""
        lo, hi, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
        check(lib().dwf_spectrum_bounds(self._h, int(eo_form), int(max_steps), float(rtol), int(seed),
                                        ctypes.byref(lo), ctypes.byref(hi), ctypes.byref(n), _stream()))
        return lo.value, hi.value, n.value

    ITERATION_KERNELS = ("p_update", "hop_a", "hop_b", "hop_c_dag", "hop_d_dag")

    def time_iteration(self, prec="f16", reps=10, flush_l2=True):
        """Per-launch device time (us) and algorithmic bytes of the five launches
        of one inner CG iteration, as {name: (us, bytes)}."""
        us = (ctypes.c_double * 5)()
        by = (ctypes.c_double * 5)()
        check(lib().dwf_time_iteration(self._h, PREC[prec], int(reps), int(bool(flush_l2)), us, by, _stream()))
        return {k: (us[i], by[i]) for i, k in enumerate(self.ITERATION_KERNELS)}


KERNEL_MATRICES = ("P", "PT", "Q", "QT", "M", "MT", "A5R", "RA5T", "NHALF", "NHALF_RBT", "NQ4", "NPT4", "ID",
                   "HALF_Q", "SRC_POST", "SRC_Y", "NQUARTER", "NMT4")


def fifth_matrix_host(Ls, M0, mf, b, c, form="standard", alpha=1.0, which=0, chirality=0):
    """(matrix, banded) without a device: which 0..3 (A5, A5^-1, B, R) or a name of
    KERNEL_MATRICES (the per-chirality matrices the kernels apply); b and c
    numbers or sequences of Ls coefficients."""
    w = which if isinstance(which, int) else 16 + KERNEL_MATRICES.index(which)
    out = (ctypes.c_double * (Ls * Ls))()
    band = ctypes.c_int()
    ba, _ = _coeffs(b, Ls)
    ca, _ = _coeffs(c, Ls)
    check(lib().dwf_fifth_matrix_host(int(Ls), float(M0), float(mf), ba, ca, FORM[form], float(alpha),
                                      int(w), int(chirality), out, ctypes.byref(band)))
    return np.array(out, dtype=np.float64).reshape(Ls, Ls), bool(band.value)


def alu_peaks():
    """Measured FP32 (scalar FMA, packed FP32x2 FMA) and FP64 FMA rates of the
    current device in TFLOP/s, and its SM count."""
    out = (ctypes.c_double * 4)()
    check(lib().dwf_alu_peaks(out, _stream()))
    return {"fp32_ffma_tflops": out[0], "fp32_ffma2_tflops": out[1], "fp64_dfma_tflops": out[2],
            "sms": int(out[3])}


def solve_batch(ops, b4s, x4s=None, allow_notconv=False, **kw):
    """Solve len(ops) systems (4D sources -> 4D solutions) in shared launches."""
    import torch
    n = len(ops)
    if x4s is None:
        x4s = [torch.empty_like(b) for b in b4s]
    H = (ctypes.c_void_p * n)(*[o.handle for o in ops])
    B = (ctypes.c_void_p * n)(*[_ptr(b).value for b in b4s])
    X = (ctypes.c_void_p * n)(*[_ptr(x).value for x in x4s])
    p = default_params(**kw)
    st = (SolveStats * n)()
    rc = lib().dwf_solve_batch(H, B, X, n, ctypes.byref(p), st, _stream())
    if rc != 0 and not (allow_notconv and rc == 4):
        check(rc)
    return x4s, [s.as_dict() for s in st]


class Slab(Operator):
    """The time slices [t0, t0 + nt) of a lattice of extents global_dims (4D
    domain decomposition in time).  set_gauge takes the global link field; the
    even-odd matrix is applied in three stages with a face exchange between
    them (dwf_slab_apply_eo, dwf_slab_faces, dwf_slab_exchange_ring)."""

    def __init__(self, global_dims, t0, nt, Ls, M0, mf, b, c, form="standard", alpha=1.0, bc=None):
        self.global_dims = tuple(int(x) for x in global_dims)
        self.t0, self.nt = int(t0), int(nt)
        self.dims = self.global_dims[:3] + (self.nt,)
        self.Ls = int(Ls)
        h = ctypes.c_void_p()
        d = (ctypes.c_int * 4)(*self.global_dims)
        bcp = (ctypes.c_int * 4)(*bc) if bc is not None else None
        check(lib().dwf_create_slab(d, self.t0, self.nt, self.Ls, float(M0), float(mf), float(b), float(c),
                                    FORM[form], float(alpha), bcp, ctypes.byref(h)))
        self._h = h
        self.b, self.c = float(b), float(c)
        self.M0, self.mf = float(M0), float(mf)
        self.form, self.alpha = form, float(alpha)
        Lx, Ly, Lz, Lt = self.dims
        self.site_shape = (Lt, Lz, Ly, Lx)
        self.V = Lx * Ly * Lz * Lt

    def apply_eo_stage(self, stage, x=None, prec="f64", dag=False, out=None):
        if stage == 2 and out is None:
            out = self._new(self.shape_eo())
        check(lib().dwf_slab_apply_eo(self._h, PREC[prec], int(stage), int(bool(dag)),
                                      _ptr(x) if x is not None else None,
                                      _ptr(out) if out is not None else None, _stream()))
        return out

    def faces(self, prec, stage):
        p = [ctypes.c_void_p() for _ in range(4)]
        n = ctypes.c_size_t()
        check(lib().dwf_slab_faces(self._h, PREC[prec], int(stage), *[ctypes.byref(q) for q in p], ctypes.byref(n)))
        return dict(send_lo=p[0].value, send_hi=p[1].value, recv_lo=p[2].value, recv_hi=p[3].value, bytes=n.value)


def slab_exchange_ring(slabs, prec, stage):
    arr = (ctypes.c_void_p * len(slabs))(*[s.handle for s in slabs])
    check(lib().dwf_slab_exchange_ring(arr, len(slabs), PREC[prec], int(stage), _stream()))


def slab_apply_eo(slabs, xs, prec="f64", dag=False):
    """The even-odd matrix on a ring of slabs on one device: the three stages
    of every slab with the face exchanges between them."""
    for sl, x in zip(slabs, xs):
        sl.apply_eo_stage(0, x=x, prec=prec, dag=dag)
    slab_exchange_ring(slabs, prec, 0)
    for sl in slabs:
        sl.apply_eo_stage(1, prec=prec, dag=dag)
    slab_exchange_ring(slabs, prec, 1)
    return [sl.apply_eo_stage(2, prec=prec, dag=dag) for sl in slabs]


def slab_cgnr_ring(slabs, bs, tol=1e-10, max_iter=20000):
    """FP64 CGNR on the even-odd matrix over a ring of slabs on one device
    (dwf_slab_cgnr_ring): returns the slabs' solutions and the residual history."""
    n = len(slabs)
    xs = [sl._new(sl.shape_eo()) for sl in slabs]
    arr = (ctypes.c_void_p * n)(*[s.handle for s in slabs])
    bp = (ctypes.c_void_p * n)(*[_ptr(b).value for b in bs])
    xp = (ctypes.c_void_p * n)(*[_ptr(x).value for x in xs])
    its = ctypes.c_int()
    hist = (ctypes.c_double * (max_iter + 1))()
    check(lib().dwf_slab_cgnr_ring(arr, n, bp, xp, float(tol), int(max_iter), ctypes.byref(its), hist, _stream()))
    return xs, list(hist[:its.value + 1])
