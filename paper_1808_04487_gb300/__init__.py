"""Python binding of the sm_103a registration library (``include/claire.h``): argument marshalling only.

Every step of the hot path runs in the library's CUDA kernels; this module only checks shapes and dtypes, passes
``data_ptr()`` of CUDA tensors and the current torch stream, and raises ``ClaireError`` on a non-OK status. There
is no CPU fallback: if ``_lib/libclaire_gb.so`` is missing, importing a context raises (build it with
``python -m paper_1808_04487_gb300.build``).

Arrays: scalars are CUDA tensors of shape (n1, n2, n3), vectors (3, n1, n2, n3), C-contiguous, float32 for a
``precision="f32"`` context and float64 for ``"f64"``.
"""
from __future__ import annotations

import ctypes
import os

__all__ = ["Context", "ClaireError", "Report", "lib", "LIB_PATH", "STATUS", "register_batch"]

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libclaire_gb.so")

STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENAN", 5: "ENOTCONV", 6: "ELINESEARCH",
          7: "EBREAKDOWN", 8: "ETIMEOUT"}
OK, EINVAL, ENOMEM, ECUDA, ENAN, ENOTCONV, ELINESEARCH, EBREAKDOWN, ETIMEOUT = range(9)


class ClaireError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class Opts(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("precision", ctypes.c_int), ("beta", ctypes.c_double),
                ("nt", ctypes.c_int), ("regnorm", ctypes.c_int), ("divfree", ctypes.c_int),
                ("gtol_rel", ctypes.c_double), ("gtol_abs", ctypes.c_double), ("max_gn", ctypes.c_int),
                ("max_krylov", ctypes.c_int), ("pcg_rtol", ctypes.c_double), ("max_ls", ctypes.c_int),
                ("armijo_c1", ctypes.c_double), ("bf16_mask", ctypes.c_int), ("beta_w", ctypes.c_double),
                ("precond", ctypes.c_int), ("pc_kappa", ctypes.c_double)]


class Report(ctypes.Structure):
    _fields_ = [("gn_iters", ctypes.c_int), ("matvecs", ctypes.c_int), ("pde_solves", ctypes.c_int),
                ("ls_trials", ctypes.c_int), ("pcg_breakdowns", ctypes.c_int), ("converged", ctypes.c_int),
                ("J0", ctypes.c_double), ("J", ctypes.c_double), ("mismatch0", ctypes.c_double),
                ("mismatch", ctypes.c_double), ("gnorm0", ctypes.c_double), ("gnorm", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("coarse_matvecs", ctypes.c_int)]

    def as_dict(self):
        d = {name: getattr(self, name) for name, _ in self._fields_}
        d["gnorm_rel"] = self.gnorm / self.gnorm0 if self.gnorm0 > 0 else 0.0
        d["mismatch_rel"] = self.mismatch / self.mismatch0 if self.mismatch0 > 0 else 0.0
        return d


class PairF32(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("mT", ctypes.c_void_p), ("mR", ctypes.c_void_p), ("v", ctypes.c_void_p),
                ("rep", Report), ("status", ctypes.c_int)]


class Counters(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("halo_x", ctypes.c_int), ("halo_y", ctypes.c_int),
                ("halo_x_heavy", ctypes.c_int), ("halo_y_heavy", ctypes.c_int), ("pcg_graph_runs", ctypes.c_longlong),
                ("gn_graph_runs", ctypes.c_longlong), ("tma_steps", ctypes.c_longlong),
                ("fft_tile", ctypes.c_int * 3)]


_VP = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_PD = ctypes.POINTER(ctypes.c_double)
_LL = ctypes.c_longlong

# exported symbol -> argument types (after the context); the suffix _f32/_f64 is added for typed calls
_TYPED = {
    "claire_transport": [_VP, _VP, _I, _VP, _VP],
    "claire_gradient": [_VP, _VP, _VP, _VP, _PD, _VP],
    "claire_gradient_data": [_VP, _VP, _VP, _VP, _PD, _VP],
    "claire_symbol": [_I, _VP, _VP, _I, _VP],
    "claire_hessvec": [_VP, _VP, _VP, _VP, _VP, _VP],
    "claire_hessvec_cached": [_VP, _VP, _VP],
    "claire_hessvec_data": [_VP, _VP, _VP],
    "claire_linearize": [_VP, _VP, _VP],
    "claire_precond": [_VP, _VP, _VP],
    "claire_register": [_VP, _VP, _VP, ctypes.POINTER(Report), _VP],
    "claire_register_host": [_VP, _VP, _VP, ctypes.POINTER(Report), _VP],
    "claire_register_continuation": [_VP, _VP, _VP, _D, _D, ctypes.POINTER(Report), _I, ctypes.POINTER(_I), _VP],
    "claire_departure": [_VP, _I, _VP, _VP],
    "claire_interp": [_VP, _VP, _VP, _VP],
    "claire_spectral": [_I, _VP, _VP, _VP],
    "claire_objective": [_VP, _VP, _VP, _PD, _VP],
    "claire_dot": [_VP, _VP, _LL, _PD, _VP],
    "claire_fft": [_VP, _VP, _VP],
    "claire_ifft": [_VP, _VP, _VP],
}

_PI = ctypes.POINTER(ctypes.c_int)
_PF = ctypes.POINTER(ctypes.c_float)
_F = ctypes.c_float
_SZ = ctypes.c_size_t

# resampling, the warm-start network and its layers: symbol -> (return type, argument types)
_UNTYPED = {
    "claire_resample_f32": (_I, [_VP, _VP, _VP, _VP, _I, _I, _I, _VP]),
    "claire_set_beta": (_I, [_VP, _D]),
    "claire_ws_create": (_I, [_I, _I, _I, _I, _F, ctypes.c_ulonglong, ctypes.POINTER(_VP)]),
    "claire_ws_destroy": (_I, [_VP]),
    "claire_ws_last_error": (ctypes.c_char_p, [_VP]),
    "claire_ws_num_params": (_LL, [_VP]),
    "claire_ws_num_layers": (_I, [_VP]),
    "claire_ws_layer": (_I, [_VP, _I, _PI]),
    "claire_ws_num_ops": (_I, [_VP]),
    "claire_ws_op": (_I, [_VP, _I, _PI]),
    "claire_ws_get_params": (_I, [_VP, _PF]),
    "claire_ws_set_params": (_I, [_VP, _PF]),
    "claire_ws_get_grads": (_I, [_VP, _PF]),
    "claire_ws_forward_f32": (_I, [_VP, _VP, _PI, _I, _VP, _VP]),
    "claire_ws_loss_f32": (_I, [_VP, _VP, _VP, _PI, _I, _I, _PD, _VP]),
    "claire_ws_adam_step": (_I, [_VP, _F, _VP]),
    "claire_ws_train_step_f32": (_I, [_VP, _VP, _VP, _PI, _I, _F, _PD, _VP]),
    "claire_ws_predict_f32": (_I, [_VP, _VP, _VP, _VP, _VP, _I, _VP]),
    "claire_nn_conv3_fwd": (_I, [_VP, _VP, _VP, _VP, _VP, _VP, _I, _I, _I, _I, _I, _I, _I, _I, _VP, _VP]),
    "claire_nn_fwd_workspace_bytes": (_SZ, [_I, _I, _I, _I, _I]),
    "claire_nn_wgrad_workspace_bytes": (_SZ, [_I, _I, _I, _I, _I, _I]),
    "claire_nn_conv3_wgrad": (_I, [_VP, _VP, _VP, _VP, _I, _I, _I, _I, _I, _I, _VP]),
    "claire_nn_weight_flip": (_I, [_VP, _VP, _I, _I, _VP]),
    "claire_nn_relu_bwd": (_I, [_VP, _VP, _VP, _VP, _LL, _VP]),
    "claire_nn_bias_workspace_bytes": (_SZ, [_I]),
    "claire_nn_bias_grad": (_I, [_VP, _LL, _I, _VP, _VP, _VP]),
    "claire_nn_pool_fwd": (_I, [_VP, _VP, _I, _I, _I, _I, _I, _VP]),
    "claire_nn_pool_bwd": (_I, [_VP, _VP, _I, _I, _I, _I, _I, _I, _VP]),
    "claire_nn_up_fwd": (_I, [_VP, _VP, _I, _I, _I, _I, _I, _VP]),
    "claire_nn_up_bwd": (_I, [_VP, _VP, _I, _I, _I, _I, _I, _I, _VP]),
    "claire_nn_mse": (_I, [_VP, _VP, _VP, _LL, _I, _I, _VP, _I, _VP]),
    "claire_nn_adam": (_I, [_VP, _VP, _VP, _VP, _VP, _LL, _F, _F, _F, _F, _I, _VP]),
    "claire_nn_status": (_I, [_VP]),
}

_lib = None


def lib():
    """Load the in-tree library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("CUDA library not built: %s is missing (run python -m paper_1808_04487_gb300.build)"
                          % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    L.claire_default_opts.argtypes = [ctypes.POINTER(Opts), _I, _I, _I, _I]
    L.claire_default_opts.restype = _I
    L.claire_last_batch_graph_launches.argtypes = []
    L.claire_last_batch_graph_launches.restype = ctypes.c_longlong
    L.claire_create.argtypes = [ctypes.POINTER(Opts), ctypes.POINTER(_VP)]
    L.claire_create.restype = _I
    L.claire_destroy.argtypes = [_VP]
    L.claire_destroy.restype = _I
    L.claire_last_error.argtypes = [_VP]
    L.claire_last_error.restype = ctypes.c_char_p
    L.claire_workspace_bytes.argtypes = [_VP]
    L.claire_workspace_bytes.restype = ctypes.c_size_t
    L.claire_get_counters.argtypes = [_VP, ctypes.POINTER(Counters)]
    L.claire_get_counters.restype = _I
    L.claire_register_batch_f32.argtypes = [ctypes.POINTER(Opts), ctypes.POINTER(PairF32), _I, _I]
    L.claire_register_batch_f32.restype = _I
    L.claire_dot_noalloc_f32.argtypes = [_VP, _VP, _LL, _D, _VP, _VP]
    L.claire_dot_noalloc_f32.restype = _I
    L.claire_profile_enable.argtypes = [_VP, _I]
    L.claire_profile_enable.restype = _I
    L.claire_profile_report.argtypes = [_VP, ctypes.c_char_p, ctypes.c_size_t]
    L.claire_profile_report.restype = _I
    for base, args in _TYPED.items():
        for sfx in ("_f32", "_f64"):
            f = getattr(L, base + sfx)
            f.argtypes = [_VP] + args
            f.restype = _I
    for name, (res, args) in _UNTYPED.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def register_batch(pairs, nworkers=4, beta=5e-3, nt=4, regnorm=1, divfree=False, gtol_rel=5e-2, max_gn=50,
                   max_krylov=100, pcg_rtol=0.0):
    """Batched FP32 registration of independent pairs [(mT, mR, v), ...] of CUDA tensors (grids may differ); v is
    updated in place. Returns [(report dict, status name), ...] in input order."""
    L = lib()
    torch = _torch()
    o = Opts()
    L.claire_default_opts(ctypes.byref(o), 4, 4, 4, 0)
    o.beta, o.nt, o.regnorm, o.divfree = float(beta), int(nt), int(regnorm), int(bool(divfree))
    o.gtol_rel, o.max_gn, o.max_krylov, o.pcg_rtol = float(gtol_rel), int(max_gn), int(max_krylov), float(pcg_rtol)
    arr = (PairF32 * len(pairs))()
    for i, (mT, mR, v) in enumerate(pairs):
        n = tuple(mT.shape)
        for t, shp in ((mT, n), (mR, n), (v, (3,) + n)):
            if t.device.type != "cuda" or t.dtype != torch.float32 or tuple(t.shape) != shp or not t.is_contiguous():
                raise ValueError("pair %d: contiguous CUDA float32 tensors of matching grids required" % i)
        for a in range(3):
            arr[i].n[a] = n[a]
        arr[i].mT, arr[i].mR, arr[i].v = mT.data_ptr(), mR.data_ptr(), v.data_ptr()
    torch.cuda.synchronize()
    st = L.claire_register_batch_f32(ctypes.byref(o), arr, len(pairs), int(nworkers))
    if st not in (OK, ENOTCONV, ELINESEARCH):
        raise ClaireError(st, "claire_register_batch_f32 failed")
    return [(arr[i].rep.as_dict(), STATUS.get(arr[i].status, arr[i].status)) for i in range(len(pairs))]


def last_batch_graph_launches():
    """Graph launches of the most recent register_batch call: 1 when the batch ran as one CUDA graph."""
    return int(lib().claire_last_batch_graph_launches())


def _torch():
    import torch
    return torch


class Context:
    """One registration problem setup (grid, precision, beta, n_t, norm, constraint) and its device workspace."""

    def __init__(self, n, precision="f32", beta=1e-2, nt=4, regnorm=1, divfree=False, gtol_rel=5e-2,
                 gtol_abs=1e-6, max_gn=50, max_krylov=100, pcg_rtol=0.0, max_ls=10, armijo_c1=1e-4, bf16_mask=0,
                 beta_w=0.0, precond=0, pc_kappa=0.1):
        L = lib()
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        self.n = tuple(int(a) for a in n)
        self.precision = precision
        self.dtype = {"f32": torch.float32, "f64": torch.float64}[precision]
        o = Opts()
        prec = 0 if precision == "f32" else 1
        L.claire_default_opts(ctypes.byref(o), self.n[0], self.n[1], self.n[2], prec)
        o.beta, o.nt, o.regnorm, o.divfree = float(beta), int(nt), int(regnorm), int(bool(divfree))
        o.gtol_rel, o.gtol_abs, o.max_gn, o.max_krylov = float(gtol_rel), float(gtol_abs), int(max_gn), int(max_krylov)
        o.pcg_rtol, o.max_ls, o.armijo_c1 = float(pcg_rtol), int(max_ls), float(armijo_c1)
        o.bf16_mask = int(bf16_mask)
        o.beta_w = float(beta_w)
        o.precond, o.pc_kappa = int(precond), float(pc_kappa)
        self.opts = o
        torch.cuda.init()
        h = _VP()
        st = L.claire_create(ctypes.byref(o), ctypes.byref(h))
        if st != OK:
            raise ClaireError(st, "claire_create failed for n=%s precision=%s" % (self.n, precision))
        self._h = h
        self._sfx = "_" + precision

    # ------------------------------------------------------------------------------------------------ plumbing
    def close(self):
        if getattr(self, "_h", None):
            lib().claire_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self):
        return self._h

    def _call(self, name, *args, allow=(OK,)):
        f = getattr(lib(), name + self._sfx)
        st = f(self._h, *args)
        if st not in allow:
            raise ClaireError(st, lib().claire_last_error(self._h).decode())
        return st

    @staticmethod
    def _stream():
        return ctypes.c_void_p(_torch().cuda.current_stream().cuda_stream)

    def _check(self, t, shape, name):
        if t.device.type != "cuda" or t.dtype != self.dtype or tuple(t.shape) != shape or not t.is_contiguous():
            raise ValueError("%s must be a contiguous CUDA %s tensor of shape %s (got %s %s %s)"
                             % (name, self.dtype, shape, t.device, t.dtype, tuple(t.shape)))
        return ctypes.c_void_p(t.data_ptr())

    def _s(self, t, name):
        return self._check(t, self.n, name)

    def _v(self, t, name):
        return self._check(t, (3,) + self.n, name)

    def empty_scalar(self):
        return _torch().empty(self.n, dtype=self.dtype, device="cuda")

    def empty_vector(self):
        return _torch().empty((3,) + self.n, dtype=self.dtype, device="cuda")

    # ------------------------------------------------------------------------------------------------ calls
    def transport(self, m0, v, direction=+1, out=None):
        out = self.empty_scalar() if out is None else out
        self._call("claire_transport", self._s(m0, "m0"), self._v(v, "v"), int(direction), self._s(out, "out"),
                   self._stream())
        return out

    def gradient(self, mT, mR, v, out=None, objective=False):
        out = self.empty_vector() if out is None else out
        J = ctypes.c_double(0.0)
        self._call("claire_gradient", self._s(mT, "mT"), self._s(mR, "mR"), self._v(v, "v"), self._v(out, "g"),
                   ctypes.byref(J) if objective else None, self._stream())
        return (out, J.value) if objective else out

    def gradient_data(self, mT, mR, v, out=None, objective=False):
        """K[int lambda grad m dt]: the reduced gradient without beta A v (Eq. (5))."""
        out = self.empty_vector() if out is None else out
        J = ctypes.c_double(0.0)
        self._call("claire_gradient_data", self._s(mT, "mT"), self._s(mR, "mR"), self._v(v, "v"),
                   self._v(out, "out"), ctypes.byref(J) if objective else None, self._stream())
        return (out, J.value) if objective else out

    SYMBOL_OPS = {"betaA": 0, "precond": 1, "K": 2}

    def symbol(self, op, spec, out=None):
        """A diagonal Fourier symbol ("betaA", "precond" or "K") on half spectra of shape
        (ncomp, n1, n2, n3//2 + 1, 2) (interleaved re/im, as returned by fft)."""
        torch = _torch()
        shp = (self.n[0], self.n[1], self.n[2] // 2 + 1, 2)
        if (spec.device.type != "cuda" or spec.dtype != self.dtype or spec.dim() != 5 or tuple(spec.shape[1:]) != shp
                or not spec.is_contiguous()):
            raise ValueError("symbol: a contiguous CUDA tensor of shape (ncomp,) + %s required" % (shp,))
        out = torch.empty_like(spec) if out is None else out
        self._call("claire_symbol", self.SYMBOL_OPS[op], ctypes.c_void_p(spec.data_ptr()),
                   ctypes.c_void_p(out.data_ptr()), int(spec.shape[0]), self._stream())
        return out

    def linearize(self, mT, v):
        self._call("claire_linearize", self._s(mT, "mT"), self._v(v, "v"), self._stream())

    def hessvec(self, mT, v, vt, out=None):
        out = self.empty_vector() if out is None else out
        self._call("claire_hessvec", self._s(mT, "mT"), None, self._v(v, "v"), self._v(vt, "vt"),
                   self._v(out, "Hvt"), self._stream())
        return out

    def hessvec_cached(self, vt, out=None):
        out = self.empty_vector() if out is None else out
        self._call("claire_hessvec_cached", self._v(vt, "vt"), self._v(out, "Hvt"), self._stream())
        return out

    def hessvec_data(self, vt, out=None):
        out = self.empty_vector() if out is None else out
        self._call("claire_hessvec_data", self._v(vt, "vt"), self._v(out, "out"), self._stream())
        return out

    def precond(self, r, out=None):
        out = self.empty_vector() if out is None else out
        self._call("claire_precond", self._v(r, "r"), self._v(out, "z"), self._stream())
        return out

    def register(self, mT, mR, v=None):
        """Solve in place on v (zeros if None); returns (v, report dict, status name)."""
        v = _torch().zeros((3,) + self.n, dtype=self.dtype, device="cuda") if v is None else v
        rep = Report()
        st = self._call("claire_register", self._s(mT, "mT"), self._s(mR, "mR"), self._v(v, "v"), ctypes.byref(rep),
                        self._stream(), allow=(OK, ENOTCONV, ELINESEARCH))
        return v, rep.as_dict(), STATUS[st]

    def register_continuation(self, mT, mR, v=None, beta_start=1.0, factor=0.1, max_levels=16):
        """Continuation in beta_v down to this context's beta (Sec. 3.6); returns (v, [report dict per level],
        status name of the last level)."""
        v = _torch().zeros((3,) + self.n, dtype=self.dtype, device="cuda") if v is None else v
        reps = (Report * max_levels)()
        nlev = ctypes.c_int(0)
        st = self._call("claire_register_continuation", self._s(mT, "mT"), self._s(mR, "mR"), self._v(v, "v"),
                        float(beta_start), float(factor), reps, int(max_levels), ctypes.byref(nlev), self._stream(),
                        allow=(OK, ENOTCONV, ELINESEARCH))
        return v, [reps[i].as_dict() for i in range(nlev.value)], STATUS[st]

    def set_beta(self, beta):
        st = lib().claire_set_beta(self._h, float(beta))
        if st != OK:
            raise ClaireError(st, "claire_set_beta(%r)" % beta)

    def register_host(self, mT, mR, v):
        """Same solve on HOST tensors (CPU, ideally pinned); v is updated in place."""
        torch = _torch()
        for t, shp, name in ((mT, self.n, "mT"), (mR, self.n, "mR"), (v, (3,) + self.n, "v")):
            if t.device.type != "cpu" or t.dtype != self.dtype or tuple(t.shape) != shp or not t.is_contiguous():
                raise ValueError("%s must be a contiguous CPU %s tensor of shape %s" % (name, self.dtype, shp))
        rep = Report()
        st = self._call("claire_register_host", ctypes.c_void_p(mT.data_ptr()), ctypes.c_void_p(mR.data_ptr()),
                        ctypes.c_void_p(v.data_ptr()), ctypes.byref(rep), self._stream(),
                        allow=(OK, ENOTCONV, ELINESEARCH))
        del torch
        return v, rep.as_dict(), STATUS[st]

    def departure(self, v, direction=+1, out=None):
        out = self.empty_vector() if out is None else out
        self._call("claire_departure", self._v(v, "v"), int(direction), self._v(out, "disp"), self._stream())
        return out

    def interp(self, f, disp, out=None):
        out = self.empty_scalar() if out is None else out
        self._call("claire_interp", self._s(f, "f"), self._v(disp, "disp"), self._s(out, "out"), self._stream())
        return out

    SPECTRAL_OPS = {"grad": (0, False, True), "div": (1, True, False), "leray": (2, True, True),
                    "A": (3, True, True), "lap": (4, False, False)}

    def spectral(self, op, x, out=None):
        code, vin, vout = self.SPECTRAL_OPS[op]
        if out is None:
            out = self.empty_vector() if vout else self.empty_scalar()
        xin = self._v(x, "in") if vin else self._s(x, "in")
        xout = self._v(out, "out") if vout else self._s(out, "out")
        self._call("claire_spectral", code, xin, xout, self._stream())
        return out

    def objective(self, m1, mR, v):
        J = ctypes.c_double(0.0)
        self._call("claire_objective", self._s(m1, "m1"), self._s(mR, "mR"), self._v(v, "v"), ctypes.byref(J),
                   self._stream())
        return J.value

    def dot(self, a, b):
        if a.dtype != self.dtype or b.dtype != self.dtype or a.numel() != b.numel() or a.device.type != "cuda":
            raise ValueError("dot: matching CUDA tensors of the context dtype required")
        out = ctypes.c_double(0.0)
        self._call("claire_dot", ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()), a.numel(),
                   ctypes.byref(out), self._stream())
        return out.value

    def fft(self, f):
        torch = _torch()
        spec = torch.empty((self.n[0], self.n[1], self.n[2] // 2 + 1, 2), dtype=self.dtype, device="cuda")
        self._call("claire_fft", self._s(f, "f"), ctypes.c_void_p(spec.data_ptr()), self._stream())
        return spec

    def ifft(self, spec):
        out = self.empty_scalar()
        self._call("claire_ifft", ctypes.c_void_p(spec.data_ptr()), self._s(out, "f"), self._stream())
        return out

    def workspace_bytes(self):
        return int(lib().claire_workspace_bytes(self._h))

    def profile(self, on=True):
        lib().claire_profile_enable(self._h, 1 if on else 0)

    def profile_report(self):
        """{kernel name: (launches, total ms)} recorded since the last report."""
        import json
        buf = ctypes.create_string_buffer(1 << 16)
        lib().claire_profile_report(self._h, buf, len(buf))
        return {k: tuple(v) for k, v in json.loads(buf.value.decode()).items()}

    def launches(self):
        c = Counters()
        lib().claire_get_counters(self._h, ctypes.byref(c))
        return int(c.launches)

    def pcg_graph_runs(self):
        """PCG solves run as one CUDA-graph launch (device-driven loop) on this context."""
        c = Counters()
        lib().claire_get_counters(self._h, ctypes.byref(c))
        return int(c.pcg_graph_runs)

    def gn_graph_runs(self):
        """Launches of the graph of the whole solve driven from the device on this context."""
        c = Counters()
        lib().claire_get_counters(self._h, ctypes.byref(c))
        return int(c.gn_graph_runs)

    def tma_steps(self):
        """Adjoint steps run with TMA-staged operands on this context."""
        c = Counters()
        lib().claire_get_counters(self._h, ctypes.byref(c))
        return int(c.tma_steps)

    def fft_tiles(self):
        """{"z", "y", "x"}: tile variant of each length-specialised FFT pass (0 default, 1 half, 2 double)."""
        c = Counters()
        lib().claire_get_counters(self._h, ctypes.byref(c))
        return {"z": int(c.fft_tile[0]), "y": int(c.fft_tile[1]), "x": int(c.fft_tile[2])}

    def gather_schedule(self):
        """{"halo_x", "halo_y", "halo_x_heavy", "halo_y_heavy"}: brick halos of the tiled gathers of the cached
        linearisation for the light and the heavy kernels (-1: plain)."""
        c = Counters()
        lib().claire_get_counters(self._h, ctypes.byref(c))
        return {"halo_x": int(c.halo_x), "halo_y": int(c.halo_y), "halo_x_heavy": int(c.halo_x_heavy),
                "halo_y_heavy": int(c.halo_y_heavy)}

    def resample_to(self, dst, f, project=False, out=None, kmax=0):
        """f ([ncomp,] n) on this grid -> dst's grid by Fourier truncation / zero padding (FP32 contexts)."""
        vec = f.dim() == 4
        nc = f.shape[0] if vec else 1
        shape = ((nc,) if vec else ()) + dst.n
        out = _torch().empty(shape, dtype=dst.dtype, device="cuda") if out is None else out
        self._check(f, ((nc,) if vec else ()) + self.n, "f")
        dst._check(out, shape, "out")
        st = lib().claire_resample_f32(self._h, dst._h, ctypes.c_void_p(f.data_ptr()),
                                       ctypes.c_void_p(out.data_ptr()), nc, int(bool(project)), int(kmax),
                                       self._stream())
        if st != OK:
            raise ClaireError(st, lib().claire_last_error(dst._h).decode())
        return out
