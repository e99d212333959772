"""Python binding of the GB300 MLBA library (libmlba.so, C ABI in include/mlba.h).

Argument marshalling only: every step of the algorithm runs in the library's
CUDA kernels.  PyTorch provides device memory and the stream the library
queues its work on.  Importing this module does not need a GPU; creating a
context does, and fails loudly if the compiled library is missing.

Names follow the paper (arXiv 1504.07234): ``bc`` is the boundary treatment
of Section 2 ('zero', 'periodic', 'reflective' or 'rect' for the rectangular
operator), ``precond`` the variant of Sections 3-5 ('none', 'bccb' =
Algorithm 1, 'krylov' = Algorithm 2, 'sym' = Algorithm 3, 'tikh' =
Algorithm 4, 'tikh_ns' = Algorithm 4-NS).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmlba.so")

BC = {"zero": 0, "periodic": 1, "reflective": 2, "rect": 3, "antireflective": 4}
PRECOND = {"none": 0, "bccb": 1, "krylov": 2, "sym": 3, "tikh": 4, "tikh_ns": 5}
TRANSFORM = {"auto": 0, "dft": 1, "dct": 2, "ar": 3}
DTYPE = {"f32": 0, "f64": 1, "bf16": 2}
ERRORS = {0: "ok", -1: "invalid argument", -2: "out of memory", -3: "CUDA runtime error",
          -4: "device wait timed out", -5: "diverged", -6: "call out of order",
          -7: "unsupported size"}


class MlbaError(RuntimeError):
    def __init__(self, code, where):
        super().__init__(f"{where}: {ERRORS.get(code, code)} ({code})")
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_double), ("alpha", ctypes.c_double), ("gamma", ctypes.c_double),
                ("q", ctypes.c_double), ("rho", ctypes.c_double), ("pcg_tol", ctypes.c_double),
                ("levels", ctypes.c_int), ("max_iter", ctypes.c_int), ("pcg_max", ctypes.c_int),
                ("dtype", ctypes.c_int), ("z_store", ctypes.c_int), ("transform", ctypes.c_int),
                ("stop", ctypes.c_int), ("rect_ns_hybrid", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("two_group", ctypes.c_int),
                ("autotune", ctypes.c_int), ("frame_shape", ctypes.c_int),
                ("blur_path", ctypes.c_int), ("formulation", ctypes.c_int),
                ("persistent", ctypes.c_int), ("wait_s", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("iter", ctypes.c_int), ("stopped", ctypes.c_int), ("stop_iter", ctypes.c_int),
                ("status", ctypes.c_int), ("resnorm", ctypes.c_double), ("alpha_n", ctypes.c_double),
                ("beta_n", ctypes.c_int), ("nres", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ProblemDesc(ctypes.Structure):
    _fields_ = [("psf", ctypes.c_void_p), ("p", ctypes.c_int), ("n", ctypes.c_int),
                ("bc", ctypes.c_int), ("precond", ctypes.c_int), ("transform", ctypes.c_int),
                ("max_iter", ctypes.c_int), ("mu", ctypes.c_double), ("alpha", ctypes.c_double),
                ("delta", ctypes.c_double), ("g", ctypes.c_void_p), ("g_on_device", ctypes.c_int)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
SIGNATURES = {
    "mlba_opts_default": (None, [ctypes.POINTER(Opts)]),
    "mlba_create": (_I, [_P, _I, _I, _I, _I, ctypes.POINTER(Opts), ctypes.POINTER(_P)]),
    "mlba_set_data": (_I, [_P, _P, _I, _D]),
    "mlba_iterate": (_I, [_P, _I]),
    "mlba_result": (_I, [_P, _P, _I]),
    "mlba_stats_get": (_I, [_P, ctypes.POINTER(Stats)]),
    "mlba_history": (_I, [_P, _P, _P, _P, _I]),
    "mlba_get_z": (_I, [_P, _P, _I]),
    "mlba_state_size": (_I, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    "mlba_get_state": (_I, [_P, _P, ctypes.c_size_t]),
    "mlba_set_state": (_I, [_P, _P, ctypes.c_size_t]),
    "mlba_destroy": (None, [_P]),
    "mlba_strerror": (ctypes.c_char_p, [_I]),
    "mlba_op_blur": (_I, [_P, _P, _P, _I]),
    "mlba_op_blur_adjoint": (_I, [_P, _P, _P, _I]),
    "mlba_op_precond": (_I, [_P, _P, _P, _D, _I, _I]),
    "mlba_op_frame": (_I, [_P, _P, _P, _P, _P, _D, _I]),
    "mlba_op_ns_alpha": (_I, [_P, _P, _D, ctypes.POINTER(_D), _I]),
    "mlba_op_spectrum": (_I, [_P, _P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "mlba_batch_create": (_I, [ctypes.POINTER(ProblemDesc), _I, ctypes.POINTER(Opts), ctypes.POINTER(_P)]),
    "mlba_batch_iterate": (_I, [_P, _I]),
    "mlba_batch_active": (_I, [_P, ctypes.POINTER(_I)]),
    "mlba_batch_result": (_I, [_P, _I, _P, _I]),
    "mlba_batch_stats": (_I, [_P, _I, ctypes.POINTER(Stats)]),
    "mlba_batch_reset": (_I, [_P]),
    "mlba_batch_set_data": (_I, [_P, _I, _P, _I, _D]),
    "mlba_batch_set_data_all": (_I, [_P, ctypes.POINTER(_P), _I, ctypes.POINTER(_D)]),
    "mlba_batch_result_all": (_I, [_P, ctypes.POINTER(_P), _I]),
    "mlba_batch_profile": (_I, [_P, _I, _I, ctypes.POINTER(ctypes.c_float)]),
    "mlba_batch_graph_kernels": (_I, [_P, ctypes.POINTER(_I)]),
    "mlba_batch_destroy": (None, [_P]),
    "mlba_batch_tiles": (_I, [_P] + [ctypes.POINTER(_I)] * 5 + [ctypes.POINTER(ctypes.c_float)]),
    "mlba_tiles": (_I, [_P] + [ctypes.POINTER(_I)] * 5 + [ctypes.POINTER(ctypes.c_float)]),
    "mlba_batch_blur_fft": (_I, [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "mlba_residual_noalloc": (_I, [_P, _P, _P, _I, _I, _I, _P, _P, _P]),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libmlba.so (no GPU needed) and declare the C signatures."""
    global _lib
    if _lib is not None and path == LIB_PATH:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_1504_07234_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path == LIB_PATH:
        _lib = lib
    return lib


def _check(code, where):
    if code < 0:
        raise MlbaError(code, where)
    return code


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("the MLBA library needs a CUDA GPU")
    return torch


def make_opts(dtype="f32", z_store=None, mu=10.0 / 255.0, alpha=0.05, levels=1, max_iter=200,
              stop=True, gamma=1.0 + 1e-15, q=0.5, rho=1e-4, transform="auto", pcg_tol=1e-3,
              pcg_max=5, rect_ns_hybrid=False, stream=None, two_group=True, autotune=0,
              frame_shape=-1, blur_path=0, formulation="synthesis", persistent=False,
              wait_s=1.0) -> Opts:
    lib = load_library()
    o = Opts()
    lib.mlba_opts_default(ctypes.byref(o))
    o.mu, o.alpha, o.gamma, o.q, o.rho, o.pcg_tol = mu, alpha, gamma, q, rho, pcg_tol
    o.levels, o.max_iter, o.pcg_max = levels, max_iter, pcg_max
    o.dtype = DTYPE[dtype]
    o.z_store = DTYPE[z_store or dtype]
    o.transform = TRANSFORM[transform]
    o.stop = 1 if stop else 0
    o.rect_ns_hybrid = 1 if rect_ns_hybrid else 0
    o.stream = stream
    o.two_group = 1 if two_group else 0
    o.autotune = int(autotune)
    o.frame_shape = int(frame_shape)
    o.blur_path = {"direct": 0, "fft": 1, "auto": 2}.get(blur_path, blur_path)
    o.formulation = {"synthesis": 0, "balanced": 1}.get(formulation, formulation)
    o.persistent = 1 if persistent else 0
    o.wait_s = float(wait_s)
    return o


def _tiles(fn, h):
    v = [ctypes.c_int() for _ in range(5)]
    us = ctypes.c_float()
    _check(fn(h, *[ctypes.byref(x) for x in v], ctypes.byref(us)), "tiles")
    how = {0: "default", 1: "measured", 2: "cache", 3: "forced"}[v[4].value]
    return {"frame_shape": v[0].value, "tile_x": v[1].value, "tile_y": v[2].value,
            "prefetch": v[3].value, "how": how, "us": us.value}


class _Base:
    """Shared stream handling: the library works on a dedicated torch stream
    that is ordered against torch's current stream around every call."""

    def _init_stream(self):
        torch = _torch()
        self.torch = torch
        self.stream = torch.cuda.Stream()
        return self.stream.cuda_stream

    def _enter(self):
        self.stream.wait_stream(self.torch.cuda.current_stream())

    def _leave(self):
        self.torch.cuda.current_stream().wait_stream(self.stream)

    def _np_dtype(self):
        return np.float64 if self.dtype == "f64" else np.float32

    def _torch_dtype(self):
        return self.torch.float64 if self.dtype == "f64" else self.torch.float32

    def _zdtype(self):
        t = self.torch
        return {"f64": t.float64, "f32": t.float32, "bf16": t.bfloat16}[self.z_store]

    def _arg(self, x):
        """(pointer, on_device, keepalive) for a host numpy array or device tensor."""
        t = self.torch
        if isinstance(x, t.Tensor):
            if not x.is_cuda:
                x = x.numpy()
            else:
                x = x.contiguous()
                return ctypes.c_void_p(x.data_ptr()), 1, x
        a = np.ascontiguousarray(x, dtype=self._np_dtype())
        return a.ctypes.data_as(ctypes.c_void_p), 0, a


class Context(_Base):
    """One deblurring problem (mlba_create ... mlba_destroy)."""

    def __init__(self, psf, n, bc, precond, dtype="f32", z_store=None, **kw):
        self.lib = load_library()
        stream = self._init_stream()
        self.dtype = dtype
        self.z_store = z_store or dtype
        if dtype == "f64":
            self.z_store = "f64"
        self.psf = np.ascontiguousarray(psf, dtype=np.float64)
        self.p = self.psf.shape[0]
        self.n = int(n)
        self.bc = bc
        self.levels = kw.get("levels", 1)
        self.nf = self.n + self.p - 1 if bc == "rect" else self.n
        self.nbands = 8 * self.levels + 1
        self.opts = make_opts(dtype=dtype, z_store=self.z_store, stream=stream, **kw)
        h = ctypes.c_void_p()
        _check(self.lib.mlba_create(self.psf.ctypes.data_as(ctypes.c_void_p), self.p, self.n,
                                    BC[bc], PRECOND[precond], ctypes.byref(self.opts),
                                    ctypes.byref(h)), "mlba_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.stream.synchronize()
            self.lib.mlba_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- loop ------------------------------------------------------------
    def set_data(self, g, delta):
        ptr, dev, keep = self._arg(g)
        self._enter()
        _check(self.lib.mlba_set_data(self.h, ptr, dev, float(delta)), "mlba_set_data")

    def iterate(self, k):
        _check(self.lib.mlba_iterate(self.h, int(k)), "mlba_iterate")
        self._leave()

    def run(self, max_iter=None):
        """Iterate until stopped (at most max_iter + 1 steps)."""
        k = (max_iter if max_iter is not None else self.opts.max_iter) + 1
        self.iterate(k)
        return self.stats()

    def result(self, device=False):
        t = self.torch
        if device:
            out = t.empty((self.nf, self.nf), dtype=self._torch_dtype(), device="cuda")
            _check(self.lib.mlba_result(self.h, ctypes.c_void_p(out.data_ptr()), 1), "mlba_result")
            self._leave()
            return out
        out = np.empty((self.nf, self.nf), dtype=self._np_dtype())
        _check(self.lib.mlba_result(self.h, out.ctypes.data_as(ctypes.c_void_p), 0), "mlba_result")
        return out

    def stats(self):
        s = Stats()
        _check(self.lib.mlba_stats_get(self.h, ctypes.byref(s)), "mlba_stats_get")
        return s.as_dict()

    def tiles(self):
        """Tile shape of the framelet launch and how it was chosen."""
        return _tiles(self.lib.mlba_tiles, self.h)

    def history(self):
        cap = self.opts.max_iter + 2
        res = np.zeros(cap)
        al = np.zeros(cap)
        be = np.zeros(cap, dtype=np.int32)
        n = _check(self.lib.mlba_history(self.h, res.ctypes.data_as(ctypes.c_void_p),
                                         al.ctypes.data_as(ctypes.c_void_p),
                                         be.ctypes.data_as(ctypes.c_void_p), cap), "mlba_history")
        it = self.stats()["iter"]
        return res[:n], al[:it], be[:it]

    def get_z(self):
        t = self.torch
        out = t.empty((self.nbands, self.nf, self.nf), dtype=self._zdtype(), device="cuda")
        _check(self.lib.mlba_get_z(self.h, ctypes.c_void_p(out.data_ptr()), 1), "mlba_get_z")
        self._leave()
        return out

    def get_state(self):
        """Checkpoint: the state blob (bytes) from which set_state resumes."""
        n = ctypes.c_size_t()
        _check(self.lib.mlba_state_size(self.h, ctypes.byref(n)), "mlba_state_size")
        buf = (ctypes.c_ubyte * n.value)()
        self._enter()
        _check(self.lib.mlba_get_state(self.h, ctypes.cast(buf, ctypes.c_void_p), n.value),
               "mlba_get_state")
        return bytes(buf)

    def set_state(self, blob):
        """Resume from a blob of get_state (call set_data first)."""
        buf = (ctypes.c_ubyte * len(blob)).from_buffer_copy(blob)
        self._enter()
        _check(self.lib.mlba_set_state(self.h, ctypes.cast(buf, ctypes.c_void_p), len(blob)),
               "mlba_set_state")

    # -- operators -------------------------------------------------------------
    def _op_out(self, shape, device):
        if device:
            return self.torch.empty(shape, dtype=self._torch_dtype(), device="cuda")
        return np.empty(shape, dtype=self._np_dtype())

    def _call_op(self, fn, name, x, shape, *extra):
        ptr, dev, keep = self._arg(x)
        out = self._op_out(shape, dev)
        optr = ctypes.c_void_p(out.data_ptr()) if dev else out.ctypes.data_as(ctypes.c_void_p)
        self._enter()
        _check(fn(self.h, ptr, optr, *extra, dev), name)
        self._leave()
        return out

    def blur(self, f):
        """A f (Section 2)."""
        return self._call_op(self.lib.mlba_op_blur, "mlba_op_blur", f, (self.n, self.n))

    def blur_adjoint(self, t):
        """A^T t."""
        return self._call_op(self.lib.mlba_op_blur_adjoint, "mlba_op_blur_adjoint", t,
                             (self.nf, self.nf))

    def precond(self, r, alpha, which="inv"):
        """(CC^T + alpha I)^{-1} r ('inv') or C^T (CC^T + alpha I)^{-1} r ('tikh')."""
        return self._call_op(self.lib.mlba_op_precond, "mlba_op_precond", r, (self.n, self.n),
                             float(alpha), 0 if which == "inv" else 1)

    def frame(self, z_in, u, mu):
        """One fused framelet pass: (z_in + W u, W^T S_mu(z_in + W u))."""
        t = self.torch
        zi = t.as_tensor(np.asarray(z_in) if not isinstance(z_in, t.Tensor) else z_in)
        zi = zi.to(device="cuda", dtype=self._zdtype()).contiguous()
        uu = t.as_tensor(np.asarray(u) if not isinstance(u, t.Tensor) else u)
        uu = uu.to(device="cuda", dtype=self._torch_dtype()).contiguous()
        zo = t.empty_like(zi)
        f = t.empty((self.nf, self.nf), dtype=self._torch_dtype(), device="cuda")
        self._enter()
        _check(self.lib.mlba_op_frame(self.h, ctypes.c_void_p(zi.data_ptr()),
                                      ctypes.c_void_p(uu.data_ptr()), ctypes.c_void_p(zo.data_ptr()),
                                      ctypes.c_void_p(f.data_ptr()), float(mu), 1), "mlba_op_frame")
        self._leave()
        return zo, f

    def ns_alpha(self, r, qn):
        """alpha solving alpha ||(CC^T + alpha I)^{-1} r|| = qn ||r|| (Eq. Alg4_rev_7)."""
        ptr, dev, keep = self._arg(r)
        out = ctypes.c_double()
        self._enter()
        _check(self.lib.mlba_op_ns_alpha(self.h, ptr, float(qn), ctypes.byref(out), dev),
               "mlba_op_ns_alpha")
        return out.value

    def spectrum(self):
        rows, cols, cplx = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        buf = np.zeros(self.n * (self.n + 2) * 2)
        self.stream.synchronize()
        _check(self.lib.mlba_op_spectrum(self.h, buf.ctypes.data_as(ctypes.c_void_p),
                                         ctypes.byref(rows), ctypes.byref(cols),
                                         ctypes.byref(cplx)), "mlba_op_spectrum")
        r, c = rows.value, cols.value
        if cplx.value:
            v = buf[:2 * r * c].reshape(r, c, 2)
            return v[..., 0] + 1j * v[..., 1]
        return buf[:r * c].reshape(r, c)


class Batch(_Base):
    """Independent problems advanced together by one graph launch per step."""

    def __init__(self, problems, dtype="f32", z_store=None, **kw):
        """``problems``: sequence of dicts with keys psf, g, delta, bc, precond
        and optionally mu, alpha, transform, max_iter."""
        self.lib = load_library()
        stream = self._init_stream()
        self.dtype = dtype
        self.z_store = z_store or dtype
        self.opts = make_opts(dtype=dtype, z_store=self.z_store, stream=stream, **kw)
        self.count = len(problems)
        self._keep = []
        descs = (ProblemDesc * self.count)()
        self.shapes = []
        for i, pr in enumerate(problems):
            psf = np.ascontiguousarray(pr["psf"], dtype=np.float64)
            ptr, dev, keep = self._arg(pr["g"])
            self._keep += [psf, keep]
            d = descs[i]
            d.psf = psf.ctypes.data_as(ctypes.c_void_p)
            d.p = psf.shape[0]
            d.n = int(np.shape(pr["g"])[0])
            d.bc = BC[pr["bc"]]
            d.precond = PRECOND[pr["precond"]]
            d.transform = TRANSFORM[pr.get("transform", "auto")]
            d.max_iter = int(pr.get("max_iter", self.opts.max_iter))
            d.mu = float(pr.get("mu", self.opts.mu))
            d.alpha = float(pr.get("alpha", self.opts.alpha))
            d.delta = float(pr["delta"])
            d.g = ptr
            d.g_on_device = dev
            nf = d.n + d.p - 1 if pr["bc"] == "rect" else d.n
            self.shapes.append((d.n, nf))
        h = ctypes.c_void_p()
        self._enter()
        _check(self.lib.mlba_batch_create(descs, self.count, ctypes.byref(self.opts),
                                          ctypes.byref(h)), "mlba_batch_create")
        self.h = h
        self._keep = []

    def close(self):
        if getattr(self, "h", None):
            self.stream.synchronize()
            self.lib.mlba_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def iterate(self, k):
        _check(self.lib.mlba_batch_iterate(self.h, int(k)), "mlba_batch_iterate")
        self._leave()

    def active(self):
        a = ctypes.c_int()
        _check(self.lib.mlba_batch_active(self.h, ctypes.byref(a)), "mlba_batch_active")
        return a.value

    def reset(self):
        _check(self.lib.mlba_batch_reset(self.h), "mlba_batch_reset")

    def result(self, i, device=False, out=None):
        nf = self.shapes[i][1]
        if out is not None:       # caller-provided host array (e.g. pinned)
            assert out.flags.c_contiguous and out.dtype == self._np_dtype() and out.shape == (nf, nf)
            _check(self.lib.mlba_batch_result(self.h, i, out.ctypes.data_as(ctypes.c_void_p), 0),
                   "mlba_batch_result")
            return out
        if device:
            out = self.torch.empty((nf, nf), dtype=self._torch_dtype(), device="cuda")
            _check(self.lib.mlba_batch_result(self.h, i, ctypes.c_void_p(out.data_ptr()), 1),
                   "mlba_batch_result")
            self._leave()
            return out
        out = np.empty((nf, nf), dtype=self._np_dtype())
        _check(self.lib.mlba_batch_result(self.h, i, out.ctypes.data_as(ctypes.c_void_p), 0),
               "mlba_batch_result")
        return out

    def stats(self, i):
        s = Stats()
        _check(self.lib.mlba_batch_stats(self.h, i, ctypes.byref(s)), "mlba_batch_stats")
        return s.as_dict()

    def set_data(self, i, g, delta):
        ptr, dev, keep = self._arg(g)
        self._enter()
        _check(self.lib.mlba_batch_set_data(self.h, int(i), ptr, dev, float(delta)),
               "mlba_batch_set_data")

    def set_data_all(self, gs, deltas):
        """Every problem's g and delta, one synchronisation (all on the host or
        all on the device)."""
        if len(gs) != len(self.shapes) or len(deltas) != len(self.shapes):
            raise ValueError("one g and one delta per problem")
        args = [self._arg(g) for g in gs]
        devs = {a[1] for a in args}
        if len(devs) != 1:
            raise ValueError("all g on the host or all on the device")
        ptrs = (_P * len(args))(*[a[0] for a in args])
        d = (_D * len(args))(*[float(x) for x in deltas])
        self._enter()
        _check(self.lib.mlba_batch_set_data_all(self.h, ptrs, devs.pop(), d),
               "mlba_batch_set_data_all")

    def result_all(self, outs=None):
        """Every problem's f, one synchronisation; into caller-provided host
        arrays (e.g. pinned) when outs is given."""
        if outs is None:
            outs = [np.empty((nf, nf), dtype=self._np_dtype()) for _, nf in self.shapes]
        if len(outs) != len(self.shapes):
            raise ValueError("one output per problem")
        for o, (_, nf) in zip(outs, self.shapes):
            assert o.flags.c_contiguous and o.dtype == self._np_dtype() and o.shape == (nf, nf)
        ptrs = (_P * len(outs))(*[o.ctypes.data_as(ctypes.c_void_p) for o in outs])
        _check(self.lib.mlba_batch_result_all(self.h, ptrs, 0), "mlba_batch_result_all")
        return outs

    def profile(self, stage, reps):
        """Mean milliseconds per launch of one stage (0 = whole step)."""
        ms = ctypes.c_float()
        self._enter()
        _check(self.lib.mlba_batch_profile(self.h, int(stage), int(reps), ctypes.byref(ms)),
               "mlba_batch_profile")
        return ms.value

    def tiles(self):
        """Tile shape of the framelet launch and how it was chosen."""
        return _tiles(self.lib.mlba_batch_tiles, self.h)

    def blur_fft(self, i):
        """(uses FFT convolution, convolution size) of problem i."""
        u, m = ctypes.c_int(), ctypes.c_int()
        _check(self.lib.mlba_batch_blur_fft(self.h, int(i), ctypes.byref(u), ctypes.byref(m)),
               "mlba_batch_blur_fft")
        return bool(u.value), m.value

    def graph_kernels(self):
        k = ctypes.c_int()
        _check(self.lib.mlba_batch_graph_kernels(self.h, ctypes.byref(k)), "mlba_batch_graph_kernels")
        return k.value
