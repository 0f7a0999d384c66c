"""ctypes binding of libnmf.so (include/nmf.h): argument marshalling only.

Every computation runs in the library's CUDA kernels; this module only turns
torch tensors into device pointers and status codes into exceptions. If the
library is missing, `load()` raises: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnmf.so")

NMF_OK, NMF_EINVAL, NMF_ENOMEM, NMF_ECUDA, NMF_ENONFINITE, NMF_ETIMEOUT, NMF_EUNSUPPORTED, NMF_ENOTREADY = range(8)
FP64, FP32, TF32, BF16 = range(4)
W_FIRST, H_FIRST, ORDER_AUTO = range(3)
PRECISIONS = {"fp64": FP64, "fp32": FP32, "tf32": TF32, "bf16": BF16}
ORDERS = {"W": W_FIRST, "H": H_FIRST, "auto": ORDER_AUTO}

EXPORTS = [
    "nmf_create", "nmf_batch_create", "nmf_set_options", "nmf_set_floor", "nmf_autotune",
    "nmf_set_subiterations", "nmf_set_dense",
    "nmf_set_csr", "nmf_set_factors", "nmf_batch_set_packed", "nmf_step_joint",
    "nmf_step_alternating", "nmf_loss", "nmf_grad", "nmf_kkt", "nmf_batch_get_losses",
    "nmf_get_status", "nmf_step_joint_host", "nmf_set_timing", "nmf_get_timing", "nmf_reset_timing",
    "nmf_loss_noalloc", "nmf_set_barrier_test", "nmf_step_joint_async", "nmf_step_alternating_async", "nmf_destroy", "nmf_status_string",
]

_lib = None


class NMFError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {status_string(code)}")


def status_string(code):
    return load().nmf_status_string(code).decode()


def _declare(lib):
    P = ctypes.c_void_p
    I64, I32, D = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    PD = ctypes.POINTER(ctypes.c_double)
    sigs = {
        "nmf_create": [I64, I64, I32, D, ctypes.POINTER(P)],
        "nmf_batch_create": [I32, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I32), D,
                             ctypes.POINTER(P)],
        "nmf_set_options": [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, D, ctypes.c_int, P],
        "nmf_set_floor": [P, D],
        "nmf_autotune": [P, I32, ctypes.POINTER(I32)],
        "nmf_set_subiterations": [P, I32],
        "nmf_set_dense": [P, P, I64],
        "nmf_set_csr": [P, I64, P, P, P],
        "nmf_set_factors": [P, P, P],
        "nmf_batch_set_packed": [P, P, P, P],
        "nmf_step_joint": [P, I32, PD],
        "nmf_step_alternating": [P, I32, PD],
        "nmf_step_joint_async": [P, I32, P],
        "nmf_step_alternating_async": [P, I32, P],
        "nmf_loss": [P, PD],
        "nmf_grad": [P, P, P, PD],
        "nmf_kkt": [P, PD, PD],
        "nmf_batch_get_losses": [P, PD],
        "nmf_get_status": [P],
        "nmf_step_joint_host": [P, P, P, P, I32, PD],
        "nmf_set_timing": [P, ctypes.c_int],
        "nmf_get_timing": [P, I32, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(I64), PD],
        "nmf_reset_timing": [P],
        "nmf_loss_noalloc": [I64, I64, I32, D, D, ctypes.c_int, P, I64, P, P, P, P],
        "nmf_set_barrier_test": [P, I64, I32],
    }
    for name, args in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.nmf_destroy.argtypes = [P]
    lib.nmf_destroy.restype = None
    lib.nmf_status_string.argtypes = [ctypes.c_int]
    lib.nmf_status_string.restype = ctypes.c_char_p


def load(path: str | None = None):
    """Loads libnmf.so (built by build.py); raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libnmf.so not built ({p}); run `python -m paper_2106_15214_gb300.build`")
    lib = ctypes.CDLL(p)
    _declare(lib)
    _lib = lib
    return lib


def check(code, where):
    if code != NMF_OK:
        raise NMFError(code, where)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dtype_for(precision):
    import torch
    return torch.float64 if precision == FP64 else torch.float32


def loss_noalloc(V, W, H, beta, kappa=0.0, out=None, stream=None):
    """nmf_loss_noalloc: the objective into a device double, with no device
    allocation inside the library (for callers that cannot call cudaMalloc).
    V, W, H are CUDA tensors (float64 or float32, row-major); `out` is a
    one-element float64 CUDA tensor (allocated here by torch if not given).
    Asynchronous on the stream; returns `out`."""
    import torch
    lib = load()
    for t, nm in ((V, "V"), (W, "W"), (H, "H")):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dim() == 2):
            raise TypeError(f"{nm} must be a 2-D CUDA tensor")
        if t.dtype not in (torch.float64, torch.float32) or t.dtype != V.dtype:
            raise TypeError(f"V, W and H must share one dtype, float64 or float32 (got {nm}: {t.dtype})")
        if t.device != V.device:
            raise ValueError("V, W and H must be on one device")
    F, N = V.shape
    K = W.shape[1]
    if V.stride(1) != 1 or V.stride(0) < N:
        raise ValueError("V must be row-major with unit column stride")
    if tuple(W.shape) != (F, K) or tuple(H.shape) != (K, N):
        raise ValueError(f"W must be {F} x K and H K x {N}")
    if not (W.is_contiguous() and H.is_contiguous()):
        raise ValueError("W and H must be contiguous")
    if out is not None and not (out.is_cuda and out.dtype == torch.float64 and out.numel() >= 1):
        raise TypeError("out must be a float64 CUDA tensor")
    prec = FP64 if V.dtype == torch.float64 else FP32
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=V.device)
    s = ctypes.c_void_p(stream) if stream is not None else _stream()
    check(lib.nmf_loss_noalloc(F, N, K, float(beta), float(kappa), prec, _ptr(V), V.stride(0), _ptr(W),
                               _ptr(H), _ptr(out), s), "nmf_loss_noalloc")
    return out


class NMF:
    """One beta-NMF problem on the GPU. V, W, H are CUDA tensors (row-major,
    contiguous); W and H are updated in place by the step calls."""

    def __init__(self, F, N, K, beta, precision="fp32", order="W", normalize=True, kappa=0.0,
                 L=1, stream=None, floor=None):
        lib = load()
        self._lib = lib
        self.F, self.N, self.K, self.beta = int(F), int(N), int(K), float(beta)
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.order = ORDERS[order] if isinstance(order, str) else int(order)
        self.normalize = bool(normalize)
        self.kappa = float(kappa)
        self._ctx = ctypes.c_void_p()
        check(lib.nmf_create(self.F, self.N, self.K, self.beta, ctypes.byref(self._ctx)), "nmf_create")
        self._stream = stream
        self.set_options(stream)
        if L != 1:
            check(lib.nmf_set_subiterations(self._ctx, int(L)), "nmf_set_subiterations")
        if floor is not None:
            self.set_floor(floor)
        self._keep = []

    def autotune(self, trials=3):
        """nmf_autotune (FP64 / FP32 contexts): returns the chosen chunk cap."""
        cap = ctypes.c_int32(0)
        check(self._lib.nmf_autotune(self._ctx, int(trials), ctypes.byref(cap)), "nmf_autotune")
        return cap.value

    def set_floor(self, eps):
        """Clamp every update to eps (nmf_set_floor); eps < 0 restores the default."""
        check(self._lib.nmf_set_floor(self._ctx, float(eps)), "nmf_set_floor")

    def set_options(self, stream=None):
        s = ctypes.c_void_p(stream) if stream is not None else _stream()
        check(self._lib.nmf_set_options(self._ctx, self.precision, self.order, int(self.normalize),
                                        self.kappa, 1, s), "nmf_set_options")

    @property
    def dtype(self):
        return _dtype_for(self.precision)

    def _check_tensor(self, t, shape, name):
        import torch
        if not (isinstance(t, torch.Tensor) and t.is_cuda):
            raise TypeError(f"{name} must be a CUDA tensor")
        if t.dtype != self.dtype:
            raise TypeError(f"{name} must be {self.dtype} for this precision, got {t.dtype}")
        if tuple(t.shape) != shape:
            raise ValueError(f"{name} must have shape {shape}, got {tuple(t.shape)}")

    def set_dense(self, V):
        self._check_tensor(V, (self.F, V.shape[1]), "V")
        if V.stride(1) != 1 or V.shape[1] != self.N:
            raise ValueError("V must be F x N with unit column stride")
        self._V = V
        check(self._lib.nmf_set_dense(self._ctx, _ptr(V), V.stride(0)), "nmf_set_dense")

    def set_csr(self, rowptr, col, val):
        import torch
        for t, dt in ((rowptr, torch.int32), (col, torch.int32), (val, torch.float32)):
            if not (t.is_cuda and t.dtype == dt and t.is_contiguous()):
                raise TypeError("CSR arrays must be contiguous CUDA tensors (int32, int32, float32)")
        self._csr = (rowptr, col, val)
        check(self._lib.nmf_set_csr(self._ctx, int(col.numel()), _ptr(rowptr), _ptr(col), _ptr(val)),
              "nmf_set_csr")

    def set_factors(self, W, H):
        self._check_tensor(W, (self.F, self.K), "W")
        self._check_tensor(H, (self.K, self.N), "H")
        if not (W.is_contiguous() and H.is_contiguous()):
            raise ValueError("W and H must be contiguous")
        self.W, self.H = W, H
        check(self._lib.nmf_set_factors(self._ctx, _ptr(W), _ptr(H)), "nmf_set_factors")

    def step_joint(self, iters=1, want_loss=True):
        loss = ctypes.c_double(float("nan"))
        check(self._lib.nmf_step_joint(self._ctx, int(iters), ctypes.byref(loss) if want_loss else None),
              "nmf_step_joint")
        return loss.value if want_loss else None

    def step_alternating(self, iters=1, want_loss=True):
        loss = ctypes.c_double(float("nan"))
        check(self._lib.nmf_step_alternating(self._ctx, int(iters),
                                             ctypes.byref(loss) if want_loss else None),
              "nmf_step_alternating")
        return loss.value if want_loss else None

    def step_joint_async(self, loss_dev, iters=1):
        """Asynchronous JMM step; the loss goes to the device tensor loss_dev (float64)."""
        check(self._lib.nmf_step_joint_async(self._ctx, int(iters), _ptr(loss_dev)), "nmf_step_joint_async")

    def step_alternating_async(self, loss_dev, iters=1):
        check(self._lib.nmf_step_alternating_async(self._ctx, int(iters), _ptr(loss_dev)),
              "nmf_step_alternating_async")

    def step_joint_host(self, V_host, W_host, H_host, iters=1):
        """Host (ideally pinned) CPU tensors in, W_host/H_host updated in place."""
        loss = ctypes.c_double(float("nan"))
        check(self._lib.nmf_step_joint_host(self._ctx, _ptr(V_host), _ptr(W_host), _ptr(H_host),
                                            int(iters), ctypes.byref(loss)), "nmf_step_joint_host")
        return loss.value

    def loss(self):
        out = ctypes.c_double()
        check(self._lib.nmf_loss(self._ctx, ctypes.byref(out)), "nmf_loss")
        return out.value

    def grad(self, gW, gH, want_loss=False):
        loss = ctypes.c_double(float("nan"))
        check(self._lib.nmf_grad(self._ctx, _ptr(gW), _ptr(gH), ctypes.byref(loss) if want_loss else None),
              "nmf_grad")
        return loss.value if want_loss else None

    def kkt(self):
        rw, rh = ctypes.c_double(), ctypes.c_double()
        check(self._lib.nmf_kkt(self._ctx, ctypes.byref(rw), ctypes.byref(rh)), "nmf_kkt")
        return rw.value, rh.value

    def status(self):
        return self._lib.nmf_get_status(self._ctx)

    def close(self):
        if self._ctx:
            self._lib.nmf_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchedNMF:
    """Many independent problems; V, W, H packed back to back (see nmf_batch_set_packed)."""

    def __init__(self, shapes, beta, precision="fp32", order="W", normalize=True, stream=None):
        lib = load()
        self._lib = lib
        self.shapes = [(int(f), int(n), int(k)) for f, n, k in shapes]
        c = len(self.shapes)
        Fa = (ctypes.c_int64 * c)(*[s[0] for s in self.shapes])
        Na = (ctypes.c_int64 * c)(*[s[1] for s in self.shapes])
        Ka = (ctypes.c_int32 * c)(*[s[2] for s in self.shapes])
        self._ctx = ctypes.c_void_p()
        check(lib.nmf_batch_create(c, Fa, Na, Ka, float(beta), ctypes.byref(self._ctx)), "nmf_batch_create")
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.order = ORDERS[order] if isinstance(order, str) else int(order)
        s = ctypes.c_void_p(stream) if stream is not None else _stream()
        check(lib.nmf_set_options(self._ctx, self.precision, self.order, int(normalize), 0.0, 1, s),
              "nmf_set_options")

    def autotune(self, trials=3):
        """nmf_autotune: time each chunk cap over `trials` steps, keep the fastest; returns it."""
        cap = ctypes.c_int32(0)
        check(self._lib.nmf_autotune(self._ctx, int(trials), ctypes.byref(cap)), "nmf_autotune")
        return cap.value

    def set_packed(self, Vp, Wp, Hp):
        self._keep = (Vp, Wp, Hp)
        check(self._lib.nmf_batch_set_packed(self._ctx, _ptr(Vp), _ptr(Wp), _ptr(Hp)), "nmf_batch_set_packed")

    def step_joint(self, iters=1, want_loss=True):
        loss = ctypes.c_double(float("nan"))
        check(self._lib.nmf_step_joint(self._ctx, int(iters), ctypes.byref(loss) if want_loss else None),
              "nmf_step_joint")
        return loss.value if want_loss else None

    def step_alternating(self, iters=1, want_loss=True):
        loss = ctypes.c_double(float("nan"))
        check(self._lib.nmf_step_alternating(self._ctx, int(iters), ctypes.byref(loss) if want_loss else None),
              "nmf_step_alternating")
        return loss.value if want_loss else None

    def losses(self):
        out = (ctypes.c_double * len(self.shapes))()
        check(self._lib.nmf_batch_get_losses(self._ctx, out), "nmf_batch_get_losses")
        return list(out)

    def close(self):
        if self._ctx:
            self._lib.nmf_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_beta_divergence_fn = None
_grad_contexts = {}


def _grad_context(F, N, K, beta, kappa, dtype, device, fused=False):
    """A context per (shape, beta, kappa, precision, device, stream), kept for
    reuse by the autograd function (contexts own device scratch: creating one
    per call would allocate every time). fused (float32 only): a BF16 context,
    whose nmf_grad is the fused single-read sweep's adjoint mode."""
    import torch
    prec = "fp64" if dtype == torch.float64 else ("bf16" if fused else "fp32")
    stream = torch.cuda.current_stream(device).cuda_stream
    key = (F, N, K, float(beta), float(kappa), prec, device.index, stream)
    m = _grad_contexts.get(key)
    if m is None:
        if len(_grad_contexts) >= 16:
            _grad_contexts.pop(next(iter(_grad_contexts))).close()
        m = NMF(F, N, K, float(beta), precision=prec, order="H" if prec == "bf16" else "W", normalize=False,
                kappa=float(kappa), stream=stream)
        _grad_contexts[key] = m
    return m


def _beta_divergence_function():
    """The torch.autograd.Function, made on first use (torch is imported lazily)."""
    global _beta_divergence_fn
    if _beta_divergence_fn is not None:
        return _beta_divergence_fn
    import torch

    class BetaDivergence(torch.autograd.Function):
        """D_beta(V + kappa | WH + kappa) (eq. obj_fct, eq. beta-div) with the
        gradient of nmf_grad: grad_W = [(WH)^(beta-2) . (WH - V)] H^T and
        grad_H = W^T [(WH)^(beta-2) . (WH - V)], the difference of the MU
        ratio's denominator and numerator (Sec. 4.1.5). Forward evaluates the
        objective only (stream-ordered, into device memory, when the problem
        fits nmf_loss_noalloc's scratch); backward runs one nmf_grad pass
        over the saved tensors, recomputing the product tile by tile. V is not
        differentiated. Contexts are cached per shape and reused."""

        @staticmethod
        def forward(ctx, V, W, H, beta, kappa, fused):
            F, K = W.shape
            N = H.shape[1]
            Vc, Wc, Hc = V.detach().contiguous(), W.detach().contiguous(), H.detach().contiguous()
            if ((F + 31) // 32) * ((N + 31) // 32) <= 65536:
                loss = loss_noalloc(Vc, Wc, Hc, beta, kappa)[0].to(W.dtype)
            else:
                m = _grad_context(F, N, K, beta, kappa, W.dtype, W.device)
                m.set_dense(Vc)
                m.set_factors(Wc, Hc)
                loss = torch.tensor(m.loss(), dtype=W.dtype, device=W.device)
            ctx.save_for_backward(Vc, Wc, Hc)
            ctx.beta, ctx.kappa, ctx.fused = float(beta), float(kappa), bool(fused) and W.dtype == torch.float32
            return loss

        @staticmethod
        def backward(ctx, g):
            Vc, Wc, Hc = ctx.saved_tensors
            F, K = Wc.shape
            N = Hc.shape[1]
            m = _grad_context(F, N, K, ctx.beta, ctx.kappa, Wc.dtype, Wc.device, ctx.fused)
            m.set_dense(Vc)
            m.set_factors(Wc, Hc)
            gW, gH = torch.empty_like(Wc), torch.empty_like(Hc)
            m.grad(gW, gH)                 # asynchronous: no host round trip
            return None, g * gW, g * gH, None, None, None

    _beta_divergence_fn = BetaDivergence
    return BetaDivergence


def beta_divergence(V, W, H, beta, kappa=0.0, fused=False):
    """Differentiable D_beta(V + kappa | WH + kappa) of CUDA tensors V (F x N),
    W (F x K), H (K x N), float32 or float64; backward gives grad_W, grad_H
    (nmf_grad). fused=True (float32): the gradients come from the fused
    single-read sweep's adjoint mode (bf16 contractions, ~1e-2 relative error
    of each term; K <= 32, F <= 1024, else the FP32 sweeps). Returns a 0-d
    tensor on W's device."""
    return _beta_divergence_function().apply(V, W, H, beta, kappa, fused)
