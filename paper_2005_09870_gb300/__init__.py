"""Python binding of libpcwave (the C-ABI in include/pcwave.h).

Argument marshalling only: every step of the assembly, the apply and the backward runs in
the CUDA kernels of libpcwave.so.  PyTorch provides device memory and streams.  There is no
CPU fallback: importing this package fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpcwave.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libpcwave.so is not built ({LIB_PATH}); run __graft_entry__.build() "
                      "or python paper_2005_09870_gb300/build.py")
_lib = ctypes.CDLL(LIB_PATH)

PC_DAUBECHIES, PC_SYMMLET = 0, 1
PC_OK, PC_ERR_INVALID_ARG, PC_ERR_UNSUPPORTED, PC_ERR_OOM, PC_ERR_CUDA, PC_ERR_TIMEOUT, \
    PC_ERR_NOT_ASSEMBLED, PC_ERR_DEVICE = range(8)
PC_ORDER_MULT_THEN_CONV, PC_ORDER_CONV_THEN_MULT = 0, 1
PC_FP32, PC_FP64 = 0, 1
PC_ALG1_SCHUR, PC_ALG1_HARD = 0, 1
PC_ALG1_DISCARD = 1
_STATUS = ["PC_OK", "PC_ERR_INVALID_ARG", "PC_ERR_UNSUPPORTED", "PC_ERR_OOM", "PC_ERR_CUDA",
           "PC_ERR_TIMEOUT", "PC_ERR_NOT_ASSEMBLED", "PC_ERR_DEVICE"]


class pc_desc(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int) for f in
                ("dim", "n", "levels", "delta", "m", "radius", "gap", "order", "precision", "store_bf16",
                 "family")]


class PCError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS[status] if 0 <= status < len(_STATUS) else status}: {msg}")
        self.status = status


_H = ctypes.c_void_p
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I64P = ctypes.POINTER(ctypes.c_int64)
_DP = ctypes.POINTER(pc_desc)

_sig = {
    "pc_plan_check": ([_DP], ctypes.c_int),
    "pc_plan_nnz": ([_DP, _I64P], ctypes.c_int),
    "pc_plan_row": ([_DP, _I64, _I64P, _I64P], ctypes.c_int),
    "pc_create": ([_DP, _P, _P, _P, ctypes.POINTER(_H)], ctypes.c_int),
    "pc_set_params": ([_H, _P, _P, _P], ctypes.c_int),
    "pc_destroy": ([_H], None),
    "pc_assemble": ([_H, _P], ctypes.c_int),
    "pc_apply": ([_H, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P], ctypes.c_int),
    "pc_assemble_stage": ([_H, ctypes.c_int, _P], ctypes.c_int),
    "pc_backward": ([_H, _P, _P, _P, _P], ctypes.c_int),
    "pc_launch_counter": ([], ctypes.c_int64),
    "pc_backward_noalloc": ([_H, _P, _P, _P, _P], ctypes.c_int),
    "pc_batch_assemble": ([ctypes.POINTER(_H), ctypes.c_int, _P], ctypes.c_int),
    "pc_batch_create": ([ctypes.POINTER(_H), ctypes.c_int, _P, ctypes.POINTER(_H)], ctypes.c_int),
    "pc_batch_run": ([_H, _P], ctypes.c_int),
    "pc_batch_info": ([_H, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "pc_batch_destroy": ([_H], None),
    "pc_autotune": ([_H, _P], ctypes.c_int),
    "pc_info": ([_H, _I64P, _I64P], ctypes.c_int),
    "pc_theta": ([_H, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P)], ctypes.c_int),
    "pc_lookup": ([_H, _I64, _I64P, _I64P, _I64P], ctypes.c_int),
    "pc_sync": ([_H, _P], ctypes.c_int),
    "pc_last_error": ([_H], ctypes.c_char_p),
    "pc_apply_adjoint": ([_H, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P], ctypes.c_int),
    "pc_jacobi": ([_H, _P, _P], ctypes.c_int),
    "pc_power_norm": ([_H, _P, ctypes.c_int, ctypes.POINTER(ctypes.c_double), _P], ctypes.c_int),
    "pc_fista": ([_H, _P, _P, _P, _P, ctypes.c_int, ctypes.c_double, _P], ctypes.c_int),
    "pc_filter_taps": ([ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "pc_export": ([_H, _I64P, _I64P, ctypes.POINTER(ctypes.c_double), _P], ctypes.c_int),
    "pc_svir_expansion": ([_P, _I64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, _P,
                           ctypes.POINTER(ctypes.c_double), _P], ctypes.c_int),
    "pc_alg1_create": ([_DP, _P, _P, ctypes.c_double, ctypes.c_int, ctypes.c_int, _P, ctypes.POINTER(_H)],
                       ctypes.c_int),
    "pc_alg1_info": ([_H, _I64P, ctypes.POINTER(ctypes.c_double), _I64P, ctypes.POINTER(ctypes.c_double)],
                     ctypes.c_int),
    "pc_alg1_export": ([_H, _I64P, _I64P, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "pc_alg1_row": ([_H, _I64, _I64P, ctypes.POINTER(ctypes.c_double), _I64P], ctypes.c_int),
    "pc_alg1_destroy": ([_H], None),
}
for _name, (_args, _ret) in _sig.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _ret


def _check(st, h=None):
    if st != PC_OK:
        raise PCError(st, _lib.pc_last_error(h).decode())


def make_desc(dim, n, levels, delta, m, radius, gap=2, order=0, precision=PC_FP32, store_bf16=0,
              family=0) -> pc_desc:
    return pc_desc(dim, n, levels, delta, m, radius, gap, order, precision, int(store_bf16), int(family))


def desc_of(op, precision=PC_FP32, store_bf16=0) -> pc_desc:
    """Descriptor for a pc_inputs.Operator-like object (fields d, n, levels, delta, m, r, gap,
    order and optionally family)."""
    return make_desc(op.d, op.n, op.levels, op.delta, op.m, op.r, op.gap, op.order, precision, store_bf16,
                     getattr(op, "family", 0))


def pc_export(h, nnz, N, stream=None):
    """Theta as host CSR arrays (row_ptr, cols, vals), ascending columns per row."""
    import numpy as np
    row_ptr = np.zeros(N + 1, dtype=np.int64)
    cols = np.zeros(nnz, dtype=np.int64)
    vals = np.zeros(nnz, dtype=np.float64)
    _check(_lib.pc_export(h, row_ptr.ctypes.data_as(_I64P), cols.ctypes.data_as(_I64P),
                          vals.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _stream(stream)), h)
    return row_ptr, cols, vals


def pc_svir_expansion(S, m, omega, power_iters=2, stream=None):
    """Rank-m product-convolution expansion of an SVIR S (N x K, FP32 CUDA tensor) by randomized
    SVD with the test matrix omega (K x l, FP32 CUDA tensor): returns (u (m x K), v (m x N),
    singular values of the projected matrix (l,), numpy)."""
    t = _torch()
    N, K = S.shape
    l = omega.shape[1]
    u = t.empty((m, K), dtype=t.float32, device=S.device)
    v = t.empty((m, N), dtype=t.float32, device=S.device)
    sing = np.zeros(l)
    _check(_lib.pc_svir_expansion(_ptr(S), int(N), int(K), int(m), int(l), int(power_iters), _ptr(omega), _ptr(u),
                                  _ptr(v), sing.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _stream(stream)))
    return u, v, sing


class PCAlg1:
    """Thresholded Algorithm 1 (pc_alg1_create): Theta~ = sum_k A~_k B_k, built on the device;
    rule PC_ALG1_SCHUR (within eta of Theta in the 2-norm) or PC_ALG1_HARD (tau_k = eps_k).
    u (m x K) and v (m x N) are FP64 (numpy or CUDA tensors); desc as for pc_create with
    order 0.  Attributes: nnz, tau (m,), kept (m,), stage_ms (4,)."""

    def __init__(self, desc: pc_desc, u, v, eta: float, rule: int = 0, flags: int = 0, stream=None):
        self.h = _H()
        self.m = int(desc.m)
        self.N = int(desc.n) ** int(desc.dim)
        self._keep = []
        _check(_lib.pc_alg1_create(ctypes.byref(desc), self._f64(u), self._f64(v), float(eta), int(rule), int(flags),
                                   _stream(stream), ctypes.byref(self.h)))
        self._keep = []
        nnz = ctypes.c_int64()
        self.tau = np.zeros(self.m)
        self.kept = np.zeros(self.m, dtype=np.int64)
        self.stage_ms = np.zeros(4)
        _check(_lib.pc_alg1_info(self.h, ctypes.byref(nnz), self.tau.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                 self.kept.ctypes.data_as(_I64P),
                                 self.stage_ms.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        self.nnz = int(nnz.value)

    def _f64(self, a):
        if hasattr(a, "is_cuda"):
            t = _torch()
            a = a.to(t.float64).contiguous()
            self._keep.append(a)
            return _ptr(a) if a.is_cuda else a.data_ptr()
        a = np.ascontiguousarray(a, dtype=np.float64)
        self._keep.append(a)
        return a.ctypes.data

    def export(self):
        """Host CSR (row_ptr, cols, vals) in canonical row order."""
        row_ptr = np.zeros(self.N + 1, dtype=np.int64)
        cols = np.zeros(max(self.nnz, 1), dtype=np.int64)
        vals = np.zeros(max(self.nnz, 1), dtype=np.float64)
        _check(_lib.pc_alg1_export(self.h, row_ptr.ctypes.data_as(_I64P), cols.ctypes.data_as(_I64P),
                                   vals.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return row_ptr, cols[:self.nnz], vals[:self.nnz]

    def row(self, mu: int):
        """Row mu of Theta~: (columns, values), storage order."""
        cnt = ctypes.c_int64(0)
        _check(_lib.pc_alg1_row(self.h, int(mu), None, None, ctypes.byref(cnt)))
        cols = np.zeros(max(cnt.value, 1), dtype=np.int64)
        vals = np.zeros(max(cnt.value, 1))
        _check(_lib.pc_alg1_row(self.h, int(mu), cols.ctypes.data_as(_I64P),
                                vals.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(cnt)))
        return cols[:cnt.value], vals[:cnt.value]

    def dense(self):
        """Theta~ as a dense N x N numpy array (small N)."""
        row_ptr, cols, vals = self.export()
        T = np.zeros((self.N, self.N))
        rows = np.repeat(np.arange(self.N), np.diff(row_ptr))
        np.add.at(T, (rows, cols), vals)
        return T

    def close(self):
        if self.h:
            _lib.pc_alg1_destroy(self.h)
            self.h = _H()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pc_filter_taps(family: int, delta: int):
    """Host-only: the library's low-pass taps for a family (0 Daubechies, 1 Symmlet) and order."""
    import numpy as np
    h = np.zeros(2 * int(delta))
    _check(_lib.pc_filter_taps(int(family), int(delta), h.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return h


# ----------------------------------------------------------------- host-only planning
def pc_plan_check(desc: pc_desc) -> None:
    _check(_lib.pc_plan_check(ctypes.byref(desc)))


def pc_plan_nnz(desc: pc_desc) -> int:
    nnz = ctypes.c_int64()
    _check(_lib.pc_plan_nnz(ctypes.byref(desc), ctypes.byref(nnz)))
    return nnz.value


def pc_plan_row(desc: pc_desc, row: int) -> np.ndarray:
    cnt = ctypes.c_int64()
    _check(_lib.pc_plan_row(ctypes.byref(desc), int(row), None, ctypes.byref(cnt)))
    cols = np.zeros(cnt.value, dtype=np.int64)
    _check(_lib.pc_plan_row(ctypes.byref(desc), int(row), cols.ctypes.data_as(_I64P), ctypes.byref(cnt)))
    return cols


# ----------------------------------------------------------------- device helpers
def _torch():
    import torch
    return torch


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(_torch().cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class _DevArray:
    """A view of library-owned device memory for torch.as_tensor (no copy)."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3}


def _ptr(t):
    """Device (or host) address of a torch tensor / numpy array."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(t.data_ptr())
    return ctypes.c_void_p(t.ctypes.data)


# ----------------------------------------------------------------- C-ABI with the same names
def pc_create(desc: pc_desc, u, v, stream=None) -> int:
    h = _H()
    _check(_lib.pc_create(ctypes.byref(desc), _ptr(u), _ptr(v), _stream(stream), ctypes.byref(h)))
    return h.value


def pc_set_params(h, u, v, stream=None):
    _check(_lib.pc_set_params(h, _ptr(u), _ptr(v), _stream(stream)), h)


def pc_destroy(h):
    _lib.pc_destroy(h)


def pc_assemble(h, stream=None):
    _check(_lib.pc_assemble(h, _stream(stream)), h)


def pc_assemble_stage(h, stage, stream=None):
    _check(_lib.pc_assemble_stage(h, int(stage), _stream(stream)), h)


def pc_launch_counter() -> int:
    return int(_lib.pc_launch_counter())


def pc_apply(h, x, y, nrhs=None, ldx=None, ldy=None, stream=None):
    if nrhs is None:
        nrhs = 1 if x.dim() == 1 else x.shape[1]
    ldx = nrhs if ldx is None else ldx
    ldy = nrhs if ldy is None else ldy
    _check(_lib.pc_apply(h, _ptr(x), _ptr(y), nrhs, ldx, ldy, _stream(stream)), h)


def pc_apply_adjoint(h, x, y, nrhs=None, ldx=None, ldy=None, stream=None):
    if nrhs is None:
        nrhs = 1 if x.dim() == 1 else x.shape[1]
    ldx = nrhs if ldx is None else ldx
    ldy = nrhs if ldy is None else ldy
    _check(_lib.pc_apply_adjoint(h, _ptr(x), _ptr(y), nrhs, ldx, ldy, _stream(stream)), h)


def pc_jacobi(h, diag, stream=None):
    _check(_lib.pc_jacobi(h, _ptr(diag), _stream(stream)), h)


def pc_power_norm(h, sigma=None, iters=50, stream=None) -> float:
    out = ctypes.c_double(0.0)
    _check(_lib.pc_power_norm(h, _ptr(sigma), int(iters), ctypes.byref(out), _stream(stream)), h)
    return out.value


def pc_fista(h, z0, w, sigma, z, iters, tau, stream=None):
    _check(_lib.pc_fista(h, _ptr(z0), _ptr(w), _ptr(sigma), _ptr(z), int(iters), float(tau), _stream(stream)), h)


def pc_backward(h, dtheta, du, dv, stream=None):
    _check(_lib.pc_backward(h, _ptr(dtheta), _ptr(du), _ptr(dv), _stream(stream)), h)


def pc_backward_noalloc(h, dtheta, du, dv, stream=None):
    """pc_backward without any device allocation (static library scratch; see pcwave.h)."""
    _check(_lib.pc_backward_noalloc(h, _ptr(dtheta), _ptr(du), _ptr(dv), _stream(stream)), h)


def pc_batch_assemble(handles, stream=None):
    arr = (_H * len(handles))(*handles)
    first = handles[0] if handles else None
    _check(_lib.pc_batch_assemble(arr, len(handles), _stream(stream)), first)


def pc_batch_create(handles, stream=None) -> int:
    arr = (_H * len(handles))(*handles)
    b = _H()
    _check(_lib.pc_batch_create(arr, len(handles), _stream(stream), ctypes.byref(b)))
    return b.value


def pc_batch_run(b, stream=None):
    _check(_lib.pc_batch_run(b, _stream(stream)))


def pc_batch_info(b):
    it, k = ctypes.c_int(), ctypes.c_int()
    _check(_lib.pc_batch_info(b, ctypes.byref(it), ctypes.byref(k)))
    return it.value, k.value


def pc_batch_destroy(b):
    _lib.pc_batch_destroy(b)


def pc_autotune(h, stream=None):
    _check(_lib.pc_autotune(h, _stream(stream)), h)


def pc_info(h):
    nnz, by = ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.pc_info(h, ctypes.byref(nnz), ctypes.byref(by)), h)
    return nnz.value, by.value


def pc_theta(h):
    a, b, c = _P(), _P(), _P()
    _check(_lib.pc_theta(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), h)
    return a.value, b.value, c.value


def pc_lookup(h, mu, lam) -> np.ndarray:
    mu = np.ascontiguousarray(mu, dtype=np.int64)
    lam = np.ascontiguousarray(lam, dtype=np.int64)
    pos = np.zeros(mu.size, dtype=np.int64)
    _check(_lib.pc_lookup(h, mu.size, mu.ctypes.data_as(_I64P), lam.ctypes.data_as(_I64P),
                          pos.ctypes.data_as(_I64P)), h)
    return pos


def pc_sync(h, stream=None):
    _check(_lib.pc_sync(h, _stream(stream)), h)


def pc_last_error(h=None) -> str:
    return _lib.pc_last_error(h).decode()


# ----------------------------------------------------------------- convenience object
class PCOperator:
    """One operator: owns a libpcwave handle.  u, v may be torch tensors (CUDA or CPU) or
    numpy arrays of the precision's dtype."""

    def __init__(self, desc: pc_desc, u, v, stream=None):
        self.desc = desc
        self._keep = (u, v)
        self.h = pc_create(desc, u, v, stream)
        self.nnz, self.device_bytes = pc_info(self.h)
        self.N = desc.n ** desc.dim

    @property
    def dtype(self):
        t = _torch()
        return t.float64 if self.desc.precision == PC_FP64 else t.float32

    def assemble(self, stream=None):
        pc_assemble(self.h, stream)

    def values(self):
        """torch view (no copy) of the stored values on the device."""
        t = _torch()
        vals, _, _ = pc_theta(self.h)
        ts = "<f8" if self.desc.precision == PC_FP64 else "<f4"
        return t.as_tensor(_DevArray(vals, (self.nnz,), ts), device="cuda")

    def values_bf16(self):
        t = _torch()
        _, v16, _ = pc_theta(self.h)
        if not v16:
            return None
        raw = t.as_tensor(_DevArray(v16, (self.nnz,), "<i2"), device="cuda")
        return raw.view(t.bfloat16)

    def apply(self, x, stream=None):
        t = _torch()
        y = t.empty_like(x)
        pc_apply(self.h, x, y, stream=stream)
        return y

    def apply_adjoint(self, x, stream=None):
        t = _torch()
        y = t.empty_like(x)
        pc_apply_adjoint(self.h, x, y, stream=stream)
        return y

    def jacobi(self, stream=None):
        t = _torch()
        d = t.empty(self.N, dtype=self.dtype, device="cuda")
        pc_jacobi(self.h, d, stream)
        return d

    def power_norm(self, sigma=None, iters=50, stream=None) -> float:
        return pc_power_norm(self.h, sigma, iters, stream)

    def fista(self, z0, w, iters, tau, z=None, sigma=None, stream=None):
        """FISTA-W (sigma None) or FISTA-WP iterates from z (zeros when None); returns z."""
        t = _torch()
        z = t.zeros_like(z0) if z is None else z
        if not t.is_tensor(w):
            w = t.full_like(z0, float(w))
        pc_fista(self.h, z0, w, sigma, z, iters, tau, stream)
        return z

    def backward(self, dtheta, stream=None):
        t = _torch()
        K = (2 * self.desc.radius + 1) ** self.desc.dim
        du = t.empty((self.desc.m, K), dtype=self.dtype, device="cuda")
        dv = t.empty((self.desc.m, self.N), dtype=self.dtype, device="cuda")
        pc_backward(self.h, dtheta, du, dv, stream)
        return du, dv

    def export(self, stream=None):
        """(row_ptr, cols, vals) of Theta on the host (CSR, ascending columns)."""
        return pc_export(self.h, self.nnz, self.N, stream)

    def lookup(self, mu, lam):
        return pc_lookup(self.h, mu, lam)

    def sync(self, stream=None):
        pc_sync(self.h, stream)

    def close(self):
        if self.h:
            pc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PCBatch:
    """A captured batch over PCOperator objects (kept alive by the batch)."""

    def __init__(self, operators, stream=None):
        self.operators = list(operators)
        self.b = pc_batch_create([o.h for o in self.operators], stream)
        self.items, self.kernels_per_run = pc_batch_info(self.b)

    def run(self, stream=None):
        pc_batch_run(self.b, stream)

    def close(self):
        if self.b:
            pc_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------- autograd
def theta(u, v, op: "PCOperator"):
    """Differentiable Theta: the stored values (nnz,) as a function of kernels u (m, K) and
    windows v (m, N).  Backward runs pc_backward (the adjoint kernels)."""
    return _theta_fn().apply(u, v, op)


_THETA_FN = None


def _theta_fn():
    global _THETA_FN
    if _THETA_FN is None:
        torch = _torch()

        class PCTheta(torch.autograd.Function):
            @staticmethod
            def forward(ctx, u, v, op):
                u = u.detach().contiguous()
                v = v.detach().contiguous()
                pc_set_params(op.h, u, v)
                op.assemble()
                ctx.op = op
                ctx.save_for_backward(u, v)
                return op.values().clone()

            @staticmethod
            def backward(ctx, g):
                u, v = ctx.saved_tensors
                pc_set_params(ctx.op.h, u, v)
                du, dv = ctx.op.backward(g.contiguous())
                return du, dv, None

        _THETA_FN = PCTheta
    return _THETA_FN
