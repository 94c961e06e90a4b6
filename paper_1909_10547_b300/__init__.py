"""B300-native FK-table convolution (arXiv:1909.10547, Sec. 3).

A thin binding over libfk.so: every function marshals torch tensors (device
memory and the current CUDA stream) into the C ABI of include/fk.h and raises
FKError on a non-zero status.  All arithmetic runs in the library's CUDA
kernels; there is no CPU fallback.

    t  = Table.had(fk, ca, cb, xmap=None, nx_grid=None, precs=("fp64", "fp32"))
    O  = conv(t, F, "fp32")                 # F [R][14][nx_grid] on cuda
    gF = conv_backward(t, F, gO, "fp32")
    cov = Cov(blocks);  chi2_r, gO = chi2(cov, O, D)
    O  = FKConv.apply(F, t, "fp32")         # autograd
    td = Table.dense(fk2d, precs=("bf16x3",))   # the paper's Table 3 product
    O  = dense_conv(td, luminosity(t, F), "bf16x3")
"""
import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import FKError, PRECS

__all__ = ["Table", "conv", "dis_conv", "had_conv", "conv_backward", "saved_size", "saved_buffer", "dense_conv",
           "luminosity", "Cov", "chi2", "chi2_white", "FKConv", "Server", "FKError", "PRECS", "lib_path"]

NFL = 14


def lib_path() -> str:
    return _lib.path()


def _p(x):
    if x is None:
        return None
    if isinstance(x, torch.Tensor):
        return ctypes.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        return x.ctypes.data_as(ctypes.c_void_p)
    return x


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _prec(p):
    if isinstance(p, int):
        return p
    return PRECS[p]


def _io_dtype(prec):
    return torch.float64 if _prec(prec) in (_lib.FK_FP64, _lib.FK_FP64_TC) else torch.float32


def _mask(precs):
    m = 0
    for p in precs:
        m |= 1 << _prec(p)
    return m


class Table:
    """A device-resident FK table (owned by the library)."""

    def __init__(self, handle, kind, ndata, nch, nx, nxg):
        self._h = handle
        self.kind, self.ndata, self.nch, self.nx, self.nxg = kind, ndata, nch, nx, nxg

    @classmethod
    def dis(cls, fk_compact, flav, xmap=None, nx_grid=None, precs=("fp64", "fp32")):
        """fk_compact [ndata][nflav][nx] (host, FP64) for active flavours flav."""
        fk = np.ascontiguousarray(fk_compact, dtype=np.float64)
        nd, nfl, nx = fk.shape
        flav = np.ascontiguousarray(flav, dtype=np.int32)
        xm = None if xmap is None else np.ascontiguousarray(xmap, dtype=np.int32)
        nxg = nx if nx_grid is None else int(nx_grid)
        h = ctypes.c_void_p()
        _lib.call("fk_table_create_dis", _p(fk), nd, _p(flav), nfl, nx, _p(xm), nxg, _mask(precs),
                  ctypes.byref(h))
        return cls(h, 0, nd, nfl, nx, nxg)

    @classmethod
    def had(cls, fk, ca, cb, xmap=None, nx_grid=None, precs=("fp64", "fp32"), form=None):
        """fk [ndata][nc][nx][nx] (host, FP64); channel c = (ca[c], cb[c]).
        form: None (the library's choice), "factored" or "lumi" (the
        reduced-mode forward's formulation, FK_TABLE_FACTORED / FK_TABLE_LUMI)."""
        fk = np.ascontiguousarray(fk, dtype=np.float64)
        nd, nc, nx, _ = fk.shape
        ca = np.ascontiguousarray(ca, dtype=np.int32)
        cb = np.ascontiguousarray(cb, dtype=np.int32)
        xm = None if xmap is None else np.ascontiguousarray(xmap, dtype=np.int32)
        nxg = nx if nx_grid is None else int(nx_grid)
        h = ctypes.c_void_p()
        mask = _mask(precs) | {None: 0, "factored": _lib.FK_TABLE_FACTORED, "lumi": _lib.FK_TABLE_LUMI}[form]
        _lib.call("fk_table_create_had", _p(fk), nd, _p(ca), _p(cb), nc, nx, _p(xm), nxg,
                  mask, ctypes.byref(h))
        return cls(h, 1, nd, nc, nx, nxg)

    @classmethod
    def dense(cls, fk, precs=("fp64", "fp32")):
        """fk [ndata][K] (host, FP64): the flattened table of the dense product
        the paper times in Table 3 (kind 2)."""
        fk = np.ascontiguousarray(fk, dtype=np.float64)
        nd, K = fk.shape
        h = ctypes.c_void_p()
        _lib.call("fk_table_create_dense", _p(fk), nd, K, _mask(precs), ctypes.byref(h))
        t = cls(h, 2, nd, 0, 0, 0)
        t.K = K
        return t

    @classmethod
    def from_workload(cls, t, precs=("fp64", "fp32"), form=None):
        """Builds a device table from a workloads.DisTable / HadTable (form:
        see had(); hadronic tables only)."""
        if hasattr(t, "ca"):
            return cls.had(t.fk, t.ca, t.cb, t.xmap, t.nxg, precs, form)
        if form is not None:
            raise ValueError("form applies to hadronic tables")
        return cls.dis(t.compact(), t.flav, t.xmap, t.nxg, precs)

    def device_bytes(self) -> int:
        n = ctypes.c_size_t()
        _lib.call("fk_table_info", self._h, None, None, None, None, None, None, ctypes.byref(n))
        return n.value

    @property
    def lumi(self) -> bool:
        """True when the reduced-mode forward uses the dense formulation with
        the PDF matrix formed in shared memory (FK_TABLE_LUMI)."""
        m = ctypes.c_uint()
        _lib.call("fk_table_info", self._h, None, None, None, None, None, ctypes.byref(m), None)
        return bool(m.value & _lib.FK_TABLE_LUMI)

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h is not None and self._h.value:
            _lib.load().fk_table_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _check_f(t, F, prec):
    dt = _io_dtype(prec)
    if not (F.is_cuda and F.dtype == dt and F.is_contiguous() and F.dim() == 3
            and F.shape[1] == NFL and F.shape[2] == t.nxg):
        raise ValueError(f"F must be a contiguous cuda {dt} tensor [R][14][{t.nxg}]")


def conv(t: Table, F: torch.Tensor, prec="fp32", out: torch.Tensor = None,
         save: torch.Tensor = None) -> torch.Tensor:
    """Observables O [R][ndata] of table t for replicas F [R][14][nx_grid].

    out may be a column slice out[:, off:off+ndata] of a wider [R][n] tensor
    (unit stride along data points): the row stride is passed as ldo.
    save (hadronic tables, tensor-core modes): a buffer from saved_buffer
    that receives the forward's products for conv_backward(..., saved=save)."""
    _check_f(t, F, prec)
    R = F.shape[0]
    O = out if out is not None else torch.empty((R, t.ndata), dtype=F.dtype, device=F.device)
    if O.shape != (R, t.ndata) or O.stride(1) != 1 or O.dtype != F.dtype:
        raise ValueError("out must be [R][ndata] with unit column stride and F's dtype")
    if save is not None:
        _lib.call("fk_had_conv_save", t.handle, _p(F), R, _p(O), O.stride(0), _p(save), _nbytes(save),
                  _prec(prec), _stream())
        return O
    name = "fk_had_conv" if t.kind == 1 else "fk_dis_conv"
    _lib.call(name, t.handle, _p(F), R, _p(O), O.stride(0), _prec(prec), _stream())
    return O


def saved_size(t: Table, R: int, prec) -> int:
    """Bytes of the saved-product buffer of table t for R replicas (fk_saved_size)."""
    n = ctypes.c_size_t()
    _lib.call("fk_saved_size", t.handle, int(R), _prec(prec), ctypes.byref(n))
    return int(n.value)


def saved_buffer(t: Table, R: int, prec, device="cuda") -> torch.Tensor:
    """A device buffer for the forward's saved products (see conv's save)."""
    return torch.empty(saved_size(t, R, prec) // 4, dtype=torch.float32, device=device)


def _nbytes(x: torch.Tensor) -> int:
    if not (x.is_cuda and x.is_contiguous()):
        raise ValueError("the saved buffer must be a contiguous cuda tensor")
    return x.numel() * x.element_size()


def dis_conv(t, F, prec="fp32", out=None):
    assert t.kind == 0
    return conv(t, F, prec, out)


def had_conv(t, F, prec="fp32", out=None):
    assert t.kind == 1
    return conv(t, F, prec, out)


def dense_conv(t: Table, L: torch.Tensor, prec="fp32", out: torch.Tensor = None) -> torch.Tensor:
    """O [R][ndata] = FK L for a dense table: L [R][K] on cuda (the PDF
    matrix, replica-major; float64 for fp64, float32 otherwise)."""
    if t.kind != 2:
        raise ValueError("dense_conv needs a dense table")
    dt = _io_dtype(prec)
    if not (L.is_cuda and L.dtype == dt and L.is_contiguous() and L.dim() == 2 and L.shape[1] == t.K):
        raise ValueError(f"L must be a contiguous cuda {dt} tensor [R][{t.K}]")
    R = L.shape[0]
    O = out if out is not None else torch.empty((R, t.ndata), dtype=dt, device=L.device)
    if O.shape != (R, t.ndata) or O.stride(1) != 1 or O.dtype != dt:
        raise ValueError("out must be [R][ndata] with unit column stride and L's dtype")
    _lib.call("fk_dense_conv", t.handle, _p(L), R, _p(O), O.stride(0), _prec(prec), _stream())
    return O


def luminosity(t: Table, F: torch.Tensor, prec="fp32", out: torch.Tensor = None) -> torch.Tensor:
    """The PDF matrix L [R][nc * nx * nx] of hadronic table t for replicas F,
    L[r][(c*nx + i)*nx + j] = F[r][a_c][x_i] F[r][b_c][x_j]."""
    if t.kind != 1:
        raise ValueError("luminosity needs a hadronic table")
    _check_f(t, F, prec)
    R = F.shape[0]
    K = t.nch * t.nx * t.nx
    L = out if out is not None else torch.empty((R, K), dtype=F.dtype, device=F.device)
    if L.shape != (R, K) or not L.is_contiguous() or L.dtype != F.dtype:
        raise ValueError("out must be a contiguous [R][nc*nx*nx] tensor of F's dtype")
    _lib.call("fk_luminosity", t.handle, _p(F), R, _p(L), _prec(prec), _stream())
    return L


def conv_backward(t: Table, F, gO, prec="fp32", gF=None, accumulate=False, saved=None):
    """gF [R][14][nx_grid] (+)= sum_d gO[r][d] dO[r][d]/dF[r].

    saved: the buffer a conv(..., save=saved) of the same F wrote before
    (stream-ordered); the first-flavour term is then formed from it."""
    dt = _io_dtype(prec)
    R = gO.shape[0]
    if gF is None:
        gF = torch.empty((R, NFL, t.nxg), dtype=dt, device=gO.device)
        accumulate = False
    if gO.stride(1) != 1:
        raise ValueError("gO needs unit stride along data points")
    if saved is not None:
        _lib.call("fk_conv_backward_saved", t.handle, _p(F), _p(gO), gO.stride(0), R, _p(saved),
                  _nbytes(saved), _p(gF), int(bool(accumulate)), _prec(prec), _stream())
        return gF
    _lib.call("fk_conv_backward", t.handle, _p(F), _p(gO), gO.stride(0), R, _p(gF),
              int(bool(accumulate)), _prec(prec), _stream())
    return gF


def grad_sum(parts, out, accumulate=False):
    """out (+)= parts[0] + parts[1] + ... in that order (fk_grad_sum)."""
    n = out.numel()
    for p in parts:
        if p.numel() != n or p.dtype != out.dtype or not p.is_contiguous():
            raise ValueError("parts must be contiguous and match out")
    arr = (ctypes.c_void_p * len(parts))(*[p.data_ptr() for p in parts])
    prec = _lib.FK_FP64 if out.dtype == torch.float64 else _lib.FK_FP32
    _lib.call("fk_grad_sum", arr, len(parts), n, _p(out), int(bool(accumulate)), prec, _stream())
    return out


class Cov:
    """Block-diagonal covariance factorised on the device (FP64)."""

    def __init__(self, blocks):
        sizes = np.array([b.shape[0] for b in blocks], dtype=np.int32)
        flat = np.ascontiguousarray(np.concatenate([np.asarray(b, np.float64).ravel() for b in blocks]))
        h = ctypes.c_void_p()
        _lib.call("fk_cov_create", _p(flat), _p(sizes), len(blocks), ctypes.byref(h))
        self._h = h
        self.n = int(sizes.sum())
        self.sizes = sizes

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h is not None and self._h.value:
            _lib.load().fk_cov_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def chi2(cov: Cov, O: torch.Tensor, D: torch.Tensor, grad=True, out=None, gO=None):
    """chi2 [R] (FP64) and, if grad, dchi2/dO [R][n] in O's dtype.  O may be
    FP64 or FP32; the arithmetic is FP64 on the device either way."""
    R = O.shape[0]
    if not O.is_contiguous() or O.shape[1] != cov.n:
        raise ValueError(f"O must be contiguous [R][{cov.n}]")
    io = _lib.FK_FP64 if O.dtype == torch.float64 else _lib.FK_FP32
    c = out if out is not None else torch.empty(R, dtype=torch.float64, device=O.device)
    g = None
    if grad:
        g = gO if gO is not None else torch.empty_like(O)
    _lib.call("fk_chi2", cov.handle, _p(O), _p(D), R, _p(c), _p(g), io, _stream())
    return c, g


def chi2_white(Z: torch.Tensor, Dw: torch.Tensor, grad=True, out=None, gO=None):
    """chi2 [R] (FP64) = |Z_r - Dw|^2 of whitened observables Z [R][n] (rows
    of unit stride, FP64 or FP32; Dw [n] FP64 on cuda) and, if grad,
    dchi2/dZ = 2 (Z - Dw) in Z's dtype (fk_chi2_white)."""
    R, n = Z.shape
    if Z.stride(1) != 1 or Dw.dtype != torch.float64 or Dw.numel() != n or not Dw.is_contiguous():
        raise ValueError("Z must have unit column stride and Dw be a contiguous float64 [n]")
    io = _lib.FK_FP64 if Z.dtype == torch.float64 else _lib.FK_FP32
    c = out if out is not None else torch.empty(R, dtype=torch.float64, device=Z.device)
    g = None
    if grad:
        g = gO if gO is not None else torch.empty((R, n), dtype=Z.dtype, device=Z.device)
        if g.stride(1) != 1 or g.shape != (R, n) or g.dtype != Z.dtype:
            raise ValueError("gO must be [R][n] with unit column stride and Z's dtype")
    _lib.call("fk_chi2_white", _p(Z), Z.stride(0), _p(Dw), n, R, _p(c), _p(g), g.stride(0) if g is not None else 0,
              io, _stream())
    return c, g


class Server:
    """Continuously batched serving over device-resident tables (fk_serve_*)."""

    def __init__(self, budget_bytes: int, max_inflight: int = 4):
        h = ctypes.c_void_p()
        _lib.call("fk_serve_create", ctypes.c_size_t(int(budget_bytes)), int(max_inflight),
                  ctypes.byref(h))
        self._h = h
        self._tables = []
        self._meta = {}

    def add_table(self, t: Table) -> int:
        tid = ctypes.c_int()
        _lib.call("fk_serve_add_table", self._h, t.handle, ctypes.byref(tid))
        self._tables.append(t)
        return tid.value

    def submit(self, table_id: int, F: np.ndarray, prec="fp32") -> int:
        """F: host [R][14][nx_grid] (float64 for fp64, float32 otherwise)."""
        dt = np.float64 if _prec(prec) in (_lib.FK_FP64, _lib.FK_FP64_TC) else np.float32
        F = np.ascontiguousarray(F, dtype=dt)
        tk = ctypes.c_uint64()
        _lib.call("fk_serve_submit", self._h, int(table_id), _p(F), F.shape[0], _prec(prec),
                  ctypes.byref(tk))
        self._meta[tk.value] = (F.shape[0], self._tables[table_id].ndata, dt)
        return tk.value

    def _out(self, ticket):
        if ticket not in self._meta:  # let the library report the unknown ticket
            return None
        R, nd, dt = self._meta[ticket]
        return np.empty((R, nd), dtype=dt)

    def poll(self, ticket: int):
        """(True, O) when done, (False, None) while pending; raises on failure."""
        O = self._out(ticket)
        done = ctypes.c_int()
        rc = _lib.load().fk_serve_poll(self._h, ctypes.c_uint64(ticket), _p(O), ctypes.byref(done))
        if rc == _lib.FK_EPENDING:
            return False, None
        self._meta.pop(ticket, None)
        if rc != 0:
            raise FKError("fk_serve_poll", rc, _lib.load())
        return True, O

    def wait(self, ticket: int, timeout_ms: int = 60000) -> np.ndarray:
        O = self._out(ticket)
        rc = _lib.load().fk_serve_wait(self._h, ctypes.c_uint64(ticket), _p(O), int(timeout_ms))
        if rc == _lib.FK_EPENDING:
            raise TimeoutError(f"ticket {ticket} still running after {timeout_ms} ms")
        self._meta.pop(ticket, None)
        if rc != 0:
            raise FKError("fk_serve_wait", rc, _lib.load())
        return O

    def cancel(self, ticket: int):
        """Cancels a request (fk_serve_cancel): its poll/wait then raises
        FKError with FK_ECANCELED, unless it had finished already."""
        _lib.call("fk_serve_cancel", self._h, ctypes.c_uint64(ticket))

    def inject(self, fault: str, count: int = 1):
        """Arms `count` host-side faults (fk_serve_inject): "pinned", "device",
        "launch" or "drop" (a lost completion message)."""
        kind = {"pinned": _lib.FK_FAULT_PINNED, "device": _lib.FK_FAULT_DEVICE, "launch": _lib.FK_FAULT_LAUNCH,
                "drop": _lib.FK_FAULT_DROP}[fault]
        _lib.call("fk_serve_inject", self._h, kind, int(count))

    def stats(self) -> dict:
        c, d, n = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        pk, q = ctypes.c_size_t(), ctypes.c_int()
        _lib.call("fk_serve_stats", self._h, ctypes.byref(c), ctypes.byref(d), ctypes.byref(n),
                  ctypes.byref(pk), ctypes.byref(q))
        return dict(completed=c.value, datapoint_replicas=d.value, launches=n.value,
                    peak_bytes=pk.value, queued=q.value)

    def close(self):
        if self._h is not None and self._h.value:
            _lib.load().fk_serve_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FKConv(torch.autograd.Function):
    """O = conv(t, F); backward gives dL/dF through the library's adjoint."""

    @staticmethod
    def forward(ctx, F, t, prec="fp32"):
        ctx.t, ctx.prec = t, prec
        ctx.save_for_backward(F)
        return conv(t, F.contiguous(), prec)

    @staticmethod
    def backward(ctx, gO):
        (F,) = ctx.saved_tensors
        gF = conv_backward(ctx.t, F.contiguous(), gO.contiguous(), ctx.prec)
        return gF, None, None
