"""FP64 CPU oracle of the FK-table convolution (arXiv:1909.10547, Sec. 3, Eq. 1).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
CPU-baseline leg of the benchmark, never by the library.  It shares no code with
the CUDA path.  The arithmetic lives in fk_oracle.c (plain loops, FP64,
compensated sums); this module only marshals numpy arrays.

Functions (all FP64, numpy in / numpy out):
  dis(table, F)            -> (O, S)   DIS observables, Table 1 "DIS"
  had(table, F)            -> (O, S)   hadronic observables, Eq. 1
  dis_grad(table, gO)      -> gF       sum_d gO[r,d] dO[r,d]/dF[r,a,x]
  had_grad(table, F, gO)   -> gF       the same for Eq. 1 (product rule)
  luminosity(table, F)     -> L        the PDF matrix of Table 3, L[r][(c,i,j)] = f_a(x_i) f_b(x_j)
  dense(fk2d, L)           -> (O, S)   the dense product of Table 3, O[r][d] = sum_k fk[d][k] L[r][k]
  cholesky(C)              -> L        C = L L^T
  chi2(L, O, D)            -> (chi2, gO)  (O-D)^T C^-1 (O-D) and its O-gradient
S is the sum of |terms| of each observable (the scale of its rounding error).
"""
import ctypes
import os

import numpy as np

from .build import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        I = ctypes.c_int
        L.fk_oracle_dis.argtypes = [I, I, P, P, I, I, P, P, P]
        L.fk_oracle_had.argtypes = [I, I, P, P, I, P, P, I, I, P, P, P]
        L.fk_oracle_dis_grad.argtypes = [I, I, P, P, I, I, P, P]
        L.fk_oracle_had_grad.argtypes = [I, I, P, P, I, P, P, I, I, P, P, P]
        L.fk_oracle_luminosity.argtypes = [I, P, P, I, P, I, I, P, P]
        L.fk_oracle_dense.argtypes = [I, ctypes.c_longlong, P, I, P, P, P]
        L.fk_oracle_cholesky.argtypes = [I, P, P]
        L.fk_oracle_chi2.argtypes = [I, P, I, P, P, P, P]
        L.fk_oracle_set_threads.argtypes = [I]
        for f in (L.fk_oracle_dis, L.fk_oracle_had, L.fk_oracle_dis_grad,
                  L.fk_oracle_had_grad, L.fk_oracle_luminosity, L.fk_oracle_dense,
                  L.fk_oracle_cholesky, L.fk_oracle_chi2,
                  L.fk_oracle_threads, L.fk_oracle_set_threads):
            f.restype = I
        _lib = L
    return _lib


def threads() -> int:
    return lib().fk_oracle_threads()


def set_threads(n: int) -> int:
    """OpenMP threads of later calls (timing only); returns the count in effect."""
    return lib().fk_oracle_set_threads(int(n))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def dis(t, F):
    """t: DisTable-like (fk [ndata][14][nx], xmap, nxg); F [R][14][nxg]."""
    fk = _f64(t.fk)
    F = _f64(F)
    R = F.shape[0]
    nd, nfl, nx = fk.shape
    assert nfl == 14 and F.shape[1:] == (14, t.nxg)
    xm = _i32(t.xmap)
    O = np.empty((R, nd))
    S = np.empty((R, nd))
    _check(lib().fk_oracle_dis(nd, nx, _p(fk), _p(xm), t.nxg, R, _p(F), _p(O), _p(S)), "dis")
    return O, S


def had(t, F):
    """t: HadTable-like (fk [ndata][nc][nx][nx], ca, cb, xmap, nxg); F [R][14][nxg]."""
    fk = _f64(t.fk)
    F = _f64(F)
    R = F.shape[0]
    nd, nc, nx, nx2 = fk.shape
    assert nx == nx2 and F.shape[1:] == (14, t.nxg)
    ca, cb, xm = _i32(t.ca), _i32(t.cb), _i32(t.xmap)
    O = np.empty((R, nd))
    S = np.empty((R, nd))
    _check(lib().fk_oracle_had(nd, nc, _p(ca), _p(cb), nx, _p(fk), _p(xm), t.nxg, R,
                               _p(F), _p(O), _p(S)), "had")
    return O, S


def dis_grad(t, gO):
    fk = _f64(t.fk)
    gO = _f64(gO)
    R, nd = gO.shape
    nx = fk.shape[2]
    xm = _i32(t.xmap)
    gF = np.empty((R, 14, t.nxg))
    _check(lib().fk_oracle_dis_grad(nd, nx, _p(fk), _p(xm), t.nxg, R, _p(gO), _p(gF)), "dis_grad")
    return gF


def had_grad(t, F, gO):
    fk = _f64(t.fk)
    F = _f64(F)
    gO = _f64(gO)
    R, nd = gO.shape
    nc, nx = fk.shape[1], fk.shape[2]
    ca, cb, xm = _i32(t.ca), _i32(t.cb), _i32(t.xmap)
    gF = np.empty((R, 14, t.nxg))
    _check(lib().fk_oracle_had_grad(nd, nc, _p(ca), _p(cb), nx, _p(fk), _p(xm), t.nxg, R,
                                    _p(F), _p(gO), _p(gF)), "had_grad")
    return gF


def conv(t, F):
    """Dispatch on the table kind: (O, S)."""
    return had(t, F) if hasattr(t, "ca") else dis(t, F)


def conv_grad(t, F, gO):
    return had_grad(t, F, gO) if hasattr(t, "ca") else dis_grad(t, gO)


def luminosity(t, F):
    """The PDF matrix of Table 3 for a HadTable-like t: [R][nc * nx * nx]."""
    F = _f64(F)
    R = F.shape[0]
    nc, nx = len(t.ca), len(t.xmap)
    assert F.shape[1:] == (14, t.nxg)
    ca, cb, xm = _i32(t.ca), _i32(t.cb), _i32(t.xmap)
    L = np.empty((R, nc * nx * nx))
    _check(lib().fk_oracle_luminosity(nc, _p(ca), _p(cb), nx, _p(xm), t.nxg, R, _p(F), _p(L)), "luminosity")
    return L


def dense(fk, L):
    """fk [ndata][K], L [R][K] (the PDF matrix, replica-major) -> (O [R][ndata], S)."""
    fk = _f64(fk)
    L = _f64(L)
    nd, K = fk.shape
    R = L.shape[0]
    assert L.shape[1] == K
    O = np.empty((R, nd))
    S = np.empty((R, nd))
    _check(lib().fk_oracle_dense(nd, K, _p(fk), R, _p(L), _p(O), _p(S)), "dense")
    return O, S


def cholesky(C):
    C = _f64(C)
    n = C.shape[0]
    L = np.empty_like(C)
    rc = lib().fk_oracle_cholesky(n, _p(C), _p(L))
    if rc != 0:
        raise np.linalg.LinAlgError(f"oracle cholesky: pivot {rc - 1} not positive")
    return L


def chi2(L, O, D, grad=True):
    """L [n][n] lower factor, O [R][n], D [n] -> chi2 [R], gO [R][n] (or None)."""
    L = _f64(L)
    O = _f64(O)
    D = _f64(D)
    R, n = O.shape
    c = np.empty(R)
    g = np.empty((R, n)) if grad else None
    _check(lib().fk_oracle_chi2(n, _p(L), R, _p(O), _p(D), _p(c), _p(g)), "chi2")
    return c, g
