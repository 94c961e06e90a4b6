"""Seeded synthetic inputs shaped like the paper's FK-convolution workloads.

This module only draws numbers: x grids, FK tables, active channel lists, PDF
replicas, block covariances, pseudo-data and request arrivals.  It contains none
of the convolution, gradient or chi^2 arithmetic, so that both the FP64 oracle
and the CUDA path can take their inputs from here without sharing any of the
method's code.

Shapes follow the paper's setting (Sec. 3, Eq. 1): an FK table per dataset with
one entry per data point, flavour pair and pair of x-grid points, convolved with
the PDFs f_a(x_i) of 14 evolution-basis flavours sampled on a log-spaced x grid.
The paper publishes no tables, so every value here is synthetic:

* x grid: x_i = 10**(log10(xmin) * (1 - i/nx)), i = 0..nx-1 (half-open [xmin, 1)).
* PDF:    f_a(x) = A_a x**alpha_a (1-x)**beta_a, alpha ~ U(-0.2, 0.8),
          beta ~ U(1, 5), A ~ U(0.5, 2) per flavour; replicas jitter alpha and
          beta by a factor U(0.9, 1.1) each (A is shared).
* DIS FK:      |N(0,1)| * x_i**0.3 on active flavours, 0 elsewhere.
* hadronic FK: N(0,1) * x_i**0.2 * x_j**0.2 per active ordered pair (a, b).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

NFL = 14          # evolution-basis flavours
NPAIR = NFL * NFL  # ordered flavour pairs
SEED_BASE = 10547


def xgrid(nx: int, xmin: float) -> np.ndarray:
    """nx log-spaced points on the half-open interval [xmin, 1)."""
    i = np.arange(nx, dtype=np.float64)
    return 10.0 ** (math.log10(xmin) * (1.0 - i / nx))


@dataclasses.dataclass
class PdfParams:
    A: np.ndarray       # [14]
    alpha: np.ndarray   # [14]
    beta: np.ndarray    # [14]


def pdf_params(rng: np.random.Generator) -> PdfParams:
    A = rng.uniform(0.5, 2.0, NFL)
    alpha = rng.uniform(-0.2, 0.8, NFL)
    beta = rng.uniform(1.0, 5.0, NFL)
    return PdfParams(A, alpha, beta)


def pdf_replicas(x: np.ndarray, p: PdfParams, R: int, rng: np.random.Generator | None,
                 jitter: float = 0.1) -> np.ndarray:
    """F[R][14][nx] = A_a x^alpha_{r,a} (1-x)^beta_{r,a}.

    With rng=None (or jitter=0) every replica is the central PDF."""
    if rng is None or jitter == 0.0:
        ja = np.ones((R, NFL))
        jb = np.ones((R, NFL))
    else:
        ja = rng.uniform(1.0 - jitter, 1.0 + jitter, (R, NFL))
        jb = rng.uniform(1.0 - jitter, 1.0 + jitter, (R, NFL))
    al = p.alpha[None, :] * ja
    be = p.beta[None, :] * jb
    lx = np.log(x)[None, None, :]
    l1x = np.log1p(-x)[None, None, :]
    F = p.A[None, :, None] * np.exp(al[:, :, None] * lx + be[:, :, None] * l1x)
    return np.ascontiguousarray(F)


@dataclasses.dataclass
class DisTable:
    """DIS FK table.  fk is dense over all 14 flavours: [ndata][14][nx]."""
    fk: np.ndarray
    flav: np.ndarray       # active flavours, sorted, int32
    xmap: np.ndarray       # [nx] indices into the PDF grid, int32
    nxg: int               # size of the PDF grid that xmap indexes

    @property
    def ndata(self) -> int:
        return self.fk.shape[0]

    @property
    def nx(self) -> int:
        return self.fk.shape[2]

    def compact(self) -> np.ndarray:
        """[ndata][nflav][nx]: the active-flavour slices only."""
        return np.ascontiguousarray(self.fk[:, self.flav, :])


@dataclasses.dataclass
class HadTable:
    """Hadronic FK table per active channel: fk[ndata][nc][nx][nx].

    Channel c couples flavour ca[c] at x_i with flavour cb[c] at x_j."""
    fk: np.ndarray
    ca: np.ndarray         # [nc] int32
    cb: np.ndarray         # [nc] int32
    xmap: np.ndarray       # [nx] int32
    nxg: int

    @property
    def ndata(self) -> int:
        return self.fk.shape[0]

    @property
    def nc(self) -> int:
        return self.fk.shape[1]

    @property
    def nx(self) -> int:
        return self.fk.shape[2]


def dis_table(rng: np.random.Generator, ndata: int, nact: int, x: np.ndarray,
              xmap: np.ndarray | None = None, nxg: int | None = None) -> DisTable:
    nx = len(x)
    flav = np.sort(rng.choice(NFL, nact, replace=False)).astype(np.int32)
    fk = np.zeros((ndata, NFL, nx))
    vals = np.abs(rng.standard_normal((ndata, nact, nx))) * (x ** 0.3)[None, None, :]
    fk[:, flav, :] = vals
    if xmap is None:
        xmap = np.arange(nx, dtype=np.int32)
        nxg = nx
    return DisTable(fk, flav, np.asarray(xmap, np.int32), int(nxg))


def channels(rng: np.random.Generator, nc: int) -> tuple[np.ndarray, np.ndarray]:
    """nc distinct ordered flavour pairs (a, b), drawn without replacement."""
    pick = np.sort(rng.choice(NPAIR, nc, replace=False))
    return (pick // NFL).astype(np.int32), (pick % NFL).astype(np.int32)


def had_table(rng: np.random.Generator, ndata: int, nc: int, x: np.ndarray,
              xmap: np.ndarray | None = None, nxg: int | None = None,
              dtype=np.float64) -> HadTable:
    nx = len(x)
    ca, cb = channels(rng, nc)
    w = x ** 0.2
    fk = rng.standard_normal((ndata, nc, nx, nx)).astype(dtype)
    fk *= (w[:, None] * w[None, :]).astype(dtype)[None, None]
    if xmap is None:
        xmap = np.arange(nx, dtype=np.int32)
        nxg = nx
    return HadTable(fk, ca, cb, np.asarray(xmap, np.int32), int(nxg))


# ---------------------------------------------------------------------------
# The five workloads.
# ---------------------------------------------------------------------------

def config0(seed: int = SEED_BASE + 0):
    """Plain DIS convolution: ndata=64, 9 of 14 flavours active, nx=40 on
    [1e-7, 1), one PDF."""
    rng = np.random.default_rng(seed)
    x = xgrid(40, 1e-7)
    t = dis_table(rng, 64, 9, x)
    F = pdf_replicas(x, pdf_params(rng), 1, None)
    return t, F


def config1(R: int = 1, seed: int = SEED_BASE + 1, ndata: int = 200, nc: int = 60,
            nx: int = 30):
    """Plain hadronic convolution: ndata=200, nx=30 on [1e-6, 1), 60 active
    ordered channels, R jittered replicas (R=1: the central PDF)."""
    rng = np.random.default_rng(seed)
    x = xgrid(nx, 1e-6)
    t = had_table(rng, ndata, nc, x)
    p = pdf_params(rng)
    F = pdf_replicas(x, p, R, rng if R > 1 else None)
    return t, F


def config2(R: int = 512, seed: int = SEED_BASE + 2):
    """Config 1's table at R=512 replicas (reduced-precision study)."""
    return config1(R=R, seed=seed)


@dataclasses.dataclass
class GlobalSet:
    """40 datasets on a shared 50-point x grid, plus replicas on that grid."""
    x: np.ndarray                   # master grid [50]
    tables: list                    # DisTable | HadTable
    F: np.ndarray                   # [R][14][50] jittered replicas
    F_true: np.ndarray              # [1][14][50] central PDF
    params: PdfParams


def global_ndata(rng: np.random.Generator, n: int = 40, total: int = 4500,
                 lo: int = 10, hi: int = 600) -> np.ndarray:
    """Log-uniform sizes in [lo, hi], rescaled until they sum to total +- 5%."""
    v = np.exp(rng.uniform(math.log(lo), math.log(hi), n))
    for _ in range(100):
        v = np.clip(v * (total / v.sum()), lo, hi)
        if abs(v.sum() - total) <= 0.05 * total:
            break
    return np.maximum(lo, np.round(v)).astype(int)


def config3(R: int = 100, seed: int = SEED_BASE + 3, n_dis: int = 12, n_had: int = 28,
            total: int = 4500, scale: float = 1.0) -> GlobalSet:
    """Global-shaped fit set: 12 DIS + 28 hadronic datasets, ~4500 points,
    nx 20..50 drawn from a 50-point master grid on [1e-7, 1), 20..120 active
    channels per hadronic set, 5..14 active flavours per DIS set.

    scale < 1 shrinks every ndata (for oracle-sized tests) keeping the mix."""
    rng = np.random.default_rng(seed)
    nxg = 50
    x = xgrid(nxg, 1e-7)
    kinds = np.array(["dis"] * n_dis + ["had"] * n_had)
    rng.shuffle(kinds)
    nd = global_ndata(rng, len(kinds), total)
    tables = []
    for k, n in zip(kinds, nd):
        n = max(1, int(round(n * scale)))
        nx = int(rng.integers(20, 51))
        xmap = np.sort(rng.choice(nxg, nx, replace=False)).astype(np.int32)
        if k == "dis":
            tables.append(dis_table(rng, n, int(rng.integers(5, 15)), x[xmap], xmap, nxg))
        else:
            tables.append(had_table(rng, n, int(rng.integers(20, 121)), x[xmap], xmap, nxg))
    p = pdf_params(rng)
    F = pdf_replicas(x, p, R, rng)
    F_true = pdf_replicas(x, p, 1, None)
    return GlobalSet(x, tables, F, F_true, p)


@dataclasses.dataclass
class CovBlocks:
    """Block-diagonal covariance: one dense SPD block per dataset."""
    blocks: list     # each [n_k][n_k] float64


def covariance(o_true: list, seed: int, rank: int = 10, corr: float = 0.05,
               stat: float = 0.03, floor: float = 1e-3) -> CovBlocks:
    """C_k = G G^T + diag(s^2) with G[d,m] ~ N(0,1)*corr*|o_d| (m < min(n,rank))
    and s_d = stat*|o_d| + floor*mean|o| per dataset block.  o_true[k] is the
    central prediction of block k, supplied by the caller."""
    rng = np.random.default_rng(seed)
    out = []
    for o in o_true:
        o = np.abs(np.asarray(o, np.float64))
        n = len(o)
        m = min(n, rank)
        G = rng.standard_normal((n, m)) * corr * o[:, None]
        s = stat * o + floor * max(o.mean(), 1e-300)
        out.append(G @ G.T + np.diag(s * s))
    return CovBlocks(out)


def pseudo_data(o_true: list, seed: int, rank: int = 10, corr: float = 0.05,
                stat: float = 0.03, floor: float = 1e-3) -> list:
    """D_k = o_k + G z1 + s * z2: one draw from N(o_k, C_k) with C_k as in
    covariance() (same seed gives the same G)."""
    rng = np.random.default_rng(seed)
    rz = np.random.default_rng(seed + 7919)
    out = []
    for o in o_true:
        o = np.asarray(o, np.float64)
        a = np.abs(o)
        n = len(o)
        m = min(n, rank)
        G = rng.standard_normal((n, m)) * corr * a[:, None]
        s = stat * a + floor * max(a.mean(), 1e-300)
        out.append(o + G @ rz.standard_normal(m) + s * rz.standard_normal(n))
    return out


# ---------------------------------------------------------------------------
# Served workload.
# ---------------------------------------------------------------------------

STRESS_SHAPE = dict(ndata=2000, nc=196, nx=50)


def stress_table(seed: int = SEED_BASE + 4, ndata: int = 2000, nx: int = 50,
                 dtype=np.float64) -> HadTable:
    """Hadronic stress table: every one of the 196 ordered channels, nx=50 on
    [1e-7, 1).  Row d is drawn from its own generator (seed, d), so any data
    point can be regenerated alone with stress_row()."""
    x = xgrid(nx, 1e-7)
    ca = (np.arange(NPAIR) // NFL).astype(np.int32)
    cb = (np.arange(NPAIR) % NFL).astype(np.int32)
    fk = np.empty((ndata, NPAIR, nx, nx), dtype=dtype)
    for d in range(ndata):
        fk[d] = stress_row(seed, d, nx).astype(dtype)
    return HadTable(fk, ca, cb, np.arange(nx, dtype=np.int32), nx)


def stress_row(seed: int, d: int, nx: int = 50) -> np.ndarray:
    x = xgrid(nx, 1e-7)
    w = x ** 0.2
    r = np.random.default_rng([seed, d])
    return r.standard_normal((NPAIR, nx, nx)) * (w[:, None] * w[None, :])[None]


def arrivals(rng: np.random.Generator, rate: float, n: int) -> np.ndarray:
    """Poisson arrival times (seconds) of n requests at the given rate."""
    return np.cumsum(rng.exponential(1.0 / rate, n))


REPLICA_CHOICES = (1, 10, 100, 1000)


# ---------------------------------------------------------------------------
# The dense product of the paper's timing study (Sec. 3, Table 3).
# ---------------------------------------------------------------------------

TABLE3_SHAPE = dict(nc=49, nx=27)  # K = 49 * 27 * 27 = 35721 elements per data point


def table3(ndata: int, R: int, seed: int = SEED_BASE + 5):
    """The base table of the paper's Table 3: 49 flavour combinations (all
    ordered pairs of 7 seeded flavours) on 27 x points in [1e-6, 1), so
    K = 35721 elements per data point; FK ~ N(0,1) x_i^0.2 x_j^0.2 as in
    config 1, and R jittered replicas of the config-0 PDF family.
    Returns (HadTable, F [R][14][27]); the dense product takes the table
    flattened to [ndata][K] and the PDF matrix built from F."""
    rng = np.random.default_rng(seed)
    nx = TABLE3_SHAPE["nx"]
    x = xgrid(nx, 1e-6)
    fl = np.sort(rng.choice(NFL, 7, replace=False))
    ca = np.repeat(fl, 7).astype(np.int32)
    cb = np.tile(fl, 7).astype(np.int32)
    w = x ** 0.2
    fk = rng.standard_normal((ndata, len(ca), nx, nx))
    fk *= (w[:, None] * w[None, :])[None, None]
    t = HadTable(fk, ca, cb, np.arange(nx, dtype=np.int32), nx)
    F = pdf_replicas(x, pdf_params(rng), R, rng if R > 1 else None)
    return t, F
