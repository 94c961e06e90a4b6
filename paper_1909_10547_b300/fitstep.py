"""One gradient-descent fit step over a set of device-resident FK tables.

The step is the hot path of the paper's fit (Sec. 2: gradient descent; Sec. 3:
the convolution is the most time-consuming operation):

  forward   O_k = conv(table_k, F)                      for every dataset k
  loss      chi2_k[r] = (O_k,r - D_k)^T C_k^{-1} (O_k,r - D_k),  gO_k = d chi2_k / d O_k
  backward  gF = sum_k conv_backward(table_k, F, gO_k)
  chi2      = sum_k chi2_k

The covariance is block diagonal with one block per dataset, so the three
stages of dataset k depend only on each other.  All run in libfk.so kernels.

pipelined=True (default): each table's chain forward -> chi^2 block ->
adjoint runs on its own CUDA stream, so the work of one dataset overlaps the
convolutions of the others (with the FP64 substitutions, the chi^2 is forked
onto a high-priority stream of its own and joined back; on whitened tables
it is one short kernel on the chain's stream); the per-stream gradient
buffers and the per-dataset chi^2 values are then added by fk_grad_sum in a
fixed order.  capture() records the step as one CUDA graph whose streams are
parallel branches.

pipelined=False: three phases (all forwards, one chi^2 launch over all
blocks, all adjoints), each its own graph, for per-phase timing.

Either way the result does not depend on how the streams interleave: every
table writes its own outputs and every sum runs in a fixed order.

save_products (hadronic tables in the tensor-core modes): the forward also
keeps its tensor-core products (fk_had_conv_save) and the adjoint forms its
first-flavour term from them (fk_conv_backward_saved) instead of a second
pass over the table; the results are bit for bit those of the plain calls.
Saving writes 4 * ndata * groups * nx * R_pad bytes, where a pass over a
BF16 hi+lo table reads 4 * ndata * nc * nx^2, so it pays where
rho = nc * nx / (groups * R_pad) is large: measured alone (R = 100, BF16
hi+lo) the ten largest tables of the global set gained 29-62 us per step
from saving at rho >= 1.7, about nothing at rho = 1.1-1.4 and lost at
rho < 1.  "auto" (default) saves where rho >= save_ratio (1.25); True
everywhere; False nowhere.

whiten (default: every mode but FP64 and FP64 on the tensor cores): the
covariance does not change during a fit, so each block's factor is folded
into its table and data once, at set-up (whiten_tables): with C_k = L_k L_k^T,
the whitened table L_k^{-1} FK_k convolves to Z_k = L_k^{-1} O_k, and
chi2_k = |Z_k - L_k^{-1} D_k|^2 with d chi2 / d Z_k = 2 (Z_k - L_k^{-1} D_k),
which the adjoint of the whitened table turns into d chi2 / dF
(fk_chi2_white).  The step then has no triangular solve.  The FP64 modes keep
the substitutions of fk_chi2 and their 1e-12 contract.
"""
import dataclasses

import numpy as np
import torch

from . import Cov, Table, _lib, chi2, chi2_white, conv, conv_backward, dense_conv, grad_sum, saved_buffer

NFL = 14


def _lower_inverse(L):
    """L^{-1} of a lower-triangular L by forward substitution, row by row
    (exact zeros above the diagonal)."""
    n = L.shape[0]
    X = np.zeros((n, n))
    for i in range(n):
        X[i, :i + 1] = -(L[i, :i] @ X[:i, :i + 1])
        X[i, i] += 1.0
        X[i, :i + 1] /= L[i, i]
    return X


def whiten_tables(tables, cov_blocks, D_parts, device="cuda"):
    """(whitened tables, whitened data): per dataset k, with C_k = L_k L_k^T,
    the table L_k^{-1} FK_k (rows of the table mixed over its data points,
    the same channels and grid) and L_k^{-1} D_k.  The product runs on the
    device in FP64 through the dense product (fk_dense_conv with L_k^{-1} as
    the table and the table's transpose as the operand); L_k^{-1} and the data
    are formed on the host (at most a few hundred rows per block)."""
    out, Dw = [], []
    for t, C, Dk in zip(tables, cov_blocks, D_parts):
        n = t.ndata
        L = np.linalg.cholesky(np.asarray(C, np.float64))
        Li = _lower_inverse(L)
        dtab = Table.dense(Li, precs=("fp64",))
        E = t.fk.size // n
        FKT = torch.tensor(np.ascontiguousarray(np.asarray(t.fk, np.float64).reshape(n, E).T), device=device)
        Wt = dense_conv(dtab, FKT, "fp64")  # [E][n] = (L^{-1} FK)^T
        fkw = Wt.t().contiguous().cpu().numpy().reshape(t.fk.shape)
        dtab.close()
        del FKT, Wt
        out.append(dataclasses.replace(t, fk=fkw))
        Dw.append(Li @ np.asarray(Dk, np.float64))
    return out, Dw


class GlobalFit:
    def __init__(self, tables, F, cov_blocks, D, prec="fp32", store=None, device="cuda",
                 nstreams=None, pipelined=True, waves=1, save_products="auto", save_ratio=1.25, whiten=None):
        """tables: workloads.DisTable/HadTable list sharing one x grid;
        F: [R][14][nxg] replicas (host numpy); cov_blocks: one SPD block per
        table; D: [sum ndata] pseudo-data."""
        self.prec = prec
        io = torch.float64 if prec in ("fp64", "fp64tc") else torch.float32
        self.whiten = prec not in ("fp64", "fp64tc") if whiten is None else bool(whiten)
        if self.whiten:
            nd0 = np.cumsum([0] + [t.ndata for t in tables])
            D = np.asarray(D, np.float64)
            tables, Dw = whiten_tables(tables, cov_blocks, [D[a:b] for a, b in zip(nd0, nd0[1:])], device)
            D = np.concatenate(Dw)
        if store is None:
            store = ("fp64", "fp32") if prec in ("fp64", "fp32") else (prec,)
        self.tabs = [Table.from_workload(t, store) for t in tables]
        self.kinds = ["had" if hasattr(t, "ca") else "dis" for t in tables]
        # every table runs in the step's mode: in the reduced modes the DIS
        # tables are plain products on the tensor cores, like the hadronic ones
        self.tprec = [prec for _ in tables]
        # per table: the buffer of its saved forward products, or None
        tc = prec in ("bf16", "bf16x3", "tf32")
        R_pad = -(-F.shape[0] // 128) * 128
        self.saved = []
        for t, tab, kind in zip(tables, self.tabs, self.kinds):
            use = tc and kind == "had" and not tab.lumi and save_products is not False
            if use and save_products == "auto":
                groups = len(set(np.asarray(t.ca).tolist()))
                use = t.nc * t.nx >= save_ratio * groups * R_pad
            self.saved.append(saved_buffer(tab, F.shape[0], prec, device) if use else None)
        nd = [t.ndata for t in tables]
        self.offs = np.concatenate([[0], np.cumsum(nd)]).astype(int)
        self.ntot = int(self.offs[-1])
        self.R = F.shape[0]
        self.nxg = F.shape[2]
        self.io = io
        self.pipelined = pipelined
        self.D = torch.tensor(np.asarray(D, np.float64), device=device)
        self.F = torch.tensor(np.asarray(F), dtype=io, device=device)
        self.gF = torch.empty_like(self.F)
        self.chi2 = torch.empty(self.R, dtype=torch.float64, device=device)
        if pipelined:
            # per dataset: its covariance block, and O_k, gO_k as contiguous
            # [R][n_k] blocks of one buffer
            self.covs = None if self.whiten else [Cov([b]) for b in cov_blocks]
            assert self.whiten or sum(c.n for c in self.covs) == self.ntot
            self.Obuf = torch.empty(self.R * self.ntot, dtype=io, device=device)
            self.gObuf = torch.empty_like(self.Obuf)
            self.Ok = [self.Obuf[self.R * a:self.R * b].view(self.R, b - a) for a, b in zip(self.offs, self.offs[1:])]
            self.gOk = [self.gObuf[self.R * a:self.R * b].view(self.R, b - a) for a, b in zip(self.offs, self.offs[1:])]
            self.Dk = [self.D[a:b] for a, b in zip(self.offs, self.offs[1:])]
            self.chi2_parts = torch.empty((len(tables), self.R), dtype=torch.float64, device=device)
        else:
            self.cov = None if self.whiten else Cov(cov_blocks)
            assert self.whiten or self.cov.n == self.ntot
            self.O = torch.empty((self.R, self.ntot), dtype=io, device=device)
            self.gO = torch.empty_like(self.O)
        self.graphs = None
        # algorithmic work per step (multiply-adds counted as 2 flops) and the
        # table elements each phase streams
        fwd = bwd = 0
        work = []
        self.elems = {"had": 0, "dis": 0}
        for t in tables:
            if hasattr(t, "ca"):
                e = t.ndata * t.nc * t.nx * t.nx
                fwd += 2 * e * self.R
                bwd += (4 * e) * self.R
                self.elems["had"] += e
            else:
                e = t.ndata * len(t.flav) * t.nx
                fwd += 2 * e * self.R
                bwd += 2 * e * self.R
                self.elems["dis"] += e
            work.append(e)
        # the loss: both substitutions (n_k^2 multiply-adds per replica), or for
        # whitened tables one subtraction and one multiply-add per data point
        loss = 2 * self.ntot * self.R if self.whiten else 2 * int(sum(n * n for n in nd)) * self.R
        self.flops = {"forward": fwd, "loss": loss, "backward": bwd}
        # streams: greedy assignment of tables (largest first) to the least
        # loaded stream; by default one stream per table (up to the 64
        # gradient parts that grad_sum combines), so that the small per-table
        # launches overlap
        self.nstreams = max(1, min(nstreams or 64, len(tables), 64))
        load = [0] * self.nstreams
        self.groups = [[] for _ in range(self.nstreams)]
        for k in sorted(range(len(tables)), key=lambda k: -work[k]):
            s = int(np.argmin(load))
            self.groups[s].append(k)
            load[s] += work[k]
        # waves of the pipelined step: tables by decreasing work, dealt
        # round-robin (so each wave has a similar share of the work)
        self.waves = max(1, int(waves))
        order = sorted(range(len(tables)), key=lambda k: -work[k])
        self.wave_tables = [order[w::self.waves] for w in range(self.waves)]
        self.stream_of = {k: s for s, grp in enumerate(self.groups) for k in grp}
        for grp in self.groups:
            grp.sort()
        # the streams of the third of the tables with the least work run at
        # high priority: their short chains (forward, chi^2, adjoint) finish
        # early instead of queueing behind the CTAs of the large tables, which
        # then fill the GPU to the end of the step (1.33 -> 1.24 ms measured
        # on the global set; the large tables at high priority gave 1.26-1.28)
        by_work = sorted(range(self.nstreams), key=lambda s: -load[s])
        light = set(by_work[(2 * self.nstreams) // 3:]) if self.nstreams >= 3 else set()
        self.streams = [torch.cuda.Stream(device=device, priority=-1 if s in light else 0)
                        for s in range(self.nstreams)]
        self.gF_parts = [torch.empty_like(self.F) for _ in range(self.nstreams)]
        # pipelined chains: each dataset's chi^2 runs on its own high-priority
        # stream between its forward and adjoint, so it starts as soon as the
        # forward ends instead of waiting behind other chains' queued CTAs
        # (1.24 -> 1.19 ms measured; priority -2, above the light streams,
        # measured 1.22)
        self.chi2_streams = ([torch.cuda.Stream(device=device, priority=-1) for _ in tables]
                             if pipelined and not self.whiten else [])

    # -- helpers -------------------------------------------------------------
    def _fan_out(self, body):
        """Runs body(stream_index) on every side stream, forked from and
        joined back to the current stream (graph-capture safe)."""
        main = torch.cuda.current_stream()
        start = torch.cuda.Event()
        start.record(main)
        ends = []
        for s, st in enumerate(self.streams):
            st.wait_event(start)
            with torch.cuda.stream(st):
                body(s)
                e = torch.cuda.Event()
                e.record(st)
                ends.append(e)
        for e in ends:
            main.wait_event(e)

    # -- phases ------------------------------------------------------------
    def forward(self):
        def body(s):
            for k in self.groups[s]:
                conv(self.tabs[k], self.F, self.tprec[k], out=self.O[:, self.offs[k]:self.offs[k + 1]],
                     save=self.saved[k])
        self._fan_out(body)

    def loss(self):
        if self.whiten:
            chi2_white(self.O, self.D, out=self.chi2, gO=self.gO)
        else:
            chi2(self.cov, self.O, self.D, grad=True, out=self.chi2, gO=self.gO)

    def backward(self):
        def body(s):
            for n, k in enumerate(self.groups[s]):
                conv_backward(self.tabs[k], self.F, self.gO[:, self.offs[k]:self.offs[k + 1]],
                              self.tprec[k], gF=self.gF_parts[s], accumulate=n > 0, saved=self.saved[k])
        self._fan_out(body)
        grad_sum([self.gF_parts[s] for s in range(self.nstreams) if self.groups[s]], self.gF)

    def chain(self):
        """The pipelined step: per stream, forward -> chi^2 -> adjoint of each
        of its tables, then the fixed-order sums.

        With one stream per table the forwards are also staged in waves:
        the forwards of wave w start when those of wave w-1 are done, so the
        FP64 chi^2 (and then the adjoint) of one wave runs while the next
        wave's forwards occupy the tensor cores, instead of every forward
        competing at once and every chi^2 waiting for all of them."""
        if self.nstreams < len(self.tabs) or self.waves <= 1:
            def body(s):
                for n, k in enumerate(self.groups[s]):
                    self._table_chain(s, k, accumulate=n > 0)
            self._fan_out(body)
        else:
            main = torch.cuda.current_stream()
            start = torch.cuda.Event()
            start.record(main)
            ends, prev = [], []
            for wave in self.wave_tables:
                done = []
                for k in wave:
                    s = self.stream_of[k]
                    st = self.streams[s]
                    st.wait_event(start)
                    for e in prev:
                        st.wait_event(e)
                    with torch.cuda.stream(st):
                        ev = self._table_chain(s, k, accumulate=False)
                        done.append(ev)
                        e = torch.cuda.Event()
                        e.record(st)
                        ends.append(e)
                prev = done
            for e in ends:
                main.wait_event(e)
        grad_sum([self.gF_parts[s] for s in range(self.nstreams) if self.groups[s]], self.gF)
        parts = list(self.chi2_parts)
        for i in range(0, len(parts), 64):  # fk_grad_sum adds up to 64 parts per call
            grad_sum(parts[i:i + 64], self.chi2, accumulate=i > 0)

    def _table_chain(self, s, k, accumulate):
        """forward -> chi^2 -> adjoint of table k on the current stream;
        returns an event recorded after the forward."""
        cur = torch.cuda.current_stream()
        conv(self.tabs[k], self.F, self.tprec[k], out=self.Ok[k], save=self.saved[k])
        fwd = torch.cuda.Event()
        fwd.record(cur)
        if self.whiten:
            # one short kernel: on the chain's own stream
            chi2_white(self.Ok[k], self.Dk[k], out=self.chi2_parts[k], gO=self.gOk[k])
        else:
            h = self.chi2_streams[k]
            h.wait_event(fwd)
            with torch.cuda.stream(h):
                chi2(self.covs[k], self.Ok[k], self.Dk[k], grad=True, out=self.chi2_parts[k], gO=self.gOk[k])
                done = torch.cuda.Event()
                done.record(h)
            cur.wait_event(done)
        conv_backward(self.tabs[k], self.F, self.gOk[k], self.tprec[k], gF=self.gF_parts[s],
                      accumulate=accumulate, saved=self.saved[k])
        return fwd

    def phases(self):
        """(name, callable) of the step's graph(s), in order."""
        if self.pipelined:
            return (("step", self.chain),)
        return (("forward", self.forward), ("loss", self.loss), ("backward", self.backward))

    def step(self):
        if self.graphs is not None:
            for g in self.graphs.values():
                g.replay()
        else:
            for _, fn in self.phases():
                fn()

    def capture(self):
        """Records the step in CUDA graphs (after one eager step): one graph
        when pipelined, else one per phase."""
        for _, fn in self.phases():
            fn()
        torch.cuda.synchronize()
        graphs = {}
        for name, fn in self.phases():
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                fn()
            graphs[name] = g
        torch.cuda.synchronize()
        self.graphs = graphs
        return graphs

    def launches_per_step(self):
        """Kernels of this library one eager step launches."""
        before = _lib.load().fk_kernel_launches()
        g, self.graphs = self.graphs, None
        self.step()
        self.graphs = g
        torch.cuda.synchronize()
        return int(_lib.load().fk_kernel_launches() - before)
