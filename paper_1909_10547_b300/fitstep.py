"""One gradient-descent fit step over a set of device-resident FK tables.

The step is the hot path of the paper's fit (Sec. 2: gradient descent; Sec. 3:
the convolution is the most time-consuming operation):

  forward   O[:, off_k : off_k + n_k] = conv(table_k, F)   for every dataset k
  loss      chi2[r] = (O_r - D)^T C^{-1} (O_r - D),  gO = d chi2 / d O  (FP64)
  backward  gF = sum_k conv_backward(table_k, F, gO[:, off_k : off_k + n_k])

All three run in libfk.so kernels.  The tables are spread over `nstreams`
CUDA streams (balanced by their work) so that small tables run side by side
on the 148 SMs: in the forward each table writes its own columns of O; in the
backward each stream accumulates into its own gradient buffer and
fk_grad_sum adds the buffers in a fixed order, so the result does not depend
on how the streams interleave.  capture() records each phase in a CUDA graph
(the streams become parallel branches), so a step costs three graph launches.
"""
import numpy as np
import torch

from . import Cov, Table, _lib, chi2, conv, conv_backward, grad_sum

NFL = 14


class GlobalFit:
    def __init__(self, tables, F, cov_blocks, D, prec="fp32", store=None, device="cuda",
                 nstreams=8):
        """tables: workloads.DisTable/HadTable list sharing one x grid;
        F: [R][14][nxg] replicas (host numpy); cov_blocks: one SPD block per
        table; D: [sum ndata] pseudo-data."""
        self.prec = prec
        io = torch.float64 if prec == "fp64" else torch.float32
        if store is None:
            store = ("fp64", "fp32") if prec in ("fp64", "fp32") else (prec,)
        self.tabs = []
        for t in tables:
            st = store if hasattr(t, "ca") else tuple(p for p in store if p in ("fp64", "fp32")) or ("fp32",)
            self.tabs.append(Table.from_workload(t, st))
        self.kinds = ["had" if hasattr(t, "ca") else "dis" for t in tables]
        # DIS tables are small linear contractions: in the reduced modes they
        # run in FP32 on the CUDA cores (the tensor-core modes are hadronic)
        self.tprec = [prec if (k == "had" or prec in ("fp64", "fp32")) else "fp32" for k in self.kinds]
        nd = [t.ndata for t in tables]
        self.offs = np.concatenate([[0], np.cumsum(nd)]).astype(int)
        self.ntot = int(self.offs[-1])
        self.R = F.shape[0]
        self.nxg = F.shape[2]
        self.io = io
        self.cov = Cov(cov_blocks)
        assert self.cov.n == self.ntot
        self.D = torch.tensor(np.asarray(D, np.float64), device=device)
        self.F = torch.tensor(np.asarray(F), dtype=io, device=device)
        self.O = torch.empty((self.R, self.ntot), dtype=io, device=device)
        self.gO = torch.empty_like(self.O)
        self.gF = torch.empty_like(self.F)
        self.chi2 = torch.empty(self.R, dtype=torch.float64, device=device)
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
        self.flops = {"forward": fwd, "loss": 2 * int(sum(n * n for n in nd)) * self.R, "backward": bwd}
        # streams: greedy assignment of tables (largest first) to the least
        # loaded stream
        self.nstreams = max(1, min(nstreams, len(tables)))
        load = [0] * self.nstreams
        self.groups = [[] for _ in range(self.nstreams)]
        for k in sorted(range(len(tables)), key=lambda k: -work[k]):
            s = int(np.argmin(load))
            self.groups[s].append(k)
            load[s] += work[k]
        for grp in self.groups:
            grp.sort()
        self.streams = [torch.cuda.Stream(device=device) for _ in range(self.nstreams)]
        self.gF_parts = [torch.empty_like(self.F) for _ in range(self.nstreams)]

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
                conv(self.tabs[k], self.F, self.tprec[k], out=self.O[:, self.offs[k]:self.offs[k + 1]])
        self._fan_out(body)

    def loss(self):
        chi2(self.cov, self.O, self.D, grad=True, out=self.chi2, gO=self.gO)

    def backward(self):
        def body(s):
            for n, k in enumerate(self.groups[s]):
                conv_backward(self.tabs[k], self.F, self.gO[:, self.offs[k]:self.offs[k + 1]],
                              self.tprec[k], gF=self.gF_parts[s], accumulate=n > 0)
        self._fan_out(body)
        grad_sum([self.gF_parts[s] for s in range(self.nstreams) if self.groups[s]], self.gF)

    def step(self):
        if self.graphs is not None:
            for g in self.graphs.values():
                g.replay()
        else:
            self.forward()
            self.loss()
            self.backward()

    def capture(self):
        """Records the three phases in CUDA graphs (after one eager step)."""
        self.forward()
        self.loss()
        self.backward()
        torch.cuda.synchronize()
        graphs = {}
        for name, fn in (("forward", self.forward), ("loss", self.loss), ("backward", self.backward)):
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
