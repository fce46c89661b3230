"""Batched search over many series of uneven length (dispersion trials).

One BatchSearch holds every trial's series and spectrum, one template bank,
and a reusable pool for f-fdot planes.  Trials are grouped into waves whose
planes fit the pool; each wave is one persistent fdas_correlate_batched
launch with the threshold fused, so the candidates of every trial come out
while the pool is reused.  The whole batch (bank, every front end, every
wave) can be captured once into a CUDA graph and replayed.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import (fdas_bank_floats, fdas_batch_plan, fdas_bluestein_bytes, fdas_bluestein_prepare,
               fdas_correlate_batched, fdas_fused_threshold, fdas_make_templates,
               fdas_normalise, fdas_normalise_prepared, fdas_normalise_workspace_bytes, fdas_num_templates,
               fdas_plane_width, fdas_trial, params)


class BatchSearch:
    def __init__(self, ns, L: int, M: int, zmin: int, zmax: int, zstep: int, interbin: int = 1,
                 median_block: int = 1024, thr: float = 20.0, cap_per_wave: int = 1 << 16,
                 pool_bytes: int = 32 << 30, ctas_per_sm: int = 0, templates_per_block: int = 0,
                 prepare_chirps: bool = True, device="cuda"):
        self.ns = [int(n) for n in ns]
        self.p = params(L, M, zmin, zmax, zstep, interbin)
        self.K = fdas_num_templates(self.p)
        self.L, self.M = int(L), int(M)
        self.median_block = int(median_block)
        self.thr = float(thr)
        self.ctas_per_sm = int(ctas_per_sm)
        self.templates_per_block = int(templates_per_block)
        dev = torch.device(device)
        self.device = dev
        nbs = [n // 2 for n in self.ns]
        self.widths = [fdas_plane_width(self.p, nb) for nb in nbs]
        self.strides = [(w + 3) // 4 * 4 for w in self.widths]
        self.plane_points = int(sum(self.K * w for w in self.widths))
        # series and spectra, one flat buffer each (offsets keep 16-byte alignment)
        self.s_off = np.concatenate([[0], np.cumsum(self.ns)]).astype(np.int64)
        self.series = torch.empty(int(self.s_off[-1]), dtype=torch.float32, device=dev)
        self.b_off = np.concatenate([[0], np.cumsum(nbs)]).astype(np.int64)
        self.spec = torch.empty(int(self.b_off[-1]), dtype=torch.complex64, device=dev)
        self.work_bytes = max(fdas_normalise_workspace_bytes(n) for n in self.ns)
        self.work = torch.empty(self.work_bytes, dtype=torch.uint8, device=dev)
        # Bluestein kernel spectra, one per distinct length that is not a power
        # of two, computed once here (input-independent) and read by every run
        self.chirp_off = {}
        if prepare_chirps:
            off = 0
            for n in sorted(set(self.ns)):
                cb = fdas_bluestein_bytes(n)
                if cb:
                    self.chirp_off[n] = off
                    off += cb
            self.chirps = torch.empty(max(off, 16), dtype=torch.uint8, device=dev)
            for n, o in self.chirp_off.items():
                fdas_bluestein_prepare(n, int(self.chirps.data_ptr()) + o, self.work,
                                       self.work_bytes)
        self.bank = torch.empty(fdas_bank_floats(self.p), dtype=torch.float32, device=dev)
        # waves: consecutive trials whose planes fit the pool
        sizes = [self.K * st * 4 for st in self.strides]
        if max(sizes) > pool_bytes:
            raise ValueError("pool_bytes smaller than one plane")
        self.waves = []
        cur, used = [], 0
        for i, sz in enumerate(sizes):
            if used + sz > pool_bytes and cur:
                self.waves.append(cur)
                cur, used = [], 0
            cur.append(i)
            used += sz
        if cur:
            self.waves.append(cur)
        pool_floats = max(sum(sizes[i] for i in w) for w in self.waves) // 4
        self.pool = torch.empty(pool_floats, dtype=torch.float32, device=dev)
        self.plane_off = {}
        self.wave_tables = []
        self.wave_items = []
        for w in self.waves:
            arr = (fdas_trial * len(w))()
            off = 0
            for j, i in enumerate(w):
                self.plane_off[i] = off
                arr[j].spec = int(self.spec.data_ptr()) + 8 * int(self.b_off[i])
                arr[j].nb = nbs[i]
                arr[j].plane = int(self.pool.data_ptr()) + 4 * off
                arr[j].row_stride = self.strides[i]
                off += self.K * self.strides[i]
            items = fdas_batch_plan(self.p, arr)
            raw = np.frombuffer(bytes(arr), dtype=np.uint8).copy()
            self.wave_tables.append(torch.from_numpy(raw).to(dev))
            self.wave_items.append(items)
        self.cap = int(cap_per_wave)
        self.cand = [torch.empty(4 * self.cap, dtype=torch.int32, device=dev) for _ in self.waves]
        self.count = torch.zeros(len(self.waves), dtype=torch.int32, device=dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        self.fused = [fdas_fused_threshold(self.thr, int(c.data_ptr()), self.cap,
                                           int(self.count.data_ptr()) + 4 * k)
                      for k, c in enumerate(self.cand)]
        self.graph = None

    # ---- inputs and views ----
    def set_series(self, i: int, x) -> None:
        self.series[int(self.s_off[i]):int(self.s_off[i + 1])].copy_(torch.as_tensor(x))

    def spec_of(self, i: int) -> torch.Tensor:
        return self.spec[int(self.b_off[i]):int(self.b_off[i + 1])]

    def plane_of(self, i: int) -> torch.Tensor:
        """Trial i's plane; valid only until the next wave reuses the pool."""
        o = self.plane_off[i]
        return self.pool[o: o + self.K * self.strides[i]].view(self.K, self.strides[i])[
            :, : self.widths[i]]

    # ---- the work ----
    def front(self, stream=None) -> None:
        fdas_make_templates(self.p, self.bank, stream)
        for i, n in enumerate(self.ns):
            chirp = (int(self.chirps.data_ptr()) + self.chirp_off[n]) if n in self.chirp_off else None
            if chirp is None and (n & (n - 1)):
                # no prepared spectrum: fdas_normalise computes it itself
                fdas_normalise(int(self.series.data_ptr()) + 4 * int(self.s_off[i]), n,
                               self.median_block,
                               int(self.spec.data_ptr()) + 8 * int(self.b_off[i]),
                               self.work, self.work_bytes, stream)
                continue
            fdas_normalise_prepared(int(self.series.data_ptr()) + 4 * int(self.s_off[i]), n,
                                    self.median_block,
                                    int(self.spec.data_ptr()) + 8 * int(self.b_off[i]),
                                    self.work, self.work_bytes, chirp, stream)

    def correlate_wave(self, k: int, stream=None) -> None:
        fdas_correlate_batched(self.p, self.wave_tables[k], len(self.waves[k]),
                               self.wave_items[k], self.bank, self.fused[k], self.ctas_per_sm,
                               self.status, stream, self.templates_per_block)

    def run(self, stream=None) -> None:
        self.front(stream)
        for k in range(len(self.waves)):
            self.correlate_wave(k, stream)

    def capture(self) -> None:
        """Run once, then capture the whole batch into one CUDA graph."""
        self.run()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                self.run(stream=s)
        torch.cuda.current_stream().wait_stream(s)
        self.graph = g

    def replay(self) -> None:
        self.graph.replay()

    def candidates(self):
        """List of (trial, rows, cols, power) per trial, sorted; syncs."""
        out = {i: [] for i in range(len(self.ns))}
        counts = self.count.cpu().numpy()
        for k, w in enumerate(self.waves):
            c = min(int(counts[k]), self.cap)
            a = self.cand[k][: 4 * c].view(c, 4).cpu().numpy()
            for row, col, pw, fl in a:
                # flags carry the trial's index within this wave's table
                out[w[int(fl) >> 8]].append((int(row), int(col),
                                             float(np.int32(pw).view(np.float32))))
        res = {}
        for i, lst in out.items():
            lst.sort()
            res[i] = (np.array([x[0] for x in lst], np.int32), np.array([x[1] for x in lst], np.int32),
                      np.array([x[2] for x in lst], np.float32))
        return res, counts
