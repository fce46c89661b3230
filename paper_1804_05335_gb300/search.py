"""Device buffers for one FDAS search and the calls that fill them.

A convenience layer over the C ABI: torch provides the device memory and the
stream, the library's kernels do all the work.  One ``Search`` holds, for a
series of n samples: the series, the normalised spectrum (n/2 bins), the
front-end workspace, the template bank, the f-fdot plane (K rows) and a
candidate buffer.
"""
from __future__ import annotations

import numpy as np
import torch

from . import (fdas_bank_floats, fdas_bank_rows, fdas_correlate, fdas_correlate_split,
               fdas_fused_threshold, fdas_make_templates,
               fdas_normalise, fdas_normalise_workspace_bytes, fdas_num_segments,
               fdas_num_templates, fdas_plane_width, fdas_threshold, params)


class Search:
    def __init__(self, n: int, L: int, M: int, zmin: int, zmax: int, zstep: int,
                 interbin: int = 1, median_block: int = 1024, thr: float = 20.0,
                 cap: int = 1 << 16, device="cuda", plane: bool = True):
        self.n = int(n)
        self.nb = self.n // 2
        self.p = params(L, M, zmin, zmax, zstep, interbin)
        self.K = fdas_num_templates(self.p)
        self.Kb = fdas_bank_rows(self.p)
        self.L, self.M = int(L), int(M)
        self.median_block = int(median_block)
        self.thr = float(thr)
        self.cap = int(cap)
        self.width = fdas_plane_width(self.p, self.nb)
        self.row_stride = (self.width + 3) // 4 * 4
        self.nseg = fdas_num_segments(self.p, self.nb)
        dev = torch.device(device)
        self.device = dev
        self.series = torch.empty(self.n, dtype=torch.float32, device=dev)
        self.spec = torch.empty(self.nb, dtype=torch.complex64, device=dev)
        self.work_bytes = fdas_normalise_workspace_bytes(self.n)
        self.work = torch.empty(max(self.work_bytes, 16), dtype=torch.uint8, device=dev)
        self.bank = torch.empty(fdas_bank_floats(self.p), dtype=torch.float32, device=dev)
        self.plane = (torch.empty(self.K * self.row_stride, dtype=torch.float32, device=dev)
                      if plane else None)
        self.cand = torch.empty(self.cap * 4, dtype=torch.int32, device=dev)
        self.count = torch.zeros(1, dtype=torch.int32, device=dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        self.fused = fdas_fused_threshold(self.thr, int(self.cand.data_ptr()), self.cap,
                                          int(self.count.data_ptr()))
        self.prec = 0   # DFT arithmetic of step() and stream() (FDAS_PREC_*)

    # ---- the calls ----
    def make_templates(self, stream=None):
        fdas_make_templates(self.p, self.bank, stream)

    def normalise(self, stream=None, series=None):
        fdas_normalise(self.series if series is None else series, self.n, self.median_block,
                       self.spec, self.work, self.work_bytes, stream)

    def correlate(self, fused: bool = True, spec=None, nb=None, stream=None, prec: int = 0):
        """The plane (and fused candidates); prec selects the DFT arithmetic
        (FDAS_PREC_*: 0 = FP32, 1 / 2 = FP16 / BF16 split tensor-core passes)."""
        args = (self.spec if spec is None else spec, self.nb if nb is None else nb, self.bank,
                self.plane, self.row_stride, self.fused if fused else None, self.status, stream)
        if prec == 0:
            fdas_correlate(self.p, *args)
        else:
            fdas_correlate_split(self.p, prec, *args)

    def threshold(self, want_peaks: bool = True, stream=None):
        fdas_threshold(self.plane, self.K, self.width, self.row_stride, self.thr,
                       1 if want_peaks else 0, self.cand, self.cap, self.count, self.status,
                       stream)

    def front(self, series=None):
        """The template bank and the normalised spectrum, which do not depend on
        each other: the bank is built on a second stream while the spectrum is
        formed on the current one, which then waits for both.  Returns the
        (start, end) events of the bank on its stream."""
        main = torch.cuda.current_stream(self.device)
        if not hasattr(self, "_side"):
            self._side = torch.cuda.Stream(self.device)
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        go = torch.cuda.Event()
        go.record(main)
        self._side.wait_event(go)
        with torch.cuda.stream(self._side):
            t0.record(self._side)
            self.make_templates()
            t1.record(self._side)
        self.normalise(series=series)
        main.wait_event(t1)
        return t0, t1

    def step(self, series=None):
        """One pass of the hot path on the current stream: bank and spectrum
        (overlapped, see front), plane + fused candidates."""
        self.front(series)
        self.correlate(True, prec=self.prec)

    def stream(self, host_series, host_out):
        """Search the pinned host series host_series[i] (n float32 each) one
        after another on the current CUDA stream, copying series i+1 to the
        device on a second stream while series i is searched.  The candidate
        count and list of series i land in the pinned int32 tensor host_out[i]
        (1 + 4*cap values: count, then (row, col, power bits, flags) per
        candidate); entries may alias when only the last result is wanted.
        Returns once everything is queued; synchronise before reading host_out."""
        main = torch.cuda.current_stream(self.device)
        if not hasattr(self, "_copy"):
            self._copy = torch.cuda.Stream(self.device)
            self._inbuf = [self.series, torch.empty_like(self.series)]
        loaded = [torch.cuda.Event(), torch.cuda.Event()]
        start = torch.cuda.Event()
        start.record(main)                 # earlier work on the input buffers
        self._copy.wait_event(start)
        free = [None, None]
        for i, hs in enumerate(host_series):
            j = i & 1
            with torch.cuda.stream(self._copy):
                if free[j] is not None:
                    self._copy.wait_event(free[j])   # series i-2 has been read
                self._inbuf[j].copy_(hs, non_blocking=True)
                loaded[j].record(self._copy)
            main.wait_event(loaded[j])
            self.front(series=self._inbuf[j])
            free[j] = torch.cuda.Event()
            free[j].record(main)
            self.correlate(True, prec=self.prec)
            host_out[i][:1].copy_(self.count, non_blocking=True)
            host_out[i][1:].copy_(self.cand, non_blocking=True)

    # ---- views ----
    def plane2d(self) -> torch.Tensor:
        return self.plane.view(self.K, self.row_stride)[:, : self.width]

    def candidates(self):
        """(rows, cols, power, flags, total) sorted by (row, col); syncs."""
        total = int(self.count.item())
        k = min(total, self.cap)
        c = self.cand[: 4 * k].view(k, 4).cpu().numpy()
        rows, cols = c[:, 0].copy(), c[:, 1].copy()
        pw = c[:, 2].copy().view(np.float32)
        fl = c[:, 3].copy()
        o = np.lexsort((cols, rows))
        return rows[o], cols[o], pw[o], fl[o], total
