"""Batched, graph-captured, autotuned evaluation of many requests.

A request is (PDF, member, pid subset of up to 16 pids, x, Q^2, out) with
device tensors; ``Batch.prepare`` tunes the persistent launch (block size,
points per thread, shared-memory staging) and captures it in a CUDA graph;
``Batch.run`` replays it on the current stream.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from ._lib import BatchDesc, check, lib
from .pdf import PDF, _stream


class Batch:
    def __init__(self, requests, autotune=True):
        """``requests``: iterable of (pdf, member, pids, x, q2, out) with
        float64 CUDA tensors x, q2 [n] and out [n][len(pids)]."""
        self.requests = list(requests)
        n = len(self.requests)
        arr = (BatchDesc * n)()
        self._keep = []
        dev = None
        for i, (pdf, member, pids, x, q2, out) in enumerate(self.requests):
            p = np.atleast_1d(np.asarray(pids, dtype=np.int32))
            assert 1 <= p.size <= 16
            assert x.dtype == torch.float64 and x.is_contiguous() and q2.is_contiguous()
            assert out.shape == (x.numel(), p.size) and out.is_contiguous()
            arr[i].grid = pdf.handle
            arr[i].member = int(member)
            arr[i].n_pid = p.size
            for k in range(p.size):
                arr[i].pids[k] = int(p[k])
            arr[i].x = x.data_ptr()
            arr[i].q2 = q2.data_ptr()
            arr[i].n = x.numel()
            arr[i].out = out.data_ptr()
            self._keep += [x, q2, out, pdf]
            dev = pdf.device
        self.device = dev
        h = C.c_void_p()
        check("pdf_batch_prepare", lib().pdf_batch_prepare(arr, n, int(bool(autotune)),
                                                           _stream(dev), C.byref(h)))
        self.handle = h

    def run(self):
        check("pdf_batch_run", lib().pdf_batch_run(self.handle, _stream(self.device)))

    def info(self):
        b, q, s, c = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        ms = C.c_float()
        check("pdf_batch_info", lib().pdf_batch_info(self.handle, C.byref(b), C.byref(q), C.byref(s),
                                                     C.byref(c), C.byref(ms)))
        return {"block": b.value, "qpt": q.value, "stage": s.value, "ctas": c.value,
                "tuned_ms": ms.value}

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().pdf_batch_free(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
