"""Host-to-host pipelining of an element-wise program over chunks.

A program whose inputs and outputs live in host memory (pinned, for
asynchronous copies) pays for the uploads and downloads as well as the
kernel.  ChunkPipeline cuts the arrays into chunks and deals the chunks
round-robin to several runtime contexts, each with its own CUDA stream: while
one chunk's results come back, the next chunks are uploaded and computed on
the other streams, so the host-to-device copies, the kernels and the
device-to-host copies of different chunks overlap.

Every chunk runs the same fused window (the program is traced once per
context and chunk size, then memoised), so the results are those of running
the program on each chunk alone; for an element-wise program that is the
result of running it on the whole arrays.
"""
from __future__ import annotations

from collections import deque

import numpy as np

from . import arrays as A


class ChunkPipeline:
    """fn(*inputs) -> tuple of outputs, over `nctx` contexts.

    runtimes: the contexts (one stream each); chunk: elements per chunk;
    in_dtypes: dtypes of the 1-D inputs.  Device buffers for one chunk of
    every input are kept per context and size, so steady use allocates
    nothing but the outputs' stream-ordered memory.
    """

    def __init__(self, runtimes, fn, chunk: int, in_dtypes):
        if not runtimes:
            raise ValueError("at least one runtime context")
        self.rts = list(runtimes)
        self.fn = fn
        self.chunk = int(chunk)
        self.in_dtypes = [np.dtype(d) for d in in_dtypes]
        self._slots = {}

    def _inputs(self, k: int, size: int):
        key = (k, size)
        if key not in self._slots:
            rt = self.rts[k]
            self._slots[key] = [rt.empty((size,), d) for d in self.in_dtypes]
        return self._slots[key]

    def run(self, host_in, host_out) -> None:
        """Computes host_out[j][:] = fn(host_in...)[j] for 1-D host arrays of
        one length (pinned memory lets the copies overlap)."""
        n = len(host_in[0])
        nctx = len(self.rts)
        inflight = deque()

        def retire():
            k, outs, lo, hi = inflight.popleft()
            for dev, host in zip(outs, host_out):
                dev.read_into(host[lo:hi])       # waits for this context's stream only

        for idx, lo in enumerate(range(0, n, self.chunk)):
            hi = min(n, lo + self.chunk)
            k = idx % nctx
            if len(inflight) == nctx:
                retire()
            ins = self._inputs(k, hi - lo)
            for dev, host in zip(ins, host_in):
                dev.write(host[lo:hi])           # asynchronous from pinned memory
            outs = self.fn(*ins)
            self.rts[k].flush()
            inflight.append((k, outs, lo, hi))
        while inflight:
            retire()


def pipelined_runtimes(nctx: int, device: int = 0, **kw):
    """nctx runtime contexts on one device, each creating its own stream."""
    return [A.Runtime(device=device, **kw) for _ in range(nctx)]
