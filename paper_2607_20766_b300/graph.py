"""CUDA-graph capture of a sequence of library calls.

A screening step is a handful of stream-ordered launches: closed-form and
sampled self-overlaps of both sets, then one persistent screen kernel whose
per-pair sample loop (fixed or adaptive) runs on the device. ``StepGraph``
records such a step once and replays it with a single graph launch; the
persistent kernels' work-queue counters become graph memory nodes, and the
outputs live in the graph's private memory pool, so ``out`` is refreshed in
place by every ``replay()``.

The library issues no host synchronisation and no blocking allocation
between the launches of these calls, which is what makes them capturable.
Launch variants (the autotuner's choice) are fixed at capture time: tune
first, then capture.
"""
from __future__ import annotations

import torch


class StepGraph:
    """Capture ``fn(*args, **kwargs)`` (library calls on the current CUDA
    stream) into a CUDA graph.

    ``out`` holds whatever ``fn`` returned during capture; each ``replay()``
    reruns every recorded launch on the current stream and rewrites those
    tensors. Inputs are read from the addresses seen at capture time, so
    update them in place (``copy_``) rather than rebinding them.
    """

    def __init__(self, fn, *args, warmup: int = 1, **kwargs):
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(warmup):  # first calls pay one-off set-up (function attributes, pools)
                fn(*args, **kwargs)
        torch.cuda.current_stream().wait_stream(side)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, capture_error_mode="thread_local"):
            self.out = fn(*args, **kwargs)

    def replay(self):
        self.graph.replay()
        return self.out
