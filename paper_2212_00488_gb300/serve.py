"""Serving form: a continuous-batching request loop over device-resident frames.

Requests (a left/right pair of uint8 CUDA tensors and Dmax) are admitted
against a device-memory budget, grouped as they arrive into batches for
``stereo_compute_batch`` and run on one of several lanes (a library context
with its own CUDA stream each), so a batch formed while others are still on
the GPU starts at once and overlaps them. A request's result is the float
disparity map on the device; it is the same whether the request ran alone or
in a mix (the batch path is exact per frame).
"""
from __future__ import annotations

import collections
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field

import torch

from . import _lib
from .stereo import Stereo, stream_handle


def frame_bytes(W: int, H: int, dmax: int, params=None) -> int:
    """Device bytes one request holds while it runs: the library's batch
    workspace for the frame (stereo_job_bytes) plus its float output map.
    params: the lanes' stereo_params (None: the library's defaults)."""
    ws = _lib.stereo_job_bytes(params, W, H, dmax)
    if ws == 0:
        raise ValueError(f"the library rejects a {W}x{H} frame with Dmax {dmax}")
    return ws + W * H * 4


class Admission:
    """First-come first-served admission against a byte budget."""

    def __init__(self, cap_bytes: int):
        if cap_bytes <= 0:
            raise ValueError("cap must be positive")
        self.cap = cap_bytes
        self.used = 0
        self.peak = 0
        self.waiting = collections.deque()

    def offer(self, item, nbytes: int):
        if nbytes > self.cap:
            raise ValueError(f"request needs {nbytes} bytes, more than the cap of {self.cap}")
        self.waiting.append((item, nbytes))

    def admit(self):
        """Admitted items, in arrival order, while the budget allows."""
        out = []
        while self.waiting and self.used + self.waiting[0][1] <= self.cap:
            item, nbytes = self.waiting.popleft()
            self.used += nbytes
            self.peak = max(self.peak, self.used)
            out.append((item, nbytes))
        return out

    def release(self, nbytes: int):
        self.used -= nbytes
        assert self.used >= 0


@dataclass
class Request:
    left: torch.Tensor
    right: torch.Tensor
    dmax: int
    future: Future
    t_submit: float
    ready: torch.cuda.Event | None = None     # the inputs are complete on the caller's stream
    nbytes: int = 0
    out: torch.Tensor | None = None
    t_done: float = 0.0


@dataclass
class _Lane:
    st: Stereo
    stream: torch.cuda.Stream
    event: torch.cuda.Event
    batch: list = field(default_factory=list)


class StereoServer:
    """Continuous batching on one GPU.

    mem_cap_bytes bounds the device memory the server holds for requests.
    Each of the `lanes` lanes (the batches that may be on the GPU at once) owns
    an equal share of it: its library context is created with that share as
    its memory cap, so the library itself refuses a batch workspace beyond it,
    and a lane's batch takes requests only while their bytes (frame_bytes:
    workspace plus output map) fit the share. Admission counts the same bytes
    against the whole cap. A request larger than one share is rejected at
    submit. max_batch caps a batch (at most 32). tile fixes the fused kernel's
    tile shape; None lets the library's autotuner time the shapes for each new
    batch signature, which costs a few ms the first time a signature appears.
    A batch whose fused kernel gave up a bounded wait (STEREO_ETIMEOUT) fails
    its requests' futures with the library's error.
    """

    def __init__(self, device: int = 0, mem_cap_bytes: int = 8 << 30, lanes: int = 2, max_batch: int = 16,
                 tile: int | None = None, **params):
        self.device = torch.device("cuda", device)
        self.max_batch = min(max_batch, 32)
        self.adm = Admission(mem_cap_bytes)
        self.lane_cap = mem_cap_bytes // lanes
        self.ready = collections.deque()          # admitted, not yet on a lane
        self.lanes = []
        for _ in range(lanes):
            s = torch.cuda.Stream(self.device)
            ln = _Lane(Stereo(device, mem_cap_bytes=self.lane_cap, **params), s, torch.cuda.Event())
            if tile is not None:
                _lib.stereo_set_tile(ln.st.ctx, tile)
            self.lanes.append(ln)
        self.params = self.lanes[0].st.params
        self.lock = threading.Condition()
        self.latencies = []
        self.completed = 0
        self.failed = 0
        self.batches = 0
        self._stop = False
        self._error = None
        self.thread = threading.Thread(target=self._loop, daemon=True)
        self.thread.start()

    def submit(self, left: torch.Tensor, right: torch.Tensor, dmax: int) -> Future:
        if left.dtype != torch.uint8 or left.dim() != 3 or left.shape != right.shape or left.device != self.device:
            raise ValueError("left and right must be uint8 [H, W, 3] tensors on the server's device")
        H, W = int(left.shape[0]), int(left.shape[1])
        fut = Future()
        ev = torch.cuda.Event()
        ev.record(torch.cuda.current_stream(self.device))
        req = Request(left, right, dmax, fut, time.perf_counter(), ev)
        with self.lock:
            if self._error is not None:
                raise RuntimeError("server stopped") from self._error
            req.nbytes = frame_bytes(W, H, dmax, self.params)
            if req.nbytes > self.lane_cap:
                raise ValueError(f"request needs {req.nbytes} bytes, more than a lane's share of "
                                 f"{self.lane_cap}")
            self.adm.offer(req, req.nbytes)
            self.lock.notify()
        return fut

    def close(self):
        with self.lock:
            self._stop = True
            self.lock.notify()
        self.thread.join()
        for ln in self.lanes:
            ln.st.close()

    def stats(self):
        lat = sorted(self.latencies)

        def q(p):
            return lat[min(len(lat) - 1, int(p * len(lat)))] if lat else None
        return {"completed": self.completed, "failed": self.failed, "batches": self.batches,
                "p50_ms": q(0.50) and q(0.50) * 1e3, "p99_ms": q(0.99) and q(0.99) * 1e3,
                "peak_admitted_bytes": self.adm.peak, "cap_bytes": self.adm.cap}

    # ------------------------------------------------------------ scheduler
    def _finish(self, ln: _Lane):
        # the lane's stream is idle: reading the context's error word costs a
        # small copy, and a bounded wait that gave up fails the whole batch
        err = None
        try:
            _lib.stereo_sync(ln.st.ctx)
        except _lib.StereoError as e:
            err = e
        now = time.perf_counter()
        for req in ln.batch:
            req.t_done = now
            self.adm.release(req.nbytes)
            if err is None:
                self.latencies.append(now - req.t_submit)
                req.future.set_result(req.out)
            else:
                req.future.set_exception(err)
        if err is None:
            self.completed += len(ln.batch)
        else:
            self.failed += len(ln.batch)
        ln.batch = []

    def _launch(self, ln: _Lane, reqs):
        jobs = []
        with torch.cuda.stream(ln.stream):
            for req in reqs:
                ln.stream.wait_event(req.ready)
                H, W = int(req.left.shape[0]), int(req.left.shape[1])
                req.out = torch.empty((H, W), dtype=torch.float32, device=self.device)
                jobs.append(_lib.stereo_job(req.left.data_ptr(), req.right.data_ptr(), W, H, req.dmax,
                                            req.out.data_ptr(), None, None, None))
            _lib.stereo_compute_batch(ln.st.ctx, jobs, stream_handle(ln.stream))
            ln.event.record(ln.stream)
        ln.batch = list(reqs)
        self.batches += 1

    def _loop(self):
        torch.cuda.set_device(self.device)
        try:
            while True:
                with self.lock:
                    for ln in self.lanes:
                        if ln.batch and ln.event.query():
                            self._finish(ln)
                    self.ready.extend(r for r, _ in self.adm.admit())
                    for ln in self.lanes:
                        if not ln.batch and self.ready:
                            # requests in arrival order while they fit the lane's share
                            take, used = [], 0
                            while (self.ready and len(take) < self.max_batch
                                   and used + self.ready[0].nbytes <= self.lane_cap):
                                used += self.ready[0].nbytes
                                take.append(self.ready.popleft())
                            self._launch(ln, take)
                    busy = any(ln.batch for ln in self.lanes)
                    if self._stop and not busy and not self.ready and not self.adm.waiting:
                        return
                    if not busy and not self.ready and not self.adm.waiting:
                        self.lock.wait(timeout=0.01)
                if busy:
                    time.sleep(20e-6)
        except BaseException as e:           # surface failures to every waiting request
            with self.lock:
                self._error = e
                for ln in self.lanes:
                    for req in ln.batch:
                        req.future.set_exception(e)
                    ln.batch = []
                for req in self.ready:
                    req.future.set_exception(e)
                while self.adm.waiting:
                    req, _ = self.adm.waiting.popleft()
                    req.future.set_exception(e)
