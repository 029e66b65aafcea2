"""Serving loop: continuous batching of exact-match queries on one GPU.

Requests arrive at any time (``Server.submit``); each names a resident
corpus (a device text loaded once) or carries its own text.  A scheduler
thread repeatedly

  1. retires finished batches (their stream's event has fired): reads the
     counts and positions copied back on that stream, completes the
     requests' futures, re-queues any request whose output was truncated
     with its exact count as the new capacity, and returns its memory to
     the budget;
  2. admits pending requests while their device memory (own text, plan,
     output capacity, count) plus the batch workspace fits the budget,
     taking requests of one length class (floor(log2 m): the class of the
     oldest pending request) in arrival order, up to ``max_batch`` requests
     and ``max_batch_scan_bytes`` of text to scan (which bounds the GPU
     time of a batch, and so the wait of the requests behind it);
  3. launches the batch on a free stream with ``sm_search_batch_async``
     (one persistent launch per kernel family, in memory the server owns),
     followed by the copy of the counts and an event; once the counts are
     on the host, exactly the valid positions of each request are copied
     back (a second event): small results through a per-stream pinned
     staging buffer, large ones straight into a pinned block of their own
     that the client receives without a copy (``PinnedPool``).

Up to ``streams`` batches are in flight at once, so requests that arrive
while others run are admitted as slots and memory free up and their work
overlaps on the device.  Every request records arrival and completion times
(p50 / p99 latency).  ``Policy`` holds the host-side decisions (admission,
length classes, batch size) and needs no GPU.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import ctypes
import itertools
import threading
import time
import weakref
from dataclasses import dataclass, field

import numpy as np


def length_class(m: int) -> int:
    """floor(log2 m) capped at 11 (the tuning table's m bucket)."""
    return min(11, max(0, int(m).bit_length() - 1))


@dataclass
class Request:
    rid: int
    pattern: bytes
    corpus: str | None
    text: np.ndarray | None
    cap: int
    t_arrival: float
    future: cf.Future = field(default_factory=cf.Future)
    attempts: int = 0

    @property
    def m(self) -> int:
        return len(self.pattern)


def plan_bytes_estimate(m: int) -> int:
    """Upper bound of a plan's device bytes (header, masks, pattern, q-gram
    table, border table, and for m > 16 an automaton of at most 32 KiB),
    for admission only."""
    return 4096 + 64 * m + (32768 if m > 16 else 0)


class Policy:
    """Host-side scheduling decisions.  No GPU work."""

    def __init__(self, budget_bytes: int, max_batch: int = 512, max_wait: float = 0.0005,
                 corpus_bytes=None, workspace_per_batch: int = 128 << 20,
                 max_batch_out_bytes: int = 1 << 62, max_batch_scan_bytes: int = 1 << 62,
                 scan_backlog: int = 512):
        self.budget = int(budget_bytes)
        self.max_batch_out = int(max_batch_out_bytes)
        # Text bytes one batch may scan: bounds a batch's GPU time, so a
        # request never waits behind hundreds of long scans.  The bound
        # grows by one step per `scan_backlog` pending requests: a backlog
        # is drained in large batches (throughput), a short queue in small
        # ones (latency).
        self.max_batch_scan = int(max_batch_scan_bytes)
        self.scan_backlog = max(1, int(scan_backlog))
        self.max_batch = int(max_batch)
        self.max_wait = float(max_wait)
        self.used = 0
        self.pending: collections.deque[Request] = collections.deque()
        self.corpus_bytes = dict(corpus_bytes or {})
        self.workspace_per_batch = int(workspace_per_batch)

    def need(self, r: Request) -> int:
        own = 0 if r.text is None else len(r.text)
        return own + plan_bytes_estimate(r.m) + 8 * max(r.cap, 1) + 8

    def scan_bytes(self, r: Request) -> int:
        return len(r.text) if r.text is not None else int(self.corpus_bytes.get(r.corpus, 0))

    def push(self, r: Request, front: bool = False) -> None:
        (self.pending.appendleft if front else self.pending.append)(r)

    def ready(self, now: float, busy: int) -> bool:
        """Launch now?  A full batch, an old enough request, or an idle GPU."""
        if not self.pending:
            return False
        return (len(self.pending) >= self.max_batch or busy == 0
                or now - self.pending[0].t_arrival >= self.max_wait)

    def take(self) -> tuple[list[Request], int, list[Request]]:
        """Pick the next batch: requests of the oldest request's length class,
        in arrival order, while they fit the budget.  Returns (batch, bytes
        reserved, requests rejected because they can never fit)."""
        rejected, batch = [], []
        while self.pending and self.need(self.pending[0]) + self.workspace_per_batch > self.budget:
            rejected.append(self.pending.popleft())
        if not self.pending:
            return [], 0, rejected
        cls = length_class(self.pending[0].m)
        reserved = self.workspace_per_batch
        if self.used + reserved > self.budget:
            return [], 0, rejected
        keep = collections.deque()
        out_bytes = scan = 0
        scan_cap = self.max_batch_scan * (1 + len(self.pending) // self.scan_backlog)
        while self.pending and len(batch) < self.max_batch:
            r = self.pending.popleft()
            need = self.need(r)
            fits_out = not batch or out_bytes + 8 * r.cap <= self.max_batch_out
            fits_scan = not batch or scan + self.scan_bytes(r) <= scan_cap
            if length_class(r.m) == cls and self.used + reserved + need <= self.budget and fits_out and fits_scan:
                batch.append(r)
                reserved += need
                out_bytes += 8 * r.cap
                scan += self.scan_bytes(r)
            else:
                keep.append(r)
                if self.used + reserved + need > self.budget and length_class(r.m) == cls:
                    break  # memory is full: later requests of this class wait too
        keep.extend(self.pending)
        self.pending = keep
        if not batch:
            return [], 0, rejected
        self.used += reserved
        return batch, reserved, rejected

    def release(self, nbytes: int) -> None:
        self.used -= nbytes


class PinnedPool:
    """Pinned host blocks for large results, recycled when the result they
    back is freed.  Block sizes are 1, 1.25, 1.5 or 1.75 times a power of
    two (at least 1 MiB), so a block wastes under a fifth of its bytes; a
    result is handed out as a numpy array over its block, and a
    finalizer puts the block back on its free list once that array and every
    view of it are gone, so steady-state serving allocates no pinned
    memory."""

    MIN_BYTES = 1 << 20

    def __init__(self, torch, max_bytes: int = 4 << 30):
        self._torch = torch
        self._free = collections.defaultdict(list)
        self._lock = threading.Lock()
        self.allocated_bytes = 0
        self.max_bytes = int(max_bytes)

    @classmethod
    def size_class(cls, nbytes: int) -> int:
        """Smallest block size (k/4 * 2**e, k in 4..7) holding nbytes."""
        n = max(int(nbytes), cls.MIN_BYTES)
        e = (n - 1).bit_length() - 1          # 2**e < n <= 2**(e+1)
        for k in (5, 6, 7, 8):
            if (k << e) >> 2 >= n:
                return (k << e) >> 2
        return 1 << (e + 1)

    def take(self, nbytes: int):
        """A free block of at least nbytes (the smallest one up to twice the
        size class), else a new block of the size class, else (the pool is
        at max_bytes) (None, 0)."""
        size = self.size_class(nbytes)
        with self._lock:
            fits = [c for c, blocks in self._free.items() if blocks and size <= c <= 2 * size]
            if fits:
                c = min(fits)
                return self._free[c].pop(), c
            if self.allocated_bytes + size > self.max_bytes:
                return None, 0
            self.allocated_bytes += size
        return self._torch.empty(size, dtype=self._torch.uint8, pin_memory=True), size

    def _give(self, block, cls: int) -> None:
        with self._lock:
            self._free[cls].append(block)

    _shared = None

    @classmethod
    def shared(cls, torch, max_bytes: int):
        """The process-wide pool (servers of one process share warm blocks),
        allowed at least max_bytes."""
        if cls._shared is None:
            cls._shared = cls(torch, max_bytes)
        cls._shared.max_bytes = max(cls._shared.max_bytes, int(max_bytes))
        return cls._shared

    def view(self, block, cls: int, count: int) -> np.ndarray:
        """The first `count` 64-bit values of `block` as a uint64 array.
        The array is made over a ctypes buffer, which every numpy view of it
        references (numpy collapses view chains to the buffer's owner); the
        finalizer on that buffer keeps the block until the last view is
        gone, then returns it to the pool."""
        buf = (ctypes.c_uint64 * max(count, 1)).from_address(block.data_ptr())
        weakref.finalize(buf, self._give, block, cls)
        return np.frombuffer(buf, dtype=np.uint64, count=count)


class Server:
    """Continuous-batching exact-match server on one GPU (see module doc)."""

    SMALL_RESULT = 8192  # positions; larger results get a pinned block of their own

    def __init__(self, corpora: dict, budget_bytes: int = 40 << 30, streams: int = 4,
                 max_batch: int = 512, max_wait: float = 0.0005, first_cap: int = 256,
                 sigma_hints: dict | None = None, own_text_sigma: int = 0,
                 staging_bytes: int = 256 << 20, pinned_pool_bytes: int | None = None,
                 max_batch_scan_bytes: int = 16 << 30):
        import torch

        import paper_1012_2547_gb300 as smg
        self._torch = torch
        self._smg = smg
        self.corpora = dict(corpora)
        # Alphabet-size hints per corpus; a corpus without one gets the
        # effective alphabet size of its first MiB (hints.effective_sigma).
        from .hints import effective_sigma
        self.sigma_hints = dict(sigma_hints or {})
        for name, t in self.corpora.items():
            if name not in self.sigma_hints:
                self.sigma_hints[name] = effective_sigma(t[: 1 << 20].cpu().numpy())
        self.own_text_sigma = own_text_sigma
        self.first_cap = int(first_cap)
        self.policy = Policy(budget_bytes, max_batch, max_wait,
                             {k: v.numel() for k, v in self.corpora.items()},
                             max_batch_scan_bytes=max_batch_scan_bytes)
        self.streams = [torch.cuda.Stream() for _ in range(streams)]
        self.inflight: list[dict | None] = [None] * streams
        # Per-stream pinned staging for the copy-back of small results
        # (at most max_batch * SMALL_RESULT positions a batch), allocated up
        # front; large results use blocks of the pool.
        staging = max(staging_bytes // 8, max_batch * self.SMALL_RESULT)
        self._staging: list = [torch.empty(staging, dtype=torch.int64, pin_memory=True)
                               for _ in range(streams)]
        # Results in flight are bounded by the device budget (their device
        # buffers fit it), so the pinned pool gets the budget plus slack for
        # its size classes; a result that finds it full is copied to
        # ordinary host memory instead.
        self.pool = PinnedPool.shared(torch, budget_bytes + (8 << 30) if pinned_pool_bytes is None
                                      else pinned_pool_bytes)
        self.latencies: list[float] = []
        self.completed = 0
        self.retries = 0
        self.batches = 0
        self.host_s = collections.Counter()  # host seconds per scheduler phase
        self._ids = itertools.count()
        self._lock = threading.Lock()
        self._wake = threading.Event()
        self._stop = False
        self._error: BaseException | None = None
        self._thread = threading.Thread(target=self._run, name="smgpu-serve", daemon=True)
        self._thread.start()

    # ---------------------------------------------------------------- API

    def submit(self, pattern, corpus: str | None = None, text=None,
               t_arrival: float | None = None) -> cf.Future:
        p = bytes(pattern)
        if not p:
            raise ValueError("empty pattern")
        if (corpus is None) == (text is None):
            raise ValueError("give exactly one of corpus and text")
        if corpus is not None and corpus not in self.corpora:
            raise KeyError(corpus)
        t = None if text is None else np.ascontiguousarray(np.frombuffer(bytes(text), np.uint8)
                                                          if isinstance(text, (bytes, bytearray))
                                                          else text, dtype=np.uint8)
        n = len(t) if t is not None else self.corpora[corpus].numel()
        r = Request(next(self._ids), p, corpus, t, self._first_cap(n, len(p), corpus),
                    time.perf_counter() if t_arrival is None else t_arrival)
        with self._lock:
            self.policy.push(r)
        self._wake.set()
        return r.future

    def _first_cap(self, n: int, m: int, corpus: str | None) -> int:
        """Output capacity of a first attempt: for a corpus with an alphabet
        hint, twice the count expected on a uniform text, (n-m+1)/sigma^m,
        plus first_cap; else first_cap.  A larger true count costs a retry."""
        starts = max(n - m + 1, 1)
        sigma = self.sigma_hints.get(corpus, 0) if corpus is not None else self.own_text_sigma
        cap = self.first_cap
        if sigma >= 2 and m * np.log2(sigma) < 62:
            cap += int(2 * starts / float(sigma) ** m)
        return min(cap, starts)

    def close(self, timeout: float | None = None) -> None:
        self._stop = True
        self._wake.set()
        self._thread.join(timeout)
        if self._error is not None:
            raise self._error

    def stats(self) -> dict:
        lat = np.array(self.latencies) if self.latencies else np.zeros(1)
        return {"completed": self.completed, "batches": self.batches, "retries": self.retries,
                "pinned_pool_bytes": self.pool.allocated_bytes,
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "host_s": {k: round(v, 4) for k, v in self.host_s.items()}}

    # ---------------------------------------------------------------- loop

    def _run(self):
        torch = self._torch
        try:
            while True:
                progressed = self._retire()
                with self._lock:
                    busy = sum(x is not None for x in self.inflight)
                    slot = next((i for i, x in enumerate(self.inflight) if x is None), None)
                    batch, reserved, rejected = ([], 0, [])
                    if slot is not None and self.policy.ready(time.perf_counter(), busy):
                        batch, reserved, rejected = self.policy.take()
                    idle = not self.policy.pending and busy == 0
                for r in rejected:
                    r.future.set_exception(MemoryError("request larger than the device budget"))
                if batch:
                    self._launch(slot, batch, reserved)
                    progressed = True
                if self._stop and idle and not batch:
                    break
                if not progressed:
                    self._wake.wait(0.0002)
                    self._wake.clear()
        except BaseException as e:  # surface errors to close()
            self._error = e
            with self._lock:
                pending = list(self.policy.pending)
            for r in pending:
                if not r.future.done():
                    r.future.set_exception(e)
        finally:
            torch.cuda.synchronize()

    def _launch(self, slot: int, batch: list[Request], reserved: int) -> None:
        torch, smg = self._torch, self._smg
        s = self.streams[slot]
        dev = torch.device("cuda")
        t0 = time.perf_counter()
        with torch.cuda.stream(s):
            texts = []
            for r in batch:
                if r.text is not None:
                    texts.append(torch.from_numpy(r.text).to(dev, non_blocking=False))
                else:
                    texts.append(self.corpora[r.corpus])
            t1 = time.perf_counter()
            hint = self.sigma_hints.get(batch[0].corpus, self.own_text_sigma)
            plans = smg.prepare_many([r.pattern for r in batch], sigma_hint=hint)
            t2 = time.perf_counter()
            caps = np.array([r.cap for r in batch], dtype=np.int64)
            offs = np.concatenate([[0], np.cumsum(caps)])
            out = torch.empty(int(offs[-1]) or 1, dtype=torch.int64, device=dev)
            cnt = torch.empty(len(batch), dtype=torch.int64, device=dev)
            qarr = smg.query_array(
                np.array([t.data_ptr() for t in texts], dtype=np.uint64),
                np.array([t.numel() for t in texts], dtype=np.uint64), plans,
                np.uint64(out.data_ptr()) + 8 * offs[:-1].astype(np.uint64), caps.astype(np.uint64),
                np.uint64(cnt.data_ptr()) + 8 * np.arange(len(batch), dtype=np.uint64))
            need = max(smg.batch_workspace_size_array(qarr), 256)
            ws = torch.empty(need, dtype=torch.uint8, device=dev)
            smg.search_batch_async_array(qarr, ws.data_ptr(), need, stream=s)
            cnt_h = torch.empty(len(batch), dtype=torch.int64, pin_memory=True)
            cnt_h.copy_(cnt, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s)
        t3 = time.perf_counter()
        self.host_s["h2d_own_texts"] += t1 - t0
        self.host_s["prepare"] += t2 - t1
        self.host_s["launch"] += t3 - t2
        self.inflight[slot] = {"batch": batch, "event": ev, "cnt_h": cnt_h, "out_h": None,
                               "offs": offs, "keep": (texts, plans, out, cnt, ws), "reserved": reserved,
                               "phase": 0}
        self.batches += 1

    def _copy_back(self, i: int, rec: dict) -> None:
        """Counts are on the host: copy back exactly the valid positions of
        each complete request (not the whole capacity), then an event.
        Small results go through the stream's staging buffer, large ones
        into a pinned block of their own."""
        torch = self._torch
        counts = rec["cnt_h"].numpy()
        caps = np.array([r.cap for r in rec["batch"]], dtype=np.int64)
        take = np.where(counts <= caps, counts, 0)
        small = np.where(take < self.SMALL_RESULT, take, 0)
        dst_offs = np.concatenate([[0], np.cumsum(small)])
        out_h = self._staging[i]
        out = rec["keep"][2]
        blocks = {}
        s = self.streams[i]
        with torch.cuda.stream(s):
            for j in np.flatnonzero(take):
                a = int(rec["offs"][j])
                c = int(take[j])
                if c < self.SMALL_RESULT:
                    out_h[int(dst_offs[j]):int(dst_offs[j + 1])].copy_(out[a:a + c], non_blocking=True)
                else:
                    block, cls = self.pool.take(8 * c)
                    if block is None:  # pool full: an ordinary host array (a blocking copy)
                        blocks[j] = out[a:a + c].cpu().numpy().view(np.uint64)
                        continue
                    block[: 8 * c].view(torch.int64).copy_(out[a:a + c], non_blocking=True)
                    blocks[j] = (block, cls)
            ev = torch.cuda.Event()
            ev.record(s)
        rec.update(out_h=out_h, dst_offs=dst_offs, blocks=blocks, event=ev, phase=1)

    def _retire(self) -> bool:
        done_any = False
        for i, rec in enumerate(self.inflight):
            if rec is None or not rec["event"].query():
                continue
            done_any = True
            if rec["phase"] == 0:
                tc = time.perf_counter()
                self._copy_back(i, rec)
                self.host_s["copy_back"] += time.perf_counter() - tc
                continue
            now = time.perf_counter()
            counts = rec["cnt_h"].numpy()
            out_h = rec["out_h"].numpy()
            offs = rec["dst_offs"]
            requeue = []
            for j, r in enumerate(rec["batch"]):
                c = int(counts[j])
                if c > r.cap:
                    r.cap = c
                    r.attempts += 1
                    requeue.append(r)
                    continue
                if j in rec["blocks"]:
                    b = rec["blocks"][j]
                    pos = b if isinstance(b, np.ndarray) else self.pool.view(*b, c)  # no copy
                else:
                    # out of the stream's reusable staging buffer
                    pos = out_h[int(offs[j]):int(offs[j]) + c].astype(np.uint64)
                self.latencies.append(now - r.t_arrival)
                self.completed += 1
                r.future.set_result(pos)
            for p in rec["keep"][1]:
                p.free()
            with self._lock:
                self.policy.release(rec["reserved"])
                for r in reversed(requeue):
                    self.policy.push(r, front=True)
                self.retries += len(requeue)
                self.inflight[i] = None
            self.host_s["retire"] += time.perf_counter() - now
        return done_any
