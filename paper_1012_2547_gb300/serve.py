"""Serving loop: continuous batching of exact-match queries on one GPU.

Requests arrive at any time (``Server.submit``); each names a resident
corpus (a device text loaded once) or carries its own text.  A scheduler
thread repeatedly

  1. retires finished work: when a batch's counts are on the host, requests
     whose output was truncated go back to the front of the queue with
     their exact count as the new capacity, and the valid positions of the
     others are copied back; each request completes (its future gets its
     positions) as soon as its own copy is done, and the batch's memory
     returns to the budget when all of it is;
  2. admits pending requests while their device memory (own text, plan,
     output capacity, count) plus the batch workspace fits the budget,
     taking requests of one length class (floor(log2 m): the class of the
     oldest pending request) in arrival order, up to ``max_batch`` requests
     and an estimated GPU time of ``max_batch_seconds`` (scan bytes and
     output bytes over rates measured on the batches already run), which
     bounds how long the requests behind a batch wait; the bound grows with
     the backlog, so a long queue drains in large batches;
  3. launches the batch on a free stream with ``sm_search_batch_async``
     (one persistent launch per kernel family, in memory the server owns),
     followed by the copy of the counts and an event; small results come
     back through a per-stream pinned staging buffer, large ones straight
     into a pinned block of their own that the client receives without a
     copy (``PinnedPool``).

A first attempt's output capacity is sized from the count expected for the
pattern's bytes under the text's byte frequencies, so few requests need a
second attempt.  A request's own text is copied into pinned memory by the
caller's thread at submission, so the scheduler uploads it asynchronously.  Up to ``streams`` batches are in flight at once, so
requests that arrive while others run are admitted as slots and memory
free up and their work overlaps on the device.  Every request records
arrival and completion times (p50 / p99 latency, also per length class).
``Policy`` holds the host-side decisions (admission, length classes, batch
size) and needs no GPU.
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
    t_launch: float = 0.0  # host time its (last) batch was launched
    staged: tuple | None = None  # (pinned block, size class) holding its own text

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
                 scan_backlog: int = 512, max_batch_seconds: float = 1e9,
                 scan_rate: float = 3e12, copy_rate: float = 1.5e11):
        self.budget = int(budget_bytes)
        self.max_batch_out = int(max_batch_out_bytes)
        # Bounds of one batch's GPU time, so a request never waits behind
        # hundreds of long scans or copies: a hard bound on the text bytes it
        # scans, and a bound on its estimated time (scan_bytes / scan_rate +
        # output bytes / copy_rate, the rates measured on the batches that
        # ran: observe()).  Both grow by one step per `scan_backlog` pending
        # requests: a backlog is drained in large batches (throughput), a
        # short queue in small ones (latency).
        self.max_batch_scan = int(max_batch_scan_bytes)
        self.max_batch_seconds = float(max_batch_seconds)
        self.scan_rate = float(scan_rate)
        self.copy_rate = float(copy_rate)
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

    def cost(self, r: Request) -> float:
        """Estimated GPU seconds of a request: its scan and its copy-back."""
        return self.scan_bytes(r) / self.scan_rate + 8 * max(r.cap, 1) / self.copy_rate

    def observe(self, scan_bytes: int, scan_s: float, out_bytes: int, copy_s: float) -> None:
        """Measured timings of a finished batch update the rate estimates
        (exponential moving averages, each sample bounded to a factor of 4
        of the current estimate)."""
        if scan_s > 0 and scan_bytes > (64 << 20):
            r = min(max(scan_bytes / scan_s, self.scan_rate / 4), self.scan_rate * 4)
            self.scan_rate = 0.8 * self.scan_rate + 0.2 * r
        if copy_s > 0 and out_bytes > (8 << 20):
            r = min(max(out_bytes / copy_s, self.copy_rate / 4), self.copy_rate * 4)
            self.copy_rate = 0.8 * self.copy_rate + 0.2 * r

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
        secs = 0.0
        steps = 1 + len(self.pending) // self.scan_backlog
        scan_cap = self.max_batch_scan * steps
        time_cap = self.max_batch_seconds * steps
        while self.pending and len(batch) < self.max_batch:
            r = self.pending.popleft()
            need = self.need(r)
            fits_out = not batch or out_bytes + 8 * r.cap <= self.max_batch_out
            fits_scan = not batch or (scan + self.scan_bytes(r) <= scan_cap and secs + self.cost(r) <= time_cap)
            if length_class(r.m) == cls and self.used + reserved + need <= self.budget and fits_out and fits_scan:
                batch.append(r)
                reserved += need
                out_bytes += 8 * r.cap
                scan += self.scan_bytes(r)
                secs += self.cost(r)
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
                 max_batch_scan_bytes: int = 64 << 30, max_batch_seconds: float = 0.008,
                 cap_factor: float = 2.0):
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
        self.cap_factor = float(cap_factor)
        # Byte frequencies of each corpus (a histogram of its first 16 MiB,
        # on the device): a first attempt's capacity is sized from the count
        # expected for the pattern's own bytes.
        self.freqs = {}
        for name, t in self.corpora.items():
            h = torch.bincount(t[: 16 << 20].to(torch.int32), minlength=256).double()
            self.freqs[name] = (h / max(float(h.sum()), 1.0)).cpu().numpy()
        self.policy = Policy(budget_bytes, max_batch, max_wait,
                             {k: v.numel() for k, v in self.corpora.items()},
                             max_batch_scan_bytes=max_batch_scan_bytes,
                             max_batch_seconds=max_batch_seconds)
        self.lat_by_class = collections.defaultdict(list)
        self.streams = [torch.cuda.Stream() for _ in range(streams)]
        self._prep_stream = torch.cuda.Stream()
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
        self.queue_s: list[float] = []   # arrival -> launch of the batch that completed it
        self.host_max = collections.Counter()  # longest single scheduler phase, seconds
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
        r = Request(next(self._ids), p, corpus, t, self._first_cap(n, p, corpus, t),
                    time.perf_counter() if t_arrival is None else t_arrival)
        if t is not None and len(t):
            # The caller's thread copies its text into a pinned block, so the
            # scheduler uploads it asynchronously instead of copying from
            # pageable memory itself (which blocked it for up to ~10 ms).
            block, cls = self.pool.take(len(t))
            if block is not None:
                block[: len(t)].numpy()[:] = t
                r.staged = (block, cls)
        with self._lock:
            self.policy.push(r)
        self._wake.set()
        return r.future

    def _first_cap(self, n: int, p: bytes, corpus: str | None, text) -> int:
        """Output capacity of a first attempt: first_cap plus cap_factor
        times the count expected if the text's bytes were independent with
        its byte frequencies, (n-m+1) * prod_j f(p[j]) (the corpus's
        histogram, or that of the first 64 KiB of an own text).  A larger true
        count costs a retry."""
        m = len(p)
        starts = max(n - m + 1, 1)
        if corpus is not None:
            f = self.freqs[corpus]
        else:
            sample = text[: 1 << 16]
            f = np.bincount(sample, minlength=256) / max(len(sample), 1)
        pr = float(np.prod(f[np.frombuffer(p, np.uint8)]))
        return int(min(self.first_cap + np.ceil(self.cap_factor * starts * pr), starts))

    def close(self, timeout: float | None = None) -> None:
        self._stop = True
        self._wake.set()
        self._thread.join(timeout)
        if self._error is not None:
            raise self._error

    def stats(self) -> dict:
        lat = np.array(self.latencies) if self.latencies else np.zeros(1)
        by_class = {}
        for c, v in sorted(self.lat_by_class.items()):
            a = np.array(v)
            by_class[f"m{1 << c}-{(2 << c) - 1}"] = {"n": len(v), "p50_ms": round(float(np.percentile(a, 50)) * 1e3, 3),
                                                  "p99_ms": round(float(np.percentile(a, 99)) * 1e3, 3)}
        qs = np.array(self.queue_s) if self.queue_s else np.zeros(1)
        return {"completed": self.completed, "batches": self.batches, "retries": self.retries,
                "pinned_pool_bytes": self.pool.allocated_bytes,
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "queue_p50_ms": round(float(np.percentile(qs, 50)) * 1e3, 3),
                "queue_p99_ms": round(float(np.percentile(qs, 99)) * 1e3, 3),
                "host_max_ms": {k: round(v * 1e3, 3) for k, v in self.host_max.items()},
                "by_length_class": by_class,
                "rates": {"scan_GBs": round(self.policy.scan_rate / 1e9, 1),
                          "copy_GBs": round(self.policy.copy_rate / 1e9, 1)},
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
                    if r.staged is not None:
                        self.pool._give(*r.staged)
                        r.staged = None
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
            ev0 = torch.cuda.Event(enable_timing=True)
            ev0.record(s)
            texts = []
            for r in batch:
                if r.staged is not None:
                    texts.append(r.staged[0][: len(r.text)].to(dev, non_blocking=True))
                elif r.text is not None:
                    texts.append(torch.from_numpy(r.text).to(dev, non_blocking=False))
                else:
                    texts.append(self.corpora[r.corpus])
            t1 = time.perf_counter()
            hint = self.sigma_hints.get(batch[0].corpus, self.own_text_sigma)
            # Plans upload on a stream of their own: the prepare call waits for
            # its stream, which must not hold this batch's text uploads.
            plans = smg.prepare_array([r.pattern for r in batch], sigma_hint=hint, stream=self._prep_stream)
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
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(s)
        t3 = time.perf_counter()
        for r in batch:
            r.t_launch = t0
        for k, v in (("h2d_own_texts", t1 - t0), ("prepare", t2 - t1), ("launch", t3 - t2)):
            self.host_s[k] += v
            self.host_max[k] = max(self.host_max[k], v)
        self.inflight[slot] = {"batch": batch, "event": ev, "ev0": ev0, "cnt_h": cnt_h, "offs": offs,
                               "keep": (texts, plans, out, cnt, ws), "reserved": reserved, "phase": 0,
                               "scan": sum(self.policy.scan_bytes(r) for r in batch)}
        self.batches += 1

    def _complete(self, r: Request, pos, now: float) -> None:
        if r.staged is not None:  # its upload finished before its search ran
            self.pool._give(*r.staged)
            r.staged = None
        lat = now - r.t_arrival
        self.latencies.append(lat)
        self.queue_s.append(r.t_launch - r.t_arrival)
        self.lat_by_class[length_class(r.m)].append(lat)
        self.completed += 1
        r.future.set_result(pos)

    def _copy_back(self, i: int, rec: dict) -> None:
        """Counts are on the host.  Requests whose output was truncated go
        back to the front of the queue at once, with their exact count as
        the capacity.  For the others exactly the valid positions are copied
        back (not the whole capacity): the small results first, through the
        stream's staging buffer, then one event; then each large result into
        a pinned block of its own, each followed by its own event, so every
        request completes as soon as its own positions are on the host."""
        torch = self._torch
        counts = rec["cnt_h"].numpy()
        batch = rec["batch"]
        caps = np.array([r.cap for r in batch], dtype=np.int64)
        requeue = [j for j in range(len(batch)) if counts[j] > caps[j]]
        for j in requeue:
            batch[j].cap = int(counts[j])
            batch[j].attempts += 1
        if requeue:
            with self._lock:
                for j in reversed(requeue):
                    self.policy.push(batch[j], front=True)
                self.retries += len(requeue)
            self._wake.set()
        take = np.where(counts <= caps, counts, 0)
        small = np.where(take < self.SMALL_RESULT, take, 0)
        dst_offs = np.concatenate([[0], np.cumsum(small)])
        out_h = self._staging[i]
        out = rec["keep"][2]
        large = []
        s = self.streams[i]
        with torch.cuda.stream(s):
            ev_c = torch.cuda.Event(enable_timing=True)
            ev_c.record(s)
            for j in np.flatnonzero(small):
                a = int(rec["offs"][j])
                out_h[int(dst_offs[j]):int(dst_offs[j + 1])].copy_(out[a:a + int(small[j])], non_blocking=True)
            ev_small = torch.cuda.Event()
            ev_small.record(s)
            for j in np.flatnonzero(take >= self.SMALL_RESULT):
                a = int(rec["offs"][j])
                c = int(take[j])
                block, cls = self.pool.take(8 * c)
                if block is None:  # pool full: an ordinary host array (a blocking copy)
                    large.append([j, out[a:a + c].cpu().numpy().view(np.uint64), None])
                    continue
                block[: 8 * c].view(torch.int64).copy_(out[a:a + c], non_blocking=True)
                e = torch.cuda.Event()
                e.record(s)
                large.append([j, (block, cls), e])
            ev_end = torch.cuda.Event(enable_timing=True)
            ev_end.record(s)
        todo = [j for j in range(len(batch)) if j not in set(requeue)]
        rec.update(out_h=out_h, dst_offs=dst_offs, small=small, ev_small=ev_small, large=large,
                   ev_c=ev_c, event=ev_end, phase=1, todo=set(todo), small_done=False,
                   out_bytes=int(8 * take.sum()))

    def _retire(self) -> bool:
        done_any = False
        for i, rec in enumerate(self.inflight):
            if rec is None:
                continue
            if rec["phase"] == 0:
                if not rec["event"].query():
                    continue
                done_any = True
                tc = time.perf_counter()
                self._copy_back(i, rec)
                dt = time.perf_counter() - tc
                self.host_s["copy_back"] += dt
                self.host_max["copy_back"] = max(self.host_max["copy_back"], dt)
                continue
            now = time.perf_counter()
            t_r = now
            batch = rec["batch"]
            counts = rec["cnt_h"].numpy()
            if not rec["small_done"] and rec["ev_small"].query():
                out_h = rec["out_h"].numpy()
                offs = rec["dst_offs"]
                for j in np.flatnonzero(rec["small"]):
                    self._complete(batch[j], out_h[int(offs[j]):int(offs[j + 1])].astype(np.uint64), now)
                    rec["todo"].discard(int(j))
                for j in list(rec["todo"]):  # empty results
                    if counts[j] == 0:
                        self._complete(batch[j], np.zeros(0, dtype=np.uint64), now)
                        rec["todo"].discard(j)
                rec["small_done"] = True
                done_any = True
            for item in rec["large"]:
                j, b, e = item
                if j in rec["todo"] and (e is None or e.query()):
                    pos = b if isinstance(b, np.ndarray) else self.pool.view(*b, int(counts[j]))  # no copy
                    self._complete(batch[j], pos, now)
                    rec["todo"].discard(j)
                    done_any = True
            if rec["todo"] or not rec["event"].query():
                self.host_s["retire"] += time.perf_counter() - t_r
                continue
            # Whole batch done: measured scan and copy times update the
            # policy's rate estimates; plans and memory are released.
            scan_s = rec["ev0"].elapsed_time(rec["ev_c"]) / 1e3
            copy_s = rec["ev_c"].elapsed_time(rec["event"]) / 1e3
            rec["keep"][1].free()
            with self._lock:
                self.policy.observe(rec["scan"], scan_s, rec["out_bytes"], copy_s)
                self.policy.release(rec["reserved"])
                self.inflight[i] = None
            done_any = True
            self.host_s["retire"] += time.perf_counter() - t_r
        return done_any
