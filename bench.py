#!/usr/bin/env python
"""Benchmark of the GB300 exact string matching library.

Default workload (the paper-shaped sweep): ten 4 MiB synthetic texts shaped
like the paper's text buffers (Section 2), m in {2, 4, ..., 1024}, 100
substring patterns per (text, m): 10,000 searches = 41.9 GB scanned per
step.  A step runs every search once, as one persistent, graph-captured
launch per kernel family (sm_batch_launch), with plans and texts resident in
HBM.  L2 is flushed (a 256 MiB write) before every timed step, outside the
timed events.

Prints ONE JSON line (rank 0):
  metric/value      scanned text GB/s (sum of n over all searches / step time)
  roofline          dominant kernel family: algorithmic bytes (n per search +
                    8 bytes per reported position) / its mean launch time,
                    against the measured HBM copy bandwidth
  e2e               the same metric through the C ABI from pinned host
                    buffers: texts H2D, sm_prepare_many, sm_search_batch,
                    positions D2H, all inside the timed region
  cpu_baseline      the CPU oracle (naive definition) on a bounded sample
  clocks            nvidia-smi samples taken during the timed region

--impl reference times the CPU oracle (the reference arm of this tier) on a
bounded sample of the same workload.  --workload bandwidth runs the 8 GiB
single-pattern scans (Section 2's bandwidth-style run at GB300 scale);
--workload single the 1 MiB single search.

Multi-GPU (--gpus N under torchrun): every rank runs the full per-GPU
workload on its own GPU (independent replicas, weak scaling); the step time
is the max over ranks.
"""
from __future__ import annotations

import argparse
import functools
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

FALLBACK_HBM_GBS = 6800.0
SM_MAX_MHZ = 2070.0
METRIC = "scanned text GB/s (% of HBM peak) per sigma,m; served queries/s + p50/p99 latency"
L2_FLUSH_BYTES = 256 << 20


# ---------------------------------------------------------------- helpers

def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value: float, world: int, device=None) -> float:
    """Max of a float over all ranks (identity for world == 1)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# CUDA sources the bit-parallel kernels (the dominant family) are built from.
SHIFTAND_SOURCES = ("sm_common.cuh", "sm_internal.h", "sm_shiftor.cu")


def _code_only(src: str) -> str:
    """C++/CUDA source without comments and whitespace (string literals are
    kept as they are), so that editing a comment leaves the hash alone."""
    import re
    tok = re.compile(r'"(?:\\.|[^"\\])*"|//[^\n]*|/\*.*?\*/|\s+', re.S)
    return tok.sub(lambda m: m.group(0) if m.group(0).startswith('"') else "", src)


def source_hash(files=SHIFTAND_SOURCES) -> str:
    """Hash of the code (comments and whitespace left out) of the CUDA
    sources a kernel is compiled from: ties committed ncu traffic to the
    build of that kernel."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1012_2547_gb300", "csrc")
    for f in sorted(files):
        h.update(f.encode())
        with open(os.path.join(csrc, f), encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def committed_profile(kernel: str, path: str | None = None) -> dict:
    """Per-launch ncu figures of `kernel` (dram bytes, thread instructions)
    from profiles/traffic.txt (or `path`), when they were taken on the
    current sources; else {}."""
    path = path or os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return {}
    cur = source_hash()
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        kv = dict(x.split("=", 1) for x in line.split() if "=" in x)
        if kv.get("kernel") == kernel and kv.get("source") == cur:
            out = {}
            for k in ("bytes_per_launch", "inst_per_launch"):
                if k in kv:
                    out[k] = float(kv[k])
            return out
    return {}


# ---------------------------------------------------------------- CPU oracle timing

def cpu_sample_time(texts, queries, budget_s: float, threads: int):
    """Time the oracle (threaded naive) on a deterministic sample of the
    queries, stopping after ~budget_s seconds.  Returns (bytes, seconds,
    searches)."""
    import oracle
    lib = oracle.load()
    done_b, done_n = 0, 0
    t0 = time.perf_counter()
    order = list(range(len(queries)))
    # spread the sample over texts and lengths
    step = max(1, len(order) // 997)
    sample = order[::step] + [i for i in order if i % step]
    for qi in sample:
        q = queries[qi]
        t = texts[q.text_id]
        n = len(t) if q.n is None else q.n
        oracle.count_mt(t[:n], q.pattern, threads=threads, lib=lib)
        done_b += n
        done_n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    return done_b, time.perf_counter() - t0, done_n


# ---------------------------------------------------------------- our arm

def load_tuning(args, sigmas=None):
    """Apply the committed GB300 tuning table (or, with --tune, re-measure
    it on this device); None with --no-tune."""
    if args.no_tune:
        return None
    from paper_1012_2547_gb300 import tuner
    if args.tune or not os.path.exists(tuner.GB300_TABLE):
        kw = {"sigmas": sigmas} if sigmas else {}
        return {"seconds": tuner.tune(**kw)["seconds"], "source": "measured now"}
    tr = tuner.load(tuner.GB300_TABLE)
    return {"seconds": tr["seconds"],
            "source": "paper_1012_2547_gb300/tuning_gb300.json (measured on GB300 by tuner.tune)"}


def workload_config(w, world: int) -> dict:
    """The `config` object of both arms' JSON lines."""
    return {"workload": w.name, "searches": len(w.queries), "scanned_bytes_per_step": w.scanned_bytes,
            "parallelism": f"replicas{world}",
            "l2": "GPU arm: L2 flushed by a 256 MiB write before each timed step"}


def sweep_kwargs(args) -> dict:
    """Subset of the sweep for profiling small cases (--ms, --per-m)."""
    kw = {}
    if args.ms:
        kw["ms"] = tuple(int(x) for x in args.ms.split(","))
    if args.per_m:
        kw["per_m"] = args.per_m
    return kw


def roofline_record(alg_bytes: float, scanned: float, t: float, prof: dict, hbm: float, peak_kind: str,
                    sms: int, mhz: float) -> dict:
    """Roofline of the dominant family from its algorithmic bytes per launch,
    its live launch time `t` (s) and its committed ncu figures `prof`
    (bytes_per_launch = DRAM traffic, inst_per_launch = thread instructions;
    either may be absent).  The family is L2-fed, and so bound by instruction
    issue, when its DRAM traffic is under half its algorithmic bytes; then
    `achieved` is thread instructions per second against the issue ceiling
    (SMs x 4 schedulers x 32 lanes x the SM clock).  Otherwise it is HBM
    bound: algorithmic bytes per second against the measured copy peak."""
    traffic = prof.get("bytes_per_launch")
    achieved = alg_bytes / t / 1e9
    hbm_view = {"achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(achieved / hbm, 4), "peak_kind": peak_kind}
    issue_peak = sms * 128 * mhz * 1e6 / 1e9  # G thread instructions / s
    issue = {"peak": round(issue_peak, 1), "unit": "Ginst/s",
             "peak_basis": f"{sms} SMs x 128 lanes x {mhz:.0f} MHz"}
    if "inst_per_launch" in prof:
        ach_i = prof["inst_per_launch"] / t / 1e9
        issue.update({"achieved": round(ach_i, 1), "frac": round(ach_i / issue_peak, 4),
                      "inst_per_scanned_byte": round(prof["inst_per_launch"] / scanned, 3),
                      "inst_basis": "smsp__thread_inst_executed.sum per launch, committed ncu capture"})
    l2_fed = traffic is not None and traffic < 0.5 * alg_bytes
    if l2_fed and "achieved" in issue:
        return {"bound": "alu", "achieved": issue["achieved"], "peak": issue["peak"], "unit": "Ginst/s",
                "frac": issue["frac"], "traffic": traffic, "hbm_view": hbm_view}
    return {"bound": "hbm", "achieved": hbm_view["achieved"], "peak": hbm, "unit": "GB/s",
            "frac": hbm_view["frac"], "traffic": traffic, "issue": issue}


KERNEL_NAMES = ["so_kernel<u32,u8,H>", "so_kernel<u32,u16,H>", "so_kernel<u32,u32,H>",
                "so_kernel<u32,u32,A>", "so_kernel<u64,u64,H>", "so_kernel<u64,u64,A>",
                "qg_kernel<qgram>", "qg_kernel<linear>", "mp_kernel", "qg_kernel<dfa>",
                "so_kernel<u32,u8,H,pair>", "so_kernel<u32,u8,H,quad>"]


def family_key(plan) -> int:
    """The library runs one persistent launch per kernel id."""
    return plan.info().kernel


def family_name(key) -> str:
    return KERNEL_NAMES[key] if 0 <= key < len(KERNEL_NAMES) else str(key)


def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    import __graft_entry__
    if rank == 0 or world > 1:
        __graft_entry__.build()
    import paper_1012_2547_gb300 as smg
    from paper_1012_2547_gb300 import workloads

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    tuning = None
    if not args.no_tune:
        # The kernel per (m bucket, sigma bucket) comes from the autotuner's
        # table measured on GB300 (committed JSON), or, with --tune, from a
        # fresh measurement on this device before anything is timed.
        from paper_1012_2547_gb300 import tuner
        if args.tune or not os.path.exists(tuner.GB300_TABLE):
            tr = tuner.tune(ms=tuple(int(x) for x in args.ms.split(",")) if args.ms else
                            tuple(__import__("paper_1012_2547_gb300").gen.SWEEP_M),
                            per=args.per_m or workloads.SWEEP_PER_M)
            source = "measured now"
        else:
            tr = tuner.load(tuner.GB300_TABLE)
            source = "paper_1012_2547_gb300/tuning_gb300.json (measured on GB300 by tuner.tune)"
        tuning = {"source": source, "seconds": tr["seconds"],
                  "choices": {f"s{r['sigma']}m{r['m']}": r["best"] for r in tr["report"]}}

    if args.workload == "sweep":
        w = workloads.sweep(**sweep_kwargs(args))
    elif args.workload == "single":
        w = workloads.single()
    else:
        raise SystemExit("--workload bandwidth is driven by bench_bandwidth() below")
    texts_h = w.texts
    texts_d = [torch.from_numpy(t).to(dev) for t in texts_h]
    queries = w.queries
    nq = len(queries)

    # plans, grouped by sigma hint to keep the tuning buckets right
    plans = [None] * nq
    by_sigma = {}
    for i, q in enumerate(queries):
        by_sigma.setdefault(q.sigma_hint, []).append(i)
    for sg, idx in by_sigma.items():
        ps = smg.prepare_many([queries[i].pattern for i in idx], sigma_hint=sg)
        for i, p in zip(idx, ps):
            plans[i] = p

    # count pass (sizes the outputs), then exact output buffers
    counts = torch.zeros(nq, dtype=torch.int64, device=dev)
    items = [(texts_d[q.text_id], plans[i], None, counts[i:i + 1]) for i, q in enumerate(queries)]
    smg.search_batch(items)
    smg.sync()
    cnt_h = counts.cpu().numpy()
    total_hits = int(cnt_h.sum())
    outbuf = torch.empty(max(total_hits, 1), dtype=torch.int64, device=dev)
    offs = np.concatenate([[0], np.cumsum(cnt_h)])

    fam = {}
    for i in range(nq):
        fam.setdefault(family_key(plans[i]), []).append(i)
    batches = []
    for key, idx in sorted(fam.items()):
        its = [(texts_d[queries[i].text_id], plans[i],
                outbuf[int(offs[i]):int(offs[i + 1])], counts[i:i + 1]) for i in idx]
        alg = sum(len(texts_h[queries[i].text_id]) for i in idx) + 8 * int(cnt_h[idx].sum())
        batches.append({"key": key, "batch": smg.Batch(its, graph=True), "alg_bytes": alg,
                        "scanned": sum(len(texts_h[queries[i].text_id]) for i in idx),
                        "n": len(idx), "times": []})

    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in batches]
    ev_step = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))

    def step(record: bool):
        # One event pair around the whole step (gaps between the families'
        # graph launches included); one pair per family inside it gives the
        # families' shares.
        ev_step[0].record(stream)
        for b, (e0, e1) in zip(batches, ev):
            e0.record(stream)
            b["batch"].launch(stream)
            e1.record(stream)
        ev_step[1].record(stream)
        if record:
            torch.cuda.synchronize()
            for b, (e0, e1) in zip(batches, ev):
                b["times"].append(e0.elapsed_time(e1) / 1e3)
            return ev_step[0].elapsed_time(ev_step[1]) / 1e3
        return None

    # The steps run inside an NVTX range, so a profiler can be limited to
    # them (ncu --nvtx --nvtx-include bench_steps/) and skip the tuner's
    # and the count pass's launches.
    nvtx = getattr(torch.cuda, "nvtx", None)
    if nvtx is not None:
        nvtx.range_push("bench_steps")
    for _ in range(args.warmup):
        flush.zero_()
        step(False)
    torch.cuda.synchronize()
    smg.sync()
    for b in batches:
        b["times"].clear()

    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    launches0 = smg.kernel_launches()
    step_times = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        step_times.append(step(True))
    torch.cuda.synchronize()
    launches = smg.kernel_launches() - launches0
    if nvtx is not None:
        nvtx.range_pop()
    barrier(world)
    clk = clocks.stop()
    smg.sync()

    per_step = sum(step_times) / len(step_times)
    per_step_max = max_over_ranks(per_step, world, dev)
    scanned = w.scanned_bytes
    value = world * scanned / per_step_max / 1e9

    # GB/s per (text, m) cell: each cell's searches as one graph-captured
    # batch, timed alone (L2 flushed before each), outside the step timing.
    per_cell = {}
    if w.name.startswith("sweep") and not args.no_cells:
        cells = {}
        for i, q in enumerate(queries):
            cells.setdefault((q.text_id, len(q.pattern)), []).append(i)
        for (ti, m), idx in sorted(cells.items()):
            b = smg.Batch([(texts_d[ti], plans[i], outbuf[int(offs[i]):int(offs[i + 1])], counts[i:i + 1])
                           for i in idx], graph=True)
            ts = []
            for r in range(3):
                flush.zero_()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                b.launch(stream)
                e1.record(stream)
                torch.cuda.synchronize()
                if r:
                    ts.append(e0.elapsed_time(e1) / 1e3)
            b.free()
            t = min(ts)
            name = w.specs[ti].name or f"text{ti}"
            per_cell.setdefault(name, {})[str(m)] = round(len(idx) * len(texts_h[ti]) / t / 1e9, 1)

    # parity sample (outside the timed region)
    import oracle
    rng = np.random.default_rng(0)
    sample = sorted(set(rng.integers(0, nq, 12).tolist()) | {0, nq - 1})
    parity_ok = True
    for i in sample:
        q = queries[i]
        got = outbuf[int(offs[i]):int(offs[i + 1])].cpu().numpy().astype(np.uint64)
        exp = oracle.kmp(texts_h[q.text_id], q.pattern) if len(q.pattern) > 64 else \
            oracle.naive_mt(texts_h[q.text_id], q.pattern)
        parity_ok &= bool(np.array_equal(got, exp))

    # roofline: dominant family
    hbm, peak_kind = peaks()
    dom = max(batches, key=lambda b: statistics.mean(b["times"]))
    dom_t = statistics.mean(dom["times"])
    kname = family_name(dom["key"])
    prof = committed_profile(kname + ":" + w.name)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = (clk or {}).get("sm_mhz") or SM_MAX_MHZ
    roofline = roofline_record(dom["alg_bytes"], dom["scanned"], dom_t, prof, hbm, peak_kind, sms, mhz)
    roofline.update({
        "kernel": kname, "peak_kind": peak_kind, "alg_bytes_per_launch": dom["alg_bytes"],
        "kernel_ms": round(dom_t * 1e3, 4), "kernel_share": round(dom_t / per_step, 4),
        "families": {family_name(b["key"]): {"searches": b["n"],
                                             "ms": round(statistics.mean(b["times"]) * 1e3, 4)}
                     for b in batches}})

    # e2e through the C ABI from pinned host buffers, pipelined per text:
    # the texts go H2D on a copy stream; for each text, its patterns' plans
    # are built and uploaded (sm_prepare_many, on a third stream), its
    # searches are enqueued as one asynchronous batch (sm_search_batch_async
    # in a workspace allocated once, outside the timed region) on the
    # compute stream, and its positions and counts go D2H on the copy
    # stream as soon as that batch is done.  So the host builds text g+1's
    # plans while the GPU searches text g and copies text g-1's results.
    e2e = None
    if not args.no_e2e:
        pinned = [torch.from_numpy(t).pin_memory() for t in texts_h]
        outs_h = torch.empty(max(total_hits, 1), dtype=torch.int64).pin_memory()
        cnts_h = torch.empty(nq, dtype=torch.int64).pin_memory()
        h2d = sum(len(t) for t in texts_h)
        by_text = {}
        for i, q in enumerate(queries):
            by_text.setdefault(q.text_id, []).append(i)
        groups = []
        for ti, idx in sorted(by_text.items()):
            idx = np.asarray(idx)
            assert np.all(np.diff(idx) == 1)  # a text's searches are contiguous
            groups.append((ti, idx, queries[idx[0]].sigma_hint))
        s_in, s_run, s_prep = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        out_ptr0 = np.uint64(outbuf.data_ptr())
        cnt_ptr0 = np.uint64(counts.data_ptr())

        # The inputs a caller holds before the timed region: each text's
        # patterns (a list of bytes) and the pointer columns of its query
        # descriptors (text, output and count pointers, capacities); the
        # plans come from the prepare call inside it.
        group_pats = [[queries[i].pattern for i in idx] for _, idx, _ in groups]
        group_cols = [(np.full(len(idx), texts_d[ti].data_ptr(), dtype=np.uint64),
                       np.full(len(idx), texts_d[ti].numel(), dtype=np.uint64),
                       out_ptr0 + 8 * offs[idx].astype(np.uint64), cnt_h[idx].astype(np.uint64),
                       cnt_ptr0 + 8 * idx.astype(np.uint64)) for ti, idx, _ in groups]

        def group_array(g, pl):
            t_i, n_i, o_i, c_i, k_i = group_cols[g]
            return smg.query_array(t_i, n_i, pl, o_i, c_i, k_i)

        # Workspace for the largest group (one compute stream runs the
        # groups in order, so they can share it).
        ws_bytes = 0
        for g, (ti, idx, sg) in enumerate(groups):
            pl = smg.prepare_array(group_pats[g], sigma_hint=sg)
            ws_bytes = max(ws_bytes, smg.batch_workspace_size_array(group_array(g, pl)))
            pl.free()
        ws = torch.empty(ws_bytes + 256, dtype=torch.uint8, device=dev)
        ws_ptr = (ws.data_ptr() + 255) & ~255
        e2e_times = []
        plan_bytes = 0
        for r in range(max(1, args.e2e_steps) + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ev_in = []
            with torch.cuda.stream(s_in):
                for td, th in zip(texts_d, pinned):
                    td.copy_(th, non_blocking=True)
                    ev_in.append(torch.cuda.Event())
                    ev_in[-1].record(s_in)
            keep = []
            for g, (ti, idx, sg) in enumerate(groups):
                pl = smg.prepare_array(group_pats[g], sigma_hint=sg, stream=s_prep)
                keep.append(pl)
                s_run.wait_event(ev_in[ti])
                smg.search_batch_async_array(group_array(g, pl), ws_ptr, ws_bytes, stream=s_run)
                done = torch.cuda.Event()
                done.record(s_run)
                s_in.wait_event(done)
                lo, hi = int(offs[idx[0]]), int(offs[idx[-1] + 1])
                with torch.cuda.stream(s_in):
                    outs_h[lo:hi].copy_(outbuf[lo:hi], non_blocking=True)
                    cnts_h[idx[0]:idx[-1] + 1].copy_(counts[idx[0]:idx[-1] + 1], non_blocking=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            if r > 0:
                e2e_times.append(dt)
            plan_bytes = sum(pl.info(i).device_bytes for pl in keep for i in range(len(pl)))
            for pl in keep:
                pl.free()
        smg.sync(s_run)
        ok = bool(np.array_equal(cnts_h.numpy(), cnt_h)) and bool(torch.equal(outs_h, outbuf.cpu()))
        e2e_t = max_over_ranks(statistics.mean(e2e_times), world, dev)
        e2e = {"value": round(world * scanned / e2e_t / 1e9, 2), "unit": "GB/s",
               "h2d_bytes_per_step": int(h2d + plan_bytes),
               "d2h_bytes_per_step": int(8 * total_hits + 8 * nq),
               "ms_per_step": round(e2e_t * 1e3, 3), "counts_match": ok,
               "path": "per text: sm_prepare_many (prepare_array) -> sm_search_batch_async -> D2H, "
                       "pipelined over 3 streams"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        b, s, k = cpu_sample_time(texts_h, queries, args.cpu_seconds, threads)
        cpu = {"value": round(b / s / 1e9, 4), "unit": "GB/s", "cores": threads, "kind": "oracle",
               "sample": f"{k} of {nq} sweep searches ({b / 1e9:.2f} GB), threaded naive"}

    return {
        "metric": METRIC,
        "value": round(value, 2),
        "unit": "GB/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(per_step_max * 1e3, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u8",
        "data": "synthetic",
        "config": workload_config(w, world),
        "positions_per_step": total_hits,
        "scanned_over_copy_peak_pct": round(100 * value / world / hbm, 2),
        "roofline": roofline,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "clocks": clk,
        "gpu_launches": int(launches),
        "parity_sample": {"searches": len(sample), "ok": parity_ok},
        "per_sigma_m_GBs": per_cell or None,
        "tuning": tuning,
    }


# ---------------------------------------------------------------- bandwidth workload

def _kernel_of(plan) -> str:
    return family_name(plan.info().kernel)


def bandwidth_record(args, local, compact: bool = False) -> dict:
    """Single-pattern scans of the 8 GiB sigma = 4 text (m in {4, 32, 256,
    1024}: 20 substring and 20 random patterns each, one search at a time,
    median of the timed repetitions), the a^m dense stress on its 64 MiB
    a^n-dominated prefix, and m = 8 scans of the text's last GiB and of the
    whole text.  The text
    is larger than L2, so no flush is needed between repetitions.  Full mode
    adds the automaton family beside the automatic choice and sampled oracle
    parity; compact mode (the default bench line) keeps the per-m medians."""
    import numpy as np
    import torch

    import paper_1012_2547_gb300 as smg
    from paper_1012_2547_gb300 import gen, workloads

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    n = args.bw_bytes
    ms = tuple(int(x) for x in args.ms.split(",")) if args.ms and not compact else workloads.BANDWIDTH_M
    per_m = args.per_m if args.per_m and not compact else 20
    warmup, reps = (2, 5) if compact else (args.warmup, args.steps)
    w = workloads.bandwidth(n=n, per_m=per_m, ms=ms)
    spec = w.specs[0]
    text = torch.empty(n, dtype=torch.uint8, device=dev)
    smg.gen_text(text, 0, spec.key, 4)
    # dense stress region: a^n-dominated first 64 MiB
    dense = workloads.bandwidth_dense(ms=ms)
    pre = min(workloads.DENSE_PREFIX, n)
    host_pre = spec.window(0, pre).copy()
    gen.plant_prefix(host_pre, pre, 4096, seed=77)
    text[:pre].copy_(torch.from_numpy(host_pre))
    smg.sync()
    queries = w.queries + dense
    plans = smg.prepare_many([q.pattern for q in queries], sigma_hint=4)
    cnt = torch.zeros(len(queries), dtype=torch.int64, device=dev)
    for i, q in enumerate(queries):
        smg.search_into(text, plans[i], None, cnt[i:i + 1], n=q.n or n, cap=0)
    smg.sync()
    caps = cnt.cpu().numpy()
    outs = [torch.empty(max(int(c), 1), dtype=torch.int64, device=dev) for c in caps]

    def time_search(t_text, plan, out, cnt1, nn, cap):
        # `reps` searches back to back between two events (the host enqueues
        # ahead, so no search waits for the host), three times: the median
        # of the per-search means.
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(warmup):
            smg.search_into(t_text, plan, out, cnt1, n=nn, cap=cap)
        ts = []
        for _ in range(3):
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(reps):
                smg.search_into(t_text, plan, out, cnt1, n=nn, cap=cap)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3 / reps)
        return statistics.median(ts)

    res = []
    for i, q in enumerate(queries):
        nn = q.n or n
        t = time_search(text, plans[i], outs[i], cnt[i:i + 1], nn, int(caps[i]))
        res.append({"m": len(q.pattern), "n": nn, "hits": int(caps[i]), "ms": round(t * 1e3, 4),
                    "GBs": round(nn / t / 1e9, 1), "variant": plans[i].info().variant,
                    "kernel": _kernel_of(plans[i]),
                    "kind": "dense" if q.n else ("substring" if i % (2 * per_m) < per_m else "random")})
    hbm, kind = peaks()
    for r in res:
        r["frac"] = round(r["GBs"] / hbm, 4)
    summary = {}
    for m in ms:
        for k in ("substring", "random"):
            rs = [r for r in res if r["m"] == m and r["kind"] == k]
            if rs:
                g = statistics.median(r["GBs"] for r in rs)
                summary.setdefault(str(m), {})[k] = {"GBs": round(g, 1), "frac": round(g / hbm, 4),
                                                     "kernel": rs[0]["kernel"]}
        d = [r for r in res if r["m"] == m and r["kind"] == "dense"]
        if d:
            summary[str(m)]["dense_64MiB"] = {"ms": d[0]["ms"], "hits": d[0]["hits"], "kernel": d[0]["kernel"]}
    out = {"text": f"{n} bytes uniform sigma=4 (device-built), L2 not flushed (text > L2)",
           "peak_gbs": hbm, "peak_kind": kind, "searches_per_m": f"{per_m} substring + {per_m} random",
           "timing": f"per search: {reps} back-to-back searches between CUDA events, median of 3, "
                     f"after {warmup} warm-up", "per_m": summary}
    del outs
    # m = 8 single scans (10 substring patterns): of the text's last GiB, and
    # of the whole text.
    pats = gen.substring_patterns_spec(spec, 8, 10, seed=23)
    pl8 = smg.prepare_many(pats, sigma_hint=4)
    c1 = torch.zeros(1, dtype=torch.int64, device=dev)
    for key, n1 in (("scan1GiB_m8", min(1 << 30, n)), ("scan_m8", n)):
        sub = text[n - n1:]
        g8 = []
        for p in pl8:
            smg.search_into(sub, p, None, c1, cap=0)
            smg.sync()
            o1 = torch.empty(max(int(c1.item()), 1), dtype=torch.int64, device=dev)
            t = time_search(sub, p, o1, c1, n1, o1.numel())
            g8.append(n1 / t / 1e9)
            del o1
        g = statistics.median(g8)
        out[key] = {"n": n1, "GBs": round(g, 1), "frac": round(g / hbm, 4), "patterns": len(pl8),
                    "kernel": _kernel_of(pl8[0])}
    if compact:
        del text
        torch.cuda.empty_cache()
        return out
    # The automaton family (explicit DFA plans) beside the automatic choice:
    # the dense stress and one substring pattern per m, where the table fits.
    outs = [torch.empty(max(int(c), 1), dtype=torch.int64, device=dev) for c in caps]
    for i, q in enumerate(queries):
        smg.search_into(text, plans[i], outs[i], cnt[i:i + 1], n=q.n or n, cap=int(caps[i]))
    smg.sync()
    dfa = {}
    for i, q in enumerate(queries):
        m = len(q.pattern)
        dense_q = bool(q.n)
        if not dense_q and i % (2 * per_m) != 0:
            continue
        if (m + 1) * (len(set(q.pattern)) + 1) * 2 > 32768 - 256:
            continue
        nn = q.n or n
        plan = smg.prepare(q.pattern, sigma_hint=4, variant="dfa")
        out_d = torch.empty(max(int(caps[i]), 1), dtype=torch.int64, device=dev)
        cnt_d = torch.zeros(1, dtype=torch.int64, device=dev)
        t = time_search(text, plan, out_d, cnt_d, nn, int(caps[i]))
        same = int(cnt_d.item()) == int(caps[i]) and bool(torch.equal(out_d[:int(caps[i])], outs[i][:int(caps[i])]))
        key = "dense" if dense_q else "substring"
        dfa.setdefault(str(m), {})[key] = {
            "ms": round(t * 1e3, 4), "hits": int(caps[i]), "GBs": round(nn / t / 1e9, 1),
            "alg_GBs": round((nn + 8 * int(caps[i])) / t / 1e9, 1), "auto_ms": res[i]["ms"],
            "auto_variant": res[i]["variant"], "equal_to_auto": same}
    # Parity on samples: every hit the GPU reports inside a few windows of the
    # text, and the count there, against the oracle on the host's copy of the
    # window (regenerated from the seed).
    import oracle
    rng = np.random.default_rng(5)
    checked, ok = 0, True
    sample = sorted(set(rng.integers(0, len(w.queries), 6).tolist())) if n > workloads.DENSE_PREFIX + (4 << 20) else []
    for i in sample:
        q = w.queries[i]
        m = len(q.pattern)
        got_all = outs[i][:int(caps[i])]
        for _ in range(3):
            lo = int(rng.integers(workloads.DENSE_PREFIX, n - (1 << 20)))
            hi = lo + (1 << 20)
            win = spec.window(lo, hi - lo + m - 1)
            exp = oracle.naive(win, q.pattern).astype(np.int64) + lo
            a0 = int(torch.searchsorted(got_all, torch.tensor([lo], device=dev)).item())
            b0 = int(torch.searchsorted(got_all, torch.tensor([hi], device=dev)).item())
            ok &= bool(np.array_equal(got_all[a0:b0].cpu().numpy(), exp))
            checked += 1
    out.update({"workload": w.name, "metric": METRIC,
                "parity_sample": {"windows": checked, "window_bytes": 1 << 20, "ok": ok},
                "dfa": dfa, "results": res})
    return out


def bench_bandwidth(args, world, rank, local):
    import __graft_entry__
    __graft_entry__.build()
    tuning = load_tuning(args, sigmas=(4,))
    rec = bandwidth_record(args, local)
    rec["tuning"] = tuning
    print(json.dumps(rec))


# ---------------------------------------------------------------- batched workload

def device_text(smg, spec, dev):
    """A counter-based TextSpec built on the device by sm_gen_text."""
    import numpy as np
    import torch
    t = torch.empty(spec.n, dtype=torch.uint8, device=dev)
    if spec.kind == "uniform":
        smg.gen_text(t, 0, spec.key, spec.sigma)
    else:
        thr = torch.tensor(np.asarray(spec.thresholds, dtype=np.uint32).view(np.int32), device=dev)
        bm = torch.tensor(np.asarray(spec.byte_map, dtype=np.uint8), device=dev)
        smg.gen_text(t, 0, spec.key, 0, thr, bm)
    return t


def bench_batched(args, world, rank, local):
    """Batched queries: (i) 4096 patterns of log-uniform length on one shared
    1 GiB sigma = 20 skewed text, (ii) 10,000 (pattern, text) pairs with
    texts of 4 KiB .. 64 MiB over sigma 4 / 64.  Each part runs as one
    graph-captured batch (one persistent launch per kernel family, kernels
    picked by the autotuned table) and, for comparison, as one launch per
    query (sm_search_plan on the same plans and outputs).  L2 is flushed
    before each timed pass.  Reports queries/s and scanned GB/s of both."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import paper_1012_2547_gb300 as smg
    from paper_1012_2547_gb300 import workloads

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    tuning = load_tuning(args, sigmas=(4, 16, 64))
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    rng = np.random.default_rng(3)
    parts = {}
    for name, w in (("shared_1GiB_sigma20_q4096", workloads.batched_shared()),
                    ("pairs_10000_4KiB-64MiB_sigma4-64", workloads.batched_pairs())):
        base = [device_text(smg, sp, dev) for sp in w.specs]
        texts = [base[q.text_id][q.offset:q.offset + (q.n or w.specs[q.text_id].n)] for q in w.queries]
        smg.sync()
        nq = len(w.queries)
        plans = [None] * nq
        by_sigma = {}
        for i, q in enumerate(w.queries):
            by_sigma.setdefault(q.sigma_hint, []).append(i)
        for sg, idx in by_sigma.items():
            for i, p in zip(idx, smg.prepare_many([w.queries[i].pattern for i in idx], sigma_hint=sg)):
                plans[i] = p
        cnt = torch.zeros(nq, dtype=torch.int64, device=dev)
        smg.search_batch([(texts[i], plans[i], None, cnt[i:i + 1]) for i in range(nq)])
        smg.sync()
        c = cnt.cpu().numpy()
        offs = np.concatenate([[0], np.cumsum(c)])
        out = torch.empty(max(int(c.sum()), 1), dtype=torch.int64, device=dev)
        items = [(texts[i], plans[i], out[int(offs[i]):int(offs[i + 1])], cnt[i:i + 1]) for i in range(nq)]
        batch = smg.Batch(items, graph=True)
        scanned = sum(t.numel() for t in texts)

        def timed(fn, reps):
            ts = []
            for r in range(args.warmup + reps):
                flush.zero_()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                torch.cuda.synchronize()
                if r >= args.warmup:
                    ts.append(e0.elapsed_time(e1) / 1e3)
            return statistics.median(ts)

        l0 = smg.kernel_launches()
        tb = timed(lambda: batch.launch(stream), args.steps)
        launches_b = (smg.kernel_launches() - l0) // (args.warmup + args.steps)

        def per_query():
            for i in range(nq):
                smg.search_into(texts[i], plans[i], items[i][2], cnt[i:i + 1], cap=int(c[i]))
        l0 = smg.kernel_launches()
        tq = timed(per_query, max(1, min(args.steps, 3)))
        launches_q = (smg.kernel_launches() - l0) // (args.warmup + max(1, min(args.steps, 3)))
        smg.sync()
        # parity: a sample of queries against the oracle (whole text when it
        # is small, else every hit in a few 1 MiB windows)
        ok, checked = True, 0
        for i in sorted(set(rng.integers(0, nq, 8).tolist())):
            q = w.queries[i]
            spec = w.specs[q.text_id]
            n = q.n or spec.n
            got = out[int(offs[i]):int(offs[i + 1])]
            m = len(q.pattern)
            if n <= (8 << 20):
                exp = oracle.naive(spec.window(q.offset, n), q.pattern)
                ok &= int(cnt[i].item()) == len(exp) and bool(np.array_equal(got.cpu().numpy().astype(np.uint64), exp))
            else:
                for _ in range(2):
                    lo = int(rng.integers(0, n - (1 << 20)))
                    exp = oracle.naive(spec.window(q.offset + lo, (1 << 20) + m - 1), q.pattern).astype(np.int64) + lo
                    a = int(torch.searchsorted(got, torch.tensor([lo], device=dev)).item())
                    b = int(torch.searchsorted(got, torch.tensor([lo + (1 << 20)], device=dev)).item())
                    ok &= bool(np.array_equal(got[a:b].cpu().numpy(), exp))
            checked += 1
        parts[name] = {
            "queries": nq, "scanned_bytes": scanned, "positions": int(c.sum()),
            "batched": {"ms": round(tb * 1e3, 3), "queries_per_s": round(nq / tb, 1),
                        "scanned_GBs": round(scanned / tb / 1e9, 1), "launches": int(launches_b)},
            "per_query": {"ms": round(tq * 1e3, 3), "queries_per_s": round(nq / tq, 1),
                          "scanned_GBs": round(scanned / tq / 1e9, 1), "launches": int(launches_q)},
            "speedup": round(tq / tb, 2),
            "parity_sample": {"queries": checked, "ok": ok},
        }
        batch.free()
        for p in plans:
            p.free()
        del out, texts, base, items, batch
        torch.cuda.empty_cache()
    hbm, kind = peaks()
    print(json.dumps({"workload": "batched", "metric": "queries/s and scanned GB/s, batched vs one launch per query",
                      "peak_gbs": hbm, "peak_kind": kind, "l2": "flushed (256 MiB write) before each pass",
                      "tuning": tuning, "parts": parts}))


# ---------------------------------------------------------------- serving workload

def serve_record(args, local, loads=None) -> dict:
    """Serving (continuous batching) vs one launch per query, on two resident
    corpora (uniform sigma = 4 and Zipf English-like), m log-uniform in
    [2, 512], 70 % corpus queries and 30 % carrying their own text
    (log-uniform 4 KiB .. 16 MiB).  Reports saturated queries/s of both
    paths and p50/p99 latency under Poisson arrivals at fractions of the
    batched capacity."""
    import numpy as np
    import torch

    import paper_1012_2547_gb300 as smg
    from paper_1012_2547_gb300 import gen
    from paper_1012_2547_gb300.serve import Server

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    C = args.serve_corpus
    specs = {"rand4": gen.uniform_text(C, 4, 61), "english": gen.english_text(C, 62)}
    corp = {}
    for k, sp in specs.items():
        t = torch.empty(C, dtype=torch.uint8, device=dev)
        if sp.kind == "uniform":
            smg.gen_text(t, 0, sp.key, sp.sigma)
        else:
            thr = torch.tensor(np.asarray(sp.thresholds, dtype=np.uint32).view(np.int32), device=dev)
            bm = torch.tensor(np.asarray(sp.byte_map, dtype=np.uint8), device=dev)
            smg.gen_text(t, 0, sp.key, 0, thr, bm)
        corp[k] = t
    smg.sync()
    pool = {4: gen.uniform_text(64 << 20, 4, 63).host(), 90: gen.english_text(64 << 20, 64).host()}
    key = gen.stream_key(65, 1)
    reqs = []
    for i in range(args.serve_queries):
        m = gen.log_uniform_int(key, 4 * i, 2, 512)
        if gen.draw_int(key, 4 * i + 1) % 10 < 7:
            name = "rand4" if i % 2 else "english"
            off = gen.draw_int(key, 4 * i + 2) % (C - m)
            pat = bytes(specs[name].window(off, m))
            reqs.append((pat, name, None))
        else:
            sg = 4 if i % 2 else 90
            n = gen.log_uniform_int(key, 4 * i + 3, 4096, 16 << 20)
            off = gen.draw_int(key, 4 * i + 2) % ((64 << 20) - n)
            t = pool[sg][off:off + n]
            pat = bytes(t[(n - m) // 2:(n - m) // 2 + m]) if n > m else bytes(m)
            reqs.append((pat, None, t))
    scanned = sum(C if r[1] else len(r[2]) for r in reqs)

    def run_server(arrival_rate=None):
        srv = Server(corp, budget_bytes=args.serve_budget, streams=4, max_batch=512)
        # Each result is consumed when it is ready, as the clients of a
        # service would (a callback keeps its length and lets it go), so
        # finished results do not pile up behind slower ones.
        lens = [None] * len(reqs)
        cond = threading.Condition()
        ndone = [0]

        def consume(f, k):
            lens[k] = len(f.result())
            with cond:
                ndone[0] += 1
                cond.notify()

        t0 = time.perf_counter()
        if arrival_rate:
            # Poisson arrivals: every request whose scheduled arrival has
            # passed is submitted with that time as its arrival (so any lag
            # of this loop counts as latency), then the loop sleeps.
            arrive = t0 + np.cumsum(np.random.default_rng(1).exponential(1.0 / arrival_rate, len(reqs)))
            k = 0
            while k < len(reqs):
                now = time.perf_counter()
                while k < len(reqs) and arrive[k] <= now:
                    pat, name, own = reqs[k]
                    srv.submit(pat, corpus=name, text=own, t_arrival=float(arrive[k])).add_done_callback(
                        functools.partial(consume, k=k))
                    k += 1
                if k < len(reqs):
                    time.sleep(min(max(arrive[k] - time.perf_counter(), 0.0), 0.001))
        else:
            for k, (pat, name, own) in enumerate(reqs):
                srv.submit(pat, corpus=name, text=own).add_done_callback(functools.partial(consume, k=k))
        with cond:
            while ndone[0] < len(reqs):
                cond.wait(60.0)
        dt = time.perf_counter() - t0
        srv.close()
        st = srv.stats()
        st["seconds"] = round(dt, 3)
        st["qps"] = round(len(reqs) / dt, 1)
        return st, lens

    run_server()  # warm-up (allocator, module load)
    sat, results = run_server()
    # one launch per query, same queries, synchronous
    t0 = time.perf_counter()
    lat1 = []
    unb_counts = []
    for pat, name, own in reqs:
        ts = time.perf_counter()
        text = corp[name] if name else torch.from_numpy(own).to(dev)
        pos = smg.search(text, pat).cpu()  # positions delivered to the host, as served
        unb_counts.append(pos.numel())
        lat1.append(time.perf_counter() - ts)
    unb_dt = time.perf_counter() - t0
    same = all(r == c for r, c in zip(results, unb_counts))
    by_load = {}
    for frac in (args.serve_loads if loads is None else loads):
        st, _ = run_server(arrival_rate=frac * sat["qps"])
        by_load[str(frac)] = {"offered_qps": round(frac * sat["qps"], 1), "qps": st["qps"],
                            "served_over_offered": round(st["qps"] / (frac * sat["qps"]), 3),
                            "p50_ms": round(st["p50_ms"], 3), "p99_ms": round(st["p99_ms"], 3),
                            "queue_p50_ms": st["queue_p50_ms"], "queue_p99_ms": st["queue_p99_ms"],
                            "host_max_ms": st["host_max_ms"],
                            "by_length_class": st["by_length_class"], "batches": st["batches"],
                            "retries": st["retries"], "rates": st["rates"], "host_s": st["host_s"]}
    out = {
        "workload": f"serve_{len(reqs)}q_corpus{C}", "metric": "served queries/s, p50/p99 latency",
        "queries": len(reqs), "scanned_bytes": scanned,
        "batched": {"qps": sat["qps"], "scanned_GBs": round(scanned / sat["seconds"] / 1e9, 1),
                    "batches": sat["batches"], "retries": sat["retries"], "host_s": sat["host_s"],
                    "pinned_pool_bytes": sat["pinned_pool_bytes"],
                    "seconds": sat["seconds"]},
        "unbatched": {"qps": round(len(reqs) / unb_dt, 1),
                      "p50_ms": round(float(np.percentile(lat1, 50)) * 1e3, 3),
                      "p99_ms": round(float(np.percentile(lat1, 99)) * 1e3, 3)},
        "speedup_qps": round(sat["qps"] / (len(reqs) / unb_dt), 2),
        "poisson": by_load, "counts_match_unbatched": same,
    }
    del corp
    torch.cuda.empty_cache()
    return out


def bench_serve(args, world, rank, local):
    import __graft_entry__
    __graft_entry__.build()
    print(json.dumps(serve_record(args, local)), flush=True)


# ---------------------------------------------------------------- reference arm

def run_reference(args, world, rank):
    """The reference arm of this tier: the CPU oracle (threaded naive) on the
    host cores.  Each step times a bounded sample of the workload's searches
    (spread over texts and lengths); value = sample bytes / sample time, and
    ms_per_step is the measured time of one sample."""
    from paper_1012_2547_gb300 import workloads
    w = workloads.sweep(**sweep_kwargs(args)) if args.workload == "sweep" else workloads.single()
    threads = os.cpu_count() or 1
    budget = max(1.0, args.ref_seconds / max(1, args.steps + args.warmup))
    secs, nbytes, nsearch = [], [], []
    for r in range(args.warmup + args.steps):
        b, s, k = cpu_sample_time(w.texts, w.queries, budget, threads)
        if r >= args.warmup:
            secs.append(s)
            nbytes.append(b)
            nsearch.append(k)
    value = sum(nbytes) / sum(secs) / 1e9
    sample = (f"each step: the first ~{budget:.1f} s of searches of the workload, spread over its texts "
              f"and lengths ({min(nsearch)}-{max(nsearch)} of {len(w.queries)} searches, "
              f"{min(nbytes) / 1e9:.2f}-{max(nbytes) / 1e9:.2f} GB), threaded naive oracle")
    return {
        "impl": "reference",
        "metric": METRIC,
        "value": round(value, 4), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(statistics.mean(secs) * 1e3, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic",
        "config": workload_config(w, world),
        "sample_bytes_per_step": round(statistics.mean(nbytes)),
        "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["sweep", "single", "bandwidth", "batched", "serve"], default="sweep")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cells", action="store_true", help="skip the per-(sigma, m) table")
    ap.add_argument("--no-tune", action="store_true", help="keep the built-in kernel rule")
    ap.add_argument("--tune", action="store_true", help="re-measure the tuning table on this device")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=60.0)
    ap.add_argument("--bw-bytes", type=int, default=8 << 30)
    ap.add_argument("--ms", default="", help="sweep subset: comma-separated pattern lengths")
    ap.add_argument("--per-m", type=int, default=0, help="sweep subset: patterns per (text, m)")
    ap.add_argument("--serve-queries", type=int, default=4000)
    ap.add_argument("--serve-corpus", type=int, default=2 << 30)
    ap.add_argument("--serve-budget", type=int, default=40 << 30)
    ap.add_argument("--serve-loads", type=float, nargs="*", default=[0.5, 0.8, 0.95])
    ap.add_argument("--serve-no-unbatched", action="store_true")
    ap.add_argument("--no-side", action="store_true",
                    help="default line without the bandwidth and serving records")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    world, rank, local = dist_env()
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, world, rank)), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    try:
        if args.workload == "bandwidth":
            if rank == 0:
                bench_bandwidth(args, world, rank, local)
            return
        if args.workload == "serve":
            if rank == 0:
                bench_serve(args, world, rank, local)
            return
        if args.workload == "batched":
            if rank == 0:
                bench_batched(args, world, rank, local)
            return
        out = run_ours(args, world, rank, local)
        if rank == 0 and args.workload == "sweep" and not args.no_side:
            # The single-pattern bandwidth scans and the serving loop, in
            # compact form, so one default run reports every half of the
            # metric (each also runs alone: --workload bandwidth / serve).
            # The sweep leaves tens of thousands of Python objects behind;
            # freezing them keeps the garbage collector's full passes (which
            # stop the serving scheduler thread) short.
            import gc
            gc.collect()
            gc.freeze()
            out["bandwidth"] = bandwidth_record(args, local, compact=True)
            # The committed tuning table is measured on the sweep's 4 MiB
            # texts; the server's 2 GiB corpora run with the built-in rule,
            # as in the standalone serving bench.
            import paper_1012_2547_gb300 as smg
            smg.tuning_reset()
            out["serve"] = serve_record(args, local, loads=[0.5, 0.8, 0.95])
            out["serve"]["kernel_choice"] = "built-in rule (tuning table reset)"
        if rank == 0:
            print(json.dumps(out), flush=True)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
