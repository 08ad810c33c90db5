#!/usr/bin/env python
"""Throughput of the gather-and-refine scoring path (QPS, p50/p99 batch latency).

One step = one batch of queries through all four steps (top centroids, gather,
refine, top-k) on synthetic data shaped like the full-scale passage-ranking
workload (8.8M docs, ~594M tokens, 2,097,152 bf16 centroids, 16-byte PQ codes,
batches of 256 queries x 32 tokens, k = 10); --workload picks another one
(msmarco-1M: 1M docs, batches of 64; lotte-2.8M: 2.8M docs, 32-byte codes,
512 queries of 8-32 tokens). Every reported number states its accuracy against
the FP64 oracle on a sample of the timed queries.

  python bench.py [--gpus N --steps K --warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the only other implementation of
this path) on the host cores, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD = "msmarco-8.8M"
# per workload: queries per batch, token count range of a query
SHAPES = {"tiny": (16, 32, 32), "msmarco-1M": (64, 32, 32), "msmarco-8.8M": (256, 32, 32),
          "lotte-2.8M": (512, 8, 32)}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--batch", type=int, default=0, help="queries per batch (0: the workload's)")
    ap.add_argument("--k", type=int, default=10)
    ap.add_argument("--kc", type=int, default=40)
    ap.add_argument("--kd", type=int, default=1000)
    ap.add_argument("--precision", default="auto", choices=["auto", "fp32", "bf16", "fp8"])
    ap.add_argument("--oracle-queries", type=int, default=0,
                    help="queries checked against the oracle (0: one per host core, at most 16)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--profile-only", action="store_true", help="short run for ncu captures")
    ap.add_argument("--single-queries", type=int, default=32,
                    help="queries of the FP32 one-query-at-a-time comparator")
    ap.add_argument("--no-single", action="store_true")
    ap.add_argument("--no-rerank", action="store_true", help="skip the rerank-only measurement")
    ap.add_argument("--no-sweep", action="store_true", help="skip the k = 100 / 1000 and FP32 batched lines")
    ap.add_argument("--rescore-margin", type=float, default=0.0,
                    help="FP8 repair window of the timed path (0: the library's default)")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving measurement")
    ap.add_argument("--tune-budgets", action="store_true",
                    help="pick kappa_c and kappa_d with the library's autotuner (default on lotte-2.8M)")
    ap.add_argument("--tune-queries", type=int, default=64)
    ap.add_argument("--serving-workload", default="msmarco-1M")
    ap.add_argument("--serving-rates", type=float, nargs="*", default=[1000, 10000, 20000])
    ap.add_argument("--serving-seconds", type=float, default=10.0)
    ap.add_argument("--fp8-windows", type=float, nargs="*", default=[0.1],
                    help="FP8 repair windows (multiples of the rigorous bound) timed in the sweep")
    a = ap.parse_args()
    shape = SHAPES.get(a.workload, (64, 32, 32))
    if a.batch <= 0:
        a.batch = shape[0]
    a.ntok_min, a.ntok_max = shape[1], shape[2]
    if a.oracle_queries <= 0:
        a.oracle_queries = min(16, host_cores())
    if a.workload == "lotte-2.8M":
        a.tune_budgets = True
    return a


def host_cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


# clock-event reason bits of NVML (nvmlClocksEventReason*), the ones a bench line reports
_NVML_REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown"}


def _nvml_open(dev):
    """A function returning (SM MHz, max SM MHz, clock-event reason bits) of CUDA device `dev`, read
    through NVML - the pynvml module where it is installed, else the driver's libnvidia-ml through
    ctypes - or None when neither answers. Only read calls; the device is matched by PCI bus id."""
    bus = []
    try:
        import torch
        p = torch.cuda.get_device_properties(dev)
        bus = [f.format(p.pci_domain_id, p.pci_bus_id, p.pci_device_id).encode()
               for f in ("{:08X}:{:02X}:{:02X}.0", "{:04X}:{:02X}:{:02X}.0")]
    except Exception:
        pass
    try:
        import pynvml
        pynvml.nvmlInit()
        h = None
        for b in bus:
            try:
                h = pynvml.nvmlDeviceGetHandleByPciBusId(b)
                break
            except Exception:
                pass
        if h is None:
            h = pynvml.nvmlDeviceGetHandleByIndex(dev)
        get = getattr(pynvml, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            pynvml.nvmlDeviceGetCurrentClocksThrottleReasons
        return lambda: (pynvml.nvmlDeviceGetClockInfo(h, pynvml.NVML_CLOCK_SM),
                        pynvml.nvmlDeviceGetMaxClockInfo(h, pynvml.NVML_CLOCK_SM), int(get(h)))
    except Exception:
        pass
    try:
        import ctypes
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        ptr, u, ull = ctypes.c_void_p, ctypes.c_uint, ctypes.c_ulonglong
        lib.nvmlInit_v2.restype = ctypes.c_int
        lib.nvmlDeviceGetHandleByPciBusId_v2.argtypes = [ctypes.c_char_p, ctypes.POINTER(ptr)]
        lib.nvmlDeviceGetHandleByIndex_v2.argtypes = [u, ctypes.POINTER(ptr)]
        lib.nvmlDeviceGetClockInfo.argtypes = [ptr, ctypes.c_int, ctypes.POINTER(u)]
        lib.nvmlDeviceGetMaxClockInfo.argtypes = [ptr, ctypes.c_int, ctypes.POINTER(u)]
        rfn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        rfn.argtypes = [ptr, ctypes.POINTER(ull)]
        if lib.nvmlInit_v2() != 0:
            return None
        h = ptr()
        if not (any(lib.nvmlDeviceGetHandleByPciBusId_v2(b, ctypes.byref(h)) == 0 for b in bus) or
                lib.nvmlDeviceGetHandleByIndex_v2(dev, ctypes.byref(h)) == 0):
            return None
        nvml_clock_sm = 1

        def read():
            sm, mx, bits = u(), u(), ull()
            if (lib.nvmlDeviceGetClockInfo(h, nvml_clock_sm, ctypes.byref(sm)) or
                    lib.nvmlDeviceGetMaxClockInfo(h, nvml_clock_sm, ctypes.byref(mx)) or
                    rfn(h, ctypes.byref(bits))):
                raise RuntimeError("NVML read failed")
            return sm.value, mx.value, bits.value
        read()
        return read
    except Exception:
        return None


class Clocks:
    """SM clock and clock-event (throttle) reasons sampled during the timed region: NVML reads
    every 2 ms from a thread plus the samples the timing loop takes with mark() while the device
    is busy (a step takes a few ms, too short for nvidia-smi's polling); nvidia-smi at 100 ms
    when NVML is unavailable. Reads only: no clock or other setting is changed."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.samples = []   # (sm MHz, max sm MHz, set of active reasons)
        self.proc = None
        self.read = None
        self.stop = threading.Event()
        self.t = None

    def _nvml_sample(self):
        try:
            sm, mx, bits = self.read()
        except Exception:
            return
        self.samples.append((float(sm), float(mx), {n for b, n in _NVML_REASONS.items() if bits & b}))

    def mark(self):
        """One sample now (call while the device runs the timed work)."""
        if self.read is not None:
            self._nvml_sample()

    def _poll(self):
        while not self.stop.is_set():
            self._nvml_sample()
            self.stop.wait(0.002)

    def __enter__(self):
        self.read = _nvml_open(self.dev)
        if self.read is not None:
            self.t = threading.Thread(target=self._poll, daemon=True)
            self.t.start()
            return self
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.proc.stdout:
            r = [x.strip() for x in line.split(",")]
            try:
                sm, mx = float(r[1]), float(r[2])
            except (IndexError, ValueError):
                continue
            self.samples.append((sm, mx, {n for i, n in enumerate(names) if len(r) > 5 + i and
                                          r[5 + i].lower() == "active"}))

    def __exit__(self, *a):
        self.stop.set()
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.t is not None and self.read is not None:
            self.t.join(timeout=1)

    def summary(self):
        return clocks_summary(self.samples, "nvml" if self.read is not None else "nvidia-smi")


def clocks_summary(samples, source):
    """Median SM clock, max SM clock and the union of active reasons over the samples."""
    if not samples:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0, "source": source}
    reasons = set()
    for _, _, r in samples:
        reasons |= r
    return {"sm_mhz": float(np.median([x[0] for x in samples])), "sm_max_mhz": max(x[1] for x in samples),
            "reasons": sorted(reasons), "samples": len(samples), "source": source}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_query_seed(cfg, rank):
    """Each replica draws its own query stream."""
    return cfg.query_seed + 7919 * rank


def combine_over_ranks(elapsed, units, world, device="cpu"):
    """(max elapsed over the ranks, units summed over the ranks): the whole job's
    throughput is units / elapsed. Plain values with one rank."""
    if world <= 1:
        return float(elapsed), float(units)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(elapsed)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def load_workload(name, device, rank, world, log):
    """Index (cached on local disk) + the query stream."""
    import torch
    if world > 1:
        import torch.distributed as dist
        if rank == 0:
            ix = synth.load_or_make(name, device=device, log=log)
        dist.barrier()
        if rank != 0:
            ix = synth.load_or_make(name, device=device, log=log)
    else:
        ix = synth.load_or_make(name, device=device, log=log)
    return ix


def measured_traffic(kernels, workload, batch):
    """DRAM bytes per launch summed over the kernels of one launcher, from the committed ncu
    capture of this workload; None when there is none, it was taken at another batch size, or a
    kernel's source has changed since."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"dram_traffic_{workload}.txt")
    if not os.path.exists(path):
        return None
    got = {}
    for line in open(path):
        if line.startswith("# batch ") and int(line.split()[2]) != batch:
            return None
        f = line.split()
        if len(f) != 4 or line.startswith("#") or f[0] not in kernels:
            continue
        src = os.path.join(ROOT, f[2])
        if not os.path.exists(src) or hashlib.sha256(open(src, "rb").read()).hexdigest() != f[3]:
            return None
        got[f[0]] = got.get(f[0], 0) + int(f[1])
    return sum(got.values()) if all(k in got for k in kernels) else None


def data_desc(a):
    shape = "long-tail QA" if a.workload.startswith("lotte") else "passage-ranking"
    return f"synthetic (seeded generator shaped like the {shape} workload)"


def workload_desc(a, ix):
    return (f"{a.workload}: {ix['doc_offsets'].shape[0] - 1} docs, {int(ix['doc_offsets'][-1])} tokens, "
            f"C={ix['centroids'].shape[0]} {ix['centroid_dtype']}, PQ {ix['pq_codebooks'].shape[0]}x8b")


def tok_desc(a):
    return a.ntok_min if a.ntok_min == a.ntok_max else f"{a.ntok_min}-{a.ntok_max} (uniform, packed)"


def time_batches(G, params, batches, idx, k, flush, torch):
    """CUDA-event time of G.search over the batches idx (k per query), L2 flushed between
    batches outside the events; returns the per-batch ms and the status flags."""
    stream = torch.cuda.current_stream()
    out = []
    for b in idx[:2]:  # sizes the scratch for this k
        nq = len(batches[b][1])
        oi = torch.empty(nq * k, dtype=torch.int32, device="cuda")
        os_ = torch.empty(nq * k, dtype=torch.float32, device="cuda")
        G.search(params, batches[b][0], batches[b][1], np.full(nq, k, np.int32), oi, os_)
    torch.cuda.synchronize()
    G.stream_status()
    for b in idx:
        nq = len(batches[b][1])
        kk = np.full(nq, k, np.int32)
        oi = torch.empty(nq * k, dtype=torch.int32, device="cuda")
        os_ = torch.empty(nq * k, dtype=torch.float32, device="cuda")
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        G.search(params, batches[b][0], batches[b][1], kk, oi, os_)
        e1.record(stream)
        torch.cuda.synchronize()
        out.append(e0.elapsed_time(e1))
    return np.array(out), G.stream_status()


def fp32_one_at_a_time(T, G, a, batch, batched_ids, torch):
    """The plain FP32 path (no tensor cores, no batching) on the first queries of a timed
    batch, one query per search call; per-query latency from CUDA events, and whether
    every result equals the batched reduced-precision one."""
    dq, ntok = batch
    n = min(a.single_queries, len(ntok))
    off = np.concatenate([[0], np.cumsum(ntok)])
    p32 = T.SearchParams(kappa_c=a.kc, kappa_d=a.kd, precision=T.PREC_FP32)
    oi = torch.empty(a.k, dtype=torch.int32, device="cuda")
    os_ = torch.empty(a.k, dtype=torch.float32, device="cuda")
    k1 = np.array([a.k], np.int32)
    stream = torch.cuda.current_stream()
    same = True
    lat = []
    for rep in range(2):  # the first pass sizes the scratch and warms the caches
        for u in range(n):
            qu = dq[off[u]:off[u + 1]]
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            G.search(p32, qu, ntok[u:u + 1], k1, oi, os_)
            e1.record(stream)
            torch.cuda.synchronize()
            if rep == 1:
                lat.append(e0.elapsed_time(e1))
                same = same and bool(torch.equal(oi, batched_ids[u * a.k:(u + 1) * a.k]))
    lat = np.array(lat)
    return {"value": float(n / (lat.sum() / 1e3)), "unit": "queries/s", "queries": int(n),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "ids_equal_to_batched": same}


def rerank_only(T, G, a, params, batches, n_docs, flush, torch):
    """Steps (c)-(d) alone (tachiom_refine) over candidate lists that come from outside the
    cascade, as a reranker of another retriever's output gets them: per query kappa_d distinct
    seeded document ids in random order. Inputs device-resident, L2 flushed between batches
    outside the events; CUDA events per batch on the launching stream."""
    rng = np.random.default_rng(20260428)
    nl = min(6, len(batches))
    cands = []
    for _ in range(nl):
        rows = []
        for _ in range(a.batch):
            ids = np.unique(rng.integers(0, n_docs, size=2 * a.kd))
            if ids.size < a.kd:
                ids = rng.choice(n_docs, size=a.kd, replace=False)
            rows.append(rng.permutation(ids[:a.kd]).astype(np.int32))
        cands.append(torch.from_numpy(np.stack(rows)).cuda())
    kk = np.full(a.batch, a.k, np.int32)
    oi = torch.empty(a.batch * a.k, dtype=torch.int32, device="cuda")
    os_ = torch.empty(a.batch * a.k, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    for b in range(min(2, nl)):
        G.refine(params, batches[b][0], batches[b][1], kk, cands[b], oi, os_)
    torch.cuda.synchronize()
    ms = []
    for b in range(nl):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        G.refine(params, batches[b][0], batches[b][1], kk, cands[b], oi, os_)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    ms = np.array(ms)
    return {"value": float(a.batch * nl / (ms.sum() / 1e3)), "unit": "queries/s", "batches": nl,
            "ms_per_batch": float(ms.mean()), "batch": a.batch, "kappa_d": a.kd, "k": a.k,
            "lists": "per query kappa_d distinct seeded document ids, random order"}


def oracle_check(ix, qs, ntok, gi, gs, k, kc, kd, nsample):
    """Top-10 overlap and score error of the GPU result vs the FP64 oracle on a sample."""
    from oracle import Oracle
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    O = Oracle(ix)
    qoff = np.concatenate([[0], np.cumsum(ntok)])
    sel = np.arange(min(nsample, len(ntok)))
    rows = np.concatenate([np.arange(qoff[u], qoff[u + 1]) for u in sel])
    t0 = time.perf_counter()
    res = O.search(qs[rows], ntok[sel], k, kc, kd)
    dt = time.perf_counter() - t0
    return accuracy_vs(res, sel, gi, gs, k), dt, len(sel), res


def accuracy_vs(res, sel, gi, gs, k):
    """Top-10 overlap and score error of a GPU result against the oracle's result on queries sel."""
    ov, err = [], []
    for j, u in enumerate(sel):
        g = gi[u * k:(u + 1) * k]
        o = res["ids"][j * k:(j + 1) * k]
        a = set(g[:10].tolist()) - {-1}
        b = set(o[:10].tolist()) - {-1}
        ov.append(len(a & b) / max(1, len(b)))
        os_ = res["scores"][j * k:(j + 1) * k]
        m = np.isfinite(os_)
        err.append(float(np.max(np.abs(gs[u * k:(u + 1) * k][m] - os_[m]) / np.maximum(1, np.abs(os_[m])))
                   if m.any() else 0.0))
    return {"queries": int(len(sel)), "overlap_at_10": float(np.mean(ov)), "min_overlap_at_10": float(np.min(ov)),
            "max_rel_score_err": float(np.max(err))}


def algorithmic_traffic(T_idx, ix, params, dq, ntok, k, kc, kd, torch):
    """Per-launch algorithmic bytes of gather and refine for one batch (counted, not modelled)."""
    R = int(ntok.sum())
    nq = len(ntok)
    top = torch.empty((R, kc), dtype=torch.int32, device="cuda")
    tops = torch.empty((R, kc), dtype=torch.float32, device="cuda")
    T_idx.top_centroids(params, dq, top, tops)
    cid = torch.empty((nq, kd), dtype=torch.int32, device="cuda")
    cs = torch.empty((nq, kd), dtype=torch.float32, device="cuda")
    nc = torch.empty(nq, dtype=torch.int32, device="cuda")
    T_idx.gather(params, dq, ntok, top, cid, cs, nc)
    torch.cuda.synchronize()
    off = ix["_list_off"]
    t = top.cpu().numpy()
    lens = (off[t + 1] - off[t]).astype(np.int64)
    entries = int(lens.sum())
    D = ix["doc_offsets"].shape[0] - 1
    # the algorithmic bytes of step (b): every list entry walked (4 B), every Top_i entry (id and
    # score, 8 B) and the kappa_d (doc, score) outputs of each query (8 B)
    gather_bytes = entries * 4 + R * kc * 8 + nq * kd * 8
    cand = cid.cpu().numpy()
    doff = ix["doc_offsets"]
    c = cand[cand >= 0]
    ntoks = int((doff[c + 1] - doff[c]).sum())
    M = ix["pq_codebooks"].shape[0]
    cbytes = 2 if ix["centroid_dtype"] == "bf16" else 4
    refine_bytes = ntoks * (4 + M + 2 + 128 * cbytes)
    return {"list_entries": entries, "gather_bytes": gather_bytes, "refine_tokens": ntoks,
            "refine_bytes": refine_bytes, "select_bytes": nq * kd * 8, "_cand": cid}


def run_ours(a):
    import torch
    import paper_2604_28142_b300 as T
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    log = (lambda m: print(f"[bench] {m}", file=sys.stderr, flush=True)) if rank == 0 else None
    cfg = synth.CONFIGS[a.workload]
    t0 = time.time()
    ix = load_workload(a.workload, "cuda", rank, world, log)
    if log:
        log(f"index ready in {time.time() - t0:.1f}s: T={ix['doc_offsets'][-1]}")
    G = T.Index(ix, local)
    if a.precision == "auto":
        prec = T.PREC_BF16 if T.tc_available() else T.PREC_FP32
    else:
        prec = {"bf16": T.PREC_BF16, "fp8": T.PREC_FP8, "fp32": T.PREC_FP32}[a.precision]
    budget_tune = None
    if a.tune_budgets:
        # candidate budgets from the paper's grid, by cost subject to recall@10 >= 0.95 against the
        # exhaustive top-10 (every document refined) on a tuning split of queries not in the timed ones
        tq = synth.make_queries(cfg, n_queries=a.tune_queries, seed=cfg.query_seed + 77, ntok_min=a.ntok_min,
                                ntok_max=a.ntok_max)
        tdq = torch.from_numpy(tq["queries"]).cuda()
        t0 = time.time()
        (kc_t, kd_t), rec_t, ms_t, table = G.autotune_budgets(prec, tdq, tq["ntok"], 10, [15, 20, 40, 80, 120],
                                                              [250, 500, 1000, 2000, 4000], min_recall=0.95)
        a.kc, a.kd = int(kc_t), int(kd_t)
        budget_tune = {"kappa_c": a.kc, "kappa_d": a.kd, "recall_at_10_vs_exhaustive": rec_t,
                       "tuning_ms_per_batch": ms_t, "tuning_queries": a.tune_queries, "target_recall": 0.95,
                       "grid": [[int(r[0]), int(r[1]), float(r[2]), float(r[3])] for r in table.reshape(-1, 4)],
                       "tuner_seconds": time.time() - t0}
        if log:
            log(f"budgets: kappa_c {a.kc} kappa_d {a.kd} recall {rec_t:.3f} ({time.time() - t0:.1f} s)")
    params = T.SearchParams(kappa_c=a.kc, kappa_d=a.kd, precision=prec, rescore_margin=a.rescore_margin)
    nb = a.warmup + a.steps
    q = synth.make_queries(cfg, n_queries=nb * a.batch, seed=rank_query_seed(cfg, rank), ntok_min=a.ntok_min,
                           ntok_max=a.ntok_max)
    qs, ntok = q["queries"], q["ntok"]
    qoff = np.concatenate([[0], np.cumsum(ntok)])
    batches = []
    for b in range(nb):
        lo, hi = b * a.batch, (b + 1) * a.batch
        batches.append((torch.from_numpy(qs[qoff[lo]:qoff[hi]]).cuda(), ntok[lo:hi].copy()))
    kk = np.full(a.batch, a.k, np.int32)
    out_i = [torch.empty(a.batch * a.k, dtype=torch.int32, device="cuda") for _ in range(nb)]
    out_s = [torch.empty(a.batch * a.k, dtype=torch.float32, device="cuda") for _ in range(nb)]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for b in range(a.warmup):
        G.search(params, batches[b][0], batches[b][1], kk, out_i[b], out_s[b])
    torch.cuda.synchronize()
    if a.profile_only:
        for b in range(a.warmup, nb):
            G.search(params, batches[b][0], batches[b][1], kk, out_i[b], out_s[b])
        torch.cuda.synchronize()
        print(json.dumps({"profile_only": True, "status_flags": G.stream_status()}))
        return
    # ---- timed region (device-resident inputs) ----
    T.profile_enable(True)
    T.profile_read()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        for s in range(a.steps):
            b = a.warmup + s
            flush.zero_()  # L2 flush between steps, outside the step's events
            evs[s][0].record(stream)
            G.search(params, batches[b][0], batches[b][1], kk, out_i[b], out_s[b])
            evs[s][1].record(stream)
            clk.mark()
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    prof = T.profile_read()
    T.profile_enable(False)
    step_ms = np.array([e0.elapsed_time(e1) for e0, e1 in evs])
    tot_ms, queries_total = combine_over_ranks(float(step_ms.sum()), a.steps * a.batch, world, "cuda")
    flags = G.stream_status()
    qps = queries_total / (tot_ms / 1e3)
    # ---- end to end through the host-buffer entry point ----
    e2e = None
    if not a.no_e2e:
        hq = [qs[qoff[(a.warmup + s) * a.batch]:qoff[(a.warmup + s + 1) * a.batch]] for s in range(a.steps)]
        for s in range(min(2, a.steps)):
            G.search_host(params, hq[s], batches[a.warmup + s][1], kk)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for s in range(a.steps):
            G.search_host(params, hq[s], batches[a.warmup + s][1], kk)
        e2e_s, _ = combine_over_ranks(time.perf_counter() - t1, 0, world, "cuda")
        h2d = int(hq[0].nbytes) + (4 * a.batch + 2) * 4
        d2h = a.batch * a.k * 8
        e2e = {"value": queries_total / e2e_s, "unit": "queries/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    # ---- comparator: the plain FP32 path, one query per launch sequence ----
    single = None
    if not a.no_single:
        single = fp32_one_at_a_time(T, G, a, batches[a.warmup], out_i[a.warmup], torch)
    # ---- the same batches with k = 100 and k = 1000 (kappa_d = max(1000, 4k)), and the FP32 path batched ----
    sweep = None
    if not a.no_sweep:
        idx = list(range(a.warmup, min(nb, a.warmup + 5)))
        sweep = {}
        for kx in (100, 1000):
            pk = T.SearchParams(kappa_c=a.kc, kappa_d=0, precision=prec)
            ms, fl = time_batches(G, pk, batches, idx, kx, flush, torch)
            sweep[f"k{kx}"] = {"value": float(a.batch * len(ms) / (ms.sum() / 1e3)), "unit": "queries/s",
                               "ms_per_step": float(ms.mean()), "kappa_d": min(4096, max(1000, 4 * kx)),
                               "status_flags": int(fl)}
        T.profile_enable(True)
        others = [("fp32_batched", T.PREC_FP32, 0.0)]
        if T.tc_available():
            others += [("bf16", T.PREC_BF16, 0.0)] + [(f"fp8_window{w}", T.PREC_FP8, w) for w in a.fp8_windows]
        for nm, pr, w in others:
            if pr == prec and pr != T.PREC_FP8:
                continue
            pp = T.SearchParams(kappa_c=a.kc, kappa_d=a.kd, precision=pr, rescore_margin=w)
            T.profile_read()
            ms, fl = time_batches(G, pp, batches, idx, a.k, flush, torch)
            pf = T.profile_read()
            sweep[nm] = {"value": float(a.batch * len(ms) / (ms.sum() / 1e3)), "unit": "queries/s",
                         "ms_per_step": float(ms.mean()), "k": a.k, "status_flags": int(fl),
                         "stage_ms_per_step": {kk: v[1] / (len(ms) + 2) for kk, v in pf.items()}}
            if pr == T.PREC_FP8:
                kg = G.debug_topc_groups(pp, batches[a.warmup][0])
                sweep[nm]["rescore_margin"] = w
                sweep[nm]["topc_candidates_per_row"] = {"mean": float(kg.mean()), "p99": float(np.percentile(kg, 99)),
                                                        "max": int(kg.max())}
        T.profile_enable(False)
    # ---- the same batches through captured CUDA graphs (tachiom_graph_*: one graph per batch shape,
    # captured outside the events; a launch copies the batch's queries in and replays the search) ----
    graph_rec = None
    if not a.no_sweep:
        idx = list(range(a.warmup, min(nb, a.warmup + 5)))
        graphs = [G.graph(params, batches[b][1], kk) for b in idx]
        gi_ = torch.empty(a.batch * a.k, dtype=torch.int32, device="cuda")
        gs_ = torch.empty(a.batch * a.k, dtype=torch.float32, device="cuda")
        for g_, b in zip(graphs, idx):
            g_.launch(batches[b][0], gi_, gs_)
        torch.cuda.synchronize()
        same = bool(torch.equal(gi_, out_i[idx[-1]]))
        gms = []
        for g_, b in zip(graphs, idx):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g_.launch(batches[b][0], gi_, gs_)
            e1.record(stream)
            torch.cuda.synchronize()
            gms.append(e0.elapsed_time(e1))
        for g_ in graphs:
            g_.close()
        gms = np.array(gms)
        graph_rec = {"value": float(a.batch * len(gms) / (gms.sum() / 1e3)), "unit": "queries/s",
                     "ms_per_step": float(gms.mean()), "batches": len(gms), "ids_equal_to_stream_launch": same}
    # ---- the rerank-only use of steps (c)-(d): external candidate lists ----
    rerank = None
    if not a.no_rerank:
        rerank = rerank_only(T, G, a, params, batches, int(ix["doc_offsets"].shape[0] - 1), flush, torch)
    # ---- accuracy on a sample of the timed queries, and the oracle's own time ----
    b0 = a.warmup
    gi = out_i[b0].cpu().numpy()
    gs = out_s[b0].cpu().numpy()
    qb = qs[qoff[b0 * a.batch]:qoff[(b0 + 1) * a.batch]]
    acc, odt, on, ores = oracle_check(ix, qb, batches[b0][1], gi, gs, a.k, a.kc, a.kd, a.oracle_queries)
    for nm, v in (sweep or {}).items():
        if not nm.startswith("fp8"):
            continue
        # the FP8 path's result on the same queries against the same oracle result
        nq0 = len(batches[b0][1])
        oi8 = torch.empty(nq0 * a.k, dtype=torch.int32, device="cuda")
        os8 = torch.empty(nq0 * a.k, dtype=torch.float32, device="cuda")
        G.search(T.SearchParams(kappa_c=a.kc, kappa_d=a.kd, precision=T.PREC_FP8, rescore_margin=v["rescore_margin"]),
                 batches[b0][0], batches[b0][1], np.full(nq0, a.k, np.int32), oi8, os8)
        torch.cuda.synchronize()
        v["accuracy"] = accuracy_vs(ores, np.arange(on), oi8.cpu().numpy(), os8.cpu().numpy(), a.k)
    # ---- roofline of the dominant launcher ----
    ix["_list_off"] = G.lists()[0]
    traffic = algorithmic_traffic(G, ix, params, batches[b0][0], batches[b0][1], a.k, a.kc, a.kd, torch)
    if prec == T.PREC_BF16:
        kg = G.debug_topc_groups(params, batches[b0][0])
        traffic["topc_candidates_per_row"] = {"mean": float(kg.mean()), "p99": float(np.percentile(kg, 99)),
                                              "max": int(kg.max())}
        # documents the decode-and-MMA refine leaves to the FP32 kernel (same rule as the window kernel)
        cand = traffic["_cand"]
        sa = torch.empty(cand.shape, dtype=torch.float32, device="cuda")
        da = torch.empty(cand.shape, dtype=torch.float32, device="cuda")
        G.debug_refine_scores(params, batches[b0][0], batches[b0][1], cand, sa, da)
        torch.cuda.synchronize()
        cn, san, dan = cand.cpu().numpy(), sa.cpu().numpy(), da.cpu().numpy()
        wins = []
        for u in range(cn.shape[0]):
            ok = (cn[u] >= 0) & np.isfinite(san[u])
            lo, up = (san[u] - dan[u])[ok], (san[u] + dan[u])[ok]
            L = np.sort(lo)[-a.k] if lo.size >= a.k else -np.inf
            wins.append(int((up >= L).sum()))
        traffic["refine_window_docs"] = {"mean": float(np.mean(wins)), "max": int(np.max(wins)),
                                         "mean_bound": float(dan[cn >= 0].mean())}
    traffic.pop("_cand", None)
    import json as _j
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = _j.load(open(pk))
    hbm_peak = peaks.get("hbm_gbs", 6400.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    dom = max(prof.items(), key=lambda kv: kv[1][1])
    name, (launches, ms) = dom
    per_launch_ms = ms / max(1, launches)
    clocks = clk.summary()
    R = float(np.mean([len(batches[a.warmup + s][0]) for s in range(a.steps)]))  # query rows per batch
    C = ix["centroids"].shape[0]
    gemm_flops = 2.0 * R * C * 128
    hbm_kernels = {"gather": (["k_gather_pool"], traffic["gather_bytes"]),
                   "refine": (["k_refine"], traffic["refine_bytes"]),
                   "refine_tc": (["k_refine_tc"], traffic["refine_bytes"]),
                   "refine_dec": (["k_refine_dec"], traffic["refine_bytes"]),
                   "select_kd": (["k_pool_select"], traffic["select_bytes"])}
    tkern = None
    if name in hbm_kernels:
        tkern, nbytes = hbm_kernels[name]
        roof = {"kernel": " + ".join(tkern), "bound": "hbm", "achieved": nbytes / (per_launch_ms * 1e-3) / 1e9,
                "peak": hbm_peak, "unit": "GB/s"}
    elif name == "topc_f32_scan":
        sm = clocks.get("sm_mhz") or 1900.0
        peak_alu = 148 * 128 * 2 * sm * 1e6 / 1e12
        roof = {"kernel": "k_topc_f32_scan", "bound": "alu", "achieved": gemm_flops / (per_launch_ms * 1e-3) / 1e12,
                "peak": peak_alu, "unit": "TFLOP/s"}
        peak_src = "derived: 148 SMs x 128 FP32 lanes x 2 x median SM clock"
    elif name == "topc_tc1":
        pk_t = peaks.get("bf16_tflops", 1800.0)
        roof = {"kernel": "k_topc_tc1", "bound": "tensor",
                "achieved": gemm_flops / (per_launch_ms * 1e-3) / 1e12, "peak": pk_t, "unit": "TFLOP/s"}
    else:
        # the tensor-core launcher timed as one: BF16 - group-maxima pass, threshold, group
        # selection and exact rescoring; FP8 - sample pass, threshold, emission pass and exact
        # rescoring (against twice the measured BF16 peak, the nominal dense E4M3 : BF16 ratio)
        pk_t = peaks.get("bf16_tflops", 1800.0) * (2.0 if prec == T.PREC_FP8 else 1.0)
        tkern = (["k_topc_tc", "k_gsel_lim", "k_gsel_collect", "k_group_rescore"] if prec != T.PREC_FP8 else
                 ["k_topc_tc", "k_gsel_lim", "k_cand_rescore"])
        roof = {"kernel": " + ".join(tkern), "bound": "tensor",
                "achieved": gemm_flops / (per_launch_ms * 1e-3) / 1e12, "peak": pk_t, "unit": "TFLOP/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["peak_source"] = peak_src
    roof["traffic"] = measured_traffic(tkern, a.workload, a.batch) if tkern else None
    roof["per_launch_ms"] = per_launch_ms
    # the HBM-bound kernels beside it: achieved algorithmic bytes per launch and the ncu DRAM bytes
    hbm_side = {}
    for lname, (kl, nbytes) in hbm_kernels.items():
        if lname in prof and lname != name:
            ms = prof[lname][1] / max(1, prof[lname][0])
            ach = nbytes / (ms * 1e-3) / 1e9
            hbm_side[lname] = {"kernel": " + ".join(kl), "algorithmic_bytes": int(nbytes), "per_launch_ms": ms,
                               "achieved_gbs": ach, "frac": ach / hbm_peak,
                               "traffic": measured_traffic(kl, a.workload, a.batch)}
    roof["hbm_kernels"] = hbm_side
    ncores = min(on, host_cores())  # the oracle runs one thread per query
    lat = step_ms
    line = {
        "metric": "QPS at top-10 overlap >=0.99 vs FP64 oracle; p50/p99 latency ms",
        "value": qps,
        "unit": "queries/s",
        "n_gpus": world,
        "steps": a.steps,
        "warmup": a.warmup,
        "ms_per_step": float(lat.mean()),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {T.PREC_BF16: "bf16/f32", T.PREC_FP8: "e4m3/f32"}.get(prec, "f32"),
        "data": data_desc(a),
        "config": {"workload": workload_desc(a, ix),
                   "batch": a.batch, "tokens_per_query": tok_desc(a), "k": a.k, "kappa_c": a.kc, "kappa_d": a.kd,
                   "precision": {T.PREC_BF16: "bf16", T.PREC_FP8: "fp8"}.get(prec, "fp32"),
                   "l2": "flushed between steps (256 MiB write outside the step's events)",
                   "parallelism": f"replicas x{world}"},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "note": "per batch; every query of a batch completes with its batch"},
        "accuracy": acc,
        "stage_ms_per_step": {k: v[1] / a.steps for k, v in prof.items()},
        "status_flags": flags,
        "roofline": roof,
        "traffic_counts": traffic,
        "cpu_baseline": {"value": on / odt, "unit": "queries/s", "cores": ncores, "kind": "oracle",
                         "sample": f"{on} queries of the first timed batch, full cascade in FP64, OpenMP over queries"},
        "clocks": clocks,
        "e2e": e2e,
        "fp32_one_query_at_a_time": single,
        "sweep": sweep,
        "rerank_only": rerank,
        "budget_autotune": budget_tune,
        "graph": graph_rec,
        "gpu_launches": _count_launches(prof),
    }
    if not a.no_serving:
        # the request loop on a resident index: free this workload's index first
        torch.cuda.synchronize()
        G.close()
        line["serving"] = serving_record(a, T, torch, log)
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def _count_launches(prof):
    # kernels per launcher call: topc_tc 4 (GEMM, lim, collect, rescoring), topc_merge 2, the others 1
    per = {"topc_merge": 2, "topc_tc": 4}
    return sum(v[0] * per.get(k, 1) for k, v in prof.items())


def serving_record(a, T, torch, log):
    """Continuous batching under open-loop Poisson arrivals (8-32 tokens per request, k in {10, 100,
    1000} with p = {0.7, 0.25, 0.05}) on the resident index of a.serving_workload: per rate the
    achieved QPS and p50/p95/p99 latency from submission to results on the host, for the batched
    tensor-core path and for the plain FP32 path one query per batch."""
    from paper_2604_28142_b300 import serving
    cfg = synth.CONFIGS[a.serving_workload]
    ix = synth.load_or_make(a.serving_workload, device="cuda", log=log)
    G = T.Index(ix, 0)
    pool = serving.request_pool(synth, cfg)
    out = {"workload": a.serving_workload, "seconds_per_rate": a.serving_seconds, "runs": []}
    paths = [("fp32_one_query", T.PREC_FP32, 1)]
    if T.tc_available():
        paths = [("bf16_batched", T.PREC_BF16, 128)] + paths
    for name, pr, mb in paths:
        params = T.SearchParams(kappa_c=a.kc, kappa_d=0, precision=pr)
        serving.run_rate(T, G, params, pool, 2000, 0.5, 99, 3, mb, 500)  # warm-up: scratch of every slot
        rates = a.serving_rates if mb > 1 else [min(a.serving_rates)]
        for r in rates:
            res = serving.run_rate(T, G, params, pool, r, a.serving_seconds, int(r), 3, mb, 500)
            res["path"] = name
            out["runs"].append(res)
            if log:
                log(f"serving {name} {r}: {res['achieved_qps']:.0f} q/s p50 {res['p50_ms']:.2f} p99 {res['p99_ms']:.2f}")
    return out


def run_reference(a):
    rank, world, local = dist_env()
    if rank != 0:
        return
    import torch
    from oracle import Oracle
    cfg = synth.CONFIGS[a.workload]
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    ix = synth.load_or_make(a.workload, device=dev)
    O = Oracle(ix)
    # the oracle runs its queries in parallel, one per thread; a step's time is one query's latency
    # (its exhaustive step (a) streams the whole centroid table per query token: about 22 s on the
    # 8.8M-document workload whether 4 or 16 queries run at once), so a step takes one query per core
    per_step = max(1, min(16, host_cores()))
    nb = a.warmup + a.steps
    q = synth.make_queries(cfg, n_queries=nb * per_step, seed=cfg.query_seed, ntok_min=a.ntok_min,
                           ntok_max=a.ntok_max)
    qs, ntok = q["queries"], q["ntok"]
    qoff = np.concatenate([[0], np.cumsum(ntok)])
    times = []
    for b in range(nb):
        lo, hi = b * per_step, (b + 1) * per_step
        t0 = time.perf_counter()
        O.search(qs[qoff[lo]:qoff[hi]], ntok[lo:hi], a.k, a.kc, a.kd)
        if b >= a.warmup:
            times.append(time.perf_counter() - t0)
    tot = sum(times)
    qps = a.steps * per_step / tot
    ncores = min(per_step, host_cores())
    line = {
        "impl": "reference",
        "metric": "QPS at top-10 overlap >=0.99 vs FP64 oracle; p50/p99 latency ms",
        "value": qps, "unit": "queries/s", "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": 1e3 * tot / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": data_desc(a),
        "config": {"workload": workload_desc(a, ix), "batch": per_step, "tokens_per_query": tok_desc(a), "k": a.k,
                   "kappa_c": a.kc, "kappa_d": a.kd},
        "latency_ms": {"p50": float(np.percentile(times, 50) * 1e3), "p99": float(np.percentile(times, 99) * 1e3)},
        "cpu_baseline": {"value": qps, "unit": "queries/s", "cores": ncores, "kind": "oracle",
                         "sample": f"{per_step} queries per step, full cascade in FP64, OpenMP over queries"},
        "e2e": {"value": qps, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
