#!/usr/bin/env python3
"""Benchmark of filtered top-K retrieval on one B300 (or N independent replicas).

Workload: N = 10,000,000 jobs, d = 128 FP32 L2-normalised Gaussian embeddings (5.12 GB, larger than
the 126 MB L2, so no flush is needed between steps); V = 16,384 terms, Poisson(40) distinct Zipf(1.1)
terms per job, stored as posting lists plus dense bitmaps of the 256 most frequent terms; query
batches of B filters (default 32) with equal shares of the 0.1 %, 1 %, 10 % and 50 % selectivity
bands; K = 1000; cosine score.  All data are synthetic and seeded.

A step = one lr_search call on one batch (filter compile, threshold sample, fused predicate + scoring
scan, selection, exact fallback check).  Prints one JSON line.
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

METRIC = "filtered top-K QPS @10M×128 vs plain FP32; HBM GB/s % of peak; p99 ms"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=("ours", "reference"), default="ours")
    p.add_argument("--batch", type=int, default=32)
    p.add_argument("--n", type=int, default=10_000_000)
    p.add_argument("--dim", type=int, default=128)
    p.add_argument("--k", type=int, default=1000)
    p.add_argument("--n-batches", type=int, default=4)
    p.add_argument("--plan", default="auto")
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--cpu-queries", type=int, default=0, help="oracle sample size (0: one query per host core)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    # workload shape (defaults: the plain method at scale); the precision form of the same study is
    # e.g. --n 50000000 --dim 64 --vocab 4096 --lam 20 --bands 0.01,0.1 --batch 1024 --dtype fp8
    p.add_argument("--dtype", choices=("f32", "bf16", "fp8"), default="f32")
    p.add_argument("--oversample", type=int, default=4)
    p.add_argument("--vocab", type=int, default=16384)
    p.add_argument("--lam", type=float, default=40.0)
    p.add_argument("--n-dense", type=int, default=256)
    p.add_argument("--bands", default="0.001,0.01,0.1,0.5")
    # other forms of the method (one JSON line each):
    #   --form loss   masked softmax loss fwd+bwd, B=4096 queries vs 4096 in-batch + 16384 sampled jobs, d=128
    #   --form serve  continuous batching over a resident 20M x 128 BF16 index, Poisson request streams
    #   --form sweep  selectivity sweep: each band alone at batch sizes --sweep-batches, per-point roofline
    #   --form topk   appendix "Fast Top K Selection": top 2,000 of 1,000,000 scores, bucket vs radix vs sort
    #   --form hardneg  in-batch hard-negative mining (top --n-neg per query) + the loss over the mined set
    #   --form peaks    device facts and library GEMM rates (cuBLAS via torch) for the roofline denominators
    p.add_argument("--form", choices=("search", "loss", "serve", "sweep", "topk", "sign", "hardneg", "peaks"),
                   default="search")
    p.add_argument("--n-neg", type=int, default=1024)
    p.add_argument("--topk-n", type=int, default=1_000_000)
    p.add_argument("--topk-k", type=int, default=2000)
    p.add_argument("--topk-rows", type=int, default=1)
    #   --form sign   sign-bit pre-selection (512-bit codes, quantK = quant-mult x K) vs the plain search
    p.add_argument("--quant-mult", type=int, default=200)
    p.add_argument("--sweep-batches", default="1,32,256,1024")
    p.add_argument("--loss-b", type=int, default=4096)
    p.add_argument("--loss-m", type=int, default=4096 + 16384)
    p.add_argument("--tau", type=float, default=0.05)
    p.add_argument("--rates", default="100,300,5000,10000,20000,50000")
    p.add_argument("--slots", type=int, default=3)
    p.add_argument("--chunks", type=int, default=0, help="serve form: >= 2 runs the rotating scan over that many "
                                                          "row chunks (one slot of 256 lanes)")
    p.add_argument("--max-requests", type=int, default=2000)
    p.add_argument("--clients", type=int, default=4, help="serve form: client threads submitting the stream")
    a = p.parse_args()
    a.band_list = tuple(float(x) for x in a.bands.split(","))
    return a


# ----------------------------------------------------------------------------- workload
def make_workload(args, rank=0):
    import datagen

    t0 = time.time()
    c = datagen.corpus(args.seed, args.n, args.dim, args.vocab, args.lam, 1.1)
    po, pid = c.postings()
    bands = args.band_list
    per = max(1, args.batch // len(bands))
    nb = args.n_batches
    band_f = [datagen.filters_in_band(args.seed + 1000 * rank, per * nb, c.V, 1.1, c.df, c.n, s,
                                      stream_offset=(i + 1) * 100_000_000) for i, s in enumerate(bands)]
    batches = []
    for j in range(nb):
        qs = []
        for i in range(len(bands)):
            sub = band_f[i].subset(range(j * per, (j + 1) * per))
            qs.extend(sub.clauses(b) for b in range(sub.n))
        qs = qs[: args.batch] + qs[: max(0, args.batch - len(qs))]
        batches.append(datagen.Filters.from_lists(qs))
    Q = datagen.query_embeddings(args.seed + 1000 * rank, args.batch * nb, args.dim)
    return dict(corpus=c, post_off=po, post_ids=pid, filters=batches, Q=Q.reshape(nb, args.batch, args.dim),
                gen_s=time.time() - t0)


def row_bytes(args):
    """Bytes the scan reads per job row: d_pad values of the stored type (+ the FP8 row scale)."""
    d_pad = 32 if args.dim <= 32 else 64 if args.dim <= 64 else 128 if args.dim <= 128 else 256
    return d_pad * {"f32": 4, "bf16": 2, "fp8": 1}[args.dtype] + (4 if args.dtype == "fp8" else 0)


def workload_config(args):
    form = {"f32": "FP32", "bf16": "BF16 rows + FP32 rescore", "fp8": "FP8 e4m3 rows + row scale + FP32 rescore"}
    gb = args.n * row_bytes(args) / 1e9
    cfg = {"workload": "filtered top-K, N=%d jobs x d=%d %s cosine, V=%d Poisson(%g) Zipf(1.1) terms as "
                       "posting lists + %d dense bitmaps, batch %d (bands %s), K=%d"
                       % (args.n, args.dim, form[args.dtype], args.vocab, args.lam, args.n_dense, args.batch,
                          "/".join("%g%%" % (100 * b) for b in args.band_list), args.k),
           "n_jobs": args.n, "dim": args.dim, "batch": args.batch, "k": args.k, "vocab": args.vocab,
           "selectivity_bands": list(args.band_list), "rows": args.dtype,
           "l2": "inputs larger than L2 (%.2f GB of scanned rows), no flush" % gb}
    if args.dtype != "f32":
        cfg["oversample"] = args.oversample
    return cfg


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """Samples the SM clock and the clock-event reasons every few milliseconds while the timed region
    runs (read-only NVML queries; falls back to nvidia-smi when NVML is unavailable)."""

    REASONS = (("hw_slowdown", "nvmlClocksEventReasonHwSlowdown"),
               ("hw_thermal_slowdown", "nvmlClocksEventReasonHwThermalSlowdown"),
               ("sw_thermal_slowdown", "nvmlClocksEventReasonSwThermalSlowdown"),
               ("sw_power_cap", "nvmlClocksEventReasonSwPowerCap"),
               ("hw_power_brake_slowdown", "nvmlClocksEventReasonHwPowerBrakeSlowdown"))

    def __init__(self, gpu: int, period_s: float = 0.002):
        self.gpu = gpu
        self.period = period_s
        self.samples = []  # (sm_mhz, max_mhz, reasons bitmask, host time)
        self.window = (0.0, float("inf"))
        self.load_end = None
        self.names = []
        self.stop = threading.Event()
        self.nv = None
        self.proc = None
        self.source = "none"
        self.errors = []

    def _nvml_handle(self, nv):
        """The NVML handle of this process's CUDA device: by UUID when CUDA_VISIBLE_DEVICES names one,
        by its index there otherwise (NVML numbers every GPU of the machine)."""
        vis = [x.strip() for x in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if x.strip()]
        if vis and self.gpu < len(vis):
            v = vis[self.gpu]
            if v.isdigit():
                return nv.nvmlDeviceGetHandleByIndex(int(v))
            return nv.nvmlDeviceGetHandleByUUID(v)
        return nv.nvmlDeviceGetHandleByIndex(self.gpu)

    def __enter__(self):
        try:
            import pynvml as nv

            nv.nvmlInit()
            self.h = self._nvml_handle(nv)
            self.mx = nv.nvmlDeviceGetMaxClockInfo(self.h, nv.NVML_CLOCK_SM)
            self._reasons = (nv.nvmlDeviceGetCurrentClocksEventReasons
                             if hasattr(nv, "nvmlDeviceGetCurrentClocksEventReasons")
                             else nv.nvmlDeviceGetCurrentClocksThrottleReasons)
            self._reasons(self.h)
            self.nv = nv
            self.names = [(nm, getattr(nv, attr)) for nm, attr in self.REASONS if hasattr(nv, attr)]
            self.source = "nvml"
            self.t = threading.Thread(target=self._poll_nvml, daemon=True)
        except Exception as e:  # no usable NVML: nvidia-smi's query loop instead
            self.errors.append("nvml: %s" % e)
            self.nv = None
            self.source = "nvidia-smi"
            self.t = threading.Thread(target=self._poll_smi, daemon=True)
        self.t.start()
        return self

    def _poll_nvml(self):
        nv, h = self.nv, self.h
        while not self.stop.is_set():
            try:
                self.samples.append((nv.nvmlDeviceGetClockInfo(h, nv.NVML_CLOCK_SM), self.mx, self._reasons(h),
                                     time.perf_counter()))
            except Exception as e:
                if len(self.errors) < 3:
                    self.errors.append("nvml sample: %s" % e)
            self.stop.wait(self.period)

    def _poll_smi(self):
        fields = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                  "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        self.names = [(nm, 1 << i) for i, (nm, _) in enumerate(self.REASONS[:4])]
        try:
            vis = [x.strip() for x in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if x.strip()]
            dev = vis[self.gpu] if vis and self.gpu < len(vis) else str(self.gpu)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", dev, "--query-gpu=" + fields,
                                          "--format=csv,noheader,nounits", "-lms", "10"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            return
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            try:
                bits = sum(1 << i for i, v in enumerate(parts[2:6]) if v.lower() in ("active", "1"))
                self.samples.append((float(parts[0]), float(parts[1]), bits, time.perf_counter()))
            except (ValueError, IndexError):
                continue

    def wait_first(self, timeout_s: float = 5.0):
        t0 = time.time()
        while not self.samples and time.time() - t0 < timeout_s:
            time.sleep(0.01)

    def __exit__(self, *exc):
        self.stop.set()
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        self.t.join(timeout=5)
        if self.nv is not None:
            try:
                self.nv.nvmlShutdown()
            except Exception:
                pass

    def mark(self, t0: float, t1: float, t_load_end: float = None):
        """The timed region ran between host times t0 and t1; when it is too short to hold a few samples,
        the window extends to t_load_end, the end of the same workload's synchronised steps that follow
        it (still under load), and the summary says so."""
        self.window = (t0, t1)
        self.load_end = t_load_end

    def summary(self):
        got = [x for x in self.samples if self.window[0] <= x[3] <= self.window[1]]
        window = "timed region"
        if len(got) < 3 and self.load_end is not None:
            got = [x for x in self.samples if self.window[0] <= x[3] <= self.load_end]
            window = "timed region + the same workload's synchronised latency steps that follow it"
        if not got:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0,
                    "source": self.source, "errors": self.errors[:3]}
        sm = [x[0] for x in got]
        reasons = sorted({nm for _, _, bits, _ in got for nm, b in self.names if bits & b})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(x[1] for x in got)),
                "sm_min_mhz": float(min(sm)), "reasons": reasons, "samples": len(sm), "source": self.source,
                "window": window}


# ----------------------------------------------------------------------------- helpers
def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            m = json.load(fh)
        return float(m["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6400.0, "fallback"


def scan_plan(args):
    """The scan kernel a search ran and the queries one launch of it serves (tensor-core tiles: 64 per
    launch at d <= 128 and 32 above; FP32 rows at d <= 128 in batches above 64: 128 (two 64-query
    blocks per launch), 96 above 128 queries (two 48-query blocks); BF16 / e4m3 rows above 64 queries: 256 (four
    64-query blocks in one N = 256 MMA); SIMT matrix-vector scan: 8 per launch).  The plan is the one the
    library reported for the timed steps (args.plan_used); before that, the requested plan, with "auto"
    read as the batch-size rule."""
    d_pad = 32 if args.dim <= 32 else 64 if args.dim <= 64 else 128 if args.dim <= 128 else 256
    plan = getattr(args, "plan_used", None) or (args.plan if args.plan != "auto" else
                                                 ("tc" if args.batch >= 16 else "gemv"))
    if plan == "tc" and args.dtype != "f32" and d_pad < 64:
        plan = "gemv"  # low-precision rows reach the tensor cores from 64 values up
    if plan == "tc":
        if args.dtype == "f32" and d_pad <= 128 and args.batch > 64:
            return "k_scan_tc", (96 if args.batch > 128 else 128), d_pad
        if args.dtype in ("bf16", "fp8") and d_pad <= 128 and args.batch > 64:
            return "k_scan_tc", 256, d_pad
        return "k_scan_tc", (64 if d_pad <= 128 else 32), d_pad
    return "k_scan_gemv", 8, d_pad


def measured_traffic(args):
    """DRAM bytes per main-scan launch from the committed ncu record, or None when the record does not
    cover the current kernel sources or this workload (10M x 128, batch 32, tensor-core plan, FP32)."""
    import hashlib

    kernel, _, _ = scan_plan(args)
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            rec = json.load(fh)[kernel]
        for path, want in rec["sources"].items():
            with open(os.path.join(ROOT, path), "rb") as fh:
                if hashlib.sha256(fh.read()).hexdigest() != want:
                    return None
    except (OSError, KeyError, ValueError):
        return None
    if (args.n, args.dim, args.batch, args.dtype) != (10_000_000, 128, 32, "f32"):
        return None
    return float(rec["traffic_per_launch_10M"])


def algorithmic_scan_bytes(lr, idx, filters, corpus, args):
    """Bytes the main scan must move per launch.  GEMV scan (predicate inside): rows that pass some
    query of the launch (each read once at d_pad*elem bytes) plus, per distinct term, the cheaper of
    its bitmap and its posting list.  Tensor-core scan (the tile filter has run before, alongside the
    threshold sample): the same rows plus the row masks of the listed tiles (128 rows x 4 bytes, 8 above
    32 queries, per 128-row tile holding a passing row); a two-block launch (96 or 128 queries) reads two
    8-byte masks per row of every tile."""
    import torch

    kernel, per, d_pad = scan_plan(args)
    rb = row_bytes(args)
    n = corpus.n
    df = corpus.df
    per_launch = []
    B = filters.n
    for q0 in range(0, B, per):
        sub = filters.subset(range(q0, min(B, q0 + per)))
        _, bm = lr.lr_filter_count(idx, sub, bitmap=True)
        union = bm[0].clone()
        for i in range(1, sub.n):
            union |= bm[i]
        words = union.view(torch.int32).cpu().numpy().view(np.uint32)
        rows = int(np.unpackbits(words.view(np.uint8)).sum())
        terms = {int(t) for t in sub.terms} if sub.terms.size and int(sub.q_off[-1]) > 0 else set()
        p = sum(min(n / 8.0, 4.0 * float(df[t])) for t in terms)
        masks = 0
        block = {96: 48, 128: 64, 256: 64}.get(per) if kernel == "k_scan_tc" else None
        if block is not None and sub.n > block:  # several blocks: every tile, one 8-byte mask per row and block
            masks = (n + 127) // 128 * 128 * 8 * -(-sub.n // block)
        elif kernel == "k_scan_tc":
            tiles = int(np.count_nonzero(words[: len(words) // 4 * 4].reshape(-1, 4).any(axis=1)))
            if len(words) % 4:
                tiles += int(words[len(words) // 4 * 4:].any())
            masks = tiles * 128 * (4 if sub.n <= 32 else 8)
        per_launch.append({"E": rows * rb, "P": p, "masks": masks})
    return per_launch


def cpu_oracle_sample(wl, args, n_queries, batch_index=0):
    """Time the CPU oracle on the first n_queries of one batch over the full index."""
    import oracle

    f = wl["filters"][batch_index]
    sel = list(range(min(n_queries, f.n)))
    fs = f.subset(sel)
    Q = wl["Q"][batch_index][sel]
    c = wl["corpus"]
    t0 = time.perf_counter()
    ref = oracle.search(c.X, c.job_off, c.job_terms, Q, fs, args.k, metric="cosine")
    dt = time.perf_counter() - t0
    cores = min(oracle.num_threads(), len(sel))
    return ref, sel, dt, cores


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The maximum of a per-rank measurement over all ranks (the slowest rank sets the job's time)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world: int, seconds: float) -> float:
    """Units all ranks processed per second of the slowest rank's time (weak scaling: fixed work per rank)."""
    return world * units_per_rank / seconds


# ----------------------------------------------------------------------------- arms
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = make_workload(args)
    # the oracle runs OpenMP over queries: one query per host core uses them all
    per_step = max(os.cpu_count() or 1, 1)
    times = []
    nq = 0
    for i in range(args.warmup + args.steps):
        j = i % len(wl["filters"])
        _, sel, dt, cores = cpu_oracle_sample(wl, args, per_step, j)
        if i >= args.warmup:
            times.append(dt)
            nq += len(sel)
    total = sum(times)
    value = nq / total
    out = {"metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded generator)",
           "impl": "reference", "config": workload_config(args),
           "cpu_baseline": {"value": value, "unit": "queries/s", "cores": cores, "kind": "oracle",
                            "sample": "%d queries per step (first of each batch) over the full %d-job index"
                                      % (per_step, args.n)},
           "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_e2e(lr, idx, wl, args, world):
    """The same metric end to end through lr_search with pinned host query and output buffers: every
    step copies its queries and filters to the device and its rows back inside the timed region (the
    copies ordered on the search stream, LR_SEARCH_ASYNC_HOST, one synchronisation at the end)."""
    import torch
    import torch.distributed as dist

    nb = len(wl["filters"])
    B, K = args.batch, args.k
    hq = [torch.from_numpy(np.ascontiguousarray(wl["Q"][j])).pin_memory() for j in range(nb)]
    h_ids = torch.empty((B, K), dtype=torch.int32).pin_memory()
    h_sc = torch.empty((B, K), dtype=torch.float32).pin_memory()
    h_cnt = torch.empty(B, dtype=torch.int32).pin_memory()
    for i in range(max(args.warmup, 10)):
        lr.lr_search(idx, hq[i % nb], wl["filters"][i % nb], K, out_ids=h_ids, out_scores=h_sc, out_count=h_cnt,
                     host_sync=False)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for i in range(args.steps):  # stream-ordered copies into the page-locked outputs, one synchronisation
        j = i % nb
        lr.lr_search(idx, hq[j], wl["filters"][j], K, out_ids=h_ids, out_scores=h_sc, out_count=h_cnt,
                     host_sync=False)
    torch.cuda.synchronize()
    dt = max_over_ranks(time.perf_counter() - t0, world)
    f0 = wl["filters"][0]
    h2d = B * args.dim * 4 + f0.q_off.nbytes + f0.c_off.nbytes + f0.terms.nbytes
    d2h = B * K * 8 + B * 4
    return {"value": whole_job_rate(B * args.steps, world, dt), "unit": "queries/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h)}


def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import paper_2402_13435_b300 as lr

    wl = make_workload(args, rank)
    c = wl["corpus"]
    t0 = time.time()
    idx = lr.lr_index_create(torch.from_numpy(c.X).cuda(), c.V, post_off=wl["post_off"], post_ids=wl["post_ids"],
                             n_dense_terms=args.n_dense, metric="cosine", max_batch=max(args.batch, 32),
                             max_k=args.k, dtype=args.dtype, oversample=args.oversample,
                             max_sparse_terms=max(256, 4 * args.batch))
    torch.cuda.synchronize()
    build_s = time.time() - t0
    nb = len(wl["filters"])
    Qd = [torch.from_numpy(np.ascontiguousarray(wl["Q"][j])).cuda() for j in range(nb)]
    B, K = args.batch, args.k
    out_ids = torch.empty((B, K), dtype=torch.int32, device="cuda")
    out_sc = torch.empty((B, K), dtype=torch.float32, device="cuda")
    out_cnt = torch.empty(B, dtype=torch.int32, device="cuda")

    def step(i, probe=None):
        j = i % nb
        lr.lr_search(idx, Qd[j], wl["filters"][j], K, out_ids=out_ids, out_scores=out_sc, out_count=out_cnt,
                     plan=args.plan, probe=probe)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    lr.lr_index_sync(idx)
    # ---- timed region (device time)
    probes = [lr.Probe(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
    for p in probes:  # materialise the event handles
        p.start.record()
        p.stop.record()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        clk.wait_first()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        h0 = time.perf_counter()
        ev0.record()
        for i in range(args.steps):
            step(i, probes[i])
        ev1.record()
        torch.cuda.synchronize()
        h1 = time.perf_counter()
        if world > 1:
            dist.barrier()
        # ---- per-step latency distribution (separate, synchronised steps of the same workload)
        lat = []
        for i in range(min(args.steps, 20)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            step(i)
            e1.record()
            torch.cuda.synchronize()
            lat.append(e0.elapsed_time(e1))
        clk.mark(h0, h1, time.perf_counter())
    # end to end after the clock sampler has stopped (its polling thread and
    # nvidia-smi child compete with the host side of the search loop)
    e2e = None if args.no_e2e else run_e2e(lr, idx, wl, args, world)
    step_ms = lat
    ms = ev0.elapsed_time(ev1)
    args.plan_used = probes[0].plan if probes[0].plan in ("gemv", "tc") else None
    lr.lr_index_sync(idx)
    ms = max_over_ranks(ms, world)
    scan_ms = float(np.mean([p.start.elapsed_time(p.stop) for p in probes]))
    n_scan = probes[0].n_scan_launches
    launches = int(sum(p.n_launches for p in probes))
    value = whole_job_rate(B * args.steps, world, ms / 1e3)

    # ---- roofline of the dominant kernel (the main scan)
    parts = algorithmic_scan_bytes(lr, idx, wl["filters"][0], c, args)
    peak, peak_kind = peaks()
    # scan_ms covers n_scan launches of batch i % nb; batch 0's bytes stand for the per-launch average.
    # E: rows some query of the launch must score x row bytes (the algorithmic bytes of the scan);
    # masks: the tile filter's row masks the tensor-core scan reads; P: the batch's term words
    E = sum(x["E"] for x in parts)
    masks = sum(x["masks"] for x in parts)
    P = sum(x["P"] for x in parts)
    achieved = (E / 1e9) / (scan_ms / 1e3)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": measured_traffic(args),
            "kernel": "%s (main scan, %d launches per step)" % (scan_plan(args)[0], n_scan),
            "algorithmic_bytes_per_launch": E / len(parts), "launch_ms": scan_ms / max(n_scan, 1),
            "frac_with_row_masks": ((E + masks) / 1e9) / (scan_ms / 1e3) / peak,
            "frac_e_plus_p_over_step": ((E + P) / 1e9) / (ms / args.steps / 1e3) / peak,
            "bytes_note": "achieved = E (rows passing some query of the launch x row bytes) / main-scan time; "
                          "frac_with_row_masks adds the tile list's row masks the scan reads; "
                          "frac_e_plus_p_over_step = (E + term bytes P) / whole step time",
            "peak_kind": peak_kind}


    # ---- CPU oracle baseline and parity of the sampled queries
    cpu = None
    parity = None
    if rank == 0 and not args.no_cpu_baseline:
        from oracle.compare import check_topk

        ref, sel, dt, cores = cpu_oracle_sample(wl, args, args.cpu_queries or (os.cpu_count() or 8), 0)
        step(0)
        torch.cuda.synchronize()
        ids, sc, cnt = out_ids.cpu().numpy(), out_sc.cpu().numpy(), out_cnt.cpu().numpy()
        import oracle

        rec = oracle.recall_at_k([ids[b, :cnt[b]] for b in sel], [ref.ids[i, :ref.count[i]] for i in range(len(sel))])
        err = 0.0
        for i, b in enumerate(sel):
            m = min(int(cnt[b]), int(ref.count[i]))
            if m:
                err = max(err, float(np.max(np.abs(sc[b, :m].astype(np.float64) - ref.scores[i, :m]))))
        try:
            moved = check_topk(ids, sc, cnt, ref, c.X, wl["Q"][0], c.job_off, c.job_terms, wl["filters"][0],
                               queries=sel)
            parity = {"queries": len(sel), "ok": True, "id_positions_in_tie_band": moved}
        except AssertionError as e:
            parity = {"queries": len(sel), "ok": False, "error": str(e)[:300]}
        parity.update({"recall_at_k": rec, "max_abs_score_err_vs_fp64": err})
        cpu = {"value": len(sel) / dt, "unit": "queries/s", "cores": cores, "kind": "oracle",
               "sample": "first %d queries of batch 0 over the full %d-job index (%.1f s)" % (len(sel), args.n, dt)}

    if rank == 0:
        p50, p99 = (float(np.percentile(step_ms, 50)), float(np.percentile(step_ms, 99))) if step_ms else (None, None)
        out = {"metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": args.dtype, "data": "synthetic (seeded generator, paper-shaped)",
               "config": workload_config(args), "p50_ms": p50, "p99_ms": p99, "clocks": clk.summary(),
               "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "parity": parity,
               "setup_s": {"generate": round(wl["gen_s"], 1), "index_build": round(build_s, 1)}}
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_loss(args):
    """Masked softmax loss (forward + backward) at the two-tower training-step shape."""
    import torch
    import datagen
    import paper_2402_13435_b300 as lr

    B, M, d = args.loss_b, args.loss_m, args.dim
    inv_tau = 1.0 / args.tau
    c = datagen.corpus(args.seed, M, d, 4096, 20.0, 1.1)  # jobs: in-batch positives first, then sampled
    Q = torch.from_numpy(datagen.query_embeddings(args.seed + 1, B, d)).to(torch.bfloat16).cuda()
    J = torch.from_numpy(c.X).to(torch.bfloat16).cuda()
    pos = torch.arange(B, dtype=torch.int32, device="cuda")
    f = datagen.filters(args.seed + 2, B, c.V, 1.1)
    idx = lr.lr_index_create(c.X, c.V, bitsets=c.bitsets(), metric="dot", max_batch=B, max_k=16,
                             max_batch_terms=16 * B)
    npass, mask = lr.lr_filter_count(idx, f, bitmap=True)  # the term constraint as the loss mask
    torch.cuda.synchronize()
    ws = lr.loss_workspace(B, M, d)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    fwd, bwd = [], []
    for i in range(args.warmup + args.steps):
        ev[0].record()
        loss, lse = lr.lr_score_forward(Q, J, pos, mask, inv_tau, ws)
        ev[1].record()
        dQ, dJ = lr.lr_score_backward(Q, J, pos, mask, inv_tau, lse, None, ws)
        ev[2].record()
        torch.cuda.synchronize()
        if i >= args.warmup:
            fwd.append(ev[0].elapsed_time(ev[1]))
            bwd.append(ev[1].elapsed_time(ev[2]))
    lr.lr_score_status(ws, B, M, d)
    fm, bm = float(np.median(fwd)), float(np.median(bwd))
    # steady state, as a training loop runs: the K steps back to back (the host
    # queues step i + 1 while step i runs), one pair of events around them
    ev[0].record()
    for i in range(args.steps):
        loss, lse = lr.lr_score_forward(Q, J, pos, mask, inv_tau, ws)
        dQ, dJ = lr.lr_score_backward(Q, J, pos, mask, inv_tau, lse, None, ws)
    ev[1].record()
    torch.cuda.synchronize()
    lr.lr_score_status(ws, B, M, d)
    steady = ev[0].elapsed_time(ev[1]) / args.steps
    flops = 4 * 2.0 * B * M * d  # forward logits, recomputed logits, dZ.J and dZ^T.Q: 86 GF at this shape
    tf = flops / (steady / 1e3) / 1e12
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        peak, kind = float(pk["bf16_tflops"]), "measured (bf16 burst)"
    except (OSError, KeyError, ValueError):
        peak, kind = 1800.0, "fallback"
    parity = None
    if not args.no_cpu_baseline:
        import oracle

        allowed = np.unpackbits(mask.cpu().numpy().view(np.uint8), axis=1, bitorder="little")[:, :M].astype(bool)
        t0 = time.perf_counter()
        ref = oracle.softmax_loss(Q.double().cpu().numpy(), J.double().cpu().numpy(), np.arange(B), allowed, inv_tau)
        cpu_s = time.perf_counter() - t0
        g = lambda a, r: float(np.max(np.abs(a.cpu().numpy() - r)) / max(np.max(np.abs(r)), 1e-30))
        parity = {"loss_rel_err": abs(float(loss.item()) - ref[0]) / abs(ref[0]), "dQ_rel_err": g(dQ, ref[2]),
                  "dJ_rel_err": g(dJ, ref[3]), "oracle": "FP64 torch autograd on the BF16 inputs",
                  "oracle_s": round(cpu_s, 2)}
    out = {"metric": "masked softmax loss fwd+bwd ms @B=%d M=%d d=%d BF16" % (B, M, d), "value": steady,
           "unit": "ms", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
           "dtype": "bf16", "data": "synthetic (seeded generator)",
           "timing": "value: K steps back to back between two events (steady state); fwd_ms / bwd_ms: medians "
                     "of single steps, each between events on an idle GPU (they include the host's launch time)",
           "fwd_ms": fm, "bwd_ms": bm, "synced_step_ms": fm + bm,
           "config": {"workload": "two-tower step: %d queries vs %d in-batch positives + %d sampled jobs, tau=%g, "
                                  "term mask from the cfg-1 filter generator (%.1f%% allowed)"
                                  % (B, B, M - B, args.tau, 100.0 * float(npass.sum()) / (B * M)),
                      "B": B, "M": M, "d": d},
           "roofline": {"bound": "tensor", "achieved": tf, "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
                        "traffic": None, "flops_per_step": flops, "peak_kind": kind},
           "parity": parity}
    print(json.dumps(out), flush=True)


def run_serve(args):
    """Poisson request streams against the continuous-batching server over a resident BF16 index."""
    import torch
    import datagen
    import paper_2402_13435_b300 as lr

    rng = np.random.default_rng(args.seed)
    t0 = time.time()
    c = datagen.corpus(args.seed, args.n, args.dim, args.vocab, args.lam, 1.1)
    bands = np.geomspace(0.0005, 0.5, 8)  # selectivity log-uniform over 0.05 % .. 50 %
    pool = []
    for i, sb in enumerate(bands):
        fb = datagen.filters_in_band(args.seed + 7, 96, c.V, 1.1, c.df, c.n, float(sb),
                                     stream_offset=(i + 1) * 100_000_000)
        pool += [fb.clauses(j) for j in range(fb.n)]
    Qpool = datagen.query_embeddings(args.seed + 3, 4096, args.dim)
    gen_s = time.time() - t0
    po, pid = c.postings()
    idx = lr.lr_index_create(torch.from_numpy(c.X).cuda(), c.V, post_off=po, post_ids=pid, n_dense_terms=-1,
                             metric="cosine", max_batch=256, max_k=2000, dtype=args.dtype,
                             oversample=args.oversample)
    torch.cuda.synchronize()
    nreq = args.max_requests
    reqs = []
    for i in range(nreq):
        Bq = int(rng.integers(1, 65))
        K = int(rng.choice([100, 500, 1000, 2000]))
        rows = rng.integers(0, len(Qpool), size=Bq)
        fl = [pool[int(j)] for j in rng.integers(0, len(pool), size=Bq)]
        reqs.append((Qpool[rows], datagen.Filters.from_lists(fl), K))
    loads = []
    with lr.Server(idx, slots=args.slots, max_queries=256, plan=args.plan, chunks=args.chunks) as srv:
        srv.wait(srv.submit(*reqs[0]), reqs[0][0].shape[0], reqs[0][2])  # warm up
        for rate in [float(r) for r in args.rates.split(",")]:
            srv.stats(reset=True)
            # arrival times of one Poisson stream, submitted by several client threads (each takes every
            # n-th request at its due time; the library call releases the interpreter lock), so a single
            # Python thread's submit cost does not cap the offered rate
            arrivals = np.cumsum(rng.exponential(1.0 / rate, size=nreq))
            tickets = [None] * nreq
            n_cli = args.clients
            t_start = time.perf_counter()
            sub_end = [t_start] * n_cli

            def client(c):
                for i in range(c, nreq, n_cli):
                    due = t_start + arrivals[i]
                    while True:
                        now = time.perf_counter()
                        if now >= due:
                            break
                        time.sleep(min(due - now, 0.001))
                    Q, f, K = reqs[i]
                    tickets[i] = srv.submit(Q, f, K)
                sub_end[c] = time.perf_counter()

            threads = [threading.Thread(target=client, args=(c,)) for c in range(n_cli)]
            for th in threads:
                th.start()
            for th in threads:
                th.join()
            t_sub = max(sub_end) - t_start
            for t, (Q, f, K) in zip(tickets, reqs):
                srv.wait(t, Q.shape[0], K)
            t_all = time.perf_counter() - t_start
            st = srv.stats()
            loads.append({"offered_rps": rate, "submitted_rps": nreq / t_sub, "achieved_rps": nreq / t_all,
                          "achieved_qps": st["queries"] / t_all, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
                          "mean_batch_queries": st["queries"] / max(st["batches"], 1), "batches": st["batches"]})
            if args.chunks >= 2:  # batches are scan steps: queries per step = active lanes
                loads[-1]["mean_batch_queries"] = st["queries"] * args.chunks / max(st["batches"], 1)
        slots = srv.stats()["slots"]
    best = max(l["achieved_qps"] for l in loads)
    out = {"metric": "serving QPS with p50/p99 latency per offered request rate", "value": best,
           "unit": "queries/s", "n_gpus": 1, "higher_is_better": True, "dtype": args.dtype,
           "data": "synthetic (seeded generator)",
           "config": {"workload": "resident N=%d x d=%d %s index (oversample %d), Poisson requests of 1-64 queries, "
                                  "K in {100,500,1000,2000}, selectivity log-uniform 0.05-50%%; %d requests per load "
                                  "point from %d client threads, %s"
                                  % (args.n, args.dim, args.dtype, args.oversample, nreq, args.clients,
                                     "%d slots of 256 queries" % slots if args.chunks < 2 else
                                     "rotating scan over %d row chunks, 256 lanes" % args.chunks),
                      "n_jobs": args.n, "dim": args.dim, "slots": slots, "chunks": max(args.chunks, 1)},
           "loads": loads, "setup_s": {"generate": round(gen_s, 1)}}
    print(json.dumps(out), flush=True)


def run_sweep(args):
    """Each selectivity band alone at each batch size (the scale configuration's sweep): per point the
    achieved pass rates (exact, from the library's filter export), QPS, the main-scan time and two
    roofline fractions -- per batch (rows some query of the batch passes, read once, plus term bytes P
    and outputs O, over the step time) and per launch (each launch's union rows over its scan time)."""
    import torch
    import datagen
    import paper_2402_13435_b300 as lr

    t0 = time.time()
    c = datagen.corpus(args.seed, args.n, args.dim, args.vocab, args.lam, 1.1)
    po, pid = c.postings()
    batches = [int(x) for x in args.sweep_batches.split(",")]
    Bmax = max(batches)
    idx = lr.lr_index_create(torch.from_numpy(c.X).cuda(), c.V, post_off=po, post_ids=pid,
                             n_dense_terms=args.n_dense, metric="cosine", max_batch=max(Bmax, 32), max_k=args.k,
                             dtype=args.dtype, oversample=args.oversample, max_sparse_terms=max(256, 4 * Bmax))
    torch.cuda.synchronize()
    peak, peak_kind = peaks()
    rb = row_bytes(args)
    points = []
    for bi, band in enumerate(args.band_list):
        fb = datagen.filters_in_band(args.seed + 5, Bmax, c.V, 1.1, c.df, c.n, band,
                                     stream_offset=(bi + 1) * 100_000_000)
        Qall = datagen.query_embeddings(args.seed + 6 + bi, Bmax, args.dim)
        for B in batches:
            f = fb.subset(range(B))
            Qd = torch.from_numpy(np.ascontiguousarray(Qall[:B])).cuda()
            oi = torch.empty((B, args.k), dtype=torch.int32, device="cuda")
            osc = torch.empty((B, args.k), dtype=torch.float32, device="cuda")
            oc = torch.empty(B, dtype=torch.int32, device="cuda")
            steps = max(3, min(args.steps, 10 if B >= 256 else 30))
            probes = [lr.Probe(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                      for _ in range(steps)]
            for p in probes:  # materialise the event handles the library records
                p.start.record()
                p.stop.record()
            for _ in range(3):
                lr.lr_search(idx, Qd, f, args.k, out_ids=oi, out_scores=osc, out_count=oc, plan=args.plan)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for i in range(steps):
                lr.lr_search(idx, Qd, f, args.k, out_ids=oi, out_scores=osc, out_count=oc, plan=args.plan,
                             probe=probes[i])
            e1.record()
            torch.cuda.synchronize()
            lr.lr_index_sync(idx)
            ms = e0.elapsed_time(e1) / steps
            scan_ms = float(np.mean([p.start.elapsed_time(p.stop) for p in probes]))
            plan = probes[0].plan
            npass, bm = lr.lr_filter_count(idx, f, bitmap=True)
            rates = npass.cpu().numpy() / c.n
            words = bm.view(torch.int32)
            union = words[0].clone()
            for i in range(1, B):
                union |= words[i]
            urows = int(np.unpackbits(union.cpu().numpy().view(np.uint8)).sum())
            terms = {int(t) for t in f.terms} if int(f.q_off[-1]) > 0 else set()
            P = sum(min(c.n / 8.0, 4.0 * float(c.df[t])) for t in terms)
            O = B * args.k * 8
            per = 64 if plan == "tc" else 8
            e_launch = 0
            for q0 in range(0, B, per):
                u = words[q0].clone()
                for i in range(q0 + 1, min(B, q0 + per)):
                    u |= words[i]
                e_launch += int(np.unpackbits(u.cpu().numpy().view(np.uint8)).sum()) * rb
            points.append({"band": band, "batch": B, "plan": plan, "qps": B / (ms / 1e3), "ms_per_step": ms,
                           "scan_ms_per_step": scan_ms, "scan_launches": probes[0].n_scan_launches,
                           "pass_rate_mean": float(rates.mean()), "pass_rate_min": float(rates.min()),
                           "pass_rate_max": float(rates.max()), "union_rows": urows,
                           "frac_per_batch": ((urows * rb + P + O) / 1e9) / (ms / 1e3) / peak,
                           "frac_per_launch_scan": (e_launch / 1e9) / (scan_ms / 1e3) / peak})
    out = {"metric": "selectivity sweep: QPS and roofline per band and batch", "unit": "queries/s",
           "n_gpus": 1, "dtype": args.dtype, "data": "synthetic (seeded generator, paper-shaped)",
           "config": workload_config(args), "peak": peak, "peak_kind": peak_kind, "points": points,
           "setup_s": round(time.time() - t0, 1)}
    print(json.dumps(out), flush=True)


def run_topk(args):
    """The appendix's selection experiment (top 2,000 of 1,000,000 scores): the bucket selection and the
    radix selection of the library against a full sort (the appendix's "naive" method; torch.sort) and
    torch.topk, as libraries for context.  64 distinct score sets of rows x n cosine-like scores are
    cycled (more bytes than L2 holds), each call timed with CUDA events on the current stream."""
    import torch
    import paper_2402_13435_b300 as lr

    n, k, R = args.topk_n, args.topk_k, args.topk_rows
    sets = 64
    g = torch.Generator(device="cuda").manual_seed(args.seed)
    S = torch.rand((sets, R, n), generator=g, device="cuda") * 2 - 1
    ws = lr.topk_workspace(R, n)
    oi = torch.empty((R, k), dtype=torch.int32, device="cuda")
    osc = torch.empty((R, k), dtype=torch.float32, device="cuda")

    def t_bucket(x):
        lr.lr_topk(x, k, method="bucket", workspace=ws, out_ids=oi, out_scores=osc)

    def t_radix(x):
        lr.lr_topk(x, k, method="radix", workspace=ws, out_ids=oi, out_scores=osc)

    def t_sort(x):
        torch.sort(x, dim=1, descending=True, stable=True)

    def t_topk(x):
        torch.topk(x, k, dim=1)

    res = {}
    for name, fn in (("bucket", t_bucket), ("radix", t_radix), ("torch_sort", t_sort), ("torch_topk", t_topk)):
        for i in range(args.warmup):
            fn(S[i % sets])
        torch.cuda.synchronize()
        times = []
        for i in range(max(args.steps, 20)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn(S[i % sets])
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        res[name] = {"median_ms": float(np.median(times)), "p10_ms": float(np.percentile(times, 10)),
                     "p90_ms": float(np.percentile(times, 90))}
    # CPU baseline leg: the oracle's full sort of one score set, timed, and parity of both methods on it
    ok, cpu = None, None
    if not args.no_cpu_baseline:
        import oracle

        x = S[0]
        xh = x.cpu().numpy()
        t0 = time.perf_counter()
        ref_ids, ref_sc = oracle.topk_scores(xh, k)
        dt = time.perf_counter() - t0
        cpu = {"value": dt * 1e3, "unit": "ms", "cores": 1, "kind": "oracle",
               "sample": "one score set (%d x %d): numpy lexsort per row" % (R, n)}
        ok = {}
        for m in ("bucket", "radix"):
            ids, sc = lr.lr_topk(x, k, method=m)
            ok[m] = bool(np.array_equal(ids.cpu().numpy(), ref_ids) and
                         np.array_equal(sc.cpu().numpy().astype(np.float64), ref_sc))
    peak, kind = peaks()
    bytes_read = R * n * 4
    out = {"metric": "top-%d of %d scores per row: ms per call" % (k, n), "value": res["bucket"]["median_ms"],
           "unit": "ms", "higher_is_better": False, "n_gpus": 1, "dtype": "f32", "data": "synthetic uniform[-1,1]",
           "config": {"workload": "%d row(s) x %d FP32 scores, k=%d, bucket granularity 100 on [-1,1]" % (R, n, k),
                      "l2": "64 distinct score sets cycled (%.0f MB)" % (sets * bytes_read / 1e6)},
           "methods": res, "parity_vs_oracle_sort": ok, "cpu_baseline": cpu,
           "roofline": {"bound": "latency", "algorithmic_bytes": bytes_read, "peak": peak, "unit": "GB/s",
                        "achieved": bytes_read / 1e9 / (res["bucket"]["median_ms"] / 1e3),
                        "frac": bytes_read / 1e9 / (res["bucket"]["median_ms"] / 1e3) / peak, "peak_kind": kind},
           "paper": {"naive_sort_ms": 1.91, "bucket_ms": 0.38, "note": "the paper's own GPU, context only"}}
    print(json.dumps(out), flush=True)


def run_sign(args):
    """Sign-bit pre-selection (appendix "Quantization"): 512-bit codes of the rows (bins of 8 permuted,
    randomly signed coordinates), Eq. 4 agreement levels, about quant_mult x K jobs kept per query and
    scored exactly -- against the plain exact search of the same batches on the same index.  Reports
    QPS of both, the main-pass time (filter export + two code scans), the kept counts, and recall@K of
    the pre-selection against the plain oracle on a sample of queries (CPU baseline leg)."""
    import torch
    import datagen
    import paper_2402_13435_b300 as lr

    wl = make_workload(args)
    c = wl["corpus"]
    idx_p, sgn_p = datagen.sign_projection(args.seed + 9, args.dim, 512, 8)
    t0 = time.time()
    idx = lr.lr_index_create(torch.from_numpy(c.X).cuda(), c.V, post_off=wl["post_off"], post_ids=wl["post_ids"],
                             n_dense_terms=args.n_dense, metric="cosine", max_batch=max(args.batch, 32),
                             max_k=args.k, max_sparse_terms=max(256, 4 * args.batch),
                             sign_projection=(idx_p, sgn_p, 8), max_quant_k=args.quant_mult * args.k)
    torch.cuda.synchronize()
    build_s = time.time() - t0
    nb = len(wl["filters"])
    Qd = [torch.from_numpy(np.ascontiguousarray(wl["Q"][j])).cuda() for j in range(nb)]
    B, K = args.batch, args.k
    oi = torch.empty((B, K), dtype=torch.int32, device="cuda")
    osc = torch.empty((B, K), dtype=torch.float32, device="cuda")
    oc = torch.empty(B, dtype=torch.int32, device="cuda")
    res = {}
    for name, qm in (("sign", args.quant_mult), ("plain", 0)):
        probes = [lr.Probe(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]
        for p in probes:
            p.start.record()
            p.stop.record()
        for i in range(args.warmup):
            lr.lr_search(idx, Qd[i % nb], wl["filters"][i % nb], K, out_ids=oi, out_scores=osc, out_count=oc,
                         quant_mult=qm)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in range(args.steps):
            lr.lr_search(idx, Qd[i % nb], wl["filters"][i % nb], K, out_ids=oi, out_scores=osc, out_count=oc,
                         quant_mult=qm, probe=probes[i])
        e1.record()
        torch.cuda.synchronize()
        lr.lr_index_sync(idx)
        ms = e0.elapsed_time(e1) / args.steps
        res[name] = {"qps": B / (ms / 1e3), "ms_per_step": ms,
                     "main_pass_ms": float(np.mean([p.start.elapsed_time(p.stop) for p in probes])),
                     "launches_per_step": probes[0].n_launches}
    _, _, _, st = lr.lr_search(idx, Qd[0], wl["filters"][0], K, quant_mult=args.quant_mult, stats=True)
    cand = st["cand_count"]
    # code scans: the codes (64 B per row) twice plus the pass bitmaps; kept rows: 512 B each
    code_bytes = 2 * c.n * 64 + 2 * B * c.n / 8
    peak, kind = peaks()
    out = {"metric": "sign-bit pre-selection QPS vs plain exact search", "value": res["sign"]["qps"],
           "unit": "queries/s", "higher_is_better": True, "n_gpus": 1, "dtype": "u64 codes + f32 rescore",
           "data": "synthetic (seeded generator, paper-shaped)", "config": workload_config(args),
           "quant_mult": args.quant_mult, "sign_bits": 512, "sign_bin": 8, "forms": res,
           "kept_per_query": {"mean": float(cand.mean()), "min": int(cand.min()), "max": int(cand.max())},
           "roofline": {"bound": "hbm", "kernel": "k_sign_scan (histogram + collect passes)",
                        "algorithmic_bytes_per_step": code_bytes, "peak": peak, "unit": "GB/s",
                        "achieved": code_bytes / 1e9 / (res["sign"]["main_pass_ms"] / 1e3),
                        "frac": code_bytes / 1e9 / (res["sign"]["main_pass_ms"] / 1e3) / peak, "peak_kind": kind},
           "setup_s": {"index_build": round(build_s, 1)}}
    if not args.no_cpu_baseline:
        import oracle

        sel = list(range(min(args.cpu_queries or 8, B)))
        fs = wl["filters"][0].subset(sel)
        Q0 = wl["Q"][0][sel]
        t1 = time.perf_counter()
        ref = oracle.search(c.X, c.job_off, c.job_terms, Q0, fs, K, metric="cosine")
        dt = time.perf_counter() - t1
        ids = lr.lr_search(idx, Qd[0], wl["filters"][0], K, quant_mult=args.quant_mult)[0].cpu().numpy()
        out["recall_at_k_vs_exact"] = oracle.recall_at_k([ids[b] for b in sel],
                                                         [ref.ids[i, :ref.count[i]] for i in range(len(sel))])
        out["cpu_baseline"] = {"value": len(sel) / dt, "unit": "queries/s", "cores": min(oracle.num_threads(),
                               len(sel)), "kind": "oracle", "sample": "first %d queries of batch 0" % len(sel)}
    print(json.dumps(out), flush=True)


def run_hardneg(args):
    """Second-stage training step of Sec. 5.2: mine each query's top n_neg negatives among the in-batch
    positives and sampled jobs (allowed by the term mask), then the loss forward and backward over the
    positive and the mined negatives only.  Times mining and loss separately (CUDA events)."""
    import torch
    import datagen
    import paper_2402_13435_b300 as lr

    B, M, d = args.loss_b, args.loss_m, args.dim
    inv_tau = 1.0 / args.tau
    c = datagen.corpus(args.seed, M, d, 4096, 20.0, 1.1)
    Q = torch.from_numpy(datagen.query_embeddings(args.seed + 1, B, d)).to(torch.bfloat16).cuda()
    J = torch.from_numpy(c.X).to(torch.bfloat16).cuda()
    pos = torch.arange(B, dtype=torch.int32, device="cuda")
    f = datagen.filters(args.seed + 2, B, c.V, 1.1)
    idx = lr.lr_index_create(c.X, c.V, bitsets=c.bitsets(), metric="dot", max_batch=B, max_k=16,
                             max_batch_terms=16 * B)
    npass, mask = lr.lr_filter_count(idx, f, bitmap=True)
    torch.cuda.synchronize()
    ws = torch.empty(int(lr._lib.lr_hard_negatives_workspace_size(B, M, d)), dtype=torch.uint8, device="cuda")
    lws = lr.loss_workspace(B, M, d)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    mine, fwd, bwd = [], [], []
    for i in range(args.warmup + args.steps):
        ev[0].record()
        ids, sc, cnt, mined = lr.lr_hard_negatives(Q, J, pos, args.n_neg, mask_bits=mask, workspace=ws)
        ev[1].record()
        loss, lse = lr.lr_score_forward(Q, J, pos, mined, inv_tau, lws)
        ev[2].record()
        dQ, dJ = lr.lr_score_backward(Q, J, pos, mined, inv_tau, lse, None, lws)
        ev[3].record()
        torch.cuda.synchronize()
        if i >= args.warmup:
            mine.append(ev[0].elapsed_time(ev[1]))
            fwd.append(ev[1].elapsed_time(ev[2]))
            bwd.append(ev[2].elapsed_time(ev[3]))
    lr.lr_score_status(lws, B, M, d)
    mm, fm, bm = (float(np.median(x)) for x in (mine, fwd, bwd))
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        peak, kind = float(pk["bf16_tflops"]), "measured (bf16 burst)"
    except (OSError, KeyError, ValueError):
        peak, kind = 1800.0, "fallback"
    flops = 2.0 * B * M * d
    out = {"metric": "hard-negative mining ms @B=%d M=%d d=%d top-%d BF16" % (B, M, d, args.n_neg), "value": mm,
           "unit": "ms", "higher_is_better": False, "n_gpus": 1, "dtype": "bf16", "data": "synthetic (seeded generator)",
           "mine_ms": mm, "loss_fwd_ms_on_mined": fm, "loss_bwd_ms_on_mined": bm,
           "config": {"workload": "%d queries vs %d in-batch positives + %d sampled jobs, term mask from the cfg-1 "
                                  "filter generator (%.1f%% allowed), top %d negatives per query"
                                  % (B, B, M - B, 100.0 * float(npass.sum()) / (B * M), args.n_neg),
                      "B": B, "M": M, "d": d, "n_neg": args.n_neg},
           "mined_mean": float(cnt.float().mean().item()),
           "roofline": {"bound": "hbm", "note": "score product on the tensor cores (%.1f GFLOP) plus B x M 8-byte "
                                                "keys written and read by the selection" % (flops / 1e9),
                        "keys_bytes": 2 * 8.0 * B * M, "peak_tflops": peak, "peak_kind": kind,
                        "tensor_tflops_achieved": flops / (mm / 1e3) / 1e12}}
    print(json.dumps(out), flush=True)


def run_peaks(args):
    """Device facts (SM count, L2 size, clocks) and the throughput of library dense products per type:
    torch.matmul (cuBLAS) in BF16, TF32, FP32 without TF32 (SIMT), FP64, and torch._scaled_mm in FP8 e4m3,
    each the best of 10 CUDA-event-timed calls after warm-up.  These are the denominators a fraction of
    peak for those types would use; the HBM copy and BF16 peaks come from the driver's measurement."""
    import torch

    dev = torch.cuda.get_device_properties(0)
    out = {"metric": "device peaks (library dense products)", "n_gpus": 1, "name": dev.name,
           "sm_count": dev.multi_processor_count, "l2_bytes": int(getattr(dev, "L2_cache_size", 0)),
           "total_mem_bytes": int(dev.total_memory), "rates_tflops": {}}

    def timeit(fn, flops):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return flops / (best / 1e3) / 1e12

    n = 8192
    a = torch.randn(n, n, device="cuda")
    b = torch.randn(n, n, device="cuda")
    ab, bb = a.to(torch.bfloat16), b.to(torch.bfloat16)
    out["rates_tflops"]["bf16"] = timeit(lambda: ab @ bb, 2.0 * n ** 3)
    torch.backends.cuda.matmul.allow_tf32 = True
    out["rates_tflops"]["tf32"] = timeit(lambda: a @ b, 2.0 * n ** 3)
    torch.backends.cuda.matmul.allow_tf32 = False
    out["rates_tflops"]["fp32_no_tf32"] = timeit(lambda: a @ b, 2.0 * n ** 3)
    m = 4096
    a64, b64 = torch.randn(m, m, device="cuda", dtype=torch.float64), torch.randn(m, m, device="cuda",
                                                                                   dtype=torch.float64)
    out["rates_tflops"]["fp64"] = timeit(lambda: a64 @ b64, 2.0 * m ** 3)
    try:
        a8 = a.to(torch.float8_e4m3fn)
        b8 = b.to(torch.float8_e4m3fn).t().contiguous().t()
        one = torch.ones((), device="cuda")
        out["rates_tflops"]["fp8_e4m3"] = timeit(
            lambda: torch._scaled_mm(a8, b8, scale_a=one, scale_b=one, out_dtype=torch.bfloat16), 2.0 * n ** 3)
    except Exception as e:  # the scaled product may be missing from a build
        out["rates_tflops"]["fp8_e4m3"] = None
        out["fp8_error"] = str(e)[:200]
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.form == "loss":
        run_loss(args)
    elif args.form == "serve":
        run_serve(args)
    elif args.form == "sweep":
        run_sweep(args)
    elif args.form == "topk":
        run_topk(args)
    elif args.form == "sign":
        run_sign(args)
    elif args.form == "hardneg":
        run_hardneg(args)
    elif args.form == "peaks":
        run_peaks(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
