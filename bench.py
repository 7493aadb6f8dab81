#!/usr/bin/env python3
"""Benchmark of the range-domain block search on GB300.

Workload: the 512 x 512 precision workload (1/f texture, alpha = 2, seed 2,
plus 16 axis-aligned step edges), quadtree 16 -> 8 -> 4, domains at step
L = 1 with the full pool ((N - 2B + 1)^2 positions per step), 8 isometries,
the paper's predefined S per step, RMS tolerance 8.  One step = one full
encode of the image (every step of the hot path), device-resident image to
device-resident records.

Metric: Gmatch/s = (sum over steps of ranges x pool domains x 8 isometries)
/ encode time, for the tensor-core engine; ms per 512^2 encode, the CUDA-core
engine's Gmatch/s and the records' equality across engines ride along.  The
default line also carries the roofline of the contraction (against the dense
FP16 peak), the same encode end to end through host buffers, the oracle on a
bounded sample (cpu_baseline), and, on one GPU, the 64-image batching
workload and a below-capacity serving run.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
  python bench.py --workload batch64|serving|compare|graph|ratedist|peaks

Under torchrun each rank encodes its own copy (independent replicas, weak
scaling); rank 0 prints one JSON line.  ``--impl reference`` times the CPU
oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import datetime
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import fic_synth  # noqa: E402

WORKLOAD = "precision512"
METRIC = "Gmatch/s and ms per 512² encode, tensor-core vs plain GPU at bit-identical codes"
L2_FLUSH_BYTES = 512 * 1024 * 1024


def workload():
    w = dict(fic_synth.WORKLOADS[WORKLOAD])
    img = fic_synth.workload_image(WORKLOAD)
    S = {16: (10, [1]), 8: (10, [2, 4]), 4: (10, [3, 8])}
    ss = [S[b] for b in (16, 8, 4)]
    return w, img, ss


def config_dict(w, extra=None):
    d = {"workload": "precision512: 512x512 uint8 1/f (alpha 2, seed 2) + 16 step edges; "
                     "quadtree 16->8->4, L=1, full pool, 8 isometries, S {0.1},{0.2,0.4},"
                     "{0.3,0.8}, RMS tol 8",
         "N": 512, "B_max": w["B_max"], "B_min": w["B_min"], "L": w["L"],
         "entropy_thresh": None, "err_tol": w["err_tol"],
         "l2": "flushed between timed steps (512 MiB write)"}
    if extra:
        d.update(extra)
    return d


def contraction_profile():
    """The committed ncu capture of the three contraction launches of one
    encode, or None when the kernel sources changed since it was taken."""
    import hashlib
    try:
        prof = json.load(open(os.path.join(ROOT, "profiles", "contract_traffic_precision512.json")))
        h = hashlib.sha1()
        for f in prof["sources"]:
            h.update(open(os.path.join(ROOT, f), "rb").read())
        return prof if h.hexdigest() == prof["sources_sha1"] else None
    except Exception:
        return None


def measured_traffic():
    """Mean DRAM bytes per contraction launch of one encode from the committed
    ncu capture, or None when the kernel sources changed since."""
    prof = contraction_profile()
    if prof is None:
        return None
    ls = prof["launches"]
    return sum(x["dram_read_bytes"] + x["dram_write_bytes"] for x in ls) / len(ls)


def contraction_only(flops_per_step, peak_tf):
    """The MMA pipeline alone: the encode's algorithmic flops over the time
    the tensor pipe was active in the committed capture (per launch,
    duration x sm__pipe_tensor_cycles_active), against the same peak.  The
    epilogue is not skipped (nothing is switched off in the product); the
    counter separates the MMA's own busy time inside the fused kernels."""
    prof = contraction_profile()
    if prof is None or len(prof["launches"]) != len(flops_per_step):
        return None
    act = [x["duration_ms_under_ncu"] * x["tensor_pipe_active_pct"] / 100.0
           for x in prof["launches"]]
    tf = sum(flops_per_step) / (sum(act) / 1e3) / 1e12
    return {"tflops_while_tensor_pipe_active": tf, "frac": tf / peak_tf,
            "tensor_pipe_active_pct": [x["tensor_pipe_active_pct"] for x in prof["launches"]],
            "fused_frac_per_step": [f / (x["duration_ms_under_ncu"] / 1e3) / 1e12 / peak_tf
                                    for f, x in zip(flops_per_step, prof["launches"])],
            "source": "profiles/contract_traffic_precision512.json (ncu --set full, one encode)"}


def load_peaks():
    """The driver's measured peaks (MEASURED_PEAKS.json: HBM copy GB/s, bf16
    GEMM TFLOP/s), or {} when absent."""
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def fp16_peak(peaks):
    """Dense FP16 tensor peak (TFLOP/s) for the contraction, which runs
    tcgen05 kind::f16 on FP16 operands: the larger of the FP16 GEMM burst
    measured on the GB300s (profiles/peak_gemm_fp16_bf16.json,
    written by ``bench.py --workload peaks``) and the driver's bf16 burst
    (fp16 and bf16 have the same nominal dense rate), so that the fraction is
    never flattered by a low measurement; else the recipe's fallback."""
    cands, notes = [], []
    try:
        pk = json.load(open(os.path.join(ROOT, "profiles", "peak_gemm_fp16_bf16.json")))
        cands.append(float(pk["fp16"]["burst_tflops"]))
        notes.append(f"fp16 GEMM burst {cands[-1]:.1f} (profiles/peak_gemm_fp16_bf16.json)")
    except Exception:
        pass
    if "bf16_tflops" in peaks:
        cands.append(float(peaks["bf16_tflops"]))
        notes.append(f"bf16 GEMM burst {cands[-1]:.1f} (MEASURED_PEAKS.json, fp16 nominal equal)")
    if not cands:
        return 1900.0, "of fallback: 1.9 PFLOP/s bf16 burst (fp16 nominal equal)"
    return max(cands), "of measured: max of " + "; ".join(notes)


# ---------------------------------------------------------------- clocks
def smi_device_id(dev):
    """The nvidia-smi --id of torch device `dev`.  torch numbers the devices
    CUDA_VISIBLE_DEVICES leaves visible from 0, nvidia-smi numbers every GPU of
    the machine, so torch's index can name another process's GPU.  Candidates,
    first accepted by nvidia-smi wins: the device's UUID, its entry in
    CUDA_VISIBLE_DEVICES, torch's index."""
    import torch
    cands = []
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid).strip()
        if u:
            cands.append(u if u.startswith(("GPU-", "MIG-")) else "GPU-" + u)
    except Exception:
        pass
    vis = [v.strip() for v in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if v.strip()]
    if dev.index is not None and dev.index < len(vis):
        cands.append(vis[dev.index])
    cands.append(str(dev.index or 0))
    for c in cands:
        try:
            out = subprocess.run(["nvidia-smi", f"--id={c}", "--query-gpu=index",
                                  "--format=csv,noheader"], capture_output=True, text=True,
                                 timeout=20)
            if out.returncode == 0 and out.stdout.strip():
                return c
        except Exception:
            pass
    return cands[-1]


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons.  Each sample carries
    nvidia-smi's own timestamp, so only the samples taken between begin() and
    end() (the timed steps) are reported; when none fell inside (a region
    shorter than the sampling period), the samples of the whole run are, and
    'window' says so."""

    QUERY = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, index, period_ms=50):
        self.index = index
        self.period_ms = period_ms
        self.proc = None
        self.lines = []
        self.t = None
        self.region = [None, None]

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", str(self.period_ms)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def begin(self):
        self.region[0] = datetime.datetime.now()

    def end(self):
        self.region[1] = datetime.datetime.now()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    @staticmethod
    def _when(text):
        try:
            return datetime.datetime.strptime(text, "%Y/%m/%d %H:%M:%S.%f")
        except ValueError:
            return None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t is not None:
            self.t.join(timeout=5)
        rows = []
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 10:
                continue
            try:
                sm, smax = float(parts[2]), float(parts[3])
            except ValueError:
                continue
            act = {nm for nm, v in zip(self.REASONS, parts[6:10]) if v.lower().startswith("active")}
            rows.append((self._when(parts[0]), sm, smax, act))
        t0, t1 = self.region
        inside = [r for r in rows
                  if t0 is not None and t1 is not None and r[0] is not None and t0 <= r[0] <= t1]
        use = inside if inside else rows
        return {"sm_mhz": statistics.median([r[1] for r in use]) if use else None,
                "sm_max_mhz": use[-1][2] if use else None,
                "reasons": sorted(set().union(*[r[3] for r in use])) if use else [],
                "samples": len(use),
                "window": "timed steps" if inside else "whole run (no sample inside the timed steps)",
                "period_ms": self.period_ms, "gpu": str(self.index)}


# ---------------------------------------------------------------- CPU oracle timing
def oracle_sample(img, ss, per_level=(2, 4, 16), seed=0, nthreads=0):
    """Time the oracle's search on a bounded sample of ranges per step.
    Returns (matches, seconds, description)."""
    import oracle
    rng = np.random.default_rng(seed)
    matches, secs = 0, 0.0
    desc = []
    for lvl, B in enumerate((16, 8, 4)):
        k = per_level[lvl]
        if k == 0:
            continue
        pool = oracle.Pool(img, B, 1, -1.0)
        per = 512 // B
        idx = rng.choice(per * per, k, replace=False)
        rx = (idx % per) * B
        ry = (idx // per) * B
        t0 = time.perf_counter()
        pool.search(rx, ry, ss[lvl], nthreads=nthreads)
        secs += time.perf_counter() - t0
        matches += k * pool.dn * 8
        desc.append(f"{k} ranges x {pool.dn} domains x 8 at B={B}")
    return matches, secs, "; ".join(desc)


def oracle_encode_matches():
    """Matches per quadtree step of the oracle's own full encode of this
    workload (tests/golden/precision512_oracle.json, written from the oracle
    alone), or None when the file is absent."""
    try:
        g = json.load(open(os.path.join(ROOT, "tests", "golden", "precision512_oracle.json")))
        return [int(m) for m in g["matches"]]
    except Exception:
        return None


def run_reference(args):
    """The oracle (plain C, OpenMP over ranges) on the host cores.  Each step
    times a bounded sample of ranges at every quadtree step; the value weights
    the per-step rates by the matches of each step in a whole encode, as the
    GPU arm's cpu_baseline does."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    w, img, ss = workload()
    cores = oracle.max_threads()
    for _ in range(args.warmup):
        oracle_sample(img, ss, per_level=(1, 1, 2), seed=99)
    per_level = (16, 16, 32)
    lvl_m, lvl_s = [0, 0, 0], [0.0, 0.0, 0.0]
    tot_s, descs = 0.0, []
    for k in range(args.steps):
        for lvl in range(3):
            pl = [0, 0, 0]
            pl[lvl] = per_level[lvl]
            m, s, d = oracle_sample(img, ss, per_level=tuple(pl), seed=k)
            lvl_m[lvl] += m
            lvl_s[lvl] += s
            tot_s += s
            if k == 0:
                descs.append(d)
    rates = [m / s for m, s in zip(lvl_m, lvl_s)]
    weights = oracle_encode_matches()
    if weights is not None:
        how = "rates weighted by the matches per step of the oracle's full encode"
    else:
        weights, how = lvl_m, "rates weighted by the sample's own matches per step"
    est_s = sum(wm / r for wm, r in zip(weights, rates))
    value = sum(weights) / est_s / 1e9
    desc = "; ".join(f"{d} ({r / 1e9:.4f} Gmatch/s)" for d, r in zip(descs, rates))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gmatch/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * tot_s / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": config_dict(w, {"sample_per_step": desc}),
        "cpu_baseline": {"value": value, "unit": "Gmatch/s", "cores": cores, "kind": "oracle",
                         "sample": f"per step: {desc}; {how}",
                         "est_ms_per_image": 1e3 * est_s},
        "e2e": {"value": value, "unit": "Gmatch/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU arm
def rank_reduce(times, work, device):
    """Across the ranks of the default process group: the max of each time
    and the sum of each work count (replicas: no other exchange)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x) for x in times], dtype=torch.float64, device=device)
    w = torch.tensor([float(x) for x in work], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return t.tolist(), w.tolist()


def run_gpu(args):
    import torch
    import paper_1502_00324_gb300 as pkg

    legs = set(args.legs.split(","))

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()

    w, img, ss = workload()
    pkg.fic_tune_mode(args.tune_mode)
    if args.only_side:
        # profiling aid: one quadtree step at side B over all (512 / B)^2 ranges
        lvl = {16: 0, 8: 1, 4: 2}[args.only_side]
        w = dict(w, B_max=args.only_side, B_min=args.only_side)
        ss = [ss[lvl]]
    N = img.shape[0]
    dimg = torch.from_numpy(img).to(dev)
    cap = (N // w["B_min"]) ** 2
    dcodes = torch.empty(cap * 16, dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def enc(engine, src=dimg, out=dcodes):
        return pkg.fic_encode_ex(src, N, w["B_max"], w["B_min"], w["L"], -1.0, ss,
                                 w["err_tol"], engine=engine, stream=stream, codes_out=out)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def timed(engine, steps, warmup, timing, sampler=None):
        for _ in range(warmup):
            enc(engine)
        torch.cuda.synchronize()
        pkg.fic_stats_reset(timing=timing)
        evs = []
        barrier()
        torch.cuda.synchronize()
        if sampler is not None:
            sampler.begin()
        t_wall = time.perf_counter()
        matches = 0
        for _ in range(steps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = enc(engine)
            e1.record(stream)
            evs.append((e0, e1))
            matches += r.total_matches
        torch.cuda.synchronize()
        if sampler is not None:
            sampler.end()
        barrier()
        wall = time.perf_counter() - t_wall
        ms = sum(a.elapsed_time(b) for a, b in evs)
        stats = pkg.fic_stats_read()
        return ms, matches, stats, r, wall

    # tensor-core engine (the headline): the production path as a user runs it
    # (no per-stage events), clocks sampled during the timed steps
    sampler = ClockSampler(smi_device_id(dev))
    sampler.start()
    ms_t, m_t, st_u, r_t, wall_t = timed(pkg.ENGINE_TENSOR, args.steps, args.warmup, False,
                                         sampler)
    clocks = sampler.stop()
    codes_t = dcodes[: r_t.n_codes * 16].cpu().numpy().copy()
    # the same steps again with the library's per-stage CUDA events on the
    # launching stream: kernel times for the roofline and the stage rates
    ms_i, _, st_t, r_i, _ = timed(pkg.ENGINE_TENSOR, args.steps, 3, True)
    assert r_i.n_codes == r_t.n_codes

    # CUDA-core engine on the same workload (fewer steps; it is much slower)
    psteps = max(1, min(args.steps, 3))
    ms_p, m_p, identical = float("nan"), 0, None
    if "plain" in legs:
        ms_p, m_p, st_p, r_p, _ = timed(pkg.ENGINE_PLAIN, psteps, 1, False)
        codes_p = dcodes[: r_p.n_codes * 16].cpu().numpy().copy()
        identical = bool(r_t.n_codes == r_p.n_codes and np.array_equal(codes_t, codes_p))

    # end to end through the C ABI with host buffers (H2D image, D2H records)
    # (each call timed on its own, host clock around the synchronous call,
    # L2 flushed before it exactly as before each device-timed step)
    e2e_m, e2e_s = 0, float("nan")
    if "e2e" in legs:
        himg = torch.from_numpy(img).pin_memory()
        hcodes = torch.empty(cap * 16, dtype=torch.uint8).pin_memory()
        for _ in range(max(1, args.warmup)):
            enc(pkg.ENGINE_TENSOR, src=himg, out=hcodes)
        torch.cuda.synchronize()
        barrier()
        e2e_s = 0.0
        for _ in range(args.steps):
            flush.fill_(1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = enc(pkg.ENGINE_TENSOR, src=himg, out=hcodes)
            e2e_s += time.perf_counter() - t0
            e2e_m += r.total_matches
        torch.cuda.synchronize()
        barrier()

    # max over ranks of the times; sum of work
    if world > 1:
        (ms_t, e2e_s, ms_p), (m_t, e2e_m, m_p) = rank_reduce([ms_t, e2e_s, ms_p],
                                                             [m_t, e2e_m, m_p], dev)
    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return 0

    gmatch_t = m_t / (ms_t / 1e3) / 1e9
    gmatch_p = m_p / (ms_p / 1e3) / 1e9 if m_p else None
    ms_per_img = ms_t / args.steps

    # roofline of the dominant kernel (the fused contraction + scoring)
    peaks = load_peaks()
    peak_tf, peak_note = fp16_peak(peaks)
    tc = st_t["contract_tc"]
    achieved = tc["flops"] / (tc["ms"] / 1e3) / 1e12 if tc["ms"] > 0 else None
    kern_ms = {k: v["ms"] / args.steps for k, v in st_t.items() if isinstance(v, dict)}
    # the memory-bound stages against the measured HBM copy bandwidth
    hbm = peaks.get("hbm_gbs", 6800.0)
    stages = {}
    for k in ("entropy", "scan", "gather", "range_prep", "split", "order"):
        v = st_t.get(k)
        if isinstance(v, dict) and v["ms"] > 0 and v["bytes"] > 0:
            gbs = v["bytes"] / (v["ms"] / 1e3) / 1e9
            stages[k] = {"ms_per_step": v["ms"] / args.steps,
                         "bytes_per_step": v["bytes"] / args.steps,
                         "GB/s": gbs, "frac_of_hbm": gbs / hbm}
    launches = sum(v["launches"] for k, v in st_u.items() if isinstance(v, dict))

    cpu = None
    if "cpu" in legs and not args.only_side:
        # oracle rate per step on a bounded sample, weighted by the matches
        # per step of the oracle's own full encode (stored), else of this
        # encode (equal under parity)
        import oracle
        weights = oracle_encode_matches()
        how = "the oracle's full encode"
        if weights is None:
            weights, how = list(r_t.matches), "this encode"
        est_s, descs = 0.0, []
        for lvl, k in enumerate((32, 64, 128)):
            pl = [0, 0, 0]
            pl[lvl] = k
            m, s, desc = oracle_sample(img, ss, per_level=tuple(pl), seed=1)
            est_s += weights[lvl] / (m / s)
            descs.append(f"{desc} ({m / s / 1e9:.4f} Gmatch/s)")
        cpu = {"value": sum(weights) / est_s / 1e9, "unit": "Gmatch/s",
               "cores": oracle.max_threads(), "kind": "oracle",
               "sample": "; ".join(descs) + f"; rates weighted by the matches per step of {how}",
               "est_ms_per_image": 1e3 * est_s}

    tuned = [[t["K"], t["iso_tiles"], t["refill"], t["epi_warps"], round(t["ms"], 3)]
             for t in pkg.fic_tune_read()]

    # the batching and serving forms, after the headline's timed steps (one GPU)
    batch_res = serving_res = None
    if world == 1 and not args.only_side:
        if "batch" in legs:
            batch_res = measure_batch(max(3, min(args.steps, 5)), 2)
        if "serving" in legs:
            t_arr, sides, simgs = serving_images(40, 4.0)
            serving_res = measure_serving(t_arr, sides, simgs, 4.0)

    line = {
        "metric": METRIC, "value": gmatch_t, "unit": "Gmatch/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_img,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "fp16->fp32 (exact int)",
        "data": "synthetic (seeded 1/f images, stand-ins for the paper's test images)",
        "config": config_dict(w, {"parallelism": f"replicas x{world}",
                                  "only_side": args.only_side or None}),
        "ms_per_image": ms_per_img,
        "plain": {"value": gmatch_p, "unit": "Gmatch/s",
                  "ms_per_image": (ms_p / psteps) if m_p else None},
        "tensor_over_plain": (gmatch_t / gmatch_p) if gmatch_p else None,
        "codes_identical_tensor_vs_plain": identical,
        "matches_per_image": r_t.total_matches,
        "per_level": {"ranges": r_t.ranges, "pool": r_t.pool_size, "matches": r_t.matches},
        "kernel_ms_per_step": kern_ms,
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak_tf,
                     "unit": "TFLOP/s", "frac": (achieved / peak_tf) if achieved else None,
                     "traffic": None if args.only_side else measured_traffic(),
                     "traffic_unit": "bytes per contraction launch (mean of the 3 steps)",
                     "kernel": "contraction (the tuner's kernel per step: contract_tc_kernel "
                               "at 16x16, contract_tc_red_kernel at 8x8 and 4x4)",
                     "algorithmic_flops_per_encode": tc["flops"] / max(args.steps, 1),
                     "timing": "library CUDA events around each contraction launch on the "
                               "launching stream, over a second pass of the same steps with "
                               "per-stage events on (ms per encode with events: "
                               f"{ms_i / args.steps:.3f})",
                     "peak_note": peak_note,
                     "contraction_only": None if args.only_side else contraction_only(
                         [2.0 * 8 * R * D * (w["B_max"] >> l) ** 2
                          for l, (R, D) in enumerate(zip(r_t.ranges, r_t.pool_size))], peak_tf)},
        "stages_hbm": {"peak_gbs": hbm, "note": "algorithmic bytes / CUDA-event time of the "
                       "stage's launches; peak = measured HBM copy bandwidth "
                       "(MEASURED_PEAKS.json)", "stages": stages},
        "cpu_baseline": cpu,
        "e2e": {"value": (e2e_m / e2e_s / 1e9) if e2e_m else None, "unit": "Gmatch/s",
                "h2d_bytes_per_step": int(N * N), "d2h_bytes_per_step": int(r_t.n_codes * 16)},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "wall_s_tensor": wall_t,
        # contraction shapes the tuner kept: (K, isometry tiles, refill, epilogue warps, ms)
        "tuned_shapes": tuned,
        "batch64": batch_res,
        "serving": serving_res,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------- batching form
BATCH_DESC = ("batch64: 64 uint8 1/f images, seeds 100..163, side uniform over {128, 256, 384, "
              "512, 768, 1024}, alpha uniform in [1.5, 2.5]; quadtree 16->8->4, L=2, entropy > "
              "4.0 bits, S {0.1},{0.2,0.4},{0.3,0.8}, RMS tol 8")


def entropy_updates(results, L=2, B_max=16):
    """Histogram updates the entropy kernel makes for the steps that ran: per
    row run of 32 positions one full window (4n pixels), then per further
    position 2 x min(L, 2B) x 2B (the columns that leave and enter)."""
    tot = 0
    for r in results:
        N = int(r.N)
        for lvl in range(len(r.ranges)):
            if int(r.ranges[lvl]) <= 0:
                continue
            B = B_max >> lvl
            S = 2 * B
            per = (N - S) // L + 1 if N >= S else 0
            if per <= 0:
                continue
            runs = per * ((per + 31) // 32)
            tot += runs * S * S + (per * per - runs) * 2 * min(L, S) * S
    return tot


def smem_atomic_peak(sm_mhz, n_sms=152):
    """Nominal bound of the entropy stage: the shared-memory pipe serves one
    32-lane access per clock per SM, and a histogram update (atomic
    increment) needs at least one."""
    return n_sms * 32 * (sm_mhz or 2070.0) * 1e6


def measure_batch(steps, warmup, one_by_one_steps=0, sampler_dev=None):
    """The 64-image batching workload: every image in one fic_encode_batch
    call (one grouped contraction launch per quadtree step, the whole call
    one CUDA graph from the second call on); optionally against the same
    images encoded one call at a time.  Returns the measurement dict."""
    import torch
    import paper_1502_00324_gb300 as pkg

    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    imgs = fic_synth.batch_images(64)
    dimgs = [torch.from_numpy(im).to(dev) for im in imgs]
    ss = pkg.paper_ssets(16, 4)
    args_enc = (16, 4, 2, 4.0, ss, 8.0)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def batch():
        return pkg.fic_encode_batch(dimgs, *args_enc, stream=stream)

    def one_by_one():
        return [pkg.fic_encode_ex(d, d.shape[0], *args_enc, stream=stream) for d in dimgs]

    def timed(fn, steps, warmup, timing=False, sampler=None):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        pkg.fic_stats_reset(timing=timing)
        ms, out = [], None
        if sampler is not None:
            sampler.begin()
        for _ in range(steps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        if sampler is not None:
            sampler.end()
        return ms, out, pkg.fic_stats_read()

    sampler = ClockSampler(smi_device_id(dev))
    sampler.start()
    ms_b, out_b, st_u = timed(batch, steps, warmup, False, sampler)
    clocks = sampler.stop()
    # kernel times: the same call again with per-stage events on
    ms_e, _, st_b = timed(batch, steps, 2, True)
    matches = sum(r.total_matches for r in out_b)
    med_b = statistics.median(ms_b)
    launches = sum(v["launches"] for v in st_u.values() if isinstance(v, dict))
    tc = st_b["contract_tc"]
    peak_tf, peak_note = fp16_peak(load_peaks())
    achieved = tc["flops"] / (tc["ms"] / 1e3) / 1e12 if tc["ms"] > 0 else None
    kern_ms = {k: v["ms"] / steps for k, v in st_b.items() if isinstance(v, dict)}
    upd = entropy_updates(out_b)
    ent_ms = kern_ms.get("entropy", 0.0)
    ent_rate = upd / (ent_ms / 1e3) if ent_ms > 0 else None
    ent_peak = smem_atomic_peak(clocks.get("sm_mhz"))
    res = {
        "metric": "aggregate Gmatch/s and ms per image, 64-image batch", "workload": "batch64",
        "value": matches / (med_b / 1e3) / 1e9, "unit": "Gmatch/s", "n_gpus": 1,
        "steps": steps, "warmup": warmup, "ms_per_step": med_b,
        "higher_is_better": True, "dtype": "fp16->fp32 (exact int)", "data": "synthetic",
        "config": {"workload": BATCH_DESC, "images": len(imgs),
                   "sides": sorted(int(i.shape[0]) for i in imgs),
                   "l2": "flushed between timed steps (512 MiB write)",
                   "timed": "device-resident images -> host records (D2H of records inside)"},
        "ms_per_image": med_b / len(imgs), "images_per_s": len(imgs) / (med_b / 1e3),
        "matches_per_batch": matches,
        "kernel_ms_per_step": kern_ms,
        "ms_per_step_with_stage_events": statistics.median(ms_e),
        "contraction_tflops": achieved, "contraction_frac_of_fp16_peak":
            (achieved / peak_tf) if achieved else None, "peak_note": peak_note,
        "entropy": {"updates_per_batch": upd, "ms_per_batch": ent_ms,
                    "updates_per_s": ent_rate, "bound": "alu",
                    "peak_updates_per_s": ent_peak,
                    "frac": (ent_rate / ent_peak) if ent_rate else None,
                    "peak_note": "nominal: 152 SMs x one 32-lane shared-memory access per "
                                 "clock (an atomic histogram update needs at least one) x "
                                 "the median SM clock sampled"},
        "gpu_launches": int(launches / steps), "clocks": clocks,
    }
    if one_by_one_steps:
        ms_s, out_s, _ = timed(one_by_one, one_by_one_steps, 1)
        med_s = statistics.median(ms_s)
        res["one_call_per_image"] = {"ms_per_batch": med_s,
                                     "value": matches / (med_s / 1e3) / 1e9, "unit": "Gmatch/s"}
        res["batch_over_one_by_one"] = med_s / med_b
        res["codes_identical_batch_vs_single"] = all(
            np.array_equal(a.codes, b.codes) for a, b in zip(out_b, out_s))
    return res


def run_batch(args):
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    res = measure_batch(args.steps, args.warmup,
                        one_by_one_steps=max(1, min(args.steps, 3)) if args.single else 0)
    print(json.dumps(res), flush=True)
    return 0


# ---------------------------------------------------------------- serving form
def serving_desc(rate_hz):
    return (f"serving: Poisson arrivals (seed 7, mean {rate_hz:g} images/s) of uint8 1/f images "
            "(alpha 2, seed 700000 + i), side uniform over {256, 512, 1024, 2048}; quadtree "
            "16->8->4, L=2, entropy > 4.0 bits, S {0.1},{0.2,0.4},{0.3,0.8}, RMS tol 8")


def _serving_image(args):
    side, seed = args
    return fic_synth.one_over_f(int(side), int(seed), 2.0)


def serving_images(requests, rate_hz):
    """Arrival times, sides and images of the request stream, generated in
    spawned workers (safe after the parent has used the GPU)."""
    import multiprocessing as mp
    t_arr, sides = fic_synth.poisson_requests(requests, seed=7, mean_rate_hz=rate_hz)
    jobs = [(int(n), 7 * 100000 + i) for i, n in enumerate(sides)]
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        imgs = pool.map(_serving_image, jobs)
    return t_arr, sides, imgs


def measure_serving(t_arr, sides, imgs, rate_hz, policy=0):
    """Request loop: a feeder thread submits each image at its Poisson arrival
    time to one fic_server (host images); the main thread polls.  Latency =
    records on the host - submit, on the server's clock.  Before the stream,
    each side is served alone (nothing else in the server) to give the
    service latency without queueing."""
    import torch
    import paper_1502_00324_gb300 as pkg
    dev = torch.device("cuda", torch.cuda.current_device())
    ss = pkg.paper_ssets(16, 4)
    # warm-up, then the service latency of each side alone (second pass)
    alone = {}
    with pkg.Server(16, 4, 2, 4.0, ss, 8.0) as w:
        for rep in range(2):
            for side in sorted(set(int(n) for n in sides)):
                _, tm = w.poll(w.submit(fic_synth.one_over_f(side, 1, 2.0)))
                if rep == 1:
                    alone[str(side)] = tm["done_ms"] - tm["submit_ms"]
    srv = pkg.Server(16, 4, 2, 4.0, ss, 8.0, policy=policy)
    tickets = [None] * len(imgs)
    sampler = ClockSampler(smi_device_id(dev))
    sampler.start()
    sampler.begin()
    t0 = time.perf_counter()

    def feed():
        for i, im in enumerate(imgs):
            dt = t0 + float(t_arr[i]) - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            tickets[i] = srv.submit(im)

    th = threading.Thread(target=feed)
    th.start()
    results = []
    for i in range(len(imgs)):
        while tickets[i] is None:
            time.sleep(0.0005)
        results.append(srv.poll(tickets[i], wait_ms=-1))
    th.join()
    wall = time.perf_counter() - t0
    sampler.end()
    clocks = sampler.stop()
    st = srv.stats()
    srv.close()
    lat = np.array([tm["done_ms"] - tm["submit_ms"] for _, tm in results])
    wait = np.array([tm["admit_ms"] - tm["submit_ms"] for _, tm in results])
    span_ms = max(tm["done_ms"] for _, tm in results) - min(tm["submit_ms"] for _, tm in results)
    matches = sum(enc.total_matches for enc, _ in results)
    by_side = {}
    for (enc, tm), n in zip(results, sides):
        by_side.setdefault(int(n), []).append(tm["done_ms"] - tm["submit_ms"])
    offered = len(results) / max(float(t_arr[-1]), 1e-9)
    return {
        "metric": "p50/p99 encode latency and images/s under a Poisson request stream",
        "workload": "serving", "value": len(results) / (span_ms / 1e3), "unit": "images/s",
        "n_gpus": 1, "requests": len(results), "higher_is_better": True,
        "dtype": "fp16->fp32 (exact int)", "data": "synthetic",
        "config": {"workload": serving_desc(rate_hz), "arrival_span_s": float(t_arr[-1]),
                   "sides": {str(k): len(v) for k, v in sorted(by_side.items())},
                   "server": {"hbm_budget": st["hbm_budget"], "max_inflight": 64,
                              "policy": ["fifo", "smallest first, 2 s aging"][policy]}},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p90": float(np.percentile(lat, 90)),
                       "p99": float(np.percentile(lat, 99)), "max": float(lat.max()),
                       "mean_queue_wait": float(wait.mean())},
        "latency_ms_by_side_p50": {str(k): float(np.percentile(v, 50))
                                   for k, v in sorted(by_side.items())},
        "service_ms_alone_by_side": alone,
        "gmatch_per_s": matches / (span_ms / 1e3) / 1e9,
        "server": {k: st[k] for k in ("iterations", "contraction_launches", "mean_inflight",
                                      "peak_inflight", "hbm_peak", "busy_ms", "failed")},
        "offered_load_images_per_s": offered,
        "busy_fraction": st["busy_ms"] / max(span_ms, 1e-9),
        "wall_s": wall, "clocks": clocks,
    }


def run_serving(args):
    t_arr, sides, imgs = serving_images(args.requests, args.rate)
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    print(json.dumps(measure_serving(t_arr, sides, imgs, args.rate, args.policy)), flush=True)
    return 0


# ---------------------------------------------------------------- proposed vs entropy-based
COMPARE_DESC = ("compare: the 512x512 precision image (1/f texture, alpha 2, seed 2, 16 step "
                "edges), quadtree 16->8->4->2 (the paper's four steps), L=2, top-DN pools "
                "DN in {32, 64, 144, 192, 256}, RMS tol 8; proposed = the paper's predefined S "
                "per step ({0.1}, {0.2,0.4}, {0.3,0.8}, {0.5,0.9}); entropy-based baseline = "
                "S = k/10, k = 1..10, at every step")


def run_graph(args):
    """Latency of one synchronous encode call, steps one by one (the host
    reads the counts back between steps) against one captured graph of the
    whole quadtree, over image sides; quadtree 16 -> 4, L = 2, entropy > 4.0
    bits (the batching and serving configuration), device-resident images
    and records, different images per call (the quadtrees differ)."""
    import torch
    import paper_1502_00324_gb300 as pkg
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    ss = [pkg.PAPER_S[b] for b in (16, 8, 4)]
    rows = []
    for n in (128, 256, 512, 1024):
        imgs = [torch.from_numpy(fic_synth.one_over_f(n, 900 + i, 2.0)).to(dev) for i in range(8)]
        out = torch.empty((n // 4) ** 2 * 16, dtype=torch.uint8, device=dev)
        row = {"N": n}
        for name, mode in (("eager", 0), ("graph", 1)):
            pkg.fic_graph_mode(mode)

            def enc(im):
                return pkg.fic_encode_ex(im, n, 16, 4, 2, 4.0, ss, 8.0, stream=stream,
                                         codes_out=out)
            for _ in range(max(args.warmup, 3)):
                for im in imgs[:2]:
                    enc(im)
            torch.cuda.synchronize()
            cap0, rep0 = pkg.fic_graph_counts()
            t0 = time.perf_counter()
            reps = max(args.steps, 1)
            codes = []
            for _ in range(reps):
                for im in imgs:
                    r = enc(im)
            torch.cuda.synchronize()
            ms = (time.perf_counter() - t0) * 1e3 / (reps * len(imgs))
            cap1, rep1 = pkg.fic_graph_counts()
            for im in imgs[:3]:
                r = enc(im)
                codes.append(out[: r.n_codes * 16].cpu().numpy().tobytes())
            row[name] = {"ms_per_encode": ms, "graph_replays": rep1 - rep0,
                         "graph_captures": cap1 - cap0}
            row[name + "_codes"] = codes
        row["codes_identical"] = row.pop("eager_codes") == row.pop("graph_codes")
        row["graph_speedup"] = row["eager"]["ms_per_encode"] / row["graph"]["ms_per_encode"]
        rows.append(row)
    pkg.fic_graph_mode(1)
    line = {"metric": "ms per synchronous encode call, steps one by one vs one CUDA graph",
            "workload": "graph", "unit": "ms", "higher_is_better": False, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "dtype": "fp16->fp32 (exact int)",
            "data": "synthetic",
            "config": {"workload": "graph: 8 uint8 1/f images (alpha 2, seeds 900-907) per "
                                   "side, quadtree 16->8->4, L=2, entropy > 4.0 bits, "
                                   "S {0.1},{0.2,0.4},{0.3,0.8}, RMS tol 8; host wall time of "
                                   "the synchronous call, device-resident input and records"},
            "rows": rows}
    print(json.dumps(line), flush=True)
    return 0


def run_compare(args):
    """Encode time, quality and stored size of the proposed method
    (predefined S per step) against the entropy-based baseline (ten S values
    per step) on the same top-DN pools (Sec. 4, Tables 2-3, eq. 9); the
    stream is Sec. 3.3 / Fig. 7 / eq. 8 with the domain lists in its
    header."""
    import torch
    import paper_1502_00324_gb300 as pkg
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    img = fic_synth.workload_image("precision512")
    dimg = torch.from_numpy(img).to(dev)
    prop = [pkg.PAPER_S[b] for b in (16, 8, 4, 2)]
    base = [(10, list(range(1, 11)))] * 4
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    rows = []
    for dn in (32, 64, 144, 192, 256):
        row = {"pool": dn}
        for name, ss in (("proposed", prop), ("entropy_based", base)):
            def enc():
                return pkg.fic_encode_ex(dimg, 512, 16, 2, 2, -1.0, ss, 8.0, stream=stream,
                                         pool_dn=dn)
            for _ in range(args.warmup):
                enc()
            ms = []
            for _ in range(args.steps):
                flush.fill_(1)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                r = enc()
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            rec, _ = pkg.fic_decode(r, iters_max=64)
            mse = float(np.mean((rec.astype(np.float64) - img) ** 2))
            packed, rec_bits = pkg.fic_pack(dimg, r, 16, 2, 2, -1.0, ss, 8.0, pool_dn=dn,
                                            stream=stream)
            row[name] = {"ms": statistics.median(ms), "records": r.n_codes,
                         "stream_bytes": len(packed), "record_bits": rec_bits,
                         "compression_ratio": 512 * 512 / len(packed),
                         "compression_ratio_records_only": 512 * 512 * 8 / rec_bits,
                         "bpp": 8.0 * len(packed) / (512 * 512),
                         "records_per_step": [int((r.codes["level"] == l).sum())
                                              for l in range(4)],
                         "psnr_db": 10 * np.log10(255.0 ** 2 / mse) if mse > 0 else None,
                         "gmatch_per_s": r.total_matches / (statistics.median(ms) / 1e3) / 1e9}
        row["time_ratio_proposed_over_baseline"] = row["proposed"]["ms"] / row["entropy_based"]["ms"]
        rows.append(row)
    line = {"metric": "encode ms, proposed vs entropy-based (ten S values) on top-DN pools",
            "workload": "compare", "unit": "ms", "higher_is_better": False, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "dtype": "fp16->fp32 (exact int)",
            "data": "synthetic", "config": {"workload": COMPARE_DESC}, "rows": rows}
    print(json.dumps(line), flush=True)
    return 0


def run_peaks(args):
    """Dense GEMM peaks of this GPU through cuBLAS (torch.matmul, 8192^3,
    FP32 accumulation): FP16 and BF16, as a burst (50 back-to-back GEMMs
    after warm-up) and sustained (a loop of about 8 s, median of 0.5 s
    windows after the first 2 s), CUDA events on the launching stream, with
    the SM clocks sampled during each."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    torch.backends.cuda.matmul.allow_fp16_reduced_precision_reduction = False
    torch.backends.cuda.matmul.allow_bf16_reduced_precision_reduction = False
    n = 8192
    flop = 2.0 * n * n * n
    out = {}
    for name, dt in (("fp16", torch.float16), ("bf16", torch.bfloat16)):
        g = torch.Generator(device=dev).manual_seed(5)
        a = torch.randn(n, n, device=dev, dtype=dt, generator=g)
        b = torch.randn(n, n, device=dev, dtype=dt, generator=g)
        c = torch.empty(n, n, device=dev, dtype=dt)
        for _ in range(20):
            torch.matmul(a, b, out=c)
        torch.cuda.synchronize()
        sampler = ClockSampler(smi_device_id(dev))
        sampler.start()
        time.sleep(0.2)
        sampler.begin()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(50):
            torch.matmul(a, b, out=c)
        e1.record(stream)
        torch.cuda.synchronize()
        sampler.end()
        burst = 50 * flop / (e0.elapsed_time(e1) / 1e3) / 1e12
        clk_burst = sampler.stop()
        sampler = ClockSampler(smi_device_id(dev))
        sampler.start()
        time.sleep(0.2)
        sampler.begin()
        wins, t_end = [], time.perf_counter() + 8.0
        while time.perf_counter() < t_end:
            w0 = torch.cuda.Event(enable_timing=True)
            w1 = torch.cuda.Event(enable_timing=True)
            w0.record(stream)
            for _ in range(200):
                torch.matmul(a, b, out=c)
            w1.record(stream)
            w1.synchronize()
            wins.append(200 * flop / (w0.elapsed_time(w1) / 1e3) / 1e12)
        sampler.end()
        clk_sus = sampler.stop()
        keep = wins[max(1, len(wins) // 4):]
        out[name] = {"burst_tflops": burst, "sustained_tflops": statistics.median(keep),
                     "sustained_windows": len(keep), "clocks_burst": clk_burst,
                     "clocks_sustained": clk_sus}
        del a, b, c
        torch.cuda.empty_cache()
    line = {"metric": "dense GEMM TFLOP/s (cuBLAS through torch.matmul, 8192^3, fp32 accumulate)",
            "workload": "peaks", "unit": "TFLOP/s", "n_gpus": 1, "higher_is_better": True,
            "device": torch.cuda.get_device_name(dev), "fp16_over_bf16_burst":
                out["fp16"]["burst_tflops"] / out["bf16"]["burst_tflops"], **out}
    print(json.dumps(line), flush=True)
    return 0


RATEDIST_DESC = ("ratedist: the 512x512 precision image (1/f texture, alpha 2, seed 2, 16 step "
                 "edges), quadtree 16->8->4->2 (the paper's four steps), L=2, top-DN pools DN in "
                 "{64, 256}, the paper's predefined S per step ({0.1}, {0.2,0.4}, {0.3,0.8}, "
                 "{0.5,0.9}); RMS tolerance swept over {2, 4, 6, 8, 12, 16}")


def run_ratedist(args):
    """Rate against distortion over the split tolerance (Sec. 4, Fig. 9):
    per point the stored stream's size (Sec. 3.3, Fig. 7, eq. 8: records and
    the header with the domain lists), the records alone, the compression
    ratio and the decoded PSNR (eq. 4), with the encode time."""
    import torch
    import paper_1502_00324_gb300 as pkg
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    img = fic_synth.workload_image("precision512")
    N = img.shape[0]
    dimg = torch.from_numpy(img).to(dev)
    ss = [pkg.PAPER_S[b] for b in (16, 8, 4, 2)]
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    rows = []
    for dn in (64, 256):
        for tol in (2.0, 4.0, 6.0, 8.0, 12.0, 16.0):
            def enc():
                return pkg.fic_encode_ex(dimg, N, 16, 2, 2, -1.0, ss, tol, stream=stream,
                                         pool_dn=dn)
            for _ in range(max(args.warmup, 1)):
                enc()
            ms = []
            for _ in range(max(args.steps, 1)):
                flush.fill_(1)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                r = enc()
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            rec, iters = pkg.fic_decode(r, iters_max=64)
            mse = float(np.mean((rec.astype(np.float64) - img) ** 2))
            packed, rec_bits = pkg.fic_pack(dimg, r, 16, 2, 2, -1.0, ss, tol, pool_dn=dn,
                                            stream=stream)
            rows.append({"pool": dn, "tol": tol, "records": r.n_codes,
                         "records_per_step": [int((r.codes["level"] == lv).sum())
                                              for lv in range(4)],
                         "stream_bytes": len(packed), "record_bits": rec_bits,
                         "bpp": 8.0 * len(packed) / (N * N),
                         "bpp_records_only": rec_bits / (N * N),
                         "compression_ratio": N * N / len(packed),
                         "compression_ratio_records_only": N * N * 8 / rec_bits,
                         "psnr_db": 10 * np.log10(255.0 ** 2 / mse) if mse > 0 else None,
                         "decode_passes": iters, "encode_ms": statistics.median(ms)})
    line = {"metric": "bits per pixel and decoded PSNR over the RMS split tolerance",
            "workload": "ratedist", "unit": "bpp / dB", "higher_is_better": None, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "dtype": "fp16->fp32 (exact int)",
            "data": "synthetic", "config": {"workload": RATEDIST_DESC}, "rows": rows}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--legs", default="tensor,plain,e2e,cpu,batch,serving",
                    help="measurements to run (profiling runs use 'tensor' alone)")
    ap.add_argument("--workload", default="precision512",
                    choices=["precision512", "batch64", "serving", "compare", "graph", "peaks",
                             "ratedist"],
                    help="precision512: the headline line; batch64: the 64-image batching "
                         "form; serving: the request server under a Poisson stream")
    ap.add_argument("--requests", type=int, default=200, help="serving: number of requests")
    ap.add_argument("--no-single", dest="single", action="store_false",
                    help="batch64: skip the one-call-per-image comparison")
    ap.add_argument("--rate", type=float, default=200.0,
                    help="serving: mean arrival rate of the Poisson stream (images/s)")
    ap.add_argument("--policy", type=int, default=0, choices=[0, 1],
                    help="serving: admission order (0 FIFO, 1 smallest image first with aging)")
    ap.add_argument("--tune-mode", type=int, default=1,
                    help="contraction shapes: 0 fixed, 1 measured on first use (default), "
                         "2 + i candidate i (profiling aid: no tuning launches)")
    ap.add_argument("--only-side", type=int, default=0, choices=[0, 16, 8, 4],
                    help="profiling aid: encode one quadtree step at this side (all ranges)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    import __graft_entry__
    __graft_entry__.build()
    if args.workload == "batch64":
        return run_batch(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "compare":
        return run_compare(args)
    if args.workload == "graph":
        return run_graph(args)
    if args.workload == "peaks":
        return run_peaks(args)
    if args.workload == "ratedist":
        return run_ratedist(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
