#!/usr/bin/env python3
"""Benchmark of the B300 single-pulse search hot path.

One step = one full search (downsampling when the plan has it, SB-gather +
dedispersion, statistics, boxcar S/N, threshold + compaction) of one 1.024 s
chunk of synthetic ARTS-shaped data, through the C ABI.  Metric: DM-trial
samples per second (SBs x DM trials x output samples, each range counted at
its own rate), whole job over all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl fdd|reference]

Prints ONE JSON line (rank 0).  --impl reference times the CPU oracle (the
only reference this project has: the paper's AMBER code is not part of it)
on a bounded sample of the same workload.
"""
import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

K_DM = 4148.808  # s MHz^2 / (pc cm^-3), for placing injected pulses only
WIDTHS = [1, 2, 4, 8, 16, 32, 64]

WORKLOADS = {
    # 1 beam, 128 ch, 4096 samples, DM 0-255 step 1, widths 1..16 (the small parity case)
    "tiny": dict(n_tab=1, n_sb=1, n_chan=128, n_out=4096, seed=1, n_pulses=1, pulse_tabs=[0], thr=8.0,
                 ranges=[dict(dm0=0.0, ddm=1.0, n_dm=256, downsamp=1, widths=[1, 2, 4, 8, 16])]),
    # 1 SB, 1536 ch, 1.024 s chunk, DM 0-409.4 step 0.2 (2048 trials), widths 1..64
    "arts_single_sb": dict(n_tab=1, n_sb=1, n_chan=1536, n_out=synth.ARTS_CHUNK, seed=2, n_pulses=10,
                           pulse_tabs=[0], thr=8.0,
                           ranges=[dict(dm0=0.0, ddm=0.2, n_dm=2048, downsamp=1, widths=WIDTHS)]),
    # 12 TABs -> 71 SBs (seeded piecewise-constant SB table), same DM plan
    "arts_71sb": dict(n_tab=12, n_sb=71, n_chan=1536, n_out=synth.ARTS_CHUNK, seed=3, n_pulses=5,
                      pulse_tabs=[0, 3, 5, 8, 11], thr=8.0,
                      ranges=[dict(dm0=0.0, ddm=0.2, n_dm=2048, downsamp=1, widths=WIDTHS)]),
    # 71 SBs from the array geometry (Apertif-10, TABs combined in 48-channel subbands), DM plan as above
    "arts_71sb_geom": dict(n_tab=12, n_sb=71, n_chan=1536, n_out=synth.ARTS_CHUNK, seed=3, n_pulses=5,
                           pulse_tabs=[0, 3, 5, 8, 11], thr=8.0, sb_table="geometry",
                           ranges=[dict(dm0=0.0, ddm=0.2, n_dm=2048, downsamp=1, widths=WIDTHS)]),
    # 71 SBs, DM 0-25.4 (128 trials): a small case of the 71-SB kernels for detailed profiles
    "arts_71sb_128dm": dict(n_tab=12, n_sb=71, n_chan=1536, n_out=synth.ARTS_CHUNK, seed=3, n_pulses=5,
                            pulse_tabs=[0, 3, 5, 8, 11], thr=8.0,
                            ranges=[dict(dm0=0.0, ddm=0.2, n_dm=128, downsamp=1, widths=WIDTHS)]),
    # 71 SBs, 4-range plan 0-5000 with downsampling 1/2/4/8
    "arts_71sb_4range": dict(n_tab=12, n_sb=71, n_chan=1536, n_out=synth.ARTS_CHUNK, seed=4, n_pulses=5,
                             pulse_tabs=[0, 3, 5, 8, 11], thr=8.0,
                             ranges=[dict(dm0=0.0, ddm=0.2, n_dm=2048, downsamp=1, widths=WIDTHS),
                                     dict(dm0=409.6, ddm=0.8, n_dm=1024, downsamp=2, widths=WIDTHS),
                                     dict(dm0=1228.8, ddm=1.6, n_dm=1024, downsamp=4, widths=WIDTHS),
                                     dict(dm0=2867.2, ddm=3.2, n_dm=667, downsamp=8, widths=WIDTHS)]),
}

N_SM = 148
INT_LANES_PER_SM = 128
ADDS_PER_LANE_OP = 2        # one IADD3 adds two operands
SM_MAX_MHZ_NOMINAL = 2032.0
CSRC = os.path.join(ROOT, "paper_2205_12362_b300", "csrc")


# ----------------------------------------------------------------- workload
def arrivals(freqs, dm, t_samp):
    """Per-channel arrival offsets (samples) of a dispersed pulse: the signal model."""
    f_top = freqs.max()
    return np.rint(K_DM * dm * (freqs ** -2 - f_top ** -2) / t_samp).astype(np.int64)


def max_delay_native(freqs, ranges, t_samp):
    out = 0
    for r in ranges:
        dm_last = r["dm0"] + (r["n_dm"] - 1) * r["ddm"]
        d = np.rint(K_DM * dm_last * (freqs.min() ** -2 - freqs.max() ** -2) / (r["downsamp"] * t_samp))
        out = max(out, int(d + 1) * r["downsamp"])
    return out


def make_workload(name, sb_table_fn=None):
    """sb_table_fn(n_tab, n_sb, freqs, chan_per_subband) builds the geometry SB
    table of workloads that ask for one (the library's on the measured arm,
    the oracle's on the reference arm)."""
    w = dict(WORKLOADS[name])
    f = synth.channel_freqs(w["n_chan"])
    t = synth.ARTS_T_SAMP_S
    n_in = w["n_out"] + max_delay_native(f, w["ranges"], t) + 16
    dm_hi = min(400.0, w["ranges"][-1]["dm0"] + w["ranges"][-1]["n_dm"] * w["ranges"][-1]["ddm"])
    dm_lo = min(50.0, 0.5 * dm_hi)
    prm = synth.random_pulses(w["seed"], w["n_pulses"], w["pulse_tabs"], dm_lo, dm_hi, [1, 2, 4, 8, 16, 32],
                              8.0, 50.0, 200, w["n_out"] - 200)
    pulses = [dict(tab=p["tab"], start=p["t0"] + arrivals(f, p["dm"], t), width=p["width"],
                   amp=synth.pulse_amplitude(p["snr"], w["n_chan"], p["width"])) for p in prm]
    x = synth.filterbank(w["seed"], w["n_tab"], w["n_chan"], n_in, pulses=pulses)
    if w["n_tab"] == 1:
        sb = np.zeros((w["n_sb"], w["n_chan"]), np.int16)
    elif w.get("sb_table") == "geometry":
        sb = np.asarray(sb_table_fn(w["n_tab"], w["n_sb"], f, 48), dtype=np.int16)
    else:
        sb = synth.sb_map_piecewise(w["seed"], w["n_sb"], w["n_chan"], w["n_tab"]).astype(np.int16)
    return w, f, t, x, sb, n_in


def units_per_step(w):
    return sum(w["n_sb"] * r["n_dm"] * (w["n_out"] // r["downsamp"]) for r in w["ranges"])


def adds_per_step(w):
    return sum(w["n_sb"] * r["n_dm"] * (w["n_out"] // r["downsamp"]) * w["n_chan"] for r in w["ranges"])


# ----------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        self.t0 = time.time()

    def mark(self):
        return time.time()

    def stop(self, t_lo, t_hi):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        rows = []
        if self.path and os.path.exists(self.path):
            for ln in open(self.path):
                parts = [p.strip() for p in ln.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        # samples are ~100 ms apart from start(); keep those inside [t_lo, t_hi] by position
        n = len(rows)
        span = max(time.time() - self.t0, 1e-3)
        lo = int(max(0, (t_lo - self.t0) / span * n))
        hi = int(min(n, (t_hi - self.t0) / span * n + 1))
        sel = rows[lo:hi] or rows
        sm = [float(r[1]) for r in sel if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in sel if r[2].replace(".", "").isdigit()]
        reasons = set()
        for r in sel:
            for name, val in (("hw_slowdown", r[5]), ("hw_thermal_slowdown", r[6]),
                              ("sw_thermal_slowdown", r[7]), ("sw_power_cap", r[8])):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sel),
                "power_w_max": max(float(r[3]) for r in sel if re.match(r"^[0-9.]+$", r[3])) if any(
                    re.match(r"^[0-9.]+$", r[3]) for r in sel) else None}


# ----------------------------------------------------------------- oracle (CPU baseline)
def oracle_sample_rate(x, sb, f, t, w, n_in, target_s):
    """Time the oracle as it stands on a bounded sample (leading DM trials of
    each range, first SB) and return (samples/s, cores, description)."""
    import oracle
    cores = oracle.get_threads()

    def run(frac):
        rr = [dict(r, n_dm=max(1, int(r["n_dm"] * frac))) for r in w["ranges"]]
        units = sum(r["n_dm"] * (w["n_out"] // r["downsamp"]) for r in rr)
        t0 = time.perf_counter()
        oracle.search(x, sb[:1], f, t, rr, w["thr"], w["n_out"], n_in=n_in)
        return units, time.perf_counter() - t0, rr

    frac = 1.0 / 64
    u, dt, rr = run(frac)
    for _ in range(4):                       # grow the sample toward target_s of CPU work
        if dt >= 0.5 * target_s or frac >= 1.0:
            break
        frac = min(1.0, frac * 0.9 * target_s / max(dt, 1e-3))
        u, dt, rr = run(frac)
    desc = "SB 0 of %d, first %s DM trials of each range (%s), full %d-sample chunk, %d channels" % (
        w["n_sb"], "/".join(str(r["n_dm"]) for r in rr), "/".join(str(r["n_dm"]) for r in w["ranges"]),
        w["n_out"], w["n_chan"])
    return u / dt, cores, desc, dt, rr


# ----------------------------------------------------------------- profile evidence
def profile_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu
    summary profiles/<kernel>_<workload>.md, or None when there is none or the
    kernel source changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "%s_%s.md" % (kernel, workload))
    src = os.path.join(CSRC, kernel + ".cu")
    if not os.path.exists(path) or not os.path.exists(src):
        return None
    text = open(path).read()
    m_sha = re.search(r"source_sha1:\s*([0-9a-f]{40})", text)
    m_b = re.search(r"dram_bytes_per_launch_full:\s*([0-9.eE+]+)", text)
    if not m_sha or not m_b:
        return None
    sha = hashlib.sha1(open(src, "rb").read()).hexdigest()
    return float(m_b.group(1)) if sha == m_sha.group(1) else None


# ----------------------------------------------------------------- arms
def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "fdd" else "gloo"
        if backend == "nccl":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def reduce_max(value, dist, device):
    """Max of a per-rank scalar over all ranks (the job's time is the slowest rank's)."""
    if not dist:
        return value
    import torch
    tt = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def run_fdd(args):
    import torch

    import paper_2205_12362_b300 as fdd

    world, rank, local, dist = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w, f, t, x, sb, n_in = make_workload(
        args.workload, lambda nt, ns, fr, g: fdd.sb_table(nt, ns, fr, chan_per_subband=g))
    mode = args.mode or w.get("mode", "plain")
    plan = fdd.Plan(w["n_tab"], w["n_chan"], w["n_sb"], f, t, w["ranges"], w["thr"], sb)
    if args.scratch_mb:
        plan.set_scratch_limit(args.scratch_mb << 20)
    if args.subband:
        sg, sk = (int(v) for v in args.subband.split(","))
        for r in range(len(w["ranges"])):
            plan.set_subband(r, sg, sk)
        n_in = max(n_in, w["n_out"] + plan.max_delay + 16)
        x = np.ascontiguousarray(np.pad(x, ((0, 0), (0, 0), (0, max(0, synth.padded_pitch(n_in) - x.shape[2])))))
    host = torch.from_numpy(x).pin_memory()
    tabs = host.to(dev)
    cap = 1 << 22
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 126 MB L2
    stream = torch.cuda.current_stream()
    plans = [plan]
    if mode in ("plain", "per_sb"):
        ws = torch.empty(plan.workspace_size(n_in, w["n_out"], with_series=True), dtype=torch.uint8, device=dev)
        cands = torch.empty((cap, 8), dtype=torch.int32, device=dev)
        count = torch.zeros(1, dtype=torch.int64, device=dev)
        if not args.no_autotune:
            plan.autotune(tabs, n_in, w["n_out"], reps=3, workspace=ws, stream=stream)
        if args.variant is not None:
            for r in range(len(w["ranges"])):
                try:
                    plan.set_config(r, args.variant, args.cc)
                except fdd.FddError:
                    pass  # variant for the other sample width
        if mode == "per_sb":
            # the plain per-beam path: one single-SB plan per SB, searched one after another, each
            # with the configuration tuned for a single-SB plan
            plans = []
            for s_i in range(w["n_sb"]):
                plans.append(fdd.Plan(w["n_tab"], w["n_chan"], 1, f, t, w["ranges"], w["thr"], sb[s_i:s_i + 1]))
            ws = torch.empty(plans[0].workspace_size(n_in, w["n_out"], with_series=True), dtype=torch.uint8,
                             device=dev)
            if not args.no_autotune:
                plans[0].autotune(tabs, n_in, w["n_out"], reps=3, workspace=ws, stream=stream)
            cfgs = [plans[0].get_config(r) for r in range(len(w["ranges"]))]
            for p1 in plans[1:]:
                for r, c in enumerate(cfgs):
                    p1.set_config(r, c["variant"], c["chan_per_stage"])
        for p_ in plans:
            p_.set_timing(True)

        def step(src=None, out=None):
            c_, n_ = (cands, count) if out is None else out
            for p_ in plans:
                p_.search(tabs if src is None else src, n_in, w["n_out"], cap=cap, workspace=ws, cands=c_,
                          count=n_, stream=stream)
    else:
        job = plan.make_job(tabs, n_in, w["n_out"], cap=cap)
        cands, count = job.cands, job.count
        plan.batch_prepare(w["n_out"])
        if not args.no_autotune:
            plan.batch_autotune([job], w["n_out"], reps=2, stream=stream)
        plan.set_timing(True)
        if mode == "graph":
            graph = fdd.Graph(plan, [job], w["n_out"])

            def step():
                graph.launch(stream)
        else:
            def step():
                plan.search_batch([job], w["n_out"], stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_lo = time.time()
    step_ms, stage_ms, launches = [], {}, 0
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    wall0 = time.perf_counter()
    torch.cuda.nvtx.range_push("timed")
    for _ in range(args.steps):
        flush.zero_()                      # evict the input from L2 between steps
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        per_step = {}
        for p_ in (plans if mode != "graph" else []):
            st = p_.stage_times()
            launches += p_.last_launches()
            for name, r, ms in st:
                key = "%s[%d]" % (name, r)
                per_step[key] = per_step.get(key, 0.0) + ms
        for key, ms in per_step.items():
            stage_ms.setdefault(key, []).append(ms)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    wall1 = time.perf_counter()
    if mode == "graph":
        # graphs carry no stage events: the kernels' own times come from the
        # same batched launches run directly, right after the timed loop
        launches = 0
        for k in range(min(args.steps, 20)):
            flush.zero_()
            plan.search_batch([job], w["n_out"], stream=stream)
            stream.synchronize()
            if k == 0:
                launches = plan.last_launches() * args.steps   # the graph replays these kernels
            for name, r, ms in plan.stage_times():
                stage_ms.setdefault("%s[%d]" % (name, r), []).append(ms)
    if dist:
        dist.barrier()
    t_hi = time.time()
    clocks = sampler.stop(t_lo, t_hi)
    for p_ in plans:
        if p_.status() != 0:               # a tile-copy wait gave up: the timed output is incomplete
            raise RuntimeError("device status word set (FDD_STATUS_TILE_WAIT): the measurement is void")

    dev_s = reduce_max(sum(step_ms) / 1e3, dist, dev)
    units = units_per_step(w) * args.steps * world
    value = units / dev_s

    # end-to-end through the public API with host buffers: every step copies its
    # chunk host-to-device from pinned memory and reads its count and candidate
    # records back.  Per-range modes double-buffer the input and the outputs, as a
    # pipelined caller would: the copy of step k+1 (copy stream) overlaps the search
    # of step k, and step k-1's results are read back (their own stream) while step
    # k runs; batched/graph modes search a fixed job buffer, copied in turn.
    e2e_units, h2d, d2h = 0, 0, 0
    e2e_steps = max(1, min(args.steps, 200))
    pipelined = mode in ("plain", "per_sb")
    bufs = [tabs, torch.empty_like(tabs)] if pipelined else [tabs]
    outs = [(cands, count), (torch.empty_like(cands), torch.zeros_like(count))] if pipelined else [(cands, count)]
    cnt_host = [torch.zeros(1, dtype=torch.int64).pin_memory() for _ in outs]
    cnt_ev = [torch.cuda.Event() for _ in outs]
    copy_stream = torch.cuda.Stream(device=dev)
    d2h_stream = torch.cuda.Stream(device=dev)
    ready = [torch.cuda.Event() for _ in bufs]
    done = [torch.cuda.Event() for _ in bufs]
    torch.cuda.synchronize()
    te0 = time.perf_counter()

    def issue_copy(k):
        b = k % len(bufs)
        with torch.cuda.stream(copy_stream):
            if k >= len(bufs):
                copy_stream.wait_event(done[b])       # the buffer's previous search has finished
            bufs[b].copy_(host, non_blocking=True)
            ready[b].record(copy_stream)

    def read_back(b):
        """Host copy of the count and candidates of the step that wrote outs[b]."""
        cnt_ev[b].synchronize()
        n = min(int(cnt_host[b].item()), cap)
        with torch.cuda.stream(d2h_stream):
            d2h_stream.wait_event(done[b])
            got = outs[b][0][:n].to("cpu")            # waits for this copy only
        return 8 + got.numel() * 4

    issue_copy(0)
    pending = None
    for k in range(e2e_steps):
        b = k % len(bufs)
        if pipelined and k + 1 < e2e_steps:
            issue_copy(k + 1)
        stream.wait_event(ready[b])
        if pipelined:
            step(bufs[b], outs[b])
        else:
            step()
        done[b].record(stream)
        cnt_host[b].copy_(outs[b][1], non_blocking=True)
        cnt_ev[b].record(stream)
        if pipelined:
            if pending is not None:
                d2h += read_back(pending)              # step k-1, while step k runs
            pending = b
        else:
            d2h += read_back(b)
            if k + 1 < e2e_steps:
                issue_copy(k + 1)
        h2d += host.numel()
        e2e_units += units_per_step(w)
    if pending is not None:
        d2h += read_back(pending)
    torch.cuda.synchronize()
    te1 = time.perf_counter()
    e2e_s = reduce_max(te1 - te0, dist, dev)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return None

    # roofline of the dominant kernel (dedispersion): channel-adds per launch
    ded = [v for k, v in stage_ms.items() if k.startswith("dedisperse")]
    ded_ms_step = float(sum(np.mean(v) for v in ded)) if ded else None   # all dedispersion work of a step
    n_ded_launches = len(ded) * len(plans)
    ded_ms = ded_ms_step / max(1, n_ded_launches) if ded else None
    adds_launch = adds_per_step(w) / max(1, n_ded_launches)
    sm_mhz = clocks.get("sm_mhz")
    peak = N_SM * INT_LANES_PER_SM * ADDS_PER_LANE_OP * SM_MAX_MHZ_NOMINAL * 1e6 / 1e12
    achieved = adds_launch / (ded_ms / 1e3) / 1e12 if ded_ms else None
    cfgs = [plan.get_config(r) for r in range(len(w["ranges"]))] if mode in ("plain", "per_sb") else []
    kinds = {v["index"]: v["kind"] for v in fdd.variants()}
    kind_names = {0: "k_dedisp", 1: "k_dedisp_fact", 2: "k_sbf"}
    if mode in ("batched", "graph"):
        sbf_batch = plan.batch_config()["variant"] == fdd.FDD_BATCH_SB_FACTORED
        kname = "k_sbf" if sbf_batch else "k_batch"
        if sbf_batch:
            cfgs = [plan.get_config(r) for r in range(len(w["ranges"]))]
    else:
        kname = kind_names[kinds[cfgs[0]["variant"]]] if cfgs else "k_dedisp"
    ratio = float(np.mean([c["work_ratio"] for c in cfgs])) if cfgs else 1.0
    if args.subband:
        # approximate two-step mode: step 1 (k_sbf_part over each coarse DM's subbands) + step 2
        # (k_dedisp over the subband rows); adds per (trial, sample) against the exact method's n_chan
        sg, sk = (int(v) for v in args.subband.split(","))
        kname = "k_sbf_part+k_dedisp (two-step subband, approximate)"
        n_chan = w["n_chan"]
        ratio = (n_chan / sk + -(-n_chan // sg)) / n_chan
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tadd/s",
            "frac": (achieved / peak) if achieved else None, "traffic": profile_traffic(kname, args.workload),
            "kernel": kname, "units_per_launch": adds_launch,
            "method_adds_per_launch": adds_launch * ratio,
            "method_note": "achieved counts brute-force channel-adds; the configured kernel performs "
                           "method_adds_per_launch integer adds (the pattern-factored kernel reuses partial sums "
                           "across DM trials, the SB-factored kernels (k_sbf_part + k_sbf_comb) reuse TAB x "
                           "segment partial sums across SBs" + (
                               "; the two-step subband mode is approximate: it does not compute the exact "
                               "sums, so its brute-force-equivalent rate is not comparable" if args.subband
                               else "") + ")",
            "peak_basis": "148 SM x 128 INT32 lanes x 2 adds/IADD3 x 2032 MHz (derived; no measured INT peak)",
            "peak_at_sampled_clock": (peak * sm_mhz / SM_MAX_MHZ_NOMINAL) if sm_mhz else None,
            "avg_launch_ms": ded_ms}

    cpu = None
    if not args.no_cpu_baseline:
        rate, cores, desc, secs, _ = oracle_sample_rate(x, sb, f, t, w, n_in, args.cpu_seconds)
        cpu = {"value": rate, "unit": "samples/s", "cores": cores, "kind": "oracle", "sample": desc,
               "seconds": secs}
        if w["n_sb"] == 1:
            # the same oracle on one host thread, on a smaller sample of the same workload
            import oracle
            oracle.set_threads(1)
            try:
                rate1, _, desc1, secs1, _ = oracle_sample_rate(x, sb, f, t, w, n_in, max(1.0, args.cpu_seconds / 4))
            finally:
                oracle.set_threads(cores)
            cpu["single_thread"] = {"value": rate1, "unit": "samples/s", "cores": 1, "sample": desc1,
                                    "seconds": secs1}

    line = {
        "metric": "DM-trial samples/s (beams x DMs x samples)",
        "value": value,
        "unit": "samples/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": sum(step_ms) / len(step_ms),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u8",
        "data": "synthetic",
        "config": {"workload": args.workload, "n_tab": w["n_tab"], "n_sb": w["n_sb"], "n_chan": w["n_chan"],
                   "n_out": w["n_out"], "n_in": n_in,
                   "dm_plan": [[r["dm0"], r["ddm"], r["n_dm"], r["downsamp"]] for r in w["ranges"]],
                   "widths": WIDTHS, "snr_thresh": w["thr"], "l2": "flushed (256 MB write) between steps",
                   "parallelism": "replicas" if world > 1 else "single", "mode": mode,
                   "dedispersion": ("two-step subband %s (approximate)" % args.subband) if args.subband
                   else "exact"},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_units * world / e2e_s, "unit": "samples/s",
                "h2d_bytes_per_step": h2d / e2e_steps, "d2h_bytes_per_step": d2h / e2e_steps,
                "steps": e2e_steps, "h2d_overlapped": pipelined},
        "gpu_launches": launches,
        "clocks": clocks,
        "stages_ms": {k: float(np.mean(v)) for k, v in stage_ms.items()},
        "kernel_config": ([plan.get_config(r) for r in range(len(w["ranges"]))] if mode in ("plain", "per_sb")
                          else plan.batch_config()),
        "wall_s": wall1 - wall0,
    }
    if dist:
        dist.destroy_process_group()
    return line


def run_reference(args):
    world, rank, local, dist = dist_setup(args)
    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return None
    import oracle
    w, f, t, x, sb, n_in = make_workload(
        args.workload, lambda nt, ns, fr, g: oracle.sb_table(nt, ns, fr, 1500.0, 0.80, 1296.0, 144.0, g))
    per_step = max(0.05, min(args.cpu_seconds, 150.0 / max(1, args.steps + args.warmup)))
    _, cores, desc, _, rr = oracle_sample_rate(x, sb, f, t, w, n_in, per_step)
    units = sum(r["n_dm"] * (w["n_out"] // r["downsamp"]) for r in rr)
    for _ in range(args.warmup):
        oracle.search(x, sb[:1], f, t, rr, w["thr"], w["n_out"], n_in=n_in)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.search(x, sb[:1], f, t, rr, w["thr"], w["n_out"], n_in=n_in)
    dt = time.perf_counter() - t0
    value = units * args.steps / dt
    line = {
        "impl": "reference",
        "metric": "DM-trial samples/s (beams x DMs x samples)",
        "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / max(1, args.steps) * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64/f64", "data": "synthetic",
        "config": {"workload": args.workload, "n_tab": w["n_tab"], "n_sb": w["n_sb"], "n_chan": w["n_chan"],
                   "n_out": w["n_out"], "n_in": n_in,
                   "dm_plan": [[r["dm0"], r["ddm"], r["n_dm"], r["downsamp"]] for r in w["ranges"]],
                   "widths": WIDTHS, "snr_thresh": w["thr"]},
        "cpu_baseline": {"value": value, "unit": "samples/s", "cores": cores, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return line


def run_serve(args):
    """Serving measurement: N beams deliver 1.024 s chunks at real-time cadence
    (seeded +-50 ms jitter) into the library's serving runtime; per window
    latency = results seen - arrival of the chunk that completed the window."""
    import torch

    import paper_2205_12362_b300 as fdd
    torch.cuda.set_device(0)
    w = dict(WORKLOADS[args.workload])
    f = synth.channel_freqs(w["n_chan"])
    t = synth.ARTS_T_SAMP_S
    chunk = w["n_out"]
    rng = np.random.Generator(np.random.Philox(w["seed"] + 55))
    # a pinned pool of pre-generated chunks (noise + injected pulses whose whole sweep lies inside the
    # chunk, so the window starting with a chunk holds its pulses whatever the chunk order)
    n_pool = args.pool
    pool, pool_pulses = [], []
    sweep = int(arrivals(f, 400.0, t).max())
    sb = synth.sb_map_piecewise(w["seed"], w["n_sb"], w["n_chan"], w["n_tab"]).astype(np.int16)
    for k in range(n_pool):
        # sources at seeded SB positions: each pulse goes into the TAB its SB takes in every channel
        prm = synth.random_pulses(w["seed"] * 100 + k, 2, list(range(w["n_sb"])), 50.0, 400.0, [1, 2, 4, 8],
                                  15.0, 40.0, 200, chunk - sweep - 200)
        pulses = []
        for p_ in prm:
            pulses += synth.sb_pulses(sb[p_["tab"]], p_["t0"] + arrivals(f, p_["dm"], t), p_["width"],
                                      synth.pulse_amplitude(p_["snr"], w["n_chan"], p_["width"]))
        x = synth.filterbank(w["seed"] * 1000 + k, w["n_tab"], w["n_chan"], chunk, pitch=chunk, pulses=pulses)
        pool.append(torch.from_numpy(x).pin_memory())
        pool_pulses.append(prm)
    plan = fdd.Plan(w["n_tab"], w["n_chan"], w["n_sb"], f, t, w["ranges"], w["thr"], sb)
    # tune the batched search on one window
    n_in = chunk + plan.max_delay
    win = torch.zeros((w["n_tab"], w["n_chan"], synth.padded_pitch(n_in)), dtype=torch.uint8, device="cuda")
    job = plan.make_job(win, n_in, chunk, cap=1 << 15)
    plan.batch_prepare(chunk)
    if not args.no_autotune:
        plan.batch_autotune([job], chunk, reps=1)
    del job, win
    torch.cuda.empty_cache()
    out = {"metric": "p99 chunk latency (s) at real-time cadence", "unit": "s", "higher_is_better": False,
           "data": "synthetic", "config": {"workload": args.workload, "chunk_s": chunk * t, "jitter_ms": 50,
                                           "pool_chunks": n_pool, "stream_s": args.seconds},
           "batch_config": plan.batch_config(), "runs": []}
    for n_beams in [int(v) for v in args.beams.split(",")]:
        srv = fdd.Server(plan, n_beams, chunk, cap_per_window=1 << 15)
        info = srv.info()
        n_chunks = int(args.seconds / 1.024)
        jitter = rng.uniform(-0.05, 0.05, size=(n_beams, n_chunks))
        t0 = fdd.now() + 0.5
        arrive = t0 + np.arange(n_chunks)[None, :] * 1.024 + jitter
        nxt = np.zeros(n_beams, dtype=np.int64)
        busy = 0
        while (nxt < n_chunks).any():
            now = fdd.now()
            progressed = False
            for b in range(n_beams):
                k = int(nxt[b])
                if k < n_chunks and arrive[b, k] <= now:
                    code = srv.push(b, k, pool[(k + 3 * b) % n_pool], t_arrival=float(arrive[b, k]))
                    if code == 0:
                        nxt[b] += 1
                        progressed = True
                    else:
                        busy += 1
            srv.poll()
            if not progressed:
                time.sleep(0.001)
        srv.drain()
        res = srv.results(max_results=n_beams * n_chunks + 8)
        lat = np.array([r["t_done"] - r["t_arrival"] for r, _ in res])
        gpu = np.array([r["t_done"] - r["t_launch"] for r, _ in res])
        wait = np.array([r["t_launch"] - r["t_ready"] for r, _ in res])
        span = max(r["t_done"] for r, _ in res) - min(r["t_launch"] for r, _ in res) if res else 1.0
        st = srv.info()
        # injected-pulse recall: window w of beam b starts with chunk w, whose pulses it must hold
        injected = recovered = 0
        for r, c in res:
            for p_ in pool_pulses[(int(r["window"]) + 3 * int(r["beam"])) % n_pool]:
                injected += 1
                t_abs = int(r["window"]) * chunk + p_["t0"]
                near = ((c["sb"] == p_["tab"]) & (np.abs(c["dm"] - p_["dm"]) < 0.02 * p_["dm"] + 2.0)
                        & (np.abs(c["t_native"] - t_abs) < 4 * p_["width"] + 64))
                recovered += int(near.any())
        p99 = float(np.percentile(lat, 99)) if len(lat) else None
        run = {"beams": n_beams, "windows": len(res), "p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
               "p99_s": p99, "max_s": float(lat.max()) if len(lat) else None,
               "p50_gpu_s": float(np.percentile(gpu, 50)) if len(gpu) else None,
               "p50_wait_s": float(np.percentile(wait, 50)) if len(wait) else None,
               "sustained": bool(p99 is not None and p99 < 1.024),
               "busy_retries": busy, "slots": st["n_slots"], "max_queued": st["max_queued"],
               "batches": st["batches"], "mean_batch": st["done"] / max(1, st["batches"]),
               "windows_per_s": len(res) / span,
               "dm_trial_samples_per_s": len(res) * units_per_step(w) / span,
               "ring_gb_per_beam": info["ring_bytes_per_beam"] / 1e9, "slot_gb": info["slot_bytes"] / 1e9,
               "candidates": int(sum(len(c) for _, c in res)),
               "injected_pulses": injected, "recovered_pulses": recovered,
               "recall": recovered / injected if injected else None}
        out["runs"].append(run)
        print(json.dumps(run), file=sys.stderr, flush=True)
        srv.close()
        torch.cuda.empty_cache()
    ok = [r["beams"] for r in out["runs"] if r["sustained"]]
    out["max_sustained_beams"] = max(ok) if ok else 0
    best = [r for r in out["runs"] if r["beams"] == out["max_sustained_beams"]]
    out["value"] = best[0]["p99_s"] if best else None
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--workload", default="arts_single_sb", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="fdd", choices=["fdd", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--variant", type=int, default=None, help="force this dedispersion kernel variant")
    ap.add_argument("--cc", type=int, default=0, help="with --variant: channels per stage (0 = largest fitting)")
    ap.add_argument("--subband", default=None,
                    help="G,K: approximate two-step subband dedispersion (G channels per subband, K fine trials per "
                         "coarse DM) instead of the exact kernels; not the benchmark's default")
    ap.add_argument("--scratch-mb", type=int, default=0,
                    help="cap on the SB-factored kernel's partial-sum scratch (0 = library default)")
    ap.add_argument("--serve", action="store_true", help="serving measurement instead of the step benchmark")
    ap.add_argument("--beams", default="1,2,3,4,8", help="--serve: compound-beam counts to run")
    ap.add_argument("--seconds", type=float, default=20.0, help="--serve: stream length per run")
    ap.add_argument("--pool", type=int, default=6, help="--serve: pre-generated chunks in the pinned pool")
    ap.add_argument("--mode", default=None, choices=["plain", "per_sb", "batched", "graph"],
                    help="plain: per-range launches over all SBs; per_sb: one plan per SB (the plain per-beam "
                         "path); batched: one persistent launch over everything; graph: the batched search "
                         "replayed from a CUDA graph (default: the workload's own)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.serve:
        if args.workload == "arts_single_sb" and not any(a.startswith("--workload") for a in sys.argv):
            args.workload = "arts_71sb_4range"
        line = run_serve(args)
    else:
        line = run_fdd(args) if args.impl == "fdd" else run_reference(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
