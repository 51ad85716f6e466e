#!/usr/bin/env python3
"""Benchmark of the B300 single-pulse search hot path.

One step = one full search (downsampling, SB-gather + dedispersion,
statistics, boxcar S/N, threshold + compaction) of one 1.024 s chunk of one
compound beam of synthetic ARTS-shaped data, through the C ABI.  Metric:
DM-trial samples per second (SBs x DM trials x output samples, each range
counted at its own rate), whole job over all ranks.

Default workload: 12 TABs -> 71 SBs, the four-range DM plan 0-5000 (D = 1, 2,
4, 8), batched search replayed from a CUDA graph.  The same JSON line also
carries: the measured integer-add / permute / shared-memory peaks (issue-rate
probe, the roofline denominators), the roofline of the dedispersion stage on
brute-force-equivalent and on performed adds, an end-to-end figure with the
new 1.024 s chunk copied host-to-device each step (the beam's delay overlap
stays on the device, as in streaming), the plain per-SB path on the same GPU,
serving (p50/p99 chunk latency at real-time cadence for 8 beams, for the count
the measured step time suggests and for one more; the largest sustained count
is reported next to the plain per-SB path at that count) and the oracle on the
host cores.

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
    # the 71-SB four-range plan with 1/16 of each range's DM trials: a small case of the same kernels
    # and launch structure for detailed profiles (traffic per trial as in the full plan)
    "arts_71sb_4range_16th": dict(n_tab=12, n_sb=71, n_chan=1536, n_out=synth.ARTS_CHUNK, seed=4, n_pulses=5,
                                  pulse_tabs=[0, 3, 5, 8, 11], thr=8.0, mode="graph",
                                  ranges=[dict(dm0=0.0, ddm=0.2, n_dm=128, downsamp=1, widths=WIDTHS),
                                          dict(dm0=409.6, ddm=0.8, n_dm=64, downsamp=2, widths=WIDTHS),
                                          dict(dm0=1228.8, ddm=1.6, n_dm=64, downsamp=4, widths=WIDTHS),
                                          dict(dm0=2867.2, ddm=3.2, n_dm=42, downsamp=8, widths=WIDTHS)]),
    # 71 SBs, 4-range plan 0-5000 with downsampling 1/2/4/8
    "arts_71sb_4range": dict(n_tab=12, n_sb=71, n_chan=1536, n_out=synth.ARTS_CHUNK, seed=4, n_pulses=5,
                             pulse_tabs=[0, 3, 5, 8, 11], thr=8.0, mode="graph",
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
    """Time the oracle as it stands on a bounded sample of the workload: the
    leading DM trials of each range of the first SB, grown toward target_s of
    CPU work (all trials first, then more SBs).  Returns (samples/s, cores,
    description, seconds, ranges of the sample, SBs of the sample)."""
    import oracle
    cores = oracle.get_threads()

    def run(frac, n_sb):
        rr = [dict(r, n_dm=max(1, int(round(r["n_dm"] * frac)))) for r in w["ranges"]]
        units = n_sb * sum(r["n_dm"] * (w["n_out"] // r["downsamp"]) for r in rr)
        t0 = time.perf_counter()
        oracle.search(x, sb[:n_sb], f, t, rr, w["thr"], w["n_out"], n_in=n_in)
        return units, time.perf_counter() - t0, rr

    frac, n_sb = 1.0 / 16, 1
    u, dt, rr = run(frac, n_sb)
    for _ in range(6):                       # grow the sample toward target_s of CPU work
        if dt >= 0.5 * target_s:
            break
        grow = 0.9 * target_s / max(dt, 1e-3)
        if frac < 1.0:
            frac = min(1.0, frac * grow)
        elif n_sb < w["n_sb"]:
            n_sb = max(n_sb + 1, min(w["n_sb"], int(n_sb * grow)))
        else:
            break
        u, dt, rr = run(frac, n_sb)
    desc = "SBs 0-%d of %d, first %s DM trials of each range (%s), full %d-sample chunk, %d channels" % (
        n_sb - 1, w["n_sb"], "/".join(str(r["n_dm"]) for r in rr), "/".join(str(r["n_dm"]) for r in w["ranges"]),
        w["n_out"], w["n_chan"])
    return u / dt, cores, desc, dt, rr, n_sb


# ----------------------------------------------------------------- profile evidence
def profile_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu
    summary profiles/<kernel>_<workload>.md, or None when there is none or a
    source file it names changed since the counters were taken (the summary's
    source_sha1 is the SHA-1 of its source_files, concatenated in order)."""
    path = os.path.join(ROOT, "profiles", "%s_%s.md" % (kernel, workload))
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_sha = re.search(r"source_sha1:\s*([0-9a-f]{40})", text)
    m_b = re.search(r"dram_bytes_per_launch_full:\s*([0-9.eE+]+)", text)
    m_f = re.search(r"source_files:\s*(.+)", text)
    if not m_sha or not m_b:
        return None
    files = m_f.group(1).split() if m_f else [kernel + ".cu"]
    h = hashlib.sha1()
    for name in files:
        src = os.path.join(CSRC, name)
        if not os.path.exists(src):
            return None
        h.update(open(src, "rb").read())
    return float(m_b.group(1)) if h.hexdigest() == m_sha.group(1) else None


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


def measure_int_peaks(fdd, gpu_index, target_s=0.25):
    """Issue-rate probes (include/fdd.h: fdd_probe_issue_rate) at full
    occupancy, timed with CUDA events, with nvidia-smi clocks sampled while
    they run: integer adds/s on the ALU pipe (three-input adds), on the FMA
    pipe (multiply-adds) and on both together (the roofline peak of the
    dedispersion kernels), ALU-pipe permutes/s and shared-memory bytes/s."""
    sampler = ClockSampler(gpu_index)
    sampler.start()
    time.sleep(0.25)
    t_lo = time.time()
    out = {}
    for kind, name in ((0, "add"), (1, "prmt"), (2, "lds"), (3, "imad"), (4, "mix")):
        r = fdd.probe_issue_rate(kind, 8, 1 << 12)            # calibrate the iteration count
        iters = int(min(1 << 30, max(1 << 12, (1 << 12) * target_s * 1e3 / max(r["ms"], 1e-3))))
        r = fdd.probe_issue_rate(kind, 8, iters)
        out[name] = dict(per_second=r["per_second"], ms=r["ms"], iters=iters, n_sm=r["n_sm"])
    clocks = sampler.stop(t_lo, time.time())
    mhz = clocks.get("sm_mhz") or SM_MAX_MHZ_NOMINAL
    n_sm = out["add"]["n_sm"]
    per_clk = lambda v: v / (n_sm * mhz * 1e6)
    best = max(out["add"]["per_second"], out["mix"]["per_second"])
    return {
        "adds_per_s": best,
        "adds_per_s_basis": "the larger of three-input adds alone and interleaved with multiply-adds",
        "iadd3_adds_per_s": out["add"]["per_second"],
        "iadd3_thread_instr_per_sm_per_clk": per_clk(out["add"]["per_second"]) / 2.0,
        "imad_per_s": out["imad"]["per_second"],
        "imad_thread_instr_per_sm_per_clk": per_clk(out["imad"]["per_second"]),
        "mixed_adds_per_s": out["mix"]["per_second"],
        "prmt_per_s": out["prmt"]["per_second"],
        "prmt_thread_instr_per_sm_per_clk": per_clk(out["prmt"]["per_second"]),
        "lds_bytes_per_s": out["lds"]["per_second"],
        "lds_bytes_per_sm_per_clk": per_clk(out["lds"]["per_second"]),
        "sm_mhz": clocks.get("sm_mhz"), "clock_reasons": clocks.get("reasons"),
        "config": "%d SMs x 8 blocks x 256 threads, 16 independent chains per thread, CUDA events" % n_sm,
        "ms": {k: v["ms"] for k, v in out.items()},
    }


def range_variant(spec, r):
    """--variant: one variant for every range, or a comma-separated one per range."""
    vals = [int(v) for v in str(spec).split(",")]
    return vals[r] if r < len(vals) else vals[-1]


class Arm:
    """One way of running the search of a workload on the device: `step()`
    searches the resident chunk; `search(b)` searches window buffer b into
    its own outputs (end-to-end loop); `stage_pass(k)` runs k searches with
    the library's per-stage events on and returns (stage ms lists, kernels
    per step)."""

    def __init__(self, fdd, args, w, f, t, sb, wins, n_in, cap, stream):
        import torch
        self.fdd, self.w, self.stream, self.n_in, self.cap = fdd, w, stream, n_in, cap
        self.mode = args.mode or w.get("mode", "plain")
        self.wins = wins
        n_out = w["n_out"]
        self.n_out = n_out
        plan = fdd.Plan(w["n_tab"], w["n_chan"], w["n_sb"], f, t, w["ranges"], w["thr"], sb)
        if args.scratch_mb:
            plan.set_scratch_limit(args.scratch_mb << 20)
        if getattr(args, "subband", None):
            sg, sk = (int(v) for v in args.subband.split(","))
            for r in range(len(w["ranges"])):
                plan.set_subband(r, sg, sk)
        self.plan = plan
        self.plans = [plan]
        dev = wins[0].device
        if self.mode in ("plain", "per_sb"):
            if self.mode == "per_sb":
                # the plain per-beam path: one single-SB plan per SB, searched one after another, each with
                # the configuration tuned for a single-SB plan
                self.plans = [fdd.Plan(w["n_tab"], w["n_chan"], 1, f, t, w["ranges"], w["thr"], sb[s:s + 1])
                              for s in range(w["n_sb"])]
            p0 = self.plans[0]
            self.ws = torch.empty(p0.workspace_size(n_in, n_out, with_series=True), dtype=torch.uint8, device=dev)
            if not args.no_autotune:
                p0.autotune(wins[0], n_in, n_out, reps=2 if self.mode == "per_sb" else 3, workspace=self.ws,
                            stream=stream)
            if args.variant is not None:
                for r in range(len(w["ranges"])):
                    try:
                        p0.set_config(r, range_variant(args.variant, r), range_variant(args.cc, r))
                    except fdd.FddError:
                        pass  # variant for the other sample width
            cfgs = [p0.get_config(r) for r in range(len(w["ranges"]))]
            for p1 in self.plans[1:]:
                for r, c in enumerate(cfgs):
                    p1.set_config(r, c["variant"], c["chan_per_stage"])
            ncap = cap if self.mode == "plain" else min(cap, 1 << 16)
            self.outs = [[(torch.empty((ncap, 8), dtype=torch.int32, device=dev),
                           torch.zeros(1, dtype=torch.int64, device=dev)) for _ in self.plans] for _ in wins]
        else:
            self.jobs = [plan.make_job(wb, n_in, n_out, cap=cap) for wb in wins]
            if args.variant is not None:  # per-range kernel of the SB-factored batch mode
                for r in range(len(w["ranges"])):
                    try:
                        plan.set_config(r, range_variant(args.variant, r), range_variant(args.cc, r))
                    except fdd.FddError:
                        pass  # variant for the other sample width
            plan.batch_prepare(n_out, args.batch_variant if args.batch_variant is not None else -1)
            if not args.no_autotune and args.batch_variant is None:
                plan.batch_autotune(self.jobs[:1], n_out, reps=2, stream=stream)
            self.graphs = [fdd.Graph(plan, [j], n_out) for j in self.jobs] if self.mode == "graph" else None
            self.outs = [[(j.cands, j.count)] for j in self.jobs]
        for p_ in self.plans:
            p_.set_timing(False)

    def search(self, b):
        if self.mode in ("plain", "per_sb"):
            for p_, (c_, n_) in zip(self.plans, self.outs[b]):
                p_.search(self.wins[b], self.n_in, self.n_out, cap=int(c_.shape[0]), workspace=self.ws, cands=c_,
                          count=n_, stream=self.stream)
        elif self.mode == "graph":
            self.graphs[b].launch(self.stream)
        else:
            self.plan.search_batch([self.jobs[b]], self.n_out, stream=self.stream)

    def step(self):
        self.search(0)

    def stage_pass(self, k, flush):
        """Per-stage times from the library's own event pairs, outside the
        timed region (graphs carry no stage events: the batched launches they
        replay are run directly)."""
        for p_ in self.plans:
            p_.set_timing(True)
        stage_ms, launches = {}, 0
        for it in range(k):
            flush.zero_()
            if self.mode in ("plain", "per_sb"):
                self.search(0)
            else:
                self.plan.search_batch([self.jobs[0]], self.n_out, stream=self.stream)
            self.stream.synchronize()
            per_step, n_l = {}, 0
            for p_ in self.plans:
                n_l += p_.last_launches()
                for name, r, ms in p_.stage_times():
                    key = "%s[%d]" % (name, r)
                    per_step[key] = per_step.get(key, 0.0) + ms
            for key, ms in per_step.items():
                stage_ms.setdefault(key, []).append(ms)
            launches = n_l
        for p_ in self.plans:
            p_.set_timing(False)
        return stage_ms, launches

    def configs(self):
        if self.mode in ("plain", "per_sb"):
            return [self.plans[0].get_config(r) for r in range(len(self.w["ranges"]))]
        return [self.plan.get_config(r) for r in range(len(self.w["ranges"]))]

    def close(self):
        for g in (self.graphs or []) if self.mode == "graph" else []:
            g.close()


def timed_steps(arm, steps, flush, dist):
    """Time `steps` searches of the resident chunk: CUDA events on the
    launching stream around each step, an L2-flushing write between steps,
    a barrier and a synchronize on both sides.  Returns per-step ms."""
    import torch
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    out = []
    torch.cuda.nvtx.range_push("timed")    # the range a profiler's launch list is restricted to
    for _ in range(steps):
        flush.zero_()                      # evict the input from L2 between steps
        e0.record(arm.stream)
        arm.step()
        e1.record(arm.stream)
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    return out


def e2e_streaming(arm, host_chunk, steps):
    """End to end through the public API, as a real-time caller streams one
    compound beam: every step copies the new 1.024 s chunk host-to-device
    (pinned) into a window buffer whose head (the delay overlap) is the
    previous window's tail (device-to-device), searches it, and reads the
    count and candidate records back.  Two window buffers alternate: the
    copies of step k+1 and the read-back of step k-1 overlap the search of
    step k.  Returns (seconds, h2d bytes, d2h bytes)."""
    import torch
    wins, L, n_in, stream = arm.wins, arm.n_out, arm.n_in, arm.stream
    keep = n_in - L
    pitch = int(wins[0].shape[-1])
    rows = int(wins[0].shape[0] * wins[0].shape[1])
    assert tuple(host_chunk.shape) == (wins[0].shape[0], wins[0].shape[1], L) and host_chunk.is_contiguous()
    copy_stream = torch.cuda.Stream(device=wins[0].device)
    ready = [torch.cuda.Event() for _ in wins]
    done = [torch.cuda.Event() for _ in wins]
    cnt_host = [[torch.zeros(1, dtype=torch.int64).pin_memory() for _ in arm.outs[b]] for b in range(len(wins))]
    cnt_ev = [torch.cuda.Event() for _ in wins]
    h2d = d2h = 0

    def read_back(b):
        cnt_ev[b].synchronize()
        nb = 0
        for (c_, n_), h in zip(arm.outs[b], cnt_host[b]):
            n = min(int(h.item()), int(c_.shape[0]))
            if n:
                nb += c_[:n].to("cpu").numel() * 4
            nb += 8
        return nb

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pending = None
    for k in range(steps):
        b, o = k % 2, 1 - k % 2
        with torch.cuda.stream(copy_stream):
            if k >= 2:
                copy_stream.wait_event(done[b])          # search k-2 has finished reading buffer b
            # 2-D copies on a copy engine: the overlap carried on, then the new chunk from host memory
            arm.fdd.copy_rows(wins[b], 0, pitch, wins[o], L, pitch, keep, rows, stream=copy_stream)
            arm.fdd.copy_rows(wins[b], keep, pitch, host_chunk, 0, L, L, rows, stream=copy_stream)
            ready[b].record(copy_stream)
        h2d += host_chunk.numel()
        stream.wait_event(ready[b])
        arm.search(b)
        done[b].record(stream)
        for (c_, n_), h in zip(arm.outs[b], cnt_host[b]):
            h.copy_(n_, non_blocking=True)
        cnt_ev[b].record(stream)
        if pending is not None:
            d2h += read_back(pending)                  # step k-1's results while step k runs
        pending = b
    if pending is not None:
        d2h += read_back(pending)
    torch.cuda.synchronize()
    return time.perf_counter() - t0, h2d, d2h


def run_fdd(args):
    import torch

    import paper_2205_12362_b300 as fdd

    world, rank, local, dist = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w, f, t, x, sb, n_in = make_workload(
        args.workload, lambda nt, ns, fr, g: fdd.sb_table(nt, ns, fr, chan_per_subband=g))
    n_out = w["n_out"]
    if args.subband:
        if (args.mode or w.get("mode", "plain")) != "plain":
            raise SystemExit("--subband runs with --mode plain (batched searches refuse the two-step mode)")
        sg, sk = (int(v) for v in args.subband.split(","))
        probe = fdd.Plan(w["n_tab"], w["n_chan"], w["n_sb"], f, t, w["ranges"], w["thr"], sb)
        for r in range(len(w["ranges"])):
            probe.set_subband(r, sg, sk)
        n_in = max(n_in, n_out + probe.max_delay + 16)
        x = np.ascontiguousarray(np.pad(x, ((0, 0), (0, 0), (0, max(0, synth.padded_pitch(n_in) - x.shape[2])))))
        probe.close()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 126 MB L2
    host = torch.from_numpy(x).pin_memory()
    wins = [host.to(dev), host.to(dev)]            # window buffers: [0] holds the benchmark chunk
    cap = 1 << 22

    peaks = None
    if not args.no_int_peak:
        peaks = measure_int_peaks(fdd, local)

    arm = Arm(fdd, args, w, f, t, sb, wins, n_in, cap, stream)
    mode = arm.mode

    for _ in range(args.warmup):
        arm.step()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    t_lo = time.time()
    wall0 = time.perf_counter()
    step_ms = timed_steps(arm, args.steps, flush, dist)
    wall1 = time.perf_counter()
    t_hi = time.time()
    clocks = sampler.stop(t_lo, t_hi)
    for p_ in arm.plans:
        if p_.status() != 0:               # a tile-copy wait gave up: the timed output is incomplete
            raise RuntimeError("device status word set (FDD_STATUS_TILE_WAIT): the measurement is void")

    dev_s = reduce_max(sum(step_ms) / 1e3, dist, dev)
    units = units_per_step(w) * args.steps * world
    value = units / dev_s
    ms_step = sum(step_ms) / len(step_ms)

    # per-stage times and kernels per step, outside the timed region
    stage_ms, launches_per_step = arm.stage_pass(min(args.steps, 10), flush)

    # end to end (streaming: the new chunk host-to-device every step)
    e2e_steps = max(3, min(args.steps, 100))
    host_chunk = torch.from_numpy(np.ascontiguousarray(x[:, :, n_in - n_out:n_in])).pin_memory()
    e2e_s, h2d, d2h = e2e_streaming(arm, host_chunk, e2e_steps)
    e2e_s = reduce_max(e2e_s, dist, dev)
    e2e_value = units_per_step(w) * e2e_steps * world / e2e_s

    if rank != 0:
        arm.close()
        if dist:
            dist.destroy_process_group()
        return None

    # roofline of the dominant kernel (dedispersion): channel-adds per launch
    cfgs = arm.configs()
    ded = [v for k, v in stage_ms.items() if k.startswith("dedisperse")]
    ded_ms_step = float(sum(np.mean(v) for v in ded)) if ded else None   # all dedispersion work of a step
    batched_sbf = mode in ("batched", "graph") and arm.plan.batch_config()["variant"] == fdd.FDD_BATCH_SB_FACTORED
    # the SB-factored batch times its part/comb launches of every range as one stage: one "launch"
    n_ded_launches = 1 if batched_sbf else len(ded) * len(arm.plans)
    ded_ms = ded_ms_step / max(1, n_ded_launches) if ded else None
    adds_launch = adds_per_step(w) / max(1, n_ded_launches)
    brute_r = [w["n_sb"] * r["n_dm"] * (n_out // r["downsamp"]) * w["n_chan"] for r in w["ranges"]]
    if args.subband:
        sg, sk = (int(v) for v in args.subband.split(","))
        ratios = [(w["n_chan"] / sk + -(-w["n_chan"] // sg)) / w["n_chan"]] * len(w["ranges"])
    else:
        ratios = [c["work_ratio"] for c in cfgs]
    method_adds_step = float(sum(b_ * q for b_, q in zip(brute_r, ratios)))
    kinds = {v["index"]: v["kind"] for v in fdd.variants()}
    kind_names = {0: "k_dedisp", 1: "k_dedisp_fact", 2: "k_sbf", 3: "k_sbf"}
    if mode in ("batched", "graph"):
        kname = "k_sbf" if batched_sbf else "k_batch"
    else:
        kname = kind_names[kinds[cfgs[0]["variant"]]] if cfgs else "k_dedisp"
    if args.subband:
        kname = "k_sbf_part+k_dedisp (two-step subband, approximate)"
    sm_mhz = clocks.get("sm_mhz")
    derived = N_SM * INT_LANES_PER_SM * ADDS_PER_LANE_OP * SM_MAX_MHZ_NOMINAL * 1e6 / 1e12
    peak = peaks["adds_per_s"] / 1e12 if peaks else derived
    achieved = adds_launch / (ded_ms / 1e3) / 1e12 if ded_ms else None
    method_achieved = (method_adds_step / max(1, n_ded_launches)) / (ded_ms / 1e3) / 1e12 if ded_ms else None
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tadd/s",
            "frac": (achieved / peak) if achieved else None,
            "method_achieved": method_achieved,
            "frac_method": (method_achieved / peak) if method_achieved else None,
            "traffic": profile_traffic(kname, args.workload),
            "kernel": kname, "launches_per_step": n_ded_launches, "units_per_launch": adds_launch,
            "method_adds_per_launch": method_adds_step / max(1, n_ded_launches),
            "method_note": "achieved counts brute-force channel-adds (n_chan per DM-trial output sample); "
                           "method_achieved counts the integer adds the configured kernels perform (the SB-factored "
                           "kernels k_sbf_part + k_sbf_comb reuse TAB x segment partial sums across SBs: "
                           "n_tab*n_chan + n_sb*n_seg per trial and sample; the pattern-factored kernel reuses "
                           "partial sums across DM trials)" + (
                               "; the two-step subband mode is approximate: it does not compute the exact sums"
                               if args.subband else ""),
            "peak_basis": ("measured: fdd_probe_issue_rate (three-input add chains, alone and interleaved with "
                           "multiply-add chains, full occupancy), %.1f T adds/s at %s MHz"
                           % (peaks["adds_per_s"] / 1e12, peaks["sm_mhz"]))
            if peaks else "derived: 148 SM x 128 INT32 lanes x 2 adds/IADD3 x 2032 MHz",
            "peak_derived": derived,
            "smem_bound_adds_per_s": peaks["lds_bytes_per_s"] if peaks else None,
            "smem_note": "the byte-SWAR dedispersion reads one shared-memory byte per channel-add, so the measured "
                         "shared-memory load bandwidth (bytes/s) is also a bound in adds/s",
            "avg_launch_ms": ded_ms}

    cpu = None
    if not args.no_cpu_baseline:
        rate, cores, desc, secs, _, _ = oracle_sample_rate(x, sb, f, t, w, n_in, args.cpu_seconds)
        cpu = {"value": rate, "unit": "samples/s", "cores": cores, "kind": "oracle", "sample": desc,
               "seconds": secs}
        if w["n_sb"] == 1:
            # the same oracle on one host thread, on a smaller sample of the same workload
            import oracle
            oracle.set_threads(1)
            try:
                rate1, _, desc1, secs1, _, _ = oracle_sample_rate(x, sb, f, t, w, n_in,
                                                                   max(1.0, args.cpu_seconds / 4))
            finally:
                oracle.set_threads(cores)
            cpu["single_thread"] = {"value": rate1, "unit": "samples/s", "cores": 1, "sample": desc1,
                                    "seconds": secs1}

    kernel_config = ([arm.plans[0].get_config(r) for r in range(len(w["ranges"]))] if mode in ("plain", "per_sb")
                     else dict(arm.plan.batch_config(), ranges=cfgs))
    arm.close()
    sb_plans_tuned = None

    plain = None
    if w["n_sb"] > 1 and mode != "per_sb" and not args.no_plain_path:
        # the plain per-beam path on the same GPU: one single-SB search per SB
        pargs = argparse.Namespace(**dict(vars(args), mode="per_sb", variant=None, scratch_mb=0))
        parm = Arm(fdd, pargs, w, f, t, sb, wins[:1], n_in, cap, stream)
        parm.step()
        p_ms = timed_steps(parm, args.plain_steps, flush, None)
        pm = float(np.mean(p_ms))
        plain = {"mode": "per_sb", "ms_per_step": pm, "steps": args.plain_steps,
                 "value": units_per_step(w) / (pm / 1e3), "unit": "samples/s",
                 "ratio_plain_over_headline": pm / ms_step,
                 "note": "%d single-SB searches (one per SB) per step, each with the configuration tuned for a "
                         "single-SB plan, against the %s step" % (w["n_sb"], mode)}
        sb_plans_tuned = parm.plans
        del parm

    line = {
        "metric": "DM-trial samples/s (beams x DMs x samples)",
        "value": value,
        "unit": "samples/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u8",
        "data": "synthetic",
        "config": {"workload": args.workload, "n_tab": w["n_tab"], "n_sb": w["n_sb"], "n_chan": w["n_chan"],
                   "n_out": w["n_out"], "n_in": n_in,
                   "dm_plan": [[r["dm0"], r["ddm"], r["n_dm"], r["downsamp"]] for r in w["ranges"]],
                   "widths": WIDTHS, "snr_thresh": w["thr"],
                   "l2": "flushed (256 MB write) between steps; input %.2f GB > L2" % (x.nbytes / 1e9),
                   "parallelism": "replicas" if world > 1 else "single", "mode": mode,
                   "stage_timing": "off in the timed steps; stage times from a separate pass",
                   "dedispersion": ("two-step subband %s (approximate)" % args.subband) if args.subband
                   else "exact"},
        "roofline": roof,
        "int_peak": peaks,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "samples/s",
                "h2d_bytes_per_step": h2d / e2e_steps, "d2h_bytes_per_step": d2h / e2e_steps,
                "steps": e2e_steps, "h2d_overlapped": True,
                "note": "streaming: each step copies the new 1.024 s chunk from pinned host memory and carries the "
                        "delay overlap on the device"},
        "gpu_launches": launches_per_step * args.steps,
        "launches_per_step": launches_per_step,
        "clocks": clocks,
        "stages_ms": {k: float(np.mean(v)) for k, v in stage_ms.items()},
        "kernel_config": kernel_config,
        "plain_path": plain,
        "wall_s": wall1 - wall0,
    }
    plan = arm.plan
    del arm
    wins.clear()
    torch.cuda.empty_cache()
    if not args.no_serving and w["n_sb"] > 1 and mode in ("batched", "graph") and len(w["ranges"]) > 1:
        auto = max(1, int(0.97 * 1024.0 / ms_step))           # beams the measured step time would sustain
        beams = sorted({8, auto, auto + 1})                    # the estimate sits on a boundary: try one more
        line["serving"] = serving_summary(fdd, args, w, f, t, sb, plan, beams, auto, sb_plans_tuned)
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
    _, cores, desc, _, rr, n_sb = oracle_sample_rate(x, sb, f, t, w, n_in, per_step)
    units = n_sb * sum(r["n_dm"] * (w["n_out"] // r["downsamp"]) for r in rr)
    for _ in range(args.warmup):
        oracle.search(x, sb[:n_sb], f, t, rr, w["thr"], w["n_out"], n_in=n_in)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.search(x, sb[:n_sb], f, t, rr, w["thr"], w["n_out"], n_in=n_in)
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


def make_pool(w, f, t, sb, n_pool):
    """A pinned pool of pre-generated chunks: noise plus two sources per chunk
    at seeded SB positions (each pulse put into the TAB its SB takes in every
    channel), each sweep wholly inside its chunk, so a window starting with a
    chunk holds that chunk's pulses whatever the chunk order."""
    import torch
    chunk = w["n_out"]
    sweep = int(arrivals(f, 400.0, t).max())
    pool, pool_pulses = [], []
    for k in range(n_pool):
        prm = synth.random_pulses(w["seed"] * 100 + k, 2, list(range(w["n_sb"])), 50.0, 400.0, [1, 2, 4, 8],
                                  15.0, 40.0, 200, chunk - sweep - 200)
        pulses = []
        for p_ in prm:
            pulses += synth.sb_pulses(sb[p_["tab"]], p_["t0"] + arrivals(f, p_["dm"], t), p_["width"],
                                      synth.pulse_amplitude(p_["snr"], w["n_chan"], p_["width"]))
        x = synth.filterbank(w["seed"] * 1000 + k, w["n_tab"], w["n_chan"], chunk, pitch=chunk, pulses=pulses)
        pool.append(torch.from_numpy(x).pin_memory())
        pool_pulses.append(prm)
    return pool, pool_pulses


def pool_index(window_or_chunk, beam, n_pool):
    return (window_or_chunk + 3 * beam) % n_pool


def serve_run(fdd, plan, w, pool, pool_pulses, n_beams, seconds, rng, sb_plans=None):
    """N beams deliver 1.024 s chunks at real-time cadence (seeded +-50 ms
    jitter) into the serving runtime; per window latency = results seen -
    arrival of the chunk that completed the window.  Returns (run summary,
    window results, window length)."""
    import torch
    chunk = w["n_out"]
    n_pool = len(pool)
    srv = fdd.Server(plan, n_beams, chunk, cap_per_window=1 << 15, sb_plans=sb_plans)
    info = srv.info()
    n_chunks = max(int(seconds / 1.024), -(-info["window_len"] // chunk) + 1)
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
                code = srv.push(b, k, pool[pool_index(k, b, n_pool)], t_arrival=float(arrive[b, k]))
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
    st = srv.info()
    srv.close()
    torch.cuda.empty_cache()
    lat = np.array([r["t_done"] - r["t_arrival"] for r, _ in res])
    gpu = np.array([r["t_done"] - r["t_launch"] for r, _ in res])
    wait = np.array([r["t_launch"] - r["t_ready"] for r, _ in res])
    span = max(r["t_done"] for r, _ in res) - min(r["t_launch"] for r, _ in res) if res else 1.0
    # injected-pulse recall: window w of beam b starts with chunk w, whose pulses it must hold
    injected = recovered = 0
    for r, c in res:
        for p_ in pool_pulses[pool_index(int(r["window"]), int(r["beam"]), n_pool)]:
            injected += 1
            t_abs = int(r["window"]) * chunk + p_["t0"]
            near = ((c["sb"] == p_["tab"]) & (np.abs(c["dm"] - p_["dm"]) < 0.02 * p_["dm"] + 2.0)
                    & (np.abs(c["t_native"] - t_abs) < 4 * p_["width"] + 64))
            recovered += int(near.any())
    p99 = float(np.percentile(lat, 99)) if len(lat) else None
    run = {"beams": n_beams, "path": "plain per-SB" if sb_plans else "batched", "windows": len(res),
           "p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
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
           "recall": recovered / injected if injected else None, "stream_s": n_chunks * 1.024}
    print(json.dumps(run), file=sys.stderr, flush=True)
    return run, res, info["window_len"]


def serving_oracle_check(w, f, t, sb, pool, pool_pulses, res, n_in, n_windows=2):
    """CPU-baseline leg of the serving measurement: the oracle, as it stands,
    on sampled served windows (the window's host samples rebuilt from the
    pool), on two SBs per window (the first injected pulse's SB and one
    other), timed, and compared with the served candidates of those SBs
    (tests/_cmp.py tolerances)."""
    import oracle
    from tests._cmp import compare_candidates, oracle_candidate_superset
    chunk = w["n_out"]
    n_pool = len(pool)
    cpw = -(-n_in // chunk)
    picked = [rc for rc in res if rc[0]["window"] >= 1][:n_windows] or res[:n_windows]
    out = {"checked_windows": 0, "agree": 0, "sbs_per_window": 2, "oracle_s": 0.0, "cores": oracle.get_threads(),
           "failures": []}
    for r, c in picked:
        b, win = int(r["beam"]), int(r["window"])
        x = np.concatenate([pool[pool_index(k, b, n_pool)].numpy() for k in range(win, win + cpw)], axis=2)
        x = np.ascontiguousarray(x[:, :, :n_in])
        s0 = int(pool_pulses[pool_index(win, b, n_pool)][0]["tab"])
        sel = [s0, (s0 + w["n_sb"] // 2) % w["n_sb"]]
        t0 = time.perf_counter()
        ora, _ = oracle_candidate_superset(x, sb[sel], f, t, w["ranges"], w["thr"], chunk, n_in,
                                           t_offset=win * chunk, bins_absolute=True)
        out["oracle_s"] += time.perf_counter() - t0
        ora = ora.copy()
        ora["sb"] = np.asarray(sel, dtype=np.int32)[ora["sb"]]
        gpu = c[np.isin(c["sb"], sel)]
        out["checked_windows"] += 1
        try:
            compare_candidates(gpu, ora, w["thr"])
            out["agree"] += 1
        except AssertionError as e:
            out["failures"].append("beam %d window %d: %s" % (b, win, str(e)[:200]))
    units = sum(r_["n_dm"] * (chunk // r_["downsamp"]) for r_ in w["ranges"]) * 2 * out["checked_windows"]
    out["oracle_samples_per_s"] = units / out["oracle_s"] if out["oracle_s"] else None
    return out


def serving_summary(fdd, args, w, f, t, sb, plan, beams, auto, sb_plans):
    rng = np.random.Generator(np.random.Philox(w["seed"] + 55))
    pool, pool_pulses = make_pool(w, f, t, sb, args.pool)
    runs = []
    res_by, n_in = {}, None
    for nb in beams:
        run, res, n_in = serve_run(fdd, plan, w, pool, pool_pulses, nb, args.seconds, rng)
        runs.append(run)
        res_by[nb] = res
    ok = [r["beams"] for r in runs if r["sustained"]]
    by = {r["beams"]: r for r in runs}
    served = max(ok) if ok else auto  # the largest count tried that was sustained
    plain = None
    if sb_plans and not args.no_plain_path:
        plain, _, _ = serve_run(fdd, plan, w, pool, pool_pulses, served, args.plain_seconds, rng, sb_plans=sb_plans)
    check = None
    if res_by.get(served) and not args.no_cpu_baseline:
        check = serving_oracle_check(w, f, t, sb, pool, pool_pulses, res_by[served], n_in)
    return {"metric": "p99 chunk latency (s) at real-time cadence", "unit": "s", "higher_is_better": False,
            "deadline_s": 1.024, "jitter_ms": 50, "pool_chunks": args.pool,
            "max_sustained_beams_tried": max(ok) if ok else 0, "beams_tried": beams,
            "auto_beams": auto, "auto_basis": "floor(0.97 x 1024 ms / measured step ms); auto + 1 tried too",
            "served_beams": served,
            "p50_s_8": by.get(8, {}).get("p50_s"), "p99_s_8": by.get(8, {}).get("p99_s"),
            "p50_s_auto": by.get(auto, {}).get("p50_s"), "p99_s_auto": by.get(auto, {}).get("p99_s"),
            "p50_s_served": by.get(served, {}).get("p50_s"), "p99_s_served": by.get(served, {}).get("p99_s"),
            "plain_beams": served if plain else None,
            "plain_p99_s_served": plain["p99_s"] if plain else None,
            "runs": runs + ([plain] if plain else []),
            "oracle_check": check}


def run_serve(args):
    """--serve: the serving measurement alone, at the beam counts given."""
    import torch

    import paper_2205_12362_b300 as fdd
    torch.cuda.set_device(0)
    w = dict(WORKLOADS[args.workload])
    f = synth.channel_freqs(w["n_chan"])
    t = synth.ARTS_T_SAMP_S
    chunk = w["n_out"]
    sb = synth.sb_map_piecewise(w["seed"], w["n_sb"], w["n_chan"], w["n_tab"]).astype(np.int16)
    plan = fdd.Plan(w["n_tab"], w["n_chan"], w["n_sb"], f, t, w["ranges"], w["thr"], sb)
    n_in = chunk + plan.max_delay
    win = torch.zeros((w["n_tab"], w["n_chan"], synth.padded_pitch(n_in)), dtype=torch.uint8, device="cuda")
    job = plan.make_job(win, n_in, chunk, cap=1 << 15)
    plan.batch_prepare(chunk)
    if not args.no_autotune:
        plan.batch_autotune([job], chunk, reps=1)
    del job, win
    torch.cuda.empty_cache()
    rng = np.random.Generator(np.random.Philox(w["seed"] + 55))
    pool, pool_pulses = make_pool(w, f, t, sb, args.pool)
    out = {"metric": "p99 chunk latency (s) at real-time cadence", "unit": "s", "higher_is_better": False,
           "data": "synthetic", "config": {"workload": args.workload, "chunk_s": chunk * t, "jitter_ms": 50,
                                           "pool_chunks": args.pool, "stream_s": args.seconds},
           "batch_config": plan.batch_config(), "runs": []}
    for n_beams in [int(v) for v in args.beams.split(",")]:
        run, _, _ = serve_run(fdd, plan, w, pool, pool_pulses, n_beams, args.seconds, rng)
        out["runs"].append(run)
    ok = [r["beams"] for r in out["runs"] if r["sustained"]]
    out["max_sustained_beams"] = max(ok) if ok else 0
    best = [r for r in out["runs"] if r["beams"] == out["max_sustained_beams"]]
    out["value"] = best[0]["p99_s"] if best else None
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="arts_71sb_4range", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="fdd", choices=["fdd", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-int-peak", action="store_true", help="skip the issue-rate probes (roofline peaks)")
    ap.add_argument("--no-plain-path", action="store_true", help="skip the plain per-SB path (step and serving)")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving runs of the default bench")
    ap.add_argument("--plain-steps", type=int, default=3, help="timed steps of the plain per-SB path")
    ap.add_argument("--variant", default=None,
                    help="force this dedispersion kernel variant (one index, or one per DM range, comma-separated)")
    ap.add_argument("--cc", default="0",
                    help="with --variant: channels per stage (0 = largest fitting), one for every range or "
                         "a comma-separated one per range")
    ap.add_argument("--batch-variant", type=int, default=None,
                    help="batched/graph modes: this batch variant instead of the tuner's choice (1000 SB-factored "
                         "launches, 1001 one persistent SB-factored launch, 0.. brute-force persistent)")
    ap.add_argument("--subband", default=None,
                    help="G,K: approximate two-step subband dedispersion (G channels per subband, K fine trials per "
                         "coarse DM) instead of the exact kernels; not the benchmark's default")
    ap.add_argument("--scratch-mb", type=int, default=0,
                    help="cap on the SB-factored kernel's partial-sum scratch (0 = library default)")
    ap.add_argument("--serve", action="store_true", help="serving measurement instead of the step benchmark")
    ap.add_argument("--beams", default="1,2,3,4,8", help="--serve: compound-beam counts to run")
    ap.add_argument("--seconds", type=float, default=8.0, help="serving: stream length per run")
    ap.add_argument("--plain-seconds", type=float, default=4.0, help="serving: stream length of the plain path run")
    ap.add_argument("--pool", type=int, default=4, help="serving: pre-generated chunks in the pinned pool")
    ap.add_argument("--mode", default=None, choices=["plain", "per_sb", "batched", "graph"],
                    help="plain: per-range launches over all SBs; per_sb: one plan per SB (the plain per-beam "
                         "path); batched: the batched search; graph: the batched search replayed from a CUDA "
                         "graph (default: the workload's own)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.serve:
        line = run_serve(args)
    else:
        line = run_fdd(args) if args.impl == "fdd" else run_reference(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
