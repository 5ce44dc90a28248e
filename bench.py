#!/usr/bin/env python
"""Throughput of the coherent-receiver DSP chain on one GB300 (per rank).

Workload: the 10,000 km straight-line shape -- DP-QPSK 10 GBd, 2 samples per
symbol, 2^24 symbols per polarisation (2^25 sample-times) streamed as int8
ADC samples, with dispersion D = 17 ps/(nm km), slowly varying PMD
(0.1 ps/sqrt(km)), 100 kHz laser phase noise, a 200 MHz frequency offset and
AWGN at Es/N0 = 9.8 dB (pre-FEC BER ~1e-3).  Synthetic, seeded input from
``linksim`` stands in for the paper's lab link.

One step = one pass of the whole chain over the stream: reset, one
rx_process call with all samples (CDC -> FO removal -> butterfly CMA/DD-LMS
-> BPS/unwrap -> demap), the flush call, and rx_ber (synchronised BER count).
Inputs (128 MiB int8) and intermediates (512 MiB CDC output) are larger than
L2, so no L2 flush is inserted between steps.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GSa/s and decoded Gb/s per GB300 at oracle-matched BER; % HBM roofline"
FP32_LANES_PER_SM = 128
N_SM = 152


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 150; 40 for --impl reference, ~1 s of CPU each)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n-sym", type=int, default=1 << 24, help="symbols per pol (default: the full workload)")
    ap.add_argument("--cpu-sample", type=int, default=1 << 21, help="sample-times the oracle baseline processes")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--precision", choices=["fp32", "fp16", "bf16"], default="fp32",
                    help="storage of the CDC transform and its output (single-stream workloads)")
    ap.add_argument("--workload", choices=["c2", "c3", "c4", "c5", "kk"], default="c2",
                    help="c2: the 10,000 km single stream (default); c4: the 64-channel batched form; "
                         "c5: the chain plus the learned post-equaliser on a Kerr-nonlinear link")
    ap.add_argument("--channels", type=int, default=64, help="c4: number of channels")
    ap.add_argument("--dft-tc", type=int, default=0,
                    help="precision form: 1 = CDC radix-16 passes on tensor cores, 0 = register butterflies")
    ap.add_argument("--train-symbols", type=int, default=1 << 14, help="c5: symbols per training sequence")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 40 if args.impl == "reference" else 150
    return args


# ncu dram__bytes_read.sum + dram__bytes_write.sum of one step's eq_kernel launches per
# symbol on the 10,000 km QPSK workload (13 launches of a 2^22-symbol step); None when
# the kernel has changed since the counters were taken
EQ_DRAM_BYTES_PER_SYMBOL = 32.4
# algorithmic equaliser work per dual-pol sample-time: FIR 2x2x15 complex MACs per
# symbol (240 flop per sample-time) and the same for the LMS gradient
EQ_FLOP_PER_SAMPLE_TIME = 480.0
_ALU_PEAK = {}


def alu_peak_tflops(stream=None):
    """FP32 FMA peak measured on this GPU in this run (rx_measure_alu_peak), cached."""
    if "fp32" not in _ALU_PEAK:
        from paper_2104_06311_gb300.rx import measure_alu_peak
        sid = stream.cuda_stream if stream is not None else None
        best = max(measure_alu_peak("fp32", 32768, sid)[0] for _ in range(3))
        _ALU_PEAK["fp32"] = best
        _ALU_PEAK["fp64"] = max(measure_alu_peak("fp64", 512, sid)[0] for _ in range(2))
    return _ALU_PEAK["fp32"], (f"FP32 FMA chains measured in this run (best of 3): {_ALU_PEAK['fp32']:.1f} TFLOP/s; "
                               f"FP64 {_ALU_PEAK['fp64']:.2f} TFLOP/s")


def max_over_ranks(ms, dist=None, device="cpu"):
    """The slowest rank's time (every rank gets it); ms itself on one rank."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, steps, world, ms):
    """Units all ranks processed (replicas: each rank its own full workload) per second, in 1e9/s."""
    return units_per_rank * steps * world / (ms / 1e3) / 1e9


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "500"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows if len(r) >= 9 for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


WORKLOADS = {
    "c2": "10,000 km straight-line DP-QPSK 10 GBd, 2 sps, 2^24 symbols/pol, int8 ADC, "
          "PMD 0.1 ps/sqrt(km), 100 kHz PN, 200 MHz FO, Es/N0 9.8 dB",
    "c3": "DP-16QAM 32 GBd, 2 sps, 2^22 symbols/pol, 6000 km, 100 kHz PN, Es/N0 18 dB, int8 ADC",
}


def make_input(n_sym, name="c2"):
    import linksim as L
    lk = L.workload(name, n_sym=n_sym)
    return lk, L.generate(lk)


def cpu_oracle_run(g, n_samples):
    """Time the FP64 oracle (as it stands) on the first n_samples sample-times."""
    import oracle as O
    lk = g.link
    p = O.RxParams(baud=lk.baud, L_km=lk.L_km, D=lk.D, mod=lk.mod, in_scale=g.in_scale)
    x = g.samples[:n_samples]
    t0 = time.perf_counter()
    out = O.run_chain(x, p)
    dt = time.perf_counter() - t0
    return out, dt, p


def _oracle_replica(args):
    """One independent replica of the oracle on a bounded sample (all-cores baseline)."""
    samples, baud, L_km, D, mod, in_scale = args
    import oracle as O
    if samples is None:
        return 0.0
    p = O.RxParams(baud=baud, L_km=L_km, D=D, mod=mod, in_scale=in_scale)
    t0 = time.perf_counter()
    O.run_chain(samples, p)
    return time.perf_counter() - t0


def oracle_all_cores(g, ns):
    """The oracle on every host core: independent replicas of the first ns sample-times
    (the chain's waves are sequential, so more cores serve more streams), one process
    each, started with spawn (the parent holds a CUDA context)."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0))
    lk = g.link
    job = (g.samples[:ns], lk.baud, lk.L_km, lk.D, lk.mod, g.in_scale)
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_replica, [(None,) + job[1:]] * cores)     # start-up and imports, untimed
        t0 = time.perf_counter()
        pool.map(_oracle_replica, [job] * cores)
        wall = time.perf_counter() - t0
    return {"value": cores * ns / wall / 1e9, "unit": "GSa/s", "cores": cores, "kind": "oracle",
            "sample": f"{cores} independent replicas of the first {ns} sample-times, FP64 numpy oracle, "
                      "one process per core"}


def reference_arm(args, rank, world):
    if rank != 0:
        return
    # each step a bounded sample (2^19 sample-times, ~2 s of FP64 numpy) so that a
    # default --steps 40 --warmup 3 run ends within a few minutes (each step ~1 s)
    lk, g = make_input(min(args.cpu_sample, 1 << 19) // 2)
    n = g.samples.shape[0]
    times = []
    for i in range(args.warmup + args.steps):
        _, dt, p = cpu_oracle_run(g, n)
        if i >= args.warmup:
            times.append(dt)
    t = sum(times)
    value = n * args.steps / t / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GSa/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded linksim 10,000 km link)",
        "config": {"workload": "10,000 km straight-line DP-QPSK 10 GBd int8, 2^24 symbols/pol (bounded sample)",
                   "sample_times_per_step": n},
        "cpu_baseline": {"value": value, "unit": "GSa/s", "cores": 1, "kind": "oracle",
                         "sample": f"first {n} sample-times of the workload per step (FP64 numpy oracle)"},
        "e2e": {"value": value, "unit": "GSa/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _gen_one(lk):
    import linksim as L
    g = L.generate(lk)
    return g.samples, L.pack_bits(g.tx_bits), g.in_scale


def bench_batch(args, rank, world, local):
    """The batched form: 64 WDM channels of uneven length / rate / dispersion / format."""
    import multiprocessing as mp
    import numpy as np
    import linksim as L
    from paper_2104_06311_gb300.shard import channel_cost, merge_counts, shard_channels
    links_all = L.workload_batch(args.channels)
    n_all = sum(2 * lk.n_sym for lk in links_all)
    # N > 1: the channels are independent, so each rank takes a cost-balanced share
    # (no exchange on the data path; the error counts are merged at the end)
    mine = shard_channels([channel_cost(2 * lk.n_sym, 4 if lk.mod == "16qam" else 2) for lk in links_all],
                          world)[rank]
    links = [links_all[c] for c in mine]
    # generate before the first CUDA call (spawned workers, no CUDA state)
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        gens = pool.map(_gen_one, links, chunksize=1)
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2104_06311_gb300 import Batch, build
    if not os.path.exists(build.OUT):
        build.build()
    stream = torch.cuda.current_stream()
    xs = [torch.from_numpy(s).cuda() for s, _, _ in gens]
    refs = [torch.from_numpy(w.view(np.int32)).cuda() for _, w, _ in gens]
    # the workload's channels carry neither a frequency offset nor laser phase noise:
    # frequency tracking off, and a longer BPS window for 16QAM (no phase noise to track)
    cfgs = [dict(baud=lk.baud, L_km=lk.L_km, in_scale=sc, max_samples=s.shape[0],
                 mod_bits=4 if lk.mod == "16qam" else 2, flags=1, bps_halfwin=64 if lk.mod == "16qam" else 16)
            for lk, (s, _, sc) in zip(links, gens)]
    b = Batch(cfgs, stream=stream)
    outs = b.alloc_outs(xs)
    n_total = sum(x.shape[0] for x in xs)
    K_total = n_total // 2
    bits_total = sum(x.shape[0] // 2 * 2 * c["mod_bits"] for x, c in zip(xs, cfgs))

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):      # eager, captured, then replayed
        b.process(xs, outs)
    torch.cuda.synchronize()
    b.profile(reset=True)
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        b.process(xs, outs)
    t1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = t0.elapsed_time(t1)
    launches = sum(v[1] for v in b.profile(reset=True).values())
    ms = max_over_ranks(ms, dist, "cuda")
    value = whole_job_rate(n_all, args.steps, 1, ms)     # every rank's channels in the slowest rank's time
    # stage split from profiled (eager) calls
    b.set_param("PROFILE", 1)
    for _ in range(args.steps):
        b.process(xs, outs)
    prof = b.profile(reset=True)
    b.set_param("PROFILE", 0)
    # BER per channel (after the timed region)
    # each channel's last V/2 symbols are not counted: the generator applies the fibre's
    # dispersion circularly over the finite stream, so the tail carries the head's
    # dispersed energy, which no linear receiver undoes (the head is skipped anyway)
    errs = []
    for ch in range(len(xs)):
        edge = int(b.get_param(ch, "OVERLAP")) // 2
        e, nb, _ = b.ber(ch, outs[ch]["bits"], refs[ch], xs[ch].shape[0] // 2 - edge)
        errs.append((e, nb))
    errs_all = merge_counts(errs, len(links_all), mine, dist, "cuda")
    ber = [e / nb if nb else None for e, nb in errs_all]
    import oracle as O_
    theory = [O_.ber_theory(lk.mod, lk.snr_db) for lk in links_all]

    def snr_penalty_db(lk, b_):
        """Es/N0 at which AWGN theory gives this BER, below the channel's own (None: error-free)."""
        if b_ is None or b_ <= 0.0:
            return None
        if b_ >= O_.ber_theory(lk.mod, -10.0):
            return float("inf")
        from scipy.optimize import brentq
        eff = brentq(lambda x: O_.ber_theory(lk.mod, x) - b_, -10.0, 40.0)
        return lk.snr_db - eff

    pen = [snr_penalty_db(lk, b_) for lk, b_ in zip(links_all, ber)]
    hi_snr = [q for q, lk in zip(pen, links_all) if q is not None and lk.snr_db >= 12.0]
    hi_free = sum(1 for q, lk in zip(pen, links_all) if q is None and lk.snr_db >= 12.0)
    lo_snr = [(ch, lk.mod, round(lk.snr_db, 1), ber[ch]) for ch, lk in enumerate(links_all) if lk.snr_db < 12.0]
    correct_bits = sum(2 * lk.n_sym * (4 if lk.mod == "16qam" else 2) * (1.0 - (b_ or 0.0))
                       for lk, b_ in zip(links_all, ber))
    bits_total = sum(2 * lk.n_sym * (4 if lk.mod == "16qam" else 2) for lk in links_all)
    e2e = None
    if not args.no_e2e:
        xh = [torch.from_numpy(s).pin_memory() for s, _, _ in gens]
        bits_h = [torch.empty_like(o["bits"], device="cpu").pin_memory() for o in outs]
        xd = xs

        def step_e2e():
            for d, h in zip(xd, xh):
                d.copy_(h, non_blocking=True)
            b.process(xd, outs)
            for h, o in zip(bits_h, outs):
                h.copy_(o["bits"], non_blocking=True)

        for _ in range(2):
            step_e2e()
        torch.cuda.synchronize()
        a_ = torch.cuda.Event(enable_timing=True)
        b_ = torch.cuda.Event(enable_timing=True)
        a_.record(stream)
        for _ in range(args.steps):
            step_e2e()
        b_.record(stream)
        torch.cuda.synchronize()
        ems = max_over_ranks(a_.elapsed_time(b_), dist, "cuda")
        e2e = {"value": n_all * args.steps / (ems / 1e3) / 1e9, "unit": "GSa/s",
               "h2d_bytes_per_step": int(sum(x.numel() * x.element_size() for x in xs)),
               "d2h_bytes_per_step": int(sum(o["bits"].numel() * 4 for o in outs))}
    pk, pk_kind = peaks()
    T, W, S = 15, 128, 1024
    stage = max(("cdc", "eq", "bps"), key=lambda s: prof[s][0])
    if stage == "eq":
        flop = EQ_FLOP_PER_SAMPLE_TIME * n_total
        peak, peak_note = alu_peak_tflops(stream)
        achieved = flop / (prof[stage][0] / args.steps / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": "eq_batch_kernel", "peak_note": peak_note}
    else:
        per = {"cdc": 4 + 16, "bps": 16 + 16 + 1 + 0.25 * 2}[stage]
        achieved = per * n_total / (prof[stage][0] / args.steps / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / pk["hbm_gbs"], "traffic": None, "kernel": stage}
    roof["peak_source"] = "measured (FMA chains, this run)" if roof["bound"] == "alu" else pk_kind
    Ns = sorted({int(b.get_param(ch, "FFT_N")) for ch in range(len(xs))})
    # channels per (FFT size, CDC engine) the autotuner picked (engine 1: four-step)
    picks = {}
    for ch in range(len(xs)):
        k = f"{int(b.get_param(ch, 'FFT_N'))}/{'four-step' if b.get_param(ch, 'CDC_ENGINE') else 'radix-16'}"
        picks[k] = picks.get(k, 0) + 1
    line = {
        "metric": METRIC, "value": value, "unit": "GSa/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "strong" if world > 1 else "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded linksim WDM channels), resident in HBM",
        "config": {"workload": f"{len(links_all)} WDM channels, 2^18-2^22 symbols/pol, 2000-10000 km, 10-32 GBd, "
                               "QPSK/16QAM, Es/N0 10-18 dB, int8 ADC; one enqueue per step (CUDA graph replay)",
                   "sample_times": n_all, "fft_n_autotuned": Ns, "cdc_autotuned": picks,
                   "eq_ctas": int(b.get_param(-1, "EQ_CTAS")),
                   "l2": f"inputs ({n_all * 4 >> 20} MiB) and CDC intermediates exceed L2; no flush",
                   "parallelism": (f"channels sharded over {world} ranks (cost-balanced, no data-path collective)"
                                   if world > 1 else "one batch")},
        "decoded_gbps": bits_total * args.steps / (ms / 1e3) / 1e9,
        "goodput_gbps": correct_bits * args.steps / (ms / 1e3) / 1e9,
        "ber_per_channel": {"min": min(x for x in ber if x is not None),
                            "median": statistics.median(x for x in ber if x is not None),
                            "max": max(x for x in ber if x is not None),
                            "channels_above_0.1": sum(1 for x in ber if x is not None and x > 0.1),
                            "snr_penalty_db_at_or_above_12dB": {
                                "channels_with_errors": len(hi_snr), "error_free": hi_free,
                                "max": max(hi_snr) if hi_snr else None,
                                "median": statistics.median(hi_snr) if hi_snr else None,
                                "worst": sorted(((round(q, 2), ch) for ch, q in enumerate(pen)
                                                 if q is not None and links_all[ch].snr_db >= 12.0),
                                                reverse=True)[:5]},
                            "below_12dB": lo_snr,
                            "config": "per channel: frequency tracking off (the channels carry no offset), "
                                      "BPS half window 64 for 16QAM, 16 for QPSK (no laser phase noise)",
                            "counted": "symbols [A + 8192, K - V/2) of each channel (the synthetic stream's "
                                       "dispersion is circular: its last V/2 symbols hold wrapped energy)"},
        "stage_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
        "gpu_launches": int(launches),
        "roofline": roof,
        "clocks": clk,
        "e2e": e2e,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as O
        lk0, (s0, _, sc0) = links[0], gens[0]
        ns = min(args.cpu_sample, s0.shape[0])
        p = O.RxParams(baud=lk0.baud, L_km=lk0.L_km, D=lk0.D, mod=lk0.mod, in_scale=sc0)
        t0_ = time.perf_counter()
        O.run_chain(s0[:ns], p)
        dt = time.perf_counter() - t0_
        line["cpu_baseline"] = {"value": ns / dt / 1e9, "unit": "GSa/s", "cores": 1, "kind": "oracle",
                                "sample": f"first {ns} sample-times of channel 0, FP64 numpy oracle, one core"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def bench_learned(args, rank, world, local):
    """Chain + CNN post-equaliser on a split-step (Kerr) link: training and inference."""
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    from paper_2104_06311_gb300 import CNN, Receiver, build
    if not os.path.exists(build.OUT):
        build.build()
    import linksim as L
    from linksim import ssfm as F
    n_sym = min(args.n_sym, 1 << 22)
    spec = dict(mod="16qam", baud=10e9, spans=10, span_km=100.0, launch_dbm=2.0, n_sym=n_sym, step_km=1.0)
    stream = torch.cuda.current_stream()
    sets = {}
    for name, seed in (("train", 2104063115), ("test", 2104063116)):
        g = F.generate(F.SSFMLink(seed=seed, **spec), device="cuda", dtype="float32")
        x = torch.from_numpy(np.ascontiguousarray(g.samples)).cuda()
        rx = Receiver(spec["baud"], g.link.L_km, stream=stream, MOD=4, IN_SCALE=g.in_scale, FO_TRACK=0, SYM_OUT=1)
        out = rx.run_stream(x, sym=True)
        K = out["n"]
        ref = torch.from_numpy(L.pack_bits(g.tx_bits).view(np.int32)).cuda()
        e, nb, sync = rx.ber(out["bits"], ref, K)
        k0, k1 = 16384 + 8192, K - 64
        t = np.zeros((2, k1 - k0), np.complex64)
        for pp, (q, r, d) in enumerate(sync):
            t[pp] = (1j ** r) * g.tx_symbols[q, k0 + d:k1 + d]
        zc = out["sym"][:, k0:k1].contiguous()
        t = L.align_rotation(zc.cpu().numpy(), t).astype(np.complex64)
        sets[name] = dict(x=x, rx=rx, z=zc, t=torch.from_numpy(t).cuda(), ber=e / max(nb, 1), K=K)
    B, BI = args.train_symbols, 1 << 20   # training sequences / inference sequences (symbols)
    tr, te = sets["train"], sets["test"]
    n_tr = tr["z"].shape[1] // B * B
    net = CNN(BI, stream=stream)
    net.set_params(L.cnn_init_params(3))     # seeded He-normal initial weights

    def epoch(lr):
        for s in range(0, n_tr, B):
            net.train_step(tr["z"][:, s:s + B], tr["t"][:, s:s + B], lr=lr)

    for _ in range(args.warmup):
        epoch(3e-4)
    net.set_profile(True)
    net.profile(reset=True)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        epoch(3e-4)
    t1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    train_ms = t0.elapsed_time(t1) / args.steps
    prof_train = net.profile(reset=True)
    # inference over the test stream, in sequences of B symbols
    zt = te["z"]
    y = torch.empty_like(zt)

    def infer():
        for s in range(0, zt.shape[1], BI):
            e = min(s + BI, zt.shape[1])
            net.apply(zt[:, s:e], out=y[:, s:e])

    infer()
    net.profile(reset=True)
    a_ = torch.cuda.Event(enable_timing=True)
    b_ = torch.cuda.Event(enable_timing=True)
    a_.record(stream)
    for _ in range(args.steps):
        infer()
    b_.record(stream)
    torch.cuda.synchronize()
    infer_ms = a_.elapsed_time(b_) / args.steps
    prof_inf = net.profile(reset=True)
    net.set_profile(False)
    # end to end: chain + CNN over the test stream (whole-stream steps)
    xt = te["x"]
    n = xt.shape[0]
    c0 = torch.cuda.Event(enable_timing=True)
    c1 = torch.cuda.Event(enable_timing=True)
    outc = te["rx"].alloc_out(n // 2 + 64, sym=True)
    c0.record(stream)
    for _ in range(args.steps):
        te["rx"].run_stream(xt, sym=True, out=outc)
        infer()
    c1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = c0.elapsed_time(c1) / args.steps
    yh = y.cpu().numpy().astype(np.complex128)
    zh, th = zt.cpu().numpy().astype(np.complex128), te["t"].cpu().numpy().astype(np.complex128)
    mse_c, mse_n = float(np.mean(np.abs(zh - th) ** 2)), float(np.mean(np.abs(yh - th) ** 2))
    flop_sym = 2 * 15 * (4 * 64 + 64 * 64 * 2 + 64 * 4)          # forward, per symbol
    n_inf = zt.shape[1]
    pk, pk_kind = peaks()
    # the 64 -> 64 forward convolutions: (layers - 2) per pass, 2*15*64*64 flop per symbol each
    hid_ms, hid_n = prof_inf["fwd_hidden"]
    per_launch_flop = args.steps * 2 * (2 * 15 * 64 * 64 * n_inf) / max(1, hid_n)
    per_launch_ms = hid_ms / max(1, hid_n)
    achieved = per_launch_flop / (per_launch_ms / 1e3) / 1e12
    roof = {"bound": "tensor", "achieved": achieved, "peak": pk["bf16_tflops"], "unit": "TFLOP/s",
            "frac": achieved / pk["bf16_tflops"], "traffic": None, "kernel": "conv_tc_kernel (64 -> 64 forward)",
            "peak_source": pk_kind,
            "note": "tcgen05.mma kind::f16 M128 N64 K16, BF16 in, FP32 in tensor memory; "
                    "peak = measured cuBLAS bf16 burst"}
    line = {
        "metric": METRIC, "value": n / (e2e_ms / 1e3) / 1e9, "unit": "GSa/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": e2e_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic split-step (Manakov) link, seeded; train and test seeds differ",
        "config": {"workload": "DP-16QAM 10 GBd, 10 x 100 km SSMF (0.2 dB/km, gamma 1.3 /W/km, NF 5 dB), 2 dBm, "
                               f"{n_sym} symbols/pol; chain + 4-layer CNN (64 ch, k 15) post-equaliser",
                   "sample_times": n, "batch_symbols": B, "l2": "CNN activations (512 MiB per layer) exceed L2"},
        "step": "e2e: whole-stream chain + CNN inference; training epochs timed separately",
        "train": {"ms_per_epoch": train_ms, "symbols_per_epoch": n_tr,
                  "tflops": 3 * flop_sym * n_tr / (train_ms / 1e3) / 1e12,
                  "kernel_ms_per_epoch": {k: v[0] / args.steps for k, v in prof_train.items()}},
        "inference": {"ms": infer_ms, "symbols": n_inf, "gsym_per_s": n_inf / (infer_ms / 1e3) / 1e9,
                      "tflops": flop_sym * n_inf / (infer_ms / 1e3) / 1e12},
        "gain": {"mse_chain": mse_c, "mse_cnn": mse_n, "effective_snr_gain_db": 10 * math.log10(mse_c / mse_n),
                 "chain_ber_test": te["ber"]},
        "roofline": roof, "clocks": clk,
        "gpu_launches": int(sum(v[1] for v in prof_train.values())),
        "e2e": {"value": n / (e2e_ms / 1e3) / 1e9, "unit": "GSa/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0,
                "note": "inputs resident on the device"},
    }
    if rank == 0 and not args.no_cpu_baseline:
        import oracle.cnn as OC
        ns = 1 << 12
        params = net.unflatten(net.get_params())
        zs = zh[:, :ns]
        t0_ = time.perf_counter()
        OC.forward(params, OC.features(zs))
        dt = time.perf_counter() - t0_
        line["cpu_baseline"] = {"value": 2 * ns / dt / 1e9, "unit": "GSa/s", "cores": 1, "kind": "oracle",
                                "sample": f"FP64 CNN forward (oracle) on the first {ns} test symbols, one core; "
                                          "GSa/s = 2 samples per symbol"}
    print(json.dumps(line), flush=True)


def bench_kk(args, rank, world, local):
    """The paper's own chain: Kramers-Kronig front end, four-tap widely-linear
    DD-LMS and demapping, over 2^22-sample ADC buffers.  Like the paper, buffers
    run on several streams: the front end of buffer i+1 overlaps the equaliser of
    buffer i, and the equaliser of buffer i+1 waits (event) for both its own field
    and the taps the equaliser of buffer i left."""
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    from paper_2104_06311_gb300 import KKFrontEnd, WLEqualiser, build
    if not os.path.exists(build.OUT):
        build.build()
    import linksim.kk as LK
    n_buf, slots = 4, 8                    # 4 distinct 2^22-sample buffers, each in 2 device slots
    # the carrier on the recording's frequency grid: replaying the 4 buffers in a loop is
    # one continuous periodic stream (dispersion is applied circularly by the generator)
    fc = round(0.516e9 / 4e9 * (n_buf << 22)) * 4e9 / (n_buf << 22)
    lk = LK.KKLink(n_sym=n_buf << 20, L_km=5600.0, cspr_db=12.0, snr_db=24.0, adc="int8",
                   iq_gain_db=1.0, iq_phase_deg=5.0, carrier_hz=fc)
    g = LK.generate(lk)
    n = 1 << 22                            # samples per buffer
    K = n // 4                             # symbols per buffer
    words = K * 4 // 32
    main = torch.cuda.current_stream()
    s_fe, s_eq = torch.cuda.Stream(), torch.cuda.Stream()
    fe = KKFrontEnd(lk.baud, lk.carrier_hz, lk.L_km, n, stream=s_fe)
    eq = WLEqualiser(4, K, stream=s_eq)
    host = torch.from_numpy(np.ascontiguousarray(g.samples[:n_buf * n])).view(n_buf, n)
    x = torch.empty(slots, n, dtype=torch.int8, device="cuda")
    for i in range(slots):
        x[i].copy_(host[i % n_buf].cuda())
    y = torch.empty(slots, n // 2, dtype=torch.complex64, device="cuda")
    bits = torch.empty(slots, words, dtype=torch.int32, device="cuda")
    ev_fe = [torch.cuda.Event() for _ in range(slots)]

    def step():
        start = torch.cuda.Event()
        start.record(main)
        for st_ in (s_fe, s_eq):
            st_.wait_event(start)
        for i in range(slots):
            fe.process(x[i], g.in_scale, g.in_offset, out=y[i])
            ev_fe[i].record(s_fe)
            s_eq.wait_event(ev_fe[i])
            eq.process(y[i], bits=bits[i])
        main.wait_stream(s_fe)
        main.wait_stream(s_eq)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(main)
    for _ in range(args.steps):
        step()
    t1.record(main)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = max_over_ranks(t0.elapsed_time(t1), None) / args.steps
    # per-stage device time (serialised by the profiling events of each object)
    fe.profile(on=True, reset=True)
    eq.profile(on=True, reset=True)
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    prof = fe.profile(on=False, reset=True)
    wprof = eq.profile(on=False, reset=True)
    # e2e through the real-time pipeline (rx_rt.h): each buffer copied from pinned host memory
    # (the ADC's DMA buffers) to the device, front end, DD-LMS, BER count, bits back to the
    # pinned host ring; host wall clock from the first submit to the drain
    from paper_2104_06311_gb300 import RealTime
    rt = RealTime(lk.baud, lk.carrier_hz, lk.L_km, n, mod_bits=4, depth=6, in_scale=g.in_scale,
                  in_offset=g.in_offset, ref_bits=g.tx_bits, bin_symbols=21_000_000)
    pinned = host.pin_memory()             # the recorded buffers as the ADC's pinned DMA buffers
    for b in range(4):
        rt.submit_from(pinned[b % n_buf])
    rt.drain()
    t0_ = time.perf_counter()
    for b in range(4, 4 + args.steps * slots):
        rt.submit_from(pinned[b % n_buf])
    rt.drain()
    ems = (time.perf_counter() - t0_) * 1e3 / args.steps
    rtbins = rt.bins()
    rt.close()
    # decisions of the last step against the transmitted bits
    bb = np.unpackbits(bits.cpu().numpy().view(np.uint8), bitorder="little").reshape(slots, K, 4)
    # the front end streams with a delay of 1536 samples: output symbol k of slot i is
    # stream symbol i K - 384 + k (the periodic stream repeats every n_buf buffers)
    txs = g.tx_bits.reshape(n_buf * K, 4)
    sidx = (np.arange(slots)[:, None] * K - 384 + np.arange(K)[None, :]) % (n_buf * K)
    errs = int(np.count_nonzero(bb != txs[sidx]))
    ber = errs / (slots * K * 4)
    pk, pk_kind = peaks()
    stage = max(prof, key=lambda k: prof[k])
    per = {"hilbert": 1 + 8, "filter": 8 + 4}[stage]          # algorithmic bytes per input sample
    achieved = per * n * slots / (prof[stage] / args.steps / 1e3) / 1e9
    total = slots * n
    line = {
        "metric": METRIC, "value": total / (ms / 1e3) / 1e9, "unit": "GSa/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32",
        "data": "synthetic seeded self-coherent link (linksim.kk), resident in HBM",
        "config": {"workload": "Kramers-Kronig chain (front end, 4-tap widely-linear DD-LMS, Gray demap): 16QAM "
                               "1 GBd + 0.516 GHz carrier (CSPR 12 dB), TX IQ imbalance 1 dB / 5 deg, 4 sps, "
                               "5600 km, int8 ADC, eight consecutive 2^22-sample buffers of one continuous stream per "
                               "step (a recorded 4-buffer period, looped), front end and DD-LMS on 2 streams",
                   "sample_times": total, "buffers_per_step": slots,
                   "l2": "8 x 4 MiB int8 in, 8 x 16 MiB fields at 2 sps, 8 x 0.5 MiB bits: 164 MiB per step, "
                         "more than the 129 MB L2 (the 32 MiB front-end scratch stays L2-resident); no flush"},
        "decoded_gbps": total / 4 * 4 / (ms / 1e3) / 1e9,
        "ber": ber,
        "stage_ms_per_step": {**{k: v / args.steps for k, v in prof.items()},
                              **{"wl_" + k: v / args.steps for k, v in wprof.items()}},
        "gpu_launches": 3 * slots * args.steps,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / pk["hbm_gbs"], "traffic": None, "kernel": f"kk_{stage}_kernel",
                     "peak_source": pk_kind},
        "clocks": clk,
        "e2e": {"value": total / (ems / 1e3) / 1e9, "unit": "GSa/s", "h2d_bytes_per_step": int(total),
                "d2h_bytes_per_step": int(slots * words * 4),
                "api": "rx_rt_submit_from (pinned host buffers, 4 streams, device BER count), host wall clock",
                "q_db_21ms_bins": [round(float(q), 2) for q in rtbins["q_db"]]},
        "paper_realtime_rate": "4 GS/s ADC (the paper's real-time figure on its own GPU)",
    }
    if not args.no_cpu_baseline:
        import oracle.kk as OK
        import oracle.wl as OW
        ns = 1 << 17
        t0_ = time.perf_counter()
        yo, _, _ = OK.kk_frontend(g.samples[:ns], g.in_scale, g.in_offset, lk.baud, lk.sps, lk.carrier_hz,
                                  lk.L_km)
        OW.wl_equalise(yo, OW.WLParams(mod="16qam"))
        dt = time.perf_counter() - t0_
        line["cpu_baseline"] = {"value": ns / dt / 1e9, "unit": "GSa/s", "cores": 1, "kind": "oracle",
                                "sample": f"first {ns} samples, FP64 numpy KK front end + widely-linear "
                                          "DD-LMS, one core"}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    if args.workload == "c4":
        bench_batch(args, rank, world, local)
        return
    if args.workload == "c5":
        bench_learned(args, rank, world, local)
        return
    if args.workload == "kk":
        bench_kk(args, rank, world, local)
        return
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2104_06311_gb300 import Receiver, build
    if not os.path.exists(build.OUT):
        build.build()
    import linksim as L

    n_sym = args.n_sym if args.workload == "c2" else min(args.n_sym, 1 << 22)
    lk, g = make_input(n_sym, args.workload)
    n = g.samples.shape[0]
    K = n // 2
    x = torch.from_numpy(g.samples).cuda()
    ref = torch.from_numpy(L.pack_bits(g.tx_bits).view(np.int32)).cuda()
    stream = torch.cuda.current_stream()
    mbits = L.bits_per_symbol(lk.mod)
    prec = {"fp32": 0, "fp16": 1, "bf16": 2}[args.precision]
    rx = Receiver(lk.baud, lk.L_km, D=lk.D, stream=stream, MOD=mbits, IN_SCALE=g.in_scale, PRECISION=prec,
                  DFT_TC=args.dft_tc)
    rx.reserve(n)
    out = rx.alloc_out(K + 64)

    def step(inp):
        rx.reset()
        _, c1, _, _ = rx.process(inp, out, 0)
        _, c2, _, _ = rx.process(None, out, c1)
        assert c1 + c2 == K
        return rx.ber(out["bits"], ref, K)

    for _ in range(args.warmup):
        e, nb, sync = step(x)
    ber = e / nb

    def barrier():
        if dist is not None:
            dist.barrier()

    clocks = ClockSampler(local)
    rx.set_param("PROFILE", 1)
    rx.profile(reset=True)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step(x)
    t1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = t0.elapsed_time(t1)
    prof = rx.profile(reset=True)
    rx.set_param("PROFILE", 0)
    ms = max_over_ranks(ms, dist, "cuda")
    value = whole_job_rate(n, args.steps, world, ms)
    launches = sum(v[1] for v in prof.values())

    # ---- end to end: pinned host samples -> device -> chain -> bits + BER back to the host
    e2e = None
    if not args.no_e2e:
        xh = torch.from_numpy(g.samples).pin_memory()
        xd = torch.empty_like(x)
        bits_h = torch.empty_like(out["bits"], device="cpu").pin_memory()

        def step_e2e():
            xd.copy_(xh, non_blocking=True)
            r = step(xd)
            bits_h.copy_(out["bits"], non_blocking=True)
            return r

        for _ in range(2):
            step_e2e()
        torch.cuda.synchronize()
        barrier()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            step_e2e()
        b.record(stream)
        torch.cuda.synchronize()
        ems = a.elapsed_time(b)
        ems = max_over_ranks(ems, dist, "cuda")
        e2e = {"value": whole_job_rate(n, args.steps, world, ems), "unit": "GSa/s",
               "h2d_bytes_per_step": int(x.numel() * x.element_size()),
               "d2h_bytes_per_step": int(out["bits"].numel() * 4 + 16)}

    # ---- roofline of the dominant kernel (stage times from CUDA events on the launch stream)
    pk, pk_kind = peaks()
    stage = max(("cdc", "eq", "bps"), key=lambda s: prof[s][0])
    T, W, S = 15, 128, 1024
    if stage == "eq":
        # algorithmic work: FIR 240 + LMS gradient 240 flop per sample-time (the
        # W pre-training and the inner phase search are executed but not counted)
        flop = EQ_FLOP_PER_SAMPLE_TIME * n
        peak, peak_note = alu_peak_tflops(stream)
        achieved = flop / (prof[stage][0] / args.steps / 1e3) / 1e12
        # DRAM bytes of one step's equaliser launches, scaled from an ncu capture of a
        # 2^22-symbol stream (each launch reads in proportion to its symbols); None until
        # a capture of the current kernel exists
        traffic = (EQ_DRAM_BYTES_PER_SYMBOL * K
                   if EQ_DRAM_BYTES_PER_SYMBOL and args.workload == "c2" and args.precision == "fp32" else None)
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": "eq_kernel", "peak_note": peak_note}
    else:
        per = {"cdc": 4 + 16, "bps": 16 + 16 + 1 + 0.25 * 2}[stage]   # bytes per sample-time
        bytes_ = per * n
        achieved = bytes_ / (prof[stage][0] / args.steps / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / pk["hbm_gbs"], "traffic": None, "kernel": stage}
    roof["peak_source"] = "measured (FMA chains, this run)" if roof["bound"] == "alu" else pk_kind
    # every stage against both ceilings (algorithmic bytes and flops per sample-time)
    alu_peak = alu_peak_tflops(stream)[0] * 1e12
    work = {"cdc": (4 + 16, 290.0),                                   # int8 in, 2 pols complex64 out
            "eq": (16 + 8, EQ_FLOP_PER_SAMPLE_TIME),
            "bps": (8 + 1 + 0.25, 32 * 11.0 + 8)}                        # per symbol-pol = per sample-time
    stage_roofs = {}
    for st_, (bpu, fpu) in work.items():
        t_s = prof[st_][0] / args.steps / 1e3
        if t_s <= 0:
            continue
        stage_roofs[st_] = {"ms": t_s * 1e3, "gsa_s": n / t_s / 1e9,
                            "hbm_frac": bpu * n / t_s / (pk["hbm_gbs"] * 1e9),
                            "alu_frac": fpu * n / t_s / alu_peak,
                            "bytes_per_sample_time": bpu, "flop_per_sample_time": fpu}

    line = {
        "metric": METRIC, "value": value, "unit": "GSa/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == 0 else f"f32 ({args.precision} CDC storage)",
        "data": f"synthetic (seeded linksim {lk.L_km:.0f} km link), resident in HBM",
        "config": {"workload": WORKLOADS[args.workload], "precision": args.precision,
                   "cdc_dft": ("tensor-core DFT-16 (FP32 accumulate)" if args.dft_tc and prec else
                               "register butterflies"),
                   "sample_times": n, "fft_n": int(rx.get_param("FFT_N")), "overlap": int(rx.get_param("OVERLAP")),
                   "taps": T, "bps_angles": 32, "segments_per_wave": 32,
                   "l2": f"inputs ({n * 4 >> 20} MiB) and CDC intermediates ({n * 16 >> 20} MiB) exceed L2; no flush",
                   "parallelism": f"replicas x{world}" if world > 1 else "single stream"},
        "decoded_gbps": value / 2 * 2 * mbits,
        "hbm_roofline_frac": value / (pk["hbm_gbs"] / 4.25),
        "ber": ber, "ber_sync": sync,
        "stage_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
        "stage_rooflines": stage_roofs,
        "alu_peaks_measured": {"fp32_tflops": _ALU_PEAK.get("fp32"), "fp64_tflops": _ALU_PEAK.get("fp64"),
                               "fp32_nominal_at_max_clock": N_SM * FP32_LANES_PER_SM * 2 * 2.07e9 / 1e12},
        "gpu_launches": int(launches),
        "roofline": roof,
        "clocks": clk,
        "e2e": e2e,
    }

    # ---- CPU baseline: the oracle as it stands, bounded sample, rank 0 at N = 1
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ns = min(args.cpu_sample, n)
        orc, dt, p = cpu_oracle_run(g, ns)
        line["cpu_baseline"] = {"value": ns / dt / 1e9, "unit": "GSa/s", "cores": 1, "kind": "oracle",
                                "sample": f"first {ns} sample-times of the workload, FP64 numpy oracle, one core"}
        line["cpu_baseline_all_cores"] = oracle_all_cores(g, min(ns, 1 << 20))
        line["oracle_parity_sample"] = oracle_parity(g, x, ns, lk, mbits, prec, stream, orc, p)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def oracle_parity(g, x, ns, lk, mbits, prec, stream, orc_free, p):
    """Bits of the CUDA chain against the FP64 oracle on the first ns sample-times.

    The oracle runs on its own decisions (`orc_free`, the timed baseline run);
    a second oracle run follows the device's choice at near-ties of its
    discrete decisions (inner BPS sums within 1e-4, tracker roundings within
    2e-3 of half-way: both candidates correct), which is the run the bits are
    compared with.  Exempt: bits whose oracle soft value lies within 1e-5 of a
    decision boundary, and symbols at an outer BPS near-tie."""
    import numpy as np
    import torch
    import linksim as L
    import oracle as O
    sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests"))
    from chain_helpers import boundary_mask, bps_near_tie, device_ties, inner_capacity
    from paper_2104_06311_gb300 import Receiver
    K = ns // 2
    rxs = Receiver(lk.baud, lk.L_km, D=lk.D, stream=stream, MOD=mbits, IN_SCALE=g.in_scale, PRECISION=prec,
                   INNER_TRACE=inner_capacity(p.resolved(), K))
    o2 = rxs.run_stream(x[:ns].contiguous())
    torch.cuda.synchronize()
    gb = L.unpack_bits(o2["bits"].cpu().numpy().view(np.uint32), K * mbits)
    ties = device_ties(rxs, p.resolved(), K)
    tr = {}
    orc = O.run_chain(g.samples[:ns], p, tr, ties)
    exempt = boundary_mask(orc["z"], p.mod) | np.repeat(bps_near_tie(orc["y"], p.resolved()), mbits, axis=1)
    diff = gb != orc["bits"]
    eo, no, _ = O_ber(orc["bits"], g.tx_bits[:, :K * mbits], p)
    e3, n3, _ = rxs.ber(o2["bits"], torch.from_numpy(L.pack_bits(g.tx_bits[:, :K * mbits]).view(np.int32)).cuda(), K)
    rxs.close()
    return {"bits": int(gb.size), "mismatched_bits": int(diff.sum()), "exempt_mismatches": int((diff & exempt).sum()),
            "non_exempt_mismatches": int((diff & ~exempt).sum()),
            "mismatched_bits_vs_free_oracle": int(np.sum(gb != orc_free["bits"])),
            "near_tie_choices_followed": len(tr["ties"]),
            "tracker_identical": bool(ties["acq_units"] == tr["acq_units"] and ties["wave_units"] == tr["wave_units"]),
            "ber_oracle": eo / max(no, 1), "ber_gpu": e3 / max(n3, 1)}


def O_ber(bits, tx_bits, p):
    import oracle as O
    return O.ber_sync_count(bits, tx_bits, p.mod, p.acq_len(bits.shape[1] // p.bits))


if __name__ == "__main__":
    main()
