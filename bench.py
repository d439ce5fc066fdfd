#!/usr/bin/env python3
"""Benchmark of the per-time-step path on the 6-level synthetic streamer.

Workload (one "step"): the 16 mm cube on a 64^3 base grid refined 6 levels
around a synthetic positive streamer (2.4e6 leaf cells), 25 kV between the
z plates: reset the densities from a device-resident copy, Eq. 5 charge
right-hand side, FMG Poisson solve to relative residual 1e-8, field, time
step, one Heun fluid step with two more Poisson solves to 1e-8.  Three
Poisson solves per step; the metric is solves per second (and leaf
Mcells x V-cycles per second).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

N > 1 runs under torchrun as N independent replicas (one per GPU, no data
exchange): the path has no exchange step between independent solves.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = "streamer6"
TOL = 1e-8
MAX_CYCLES = 40
SOLVES_PER_STEP = 3
PAPER_VCYCLES = 2   # V-cycles per potential update in the paper's runs (Sec. 2.1.2)
L2_BYTES = 129 * 2 ** 20
NO_GRAPHS = False
NO_PDL = False
PERSIST = False
ROW_KERNELS = None


# DRAM bytes (read + write) per k_fcolor launch, mean over the colour
# passes of one kernel-bench sweep of every level of the benchmark mesh (the
# mix the roofline's achieved figure averages); taken with
#   python bench.py --mode kernels &&
#   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum \
#       --clock-control none -k regex:k_fcolor --csv --log-file fcolor_dram.csv \
#       python bench.py --mode kernels
# Mean of the first 36 launches (the kernel-bench mix): 3.118 MB read, 0
# written, taken with the command above.
FCOLOR_TRAFFIC_PER_LAUNCH = 3118798
FCOLOR_TRAFFIC_NOTE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum, mean over the 36 k_fcolor_half launches "
                       "of one kernel-bench sweep of every level (cold caches): 0.85x the algorithmic bytes per "
                       "launch, the colour's stores staying in L2")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-threads", type=int, default=0,
                    help="--impl reference: oracle threads (0 = all host cores)")
    ap.add_argument("--no-profile", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-paper", action="store_true", help="skip the fixed 2-V-cycle (paper) schedule")
    ap.add_argument("--no-large", action="store_true", help="skip the 1e8-cell mesh (streamer9)")
    ap.add_argument("--no-axi", action="store_true", help="skip the axisymmetric (2-D) variant")
    ap.add_argument("--no-graphs", action="store_true",
                    help="launch the same kernels from the host instead of CUDA graphs "
                         "(profilers cannot see kernels inside conditional graph nodes)")
    ap.add_argument("--persistent", action="store_true",
                    help="run V-cycles as one persistent cooperative launch instead of per-level launches")
    ap.add_argument("--row-kernels", type=int, default=None, metavar="MIN_BOXES",
                    help="levels of at least MIN_BOXES boxes run the row kernels (library default 2048; 0: all)")
    ap.add_argument("--no-pdl", action="store_true",
                    help="launch the solver kernels without programmatic dependent launch")
    ap.add_argument("--workload", default=WORKLOAD,
                    help="mesh of --mode kernels and --mode vcycle (the step and its metric use streamer6)")
    ap.add_argument("--mode", default="step",
                    choices=["step", "vcycle", "kernels", "batch", "large", "axi", "learned", "network"],
                    help="vcycle: build the workload, then only run --steps V-cycles; "
                         "batch: only the batched solves, --steps solves with the default "
                         "schedule (small, fixed launch sequences for ncu captures); "
                         "large: the 1e8-cell mesh alone; axi: the axisymmetric variant alone; "
                         "network: the network kernels alone (--steps launches each)")
    ap.add_argument("--net-samples", type=int, default=4096,
                    help="--mode network only: synthetic samples (boxes) per launch")
    ap.add_argument("--batch-solves", type=int, default=256,
                    help="--mode batch only: solve the first N of the 256 batched problems (small ncu captures)")
    ap.add_argument("--batch-schedule", type=int, nargs=2, default=None, metavar=("SHAPE", "BLOCKS_PER_SM"),
                    help="--mode batch only: restriction schedule (0-3 tiles, 4 columns) and blocks per SM "
                         "instead of the library default (tiles 0, 4 per SM)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value: float, dev=None) -> float:
    """Max of a per-rank float over all ranks of the initialised process
    group (NCCL on GPUs, gloo in the CPU tests); the value itself on one
    process.  Replicas are timed by their slowest rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, ms_max: float) -> float:
    """Units per second of the whole job: every rank's units over the time
    of the slowest rank (weak scaling: the per-rank work is fixed)."""
    return units_per_rank * world / (ms_max * 1e-3)


def bf16_peak_tflops():
    """Measured dense BF16 matmul throughput of this GPU (burst), TFLOP/s."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f).get("bf16_tflops", 1900.0))
    return 1900.0


def network_kernels(net, n, reps):
    """Forward and training-gradient-pass timing of the network kernels over
    the first n recorded samples, against the measured BF16 peak."""
    bf16_peak = bf16_peak_tflops()
    kern = {}
    for kind, name in ((0, "forward (k_cnn_forward)"), (1, "gradient pass (k_cnn_train + reduce)")):
        us, fl, tf = net.kernel_bench(kind, n, reps)
        kern[name] = {"us": round(us, 1), "tflops_model": round(fl / (us * 1e-6) / 1e12, 2),
                      "tensor_tflops": round(tf / (us * 1e-6) / 1e12, 2),
                      "tensor_frac_of_bf16_peak": round(tf / (us * 1e-6) / 1e12 / bf16_peak, 4)}
    note = ("%d boxes per launch, CUDA events; model FLOPs 16416 per voxel forward, 3x for a gradient pass; "
            "tensor FLOPs = the tcgen05 MMAs issued per box (forward 135 of 128x16x16; a gradient pass adds "
            "405 of 128x16x16 and 288 of 128x48x16), discarded tile rows included; peak = measured BF16 "
            "burst %.1f TFLOP/s" % (n, bf16_peak))
    return kern, note


def run_network(args):
    """The network kernels alone on seeded synthetic samples (inputs uniform
    in [-1, 1], targets normal with deviation 0.3): a small command for
    kernel captures."""
    import torch
    import synth
    import __graft_entry__
    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    __graft_entry__.build()
    import paper_1708_08434_gb300 as pkg
    n = args.net_samples
    net = pkg.Network(n, n)
    rng = np.random.default_rng(7)
    p = synth.cnn_initial_params().astype(np.float32)
    net.set_params(p)
    net.load_samples(rng.uniform(-1.0, 1.0, (n, 1000, 2)).astype(np.float32),
                     (0.3 * rng.standard_normal((n, 512))).astype(np.float32))
    kern, note = network_kernels(net, n, max(1, args.steps))
    net.close()
    print(json.dumps({"mode": "network", "samples": n, "network_kernels": kern, "note": note}), flush=True)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


_FP64 = {}


def fp64_rate():
    """Measured FP64-pipe throughput in G instructions/s (probed once)."""
    if "v" not in _FP64:
        _FP64["v"] = fp64_peak()
    return _FP64["v"]["ginstr_per_s"]


def fp64_peak():
    """The FP64 pipe's throughput measured on this GPU (sm_fp64_probe: 8
    independent fused multiply-add chains per thread on every SM), with the
    SM clocks sampled while it ran: G FP64 instructions/s."""
    import torch
    import paper_1708_08434_gb300 as pkg
    pkg.fp64_probe(1 << 12)
    torch.cuda.synchronize()
    clk = Clocks(torch.cuda.current_device())
    clk.start()
    rate, ms = pkg.fp64_probe(1 << 18)
    clocks = clk.stop()
    return {"ginstr_per_s": round(rate / 1e9, 1), "probe_ms": round(ms, 2), "clocks": clocks,
            "how": "sm_fp64_probe: 8 x 256 threads per SM, 8 independent DFMA chains each"}


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def start(self):
        """Start sampling every 100 ms; returns once the first sample (taken
        before the region, and left out) has arrived."""
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.p.stdout.readline()
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def build_gpu_case(precision=0):
    import torch
    import synth
    import paper_1708_08434_gb300 as pkg
    dom, st = synth.workload(WORKLOAD)
    g = pkg.Solver(dom, max_boxes=8192 if WORKLOAD == "streamer6" else 1 << 18, precision=precision)
    if NO_GRAPHS:
        g.set_graphs(False)
    if NO_PDL:
        g.set_pdl(False)
    if PERSIST:
        g.set_persistent(True)
    if ROW_KERNELS is not None:
        g.set_row_kernels(ROW_KERNELS)
    g.build_octree()
    synth.refine_all(dom, st, g.level_ijk, g.refine_level)
    t = g.tables()
    ne, ni = synth.streamer_densities(dom, st, t["level"], t["ijk"])
    g.set_table(synth.coefficient_table())
    return dom, st, g, t, ne, ni


def run_batch_only(args):
    import torch
    import __graft_entry__
    torch.cuda.set_device(0)
    __graft_entry__.build()
    b, _ = make_batch_workload(args.batch_solves)
    if args.no_graphs:
        b.set_graphs(False)
    if args.batch_schedule:
        b.set_schedule(*args.batch_schedule)
    for _ in range(args.steps):
        b.phi.zero_()
        rc, cyc, rel = b.solve(TOL, MAX_CYCLES)
    torch.cuda.synchronize()
    print(json.dumps({"mode": "batch", "solves": args.steps, "max_corrections": int(cyc.max())}), flush=True)
    b.close()


def run_large(args):
    import torch
    import __graft_entry__
    torch.cuda.set_device(0)
    __graft_entry__.build()
    print(json.dumps(large_mesh()), flush=True)


def run_axi(args):
    import torch
    import __graft_entry__
    torch.cuda.set_device(0)
    __graft_entry__.build()
    dev = torch.device("cuda", 0)
    print(json.dumps({"mode": "axi", **bench_axisymmetric(args, dev, 1)}), flush=True)


def large_mesh():
    """The largest mesh of the paper's runs (~1e8 cells, streamer9): FMG to
    1e-8, one Heun step, and the FP64 V-cycle and smoother against their
    rooflines; the same for the mixed-precision form (about 16 GB of device
    memory per solver, one solver at a time)."""
    import torch
    import synth
    import paper_1708_08434_gb300 as pkg
    Q, E0 = synth.E_CHARGE, synth.EPS0
    dom, st = synth.workload("streamer9")
    out = {"mode": "large", "workload": "streamer9"}
    ne = ni = None
    for prec, name in ((0, "fp64"), (pkg.MIXED, "mixed")):
        t0 = time.perf_counter()
        g = pkg.Solver(dom, max_boxes=1 << 18, precision=prec)
        if ROW_KERNELS is not None:
            g.set_row_kernels(ROW_KERNELS)
        g.build_octree()
        synth.refine_all(dom, st, g.level_ijk, g.refine_level)
        g.set_table(synth.coefficient_table())
        if ne is None:
            t = g.tables()
            ne, ni = synth.streamer_densities(dom, st, t["level"], t["ijk"])
            out["boxes"], out["leaf_cells"], out["levels"] = g.n_boxes, g.n_leaves * 512, g.n_levels
        g.upload(pkg.NE, ne)
        g.upload(pkg.NI, ni)
        g.charge_rhs(Q, E0)
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t0

        def ev(fn):
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(g.stream)
            r = fn()
            b.record(g.stream)
            torch.cuda.synchronize()
            return a.elapsed_time(b), r

        g.fmg(TOL, MAX_CYCLES)  # warm-up (captures the graphs)
        g.charge_rhs(Q, E0)
        fmg_ms, (rc, rel, cyc) = ev(lambda: g.fmg(TOL, MAX_CYCLES))
        g.compute_field()
        dt = g.dt_limit(Q, E0)
        step_ms, (rc2, dtn, c1, c2) = ev(lambda: g.advance(dt, Q, E0, TOL, MAX_CYCLES))
        r = {"setup_s": round(setup_s, 1), "fmg_ms": round(fmg_ms, 2), "fmg_cycles": cyc,
             "heun_step_ms": round(step_ms, 2), "step_cycles": [c1, c2],
             "solves_per_s": round(3 / ((fmg_ms + step_ms) * 1e-3), 3)}
        peak, _ = measured_peaks()
        kc = pkg.K_VCYCLE if prec == 0 else pkg.K_VCYCLE32
        us, n, by, fl = g.kernel_bench(kc, 5)
        r["vcycle"] = {"us": round(us, 1), "bytes": int(by), "hbm_frac": round(by / (us * 1e-6) / 1e9 / peak, 4)}
        r["vcycle"]["gbs"] = round(by / (us * 1e-6) / 1e9, 1)
        if prec == 0:
            us, n, by, fl = g.kernel_bench(pkg.K_SMOOTH, 5)
            r["colour_pass"] = {"avg_launch_us": round(us, 2), "launches": n,
                                "gbs": round(by / (us * 1e-6) / 1e9, 1),
                                "hbm_frac": round(by / (us * 1e-6) / 1e9 / peak, 4),
                                "kernels": "k_fcolor_rows on levels of >= 2048 boxes, k_fcolor_half below"}
        out[name] = r
        g.close()
        del g
        torch.cuda.empty_cache()
    return out


def run_gpu(args):
    import numpy as np
    import torch
    import synth
    import paper_1708_08434_gb300 as pkg
    import __graft_entry__
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    __graft_entry__.build()
    Q, E0 = synth.E_CHARGE, synth.EPS0
    dom, st, g, t, ne, ni = build_gpu_case()
    n_boxes = g.n_boxes
    leaf_cells = g.n_leaves * 512
    dev = torch.device("cuda", torch.cuda.current_device())
    ne_d = torch.from_numpy(ne).to(dev)
    ni_d = torch.from_numpy(ni).to(dev)
    ne_h = torch.from_numpy(ne).pin_memory()
    ni_h = torch.from_numpy(ni).pin_memory()
    phi_out = torch.empty((n_boxes, 512), dtype=torch.float64).pin_memory()
    ne_out = torch.empty((n_boxes, 512), dtype=torch.float64).pin_memory()
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=dev)
    stream = g.stream

    def make_step(g):
        def step(host_io=False):
            if host_io:
                g.upload(pkg.NE, ne_h)
                g.upload(pkg.NI, ni_h)
            else:
                g.var(pkg.NE).copy_(ne_d)
                g.var(pkg.NI).copy_(ni_d)
            g.charge_rhs(Q, E0)
            rc0, rel0, c0 = g.fmg(TOL, MAX_CYCLES)
            g.compute_field()
            dt = g.dt_limit(Q, E0)
            rc1, dtn, c1, c2 = g.advance(dt, Q, E0, TOL, MAX_CYCLES)
            if host_io:
                g.download(pkg.PHI, phi_out)
                g.download(pkg.NE, ne_out)
            assert rc0 == 0 and rc1 == 0, (rc0, rc1)
            return c0 + c1 + c2

        def timed(n, host_io=False):
            total_ms, cycles = 0.0, 0
            l0 = g.launch_count()
            for _ in range(n):
                flush.fill_(1)
                torch.cuda.synchronize()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                cycles += step(host_io)
                b.record(stream)
                torch.cuda.synchronize()
                total_ms += a.elapsed_time(b)
            return total_ms, cycles, g.launch_count() - l0
        return step, timed

    step, timed = make_step(g)

    if args.mode == "kernels":
        # one kernel-bench pass of the colour kernel over every level and one
        # V-cycle (the launches the roofline times; a small command for ncu)
        g.var(pkg.NE).copy_(ne_d)
        g.var(pkg.NI).copy_(ni_d)
        g.charge_rhs(Q, E0)
        out = {"mode": "kernels"}
        for kc, name in ((pkg.K_SMOOTH, "k_fcolor"), (pkg.K_VCYCLE, "vcycle")):
            us, n, by, fl = g.kernel_bench(kc, 1)
            out[name] = {"avg_launch_us": round(us, 3), "launches": n, "bytes_per_launch": round(by)}
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps(out), flush=True)
        g.close()
        return
    if args.mode == "vcycle":
        g.var(pkg.NE).copy_(ne_d)
        g.var(pkg.NI).copy_(ni_d)
        g.charge_rhs(Q, E0)
        rel = g.vcycles(args.steps)
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"mode": "vcycle", "cycles": args.steps, "rel": rel}), flush=True)
        g.close()
        return
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = Clocks(torch.cuda.current_device())
    clk.start()
    ms, cycles, launches = timed(args.steps)
    clocks = clk.stop()
    if world > 1:
        dist.barrier()
    ms = max_over_ranks(ms, dev)
    # the FMG solve alone (the unit the CPU oracle's single-solve figure times)
    fmg_only = None
    if not args.no_profile:
        g.var(pkg.NE).copy_(ne_d)
        g.var(pkg.NI).copy_(ni_d)
        g.charge_rhs(Q, E0)
        g.fmg(TOL, MAX_CYCLES)
        torch.cuda.synchronize()
        fa = torch.cuda.Event(enable_timing=True)
        fb = torch.cuda.Event(enable_timing=True)
        fa.record(stream)
        for _ in range(10):
            g.charge_rhs(Q, E0)
            _, _, fcyc = g.fmg(TOL, MAX_CYCLES)
        fb.record(stream)
        torch.cuda.synchronize()
        fmg_only = {"solves_per_s": round(10 / (fa.elapsed_time(fb) * 1e-3), 2), "vcycles": fcyc,
                    "note": "FMG to 1e-8 from phi = 0 on the same workload, 10 solves timed with CUDA events "
                            "(L2 not flushed)"}
    # where the step's time goes: CUDA events on the library's stream
    # between the calls of one step (after an L2 flush, like a timed step;
    # host gaps such as the time-step read are inside the phase that waits),
    # and the fixed and per-cycle cost of a solve from warm-started solves
    # run to tol 0 for 1 and 4 V-cycles
    step_phases = None
    if not args.no_profile:
        step_phases = phase_breakdown(g, ne_d, ni_d, flush, Q, E0)
    # end to end through the C ABI with host buffers (H2D + D2H every step)
    e2e_ms, _, _ = timed(args.steps, host_io=True)
    e2e_ms = max_over_ranks(e2e_ms, dev)
    # roofline of the dominant kernel: a colour pass of the red-black
    # smoother (k_fcolor), timed with CUDA events around a graph of its
    # launches in the V-cycle mix (every level, both colours), or with
    # --persistent the persistent V-cycle kernel (one cooperative launch per
    # V-cycle); beside it the whole FP64 V-cycle of the per-level path
    roof = None
    f64 = None
    if not args.no_profile:
        fp64_rate()
        f64 = _FP64["v"]
    if not args.no_profile:
        kclass = pkg.K_PERSIST if PERSIST else pkg.K_SMOOTH
        us, kn, kbytes, kflops = g.kernel_bench(kclass, 20)
        peak, kind = measured_peaks()
        gbs = kbytes / (us * 1e-6) / 1e9
        roof = {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                "frac": round(gbs / peak, 4), "peak_kind": kind + " (copy bandwidth)",
                "traffic": None if PERSIST else FCOLOR_TRAFFIC_PER_LAUNCH,
                "traffic_note": None if PERSIST else FCOLOR_TRAFFIC_NOTE,
                "kernel": "k_persistx" if PERSIST else "k_fcolor", "launches": kn,
                "avg_launch_us": round(us, 3), "bytes_per_launch": round(kbytes),
                "bytes_model": ("12 B per cell of the level and colour pass: the other colour's potential "
                                "and this colour's G read (4 + 4), this colour written (4); int64 fixed point"
                                if not PERSIST else "V-cycle model, 24 B per cell and sweep"),
                "fp64_instr_per_launch": round(kflops),
                "note": ("mean over %d graph-launched colour passes of every level "
                         "(the V-cycle mix), CUDA events on the launching stream; the level "
                         "kernels use no FP64 instruction" % kn) if not PERSIST else
                        ("mean over %d launches, each one whole V-cycle, CUDA events on the "
                         "launching stream; bytes from the per-level model" % kn)}
        if not PERSIST:
            vus, vn, vbytes, vinstr = g.kernel_bench(pkg.K_VCYCLE, 10)
            roof["vcycle"] = {"us": round(vus, 2), "cycles": vn, "bytes": round(vbytes),
                              "gbs": round(vbytes / (vus * 1e-6) / 1e9, 1),
                              "hbm_frac": round(vbytes / (vus * 1e-6) / 1e9 / peak, 4),
                              "fp64_instr": round(vinstr),
                              "note": "whole FP64 V-cycle (fixed-point level kernels, FP64 level-0 solve), "
                                      "per-level launches in a CUDA graph, bytes from the per-level model"}
    # the same step with the mixed-precision solve (FP32 error equation in an
    # FP64 defect-correction loop) on a second solver of the same workload
    mixed = None
    if not args.no_mixed:
        gm = build_gpu_case(precision=pkg.MIXED)[2]
        step_m, timed_m = make_step(gm)
        for _ in range(args.warmup):
            step_m()
        torch.cuda.synchronize()
        mms, mcyc, mlaunch = timed_m(args.steps)
        mms = max_over_ranks(mms, dev)
        mixed = {"value": round(SOLVES_PER_STEP * args.steps * world / (mms * 1e-3), 3),
                 "unit": "solves/s", "ms_per_step": round(mms / args.steps, 4),
                 "corrections_per_step": mcyc / args.steps, "gpu_launches": mlaunch,
                 "speedup_vs_fp64": round(ms / mms, 3),
                 "dtype": "f32 error equation, f64 residual/accumulation/level-0 solve"}
        if not args.no_profile:
            vus32, _, vby32, _ = gm.kernel_bench(pkg.K_VCYCLE32, 10)
            mixed["fp32_vcycle_us"] = round(vus32, 2)
        # accuracy of the form: the same charge solved by the mixed form to
        # 1e-8 and by the FP64 path to 1e-12 (the FP64 path matches the CPU
        # oracle element by element); potential and |E| on leaf cells
        for gg in (g, gm):
            gg.var(pkg.NE).copy_(ne_d)
            gg.var(pkg.NI).copy_(ni_d)
            gg.charge_rhs(Q, E0)
        g.fmg(1e-12, 60)
        gm.fmg(TOL, MAX_CYCLES)
        g.compute_field()
        gm.compute_field()
        leaf = torch.from_numpy(np.asarray(g.tables()["leaf"], dtype=np.int64)).to(dev)
        p64, p32 = g.var(pkg.PHI)[leaf], gm.var(pkg.PHI)[leaf]
        e64, e32 = g.var(pkg.EMAG)[leaf], gm.var(pkg.EMAG)[leaf]
        mixed["error_vs_fp64"] = {
            "phi_max_rel": float((p32 - p64).abs().max() / p64.abs().max()),
            "emag_max_rel": float((e32 - e64).abs().max() / e64.abs().max()),
            "reference": "FP64 path converged to 1e-12 (element-wise parity with the CPU oracle)"}
        gm.close()
    # field (Sec. 2.3) and one Euler stage of the fluid update (Eq. 2-3, 6-7)
    # against their rooflines: CUDA events around 20 calls each; the field
    # call is the refinement-face fill + k_field, the stage is the face
    # fill, the refinement fluxes, k_update and the density restriction
    fluid = None
    if not args.no_profile:
        g.var(pkg.NE).copy_(ne_d)
        g.var(pkg.NI).copy_(ni_d)
        g.charge_rhs(Q, E0)
        g.fmg(TOL, MAX_CYCLES)
        g.compute_field()
        dt = g.dt_limit(Q, E0)

        def per_call(fn, n=20):
            fn()
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(n):
                fn()
            b.record(stream)
            torch.cuda.synchronize()
            return a.elapsed_time(b) * 1e3 / n

        peak, _ = measured_peaks()
        fpk = f64["ginstr_per_s"] if f64 else None
        fus = per_call(g.compute_field)
        sus = per_call(lambda: g.fluid_stage(dt))
        fluid = {"fp64_peak": f64}
        # FP64 instructions per leaf cell as counted by ncu on this workload
        # (32 x smsp__inst_executed_pipe_fp64 / leaf cells: k_field 17.4 with
        # the FP64 square root of |E|, stage-1 k_update 64.0); bytes:
        # compulsory traffic
        for name, us, bpc, ipc in (("field (k_field)", fus, 16.0, 17.4), ("euler stage (k_update)", sus, 72.0, 64.0)):
            fluid[name] = {"us": round(us, 2), "gbs": round(leaf_cells * bpc / (us * 1e-6) / 1e9, 1),
                           "hbm_frac": round(leaf_cells * bpc / (us * 1e-6) / 1e9 / peak, 4),
                           "fp64_ginstr": round(leaf_cells * ipc / (us * 1e-6) / 1e9, 1),
                           "fp64_frac": (round(leaf_cells * ipc / (us * 1e-6) / 1e9 / fpk, 4) if fpk else None),
                           "model_per_leaf_cell": {"bytes": bpc, "fp64_instr": ipc}}
    # the paper's schedule (Sec. 2.1.2, 2.4): one FMG solve, then Heun steps
    # with exactly two V-cycles per potential update and the time step from
    # the limits of Sec. 2.4
    paper = None
    if not args.no_paper:
        g.var(pkg.NE).copy_(ne_d)
        g.var(pkg.NI).copy_(ni_d)
        g.charge_rhs(Q, E0)
        g.fmg(TOL, MAX_CYCLES)
        g.compute_field()
        dt = g.dt_limit(Q, E0)
        for _ in range(2):
            _, dt, _, _ = g.advance(dt, Q, E0, 0.0, PAPER_VCYCLES)
        nsteps = 20
        l0 = g.launch_count()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(nsteps):
            _, dt, c1, c2 = g.advance(dt, Q, E0, 0.0, PAPER_VCYCLES)
            assert (c1, c2) == (PAPER_VCYCLES, PAPER_VCYCLES)
        b.record(stream)
        torch.cuda.synchronize()
        pms = a.elapsed_time(b)
        paper = {"steps_per_s": round(nsteps * world / (pms * 1e-3), 2),
                 "solves_per_s": round(2 * nsteps * world / (pms * 1e-3), 2),
                 "ms_per_step": round(pms / nsteps, 4),
                 "mcells_vcycles_per_s": round(leaf_cells * 4 * nsteps * world / (pms * 1e-3) / 1e6, 1),
                 "steps": nsteps, "gpu_launches": g.launch_count() - l0,
                 "schedule": "2 V-cycles per solve, 2 solves per Heun step, dt from the Sec. 2.4 limits "
                             "(host reads dt each step)"}
    # refinement criterion (Eq. 8) and regridding on the benchmark mesh:
    # flags with the paper's constants, then a regrid that changes the mesh
    # (a stricter c0 refines), timed with CUDA events, and the way back
    regrid = None
    if not args.no_paper:
        g.var(pkg.NE).copy_(ne_d)
        g.var(pkg.NI).copy_(ni_d)
        g.charge_rhs(Q, E0)
        g.fmg(TOL, MAX_CYCLES)
        g.compute_field()

        def timed_ms(fn):
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            out = fn()
            b.record(stream)
            torch.cuda.synchronize()
            return a.elapsed_time(b), out

        g.refine_flags()  # warm-up
        warm_regrid(False)
        fl_ms, flags = timed_ms(lambda: g.refine_flags())
        nb0 = g.n_boxes
        strict = g.refine_flags(0.25, 1.2, 0.125, 30e-6, 3)
        room = (8192 - nb0) // 8 - 16            # the solver's max_boxes
        strict[np.where(strict == 1)[0][max(room, 0):]] = 0
        rg_ms, (nref, nder, ndrop) = timed_ms(lambda: g.regrid(strict))
        nb1 = g.n_boxes
        regrid = {"flags_ms": round(fl_ms, 3), "paper_flags": {"refine": int((flags == 1).sum()),
                                                                "derefine": int((flags == -1).sum())},
                  "regrid_ms": round(rg_ms, 3), "boxes": [nb0, nb1], "refined": nref, "derefined": nder,
                  "dropped": ndrop, "criterion": "c0=0.25 (paper: 1), c1=1.2, buffer 3; flags with the paper's "
                                                 "c0=1, c0_deref=1/8, dx_deref=30 um"}
    large = None if (args.no_large or rank != 0) else large_mesh()
    configs = None if (args.no_large or rank != 0) else bench_configs()
    axi = None if args.no_axi else bench_axisymmetric(args, dev, world)
    batched = None if args.no_batch else bench_batch(args, dev, world)
    learned = None if args.no_learned else bench_learned(args, dev, world)
    steps = args.steps
    solves = SOLVES_PER_STEP * steps * world
    value = whole_job_rate(SOLVES_PER_STEP * steps, world, ms)
    e2e_value = whole_job_rate(SOLVES_PER_STEP * steps, world, e2e_ms)
    mcell_vc = leaf_cells * cycles * world / (ms * 1e-3) / 1e6
    res = {
        "metric": "Poisson solves/s to rel residual 1e-8 (octree FMG + Heun step, 3 solves/step)",
        "value": round(value, 3), "unit": "solves/s", "n_gpus": world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": round(ms / steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "leaf_cells": leaf_cells, "boxes": n_boxes,
                   "levels": g.n_levels, "tol": TOL, "nu": [2, 2],
                   "l2": "flushed between steps (258 MB write)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "mcells_vcycles_per_s": round(mcell_vc, 2),
        "vcycles_per_step": cycles / steps,
        "e2e": {"value": round(e2e_value, 3), "unit": "solves/s",
                "h2d_bytes_per_step": int(2 * ne_h.numel() * 8),
                "d2h_bytes_per_step": int(2 * phi_out.numel() * 8)},
        "gpu_launches": launches,
        "clocks": clocks,
        "fmg_only": fmg_only,
        "step_phases": step_phases,
        "roofline": roof,
        "mixed_precision": mixed,
        "field_and_fluid": fluid,
        "paper_schedule": paper,
        "large_mesh": large,
        "other_configs": configs,
        "regrid": regrid,
        "axisymmetric": axi,
        "batched": batched,
        "learned_warm_start": learned,
    }
    if rank == 0 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline()
    g.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(res), flush=True)


def phase_breakdown(g, ne_d, ni_d, flush, q, eps, reps=10):
    """Mean microseconds of each call of the benchmark step (CUDA events
    recorded on the library's stream between the calls, L2 flushed before
    each step), and the cost of a warm-started FP64 solve as a fixed part
    plus a part per V-cycle, from solves of 1 and 4 cycles (tol 0)."""
    import torch
    import paper_1708_08434_gb300 as pkg
    s = g.stream
    names = ("density copy", "charge", "fmg", "field", "dt limit", "heun step")
    acc = [0.0] * len(names)
    for _ in range(reps):
        flush.fill_(1)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 1)]
        ev[0].record(s)
        g.var(pkg.NE).copy_(ne_d)
        g.var(pkg.NI).copy_(ni_d)
        ev[1].record(s)
        g.charge_rhs(q, eps)
        ev[2].record(s)
        g.fmg(TOL, MAX_CYCLES)
        ev[3].record(s)
        g.compute_field()
        ev[4].record(s)
        dt = g.dt_limit(q, eps)
        ev[5].record(s)
        g.advance(dt, q, eps, TOL, MAX_CYCLES)
        ev[6].record(s)
        torch.cuda.synchronize()
        for i in range(len(names)):
            acc[i] += ev[i].elapsed_time(ev[i + 1]) * 1e3
    out = {n: round(a / reps, 1) for n, a in zip(names, acc)}

    def solve_us(k):
        g.solve(0.0, k)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s)
        for _ in range(reps):
            g.solve(0.0, k)
        b.record(s)
        torch.cuda.synchronize()
        return a.elapsed_time(b) * 1e3 / reps

    t1, t4 = solve_us(1), solve_us(4)
    per_cycle = (t4 - t1) / 3.0
    out["solve_cost"] = {"fixed_us": round(t1 - per_cycle, 1), "per_vcycle_us": round(per_cycle, 1),
                         "note": "warm-started FP64 solve (CUDA graph with a device-side loop): scale, "
                                 "conversions and ghost fills before and after the loop, the graph launch "
                                 "and the read of the cycle count; per V-cycle the cycle and its stopping test"}
    return out


def bench_configs():
    """The other single-GPU configurations at their own sizes:
    uniform64 -- FP64 V(2,2) cycles to rel residual 1e-10 on the unit cube,
    64^3 cells in 512 boxes, Gaussian charge plus 1e-3 seeded noise: solves
    from phi = 0 and FMG, timed with CUDA events;
    streamer8 -- the mixed-precision form on the 8-level mesh (1.7e7 leaf
    cells): FMG to 1e-8, and its potential and |E| against the FP64 path
    solved to 1e-12 on the same charge (the FP64 path matches the CPU oracle
    element by element)."""
    import numpy as np
    import torch
    import synth
    import paper_1708_08434_gb300 as pkg
    Q, E0 = synth.E_CHARGE, synth.EPS0
    out = {}

    def ev(g, fn, n=1):
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(g.stream)
        for _ in range(n):
            r = fn()
        b.record(g.stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / n, r

    dom = synth.domain_uniform_cube(64)
    g = pkg.Solver(dom, 1024)
    g.build_octree()
    t = g.tables()
    rho = synth.gaussian_charge(dom, t["level"], t["ijk"], np.arange(len(t["level"])))
    g.upload(pkg.RHO, rho)
    g.charge_rhs(1.0, 1.0, True)
    cells = g.n_leaves * 512

    def from_zero():
        g.var(pkg.PHI).zero_()
        return g.solve(1e-10, 100)

    from_zero()
    ms_v, (rc, rel, cyc) = ev(g, from_zero, 10)
    ms_f, (rcf, relf, cycf) = ev(g, lambda: g.fmg(1e-10, 100), 10)
    us_vc, _, by_vc, _ = g.kernel_bench(pkg.K_VCYCLE, 20)
    out["uniform64"] = {
        "cells": cells, "levels": g.n_levels, "tol": 1e-10,
        "vcycles_from_zero": {"solves_per_s": round(1e3 / ms_v, 1), "ms": round(ms_v, 3), "vcycles": cyc,
                              "rel_residual": rel},
        "fmg": {"solves_per_s": round(1e3 / ms_f, 1), "ms": round(ms_f, 3), "vcycles": cycf, "rel_residual": relf},
        "vcycle_us": round(us_vc, 2),
        "mcells_vcycles_per_s": round(cells * cyc / (ms_v * 1e-3) / 1e6, 1),
        "note": "the working set (about 40 MB) stays in L2; L2 not flushed"}
    g.close()

    dom, st = synth.workload("streamer8")
    sides = {}
    ne = ni = None
    for prec, name in ((0, "fp64"), (pkg.MIXED, "mixed")):
        g = pkg.Solver(dom, max_boxes=1 << 16, precision=prec)
        g.build_octree()
        synth.refine_all(dom, st, g.level_ijk, g.refine_level)
        if ne is None:
            t = g.tables()
            ne, ni = synth.streamer_densities(dom, st, t["level"], t["ijk"])
        g.upload(pkg.NE, ne)
        g.upload(pkg.NI, ni)
        g.charge_rhs(Q, E0)
        sides[name] = g
    gf, gm = sides["fp64"], sides["mixed"]
    gm.fmg(TOL, MAX_CYCLES)
    ms_m, (rcm, relm, cycm) = ev(gm, lambda: gm.fmg(TOL, MAX_CYCLES), 5)
    ms_d, (rcd, reld, cycd) = ev(gf, lambda: gf.fmg(TOL, MAX_CYCLES), 5)
    gf.fmg(1e-12, 60)
    gm.fmg(TOL, MAX_CYCLES)
    gf.compute_field()
    gm.compute_field()
    leaf = torch.from_numpy(np.asarray(gf.tables()["leaf"], dtype=np.int64)).to(gf.var(pkg.PHI).device)
    p64, p32 = gf.var(pkg.PHI)[leaf], gm.var(pkg.PHI)[leaf]
    e64, e32 = gf.var(pkg.EMAG)[leaf], gm.var(pkg.EMAG)[leaf]
    out["streamer8_mixed"] = {
        "leaf_cells": gf.n_leaves * 512, "boxes": gf.n_boxes, "levels": gf.n_levels, "tol": TOL,
        "mixed": {"solves_per_s": round(1e3 / ms_m, 2), "ms": round(ms_m, 3), "corrections": cycm},
        "fp64": {"solves_per_s": round(1e3 / ms_d, 2), "ms": round(ms_d, 3), "vcycles": cycd},
        "speedup_mixed_vs_fp64": round(ms_d / ms_m, 3),
        "error_vs_fp64": {"phi_max_rel": float((p32 - p64).abs().max() / p64.abs().max()),
                          "emag_max_rel": float((e32 - e64).abs().max() / e64.abs().max()),
                          "reference": "FP64 path converged to 1e-12"},
        "note": "FMG from phi = 0 to 1e-8, 5 solves each timed with CUDA events"}
    gf.close()
    gm.close()
    return out


def warm_regrid(two_d):
    """One regrid of a small mesh that refines and one that derefines, so
    that the regrid kernels are loaded (lazy module loading) before a
    regrid is timed."""
    import synth
    import paper_1708_08434_gb300 as pkg
    if two_d:
        dom, st = synth.workload2("axi_small")
        w = pkg.Quad(dom, 1 << 12)
        synth.refine_all2(dom, st, w.level_ij, w.refine_level)
    else:
        dom, st = synth.workload("streamer_small")
        w = pkg.Solver(dom, max_boxes=1 << 14)
        w.build_octree()
        synth.refine_all(dom, st, w.level_ijk, w.refine_level)
    t = w.tables()
    leaf = t["child"][:, 0] < 0
    top = t["level"] == t["level"].max()
    f = np.zeros(len(leaf), np.int8)
    f[np.where(leaf & ~top)[0][:16]] = 1
    w.regrid(f)
    t = w.tables()
    w.regrid(np.where(t["child"][:, 0] < 0, -1, 0).astype(np.int8))
    w.close()


def bench_axisymmetric(args, dev, world):
    """The axisymmetric variant (quadtree of 8^2 boxes, cylindrical
    operators): the streamer on its symmetry axis, 16 mm, base 512^2 cells +
    8 levels (10113 boxes, 4.9e5 leaf cells, finest spacing 0.12 um).  A step
    is the headline step in 2-D: FMG to 1e-8, field, dt, one Heun step (3
    solves), densities copied in from device buffers; CUDA events on the
    solver's stream, L2 flushed between steps.  Beside it the V-cycle alone
    (10 back-to-back cycles) and its launch count."""
    import torch
    import synth
    import paper_1708_08434_gb300 as pkg
    Q, E0 = synth.E_CHARGE, synth.EPS0
    dom, st = synth.workload2("axi_streamer")
    g = pkg.Quad(dom, 1 << 15)
    synth.refine_all2(dom, st, g.level_ij, g.refine_level)
    t = g.tables()
    ne, ni = synth.streamer_densities2(dom, st, t["level"], t["ij"])
    g.set_table(synth.coefficient_table())
    ne_d, ni_d = torch.from_numpy(ne).to(dev), torch.from_numpy(ni).to(dev)
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=dev)
    stream = g.stream

    def step():
        g.view(pkg.NE).copy_(ne_d)
        g.view(pkg.NI).copy_(ni_d)
        g.charge_rhs(Q, E0)
        rc0, _, c0 = g.fmg(TOL, MAX_CYCLES)
        g.compute_field()
        dt = g.dt_limit(Q, E0)
        rc1, _, c1, c2 = g.advance(dt, Q, E0, TOL, MAX_CYCLES)
        assert rc0 == 0 and rc1 == 0, (rc0, rc1)
        return c0 + c1 + c2

    def events():
        return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    for _ in range(max(args.warmup, 3)):
        step()
    n = max(args.steps, 5)
    total, cycles = 0.0, 0
    l0 = g.launch_count()
    for _ in range(n):
        flush.fill_(1)
        torch.cuda.synchronize()
        a, b = events()
        a.record(stream)
        cycles += step()
        b.record(stream)
        torch.cuda.synchronize()
        total += a.elapsed_time(b)
    launches = g.launch_count() - l0
    total = max_over_ranks(total, dev)
    # the paper's schedule (Sec. 2.1.2, 2.4): from the solved state, Heun
    # steps with exactly two V-cycles per solve and dt from the limits
    paper_steps = 20
    g.compute_field()
    dt = g.dt_limit(Q, E0)
    torch.cuda.synchronize()
    a, b = events()
    a.record(stream)
    for _ in range(paper_steps):
        rc_, dt, c1_, c2_ = g.advance(dt, Q, E0, 0.0, PAPER_VCYCLES)
    b.record(stream)
    torch.cuda.synchronize()
    pms = max_over_ranks(a.elapsed_time(b), dev)
    paper = {"steps_per_s": round(paper_steps * world / (pms * 1e-3), 2),
             "solves_per_s": round(2 * paper_steps * world / (pms * 1e-3), 2),
             "ms_per_step": round(pms / paper_steps, 4), "steps": paper_steps,
             "schedule": "2 V-cycles per solve, 2 solves per Heun step, dt from the Sec. 2.4 limits"}
    # the V-cycle alone
    g.vcycles(2)
    torch.cuda.synchronize()
    lv = g.launch_count()
    a, b = events()
    a.record(stream)
    g.vcycles(10)
    b.record(stream)
    torch.cuda.synchronize()
    vus = a.elapsed_time(b) * 100.0
    lv = (g.launch_count() - lv) // 10
    leaf_cells = int((t["child"][:, 0] < 0).sum()) * 64
    all_cells = len(t["level"]) * 64
    # refinement criterion (Eq. 8) with the paper's constants, then a regrid
    # with a stricter c0 that changes the mesh (CUDA events around each)
    g.compute_field()

    def timed_ms(fn):
        torch.cuda.synchronize()
        a_, b_ = events()
        a_.record(stream)
        out = fn()
        b_.record(stream)
        torch.cuda.synchronize()
        return a_.elapsed_time(b_), out

    g.refine_flags()
    warm_regrid(True)
    fl_ms, flags = timed_ms(lambda: g.refine_flags())
    strict = g.refine_flags(0.25, 1.2, 0.125, 30e-6, 3)
    nb0 = g.n_boxes
    rg_ms, (nref, nder, ndrop) = timed_ms(lambda: g.regrid(strict))
    regrid = {"flags_ms": round(fl_ms, 3), "paper_flags": {"refine": int((flags == 1).sum()),
                                                            "derefine": int((flags == -1).sum())},
              "regrid_ms": round(rg_ms, 3), "boxes": [nb0, g.n_boxes], "refined": nref, "derefined": nder,
              "dropped": ndrop, "criterion": "c0=0.25 (paper: 1), c1=1.2, buffer 3"}
    res = {"value": round(whole_job_rate(SOLVES_PER_STEP * n, world, total), 3), "unit": "solves/s",
           "ms_per_step": round(total / n, 4), "vcycles_per_step": cycles / n, "gpu_launches": launches,
           "vcycle_us": round(vus, 2), "launches_per_vcycle": int(lv),
           "gcells_per_s_vcycle": round(all_cells / (vus * 1e-6) / 1e9, 3),
           "workload": "axi_streamer", "geometry": "axisymmetric (r, z)", "boxes": len(t["level"]),
           "leaf_cells": leaf_cells, "levels": int(len(t["level_offset"]) - 1), "tol": TOL,
           "dtype": "f64", "l2": "flushed between steps",
           "note": "per-level launches, each V-cycle a CUDA graph (one per top level), one residual "
                   "read per V-cycle", "paper_schedule": paper, "regrid": regrid}
    g.close()
    return res


def bench_learned(args, dev, world):
    """The learned warm start on the benchmark workload: record the
    (input, solved change) pairs of the first 6 Heun steps, train the
    network on the GPU, then time 4 more steps with predictions (judged by
    the multigrid residual) and the same 4 steps without."""
    import torch
    import synth
    import paper_1708_08434_gb300 as pkg
    Q, E0 = synth.E_CHARGE, synth.EPS0
    n_train, n_eval = 6, 4

    def start():
        dom, st, g, t, ne, ni = build_gpu_case()
        g.upload(pkg.NE, ne)
        g.upload(pkg.NI, ni)
        g.charge_rhs(Q, E0)
        g.fmg(TOL, MAX_CYCLES)
        g.compute_field()
        return g, g.dt_limit(Q, E0)

    def steps(g, dt, n):
        ms, cyc = 0.0, []
        for _ in range(n):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(g.stream)
            rc, dt, c1, c2 = g.advance(dt, Q, E0, TOL, MAX_CYCLES)
            e1.record(g.stream)
            torch.cuda.synchronize()
            assert rc == 0, rc
            ms += e0.elapsed_time(e1)
            cyc += [c1, c2]
        return ms, cyc, dt

    net = pkg.Network(16384, 4096)
    net.set_params(synth.cnn_initial_params())
    g, dt = start()
    net.attach(g, 1, per_solve=4096)
    steps(g, dt, n_train)
    samples = net.stats()["samples"]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss = net.train(30, 64, 1e-3)
    train_s = time.perf_counter() - t0
    g.close()
    res = {"train_samples": samples, "train_epochs": 30, "train_s": round(train_s, 3),
           "final_loss": round(loss, 6)}
    # the network kernels against the tensor-core roof: forward (inference)
    # and a training gradient pass over 4096 recorded samples
    res["network_kernels"], res["network_kernels_note"] = network_kernels(net, 4096, 10)
    for mode in ("plain", "learned"):
        g, dt = start()
        _, _, dt = steps(g, dt, n_train)
        if mode == "learned":
            net.attach(g, 2, per_solve=4096, taper=True)
        ms, cyc, _ = steps(g, dt, n_eval)
        res[mode] = {"solves_per_s": round(2 * n_eval / (ms * 1e-3), 2), "vcycles": cyc,
                     "mean_vcycles": sum(cyc) / len(cyc)}
        g.close()
    s = net.stats()
    res["predictions_kept"] = "%d/%d" % (s["kept"], s["predictions"])
    res["vcycles_saved_per_solve"] = res["plain"]["mean_vcycles"] - res["learned"]["mean_vcycles"]
    res["workload"] = "streamer6; train on Heun steps 1-6 (12 solves), evaluate steps 7-10"
    return res


def bench_learned_c4(n_rec=100, n_eval=100, epochs=10):
    """The learned warm start at its own configuration: streamer9 with the
    seeded stochastic background (1.02e8 leaf cells, mean background 1e13
    m^-3), Heun steps with solves to 1e-8.  The plain FP64 run records
    (input, solved change) pairs of the two finest levels during steps
    1..n_rec and then times steps n_rec+1..n_rec+n_eval; the network trains
    on the GPU; the state after step n_rec is restored into the other arms --
    FP64 with predictions, mixed precision, mixed precision with predictions
    -- which time the same n_eval steps with the plain run's time steps.
    Reported per arm: V-cycles (or corrections) per solve, solves/s, and the
    potential and electron density after the last step against the plain
    FP64 run."""
    import numpy as np
    import torch
    import synth
    import paper_1708_08434_gb300 as pkg
    Q, E0 = synth.E_CHARGE, synth.EPS0
    dom, st = synth.workload("streamer9_bg")
    tab = synth.coefficient_table()
    out = {"mode": "learned", "workload": "streamer9_bg", "steps_recorded": n_rec, "steps_evaluated": n_eval,
           "tol": TOL}

    def solver(prec):
        g = pkg.Solver(dom, max_boxes=1 << 18, precision=prec)
        if ROW_KERNELS is not None:
            g.set_row_kernels(ROW_KERNELS)
        g.build_octree()
        synth.refine_all(dom, st, g.level_ijk, g.refine_level)
        g.set_table(tab)
        return g

    def run(g, dts, timed):
        ms, cyc = 0.0, []
        for dt in dts:
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(g.stream)
            rc, dtn, c1, c2 = g.advance(dt, Q, E0, TOL, MAX_CYCLES)
            b.record(g.stream)
            torch.cuda.synchronize()
            assert rc == 0, rc
            if timed:
                ms += a.elapsed_time(b)
            cyc += [c1, c2]
        return ms, cyc, dtn

    t0 = time.perf_counter()
    g = solver(0)
    t = g.tables()
    ne, ni = synth.streamer_densities(dom, st, t["level"], t["ijk"])
    out["boxes"], out["leaf_cells"], out["levels"] = g.n_boxes, g.n_leaves * 512, g.n_levels
    g.upload(pkg.NE, ne)
    g.upload(pkg.NI, ni)
    g.charge_rhs(Q, E0)
    g.fmg(TOL, MAX_CYCLES)
    g.compute_field()
    dt = g.dt_limit(Q, E0)
    lv = np.asarray(t["level"])
    fine = int(((lv >= g.n_levels - 2) & (np.asarray(t["child"])[:, 0] < 0)).sum())
    per_solve = 256
    max_samples = per_solve * 2 * n_rec
    net = pkg.Network(max_samples, 16384)
    net.set_params(synth.cnn_initial_params())
    net.attach(g, 1, per_solve=per_solve, stride=max(1, fine // per_solve))
    # steps 1..n_rec with recording, keeping the time steps
    dts = []
    for _ in range(n_rec):
        dts.append(dt)
        _, _, dt = run(g, [dt], False)
    net.attach(g, 0)
    samples = net.stats()["samples"]
    state = {v: g.download(v) for v in (pkg.NE, pkg.NI, pkg.PHI)}
    # the restored arms start from these densities and potential with the
    # field recomputed; the plain run does the same so that all four arms
    # take identical steps
    g.charge_rhs(Q, E0)
    g.compute_field()
    # plain FP64: steps n_rec+1 .. n_rec+n_eval
    eval_dts = []
    ms_plain, cyc_plain = 0.0, []
    for _ in range(n_eval):
        eval_dts.append(dt)
        m, c, dt = run(g, [dt], True)
        ms_plain += m
        cyc_plain += c
    ref = {v: g.download(v) for v in (pkg.PHI, pkg.NE)}
    leaf = np.asarray(t["child"])[:, 0] < 0
    g.close()
    torch.cuda.synchronize()
    tt = time.perf_counter()
    loss = net.train(epochs, 64, 1e-3)
    train_s = time.perf_counter() - tt
    out["network"] = {"samples": samples, "epochs": epochs, "train_s": round(train_s, 2), "final_loss": round(loss, 6),
                      "sampled_boxes": "%d per solve, every %d-th leaf of the two finest levels (%d leaves)"
                                       % (per_solve, max(1, fine // per_solve), fine)}
    out["plain_fp64"] = {"solves_per_s": round(2 * n_eval / (ms_plain * 1e-3), 3),
                         "mean_vcycles": sum(cyc_plain) / len(cyc_plain), "ms": round(ms_plain, 1)}
    for name, prec, learned in (("learned_fp64", 0, True), ("mixed", pkg.MIXED, False),
                                ("learned_mixed", pkg.MIXED, True)):
        g = solver(prec)
        for v, a in state.items():
            g.upload(v, a)
        g.charge_rhs(Q, E0)
        g.compute_field()
        if learned:
            net.attach(g, 2, per_solve=16384, stride=max(1, fine // 16384), taper=True)
            p0, k0 = net.stats()["predictions"], net.stats()["kept"]
        ms, cyc, _ = run(g, eval_dts, True)
        r = {"solves_per_s": round(2 * n_eval / (ms * 1e-3), 3), "mean_vcycles": sum(cyc) / len(cyc),
             "ms": round(ms, 1), "speedup_vs_plain_fp64": round(ms_plain / ms, 3)}
        if learned:
            s_ = net.stats()
            r["predictions_kept"] = "%d/%d" % (s_["kept"] - k0, s_["predictions"] - p0)
            r["vcycles_saved_per_solve"] = round(out["plain_fp64"]["mean_vcycles"] - r["mean_vcycles"], 3)
            net.attach(g, 0)
        phi, n_e = g.download(pkg.PHI), g.download(pkg.NE)
        r["vs_plain_fp64_after_last_step"] = {
            "phi_max_rel": float(np.abs(phi[leaf] - ref[pkg.PHI][leaf]).max() / np.abs(ref[pkg.PHI][leaf]).max()),
            "ne_max_rel": float(np.abs(n_e[leaf] - ref[pkg.NE][leaf]).max() / np.abs(ref[pkg.NE][leaf]).max())}
        out[name] = r
        g.close()
        torch.cuda.empty_cache()
    net.close()
    out["wall_s"] = round(time.perf_counter() - t0, 1)
    out["note"] = ("every arm from the same state after step %d, the plain run's time steps, solves to 1e-8 "
                   "(the learned arms predict on up to 16384 of the finest leaves per solve, kept only when "
                   "the relative residual drops)" % n_rec)
    return out


def run_learned(args):
    import torch
    import __graft_entry__
    torch.cuda.set_device(0)
    __graft_entry__.build()
    print(json.dumps(bench_learned_c4(n_rec=args.steps if args.steps != 40 else 100,
                                      n_eval=args.steps if args.steps != 40 else 100)), flush=True)


def make_batch_workload(n=256):
    """The first n solves of the seeded 256-solve workload."""
    import torch
    import synth
    import paper_1708_08434_gb300 as pkg
    sides = synth.batch_sizes(256)[:n]
    b = pkg.Batch(sides, 1.0, (0, 0, 0, 0, 1, 1), (0, 0, 0, 0, 0, 1.0))
    blobs = synth.batch_blobs(len(sides))
    for s, n in enumerate(sides):
        b.grid(b.rhs, s).copy_(torch.from_numpy(-synth.blob_rho(int(n), blobs[s])))
    return b, sides


def bench_batch(args, dev, world):
    """The batched form: 256 independent unit-cube solves of 32^3..128^3
    cells (log-uniform sizes, 1-8 Gaussian charge blobs each), autotuned,
    solved from phi = 0 to 1e-8; value = solves per second."""
    import torch
    import synth
    import paper_1708_08434_gb300 as pkg
    if world > 1:
        import torch.distributed as dist
    b, sides = make_batch_workload()
    if NO_GRAPHS:
        b.set_graphs(False)
    shape, gmult, tune_ms = b.tune(2)
    for _ in range(args.warmup):
        b.phi.zero_()
        b.solve(TOL, MAX_CYCLES)
    total, cycles = 0.0, 0
    l0 = b.info()[2]
    for _ in range(args.steps):
        b.phi.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(b.stream)
        rc, cyc, rel = b.solve(TOL, MAX_CYCLES)
        e1.record(b.stream)
        torch.cuda.synchronize()
        assert rc == 0, rc
        total += e0.elapsed_time(e1)
        cycles += int(cyc.max())
    total = max_over_ranks(total, dev)
    cells, levels, launches = b.info()
    # per-kernel rooflines of the cycle (after the timed solves: the bench
    # launches overwrite the error arrays)
    hbm = measured_peaks()[0]
    kern = {}
    for kc, name in ((0, "k_bt_sweep level 0"), (1, "k_bt_outer (residual, fixed-point sum)"),
                     (2, "k_bt_prolong level 0"), (3, "k_bt_restrict level 0->1")):
        us, by, fl = b.kernel_bench(kc, 10)
        e = {"us": round(us, 2), "bytes": int(by), "gbs": round(by / (us * 1e-6) / 1e9, 1),
             "hbm_frac": round(by / (us * 1e-6) / 1e9 / hbm, 4)}
        if fl:
            e["fp64_ginstr"] = round(fl / (us * 1e-6) / 1e9, 1)
            e["fp64_frac"] = round(fl / (us * 1e-6) / 1e9 / fp64_rate(), 4)
        kern[name] = e
    # the same problems one at a time (a batch of one each, same kernels and
    # schedule): 16 problems spread over the size range, timed after a
    # warm-up solve each, scaled to the 256 solves by their cell counts
    order = np.argsort(sides)
    pick = [int(order[i]) for i in np.linspace(0, len(sides) - 1, 16).round().astype(int)]
    blobs = synth.batch_blobs(len(sides))
    one_ms, one_cells = 0.0, 0
    for s_ in pick:
        n_ = int(sides[s_])
        b1 = pkg.Batch([n_], 1.0, (0, 0, 0, 0, 1, 1), (0, 0, 0, 0, 0, 1.0))
        b1.grid(b1.rhs, 0).copy_(torch.from_numpy(-synth.blob_rho(n_, blobs[s_])))
        b1.set_schedule(shape, gmult)
        b1.phi.zero_()
        b1.solve(TOL, MAX_CYCLES)
        b1.phi.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(b1.stream)
        rc1, _, _ = b1.solve(TOL, MAX_CYCLES)
        e1.record(b1.stream)
        torch.cuda.synchronize()
        assert rc1 == 0, rc1
        one_ms += e0.elapsed_time(e1)
        one_cells += n_ ** 3
        b1.close()
    one_total_ms = one_ms * float(np.sum(np.asarray(sides, np.float64) ** 3)) / one_cells
    one = {"sample": "16 of the 256 problems spread over the size range, each solved alone (a batch of one, "
                     "same kernels and schedule) after a warm-up solve; time scaled to all 256 by cell count",
           "solves_per_s": round(256 / (one_total_ms * 1e-3), 2),
           "batched_speedup": round((256 * args.steps / (total * 1e-3)) / (256 / (one_total_ms * 1e-3)), 2)}
    res = {"value": round(256 * args.steps * world / (total * 1e-3), 2), "unit": "solves/s",
           "one_at_a_time": one,
           "ms_per_batch": round(total / args.steps, 3), "solves_per_batch": 256, "cells": cells,
           "max_corrections": cycles / args.steps,
           "gcells_corrections_per_s": round(cells * cycles * world / (total * 1e-3) / 1e9, 3),
           "schedule": {"tile": pkg.Batch.SHAPES[shape], "blocks_per_sm": gmult, "tuned_ms": round(tune_ms, 3)},
           "gpu_launches": launches - l0,
           "dtype": "f32 cycles; f64 residual (stencil sum exact in int64 fixed point), accumulation, coarsest solve",
           "workload": "256 unit-cube solves, sides 8*round(32*4^u/8), phi=0/1 on z plates",
           "kernels": kern,
           "kernels_note": "CUDA events around 10 back-to-back launches over all 256 solves; bytes = "
                           "compulsory traffic (sweep 12 B, outer 20 B + 2 FP64-pipe instr, prolong/restrict "
                           "8.5 B per fine cell); hbm peak %.1f GB/s measured, FP64 peak %.0f G instr/s "
                           "measured (sm_fp64_probe)" % (hbm, fp64_rate())}
    b.close()
    return res


def oracle_case():
    import oracle
    import synth
    dom, st = synth.workload(WORKLOAD)
    o = oracle.build_mesh(dom, st)
    t = o.tables()
    ne, ni = synth.streamer_densities(dom, st, t["level"], t["ijk"])
    o.set_table(synth.coefficient_table())
    return o, ne, ni


def oracle_solve(o, ne, ni):
    import oracle
    import synth
    o.set(oracle.NE, ne)
    o.set(oracle.NI, ni)
    o.charge_rhs(synth.E_CHARGE, synth.EPS0)
    t0 = time.perf_counter()
    st, rel, cyc = o.fmg(TOL, MAX_CYCLES)
    return time.perf_counter() - t0, cyc


def oracle_step(o, ne, ni):
    """The GPU arm's step on the oracle: charge, FMG to 1e-8, field, time
    step, one Heun step with its two solves to 1e-8 (3 solves)."""
    import oracle
    import synth
    Q, E0 = synth.E_CHARGE, synth.EPS0
    o.set(oracle.NE, ne)
    o.set(oracle.NI, ni)
    t0 = time.perf_counter()
    o.charge_rhs(Q, E0)
    _, _, c0 = o.fmg(TOL, MAX_CYCLES)
    o.compute_field()
    dt = o.dt_limit(Q, E0)
    r = o.advance(dt, Q, E0, TOL, MAX_CYCLES)
    return time.perf_counter() - t0, c0 + r[2] + r[3]


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline():
    """The oracle as it stands on one step of the same workload (the GPU
    arm's step: FMG, field, time step, Heun step; 3 solves) on all host
    cores (OpenMP over boxes, the paper's own CPU scheme), and one FMG solve
    on one thread (about 10-30 s of CPU work in all)."""
    import oracle
    o, ne, ni = oracle_case()
    cores = oracle.set_threads(host_cores())
    try:
        sec_all, cyc = oracle_step(o, ne, ni)
        oracle.set_threads(1)
        sec_one, cyc1 = oracle_solve(o, ne, ni)
    finally:
        oracle.set_threads(1)
    return {"value": round(SOLVES_PER_STEP / sec_all, 5), "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": "one step of the %s workload (FMG to 1e-8, field, time step, Heun step with two solves "
                      "to 1e-8; %d V-cycles), plain C oracle, OpenMP over boxes on %d threads"
                      % (WORKLOAD, cyc, cores),
            "single_thread": {"value": round(1.0 / sec_one, 5), "unit": "solves/s", "cores": 1,
                              "sample": "one FMG solve to 1e-8 (%d V-cycles)" % cyc1},
            "axisymmetric": cpu_baseline_axi()}


def cpu_baseline_axi():
    """The 2-D oracle on all host cores: one FMG solve to 1e-8 of the
    axisymmetric workload (the GPU's axisymmetric line beside it)."""
    import synth
    from oracle import quad
    dom, st = synth.workload2("axi_streamer")
    o = quad.build_mesh(dom, st)
    t = o.tables()
    ne, ni = synth.streamer_densities2(dom, st, t["level"], t["ij"])
    o.set(quad.NE, ne)
    o.set(quad.NI, ni)
    o.charge_rhs(synth.E_CHARGE, synth.EPS0)
    cores = quad.set_threads(host_cores())
    try:
        t0 = time.perf_counter()
        st_, rel, cyc = o.fmg(TOL, MAX_CYCLES)
        sec = time.perf_counter() - t0
    finally:
        quad.set_threads(1)
    return {"value": round(1.0 / sec, 4), "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": "one FMG solve to 1e-8 of axi_streamer (%d V-cycles), plain C oracle "
                      "(oracle/quad.c), OpenMP over boxes" % cyc}


def run_reference(args):
    """The reference arm: the CPU oracle as it stands, timed on the GPU arm's
    own step (FMG + field + time step + Heun step: 3 solves to 1e-8) of the
    same workload, on the host cores."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    import oracle
    o, ne, ni = oracle_case()
    nthr = getattr(args, "ref_threads", 0)
    cores = oracle.set_threads(nthr if nthr > 0 else host_cores())
    for _ in range(args.warmup):
        oracle_step(o, ne, ni)
    total, cycles = 0.0, 0
    for _ in range(args.steps):
        sec, cyc = oracle_step(o, ne, ni)
        total += sec
        cycles += cyc
    oracle.set_threads(1)
    value = SOLVES_PER_STEP * args.steps / total
    res = {
        "metric": "Poisson solves/s to rel residual 1e-8 (octree FMG + Heun step, 3 solves/step)",
        "value": round(value, 5), "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(1e3 * total / args.steps, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": WORKLOAD, "tol": TOL, "nu": [2, 2]},
        "vcycles_per_step": cycles / args.steps,
        "cpu_baseline": {"value": round(value, 5), "unit": "solves/s", "cores": cores, "kind": "oracle",
                         "sample": "each step = the GPU arm's step (charge, FMG to 1e-8, field, time step, "
                                   "Heun step with two solves to 1e-8) of the workload, plain C oracle, "
                                   "OpenMP over boxes on %d threads" % cores},
        "e2e": {"value": round(value, 5), "unit": "solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(res), flush=True)


def main():
    global NO_GRAPHS, NO_PDL, PERSIST, WORKLOAD, ROW_KERNELS
    args = parse()
    if args.mode in ("kernels", "vcycle"):
        WORKLOAD = args.workload
    NO_GRAPHS = args.no_graphs
    NO_PDL = args.no_pdl
    PERSIST = args.persistent
    ROW_KERNELS = args.row_kernels
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "batch":
        run_batch_only(args)
    elif args.mode == "large":
        run_large(args)
    elif args.mode == "axi":
        run_axi(args)
    elif args.mode == "learned":
        run_learned(args)
    elif args.mode == "network":
        run_network(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
