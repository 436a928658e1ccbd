#!/usr/bin/env python
"""CGNE throughput on the paper-shaped workload (Sec. 3 of arXiv:1312.3265).

Workload (one "step" = one gauge configuration, every row of the hot path):
  16^3x32 lattice, SU(3) links exp(i eps H) with eps tuned to mean plaquette
  0.59 (stand-in for the paper's quenched beta = 6 ensemble, which is not
  available), configuration seed = step index mod 10;
  hypercube transports built on the device for that configuration;
  staggered Wilson (r = 1): 4 bare masses x 3 colour point sources = 12 solves;
  Wilson (r = 1):           4 bare masses x 12 spin-colour point sources = 48 solves;
  unpreconditioned CGNE (Eq. 2) to an FP64 true relative residual of 1e-8,
  FP32 inner iterations with FP64 reliable updates, one batched call per
  operator.
value = solves per second (device-resident inputs); e2e = the same through
the public API with inputs copied from pinned host memory and solutions
copied back inside the timed region.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "CG solves/sec to 1e-8 residual and Dslash GB/s vs HBM roofline; p50/p99 latency"
DIMS = (16, 16, 16, 32)
MASSES = (0.02, 0.05, 0.1, 0.2)
TOL = 1e-8
R_WILSON = 1.0
N_SEEDS = 10
WORKLOAD = "16^3x32 paper-shaped CGNE: staggered Wilson 4 masses x 3 colour sources + Wilson 4 masses x 12 spin-colour sources per configuration"

# Mean CG iterations per (operator, mass) of the workload above, used only to
# turn the CPU oracle's seconds per iteration into solves/s in the reference
# arm (which cannot afford full solves).  Measured with this bench's
# reliable-update solves on configurations 3-5.
ITERS_TABLE = {"sw": {0.02: 41.0, 0.05: 39.0, 0.1: 36.9, 0.2: 32.0},
               "wilson": {0.02: 118.0, 0.05: 113.6, 0.1: 107.0, 0.2: 94.9}}


# DRAM traffic of a kernel class from one ncu capture of the current kernel
# build (dram__bytes_read.sum + dram__bytes_write.sum): bytes of one launch
# over `systems` running systems and the algorithmic bytes of that launch.  A
# bench launch's traffic is scaled by its algorithmic bytes (traffic grows
# with the systems computed).  Entries are removed when the kernel changes.
NCU_TRAFFIC = {
    # profiles/ncu_sw_k1k2k3_fp32_16x16x16x32_12sys.md
    "sw.k1.f32": {"bytes": 195.3e6, "algorithmic": 188.7e6, "systems": 12},
    "sw.k2.f32": {"bytes": 236.8e6, "algorithmic": 226.5e6, "systems": 12},
    # profiles/ncu_wilson_k1k2k3_fp32_16x16x16x32_12sys.md (the 48-system section:
    # the headline's batch, every system running)
    "wilson.k1.f32": {"bytes": 1582.8e6, "algorithmic": 1245.7e6, "systems": 48},
    "wilson.k2.f32": {"bytes": 2206.5e6, "algorithmic": 1849.7e6, "systems": 48},
}

# FP64 peak of a GB300 when no measurement is given (nominal 1.25 TFLOP/s; the
# measured-peaks file has no FP64 figure): the bench measures it with the
# library's FMA-throughput kernel (sw_measure_fp64_peak) and passes that in.
FP64_PEAK_TFLOPS = 1.25


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["mixed", "f16", "f64"], default="mixed",
                    help="inner iterations: FP32 (mixed), FP16 storage (f16) or FP64")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--delta", type=float, default=None, help="reliable-update delta (library default if unset)")
    ap.add_argument("--chunk", type=int, default=None, help="CG iterations between status reads")
    ap.add_argument("--ns-sw", type=int, default=None, help="systems per thread, staggered Wilson FP32 stencils")
    ap.add_argument("--ns-wilson", type=int, default=None, help="systems per thread, Wilson FP32 stencils")
    ap.add_argument("--serving-requests", type=int, default=2000,
                    help="requests in the Poisson serving phase (0: skip)")
    ap.add_argument("--serving-lattices", default="8x8x8x8,12x12x12x24,16x16x16x32,24x24x24x48")
    ap.add_argument("--no-f64", action="store_true", help="skip the plain-FP64 comparison step")
    ap.add_argument("--masses", default=None, help="comma-separated bare masses (default: the workload's four)")
    ap.add_argument("--w-sources", type=int, default=12, help="Wilson spin-colour sources per mass (<= 12)")
    ap.add_argument("--dims", default="16x16x16x32", help="lattice L0xL1xL2xL3 (L3 = time)")
    ap.add_argument("--graphs", type=int, default=None, help="1/0: replay chunks as CUDA graphs (library default 1)")
    ap.add_argument("--site-blocking", type=int, default=None,
                    help="site order of the packed fields: 0 lexicographic, 1-5 site-block shapes")
    ap.add_argument("--group-fast", type=int, default=None, help="1/0: system groups fastest in the stencil grid")
    ap.add_argument("--autotune", action="store_true",
                    help="before the warm-up, pick each operator's systems per thread and the shared site order "
                         "with the library's width x site-order autotuner (overrides --ns-* / --site-blocking)")
    ap.add_argument("--concurrent-ops", action="store_true",
                    help="solve the staggered Wilson and Wilson batches at the same time, each on its own stream "
                         "and host thread (the per-kernel event timings then include the other batch's kernels)")
    ap.add_argument("--ops", choices=["both", "sw", "wilson"], default="both",
                    help="operators of a step (the large-volume runs take one per lattice)")
    ap.add_argument("--sources", default="point",
                    help="'point': 3 colour (SW) / 12 spin-colour (W) point sources per mass; "
                         "'z2:N': N real Z2-noise sources per mass for both operators")
    ap.add_argument("--no-large-volume", action="store_true",
                    help="skip the large-volume block (48^3x96 staggered Wilson, 32^3x64 Wilson; FP32 and FP16)")
    ap.add_argument("--no-even-odd", action="store_true",
                    help="skip the even-odd Wilson block (run after the timed region in the default configuration)")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched block (24^3x48, 12 Z2 sources x 6 masses per operator)")
    return ap.parse_args()


# ------------------------------------------------------------------ distributed plumbing
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def seed_for(step, rank, world):
    """Configuration of a replica's step: ranks take disjoint configurations in
    each step (weak scaling: every rank solves a full configuration)."""
    return (step * world + rank) % N_SEEDS


def max_over_ranks(ms, device=None):
    """Slowest rank's time (the job's time) when running under torch.distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([float(ms)], device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        busy = [v for v in sm if v > 0.5 * max(sm)] if sm else []
        return {"sm_mhz": statistics.median(busy) if busy else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------ workload inputs
def host_inputs(seeds, masses=MASSES, w_sources=12, dims=DIMS, sources="point"):
    """Links per configuration seed and the sources of one configuration's solves
    (mass-major: all sources of the first mass, then the next mass, ...)."""
    import lattice_synth as ls
    V = ls.volume(dims)
    nproc = min(16, os.cpu_count() or 1)
    U = {s: ls.su3_links(dims, s, ls.PLAQ_EPS, processes=nproc) for s in seeds}
    if sources.startswith("z2:"):
        nz = int(sources.split(":")[1])
        z_sw = [ls.z2_source(dims, 3, k) for k in range(nz)]
        z_w = [ls.z2_source(dims, 12, k).reshape(V, 4, 3) for k in range(nz)]
    else:
        z_sw = [ls.point_source(dims, 3, a) for a in range(3)]
        z_w = [ls.point_source(dims, 12, a).reshape(V, 4, 3) for a in range(w_sources)]
    chi_sw = np.zeros((len(masses) * len(z_sw), V, 3), dtype=np.complex128)
    chi_w = np.zeros((len(masses) * len(z_w), V, 4, 3), dtype=np.complex128)
    m_sw, m_w = [], []
    for i, m in enumerate(masses):
        for a, z in enumerate(z_sw):
            chi_sw[len(z_sw) * i + a] = z
            m_sw.append(m)
        for a, z in enumerate(z_w):
            chi_w[len(z_w) * i + a] = z
            m_w.append(m)
    return U, chi_sw, m_sw, chi_w, m_w


def workload_config(workload, dims, masses):
    """The `config` object of the JSON line: the workload only, the same keys
    and values in both arms."""
    return {"workload": workload, "lattice": "x".join(map(str, dims)), "masses": list(masses), "tol": TOL,
            "l2": "inputs larger than L2: a step touches ~10 GB and each step uses a new configuration"}


# ------------------------------------------------------------------ rooflines
# FP32 peak of a GB300 from its unit counts and clock: 152 SMs x 128 FP32
# lanes x 2 flop (FMA) x 2.07 GHz (the maximum SM clock).
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def classify_kernels(prof, hbm_peak, peak_kind, fp64_peak=None):
    """Per kernel class: time per launch, and the fraction of the roofline
    that bounds it.  FP32/FP16 stencils: algorithmic bytes against the
    measured HBM bandwidth and the paper's flops (Eq. 4) against the FP32 peak;
    the bound is the resource whose roofline time is longer (the launch's
    arithmetic intensity against the ridge).  FP64 matvecs: flops against the
    measured FP64 FMA throughput (fp64_peak, TFLOP/s), else the nominal one.  A class's time in the timed region is its mean timed
    launch times the launches it issued (only some launches are timed).
    Returns (kernels, roofline of the kernel class with the most time,
    roofline of the HBM-bound class with the most time)."""
    kernels, cand = {}, []
    for k, v in prof.items():
        if not v["launches"]:
            continue
        ms = v["ms"] / v["launches"]
        bpl, fpl = v["bytes"] / v["launches"], v.get("flops", 0.0) / v["launches"]
        issued = max(v.get("issued", 0), v["launches"])
        e = {"launches": v["launches"], "issued": issued, "ms_per_launch": round(ms, 4),
             "ms_total_est": round(ms * issued, 2)}
        res = []
        if bpl > 0:
            gbs = bpl / (ms / 1e3) / 1e9
            e.update({"GB/s": round(gbs, 1), "frac_hbm": round(gbs / hbm_peak, 4)})
            res.append(("hbm", bpl / (hbm_peak * 1e9), gbs, hbm_peak, "GB/s", bpl, peak_kind))
        if fpl > 0:
            tf = fpl / (ms / 1e3) / 1e12
            fp64 = bpl == 0
            pk = (fp64_peak or FP64_PEAK_TFLOPS) if fp64 else FP32_PEAK_TFLOPS
            e.update({"TFLOP/s": round(tf, 3), ("frac_fp64" if fp64 else "frac_fp32"): round(tf / pk, 4)})
            res.append(("alu", fpl / (pk * 1e12), tf, pk, "TFLOP/s", fpl,
                        ("measured FP64 FMA throughput" if fp64_peak else "nominal FP64") if fp64
                        else "FP32 from unit counts and clock"))
        if not res:
            continue
        bound = max(res, key=lambda r: r[1])
        e["bound"] = bound[0] if bound[0] == "hbm" else ("alu-fp64" if bpl == 0 else "alu-fp32")
        kernels[k] = e
        cand.append((ms * issued, k, bound, ms))

    def roof_of(item):
        total, name, b, ms = item
        kind, _, ach, pk, unit, amount, pkind = b
        cap = NCU_TRAFFIC.get(name)
        traffic = None
        if cap and prof[name]["bytes"] > 0:
            traffic = round(cap["bytes"] * (prof[name]["bytes"] / prof[name]["launches"]) / cap["algorithmic"])
        return {"kernel": name, "bound": kind, "achieved": round(ach, 3), "peak": round(pk, 2), "unit": unit,
                "frac": round(ach / pk, 4), "traffic": traffic, "peak_kind": pkind,
                ("bytes_per_launch" if unit == "GB/s" else "flops_per_launch"): amount, "launch_ms": ms}

    top = max(cand, default=None)
    top_hbm = max((c for c in cand if c[2][0] == "hbm"), default=None)
    # one whole inner-precision CG iteration (k1 + k2 + k3) of each operator:
    # the algorithmic bytes of the three launches over their summed time
    for op in ("wilson", "sw"):
        ks = [k for k in prof if k.startswith(op + ".k") and prof[k]["launches"]]
        if len(ks) == 3:
            ms = sum(prof[k]["ms"] / prof[k]["launches"] for k in ks)
            by = sum(prof[k]["bytes"] / prof[k]["launches"] for k in ks)
            gbs = by / (ms / 1e3) / 1e9
            kernels[op + ".iteration"] = {"kernels": sorted(ks), "ms": round(ms, 4), "GB/s": round(gbs, 1),
                                          "frac_hbm": round(gbs / hbm_peak, 4)}
    return kernels, (roof_of(top) if top else None), (roof_of(top_hbm) if top_hbm else None)


# ------------------------------------------------------------------ our arm
def autotune_layout(sw, dims, Ud, W, prec, n_sw, n_w, stream, iters=48):
    """Width x site order for this step's batches: sw_autotune_layout per
    operator on the first configuration, then the site order (one setting for
    both operators: lexicographic or a site-block shape) with the smallest sum
    of the operators' best times, and per operator the fastest width under
    that order."""
    if prec == sw.SW_PREC_F64:
        return {"skipped": "the FP64 path has one layout"}
    times = {}
    if n_sw:
        sw.sw_hypercube_build(dims, Ud, W, stream=stream)
        _, times["sw"] = sw.sw_autotune_layout(dims, sw.SW_OP_STAGGERED_WILSON, Ud, W, n_sw, prec, 1.0, iters,
                                               stream=stream)
    if n_w:
        _, times["wilson"] = sw.sw_autotune_layout(dims, sw.SW_OP_WILSON, Ud, None, n_w, prec, R_WILSON, iters,
                                                   stream=stream)
    shapes = range(sw.SW_SITE_SHAPES)
    total = {b: sum(min(t[(w, b)] for w in (1, 2, 4)) for t in times.values()) for b in shapes}
    blk = min(total, key=total.get)
    sw.sw_set_param(sw.SW_PARAM_SITE_BLOCKING, blk)
    keys = {"sw": sw.SW_PARAM_NS_SW, "wilson": sw.SW_PARAM_NS_WILSON}
    for op, t in times.items():
        sw.sw_set_param(keys[op], min((1, 2, 4), key=lambda w: t[(w, blk)]))
    return {"iters": iters, "site_blocking": blk,
            "ms": {op: {f"ns{w}_shape{b}": round(v, 2) for (w, b), v in sorted(t.items())} for op, t in times.items()}}


def run_ours(args):
    import torch
    import paper_1312_3265_gb300 as sw

    rank, world, local = dist_env()
    use_dist = world > 1
    if use_dist:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if use_dist else 0)
    torch.cuda.set_device(dev)
    sw.lib()
    prec = {"mixed": sw.SW_PREC_F32_RELIABLE, "f16": sw.SW_PREC_F16_RELIABLE, "f64": sw.SW_PREC_F64}[args.precision]
    if args.delta is not None:
        sw.sw_set_param(sw.SW_PARAM_RELIABLE_DELTA_F16 if args.precision == "f16" else sw.SW_PARAM_RELIABLE_DELTA,
                        args.delta)
    if args.chunk is not None:
        sw.sw_set_param(sw.SW_PARAM_CHUNK, args.chunk)
    if args.graphs is not None:
        sw.sw_set_param(sw.SW_PARAM_GRAPHS, args.graphs)
    if args.site_blocking is not None:
        sw.sw_set_param(sw.SW_PARAM_SITE_BLOCKING, args.site_blocking)
    if args.group_fast is not None:
        sw.sw_set_param(sw.SW_PARAM_GROUP_FAST, args.group_fast)
    if args.ns_sw is not None:
        sw.sw_set_param(sw.SW_PARAM_NS_SW, args.ns_sw)
    if args.ns_wilson is not None:
        sw.sw_set_param(sw.SW_PARAM_NS_WILSON, args.ns_wilson)
    K, Wm = args.steps, args.warmup
    seeds = sorted({seed_for(s, rank, world) for s in range(K + Wm)})
    masses = MASSES if args.masses is None else tuple(float(v) for v in args.masses.split(","))
    dims = tuple(int(v) for v in args.dims.split("x"))
    Uh, chi_sw_h, m_sw, chi_w_h, m_w = host_inputs(seeds, masses, args.w_sources, dims, args.sources)
    V = int(np.prod(dims))

    if args.ops == "sw":
        chi_w_h, m_w = chi_w_h[:0], []
    if args.ops == "wilson":
        chi_sw_h, m_sw = chi_sw_h[:0], []
    U = {s: torch.from_numpy(Uh[s]).to(dev) for s in seeds}
    W = torch.empty((V if args.ops != "wilson" else 1, 8, 3, 3), dtype=torch.complex128, device=dev)
    chi_sw = torch.from_numpy(chi_sw_h).to(dev)
    chi_w = torch.from_numpy(chi_w_h).to(dev)
    x_sw = torch.empty_like(chi_sw)
    x_w = torch.empty_like(chi_w)
    stream = torch.cuda.current_stream(dev)
    tune = (autotune_layout(sw, dims, U[seeds[0]], W, prec, len(m_sw), len(m_w), stream)
            if args.autotune else None)

    # The staggered Wilson batch (its FP64 hypercube build and reliable
    # updates are bound by the FP64 pipe) and the Wilson batch (bound by HBM)
    # are independent.  By default they run one after the other, so that the
    # kernel timings of the roofline report are those of each kernel alone;
    # with --concurrent-ops they run at once, each on its own stream from its
    # own host thread (the library's entry points are thread-safe).
    stream_sw = torch.cuda.Stream(dev) if (args.ops == "both" and args.concurrent_ops) else stream
    ev_start, ev_sw = torch.cuda.Event(), torch.cuda.Event()

    def step(seed, Ud, csw, cw, xsw, xw, precision=None):
        pr = prec if precision is None else precision
        res = {"sw": [], "w": []}

        def solve_sw():
            try:
                stream_sw.wait_event(ev_start)
                with torch.cuda.stream(stream_sw):
                    sw.sw_hypercube_build(dims, Ud, W, stream=stream_sw)
                    xsw.zero_()
                    rc1, res["sw"] = sw.cgne_solve_batch(dims, sw.SW_OP_STAGGERED_WILSON, Ud, W, csw, xsw, m_sw,
                                                         1.0, TOL, 100000, pr, stream=stream_sw)
                ev_sw.record(stream_sw)
            except BaseException as exc:  # re-raised by the caller after the join
                res["err"] = exc

        ev_start.record(stream)
        th = None
        if args.ops in ("both", "sw"):
            if stream_sw is stream:
                solve_sw()
            else:
                th = threading.Thread(target=solve_sw)
                th.start()
        if args.ops in ("both", "wilson"):
            xw.zero_()
            rc2, res["w"] = sw.cgne_solve_batch(dims, sw.SW_OP_WILSON, Ud, None, cw, xw, m_w, R_WILSON, TOL, 100000,
                                                pr, stream=stream)
        if th is not None:
            th.join()
        if "err" in res:
            raise res["err"]
        if args.ops in ("both", "sw"):
            stream.wait_event(ev_sw)
        inf_sw, inf_w = res["sw"], res["w"]
        for inf in inf_sw + inf_w:
            if inf.status != sw.SW_OK or not (inf.true_rel_resid <= TOL):
                raise RuntimeError(f"solve failed: {inf}")
        return inf_sw, inf_w

    for s in range(Wm):
        step(seed_for(s, rank, world), U[seed_for(s, rank, world)], chi_sw, chi_w, x_sw, x_w)
    # FP64 FMA throughput of this GPU (the FP64 matvecs' roofline denominator),
    # measured before the timed region
    fp64_peak = sw.sw_measure_fp64_peak(stream)

    # ---- timed region: device-resident inputs
    clocks = ClockSampler(dev.index)
    sw.sw_profile_reset()
    sw.sw_profile_enable(True)
    launches0 = sw.sw_kernel_launches()
    if use_dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    infos = []
    for s in range(Wm, Wm + K):
        sd = seed_for(s, rank, world)
        infos.append(step(sd, U[sd], chi_sw, chi_w, x_sw, x_w))
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ck = clocks.stop()
    ms = e0.elapsed_time(e1)
    launches = sw.sw_kernel_launches() - launches0
    sw.sw_profile_enable(False)
    prof = sw.sw_profile_read()
    ms = max_over_ranks(ms, dev)
    if use_dist:
        dist.barrier()

    n_solves = (len(m_sw) + len(m_w)) * K * world
    value = n_solves / (ms / 1e3)

    # ---- end to end through the public API, host buffers in pinned memory.
    # Every step copies its links and sources from pinned host memory and
    # reads its solutions back.  The copies run on a second stream into
    # double buffers: step s+1's inputs go up while step s solves, and step
    # s's solutions come down while step s+1 solves (a serving loop's
    # pipelining); the timed region spans all copies and solves.
    e2e = None
    if not args.no_e2e:
        U_pin = {s: torch.from_numpy(Uh[s]).pin_memory() for s in seeds}
        csw_pin = torch.from_numpy(chi_sw_h).pin_memory()
        cw_pin = torch.from_numpy(chi_w_h).pin_memory()
        xsw_pin = [torch.empty(chi_sw_h.shape, dtype=torch.complex128).pin_memory() for _ in range(2)]
        xw_pin = [torch.empty(chi_w_h.shape, dtype=torch.complex128).pin_memory() for _ in range(2)]
        Ud = [torch.empty_like(U[seeds[0]]) for _ in range(2)]
        csw_d = [torch.empty_like(chi_sw) for _ in range(2)]
        cw_d = [torch.empty_like(chi_w) for _ in range(2)]
        xsw_d = [torch.empty_like(chi_sw) for _ in range(2)]
        xw_d = [torch.empty_like(chi_w) for _ in range(2)]
        cs = torch.cuda.Stream(dev)
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_done = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]

        def upload(k, sd):
            b = k % 2
            with torch.cuda.stream(cs):
                cs.wait_event(ev_done[b])  # the solve that last read buffer b has finished
                Ud[b].copy_(U_pin[sd], non_blocking=True)
                csw_d[b].copy_(csw_pin, non_blocking=True)
                cw_d[b].copy_(cw_pin, non_blocking=True)
                ev_in[b].record(cs)

        if use_dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        steps = list(range(Wm, Wm + K))
        upload(0, seed_for(steps[0], rank, world))
        for k, s in enumerate(steps):
            b = k % 2
            stream.wait_event(ev_in[b])
            stream.wait_event(ev_out[b])  # solutions of step k-2 are on the host
            if k + 1 < len(steps):
                upload(k + 1, seed_for(steps[k + 1], rank, world))
            step(seed_for(s, rank, world), Ud[b], csw_d[b], cw_d[b], xsw_d[b], xw_d[b])
            ev_done[b].record(stream)
            with torch.cuda.stream(cs):
                cs.wait_event(ev_done[b])
                xsw_pin[b].copy_(xsw_d[b], non_blocking=True)
                xw_pin[b].copy_(xw_d[b], non_blocking=True)
                ev_out[b].record(cs)
        stream.wait_stream(cs)
        f1.record(stream)
        torch.cuda.synchronize(dev)
        ems = f0.elapsed_time(f1)
        ems = max_over_ranks(ems, dev)
        h2d = Uh[seeds[0]].nbytes + chi_sw_h.nbytes + chi_w_h.nbytes
        d2h = chi_sw_h.nbytes + chi_w_h.nbytes
        e2e = {"value": n_solves / (ems / 1e3), "unit": "solves/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": ems / K,
               "note": "inputs up and solutions down on a second stream, double-buffered across steps"}

    # ---- plain FP64 CG on one configuration of the same workload (comparison)
    f64 = None
    if not args.no_f64 and prec != sw.SW_PREC_F64:
        torch.cuda.synchronize(dev)
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sd = seed_for(Wm, rank, world)
        g0.record(stream)
        step(sd, U[sd], chi_sw, chi_w, x_sw, x_w, precision=sw.SW_PREC_F64)
        g1.record(stream)
        torch.cuda.synchronize(dev)
        fms = g0.elapsed_time(g1)
        f64 = {"value": round((len(m_sw) + len(m_w)) / (fms / 1e3), 3), "unit": "solves/s",
               "ms_per_step": round(fms, 1), "note": "same workload, one configuration, FP64 inner iterations"}

    serving = None
    if args.serving_requests > 0 and world == 1:
        serving = run_serving(sw, torch, dev, args)
    even_odd = None
    if (not args.no_even_odd and args.ops in ("both", "wilson") and dims == DIMS and args.sources == "point"
            and prec != sw.SW_PREC_F16_RELIABLE):
        sd = seed_for(Wm, rank, world)
        even_odd = run_even_odd(sw, torch, dev, U[sd], chi_w, m_w, prec)
    batched = None if (args.no_batched or world > 1) else run_batched(sw, torch, dev)
    large = None if (args.no_large_volume or world > 1) else run_large_volume(sw, torch, dev)

    # ---- per-operator statistics
    it_sw = [i.iters for st in infos for i in st[0]]
    it_w = [i.iters for st in infos for i in st[1]]
    by_mass = {"sw": {}, "wilson": {}}
    kap = {"sw": {}, "wilson": {}}  # sqrt(kappa) of (D+m)^+(D+m) from each solve's Ritz values
    for st in infos:
        for m, i in zip(m_sw, st[0]):
            by_mass["sw"].setdefault(m, []).append(i.iters)
            kap["sw"].setdefault(m, []).append(float(np.sqrt(i.kappa)))
        for m, i in zip(m_w, st[1]):
            by_mass["wilson"].setdefault(m, []).append(i.iters)
            kap["wilson"].setdefault(m, []).append(float(np.sqrt(i.kappa)))
    kmean = {op: {str(m): round(float(np.mean(v)), 2) for m, v in kap[op].items()} for op in kap}
    kratio = {str(m): round(float(np.mean(kap["wilson"][m]) / np.mean(kap["sw"][m])), 3)
              for m in kap["sw"] if m in kap["wilson"]}
    lat_sw = [st[0][0].seconds * 1e3 for st in infos if st[0]]
    lat_w = [st[1][0].seconds * 1e3 for st in infos if st[1]]
    lats = sorted([v for v in lat_sw for _ in m_sw] + [v for v in lat_w for _ in m_w]) or [0.0]

    peak, peak_kind = measured_peaks()
    kernels, roof, roof_hbm = classify_kernels(prof, peak, peak_kind, fp64_peak)

    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "solves/s", "n_gpus": world, "steps": K,
        "warmup": Wm, "ms_per_step": round(ms / K, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": {sw.SW_PREC_F32_RELIABLE: "f32+f64", sw.SW_PREC_F16_RELIABLE: "f16-storage/f32+f64"}.get(prec, "f64"),
        "data": "synthetic",
        "config": workload_config(WORKLOAD if (dims == DIMS and args.sources == "point") else
                                  f"CGNE batch per configuration: {len(m_sw)} staggered Wilson + {len(m_w)} Wilson "
                                  f"solves, {args.sources} sources", dims, masses),
        "settings": {"solves_per_step": len(m_sw) + len(m_w), "r": 1.0,
                     "precision": args.precision, "configurations": "seeds 0-9, mean plaquette 0.59",
                     "reliable_delta": sw.sw_get_param(sw.SW_PARAM_RELIABLE_DELTA_F16 if args.precision == "f16"
                                                       else sw.SW_PARAM_RELIABLE_DELTA),
                     "chunk": int(sw.sw_get_param(sw.SW_PARAM_CHUNK)),
                     "graphs": int(sw.sw_get_param(sw.SW_PARAM_GRAPHS)),
                     "site_blocking": int(sw.sw_get_param(sw.SW_PARAM_SITE_BLOCKING)),
                     "group_fast": int(sw.sw_get_param(sw.SW_PARAM_GROUP_FAST)),
                     "autotune": tune,
                     "systems_per_thread": {"sw": int(sw.sw_get_param(sw.SW_PARAM_NS_SW)),
                                            "wilson": int(sw.sw_get_param(sw.SW_PARAM_NS_WILSON))},
                     "parallelism": f"replicas x{world}",
                     "operator_batches": ("concurrent, one stream and host thread each"
                                          if (args.concurrent_ops and args.ops == "both") else "one after the other")},
        "clocks": ck, "gpu_launches": int(launches), "roofline": roof, "roofline_hbm_top": roof_hbm,
        "fp64_peak_tflops": {"value": round(fp64_peak, 4), "kind": "measured",
                             "how": "library FMA-throughput kernel (sw_measure_fp64_peak): every SM filled with "
                                    "independent FP64 FMA chains, best of 3 event-timed launches"},
        "kernels": kernels,
        "latency_ms": {"p50": round(float(np.percentile(lats, 50)), 2),
                       "p99": round(float(np.percentile(lats, 99)), 2),
                       "note": "time to solution of each solve's batch"},
        "operators": {
            "sw": {"solves": len(m_sw), "iters_mean": float(np.mean(it_sw)) if it_sw else None,
                   "batch_ms_mean": float(np.mean(lat_sw)) if lat_sw else None,
                   "iters_by_mass": {str(m): float(np.mean(v)) for m, v in by_mass["sw"].items()}},
            "wilson": {"solves": len(m_w), "iters_mean": float(np.mean(it_w)) if it_w else None,
                       "batch_ms_mean": float(np.mean(lat_w)) if lat_w else None,
                       "iters_by_mass": {str(m): float(np.mean(v)) for m, v in by_mass["wilson"].items()}},
            "iters_ratio_w_over_sw": float(np.mean(it_w) / np.mean(it_sw)) if it_sw and it_w else None,
            "sqrt_kappa_by_mass": kmean,
            "sqrt_kappa_ratio_w_over_sw": kratio,
            "kappa_note": ("sqrt of lambda_max/lambda_min of (D+m)^+(D+m) from each solve's CG coefficients "
                           "(Lanczos Ritz values, a lower bound on kappa); the paper's free-field ratio "
                           "kappa_W^1/2 / kappa_SW^1/2 tends to 8/sqrt(5) = 3.58 as m -> 0 (Sec. 3)"),
            "paper_context": "Sec. 3: iteration ratio W/SW almost 2 on thermalised beta=6 fields "
                             "(not comparable: synthetic links)"},
    }
    if e2e:
        line["e2e"] = e2e
    if f64:
        line["f64_baseline"] = f64
    if serving:
        line["serving"] = serving
    if even_odd:
        line["even_odd"] = even_odd
    if batched:
        line["batched"] = batched
    if large:
        line["large_volume"] = large
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(Uh[seeds[0]], by_mass, dims)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if use_dist:
        dist.destroy_process_group()


# ------------------------------------------------------------------ further workloads
def run_workload(sw, torch, dev, dims, op, precision, nsrc, masses, steps=1, warmup=1, persistent=False):
    """One operator's batch on one lattice (configuration seed 0, mean
    plaquette 0.59): nsrc real Z2-noise sources x the masses, one
    cgne_solve_batch per step to the FP64 true residual 1e-8.  The timed steps
    run with kernel timing on (host-driven rounds) unless `persistent`, which
    runs each batch as one device-driven CUDA graph launch (no kernel timing).
    Returns solves/s (CUDA events on the stream), iterations and the stencil
    kernels' roofline fractions."""
    import lattice_synth as ls
    V = ls.volume(dims)
    nc = 3 if op == sw.SW_OP_STAGGERED_WILSON else 12
    shape = (V, 3) if nc == 3 else (V, 4, 3)
    U = torch.from_numpy(ls.su3_links(dims, 0, ls.PLAQ_EPS, processes=min(16, os.cpu_count() or 1))).to(dev)
    W = None
    if nc == 3:
        W = torch.empty((V, 8, 3, 3), dtype=torch.complex128, device=dev)
        sw.sw_hypercube_build(dims, U, W)
    ms = [m for m in masses for _ in range(nsrc)]
    chi = torch.empty((len(ms),) + shape, dtype=torch.complex128, device=dev)
    for k in range(nsrc):
        z = torch.from_numpy(ls.z2_source(dims, nc, k).reshape(shape)).to(dev)
        for i in range(len(masses)):
            chi[i * nsrc + k] = z
        del z
    x = torch.zeros_like(chi)
    stream = torch.cuda.current_stream(dev)
    old = sw.sw_get_param(sw.SW_PARAM_PERSISTENT)

    def solve():
        x.zero_()
        rc, infos = sw.cgne_solve_batch(dims, op, U, W, chi, x, ms, 1.0, TOL, 100000, precision, stream=stream)
        for inf in infos:
            if inf.status != sw.SW_OK or not (inf.true_rel_resid <= TOL):
                raise RuntimeError(f"solve failed: {inf}")
        return infos

    try:
        sw.sw_set_param(sw.SW_PARAM_PERSISTENT, 1 if persistent else 0)
        for _ in range(warmup):
            solve()
        if not persistent:
            sw.sw_profile_reset()
            sw.sw_profile_enable(True)
        launches0 = sw.sw_kernel_launches()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos = []
        for _ in range(steps):
            infos += solve()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        sw.sw_profile_enable(False)
    finally:
        sw.sw_set_param(sw.SW_PARAM_PERSISTENT, old)
    tms = e0.elapsed_time(e1)
    by_mass = {}
    for m, inf in zip(ms * steps, infos):
        by_mass.setdefault(m, []).append(inf.iters)
    out = {"lattice": "x".join(map(str, dims)), "operator": "sw" if nc == 3 else "wilson",
           "precision": {sw.SW_PREC_F32_RELIABLE: "f32", sw.SW_PREC_F16_RELIABLE: "f16"}.get(precision, "f64"),
           "systems": len(ms), "sources": f"{nsrc} Z2", "masses": list(masses), "steps": steps,
           "solves_per_s": round(len(ms) * steps / (tms / 1e3), 3), "ms_per_step": round(tms / steps, 1),
           "iters_by_mass": {str(m): float(np.mean(v)) for m, v in by_mass.items()},
           "gpu_launches": int(sw.sw_kernel_launches() - launches0),
           "sqrt_kappa_by_mass": {str(m): round(float(np.mean([np.sqrt(i.kappa) for mm, i in zip(ms * steps, infos)
                                                                if mm == m])), 2) for m in masses}}
    if persistent:
        out["launch"] = "one device-driven CUDA graph launch per batch (conditional WHILE node over rounds)"
    else:
        peak, kind = measured_peaks()
        kernels, _, _ = classify_kernels(sw.sw_profile_read(), peak, kind)
        out["dslash"] = {k: {kk: v[kk] for kk in ("ms_per_launch", "frac_hbm", "frac_fp32", "bound") if kk in v}
                         for k, v in kernels.items() if ".k1." in k or ".k2." in k}
        out["iteration_frac_hbm"] = {k: v["frac_hbm"] for k, v in kernels.items() if k.endswith(".iteration")}
    del chi, x, U, W
    torch.cuda.empty_cache()
    sw.sw_trim_workspace()
    return out


def run_even_odd(sw, torch, dev, U, chi_w, m_w, prec, steps=2):
    """The headline configuration's Wilson batch (48 systems) solved on the
    even-odd Schur complement (outside the paper's unpreconditioned
    comparison), beside the same batch unpreconditioned, both to the full
    system's FP64 true residual 1e-8."""
    stream = torch.cuda.current_stream(dev)
    out = {}
    for name, op in (("unpreconditioned", sw.SW_OP_WILSON), ("even_odd", sw.SW_OP_WILSON_EVEN_ODD)):
        x = torch.zeros_like(chi_w)

        def solve():
            x.zero_()
            rc, infos = sw.cgne_solve_batch(DIMS, op, U, None, chi_w, x, m_w, R_WILSON, TOL, 100000, prec,
                                            stream=stream)
            for inf in infos:
                if inf.status != sw.SW_OK or not (inf.true_rel_resid <= TOL):
                    raise RuntimeError(f"solve failed: {inf}")
            return infos

        solve()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos = []
        for _ in range(steps):
            infos += solve()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        tms = e0.elapsed_time(e1)
        out[name] = {"solves_per_s": round(len(m_w) * steps / (tms / 1e3), 3),
                     "iters_mean": float(np.mean([i.iters for i in infos]))}
        del x
    out["speedup"] = round(out["even_odd"]["solves_per_s"] / out["unpreconditioned"]["solves_per_s"], 3)
    out["workload"] = ("the 16^3x32 configuration's 48 Wilson systems (12 spin-colour point sources x 4 masses), "
                       "FP32 inner iterations, CGNE on D^ = M - D_eo D_oe / M over the even sites")
    return out


def run_large_volume(sw, torch, dev):
    """48^3x96 staggered Wilson and 32^3x64 Wilson at the smallest bare mass
    0.01 and three more, 4 Z2 sources each, FP32 storage and FP16 storage
    (12-real links, per-site-scaled vectors), FP64 reliable updates."""
    masses = (0.01, 0.02, 0.05, 0.1)
    out = []
    for dims, op in (((48, 48, 48, 96), sw.SW_OP_STAGGERED_WILSON), ((32, 32, 32, 64), sw.SW_OP_WILSON)):
        for prec in (sw.SW_PREC_F32_RELIABLE, sw.SW_PREC_F16_RELIABLE):
            out.append(run_workload(sw, torch, dev, dims, op, prec, 4, masses))
    return out


def run_batched(sw, torch, dev):
    """24^3x48, 12 Z2 sources x 6 masses per operator (72 systems each), FP32
    inner iterations with FP64 reliable updates: each operator's batch as one
    device-driven CUDA graph launch, then one host-driven step with kernel timing."""
    masses = (0.02, 0.04, 0.06, 0.1, 0.15, 0.2)
    out = {}
    for op, name in ((sw.SW_OP_STAGGERED_WILSON, "sw"), (sw.SW_OP_WILSON, "wilson")):
        out[name] = {"persistent": run_workload(sw, torch, dev, (24, 24, 24, 48), op, sw.SW_PREC_F32_RELIABLE, 12,
                                                masses, persistent=True),
                     "profiled": run_workload(sw, torch, dev, (24, 24, 24, 48), op, sw.SW_PREC_F32_RELIABLE, 12,
                                              masses, warmup=0)}
    tot = sum(v["persistent"]["systems"] for v in out.values())
    secs = sum(v["persistent"]["systems"] / v["persistent"]["solves_per_s"] for v in out.values())
    out["solves_per_s_both_operators"] = round(tot / secs, 3)
    return out


# ------------------------------------------------------------------ serving phase
def run_serving(sw, torch, dev, args, seed=0, slots=8):
    """Poisson stream of solve requests through the continuous-batching server:
    lattices drawn uniformly from --serving-lattices (one resident gauge field
    each), operator uniform (staggered Wilson or Wilson), inner precision
    uniform (FP32 or FP16 storage; FP64 reliable updates), bare mass uniform in
    [0.02, 0.2], complex Gaussian sources, tol 1e-8.  Requests name a field,
    operator and precision; the server admits them by device memory, creating
    each (field, operator, precision) engine on demand within its budget.  The
    rate is 80% of the capacity measured by a burst of requests first (after
    one warm-up request per engine)."""
    import lattice_synth as ls
    lats = [tuple(int(v) for v in t.split("x")) for t in args.serving_lattices.split(",")]
    rng = np.random.default_rng(seed)
    srv = sw.Server(200 << 30)
    classes, pools, fields = [], [], []
    precs = (sw.SW_PREC_F32_RELIABLE, sw.SW_PREC_F16_RELIABLE)
    for li, dims in enumerate(lats):
        Ud = torch.from_numpy(ls.su3_links(dims, 100 + li, ls.PLAQ_EPS, processes=min(16, os.cpu_count() or 1))).to(dev)
        f = srv.add_field(dims, Ud, slots)
        del Ud
        V = ls.volume(dims)
        for op in (sw.SW_OP_STAGGERED_WILSON, sw.SW_OP_WILSON):
            nc = 3 if op == sw.SW_OP_STAGGERED_WILSON else 12
            srcs = []
            for j in range(2):
                c = torch.empty((V, nc), dtype=torch.complex128).pin_memory().numpy()
                c[:] = ls.gaussian_source(dims, nc, 1000 * li + 10 * op + j)
                srcs.append(c)
            for prec in precs:
                outs = [torch.empty((V, nc), dtype=torch.complex128).pin_memory().numpy() for _ in range(3 * slots)]
                classes.append((dims, op, prec, f))
                pools.append({"src": srcs, "free": list(range(len(outs))), "out": outs})
    pending = {}

    def submit(k):
        pool = pools[k]
        if not pool["free"]:
            return False
        o = pool["free"].pop()
        dims, op, prec, f = classes[k]
        rid = srv.submit_field(f, op, pool["src"][int(rng.integers(0, 2))], pool["out"][o],
                               float(rng.uniform(0.02, 0.2)), prec, tol=TOL)
        pending[rid] = (k, o)
        return True

    def collect(res):
        for rid, info in srv.poll(4096):
            k, o = pending.pop(rid)
            pools[k]["free"].append(o)
            res.append((k, info))

    def drain(res):
        while pending:
            collect(res)
            time.sleep(0.0005)

    warm = []
    for k in range(len(classes)):  # every engine created on demand once
        submit(k)
    drain(warm)
    # capacity: a burst of requests with every engine busy
    burst = []
    t0 = time.perf_counter()
    nb = 0
    for _ in range(3):
        for k in range(len(classes)):
            nb += submit(k)
    drain(burst)
    cap = nb / (time.perf_counter() - t0)
    rate = 0.8 * cap
    # Poisson stream at 80% of capacity
    n = args.serving_requests
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n))
    picks = rng.integers(0, len(classes), size=n)
    res = []
    t0 = time.perf_counter()
    for a, k in zip(arrivals, picks):
        while time.perf_counter() - t0 < a:
            collect(res)
            time.sleep(0.0002)
        while not submit(int(k)):  # this class's output buffers are all in flight
            collect(res)
            time.sleep(0.0002)
    drain(res)
    wall = time.perf_counter() - t0
    stats = srv.stats()
    srv.close()
    bad = [i for _, i in warm + burst + res if i.status != sw.SW_OK or not i.true_rel_resid <= TOL]
    if bad:
        raise RuntimeError(f"serving: {len(bad)} requests failed, e.g. {bad[0]}")
    lat = np.array([i.seconds * 1e3 for _, i in res])
    per = {}
    for k, i in res:
        d, op, prec, _ = classes[k]
        key = ("x".join(map(str, d)) + ("/sw" if op == sw.SW_OP_STAGGERED_WILSON else "/wilson") +
               ("/f16" if prec == sw.SW_PREC_F16_RELIABLE else "/f32"))
        per.setdefault(key, []).append(i.seconds * 1e3)
    return {"requests": n, "solves_per_s": round(n / wall, 2), "capacity_burst_solves_per_s": round(cap, 2),
            "offered_rate_per_s": round(rate, 2),
            "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 2),
                           "p99": round(float(np.percentile(lat, 99)), 2)},
            "latency_p50_ms_by_engine": {k: round(float(np.median(v)), 2) for k, v in sorted(per.items())},
            "slots_per_engine": slots, "engines": len(classes),
            "admission": {k: stats[k] for k in ("engines_created", "engines_retired", "requests_waited_for_memory",
                                                "bytes_charged", "budget")},
            "workload": "Poisson arrivals at 80% of burst capacity; lattices " + args.serving_lattices +
                        "; operator uniform; inner precision uniform over FP32 / FP16 storage (FP64 reliable "
                        "updates); mass U[0.02,0.2]; Gaussian sources; tol 1e-8; requests name a resident field "
                        "and the server creates each (field, operator, precision) engine on demand within its "
                        "device-memory budget"}


# ------------------------------------------------------------------ CPU oracle sample
def oracle_iteration_seconds(Uflat, k_sw=2, k_w=3, dims=DIMS):
    """Seconds per CG iteration of the oracle (numpy FP64) on the 16^3x32
    systems at m = 0.1: cg() run for k iterations, minus its final true-residual
    recomputation (two A applications, timed separately)."""
    import lattice_synth as ls
    from oracle import Lattice, operators as ops
    from oracle.cg import cg
    lat = Lattice(dims)
    U4 = lat.links(Uflat)
    out = {}
    for name, k, nc in (("sw", k_sw, 3), ("wilson", k_w, 12)):
        internal = (3,) if nc == 3 else (4, 3)
        if nc == 3:
            A = lambda v: ops.sw_dslash(lat, U4, ops.sw_dslash(lat, U4, v, 0.1), 0.1, dagger=True)
        else:
            A = lambda v: ops.wilson_dslash(lat, U4, ops.wilson_dslash(lat, U4, v, 0.1), 0.1, dagger=True)
        b = lat.field(ls.point_source(dims, nc, 0).reshape((-1,) + internal), internal)
        t0 = time.perf_counter()
        A(b)
        tA = time.perf_counter() - t0
        t0 = time.perf_counter()
        cg(A, b, 0.0, k)
        tk = time.perf_counter() - t0
        out[name] = {"s_per_iter": (tk - 2 * tA) / k, "s_per_A": tA, "iters_sampled": k}
    return out


def cpu_solves_per_s(per_iter, iters_by_mass, nsrc=None):
    """Solves/s of the oracle on one configuration's 60 solves: per solve, its
    iteration count times the seconds per iteration, plus b = (D+m)^+ chi and the
    final residual (about 1.5 A applications)."""
    total, n = 0.0, 0
    nsrc = nsrc or {"sw": 3, "wilson": 12}
    for op in ("sw", "wilson"):
        for m, its in iters_by_mass[op].items():
            mean_it = float(np.mean(its)) if isinstance(its, (list, tuple)) else float(its)
            k = len(its) if isinstance(its, (list, tuple)) else nsrc[op]
            total += k * (mean_it * per_iter[op]["s_per_iter"] + 1.5 * per_iter[op]["s_per_A"])
            n += k
    return n / total


def _oracle_worker_init(barrier):
    global _BARRIER
    _BARRIER = barrier


def _oracle_worker(job):
    """One oracle sample in a worker process: load the links, wait for every
    worker (so the timed regions run concurrently on all cores), time."""
    path, dims, k_sw, k_w = job
    Uflat = np.load(path)
    _BARRIER.wait()
    return oracle_iteration_seconds(Uflat, k_sw, k_w, dims)


def oracle_parallel(Uflat, dims, k_sw, k_w):
    """The oracle sample run concurrently by one process per host core (spawned:
    the parent already holds a CUDA context).  Returns the per-process results
    and the process count."""
    import multiprocessing as mp
    import tempfile
    n = max(1, min(os.cpu_count() or 1, 64))
    ctx = mp.get_context("spawn")
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "links.npy")
        np.save(path, Uflat)
        env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in env:
            os.environ[k] = "1"  # one thread per oracle process (inherited by the spawned workers)
        try:
            barrier = ctx.Barrier(n)
            with ctx.Pool(n, initializer=_oracle_worker_init, initargs=(barrier,)) as pool:
                res = pool.map(_oracle_worker, [(path, dims, k_sw, k_w)] * n, chunksize=1)
        finally:
            for k, v in env.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
    return res, n


def cpu_baseline(Uflat, iters_by_mass, dims=DIMS):
    t0 = time.perf_counter()
    res, n = oracle_parallel(Uflat, dims, 2, 3)
    spent = time.perf_counter() - t0
    value = sum(cpu_solves_per_s(per, iters_by_mass) for per in res)
    s_sw = float(np.mean([p["sw"]["s_per_iter"] for p in res]))
    s_w = float(np.mean([p["wilson"]["s_per_iter"] for p in res]))
    return {"value": round(value, 6), "unit": "solves/s", "cores": n, "kind": "oracle",
            "sample": (f"oracle (numpy FP64; staggered Wilson with the literal symmetrised C-product form of "
                       f"Gamma55, the oracle as it stands) CG on {'x'.join(map(str, dims))} links, m=0.1, one process per "
                       f"host core ({n}), all timed concurrently: each 2 staggered Wilson + 3 Wilson "
                       f"iterations ({spent:.1f} s wall); mean s/iter SW {s_sw:.2f}, W {s_w:.2f}; each "
                       f"process's rate scaled to the workload's 60 solves with this run's iteration counts "
                       f"per operator and mass, summed over the processes")}


# ------------------------------------------------------------------ reference arm (the oracle)
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import lattice_synth as ls
    if not all(ITERS_TABLE[op][m] > 0 for op in ITERS_TABLE for m in MASSES):
        print(json.dumps({"impl": "reference", "unavailable": "iteration table not filled"}))
        return
    vals, cores = [], 1
    for s in range(args.warmup + args.steps):
        Uflat = ls.su3_links(DIMS, s % N_SEEDS, ls.PLAQ_EPS, processes=min(16, os.cpu_count() or 1))
        t0 = time.perf_counter()
        res, cores = oracle_parallel(Uflat, DIMS, 1, 1)
        v = sum(cpu_solves_per_s(per, ITERS_TABLE) for per in res)
        if s >= args.warmup:
            vals.append((v, time.perf_counter() - t0))
    value = float(np.mean([v for v, _ in vals]))
    ms = float(np.mean([t for _, t in vals])) * 1e3
    sample = (f"per step: 1 staggered Wilson + 1 Wilson CG iteration of the oracle (numpy FP64; literal "
              f"symmetrised C-product form of Gamma55) on that step's "
              f"16^3x32 configuration at m=0.1, in one process per host core ({cores}) timed concurrently; each "
              f"process's rate scaled to the 60 solves with the mean iteration counts per operator and mass of "
              f"the workload, summed over the processes")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(WORKLOAD, DIMS, MASSES),
        "settings": {"parallelism": "cpu oracle, rank 0 only"},
        "cpu_baseline": {"value": round(value, 6), "unit": "solves/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 6), "unit": "solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
