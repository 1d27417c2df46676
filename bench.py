"""Benchmark of the GB300 relativistic space-charge FMM.

python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--passes fwd|fwd+adj]
                [--impl ours|reference] [--eta E] [--eta-alt E2] [--recompute] [--no-extras]

A step is one pass of the whole hot path on one batch of synthetic input:
setup (gbar), tree build, upward pass, dual tree traversal with the list
ordering, M2L, L2L, P2P and L2P (the forward field), and with --passes
fwd+adj the adjoint (the gradients of sum wE.E + wB.B with respect to x, p
and q).  The metric is particles per second of that step.  The default
workload is the largest single-GPU beam: 2^24 particles of a core-halo
bunch at gamma 200 (n = 8, N0 = 256, eta = 0.5), FP32, forward + adjoint,
with one set of per-level expansions (FMM_RECOMPUTE), as that beam's
configuration asks.
Inputs are resident on the GPU when the timed region starts; they are
larger than L2, and L2 is flushed (a 512 MiB write) before every timed step
anyway.  Under torchrun every rank runs its own replica of the workload (the
problems are independent, no data-path collective) and the reported value is
the sum over ranks of particles per second at the slowest rank's time
("scaling": "weak").

Beside the timed steps rank 0 measures, each bounded in time: the FP32 FMA
rate of the GPU (the roofline peak); every hot kernel alone, in a plan that
runs the stages one after another (the roofline's kernel durations); the
same beam at a second admissibility parameter with its own error; the FP64
GPU FMM against FP32 on a 2^20 draw of the beam; and the CPU oracle on all
host cores and on one core.

--impl reference times the FP64 CPU oracle (serial BLDTT + autograd adjoint)
on the host cores on a bounded sample of the same workload; it is a
deliberately plain program, reported as a baseline, not a target.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2302_07567_gb300.workloads import WORKLOADS, make_beam, make_weights, sample_targets  # noqa: E402

METRIC = "particles/s (E,B on all N; fwd and fwd+adjoint) at fixed rel. L2 error vs FP64"
# ALU-bound hot kernels: stage name -> (algorithmic flop per unit, stats key
# counting the units).  The FP32 adjoint without the gbar term evaluates both
# roles of every near-field pair in one kernel (stage adj_near, 84 flop per
# pair; its adj_source stage is then the far field and the chain rule only);
# otherwise adj_near is the target side (46) and adj_source the source side (67).
HOT = {"m2l": (32.0, "m2l_interactions"), "p2p_l2p": (32.0, "p2p_interactions"),
       "adj_m2lt": (32.0, "m2l_interactions")}
HOT_FUSED = {"adj_near": (84.0, "p2p_interactions")}
HOT_SPLIT = {"adj_near": (46.0, "p2p_interactions"), "adj_source": (67.0, "p2p_interactions")}
# Stage name of each hot kernel in the DRAM capture summary
KERNEL_OF = {"m2l": "k_m2l_pair", "p2p_l2p": "k_p2p_l2p", "adj_m2lt": "k_adj_m2l_pair", "adj_near": "k_adj_near"}
CONCURRENT = ("adj_near", "adj_m2lt")  # stages that share the GPU by default (two streams)
CONCURRENT_FP32_FWD = ("p2p_l2p", "m2l")  # FP32 forward: near-field P2P beside M2L and L2L
# HBM-bound stages: algorithmic bytes per particle (reads + writes of the
# data each stage must move once, FP32 plans; the bytes of the tree follow
# the passes of its algorithm, see hbm_bytes below)
HBM_FALLBACK_GBS = 6800.0  # only if the driver's measured peaks are absent
ELECTRON_MASS = 9.1093837015e-31  # kg (CODATA 2018), the tracking leg's particle mass
SMI_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="corehalo16m", choices=sorted(WORKLOADS))
    ap.add_argument("--N", type=int, default=None, help="particles (default: the workload's); a draw of the same beam")
    ap.add_argument("--eta", type=float, default=None, help="admissibility parameter (default: the workload's)")
    ap.add_argument("--eta-alt", type=float, default=0.4,
                    help="second admissibility parameter measured beside the line, with its own error (0: none)")
    ap.add_argument("--recompute", dest="recompute", action="store_true", default=None,
                    help="FMM_RECOMPUTE: one set of per-level expansions, the adjoint's written over the forward's "
                         "(default for the 2^24 core-halo beam, whose configuration names it)")
    ap.add_argument("--no-recompute", dest="recompute", action="store_false")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the serial per-kernel pass, the second eta, the FP64 side leg and the CPU baselines")
    ap.add_argument("--passes", default="fwd+adj", choices=["fwd", "fwd+adj"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-fp64-side", action="store_true", help="skip the FP64 GPU FMM side measurement")
    ap.add_argument("--sweep", action="store_true",
                    help="the paper's uniform-cube experiments (Figs. 2-4, Section 11) instead of the bench line")
    ap.add_argument("--sweep-part", default="all", choices=["all", "fig2", "fig3", "fig4", "sec11"],
                    help="with --sweep: one experiment only")
    ap.add_argument("--size-aware", action="store_true",
                    help="admissible pairs with fewer particle pairs than proxy-point pairs go to P2P (not in the paper)")
    ap.add_argument("--gbar-term", action="store_true",
                    help="adjoint with gbar as a function of p (FMM_GBAR_TERM): dL/dp includes dL/dgbar dgbar/dp")
    ap.add_argument("--profile", action="store_true",
                    help="run only the warm-up and the timed steps, print nothing (for profiler captures)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value: float, world: int, device=None) -> float:
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
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={SMI_FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except FileNotFoundError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                f = [c.strip() for c in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        busy = [s for s in sm if s > 0.5 * (max(smax) if smax else 1)]
        return {"sm_mhz": statistics.median(busy or sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons, "samples": len(rows)}


def hbm_peak():
    """Measured STREAM-style copy bandwidth of the GB300s (GB/s)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return HBM_FALLBACK_GBS, "fallback"


def hbm_bytes(st, w, N):
    """Algorithmic bytes of the HBM-bound stages of one FP32 forward.

    tree: the presort (8 passes of 8-bit digits over the 3N 12-byte (key,
      index) records, each read and written once per pass: 576 B/particle),
      the partition levels above the 4096-slot subtrees (per level each of the
      3 index arrays is read and written and its ranks read: 36 B/particle)
      and the subtree pass (the 3 index arrays and x read, the leaf order
      written: 40 B/particle);
    p2m: the particles' positions and masses (two float4) read once and the
      leaves' multipoles written once (4 m floats per leaf);
    l2p: positions (two float4) and near-field partial sums (two float4) read,
      the leaf's cumulative local (6 m floats) read once per leaf, the leaf
      order index read, E and B (6 floats) written.
    """
    kappa, m = st["kappa"], (w.n + 1) ** 3
    leaves = 1 << kappa
    top = max(0, kappa - max(0, (4096 // max(1, w.leaf)).bit_length() - 1))
    tree = N * (576 + 36 * top + 40)
    p2m = N * 32 + leaves * 4 * m * 4
    l2p = N * (32 + 32 + 4 + 24) + leaves * 6 * m * 4
    return {"tree": tree, "p2m": p2m, "l2p": l2p}


def fp32_peak(fmm, dev):
    """FP32 FMA throughput measured on this GPU (scalar and paired forms)."""
    r = {"scalar_tflops": fmm.fp32_fma_rate(False, dev), "paired_tflops": fmm.fp32_fma_rate(True, dev)}
    r["tflops"] = max(r["scalar_tflops"], r["paired_tflops"])
    return r


def traffic_of(kernel_stage, workload, N):
    """DRAM bytes per launch of a hot kernel from the committed ncu capture
    summary, scaled from the captured size to N particles.  None when there is
    no capture for this workload, or when the kernel's source changed since it
    was taken (the summary records the SHA-256 of the source file)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "dram_traffic_corehalo.json")
    try:
        with open(path) as f:
            cap = json.load(f)
    except (OSError, ValueError):
        return None, "no capture summary"
    k = KERNEL_OF.get(kernel_stage)
    e = cap.get("kernels", {}).get(k)
    if e is None or cap.get("workload") != workload:
        return None, f"no capture of {k} on {workload}"
    src = os.path.join(ROOT, "paper_2302_07567_gb300", "csrc", e["source"])
    with open(src, "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()
    if sha != e["source_sha256"]:
        return None, f"{e['source']} changed since the capture"
    return e["bytes"] * N / cap["N"], f"ncu capture at N={cap['N']} scaled by N ({e['source']} unchanged)"


def run_ours(args, rank, world, local):
    import torch

    from paper_2302_07567_gb300 import fmm

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = WORKLOADS[args.workload]
    N = w.N if args.N is None else int(args.N)
    eta = w.eta if args.eta is None else args.eta
    if args.recompute is None:
        args.recompute = bool(w.extra.get("recompute", False))
    x, p, q = make_beam(args.workload, N=N)
    wE, wB = make_weights(N)
    out_dt = torch.float32 if args.precision == "fp32" else torch.float64
    X, Pm, Q = (torch.as_tensor(a, device=dev) for a in (x, p, q))
    WE, WB = torch.as_tensor(wE, device=dev, dtype=out_dt), torch.as_tensor(wB, device=dev, dtype=out_dt)
    adj = args.passes == "fwd+adj"
    flags = (fmm.FMM_SIZE_AWARE if args.size_aware else 0) | (fmm.FMM_GBAR_TERM if args.gbar_term else 0)
    flags |= fmm.FMM_RECOMPUTE if args.recompute else 0
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    peak32 = fp32_peak(fmm, dev) if args.precision == "fp32" and not args.profile else None

    def make_plan(extra=0, e=eta):
        return fmm.Plan(N, w.n, w.leaf, e, precision=args.precision, flags=flags | extra)

    plan = make_plan(fmm.FMM_TIMING)

    def step(pl):
        E, B = pl.field(X, Pm, Q)
        if adj:
            return pl.adjoint(X, Pm, Q, WE, WB)
        return E, B

    warm = max(args.warmup, 3)
    for _ in range(warm):
        step(plan)
    torch.cuda.synchronize()
    st0 = plan.stats()
    hot = dict(HOT, **(HOT_FUSED if args.precision == "fp32" and not args.gbar_term else HOT_SPLIT))
    stage_hist = {}
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    launches0 = fmm.kernel_launches()
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()
            ev0[k].record(stream)
            step(plan)
            ev1[k].record(stream)
            for name, v in plan.stats()["stage_ms"].items():  # this step's stage events (same stream)
                stage_hist.setdefault(name, []).append(v)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    launches = fmm.kernel_launches() - launches0
    barrier(world)
    if args.profile:
        plan.close()
        return
    step_ms = [ev0[k].elapsed_time(ev1[k]) for k in range(args.steps)]
    t_steps = sum(step_ms) / 1e3
    t_max = max_over_ranks(t_steps, world, dev)
    value = N * world * args.steps / t_max
    stage_med = {k: statistics.median(v) for k, v in stage_hist.items()}

    # end to end through the public API with host buffers: H2D of the step's
    # inputs from pinned memory, the step, D2H of its results into pinned
    # memory, all inside the timed region, and the host waits for the results
    # at the end of every step (as a host-side integrator must).  The loss
    # weights go up on a copy stream while the forward runs and E, B come down
    # on it while the adjoint runs (copy engine); x, p, q go up before the
    # forward and the gradients come down after the adjoint, on the compute
    # stream, by the SMs (fmm.copy_).  The plan
    # is warm from the device-resident timing: one more warm-up step, then up
    # to five timed steps.
    hx, hp, hq = (torch.as_tensor(a).pin_memory() for a in (x, p, q))
    hwE, hwB = torch.as_tensor(wE, dtype=out_dt).pin_memory(), torch.as_tensor(wB, dtype=out_dt).pin_memory()
    h2d = (hx.numel() + hp.numel() + hq.numel()) * 8 + ((hwE.numel() + hwB.numel()) * hwE.element_size() if adj else 0)
    cstream = torch.cuda.Stream(dev)
    o_field = [torch.empty((N, 3), dtype=out_dt, pin_memory=True) for _ in range(2)]
    o_grad = [torch.empty(sh, dtype=torch.float64, pin_memory=True) for sh in ((N, 3), (N, 3), (N,))] if adj else []
    outs = o_grad + o_field
    Xd, Pd, Qd = (torch.empty(h.shape, dtype=h.dtype, device=dev) for h in (hx, hp, hq))

    def up_or_down(dst, src):
        # the copies the compute waits for go through the SMs (fmm.copy_),
        # which the first transfer of a buffer after a step takes faster
        # than the copy engine; rows of an odd N are not 16-byte multiples
        if (dst.numel() * dst.element_size()) % 16 == 0:
            fmm.copy_(dst, src)
        else:
            dst.copy_(src, non_blocking=True)

    e2e_steps = min(args.steps, 5)
    e2e_ms = []
    for k in range(1 + e2e_steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for d_, h_ in zip((Xd, Pd, Qd), (hx, hp, hq)):
            up_or_down(d_, h_)
        if adj:
            with torch.cuda.stream(cstream):
                WEd, WBd = hwE.to(dev, non_blocking=True), hwB.to(dev, non_blocking=True)
            w_ready = cstream.record_event()
        E, B = plan.field(Xd, Pd, Qd)
        f_done = stream.record_event()
        with torch.cuda.stream(cstream):
            cstream.wait_event(f_done)
            for o, r in zip(o_field, (E, B)):
                o.copy_(r, non_blocking=True)
        if adj:
            stream.wait_event(w_ready)
            for o, r in zip(o_grad, plan.adjoint(Xd, Pd, Qd, WEd, WBd)):
                up_or_down(o, r)
        torch.cuda.synchronize()
        if k >= 1:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
        del E, B
        if adj:
            del WEd, WBd
    d2h = sum(o.numel() * o.element_size() for o in outs)
    e2e_t = max_over_ranks(sum(e2e_ms) / 1e3, world, dev)
    e2e_value = N * world * e2e_steps / e2e_t
    del outs, o_field, o_grad, hx, hp, hq, hwE, hwB, Xd, Pd, Qd

    def rel(a, b):
        return float(torch.linalg.norm(a.double() - b) / torch.linalg.norm(b))

    # accuracy of this configuration against the FP64 brute force on sampled targets
    tg = torch.as_tensor(sample_targets(N, 4096), device=dev)
    E, B = plan.field(X, Pm, Q)
    gbar = plan.stats()["gbar"]
    Ed, Bd = fmm.direct_field(X, Pm, Q, gbar=gbar, targets=tg)
    err = max(rel(E[tg], Ed), rel(B[tg], Bd))
    del E, B
    plan.close()
    del plan
    torch.cuda.empty_cache()

    extra = {}
    if rank == 0 and not args.no_extras:
        extra = run_extras(args, fmm, torch, dev, w, N, eta, x, p, q, X, Pm, Q, WE, WB, adj, flags, step, rel, tg,
                           Ed, Bd, hot, st0)
    del X, Pm, Q, WE, WB
    torch.cuda.empty_cache()

    # roofline of the dominant kernel: the ALU-bound kernels against the
    # measured FP32 FMA rate, each timed alone in the serial pass (its own
    # duration), beside the stage time it takes inside the overlapped step
    clocks = clk.summary()
    kernels = {}
    serial = extra.get("serial_stage_ms", {})
    conc = set(CONCURRENT) | (set(CONCURRENT_FP32_FWD) if args.precision == "fp32" else set())
    for k, (per, unit) in hot.items():
        flop = per * st0[unit]
        in_step = stage_med.get(k, 0.0)
        alone = serial.get(k, 0.0)
        d = {"flop": flop, "ms_in_step": in_step, "shares_gpu_in_step": k in conc}
        if alone > 0:
            d.update(ms=alone, tflops=flop / (alone / 1e3) / 1e12)
            if peak32:
                d["frac"] = d["tflops"] / peak32["tflops"]
        if in_step > 0 and peak32:
            d["frac_in_step"] = flop / (in_step / 1e3) / 1e12 / peak32["tflops"]
        kernels[k] = d
    timed = [k for k in kernels if "ms" in kernels[k]]
    roof = None
    if timed:
        dom = max(timed, key=lambda k: kernels[k]["ms"])
        traffic, traffic_basis = traffic_of(dom, args.workload, N)
        roof = {"kernel": dom, "bound": "alu", "achieved": kernels[dom]["tflops"],
                "peak": peak32["tflops"] if peak32 else None, "unit": "TFLOP/s",
                "frac": kernels[dom].get("frac"), "traffic": traffic, "traffic_basis": traffic_basis,
                "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
                "timing": "kernel alone: stage events of an FMM_SERIAL plan (every stage on one stream, "
                          "one kernel after another), median of its steps",
                "peak_basis": (f"measured: FP32 FMA-rate kernel on this GPU, {peak32['scalar_tflops']:.1f} TFLOP/s "
                               f"scalar, {peak32['paired_tflops']:.1f} paired; SM clock median "
                               f"{clocks['sm_mhz']} MHz during the timed steps") if peak32 else None,
                "flop_basis": "algorithmic flop per pair (FMA = 2): M2L and M2L^T 32 per point pair, P2P 32, "
                              "adjoint near field 84 per particle pair for both roles in one kernel (FP32), "
                              "else 46 (target side) and 67 (source side)",
                "kernels": kernels}
        # kernels that share the GPU in the step (two streams) have no
        # duration of their own there: report each pair of branches over the
        # span they share, from the first one's start to the last one's end
        branches = {}
        pairs = (("forward", ("m2l", "p2p_l2p"), stage_med.get("p2p_l2p", 0.0)),
                 ("adjoint", ("adj_near", "adj_m2lt"),
                  stage_med.get("adj_total", 0.0) - stage_med.get("adj_lists", 0.0) - stage_med.get("adj_source", 0.0)))
        for name, ks, span in pairs:
            if all(k in kernels and kernels[k]["shares_gpu_in_step"] for k in ks) and span > 0 and peak32:
                fl = sum(kernels[k]["flop"] for k in ks)
                branches[name] = {"kernels": list(ks), "ms_in_step": span, "tflops": fl / (span / 1e3) / 1e12,
                                  "frac": fl / (span / 1e3) / 1e12 / peak32["tflops"]}
        roof["branches_in_step"] = branches
        # the whole step: every hot kernel's algorithmic flop over the timed
        # step (branches that share the GPU counted once, by their flop)
        step_flop = sum(kd["flop"] for kd in kernels.values())
        step_s = t_max / args.steps  # one rank's step (replicas: every rank runs the same work)
        roof["step"] = {"flop": step_flop, "ms": step_s * 1e3, "tflops": step_flop / step_s / 1e12,
                        "frac": step_flop / step_s / 1e12 / peak32["tflops"] if peak32 else None}

    # HBM-bound stages of the forward (tree with its presort, P2M, L2P)
    hpk, hbasis = hbm_peak()
    hbm = {}
    if args.precision == "fp32":
        for k, b in hbm_bytes(st0, w, N).items():
            ms = stage_med.get({"tree": "tree", "p2m": "p2m", "l2p": "l2p"}[k], 0.0)
            if ms > 0:
                hbm[k] = {"ms": ms, "bytes": b, "gbs": b / (ms / 1e3) / 1e9, "frac": b / (ms / 1e3) / 1e9 / hpk}
        hbm["peak_gbs"] = hpk
        hbm["peak_basis"] = hbasis
        hbm["bytes_basis"] = hbm_bytes.__doc__.split("\n\n")[0] + " (see bench.py hbm_bytes)"

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": world, "steps": args.steps,
            "warmup": warm, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64",
            "data": "synthetic (seeded beam generator)",
            "config": {"workload": args.workload, "N": N, "degree": w.n, "leaf": w.leaf, "eta": eta,
                       "passes": args.passes, "precision": args.precision, "replicas": world,
                       "recompute": bool(args.recompute),
                       "lists": "size-aware (M2L -> P2P below m^2 pairs)" if args.size_aware else "paper (Alg. 17)",
                       "adjoint_gbar": "gbar(p) live" if args.gbar_term else "gbar held fixed",
                       "l2": ("inputs larger than L2, and L2 flushed before every timed step (512 MiB write)"
                              if N * 56 > (129 << 20) else "L2 flushed before every timed step (512 MiB write)"),
                       "note": w.note},
            "rel_l2_error_vs_fp64_direct": err, "error_targets": 4096,
            "stage_ms": {k: round(v, 4) for k, v in stage_med.items() if v},
            "lists": {"p2p_pairs": st0["p2p_pairs"], "m2l_pairs": st0["m2l_pairs"], "kappa": st0["kappa"],
                      "p2p_interactions": st0["p2p_interactions"], "m2l_interactions": st0["m2l_interactions"]},
            "wall_ms_per_step": 1e3 * t_wall / args.steps,
            "e2e": {"value": e2e_value, "unit": "particles/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps": e2e_steps},
            "gpu_launches": launches, "launches_per_step": launches / args.steps,
            "roofline": roof, "hbm": hbm, "fp32_peak": peak32, "clocks": clocks,
            **{k: v for k, v in extra.items() if k not in ("serial_stage_ms", "cpu_baseline")},
        }
        if "cpu_baseline" in extra:
            line["cpu_baseline"] = extra["cpu_baseline"]
        print(json.dumps(line), flush=True)
    barrier(world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_extras(args, fmm, torch, dev, w, N, eta, x, p, q, X, Pm, Q, WE, WB, adj, flags, step, rel, tg, Ed, Bd, hot,
               st0):
    """Rank 0: per-kernel attribution, the second eta, the FP64 side leg and
    the CPU baselines (each bounded so the whole bench ends in minutes)."""
    out = {}
    # every kernel timed alone: a serial plan, one warm-up and two timed steps
    sp = fmm.Plan(N, w.n, w.leaf, eta, precision=args.precision, flags=flags | fmm.FMM_SERIAL | fmm.FMM_TIMING)
    step(sp)
    hist = {}
    for _ in range(2):
        step(sp)
        for k, v in sp.stats()["stage_ms"].items():
            hist.setdefault(k, []).append(v)
    torch.cuda.synchronize()
    out["serial_stage_ms"] = {k: statistics.median(v) for k, v in hist.items()}
    out["serial_stage_ms_report"] = {k: round(v, 3) for k, v in out["serial_stage_ms"].items() if v}
    sp.close()
    del sp
    torch.cuda.empty_cache()

    # the same beam at a second admissibility parameter, with its own error
    if args.eta_alt and args.eta_alt != eta:
        ap = fmm.Plan(N, w.n, w.leaf, args.eta_alt, precision=args.precision, flags=flags)
        step(ap)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 2
        a.record()
        for _ in range(reps):
            step(ap)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / reps
        E, B = ap.field(X, Pm, Q)
        e2 = max(rel(E[tg], Ed), rel(B[tg], Bd))
        out["eta_alt"] = {"eta": args.eta_alt, "value": N / (ms / 1e3), "unit": "particles/s", "ms_per_step": ms,
                          "steps": reps, "rel_l2_error_vs_fp64_direct": e2, "error_targets": 4096}
        del E, B
        ap.close()
        del ap
        torch.cuda.empty_cache()

    # the step recorded as CUDA graphs (fmm_step_graph_*) and replayed: the
    # same kernels in the same order, without a host launch for each; timed
    # on the host per replay, which waits for its forward's list check and
    # for its end
    gp = fmm.Plan(N, w.n, w.leaf, eta, precision=args.precision, flags=flags)
    Xg, Pg, Qg = X.clone(), Pm.clone(), Q.clone()
    gout = gp.record_step(Xg, Pg, Qg, *((WE, WB) if adj else ()))
    greps = 5 if N <= (1 << 22) else 2
    gp.replay()
    torch.cuda.synchronize()
    k0 = fmm.kernel_launches()
    t0 = time.perf_counter()
    for _ in range(greps):
        gp.replay()
    gms = (time.perf_counter() - t0) * 1e3 / greps
    out["graph"] = {"value": N / (gms / 1e3), "unit": "particles/s", "ms_per_step": gms, "steps": greps,
                    "kernels_per_step": (fmm.kernel_launches() - k0) / greps,
                    "timing": "host clock per replay (each replay waits for its end)"}
    del gout
    gp.close()
    del gp, Xg, Pg, Qg
    torch.cuda.empty_cache()

    # tracking: per step the forward field and a Boris push (electron
    # charge and mass per particle, dt = 1 ps), with the tree and lists kept
    # while admissible (fmm_field_reuse) and built anew every step (fmm_field)
    track = {"dt_s": 1e-12, "steps": 3}
    for reuse in (True, False):
        Xt, Pt = X.clone(), Pm.clone()
        tp = fmm.Plan(N, w.n, w.leaf, eta, precision=args.precision, flags=flags & ~fmm.FMM_RECOMPUTE)
        fmm.track(tp, Xt, Pt, Q, ELECTRON_MASS, 1e-12, 1, reuse)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        rebuilt = fmm.track(tp, Xt, Pt, Q, ELECTRON_MASS, 1e-12, track["steps"], reuse)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / track["steps"]
        track["reuse" if reuse else "rebuild"] = {"value": N / (ms / 1e3), "unit": "particles/s", "ms_per_step": ms,
                                                   "tree_and_lists_built": rebuilt}
        tp.close()
        del tp, Xt, Pt
        torch.cuda.empty_cache()
    out["tracking"] = track

    # FP64 GPU FMM against FP32 on a 2^20 draw of the same beam (the FP64
    # forward at 2^24 would take minutes)
    if args.precision == "fp32" and not args.no_fp64_side:
        Ns = min(N, 1 << 20)
        xs, ps, qs = make_beam(args.workload, N=Ns)
        Xs, Ps, Qs = (torch.as_tensor(v, device=dev) for v in (xs, ps, qs))
        tgs = torch.as_tensor(sample_targets(Ns, 4096), device=dev)
        side = {"sample": f"{args.workload} beam drawn at N={Ns} (same distribution), forward only, "
                          f"error vs FP64 brute force on 4096 sampled targets"}
        ref = None
        for prec in ("fp32", "fp64"):
            pl = fmm.Plan(Ns, w.n, w.leaf, eta, precision=prec)
            pl.field(Xs, Ps, Qs)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            E, B = pl.field(Xs, Ps, Qs)
            b.record()
            torch.cuda.synchronize()
            if ref is None:
                ref = fmm.direct_field(Xs, Ps, Qs, gbar=pl.stats()["gbar"], targets=tgs)
            side[f"{prec}_fwd_particles_per_s"] = Ns / (a.elapsed_time(b) / 1e3)
            side[f"{prec}_fwd_err"] = max(rel(E[tgs], ref[0]), rel(B[tgs], ref[1]))
            pl.close()
            del pl, E, B
            torch.cuda.empty_cache()
        out["fp64_side"] = side
        del Xs, Ps, Qs

    out["cpu_baseline"] = cpu_baseline(args.workload, adj)
    return out


def _oracle_step(x, p, q, wE, wB, w, adj):
    from oracle import bldtt, gradient
    plan = bldtt.build_plan(x, p, w.n, w.leaf, w.eta)
    if adj:
        gradient.fmm_gradient(x, p, q, wE, wB, plan)
    else:
        bldtt.fmm_fields(x, p, q, w.n, w.leaf, w.eta, plan=plan)


def _cpu_leg(workload: str, adj: bool, budget_s: float, threads: int, Ns: int):
    """Time the oracle on fresh draws of Ns particles until budget_s of CPU time is spent (at most 3 draws)."""
    import torch
    torch.set_num_threads(threads)
    w = WORKLOADS[workload]
    Ns = min(w.N, Ns)
    done, t_all, n_all = 0, 0.0, 0
    while t_all < budget_s and done < 3:
        x, p, q = make_beam(workload, N=Ns, seed_offset=done)
        wE, wB = make_weights(Ns, seed_offset=done)
        t0 = time.perf_counter()
        _oracle_step(x, p, q, wE, wB, w, adj)
        t_all += time.perf_counter() - t0
        n_all += Ns
        done += 1
    return {"value": n_all / t_all, "unit": "particles/s", "cores": torch.get_num_threads(), "kind": "oracle",
            "sample": f"{done} x serial FP64 BLDTT {'forward+autograd adjoint' if adj else 'forward'} on "
                      f"N={Ns} draws of {workload} (n={w.n}, leaf={w.leaf}, eta={w.eta}); {t_all:.1f} s of CPU time"}


def cpu_baseline(workload: str, adj: bool, budget_s: float = 10.0):
    """The oracle, as it stands, on bounded samples of the workload: on all the
    host's cores, and on one core (the paper's CPU baseline is a single core,
    Section 11), the latter in a child process pinned to one CPU with one
    thread in every numerical library."""
    allc = _cpu_leg(workload, adj, budget_s, os.cpu_count() or 1, 16384)
    code = ("import os, sys, json; os.sched_setaffinity(0, {min(os.sched_getaffinity(0))}); "
            f"sys.path.insert(0, {ROOT!r}); import bench; "
            f"print(json.dumps(bench._cpu_leg({workload!r}, {bool(adj)}, {budget_s}, 1, 4096)))")
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
        one = json.loads(r.stdout.strip().splitlines()[-1]) if r.returncode == 0 else {"error": r.stderr[-300:]}
    except (subprocess.TimeoutExpired, ValueError, IndexError) as e:
        one = {"error": str(e)[:300]}
    allc["single_core"] = one
    return allc


def run_reference(args, rank, world):
    if rank != 0:
        return
    import torch
    torch.set_num_threads(os.cpu_count() or 1)
    w = WORKLOADS[args.workload]
    adj = args.passes == "fwd+adj"
    Ns = min(w.N, 4096)
    times = []
    for k in range(max(args.warmup, 3) + args.steps):
        x, p, q = make_beam(args.workload, N=Ns, seed_offset=k)
        wE, wB = make_weights(Ns, seed_offset=k)
        t0 = time.perf_counter()
        _oracle_step(x, p, q, wE, wB, w, adj)
        if k >= max(args.warmup, 3):
            times.append(time.perf_counter() - t0)
    t = sum(times)
    value = Ns * args.steps / t
    line = {"metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded beam generator)",
            "impl": "reference",
            "config": {"workload": args.workload, "N_sample": Ns, "degree": w.n, "leaf": w.leaf, "eta": w.eta,
                       "passes": args.passes},
            "cpu_baseline": {"value": value, "unit": "particles/s", "cores": torch.get_num_threads(), "kind": "oracle",
                             "sample": f"each step: serial FP64 BLDTT on a fresh N={Ns} draw of {args.workload}"},
            "e2e": {"value": value, "unit": "particles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_sweep(args):
    """The paper's own experiments on its uniform-cube workload (Section 5), on this GPU.

    Fig. 2: forward time against the error of Eq. 5.1 for eta in {0.3, 0.4, 0.5} and
    n in {2, 4, 6, 8, 10} with N0 = (n+1)^3, N = 1.28e6.  Fig. 3: forward time against N
    for n = 4, N0 = 125, eta = 0.5.  Fig. 4: the stage times (each stage alone) and the
    interaction counts at, just above and halfway past the transitions N_t = 2^kappa N0
    of the same case.  Section 11 (Fig. 7): N = 2.56e7 with the same
    parameters.  Times are CUDA-event medians of the whole fmm_field call (inputs in HBM);
    errors are max over E, B of the relative L2 error on 4096 sampled targets against the
    FP64 brute force.  One JSON line per point.
    """
    import torch

    from paper_2302_07567_gb300 import fmm

    dev = torch.device("cuda", 0)

    def point(N, n, N0, eta, prec, reps=3, err=True, exp="", stages=False):
        x, p, q = make_beam("cube", N=N)
        X, Pm, Q = (torch.as_tensor(a, device=dev) for a in (x, p, q))
        # stages: every stage alone (FMM_SERIAL) with its own events
        plan = fmm.Plan(N, n, N0, eta, precision=prec, flags=(fmm.FMM_TIMING | fmm.FMM_SERIAL) if stages else 0)
        for _ in range(2):
            plan.field(X, Pm, Q)
        times = []
        for _ in range(reps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            E, B = plan.field(X, Pm, Q)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        out = {"sweep": exp, "N": N, "n": n, "N0": N0, "eta": eta, "precision": prec,
               "ms": statistics.median(times), "particles_per_s": N / (statistics.median(times) / 1e3)}
        if stages:
            st = plan.stats()
            out["kappa"] = st["kappa"]
            out["stage_ms"] = {k: round(st["stage_ms"][k], 4) for k in ("tree", "p2m", "upward", "traversal", "m2l",
                                                                         "l2l", "p2p_l2p", "l2p")}
            out["p2p_interactions"], out["m2l_interactions"] = st["p2p_interactions"], st["m2l_interactions"]
            out["p2p_pairs"], out["m2l_pairs"] = st["p2p_pairs"], st["m2l_pairs"]
        if err:
            st = plan.stats()
            tg = torch.as_tensor(sample_targets(N, 4096, tag=9), device=dev)
            Ed, Bd = fmm.direct_field(X, Pm, Q, gbar=st["gbar"], targets=tg)
            rel = lambda a, b: float(torch.linalg.norm(a.double() - b) / torch.linalg.norm(b))  # noqa: E731
            out["error"] = max(rel(E[tg], Ed), rel(B[tg], Bd))
            out["m2l_pairs"], out["p2p_pairs"] = st["m2l_pairs"], st["p2p_pairs"]
        print(json.dumps(out), flush=True)
        del plan
        torch.cuda.empty_cache()

    part = args.sweep_part
    if part in ("all", "fig2"):
        for eta in (0.3, 0.4, 0.5):
            for n in (2, 4, 6, 8, 10):
                point(1_280_000, n, (n + 1) ** 3, eta, "fp32", exp="fig2")
        for eta in (0.5,):
            for n in (2, 4, 6):
                point(1_280_000, n, (n + 1) ** 3, eta, "fp64", exp="fig2")
    if part in ("all", "fig3"):
        for N in (10_000, 20_000, 50_000, 100_000, 200_000, 500_000, 1_000_000, 2_000_000, 4_000_000, 8_000_000,
                  16_000_000):
            point(N, 4, 125, 0.5, "fp32", err=False, exp="fig3")
    if part in ("all", "fig4"):
        # the stages against N across the transitions N_t = 2^kappa N0, where
        # the tree gains a level (Section 5's model: P2P work halves, M2L work
        # doubles just above N_t)
        for kappa in (10, 11, 12, 13):
            Nt = (1 << kappa) * 125
            for N in (Nt, Nt + 1, (3 * Nt) // 2):
                point(N, 4, 125, 0.5, "fp32", err=False, exp="fig4", stages=True)
    if part in ("all", "sec11"):
        point(25_600_000, 4, 125, 0.5, "fp32", exp="sec11")
        point(25_600_000, 4, 125, 0.5, "fp64", reps=1, err=False, exp="sec11")


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.sweep:
        run_sweep(args)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
