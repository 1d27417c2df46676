"""Benchmark of the GB300 relativistic space-charge FMM.

python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--passes fwd|fwd+adj]
                [--impl ours|reference]

A step is one pass of the whole hot path on one batch of synthetic input:
setup (gbar), tree build, upward pass, dual tree traversal, list sort, M2L,
L2L, P2P + L2P (the forward field), and with --passes fwd+adj the adjoint
(the gradients of sum wE.E + wB.B with respect to x, p and q).  The metric
is particles per second of that step.  Inputs are resident on the GPU when
the timed region starts; L2 is flushed (a 512 MiB write) before every timed
step because one batch is smaller than L2.  Under torchrun every rank runs
its own replica of the workload (the problems are independent, no data-path
collective) and the reported value is the sum over ranks of particles per
second at the slowest rank's time ("scaling": "weak").

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
# hot kernels: stage name -> (algorithmic flop per unit, stats key counting the units).
# The FP32 adjoint without the gbar term evaluates both roles of every
# near-field pair in one kernel (stage adj_near, 84 flop per pair; its
# adj_source stage is then the far field and the chain rule only); otherwise
# adj_near is the target side (46) and adj_source the source side (67).
HOT = {"m2l": (32.0, "m2l_interactions"), "p2p_l2p": (32.0, "p2p_interactions"),
       "adj_m2lt": (32.0, "m2l_interactions")}
HOT_FUSED = {"adj_near": (84.0, "p2p_interactions")}
HOT_SPLIT = {"adj_near": (46.0, "p2p_interactions"), "adj_source": (67.0, "p2p_interactions")}
# DRAM bytes (read + write) per launch of each hot kernel on the cylinder64k
# fwd+adj step, from one `ncu --set full` capture per kernel (summary and
# command in profiles/hot_kernels_cylinder64k.md).  Valid only while the
# kernel is unchanged since that capture; reported for that workload only.
TRAFFIC_CYL64K = {"m2l": 2674688, "adj_m2lt": 3963392, "adj_near": 9885696 + 15360, "p2p_l2p": 3494144}
CONCURRENT = ("adj_near", "adj_m2lt")  # stages that overlap each other (two streams)
CONCURRENT_FP32_FWD = ("p2p_l2p", "m2l")  # FP32 forward: near-field P2P beside M2L and L2L
SMS = 152          # GB300 streaming multiprocessors
FP32_LANES = 128   # FP32 FMA lanes per SM
SMI_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="cylinder64k", choices=sorted(WORKLOADS))
    ap.add_argument("--passes", default="fwd+adj", choices=["fwd", "fwd+adj"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-fp64-side", action="store_true", help="skip the FP64 GPU FMM side measurement")
    ap.add_argument("--sweep", action="store_true",
                    help="the paper's uniform-cube experiments (Figs. 2, 3, Section 11) instead of the bench line")
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


def run_ours(args, rank, world, local):
    import torch

    from paper_2302_07567_gb300 import fmm

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = WORKLOADS[args.workload]
    N = w.N
    x, p, q = make_beam(args.workload)
    wE, wB = make_weights(N)
    out_dt = torch.float32 if args.precision == "fp32" else torch.float64
    X, Pm, Q = (torch.as_tensor(a, device=dev) for a in (x, p, q))
    WE, WB = torch.as_tensor(wE, device=dev, dtype=out_dt), torch.as_tensor(wB, device=dev, dtype=out_dt)
    adj = args.passes == "fwd+adj"
    sa_flag = fmm.FMM_SIZE_AWARE if args.size_aware else 0
    gb_flag = fmm.FMM_GBAR_TERM if args.gbar_term else 0
    plan = fmm.Plan(N, w.n, w.leaf, w.eta, precision=args.precision, flags=fmm.FMM_TIMING | sa_flag | gb_flag)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        E, B = plan.field(X, Pm, Q)
        if adj:
            return plan.adjoint(X, Pm, Q, WE, WB)
        return E, B

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    st0 = plan.stats()
    hot = dict(HOT, **(HOT_FUSED if args.precision == "fp32" and not args.gbar_term else HOT_SPLIT))
    stage_hist = {k: [] for k in hot}
    step_ms = []
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
            step()
            ev1[k].record(stream)
            st = plan.stats()  # stage events of this step (same stream)
            for k in hot:
                stage_hist[k].append(st["stage_ms"][k])
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    launches = fmm.kernel_launches() - launches0
    barrier(world)
    if args.profile:
        plan.close()
        return
    for k in range(args.steps):
        step_ms.append(ev0[k].elapsed_time(ev1[k]))
    t_steps = sum(step_ms) / 1e3
    t_max = max_over_ranks(t_steps, world, dev)
    value = N * world * args.steps / t_max

    # end to end through the public API with host buffers: H2D of the step's
    # inputs from pinned memory, the step, D2H of its results into pinned
    # memory, all inside the timed region, and the host waits for the results
    # at the end of every step (as a host-side integrator must)
    hx, hp, hq = (torch.as_tensor(a).pin_memory() for a in (x, p, q))
    hwE, hwB = torch.as_tensor(wE, dtype=out_dt).pin_memory(), torch.as_tensor(wB, dtype=out_dt).pin_memory()
    outs = None
    h2d = (hx.numel() + hp.numel() + hq.numel()) * 8 + ((hwE.numel() + hwB.numel()) * hwE.element_size() if adj else 0)
    e2e_ms = []
    for k in range(max(args.warmup, 3) + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Xd, Pd, Qd = hx.to(dev, non_blocking=True), hp.to(dev, non_blocking=True), hq.to(dev, non_blocking=True)
        E, B = plan.field(Xd, Pd, Qd)
        res = [E, B]
        if adj:
            WEd, WBd = hwE.to(dev, non_blocking=True), hwB.to(dev, non_blocking=True)
            res = list(plan.adjoint(Xd, Pd, Qd, WEd, WBd)) + res
        if outs is None:
            outs = [torch.empty(r.shape, dtype=r.dtype, pin_memory=True) for r in res]
        for o, r in zip(outs, res):
            o.copy_(r, non_blocking=True)
        torch.cuda.synchronize()
        if k >= max(args.warmup, 3):
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    d2h = sum(o.numel() * o.element_size() for o in outs)
    e2e_t = max_over_ranks(sum(e2e_ms) / 1e3, world, dev)
    e2e_value = N * world * args.steps / e2e_t

    # accuracy of this configuration against the FP64 brute force on sampled targets
    tg = torch.as_tensor(sample_targets(N, 4096), device=dev)
    E, B = plan.field(X, Pm, Q)
    st = plan.stats()
    Ed, Bd = fmm.direct_field(X, Pm, Q, gbar=st["gbar"], targets=tg)

    def rel(a, b):
        return float(torch.linalg.norm(a.double() - b) / torch.linalg.norm(b))

    err = max(rel(E[tg], Ed), rel(B[tg], Bd))

    side = {}
    if rank == 0 and not args.no_fp64_side and args.precision == "fp32":
        p64 = fmm.Plan(N, w.n, w.leaf, w.eta, precision="fp64", flags=sa_flag)
        for _ in range(2):
            p64.field(X, Pm, Q)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 3
        a.record(stream)
        for _ in range(reps):
            E64, B64 = p64.field(X, Pm, Q)
        b.record(stream)
        torch.cuda.synchronize()
        t64 = a.elapsed_time(b) / 1e3 / reps
        err64 = max(rel(E64[tg], Ed), rel(B64[tg], Bd))
        side = {"fp64_fwd_particles_per_s": N / t64, "fp64_fwd_err": err64, "fp32_fwd_err": err}
        p64.close()

    # roofline of the dominant kernel, ALU bound: FP32 SIMT peak
    # = SMs x 128 lanes x 2 flop x SM clock (median sampled under load)
    clocks = clk.summary()
    mhz = clocks["sm_mhz"] or 2070.0
    peak = SMS * FP32_LANES * 2 * mhz * 1e6 / 1e12 if args.precision == "fp32" else None
    kernels = {}
    for k, (per, unit) in hot.items():
        ms = statistics.median(stage_hist[k]) if stage_hist[k] else 0.0
        if ms <= 0.0:
            continue
        flop = per * st0[unit]
        traffic = (TRAFFIC_CYL64K.get(k) if args.workload == "cylinder64k" and args.precision == "fp32" and not args.size_aware
                   and not args.gbar_term and args.passes == "fwd+adj" else None)
        kernels[k] = {"ms": ms, "tflops": flop / (ms / 1e3) / 1e12,
                      "frac": (flop / (ms / 1e3) / 1e12 / peak) if peak else None, "traffic": traffic}
    # the adjoint runs its target side and M2L^T on two streams at once: their
    # stage times are shared-GPU times, so the dominant kernel is chosen among
    # the stages that have the GPU to themselves
    conc = set(CONCURRENT) | (set(CONCURRENT_FP32_FWD) if args.precision == "fp32" else set())
    for k in conc:
        if k in kernels:
            kernels[k]["concurrent"] = True
    # the longest stage that has the GPU to itself, else (every hot stage
    # overlapping another) the longest stage, measured while sharing the GPU
    alone = [k for k in kernels if k not in conc]
    dom = max(alone or list(kernels), key=lambda k: kernels[k]["ms"])
    roof = {"kernel": dom, "bound": "alu", "achieved": kernels[dom]["tflops"], "peak": peak, "unit": "TFLOP/s",
            "frac": kernels[dom]["frac"], "traffic": kernels[dom]["traffic"],
            "concurrent": kernels[dom].get("concurrent", False),
            "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
            "peak_basis": f"{SMS} SMs x {FP32_LANES} FP32 lanes x 2 x {mhz:.0f} MHz (median sampled SM clock)",
            "flop_basis": "algorithmic flop per pair (FMA = 2): M2L and M2L^T 32 per point pair, P2P 32, "
                          "adjoint near field 84 per particle pair for both roles in one kernel (FP32), "
                          "else 46 (target side) and 67 (source side)",
            "kernels": kernels}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64",
            "data": "synthetic (seeded beam generator)",
            "config": {"workload": args.workload, "N": N, "degree": w.n, "leaf": w.leaf, "eta": w.eta,
                       "passes": args.passes, "precision": args.precision, "replicas": world,
                       "lists": "size-aware (M2L -> P2P below m^2 pairs)" if args.size_aware else "paper (Alg. 17)",
                       "adjoint_gbar": "gbar(p) live" if args.gbar_term else "gbar held fixed",
                       "l2": "flushed before every timed step (512 MiB write)", "note": w.note},
            "rel_l2_error_vs_fp64_direct": err, "error_targets": 4096,
            "stage_ms": {k: round(v, 4) for k, v in st0["stage_ms"].items() if v},
            "lists": {"p2p_pairs": st0["p2p_pairs"], "m2l_pairs": st0["m2l_pairs"], "kappa": st0["kappa"]},
            "wall_ms_per_step": 1e3 * t_wall / args.steps,
            "e2e": {"value": e2e_value, "unit": "particles/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches, "launches_per_step": launches / args.steps,
            "roofline": roof, "clocks": clocks, **side,
        }
        if world == 1:
            line["cpu_baseline"] = cpu_baseline(args.workload, adj)
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _oracle_step(x, p, q, wE, wB, w, adj):
    from oracle import bldtt, gradient
    plan = bldtt.build_plan(x, p, w.n, w.leaf, w.eta)
    if adj:
        gradient.fmm_gradient(x, p, q, wE, wB, plan)
    else:
        bldtt.fmm_fields(x, p, q, w.n, w.leaf, w.eta, plan=plan)


def cpu_baseline(workload: str, adj: bool, budget_s: float = 12.0):
    """The oracle, as it stands, on a bounded sample of the workload on the host cores."""
    import torch
    torch.set_num_threads(os.cpu_count() or 1)
    w = WORKLOADS[workload]
    Ns = min(w.N, 16384)
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
    for n = 4, N0 = 125, eta = 0.5.  Section 11 (Fig. 7): N = 2.56e7 with the same
    parameters.  Times are CUDA-event medians of the whole fmm_field call (inputs in HBM);
    errors are max over E, B of the relative L2 error on 4096 sampled targets against the
    FP64 brute force.  One JSON line per point.
    """
    import torch

    from paper_2302_07567_gb300 import fmm

    dev = torch.device("cuda", 0)

    def point(N, n, N0, eta, prec, reps=3, err=True, exp=""):
        x, p, q = make_beam("cube", N=N)
        X, Pm, Q = (torch.as_tensor(a, device=dev) for a in (x, p, q))
        plan = fmm.Plan(N, n, N0, eta, precision=prec)
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

    for eta in (0.3, 0.4, 0.5):
        for n in (2, 4, 6, 8, 10):
            point(1_280_000, n, (n + 1) ** 3, eta, "fp32", exp="fig2")
    for eta in (0.5,):
        for n in (2, 4, 6):
            point(1_280_000, n, (n + 1) ** 3, eta, "fp64", exp="fig2")
    for N in (10_000, 20_000, 50_000, 100_000, 200_000, 500_000, 1_000_000, 2_000_000, 4_000_000, 8_000_000,
              16_000_000):
        point(N, 4, 125, 0.5, "fp32", err=False, exp="fig3")
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
