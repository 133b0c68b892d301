#!/usr/bin/env python
"""sFMM benchmark: Mpts/s of a full potential + deflection solve on GB300.

Workload (default): N = M = 1.6e7, sources and targets drawn independently from
one clustered sky (20,000 shared NFW clumps, 70 % clustered, 30 % uniform),
float64 positions, float32 equal masses.  One step = one complete
sfmm_deflection (keys, sort, tree, up-pass, lists, M2L, L2L, L2P + near field)
with inputs resident in HBM; value = M / step time.  Inputs (384 MB of
positions each) are larger than L2, so no flush is needed between steps.

Also reported: e2e through the host-array entry point (host<->device copies
inside the timed region), the roofline of the dominant kernel (the evaluation
kernel: near field + L2P), the oracle timed on the host cores on a bounded
sample of targets, the relative error against the oracle on a seeded sample,
and the SM clocks during the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl sfmm|reference]

Under torchrun (N > 1) every rank solves its own independent sky (weak
scaling; the path has no exchange step between independent problems).
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sFMM Mpts/s (N=M=1.6e7) FP64 vs mixed precision, at stated relative error"
# (path name, precision enum value, order p, stated relative error, leaf size m, c_s, c_t).
# mixed (1e-6): the setting that holds 1e-6 on every sky of the tests (uniform sky at its own
#   points, clustered sky on the N_side 512 grid, largest shell on N_side 256), not only on this one
#   (p = 16 suffices here: 2.8e-7);
# mixed_df and fp64 (1e-10): the fastest settings within half the stated error on this workload
#   (tune.autotune over the default candidate grids: errors 2.2e-11 and 3.0e-11);
# fp32 (3e-5): the all-FP32 path with tensor-core M2L.
MODES = [("mixed", 1, 20, 1e-6, 96, 1.5, 0.5), ("mixed_df", 2, 28, 1e-10, 64, 1.6, 0.45),
         ("fp64", 0, 32, 1e-10, 32, 1.5, 0.45), ("fp32", 3, 20, 3e-5, 64, 1.3, 0.5)]
# the FP64 reference every path is compared with on all M targets: error ~3e-13 on this workload
REF_SETTINGS = dict(p=32, leaf_size=32, c_s=2.0, c_t=0.45)
# operations per near-field pair of the unit of the roofline: d^2 (3 sub, 3 mul, 2 add), the
# alpha accumulation (q/d^2 times 3 components, 3 adds) and sum q: 12 flop, plus one reciprocal
# and one logarithm (psi): 14 operations
OPS_PER_PAIR = 14
MUFU_PER_PAIR = 2           # rcp and lg2 (the FP32 pair loop's special-function operations)
DTYPES = {"mixed": "f32+f32x2", "mixed_df": "f32x2+f64", "fp64": "f64", "fp32": "f32+bf16"}
EVAL_KERNEL = {"mixed": "k_eval32 (FP32 near field; its double-float L2P and combination are k_finish_dfar)",
               "mixed_df": "k_eval_df (near field and L2P in double-float)",
               "fp64": "k_eval (near field and L2P in FP64)",
               "fp32": "k_eval32 (near field and L2P in FP32)"}
# DRAM bytes of one k_eval32 launch of the headline path (p = 20, m = 96, c_s = 1.5 at N = M = 1.6e7):
# ncu at N = M = 2e6 (profiles/k_eval32_mixed_clustered_2e6.md), scaled by the near-field pairs
K_EVAL32_TRAFFIC = (225.2e6 + 55.6e6) * (1.3399e10 / 1.1019e9)
K_EVAL32_TRAFFIC_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one k_eval32 launch at N = M = 2e6 "
                           "(225.2 + 55.6 MB, 1.10e9 pairs), scaled by the near-field pairs to this launch (x 12.16)")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sfmm", choices=["sfmm", "reference"])
    ap.add_argument("--n", type=int, default=16_000_000, help="N = M")
    ap.add_argument("--clumps", type=int, default=20_000)
    ap.add_argument("--modes", default="mixed,mixed_df,fp64,fp32", help="paths to run; the first is the headline value")
    ap.add_argument("--leaf", type=int, default=0, help="leaf size m for every path (0 = each path's own)")
    ap.add_argument("--check", type=int, default=1000,
                    help="oracle targets per stratum (near clump, empty sky) for the error check and CPU baseline")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the oracle CPU baseline (extra legs)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--shells", action="store_true",
                    help="also time the batched-shell workload (64 shells, 9.3e7 sources; slow to generate)")
    ap.add_argument("--no-adjoint", action="store_true",
                    help="skip the gradient, shear and Near Particle Model measurements")
    ap.add_argument("--solve-only", action="store_true",
                    help="time the chosen paths only (no reference solve, oracle, e2e or extra legs): "
                         "the driver of the ncu captures under profiles/")
    return ap.parse_args()


def dist_env():
    from paper_2210_07021_gb300.shard import dist_env as env
    return env()


class ClockSampler:
    """nvidia-smi samples (every 50 ms) of SM clock and throttle reasons during a
    region: the sampler is running (its first line written) before the region
    opens, and only samples stamped inside the region are summarised (if none
    are, the one nearest to the region is reported with in_region false).  The
    GPU is selected by the UUID of the CUDA device (CUDA ordinals and nvidia-smi
    indices differ under CUDA_VISIBLE_DEVICES); every sample's UUID is checked."""
    Q = ("timestamp,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, cuda_device, uuid=None):
        self.uuid = uuid or device_uuid(cuda_device)
        self.proc = None
        self.f = None
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", self.uuid, "-lms", "50"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
            deadline = time.time() + 5.0
            while time.time() < deadline and os.path.getsize(self.f.name) == 0:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        self.t0 = time.time()
        return self

    def __exit__(self, *a):
        self.t1 = time.time()
        if self.proc:
            time.sleep(0.06)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.f:
            return None
        try:
            rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
            os.unlink(self.f.name)
        except Exception:
            return None
        import datetime
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        parsed = []
        uuid_ok = True
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(r[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                uuid_ok &= r[1] == self.uuid
                parsed.append((ts, float(r[2]), float(r[3]), [n for n, v in zip(names, r[6:10]) if v.lower() == "active"]))
            except ValueError:
                continue
        if not parsed:
            return None
        inside = [x for x in parsed if self.t0 - 0.01 <= x[0] <= self.t1 + 0.01]
        in_region = bool(inside)
        if not inside:
            mid = 0.5 * (self.t0 + self.t1)
            inside = [min(parsed, key=lambda x: abs(x[0] - mid))]
        reasons = sorted({n for x in inside for n in x[3]})
        return {"sm_mhz": float(np.median([x[1] for x in inside])), "sm_max_mhz": inside[-1][2], "reasons": reasons,
                "samples": len(inside), "in_region": in_region, "gpu_uuid": self.uuid, "uuid_matches": uuid_ok}


def device_uuid(cuda_device):
    """nvidia-smi's UUID string ("GPU-...") of a CUDA device ordinal."""
    import torch
    u = str(torch.cuda.get_device_properties(cuda_device).uuid)
    return u if u.startswith("GPU-") else "GPU-" + u


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def make_workload(args, rank):
    from paper_2210_07021_gb300 import workloads
    from paper_2210_07021_gb300.shard import rank_config_index
    d = workloads.clustered_pair(n=args.n, n_clumps=args.clumps, config_index=rank_config_index(3, rank))
    return d


def run_adjoint(args, dev, clock_sampler):
    """One training step of the gradient workload: the 1e-10 forward solve, the
    loss gradient dL/dalpha = 2 w (alpha - alpha_ref) on the device, and the
    double-float adjoint sFMM (dL/dq, dL/dy); CUDA events around each part."""
    import torch
    from paper_2210_07021_gb300 import sfmm, workloads
    d = workloads.loss_sky()
    N, M = d["src"].shape[0], d["tgt"].shape[0]
    src = torch.as_tensor(d["src"], device=dev)
    q = torch.as_tensor(d["q"], device=dev)
    tgt = torch.as_tensor(d["tgt"], device=dev)
    w = torch.as_tensor(d["w"], device=dev)
    plan = sfmm.Plan(p=28, leaf_size=64, c_s=2.0, c_t=0.45, precision=sfmm.SFMM_MIXED_DF, n_max=max(N, M), m_max=max(N, M))
    psi, alpha = plan.deflection(src, q, tgt)
    s = float(torch.sqrt((alpha ** 2).mean()))
    a_ref = s * torch.as_tensor(d["xi"], device=dev)

    def step():
        _, al = plan.deflection(src, q, tgt, with_psi=False)
        ev_mid.record(torch.cuda.current_stream())
        g_alpha = (2.0 * w[:, None] * (al - a_ref)).contiguous()
        gq, gs = plan.adjoint(src, q, tgt, g_alpha=g_alpha)
        return g_alpha, gq, gs

    ev_mid = torch.cuda.Event(enable_timing=True)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    t_f, t_b = [], []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with clock_sampler as clk:
        for _ in range(args.steps):
            ev0.record(torch.cuda.current_stream())
            g_alpha, gq, gs = step()
            ev1.record(torch.cuda.current_stream())
            torch.cuda.synchronize()
            t_f.append(ev0.elapsed_time(ev_mid))
            t_b.append(ev_mid.elapsed_time(ev1))
    from oracle.direct import adjoint as oracle_adjoint
    idx = workloads.subsample(N, args.check, 5, stream=9)
    rq, rs = oracle_adjoint(d["src"][idx], d["q"][idx], d["tgt"], g_alpha.cpu().numpy(), None)
    plan.close()
    ms = float(np.mean(t_f) + np.mean(t_b))
    return {"workload": d["workload"], "N": N, "M": M, "forward": "mixed_df (stated 1e-10), p=28, m=64, c_t=0.45",
            "backward": "adjoint sFMM, double-float (charges and dipoles), same p and tree settings",
            "backward_over_forward": float(np.mean(t_b) / np.mean(t_f)), "steps": args.steps,
            "ms_per_step": ms, "ms_forward": float(np.mean(t_f)), "ms_backward": float(np.mean(t_b)),
            "value": (N + M) * 1e-3 / ms, "unit": "Mpts/s (sources + targets per forward+backward step)",
            "error_vs_oracle": {"dq_rel": rel(gq.cpu().numpy()[idx], rq), "dy_rel": rel(gs.cpu().numpy()[idx], rs),
                                "sample": int(idx.size), "norm": "l2 over the sampled sources (relative)"},
            "clocks": clk.summary()}


def run_shear(args, dev, clock_sampler):
    """Shear (gamma_1, gamma_2) and magnification on the gradient workload's sky,
    FP64 path at p = 32; error vs the oracle's Hessian on a target sample."""
    import torch
    from paper_2210_07021_gb300 import sfmm, workloads
    d = workloads.loss_sky()
    N, M = d["src"].shape[0], d["tgt"].shape[0]
    src = torch.as_tensor(d["src"], device=dev)
    q = torch.as_tensor(d["q"], device=dev)
    tgt = torch.as_tensor(d["tgt"], device=dev)
    plan = sfmm.Plan(p=32, leaf_size=64, c_t=0.45, n_max=N, m_max=M)
    for _ in range(args.warmup):
        g, _, _, mu = plan.shear(src, q, tgt, with_mu=True)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with clock_sampler as clk:
        ev0.record(torch.cuda.current_stream())
        for _ in range(args.steps):
            g, _, _, mu = plan.shear(src, q, tgt, with_mu=True)
        ev1.record(torch.cuda.current_stream())
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    from oracle.direct import lensing
    idx = workloads.subsample(M, args.check, 6, stream=9)
    ref = lensing(d["src"], d["q"], d["tgt"][idx])
    plan.close()
    return {"workload": d["workload"].split(", loss")[0], "N": N, "M": M, "path": "FP64, p=32, m=64, c_t=0.45",
            "ms_per_step": ms, "value": M * 1e-3 / ms, "unit": "Mpts/s (targets per shear solve)",
            "error_vs_oracle": {"gamma_rel": rel(g.cpu().numpy()[idx], ref["gamma"]),
                                "mu_rel": rel(mu.cpu().numpy()[idx], ref["mu"]), "sample": int(idx.size),
                                "stated": 1e-9},
            "clocks": clk.summary()}


def run_npm(args, dev, clock_sampler):
    """Near Particle Model solve (sigma = sqrt(4 pi / N), the paper's choice) on
    the gradient workload's sky, FP64 path at p = 32; error vs the oracle's
    NPM sum on a target sample."""
    import torch
    from paper_2210_07021_gb300 import sfmm, workloads
    d = workloads.loss_sky()
    N, M = d["src"].shape[0], d["tgt"].shape[0]
    sigma = float(np.sqrt(4 * np.pi / N))
    src = torch.as_tensor(d["src"], device=dev)
    q = torch.as_tensor(d["q"], device=dev)
    tgt = torch.as_tensor(d["tgt"], device=dev)
    plan = sfmm.Plan(p=32, leaf_size=64, c_t=0.45, sigma=sigma, n_max=N, m_max=M)
    for _ in range(args.warmup):
        psi, alpha = plan.deflection(src, q, tgt)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with clock_sampler as clk:
        ev0.record(torch.cuda.current_stream())
        for _ in range(args.steps):
            psi, alpha = plan.deflection(src, q, tgt)
        ev1.record(torch.cuda.current_stream())
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    from oracle.direct import direct_sum
    idx = workloads.subsample(M, args.check, 7, stream=9)
    ref = direct_sum(d["src"], d["q"], d["tgt"][idx], sigma=sigma)
    plan.close()
    return {"workload": d["workload"].split(", loss")[0], "N": N, "M": M, "sigma": sigma,
            "path": "FP64, p=32, m=64, c_t=0.45, NPM near field", "ms_per_step": ms, "value": M * 1e-3 / ms,
            "unit": "Mpts/s (targets per solve)",
            "error_vs_oracle": {"psi_rel": rel(psi.cpu().numpy()[idx], ref["psi"]),
                                "alpha_rel": rel(alpha.cpu().numpy()[idx], ref["alpha"]), "sample": int(idx.size)},
            "clocks": clk.summary()}


def run_shells(args, dev, clock_sampler, ws=1, rank=0):
    """Batched shells: the 64-shell set split over the ranks by the longest-first
    rule (shard.assign_shells; every rank builds and solves only its shells),
    each rank's shells solved per step with 4 concurrent lanes and with 1, for
    the 1e-6 and 1e-10 paths; the whole job's targets over the slowest rank's
    time; error of rank 0's largest shell vs the oracle on a target sample."""
    import torch
    from paper_2210_07021_gb300 import sfmm, shard, workloads
    sizes = workloads.shell_sizes()
    tgt_h = workloads.healpix_ring_centres(256)
    M = tgt_h.shape[0]
    mine = shard.assign_shells([shard.shell_cost(n, M) for n in sizes], ws)[rank]
    tgt = torch.as_tensor(tgt_h, device=dev)
    host = {k: workloads.shell(k, sizes[k]) for k in mine}
    sh = [(torch.as_tensor(host[k][0], device=dev), torch.as_tensor(host[k][1], device=dev), tgt) for k in mine]
    out = {"workload": f"{len(sizes)} shells, N_k log-uniform in [1e4, 1e7] (sum {int(sizes.sum())}), clustered "
                       f"(N_k/500 clumps), M = {M} N_side=256 pixel centres each",
           "n_shells": len(sizes), "sum_N": int(sizes.sum()), "M_per_shell": M, "ranks": ws,
           "shells_per_rank_0": len(mine), "split": "longest-first greedy on N_k + M (shard.assign_shells)"}
    from oracle.direct import direct_sum
    big = mine[int(np.argmax([sizes[k] for k in mine]))] if mine else None
    idx = workloads.subsample(M, min(args.check, 100), 8, stream=9)
    for name, prec, kw in (("mixed", sfmm.SFMM_MIXED, dict(p=20, leaf_size=96, c_s=1.5, c_t=0.5)),
                           ("mixed_df", sfmm.SFMM_MIXED_DF, dict(p=28, leaf_size=64, c_s=1.6, c_t=0.45))):
        plan = sfmm.Plan(precision=prec, **kw)
        for lanes in (4, 1):
            outs = plan.deflection_batch(sh, with_psi=False, lanes=lanes) if sh else []
            torch.cuda.synchronize()
            if ws > 1:
                import torch.distributed as dist
                dist.barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with clock_sampler as clk:
                e0.record(torch.cuda.current_stream())
                for _ in range(args.steps):
                    outs = plan.deflection_batch(sh, with_psi=False, lanes=lanes) if sh else []
                e1.record(torch.cuda.current_stream())
                torch.cuda.synchronize()
            ms = shard.max_over_ranks(e0.elapsed_time(e1) / args.steps, device=dev)
            out[f"{name}_lanes{lanes}"] = {"ms_per_step": ms, "value": len(sizes) * M * 1e-3 / ms,
                                           "unit": "Mpts/s (targets of all shells per step, whole job)",
                                           "clocks": clk.summary()}
        plan.close()
        # the same shells replayed as one CUDA graph (sfmm_graph_capture / sfmm_graph_launch):
        # no host synchronisation inside; one for the whole batch after each replay
        gouts, graph = [], None
        if sh:
            gplan = sfmm.Plan(precision=prec, **kw)
            gouts = gplan.graph_capture(sh, with_psi=False)
            for _ in range(max(1, args.warmup)):
                gplan.graph_launch()
            if ws > 1:
                import torch.distributed as dist
                dist.barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with clock_sampler as clk:
                for _ in range(args.steps):
                    gplan.graph_launch()
            ms_g = 1e3 * (time.perf_counter() - t0) / args.steps
            info = gplan.graph_info()
            agree = max(float((g[1] - l[1]).abs().max() / l[1].abs().max()) for g, l in zip(gouts, outs))
            graph = {"ms_per_step": ms_g, "kernel_nodes": info["kernel_nodes"], "overflows": info["overflows"],
                     "recaptures": info["recaptures"], "max_rel_diff_vs_lanes": agree,
                     "timing": "host clock around synchronous replays (each replay waits for its graph)",
                     "clocks": clk.summary()}
        ms_g = shard.max_over_ranks(graph["ms_per_step"] if graph else 0.0, device=dev)
        out[f"{name}_graph"] = dict(graph or {}, ms_per_step=ms_g, value=len(sizes) * M * 1e-3 / ms_g,
                                    unit="Mpts/s (targets of all shells per step, whole job)",
                                    speedup_vs_lanes4=out[f"{name}_lanes4"]["ms_per_step"] / ms_g)
        if rank == 0 and big is not None:
            ref = direct_sum(host[big][0], host[big][1], tgt_h[idx])
            err = rel(outs[mine.index(big)][1].cpu().numpy()[idx], ref["alpha"])
            err_g = rel(gouts[mine.index(big)][1].cpu().numpy()[idx], ref["alpha"])
            stated = 1e-6 if prec == sfmm.SFMM_MIXED else 1e-10
            out[f"{name}_error_vs_oracle"] = {"alpha_rel": err, "alpha_rel_graph": err_g, "shell": int(big),
                                              "sample": int(idx.size), "stated": stated,
                                              "within_stated": bool(max(err, err_g) < stated)}
        if sh:
            gplan.close()
    return out


def run_reference(args):
    ws, rank, local = dist_env()
    if ws > 1 and rank != 0:
        return
    d = make_workload(args, 0)
    from oracle.direct import direct_sum, threads
    from paper_2210_07021_gb300 import workloads
    src, q, tgt = d["src"], d["q"].astype(np.float64), d["tgt"]
    n_probe = 2 * threads()
    probe = workloads.subsample(tgt.shape[0], n_probe, 3, stream=11)
    t0 = time.perf_counter()
    direct_sum(src, q, tgt[probe])
    t_probe = max(time.perf_counter() - t0, 1e-3)
    per_step_s = min(20.0, 150.0 / max(1, args.steps + args.warmup))
    k = int(max(n_probe, min(tgt.shape[0], n_probe * per_step_s / t_probe)))
    for w in range(args.warmup):
        direct_sum(src, q, tgt[workloads.subsample(tgt.shape[0], k, 3, stream=20 + w)])
    t0 = time.perf_counter()
    for s in range(args.steps):
        direct_sum(src, q, tgt[workloads.subsample(tgt.shape[0], k, 3, stream=40 + s)])
    t = time.perf_counter() - t0
    value = args.steps * k / t / 1e6
    line = {"metric": METRIC, "value": value, "unit": "Mpts/s", "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": d["workload"], "N": int(src.shape[0]), "M": int(tgt.shape[0]),
                       "parallelism": "host cores (OpenMP)"},
            "cpu_baseline": {"value": value, "unit": "Mpts/s", "cores": threads(), "kind": "oracle",
                             "sample": f"{k} seeded targets per step against all {src.shape[0]} sources "
                                       f"(FP64 direct sum, Neumaier sums)"},
            "e2e": {"value": value, "unit": "Mpts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def errors(psi, alpha, ref_psi, ref_alpha):
    """Norm-wise relative errors of psi and alpha, and the largest pointwise
    deflection error relative to the largest deflection (numpy or torch)."""
    if hasattr(psi, "cpu"):
        import torch
        e_psi = float(torch.linalg.norm(psi - ref_psi) / torch.linalg.norm(ref_psi))
        e_al = float(torch.linalg.norm(alpha - ref_alpha) / torch.linalg.norm(ref_alpha))
        e_max = float((alpha - ref_alpha).norm(dim=1).max() / ref_alpha.norm(dim=1).max())
    else:
        e_psi, e_al = rel(psi, ref_psi), rel(alpha, ref_alpha)
        e_max = float(np.linalg.norm(alpha - ref_alpha, axis=1).max() / np.linalg.norm(ref_alpha, axis=1).max())
    return {"psi_rel": e_psi, "alpha_rel": e_al, "alpha_max_rel": e_max}


def run_solve_only(args):
    """W untimed and K timed solves of each chosen path on the benchmark sky (or
    --n), printing one JSON line of times and solver statistics."""
    import torch
    from paper_2210_07021_gb300 import sfmm, workloads
    torch.cuda.set_device(0)
    d = workloads.clustered_pair(n=args.n, n_clumps=args.clumps)
    N, M = d["src"].shape[0], d["tgt"].shape[0]
    src, q, tgt = (torch.as_tensor(d[k], device="cuda") for k in ("src", "q", "tgt"))
    out = {"workload": d["workload"], "steps": args.steps, "warmup": args.warmup, "paths": {}}
    for name, prec, p, stated, leaf, c_s, c_t in [m for m in MODES if m[0] in args.modes.split(",")]:
        plan = sfmm.Plan(p=p, leaf_size=args.leaf or leaf, c_s=c_s, c_t=c_t, precision=prec, q_f32=True,
                         n_max=N, m_max=M)
        for _ in range(args.warmup):
            plan.deflection(src, q, tgt)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            plan.deflection(src, q, tgt)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / max(args.steps, 1)
        plan.set_timing(2)                    # one more solve: phase times and the near-field pair count
        plan.deflection(src, q, tgt)
        out["paths"][name] = {"ms_per_step": ms, "stats": plan.stats()}
        plan.close()
    print(json.dumps(out), flush=True)


def run_sfmm(args):
    import torch
    from paper_2210_07021_gb300 import sfmm, workloads

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    d = make_workload(args, rank)
    N, M = d["src"].shape[0], d["tgt"].shape[0]
    src = torch.as_tensor(d["src"], device=dev)
    q = torch.as_tensor(d["q"], device=dev)
    tgt = torch.as_tensor(d["tgt"], device=dev)
    psi = torch.empty(M, dtype=torch.float64, device=dev)
    alpha = torch.empty((M, 2), dtype=torch.float64, device=dev)

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(v):
        from paper_2210_07021_gb300.shard import max_over_ranks as mor
        return mor(v, device=dev)

    # measured arithmetic rates of this GPU: the rooflines' denominators
    peaks = {k: sfmm.peak_rate(w) for k, w in (("fp32", sfmm.PEAK_FP32), ("fp32x2", sfmm.PEAK_FP32X2),
                                               ("fp64", sfmm.PEAK_FP64), ("mufu", sfmm.PEAK_MUFU))}
    # the FP64 reference on every target (untimed)
    ref_plan = sfmm.Plan(precision=sfmm.SFMM_FP64, q_f32=True, n_max=N, m_max=M, **REF_SETTINGS)
    ref_psi, ref_alpha = ref_plan.deflection(src, q, tgt)
    ref_plan.close()
    # oracle targets: seeded samples near clumps and in empty sky (rank 0)
    strata = None
    if rank == 0:
        near, empty = workloads.clump_strata(d["tgt"], d["clumps"], args.check, 3)
        strata = {"near_clump": near, "empty_sky": empty}

    wanted = [m for m in MODES if m[0] in args.modes.split(",")]
    wanted.sort(key=lambda m: args.modes.split(",").index(m[0]))
    results, outputs = {}, {}
    for name, prec, p, stated, leaf, c_s, c_t in wanted:
        leaf = args.leaf or leaf
        plan = sfmm.Plan(p=p, leaf_size=leaf, c_s=c_s, c_t=c_t, precision=prec, q_f32=True, n_max=N, m_max=M)
        for _ in range(args.warmup):
            plan.deflection(src, q, tgt, psi=psi, alpha=alpha)
        # the near-field pair count (one more kernel) from an untimed solve; the
        # timed steps record phase times only
        plan.set_timing(2)
        plan.deflection(src, q, tgt, psi=psi, alpha=alpha)
        n_pairs = plan.stats()["p2p_interactions"]
        plan.set_timing(1)
        stream = torch.cuda.current_stream()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        eval_ms, launches, phase = [], 0, np.zeros(8)
        barrier()
        with ClockSampler(local) as clk:
            ev0.record(stream)
            for _ in range(args.steps):
                plan.deflection(src, q, tgt, psi=psi, alpha=alpha)
                st = plan.stats()
                # the near-field kernel's own time (the 1e-6 path runs it beside M2L and L2L),
                # else the evaluation phase
                eval_ms.append(st["near_ms"] if st["near_ms"] > 0 else st["ms"][6])
                launches += st["launches"]
                phase += np.array(st["ms"])
            ev1.record(stream)
            barrier()
        elapsed_ms = max_over_ranks(ev0.elapsed_time(ev1))
        plan.set_timing(False)
        r = {"precision": name, "p": p, "stated_error": stated, "leaf_size": leaf, "c_s": c_s, "c_t": c_t,
             "value": M * args.steps * ws / (elapsed_ms / 1e3) / 1e6, "ms_per_step": elapsed_ms / args.steps,
             "gpu_launches": int(launches), "eval_ms": float(np.mean(eval_ms)), "pairs": float(n_pairs),
             "phase_ms": {k: v / args.steps for k, v in zip(
                 ["keys_sort", "tree_geometry", "up_pass", "lists", "m2l", "l2l", "evaluation", "total"], phase)},
             "clocks": clk.summary(),
             "error_vs_fp64_all_M": dict(errors(psi, alpha, ref_psi, ref_alpha), targets=M,
                                         reference="FP64 sFMM, p=32, m=32, c_s=2, c_t=0.45")}
        if rank == 0:
            idx = np.concatenate([strata["near_clump"], strata["empty_sky"]])
            outputs[name] = (psi.cpu().numpy()[idx], alpha.cpu().numpy()[idx])
        # end to end through the host-array entry point (headline path only)
        if not args.no_e2e and name == wanted[0][0]:
            hs = torch.empty((N, 3), dtype=torch.float64, pin_memory=True).numpy()
            hq = torch.empty(N, dtype=torch.float32, pin_memory=True).numpy()
            ht = torch.empty((M, 3), dtype=torch.float64, pin_memory=True).numpy()
            hpsi = torch.empty(M, dtype=torch.float64, pin_memory=True).numpy()
            halpha = torch.empty((M, 2), dtype=torch.float64, pin_memory=True).numpy()
            hs[:] = d["src"]
            hq[:] = d["q"]
            ht[:] = d["tgt"]
            plan.deflection_host(hs, hq, ht, psi=hpsi, alpha=halpha)
            barrier()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                plan.deflection_host(hs, hq, ht, psi=hpsi, alpha=halpha)
            barrier()
            t_e2e = max_over_ranks(time.perf_counter() - t0)
            r["e2e"] = {"value": M * args.steps * ws / t_e2e / 1e6, "unit": "Mpts/s",
                        "h2d_bytes_per_step": int(N * 24 + N * 4 + M * 24), "d2h_bytes_per_step": int(M * 8 + M * 16)}
        results[name] = r
        plan.close()
    del ref_psi, ref_alpha
    shl = run_shells(args, dev, ClockSampler(local), ws, rank) if args.shells else None
    if rank != 0:
        if dist:
            dist.barrier()
        return
    # the oracle on the stratified targets: the error of every path per stratum, and
    # its own time on the host cores (the CPU baseline)
    from oracle.direct import direct_sum, threads
    idx = np.concatenate([strata["near_clump"], strata["empty_sky"]])
    t0 = time.perf_counter()
    ref = direct_sum(d["src"], d["q"].astype(np.float64), d["tgt"][idx])
    t_or = time.perf_counter() - t0
    n_near = strata["near_clump"].size
    cpu = {"value": idx.size / t_or / 1e6, "unit": "Mpts/s", "cores": threads(), "kind": "oracle",
           "sample": f"{idx.size} seeded targets ({n_near} near clumps, {idx.size - n_near} in empty sky) against "
                     f"all {N} sources, FP64 direct sum, {t_or:.1f} s"}
    for name, (ps, al) in outputs.items():
        ev = {"all": errors(ps, al, ref["psi"], ref["alpha"]),
              "near_clump": errors(ps[:n_near], al[:n_near], ref["psi"][:n_near], ref["alpha"][:n_near]),
              "empty_sky": errors(ps[n_near:], al[n_near:], ref["psi"][n_near:], ref["alpha"][n_near:])}
        ev["within_stated"] = bool(max(ev["all"]["psi_rel"], ev["all"]["alpha_rel"],
                                       ev["near_clump"]["alpha_rel"], ev["empty_sky"]["alpha_rel"])
                                   < results[name]["stated_error"])
        ev["targets"] = f"{n_near} near clumps + {idx.size - n_near} in empty sky (norm-wise relative errors)"
        results[name]["error_vs_oracle"] = ev
    head = results[wanted[0][0]]
    adj = shr = npm = None
    if ws == 1 and not args.no_adjoint:
        adj = run_adjoint(args, dev, ClockSampler(local))
        shr = run_shear(args, dev, ClockSampler(local))
        npm = run_npm(args, dev, ClockSampler(local))

    def roofline_of(r):
        fp64 = r["precision"] == "fp64"
        peak = peaks["fp64"] if fp64 else peaks["fp32"]
        secs = r["eval_ms"] / 1e3
        ach = r["pairs"] * OPS_PER_PAIR / secs
        out = {"bound": "alu", "kernel": EVAL_KERNEL[r["precision"]], "achieved": ach / 1e12, "peak": peak / 1e12,
               "unit": "TFLOP/s", "frac": ach / peak,
               "peak_source": ("measured in this run: sfmm_peak_rate, a loop of independent "
                               + ("FP64" if fp64 else "FP32") + " FMA chains on a full grid"),
               "work_per_unit": f"{OPS_PER_PAIR} operations per near-field pair (12 flop + 1 reciprocal + 1 log)",
               "pairs_per_launch": r["pairs"], "launch_ms": r["eval_ms"], "traffic": None}
        if not fp64:
            out["mufu_frac"] = r["pairs"] * MUFU_PER_PAIR / secs / peaks["mufu"]
        if (K_EVAL32_TRAFFIC is not None and r["precision"] == "mixed" and r["leaf_size"] == 96
                and r["c_s"] == 1.5 and N == 16_000_000 and M == 16_000_000 and args.clumps == 20_000):
            out["traffic"] = K_EVAL32_TRAFFIC
            out["traffic_source"] = K_EVAL32_TRAFFIC_SOURCE
        return out

    modes = {}
    for name, *_ in wanted:
        r = dict(results[name])
        r["roofline"] = roofline_of(r)
        modes[name] = r
    line = {"metric": METRIC, "value": head["value"], "unit": "Mpts/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPES[head["precision"]], "data": "synthetic",
            "config": {"workload": d["workload"], "N": N, "M": M, "precision": head["precision"], "p": head["p"],
                       "stated_error": head["stated_error"], "leaf_size": head["leaf_size"], "c_s": head["c_s"],
                       "c_t": head["c_t"],
                       "l2": "inputs larger than L2 (384 MB of positions each), no flush"},
            "error_vs_oracle": head.get("error_vs_oracle"), "error_vs_fp64_all_M": head["error_vs_fp64_all_M"],
            "roofline": modes[head["precision"]]["roofline"],
            "cpu_baseline": cpu, "e2e": head.get("e2e"), "gpu_launches": head["gpu_launches"],
            "phase_ms": head["phase_ms"], "clocks": head["clocks"],
            "peaks_measured": {k: v / 1e12 for k, v in peaks.items()},
            "peaks_unit": "TFLOP/s (FMA = 2 flop); mufu: Tops/s (rcp + lg2)",
            "adjoint": adj, "shear": shr, "npm": npm, "shells": shl,
            "modes": {k: {kk: vv for kk, vv in v.items()} for k, v in modes.items()}}
    if "fp64" in results:
        line["speedup_vs_fp64"] = {k: results[k]["value"] / results["fp64"]["value"] for k in results if k != "fp64"}
    print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.solve_only:
        run_solve_only(args)
    else:
        run_sfmm(args)


if __name__ == "__main__":
    main()
