"""Throughput benchmark of the fused axisymmetric MRT-LB step on GB300.

Workload (one GPU): the single large porous annulus, nr x nz = 4096 x 8192, R* = 2,
porosity = seeded uniform[0.3, 0.9] white noise smoothed by a Gaussian of sigma = 16
cells (seed 2), Da = 1e-4, Ra = 1e6, Pr = 0.71, Ergun drag, FP32 arithmetic; storage
FP32 by default (--storage f16 / bf16 for deviation storage).  A step is one pass
of the whole hot path over the domain: pull streaming, wall rebuild, recovery,
MRT + D2Q5 collision, store.  The state (3.8 GB in FP32) is far larger than L2,
so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank advances its own replica of the domain (no data
exchange; weak scaling); value = all ranks' node updates / max time over ranks.
--impl reference times the FP64 CPU oracle on the host cores on a bounded sample
of the same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NR, NZ = 4096, 8192
WORKLOAD = dict(nr=NR, nz=NZ, radius_ratio=2.0, Ra=1e6, Da=1e-4, Pr=0.71, F_eps=-1.0)
PHI_RECIPE = dict(lo=0.3, hi=0.9, sigma=16.0, seed=2)
METRIC = "MLUPS & % HBM roofline; time-to-steady vs plain FP32 GPU at |ΔNu|≤1e-3"
SAMPLE_NR, SAMPLE_NZ = 256, 512   # bounded CPU sample: the same recipe on a 256 x 512 annulus
E2E_STEPS = 50                    # minimum length of the end-to-end window (steps)


# DRAM traffic of one k_bulk launch on the 4096 x 8192 workload (dram__bytes_read.sum +
# dram__bytes_write.sum of the bulk kernel in one single-pass ncu capture of this
# benchmark), valid only for the bulk kernel's source it was taken on (_kernel_hash).
TRAFFIC = {("f32", 4096, 8192): ("e47fb4700593f444", 2089953280 + 1827634944),
           ("f16", 4096, 8192): ("e47fb4700593f444", 1690808064 + 1227835648),
           ("bf16", 4096, 8192): ("e47fb4700593f444", 1689640704 + 1228074496)}


def _kernel_hash() -> str:
    """Hash of the bulk kernels' own source: csrc/lbm_physics.cuh, csrc/lbm_pair.cuh and
    csrc/lbm.cu up to the end of the bulk kernels (where k_wall begins); host code and
    other kernels further down do not change the traffic record's validity."""
    import hashlib

    d = os.path.join(ROOT, "paper_1409_5929_gb300", "csrc")
    h = hashlib.sha256()
    h.update(open(os.path.join(d, "lbm_physics.cuh"), "rb").read())
    h.update(open(os.path.join(d, "lbm_pair.cuh"), "rb").read())
    src = open(os.path.join(d, "lbm.cu"), "rb").read()
    k = src.find(b"__global__ void k_wall(")
    cut = src.rfind(b"template <", 0, k) if k > 0 else -1
    h.update(src[:cut] if cut > 0 else src + b"(no k_wall marker)")
    return h.hexdigest()[:16]


def _traffic(storage: str):
    rec = TRAFFIC.get((storage, NR, NZ))
    return rec[1] if rec and rec[0] == _kernel_hash() else None


def _set_grid(nr: int, nz: int):
    global NR, NZ
    NR, NZ = nr, nz
    WORKLOAD.update(nr=nr, nz=nz)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _workload_name(storage):
    return (f"porous annulus {NR}x{NZ}, R*=2, phi~U[0.3,0.9] smoothed sigma=16 (seed 2), "
            f"Ra=1e6, Da=1e-4, Pr=0.71, Ergun drag, {storage} storage")


class Clocks:
    """nvidia-smi samples during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.05)
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            return None
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = max(mx, float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def aggregate(local_ms: float, local_units: float, device=None) -> tuple[float, float]:
    """Whole-job throughput of independent replicas: the units all ranks processed
    divided by the slowest rank's time (MAX over ranks).  Returns (units per second,
    max milliseconds).  Works with any initialised process group (NCCL or gloo)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([local_ms, local_units], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        tm = t[:1].clone()
        dist.all_reduce(tm, op=dist.ReduceOp.MAX)
        tu = t[1:].clone()
        dist.all_reduce(tu, op=dist.ReduceOp.SUM)
        ms, units = float(tm.item()), float(tu.item())
    else:
        ms, units = local_ms, local_units
    return units / (ms * 1e-3), ms


def _time_steps(lbm, s, stream, steps):
    """Device time of `steps` steps on the solver's stream (CUDA events around the loop and
    around every bulk and wall launch), with nvidia-smi clock samples taken meanwhile."""
    import torch

    torch.cuda.synchronize()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    lbm.lbm_set_timing(s.h, True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    s.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    bulk_ms, bulk_n, wall_ms, wall_n = lbm.lbm_kernel_times(s.h)
    lbm.lbm_set_timing(s.h, False)
    return ms, bulk_ms / max(bulk_n, 1), wall_ms / max(wall_n, 1), clocks.stop()


def _solver(lbm, storage, phi, stream, inplace=0):
    p = lbm.lbm_params_default(storage=storage, eps_mean=float(phi.mean(dtype=np.float64)), inplace=inplace,
                               **WORKLOAD)
    s = lbm.Solver(p)
    s.set_stream(stream.cuda_stream)
    s.set_porosity(phi)
    s.init_fields()
    return s


def _bulk_bytes(info):
    """Algorithmic bytes of one bulk launch: every non-wall node reads and writes its
    populations and reads its porosity (and the reference planes its storage type
    keeps); bytes per node as the library states them for the storage type."""
    return (NR - 2) * (NZ - 2) * (info.bytes_per_step // (NR * NZ))


def _bulk_kernel(storage: str, inplace: int) -> str:
    """The bulk kernel this workload launches: one node per thread for FP32 storage and in
    place, the staged two-column kernel for 16-bit storage on two buffers."""
    return f"k_bulk<{storage}>" if storage == "f32" or inplace else f"k_bulk_stage<{storage}>"


def storage_variant(lbm, storage, phi, steps, warmup, peak, inplace=0):
    """Single-domain line for another storage type (or in-place storage): MLUPS, the bulk
    kernel's roofline fraction on its own bytes per node, and each kernel's mean launch
    time."""
    import torch

    stream = torch.cuda.Stream()
    s = _solver(lbm, storage, phi, stream, inplace)
    s.step(warmup)
    ms, bulk_avg, wall_avg, ck = _time_steps(lbm, s, stream, steps)
    info = s.info()
    s.close()
    achieved = _bulk_bytes(info) / (bulk_avg * 1e-3) / 1e9
    return {"value": round(NR * NZ * steps / (ms * 1e-3) / 1e6, 2), "unit": "MLUPS", "kernel": _bulk_kernel(storage, inplace),
            "ms_per_step": round(ms / steps, 5), "bytes_per_node": info.bytes_per_step // (NR * NZ),
            "bulk_avg_ms": round(bulk_avg, 5), "wall_avg_ms": round(wall_avg, 5),
            "achieved_gbs": round(achieved, 1), "frac": round(achieved / peak, 4),
            "traffic": None if inplace else _traffic(storage), "clocks": ck}


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_1409_5929_gb300 import inputs, lbm

    torch.cuda.set_device(local_rank)
    phi = inputs.porosity_field(NR, NZ, PHI_RECIPE["lo"], PHI_RECIPE["hi"], PHI_RECIPE["sigma"], PHI_RECIPE["seed"])
    stream = torch.cuda.Stream()
    s = _solver(lbm, args.storage, phi, stream, int(args.inplace))
    info = s.info()
    nodes = NR * NZ
    bulk_bytes = _bulk_bytes(info)

    s.step(args.warmup)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms, bulk_avg, wall_avg, ck = _time_steps(lbm, s, stream, args.steps)
    if world > 1:
        dist.barrier()
    ups, ms_max = aggregate(ms, float(nodes) * args.steps, device="cuda")
    value = ups / 1e6

    # end to end through the C ABI with host buffers: every step uploads its porosity field
    # from pinned host memory (the upload of step n + 1's input runs on the handle's copy
    # stream while step n computes) and copies its two Nusselt numbers back to pinned host
    # memory; the host waits once, at the end of the timed region, and checks every result.
    # The window is E2E_STEPS steps whatever --steps is, so that the first upload, which
    # nothing overlaps, does not dominate it.
    ke = max(E2E_STEPS, args.steps)
    phi_pinned = torch.from_numpy(phi).pin_memory()
    nus = torch.full((ke, 2), float("nan"), dtype=torch.float64).pin_memory()
    lbm.lbm_porosity_errors(s.h)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lbm.lbm_set_porosity_async(s.h, phi_pinned.data_ptr())          # input of the first step
    for n in range(ke):
        s.step(1)
        if n + 1 < ke:
            lbm.lbm_set_porosity_async(s.h, phi_pinned.data_ptr())  # input of step n + 1
        lbm.lbm_nusselt_async(s.h, nus[n])
    lbm.lbm_sync(s.h)
    t1 = time.perf_counter()
    nu = nus[-1].tolist()
    if not bool(torch.isfinite(nus).all()):
        raise RuntimeError("a step's Nusselt numbers did not arrive or are not finite")
    if lbm.lbm_porosity_errors(s.h):
        raise RuntimeError("porosity upload saw values outside (0, 1]")
    e2e_ups, _ = aggregate((t1 - t0) * 1e3, float(nodes) * ke, device="cuda")
    e2e_val = e2e_ups / 1e6
    s.close()
    if rank != 0:
        return None

    peak, peak_kind = _peaks()
    achieved = bulk_bytes / (bulk_avg * 1e-3) / 1e9
    line = {
        "metric": METRIC,
        "value": round(value, 2),
        "unit": "MLUPS",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_max / args.steps, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": _workload_name(args.storage), "storage": args.storage, "nodes": nodes,
                   "parallelism": f"replicas{world}" if world > 1 else "single",
                   "l2": "state larger than L2 (no flush)",
                   "bytes_per_step": info.bytes_per_step, "inplace": bool(args.inplace)},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4),
                     "traffic": None if args.inplace else _traffic(args.storage),
                     "kernel": _bulk_kernel(args.storage, int(args.inplace)), "peak_source": f"{peak_kind} hbm_gbs",
                     "avg_launch_ms": round(bulk_avg, 5), "bytes_per_launch": bulk_bytes,
                     "wall_kernel_avg_ms": round(wall_avg, 5)},
        "e2e": {"value": round(e2e_val, 2), "unit": "MLUPS", "h2d_bytes_per_step": nodes * 4,
                "d2h_bytes_per_step": 16, "steps": ke, "nusselt": list(nu) if nu else None},
        "gpu_launches": 2 * args.steps,
        "clocks": ck,
    }
    if world == 1 and not args.no_extras:
        line["storage_variants"] = {sto: storage_variant(lbm, sto, phi, args.steps, args.warmup, peak)
                                    for sto in ("f32", "f16", "bf16") if sto != args.storage}
        # one state buffer updated in place: half the state memory, one node per thread
        line["inplace_variants"] = {sto: storage_variant(lbm, sto, phi, args.steps, args.warmup, peak, 1)
                                    for sto in ("f32", "f16")}
    return line


def _sweep_params(lbm, n, seed, storage, nr_lo=64, nr_hi=512):
    from paper_1409_5929_gb300 import inputs

    return [lbm.lbm_params_default(nr=d["nr"], nz=d["nz"], Ra=d["Ra"], Da=d["Da"], eps_mean=d["eps"], Pr=d["Pr"],
                                   radius_ratio=d["radius_ratio"], storage=storage)
            for d in inputs.sweep_instances(n, seed=seed, nr_lo=nr_lo, nr_hi=nr_hi)]


def sweep_throughput(steps: int):
    """Batched sweep (256 annulus instances, Nr ~ U{64..512}, Nz = 2 Nr, Ra log-U[1e3, 1e6],
    Da log-U[1e-5, 1e-1], eps ~ U[0.3, 0.9], Pr in {0.71, 1, 7}, R* ~ U[1.5, 4], seed 3,
    FP16 storage): node updates per second of the batched launches vs the same
    instances stepped one at a time."""
    import torch

    from paper_1409_5929_gb300 import lbm

    params = _sweep_params(lbm, 256, 3, "f16")
    nodes = sum(p.nr * p.nz for p in params)
    b = lbm.Batch(params)
    cols, rows, _ = b.tune(10)
    steps += steps % 2   # even: the A/B parity at the timed replay is the one the graph was captured at
    b.step(10)
    b.run(steps, steps, -1.0)   # captures the check interval's CUDA graph, once per run as in a long sweep
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.step(steps)
    b.run(steps, steps, -1.0)   # graph-replayed steps
    torch.cuda.synchronize()
    tb = (time.perf_counter() - t0) / (2 * steps)
    b.close()
    singles = [lbm.Solver(p) for p in params]
    for s in singles:
        s.step(3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in singles:
        s.step(steps)
    torch.cuda.synchronize()
    ts = (time.perf_counter() - t0) / steps
    for s in singles:
        s.close()
    return {"workload": "256 annulus instances of the sweep draws (seed 3), 48.6 M nodes, FP16 storage",
            "batched_mlups": round(nodes / tb / 1e6, 1), "one_at_a_time_mlups": round(nodes / ts / 1e6, 1),
            "speedup": round(ts / tb, 2), "tile": "staged, 256 columns x up to 16 rows (even nz)",
            "tuned_tile": f"{cols}x{rows}", "steps": 2 * steps, "graph": "captured before the timed steps"}


def _tts_subset(n: int = 16):
    """The n draws of the 256-instance sweep (seed 3, Nr ~ U{64..512}) with the shortest
    diffusive time, estimated as 3 L^2 Pr / (tau - 1/2) = 17.3 L sqrt(Pr Ra) steps at the
    Ma = 0.1 of Eq. 39: a subset at the sweep's real sizes that finishes in bounded time."""
    from paper_1409_5929_gb300 import inputs

    draws = inputs.sweep_instances(256, seed=3)
    est = sorted((17.3 * (d["nr"] - 1) * (d["Pr"] * d["Ra"]) ** 0.5, i) for i, d in enumerate(draws))
    return sorted(i for _, i in est[:n])


def _settle_time(times, nus, ref, tol):
    """Wall time at the first check after which |Nu - ref| <= tol on both walls holds to the
    end of the record (None if it never does)."""
    ok = np.abs(np.asarray(nus) - ref[None]).max(axis=-1) <= tol
    for k in range(len(ok)):
        if ok[k:].all():
            return times[k]
    return None


def time_to_steady(max_steps: int = 400000, check: int = 1000, tol: float = 1e-8, dnu_tol: float = 1e-3):
    """Time to steady state for a subset of the batched sweep (_tts_subset): each instance
    alone with FP32 storage (plain), the batch with FP32 storage, the batch with FP16
    storage.  Two criteria: (a) the method's residual criterion (interval mean change per
    step <= tol, lbm_run / lbm_batch_run), and (b) the metric's: the wall time after which
    both Nusselt numbers stay within dnu_tol of the plain FP32 run's final values."""
    import torch

    from paper_1409_5929_gb300 import inputs, lbm

    idx = _tts_subset()
    draws = inputs.sweep_instances(256, seed=3)

    def params(sto):
        return [lbm.lbm_params_default(nr=draws[i]["nr"], nz=draws[i]["nz"], Ra=draws[i]["Ra"], Da=draws[i]["Da"],
                                       eps_mean=draws[i]["eps"], Pr=draws[i]["Pr"],
                                       radius_ratio=draws[i]["radius_ratio"], storage=sto) for i in idx]

    out = {"workload": f"{len(idx)} draws of the 256-instance sweep (seed 3) with the shortest estimated diffusive "
                       f"time: Nr {min(draws[i]['nr'] for i in idx)}..{max(draws[i]['nr'] for i in idx)}, Nz = 2 Nr, "
                       f"{sum(draws[i]['nr'] * draws[i]['nz'] for i in idx) / 1e6:.2f} M nodes",
           "criterion_residual": f"interval residual <= {tol:g}, checked every {check} steps, cap {max_steps} steps",
           "criterion_nu": f"|Nu - Nu_ref| <= {dnu_tol:g} on both walls from then on; Nu_ref = plain FP32 at its end",
           "criterion_consecutive": "residual between the last two states (lbm_residual), reported at the end of each "
                                    "plain run: rounding jitter keeps it above the interval mean, so it is not the "
                                    "stopping test"}
    # plain FP32: one instance at a time, Nusselt numbers recorded at every check
    recs, t_total = [], 0.0
    for p in params("f32"):
        s = lbm.Solver(p)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        times, nus, done, res = [], [], 0, np.inf
        while done < max_steps and not res <= tol:
            n, res = s.run(check, check, tol)
            done += n
            nus.append(s.nusselt())
            times.append(time.perf_counter() - t0)
        t_total += times[-1]
        recs.append((times, nus, done, res, s.residual()[0]))
        s.close()
    nu_ref = np.array([r[1][-1] for r in recs])
    settle = [_settle_time(r[0], r[1], nu_ref[k], dnu_tol) for k, r in enumerate(recs)]
    out["plain_fp32"] = {"s": round(t_total, 3), "converged": int(sum(r[3] <= tol for r in recs)), "of": len(recs),
                         "steps_max": int(max(r[2] for r in recs)),
                         "nu_settle_s_sum": round(sum(x for x in settle if x is not None), 3),
                         "nu_settled": int(sum(x is not None for x in settle)),
                         "interval_residual_max_end": float(max(r[3] for r in recs)),
                         "consecutive_residual_max_end": float(max(r[4] for r in recs))}
    for name, sto in (("batched_fp32", "f32"), ("batched_fp16", "f16")):
        b = lbm.Batch(params(sto))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        times, nus, total = [], [], 0
        res = np.full(len(idx), np.inf)
        while total < max_steps and not (res <= tol).all():
            _, r = b.run(check, check, tol)
            res = np.where(np.isfinite(r), r, res)       # instances stopped earlier report inf
            total += check
            nus.append(np.stack(b.nusselt(), axis=1))
            times.append(time.perf_counter() - t0)
        b.close()
        nus = np.array(nus)
        settle = [_settle_time(times, nus[:, k], nu_ref[k], dnu_tol) for k in range(len(idx))]
        t_nu = max(x for x in settle if x is not None) if all(x is not None for x in settle) else None
        out[name] = {"s": round(times[-1], 3), "converged": int((res <= tol).sum()), "of": len(idx),
                     "steps": int(total), "speedup_vs_plain": round(out["plain_fp32"]["s"] / times[-1], 2),
                     "nu_settled": int(sum(x is not None for x in settle)),
                     "nu_settle_s": round(t_nu, 3) if t_nu is not None else None,
                     "nu_speedup_vs_plain": round(out["plain_fp32"]["nu_settle_s_sum"] / t_nu, 2) if t_nu else None,
                     "max_abs_dNu_end": float(np.abs(nus[-1] - nu_ref).max()),
                     "residual_max_end": float(np.max(res))}
    return out


def warm_start_section(nr: int = 64, nz: int = 128, ntrain: int = 256, nheld: int = 32, check: int = 1000,
                       tol: float = 1e-8, max_steps: int = 200000, dnu_tol: float = 1e-3):
    """Bounded learned-warm-start measurement (the config-4 pipeline at a reduced size):
    steady fields of ntrain sweep-range instances from the batched solver, the network
    trained on them on the GPU, then nheld held-out instances run to the residual
    criterion (batched, FP32) from the cold start and from the network's fields.  Warm
    time includes the network's inference and the upload of its fields."""
    import torch

    from paper_1409_5929_gb300 import fno as F, lbm, warmstart as W

    t0 = time.perf_counter()
    train_inst = W.make_instances(ntrain, 40000, nr, nz)
    held = W.make_instances(nheld, 50000, nr, nz)
    _, res_tr, _, fields, dt_gen = W.run_batch(train_inst, max_steps, check, tol)
    X = torch.tensor(W.features(train_inst, nr, nz), device="cuda")
    Y = torch.tensor(np.stack([W.targets_from_fields(f[1], f[2], f[3]) for f in fields]), device="cuda")
    # one untimed epoch of a throwaway network on 16 samples: first-use costs of the process
    # (module loading, PyTorch's own kernels built for this GPU on first use) stay outside
    # the timed training
    tw = time.perf_counter()
    W.train(F.make_fno(nr, nz, width=32, modes=16, seed=2), X[:16], Y[:16], epochs=1, batch=8, lr=2e-3)
    torch.cuda.synchronize()
    t_warmup = time.perf_counter() - tw
    net = F.make_fno(nr, nz, width=32, modes=16, seed=1)
    t1 = time.perf_counter()
    losses = W.train(net, X, Y, epochs=20, batch=8, lr=2e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1

    def run(warm):
        b = lbm.Batch([p for p, _, _ in held])
        for i, (p, phi, _) in enumerate(held):
            b.set_porosity(i, phi)
        torch.cuda.synchronize()
        ts = time.perf_counter()
        if warm:
            pred = W.predict(net, torch.tensor(W.features(held, nr, nz), device="cuda"))
            ur, uz, T = W.fields_from_targets(pred)
            for i in range(len(held)):
                b.init_fields(i, ur[i], uz[i], T[i])
        else:
            for i in range(len(held)):
                b.init_fields(i)
        torch.cuda.synchronize()
        t_start = time.perf_counter() - ts
        times, nus, total = [], [], 0
        res = np.full(len(held), np.inf)
        steps = np.zeros(len(held), np.int64)
        while total < max_steps and not (res <= tol).all():
            st, r = b.run(check, check, tol)
            res = np.where(np.isfinite(r), r, res)       # instances stopped earlier report inf
            steps += st
            total += check
            nus.append(np.stack(b.nusselt(), axis=1))
            times.append(time.perf_counter() - ts)
        b.close()
        return t_start, np.array(times), np.array(nus), steps, res

    c_start, c_t, c_nu, c_steps, c_res = run(False)
    w_start, w_t, w_nu, w_steps, w_res = run(True)
    both = (c_res <= tol) & (w_res <= tol)
    ref = c_nu[-1]
    agree = np.abs(w_nu[-1] - ref).max(axis=1) <= dnu_tol
    settle_c = [_settle_time(c_t, c_nu[:, k], ref[k], dnu_tol) for k in range(len(held))]
    settle_w = [_settle_time(w_t, w_nu[:, k], ref[k], dnu_tol) for k in range(len(held))]
    ok = [k for k in range(len(held)) if both[k] and settle_c[k] is not None and settle_w[k] is not None]
    return {
        "workload": f"{nr}x{nz} annuli, sweep parameter ranges, smoothed porosity; {ntrain} training fields, "
                    f"{nheld} held-out; FNO 4 layers, width 32, 16 modes, 20 epochs",
        "data_generation_s": round(dt_gen, 2), "train_s": round(t_train, 2), "train_warmup_s": round(t_warmup, 2),
        "train_converged": int((res_tr <= tol).sum()), "loss_first_last": [losses[0], losses[-1]],
        "cold": {"converged": int((c_res <= tol).sum()), "s_to_all_converged_or_cap": round(float(c_t[-1]), 3),
                 "steps_sum": int(c_steps.sum()), "start_s": round(c_start, 3)},
        "warm": {"converged": int((w_res <= tol).sum()), "s_to_all_converged_or_cap": round(float(w_t[-1]), 3),
                 "steps_sum": int(w_steps.sum()), "start_s_incl_inference": round(w_start, 3)},
        "both_converged": int(both.sum()), "warm_agrees_with_cold_within_dNu_tol": int((agree & both).sum()),
        "steps_ratio_cold_over_warm": round(float(c_steps[both].sum()) / max(float(w_steps[both].sum()), 1.0), 3)
        if both.any() else None,
        "nu_settle_s_cold_sum": round(sum(settle_c[k] for k in ok), 3) if ok else None,
        "nu_settle_s_warm_sum": round(sum(settle_w[k] for k in ok), 3) if ok else None,
        "wall_s_ratio_cold_over_warm": round(float(c_t[-1]) / float(w_t[-1]), 3),
        "total_s": round(time.perf_counter() - t0, 1),
    }


def _oracle_sample_state():
    from oracle import oracle as O

    from paper_1409_5929_gb300 import inputs

    O.build()
    phi = inputs.porosity_field(SAMPLE_NR, SAMPLE_NZ, PHI_RECIPE["lo"], PHI_RECIPE["hi"], PHI_RECIPE["sigma"],
                                PHI_RECIPE["seed"])
    p = O.params(nr=SAMPLE_NR, nz=SAMPLE_NZ, radius_ratio=2.0, Ra=1e6, Da=1e-4, Pr=0.71, F_eps=-1.0,
                 eps_mean=float(phi.mean(dtype=np.float64)))
    return O.State(p, phi=phi.astype(np.float64))


def _oracle_mlups(threads: int, seconds: float):
    st = _oracle_sample_state()
    st.run(2, threads)
    steps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        st.run(5 if threads == 1 else 10, threads)
        steps += 5 if threads == 1 else 10
    dt = time.perf_counter() - t0
    return SAMPLE_NR * SAMPLE_NZ * steps / dt / 1e6, steps, dt


def cpu_sample(seconds: float):
    """The oracle as it stands on a bounded sample: the same recipe on a 256 x 512
    annulus, on all host cores for about `seconds` and on one core for about half that."""
    cores = os.cpu_count() or 1
    v, steps, dt = _oracle_mlups(cores, seconds)
    v1, steps1, dt1 = _oracle_mlups(1, 0.5 * seconds)
    return {"value": round(v, 3), "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle, same recipe on a {SAMPLE_NR}x{SAMPLE_NZ} annulus, {steps} steps, {dt:.1f} s",
            "single_thread": {"value": round(v1, 3), "unit": "MLUPS", "cores": 1,
                              "sample": f"same, one thread, {steps1} steps, {dt1:.1f} s"}}


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores, bounded sample per step."""
    from oracle import oracle as O

    from paper_1409_5929_gb300 import inputs

    O.build()
    phi = inputs.porosity_field(SAMPLE_NR, SAMPLE_NZ, PHI_RECIPE["lo"], PHI_RECIPE["hi"], PHI_RECIPE["sigma"],
                                PHI_RECIPE["seed"])
    p = O.params(nr=SAMPLE_NR, nz=SAMPLE_NZ, radius_ratio=2.0, Ra=1e6, Da=1e-4, Pr=0.71, F_eps=-1.0,
                 eps_mean=float(phi.mean(dtype=np.float64)))
    st = O.State(p, phi=phi.astype(np.float64))
    cores = os.cpu_count() or 1
    st.run(args.warmup, cores)
    t0 = time.perf_counter()
    st.run(args.steps, cores)
    dt = time.perf_counter() - t0
    value = SAMPLE_NR * SAMPLE_NZ * args.steps / dt / 1e6
    sample = f"FP64 oracle, same recipe on a {SAMPLE_NR}x{SAMPLE_NZ} annulus, {args.steps} steps"
    return {
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "MLUPS", "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": _workload_name("f64") + f" (sampled at {SAMPLE_NR}x{SAMPLE_NZ})"},
        "cpu_baseline": {"value": round(value, 3), "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--storage", choices=["f32", "f16", "bf16"], default="f32")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-extras", action="store_true", help="skip the sweep and time-to-steady sections")
    ap.add_argument("--nr", type=int, default=NR, help="override the grid (profiling of small cases only)")
    ap.add_argument("--nz", type=int, default=NZ)
    ap.add_argument("--inplace", action="store_true", help="one state buffer updated in place (AA pattern)")
    args = ap.parse_args()
    _set_grid(args.nr, args.nz)
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank == 0:
            ref_args = argparse.Namespace(steps=min(args.steps, 40), warmup=min(args.warmup, 3))
            print(json.dumps(run_reference(ref_args)), flush=True)
        return

    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    from paper_1409_5929_gb300 import build

    if rank == 0:
        build.build()
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
    line = run_ours(args, rank, world, local_rank)
    if rank == 0 and world == 1 and not args.no_extras:
        line["sweep"] = sweep_throughput(100)
        line["time_to_steady"] = time_to_steady()
        line["warm_start"] = warm_start_section()
    if rank == 0:
        line["cpu_baseline"] = cpu_sample(args.cpu_seconds) if world == 1 and args.cpu_seconds > 0 else None
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
