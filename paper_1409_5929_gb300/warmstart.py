"""Learned warm start of the steady-state iteration.

Pipeline (all compute on the GPU: the lattice Boltzmann step in liblbm.so, the network
in libfno.so):
  1. instances: parameter draws of the batched sweep (Ra log-U[1e3, 1e6], Da log-U[1e-5,
     1e-1], eps ~ U[0.3, 0.9], Pr in {0.71, 1, 7}, R* ~ U[1.5, 4]) on an nr x nz annulus,
     each with a smoothed porosity field of mean eps (inputs.porosity_field_around);
  2. targets: the solver's own steady fields (lbm_batch_run to the steady criterion,
     capped at max_steps);
  3. training: the FNO (4 Fourier layers, width 32, 16 modes) on normalised inputs
     (porosity, five parameter planes, r, z) and outputs (u_r / U, u_z / U, 2 (T - T0) / dT
     with U = Ma c_s), MSE, Adam, BF16 tensor-core GEMMs with FP32 accumulation;
  4. warm start of held-out instances: the network's fields through lbm_init_fields,
     then the same iteration from them, which decides the result; cold and warm runs
     record their Nusselt numbers along a long run, and the steps each needs to come
     within dNu_tol of the cold run's final values are compared on the instances where
     both runs are stationary (summarize).

    python -m paper_1409_5929_gb300.warmstart [--ntrain 2000] [--nheld 256] ...
prints one JSON line with the measurements.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import inputs, lbm
from . import fno as F

U_LATTICE = 0.1 / math.sqrt(3.0)   # U = Ma c_s with the Ma = 0.1 of Eq. 39


def make_instances(n: int, seed: int, nr: int, nz: int, amp: float = 0.05, sigma: float = 8.0):
    draws = inputs.sweep_instances(n, seed=seed, nr_lo=nr, nr_hi=nr)
    out = []
    for k, d in enumerate(draws):
        phi = inputs.porosity_field_around(nr, nz, d["eps"], amp, sigma, seed * 100003 + k)
        p = lbm.lbm_params_default(nr=nr, nz=nz, Ra=d["Ra"], Da=d["Da"], Pr=d["Pr"],
                                   radius_ratio=d["radius_ratio"], eps_mean=float(phi.mean(dtype=np.float64)))
        out.append((p, phi, d))
    return out


def features(inst, nr: int, nz: int) -> np.ndarray:
    """[n, nr, nz, 8] float32: porosity, log Ra, log Da, eps, log Pr, R*, r, z (scaled to ~[-1, 1])."""
    X = np.empty((len(inst), nr, nz, 8), np.float32)
    rr = np.linspace(-1, 1, nr, dtype=np.float32)[:, None]
    zz = np.linspace(-1, 1, nz, dtype=np.float32)[None, :]
    for i, (p, phi, d) in enumerate(inst):
        X[i, :, :, 0] = (phi - 0.6) / 0.3
        X[i, :, :, 1] = (math.log10(d["Ra"]) - 4.5) / 1.5
        X[i, :, :, 2] = (math.log10(d["Da"]) + 3.0) / 2.0
        X[i, :, :, 3] = (d["eps"] - 0.6) / 0.3
        X[i, :, :, 4] = math.log10(d["Pr"]) / 0.85
        X[i, :, :, 5] = (d["radius_ratio"] - 2.75) / 1.25
        X[i, :, :, 6] = rr
        X[i, :, :, 7] = zz
    return X


def targets_from_fields(ur, uz, T, T0=0.5, dT=1.0):
    return np.stack([ur / U_LATTICE, uz / U_LATTICE, 2.0 * (T - T0) / dT], axis=-1).astype(np.float32)


def fields_from_targets(Y, T0=0.5, dT=1.0):
    return Y[..., 0] * U_LATTICE, Y[..., 1] * U_LATTICE, T0 + 0.5 * dT * Y[..., 2]


def run_batch(inst, max_steps, check, tol, warm=None):
    """Batched run of instances to the criterion; returns steps, criterion values, Nu
    (inner, outer), the fields and the wall time.  warm: optional (ur, uz, T) arrays
    [n, nr, nz] as start fields."""
    import torch

    b = lbm.Batch([p for p, _, _ in inst])
    for i, (p, phi, _) in enumerate(inst):
        b.set_porosity(i, phi)
        if warm is None:
            b.init_fields(i)
        else:
            b.init_fields(i, warm[0][i], warm[1][i], warm[2][i])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steps, res = b.run(max_steps, check, tol)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    nu = np.stack(b.nusselt(), axis=1)
    fields = [b.moments(i) for i in range(len(inst))]
    b.close()
    return steps, res, nu, fields, dt


def nu_trajectory(inst, total, chunk, warm=None):
    """Advance every instance `total` steps (batched, graph-replayed chunks, no early
    stop) and record both Nusselt numbers after each chunk: [nchunks, n, 2]."""
    import torch

    b = lbm.Batch([p for p, _, _ in inst])
    for i, (p, phi, _) in enumerate(inst):
        b.set_porosity(i, phi)
        if warm is None:
            b.init_fields(i)
        else:
            b.init_fields(i, warm[0][i], warm[1][i], warm[2][i])
    torch.cuda.synchronize()
    traj, done = [], 0
    t0 = time.perf_counter()
    while done < total:
        b.run(chunk, chunk, -1.0)
        done += chunk
        traj.append(np.stack(b.nusselt(), axis=1))
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    fields = [b.moments(i) for i in range(len(inst))]
    b.close()
    return np.stack(traj), dt, fields


def steps_to_nu(traj, ref, tol, chunk):
    """First step count after which |Nu - ref| <= tol (both walls) holds to the end of the
    trajectory; -1 where it never settles."""
    err = np.abs(traj - ref[None]).max(axis=2)          # [nchunks, n]
    ok = err <= tol
    settled = np.flip(np.logical_and.accumulate(np.flip(ok, 0), 0), 0)   # ok from t to the end
    first = np.where(settled.any(0), settled.argmax(0), -1)
    return np.where(first >= 0, (first + 1) * chunk, -1)


def summarize(traj_c, traj_w, chunk, tol, window, drift, groups=None):
    """Time-to-steady comparison of cold and warm Nusselt trajectories [nchunks, n, 2]
    recorded every `chunk` steps.

    An instance is stationary when, over the last `window` steps, both runs' Nusselt
    numbers stay within `drift` of their final values; only then does "time to steady" mean
    something.  Among stationary instances, the warm run agrees when its final Nusselt
    numbers are within `tol` of the cold run's; for those, steps to |Nu - Nu_cold,end| <= tol
    (held to the end) are compared.  `groups` (optional, one label per instance) splits
    the three counts by label."""
    w = max(1, window // chunk)
    ref = traj_c[-1]
    d_c = np.abs(traj_c[-w:] - traj_c[-1][None]).max(axis=(0, 2))
    d_w = np.abs(traj_w[-w:] - traj_w[-1][None]).max(axis=(0, 2))
    stat = (d_c <= drift) & (d_w <= drift)
    dnu = np.abs(traj_w[-1] - ref).max(axis=1)
    agree = dnu <= tol
    s_c = steps_to_nu(traj_c, ref, tol, chunk)
    s_w = steps_to_nu(traj_w, ref, tol, chunk)
    ok = stat & agree & (s_c > 0) & (s_w > 0)
    dis = stat & ~agree
    out = {"stationary": int(stat.sum()), "stationary_agree": int(ok.sum()),
           "stationary_disagree": int(dis.sum()), "nonstationary": int((~stat).sum()),
           "disagree_dNu_quantiles_50_90_max": [float(np.quantile(dnu[dis], q)) for q in (0.5, 0.9, 1.0)]
           if dis.any() else None}
    if ok.any():
        out.update({"cold_steps_median": int(np.median(s_c[ok])), "warm_steps_median": int(np.median(s_w[ok])),
                    "cold_steps_max": int(s_c[ok].max()), "warm_steps_max": int(s_w[ok].max()),
                    "steps_ratio_cold_over_warm_sum": round(float(s_c[ok].sum()) / float(s_w[ok].sum()), 3)})
    if groups is not None:
        g = np.asarray(groups)
        out["by_group"] = {str(v): {"stationary_agree": int((ok & (g == v)).sum()),
                                    "stationary_disagree": int((dis & (g == v)).sum()),
                                    "nonstationary": int((~stat & (g == v)).sum())} for v in np.unique(g)}
    return out, ok


def train(net, X, Y, epochs, batch, lr, seed=0, log=None):
    import torch

    n = X.shape[0]
    rng = np.random.default_rng(seed)
    steps_per_epoch = n // batch
    total = epochs * steps_per_epoch
    losses = []
    it = 0
    for ep in range(epochs):
        perm = torch.tensor(rng.permutation(n)[: steps_per_epoch * batch], device="cuda").view(steps_per_epoch, batch)
        acc = torch.zeros((), dtype=torch.float64, device="cuda")
        for s in range(steps_per_epoch):
            idx = perm[s]
            xb = X.index_select(0, idx).contiguous()
            yb = Y.index_select(0, idx).contiguous()
            net.zero_grad()
            l = net.loss_and_grad(xb, yb)
            acc += l[0]
            cur_lr = lr * 0.5 * (1 + math.cos(math.pi * it / total))
            net.adam_step(cur_lr)
            it += 1
        losses.append(float(acc.item()) / steps_per_epoch)
        if log:
            log(f"epoch {ep} loss {losses[-1]:.4e}")
    return losses


def predict(net, X, batch=8):
    import torch

    out = []
    for s in range(0, X.shape[0], batch):
        xb = X[s:s + batch].contiguous()
        out.append(net.forward(xb).clone())
    torch.cuda.synchronize()
    return torch.cat(out).cpu().numpy()


def compare(cold_steps, cold_res, cold_nu, cold_fields, cold_dt, warm_steps, warm_res, warm_nu, warm_fields, warm_dt,
            pred, tol, dnu_tol):
    """Cold against warm start.  The iteration decides: where both runs reach the
    criterion their Nusselt numbers must agree within dnu_tol, else the instance falls
    back to the cold start (its cost then counts both runs); a warm run that fails to
    converge where the cold one converges also falls back."""
    ok_c = cold_res <= tol
    ok_w = (warm_res <= tol) & np.isfinite(warm_nu).all(axis=1)
    dnu = np.abs(warm_nu - cold_nu).max(axis=1)
    both = ok_c & ok_w
    agree = both & (dnu <= dnu_tol)
    fallback = (both & ~agree) | (ok_c & ~ok_w)
    rel = []
    for i in np.nonzero(both)[0]:
        g, c = warm_fields[i], cold_fields[i]
        rel.append(max(np.linalg.norm(g[3] - c[3]) / np.linalg.norm(c[3]),
                       np.linalg.norm(np.stack(g[1:3]) - np.stack(c[1:3])) / max(np.linalg.norm(np.stack(c[1:3])), 1e-30)))
    Yc = np.stack([targets_from_fields(f[1], f[2], f[3]) for f in cold_fields])
    steps_w = np.where(fallback, warm_steps + cold_steps, warm_steps)
    return {
        "cold": {"s": round(cold_dt, 2), "converged": int(ok_c.sum()), "steps_median": int(np.median(cold_steps))},
        "warm": {"s": round(warm_dt, 2), "converged": int(ok_w.sum()), "steps_median": int(np.median(warm_steps)),
                 "fallback_to_cold": int(fallback.sum()), "converged_only_warm": int((ok_w & ~ok_c).sum())},
        "both_converged": {
            "instances": int(both.sum()), "agree_within_dNu_tol": int(agree.sum()),
            "cold_steps_median": int(np.median(cold_steps[both])) if both.any() else None,
            "warm_steps_median": int(np.median(steps_w[both])) if both.any() else None,
            "steps_ratio_cold_over_warm": round(float(cold_steps[both].sum()) / max(float(steps_w[both].sum()), 1.0), 3)
            if both.any() else None,
            "max_abs_dNu": float(dnu[both].max()) if both.any() else None,
            "max_rel_l2_fields": float(max(rel)) if rel else None},
        "batch_time_ratio_cold_over_warm": round(cold_dt / warm_dt, 3) if warm_dt > 0 else None,
        "start_field_rms_error": {"trained_network": float(np.sqrt(((pred - Yc) ** 2).mean())),
                                  "rest_state": float(np.sqrt((Yc ** 2).mean()))},
    }


def main():
    import torch

    ap = argparse.ArgumentParser()
    ap.add_argument("--nr", type=int, default=128)
    ap.add_argument("--nz", type=int, default=256)
    ap.add_argument("--ntrain", type=int, default=2000)
    ap.add_argument("--nheld", type=int, default=256)
    ap.add_argument("--max-steps", type=int, default=300000)
    ap.add_argument("--check", type=int, default=1000)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--width", type=int, default=32)
    ap.add_argument("--modes", type=int, default=16)
    ap.add_argument("--dnu-tol", type=float, default=1e-3)
    ap.add_argument("--held-max-steps", type=int, default=800000)
    ap.add_argument("--nu-chunk", type=int, default=5000)
    ap.add_argument("--window", type=int, default=200000, help="stationarity window (steps)")
    ap.add_argument("--drift", type=float, default=1e-4, help="stationarity bound on |Nu - Nu_end|")
    ap.add_argument("--save", default="", help="write per-instance trajectories and parameters (npz) here")
    ap.add_argument("--verbose", action="store_true")
    a = ap.parse_args()
    log = (lambda s: print(s, flush=True)) if a.verbose else None
    nr, nz = a.nr, a.nz
    out = {"workload": f"warm start, {nr}x{nz} annulus, sweep parameter ranges, smoothed porosity (sigma 8)",
           "ntrain": a.ntrain, "nheld": a.nheld, "criterion": f"interval residual <= {a.tol:g}",
           "max_steps": a.max_steps}
    t0 = time.perf_counter()
    train_inst = make_instances(a.ntrain, 40000, nr, nz)
    held = make_instances(a.nheld, 50000, nr, nz)
    steps, res, nu, fields, dt = run_batch(train_inst, a.max_steps, a.check, a.tol)
    out["data_generation_s"] = round(dt, 2)
    out["train_converged"] = int((res <= a.tol).sum())
    Y = np.stack([targets_from_fields(f[1], f[2], f[3]) for f in fields])
    X = features(train_inst, nr, nz)
    Xd, Yd = torch.tensor(X, device="cuda"), torch.tensor(Y, device="cuda")
    net = F.make_fno(nr, nz, width=a.width, modes=a.modes, seed=1)
    t1 = time.perf_counter()
    losses = train(net, Xd, Yd, a.epochs, a.batch, a.lr, log=log)
    torch.cuda.synchronize()
    out["train_s"] = round(time.perf_counter() - t1, 2)
    out["train_loss_first_last"] = [losses[0], losses[-1]]
    Xh = torch.tensor(features(held, nr, nz), device="cuda")
    pred = predict(net, Xh)
    warm = fields_from_targets(pred)
    hm, ch = a.held_max_steps, a.nu_chunk
    traj_c, dt_c, f_c = nu_trajectory(held, hm, ch)
    traj_w, dt_w, f_w = nu_trajectory(held, hm, ch, warm=warm)
    pr = np.array([d["Pr"] for _, _, d in held])
    summ, ok = summarize(traj_c, traj_w, ch, a.dnu_tol, a.window, a.drift, groups=pr)
    if a.save:
        np.savez_compressed(a.save, traj_cold=traj_c, traj_warm=traj_w, chunk=ch,
                            Ra=np.array([d["Ra"] for _, _, d in held]), Da=np.array([d["Da"] for _, _, d in held]),
                            eps=np.array([d["eps"] for _, _, d in held]), Pr=pr,
                            Rstar=np.array([d["radius_ratio"] for _, _, d in held]))
    rel = [max(np.linalg.norm(f_w[i][3] - f_c[i][3]) / np.linalg.norm(f_c[i][3]),
               np.linalg.norm(np.stack(f_w[i][1:3]) - np.stack(f_c[i][1:3]))
               / max(np.linalg.norm(np.stack(f_c[i][1:3])), 1e-30)) for i in np.nonzero(ok)[0]]
    Yc = np.stack([targets_from_fields(f[1], f[2], f[3]) for f in f_c])
    ms_step = dt_c / hm * 1e3
    if ok.any():
        summ["time_to_steady_cold_s"] = round(summ["cold_steps_max"] * ms_step / 1e3, 2)
        summ["time_to_steady_warm_s"] = round(summ["warm_steps_max"] * ms_step / 1e3, 2)
    out.update({
        "time_to_steady_definition": f"steps until |Nu - Nu_ref| <= {a.dnu_tol:g} on both walls for the rest "
                                     f"of a {hm}-step run; Nu_ref = cold start at {hm} steps; checked every {ch}; "
                                     f"stationary = both runs within {a.drift:g} of their final Nu over the last "
                                     f"{a.window} steps",
        "batched_ms_per_step": round(ms_step, 4),
        "held_out": summ,
        "max_rel_l2_fields_warm_vs_cold_at_end": float(max(rel)) if rel else None,
        "start_field_rms_error": {"trained_network": float(np.sqrt(((pred - Yc) ** 2).mean())),
                                  "rest_state": float(np.sqrt((Yc ** 2).mean()))},
        "held_steps": hm,
        "total_s": round(time.perf_counter() - t0, 1),
    })
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
