"""Measurement of the warm-start network's GPU work: one training step (forward,
backward, Adam) of the FNO at its training size, and every GEMM of that step timed on
its own with CUDA events, for both tensor-core paths of libfno.so (mma.sync and
tcgen05.mma).

Each GEMM reads A (M x K) and B (K x N) and writes C (M x N) in FP32 (and reads C when
beta != 0); the operands are rounded to BF16 on the way into shared memory, so the
algorithmic traffic is 4 (M K + K N + M N (1 + [beta != 0])) bytes per batch entry and the
work 2 M N K flops.  With K, N <= 256 (mostly 32) these contractions carry under 16 flops
per byte: they are bound by HBM, not by the tensor cores, and the roofline is the
measured copy bandwidth.

    python -m paper_1409_5929_gb300.fno_bench [--nr 128 --nz 256 --batch 8]

prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import fno as F

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, 1900.0, "fallback"


def _gemm_calls(net, x, t):
    """The fno_gemm calls of one loss_and_grad, with their arguments."""
    calls = []
    orig = F.fno_gemm

    def rec(*a, **kw):
        calls.append((a, kw))
        return orig(*a, **kw)

    F.fno_gemm = rec
    try:
        net.zero_grad()
        net.loss_and_grad(x, t)
    finally:
        F.fno_gemm = orig
    return calls


def _time_calls(calls, reps):
    """Mean device time of each call over `reps` replays (CUDA events on the stream the
    kernels are launched on)."""
    import torch

    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in calls]
    tot = np.zeros(len(calls))
    for _ in range(reps):
        for (a, kw), (e0, e1) in zip(calls, ev):
            e0.record(stream)
            F.fno_gemm(*a, **kw)
            e1.record(stream)
        torch.cuda.synchronize()
        tot += [e0.elapsed_time(e1) for e0, e1 in ev]
    return tot / reps


def main():
    import torch

    ap = argparse.ArgumentParser()
    ap.add_argument("--nr", type=int, default=128)
    ap.add_argument("--nz", type=int, default=256)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--fused-only", action="store_true", help="time only the fused path (profiling)")
    a = ap.parse_args()
    hbm, tc, src = _peaks()
    rng = np.random.default_rng(0)
    x = torch.tensor(rng.normal(size=(a.batch, a.nr, a.nz, 8)).astype(np.float32), device="cuda")
    t = torch.tensor(rng.normal(size=(a.batch, a.nr, a.nz, 3)).astype(np.float32), device="cuda")
    out = {"workload": f"FNO training step, batch {a.batch} x {a.nr} x {a.nz}, width 32, 16 modes, 4 layers",
           "peaks": {"hbm_gbs": hbm, "bf16_tflops": tc, "source": src}, "paths": {}}
    for path, name in ((0, "mma.sync"), (1, "tcgen05")) if not a.fused_only else ():
        F.fno_set_tensor_path(path)
        net = F.FNO2d(a.nr, a.nz, seed=1)
        for _ in range(3):
            net.zero_grad()
            net.loss_and_grad(x, t)
            net.adam_step(1e-3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(a.steps):
            net.zero_grad()
            net.loss_and_grad(x, t)
            net.adam_step(1e-3)
        torch.cuda.synchronize()
        step_ms = (time.perf_counter() - t0) / a.steps * 1e3
        calls = _gemm_calls(net, x, t)
        ms = _time_calls(calls, 5)
        shapes = {}
        for (args, kw), m in zip(calls, ms):
            tA, tB, M, N, K = args[:5]
            beta = args[12]
            batch = kw.get("batch", args[16] if len(args) > 16 else 1)
            key = f"{'T' if tA else 'N'}{'T' if tB else 'N'} M={M} N={N} K={K} batch={batch}"
            byt = 4.0 * batch * (M * K + K * N + M * N * (2 if beta != 0 else 1))
            fl = 2.0 * batch * M * N * K
            s = shapes.setdefault(key, {"calls": 0, "ms": 0.0, "bytes": 0.0, "flops": 0.0})
            s["calls"] += 1
            s["ms"] += float(m)
            s["bytes"] += byt
            s["flops"] += fl
        gemm_ms = float(ms.sum())
        top = sorted(shapes.items(), key=lambda kv: -kv[1]["ms"])[:6]
        out["paths"][name] = {
            "train_step_ms": round(step_ms, 3),
            "gemm_ms_per_step": round(gemm_ms, 3),
            "gemm_calls": len(calls),
            "gemm_gbs": round(sum(s["bytes"] for s in shapes.values()) / (gemm_ms * 1e-3) / 1e9, 1),
            "gemm_frac_of_hbm": round(sum(s["bytes"] for s in shapes.values()) / (gemm_ms * 1e-3) / 1e9 / hbm, 4),
            "gemm_tflops": round(sum(s["flops"] for s in shapes.values()) / (gemm_ms * 1e-3) / 1e12, 2),
            "top_shapes": [{"shape": k, "calls": v["calls"], "ms": round(v["ms"], 4),
                            "gbs": round(v["bytes"] / (v["ms"] * 1e-3) / 1e9, 1),
                            "frac_of_hbm": round(v["bytes"] / (v["ms"] * 1e-3) / 1e9 / hbm, 4),
                            "tflops": round(v["flops"] / (v["ms"] * 1e-3) / 1e12, 2)} for k, v in top],
            "tensor_path_status": F.fno_tensor_path_status(True),
        }
    F.fno_set_tensor_path(0)
    out["paths"]["fused"] = fused_step(a, x, t, hbm)
    print(json.dumps(out), flush=True)


def fused_bytes(B, nr, nz, width=32, in_ch=8, out_ch=3, layers=4):
    """Algorithmic HBM bytes of one fused training step's pixel-space kernels (BF16
    activations): lift reads x and writes h0; each layer reads h and writes pre and
    GELU(pre) (the last only pre); the projection reads hL and the targets and writes y and
    dL/dhL; the backward kernels read dL/dpre, pre and h and write the next dL/dpre (the
    last layer's kernel reads two of them, the lift's dL/dpre and x).  The spectra and
    weights (under 1 %) are left out."""
    P = B * nr * nz
    act = 2 * P * width
    return (P * in_ch * 4 + act                                   # lift
            + (layers - 1) * 3 * act + 2 * act                    # layers
            + act + P * out_ch * 8 + act                          # projection
            + 2 * act + (layers - 1) * 4 * act + act + P * in_ch * 4)   # backward


def fused_step(a, x, t, hbm):
    """The fused tcgen05 network: training step (forward, loss, backward, Adam) and its
    forward and backward halves timed with CUDA events."""
    import torch

    if not F.net_supported(a.batch, a.nr, a.nz, 32, 16, 128, 8, 3):
        return {"unsupported": True}
    net = F.FusedFNO2d(a.nr, a.nz, seed=1)
    for _ in range(3):
        net.zero_grad()
        net.loss_and_grad(x, t)
        net.adam_step(1e-3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        net.zero_grad()
        net.loss_and_grad(x, t)
        net.adam_step(1e-3)
    torch.cuda.synchronize()
    step_ms = (time.perf_counter() - t0) / a.steps * 1e3
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    fw = bw = 0.0
    for _ in range(a.steps):
        ev[0].record()
        net.forward(x, train=True, t=t)
        ev[1].record()
        net._backward_layers(x, x.shape[0])
        ev[2].record()
        torch.cuda.synchronize()
        fw += ev[0].elapsed_time(ev[1])
        bw += ev[1].elapsed_time(ev[2])
    fw, bw = fw / a.steps, bw / a.steps
    byt = fused_bytes(a.batch, a.nr, a.nz)
    return {"train_step_ms": round(step_ms, 3), "forward_loss_ms": round(fw, 4), "backward_ms": round(bw, 4),
            "pixel_bytes_per_step": byt, "fwd_bwd_gbs": round(byt / ((fw + bw) * 1e-3) / 1e9, 1),
            "fwd_bwd_frac_of_hbm": round(byt / ((fw + bw) * 1e-3) / 1e9 / hbm, 4),
            "status": F.fno_net_status(True)}


if __name__ == "__main__":
    main()
