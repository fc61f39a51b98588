"""16-bit flow storage against the flow reference (GPU) checked against the emulation of
the same codec on the FP64 oracle (tests/storage_emulation.py), and the steady-state bar of
the precision target: |Delta Nu| <= 1e-3 against FP32 storage on convective cases.

The emulation rounds the stored values exactly as the GPU's codec defines them, around
the oracle's FP64 step; the GPU differs from it by FP32 arithmetic and by where each
16-bit rounding falls.  Both must sit at the codec's error level against plain FP64, which
the same emulation without the reference (stored against the rest state, as the CUDA path
stored them before) exceeds by two orders of magnitude on these cases.
"""
import os

import numpy as np
import pytest

from paper_1409_5929_gb300 import inputs
from storage_emulation import Emulated16

pytestmark = pytest.mark.gpu
THREADS = min(16, os.cpu_count() or 1)


@pytest.fixture(scope="module")
def lbm():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1409_5929_gb300 import build, lbm as L

    build.build()
    L.load()
    return L


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _sweep_case(k):
    """Instance k of the time-to-steady set (sweep parameter ranges, Nr ~ U{24..48}, seed 4)."""
    d = inputs.sweep_instances(16, seed=4, nr_lo=24, nr_hi=48)[k]
    return dict(nr=d["nr"], nz=d["nz"], Ra=d["Ra"], Da=d["Da"], eps_mean=d["eps"], Pr=d["Pr"],
                radius_ratio=d["radius_ratio"])


def _oparams(oracle, kw):
    return oracle.params(**kw)


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("case", [6, 13])
def test_codec_against_emulation(lbm, oracle, storage, case):
    kw = _sweep_case(case)
    steps = 5000                       # four reference refreshes (every 1024 steps)
    s = lbm.Solver(lbm.lbm_params_default(storage=storage, **kw))
    s.step(steps)
    gm, nu_g = s.moments(), np.array(s.nusselt())
    em = Emulated16(oracle, _oparams(oracle, kw), storage=storage).run(steps)
    rest = Emulated16(oracle, _oparams(oracle, kw), storage=storage, reference=False).run(steps)
    st = oracle.State(_oparams(oracle, kw)).run(steps, THREADS)
    om, nu_o = st.moments(), np.array(st.nusselt())
    u = lambda m: np.stack(m[1:3])
    e_gpu, e_em, e_rest = _rel(u(gm), u(om)), _rel(u(em.moments()), u(om)), _rel(u(rest.moments()), u(om))
    d_gpu = np.abs(nu_g - nu_o).max()
    d_em = np.abs(np.array(em.nusselt()) - nu_o).max()
    d_rest = np.abs(np.array(rest.nusselt()) - nu_o).max()
    print(storage, case, "u rel L2 vs FP64: gpu", e_gpu, "emulated", e_em, "emulated rest-state", e_rest,
          "|dNu| gpu", d_gpu, "emulated", d_em, "rest", d_rest, "stored max", em.stored_magnitude())
    # the GPU carries the codec's error, not more (FP32 arithmetic adds ~1e-6)
    assert e_gpu <= 3 * e_em + 2e-5
    assert d_gpu <= 3 * d_em + 1e-5
    if storage == "f16":
        # in this transient; BF16 (8-bit significand) reaches the bar at steady state only
        # (test_steady_state_within_1e3_of_fp32), as its emulation does (3.4e-3 here)
        assert d_gpu <= 1e-3
    # and the reference is what brings it there
    assert e_em < 0.1 * e_rest


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_reference_refresh_keeps_the_state(lbm, storage):
    """A refresh re-encodes every flow population against a new reference: the populations
    change by the storage rounding of the (small) re-encoded values only, and a second
    refresh right after it by less than the first."""
    kw = _sweep_case(6)
    s = lbm.Solver(lbm.lbm_params_default(storage=storage, **kw))
    s.step(700)
    f0, _ = s.export_populations()
    s.rebase()
    f1, _ = s.export_populations()
    s.rebase()
    f2, _ = s.export_populations()
    r = s.info().r0 + np.arange(kw["nr"])
    W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    dev = np.abs(f0 - r[None, :, None] * W9[:, None, None]).max()
    ulp = 2.0 ** -11 if storage == "f16" else 2.0 ** -8
    d01, d12 = np.abs(f1 - f0).max(), np.abs(f2 - f1).max()
    print(storage, "refresh changes", d01, d12, "deviation scale", dev)
    assert d01 <= ulp * dev
    assert d12 <= d01


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_steady_state_within_1e3_of_fp32(lbm, storage):
    """Convective instances of the time-to-steady set run to steady state: the 16-bit
    steady Nusselt numbers lie within 1e-3 of the FP32 ones (absolute), as the precision
    target requires; the interval residual each storage reaches is reported."""
    for k in (6, 10, 13):
        kw = _sweep_case(k)
        out = {}
        for sto in ("f32", storage):
            s = lbm.Solver(lbm.lbm_params_default(storage=sto, **kw))
            n, res = s.run(300_000, 1000, 1e-8)
            out[sto] = (np.array(s.nusselt()), n, res)
            s.close()
        d = np.abs(out[storage][0] - out["f32"][0]).max()
        print(storage, k, kw["nr"], "Ra %.3g" % kw["Ra"], "Nu f32", out["f32"][0], "|dNu|", d,
              "steps/res f32", out["f32"][1:], storage, out[storage][1:])
        assert d <= 1e-3
