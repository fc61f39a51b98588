"""Storage-codec experiment on the FP64 oracle (opt-in, LBM_SLOW=1, about 6 min): the
16-bit flow storage of the CUDA path is emulated by rounding the stored flow deviations to
FP16 (and the temperature deviations to FP32) after every oracle step.

It backs two statements about the 16-bit path on a convective instance of the
time-to-steady set (28 x 56 annulus, Ra = 8.4e4, Da = 0.057, Pr = 1):
  - as built (deviations from the rest state r w_i + e_ir w_i / 2), the steady Nusselt
    numbers miss the FP64 ones by more than 1e-3 and keep drifting;
  - stored against a per-node reference equilibrium f_eq(rho_ref, u_ref) + e_ir w_i / 2
    (rho_ref - 1 and u_ref held in FP16, refreshed every 1000 steps), they land within
    3e-4 and the drift falls by more than an order of magnitude.
The equilibrium here is Eq. 32's, written out for the emulation."""
import os

import numpy as np
import pytest

from paper_1409_5929_gb300 import inputs

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], float)
EZ = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], float)
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
WT = np.array([0.6, 0.1, 0.1, 0.1, 0.1])
CS2 = 1.0 / 3.0


def _q16(x):
    return x.astype(np.float16).astype(np.float64)


def _q32(x):
    return x.astype(np.float32).astype(np.float64)


@pytest.mark.slow
@pytest.mark.skipif(not os.environ.get("LBM_SLOW"), reason="set LBM_SLOW=1 (about 6 min on one core)")
def test_flow_reference_tames_fp16_storage(oracle):
    d = inputs.sweep_instances(16, seed=4, nr_lo=24, nr_hi=48)[6]
    p = oracle.params(nr=d["nr"], nz=d["nz"], Ra=d["Ra"], Da=d["Da"], eps_mean=d["eps"], Pr=d["Pr"],
                      radius_ratio=d["radius_ratio"])
    c = oracle.derive(p)
    r = c["r0"] + np.arange(p.nr)
    half_er = (0.5 * EX[:, None] * W9[:, None])[:, :, None]
    rest_f = (r[None, :, None] * W9[:, None, None]) + half_er
    rest_g = (WT * c["T0"])[:, None, None]

    def feq(rho, ur, uz):
        u2 = ur * ur + uz * uz
        eu = EX[:, None, None] * ur[None] + EZ[:, None, None] * uz[None]
        phi = d["eps"]
        return W9[:, None, None] * r[None, :, None] * rho[None] * (
            1 + eu / CS2 + eu * eu / (2 * phi * CS2 * CS2) - u2[None] / (2 * phi * CS2))

    def run(mode, chunks=200, chunk=1000):
        st = oracle.State(p)
        fref = rest_f
        nus = []
        for _ in range(chunks):
            if mode == "reference":
                rho, ur, uz, _ = st.moments()
                fref = feq(_q16(rho - 1) + 1, _q16(ur), _q16(uz)) + half_er
            for _ in range(chunk):
                if mode != "fp64":
                    st.f[:] = _q16(st.f - fref) + fref
                    st.g[:] = _q32(st.g - rest_g) + rest_g
                st.run(1, 1)
            nus.append(st.nusselt())
        return np.array(nus)

    nus64 = run("fp64")
    nu64 = nus64[-1]
    assert np.abs(nus64[-21:] - nu64).max() < 1e-7
    # largest |dNu| and drift over the last 2e4 steps (the emulated 16-bit runs wander)
    window = {mode: run(mode)[-21:] for mode in ("rest", "reference")}
    err_rest, err_ref = (np.abs(window[m] - nu64).max() for m in ("rest", "reference"))
    drift_rest, drift_ref = (np.ptp(window[m], axis=0).max() for m in ("rest", "reference"))
    print("FP16 flow storage |dNu|: rest-state deviation", err_rest, "reference", err_ref,
          "drift", drift_rest, drift_ref)
    assert err_rest > 1e-3 and err_ref < 3e-4
    assert drift_ref < 0.1 * drift_rest
