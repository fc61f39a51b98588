"""Writes slow_annulus_nusselt.txt: the FP64 oracle's steady Nusselt numbers (Eq. 42)
of a slowly converging porous annulus (Pr = 7, Ra ~ 1.1e3, 128 x 256, smoothed
porosity), from the cold start and from the conduction start.  Uses only the oracle
and the seeded input generators.

    python tests/golden/slow_annulus_case.py      (about 25 min on 8 cores)
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
from oracle import oracle as O  # noqa: E402
from paper_1409_5929_gb300 import inputs  # noqa: E402

NR, NZ, SEED, K = 128, 256, 50000, 8
STEPS, CHUNK = 400000, 50000


def case():
    """Parameters and porosity of draw K of the seeded sweep at NR x NZ."""
    d = inputs.sweep_instances(K + 1, seed=SEED, nr_lo=NR, nr_hi=NR)[K]
    phi = inputs.porosity_field_around(NR, NZ, d["eps"], 0.05, 8.0, SEED * 100003 + K)
    kw = dict(nr=NR, nz=NZ, Ra=d["Ra"], Da=d["Da"], Pr=d["Pr"], radius_ratio=d["radius_ratio"],
              eps_mean=float(phi.mean(dtype=np.float64)))
    return kw, phi


def conduction_T(p):
    d = O.derive(p)
    r = d["r0"] + np.arange(p.nr, dtype=np.float64)
    T = p.T_cold + (p.T_hot - p.T_cold) * np.log(r[-1] / r) / np.log(r[-1] / r[0])
    return np.repeat(T[:, None], p.nz, 1)


def main():
    kw, phi = case()
    p = O.params(**kw)
    out = {}
    for start in ("cold", "conduction"):
        if start == "cold":
            st = O.State(p, phi)
        else:
            z = np.zeros((p.nr, p.nz))
            st = O.State(p, phi, z, z, conduction_T(p))
        traj = []
        for _ in range(STEPS // CHUNK):
            st.run(CHUNK)
            traj.append(st.nusselt())
        out[start] = traj
    with open(os.path.join(HERE, "slow_annulus_nusselt.txt"), "w") as f:
        f.write("# FP64 oracle, Eq. 42 (Nu_inner, Nu_outer) every %d steps up to %d, from the cold start\n"
                "# and from the conduction profile (u = 0); written by slow_annulus_case.py\n" % (CHUNK, STEPS))
        f.write("# case: %s\n" % json.dumps(kw))
        for start, traj in out.items():
            for k, (a, b) in enumerate(traj):
                f.write("%s %d %.12f %.12f\n" % (start, (k + 1) * CHUNK, a, b))


if __name__ == "__main__":
    main()
