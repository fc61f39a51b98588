"""Emulation of the 16-bit storage codec on the FP64 oracle (test helper).

The CUDA path stores each flow population as
    s_i = f+_i - (r w_i + e_ir w_i / 2) - D_i,   D_i = w_i (A + 3 e_i.J),
rounded to FP16 (or BF16), with the node's reference A = sum of the post-collision
deviations f+_i - rest_i and J their e-weighted sums, both held in FP16; the temperature
populations in FP32 as g+_i - w~_i (T0 + R), with R = T - T0 of the node in FP16.  The
references come from the start state and are refreshed from the state every `refresh`
steps.  This module reproduces that storage around the oracle's FP64 step: after the
start state and after every step the stored values are rounded as the GPU rounds them,
so the emulated run carries the codec's error and nothing else.

The linear part of Eq. 32's equilibrium written out here is the codec's reference, a
storage choice of the GPU path, not part of the paper's method.
"""
import numpy as np

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], float)
EZ = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], float)
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
WT = np.array([0.6, 0.1, 0.1, 0.1, 0.1])


def round_f16(x):
    return np.asarray(x, np.float64).astype(np.float16).astype(np.float64)


def round_f32(x):
    return np.asarray(x, np.float64).astype(np.float32).astype(np.float64)


def round_bf16(x):
    """Round to nearest even in BF16 (via the FP32 bit pattern), back to float64."""
    a = np.asarray(x, np.float64).astype(np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


ROUND = {"f16": round_f16, "bf16": round_bf16}


class Emulated16:
    """An oracle State whose flow populations live in 16-bit storage against the flow
    reference, refreshed every `refresh` steps (as lbm_step does)."""

    def __init__(self, oracle, p, phi=None, storage="f16", refresh=1024, reference=True):
        self.o = oracle
        self.st = oracle.State(p, phi=phi)
        self.p = p
        self.rnd = ROUND[storage]
        self.refresh = refresh
        self.reference = reference
        c = oracle.derive(p)
        self.T0 = c["T0"]
        self.r = c["r0"] + np.arange(p.nr)
        self.rest_f = self.r[None, :, None] * W9[:, None, None] + (0.5 * EX * W9)[:, None, None]
        self.since = 0
        self._make_reference()
        self._store()

    def _make_reference(self):
        T = self.st.g.sum(0)
        self.R = round_f16(np.clip(T - self.T0, -60000, 60000))
        self.rest_g = WT[:, None, None] * (self.T0 + self.R)[None]
        if not self.reference:
            self.ref = np.zeros_like(self.st.f)
            return
        d = self.st.f - self.rest_f
        A, Jr, Jz = (round_f16(np.clip(x, -60000, 60000))
                     for x in (d.sum(0), np.tensordot(EX, d, 1), np.tensordot(EZ, d, 1)))
        eJ = EX[:, None, None] * Jr[None] + EZ[:, None, None] * Jz[None]
        self.ref = W9[:, None, None] * (A[None] + 3 * eJ)

    def _store(self):
        base = self.rest_f + self.ref
        self.st.f[:] = self.rnd(self.st.f - base) + base
        self.st.g[:] = round_f32(self.st.g - self.rest_g) + self.rest_g

    def stored_magnitude(self):
        """Largest |s_i| currently stored (the values the 16-bit format rounds)."""
        return float(np.abs(self.st.f - self.rest_f - self.ref).max())

    def run(self, nsteps):
        for _ in range(nsteps):
            if self.since >= self.refresh:
                self._make_reference()
                self._store()
                self.since = 0
            self.st.run(1, 1)
            self._store()
            self.since += 1
        return self

    def moments(self):
        return self.st.moments()

    def nusselt(self):
        return self.st.nusselt()
