"""Emulation of the 16-bit storage codec on the FP64 oracle (test helper).

The CUDA path stores each flow population as
    s_i = f+_i - (r w_i + e_ir w_i / 2) - D_i(Q),
    D_i(Q) = w_i [A + 3 e_i.J + (4.5 (e_i.J)^2 - 1.5 |J|^2) P / 1024],
rounded to FP16 (or BF16), with the per-node reference Q = (A, J_r, J_z, P) itself held in
FP16: A and J the sum and e-weighted sums of the node's post-collision deviations
f+_i - rest_i, P = 1024 / (r rho phi), rho = 1 + A / r.  Q is taken from the start state
and refreshed from the state every `refresh` steps.  Temperature populations are kept in
FP32 against w~_i T0.  This module reproduces that storage around the oracle's FP64 step:
after the start state and after every step the stored values are rounded as the GPU
rounds them, so the emulated run carries the codec's error and nothing else.

The equilibrium written out here is Eq. 32's deviation part; the codec is a storage
choice of the GPU path, not part of the paper's method.
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
        self.r = c["r0"] + np.arange(p.nr)
        self.rest_f = self.r[None, :, None] * W9[:, None, None] + (0.5 * EX * W9)[:, None, None]
        self.rest_g = (WT * c["T0"])[:, None, None]
        self.since = 0
        self.Q = None
        self._make_reference()
        self._store()

    def _make_reference(self):
        if not self.reference:
            self.ref = np.zeros_like(self.st.f)
            return
        d = self.st.f - self.rest_f
        A = d.sum(0)
        Jr = np.tensordot(EX, d, 1)
        Jz = np.tensordot(EZ, d, 1)
        r = self.r[:, None]
        rho = 1 + A / r
        with np.errstate(divide="ignore", invalid="ignore"):
            P = np.clip(np.nan_to_num(1024.0 / (r * rho * self.st.phi), nan=0.0, posinf=60000.0), 0, 60000)
        A, Jr, Jz = (np.clip(x, -60000, 60000) for x in (A, Jr, Jz))
        A, Jr, Jz, P = (round_f16(x) for x in (A, Jr, Jz, P))
        eJ = EX[:, None, None] * Jr[None] + EZ[:, None, None] * Jz[None]
        quad = 4.5 * eJ * eJ - 1.5 * (Jr * Jr + Jz * Jz)[None]
        self.ref = W9[:, None, None] * (A[None] + 3 * eJ + quad * (P / 1024.0)[None])
        self.Q = (A, Jr, Jz, P)

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
