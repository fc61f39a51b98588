"""Learned warm start: a 2-D Fourier neural operator (FNO) trained on steady fields of the
lattice Boltzmann solver, mapping the porosity field and the problem parameters to an
initial (u_r, u_z, T).  The paper has no counterpart; the solver always runs to
convergence from the proposed field, and the cold start remains the fallback.

Network (channels-last activations [batch, nr, nz, channels], FP32 in memory; every
contraction runs in the BF16 tensor-core GEMM of libfno.so with FP32 accumulation):
  lift      h = x P + p                        8 -> width
  layers    pre = h W + b + K(h);  h = GELU(pre)   (no GELU after the last layer)
  project   q = GELU(h Q1 + q1);  y = q Q2 + q2      width -> hidden -> 3
K is the truncated spectral convolution: rfft2, keep kr in [0, m) U [nr - m, nr) and
kz in [0, m), multiply by complex weights per mode, irfft2 -- evaluated as dense
GEMMs against truncated DFT matrices (z: real -> complex, r: complex), the per-mode
channel mixing, then the inverse pair, all in fno.h kernels.  Torch is used for device
buffers only.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
FNO_LIB_PATH = os.path.join(HERE, "libfno.so")

_lock = threading.Lock()
_lib = None
_vp = C.c_void_p
_i64 = C.c_int64
_SIGS = {
    "fno_gemm": [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_float, _vp, _i64, _i64, _vp, _i64, _i64, C.c_float,
                 _vp, _i64, _i64, C.c_int, _vp, _vp],
    "fno_gelu_fwd": [_vp, _vp, _i64, _vp],
    "fno_gelu_bwd": [_vp, _vp, _vp, _i64, C.c_int, _vp],
    "fno_mix_fwd": [_vp, _vp, _vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _vp],
    "fno_mix_bwd": [_vp, _vp, _vp, _vp, _vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _vp],
    "fno_colsum": [_vp, _i64, C.c_int, _i64, _vp, C.c_int, _vp],
    "fno_mse": [_vp, _vp, _vp, _vp, _i64, _vp],
    "fno_adam": [_vp, _vp, _vp, _vp, _i64, C.c_float, C.c_float, C.c_float, C.c_float, C.c_int, _vp],
    "fno_set_tensor_path": [C.c_int],
    "fno_tensor_path_status": [C.c_int],
    "fno_test_wait_timeout": [C.c_int],
    "fno_test_set_tc_error": [C.c_int],
}


def load():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(FNO_LIB_PATH):
                from . import build as _b

                _b.build()
            lib = C.CDLL(FNO_LIB_PATH)
            for name, args in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = C.c_int
                fn.argtypes = args
            lib.fno_last_error.restype = C.c_char_p
            _lib = lib
    return _lib


def _check(rc):
    if rc != 0:
        raise RuntimeError(f"fno error {rc}: {load().fno_last_error().decode()}")


def _p(t):
    return None if t is None else t.data_ptr()


def _stream():
    import torch

    return torch.cuda.current_stream().cuda_stream


# ---- C-named wrappers (argument marshalling only) ---------------------------
def fno_gemm(transA, transB, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, Cm, ldc, sC, batch=1, bias=None,
             a_off=0, b_off=0, c_off=0):
    """Pointers may be offset by a_off / b_off / c_off elements (views into a buffer)."""
    _check(load().fno_gemm(int(transA), int(transB), int(M), int(N), int(K), float(alpha), _p(A) + 4 * a_off,
                           int(lda), int(sA), _p(B) + 4 * b_off, int(ldb), int(sB), float(beta), _p(Cm) + 4 * c_off,
                           int(ldc), int(sC), int(batch), _p(bias), _stream()))


def fno_gelu_fwd(x, y):
    _check(load().fno_gelu_fwd(_p(x), _p(y), x.numel(), _stream()))


def fno_gelu_bwd(x, dy, dx, accumulate=False):
    _check(load().fno_gelu_bwd(_p(x), _p(dy), _p(dx), x.numel(), int(accumulate), _stream()))


def fno_mix_fwd(X, R, Y, batch, nkr, nkz, Cin, O):
    _check(load().fno_mix_fwd(_p(X), _p(R), _p(Y), batch, nkr, nkz, Cin, O, _stream()))


def fno_mix_bwd(X, R, dY, dX, dR, batch, nkr, nkz, Cin, O, accumulate=False):
    _check(load().fno_mix_bwd(_p(X), _p(R), _p(dY), _p(dX), _p(dR), batch, nkr, nkz, Cin, O, int(accumulate),
                              _stream()))


def fno_colsum(X, rows, N, ldx, out, accumulate=False):
    _check(load().fno_colsum(_p(X), int(rows), int(N), int(ldx), _p(out), int(accumulate), _stream()))


def fno_mse(y, t, dy, loss):
    _check(load().fno_mse(_p(y), _p(t), _p(dy), _p(loss), y.numel(), _stream()))


def fno_adam(w, g, m, v, lr, b1, b2, eps, step):
    _check(load().fno_adam(_p(w), _p(g), _p(m), _p(v), w.numel(), float(lr), float(b1), float(b2), float(eps),
                           int(step), _stream()))


def fno_set_tensor_path(path: int):
    """0: mma.sync m16n8k16; 1: tcgen05.mma with the accumulator in tensor memory."""
    _check(load().fno_set_tensor_path(int(path)))


def fno_tensor_path_status(clear: bool = True) -> int:
    return int(load().fno_tensor_path_status(int(clear)))


def fno_test_wait_timeout(enable: bool):
    """Test hook: tcgen05 GEMM CTAs replace their first commit wait by a short wait that
    runs out (see include/fno.h)."""
    _check(load().fno_test_wait_timeout(int(enable)))


def fno_test_set_tc_error(value: int):
    """Test hook: write the device error flag that fno_tensor_path_status reads."""
    _check(load().fno_test_set_tc_error(int(value)))


# ---- the operator -------------------------------------------------------------
PARAM_ORDER = ["P", "p"] + [f"{n}{l}" for l in range(4) for n in ("R", "W", "b")] + ["Q1", "q1", "Q2", "q2"]


def kr_values(nr: int, m: int):
    """Retained radial wavenumbers: 0..m-1 and nr-m..nr-1."""
    return list(range(m)) + list(range(nr - m, nr))


def init_params(nr, nz, width=32, modes=16, layers=4, in_ch=8, out_ch=3, hidden=128, seed=0):
    """FP32 parameters (numpy) in the layout of the kernels: matrices [in, out], spectral
    weights [nkr, nkz, in, out, 2]."""
    rng = np.random.default_rng(seed)
    nkr, nkz = 2 * modes, modes

    def lin(i, o):
        a = 1.0 / math.sqrt(i)
        return rng.uniform(-a, a, (i, o)).astype(np.float32), rng.uniform(-a, a, o).astype(np.float32)

    P = {}
    P["P"], P["p"] = lin(in_ch, width)
    for l in range(layers):
        P[f"R{l}"] = (rng.uniform(0, 1, (nkr, nkz, width, width, 2)) / (width * width)).astype(np.float32)
        P[f"W{l}"], P[f"b{l}"] = lin(width, width)
    P["Q1"], P["q1"] = lin(width, hidden)
    P["Q2"], P["q2"] = lin(hidden, out_ch)
    return P


def dft_matrices(nr, nz, modes):
    """Truncated DFT matrices (float64 numpy): Fz [nz, 2m] (cos | -sin) for the z
    transform, Cr, Sr [2m, nr] for the r transform, Gz [2m, nz] for the inverse z
    transform with the one-sided weights (1 for kz = 0, 2 otherwise) and 1/(nr nz)."""
    m = modes
    z = np.arange(nz)[:, None]
    kz = np.arange(m)[None, :]
    ang = 2 * np.pi * z * kz / nz
    Fz = np.concatenate([np.cos(ang), -np.sin(ang)], axis=1)
    kr = np.array(kr_values(nr, m))[:, None]
    r = np.arange(nr)[None, :]
    angr = 2 * np.pi * kr * r / nr
    Cr, Sr = np.cos(angr), np.sin(angr)
    w = np.where(np.arange(m) == 0, 1.0, 2.0)[:, None] / (nr * nz)
    angz = 2 * np.pi * np.arange(m)[:, None] * np.arange(nz)[None, :] / nz
    Gz = np.concatenate([w * np.cos(angz), -w * np.sin(angz)], axis=0)
    return Fz, Cr, Sr, Gz


class FNO2d:
    """Forward, backward and Adam on the GPU through libfno.so."""

    def __init__(self, nr, nz, width=32, modes=16, layers=4, in_ch=8, out_ch=3, hidden=128, seed=0, params=None):
        import torch

        self.nr, self.nz, self.width, self.m, self.L = nr, nz, width, modes, layers
        self.in_ch, self.out_ch, self.hidden = in_ch, out_ch, hidden
        self.nkr, self.nkz = 2 * modes, modes
        P = params if params is not None else init_params(nr, nz, width, modes, layers, in_ch, out_ch, hidden, seed)
        dev = "cuda"
        self.w = {k: torch.tensor(np.ascontiguousarray(v, dtype=np.float32), device=dev) for k, v in P.items()}
        self.g = {k: torch.zeros_like(v) for k, v in self.w.items()}
        self.adam_m = {k: torch.zeros_like(v) for k, v in self.w.items()}
        self.adam_v = {k: torch.zeros_like(v) for k, v in self.w.items()}
        self.step_count = 0
        Fz, Cr, Sr, Gz = dft_matrices(nr, nz, modes)
        f32 = lambda a: torch.tensor(np.ascontiguousarray(a, dtype=np.float32), device=dev)
        self.Fz, self.Cr, self.Sr, self.Gz = f32(Fz), f32(Cr), f32(Sr), f32(Gz)
        self.Ci, self.Si = f32(Cr.T), f32(Sr.T)
        self._buf = {}
        load()

    # -- buffers ------------------------------------------------------------
    def _b(self, name, shape):
        import torch

        t = self._buf.get(name)
        if t is None or tuple(t.shape) != tuple(shape):
            t = torch.empty(shape, dtype=torch.float32, device="cuda")
            self._buf[name] = t
        return t

    def params_numpy(self):
        return {k: v.detach().cpu().numpy() for k, v in self.w.items()}

    # -- spectral convolution pieces (B = batch) -------------------------------
    def _zdft(self, v, Z, B, Cc):
        """Z[b, r, kz2, c] = sum_z Fz[z, kz2] v[b, r, z, c]."""
        nz, m2 = self.nz, 2 * self.m
        fno_gemm(1, 0, m2, Cc, nz, 1.0, self.Fz, m2, 0, v, Cc, nz * Cc, 0.0, Z, Cc, m2 * Cc, B * self.nr)

    def _zdft_T(self, dZ, dv, B, Cc):
        """dv[b, r, z, c] += sum_kz2 Fz[z, kz2] dZ[b, r, kz2, c]."""
        nz, m2 = self.nz, 2 * self.m
        fno_gemm(0, 0, nz, Cc, m2, 1.0, self.Fz, m2, 0, dZ, Cc, m2 * Cc, 1.0, dv, Cc, nz * Cc, B * self.nr)

    def _rdft(self, Z, W, B, Cc, M1, M2, rows_in, rows_out):
        """W_re = M1 Z_re + M2 Z_im, W_im = M1 Z_im - M2 Z_re, per batch; Z [rows_in, 2 m C],
        W [rows_out, 2 m C]; M1, M2 [rows_out, rows_in]."""
        mc = self.m * Cc
        sz, sw = rows_in * 2 * mc, rows_out * 2 * mc
        K = rows_in
        fno_gemm(0, 0, rows_out, mc, K, 1.0, M1, K, 0, Z, 2 * mc, sz, 0.0, W, 2 * mc, sw, B)
        fno_gemm(0, 0, rows_out, mc, K, 1.0, M2, K, 0, Z, 2 * mc, sz, 1.0, W, 2 * mc, sw, B, b_off=mc)
        fno_gemm(0, 0, rows_out, mc, K, 1.0, M1, K, 0, Z, 2 * mc, sz, 0.0, W, 2 * mc, sw, B, b_off=mc, c_off=mc)
        fno_gemm(0, 0, rows_out, mc, K, -1.0, M2, K, 0, Z, 2 * mc, sz, 1.0, W, 2 * mc, sw, B, c_off=mc)

    def _irdft(self, Y, V, B, Cc, M1, M2, rows_in, rows_out):
        """V_re = M1 Y_re - M2 Y_im, V_im = M2 Y_re + M1 Y_im."""
        mc = self.m * Cc
        sy, sv = rows_in * 2 * mc, rows_out * 2 * mc
        K = rows_in
        fno_gemm(0, 0, rows_out, mc, K, 1.0, M1, K, 0, Y, 2 * mc, sy, 0.0, V, 2 * mc, sv, B)
        fno_gemm(0, 0, rows_out, mc, K, -1.0, M2, K, 0, Y, 2 * mc, sy, 1.0, V, 2 * mc, sv, B, b_off=mc)
        fno_gemm(0, 0, rows_out, mc, K, 1.0, M2, K, 0, Y, 2 * mc, sy, 0.0, V, 2 * mc, sv, B, c_off=mc)
        fno_gemm(0, 0, rows_out, mc, K, 1.0, M1, K, 0, Y, 2 * mc, sy, 1.0, V, 2 * mc, sv, B, b_off=mc, c_off=mc)

    def _izdft(self, V, out, B, Cc):
        """out[b, r, z, c] += sum_kz2 Gz[kz2, z] V[b, r, kz2, c]."""
        nz, m2 = self.nz, 2 * self.m
        fno_gemm(1, 0, nz, Cc, m2, 1.0, self.Gz, nz, 0, V, Cc, m2 * Cc, 1.0, out, Cc, nz * Cc, B * self.nr)

    def _izdft_T(self, dout, dV, B, Cc):
        """dV[b, r, kz2, c] = sum_z Gz[kz2, z] dout[b, r, z, c]."""
        nz, m2 = self.nz, 2 * self.m
        fno_gemm(0, 0, m2, Cc, nz, 1.0, self.Gz, nz, 0, dout, Cc, nz * Cc, 0.0, dV, Cc, m2 * Cc, B * self.nr)

    def _wgrad(self, X, dY, K, Min, Nout, dW):
        """dW [Min, Nout] = X^T dY with X [K, Min], dY [K, Nout]; split over K into up to 512
        slices of >= 512 rows (one CTA each: 64 slices left most of the 152 SMs idle), the
        slices summed by fno_colsum."""
        S = max(1, min(512, K // 512))
        while K % S:
            S -= 1
        tmp = self._b(f"wg_{Min}_{Nout}_{S}", (S, Min, Nout))
        ks = K // S
        fno_gemm(1, 0, Min, Nout, ks, 1.0, X, Min, ks * Min, dY, Nout, ks * Nout, 0.0, tmp, Nout, Min * Nout, S)
        fno_colsum(tmp, S, Min * Nout, Min * Nout, dW, accumulate=True)

    # -- forward / backward -------------------------------------------------
    def forward(self, x, train=False):
        """x: [B, nr, nz, in_ch] float32 CUDA tensor -> [B, nr, nz, out_ch]."""
        B = x.shape[0]
        px = B * self.nr * self.nz
        Wd, m = self.width, self.m
        w = self.w
        h = self._b("h0", (B, self.nr, self.nz, Wd))
        fno_gemm(0, 0, px, Wd, self.in_ch, 1.0, x, self.in_ch, 0, w["P"], Wd, 0, 0.0, h, Wd, 0, 1, bias=w["p"])
        self._x = x
        self._hs = [h]
        for l in range(self.L):
            Z = self._b(f"Z{l}", (B, self.nr, 2 * m, Wd))
            Wm = self._b(f"Wm{l}", (B, self.nkr, 2 * m, Wd))
            Y = self._b(f"Y{l}", (B, self.nkr, 2 * m, Wd))
            V = self._b(f"V{l}", (B, self.nr, 2 * m, Wd))
            pre = self._b(f"pre{l}", (B, self.nr, self.nz, Wd))
            self._zdft(h, Z, B, Wd)
            self._rdft(Z, Wm, B, Wd, self.Cr, self.Sr, self.nr, self.nkr)
            fno_mix_fwd(Wm, w[f"R{l}"], Y, B, self.nkr, self.nkz, Wd, Wd)
            self._irdft(Y, V, B, Wd, self.Ci, self.Si, self.nkr, self.nr)
            fno_gemm(0, 0, px, Wd, Wd, 1.0, h, Wd, 0, w[f"W{l}"], Wd, 0, 0.0, pre, Wd, 0, 1, bias=w[f"b{l}"])
            self._izdft(V, pre, B, Wd)
            if l < self.L - 1:
                h = self._b(f"h{l + 1}", (B, self.nr, self.nz, Wd))
                fno_gelu_fwd(pre, h)
            else:
                h = pre
            self._hs.append(h)
        qp = self._b("qpre", (B, self.nr, self.nz, self.hidden))
        q = self._b("q", (B, self.nr, self.nz, self.hidden))
        y = self._b("y", (B, self.nr, self.nz, self.out_ch))
        fno_gemm(0, 0, px, self.hidden, Wd, 1.0, h, Wd, 0, w["Q1"], self.hidden, 0, 0.0, qp, self.hidden, 0, 1,
                 bias=w["q1"])
        fno_gelu_fwd(qp, q)
        fno_gemm(0, 0, px, self.out_ch, self.hidden, 1.0, q, self.hidden, 0, w["Q2"], self.out_ch, 0, 0.0, y,
                 self.out_ch, 0, 1, bias=w["q2"])
        return y

    def zero_grad(self):
        for g in self.g.values():
            g.zero_()

    def backward(self, dy):
        """Accumulate parameter gradients for dL/dy of the last forward."""
        B = dy.shape[0]
        px = B * self.nr * self.nz
        Wd, m, hid = self.width, self.m, self.hidden
        w, g = self.w, self.g
        q, qp = self._buf["q"], self._buf["qpre"]
        h = self._hs[-1]
        # projection
        self._wgrad(q, dy, px, hid, self.out_ch, g["Q2"])
        fno_colsum(dy, px, self.out_ch, self.out_ch, g["q2"], accumulate=True)
        dq = self._b("dq", (B, self.nr, self.nz, hid))
        fno_gemm(0, 1, px, hid, self.out_ch, 1.0, dy, self.out_ch, 0, w["Q2"], self.out_ch, 0, 0.0, dq, hid, 0, 1)
        fno_gelu_bwd(qp, dq, dq)
        self._wgrad(h, dq, px, Wd, hid, g["Q1"])
        fno_colsum(dq, px, hid, hid, g["q1"], accumulate=True)
        dh = self._b("dh_a", (B, self.nr, self.nz, Wd))
        fno_gemm(0, 1, px, Wd, hid, 1.0, dq, hid, 0, w["Q1"], hid, 0, 0.0, dh, Wd, 0, 1)
        other = "dh_b"
        for l in reversed(range(self.L)):
            pre = self._buf[f"pre{l}"]
            hin = self._hs[l]
            dpre = self._b("dpre", (B, self.nr, self.nz, Wd))
            if l < self.L - 1:
                fno_gelu_bwd(pre, dh, dpre)
            else:
                dpre.copy_(dh)
            # pointwise path
            self._wgrad(hin, dpre, px, Wd, Wd, g[f"W{l}"])
            fno_colsum(dpre, px, Wd, Wd, g[f"b{l}"], accumulate=True)
            dhin = self._b(other, (B, self.nr, self.nz, Wd))
            fno_gemm(0, 1, px, Wd, Wd, 1.0, dpre, Wd, 0, w[f"W{l}"], Wd, 0, 0.0, dhin, Wd, 0, 1)
            # spectral path
            dV = self._b("dV", (B, self.nr, 2 * m, Wd))
            dY = self._b("dY", (B, self.nkr, 2 * m, Wd))
            dWm = self._b("dWm", (B, self.nkr, 2 * m, Wd))
            dZ = self._b("dZ", (B, self.nr, 2 * m, Wd))
            self._izdft_T(dpre, dV, B, Wd)
            # V = irdft(Y) with (Ci, Si): dY_re = Cr dV_re + Sr dV_im, dY_im = Cr dV_im - Sr dV_re
            self._rdft(dV, dY, B, Wd, self.Cr, self.Sr, self.nr, self.nkr)
            fno_mix_bwd(self._buf[f"Wm{l}"], w[f"R{l}"], dY, dWm, g[f"R{l}"], B, self.nkr, self.nkz, Wd, Wd,
                        accumulate=True)
            # Wm = rdft(Z) with (Cr, Sr): dZ_re = Ci dW_re - Si dW_im, dZ_im = Si dW_re + Ci dW_im
            self._irdft(dWm, dZ, B, Wd, self.Ci, self.Si, self.nkr, self.nr)
            self._zdft_T(dZ, dhin, B, Wd)
            dh, other = dhin, ("dh_a" if other == "dh_b" else "dh_b")
        # lift
        self._wgrad(self._x, dh, px, self.in_ch, Wd, g["P"])
        fno_colsum(dh, px, Wd, Wd, g["p"], accumulate=True)

    def loss_and_grad(self, x, t):
        """MSE loss (device double, accumulated) and parameter gradients for one batch."""
        import torch

        y = self.forward(x, train=True)
        dy = self._b("dy", tuple(y.shape))
        lbuf = self._buf.get("lossd")
        if lbuf is None:
            lbuf = torch.zeros(1, dtype=torch.float64, device="cuda")
            self._buf["lossd"] = lbuf
        lbuf.zero_()
        fno_mse(y, t, dy, lbuf)
        self.backward(dy)
        return lbuf

    def adam_step(self, lr, b1=0.9, b2=0.999, eps=1e-8):
        self.step_count += 1
        for k in self.w:
            fno_adam(self.w[k], self.g[k], self.adam_m[k], self.adam_v[k], lr, b1, b2, eps, self.step_count)


# ---- fused tensor-core network (libfnonet.so, include/fno_net.h) --------------------
FNO_NET_LIB_PATH = os.path.join(HERE, "libfnonet.so")
_net_lib = None
_NET_SIGS = {
    "fno_net_supported": [_vp],
    "fno_net_pack": [_vp, _i64, _i64, C.c_int, C.c_int, _vp, C.c_int, C.c_int, _vp],
    "fno_net_pack_many": [_vp, C.c_int, _vp],
    "fno_net_fwd": [C.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "fno_net_proj": [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "fno_net_bwd": [C.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "fno_net_r2k": [_vp, _vp, _vp, _vp, _vp],
    "fno_net_k2r": [_vp, _vp, _vp, _vp, _vp],
    "fno_net_mix_fwd": [_vp, _vp, _vp, _vp, _vp],
    "fno_net_mix_bwd": [_vp, _vp, _vp, _vp, _vp, _vp, C.c_int, _vp],
    "fno_net_status": [C.c_int],
}


class fno_net_dims(C.Structure):
    _fields_ = [(n, C.c_int32) for n in ("batch", "nr", "nz", "width", "modes", "hidden", "in_ch", "out_ch")]


class fno_net_pack_job(C.Structure):
    _fields_ = [("src", _vp), ("so", _i64), ("si", _i64), ("O", C.c_int32), ("I", C.c_int32),
                ("Opad", C.c_int32), ("Ipad", C.c_int32), ("dst", _vp)]


def load_net():
    global _net_lib
    with _lock:
        if _net_lib is None:
            if not os.path.exists(FNO_NET_LIB_PATH):
                from . import build as _b

                _b.build()
            lib = C.CDLL(FNO_NET_LIB_PATH)
            for name, args in _NET_SIGS.items():
                fn = getattr(lib, name)
                fn.restype = C.c_int
                fn.argtypes = args
            lib.fno_net_last_error.restype = C.c_char_p
            _net_lib = lib
    return _net_lib


def _ncheck(rc):
    if rc != 0:
        raise RuntimeError(f"fno_net error {rc}: {load_net().fno_net_last_error().decode()}")


def net_supported(batch, nr, nz, width, modes, hidden, in_ch, out_ch) -> bool:
    d = fno_net_dims(batch, nr, nz, width, modes, hidden, in_ch, out_ch)
    return bool(load_net().fno_net_supported(C.byref(d)))


def fno_net_status(clear: bool = True) -> int:
    return int(load_net().fno_net_status(int(clear)))


class FusedFNO2d:
    """The operator of FNO2d on the fused tcgen05 kernels of libfnonet.so: BF16
    activations, FP32 master weights and Adam state (same layouts as FNO2d, views into one
    flat buffer each, so that one Adam launch updates them all), BF16 operand images of the
    weights refreshed by one launch after every update.  Torch provides device buffers
    only; every step runs in libfnonet.so (and Adam in libfno.so)."""

    def __init__(self, nr, nz, width=32, modes=16, layers=4, in_ch=8, out_ch=3, hidden=128, seed=0, params=None):
        import torch

        self.nr, self.nz, self.width, self.m, self.L = nr, nz, width, modes, layers
        self.in_ch, self.out_ch, self.hidden = in_ch, out_ch, hidden
        self.nkr, self.nkz = 2 * modes, modes
        if not net_supported(1, nr, nz, width, modes, hidden, in_ch, out_ch):
            raise ValueError("sizes outside the fused kernels' range (include/fno_net.h)")
        P = params if params is not None else init_params(nr, nz, width, modes, layers, in_ch, out_ch, hidden, seed)
        dev = "cuda"
        total = sum(int(np.prod(v.shape)) for v in P.values())
        self._flat = {n: torch.zeros(total, dtype=torch.float32, device=dev) for n in ("w", "g", "m", "v")}
        self.w, self.g, self.adam_m, self.adam_v = {}, {}, {}, {}
        off = 0
        for k, v in P.items():
            n = int(np.prod(v.shape))
            for name, d in (("w", self.w), ("g", self.g), ("m", self.adam_m), ("v", self.adam_v)):
                d[k] = self._flat[name][off:off + n].view(v.shape)
            self.w[k].copy_(torch.tensor(np.ascontiguousarray(v, dtype=np.float32), device=dev))
            off += n
        self.step_count = 0
        load()
        load_net()
        Fz, Cr, Sr, Gz = dft_matrices(nr, nz, modes)
        f32 = lambda a: torch.tensor(np.ascontiguousarray(a, dtype=np.float32), device=dev)
        F2 = np.block([[Cr, Sr], [-Sr, Cr]])                 # [W_re; W_im] = F2 [Z_re; Z_im]
        F2i = np.block([[Cr.T, -Sr.T], [Sr.T, Cr.T]])        # [V_re; V_im] = F2i [Y_re; Y_im]
        m2 = 2 * modes
        self.img = {}
        self.img["fz"] = self._pack(f32(Fz), m2, 1, nz, m2, nz, m2)
        self.img["gzt"] = self._pack(f32(Gz), 1, nz, nz, m2, nz, m2)
        self.img["f2"] = self._pack(f32(F2), 2 * nr, 1, 2 * m2, 2 * nr, 128, 2 * nr)
        self.img["f2i"] = self._pack(f32(F2i), 2 * m2, 1, 2 * nr, 2 * m2, 2 * nr, 2 * m2)
        self._dirty = True
        self._buf = {}
        self._parts = None

    # -- helpers ------------------------------------------------------------------
    def _pack(self, src, so, si, O, I, Opad, Ipad, out=None):
        import torch

        if out is None:
            out = torch.empty(Opad * Ipad, dtype=torch.bfloat16, device="cuda")
        _ncheck(load_net().fno_net_pack(src.data_ptr(), so, si, O, I, out.data_ptr(), Opad, Ipad, _stream()))
        return out

    def _pack_jobs(self):
        """The weight images as one table of pack jobs (built once: the weights are views
        into the flat buffer and the images never move)."""
        import torch

        C, H, CI, CO, w, im = self.width, self.hidden, self.in_ch, self.out_ch, self.w, self.img
        spec = [("P", w["P"], 1, C, C, CI, C, 16)]                                   # P^T: (c, ci)
        for l in range(self.L):
            spec.append((f"Wf{l}", w[f"W{l}"], 1, C, C, C, C, C))                   # W^T: (c_out, c_in)
            spec.append((f"Wn{l}", w[f"W{l}"], C, 1, C, C, C, C))                   # W: (c_in, c_out)
        spec += [("q1w", w["Q1"], 1, H, H, C, H, C), ("q1n", w["Q1"], H, 1, C, H, C, H),   # Q1^T, Q1
                 ("q2w", w["Q2"], 1, CO, CO, H, 16, H), ("q2n", w["Q2"], CO, 1, H, CO, H, 16)]   # Q2^T, Q2
        jobs = (fno_net_pack_job * len(spec))()
        for j, (name, src, so, si, O, I, Op, Ip) in enumerate(spec):
            im[name] = torch.empty(Op * Ip, dtype=torch.bfloat16, device="cuda")
            jobs[j] = fno_net_pack_job(src.data_ptr(), so, si, O, I, Op, Ip, im[name].data_ptr())
        return jobs

    def _refresh_images(self):
        """BF16 operand images of the current FP32 weights (after every update)."""
        if not self._dirty:
            return
        if getattr(self, "_jobs", None) is None:
            self._jobs = self._pack_jobs()
        _ncheck(load_net().fno_net_pack_many(self._jobs, len(self._jobs), _stream()))
        self._dirty = False

    def _dims(self, B):
        return fno_net_dims(B, self.nr, self.nz, self.width, self.m, self.hidden, self.in_ch, self.out_ch)

    def _b(self, name, shape, dtype=None):
        import torch

        dtype = dtype or torch.bfloat16
        t = self._buf.get(name)
        if t is None or tuple(t.shape) != tuple(shape) or t.dtype != dtype:
            t = torch.empty(shape, dtype=dtype, device="cuda")
            self._buf[name] = t
        return t

    def params_numpy(self):
        return {k: v.detach().cpu().numpy() for k, v in self.w.items()}

    # -- forward ------------------------------------------------------------------
    def forward(self, x, train=False, t=None):
        """x: [B, nr, nz, in_ch] float32 CUDA tensor -> y [B, nr, nz, out_ch] (float32).
        With t (targets) also the loss and the projection's backward (see loss_and_grad)."""
        import torch

        lib = load_net()
        B = x.shape[0]
        d = self._dims(B)
        dp = C.byref(d)
        nr, nz, Cw, M, L = self.nr, self.nz, self.width, self.m, self.L
        s = _stream()
        self._refresh_images()
        im, w = self.img, self.w
        x = x.contiguous()
        act = (B, nr, nz, Cw)
        zs = (B, M, 2, nr, Cw)
        ks = (M, 2 * M, 2, B, Cw)
        h = [self._b(f"h{l}", act) for l in range(L + 1)]
        Z = [self._b(f"Z{l}", zs) for l in range(L)]
        V = [self._b(f"V{l}", zs) for l in range(L)]
        Wk = [self._b(f"Wk{l}", ks, torch.float32) for l in range(L)]
        Yk = self._b("Yk", ks, torch.float32)
        _ncheck(lib.fno_net_fwd(0, dp, x.data_ptr(), None, im["P"].data_ptr(), w["p"].data_ptr(), None,
                                im["fz"].data_ptr(), None, h[0].data_ptr(), None, Z[0].data_ptr(), s))
        for l in range(L):
            _ncheck(lib.fno_net_r2k(dp, Z[l].data_ptr(), im["f2"].data_ptr(), Wk[l].data_ptr(), s))
            _ncheck(lib.fno_net_mix_fwd(dp, Wk[l].data_ptr(), w[f"R{l}"].data_ptr(), Yk.data_ptr(), s))
            _ncheck(lib.fno_net_k2r(dp, Yk.data_ptr(), im["f2i"].data_ptr(), V[l].data_ptr(), s))
            if l < L - 1:
                pre = self._b(f"pre{l}", act)
                _ncheck(lib.fno_net_fwd(1, dp, None, h[l].data_ptr(), im[f"Wf{l}"].data_ptr(), w[f"b{l}"].data_ptr(),
                                        im["gzt"].data_ptr(), im["fz"].data_ptr(), V[l].data_ptr(), pre.data_ptr(),
                                        h[l + 1].data_ptr(), Z[l + 1].data_ptr(), s))
            else:
                _ncheck(lib.fno_net_fwd(2, dp, None, h[l].data_ptr(), im[f"Wf{l}"].data_ptr(), w[f"b{l}"].data_ptr(),
                                        im["gzt"].data_ptr(), None, V[l].data_ptr(), h[L].data_ptr(), None, None, s))
        y = self._b("y", (B, nr, nz, self.out_ch), torch.float32)
        if t is None:
            _ncheck(lib.fno_net_proj(dp, h[L].data_ptr(), im["q1w"].data_ptr(), None, w["q1"].data_ptr(),
                                     im["q2w"].data_ptr(), None, w["q2"].data_ptr(), None, y.data_ptr(), None, None,
                                     None, None, None, None, s))
            return y
        dhL = self._b("dhL", act)
        lbuf = self._b("lossd", (1,), torch.float64)
        lbuf.zero_()
        g = self.g
        _ncheck(lib.fno_net_proj(dp, h[L].data_ptr(), im["q1w"].data_ptr(), im["q1n"].data_ptr(), w["q1"].data_ptr(),
                                 im["q2w"].data_ptr(), im["q2n"].data_ptr(), w["q2"].data_ptr(), t.data_ptr(),
                                 y.data_ptr(), dhL.data_ptr(), lbuf.data_ptr(), g["Q1"].data_ptr(), g["q1"].data_ptr(),
                                 g["Q2"].data_ptr(), g["q2"].data_ptr(), s))
        return y

    def zero_grad(self):
        self._flat["g"].zero_()

    def _backward_layers(self, x, B):
        import torch

        lib = load_net()
        d = self._dims(B)
        dp = C.byref(d)
        nr, nz, Cw, M, L = self.nr, self.nz, self.width, self.m, self.L
        s = _stream()
        im, w, g = self.img, self.w, self.g
        act = (B, nr, nz, Cw)
        zs = (B, M, 2, nr, Cw)
        ks = (M, 2 * M, 2, B, Cw)
        dV = self._b("dV", zs)
        dZ = self._b("dZ", zs)
        dYk = self._b("dYk", ks, torch.float32)
        dWk = self._b("dWk", ks, torch.float32)
        dpre = [self._b("dpre_a", act), self._b("dpre_b", act)]
        h = [self._buf[f"h{l}"] for l in range(L + 1)]
        cur = self._buf["dhL"]   # dL/dpre_{L-1} (h_L = pre_{L-1})
        _ncheck(lib.fno_net_bwd(0, dp, cur.data_ptr(), None, None, None, None, h[L - 1].data_ptr(), None,
                                im["gzt"].data_ptr(), None, dV.data_ptr(), g[f"W{L - 1}"].data_ptr(),
                                g[f"b{L - 1}"].data_ptr(), s))
        for l in range(L - 1, -1, -1):
            _ncheck(lib.fno_net_r2k(dp, dV.data_ptr(), im["f2"].data_ptr(), dYk.data_ptr(), s))
            _ncheck(lib.fno_net_mix_bwd(dp, self._buf[f"Wk{l}"].data_ptr(), w[f"R{l}"].data_ptr(), dYk.data_ptr(),
                                        dWk.data_ptr(), g[f"R{l}"].data_ptr(), 1, s))
            _ncheck(lib.fno_net_k2r(dp, dWk.data_ptr(), im["f2i"].data_ptr(), dZ.data_ptr(), s))
            if l > 0:
                nxt = dpre[l % 2]
                _ncheck(lib.fno_net_bwd(1, dp, cur.data_ptr(), dZ.data_ptr(), im[f"Wn{l}"].data_ptr(),
                                        im["fz"].data_ptr(), self._buf[f"pre{l - 1}"].data_ptr(), h[l - 1].data_ptr(),
                                        None, im["gzt"].data_ptr(), nxt.data_ptr(), dV.data_ptr(),
                                        g[f"W{l - 1}"].data_ptr(), g[f"b{l - 1}"].data_ptr(), s))
                cur = nxt
            else:
                _ncheck(lib.fno_net_bwd(2, dp, cur.data_ptr(), dZ.data_ptr(), im["Wn0"].data_ptr(),
                                        im["fz"].data_ptr(), None, None, x.data_ptr(), None, None, None,
                                        g["P"].data_ptr(), g["p"].data_ptr(), s))

    def loss_and_grad(self, x, t):
        """MSE loss (device double) and parameter gradients (accumulated into self.g) of
        one batch."""
        x = x.contiguous()
        t = t.contiguous()
        self.forward(x, train=True, t=t)
        self._backward_layers(x, x.shape[0])
        return self._buf["lossd"]

    def adam_step(self, lr, b1=0.9, b2=0.999, eps=1e-8):
        self.step_count += 1
        f = self._flat
        fno_adam(f["w"], f["g"], f["m"], f["v"], lr, b1, b2, eps, self.step_count)
        self._dirty = True


def make_fno(nr, nz, width=32, modes=16, layers=4, in_ch=8, out_ch=3, hidden=128, seed=0, params=None, fused=None):
    """The warm-start network: the fused tcgen05 kernels where they cover the sizes (the
    default), else FNO2d on the batched GEMM."""
    if fused is None:
        fused = net_supported(1, nr, nz, width, modes, hidden, in_ch, out_ch)
    cls = FusedFNO2d if fused else FNO2d
    return cls(nr, nz, width, modes, layers, in_ch, out_ch, hidden, seed, params)
