"""FP64 CPU reference of the warm-start Fourier neural operator (test infrastructure
only; the library package never imports it).

Plain PyTorch CPU ops in float64 with autograd for gradients.  The spectral
convolution uses torch.fft.rfft2 / irfft2 with mode truncation (keep radial
wavenumbers 0..m-1 and nr-m..nr-1, axial 0..m-1), a per-mode complex channel
contraction, and zero elsewhere -- the textbook FNO layer (Li et al., ICLR 2021),
independent of the truncated-DFT-as-GEMM evaluation on the GPU.  Parameter layout:
matrices [in, out], spectral weights [2m, m, in, out, 2] (re, im).
"""
from __future__ import annotations

import torch
import torch.nn.functional as F


def _kr_index(nr: int, m: int):
    return list(range(m)) + list(range(nr - m, nr))


def forward(params: dict, x: torch.Tensor, modes: int, layers: int) -> torch.Tensor:
    """x [B, nr, nz, in] float64 -> [B, nr, nz, out]."""
    B, nr, nz, _ = x.shape
    idx = _kr_index(nr, modes)
    h = x @ params["P"] + params["p"]
    for l in range(layers):
        R = torch.complex(params[f"R{l}"][..., 0], params[f"R{l}"][..., 1])   # [2m, m, C, O]
        X = torch.fft.rfft2(h.permute(0, 3, 1, 2))                              # [B, C, nr, nz/2+1]
        Xs = X[:, :, idx, :modes]                                               # [B, C, 2m, m]
        Ys = torch.einsum("bcxy,xyco->boxy", Xs, R)
        Yf = torch.zeros(B, R.shape[-1], nr, nz // 2 + 1, dtype=X.dtype)
        Yf[:, :, idx, :modes] = Ys
        s = torch.fft.irfft2(Yf, s=(nr, nz)).permute(0, 2, 3, 1)
        pre = h @ params[f"W{l}"] + params[f"b{l}"] + s
        h = F.gelu(pre) if l < layers - 1 else pre
    q = F.gelu(h @ params["Q1"] + params["q1"])
    return q @ params["Q2"] + params["q2"]


def loss_and_grads(params_np: dict, x_np, t_np, modes: int, layers: int):
    """MSE loss and its gradient for every parameter, float64."""
    params = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in params_np.items()}
    x = torch.tensor(x_np, dtype=torch.float64)
    t = torch.tensor(t_np, dtype=torch.float64)
    y = forward(params, x, modes, layers)
    loss = ((y - t) ** 2).mean()
    loss.backward()
    return y.detach().numpy(), float(loss.detach()), {k: v.grad.numpy() for k, v in params.items()}
