"""Warm-start network: the GPU kernels (BF16 tensor-core GEMM, FP32 accumulation)
against FP64 references.  GEMM against an FP64 matmul; the whole operator's output
and every parameter gradient against the FP64 autograd oracle (oracle/fno_oracle.py),
which evaluates the spectral layers with FFTs instead of DFT GEMMs."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fno():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1409_5929_gb300 import build, fno as F

    build.build()
    F.load()
    return F


def _bf16_tol(a, b):
    """BF16 operands (8-bit significand): relative rounding 2^-9 per operand."""
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("path", [0, 1])
@pytest.mark.parametrize("ta,tb", [(0, 0), (0, 1), (1, 0), (1, 1)])
@pytest.mark.parametrize("shape", [(1, 64, 64, 32), (3, 77, 45, 130), (2, 300, 3, 8), (1, 5, 200, 513),
                                   (1, 1000, 300, 96), (4, 640, 32, 256), (2, 260, 48, 20)])
@pytest.mark.parametrize("beta", [2.0, 0.0])
def test_gemm_against_fp64(fno, path, ta, tb, shape, beta):
    """Both tensor-core paths: mma.sync (0) and tcgen05 with a tensor-memory accumulator (1);
    aligned and ragged shapes, several K chunks, beta = 0 (vector stores) and beta != 0."""
    import torch

    fno.fno_set_tensor_path(path)
    batch, M, N, K = shape
    rng = np.random.default_rng(M * 7 + N)
    A = rng.normal(size=(batch, K, M) if ta else (batch, M, K)).astype(np.float32)
    B = rng.normal(size=(batch, N, K) if tb else (batch, K, N)).astype(np.float32)
    C0 = rng.normal(size=(batch, M, N)).astype(np.float32)
    bias = rng.normal(size=N).astype(np.float32)
    Ad, Bd, Cd, bd = (torch.tensor(v, device="cuda") for v in (A, B, C0, bias))
    lda = M if ta else K
    ldb = K if tb else N
    fno.fno_gemm(ta, tb, M, N, K, 0.5, Ad, lda, A[0].size, Bd, ldb, B[0].size, beta, Cd, N, M * N, batch, bias=bd)
    torch.cuda.synchronize()
    opA = np.swapaxes(A, 1, 2) if ta else A
    opB = np.swapaxes(B, 1, 2) if tb else B
    ref = 0.5 * np.einsum("bmk,bkn->bmn", opA.astype(np.float64), opB.astype(np.float64)) + beta * C0 + bias
    # bound: |sum a b| error <= K * 2 * 2^-9 * max|a b| per element; L2-relative check
    got = Cd.cpu().numpy()
    fno.fno_set_tensor_path(0)
    assert fno.fno_tensor_path_status(True) == 0
    assert _bf16_tol(got, ref) < 2e-2


@pytest.mark.parametrize("path", [0, 1])
def test_operator_and_gradients_against_fp64_oracle(fno, path):
    import torch

    from oracle import fno_oracle

    nr, nz, width, modes, layers, hidden = 16, 32, 8, 4, 4, 16
    P = fno.init_params(nr, nz, width, modes, layers, in_ch=8, out_ch=3, hidden=hidden, seed=3)
    rng = np.random.default_rng(5)
    x = rng.normal(size=(2, nr, nz, 8)).astype(np.float32)
    t = rng.normal(size=(2, nr, nz, 3)).astype(np.float32)
    # larger spectral weights so the spectral path carries a visible share of the output
    for l in range(layers):
        P[f"R{l}"] = (P[f"R{l}"] * width).astype(np.float32)
    fno.fno_set_tensor_path(path)
    net = fno.FNO2d(nr, nz, width, modes, layers, 8, 3, hidden, params=P)
    xd, td = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
    net.zero_grad()
    loss = net.loss_and_grad(xd, td)
    torch.cuda.synchronize()
    y_ref, loss_ref, g_ref = fno_oracle.loss_and_grads(P, x, t, modes, layers)
    y = net._buf["y"].cpu().numpy()
    assert _bf16_tol(y, y_ref) < 2e-2
    assert abs(float(loss.item()) - loss_ref) < 2e-2 * loss_ref
    fno.fno_set_tensor_path(0)
    assert fno.fno_tensor_path_status(True) == 0
    for k in P:
        g = net.g[k].cpu().numpy()
        assert _bf16_tol(g, g_ref[k]) < 5e-2, (k, _bf16_tol(g, g_ref[k]))


def test_adam_step_matches_formula(fno):
    import torch

    rng = np.random.default_rng(1)
    w, g = rng.normal(size=100).astype(np.float32), rng.normal(size=100).astype(np.float32)
    m, v = np.zeros(100, np.float32), np.zeros(100, np.float32)
    wd, gd, md, vd = (torch.tensor(a, device="cuda") for a in (w, g, m, v))
    for step in (1, 2):
        fno.fno_adam(wd, gd, md, vd, 1e-2, 0.9, 0.999, 1e-8, step)
        m = 0.9 * m + 0.1 * g
        v = 0.999 * v + 0.001 * g * g
        w = w - 1e-2 * (m / (1 - 0.9 ** step)) / (np.sqrt(v / (1 - 0.999 ** step)) + 1e-8)
    torch.cuda.synchronize()
    assert np.allclose(wd.cpu().numpy(), w, rtol=1e-5, atol=1e-6)


# ---- fused tcgen05 network (libfnonet.so) -------------------------------------------
def _fused_case(fno, nr, nz, width, modes, batch, seed=3, scale_r=True):
    layers, hidden = 4, 128
    P = fno.init_params(nr, nz, width, modes, layers, in_ch=8, out_ch=3, hidden=hidden, seed=seed)
    if scale_r:   # larger spectral weights so the spectral path carries a visible share
        for l in range(layers):
            P[f"R{l}"] = (P[f"R{l}"] * width).astype(np.float32)
    rng = np.random.default_rng(seed + 2)
    x = rng.normal(size=(batch, nr, nz, 8)).astype(np.float32)
    t = rng.normal(size=(batch, nr, nz, 3)).astype(np.float32)
    return P, x, t, layers, hidden


@pytest.mark.parametrize("width,modes", [(32, 8), (32, 16), (64, 8)])
def test_fused_operator_and_gradients_against_fp64_oracle(fno, width, modes):
    """The fused path (BF16 activations, tcgen05 MMAs, MN-major operand images) against
    the FP64 autograd oracle: output, loss and every parameter gradient on a 64 x 128 grid
    (two row tiles of the inverse r transform, one z tile), batch 2."""
    import torch

    from oracle import fno_oracle

    nr, nz = 64, 128
    P, x, t, layers, hidden = _fused_case(fno, nr, nz, width, modes, 2)
    net = fno.FusedFNO2d(nr, nz, width, modes, layers, 8, 3, hidden, params=P)
    xd, td = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
    net.zero_grad()
    loss = net.loss_and_grad(xd, td)
    torch.cuda.synchronize()
    assert fno.fno_net_status(True) == 0
    y_ref, loss_ref, g_ref = fno_oracle.loss_and_grads(P, x, t, modes, layers)
    y = net._buf["y"].cpu().numpy()
    print("y", _bf16_tol(y, y_ref), "loss", float(loss.item()), loss_ref)
    assert _bf16_tol(y, y_ref) < 2e-2
    assert abs(float(loss.item()) - loss_ref) < 2e-2 * loss_ref
    errs = {k: _bf16_tol(net.g[k].cpu().numpy(), g_ref[k]) for k in P}
    print("grad rel L2", errs)
    for k, e in errs.items():
        assert e < 5e-2, (k, e)
    # the forward alone (no targets) gives the same output
    y2 = net.forward(xd).cpu().numpy()
    assert np.array_equal(y2, y)


def test_fused_matches_gemm_path_at_training_size(fno):
    """128 x 256, width 32, 16 modes (the warm start's training size), batch 2: the fused
    path's loss and gradients against FNO2d on the batched GEMM (FP32 activations, BF16
    operands) -- the two differ by BF16 activation rounding only."""
    import torch

    nr, nz, width, modes = 128, 256, 32, 16
    P, x, t, layers, hidden = _fused_case(fno, nr, nz, width, modes, 2, seed=7)
    xd, td = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
    fno.fno_set_tensor_path(0)
    ref = fno.FNO2d(nr, nz, width, modes, layers, 8, 3, hidden, params=P)
    ref.zero_grad()
    lr_ = float(ref.loss_and_grad(xd, td).item())
    net = fno.FusedFNO2d(nr, nz, width, modes, layers, 8, 3, hidden, params=P)
    net.zero_grad()
    lf = float(net.loss_and_grad(xd, td).item())
    torch.cuda.synchronize()
    assert fno.fno_net_status(True) == 0
    print("loss gemm", lr_, "fused", lf)
    assert abs(lf - lr_) < 1e-2 * lr_
    for k in P:
        e = _bf16_tol(net.g[k].cpu().numpy(), ref.g[k].cpu().numpy())
        assert e < 5e-2, (k, e)


def test_fused_training_follows_gemm_path(fno):
    """Fifteen Adam steps on one batch with learnable targets (a fixed linear map of the
    input channels): the fused path's loss falls and stays within 2 % of the GEMM path's
    trajectory from the same parameters (the weight images follow every update)."""
    import torch

    nr, nz, width, modes = 64, 128, 32, 16
    P, x, _, layers, hidden = _fused_case(fno, nr, nz, width, modes, 4, seed=11, scale_r=False)
    A = np.random.default_rng(12).normal(size=(8, 3)).astype(np.float32) / np.sqrt(8)
    t = (x @ A).astype(np.float32)
    xd, td = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
    runs = {}
    fno.fno_set_tensor_path(0)
    for name, net in (("gemm", fno.FNO2d(nr, nz, width, modes, layers, 8, 3, hidden, params=P)),
                      ("fused", fno.make_fno(nr, nz, width, modes, layers, 8, 3, hidden, params=P))):
        losses = []
        for _ in range(15):
            net.zero_grad()
            losses.append(float(net.loss_and_grad(xd, td).item()))
            net.adam_step(2e-3)
        runs[name] = np.array(losses)
    assert isinstance(net, fno.FusedFNO2d)
    assert fno.fno_net_status(True) == 0
    print("losses gemm", runs["gemm"][[0, -1]], "fused", runs["fused"][[0, -1]])
    assert runs["fused"][-1] < 0.85 * runs["fused"][0]
    assert np.all(np.abs(runs["fused"] / runs["gemm"] - 1) < 2e-2)
