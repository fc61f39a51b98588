"""Failure detection without a GPU fault.

- A non-finite value planted in a host input (the start temperature) spreads through the
  state, and every convergence check reports LBM_ERR_DIVERGED instead of a number; the
  handle stays usable afterwards.
- The tcgen05 GEMM of the warm-start network gives up a bounded wait (a test hook makes
  one wait on a barrier that nothing arrives at), reports it through
  fno_tensor_path_status and leaves the next GEMM unaffected; the host's handling of the
  worse status (a recovery wait that ran out) is driven by writing that status itself.

Collected after the tensor-core tests of test_fno.py and before the allocation-free
residual's file, which comes last."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1409_5929_gb300 import build, lbm as L

    build.build()
    L.load()
    return L


def _poisoned_T(nr, nz):
    T = np.full((nr, nz), 0.5, np.float32)
    T[nr // 2, nz // 2] = np.nan
    return T


def test_single_problem_reports_divergence(lbm):
    import torch

    nr, nz = 24, 40
    s = lbm.Solver(lbm.lbm_params_default(nr=nr, nz=nz, Ra=1e4))
    s.init_fields(T=_poisoned_T(nr, nz))
    s.step(20)
    with pytest.raises(lbm.LbmError) as e:
        s.residual()
    assert e.value.code == lbm.LBM_ERR_DIVERGED
    with pytest.raises(lbm.LbmError) as e:
        s.run(400, 100, 1e-8)
    assert e.value.code == lbm.LBM_ERR_DIVERGED
    # a cold start on the same handle runs and checks as before
    s.init_fields()
    s.step(20)
    res, mass = s.residual()
    assert np.isfinite(res) and np.isfinite(mass)
    # the allocation-free residual reads device snapshots and reports the same
    N = nr * nz
    cur = torch.zeros(4 * N, dtype=torch.float32, device="cuda")
    prev = torch.zeros(4 * N, dtype=torch.float32, device="cuda")
    cur[3 * N + 3 * nz + 5] = float("nan")
    torch.cuda.synchronize()
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_field_residual_noalloc(0, nr, nz, s.info().r0, cur, prev, N)
    assert e.value.code == lbm.LBM_ERR_DIVERGED
    s.close()


def test_batch_stops_the_diverged_instance_only(lbm):
    params = [lbm.lbm_params_default(nr=24, nz=40, Ra=1e4), lbm.lbm_params_default(nr=30, nz=50, Ra=1e4)]
    b = lbm.Batch(params)
    b.init_fields(1, T=_poisoned_T(30, 50))
    with pytest.raises(lbm.LbmError) as e:
        b.run(400, 100, 1e-8)
    assert e.value.code == lbm.LBM_ERR_DIVERGED and "instance 1" in str(e.value)
    steps, res = b.run(400, 100, 1e-8)   # instance 0 carries on alone
    assert steps[0] > 0 and np.isfinite(res[0])
    assert all(np.isfinite(f).all() for f in b.moments(0))
    b.close()


@pytest.fixture(scope="module")
def fno():
    from paper_1409_5929_gb300 import build, fno as F

    build.build()
    F.load()
    return F


def _gemm_case(fno, seed=0):
    import torch

    batch, M, N, K = 2, 300, 96, 200
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(batch, M, K)).astype(np.float32)
    B = rng.normal(size=(batch, K, N)).astype(np.float32)
    Ad, Bd = torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda")
    Cd = torch.zeros((batch, M, N), dtype=torch.float32, device="cuda")
    ref = np.einsum("bmk,bkn->bmn", A.astype(np.float64), B.astype(np.float64))

    def run():
        Cd.zero_()
        fno.fno_gemm(0, 0, M, N, K, 1.0, Ad, K, M * K, Bd, N, K * N, 0.0, Cd, N, M * N, batch)
        torch.cuda.synchronize()
        got = Cd.cpu().numpy()
        return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))

    return run


def test_tcgen05_wait_timeout_is_reported_and_recovered(fno):
    run = _gemm_case(fno)
    fno.fno_set_tensor_path(1)
    assert fno.fno_tensor_path_status(True) == 0
    fno.fno_test_wait_timeout(True)
    try:
        err = run()
    finally:
        fno.fno_test_wait_timeout(False)
    # the wait ran out, every issued MMA was seen complete before the tensor memory was
    # freed (status 1), and the output of that GEMM is not trusted
    assert fno.fno_tensor_path_status(False) == 1
    assert err > 1e-3
    assert fno.fno_tensor_path_status(True) == 1
    # the next GEMM on the same path runs clean
    assert run() < 2e-2
    assert fno.fno_tensor_path_status(True) == 0
    fno.fno_set_tensor_path(0)


def test_tcgen05_path_disabled_after_unrecovered_wait(fno):
    """Status 2 (a recovery wait ran out as well) turns the tcgen05 path off for the rest
    of the process: GEMMs fall back to mma.sync and stay correct.  Runs after every other
    tensor-core test of the suite."""
    run = _gemm_case(fno, seed=1)
    fno.fno_set_tensor_path(1)
    fno.fno_test_set_tc_error(2)
    assert fno.fno_tensor_path_status(True) == 2
    assert fno.fno_tensor_path_status(True) == 2        # sticky, although the flag was cleared
    with pytest.raises(RuntimeError):
        fno.fno_set_tensor_path(1)
    assert run() < 2e-2                                 # served by the mma.sync kernel
    fno.fno_set_tensor_path(0)
