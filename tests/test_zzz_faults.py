"""Failure detection without a GPU fault: a non-finite value planted in a host input
(the start temperature) spreads through the state, and every convergence check reports
LBM_ERR_DIVERGED instead of a number; the handle stays usable afterwards.  Collected last,
after the allocation-free residual's file."""
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
