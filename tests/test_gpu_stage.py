"""GPU tests of the staged 16-bit bulk kernel (each row's source segments copied into
shared memory by bulk copies, the e_z = +-1 columns read from there) against the
global-load pair update of the batched runner, on grids large enough for the
single-problem step to pick the staged kernel (nz a multiple of 8, 16 blocks per SM):
ragged row blocks and a ragged last column block, every geometry class (walls at both
rows, periodic z, the pipe axis row with its mirror sources); and its bounded waits,
made to run out on purpose."""
import numpy as np
import pytest

from paper_1409_5929_gb300 import inputs

pytestmark = pytest.mark.gpu

BULK_THREADS = 128   # threads per bulk block; a block covers 2 BULK_THREADS columns
BULK_RPT = 4         # rows per thread once the grid keeps 16 blocks per SM
RPT_MIN_BLOCKS = 16


@pytest.fixture(scope="module")
def lbm():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1409_5929_gb300 import build, lbm as L

    build.build()
    L.load()
    return L


def _rows_for_staging(nz):
    """Smallest nr (≡ 2 mod 4, so the last row block is ragged) at which the step runs
    BULK_RPT rows per thread, the condition under which it launches the staged kernel."""
    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    zblocks = -(-nz // (2 * BULK_THREADS))
    rblocks = -(-RPT_MIN_BLOCKS * sms // zblocks)
    return BULK_RPT * rblocks + 2


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("geometry", [0, 1, 2])
def test_staged_kernel_follows_global_load_path(lbm, storage, geometry):
    nz = 2104   # 9 column blocks: the first and the last (ragged) run the global-load path
    nr = _rows_for_staging(nz)
    kw = dict(nr=nr, nz=nz, geometry=geometry, storage=storage)
    if geometry == 2:
        kw.update(Ra=0.0, tau_nu=0.8, Da=0.05, F_eps=0.0, eps_mean=1.0, body_accel_z=1e-5)
    else:
        kw.update(Ra=1e5, Da=1e-3, Pr=0.71)
    phi = inputs.porosity_field(nr, nz, 0.3, 0.9, 4.0, seed=11) if geometry != 2 else None
    p = lbm.lbm_params_default(**kw)
    if phi is not None:
        p.eps_mean = float(phi.mean(dtype=np.float64))
    s, b = lbm.Solver(p), lbm.Batch([p])
    if phi is not None:
        s.set_porosity(phi)
        b.set_porosity(0, phi)
    s.init_fields()
    b.init_fields(0)
    s.step(200)
    b.step(200)
    g, o = b.moments(0), s.moments()
    for a, c in zip(g, o):
        a, c = np.asarray(a, np.float64), np.asarray(c, np.float64)
        assert np.isfinite(c).all()
        # both kernels evaluate the same per-node source; a multiply-add fused differently
        # flips a 16-bit storage rounding (2^-11 of a stored deviation), nothing larger
        assert np.abs(a - c).max() <= 2e-5, np.abs(a - c).max()
    nb, nu = b.nusselt(), s.nusselt()
    for k in (0, 1) if geometry != 2 else (1,):
        assert abs(nb[k][0] - nu[k]) <= 1e-4 * abs(nu[k]) + 1e-9
    assert lbm.lbm_wait_status(s.h) == lbm.LBM_OK
    s.close()
    b.close()


def _staged_solver(lbm, storage):
    nz = 1032
    nr = _rows_for_staging(nz)
    phi = inputs.porosity_field(nr, nz, 0.3, 0.9, 4.0, seed=5)
    p = lbm.lbm_params_default(nr=nr, nz=nz, Ra=1e5, Da=1e-3, Pr=0.71, storage=storage,
                               eps_mean=float(phi.mean(dtype=np.float64)))
    s = lbm.Solver(p)
    s.set_porosity(phi)
    s.init_fields()
    return s


@pytest.mark.parametrize("storage", ["f16"])
def test_staged_kernel_wait_runs_out(lbm, storage):
    """A per-row wait limited to zero polls runs out at once: the step is reported as
    LBM_ERR_TIMEOUT (by lbm_wait_status and by lbm_run), the blocks drain their copies
    (the drain keeps its normal bound) and stop, and the context stays usable: after the
    limit is restored and the fields re-initialised, the solver steps like a fresh one."""
    s = _staged_solver(lbm, storage)
    assert lbm.lbm_wait_status(s.h) == lbm.LBM_OK
    lbm.lbm_set_wait_limit(s.h, 0)
    s.step(1)
    assert lbm.lbm_wait_status(s.h) == lbm.LBM_ERR_TIMEOUT
    assert lbm.lbm_wait_status(s.h, True) == lbm.LBM_ERR_TIMEOUT   # cleared
    assert lbm.lbm_wait_status(s.h) == lbm.LBM_OK
    with pytest.raises(lbm.LbmError) as err:
        s.run(2, 1, -1.0)
    assert err.value.code == lbm.LBM_ERR_TIMEOUT
    lbm.lbm_wait_status(s.h, True)
    lbm.lbm_set_wait_limit(s.h, -1)
    s.init_fields()
    ref = _staged_solver(lbm, storage)
    s.step(50)
    ref.step(50)
    assert lbm.lbm_wait_status(s.h) == lbm.LBM_OK
    for a, c in zip(s.moments(), ref.moments()):
        assert np.isfinite(a).all()
        assert np.abs(np.asarray(a, np.float64) - c).max() <= 2e-5
    s.close()
    ref.close()
