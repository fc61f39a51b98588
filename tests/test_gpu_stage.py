"""GPU tests of the staged 16-bit bulk kernels: each row's source runs copied into shared
memory by bulk copies, with the e_z = +-1 columns read from there.  Both the
single-problem kernel (blocks of 256 columns) and the batch kernel (blocks of 128
columns) are compared with the global-load pair update that lbm_set_staging(0) selects,
on the same grids:
- nz a multiple of 8 and nz = 6 mod 8, so the row windows are aligned differently;
- ragged row blocks and ragged last column blocks;
- every geometry class: walls at both rows, periodic z with its end blocks on global
  loads, and the pipe axis row with its mirror sources.
The bounded waits are made to run out on purpose."""
import numpy as np
import pytest

from paper_1409_5929_gb300 import inputs

pytestmark = pytest.mark.gpu

BULK_THREADS = 128   # threads per single-problem bulk block; a block covers 2 BULK_THREADS columns
BULK_RPT = 4         # rows per thread once the grid keeps 16 blocks per SM
RPT_MIN_BLOCKS = 16
TOL = 2e-5           # see _compare


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


def _kw(**kw):
    if kw["geometry"] == 2:
        kw.update(Ra=0.0, tau_nu=0.8, Da=0.05, F_eps=0.0, eps_mean=1.0, body_accel_z=1e-5)
    else:
        kw.update(Ra=1e5, Da=1e-3, Pr=0.71)
    return kw


def _compare(a_fields, b_fields):
    """Both kernels evaluate the same per-node update on the same loaded values; a
    multiply-add the compiler fuses differently in the two kernels flips a 16-bit storage
    rounding (2^-11 of a stored deviation), nothing larger."""
    worst = 0.0
    for a, c in zip(a_fields, b_fields):
        a, c = np.asarray(a, np.float64), np.asarray(c, np.float64)
        assert np.isfinite(a).all() and np.isfinite(c).all()
        worst = max(worst, float(np.abs(a - c).max()))
    assert worst <= TOL, worst
    return worst


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("geometry", [0, 1, 2])
@pytest.mark.parametrize("nz", [2104, 2102])
def test_staged_kernel_matches_global_loads(lbm, storage, geometry, nz):
    nr = _rows_for_staging(nz)
    p = lbm.lbm_params_default(**_kw(nr=nr, nz=nz, geometry=geometry, storage=storage))
    phi = inputs.porosity_field(nr, nz, 0.3, 0.9, 4.0, seed=11) if geometry != 2 else None
    if phi is not None:
        p.eps_mean = float(phi.mean(dtype=np.float64))
    s, g = lbm.Solver(p), lbm.Solver(p)
    lbm.lbm_set_staging(g.h, False)
    for x in (s, g):
        if phi is not None:
            x.set_porosity(phi)
        x.init_fields()
        x.step(200)
    _compare(s.moments(), g.moments())
    ns, ng = s.nusselt(), g.nusselt()
    for k in (0, 1) if geometry != 2 else (1,):
        assert abs(ns[k] - ng[k]) <= 1e-4 * abs(ng[k]) + 1e-9
    assert lbm.lbm_wait_status(s.h) == lbm.LBM_OK
    s.close()
    g.close()


def _batch_params(lbm, storage):
    """Instances with interior column blocks of the 128-column batch tiles, nz = 6 mod 8
    and 0 mod 8, every geometry, one odd nz (global loads in either mode)."""
    specs = [dict(nr=40, nz=262, geometry=0), dict(nr=37, nz=390, geometry=0, radius_ratio=3.0),
             dict(nr=21, nz=520, geometry=1, body_accel_z=2e-6), dict(nr=25, nz=646, geometry=2),
             dict(nr=30, nz=131, geometry=0), dict(nr=48, nz=96, geometry=0)]
    return [lbm.lbm_params_default(storage=storage, **_kw(**sp)) for sp in specs]


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_batch_staged_matches_global_loads(lbm, storage):
    params = _batch_params(lbm, storage)
    phi = inputs.porosity_field(37, 390, 0.3, 0.9, 2.0, seed=7)
    params[1].eps_mean = float(phi.mean(dtype=np.float64))
    a, c = lbm.Batch(params), lbm.Batch(params)
    lbm.lbm_batch_set_staging(c.b, False)
    for x in (a, c):
        x.set_porosity(1, phi)
        x.init_fields(1)
        x.step(150)
        x.run(150 + 150 % 2, 150 + 150 % 2, -1.0)   # graph-replayed steps as well
    for i in range(len(params)):
        _compare(a.moments(i), c.moments(i))
    assert lbm.lbm_batch_wait_status(a.b) == lbm.LBM_OK
    a.close()
    c.close()


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


def test_staged_kernel_wait_runs_out(lbm):
    """A per-row wait limited to zero polls runs out at once: the step is reported as
    LBM_ERR_TIMEOUT (by lbm_wait_status and by lbm_run), the blocks drain their copies
    (the drain keeps its normal bound) and stop, and the context stays usable: after the
    limit is restored and the fields re-initialised, the solver steps like a fresh one."""
    s = _staged_solver(lbm, "f16")
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
    ref = _staged_solver(lbm, "f16")
    s.step(50)
    ref.step(50)
    assert lbm.lbm_wait_status(s.h) == lbm.LBM_OK
    _compare(s.moments(), ref.moments())
    s.close()
    ref.close()


def test_batch_staged_wait_runs_out(lbm):
    """The same for the batch kernel: lbm_batch_run reports LBM_ERR_TIMEOUT; with the limit
    restored and every instance re-initialised, the batch steps like a fresh one."""
    params = _batch_params(lbm, "f16")
    b = lbm.Batch(params)
    lbm.lbm_batch_set_wait_limit(b.b, 0)
    b.step(1)
    assert lbm.lbm_batch_wait_status(b.b, True) == lbm.LBM_ERR_TIMEOUT
    with pytest.raises(lbm.LbmError) as err:
        b.run(2, 2, -1.0)
    assert err.value.code == lbm.LBM_ERR_TIMEOUT
    lbm.lbm_batch_wait_status(b.b, True)
    lbm.lbm_batch_set_wait_limit(b.b, -1)
    ref = lbm.Batch(params)
    for i in range(len(params)):
        b.init_fields(i)
    b.step(40)
    ref.step(40)
    assert lbm.lbm_batch_wait_status(b.b) == lbm.LBM_OK
    for i in range(len(params)):
        _compare(b.moments(i), ref.moments(i))
    b.close()
    ref.close()
