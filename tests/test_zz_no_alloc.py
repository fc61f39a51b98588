"""The allocation-free residual entry point, checked against lbm_residual.

Some callers cannot allocate device memory at the moment they need the convergence
check: their own allocator owns all device memory, or they must not trigger the
device-wide synchronisation that cudaMalloc / cudaFree can cause.
lbm_field_residual_noalloc serves them from a static device array; the caller only
passes the two field snapshots and receives the result.  This file is collected last
so that a run stopping at its first failure has already run every other test.
"""
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


def _snapshot(lbm, s, buf, N):
    """Fields of the solver's current state into one device buffer of 4 planes."""
    import torch

    base, es = buf.data_ptr(), buf.element_size()
    lbm.lbm_moments(s.h, base, base + N * es, base + 2 * N * es, base + 3 * N * es, True)
    torch.cuda.synchronize()


@pytest.mark.parametrize("geometry,nr,nz", [(0, 64, 300), (2, 64, 300), (0, 600, 600)])
def test_noalloc_residual_matches_lbm_residual(lbm, geometry, nr, nz):
    """64 x 300 needs 75 reduction blocks; 600 x 600 (360,000 nodes) is more than the
    1024 blocks x 256 threads of the static scratch cover in one pass, so its partial
    rows accumulate over the grid-stride loop."""
    import torch

    kw = dict(nr=nr, nz=nz, geometry=geometry)
    kw.update(dict(Ra=1e5) if geometry == 0 else dict(Ra=0.0, tau_nu=0.8, Da=0.05, F_eps=0.0, eps_mean=1.0,
                                                        body_accel_z=1e-5))
    s = lbm.Solver(lbm.lbm_params_default(**kw))
    N = nr * nz
    r0 = s.info().r0
    prev = torch.empty(4 * N, dtype=torch.float32, device="cuda")
    cur = torch.empty(4 * N, dtype=torch.float32, device="cuda")
    for nsteps in (99, 400):
        s.step(nsteps)
        _snapshot(lbm, s, prev, N)
        s.step(1)
        _snapshot(lbm, s, cur, N)
        res_ref, mass_ref = s.residual()
        assert res_ref > 0 and np.isfinite(res_ref)
        # two calls in a row on the same inputs: the shared scratch keeps the first
        # call's contents, which must not leak into the second result
        for _ in range(2):
            res, mass = lbm.lbm_field_residual_noalloc(geometry, nr, nz, r0, cur, prev, N)
            assert res == pytest.approx(res_ref, rel=1e-12, abs=0.0)
            assert mass == pytest.approx(mass_ref, rel=1e-12, abs=0.0)
    s.close()


def test_noalloc_residual_rejects_oversize(lbm):
    import torch

    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    for nr, nz in ((2, 10), (70000, 10), (65535, 65535)):
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_field_residual_noalloc(0, nr, nz, 10.0, buf, buf, nr * nz)
        assert e.value.code == lbm.LBM_ERR_INVALID


def test_noalloc_residual_allocates_nothing(lbm):
    """Around repeated calls neither the device's free memory nor PyTorch's reserved
    pool changes (after one warm-up call, which may load the library's device code)."""
    import torch

    nr, nz = 64, 300
    s = lbm.Solver(lbm.lbm_params_default(nr=nr, nz=nz, Ra=1e5))
    N = nr * nz
    r0 = s.info().r0
    prev = torch.empty(4 * N, dtype=torch.float32, device="cuda")
    cur = torch.empty(4 * N, dtype=torch.float32, device="cuda")
    s.step(50)
    _snapshot(lbm, s, prev, N)
    s.step(1)
    _snapshot(lbm, s, cur, N)
    first = lbm.lbm_field_residual_noalloc(0, nr, nz, r0, cur, prev, N)
    torch.cuda.synchronize()
    free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    for _ in range(5):
        assert lbm.lbm_field_residual_noalloc(0, nr, nz, r0, cur, prev, N) == first
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_reserved() == reserved0
    s.close()


def test_noalloc_residual_rejects_bad_pointers(lbm):
    """Host memory (pageable or pinned) and a device allocation shorter than the four
    planes are refused before any kernel runs."""
    import torch

    nr, nz = 600, 600
    N = nr * nz
    host = np.zeros(4 * N, np.float32)
    pinned = torch.zeros(4 * N, dtype=torch.float32).pin_memory()
    dev = torch.zeros(4 * N, dtype=torch.float32, device="cuda")
    # a small tensor lies in one of PyTorch's 2 MiB small-block segments, far shorter than
    # the 5.76 MB the four planes of a 600 x 600 grid need
    short = torch.zeros(16, dtype=torch.float32, device="cuda")
    for bad in (host.ctypes.data, pinned.data_ptr(), short.data_ptr()):
        for cur, prev in ((bad, dev.data_ptr()), (dev.data_ptr(), bad)):
            with pytest.raises(lbm.LbmError) as e:
                lbm.lbm_field_residual_noalloc(0, nr, nz, 10.0, cur, prev, N)
            assert e.value.code == lbm.LBM_ERR_INVALID
    with pytest.raises(TypeError):
        lbm.lbm_field_residual_noalloc(0, nr, nz, 10.0, host, dev, N)
