"""GPU tests of the batched runner: every instance of a batch must follow the
single-problem path (the same per-node source; the compiler may fuse multiply-adds
differently in the two kernels, so agreement is at rounding level), and the oracle."""
import os

import numpy as np
import pytest

from paper_1409_5929_gb300 import inputs

pytestmark = pytest.mark.gpu
THREADS = min(16, os.cpu_count() or 1)


@pytest.fixture(scope="module")
def lbm():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1409_5929_gb300 import build, lbm as L

    build.build()
    L.load()
    return L


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(np.asarray(b, np.float64)), 1e-300))


def _mixed_params(lbm, storage="f32"):
    """Uneven sizes (ragged tails, several tiles), all geometries, variable porosity."""
    specs = [dict(nr=48, nz=96), dict(nr=37, nz=300, Ra=3e4, Da=1e-3, Pr=0.71, radius_ratio=3.0),
             dict(nr=64, nz=128, Ra=1e5, Da=1e-2, Pr=7.0, radius_ratio=1.5),
             dict(nr=21, nz=130, geometry=1, Ra=1e4, Da=5e-3, body_accel_z=2e-6),
             dict(nr=25, nz=66, geometry=2, Ra=0.0, tau_nu=0.8, Da=0.05, F_eps=0.0, eps_mean=1.0, body_accel_z=1e-5),
             dict(nr=3, nz=3, Ra=1e4)]
    return [lbm.lbm_params_default(storage=storage, **s) for s in specs]


def _fields(solver_or_batch, i=None):
    return solver_or_batch.moments() if i is None else solver_or_batch.moments(i)


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_batch_instances_follow_single_path(lbm, storage):
    params = _mixed_params(lbm, storage)
    phi = inputs.porosity_field(37, 300, 0.3, 0.9, 2.0, seed=7)
    params[1].eps_mean = float(phi.mean(dtype=np.float64))
    b = lbm.Batch(params)
    b.set_porosity(1, phi)
    b.init_fields(1)
    singles = []
    for i, p in enumerate(params):
        s = lbm.Solver(p)
        if i == 1:
            s.set_porosity(phi)
            s.init_fields()
        singles.append(s)
    b.step(300)
    for s in singles:
        s.step(300)
    for i, s in enumerate(singles):
        g, o = _fields(b, i), _fields(s)
        pairs = ((g[0], o[0]), (np.stack(g[1:3]), np.stack(o[1:3])), (g[3], o[3]))   # rho, u, T
        if storage == "f32":
            for a, c in pairs:
                assert _rel(a, c) <= 2e-6, (i, _rel(a, c))
        else:
            # 16-bit stored deviations turn an FP32 rounding difference into a flipped
            # storage rounding (2^-11 of a deviation): absolute bound, far below what a
            # wrong offset or constant gives
            for a, c in pairs:
                assert np.abs(np.asarray(a, np.float64) - c).max() <= 2e-5, (i, np.abs(a - c).max())
    nb = b.nusselt()
    tol = 1e-5 if storage == "f32" else 1e-3
    for i, s in enumerate(singles):
        nu = s.nusselt()
        if params[i].geometry != 2:
            assert abs(nb[0][i] - nu[0]) <= tol * abs(nu[0]) + 1e-9
        assert abs(nb[1][i] - nu[1]) <= tol * abs(nu[1]) + 1e-9


def test_batch_matches_oracle(lbm, oracle):
    params = _mixed_params(lbm)[:1] + _mixed_params(lbm)[3:5]
    b = lbm.Batch(params)
    b.step(1000)
    for i, p in enumerate(params):
        op = oracle.params(nr=p.nr, nz=p.nz, geometry=p.geometry, radius_ratio=p.radius_ratio, Ra=p.Ra, Da=p.Da,
                           Pr=p.Pr, J=p.J, lam=p.lam, Ma=p.Ma, tau_nu=p.tau_nu, F_eps=p.F_eps, eps_mean=p.eps_mean,
                           T_hot=p.T_hot, T_cold=p.T_cold, body_accel_z=p.body_accel_z, init_noise=p.init_noise,
                           seed=p.seed)
        st = oracle.State(op)
        st.run(1000, THREADS)
        g, o = b.moments(i), st.moments()
        assert _rel(g[0], o[0]) < 1e-5 and _rel(np.stack(g[1:3]), np.stack(o[1:3])) < 1e-5 and _rel(g[3], o[3]) < 1e-5


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_batch_graph_run_equals_plain_steps(lbm, storage):
    """lbm_batch_run replays a captured graph of check_every steps; with tol = 0 it
    must leave every instance exactly where plain stepping (with the same reference
    refreshes) does.  With 16-bit storage the 1200-step intervals also hold the flow
    reference's own refresh after 1024 steps, inside the graph."""
    params = _mixed_params(lbm, storage)
    if storage == "f16":
        a, c = lbm.Batch(params), lbm.Batch(params)
        steps, res = a.run(2400, 1200, 0.0)
        assert (steps == 2400).all() and np.isfinite(res).all()
        for _ in range(2):
            c.rebase()
            c.step(1200)
        for i in range(len(params)):
            for x, y in zip(a.moments(i), c.moments(i)):
                assert np.array_equal(x, y)
        return
    a, c = lbm.Batch(params), lbm.Batch(params)
    steps, res = a.run(600, 200, 0.0)
    assert (steps == 600).all() and np.isfinite(res).all()
    for _ in range(3):                           # the run refreshes the reference before each interval
        c.rebase()
        c.step(200)
    for i in range(len(params)):
        for x, y in zip(a.moments(i), c.moments(i)):
            assert np.array_equal(x, y)


def test_batch_run_stops_converged_instances(lbm):
    """Each instance stops at its own check once the criterion holds; its result is
    the single-problem lbm_run result with the same criterion."""
    specs = [dict(nr=20, nz=40, Ra=1e3), dict(nr=32, nz=64, Ra=1e4, Da=1e-2), dict(nr=24, nz=48, Ra=0.0,
                                                                                   tau_nu=0.8)]
    params = [lbm.lbm_params_default(**s) for s in specs]
    b = lbm.Batch(params)
    steps, res = b.run(400000, 1000, 1e-9)
    assert (res <= 1e-9).all()
    assert len(set(steps.tolist())) > 1          # uneven convergence
    nb = b.nusselt()
    for i, p in enumerate(params):
        s = lbm.Solver(p)
        n, r = s.run(400000, 1000, 1e-9)
        # the batch sums each instance's residual in a different order, so the
        # threshold may be met one check apart
        assert abs(n - steps[i]) <= 1000
        nu = s.nusselt()
        assert abs(nu[0] - nb[0][i]) <= 1e-6 * abs(nu[0]) + 1e-12


def test_batch_autotune(lbm):
    params = _mixed_params(lbm)
    b, c = lbm.Batch(params), lbm.Batch(params)
    cols, rows, ms = b.tune(4)
    assert cols * rows <= 8 * 256 and ms > 0
    c.step(b.info(0).steps)                     # the steps the tuner ran
    b.step(10)
    c.step(10)
    # the tuner ran several rows-per-thread instantiations, which may fuse multiply-adds
    # differently: rounding-level agreement on rho, the velocity vector and T
    for i in range(len(params)):
        g, o = b.moments(i), c.moments(i)
        for x, y in ((g[0], o[0]), (np.stack(g[1:3]), np.stack(o[1:3])), (g[3], o[3])):
            assert _rel(x, y) <= 2e-6, (i, _rel(x, y))
