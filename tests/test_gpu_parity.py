"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on the
same seeded inputs.

Tolerances.  FP32 arithmetic on FP32 storage: relative L2 <= 1e-5 on each field
(rho, the velocity vector u, T) after 10^4 steps, the bar stated for the plain method.  FP16 /
BF16 deviation storage: |Delta Nu| <= 1e-3 against the oracle, with each field's
error reported.  Node classes: bit-exact.
"""
import os

import numpy as np
import pytest

from paper_1409_5929_gb300 import inputs

pytestmark = pytest.mark.gpu
THREADS = min(16, os.cpu_count() or 1)
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
WT = np.array([0.6, 0.1, 0.1, 0.1, 0.1])


@pytest.fixture(scope="module")
def lbm():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1409_5929_gb300 import build, lbm as L

    build.build()
    L.load()
    return L


def _oparams(oracle, p):
    return oracle.params(nr=p.nr, nz=p.nz, geometry=p.geometry, radius_ratio=p.radius_ratio, Ra=p.Ra, Da=p.Da,
                         Pr=p.Pr, J=p.J, lam=p.lam, Ma=p.Ma, tau_nu=p.tau_nu, F_eps=p.F_eps, eps_mean=p.eps_mean,
                         T_hot=p.T_hot, T_cold=p.T_cold, body_accel_z=p.body_accel_z, init_noise=p.init_noise,
                         seed=p.seed, u_in=p.u_in, heater_len=p.heater_len, heater_center=p.heater_center,
                         collision=p.collision)


def _quantise_phi(phi, storage):
    """The porosity field as the library holds it (FP32 for every storage type)."""
    return np.asarray(phi, np.float32).astype(np.float64)


def _pair(lbm, oracle, storage="f32", phi=None, **kw):
    p = lbm.lbm_params_default(storage=storage, **kw)
    if phi is not None:
        p.eps_mean = float(np.mean(phi, dtype=np.float64))
    s = lbm.Solver(p)
    if phi is not None:
        s.set_porosity(phi)
        s.init_fields()
    phi_o = _quantise_phi(phi if phi is not None else np.full((p.nr, p.nz), p.eps_mean, np.float32), storage)
    st = oracle.State(_oparams(oracle, p), phi=phi_o)
    return s, st


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _field_errors(g, o):
    """Relative L2 errors of rho, the velocity vector u = (u_r, u_z) and T; the
    deviation rho - 1 and the components are reported too (a component that is
    zero in exact arithmetic, like u_r of an axial flow, has no meaningful
    relative error of its own)."""
    errs = {"rho": _rel(g[0], o[0]), "u": _rel(np.stack(g[1:3]), np.stack(o[1:3])), "T": _rel(g[3], o[3])}
    errs.update(drho=_rel(g[0] - 1.0, o[0] - 1.0), ur=_rel(g[1], o[1]), uz=_rel(g[2], o[2]))
    return errs


def _fields_close(s, st, tol):
    errs = _field_errors(s.moments(), st.moments())
    bad = {k: errs[k] for k in ("rho", "u", "T") if errs[k] > tol}
    assert not bad, errs
    return errs


def _nusselt_within_bound(s, st):
    """Eq. 42 is a fixed linear functional of T (trapezoid weights summing to H, the
    one-sided stencil (-3, 4, -1)/2), so |Nu_gpu - Nu_oracle| <= r_w * 4 * max|dT| / dT
    over the three wall rows.  The GPU reduction reads T in FP64 from the state; the
    moments it is compared through are FP32, hence one FP32 ulp of slack."""
    Tg, To = s.moments()[3], st.moments()[3]
    info = s.info()
    dTw = s.params.T_hot - s.params.T_cold
    nu_g, nu_o = s.nusselt(), st.nusselt()
    for j, rows, rw in ((0, slice(0, 3), info.r0), (1, slice(-3, None), info.r0 + s.nr - 1)):
        dmax = np.abs(Tg[rows].astype(np.float64) - To[rows]).max() + 6e-8
        bound = rw * 4 * dmax / dTw
        assert abs(nu_g[j] - nu_o[j]) <= bound, (j, nu_g, nu_o, bound)
        assert abs(nu_g[j] - nu_o[j]) <= 1e-4 * abs(nu_o[j]), (j, nu_g, nu_o)
    return nu_g, nu_o


@pytest.mark.parametrize("geom", [0, 1, 2])
@pytest.mark.parametrize("shape", [(3, 3), (5, 130), (48, 96), (37, 300)])
def test_node_classes_bit_exact(lbm, oracle, geom, shape):
    nr, nz = shape
    s = lbm.Solver(lbm.lbm_params_default(nr=nr, nz=nz, geometry=geom))
    o = oracle.node_class(_oparams(oracle, s.params))
    assert np.array_equal(s.node_class(), o)


def test_start_state(lbm, oracle):
    phi = inputs.porosity_field(37, 300, 0.3, 0.9, 2.0, seed=11)
    s, st = _pair(lbm, oracle, phi=phi, nr=37, nz=300, Ra=1e4, Da=1e-3, init_noise=0.05)
    f, g = s.export_populations()
    r = s.info().r0 + np.arange(37)
    df = (f - st.f) / np.maximum(np.abs(st.f - r[None, :, None] * W9[:, None, None]).max(), 1e-30)
    assert np.abs(df).max() < 1e-6
    assert np.abs(g - st.g).max() < 1e-7
    gm, om = s.moments(), st.moments()
    assert _rel(gm[0], om[0]) < 1e-6 and _rel(gm[3], om[3]) < 1e-6
    # at rest u is zero up to rounding on both sides: compare against the buoyancy velocity scale
    uscale = s.info().gbeta * s.info().L
    assert np.abs(np.stack(gm[1:3]) - np.stack(om[1:3])).max() < 1e-6 * uscale


@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("geometry", [0, 2])
def test_warm_start_init_fields(lbm, oracle, storage, geometry):
    """lbm_init_fields with caller-given (u_r, u_z, T), u != 0 (the call the learned warm
    start feeds), against orc_init on the same fields: every stored population, element by
    element, and the fields of the start state.  Porous field, Ergun drag, buoyancy, walls;
    FP32 storage to FP32 rounding of the deviations, 16-bit flow storage to its rounding."""
    nr, nz = 37, 300
    phi = inputs.porosity_field(nr, nz, 0.3, 0.9, 2.0, seed=13)
    rng = np.random.default_rng(17)
    ur = (0.01 * rng.standard_normal((nr, nz))).astype(np.float32)
    uz = (0.01 * rng.standard_normal((nr, nz))).astype(np.float32)
    T = (0.5 + 0.2 * rng.standard_normal((nr, nz))).astype(np.float32)
    kw = dict(nr=nr, nz=nz, geometry=geometry, Ra=1e4, Da=1e-3, Pr=0.71)
    if geometry == 2:
        kw.update(body_accel_z=1e-5)
    s, st0 = _pair(lbm, oracle, storage=storage, phi=phi, **kw)
    s.init_fields(ur, uz, T)
    st = oracle.State(st0.p, phi=st0.phi, ur=ur.astype(np.float64), uz=uz.astype(np.float64),
                      T=T.astype(np.float64))
    f, g = s.export_populations()
    r = s.info().r0 + np.arange(nr)
    dev = st.f - r[None, :, None] * W9[:, None, None]
    scale = np.abs(dev).max()
    rel_f = np.abs(f - st.f).max() / scale
    tol_f = 1e-6 if storage == "f32" else 2.0 ** -10
    assert rel_f < tol_f, rel_f
    assert np.abs(g - st.g).max() < 1e-6
    gm, om = s.moments(), st.moments()
    errs = _field_errors(gm, om)
    print(storage, geometry, "start-state populations", rel_f, "fields", errs)
    assert errs["u"] < (1e-5 if storage == "f32" else 2e-3) and errs["T"] < 1e-6


def test_config1_plain_method_10k_steps(lbm, oracle):
    """Porous annulus 48 x 96, R* = 2, eps = 0.6, Da = 1e-2, Ra = 1e3, Pr = 1, Ergun
    F_eps, hot inner / cold outer wall, adiabatic ends, seeded +-1e-3 noise, 10^4
    steps: relative L2 <= 1e-5 per field; Nusselt numbers and residual agree."""
    s, st = _pair(lbm, oracle)
    s.step(9999)
    st.run(9999, THREADS)
    prev_o = st.moments()
    s.step(1)
    st.run(1, THREADS)
    errs = _fields_close(s, st, 1e-5)
    print("config1 field errors", errs)
    _nusselt_within_bound(s, st)
    res_g, mass_g = s.residual()
    res_o, mass_o = oracle.residual(st.p, st.moments(), prev_o)
    assert abs(res_g - res_o) <= 1e-3 * res_o + 1e-12
    assert abs(mass_g - mass_o) <= 1e-9 * mass_o


@pytest.mark.parametrize("case", ["porous_field", "periodic_body_force", "pipe_brinkman", "forchheimer_pipe"])
def test_parity_small_grids(lbm, oracle, case):
    """Several blocks along z with a ragged tail (nz = 300 = 2 x 128 + 44), every
    geometry, variable porosity, body force, Forchheimer drag."""
    if case == "porous_field":
        phi = inputs.porosity_field(37, 300, 0.3, 0.9, 2.0, seed=7)
        s, st = _pair(lbm, oracle, phi=phi, nr=37, nz=300, Ra=3e4, Da=1e-3, Pr=0.71, radius_ratio=3.0)
    elif case == "periodic_body_force":
        s, st = _pair(lbm, oracle, nr=21, nz=300, geometry=1, Ra=1e4, Da=5e-3, body_accel_z=2e-6)
    elif case == "pipe_brinkman":
        s, st = _pair(lbm, oracle, nr=25, nz=300, geometry=2, Ra=0.0, tau_nu=0.8, Da=0.05, F_eps=0.0,
                      eps_mean=1.0, body_accel_z=1e-5)
    else:
        phi = inputs.porosity_field(25, 300, 0.4, 0.8, 1.5, seed=9)
        s, st = _pair(lbm, oracle, phi=phi, nr=25, nz=300, geometry=2, Ra=0.0, tau_nu=0.7, Da=2e-3, F_eps=1.0,
                      body_accel_z=5e-4)
    s.step(2000)
    st.run(2000, THREADS)
    _fields_close(s, st, 1e-5)


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_bgk_collision_parity(lbm, oracle, storage):
    """LBM_BGK (every rate 1/tau, Sec. 3.1) on the porous annulus with a smoothed porosity
    field (37 x 300, Ra = 3e4), 3000 steps against the oracle's BGK option: FP32 fields
    within 1e-5, 16-bit flow storage |Delta Nu| <= 1e-3; and the run differs from MRT."""
    phi = inputs.porosity_field(37, 300, 0.3, 0.9, 2.0, seed=7)
    s, st = _pair(lbm, oracle, storage=storage, phi=phi, nr=37, nz=300, Ra=3e4, Da=1e-3, Pr=0.71, radius_ratio=3.0,
                  collision=1)
    assert st.p.collision == 1
    s.step(3000)
    st.run(3000, THREADS)
    if storage == "f32":
        _fields_close(s, st, 1e-5)
    else:
        nu_g, nu_o = s.nusselt(), st.nusselt()
        assert abs(nu_g[0] - nu_o[0]) <= 1e-3 and abs(nu_g[1] - nu_o[1]) <= 1e-3
    m, _ = _pair(lbm, oracle, storage=storage, phi=phi, nr=37, nz=300, Ra=3e4, Da=1e-3, Pr=0.71, radius_ratio=3.0)
    m.step(3000)
    assert _rel(m.moments()[2], s.moments()[2]) > 1e-4


def test_full_size_sampled_nodes(lbm, oracle):
    """Single large domain 4096 x 8192 (variable porosity uniform[0.3, 0.9] smoothed
    by sigma = 16, Da = 1e-4, Ra = 1e6, Pr = 0.71), in the benchmark's launch
    configuration: for sampled nodes (corners, walls, interior, last column block)
    the oracle recomputes one step from the GPU's own pre-step state."""
    nr, nz = 4096, 8192
    phi = inputs.porosity_field(nr, nz, 0.3, 0.9, 16.0, seed=2)
    p = lbm.lbm_params_default(nr=nr, nz=nz, Ra=1e6, Da=1e-4, Pr=0.71, eps_mean=float(phi.mean(dtype=np.float64)))
    s = lbm.Solver(p)
    s.set_porosity(phi)
    s.init_fields()
    s.step(20)
    rng = np.random.default_rng(0)
    samples = [(0, 0), (0, nz - 1), (nr - 1, 0), (nr - 1, nz - 1), (0, 4000), (nr - 1, 77), (1, 0), (2000, nz - 1),
               (1, 1), (nr - 2, nz - 2), (1, nz - 2), (nr - 2, 1), (2, 8191 - 44)]
    samples += [(int(a), int(b)) for a, b in zip(rng.integers(0, nr, 24), rng.integers(0, nz, 24))]
    op = _oparams(oracle, p)
    r0 = s.info().r0
    # lazily allocated full-size arrays; only rows around the samples are filled
    F = np.zeros((9, nr, nz))
    G = np.zeros((5, nr, nz))
    PHI = np.zeros((nr, nz))
    rows = sorted({k for kr, _ in samples for k in range(max(0, kr - 2), min(nr, kr + 3))})
    for kr in rows:
        f, g = s.export_populations(kr, 1)
        F[:, kr] = f[:, 0]
        G[:, kr] = g[:, 0]
        PHI[kr] = phi[kr].astype(np.float64)
    s.step(1)
    worst = 0.0
    for kr, kz in samples:
        fo, go, _ = oracle.node_update(op, PHI, F, G, kr, kz)
        f, g = s.export_populations(kr, 1)
        dev_o = fo - (r0 + kr) * W9
        dev_g = f[:, 0, kz] - (r0 + kr) * W9
        scale = np.abs(dev_o).max()
        worst = max(worst, np.abs(dev_g - dev_o).max() / scale)
        assert np.abs(g[:, 0, kz] - go).max() < 1e-6
    assert worst < 1e-5, worst


def test_edge_cases(lbm, oracle):
    s = lbm.Solver(lbm.lbm_params_default(nr=3, nz=3))
    with pytest.raises(lbm.LbmError):
        s.residual()                                  # needs a step
    s.step(0)
    assert s.info().steps == 0
    s.step(5)
    rho, ur, uz, T = s.moments()
    assert np.isfinite(rho).all() and np.isfinite(T).all()
    bad = np.full((3, 3), 0.5, np.float32)
    bad[1, 1] = 0.0
    with pytest.raises(lbm.LbmError) as e:
        s.set_porosity(bad)
    assert e.value.code == lbm.LBM_ERR_INVALID
    # minimum grid matches the oracle too
    s2, st = _pair(lbm, oracle, nr=3, nz=3, Ra=1e4)
    s2.step(50)
    st.run(50, 1)
    _fields_close(s2, st, 1e-5)


def test_deterministic(lbm):
    out = []
    for _ in range(2):
        s = lbm.Solver(lbm.lbm_params_default(nr=64, nz=200, Ra=1e5))
        s.step(300)
        out.append(s.export_populations())
    assert all(np.array_equal(a, b) for a, b in zip(out[0], out[1]))


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("nz", [3, 129, 301])
def test_boundary_nodes_written_once_odd_nz(lbm, storage, nz):
    """The wall kernel runs beside the bulk kernel, so a boundary node written by both would
    race.  With odd nz the two-column bulk kernel's last pair starts on the closed end
    column; it must leave that node to the wall kernel: three runs of the same problem are
    bit-identical.  (test_gpu_batch's 3 x 3 instance, stepped by other kernels, compares
    the result itself.)"""
    out = []
    for _ in range(3):
        s = lbm.Solver(lbm.lbm_params_default(nr=21, nz=nz, Ra=1e4, storage=storage))
        s.step(200)
        out.append(s.export_populations())
    for o in out[1:]:
        assert all(np.array_equal(a, b, equal_nan=True) for a, b in zip(out[0], o))


def test_largest_domain_runs(lbm):
    """8192 x 8192 (the stress case's size), FP16 storage, tau_nu = 0.51."""
    phi = _config5_phi()
    p = lbm.lbm_params_default(nr=8192, nz=8192, Ra=1e7, Da=1e-6, Pr=0.71, tau_nu=0.51, storage="f16",
                               eps_mean=float(phi.mean(dtype=np.float64)))
    s = lbm.Solver(p)
    s.set_porosity(phi)
    s.init_fields()
    s.step(20)
    nu = s.nusselt()
    assert np.isfinite(nu).all()


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_half_storage_config1(lbm, oracle, storage):
    """FP16 / BF16 deviation storage, FP32 arithmetic, config 1 for 10^4 steps:
    |Delta Nu| <= 1e-3 against the FP64 oracle; field errors reported."""
    s, st = _pair(lbm, oracle, storage=storage)
    s.step(10000)
    st.run(10000, THREADS)
    errs = _field_errors(s.moments(), st.moments())
    nu_g, nu_o = s.nusselt(), st.nusselt()
    print(storage, "field errors", errs, "Nu", nu_g, nu_o)
    assert abs(nu_g[0] - nu_o[0]) <= 1e-3 and abs(nu_g[1] - nu_o[1]) <= 1e-3
    assert errs["T"] < 1e-3


def test_table2_free_annulus(lbm):
    """Table 2 (Sec. 4.2): free-fluid annulus, phi = 1, Da = 1e8, Pr = 0.7,
    R* = A = 2, 100 x 200, run to steady state: Nu_i within 2 % of the printed
    values (the paper's own scatter against the literature is about 1 %).  With adiabatic
    top and bottom the steady heat flux through both walls is the same, Nu_i = Nu_o; the
    non-equilibrium wall rebuild balances neither the mass nor the heat that streams across
    a wall exactly, and at the fixed Ma = 0.1 of Eq. 39 its relaxation-time-dependent part
    leaves Nu_o 1.3 % below Nu_i at Ra = 1e3 on this grid (the FP64 oracle gives the same
    1.29 %; with tau fixed the imbalance falls at first order under refinement, a CPU pin
    of the oracle).  Asserted: within the 2 % of the paper's own scatter."""
    path = os.path.join(os.path.dirname(__file__), "golden", "table2_annulus_nusselt.txt")
    rows = [tuple(map(float, l.split())) for l in open(path) if l.strip() and not l.startswith("#")]
    for ra, nu_paper in rows:
        s = lbm.Solver(lbm.lbm_params_default(nr=100, nz=200, Ra=ra, Pr=0.7, Da=1e8, eps_mean=1.0, F_eps=0.0))
        steps, res = s.run(3_000_000, 2000, 1e-9)
        nu_i, nu_o = s.nusselt()
        print("Table 2", ra, nu_i, nu_o, nu_paper, steps, res)
        assert abs(nu_i / nu_paper - 1) < 0.02
        assert abs(nu_i - nu_o) < 0.02 * nu_i


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_config2_recipe_256x512(lbm, oracle, storage):
    """The single-domain workload's recipe at 256 x 512 (porosity uniform[0.3, 0.9]
    smoothed by sigma = 16, seed 2; Ra = 1e6, Da = 1e-4, Pr = 0.71; tau_nu = 0.5372 at this
    size), 10^4 steps, per storage type.  FP32: relative L2 <= 1e-5 per field and Nu within
    the linear bound; 16-bit flow storage: |Delta Nu| <= 1e-3 and T within 1e-3, the field
    errors reported."""
    phi = inputs.porosity_field(256, 512, 0.3, 0.9, 16.0, seed=2)
    s, st = _pair(lbm, oracle, storage=storage, phi=phi, nr=256, nz=512, Ra=1e6, Da=1e-4, Pr=0.71)
    assert abs(s.info().tau_nu - 0.5372) < 1e-4
    s.step(10000)
    st.run(10000, THREADS)
    errs = _field_errors(s.moments(), st.moments())
    nu_g, nu_o = s.nusselt(), st.nusselt()
    print(storage, "256x512 field errors", errs, "Nu", nu_g, nu_o)
    if storage == "f32":
        _fields_close(s, st, 1e-5)
        _nusselt_within_bound(s, st)
    else:
        assert abs(nu_g[0] - nu_o[0]) <= 1e-3 and abs(nu_g[1] - nu_o[1]) <= 1e-3
        assert errs["T"] < 1e-3


def test_config5_corner_crop_512(lbm, oracle):
    """The stress case on the 512 x 512 corner crop of its porosity field (uniform[0.3,
    0.5] smoothed by sigma = 32 at 8192 x 8192, seed 5; crop first, then the annulus built
    at 512 x 512): Ra = 1e7, Da = 1e-6, Pr = 0.71, tau_nu = 0.51, FP16 flow storage, 10^4 steps
    against the FP64 oracle."""
    phi = _config5_phi()[:512, :512].copy()
    s, st = _pair(lbm, oracle, storage="f16", phi=phi, nr=512, nz=512, Ra=1e7, Da=1e-6, Pr=0.71, tau_nu=0.51)
    s.step(10000)
    st.run(10000, THREADS)
    errs = _field_errors(s.moments(), st.moments())
    nu_g, nu_o = s.nusselt(), st.nusselt()
    print("config5 crop field errors", errs, "Nu", nu_g, nu_o)
    assert np.isfinite(nu_g).all()
    assert abs(nu_g[0] - nu_o[0]) <= 1e-3 and abs(nu_g[1] - nu_o[1]) <= 1e-3
    assert errs["T"] < 1e-3


_CONFIG5_PHI = {}


def _config5_phi():
    """Porosity of the stress case (uniform[0.3, 0.5] smoothed by sigma = 32 at 8192 x 8192,
    seed 5), generated once per test session."""
    if "phi" not in _CONFIG5_PHI:
        _CONFIG5_PHI["phi"] = inputs.porosity_field(8192, 8192, 0.3, 0.5, 32.0, seed=5)
    return _CONFIG5_PHI["phi"]


def _config5_drift(L, chunks, chunk):
    """Nu of the full-size stress case (8192 x 8192, tau_nu = 0.51, Ra = 1e7, Da = 1e-6) every
    `chunk` steps for three runs: FP32 storage, FP32 storage perturbed at its own rounding
    level (one temperature-reference refresh after 1000 steps re-rounds every thermal
    population), and FP16 flow storage.  Returns (|FP16 - FP32|, |perturbed - FP32|)."""
    phi = _config5_phi()
    nus = {}
    for name, storage in (("f32", "f32"), ("f32_perturbed", "f32"), ("f16", "f16")):
        p = L.lbm_params_default(nr=8192, nz=8192, Ra=1e7, Da=1e-6, Pr=0.71, tau_nu=0.51, storage=storage,
                                 eps_mean=float(phi.mean(dtype=np.float64)))
        s = L.Solver(p)
        s.set_porosity(phi)
        s.init_fields()
        traj = []
        for k in range(chunks):
            if name == "f32_perturbed" and k == 0:
                s.step(1000)
                s.rebase()
                s.step(chunk - 1000)
            else:
                s.step(chunk)
            traj.append(s.nusselt())
        nus[name] = np.array(traj)
        s.close()
    d16 = np.abs(nus["f16"] - nus["f32"])
    d32 = np.abs(nus["f32_perturbed"] - nus["f32"])
    print("config5 Nu f32", nus["f32"].tolist(), "f16", nus["f16"].tolist(), "|dNu| f16-f32", d16.tolist(),
          "|dNu| perturbed f32 - f32", d32.tolist())
    assert all(np.isfinite(v).all() for v in nus.values())
    return d16, d32


def test_config5_nusselt_drift_fp16_vs_fp32(lbm):
    """Stress case at full size (8192 x 8192, tau_nu = 0.51, Ra = 1e7): over 2 x 10^4 steps,
    Nu compared every 5000 steps, all runs finite.  This transient is unsteady: two FP32 runs
    that differ only by one re-rounding of the thermal populations drift apart by far more
    than 1e-3 in Nu (Nu ~ 240-940), so the FP16 run is held to that sensitivity: its
    distance from FP32 stays within 3 times the perturbed FP32 run's, or 1e-3.  The
    absolute bar |Delta Nu| <= 1e-3 against FP64 is checked on the 512 x 512 crop."""
    d16, d32 = _config5_drift(lbm, 4, 5000)
    assert (d16 <= np.maximum(1e-3, 3 * d32.max(axis=0))).all(), (d16, d32)


@pytest.mark.slow
@pytest.mark.skipif(not os.environ.get("LBM_SLOW"), reason="set LBM_SLOW=1 (about 8 min on one GB300)")
def test_config5_nusselt_drift_fp16_vs_fp32_long(lbm):
    """The same over 10^5 steps, Nu compared every 10^4 steps."""
    d16, d32 = _config5_drift(lbm, 10, 10000)
    assert (d16 <= np.maximum(1e-3, 3 * d32.max(axis=0))).all(), (d16, d32)


def test_async_porosity_upload(lbm):
    """lbm_set_porosity_async: the same fields as lbm_set_porosity when the uploads are
    pipelined behind queued steps (each step sees the field set before it), an upload no
    step read replaced by the next one, and invalid values counted by lbm_porosity_errors."""
    import torch

    p = lbm.lbm_params_default(nr=64, nz=200, Ra=1e5, Da=1e-3)
    phis = [inputs.porosity_field(64, 200, 0.3, 0.9, 2.0, seed=k) for k in (1, 2, 3)]
    pins = [torch.from_numpy(f).pin_memory() for f in phis]
    a, b = lbm.Solver(p), lbm.Solver(p)
    for f in phis:
        a.set_porosity(f)
        a.step(7)
    lbm.lbm_set_porosity_async(b.h, pins[0].data_ptr())
    b.step(7)
    lbm.lbm_set_porosity_async(b.h, pins[1].data_ptr())   # queued behind the first 7 steps
    b.step(7)
    lbm.lbm_set_porosity_async(b.h, pins[2].data_ptr())
    b.step(7)
    for x, y in zip(a.moments(), b.moments()):
        assert np.array_equal(x, y)
    assert lbm.lbm_porosity_errors(b.h) == 0
    bad = phis[0].copy()
    bad[3, 3] = 0.0
    bad[5, 7] = 1.5
    pin_bad = torch.from_numpy(bad).pin_memory()
    lbm.lbm_set_porosity_async(b.h, pin_bad.data_ptr())
    assert lbm.lbm_porosity_errors(b.h) == 2
    assert lbm.lbm_porosity_errors(b.h) == 0
    # uploads that no reader saw are replaced by the newest one (three in a row: both
    # staging buffers reused)
    c, d = lbm.Solver(p), lbm.Solver(p)
    c.set_porosity(phis[2])
    c.step(5)
    for pin in pins:
        lbm.lbm_set_porosity_async(d.h, pin.data_ptr())
    d.step(5)
    for x, y in zip(c.moments(), d.moments()):
        assert np.array_equal(x, y)
    for s in (a, b, c, d):
        s.close()


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_porosity_range_count_ragged(lbm, storage):
    """The porosity kernels read four values at a time and the ragged tail one at a time:
    values outside (0, 1] in either part are all counted (asynchronous upload; synchronous
    upload from host memory and from a device pointer that is not 16-byte aligned), and the
    field a step then sees is the one uploaded."""
    import torch

    p = lbm.lbm_params_default(nr=5, nz=7, storage=storage)   # 35 values: 8 groups of 4 + 3
    f = np.full((5, 7), 0.5, np.float32)
    f[0, 1] = 0.0          # in a group of four
    f[4, 5] = 2.0          # in the tail
    f[4, 6] = -1.0         # in the tail
    e = lbm.Solver(p)
    pin = torch.from_numpy(f).pin_memory()
    lbm.lbm_set_porosity_async(e.h, pin.data_ptr())
    assert lbm.lbm_porosity_errors(e.h) == 3
    with pytest.raises(RuntimeError, match="3 porosity values"):
        e.set_porosity(f)
    dev = torch.full((36,), 0.5, dtype=torch.float32, device="cuda")
    dev[1:] = torch.from_numpy(f.ravel()).cuda()
    torch.cuda.synchronize()
    assert dev[1:].data_ptr() % 16 != 0
    with pytest.raises(RuntimeError, match="3 porosity values"):
        e.set_porosity(dev[1:])
    good = np.linspace(0.31, 0.89, 35, dtype=np.float32).reshape(5, 7)
    dev[1:] = torch.from_numpy(good.ravel()).cuda()
    torch.cuda.synchronize()
    e.set_porosity(dev[1:])
    ref = lbm.Solver(p)
    ref.set_porosity(good)
    e.init_fields()
    ref.init_fields()
    e.step(20)
    ref.step(20)
    for x, y in zip(e.moments(), ref.moments()):
        assert np.array_equal(x, y)
    e.close()
    ref.close()


@pytest.mark.parametrize("pinned", [False, True])
@pytest.mark.parametrize("geom", [0, 2])
def test_nusselt_async(lbm, geom, pinned):
    """lbm_nusselt_async + lbm_sync give what lbm_nusselt gives after the same steps,
    with several reads queued before one wait (inner value NaN for the periodic pipe), into
    pageable memory (copied) and pinned memory (written by the device)."""
    import torch

    kw = dict(nr=40, nz=130, Ra=1e5, Da=1e-3) if geom == 0 else dict(nr=25, nz=130, geometry=2, Ra=0.0, tau_nu=0.8,
                                                                         Da=0.05, F_eps=0.0, eps_mean=1.0,
                                                                         body_accel_z=1e-5)
    a, b = lbm.Solver(lbm.lbm_params_default(**kw)), lbm.Solver(lbm.lbm_params_default(**kw))
    out = torch.full((3, 2), -1.0, dtype=torch.float64)
    if pinned:
        out = out.pin_memory()
    ref = []
    for k in range(3):
        a.step(40)
        lbm.lbm_nusselt_async(a.h, out[k])
        b.step(40)
        ref.append(b.nusselt())
    lbm.lbm_sync(a.h)
    out = out.numpy()
    np.testing.assert_array_equal(out, np.array(ref))
    assert np.isnan(out[:, 0]).all() == (geom == 2)
    a.close()
    b.close()
