"""In-place storage (one state buffer, AA pattern) against the two-buffer path (GPU).

With in-place storage each step reads the populations from one layout and writes them
to the other in the same buffer: after an even number of steps node n holds its own
post-collision population i in slot opp(i) (layout S), after an odd number population i
sits at the node it streams to, n + e_i, in slot i (layout L), with the pipe axis
reflecting e_r < 0 into the mirrored slot and populations that leave the domain dropped.
The arithmetic of a node update is the same source as the two-buffer path's, compiled
in another kernel instantiation: with FP32 storage every field, Nusselt number and
exported population agrees to FP32 rounding (the compiler fuses a few multiply-adds
differently, which moves isolated values by an ulp), and the set of dropped populations is
exact; with 16-bit storage the two paths run different bulk kernels (one node per thread
against two) and agree to the storage codec's level.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EZ = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


@pytest.fixture(scope="module")
def lbm():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1409_5929_gb300 import build, lbm as L

    build.build()
    L.load()
    return L


def _params(lbm, geometry, nr, nz, storage="f32", **kw):
    if geometry == lbm.LBM_PIPE_INFLOW:
        base = dict(Ra=0.0, Da=1e-2, eps_mean=1.0, F_eps=0.0, Pr=0.7, tau_nu=0.62, u_in=0.05, init_noise=0.0)
    elif geometry == lbm.LBM_PIPE_PERIODIC_Z:
        base = dict(Ra=0.0, tau_nu=0.8, Da=0.05, F_eps=0.0, body_accel_z=2e-6)
    elif geometry == lbm.LBM_ANNULUS_PERIODIC_Z:
        base = dict(Ra=1e4, Da=5e-3, body_accel_z=2e-6)
    else:
        base = dict(Ra=1e5, Da=1e-3, Pr=0.71)
    base.update(kw)
    return lbm.lbm_params_default(nr=nr, nz=nz, geometry=geometry, storage=storage, **base)


def _pair(lbm, geometry, nr, nz, storage="f32", **kw):
    a = lbm.Solver(_params(lbm, geometry, nr, nz, storage, inplace=0, **kw))
    b = lbm.Solver(_params(lbm, geometry, nr, nz, storage, inplace=1, **kw))
    return a, b


def _dropped_mask(lbm, geometry, nr, nz):
    """Populations the odd-step layout does not keep: those leaving the domain."""
    kr = np.arange(nr)[:, None, None]
    kz = np.arange(nz)[None, :, None]
    r = kr + EX[None, None, :]
    z = kz + EZ[None, None, :]
    pipe = geometry in (lbm.LBM_PIPE_PERIODIC_Z, lbm.LBM_PIPE_INFLOW)
    periodic = geometry in (lbm.LBM_ANNULUS_PERIODIC_Z, lbm.LBM_PIPE_PERIODIC_Z)
    out = (r >= nr) | ((r < 0) & (not pipe)) | np.zeros(z.shape, bool)
    if not periodic:
        out = out | (z < 0) | (z >= nz)
    return np.moveaxis(out, 2, 0)          # [9, nr, nz]


# FP32 rounding: an ulp here and there, carried by the flow over a few hundred steps (the
# bar of the oracle parity tests), with an absolute floor for fields that are near zero
# everywhere (u_r of the periodic cases, of order 1e-7 to 1e-11)
RTOL, ATOL = 1e-5, 1e-9


def _close(x, y, what):
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    assert np.array_equal(np.isnan(x), np.isnan(y)), what
    ok = ~np.isnan(x)
    if not ok.any():
        return
    d, ref = (x[ok] - y[ok]).ravel(), y[ok].ravel()
    err = float(np.linalg.norm(d)) if d.size > 1 else abs(float(d[0]))
    scale = float(np.linalg.norm(ref)) if d.size > 1 else abs(float(ref[0]))
    floor = ATOL * np.sqrt(d.size)
    assert err <= RTOL * scale + floor, (what, err, scale)


def _same_state(a, b, odd, mask=None):
    for k, (x, y) in enumerate(zip(a.moments(), b.moments())):
        _close(y, x, f"moment field {k}")
    _close(b.nusselt(), a.nusselt(), "Nusselt")
    if a.params.geometry == 3:
        _close(b.pipe_nusselt(), a.pipe_nusselt(), "pipe Nusselt")
    (psi_a, m_a), (psi_b, m_b) = a.stream_function(), b.stream_function()
    _close(psi_b, psi_a, "stream function")
    _close(m_b, m_a, "max |psi|")
    fa, ga = a.export_populations()
    fb, gb = b.export_populations()
    if not odd:
        _close(fb, fa, "f")
        _close(gb, ga, "g")
        return
    nan_f, nan_g = np.isnan(fb), np.isnan(gb)
    assert np.array_equal(nan_f, mask) and np.array_equal(nan_g, mask[:5])
    _close(fb[~nan_f], fa[~nan_f], "f kept")
    _close(gb[~nan_g], ga[~nan_g], "g kept")


GEOMS = [(0, 37, 141), (1, 23, 130), (2, 25, 131), (3, 21, 200)]


@pytest.mark.parametrize("geometry,nr,nz", GEOMS)
def test_fp32_matches_two_buffers(lbm, geometry, nr, nz):
    """Annulus, periodic annulus, periodic pipe (axis reflection) and pipe with inlet and
    outlet, ragged sizes: after 1, 2, 37 and 600 steps every field, the Nusselt numbers and
    the exported populations agree to FP32 rounding, with NaN exactly at the dropped
    populations after odd step counts."""
    a, b = _pair(lbm, geometry, nr, nz)
    mask = _dropped_mask(lbm, geometry, nr, nz)
    done = 0
    for total in (1, 2, 37, 600):
        a.step(total - done)
        b.step(total - done)
        done = total
        _same_state(a, b, total % 2 == 1, mask)
    assert b.info().steps == 600


def test_fp32_heater_matches_two_buffers(lbm):
    """The discrete-heater wall (Sec. 4.4), whose update also reads the second node inward."""
    kw = dict(radius_ratio=2.0, Ra=1e5, Da=1e-3, Pr=0.7, eps_mean=0.9, F_eps=0.0, T_hot=11.0, T_cold=1.0,
              heater_len=0.4, heater_center=0.5)
    a, b = _pair(lbm, 0, 41, 41, **kw)
    mask = _dropped_mask(lbm, 0, 41, 41)
    for n in (501, 500):
        a.step(n)
        b.step(n)
        _same_state(a, b, a.info().steps % 2 == 1, mask)
    (ma, za), (mb, zb) = a.heater_nusselt(), b.heater_nusselt()
    _close(mb, ma, "mean heater Nusselt")
    _close(zb, za, "heater Nu(z)")


@pytest.mark.parametrize("geometry,nr,nz", [GEOMS[0], GEOMS[2]])
def test_fp32_rebase_and_run(lbm, geometry, nr, nz):
    """A refresh after an even step count and after an odd one (where boundary nodes with
    dropped populations keep their references) leaves the state equal to the two-buffer
    path's to FP32 rounding.  lbm_run with an even check interval (refreshes in layout S)
    takes the same number of steps to its criterion, with the same residual to rounding."""
    a, b = _pair(lbm, geometry, nr, nz)
    a.step(200)
    b.step(200)
    a.rebase()
    b.rebase()
    _same_state(a, b, False)
    a.step(301)
    b.step(301)
    a.rebase()
    b.rebase()
    mask = _dropped_mask(lbm, geometry, nr, nz)
    fa, _ = a.export_populations()
    fb, _ = b.export_populations()
    keep = ~mask
    assert np.isnan(fb[mask]).all()
    _close(fb[keep], fa[keep], "f after an odd-count refresh")
    _same_state(a, b, True, mask)
    a2, b2 = _pair(lbm, geometry, nr, nz)
    na, ra = a2.run(4000, 200, 1e-12)
    nb, rb = b2.run(4000, 200, 1e-12)
    assert na == nb and abs(rb - ra) <= 1e-3 * ra
    _same_state(a2, b2, na % 2 == 1, mask)


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("geometry,nr,nz", [GEOMS[0], GEOMS[3]])
def test_16bit_against_two_buffers(lbm, storage, geometry, nr, nz):
    """16-bit storage: 2100 steps (two reference refreshes).  Both paths carry the codec's
    error against FP32 storage, the in-place one no more than the two-buffer one, in the
    fields and in the Nusselt numbers."""
    ref = lbm.Solver(_params(lbm, geometry, nr, nz, "f32"))
    a, b = _pair(lbm, geometry, nr, nz, storage)
    for s in (ref, a, b):
        s.step(2100)
    u = lambda s: np.stack(s.moments()[1:3]).astype(np.float64)
    rel = lambda x, y: float(np.linalg.norm(x - y) / np.linalg.norm(y))
    e_a, e_b = rel(u(a), u(ref)), rel(u(b), u(ref))
    nu = lambda s: np.array(s.nusselt() if geometry != lbm.LBM_PIPE_INFLOW else s.pipe_nusselt())
    d_a = np.nanmax(np.abs(nu(a) - nu(ref)))
    d_b = np.nanmax(np.abs(nu(b) - nu(ref)))
    print(storage, geometry, "u rel vs FP32: two-buffer", e_a, "in-place", e_b, "|dNu| vs FP32: two-buffer", d_a,
          "in-place", d_b)
    assert e_b <= 1.5 * e_a + 1e-5
    assert d_b <= 1.5 * d_a + 1e-4


def test_full_size_matches_two_buffers(lbm):
    """The bench's 4096 x 8192 annulus (several rows per thread), 9 steps: FP32 fields
    equal to the two-buffer path's to FP32 rounding."""
    a, b = _pair(lbm, 0, 4096, 8192, Ra=1e6, Da=1e-4)
    a.step(9)
    b.step(9)
    for k, (x, y) in enumerate(zip(a.moments(), b.moments())):
        _close(y, x, f"moment field {k}")
    _close(b.nusselt(), a.nusselt(), "Nusselt")


def test_half_the_state_memory(lbm):
    import torch

    torch.cuda.synchronize()
    sizes = []
    for inplace in (0, 1):
        free0 = torch.cuda.mem_get_info()[0]
        s = lbm.Solver(_params(lbm, 0, 2048, 4096, inplace=inplace))
        sizes.append(free0 - torch.cuda.mem_get_info()[0])
        s.close()
    state = 2048 * 4096 * 14 * 4
    print("allocated two-buffer", sizes[0], "in-place", sizes[1], "one state", state)
    assert abs((sizes[0] - sizes[1]) - state) <= 0.05 * state


def test_residual_rejected_and_batch_rejected(lbm):
    s = lbm.Solver(_params(lbm, 0, 21, 40, inplace=1))
    s.step(3)
    with pytest.raises(lbm.LbmError) as e:
        s.residual()
    assert e.value.code == lbm.LBM_ERR_INVALID
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_batch_create([_params(lbm, 0, 21, 40, inplace=1)])
    assert e.value.code == lbm.LBM_ERR_INVALID


def test_kernel_times_count_both_kernels(lbm):
    s = lbm.Solver(_params(lbm, 0, 64, 256, inplace=1))
    lbm.lbm_set_timing(s.h, True)
    s.step(5)
    bulk_ms, nb, wall_ms, nw = lbm.lbm_kernel_times(s.h)
    assert nb == 5 and nw == 5 and bulk_ms > 0 and wall_ms > 0
