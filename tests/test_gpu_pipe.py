"""GPU tests of the pipe with inlet and outlet (Sec. 4.1, Fig. 1): parity with the FP64
oracle, and Table 1 (fully developed Nusselt numbers for seven Darcy numbers)."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
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
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _pipe_params(lbm, nr, nz, Da, tau, u_in, Pr=0.7, storage="f32"):
    # Da = 0 stands for the pipe without porous matrix (no drag)
    return lbm.lbm_params_default(nr=nr, nz=nz, geometry=lbm.LBM_PIPE_INFLOW, Ra=0.0, Da=Da if Da > 0 else 1e8,
                                  eps_mean=1.0, F_eps=0.0, Pr=Pr, tau_nu=tau, u_in=u_in, init_noise=0.0,
                                  storage=storage)


@pytest.mark.parametrize("Da", [1e-2, 0.0])
def test_pipe_inflow_parity(lbm, oracle, Da):
    """21 x 200 pipe (inlet, outlet, axis, wall; Brinkman drag or none), 3000 steps from
    the start state: fields within relative L2 1e-5 of the oracle, the local Nusselt
    numbers of Eq. 40 and the stream function (from the axis) within 1e-5 relative."""
    p = _pipe_params(lbm, 21, 200, Da, 0.62, 0.05)
    s = lbm.Solver(p)
    op = oracle.params(nr=p.nr, nz=p.nz, geometry=oracle.PIPE_INFLOW, Ra=0.0, Da=p.Da, eps_mean=1.0, F_eps=0.0,
                       Pr=p.Pr, tau_nu=p.tau_nu, u_in=p.u_in, init_noise=0.0)
    st = oracle.State(op)
    assert np.array_equal(s.node_class(), oracle.node_class(op))
    s.step(3000)
    st.run(3000, THREADS)
    g, o = s.moments(), st.moments()
    errs = [_rel(g[0], o[0]), _rel(np.stack(g[1:3]), np.stack(o[1:3])), _rel(g[3], o[3])]
    print("pipe parity", Da, errs)
    assert max(errs) <= 1e-5, errs
    nu_g, nu_o = s.pipe_nusselt(), st.pipe_nusselt()
    assert np.isnan(nu_g[0]) and np.isnan(nu_o[0])
    assert np.abs(nu_g[1:] - nu_o[1:]).max() <= 1e-5 * np.abs(nu_o[1:]).max()
    (psi_g, m_g), (psi_o, m_o) = s.stream_function(), oracle.stream_function(op, o[2])
    assert _rel(psi_g, psi_o) <= 1e-5 and abs(m_g - m_o) <= 1e-5 * m_o


def test_table1_pipe(lbm):
    """Table 1: 81 x 648 in the paper (diameter x length), i.e. 41 radial nodes from the
    axis image row at r = 1/2 to the wall node at r_i = 40.5 and 648 columns; Pr = 0.7,
    phi = 1, F_phi = 0, Re = r_i U_in / nu = 100.  U_in is not stated; it is taken as 0.05,
    lowered where the Darcy pressure drop would compress the fluid (density change
    3 nu U_in H / (c_s^2 K) ~ 0.48 U_in^2 / Da kept at 3 %).  All seven cases in one batch,
    run to the steady criterion; the fully developed value is Nu at z = 0.9 H.  Measured
    0.6 - 3.1 % above the paper's column, which is itself 0.8 % from Ref. [6]: the scheme's
    wall error is first order (3.757 -> 3.706 from r_i = 20.5 to 40.5 in the oracle's Graetz
    case), so 3.5 % is the bound."""
    rows = [tuple(map(float, l.split())) for l in open(os.path.join(HERE, "golden", "table1_pipe_nusselt.txt"))
            if l.strip() and not l.startswith("#")]
    nr, nz = 41, 648
    params = []
    for Da, _, _ in rows:
        U = 0.05 if Da == 0 else min(0.05, (0.03 * Da / 0.48) ** 0.5)
        params.append(_pipe_params(lbm, nr, nz, Da, 0.5 + 3 * (nr - 0.5) * U / 100.0, U))
    b = lbm.Batch(params)
    steps, res = b.run(2000000, 2000, 4e-10)
    out = []
    for i, (Da, nu_ref6, nu_paper) in enumerate(rows):
        val = b.pipe_nusselt(i)[int(round(0.9 * (nz - 1)))]
        out.append((Da, val, nu_paper))
        print("Table 1", Da, val, nu_paper, nu_ref6, steps[i], res[i])
    for Da, val, nu_paper in out:
        assert abs(val / nu_paper - 1) < 0.035, out
    # Nu grows as Da falls (Sec. 4.1)
    vals = [v for _, v, _ in out[:-1]]
    assert all(a > b for a, b in zip(vals, vals[1:])) and vals[-1] > out[-1][1]
