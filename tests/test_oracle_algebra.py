"""Pins of the FP64 oracle's per-node algebra against facts the paper and the
mathematics fix (not against a retyping of the oracle's own formulas)."""
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")
EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=float)
EZ = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=float)
CS2 = 1.0 / 3.0


def _read_blocks(name):
    blocks, cur = [], None
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line.startswith("# block"):
            cur = []
            blocks.append(cur)
        elif line and not line.startswith("#"):
            cur.append([float(x) for x in line.split()])
    return [np.array(b) for b in blocks]


def _guo_forcing(r, rho, ur, uz, phi, Ftr, Ftz):
    """Velocity-space porous forcing of Guo & Zhao (ref. [41]) with the factor r
    of Eq. 17: w_i r rho [e.F/cs2 + (e.F)(e.u)/(phi cs2^2) - F.u/(phi cs2)]."""
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    eF = EX * Ftr + EZ * Ftz
    eu = EX * ur + EZ * uz
    Fu = Ftr * ur + Ftz * uz
    return w * r * rho * (eF / CS2 + eF * eu / (phi * CS2 ** 2) - Fu / (phi * CS2))


def test_moment_matrix_orthogonal(oracle):
    """Eq. 18: the rows of M are mutually orthogonal with the Lallemand-Luo norms,
    and M^-1 inverts M."""
    M, Mi = oracle.matrices()
    G = M @ M.T
    assert np.array_equal(G, np.diag([9, 36, 36, 6, 12, 6, 12, 4, 4]).astype(float))
    assert np.allclose(Mi @ M, np.eye(9), atol=1e-15)
    assert np.allclose(M @ Mi, np.eye(9), atol=1e-15)


def test_streaming_matrices_match_appendix(oracle):
    """App. A: C_j = M (e_j I) M^-1 equals the printed C_r and C_z.  Pins both the
    transcription of Eq. 18 and the velocity ordering of Eq. 14."""
    Cr, Cz = _read_blocks("appendix_A_C_matrices.txt")
    M, Mi = oracle.matrices()
    assert np.allclose(M @ np.diag(EX) @ Mi * 6, Cr, atol=1e-12)
    assert np.allclose(M @ np.diag(EZ) @ Mi * 6, Cz, atol=1e-12)


def test_lattice_isotropy(oracle):
    """D2Q9 weights of Eq. 32: zeroth, first and second moments of f_eq at rest are
    r rho, 0 and r rho c_s^2 delta (textbook lattice isotropy)."""
    f = oracle.feq(2.5, 1.3, 0.0, 0.0, 0.7)
    assert np.isclose(f.sum(), 2.5 * 1.3)
    assert np.isclose((EX * f).sum(), 0) and np.isclose((EZ * f).sum(), 0)
    assert np.isclose((EX * EX * f).sum(), 2.5 * 1.3 * CS2)
    assert np.isclose((EZ * EZ * f).sum(), 2.5 * 1.3 * CS2)
    assert np.isclose((EX * EZ * f).sum(), 0)


@pytest.mark.parametrize("seed", range(5))
def test_equilibrium_moments(oracle, seed):
    """M f_eq(Eq. 32) = m_eq(Eq. 19-20): the BGK-equivalence statement of Sec. 3.1."""
    rng = np.random.default_rng(seed)
    r, rho, ur, uz, phi = rng.uniform(0.5, 50), rng.uniform(0.9, 1.1), *rng.normal(0, 0.05, 2), rng.uniform(0.3, 1)
    M, _ = oracle.matrices()
    assert np.allclose(M @ oracle.feq(r, rho, ur, uz, phi), oracle.meq(r, rho, ur, uz, phi), rtol=1e-13, atol=1e-13 * r)


@pytest.mark.parametrize("seed", range(5))
def test_source_is_guo_forcing_in_moment_space(oracle, seed):
    """Eq. 24 is M applied to the porous Guo forcing of ref. [41] (times r)."""
    rng = np.random.default_rng(100 + seed)
    r, rho, ur, uz, phi = rng.uniform(0.5, 50), rng.uniform(0.9, 1.1), *rng.normal(0, 0.05, 2), rng.uniform(0.3, 1)
    Ftr, Ftz = rng.normal(0, 1e-3, 2)
    M, _ = oracle.matrices()
    S = oracle.source(r, rho, ur, uz, phi, Ftr, Ftz)
    assert np.allclose(M @ _guo_forcing(r, rho, ur, uz, phi, Ftr, Ftz), S, rtol=1e-12, atol=1e-16)


def _random_node(rng, oracle, r, phi=0.6):
    rho = rng.uniform(0.98, 1.02)
    ur, uz = rng.normal(0, 0.02, 2)
    f = oracle.feq(r, rho, ur, uz, phi) * (1 + rng.normal(0, 1e-2, 9))
    T = rng.uniform(0, 1)
    w5 = np.array([0.6, 0.1, 0.1, 0.1, 0.1])
    g = w5 * T * (1 + rng.normal(0, 0.05, 5))
    return f, g


def test_collision_conserves_without_axisymmetric_terms(oracle):
    """With the cylindrical terms and all forces off, the MRT collision conserves
    m_0, m_3, m_5 (Sec. 3.1: the conserved moments) and the D2Q5 step conserves
    sum g (Eq. 38)."""
    p = oracle.params(Ra=0.0, tau_nu=0.8, Da=0.0, F_eps=0.0)
    M, _ = oracle.matrices()
    rng = np.random.default_rng(7)
    for _ in range(10):
        r = rng.uniform(1, 40)
        f, g = _random_node(rng, oracle, r)
        fo, go, _ = oracle.collide_node(p, r, 0.6, f, g, cartesian=True)
        m, mo = M @ f, M @ fo
        assert np.allclose(mo[[0, 3, 5]], m[[0, 3, 5]], rtol=0, atol=1e-13 * r)
        assert np.isclose(go.sum(), g.sum(), rtol=0, atol=1e-14)


def test_collision_axisymmetric_closed_forms(oracle):
    """With every term on: m_0 is unchanged; for s_j = 1, m_3+ = r rho u_r + S_3 / 2
    (Eq. 21); and the change of sum g is the closed form obtained by summing
    Eq. 33 with Eq. 35-37:  -(tau_T / (r (tau_T + 1/2))) [(g1-g3) - (g1-g3)_eq] - u_r T / r."""
    p = oracle.params()
    c = oracle.derive(p)
    M, _ = oracle.matrices()
    rng = np.random.default_rng(8)
    for _ in range(10):
        r = rng.uniform(c["r0"], c["r0"] + 47)
        f, g = _random_node(rng, oracle, r)
        fo, go, (rho, ur, uz, T) = oracle.collide_node(p, r, 0.6, f, g)
        assert np.isclose((M @ fo)[0], (M @ f)[0], rtol=1e-14)
        # S_3 from Eq. 24 with F~_r = F_r + a_r (Eq. 6, 7, 25)
        lin = c["nu"] / c["Kbar"]
        nl = 1.75 / np.sqrt(150 * 0.6 ** 3) / np.sqrt(c["Kbar"])
        um = np.hypot(ur, uz)
        Fr = -0.6 * lin * ur - 0.6 * nl * um * ur
        ar = CS2 * (1 - 2 * (c["tau"] - 0.5) * ur / r) / r
        S3 = r * rho * (Fr + ar)
        assert np.isclose((M @ fo)[3], r * rho * ur + S3 / 2, rtol=1e-12, atol=1e-15)
        tT = c["tauT"]
        geq13 = 0.1 * T * (1 + 5 * ur) - 0.1 * T * (1 - 5 * ur)
        expect = -(tT / (r * (tT + 0.5))) * ((g[1] - g[3]) - geq13) - ur * T / r
        assert np.isclose(go.sum() - g.sum(), expect, rtol=1e-9, atol=1e-15)


def test_result_independent_of_momentum_rate(oracle):
    """Derived from Eq. 21, 24, 25 and 27: m_3 + S_3 / 2 = r rho u_r, so s_j drops out
    of the collision.  Holds exactly where Eq. 28 is exact (no Forchheimer term)."""
    p = oracle.params(F_eps=0.0)
    c = oracle.derive(p)
    rng = np.random.default_rng(9)
    base = np.array([1.0, 1.1, 1.1, 1.0, 1.2, 1.0, 1.2, 1 / c["tau"], 1 / c["tau"]])
    for _ in range(5):
        r = rng.uniform(c["r0"], c["r0"] + 47)
        f, g = _random_node(rng, oracle, r)
        ref, _, _ = oracle.collide_node(p, r, 0.6, f, g, s=base)
        for sj in (0.6, 1.4, 1.9):
            s = base.copy()
            s[3] = s[5] = sj
            out, _, _ = oracle.collide_node(p, r, 0.6, f, g, s=s)
            assert np.allclose(out, ref, rtol=1e-12, atol=1e-14 * r)


def test_bgk_limit(oracle):
    """Sec. 3.1: with every rate 1/tau the model is the BGK model with Eq. 32, i.e.
    f+ = f - (f - f_eq) / tau + (1 - 1/(2 tau)) * Guo forcing."""
    p = oracle.params()
    c = oracle.derive(p)
    tau = c["tau"]
    rng = np.random.default_rng(10)
    for _ in range(5):
        r = rng.uniform(c["r0"], c["r0"] + 47)
        f, g = _random_node(rng, oracle, r)
        fo, _, (rho, ur, uz, T) = oracle.collide_node(p, r, 0.6, f, g, s=np.full(9, 1 / tau))
        lin = c["nu"] / c["Kbar"]
        nl = 1.75 / np.sqrt(150 * 0.6 ** 3) / np.sqrt(c["Kbar"])
        um = np.hypot(ur, uz)
        Gz = c["gbeta"] * (T - c["T0"])
        Ftr = -0.6 * lin * ur - 0.6 * nl * um * ur + CS2 * (1 - 2 * (tau - 0.5) * ur / r) / r
        Ftz = -0.6 * lin * uz - 0.6 * nl * um * uz + 0.6 * Gz
        w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
        eu = EX * ur + EZ * uz
        feq = w * r * rho * (1 + eu / CS2 + eu ** 2 / (2 * 0.6 * CS2 ** 2) - (ur ** 2 + uz ** 2) / (2 * 0.6 * CS2))
        bgk = f - (f - feq) / tau + (1 - 1 / (2 * tau)) * _guo_forcing(r, rho, ur, uz, 0.6, Ftr, Ftz)
        assert np.allclose(fo, bgk, rtol=1e-12, atol=1e-14 * r)


def test_velocity_solves_quadratic_drag(oracle):
    """Eq. 28 with l_1 > 0 solves u (2 l_0 + l_1 |u|) = v exactly when l_r0 = l_z0
    (the Cartesian limit): pins l_1 of Eq. 30 and the root choice of Eq. 28."""
    p = oracle.params(Ra=0.0, tau_nu=0.8, Da=1e-3, F_eps=0.5, eps_mean=0.5)
    c = oracle.derive(p)
    rng = np.random.default_rng(11)
    r, phi = 20.0, 0.5
    f, g = _random_node(rng, oracle, r, phi)
    _, _, (rho, ur, uz, T) = oracle.collide_node(p, r, phi, f, g, cartesian=True)
    K = c["Kbar"]
    l0 = 0.5 * (r + r * phi * 0.5 * c["nu"] / K)
    l1 = r * phi * 0.5 * 0.5 / np.sqrt(K)
    vr = (EX * f).sum() / rho
    vz = (EZ * f).sum() / rho
    um = np.hypot(ur, uz)
    assert np.isclose(ur * (2 * l0 + l1 * um), vr, rtol=1e-12)
    assert np.isclose(uz * (2 * l0 + l1 * um), vz, rtol=1e-12)


def test_relaxation_times_reproduce_groups(oracle):
    """Eq. 39 and Eq. 31, checked against the definitions of Eq. 9: the derived
    nu, alpha, g beta give back Ra and Pr, and U = sqrt(g beta dT L) = Ma c_s."""
    for Ra, Pr, nr in ((1e3, 1.0, 48), (1e6, 0.71, 256), (1e4, 7.0, 100)):
        p = oracle.params(Ra=Ra, Pr=Pr, nr=nr, nz=2 * nr)
        c = oracle.derive(p)
        nu = c["nu"]
        alpha = 0.2 * c["tauT"]  # alpha_e = c_sT^2 tau_T (Sec. 3.2), lambda = 1
        L = c["L"]
        assert np.isclose(c["gbeta"] * 1.0 * L ** 3 / (nu * alpha), Ra, rtol=1e-12)
        assert np.isclose(nu / alpha, Pr, rtol=1e-12)
        assert np.isclose(np.sqrt(c["gbeta"] * L), 0.1 / np.sqrt(3), rtol=1e-12)
    c = oracle.derive(oracle.params())
    assert c["L"] == 47 and c["r0"] == 47  # config 1: r_i = L / (R* - 1)


def test_splitmix64_reference_vectors(oracle):
    for line in open(os.path.join(GOLD, "splitmix64_vectors.txt")):
        if line.startswith("#") or not line.strip():
            continue
        seed, n, out = (int(x) for x in line.split())
        assert oracle.splitmix64(seed, n) == out


@pytest.mark.parametrize("geom", [0, 1, 2])
def test_node_classes_brute_force(oracle, geom):
    """Fig. 1 and Fig. 3 boundaries on tiny grids: walls on the outermost nodes,
    corners belong to the side walls, axis row for the pipe."""
    for nr, nz in ((3, 3), (4, 7), (6, 5)):
        p = oracle.params(nr=nr, nz=nz, geometry=geom)
        cls = oracle.node_class(p)
        for kr in range(nr):
            for kz in range(nz):
                if kr == nr - 1:
                    want = oracle.WALL_OUT
                elif kr == 0:
                    want = oracle.AXIS if geom == 2 else oracle.WALL_IN
                elif geom == 0 and kz == 0:
                    want = oracle.BOTTOM
                elif geom == 0 and kz == nz - 1:
                    want = oracle.TOP
                else:
                    want = oracle.FLUID
                assert cls[kr, kz] == want, (nr, nz, kr, kz)


def test_bgk_collision_option(oracle):
    """collision = 1 selects the BGK limit (Sec. 3.1): a node update equals the MRT update
    with every rate 1/tau (itself pinned against the BGK formula by test_bgk_limit) and
    differs from the MRT rates of Sec. 4."""
    p_mrt, p_bgk = oracle.params(), oracle.params(collision=1)
    tau = oracle.derive(p_mrt)["tau"]
    rng = np.random.default_rng(12)
    r = 60.0
    f, g = _random_node(rng, oracle, r)
    fo_bgk, go_bgk, _ = oracle.collide_node(p_bgk, r, 0.6, f, g)
    fo_ref, go_ref, _ = oracle.collide_node(p_mrt, r, 0.6, f, g, s=np.full(9, 1 / tau))
    fo_mrt, _, _ = oracle.collide_node(p_mrt, r, 0.6, f, g)
    assert np.array_equal(fo_bgk, fo_ref) and np.array_equal(go_bgk, go_ref)
    assert np.abs(fo_bgk - fo_mrt).max() > 1e-6 * np.abs(fo_mrt).max()
