"""CPU checks of the C ABI: the library builds, loads and exports every entry
point the headers declare; host-side parameter derivation agrees with the oracle
and rejects invalid input.  No device call is made here."""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(lbm_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lbm():
    from paper_1409_5929_gb300 import build, lbm as L

    build.build()
    L.load()
    return L


def test_every_declared_symbol_is_exported(lbm):
    names = _declared()
    assert len(names) >= 15
    lib = C.CDLL(lbm.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


@pytest.mark.parametrize("header,lib_name", [("fno.h", "libfno.so"), ("fno_net.h", "libfnonet.so")])
def test_network_libraries_export_their_headers(lbm, header, lib_name):
    """The warm-start network's libraries (built by the same build step) load without a
    GPU and export every function their header declares."""
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", header)).read(), flags=re.S)
    names = sorted({m.group(1) for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(fno_\w+)\s*\(", text, flags=re.M)})
    assert len(names) >= 8
    lib = C.CDLL(os.path.join(ROOT, "paper_1409_5929_gb300", lib_name))
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_fused_network_size_checks(lbm):
    """Host-side size checks of the fused network (no device call)."""
    from paper_1409_5929_gb300 import fno as F

    assert F.net_supported(8, 128, 256, 32, 16, 128, 8, 3)
    assert F.net_supported(8, 64, 128, 32, 8, 128, 8, 3)
    assert F.net_supported(2, 64, 128, 64, 8, 128, 8, 3)
    assert not F.net_supported(2, 16, 32, 8, 4, 16, 8, 3)      # width, nz, hidden
    assert not F.net_supported(2, 16, 128, 32, 8, 128, 8, 3)   # 2 nr not a multiple of 128
    assert not F.net_supported(2, 64, 100, 32, 8, 128, 8, 3)   # nz
    assert not F.net_supported(2, 64, 128, 32, 12, 128, 8, 3)  # 2 modes not 16 or 32
    assert not F.net_supported(2, 64, 128, 32, 8, 64, 8, 3)    # hidden


def _oracle_params(oracle, p):
    return oracle.params(nr=p.nr, nz=p.nz, geometry=p.geometry, radius_ratio=p.radius_ratio, Ra=p.Ra, Da=p.Da,
                         Pr=p.Pr, J=p.J, lam=p.lam, Ma=p.Ma, tau_nu=p.tau_nu, F_eps=p.F_eps, eps_mean=p.eps_mean,
                         T_hot=p.T_hot, T_cold=p.T_cold, body_accel_z=p.body_accel_z, init_noise=p.init_noise,
                         seed=p.seed, u_in=p.u_in, heater_len=p.heater_len, heater_center=p.heater_center,
                         collision=p.collision)


@pytest.mark.parametrize("kw", [
    {},
    dict(nr=4096, nz=8192, Ra=1e6, Da=1e-4, Pr=0.71),
    dict(nr=8192, nz=8192, Ra=1e7, Da=1e-6, Pr=0.71, tau_nu=0.51, eps_mean=0.4, storage="f16"),
    dict(nr=33, nz=4, geometry=2, Ra=0.0, tau_nu=0.8, Da=0.0625, F_eps=0.0, eps_mean=1.0, body_accel_z=1e-5),
    dict(nr=100, nz=200, Ra=1e5, Pr=0.7, Da=1e8, eps_mean=1.0, F_eps=0.0),
    dict(nr=41, nz=648, geometry=3, Ra=0.0, tau_nu=0.5096, Da=1e-3, eps_mean=1.0, F_eps=0.0, Pr=0.7, u_in=0.0079),
    dict(nr=200, nz=200, Ra=1e7, Da=1e-4, Pr=0.7, eps_mean=0.9, F_eps=0.0, T_hot=11.0, T_cold=1.0,
         heater_len=0.4, heater_center=0.5),
    dict(nr=37, nz=300, Ra=3e4, Da=1e-3, Pr=0.71, radius_ratio=3.0, collision=1),
])
def test_derivation_matches_oracle(lbm, oracle, kw):
    p = lbm.lbm_params_default(**kw)
    info = lbm.lbm_derive(p)
    ref = oracle.derive(_oracle_params(oracle, p))
    for k_lib, k_ref in (("L", "L"), ("H", "H"), ("r0", "r0"), ("tau_nu", "tau"), ("tau_T", "tauT"),
                         ("nu_e", "nu_e"), ("nu", "nu"), ("gbeta", "gbeta"), ("T0", "T0"), ("Kbar", "Kbar")):
        assert np.isclose(getattr(info, k_lib), ref[k_ref], rtol=1e-14, atol=0), k_lib
    ef = 4 if p.storage == 0 else 2           # flow populations; temperature populations stay FP32
    # populations read and written, the FP32 porosity, and the references a pull reads: the
    # FP16 temperature offset (FP32 storage) or the 4 x FP16 reference word (16-bit storage)
    assert info.bytes_per_step == p.nr * p.nz * (2 * (9 * ef + 5 * 4) + 4 + (2 if p.storage == 0 else 8))


@pytest.mark.parametrize("bad", [
    dict(nr=2), dict(nz=1), dict(tau_nu=0.5), dict(radius_ratio=1.0), dict(eps_mean=0.0), dict(eps_mean=1.5),
    dict(geometry=7), dict(storage=5), dict(Ra=0.0, tau_nu=0.0), dict(Pr=0.0), dict(T_hot=0.0, T_cold=0.0),
    dict(nr=70000), dict(collision=2), dict(heater_len=1.5), dict(heater_len=0.4, heater_center=1.2),
    dict(heater_len=0.4, geometry=2, Ra=0.0, tau_nu=0.8), dict(geometry=3, Ra=0.0, tau_nu=0.8, u_in=-0.01),
    dict(geometry=3, Ra=0.0, tau_nu=0.8, u_in=0.6),
])
def test_invalid_parameters_rejected(lbm, bad):
    p = lbm.lbm_params_default(**bad)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_derive(p)
    assert e.value.code == lbm.LBM_ERR_INVALID
    assert lbm.load().lbm_last_error().decode()


def test_product_path_has_no_oracle_dependency():
    """The library package never imports, links or loads the oracle (no CPU fallback)."""
    pkg = os.path.join(ROOT, "paper_1409_5929_gb300")
    pat = re.compile(r"(import\s+oracle|from\s+oracle|liblbm_oracle|\borc_\w+|lbm_oracle)")
    for path in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if path.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
            assert not pat.search(open(path).read()), path
