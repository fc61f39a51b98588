"""What the trained network gains over the method without it (the cold start), on a
small version of the warm-start workload: 256 training fields and 32 held-out
instances on a 32 x 64 annulus, sweep parameter ranges.  The iteration always runs to
the criterion from the proposed field and decides the result."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_trained_network_gains_over_cold_start():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1409_5929_gb300 import build, fno as F, warmstart as W

    build.build()
    nr, nz, tol = 32, 64, 1e-8
    train_inst = W.make_instances(256, 40000, nr, nz)
    held = W.make_instances(32, 50000, nr, nz)
    _, _, _, fields, _ = W.run_batch(train_inst, 60000, 1000, tol)
    X = torch.tensor(W.features(train_inst, nr, nz), device="cuda")
    Y = torch.tensor(np.stack([W.targets_from_fields(f[1], f[2], f[3]) for f in fields]), device="cuda")
    net = F.FNO2d(nr, nz, width=32, modes=8, seed=1)
    losses = W.train(net, X, Y, epochs=15, batch=8, lr=2e-3)
    assert losses[-1] < 0.2 * losses[0]
    pred = W.predict(net, torch.tensor(W.features(held, nr, nz), device="cuda"))
    cold = W.run_batch(held, 120000, 1000, tol)
    warm = W.run_batch(held, 120000, 1000, tol, warm=W.fields_from_targets(pred))
    r = W.compare(*cold, *warm, pred, tol, 1e-3)
    print(r)
    err = r["start_field_rms_error"]
    assert err["trained_network"] < 0.2 * err["rest_state"]          # far closer start than the rest state
    bc = r["both_converged"]
    assert bc["instances"] >= 8
    assert bc["agree_within_dNu_tol"] == bc["instances"]            # the iteration reaches the same answer
    assert bc["steps_ratio_cold_over_warm"] > 1.0                   # and needs fewer steps to get there
    assert r["warm"]["converged"] >= r["cold"]["converged"]
