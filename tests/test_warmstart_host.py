"""Host logic of the warm-start measurement (no GPU): the time-to-steady summary on
synthetic Nusselt trajectories with known answers."""
import numpy as np

from paper_1409_5929_gb300.warmstart import steps_to_nu, summarize


def _traj(nchunks, chunk, final, start, rate, wobble=0.0):
    t = (np.arange(nchunks) + 1) * chunk
    nu = final + (start - final) * np.exp(-rate * t) + wobble * np.sin(t / (7.0 * chunk))
    return np.stack([nu, 2 * nu], axis=1)            # both walls


def test_steps_to_nu_first_settled_chunk():
    traj = np.array([[[3.0, 3.0]], [[1.0, 1.0]], [[2.0, 2.0]], [[1.0005, 1.0]], [[1.0, 1.0]]])
    assert steps_to_nu(traj, np.array([[1.0, 1.0]]), 1e-3, 10).tolist() == [40]   # the dip at 20 does not count
    assert steps_to_nu(traj, np.array([[5.0, 5.0]]), 1e-3, 10).tolist() == [-1]


def test_summarize_classifies_and_counts_steps():
    n, ch = 200, 1000
    cases = [
        # (cold, warm, group): converging to the same value, warm starts closer
        (_traj(n, ch, 2.0, 1.0, 1e-4), _traj(n, ch, 2.0, 1.9, 1e-4), "a"),
        (_traj(n, ch, 3.0, 1.0, 6e-5), _traj(n, ch, 3.0, 3.1, 6e-5), "a"),
        # stationary, but the warm run ends 1e-2 away
        (_traj(n, ch, 2.0, 1.0, 1e-4), _traj(n, ch, 2.01, 1.9, 1e-4), "b"),
        # still oscillating at the end
        (_traj(n, ch, 2.0, 1.0, 1e-4, wobble=1e-2), _traj(n, ch, 2.0, 1.9, 1e-4), "b"),
    ]
    tc = np.stack([c[0] for c in cases], axis=1)
    tw = np.stack([c[1] for c in cases], axis=1)
    out, ok = summarize(tc, tw, ch, 1e-3, 20 * ch, 1e-4, groups=[c[2] for c in cases])
    assert ok.tolist() == [True, True, False, False]
    assert (out["stationary"], out["stationary_agree"], out["stationary_disagree"], out["nonstationary"]) == (3, 2, 1, 1)
    # analytic first settle times against the value at the end T of the run (the outer
    # wall dominates): 2 |a| (e^{-r t} - e^{-r T}) <= 1e-3, rounded up to a recorded step
    T = n * ch
    want = lambda a, r: int(np.ceil(-np.log(1e-3 / (2 * abs(a)) + np.exp(-r * T)) / r / ch)) * ch
    s_c, s_w = [want(1.0, 1e-4), want(2.0, 6e-5)], [want(0.1, 1e-4), want(0.1, 6e-5)]
    assert out["cold_steps_max"] == max(s_c) and out["warm_steps_max"] == max(s_w)
    assert out["steps_ratio_cold_over_warm_sum"] == round(sum(s_c) / sum(s_w), 3)
    assert out["by_group"]["a"]["stationary_agree"] == 2 and out["by_group"]["b"]["nonstationary"] == 1
    assert abs(out["disagree_dNu_quantiles_50_90_max"][2] - 0.02) < 1e-6      # outer wall: 2 x 0.01
