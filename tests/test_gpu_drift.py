"""GPU parity of the drift-trajectory forecast and its error measures E(t)
and RMSE(t) (Sec. 5.2) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1910_01031_gb300 import synth

from gpu_common import ensemble, oracle_problem, rel_l2, start_state

pytestmark = pytest.mark.gpu


def test_drift_forecast_errors_match_oracle():
    cfg = synth.config1(n_particles=6)
    ne, nd = 6, 3
    U32, U64 = start_state(cfg, ne)
    P = oracle_problem(cfg)
    xy0 = synth.drifter_positions(cfg, nd)
    hours, every = 40.0 / 60.0, 600.0
    n_out = 5
    # a synthetic truth trajectory (any positions serve for the error measures)
    truth = np.stack([xy0 + o * np.array([[150.0, -80.0]]) for o in range(n_out)])
    ens = ensemble(cfg, n_drifters_max=nd)
    ens.set_state(U32)
    E, R, traj = ens.drifter_forecast_errors(xy0, hours, every, truth, want_traj=True)
    # oracle: the same model steps with model error, drifters after every scheme step
    ref = U64
    xy = np.repeat(xy0[None], ne, axis=0)
    otraj = [xy.copy()]
    for o in range(1, n_out):
        ref, _, xy = O.forecast(P, ref, 10, True, t0=10 * (o - 1), xy=xy)
        otraj.append(xy.copy())
    otraj = np.stack(otraj)
    assert rel_l2(ens.get_state(), ref) < 1e-5
    disp_g, disp_o = traj - xy0, otraj - xy0
    assert np.max(np.abs(disp_g - disp_o)) < 1e-4 * np.max(np.abs(disp_o))
    Eo, Ro = O.forecast_errors(otraj, truth)
    assert np.allclose(E, Eo, rtol=1e-6, atol=1e-9)
    assert np.allclose(R, Ro, rtol=1e-3, atol=1e-6)
    assert R[0] == 0.0 and np.all(R[1:] > 0)
    # the device reductions against the oracle's formula on the GPU's own positions
    Eg, Rg = O.forecast_errors(traj, truth)
    assert np.allclose(E, Eg, rtol=1e-12, atol=0)
    assert np.allclose(R, Rg, rtol=1e-10, atol=1e-12)


def test_drift_forecast_error_equals_rmse_when_truth_is_the_mean():
    cfg = synth.config1(n_particles=4)
    U32, _ = start_state(cfg, 4)
    ens = ensemble(cfg, n_drifters_max=2)
    ens.set_state(U32)
    xy0 = synth.drifter_positions(cfg, 2)
    # first pass: get the trajectories; second pass from the same start with
    # their ensemble mean as the truth
    E, R, traj = ens.drifter_forecast_errors(xy0, 0.5, 600.0, np.repeat(xy0[None], 4, axis=0), want_traj=True)
    mean = traj.mean(axis=1)
    ens2 = ensemble(cfg, n_drifters_max=2)
    ens2.set_state(U32)
    E2, R2, traj2 = ens2.drifter_forecast_errors(xy0, 0.5, 600.0, mean, want_traj=True)
    assert np.array_equal(traj2, traj)
    assert np.allclose(E2, R2, rtol=1e-12, atol=1e-12)
