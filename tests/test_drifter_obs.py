"""Drifter observations from two GPS fixes (Sec. 3.3, eq. drifterObservation):
the oracle against uniform flow (closed form) including a crossing of the
periodic boundary, and the library's host-side form against the oracle,
bit for bit (no GPU needed)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1910_01031_gb300 import iewpf, synth


def test_uniform_flow_gives_h_times_the_velocity_across_the_boundary():
    P = O.Problem(nx=64, ny=48, dx=2000.0, dy=2500.0)
    Lx, Ly = 64 * 2000.0, 48 * 2500.0
    u, v, dt = np.array([0.31, -0.12, 0.0]), np.array([-0.05, 0.22, 0.4]), 300.0
    xy_prev = np.array([[Lx - 20.0, 100.0], [10.0, Ly - 5.0], [5e4, 6e4]])
    xy = np.stack([np.mod(xy_prev[:, 0] + u * dt, Lx), np.mod(xy_prev[:, 1] + v * dt, Ly)], axis=1)
    got = O.drifter_observation(P, xy, xy_prev, dt)
    assert np.allclose(got[:, 0], u * P.H, rtol=1e-9, atol=1e-9)
    assert np.allclose(got[:, 1], v * P.H, rtol=1e-9, atol=1e-9)


def test_library_form_equals_the_oracle_bitwise():
    cfg = synth.config2()
    P = O.Problem(nx=cfg.nx, ny=cfg.ny, dx=cfg.dx, dy=cfg.dy, H=cfg.H)
    rng = np.random.default_rng(4)
    xy_prev = rng.uniform(0, 1, (64, 2)) * np.array([cfg.nx * cfg.dx, cfg.ny * cfg.dy])
    xy = xy_prev + rng.normal(0, 200.0, (64, 2))
    xy[:5] = xy_prev[:5] + np.array([cfg.nx * cfg.dx, 0.0]) * 0.999     # large jumps wrap
    got = iewpf.drifter_obs(iewpf.params_from_config(cfg), xy, xy_prev, 300.0)
    ref = O.drifter_observation(P, xy, xy_prev, 300.0)
    assert np.array_equal(got, ref)


def test_library_form_rejects_bad_arguments():
    p = iewpf.params_from_config(synth.config1())
    with pytest.raises(iewpf.IewpfError):
        iewpf.drifter_obs(p, np.zeros((2, 2)), np.zeros((2, 2)), 0.0)
    with pytest.raises(iewpf.IewpfError):
        iewpf.drifter_obs(p, np.array([[np.nan, 0.0]]), np.zeros((1, 2)), 60.0)


def test_observation_structure_of_the_binding():
    # values given: xy_prev is not passed; values None: both fixes and dt
    xy = np.array([[1.0, 2.0], [3.0, 4.0]])
    vals = np.array([[0.5, -0.5], [1.5, 2.5]])
    obs, keep = iewpf.make_obs(xy, vals)
    assert obs.n_obs == 2 and obs.xy[3] == 4.0 and obs.value[2] == 1.5 and not obs.xy_prev
    obs, keep = iewpf.make_obs(xy, None, xy_prev=xy - 1.0, dt=60.0)
    assert obs.n_obs == 2 and not obs.value and obs.xy_prev[0] == 0.0 and obs.dt == 60.0
    obs, keep = iewpf.make_obs(None, vals)                      # moorings: positions fixed at creation
    assert not obs.xy and obs.value[1] == -0.5
    with pytest.raises(ValueError):
        iewpf.make_obs(xy, None)


def test_binding_refuses_mismatched_observation_arrays():
    # the C side reads 2 n doubles from every pointer it is given, so a short
    # array must be refused in the binding before any call
    xy = np.array([[1.0, 2.0], [3.0, 4.0]])
    with pytest.raises(ValueError):
        iewpf.make_obs(xy, None, xy_prev=xy[:1], dt=60.0)
    with pytest.raises(ValueError):
        iewpf.make_obs(xy, np.zeros((3, 2)))
    cfg = synth.config1()
    with pytest.raises(ValueError):
        iewpf.drifter_obs(iewpf.params_from_config(cfg), xy, xy[:1], 60.0)
