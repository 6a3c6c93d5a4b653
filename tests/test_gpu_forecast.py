"""GPU parity of the forecast path (stepper, CFL, model error, drifters)
against the FP64 oracle, through the C ABI.  Tolerance: relative L2 <= 1e-5
per model step (FP32 state against FP64)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1910_01031_gb300 import iewpf, synth

from gpu_common import ensemble, oracle_problem, ragged_config, rel_l2, start_state

pytestmark = pytest.mark.gpu
TOL = 1e-5


def test_philox_blocks_are_bit_exact():
    for (p, t, s) in [(0, 0, 0), (7, 123, 1), (999, 4, 2 + 16 * 3)]:
        g = iewpf.philox_blocks(0x1910_01031, p, t, s, 2000)
        key = [0x1910_01031 & 0xFFFFFFFF, 0x1910_01031 >> 32]
        for b in (0, 1, 2, 3, 511, 1999):
            assert list(g[b]) == O.philox([b, p, t, s], key)
    # all 2000 blocks of one stream against the oracle's normals' words
    g = iewpf.philox_blocks(42, 3, 5, 1, 2000)
    ref = np.array([O.philox([b, 3, 5, 1], [42, 0]) for b in range(2000)], dtype=np.uint32)
    assert np.array_equal(g, ref)


def test_normals_match_oracle():
    z64, z32 = iewpf.normals(0x1910_01031, 5, 17, 2, 100_000)
    ref = O.normals(0x1910_01031, 5, 17, 2, 100_000)
    assert np.max(np.abs(z64 - ref) / np.maximum(1.0, np.abs(ref))) < 1e-13
    err = np.abs(z32.astype(np.float64) - ref)
    assert err.max() < 2e-5 and err.mean() < 1e-6


def test_lake_at_rest_is_exactly_steady_on_gpu():
    cfg = synth.config1(n_particles=2)
    ens = ensemble(cfg)
    ens.set_state(np.zeros(ens.shape, np.float32))
    ens.forecast_fixed(3, False, 7)
    assert np.array_equal(ens.get_state(), np.zeros(ens.shape, np.float32))
    ens.forecast(2, False)
    assert np.array_equal(ens.get_state(), np.zeros(ens.shape, np.float32))


@pytest.mark.parametrize("maker", [synth.config1, ragged_config])
def test_fixed_substeps_match_oracle(maker):
    cfg = maker()
    ne = 3
    U32, U64 = start_state(cfg, ne)
    P = oracle_problem(cfg)
    ens = ensemble(synth.Config(**{**cfg.as_dict(), "n_particles": ne}))
    ens.set_state(U32)
    ref = U64
    for step in range(4):
        ens.forecast_fixed(1, False, 9)
        ref, _, _ = O.forecast(P, ref, 1, False, t0=step, fixed_n_sub=9)
        assert rel_l2(ens.get_state(), ref) < TOL, step


def test_mass_is_conserved_on_gpu():
    cfg = ragged_config()
    U32, _ = start_state(cfg, cfg.n_particles)
    ens = ensemble(cfg)
    ens.set_state(U32)
    m0 = U32[:, 0].astype(np.float64).sum(axis=(1, 2))
    ens.forecast_fixed(5, False, 10)
    out = ens.get_state()
    m1 = out[:, 0].astype(np.float64).sum(axis=(1, 2))
    scale = np.abs(U32[:, 0]).astype(np.float64).sum(axis=(1, 2))
    assert np.all(np.abs(m1 - m0) < 2e-6 * scale)


def test_add_qhalf_matches_oracle():
    cfg = ragged_config()
    ens = ensemble(cfg)
    P = oracle_problem(cfg)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((cfg.n_particles, P.N_R)).astype(np.float32)
    ens.set_state(np.zeros(ens.shape, np.float32))
    ens.add_qhalf(x)
    got = ens.get_state()
    for i in range(cfg.n_particles):
        ref = O.add_qhalf(P, x[i].astype(np.float64), np.zeros((3, cfg.ny, cfg.nx)))
        assert rel_l2(got[i], ref) < TOL


@pytest.mark.parametrize("maker", [synth.config1, ragged_config])
def test_forecast_with_cfl_and_model_error_matches_oracle(maker):
    """Model steps with CFL-chosen substeps and SOAR model error: the GPU and
    the oracle must pick the same substep counts and stay within 1e-5."""
    cfg = maker()
    ne = 4 if maker is ragged_config else cfg.n_particles
    cfg = synth.Config(**{**cfg.as_dict(), "n_particles": ne})
    U32, U64 = start_state(cfg, ne)
    P = oracle_problem(cfg)
    ens = ensemble(cfg)
    ens.set_state(U32)
    ref = U64
    for step in range(12):
        err = step % 5 != 4               # no model error before an observation time
        ens.forecast(1, err)
        nsub_gpu = ens.last_nsub()
        ref, nsub, _ = O.forecast(P, ref, 1, err, t0=step)
        assert np.array_equal(nsub_gpu, nsub[:, 0]), step
        e = rel_l2(ens.get_state(), ref)
        assert e < TOL, (step, e)
    assert ens.counters() == (12, 0)


def test_drifters_match_oracle():
    cfg = synth.config1(n_particles=3)
    U32, U64 = start_state(cfg, 3)
    P = oracle_problem(cfg)
    ens = ensemble(cfg, n_drifters_max=5)
    ens.set_state(U32)
    xy0 = synth.drifter_positions(cfg, 5)
    xy = np.repeat(xy0[None], 3, axis=0)
    ens.set_drifters(xy)
    ens.forecast(3, True)
    ref, _, rxy = O.forecast(P, U64, 3, True, t0=0, xy=xy)
    got = ens.get_drifters()
    # displacements agree to the FP32 velocity precision
    disp_g, disp_r = got - xy, rxy - xy
    assert np.max(np.abs(disp_g - disp_r)) < 1e-4 * np.max(np.abs(disp_r)) + 1e-6


def test_state_roundtrip_through_torch_device_pointers():
    torch = pytest.importorskip("torch")
    cfg = synth.config1(n_particles=2)
    U32, _ = start_state(cfg, 2)
    ens = ensemble(cfg)
    t = torch.from_numpy(U32).cuda()
    ens.set_state(t)
    out = torch.empty_like(t)
    ens.get_state(out)
    torch.cuda.synchronize()
    assert torch.equal(out, t)


def test_checkpoint_resume_is_bit_identical(tmp_path):
    cfg = synth.config1(n_particles=2)
    U32, _ = start_state(cfg, 2)
    a = ensemble(cfg)
    a.set_state(U32)
    a.forecast(2, True)
    a.save(tmp_path / "ck.bin")
    a.forecast(2, True)
    b = ensemble(cfg)
    b.load_checkpoint(tmp_path / "ck.bin")
    b.forecast(2, True)
    assert np.array_equal(a.get_state(), b.get_state())
    assert a.counters() == b.counters()


def test_nonfinite_state_is_reported():
    cfg = synth.config1(n_particles=2)
    U32, _ = start_state(cfg, 2)
    U32[1, 0, 5, 5] = np.nan
    ens = ensemble(cfg)
    ens.set_state(U32)
    with pytest.raises(iewpf.IewpfError) as e:
        ens.forecast_fixed(1, False, 2)
    assert e.value.name == "ENONFINITE"


@pytest.mark.parametrize("maker", [synth.config1, ragged_config])
def test_marching_shapes_are_bitwise_identical(maker):
    """Every tile shape of the marching scheme step, scalar or with the two
    stages paired in packed f32x2 registers, computes each cell with the same
    operations, so the results agree bit for bit."""
    cfg = maker(n_particles=3)
    U32, _ = start_state(cfg, 3)
    outs = []
    for shape in [(1, 2, 64, 4), (1, 2, 16, 2), (1, 3, 32, 8), (1, 4, 128, 1), (1, 3, 7, 3),
                  (2, 2, 64, 4), (2, 3, 16, 2), (2, 3, 256, 2), (2, 4, 128, 1), (2, 2, 7, 3)]:
        ens = ensemble(cfg)
        ens.set_stepper(*shape)
        ens.set_state(U32)
        ens.forecast_fixed(2, True, 5)
        outs.append(ens.get_state())
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


def test_autotuner_keeps_the_state():
    cfg = synth.config1(n_particles=2)
    U32, _ = start_state(cfg, 2)
    ens = ensemble(cfg)
    ens.set_state(U32)
    shape = ens.tune()
    assert shape[0] in (1, 2) and shape[1] in (2, 3, 4)
    assert np.array_equal(ens.get_state(), U32)
