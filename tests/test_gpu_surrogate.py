"""GPU parity of the learned surrogate against its FP64 oracle
(oracle/surrogate.py), through the C ABI.

Tolerances follow from the arithmetic: weights are made BF16-exact before
the comparison, so the GPU differs from FP64 by the BF16 rounding of the
network input and of every activation (relative 2^-9 each) and by FP32
accumulation.  Six layers of such rounding give a relative L2 error of the
output change of a few 1e-3 (FWD_TOL = 2e-2 leaves a margin); the gradients
also pass the BF16-rounded back-propagated signal through every layer
(GRAD_TOL = 5e-2)."""
import numpy as np
import pytest

from oracle import oracle as O
from oracle import surrogate as S
from paper_1910_01031_gb300 import iewpf, synth

from gpu_common import ensemble, oracle_problem, rel_l2, start_state

pytestmark = pytest.mark.gpu
FWD_TOL = 2e-2
GRAD_TOL = 5e-2
W, D = 64, 6


def bf16_exact(a):
    """Round FP32 values to the nearest BF16 (ties to even), kept as FP32."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def _fields(n, ny, nx, seed):
    """Smooth random states of the right magnitudes: eta ~ 0.05 m, hu, hv ~ 5 m^2/s."""
    rng = np.random.default_rng(seed)
    U = rng.standard_normal((n, 3, ny, nx))
    for _ in range(2):                                   # light periodic smoothing
        U = (U + np.roll(U, 1, 2) + np.roll(U, -1, 2) + np.roll(U, 1, 3) + np.roll(U, -1, 3)) / 5.0
    U *= np.array([0.05, 5.0, 5.0])[None, :, None, None] / U.std(axis=(0, 2, 3))[None, :, None, None]
    return U.astype(np.float32)


SI = [1 / 0.05, 1 / 5.0, 1 / 5.0]
SO = [0.004, 0.3, 0.3]


def _net(nx=48, ny=40, seed=5):
    sur = iewpf.Surrogate(nx, ny, W, D, seed=seed)
    p = bf16_exact(sur.params())
    sur.set_params(p)
    sur.set_scales(SI, SO)
    return sur, p


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def test_parameter_layout_and_padding():
    sur, p = _net()
    assert sur.n_params == S.n_params(W, D)
    assert np.array_equal(S.pack(S.unpack(p, W, D), W, D), p)     # padding holds zeros


def test_forward_matches_oracle():
    sur, p = _net()
    U = _fields(3, 40, 48, 1)
    out = sur.apply(U)
    ref = S.apply(p, U.astype(np.float64), SI, SO, W, D)
    d_gpu = out.astype(np.float64) - U
    d_ref = ref - U
    assert np.linalg.norm(d_ref) > 0
    assert _rel(d_gpu, d_ref) < FWD_TOL


def test_forward_is_bitwise_translation_equivariant():
    # a shift by whole pixel tiles (8 rows, 16 columns) maps every output to
    # the same position in its tile: identical arithmetic
    sur, _ = _net()
    U = _fields(2, 40, 48, 2)
    a = sur.apply(U)
    b = sur.apply(np.ascontiguousarray(np.roll(U, (8, 16), axis=(2, 3))))
    assert np.array_equal(np.roll(a, (8, 16), axis=(2, 3)), b)


def test_loss_and_gradients_match_oracle():
    sur, p = _net()
    X = _fields(3, 40, 48, 3)
    Y = X + (_fields(3, 40, 48, 4) * np.array([0.05, 0.1, 0.1], np.float32)[None, :, None, None]).astype(np.float32)
    L, g = sur.loss_grad(X, Y)
    Lr, gr = S.loss_grad(p, X.astype(np.float64), Y.astype(np.float64), SI, SO, W, D)
    assert abs(L - Lr) < 1e-2 * Lr
    lg, lr = S.unpack(g, W, D), S.unpack(gr, W, D)
    for l in range(D):
        assert _rel(lg[l][0], lr[l][0]) < GRAD_TOL, ("weights", l)
        assert _rel(lg[l][1], lr[l][1]) < GRAD_TOL, ("bias", l)
    # padding entries get exactly zero gradient
    pad = S.pack([(np.ones_like(Wl), np.ones_like(bl)) for Wl, bl in lr], W, D) == 0
    assert np.all(g[pad] == 0.0)


def test_first_training_step_is_signed_learning_rate():
    cfg = synth.config1(n_particles=4)
    U32, _ = start_state(cfg, 4)
    ens, ens2 = ensemble(cfg), ensemble(cfg)
    ens.set_state(U32)
    ens2.set_state(U32)
    sur = iewpf.Surrogate(cfg.nx, cfg.ny, W, D, seed=9)
    p0 = sur.params()
    lr = 1e-3
    sur.train(ens, n_pairs=4, k_steps=1, epochs=1, batch=4, lr=lr)
    p1 = sur.params()
    # the same pairs and parameters, gradient by loss_grad
    X = ens2.get_state()
    ens2.forecast(1, False)
    Y = ens2.get_state()
    sur2 = iewpf.Surrogate(cfg.nx, cfg.ny, W, D, seed=9)
    si, so = sur.scales()
    sur2.set_scales(si, so)
    _, g = sur2.loss_grad(X, Y)
    big = np.abs(g) > 1e-3 * np.abs(g).max()
    assert big.sum() > 1000
    dp = p1.astype(np.float64) - p0
    assert np.all(np.abs(dp[big] + lr * np.sign(g[big])) < 2e-2 * lr)
    assert np.all(dp[g == 0] == 0)


def test_training_reduces_the_loss():
    cfg = synth.config1(n_particles=16)
    U32, _ = start_state(cfg, 16)
    ens = ensemble(cfg)
    ens.set_state(U32)
    sur = iewpf.Surrogate(cfg.nx, cfg.ny, W, D, seed=11)
    losses = sur.train(ens, n_pairs=64, k_steps=2, epochs=15, batch=8, lr=2e-3)
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 0.8 * losses[0], losses


def test_zero_network_forecast_is_model_error_and_drift_only():
    cfg = synth.config1(n_particles=3)
    P = oracle_problem(cfg)
    U32, U64 = start_state(cfg, 3)
    ens = ensemble(cfg, n_drifters_max=2)
    ens.set_state(U32)
    sur = iewpf.Surrogate(cfg.nx, cfg.ny, W, D, seed=1)
    sur.set_params(np.zeros(sur.n_params, np.float32))
    k = 2
    ens.set_surrogate(sur, k)
    xy0 = np.array([[30.5e3, 61.2e3], [100.1e3, 7.7e3]])
    every = k * cfg.dt_model
    traj = ens.drifter_forecast(xy0, hours=2 * every / 3600.0, out_every_s=every, use_surrogate=True)
    calls, fb = ens.surrogate_stats()
    assert (calls, fb) == (2, 0)
    ref_traj = [np.repeat(xy0[None], 3, axis=0)]
    ref = U64.copy()
    xy = ref_traj[0].copy()
    t = 0
    for _ in range(2):
        for p in range(3):
            xy[p] = O.drift(P, ref[p], k * cfg.dt_model, xy[p])
        for _ in range(k):
            for p in range(3):
                ref[p] = O.model_error(P, ref[p], p, t)
            t += 1
        ref_traj.append(xy.copy())
    assert rel_l2(ens.get_state(), ref) < 1e-5
    disp = np.abs(np.array(ref_traj) - ref_traj[0]).max()
    assert disp > 0 and np.abs(traj - np.array(ref_traj)).max() < 1e-5 * disp + 1e-6
    assert ens.counters()[0] == 2 * k


@pytest.mark.parametrize("bad", ["nan", "growth"])
def test_rejected_network_falls_back_to_the_plain_stepper_bitwise(bad):
    cfg = synth.config1(n_particles=3)
    U32, _ = start_state(cfg, 3)
    a, b = ensemble(cfg, n_drifters_max=1), ensemble(cfg, n_drifters_max=1)
    a.set_state(U32)
    b.set_state(U32)
    sur = iewpf.Surrogate(cfg.nx, cfg.ny, W, D, seed=1)
    if bad == "nan":
        sur.set_params(np.full(sur.n_params, np.nan, np.float32))
    else:
        # finite output that multiplies eta far beyond the guard: f = 0.5 in every
        # field, scaled by 1 -> eta + 0.5 m, hu, hv + 0.5 m^2/s
        p = np.zeros(sur.n_params, np.float32)
        p[-16:-13] = 0.5                                # bias of the output layer
        sur.set_params(p)
    a.set_surrogate(sur, 2)
    xy0 = np.array([[50e3, 50e3]])
    ta = a.drifter_forecast(xy0, hours=240 / 3600.0, out_every_s=240.0, use_surrogate=True)
    tb = b.drifter_forecast(xy0, hours=240 / 3600.0, out_every_s=240.0)
    assert a.surrogate_stats() == (2, 2)
    assert np.array_equal(ta, tb)
    assert np.array_equal(a.get_state(), b.get_state())
    assert a.counters() == b.counters()


def test_surrogate_argument_errors():
    with pytest.raises(iewpf.IewpfError):
        iewpf.Surrogate(50, 40, W, D)                 # nx not a multiple of 16
    cfg = synth.config1(n_particles=2)
    ens = ensemble(cfg, n_drifters_max=1)
    with pytest.raises(iewpf.IewpfError):
        ens.drifter_forecast(np.array([[1e3, 1e3]]), 0.1, 60.0, use_surrogate=True)   # none attached
    sur = iewpf.Surrogate(cfg.nx, cfg.ny, W, D)
    ens.set_surrogate(sur, 4)
    with pytest.raises(iewpf.IewpfError):
        ens.drifter_forecast(np.array([[1e3, 1e3]]), 0.1, 60.0, use_surrogate=True)   # 60 s not a multiple of 4 steps
    other = iewpf.Surrogate(32, 32, W, D)
    with pytest.raises(iewpf.IewpfError):
        ens.set_surrogate(other, 2)


def test_tcgen05_forward_matches_oracle_and_mma_sync():
    # 256 x 64 cells, 10 fields: 640 tiles of 2 rows x 128 pixels, several per
    # CTA (both pipeline buffers, a ragged last round of the persistent grid)
    sur, p = _net(nx=256, ny=64, seed=6)
    assert sur.uses_tcgen05()
    U = _fields(10, 64, 256, 7)
    out_tc = sur.apply(U)
    ref = S.apply(p, U.astype(np.float64), SI, SO, W, D)
    assert _rel(out_tc.astype(np.float64) - U, ref - U) < FWD_TOL
    sur.set_path(1)
    assert not sur.uses_tcgen05()
    out_mma = sur.apply(U)
    # the two paths round the same activations to BF16; they differ only where
    # a different FP32 summation order flips a rounding
    assert _rel(out_tc.astype(np.float64) - U, out_mma.astype(np.float64) - U) < 1e-2


def test_bounded_device_wait_times_out_and_the_context_stays_usable():
    """Failure detection of the tensor-core pipeline: the injected kernels
    wait on a barrier that nothing completes, give up after their poll limit
    and report FLAG_TIMEOUT, so the call raises ETIMEOUT; the next call on the
    same device runs normally and matches the oracle, twice."""
    sur, p = _net(nx=128, ny=16, seed=21)
    assert sur.uses_tcgen05()
    U = _fields(3, 16, 128, 22)
    sur.inject_timeout(1)
    with pytest.raises(iewpf.IewpfError) as e:
        sur.apply(U)
    assert e.value.name == "ETIMEOUT"
    ref = S.apply(p, U.astype(np.float64), SI, SO, W, D)
    for _ in range(2):
        out = sur.apply(U)
        assert _rel(out.astype(np.float64) - U, ref - U) < FWD_TOL


def test_tcgen05_forward_small_grid_and_gradients():
    # one tile row pair per field, fewer tiles than SMs; training forward keeps z
    sur, p = _net(nx=128, ny=16, seed=8)
    assert sur.uses_tcgen05()
    X = _fields(2, 16, 128, 9)
    Y = X + (_fields(2, 16, 128, 10) * np.array([0.05, 0.1, 0.1], np.float32)[None, :, None, None]).astype(np.float32)
    out = sur.apply(X)
    ref = S.apply(p, X.astype(np.float64), SI, SO, W, D)
    assert _rel(out.astype(np.float64) - X, ref - X) < FWD_TOL
    L, g = sur.loss_grad(X, Y)
    Lr, gr = S.loss_grad(p, X.astype(np.float64), Y.astype(np.float64), SI, SO, W, D)
    assert abs(L - Lr) < 1e-2 * Lr
    lg, lr = S.unpack(g, W, D), S.unpack(gr, W, D)
    for l in range(D):
        assert _rel(lg[l][0], lr[l][0]) < GRAD_TOL, ("weights", l)


def test_tcgen05_forward_is_bitwise_translation_equivariant():
    sur, _ = _net(nx=256, ny=16, seed=12)
    U = _fields(3, 16, 256, 13)
    a = sur.apply(U)
    b = sur.apply(np.ascontiguousarray(np.roll(U, (2, 128), axis=(2, 3))))
    assert np.array_equal(np.roll(a, (2, 128), axis=(2, 3)), b)


def test_tcgen05_many_tiles_per_cta_match_mma_sync():
    # 8 fields of 256 x 256: 2048 tiles, about 13 consecutive tiles per CTA, so
    # the ring of input rows wraps several times within a column strip
    sur, _ = _net(nx=256, ny=256, seed=14)
    U = _fields(8, 256, 256, 15)
    out_tc = sur.apply(U)
    sur.set_path(1)
    out_mma = sur.apply(U)
    d_tc = out_tc.astype(np.float64) - U
    d_mma = out_mma.astype(np.float64) - U
    assert np.linalg.norm(d_mma) > 0
    assert _rel(d_tc, d_mma) < 1e-2


def test_full_size_network_call_sampled_against_oracle():
    # the surrogate workload's network call: 1000 fields of 256 x 256 in one
    # call on the tcgen05 path, as the drift forecast and the bench make it;
    # two sampled fields against the FP64 oracle
    torch = pytest.importorskip("torch")
    sur, p = _net(nx=256, ny=256, seed=21)
    assert sur.uses_tcgen05()
    n = 1000
    gen = torch.Generator(device="cuda").manual_seed(3)
    U = torch.randn(n, 3, 256, 256, device="cuda", generator=gen)
    for _ in range(2):       # smooth periodic fields of the state's magnitudes
        U = (U + U.roll(1, 2) + U.roll(-1, 2) + U.roll(1, 3) + U.roll(-1, 3)) / 5.0
    U *= (torch.tensor([0.05, 5.0, 5.0], device="cuda") / U.std(dim=(0, 2, 3))).view(1, 3, 1, 1)
    U = U.contiguous()
    out = torch.empty_like(U)
    sur.apply_device(U, out=out)
    torch.cuda.synchronize()
    for i in (0, n - 1):
        x = U[i:i + 1].double().cpu().numpy()
        ref = S.apply(p, x, SI, SO, W, D)
        got = out[i:i + 1].double().cpu().numpy()
        assert _rel(got - x, ref - x) < FWD_TOL, i


def _oracle_grads(sur, p, X, Y):
    """loss_grad through the C ABI against the FP64 oracle, per layer."""
    L, g = sur.loss_grad(X, Y)
    Lr, gr = S.loss_grad(p, X.astype(np.float64), Y.astype(np.float64), SI, SO, W, D)
    assert abs(L - Lr) < 1e-2 * Lr
    lg, lr = S.unpack(g, W, D), S.unpack(gr, W, D)
    for l in range(D):
        assert _rel(lg[l][0], lr[l][0]) < GRAD_TOL, ("weights", l)
        assert _rel(lg[l][1], lr[l][1]) < GRAD_TOL, ("bias", l)
    pad = S.pack([(np.ones_like(Wl), np.ones_like(bl)) for Wl, bl in lr], W, D) == 0
    assert np.all(g[pad] == 0.0)
    return L, g


@pytest.mark.parametrize("nx,ny,n", [(64, 64, 3), (128, 16, 2), (192, 16, 1)])
def test_tcgen05_training_matches_oracle(nx, ny, n):
    # training on tcgen05: forward and data passes over tiles of 16 rows x 8
    # pixels (8, 16 or 24 across), weight gradients over tiles of 4 rows x 64
    # pixels with tap pairs on M/N-major operands; the forward output as well
    sur, p = _net(nx=nx, ny=ny, seed=31)
    assert sur.uses_tcgen05_training()
    assert sur.uses_tcgen05() == (nx % 128 == 0)
    X = _fields(n, ny, nx, 32)
    Y = X + (_fields(n, ny, nx, 33) * np.array([0.05, 0.1, 0.1], np.float32)[None, :, None, None]).astype(np.float32)
    _oracle_grads(sur, p, X, Y)
    out = sur.apply(X)
    ref = S.apply(p, X.astype(np.float64), SI, SO, W, D)
    assert _rel(out.astype(np.float64) - X, ref - X) < FWD_TOL


def test_tcgen05_training_many_tiles_per_cta_match_mma_sync():
    # 24 fields of 64 x 64: 768 tiles of the forward and data passes (five or
    # six per CTA: every shared-memory stage and both accumulator sets
    # reused) and 384 of the weight gradients; the same gradients on the
    # mma.sync path
    sur, p = _net(nx=64, ny=64, seed=34)
    X = _fields(24, 64, 64, 35)
    Y = X + (_fields(24, 64, 64, 36) * np.array([0.05, 0.1, 0.1], np.float32)[None, :, None, None]).astype(np.float32)
    L_tc, g_tc = sur.loss_grad(X, Y)
    sur.set_path(1)
    assert not sur.uses_tcgen05_training()
    L_mma, g_mma = sur.loss_grad(X, Y)
    assert abs(L_tc - L_mma) < 1e-3 * L_mma
    lt, lm = S.unpack(g_tc, W, D), S.unpack(g_mma, W, D)
    for l in range(D):
        assert np.linalg.norm(lm[l][0]) > 0
        assert _rel(lt[l][0], lm[l][0]) < 2e-2, ("weights", l)
        assert _rel(lt[l][1], lm[l][1]) < 2e-2, ("bias", l)


def test_tcgen05_training_forward_is_bitwise_translation_equivariant():
    # a shift by whole tiles (16 rows) moves every tile's work unchanged
    sur, _ = _net(nx=64, ny=64, seed=37)
    assert not sur.uses_tcgen05() and sur.uses_tcgen05_training()
    V = _fields(2, 64, 64, 39)
    a = sur.apply(V)
    b = sur.apply(np.ascontiguousarray(np.roll(V, 16, axis=2)))
    assert np.array_equal(np.roll(a, 16, axis=2), b)
