"""Host helpers of the rank-histogram harness (Sec. 5.1), on the CPU: the
state values at integer cells and the mooring observations built from them
(eq. buoyObservation: (hu, hv) H / (H + eta) plus the observation error)."""
import numpy as np
import pytest

from paper_1910_01031_gb300 import rank_histogram, synth

torch = pytest.importorskip("torch")


def test_values_at_reads_cells_as_x_then_y():
    n, ny, nx = 2, 5, 7
    # every entry encodes (particle, field, y, x) so a swapped index shows
    U = torch.zeros((n, 3, ny, nx), dtype=torch.float32)
    for p in range(n):
        for f in range(3):
            for y in range(ny):
                for x in range(nx):
                    U[p, f, y, x] = 1000 * p + 100 * f + 10 * y + x
    cells = np.array([[3, 1], [0, 4], [6, 0]])          # (x, y)
    v = rank_histogram._values_at(torch, U, cells)
    assert v.shape == (n, len(cells), 3)
    assert v.dtype == np.float64
    for p in range(n):
        for m, (x, y) in enumerate(cells):
            for f in range(3):
                assert v[p, m, f] == 1000 * p + 100 * f + 10 * y + x


def test_observe_is_the_mooring_observation():
    cfg = synth.config_rank()
    H = cfg.H
    vals = np.array([[0.0, 2.0, -3.0],                 # eta = 0: (hu, hv) unchanged
                     [H, 4.0, 6.0],                    # eta = H: halved
                     [-0.5 * H, 1.0, -1.0]])           # eta = -H/2: doubled
    noise = np.array([[0.1, -0.2], [0.0, 0.0], [0.5, 0.5]])
    y = rank_histogram._observe(cfg, vals, noise)
    expect = np.array([[2.1, -3.2], [2.0, 3.0], [2.5, -1.5]])
    np.testing.assert_allclose(y, expect, rtol=0, atol=1e-12)
