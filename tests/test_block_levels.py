"""Levels of the 7 x 7 local blocks (Sec. 4.6): overlapping blocks act in
observation order, blocks that share no coarse point commute, so a fixed
layout is applied level by level.  The library's host-side schedule against
a reference built from the blocks' actual cell sets on the periodic coarse
grid (no distance rule), on random layouts, at the wrap, along overlap
chains and on the two mooring layouts of the benchmark (no GPU needed)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1910_01031_gb300 import iewpf, synth


def reference_levels(block0, nRx, nRy):
    """level(l) = 1 + the highest level among earlier blocks that share a
    coarse point with block l (-1 + 1 = 0 when none): each coarse point keeps
    the highest level of the blocks that covered it so far."""
    last = np.full((nRy, nRx), -1, dtype=np.int64)
    out = []
    for a, b in np.asarray(block0).reshape(-1, 2):
        ys = (b + np.arange(-3, 4)) % nRy
        xs = (a + np.arange(-3, 4)) % nRx
        v = int(last[np.ix_(ys, xs)].max()) + 1
        out.append(v)
        last[np.ix_(ys, xs)] = np.maximum(last[np.ix_(ys, xs)], v)
    return np.array(out)


@pytest.mark.parametrize("nRx,nRy,n,seed", [(5, 6, 12, 1), (7, 13, 20, 2), (12, 12, 30, 3), (13, 14, 40, 4),
                                            (40, 25, 60, 5), (171, 171, 200, 6)])
def test_random_layouts_match_the_cell_sets(nRx, nRy, n, seed):
    rng = np.random.default_rng(seed)
    b0 = np.stack([rng.integers(0, nRx, n), rng.integers(0, nRy, n)], axis=1)
    b0[n // 2] = b0[0]                       # a repeated centre
    got = iewpf.block_levels(b0, nRx, nRy)
    assert np.array_equal(got, reference_levels(b0, nRx, nRy))


def test_distance_six_overlaps_seven_does_not_across_the_wrap():
    n = 40
    assert list(iewpf.block_levels([[1, 5], [n - 5, 5]], n, n)) == [0, 1]       # 6 apart through the seam
    assert list(iewpf.block_levels([[1, 5], [n - 6, 5]], n, n)) == [0, 0]       # 7 apart
    assert list(iewpf.block_levels([[3, 0], [3, n - 6]], n, n)) == [0, 1]
    assert list(iewpf.block_levels([[3, 0], [3, n - 7]], n, n)) == [0, 0]
    # overlapping in x only is no overlap
    assert list(iewpf.block_levels([[3, 3], [5, 20]], n, n)) == [0, 0]


def test_a_chain_of_overlaps_gives_one_level_per_block():
    # centres 5 apart: each block meets only its predecessor, so the order
    # forces a new level every time
    b0 = [[5 * k, 7] for k in range(8)]
    assert list(iewpf.block_levels(b0, 64, 30)) == list(range(8))
    # the same blocks in the order 0, 2, 4, ..., 1, 3, ...: two levels
    b1 = [[5 * k, 7] for k in list(range(0, 8, 2)) + list(range(1, 8, 2))]
    assert list(iewpf.block_levels(b1, 64, 30)) == [0] * 4 + [1] * 4


@pytest.mark.parametrize("which", ["headline", "coupled"])
def test_mooring_layouts(which):
    cfg = synth.config4() if which == "headline" else synth.coupled_moorings()
    spacing = 26 if which == "headline" else synth.COUPLED_SPACING
    cells = synth.mooring_cells(cfg, spacing)
    c = cfg.c_omega
    nRx, nRy = -(-cfg.nx // c), -(-cfg.ny // c)
    b0 = np.array([[O.nearest_coarse(cfg.nx, nRx, c, int(x)), O.nearest_coarse(cfg.ny, nRy, c, int(y))]
                   for x, y in cells])
    got = iewpf.block_levels(b0, nRx, nRy)
    assert np.array_equal(got, reference_levels(b0, nRx, nRy))
    if which == "headline":
        assert got.max() == 0                # 26 cells = 8.7 coarse points apart: one level
    else:
        assert got.max() >= 1


def test_arguments_are_checked():
    with pytest.raises(iewpf.IewpfError):
        iewpf.block_levels([[0, 0]], 0, 5)
    with pytest.raises(iewpf.IewpfError):
        iewpf.block_levels([[5, 0]], 5, 5)
    assert iewpf.block_levels(np.zeros((0, 2), np.int32), 5, 5).size == 0
