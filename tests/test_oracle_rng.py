"""Pins of the oracle's counter-based generator (Philox4x32-10) and of its
Box-Muller normals, against things other than the oracle itself."""
import ctypes
import math
import os

import numpy as np
import pytest

from oracle import oracle as O


def _curand_host():
    for path in ("/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"):
        try:
            return ctypes.CDLL(path)
        except OSError:
            continue
    return None


def test_philox_matches_curand_host_generator():
    """cuRAND's host-side Philox4_32_10 generator (run, not read) emits the
    Philox block of counter (n // 65536, 0, n % 65536, 0) with key = seed as
    its n-th group of four words; every such block must equal ours."""
    cur = _curand_host()
    if cur is None:
        pytest.skip("libcurand not available")
    for seed in (0x0123456789ABCDEF, 42, 0xFFFFFFFFFFFFFFFF):
        # a fresh generator per seed: re-seeding keeps the stream offset
        gen = ctypes.c_void_p()
        if cur.curandCreateGeneratorHost(ctypes.byref(gen), 161) != 0:
            pytest.skip("cuRAND host generator unavailable")
        try:
            assert cur.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
            n_blocks = 2 * 65536 + 8
            out = np.zeros(4 * n_blocks, dtype=np.uint32)
            assert cur.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p),
                                      ctypes.c_size_t(out.size)) == 0
        finally:
            cur.curandDestroyGenerator(gen)
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for n in (0, 1, 2, 3, 777, 65535, 65536, 65537, 2 * 65536 + 5):
            ref = [int(x) for x in out[4 * n:4 * n + 4]]
            assert O.philox([n // 65536, 0, n % 65536, 0], key) == ref


def test_philox_counter_words_all_matter():
    key = [1, 2]
    base = O.philox([5, 6, 7, 8], key)
    for i in range(4):
        c = [5, 6, 7, 8]
        c[i] ^= 1
        assert O.philox(c, key) != base
    assert O.philox([5, 6, 7, 8], [1, 3]) != base


def test_normals_are_standard_normal():
    from scipy import stats
    z = O.normals(1234, 3, 9, 0, 200_000)
    assert abs(z.mean()) < 5 / math.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-4


def test_normals_box_muller_layout():
    """Normals 4b..4b+3 come from the Philox block (b, p, t, stream): words
    (0,1) and (2,3) form Box-Muller pairs whose squared radius is -2 ln u_a."""
    seed, p, t, s = 99, 4, 17, 2
    z = O.normals(seed, p, t, s, 40)
    for b in range(10):
        w = O.philox([b, p, t, s], [seed & 0xFFFFFFFF, seed >> 32])
        for pair in range(2):
            ua = (w[2 * pair] + 0.5) * 2.0 ** -32
            ub = (w[2 * pair + 1] + 0.5) * 2.0 ** -32
            z0, z1 = z[4 * b + 2 * pair], z[4 * b + 2 * pair + 1]
            assert math.isclose(z0 * z0 + z1 * z1, -2.0 * math.log(ua), rel_tol=1e-13)
            ang = math.atan2(z1, z0) % (2 * math.pi)
            assert math.isclose(ang, 2 * math.pi * ub, rel_tol=1e-9, abs_tol=1e-9)


def test_streams_and_particles_are_independent():
    a = O.normals(5, 0, 0, 0, 1000)
    b = O.normals(5, 1, 0, 0, 1000)
    c = O.normals(5, 0, 1, 0, 1000)
    d = O.normals(5, 0, 0, 1, 1000)
    for other in (b, c, d):
        assert abs(np.corrcoef(a, other)[0, 1]) < 0.15
