"""The seeded input generators against their plain definitions (no GPU)."""
import numpy as np
import pytest

from inputs import generate as gen


def rsa_sequential(n, L, dmin, seed, batch=4096):
    """Random sequential addition written out candidate by candidate (the definition)."""
    kept = []
    t = 0
    while len(kept) < n:
        cnt = np.arange(3 * t, 3 * (t + batch), dtype=np.uint64)
        cand = gen.uniform01(gen.counter_u64(seed, gen.STREAM_RSA, cnt)).reshape(batch, 3) * L
        t += batch
        for p in cand:
            if kept:
                q = np.asarray(kept)
                dx = q - p
                dx -= L * np.round(dx / L)
                if np.any((dx * dx).sum(axis=1) < dmin * dmin):
                    continue
            kept.append(p)
            if len(kept) == n:
                break
    return np.asarray(kept)


@pytest.mark.parametrize("n,rho,dmin,seed", [(300, 1.2, 0.7, 3), (800, 1.2, 0.7, 5),
                                             (500, 0.8, 0.9, 11), (1200, 1.2, 0.62, 33)])
def test_rsa_equals_sequential_definition(n, rho, dmin, seed):
    L = gen.box_for(n, rho)
    fast = gen.rsa_positions(n, L, dmin, seed, batch=256)
    ref = rsa_sequential(n, L, dmin, seed, batch=256)
    assert np.array_equal(fast, ref)


def test_rsa_batch_size_does_not_change_the_result():
    n, L = 700, gen.box_for(700, 1.2)
    assert np.array_equal(gen.rsa_positions(n, L, 0.7, 2, batch=64),
                          gen.rsa_positions(n, L, 0.7, 2, batch=4096))


def test_rsa_minimum_distance():
    n = 5000
    L = gen.box_for(n, 1.2)
    p = gen.rsa_positions(n, L, 0.7, 1)
    from scipy.spatial import cKDTree

    d, _ = cKDTree(p % L, boxsize=L).query(p % L, k=2)
    assert d[:, 1].min() >= 0.7 - 1e-12


def test_replica_sizes_range_and_rounding():
    ns = gen.replica_sizes(64, 2048, 32768, 0)
    assert len(ns) == 64 and all(2048 <= n <= 32768 and n % 5 == 0 for n in ns)
    assert len(set(ns)) > 50  # uneven sizes
    assert ns == gen.replica_sizes(64, 2048, 32768, 0)


def test_fcc_sites_equal_the_lattice():
    L = gen.box_for(4 * 9 ** 3, 1.2)
    full = gen.fcc_lattice(9, L)
    idx = np.random.default_rng(0).permutation(full.shape[0])[:500]
    assert np.array_equal(gen.fcc_sites(9, L, idx), full[idx])


def test_fcc_jitter_is_bounded_seeded_and_counter_addressed():
    ncell, L = 6, gen.box_for(4 * 6 ** 3, 1.2)
    n = 4 * ncell ** 3
    idx = np.arange(n)
    base = gen.fcc_sites(ncell, L, idx)
    a = gen.fcc_sites(ncell, L, idx, jitter=0.05, seed=3)
    d = a - base
    assert np.abs(d).max() <= 0.05 and np.abs(d).max() > 0.045
    assert abs(d.mean()) < 0.005  # centred
    # the same draws whatever subset is asked for (counter-based), another seed differs
    sub = np.array([5, 17, n - 1])
    assert np.array_equal(gen.fcc_sites(ncell, L, sub, jitter=0.05, seed=3), a[sub])
    assert not np.array_equal(gen.fcc_sites(ncell, L, idx, jitter=0.05, seed=4), a)
