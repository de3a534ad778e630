"""Pins for the seeded input generators (no GPU)."""
import numpy as np
import pytest

import workloads as wl


def test_splitmix64_reference_outputs():
    """SplitMix64 (Steele, Lea & Flood 2014) seeded 1234567: first outputs."""
    state = np.uint64(1234567)
    outs = []
    for k in range(1, 4):
        outs.append(int(wl.mix64(np.array([state + np.uint64(k) * wl.GAMMA], np.uint64))[0]))
    assert outs == [6457827717110365317, 3203168211198807973, 9817491932198370423]


def test_draws_deterministic_and_windowed():
    a = wl.draws_range(7, 3, 1000)
    b = wl.draws_range(7, 3, 600, start=400)
    np.testing.assert_array_equal(a[400:], b)
    assert len(np.unique(a)) == 1000
    assert not np.array_equal(a, wl.draws_range(7, 4, 1000))


def test_uniform_below_range_and_mean():
    x = wl.uniform_below(wl.draws_range(1, 1, 200000), 10)
    assert x.min() == 0 and x.max() == 9
    assert abs(x.mean() - 4.5) < 0.05


@pytest.mark.parametrize("n,q", [(10, 0.99), (50, 0.9), (7, 1.0), (20, 1.5)])
def test_zipf_matches_pmf(n, q):
    """Rejection-inversion reproduces P(k) ~ k^-q (chi-square at 200k draws)."""
    z = wl.Zipf(n, q)
    k = z.sample(3, 9, 200000)
    assert k.min() >= 1 and k.max() <= n
    obs = np.bincount(k, minlength=n + 1)[1:]
    exp = z.pmf(np.arange(1, n + 1)) * k.size
    chi2 = ((obs - exp) ** 2 / exp).sum()
    assert chi2 < 3 * n + 30


def test_zipf_hot_rank_at_2_28():
    """p(rank 1) of Zipf(0.99) over 2^28 is ~1/20 (H_{N,0.99} ~ 20)."""
    z = wl.Zipf(1 << 28, 0.99)
    k = z.sample(0, 1, 400000)
    p1 = (k == 1).mean()
    assert 1 / 25 < p1 < 1 / 17


def test_rank_bijection():
    idx = wl.rank_to_index(np.arange(1, (1 << 12) + 1), 12)
    assert sorted(idx.tolist()) == list(range(1 << 12))


def test_permutation():
    p = wl.permutation(5, 5, 1000)
    assert sorted(p.tolist()) == list(range(1000))


def test_bank_round_shapes():
    b = wl.bank_round(seed=0, n_accounts=1 << 10, n_gpu=500, cpu_threads=3, cpu_tx_per_thread=20)
    assert (b.gpu_tx["src"] != b.gpu_tx["dst"]).all()
    assert b.gpu_tx["amount"].min() >= 1 and b.gpu_tx["amount"].max() <= 10
    log = b.cpu_log
    assert len(log) == 3 * 20 * 2
    assert sorted(log["ts"].tolist()) == sorted(np.repeat(np.arange(1, 61), 2).tolist())
    p = wl.bank_round(seed=0, n_accounts=1 << 10, n_gpu=500, partitioned=True,
                      cpu_threads=2, cpu_tx_per_thread=20)
    assert p.gpu_tx["src"].min() >= 512 and p.cpu_log["addr"].max() < 512


def test_validation_round_recipe():
    v = wl.validation_round(seed=1, log2_words=16, n_log=1 << 12, cpu_threads=4)
    n_gran = (1 << 16) // 16
    assert v.read_granules.size == round(0.05 * n_gran)
    assert len(np.unique(v.read_granules)) == v.read_granules.size
    assert sorted(v.log["ts"].tolist()) == list(range(1, (1 << 12) + 1))
    seg = (1 << 12) // 4
    for t in range(4):
        s = v.log["ts"][t * seg:(t + 1) * seg]
        assert (np.diff(s.astype(np.int64)) > 0).all()
    hit = np.isin(v.log["addr"] // 16, v.read_granules)
    assert hit.sum() == v.n_hits_planted
    assert np.isin(v.plant_addr // 16, v.read_granules).all()


def test_rmw_batch_distinct_addresses():
    t = wl.rmw_batch(seed=2, batch=0, n_tx=20000, log2_words=20)
    a = t["addr"]
    for i in range(4):
        for j in range(i):
            assert (a[:, i] != a[:, j]).all()
    assert 0.08 < t["flags"].mean() < 0.12
    u = wl.rmw_batch(seed=2, batch=0, n_tx=1000, log2_words=20, uniform=True, lo=100, hi=200)
    assert u["addr"].min() >= 100 and u["addr"].max() < 200


def test_cache_prefill_and_requests():
    lay = wl.CacheLayout(log2_sets=8)
    img = lay and wl.cache_prefill(lay, 1 << 11)
    keys = img[lay.key_base:lay.val_base].view(np.uint64).reshape(-1, 8)
    vals = img[lay.val_base:lay.gpu_lru_base].view(np.uint64).reshape(-1, 8)
    present = keys[keys != 0]
    assert len(np.unique(present)) == present.size
    sets = wl.set_of_key(present, 8)
    rows = np.nonzero(keys != 0)[0]
    np.testing.assert_array_equal(sets, rows)
    np.testing.assert_array_equal(vals[keys != 0], present * np.uint64(3))
    r = wl.cache_batch(seed=3, batch=0, n_req=10000, n_keys=1 << 12)
    assert r["key"].min() >= 1 and r["key"].max() <= 1 << 12
    assert 0.07 < r["op"].mean() < 0.13
