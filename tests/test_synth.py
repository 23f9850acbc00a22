"""The seeded input generators against the recipes they state (CPU): the
recommendation-shaped Zipf matrices (exact nnz, distinct in-range pairs,
row degrees water-filled within [1, n/2], integer ratings in range,
heavy-tailed degrees, lambda = 0.05 max|A|), the planted uniform problem,
the water-filling itself, the serving stream, and that every array is a
function of the parameters and the seed alone."""
import numpy as np
import pytest

from synth import gen
from synth import named_config, planted_uniform, random_factors, serving_requests


def _distinct_pairs(rows, cols, n):
    key = rows.astype(np.int64) * n + cols.astype(np.int64)
    return np.unique(key).shape[0] == key.shape[0]


@pytest.mark.parametrize("m, n, nnz", [(6000, 1500, 200_000), (900, 5000, 150_000), (2000, 60, 50_000)])
def test_zipf_matrix_follows_its_recipe(m, n, nnz):
    p = named_config("small", m=m, n=n, nnz=nnz, seed=11)
    assert (p.m, p.n, p.nnz) == (m, n, nnz)
    assert p.rows.dtype == np.int32 and p.cols.dtype == np.int32 and p.vals.dtype == np.float32
    assert p.rows.min() >= 0 and p.rows.max() < m and p.cols.min() >= 0 and p.cols.max() < n
    assert _distinct_pairs(p.rows, p.cols, n)
    deg = np.bincount(p.rows, minlength=m)
    assert deg.min() >= 1 and deg.max() <= max(1, n // 2) and deg.sum() == nnz
    assert np.all(p.vals == np.round(p.vals)) and p.vals.min() >= 1 and p.vals.max() <= 5
    assert p.lam == pytest.approx(0.05 * float(np.abs(p.vals).max()))
    # heavy tails: the busiest column holds many times the mean column degree
    # (where a column can: at most m entries fit in one)
    cdeg = np.bincount(p.cols, minlength=n)
    if 5 * cdeg.mean() <= m:
        assert cdeg.max() >= 5 * cdeg.mean()
    else:
        assert cdeg.max() == m


def test_generators_depend_on_the_seed_alone():
    a = named_config("small", m=3000, n=800, nnz=100_000, seed=3)
    b = named_config("small", m=3000, n=800, nnz=100_000, seed=3)
    c = named_config("small", m=3000, n=800, nnz=100_000, seed=4)
    for x, y in ((a.rows, b.rows), (a.cols, b.cols), (a.vals, b.vals)):
        assert np.array_equal(x, y)
    assert not (np.array_equal(a.rows, c.rows) and np.array_equal(a.cols, c.cols))
    W1, H1 = random_factors(50, 40, 3, seed=7)
    W2, H2 = random_factors(50, 40, 3, seed=7)
    assert np.array_equal(W1, W2) and np.array_equal(H1, H2) and W1.dtype == np.float32


def test_planted_uniform_problem():
    p = named_config("tiny")
    assert (p.m, p.n, p.nnz) == (500, 300, 15_000) and p.lam == 0.5 and p.k_init == 8
    assert _distinct_pairs(p.rows, p.cols, p.n)
    q = planted_uniform(m=40, n=30, rank=2, frac=0.6, noise_sd=0.0, seed=9)
    assert q.nnz == 720 and _distinct_pairs(q.rows, q.cols, q.n)
    # noise-free values are the planted rank-2 product: every fully observed
    # 3 x 3 minor vanishes (to the float32 rounding of the stored values)
    M = np.full((40, 30), np.nan)
    M[q.rows, q.cols] = q.vals
    obs = np.isfinite(M)
    found = 0
    for a in range(0, 40, 3):
        for b in range(a + 1, 40, 5):
            for c in range(b + 1, 40, 7):
                common = np.nonzero(obs[a] & obs[b] & obs[c])[0]
                if common.shape[0] >= 3:
                    S = M[np.ix_([a, b, c], common[:3])].astype(np.float64)
                    assert abs(np.linalg.det(S)) <= 1e-5 * np.prod(np.linalg.norm(S, axis=1))
                    found += 1
    assert found >= 20


@pytest.mark.parametrize("total, cap", [(1000, 40), (5000, 100), (200, 1)])
def test_waterfill_degrees(total, cap):
    rng = np.random.default_rng(1)
    w = rng.pareto(1.2, 200) + 1e-3
    d = gen._waterfill(w, total, cap=cap, floor=1)
    assert d.sum() == total and d.min() >= 1 and d.max() <= cap
    # heavier weights never get fewer entries (up to the one unit of rounding)
    order = np.argsort(w)
    assert np.all(np.diff(d[order]) >= -1)
    with pytest.raises(ValueError):
        gen._waterfill(w, 100, cap=cap, floor=1)          # below one entry per row
    with pytest.raises(ValueError):
        gen._waterfill(w, 200 * cap + 1, cap=cap, floor=1)


def test_serving_stream_within_its_ranges():
    probs, arr = serving_requests(count=12, seed=4, m_range=(1000, 4000), n_range=(500, 2000),
                                  density_range=(0.002, 0.02), rate=5.0, max_nnz=60_000,
                                  lam_grid2=(3.0, 5.0, 8.0))
    assert len(probs) == 12 and np.all(np.diff(arr) > 0)
    for p in probs:
        assert 1000 <= p.m <= 4000 and 500 <= p.n <= 2000
        assert max(p.m, p.n) <= p.nnz <= max(60_000, p.m, p.n)
        assert _distinct_pairs(p.rows, p.cols, p.n)
        assert p.k_max == min(32, p.m, p.n)
        ratio = p.lam / float(np.abs(p.vals).max())
        assert any(abs(ratio - g) <= 1e-9 * g for g in (0.02, 0.05, 0.1, 0.2, 0.5, 3.0, 5.0, 8.0))
