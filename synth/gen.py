"""Seeded generators for the matrix-completion workloads.

Every array here is a function of (shape parameters, seed) only.  The
generators use numpy's Philox bit generator so that the same call gives the
same bytes on x86 and on Arm.  Nothing in this file evaluates the objective,
a gradient or a proximal step.

Workload shapes follow the matrix-completion experiments of the paper
(Sec. 5.1, Table "data"): a small planted-rank problem with uniformly
sampled entries, and recommendation-shaped problems whose row and column
degrees follow a Zipf law with integer ratings.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

MASK64 = (1 << 64) - 1


@dataclasses.dataclass
class Problem:
    """One observed matrix in the caller's orientation (m x n, 0-based COO)."""

    name: str
    m: int
    n: int
    rows: np.ndarray  # int32 [nnz]
    cols: np.ndarray  # int32 [nnz]
    vals: np.ndarray  # float32 [nnz]
    lam: float
    k_init: int
    k_max: int
    seed: int
    recipe: str

    @property
    def nnz(self) -> int:
        return int(self.rows.shape[0])


def _rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[seed & MASK64, stream & MASK64]))


def _round_half_away(x: np.ndarray) -> np.ndarray:
    return np.sign(x) * np.floor(np.abs(x) + 0.5)


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------
def planted_uniform(m=500, n=300, rank=5, frac=0.10, noise_sd=0.1, lam=0.5, k_init=8,
                    k_max=None, seed=0, factor_var=1.0 / math.sqrt(5.0), name="planted") -> Problem:
    """Planted low-rank matrix with uniformly sampled observations.

    W*, H* entries are N(0, factor_var) (the second argument of N(.,.) read as a
    variance), |Omega| = round(frac*m*n) entries drawn uniformly without
    replacement, A = W* H*^T + N(0, noise_sd^2) on Omega.
    """
    rng = _rng(seed, 1)
    sd = math.sqrt(factor_var)
    Ws = rng.standard_normal((m, rank)) * sd
    Hs = rng.standard_normal((n, rank)) * sd
    nnz = int(round(frac * m * n))
    flat = np.sort(rng.choice(m * n, size=nnz, replace=False))
    flat = rng.permutation(flat)  # callers receive COO in no particular order
    rows = (flat // n).astype(np.int32)
    cols = (flat % n).astype(np.int32)
    vals = np.einsum("ij,ij->i", Ws[rows], Hs[cols]) + noise_sd * rng.standard_normal(nnz)
    if k_max is None:
        k_max = min(m, n, 64)
    return Problem(name, m, n, rows, cols, vals.astype(np.float32), float(lam), int(k_init),
                   int(k_max), seed,
                   f"planted rank {rank}, factors N(0,{factor_var:.4g}), {frac:.0%} uniform, noise sd {noise_sd}")


def _zipf_weights(count: int, s: float, rng: np.random.Generator) -> np.ndarray:
    rank = rng.permutation(count).astype(np.float64) + 1.0
    return rank ** (-s)


def _waterfill(w: np.ndarray, total: int, cap: int, floor: int = 1) -> np.ndarray:
    """Integer degrees d_i = clip(c*w_i, floor, cap) summing exactly to total."""
    count = w.shape[0]
    if not (floor * count <= total <= cap * count):
        raise ValueError("total outside [floor*count, cap*count]")
    lo, hi = 0.0, 1.0
    while np.clip(hi * w, floor, cap).sum() < total:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if np.clip(mid * w, floor, cap).sum() < total:
            lo = mid
        else:
            hi = mid
    real = np.clip(lo * w, floor, cap)
    d = np.floor(real).astype(np.int64)
    rem = total - int(d.sum())
    if rem > 0:
        frac = real - d
        frac[d >= cap] = -1.0
        order = np.lexsort((np.arange(count), -frac))
        d[order[:rem]] += 1
    assert int(d.sum()) == total and d.max() <= cap and d.min() >= floor
    return d


def _class_counts(deg_u: np.ndarray, size: np.ndarray, wc: np.ndarray) -> np.ndarray:
    """Integer counts K[u, c] <= size[c] with sum_c K[u, c] = deg_u[u], proportional
    to the class weights wc and water-filled where a class saturates."""
    lo = np.zeros(deg_u.shape[0])
    hi = np.full(deg_u.shape[0], 1.0)
    while True:
        s = np.minimum(size[None, :], hi[:, None] * wc[None, :]).sum(1)
        if np.all(s >= deg_u):
            break
        hi = np.where(s >= deg_u, hi, hi * 2.0)
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        s = np.minimum(size[None, :], mid[:, None] * wc[None, :]).sum(1)
        below = s < deg_u
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    real = np.minimum(size[None, :], hi[:, None] * wc[None, :])
    K = np.minimum(np.floor(real).astype(np.int64), size[None, :])
    rem = deg_u - K.sum(1)
    frac = np.where(K < size[None, :], real - K, -1.0)
    order = np.argsort(-frac, axis=1, kind="stable")
    rank = np.empty_like(order)
    np.put_along_axis(rank, order, np.arange(K.shape[1])[None, :].repeat(K.shape[0], 0), axis=1)
    K += (rank < rem[:, None]) & (frac >= 0)
    assert np.all(K.sum(1) == deg_u) and np.all(K <= size[None, :])
    return K


def _sample_columns(deg: np.ndarray, colw: np.ndarray, rng: np.random.Generator):
    """Choose deg[r] distinct columns for every row r, favouring heavy columns.

    Columns are ranked by weight and grouped into classes of ranks
    [2^c - 1, 2^(c+1) - 1).  Row r takes from class c a count proportional to
    the class weight (water-filled where a class is exhausted), and picks
    them as a strided walk (o + t*g) mod |class| through a random permutation
    of the class, with a random offset o and a random odd stride g (g = 1 in
    the last, non power-of-two class).  The walk never repeats, so every
    row's columns are distinct without a sort, and the work is O(nnz).
    """
    m = deg.shape[0]
    n = colw.shape[0]
    order = np.argsort(-colw, kind="stable")
    bounds = [0]
    while bounds[-1] < n:
        bounds.append(min(n, 2 * bounds[-1] + 1))
    bounds = np.array(bounds, dtype=np.int64)
    size = np.diff(bounds)
    wc = np.add.reduceat(colw[order], bounds[:-1])
    ncls = size.shape[0]
    # a random permutation inside each class
    slot = order.copy()
    for c in range(ncls):
        slot[bounds[c]:bounds[c + 1]] = rng.permutation(order[bounds[c]:bounds[c + 1]])
    deg_u, inv = np.unique(deg, return_inverse=True)
    K = _class_counts(deg_u.astype(np.float64), size.astype(np.float64), wc).astype(np.int64)
    Kr = K[inv]                                   # m x ncls
    pr, pc = np.nonzero(Kr)                       # (row, class) pairs in row-major order
    pk = Kr[pr, pc]
    psize = size[pc]
    off = np.floor(rng.random(pr.shape[0]) * psize).astype(np.int64)
    g = 2 * np.floor(rng.random(pr.shape[0]) * np.maximum(1, psize // 2)).astype(np.int64) + 1
    pow2 = (psize & (psize - 1)) == 0
    g = np.where(pow2, g % np.maximum(psize, 1), 1)
    g = np.where(g == 0, 1, g)
    start = np.cumsum(pk) - pk
    total = int(pk.sum())
    rows = np.repeat(pr.astype(np.int32), pk)
    t = np.arange(total, dtype=np.int64) - np.repeat(start, pk)
    local = (np.repeat(off, pk) + t * np.repeat(g, pk)) % np.repeat(psize, pk)
    cols = slot[np.repeat(bounds[pc], pk) + local].astype(np.int32)
    return rows, cols


def zipf_ratings(m, n, nnz, rank, mean, sd, lo, hi, noise_sd=0.0, zipf_s=1.2, lam=None,
                 lam_frac=0.05, k_init=8, k_max=64, seed=1, name="zipf", shuffle=False) -> Problem:
    """Recommendation-shaped matrix with Zipf(zipf_s) row and column degrees.

    Row and column weights are rank^-s over random permutations.  Row degrees
    are water-filled to exactly nnz with 1 <= d <= n//2; each row's columns
    are spread over popularity classes in proportion to the class weight
    (see _sample_columns).  Values are
    round(clip(mean + sd*z + noise, lo, hi)) with z the planted rank-`rank`
    product <w*_i, h*_j> (N(0,1) factors) standardised over Omega; rounding is
    half away from zero.  lam defaults to lam_frac * max|A|.
    """
    rng = _rng(seed, 2)
    roww = _zipf_weights(m, zipf_s, rng)
    colw = _zipf_weights(n, zipf_s, rng)
    deg = _waterfill(roww, nnz, cap=max(1, n // 2), floor=1)
    rows, cols = _sample_columns(deg, colw, rng)
    Ws = rng.standard_normal((m, rank)).astype(np.float32)
    Hs = rng.standard_normal((n, rank)).astype(np.float32)
    x = np.empty(nnz, dtype=np.float64)
    step = 1 << 22
    for s in range(0, nnz, step):
        e = min(nnz, s + step)
        x[s:e] = np.einsum("ij,ij->i", Ws[rows[s:e]], Hs[cols[s:e]], dtype=np.float64)
    mu = x.mean()
    sg = x.std()
    z = (x - mu) / (sg if sg > 0 else 1.0)
    del x
    v = mean + sd * z
    if noise_sd > 0:
        v += noise_sd * rng.standard_normal(nnz)
    vals = _round_half_away(np.clip(v, lo, hi)).astype(np.float32)
    del v, z
    if shuffle:
        p = rng.permutation(nnz)
        rows, cols, vals = rows[p], cols[p], vals[p]
    if lam is None:
        lam = lam_frac * float(np.abs(vals).max())
    recipe = (f"Zipf({zipf_s}) degrees, rank-{rank} planted ratings mean {mean} sd {sd} "
              f"noise {noise_sd} clipped to [{lo},{hi}]")
    return Problem(name, m, n, rows, cols, vals, float(lam), int(k_init), int(k_max), seed, recipe)


def named_config(name: str, **kw) -> Problem:
    """The workloads by name.

    tiny     : 500 x 300 planted rank 5, 10% uniform, lambda 0.5, k0 = 8
    tiny5    : same matrix, lambda 5 (planted-rank recovery case)
    netflix  : 480,189 x 17,770, 100,480,507 Zipf(1.2) ratings 1..5, k <= 64
    netflix_quarter : 120,047 x 17,770, 25,120,127 ratings, the same recipe (a
               quarter of the users and entries: profiling captures)
    yahoo    : 1,000,990 x 624,961, 252,800,275 ratings 0..100, k <= 128
    small    : a scaled netflix-shaped case for parity runs (kw: m, n, nnz)
    """
    if name == "tiny":
        return planted_uniform(seed=0, lam=0.5, name=name, **kw)
    if name == "tiny5":
        return planted_uniform(seed=0, lam=5.0, name=name, **kw)
    if name == "netflix":
        return zipf_ratings(480_189, 17_770, 100_480_507, rank=20, mean=3.6, sd=1.0, lo=1, hi=5,
                            k_max=64, seed=1, name=name, **kw)
    if name == "netflix_quarter":
        return zipf_ratings(120_047, 17_770, 25_120_127, rank=20, mean=3.6, sd=1.0, lo=1, hi=5,
                            k_max=64, seed=1, name=name, **kw)
    if name == "yahoo":
        return zipf_ratings(1_000_990, 624_961, 252_800_275, rank=32, mean=50.0, sd=20.0, lo=0,
                            hi=100, noise_sd=10.0, k_max=128, seed=2, name=name, **kw)
    if name == "small":
        m = kw.pop("m", 6000)
        n = kw.pop("n", 1500)
        nnz = kw.pop("nnz", 200_000)
        seed = kw.pop("seed", 5)
        return zipf_ratings(m, n, nnz, rank=8, mean=3.6, sd=1.0, lo=1, hi=5, seed=seed,
                            name=name, **kw)
    raise KeyError(name)


def random_factors(m: int, n: int, k: int, seed: int, scale: float = 0.3):
    """W (m x k), H (n x k) with N(0, scale^2) entries, float32."""
    rng = _rng(seed, 3)
    W = (scale * rng.standard_normal((m, k))).astype(np.float32)
    H = (scale * rng.standard_normal((n, k))).astype(np.float32)
    return W, H


@dataclasses.dataclass
class PairProblem:
    """Distance data on a point set: pairs (i < j) with noisy distances d_ij."""

    name: str
    n: int
    i: np.ndarray      # int32 [npairs]
    j: np.ndarray      # int32 [npairs]
    d: np.ndarray      # float32 [npairs]
    X_true: np.ndarray  # float64 [n, 3]
    seed: int
    recipe: str

    @property
    def npairs(self) -> int:
        return int(self.i.shape[0])


def self_avoiding_chain(n=30_000, cutoff=6.0, noise=0.10, exclusion=1.0, seed=3, name="chain") -> PairProblem:
    """3-D self-avoiding random walk with unit bonds; all pairs within `cutoff`.

    Each step draws a direction uniformly on the sphere and is redrawn while
    the new point lies within `exclusion` of any earlier, non-bonded point
    (checked through a uniform grid of cell size `exclusion`).  Omega is every
    pair i < j at true distance <= cutoff; d_ij = true * (1 + U(-noise, noise)).
    """
    import scipy.spatial

    rng = _rng(seed, 4)
    X = np.zeros((n, 3))
    cells: dict = {}

    def key(p):
        return (int(np.floor(p[0] / exclusion)), int(np.floor(p[1] / exclusion)), int(np.floor(p[2] / exclusion)))

    cells.setdefault(key(X[0]), []).append(0)
    for t in range(1, n):
        for _ in range(1000):
            v = rng.standard_normal(3)
            p = X[t - 1] + v / np.linalg.norm(v)
            c = key(p)
            ok = True
            for dx in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dz in (-1, 0, 1):
                        for q in cells.get((c[0] + dx, c[1] + dy, c[2] + dz), ()):
                            if q != t - 1 and np.sum((X[q] - p) ** 2) < exclusion ** 2:
                                ok = False
                                break
                        if not ok:
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if ok:
                break
        X[t] = p
        cells.setdefault(c, []).append(t)
    tree = scipy.spatial.cKDTree(X)
    pairs = np.array(sorted(tree.query_pairs(cutoff)), dtype=np.int64)
    dtrue = np.sqrt(np.sum((X[pairs[:, 0]] - X[pairs[:, 1]]) ** 2, axis=1))
    d = dtrue * (1.0 + rng.uniform(-noise, noise, size=dtrue.shape[0]))
    return PairProblem(name, n, pairs[:, 0].astype(np.int32), pairs[:, 1].astype(np.int32), d.astype(np.float32),
                       X, seed, f"3-D self-avoiding walk, unit bonds, exclusion {exclusion}, pairs within {cutoff}, "
                                f"d = true*(1+U(-{noise},{noise}))")


def serving_requests(count=2000, seed=4, m_range=(1_000, 200_000), n_range=(500, 20_000),
                     density_range=(0.001, 0.02), rank_range=(2, 16), lam_grid=(0.02, 0.05, 0.1, 0.2, 0.5),
                     rate=None, k_max=32, max_nnz=None, lam_grid2=None, share2=0.5):
    """A stream of completion requests: m, n and the density log-uniform in
    their ranges, nnz = density*m*n (capped at max_nnz), planted rank uniform
    in rank_range, ratings as in the recommendation workload, lambda = a grid
    value times max|A|; with lam_grid2, a share `share2` of the requests
    (chosen by a separate draw) takes its lambda from lam_grid2 instead;
    arrival times from a Poisson process of the given rate (requests per
    second; None: all at 0).  Returns (problems, arrivals)."""
    rng = _rng(seed, 5)
    lu = lambda lo, hi, size: np.exp(rng.uniform(np.log(lo), np.log(hi), size))
    ms = np.round(lu(*m_range, count)).astype(np.int64)
    ns = np.round(lu(*n_range, count)).astype(np.int64)
    ds = lu(*density_range, count)
    ranks = rng.integers(rank_range[0], rank_range[1] + 1, count)
    lams = rng.choice(np.asarray(lam_grid), count)
    if lam_grid2 is not None:
        rng2 = _rng(seed, 6)
        pick = rng2.uniform(size=count) < share2
        lams = np.where(pick, rng2.choice(np.asarray(lam_grid2), count), lams)
    probs = []
    for t in range(count):
        m, n = int(ms[t]), int(ns[t])
        nnz = int(round(ds[t] * m * n))
        if max_nnz is not None:
            nnz = min(nnz, max_nnz)
        nnz = max(nnz, max(m, n))
        nnz = min(nnz, m * (n // 2))
        p = zipf_ratings(m, n, nnz, rank=int(ranks[t]), mean=3.6, sd=1.0, lo=1, hi=5, seed=seed * 100003 + t,
                         lam_frac=float(lams[t]), k_max=min(k_max, m, n), name=f"req{t}", shuffle=True)
        probs.append(p)
    if rate is None:
        arrivals = np.zeros(count)
    else:
        arrivals = np.cumsum(rng.exponential(1.0 / rate, count))
    return probs, arrivals
