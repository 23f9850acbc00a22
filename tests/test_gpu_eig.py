"""The one-block symmetric eigensolver (bm_sym_eig) in its three modes against
LAPACK's eigh in FP64 (sizes on both sides of the divide-and-conquer
range 24 ... 150 of mode 0), on the spectra the PG step produces: random
symmetric, graded positive definite (Rayleigh-Ritz matrices of Algorithm 2,
whose Ritz values span many decades), clustered and rank-deficient Grams
(Eq. "orth-W"), a diagonal input and a single entry.

Checked: eigenvalues (absolute error against ||S|| in mode 0, relative error
of a positive definite spectrum in modes 1 and 2), descending order, the
residual ||S V - V diag(evals)||_F / ||S||_F, orthogonality of V, and for
eigenvalues separated by more than 1e-3 ||S|| the vectors themselves (up to
sign)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

EPS32 = float(np.finfo(np.float32).eps)


@pytest.fixture(scope="module")
def B():
    import paper_2204_14067_gb300 as B
    B.lib()
    return B


def _orth(n, rng):
    q, r = np.linalg.qr(rng.standard_normal((n, n)))
    return q * np.sign(np.diag(r))


def _spectrum(kind, n, rng):
    if kind == "random":
        a = rng.standard_normal((n, n))
        return (a + a.T) / 2
    if kind == "graded":     # positive definite, 1e4 ... 1e-4
        lam = 1e4 * 10.0 ** (-8.0 * np.arange(n) / max(n - 1, 1))
    elif kind == "cluster":  # half the values near 1 (within 1e-7), the rest tiny
        lam = np.where(np.arange(n) < n // 2, 1.0 + 1e-7 * np.arange(n), 1e-9 * np.arange(n))
    elif kind == "deficient":  # a PSD Gram of rank n // 3
        x = rng.standard_normal((n, max(1, n // 3)))
        return x @ x.T
    else:                    # diagonal with repeated values
        return np.diag(rng.integers(-3, 4, size=n).astype(np.float64))
    u = _orth(n, rng)
    return (u * lam) @ u.T


def _run(B, S, mode):
    torch = pytest.importorskip("torch")
    n = S.shape[0]
    Sd = torch.from_numpy(np.ascontiguousarray(S)).cuda()
    ev = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    V = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
    B.bm_sym_eig(Sd, ev, V, mode)
    torch.cuda.synchronize()
    return ev.cpu().numpy(), V.cpu().numpy()


def _check_common(S, ev, V, n):
    assert np.all(np.isfinite(ev)) and np.all(np.isfinite(V))
    assert np.all(np.diff(ev) <= 0), "eigenvalues must leave sorted descending"
    nS = np.linalg.norm(S)
    res = np.linalg.norm(S @ V - V * ev) / max(nS, 1e-300)
    orth = np.abs(V.T @ V - np.eye(n)).max()
    assert res <= 20 * np.sqrt(n) * EPS32, res
    assert orth <= 20 * np.sqrt(n) * EPS32, orth


@pytest.mark.parametrize("n", [1, 2, 3, 16, 23, 24, 65, 130, 150, 151, 200, 256])
@pytest.mark.parametrize("kind", ["random", "graded", "cluster", "deficient", "diagonal"])
def test_fast_mode_against_eigh(B, n, kind):
    rng = np.random.default_rng(1000 * n + len(kind))
    S = _spectrum(kind, n, rng)
    ev, V = _run(B, S, 0)
    ref, U = np.linalg.eigh(S)
    ref, U = ref[::-1], U[:, ::-1]
    norm2 = max(np.abs(ref).max(), 1e-300)
    assert np.abs(ev - ref).max() <= 8 * np.sqrt(n) * EPS32 * norm2
    _check_common(S, ev, V, n)
    # vectors of well separated eigenvalues, up to sign
    gap = np.full(n, np.inf)
    if n > 1:
        d = np.abs(np.diff(ref))
        gap[:-1] = d
        gap[1:] = np.minimum(gap[1:], d)
    sep = gap > 1e-3 * norm2
    if sep.any():
        # angle between the computed and the exact vector (Davis-Kahan: the
        # residual over the gap); the computed vectors' norms differ from 1
        # by the orthogonality error, so they are normalised first
        v = V[:, sep] / np.linalg.norm(V[:, sep], axis=0)
        cos = np.minimum(np.abs(np.sum(v * U[:, sep], axis=0)), 1.0)
        sin = np.sqrt(1.0 - cos * cos)
        assert np.all(sin <= 10 * np.sqrt(n) * EPS32 * norm2 / gap[sep]), (sin * gap[sep] / norm2).max()


@pytest.mark.parametrize("n", [16, 65, 130, 160])
@pytest.mark.parametrize("mode", [1, 2])
def test_refined_modes_accuracy(B, n, mode):
    """Modes 1 and 2 on a graded positive definite spectrum (1e4 ... 1e-4, the
    shape of the Rayleigh-Ritz matrices, whose small Ritz values near the
    threshold lambda * alpha decide the rank).

    Mode 1 (FP32 refinement sweeps) resolves each eigenvalue to a few units
    of FP32 rounding relative to itself, down to the sweeps' absolute floor:
    rotations stop below 2e-9 ||S||_F (the relative threshold 2e-6 times
    1e-3).  Measured on GB300 for n = 16 ... 160: relative error <= 5.2e-8
    for lam / lam_1 > 1e-2, absolute error <= 1.5e-8 ||S||_F everywhere.
    Mode 2 (FP64 sweeps for n <= 112, FP64 Householder + QL above):
    relative error <= 4.4e-12, absolute <= 1.6e-12 ||S||_F.  The bounds are
    those figures times about four to ten."""
    rng = np.random.default_rng(7 * n + mode)
    u = _orth(n, rng)
    lam = 1e4 * 10.0 ** (-8.0 * np.arange(n) / (n - 1))
    S = (u * lam) @ u.T
    ev, V = _run(B, S, mode)
    fro = np.linalg.norm(S)
    if mode == 1:
        bound = 4 * EPS32 * lam + 8e-9 * fro
    else:
        bound = 1e-10 * lam + 1e-11 * fro
    err = np.abs(ev - lam)
    assert np.all(err <= bound), (err / bound).max()
    _check_common(S, ev, V, n)


def test_rejects_bad_arguments(B):
    torch = pytest.importorskip("torch")
    S = torch.eye(4, dtype=torch.float64, device="cuda")
    ev = torch.empty(4, dtype=torch.float64, device="cuda")
    V = torch.empty((4, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(B.BMError):
        B.bm_sym_eig(S, ev, V, 3)
    with pytest.raises(B.BMError):
        B.bm_sym_eig(S.cpu(), ev, V, 0)
