"""Dense k-wide Grams C = A^T B (bm_dense_gram) in the three arithmetic modes
against the FP64 product, element by element, relative to the sum of the
absolute products |A|^T |B| (the scale FP32 rounding works on).

Measured on GB300 (this file's shapes): FP32 pipes <= 5e-8, compensated
<= 2e-14, tensor cores (bfloat16 slices, tcgen05.mma) <= 2.7e-6 with one
accumulator and <= 5e-7 with the small slice products in their own
accumulator.  The bounds are those figures times about four."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

BOUND = {0: 2e-7, 1: 1e-13, 2: 1e-5}
SHAPES = [(1000, 64, 64, True), (1000, 64, 65, False), (4097, 3, 17, False), (20000, 130, 130, True),
          (20000, 64, 130, False), (333, 200, 256, False), (1, 5, 7, False), (250_000, 65, 65, True)]


@pytest.fixture(scope="module")
def B():
    import paper_2204_14067_gb300 as B
    B.lib()
    return B


@pytest.mark.parametrize("L,a,b,sym", SHAPES)
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_dense_gram_modes(B, L, a, b, sym, mode):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(L + a + b)
    lda = (a + 3) // 4 * 4
    An = rng.standard_normal((L, lda)).astype(np.float32)
    if sym:
        b, Bn = a, An
    else:
        Bn = rng.standard_normal((L, (b + 3) // 4 * 4)).astype(np.float32)
    A = torch.from_numpy(An).cuda()
    Bt = A if sym else torch.from_numpy(Bn).cuda()
    C = torch.full((a, b), float("nan"), dtype=torch.float64, device="cuda")
    B.bm_dense_gram(A, Bt, C, mode)
    ref = An[:, :a].astype(np.float64).T @ Bn[:, :b].astype(np.float64)
    scale = np.abs(An[:, :a].astype(np.float64)).T @ np.abs(Bn[:, :b].astype(np.float64))
    err = float(np.max(np.abs(C.cpu().numpy() - ref) / np.maximum(scale, 1e-300)))
    assert err <= BOUND[mode], (mode, err)


def test_dense_gram_rejects_bad_arguments(B):
    torch = pytest.importorskip("torch")
    A = torch.zeros((16, 8), device="cuda")
    C = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(B.BMError):
        B.bm_dense_gram(A, A, C, 3)                                   # unknown mode
    wide = torch.zeros((16, 260), device="cuda")
    Cw = torch.zeros((257, 257), dtype=torch.float64, device="cuda")
    with pytest.raises(B.BMError):
        B.bm_dense_gram(wide, wide, Cw, 2)                            # wider than 256 (and than lda)
    off = torch.zeros(16 * 8 + 1, device="cuda")[1:].view(16, 8)
    with pytest.raises(B.BMError, match="16-byte"):
        B.bm_dense_gram(off, A, C, 2)
