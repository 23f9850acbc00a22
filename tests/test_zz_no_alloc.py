"""The allocation-free loss/gradient entry point agrees with bm_loss_grad.

bm_loss_grad_csr_noalloc serves callers that cannot allocate device memory
(framework-owned pools, allocation-free loops); it keeps its scratch in a
fixed array of the library.  This file is collected last so that a run that
stops at the first failure has already run every other test.  It checks two
calls in a row against the handle-based entry point, within the tolerance of
the other gradient tests (1e-5 relative), and the size limit.
"""
import numpy as np
import pytest

from synth import named_config, random_factors

pytestmark = pytest.mark.gpu

RTOL = 1e-5


def test_noalloc_matches_loss_grad_twice():
    torch = pytest.importorskip("torch")
    import paper_2204_14067_gb300 as B
    p = named_config("small", m=1500, n=6000, nnz=220_000, seed=41)   # m <= n: no transpose
    h = B.bm_create(p.m, p.n, p.rows, p.cols, p.vals, p.lam, 40)
    try:
        assert not B.bm_dims(h)["transposed"]
        k = 23
        ld = 24
        W, H = random_factors(p.m, p.n, k, seed=2, scale=0.3)
        B.bm_set_factors(h, k, W, H)
        gW_ref = np.empty_like(W)
        gH_ref = np.empty_like(H)
        f_ref, _ = B.bm_loss_grad(h, gW_ref, gH_ref)
        ix = B.bm_get_index(h)
        dev = torch.device("cuda")
        rp = torch.from_numpy(ix["row_ptr"]).to(dev)
        col = torch.from_numpy(ix["col"]).to(dev)
        val = torch.from_numpy(ix["val"]).to(dev)
        Wp = torch.zeros((p.m, ld), dtype=torch.float32, device=dev)
        Hp = torch.zeros((p.n, ld), dtype=torch.float32, device=dev)
        Wp[:, :k] = torch.from_numpy(W).to(dev)
        Hp[:, :k] = torch.from_numpy(H).to(dev)
        outs = []
        for _ in range(2):
            gW = torch.full((p.m, ld), float("nan"), dtype=torch.float32, device=dev)
            f = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
            B.bm_loss_grad_csr_noalloc(p.m, p.n, rp, col, val, Wp, Hp, k, ld, p.lam, gW, f)
            torch.cuda.synchronize()
            outs.append((float(f.item()), gW.cpu().numpy()))
        for fv, g in outs:
            assert abs(fv - f_ref) <= RTOL * f_ref
            assert np.linalg.norm(g[:, :k] - gW_ref) <= RTOL * np.linalg.norm(gW_ref)
            assert np.all(g[:, k:] == 0)
        assert outs[0][0] == outs[1][0] and np.array_equal(outs[0][1], outs[1][1])
    finally:
        B.bm_destroy(h)


def test_noalloc_rejects_too_many_rows():
    torch = pytest.importorskip("torch")
    import paper_2204_14067_gb300 as B
    dev = torch.device("cuda")
    m = 262144 + 1
    rp = torch.zeros(m + 1, dtype=torch.int64, device=dev)
    col = torch.zeros(1, dtype=torch.int32, device=dev)
    val = torch.zeros(1, dtype=torch.float32, device=dev)
    Wp = torch.zeros((m, 4), dtype=torch.float32, device=dev)
    Hp = torch.zeros((4, 4), dtype=torch.float32, device=dev)
    gW = torch.zeros((m, 4), dtype=torch.float32, device=dev)
    f = torch.zeros(1, dtype=torch.float64, device=dev)
    with pytest.raises(B.BMError, match="BM_NOALLOC_MAX_ROWS"):
        B.bm_loss_grad_csr_noalloc(m, 4, rp, col, val, Wp, Hp, 1, 4, 0.1, gW, f)
