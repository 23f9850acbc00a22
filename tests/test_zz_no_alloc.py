"""The allocation-free loss/gradient entry point.

bm_loss_grad_csr_noalloc serves callers that cannot allocate device memory
where they need a gradient (code running inside another framework's memory
pool, allocation-free loops, callers holding only borrowed buffers); it keeps
its scratch in a fixed array of the library.  This file is collected last so
that a run that stops at the first failure has already run every other test.

Checked, for several ranks and row strides (which select different kernel
instances, including row widths whose float4 chunk count is not a multiple
of four), on two calls in a row:
  * against the handle-based entry point bm_loss_grad, within the tolerance
    of the other gradient tests (1e-5 relative, row by row);
  * against the FP64 oracle's loss and gradient, element-wise per row;
  * that both calls give identical results (the shared scratch is rewritten).
Also: the row limit and misaligned buffers are rejected before any launch.
"""
import numpy as np
import pytest

from oracle import bm_oracle as O
from synth import named_config, random_factors
from tests.parity import assert_rows_close, grad_rounding_scales

pytestmark = pytest.mark.gpu

RTOL = 1e-5


@pytest.fixture(scope="module")
def prob():
    return named_config("small", m=1500, n=6000, nnz=220_000, seed=41)   # m <= n: no transpose


@pytest.mark.parametrize("k,ld", [(23, 24), (37, 40), (64, 64), (127, 128)])
def test_noalloc_matches_loss_grad_and_oracle_twice(prob, k, ld):
    torch = pytest.importorskip("torch")
    import paper_2204_14067_gb300 as B
    p = prob
    h = B.bm_create(p.m, p.n, p.rows, p.cols, p.vals, p.lam, 127)
    try:
        assert not B.bm_dims(h)["transposed"]
        W, H = random_factors(p.m, p.n, k, seed=2, scale=0.3)
        B.bm_set_factors(h, k, W, H)
        gW_ref = np.empty_like(W)
        gH_ref = np.empty_like(H)
        f_ref, _ = B.bm_loss_grad(h, gW_ref, gH_ref)
        ix = B.bm_get_index(h)
        oix = O.build_index(p.m, p.n, p.rows, p.cols, p.vals.astype(np.float64))
        f_o, _, gW_o, _, r_o = O.loss_grad(oix, W.astype(np.float64), H.astype(np.float64), p.lam)
        aW, _ = grad_rounding_scales(oix, r_o, W, H, p.lam)
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
            assert_rows_close(g[:, :k], gW_ref, RTOL, what="gW vs bm_loss_grad", extra=aW)
            assert abs(fv - f_o) <= RTOL * f_o
            assert_rows_close(g[:, :k], gW_o, RTOL, what="gW vs oracle", extra=aW)
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


def test_noalloc_rejects_misaligned_buffers_and_huge_lambda():
    """A view with a storage offset of one float is not 16-byte aligned: the
    call returns BM_ERR_INVALID before anything is launched."""
    torch = pytest.importorskip("torch")
    import paper_2204_14067_gb300 as B
    dev = torch.device("cuda")
    m, n, ld = 8, 8, 4
    rp = torch.zeros(m + 1, dtype=torch.int64, device=dev)
    col = torch.zeros(1, dtype=torch.int32, device=dev)
    val = torch.zeros(1, dtype=torch.float32, device=dev)
    f = torch.zeros(1, dtype=torch.float64, device=dev)
    good_W = torch.zeros((m, ld), dtype=torch.float32, device=dev)
    good_H = torch.zeros((n, ld), dtype=torch.float32, device=dev)
    good_g = torch.zeros((m, ld), dtype=torch.float32, device=dev)
    base = torch.zeros(m * ld + 1, dtype=torch.float32, device=dev)
    off = base[1:].view(m, ld)                        # 4-byte offset
    assert off.data_ptr() % 16 != 0
    for W, H, g in ((off, good_H, good_g), (good_W, off, good_g), (good_W, good_H, off)):
        with pytest.raises(B.BMError, match="16-byte"):
            B.bm_loss_grad_csr_noalloc(m, n, rp, col, val, W, H, 1, ld, 0.1, g, f)
    with pytest.raises(B.BMError, match="lambda"):
        B.bm_loss_grad_csr_noalloc(m, n, rp, col, val, good_W, good_H, 1, ld, 1e300, good_g, f)
