"""The tensor-core delayed update on CTA pairs (GB_OPT_TC_UPDATE = 2).

The two CTAs of a cluster compute a 256 x 256 tile with pair MMAs (M = 256,
tcgen05 cta_group::2): each stages 128 rows of A and half of B, and each
CTA's tensor memory holds its 128 x 256 half of the accumulator.  Every
product and every accumulation order is the same as with one CTA per
128 x 256 tile, so:

* small-integer operands (exact products and sums) reproduce C - X op(Y) bit
  for bit, over shapes that leave the second tile of the last pair outside
  the matrix, ragged columns, one row, lower and full updates;
* on random operands the cluster kernel equals the one-CTA kernel bit for bit;
* factorizations run with the cluster update equal those run with the
  one-CTA update bit for bit.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DEV = "cuda:0"


@pytest.fixture(scope="module")
def h():
    from paper_1812_02056_gb300 import _build, binding
    _build.build()
    hd = binding.Handle(0)
    yield hd
    hd.close()


def _update(h, dt, lower, kxn, C, X, Y, mode):
    from paper_1812_02056_gb300 import binding
    prev = h.get_option(binding.GB_OPT_TC_UPDATE)
    h.set_option(binding.GB_OPT_TC_UPDATE, mode)
    try:
        M, N = C.shape
        st = h.gb_rank_update(binding.DTYPES[dt], lower, kxn, M, N, X.shape[1], C, C.stride(0), X,
                              X.stride(0), Y, Y.stride(0))
        binding.check(st, "gb_rank_update")
        torch.cuda.synchronize()
    finally:
        h.set_option(binding.GB_OPT_TC_UPDATE, prev)
    return C


def test_option_range(h):
    from paper_1812_02056_gb300 import binding
    assert h.get_option(binding.GB_OPT_TC_UPDATE) == 2  # the pair kernel is the default
    for v in (0, 1, 2):
        h.set_option(binding.GB_OPT_TC_UPDATE, v)
        assert h.get_option(binding.GB_OPT_TC_UPDATE) == v
    assert h.lib.gb_set_option(h.h, binding.GB_OPT_TC_UPDATE, 3) == -3
    assert h.lib.gb_set_option(h.h, binding.GB_OPT_TC_UPDATE, -1) == -3
    assert h.get_option(binding.GB_OPT_TC_UPDATE) == 2


@pytest.mark.parametrize("dt", ["mix_bf16", "mix_f16", "mix_bf16x3"])
@pytest.mark.parametrize("M,N,K,lower,kxn", [
    (300, 300, 117, 1, 0),    # 3 row tiles: the last pair's second tile is empty
    (129, 129, 16, 1, 0),     # 2 row tiles, one pair
    (520, 520, 1024, 1, 0),   # 5 row tiles, deep K
    (1, 1, 1, 1, 0),
    (200, 520, 64, 0, 1),     # ragged columns, K x N operand
    (384, 256, 200, 0, 1),    # 3 row tiles, full update
    (77, 333, 1000, 0, 0),    # one row tile
    (1100, 700, 96, 0, 0)])   # 9 row tiles, 3 column tiles
def test_cluster_exact_integers(h, dt, M, N, K, lower, kxn):
    g = torch.Generator().manual_seed(M * 5 + N * 11 + K)
    X = torch.randint(-4, 5, (M, K), generator=g).float()
    Y = torch.randint(-4, 5, (K, N) if kxn else (N, K), generator=g).float()
    if lower and M == N:
        Y = X.clone()
    C0 = torch.randint(-1000, 1000, (M, N), generator=g).float()
    P = X.double() @ (Y.double() if kxn else Y.double().T)
    exp = C0.double() - P
    C = _update(h, dt, lower, kxn, C0.to(DEV), X.to(DEV), Y.to(DEV), 2).cpu().double()
    if lower:
        mask = torch.tril(torch.ones(M, N, dtype=torch.bool))
        assert torch.equal(C[mask], exp[mask])
        assert torch.equal(C[~mask], C0.double()[~mask])
    else:
        assert torch.equal(C, exp)


@pytest.mark.parametrize("dt", ["mix_bf16", "mix_f16", "mix_bf16x3"])
@pytest.mark.parametrize("M,N,K,lower,kxn", [(1000, 1000, 256, 1, 0), (515, 515, 117, 1, 0),
                                             (640, 384, 320, 0, 1), (2048, 2048, 512, 1, 0)])
def test_cluster_equals_single_cta(h, dt, M, N, K, lower, kxn):
    g = torch.Generator().manual_seed(3 * M + K)
    X = torch.randn((M, K), generator=g)
    Y = X.clone() if (lower and M == N) else torch.randn((K, N) if kxn else (N, K), generator=g)
    C0 = torch.randn((M, N), generator=g) * 10
    Xd, Yd = X.to(DEV), Y.to(DEV)
    C1 = _update(h, dt, lower, kxn, C0.to(DEV), Xd, Yd, 1)
    C2 = _update(h, dt, lower, kxn, C0.to(DEV), Xd, Yd, 2)
    assert torch.equal(C1, C2)


@pytest.mark.parametrize("dt", ["mix_bf16", "mix_bf16x3"])
@pytest.mark.parametrize("kind", ["chol", "lu"])
def test_factorization_with_cluster_update(h, dt, kind):
    from paper_1812_02056_gb300 import binding, inputs as I
    n, s = 1500, 256
    A = I.spd_gram(n, 21) if kind == "chol" else I.lu_diag_dominant(n, 21)
    Ad = torch.from_numpy(A).to(DEV)
    f = h.chol_factor if kind == "chol" else h.lu_factor
    h.set_option(binding.GB_OPT_TC_UPDATE, 1)
    try:
        F1, info1 = f(Ad, s, dt)
    finally:
        h.set_option(binding.GB_OPT_TC_UPDATE, 2)
    F2, info2 = f(Ad, s, dt)
    assert int(info1.item()) == 0 and int(info2.item()) == 0
    assert torch.equal(F1, F2)
