"""hlu_rhs_manufactured_noalloc (fixed device scratch, no allocation) against
hlu_rhs_manufactured, through the C ABI.  Collected last on purpose: it must
pass alone and after every other test."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-13  # atomics change only the order of the additions


@pytest.fixture(scope="module")
def hlu():
    import __graft_entry__ as g
    g.build()
    from paper_2211_11303_gb300 import hlu as H
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return H


@pytest.mark.parametrize("n,kappa", [(2, 1.0), (5, 3.0), (24, 8.0)])  # 24: the largest mesh the scratch holds
def test_noalloc_rhs_matches_allocating_entry(hlu, n, kappa):
    h = hlu.hlu_build(n, kappa, 32, 2.0, 1e-4)
    try:
        N = hlu.hlu_n(h)
        ref = torch.zeros(N, dtype=torch.float64, device="cuda")
        hlu.hlu_rhs_manufactured(h, ref)
        warm = torch.zeros(N, dtype=torch.float64, device="cuda")
        hlu.hlu_rhs_manufactured_noalloc(h, warm)  # first call on the device: set-up
        torch.cuda.synchronize()
        outs = [torch.full((N,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(2)]
        free0 = torch.cuda.mem_get_info()[0]
        for b in outs:  # two calls in a row
            hlu.hlu_rhs_manufactured_noalloc(h, b)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        scale = float(ref.abs().max())
        assert scale > 0
        for b in [warm] + outs:
            assert torch.isfinite(b).all()
            assert float((b - ref).abs().max()) <= RTOL * scale
    finally:
        hlu.hlu_destroy(h)


def test_noalloc_rhs_rejects_meshes_beyond_the_scratch(hlu):
    h = hlu.hlu_build(25, 1.0, 64, 2.0, 1e-2)
    try:
        b = torch.full((hlu.hlu_n(h),), 7.0, dtype=torch.float64, device="cuda")
        with pytest.raises(hlu.HluError):
            hlu.hlu_rhs_manufactured_noalloc(h, b)
        torch.cuda.synchronize()
        assert bool((b == 7.0).all())  # nothing written
    finally:
        hlu.hlu_destroy(h)
