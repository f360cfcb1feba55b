"""The allocation-free projection entry point (ncs_block_dots_noalloc), for callers
that cannot call cudaMalloc, against the allocating ncs_block_dots: same results on
two calls in a row (the fixed scratch is reused), and sizes beyond its fixed scratch
are refused. Kept in a file of its own that pytest collects last."""
import numpy as np
import pytest

from paper_1906_04209_gb300 import ncs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda(libncs):
    assert torch.cuda.is_available(), "GPU test without a GPU"
    torch.cuda.set_device(0)


def _case(n, k, seed):
    rng = np.random.default_rng(seed)
    V = torch.tensor(rng.standard_normal((k, n)), device="cuda")
    w = torch.tensor(rng.standard_normal(n), device="cuda")
    return V, w


def test_noalloc_matches_allocating_entry_point_twice():
    stream = torch.cuda.current_stream().cuda_stream
    for (n, k, seed) in [(100_003, 37, 1), (65_536, 1024, 2)]:
        V, w = _case(n, k, seed)
        ref = torch.empty(k, dtype=torch.float64, device="cuda")
        out = torch.full((k,), float("nan"), dtype=torch.float64, device="cuda")
        ncs.block_dots(n, k, V.data_ptr(), n, w.data_ptr(), ref.data_ptr(), stream)
        ncs.block_dots_noalloc(n, k, V.data_ptr(), n, w.data_ptr(), out.data_ptr(), stream)
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        scale = np.sqrt(n) * float(V.abs().max()) * float(w.abs().max())
        assert np.isfinite(o).all()
        assert np.abs(o - r).max() <= 1e-12 * scale
        exact = V.cpu().numpy() @ w.cpu().numpy()
        assert np.abs(o - exact).max() <= 1e-12 * scale


def test_noalloc_refuses_more_vectors_than_its_scratch():
    V, w = _case(1000, 2, 3)
    out = torch.empty(1025, dtype=torch.float64, device="cuda")
    with pytest.raises(ncs.NcsError) as e:
        ncs.block_dots_noalloc(1000, 1025, V.data_ptr(), 1000, w.data_ptr(), out.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)
    assert e.value.code == ncs.NCS_E_INPUT
