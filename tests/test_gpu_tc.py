"""Tensor-core (tcgen05 kind::tf32, 3xTF32 split) GEMM behind the per-patch operator
contractions, through the C ABI: against an FP64 numpy product on ragged sizes, and
the FP32 product with and without tensor cores."""
import numpy as np
import pytest

from oracle import operator as O
from oracle.kernels import INTERIOR
from paper_1906_04209_gb300 import layouts as L, ncs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda(libncs):
    assert torch.cuda.is_available(), "GPU test without a GPU"
    torch.cuda.set_device(0)


@pytest.mark.parametrize("rows,cols,kdim", [(300, 200, 136), (1, 17, 5), (129, 130, 33), (256, 128, 496),
                                            (1000, 700, 136)])
def test_tc_gemm(rows, cols, kdim):
    rng = np.random.default_rng(rows + cols + kdim)
    A = rng.standard_normal((rows, kdim)).astype(np.float32)
    B = rng.standard_normal((cols, kdim)).astype(np.float32)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    Ad = torch.tensor(A, device="cuda")
    Bd = torch.tensor(B, device="cuda")
    Dd = torch.full((rows, cols), float("nan"), dtype=torch.float32, device="cuda")
    ncs.tc_gemm_f32(rows, cols, kdim, Ad.data_ptr(), Bd.data_ptr(), Dd.data_ptr(),
                    torch.cuda.current_stream().cuda_stream)
    D = Dd.cpu().numpy().astype(np.float64)
    scale = np.sqrt(kdim) * np.abs(A).max() * np.abs(B).max()
    assert np.isfinite(D).all()
    assert np.abs(D - ref).max() <= 2e-6 * scale


def test_fp32_product_with_and_without_tensor_cores(small_pre):
    N = 300
    c = L.uniform(N, 0.03, L.rng(99))
    pre = small_pre(INTERIOR, eps=0.03)
    x = np.random.default_rng(17).standard_normal(N * pre.K)
    out = {}
    for tc in (0, 1):
        ctx = ncs.Context(pre.eps, pre.mode, pre.K,
                          operator=(pre.idr.T, pre.idr.t_skel, pre.idr.th_skel, pre.op.I),
                          method=ncs.METHOD_DIRECT, tensor_cores=tc)
        ctx.set_patches(c)
        out[tc] = ctx.matvec(x, ncs.FP32)
    ref = O.id_matvec(pre, c, x)
    scale = np.abs(ref).max()
    assert np.abs(out[1] - ref).max() <= 5e-6 * scale
    assert np.abs(out[1] - out[0]).max() <= 5e-6 * scale
