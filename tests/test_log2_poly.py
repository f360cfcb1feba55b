"""The FP32 log2 polynomial of the pair kernels (lg2_poly): its coefficients in the
CUDA header are the ones the committed fit produces, and its FP32 evaluation (step for
step as in the kernel) stays within its stated error bound."""
import importlib.util
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1906_04209_gb300", "csrc")


def _gen():
    spec = importlib.util.spec_from_file_location("gen_log2_poly", os.path.join(CSRC, "gen_log2_poly.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_header_coefficients_match_fit():
    g = _gen()
    c = g.fit()
    src = open(os.path.join(CSRC, "device_common.cuh")).read()
    body = src[src.index("float lg2_poly("):]
    body = body[:body.index("return")]
    vals = [float(v) for v in re.findall(r"([-+]?\d\.\d+e[-+]\d+)f", body)]
    # Horner order: highest coefficient first
    assert np.array_equal(np.float32(vals), c[::-1])


def test_error_bound():
    g = _gen()
    c = g.fit()
    x = np.exp(np.linspace(np.log(1e-6), np.log(1e6), 400_001)).astype(np.float32)
    x = np.concatenate([x, np.float32([0.5, 1.0, 2.0, np.sqrt(0.5), np.sqrt(2.0), 1e-30, 3e38])])
    tr = np.log2(x.astype(np.float64))
    y = g.eval32(c, x).astype(np.float64)
    small = np.abs(tr) < 1
    assert np.abs(y - tr)[small].max() <= 1e-7
    ulp = np.spacing(np.abs(tr).astype(np.float32)).astype(np.float64)
    assert (np.abs(y - tr)[~small] / ulp[~small]).max() <= 3.0
    # exact at powers of two
    p2 = np.float32(2.0) ** np.arange(-60, 60, dtype=np.float32)
    assert np.array_equal(g.eval32(c, p2), np.arange(-60, 60, dtype=np.float32))
