"""The kernels evaluate sin(pi x) and cos(pi x) on |x| <= 1/2 (fractional delays delta and
delta/K) with Taylor series truncated after x^13 and x^14.  This checks, independently of the
CUDA code, that those truncations stay far below the RIR tolerance (1e-5 of the peak): the
series coefficients are rebuilt from factorials here and compared with numpy's sin/cos in FP64.
"""
import math

import numpy as np


def test_taylor_truncation_bounds():
    x = np.linspace(-0.5 - 1e-6, 0.5 + 1e-6, 200001)
    s = sum(((-1) ** k) * math.pi ** (2 * k + 1) / math.factorial(2 * k + 1) * x ** (2 * k + 1) for k in range(7))
    c = sum(((-1) ** k) * math.pi ** (2 * k) / math.factorial(2 * k) * x ** (2 * k) for k in range(8))
    assert np.max(np.abs(s - np.sin(np.pi * x))) < 7e-10
    assert np.max(np.abs(c - np.cos(np.pi * x))) < 7e-11


def test_float32_horner_error():
    # Horner evaluation in float32 (as on the GPU, with separate rounding per step) stays
    # within a few float32 ulps of the true values.
    x = np.linspace(-0.5, 0.5, 100001).astype(np.float32)
    x2 = x * x
    cs = [((-1) ** k) * math.pi ** (2 * k + 1) / math.factorial(2 * k + 1) for k in range(7)][::-1]
    p = np.float32(cs[0])
    for ck in cs[1:]:
        p = (p * x2 + np.float32(ck)).astype(np.float32)
    s = (p * x).astype(np.float32)
    assert np.max(np.abs(s.astype(np.float64) - np.sin(np.pi * x.astype(np.float64)))) < 5e-7
