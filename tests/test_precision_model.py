"""The tensor-core gradient tolerances cover the error the FP16 / BF16 rounding
points themselves produce (emulated in FP64) on the cases the GPU tests use."""
import numpy as np
import pytest

import oracle as O
from paper_2207_11620_gb300 import configs as CF
from paper_2207_11620_gb300 import inputs as I
from tests.precision_model import expected_errors, round_bf16, round_fp16
from tests.test_gpu_tc import GRAD_TOL, TABLE_TOL


def test_rounding_helpers():
    assert round_fp16(1.0 + 2 ** -12) == 1.0 and round_fp16(1.0 + 2 ** -10) == 1.0 + 2 ** -10
    assert round_bf16(1.0 + 2 ** -9) == 1.0 and round_bf16(1.0 + 2 ** -7) == 1.0 + 2 ** -7
    assert round_bf16(3.0) == 3.0 and round_fp16(-0.5) == -0.5


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_tolerances_cover_rounding_model(prec):
    c = CF.CFG2_NET
    net = O.Net(L=c.L, F=c.F, log2T=c.log2T, Nmin=c.Nmin, b=c.b, dims=c.dims)
    params = I.uniform_params(net.n_params, seed=43, scale=0.5)
    n = 2000
    x = I.uniform_points(n, seed=44)
    dy = np.random.default_rng(45).uniform(0.5, 1.5, size=n) / n
    err = expected_errors(net, params, x, dy, prec)
    # the per-point dF (the table gradient before the scatter) carries the
    # ReLU decisions the rounded forward flips; the weight gradients average them
    assert err["dF"] * 1.25 <= TABLE_TOL[prec], err
    for k in ("dW0", "dW1", "dW2"):
        assert err[k] * 1.25 <= GRAD_TOL[prec], err
    assert err["dF"] > 3 * err["dW1"]
