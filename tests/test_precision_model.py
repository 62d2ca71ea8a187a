"""The tensor-core gradient tolerances cover the error the FP16 / BF16 rounding
points themselves produce (emulated in FP64) on the cases the GPU tests use."""
import numpy as np
import pytest

import oracle as O
from paper_2207_11620_gb300 import configs as CF
from paper_2207_11620_gb300 import inputs as I
from tests.precision_model import (backward_model, coord_grad_from_df, expected_errors, normwise, round_bf16,
                                   round_fp16)
from tests.test_gpu_coord_grad import NORM_TOL as COORD_TOL
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


def test_coord_grad_model_matches_the_oracle_without_rounding():
    """The model's Jacobian applied to the exact dF is the oracle's dL/dx."""
    c = CF.CFG1_NET
    net = O.Net(L=c.L, F=c.F, log2T=c.log2T, Nmin=c.Nmin, b=c.b, dims=c.dims)
    params = I.uniform_params(net.n_params, seed=54, scale=0.5)
    x = I.uniform_points(300, seed=55)
    dy = np.random.default_rng(56).uniform(0.5, 1.5, size=300)
    dF = backward_model(net, params, x, dy, "exact")[0]
    want = O.backward_x(net, params, x, dy)
    np.testing.assert_allclose(coord_grad_from_df(net, params, x, dF), want, rtol=1e-9,
                               atol=1e-12 * np.abs(want).max())


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("shape", ["cfg1", "cfg2"])
def test_coord_grad_tolerance_covers_rounding_model(prec, shape):
    c = CF.CFG1_NET if shape == "cfg1" else CF.CFG2_NET
    net = O.Net(L=c.L, F=c.F, log2T=c.log2T, Nmin=c.Nmin, b=c.b, dims=c.dims)
    params = I.uniform_params(net.n_params, seed=54, scale=0.5)
    n = 2000
    x = I.uniform_points(n, seed=55)
    dy = np.random.default_rng(56).uniform(0.5, 1.5, size=n)
    exact = coord_grad_from_df(net, params, x, backward_model(net, params, x, dy, "exact")[0])
    got = coord_grad_from_df(net, params, x, backward_model(net, params, x, dy, prec)[0])
    assert normwise(got, exact) * 1.25 <= COORD_TOL[prec], normwise(got, exact)
