"""Pins of the oracle's error magnitudes (the per-element M(q) >= |q| that the
FP32 parity bound |g - o| <= 1e-5 M scales with).

M(q) bounds the first-order sensitivity of q to relative perturbations of
every input that carries a rounding error: changing each table entry, weight,
voxel or upstream gradient by at most delta times its own size moves q by at
most k delta M(q), k the number of perturbed factors a term of q carries (k =
1 for the features, which are linear in the tables: there the sign-aligned
perturbation reaches the bound exactly; 4 for a network output, whose terms
carry a table entry and three weights; 8 for a gradient entry; 3 for a
composited pixel, whose terms carry a transmittance, an opacity and a colour).
Where nothing cancels M is the value itself.  The tests below check these
properties, with the oracle's own FP64 evaluation as the function perturbed.
"""
import numpy as np
import pytest

import oracle as O
from paper_2207_11620_gb300 import inputs as I

NET = O.Net(L=4, F=2, log2T=10, Nmin=4, b=1.6, dims=(8, 16, 16, 1))
DELTA = 1e-7


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _relative_perturbation(p, seed, delta=DELTA, sign=None):
    s = _rng(seed).choice([-1.0, 1.0], size=p.shape) if sign is None else sign
    return p + delta * s * np.abs(p)


def _params(seed, scale=0.5, nonneg=False):
    p = _rng(seed).uniform(0.0 if nonneg else -scale, scale, size=NET.n_params)
    return p.astype(np.float64)


def test_encode_mag_is_the_value_for_nonnegative_tables():
    p = _params(1, nonneg=True)
    x = I.uniform_points(300, seed=2)
    np.testing.assert_allclose(O.encode_mag(NET, p, x), O.encode(NET, p, x), rtol=1e-14)


def test_encode_mag_is_the_reachable_sensitivity():
    # features are linear in the tables: the sign-aligned relative perturbation
    # of the tables moves each feature by exactly delta M, a random one by less
    p = _params(3)
    x = I.uniform_points(200, seed=4)
    f, fm = O.encode(NET, p, x), O.encode_mag(NET, p, x)
    assert np.all(fm >= np.abs(f))
    df = O.encode(NET, _relative_perturbation(p, 5), x) - f
    assert np.all(np.abs(df) <= DELTA * fm * (1 + 1e-6) + 1e-300)
    # raising every entry by delta |theta| raises every term w |theta|: the gain is delta M
    gain = O.encode(NET, p + DELTA * np.abs(p), x) - f
    np.testing.assert_allclose(gain, DELTA * fm, rtol=1e-6, atol=1e-300)
    # with constant-magnitude entries of random sign the magnitude is that
    # magnitude times the partition of unity, whatever the signs
    a = 0.37
    q = a * _rng(6).choice([-1.0, 1.0], size=NET.n_params)
    np.testing.assert_allclose(O.encode_mag(NET, q, x), a, rtol=1e-13)


def test_forward_mag_closed_form_for_nonnegative_parameters():
    # nothing cancels: every hidden magnitude is the hidden value, so M(y) = y +
    # sigma'(z) z with z = logit(y), and every pre-activation is its own magnitude
    p = _params(7, scale=0.3, nonneg=True)
    x = I.uniform_points(300, seed=8)
    y, ym, kink = O.forward_mag(NET, p, x)
    np.testing.assert_array_equal(y, O.forward(NET, p, x))
    z = np.log(y / (1 - y))
    np.testing.assert_allclose(ym, y + y * (1 - y) * z, rtol=1e-12)
    np.testing.assert_allclose(kink, 1.0, rtol=1e-12)


def test_forward_mag_bounds_relative_perturbations():
    p = _params(9)
    x = I.uniform_points(400, seed=10)
    y, ym, kink = O.forward_mag(NET, p, x)
    assert np.all(ym >= np.abs(y))
    for seed in range(3):
        dy = O.forward(NET, _relative_perturbation(p, 11 + seed), x) - y
        ok = kink > 1e-4  # a unit this close to its kink may switch under the perturbation
        assert ok.mean() > 0.9
        assert np.all(np.abs(dy[ok]) <= 4 * DELTA * ym[ok])


def test_forward_mag_bounds_an_fp32_evaluation():
    # what the bound is for: the same network evaluated in FP32 (features rounded,
    # float32 products in numpy's order) stays within 1e-5 M of the FP64 value
    p = _params(12)
    x = I.uniform_points(2000, seed=13)
    y, ym, _ = O.forward_mag(NET, p, x)
    d = NET.dims
    W = p[NET.n_table:].astype(np.float32)
    W0 = W[: d[1] * d[0]].reshape(d[1], d[0])
    W1 = W[d[1] * d[0]: d[1] * d[0] + d[2] * d[1]].reshape(d[2], d[1])
    W2 = W[-d[2]:]
    f = O.encode(NET, p.astype(np.float32).astype(np.float64), x).astype(np.float32)
    h = np.maximum(f @ W0.T, np.float32(0))
    h = np.maximum(h @ W1.T, np.float32(0))
    y32 = (np.float32(1) / (np.float32(1) + np.exp(-(h @ W2)))).astype(np.float64)
    y64 = O.forward(NET, p.astype(np.float32).astype(np.float64), x)
    assert np.max(np.abs(y32 - y64) / ym) <= 1e-5


def test_backward_mag_equals_backward_when_nothing_cancels():
    # nonnegative parameters and upstream gradients: the magnitude recursion is
    # the backward recursion itself, with the output derivative sigma' replaced
    # by its magnitude sigma' + |1 - 2y| M(y)
    p = _params(14, scale=0.3, nonneg=True)
    x = I.uniform_points(300, seed=15)
    dym = _rng(16).uniform(0.1, 1.0, size=300)
    y, ym, _ = O.forward_mag(NET, p, x)
    s = y * (1 - y)
    want = O.backward(NET, p, x, dym * (s + np.abs(1 - 2 * y) * ym) / s)
    np.testing.assert_allclose(O.backward_mag(NET, p, x, dym), want, rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("masked", [True, False])
def test_backward_mag_bounds_relative_perturbations(masked):
    p = _params(17)
    x = I.uniform_points(500, seed=18)
    _, _, kink = O.forward_mag(NET, p, x)
    x = x[kink > 1e-3]  # the masks cannot switch under a 1e-7 perturbation
    dy = _rng(19).normal(size=x.shape[0])
    g = O.backward(NET, p, x, dy)
    gm = O.backward_mag(NET, p, x, np.abs(dy), masked=masked)
    assert np.all(gm >= np.abs(g) * (1 - 1e-12))
    assert np.array_equal(gm == 0, g == 0) if masked else np.all(gm[g != 0] > 0)
    for seed in range(2):
        q = _relative_perturbation(p, 20 + seed)
        dq = _relative_perturbation(dy, 30 + seed)
        dg = O.backward(NET, q, x, dq) - g
        assert np.all(np.abs(dg) <= 8 * DELTA * gm + 1e-300)


def _render(vol, lut, opts, cam, with_mag=True, **kw):
    pix = np.arange(cam["width"] * cam["height"])
    return O.render_pixels(cam, lut, opts, pix, vol=vol, with_mag=with_mag, **kw)


@pytest.mark.parametrize("lut_kind", ["ramp_floor", "soft"])
@pytest.mark.parametrize("alpha_exp", [1.0, 0.5])
def test_render_mag_bounds_relative_perturbations(lut_kind, alpha_exp):
    # no early termination (et > 1), so every pixel is a smooth function of the voxels
    vol = I.blob_volume(24, seed=21)
    lut = I.ramp_lut(alpha_floor=0.1) if lut_kind == "ramp_floor" else I.ramp_lut_soft(0.1)
    cam = I.perspective_camera(24, 16)
    opts = dict(step=0.5 / 24, alpha_exp=alpha_exp, et=2.0)
    rgba, mag = _render(vol, lut, opts, cam)
    assert np.all(mag >= np.abs(rgba) * (1 - 1e-12))
    assert rgba[:, 3].max() > 0.3
    delta = 1e-6
    for seed in range(2):
        s = _rng(40 + seed).choice([-1.0, 1.0], size=vol.shape)
        v2 = (vol.astype(np.float64) * (1 + delta * s)).astype(np.float32)
        # the FP32 store of the perturbed volume rounds: use the realised perturbation
        real = np.abs(v2.astype(np.float64) - vol) / np.maximum(np.abs(vol), 1e-30)
        assert real.max() <= delta + 2.0 ** -24
        d = O.render_pixels(cam, lut, opts, np.arange(24 * 16), vol=v2) - rgba
        assert np.all(np.abs(d) <= 3 * real.max() * mag + 1e-15)


def test_render_mag_of_a_network_bounds_relative_perturbations():
    p = _params(50)
    cam = I.ortho_camera_z(12, 10)
    lut = I.ramp_lut()
    opts = dict(step=1 / 64, alpha_exp=1.0, et=2.0)
    pix = np.arange(120)
    rgba, mag = O.render_pixels(cam, lut, opts, pix, net=NET, params=p, with_mag=True)
    assert np.all(mag >= np.abs(rgba) * (1 - 1e-12))
    d = O.render_pixels(cam, lut, opts, pix, net=NET, params=_relative_perturbation(p, 51)) - rgba
    assert np.all(np.abs(d) <= 3 * 4 * DELTA * mag + 1e-15)


def test_render_mag_with_shadows_bounds_value():
    vol = I.blob_volume(20, seed=52)
    lut = I.ramp_lut_soft(0.1)
    cam = I.perspective_camera(16, 12)
    opts = dict(step=0.5 / 20, alpha_exp=0.5, et=0.99, shade=1, light=(0.0, 0.8, -0.6), ambient=0.25)
    rgba, mag = _render(vol, lut, opts, cam)
    assert np.all(mag >= np.abs(rgba) * (1 - 1e-12))
    plain = _render(vol, lut, dict(opts, shade=0), cam, with_mag=False)
    assert np.all(rgba[:, :3] <= plain[:, :3] + 1e-15)


def test_coordinate_gradient_mag_bounds_relative_perturbations():
    p = _params(60)
    x = I.uniform_points(400, seed=61)
    _, _, kink = O.forward_mag(NET, p, x)
    x = x[kink > 1e-3]
    dy = _rng(62).normal(size=x.shape[0])
    g = O.backward_x(NET, p, x, dy)
    gm = O.backward_x_mag(NET, p, x, np.abs(dy))
    assert np.all(gm >= np.abs(g) * (1 - 1e-12))
    assert np.all(O.backward_x_mag(NET, p, x, np.abs(dy), masked=False) >= gm)
    for seed in range(2):
        dg = O.backward_x(NET, _relative_perturbation(p, 63 + seed), x, _relative_perturbation(dy, 70 + seed)) - g
        assert np.all(np.abs(dg) <= 8 * DELTA * gm + 1e-300)
