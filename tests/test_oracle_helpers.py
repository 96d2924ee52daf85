"""Pins of the oracle's smaller helpers against hand-worked values:
halfmax_width (the beam fit's start, reading of Sect. 3), component_terms'
box and clipping (reading 11), the xtol scales of the LM test (reading 9)
and the inclusive box overlap of the active set (reading 6)."""
import math

import numpy as np
import pytest

import oracle as O
import oracle.asp_oracle as OA


def _cone_psf(H, W, radii):
    """B with a linear profile 1 - r / R_d along each axis direction d
    (right, left, down, up), zero elsewhere: linear interpolation of the
    half-maximum crossing is exact there, at R_d / 2."""
    B = np.zeros((2 * H, 2 * W))
    B[H, W] = 1.0
    for (dy, dx), R in zip(((0, 1), (0, -1), (1, 0), (-1, 0)), radii):
        for s in range(1, min(H, W)):
            B[H + dy * s, W + dx * s] = max(0.0, 1.0 - s / R)
    return B


def test_halfmax_width_is_exact_on_linear_profiles():
    for radii in ((8.0, 8.0, 8.0, 8.0), (6.0, 9.0, 7.5, 10.0)):
        B = _cone_psf(20, 24, radii)
        want = (sum(R / 2.0 for R in radii) / 4.0) / math.sqrt(2.0 * math.log(2.0))
        assert OA.halfmax_width(B) == pytest.approx(want, rel=1e-14)


def test_halfmax_width_of_a_sampled_gaussian():
    # the crossing of a sampled Gaussian, interpolated linearly between
    # samples, lies within the chord error of sigma sqrt(2 ln 2)
    for sigma in (1.5, 2.7, 6.0):
        B = O.gauss_model(np.array([1.0, 30.0, 25.0, sigma]), *np.meshgrid(np.arange(60.0), np.arange(50.0)))
        w = OA.halfmax_width(B)
        assert abs(w - sigma) < 0.06 * sigma


def test_component_terms_box_extent_and_normalisation():
    H, W = 40, 50
    x, y, w = 20.4, 17.7, 1.3
    qx0, wx, qy0, wy, F = O.component_terms(3.0, x, y, w, False, H, W)
    h = math.ceil(5 * w) + 1                                   # 8
    assert qx0 == math.ceil(x - h) and len(wx) == math.floor(x + h) - math.ceil(x - h) + 1
    assert qy0 == math.ceil(y - h) and len(wy) == math.floor(y + h) - math.ceil(y - h) + 1
    assert wx.sum() == pytest.approx(1.0, rel=1e-15) and wy.sum() == pytest.approx(1.0, rel=1e-15)
    cols = np.arange(qx0, qx0 + len(wx))
    e = np.exp(-((cols - x) ** 2) / (2 * w * w))
    np.testing.assert_allclose(wx, e / e.sum(), rtol=1e-15)
    assert F == 3.0


def test_component_terms_clipped_at_the_edge_without_renormalisation():
    H, W = 30, 30
    full = O.component_terms(1.0, 15.0, 15.0, 2.0, False, 100, 100)     # far from every edge
    edge = O.component_terms(1.0, 1.2, 15.0, 2.0, False, H, W)
    qx0, wx, _, wy, _ = edge
    assert qx0 == 0
    # the kept columns carry the weights they have unclipped; the flux
    # that fell outside the image is lost, not spread over the rest
    cols = np.arange(math.ceil(1.2 - 11), math.floor(1.2 + 11) + 1)
    e = np.exp(-((cols - 1.2) ** 2) / (2 * 4.0))
    e /= e.sum()
    np.testing.assert_allclose(wx, e[cols >= 0], rtol=1e-14)
    assert wx.sum() < 1.0 - 1e-3 and wy.sum() == pytest.approx(1.0, rel=1e-15)
    assert full[1].sum() == pytest.approx(1.0, rel=1e-15)
    assert O.component_terms(1.0, -30.0, 15.0, 2.0, False, H, W) is None


def test_point_and_narrow_components_are_bilinear():
    for w, is_point in ((0.0, True), (0.49, False)):
        qx0, wx, qy0, wy, _ = O.component_terms(2.0, 5.75, 9.25, w, is_point, 20, 20)
        assert (qx0, qy0) == (5, 9)
        np.testing.assert_allclose(wx, [0.25, 0.75], rtol=1e-15)
        np.testing.assert_allclose(wy, [0.75, 0.25], rtol=1e-15)
    assert len(O.component_terms(2.0, 5.75, 9.25, 0.5, False, 20, 20)[1]) > 2   # 0.5 px is extended


def test_step_scales_of_the_xtol_test():
    theta = np.array([-0.3, 12.0, 7.0, 2.5, 0.0, 1.0, 2.0, 0.8])
    np.testing.assert_array_equal(OA._step_scale(theta), [0.3, 2.5, 2.5, 2.5, 1.0, 0.8, 0.8, 0.8])


def test_boxes_overlap_is_inclusive():
    a = (0, 10, 0, 10)
    assert O.boxes_overlap(a, (10, 20, 10, 20))            # sharing one corner pixel
    assert not O.boxes_overlap(a, (11, 20, 0, 10))
    assert not O.boxes_overlap(a, (0, 10, -20, -1))
    assert O.boxes_overlap(a, (3, 4, 3, 4)) and O.boxes_overlap((3, 4, 3, 4), a)


def test_round_half_up_on_halves():
    np.testing.assert_array_equal(O.round_half_up([-1.5, -0.5, 0.5, 1.5, 2.49999, -2.50001]), [-1, 0, 1, 2, 2, -3])


# ---------------------------------------------------------------- planted mistakes

def test_halfmax_without_interpolation_is_caught(monkeypatch):
    def bad(B):                                            # first sample below half, no interpolation
        B = np.asarray(B, dtype=np.float64)
        H, W = B.shape[0] // 2, B.shape[1] // 2
        half, radii = 0.5 * B[H, W], []
        for dy, dx in ((0, 1), (0, -1), (1, 0), (-1, 0)):
            s = 1
            while B[H + dy * s, W + dx * s] >= half:
                s += 1
            radii.append(float(s))
        return (sum(radii) / 4.0) / math.sqrt(2.0 * math.log(2.0))

    monkeypatch.setattr(OA, "halfmax_width", bad)
    with pytest.raises(AssertionError):
        test_halfmax_width_is_exact_on_linear_profiles()


def test_renormalised_clipping_is_caught(monkeypatch):
    orig = OA.component_terms

    def bad(F, x, y, w, is_point, H, W):
        t = orig(F, x, y, w, is_point, H, W)
        if t is None:
            return t
        qx0, wx, qy0, wy, s = t
        return qx0, wx / wx.sum(), qy0, wy / wy.sum(), s     # the lost flux spread over the kept pixels

    monkeypatch.setattr(OA, "component_terms", bad)
    monkeypatch.setattr(O, "component_terms", bad)
    with pytest.raises(AssertionError):
        test_component_terms_clipped_at_the_edge_without_renormalisation()
