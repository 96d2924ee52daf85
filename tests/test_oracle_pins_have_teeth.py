"""Plant plausible mistakes in the oracle (on the CPU) and check that the
pins of test_oracle_closed_forms.py catch each one."""
import math

import numpy as np
import pytest

import oracle as O
import oracle.asp_oracle as OA
import tests.test_oracle_closed_forms as pins


def _patch(monkeypatch, name, fn):
    monkeypatch.setattr(OA, name, fn)
    monkeypatch.setattr(O, name, fn)


def test_flipped_jacobian_sign_is_caught(monkeypatch):
    orig = OA.model_and_jacobian

    def bad(theta, xs, ys):
        m, J = orig(theta, xs, ys)
        J = J.copy()
        J[:, 1::4] *= -1.0          # d/dx0 with the wrong sign
        return m, J

    _patch(monkeypatch, "model_and_jacobian", bad)
    with pytest.raises(AssertionError):
        pins.test_jacobian_against_central_differences()


def test_missing_factor_two_in_width_is_caught(monkeypatch):
    def bad(theta, xs, ys):
        theta = np.asarray(theta, float)
        out = np.zeros(np.broadcast(xs, ys).shape)
        for k in range(len(theta) // 4):
            a, x0, y0, w = theta[4 * k: 4 * k + 4]
            out += a * np.exp(-((xs - x0) ** 2 + (ys - y0) ** 2) / (w * w))
        return out

    _patch(monkeypatch, "gauss_model", bad)
    with pytest.raises(AssertionError):
        pins.test_model_against_python_loop()


def test_widths_added_instead_of_subtracted_is_caught(monkeypatch):
    def bad(a_ic, w_ic, alpha_b, omega_b):
        F = a_ic * w_ic * w_ic / (alpha_b * omega_b * omega_b)
        wi = math.sqrt(w_ic * w_ic + omega_b * omega_b)
        return F, F / (2 * math.pi * wi * wi), wi, False

    _patch(monkeypatch, "deconvolve", bad)
    with pytest.raises(AssertionError):
        pins.test_eq7_eq8_against_numerical_convolution(0.3, 2.0, 1.0, 1.5)


def test_transposed_psf_index_is_caught(monkeypatch):
    orig = OA.subtract_terms

    def bad(R, B, terms):
        return orig(R, np.asarray(B)[::-1, ::-1], terms)   # B(q - p) instead of B(p - q)

    _patch(monkeypatch, "subtract_terms", bad)
    with pytest.raises(AssertionError):
        pins.test_subtraction_separable_against_definition(9, 11)


def test_unit_sum_smoothing_kernel_is_caught(monkeypatch):
    def bad(s):
        m = int(math.ceil(4.0 * s))
        u = np.arange(-m, m + 1, dtype=np.float64)
        e = np.exp(-u * u / (2.0 * s * s))
        return e / e.sum()

    _patch(monkeypatch, "smoothing_kernel_1d", bad)
    with pytest.raises(AssertionError):
        pins.test_smoothing_init_recovers_gaussian_scale_and_amplitude()


def test_signed_argmax_is_caught(monkeypatch):
    def bad(R):
        flat = np.asarray(R).ravel()
        i = int(np.argmax(flat))
        return i, float(flat[i])

    _patch(monkeypatch, "peak_simple", bad)
    with pytest.raises(AssertionError):
        pins.test_argmax_against_python_scan_with_ties()


def test_gain_on_wrong_side_is_caught(monkeypatch):
    orig = OA.MinorCycle._component_from_fit

    def bad(self, a, x, y, w, gain=1.0):
        return orig(self, a, x, y, w, gain=1.0 / gain if gain != 1.0 else 1.0)

    monkeypatch.setattr(OA.MinorCycle, "_component_from_fit", bad)
    with pytest.raises(AssertionError):
        pins.test_first_iteration_on_point_source_gaussian_psf()


def test_mad_without_normal_factor_is_caught(monkeypatch):
    def bad(img):
        v = np.asarray(img, dtype=np.float64).ravel()
        return float(np.median(np.abs(v - np.median(v))))

    _patch(monkeypatch, "mad_sigma", bad)
    with pytest.raises(AssertionError):
        pins.test_mad_sigma_hand_computed_and_normal_consistency()


def test_mad_as_mean_deviation_is_caught(monkeypatch):
    def bad(img):
        v = np.asarray(img, dtype=np.float64).ravel()
        return 1.4826 * float(np.mean(np.abs(v - np.median(v))))

    _patch(monkeypatch, "mad_sigma", bad)
    with pytest.raises(AssertionError):
        pins.test_mad_sigma_hand_computed_and_normal_consistency()


def test_switch_on_widths_instead_of_areas_is_caught(monkeypatch):
    def bad(self):
        if self.t > 0 and self.last_wi < self.p.area_frac * self.last_w0:
            return O.MODE_SIMPLE
        return O.MODE_SMOOTH

    monkeypatch.setattr(OA.MinorCycle, "choose_mode", bad)
    with pytest.raises(AssertionError):
        pins.test_choose_mode_five_percent_area_rule()


def test_switch_with_non_strict_threshold_is_caught(monkeypatch):
    def bad(self):
        if self.t > 0 and self.last_wi ** 2 <= self.p.area_frac * self.last_w0 ** 2:
            return O.MODE_SIMPLE
        return O.MODE_SMOOTH

    monkeypatch.setattr(OA.MinorCycle, "choose_mode", bad)
    with pytest.raises(AssertionError):
        pins.test_choose_mode_five_percent_area_rule()


def test_member_box_with_half_even_rounding_is_caught(monkeypatch):
    def bad(x, y, w):
        h = max(5, int(math.ceil(4.0 * w)))
        rx, ry = int(round(x)), int(round(y))       # Python rounds halves to even
        return (rx - h, rx + h, ry - h, ry + h)

    _patch(monkeypatch, "member_box", bad)
    with pytest.raises(AssertionError):
        pins.test_member_box_half_width_and_rounding()


def test_window_without_clipping_is_caught(monkeypatch):
    orig = OA.MinorCycle.select

    def bad(self, init):
        chosen, _ = orig(self, init)
        boxes = [OA.member_box(init["x0"], init["y0"], init["w0"])] + [OA.member_box(*self.G(k)[1:4]) for k in chosen]
        return chosen, (min(b[0] for b in boxes), max(b[1] for b in boxes), min(b[2] for b in boxes),
                        max(b[3] for b in boxes))

    monkeypatch.setattr(OA.MinorCycle, "select", bad)
    with pytest.raises(AssertionError):
        pins.test_window_is_clipped_bounding_box_of_member_boxes()


def test_beam_image_with_widths_added_linearly_is_caught(monkeypatch):
    def bad(x, y, w, alpha_b, omega_b, H, W):
        w_ic = w + omega_b
        a_ic = alpha_b * omega_b * omega_b / (w_ic * w_ic)
        h = math.ceil(5.0 * w_ic) + 1
        x0, x1 = max(math.ceil(x - h), 0), min(math.floor(x + h), W - 1)
        y0, y1 = max(math.ceil(y - h), 0), min(math.floor(y + h), H - 1)
        ys, xs = np.mgrid[y0: y1 + 1, x0: x1 + 1].astype(np.float64)
        return x0, y0, a_ic * np.exp(-((xs - x) ** 2 + (ys - y) ** 2) / (2.0 * w_ic * w_ic))

    _patch(monkeypatch, "beam_image_box", bad)
    with pytest.raises(AssertionError):
        pins.test_beam_image_is_full_psf_subtraction_through_a_gaussian_psf(1.3, 20.4, 18.7, 2.5)


def test_2004_jacobian_without_the_psf_is_caught(monkeypatch):
    def bad(B, theta, H, W):
        ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
        m, J = OA.model_and_jacobian(theta, xs.ravel(), ys.ravel())
        return OA.psf_convolve(B, m.reshape(H, W)).ravel(), J      # columns not convolved

    _patch(monkeypatch, "model_jac_2004", bad)
    with pytest.raises(AssertionError):
        pins.test_2004_jacobian_against_central_differences()


def test_psf_convolve_with_flipped_psf_is_caught(monkeypatch):
    orig = OA.psf_convolve

    def bad(B, img):
        return orig(np.asarray(B)[::-1, ::-1], img)

    _patch(monkeypatch, "psf_convolve", bad)
    with pytest.raises(AssertionError):
        pins.test_psf_convolve_is_the_direct_convolution(9, 11)
