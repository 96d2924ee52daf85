"""CPU checks of the test helpers that hold the GPU to the oracle: the
brute-force sampled subtraction and the FP32 step bound."""
import numpy as np

import oracle as O
import synth
from tests import fp32_bounds as FB
from tests import teacher


def test_sampled_subtraction_equals_oracle_subtraction():
    c = synth.small_case(40, 36, seed=2)
    terms = [O.component_terms(0.7, 12.3, 20.6, 2.5, False, 40, 36), O.component_terms(-0.4, 30.2, 5.9, 0.0, True, 40, 36)]
    ref = O.subtract_definition(np.zeros((40, 36)), c.psf, O.terms_to_image(terms, 40, 36))
    rng = np.random.default_rng(0)
    py, px = rng.integers(0, 40, 50), rng.integers(0, 36, 50)
    got = -teacher.subtraction_at(c.psf.astype(np.float64), terms, 40, 36, py, px)
    np.testing.assert_allclose(got, ref[py, px], rtol=1e-12, atol=1e-15)


def test_step_bound_covers_perturbed_solves():
    """Perturb A and g entrywise within the FP32 bounds (random signs,
    full size) and solve in FP64: every step stays within the first-order
    bound."""
    rng = np.random.default_rng(4)
    H = W = 40
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    xs, ys = xs.ravel(), ys.ravel()
    truth = np.array([0.8, 18.2, 21.1, 3.0, -0.3, 22.0, 19.4, 2.2, 0.2, 20.5, 20.1, 6.0])
    T = O.gauss_model(truth, xs, ys) + rng.normal(0, 1e-3, xs.size)
    theta = truth * np.array([1.05, 1, 1, 0.97] * 3) + np.array([0, 0.2, -0.1, 0] * 3)
    pb = FB.pass_bounds(T, xs, ys, theta)
    for lam in (1e-12, 1e-3, 10.0):
        d = FB.marquardt_diag(pb["A"])
        M = pb["A"] + lam * np.diag(d)
        delta = np.linalg.solve(M, pb["g"])
        bound, kappa = FB.step_bound(pb["A"], pb["g"], lam, pb["bA"], pb["bg"], delta)
        assert kappa < 0.5
        for _ in range(20):
            sA = rng.choice([-1.0, 1.0], size=pb["A"].shape)
            sA = np.triu(sA) + np.triu(sA, 1).T
            A2 = pb["A"] + sA * pb["bA"]
            g2 = pb["g"] + rng.choice([-1.0, 1.0], size=pb["g"].shape) * pb["bg"]
            d2 = FB.marquardt_diag(A2)
            delta2 = np.linalg.solve(A2 + lam * np.diag(d2), g2)
            assert np.all(np.abs(delta2 - delta) <= bound), np.max(np.abs(delta2 - delta) / bound)


def test_step_backward_accepts_perturbed_solutions_and_rejects_wrong_steps():
    rng = np.random.default_rng(5)
    ys, xs = np.mgrid[0:32, 0:32].astype(np.float64)
    xs, ys = xs.ravel(), ys.ravel()
    truth = np.array([0.8, 15.2, 16.1, 2.5, -0.3, 17.0, 14.4, 1.9])
    T = O.gauss_model(truth, xs, ys) + rng.normal(0, 1e-3, xs.size)
    theta = truth * np.array([1.05, 1, 1, 0.97] * 2)
    pb = FB.pass_bounds(T, xs, ys, theta)
    lam = 1e-3
    d = FB.marquardt_diag(pb["A"])
    A2 = pb["A"] + 0.5 * pb["bA"]
    g2 = pb["g"] - 0.5 * pb["bg"]
    delta2 = np.linalg.solve(A2 + lam * np.diag(FB.marquardt_diag(A2)), g2)
    resid, allowed = FB.step_backward(pb["A"], pb["g"], lam, pb["bA"], pb["bg"], delta2)
    assert np.all(resid <= allowed)
    wrong = delta2 * 1.01                                    # a 1 % wrong step is far outside
    resid, allowed = FB.step_backward(pb["A"], pb["g"], lam, pb["bA"], pb["bg"], wrong)
    assert np.any(resid > 2 * allowed)

