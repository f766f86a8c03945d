"""Pins of the ASPC predictor weights (density extrapolation for MD, Sec. "Common Setup")."""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("K", range(0, 7))
def test_weights_reproduce_constant_and_linear_histories(K):
    B = oracle.aspc_coefficients(K)
    j = np.arange(1, K + 2)
    assert abs(B.sum() - 1.0) < 1e-14                 # a constant density is predicted exactly
    if K >= 1:
        assert abs(np.sum(B * (-j))) < 1e-13          # so is a linear drift (t - j -> t = 0)


def test_low_orders_are_the_textbook_extrapolations():
    assert np.allclose(oracle.aspc_coefficients(0), [1.0])            # previous step
    assert np.allclose(oracle.aspc_coefficients(1), [2.0, -1.0])      # linear extrapolation


def test_predict_on_matrices():
    rng = np.random.default_rng(5)
    A, Bm = rng.normal(size=(4, 4)), rng.normal(size=(4, 4))
    hist = [A + Bm * (-j) for j in range(1, 5)]  # linear in time, t = 0 is the prediction
    assert np.max(np.abs(oracle.aspc_predict(hist) - A)) < 1e-12
