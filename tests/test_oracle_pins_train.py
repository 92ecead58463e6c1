"""Pins of the oracle's training-loop pieces (parameter activations, Adam)
against closed forms of Adam (Kingma and Ba) and central differences."""
import numpy as np
import pytest

import oracle


def _raw(rng, M=5):
    raw = np.zeros((M, 11))
    raw[:, 0:3] = rng.normal(size=(M, 3))
    raw[:, 3:6] = np.log(rng.uniform(1.0, 3.0, size=(M, 3)))
    raw[:, 6:10] = rng.normal(size=(M, 4))
    raw[:, 10] = np.log(rng.uniform(0.5, 1.5, size=M))
    return raw


def test_activation_closed_form():
    raw = _raw(np.random.default_rng(90))
    p = oracle.activate(raw)
    np.testing.assert_array_equal(p[:, 0:3], raw[:, 0:3])
    np.testing.assert_array_equal(p[:, 6:10], raw[:, 6:10])
    np.testing.assert_allclose(np.log(p[:, 3:6]), raw[:, 3:6], rtol=1e-15)
    np.testing.assert_allclose(np.log(p[:, 10]), raw[:, 10], rtol=1e-15)


def test_first_step_moves_by_the_learning_rate():
    """After one step m^ = g and v^ = g^2, so each raw entry moves by
    -lr g / (|g| + eps): lr times the sign of the raw gradient."""
    rng = np.random.default_rng(91)
    raw = _raw(rng)
    g = rng.normal(size=raw.shape)
    lr = [0.1, 0.01, 0.001, 0.05]
    z = np.zeros_like(raw)
    new, m, v, params = oracle.adam_step(raw, z, z, g, lr, 1, eps=1e-12)
    p = oracle.activate(raw)
    graw = g.copy()
    graw[:, [3, 4, 5, 10]] *= p[:, [3, 4, 5, 10]]
    lrs = np.array(lr)[[0, 0, 0, 1, 1, 1, 2, 2, 2, 2, 3]]
    np.testing.assert_allclose(new - raw, -lrs * np.sign(graw), rtol=1e-9)
    np.testing.assert_allclose(params, oracle.activate(new), rtol=1e-15)


def test_constant_gradient_steps_are_constant():
    """With a constant raw gradient the bias-corrected moments are exactly g
    and g^2 at every step: t steps move centre and quaternion entries by
    -t lr g / (|g| + eps)."""
    rng = np.random.default_rng(92)
    raw = _raw(rng)
    g = rng.normal(size=raw.shape)
    g[:, [3, 4, 5, 10]] = 0.0  # the log entries' raw gradient would change with the scale
    lr = [0.2, 0.0, 0.03, 0.0]
    m = np.zeros_like(raw)
    v = np.zeros_like(raw)
    r = raw
    for t in range(1, 8):
        r, m, v, _ = oracle.adam_step(r, m, v, g, lr, t, eps=1e-8)
    lrs = np.array(lr)[[0, 0, 0, 1, 1, 1, 2, 2, 2, 2, 3]]
    np.testing.assert_allclose(r - raw, -7 * lrs * g / (np.abs(g) + 1e-8), rtol=1e-9, atol=1e-15)


def test_chain_rule_through_the_activations():
    """The raw gradient the step uses is d f(activate(raw)) / d raw, checked by
    central differences on f(params) = sum c * params."""
    rng = np.random.default_rng(93)
    raw = _raw(rng, M=3)
    c = rng.normal(size=raw.shape)
    f = lambda r: float(np.sum(c * oracle.activate(r)))
    # one Adam step with beta1 = beta2 = 0 and eps tiny: new - raw = -lr g_raw / |g_raw|;
    # recover g_raw's sign and compare with the differences
    z = np.zeros_like(raw)
    new, _, _, _ = oracle.adam_step(raw, z, z, c, [1, 1, 1, 1], 1, beta1=0.0, beta2=0.0, eps=1e-300)
    for j in range(3):
        for k in range(11):
            h = 1e-6
            rp, rm = raw.copy(), raw.copy()
            rp[j, k] += h
            rm[j, k] -= h
            fd = (f(rp) - f(rm)) / (2 * h)
            assert np.sign(fd) == -np.sign(new[j, k] - raw[j, k])


def test_iso_scale_is_imposed_and_moments_kept():
    rng = np.random.default_rng(94)
    raw = _raw(rng)
    g = rng.normal(size=raw.shape)
    m = rng.normal(size=raw.shape) * 0.1
    v = np.abs(rng.normal(size=raw.shape)) * 0.1
    iso = rng.uniform(0.5, 2.0, size=raw.shape[0])
    new, m2, v2, params = oracle.adam_step(raw, m, v, g, [0.1] * 4, 3, iso_scale=iso)
    np.testing.assert_array_equal(params[:, 3:6], np.repeat(iso[:, None], 3, 1))
    np.testing.assert_allclose(new[:, 3:6], np.log(iso)[:, None].repeat(3, 1))
    np.testing.assert_array_equal(m2[:, 3:6], m[:, 3:6])
    np.testing.assert_array_equal(v2[:, 3:6], v[:, 3:6])
