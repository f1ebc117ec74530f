"""Pins of the learned tagger's oracle (oracle/cnn.py) against things other
than itself: exact bfloat16 encodings, brute-force loops, a library
correlation, finite differences of the loss, Adam's first step in closed
form, and the input scaling on linear data."""
import numpy as np
import pytest

from oracle import cnn


def test_bf16_rounding_exact_values():
    one = 1.0
    assert cnn.bf16([one])[0] == 1.0
    assert cnn.bf16([1 + 2.0 ** -8])[0] == 1.0                 # tie -> even (1.0)
    assert cnn.bf16([1 + 3 * 2.0 ** -8])[0] == 1 + 2.0 ** -6    # tie -> even (mantissa ...10)
    assert cnn.bf16([1 + 2.0 ** -8 + 2.0 ** -20])[0] == 1 + 2.0 ** -7  # above the tie
    assert cnn.bf16([np.pi])[0] == 3.140625
    assert cnn.bf16([-np.pi])[0] == -3.140625
    r = np.random.default_rng(0).normal(size=1000) * 10.0 ** np.random.default_rng(1).integers(-20, 20, 1000)
    b = cnn.bf16(r)
    assert np.all((b.astype(np.float32).view(np.uint32) & 0xFFFF) == 0)
    assert np.all(np.abs(b - r) <= np.abs(r) * 2.0 ** -8 * (1 + 1e-12))


def test_conv_matches_brute_force_and_library():
    scipy_signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(3)
    A = rng.normal(size=(2, 3, 6, 7))
    W = rng.normal(size=(4, 3, 3, 3))
    got = cnn.conv3x3_valid(A, W)
    ref = np.zeros_like(got)
    for p in range(2):
        for g in range(4):
            for y in range(4):
                for x in range(5):
                    ref[p, g, y, x] = sum(W[g, f, ky, kx] * A[p, f, y + ky, x + kx]
                                          for f in range(3) for ky in range(3) for kx in range(3))
            lib = sum(scipy_signal.correlate2d(A[p, f], W[g, f], mode="valid") for f in range(3))
            assert np.allclose(lib, ref[p, g], rtol=0, atol=1e-12)
    assert np.allclose(got, ref, rtol=0, atol=1e-12)


def _problem(seed, P=3, C=2, S=8):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(P, C, S, S))
    level = rng.integers(0, 4, size=P)
    params = rng.normal(size=cnn.param_count(C)) * 0.3
    label = rng.integers(0, 2, size=P).astype(float)
    omega = rng.uniform(0.5, 2.0, size=P)
    return X, level, params, label, omega


def test_forward_max_pool_and_head_brute_force():
    X, level, params, label, omega = _problem(5)
    logit, M, arg, mid = cnn.forward(X, level, params, 2)
    w = cnn.unpack(params, 2)
    Z2 = mid["Z2"]
    for p in range(X.shape[0]):
        for g in range(cnn.F):
            best, bi = -np.inf, -1
            for y in range(Z2.shape[2]):
                for x in range(Z2.shape[3]):
                    if Z2[p, g, y, x] > best:
                        best, bi = Z2[p, g, y, x], y * Z2.shape[3] + x
            assert M[p, g] == max(best, 0.0)
            assert arg[p, g] == (bi if best > 0 else -1)
        assert np.isclose(logit[p], sum(w["w3"][g] * M[p, g] for g in range(cnn.F)) + w["b3"][0], rtol=1e-13)
    # layer-1 activations are BF16 values
    assert np.array_equal(mid["A1"], cnn.bf16(mid["A1"]))


def test_backward_matches_finite_differences():
    X, level, params, label, omega = _problem(7)
    g = cnn.backward(X, level, params, 2, label, omega, exact=True)
    rng = np.random.default_rng(11)
    n = len(params)
    idx = np.unique(np.concatenate([rng.choice(n, 150, replace=False), np.arange(n - 2 * cnn.F - 1, n)]))
    eps = 1e-6
    for i in idx:
        pp, pm = params.copy(), params.copy()
        pp[i] += eps
        pm[i] -= eps
        lp = cnn.loss(cnn.forward(X, level, pp, 2, exact=True)[0], label, omega)
        lm = cnn.loss(cnn.forward(X, level, pm, 2, exact=True)[0], label, omega)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
    # every parameter block receives some gradient
    sizes = [cnn.F * 2 * 9, cnn.NLEVEL * cnn.F, cnn.F * cnn.F * 9, cnn.F, cnn.F, 1]
    o = 0
    for s in sizes:
        assert np.abs(g[o:o + s]).max() > 0
        o += s


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(2)
    p0, g = rng.normal(size=50), rng.normal(size=50)
    p1, m, v = cnn.adam(p0, np.zeros(50), np.zeros(50), g, 1, 0.01)
    # bias-corrected moments are g and g^2 at step 1: the step is lr * g / (|g| + eps)
    assert np.allclose(p1, p0 - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_inputs_scale_makes_the_threshold_a_unit_difference():
    n, thr, dx0, lev = 8, 3.0, 0.1, 2
    h = dx0 / 4
    W = n + 5
    idx = np.arange(W) - 2
    slope = 2.5                      # Q = slope * x: indicator |dQ| / (2h) = slope
    Q = slope * (idx[None, :] + 0.5) * h * np.ones((W, 1))
    X = cnn.inputs(Q[None, None], n, np.array([lev]), dx0, thr)
    assert X.shape == (1, 1, n + 4, n + 4)
    cd = X[0, 0, 2:-2, 3:-1] - X[0, 0, 2:-2, 1:-3]
    assert np.allclose(cd, slope / thr, rtol=2 ** -7)
    assert abs(X[0, 0, 2:n + 2, 2:n + 2].mean()) < 1e-2


def test_combine_tags_fallback_rules():
    logit = np.array([5.0, -5.0, 0.1, -0.1, 5.0, -5.0])
    plain = np.array([0, 1, 1, -1, -1, -1], np.int8)
    tags, nfall = cnn.combine_tags(logit, plain, 0.5)
    assert tags.tolist() == [1, 0, 1, -1, 1, -1]
    assert nfall == 2
