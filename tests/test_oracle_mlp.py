"""Pins for the predictor's CPU oracle: its backpropagated gradient against
central finite differences of its loss (a check independent of the chain-rule
formulas), the loss at a hand-computable point, and one Adam step against the
closed form of the first step."""
import numpy as np
import pytest

from oracle import mlp


def random_params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    p = np.zeros(mlp.TOTAL)
    p[:mlp.TRAINABLE] = scale * rng.standard_normal(mlp.TRAINABLE)
    p[mlp.TRAINABLE:mlp.TRAINABLE + 35] = rng.standard_normal(35)          # mu
    p[mlp.TRAINABLE + 35:mlp.TRAINABLE + 70] = 0.5 + rng.random(35)        # sigma
    p[-2], p[-1] = 7.0, 2.0                                                 # y_mu, y_sigma
    return p


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    p = random_params(2)
    x = rng.standard_normal((9, 35))
    t = 7.0 + 2.0 * rng.standard_normal(9)
    L, g = mlp.loss_grad(p, x, t)
    assert L == mlp.loss(p, x, t)
    idx = np.concatenate([rng.choice(mlp.TRAINABLE, 60, replace=False),
                          [0, 35 * 128 - 1, mlp.TRAINABLE - 1, mlp.TRAINABLE - 2]])
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.loss(pp, x, t) - mlp.loss(pm, x, t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_loss_closed_form_at_zero_weights():
    """With all weights zero the output is b3 everywhere: L = mean((b3 - t_std)^2)."""
    p = random_params(3)
    p[:mlp.TRAINABLE] = 0.0
    p[mlp.TRAINABLE - 1] = 0.25  # b3
    t = np.array([7.0, 9.0, 5.0])
    t_std = (t - 7.0) / 2.0
    assert abs(mlp.loss(p, np.zeros((3, 35)), t) - np.mean((0.25 - t_std) ** 2)) < 1e-15
    assert np.allclose(mlp.forward(p, np.zeros((3, 35))), 0.25 * 2.0 + 7.0)


def test_first_adam_step_closed_form():
    """At step 1 the bias-corrected moments are g and g^2, so the update is
    -lr * g / (|g| + eps)."""
    rng = np.random.default_rng(4)
    p = random_params(5)
    g = rng.standard_normal(mlp.TRAINABLE)
    p1, m1, m2 = mlp.adam(p, g, np.zeros_like(g), np.zeros_like(g), 1, 1e-3)
    np.testing.assert_allclose(p1[:mlp.TRAINABLE] - p[:mlp.TRAINABLE], -1e-3 * g / (np.abs(g) + 1e-8),
                               rtol=1e-9)
    np.testing.assert_array_equal(p1[mlp.TRAINABLE:], p[mlp.TRAINABLE:])


def test_adam_moments_are_bias_corrected_weighted_averages():
    """Kingma and Ba's bias correction turns the moment recursions into
    normalised exponential averages: after steps 1..t with gradients g_1..g_t,
    m_hat_t = sum_i b1^(t-i) g_i / sum_i b1^(t-i) and likewise v_hat_t with
    b2 and g_i^2.  Three different gradients make both betas show: swapped or
    wrong betas, a missing bias correction or a stale moment all change the
    result.  Weights at b1 = 0.9, b2 = 0.999 written out: (0.81, 0.9, 1) / 2.71
    and (0.998001, 0.999, 1) / 2.997001 at step 3."""
    rng = np.random.default_rng(6)
    p = random_params(7)
    G = [rng.standard_normal(mlp.TRAINABLE) for _ in range(3)]
    lr = 2e-3
    m1 = np.zeros(mlp.TRAINABLE)
    m2 = np.zeros(mlp.TRAINABLE)
    q = p.copy()
    expect = p[:mlp.TRAINABLE].copy()
    w1 = {1: [1.0], 2: [0.9, 1.0], 3: [0.81, 0.9, 1.0]}
    w2 = {1: [1.0], 2: [0.999, 1.0], 3: [0.998001, 0.999, 1.0]}
    for t in (1, 2, 3):
        q, m1, m2 = mlp.adam(q, G[t - 1], m1, m2, t, lr)
        mh = sum(w * g for w, g in zip(w1[t], G[:t])) / sum(w1[t])
        vh = sum(w * g * g for w, g in zip(w2[t], G[:t])) / sum(w2[t])
        expect -= lr * mh / (np.sqrt(vh) + 1e-8)
    np.testing.assert_allclose(q[:mlp.TRAINABLE], expect, rtol=0, atol=1e-12)
    assert sum(w1[3]) == pytest.approx(2.71) and sum(w2[3]) == pytest.approx(2.997001)
    # the betas matter: the same three steps with them swapped land elsewhere
    r, a, c = p.copy(), np.zeros(mlp.TRAINABLE), np.zeros(mlp.TRAINABLE)
    for t in (1, 2, 3):
        r, a, c = mlp.adam(r, G[t - 1], a, c, t, lr, b1=0.999, b2=0.9)
    assert np.abs(r[:mlp.TRAINABLE] - expect).max() > 1e-4


def test_features_definition():
    f = mlp.features(np.array([4.0, 2.0, 1.0]), 1000, 10, 1e-6)
    assert f[0] == 0.0 and abs(f[1] - np.log10(0.5)) < 1e-15 and abs(f[2] - np.log10(0.25)) < 1e-15
    assert f[3] == -30.0  # missing pivots read as the floor
    assert (f[32], f[33], f[34]) == (3.0, 1.0, -6.0)


def test_ranks_from_trace_equal_runs_at_each_tolerance():
    """The predictor's labels at scale: one run of Algorithm 1 at the tightest
    tolerance gives, through its estimates E^(t), the rank a run at each looser
    tolerance returns (the loop stops at the first t with E^(t) <= tol ||A||_F and
    the estimates do not depend on tol).  Checked against separate oracle runs."""
    import oracle
    from paper_2310_09417_gb300 import workloads as W
    from paper_2310_09417_gb300.predictor import ranks_from_trace
    m, n, b = 500, 300, 16
    for kind in ("geometric", "poly", "fast_decay"):
        A = W.spectral_matrix(m, n, W.spectrum(kind, n), seed=len(kind))
        Om = W.gaussian_omega(5, oracle.rows_needed(n, b), m)
        nA = oracle.fro_norm(A)
        tols = [10.0 ** -e for e in (2, 3, 4, 5, 6, 8, 10, 13)]
        tight = oracle.id_adaptive(A, Om, b, min(tols) * nA)
        ks = ranks_from_trace(tight["trace"], nA, tols, b, n)
        for tol, k in zip(tols, ks):
            assert oracle.id_adaptive(A, Om, b, tol * nA)["k"] == k, (kind, tol)
