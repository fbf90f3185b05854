"""Pins of the oracle's training side (StatNet / RRSNet losses, gradients, optimizer,
reverse pass) against closed forms, exact variances and finite differences."""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2510_07868_b300 import inputs as I
from tests.conftest import paper_constant


def _params(n_out, seed):
    rng = np.random.default_rng(seed)
    n = oracle.mlpn_param_count(n_out)
    return rng.normal(scale=0.3, size=n)


def test_mlpn_backward_finite_differences():
    P = _params(6, 1)
    rng = np.random.default_rng(2)
    x = rng.normal(size=16)
    dout = rng.normal(size=6)
    G = oracle.mlpn_backward(P, 6, x, dout)
    h = 1e-6
    for i in list(rng.choice(len(P), 50, replace=False)) + [0, len(P) - 1]:
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += h
        Pm[i] -= h
        fd = (dout @ oracle.mlpn_forward(Pp, 6, x) - dout @ oracle.mlpn_forward(Pm, 6, x)) / (2 * h)
        assert abs(fd - G[i]) < 1e-7 + 1e-6 * abs(G[i])


def test_mlpn_single_output_is_rrsnet_preactivation():
    """With one output the generic MLP is RRSNet before its output activation."""
    P = I.rrsnet_init_params(3).astype(np.float64)
    for x in I.random_features(5, seed=4).astype(np.float64):
        q, z, _, _ = oracle.mlp_forward(P, x)
        assert oracle.mlpn_forward(P, 1, x)[0] == z


def test_statnet_relative_l2():
    """Eq. loss-function_StatNet with the stop-gradient on the prediction: zero at the
    targets; the mean gradient over a set of one-sample targets vanishes exactly at their
    mean (so noisy targets, most of them zero, do not bias the prediction — normalising
    by the targets instead would stop at a weighted mean); relative (scale invariant)."""
    L = np.array([0.3, 2.0, 0.0])
    loss, d = oracle.statnet_dloss(np.r_[L, L * L], L)
    assert loss == 0.0 and np.all(d == 0)
    targets = [np.array([0.0, 0.0, 0.0]), np.array([0.0, 1.0, 0.0]),
               np.array([4.0, 0.0, 0.5]), np.array([0.0, 3.0, 0.5])]
    mean1 = np.mean(targets, axis=0)
    mean2 = np.mean([t * t for t in targets], axis=0)
    grads = np.array([oracle.statnet_dloss(np.r_[mean1, mean2], t)[1] for t in targets])
    np.testing.assert_allclose(grads.sum(axis=0), 0.0, atol=1e-12)
    # away from the mean the summed gradient points back towards it
    g_hi = sum(oracle.statnet_dloss(np.r_[mean1 * 1.5 + 0.1, mean2], t)[1] for t in targets)
    assert np.all(g_hi[:3] > 0)
    # relative: scaling targets and predictions together by c leaves the loss unchanged
    # when eps is negligible
    pred = np.random.default_rng(5).normal(size=6)
    l1, _ = oracle.statnet_dloss(pred * 1.5, L + 0.1, eps=1e-30)
    l2, _ = oracle.statnet_dloss(np.r_[pred[:3] * 1.5e3, pred[3:] * 1.5e6], (L + 0.1) * 1e3,
                                 eps=1e-30)
    assert l1 == pytest.approx(l2, rel=1e-9)


def test_pixel_error_closed_form():
    # two samples a, b per pixel: unbiased variance (a-b)^2/2, of the mean: /2
    S1 = np.array([[[1.0, 1, 1], [3.0, 3, 3]], [[2.0, 0, 4], [2.0, 0, 4]]])
    ref = np.array([[2.0, 2, 2], [1.0, 1, 1]])
    V, E = oracle.pixel_error(S1, 2, ref, eps=0.01)
    assert V[0] == pytest.approx(1.0) and V[1] == 0.0
    assert E[0] == pytest.approx(1.0 / (4.0 + 0.01))


def _exact_rrs_variance(q, hv, hp):
    """Exact variance of Y = (1/q) sum_{j < X} H_j, X = floor(q) + Bernoulli(q - floor q),
    H_j i.i.d. over values hv with probabilities hp (enumeration)."""
    k = math.floor(q)
    r = q - k
    EY = EY2 = 0.0
    for X, px in ((k, 1 - r), (k + 1, r)):
        if px == 0:
            continue
        for combo in itertools.product(range(len(hv)), repeat=X):
            p = px * np.prod([hp[c] for c in combo]) if X else px
            y = sum(hv[c] for c in combo) / q
            EY += p * y
            EY2 += p * y * y
    return EY2 - EY * EY


def test_gradient_transfer_matches_exact_variance_derivative():
    """Eq. gradient_transfer_rr_mc / splitting_mc: for roulette (q < 1)
    dV/dq = -t^2 E[H^2] / q^2, for integer splitting dV/dq = -t^2 V[H] / q^2.  The oracle's
    dq (with g2 = 1, k = 1, I^2 + eps = 1, F = 1, t = 1) must equal the derivative of the
    exact variance of the estimator, by central differences."""
    hv, hp = [0.2, 1.5], [0.7, 0.3]
    m1 = hv[0] * hp[0] + hv[1] * hp[1]
    m2 = hv[0] ** 2 * hp[0] + hv[1] ** 2 * hp[1]
    for q in (0.3, 0.7, 2.0, 3.0):
        h = 1e-4 if q < 1 else 0.0
        if q < 1:
            fd = (_exact_rrs_variance(q + h, hv, hp) - _exact_rrs_variance(q - h, hv, hp)) / (2 * h)
        else:
            # integer splitting: V(q) = V[H]/q on integers; the paper ignores the rounding
            # term, so compare with the derivative of V[H]/q through q -> q +- 1
            v_m = _exact_rrs_variance(q - 1, hv, hp) * (q - 1)  # = V[H]
            fd = -v_m / q ** 2
            assert _exact_rrs_variance(q, hv, hp) == pytest.approx(v_m / q, rel=1e-12)
        dq, _ = oracle.rrsnet_dloss([q], [1.0], [0.0], [1.0], [0], [m1], [m2], E=[0.0],
                                    Iref=[math.sqrt(1 - 0.01)], k=[1], g=(0.0, 1.0, 0.0))
        assert dq[0] == pytest.approx(fd, rel=1e-6)


def test_pixel_loss_derivative_matches_finite_differences():
    """d(g1 L_avg + g2 L_min)/dE_i = g1 2 (E_i - Ebar) + g2: the Ebar terms cancel."""
    g1, g2 = paper_constant("gamma1"), paper_constant("gamma2")
    rng = np.random.default_rng(7)
    E = rng.uniform(0, 2, 9)
    Iref = np.full(9, math.sqrt(1 - 0.01))
    k = np.ones(9, dtype=np.int64)
    for i in range(9):
        dq, _ = oracle.rrsnet_dloss([0.5], [1.0], [0.0], [1.0], [i], [0.0], [1.0], E, Iref, k,
                                    g=(g1, g2, 0.0))
        # dq = dL/dE_i * dV/dq with dV/dq = -1/0.25 = -4
        dLdE = dq[0] / -4.0

        def L(Ev):
            _, t = oracle.rrsnet_dloss([0.5], [1.0], [0.0], [1.0], [0], [0.0], [1.0], Ev, Iref, k)
            return g1 * t[0] + g2 * t[1]

        e = np.zeros(9)
        e[i] = 1e-6
        assert dLdE == pytest.approx((L(E + e) - L(E - e)) / 2e-6, rel=1e-5)


def test_bound_loss_and_sharing():
    # L_rrs with Fn = 0: (q - 0)^2, gradient 2 q; with Fn = 1: zero
    dq, t = oracle.rrsnet_dloss([1.7], [1.0], [0.0], [1.0], [0], [0.0], [0.0], [0.0], [1.0], [1],
                                g=(0, 0, 1.0))
    assert t[2] == pytest.approx(1.7 ** 2) and dq[0] == pytest.approx(3.4)
    dq, t = oracle.rrsnet_dloss([1.7], [1.0], [1.0], [1.0], [0], [0.0], [0.0], [0.0], [1.0], [1],
                                g=(0, 0, 1.0))
    assert t[2] == 0 and dq[0] == 0
    # the pixel loss is shared: k_i samples each get 1/k_i
    args = dict(Fn=[0.0], t=[1.0], pixel=[0], m1=[0.0], m2=[1.0], E=[0.5], Iref=[1.0])
    d1, _ = oracle.rrsnet_dloss([0.5], [1.0], k=[1], g=(0, 1, 0), **args)
    d4, _ = oracle.rrsnet_dloss([0.5], [1.0], k=[4], g=(0, 1, 0), **args)
    assert d4[0] == pytest.approx(d1[0] / 4)


def test_adam_first_step_and_convergence():
    """Adam's first step moves each weight by -lr sign(g) (bias-corrected moments),
    and it minimises a quadratic."""
    P = np.array([1.0, -2.0, 3.0])
    m = np.zeros(3)
    v = np.zeros(3)
    oracle.adam_step(P, np.array([0.5, -4.0, 1e-3]), m, v, 1, 0.01)
    np.testing.assert_allclose(P, [0.99, -1.99, 2.99], atol=1e-7)
    P = np.array([5.0, -3.0])
    m = np.zeros(2)
    v = np.zeros(2)
    for step in range(1, 3001):
        oracle.adam_step(P, 2 * (P - np.array([1.0, 2.0])), m, v, step, 0.05)
    np.testing.assert_allclose(P, [1.0, 2.0], atol=1e-3)


def test_ema_closed_form():
    E = np.array([0.0, 10.0])
    P = np.array([1.0, 2.0])
    for _ in range(7):
        oracle.ema(E, P, 0.99)
    np.testing.assert_allclose(E, P + 0.99 ** 7 * (np.array([0.0, 10.0]) - P), rtol=1e-12)


def test_reverse_pass_furnace_closed_form():
    """In the furnace (albedo a = 0.5, emission 1, no RRS) the outgoing radiance estimate
    S / t of a vertex at depth d is exactly sum_{k <= D-d} a^k."""
    s = I.box_scene(1, furnace=True)
    D = 6
    img, st, _ = oracle.render(s, 8, 8, 2, D, oracle.MODE_NONE, record=True)
    for d in range(D):
        r = st["rec"][d]
        Lo = r[:, 0:3] / r[:, 6:9]
        assert np.all(Lo == (1 - 0.5 ** (D - d)) / 0.5)


def test_reverse_pass_sums_to_the_image():
    """Per pixel, the mean over spp of the depth-1 suffix sums is the rendered value."""
    s = I.box_scene(2)
    P = I.rrsnet_init_params(2).astype(np.float64)
    img, st, _ = oracle.render(s, 12, 10, 3, 7, oracle.MODE_NET, params=P, record=True)
    S1 = st["rec"][0][:, 0:3].reshape(120, 3, 3)
    np.testing.assert_allclose(S1.mean(1), img.reshape(-1, 3), rtol=1e-12, atol=1e-15)
    # children bookkeeping: sum of X at depth d = requested children
    for d in range(6):
        assert st["rec"][d][:, 11].sum() == st["requested"][d]
