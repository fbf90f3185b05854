"""The NRRS network inputs in the FP64 oracle (CPU), Sec. 4 "Input Encoding".

RRSNet's inputs are observed through its output: a selector network whose output is
(1 + 1e-6) x input k for either sign (two hidden units carry +x and -x through the Leaky
ReLUs, the last layer takes their difference), so each depth-1 factor q_orig of a
recorded frame reveals input k of that vertex.  StatNet is a selector too (E[L_o]_c =
(1 + 1e-6) albedo_c, E[L_o^2]_c = (1 + 1e-6) albedo of another channel), so every
input has a closed-form value from the scene: Box-Cox(lambda 0.5) of the statistics and of the throughput (1 at depth
1), Box-Cox of the pixel estimate's mean, 1 - exp(-roughness), zeros after that."""
import numpy as np
import pytest

import oracle
from paper_2510_07868_b300 import inputs as I

NF, NH = 16, 32
K = 1.0 + 1e-6


def _softplus_mod(x):
    return np.where(x < 0, np.log1p(np.exp(np.minimum(x, 0))), 0.5 * x + np.log(2.0))


def _boxcox(x):
    return 2.0 * (np.sqrt(x) - 1.0)


def _selector(n_out, picks):
    """MLP 16 -> 32 -> 32 -> 32 -> n_out whose output o is K * x[picks[o]]."""
    W1 = np.zeros((NH, NF))
    W2 = np.zeros((NH, NH))
    W3 = np.zeros((NH, NH))
    W4 = np.zeros((n_out, NH))
    for o, k in enumerate(picks):
        a, b = 2 * o, 2 * o + 1
        W1[a, k], W1[b, k] = 1.0, -1.0
        W2[a, a] = W2[b, b] = W3[a, a] = W3[b, b] = 1.0
        W4[o, a], W4[o, b] = 1.0, -1.0
    return np.concatenate([W1.ravel(), W2.ravel(), W3.ravel(), W4.ravel()])


def _depth1(scene, k, stat, ref_value, W=8, H=8, spp=2):
    ref = np.full((H * W, 3), ref_value)
    _, st, tr = oracle.render(scene, W, H, spp, 2, oracle.MODE_NET, params=_selector(1, [k]),
                              stat_params=stat, rrsnet_inputs=1, pixel_ref=ref, record=True,
                              trace=True)
    rec = st["rec"][0]
    tri = tr[0][:, 3].astype(np.int64)
    went_on = rec[:, 9] > 0
    return rec[went_on, 9], tri[went_on]


def test_selector_network_reads_one_input():
    x = np.linspace(-2, 3, NF)
    for k in (0, 5, 15):
        out = oracle.mlpn_forward(_selector(1, [k]), 1, x)
        assert abs(out[0] - K * x[k]) <= 1e-12 * max(1.0, abs(x[k]))


@pytest.mark.parametrize("k", list(range(16)))
def test_nrrs_inputs_box_scene(k):
    s = I.box_scene(4)
    stat = _selector(6, [9, 10, 11, 11, 9, 10])  # E[L] <- albedo, E[L^2] <- albedo rotated
    ref_value = 2.5
    q, tri = _depth1(s, k, stat, ref_value)
    assert q.size > 50
    alb = s.mats["albedo"][s.mat_id[tri]].astype(np.float64)
    if k <= 2:
        f = _boxcox(K * alb[:, k])
    elif k <= 5:
        f = _boxcox(K * alb[:, [2, 0, 1][k - 3]])
    elif k <= 8:
        f = np.zeros_like(q)  # Box-Cox of the depth-1 throughput 1
    elif k == 9:
        f = np.full_like(q, _boxcox(ref_value))
    elif k == 10:
        f = np.full_like(q, 1.0 - np.exp(-1.0))  # Lambertian: roughness 1
    else:
        f = np.zeros_like(q)
    # the recorded q_orig is the FP32 value the split decides on
    np.testing.assert_allclose(q, _softplus_mod(K * f), rtol=1e-7, atol=0)


def test_nrrs_roughness_input_ggx():
    s = I.icosphere_room(5, min_triangles=1500, subdiv=2)
    stat = _selector(6, [9, 10, 11, 6, 7, 8])
    q, tri = _depth1(s, 10, stat, 1.0, W=12, H=12)
    m = s.mats[s.mat_id[tri]]
    alpha = np.where(m["type"] == I.MAT_GGX, m["roughness"].astype(np.float64), 1.0)
    assert (m["type"] == I.MAT_GGX).any() and (m["type"] == I.MAT_LAMBERT).any()
    np.testing.assert_allclose(q, _softplus_mod(K * (1.0 - np.exp(-alpha))), rtol=1e-7)


def test_nrrs_statistics_clamped_at_zero():
    """A StatNet predicting negative statistics: the inputs are Box-Cox(0) = -2."""
    s = I.box_scene(4)
    stat = _selector(6, [9, 10, 11, 9, 10, 11])
    stat[-6 * NH:] *= -1.0  # negated last layer: E[L]_c = -K albedo_c < 0
    q, _ = _depth1(s, 0, stat, 1.0)
    np.testing.assert_allclose(q, _softplus_mod(K * np.full_like(q, -2.0)), rtol=1e-7)


def test_nrrs_inputs_need_statnet():
    with pytest.raises(RuntimeError):
        oracle.render(I.box_scene(1), 4, 4, 1, 2, oracle.MODE_NET, params=_selector(1, [0]),
                      rrsnet_inputs=1)


# ------------------------------------------------------------------ AID-NRRS inputs
def _selector32(k):
    """RRSNet with 32 inputs whose pre-activation is K * x[k] for either sign."""
    W1 = np.zeros((NH, 32))
    W2 = np.zeros((NH, NH))
    W3 = np.zeros((NH, NH))
    W4 = np.zeros((1, NH))
    W1[0, k], W1[1, k] = 1.0, -1.0
    W2[0, 0] = W2[1, 1] = W3[0, 0] = W3[1, 1] = 1.0
    W4[0, 0], W4[0, 1] = 1.0, -1.0
    return np.concatenate([W1.ravel(), W2.ravel(), W3.ravel(), W4.ravel()])


def test_aid_inputs_layout():
    tab = np.random.default_rng(11).normal(size=oracle.grid_param_count())
    p = np.array([0.25, 0.5, 0.75])
    x = oracle.aid_inputs(tab, p, [0.0, 0.0, 1.0], [1.0, 4.0, 0.25], 4.0, 0.0)
    np.testing.assert_allclose(x[:16], oracle.grid_encode(tab, p)[0], atol=1e-15)
    np.testing.assert_allclose(x[16:20], oracle.one_blob(0.0, 4), atol=1e-15)
    np.testing.assert_allclose(x[20:24], oracle.one_blob(0.5, 4), atol=1e-15)
    np.testing.assert_allclose(x[24:27], [0.0, 2.0, -1.0], atol=1e-15)  # Box-Cox of t
    assert x[27] == 2.0  # Box-Cox of I = 4
    np.testing.assert_allclose(x[28:32], oracle.one_blob(0.0, 4), atol=1e-15)
    x = oracle.aid_inputs(tab, p, [0.0, 0.0, 1.0], [1.0, 1.0, 1.0], -3.0, 1.0)
    assert x[27] == -2.0  # a negative estimate counts as 0
    np.testing.assert_allclose(x[28:32], oracle.one_blob(1 - np.exp(-1.0), 4), atol=1e-15)


@pytest.mark.parametrize("k", [16, 20, 24, 25, 26, 27, 28, 29, 30, 31])
def test_aid_inputs_in_render(k):
    """The render's AID-NRRS path feeds RRSNet the encoding: at depth 1 (throughput 1)
    of the Lambertian box each input has a closed form or the oracle's encoding value."""
    s = I.box_scene(4)
    tab = np.random.default_rng(12).normal(size=oracle.grid_param_count()) * 0.1
    ref_value = 2.25
    W = H = 8
    ref = np.full((H * W, 3), ref_value)
    _, st, tr = oracle.render(s, W, H, 2, 2, oracle.MODE_NET, params=_selector32(k),
                              rrsnet_inputs=2, rrs_grid=tab, pixel_ref=ref, record=True,
                              trace=True)
    rec = st["rec"][0]
    went_on = rec[:, 9] > 0
    q = rec[went_on, 9]
    assert q.size > 50
    if 24 <= k <= 26:
        f = np.zeros_like(q)
    elif k == 27:
        f = np.full_like(q, _boxcox(ref_value))
    elif k >= 28:
        f = np.full_like(q, oracle.one_blob(1 - np.exp(-1.0), 4)[k - 28])
    else:  # one-blob of w_o: in (0, 1], recomputed from each camera ray
        pix = tr[0][went_on, 0].astype(np.int64)
        smp = tr[0][went_on, 1]
        f = np.empty_like(q)
        for j, (pp, ss) in enumerate(zip(pix, smp)):
            w = oracle.philox([pp, ss, 0, 0], [1, 0])
            _, d = oracle.camera_ray(s, W, H, int(pp % W), int(pp // W), (w[0] >> 8) / 2 ** 24,
                                     (w[1] >> 8) / 2 ** 24)
            x = oracle.aid_inputs(tab, [0.5, 0.5, 0.5], -d, [1.0, 1.0, 1.0], 0.0, 1.0)
            f[j] = x[k]
    np.testing.assert_allclose(q, _softplus_mod(K * f), rtol=1e-6)


def test_aid_inputs_need_grid():
    with pytest.raises(RuntimeError):
        oracle.render(I.box_scene(1), 4, 4, 1, 2, oracle.MODE_NET, params=_selector32(0),
                      rrsnet_inputs=2)
