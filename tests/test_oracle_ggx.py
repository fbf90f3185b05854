"""Pins of the oracle's GGX lobe, heuristic factor and error-map smoothing (CPU).

The paper prints no BSDF, so the GGX + Lambert mixture (Walter et al. 2007, Smith
masking, Schlick Fresnel) is pinned by identities of the microfacet model that any
correct implementation satisfies, each evaluated by quadrature written here:

* D is normalised: the integral of D(h) (n.h) over the hemisphere is 1;
* Smith's masking identity: G1(o) times the integral of max(0, o.h) D(h) over the
  hemisphere equals o.n;
* the expected sampling weight E[f cos / pdf] over the sampler's random numbers equals
  the integral of f cos over the hemisphere (so the sampler draws from the pdf it
  divides by);
* at normal incidence f cos and pdf take closed forms (D(n) = 1 / (pi a^2), G1 = 1,
  Fresnel = F0);
* away from normal incidence the Fresnel term stays within Schlick's published error of
  the exact Fresnel equations of the dielectric with the same normal reflectance.

A dropped 1/pi in D, a instead of a^2, a wrong Smith term, a missing factor 4 in the
half-vector Jacobian, a wrong Fresnel base or a wrong Schlick exponent each fail one of
them.  The heuristic factor
of Sec. 4 ("Compromise": the reference is the accumulated estimate) is pinned by its
closed form at depth 1, where the throughput is 1; the temporal EMA and the spatial
filter of Sec. 4 "Tackle Low Spp" by closed forms and by library convolutions.
"""
import math

import numpy as np
import pytest
from scipy import integrate, ndimage

import oracle
from paper_2510_07868_b300 import inputs as I

ROUGH = (0.05, 0.2, 0.5)


def _theta_points(a):
    # the lobe of D has its width near atan(a): help the adaptive quadrature find it
    return [math.atan(a * s) for s in (0.25, 1.0, 4.0, 16.0) if math.atan(a * s) < math.pi / 2]


@pytest.mark.parametrize("a", ROUGH)
def test_ggx_D_projected_area_is_one(a):
    f = lambda th: oracle.ggx_D(math.cos(th), a) * math.cos(th) * math.sin(th)  # noqa: E731
    v, err = integrate.quad(f, 0.0, math.pi / 2, points=_theta_points(a), limit=400,
                            epsabs=1e-13, epsrel=1e-12)
    assert abs(2.0 * math.pi * v - 1.0) < 1e-9, (a, 2 * math.pi * v)


def _phi_integral_of_positive_cos(A, B):
    """Integral over phi in [0, 2 pi) of max(0, A cos(phi) + B), A >= 0, B >= 0."""
    if B >= A:
        return 2.0 * math.pi * B
    p0 = math.acos(-B / A)
    return 2.0 * (A * math.sin(p0) + B * p0)


@pytest.mark.parametrize("a", ROUGH)
@pytest.mark.parametrize("theta_o_deg", [0.0, 30.0, 60.0, 80.0])
def test_smith_masking_identity(a, theta_o_deg):
    """G1(o) * integral of max(0, o.h) D(h) dw_h = cos(theta_o) (Smith's G1 normalises the
    visible projected microfacet area to the projected macro-surface area)."""
    to = math.radians(theta_o_deg)
    so, co = math.sin(to), math.cos(to)

    def f(th):
        A, B = so * math.sin(th), co * math.cos(th)
        return oracle.ggx_D(math.cos(th), a) * math.sin(th) * _phi_integral_of_positive_cos(A, B)

    v, _ = integrate.quad(f, 0.0, math.pi / 2, points=_theta_points(a), limit=400,
                          epsabs=1e-13, epsrel=1e-11)
    g1 = oracle.ggx_G1(co, a) if theta_o_deg > 0 else 1.0
    assert abs(g1 * v - co) < 1e-8 * max(co, 1e-3), (a, theta_o_deg, g1 * v, co)
    if theta_o_deg == 0.0:
        assert oracle.ggx_G1(1.0, a) == 1.0


def _hemisphere_grid(n_mu, n_phi):
    """Midpoint grid over (cos theta, phi) of the upper hemisphere: directions and the
    solid-angle weight of each cell (d omega = d cos(theta) d phi)."""
    mu = (np.arange(n_mu) + 0.5) / n_mu
    phi = (np.arange(n_phi) + 0.5) * (2.0 * math.pi / n_phi)
    M, P = np.meshgrid(mu, phi, indexing="ij")
    st = np.sqrt(1.0 - M * M)
    dirs = np.stack([st * np.cos(P), st * np.sin(P), M], axis=-1).reshape(-1, 3)
    return dirs, (1.0 / n_mu) * (2.0 * math.pi / n_phi)


@pytest.mark.parametrize("a", ROUGH)
@pytest.mark.parametrize("theta_o_deg", [20.0, 60.0])
def test_ggx_expected_sampling_weight_is_the_directional_albedo(a, theta_o_deg):
    n = np.array([0.0, 0.0, 1.0])
    to = math.radians(theta_o_deg)
    wo = np.array([math.sin(to), 0.0, math.cos(to)])
    albedo = np.array([0.5, 0.3, 0.8])
    F0 = 0.04
    # integral of f cos over the hemisphere; the narrow lobe (a = 0.05) needs a fine grid
    # around the mirror direction, so the quadrature splits cos(theta) near it
    dirs, dw = _hemisphere_grid(1600, 1600)
    fc, _ = oracle.eval_ggx_batch(n, wo, dirs, albedo, a, F0)
    albedo_quad = fc.sum(axis=0) * dw
    # expected weight over (ulobe, u1, u2): each lobe half on a midpoint grid of (u1, u2)
    k = 1024
    u1, u2 = np.meshgrid((np.arange(k) + 0.5) / k, (np.arange(k) + 0.5) / k, indexing="ij")
    est = np.zeros(3)
    for ulobe in (0.25, 0.75):
        u = np.stack([np.full(k * k, ulobe), u1.ravel(), u2.ravel()], axis=1)
        _, w = oracle.sample_ggx_batch(n, wo, albedo, a, F0, u)
        est += 0.5 * w.mean(axis=0)
    # the midpoint grids resolve the lobes to ~1e-4; the horizon cut-off leaves O(1/k)
    np.testing.assert_allclose(est, albedo_quad, rtol=2e-3)
    assert np.all(albedo_quad < 1.0)


@pytest.mark.parametrize("a", ROUGH)
def test_ggx_normal_incidence_closed_form(a):
    n = np.array([0.0, 0.0, 1.0])
    albedo = np.array([0.2, 0.5, 0.9])
    F0 = 0.04
    ok, fc, pdf = oracle.eval_ggx(n, n, n, albedo, a, F0)
    assert ok == 1
    # materials hold FP32 parameters: the closed form takes the same rounded values
    a32, F032 = float(np.float32(a)), float(np.float32(F0))
    alb32 = albedo.astype(np.float32).astype(np.float64)
    spec = F032 / (4.0 * math.pi * a32 * a32)  # D(n) G1^2 F0 / (4 cos cos), D(n) = 1/(pi a^2)
    np.testing.assert_allclose(fc, spec + (1.0 - F032) * alb32 / math.pi, rtol=1e-12)
    assert math.isclose(pdf, 0.5 / (4.0 * math.pi * a32 * a32) + 0.5 / math.pi, rel_tol=1e-12)
    assert math.isclose(oracle.ggx_D(1.0, a), 1.0 / (math.pi * a * a), rel_tol=1e-12)


def _fresnel_dielectric(cos_i, eta):
    """Unpolarised Fresnel reflectance of a smooth dielectric interface (the exact
    equations for the s and p polarisations, averaged)."""
    sin_t = math.sqrt(max(0.0, 1.0 - cos_i * cos_i)) / eta
    cos_t = math.sqrt(1.0 - sin_t * sin_t)
    rs = (cos_i - eta * cos_t) / (cos_i + eta * cos_t)
    rp = (cos_t - eta * cos_i) / (cos_t + eta * cos_i)
    return 0.5 * (rs * rs + rp * rp)


@pytest.mark.parametrize("a", ROUGH)
def test_ggx_fresnel_term_follows_the_dielectric_away_from_normal_incidence(a):
    """The lobe's Fresnel term, read back at the mirror direction, against the exact
    Fresnel equations of the dielectric whose normal reflectance is F0 (eta = 1.5 for
    F0 = 0.04).  Along the mirror direction h = n, so with albedo 0 the value is
    D(n) G1(o)^2 F(cos t) / (4 cos^2 t) and F follows from the separately pinned D and G1.
    Schlick's approximation stays within 0.036 of the exact reflectance up to 85 degrees;
    an exponent of 4 or 6 in place of 5 misses by 0.10 or 0.055."""
    n = np.array([0.0, 0.0, 1.0])
    F0 = float(np.float32(0.04))
    eta = (1.0 + math.sqrt(F0)) / (1.0 - math.sqrt(F0))
    a32 = float(np.float32(a))
    worst = 0.0
    for deg in np.linspace(0.0, 85.0, 35):
        t = math.radians(deg)
        wo = np.array([math.sin(t), 0.0, math.cos(t)])
        wi = np.array([-math.sin(t), 0.0, math.cos(t)])
        ok, fc, _ = oracle.eval_ggx(n, wo, wi, np.zeros(3), a, 0.04)
        assert ok == 1
        c = math.cos(t)
        F = fc[0] * 4.0 * c / (oracle.ggx_D(1.0, a32) * oracle.ggx_G1(c, a32) ** 2)
        assert abs(fc[0] - fc[1]) <= 1e-15 * abs(fc[0]) and abs(fc[0] - fc[2]) <= 1e-15 * abs(fc[0])
        worst = max(worst, abs(F - _fresnel_dielectric(c, eta)))
        if deg == 0.0:
            assert math.isclose(F, F0, rel_tol=1e-12)
    assert worst <= 0.037, worst


# ----------------------------------------------------------------------------- HEUR
def test_heuristic_factor_closed_form_at_depth_one():
    """Depth-1 vertices carry throughput 1, so HEUR's factor is
    min(lum(1,1,1) / max(mean_rgb(I_px), eps_I), q_max) = min(1 / max(I, eps_I), q_max),
    eps_I = 0.01 mean(I).  A coloured reference separates the mean over RGB from a
    luminance; dark pixels take the floor; a dim pixel hits the q_max clamp."""
    s = I.box_scene(1)
    W = H = 16
    spp, D = 2, 3
    rng = np.random.default_rng(7)
    ref = np.zeros((H, W, 3))
    kind = rng.integers(0, 3, W * H)
    cols = np.array([[30.0, 10.0, 2.0], [0.0, 0.0, 0.0], [0.02, 0.01, 0.03]])
    ref.reshape(-1, 3)[:] = cols[kind]
    eps_I = 0.01 * ref.mean()
    _, st, _ = oracle.render(s, W, H, spp, D, oracle.MODE_HEUR_NORM, pixel_ref=ref, record=True,
                             q_max=16.0)
    rec = st["rec"][0]
    pix = rec[:, 13].astype(np.int64)
    went_on = rec[:, 14:30].any(axis=1)  # vertices that reached the factor decision
    assert went_on.sum() > 100
    den = np.maximum(ref.reshape(-1, 3).mean(axis=1)[pix], eps_I)
    expect = np.minimum(1.0 / den, 16.0).astype(np.float32).astype(np.float64)
    np.testing.assert_array_equal(rec[went_on, 9], expect[went_on])
    for k in range(3):  # every case occurs: plain ratio, floor (dark), clamp (dim)
        assert np.any(went_on & (kind[pix] == k))
    assert np.any(expect[went_on] == 16.0) and np.any(expect[went_on] < 1.0)
    # without a reference the factor is lum(t) = 1
    _, st2, _ = oracle.render(s, W, H, spp, D, oracle.MODE_HEUR_NORM, record=True)
    r2 = st2["rec"][0]
    on2 = r2[:, 14:30].any(axis=1)
    assert np.all(r2[on2, 9] == 1.0)


# ------------------------------------------------------------------ error-map smoothing
def test_error_temporal_is_a_geometric_mixture():
    """E_acc after frames e_1 .. e_k: (1 - a)^(k-1) e_1 + sum_{j >= 2} a (1 - a)^(k-j) e_j."""
    rng = np.random.default_rng(2)
    frames = rng.exponential(size=(6, 50))
    for a in (0.5, 0.2):
        acc = None
        for k, e in enumerate(frames, start=1):
            acc = oracle.error_temporal(e, acc, alpha=a, first=(k == 1))
            w = np.array([(1 - a) ** (k - 1)] + [a * (1 - a) ** (k - j) for j in range(2, k + 1)])
            assert math.isclose(w.sum(), 1.0, rel_tol=1e-12)
            np.testing.assert_allclose(acc, w @ frames[:k], rtol=1e-12)
    const = oracle.error_temporal(np.full(5, 3.0), np.full(5, 3.0), alpha=0.5)
    assert np.all(const == 3.0)


def _box_mean(E, W, H, r, mask=None):
    """Mean over the clipped (2r+1)^2 window by convolution (scipy.ndimage)."""
    img = E.reshape(H, W)
    m = np.ones_like(img) if mask is None else mask.reshape(H, W).astype(np.float64)
    k = np.ones((2 * r + 1, 2 * r + 1))
    s = ndimage.convolve(img * m, k, mode="constant", cval=0.0)
    c = ndimage.convolve(m, k, mode="constant", cval=0.0)
    return (s / c).ravel()


def test_error_filter_unguided_is_the_clipped_box_mean():
    W, H, r = 23, 17, 2
    E = np.random.default_rng(3).exponential(size=W * H)
    np.testing.assert_allclose(oracle.error_filter(E, W, H, r), _box_mean(E, W, H, r), rtol=1e-12)
    # a flat normal field weighs every neighbour by 1 as well
    N = np.tile([0.0, 1.0, 0.0, 1.0], (W * H, 1))
    np.testing.assert_allclose(oracle.error_filter(E, W, H, r, N, 8.0), _box_mean(E, W, H, r),
                               rtol=1e-12)
    assert np.all(oracle.error_filter(np.full(W * H, 2.5), W, H, r) == 2.5)


def test_error_filter_orthogonal_normals_do_not_mix():
    """A checkerboard of two orthogonal normals: each pixel averages only the pixels of
    its own colour (weight cos^p(90 deg) = 0)."""
    W, H, r = 20, 14, 2
    E = np.random.default_rng(4).exponential(size=W * H)
    y, x = np.divmod(np.arange(W * H), W)
    black = (x + y) % 2 == 0
    N = np.where(black[:, None], [1.0, 0.0, 0.0, 1.0], [0.0, 0.0, 1.0, 1.0])
    out = oracle.error_filter(E, W, H, r, N, 8.0)
    expect = np.where(black, _box_mean(E, W, H, r, black), _box_mean(E, W, H, r, ~black))
    np.testing.assert_allclose(out, expect, rtol=1e-12)


def test_error_filter_two_pixel_weights():
    """Two pixels with normals at angle t: out_0 = (E_0 + c E_1) / (1 + c), c = cos(t)^p;
    a neighbour without a normal weighs 0, a pixel without one weighs all by 1."""
    t, p = 0.6, 5.0
    N = np.array([[0.0, 0.0, 1.0, 1.0], [math.sin(t), 0.0, math.cos(t), 1.0]])
    E = np.array([1.0, 4.0])
    c = math.cos(t) ** p
    out = oracle.error_filter(E, 2, 1, 1, N, p)
    np.testing.assert_allclose(out, [(1 + 4 * c) / (1 + c), (4 + c) / (1 + c)], rtol=1e-13)
    N[1, 3] = 0.0
    out = oracle.error_filter(E, 2, 1, 1, N, p)
    np.testing.assert_allclose(out, [1.0, 2.5], rtol=1e-13)


def test_pixel_normals_mean_of_the_vertices_that_went_on():
    spp = 3
    feat = np.zeros((2 * spp, 16))
    q = np.array([1.0, 0.0, 2.0, 0.0, 0.0, 0.0])
    feat[0, 6:9] = [1.0, 0.0, 0.0]
    feat[1, 6:9] = [0.0, 0.0, 1.0]  # q = 0: left out
    feat[2, 6:9] = [0.0, 1.0, 0.0]
    out = oracle.pixel_normals(feat, q, 2, spp)
    np.testing.assert_allclose(out[0], [1 / math.sqrt(2), 1 / math.sqrt(2), 0.0, 1.0], rtol=1e-14)
    assert np.all(out[1] == 0.0)
