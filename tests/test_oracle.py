"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published test
vectors, closed forms, invariants, exhaustive enumeration or finite differences.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2510_07868_b300 import inputs as I
from tests.conftest import golden, paper_constant


# ----------------------------------------------------------------------------- Philox
def test_philox_known_answers():
    """Salmon et al. 2011 known-answer vectors for Philox4x32-10."""
    rows = golden("philox4x32_10_kat.txt")
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox(v[0:4], v[4:6])
        assert list(out) == v[6:10]


# ----------------------------------------------------------------------------- camera / geometry
def test_camera_center_and_fov():
    s = I.box_scene(1)
    # odd image: the centre pixel with jitter 0.5 looks straight along +z
    o, d = oracle.camera_ray(s, 33, 33, 16, 16, 0.5, 0.5)
    np.testing.assert_allclose(o, [0.5, 0.5, 0.01], atol=1e-7)
    np.testing.assert_allclose(d, [0, 0, 1], atol=1e-15)
    # top edge of the image sits at half the vertical field of view (30 degrees)
    o, d = oracle.camera_ray(s, 33, 33, 16, 0, 0.5, 0.0)
    assert math.isclose(math.degrees(math.atan2(d[1], d[2])), 30.0, rel_tol=1e-12)
    # row 0 is the top of the image, column 0 the left (x grows to the right)
    _, d_left = oracle.camera_ray(s, 33, 33, 0, 16, 0.0, 0.5)
    assert d_left[0] < 0 and abs(d_left[1]) < 1e-15
    assert np.isclose(np.linalg.norm(d_left), 1.0)


def test_intersect_known_distances_and_ties():
    s = I.box_scene(1, n_random=0)
    # straight up from the box centre: emitter at y = 0.999 (triangles 12, 13)
    tri, t = oracle.intersect(s, [0.5, 0.5, 0.5], [0, 1, 0])
    assert tri in (12, 13) and math.isclose(t, 0.499, rel_tol=1e-6)
    # straight down: floor at y = 0
    tri, t = oracle.intersect(s, [0.3, 0.5, 0.3], [0, -1, 0])
    assert tri in (0, 1) and math.isclose(t, 0.5, rel_tol=1e-12)
    # outside the box, pointing away: miss
    tri, t = oracle.intersect(s, [0.5, 2.0, 0.5], [0, 1, 0])
    assert tri == -1 and math.isinf(t)
    # two identical triangles: the tie goes to the lower index
    dup = I.Scene(np.vstack([s.tri[0:1], s.tri[0:1]]), [0, 0], s.mats[:1], s.cam, "dup")
    tri, t = oracle.intersect(dup, [0.2, 0.5, 0.6], [0, -1, 0])
    assert tri == 0 and math.isclose(t, 0.5, rel_tol=1e-12)
    # a ray parallel to the triangle's plane never hits it
    tri, _ = oracle.intersect(dup, [0.2, 0.0, 0.6], [1, 0, 0])
    assert tri == -1


# ----------------------------------------------------------------------------- BSDF sampling
def _sphere_dirs(n, seed):
    g = np.random.default_rng(seed).normal(size=(n, 3))
    return g / np.linalg.norm(g, axis=1, keepdims=True)


def test_lambert_cosine_distribution():
    """Cosine-weighted hemisphere: P(cos <= c) = c^2, E[cos] = 2/3, E[wi] = 2/3 n."""
    rng = np.random.default_rng(3)
    normals = _sphere_dirs(8, 4)
    normals = np.vstack([normals, [[0, 0, 1], [0, 0, -1], [0.6, 0.8, -0.0]]])
    for n in normals:
        n = n / np.linalg.norm(n)
        m = 4000
        u = rng.uniform(size=(m, 2))
        W = np.array([oracle.sample_lambert(n, a, b) for a, b in u])
        np.testing.assert_allclose(np.linalg.norm(W, axis=1), 1.0, atol=1e-12)
        c = W @ n
        assert c.min() >= -1e-12
        for cut in (0.25, 0.5, 0.75):
            frac = np.mean(c <= cut)
            se = math.sqrt(cut * cut * (1 - cut * cut) / m)
            assert abs(frac - cut * cut) < 4 * se + 1e-9
        mean = W.mean(0)
        se = W.std(0) / math.sqrt(m)
        assert np.all(np.abs(mean - 2.0 / 3.0 * n) < 4 * se + 1e-9)


def test_lambert_concentric_corners():
    """Concentric map: u = (0.5, 0.5) is the disk centre -> wi = n exactly."""
    n = np.array([0.0, 1.0, 0.0])
    np.testing.assert_allclose(oracle.sample_lambert(n, 0.5, 0.5), n, atol=1e-15)


def test_ggx_mirror_limit_and_hemisphere():
    """GGX lobe: as roughness -> 0 the specular sample is the mirror direction; every
    accepted sample lies in the upper hemisphere with a finite, non-negative weight."""
    n = np.array([0.0, 0.0, 1.0])
    wo = np.array([0.6, 0.0, 0.8])
    ok, wi, w = oracle.sample_ggx(n, wo, [0.5] * 3, 1e-4, 0.04, 0.1, 0.3, 0.7)
    assert ok == 1
    np.testing.assert_allclose(wi, [-0.6, 0.0, 0.8], atol=1e-3)
    rng = np.random.default_rng(1)
    for _ in range(2000):
        ok, wi, w = oracle.sample_ggx(n, wo, [0.5] * 3, 0.3, 0.04, *rng.uniform(size=3))
        if ok:
            assert wi @ n > 0 and np.all(np.isfinite(w)) and np.all(w >= 0)
        else:
            assert np.all(w == 0)


# ----------------------------------------------------------------------------- RRSNet
def test_softplus_variant_closed_form():
    """Eq. rrsnet_activation: continuous at 0 with value ln 2, slope 1/2 for x >= 0,
    ln(1 + e^x) for x < 0."""
    ln2 = paper_constant("softplus_at_zero")
    assert oracle.softplus_mod(0.0) == ln2
    assert math.isclose(oracle.softplus_mod(-1e-12), ln2, rel_tol=1e-11)
    for x in (0.0, 0.5, 3.0, 100.0):
        assert math.isclose(oracle.softplus_mod(x), 0.5 * x + ln2, rel_tol=1e-15)
        assert oracle.softplus_mod_grad(x) == 0.5
    for x in (-0.5, -3.0, -30.0):
        assert math.isclose(oracle.softplus_mod(x), np.logaddexp(0.0, x), rel_tol=1e-14)
        assert math.isclose(oracle.softplus_mod_grad(x), 1 / (1 + math.exp(-x)), rel_tol=1e-14)
    assert math.isclose(oracle.softplus_mod_grad(-1e-12), 0.5, rel_tol=1e-11)


def test_mlp_zero_weights_and_selector_network():
    P = np.zeros(I.RRSNET_N_PARAMS)
    x = I.random_features(1, seed=2)[0].astype(np.float64)
    q, z, _, _ = oracle.mlp_forward(P, x)
    assert z == 0.0 and q == math.log(2.0)
    # a chain that routes feature 0 through neuron 0 of every layer: z = lrelu^3(x0)
    P = np.zeros(I.RRSNET_N_PARAMS)
    P[0] = 1.0                        # W1[0][0]
    P[512] = 1.0                      # W2[0][0]
    P[512 + 1024] = 1.0               # W3[0][0]
    P[512 + 2048] = 2.0               # W4[0][0]
    for x0 in (0.7, -0.7):
        x = np.zeros(16)
        x[0] = x0
        q, z, _, _ = oracle.mlp_forward(P, x)
        expect_z = 2.0 * (x0 if x0 > 0 else 1e-6 * x0)
        assert math.isclose(z, expect_z, rel_tol=1e-14)


def test_mlp_positive_homogeneity():
    """Bias-free Leaky-ReLU network: z(c x) = c z(x) for c > 0, and scaling any one
    layer's weights by c scales z by c (catches a stray bias or a wrong activation)."""
    P = I.rrsnet_init_params(5).astype(np.float64)
    X = I.random_features(20, seed=6).astype(np.float64)
    for x in X:
        _, z, _, _ = oracle.mlp_forward(P, x)
        _, z2, _, _ = oracle.mlp_forward(P, 3.0 * x)
        assert math.isclose(z2, 3.0 * z, rel_tol=1e-12, abs_tol=1e-14)
        for lo, hi in ((0, 512), (512, 1536), (1536, 2560), (2560, 2592)):
            Q = P.copy()
            Q[lo:hi] *= 2.5
            _, zq, _, _ = oracle.mlp_forward(Q, x)
            assert math.isclose(zq, 2.5 * z, rel_tol=1e-12, abs_tol=1e-14)


def test_mlp_backward_matches_finite_differences():
    P = I.rrsnet_init_params(7).astype(np.float64)
    X = I.random_features(3, seed=8).astype(np.float64)
    rng = np.random.default_rng(9)
    for x in X:
        G = oracle.mlp_backward(P, x, 1.0)
        idx = rng.choice(I.RRSNET_N_PARAMS, 60, replace=False)
        idx = np.r_[idx, [0, 511, 512, 1535, 1536, 2559, 2560, 2591]]
        h = 1e-6
        for i in idx:
            Pp = P.copy()
            Pm = P.copy()
            Pp[i] += h
            Pm[i] -= h
            fd = (oracle.mlp_forward(Pp, x)[0] - oracle.mlp_forward(Pm, x)[0]) / (2 * h)
            assert abs(fd - G[i]) < 1e-7 + 1e-5 * abs(G[i])
        # linear in the upstream gradient
        np.testing.assert_allclose(oracle.mlp_backward(P, x, -2.0), -2.0 * G, rtol=1e-14, atol=0)


def test_boxcox():
    assert oracle.boxcox(1.0, 0.5) == 0.0
    assert oracle.boxcox(4.0, 0.5) == 2.0
    assert math.isclose(oracle.boxcox(0.25, 0.5), -1.0, rel_tol=1e-15)
    # lambda -> 0 tends to log
    assert math.isclose(oracle.boxcox(3.0, 1e-9), math.log(3.0), rel_tol=1e-6)
    assert oracle.boxcox(3.0, 0.0) == math.log(3.0)


# ----------------------------------------------------------------------------- normalisation
def test_normalize_closed_forms():
    # downscale only (Sec. 4 "Compromise"): small totals keep F = 1
    F, s = oracle.normalize(np.ones(100), budget=200, f_rate=0.85)
    assert F == 1.0 and s == 100.0
    # Eq. F_norm * f_rate: 1000 unit factors, budget 200 -> F = 0.85 * 200 / 1000
    F, s = oracle.normalize(np.ones(1000), budget=200, f_rate=0.85)
    assert math.isclose(F, 0.17, rel_tol=1e-15)
    # alpha scales the target (Eq. f_rate_prime)
    F2, _ = oracle.normalize(np.ones(1000), budget=200, f_rate=0.85, alpha=0.99)
    assert math.isclose(F2, 0.17 * 0.99, rel_tol=1e-15)
    # an empty or all-zero queue is left alone
    assert oracle.normalize(np.zeros(5), budget=10)[0] == 1.0
    assert oracle.normalize(np.zeros(0), budget=10)[0] == 1.0
    # sum of normalised factors equals f * alpha * budget whenever F < 1
    q = I.random_q(5000, seed=3, scale=8).astype(np.float64)
    F, s = oracle.normalize(q, budget=1000, f_rate=0.85, alpha=0.97)
    assert F < 1 and math.isclose((F * q).sum(), 0.85 * 0.97 * 1000, rel_tol=1e-12)


def test_bernstein_exponent_matches_paper():
    c = oracle.bernstein_exponent(0.85)
    assert math.isclose(c, paper_constant("bernstein_exponent_f085"), rel_tol=1e-3)
    assert oracle.bernstein_exponent(1.0) == 0.0


# ----------------------------------------------------------------------------- split
def _ids(n):
    return np.arange(n, dtype=np.uint32), np.zeros(n, np.uint32), np.zeros(n, np.uint32)


def test_split_integer_factors_are_deterministic():
    q = np.array([0, 1, 2, 3, 0, 5], dtype=np.float32)
    pix, smp, lin = _ids(len(q))
    X, prefix, cp, cl, S, drop = oracle.split(q, 1.0, pix, smp, lin, depth=1)
    assert list(X) == [0, 1, 2, 3, 0, 5]
    assert list(prefix) == [0, 0, 1, 3, 6, 6]
    assert S == 11 and drop == 0
    assert list(cp) == [1, 2, 2, 3, 3, 3, 5, 5, 5, 5, 5]
    # lineages of siblings differ by the golden-ratio step
    assert (int(cl[2]) - int(cl[1])) % 2**32 == 0x9E3779B9


def test_split_cap_drops_and_counts():
    q = np.array([3, 3, 3], dtype=np.float32)
    pix, smp, lin = _ids(3)
    X, prefix, cp, cl, S, drop = oracle.split(q, 1.0, pix, smp, lin, depth=2, cap=7)
    assert S == 9 and drop == 2 and len(cp) == 7 and list(cp) == [0, 0, 0, 1, 1, 1, 2]


def test_split_matches_exhaustive_enumeration():
    """Sec. 3.1 "Boundedness": with X_i = k_i + Bernoulli(r_i) independent, the law of
    S is the convolution over all 2^n Bernoulli outcomes.  Compare the oracle's split
    over many Philox keys with that law (chi-square) and with E[S] = sum q,
    Var(S) = sum r(1-r) <= rho <= N and <= n/4."""
    rng = np.random.default_rng(11)
    n = 10
    q = rng.uniform(0, 2.5, n).astype(np.float32)
    F32 = np.float32(0.8)
    qu = (F32 * q).astype(np.float32)
    k = np.floor(qu).astype(np.int64)
    r = (qu - k).astype(np.float64)
    law = {}
    for bits in itertools.product((0, 1), repeat=n):
        p = 1.0
        for b, ri in zip(bits, r):
            p *= ri if b else 1 - ri
        s = int(k.sum() + sum(bits))
        law[s] = law.get(s, 0.0) + p
    pix, smp, lin = _ids(n)
    trials = 4000
    counts = {}
    for frame in range(trials):
        _, _, _, _, S, _ = oracle.split(q, F32, pix, smp, lin, depth=3, frame=frame)
        counts[S] = counts.get(S, 0) + 1
    assert set(counts) <= set(law)
    chi2, dof = 0.0, -1
    for s, p in law.items():
        if p * trials >= 5:
            chi2 += (counts.get(s, 0) - p * trials) ** 2 / (p * trials)
            dof += 1
    assert chi2 < dof + 5 * math.sqrt(2 * dof)
    mean = sum(s * p for s, p in law.items())
    var = sum((s - mean) ** 2 * p for s, p in law.items())
    assert math.isclose(mean, float(qu.astype(np.float64).sum()), rel_tol=1e-12)
    assert math.isclose(var, float((r * (1 - r)).sum()), rel_tol=1e-9)
    rho = r.sum()
    assert var <= rho <= qu.astype(np.float64).sum() and var <= n / 4


def test_split_per_path_unbiased():
    """E[X_i] = q_used_i (Sec. 3.1, proof step (1)), per path, over many keys."""
    q = np.array([0.05, 0.5, 0.95, 1.3, 2.75], dtype=np.float32)
    pix, smp, lin = _ids(len(q))
    trials = 6000
    tot = np.zeros(len(q))
    for frame in range(trials):
        X, *_ = oracle.split(q, 1.0, pix, smp, lin, depth=1, frame=frame)
        tot += X
    mean = tot / trials
    r = q - np.floor(q)
    se = np.sqrt(r * (1 - r) / trials)
    assert np.all(np.abs(mean - q) < 4 * se + 1e-12)


def test_bernstein_bound_holds_empirically():
    """Eq. bernstein_frate: P(S' >= N) <= exp(-c(f) N) for normalised, rate-controlled q."""
    rng = np.random.default_rng(12)
    N = 64
    f = 0.5
    qo = rng.uniform(0.1, 3.0, 100)
    F, _ = oracle.normalize(qo, budget=N, f_rate=f)
    q = (F * qo).astype(np.float32)
    pix, smp, lin = _ids(len(q))
    over = 0
    trials = 3000
    for frame in range(trials):
        _, _, _, _, S, _ = oracle.split(q, 1.0, pix, smp, lin, depth=1, frame=frame)
        over += S >= N
    bound = math.exp(-oracle.bernstein_exponent(f) * N)
    assert over / trials <= bound + 3 * math.sqrt(bound / trials)


# ----------------------------------------------------------------------------- render
def test_furnace_closed_form_exact():
    """Closed box, albedo a = 0.5 and emission 1 everywhere, no RRS: every sample
    deposits sum_{k<D} a^k = (1 - a^D)/(1 - a) exactly (Lambertian weight = albedo)."""
    s = I.box_scene(1, furnace=True)
    for D in (1, 2, 5, 8):
        img, st, _ = oracle.render(s, 16, 12, 2, D, oracle.MODE_NONE)
        assert np.all(img == (1 - 0.5 ** D) / (1 - 0.5))
        assert st["segments"] == 16 * 12 * 2 * D


@pytest.mark.parametrize("mode", [oracle.MODE_PLAIN_RR, oracle.MODE_HEUR_NORM, oracle.MODE_NET])
def test_furnace_unbiased_with_rrs(mode):
    """With Russian roulette / splitting the furnace stays unbiased: the image mean
    over independent frames is within 3 standard errors of the closed form."""
    s = I.box_scene(1, furnace=True)
    P = I.rrsnet_init_params(1).astype(np.float64)
    means = []
    ref = None
    for frame in range(12):
        img, st, _ = oracle.render(s, 16, 16, 4, 8, mode, frame=frame, params=P, pixel_ref=ref)
        means.append(img.mean())
        ref = img if mode == oracle.MODE_HEUR_NORM else None
    m = np.mean(means)
    se = np.std(means, ddof=1) / math.sqrt(len(means))
    assert abs(m - 1.9921875) < 3 * se + 1e-12


def test_rrs_unbiased_against_no_rrs():
    """Normalised RRS (heuristic and network factors) is unbiased: per-frame image
    means agree with the no-RRS estimator within 3 standard errors."""
    s = I.box_scene(2)
    P = I.rrsnet_init_params(2).astype(np.float64)
    res = {}
    for mode in (oracle.MODE_NONE, oracle.MODE_HEUR_NORM, oracle.MODE_NET):
        vals = []
        ref = None
        for frame in range(16):
            img, st, _ = oracle.render(s, 16, 16, 4, 6, mode, frame=frame, params=P,
                                       pixel_ref=ref, cap=16 * 16 * 4)
            vals.append(img.mean())
            if mode == oracle.MODE_HEUR_NORM:
                ref = img if ref is None else (ref * frame + img) / (frame + 1)
        res[mode] = np.array(vals)
    base = res[oracle.MODE_NONE]
    for mode in (oracle.MODE_HEUR_NORM, oracle.MODE_NET):
        v = res[mode]
        se = math.sqrt(v.var(ddof=1) / len(v) + base.var(ddof=1) / len(base))
        assert abs(v.mean() - base.mean()) < 3 * se


def test_direct_view_of_emitter_and_sidedness():
    """A camera below the emitter looking up sees radiance 10 at depth 1 in every
    pixel; from above (the back side of a one-sided emitter) it sees nothing."""
    s = I.box_scene(1, n_random=0)
    cam = s.cam.copy()
    cam["pos"] = (0.5, 0.5, 0.5)
    cam["look"] = (0, 1, 0)
    cam["up"] = (0, 0, 1)
    cam["vfov_deg"] = 10.0
    below = I.Scene(s.tri, s.mat_id, s.mats, cam, "below")
    img, _, _ = oracle.render(below, 8, 8, 2, 1, oracle.MODE_NONE)
    assert np.all(img == 10.0)
    # push the camera above the emitter plane (inside the box, y = 0.9995)
    cam2 = cam.copy()
    cam2["pos"] = (0.5, 0.9995, 0.5)
    cam2["look"] = (0, -1, 0)
    above = I.Scene(s.tri, s.mat_id, s.mats, cam2, "above")
    img, _, _ = oracle.render(above, 8, 8, 2, 1, oracle.MODE_NONE)
    assert np.all(img == 0.0)


def test_pixel_subset_matches_full_render():
    """Without normalisation pixels are independent, so rendering a subset of pixels
    gives exactly the full render's values there (used for full-size sampling)."""
    s = I.box_scene(3)
    full, _, _ = oracle.render(s, 24, 16, 3, 6, oracle.MODE_PLAIN_RR, frame=4)
    pix = np.array([0, 5, 17, 100, 383], dtype=np.int32)
    sub, _, _ = oracle.render(s, 24, 16, 3, 6, oracle.MODE_PLAIN_RR, frame=4, pixels=pix)
    flat_full = full.reshape(-1, 3)
    flat_sub = sub.reshape(-1, 3)
    np.testing.assert_array_equal(flat_sub[pix], flat_full[pix])
    mask = np.ones(24 * 16, bool)
    mask[pix] = False
    assert np.all(flat_sub[mask] == 0)


def test_queue_bookkeeping_and_trace():
    s = I.box_scene(1)
    img, st, tr = oracle.render(s, 16, 16, 4, 8, oracle.MODE_HEUR_NORM, frame=0, trace=True)
    C = 2 * 16 * 16 * 4
    for d in range(7):
        X = tr[d][:, 4].astype(np.int64)
        assert X.sum() == st["requested"][d]
        assert st["live"][d + 1] == min(st["requested"][d], C)
        assert len(tr[d]) == st["live"][d]
        # the queue stays pixel-major (sorted by pixel) at every depth
        assert np.all(np.diff(tr[d][:, 0].astype(np.int64)) >= 0)
    assert np.all(tr[7][:, 4] == 0)  # the last depth never continues


def test_adaptive_alpha_backoff():
    """Eq. f_rate_prime: alpha shrinks by (1 - 0.01) after every depth that overflows
    the queue; with f_rate = 1 the expected count equals the capacity, so overflows
    happen often."""
    s = I.box_scene(1)
    ref, _, _ = oracle.render(s, 16, 16, 4, 8, oracle.MODE_NONE)
    img, st, _ = oracle.render(s, 16, 16, 4, 12, oracle.MODE_HEUR_NORM, frame=1, pixel_ref=ref,
                               f_rate=1.0, cap=16 * 16 * 4)
    eps = paper_constant("alpha_epsilon")
    alpha = 1.0
    assert st["dropped"].sum() > 0
    for d in range(12):
        assert st["alpha"][d] == alpha
        if st["dropped"][d] > 0:
            alpha *= 1 - eps
    # the realised count never exceeds the capacity
    assert np.all(st["live"] <= 16 * 16 * 4)


def test_downscale_only_normalisation():
    """Sec. 4 "Compromise": F >= 1 is never applied (q is only scaled down)."""
    s = I.box_scene(1)
    P = 16 * 16 * 4
    img, st, _ = oracle.render(s, 16, 16, 4, 8, oracle.MODE_HEUR_NORM, frame=0)
    assert np.all(st["F"] <= 1.0)
    # budget N_px = P (the primary queue): F = min(1, 0.85 P / sum q) at every depth; the
    # first frame has q = lum(t) <= 1, so only the first depths can exceed 0.85 P
    sq = st["sum_q"]
    expect = np.where(sq > 0, np.minimum(1.0, 0.85 * P / np.where(sq > 0, sq, 1.0)), 1.0)
    np.testing.assert_array_equal(st["F"], expect.astype(np.float32))
    assert st["F"][0] < 1.0 and st["F"][-1] == 1.0
    # budget 2 P: the queue never asks for more than 0.85 x 2 P, so no depth is rescaled
    _, st2, _ = oracle.render(s, 16, 16, 4, 8, oracle.MODE_HEUR_NORM, frame=0, budget=2 * P)
    assert np.all(st2["F"] == 1.0)


def test_nonfinite_network_factors_fall_back_to_the_heuristic():
    """A network whose factors come out non-finite degrades to plain heuristic normalised
    RRS: the NET render equals the HEUR_NORM render exactly, with every network
    evaluation counted as non-finite."""
    s = I.box_scene(1)
    P = I.rrsnet_init_params(1).astype(np.float64)
    P[2560:] = np.inf
    ref = np.full((8 * 8, 3), 0.3) * np.linspace(0.5, 1.5, 64)[:, None]
    net, st, _ = oracle.render(s, 8, 8, 2, 5, oracle.MODE_NET, params=P, pixel_ref=ref)
    heur, sth, _ = oracle.render(s, 8, 8, 2, 5, oracle.MODE_HEUR_NORM, pixel_ref=ref)
    np.testing.assert_array_equal(net, heur)
    np.testing.assert_array_equal(st["live"], sth["live"])
    # every vertex that was not a miss, black or at the last depth asked the network
    assert st["nonfinite"] > 0 and sth["nonfinite"] == 0
    assert st["nonfinite"] <= st["live"][:4].sum()


def test_forced_F_subset_equals_whole_frame():
    """The sampled-pixel hook: a pixel subset rendered with the whole frame's per-depth
    normalisation factors reproduces those pixels of the whole-frame render exactly
    (pixels interact only through F; the random numbers are keyed per path)."""
    s = I.box_scene(2)
    P = (I.rrsnet_init_params(3) * 3.0).astype(np.float64)
    img, st, _ = oracle.render(s, 24, 16, 2, 6, oracle.MODE_NET, params=P)
    assert np.any(st["F"] < 1.0)
    pix = np.array([0, 5, 77, 200, 383], dtype=np.int32)
    sub, _, _ = oracle.render(s, 24, 16, 2, 6, oracle.MODE_NET, params=P, pixels=pix,
                              forced_F=st["F"])
    np.testing.assert_array_equal(sub.reshape(-1, 3)[pix], img.reshape(-1, 3)[pix])
    with pytest.raises(RuntimeError):
        oracle.render(s, 24, 16, 2, 6, oracle.MODE_NET, params=P, pixels=pix)


def _statnet_params(seed):
    """StatNet weights with a non-negative output layer (positive predicted radiance)."""
    n = oracle.mlpn_param_count(6)
    rng = np.random.default_rng(seed)
    P = rng.normal(size=n) * 0.3
    P[n - 6 * 32:] = np.abs(P[n - 6 * 32:])
    return P


def _adrrs_gate(D, adrrs_depths):
    g = 0
    for d in range(D):
        g |= (oracle.GATE_ADRRS if d in adrrs_depths else oracle.GATE_FIXED) << (2 * d)
    return g


def test_adrrs_without_reference_is_the_heuristic():
    """ADRRS (NN) compares a path's expected contribution with the pixel estimate; before
    any estimate exists it is the throughput heuristic, so an all-ADRRS Mix-Depth render
    equals the HEUR_NORM render exactly."""
    s = I.box_scene(2)
    D = 6
    gate = _adrrs_gate(D, range(D))
    a, sa, _ = oracle.render(s, 16, 12, 2, D, oracle.MODE_NET_MIX, gate=gate,
                             stat_params=_statnet_params(1))
    b, sb, _ = oracle.render(s, 16, 12, 2, D, oracle.MODE_HEUR_NORM)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(sa["live"], sb["live"])


def test_adrrs_factor_scales_with_statnet_output():
    """q_ADRRS is linear in StatNet's predicted mean outside ADRRS's weight window:
    doubling the output layer doubles every such depth-1 factor exactly (powers of two);
    inside the window the factor is 1."""
    s = I.box_scene(3)
    D = 4
    ref = np.ones((16 * 12, 3)) * np.logspace(-3, 1, 16 * 12)[:, None]  # r across the window
    P = _statnet_params(2)
    P2 = P.copy()
    n = P.size
    P2[n - 6 * 32:] *= 2.0
    gate = _adrrs_gate(D, range(D))
    qs = []
    for params in (P, P2):
        _, st, _ = oracle.render(s, 16, 12, 2, D, oracle.MODE_NET_MIX, gate=gate, q_max=1e9,
                                 stat_params=params, pixel_ref=ref, record=True)
        qs.append(st["rec"][0][:, 9])  # q_orig of the depth-1 vertices
    q1, q2 = qs
    # outside the weight window [1/3, 5/3] and above the floor in both renders
    free = (q1 > 0.05) & ((q1 < 1 / 6) | (q1 > 5 / 3))
    assert free.sum() > 20
    np.testing.assert_array_equal(q2[free], 2.0 * q1[free])
    # no factor falls strictly inside the window except the window's own 1
    hits = 0
    for q in (q1, q2):
        inwin = (q >= 1 / 3) & (q <= 5 / 3)
        assert np.all(q[inwin] == 1.0)
        hits += int(inwin.sum())
    assert hits > 0


def test_adrrs_is_unbiased_against_no_rrs():
    """Mix-Depth with ADRRS (NN) depths stays unbiased (every factor is positive): frame
    means agree with the no-RRS estimator within 3 standard errors."""
    s = I.box_scene(2)
    D = 6
    gate = _adrrs_gate(D, {1, 2, 3, 4})
    SP = _statnet_params(3)
    ref = np.full((16 * 16, 3), 0.25)
    vals = {0: [], 1: []}
    for frame in range(16):
        a, _, _ = oracle.render(s, 16, 16, 4, D, oracle.MODE_NONE, frame=frame)
        b, _, _ = oracle.render(s, 16, 16, 4, D, oracle.MODE_NET_MIX, frame=frame, gate=gate,
                                stat_params=SP, pixel_ref=ref)
        vals[0].append(a.mean())
        vals[1].append(b.mean())
    x, y = np.array(vals[0]), np.array(vals[1])
    se = math.sqrt(x.var(ddof=1) / len(x) + y.var(ddof=1) / len(y))
    assert abs(x.mean() - y.mean()) < 3 * se
