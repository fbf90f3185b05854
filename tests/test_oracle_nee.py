"""Next-event estimation in the FP64 oracle (CPU).

The paper's experiments run with next-event estimation on (Sec. 5).  The oracle's
version (one emitter point per vertex, chosen by area; power-heuristic MIS against
emitters found by BSDF sampling) is pinned by what holds whatever the implementation:

* direct light at a point under a rectangular emitter has a closed form (the form factor
  of a differential area to a parallel rectangle with the normal through a corner), which
  the test also checks by quadrature;
* with and without NEE the estimator is unbiased, so the two agree in expectation on
  glossy scenes and in the furnace (closed form Le (1 - a^D) / (1 - a));
* at depth limit 1 nothing but the camera ray's emission counts, with or without NEE;
* normalised RRS stays unbiased with NEE on.
"""
import numpy as np
import pytest

import oracle
from paper_2510_07868_b300 import inputs as I


def _corner_form_factor(X, Y):
    """Form factor from a differential area to a parallel X x Y rectangle (sizes over the
    height) whose corner lies on the area's normal."""
    sx, sy = np.sqrt(1 + X * X), np.sqrt(1 + Y * Y)
    return (X / sx * np.arctan(Y / sx) + Y / sy * np.arctan(X / sy)) / (2 * np.pi)


def _frame_values(scene, W, H, spp, D, mode, frames, nee, **kw):
    """Mean image value of each of `frames` independent frames."""
    out = []
    for f in range(frames):
        img, _, _ = oracle.render(scene, W, H, spp, D, mode, frame=f, nee=nee, **kw)
        out.append(img.mean())
    return np.array(out)


def _agree(a, b, k=4.0):
    se = np.sqrt(a.var(ddof=1) / a.size + b.var(ddof=1) / b.size)
    return abs(a.mean() - b.mean()) <= k * se, a.mean(), b.mean(), se


def test_corner_form_factor_by_quadrature():
    a, b, c = 0.6, 0.4, 0.5
    n = 800
    x = (np.arange(n) + 0.5) / n * a
    z = (np.arange(n) + 0.5) / n * b
    X, Z = np.meshgrid(x, z)
    r2 = X * X + Z * Z + c * c
    quad = np.sum(c * c / (np.pi * r2 * r2)) * (a / n) * (b / n)
    assert abs(_corner_form_factor(a / c, b / c) - quad) < 1e-6


@pytest.mark.parametrize("nee", [1, 0])
def test_direct_light_under_rectangle_closed_form(nee):
    """Radiance reflected by a Lambertian point: albedo x Le x form factor.  Depth limit 2:
    the floor vertex and the emitter hit (MIS-weighted when NEE is on).  The emitter is
    three triangles of unequal area, so a choice not by area would be biased."""
    a, b, c, Le, rho = 0.6, 0.4, 0.5, 10.0, 0.5
    s = I.lit_floor(a, b, c, Le, rho)
    expected = rho * Le * _corner_form_factor(a / c, b / c)
    v = np.array([oracle.render(s, 1, 1, 4096, 2, oracle.MODE_NONE, frame=f, nee=nee)[0][0, 0, 0]
                  for f in range(16)])
    se = v.std(ddof=1) / np.sqrt(v.size)
    assert abs(v.mean() - expected) <= 4 * se, (v.mean(), expected, se)
    if nee:  # one emitter sample per vertex already pins it to 0.5 %
        assert abs(v.mean() / expected - 1) < 5e-3


def test_nee_and_bsdf_sampling_agree_on_glossy_floor():
    """A GGX floor (roughness 0.2) under the same emitter: no closed form, but the two
    estimators must agree; the MIS weights of both sides enter."""
    s = I.lit_floor(floor_type=I.MAT_GGX, roughness=0.2)
    on = np.array([oracle.render(s, 1, 1, 4096, 2, oracle.MODE_NONE, frame=f, nee=1)[0][0, 0, 0]
                   for f in range(16)])
    off = np.array([oracle.render(s, 1, 1, 4096, 2, oracle.MODE_NONE, frame=f, nee=0)[0][0, 0, 0]
                    for f in range(16)])
    ok, m_on, m_off, se = _agree(on, off)
    assert ok, (m_on, m_off, se)
    assert on.std() < off.std()  # NEE's point: less noise per sample


def test_nee_and_bsdf_sampling_agree_in_glossy_room():
    s = I.icosphere_room(2, min_triangles=1500, subdiv=2)
    on = _frame_values(s, 16, 16, 4, 4, oracle.MODE_NONE, 24, 1)
    off = _frame_values(s, 16, 16, 4, 4, oracle.MODE_NONE, 24, 0)
    ok, m_on, m_off, se = _agree(on, off)
    assert ok, (m_on, m_off, se)


def test_furnace_closed_form_with_nee():
    """Every surface emits 1 and reflects 0.5: the expected pixel value is
    Le (1 - a^D) / (1 - a) = 1.9921875 at D = 8, with NEE as without."""
    s = I.box_scene(3, furnace=True)
    v = _frame_values(s, 8, 8, 4, 8, oracle.MODE_NONE, 16, 1)
    se = v.std(ddof=1) / np.sqrt(v.size)
    assert abs(v.mean() - 1.9921875) <= 4 * se + 1e-12, (v.mean(), se)


def test_depth_one_is_unchanged_by_nee():
    s = I.box_scene(1)
    a, _, _ = oracle.render(s, 16, 16, 2, 1, oracle.MODE_NONE, nee=0)
    b, _, _ = oracle.render(s, 16, 16, 2, 1, oracle.MODE_NONE, nee=1)
    assert np.array_equal(a, b)


def test_normalized_rrs_with_nee_is_unbiased():
    """Plain normalised RRS (heuristic factors, Eq. F_norm) against no RRS, NEE on: both
    estimate the same image."""
    s = I.box_scene(2)
    ref = oracle.render(s, 16, 16, 16, 6, oracle.MODE_NONE, nee=1, frame=99)[0]
    heur = _frame_values(s, 16, 16, 4, 6, oracle.MODE_HEUR_NORM, 24, 1, pixel_ref=ref)
    none = _frame_values(s, 16, 16, 4, 6, oracle.MODE_NONE, 24, 1)
    ok, m_h, m_n, se = _agree(heur, none)
    assert ok, (m_h, m_n, se)
