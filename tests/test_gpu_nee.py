"""Next-event estimation on the GPU against the FP64 oracle (GPU).

With NEE on, every vertex that goes on samples one emitter point and traces a shadow
ray; a pixel's value then also depends on that shadow test, which FP32 and FP64 can
decide differently for points near an occluder's silhouette.  So besides the decision
records (triangle and split count per path, compared as in the other render tests), the
bar is: decision-matched pixels within 1e-5 relative for at least 99 % of them, and
the image means, over many frames, equal to the closed form where one exists."""
import numpy as np
import pytest

import oracle
from paper_2510_07868_b300 import inputs as I
from test_gpu_render import RTOL, gpu_render, pixel_hashes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def nrrs():
    from paper_2510_07868_b300 import nrrs as m

    assert torch.cuda.is_available()
    return m


def _corner_form_factor(X, Y):
    sx, sy = np.sqrt(1 + X * X), np.sqrt(1 + Y * Y)
    return (X / sx * np.arctan(Y / sx) + Y / sy * np.arctan(X / sy)) / (2 * np.pi)


def _compare_nee(gimg, gtr, oimg, otr, W, H, min_match=0.98, min_close=0.99):
    hg, cg = pixel_hashes(gtr, W * H)
    ho, co = pixel_hashes(otr, W * H)
    match = (hg == ho) & (cg == co)
    assert match.mean() >= min_match, match.mean()
    g = gimg.reshape(-1, 3)[match]
    o = oimg.reshape(-1, 3)[match]
    rel = np.max(np.abs(g - o) / np.maximum(np.abs(o), 1e-30), axis=1)
    rel[np.all(o == 0, axis=1) & np.all(g == 0, axis=1)] = 0.0
    close = np.mean(rel <= RTOL)
    assert close >= min_close, (close, np.sort(rel)[-5:])
    return match.mean(), close


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_nee_box_scene_parity(nrrs, mode):
    s = I.box_scene(1)
    P = I.rrsnet_init_params(1)
    W = H = 48
    gimg, gst, gtr = gpu_render(nrrs, s, W, H, 4, 8, mode, params=P, nee=1)
    oimg, ost, otr = oracle.render(s, W, H, 4, 8, mode, params=P.astype(np.float64), trace=True,
                                   nee=1)
    m, c = _compare_nee(gimg, gtr, oimg, otr, W, H)
    np.testing.assert_allclose(gst["F"], ost["F"], rtol=1e-5)
    # NEE changes the deposits only: the factors, and so the decisions and the traced
    # records, are the NEE-off render's
    _, _, gtr0 = gpu_render(nrrs, s, W, H, 4, 8, mode, params=P, nee=0)
    for d in range(8):
        np.testing.assert_array_equal(gtr[d], gtr0[d])


@pytest.mark.parametrize("mode", [0, 2])
def test_nee_ggx_scene_parity(nrrs, mode):
    s = I.icosphere_room(4, min_triangles=3000, subdiv=2)
    W = H = 40
    gimg, _, gtr = gpu_render(nrrs, s, W, H, 4, 6, mode, nee=1)
    oimg, _, otr = oracle.render(s, W, H, 4, 6, mode, trace=True, nee=1)
    _compare_nee(gimg, gtr, oimg, otr, W, H)


def test_nee_net_mix_parity(nrrs):
    s = I.occluded_room(2, n_random=300)
    P = I.rrsnet_init_params(2)
    gate = 0
    for d, g in enumerate([2, 0, 1, 0, 2, 1, 0, 0]):
        gate |= g << (2 * d)
    W = H = 40
    gimg, _, gtr = gpu_render(nrrs, s, W, H, 4, 8, nrrs.RRS_NET_MIX, params=P, gate=gate, nee=1)
    oimg, _, otr = oracle.render(s, W, H, 4, 8, oracle.MODE_NET_MIX, params=P.astype(np.float64),
                                 gate=gate, trace=True, nee=1)
    _compare_nee(gimg, gtr, oimg, otr, W, H)


@pytest.mark.parametrize("floor_type", [0, 1])
def test_nee_direct_light_closed_form(nrrs, floor_type):
    """The pencil camera's point under a rectangular emitter: the Lambertian floor
    reflects albedo x Le x form factor; the GGX floor has no closed form but NEE and
    BSDF sampling must agree."""
    a, b, c, Le, rho = 0.6, 0.4, 0.5, 10.0, 0.5
    s = I.lit_floor(a, b, c, Le, rho, floor_type=floor_type)
    sc = nrrs.Scene(s)
    vals = {0: [], 1: []}
    for nee in (0, 1):
        for f in range(16):
            img, _ = sc.render(1, 1, 65536, 2, nrrs.RRS_NONE, frame=f, nee=nee, stats=False)
            vals[nee].append(float(img[0, 0, 0]))
    sc.close()
    on, off = np.array(vals[1]), np.array(vals[0])
    se = np.sqrt(on.var(ddof=1) / on.size + off.var(ddof=1) / off.size)
    assert abs(on.mean() - off.mean()) <= 4 * se, (on.mean(), off.mean(), se)
    if floor_type == 0:
        expected = rho * Le * _corner_form_factor(a / c, b / c)
        se_on = on.std(ddof=1) / np.sqrt(on.size)
        assert abs(on.mean() - expected) <= 4 * se_on + 1e-6 * expected, (on.mean(), expected)
        assert abs(on.mean() / expected - 1) < 2e-3


def test_nee_normalized_rrs_unbiased(nrrs):
    """Normalised heuristic RRS against no RRS with NEE on (GPU): same image mean."""
    s = I.occluded_room(3, n_random=400)
    sc = nrrs.Scene(s)
    W = H = 64
    ref, _ = sc.render(W, H, 64, 8, nrrs.RRS_NONE, frame=500, nee=1, update_ref=0)
    ref = ref.clone()
    means = {nrrs.RRS_NONE: [], nrrs.RRS_HEUR_NORM: []}
    for m in means:
        for f in range(24):
            img, _ = sc.render(W, H, 4, 8, m, frame=f, nee=1, update_ref=0,
                               d_pixel_ref=ref.data_ptr())
            means[m].append(float(img.double().mean()))
    sc.close()
    a, b = np.array(means[nrrs.RRS_NONE]), np.array(means[nrrs.RRS_HEUR_NORM])
    se = np.sqrt(a.var(ddof=1) / a.size + b.var(ddof=1) / b.size)
    assert abs(a.mean() - b.mean()) <= 4 * se, (a.mean(), b.mean(), se)


def test_nee_graph_captured_is_bit_identical(nrrs):
    s = I.occluded_room(1, n_random=500)
    P = I.rrsnet_init_params(3)
    sc = nrrs.Scene(s)
    sc.set_params(P)
    outs = []
    for g in (0, 1, 1):
        img, st = sc.render(64, 64, 4, 10, nrrs.RRS_NET, frame=2, update_ref=0, graph=g, nee=1)
        outs.append((img.clone(), st))
    sc.close()
    for img, st in outs[1:]:
        assert torch.equal(img, outs[0][0])
        np.testing.assert_array_equal(st["live"], outs[0][1]["live"])


def test_nee_batch_jobs_equal_single_renders(nrrs):
    jobs = [(I.box_scene(1), 24, 16, 3, 6),
            (I.occluded_room(2, n_random=200), 16, 16, 2, 8),
            (I.icosphere_room(3, min_triangles=1500, subdiv=2), 20, 12, 4, 5)]
    P = (I.rrsnet_init_params(2) * 2.0).astype(np.float32)
    b = nrrs.Batch(jobs)
    b.set_params(P)
    kw = dict(frame=3, update_ref=0, nee=1)
    imgs, st, live, F, sq = b.render(nrrs.RRS_NET, **kw)
    torch.cuda.synchronize()
    for j, (scene, W, H, spp, D) in enumerate(jobs):
        sc = nrrs.Scene(scene)
        sc.set_params(P)
        ref, rst = sc.render(W, H, spp, D, nrrs.RRS_NET, **kw)
        torch.cuda.synchronize()
        if np.array_equal(F[j, :D], rst["F"][:D]):
            assert torch.equal(imgs[j], ref), j
        sc.close()
        oimg, _, _ = oracle.render(scene, W, H, spp, D, oracle.MODE_NET, frame=3,
                                   params=P.astype(np.float64), nee=1)
        g = imgs[j].cpu().numpy().astype(np.float64)
        close = np.all(np.abs(g - oimg) <= RTOL * np.abs(oimg) + 1e-30, axis=2)
        assert close.mean() >= 0.95, (j, close.mean())
    b.close()


def test_nee_full_size_occluded_room_sampled_pixels(nrrs):
    """The bench scene at full size (256 x 256 x 16 spp, depth 16) with NEE: sampled
    pixels rendered one by one by the oracle."""
    s = I.occluded_room(1)
    W = H = 256
    spp, D = 16, 16
    for mode in (nrrs.RRS_NONE, nrrs.RRS_PLAIN_RR):
        gimg, gst, _ = gpu_render(nrrs, s, W, H, spp, D, mode, trace=False, nee=1)
        assert gst["status_bits"] == 0
        rng = np.random.default_rng(10 + mode)
        pix = np.sort(rng.choice(W * H, 32, replace=False)).astype(np.int32)
        oimg, _, _ = oracle.render(s, W, H, spp, D, mode, pixels=pix, nee=1)
        g = gimg.reshape(-1, 3)[pix]
        o = oimg.reshape(-1, 3)[pix]
        close = np.all(np.abs(g - o) <= RTOL * np.abs(o) + 1e-30, axis=1)
        assert close.mean() >= 0.9, close.mean()


def test_nee_train_step(nrrs):
    """A training step on an NEE frame: finite losses, samples drawn."""
    s = I.occluded_room(1, n_random=500)
    sc = nrrs.Scene(s)
    sc.set_params(I.rrsnet_init_params(1))
    for _ in range(3):
        sc.render(64, 64, 4, 8, nrrs.RRS_HEUR_NORM, nee=1)
    for _ in range(3):
        st = sc.train_step(width=64, height=64, spp=2, max_depth=8, nee=1)
    assert st["samples"] > 0 and np.isfinite(st["loss_statnet"]) and not st["fallback"]
    sc.close()


def test_nee_without_emitters(nrrs):
    """A scene with no emitting triangle: NEE has nothing to sample and the image is 0,
    alone and as a job next to a lit one (each job samples its own emitters)."""
    dark = I.box_scene(2)
    dark.mats["Le"][:] = 0.0
    sc = nrrs.Scene(dark)
    img, st = sc.render(32, 32, 4, 6, nrrs.RRS_HEUR_NORM, nee=1)
    torch.cuda.synchronize()
    assert st["status_bits"] == 0 and float(img.abs().max()) == 0.0
    sc.close()
    b = nrrs.Batch([(dark, 16, 16, 2, 5), (I.box_scene(1), 16, 16, 2, 5)])
    imgs, st, _, _, _ = b.render(nrrs.RRS_HEUR_NORM, nee=1, update_ref=0)
    torch.cuda.synchronize()
    assert float(imgs[0].abs().max()) == 0.0 and float(imgs[1].max()) > 0.0
    b.close()
