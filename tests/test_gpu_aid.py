"""AID-NRRS on the GPU (Sec. 4 "Input Encoding"): RRSNet reads its own hash grid of the
position, one-blob direction and roughness, Box-Cox throughput and pixel estimate.
Renders are compared with the FP64 oracle on decision-matched pixels; training moves the
grid; the mode's limits fail loudly."""
import numpy as np
import pytest

import oracle
from paper_2510_07868_b300 import inputs as I
from test_gpu_render import pixel_hashes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def nrrs():
    from paper_2510_07868_b300 import nrrs as m

    assert torch.cuda.is_available()
    return m


def _aid_scene(nrrs, s, seed):
    sc = nrrs.Scene(s)
    sc.set_rrsnet_inputs(2)
    rng = np.random.default_rng(seed)
    P = (rng.normal(size=nrrs.AID_RRSNET_PARAMS) * 0.3).astype(np.float32)
    G = (rng.normal(size=nrrs.GRID_PARAMS) * 0.3).astype(np.float32)
    sc.set_params(P)
    nrrs.nrrs_set_params(sc.handle, nrrs.NET_RRSNET_GRID, G)
    return sc, P, G


def _render_traced(nrrs, sc, W, H, spp, D, mode, ref, **kw):
    C = 2 * W * H * spp
    tr = torch.zeros((D, C, 5), dtype=torch.int32, device="cuda")
    dref = torch.from_numpy(ref.astype(np.float32)).cuda()
    img, st = sc.render(W, H, spp, D, mode, d_trace=tr.data_ptr(), d_pixel_ref=dref.data_ptr(),
                        **kw)
    torch.cuda.synchronize()
    trn = tr.cpu().numpy().view(np.uint32)
    return img.cpu().numpy().astype(np.float64), st, [trn[d, :st["live"][d]] for d in range(D)]


def _matched(gimg, gtr, oimg, otr, W, H, min_match):
    """Decision-matched pixels; the grid's FP32 positions (scaled by up to 2048) put ~1e-4
    relative error on the factors, which the path weights t / q inherit."""
    hg, cg = pixel_hashes(gtr, W * H)
    ho, co = pixel_hashes(otr, W * H)
    match = (hg == ho) & (cg == co)
    assert match.mean() >= min_match, match.mean()
    g, o = gimg.reshape(-1, 3)[match], oimg.reshape(-1, 3)[match]
    rel = np.max(np.abs(g - o) / np.maximum(np.abs(o), 1e-30), axis=1)
    rel[np.all(o == 0, axis=1) & np.all(g == 0, axis=1)] = 0.0
    assert rel.max() <= 2e-3, rel.max()
    return match.mean()


@pytest.mark.parametrize("scene_name", ["box", "ggx"])
def test_aid_parity(nrrs, scene_name):
    s = I.box_scene(3) if scene_name == "box" else I.icosphere_room(4, min_triangles=3000,
                                                                      subdiv=2)
    sc, P, G = _aid_scene(nrrs, s, 21)
    W = H = 40 if scene_name == "box" else 32
    D = 8 if scene_name == "box" else 6
    ref = (np.full((H * W, 3), 0.3) * np.linspace(0.2, 2.0, H * W)[:, None]).astype(np.float32)
    gimg, gst, gtr = _render_traced(nrrs, sc, W, H, 4, D, nrrs.RRS_NET, ref)
    assert gst["net_evals"] > 0 and gst["nonfinite"] == 0
    oimg, ost, otr = oracle.render(s, W, H, 4, D, oracle.MODE_NET, params=P.astype(np.float64),
                                   rrsnet_inputs=2, rrs_grid=G.astype(np.float64),
                                   pixel_ref=ref.astype(np.float64), trace=True)
    np.testing.assert_allclose(gst["sum_q"][0], ost["sum_q"][0], rtol=1e-4)
    _matched(gimg, gtr, oimg, otr, W, H, 0.95)
    sc.close()


def test_aid_net_mix_parity(nrrs):
    s = I.occluded_room(2, n_random=300)
    sc, P, G = _aid_scene(nrrs, s, 22)
    gate = 0
    for d, g in enumerate([2, 0, 1, 0, 2, 0, 0, 1]):
        gate |= g << (2 * d)
    W = H = 40
    ref = np.full((H * W, 3), 0.8, dtype=np.float32)
    gimg, _, gtr = _render_traced(nrrs, sc, W, H, 4, 8, nrrs.RRS_NET_MIX, ref, gate=gate)
    oimg, _, otr = oracle.render(s, W, H, 4, 8, oracle.MODE_NET_MIX, params=P.astype(np.float64),
                                 rrsnet_inputs=2, rrs_grid=G.astype(np.float64), gate=gate,
                                 pixel_ref=ref.astype(np.float64), trace=True)
    _matched(gimg, gtr, oimg, otr, W, H, 0.95)
    sc.close()


def test_aid_training_moves_the_grid(nrrs):
    s = I.occluded_room(1, n_random=500)
    sc = nrrs.Scene(s)
    sc.set_rrsnet_inputs(2)
    assert nrrs.nrrs_get_rrsnet_params(sc.handle, n=nrrs.AID_RRSNET_PARAMS).size == 3104
    G0 = nrrs.nrrs_get_params(sc.handle, nrrs.NET_RRSNET_GRID_TRAIN)
    for _ in range(3):
        sc.render(64, 64, 4, 8, nrrs.RRS_HEUR_NORM)
    for k in range(40):
        st = sc.train_step(width=64, height=64, spp=2, max_depth=8, warmup_steps=20, frame=k)
        assert np.isfinite(st["loss_rrsnet"]) and not st["fallback"]
    assert st["phase"] == 2
    G1 = nrrs.nrrs_get_params(sc.handle, nrrs.NET_RRSNET_GRID_TRAIN)
    Gr = nrrs.nrrs_get_params(sc.handle, nrrs.NET_RRSNET_GRID)
    assert np.count_nonzero(G1 != G0) > 1000
    assert np.count_nonzero(Gr != G0) > 1000  # the rendering grid follows by EMA
    img, st = sc.render(64, 64, 4, 8, nrrs.RRS_NET, update_ref=0, graph=1)
    assert torch.isfinite(img).all() and st["net_evals"] > 0
    img2, _ = sc.render(64, 64, 4, 8, nrrs.RRS_NET, update_ref=0, graph=0)
    assert torch.equal(img, img2)
    # the mode's limits fail loudly
    with pytest.raises(nrrs.NrrsError):
        sc.render(64, 64, 4, 8, nrrs.RRS_NET, precision=16)
    with pytest.raises(nrrs.NrrsError):
        sc.query(torch.zeros((64, 16), device="cuda"))
    sc.set_rrsnet_inputs(0)  # back to 16 inputs: a fresh network of that shape
    assert nrrs.nrrs_get_rrsnet_params(sc.handle).size == 2592
    with pytest.raises(nrrs.NrrsError):
        nrrs.nrrs_get_params(sc.handle, nrrs.NET_RRSNET_GRID)
    sc.close()
