"""RRSNet on the NRRS inputs of Sec. 4 "Input Encoding" (GPU): StatNet's statistics,
the throughput, the pixel estimate and the remapped roughness, Box-Cox encoded.  Renders
are compared with the FP64 oracle on its decision records as the other render tests are;
training steps and graph capture run with the encoding."""
import numpy as np
import pytest

import oracle
from paper_2510_07868_b300 import inputs as I
from test_gpu_render import compare, pixel_hashes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def nrrs():
    from paper_2510_07868_b300 import nrrs as m

    assert torch.cuda.is_available()
    return m


def _statnet(nrrs, seed):
    SP = np.random.default_rng(seed).normal(size=nrrs.STATNET_PARAMS).astype(np.float32) * 0.3
    SP[-6 * 32:] = np.abs(SP[-6 * 32:])  # mostly positive statistics
    return SP


def _render(nrrs, s, W, H, spp, D, mode, P, SP, ref, **kw):
    sc = nrrs.Scene(s)
    sc.set_params(P)
    nrrs.nrrs_set_params(sc.handle, nrrs.NET_STATNET, SP)
    sc.set_rrsnet_inputs(1)
    C = 2 * W * H * spp
    tr = torch.zeros((D, C, 5), dtype=torch.int32, device="cuda")
    dref = torch.from_numpy(ref.astype(np.float32)).cuda() if ref is not None else None
    img, st = sc.render(W, H, spp, D, mode, d_trace=tr.data_ptr(),
                        d_pixel_ref=dref.data_ptr() if dref is not None else None, **kw)
    torch.cuda.synchronize()
    trn = tr.cpu().numpy().view(np.uint32)
    sc.close()
    return img.cpu().numpy().astype(np.float64), st, [trn[d, :st["live"][d]] for d in range(D)]


@pytest.mark.parametrize("scene_name", ["box", "ggx"])
def test_nrrs_inputs_parity(nrrs, scene_name):
    s = I.box_scene(3) if scene_name == "box" else I.icosphere_room(4, min_triangles=3000,
                                                                      subdiv=2)
    P = I.rrsnet_init_params(2)
    SP = _statnet(nrrs, 11)
    W = H = 40
    ref = (np.full((H * W, 3), 0.3) * np.linspace(0.2, 2.0, H * W)[:, None])
    gimg, gst, gtr = _render(nrrs, s, W, H, 4, 6, nrrs.RRS_NET, P, SP, ref)
    assert gst["net_evals"] > 0 and gst["nonfinite"] == 0
    oimg, ost, otr = oracle.render(s, W, H, 4, 6, oracle.MODE_NET, params=P.astype(np.float64),
                                   stat_params=SP.astype(np.float64), rrsnet_inputs=1,
                                   pixel_ref=ref.astype(np.float32).astype(np.float64), trace=True)
    # depth 1: the same vertices on both sides, so the sums of the factors agree closely
    np.testing.assert_allclose(gst["sum_q"][0], ost["sum_q"][0], rtol=1e-6)
    if scene_name == "box":
        compare(gimg, gtr, oimg, otr, W, H, min_match=0.98)
    else:  # GGX directions: the bar of the GGX render test (99 % of matched pixels)
        hg, cg = pixel_hashes(gtr, W * H)
        ho, co = pixel_hashes(otr, W * H)
        match = (hg == ho) & (cg == co)
        assert match.mean() >= 0.98
        g, o = gimg.reshape(-1, 3)[match], oimg.reshape(-1, 3)[match]
        rel = np.max(np.abs(g - o) / np.maximum(np.abs(o), 1e-30), axis=1)
        rel[np.all(o == 0, axis=1) & np.all(g == 0, axis=1)] = 0.0
        assert np.mean(rel <= 1e-5) >= 0.99


def test_nrrs_inputs_net_mix_parity(nrrs):
    s = I.occluded_room(2, n_random=300)
    P = I.rrsnet_init_params(3)
    SP = _statnet(nrrs, 12)
    gate = 0
    for d, g in enumerate([2, 0, 1, 0, 2, 0, 0, 1]):
        gate |= g << (2 * d)
    W = H = 40
    ref = np.full((H * W, 3), 0.8)
    gimg, _, gtr = _render(nrrs, s, W, H, 4, 8, nrrs.RRS_NET_MIX, P, SP, ref, gate=gate)
    oimg, _, otr = oracle.render(s, W, H, 4, 8, oracle.MODE_NET_MIX, params=P.astype(np.float64),
                                 stat_params=SP.astype(np.float64), rrsnet_inputs=1, gate=gate,
                                 pixel_ref=ref, trace=True)
    compare(gimg, gtr, oimg, otr, W, H, min_match=0.98)


@pytest.mark.parametrize("precision", [16, 8])
def test_nrrs_inputs_tensor_core_precisions(nrrs, precision):
    """The tensor-core kernels on the encoded inputs: factors within the precision's
    error of FP32 (same decisions for nearly every path)."""
    s = I.occluded_room(1, n_random=500)
    P = I.rrsnet_init_params(1)
    SP = _statnet(nrrs, 13)
    W = H = 64
    ref = np.full((H * W, 3), 0.5)
    g32, st32, tr32 = _render(nrrs, s, W, H, 4, 8, nrrs.RRS_NET, P, SP, ref, precision=32)
    gp, stp, trp = _render(nrrs, s, W, H, 4, 8, nrrs.RRS_NET, P, SP, ref, precision=precision)
    assert stp["status_bits"] == 0 and np.isfinite(gp).all()
    h32, c32 = pixel_hashes(tr32, W * H)
    hp, cp = pixel_hashes(trp, W * H)
    same = np.mean((h32 == hp) & (c32 == cp))
    assert same >= (0.97 if precision == 16 else 0.6), same


def test_nrrs_inputs_training_and_graph(nrrs):
    """Training steps on the encoded inputs stay finite; graph-captured renders equal
    stream-launched ones."""
    s = I.occluded_room(1, n_random=500)
    sc = nrrs.Scene(s)
    sc.set_params(I.rrsnet_init_params(1))
    sc.set_rrsnet_inputs(1)
    for _ in range(3):
        sc.render(64, 64, 4, 8, nrrs.RRS_HEUR_NORM)
    for k in range(30):
        st = sc.train_step(width=64, height=64, spp=2, max_depth=8, warmup_steps=10, frame=k)
        assert np.isfinite(st["loss_statnet"]) and np.isfinite(st["loss_rrsnet"])
    assert st["phase"] == 2 and not st["fallback"]
    outs = []
    for g in (0, 1, 1):
        img, _ = sc.render(64, 64, 4, 8, nrrs.RRS_NET, frame=5, update_ref=0, graph=g)
        outs.append(img.clone())
    assert torch.isfinite(outs[0]).all()
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])
    with pytest.raises(nrrs.NrrsError):
        sc.set_rrsnet_inputs(3)  # 0, 1 (NRRS inputs) and 2 (AID-NRRS) exist
    sc.close()
