"""Parity of whole renders (camera -> D bounces -> accumulation) with the FP64 oracle.

Decisions are compared on integers: per depth and queue slot the traced
(pixel, sample, lineage, triangle, X) records.  Pixels whose decision multiset matches
the oracle's must agree to 1e-5 relative (FP32 path on identical decisions); the
matching fraction must stay near 1 (FP32 and FP64 geometry can differ on near-ties).
"""
import numpy as np
import pytest

import oracle
from paper_2510_07868_b300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

RTOL = 1e-5


@pytest.fixture(scope="module")
def nrrs():
    from paper_2510_07868_b300 import nrrs as m

    assert torch.cuda.is_available()
    return m


def _mix(x):
    x = x.astype(np.uint64)
    with np.errstate(over="ignore"):
        x = (x ^ (x >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        x = (x ^ (x >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        x = x ^ (x >> np.uint64(31))
    return x


def pixel_hashes(trace_per_depth, npix):
    """Order-insensitive per-pixel hash of every (depth, sample, lineage, tri, X) record."""
    h = np.zeros(npix, dtype=np.uint64)
    cnt = np.zeros(npix, dtype=np.int64)
    with np.errstate(over="ignore"):
        for d, tr in enumerate(trace_per_depth):
            if len(tr) == 0:
                continue
            tr = tr.astype(np.uint64)
            v = _mix(tr[:, 1] + np.uint64(d) * np.uint64(1 << 40))
            v = _mix(v ^ tr[:, 2])
            v = _mix(v ^ (tr[:, 3] << np.uint64(8)))
            v = _mix(v ^ tr[:, 4])
            np.add.at(h, tr[:, 0].astype(np.int64), v)
            np.add.at(cnt, tr[:, 0].astype(np.int64), 1)
    return h, cnt


def gpu_render(nrrs, scene, W, H, spp, D, mode, params=None, ref=None, trace=True, **kw):
    sc = nrrs.Scene(scene)
    if params is not None:
        sc.set_params(params)
    C = 2 * W * H * spp
    tr = torch.zeros((D, C, 5), dtype=torch.int32, device="cuda") if trace else None
    dref = torch.from_numpy(ref.astype(np.float32)).cuda() if ref is not None else None
    img, st = sc.render(W, H, spp, D, mode, d_trace=tr.data_ptr() if trace else None,
                        d_pixel_ref=dref.data_ptr() if dref is not None else None, **kw)
    torch.cuda.synchronize()
    out = img.cpu().numpy().astype(np.float64)
    trace_list = None
    if trace:
        trn = tr.cpu().numpy().view(np.uint32)
        trace_list = [trn[d, :st["live"][d]] for d in range(D)]
    sc.close()
    return out, st, trace_list


def compare(gimg, gtr, oimg, otr, W, H, min_match=0.995):
    hg, cg = pixel_hashes(gtr, W * H)
    ho, co = pixel_hashes(otr, W * H)
    match = (hg == ho) & (cg == co)
    frac = match.mean()
    assert frac >= min_match, f"only {frac:.4f} of pixels share every decision"
    g = gimg.reshape(-1, 3)[match]
    o = oimg.reshape(-1, 3)[match]
    err = np.abs(g - o)
    bad = err > RTOL * np.abs(o) + 1e-30
    assert not bad.any(), f"max rel err {np.max(err / np.maximum(np.abs(o), 1e-30)):.3e}"
    return frac


def test_furnace_exact(nrrs):
    """Closed furnace, no RRS: every pixel is exactly (1 - 0.5^8) / (1 - 0.5)."""
    s = I.box_scene(1, furnace=True)
    img, st, _ = gpu_render(nrrs, s, 64, 64, 4, 8, nrrs.RRS_NONE, trace=False)
    exact = np.mean(img == 1.9921875)
    assert exact >= 0.999, exact
    assert np.all(np.abs(img - 1.9921875) <= 1.9921875 * 0.51)
    assert st["segments"] <= 64 * 64 * 4 * 8


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_box_scene_parity(nrrs, mode):
    s = I.box_scene(1)
    P = I.rrsnet_init_params(1)
    W = H = 64
    spp, D = 4, 8
    gimg, gst, gtr = gpu_render(nrrs, s, W, H, spp, D, mode, params=P)
    oimg, ost, otr = oracle.render(s, W, H, spp, D, mode, params=P.astype(np.float64), trace=True)
    # depth-1 queue and decisions are identical slot by slot
    assert gst["live"][0] == ost["live"][0] == W * H * spp
    np.testing.assert_array_equal(gtr[0][:, [0, 1, 2]], otr[0][:, [0, 1, 2]])
    same_tri = gtr[0][:, 3] == otr[0][:, 3]
    assert same_tri.mean() > 0.999
    np.testing.assert_array_equal(gtr[0][same_tri, 4], otr[0][same_tri, 4])
    compare(gimg, gtr, oimg, otr, W, H)
    np.testing.assert_allclose(gst["F"], ost["F"], rtol=1e-6)


def test_heuristic_with_reference_parity(nrrs):
    """Normalised heuristic RRS with a reference image: F < 1 at every depth."""
    s = I.box_scene(2)
    W = H = 48
    spp, D = 4, 8
    ref, _, _ = oracle.render(s, W, H, 4, D, oracle.MODE_NONE, frame=9)
    ref32 = ref.astype(np.float32)
    gimg, gst, gtr = gpu_render(nrrs, s, W, H, spp, D, nrrs.RRS_HEUR_NORM, ref=ref32, frame=1)
    oimg, ost, otr = oracle.render(s, W, H, spp, D, oracle.MODE_HEUR_NORM, frame=1,
                                   pixel_ref=ref32.astype(np.float64), trace=True)
    assert np.all(ost["F"][:-1] < 1)
    np.testing.assert_allclose(gst["sum_q"][:2], ost["sum_q"][:2], rtol=1e-5)
    assert gst["F"][0] == ost["F"][0]
    compare(gimg, gtr, oimg, otr, W, H, min_match=0.98)


def test_net_mix_gate_parity(nrrs):
    s = I.box_scene(3)
    P = I.rrsnet_init_params(2)
    gate = 0
    for d, g in enumerate([2, 0, 1, 0, 2, 1, 0, 0]):
        gate |= g << (2 * d)
    W = H = 40
    gimg, gst, gtr = gpu_render(nrrs, s, W, H, 4, 8, nrrs.RRS_NET_MIX, params=P, gate=gate)
    oimg, ost, otr = oracle.render(s, W, H, 4, 8, oracle.MODE_NET_MIX, params=P.astype(np.float64),
                                   gate=gate, trace=True)
    compare(gimg, gtr, oimg, otr, W, H)


def test_net_mix_with_adrrs_parity(nrrs):
    """Mix-Depth with all four methods, ADRRS (NN) among them (StatNet's predicted
    radiance over the pixel reference): decision-matched pixels equal the oracle's."""
    s = I.box_scene(3)
    P = I.rrsnet_init_params(2)
    SP = np.random.default_rng(7).normal(size=nrrs.STATNET_PARAMS).astype(np.float32) * 0.3
    SP[-6 * 32:] = np.abs(SP[-6 * 32:])
    gate = 0
    for d, g in enumerate([2, 3, 0, 3, 1, 3, 0, 3]):
        gate |= g << (2 * d)
    W = H = 40
    ref = (np.full((H * W, 3), 0.3) * np.linspace(0.4, 1.6, H * W)[:, None]).astype(np.float32)
    sc = nrrs.Scene(s)
    sc.set_params(P)
    nrrs.nrrs_set_params(sc.handle, nrrs.NET_STATNET, SP)
    C = 2 * W * H * 4
    tr = torch.zeros((8, C, 5), dtype=torch.int32, device="cuda")
    dref = torch.from_numpy(ref).cuda()
    img, st = sc.render(W, H, 4, 8, nrrs.RRS_NET_MIX, gate=gate, d_trace=tr.data_ptr(),
                        d_pixel_ref=dref.data_ptr())
    torch.cuda.synchronize()
    trn = tr.cpu().numpy().view(np.uint32)
    gtr = [trn[d, :st["live"][d]] for d in range(8)]
    assert st["net_evals"] > 0 and st["nonfinite"] == 0
    oimg, ost, otr = oracle.render(s, W, H, 4, 8, oracle.MODE_NET_MIX, params=P.astype(np.float64),
                                   gate=gate, stat_params=SP.astype(np.float64),
                                   pixel_ref=ref.astype(np.float64), trace=True)
    compare(img.cpu().numpy().astype(np.float64), gtr, oimg, otr, W, H)
    sc.close()


def test_overflow_and_alpha_backoff(nrrs):
    """Tight capacity with f_rate = 1: drops happen, the queue never exceeds C, alpha
    backs off by 0.99 per overflowing depth (Eq. f_rate_prime), like the oracle."""
    s = I.box_scene(1)
    W = H = 32
    ref, _, _ = oracle.render(s, W, H, 4, 8, oracle.MODE_NONE, frame=3)
    ref32 = ref.astype(np.float32)
    gimg, gst, gtr = gpu_render(nrrs, s, W, H, 4, 10, nrrs.RRS_HEUR_NORM, ref=ref32, f_rate=1.0,
                                cap_factor=1, trace=False)
    C = W * H * 4
    assert np.all(gst["live"] <= C)
    assert gst["dropped"].sum() > 0 and gst["status_bits"] & nrrs.STATUS_OVERFLOW_DROPPED
    alpha = 1.0
    for d in range(10):
        assert gst["alpha"][d] == pytest.approx(alpha, rel=1e-15)
        if gst["dropped"][d] > 0:
            alpha *= 0.99


def test_determinism(nrrs):
    s = I.box_scene(1)
    P = I.rrsnet_init_params(1)
    a, sa, _ = gpu_render(nrrs, s, 64, 64, 4, 8, nrrs.RRS_NET, params=P, trace=False)
    b, sb, _ = gpu_render(nrrs, s, 64, 64, 4, 8, nrrs.RRS_NET, params=P, trace=False)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(sa["live"], sb["live"])


@pytest.mark.parametrize("precision,fuse", [(32, 1), (16, 1), (16, 0), (17, 1), (17, 0),
                                            (8, 1)])
def test_nonfinite_network_falls_back_to_heuristic(nrrs, precision, fuse):
    """Non-finite network factors take the throughput heuristic's factor: with an
    infinite output layer the NET render is the HEUR_NORM render, bit for bit, and every
    network evaluation is reported non-finite (tensor-core precisions with the fused
    shade + RRSNet kernel and with the separate kernels)."""
    s = I.box_scene(1)
    P = I.rrsnet_init_params(1)
    P[2560:] = np.inf
    ref = torch.from_numpy((np.full((16 * 16, 3), 0.3, dtype=np.float32) *
                            np.linspace(0.5, 1.5, 256, dtype=np.float32)[:, None])).cuda()
    sc = nrrs.Scene(s)
    sc.set_params(P)
    sc.set_shade_fusion(fuse)
    kw = dict(d_pixel_ref=ref.data_ptr(), update_ref=0, precision=precision)
    net, st = sc.render(16, 16, 2, 5, nrrs.RRS_NET, **kw)
    heur, sth = sc.render(16, 16, 2, 5, nrrs.RRS_HEUR_NORM, **kw)
    torch.cuda.synchronize()
    assert torch.equal(net, heur)
    np.testing.assert_array_equal(st["live"], sth["live"])
    assert st["nonfinite"] == st["net_evals"] > 0
    assert st["status_bits"] & nrrs.STATUS_NONFINITE and np.all(np.isfinite(net.cpu().numpy()))
    sc.close()


def test_full_size_occluded_room_sampled_pixels(nrrs):
    """256 x 256 x 16 spp, depth 16, the bench workload's scene: without normalisation
    pixels are independent, so the oracle renders sampled pixels one by one."""
    s = I.occluded_room(1)
    W = H = 256
    spp, D = 16, 16
    for mode in (nrrs.RRS_NONE, nrrs.RRS_PLAIN_RR):
        gimg, gst, _ = gpu_render(nrrs, s, W, H, spp, D, mode, trace=False)
        rng = np.random.default_rng(mode)
        pix = np.sort(rng.choice(W * H, 48, replace=False)).astype(np.int32)
        oimg, _, _ = oracle.render(s, W, H, spp, D, mode, pixels=pix)
        g = gimg.reshape(-1, 3)[pix]
        o = oimg.reshape(-1, 3)[pix]
        close = np.all(np.abs(g - o) <= RTOL * np.abs(o) + 1e-30, axis=1)
        assert close.mean() >= 0.95, close.mean()


def test_full_size_net_properties(nrrs):
    """Full-size NET render: counts bounded by C, requested children consistent with
    the next queue, finite non-negative image, F within (0, 1]."""
    s = I.occluded_room(1)
    P = I.rrsnet_init_params(1)
    W = H = 256
    spp, D = 16, 16
    img, st, _ = gpu_render(nrrs, s, W, H, spp, D, nrrs.RRS_NET, params=P, trace=False)
    C = 2 * W * H * spp
    assert st["capacity"] == C and np.all(st["live"] <= C)
    for d in range(D - 1):
        assert st["live"][d + 1] == min(st["requested"][d], C)
    assert np.all(np.isfinite(img)) and img.min() >= 0
    assert np.all((st["F"] > 0) & (st["F"] <= 1))
    assert st["net_evals"] > 0 and st["segments"] == st["live"].sum()
    assert not st["status_bits"] & nrrs.STATUS_TIMEOUT


def test_invalid_arguments(nrrs):
    s = nrrs.Scene(I.box_scene(1))
    out = torch.empty((8, 8, 3), device="cuda")
    for bad in ({"width": 0}, {"max_depth": 33}, {"mode": 7}):
        args = dict(width=8, height=8, spp=1, max_depth=4, mode=0)
        args.update(bad)
        with pytest.raises(nrrs.NrrsError) as e:
            s.render(args["width"], args["height"], args["spp"], args["max_depth"], args["mode"],
                     out=out)
        assert e.value.code == 1
    s.close()


@pytest.mark.parametrize("mode", [0, 2])
def test_ggx_scene_parity(nrrs, mode):
    """Half the objects are GGX + Lambert plastic: their sampled weights depend on the
    geometry, so this checks the GPU GGX lobe against the oracle's on identical decisions.
    At roughness 0.05 the GGX density changes by ~4 tan(theta_h) / (alpha^2 +
    tan(theta_h)^2) relative per radian, which turns FP32 direction differences (~1e-7)
    into a few 1e-6 per bounce; over 6 bounces the bar is 1e-5 relative for 99 % of the
    decision-matched pixels and 1e-4 for all."""
    s = I.icosphere_room(4, min_triangles=3000, subdiv=2)
    assert (s.mats["type"] == I.MAT_GGX).any()
    W = H = 40
    gimg, gst, gtr = gpu_render(nrrs, s, W, H, 4, 6, mode)
    oimg, ost, otr = oracle.render(s, W, H, 4, 6, mode, trace=True)
    hg, cg = pixel_hashes(gtr, W * H)
    ho, co = pixel_hashes(otr, W * H)
    match = (hg == ho) & (cg == co)
    assert match.mean() >= 0.98
    g = gimg.reshape(-1, 3)[match]
    o = oimg.reshape(-1, 3)[match]
    rel = np.max(np.abs(g - o) / np.maximum(np.abs(o), 1e-30), axis=1)
    rel[np.all(o == 0, axis=1) & np.all(g == 0, axis=1)] = 0.0
    assert np.mean(rel <= RTOL) >= 0.99, np.mean(rel <= RTOL)
    assert rel.max() <= 1e-4, rel.max()


def _same_stats(a, b):
    for k in ("live", "sum_q", "F", "alpha", "requested", "dropped"):
        np.testing.assert_array_equal(a[k], b[k])
    assert a["segments"] == b["segments"] and a["net_evals"] == b["net_evals"]


@pytest.mark.parametrize("mode,prec", [("RRS_NET", 32), ("RRS_HEUR_NORM", 32),
                                       ("RRS_NET_MIX", 32), ("RRS_NET", 16), ("RRS_PLAIN_RR", 32)])
def test_graph_captured_render_is_bit_identical(nrrs, mode, prec):
    """The bounce loop captured into a CUDA graph (opts.graph) renders exactly what the
    stream-launched loop renders, frame after frame (the cached graph is updated in place
    with each frame's seeds) and across alternating image shapes (one graph per shape)."""
    s = I.box_scene(2)
    P = I.rrsnet_init_params(5)
    sg, sp = nrrs.Scene(s), nrrs.Scene(s)
    sg.set_params(P)
    sp.set_params(P)
    m = getattr(nrrs, mode)
    gate = 0
    for d, g in enumerate([2, 1, 0, 0, 1, 0, 2, 1]):
        gate |= g << (2 * d)
    shapes = [(64, 48, 4), (32, 32, 2), (64, 48, 4), (64, 48, 4), (32, 32, 2)]
    for frame, (W, H, spp) in enumerate(shapes):
        kw = dict(frame=frame, precision=prec, gate=gate if m == nrrs.RRS_NET_MIX else 0)
        ig, stg = sg.render(W, H, spp, 8, m, graph=1, **kw)
        ip, stp = sp.render(W, H, spp, 8, m, graph=0, **kw)
        torch.cuda.synchronize()
        assert torch.equal(ig, ip), (frame, W, H)
        _same_stats(stg, stp)
    # profiling inside the graph: the event pairs become graph nodes
    _, st = sg.render(64, 48, 4, 8, m, graph=1, profile=1, frame=9, precision=prec)
    assert st["stage_launches"][1] == 8 and st["stage_ms"][1] > 0
    sg.close()
    sp.close()


def test_graph_captured_train_step_matches(nrrs):
    """The training frame recorded through a graph gives the same step as without."""
    out = []
    for graph in (0, 1):
        sc = nrrs.Scene(I.box_scene(1))
        sc.set_params(I.rrsnet_init_params(1))
        sts = [sc.train_step(width=32, height=32, spp=2, max_depth=6, warmup_steps=2,
                             graph=graph) for _ in range(4)]
        out.append((sts, nrrs.nrrs_get_params(sc.handle, nrrs.NET_RRSNET)))
        sc.close()
    for a, b in zip(out[0][0], out[1][0]):
        assert a["loss_rrsnet"] == b["loss_rrsnet"] and a["segments"] == b["segments"]
    np.testing.assert_array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("scene_name", ["box", "occluded", "ggx", "three_rooms"])
def test_tree_formats_give_identical_renders(nrrs, scene_name):
    """The BVH2 with FP16 boxes rounded outward (the default), the BVH2 with FP32 boxes
    and the four-wide tree collapsed from it find the same closest hits (same triangle
    test, same tie rule; the FP16 boxes contain the FP32 ones), so whole renders are
    bit-identical; so are next-event estimation's any-hit shadow queries."""
    s = {"box": lambda: I.box_scene(2), "occluded": lambda: I.occluded_room(1),
         "ggx": lambda: I.icosphere_room(4, min_triangles=20000, subdiv=2),
         "three_rooms": lambda: I.three_rooms(1)}[scene_name]()
    P = I.rrsnet_init_params(3)
    W, H, spp, D = (128, 96, 8, 12) if scene_name != "three_rooms" else (320, 180, 4, 16)
    runs = [(nrrs.RRS_NONE, 0), (nrrs.RRS_NET, 0), (nrrs.RRS_NET, 1)]
    out = []
    for width, bits in ((2, 16), (2, 32), (4, 32)):
        sc = nrrs.Scene(s)
        sc.set_params(P)
        sc.set_bvh_precision(bits)
        sc.set_traversal(width)
        for mode, nee in runs:
            img, st = sc.render(W, H, spp, D, mode, frame=1, nee=nee)
            torch.cuda.synchronize()
            out.append((img.cpu().numpy(), st))
        sc.close()
    n = len(runs)
    if scene_name != "three_rooms":  # there light from the third room seldom reaches room 1
        assert np.abs(out[0][0]).sum() > 0
    for k in (1, 2):
        for (a, sa), (b, sb) in zip(out[:n], out[k * n:(k + 1) * n]):
            np.testing.assert_array_equal(a, b)
            np.testing.assert_array_equal(sa["live"], sb["live"])


def test_scene_far_from_origin_renders_the_same_with_either_node_format(nrrs):
    """At x ~ 2000 binary16 is coarse (spacing 1 or 2), so the rounded boxes are far
    larger than the FP32 ones: the scene defaults to FP32 nodes, and the FP16 nodes,
    still conservative, give the same image, only slower."""
    s = I.box_scene(2)
    tri = s.tri.copy()
    tri[:, 0::3] += 2000.0
    cam = s.cam.copy()
    cam["pos"][:, 0] += 2000.0
    far = I.Scene(tri, s.mat_id, s.mats, cam, "box_far")
    sc = nrrs.Scene(far)
    imgs = []
    for bits in (None, 16, 32):
        if bits:
            sc.set_bvh_precision(bits)
        img, _ = sc.render(64, 48, 4, 8, nrrs.RRS_HEUR_NORM, frame=3, update_ref=0)
        torch.cuda.synchronize()
        imgs.append(img.clone())
    assert torch.abs(imgs[0]).sum() > 0
    assert torch.equal(imgs[0], imgs[1]) and torch.equal(imgs[0], imgs[2])
    sc.close()


def test_bvh_precision_arguments_and_graph_switch(nrrs):
    """Bad widths fail loudly; switching the node format between graph-launched renders
    of one scene takes effect (the graph is keyed by the tree it reads) and gives the
    same image."""
    sc = nrrs.Scene(I.occluded_room(1))
    for bad in (0, 8, 64):
        with pytest.raises(nrrs.NrrsError):
            sc.set_bvh_precision(bad)
    imgs = []
    for bits in (16, 32, 16):
        sc.set_bvh_precision(bits)
        img, _ = sc.render(96, 64, 4, 8, nrrs.RRS_HEUR_NORM, frame=2, update_ref=0, graph=1)
        torch.cuda.synchronize()
        imgs.append(img.clone())
    assert torch.equal(imgs[0], imgs[1]) and torch.equal(imgs[0], imgs[2])
    sc.close()
