"""StatNet on the encodings of Sec. 4 "Input Encoding" (GPU): hash grid of the position,
one-blob direction and roughness.  The encoding, its backward pass and the 32-input
network's gradients are compared with the FP64 oracle; renders that run StatNet (ADRRS
(NN), the NRRS inputs) are compared with the oracle's on decision-matched pixels; training
steps move the grid and lower StatNet's loss."""
import numpy as np
import pytest

import oracle
from paper_2510_07868_b300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def nrrs():
    from paper_2510_07868_b300 import nrrs as m

    assert torch.cuda.is_available()
    return m


def _grid_scene(nrrs, s, seed, grid_scale=0.5):
    sc = nrrs.Scene(s)
    sc.set_statnet_encoding(1)
    rng = np.random.default_rng(seed)
    SP = (rng.normal(size=nrrs.STATNET_GRID_PARAMS) * 0.3).astype(np.float32)
    SP[-6 * 32:] = np.abs(SP[-6 * 32:])
    G = (rng.normal(size=nrrs.GRID_PARAMS) * grid_scale).astype(np.float32)
    nrrs.nrrs_set_params(sc.handle, nrrs.NET_STATNET, SP)
    nrrs.nrrs_set_params(sc.handle, nrrs.NET_STATNET_GRID, G)
    return sc, SP, G


def _features(n, seed):
    rng = np.random.default_rng(seed)
    f = np.zeros((n, 16), dtype=np.float32)
    f[:, :3] = rng.random((n, 3))
    w = rng.normal(size=(n, 3))
    f[:, 3:6] = w / np.linalg.norm(w, axis=1, keepdims=True)
    rough = np.where(rng.random(n) < 0.5, 1.0, rng.uniform(0.05, 0.5, n)).astype(np.float32)
    return f, rough


def test_statnet_inputs_match_oracle(nrrs):
    sc, _, G = _grid_scene(nrrs, I.box_scene(1), 1)
    n = 512
    f, rough = _features(n, 2)
    out = torch.empty((n, 32), device="cuda")
    nrrs.nrrs_statnet_inputs(sc.handle, torch.from_numpy(f).cuda(), torch.from_numpy(rough).cuda(),
                             n, out)
    torch.cuda.synchronize()
    g = out.cpu().numpy()
    G64 = G.astype(np.float64)
    o = np.stack([oracle.statnet_grid_inputs(G64, f[i, :3].astype(np.float64),
                                             f[i, 3:6].astype(np.float64), float(rough[i]))
                  for i in range(n)])
    np.testing.assert_allclose(g, o, rtol=0, atol=5e-5)
    sc.close()


def test_grid_backward_matches_oracle(nrrs):
    sc, _, _ = _grid_scene(nrrs, I.box_scene(1), 3)
    n = 64
    f, _ = _features(n, 4)
    dx = np.random.default_rng(5).normal(size=(n, 16)).astype(np.float32)
    grad = torch.zeros(nrrs.GRID_PARAMS, device="cuda")
    nrrs.nrrs_grid_backward(sc.handle, torch.from_numpy(f).cuda(), torch.from_numpy(dx).cuda(), n,
                            grad)
    torch.cuda.synchronize()
    o = oracle.grid_backward(f[:, :3].astype(np.float64), dx.astype(np.float64))
    g = grad.cpu().numpy()
    assert np.count_nonzero(o) > 0
    np.testing.assert_allclose(g, o, rtol=0, atol=2e-5 * np.abs(o).max())
    sc.close()


def test_statnet_grad32_matches_oracle(nrrs):
    sc = nrrs.Scene(I.box_scene(1))
    rng = np.random.default_rng(6)
    n = 300
    P = (rng.normal(size=nrrs.STATNET_GRID_PARAMS) * 0.3).astype(np.float32)
    x = rng.normal(size=(n, 32)).astype(np.float32)
    gout = rng.normal(size=(n, 6)).astype(np.float32)
    d_grad = torch.empty(nrrs.STATNET_GRID_PARAMS, device="cuda")
    nrrs.nrrs_statnet_grad(sc.handle, torch.from_numpy(P).cuda(), torch.from_numpy(x).cuda(),
                           torch.from_numpy(gout).cuda(), n, d_grad)
    torch.cuda.synchronize()
    G = np.zeros(P.size)
    for i in range(n):
        Gi, _ = oracle.mlpk_backward(P.astype(np.float64), 32, 6, x[i].astype(np.float64),
                                     gout[i].astype(np.float64))
        G += Gi
    np.testing.assert_allclose(d_grad.cpu().numpy(), G, rtol=1e-4, atol=1e-4 * np.abs(G).max())
    sc.close()


def test_adrrs_with_grid_statnet_parity(nrrs):
    s = I.box_scene(3)
    P = I.rrsnet_init_params(2)
    sc, SP, G = _grid_scene(nrrs, s, 7, grid_scale=0.3)
    sc.set_params(P)
    gate = 0
    for d, g in enumerate([2, 3, 0, 3, 1, 3, 0, 3]):
        gate |= g << (2 * d)
    W = H = 40
    ref = (np.full((H * W, 3), 0.3) * np.linspace(0.4, 1.6, H * W)[:, None]).astype(np.float32)
    C = 2 * W * H * 4
    tr = torch.zeros((8, C, 5), dtype=torch.int32, device="cuda")
    dref = torch.from_numpy(ref).cuda()
    img, st = sc.render(W, H, 4, 8, nrrs.RRS_NET_MIX, gate=gate, d_trace=tr.data_ptr(),
                        d_pixel_ref=dref.data_ptr())
    torch.cuda.synchronize()
    trn = tr.cpu().numpy().view(np.uint32)
    gtr = [trn[d, :st["live"][d]] for d in range(8)]
    assert st["net_evals"] > 0 and st["nonfinite"] == 0
    oimg, _, otr = oracle.render(s, W, H, 4, 8, oracle.MODE_NET_MIX, params=P.astype(np.float64),
                                 gate=gate, stat_params=SP.astype(np.float64),
                                 stat_grid=G.astype(np.float64), pixel_ref=ref.astype(np.float64),
                                 trace=True)
    # FP32 positions scaled by 2048 at the finest grid level carry ~1e-4 relative error in
    # the interpolation weights; ADRRS factors inherit it (q = r outside the weight window)
    # and so do the weights t / q of the paths, so matched pixels agree to 2e-3
    from test_gpu_render import pixel_hashes
    hg, cg = pixel_hashes(gtr, W * H)
    ho, co = pixel_hashes(otr, W * H)
    match = (hg == ho) & (cg == co)
    assert match.mean() >= 0.97
    g = img.cpu().numpy().reshape(-1, 3)[match].astype(np.float64)
    o = oimg.reshape(-1, 3)[match]
    rel = np.max(np.abs(g - o) / np.maximum(np.abs(o), 1e-30), axis=1)
    rel[np.all(o == 0, axis=1) & np.all(g == 0, axis=1)] = 0.0
    assert rel.max() <= 2e-3 and np.mean(rel <= 1e-5) >= 0.8, (rel.max(), np.mean(rel <= 1e-5))
    sc.close()


def test_nrrs_inputs_with_grid_statnet_parity(nrrs):
    s = I.icosphere_room(4, min_triangles=3000, subdiv=2)
    P = I.rrsnet_init_params(3)
    sc, SP, G = _grid_scene(nrrs, s, 8, grid_scale=0.3)
    sc.set_params(P)
    sc.set_rrsnet_inputs(1)
    W = H = 32
    ref = np.full((H * W, 3), 0.7, dtype=np.float32)
    C = 2 * W * H * 4
    tr = torch.zeros((6, C, 5), dtype=torch.int32, device="cuda")
    dref = torch.from_numpy(ref).cuda()
    img, st = sc.render(W, H, 4, 6, nrrs.RRS_NET, d_trace=tr.data_ptr(), d_pixel_ref=dref.data_ptr())
    torch.cuda.synchronize()
    trn = tr.cpu().numpy().view(np.uint32)
    gtr = [trn[d, :st["live"][d]] for d in range(6)]
    oimg, ost, otr = oracle.render(s, W, H, 4, 6, oracle.MODE_NET, params=P.astype(np.float64),
                                   stat_params=SP.astype(np.float64), rrsnet_inputs=1,
                                   stat_grid=G.astype(np.float64),
                                   pixel_ref=ref.astype(np.float64), trace=True)
    np.testing.assert_allclose(st["sum_q"][0], ost["sum_q"][0], rtol=1e-5)
    from test_gpu_render import pixel_hashes
    hg, cg = pixel_hashes(gtr, W * H)
    ho, co = pixel_hashes(otr, W * H)
    match = (hg == ho) & (cg == co)
    assert match.mean() >= 0.95
    g, o = img.cpu().numpy().reshape(-1, 3)[match].astype(np.float64), oimg.reshape(-1, 3)[match]
    rel = np.max(np.abs(g - o) / np.maximum(np.abs(o), 1e-30), axis=1)
    rel[np.all(o == 0, axis=1) & np.all(g == 0, axis=1)] = 0.0
    assert np.mean(rel <= 1e-4) >= 0.98
    sc.close()


def test_training_moves_the_grid_and_lowers_statnet_loss(nrrs):
    s = I.occluded_room(1, n_random=500)
    sc = nrrs.Scene(s)
    sc.set_params(I.rrsnet_init_params(1))
    sc.set_statnet_encoding(1)
    G0 = nrrs.nrrs_get_params(sc.handle, nrrs.NET_STATNET_GRID)
    assert np.all(np.abs(G0) <= 1e-4) and np.any(G0 != 0)
    for _ in range(3):
        sc.render(64, 64, 4, 8, nrrs.RRS_HEUR_NORM)
    losses = []
    for k in range(60):
        st = sc.train_step(width=64, height=64, spp=2, max_depth=8, warmup_steps=20, frame=k)
        assert np.isfinite(st["loss_statnet"]) and not st["fallback"]
        losses.append(st["loss_statnet"])
    G1 = nrrs.nrrs_get_params(sc.handle, nrrs.NET_STATNET_GRID)
    assert np.count_nonzero(G1 != G0) > 1000
    assert np.mean(losses[-10:]) < np.mean(losses[:10]), (losses[:10], losses[-10:])
    # ADRRS (NN) renders on the trained grid StatNet
    gate = sum(nrrs.GATE_ADRRS << (2 * d) for d in range(8))
    img, st = sc.render(64, 64, 4, 8, nrrs.RRS_NET_MIX, gate=gate, update_ref=0)
    assert torch.isfinite(img).all() and st["status_bits"] & nrrs.STATUS_NONFINITE == 0
    sc.close()
