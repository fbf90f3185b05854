"""Parity of the training kernels with the FP64 oracle, and train-step behaviour (GPU)."""
import math

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


def _dev(a, dtype=None):
    return torch.from_numpy(np.ascontiguousarray(a if dtype is None else a.astype(dtype))).cuda()


@pytest.mark.parametrize("n_out,n", [(1, 1), (1, 5000), (6, 777), (6, 20000)])
def test_mlp_grad_matches_oracle(nrrs, n_out, n):
    """Summed weight gradients of the MLP backward.  FP32 sums of n per-sample products
    against FP64: bar 1e-4 of the largest gradient entry (each entry sums at most n
    products; block sums of 128 then a fixed-order sum over blocks)."""
    sc = nrrs.Scene(I.box_scene(1))
    rng = np.random.default_rng(n + n_out)
    P = (rng.normal(size=oracle.mlpn_param_count(n_out)) * 0.25).astype(np.float32)
    X = I.random_features(n, seed=n)
    gout = rng.normal(size=(n, n_out)).astype(np.float32)
    grad = torch.zeros(P.size, dtype=torch.float32, device="cuda")
    nrrs.nrrs_mlp_grad(sc.handle, n_out, _dev(P), _dev(X), _dev(gout), n, grad)
    torch.cuda.synchronize()
    G = np.zeros(P.size)
    P64 = P.astype(np.float64)
    for s in range(n):
        G += oracle.mlpn_backward(P64, n_out, X[s].astype(np.float64), gout[s].astype(np.float64))
    g = grad.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(g - G)) <= 1e-4 * np.max(np.abs(G))
    sc.close()


def test_rrsnet_dloss_matches_oracle(nrrs):
    rng = np.random.default_rng(3)
    n, npix = 50_000, 997
    q = rng.uniform(0.05, 3.0, n)
    F = rng.uniform(0.2, 1.0, n)
    Fn = rng.uniform(0.2, 1.0, n)
    t = rng.uniform(0.01, 2.0, n)
    pix = rng.integers(0, npix, n).astype(np.int32)
    m1 = rng.uniform(0.0, 2.0, n)
    m2 = m1 * m1 * rng.uniform(0.5, 3.0, n)
    E = rng.uniform(0.0, 2.0, npix)
    Iref = rng.uniform(0.0, 3.0, npix)
    k = rng.integers(1, 9, npix).astype(np.int64)
    f32 = lambda a: a.astype(np.float32).astype(np.float64)  # noqa: E731
    args32 = [f32(v) for v in (q, F, Fn, t)]
    dq_o, _ = oracle.rrsnet_dloss(*args32, pix, f32(m1), f32(m2), f32(E), f32(Iref), k,
                                  eps=0.01, g=(0.01, 0.05, 0.01))
    Ebar = float(f32(E).mean())
    out = torch.zeros(n, dtype=torch.float32, device="cuda")
    nrrs.nrrs_rrsnet_dloss(_dev(q, np.float32), _dev(F, np.float32), _dev(Fn, np.float32),
                           _dev(t, np.float32), _dev(pix), _dev(m1, np.float32),
                           _dev(m2, np.float32), _dev(E, np.float32), Ebar, _dev(Iref, np.float32),
                           _dev(k, np.int32), n, 0.01, 0.01, 0.05, 0.01, out)
    torch.cuda.synchronize()
    dq = out.cpu().numpy().astype(np.float64)
    qu = f32(F) * f32(q)
    assert np.any(qu < 1) and np.any(qu >= 1)  # both gradient-transfer branches
    # dq is the sum of the transfer term and the bound term, which can cancel; each is an
    # FP32 chain of about 12 roundings, so the bar is 2e-5 of their summed magnitudes
    t1, _ = oracle.rrsnet_dloss(*args32, pix, f32(m1), f32(m2), f32(E), f32(Iref), k,
                                eps=0.01, g=(0.01, 0.05, 0.0))
    t2, _ = oracle.rrsnet_dloss(*args32, pix, f32(m1), f32(m2), f32(E), f32(Iref), k,
                                eps=0.01, g=(0.0, 0.0, 0.01))
    np.testing.assert_allclose(t1 + t2, dq_o, rtol=1e-12, atol=1e-18)
    assert np.all(np.abs(dq - dq_o) <= 2e-5 * (np.abs(t1) + np.abs(t2)) + 1e-12)


def test_adam_matches_oracle(nrrs):
    rng = np.random.default_rng(4)
    n = 2752
    P = rng.normal(size=n).astype(np.float32)
    dP, dm, dv = _dev(P), torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
    Po, mo, vo = P.astype(np.float64), np.zeros(n), np.zeros(n)
    for step in range(1, 4):
        G = rng.normal(size=n).astype(np.float32)
        nrrs.nrrs_adam_step(dP, _dev(G), dm, dv, n, step, 0.005)
        oracle.adam_step(Po, G.astype(np.float64), mo, vo, step, 0.005)
    torch.cuda.synchronize()
    np.testing.assert_allclose(dP.cpu().numpy(), Po, rtol=1e-5, atol=1e-7)


def _render_suffix(nrrs, scene, W, H, spp, D, mode, params=None, **kw):
    sc = nrrs.Scene(scene)
    if params is not None:
        sc.set_params(params)
    C = 2 * W * H * spp
    suf = torch.zeros((D, C, 4), dtype=torch.float32, device="cuda")
    tr = torch.zeros((D, C, 5), dtype=torch.int32, device="cuda")
    img, st = sc.render(W, H, spp, D, mode, d_suffix=suf.data_ptr(), d_trace=tr.data_ptr(), **kw)
    torch.cuda.synchronize()
    S = suf.cpu().numpy()
    T = tr.cpu().numpy().view(np.uint32)
    sc.close()
    return img.cpu().numpy(), st, [S[d, :st["live"][d], :3] for d in range(D)], \
        [T[d, :st["live"][d]] for d in range(D)]


def test_reverse_pass_furnace_exact(nrrs):
    """Furnace (albedo 0.5, emission 1), no RRS: a vertex at depth d has suffix sum
    t * sum_{k <= D-d} 0.5^k, exactly in FP32."""
    s = I.box_scene(1, furnace=True)
    D = 6
    img, st, S, T = _render_suffix(nrrs, s, 32, 32, 2, D, nrrs.RRS_NONE)
    for d in range(D):
        t = 0.5 ** d
        expect = t * (1 - 0.5 ** (D - d)) / 0.5
        assert np.mean(S[d] == expect) > 0.999


def test_reverse_pass_matches_oracle(nrrs):
    """Per-vertex suffix sums of a normalised-RRS render agree with the oracle's reverse
    pass on vertices of pixels whose decisions all match (1e-5 relative)."""
    from tests.test_gpu_render import pixel_hashes

    s = I.box_scene(2)
    P = I.rrsnet_init_params(5)
    W = H = 32
    spp, D = 4, 7
    img, st, S, T = _render_suffix(nrrs, s, W, H, spp, D, nrrs.RRS_NET, params=P)
    oimg, ost, otr = oracle.render(s, W, H, spp, D, oracle.MODE_NET, params=P.astype(np.float64),
                                   trace=True, record=True)
    hg, cg = pixel_hashes(T, W * H)
    ho, co = pixel_hashes(otr, W * H)
    good = (hg == ho) & (cg == co)
    assert good.mean() > 0.99
    checked = 0
    for d in range(D):
        okey = {(int(r[0]), int(r[1]), int(r[2])): i for i, r in enumerate(otr[d])}
        Od = ost["rec"][d][:, 0:3]
        for i, r in enumerate(T[d]):
            if not good[int(r[0])]:
                continue
            j = okey[(int(r[0]), int(r[1]), int(r[2]))]
            np.testing.assert_allclose(S[d][i], Od[j], rtol=1e-5, atol=1e-30)
            checked += 1
    assert checked > 0.9 * sum(len(t) for t in T)


def test_train_step_warmup_converges_and_ema(nrrs):
    """Step (1) of Sec. 4: RRSNet regressed to 1 -- its loss falls and the trained
    network's factors approach 1; the rendering weights follow as the EMA."""
    sc = nrrs.Scene(I.box_scene(1))
    sc.set_params(I.rrsnet_init_params(1))
    losses, stat = [], []
    for k in range(30):
        st = sc.train_step(width=64, height=64, spp=4, max_depth=8, warmup_steps=100,
                           lr_rrsnet=3e-3)
        assert st["fallback"] == 0 and st["phase"] == 1 and st["samples"] > 0
        losses.append(st["loss_rrsnet"])
        stat.append(st["loss_statnet"])
    assert losses[-1] < 0.2 * losses[0]
    assert np.mean(stat[-5:]) < np.mean(stat[:5])
    raw = nrrs.nrrs_get_params(sc.handle, nrrs.NET_RRSNET_TRAIN)
    X = I.random_features(4096, seed=9).astype(np.float64)
    q = oracle.mlp_forward_batch(raw.astype(np.float64), X.astype(np.float32))
    assert np.median(np.abs(q - 1.0)) < 0.15
    ema = nrrs.nrrs_get_params(sc.handle, nrrs.NET_RRSNET)
    assert not np.array_equal(ema, raw) and np.all(np.isfinite(ema))
    sc.close()


def test_train_step_full_phase_runs(nrrs):
    sc = nrrs.Scene(I.box_scene(3))
    sc.set_params(I.rrsnet_init_params(3))
    for k in range(12):
        st = sc.train_step(width=64, height=64, spp=4, max_depth=8, warmup_steps=4)
        assert math.isfinite(st["loss_rrsnet"]) and math.isfinite(st["loss_statnet"])
    assert st["phase"] == 2 and st["step"] >= 8
    assert st["loss_min"] > 0 and st["loss_rrs"] >= 0
    sc.close()


def test_train_step_nonfinite_weights_fall_back(nrrs):
    sc = nrrs.Scene(I.box_scene(1))
    P = I.rrsnet_init_params(1)
    sc.set_params(P)
    sc.train_step(width=32, height=32, spp=2, max_depth=6)
    good = nrrs.nrrs_get_params(sc.handle, nrrs.NET_RRSNET_TRAIN)
    bad = good.copy()
    bad[:512] = np.nan
    nrrs.nrrs_set_params(sc.handle, nrrs.NET_RRSNET_TRAIN, bad)
    st = sc.train_step(width=32, height=32, spp=2, max_depth=6)
    assert st["fallback"] == 1 and st["step"] == 1
    np.testing.assert_array_equal(nrrs.nrrs_get_params(sc.handle, nrrs.NET_RRSNET_TRAIN), good)
    # the next frame renders with the heuristic at the network's depths, the one after
    # with the network again
    _, r1 = sc.render(32, 32, 2, 6, nrrs.RRS_NET)
    assert r1["status_bits"] & nrrs.STATUS_HEUR_FALLBACK and r1["net_evals"] == 0
    _, r2 = sc.render(32, 32, 2, 6, nrrs.RRS_NET)
    assert not r2["status_bits"] & nrrs.STATUS_HEUR_FALLBACK and r2["net_evals"] > 0
    sc.close()


def test_rrsnet_autograd_matches_oracle_and_finite_differences(nrrs):
    """The differentiable RRSNet (library forward and backward behind a
    torch.autograd.Function): its weight gradient of L = sum_s c_s q_s equals the FP64
    oracle's chain rule through Eq. rrsnet_activation (1e-4 of the largest entry: FP32
    sums of n products), and a central difference of the library's own forward along a
    random direction (relative 2e-3: FP32 forward noise over the step)."""
    sc = nrrs.Scene(I.box_scene(1))
    rng = np.random.default_rng(21)
    P = (I.rrsnet_init_params(8) * 2.0).astype(np.float32)  # both activation branches
    n = 3000
    X = I.random_features(n, seed=21)
    c = rng.normal(size=n).astype(np.float32)
    w = torch.tensor(P, device="cuda", requires_grad=True)
    xs = _dev(X)
    q = nrrs.rrsnet(sc, xs, w)
    # the forward is the query kernel with these weights
    sc.set_params(P)
    np.testing.assert_array_equal(q.detach().cpu().numpy(), sc.query(xs).cpu().numpy())
    (q * _dev(c)).sum().backward()
    g = w.grad.cpu().numpy().astype(np.float64)
    G = np.zeros(P.size)
    P64 = P.astype(np.float64)
    zs = [oracle.mlp_forward(P64, X[s])[1] for s in range(n)]
    assert min(zs) < 0 < max(zs)
    for s in range(n):
        G += oracle.mlp_backward(P64, X[s].astype(np.float64), float(c[s]))
    assert np.max(np.abs(g - G)) <= 1e-4 * np.max(np.abs(G))
    # central difference of the library forward along v (sums in FP64 on the host)
    v = rng.normal(size=P.size).astype(np.float32)
    h = 1e-2 / np.linalg.norm(v)

    def L(p):
        with torch.no_grad():
            qq = nrrs.rrsnet(sc, xs, _dev(p.astype(np.float32)))
        return float(np.dot(qq.cpu().numpy().astype(np.float64), c.astype(np.float64)))

    fd = (L(P + h * v) - L(P - h * v)) / (2 * h)
    assert abs(fd - float(g @ v)) <= 2e-3 * abs(float(g @ v)) + 1e-3
    sc.close()


def test_rrsnet_autograd_trains(nrrs):
    """A few Adam steps through the autograd path regress RRSNet towards a target factor
    (the warm-up objective of Sec. 4 "Training", here with torch's optimizer)."""
    sc = nrrs.Scene(I.box_scene(1))
    w = torch.tensor(I.rrsnet_init_params(3), device="cuda", requires_grad=True)
    xs = _dev(I.random_features(8192, seed=4))
    opt = torch.optim.Adam([w], lr=3e-3)
    losses = []
    for _ in range(60):
        opt.zero_grad()
        loss = ((nrrs.rrsnet(sc, xs, w) - 1.5) ** 2).mean()
        loss.backward()
        opt.step()
        losses.append(loss.item())
    assert losses[-1] < 0.1 * losses[0]
    sc.close()


def test_train_step_batch_subsampling(nrrs):
    """Sec. 4's fixed training batch: with batch_size below the recorded vertex count the
    step trains on batch_size systematic samples of the frame's vertices, so the count
    of trainable samples among them follows the frame's trainable fraction; the warm-up
    regression still converges on the smaller batches."""
    kw = dict(width=64, height=64, spp=4, max_depth=8)
    a = nrrs.Scene(I.box_scene(1))
    a.set_params(I.rrsnet_init_params(1))
    full = a.train_step(warmup_steps=100, lr_rrsnet=3e-3, **kw)
    frac = full["samples"] / full["segments"]
    assert full["segments"] > 20_000
    b = nrrs.Scene(I.box_scene(1))
    b.set_params(I.rrsnet_init_params(1))
    losses = []
    for k in range(30):
        st = b.train_step(batch_size=5000, warmup_steps=100, lr_rrsnet=3e-3, **kw)
        assert st["fallback"] == 0 and st["samples"] <= 5000
        if k == 0:  # the same recorded frame as the full step
            assert st["segments"] == full["segments"]
            assert abs(st["samples"] - 5000 * frac) <= 0.05 * 5000 * frac + 20, (st["samples"], frac)
        losses.append(st["loss_rrsnet"])
    assert losses[-1] < 0.2 * losses[0]
    a.close()
    b.close()
