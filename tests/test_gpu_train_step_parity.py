"""The training step's own gradient chain against the FP64 oracle (GPU).

nrrs_train_step records a frame, runs the reverse pass, computes the pixel errors
(Eq. loss-function_min), smooths them in time (Eq. error_temporal) and space (the
normal-guided filter standing in for the denoiser, Sec. 4 "Tackle Low Spp"), counts the
training samples per pixel, then forms StatNet's relative-L2 gradient (Eq.
loss-function_StatNet) and RRSNet's gradient: the warm-up regression to 1 (Sec. 4
"Training", step 1) or the full loss (Eq. loss-function_rrsnet through Eq.
gradient_transfer_rr_mc / splitting_mc with StatNet's moments).  Its debug record
returns what it is about to apply; the oracle composes the same chain from its own
render of the same frame (same weights, same Philox key) and its own functions.

Two steps with zero learning rates keep the weights fixed: the first is a warm-up step
(the error map's EMA starts), the second a full-loss step whose error map mixes both
frames.  The frame is small enough for every pixel's decisions to match the oracle's,
which the test checks first, so the two sides sum the same samples.  Bars: per-pixel
quantities 1e-5 relative (FP32 sums of a few terms), sample counts exact, summed weight
gradients 1e-4 of their largest entry (FP32 sums of ~10^4 per-sample products)."""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_2510_07868_b300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

W = H = 32
SPP, D = 4, 6
SEED = (3, 1)
FRAME0 = 40
EPS = 0.01
GAMMA = (0.01, 0.05, 0.01)


@pytest.fixture(scope="module")
def nrrs():
    from paper_2510_07868_b300 import nrrs as m

    assert torch.cuda.is_available()
    return m


def _decisions(trace, npix):
    per = [[] for _ in range(npix)]
    for d, tr in enumerate(trace):
        for r in tr:
            per[int(r[0])].append((d, int(r[1]), int(r[2]), int(r[3]), int(r[4])))
    return [sorted(p) for p in per]


def _oracle_step(scene, P, S, ref, frame, E_acc_prev, full):
    """One training step composed from the oracle's functions (weights fixed)."""
    npix = W * H
    _, st, tr = oracle.render(scene, W, H, SPP, D, oracle.MODE_NET, params=P, record=True,
                              trace=True, seed=SEED, frame=frame, f_rate=0.85)
    rec = st["rec"]
    # pixel errors from the depth-1 suffix sums (queue pixel-major, sample-minor)
    S1 = rec[0][:, 0:3].reshape(npix, SPP, 3)
    V, E_cur = oracle.pixel_error(S1, SPP, ref, EPS)
    E_acc = oracle.error_temporal(E_cur, E_acc_prev, alpha=0.5, first=E_acc_prev is None)
    nrm = oracle.pixel_normals(rec[0][:, 14:30], rec[0][:, 9], npix, SPP)
    E = oracle.error_filter(E_acc, W, H, 2, nrm, 8.0)
    # training samples: every vertex where the network was evaluated (q_orig > 0)
    rows = np.concatenate([np.c_[np.full(len(r), d), r] for d, r in enumerate(rec)])
    rows = rows[rows[:, 1 + 9] > 0]
    depth = rows[:, 0].astype(np.int64)
    r = rows[:, 1:]
    pix = r[:, 13].astype(np.int64)
    k = np.bincount(pix, minlength=npix).astype(np.int64)
    N = len(r)
    x = r[:, 14:30]
    # StatNet: relative L2 of both moments against the one-sample targets (S - dep) / t
    t = r[:, 6:9]
    L = np.where(t > 0, (r[:, 0:3] - r[:, 3:6]) / np.where(t > 0, t, 1.0), 0.0)
    G_stat = np.zeros(S.size)
    m1 = np.zeros(N)
    m2 = np.zeros(N)
    xs = x.copy()
    xs[:, 13:16] = 0.0
    for s in range(N):
        out = oracle.mlpn_forward(S, 6, xs[s])
        m1[s], m2[s] = out[:3].mean(), out[3:].mean()
        _, dpred = oracle.statnet_dloss(out, L[s], EPS)
        G_stat += oracle.mlpn_backward(S, 6, xs[s], dpred / N)
    # RRSNet
    q = np.array([oracle.mlp_forward(P, x[s])[0] for s in range(N)])
    G_rrs = np.zeros(P.size)
    if not full:
        dq = 2.0 * (q - 1.0) / (1.0 + EPS) / N
    else:
        N_px = W * H * SPP  # Eq. F_norm's budget: the primary queue
        F = st["F"].astype(np.float64)
        sq = st["sum_q"]
        Fn = np.where(sq > 0, np.minimum(1.0, N_px / np.where(sq > 0, sq, 1.0)), 1.0)
        Iref = ref.reshape(-1, 3).mean(axis=1)
        dq, _ = oracle.rrsnet_dloss(q, F[depth], Fn[depth], t.mean(axis=1), pix, m1, m2, E, Iref,
                                    k, eps=EPS, g=GAMMA, q_used=r[:, 10])
    for s in range(N):
        G_rrs += oracle.mlp_backward(P, x[s], dq[s])
    return {"V": V, "E": E, "E_acc": E_acc, "k": k, "N": N, "G_stat": G_stat, "G_rrs": G_rrs,
            "trace": tr, "vertices": int(sum(len(a) for a in rec))}


def test_train_step_gradients_match_the_oracle(nrrs):
    scene = I.box_scene(1)
    P = I.rrsnet_init_params(4)
    S = I.statnet_init_params(4)
    npix = W * H
    rng = np.random.default_rng(8)
    ref = (0.2 + 0.3 * rng.random((H, W, 3))).astype(np.float32)
    sc = nrrs.Scene(scene)
    sc.set_params(P)
    nrrs.nrrs_set_params(sc.handle, nrrs.NET_STATNET, S)
    dref = torch.from_numpy(ref).cuda()
    P64, S64, ref64 = P.astype(np.float64), S.astype(np.float64), ref.astype(np.float64)
    E_acc = None
    for step, full in ((0, False), (1, True)):
        frame = FRAME0 + step
        # the decisions of the recorded frame, through the public render of the same key
        tr = torch.zeros((D, 2 * npix * SPP, 5), dtype=torch.int32, device="cuda")
        _, rst = sc.render(W, H, SPP, D, nrrs.RRS_NET, d_trace=tr.data_ptr(), seed_lo=SEED[0],
                           seed_hi=SEED[1], frame=frame, update_ref=0)
        torch.cuda.synchronize()
        gtr = tr.cpu().numpy().view(np.uint32)
        o = _oracle_step(scene, P64, S64, ref64, frame, E_acc, full)
        E_acc = o["E_acc"]
        gd = _decisions([gtr[d, :rst["live"][d]] for d in range(D)], npix)
        od = _decisions(o["trace"], npix)
        assert all(a == b for a, b in zip(gd, od)), "a decision differs: pick another key"
        dbg = nrrs.TrainDebug.with_buffers(npix, nrrs.STATNET_PARAMS, nrrs.RRSNET_PARAMS)
        opts = nrrs.TrainOpts.defaults(width=W, height=H, spp=SPP, max_depth=D, seed_lo=SEED[0],
                                       seed_hi=SEED[1], frame=FRAME0, warmup_steps=1,
                                       lr_rrsnet=0.0, lr_statnet=0.0,
                                       d_pixel_ref=dref.data_ptr(), batch_size=1 << 22,
                                       debug=C.addressof(dbg))
        ts = nrrs.nrrs_train_step(sc.handle, opts)
        assert ts["phase"] == (2 if full else 1) and ts["fallback"] == 0
        a = dbg.arrays
        assert dbg.vertices == o["vertices"] and dbg.batch == dbg.vertices
        assert ts["samples"] == o["N"]
        np.testing.assert_array_equal(a["samples"], o["k"])
        Vo = o["V"]
        np.testing.assert_allclose(a["pixel_var"], Vo, rtol=1e-5, atol=1e-6 * Vo.max())
        np.testing.assert_allclose(a["pixel_error"], o["E"], rtol=1e-5, atol=1e-6 * o["E"].max())
        assert abs(dbg.ebar - o["E"].mean()) <= 1e-5 * o["E"].mean()
        for name in ("G_stat", "G_rrs"):
            g = a["grad_statnet" if name == "G_stat" else "grad_rrsnet"].astype(np.float64)
            G = o[name]
            err = np.max(np.abs(g - G))
            print(f"step {step} {name}: max |G| {np.max(np.abs(G)):.3e}, max error {err:.3e}")
            assert err <= 1e-4 * np.max(np.abs(G)), (name, step, err, np.max(np.abs(G)))
    sc.close()


def test_ema_matches_oracle(nrrs):
    """The EMA of the rendering weights (Sec. 4 "Training"): FP32 against FP64, 1e-6."""
    rng = np.random.default_rng(11)
    n = 2752
    avg = rng.normal(size=n).astype(np.float32)
    P = rng.normal(size=n).astype(np.float32)
    d_avg = torch.from_numpy(avg.copy()).cuda()
    d_P = torch.from_numpy(P).cuda()
    o = avg.astype(np.float64)
    for decay in (0.1, 0.5, 0.99):
        nrrs.nrrs_ema(d_avg, d_P, n, decay)
        oracle.ema(o, P.astype(np.float64), decay=np.float32(decay))
    torch.cuda.synchronize()
    np.testing.assert_allclose(d_avg.cpu().numpy(), o, rtol=1e-6, atol=1e-7)
