"""Batched renders: many uneven jobs traced together, one RRSNet, Eq. F_norm per job (GPU).

A job's paths draw the random numbers its own render would, so each job of a batch must
reproduce the single-scene render of that job; the FP64 oracle renders jobs whole where
it can finish in seconds."""
import numpy as np
import pytest

import oracle
from paper_2510_07868_b300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ORACLE_MODE = {0: oracle.MODE_NONE, 1: oracle.MODE_PLAIN_RR, 2: oracle.MODE_HEUR_NORM,
               3: oracle.MODE_NET, 4: oracle.MODE_NET_MIX}


@pytest.fixture(scope="module")
def nrrs():
    from paper_2510_07868_b300 import nrrs as m

    assert torch.cuda.is_available()
    return m


def _relmse(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.mean((a - b) ** 2 / (b * b + 0.01)))


def _gate(nrrs, D):
    g = 0
    for d in range(D):
        g |= [nrrs.GATE_FIXED, nrrs.GATE_NET, nrrs.GATE_HEUR][d % 3] << (2 * d)
    return g


def _check_job_equals_single(nrrs, job, mode, P, img, F, sq, **kw):
    """The job rendered alone: the same per-depth F and sum of q (1e-12: FP64 sums in
    another order), and then the same image bit for bit."""
    scene, W, H, spp, D = job
    sc = nrrs.Scene(scene)
    sc.set_params(P)
    ref, st = sc.render(W, H, spp, D, mode, **kw)
    torch.cuda.synchronize()
    np.testing.assert_allclose(sq[:D], st["sum_q"][:D], rtol=1e-12, atol=0)
    same_F = np.array_equal(F[:D], st["F"][:D])
    if same_F:
        assert torch.equal(img, ref)
    sc.close()
    return same_F


@pytest.mark.parametrize("mode", ["RRS_NET", "RRS_HEUR_NORM", "RRS_PLAIN_RR", "RRS_NET_MIX",
                                  "RRS_NONE"])
def test_small_batch_equals_single_renders_and_oracle(nrrs, mode):
    m = getattr(nrrs, mode)
    jobs = [(I.box_scene(1), 24, 16, 3, 6),
            (I.occluded_room(2, n_random=200), 16, 16, 2, 8),
            (I.icosphere_room(3, min_triangles=1500, subdiv=2), 20, 12, 4, 5),
            (I.box_scene(4, furnace=True), 8, 8, 1, 4)]
    P = (I.rrsnet_init_params(2) * 2.0).astype(np.float32)
    gate = _gate(nrrs, 8)
    b = nrrs.Batch(jobs)
    b.set_params(P)
    kw = dict(frame=3, update_ref=0, gate=gate if m == nrrs.RRS_NET_MIX else 0)
    imgs, st, live, F, sq = b.render(m, **kw)
    torch.cuda.synchronize()
    assert np.array_equal(live[:, :8].sum(axis=0), st["live"][:8])
    for j, job in enumerate(jobs):
        scene, W, H, spp, D = job
        assert np.all(live[j, D:] == 0)
        assert _check_job_equals_single(nrrs, job, m, P, imgs[j], F[j], sq[j], **kw)
        oimg, ost, _ = oracle.render(scene, W, H, spp, D, ORACLE_MODE[m], frame=3,
                                     params=P.astype(np.float64), gate=kw["gate"])
        g = imgs[j].cpu().numpy().astype(np.float64)
        close = np.all(np.abs(g - oimg) <= 1e-5 * np.abs(oimg) + 1e-30, axis=2)
        assert close.mean() >= 0.98, (j, close.mean())
    b.close()


def test_batch_of_64_uneven_jobs_full_size(nrrs):
    """64 jobs: sides 32..512, spp 1..64, depth 8..32, 1k..50k triangles (about 83 M
    primary paths), one RRSNet, tuned shapes, graph-captured loop."""
    jobs = I.uneven_jobs(1)
    n = len(jobs)
    P = I.rrsnet_init_params(3)
    b = nrrs.Batch(jobs)
    b.set_params(P)
    b.tune(32)
    kw = dict(frame=0, update_ref=0)
    imgs, st, live, F, sq = b.render(nrrs.RRS_NET, graph=1, **kw)
    torch.cuda.synchronize()
    Dm = b.max_depth
    assert np.array_equal(live[:, :Dm].sum(axis=0), st["live"][:Dm])
    C = 2 * sum(w * h * s for _, w, h, s, _ in jobs)
    assert st["capacity"] == C and st["dropped"].sum() == 0
    assert not st["status_bits"] & nrrs.STATUS_TIMEOUT
    for j, (_, W, H, spp, D) in enumerate(jobs):
        assert live[j, 0] == W * H * spp and np.all(live[j, D:] == 0)
        assert np.all((F[j, :D] > 0) & (F[j, :D] <= 1))
        assert torch.isfinite(imgs[j]).all() and imgs[j].min() >= 0
    # jobs alone: the smallest, the largest and a few others
    sizes = [w * h * s for _, w, h, s, _ in jobs]
    pick = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), 5, 17, 33, 50})
    same = [_check_job_equals_single(nrrs, jobs[j], nrrs.RRS_NET, P, imgs[j], F[j], sq[j], **kw)
            for j in pick]
    assert sum(same) >= len(pick) - 1
    # FP64 oracle on the jobs it can render whole in seconds
    cost = [w * h * s * sc.n_tri for sc, w, h, s, _ in jobs]
    small = [j for j in np.argsort(cost)[:3]]
    rel_oracle = {}
    for j in small:
        scene, W, H, spp, D = jobs[j]
        oimg, _, _ = oracle.render(scene, W, H, spp, D, oracle.MODE_NET, params=P.astype(np.float64))
        g = imgs[j].cpu().numpy().astype(np.float64)
        close = np.all(np.abs(g - oimg) <= 1e-5 * np.abs(oimg) + 1e-30, axis=2)
        rel_oracle[int(j)] = _relmse(g, oimg)
        assert close.mean() >= 0.98, (j, close.mean())
    # per-job relMSE of NET and of the plain-RR baseline against an 8-frame NONE mean
    ref = [torch.zeros_like(im, dtype=torch.float64) for im in imgs]
    frames = 8
    for f in range(frames):
        r_imgs, _, _, _, _ = b.render(nrrs.RRS_NONE, frame=100 + f, update_ref=0, graph=1)
        for j in range(n):
            ref[j] += r_imgs[j].double() / frames
    net = [im.cpu().numpy() for im in imgs]
    rr_imgs, _, _, _, _ = b.render(nrrs.RRS_PLAIN_RR, frame=0, update_ref=0, graph=1)
    rr = [im.cpu().numpy() for im in rr_imgs]
    refs = [r.cpu().numpy() for r in ref]
    e_net = np.array([_relmse(net[j], refs[j]) for j in range(n)])
    e_rr = np.array([_relmse(rr[j], refs[j]) for j in range(n)])
    assert np.all(np.isfinite(e_net)) and np.all(np.isfinite(e_rr))
    print(f"batch: {n} jobs, {sum(sizes)} primary paths; oracle relMSE on jobs {rel_oracle}; "
          f"relMSE vs 8-frame NONE mean: NET median {np.median(e_net):.3e}, plain RR median "
          f"{np.median(e_rr):.3e}, NET better on {int(np.sum(e_net < e_rr))} of {n} jobs")
    b.close()


@pytest.mark.parametrize("inputs", [1, 2])
def test_batch_with_paper_inputs_equals_single_renders(nrrs, inputs):
    """Batched jobs with RRSNet on the NRRS inputs (StatNet first) or on the AID-NRRS
    inputs (its own hash grid), NEE on: every job equals its render alone when the
    per-job factors agree."""
    jobs = [(I.box_scene(1), 24, 16, 3, 6),
            (I.icosphere_room(3, min_triangles=1500, subdiv=2), 20, 12, 4, 5)]
    rng = np.random.default_rng(40 + inputs)
    n_p = nrrs.AID_RRSNET_PARAMS if inputs == 2 else nrrs.RRSNET_PARAMS
    P = (rng.normal(size=n_p) * 0.3).astype(np.float32)
    G = (rng.normal(size=nrrs.GRID_PARAMS) * 0.3).astype(np.float32)
    ref = None

    def setup(handle):
        nrrs.nrrs_set_rrsnet_inputs(handle, inputs)
        nrrs.nrrs_set_rrsnet_params(handle, P)
        if inputs == 2:
            nrrs.nrrs_set_params(handle, nrrs.NET_RRSNET_GRID, G)

    b = nrrs.Batch(jobs)
    setup(b.handle)
    kw = dict(frame=5, update_ref=0, nee=1)
    imgs, st, live, F, sq = b.render(nrrs.RRS_NET, **kw)
    torch.cuda.synchronize()
    assert st["net_evals"] > 0 and st["nonfinite"] == 0
    same = 0
    for j, (scene, W, H, spp, D) in enumerate(jobs):
        sc = nrrs.Scene(scene)
        setup(sc.handle)
        img, rst = sc.render(W, H, spp, D, nrrs.RRS_NET, **kw)
        torch.cuda.synchronize()
        np.testing.assert_allclose(sq[j, :D], rst["sum_q"][:D], rtol=1e-12, atol=0)
        if np.array_equal(F[j, :D], rst["F"][:D]):
            assert torch.equal(imgs[j], img), j
            same += 1
        sc.close()
    assert same >= 1
    b.close()
