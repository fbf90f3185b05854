"""Full-size parity cases beyond the bench workload (GPU): the RRSNet precision sweep on
the 200k-triangle icosphere room (1024 x 1024 px, 64 spp, depth 24) and the Mix-Depth
frame sequence on the 1M-triangle three-room scene (1920 x 1080 px, 8 frames of 16 spp,
depth 32, tuned RRSNet shapes, graph-captured bounce loop).

The oracle cannot render these frames whole, so it renders 256 sampled pixels one by
one: with normalisation, pixels interact only through each depth's factor F, which the
oracle takes from the GPU frame's stats (its own F is checked at small sizes elsewhere).
Both sides trace the sampled pixels' decisions (the GPU through a pixel mask into compact
rows); pixels whose decisions all match are held to the FP32 bar, 1e-5 relative for paths
of up to 3 bounces and 50 u per bounce beyond (u = 2^-24: each bounce's FP32 throughput
update carries about 50 roundings), and the share of path vertices on which both sides
agree is reported per depth."""
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


def _relmse(a, b):
    """Sec. 5's relMSE of image a against reference b (mean over pixels and channels)."""
    a = a.astype(np.float64)
    b = b.astype(np.float64)
    return float(np.mean((a - b) ** 2 / (b * b + 0.01)))


def _frame_properties(st, C, D):
    live = st["live"][:D]
    assert st["capacity"] == C and np.all(live <= C)
    for d in range(D - 1):
        assert live[d + 1] == min(st["requested"][d], C)
    assert np.all((st["F"][:D] > 0) & (st["F"][:D] <= 1)) and st["nonfinite"] == 0
    assert st["status_bits"] == 0  # no drops, no non-finite factors, no bounded wait ran out


def _masked_trace_render(nrrs, sc, W, H, spp, D, mode, pix, **opts):
    """A frame with the decisions of the sampled pixels traced (compact rows of depth,
    pixel, sample, lineage, triangle, X); returns (image, stats, rows)."""
    mask = torch.zeros(W * H, dtype=torch.uint8, device="cuda")
    mask[torch.from_numpy(pix.astype(np.int64)).cuda()] = 1
    rows = len(pix) * spp * D * 8
    tr = torch.zeros((rows, 6), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    img, st = sc.render(W, H, spp, D, mode, d_trace=tr.data_ptr(), d_trace_mask=mask.data_ptr(),
                        d_trace_count=cnt.data_ptr(), trace_rows=rows, **opts)
    torch.cuda.synchronize()
    n = int(cnt.item())
    assert n <= rows, (n, rows)
    return img.cpu().numpy(), st, tr[:n].cpu().numpy().view(np.uint32)


U32 = 2.0 ** -24


def _pixel_bar(d_max):
    """Relative error bar of a pixel whose decisions all match, from its deepest vertex:
    each bounce carries an FP32 throughput update t w / q_used (the BSDF weight and the FP32
    RRSNet factor, about 50 roundings) against the oracle's FP64, so the error grows with
    the path length: max(1e-5, 50 u d_max), u = 2^-24 (1e-5 up to depth 3)."""
    return np.maximum(1e-5, 50.0 * U32 * d_max)


def _sampled_pixel_match(s, W, H, spp, D, mode, P, img, st, rows, pix, **kw):
    """The oracle renders the sampled pixels one by one (the GPU frame's per-depth F forced,
    since it depends on the whole frame) with its decisions traced.  Returns the fraction of
    sampled pixels whose decision multisets (per path vertex: depth, sample, lineage,
    triangle, X) equal the GPU's, their relative errors and bars, the match mask, and per
    depth the share of vertices (pixel, sample, lineage) that both sides reach with the
    same triangle and X."""
    oimg, _, otr = oracle.render(s, W, H, spp, D, mode, params=P.astype(np.float64), pixels=pix,
                                 forced_F=st["F"][:D], trace=True, **kw)
    gdec = {int(p): [] for p in pix}
    for r in rows:
        gdec[int(r[1])].append((int(r[0]) - 1, int(r[2]), int(r[3]), int(r[4]), int(r[5])))
    odec = {int(p): [] for p in pix}
    for d, tr in enumerate(otr):
        for r in tr:
            odec[int(r[0])].append((d, int(r[1]), int(r[2]), int(r[3]), int(r[4])))
    match = np.array([sorted(gdec[int(p)]) == sorted(odec[int(p)]) for p in pix])
    d_max = np.array([max((v[0] for v in odec[int(p)]), default=0) + 1 for p in pix])
    g = img.reshape(-1, 3)[pix].astype(np.float64)
    o = oimg.reshape(-1, 3)[pix]
    rel = np.max(np.abs(g - o) / np.maximum(np.abs(o), 1e-30), axis=1)
    rel[np.all(o == 0, axis=1) & np.all(g == 0, axis=1)] = 0.0
    # per-depth agreement of the vertices (keyed by pixel, sample and lineage)
    agree = []
    for d in range(D):
        gs = {(p, v[1], v[2]): v[3:] for p in gdec for v in gdec[p] if v[0] == d}
        os_ = {(p, v[1], v[2]): v[3:] for p in odec for v in odec[p] if v[0] == d}
        keys = set(gs) | set(os_)
        if not keys:
            break
        agree.append(sum(1 for k in keys if gs.get(k) == os_.get(k)) / len(keys))
    return (float(match.mean()), rel[match], _pixel_bar(d_max[match]), match,
            np.array(agree))


def _sample_pixels(img, n, seed):
    """n sampled pixels, half of them lit (as many as the frame has), the rest dark."""
    lum = img.reshape(-1, 3).max(axis=1)
    lit = np.flatnonzero(lum > 0)
    dark = np.flatnonzero(lum == 0)
    rng = np.random.default_rng(seed)
    n_lit = min(n // 2, lit.size)
    pick = [rng.choice(lit, n_lit, replace=False)] if n_lit else []
    pick.append(rng.choice(dark, n - n_lit, replace=False))
    return np.sort(np.concatenate(pick)).astype(np.int32), n_lit


def test_precision_sweep_icosphere_room_full_size(nrrs):
    s = I.icosphere_room(1)
    assert s.n_tri >= 200_000
    W = H = 1024
    spp, D = 64, 24
    C = 2 * W * H * spp
    P = I.rrsnet_init_params(1)
    sc = nrrs.Scene(s)
    sc.set_params(P)
    imgs, stats = {}, {}
    for prec in (32, 16, 8):
        img, st = sc.render(W, H, spp, D, nrrs.RRS_NET, precision=prec, frame=0, update_ref=0)
        torch.cuda.synchronize()
        _frame_properties(st, C, D)
        imgs[prec] = img.cpu().numpy()
        stats[prec] = st
        assert np.isfinite(imgs[prec]).all() and imgs[prec].min() >= 0
    # noise floor: the FP32 frame against an independent FP32 frame (other random numbers)
    other, _ = sc.render(W, H, spp, D, nrrs.RRS_NET, precision=32, frame=1, update_ref=0)
    floor = _relmse(other.cpu().numpy(), imgs[32])
    r16 = _relmse(imgs[16], imgs[32])
    r8 = _relmse(imgs[8], imgs[32])
    # split BF16 factors are within 1e-4 of FP32: a few decisions flip, far below the floor
    assert r16 <= 0.05 * floor, (r16, floor)
    # E4M3 factors move ~1 %: more flips, still no more than an independent frame
    assert r8 <= floor, (r8, floor)
    # FP64 oracle on 256 sampled pixels (half lit) of an FP32 frame with their decisions
    # traced on both sides: pixels whose decisions all match must agree to 1e-5 relative
    # (the FP32 path on identical decisions)
    pix, n_lit = _sample_pixels(imgs[32], 256, 3)
    img, st, rows = _masked_trace_render(nrrs, sc, W, H, spp, D, nrrs.RRS_NET, pix, precision=32,
                                         frame=0, update_ref=0)
    np.testing.assert_array_equal(img, imgs[32])  # tracing changes nothing
    frac, rel, bar, match, agree = _sampled_pixel_match(s, W, H, spp, D, oracle.MODE_NET, P, img,
                                                        st, rows, pix)
    print(f"precision sweep: relMSE vs FP32 bf16 {r16:.3e} e4m3 {r8:.3e} floor {floor:.3e}; "
          f"{n_lit} lit of 256 sampled pixels, decisions match on {frac:.3f}, "
          f"max rel error there {rel.max() if rel.size else 0:.2e} (max rel / bar "
          f"{(rel / bar).max() if rel.size else 0:.2f}); vertex agreement per depth "
          f"{np.array2string(agree, precision=3)}")
    assert frac >= 0.7 and match.sum() >= 150, frac
    assert np.all(rel <= bar), np.sort(rel / bar)[-5:]
    assert agree[0] >= 0.99 and np.all(agree[:4] >= 0.95), agree
    sc.close()


def test_mix_depth_three_rooms_full_size(nrrs):
    s = I.three_rooms(1)
    assert s.n_tri >= 1_000_000
    W, H = 1920, 1080
    spp, D, frames = 16, 32, 8
    C = 2 * W * H * spp
    P = I.rrsnet_init_params(2)
    gate = 0
    for d in range(D):  # FIXED, FIXED, then NET through depth 8, HEUR beyond
        g = nrrs.GATE_FIXED if d < 2 else nrrs.GATE_NET if d < 8 else nrrs.GATE_HEUR
        gate |= g << (2 * d)
    sc = nrrs.Scene(s)
    sc.set_params(P)
    sc.tune(32)
    acc = None
    lit_per_frame = []
    for f in range(frames):
        img, st = sc.render(W, H, spp, D, nrrs.RRS_NET_MIX, gate=gate, frame=f, graph=1)
        torch.cuda.synchronize()
        _frame_properties(st, C, D)
        assert st["net_evals"] > 0
        a = img.cpu().numpy().astype(np.float64)
        lit_per_frame.append(int(np.count_nonzero(a.max(axis=2))))
        acc = a if acc is None else acc + a
    final = acc / frames
    assert np.isfinite(final).all() and final.min() >= 0 and final.max() > 0
    # one more frame against an explicit reference (the mean of the 8 frames) that the
    # oracle is handed too: its HEUR depths then see the same I_px on both sides
    ref = final.astype(np.float32)
    img, st = sc.render(W, H, spp, D, nrrs.RRS_NET_MIX, gate=gate, frame=frames, graph=1,
                        d_pixel_ref=torch.from_numpy(ref).cuda().data_ptr(), update_ref=0)
    torch.cuda.synchronize()
    _frame_properties(st, C, D)
    img = img.cpu().numpy()
    lit = int(np.count_nonzero(img.reshape(-1, 3).max(axis=1)))
    print(f"mix-depth: lit pixels per frame {lit_per_frame}, checked frame {lit}")
    assert lit >= 8  # light from room 3 reaches the camera
    # 256 sampled pixels (half lit, as far as the frame has lit pixels), decisions traced on
    # both sides: decision-matched pixels must agree to 1e-5 relative
    pix, n_lit = _sample_pixels(img, 256, 5)
    dref = torch.from_numpy(ref).cuda()
    img2, st2, rows = _masked_trace_render(nrrs, sc, W, H, spp, D, nrrs.RRS_NET_MIX, pix, gate=gate,
                                           frame=frames, graph=1, d_pixel_ref=dref.data_ptr(),
                                           update_ref=0)
    np.testing.assert_array_equal(img2, img)  # the same frame, traced
    frac, rel, bar, match, agree = _sampled_pixel_match(s, W, H, spp, D, oracle.MODE_NET_MIX, P,
                                                        img2, st2, rows, pix, gate=gate,
                                                        pixel_ref=ref.astype(np.float64),
                                                        frame=frames)
    lit_match = float(match[np.isin(pix, np.flatnonzero(img.reshape(-1, 3).max(axis=1) > 0))].mean())
    print(f"mix-depth: {n_lit} lit of 256 sampled pixels; decisions match on {frac:.3f} "
          f"(lit {lit_match:.3f}), max rel error there {rel.max() if rel.size else 0:.2e}; "
          f"vertex agreement per depth {np.array2string(agree, precision=3)}")
    # a path through the dust (random triangles of size 0.01, mean free path ~0.1) is a
    # chaotic billiard: the FP32 and FP64 hit points differ by ~1e-7 and the difference
    # grows with every bounce until one side hits another triangle, so whole-pixel
    # agreement falls with depth (the lit pixels' paths are the deepest).  The early
    # depths must agree; pixels whose decisions all match are held to their bar
    assert agree[0] >= 0.99 and np.all(agree[:4] >= 0.9), agree
    assert match.sum() >= 50, frac
    assert np.all(rel <= bar), np.sort(rel / bar)[-5:]
    sc.close()
