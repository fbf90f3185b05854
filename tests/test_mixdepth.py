"""Mix-Depth (Sec. 3.3): candidate counts (CPU) and the search's choice (GPU)."""
import numpy as np
import pytest

import oracle
from paper_2510_07868_b300 import inputs as I
from tests.conftest import paper_constant


def test_candidate_counts_match_paper():
    from paper_2510_07868_b300 import nrrs

    assert nrrs.nrrs_mixdepth_candidates(6, 6) == paper_constant("mixdepth_bruteforce_d6")
    assert nrrs.nrrs_mixdepth_candidates(10, 10) == paper_constant("mixdepth_bruteforce_d10")
    assert nrrs.nrrs_mixdepth_candidates(10, 6) == paper_constant("mixdepth_heuristic_td6_d10")
    assert nrrs.nrrs_mixdepth_candidates(16, 6) == 729 + 729 + 81
    assert nrrs.nrrs_mixdepth_candidates(0, 6) == -1 and nrrs.nrrs_mixdepth_candidates(4, 0) == -1


def test_relmse_oracle_closed_form():
    ref = np.array([1.0, 0.0, 2.0])
    img = np.array([2.0, 0.1, 2.0])
    assert oracle.relmse(img, ref, 0.01) == pytest.approx((1 / 1.01 + 0.01 / 0.01 + 0) / 3)


@pytest.mark.gpu
def test_relmse_matches_oracle():
    import torch

    from paper_2510_07868_b300 import nrrs

    rng = np.random.default_rng(1)
    n = 70_001
    img = rng.uniform(0, 3, (n, 3)).astype(np.float32)
    ref = rng.uniform(0, 3, (n, 3)).astype(np.float32)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    nrrs.nrrs_relmse(torch.from_numpy(img).cuda(), torch.from_numpy(ref).cuda(), n, 0.01, out)
    torch.cuda.synchronize()
    # the GPU sums in FP32 (compensated per thread, then a tree over 1024 threads): each
    # term (i - r)^2 / (r^2 + eps) carries at most 4 roundings (4 u, u = 2^-24) and the
    # tree 10 more, so the mean is within 14 u < 1e-6 relative of the FP64 oracle's
    assert out.item() == pytest.approx(oracle.relmse(img, ref, 0.01), rel=1e-6)


@pytest.mark.gpu
@pytest.mark.parametrize("D,t_d,adrrs", [(3, 3, 0), (4, 2, 0), (4, 2, 1)])
def test_search_returns_the_argmin(D, t_d, adrrs):
    """The search's gate is the lowest relMSE x segments among the candidates it may
    visit, found here by rendering every candidate through the public API."""
    import torch

    from paper_2510_07868_b300 import nrrs

    s = nrrs.Scene(I.box_scene(1))
    s.set_params(I.rrsnet_init_params(1))
    W = H = 32
    ref = torch.zeros((H, W, 3), device="cuda")
    acc = None
    for f in range(16):  # reference: mean of 16 plain frames at 8 spp
        img, _ = s.render(W, H, 8, D, nrrs.RRS_NONE, frame=100 + f, update_ref=0)
        acc = img.clone() if acc is None else acc + img
    ref.copy_(acc / 16)
    if adrrs:  # StatNet with a non-negative output layer, as after some training
        sp = np.random.default_rng(5).normal(size=nrrs.STATNET_PARAMS).astype(np.float32) * 0.3
        sp[-6 * 32:] = np.abs(sp[-6 * 32:])
        nrrs.nrrs_set_params(s.handle, nrrs.NET_STATNET, sp)
    res = nrrs.nrrs_mixdepth_search(s.handle, W, H, D, t_d=t_d, frame=7, d_pixel_ref=ref,
                                    adrrs=adrrs)
    assert res["evaluated"] == nrrs.nrrs_mixdepth_candidates(D, t_d)
    order = [nrrs.GATE_FIXED, nrrs.GATE_ADRRS if adrrs else nrrs.GATE_HEUR, nrrs.GATE_NET]
    gate = sum(nrrs.GATE_FIXED << (2 * d) for d in range(D))
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for start in range(0, D, t_d):
        length = min(t_d, D - start)
        best, best_g = np.inf, None
        for c in range(3 ** length):
            g, x = gate, c
            for k in range(length):
                g &= ~(3 << (2 * (start + k)))
                g |= order[x % 3] << (2 * (start + k))
                x //= 3
            img, st = s.render(W, H, 1, D, nrrs.RRS_NET_MIX, gate=g, frame=7, update_ref=0,
                               d_pixel_ref=ref.data_ptr())
            nrrs.nrrs_relmse(img, ref, W * H, 0.01, out)
            torch.cuda.synchronize()
            score = out.item() * st["segments"]
            if score < best:
                best, best_g = score, g
        gate = best_g
    assert res["gate"] == gate
    assert res["score"] == pytest.approx(best, rel=1e-12)
    s.close()
