"""What the trained network gains (GPU): after online training (Sec. 4 "Training"),
RRSNet's normalised RRS has a lower relMSE than the same network untrained and than plain
heuristic normalised RRS, at equal samples and against the same high-spp no-RRS
reference; the Mix-Depth gate searched with the trained network is at least as efficient
as the heuristic (Sec. 3.3).  Measured on the occluded room, where light reaches the
camera's side only through a slot, so where paths go matters."""
import numpy as np
import pytest

from paper_2510_07868_b300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

W = H = 128
SPP, D = 16, 12


@pytest.fixture(scope="module")
def nrrs():
    from paper_2510_07868_b300 import nrrs as m

    assert torch.cuda.is_available()
    return m


def _relmse(a, b):
    a = a.double()
    b = b.double()
    return float(torch.mean((a - b) ** 2 / (b * b + 0.01)))


def _mean_frames(sc, nrrs, mode, frames, first, **kw):
    acc = torch.zeros((H, W, 3), dtype=torch.float64, device="cuda")
    segs = 0
    for f in range(frames):
        img, st = sc.render(W, H, SPP, D, mode, frame=first + f, update_ref=0, **kw)
        acc += img.double()
        segs += st["segments"]
    return (acc / frames).float(), segs


def test_trained_rrsnet_beats_untrained_and_heuristic(nrrs):
    s = I.occluded_room(1)
    sc = nrrs.Scene(s)
    sc.set_params(I.rrsnet_init_params(1))
    ref, _ = _mean_frames(sc, nrrs, nrrs.RRS_NONE, 128, 50_000)
    # untrained network, same frames
    untrained, _ = _mean_frames(sc, nrrs, nrrs.RRS_NET, 16, 90_000)
    # online training: training steps interleaved with frames that build the reference
    for k in range(200):
        st = sc.train_step(width=W, height=H, spp=2, max_depth=D, frame=k)
        assert np.isfinite(st["loss_rrsnet"])
        sc.render(W, H, SPP, D, nrrs.RRS_NET, frame=20_000 + k)
    assert st["phase"] == 2
    trained, segs_net = _mean_frames(sc, nrrs, nrrs.RRS_NET, 16, 90_000)
    heur, segs_heur = _mean_frames(sc, nrrs, nrrs.RRS_HEUR_NORM, 16, 90_000)
    e_untrained = _relmse(untrained, ref)
    e_trained = _relmse(trained, ref)
    e_heur = _relmse(heur, ref)
    print(f"relMSE: untrained NET {e_untrained:.4f}, trained NET {e_trained:.4f} "
          f"({segs_net} segments), HEUR_NORM {e_heur:.4f} ({segs_heur} segments)")
    assert e_trained < 0.9 * e_untrained
    assert e_trained < 0.9 * e_heur
    # Mix-Depth with the trained network: relMSE x segments no worse than the heuristic's
    g = nrrs.nrrs_mixdepth_search(sc.handle, W, H, D, t_d=6, frame=777)
    mix, segs_mix = _mean_frames(sc, nrrs, nrrs.RRS_NET_MIX, 16, 90_000, gate=g["gate"])
    e_mix = _relmse(mix, ref)
    print(f"Mix-Depth {nrrs.gate_methods(g['gate'], D)}: relMSE {e_mix:.4f}, {segs_mix} segments")
    assert e_mix * segs_mix <= 1.05 * e_heur * segs_heur
    sc.close()
