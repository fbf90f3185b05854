"""The spatial filter of the training error map (GPU), against its definition written
out in numpy, and its schedule in the training step (Sec. 4 "Tackle Low Spp": a
normal-guided denoiser that is turned off for the last part of training)."""
import numpy as np
import pytest

from paper_2510_07868_b300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def nrrs():
    from paper_2510_07868_b300 import nrrs as m

    assert torch.cuda.is_available()
    return m


def _filter_reference(E, N, W, H, r, power):
    out = np.zeros(W * H)
    for p in range(W * H):
        x, y = p % W, p // W
        s = c = 0.0
        for yy in range(max(0, y - r), min(H - 1, y + r) + 1):
            for xx in range(max(0, x - r), min(W - 1, x + r) + 1):
                q = yy * W + xx
                w = 1.0
                if N is not None and N[p, 3] > 0 and q != p:
                    d = float(np.dot(N[p, :3].astype(np.float64), N[q, :3].astype(np.float64)))
                    w = d ** power if (N[q, 3] > 0 and d > 0) else 0.0
                s += w * E[q]
                c += w
        out[p] = s / c
    return out


@pytest.mark.parametrize("guided,power", [(False, 8.0), (True, 8.0), (True, 5.0), (True, 2.5)])
def test_error_filter_matches_definition(nrrs, guided, power):
    """Integral powers take repeated squaring, others pow; both against the definition."""
    W, H, r = 37, 23, 2
    rng = np.random.default_rng(5)
    E = rng.exponential(size=W * H).astype(np.float32)
    N = None
    if guided:
        n = rng.normal(size=(W * H, 3))
        n[: W * H // 2] = [0.0, 1.0, 0.0]  # a flat half: neighbours agree
        n /= np.linalg.norm(n, axis=1, keepdims=True)
        N = np.concatenate([n, (rng.random((W * H, 1)) > 0.1)], axis=1).astype(np.float32)
    dE = torch.from_numpy(E).cuda()
    dN = torch.from_numpy(N).cuda() if guided else None
    out = torch.empty_like(dE)
    nrrs.nrrs_error_filter(dE, dN, W, H, r, power if guided else 0.0, out)
    torch.cuda.synchronize()
    ref = _filter_reference(E, N, W, H, r, power)
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=2e-6, atol=0)
    # radius 0 copies
    nrrs.nrrs_error_filter(dE, dN, W, H, 0, power, out)
    torch.cuda.synchronize()
    assert torch.equal(out, dE)


def test_training_turns_the_filter_off_on_schedule(nrrs):
    """With error_filter_until = 2 the first two steps run the normal pass and the filter
    (two more kernel launches) and later steps do not."""
    sc = nrrs.Scene(I.occluded_room(1, n_random=300))
    sc.set_params(I.rrsnet_init_params(1))
    sc.render(64, 64, 4, 8, nrrs.RRS_HEUR_NORM)
    n = [sc.train_step(width=64, height=64, spp=2, max_depth=8, error_filter_until=2,
                       warmup_steps=0)["kernel_launches"] for _ in range(4)]
    assert n[0] == n[1] and n[2] == n[3] and n[0] - n[2] == 2, n
    sc.close()
