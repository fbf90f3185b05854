"""The fused shade + RRSNet kernel against the separate kernels (GPU).

At NET depths on the tensor cores (precision 16: split BF16, 17: BF16) the default render
shades the depth's vertices and runs RRSNet in one kernel, the 16 vertex features going
from registers into shared memory as the first layer's operand; nrrs_set_shade_fusion(0)
writes them to device memory for the separate RRSNet kernel instead.  Both evaluate the
same features with the same MMAs, so images, queue sizes, network evaluations and the
per-depth sums of q must agree bit for bit, with and without next-event estimation, in
stream and graph launches, in NET and NET_MIX modes and in a batched render.  The fused
path must also launch one kernel fewer per NET depth (the sign that it ran)."""
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


def _pair(nrrs, scene, params):
    a, b = nrrs.Scene(scene), nrrs.Scene(scene)
    for s in (a, b):
        s.set_params(params)
    b.set_shade_fusion(0)
    return a, b


def _same(sa, sb, ia, ib):
    assert torch.equal(ia, ib)
    np.testing.assert_array_equal(sa["live"], sb["live"])
    np.testing.assert_array_equal(sa["sum_q"], sb["sum_q"])
    np.testing.assert_array_equal(sa["F"], sb["F"])
    assert sa["net_evals"] == sb["net_evals"] > 0
    assert sa["segments"] == sb["segments"]
    assert sa["status_bits"] == sb["status_bits"] == 0


@pytest.mark.parametrize("precision", [16, 17])
@pytest.mark.parametrize("nee", [0, 1])
def test_fused_net_depths_equal_separate_kernels(nrrs, precision, nee):
    W, H, spp, D = 96, 64, 8, 8
    a, b = _pair(nrrs, I.occluded_room(1), I.rrsnet_init_params(3))
    for frame in range(3):
        for graph in (0, 1):
            ia, sa = a.render(W, H, spp, D, nrrs.RRS_NET, precision=precision, frame=frame,
                              graph=graph, nee=nee)
            ib, sb = b.render(W, H, spp, D, nrrs.RRS_NET, precision=precision, frame=frame,
                              graph=graph, nee=nee)
            torch.cuda.synchronize()
            _same(sa, sb, ia, ib)
            # every depth with a live vertex is a NET depth (the last one too: its shading
            # deposits, and the separate path still launches RRSNet there)
            net_depths = int(np.count_nonzero(sa["live"][:D] > 0))
            assert sb["kernel_launches"] - sa["kernel_launches"] == net_depths
    a.close()
    b.close()


def test_fused_gated_depths_equal_separate_kernels(nrrs):
    """NET_MIX with a gate that alternates NET, HEUR and FIXED depths (2 bits per depth:
    0 NET, 1 HEUR, 2 FIXED)."""
    W, H, spp, D = 80, 48, 4, 10
    gate = 0
    for d in range(D):
        gate |= (d % 3) << (2 * d)
    a, b = _pair(nrrs, I.box_scene(4), I.rrsnet_init_params(8))
    for frame in range(2):
        ia, sa = a.render(W, H, spp, D, nrrs.RRS_NET_MIX, precision=16, frame=frame, gate=gate)
        ib, sb = b.render(W, H, spp, D, nrrs.RRS_NET_MIX, precision=16, frame=frame, gate=gate)
        torch.cuda.synchronize()
        _same(sa, sb, ia, ib)
        net_depths = sum(1 for d in range(D) if d % 3 == 0 and sa["live"][d] > 0)
        assert sb["kernel_launches"] - sa["kernel_launches"] == net_depths
    a.close()
    b.close()


def test_fused_batched_render_equals_separate_kernels(nrrs):
    jobs = I.uneven_jobs(seed=2, n_jobs=6, tri_range=(1_000, 4_000), side_log2=(5, 6),
                         spp_range=(1, 4), depth_range=(4, 8))
    params = I.rrsnet_init_params(9)
    out = []
    for fuse in (1, 0):
        bt = nrrs.Batch(jobs)
        bt.set_params(params)
        nrrs.nrrs_set_shade_fusion(bt.handle, fuse)
        imgs, st, live, F, sq = bt.render(nrrs.RRS_NET, precision=17)
        torch.cuda.synchronize()
        out.append(([i.clone() for i in imgs], st, np.array(live), np.array(F), np.array(sq)))
        bt.close()
    (ia, sa, la, Fa, qa), (ib, sb, lb, Fb, qb) = out
    assert all(torch.equal(x, y) for x, y in zip(ia, ib))
    np.testing.assert_array_equal(la, lb)
    np.testing.assert_array_equal(Fa, Fb)
    np.testing.assert_array_equal(qa, qb)
    assert sa["net_evals"] == sb["net_evals"] > 0
    assert sa["segments"] == sb["segments"]
