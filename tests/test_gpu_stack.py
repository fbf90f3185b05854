"""The BVH2 traversal with its short and its long stack (GPU).

A ray holds at most one pushed sibling per inner node on its current path, so a tree
whose height (most inner nodes on a root-to-leaf path) is at most 24 is traversed with a
24-entry stack by default, otherwise with the 40-entry one.  Both must find the same
closest hits, so renders with either stack are bit-identical (the oracle parity of the
default, short-stack path is in the other render tests)."""
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


@pytest.mark.parametrize("make", [lambda: I.box_scene(2), lambda: I.occluded_room(3),
                                  lambda: I.icosphere_room(4, min_triangles=20_000)])
def test_short_and_long_stack_render_identically(nrrs, make):
    scene = make()
    sc = nrrs.Scene(scene)
    sc.set_params(I.rrsnet_init_params(2))
    h, e = sc.traversal_stack_info()
    assert 1 <= h <= 24 and e == 24, (h, e)
    W, H, spp, D = 64, 48, 4, 8
    imgs = {}
    for entries in (0, 40, 24):
        sc.set_traversal_stack(entries)
        assert sc.traversal_stack_info()[1] == (40 if entries == 40 else 24)
        out = []
        for nee in (0, 1):
            for graph in (0, 1):
                img, st = sc.render(W, H, spp, D, nrrs.RRS_HEUR_NORM, frame=5, nee=nee,
                                    graph=graph, update_ref=0)
                torch.cuda.synchronize()
                assert st["status_bits"] == 0
                out.append((img.clone(), np.array(st["live"])))
        imgs[entries] = out
    for entries in (40, 24):
        for (a, la), (b, lb) in zip(imgs[0], imgs[entries]):
            assert torch.equal(a, b)
            np.testing.assert_array_equal(la, lb)
    sc.close()


def test_stack_request_validation(nrrs):
    sc = nrrs.Scene(I.box_scene(1))
    for bad in (-1, 1, 23, 25, 39, 41):
        with pytest.raises(nrrs.NrrsError):
            sc.set_traversal_stack(bad)
    sc.set_traversal_stack(0)
    assert sc.traversal_stack_info()[1] == 24
    sc.close()
