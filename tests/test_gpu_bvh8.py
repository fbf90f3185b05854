"""The compressed eight-wide BVH built on the device (GPU).

The tree (nrrs_set_traversal(8)) is exported and checked on the CPU: every triangle is
stored exactly once with the same vertices, the tree reaches every node once, every
decoded child box (origin + byte x power-of-two scale per plane) contains what is
below it, and its depth fits the traversal stack.  Renders through it must equal the
BVH2's bit for bit: the closest hit (with the lower-id tie rule) does not depend on the
tree, so images, traced decisions and next-event shadow rays are identical."""
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


def _decode(nodes):
    """Per node: origin [n][3], scale [n][3], inner mask [n], first child [n], first
    triangle [n], meta [n][8], lo/hi bytes [n][3][8]."""
    p = nodes[:, 0:3].view(np.float32).astype(np.float64)
    w = nodes[:, 3]
    ex = (w & 0xFF).astype(np.int64), ((w >> 8) & 0xFF).astype(np.int64), ((w >> 16) & 0xFF).astype(np.int64)
    scale = np.stack([np.ldexp(1.0, e - 127) for e in ex], axis=1)
    imask = (w >> 24).astype(np.int64)
    child = nodes[:, 4].astype(np.int64)
    tri0 = nodes[:, 5].astype(np.int64)
    meta = nodes[:, 6:8].copy().view(np.uint8).reshape(-1, 8).astype(np.int64)
    b = nodes[:, 8:20].copy().view(np.uint8).reshape(-1, 6, 8).astype(np.float64)
    return p, scale, imask, child, tri0, meta, b[:, 0:3], b[:, 3:6]


def _check_tree(nrrs, sc, scene):
    """Structure and conservativeness of the exported tree.  Every decoded slot box must
    contain the geometry below it (its leaf triangles, or everything under its child
    node); the boxes of a child node need not nest inside its parent's slot box, since
    each level rounds outward on its own grid."""
    info = nrrs.nrrs_bvh8_info(sc.handle)
    n_tri = scene.n_tri
    assert info["triangles"] == n_tri and info["nodes"] >= 1
    assert 1 <= info["depth"] <= 40
    nodes, tris = nrrs.nrrs_bvh8_export(sc.handle)
    # every triangle once, with the input vertices (v0 exact, edges as FP32 differences)
    ids = tris[:, 3].view(np.uint32).astype(np.int64)
    assert np.array_equal(np.sort(ids), np.arange(n_tri))
    src = scene.tri.reshape(-1, 9).astype(np.float32)[ids]
    np.testing.assert_array_equal(tris[:, 0:3], src[:, 0:3])
    np.testing.assert_array_equal(tris[:, 4:7], src[:, 3:6] - src[:, 0:3])
    np.testing.assert_array_equal(tris[:, 8:11], src[:, 6:9] - src[:, 0:3])
    assert np.array_equal(tris[:, 7].view(np.int32), np.asarray(scene.mat_id, np.int32)[ids])
    p, scale, imask, child, tri0, meta, qlo, qhi = _decode(nodes)
    n = nodes.shape[0]
    lo = p[:, :, None] + qlo * scale[:, :, None]  # decoded slot boxes, exact in FP64
    hi = p[:, :, None] + qhi * scale[:, :, None]
    # the triangles' corners as the traversal's Moller-Trumbore sees them (v0 + e)
    v0 = tris[:, 0:3].astype(np.float64)
    corners = np.stack([v0, v0 + tris[:, 4:7], v0 + tris[:, 8:11]], axis=1)
    t_lo, t_hi = corners.min(axis=1), corners.max(axis=1)
    popc = np.array([bin(v).count("1") for v in range(256)], dtype=np.int64)
    kid = np.stack([child + popc[imask & ((1 << s) - 1)] for s in range(8)], axis=1)
    inner = np.stack([(imask >> s) & 1 == 1 for s in range(8)], axis=1)
    leaf = (~inner) & (meta != 0)
    assert np.all(kid[inner] < n) and np.all(kid[inner] > np.nonzero(inner)[0])
    # every node reached once from the root; every triangle in exactly one leaf slot
    seen = np.zeros(n, dtype=np.int64)
    seen[0] = 1
    np.add.at(seen, kid[inner], 1)
    assert np.all(seen == 1)
    cnt, off = meta >> 5, meta & 31
    assert np.all((cnt[leaf] >= 1) & (cnt[leaf] <= 3))
    owner = np.zeros(n_tri, dtype=np.int64)
    for j in range(3):
        sel = leaf & (cnt > j)
        np.add.at(owner, (tri0[:, None] + off + j)[sel], 1)
    assert np.all(owner == 1)
    # geometric boxes bottom-up (children have higher indices than their parents)
    g_lo = np.full((n, 3), np.inf)
    g_hi = np.full((n, 3), -np.inf)
    slot_lo = np.full((n, 8, 3), np.inf)
    slot_hi = np.full((n, 8, 3), -np.inf)
    for j in range(3):  # leaf slots: their triangles
        sel = leaf & (cnt > j)
        r = (tri0[:, None] + off + j)
        slot_lo[sel] = np.minimum(slot_lo[sel], t_lo[r[sel]])
        slot_hi[sel] = np.maximum(slot_hi[sel], t_hi[r[sel]])
    level_of = np.zeros(n, dtype=np.int64)
    frontier, L = np.array([0]), 0
    while frontier.size:  # levels top-down
        frontier = kid[frontier][inner[frontier]]
        L += 1
        level_of[frontier] = L
    for L in range(level_of.max(), -1, -1):
        nodes_L = np.flatnonzero(level_of == L)
        ii = inner[nodes_L]
        kk = kid[nodes_L]
        sl = slot_lo[nodes_L]
        sh = slot_hi[nodes_L]
        sl[ii] = g_lo[kk[ii]]
        sh[ii] = g_hi[kk[ii]]
        slot_lo[nodes_L] = sl
        slot_hi[nodes_L] = sh
        g_lo[nodes_L] = sl.min(axis=1)
        g_hi[nodes_L] = sh.max(axis=1)
    used = inner | leaf
    dl = np.transpose(lo, (0, 2, 1))  # [n][8][3]
    dh = np.transpose(hi, (0, 2, 1))
    assert np.all(dl[used] <= slot_lo[used]) and np.all(dh[used] >= slot_hi[used])
    return info


@pytest.mark.parametrize("name", ["box", "occluded_room", "icosphere_room", "three_rooms"])
def test_bvh8_tree_is_valid(nrrs, name):
    scene = {"box": lambda: I.box_scene(1), "occluded_room": lambda: I.occluded_room(1),
             "icosphere_room": lambda: I.icosphere_room(1),
             "three_rooms": lambda: I.three_rooms(1)}[name]()
    sc = nrrs.Scene(scene)
    sc.set_traversal(8)
    info = _check_tree(nrrs, sc, scene)
    print(f"{name}: {scene.n_tri} triangles, {info['nodes']} nodes, depth {info['depth']}, "
          f"{info['iterations']} clustering rounds, build {info['build_ms']:.1f} ms")
    sc.close()


def _render_both(nrrs, scene, W, H, spp, D, mode, trace=False, **opts):
    out = {}
    for width in (2, 8):
        sc = nrrs.Scene(scene)
        sc.set_params(I.rrsnet_init_params(1))
        sc.set_traversal(width)
        tr = None
        kw = dict(opts)
        if trace:
            tr = torch.zeros((D, 2 * W * H * spp, 5), dtype=torch.int32, device="cuda")
            kw["d_trace"] = tr.data_ptr()
        img, st = sc.render(W, H, spp, D, mode, **kw)
        torch.cuda.synchronize()
        out[width] = (img.cpu().numpy(), st, tr.cpu().numpy() if trace else None)
        sc.close()
    return out


@pytest.mark.parametrize("mode_name,nee", [("NET", 0), ("HEUR_NORM", 1), ("NONE", 0)])
def test_bvh8_renders_equal_the_bvh2(nrrs, mode_name, nee):
    mode = getattr(nrrs, "RRS_" + mode_name)
    for scene, W, H, spp, D in ((I.box_scene(1), 48, 40, 4, 8),
                                (I.occluded_room(1), 64, 64, 4, 12)):
        out = _render_both(nrrs, scene, W, H, spp, D, mode, trace=True, nee=nee, graph=1)
        np.testing.assert_array_equal(out[8][0], out[2][0])
        np.testing.assert_array_equal(out[8][2], out[2][2])
        assert np.array_equal(out[8][1]["live"], out[2][1]["live"])


def test_bvh8_full_size_scenes_render_identically(nrrs):
    for scene, W, H, spp, D, mode in ((I.icosphere_room(1), 512, 512, 4, 24, nrrs.RRS_NET),
                                      (I.three_rooms(1), 960, 540, 4, 32, nrrs.RRS_HEUR_NORM)):
        out = _render_both(nrrs, scene, W, H, spp, D, mode, graph=1)
        assert out[2][1]["segments"] > 0
        np.testing.assert_array_equal(out[8][0], out[2][0])
        assert out[8][1]["segments"] == out[2][1]["segments"]


def _render_builders(nrrs, scene, W, H, spp, D, mode, trace=False, **opts):
    out = {}
    for builder in (0, 1):
        sc = nrrs.Scene(scene)
        sc.set_params(I.rrsnet_init_params(1))
        if builder:
            ms = sc.set_bvh_builder(1)
            assert ms > 0.0
        tr = None
        kw = dict(opts)
        if trace:
            tr = torch.zeros((D, 2 * W * H * spp, 5), dtype=torch.int32, device="cuda")
            kw["d_trace"] = tr.data_ptr()
        img, st = sc.render(W, H, spp, D, mode, **kw)
        torch.cuda.synchronize()
        out[builder] = (img.cpu().numpy(), st, tr.cpu().numpy() if trace else None,
                        nrrs.nrrs_scene_info(sc.handle)[0])
        sc.close()
    return out


@pytest.mark.parametrize("mode_name,nee", [("NET", 0), ("HEUR_NORM", 1)])
def test_device_built_bvh2_renders_equal_the_host_tree(nrrs, mode_name, nee):
    """The PLOC BVH2 (nrrs_set_bvh_builder(1)) and the host SAH tree give identical
    closest hits, so identical images and traced decisions, through the FP16 and the FP32
    boxes alike."""
    mode = getattr(nrrs, "RRS_" + mode_name)
    for scene, W, H, spp, D in ((I.box_scene(1), 48, 40, 4, 8),
                                (I.occluded_room(1), 64, 64, 4, 12)):
        out = _render_builders(nrrs, scene, W, H, spp, D, mode, trace=True, nee=nee, graph=1)
        np.testing.assert_array_equal(out[1][0], out[0][0])
        np.testing.assert_array_equal(out[1][2], out[0][2])
        # one triangle per PLOC leaf: n - 1 inner nodes
        assert out[1][3] == scene.n_tri - 1


def test_device_built_bvh2_full_size_and_switching(nrrs):
    scene = I.three_rooms(1)
    out = _render_builders(nrrs, scene, 960, 540, 4, 32, nrrs.RRS_HEUR_NORM, graph=1)
    np.testing.assert_array_equal(out[1][0], out[0][0])
    assert out[1][1]["segments"] == out[0][1]["segments"] > 0
    # switching back to the host tree, after a captured graph, reproduces the first image
    sc = nrrs.Scene(scene)
    sc.set_params(I.rrsnet_init_params(1))
    a, _ = sc.render(320, 180, 2, 16, nrrs.RRS_NET, graph=1)
    sc.set_bvh_builder(1)
    sc.set_bvh_precision(32)
    b, _ = sc.render(320, 180, 2, 16, nrrs.RRS_NET, graph=1)
    sc.set_bvh_builder(0)
    c, _ = sc.render(320, 180, 2, 16, nrrs.RRS_NET, graph=1)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())
    np.testing.assert_array_equal(a.cpu().numpy(), c.cpu().numpy())
    with pytest.raises(nrrs.NrrsError):
        sc.set_bvh_builder(2)
    sc.close()
