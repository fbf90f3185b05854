"""Host logic of the BVH builder (CPU): the FP16 copy of the BVH2 that the traversal reads
by default.  Each child box bound is rounded outward to IEEE binary16 (lower bounds
toward -inf, upper toward +inf), so the FP16 box contains the FP32 box and the closest
hit cannot change; leaf codes pack (first reference, count).  The library's rounding is
checked against numpy's binary16 decoding (an independent implementation of the
format), the packed tree against the FP32 tree it came from."""
import os
import subprocess

import numpy as np
import pytest

from paper_2510_07868_b300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2510_07868_b300", "csrc")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("bvh") / "bvh_host_check")
    subprocess.run(["g++", "-O1", "-std=c++17", "-I", CSRC, "-o", exe,
                    os.path.join(os.path.dirname(__file__), "bvh_host_check.cpp"),
                    os.path.join(CSRC, "bvh.cpp")], check=True)
    return exe


def _run(driver, tmp_path, mode, payload):
    src, dst = tmp_path / "in.bin", tmp_path / "out.bin"
    src.write_bytes(payload)
    subprocess.run([driver, mode, str(src), str(dst)], check=True)
    return dst.read_bytes()


def _f16(bits):
    return np.asarray(bits, dtype=np.uint16).view(np.float16).astype(np.float64)


def test_directed_rounding_to_binary16(driver, tmp_path):
    rng = np.random.default_rng(5)
    x = (rng.uniform(-1, 1, 200_000) * np.exp2(rng.integers(-30, 20, 200_000))).astype(np.float32)
    every = np.arange(1 << 16, dtype=np.uint16).view(np.float16)
    every = every[np.isfinite(every)].astype(np.float32)  # every binary16 value exactly
    special = np.array([0.0, -0.0, 65504.0, -65504.0, 65519.0, 65520.0, 70000.0, -70000.0,
                        3.4e38, -3.4e38, 1e-8, -1e-8, 2.0 ** -24, 2.0 ** -25, 2.0 ** -14,
                        np.nextafter(np.float32(2.0 ** -14), np.float32(0))], dtype=np.float32)
    x = np.concatenate([x, every, special, np.nextafter(every, np.float32(np.inf)),
                        np.nextafter(every, np.float32(-np.inf))])
    r = np.frombuffer(_run(driver, tmp_path, "half", x.tobytes()), dtype=np.uint16).reshape(-1, 2)
    lo, hi = _f16(r[:, 0]), _f16(r[:, 1])
    xd = x.astype(np.float64)
    assert np.all(lo <= xd) and np.all(hi >= xd)
    exact = np.isin(x, every)
    assert np.all(lo[exact] == xd[exact]) and np.all(hi[exact] == xd[exact])
    # otherwise the two are neighbouring binary16 values (or +-65504 and +-inf)
    ne = ~exact
    with np.errstate(over="ignore"):  # 65504 steps to inf
        up_of_lo = np.nextafter(lo[ne].astype(np.float16), np.float16(np.inf)).astype(np.float64)
    assert np.all(up_of_lo == hi[ne])
    # the sign of zero survives; magnitudes beyond the largest finite value saturate
    assert r[np.flatnonzero(x == 0)[0], 0] in (0x0000, 0x8000)
    big = np.flatnonzero(x == np.float32(70000.0))[0]
    assert lo[big] == 65504.0 and hi[big] == np.inf


@pytest.mark.parametrize("scene", ["box", "occluded", "ggx"])
def test_packed_nodes_contain_the_fp32_boxes(driver, tmp_path, scene):
    s = {"box": lambda: I.box_scene(2), "occluded": lambda: I.occluded_room(1),
         "ggx": lambda: I.icosphere_room(4, min_triangles=3000, subdiv=2)}[scene]()
    payload = np.int32(s.n_tri).tobytes() + s.tri.astype(np.float32).tobytes()
    out = _run(driver, tmp_path, "pack", payload)
    nn = int(np.frombuffer(out[:8], dtype=np.int64)[0])
    rec = np.dtype([("a", "<f4", 4), ("b", "<f4", 4), ("c", "<f4", 4), ("d", "<i4", 4)])
    nodes = np.frombuffer(out[8:8 + 64 * nn], dtype=rec)
    ok = np.frombuffer(out[8 + 64 * nn:12 + 64 * nn], dtype=np.int32)[0]
    assert ok == 1
    half = np.frombuffer(out[12 + 64 * nn:], dtype=np.uint32).reshape(nn, 8)
    assert half.shape[0] == nn > 1
    # FP32 bounds per child: (lo.x, hi.x, lo.y, hi.y, lo.z, hi.z)
    f32 = np.stack([np.concatenate([nodes["a"], nodes["c"][:, :2]], axis=1),
                    np.concatenate([nodes["b"], nodes["c"][:, 2:]], axis=1)], axis=1)
    words = half[:, :6].reshape(nn, 2, 3)
    lo = _f16(words & 0xFFFF)
    hi = _f16(words >> 16)
    # an empty child (a leaf of no references) has no box
    used = ~((nodes["d"][:, :2] < 0) & (nodes["d"][:, 2:] == 0))
    flo, fhi = f32[..., 0::2].astype(np.float64), f32[..., 1::2].astype(np.float64)
    assert np.all((lo <= flo)[used]) and np.all((hi >= fhi)[used])
    # outward by less than one binary16 spacing (2^-10 relative, or 2^-24 near zero)
    slack = np.maximum(np.abs(flo), np.abs(fhi)) * 2.0 ** -10 + 2.0 ** -24
    assert np.all(((flo - lo) <= slack)[used]) and np.all(((hi - fhi) <= slack)[used])
    # child codes: inner nodes as they are, leaves as ~(first | count << 26)
    code = half[:, 6:8].view(np.int32)
    inner = nodes["d"][:, :2] >= 0
    assert np.array_equal(code[inner], nodes["d"][:, :2][inner])
    v = (~code[~inner]).astype(np.uint32)
    assert np.array_equal((v & ((1 << 26) - 1)).astype(np.int64),
                          (~nodes["d"][:, :2][~inner]).astype(np.int64))
    assert np.array_equal((v >> 26).astype(np.int64), nodes["d"][:, 2:][~inner].astype(np.int64))


def test_pack_refuses_leaves_beyond_the_code(driver, tmp_path):
    res = np.frombuffer(_run(driver, tmp_path, "limit", b"\0"), dtype=np.int32)
    assert res.tolist() == [1, 0, 0]  # 31 references fit; 32, or a first at 2^26, do not


def _growth_numpy(out):
    """Growth of the packed child boxes' summed surface area, from the pack output."""
    nn = int(np.frombuffer(out[:8], dtype=np.int64)[0])
    rec = np.dtype([("a", "<f4", 4), ("b", "<f4", 4), ("c", "<f4", 4), ("d", "<i4", 4)])
    nodes = np.frombuffer(out[8:8 + 64 * nn], dtype=rec)
    half = np.frombuffer(out[12 + 64 * nn:], dtype=np.uint32).reshape(nn, 8)
    f32 = np.stack([np.concatenate([nodes["a"], nodes["c"][:, :2]], axis=1),
                    np.concatenate([nodes["b"], nodes["c"][:, 2:]], axis=1)], axis=1)
    words = half[:, :6].reshape(nn, 2, 3)
    with np.errstate(over="ignore", invalid="ignore"):
        q = np.stack([_f16(words & 0xFFFF), _f16(words >> 16)], axis=-1)
        f = np.stack([f32[..., 0::2], f32[..., 1::2]], axis=-1).astype(np.float64)

        def area(b):
            e = b[..., 1] - b[..., 0]
            return 2 * (e[..., 0] * e[..., 1] + e[..., 1] * e[..., 2] + e[..., 2] * e[..., 0])

        a, qa = area(f), area(q)
        used = ~((nodes["d"][:, :2] < 0) & (nodes["d"][:, 2:] == 0))
        return float(min(qa[used].sum() / a[used].sum() - 1.0, 1e6))


def test_growth_of_packed_boxes_picks_the_default(driver, tmp_path):
    """Near the origin the rounded boxes' summed area grows by well under the 10 % that
    keeps FP16 the default; the same scene moved to x ~ 2000 (binary16 spacing 1 or 2
    there) grows far beyond it, so it defaults to the FP32 nodes.  The library's figure
    equals the one computed here from the packed tree."""
    s = I.occluded_room(1)
    far = s.tri.copy()
    far[:, 0::3] += 2000.0
    for tri, lo_bound in ((s.tri, None), (far, 0.10)):
        payload = np.int32(len(tri)).tobytes() + tri.astype(np.float32).tobytes()
        g = float(np.frombuffer(_run(driver, tmp_path, "growth", payload), dtype=np.float64)[0])
        ref = _growth_numpy(_run(driver, tmp_path, "pack", payload))
        assert g == pytest.approx(ref, rel=1e-9)
        if lo_bound is None:
            assert 0.0 < g < 0.10
        else:
            assert g > lo_bound
