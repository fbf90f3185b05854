"""Seeded synthetic inputs for the NRRS bounce: scenes, cameras, network weights, features.

This module draws random inputs only. It holds none of the method's arithmetic (no
intersection, sampling, roulette, splitting or network evaluation), so that the CUDA
path and the CPU oracle can both be fed from it without sharing any of the method.

The paper's scenes (Apartment, Bistro, Sponza, Sun Temple; Sec. 5) are not available;
these procedural scenes stand in for them:

* ``box_scene``          - closed unit box of 12 triangles, a 0.2 x 0.2 ceiling emitter
                           (radiance 10) and 20 seed-random triangles (furnace variant:
                           albedo 0.5 and emission 1 on every surface).
* ``occluded_room``      - the box split by an inner wall with a 0.1-wide slot, an
                           emitter of area 0.05 (radiance 100) behind the wall, and
                           seed-random small triangles.
* ``icosphere_room``     - a room of seed-random icospheres and boxes, half Lambertian,
                           half GGX, with 4 ceiling quad lights.
* ``lit_floor``          - a floor under an a x b rectangular emitter at height c whose
                           corner lies straight above the one point a pencil camera sees
                           (direct light there has a closed form).

Binary layouts (shared with ``include/nrrs.h``):

* triangles: float32 ``[n_tri, 9]`` = v0.xyz, v1.xyz, v2.xyz.
* material:  40-byte record ``MATERIAL_DTYPE`` (type, albedo rgb, Le rgb, roughness,
  F0, two_sided). type 0 = Lambertian, 1 = GGX/Lambert "plastic" mixture.
* camera:    40-byte record ``CAMERA_DTYPE`` (pos, look direction, up, vertical fov).
"""
from __future__ import annotations

import numpy as np

MATERIAL_DTYPE = np.dtype(
    [
        ("type", "<i4"),
        ("albedo", "<f4", (3,)),
        ("Le", "<f4", (3,)),
        ("roughness", "<f4"),
        ("F0", "<f4"),
        ("two_sided", "<i4"),
    ]
)
assert MATERIAL_DTYPE.itemsize == 40

CAMERA_DTYPE = np.dtype(
    [("pos", "<f4", (3,)), ("look", "<f4", (3,)), ("up", "<f4", (3,)), ("vfov_deg", "<f4")]
)
assert CAMERA_DTYPE.itemsize == 40

MAT_LAMBERT = 0
MAT_GGX = 1

# Number of parameters of RRSNet 16 -> 32 -> 32 -> 32 -> 1 without biases
# (Sec. 4, "Network Architecture": 3 layers of 32 neurons).
N_FEATURES = 16
HIDDEN = 32
RRSNET_SHAPES = ((HIDDEN, N_FEATURES), (HIDDEN, HIDDEN), (HIDDEN, HIDDEN), (1, HIDDEN))
RRSNET_N_PARAMS = sum(a * b for a, b in RRSNET_SHAPES)
assert RRSNET_N_PARAMS == 2592


class Scene:
    """Plain container of host arrays describing one scene."""

    def __init__(self, tri, mat_id, mats, cam, name):
        self.tri = np.ascontiguousarray(tri, dtype=np.float32).reshape(-1, 9)
        self.mat_id = np.ascontiguousarray(mat_id, dtype=np.int32)
        self.mats = np.ascontiguousarray(mats, dtype=MATERIAL_DTYPE)
        self.cam = np.ascontiguousarray(cam, dtype=CAMERA_DTYPE).reshape(1)
        self.name = name
        assert self.tri.shape[0] == self.mat_id.shape[0]
        assert self.mat_id.min() >= 0 and self.mat_id.max() < len(self.mats)

    @property
    def n_tri(self):
        return int(self.tri.shape[0])


def _material(type_=MAT_LAMBERT, albedo=0.0, Le=0.0, roughness=0.0, F0=0.04, two_sided=1):
    m = np.zeros((), dtype=MATERIAL_DTYPE)
    m["type"] = type_
    m["albedo"] = np.broadcast_to(np.float32(albedo), (3,))
    m["Le"] = np.broadcast_to(np.float32(Le), (3,))
    m["roughness"] = roughness
    m["F0"] = F0
    m["two_sided"] = two_sided
    return m


def _quad(a, b, c, d):
    """Two triangles (a, b, c) and (a, c, d); the winding fixes the geometric normal."""
    return [np.r_[a, b, c], np.r_[a, c, d]]


def _box_walls(lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
    """12 triangles of an axis-aligned box whose normals (e1 x e2) point inward."""
    x0, y0, z0 = lo
    x1, y1, z1 = hi
    P = lambda x, y, z: np.array([x, y, z], dtype=np.float64)  # noqa: E731
    tris = []
    tris += _quad(P(x0, y0, z0), P(x0, y0, z1), P(x1, y0, z1), P(x1, y0, z0))  # floor, +y
    tris += _quad(P(x0, y1, z0), P(x1, y1, z0), P(x1, y1, z1), P(x0, y1, z1))  # ceiling, -y
    tris += _quad(P(x0, y0, z0), P(x0, y1, z0), P(x0, y1, z1), P(x0, y0, z1))  # x=0 wall, +x
    tris += _quad(P(x1, y0, z0), P(x1, y0, z1), P(x1, y1, z1), P(x1, y1, z0))  # x=1 wall, -x
    tris += _quad(P(x0, y0, z0), P(x1, y0, z0), P(x1, y1, z0), P(x0, y1, z0))  # z=0 wall, +z
    tris += _quad(P(x0, y0, z1), P(x0, y1, z1), P(x1, y1, z1), P(x1, y0, z1))  # z=1 wall, -z
    return tris


def _ceiling_emitter(cx, cz, side, y=0.999):
    """Square at height y, centred (cx, cz), winding chosen so its normal points -y."""
    h = side / 2
    a = np.array([cx - h, y, cz - h])
    b = np.array([cx + h, y, cz - h])
    c = np.array([cx + h, y, cz + h])
    d = np.array([cx - h, y, cz + h])
    return _quad(a, b, c, d)


def _camera(pos, look=(0.0, 0.0, 1.0), up=(0.0, 1.0, 0.0), vfov=60.0):
    c = np.zeros((1,), dtype=CAMERA_DTYPE)
    c["pos"] = pos
    c["look"] = look
    c["up"] = up
    c["vfov_deg"] = vfov
    return c


def box_scene(seed: int = 1, furnace: bool = False, n_random: int = 20) -> Scene:
    """Closed unit box, 0.2 x 0.2 ceiling emitter, ``n_random`` random triangles.

    Walls: Lambertian albedo 0.7, one-sided emission (they emit nothing).
    Emitter: black, radiance 10 along -y.  Random triangles: centre U[0.2,0.8]^3,
    vertices centre + U[-0.15,0.15]^3, grey albedo U[0.1,0.9], two-sided.
    Furnace variant: every surface has albedo 0.5 and emits 1 on both sides, so every
    pixel of a depth-D render converges to sum_{k<D} 0.5^k.
    Camera at (0.5, 0.5, 0.01) looking +z, 60 degree vertical field of view.
    """
    rng = np.random.default_rng(seed)
    tris = _box_walls()
    mats = []
    mat_id = []
    if furnace:
        mats.append(_material(albedo=0.5, Le=1.0, two_sided=1))
        mat_id += [0] * 12
    else:
        mats.append(_material(albedo=0.7, Le=0.0, two_sided=0))
        mats.append(_material(albedo=0.0, Le=10.0, two_sided=0))
        mat_id += [0] * 12
    tris += _ceiling_emitter(0.5, 0.5, 0.2)
    mat_id += [0, 0] if furnace else [1, 1]
    for _ in range(n_random):
        c = rng.uniform(0.2, 0.8, 3)
        v = c + rng.uniform(-0.15, 0.15, (3, 3))
        tris.append(v.reshape(9))
        if furnace:
            mat_id.append(0)
        else:
            mats.append(_material(albedo=rng.uniform(0.1, 0.9), two_sided=1))
            mat_id.append(len(mats) - 1)
    return Scene(np.array(tris), mat_id, np.array(mats), _camera((0.5, 0.5, 0.01)),
                 "furnace_box" if furnace else "box")


def occluded_room(seed: int = 1, n_random: int = 2000, tri_size: float = 0.05) -> Scene:
    """Unit box split at z=0.5 by a wall with a vertical slot x in [0.45, 0.55].

    The emitter (area 0.05, radiance 100, facing -y) hangs under the ceiling at
    z=0.8, on the far side of the wall from the camera at (0.5, 0.5, 0.05).
    ``n_random`` two-sided triangles of edge scale ``tri_size`` (centre U[0,1]^3,
    vertices centre + U[-s/2, s/2]^3) with grey albedo U[0.1, 0.9].
    """
    rng = np.random.default_rng(seed)
    tris = _box_walls()
    mats = [_material(albedo=0.7, two_sided=0), _material(albedo=0.0, Le=100.0, two_sided=0),
            _material(albedo=0.7, two_sided=1)]
    mat_id = [0] * 12
    P = lambda x, y, z: np.array([x, y, z], dtype=np.float64)  # noqa: E731
    for x0, x1 in ((0.0, 0.45), (0.55, 1.0)):
        tris += _quad(P(x0, 0, 0.5), P(x1, 0, 0.5), P(x1, 1, 0.5), P(x0, 1, 0.5))
        mat_id += [2, 2]
    side = float(np.sqrt(0.05))
    tris += _ceiling_emitter(0.5, 0.8, side)
    mat_id += [1, 1]
    h = tri_size / 2
    for _ in range(n_random):
        c = rng.uniform(0.0, 1.0, 3)
        v = c + rng.uniform(-h, h, (3, 3))
        tris.append(v.reshape(9))
        mats.append(_material(albedo=rng.uniform(0.1, 0.9), two_sided=1))
        mat_id.append(len(mats) - 1)
    return Scene(np.array(tris), mat_id, np.array(mats), _camera((0.5, 0.5, 0.05)),
                 "occluded_room")


def _icosphere(subdiv: int):
    t = (1 + 5 ** 0.5) / 2
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t),
         (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    v = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in v]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
         (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
         (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(subdiv):
        cache = {}

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = v[a] + v[b]
                v.append(m / np.linalg.norm(m))
                cache[key] = len(v) - 1
            return cache[key]

        nf = []
        for a, b, c in f:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        f = nf
    V = np.array(v)
    return np.array([np.r_[V[a], V[b], V[c]] for a, b, c in f])


def _random_rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def icosphere_room(seed: int = 1, min_triangles: int = 200_000, subdiv: int = 3) -> Scene:
    """Unit room filled with seed-random icospheres and boxes until ``min_triangles``.

    Each object is, with probability 0.5, an icosphere (``subdiv`` subdivisions,
    radius U[0.02, 0.08]), else a randomly rotated box (12 triangles, half-size
    U[0.02, 0.08]).  Per object: 50% Lambertian (albedo U[0.1, 0.9]) and 50% GGX
    plastic (roughness U[0.05, 0.5], F0 0.04, base albedo U[0.1, 0.9]).  4 ceiling
    quads of 0.1 x 0.1 emit radiance U[5, 50].
    """
    rng = np.random.default_rng(seed)
    tris = _box_walls()
    mats = [_material(albedo=0.7, two_sided=0)]
    mat_id = [0] * 12
    for cx, cz in ((0.25, 0.25), (0.75, 0.25), (0.25, 0.75), (0.75, 0.75)):
        tris += _ceiling_emitter(cx, cz, 0.1)
        mats.append(_material(albedo=0.0, Le=rng.uniform(5, 50), two_sided=0))
        mat_id += [len(mats) - 1] * 2
    sphere = _icosphere(subdiv)
    cube = np.array(_box_walls((-1, -1, -1), (1, 1, 1)))
    while len(tris) < min_triangles:
        centre = rng.uniform(0.1, 0.9, 3)
        size = rng.uniform(0.02, 0.08)
        if rng.uniform() < 0.5:
            obj = sphere.reshape(-1, 3, 3) * size + centre
        else:
            R = _random_rotation(rng)
            obj = (cube.reshape(-1, 3, 3) @ R.T) * size + centre
        if rng.uniform() < 0.5:
            mats.append(_material(albedo=rng.uniform(0.1, 0.9), two_sided=1))
        else:
            mats.append(_material(MAT_GGX, albedo=rng.uniform(0.1, 0.9),
                                  roughness=rng.uniform(0.05, 0.5), F0=0.04, two_sided=1))
        tris += list(obj.reshape(-1, 9))
        mat_id += [len(mats) - 1] * obj.shape[0]
    return Scene(np.array(tris), mat_id, np.array(mats), _camera((0.5, 0.5, 0.01)),
                 "icosphere_room")


def three_rooms(seed: int = 1, n_random: int = 1_000_000, tri_size: float = 0.01,
                n_palette: int = 64, emitter_room: int = 2) -> Scene:
    """Three unit rooms along x ([0,3] x [0,1] x [0,1]) joined by doorways 0.1 wide
    (z in [0.45, 0.55]) and 0.2 high (y in [0, 0.2]) in the walls at x = 1 and x = 2.

    One 0.1 x 0.1 emitter of radiance 200 under the ceiling of room ``emitter_room``
    (centre x = room - 0.5, z = 0.5; room 2 by default: from room 3 almost no light reaches
    the camera through the dust and both doorways), the camera in room 1 at
    (0.05, 0.1, 0.5) looking +x, through both doorways.  ``n_random``
    two-sided triangles (centre uniform in the rooms, vertices centre +
    U[-s/2, s/2]^3) draw their material from a palette of ``n_palette``: 60% GGX plastic
    (roughness U[0.05, 0.5], F0 0.04), the rest Lambertian; albedo U[0.1, 0.9].
    """
    rng = np.random.default_rng(seed)
    tris = _box_walls((0.0, 0.0, 0.0), (3.0, 1.0, 1.0))
    mats = [_material(albedo=0.7, two_sided=0), _material(albedo=0.0, Le=200.0, two_sided=0),
            _material(albedo=0.7, two_sided=1)]
    mat_id = [0] * 12
    P = lambda x, y, z: np.array([x, y, z], dtype=np.float64)  # noqa: E731
    for x in (1.0, 2.0):  # inner walls minus the doorway
        for (z0, z1, y0, y1) in ((0.0, 0.45, 0.0, 1.0), (0.55, 1.0, 0.0, 1.0),
                                 (0.45, 0.55, 0.2, 1.0)):
            tris += _quad(P(x, y0, z0), P(x, y0, z1), P(x, y1, z1), P(x, y1, z0))
            mat_id += [2, 2]
    tris += _ceiling_emitter(emitter_room - 0.5, 0.5, 0.1)
    mat_id += [1, 1]
    first = len(mats)
    n_ggx = int(round(0.6 * n_palette))
    for k in range(n_palette):
        if k < n_ggx:
            mats.append(_material(MAT_GGX, albedo=rng.uniform(0.1, 0.9),
                                  roughness=rng.uniform(0.05, 0.5), F0=0.04, two_sided=1))
        else:
            mats.append(_material(albedo=rng.uniform(0.1, 0.9), two_sided=1))
    h = tri_size / 2
    c = rng.uniform(0.0, 1.0, (n_random, 3)) * np.array([3.0, 1.0, 1.0])
    v = c[:, None, :] + rng.uniform(-h, h, (n_random, 3, 3))
    tri = np.concatenate([np.array(tris).reshape(-1, 9), v.reshape(n_random, 9)])
    mat_id = np.concatenate([np.array(mat_id, dtype=np.int32),
                             first + rng.integers(0, n_palette, n_random).astype(np.int32)])
    return Scene(tri, mat_id, np.array(mats), _camera((0.05, 0.1, 0.5), look=(1.0, 0.0, 0.0)),
                 "three_rooms")


def uneven_jobs(seed: int = 1, n_jobs: int = 64, tri_range=(1_000, 50_000), side_log2=(5, 9),
                spp_range=(1, 64), depth_range=(8, 32), subdiv: int = 2):
    """Render jobs of uneven size for a batched render: per job an ``icosphere_room``
    scene with log-uniform triangle count in ``tri_range`` (half GGX), a square image of
    side round(2^U[side_log2]), spp uniform in ``spp_range`` and depth uniform in
    ``depth_range`` (bounds inclusive).  Returns a list of (Scene, W, H, spp, D)."""
    rng = np.random.default_rng(seed)
    jobs = []
    for k in range(n_jobs):
        n_tri = int(np.exp(rng.uniform(np.log(tri_range[0]), np.log(tri_range[1]))))
        side = int(round(2.0 ** rng.uniform(*side_log2)))
        spp = int(rng.integers(spp_range[0], spp_range[1] + 1))
        D = int(rng.integers(depth_range[0], depth_range[1] + 1))
        scene = icosphere_room(1000 * seed + k, min_triangles=n_tri, subdiv=subdiv)
        jobs.append((scene, side, side, spp, D))
    return jobs


def lit_floor(a: float = 0.6, b: float = 0.4, c: float = 0.5, Le: float = 10.0,
              albedo: float = 0.5, floor_type: int = MAT_LAMBERT, roughness: float = 0.2) -> Scene:
    """A 20 x 20 floor at y = 0 (two-sided) and, at height c, an a x b emitter facing
    down over [0, a] x [0, b] in (x, z), made of three triangles of areas ab/6, ab/3 and
    ab/2 (a fan from its corner at x = z = 0).  The camera sees the origin only: it sits
    at (-0.6, 0.35, -0.6), looks at the origin and has a 0.001 degree field of view."""
    A = np.array([0.0, c, 0.0])
    B = np.array([a, c, 0.0])
    E = np.array([a, c, b / 3.0])
    Cc = np.array([a, c, b])
    D = np.array([0.0, c, b])
    tris = _quad(np.array([-10.0, 0.0, -10.0]), np.array([-10.0, 0.0, 10.0]),
                 np.array([10.0, 0.0, 10.0]), np.array([10.0, 0.0, -10.0]))
    tris += [np.r_[A, B, E], np.r_[A, E, Cc], np.r_[A, Cc, D]]
    mats = [_material(floor_type, albedo, 0.0, roughness=roughness, two_sided=1),
            _material(MAT_LAMBERT, 0.0, Le, two_sided=0)]
    cam = _camera((-0.6, 0.35, -0.6), look=(0.6, -0.35, 0.6), vfov=0.001)
    return Scene(np.array(tris), [0, 0, 1, 1, 1], np.array(mats), cam, "lit_floor")


def rrsnet_init_params(seed: int = 1, dtype=np.float32) -> np.ndarray:
    """Xavier-uniform draw of the 2592 RRSNet weights, packed W1|W2|W3|W4, row-major.

    W1 is [32][16], W2 and W3 are [32][32], W4 is [1][32] (output row).
    """
    rng = np.random.default_rng(seed)
    parts = []
    for fan_out, fan_in in RRSNET_SHAPES:
        a = np.sqrt(6.0 / (fan_in + fan_out))
        parts.append(rng.uniform(-a, a, fan_out * fan_in))
    return np.concatenate(parts).astype(dtype)


def statnet_init_params(seed: int = 1, n_in: int = N_FEATURES, dtype=np.float32) -> np.ndarray:
    """Xavier-uniform draw of StatNet's weights (n_in -> 32 -> 32 -> 32 -> 6), packed
    W1|W2|W3|W4 row-major like RRSNet's; the output weights scaled by 1/4 so that the
    untrained moments start small."""
    rng = np.random.default_rng(seed + 7919)
    parts = []
    for k, (fan_out, fan_in) in enumerate(((HIDDEN, n_in), (HIDDEN, HIDDEN), (HIDDEN, HIDDEN),
                                           (6, HIDDEN))):
        a = np.sqrt(6.0 / (fan_in + fan_out)) * (0.25 if k == 3 else 1.0)
        parts.append(rng.uniform(-a, a, fan_out * fan_in))
    return np.concatenate(parts).astype(dtype)


def random_features(n: int, seed: int = 1) -> np.ndarray:
    """``n`` feature rows [n][16] with the ranges the renderer produces.

    position in [0,1]^3, unit outgoing direction, unit normal, albedo in [0.1,0.9],
    depth fraction in (0,1], throughput-feature values uniform in [-1.9, 2].
    """
    rng = np.random.default_rng(seed)
    f = np.empty((n, N_FEATURES), dtype=np.float64)
    f[:, 0:3] = rng.uniform(0, 1, (n, 3))
    w = rng.normal(size=(n, 3))
    f[:, 3:6] = w / np.linalg.norm(w, axis=1, keepdims=True)
    nn = rng.normal(size=(n, 3))
    f[:, 6:9] = nn / np.linalg.norm(nn, axis=1, keepdims=True)
    f[:, 9:12] = rng.uniform(0.1, 0.9, (n, 1))
    f[:, 12] = rng.integers(1, 17, n) / 16.0
    f[:, 13:16] = rng.uniform(-1.9, 2.0, (n, 1))
    return f.astype(np.float32)


def random_q(n: int, seed: int = 1, scale: float = 2.0) -> np.ndarray:
    """Non-negative float32 RRS factors: 10% exact zeros, the rest log-uniform."""
    rng = np.random.default_rng(seed)
    q = np.exp(rng.uniform(np.log(1e-3), np.log(scale * 4), n))
    q[rng.uniform(size=n) < 0.1] = 0.0
    return q.astype(np.float32)
