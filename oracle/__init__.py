"""ctypes front end of the FP64 CPU oracle (``nrrs_oracle.c``).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and bench.py's CPU
baseline leg load it.  The product package never imports this module, and this
module never imports the product package.

The paper prints no BSDF; the GGX lobe (``or_ggx_D``, ``or_ggx_G1``, ``or_sample_ggx``,
``or_eval_bsdf``) is pinned in tests/ by the identities of the microfacet model
(normalisation of D, Smith's masking identity, the expected sampling weight equal to the
quadrature of f cos, the normal-incidence closed form).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nrrs_oracle.c")
_SRC_TRAIN = os.path.join(_HERE, "nrrs_oracle_train.c")
_SRC_ENC = os.path.join(_HERE, "nrrs_oracle_encoding.c")
_LIB = os.path.join(_HERE, "liboracle.so")

MODE_NONE, MODE_PLAIN_RR, MODE_HEUR_NORM, MODE_NET, MODE_NET_MIX = range(5)
GATE_NET, GATE_HEUR, GATE_FIXED, GATE_ADRRS = 0, 1, 2, 3
MAX_DEPTH = 64
NO_HIT = 0xFFFFFFFF


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (gcc, -O2, OpenMP)."""
    stale = not os.path.exists(_LIB) or any(
        os.path.getmtime(_LIB) < os.path.getmtime(f) for f in (_SRC, _SRC_TRAIN, _SRC_ENC))
    if force or stale:
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fopenmp", "-fPIC", "-shared",
               "-ffp-contract=off", _SRC, _SRC_TRAIN, _SRC_ENC, "-o", _LIB, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


class Material(C.Structure):
    _fields_ = [("type", C.c_int32), ("albedo", C.c_float * 3), ("Le", C.c_float * 3),
                ("roughness", C.c_float), ("F0", C.c_float), ("two_sided", C.c_int32)]


class Camera(C.Structure):
    _fields_ = [("pos", C.c_float * 3), ("look", C.c_float * 3), ("up", C.c_float * 3),
                ("vfov_deg", C.c_float)]


class SceneC(C.Structure):
    _fields_ = [("tri", C.c_void_p), ("mat_id", C.c_void_p), ("mats", C.c_void_p),
                ("n_tri", C.c_int32), ("n_mat", C.c_int32), ("cam", C.c_void_p)]


class RenderArgs(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("spp", C.c_int32),
                ("max_depth", C.c_int32), ("mode", C.c_int32), ("seed_lo", C.c_uint32),
                ("seed_hi", C.c_uint32), ("frame", C.c_uint32), ("cap", C.c_int64),
                ("f_rate", C.c_double), ("alpha0", C.c_double), ("q_max", C.c_double),
                ("eps_rel", C.c_double), ("boxcox_lambda", C.c_double), ("gate", C.c_uint64),
                ("params", C.c_void_p), ("pixel_ref", C.c_void_p), ("pixels", C.c_void_p),
                ("n_pixels", C.c_int64), ("rec", C.c_void_p), ("forced_F", C.c_void_p),
                ("stat_params", C.c_void_p), ("nee", C.c_int32), ("rrsnet_inputs", C.c_int32),
                ("stat_encoding", C.c_int32), ("stat_grid", C.c_void_p), ("rrs_grid", C.c_void_p),
                ("budget", C.c_int64)]


class RenderStats(C.Structure):
    _fields_ = [("live", C.c_int64 * (MAX_DEPTH + 1)), ("sum_q", C.c_double * (MAX_DEPTH + 1)),
                ("F", C.c_float * (MAX_DEPTH + 1)), ("alpha", C.c_double * (MAX_DEPTH + 1)),
                ("dropped", C.c_int64 * (MAX_DEPTH + 1)),
                ("requested", C.c_int64 * (MAX_DEPTH + 1)),
                ("segments", C.c_int64), ("nonfinite", C.c_int64)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.c_void_p
        _lib.or_philox4x32_10.argtypes = [P, P, P]
        _lib.or_intersect.argtypes = [P, P, P, P]
        _lib.or_intersect.restype = C.c_int32
        _lib.or_camera_ray.argtypes = [P, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                       C.c_double, C.c_double, P, P]
        _lib.or_sample_lambert.argtypes = [P, C.c_double, C.c_double, P]
        _lib.or_sample_ggx.argtypes = [P, P, P, C.c_double, C.c_double, C.c_double, C.c_double,
                                       C.c_double, P, P]
        _lib.or_sample_ggx.restype = C.c_int
        _lib.or_ggx_D.argtypes = [C.c_double, C.c_double]
        _lib.or_ggx_D.restype = C.c_double
        _lib.or_ggx_G1.argtypes = [C.c_double, C.c_double]
        _lib.or_ggx_G1.restype = C.c_double
        _lib.or_eval_ggx.argtypes = [P, P, P, P, C.c_double, C.c_double, P, P]
        _lib.or_eval_ggx.restype = C.c_int
        _lib.or_sample_ggx_batch.argtypes = [P, P, P, C.c_double, C.c_double, P, C.c_int64, P, P]
        _lib.or_eval_ggx_batch.argtypes = [P, P, P, C.c_int64, P, C.c_double, C.c_double, P, P]
        _lib.or_error_temporal.argtypes = [P, P, C.c_int64, C.c_double, C.c_int]
        _lib.or_error_filter.argtypes = [P, P, C.c_int32, C.c_int32, C.c_int32, C.c_double, P]
        _lib.or_pixel_normals.argtypes = [P, P, C.c_int64, C.c_int32, P]
        _lib.or_softplus_mod.argtypes = [C.c_double]
        _lib.or_softplus_mod.restype = C.c_double
        _lib.or_softplus_mod_grad.argtypes = [C.c_double]
        _lib.or_softplus_mod_grad.restype = C.c_double
        _lib.or_mlp_forward.argtypes = [P, P, P, P, P]
        _lib.or_mlp_forward.restype = C.c_double
        _lib.or_mlp_backward.argtypes = [P, P, C.c_double, P]
        _lib.or_mlp_forward_batch.argtypes = [P, P, C.c_int64, P]
        _lib.or_boxcox.argtypes = [C.c_double, C.c_double]
        _lib.or_boxcox.restype = C.c_double
        _lib.or_normalize.argtypes = [P, C.c_int64, C.c_double, C.c_double, C.c_double, P]
        _lib.or_normalize.restype = C.c_double
        _lib.or_split.argtypes = [P, C.c_int64, C.c_float, P, P, P, C.c_uint32, C.c_uint32,
                                  C.c_uint32, C.c_uint32, C.c_int64, P, P, P, P, P]
        _lib.or_split.restype = C.c_int64
        _lib.or_bernstein_exponent.argtypes = [C.c_double]
        _lib.or_bernstein_exponent.restype = C.c_double
        _lib.or_render.argtypes = [P, P, P, P, P, P]
        _lib.or_render.restype = C.c_int
        _lib.or_mlpn_param_count.argtypes = [C.c_int]
        _lib.or_mlpn_param_count.restype = C.c_int64
        _lib.or_mlpn_forward.argtypes = [P, C.c_int, P, P, P, P]
        _lib.or_mlpn_backward.argtypes = [P, C.c_int, P, P, P]
        _lib.or_statnet_dloss.argtypes = [P, P, C.c_double, P]
        _lib.or_statnet_dloss.restype = C.c_double
        _lib.or_pixel_error.argtypes = [P, C.c_int64, C.c_int32, P, C.c_double, P, P]
        _lib.or_rrsnet_dloss.argtypes = [C.c_int64, P, P, P, P, P, P, P, C.c_int64, P, P, P,
                                         C.c_double, C.c_double, C.c_double, C.c_double, P, P]
        _lib.or_rrsnet_dloss_at.argtypes = [C.c_int64, P, P, P, P, P, P, P, P, C.c_int64, P, P,
                                            P, C.c_double, C.c_double, C.c_double, C.c_double,
                                            P, P]
        _lib.or_adam_step.argtypes = [P, P, P, P, C.c_int64, C.c_int64, C.c_double, C.c_double,
                                      C.c_double, C.c_double]
        _lib.or_ema.argtypes = [P, P, C.c_int64, C.c_double]
        _lib.or_relmse.argtypes = [P, P, C.c_int64, C.c_double]

        _lib.or_relmse.restype = C.c_double
        _lib.or_mlpk_param_count.argtypes = [C.c_int, C.c_int]
        _lib.or_mlpk_param_count.restype = C.c_int64
        _lib.or_mlpk_forward.argtypes = [P, C.c_int, C.c_int, P, P, P, P]
        _lib.or_mlpk_backward.argtypes = [P, C.c_int, C.c_int, P, P, P, P]
        _lib.or_grid_param_count.argtypes = []
        _lib.or_grid_param_count.restype = C.c_int64
        _lib.or_grid_index.argtypes = [C.c_int, C.c_uint32, C.c_uint32, C.c_uint32]
        _lib.or_grid_index.restype = C.c_uint32
        _lib.or_grid_encode.argtypes = [P, P, P]
        _lib.or_grid_backward.argtypes = [P, P, P]
        _lib.or_one_blob.argtypes = [C.c_double, C.c_int, P]
        _lib.or_statnet_grid_inputs.argtypes = [P, P, P, C.c_double, P]
        _lib.or_aid_inputs.argtypes = [P, P, P, P, C.c_double, C.c_double, C.c_double, P]
    return _lib


def _p(a):
    return a.ctypes.data if a is not None else None


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_p(c), _p(k), _p(out))
    return out


class _SceneHolder:
    """Keeps the numpy arrays alive while the C struct points at them."""

    def __init__(self, scene):
        self.tri = np.ascontiguousarray(scene.tri, dtype=np.float32)
        self.mat_id = np.ascontiguousarray(scene.mat_id, dtype=np.int32)
        self.mats = np.ascontiguousarray(scene.mats)
        self.cam = np.ascontiguousarray(scene.cam)
        self.c = SceneC(_p(self.tri), _p(self.mat_id), _p(self.mats), self.tri.shape[0],
                        len(self.mats), _p(self.cam))


def intersect(scene, o, d):
    h = _SceneHolder(scene)
    o = np.ascontiguousarray(o, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.float64)
    t = np.zeros(1)
    tri = lib().or_intersect(C.byref(h.c), _p(o), _p(d), _p(t))
    return int(tri), float(t[0])


def camera_ray(scene, W, H, px, py, jx, jy):
    cam = np.ascontiguousarray(scene.cam)
    o = np.zeros(3)
    d = np.zeros(3)
    lib().or_camera_ray(_p(cam), W, H, px, py, jx, jy, _p(o), _p(d))
    return o, d


def sample_lambert(n, u1, u2):
    n = np.ascontiguousarray(n, dtype=np.float64)
    wi = np.zeros(3)
    lib().or_sample_lambert(_p(n), u1, u2, _p(wi))
    return wi


def sample_ggx(n, wo, albedo, rough, F0, ulobe, u1, u2):
    n = np.ascontiguousarray(n, dtype=np.float64)
    wo = np.ascontiguousarray(wo, dtype=np.float64)
    alb = np.ascontiguousarray(albedo, dtype=np.float64)
    wi = np.zeros(3)
    w = np.zeros(3)
    ok = lib().or_sample_ggx(_p(n), _p(wo), _p(alb), rough, F0, ulobe, u1, u2, _p(wi), _p(w))
    return ok, wi, w


def ggx_D(cos_h, a):
    """GGX normal distribution at cos(theta_h) for roughness a."""
    return float(lib().or_ggx_D(float(cos_h), float(a)))


def ggx_G1(cos_w, a):
    """Smith masking term of GGX for a direction at cos(theta)."""
    return float(lib().or_ggx_G1(float(cos_w), float(a)))


def eval_ggx(n, wo, wi, albedo, rough, F0):
    """f cos_i per channel and the sampling pdf of wi for the GGX + Lambert mixture."""
    n = np.ascontiguousarray(n, dtype=np.float64)
    wo = np.ascontiguousarray(wo, dtype=np.float64)
    wi = np.ascontiguousarray(wi, dtype=np.float64)
    alb = np.ascontiguousarray(albedo, dtype=np.float64)
    fc = np.zeros(3)
    pdf = np.zeros(1)
    ok = lib().or_eval_ggx(_p(n), _p(wo), _p(wi), _p(alb), rough, F0, _p(fc), _p(pdf))
    return ok, fc, float(pdf[0])


def sample_ggx_batch(n, wo, albedo, rough, F0, u):
    """or_sample_ggx over rows of u [m][3] = (ulobe, u1, u2): directions and weights."""
    n = np.ascontiguousarray(n, dtype=np.float64)
    wo = np.ascontiguousarray(wo, dtype=np.float64)
    alb = np.ascontiguousarray(albedo, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    m = u.shape[0]
    wi = np.zeros((m, 3))
    w = np.zeros((m, 3))
    lib().or_sample_ggx_batch(_p(n), _p(wo), _p(alb), rough, F0, _p(u), m, _p(wi), _p(w))
    return wi, w


def eval_ggx_batch(n, wo, wi, albedo, rough, F0):
    """or_eval_ggx over rows of wi [m][3]: f cos per channel and the sampling pdf."""
    n = np.ascontiguousarray(n, dtype=np.float64)
    wo = np.ascontiguousarray(wo, dtype=np.float64)
    wi = np.ascontiguousarray(wi, dtype=np.float64)
    alb = np.ascontiguousarray(albedo, dtype=np.float64)
    m = wi.shape[0]
    fc = np.zeros((m, 3))
    pdf = np.zeros(m)
    lib().or_eval_ggx_batch(_p(n), _p(wo), _p(wi), m, _p(alb), rough, F0, _p(fc), _p(pdf))
    return fc, pdf


def error_temporal(E_cur, E_acc, alpha=0.5, first=False):
    """Temporal EMA of the error map; returns the new E_acc (E_acc is not modified)."""
    Ec = np.ascontiguousarray(E_cur, dtype=np.float64)
    Ea = np.array(E_acc if E_acc is not None else np.zeros_like(Ec), dtype=np.float64)
    lib().or_error_temporal(_p(Ec), _p(Ea), Ec.size, float(alpha), int(bool(first)))
    return Ea


def error_filter(E, W, H, radius, normals=None, power=8.0):
    """The normal-guided (2r+1)^2 spatial filter of the error map."""
    Ein = np.ascontiguousarray(E, dtype=np.float64)
    N = np.ascontiguousarray(normals, dtype=np.float64) if normals is not None else None
    out = np.zeros(W * H)
    lib().or_error_filter(_p(Ein), _p(N), W, H, radius, float(power), _p(out))
    return out


def pixel_normals(feat1, q1, npix, spp):
    """Per-pixel normals guiding the filter from the depth-1 features [npix*spp][16]."""
    f = np.ascontiguousarray(feat1, dtype=np.float64)
    q = np.ascontiguousarray(q1, dtype=np.float64)
    out = np.zeros((npix, 4))
    lib().or_pixel_normals(_p(f), _p(q), npix, spp, _p(out))
    return out


def softplus_mod(x):
    return lib().or_softplus_mod(float(x))


def softplus_mod_grad(x):
    return lib().or_softplus_mod_grad(float(x))


def boxcox(t, lam=0.5):
    return lib().or_boxcox(float(t), float(lam))


def mlp_forward(params, x):
    P = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    pre = np.zeros(96)
    hid = np.zeros(96)
    z = np.zeros(1)
    q = lib().or_mlp_forward(_p(P), _p(x), _p(pre), _p(hid), _p(z))
    return q, float(z[0]), pre, hid


def mlp_forward_batch(params, X):
    P = np.ascontiguousarray(params, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float32)
    q = np.zeros(X.shape[0])
    lib().or_mlp_forward_batch(_p(P), _p(X), X.shape[0], _p(q))
    return q


def mlp_backward(params, x, dq):
    P = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    G = np.zeros_like(P)
    lib().or_mlp_backward(_p(P), _p(x), float(dq), _p(G))
    return G


def normalize(q, budget, f_rate=0.85, alpha=1.0):
    q = np.ascontiguousarray(q, dtype=np.float64)
    s = np.zeros(1)
    F = lib().or_normalize(_p(q), q.shape[0], float(budget), float(f_rate), float(alpha), _p(s))
    return F, float(s[0])


def split(q_orig, F32, pixel, sample, lineage, depth, seed=(1, 0), frame=0, cap=None):
    """Eq. rrs_factor over one queue; returns X, prefix, child parent, child lineage, S, dropped."""
    q = np.ascontiguousarray(q_orig, dtype=np.float32)
    n = q.shape[0]
    pixel = np.ascontiguousarray(pixel, dtype=np.uint32)
    sample = np.ascontiguousarray(sample, dtype=np.uint32)
    lineage = np.ascontiguousarray(lineage, dtype=np.uint32)
    cap = int(cap if cap is not None else 2 * n + 16)
    X = np.zeros(n, dtype=np.uint32)
    prefix = np.zeros(n, dtype=np.int64)
    cp = np.zeros(max(cap, 1), dtype=np.uint32)
    cl = np.zeros(max(cap, 1), dtype=np.uint32)
    dropped = np.zeros(1, dtype=np.int64)
    S = lib().or_split(_p(q), n, C.c_float(F32), _p(pixel), _p(sample), _p(lineage), depth,
                       seed[0], seed[1], frame, cap, _p(X), _p(prefix), _p(cp), _p(cl),
                       _p(dropped))
    m = min(S, cap)
    return X, prefix, cp[:m], cl[:m], int(S), int(dropped[0])


def bernstein_exponent(f_rate):
    return lib().or_bernstein_exponent(float(f_rate))


def render(scene, width, height, spp, max_depth, mode, seed=(1, 0), frame=0, cap=0,
           f_rate=0.85, alpha0=1.0, q_max=16.0, eps_rel=0.01, boxcox_lambda=0.5, gate=0,
           params=None, pixel_ref=None, pixels=None, trace=False, record=False, forced_F=None,
           stat_params=None, nee=0, rrsnet_inputs=0, stat_grid=None, rrs_grid=None, budget=0):
    """One oracle render; returns (rgb [H,W,3] float64, stats dict, trace or None).
    nee=1 adds next-event estimation with MIS (power heuristic) at every vertex;
    rrsnet_inputs=1 feeds RRSNet the NRRS inputs built from StatNet (stat_params);
    with stat_grid (the hash-grid table) StatNet reads the encodings of Sec. 4 (32 inputs,
    stat_params then has 32 inputs) instead of the vertex features; rrsnet_inputs=2 with
    rrs_grid is AID-NRRS (RRSNet on 32 encoded inputs, params then has 32 inputs).
    With record=True the stats dict also holds "rec": per depth an array [live, 30] of
    (S rgb, deposit rgb, t rgb, q_orig, q_used, X, first child, pixel, the 16 vertex
    features)."""
    h = _SceneHolder(scene)
    P = np.ascontiguousarray(params, dtype=np.float64) if params is not None else None
    ref = np.ascontiguousarray(pixel_ref, dtype=np.float64) if pixel_ref is not None else None
    pix = np.ascontiguousarray(pixels, dtype=np.int32) if pixels is not None else None
    capv = cap if cap > 0 else 2 * width * height * spp
    rec = np.zeros((max_depth, capv, 30)) if record else None
    fF = np.ascontiguousarray(forced_F, dtype=np.float32) if forced_F is not None else None
    SP = np.ascontiguousarray(stat_params, dtype=np.float64) if stat_params is not None else None
    SG = np.ascontiguousarray(stat_grid, dtype=np.float64) if stat_grid is not None else None
    RG = np.ascontiguousarray(rrs_grid, dtype=np.float64) if rrs_grid is not None else None
    args = RenderArgs(width, height, spp, max_depth, mode, seed[0], seed[1], frame, cap, f_rate,
                      alpha0, q_max, eps_rel, boxcox_lambda, gate, _p(P), _p(ref), _p(pix),
                      0 if pix is None else pix.shape[0], _p(rec), _p(fF), _p(SP), int(nee),
                      int(rrsnet_inputs), 0 if SG is None else 1, _p(SG), _p(RG), int(budget))
    out = np.zeros((height, width, 3))
    st = RenderStats()
    tr = np.zeros((max_depth, capv, 5), dtype=np.uint32) if trace else None
    tc = np.zeros(max_depth, dtype=np.int64) if trace else None
    rc = lib().or_render(C.byref(h.c), C.byref(args), _p(out), C.byref(st), _p(tr), _p(tc))
    if rc != 0:
        raise RuntimeError(f"oracle render failed with code {rc}")
    D = max_depth
    stats = {
        "live": np.array(st.live[1:D + 1]), "sum_q": np.array(st.sum_q[1:D + 1]),
        "F": np.array(st.F[1:D + 1], dtype=np.float32), "alpha": np.array(st.alpha[1:D + 1]),
        "dropped": np.array(st.dropped[1:D + 1]), "requested": np.array(st.requested[1:D + 1]),
        "segments": int(st.segments), "nonfinite": int(st.nonfinite),
    }
    if record:
        stats["rec"] = [rec[d, :stats["live"][d]] for d in range(D)]
    trace_out = None
    if trace:
        trace_out = [tr[d, :tc[d]] for d in range(D)]
    return out, stats, trace_out


# ------------------------------------------------------------------ training side
def mlpn_param_count(n_out):
    return int(lib().or_mlpn_param_count(n_out))


def mlpn_forward(params, n_out, x):
    P = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(n_out)
    lib().or_mlpn_forward(_p(P), n_out, _p(x), _p(out), None, None)
    return out


def mlpk_param_count(n_in, n_out):
    return int(lib().or_mlpk_param_count(n_in, n_out))


def mlpk_forward(params, n_in, n_out, x):
    P = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(n_out)
    lib().or_mlpk_forward(_p(P), n_in, n_out, _p(x), _p(out), None, None)
    return out


def mlpk_backward(params, n_in, n_out, x, dout):
    """(gradient of sum dout . out with respect to the weights, and to the inputs)."""
    P = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    d = np.ascontiguousarray(dout, dtype=np.float64)
    G = np.zeros_like(P)
    dx = np.zeros(n_in)
    lib().or_mlpk_backward(_p(P), n_in, n_out, _p(x), _p(d), _p(G), _p(dx))
    return G, dx


GRID_LEVELS, GRID_T = 8, 1 << 18


def grid_param_count():
    return int(lib().or_grid_param_count())


def grid_index(level, x, y, z):
    return int(lib().or_grid_index(level, x, y, z))


def grid_encode(table, p):
    """Hash-grid features [n, 16] of points p [n, 3] in [0, 1]^3."""
    T = np.ascontiguousarray(table, dtype=np.float64)
    p = np.ascontiguousarray(np.atleast_2d(p), dtype=np.float64)
    out = np.zeros((p.shape[0], 16))
    for i in range(p.shape[0]):
        lib().or_grid_encode(_p(T), _p(p[i]), _p(out[i]))
    return out


def grid_backward(p, dout):
    """Table gradient of sum_i dout[i] . encode(p[i])."""
    p = np.ascontiguousarray(np.atleast_2d(p), dtype=np.float64)
    d = np.ascontiguousarray(np.atleast_2d(dout), dtype=np.float64)
    G = np.zeros(grid_param_count())
    for i in range(p.shape[0]):
        lib().or_grid_backward(_p(G), _p(p[i]), _p(d[i]))
    return G


def one_blob(v, k):
    out = np.zeros(k)
    lib().or_one_blob(float(v), int(k), _p(out))
    return out


def statnet_grid_inputs(table, p, wo, alpha):
    T = np.ascontiguousarray(table, dtype=np.float64)
    p = np.ascontiguousarray(p, dtype=np.float64)
    wo = np.ascontiguousarray(wo, dtype=np.float64)
    x = np.zeros(32)
    lib().or_statnet_grid_inputs(_p(T), _p(p), _p(wo), float(alpha), _p(x))
    return x


def aid_inputs(table, p, wo, t, I, alpha, lam=0.5):
    T = np.ascontiguousarray(table, dtype=np.float64)
    p = np.ascontiguousarray(p, dtype=np.float64)
    wo = np.ascontiguousarray(wo, dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.float64)
    x = np.zeros(32)
    lib().or_aid_inputs(_p(T), _p(p), _p(wo), _p(t), float(I), float(alpha), float(lam), _p(x))
    return x


def mlpn_backward(params, n_out, x, dout):
    P = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    d = np.ascontiguousarray(dout, dtype=np.float64)
    G = np.zeros_like(P)
    lib().or_mlpn_backward(_p(P), n_out, _p(x), _p(d), _p(G))
    return G


def statnet_dloss(pred, L, eps=0.01):
    pred = np.ascontiguousarray(pred, dtype=np.float64)
    L = np.ascontiguousarray(L, dtype=np.float64)
    d = np.zeros(6)
    loss = lib().or_statnet_dloss(_p(pred), _p(L), eps, _p(d))
    return loss, d


def pixel_error(S1, spp, ref, eps=0.01):
    S1 = np.ascontiguousarray(S1, dtype=np.float64)
    ref = np.ascontiguousarray(ref, dtype=np.float64)
    npix = ref.size // 3
    V = np.zeros(npix)
    E = np.zeros(npix)
    lib().or_pixel_error(_p(S1), npix, spp, _p(ref), eps, _p(V), _p(E))
    return V, E


def rrsnet_dloss(q_nrrs, F, Fn, t, pixel, m1, m2, E, Iref, k, eps=0.01, g=(0.01, 0.05, 0.01),
                 q_used=None):
    """d L_RRSNet / d q_nrrs per sample and (L_avg, L_min, L_rrs); q_used: the factor the
    frame was split with (default F q_nrrs)."""
    a = [np.ascontiguousarray(v, dtype=np.float64) for v in (q_nrrs, F, Fn, t, m1, m2)]
    pixel = np.ascontiguousarray(pixel, dtype=np.int32)
    E = np.ascontiguousarray(E, dtype=np.float64)
    Iref = np.ascontiguousarray(Iref, dtype=np.float64)
    k = np.ascontiguousarray(k, dtype=np.int64)
    n = a[0].shape[0]
    dq = np.zeros(n)
    terms = np.zeros(3)
    qu = np.ascontiguousarray(q_used, dtype=np.float64) if q_used is not None else None
    lib().or_rrsnet_dloss_at(n, _p(a[0]), _p(a[1]), _p(a[2]), _p(qu), _p(a[3]), _p(pixel),
                             _p(a[4]), _p(a[5]), E.shape[0], _p(E), _p(Iref), _p(k), eps, g[0],
                             g[1], g[2], _p(dq), _p(terms))
    return dq, terms


def adam_step(P, G, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    for arr in (P, m, v):
        assert arr.dtype == np.float64 and arr.flags.c_contiguous
    G = np.ascontiguousarray(G, dtype=np.float64)
    lib().or_adam_step(_p(P), _p(G), _p(m), _p(v), P.shape[0], step, lr, b1, b2, eps)


def ema(Eavg, P, decay=0.99):
    P = np.ascontiguousarray(P, dtype=np.float64)
    lib().or_ema(_p(Eavg), _p(P), P.shape[0], decay)


def relmse(img, ref, eps=0.01):
    img = np.ascontiguousarray(img, dtype=np.float64).reshape(-1)
    ref = np.ascontiguousarray(ref, dtype=np.float64).reshape(-1)
    return float(lib().or_relmse(_p(img), _p(ref), img.shape[0], eps))
