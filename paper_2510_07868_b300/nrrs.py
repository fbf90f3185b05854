"""Thin ctypes binding of the C ABI in include/nrrs.h (argument marshalling only).

Every function here forwards to the entry point of the same name in libnrrs.so; all
computation runs in the library's CUDA kernels.  Device buffers are passed as torch
CUDA tensors (or raw integer addresses); streams as torch.cuda.Stream (or raw handles).
Importing this module fails loudly when the compiled library is missing: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnrrs.so")

NRRS_OK = 0
STATUS_NAMES = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "out of device memory",
                4: "timeout", 5: "non-finite", 6: "overflow dropped", 7: "unsupported"}
RRS_NONE, RRS_PLAIN_RR, RRS_HEUR_NORM, RRS_NET, RRS_NET_MIX = range(5)
GATE_NET, GATE_HEUR, GATE_FIXED, GATE_ADRRS = 0, 1, 2, 3
STATUS_OVERFLOW_DROPPED, STATUS_NONFINITE, STATUS_TIMEOUT, STATUS_HEUR_FALLBACK = 1, 2, 4, 8
MAX_DEPTH = 32
STAGES = 11
STAGE_NAMES = ["init", "extend", "normalize", "split_count", "split_scan", "split_scatter",
               "finalize", "rrsnet", "shade", "reverse", "shadow"]
NET_RRSNET, NET_RRSNET_TRAIN, NET_STATNET, NET_STATNET_GRID = 0, 1, 2, 3
NET_RRSNET_GRID, NET_RRSNET_GRID_TRAIN = 4, 5
AID_RRSNET_PARAMS = 3104  # RRSNet on the AID-NRRS inputs (32)
STATNET_PARAMS = 2752
STATNET_GRID_PARAMS = 3264  # StatNet on the encodings (32 inputs)
GRID_PARAMS = 8 * (1 << 18) * 2
N_FEATURES = 16
RRSNET_PARAMS = 2592

EXPORTED = [
    "nrrs_status_string", "nrrs_last_error", "nrrs_create_scene", "nrrs_destroy_scene",
    "nrrs_scene_info", "nrrs_set_rrsnet_params", "nrrs_get_rrsnet_params", "nrrs_render",
    "nrrs_query_factors", "nrrs_normalize", "nrrs_split", "nrrs_split_noalloc",
    "nrrs_train_step", "nrrs_set_params", "nrrs_get_params", "nrrs_mlp_grad",
    "nrrs_rrsnet_dloss", "nrrs_adam_step", "nrrs_ema", "nrrs_mixdepth_candidates", "nrrs_mixdepth_search",
    "nrrs_relmse", "nrrs_error_filter", "nrrs_set_rrsnet_inputs", "nrrs_set_statnet_encoding",
    "nrrs_statnet_grad", "nrrs_statnet_inputs", "nrrs_grid_backward",
    "nrrs_rrsnet_forward", "nrrs_rrsnet_backward", "nrrs_tune_rrsnet",
    "nrrs_set_rrsnet_shape", "nrrs_create_batch", "nrrs_render_batch", "nrrs_batch_info",
    "nrrs_set_traversal",
    "nrrs_set_bvh_precision", "nrrs_set_bvh_builder", "nrrs_bvh8_info", "nrrs_bvh8_export",
    "nrrs_set_shade_fusion", "nrrs_set_traversal_stack", "nrrs_traversal_stack_info",
]


class NrrsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class RenderOpts(C.Structure):
    _fields_ = [("seed_lo", C.c_uint32), ("seed_hi", C.c_uint32), ("frame", C.c_uint32),
                ("cap_factor", C.c_int32), ("f_rate", C.c_float), ("alpha0", C.c_float),
                ("q_max", C.c_float), ("eps_rel", C.c_float), ("boxcox_lambda", C.c_float),
                ("precision", C.c_int32), ("gate", C.c_uint64), ("d_pixel_ref", C.c_void_p),
                ("update_ref", C.c_int32), ("reset_ref", C.c_int32), ("d_trace", C.c_void_p),
                ("profile", C.c_int32), ("graph", C.c_int32), ("d_suffix", C.c_void_p),
                ("nee", C.c_int32), ("d_trace_mask", C.c_void_p), ("d_trace_count", C.c_void_p),
                ("trace_rows", C.c_int64), ("budget_factor", C.c_int32)]

    @classmethod
    def defaults(cls, **kw):
        o = cls(seed_lo=1, seed_hi=0, frame=0, cap_factor=2, f_rate=0.85, alpha0=1.0, q_max=16.0,
                eps_rel=0.01, boxcox_lambda=0.5, precision=32, gate=0, d_pixel_ref=None,
                update_ref=1, reset_ref=0, d_trace=None, profile=0, graph=0, d_suffix=None,
                nee=0, d_trace_mask=None, d_trace_count=None, trace_rows=0, budget_factor=0)
        for k, v in kw.items():
            setattr(o, k, v)
        return o


class RenderStats(C.Structure):
    _fields_ = [("live", C.c_int64 * MAX_DEPTH), ("sum_q", C.c_double * MAX_DEPTH),
                ("F", C.c_float * MAX_DEPTH), ("alpha", C.c_double * MAX_DEPTH),
                ("requested", C.c_int64 * MAX_DEPTH), ("dropped", C.c_int64 * MAX_DEPTH),
                ("segments", C.c_int64), ("nonfinite", C.c_int64), ("net_evals", C.c_int64),
                ("capacity", C.c_int64), ("status_bits", C.c_uint32),
                ("kernel_launches", C.c_uint32), ("stage_ms", C.c_float * 12),
                ("stage_launches", C.c_int32 * 12)]

    def as_dict(self, depth):
        return {
            "live": np.array(self.live[:depth]), "sum_q": np.array(self.sum_q[:depth]),
            "F": np.array(self.F[:depth], dtype=np.float32), "alpha": np.array(self.alpha[:depth]),
            "requested": np.array(self.requested[:depth]),
            "dropped": np.array(self.dropped[:depth]), "segments": int(self.segments),
            "nonfinite": int(self.nonfinite), "net_evals": int(self.net_evals),
            "capacity": int(self.capacity), "status_bits": int(self.status_bits),
            "kernel_launches": int(self.kernel_launches),
            "stage_ms": np.array(self.stage_ms[:STAGES], dtype=np.float64),
            "stage_launches": np.array(self.stage_launches[:STAGES]),
        }


class TrainOpts(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("spp", C.c_int32),
                ("max_depth", C.c_int32), ("seed_lo", C.c_uint32), ("seed_hi", C.c_uint32),
                ("frame", C.c_uint32), ("warmup_steps", C.c_int32), ("lr_rrsnet", C.c_float),
                ("lr_statnet", C.c_float), ("gamma1", C.c_float), ("gamma2", C.c_float),
                ("gamma3", C.c_float), ("eps", C.c_float), ("ema_decay", C.c_float),
                ("f_rate", C.c_float), ("d_pixel_ref", C.c_void_p), ("alpha_mix", C.c_float),
                ("error_filter_radius", C.c_int32), ("graph", C.c_int32),
                ("batch_size", C.c_int32), ("nee", C.c_int32),
                ("error_filter_power", C.c_float), ("error_filter_until", C.c_int32),
                ("debug", C.c_void_p)]

    @classmethod
    def defaults(cls, **kw):
        o = cls(width=256, height=256, spp=2, max_depth=16, seed_lo=1, seed_hi=0, frame=0,
                warmup_steps=20, lr_rrsnet=3e-4, lr_statnet=5e-3, gamma1=0.01, gamma2=0.05,
                gamma3=0.01, eps=0.01, ema_decay=0.99, f_rate=0.85, d_pixel_ref=None,
                alpha_mix=0.5, error_filter_radius=2, graph=0, batch_size=0, nee=0,
                error_filter_power=8.0, error_filter_until=0, debug=None)
        for k, v in kw.items():
            setattr(o, k, v)
        return o


TUNE_BUCKETS = 17
MAX_JOBS = 256


class Job(C.Structure):
    _fields_ = [("tri", C.c_void_p), ("n_tri", C.c_int32), ("tri_mat", C.c_void_p),
                ("mats", C.c_void_p), ("n_mat", C.c_int32), ("cam", C.c_void_p),
                ("width", C.c_int32), ("height", C.c_int32), ("spp", C.c_int32),
                ("max_depth", C.c_int32)]


class TuneReport(C.Structure):
    _fields_ = [("precision", C.c_int32), ("n_buckets", C.c_int32),
                ("rows", C.c_int64 * TUNE_BUCKETS), ("variant", C.c_int32 * TUNE_BUCKETS),
                ("blocks_per_sm", C.c_int32 * TUNE_BUCKETS),
                ("ms_best", C.c_float * TUNE_BUCKETS), ("ms_default", C.c_float * TUNE_BUCKETS)]

    def as_dict(self):
        n = self.n_buckets
        return {"precision": self.precision, "rows": list(self.rows[:n]),
                "variant": list(self.variant[:n]), "blocks_per_sm": list(self.blocks_per_sm[:n]),
                "ms_best": list(self.ms_best[:n]), "ms_default": list(self.ms_default[:n])}


class Bvh8Stats(C.Structure):
    _fields_ = [("nodes", C.c_int64), ("triangles", C.c_int64), ("depth", C.c_int32),
                ("iterations", C.c_int32), ("build_ms", C.c_float)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class TrainDebug(C.Structure):
    """nrrs_train_debug: host buffers a training step fills before its Adam updates."""
    _fields_ = [("grad_statnet", C.c_void_p), ("grad_rrsnet", C.c_void_p),
                ("pixel_var", C.c_void_p), ("pixel_error", C.c_void_p), ("samples", C.c_void_p),
                ("ebar", C.c_float), ("vertices", C.c_int64), ("batch", C.c_int64)]

    @classmethod
    def with_buffers(cls, npix, n_stat, n_rrs):
        """A debug record with numpy buffers attached (kept alive on the object)."""
        d = cls()
        d.arrays = {"grad_statnet": np.zeros(n_stat, np.float32),
                    "grad_rrsnet": np.zeros(n_rrs, np.float32),
                    "pixel_var": np.zeros(npix, np.float32),
                    "pixel_error": np.zeros(npix, np.float32),
                    "samples": np.zeros(npix, np.int32)}
        for k, a in d.arrays.items():
            setattr(d, k, a.ctypes.data)
        return d


class TrainStats(C.Structure):
    _fields_ = [("step", C.c_int64), ("samples", C.c_int64), ("segments", C.c_int64),
                ("loss_statnet", C.c_double), ("loss_rrsnet", C.c_double),
                ("loss_avg", C.c_double), ("loss_min", C.c_double), ("loss_rrs", C.c_double),
                ("phase", C.c_int32), ("fallback", C.c_int32), ("kernel_launches", C.c_int64)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class MixDepthOpts(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("spp", C.c_int32),
                ("max_depth", C.c_int32), ("t_d", C.c_int32), ("max_candidates", C.c_int32),
                ("seed_lo", C.c_uint32), ("seed_hi", C.c_uint32), ("frame", C.c_uint32),
                ("d_pixel_ref", C.c_void_p), ("adrrs", C.c_int32), ("nee", C.c_int32),
                ("precision", C.c_int32)]


class MixDepthResult(C.Structure):
    _fields_ = [("gate", C.c_uint64), ("score", C.c_double), ("relmse", C.c_double),
                ("segments", C.c_int64), ("evaluated", C.c_int64)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -m paper_2510_07868_b300.build` (no CPU fallback exists)")
    lib = C.CDLL(LIB_PATH)
    P, I32, I64, U32, D = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_double
    sig = {
        "nrrs_status_string": ([I32], C.c_char_p),
        "nrrs_last_error": ([], C.c_char_p),
        "nrrs_create_scene": ([P, I32, P, P, I32, P, I32, P], I32),
        "nrrs_destroy_scene": ([P], I32),
        "nrrs_scene_info": ([P, P, P], I32),
        "nrrs_set_rrsnet_params": ([P, P, I32, P], I32),
        "nrrs_get_rrsnet_params": ([P, P, I32, P], I32),
        "nrrs_render": ([P, I32, I32, I32, I32, I32, P, P, P, P], I32),
        "nrrs_query_factors": ([P, P, I64, I32, P, P], I32),
        "nrrs_normalize": ([P, P, I64, D, D, D, P, P, P], I32),
        "nrrs_split": ([P, P, I64, P, P, P, P, U32, U32, U32, U32, I64, P, P, P, P, P, P, P], I32),
        "nrrs_split_noalloc": ([P, I64, P, P, P, P, U32, U32, U32, U32, I64, P, P, P, P, P, P, P],
                               I32),
        "nrrs_train_step": ([P, P, P, P], I32),
        "nrrs_set_params": ([P, I32, P, I32, P], I32),
        "nrrs_get_params": ([P, I32, P, I32, P], I32),
        "nrrs_mlp_grad": ([P, I32, P, P, P, I64, P, P], I32),
        "nrrs_rrsnet_dloss": ([P, P, P, P, P, P, P, P, D, P, P, I64, C.c_float, C.c_float,
                               C.c_float, C.c_float, P, P], I32),
        "nrrs_adam_step": ([P, P, P, P, I32, I32, C.c_float, C.c_float, C.c_float, C.c_float, P],
                           I32),
        "nrrs_ema": ([P, P, I32, C.c_float, P], I32),
        "nrrs_mixdepth_candidates": ([I32, I32], I64),
        "nrrs_mixdepth_search": ([P, P, P, P], I32),
        "nrrs_relmse": ([P, P, I64, D, P, P], I32),
        "nrrs_error_filter": ([P, P, I32, I32, I32, C.c_float, P, P], I32),
        "nrrs_set_rrsnet_inputs": ([P, I32], I32),
        "nrrs_set_statnet_encoding": ([P, I32], I32),
        "nrrs_statnet_grad": ([P, P, P, P, I64, P, P], I32),
        "nrrs_statnet_inputs": ([P, P, P, I64, P, P], I32),
        "nrrs_grid_backward": ([P, P, P, I64, P, P], I32),
        "nrrs_rrsnet_forward": ([P, P, I64, P, P], I32),
        "nrrs_rrsnet_backward": ([P, P, P, P, I64, P, P], I32),
        "nrrs_tune_rrsnet": ([P, I32, P, P], I32),
        "nrrs_set_rrsnet_shape": ([P, I32, I32, I32, I32], I32),
        "nrrs_create_batch": ([P, I32, I32, P], I32),
        "nrrs_render_batch": ([P, I32, P, P, P, P, P, P, P], I32),
        "nrrs_batch_info": ([P, P, P, P], I32),
        "nrrs_set_traversal": ([P, I32], I32),
        "nrrs_set_bvh_precision": ([P, I32], I32),
        "nrrs_set_shade_fusion": ([P, I32], I32),
        "nrrs_set_traversal_stack": ([P, I32], I32),
        "nrrs_traversal_stack_info": ([P, P, P], I32),
        "nrrs_set_bvh_builder": ([P, I32, P], I32),
        "nrrs_bvh8_info": ([P, P], I32),
        "nrrs_bvh8_export": ([P, P, I64, P, I64], I32),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


_lib = _load()


def lib():
    return _lib


def _ptr(x):
    """Device address of a torch tensor (or an int address, or None)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(s):
    if s is None:
        try:
            import torch

            return torch.cuda.current_stream().cuda_stream
        except Exception:  # pragma: no cover - torch without CUDA
            return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(rc):
    if rc != NRRS_OK:
        raise NrrsError(rc, _lib.nrrs_last_error().decode())
    return rc


# ------------------------------------------------------------------ ABI functions
def nrrs_status_string(code):
    return _lib.nrrs_status_string(code).decode()


def nrrs_last_error():
    return _lib.nrrs_last_error().decode()


def nrrs_create_scene(tri, tri_mat, mats, cam, device=0):
    tri = np.ascontiguousarray(tri, dtype=np.float32).reshape(-1, 9)
    tri_mat = np.ascontiguousarray(tri_mat, dtype=np.int32)
    mats = np.ascontiguousarray(mats)
    cam = np.ascontiguousarray(cam)
    assert mats.dtype.itemsize == 40 and cam.dtype.itemsize == 40
    out = C.c_void_p()
    _check(_lib.nrrs_create_scene(tri.ctypes.data, tri.shape[0], tri_mat.ctypes.data,
                                  mats.ctypes.data, len(mats), cam.ctypes.data, device,
                                  C.byref(out)))
    return out.value


def nrrs_create_batch(jobs, device=0):
    """jobs: sequence of (inputs.Scene, width, height, spp, max_depth)."""
    keep = []
    arr = (Job * len(jobs))()
    for k, (sc, w, h, spp, D) in enumerate(jobs):
        tri = np.ascontiguousarray(sc.tri, dtype=np.float32).reshape(-1, 9)
        tm = np.ascontiguousarray(sc.mat_id, dtype=np.int32)
        mats = np.ascontiguousarray(sc.mats)
        cam = np.ascontiguousarray(sc.cam)
        keep += [tri, tm, mats, cam]
        arr[k] = Job(tri.ctypes.data, tri.shape[0], tm.ctypes.data, mats.ctypes.data, len(mats),
                     cam.ctypes.data, w, h, spp, D)
    out = C.c_void_p()
    _check(_lib.nrrs_create_batch(arr, len(jobs), device, C.byref(out)))
    return out.value


def nrrs_render_batch(batch, rrs_mode, opts, d_rgb, n_jobs, stream=None, stats=True):
    st = RenderStats() if stats else None
    live = np.zeros((n_jobs, MAX_DEPTH), dtype=np.int64)
    F = np.zeros((n_jobs, MAX_DEPTH), dtype=np.float32)
    sq = np.zeros((n_jobs, MAX_DEPTH), dtype=np.float64)
    _check(_lib.nrrs_render_batch(batch, rrs_mode, C.byref(opts) if opts is not None else None,
                                  _ptr(d_rgb), _stream(stream),
                                  C.byref(st) if st is not None else None, live.ctypes.data,
                                  F.ctypes.data, sq.ctypes.data))
    return (st.as_dict(MAX_DEPTH) if st is not None else None), live, F, sq


def nrrs_batch_info(batch):
    n = C.c_int32()
    total = C.c_int64()
    _check(_lib.nrrs_batch_info(batch, C.byref(n), None, C.byref(total)))
    base = np.zeros(max(n.value, 1), dtype=np.int64)
    _check(_lib.nrrs_batch_info(batch, None, base.ctypes.data, None))
    return n.value, base[:n.value], total.value


def nrrs_set_traversal(scene, width):
    _check(_lib.nrrs_set_traversal(scene, width))


def nrrs_set_bvh_precision(scene, bits):
    _check(_lib.nrrs_set_bvh_precision(scene, bits))


def nrrs_set_shade_fusion(scene, on):
    _check(_lib.nrrs_set_shade_fusion(scene, on))


def nrrs_set_traversal_stack(scene, entries):
    _check(_lib.nrrs_set_traversal_stack(scene, entries))


def nrrs_traversal_stack_info(scene):
    """(BVH2 height, stack entries per ray in use)."""
    h, e = C.c_int32(), C.c_int32()
    _check(_lib.nrrs_traversal_stack_info(scene, C.byref(h), C.byref(e)))
    return h.value, e.value


def nrrs_set_bvh_builder(scene, builder):
    """Rebuilds the BVH2 with builder 0 (host binned SAH) or 1 (device PLOC); returns
    the build's wall time in ms."""
    ms = C.c_float()
    _check(_lib.nrrs_set_bvh_builder(scene, builder, C.byref(ms)))
    return ms.value


def nrrs_destroy_scene(scene):
    _check(_lib.nrrs_destroy_scene(scene))


def nrrs_scene_info(scene):
    nn, nt = C.c_int64(), C.c_int64()
    _check(_lib.nrrs_scene_info(scene, C.byref(nn), C.byref(nt)))
    return nn.value, nt.value


def nrrs_set_rrsnet_params(scene, params, stream=None):
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(_lib.nrrs_set_rrsnet_params(scene, p.ctypes.data, p.size, _stream(stream)))


def nrrs_get_rrsnet_params(scene, stream=None, n=RRSNET_PARAMS):
    """The rendering weights of RRSNet (AID_RRSNET_PARAMS with the AID-NRRS inputs)."""
    p = np.zeros(n, dtype=np.float32)
    _check(_lib.nrrs_get_rrsnet_params(scene, p.ctypes.data, p.size, _stream(stream)))
    return p


def nrrs_render(scene, width, height, spp, max_depth, rrs_mode, opts, d_rgb, stream=None,
                stats=True):
    st = RenderStats() if stats else None
    _check(_lib.nrrs_render(scene, width, height, spp, max_depth, rrs_mode,
                            C.byref(opts) if opts is not None else None, _ptr(d_rgb),
                            _stream(stream), C.byref(st) if st is not None else None))
    return st.as_dict(max_depth) if st is not None else None


def nrrs_query_factors(scene, d_features, n, precision, d_q, stream=None):
    _check(_lib.nrrs_query_factors(scene, _ptr(d_features), n, precision, _ptr(d_q),
                                   _stream(stream)))


def nrrs_normalize(scene, d_q, n, budget, f_rate, alpha, d_F, d_sum, stream=None):
    _check(_lib.nrrs_normalize(scene, _ptr(d_q), n, budget, f_rate, alpha, _ptr(d_F),
                               _ptr(d_sum), _stream(stream)))


def nrrs_split(scene, d_q_orig, n, d_F, d_pixel, d_sample, d_lineage, depth, seed_lo, seed_hi,
               frame, cap, d_X, d_prefix, d_child_parent, d_child_lineage, d_total, d_dropped,
               stream=None):
    _check(_lib.nrrs_split(scene, _ptr(d_q_orig), n, _ptr(d_F), _ptr(d_pixel), _ptr(d_sample),
                           _ptr(d_lineage), depth, seed_lo, seed_hi, frame, cap, _ptr(d_X),
                           _ptr(d_prefix), _ptr(d_child_parent), _ptr(d_child_lineage),
                           _ptr(d_total), _ptr(d_dropped), _stream(stream)))


def nrrs_split_noalloc(d_q_orig, n, d_F, d_pixel, d_sample, d_lineage, depth, seed_lo, seed_hi,
                       frame, cap, d_X, d_prefix, d_child_parent, d_child_lineage, d_total,
                       d_dropped, stream=None):
    """nrrs_split for callers that cannot allocate device memory on the call path; its
    scratch is a fixed array inside the library (n <= 67,108,864).  Runs on the current
    device; the first call on a device must precede any stream capture."""
    _check(_lib.nrrs_split_noalloc(_ptr(d_q_orig), n, _ptr(d_F), _ptr(d_pixel), _ptr(d_sample),
                                   _ptr(d_lineage), depth, seed_lo, seed_hi, frame, cap,
                                   _ptr(d_X), _ptr(d_prefix), _ptr(d_child_parent),
                                   _ptr(d_child_lineage), _ptr(d_total), _ptr(d_dropped),
                                   _stream(stream)))


def nrrs_train_step(scene, opts=None, stream=None):
    st = TrainStats()
    _check(_lib.nrrs_train_step(scene, C.byref(opts) if opts is not None else None,
                                _stream(stream), C.byref(st)))
    return st.as_dict()


def nrrs_set_params(scene, which, params, stream=None):
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(_lib.nrrs_set_params(scene, which, p.ctypes.data, p.size, _stream(stream)))


def nrrs_get_params(scene, which, stream=None, n=None):
    """Weights of network `which`; StatNet on the encodings has STATNET_GRID_PARAMS (pass
    n), its grid GRID_PARAMS."""
    if n is None:
        n = {NET_STATNET: STATNET_PARAMS, NET_STATNET_GRID: GRID_PARAMS,
             NET_RRSNET_GRID: GRID_PARAMS, NET_RRSNET_GRID_TRAIN: GRID_PARAMS}.get(which,
                                                                                    RRSNET_PARAMS)
    p = np.zeros(n, dtype=np.float32)
    _check(_lib.nrrs_get_params(scene, which, p.ctypes.data, n, _stream(stream)))
    return p


def nrrs_mlp_grad(scene, n_out, d_params, d_x, d_gout, n, d_grad, stream=None):
    _check(_lib.nrrs_mlp_grad(scene, n_out, _ptr(d_params), _ptr(d_x), _ptr(d_gout), n,
                              _ptr(d_grad), _stream(stream)))


def nrrs_tune_rrsnet(scene, precision, stream=None):
    rep = TuneReport()
    _check(_lib.nrrs_tune_rrsnet(scene, precision, _stream(stream), C.byref(rep)))
    return rep.as_dict()


def nrrs_set_rrsnet_shape(scene, precision, bucket, variant, blocks_per_sm):
    _check(_lib.nrrs_set_rrsnet_shape(scene, precision, bucket, variant, blocks_per_sm))


def nrrs_rrsnet_forward(d_params, d_x, n, d_q, stream=None):
    _check(_lib.nrrs_rrsnet_forward(_ptr(d_params), _ptr(d_x), n, _ptr(d_q), _stream(stream)))


def nrrs_rrsnet_backward(scene, d_params, d_x, d_gq, n, d_grad, stream=None):
    _check(_lib.nrrs_rrsnet_backward(scene, _ptr(d_params), _ptr(d_x), _ptr(d_gq), n,
                                     _ptr(d_grad), _stream(stream)))


def _rrsnet_function():
    import torch

    class RRSNetFunction(torch.autograd.Function):
        """q = RRSNet(x; W) with the forward and the weight gradient computed by the
        library's kernels (nrrs_rrsnet_forward / nrrs_rrsnet_backward).  Features are not
        differentiated (they come from the renderer)."""

        @staticmethod
        def forward(ctx, scene, x, params):
            x = x.contiguous()
            params = params.contiguous()
            q = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
            nrrs_rrsnet_forward(params, x, x.shape[0], q)
            ctx.scene = scene
            ctx.save_for_backward(x, params)
            return q

        @staticmethod
        def backward(ctx, gq):
            x, params = ctx.saved_tensors
            grad = torch.empty_like(params)
            nrrs_rrsnet_backward(ctx.scene, params, x, gq.contiguous(), x.shape[0], grad)
            return None, None, grad

    return RRSNetFunction


_RRSNET_FN = None


def rrsnet(scene, x, params):
    """Differentiable RRSNet: x [n][16] float32 CUDA, params [2592] float32 CUDA (requires
    grad for training) -> q [n].  `scene` supplies the backward's scratch buffers."""
    global _RRSNET_FN
    if _RRSNET_FN is None:
        _RRSNET_FN = _rrsnet_function()
    handle = scene.handle if hasattr(scene, "handle") else scene
    return _RRSNET_FN.apply(handle, x, params)


def nrrs_rrsnet_dloss(d_q_nrrs, d_F, d_Fn, d_t, d_pixel, d_m1, d_m2, d_E, Ebar, d_Iref, d_k, n,
                      eps, g1, g2, g3, d_dq, stream=None):
    _check(_lib.nrrs_rrsnet_dloss(_ptr(d_q_nrrs), _ptr(d_F), _ptr(d_Fn), _ptr(d_t), _ptr(d_pixel),
                                  _ptr(d_m1), _ptr(d_m2), _ptr(d_E), float(Ebar), _ptr(d_Iref),
                                  _ptr(d_k), n, eps, g1, g2, g3, _ptr(d_dq), _stream(stream)))


def nrrs_adam_step(d_params, d_grad, d_m, d_v, n, step, lr, b1=0.9, b2=0.999, eps=1e-8,
                   stream=None):
    _check(_lib.nrrs_adam_step(_ptr(d_params), _ptr(d_grad), _ptr(d_m), _ptr(d_v), n, step, lr,
                               b1, b2, eps, _stream(stream)))


def nrrs_ema(d_avg, d_params, n, decay, stream=None):
    _check(_lib.nrrs_ema(_ptr(d_avg), _ptr(d_params), n, decay, _stream(stream)))


def nrrs_bvh8_info(scene):
    st = Bvh8Stats()
    _check(_lib.nrrs_bvh8_info(scene, C.byref(st)))
    return st.as_dict()


def nrrs_bvh8_export(scene):
    """Host copies of the eight-wide tree: nodes [n][20] uint32, tris [n_tri][12] float32."""
    info = nrrs_bvh8_info(scene)
    nodes = np.zeros((max(1, info["nodes"]), 20), dtype=np.uint32)
    tris = np.zeros((max(1, info["triangles"]), 12), dtype=np.float32)
    _check(_lib.nrrs_bvh8_export(scene, nodes.ctypes.data, nodes.shape[0], tris.ctypes.data,
                                 tris.shape[0]))
    return nodes, tris


def nrrs_mixdepth_candidates(max_depth, t_d):
    return int(_lib.nrrs_mixdepth_candidates(max_depth, t_d))


def nrrs_mixdepth_search(scene, width, height, max_depth, t_d=6, spp=1, seed=(1, 0), frame=0,
                         d_pixel_ref=None, max_candidates=0, adrrs=0, nee=0, precision=32,
                         stream=None):
    o = MixDepthOpts(width, height, spp, max_depth, t_d, max_candidates, seed[0], seed[1], frame,
                     _ptr(d_pixel_ref), adrrs, nee, precision)
    r = MixDepthResult()
    _check(_lib.nrrs_mixdepth_search(scene, C.byref(o), _stream(stream), C.byref(r)))
    return {name: getattr(r, name) for name, _ in r._fields_}


def nrrs_set_rrsnet_inputs(scene, mode):
    _check(_lib.nrrs_set_rrsnet_inputs(scene, mode))


def nrrs_set_statnet_encoding(scene, mode):
    _check(_lib.nrrs_set_statnet_encoding(scene, mode))


def nrrs_statnet_grad(scene, d_params, d_x, d_gout, n, d_grad, stream=None):
    _check(_lib.nrrs_statnet_grad(scene, _ptr(d_params), _ptr(d_x), _ptr(d_gout), n, _ptr(d_grad),
                                  _stream(stream)))


def nrrs_statnet_inputs(scene, d_feat, d_rough, n, d_x, stream=None):
    _check(_lib.nrrs_statnet_inputs(scene, _ptr(d_feat), _ptr(d_rough), n, _ptr(d_x),
                                    _stream(stream)))


def nrrs_grid_backward(scene, d_feat, d_dx, n, d_grad, stream=None):
    _check(_lib.nrrs_grid_backward(scene, _ptr(d_feat), _ptr(d_dx), n, _ptr(d_grad),
                                   _stream(stream)))


def nrrs_error_filter(d_in, d_normals, width, height, radius, power, d_out, stream=None):
    _check(_lib.nrrs_error_filter(_ptr(d_in), _ptr(d_normals), width, height, radius, power,
                                  _ptr(d_out), _stream(stream)))


def nrrs_relmse(d_img, d_ref, n_pixels, eps, d_out, stream=None):
    _check(_lib.nrrs_relmse(_ptr(d_img), _ptr(d_ref), n_pixels, eps, _ptr(d_out), _stream(stream)))


def gate_methods(gate, max_depth):
    """Per-depth method names of a Mix-Depth gate."""
    names = {GATE_NET: "NET", GATE_HEUR: "HEUR", GATE_FIXED: "FIXED", GATE_ADRRS: "ADRRS"}
    return [names[(gate >> (2 * d)) & 3] for d in range(max_depth)]


# ------------------------------------------------------------------ convenience wrapper
class Batch:
    """Owns a batch scene of many render jobs: ``jobs`` is a sequence of
    (inputs.Scene, width, height, spp, max_depth)."""

    def __init__(self, jobs, device=0):
        self.handle = nrrs_create_batch(jobs, device)
        self.device = device
        self.shapes = [(h, w) for (_, w, h, _, _) in jobs]
        self.max_depth = max(j[4] for j in jobs)
        self.n_jobs, self.pixel_base, self.n_pixels = nrrs_batch_info(self.handle)

    def close(self):
        if self.handle:
            nrrs_destroy_scene(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        nrrs_set_rrsnet_params(self.handle, params)

    def tune(self, precision=32, stream=None):
        return nrrs_tune_rrsnet(self.handle, precision, stream)

    def render(self, mode, out=None, stream=None, **opts):
        """One frame of every job; returns (list of per-job [H, W, 3] views of the output,
        totals, per-job live [n][32], per-job F, per-job sum of q)."""
        import torch

        if out is None:
            out = torch.empty((self.n_pixels, 3), dtype=torch.float32,
                              device=f"cuda:{self.device}")
        st, live, F, sq = nrrs_render_batch(self.handle, mode, RenderOpts.defaults(**opts), out,
                                            self.n_jobs, stream)
        imgs = [out[b:b + h * w].view(h, w, 3) for b, (h, w) in zip(self.pixel_base, self.shapes)]
        return imgs, st, live, F, sq


class Scene:
    """Owns one nrrs_scene handle built from an ``inputs.Scene``."""

    def __init__(self, scene, device=0):
        self.handle = nrrs_create_scene(scene.tri, scene.mat_id, scene.mats, scene.cam, device)
        self.device = device
        self.n_tri = scene.n_tri

    def close(self):
        if self.handle:
            nrrs_destroy_scene(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        nrrs_set_rrsnet_params(self.handle, params)

    def get_params(self):
        return nrrs_get_rrsnet_params(self.handle)

    def render(self, width, height, spp, max_depth, mode, out=None, stats=True, stream=None,
               **opts):
        import torch

        if out is None:
            out = torch.empty((height, width, 3), dtype=torch.float32, device=f"cuda:{self.device}")
        o = RenderOpts.defaults(**opts)
        st = nrrs_render(self.handle, width, height, spp, max_depth, mode, o, out, stream, stats)
        return out, st

    def tune(self, precision=32, stream=None):
        return nrrs_tune_rrsnet(self.handle, precision, stream)

    def set_traversal(self, width):
        nrrs_set_traversal(self.handle, width)

    def set_bvh_precision(self, bits):
        nrrs_set_bvh_precision(self.handle, bits)

    def set_traversal_stack(self, entries):
        nrrs_set_traversal_stack(self.handle, entries)

    def traversal_stack_info(self):
        return nrrs_traversal_stack_info(self.handle)

    def set_shade_fusion(self, on):
        nrrs_set_shade_fusion(self.handle, int(on))

    def set_bvh_builder(self, builder):
        return nrrs_set_bvh_builder(self.handle, builder)

    def set_rrsnet_inputs(self, mode):
        nrrs_set_rrsnet_inputs(self.handle, mode)

    def set_statnet_encoding(self, mode):
        nrrs_set_statnet_encoding(self.handle, mode)

    def train_step(self, stream=None, **opts):
        return nrrs_train_step(self.handle, TrainOpts.defaults(**opts), stream)

    def query(self, features, precision=32, out=None, stream=None):
        import torch

        n = features.shape[0]
        if out is None:
            out = torch.empty(n, dtype=torch.float32, device=features.device)
        nrrs_query_factors(self.handle, features, n, precision, out, stream)
        return out
