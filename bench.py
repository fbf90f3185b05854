"""Benchmark of the NRRS bounce loop on B300.

Headline (`value`): the Mix-Depth workload on one GPU -- the three-room scene with
1,000,000 random triangles (60 % GGX) joined by narrow doorways, 1920 x 1080 px, depth
32, 128 spp rendered as 8 frames of 16 spp.  A step is one 16-spp frame through
nrrs_render (camera rays, then per depth the traversal, shading, RRSNet at the depths
the Mix-Depth gate marks -- BF16 tensor cores, fused with the shading of those depths --
and heuristic factors
elsewhere, normalization, split counts with the per-pixel accumulation, compaction and
BSDF sampling of the children, the frame estimate), graph-captured, with the launch
shapes the autotuner chose per queue-size bucket.  Set-up, untimed: the BVH build,
online training of RRSNet and StatNet on 480 x 270 x 4 spp frames of the same scene,
the tuner, and the Mix-Depth search on 480 x 270 x 1 spp renders.

`value` is path segments per second (rays traced, summed over depths and ranks) with the
scene, weights and queues resident on the device; `e2e` is the same metric through the
public API with the weights copied from pinned host memory and the frame read back every
step.  Second section, `online_step`: the online NRRS step on the occluded room (2,018
triangles, 256 x 256 px, 16 spp, depth 16): nrrs_train_step on a recorded 256 x 256 x
2 spp frame plus the 16-spp inference frame, with the estimators' efficiency
1 / (relMSE x s) over several seeds.  `--impl reference` times the FP64 CPU oracle on
the host cores on a bounded crop of the headline workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "efficiency 1/(relMSE·s) vs plain RR, same B300; path segments/s; RRSNet TFLOP/s"
UNIT = "path segments/s"
# headline: the Mix-Depth configuration
HL_W, HL_H, HL_SPP, HL_DEPTH = 1920, 1080, 16, 32
HL_FRAMES = 8                        # 8 frames x 16 spp = 128 spp
HL_TRAIN = (480, 270, 4)             # online training frames of the same scene
HL_PRETRAIN = 200                    # untimed training steps before the search
HL_SEARCH = (480, 270)               # Mix-Depth estimation renders (1 spp)
HL_PRECISION = 17                    # RRSNet on the tensor cores, BF16 operands
HL_WORKLOAD = ("three_rooms (1,000,000 random triangles, 60 % GGX) 1920x1080 px, depth 32, "
               "128 spp as 8 frames x 16 spp; step = one 16-spp frame, NET_MIX (searched "
               "Mix-Depth gate), RRSNet BF16 tensor cores fused with shading at gated depths, heuristic "
               "elsewhere, tuned launch shapes, CUDA-graph bounce loop, cap 2*P")
# second section: the online training step
W_IMG, H_IMG, SPP, DEPTH = 256, 256, 16, 16
TRAIN_SPP = 2          # recorded training frame: 256x256x2 spp ~ 2^19 training vertices
PRETRAIN_STEPS = 300   # untimed online training before the timed steps (20 warm-up + 280 full)
ONLINE_PRECISION = 17  # inference frame's RRSNet: BF16 tensor cores
WORKLOAD = ("occluded_room 256x256 px, 16 spp, depth 16, RRSNet BF16 tensor-core factors "
            "(NET), budget P, cap 2*P; step = online RRSNet/StatNet training step on a recorded "
            "256x256x2 spp frame + the 16 spp inference frame")
EFF_SEEDS = 5          # independent render seeds per estimator in the efficiency tables
# algorithmic bytes per unit of each stage
BYTES_PER_RAY_EXTEND = 32 + 16                  # ray in, hit record out
BYTES_PER_RAY_SHADE = 48 + 8 + 4 + 16           # path state, hit in; q, deposit out
BYTES_PER_SLOT_DEPOSIT = 16                     # last depth: deposit only
BYTES_PER_PARENT_SPLIT = 16 + 4 + 48 + 8        # deposit, q, path state, hit
BYTES_PER_CHILD_SPLIT = 48                      # child path state
RRSNET_FLOP_PER_PATH = 2 * (16 * 32 + 32 * 32 + 32 * 32 + 32)


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p["bf16_tflops"]), "measured"
    except Exception:
        return 6400.0, 1800.0, "fallback"


class ClockSampler:
    """SM clocks and clock-event (throttle) reasons during the timed region: NVML in a
    background thread when pynvml is importable, else an `nvidia-smi -lms 50` subprocess
    started before the warm-up and filtered to the timed window by timestamp."""

    REASONS = {"hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40,
               "sw_power_cap": 0x4}
    SMI_FIELDS = ("timestamp,clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
                  "clocks_event_reasons.hw_thermal_slowdown,"
                  "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.reasons = set()
        self.max_mhz = None
        self.error = None
        self._stop = None
        self._proc = None
        self._t0 = self._t1 = None

    def launch(self):
        """Start sampling (call before the warm-up so samples exist when timing starts)."""
        import threading

        try:
            import pynvml

            pynvml.nvmlInit()
            h = pynvml.nvmlDeviceGetHandleByIndex(self.index)
            self.max_mhz = float(pynvml.nvmlDeviceGetMaxClockInfo(h, pynvml.NVML_CLOCK_SM))
        except Exception as e:
            self.error = f"pynvml: {type(e).__name__}"
            self._launch_smi()
            return
        self._stop = threading.Event()

        def loop():
            while not self._stop.is_set():
                try:
                    now = time.time()
                    mhz = float(pynvml.nvmlDeviceGetClockInfo(h, pynvml.NVML_CLOCK_SM))
                    bits = pynvml.nvmlDeviceGetCurrentClocksThrottleReasons(h)
                    self.samples.append((now, mhz, bits))
                except Exception as e:
                    self.error = f"{type(e).__name__}: {e}"
                self._stop.wait(0.01)

        self._t = threading.Thread(target=loop, daemon=True)
        self._t.start()

    def _launch_smi(self):
        try:
            # the raw samples go to $NRRS_CLOCKS_DIR (default: the system temp folder)
            out_dir = os.environ.get("NRRS_CLOCKS_DIR", tempfile.gettempdir())
            os.makedirs(out_dir, exist_ok=True)
            self._path = os.path.join(out_dir, f"clocks_gpu{self.index}.csv")
            self._f = open(self._path, "w")
            self._proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.SMI_FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"], stdout=self._f,
                stderr=subprocess.DEVNULL)
            time.sleep(1.0)  # first samples before the timed region
        except Exception as e:
            self.error = (self.error or "") + f"; nvidia-smi: {type(e).__name__}"
            self._proc = None

    def start(self):
        self._t0 = time.time()

    def stop(self):
        self._t1 = time.time()
        if self._stop is not None:
            self._stop.set()
            self._t.join(timeout=2)
            names = {b: n for n, b in self.REASONS.items()}
            sm = []
            for t, mhz, bits in self.samples:
                if self._t0 - 0.05 <= t <= self._t1 + 0.05:
                    sm.append(mhz)
                    for b, n in names.items():
                        if bits & b:
                            self.reasons.add(n)
            return self._summary(sm)
        if self._proc is not None:
            time.sleep(0.2)
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except Exception:
                self._proc.kill()
            self._f.close()
            return self._parse_smi()
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"],
                "error": self.error}

    def _parse_smi(self):
        import datetime

        sm, smax = [], []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self._path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                mhz, mx = float(parts[1]), float(parts[2])
            except ValueError:
                continue
            if not (self._t0 - 0.1 <= ts <= self._t1 + 0.1):
                continue
            sm.append(mhz)
            smax.append(mx)
            for name, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    self.reasons.add(name)
        self.max_mhz = max(smax) if smax else None
        return self._summary(sm)

    def _summary(self, sm):
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["unsampled"],
                    "error": self.error}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": self.max_mhz,
                "reasons": sorted(self.reasons), "samples": len(sm)}


def profile_record(kernel_tag, key):
    """A figure `key` per unit recorded from an ncu capture of `kernel_tag` in profiles/
    (lines `<key> <tag> source_sha=<sha> value=<x>`), if the recorded source hash still
    matches the current kernel source (else None).  The traversal's hash covers its
    kernel file and the BVH builder that lays out what it reads."""
    csrc = os.path.join(ROOT, "paper_2510_07868_b300", "csrc")
    files = {"extend": ["trace.cu", "bvh.cpp"]}.get(kernel_tag, ["wavefront.cu"])
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(csrc, f), "rb").read())
    sha = h.hexdigest()[:12]
    pdir = os.path.join(ROOT, "profiles")
    for fn in sorted(os.listdir(pdir)) if os.path.isdir(pdir) else []:
        if not fn.endswith((".md", ".txt")):
            continue
        for line in open(os.path.join(pdir, fn)):
            m = re.match(r"(\w+)\s+(\S+)\s+source_sha=(\w+)\s+value=([\d.eE+-]+)", line.strip("` \n"))
            if m and m.group(1) == key and m.group(2) == kernel_tag and m.group(3) == sha:
                return float(m.group(4))
    return None


def source_sha(kernel_tag):
    csrc = os.path.join(ROOT, "paper_2510_07868_b300", "csrc")
    files = {"extend": ["trace.cu", "bvh.cpp"]}.get(kernel_tag, ["wavefront.cu"])
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:12]


# ------------------------------------------------------------------ CPU oracle legs
def crop_pixels(side, W=None, H=None):
    """Pixel ids of a side x side window at the image centre."""
    W, H = W or HL_W, H or HL_H
    x0, y0 = (W - side) // 2, (H - side) // 2
    ys, xs = np.meshgrid(np.arange(y0, y0 + side), np.arange(x0, x0 + side), indexing="ij")
    return (ys * W + xs).ravel().astype(np.int32)


def oracle_headline_sample(scene, params, gate, pixel_ref, forced_F, seconds_target=15.0,
                           frame=0):
    """Times the FP64 oracle on a centred crop of the headline frame at 1 spp (same scene,
    depth, mode and gate), growing the crop toward `seconds_target` of work; returns
    (segments/s, cores, sample description, seconds, side)."""
    import oracle

    side = 8
    while True:
        pix = crop_pixels(side)
        t0 = time.perf_counter()
        _, st, _ = oracle.render(scene, HL_W, HL_H, 1, HL_DEPTH, oracle.MODE_NET_MIX,
                                 params=params, gate=gate, pixel_ref=pixel_ref, pixels=pix,
                                 forced_F=forced_F, frame=frame)
        dt = time.perf_counter() - t0
        if dt >= 0.25 * seconds_target or side >= 128:
            break
        side = int(min(128, side * min(2.0, np.sqrt(seconds_target / max(dt, 1e-3)))))
    cores = _env_int("OMP_NUM_THREADS", os.cpu_count() or 1)
    desc = (f"three_rooms centred {side}x{side} px crop of {HL_W}x{HL_H} at 1 spp (the GPU step "
            f"renders 16 spp over {HL_W * HL_H:,} px), depth 32, NET_MIX; {st['segments']} segments "
            f"in {dt:.2f} s")
    return st["segments"] / dt, cores, desc, dt, side


def reference_gate():
    """The fixed Mix-Depth gate the reference arm uses (it cannot train): FIXED at depths
    1-2, RRSNet at depths 3-8, the heuristic beyond."""
    g = 0
    for d in range(HL_DEPTH):
        m = 2 if d < 2 else 0 if d < 8 else 1  # NRRS_GATE_FIXED / _NET / _HEUR
        g |= m << (2 * d)
    return g


def run_reference(args, rank, world):
    if rank != 0:
        return
    os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))
    import oracle
    from paper_2510_07868_b300 import inputs as I

    oracle.build()
    scene = I.three_rooms(1)
    params = I.rrsnet_init_params(2).astype(np.float64)
    gate = reference_gate()
    per_step = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    # a crop cannot see the whole frame's sum of factors: F = 1 at every depth (the frame's
    # own F stays near 1 here, its budget 2 P being far above the factors' sum)
    F1 = np.ones(HL_DEPTH, dtype=np.float32)
    _, _, _, _, side = oracle_headline_sample(scene, params, gate, None, F1,
                                              seconds_target=per_step)
    pix = crop_pixels(side)
    for k in range(args.warmup):
        oracle.render(scene, HL_W, HL_H, 1, HL_DEPTH, oracle.MODE_NET_MIX, params=params,
                      gate=gate, pixels=pix, forced_F=F1, frame=k)
    segs = 0
    t0 = time.perf_counter()
    for k in range(args.steps):
        _, st, _ = oracle.render(scene, HL_W, HL_H, 1, HL_DEPTH, oracle.MODE_NET_MIX,
                                 params=params, gate=gate, pixels=pix, forced_F=F1,
                                 frame=args.warmup + k)
        segs += st["segments"]
    dt = time.perf_counter() - t0
    value = segs / dt
    cores = _env_int("OMP_NUM_THREADS", os.cpu_count() or 1)
    sample = (f"three_rooms centred {side}x{side} px crop of {HL_W}x{HL_H} per step at 1 spp, depth "
              f"32, NET_MIX with a fixed gate (FIXED 1-2, RRSNet 3-8, heuristic beyond) and "
              f"the untrained RRSNet (the oracle cannot train; its cost per segment does not "
              f"depend on the weights' values)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": HL_WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU leg
def replica_seed(rank):
    """Philox key high word of a replica: every rank renders other random numbers."""
    return rank


def combine_ranks(dist, device, ms, e2e_s, segs, e2e_segs):
    """Whole-job figures of N replicas: the slowest rank's times (max over ranks) and the
    path segments every rank traced (sum), so value = all segments / the slowest time."""
    import torch

    t = torch.tensor([ms, e2e_s], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([segs, e2e_segs], dtype=torch.float64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t[0]), float(t[1]), int(c[0]), int(c[1])


def mean_se(xs):
    x = np.asarray(xs, dtype=np.float64)
    return float(x.mean()), float(x.std(ddof=1) / np.sqrt(len(x))) if len(x) > 1 else 0.0


def efficiency_section(nrrs, sc, torch, dev, stream, seed_hi, nee=0, seeds=EFF_SEEDS,
                       precisions=(32,)):
    """1/(relMSE x seconds) of the estimators on the same B300 -- PLAIN_RR (throughput
    roulette), HEUR_NORM (plain normalised RRS), NET (trained RRSNet at every depth),
    ADRRS_NN (StatNet's radiance over the pixel estimate at every depth), NET_MIX (the
    Mix-Depth gate over FIXED / HEUR / NET) and NET_MIX_ADRRS (over FIXED / ADRRS (NN) /
    NET, the paper's set), NET and NET_MIX again at every tensor-core precision asked
    for (17 = BF16, 16 = split BF16, 8 = E4M3) -- each averaging 16 frames of 16 spp, against a
    4096-spp plain path-traced reference (256 frames x 16 spp, no RRS), repeated with
    `seeds` independent render seeds: mean and standard error per estimator.  nee=1:
    every render, the reference and the Mix-Depth searches with next-event estimation."""
    ref = torch.zeros((H_IMG, W_IMG, 3), dtype=torch.float64, device=dev)
    img = torch.empty((H_IMG, W_IMG, 3), dtype=torch.float32, device=dev)
    n_ref = 256
    for f in range(n_ref):
        nrrs.nrrs_render(sc.handle, W_IMG, H_IMG, SPP, DEPTH, nrrs.RRS_NONE,
                         nrrs.RenderOpts.defaults(frame=50_000 + f, seed_hi=seed_hi + 1000,
                                                  update_ref=0, nee=nee),
                         img, stream, False)
        ref += img
    ref32 = (ref / n_ref).float().contiguous()
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    t0 = time.perf_counter()
    gates = {}
    for prec in precisions:
        gates[prec] = nrrs.nrrs_mixdepth_search(sc.handle, W_IMG, H_IMG, DEPTH, t_d=6,
                                                frame=777, d_pixel_ref=None, nee=nee,
                                                precision=prec, stream=stream)
    search_s = time.perf_counter() - t0
    # the paper's candidate set per depth: FIXED, ADRRS (NN), NRRS
    gate_adrrs = nrrs.nrrs_mixdepth_search(sc.handle, W_IMG, H_IMG, DEPTH, t_d=6, frame=777,
                                           d_pixel_ref=None, adrrs=1, nee=nee, stream=stream)
    all_adrrs = sum(nrrs.GATE_ADRRS << (2 * d) for d in range(DEPTH))
    modes = [("PLAIN_RR", nrrs.RRS_PLAIN_RR, 0, 32), ("HEUR_NORM", nrrs.RRS_HEUR_NORM, 0, 32),
             ("ADRRS_NN", nrrs.RRS_NET_MIX, all_adrrs, 32),
             ("NET_MIX_ADRRS", nrrs.RRS_NET_MIX, gate_adrrs["gate"], 32)]
    tag = {32: "", 17: "_BF16", 16: "_BF16X3", 8: "_E4M3"}
    for prec in precisions:
        modes.append(("NET" + tag[prec], nrrs.RRS_NET, 0, prec))
        modes.append(("NET_MIX" + tag[prec], nrrs.RRS_NET_MIX, gates[prec]["gate"], prec))
    frames = 16
    res = {}
    for name, mode, gate, prec in modes:
        per = {"relmse": [], "seconds": [], "efficiency": [], "segments": [], "ray_efficiency": []}
        # one untimed frame first, so that no mode's time holds its first graph capture
        nrrs.nrrs_render(sc.handle, W_IMG, H_IMG, SPP, DEPTH, mode,
                         nrrs.RenderOpts.defaults(frame=89_999, seed_hi=seed_hi, gate=gate,
                                                  update_ref=0, nee=nee, precision=prec,
                                                  graph=1),
                         img, stream, True)
        for k in range(seeds):
            acc = torch.zeros((H_IMG, W_IMG, 3), dtype=torch.float64, device=dev)
            segs = 0
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for f in range(frames):
                st = nrrs.nrrs_render(sc.handle, W_IMG, H_IMG, SPP, DEPTH, mode,
                                      nrrs.RenderOpts.defaults(frame=90_000 + f,
                                                               seed_hi=seed_hi + 17 * k,
                                                               gate=gate, update_ref=0, nee=nee,
                                                               precision=prec, graph=1),
                                      img, stream, True)
                segs += st["segments"]
                acc += img
            e1.record(stream)
            torch.cuda.synchronize()
            sec = e0.elapsed_time(e1) / 1000.0
            mean = (acc / frames).float().contiguous()
            nrrs.nrrs_relmse(mean, ref32, W_IMG * H_IMG, 0.01, out, stream)
            torch.cuda.synchronize()
            rel = out.item()
            per["relmse"].append(rel)
            per["seconds"].append(sec)
            per["efficiency"].append(1.0 / (rel * sec))
            per["segments"].append(segs)
            per["ray_efficiency"].append(1.0 / (rel * segs))
        res[name] = {}
        for key, xs in per.items():
            m, se = mean_se(xs)
            res[name][key] = m
            res[name][key + "_se"] = se
    base = res["PLAIN_RR"]["efficiency"]
    heur = res["HEUR_NORM"]["efficiency"]
    summary = {
        "reference": f"no-RRS path tracing{' with NEE' if nee else ''}, {n_ref * SPP} spp",
        "frames_per_seed": frames, "seeds": seeds, "modes": res,
        "mixdepth_gates": {str(p): nrrs.gate_methods(g["gate"], DEPTH) for p, g in gates.items()},
        "mixdepth_gate_adrrs": nrrs.gate_methods(gate_adrrs["gate"], DEPTH),
        "mixdepth_candidates": gates[precisions[0]]["evaluated"], "mixdepth_search_s": search_s,
    }
    for name in res:
        if name not in ("PLAIN_RR", "HEUR_NORM"):
            summary[name.lower() + "_vs_heur_norm"] = res[name]["efficiency"] / heur
    summary["heur_norm_vs_plain_rr"] = heur / base
    return summary


def time_rrsnet_queries(nrrs, sc, torch, dev, stream, I):
    """Stand-alone RRSNet throughput on a live-queue-sized batch at each precision."""
    n_q = 1 << 21
    feats = torch.from_numpy(I.random_features(n_q, seed=3)).to(dev)
    qout = torch.empty(n_q, dtype=torch.float32, device=dev)
    ms = {}
    for prec in (32, 16, 17, 8):
        for _ in range(3):
            sc.query(feats, out=qout, precision=prec)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(10):
            sc.query(feats, out=qout, precision=prec)
        e1.record(stream)
        torch.cuda.synchronize()
        ms[prec] = e0.elapsed_time(e1) / 10
    return n_q, ms


def online_section(args, nrrs, torch, dev, stream, seed_hi, local_rank, rank):
    """The online NRRS step on the occluded room: one training step and one inference
    frame per step (the first section of earlier versions of this benchmark), its stage
    breakdown and the efficiency tables."""
    from paper_2510_07868_b300 import inputs as I

    scene = I.occluded_room(1)
    params = I.rrsnet_init_params(1)
    sc = nrrs.Scene(scene, device=local_rank)
    sc.set_params(params)
    if args.bvh4:
        sc.set_traversal(4)
    out = torch.empty((H_IMG, W_IMG, 3), dtype=torch.float32, device=dev)
    graph = 0 if args.no_graph else 1
    topts = nrrs.TrainOpts.defaults(width=W_IMG, height=H_IMG, spp=TRAIN_SPP, max_depth=DEPTH,
                                    seed_hi=seed_hi, graph=graph)

    def train(frame):
        topts.frame = frame
        return nrrs.nrrs_train_step(sc.handle, topts, stream)

    def render(frame, profile=0):
        return nrrs.nrrs_render(sc.handle, W_IMG, H_IMG, SPP, DEPTH, nrrs.RRS_NET,
                                nrrs.RenderOpts.defaults(frame=frame, seed_hi=seed_hi,
                                                         profile=profile, graph=graph,
                                                         precision=ONLINE_PRECISION),
                                out, stream, True)

    tuner = {p: sc.tune(p) for p in (32, 16, 8)}
    for k in range(args.pretrain):
        train(10_000 + k)
        if k % 4 == 3 or k >= args.pretrain - 8:  # the scene's running mean of frames
            render(20_000 + k)
    warm_ms = np.zeros(nrrs.STAGES)
    warm_n = np.zeros(nrrs.STAGES, dtype=np.int64)
    for k in range(args.warmup):
        train(30_000 + k)
        st = render(k, profile=1)
        warm_ms += st["stage_ms"]
        warm_n += st["stage_launches"]
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    et0 = torch.cuda.Event(enable_timing=True)
    et1 = torch.cuda.Event(enable_timing=True)
    segs = render_segs = launches = fallbacks = 0
    train_ms = 0.0
    steps = max(1, args.online_steps)
    ev0.record(stream)
    for k in range(steps):
        et0.record(stream)
        ts = train(40_000 + k)
        et1.record(stream)
        st = render(args.warmup + k)
        train_ms += et0.elapsed_time(et1)
        segs += st["segments"] + ts["segments"]
        render_segs += st["segments"]
        launches += st["kernel_launches"] + ts["kernel_launches"]
        fallbacks += ts["fallback"] != 0
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    names = nrrs.STAGE_NAMES
    stages = {n: {"ms_per_frame": float(warm_ms[i] / max(1, args.warmup)),
                  "share": float(warm_ms[i] / warm_ms.sum())}
              for i, n in enumerate(names) if warm_n[i] > 0}
    sec = {
        "workload": WORKLOAD, "scene_triangles": scene.n_tri, "value": segs / (ms / 1000.0),
        "unit": UNIT, "steps": steps, "ms_per_step": ms / steps,
        "train_step_ms": train_ms / steps, "render_ms": (ms - train_ms) / steps,
        "render_segments_per_s": render_segs / ((ms - train_ms) / 1000.0),
        "train_phase": ts["phase"], "train_fallbacks": fallbacks,
        "train_loss_rrsnet": ts["loss_rrsnet"], "train_loss_statnet": ts["loss_statnet"],
        "pretrain_steps": args.pretrain, "gpu_launches": int(launches),
        "stages": stages,
        "tuned_shapes": {str(p): {"variant": r["variant"], "blocks_per_sm": r["blocks_per_sm"]}
                         for p, r in tuner.items()},
    }
    eff = None
    if rank == 0 and not args.no_efficiency:
        eff = efficiency_section(nrrs, sc, torch, dev, stream, seed_hi,
                                 precisions=(32, 17, 16, 8))

        def trained_scene(nee, rrsnet_inputs, statnet_encoding):
            """A second RRSNet / StatNet pair trained online like the first."""
            sc2 = nrrs.Scene(scene, device=local_rank)
            sc2.set_params(params)
            sc2.set_rrsnet_inputs(rrsnet_inputs)
            sc2.set_statnet_encoding(statnet_encoding)
            sc2.tune(32)
            t2 = nrrs.TrainOpts.defaults(width=W_IMG, height=H_IMG, spp=TRAIN_SPP,
                                         max_depth=DEPTH, seed_hi=seed_hi, graph=graph, nee=nee)
            for k in range(args.pretrain + args.warmup + steps):
                t2.frame = 10_000 + k
                nrrs.nrrs_train_step(sc2.handle, t2, stream)
                nrrs.nrrs_render(sc2.handle, W_IMG, H_IMG, SPP, DEPTH, nrrs.RRS_NET,
                                 nrrs.RenderOpts.defaults(frame=20_000 + k, seed_hi=seed_hi,
                                                          graph=graph, nee=nee),
                                 out, stream, False)
            return sc2

        # the same comparison with next-event estimation (on in the paper's experiments,
        # Sec. 5), with RRSNet on the paper's NRRS inputs (Sec. 4 "Input Encoding"), with
        # StatNet on the paper's encodings too (hash grid, one-blob), and AID-NRRS
        for key, nee, rin, enc in (("nee", 1, 0, 0), ("nrrs_inputs", 0, 1, 0),
                                   ("nrrs_inputs_grid_statnet", 0, 1, 1),
                                   ("aid_nrrs", 0, 2, 1)):
            sc2 = trained_scene(nee, rin, enc)
            eff[key] = efficiency_section(nrrs, sc2, torch, dev, stream, seed_hi, nee=nee)
            sc2.close()
    sec["efficiency"] = eff
    n_q, qms = time_rrsnet_queries(nrrs, sc, torch, dev, stream, I)
    sc.close()
    return sec, (n_q, qms, tuner)


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_2510_07868_b300 import inputs as I
    from paper_2510_07868_b300 import nrrs

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

    stream = torch.cuda.current_stream()
    seed_hi = replica_seed(rank)  # independent replicas: different Philox streams per rank
    graph = 0 if args.no_graph else 1

    # ---- set-up of the headline workload (untimed)
    scene = I.three_rooms(1)
    t_build = time.perf_counter()
    sc = nrrs.Scene(scene, device=local_rank)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t_build
    params0 = I.rrsnet_init_params(2)
    sc.set_params(params0)
    tuner = {p: sc.tune(p) for p in (HL_PRECISION, 32)}
    tw, th, tspp = HL_TRAIN
    topts = nrrs.TrainOpts.defaults(width=tw, height=th, spp=tspp, max_depth=HL_DEPTH,
                                    seed_hi=seed_hi, graph=graph)
    t_train = time.perf_counter()
    last_ts = None
    for k in range(args.hl_pretrain):
        topts.frame = 10_000 + k
        last_ts = nrrs.nrrs_train_step(sc.handle, topts, stream)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t_train
    t_search = time.perf_counter()
    search = nrrs.nrrs_mixdepth_search(sc.handle, HL_SEARCH[0], HL_SEARCH[1], HL_DEPTH, t_d=6,
                                       frame=777, d_pixel_ref=None, precision=HL_PRECISION,
                                       stream=stream)
    search_s = time.perf_counter() - t_search
    gate = search["gate"]
    out = torch.empty((HL_H, HL_W, 3), dtype=torch.float32, device=dev)

    def render(frame, profile=0, d_out=out):
        return nrrs.nrrs_render(sc.handle, HL_W, HL_H, HL_SPP, HL_DEPTH, nrrs.RRS_NET_MIX,
                                nrrs.RenderOpts.defaults(frame=frame, seed_hi=seed_hi, gate=gate,
                                                         precision=HL_PRECISION, graph=graph,
                                                         profile=profile),
                                d_out, stream, True)

    clocks = ClockSampler(local_rank)
    clocks.launch()
    # warm-up frames time every render stage (events around each launch); the timed frames
    # bracket only the dominant stage's launches, which the roofline needs
    warm_ms = np.zeros(nrrs.STAGES)
    warm_n = np.zeros(nrrs.STAGES, dtype=np.int64)
    warm = {"live": 0, "evals": 0, "children": 0, "last": 0, "live_net": 0}
    gate_names = nrrs.gate_methods(gate, HL_DEPTH)
    for k in range(args.warmup):
        st = render(k, profile=1)
        warm_ms += st["stage_ms"]
        warm_n += st["stage_launches"]
        warm["live"] += int(st["live"].sum())
        # slots of the depths whose shading runs fused with RRSNet
        warm["live_net"] += int(sum(st["live"][d] for d in range(HL_DEPTH - 1)
                                    if gate_names[d] == "NET"))
        warm["evals"] += st["net_evals"]
        warm["children"] += int(st["live"][1:].sum())
        warm["last"] += int(st["live"][HL_DEPTH - 1])
    dom = int(np.argmax(warm_ms))
    torch.cuda.synchronize()
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    segs = launches = live_total = net_evals = 0
    stage_ms = np.zeros(nrrs.STAGES)
    stage_n = np.zeros(nrrs.STAGES, dtype=np.int64)
    status = 0
    # a profiler started with "profile from start off" (ncu --profile-from-start off)
    # records the timed frames only; without a profiler these calls do nothing
    torch.cuda.profiler.start()
    ev0.record(stream)
    for k in range(args.steps):
        st = render(args.warmup + k, profile=1 << (dom + 1))
        segs += st["segments"]
        launches += st["kernel_launches"]
        stage_ms += st["stage_ms"]
        stage_n += st["stage_launches"]
        live_total += int(st["live"].sum())
        net_evals += st["net_evals"]
        status |= st["status_bits"]
    ev1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    last_F = np.array(st["F"][:HL_DEPTH], dtype=np.float32)
    last_live = [int(v) for v in st["live"][:HL_DEPTH]]

    # end to end through the public API: weights from pinned host memory in, frame out
    trained = nrrs.nrrs_get_params(sc.handle, nrrs.NET_RRSNET)
    pinned_params = torch.from_numpy(trained).pin_memory()
    pinned_out = torch.empty((HL_H, HL_W, 3), dtype=torch.float32).pin_memory()
    e2e_segs = 0
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for k in range(args.steps):
        nrrs.nrrs_set_rrsnet_params(sc.handle, pinned_params.numpy(), stream)
        st = render(70_000 + k)
        e2e_segs += st["segments"]
        pinned_out.copy_(out, non_blocking=True)
        torch.cuda.current_stream().synchronize()
    e2e_s = time.perf_counter() - t0
    ref_img = None
    if world == 1 and not args.no_cpu_baseline:
        # the reference image the gate's heuristic depths saw (the scene's running mean)
        ref_img = out.cpu().numpy().astype(np.float64)

    if dist:
        ms, e2e_s, segs, e2e_segs = combine_ranks(dist, dev, ms, e2e_s, segs, e2e_segs)
    hl_stats = {"live_total": live_total, "net_evals": net_evals, "stage_ms": stage_ms,
                "stage_n": stage_n, "warm_ms": warm_ms, "warm_n": warm_n, "warm": warm,
                "dom": dom, "status": status, "last_live": last_live}
    sc.close()

    # ---- second section: the online training step on the occluded room
    online = None
    qstats = None
    if not args.no_online:
        online, qstats = online_section(args, nrrs, torch, dev, stream, seed_hi, local_rank, rank)
    if rank != 0:
        return
    hbm, bf16, peak_kind = measured_peaks()
    value = segs / (ms / 1000.0)

    # roofline of the dominant render stage (event times on the launching stream)
    names = nrrs.STAGE_NAMES
    warm = hl_stats["warm"]
    alg_bytes_per_unit = {"extend": BYTES_PER_RAY_EXTEND}
    bytes_dom = (BYTES_PER_RAY_EXTEND * live_total) if names[dom] == "extend" else None
    per_launch_ms = stage_ms[dom] / max(1, stage_n[dom])
    achieved = (bytes_dom / (stage_ms[dom] / 1000.0) / 1e9) if bytes_dom else None
    units_per_launch = live_total / max(1, stage_n[dom])
    per_unit = profile_record(names[dom], "traffic")
    traffic = per_unit * units_per_launch if per_unit is not None else None
    inst_per_ray = profile_record(names[dom], "warp_inst_per_ray")
    issue_active = profile_record(names[dom], "issue_active")
    alu_active = profile_record(names[dom], "alu_pipe_active")
    roofline = {
        "kernel": "k_trace" if names[dom] == "extend" else names[dom], "bound": "hbm",
        "achieved": achieved, "peak": hbm, "unit": "GB/s",
        "frac": (achieved / hbm) if achieved else None, "traffic": traffic,
        "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
        else "fallback 6.4 TB/s", "avg_launch_ms": per_launch_ms,
        "launches": int(stage_n[dom]),
        "bytes_per_unit": alg_bytes_per_unit.get(names[dom]),
        "issue": {"warp_inst_per_ray_depth1": inst_per_ray,
                  "issue_active_frac": issue_active, "alu_pipe_active_frac": alu_active,
                  "source": "ncu capture in profiles/ of the same kernel on a smaller image of "
                            "the same scene (depths 1 and 2, time-weighted; null when the "
                            "kernel changed since)",
                  "issue_peak_warp_inst_per_s": 148 * 4 * 2.032e9,
                  "achieved_warp_inst_per_s": issue_active * 148 * 4 * 2.032e9
                  if issue_active else None},
        "note": ("the traversal is bound by instruction issue, not HBM: the BVH and the "
                 "triangles stay in L2; 48 B/ray algorithmic (32 B ray in, 16 B hit out)"
                 if names[dom] == "extend" else f"{names[dom]} stage against HBM"),
    }
    if issue_active:
        roofline["issue"]["frac_of_issue_peak"] = issue_active
    stage_bytes = {
        "extend": BYTES_PER_RAY_EXTEND * warm["live"],
        # the last depth only deposits (split_count); NET depths shade in the fused kernel
        "shade": BYTES_PER_RAY_SHADE * (warm["live"] - warm["last"] - warm["live_net"]),
        "rrsnet": BYTES_PER_RAY_SHADE * warm["live_net"],
        "split_count": BYTES_PER_SLOT_DEPOSIT * warm["last"],
        "split_scatter": BYTES_PER_PARENT_SPLIT * (warm["live"] - warm["last"])
        + BYTES_PER_CHILD_SPLIT * warm["children"],
    }
    stages = {"timed_over": f"{args.warmup} warm-up frames"}
    for i, n in enumerate(names):
        if warm_n[i] == 0:
            continue
        e = {"ms_per_frame": float(warm_ms[i] / args.warmup), "launches": int(warm_n[i]),
             "share": float(warm_ms[i] / warm_ms.sum())}
        if n in stage_bytes and warm_ms[i] > 0:
            gbs = stage_bytes[n] / (warm_ms[i] / 1000.0) / 1e9
            e.update({"achieved_gbs": gbs, "frac_of_hbm": gbs / hbm})
        stages[n] = e
    roofline["stages"] = stages
    rr_ms = warm_ms[names.index("rrsnet")]
    rrsnet = {
        "in_render": {"precision": "BF16 (tensor cores)",
                      "kernel": "k_shade_rrsnet_tc: shading and RRSNet fused at NET depths "
                                "(the features stay in shared memory); the time includes the "
                                "shading of those depths",
                      "evaluations_per_frame": warm["evals"] / max(1, args.warmup),
                      "ms_per_frame": float(rr_ms / max(1, args.warmup)),
                      "tflops": RRSNET_FLOP_PER_PATH * warm["evals"] / (rr_ms / 1000) / 1e12
                      if rr_ms > 0 else None,
                      "bf16_peak_tflops": bf16},
    }
    ir = rrsnet["in_render"]
    if ir["tflops"]:
        ir["frac_of_bf16_tensor_peak"] = ir["tflops"] / bf16
    if qstats:
        n_q, qms, tuner2 = qstats
        fp32_peak = 148 * 128 * 2 * 2.032e9 / 1e12  # FP32 SIMT FMA lanes x max clock
        rows_per_s_hbm = hbm * 1e9 / (16 * 4 + 4)  # FP32 features in, factor out
        tf = {p: RRSNET_FLOP_PER_PATH * n_q / (qms[p] / 1000) / 1e12 for p in qms}
        rrsnet["standalone"] = {
            "batch": n_q, "ms": qms,
            "tflops_fp32": tf[32], "fp32_simt_peak_tflops": fp32_peak,
            "frac_of_fp32_peak": tf[32] / fp32_peak,
            "tflops_tensor_bf16x3": tf[16], "tflops_tensor_bf16": tf[17],
            "tflops_tensor_e4m3": tf[8],
            "hbm_frac_bf16x3": 68 * n_q / (qms[16] / 1000) / 1e9 / hbm,
            "hbm_frac_bf16": 68 * n_q / (qms[17] / 1000) / 1e9 / hbm,
            "hbm_frac_e4m3": 68 * n_q / (qms[8] / 1000) / 1e9 / hbm,
            "flop_cap_at_hbm_tflops": RRSNET_FLOP_PER_PATH * rows_per_s_hbm / 1e12,
            "frac_of_bf16_tensor_peak": tf[16] / bf16,
            "frac_of_fp8_tensor_peak": tf[8] / (2 * bf16),
            "note": "algorithmic FLOP (5184/row); the split BF16 runs 3 MMAs per product; "
                    "FP8 peak taken as 2x the measured BF16 (nominal ratio)",
        }
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        v, cores, desc, _, _ = oracle_headline_sample(
            scene, trained.astype(np.float64), gate, ref_img, last_F)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": desc + "; the GPU run's trained weights, gate and per-depth F"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": HL_WORKLOAD, "scene_triangles": scene.n_tri,
                   "parallelism": f"replicas{world}",
                   "bounce_loop": "CUDA graph per frame" if graph else "stream launches",
                   "bvh": "BVH2, FP16 boxes rounded outward",
                   "mixdepth_gate": nrrs.gate_methods(gate, HL_DEPTH),
                   "l2": "no flush: each step writes ~3 GB of path queues (> 126 MB L2)"},
        "setup": {"bvh_build_s": build_s, "pretrain_steps": args.hl_pretrain,
                  "pretrain_s": train_s, "train_frame": list(HL_TRAIN),
                  "last_train_phase": last_ts["phase"] if last_ts else None,
                  "mixdepth_search_s": search_s, "mixdepth_candidates": search["evaluated"],
                  "search_frame": list(HL_SEARCH),
                  "tuned_shapes": {str(p): {"variant": r["variant"],
                                            "blocks_per_sm": r["blocks_per_sm"]}
                                   for p, r in tuner.items()}},
        "frame_status_bits": int(hl_stats["status"]),
        "queue_per_depth_last_frame": hl_stats["last_live"],
        "e2e": {"value": e2e_segs / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": int(trained.nbytes),
                "d2h_bytes_per_step": int(HL_W * HL_H * 3 * 4)},
        "gpu_launches": int(launches),
        "roofline": roofline,
        "rrsnet": rrsnet,
        "online_step": online,
        "cpu_baseline": cpu,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def run_rrsnet_only(args):
    """RRSNet inference alone: `warmup` untimed then `steps` timed queries of 2^21 rows."""
    import torch

    from paper_2510_07868_b300 import inputs as I
    from paper_2510_07868_b300 import nrrs

    sc = nrrs.Scene(I.box_scene(1))
    sc.set_params(I.rrsnet_init_params(1))
    if args.tuned:
        sc.tune(precision=args.rrsnet_only)
    n = 1 << 21
    feats = torch.from_numpy(I.random_features(n, seed=3)).cuda()
    q = torch.empty(n, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        sc.query(feats, precision=args.rrsnet_only, out=q)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()  # ncu --profile-from-start off sees only the timed queries
    e0.record()
    for _ in range(args.steps):
        sc.query(feats, precision=args.rrsnet_only, out=q)
    e1.record()
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    hbm, _, _ = measured_peaks()
    print(json.dumps({"metric": "RRSNet inference", "precision": args.rrsnet_only, "rows": n,
                      "launch_shape": "tuned" if args.tuned else "default", "ms_per_launch": ms,
                      "tflops": RRSNET_FLOP_PER_PATH * n / (ms / 1000) / 1e12,
                      "hbm_frac": 68 * n / (ms / 1000) / 1e9 / hbm}), flush=True)
    sc.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-efficiency", action="store_true")
    ap.add_argument("--bvh4", action="store_true",
                    help="traverse the four-wide tree instead of the binary BVH")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch the bounce loop kernel by kernel instead of as a CUDA graph")
    ap.add_argument("--pretrain", type=int, default=PRETRAIN_STEPS,
                    help="untimed online training steps of the online-step section")
    ap.add_argument("--hl-pretrain", type=int, default=HL_PRETRAIN,
                    help="untimed online training steps on the headline scene")
    ap.add_argument("--online-steps", type=int, default=20,
                    help="timed steps of the online-step section")
    ap.add_argument("--no-online", action="store_true",
                    help="skip the online-step section (occluded room)")
    ap.add_argument("--rrsnet-only", type=int, choices=[32, 16, 17, 8], default=0,
                    help="time only RRSNet inference at this precision on a 2^21-row batch "
                         "(the untuned default launch shape), for kernel profiles")
    ap.add_argument("--tuned", action="store_true",
                    help="with --rrsnet-only: run the launch-shape tuner first, so the "
                         "queries take the tuned shape of their bucket")
    ap.add_argument("--hl-image", default="",
                    help="WxH: render the headline scene at this image size instead of "
                         "1920x1080 (a smaller workload for kernel profiles; the JSON line "
                         "names the size)")
    args = ap.parse_args()
    if args.hl_image:
        global HL_W, HL_H, HL_WORKLOAD
        w, h = (int(v) for v in args.hl_image.lower().split("x"))
        HL_WORKLOAD = HL_WORKLOAD.replace(f"{HL_W}x{HL_H}", f"{w}x{h}")
        HL_W, HL_H = w, h
    if args.rrsnet_only:
        run_rrsnet_only(args)
        return
    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local_rank = _env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
