"""Benchmark of the II-LBM time step on one GB300 (or N independent replicas).

Workload (default): the 2048^2 periodic MRT membrane -- an ellipse with semi-axes 400
and 250, 2048 markers equally spaced in arc length, zero-rest-length springs of
stiffness 0.05, tau = 0.6, populations stored in FP32 as shifted deviations.  One
"step" is one whole II-LBM time step (marker forces, cut-link jump, tangential
spreading, interpolation and marker update, fused stream-collide), i.e. every row of
the hot path.  Metric: MLUPS (million lattice-node updates per second), whole job.
--storage f16 | bf16 | f64 runs it with another storage precision; FP64 storage computes
in FP64, which GB300 runs at about 1.26 TFLOP/s, so its roofline is the FP64 arithmetic
roof ("bound": "alu") with the HBM fraction beside it.

--workload batched: the sweep of 256 independent membranes (square lattices of
64..512 nodes, ellipses of aspect 1..2.5 at perimeter 0.6 n, one marker per half lattice
unit, stiffness log-uniform in [1e-3, 1e-1], tau uniform in [0.55, 1], FP32, seeded),
advanced by the batched executor (one launch per phase per step, autotuned stream-collide
variant, graph replay); the line also carries the same lattices stepped one by one
("plain per-simulation form") for comparison.

--workload channel: flow past the fixed cylinder (D = 40 at x = 256, y = 128.5, 126
markers) in the 1024 x 256 MRT channel, parabolic inflow u_max = 0.05, tau from Re,
FP32, the normal force through the jump and the tangential force by direct forcing with
5 force updates per step (the updates see the force through the jump, as the step
applies it), Re 20 by default (--re 100: tau = 0.56).  --history H adds an untimed
drag / lift record of H steps (mean C_D, lift amplitude, Strouhal number).  Its state
(19 MB) fits in L2, so its roofline is flagged so.

--workload learned: 64 rigid-cylinder channels (512 x 128, D uniform in [16, 32], Re
uniform in [10, 150], markers 1.5 lattice units apart, FP32) with the direct-forcing
iteration run to the no-slip residual 1e-6 every step.  A network trained on samples the
method generates (other channels, another seed) proposes the iteration's start; the line
reports its end-to-end MLUPS and force passes per step next to the plain iteration
(start zero) and the previous-step start, on the same channels.

--workload membrane3d: the three-dimensional method on the D3Q19 lattice -- a 256^3
periodic MRT box (tau 0.6, d'Humieres rates of section 2.2.1) holding a surface-tension
ellipsoid (semi-axes 0.31, 0.25, 0.22 of the box, a seeded rotation, 40 962 vertices, edges
about one lattice unit) whose vertices move with the fluid; FP32 populations (--storage f64
runs FP64; f16 / bf16 store 16-bit populations with FP32 arithmetic).  One step: vertex forces and normal split, the jump on every cut link of the
triangulation, tangential spreading, the stream-collide, interpolation and the vertex
update.  --size3 sets the box's side.

Prints one JSON line.  --impl reference times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2003_12186_gb300 import workloads as W  # noqa: E402

L2_BYTES = 129 * 1024 * 1024
NOMINAL_HBM_GBS = 8000.0  # GB300 HBM3e, nominal


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16", "f64"])
    ap.add_argument("--size", type=int, default=2048)
    ap.add_argument("--tma", type=int, default=0, choices=[0, 1, 2],
                    help="FP32 lean stream-collide of interior tiles by bulk tensor copies: "
                         "0 never (default), 1 every step, 2 odd steps only")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-hbm-check", action="store_true",
                    help="skip the 4096^2 out-of-L2 lean stream-collide measurement")
    ap.add_argument("--workload", default="ellipse",
                    choices=["ellipse", "batched", "learned", "channel", "membrane3d"])
    ap.add_argument("--size3", type=int, default=256, help="membrane3d: nodes per axis")
    ap.add_argument("--re", type=float, default=20.0, help="Reynolds number (channel)")
    ap.add_argument("--history", type=int, default=0,
                    help="channel: steps of drag / lift history after the timed region")
    ap.add_argument("--count", type=int, default=256, help="simulations of the batched sweep")
    a = ap.parse_args()
    if a.steps is None:
        a.steps = {"ellipse": 20000, "membrane3d": 200}.get(a.workload, 2000)
    return a


def ellipse_config(args, world=1):
    """The membrane workload's config object, the same in both arms."""
    w = workload(args.size, args.storage)
    sbytes = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2}[args.storage]
    cells = w["nx"] * w["ny"]
    return {"workload": w["name"].replace(f"_{args.storage}", "") + "_membrane",
            "lattice": [w["nx"], w["ny"]], "markers": len(w["X"]), "collision": "mrt",
            "tau": w["tau"], "storage": args.storage,
            "arithmetic": "f64" if args.storage == "f64" else "f32",
            "parallelism": "replicas" if world > 1 else "single",
            "l2": f"inputs larger than L2 ({9 * sbytes * cells / 2**20:.0f} MiB populations "
                  f"vs 129 MiB L2)" if 9 * sbytes * cells > L2_BYTES else "working set fits L2"}


def workload(size, storage):
    return W.ellipse_2048(storage) if size == 2048 else W.ellipse_scaled(size, storage)


# FP64 roof of GB300 from its unit counts and clock, and the algorithmic FP64 flops of one
# node update of the MRT collision without a body force, counted from the collision
# (density and velocity 24, moments 32, equilibrium moments 12, relaxation 12, moment
# coefficients 10, back-transform 36; a division counts as one flop).
FP64_PEAK_TFLOPS = round(152 * 2 * 2 * 2.07e9 / 1e12, 4)
FP64_MRT_FLOPS_PER_NODE = 126
# The D3Q19 MRT collision without force, per node, as the pair-symmetric form computes
# it: pair sums and differences 18, density and momentum 24, density, reciprocal,
# velocity and the equilibrium's base 13, the nine pairs' equilibrium terms 96, the
# moments (83 terms, 27 of them with a non-unit coefficient, and the rates and norms of
# 15 rows) 140, the back-transform and the pairs' reassembly 147.
D3Q19_MRT_FLOPS_PER_NODE = 438


def max_over_ranks(values, dist, device="cuda"):
    """Each value's maximum over the ranks (the slowest rank's time); the values
    themselves in a single process."""
    if not dist:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def whole_job_mlups(cells_per_rank, steps, world, seconds):
    """Lattice updates of all ranks (each runs its own replica: weak scaling) over the
    slowest rank's time."""
    return cells_per_rank * steps * world / seconds / 1e6


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks
class _Nvml:
    """The driver's management library (libnvidia-ml), read through ctypes: SM clock,
    its maximum, power and the active clock-event reasons of one device.  Read only."""

    SM = 1  # NVML_CLOCK_SM
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, torch_device):
        import ctypes as C
        self.C = C
        L = None
        for name in ("libnvidia-ml.so.1", "libnvidia-ml.so"):
            try:
                L = C.CDLL(name)
                break
            except OSError:
                continue
        if L is None or L.nvmlInit_v2() != 0:
            raise OSError("NVML unavailable")
        self.L = L
        self.h = C.c_void_p()
        import torch
        p = torch.cuda.get_device_properties(torch_device)
        ids = [f"{p.pci_domain_id:08x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0",
               f"{p.pci_domain_id:04x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0"]
        ok = False
        for bid in ids:
            if L.nvmlDeviceGetHandleByPciBusId_v2(bid.encode(), C.byref(self.h)) == 0:
                ok = True
                break
        if not ok:
            raise OSError("NVML: no device with the CUDA device's PCI bus id")
        self.reasons_fn = getattr(L, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(L, "nvmlDeviceGetCurrentClocksThrottleReasons")
        v = C.c_uint()
        self.max_mhz = float(v.value) if L.nvmlDeviceGetMaxClockInfo(self.h, self.SM,
                                                                     C.byref(v)) == 0 else None

    def sample(self):
        C = self.C
        mhz, mw, r = C.c_uint(), C.c_uint(), C.c_ulonglong()
        if self.L.nvmlDeviceGetClockInfo(self.h, self.SM, C.byref(mhz)) != 0:
            return None
        self.reasons_fn(self.h, C.byref(r))
        self.L.nvmlDeviceGetPowerUsage(self.h, C.byref(mw))
        return float(mhz.value), int(r.value), mw.value / 1000.0


class ClockSampler:
    """SM clock and clock-event reasons sampled during the timed region: a thread reads
    NVML every ~0.25 ms (so even a region of a millisecond or two gets samples), with
    nvidia-smi polling (200 ms) where NVML cannot be loaded.  begin() / end() mark the
    region; stop() summarises the samples taken between the marks."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []  # (host time, sm MHz, reason names, power W)
        self.proc = None
        self.nvml = None
        self.max_mhz = None
        self.t0 = self.t1 = None
        self._stop = threading.Event()

    def start(self):
        try:
            self.nvml = _Nvml(self.index)
            self.max_mhz = self.nvml.max_mhz
            self.t = threading.Thread(target=self._poll_nvml, daemon=True)
            self.t.start()
            return
        except Exception:
            self.nvml = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read_smi, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _poll_nvml(self):
        while not self._stop.is_set():
            v = self.nvml.sample()
            if v:
                mhz, bits, w = v
                names = sorted(n for b, n in _Nvml.REASONS.items() if bits & b)
                self.samples.append((time.perf_counter(), mhz, names, w))
            time.sleep(0.00025)

    def _read_smi(self):
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.proc.stdout:
            f = [x.strip() for x in ln.strip().split(",")]
            if len(f) < 9:
                continue
            try:
                mhz, mx = float(f[1]), float(f[2])
            except ValueError:
                continue
            self.max_mhz = mx
            act = sorted(nm for nm, v in zip(names, f[5:9]) if v.lower().startswith("active"))
            self.samples.append((time.perf_counter(), mhz, act, None))

    def begin(self):
        self.t0 = time.perf_counter()

    def end(self):
        self.t1 = time.perf_counter()

    def stop(self):
        self._stop.set()
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.nvml is None and self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clock query unavailable"],
                    "samples": 0}
        self.t.join(timeout=5)
        t0 = self.t0 if self.t0 is not None else -1e300
        t1 = self.t1 if self.t1 is not None else 1e300
        inside = [s for s in self.samples if t0 <= s[0] <= t1]
        sm = [s[1] for s in inside]
        reasons = sorted({r for s in inside for r in s[2]})
        power = [s[3] for s in inside if s[3] is not None]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": self.max_mhz,
                "sm_mhz_min": min(sm) if sm else None, "reasons": reasons,
                "samples": len(sm), "source": "nvml" if self.nvml else "nvidia-smi",
                "power_w_max": round(max(power), 1) if power else None,
                "region_s": round(t1 - t0, 6) if self.t0 is not None else None}


# -------------------------------------------------------------- cpu oracle
def oracle_rate(size, max_seconds, min_steps=1, parallel=False):
    """Time the FP64 CPU oracle (as it stands: one thread, or its OpenMP build on every
    host core) on the workload."""
    from oracle import oracle as O
    w = workload(size, "f64")
    o = O.Oracle(w["nx"], w["ny"], parallel=parallel, collision=O.MRT, tau=w["tau"],
                 s=W.mrt_rates(w["tau"]))
    o.set_interface(w["X"], model=O.SPRING, kappa=w["kappa"], dX=w["dX"])
    steps, t0 = 0, time.perf_counter()
    while steps < min_steps or time.perf_counter() - t0 < max_seconds:
        o.step(1)
        steps += 1
    dt = time.perf_counter() - t0
    o.close()
    return w["nx"] * w["ny"] * steps / dt / 1e6, steps, dt


def cpu_baseline_both(size, seconds_single, seconds_all):
    """The oracle on one thread and (OpenMP build) on every host core; the all-core
    figure leads, the single-thread one is kept beside it."""
    from oracle import oracle as O
    r1, st1, dt1 = oracle_rate(size, seconds_single)
    out = {"value": round(r1, 4), "unit": "MLUPS", "cores": 1, "kind": "oracle",
           "sample": f"{st1} FP64 oracle steps of the same {size}^2 workload, {dt1:.1f} s, "
                     f"one thread"}
    try:
        rp, stp, dtp = oracle_rate(size, seconds_all, parallel=True)
    except RuntimeError:
        return out
    return {"value": round(rp, 4), "unit": "MLUPS", "cores": O.omp_threads(), "kind": "oracle",
            "sample": f"{stp} FP64 oracle steps of the same {size}^2 workload, {dtp:.1f} s, "
                      f"OpenMP build (per-node loops on {O.omp_threads()} threads, results "
                      f"identical to the serial build)",
            "single_thread": out}


def run_reference(args):
    """Reference arm: the oracle (OpenMP build, every host core), rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    try:
        O.lib(parallel=True)
        par = True
    except RuntimeError:
        par = False
    cores = O.omp_threads() if par else 1
    K, Wm = args.steps, args.warmup
    probe, _, _ = oracle_rate(256, 0.5, parallel=par)
    # largest lattice of the same workload family whose run fits about two minutes
    size = 256
    for n in (args.size, args.size // 2, args.size // 4, args.size // 8, 256):
        if n * n * (K + min(Wm, 3)) / (probe * 1e6) <= 120.0:
            size = n
            break
    steps = K
    if size == 256:
        steps = max(1, min(K, int(120.0 * probe * 1e6 / (256 * 256))))
    w = workload(size, "f64")
    o = O.Oracle(w["nx"], w["ny"], parallel=par, collision=O.MRT, tau=w["tau"],
                 s=W.mrt_rates(w["tau"]))
    o.set_interface(w["X"], model=O.SPRING, kappa=w["kappa"], dX=w["dX"])
    o.step(min(Wm, 3))
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    value = w["nx"] * w["ny"] * steps / dt / 1e6
    sample = (f"{steps} oracle steps of the ellipse membrane "
              + (f"at {size}^2" if size == args.size else
                 f"scaled to {size}^2 (same aspect, tau, stiffness, marker density)")
              + ", FP64, " + (f"OpenMP build on {cores} threads" if par else "one thread"))
    out = {"metric": "MLUPS", "value": round(value, 4), "unit": "MLUPS", "n_gpus": args.gpus,
           "steps": K, "warmup": Wm, "ms_per_step": round(dt / steps * 1e3, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "impl": "reference",
           "config": ellipse_config(args),
           "cpu_baseline": {"value": round(value, 4), "unit": "MLUPS", "cores": cores,
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": round(value, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------- GPU arm
def make_lattice(iilbm, w, stream, tma=0):
    g = iilbm.Lattice(w["nx"], w["ny"], collision=iilbm.MRT, storage=w["storage"],
                      tau=w["tau"], s=W.mrt_rates(w["tau"]), stream=stream)
    if tma:
        g.set_option(iilbm.OPT_TMA_KERNEL, tma)
    return g


def run_ours(args):
    import torch
    from paper_2003_12186_gb300 import iilbm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    ts = torch.cuda.Stream()  # the library runs on this stream; events are recorded on it
    torch.cuda.set_stream(ts)
    stream = ts.cuda_stream
    w = workload(args.size, args.storage)
    cells = w["nx"] * w["ny"]
    sbytes = iilbm.STORAGE_BYTES[iilbm.STORAGE[args.storage]]
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    g = make_lattice(iilbm, w, stream, args.tma)
    g.set_interface(w["X"], model=iilbm.SPRING, stiffness=w["kappa"], dX=w["dX"])
    g.step(args.warmup)  # the first call captures the step graphs
    g.synchronize()

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(lat, steps, kernel_timing, mark=False):
        """One timed region of `steps` steps on stream ts, bracketed by a barrier and a
        device synchronisation; optionally with per-launch kernel events."""
        if kernel_timing:
            lat.iilbm_set_timing(True)
            lat.step(2)  # captures the graphs that record the events, outside the region
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        if mark:
            clocks.begin()
        e0.record(ts)
        lat.step(steps)
        e1.record(ts)
        barrier()
        if mark:
            clocks.end()
        ms = e0.elapsed_time(e1)
        kt = None
        if kernel_timing:
            kt = lat.iilbm_get_timing(with_tiles=True)
            lat.iilbm_set_timing(False)
        return ms, kt

    # region 1 -- the metric: the step as a user runs it (graph replay, no per-launch
    # instrumentation); the clocks are sampled during this region
    ms, _ = timed(g, args.steps, False, mark=True)
    # region 2 -- same workload and graph replay, with CUDA events recorded inside the
    # graphs around every launch of the lean stream-collide (the dominant kernel)
    ms2, (sc_ms, sc_n, launches, tiles) = timed(g, args.steps, True)
    clk = clocks.stop()
    g.synchronize()
    ms, ms2 = max_over_ranks([ms, ms2], dist)
    value = whole_job_mlups(cells, args.steps, world, ms * 1e-3)
    sc_avg_s = sc_ms / max(sc_n, 1) * 1e-3
    # the lean stream-collide updates every node outside the flagged 128 x 8 tiles (those
    # go to the forced kernel on the side stream): 2 x 9 stored values per node
    lean_cells = cells - tiles / max(sc_n, 1) * 128 * 8
    alg_bytes = int(2 * 9 * sbytes * lean_cells)
    peak, peak_kind = peaks()
    achieved = alg_bytes / sc_avg_s / 1e9
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": None,
                "kernel": ("k_stream_collide_tma + k_stream_collide_vec_edge (lean, TMA "
                           f"mode {args.tma})" if args.tma else "k_stream_collide_vec (lean)"),
                "peak_source": peak_kind,
                "flagged_tiles_per_step": round(tiles / max(sc_n, 1), 1),
                "alg_bytes_per_launch": alg_bytes, "avg_launch_us": round(sc_avg_s * 1e6, 2),
                "timed_in": "second timed region of the same steps with per-launch CUDA "
                            f"events ({ms2 / args.steps * 1e3:.2f} us/step there)",
                # the whole step (every node updated once, lean or forced) over the
                # uninstrumented step time of the metric's region
                "step_achieved": round(2 * 9 * sbytes * cells / (ms / args.steps * 1e-3) / 1e9, 1),
                "step_frac": round(2 * 9 * sbytes * cells / (ms / args.steps * 1e-3) / 1e9 / peak,
                                   4),
                # the same two figures against the nominal 8 TB/s of GB300's HBM3e
                "frac_nominal_8tbs": round(achieved / NOMINAL_HBM_GBS, 4),
                "step_frac_nominal_8tbs": round(2 * 9 * sbytes * cells /
                                                (ms / args.steps * 1e-3) / 1e9 /
                                                NOMINAL_HBM_GBS, 4)}
    tr = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tr):
        d = json.load(open(tr)).get(f"ellipse{args.size}_{args.storage}")
        if d and not args.tma:
            roofline["traffic"] = d
            # the same fraction counted in the DRAM bytes of a captured launch
            roofline["dram_achieved"] = round(d / sc_avg_s / 1e9, 1)
            roofline["dram_frac"] = round(d / sc_avg_s / 1e9 / peak, 4)
    if args.storage == "f64":
        # FP64 arithmetic: GB300 runs FP64 at about 1.25 TFLOP/s (152 SMs x 2 FP64 FMA per
        # clock x 2 flops x 2.07 GHz), so the FP64 stream-collide is bound by the FP64
        # pipe, not by HBM (126 flops per node of the MRT collision without a body force
        # against 144 bytes per node).  The HBM figures stay in the line as hbm_*.
        flops = FP64_MRT_FLOPS_PER_NODE * lean_cells
        hbm = {("hbm_" + k): roofline[k] for k in ("achieved", "peak", "frac")}
        roofline.update({"bound": "alu", "achieved": round(flops / sc_avg_s / 1e12, 4),
                         "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": round(flops / sc_avg_s / 1e12 / FP64_PEAK_TFLOPS, 4),
                         "peak_source": "derived: 152 SMs x 2 FP64 FMA/clock x 2 flops x "
                                        "2.07 GHz (nominal FP64 rate of GB300)",
                         "flops_per_node": FP64_MRT_FLOPS_PER_NODE, **hbm})
    # out of L2: the same membrane scaled to 4096^2 (populations 4x the 2048^2 ones, far
    # above the 129 MiB L2), lean stream-collide timed as in region 2
    if args.storage != "f64" and args.size < 4096 and not args.no_hbm_check:
        del g
        torch.cuda.synchronize()
        w4 = workload(4096, args.storage)
        g4 = make_lattice(iilbm, w4, stream, args.tma)
        g4.set_interface(w4["X"], model=iilbm.SPRING, stiffness=w4["kappa"], dX=w4["dX"])
        g4.step(max(args.warmup, 8))
        K4 = 256
        ms4, (sc4, n4, _, t4) = timed(g4, K4, True)
        cells4 = w4["nx"] * w4["ny"]
        lean4 = int(2 * 9 * sbytes * (cells4 - t4 / max(n4, 1) * 128 * 8))
        a4 = lean4 / (sc4 / max(n4, 1) * 1e-3) / 1e9
        s4 = 2 * 9 * sbytes * cells4 / (ms4 / K4 * 1e-3) / 1e9
        roofline["out_of_l2"] = {
            "lattice": [4096, 4096], "steps": K4,
            "populations_mib": round(9 * sbytes * cells4 / 2**20),
            "lean_achieved": round(a4, 1), "lean_frac": round(a4 / peak, 4),
            "lean_frac_nominal_8tbs": round(a4 / NOMINAL_HBM_GBS, 4),
            "avg_launch_us": round(sc4 / max(n4, 1) * 1e3, 2),
            "step_mlups": round(cells4 * K4 / (ms4 * 1e-3) / 1e6, 1),
            "step_achieved": round(s4, 1), "step_frac": round(s4 / peak, 4),
            "note": "the 2048^2 membrane scaled to 4096^2 (same aspect, tau, stiffness, "
                    "marker density), timed with per-launch events like region 2"}
        tr4 = os.path.join(ROOT, "profiles", "traffic.json")
        if os.path.exists(tr4):
            d = json.load(open(tr4)).get(f"ellipse4096_{args.storage}")
            if d:
                roofline["out_of_l2"]["traffic"] = d
        del g4
        torch.cuda.synchronize()
    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        if "g" in locals():
            del g
        torch.cuda.synchronize()
        g2 = make_lattice(iilbm, w, stream, args.tma)
        nm = len(w["X"])
        Xin = torch.from_numpy(np.ascontiguousarray(w["X"])).pin_memory()
        Xout = torch.empty((nm, 2), dtype=torch.float64).pin_memory()
        ux = torch.empty((w["ny"], w["nx"]), dtype=torch.float64).pin_memory()
        uy = torch.empty((w["ny"], w["nx"]), dtype=torch.float64).pin_memory()
        K2 = args.steps
        # warm-up outside the region: the graphs are captured here; the set_interface
        # inside the region (same marker count and parameters) keeps them
        g2.set_interface(Xin, model=iilbm.SPRING, stiffness=w["kappa"], dX=w["dX"])
        g2.step(2)
        g2.synchronize()
        barrier()
        t0 = time.perf_counter()
        g2.set_interface(Xin, model=iilbm.SPRING, stiffness=w["kappa"], dX=w["dX"])
        for _ in range(K2):
            g2.step(1)
            g2.iilbm_get_markers_into(X=Xout)
        g2.get_macros(None, ux, uy, want=(False, True, True))
        barrier()
        dt = time.perf_counter() - t0
        dt, = max_over_ranks([dt], dist)
        h2d = Xin.numel() * 8
        d2h = K2 * Xout.numel() * 8 + 2 * cells * 8
        e2e = {"value": round(whole_job_mlups(cells, K2, world, dt), 1), "unit": "MLUPS",
               "h2d_bytes_per_step": round(h2d / K2, 1), "d2h_bytes_per_step": round(d2h / K2, 1),
               "note": "inside the region: set_interface from pinned host (the same "
                       "membrane as the warm-up's, so the captured graphs are kept), per "
                       "step iilbm_step(1) + marker read-back to pinned host, final velocity "
                       "field read-back"}
        del g2
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline_both(args.size, 10.0, 8.0)
    if rank == 0:
        out = {"metric": "MLUPS", "value": round(value, 1), "unit": "MLUPS", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": round(ms / args.steps, 5), "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": args.storage,
               "data": "synthetic",
               "config": ellipse_config(args, world),
               "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
               "gpu_launches": int(launches / max(sc_n, 1) * args.steps)}
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


# ----------------------------------------------------------- batched sweep
def batch_lattice(iilbm, sim, stream=None, with_interface=True):
    g = iilbm.Lattice(sim["nx"], sim["ny"], collision=iilbm.MRT, storage="f32", tau=sim["tau"],
                      s=W.mrt_rates(sim["tau"]), stream=stream)
    if with_interface:
        g.set_interface(sim["X"], model=iilbm.SPRING, stiffness=sim["kappa"], dX=sim["dX"])
    return g


def oracle_batch_rate(sims, max_seconds):
    """The FP64 oracle stepping the sweep's simulations one after another (one thread)
    until max_seconds have passed; returns node updates / s, steps, seconds, sims used."""
    from oracle import oracle as O
    cells, used, t0 = 0, 0, time.perf_counter()
    steps_per_sim = 4
    while time.perf_counter() - t0 < max_seconds and used < len(sims):
        sim = sims[used]
        o = O.Oracle(sim["nx"], sim["ny"], collision=O.MRT, tau=sim["tau"],
                     s=W.mrt_rates(sim["tau"]))
        o.set_interface(sim["X"], model=O.SPRING, kappa=sim["kappa"], dX=sim["dX"])
        o.step(steps_per_sim)
        o.close()
        cells += sim["nx"] * sim["ny"] * steps_per_sim
        used += 1
    dt = time.perf_counter() - t0
    return cells / dt / 1e6, steps_per_sim, dt, used


def run_batched(args):
    import torch
    from paper_2003_12186_gb300 import iilbm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    ts = torch.cuda.Stream()
    torch.cuda.set_stream(ts)
    sims = W.batched_membranes(count=args.count, seed=0)
    cells = sum(s["nx"] * s["ny"] for s in sims)
    markers = sum(len(s["X"]) for s in sims)
    K, Wm = args.steps, args.warmup

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    def slowest(x):
        return max_over_ranks([x], dist)[0]

    # plain per-simulation form: every lattice on its own stream, stepped by its own calls
    lat = [batch_lattice(iilbm, s) for s in sims]
    Kp = max(32, min(K, 512) // 32 * 32)
    for g in lat:
        g.step(Wm)
    barrier()
    t0 = time.perf_counter()
    for g in lat:
        g.step(Kp)
    barrier()
    plain_s = slowest(time.perf_counter() - t0)
    plain = whole_job_mlups(cells, Kp, world, plain_s)
    # batched: one launch per phase per step for all lattices, graph replay
    if Wm % 2:
        for g in lat:  # keep every lattice at the same parity as a fresh one
            g.step(1)
    B = iilbm.Batch(lat, stream=ts.cuda_stream)
    variant, tune_us = B.autotune(64)
    B.step(max(Wm, 3))
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(ts)
    B.step(K)
    e1.record(ts)
    barrier()
    ms = slowest(e0.elapsed_time(e1))
    # second region, eager steps with events around every batched lean stream-collide
    Kt = min(K, 256)
    B.iilbm_batch_set_timing(True)
    barrier()
    B.step(Kt)
    barrier()
    sc_ms, sc_n, launches = B.iilbm_batch_get_timing()
    B.iilbm_batch_set_timing(False)
    clk = clocks.stop()
    B.synchronize()
    value = whole_job_mlups(cells, K, world, ms * 1e-3)
    peak, peak_kind = peaks()
    step_bytes = 2 * 9 * 4 * cells
    achieved = step_bytes / (ms * 1e-3 / K) / 1e9
    sc_avg = sc_ms / max(sc_n, 1) * 1e-3
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": None,
                "kernel": "whole batched step (every node updated once: lean and forced "
                          "stream-collide; interface and interpolation overlapped)",
                "peak_source": peak_kind, "alg_bytes_per_step": step_bytes,
                "lean_stream_collide_avg_us": round(sc_avg * 1e6, 2),
                "lean_stream_collide_upper_frac": round(step_bytes / sc_avg / 1e9 / peak, 4)}
    B.close()
    e2e = None
    if not args.no_e2e:
        # through the C ABI: marker polygons from pinned host memory, the batch stepped,
        # every lattice's velocity field read back to pinned host memory
        del lat
        torch.cuda.synchronize()
        lat = [batch_lattice(iilbm, s, with_interface=False) for s in sims]
        Xin = [torch.from_numpy(np.ascontiguousarray(s["X"])).pin_memory() for s in sims]
        outs = [(torch.empty((s["ny"], s["nx"]), dtype=torch.float64).pin_memory(),
                 torch.empty((s["ny"], s["nx"]), dtype=torch.float64).pin_memory()) for s in sims]
        barrier()
        t0 = time.perf_counter()
        for g, s, X in zip(lat, sims, Xin):
            g.set_interface(X, model=iilbm.SPRING, stiffness=s["kappa"], dX=s["dX"])
        B2 = iilbm.Batch(lat, stream=ts.cuda_stream)
        B2.iilbm_batch_set_variant(variant)
        B2.step(K)
        for g, (ux, uy) in zip(lat, outs):
            g.get_macros(None, ux, uy, want=(False, True, True))
        barrier()
        dt = slowest(time.perf_counter() - t0)
        B2.close()
        e2e = {"value": round(whole_job_mlups(cells, K, world, dt), 1), "unit": "MLUPS",
               "h2d_bytes_per_step": round(markers * 16 / K, 1),
               "d2h_bytes_per_step": round(2 * cells * 8 / K, 1),
               "note": "set_interface of every lattice from pinned host, batch creation, "
                       "K batched steps, every velocity field read back to pinned host"}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        rate, st, dt, used = oracle_batch_rate(sims, 12.0)
        cpu = {"value": round(rate, 4), "unit": "MLUPS", "cores": 1, "kind": "oracle",
               "sample": f"{st} FP64 oracle steps of each of the first {used} simulations of "
                         f"the sweep, one after another, {dt:.1f} s, one thread"}
    if rank == 0:
        out = {"metric": "MLUPS", "value": round(value, 1), "unit": "MLUPS", "n_gpus": world,
               "steps": K, "warmup": Wm, "ms_per_step": round(ms / K, 5),
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic",
               "config": {"workload": f"batched{args.count}_membranes_f32",
                          "simulations": args.count, "cells": cells, "markers": markers,
                          "collision": "mrt", "storage": "f32", "arithmetic": "f32",
                          "variant": iilbm.BATCH_VARIANTS[variant],
                          "autotune_us_per_step": round(tune_us, 2),
                          "parallelism": "replicas" if world > 1 else "single",
                          "l2": f"inputs larger than L2 ({36 * cells / 2**20:.0f} MiB "
                                "populations vs 129 MiB L2)"},
               "plain_per_simulation": {"value": round(plain, 1), "unit": "MLUPS",
                                        "steps": Kp, "speedup_of_batch": round(value / plain, 2),
                                        "form": "each lattice stepped by its own iilbm_step "
                                                "calls on its own stream (graph replay)"},
               "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
               "gpu_launches": int(launches / max(sc_n, 1) * K)}
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


# ------------------------------------------------------- learned warm start
def oracle_channel_rate(max_seconds):
    """The FP64 oracle stepping one learned-workload channel (iteration to 1e-6)."""
    from oracle import oracle as O
    sim = W.learned_channels(1, 2)[0]
    nx, ny = sim["nx"], sim["ny"]
    o = O.Oracle(nx, ny, collision=O.MRT, tau=sim["tau"], s=W.mrt_rates(sim["tau"]),
                 bc=O.BC_CHANNEL, u_max=sim["u_max"], jump=1)
    y = np.arange(ny) + 0.5
    o.init_equilibrium(None, np.repeat((4 * sim["u_max"] * y * (ny - y) / ny ** 2)[:, None], nx,
                                       axis=1), None)
    o.set_interface(sim["X"], model=O.DIRECT, moves=False, dX=sim["dX"], eta=2.0, mdf_iters=500,
                    mdf_tol=1e-6, UD=np.zeros((sim["n"], 2)))
    steps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < max_seconds:
        o.step(1)
        steps += 1
    dt = time.perf_counter() - t0
    o.close()
    return nx * ny * steps / dt / 1e6, steps, dt


def run_learned(args):
    import torch
    from paper_2003_12186_gb300 import learned as LL

    rank = int(os.environ.get("RANK", "0"))
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    t0 = time.perf_counter()
    X, T, _ = LL.generate(count=64, seed=1, spin_up=400, records=64, every=100)
    gen_s = time.perf_counter() - t0
    mlp, norm, rep = LL.train(X, T, epochs=30)
    rep["generate_seconds"] = round(gen_s, 2)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    ev = LL.evaluate(mlp, count=64, seed=2, spin_up=400, count_steps=32,
                     timed_steps=max(args.steps, 32))
    clk = clocks.stop()
    sims = W.learned_channels(64, 2)
    cells = sum(s["nx"] * s["ny"] for s in sims)
    peak, peak_kind = peaks()
    L, P = ev["mlp"], ev["plain"]
    step_bytes = 2 * 9 * 4 * cells
    achieved = step_bytes / (L["us_per_step"] * 1e-6) / 1e9
    cpu = None
    if rank == 0 and not args.no_cpu:
        rate, st, dt = oracle_channel_rate(10.0)
        cpu = {"value": round(rate, 4), "unit": "MLUPS", "cores": 1, "kind": "oracle",
               "sample": f"{st} FP64 oracle steps of one channel of the workload (force "
                         f"iteration to 1e-6), {dt:.1f} s, one thread"}
    if rank == 0:
        out = {"metric": "MLUPS", "value": round(L["mlups"], 1), "unit": "MLUPS", "n_gpus": 1,
               "steps": max(args.steps, 32), "warmup": 400,
               "ms_per_step": round(L["us_per_step"] / 1e3, 5), "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": "learned64_cylinder_channels_f32", "channels": 64,
                          "lattice": [512, 128], "cells": cells, "residual_tol": 1e-6,
                          "max_passes": 500, "markers_spacing": 1.5, "jump": 1,
                          "l2": "inputs larger than L2"},
               "learned": {"passes_per_step": round(L["passes_per_step"], 2),
                           "worst_residual": L["worst_residual"], "capped": L["capped"]},
               "plain_iteration": {"value": round(P["mlups"], 1), "unit": "MLUPS",
                                   "passes_per_step": round(P["passes_per_step"], 2),
                                   "worst_residual": P["worst_residual"],
                                   "speedup_of_learned": round(L["mlups"] / P["mlups"], 3),
                                   "passes_saved": round(1 - L["passes_per_step"] /
                                                         P["passes_per_step"], 3)},
               "previous_force_start": {"value": round(ev["previous"]["mlups"], 1),
                                        "unit": "MLUPS",
                                        "passes_per_step": round(ev["previous"]["passes_per_step"], 2)},
               "training": rep,
               "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                            "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": None,
                            "kernel": "whole step (the force iteration, one CTA per body, "
                                      "dominates; the stream-collide is the HBM part)",
                            "peak_source": peak_kind, "alg_bytes_per_step": step_bytes},
               "cpu_baseline": cpu, "e2e": None, "clocks": clk,
               # per step: lean and forced stream-collide, interpolation, force
               # iteration, marker and segment passes, channel ends
               "gpu_launches": 7 * max(args.steps, 32)}
        print(json.dumps(out), flush=True)


# --------------------------------------------------------------- channel
def run_channel(args):
    import torch
    from paper_2003_12186_gb300 import iilbm

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    ts = torch.cuda.Stream()
    torch.cuda.set_stream(ts)
    w = W.cylinder_channel(args.re)
    nx, ny, n = w["nx"], w["ny"], len(w["X"])
    g = iilbm.Lattice(nx, ny, collision=iilbm.MRT, storage="f32", tau=w["tau"],
                      s=W.mrt_rates(w["tau"]), bc=iilbm.BC_CHANNEL, u_max=w["u_max"],
                      stream=ts.cuda_stream)
    y = np.arange(ny) + 0.5
    u0 = np.repeat((4 * w["u_max"] * y * (ny - y) / ny ** 2)[:, None], nx, axis=1)
    g.init_equilibrium(None, u0, None)
    g.set_interface(w["X"], model=iilbm.DIRECT, moves=False, dX=w["dX"], eta=2.0, mdf_iters=5,
                    aux=np.zeros((n, 2)))
    g.step(args.warmup)
    g.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0.record(ts)
    g.step(args.steps)
    e1.record(ts)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms, = max_over_ranks([e0.elapsed_time(e1)], dist)
    g.iilbm_set_timing(True)
    g.step(min(args.steps, 128))
    sc_ms, sc_n, launches = g.iilbm_get_timing()
    g.iilbm_set_timing(False)
    clk = clocks.stop()
    F = g.iilbm_get_body_force()
    # drag / lift history (untimed): the force every 20 steps over args.history steps,
    # C = 2 F / (rho U^2 D) with U = u_max (Eqs. 52-53), St = f D / U from the lift's
    # mean-crossing period (Eq. 51)
    hist = None
    if args.history > 0:
        cd, cl = [], []
        for _ in range(args.history // 20):
            g.step(20)
            Fx, Fy = g.iilbm_get_body_force()
            cd.append(2 * Fx / (w["u_max"] ** 2 * w["D"]))
            cl.append(2 * Fy / (w["u_max"] ** 2 * w["D"]))
        cd, cl = np.array(cd), np.array(cl)
        c = cl - cl.mean()
        up = np.nonzero((c[:-1] < 0) & (c[1:] >= 0))[0]
        st = None
        if len(up) >= 3:
            period = 20.0 * (up[-1] - up[0]) / (len(up) - 1)
            st = w["D"] / (period * w["u_max"])
        hist = {"steps": args.history, "every": 20, "C_D_mean": round(float(cd.mean()), 4),
                "C_D_amplitude": round(float((cd.max() - cd.min()) / 2), 4),
                "C_L_amplitude": round(float((cl.max() - cl.min()) / 2), 4),
                "C_L_mean": round(float(cl.mean()), 4),
                "St": None if st is None else round(float(st), 4),
                "lift_periods": max(len(up) - 1, 0),
                "context": "paper, section 4.3 (its own setup: uniform inflow, D = 80 in "
                           "[0, 40D] x [0, 20D]): Re 100 C_D 1.417, C_L +-0.344, St 0.169; "
                           "here a confined channel (blockage 0.16) with a parabolic inflow, "
                           "coefficients on u_max"}
    cells = nx * ny
    value = whole_job_mlups(cells, args.steps, world, ms * 1e-3)
    peak, peak_kind = peaks()
    sc_avg = sc_ms / max(sc_n, 1) * 1e-3
    lean_bytes = 2 * 9 * 4 * cells
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        from oracle import oracle as O
        o = O.Oracle(nx, ny, collision=O.MRT, tau=w["tau"], s=W.mrt_rates(w["tau"]),
                     bc=O.BC_CHANNEL, u_max=w["u_max"])
        o.init_equilibrium(None, u0, None)
        o.set_interface(w["X"], model=O.DIRECT, moves=False, dX=w["dX"], eta=2.0, mdf_iters=5,
                        UD=np.zeros((n, 2)))
        st, t0 = 0, time.perf_counter()
        while time.perf_counter() - t0 < 10.0:
            o.step(1)
            st += 1
        dt = time.perf_counter() - t0
        o.close()
        cpu = {"value": round(cells * st / dt / 1e6, 4), "unit": "MLUPS", "cores": 1,
               "kind": "oracle", "sample": f"{st} FP64 oracle steps of the same channel, "
                                           f"{dt:.1f} s, one thread"}
    if rank == 0:
        out = {"metric": "MLUPS", "value": round(value, 1), "unit": "MLUPS", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": round(ms / args.steps, 5), "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": f"cylinder_channel_1024x256_re{args.re:g}_f32",
                          "lattice": [nx, ny], "markers": n, "tau": w["tau"],
                          "force_updates_per_step": 5,
                          "l2": "working set (19 MB) fits in L2: the roofline is not an HBM bound"},
               "drag_lift": {"Fx": F[0], "Fy": F[1],
                             "C_D": 2 * F[0] / (w["u_max"] ** 2 * 40.0),
                             "note": "after warmup + the timed steps, from the parabolic start",
                             "history": hist},
               "roofline": {"bound": "hbm", "achieved": round(lean_bytes / sc_avg / 1e9, 1),
                            "peak": peak, "unit": "GB/s",
                            "frac": round(lean_bytes / sc_avg / 1e9 / peak, 4), "traffic": None,
                            "kernel": "k_stream_collide_vec (lean), L2-resident",
                            "peak_source": peak_kind,
                            "avg_launch_us": round(sc_avg * 1e6, 2)},
               "cpu_baseline": cpu, "e2e": None, "clocks": clk,
               "gpu_launches": int(launches / max(sc_n, 1) * args.steps)}
        print(json.dumps(out), flush=True)


# ------------------------------------------------------- three dimensions
def membrane3d_config(args, w):
    sb = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2}[args.storage]
    n = w["n"]
    return {"workload": f"membrane3d_{n}^3_tension_ellipsoid", "lattice": [n, n, n],
            "vertices": len(w["X"]), "triangles": len(w["T"]), "collision": "mrt (d'Humieres D3Q19)",
            "tau": w["tau"], "gamma": w["gamma"], "storage": args.storage,
            "arithmetic": "f64" if args.storage == "f64" else "f32",
            "l2": f"inputs larger than L2 ({19 * sb * n ** 3 / 2**20:.0f} MiB populations vs "
                  f"129 MiB L2)"}


def oracle3d_rate(w, max_seconds, parallel):
    from oracle import oracle3d as O3
    n = w["n"]
    o = O3.Oracle3D(n, n, n, parallel=parallel, collision=O3.MRT, tau=w["tau"])
    o.set_surface(w["X"], w["T"], model=O3.TENSION, moves=True, gamma=w["gamma"])
    steps, t0 = 0, time.perf_counter()
    while steps < 1 or time.perf_counter() - t0 < max_seconds:
        o.step(1)
        steps += 1
    dt = time.perf_counter() - t0
    return n ** 3 * steps / dt / 1e6, steps, dt


def run_membrane3d(args):
    """The D3Q19 II-LBM membrane: a surface-tension ellipsoid in a periodic n^3 box."""
    import torch
    from paper_2003_12186_gb300 import iilbm3d

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    ts = torch.cuda.Stream()
    torch.cuda.set_stream(ts)
    w = W.membrane_3d(args.size3)
    n = w["n"]
    cells = n ** 3
    sb = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2}[args.storage]

    def lattice():
        g = iilbm3d.Lattice3D(n, n, n, collision=iilbm3d.MRT, storage=args.storage, tau=w["tau"],
                              stream=ts.cuda_stream)
        return g

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    g = lattice()
    g.set_surface(w["X"], w["T"], model=iilbm3d.TENSION, moves=True, gamma=w["gamma"])
    g.step(args.warmup)  # captures the two-step graph
    g.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    clocks.begin()
    e0.record(ts)
    g.step(args.steps)
    e1.record(ts)
    barrier()
    clocks.end()
    ms = e0.elapsed_time(e1)
    # second region: eager steps with CUDA events around every stream-collide launch
    K2 = min(args.steps, 100)
    g.set_timing(True)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    f0.record(ts)
    g.step(K2)
    f1.record(ts)
    barrier()
    ms2 = f0.elapsed_time(f1)
    sc_ms, sc_n, kernels = g.get_timing()
    g.set_timing(False)
    clk = clocks.stop()
    cut = g.get_cut_link_count()
    ms, = max_over_ranks([ms], dist)
    value = whole_job_mlups(cells, args.steps, world, ms * 1e-3)
    peak, peak_kind = peaks()
    alg = 2 * 19 * sb * cells
    sc_avg = sc_ms / max(sc_n, 1) * 1e-3
    achieved = alg / sc_avg / 1e9
    step_ach = alg / (ms / args.steps * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": None,
                "kernel": "k3_stream_collide (every node, flagged tiles with the spread force)",
                "peak_source": peak_kind, "alg_bytes_per_launch": alg,
                "avg_launch_us": round(sc_avg * 1e6, 2),
                "timed_in": f"second region of {K2} eager steps with CUDA events around each "
                            f"stream-collide ({ms2 / K2 * 1e3:.1f} us/step there)",
                "step_achieved": round(step_ach, 1), "step_frac": round(step_ach / peak, 4),
                "frac_nominal_8tbs": round(achieved / NOMINAL_HBM_GBS, 4)}
    tr = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tr):
        d = json.load(open(tr)).get(f"membrane3d_{n}_{args.storage}")
        if d:
            roofline["traffic"] = d
    if args.storage == "f64":
        # FP64 arithmetic is bound by GB300's FP64 pipe, not by HBM: the roof is the FP64
        # rate, the work the D3Q19 MRT collision's algorithmic flops per node (counted
        # from the pair-symmetric collision without force; the forced tiles are a few %)
        flops = D3Q19_MRT_FLOPS_PER_NODE * cells
        hbm = {("hbm_" + k): roofline[k] for k in ("achieved", "peak", "frac")}
        roofline.update({"bound": "alu", "achieved": round(flops / sc_avg / 1e12, 4),
                         "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": round(flops / sc_avg / 1e12 / FP64_PEAK_TFLOPS, 4),
                         "peak_source": "derived: 152 SMs x 2 FP64 FMA/clock x 2 flops x "
                                        "2.07 GHz (nominal FP64 rate of GB300)",
                         "flops_per_node": D3Q19_MRT_FLOPS_PER_NODE, **hbm})
    del g
    e2e = None
    if not args.no_e2e:
        torch.cuda.synchronize()
        g2 = lattice()
        Xin = torch.from_numpy(np.ascontiguousarray(w["X"])).pin_memory()
        Xout = torch.empty((len(w["X"]), 3), dtype=torch.float64).pin_memory()
        u = [torch.empty((n, n, n), dtype=torch.float64).pin_memory() for _ in range(3)]
        K3 = min(args.steps, 100)
        g2.set_surface(Xin.numpy(), w["T"], model=iilbm3d.TENSION, moves=True, gamma=w["gamma"])
        g2.step(2)
        g2.synchronize()
        barrier()
        t0 = time.perf_counter()
        g2.set_surface(Xin.numpy(), w["T"], model=iilbm3d.TENSION, moves=True, gamma=w["gamma"])
        for _ in range(K3):
            g2.step(1)
            g2.get_markers_into(X=Xout)
        _, ux, uy, uz = g2.get_macros()
        for a, b in zip(u, (ux, uy, uz)):
            a.copy_(torch.from_numpy(b))
        barrier()
        dt = time.perf_counter() - t0
        dt, = max_over_ranks([dt], dist)
        h2d = Xin.numel() * 8 + w["T"].size * 4
        d2h = K3 * Xout.numel() * 8 + 3 * cells * 8
        e2e = {"value": round(whole_job_mlups(cells, K3, world, dt), 1), "unit": "MLUPS",
               "h2d_bytes_per_step": round(h2d / K3, 1), "d2h_bytes_per_step": round(d2h / K3, 1),
               "note": "inside the region: the surface installed from host memory, per step "
                       "iilbm3d_step(1) + vertex read-back to pinned host, final velocity "
                       "field read-back"}
        del g2
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        from oracle import oracle3d as O3
        try:
            rp, stp, dtp = oracle3d_rate(w, 8.0, True)
            cpu = {"value": round(rp, 4), "unit": "MLUPS", "cores": O3.omp_threads(),
                   "kind": "oracle", "sample": f"{stp} FP64 oracle steps of the same "
                   f"{n}^3 workload, {dtp:.1f} s, OpenMP build"}
        except RuntimeError:
            r1, st1, dt1 = oracle3d_rate(w, 10.0, False)
            cpu = {"value": round(r1, 4), "unit": "MLUPS", "cores": 1, "kind": "oracle",
                   "sample": f"{st1} FP64 oracle steps of the same {n}^3 workload, "
                   f"{dt1:.1f} s, one thread"}
    if rank == 0:
        out = {"metric": "MLUPS", "value": round(value, 1), "unit": "MLUPS", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": round(ms / args.steps, 5), "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": args.storage,
               "data": "synthetic", "config": membrane3d_config(args, w),
               "cut_links_per_step": cut, "roofline": roofline, "cpu_baseline": cpu,
               "e2e": e2e, "clocks": clk,
               "gpu_launches": int(kernels / max(sc_n, 1) * args.steps)}
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def run_reference3d(args):
    """Reference arm of the 3-D workload: the 3-D oracle (OpenMP build), rank 0 only, a
    bounded number of steps of the same configuration."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    from oracle import oracle3d as O3
    try:
        O3.lib(parallel=True)
        par = True
    except RuntimeError:
        par = False
    w = W.membrane_3d(args.size3)
    rate, steps, dt = oracle3d_rate(w, 20.0, par)
    cores = O3.omp_threads() if par else 1
    sample = (f"{steps} FP64 oracle steps of the {w['n']}^3 membrane, "
              + (f"OpenMP build on {cores} threads" if par else "one thread"))
    out = {"metric": "MLUPS", "value": round(rate, 4), "unit": "MLUPS", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / steps * 1e3, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "impl": "reference", "config": membrane3d_config(args, w),
           "cpu_baseline": {"value": round(rate, 4), "unit": "MLUPS", "cores": cores,
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": round(rate, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference" and args.workload == "membrane3d":
        run_reference3d(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "membrane3d":
        run_membrane3d(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "learned":
        run_learned(args)
    elif args.workload == "channel":
        run_channel(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
