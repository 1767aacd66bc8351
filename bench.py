"""Benchmark: VMS Jacobian-vector products per second on the sphere LES workload (one GB300).

A step is one application of J(u) v over the whole mesh: Out elements on the 2x2x2 Gauss
rule, Intercepted elements on their adaptive sub-cell points, Nitsche surface points, scatter
through the hanging-node operator, strong rows.  The workload is a 32 x 16 x 16 box with a
sphere of diameter 1 (81,920 triangles), octree levels 4-10 with a wake cone, 2,001,176
elements, Re 1e4, BDF2 dt 0.01; inputs are seeded synthetic states (uniform inflow + N(0, 0.01)
noise, v ~ N(0, 1)).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64] [--impl ours|reference]

Multi-GPU: every rank solves its own independent problem (a replica of the workload with its own
seed), so the units shard with no data-path collective ("scaling": "weak").  --impl reference
times the FP64 CPU oracle on a bounded sample of the same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2009_00706_gb300 import inputs as I  # noqa: E402

METRIC = "VMS Jv elements/s; Newton-GMRES step time to 1e-8, mixed/learned vs FP64"
UNIT = "elements/s"
L2_BYTES = 129 * 2 ** 20

# Algorithmic FP32 work of one Out element in the forward-mode J v, counted in the nodal form:
# 8 Gauss points x (interpolation of values + tangents 896, pointwise VMS + tangent 390, weights 16)
# + contraction of 8 nodes x 4 rows over 8 points (2048).
FLOPS_JV_OUT_ELEMENT = 8 * (896 + 390 + 16) + 2048
FP64_TFLOPS_NOMINAL = 1.25


# algorithmic work per unit of the other kernels of the mixed J v step (BDF2)
FLOPS_JV_SUBCELL_POINT = 896 + 390 + 16 + 256     # a Gauss point's work incl. its share of the contraction
FLOPS_JV_SURFACE_POINT_EST = 920                  # estimate: interpolation 512, pointwise 150, rows 256
BYTES_NODE_PREP_NODE = 4 * 32 + 2 * 32            # reads u, u_prev, u_prev2, v; writes value + tangent rows
BYTES_NODE_PREP_HANGING = 3 * 2 * 32 + 2 * 32     # ~3 parents' two rows read, two rows written


def kernel_rooflines(prof, steps, info, n_nodes, pk):
    """Per kernel class of the timed step: average ms per step, bound, achieved, fraction of peak."""
    out = {}
    hbm = pk["hbm_gbs"]
    fp32 = pk["fp32_tflops"]
    work = {
        "out_elements": ("alu", FLOPS_JV_OUT_ELEMENT * info["n_out"], fp32, "TFLOP/s"),
        "cut_elements": ("alu", FLOPS_JV_SUBCELL_POINT * info["n_cut_points"], fp32, "TFLOP/s"),
        "nitsche": ("alu (estimated flop)", FLOPS_JV_SURFACE_POINT_EST * info["n_surface_points"], fp32, "TFLOP/s"),
        "node_prep": ("hbm", BYTES_NODE_PREP_NODE * n_nodes + BYTES_NODE_PREP_HANGING * info["n_hanging"], hbm, "GB/s"),
    }
    rec = step_kernel_record()
    for k, (bound, units, peak, unit) in work.items():
        ms = prof[k][0] / max(1, steps)
        if ms <= 0:
            continue
        scale = 1e12 if unit == "TFLOP/s" else 1e9
        ach = units / (ms / 1e3) / scale
        out[k] = {"ms_per_step": ms, "bound": bound, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak}
        ex = rec.get(k)
        if ex:   # executed work from the committed ncu counters of this source (per launch of the class)
            if unit == "TFLOP/s":
                f32, f64 = ex["fp32_flop"], ex["fp64_flop"]
                out[k]["executed"] = {"fp32_tflops": f32 / (ms / 1e3) / 1e12, "fp32_frac": f32 / (ms / 1e3) / 1e12 / fp32,
                                      "fp64_tflops": f64 / (ms / 1e3) / 1e12,
                                      "fp64_frac": f64 / (ms / 1e3) / 1e12 / pk["fp64_tflops"]}
            else:
                out[k]["dram"] = {"bytes": ex["dram_bytes"], "gbs": ex["dram_bytes"] / (ms / 1e3) / 1e9,
                                  "frac": ex["dram_bytes"] / (ms / 1e3) / 1e9 / hbm}
    # class 3: with the deterministic scatter (the default) the node sums, which also write the strong
    # rows: bound by the latency of two dependent loads per incidence entry (code, then a 16-byte slot
    # row); with the atomic scatter only the strong rows, a few microseconds of launch latency
    ms3 = prof["strong_rows"][0] / max(1, steps)
    out["strong_rows"] = {"ms_per_step": ms3, "nodes_per_s": n_nodes / (ms3 / 1e3) if ms3 > 0 else None,
                          "bound": "latency of dependent loads (node sums of the deterministic scatter)"
                          if ms3 > 0.05 else "launch latency (strong rows only)"}
    return out


def wpart_costs(prof, steps, info):
    """Eq. Wpart's costs on this GPU, from the per-kernel times of the timed J v steps: T_v per
    volume Gauss point (the Out elements' 8 and the Intercepted elements' kept sub-cell points),
    T_s per surface Gauss point (the Nitsche kernels), in picoseconds.  With n_Tgp = 8 for Q1,
    W(e) = n_Vgp(e) / 8 + (T_s / T_v) n_Sgp(e) / 8."""
    s = max(1, steps)
    t_out, t_cut, t_sur = (prof[k][0] / s for k in ("out_elements", "cut_elements", "nitsche"))
    n_out, n_cut, n_sur = 8 * info["n_out"], info["n_cut_points"], info["n_surface_points"]
    if n_out + n_cut == 0 or n_sur == 0:
        return None
    tv = (t_out + t_cut) / (n_out + n_cut) * 1e9
    ts = t_sur / n_sur * 1e9
    return {"T_v_ps": tv, "T_s_ps": ts, "T_s_over_T_v": ts / tv,
            "T_out_point_ps": t_out / max(1, n_out) * 1e9, "T_cut_point_ps": t_cut / max(1, n_cut) * 1e9}


def interior_record():
    """The committed ncu record of vms_interior (DRAM bytes per launch, executed flops per element),
    or an empty dict when the kernel source changed since the counters were taken."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "vms_interior_traffic.json")))
        h = hashlib.sha256()
        for f in ("paper_2009_00706_gb300/csrc/vms.cu", "paper_2009_00706_gb300/csrc/vms_device.cuh"):
            h.update(open(os.path.join(ROOT, f), "rb").read())
        return rec if h.hexdigest() == rec["source_sha256"] else {}
    except Exception:
        return {}


def step_kernel_record():
    """Executed flops / DRAM bytes per step of the Intercepted, surface and node-preparation kernels
    from the committed ncu record (profiles/step_kernel_counters.json), or {} when the kernel source
    changed since the counters were taken."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "step_kernel_counters.json")))
        h = hashlib.sha256()
        for f in ("paper_2009_00706_gb300/csrc/vms.cu", "paper_2009_00706_gb300/csrc/vms_device.cuh"):
            h.update(open(os.path.join(ROOT, f), "rb").read())
        return rec["classes"] if h.hexdigest() == rec["source_sha256"] else {}
    except Exception:
        return {}


def interior_traffic():
    """DRAM bytes per launch of vms_interior from the committed ncu record, or None when stale."""
    return interior_record().get("traffic_bytes_per_launch")


def peaks(api=None, device=0):
    """Roofline denominators.  HBM: MEASURED_PEAKS.json (the driver's copy benchmark).  FP32 / FP64:
    the library's own FMA microbenchmark on this GPU (imga_peak_flops: scalar FFMA, packed FFMA2,
    DFMA), the FP32 peak being the faster of the two FP32 forms; without a GPU the unit-count
    formula SMs x 128 lanes x 2 x max clock, with the SM count read from the device when there is
    one."""
    p = {"source": "fallback", "sm_max_mhz": 2070.0, "hbm_gbs": 6800.0}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        p.update({"source": "measured", "sm_max_mhz": float(d.get("sm_max_mhz", 2070.0)),
                  "hbm_gbs": float(d.get("hbm_gbs", 6800.0))})
    except Exception:
        pass
    sms = 152
    try:
        import torch
        sms = torch.cuda.get_device_properties(device).multi_processor_count
    except Exception:
        pass
    p["sm_count"] = sms
    p["fp32_tflops"] = sms * 128 * 2 * p["sm_max_mhz"] * 1e6 / 1e12
    p["fp64_tflops"] = FP64_TFLOPS_NOMINAL
    p["fp_source"] = f"derived: {sms} SMs x 128 FP32 lanes x 2 x max SM clock; FP64 nominal"
    if api is not None:
        try:
            f32, f32x2, f64 = (api.peak_flops(k, device) for k in (0, 1, 2))
            p.update({"fp32_ffma_tflops": f32, "fp32_ffma2_tflops": f32x2, "fp64_dfma_tflops": f64,
                      "fp32_tflops": max(f32, f32x2), "fp64_tflops": f64,
                      "fp_source": "measured: imga_peak_flops FMA microbenchmark on this GPU "
                                   "(FP32 = faster of FFMA and packed FFMA2; FP64 = DFMA)"})
        except Exception as ex:
            p["fp_source"] += f" (microbenchmark failed: {ex!r})"
    return p


class Clocks:
    """nvidia-smi samples (every 50 ms) taken while the timed region runs.

    `wait_live` keeps the GPU busy with untimed steps until the sampler has written its first line,
    so that the sampler is running when the timed region starts; `mark` records the file offset at
    the start and end of the timed region, and `summary` reads only the samples written between
    the two marks (or, if the region was shorter than one interval, the first sample after it)."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"imga_bench_clocks_{os.getpid()}.csv")
        self.marks = []

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def _size(self):
        try:
            return os.path.getsize(self.path)
        except OSError:
            return 0

    def wait_live(self, work, limit_s=5.0):
        """run `work()` (an untimed step) until the sampler has written a line, at most limit_s"""
        import torch
        t0 = time.perf_counter()
        while self.proc and self.proc.poll() is None and self._size() == 0 and time.perf_counter() - t0 < limit_s:
            for _ in range(20):
                work()
            torch.cuda.synchronize()

    def mark(self):
        self.marks.append(self._size())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        data = open(self.path, "rb").read()
        lo, hi = (self.marks + [0, len(data)])[:2] if len(self.marks) >= 2 else (0, len(data))
        lines = data[lo:hi].decode(errors="replace").splitlines()
        window = "samples written during the timed region"
        if not [x for x in lines if x.count(",") >= 8]:
            lines = data[hi:].decode(errors="replace").splitlines()[:1]
            window = "timed region shorter than the 50 ms interval: the first sample after it"
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "sm_mhz_min": min(sm), "window": window}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(x, world, dev=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, steps, max_ms, world):
    """Whole-job units/s: every rank processes units_per_rank per step; the slowest rank's time counts."""
    return world * units_per_rank * steps / (max_ms / 1e3)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------------------------------
# reference arm and CPU baseline: the FP64 oracle on a bounded sample of the workload
# ------------------------------------------------------------------------------------------
def oracle_sample(w, n_nodes_sample, seed=0):
    """Build the oracle mesh (untimed), then time residual + J v of the elements touching a
    seeded sample of nodes.  Returns (elements/s, elements per sample, seconds per sample, om)."""
    from oracle.oracle import OracleMesh
    tri = w.triangles()
    om = OracleMesh(w.lo, w.hi, w.base_level, w.regions, tri, w.lmax)
    u, up, v = I.state(om.n_nodes, seed)
    return om, u, up, v


def time_oracle(om, w, u, up, v, sel, rows=False, threads=1, prepared=False):
    """One timed residual + J v of the oracle over the elements touching the nodes `sel`, with its
    element loop on `threads` host threads (the geometry of the sample is computed untimed first,
    unless an earlier call on the same sample already did)."""
    from oracle import oracle
    if not prepared:
        om.residual_jvp(w.physics, u, up, up, v=v, nodes=sel)      # geometry of the sample, untimed
    oracle.set_threads(threads)
    try:
        t = time.perf_counter()
        R, J = om.residual_jvp(w.physics, u, up, up, v=v, nodes=sel)
        dt = time.perf_counter() - t
    finally:
        oracle.set_threads(1)
    if rows:
        return om.counters()["elements_evaluated"], dt, R, J
    return om.counters()["elements_evaluated"], dt


def parity_on_sample(mesh, ph, ud, upd, up2d, vd, sel, Ro, Jo):
    """R and J v of the GPU path (float64 and mixed) against the oracle on the sampled rows."""
    from paper_2009_00706_gb300 import api
    out = {"nodes": int(sel.size), "bound": {"fp64": 1e-10, "mixed": 2e-5}}
    for name, p in (("fp64", api.PRECISION_FP64), ("mixed", api.PRECISION_MIXED)):
        Rg = mesh.residual(ph, ud, upd, up2d, precision=p).cpu().numpy()[sel]
        Jg = mesh.jvp(ph, ud, upd, vd, up2d, precision=p).cpu().numpy()[sel]
        r = {}
        for key, g, o in (("R", Rg, Ro[sel]), ("Jv", Jg, Jo[sel])):
            r[key + "_rel_l2"] = float(np.linalg.norm(g - o) / max(np.linalg.norm(o), 1e-300))
            r[key + "_max_abs"] = float(np.abs(g - o).max())
        out[name] = r
    return out


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    w = I.sphere_les(0)
    om, u, up, v = oracle_sample(w, 0)
    # per-step sample: at most ref_sample_nodes seeded nodes, and about 4 M node samples over the
    # whole run, so that any --steps ends within a few minutes on the host cores
    nodes = max(1000, min(args.ref_sample_nodes, 4_000_000 // max(1, args.steps)))
    rng_sel = lambda k: np.unique(I.splitmix64(1000 + k, nodes) % om.n_nodes).astype(np.int64)
    cores = os.cpu_count() or 1
    # one seeded sample whose geometry (markers by a ray against every triangle, sub-cell points,
    # surface points) the oracle computes once, untimed: about 2 ms per element on one core, which
    # a fresh sample per step would pay again; every step is one timed oracle call on it (each call
    # also pays the oracle's full-size per-thread vectors)
    pool = [rng_sel(0)]
    for sel in pool:
        om.residual_jvp(w.physics, u, up, up, v=v, nodes=sel)
    for k in range(args.warmup):
        time_oracle(om, w, u, up, v, pool[k % len(pool)], threads=cores, prepared=True)
    ne_tot, t_tot = 0, 0.0
    for k in range(args.steps):
        ne, dt = time_oracle(om, w, u, up, v, pool[k % len(pool)], threads=cores, prepared=True)
        ne_tot += ne
        t_tot += dt
    val = ne_tot / t_tot
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "sphere_les", "elements": om.n_elem, "sample": "elements touching "
                       f"the same {nodes} seeded nodes every step, residual + J v", "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{ne_tot} element evaluations over {args.steps} steps, element loop on "
                                       f"{cores} threads (os.cpu_count())"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------
def run_ours(args):
    import torch

    from paper_2009_00706_gb300 import _lib, api

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _lib.build()
    w = I.sphere_les(0)
    prec = api.PRECISION_MIXED if args.precision == "mixed" else api.PRECISION_FP64
    t0 = time.perf_counter()
    mesh = api.Mesh.from_workload(w, device=local)
    build_s = time.perf_counter() - t0
    info = mesh.info
    nn = mesh.n_nodes
    n_active = info["n_out"] + info["n_cut"]
    u, up, v = I.state(nn, rank)
    up2 = up.copy()
    ud, upd, up2d, vd = (torch.from_numpy(a).to(dev) for a in (u, up, up2, v))
    out = torch.empty_like(ud)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    ph = w.physics

    def step(p=prec):
        mesh.jvp(ph, ud, upd, vd, up2d, precision=p, out=out, stream=stream)

    mesh.autotune(True)   # the first warm-up step picks the Intercepted-element tile shape
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # device-timed region: per-step events, L2 flushed (untimed) between steps
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with Clocks(local) as clk:
        clk.wait_live(step)
        mesh.profile(True)
        barrier(world)
        torch.cuda.synchronize()
        wall0 = time.perf_counter()
        clk.mark()
        for a, b in evs:
            flush.zero_()
            a.record(stream)
            step()
            b.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        clk.mark()
    prof = mesh.profile_read()
    mesh.profile(False)
    launches_per_step = sum(n for _, n in prof.values()) // max(1, args.steps)
    ms = sum(a.elapsed_time(b) for a, b in evs)
    ms = reduce_max(ms, world, dev)
    barrier(world)
    value = job_throughput(n_active, args.steps, ms, world)
    # dominant kernel roofline (Out elements, live CUDA events on the launching stream)
    k_ms, k_n = prof["out_elements"]
    k_avg = k_ms / max(k_n, 1)
    pk = peaks(api, local)
    flops = FLOPS_JV_OUT_ELEMENT * info["n_out"]
    achieved = flops / (k_avg / 1e3) / 1e12
    roof = {"kernel": "vms_interior (Out elements, J v)", "bound": "alu", "achieved": achieved,
            "peak": pk["fp32_tflops"] if prec == api.PRECISION_MIXED else None, "unit": "TFLOP/s",
            "frac": achieved / pk["fp32_tflops"] if prec == api.PRECISION_MIXED else None,
            "traffic": interior_traffic() if prec == api.PRECISION_MIXED else None,
            "peak_source": pk["fp_source"], "peaks": {k: v for k, v in pk.items() if k.endswith("tflops") or k == "sm_count"},
            "flops_per_element": FLOPS_JV_OUT_ELEMENT, "avg_launch_ms": k_avg,
            "timing": "inside the timed steps, where the Intercepted and surface kernels run beside it on side "
                      "streams and share its SMs"}
    # the same step with every kernel alone (IMGA_OPT_CONCURRENT off), L2 flushed: the per-kernel
    # rooflines, time shares and Eq. Wpart costs, and the dominant kernel's fraction by itself
    mesh.concurrent(False)
    prof_steps = 20
    for _ in range(2):
        step()
    torch.cuda.synchronize()
    mesh.profile(True)
    for _ in range(prof_steps):
        flush.zero_()
        step()
    palone = mesh.profile_read()
    mesh.profile(False)
    mesh.concurrent(True)
    ka = palone["out_elements"][0] / max(palone["out_elements"][1], 1)
    aa = flops / (ka / 1e3) / 1e12
    roof["alone"] = {"avg_launch_ms": ka, "achieved": aa,
                     "frac": aa / pk["fp32_tflops"] if prec == api.PRECISION_MIXED else None,
                     "timing": f"{prof_steps} steps with IMGA_OPT_CONCURRENT off (every kernel by itself), L2 flushed"}
    ex = interior_record().get("executed_fp32_flop_per_out_element")
    if ex and prec == api.PRECISION_MIXED:   # executed flops (ncu counters of this source), kernel alone
        roof["executed"] = {"flops_per_element": ex, "achieved": ex * info["n_out"] / (ka / 1e3) / 1e12,
                            "frac": ex * info["n_out"] / (ka / 1e3) / 1e12 / pk["fp32_tflops"],
                            "source": "profiles/vms_interior_traffic.json (ncu instruction counters)"}
    kern_share = {k: v[0] / max(1e-9, sum(x[0] for x in palone.values())) for k, v in palone.items()}
    kern_roof = kernel_rooflines(palone, prof_steps, info, nn, pk)
    try:
        wpart = wpart_costs(palone, prof_steps, info)
    except Exception as ex:          # reported, never fatal
        wpart = {"error": repr(ex)}
    # end-to-end through the C ABI with host buffers (pinned), copies inside the timed region: every
    # step copies its four input vectors in and its result out; the copies of step i+1's inputs and
    # of step i's result overlap step i's J v (double-buffered device vectors, copy streams).
    hu, hup, hup2, hv = (torch.from_numpy(a).pin_memory() for a in (u, up, up2, v))
    houts = [torch.empty_like(hu).pin_memory() for _ in range(2)]
    dsets = [(ud, upd, up2d, vd, out)] + [tuple(torch.empty_like(ud) for _ in range(5))]
    # one copy stream per input vector (the four copies of a step run side by side) and one out
    s_ins = [torch.cuda.Stream(device=dev) for _ in range(4)]
    s_out = torch.cuda.Stream(device=dev)
    ev = lambda: torch.cuda.Event()
    ev_in, ev_done, ev_read = [[ev() for _ in range(4)] for _ in range(2)], [ev(), ev()], [ev(), ev()]
    e2e_steps = max(2, min(args.steps, 20))
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def h2d(k, dep):
        for j, (dst, src) in enumerate(zip(dsets[k][:4], (hu, hup, hup2, hv))):
            s_ins[j].wait_event(dep)
            with torch.cuda.stream(s_ins[j]):
                dst.copy_(src, non_blocking=True)
                ev_in[k][j].record(s_ins[j])

    def e2e_run():
        torch.cuda.synchronize()
        ea.record(stream)
        h2d(0, ea)
        for i in range(e2e_steps):
            k = i % 2
            du_, dup_, dup2_, dv_, dout_ = dsets[k]
            for e_ in ev_in[k]:
                stream.wait_event(e_)
            if i >= 2:
                stream.wait_event(ev_read[k])          # the result copy of step i-2 has left this buffer
            mesh.jvp(ph, du_, dup_, dv_, dup2_, precision=prec, out=dout_, stream=stream)
            ev_done[k].record(stream)
            if i + 1 < e2e_steps:
                h2d(1 - k, ev_done[1 - k] if i >= 1 else ea)   # step i-1 no longer reads that set
            with torch.cuda.stream(s_out):
                s_out.wait_event(ev_done[k])
                houts[k].copy_(dout_, non_blocking=True)
                ev_read[k].record(s_out)
        stream.wait_event(ev_read[(e2e_steps - 1) % 2])
        stream.wait_event(ev_read[e2e_steps % 2])
        eb.record(stream)
        torch.cuda.synchronize()
        return ea.elapsed_time(eb)

    # three runs of e2e_steps steps (the host-memory link is shared): the median counts
    runs = sorted(e2e_run() for _ in range(3))
    # the host link alone, for context: the four input copies side by side, then the result copy
    la, lb, lc = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    torch.cuda.synchronize()
    la.record(stream)
    h2d(0, la)
    for e_ in ev_in[0]:
        stream.wait_event(e_)
    lb.record(stream)
    houts[0].copy_(out, non_blocking=True)
    lc.record(stream)
    torch.cuda.synchronize()
    host_link = {"h2d_gbs": 4 * hu.numel() * 8 / (la.elapsed_time(lb) / 1e3) / 1e9,
                 "d2h_gbs": houts[0].numel() * 8 / (lb.elapsed_time(lc) / 1e3) / 1e9}
    e2e_ms = reduce_max(runs[1], world, dev)
    e2e = {"value": world * n_active * e2e_steps / (e2e_ms / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": 4 * hu.numel() * 8, "d2h_bytes_per_step": houts[0].numel() * 8,
           "pipelined": "copies of step i+1 in and step i out overlap step i's J v (2 buffer sets, 4 input copy streams, 1 output)",
           "host_link": host_link,
           "runs_ms": runs, "steps_per_run": e2e_steps}
    ref = out.cpu().numpy()   # the same J v (float64 atomics: the sum order may differ)
    ok = np.allclose(houts[(e2e_steps - 1) % 2].numpy(), ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max())
    e2e["result_matches_device_path"] = bool(ok)
    # companion numbers (not the headline): FP64 J v, residuals
    extra = {}
    for name, fn in (("jv_fp64", lambda: mesh.jvp(ph, ud, upd, vd, up2d, precision=0, out=out, stream=stream)),
                     ("residual_mixed", lambda: mesh.residual(ph, ud, upd, up2d, precision=1, out=out, stream=stream)),
                     ("residual_fp64", lambda: mesh.residual(ph, ud, upd, up2d, precision=0, out=out, stream=stream))):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 3
        tot = 0.0
        for _ in range(reps):
            flush.zero_()
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            tot += a.elapsed_time(b)
        extra[name] = n_active * reps / (tot / 1e3)
    # the float64 Out-element kernel against the float64 pipe (GB300 nominal 1.25 TFLOP/s dense FP64)
    mesh.profile(True)
    for _ in range(3):
        mesh.jvp(ph, ud, upd, vd, up2d, precision=0, out=out, stream=stream)
    p64 = mesh.profile_read()
    mesh.profile(False)
    k64 = p64["out_elements"][0] / max(1, p64["out_elements"][1])
    a64 = FLOPS_JV_OUT_ELEMENT * info["n_out"] / (k64 / 1e3) / 1e12
    extra_roof = {"kernel": "vms_interior<double, J v>", "bound": "fp64 pipe", "avg_launch_ms": k64, "achieved": a64,
                  "peak": pk["fp64_tflops"], "unit": "TFLOP/s", "frac": a64 / pk["fp64_tflops"],
                  "peak_source": pk["fp_source"],
                  "note": "achieved counts the nodal-form 12,464 flop per element; the monomial form executes fewer"}
    ex64 = interior_record().get("executed_fp64_flop_per_out_element")
    if ex64:
        e64 = ex64 * info["n_out"] / (k64 / 1e3) / 1e12
        extra_roof["executed"] = {"flops_per_element": ex64, "achieved": e64, "frac": e64 / pk["fp64_tflops"],
                                  "source": "profiles/vms_interior_traffic.json (ncu instruction counters)"}
    # J v replayed as a CUDA graph (parallel branches for the Out / Intercepted / surface kernels)
    mesh.use_graphs(True)
    step()
    torch.cuda.synchronize()
    gms = 0.0
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(20):
        flush.zero_()
        a.record(stream)
        step()
        b.record(stream)
        torch.cuda.synchronize()
        gms += a.elapsed_time(b)
    extra["jv_mixed_graph"] = n_active * 20 / (gms / 1e3)
    mesh.use_graphs(False)
    extra["fused"] = run_fused(mesh, step, flush, stream, n_active)
    extra["scatter"] = run_scatter_modes(mesh, step, flush, stream, n_active)
    batched = run_batched(args, dev, stream) if not args.no_batched else None
    bluff = run_bluff(args, dev, stream) if not args.no_bluff else None

    # Newton-GMRES step to 1e-8 (float64 residual), block-Jacobi, J v in FP64 vs mixed precision, on the
    # small-sphere problem (7,288 elements: the size the learned preconditioner is evaluated at).  On the
    # 2M-element sphere LES nodal block-Jacobi does not bring GMRES(50) to 1e-8: after the first Newton
    # step every linear solve reaches its cap, held back by global pressure coupling.
    newton = {}
    if not args.no_newton:
        ws = I.small_sphere(0)
        smesh = api.Mesh.from_workload(ws, device=local)
        su, sup, _ = I.state(smesh.n_nodes, 16 + rank)
        sud, supd = torch.from_numpy(su).to(dev), torch.from_numpy(sup).to(dev)
        for name, p, gr, pc in (("mixed", api.PRECISION_MIXED, False, 1), ("fp64", api.PRECISION_FP64, False, 1),
                                ("mixed_graphs", api.PRECISION_MIXED, True, 1),
                                ("mixed_graphs_multilevel", api.PRECISION_MIXED, True, 4),
                                ("fp64_graphs_multilevel", api.PRECISION_FP64, True, 4)):
            smesh.use_graphs(gr)
            runs = []
            for rep in range(2):   # the first run also allocates the Krylov workspace
                uw = sud.clone()
                torch.cuda.synchronize()
                st = smesh.newton_step(ws.physics, uw, supd, precision=p, precond=pc, rtol=1e-8, gmres_m=50,
                                    krylov_rtol=args.krylov_rtol, max_newton=20, max_krylov=500, stream=stream,
                                    raise_on_failure=False)
                runs.append(st)
            st = runs[-1]
            newton[name] = {"ms": st["time_ms"], "newton_its": st["newton_its"], "krylov_its": st["krylov_its"],
                            "converged": bool(st["converged"]), "rel_residual": st["res_norm"][-1] / st["res_norm"][0],
                            "workload": "small_sphere (7,288 elements, Re 10, BE dt 0.01), "
                                        + ("multilevel V-cycle" if pc == 4 else "block-Jacobi") + ", GMRES(50)"}
        smesh.close()
        # the sphere LES itself: block-Jacobi GMRES(50) stalls on it (every linear solve after the first
        # reaches its cap); the multilevel V-cycle (precond 4) solves its linear systems.  Mixed: float32
        # elements, hierarchy and V-cycle, float64 Krylov vectors, reductions and update; fp64: everything
        # float64.  (a) One Newton step whose GMRES(50) solve reaches 1e-8 relative, mixed against fp64,
        # and the error of the mixed step against the fp64 one.  (b) The nonlinear solve toward 1e-8
        # (mixed, two smoothing sweeps): at Re 1e4 Newton converges only linearly on this residual.
        mesh.use_graphs(True)
        sol = {}
        for name, p in (("mixed", api.PRECISION_MIXED), ("fp64", api.PRECISION_FP64)):
            uw = ud.clone()
            torch.cuda.synchronize()
            st = mesh.newton_step(ph, uw, upd, up2d, precision=p, precond=4, rtol=1e-8, gmres_m=50,
                                  krylov_rtol=1e-8, max_newton=1, max_krylov=2000, stream=stream,
                                  raise_on_failure=False)
            sol[name] = uw
            r = st["res_norm"]
            newton["sphere_les_step_" + name] = {
                "ms": st["time_ms"], "krylov_its": st["krylov_its"], "linear_rel_residual": st["krylov_rel"][0],
                "linear_converged": bool(st["krylov_rel"][0] <= 1e-8 * 1.0000001),
                "nonlinear_rel_residual_after": r[-1] / r[0],
                "workload": "sphere_les (2,001,176 elements, Re 1e4, BDF2 dt 0.01): one Newton step, GMRES(50) to "
                            "1e-8 relative, multilevel V-cycle (6 Morton-consecutive blocks per aggregate, damped "
                            "block-Jacobi 0.5), whole solve as one CUDA graph"}
        d = (sol["mixed"] - sol["fp64"]).norm().item() / max((sol["fp64"] - ud).norm().item(), 1e-300)
        newton["sphere_les_step_mixed"]["rel_error_of_update_vs_fp64"] = d
        uw = ud.clone()
        st = mesh.newton_step(ph, uw, upd, up2d, precision=api.PRECISION_MIXED, precond=4, rtol=1e-8, gmres_m=50,
                              krylov_rtol=args.krylov_rtol, max_newton=20, max_krylov=600, ml_sweeps=2,
                              stream=stream, raise_on_failure=False)
        r = st["res_norm"]
        newton["sphere_les_solve_mixed"] = {
            "ms": st["time_ms"], "ms_per_newton": st["time_ms"] / max(1, st["newton_its"]),
            "newton_its": st["newton_its"], "krylov_its": st["krylov_its"],
            "krylov_per_newton": st["krylov_per_newton"], "rel_residual_history": [x / r[0] for x in r],
            "converged": bool(st["converged"]),
            "workload": "sphere_les, Newton toward 1e-8 with GMRES(50) to 1e-3 per step, multilevel V-cycle with "
                        "two sweeps, at most 20 Newton iterations"}
        rows, _ = mesh.multilevel_info()
        newton["sphere_les_multilevel_levels"] = [int(x) for x in rows]
        mesh.use_graphs(False)
    learned = run_learned(args, dev, stream, mesh, w) if not args.no_learned and rank == 0 else None
    try:
        inout = run_inout(mesh, w, dev, stream)
    except Exception as ex:          # reported in the JSON line instead of ending the run
        inout = {"error": repr(ex)}
    if not args.no_inout_table and rank == 0:
        try:
            inout["table_in_out"] = run_inout_table(dev, stream)
        except Exception as ex:
            inout["table_in_out"] = {"error": repr(ex)}
    # CPU baseline: the oracle on a bounded sample (rank 0, one GPU only)
    cpu, parity = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            om, ou, oup, ov = oracle_sample(w, 0)
            sel = np.unique(I.splitmix64(77, args.sample_nodes) % om.n_nodes).astype(np.int64)
            ne, dt, Ro, Jo = time_oracle(om, w, ou, oup, ov, sel, rows=True)
            parity = parity_on_sample(mesh, ph, ud, upd, up2d, vd, sel, Ro, Jo)
            cores = os.cpu_count() or 1
            ne_c, dt_c = time_oracle(om, w, ou, oup, ov, sel, threads=cores)
            cpu = {"value": ne_c / dt_c, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": f"residual + J v of the {ne_c} active elements touching {args.sample_nodes} seeded nodes "
                             f"of the same mesh, element loop on {cores} threads (os.cpu_count()) ({dt_c:.1f} s)",
                   "single_core": {"value": ne / dt, "cores": 1, "seconds": dt}}
        except Exception as ex:  # report, never hide
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {ex}"}
    clocks = clk.summary()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32" if prec == 1 else "f64", "data": "synthetic",
                "config": {"workload": "sphere_les (box 32x16x16 D, sphere D=1, levels 4-10 + wake cone, Re 1e4, BDF2)",
                           "elements": info["n_elem"], "active_elements": n_active, "out_elements": info["n_out"],
                           "cut_elements": info["n_cut"], "cut_points": info["n_cut_points"],
                           "surface_points": info["n_surface_points"], "nodes": nn,
                           "precision": "mixed: f32 element arithmetic, f64 node differences, scatter and reductions"
                           if prec == 1 else "fp64",
                           "l2": "flushed between timed steps (256 MiB write)", "parallelism": f"replicas x{world}"},
                "roofline": roof, "kernel_roofline": kern_roof, "fp64_roofline": extra_roof,
                "kernel_time_share": kern_share, "wpart": wpart,
                "cut_tile": dict(zip(("warps_per_block", "longest_first", "candidate_ms"), mesh.tuning()[(prec, "jvp")])),
                "out_tile": dict(zip(("blocks_per_sm", "candidate_ms"), mesh.tuning_interior()[(prec, "jvp")])),
                "clocks": clocks, "e2e": e2e,
                "gpu_launches": launches_per_step * args.steps, "cpu_baseline": cpu, "parity_vs_oracle": parity,
                "extra_elements_per_s": extra,
                "newton_step": newton, "learned_preconditioner": learned, "inout": inout, "batched": batched, "bluff_pair": bluff, "setup_s": build_s, "setup_ms": info["setup_ms"], "wall_s_timed": wall}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_fused(mesh, step, flush, stream, n_active, reps=20):
    """The same J v with the buckets in one persistent launch (IMGA_OPT_FUSED), direct and as a CUDA
    graph, L2 flushed between steps; the fused kernel's own time from events around it."""
    import torch

    res = {}
    mesh.fused(True)
    try:
        res["queue"] = mesh.fused_info()
        # warps per block that start on the costly items: keep the fastest
        split = {}
        for hw in (4, 2, 1):
            mesh.fused_split(hw)
            step()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            tot = 0.0
            for _ in range(reps):
                flush.zero_()
                a.record(stream)
                step()
                b.record(stream)
                torch.cuda.synchronize()
                tot += a.elapsed_time(b)
            split[hw] = tot / reps
        best = min(split, key=split.get)
        mesh.fused_split(best)
        res["split_ms_per_jv"] = {str(k): v for k, v in split.items()}
        res["heavy_first_warps"] = best
        for graphs in (False, True):
            mesh.use_graphs(graphs)
            step()
            torch.cuda.synchronize()
            tot = 0.0
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            for _ in range(reps):
                flush.zero_()
                a.record(stream)
                step()
                b.record(stream)
                torch.cuda.synchronize()
                tot += a.elapsed_time(b)
            res["graph" if graphs else "direct"] = {"ms_per_jv": tot / reps, "elements_per_s": n_active * reps / (tot / 1e3)}
        mesh.use_graphs(False)
        mesh.profile(True)
        for _ in range(reps):
            flush.zero_()
            step()
        prof = mesh.profile_read()
        mesh.profile(False)
        res["kernel_ms"] = {k: v[0] / max(1, v[1]) for k, v in prof.items() if v[1]}
    finally:
        mesh.use_graphs(False)
        mesh.fused_split(4)
        mesh.fused(False)
    return res


def run_scatter_modes(mesh, step, flush, stream, n_active, reps=20):
    """J v with the deterministic scatter (slots + ordered node sums, the default) against float64
    atomic additions (IMGA_OPT_DETERMINISTIC off), L2 flushed between steps, with per-kernel times."""
    import torch

    res = {}
    try:
        for det in (True, False):
            mesh.deterministic(det)
            step()
            torch.cuda.synchronize()
            mesh.profile(True)
            tot = 0.0
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            for _ in range(reps):
                flush.zero_()
                a.record(stream)
                step()
                b.record(stream)
                torch.cuda.synchronize()
                tot += a.elapsed_time(b)
            prof = mesh.profile_read()
            mesh.profile(False)
            res["deterministic" if det else "atomic"] = {
                "ms_per_jv": tot / reps, "elements_per_s": n_active * reps / (tot / 1e3),
                "kernel_ms": {k: v[0] / max(1, v[1]) for k, v in prof.items() if v[1]}}
    finally:
        mesh.deterministic(True)
    return res


def run_batched_newton(B, sep, probs, states, dev, max_newton=4, max_krylov=600):
    """One Newton solve of all 64 problems through the batched mesh (one GMRES on the block-diagonal
    system, the whole solve replayed as one CUDA graph) against 64 solves one mesh after the other
    (each also one graph).  Mixed precision, block-Jacobi, GMRES(50); capped at max_newton Newton and
    max_krylov Krylov iterations per solve, since block-Jacobi does not bring every high-Reynolds
    problem to 1e-8: the reductions reached are reported beside the times."""
    import torch

    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    kw = dict(precision=1, precond=1, rtol=1e-8, gmres_m=50, max_newton=max_newton, max_krylov=max_krylov,
              raise_on_failure=False)
    u0 = np.concatenate([s[0] for s in states])
    up = T(np.concatenate([s[1] for s in states]))
    out = {"max_newton": max_newton, "max_krylov": max_krylov}
    B.use_graphs(True)
    try:
        B.newton_step(probs[0].physics, T(u0), up, **kw)   # capture
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = B.newton_step(probs[0].physics, T(u0), up, **kw)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out["one_batched_graph"] = {"s": dt, "newton_its": st["newton_its"],
                                    "krylov_its": st["krylov_its"], "converged": bool(st["converged"]),
                                    "rel_res": st["res_norm"][-1] / max(st["res_norm"][0], 1e-300),
                                    "problem_krylov_its_per_s": len(sep) * st["krylov_its"] / dt}
    finally:
        B.use_graphs(False)
    rels, conv, kits = [], 0, 0
    for m in sep:
        m.use_graphs(True)
    try:
        ups = [T(s[1]) for s in states]
        for m, w, s, u in zip(sep, probs, states, ups):   # capture
            m.newton_step(w.physics, T(s[0]), u, **kw)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for m, w, s, u in zip(sep, probs, states, ups):
            st = m.newton_step(w.physics, T(s[0]), u, **kw)
            rels.append(st["res_norm"][-1] / max(st["res_norm"][0], 1e-300))
            conv += bool(st["converged"])
            kits += st["krylov_its"]
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out["sequential_64_graphs"] = {"s": dt, "converged": conv, "krylov_its": kits,
                                       "rel_res_max": max(rels), "rel_res_median": float(np.median(rels)),
                                       "problem_krylov_its_per_s": kits / dt}
    finally:
        for m in sep:
            m.use_graphs(False)
    return out


def run_batched(args, dev, stream):
    """64 independent sphere problems (5k-200k elements, Re 1-1e6): J v of all of them through one
    batched mesh (one launch of each kernel) vs 64 meshes called one after the other."""
    import torch

    from paper_2009_00706_gb300 import api
    probs = [wl for wl, _, _ in I.batched_spheres(64)]
    t0 = time.perf_counter()
    B = api.Mesh.batch(probs, device=dev.index)
    tb = time.perf_counter() - t0
    sep = [api.Mesh.from_workload(w, device=dev.index) for w in probs]
    n_act = B.info["n_out"] + B.info["n_cut"]
    states = [I.state(m.n_nodes, 100 + k) for k, m in enumerate(sep)]
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    ub, upb, vb = (T(np.concatenate([s[i] for s in states])) for i in range(3))
    outb = torch.empty_like(ub)
    per = [(T(s[0]), T(s[1]), T(s[2]), torch.empty_like(T(s[0]))) for s in states]
    ph = probs[0].physics
    prec = api.PRECISION_MIXED

    def batched_step():
        B.jvp(ph, ub, upb, vb, precision=prec, out=outb, stream=stream)

    def sequential_step():
        for m, w, (u, up, v, o) in zip(sep, probs, per):
            m.jvp(w.physics, u, up, v, precision=prec, out=o, stream=stream)

    res = {"problems": 64, "elements": int(B.n_elem), "active_elements": int(n_act), "batch_build_s": tb}
    B.autotune(True)
    for m in sep:
        m.autotune(True)
    for name, fn in (("one_batched_launch", batched_step), ("sequential_64_meshes", sequential_step)):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(10):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / 10
        res[name] = {"ms_per_jv": ms, "elements_per_s": n_act / (ms / 1e3)}
    res["cut_tile"] = dict(zip(("warps_per_block", "longest_first", "candidate_ms"), B.tuning()[(prec, "jvp")]))
    B.use_graphs(True)
    batched_step()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(10):
        batched_step()
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / 10
    res["one_batched_graph"] = {"ms_per_jv": ms, "elements_per_s": n_act / (ms / 1e3)}
    B.use_graphs(False)
    # the buckets of all 64 problems in one persistent launch
    B.fused(True)
    for graphs in (False, True):
        B.use_graphs(graphs)
        batched_step()
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(10):
            batched_step()
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / 10
        res["one_fused_graph" if graphs else "one_fused_launch"] = {"ms_per_jv": ms, "elements_per_s": n_act / (ms / 1e3)}
    B.use_graphs(False)
    B.fused(False)
    res["newton"] = run_batched_newton(B, sep, probs, states, dev)
    for m in sep:
        m.close()
    B.close()
    return res


def run_bluff(args, dev, stream):
    """Bluff-body pair (19.8 M elements, 397,488 triangles, Re 1e6, BDF2): mixed J v and residual,
    direct and as a CUDA graph, with the per-kernel time shares."""
    import torch

    from paper_2009_00706_gb300 import api
    w = I.bluff_pair(0)
    t0 = time.perf_counter()
    m = api.Mesh.from_workload(w, device=dev.index)
    build_s = time.perf_counter() - t0
    info = m.info
    n_act = info["n_out"] + info["n_cut"]
    u, up, v = I.state(m.n_nodes, 0)
    ud, upd, vd = (torch.from_numpy(a).to(dev) for a in (u, up, v))
    out = torch.empty_like(ud)
    ph = w.physics
    prec = api.PRECISION_MIXED
    res = {"workload": "bluff_pair (two trucks, 16L x 2L x 2L, levels 5-11, Re 1e6, BDF2)", "elements": info["n_elem"],
           "active_elements": n_act, "cut_elements": info["n_cut"], "cut_points": info["n_cut_points"],
           "surface_points": info["n_surface_points"], "triangles": info["n_tri"], "build_s": build_s}

    def timed(fn, n=10):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(n):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / n

    jv = lambda: m.jvp(ph, ud, upd, vd, upd, precision=prec, out=out, stream=stream)
    m.autotune(True)
    ms = timed(jv)
    res["jv_mixed"] = {"ms": ms, "elements_per_s": n_act / (ms / 1e3)}
    ms = timed(lambda: m.residual(ph, ud, upd, upd, precision=prec, out=out, stream=stream))
    res["residual_mixed"] = {"ms": ms, "elements_per_s": n_act / (ms / 1e3)}
    # time shares with every kernel by itself (on side streams their event spans overlap)
    m.concurrent(False)
    jv()
    m.profile(True)
    for _ in range(3):
        jv()
    prof = m.profile_read()
    m.profile(False)
    m.concurrent(True)
    tot = sum(x[0] for x in prof.values())
    res["jv_kernel_time_share"] = {k: x[0] / max(tot, 1e-9) for k, x in prof.items() if x[1]}
    res["jv_kernel_ms_alone"] = {k: x[0] / 3 for k, x in prof.items() if x[1]}
    m.use_graphs(True)
    ms = timed(jv)
    res["jv_mixed_graph"] = {"ms": ms, "elements_per_s": n_act / (ms / 1e3)}
    m.close()
    return res


def run_inout(mesh, w, dev, stream):
    """In/out classification (imga_classify) on the sphere LES: 5^3 points per Intercepted element
    (a regular grid inside the element: the normal test decides most, the rest cast warp-cooperative
    rays against 81,920 triangles), and points uniform over the box (most lie in elements without
    background triangles and take the stored marker).  As in the paper's Table in-out: P_s, the
    fraction of the normal-tested points that the normal test decides, and the time of the same
    points when every one of them is classified by ray parity."""
    import torch

    ex = mesh.export()
    mk, _ = mesh.markers()
    cut = np.where(mk == 2)[0]
    h = (2.0 ** (-ex["levels"][cut].astype(np.float64))) * max(np.subtract(w.hi, w.lo))
    x0 = np.asarray(w.lo)[None, :] + ex["anchors"][cut].astype(np.float64) * (max(np.subtract(w.hi, w.lo)) / 2.0 ** 20)
    t = (np.arange(5) + 0.5) / 5.0
    g = np.stack(np.meshgrid(t, t, t, indexing="ij"), -1).reshape(-1, 3)
    near = (x0[:, None, :] + h[:, None, None] * g[None, :, :]).reshape(-1, 3)
    uni = np.asarray(w.lo) + I.uniform(41, 3 * near.shape[0]).reshape(-1, 3) * np.subtract(w.hi, w.lo)

    def timed(P, flags, reps=3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            mesh.classify(P, flags=flags, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    out = {}
    for name, pts in (("near_surface_5x5x5_per_cut_element", near), ("uniform_in_box", uni)):
        P = torch.from_numpy(np.ascontiguousarray(pts)).to(dev)
        flags = mesh.classify(P, stream=stream)
        torch.cuda.synchronize()
        ms = timed(P, flags)
        mesh.classify_counts(reset=True)
        mesh.classify(P, flags=flags, stream=stream)
        cnt = mesh.classify_counts(reset=True)
        mesh.classify_rays_only(True)
        try:
            flags_r = mesh.classify(P, stream=stream)
            torch.cuda.synchronize()
            ms_r = timed(P, flags_r)
            differing = int((flags_r != flags).sum().item())
        finally:
            mesh.classify_rays_only(False)
            mesh.classify_counts(reset=True)
        p_s = cnt["normal_decided"] / cnt["normal_tests"] if cnt["normal_tests"] else None
        out[name] = {"points": int(P.shape[0]), "ms": ms, "points_per_s": P.shape[0] / (ms / 1e3),
                     "fraction_in": float(flags.float().mean().item()), "counts": cnt,
                     "P_s": p_s, "P_f": None if p_s is None else 1.0 - p_s,
                     "ray_only": {"ms": ms_r, "points_per_s": P.shape[0] / (ms_r / 1e3), "flags_differing": differing},
                     "speedup_vs_ray_only": ms_r / ms}
    return out


def run_inout_table(dev, stream, levels=(6, 7, 8)):
    """The analogue of Table in-out: a truck (two filleted boxes) in uniform 64^3, 128^3 and 256^3
    grids, 5^3 Gauss-Legendre points per Intercepted element, classified by the normal test with
    ray fallback and, for comparison, every point by ray parity.  Per grid: P_s (points the normal
    test decides, of all the points), both times, the time per point and the speed-up."""
    import gc

    import torch

    from paper_2009_00706_gb300 import api
    xi = np.polynomial.legendre.leggauss(5)[0]
    g = np.stack(np.meshgrid(xi, xi, xi, indexing="ij"), -1).reshape(-1, 3)
    rows = []
    for lev in levels:
        w = I.inout_truck(lev)
        m = api.Mesh.from_workload(w, device=dev.index)
        ex = m.export()
        mk, _ = m.markers()
        cut = np.where(mk == 2)[0]
        h = (w.hi[0] - w.lo[0]) / 2.0 ** lev
        x0 = np.asarray(w.lo)[None, :] + ex["anchors"][cut].astype(np.float64) * ((w.hi[0] - w.lo[0]) / 2.0 ** 20)
        pts = (x0[:, None, :] + 0.5 * h * (g[None, :, :] + 1.0)).reshape(-1, 3)
        P = torch.from_numpy(np.ascontiguousarray(pts)).to(dev)
        res = {}
        for mode in ("normal_then_ray", "ray_only"):
            m.classify_rays_only(mode == "ray_only")
            flags = m.classify(P, stream=stream)
            torch.cuda.synchronize()
            m.classify_counts(reset=True)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            m.classify(P, flags=flags, stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            res[mode] = (a.elapsed_time(b), m.classify_counts(reset=True), flags)
        m.classify_rays_only(False)
        (ms, cnt, f), (ms_r, cnt_r, f_r) = res["normal_then_ray"], res["ray_only"]
        n = int(P.shape[0])
        rows.append({"grid": "%d^3" % (1 << lev), "elements": m.n_elem, "cut_elements": int(cut.size),
                     "points": n, "triangles": int(m.info["n_tri"]),
                     "P_s": cnt["normal_decided"] / max(1, cnt["normal_tests"]),
                     "P_f": cnt["rays"] / max(1, cnt["normal_tests"]), "counts": cnt,
                     "ms": ms, "ns_per_point": 1e6 * ms / n, "ray_only_ms": ms_r, "ray_only_ns_per_point": 1e6 * ms_r / n,
                     "speedup_vs_ray_only": ms_r / ms, "flags_differing_from_ray_only": int((f != f_r).sum().item()),
                     "fraction_in": float(f.float().mean().item())})
        del m, P, res, f, f_r
        gc.collect()
        torch.cuda.empty_cache()
    return {"workload": "truck (cab + trailer, 24,576 triangles) in a 6.4 cube, uniform grids, 5^3 "
                        "Gauss-Legendre points per Intercepted element", "grids": rows}


def run_learned(args, dev, stream, les, w_les):
    """Learned block preconditioner, config 5: the network is trained by the library's kernels on
    element Jacobian blocks of small-sphere problems with geometry seeds 0-15 (the sphere's jitter and
    the state follow the seed; all active elements) and of the sphere LES (50,000 sampled active
    elements, every Intercepted one kept), then evaluated in Newton-GMRES(50) on the 16 held-out
    geometries 16-31 against block-Jacobi and no preconditioner (and, for context, the multilevel
    V-cycle); the float64 residual decides convergence."""
    import torch

    from paper_2009_00706_gb300 import api
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    t0 = time.perf_counter()
    Xs, Ts = [], []
    for seed in range(16):
        ws = I.small_sphere(seed)
        sm = api.Mesh.from_workload(ws, device=dev.index)
        mk, _ = sm.markers()
        elems = T(np.where(mk != 1)[0].astype(np.int32))
        u, up, _ = I.state(sm.n_nodes, seed)
        X, Tt, _ = sm.precond_dataset(ws.physics, T(u), T(up), elems)
        Xs.append(X)
        Ts.append(Tt)
        sm.close()
    lmk, _ = les.markers()
    cut, out_ = np.where(lmk == 2)[0], np.where(lmk == 0)[0]
    pick = np.unique(np.concatenate([cut, out_[I.splitmix64(31, 50000 - cut.size) % out_.size]])).astype(np.int32)
    u, up, _ = I.state(les.n_nodes, 0)
    X, Tt, _ = les.precond_dataset(w_les.physics, T(u), T(up), T(pick), u_prev2=T(up))
    Xs.append(X)
    Ts.append(Tt)
    X, Tt = torch.cat(Xs), torch.cat(Ts)
    del Xs, Ts
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    net = api.Mlp(seed=11, device=dev.index)
    t0 = time.perf_counter()
    hist = net.train(X, Tt, epochs=20, batch=1024, lr=1e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    n_train = int(X.shape[0])
    del X, Tt
    res = {}
    for seed in range(16, 32):
        ws = I.small_sphere(seed)
        sm = api.Mesh.from_workload(ws, device=dev.index)
        sm.use_graphs(True)
        u, up, _ = I.state(sm.n_nodes, seed)
        for name, kw in (("block_jacobi", dict(precond=1)), ("learned", dict(precond=2, learned=net, learned_omega=0.5)),
                         ("none", dict(precond=0, max_newton=10)), ("multilevel", dict(precond=4))):
            ud = T(u)
            st = sm.newton_step(ws.physics, ud, T(up), precision=api.PRECISION_MIXED, rtol=1e-8, gmres_m=50,
                                max_krylov=1000, raise_on_failure=False, **kw)
            res.setdefault(name, []).append({"ms": st["time_ms"], "newton_its": st["newton_its"],
                                             "krylov_its": st["krylov_its"], "fallbacks": st.get("fallbacks"),
                                             "converged": bool(st["converged"])})
        sm.close()
    summary = {k: {"krylov_its_median": float(np.median([r["krylov_its"] for r in v])),
                   "ms_median": float(np.median([r["ms"] for r in v])),
                   "converged": sum(r["converged"] for r in v), "problems": len(v)} for k, v in res.items()}
    net.close()
    return {"train_samples": n_train, "dataset_s": t_data, "train_s": t_train, "epochs": 20,
            "train_geometry_seeds": "0-15 (+ sphere LES sample)", "eval_geometry_seeds": "16-31",
            "loss_first_last": [float(hist[0]), float(hist[-1])],
            "precision": "mixed J v, float64 residual, graph-replayed GMRES(50)", "summary": summary, "results": res}


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--sample-nodes", type=int, default=60000)
    ap.add_argument("--ref-sample-nodes", type=int, default=20000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-inout-table", action="store_true", help="skip the 64^3-256^3 in/out comparison")
    ap.add_argument("--no-newton", action="store_true", help="skip the Newton-GMRES step timing")
    ap.add_argument("--no-batched", action="store_true", help="skip the 64-problem batched measurement")
    ap.add_argument("--no-bluff", action="store_true", help="skip the 19.8 M-element bluff-body pair measurement")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-preconditioner training and evaluation")
    ap.add_argument("--krylov-rtol", type=float, default=1e-3)
    ap.add_argument("--newton-profile", action="store_true",
                    help="only one config-2 Newton step (for ncu launch lists of the solver)")
    ap.add_argument("--kernel-profile", action="store_true",
                    help="only a few J v calls on the sphere LES (for ncu counter captures)")
    return ap.parse_args(argv)


def run_kernel_profile(args):
    """A short fixed sequence for counter captures (ncu): the sphere-LES mesh, untuned launch shapes,
    mixed-precision J v calls -- bucketed, fused (IMGA_OPT_FUSED), bucketed, bucketed -- then one
    float64 J v call, no other work.  Prints the per-call milliseconds (not a bench value)."""
    import torch

    from paper_2009_00706_gb300 import _lib, api
    _lib.build()
    dev = torch.device("cuda", 0)
    w = I.sphere_les(0)
    mesh = api.Mesh.from_workload(w, device=0)
    u, up, v = I.state(mesh.n_nodes, 0)
    ud, upd, vd = (torch.from_numpy(a).to(dev) for a in (u, up, v))
    out = torch.empty_like(ud)
    st = torch.cuda.current_stream()
    ms = []
    for prec, fused in ((1, False), (1, True), (1, False), (1, False), (0, False)):
        mesh.fused(fused)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        mesh.jvp(w.physics, ud, upd, vd, upd, precision=prec, out=out, stream=st)
        b.record(st)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    mesh.fused(False)
    print(json.dumps({"kernel_profile": "sphere_les J v: mixed, mixed fused, mixed x2, float64", "ms": ms,
                      "out_elements": mesh.info["n_out"]}))
    mesh.close()
    return 0


def run_newton_profile(args):
    """One config-2 Newton step (sphere LES, mixed precision, multilevel V-cycle, GMRES(50) to 1e-8),
    host-driven (a profiler sees every kernel as its own launch), then the same step as one CUDA
    graph; nothing else: for kernel launch lists and timings of the solver."""
    import torch

    from paper_2009_00706_gb300 import _lib, api
    _lib.build()
    dev = torch.device("cuda", 0)
    w = I.sphere_les(0)
    mesh = api.Mesh.from_workload(w, device=0)
    u, up, _ = I.state(mesh.n_nodes, 0)
    ud, upd = (torch.from_numpy(a).to(dev) for a in (u, up))
    stream = torch.cuda.current_stream()
    res = {}
    for graphs in (False, True):   # host-driven first (a profiler sees its kernels), then one graph
        mesh.use_graphs(graphs)
        uw = ud.clone()
        st = mesh.newton_step(w.physics, uw, upd, upd.clone(), precision=api.PRECISION_MIXED, precond=4, rtol=1e-8,
                              gmres_m=50, krylov_rtol=1e-8, max_newton=1, max_krylov=2000, stream=stream,
                              raise_on_failure=False)
        res["graph" if graphs else "host_driven"] = {"ms": st["time_ms"], "krylov_its": st["krylov_its"],
                                                      "linear_rel": st["krylov_rel"][0]}
    mesh.use_graphs(False)
    print(json.dumps({"newton_profile": "sphere_les, one Newton step, mixed, multilevel", **res}))
    mesh.close()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.kernel_profile:
        return run_kernel_profile(args)
    if args.newton_profile:
        return run_newton_profile(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
