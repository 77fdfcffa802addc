"""i-NOLF rendering throughput on one GB300 (Mrays/s at 4K).

Workload (default): the full synthetic object -- displaced geodesic sphere,
200 000 triangles, 16 PSH levels N = 16..2048 (band 2 cells), F = 2 FP32
features, MLP 48-64-64-4 -- rendered from 64 ring viewpoints at distance 2.5,
3840x2160 each: one step = one inolf_render call over all 64 views
(530.8 M primary rays).  Inputs (object tables, cameras) are resident in HBM
before the timed region; the RGBA output (8.5 GB) is larger than L2, and L2
is flushed between timed steps as well.

`value` is device-timed Mrays/s of the FP32 path; `e2e` is the same metric
through the C ABI with host buffers (cameras host->device and the full RGBA
frame device->host inside the timed region).  Precision variants (BF16/FP8
MLP on the tensor cores) are reported under `precisions` where built.

`--impl reference` times the FP64 CPU oracle (the only reference this
project has) on a bounded pixel sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

W4K, H4K, N_VIEWS, RING_R = 3840, 2160, 64, 2.5
SLOT_SLACK = 1.25


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--small", action="store_true", help="tiny scene, 1 view at 512x512 (profiling)")
    ap.add_argument("--views", type=int, default=N_VIEWS)
    ap.add_argument("--levels", type=int, default=16,
                    help="PSH levels of the full scene (N = 16 .. 16 * 2^(levels-1), at most 2048); the proxy "
                         "mesh is the same at any count, so a small count keeps a trace profile's footprint small")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precisions", default="fp32,bf16,fp8")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serving-seconds", type=float, default=10.0)
    ap.add_argument("--no-variant", action="store_true", help="skip the density-cube variant workload")
    ap.add_argument("--training-only", action="store_true",
                    help="run only the differentiation workload and print its JSON (profiling)")
    ap.add_argument("--serving-only", action="store_true",
                    help="run only the serving workload (policy 1) and print its JSON (profiling)")
    ap.add_argument("--variant-only", action="store_true",
                    help="run only the density-cube variant workload (--views, --steps, --warmup, --precisions) "
                         "and print its JSON (profiling)")
    return ap.parse_args()


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist_init(n_gpus):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    return rank, world, local


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(x, world, device="cuda"):
    """Slowest rank's time (timing plumbing only: the replicas exchange no data)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank, seconds_max, world):
    """Whole-job throughput of N independent replicas (weak scaling): all
    ranks' units over the slowest rank's time."""
    return units_per_rank * world / seconds_max


def make_workload(small: bool, views: int, levels: int = 16):
    from paper_2303_04086_gb300 import synth
    if small:
        scene = synth.tiny_scene(seed=0)
        cams = synth.ring_cameras(max(1, min(views, 4)), 3.0)
        return scene, cams, 512, 512, {"workload": "icosphere-1280tri L4 N16-128, %d view(s) 512x512" % len(cams)}
    top = min(2048, 16 << (levels - 1))
    scene = synth.full_scene(seed=0, n_levels=levels, top=top)
    cams = synth.ring_cameras(views, RING_R)
    desc = ("displaced geodesic sphere 200k tris, L%d PSH N16-%d band 2 cells, F2 fp32, "
            "MLP %d-64-64-4, %d ring views r=2.5 at 3840x2160" % (levels, top, 2 * levels + 16, views))
    return scene, cams, W4K, H4K, {"workload": desc}


# Per-hit-ray counters of the FP32 shade kernel on the full workload, from one
# ncu capture of one 4K view (one launch, cold L2; the capture command sits in
# the profile summary of that kernel): DRAM bytes read + written, and the
# 32-byte sectors L2 served to L1 (lts__t_sectors_srcunit_tex_op_read.sum).
# Both grow in proportion to the hit rays rendered.  Each figure is keyed by a
# hash of the kernel's sources; once they change the figure prints as null
# until it is captured again.
SHADE_SOURCES = ["render.cu", "kernels_common.cuh", "tc_ptx.cuh", "inolf_internal.h"]
SHADE_COUNTERS = {"k_shade_f32": {"src_sha": "fc072ee43e256737",
                                   # (1 106 912 256 B read + 64 595 968 B written) / 4 010 637 hit rays
                                   "dram_bytes_per_hit": (1106912256 + 64595968) / 4010637,
                                   # 59 006 194 sectors / 4 010 637 hit rays
                                   "l2_sectors_per_hit": 59006194 / 4010637}}


def shade_source_sha() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in SHADE_SOURCES:
        with open(os.path.join(ROOT, "paper_2303_04086_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def shade_counters(kernel: str) -> dict:
    """The stored per-hit counters of `kernel`, or {} when they are stale."""
    c = SHADE_COUNTERS.get(kernel)
    if not c or c["src_sha"] != shade_source_sha():
        return {}
    return c


def algorithmic_bytes_per_hit(scene) -> int:
    # per hit ray: L levels x 8 corners x (F features + 4-byte Phi entry)
    fb = 2 if scene.feature_fp16 else 4
    return scene.n_levels * 8 * (2 * fb + 4)


def kernel_stats() -> dict:
    """The library's per-kernel launch statistics, with the split BF16 / FP8
    tensor-core shade (k_encode_tc_* gathers and encodes, k_mlp_tc_* runs the
    MLP) also summed under k_shade_tc_*, the name of the fused kernel it
    replaces.  The FP32 split shade (k_encode_tc_f32, k_mlp_tc_f32) stays as
    two entries: the roofline line takes the dominant kernel of the FP32
    step, so each must stand on its own."""
    from paper_2303_04086_gb300 import inolf
    st = inolf.stats_read()
    for prec in ("bf16", "fp8"):
        enc, mlp = st.get("k_encode_tc_" + prec), st.get("k_mlp_tc_" + prec)
        if enc and mlp:
            fused = st.get("k_shade_tc_" + prec, {"launches": 0, "ms": 0.0})
            st["k_shade_tc_" + prec] = {"launches": enc["launches"] + fused["launches"],
                                        "ms": enc["ms"] + mlp["ms"] + fused["ms"],
                                        "parts_ms": {"k_encode_tc": enc["ms"], "k_mlp_tc": mlp["ms"],
                                                     "k_shade_tc": fused["ms"]}}
            del st["k_encode_tc_" + prec], st["k_mlp_tc_" + prec]
    return st


def mlp_flops_per_hit(scene) -> int:
    return 2 * (64 * scene.d_in + 64 * 64 + 4 * 64)


# nominal dense tensor rates of the GB300: TF32 1.1, BF16 2.25 PFLOP/s
TF32_PER_BF16 = 1.1 / 2.25


def tf32_k1(scene) -> int:
    return (scene.d_in + 7) // 8 * 8


def tf32_row_bytes(scene) -> int:
    # one FP32 layer-1 operand row of the split shade
    return 4 * tf32_k1(scene)


def tf32x3_flops_per_hit(scene) -> int:
    # tensor-core flops the split-TF32 MLP issues per hit: three products per
    # layer, layer 1 padded to K1 columns, layer 3 to 16 outputs
    return 3 * 2 * (64 * tf32_k1(scene) + 64 * 64 + 16 * 64)


def encode_bytes_per_hit(scene) -> int:
    # the gather's algorithmic bytes, the hit record read, the operand row written
    return algorithmic_bytes_per_hit(scene) + 8 + tf32_row_bytes(scene)


def kernel_rooflines(kernels, scene, n_rays, n_hit, steps, peaks):
    """Every kernel of a timed run against its roofline: the shade kernels'
    algorithmic gather + output bytes against the measured HBM copy bandwidth
    and their MLP flops against the peak of their arithmetic (FP32 SIMT from
    the unit counts, BF16 measured, FP8 = 2 x BF16, the nominal ratio); the
    trace / march kernels' output bytes (16 B per miss, 8 B per hit record)
    against HBM, with rays per second (their limit is ALU issue, as ncu shows)."""
    hbm = peaks.get("hbm_gbs", 6800.0)
    bf16 = peaks.get("bf16_tflops", 1900.0)
    mlp_peak = {"k_shade_f32": 80.5, "k_shade_tc_bf16": bf16, "k_shade_tc_fp8": 2.0 * bf16}
    out = {}
    for name, st in kernels.items():
        if not st.get("launches"):
            continue
        sec = st["ms"] / 1e3
        per_step_launches = max(1, st["launches"] // max(1, steps))
        if name == "k_encode_tc_f32":
            byt = encode_bytes_per_hit(scene) * n_hit * steps
            out[name] = {"gbs": byt / sec / 1e9, "frac_hbm": byt / sec / 1e9 / hbm,
                         "frac_hbm_basis": "algorithmic gather bytes (every corner row and Phi entry) + the hit "
                                           "record read + the FP32 operand row written, per second over the HBM "
                                           "copy rate; L1 and L2 serve most of the gather, so it can exceed 1",
                         "bound": "latency (dependent L1/L2 gather loads)", "launches_per_step": per_step_launches}
        elif name == "k_mlp_tc_f32":
            fl = tf32x3_flops_per_hit(scene) * n_hit * steps
            byt = (tf32_row_bytes(scene) + 16 + 8) * n_hit * steps
            out[name] = {"tensor_tflops": fl / sec / 1e12, "frac_tf32_peak": fl / sec / 1e12 / (TF32_PER_BF16 * bf16),
                         "tf32_peak_tflops": TF32_PER_BF16 * bf16,
                         "tf32_peak_basis": "measured BF16 burst x 1.1 / 2.25, the nominal dense TF32 / BF16 ratio",
                         "mlp_tflops": mlp_flops_per_hit(scene) * n_hit * steps / sec / 1e12,
                         "gbs": byt / sec / 1e9, "frac_hbm": byt / sec / 1e9 / hbm,
                         "launches_per_step": per_step_launches}
        elif name.startswith("k_shade"):
            byt = (algorithmic_bytes_per_hit(scene) + 24) * n_hit * steps
            fl = mlp_flops_per_hit(scene) * n_hit * steps
            out[name] = {"gbs": byt / sec / 1e9, "frac_hbm": byt / sec / 1e9 / hbm,
                         "frac_hbm_basis": "algorithmic bytes (every corner row and Phi entry, 1 560 B per hit) "
                                           "per second over the HBM copy rate; L1 and L2 serve most of them, "
                                           "so it can exceed 1",
                         "mlp_tflops": fl / sec / 1e12, "frac_mlp_peak": fl / sec / 1e12 / mlp_peak.get(name, bf16),
                         "mlp_peak_tflops": mlp_peak.get(name, bf16), "launches_per_step": per_step_launches}
        else:
            byt = (16 * (n_rays - n_hit) + 8 * n_hit) * steps
            out[name] = {"gbs": byt / sec / 1e9, "frac_hbm": byt / sec / 1e9 / hbm,
                         "grays_per_s": n_rays * steps / sec / 1e9, "bound": "alu (issue)",
                         "launches_per_step": per_step_launches}
    return out


def add_probed_rooflines(rooflines, probed, scene, n_rays, n_hit, steps, kernels_by_prec, tstats):
    """The same kernels against the microbenchmarked peaks (inolf_probe_peaks):
    the PSH gather's load rate (16 per level and hit ray: 8 Phi + 8 table
    entries; L1 serves most of them, so the ratio to the L2 random-read rate
    can exceed 1), the FP32 SIMT MLP against the packed-FMA rate, and the
    trace kernel's BVH node visits per second (node visits per ray from
    inolf_trace_stats on view 0)."""
    for prec, kern in kernels_by_prec.items():
        for name, st in kern.items():
            if not st.get("launches") or name not in rooflines.get(prec, {}):
                continue
            sec = st["ms"] / 1e3
            r = rooflines[prec][name]
            if name.startswith("k_shade"):
                # all 16 loads per level and hit ray, most of them L1 hits: a
                # rate, not a fraction of the L2 probe (that one needs the
                # L2-served sectors, see the roofline entry)
                loads = 16 * scene.n_levels * n_hit * steps / sec / 1e9
                r["gather_gloads_per_s"] = loads
                r["gather_loads_per_l2_random_read"] = loads / probed["l2_gather_gsps"]
                if name == "k_shade_f32":
                    r["frac_fp32_fma_probe"] = r["mlp_tflops"] / probed["fp32_tflops"]
            elif name == "k_trace" and tstats:
                r["node_visits_per_ray"] = tstats["node_visits_per_ray"]
                r["triangle_tests_per_ray"] = tstats["triangle_tests_per_ray"]
                r["gnode_visits_per_s"] = tstats["node_visits_per_ray"] * n_rays * steps / sec / 1e9


ORACLE_BATCH_RAYS = 1_000_000


def time_oracle_batches(orc, cams, W, H, n_batches, warmup=1, batch_rays=ORACLE_BATCH_RAYS, seed=0,
                        budget_s=None):
    """The FP64 oracle as it stands on seeded batches of the workload: batch
    b renders `batch_rays` random pixels (sorted) of view b mod len(cams).
    The first `warmup` batches are not timed.  Stops after n_batches timed
    batches, or earlier once budget_s seconds are spent.  Returns (rays,
    seconds, per-batch seconds).  Both CPU legs of this file time the oracle
    through this function, so their figures are comparable."""
    rng = np.random.default_rng(seed)
    rays, secs, per = 0, 0.0, []
    n = min(batch_rays, W * H)
    for b in range(warmup + n_batches):
        pix = np.sort(rng.choice(W * H, n, replace=False)).astype(np.int64)
        t0 = time.perf_counter()
        orc.render_pixels(cams[b % len(cams)], W, H, pix)
        dt = time.perf_counter() - t0
        if b >= warmup:
            rays += n
            secs += dt
            per.append(dt)
            if budget_s is not None and secs >= budget_s:
                break
    return rays, secs, per


def cpu_baseline(scene, cams, W, H, budget_s=10.0, orc=None):
    """The FP64 oracle as it stands on the machine's host cores: batches of 10^6
    seeded random pixels cycling through the views (all cores, about
    budget_s seconds), the same on one thread (one batch of 10^5 pixels),
    and full frames of the tiny scene (one 128x128 view at distance 3) and of
    the precision-sweep scene (FP16 tables, one 3840x2160 ring view at r = 3)."""
    import oracle
    if orc is None:
        oracle.build()
        orc = oracle.Oracle(scene)
    cores = oracle.max_threads()
    rays, secs, _ = time_oracle_batches(orc, cams, W, H, n_batches=1000, warmup=1, budget_s=budget_s)
    rate = rays / secs
    out = {"value": rate / 1e6, "unit": "Mrays/s", "cores": cores, "kind": "oracle",
           "sample": f"{rays} rays in batches of {min(ORACLE_BATCH_RAYS, W * H)} seeded random pixels of views 1, 2, ... "
                     f"({W}x{H}; one untimed warm-up batch of view 0), FP64 oracle, {secs:.1f} s of CPU work "
                     f"on {cores} threads"}
    try:
        oracle.set_threads(1)
        r1, s1, _ = time_oracle_batches(orc, cams, W, H, n_batches=1, warmup=0, batch_rays=100_000, seed=1)
        out["value_1thread"] = r1 / s1 / 1e6
        out["sample_1thread"] = f"{r1} seeded random pixels of view 0 on 1 thread, {s1:.1f} s"
    finally:
        oracle.set_threads(cores)
    from paper_2303_04086_gb300 import synth
    frames = {}
    for name, sc, cam, fw, fh in (
            ("tiny_128x128", synth.tiny_scene(seed=0), synth.camera((0.0, 0.0, 3.0)), 128, 128),
            ("tiny_fp16_3840x2160", synth.tiny_scene(seed=0, fp16=True), synth.ring_cameras(1, 3.0)[0],
             3840, 2160)):
        o2 = oracle.Oracle(sc)
        o2.render_pixels(cam, min(fw, 64), min(fh, 64))  # warm-up
        t0 = time.perf_counter()
        o2.render_pixels(cam, fw, fh)
        dt = time.perf_counter() - t0
        frames[name] = {"rays": fw * fh, "seconds": dt, "mrays_per_s": fw * fh / dt / 1e6, "cores": cores}
        del o2
    out["full_frames"] = frames
    return out


def serving_workload(seed: int = 0):
    """12 tiny-scene objects (seeds 0-11) placed without bounding-sphere
    overlap in a 10 m cube; 32 viewers on a 12 m sphere around the cube
    centre, each with its resolution drawn from 720p / 1080p / 4K."""
    from paper_2303_04086_gb300 import synth
    return synth.serving_scene(seed)


def run_serving(seconds=10.0, warmup=1.0, rate_hz=50.0, seed=0, prec="bf16", policy=1,
                max_rays_in_flight=64_000_000):
    """Poisson frame requests of 32 viewers against the persistent request
    loop; returns p50/p99 submit->complete latency, throughput, refusals."""
    import heapq
    from paper_2303_04086_gb300 import inolf, synth
    scenes, places, viewers = serving_workload(seed)
    srv = inolf.Server(hbm_budget=8 << 30, max_slots=64, max_width=3840, max_height=2160, max_hits=4,
                       policy=policy, max_rays_in_flight=max_rays_in_flight if policy == 1 else 0)
    for v in range(len(viewers)):
        srv.set_viewer(v, rate_hz)
    objs = [inolf.object_create(sc) for sc in scenes]
    for o, p in zip(objs, places):
        srv.add_object(o, p)
    rng = np.random.default_rng(seed + 1)
    inolf.stats_reset()
    inolf.stats_enable(True)  # events around each persistent-kernel launch: the device's busy time
    t_submit = t_poll = 0.0
    events = [(rng.exponential(1.0 / rate_hz), v) for v in range(len(viewers))]
    heapq.heapify(events)
    inflight = {}
    lat, rays_done, frames, refused, submitted = [], 0, 0, 0, 0
    t0 = time.perf_counter()
    end = warmup + seconds
    frame_no = [0] * len(viewers)
    while True:
        now = time.perf_counter() - t0
        while events and events[0][0] <= now and events[0][0] < end:
            ta, v = heapq.heappop(events)
            vw = viewers[v]
            frame_no[v] += 1
            ang = 0.02 * frame_no[v]  # small orbit per frame
            axis = np.cross(vw["dir"], [0.0, 1.0, 0.0])
            axis = axis / (np.linalg.norm(axis) + 1e-12)
            dv = vw["dir"] * np.cos(ang) + np.cross(axis, vw["dir"]) * np.sin(ang)
            cam = synth.camera(tuple(12.0 * dv))
            W, H = vw["res"]
            try:
                ts0 = time.perf_counter()
                try:
                    t = srv.submit(cam, W, H, prec, viewer_id=v)
                finally:
                    t_submit += time.perf_counter() - ts0
                inflight[t] = (ta, W * H)
                submitted += 1
            except inolf.InolfError as e:
                if e.status != inolf.E_BUDGET:
                    raise
                if ta >= warmup:
                    refused += 1
            heapq.heappush(events, (ta + rng.exponential(1.0 / rate_hz), v))
        for t in list(inflight):
            tp0 = time.perf_counter()
            st, res = srv.poll(t)
            t_poll += time.perf_counter() - tp0
            if st == inolf.PENDING:
                continue
            ta, npx = inflight.pop(t)
            done_t = time.perf_counter() - t0
            if ta >= warmup and st == inolf.OK:
                lat.append(done_t - ta)
                rays_done += npx
                frames += 1
            srv.release(t)
        if now >= end and not inflight:
            break
        time.sleep(0.0002)
    wall = time.perf_counter() - t0 - warmup
    counters = srv.counters()
    prof = srv.profile()
    srv.close()
    inolf.stats_enable(False)
    ks = kernel_stats().get("k_serve", {"launches": 0, "ms": 0.0})
    work = sum(prof[k] for k in ("trace_cycles", "shade_cycles", "composite_cycles", "done_cycles"))
    phases = {k.replace("_cycles", ""): prof[k] / max(1, work)
              for k in ("trace_cycles", "shade_cycles", "composite_cycles", "done_cycles")}
    profile = {"phase_share_of_work": phases,
               "claim_and_idle_cycles_per_work_cycle": prof["claim_cycles"] / max(1, work),
               "cycles_per_tile": work / max(1, prof["tiles"]),
               "hits_per_tile": prof["hits"] / max(1, prof["tiles"]),
               "mlp_batches_per_tile": prof["mlp_batches"] / max(1, prof["tiles"]),
               "rows_used_per_256_row_batch": prof["hits"] / max(1, prof["mlp_batches"]),
               "kernel_launches": ks["launches"], "kernel_busy_s": ks["ms"] / 1e3, "persistent_ctas": prof["ctas"],
               "launch_plan": {k: prof[k] for k in ("regs_per_thread", "static_smem", "dynamic_smem", "ctas_per_sm")},
               "sm_mhz_implied": (prof["claim_cycles"] + work) / max(1, prof["ctas"]) / max(1e-9, ks["ms"] / 1e3) / 1e6,
               "host_submit_s": t_submit, "host_poll_s": t_poll, "wall_s_incl_warmup": wall + warmup,
               "raw": prof}
    lat_ms = np.array(lat) * 1e3
    return {"viewers": len(viewers), "objects": len(objs), "rate_hz_per_viewer": rate_hz, "seconds": seconds,
            "frames": frames, "frames_per_s": frames / wall, "mrays_per_s": rays_done / wall / 1e6,
            "p50_ms": float(np.percentile(lat_ms, 50)) if len(lat_ms) else None,
            "p99_ms": float(np.percentile(lat_ms, 99)) if len(lat_ms) else None,
            "refused": refused, "submitted": submitted, "precision": prec,
            "policy": "algorithm1" if policy == 1 else "arrival-order",
            "max_rays_in_flight": max_rays_in_flight if policy == 1 else None, "counters": counters,
            "kernel_profile": profile,
            "note": "latency = arrival time -> completion seen by the poller; refused = admission (slots/HBM "
                    "budget) full at arrival"}


def run_zoom_sweep(obj, W, H, prec="bf16", distances=(6.0, 4.0, 3.0, 2.5, 2.0, 1.6, 1.35)):
    """Speed vs camera distance at 4K (the linear-in-covered-pixels claim of
    one query per ray, Sec. 8.2): one view per distance; time vs hit rays is
    fitted by a line."""
    import torch
    from paper_2303_04086_gb300 import inolf, synth
    rgba = torch.empty((1, H, W, 4), device="cuda")
    tri = torch.empty((1, H, W), dtype=torch.int32, device="cuda")
    ws = torch.empty((inolf.render_workspace_bytes(W * H) + 15) // 16 * 4, dtype=torch.int32, device="cuda")
    rows = []
    for r in distances:
        cam = synth.camera((0.0, 0.0, r))[None]
        inolf.render(obj, cam, W, H, prec, rgba_out=rgba, tri_out=tri, workspace=ws)
        torch.cuda.synchronize()
        hits = int((tri >= 0).sum().item())
        evs = []
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            inolf.render(obj, cam, W, H, prec, rgba_out=rgba, workspace=ws)
            e1.record()
            evs.append((e0, e1))
        torch.cuda.synchronize()
        ms = min(a.elapsed_time(b) for a, b in evs)
        rows.append({"distance": r, "hit_fraction": hits / (W * H), "ms": ms, "mrays_per_s": W * H / ms / 1e3})
    x = np.array([q["hit_fraction"] for q in rows]) * W * H
    y = np.array([q["ms"] for q in rows])
    A = np.stack([np.ones_like(x), x], 1)
    coef, *_ = np.linalg.lstsq(A, y, rcond=None)
    r2 = 1 - ((A @ coef - y) ** 2).sum() / max(((y - y.mean()) ** 2).sum(), 1e-30)
    return {"precision": prec, "points": rows, "fit_ms": {"intercept": float(coef[0]),
            "per_mhit": float(coef[1] * 1e6), "r2": float(r2)}}


def run_looking_glass(views=45, W=420, H=560, arc_deg=40.0, seed=0):
    """A 45-view light-field quilt (Sec. 7, Looking Glass display): 45
    consecutive viewpoints on a horizontal arc, submitted together to the
    serving loop over the 12-object scene."""
    from paper_2303_04086_gb300 import inolf, synth
    scenes, places, _ = serving_workload(seed)
    centre = np.mean(places, 0)
    srv = inolf.Server(hbm_budget=1 << 30, max_slots=64, max_width=W, max_height=H)
    objs = [inolf.object_create(sc) for sc in scenes]
    for o, p in zip(objs, places):
        srv.add_object(o, p)
    cams = []
    for k in range(views):
        a = np.radians(-arc_deg / 2 + arc_deg * k / (views - 1))
        eye = centre + 12.0 * np.array([np.sin(a), 0.15, np.cos(a)])
        cams.append(synth.camera(tuple(eye), target=tuple(centre)))
    times = []
    for rep in range(4):
        t0 = time.perf_counter()
        ts = [srv.submit(c, W, H, "bf16") for c in cams]
        for t in ts:
            st, _ = srv.wait(t)
            assert st == inolf.OK
        times.append(time.perf_counter() - t0)
        for t in ts:
            srv.release(t)
    srv.close()
    best = min(times[1:])
    return {"views": views, "view_res": [W, H], "quilt_ms": best * 1e3, "quilts_per_s": 1.0 / best,
            "mrays_per_s": views * W * H / best / 1e6, "precision": "bf16"}


def run_training(steps=40, batch=1 << 18, n_views=100, res=800, prec="bf16"):
    """Differentiation workload: a teacher object (seed 1) renders 100 target
    views at 800x800; a student (seed 2) trains toward them with batches of
    2^18 random (view, pixel) rays, L2 loss (Eq. 8), Adam lr 1e-2, forward MLP
    in `prec`, FP32 backward with atomic scatter into the feature tables."""
    import torch
    from paper_2303_04086_gb300 import inolf, synth
    teacher = inolf.object_create(synth.tiny_scene(seed=1))
    field = inolf.Field(synth.tiny_scene(seed=2))
    cams = synth.fibonacci_cameras(n_views, 3.0)
    tgt = inolf.render(teacher, cams, res, res).reshape(-1, 4)
    # rays of all target pixels (inputs: any FP32 rays will do)
    c = torch.from_numpy(np.ascontiguousarray(cams)).cuda()
    jj, ii = torch.meshgrid(torch.arange(res, device="cuda"), torch.arange(res, device="cuda"), indexing="ij")
    a = ((2 * ii + 1).float() / res - 1).reshape(-1) * c[:, 12:13]
    b = (1 - (2 * jj + 1).float() / res).reshape(-1) * c[:, 12:13]
    d = a[..., None] * c[:, None, 3:6] + b[..., None] * c[:, None, 6:9] + c[:, None, 9:12]
    d = (d / d.norm(dim=-1, keepdim=True)).reshape(-1, 3).contiguous()
    o = c[:, None, 0:3].expand(-1, res * res, -1).reshape(-1, 3).contiguous()
    opt = torch.optim.Adam(field.parameters(), lr=1e-2, betas=(0.9, 0.99), eps=1e-15, capturable=True)
    torch.manual_seed(0)
    losses = []

    def one():
        idx = torch.randint(0, o.shape[0], (batch,), device="cuda")
        pred = field.render(o[idx], d[idx], prec)
        loss = ((pred - tgt[idx]) ** 2).sum(1).mean()
        opt.zero_grad(set_to_none=False)
        loss.backward()
        opt.step()
        return loss.detach()

    # warm-up on a side stream (allocations, one-time kernel attributes), then
    # the whole step -- sampling, inolf forward, inolf backward, Adam -- is
    # captured once as a CUDA graph and replayed; eager steps if capture fails
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(3):
            losses.append(one())
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph, static_loss = None, None
    try:
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            static_loss = one()
        torch.cuda.synchronize()
    except Exception as e:  # eager fallback, reported
        graph = None
        capture_error = str(e)[:200]
        torch.cuda.synchronize()
    inolf.stats_reset()
    inolf.stats_enable(graph is None)
    t0 = time.perf_counter()
    for _ in range(steps):  # losses stay on the device: no host synchronisation inside the loop
        if graph is not None:
            graph.replay()
            losses.append(static_loss.clone())
        else:
            losses.append(one())
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    if graph is not None:  # per-kernel times from a few eager steps with launch events (outside the timed loop)
        inolf.stats_enable(True)
        for _ in range(5):
            one()
        torch.cuda.synchronize()
        n_kern = 5
    else:
        n_kern = steps
    inolf.stats_enable(False)
    kern = {k: {"launches": v["launches"], "ms_per_step": v["ms"] / n_kern} for k, v in kernel_stats().items()}
    losses = [float(x) for x in losses]
    out = {"steps_per_s": steps / dt, "rays_per_step": batch, "mrays_per_s": steps * batch / dt / 1e6,
           "loss_first": losses[0], "loss_last": losses[-1], "forward": prec, "backward": "fp32",
           "views": n_views, "res": res, "cuda_graph": graph is not None, "kernels": kern}
    if graph is None:
        out["capture_error"] = capture_error
    return out


def run_variant(steps=3, warmup=3, views=N_VIEWS, precisions=("fp32", "bf16", "fp8"), oracle_pixels=100_000):
    """The paper's decoupled variant (Sec. 4.2, Eqs. 4-7) on the same object
    as a density shell: 64 ring views at 4K, hit points from the density march
    (k_march), alpha_c input, c = c_d + t c_s.  Returns per-precision Mrays/s
    with per-kernel times, the accuracy of view 0 against the oracle on a
    pixel sample, and the march alone on 1080p frames."""
    import torch
    from paper_2303_04086_gb300 import inolf, synth
    t0 = time.time()
    scene = synth.full_density_scene(seed=0)
    hashes = inolf.build_hashes(scene, slot_slack=SLOT_SLACK)
    obj = inolf.object_create(scene, hashes)
    prep_s = time.time() - t0
    cams = synth.ring_cameras(views, RING_R)
    W, H = W4K, H4K
    n_rays = views * W * H
    dev = torch.device("cuda", torch.cuda.current_device())
    rgba = torch.empty((views, H, W, 4), dtype=torch.float32, device=dev)
    ws = torch.empty((inolf.render_workspace_bytes(n_rays) + 15) // 16 * 4, dtype=torch.int32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    kk = torch.empty((views, H, W), dtype=torch.int32, device=dev)
    inolf.render(obj, cams, W, H, "fp32", rgba_out=rgba, tri_out=kk, workspace=ws)
    torch.cuda.synchronize()
    n_hit = int((kk >= 0).sum().item())
    del kk
    out = {"workload": ("displaced-sphere density shell (half-width 2 fine cells, optical depth 12), 128^3 base "
                        "cells x 16^3 fine cells, %d cubes; L16 PSH N16-2048 over the voxels around possible hit "
                        "points; MLP 49-64-64-4 with alpha_c; %d ring views r=2.5 at 3840x2160"
                        % (scene.cubes.n, views)),
           "prep_s": round(prep_s, 1), "rays_per_step": n_rays, "hit_rays_per_step": n_hit, "precisions": {}}
    for prec in precisions:
        if prec == "fp8":
            inolf.calibrate_fp8(obj, cams[:1], W, H, workspace=ws)
        for _ in range(warmup):
            inolf.render(obj, cams, W, H, prec, rgba_out=rgba, workspace=ws, stream=stream)
        torch.cuda.synchronize()
        inolf.stats_reset()
        inolf.stats_enable(True)
        evs = []
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            inolf.render(obj, cams, W, H, prec, rgba_out=rgba, workspace=ws, stream=stream)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        inolf.stats_enable(False)
        ms = sum(e0.elapsed_time(e1) for e0, e1 in evs)
        out["precisions"][prec] = {"value": n_rays * steps / (ms / 1e3) / 1e6, "unit": "Mrays/s",
                                   "ms_per_step": ms / steps, "kernels": kernel_stats()}
    # the march alone on 1080p frames (the paper times its hit estimation per 1080p image)
    W2, H2 = 1920, 1080
    o_views = 8
    c8 = synth.ring_cameras(o_views, RING_R)
    k8 = torch.empty((o_views, H2, W2), dtype=torch.int32, device=dev)
    f8 = torch.empty((o_views, H2, W2, 4), dtype=torch.float32, device=dev)
    for _ in range(3):
        inolf.render(obj, c8, W2, H2, "bf16", rgba_out=f8, tri_out=k8, workspace=ws, stream=stream)
    torch.cuda.synchronize()
    inolf.stats_reset()
    inolf.stats_enable(True)
    for _ in range(5):
        inolf.render(obj, c8, W2, H2, "bf16", rgba_out=f8, tri_out=k8, workspace=ws, stream=stream)
    torch.cuda.synchronize()
    inolf.stats_enable(False)
    st = kernel_stats()
    if "k_march" in st:
        out["march_ms_per_1080p_frame"] = st["k_march"]["ms"] / (5 * o_views)
    # accuracy of view 0 on a pixel sample against the oracle (FP32 argmax
    # near-ties, a handful, are compared at the oracle's own decision anyway)
    try:
        if oracle_pixels <= 0:
            raise RuntimeError("accuracy check skipped")
        import oracle
        oracle.build()
        orc = oracle.Oracle(scene)
        rng = np.random.default_rng(7)
        pix = np.sort(rng.choice(W * H, oracle_pixels, replace=False)).astype(np.int64)
        ref = orc.render_variant_pixels(cams[0], W, H, pix)
        hit = ref["k"] >= 0
        pt = torch.from_numpy(pix).to(dev)
        v0 = torch.empty((1, H, W, 4), dtype=torch.float32, device=dev)
        for prec in precisions:
            inolf.render(obj, cams[:1], W, H, prec, rgba_out=v0, workspace=ws)
            got = v0.reshape(-1, 4)[pt].cpu().numpy()
            mse = float(np.mean((got[hit] - ref["rgba"][hit]) ** 2))
            out["precisions"][prec]["accuracy_vs_oracle"] = {
                "psnr_db": 10 * math.log10(1.0 / mse) if mse > 0 else 99.0,
                "max_abs": float(np.abs(got - ref["rgba"]).max()), "view": 0, "pixels": int(len(pix))}
    except Exception as e:  # the accuracy check is a report, not the measurement
        out["accuracy_error"] = str(e)[:200]
    del rgba, ws, flush, obj, f8, k8
    torch.cuda.empty_cache()
    return out


def run_precision_sweep(steps=3, warmup=3, views=N_VIEWS, pixels_per_view=4000):
    """The precision sweep on the tiny scene with FP16 feature tables: 64 ring
    views at r = 3 and 3840x2160 rendered with the FP32, BF16 and FP8 MLPs
    (Mrays/s each), and every view's PSNR / max-abs against the FP64 oracle on
    a seeded pixel sample."""
    import torch
    import oracle
    from paper_2303_04086_gb300 import inolf, synth
    scene = synth.tiny_scene(seed=0, fp16=True)
    obj = inolf.object_create(scene)
    cams = synth.ring_cameras(views, 3.0)
    W, H = W4K, H4K
    n_rays = views * W * H
    dev = torch.device("cuda", torch.cuda.current_device())
    rgba = torch.empty((views, H, W, 4), dtype=torch.float32, device=dev)
    ws = torch.empty((inolf.render_workspace_bytes(n_rays) + 15) // 16 * 4, dtype=torch.int32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    inolf.calibrate_fp8(obj, cams[:1], W, H, workspace=ws)
    oracle.build()
    orc = oracle.Oracle(scene)
    rng = np.random.default_rng(11)
    samples = [np.sort(rng.choice(W * H, pixels_per_view, replace=False)).astype(np.int64) for _ in range(views)]
    refs = [orc.render_pixels(cams[v], W, H, samples[v]) for v in range(views)]
    out = {"workload": "icosphere-1280tri L4 N16-128, FP16 feature tables, MLP 24-64-64-4, %d ring views r=3 at "
                       "3840x2160" % views,
           "accuracy": "per view, %d seeded pixels, PSNR over the 4 channels of hit pixels" % pixels_per_view,
           "precisions": {}}
    for prec in ("fp32", "bf16", "fp8"):
        for _ in range(warmup):
            inolf.render(obj, cams, W, H, prec, rgba_out=rgba, workspace=ws, stream=stream)
        torch.cuda.synchronize()
        evs = []
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            inolf.render(obj, cams, W, H, prec, rgba_out=rgba, workspace=ws, stream=stream)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        ms = sum(e0.elapsed_time(e1) for e0, e1 in evs)
        flat = rgba.reshape(views, -1, 4)
        psnrs, maxabs = [], 0.0
        for v in range(views):
            got = flat[v][torch.from_numpy(samples[v]).to(dev)].cpu().numpy()
            hit = refs[v]["tri"] >= 0
            mse = float(np.mean((got[hit] - refs[v]["rgba"][hit]) ** 2)) if hit.any() else 0.0
            psnrs.append(10 * math.log10(1.0 / mse) if mse > 0 else 99.0)
            maxabs = max(maxabs, float(np.abs(got - refs[v]["rgba"]).max()))
        out["precisions"][prec] = {"value": n_rays * steps / (ms / 1e3) / 1e6, "unit": "Mrays/s",
                                   "ms_per_step": ms / steps, "psnr_db_min": min(psnrs),
                                   "psnr_db_median": float(np.median(psnrs)), "max_abs": maxabs}
    del rgba, ws, flush, obj
    torch.cuda.empty_cache()
    return out


def run_reference(a):
    """The oracle as it stands (the reference of this project), one batch of
    10^6 seeded random pixels per step, views cycling, on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    scene, cams, W, H, cfg = make_workload(a.small, a.views, a.levels)
    import oracle
    oracle.build()
    orc = oracle.Oracle(scene)
    rays, secs, _ = time_oracle_batches(orc, cams, W, H, n_batches=a.steps, warmup=a.warmup)
    val = rays / secs / 1e6
    cfg = dict(cfg)
    cfg["sample"] = (f"{min(ORACLE_BATCH_RAYS, W * H)} seeded random pixels per step, step s on view s mod "
                     f"{len(cams)} ({W}x{H}), FP64 oracle on {oracle.max_threads()} threads")
    out = {"impl": "reference", "metric": "i-NOLF Mrays/s at 4K (FP32 plain)", "value": val, "unit": "Mrays/s",
           "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * secs / a.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": cfg,
           "cpu_baseline": {"value": val, "unit": "Mrays/s", "cores": oracle.max_threads(), "kind": "oracle",
                            "sample": cfg["sample"]},
           "e2e": {"value": val, "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_native(a):
    import torch
    from paper_2303_04086_gb300 import build, inolf, synth
    rank, world, local = _dist_init(a.gpus)
    build.build()
    scene, cams, W, H, cfg = make_workload(a.small, a.views, a.levels)
    t0 = time.time()
    hashes = inolf.build_hashes(scene, slot_slack=1.0 if a.small else SLOT_SLACK)
    obj = inolf.object_create(scene, hashes)
    prep_s = time.time() - t0
    nv = len(cams)
    n_rays = nv * W * H
    dev = torch.device("cuda", torch.cuda.current_device())
    rgba = torch.empty((nv, H, W, 4), dtype=torch.float32, device=dev)
    ws = torch.empty((inolf.render_workspace_bytes(n_rays) + 15) // 16 * 4, dtype=torch.int32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    stream = torch.cuda.current_stream()
    peaks = _peaks()

    def step(prec):
        inolf.render(obj, cams, W, H, prec, rgba_out=rgba, workspace=ws, stream=stream)

    # hit count (for per-hit algorithmic work)
    tri = torch.empty((nv, H, W), dtype=torch.int32, device=dev)
    inolf.render(obj, cams, W, H, "fp32", rgba_out=rgba, tri_out=tri, workspace=ws)
    torch.cuda.synchronize()
    n_hit = int((tri >= 0).sum().item())
    del tri

    def timed(prec, steps, warmup, with_stats=False):
        for _ in range(warmup):
            step(prec)
        torch.cuda.synchronize()
        _barrier(world)
        inolf.stats_reset()
        inolf.stats_enable(with_stats)
        evs = []
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(prec)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        _barrier(world)
        inolf.stats_enable(False)
        ms = sum(e0.elapsed_time(e1) for e0, e1 in evs)
        return ms, kernel_stats()

    with ClockSampler(local) as clk:
        ms, stats = timed("fp32", a.steps, a.warmup, with_stats=True)
    ms = _max_over_ranks(ms, world)
    clocks = clk.summary()
    value = replica_throughput(n_rays * a.steps, ms / 1e3, world) / 1e6

    # precision variants: BF16 / FP8-e4m3 MLP on the tensor cores (FP8
    # activation scales calibrated once from the FP32 path on view 0)
    precisions = {}
    for prec in [p for p in a.precisions.split(",") if p and p != "fp32"]:
        try:
            if prec == "fp8":
                inolf.calibrate_fp8(obj, cams[:1], W, H, workspace=ws)
            pms, pstats = timed(prec, a.steps, 1, with_stats=True)
            pms = _max_over_ranks(pms, world)
            precisions[prec] = {"value": n_rays * a.steps * world / (pms / 1e3) / 1e6, "unit": "Mrays/s",
                                "ms_per_step": pms / a.steps, "kernels": pstats}
        except inolf.InolfError as e:
            precisions[prec] = {"unavailable": str(e)}

    # end to end through the C ABI with host buffers: the cameras go from
    # host memory into the launch, every RGBA frame comes back to pinned host
    # memory inside the timed region (inolf_render_host: rendering of chunk
    # c + 1 overlaps the copy of chunk c)
    host_out = torch.empty((nv, H, W, 4), dtype=torch.float32, pin_memory=True)
    host_cams = np.ascontiguousarray(cams, np.float32)
    e2e_steps = max(1, min(a.steps, 3))
    vpc = 4
    staging = torch.empty((2 * vpc * H * W * 4,), dtype=torch.float32, device=dev)

    def e2e_step():
        inolf.render_host(obj, host_cams, W, H, "fp32", host_out=host_out, staging=staging, workspace=ws,
                          stream=stream, views_per_chunk=vpc)

    e2e_step()
    torch.cuda.synchronize()
    _barrier(world)
    t_e = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = _max_over_ranks(time.perf_counter() - t_e, world)
    e2e = {"value": n_rays * e2e_steps * world / e2e_s / 1e6, "unit": "Mrays/s",
           "h2d_bytes_per_step": int(host_cams.nbytes), "d2h_bytes_per_step": int(host_out.numel() * 4)}
    del host_out, staging

    # roofline of the dominant kernel (from CUDA events around each launch)
    top = max(stats, key=lambda k: stats[k]["ms"]) if stats else None
    roof = None
    if top:
        st = stats[top]
        avg_s = st["ms"] / 1e3 / st["launches"]
        hits_per_launch = n_hit / max(1, st["launches"] // a.steps) if a.steps else n_hit
        peak = peaks.get("hbm_gbs", 6800.0)
        if top == "k_encode_tc_f32":
            byt = encode_bytes_per_hit(scene) * hits_per_launch
            achieved = byt / avg_s / 1e9
            cnt = shade_counters(top) if not a.small and a.levels == 16 else {}
            dram = cnt.get("dram_bytes_per_hit")
            l2s = cnt.get("l2_sectors_per_hit")
            roof = {"kernel": top, "bound": "latency (dependent L1/L2 gather loads)", "achieved": achieved,
                    "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_source": "measured",
                    "traffic": dram * hits_per_launch if dram else None,
                    "algorithmic_bytes_per_launch": byt,
                    "frac_algorithmic_of_hbm": achieved / peak,
                    "frac_dram_of_hbm": dram * hits_per_launch / avg_s / 1e9 / peak if dram else None,
                    "l2_sectors_per_launch": l2s * hits_per_launch if l2s else None,
                    "frac_l2_served_of_l2_random_probe": None,
                    "counters_src_sha": shade_source_sha()}
        elif top == "k_mlp_tc_f32":
            fl = tf32x3_flops_per_hit(scene) * hits_per_launch
            tpk = TF32_PER_BF16 * peaks.get("bf16_tflops", 1900.0)
            achieved = fl / avg_s / 1e12
            roof = {"kernel": top, "bound": "tensor", "achieved": achieved, "peak": tpk, "unit": "TFLOP/s",
                    "frac": achieved / tpk, "peak_source": "measured BF16 burst x 1.1 / 2.25 (nominal dense TF32 / BF16 ratio)",
                    "traffic": None, "flops_per_launch": fl}
        elif top.startswith("k_shade"):
            # the gather's algorithmic bytes over the measured HBM copy rate (the
            # contract's fraction); the kernel is bound by the latency of its
            # dependent L1/L2 gathers, so the DRAM bytes it actually moves and
            # the L2-served sectors against the probed L2 random-read rate are
            # reported beside it
            byt = algorithmic_bytes_per_hit(scene) * hits_per_launch + 16 * hits_per_launch + 8 * hits_per_launch
            achieved = byt / avg_s / 1e9
            cnt = shade_counters(top) if not a.small and a.levels == 16 else {}
            dram = cnt.get("dram_bytes_per_hit")
            l2s = cnt.get("l2_sectors_per_hit")
            roof = {"kernel": top, "bound": "latency (dependent L1/L2 gather loads)", "achieved": achieved,
                    "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_source": "measured",
                    "traffic": dram * hits_per_launch if dram else None,
                    "algorithmic_bytes_per_launch": byt,
                    "frac_algorithmic_of_hbm": achieved / peak,
                    "frac_dram_of_hbm": dram * hits_per_launch / avg_s / 1e9 / peak if dram else None,
                    "l2_sectors_per_launch": l2s * hits_per_launch if l2s else None,
                    "frac_l2_served_of_l2_random_probe": None,
                    "counters_src_sha": shade_source_sha(),
                    "mlp_tflops": mlp_flops_per_hit(scene) * hits_per_launch / avg_s / 1e12,
                    "mlp_frac_of_fp32_peak": mlp_flops_per_hit(scene) * hits_per_launch / avg_s / 80.5e12}
        else:
            rays_per_launch = n_rays / max(1, st["launches"] // a.steps)
            byt = 16 * rays_per_launch + 8 * hits_per_launch
            achieved = byt / avg_s / 1e9
            roof = {"kernel": top, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": None}

    base = None
    fp32_acc = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        import oracle
        oracle.build()
        orc = oracle.Oracle(scene)
        base = cpu_baseline(scene, cams, W, H, orc=orc)
        # accuracy of every precision on view 0 (full frame) against the FP64 oracle
        ref = orc.render_pixels(cams[0], W, H)
        hit = ref["tri"] >= 0
        v0 = torch.empty((1, H, W, 4), dtype=torch.float32, device=dev)
        tri0 = torch.empty((1, H, W), dtype=torch.int32, device=dev)
        for prec in ["fp32"] + list(precisions):
            if "unavailable" in precisions.get(prec, {}):
                continue
            inolf.render(obj, cams[:1], W, H, prec, rgba_out=v0, tri_out=tri0 if prec == "fp32" else None,
                         workspace=ws)
            got = v0.cpu().numpy().reshape(-1, 4)
            mse = float(np.mean((got[hit] - ref["rgba"][hit]) ** 2))
            acc = {"psnr_db": 10 * math.log10(1.0 / mse) if mse > 0 else 99.0,
                   "max_abs": float(np.abs(got - ref["rgba"]).max()), "view": 0}
            if prec == "fp32":
                # hit triangle ids against the oracle's, and the rays whose winning hit
                # lies within 1e-6 (barycentric) of a triangle edge
                acc["tri_id_mismatches"] = int((tri0.cpu().numpy().ravel() != ref["tri"]).sum())
                acc["near_edge_rays"] = int(np.asarray(ref["near_edge"]).sum())
                fp32_acc = acc
            else:
                precisions[prec]["accuracy_vs_oracle"] = acc

    cfg = dict(cfg)
    cfg.update({"l2": "flushed between timed steps (256 MB write); output 8.5 GB > L2" if not a.small else
                "flushed between timed steps", "rays_per_step": n_rays, "hit_rays_per_step": n_hit,
                "prep_s": round(prep_s, 1), "slot_slack": 1.0 if a.small else SLOT_SLACK})
    out = {"metric": "i-NOLF Mrays/s at 4K (FP32 plain)", "value": value, "unit": "Mrays/s", "n_gpus": world,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
           "e2e": e2e, "gpu_launches": int(sum(s["launches"] for s in stats.values())),
           "kernels": stats, "roofline": roof, "cpu_baseline": base, "clocks": clocks,
           "precisions": precisions, "hit_mrays_per_s": n_hit * a.steps * world / (ms / 1e3) / 1e6}
    out["kernel_rooflines"] = {"fp32": kernel_rooflines(stats, scene, n_rays, n_hit, a.steps, peaks)}
    for prec, pr in precisions.items():
        if "kernels" in pr:
            out["kernel_rooflines"][prec] = kernel_rooflines(pr["kernels"], scene, n_rays, n_hit, a.steps, peaks)
    if rank == 0:
        try:  # measurement aids outside the timed region; the bench line stands without them
            probed = inolf.probe_peaks()
            tstats = inolf.trace_stats(obj, cams[:1], W, H)
            by_prec = {"fp32": stats}
            by_prec.update({k: v["kernels"] for k, v in precisions.items() if "kernels" in v})
            add_probed_rooflines(out["kernel_rooflines"], probed, scene, n_rays, n_hit, a.steps, by_prec, tstats)
            out["peaks_probed"] = probed
            if roof and roof.get("l2_sectors_per_launch"):
                st = stats[roof["kernel"]]
                avg_s = st["ms"] / 1e3 / st["launches"]
                roof["frac_l2_served_of_l2_random_probe"] = (roof["l2_sectors_per_launch"] / avg_s / 1e9 /
                                                             probed["l2_gather_gsps"])
            out["trace_stats_view0"] = tstats
        except Exception as e:  # noqa: BLE001
            out["peaks_probed"] = {"error": str(e)[:200]}
    if fp32_acc is not None:
        out["accuracy_vs_oracle"] = fp32_acc
    if rank == 0 and not a.small:
        out["zoom_sweep"] = run_zoom_sweep(obj, W, H)
    if rank == 0 and not a.small and not a.no_variant:
        del rgba, ws
        torch.cuda.empty_cache()
        out["variant"] = run_variant(steps=max(1, a.steps), warmup=max(1, a.warmup),
                                     precisions=[p for p in ["fp32"] + list(precisions)
                                                 if "unavailable" not in precisions.get(p, {})])
    if rank == 0 and not a.small and not a.no_variant:
        out["precision_sweep"] = run_precision_sweep(steps=max(1, a.steps), warmup=max(1, a.warmup))
    if rank == 0 and not a.no_serving and not a.small:
        rgba = ws = None
        torch.cuda.empty_cache()
        out["serving"] = run_serving(seconds=a.serving_seconds, policy=1)
        out["serving_fifo"] = run_serving(seconds=a.serving_seconds, policy=0)
        # the same scene and viewers at three times the request rate: the loop's
        # capacity once the 50 Hz load no longer saturates it
        out["serving_capacity"] = run_serving(seconds=5.0, rate_hz=150.0, policy=1)
        out["training"] = run_training()
        out["looking_glass"] = run_looking_glass()
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    a = _args()
    if a.impl == "reference":
        run_reference(a)
    elif a.training_only:
        from paper_2303_04086_gb300 import build
        build.build()
        print(json.dumps({"training": run_training(steps=max(1, a.steps))}))
    elif a.serving_only:
        from paper_2303_04086_gb300 import build
        build.build()
        print(json.dumps({"serving": run_serving(seconds=a.serving_seconds, policy=1),
                          "serving_capacity": run_serving(seconds=5.0, rate_hz=150.0, policy=1)}))
    elif a.variant_only:
        from paper_2303_04086_gb300 import build
        build.build()
        out = run_variant(steps=max(1, a.steps), warmup=max(1, a.warmup), views=a.views,
                          precisions=[p for p in a.precisions.split(",") if p],
                          oracle_pixels=0 if a.no_cpu_baseline else 100_000)
        print(json.dumps({"variant": out}))
    else:
        run_native(a)


if __name__ == "__main__":
    main()
