"""Benchmark of the MBOIT puzzle-piece render on GB300.

Workload (default, "amr"): brick octree of 81,549 leaves of 8^3 cells over
three levels (41.8 M cells, finest 832^3), float32 vertex values of the
512^3 workload's analytic field (64 Gaussian blobs + 3-octave value noise),
72 Morton pieces of uneven size (largest / smallest = 8), 2560x2560
perspective view, step 0.5 finest voxel, 4 power moments in float32.

One step = one frame: pass 1 (moments of all pieces, summed) + pass 2
(transmittance reconstruction, blend, colour sum and renormalisation),
replayed from a CUDA graph.  value = owned lattice samples per frame (each
marched once per pass) / frame time, in Gsamples/s, summed over ranks.  The
512^3 regular-grid workload, the tetrahedral and mixed-cell meshes, the
gear-teeth stress test and the precision sweep follow as further keys.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the only reference this method
has) on every host core, on a bounded pixel sample of the same workload.
Under torchrun (N > 1) every rank renders its own replica (no data-path
collective); rank 0 prints.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gsamples/s & ms/frame: batched mixed-prec vs plain FP32, RMSE vs FP64 oracle"
UNIT = "Gsamples/s"
# FP32 operations per owned sample on the algorithm's path (fma = 2, add / mul = 1;
# MUFU ops, min / max and conversions not counted):
# pass 1 on a grid: position 6, cell fractions 3, trilinear 21, table coordinate 3,
#   extinction lerp 2, depth warp 2, moments 12 (m0 add, four fma, three products);
# pass 1 on an octree: the same plus the leaf-local coordinates (p - origin) / h (6);
# pass 2 from the sample cache: table coordinate 3, extinction lerp 2, opacity
#   1 - e^-a 11 (series branch), depth warp 2, moment bound 35 (both branches'
#   arithmetic, which the kernel evaluates before selecting), exponent 1,
#   weight 1, colour 13; the split form adds the march (position, fractions,
#   trilinear: 30).
FLOP_PASS1 = {"grid": 49, "amr": 55}
FLOP_PASS2_FRAME = 68
FLOP_PASS2 = FLOP_PASS2_FRAME + 6 + 3 + 21
CACHE_BYTES_PER_SAMPLE = 4
# FP32 peak from unit counts and the maximum SM clock: 152 SMs x 128 lanes x
# 2 FLOP x 2.070 GHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# MUFU (special-function) results per second: 152 SMs x 16 per clock x 2.070 GHz;
# per owned sample pass 1 takes 1 (log2 of the depth), pass 2 from the cache 4
# (log2, rcp, rsqrt, exp2), the one-launch frame both.
MUFU_PEAK_TOPS = 152 * 16 * 2.070e9 / 1e12
MUFU_PASS1, MUFU_PASS2 = 1, 4


def roofs_of(samples, launch_ms, flop, mufu, traffic, hbm_gbs, ncu_rec):
    """The four roofs of one kernel launch (FP32 ALU, MUFU, HBM, L2) as
    fractions of their peaks, and the binding one (the largest).  ALU and MUFU
    from the algorithmic counts per owned sample and the launch time; HBM from
    the ncu DRAM bytes of the launch (None without a record) and the measured
    copy rate; L2 (and the issue slots, for reference) from the ncu record's
    percentages of peak."""
    sec = launch_ms * 1e-3
    r = {"alu": flop * samples / sec / 1e12 / FP32_PEAK_TFLOPS,
         "mufu": mufu * samples / sec / 1e12 / MUFU_PEAK_TOPS}
    r["hbm"] = traffic / sec / 1e9 / hbm_gbs if (traffic is not None and hbm_gbs) else None
    r["l2"] = ncu_rec["l2_throughput_pct"] / 100.0 if ncu_rec and "l2_throughput_pct" in ncu_rec else None
    known = {k: v for k, v in r.items() if v is not None}
    b = max(known, key=known.get)
    out = {f"{k}_frac": v for k, v in r.items()}
    out.update({"binding": b, "binding_frac": known[b],
                "issue_active_frac_ncu": ncu_rec["issue_active_pct"] / 100.0
                if ncu_rec and "issue_active_pct" in ncu_rec else None,
                "peaks": {"alu_tflops": FP32_PEAK_TFLOPS, "mufu_tops": MUFU_PEAK_TOPS, "hbm_gbs": hbm_gbs,
                          "sources": "ALU and MUFU derived from unit counts at 2.07 GHz; HBM measured copy rate; "
                                     "L2 as ncu's percentage of its peak"}})
    return out
CSRC = os.path.join(ROOT, "paper_2501_12581_gb300", "csrc")
# committed ncu records of the frame kernels (DRAM bytes per launch and the
# binding units' activity), one file per (kernel, workload), valid while the
# kernel sources are unchanged
NCU_DIR = os.path.join(ROOT, "profiles")


def ncu_record_path(kernel, workload):
    return os.path.join(NCU_DIR, f"ncu_{kernel}_{workload}.txt")


def _measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


MEASURED = _measured_peaks()


# device headers every frame kernel includes
COMMON_SOURCES = ["mboit_common.cuh", "mboit_device.cuh", "mboit_internal.h", "mboit_power.cuh", "mboit_trig.cuh"]


def kernel_sources(kernel):
    """The library sources a frame kernel is compiled from: the octree / mesh
    kernels (k_*_unit) or the grid kernels (k_*_fused), plus the shared device
    headers."""
    fam = "mboit_units" if "unit" in kernel else "mboit_grid"
    own = sorted(f for f in os.listdir(CSRC) if f.startswith(fam) and f.endswith((".cu", ".cuh")))
    return own + COMMON_SOURCES


def kernel_hash(kernel="k_frame_unit"):
    """Hash of the sources `kernel` is compiled from."""
    h = hashlib.sha256()
    for f in kernel_sources(kernel):
        h.update(f.encode())
        h.update(open(os.path.join(CSRC, f), "rb").read())
    return h.hexdigest()[:16]


def measured_ncu(kernel, workload):
    """The committed ncu record of `kernel` on `workload` (DRAM bytes per
    launch and the binding units' activity), or None when there is none for
    that kernel and workload or the kernel sources changed since."""
    try:
        kv = dict(tok.split("=", 1) for tok in open(ncu_record_path(kernel, workload)).read().split() if "=" in tok)
        if kv.get("kernel") == kernel and kv.get("workload") == workload and kv.get("kernel_sha") == kernel_hash(kernel):
            return {k: float(v) for k, v in kv.items() if k not in ("kernel", "workload", "kernel_sha", "note")}
    except (OSError, ValueError, KeyError):
        pass
    return None


def measured_traffic(kernel, workload):
    rec = measured_ncu(kernel, workload)
    return int(rec["dram_bytes_per_launch"]) if rec and "dram_bytes_per_launch" in rec else None


def write_ncu_record(csv_path, kernel, workload, samples, out_path):
    """Writes the record `measured_ncu` reads from an `ncu --page raw --csv`
    dump of one launch of the frame kernel: DRAM bytes of the launch, the
    binding units' activity and the owned samples that launch processed."""
    import csv
    rows = list(csv.reader(open(csv_path)))
    hdr, units, vals = rows[0], rows[1], rows[2]
    d = dict(zip(hdr, vals))
    u = dict(zip(hdr, units))

    def num(name):
        v = float(d[name].replace(",", ""))
        scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "Tbyte": 1e12}.get(u.get(name, ""), 1)
        return v * scale
    dram = num("dram__bytes_read.sum") + num("dram__bytes_write.sum")
    inst = num("smsp__inst_executed.sum")
    rec = {"kernel": kernel, "workload": workload, "kernel_sha": kernel_hash(kernel),
           "dram_bytes_per_launch": int(dram), "samples_per_launch": int(samples),
           "launch_ms": num("gpu__time_duration.sum") * ({"usecond": 1e-3, "msecond": 1, "nsecond": 1e-6}
                                                           .get(u.get("gpu__time_duration.sum"), 1)),
           "issue_active_pct": num("smsp__issue_active.avg.pct_of_peak_sustained_active"),
           "sm_sol_pct": num("sm__throughput.avg.pct_of_peak_sustained_elapsed"),
           "l1_data_pipe_pct": num("l1tex__throughput.avg.pct_of_peak_sustained_active"),
           "l2_throughput_pct": num("lts__throughput.avg.pct_of_peak_sustained_elapsed"),
           "dram_throughput_pct": num("gpu__dram_throughput.avg.pct_of_peak_sustained_elapsed"),
           "alu_pipe_pct": num("sm__inst_executed_pipe_alu.avg.pct_of_peak_sustained_active"),
           "fma_pipe_pct": num("sm__inst_executed_pipe_fma.avg.pct_of_peak_sustained_active"),
           "xu_pipe_pct": num("sm__inst_executed_pipe_xu.avg.pct_of_peak_sustained_active"),
           "lsu_pipe_pct": num("sm__inst_executed_pipe_lsu.avg.pct_of_peak_sustained_active"),
           "inst_per_sample": inst * 32 / samples}
    with open(out_path, "w") as f:
        f.write(" ".join(f"{k}={v:.6g}" if isinstance(v, float) else f"{k}={v}" for k, v in rec.items()) + "\n")
    return rec


class ClockSampler:
    """nvidia-smi clock/throttle samples every 25 ms while running; begin() and
    end() bracket the timed region, and the summary keeps the samples that
    arrived inside it (else the first one after it)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []          # (arrival time, line)
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "25", "-i", str(self.device)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def begin(self, wait_s=5.0):
        """Waits for the first sample (nvidia-smi takes a while to start), then
        marks the start of the timed region."""
        t_end = time.monotonic() + wait_s
        while self.proc and not self.lines and time.monotonic() < t_end:
            time.sleep(0.01)
        self.t0 = time.monotonic()

    def end(self):
        self.t1 = time.monotonic()
        t_end = self.t1 + 1.0   # one sample after the region, in case none fell inside it
        while self.proc and not any(t > self.t1 for t, _ in self.lines) and time.monotonic() < t_end:
            time.sleep(0.01)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        inside = [ln for t, ln in self.lines if self.t0 is not None and self.t0 <= t <= self.t1]
        if not inside and self.t1 is not None:
            inside = [ln for t, ln in self.lines if t > self.t1][:1]
        for ln in inside:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for n, flag in zip(names, p[5:9]):
                if flag.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm),
                "in_timed_region": bool(self.t0 is not None and any(self.t0 <= t <= self.t1 for t, _ in self.lines))}


def sample_pixels(width, height, row_stride, col_stride):
    ys, xs = np.meshgrid(np.arange(row_stride // 2, height, row_stride), np.arange(col_stride // 2, width, col_stride),
                         indexing="ij")
    return (ys * width + xs).ravel()


def host_cores():
    """Host cores this process may run on (its affinity mask)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=20).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return None


def time_oracle(sc, pixels, threads=1, want=("mboit", "exact", "nsamples")):
    """Runs the FP64 oracle on `pixels`: single-threaded as it stands
    (threads = 1), or its per-pixel entry on disjoint pixel chunks from a
    pool of `threads` host threads (ctypes releases the GIL during each call).
    Returns (results in pixel order, wall seconds)."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    if hasattr(sc, "cells"):
        sc = oracle.tet_scene_of(sc)  # the oracle's own split of mixed cells
    if threads <= 1:
        t0 = time.perf_counter()
        r = oracle.render(sc, pixels=pixels, want=want)
        return r, time.perf_counter() - t0
    chunks = [c for c in np.array_split(pixels, 8 * threads) if c.size]
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        parts = list(ex.map(lambda c: oracle.render(sc, pixels=c, want=want), chunks))
    dt = time.perf_counter() - t0
    return {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}, dt


def cpu_sample(v):
    """The bounded pixel sample of a view the CPU legs run: every 8th row and
    4th column above 512^2 pixels, else every pixel."""
    big = v.width * v.height > (1 << 18)
    return (sample_pixels(v.width, v.height, 8, 4) if big else sample_pixels(v.width, v.height, 1, 1),
            "every 8th row, 4th column" if big else "every pixel")


def workload(name):
    import scenes
    if name == "blobs512":
        return scenes.blobs512()
    if name == "blobs64":
        return scenes.blobs64()
    if name == "amr":
        return scenes.amr_blobs()
    if name == "tets":
        return scenes.tet_mesh()
    if name == "mixed":
        return scenes.mixed_mesh(n=64, n_pieces=72, width=1024, height=1024)
    raise SystemExit(f"unknown workload {name}")


def config_of(sc, name):
    v = sc.views[0]
    if hasattr(sc, "cells"):
        nc = np.bincount(sc.cell_types, minlength=7)
        return {"workload": name,
                "field": (f"mixed cells of a {int(sc.box[0])}^3 hex grid: {nc[4]} tets, {nc[5]} pyramids, {nc[6]} prisms "
                          f"({sc.verts.shape[0]} vertices), split into tets by the library, float32 vertex values"),
                "pieces": sc.n_pieces, "image": f"{v.width}x{v.height}",
                "projection": "perspective" if v.projection else "orthographic", "step_voxels": sc.step,
                "moments": "4 power, float32", "moment_bias": sc.moment_bias, "overestimation": sc.overestimation}
    if hasattr(sc, "tets"):
        return {"workload": name,
                "field": (f"tetrahedral mesh, {sc.tets.shape[0]} tets ({sc.verts.shape[0]} vertices, jittered "
                          f"{int(sc.box[0])}^3 hex grid, 5 tets per hex), float32 vertex values"),
                "pieces": sc.n_pieces, "image": f"{v.width}x{v.height}",
                "projection": "perspective" if v.projection else "orthographic", "step_voxels": sc.step,
                "moments": "4 power, float32", "moment_bias": sc.moment_bias, "overestimation": sc.overestimation,
                "l2": "mesh tables (~330 MB) larger than L2, re-read every frame"}
    if hasattr(sc, "leaves"):
        lv = np.bincount(sc.leaves[:, 3])
        field = (f"brick octree, {sc.leaves.shape[0]} leaves of 8^3 cells (per level {lv.tolist()}), "
                 f"{sc.leaves.shape[0] * 512 / 1e6:.1f} M cells, finest {sc.finest_cells}^3, float32")
    else:
        field = "x".join(str(n) for n in sc.dims) + " float32"
    return {"workload": name, "field": field,
            "pieces": sc.n_pieces, "brick_cells": 1 << sc.brick_log2, "image": f"{v.width}x{v.height}",
            "projection": "perspective" if v.projection else "orthographic", "step_voxels": sc.step,
            "moments": "4 power, float32", "moment_bias": sc.moment_bias, "overestimation": sc.overestimation,
            "l2": (lambda nb: f"inputs larger than L2 ({nb >> 20} MiB volume re-read every frame)" if nb > (129 << 20)
                   else f"volume of {nb >> 20} MiB fits in L2")((sc.values if hasattr(sc, 'leaves') else sc.field).nbytes),
            **({"step_rule": "adaptive dyadic (a level-L leaf samples every 2^(max_level - L)-th lattice point)"}
               if getattr(sc, "adaptive_step", False) else {})}


def run_reference(args, rank):
    """The reference arm: the FP64 oracle as it stands, on every host core
    (disjoint pixel chunks), on the bounded pixel sample of the workload."""
    if rank != 0:
        return
    sc = workload(args.workload)
    v = sc.views[0]
    pix, how = cpu_sample(v)
    cores = host_cores()
    for _ in range(args.warmup):
        time_oracle(sc, pix[: max(1, pix.size // 64)], cores)
    times, samples = [], 0
    for _ in range(args.steps):
        r, dt = time_oracle(sc, pix, cores, want=("mboit", "nsamples"))
        times.append(dt)
        samples = int(r["nsamples"].sum())
    total = sum(times)
    value = samples * args.steps / total / 1e9
    sample_desc = (f"{pix.size} pixels of the {v.width}x{v.height} frame ({how}), {samples} samples per step, "
                   f"FP64, {cores} threads over pixel chunks")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(config_of(sc, args.workload), parallelism="replicas" if args.gpus > 1 else "single"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample_desc,
                         "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def reduce_max(x, world, device):
    """The largest x over the ranks of the default process group (x itself
    for one rank): the whole-job time is the slowest replica's."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(samples_per_replica, world, ms_max):
    """Whole-job throughput of `world` replicas that each render the frame:
    every replica's samples over the slowest replica's frame time (Gsamples/s)."""
    return samples_per_replica * world / (ms_max * 1e-3) / 1e9


def pin_to_gpu_cpus(device):
    """Runs this process on the host cores next to the GPU (its PCI device's
    local CPU list), so that pinned host buffers land in the nearby memory;
    best effort, a no-op where the topology is not exposed."""
    try:
        bus = subprocess.run(["nvidia-smi", "--query-gpu=pci.bus_id", "--format=csv,noheader", "-i", str(device)],
                             capture_output=True, text=True, timeout=20).stdout.strip().lower()
        dom, rest = bus.split(":", 1)
        path = f"/sys/bus/pci/devices/{dom[-4:]}:{rest}/local_cpulist"
        cpus = set()
        for part in open(path).read().strip().split(","):
            a, _, b = part.partition("-")
            cpus.update(range(int(a), int(b or a) + 1))
        if cpus:
            os.sched_setaffinity(0, cpus)
    except (OSError, ValueError, subprocess.SubprocessError):
        pass


def profile_moment_set(args):
    """Frames of the workload with another moment set and storage (the biases of
    the precision sweep), for a profiler: autotune, warm-up, timed frames."""
    import torch
    import paper_2501_12581_gb300 as pkg
    mset, stor = (args.moment_set.split(":") + ["f32"])[:2]
    beta = {"f32": 5e-5, "f16": 2e-3, "bf16": 2e-2}[stor]
    sc = workload(args.workload)
    if args.image:
        for vw in sc.views:
            vw.width = vw.height = args.image
    sc.moment_set, sc.storage, sc.moment_bias = mset, stor, beta
    vol = pkg.Volume(sc)
    views = sc.views
    mom, rgba = vol.moments_for(views), pkg.Volume.color_buffer(views)
    vol.autotune(views, mom, rgba)
    for _ in range(args.warmup):
        vol.render_frame(views, mom, rgba)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(args.steps):
        vol.render_frame(views, mom, rgba)
    ev1.record()
    torch.cuda.synchronize()
    vol.synchronize()
    st = vol.stats()
    print(json.dumps({"workload": args.workload, "moments": mset, "storage": stor, "moment_bias": beta,
                      "image": f"{views[0].width}x{views[0].height}", "samples_per_frame": st["samples_pass1"],
                      "ms_per_frame": ev0.elapsed_time(ev1) / args.steps, "frame_pass1_ms": st["frame_pass1_ms"],
                      "frame_pass2_ms": st["frame_pass2_ms"]}))
    vol.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="amr", choices=["blobs512", "blobs64", "amr", "tets", "mixed"])
    ap.add_argument("--image", type=int, default=0, help="square image size for the main workload (profiling)")
    ap.add_argument("--adaptive", action="store_true", help="octree workload: the adaptive dyadic step")
    ap.add_argument("--no-amr", action="store_true", help="skip the adaptive-step octree frame")
    ap.add_argument("--no-grid", action="store_true", help="skip the 512^3 regular-grid workload")
    ap.add_argument("--no-tets", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-per-piece", action="store_true")
    ap.add_argument("--no-sortlast", action="store_true")
    ap.add_argument("--no-gear", action="store_true", help="skip the gear-teeth stress test")
    ap.add_argument("--no-multi", action="store_true", help="skip the multi-volume frame")
    ap.add_argument("--no-fp64-setup", action="store_true", help="skip the frame with every pixel set up in FP64")
    ap.add_argument("--no-orbit", action="store_true", help="skip the four-camera orbits (octree and 512^3 grid)")
    ap.add_argument("--gear-k", default="8,16,32,64,128", help="piece counts of the gear-teeth stress test")
    ap.add_argument("--heatmap", default="", help="directory for the gear-teeth segments-per-pixel images (PGM)")
    ap.add_argument("--moment-set", default="", metavar="SET:STORAGE",
                    help="profiling only: frames of --workload with another moment set (power6:f32, power8:f32, "
                         "trig6:f16, trig8:bf16, ...); prints their time, not the benchmark line")
    ap.add_argument("--ncu-record", nargs=4, metavar=("CSV", "KERNEL", "SAMPLES", "OUT"),
                    help="write the frame kernel's ncu record for --workload from a raw CSV dump and exit")
    args = ap.parse_args()
    if args.ncu_record:
        csv_path, kernel, nsamp, out_path = args.ncu_record
        print(json.dumps(write_ncu_record(csv_path, kernel, args.workload, int(nsamp), out_path)))
        return
    args.warmup = max(args.warmup, 3)
    if args.moment_set:
        profile_moment_set(args)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import torch.distributed as dist
    import __graft_entry__
    import paper_2501_12581_gb300 as pkg

    torch.cuda.set_device(local)
    pin_to_gpu_cpus(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    __graft_entry__.build()

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x):
        return reduce_max(x, world, "cuda")

    sc = workload(args.workload)
    if args.adaptive:
        assert hasattr(sc, "leaves"), "--adaptive applies to the octree workload"
        sc.adaptive_step = True
    if args.image:
        for vw in sc.views:
            assert vw.width == vw.height, "--image rescales square views only"
            vw.width = vw.height = args.image
    vol = pkg.Volume(sc)
    views = sc.views
    v = views[0]
    mom = pkg.Volume.moment_buffer(views)
    rgba = pkg.Volume.color_buffer(views)
    stream = torch.cuda.current_stream()

    def timed(fn, steps):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(steps):
            fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return ev0.elapsed_time(ev1) / steps

    tuning = vol.autotune(views, mom, rgba)   # outside the timed region
    frame = lambda: vol.render_frame(views, mom, rgba)  # noqa: E731
    for _ in range(args.warmup):
        frame()
    vol.synchronize()
    with ClockSampler(local) as clk:
        clk.begin()
        ms = timed(frame, args.steps)
        clk.end()
    vol.synchronize()
    st = vol.stats()
    samples = st["samples_pass1"]
    ms_max = max_over_ranks(ms)
    value = job_rate(samples, world, ms_max)

    # the frame's kernels (one or two): CUDA events recorded inside its graph, on
    # the launching stream, averaged over a few frames
    p1 = p2 = 0.0
    nf = max(5, args.steps // 2)
    for _ in range(nf):
        frame()
        stf = vol.stats()
        p1 += stf["frame_pass1_ms"] / nf
        p2 += stf["frame_pass2_ms"] / nf
    # the same passes as separate calls (pass 2 marches the field again)
    for _ in range(3):
        vol.render_moments(views, mom)
        vol.reconstruct_blend(views, mom, rgba, mode=pkg.MBOIT_COLOR_RESOLVED)
    k = max(5, args.steps // 2)
    ms_p1 = timed(lambda: vol.render_moments(views, mom), k)
    ms_p2 = timed(lambda: vol.reconstruct_blend(views, mom, rgba, mode=pkg.MBOIT_COLOR_RESOLVED), k)
    vol.synchronize()
    frame()
    vol.synchronize()
    hbm = MEASURED.get("hbm_gbs")

    def kstats(ms_k, flop, cache_bytes):
        d = {"launch_ms": ms_k, "flop_per_sample": flop, "achieved_tflops": flop * samples / (ms_k * 1e-3) / 1e12,
             "cache_bytes_per_sample": cache_bytes, "cache_gbs": cache_bytes * samples / (ms_k * 1e-3) / 1e9}
        d["alu_frac"] = d["achieved_tflops"] / FP32_PEAK_TFLOPS
        if hbm:
            d["hbm_frac_of_measured"] = d["cache_gbs"] / hbm
        return d
    launches = stf["frame_launches"]
    unit_scene = hasattr(sc, "leaves") or hasattr(sc, "tets") or hasattr(sc, "cells")
    flop1 = FLOP_PASS1["amr" if hasattr(sc, "leaves") else "grid"]
    if launches == 1:
        # one kernel per frame: the event pair brackets it, the second pair is empty
        k1s = kstats(p1 + p2, flop1 + FLOP_PASS2_FRAME, 2 * CACHE_BYTES_PER_SAMPLE)
        frame_kernels = {"frame_one_launch": k1s}
        dom_key = "k_frame_unit" if unit_scene else "k_frame_fused"
        dom, dflop = k1s, flop1 + FLOP_PASS2_FRAME
        dmufu = MUFU_PASS1 + MUFU_PASS2
        dname = (dom_key + ", one launch per frame (per ray tile: march + moments + sample store, "
                 "then reconstruct + blend + resolve)")
    else:
        k1s = kstats(p1, flop1, CACHE_BYTES_PER_SAMPLE)
        k2s = kstats(p2, FLOP_PASS2_FRAME, CACHE_BYTES_PER_SAMPLE)
        frame_kernels = {"frame_pass1": k1s, "frame_pass2": k2s}
        kname = "k_pass{}_unit" if unit_scene else "k_pass{}_fused"
        dom, dname, dflop = (k2s, kname.format(2) + ", frame form (reads the cached samples; reconstruct + blend + resolve)",
                             FLOP_PASS2_FRAME) if p2 >= p1 else \
            (k1s, kname.format(1) + ", frame form (march + moments + sample store)", flop1)
        dom_key = kname.format(2 if p2 >= p1 else 1) + "_frame"
        dmufu = MUFU_PASS2 if p2 >= p1 else MUFU_PASS1
    rec_traffic = measured_traffic(dom_key, args.workload)
    ncu_rec = measured_ncu(dom_key, args.workload)
    # a record taken on a reduced view scales to this launch by its owned samples
    traffic = None
    if rec_traffic is not None:
        traffic = int(rec_traffic * (samples / ncu_rec["samples_per_launch"] if "samples_per_launch" in ncu_rec else 1.0))
    roofline = {"bound": "alu", "kernel": dname, "achieved": dom["achieved_tflops"], "peak": FP32_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": dom["achieved_tflops"] / FP32_PEAK_TFLOPS, "traffic": traffic,
                "traffic_source": None if ncu_rec is None else
                ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch"
                 + (f" on {int(ncu_rec['samples_per_launch'])} owned samples, scaled by owned samples"
                    if "samples_per_launch" in ncu_rec else "")),
                "binding_units_ncu": None if ncu_rec is None else
                {k: v for k, v in ncu_rec.items() if k != "dram_bytes_per_launch"},
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz", "flop_per_sample": dflop,
                "launch_ms": dom["launch_ms"], **frame_kernels,
                "split_calls": {"pass1_ms": ms_p1, "pass2_ms": ms_p2, "pass2_flop_per_sample": FLOP_PASS2,
                                "pass2_achieved_tflops": FLOP_PASS2 * samples / (ms_p2 * 1e-3) / 1e12}}
    if traffic is not None and hbm:
        roofline["hbm"] = {"traffic_gbs": traffic / (dom["launch_ms"] * 1e-3) / 1e9, "peak_gbs": hbm,
                           "frac_of_measured": traffic / (dom["launch_ms"] * 1e-3) / 1e9 / hbm}
    roofline["roofs"] = roofs_of(samples, dom["launch_ms"], dflop, dmufu, traffic, hbm, ncu_rec)

    # end to end through the host API: field upload, frame, image download
    host_values = (sc.values if hasattr(sc, "leaves") else sc.verts[:, 3] if (hasattr(sc, "tets") or hasattr(sc, "cells"))
                   else sc.field)
    field_host = torch.from_numpy(np.ascontiguousarray(host_values, dtype=np.float32)).pin_memory()
    rgba_host = torch.empty(rgba.numel(), dtype=torch.float32).pin_memory()
    e2e_step = lambda: pkg.mboit_render_frame_host(vol.handle, field_host, views, mom, rgba, rgba_host)  # noqa: E731
    e2e_step()
    t0 = time.perf_counter()
    barrier()
    for _ in range(max(3, args.steps // 3)):
        e2e_step()
    barrier()
    e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / max(3, args.steps // 3))
    e2e = {"value": samples * world / (e2e_ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": e2e_ms,
           "h2d_bytes_per_step": int(field_host.numel() * 4), "d2h_bytes_per_step": int(rgba_host.numel() * 4)}

    # the plain per-piece FP32 form (one launch per piece and pass, K images summed)
    per_piece = None
    if not args.no_per_piece:
        K = sc.n_pieces
        per_m = pkg.Volume.moment_buffer(views, K)
        per_c = pkg.Volume.color_buffer(views, K)
        glob = pkg.Volume.moment_buffer(views)

        def plain():
            vol.render_moments(views, per_m, mode=pkg.MBOIT_MOMENTS_PER_PIECE)
            vol.composite(pkg.MBOIT_OP_MOMENTS_SUM, v.width, v.height, 1, K, per_m, glob)
            vol.reconstruct_blend(views, glob, per_c, mode=pkg.MBOIT_COLOR_PER_PIECE)
            vol.composite(pkg.MBOIT_OP_COLOR_SUM_RESOLVE, v.width, v.height, 1, K, per_c, rgba, glob)
        plain()
        ms_pp = timed(plain, max(3, args.steps // 6))
        vol.synchronize()
        per_piece = {"ms_per_frame": ms_pp, "gsamples_per_s": samples / (ms_pp * 1e-3) / 1e9,
                     "launches_per_frame": 2 * K + 2, "speedup_of_batched": ms_pp / ms}
        del per_m, per_c, glob
        torch.cuda.empty_cache()
        frame()

    # the on-GPU exact sort-last baseline (segment layers) and the MBOIT error against it
    sortlast = None
    if not args.no_sortlast:
        exact = pkg.Volume.color_buffer(views)
        vol.render_sortlast(views, exact)
        ms_sl = timed(lambda: vol.render_sortlast(views, exact), max(3, args.steps // 6))
        frame()
        vol.synchronize()
        d = (rgba - exact).view(-1, 4).double()
        st_sl = vol.stats()
        sortlast = {"ms_per_frame": ms_sl, "gsamples_per_s": samples / (ms_sl * 1e-3) / 1e9,
                    "segments": st_sl["sortlast_segments"], "max_segments_per_pixel": st_sl["sortlast_max_segments"],
                    "speedup_of_batched_mboit": ms_sl / ms,
                    "mboit_vs_exact_rmse": float(d.pow(2).mean().sqrt()), "mboit_vs_exact_max": float(d.abs().max())}
        del exact
        torch.cuda.empty_cache()

    # the 512^3 regular grid (64 pieces, 2048x2048), the 72-piece tetrahedral
    # A volume seen from four cameras on an orbit about its z axis (the
    # benchmark camera's direction (0.57, 0.49, 0.66) turned by 0, 90, 180 and
    # 270 degrees; same elevation, distance and field of view), with the tuning
    # the volume already has: one frame graph per camera; the frame rate's
    # spread over the orbit.
    def orbit_of(ovol, dims, width, height, om, orgba):
        import scenes as _scenes
        w0 = (0.57, 0.49, 0.66)
        cams, rates, mss, ns = [], [], [], []
        for deg in (0, 90, 180, 270):
            c_, s_ = np.cos(np.radians(deg)), np.sin(np.radians(deg))
            wd = (c_ * w0[0] - s_ * w0[1], s_ * w0[0] + c_ * w0[1], w0[2])
            ov = [_scenes.perspective_view(dims, wd, width, height)]
            of = lambda: ovol.render_frame(ov, om, orgba)  # noqa: E731,B023
            for _ in range(3):
                of()
            ms_o = timed(of, max(5, args.steps // 3))
            of()
            ovol.synchronize()
            so = ovol.stats()["samples_pass1"]
            cams.append(deg)
            mss.append(ms_o)
            ns.append(so)
            rates.append(so / (ms_o * 1e-3) / 1e9)
        return {"azimuth_deg": cams, "ms_per_frame": mss, "samples_per_frame": ns, "gsamples_per_s": rates,
                "mean_gsamples_per_s": float(np.mean(rates)), "min_gsamples_per_s": float(min(rates)),
                "max_gsamples_per_s": float(max(rates)), "mean_ms_per_frame": float(np.mean(mss))}

    # (1024x1024) and mixed-cell workloads as further lines of results
    def unit_block(name):
        usc = workload(name)
        uvol = pkg.Volume(usc)
        uv = usc.views
        umom, urgba = pkg.Volume.moment_buffer(uv), pkg.Volume.color_buffer(uv)
        utune = uvol.autotune(uv, umom, urgba)   # the ray packet (one window configuration here)
        uframe = lambda: uvol.render_frame(uv, umom, urgba)  # noqa: E731
        for _ in range(3):
            uframe()
        ms_u = timed(uframe, max(3, args.steps // 3))
        uvol.synchronize()
        su = uvol.stats()["samples_pass1"]
        K = usc.n_pieces
        pm, pc, gm = pkg.Volume.moment_buffer(uv, K), pkg.Volume.color_buffer(uv, K), pkg.Volume.moment_buffer(uv)
        uw, uh = uv[0].width, uv[0].height

        def uplain():
            uvol.render_moments(uv, pm, mode=pkg.MBOIT_MOMENTS_PER_PIECE)
            uvol.composite(pkg.MBOIT_OP_MOMENTS_SUM, uw, uh, 1, K, pm, gm)
            uvol.reconstruct_blend(uv, gm, pc, mode=pkg.MBOIT_COLOR_PER_PIECE)
            uvol.composite(pkg.MBOIT_OP_COLOR_SUM_RESOLVE, uw, uh, 1, K, pc, urgba, gm)
        uplain()
        ms_up = timed(uplain, 3)
        del pm, pc, gm
        torch.cuda.empty_cache()
        usl = None
        if not args.no_sortlast:
            uexact = pkg.Volume.color_buffer(uv)
            uvol.render_sortlast(uv, uexact)
            ms_usl = timed(lambda: uvol.render_sortlast(uv, uexact), 3)
            uframe()
            uvol.synchronize()
            dd = (urgba - uexact).view(-1, 4).double()
            stu = uvol.stats()
            usl = {"ms_per_frame": ms_usl, "segments": stu["sortlast_segments"],
                   "max_segments_per_pixel": stu["sortlast_max_segments"], "speedup_of_batched_mboit": ms_usl / ms_u,
                   "mboit_vs_exact_rmse": float(dd.pow(2).mean().sqrt()), "mboit_vs_exact_max": float(dd.abs().max())}
            del uexact, dd
            torch.cuda.empty_cache()
        uframe()
        uvol.synchronize()
        out_u = {"config": dict(config_of(usc, name), packet="4x8" if utune[2] == pkg.MBOIT_PACKET_4X8 else "8x4"),
                 "samples_per_frame": su, "ms_per_frame": ms_u,
                 "gsamples_per_s": su / (ms_u * 1e-3) / 1e9, "per_piece_fp32_ms_per_frame": ms_up,
                 "speedup_of_batched": ms_up / ms_u, "sortlast_gpu": usl}
        if name == "blobs512" and not args.no_orbit:
            out_u["orbit_4_cameras"] = orbit_of(uvol, usc.dims, uw, uh, umom, urgba)
            uframe()
            uvol.synchronize()
        upix = sample_pixels(uw, uh, 64, 32)
        if rank == 0 and not args.no_cpu_baseline:
            _orc = __import__("oracle")
            oscene = _orc.tet_scene_of(usc) if hasattr(usc, "cells") else usc
            r, _ = time_oracle(oscene, upix, host_cores(), want=("mboit",))
            ref = r["mboit"]
            got = urgba.view(-1, 4)[torch.from_numpy(upix).cuda()].double().cpu().numpy()
            out_u["quality"] = {"pixels": int(upix.size), "max_abs_vs_oracle": float(np.abs(got - ref).max()),
                                "rmse_vs_oracle": float(np.sqrt(((got - ref) ** 2).mean()))}
        uvol.close()
        del uvol, umom, urgba
        torch.cuda.empty_cache()
        return out_u

    # the octree workload with the adaptive dyadic step (a level-L leaf samples
    # every 2^(max_level - L)-th lattice point, each sample over that interval)
    def adaptive_block(usc, upix, ms_fixed, samples_fixed, fixed_exact):
        import copy
        asc = copy.copy(usc)
        asc.adaptive_step = True
        avol = pkg.Volume(asc)
        av = asc.views
        amom, argba = pkg.Volume.moment_buffer(av), pkg.Volume.color_buffer(av)
        atune = avol.autotune(av, amom, argba)
        aframe = lambda: avol.render_frame(av, amom, argba)  # noqa: E731
        for _ in range(3):
            aframe()
        ms_a = timed(aframe, max(3, args.steps // 3))
        avol.synchronize()
        sa = avol.stats()["samples_pass1"]
        out_a = {"packet": "4x8" if atune[2] == pkg.MBOIT_PACKET_4X8 else "8x4", "samples_per_frame": sa,
                 "sample_fraction_of_fixed_step": sa / samples_fixed, "ms_per_frame": ms_a,
                 "gsamples_per_s": sa / (ms_a * 1e-3) / 1e9,
                 "fixed_step_lattice_gsamples_per_s": samples_fixed / (ms_a * 1e-3) / 1e9,
                 "speedup_of_fixed_step_frame": ms_fixed / ms_a}
        if rank == 0 and not args.no_cpu_baseline:
            r, _ = time_oracle(asc, upix, host_cores(), want=("mboit", "exact"))
            got = argba.view(-1, 4)[torch.from_numpy(upix).cuda()].double().cpu().numpy()
            out_a["quality"] = {"pixels": int(upix.size),
                                "max_abs_vs_oracle": float(np.abs(got - r["mboit"]).max()),
                                "rmse_vs_oracle": float(np.sqrt(((got - r["mboit"]) ** 2).mean())),
                                "rmse_vs_fixed_step_exact": float(np.sqrt(((got - fixed_exact) ** 2).mean())),
                                "exact_adaptive_vs_exact_fixed_rmse":
                                    float(np.sqrt(((r["exact"] - fixed_exact) ** 2).mean()))}
        avol.close()
        del avol, amom, argba
        torch.cuda.empty_cache()
        return out_a

    headline = args.workload == "amr" and not args.image
    grid = unit_block("blobs512") if headline and not args.no_grid else None
    tets = unit_block("tets") if headline and not args.no_tets else None
    mixed = unit_block("mixed") if headline and not args.no_tets else None

    # the headline frame with every pixel's reconstruction frame set up in FP64
    # (MBOIT_FLAG_FP64_SETUP), the same tuning, against the float-float set-up
    fp64_setup = None
    if headline and not args.no_fp64_setup:
        st0 = vol.stats()
        v64 = pkg.Volume(sc, flags=pkg.MBOIT_FLAG_FP64_SETUP)
        v64.set_tuning(st0["tuning_pass1"], st0["tuning_pass2"])
        v64.set_packet(st0["packet"])
        v64.set_frame_launches(st0["frame_launches"])
        v64.set_tile_order(st0["tile_order"])
        f64 = lambda: v64.render_frame(views, mom, rgba)  # noqa: E731
        for _ in range(3):
            f64()
        ms64 = timed(f64, max(5, args.steps // 3))
        v64.synchronize()
        s64 = v64.stats()
        fp64_setup = {"ms_per_frame": ms64, "fp64_pixels": s64["fp64_pixels"],
                      "float_float_ms_per_frame": ms_max, "float_float_fp64_pixels": st0["fp64_pixels"],
                      "time_ratio": ms64 / ms_max}
        v64.close()
        del v64
        torch.cuda.empty_cache()

    orbit = orbit_of(vol, sc.dims, v.width, v.height, mom, rgba) if headline and not args.no_orbit else None
    vol.render_frame(views, mom, rgba)
    vol.synchronize()

    # several independent volumes in one persistent launch per pass: 8 grids
    # of 64^3 (the blobs64 field flipped and scaled per volume, one transfer
    # function), one 256^2 view each, against 8 single-volume frames
    multi = None
    if headline and not args.no_multi:
        import dataclasses
        import scenes as _scenes
        base = _scenes.blobs64()
        mscs = []
        for i in range(8):
            f = np.ascontiguousarray(np.flip(base.field, axis=i % 3) * np.float32(1.0 - 0.05 * i)).astype(np.float32)
            mscs.append(dataclasses.replace(base, name=f"blobs64_{i}", field=f,
                                            tf_range=(np.float32(f.min()), np.float32(f.max()))))
        mvols = [pkg.Volume(s_) for s_ in mscs]
        mviews = [_scenes.ortho_view(base.dims, (0.62 - 0.05 * i, 0.48, 0.62), 256, 256) for i in range(8)]
        mmom, mrgba = pkg.Volume.moment_buffer(mviews), pkg.Volume.color_buffer(mviews)
        owner = list(range(8))
        mframe = lambda: pkg.Volume.render_frame_multi(mvols, mviews, owner, mmom, mrgba)  # noqa: E731
        singles = [(mv, [vw], pkg.Volume.moment_buffer([vw]), pkg.Volume.color_buffer([vw]))
                   for mv, vw in zip(mvols, mviews)]

        def sframes():
            for mv, vw, m_, c_ in singles:
                mv.render_frame(vw, m_, c_)
        for _ in range(3):
            mframe()
            sframes()
        ms_m = timed(mframe, 20)
        ms_s = timed(sframes, 20)
        mframe()
        mvols[0].synchronize()
        sm = mvols[0].stats()["samples_pass1"]
        multi = {"volumes": 8, "field": "64x64x64 float32 each", "image": "256x256 per volume",
                 "samples_per_frame": sm, "multi_ms_per_frame": ms_m, "multi_gsamples_per_s": sm / (ms_m * 1e-3) / 1e9,
                 "launches_per_frame": 2, "single_volume_frames_ms": ms_s,
                 "single_volume_launches": sum(1 if mv.stats()["frame_launches"] == 1 else 2 for mv in mvols),
                 "speedup_of_one_launch_per_pass": ms_s / ms_m}
        for mv in mvols:
            mv.close()
        del mvols, singles, mmom, mrgba
        torch.cuda.empty_cache()
        # four brick octrees (the headline octree at a quarter of its base, its
        # leaf values scaled per volume), one 512^2 view each
        abase = _scenes.amr_blobs(width=512, height=512, n_pieces=8, base=8, max_level=2)
        oscs = []
        for i in range(4):
            vals = np.ascontiguousarray(abase.values * np.float32(1.0 - 0.1 * i)).astype(np.float32)
            oscs.append(dataclasses.replace(abase, name=f"amr_blobs8_{i}", values=vals,
                                            tf_range=(np.float32(vals.min()), np.float32(vals.max()))))
        ovols = [pkg.Volume(s_) for s_ in oscs]
        oviews = [_scenes.perspective_view(abase.dims, (0.57 - 0.1 * i, 0.49, 0.66), 512, 512) for i in range(4)]
        omom, orgba = pkg.Volume.moment_buffer(oviews), pkg.Volume.color_buffer(oviews)
        oframe = lambda: pkg.Volume.render_frame_multi(ovols, oviews, list(range(4)), omom, orgba)  # noqa: E731
        osingles = [(ov, [vw], pkg.Volume.moment_buffer([vw]), pkg.Volume.color_buffer([vw]))
                    for ov, vw in zip(ovols, oviews)]

        def oframes():
            for ov, vw, m_, c_ in osingles:
                ov.render_frame(vw, m_, c_)
        for _ in range(3):
            oframe()
            oframes()
        ms_om = timed(oframe, 10)
        ms_os = timed(oframes, 10)
        oframe()
        ovols[0].synchronize()
        som = ovols[0].stats()["samples_pass1"]
        multi["octrees"] = {"volumes": 4, "leaves": int(len(abase.leaves)), "image": "512x512 per volume",
                            "samples_per_frame": som, "multi_ms_per_frame": ms_om,
                            "multi_gsamples_per_s": som / (ms_om * 1e-3) / 1e9, "single_volume_frames_ms": ms_os,
                            "speedup_of_one_launch_per_pass": ms_os / ms_om}
        for ov in ovols:
            ov.close()
        del ovols, osingles, omom, orgba
        torch.cuda.empty_cache()

    # the gear-teeth stress test of Sec. 5: K pieces of 4 interleaved layers,
    # batched MBOIT against the exact sort-last baseline as K grows
    gear = None
    if headline and not args.no_gear:
        import scenes as _scenes
        gear = []
        for K in [int(x) for x in args.gear_k.split(",") if x]:
            gsc = _scenes.gear_teeth(n_pieces=K)
            gvol = pkg.Volume(gsc)
            gv = gsc.views
            gmom, grgba = gvol.moments_for(gv), pkg.Volume.color_buffer(gv)
            gframe = lambda: gvol.render_frame(gv, gmom, grgba)  # noqa: E731
            for _ in range(2):
                gframe()
            ms_g = timed(gframe, 3)
            gvol.synchronize()
            sg = gvol.stats()["samples_pass1"]
            row = {"pieces": K, "layers": 4 * K, "field": "x".join(str(n) for n in gsc.dims) + " float32",
                   "views": len(gv), "image": f"{gv[0].width}x{gv[0].height} per view", "samples_per_frame": sg,
                   "mboit_ms_per_frame": ms_g, "mboit_gsamples_per_s": sg / (ms_g * 1e-3) / 1e9}
            if not args.no_sortlast:
                gex = pkg.Volume.color_buffer(gv)
                segs = torch.zeros(sum(v.width * v.height for v in gv), dtype=torch.int32, device="cuda")
                gvol.render_sortlast(gv, gex, segs)
                ms_sl = timed(lambda: gvol.render_sortlast(gv, gex, segs), 1)
                gframe()
                gvol.synchronize()
                sn = segs.cpu().numpy()
                hit = sn[sn > 0]
                d = (grgba - gex).view(-1, 4).double()
                row.update({"sortlast_ms_per_frame": ms_sl, "speedup_of_batched_mboit": ms_sl / ms_g,
                            "segments_per_hit_pixel_mean": float(hit.mean()) if hit.size else 0.0,
                            "segments_per_pixel_max": int(sn.max()),
                            "segments_histogram": {"bin_edges": np.linspace(0, 4 * K, 9).tolist(),
                                                   "pixels": np.histogram(sn, bins=8, range=(0, 4 * K))[0].tolist()},
                            "mboit_vs_exact_rmse": float(d.pow(2).mean().sqrt())})
                if args.heatmap:
                    os.makedirs(args.heatmap, exist_ok=True)
                    off = 0
                    for i, gview in enumerate(gv):
                        w_, h_ = gview.width, gview.height
                        img = sn[off:off + w_ * h_].reshape(h_, w_)
                        off += w_ * h_
                        with open(os.path.join(args.heatmap, f"gear_teeth{K}_view{i}_segments.pgm"), "wb") as fh:
                            fh.write(f"P5 {w_} {h_} 255\n".encode())
                            fh.write(np.clip(img * 255.0 / (4 * K), 0, 255).astype(np.uint8).tobytes())
                del gex, segs
            gear.append(row)
            gvol.close()
            del gvol, gmom, grgba
            torch.cuda.empty_cache()

    # precision sweep on the octree field with the 2048^2 view: moment sets and storages
    sweep = None
    if headline and not args.no_sweep:
        import copy
        import scenes as _scenes
        import oracle as _oracle
        base = workload("amr")
        base.views = [_scenes.perspective_view(base.dims, (0.57, 0.49, 0.66), 2048, 2048)]
        spix = sample_pixels(2048, 2048, 64, 32)
        sweep = []
        exact_ref = None
        for mset, stor, beta in (("power4", "f32", 5e-5), ("power6", "f32", 5e-5), ("power8", "f32", 5e-5),
                             ("trig6", "f16", 2e-3), ("trig6", "bf16", 2e-2), ("trig8", "f16", 2e-3),
                             ("trig8", "bf16", 2e-2)):
            sc2 = copy.copy(base)
            sc2.moment_set, sc2.storage, sc2.moment_bias = mset, stor, beta
            svol = pkg.Volume(sc2)
            sv = sc2.views
            smom, srgba = svol.moments_for(sv), pkg.Volume.color_buffer(sv)
            sframe = lambda: svol.render_frame(sv, smom, srgba)  # noqa: E731
            for _ in range(2):
                sframe()
            ms_s = timed(sframe, 3)
            svol.synchronize()
            ns = svol.stats()["samples_pass1"]
            row = {"moments": mset, "storage": stor, "moment_bias": beta,
                   "moment_bytes_per_pixel": pkg.mboit_moment_image_bytes(4, 1, svol.moment_set, svol.storage) // 4,
                   "ms_per_frame": ms_s, "gsamples_per_s": ns / (ms_s * 1e-3) / 1e9}
            if rank == 0 and not args.no_cpu_baseline:
                ref = _oracle.render_amr(sc2, pixels=spix, want=("mboit", "exact") if exact_ref is None else ("mboit",))
                if exact_ref is None:
                    exact_ref = ref["exact"]
                got = srgba.view(-1, 4)[torch.from_numpy(spix).cuda()].double().cpu().numpy()
                row.update({"max_abs_vs_oracle": float(np.abs(got - ref["mboit"]).max()),
                            "rmse_vs_oracle": float(np.sqrt(((got - ref["mboit"]) ** 2).mean())),
                            "rmse_vs_exact": float(np.sqrt(((got - exact_ref) ** 2).mean())),
                            "max_abs_vs_exact": float(np.abs(got - exact_ref).max()),
                            "pixels": int(spix.size)})
            sweep.append(row)
            svol.close()
            del svol, smom, srgba
            torch.cuda.empty_cache()


    # parity on a pixel sample and the oracle's own speed (rank 0, one GPU):
    # the FP64 oracle single-threaded as it stands, and its per-pixel entry on
    # disjoint pixel chunks over every host core
    cpu_baseline, quality, adaptive = None, None, None
    if rank == 0 and not args.no_cpu_baseline:
        frame()
        vol.synchronize()
        v0 = sc.views[0]
        pix, how = cpu_sample(v0)
        cores = host_cores()
        r, dt_all = time_oracle(sc, pix, cores)
        one = pix[:: max(1, pix.size // 16384)]   # the single-thread leg on a 1/N subset of the sample
        r1, dt1 = time_oracle(sc, one, 1, want=("nsamples",))
        ns = int(r["nsamples"].sum())
        ns1 = int(r1["nsamples"].sum())
        got = rgba.view(-1, 4)[torch.from_numpy(pix).cuda()].double().cpu().numpy()
        d = got - r["mboit"]
        quality = {"pixels": int(pix.size), "max_abs_vs_oracle": float(np.abs(d).max()),
                   "rmse_vs_oracle": float(np.sqrt((d ** 2).mean())),
                   "oracle_mboit_vs_exact_rmse": float(np.sqrt(((r["mboit"] - r["exact"]) ** 2).mean())),
                   "oracle_mboit_vs_exact_max": float(np.abs(r["mboit"] - r["exact"]).max())}
        rate = ns / dt_all / 1e9
        cpu_baseline = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
                        "sample": (f"{pix.size} pixels ({how}) of the {v0.width}x{v0.height} frame, {ns} samples, "
                                   f"{dt_all:.2f} s, FP64, {cores} threads over pixel chunks"),
                        "frame_s_extrapolated": samples / (rate * 1e9),
                        "single_thread": {"value": ns1 / dt1 / 1e9, "unit": UNIT, "cores": 1,
                                          "sample": f"{one.size} pixels (every {pix.size // one.size}th of the sample), "
                                                    f"{ns1} samples, {dt1:.2f} s"}}
        if hasattr(sc, "leaves") and not args.no_amr and not args.image:
            adaptive = adaptive_block(sc, pix, ms, samples, r["exact"])

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": dict(config_of(sc, args.workload), parallelism="replicas" if world > 1 else "single"),
           "form": ("batched: 1 persistent kernel per frame (pass 1 then pass 2 per ray tile), CUDA graph"
                    if launches == 1 else "batched: 2 persistent kernels per frame, CUDA graph"),
           "tuning": {"pass1": tuning[0], "pass2": tuning[1],
                      "packet": "4x8" if tuning[2] == pkg.MBOIT_PACKET_4X8 else "8x4", "frame_launches": launches,
                      "tile_order": "longest first" if stf["tile_order"] else "raster"},
           "samples_per_frame": samples, "ms_per_frame": ms_max, "singular_pixels": st["singular_pixels"],
           "fp64_setup_pixels": st["fp64_pixels"],
           "per_piece_fp32": per_piece, "sortlast_gpu": sortlast, "adaptive_step": adaptive,
           "grid_512_64_pieces": grid, "tets_72_pieces": tets, "mixed_cells_72_pieces": mixed,
           "gear_teeth_stress": gear,
           "multi_volume_8_grids": multi,
           "fp64_setup_every_pixel": fp64_setup,
           "orbit_4_cameras": orbit,
           "precision_sweep_amr_2048": sweep,
           "quality": quality, "roofline": roofline, "cpu_baseline": cpu_baseline, "e2e": e2e,
           "gpu_launches": launches * args.steps, "clocks": clk.summary()}
    vol.close()
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
