"""Benchmark of the Wilson-clover hot path on GB300.

Workload: the 48^3 x 96 lattice (nT = 96, nZ = nY = nX = 48; 10,616,832
sites), synthetic SU(3) links exp(i 0.3 H), m0 = -0.4, c_sw = 1.0,
antiperiodic time, one Gaussian right-hand side.

Headline metric: algorithmic HBM GB/s of one D psi application (Eq. 1.13)
in the chosen precision (default FP32), inputs resident in HBM, native
layout.  One step = one full-lattice D psi.  The working set (links,
self coupling, spinors: > 8 GB) is far larger than the 129 MB L2, so no
flush is needed between steps.

Algorithmic bytes per site for N right-hand sides (every link, clover
block and spinor read once, the result written once):
  FP64 1152 + 384 N,  FP32 576 + 192 N (480 + 192 for one RHS when the
  library reads two-row FP32 links, which it does for SU(3) links),
  FP16 storage 288 + 104 N.

The JSON line also carries:
  variants    GB/s of the FP64, FP32 and FP16-storage applies, each with its
              binding roof (FP64 is bound by the FP64 pipeline on this GPU);
  e2e         the same apply through the C ABI on host buffers, copies
              included;
  solve       time to ||b - D x|| < 1e-10 ||b|| of the mixed-precision
              even-odd FGMRES with FP64 refinement against the plain FP64 GPU
              solve;
  roofline    the headline kernel against the measured HBM copy bandwidth;
  cpu_baseline the CPU oracle on a bounded sample of the same workload.

--impl reference times the CPU oracle instead (each step: D psi on a
bounded sample of sites of the same lattice).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DIMS = (96, 48, 48, 48)  # nT, nZ, nY, nX
M0, CSW, EPS = -0.4, 1.0, 0.3
WORKLOAD = "48^3x96 Wilson-clover D.psi, 1 RHS, eps=0.3 SU(3) links, m0=-0.4, c_sw=1.0, antiperiodic T"
METRIC = "D.psi HBM GB/s (algorithmic) at 48^3x96; mixed vs FP64 FGMRES time-to-1e-10"
BYTES = {"f64": (1152, 384), "f32": (576, 192), "f16": (288, 104), "df64": (1152, 384)}
PREC = {"f64": 1, "f32": 2, "f16": 4, "df64": 8}  # df64: FP64-accurate FP32-pair arithmetic
FLOPS_PER_SITE = 1848  # nominal: hopping 1320 + self coupling 504 + combine 24
# FP64-pipe instructions of the FP64 stencil per site and RHS (ncu; an FMA and
# an addition each take one slot, so the pipe roof is half the FMA FLOP peak)
F64_PIPE_INSTR_PER_SITE = 1153
# link force with the clover term, one RHS, as the kernels compute it (an FMA
# counts 2): hopping outer products 4 x 336, clover leaf derivatives 6 planes x
# (T 720 + T' 36 + 4 leaves x 8 products x 216), su(3) projection 4 x 242
FORCE_FLOPS_PER_SITE = 4 * 336 + 6 * (720 + 36 + 4 * 8 * 216) + 4 * 242


_T0 = time.time()


def log(msg):
    print(f"[bench {time.time() - _T0:7.1f}s] {msg}", file=sys.stderr, flush=True)


LINK_REALS_F32 = [18]  # reals per FP32 link read by single-RHS applies (set once the gauge exists)
LINK_REALS_F16 = [18]  # the same for FP16 links
HBM_PEAK = [6800.0]  # GB/s, replaced by the measured copy bandwidth at start


def bytes_per_site(prec, nrhs=1):
    a, b = BYTES[prec]
    if prec == "f32" and nrhs == 1:
        a -= 288 - 16 * LINK_REALS_F32[0]  # compressed FP32 links: 192 (12 reals) or 128 (8) instead of 288 B
    if prec == "f16" and nrhs == 1:
        a -= 144 - 8 * LINK_REALS_F16[0]  # two-row FP16 links: 96 instead of 144 B
    return a + b * nrhs


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ---------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi sampler running during the measurement."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id=None):
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50"]
        if gpu_id:
            cmd.insert(1, f"--id={gpu_id}")
        try:
            self.proc = subprocess.Popen(cmd, stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        self.windows = []

    def window(self, t0, t1):
        self.windows.append((t0, t1))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(5)
            except Exception:
                self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        rows = []
        for line in self.tmp.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                ts += float("0." + parts[0].split(".")[1]) if "." in parts[0] else 0.0
                rows.append((ts, float(parts[1]), float(parts[2]), parts[3], parts[4:]))
            except Exception:
                continue
        os.unlink(self.tmp.name)
        return rows

    def summary(self, rows):
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        inwin = [r for r in rows if any(a - 0.05 <= r[0] <= b + 0.05 for a, b in self.windows)]
        use = inwin if inwin else rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in use:
            for n, v in zip(names, r[4][1:]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(r[1] for r in use), "sm_max_mhz": max(r[2] for r in use),
                "reasons": sorted(reasons), "samples": len(use), "samples_in_timed_windows": len(inwin)}


# ---------------------------------------------------------------- distributed
def dist_env():
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    return rank, world, local


def init_dist(world, local):
    """One process per GPU (torchrun); NCCL on GPUs, gloo otherwise.  The
    path shards as independent replicas, so the process group only carries
    the barrier and the max-over-ranks reduction of the timings."""
    import torch
    if world <= 1:
        return None
    import torch.distributed as tdist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    tdist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return tdist


def _sync():
    import torch
    if torch.cuda.is_available():
        torch.cuda.synchronize()


def barrier(tdist):
    if tdist is not None:
        tdist.barrier()
    _sync()


def max_over_ranks(tdist, x):
    import torch
    if tdist is None:
        return x
    dev = "cuda" if (torch.cuda.is_available() and tdist.get_backend() == "nccl") else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def aggregate_gbs(bytes_per_unit, units_per_rank, world, seconds_max):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return bytes_per_unit * units_per_rank * world / seconds_max / 1e9


# ---------------------------------------------------------------- timing
def device_status(dd):
    """The library's device flag for expired waits (0: none since the last read)."""
    import ctypes
    f = ctypes.c_int(-1)
    dd.check(dd.lib.dd_device_status(ctypes.byref(f)), "dd_device_status")
    return f.value


def time_steps(fn, steps, warmup, stream, tdist, clocks):
    """W untimed steps, then exactly K timed steps bracketed by barrier + sync.
    Returns (total seconds max over ranks, per-step seconds list)."""
    import torch
    for _ in range(warmup):
        fn()
    barrier(tdist)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    w0 = time.time()
    t_start.record(stream)
    for i in range(steps):
        ev[i][0].record(stream)
        fn()
        ev[i][1].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    w1 = time.time()
    barrier(tdist)
    if clocks is not None:
        clocks.window(w0, w1)
    total = t_start.elapsed_time(t_end) * 1e-3
    per = [a.elapsed_time(b) * 1e-3 for a, b in ev]
    return max_over_ranks(tdist, total), per


# ---------------------------------------------------------------- profiles
def kernel_source_hash(units=("dd_hop_f32.cu", "dd_hop_f16.cu")):
    """sha256 (16 hex digits) of the sources the single-RHS FP32 and FP16
    stencils are compiled from: their instantiation units and every local
    header those include, transitively."""
    csrc = os.path.join(ROOT, "paper_2407_00041_gb300", "csrc")
    seen, todo = set(), list(units)
    while todo:
        f = todo.pop()
        if f in seen or not os.path.exists(os.path.join(csrc, f)):
            continue
        seen.add(f)
        with open(os.path.join(csrc, f)) as fh:
            todo += re.findall(r'^\s*#\s*include\s+"([^"]+)"', fh.read(), flags=re.M)
    h = hashlib.sha256()
    for f in sorted(seen):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profile_traffic(prec):
    """DRAM bytes per launch of the stencil from the committed ncu summary, if
    it was taken with the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", f"dslash_{prec}_48x48x48x96.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    h = re.search(r"kernel_sources_sha256_16:\s*([0-9a-f]+)", txt)
    if not m or not h or h.group(1) != kernel_source_hash():
        return None
    return float(m.group(1))


# ---------------------------------------------------------------- CPU oracle
def fill_sample(U, psi, dims, tslices):
    """Fill links and spinor of the listed time slices (lazily mapped arrays)."""
    import synthetic
    nT, nZ, nY, nX = dims
    per = nZ * nY * nX
    for t in tslices:
        sites = np.arange(t * per, (t + 1) * per, dtype=np.int64)
        U[t * per:(t + 1) * per] = synthetic.gauge_sites(sites, eps=EPS)
        psi[t * per:(t + 1) * per] = synthetic.spinor_sites(dims, sites)


def oracle_sample_rate(U, psi, dims, slices, reps):
    """Time the oracle's D psi on the sites of time slices [0, slices); the
    self coupling of the sample is built first (setup, timed separately)."""
    import oracle
    per = dims[1] * dims[2] * dims[3]
    sites = np.arange(slices * per, dtype=np.int64)
    t0 = time.perf_counter()
    A = oracle.clover_sites(U, dims, M0, CSW, sites)
    t_setup = time.perf_counter() - t0
    out = None
    t0 = time.perf_counter()
    for _ in range(reps):
        out = oracle.apply_D_sites(U, A, psi, dims, sites)
    dt = (time.perf_counter() - t0) / reps
    return sites, out, dt, t_setup


def cpu_baseline(U, psi, dims, budget_s=20.0, reps=3):
    """The oracle on a bounded sample: a number of whole time slices chosen
    from a one-slice trial so that setup plus `reps` applies take about
    `budget_s` seconds."""
    import oracle
    _, _, t1, s1 = oracle_sample_rate(U, psi, dims, 1, 1)
    slices = int(max(1, min(dims[0] - 2, (budget_s - s1 - t1) / max(s1 + reps * t1, 1e-6))))
    sites, out, dt, ts = oracle_sample_rate(U, psi, dims, slices, reps)
    gbs = bytes_per_site("f64") * sites.size / dt / 1e9
    cores = oracle.threads()
    # the same oracle on one core (one time slice, `reps` repetitions)
    oracle.set_threads(1)
    try:
        s1, _, dt1, _ = oracle_sample_rate(U, psi, dims, 1, reps)
    finally:
        oracle.set_threads(cores)
    gbs1 = bytes_per_site("f64") * s1.size / dt1 / 1e9
    return {"value": gbs, "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": f"FP64 CPU oracle D psi (Eq. 1.13) on the {sites.size} sites of time slices 0..{slices - 1} "
                      f"of the 48^3x96 lattice, {reps} repetitions, {dt:.3f} s per apply (self-coupling setup "
                      f"{ts:.1f} s not timed); GB/s counts the FP64 algorithmic 1536 B/site",
            "single_thread": {"value": gbs1, "unit": "GB/s", "cores": 1,
                              "sample": f"the {s1.size} sites of time slice 0, {reps} repetitions, "
                                        f"{dt1:.3f} s per apply",
                              "full_lattice_apply_s_est": dt1 * int(np.prod(dims)) / s1.size},
            "full_lattice_apply_s_est": dt * int(np.prod(dims)) / sites.size,
            "host_cpu": host_cpu_model()}, (sites, out)


def host_cpu_model():
    """CPU model and logical CPU count of this host (from /proc/cpuinfo and os)."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                k = ln.split(":", 1)[0].strip().lower()
                if k in ("model name", "cpu part", "hardware") and model is None:
                    model = ln.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        impl = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        m = re.search(r"Model name:\s*(.+)", impl)
        if m:
            model = m.group(1).strip()
    except Exception:
        pass
    return {"model": model, "nproc": os.cpu_count()}


def run_reference(args):
    """The CPU oracle as the reference arm: each step = D psi on a bounded
    sample of sites of the same 48^3 x 96 workload."""
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    import oracle
    import synthetic
    synthetic.build()
    oracle.build()
    dims = DIMS
    V = int(np.prod(dims))
    U = np.empty((V, 4, 3, 3), dtype=np.complex128)  # only the sample's slices are touched
    psi = np.empty((V, 4, 3), dtype=np.complex128)
    slices = 4
    fill_sample(U, psi, dims, [dims[0] - 1] + list(range(slices + 1)))
    per = dims[1] * dims[2] * dims[3]
    sites = np.arange(slices * per, dtype=np.int64)
    A = oracle.clover_sites(U, dims, M0, CSW, sites)
    for _ in range(args.warmup):
        oracle.apply_D_sites(U, A, psi, dims, sites)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.apply_D_sites(U, A, psi, dims, sites)
    total = time.perf_counter() - t0
    gbs = bytes_per_site("f64") * sites.size * args.steps / total / 1e9
    sample = (f"each step: FP64 CPU oracle D psi on the {sites.size} sites of time slices 0..{slices - 1} of the "
              f"48^3x96 lattice; GB/s counts the FP64 algorithmic 1536 B/site")
    line = {"impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": "f64", "nrhs": 1, "sites": V, "parallelism": "single GPU",
                       "sample_sites": int(sites.size)},
            "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": oracle.threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- other rows of the hot path
def _time_fn(fn, reps, warmup=3):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps * 1e-3


def extra_measurements(dd, torch, stream, op48, psi48, V48, tdist, clocks, alu_peaks):
    """Multi-RHS D psi at 32^4 x 12 RHS, the batched uneven-lattice launch
    (8^4 x 1, 16^4 x 5, 24^4 x 17, 32^4 x 32 RHS) against one launch per
    lattice, Dhat at 48^3 x 96, and the autograd adjoint at 24^4."""
    import ctypes
    import synthetic
    out = {}
    st = stream.cuda_stream
    # Dhat on the odd sites of the 48^3 x 96 lattice
    for name, p in (("f32", 2), ("f16", 4)):
        hb = op48.field_bytes(p, 1, 1)
        hi = torch.empty(hb, dtype=torch.uint8, device="cuda")
        ho = torch.empty_like(hi)
        op48.pack(p, 1, psi48[:, : V48 // 2].contiguous(), hi, 1)
        t = _time_fn(lambda: dd.check(dd.lib.dd_apply(op48.h, dd.DD_OP_DHAT, p, hi.data_ptr(), ho.data_ptr(), 1,
                                                      dd.DD_LAYOUT_NATIVE, st), "Dhat"), 20)
        # two half-lattice hops read every link twice; A_oo and A_ee^-1 once;
        # five half-field spinor passes (psi_o twice, t_e written and read, out_o)
        link, clov, spin = {"f32": (16 * LINK_REALS_F32[0], 288, 96), "f16": (8 * LINK_REALS_F16[0], 144, 52)}[name]
        bytes_ = 2 * link * V48 + clov * V48 + 5 * spin * (V48 // 2)
        out[f"dhat_{name}"] = {"ms": t * 1e3, "gbs_formula": bytes_ / t / 1e9}
    # domain-decomposed D psi (Algorithm 3 on virtual ranks of this GPU): the
    # 48^3 x 96 lattice split in T, in T and X, and in all four directions
    xi = torch.empty(op48.field_bytes(2, 0, 1), dtype=torch.uint8, device="cuda")
    op48.pack(2, 0, psi48[:1].contiguous(), xi, 1)
    xo = torch.empty_like(xi)
    t_single = _time_fn(lambda: dd.check(dd.lib.dd_apply(op48.h, dd.DD_OP_D, 2, xi.data_ptr(), xo.data_ptr(), 1,
                                                         dd.DD_LAYOUT_NATIVE, st), "D"), 20)
    dec_res = {"ms_single_domain": t_single * 1e3}
    for grid in ((2, 1, 1, 1), (2, 1, 1, 2), (2, 2, 2, 2)):
        dec = dd.Decomposition(op48, grid)
        dec.scatter(2, 0, xi, 1)
        t = _time_fn(lambda: dec.apply(dd.DD_OP_D, 2, 1, stream), 20)
        dec_res["x".join(map(str, grid))] = {"ms": t * 1e3, "overhead": t / t_single - 1.0,
                                             "boundary_sites_rank0": dec.info(0)["boundary_sites"]}
        del dec
    out["decomposed_D_48c96_f32"] = dec_res
    del xi, xo
    torch.cuda.empty_cache()
    # the batch of uneven lattices 8^4 x 1, 16^4 x 5, 24^4 x 17, 32^4 x 32 RHS
    shapes = [(8, 8, 8, 8), (16, 16, 16, 16), (24, 24, 24, 24), (32, 32, 32, 32)]
    nrhs = [1, 5, 17, 32]
    keep, ops, ins, outs = [], [], [], []
    for dims, n in zip(shapes, nrhs):
        lat = dd.Lattice(dims, -1)
        g = dd.Gauge(lat, synthetic.gauge(dims, eps=EPS), precisions=dd.DD_PREC_F64 | dd.DD_PREC_F32 | dd.DD_PREC_F16)
        o = dd.Operator(g, M0, CSW)
        keep.append((lat, g, o))
        ops.append(o)
        x = torch.from_numpy(synthetic.spinor(dims, nrhs=n)).cuda()
        nb = o.field_bytes(2, 0, n)
        xi = torch.empty(nb, dtype=torch.uint8, device="cuda")
        o.pack(2, 0, x, xi, n)
        ins.append(xi)
        outs.append(torch.empty_like(xi))
        del x
    # multi-RHS at 32^4 x 12 (the first 12 of the 32 RHS) in FP32 and FP16:
    # the paired-RHS layout (packed FP32x2 stencil) and the native layout
    lat32, g32, o32 = keep[3]
    V32 = lat32.V
    x12 = torch.from_numpy(synthetic.spinor(shapes[3], nrhs=12)).cuda()
    for name, p in (("f32", 2), ("f16", 4)):
        nb = o32.field_bytes(p, 0, 12)
        xi = torch.empty(nb, dtype=torch.uint8, device="cuda")
        xo = torch.empty_like(xi)
        o32.pack(p, 0, x12, xi, 12)
        t_nat = _time_fn(lambda: dd.check(dd.lib.dd_apply(o32.h, dd.DD_OP_D, p, xi.data_ptr(), xo.data_ptr(), 12,
                                                          dd.DD_LAYOUT_NATIVE, st), "D 12 RHS"), 20)
        o32.pack_paired(p, 0, x12, xi, 12)
        t = _time_fn(lambda: dd.check(dd.lib.dd_apply(o32.h, dd.DD_OP_D, p, xi.data_ptr(), xo.data_ptr(), 12,
                                                      dd.DD_LAYOUT_NATIVE_PAIRED, st), "D 12 RHS paired"), 20)
        out[f"mrhs_32x4_12rhs_{name}"] = {"ms": t * 1e3, "gbs": bytes_per_site(name, 12) * V32 / t / 1e9,
                                          "site_rhs_per_s": V32 * 12 / t,
                                          "hbm_frac": bytes_per_site(name, 12) * V32 / t / 1e9 / HBM_PEAK[0],
                                          "layout": "paired-RHS (packed FP32x2 stencil)",
                                          "ms_native_layout": t_nat * 1e3}
        del xi, xo
    del x12
    # two right-hand sides on the 48^3 x 96 lattice, paired layout
    x2 = torch.from_numpy(synthetic.spinor(DIMS, nrhs=2)).cuda()
    for name, p in (("f32", 2), ("f16", 4)):
        nb = op48.field_bytes(p, 0, 2)
        xi = torch.empty(nb, dtype=torch.uint8, device="cuda")
        xo = torch.empty_like(xi)
        op48.pack_paired(p, 0, x2, xi, 2)
        t = _time_fn(lambda: dd.check(dd.lib.dd_apply(op48.h, dd.DD_OP_D, p, xi.data_ptr(), xo.data_ptr(), 2,
                                                      dd.DD_LAYOUT_NATIVE_PAIRED, st), "D 2 RHS paired"), 20)
        out[f"mrhs_48c96_2rhs_{name}"] = {"ms": t * 1e3, "gbs": bytes_per_site(name, 2) * V48 / t / 1e9,
                                          "site_rhs_per_s": V48 * 2 / t,
                                          "hbm_frac": bytes_per_site(name, 2) * V48 / t / 1e9 / HBM_PEAK[0],
                                          "layout": "paired-RHS (packed FP32x2 stencil)"}
        del xi, xo
    del x2
    torch.cuda.empty_cache()
    # batched uneven lattices, FP32
    arr = lambda v, t=ctypes.c_void_p: (t * len(v))(*v)
    b = ctypes.c_void_p()
    dd.check(dd.lib.dd_batch_create(arr([o.h.value for o in ops]), len(ops), 2, arr(nrhs, ctypes.c_int),
                                    ctypes.byref(b)), "dd_batch_create")
    pin = arr([x.data_ptr() for x in ins])
    pout = arr([x.data_ptr() for x in outs])
    chosen = (ctypes.c_int * 3)()
    dd.check(dd.lib.dd_batch_tune(b, pin, pout, st, chosen), "dd_batch_tune")
    t_batch = _time_fn(lambda: dd.check(dd.lib.dd_apply_batched_graph(b, pin, pout, st), "graph"), 20)

    def separate():
        for o, n, xi, xo in zip(ops, nrhs, ins, outs):
            dd.check(dd.lib.dd_apply(o.h, dd.DD_OP_D, 2, xi.data_ptr(), xo.data_ptr(), n, dd.DD_LAYOUT_NATIVE, st),
                     "D")

    t_sep = _time_fn(separate, 20)
    units = sum(int(np.prod(d)) * n for d, n in zip(shapes, nrhs))
    bytes_ = sum(int(np.prod(d)) * bytes_per_site("f32", n) for d, n in zip(shapes, nrhs))
    out["batch_8c4_16c4_24c4_32c4_f32"] = {"ms_one_graph_launch": t_batch * 1e3, "ms_four_launches": t_sep * 1e3,
                                "gbs": bytes_ / t_batch / 1e9, "site_rhs": units,
                                "tuned_tile_threads": chosen[0], "tuned_ctas_per_sm": chosen[2]}
    dd.lib.dd_batch_destroy(b)
    # the same batch with the even-RHS lattices in the paired-RHS layout
    pins, pouts = [], []
    for o, n, xi in zip(ops, nrhs, ins):
        if n % 2 == 0:
            c = torch.empty((n, o.lattice.V, 12), dtype=torch.complex128, device="cuda")
            o.unpack(2, 0, xi, c, n)
            xp = torch.empty_like(xi)
            o.pack_paired(2, 0, c, xp, n)
            del c
            pins.append(xp)
            pouts.append(torch.empty_like(xp))
        else:
            pins.append(xi)
            pouts.append(torch.empty_like(xi))
    b = ctypes.c_void_p()
    dd.check(dd.lib.dd_batch_create(arr([o.h.value for o in ops]), len(ops), 2, arr(nrhs, ctypes.c_int),
                                    ctypes.byref(b)), "dd_batch_create")
    dd.check(dd.lib.dd_batch_set_layout(b, dd.DD_LAYOUT_NATIVE_PAIRED), "dd_batch_set_layout")
    ppin = arr([x.data_ptr() for x in pins])
    ppout = arr([x.data_ptr() for x in pouts])
    dd.check(dd.lib.dd_batch_tune(b, ppin, ppout, st, chosen), "dd_batch_tune")
    t_pb = _time_fn(lambda: dd.check(dd.lib.dd_apply_batched_graph(b, ppin, ppout, st), "graph"), 20)

    def separate_paired():
        for o, n, xi, xo in zip(ops, nrhs, pins, pouts):
            dd.check(dd.lib.dd_apply(o.h, dd.DD_OP_D, 2, xi.data_ptr(), xo.data_ptr(), n,
                                     dd.DD_LAYOUT_NATIVE_PAIRED if n % 2 == 0 else dd.DD_LAYOUT_NATIVE, st), "D")

    t_psep = _time_fn(separate_paired, 20)
    out["batch_8c4_16c4_24c4_32c4_f32_paired"] = {
        "ms_one_graph_launch": t_pb * 1e3, "ms_four_launches": t_psep * 1e3, "gbs": bytes_ / t_pb / 1e9,
        "hbm_frac": bytes_ / t_pb / 1e9 / HBM_PEAK[0], "site_rhs": units,
        "layout": "32^4 x 32 in the paired-RHS layout, the odd RHS counts native; one launch per lattice"}
    out["batch_8c4_16c4_24c4_32c4_f32"]["hbm_frac"] = bytes_ / t_batch / 1e9 / HBM_PEAK[0]
    dd.lib.dd_batch_destroy(b)
    del pins, pouts
    # autograd adjoint at 24^4 (FP64 and FP32): D^H and the link force with the clover term
    lat24, g24, o24 = keep[2]
    V24 = lat24.V
    phi = torch.from_numpy(synthetic.spinor(shapes[2], seed=synthetic.SEED_PHI)).cuda()
    ps = torch.from_numpy(synthetic.spinor(shapes[2], seed=synthetic.SEED_RHS)).cuda()
    G = torch.empty((V24, 4, 3, 3), dtype=torch.complex128, device="cuda")
    F = torch.empty_like(G)
    for name, p in (("f64", 1), ("f32", 2)):
        t_f = _time_fn(lambda: o24.force(p, phi, ps, 1, True, G=G, F=F), 5, warmup=1)
        tmp = torch.empty_like(phi)
        t_dh = _time_fn(lambda: o24.apply(dd.DD_OP_DH, p, phi, tmp, 1), 10)
        peak = alu_peaks[name]
        out[f"adjoint_24x4_{name}"] = {"ms_link_force_with_clover": t_f * 1e3, "ms_DH_canonical": t_dh * 1e3,
                                      "force_gflops_nominal": FORCE_FLOPS_PER_SITE * V24 / t_f / 1e9,
                                      "force_alu_frac": FORCE_FLOPS_PER_SITE * V24 / t_f / peak,
                                      "force_flops_per_site": FORCE_FLOPS_PER_SITE}
    return out


# ---------------------------------------------------------------- 64^3 x 128, 8 RHS
def run_solve_only(args):
    """One mixed-precision solve of the 48^3 x 96 workload, for profiling its
    kernels: the bench's `solve.mixed` leg (even-odd FGMRES(8), M_j = 64 CG
    steps on Dhat^H Dhat, inner tolerance 1e-6, FP32 inner, FP64 refinement),
    or with --solve-inner f16 its `solve.mixed_f16` leg (32 CG steps, inner
    tolerance 1e-3), and with --solve-precond cgnr16 the same with the CG
    vectors in FP16 (`solve.mixed_f16_cg16`)."""
    import torch
    import synthetic
    import paper_2407_00041_gb300 as dd
    dims = DIMS
    lat = dd.Lattice(dims, -1)
    gauge = dd.Gauge(lat, synthetic.gauge(dims, eps=EPS))
    op = dd.Operator(gauge, M0, CSW)
    b = torch.from_numpy(synthetic.spinor(dims, nrhs=1)).cuda()
    x = torch.zeros_like(b)
    cg, tol_in = (64, 1e-6) if args.solve_inner == "f32" else (32, 1e-3)
    pc = dd.DD_PRECOND_CGNR16 if args.solve_precond == "cgnr16" else dd.DD_PRECOND_CGNR
    status, st = op.solve(b, x, 1, tol=1e-10, inner_prec=PREC[args.solve_inner], restart=8, max_restarts=100,
                          max_outer=20, precond=pc, precond_iters=cg, inner_tol=tol_in)
    print(json.dumps({"metric": "time to ||b-Dx|| < 1e-10 ||b||, 48^3x96, mixed precision", "value": st["seconds"],
                      "unit": "s", "higher_is_better": False, "status": status, "stats": st}), flush=True)
    return 0 if status == dd.DD_OK else 1


def run_amg_solve(args):
    """The 48^3 x 96 mixed solve (FP32 inner vectors, FP64 refinement to
    ||b - D x|| < 1e-10 ||b||) with the two-level AMG preconditioner of
    Section 1.3 (DD_PRECOND_AMG): setup time, solve time, Arnoldi steps, for
    the settings given by --amg-settings (n_tv:aT.aZ.aY.aX:init:setup, comma
    separated), each RHS solved after one setup, next to the CG-preconditioned
    solve of the same system.  The oracle recomputes ||b - D x|| on the sites
    of the two boundary time slices."""
    import torch
    import oracle
    import synthetic
    import paper_2407_00041_gb300 as dd
    dims = DIMS
    nrhs = args.amg_rhs
    U = synthetic.gauge(dims, eps=EPS)
    lat = dd.Lattice(dims, -1)
    gauge = dd.Gauge(lat, U)
    op = dd.Operator(gauge, M0, CSW)
    b_h = synthetic.spinor(dims, nrhs=nrhs)
    b = torch.from_numpy(b_h).cuda()
    per = dims[1] * dims[2] * dims[3]
    V = int(np.prod(dims))
    sites = np.concatenate([np.arange(per), np.arange(V - per, V)]).astype(np.int64)
    A_s = oracle.clover_sites(U, dims, M0, CSW, sites)

    def certify(x):
        xh = x.cpu().numpy()
        worst = 0.0
        for r in range(nrhs):
            Dx = oracle.apply_D_sites(U, A_s, xh[r].reshape(-1, 12), dims, sites)
            bs = b_h[r].reshape(-1, 12)[sites]
            worst = max(worst, float(np.linalg.norm(bs - Dx) / np.linalg.norm(bs)))
        return worst

    out = {"metric": "time to ||b-Dx|| < 1e-10 ||b||, 48^3x96, FP32 inner, FP64 refinement", "unit": "s",
           "higher_is_better": False, "nrhs": nrhs, "legs": []}
    x = torch.zeros_like(b)
    status, st = op.solve(b, x, nrhs, tol=1e-10, inner_prec=dd.DD_PREC_F32, restart=8, max_restarts=100,
                          max_outer=20, precond=dd.DD_PRECOND_CGNR, precond_iters=64)
    out["legs"].append({"precond": "CG, 64 steps per M_j", "status": status, "solve_s": st["seconds"],
                        "arnoldi_steps": st["inner_iterations"], "applies_inner": st["applies_inner"],
                        "oracle_residual_boundary_slices": certify(x)})
    print(json.dumps(out["legs"][-1]), flush=True)
    for spec in args.amg_settings.split(","):
        ntv, agg, init, setup = spec.split(":")
        agg = tuple(int(v) for v in agg.split("."))
        w0 = torch.from_numpy(synthetic.spinor(dims, nrhs=int(ntv), seed=31)).cuda()
        amg = dd.Amg(op, dd.DD_PREC_F32, w0, aggregate=agg, n_tv=int(ntv), sap_block=(4, 4, 4, 4),
                     init_sap_iters=int(init), setup_iters=int(setup), coarse_tol=5e-2, coarse_restart=16,
                     coarse_max_restarts=4)
        del w0
        info = amg.info()
        x = torch.zeros_like(b)
        status, st = op.solve(b, x, nrhs, tol=1e-10, inner_prec=dd.DD_PREC_F32, restart=16, max_restarts=40,
                              max_outer=10, precond=dd.DD_PRECOND_AMG, amg=amg)
        out["legs"].append({"precond": f"AMG n_tv={ntv} aggregates={agg} init_sap={init} setup={setup}, "
                                       "SAP 4^4 blocks 1 cycle 4 MR steps, coarse GMRES(16) to 5e-2",
                            "status": status, "setup_s": info["setup_seconds"], "solve_s": st["seconds"],
                            "arnoldi_steps": st["inner_iterations"], "applies_inner": st["applies_inner"],
                            "coarse_dims": info["coarse_dims"], "oracle_residual_boundary_slices": certify(x)})
        print(json.dumps(out["legs"][-1]), flush=True)
        del amg
        torch.cuda.empty_cache()
    print(json.dumps(out), flush=True)
    return 0


def run_solve_64c128_8rhs(args):
    """Mixed-precision multi-RHS even-odd FGMRES with FP64 refinement to 1e-10
    on the 64^3 x 128 lattice with 8 Gaussian RHS, fitted in one GPU: FP64
    and FP16 copies of links and self coupling only, b and x resident in host
    memory, right-hand sides in batches of `rhs_batch`, FGMRES(m) with
    M_j = CG steps on the normal equations of Dhat and FP16 links / FP32
    vectors in the inner solve.  The CPU
    oracle certifies the final residual on the sites of two time slices."""
    import torch
    import oracle
    import synthetic
    import paper_2407_00041_gb300 as dd
    dims = (128, 64, 64, 64)
    N, batch, m = 8, args.rhs_batch, args.restart
    V = int(np.prod(dims))
    log("64^3x128 solve: generating links and 8 right-hand sides")
    U = synthetic.gauge(dims, eps=EPS)
    b = synthetic.spinor(dims, nrhs=N)
    x = np.zeros_like(b)
    free0, total = torch.cuda.mem_get_info()
    lat = dd.Lattice(dims, -1)
    gauge = dd.Gauge(lat, U, precisions=dd.DD_PREC_F64 | dd.DD_PREC_F16)
    del U  # 19 GB of host memory; the certification regenerates the slices it needs
    op = dd.Operator(gauge, M0, CSW, precisions=dd.DD_PREC_F64 | dd.DD_PREC_F16)
    free1, _ = torch.cuda.mem_get_info()
    log(f"handles: {(free0 - free1) / 1e9:.1f} GB of {total / 1e9:.1f} GB")
    h64 = V // 2 * 12 * 16 * batch
    h32 = V // 2 * 6 * 16 * batch
    plan = (free0 - free1) + 6 * h64 + V * 12 * 16 * batch + (2 * m + 1 + 8) * h32
    t0 = time.time()
    status, st = op.solve(b, x, N, layout=dd.DD_LAYOUT_CANONICAL_HOST, tol=1e-10, inner_prec=dd.DD_PREC_F16,
                          restart=m, rhs_batch=batch, precond=dd.DD_PRECOND_CGNR, precond_iters=args.cg_steps,
                          max_restarts=200, max_outer=10, verbose=1)
    wall = time.time() - t0
    log(f"64^3x128 solve: status {status} {st}")
    # oracle check of ||b - D x|| / ||b|| on two time slices per RHS
    per = dims[1] * dims[2] * dims[3]
    sites = np.arange(2 * per, dtype=np.int64)
    U = np.empty((V, 4, 3, 3), dtype=np.complex128)  # only the slices below are touched
    for t in (dims[0] - 1, 0, 1, 2):
        U[t * per:(t + 1) * per] = synthetic.gauge_sites(np.arange(t * per, (t + 1) * per), eps=EPS)
    A = oracle.clover_sites(U, dims, M0, CSW, sites)
    cert = []
    for r in range(N):
        Dx = oracle.apply_D_sites(U, A, x[r], dims, sites)
        bb = b[r].reshape(-1, 12)[sites]
        cert.append(float(np.linalg.norm(bb - Dx) / np.linalg.norm(bb)))
    line = {"metric": "time to ||b-Dx|| < 1e-10 ||b||, 64^3x128, 8 RHS, mixed precision, one GPU",
            "value": st["seconds"], "unit": "s", "n_gpus": 1, "steps": 1, "warmup": 0, "higher_is_better": False,
            "vs_baseline": None, "dtype": "f32 (fp16 links/clover inner, fp64 refinement)", "data": "synthetic",
            "config": {"workload": "64^3x128 Wilson-clover, eps=0.3 links, m0=-0.4, c_sw=1.0, 8 Gaussian RHS",
                       "rhs_batch": batch, "restart": m,
                       "method": f"even-odd FGMRES({m}), M_j = {args.cg_steps} CG steps on Dhat^H Dhat, FP64 refinement"},
            "status": status, "stats": st, "wall_s": wall,
            "device_memory": {"total_gb": total / 1e9, "handles_gb": (free0 - free1) / 1e9,
                              "planned_peak_gb": plan / 1e9},
            "oracle_residual_two_slices": cert}
    print(json.dumps(line), flush=True)
    return 0 if status == 0 else 1


def run_context_64x32(args):
    """Context run on the lattice shape of the thesis' two-node solves
    (64 x 32^3) at its mass m0 = -0.332, with the synthetic eps = 0.3 links
    instead of its gauge configurations (not in this container), so the
    numbers are not comparable to its tables.  Three solves to
    ||b - D x|| < 1e-10 ||b||: plain FP64 GMRES(30) on the full lattice with
    M = I (the thesis' unpreconditioned solver), the mixed FP32-inner
    even-odd FGMRES(8) with 64 CG steps per M_j and FP64 refinement, and the
    FP16-inner solve with FP16 CG vectors and FP32-pair refinement.  The
    oracle recomputes the residual on the sites of two time slices."""
    import torch
    import oracle
    import synthetic
    import paper_2407_00041_gb300 as dd
    dims = (64, 32, 32, 32)
    m0 = -0.332
    V = int(np.prod(dims))
    log("64x32^3 context run: generating links")
    U = synthetic.gauge(dims, eps=EPS)
    b = synthetic.spinor(dims, nrhs=1)
    lat = dd.Lattice(dims, -1)
    precs = dd.DD_PREC_F64 | dd.DD_PREC_F32 | dd.DD_PREC_F16 | dd.DD_PREC_DF64
    gauge = dd.Gauge(lat, U, precisions=precs)
    op = dd.Operator(gauge, m0, CSW, precisions=precs)
    bt = torch.from_numpy(b).cuda()
    per = dims[1] * dims[2] * dims[3]
    sites = np.arange(2 * per, dtype=np.int64)
    A = oracle.clover_sites(U, dims, m0, CSW, sites)
    legs = [("gmres_fp64_no_precond", dict(inner_prec=dd.DD_PREC_F64, even_odd=0, restart=30, max_outer=1,
                                           precond=dd.DD_PRECOND_NONE, max_restarts=100)),
            ("mixed", dict(inner_prec=dd.DD_PREC_F32, restart=8, precond=dd.DD_PRECOND_CGNR, precond_iters=64,
                           inner_tol=1e-6, max_outer=20, max_restarts=100)),
            ("mixed_f16_cg16_dfref", dict(inner_prec=dd.DD_PREC_F16, restart=8, precond=dd.DD_PRECOND_CGNR16,
                                          precond_iters=32, inner_tol=1e-3, max_outer=20, max_restarts=100,
                                          refine_prec=dd.DD_PREC_DF64))]
    out = {}
    for name, kw in legs:
        x = torch.zeros_like(bt)
        log(f"context solve {name}")
        status, st = op.solve(bt, x, 1, tol=1e-10, **kw)
        xn = x.cpu().numpy()[0]
        Dx = oracle.apply_D_sites(U, A, xn, dims, sites)
        bb = b[0].reshape(-1, 12)[sites]
        out[name] = {"seconds": st["seconds"], "status": status, "true_residual": st["true_residual"],
                     "applies": st["applies_inner"] + st["applies_fp64"], "outer": st["outer_iterations"],
                     "oracle_residual_two_slices": float(np.linalg.norm(bb - Dx) / np.linalg.norm(bb))}
        log(f"  {name}: {out[name]}")
    line = {"metric": "context: time to ||b-Dx|| < 1e-10 ||b|| on the 64x32^3 lattice shape at m0=-0.332",
            "unit": "s", "n_gpus": 1, "higher_is_better": False, "data": "synthetic (eps=0.3 links)",
            "config": {"workload": "64x32^3 Wilson-clover, eps=0.3 synthetic links, m0=-0.332, c_sw=1.0, "
                                   "antiperiodic T, 1 Gaussian RHS",
                       "note": "the thesis' two-node lattice shape and mass on synthetic links: "
                               "not comparable to its gauge-configuration solves"},
            "solves": out}
    print(json.dumps(line), flush=True)
    return 0 if all(v["status"] == 0 for k, v in out.items() if k != "gmres_fp64_no_precond") else 1


def run_cpu_solve(args):
    """The CPU oracle solving D x = b to ||b - D x|| < 1e-10 ||b|| in FP64 on
    the host cores, with the settings of the GPU solves: the oracle's
    even-odd Schur operator, its FGMRES(8) (Algorithm 2), M_j = 64 CG steps on
    Dhat^H Dhat (written here with the oracle's Dhat and Dhat^H), the full
    residual recomputed with the oracle's D.  Timed in full."""
    import oracle
    import synthetic
    synthetic.build()
    oracle.build()
    dims = tuple(int(v) for v in args.cpu_solve.split("x"))
    V = int(np.prod(dims))
    U = synthetic.gauge(dims, eps=EPS)
    b = synthetic.spinor(dims, nrhs=1)[0].reshape(V, 12)
    t_setup = time.perf_counter()
    A = oracle.clover(U, dims, M0, CSW)
    eo = oracle.EvenOdd(U, A, dims)
    t_setup = time.perf_counter() - t_setup
    counts = {"Dhat": 0}

    def Dhat(v):
        counts["Dhat"] += 1
        return eo.Dhat(v.reshape(-1, 12)).reshape(-1)

    def DhatH(v):
        counts["Dhat"] += 1
        return eo.DhatH(v.reshape(-1, 12)).reshape(-1)

    def cgnr(j, v, k=args.cg_steps):
        z = np.zeros_like(v)
        r = v.copy()
        zr = DhatH(r)
        p = zr.copy()
        g = np.vdot(zr, zr).real
        for i in range(k):
            w = Dhat(p)
            alpha = g / np.vdot(w, w).real
            z += alpha * p
            if i + 1 == k:
                break
            r -= alpha * w
            zr = DhatH(r)
            gn = np.vdot(zr, zr).real
            p = zr + (gn / g) * p
            g = gn
        return z

    if args.cpu_dhat_only:
        # one application of Dhat and of Dhat^H, timed; the full solve makes
        # about as many applications as the GPU solve with the same settings
        v = eo.prepare(b).reshape(-1)
        t0 = time.perf_counter()
        Dhat(v)
        t1 = time.perf_counter()
        DhatH(v)
        t2 = time.perf_counter()
        per = 0.5 * ((t1 - t0) + (t2 - t1))
        line = {"metric": f"CPU oracle time per Dhat application, {args.cpu_solve}, FP64", "value": per, "unit": "s",
                "higher_is_better": False, "cores": oracle.threads(), "host_cpu": host_cpu_model(),
                "dhat_s": t1 - t0, "dhatH_s": t2 - t1, "setup_s": t_setup,
                "solve_estimate_s_for_904_applications": 904 * per}
        print(json.dumps(line), flush=True)
        return 0
    t0 = time.perf_counter()
    bhat = eo.prepare(b).reshape(-1)
    x_o, st = oracle.fgmres(Dhat, bhat, m=args.restart, tol=1e-10, max_restarts=200, M=cgnr)
    x = eo.reconstruct(b, x_o.reshape(-1, 12))
    wall = time.perf_counter() - t0
    res = float(np.linalg.norm(b - oracle.apply_D(U, A, x, dims)) / np.linalg.norm(b))
    line = {"metric": f"CPU oracle time to ||b-Dx|| < 1e-10 ||b||, {args.cpu_solve}, FP64", "value": wall,
            "unit": "s", "higher_is_better": False, "cores": oracle.threads(), "host_cpu": host_cpu_model(),
            "dhat_applications": counts["Dhat"], "fgmres_cycles": st.cycles, "converged": bool(st.converged),
            "true_residual": res, "setup_s": t_setup,
            "method": f"even-odd FGMRES({args.restart}) (oracle, Algorithm 2), M_j = {args.cg_steps} CG steps on "
                      f"Dhat^H Dhat, FP64", "config": {"workload": f"{args.cpu_solve} Wilson-clover, eps=0.3 links, "
                                                                f"m0=-0.4, c_sw=1.0, 1 Gaussian RHS"}}
    print(json.dumps(line), flush=True)
    return 0 if st.converged and res < 1e-10 else 1


# ---------------------------------------------------------------- GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="f32", choices=["f64", "f32", "f16", "df64"], help="headline precision")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the multi-RHS, batch, Dhat and adjoint lines")
    ap.add_argument("--no-link8", action="store_true", help="skip the eight-real FP32 link apply and solve")
    ap.add_argument("--no-df64", action="store_true", help="skip the FP64-accurate FP32-pair apply")
    ap.add_argument("--solve-inner", default="f32", choices=["f32", "f16"])
    ap.add_argument("--dims", default="96x48x48x48", help="nT x nZ x nY x nX (a smaller lattice for profiling)")
    ap.add_argument("--nrhs", type=int, default=1, help="right-hand sides of the timed D psi (profiling)")
    ap.add_argument("--layout", default="native", choices=["native", "paired"],
                    help="field layout of the timed FP32 / FP16 D psi (paired: even --nrhs; profiling)")
    ap.add_argument("--solve-64x128-8rhs", action="store_true", help="run the 64^3x128, 8-RHS memory-fitted solve instead")
    ap.add_argument("--solve-only", action="store_true", help="run only the mixed 48^3x96 solve (for profiling)")
    ap.add_argument("--solve-precond", default="cgnr", choices=["cgnr", "cgnr16"],
                    help="--solve-only: CG vectors of the preconditioner in FP32 (cgnr) or FP16 (cgnr16, FP16 inner)")
    ap.add_argument("--rhs-batch", type=int, default=2, help="64^3x128 solve: right-hand sides per batch")
    ap.add_argument("--restart", type=int, default=8, help="64^3x128 solve: FGMRES restart length")
    ap.add_argument("--cg-steps", type=int, default=64, help="64^3x128 solve: CG steps per preconditioner application")
    ap.add_argument("--cpu-solve", default=None, help="nT x nZ x nY x nX: time the CPU oracle's FP64 solve in full")
    ap.add_argument("--cpu-dhat-only", action="store_true",
                    help="with --cpu-solve: time one oracle Dhat and Dhat^H application instead of the full solve")
    ap.add_argument("--amg-solve", action="store_true", help="run the 48^3x96 solve with the AMG preconditioner")
    ap.add_argument("--context-64x32", action="store_true",
                    help="context solves on the 64x32^3 lattice shape at m0=-0.332 (synthetic links)")
    ap.add_argument("--amg-settings", default="8:4.4.4.4:1:2,16:4.4.4.4:1:4",
                    help="AMG settings n_tv:aT.aZ.aY.aX:init_sap:setup_iters, comma separated")
    ap.add_argument("--amg-rhs", type=int, default=1, help="right-hand sides of the AMG solves")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.solve_64x128_8rhs:
        return run_solve_64c128_8rhs(args)
    if args.solve_only:
        return run_solve_only(args)
    if args.context_64x32:
        return run_context_64x32(args)
    if args.cpu_solve:
        return run_cpu_solve(args)
    if args.amg_solve:
        return run_amg_solve(args)

    import torch
    import synthetic
    import paper_2407_00041_gb300 as dd

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    tdist = init_dist(world, local)
    stream = torch.cuda.current_stream()
    peaks, peak_kind = measured_peaks()
    HBM_PEAK[0] = peaks["hbm_gbs"]
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
        gpu_id = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        gpu_id = None
    clocks = Clocks(gpu_id)

    dims = tuple(int(v) for v in args.dims.split("x"))
    V = int(np.prod(dims))
    log("generating links and spinor")
    U = synthetic.gauge(dims, eps=EPS)
    N = args.nrhs
    psi = synthetic.spinor(dims, nrhs=N)
    log("building gauge and operator handles")
    lat = dd.Lattice(dims, -1)
    precs = dd.DD_PREC_F64 | dd.DD_PREC_F32 | dd.DD_PREC_F16 | (0 if args.no_df64 else dd.DD_PREC_DF64)
    gauge = dd.Gauge(lat, U, precisions=precs)
    op = dd.Operator(gauge, M0, CSW, precisions=precs)
    # SU(3) links: the FP32 copy keeps two rows per link (192 instead of 288 B)
    rows32 = dd.lib.dd_gauge_stored_rows(gauge.h, dd.DD_PREC_F32)
    reals32 = gauge.link_reals(dd.DD_PREC_F32)
    LINK_REALS_F32[0] = reals32
    LINK_REALS_F16[0] = gauge.link_reals(dd.DD_PREC_F16)
    log(f"handles ready (single-RHS FP32 applies read {reals32} reals per link)")
    psi_dev = torch.from_numpy(psi).to("cuda")

    gpu_launches = 0
    variants = {}
    rooflines = {}
    f64_peak = f32_peak = None
    fl = np.zeros(1, dtype=np.float64)
    dd.check(dd.lib.dd_probe_flops(dd.DD_PREC_F64, fl.ctypes.data, stream.cuda_stream), "probe")
    f64_peak = float(fl[0])
    dd.check(dd.lib.dd_probe_flops(dd.DD_PREC_F32, fl.ctypes.data, stream.cuda_stream), "probe")
    f32_peak = float(fl[0])

    order = ["f64", "f32", "f16"] + ([] if args.no_df64 else ["df64"])
    out_f64 = None
    head = None
    for prec in order:
        p = PREC[prec]
        nbytes = op.field_bytes(p, 0, N)
        xin = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        xout = torch.empty_like(xin)
        paired = args.layout == "paired" and prec in ("f32", "f16") and N % 2 == 0
        if paired:
            op.pack_paired(p, 0, psi_dev, xin, N)
        else:
            op.pack(p, 0, psi_dev, xin, N)
        layout = dd.DD_LAYOUT_NATIVE_PAIRED if paired else dd.DD_LAYOUT_NATIVE

        def step():
            dd.check(dd.lib.dd_apply(op.h, dd.DD_OP_D, p, xin.data_ptr(), xout.data_ptr(), N,
                                     layout, stream.cuda_stream), "dd_apply")

        log(f"timing D psi in {prec}")
        steps = args.steps if prec == args.prec else max(10, min(args.steps, 50))
        total, per = time_steps(step, steps, args.warmup, stream, tdist, clocks if prec == args.prec else None)
        log(f"  {prec}: per-step ms min {min(per) * 1e3:.4f} max {max(per) * 1e3:.4f}; "
            f"device wait status {device_status(dd)}")
        if prec == args.prec:
            gpu_launches += steps
        ms = total / steps * 1e3
        gbs = aggregate_gbs(bytes_per_site(prec, N), V, world, total / steps)
        kern = statistics.mean(per)
        achieved = bytes_per_site(prec, N) * V / kern / 1e9
        gflops = FLOPS_PER_SITE * N * V / kern / 1e9
        bound = "hbm"
        peak, unit, frac = peaks["hbm_gbs"], "GB/s", achieved / peaks["hbm_gbs"]
        alu_peak = f64_peak if prec == "f64" else f32_peak
        if gflops * 1e9 / alu_peak > frac:  # the arithmetic pipe is the closer roof
            bound, peak, unit, frac = "alu", alu_peak / 1e12, "TFLOP/s", gflops * 1e9 / alu_peak
            achieved = gflops / 1e3
        variants[prec] = {"gbs": gbs, "ms_per_apply": ms, "hbm_frac": bytes_per_site(prec, N) * V / kern / 1e9 /
                          peaks["hbm_gbs"], "gflops_nominal": gflops, "bound": bound,
                          "roof_frac": frac, "bytes_per_site": bytes_per_site(prec, N),
                          "ms_min": min(per) * 1e3, "ms_median": statistics.median(per) * 1e3}
        if prec in ("f64", "df64") and not paired:  # the FP32-pair result against the FP64 one
            o = torch.empty_like(psi_dev)
            op.unpack(p, 0, xout, o, N)
            if prec == "f64":
                out_f64 = o
            elif out_f64 is not None:
                variants[prec]["rel_diff_vs_f64"] = ((o - out_f64).norm() / out_f64.norm()).item()
                variants[prec]["speedup_over_f64"] = variants["f64"]["ms_per_apply"] / ms
                out_f64 = None
            del o
        if prec == "f64":  # FP64-pipe instructions per site (ncu, profiles/dslash_f64_48x48x48x96.md)
            variants[prec]["fp64_pipe_frac"] = F64_PIPE_INSTR_PER_SITE * N * V / kern / (f64_peak / 2)
        rooflines[prec] = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": frac,
                           "traffic": (profile_traffic(prec) if N == 1 and dims == DIMS and
                                       (prec != "f32" or LINK_REALS_F32[0] == 12) and
                                       (prec != "f16" or LINK_REALS_F16[0] == 12) else None),
                           "ms_per_apply": kern * 1e3,
                           "peak_source": f"{peak_kind} MEASURED_PEAKS.json hbm_gbs" if bound == "hbm"
                           else "FMA-chain probe dd_probe_flops on this GPU (FP64 pipe)" if prec == "f64"
                           else "FMA-chain probe dd_probe_flops on this GPU (FP32 pipe)"}
        if rooflines[prec]["traffic"]:  # DRAM bytes of the ncu capture over this run's launch time
            rooflines[prec]["dram_gbs"] = rooflines[prec]["traffic"] / kern / 1e9
            rooflines[prec]["dram_frac"] = rooflines[prec]["dram_gbs"] / peaks["hbm_gbs"]
        if prec == args.prec:
            traffic = (profile_traffic(prec) if N == 1 and dims == DIMS and (prec != "f32" or LINK_REALS_F32[0] == 12) and
                       (prec != "f16" or LINK_REALS_F16[0] == 12)
                       else None)  # the captured launch: 48^3x96, one RHS, two-row FP32 links
            head = {"value": gbs, "ms": ms, "kernel_s": kern,
                    "roofline": {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": frac,
                                 "traffic": traffic,
                                 **({"dram_gbs": traffic / kern / 1e9,
                                     "dram_frac": traffic / kern / 1e9 / peaks["hbm_gbs"]} if traffic else {}),
                                 "peak_source": f"{peak_kind} MEASURED_PEAKS.json hbm_gbs" if bound == "hbm"
                                 else "FMA-chain probe dd_probe_flops on this GPU"}}
            # parity of the timed launch configuration on a sample of sites
            out_c = torch.empty_like(psi_dev)
            if paired:
                op.unpack_paired(p, 0, xout, out_c, N)
            else:
                op.unpack(p, 0, xout, out_c, N)
            head["_out"] = out_c
        del xin, xout

    # the eight-real FP32 links (dd_gauge_compress_links): the FP32 apply
    # reading 128 instead of 192 B of links per site, checked against the
    # two-row result of the same input
    if N == 1 and reals32 == 12 and not args.no_link8:
        try:
            gauge.compress_links(8)
        except dd.DDError as e:
            log(f"eight-real FP32 links not available: {e}")
        else:
            LINK_REALS_F32[0] = 8
            p = PREC["f32"]
            xin = torch.empty(op.field_bytes(p, 0, N), dtype=torch.uint8, device="cuda")
            xout = torch.empty_like(xin)
            op.pack(p, 0, psi_dev, xin, N)

            def step8():
                dd.check(dd.lib.dd_apply(op.h, dd.DD_OP_D, p, xin.data_ptr(), xout.data_ptr(), N,
                                         dd.DD_LAYOUT_NATIVE, stream.cuda_stream), "dd_apply")

            log("timing D psi in f32 with eight-real links")
            steps = max(10, min(args.steps, 50))
            total, per = time_steps(step8, steps, args.warmup, stream, tdist, None)
            kern = statistics.mean(per)
            out8 = torch.empty_like(psi_dev)
            op.unpack(p, 0, xout, out8, N)
            v = {"ms_per_apply": total / steps * 1e3, "kernel_ms": kern * 1e3,
                 "bytes_per_site": bytes_per_site("f32", N),
                 "hbm_frac": bytes_per_site("f32", N) * V / kern / 1e9 / peaks["hbm_gbs"],
                 "gbs": aggregate_gbs(bytes_per_site("f32", N), V, world, total / steps)}
            if "f32" in variants:
                v["speedup_over_two_row"] = variants["f32"]["ms_per_apply"] / v["ms_per_apply"]
            gauge.compress_links(12)
            LINK_REALS_F32[0] = 12
            step8()  # the same apply with the two-row links
            out12 = torch.empty_like(psi_dev)
            op.unpack(p, 0, xout, out12, N)
            torch.cuda.synchronize()
            v["rel_diff_vs_two_row"] = ((out8 - out12).norm() / out12.norm()).item()
            variants["f32_link8"] = v
            del xin, xout, out8, out12

    # the FP16 apply with three-row FP16 links, beside the two-row default
    if N == 1 and LINK_REALS_F16[0] == 12 and "f16" in variants and not args.no_link8:
        gauge.compress_links(18, dd.DD_PREC_F16)
        LINK_REALS_F16[0] = 18
        p = PREC["f16"]
        xin = torch.empty(op.field_bytes(p, 0, N), dtype=torch.uint8, device="cuda")
        xout = torch.empty_like(xin)
        op.pack(p, 0, psi_dev, xin, N)

        def step18():
            dd.check(dd.lib.dd_apply(op.h, dd.DD_OP_D, p, xin.data_ptr(), xout.data_ptr(), N,
                                     dd.DD_LAYOUT_NATIVE, stream.cuda_stream), "dd_apply")

        log("timing D psi in f16 with three-row links")
        steps = max(10, min(args.steps, 50))
        total, per = time_steps(step18, steps, args.warmup, stream, tdist, None)
        kern = statistics.mean(per)
        variants["f16_link18"] = {"ms_per_apply": total / steps * 1e3, "kernel_ms": kern * 1e3,
                                  "bytes_per_site": bytes_per_site("f16", N),
                                  "hbm_frac": bytes_per_site("f16", N) * V / kern / 1e9 / peaks["hbm_gbs"],
                                  "two_row_speedup": total / steps * 1e3 / variants["f16"]["ms_per_apply"]}
        del xin, xout
        gauge.compress_links(12, dd.DD_PREC_F16)
        LINK_REALS_F16[0] = 12

    # e2e through the C ABI on pinned host buffers: complex64 canonical
    # fields for the FP32 / FP16 applies (their input precision), complex128
    # for FP64 and FP32 pairs; the complex128 path is timed beside it
    p = PREC[args.prec]
    log("timing the host-buffer path")
    e2e_steps = max(3, min(args.steps, 20))
    e2e_runs = {}
    for c64 in ((True, False) if args.prec in ("f32", "f16") else (False,)):
        hin = torch.from_numpy(psi.astype(np.complex64) if c64 else psi).pin_memory()
        hout = torch.empty_like(hin).pin_memory()
        lay = dd.DD_LAYOUT_CANONICAL_HOST_C64 if c64 else dd.DD_LAYOUT_CANONICAL_HOST

        def e2e_step():
            dd.check(dd.lib.dd_apply(op.h, dd.DD_OP_D, p, hin.data_ptr(), hout.data_ptr(), N, lay,
                                     stream.cuda_stream), "dd_apply host")

        e_total, _ = time_steps(e2e_step, e2e_steps, 1, stream, tdist, None)
        esz = 8 if c64 else 16
        e2e_runs[c64] = {"value": bytes_per_site(args.prec, N) * V * world / (e_total / e2e_steps) / 1e9,
                         "unit": "GB/s", "h2d_bytes_per_step": V * 12 * esz * N, "d2h_bytes_per_step": V * 12 * esz * N,
                         "ms_per_step": e_total / e2e_steps * 1e3,
                         "host_fields": "complex64 canonical" if c64 else "complex128 canonical"}
        del hin, hout
    e2e = e2e_runs[True] if True in e2e_runs else e2e_runs[False]
    if True in e2e_runs:
        e2e["complex128_host_fields"] = e2e_runs[False]

    # solves: mixed-precision vs plain FP64, time to ||b - D x|| < 1e-10 ||b||
    solve = None
    if not args.no_solve:
        solve = {}
        b = psi_dev[:1].contiguous()
        sols = {}
        # FGMRES(8) with the flexible preconditioner M_j = 64 CG steps on the
        # normal equations of Dhat: plain restarted FGMRES stalls near 2.5e-3
        # on this lattice at m0 = -0.4
        # (name, inner precision, FGMRES restart, CG steps per M_j, inner tolerance): the
        # mixed and FP64 legs run the same algorithm; the FP16-storage leg uses the
        # settings that suit its less accurate inner operator (measured: 2.0 s
        # with 32 CG steps and inner tolerance 1e-3 against 2.8 s with the
        # FP32 settings)
        # the last field: reals per FP32 link of the inner operator
        legs = [("mixed", PREC[args.solve_inner], 8, 64, 1e-6, reals32), ("fp64", PREC["f64"], 8, 64, 1e-6, reals32)]
        if args.solve_inner != "f16":
            legs.insert(1, ("mixed_f16", PREC["f16"], 8, 32, 1e-3, reals32))
            # the same with the CG vectors in FP16 (DD_PRECOND_CGNR16)
            legs.insert(2, ("mixed_f16_cg16", PREC["f16"], 8, 32, 1e-3, reals32))
        if args.solve_inner == "f32" and "f32_link8" in variants:
            legs.insert(1, ("mixed_link8", PREC["f32"], 8, 64, 1e-6, 8))
        if "df64" in variants:  # the FP64-accuracy solve with the FP32-pair stencil (FP64 vectors)
            legs.append(("df64", PREC["df64"], 8, 64, 1e-6, reals32))
            # the refinement's operator applications (r = b - D x, preparation,
            # reconstruction) in FP32-pair arithmetic on the FP64 iterate
            legs.append(("mixed_dfref", PREC[args.solve_inner], 8, 64 if args.solve_inner == "f32" else 32,
                         1e-6 if args.solve_inner == "f32" else 1e-3, reals32))
            if args.solve_inner != "f16":
                legs.append(("mixed_f16_cg16_dfref", PREC["f16"], 8, 32, 1e-3, reals32))
        for name, inner, restart, cg, tol_in, reals in legs:
            x = torch.zeros_like(b)
            log(f"solve {name}")
            if reals != reals32:
                gauge.compress_links(reals)
            barrier(tdist)
            w0 = time.time()
            pc = dd.DD_PRECOND_CGNR16 if "_cg16" in name else dd.DD_PRECOND_CGNR
            rp = dd.DD_PREC_DF64 if name.endswith("_dfref") else dd.DD_PREC_F64
            status, st = op.solve(b, x, 1, tol=1e-10, inner_prec=inner, restart=restart, max_restarts=100,
                                  max_outer=20, precond=pc, precond_iters=cg, inner_tol=tol_in, refine_prec=rp)
            w1 = time.time()
            clocks.window(w0, w1)
            if reals != reals32:
                gauge.compress_links(reals32)
            sols[name] = x
            log(f"solve {name}: {st}")
            solve[name] = {"seconds": max_over_ranks(tdist, st["seconds"]), "status": status,
                           "true_residual": st["true_residual"], "outer": st["outer_iterations"],
                           "inner_steps": st["inner_iterations"], "applies_inner": st["applies_inner"],
                           "applies_fp64": st["applies_fp64"],
                           "inner_prec": {1: "f64", 2: "f32", 4: "f16 links/clover, f32 vectors",
                                          8: "f64 accuracy in FP32-pair arithmetic, f64 vectors"}[inner],
                           "f32_link_reals": reals,
                           "method": f"even-odd FGMRES({restart}), M_j = {cg} CG steps on Dhat^H Dhat"
                                     f"{' (FP16 CG vectors)' if '_cg16' in name else ''}, "
                                     f"inner tolerance {tol_in:g}, "
                                     + ("refinement on FP64 vectors with the FP32-pair (FP64-accurate) stencil"
                                        if rp == dd.DD_PREC_DF64 else "FP64 refinement")}
        d = (sols["mixed"] - sols["fp64"]).norm().item() / sols["fp64"].norm().item()
        solve["mixed_vs_fp64_solution_rel_diff"] = d
        solve["speedup_mixed_over_fp64"] = solve["fp64"]["seconds"] / solve["mixed"]["seconds"]
        if "mixed_f16" in solve:
            solve["mixed_f16_vs_fp64_solution_rel_diff"] = \
                (sols["mixed_f16"] - sols["fp64"]).norm().item() / sols["fp64"].norm().item()
            solve["speedup_mixed_f16_over_fp64"] = solve["fp64"]["seconds"] / solve["mixed_f16"]["seconds"]
        if "mixed_f16_cg16" in solve:
            solve["mixed_f16_cg16_vs_fp64_solution_rel_diff"] = \
                (sols["mixed_f16_cg16"] - sols["fp64"]).norm().item() / sols["fp64"].norm().item()
            solve["speedup_mixed_f16_cg16_over_fp64"] = solve["fp64"]["seconds"] / solve["mixed_f16_cg16"]["seconds"]
        if "df64" in solve:
            solve["df64_vs_fp64_solution_rel_diff"] = \
                (sols["df64"] - sols["fp64"]).norm().item() / sols["fp64"].norm().item()
            solve["speedup_df64_over_fp64"] = solve["fp64"]["seconds"] / solve["df64"]["seconds"]
        for name in ("mixed_dfref", "mixed_f16_cg16_dfref"):
            if name in solve:
                solve[f"{name}_vs_fp64_solution_rel_diff"] = \
                    (sols[name] - sols["fp64"]).norm().item() / sols["fp64"].norm().item()
                solve[f"speedup_{name}_over_fp64"] = solve["fp64"]["seconds"] / solve[name]["seconds"]
        if "mixed_link8" in solve:
            solve["mixed_link8_vs_fp64_solution_rel_diff"] = \
                (sols["mixed_link8"] - sols["fp64"]).norm().item() / sols["fp64"].norm().item()
            solve["speedup_mixed_link8_over_fp64"] = solve["fp64"]["seconds"] / solve["mixed_link8"]["seconds"]

    extra = None
    if not args.no_extra:
        log("extra measurements (multi-RHS, batch, Dhat, adjoint)")
        extra = extra_measurements(dd, torch, stream, op, psi_dev, V, tdist, clocks,
                                   {"f64": f64_peak, "f32": f32_peak})

    rows = clocks.stop()
    clk = clocks.summary(rows)

    cpu = None
    parity = None
    if rank == 0 and world == 1 and not args.no_cpu:
        log("CPU oracle baseline")
        cpu, (sites, ref) = cpu_baseline(U, psi[0], dims)
        log("CPU oracle baseline done")
        got = head["_out"][0].reshape(V, 12)[torch.from_numpy(sites).cuda()].cpu().numpy()
        tol = {"f64": 1e-13, "f32": 1e-6, "f16": 5e-3}[args.prec]
        err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        parity = {"sample_sites": int(sites.size), "rel_l2_vs_oracle": err, "tol": tol, "ok": err < tol}

    head.pop("_out", None)
    if tdist is not None:
        tdist.destroy_process_group()
    if rank != 0:
        return 0
    line = {
        "metric": METRIC,
        "value": head["value"], "unit": "GB/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": head["ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"f64": "f64", "f32": "f32", "f16": "f32 (fp16 storage)",
                  "df64": "f64 (FP32-pair arithmetic)"}[args.prec], "data": "synthetic",
        "config": {"workload": (WORKLOAD if dims == DIMS else WORKLOAD.replace("48^3x96", args.dims)).replace(
                       "1 RHS", f"{N} RHS"),
                   "precision": args.prec, "nrhs": N, "sites": V, "f32_link_rows_single_rhs": rows32,
                   "f32_link_reals_single_rhs": reals32, "f16_link_reals_single_rhs": LINK_REALS_F16[0],
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "inputs (>8 GB) larger than L2; no flush"},
        "roofline": head["roofline"], "roofline_by_precision": rooflines, "variants": variants, "e2e": e2e,
        "solve": solve,
        "cpu_baseline": cpu, "parity_sample": parity, "extra": extra, "gpu_launches": gpu_launches, "clocks": clk,
        "probe_tflops": {"f64": f64_peak / 1e12, "f32": f32_peak / 1e12},
    }
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
