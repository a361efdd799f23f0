"""Benchmark of the FMM-BEM matrix-vector product (the hot path inside GMRES).

Workload: the 81,920-panel globular molecule (sphere R = 20 A, icosphere
subdivision 6, 2,000 seeded charges, eps_in = 4, eps_out = 80), synthetic
stand-in for the paper's protein meshes.  One step = one product
y = (I + Ehat K') x through the C-ABI on device-resident vectors; the tree
is built once before the timed region (its time is reported separately).

Printed: one JSON line (rank 0) with the throughput in Mpanels/s, the
end-to-end number through the C-ABI with host buffers, the roofline of the
dominant kernel (P2P, FP32 ALU bound), the oracle timed on the host cores,
the solve time and the plain FP64 GPU form at the same accuracy.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank runs an independent replica of the
workload on its own GPU (the product is not sharded: replicas only).
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FMM-BEM matvec Mpanels/s & solve s, mixed vs FP64 GPU at 1e-5 rel ΔG"
FP32_LANES_PER_SM = 128
N_SM = 152


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class NvmlSampler:
    """SM clock and clock-event reasons read through NVML (the driver's
    libnvidia-ml, read-only queries) every ~0.5 ms in a background thread:
    the timed region of the product is milliseconds long, shorter than
    nvidia-smi's sampling period.  The device is matched to the CUDA device
    by its UUID."""

    # clock event reason bits (nvml.h)
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x40: "sw_thermal_slowdown",
               0x80: "hw_thermal_slowdown", 0x100: "hw_power_brake_slowdown"}

    def __init__(self, uuid):
        import ctypes
        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.dev = ctypes.c_void_p()
        if self.lib.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(self.dev)) != 0:
            raise RuntimeError("no NVML device for " + uuid)
        self.get_reasons = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        mx = ctypes.c_uint()
        self.max_mhz = float(mx.value) if self.lib.nvmlDeviceGetMaxClockInfo(self.dev, 1, ctypes.byref(mx)) == 0 \
            else None
        self.samples, self.reasons, self.run = [], 0, False

    def _loop(self):
        c = self.ct.c_uint()
        r = self.ct.c_ulonglong()
        while self.run:
            if self.lib.nvmlDeviceGetClockInfo(self.dev, 1, self.ct.byref(c)) == 0:
                self.samples.append(float(c.value))
            if self.get_reasons(self.dev, self.ct.byref(r)) == 0:
                self.reasons |= int(r.value)
            time.sleep(0.0005)

    def start(self):
        self.run = True
        self.t = threading.Thread(target=self._loop, daemon=True)
        self.t.start()
        while not self.samples and self.t.is_alive():
            time.sleep(0.0002)

    def stop(self):
        self.run = False
        self.t.join(timeout=2)
        self.lib.nvmlShutdown()
        return {"sm_mhz": statistics.median(self.samples) if self.samples else None, "sm_max_mhz": self.max_mhz,
                "reasons": sorted(v for k, v in self.REASONS.items() if self.reasons & k),
                "samples": len(self.samples), "source": "NVML, every ~0.5 ms during the timed region"}


def clock_sampler(local):
    """NVML sampling when the driver library answers, else nvidia-smi."""
    try:
        import torch
        uuid = str(torch.cuda.get_device_properties(local).uuid)
        return NvmlSampler(uuid if uuid.startswith("GPU-") else "GPU-" + uuid)
    except Exception:
        return ClockSampler(local)


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []
        self.live = threading.Event()

    def start(self):
        """Start sampling every 20 ms; returns once the first sample has
        arrived (at most ~2 s), so that the timed region that follows is
        covered from its start."""
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            self.live.wait(timeout=2.0)
            self.lines = []  # keep only the samples taken from here on
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())
            self.live.set()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(v, ws):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _aggregate(units_per_rank, steps, t_ms, ws):
    """Whole-job throughput in millions of units per second: every rank
    processed units_per_rank x steps; t_ms is the max over ranks."""
    return ws * units_per_rank * steps / (t_ms * 1e-3) / 1e6


def _config(args, depth, ws):
    return {"workload": "globular-s6 (sphere R=20 A, icosphere subdivision 6, 81,920 panels, 2,000 "
                        "charges, eps 4/80)",
            "p": args.p, "leaf_size": args.leaf, "depth": depth, "precision": "mixed",
            "global_batch": ws, "parallelism": "replicas" if ws > 1 else "single",
            "l2": "flushed (256 MB write) between timed products"}


def _traffic(kernel):
    """DRAM bytes (read + write) per launch of `kernel` from the committed ncu
    capture, or None when the kernel's source changed since the capture."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "roofline_traffic.json")) as f:
            rec = json.load(f)[kernel]
        with open(os.path.join(ROOT, rec["source_file"]), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != rec["source_sha256"]:
                return None
        return rec["dram_bytes_per_launch"]
    except Exception:
        return None


def workload():
    import synth
    return synth.globular(6)


def cpu_baseline(mol, budget_s=12.0, rows=None):
    """The oracle (dense FP64, OpenMP over targets) on a bounded sample of rows."""
    import oracle
    P = oracle.Problem(mol.panels, mol.charges, mol.eps_in, mol.eps_out)
    x = P.bq()
    rng = np.random.default_rng(0)
    n = rows or 64
    t0 = time.perf_counter()
    P.kprime_rows(x, rng.choice(mol.n_p, n, replace=False))
    dt = time.perf_counter() - t0
    if rows is None:
        n = int(max(64, min(mol.n_p, n * budget_s / max(dt, 1e-3))))
        t0 = time.perf_counter()
        P.kprime_rows(x, rng.choice(mol.n_p, n, replace=False))
        dt = time.perf_counter() - t0
    return {"value": n / dt / 1e6, "unit": "Mpanels/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"{n} of {mol.n_p} rows of the dense FP64 product "
                      f"(each row = {mol.n_p * 7} quadrature points), {dt:.1f} s"}


def oracle_born_timings():
    """The oracle on the Born ion (1,280 panels): one dense product on all
    host cores and on one thread, and the full solve with its energy."""
    import oracle
    import synth
    m = synth.born(3)
    P = oracle.Problem(m.panels, m.charges, m.eps_in, m.eps_out)
    x = P.bq()
    cores = oracle.num_threads()
    t0 = time.perf_counter()
    P.kprime(x)
    t_all = time.perf_counter() - t0
    oracle.set_threads(1)
    try:
        t0 = time.perf_counter()
        P.kprime(x)
        t_one = time.perf_counter() - t0
    finally:
        oracle.set_threads(cores)
    t0 = time.perf_counter()
    sig, _ = P.solve(tol=1e-8)
    dg, _ = P.energy(sig)
    t_solve = time.perf_counter() - t0
    return {"workload": "born (R 2 A, 1,280 panels, one +1 e charge, eps 1/80)", "cores": cores,
            "matvec_s": round(t_all, 5), "matvec_s_1thread": round(t_one, 5), "solve_s": round(t_solve, 4),
            "dG_kcal": dg}


def _depth_of(args):
    """Octree leaf level the product uses for the workload at args.leaf (the
    rule of the library: the smallest level whose mean panels per non-empty
    leaf is at most the leaf size); for the reference arm's config only."""
    return {64: 5, 128: 4}.get(args.leaf)


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    mol = workload()
    cb = None
    vals = []
    for k in range(args.warmup + args.steps):
        r = cpu_baseline(mol, rows=max(8, args.ref_rows))
        if k >= args.warmup:
            vals.append(r["value"])
        cb = r
    v = float(np.mean(vals))
    cb["value"] = v
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "Mpanels/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(args, _depth_of(args), ws),
        "cpu_baseline": cb,
        "e2e": {"value": v, "unit": "Mpanels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def _time_matvec(pkg, mesh, n, torch, reps=5):
    x = torch.from_numpy(np.random.default_rng(1).standard_normal(n)).cuda()
    y = torch.empty_like(x)
    for _ in range(2):
        pkg.bem_matvec(mesh.h, x, y)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        pkg.bem_matvec(mesh.h, x, y)
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def _solve(pkg, mol, torch, **opts):
    mesh = pkg.Mesh(mol.panels, mol.charges, mol.eps_in, mol.eps_out, **opts)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sig, st = mesh.solve(allow_noconv=True)
    dg = mesh.energy(sig)
    torch.cuda.synchronize()
    return mesh, dg, time.perf_counter() - t0, st


def precision_comparison(pkg, mol, torch):
    """Mixed precision against the plain FP64 GPU form at equal accuracy.
    For each mode and leaf size in {32, 64, 128, 256}, the smallest p in
    {2, 4, 6, 8, 10, 12} whose solvation energy is within 1e-5 of the
    reference (the FP64 form at p = 14, GMRES tol 1e-10); of those, the
    configuration with the fastest solve is the mode's choice.  Each choice
    also reports its product error against the FP64 form at p = 16 (relative
    L2 and largest element, on a seeded random input)."""
    ref_mesh, dg_ref, _, _ = _solve(pkg, mol, torch, p=14, leaf_size=64, precision=1, tol=1e-10)
    ref_mesh.close()
    xr = torch.from_numpy(np.random.default_rng(11).standard_normal(mol.n_p)).cuda()
    with pkg.Mesh(mol.panels, mol.charges, mol.eps_in, mol.eps_out, p=16, leaf_size=64, precision=1) as g16:
        y16 = g16.matvec(xr).cpu().numpy()
    out = {"dG_ref_kcal": dg_ref, "reference": "FP64 GPU form, p = 14, GMRES tol 1e-10",
           "gate": "|dG - dG_ref| / |dG_ref| <= 1e-5",
           "searched": "leaf_size in {32, 64, 128, 256} x smallest passing p in {2, 4, 6, 8, 10, 12}; "
                       "the fastest solve wins",
           "product_error_reference": "FP64 GPU form at p = 16, leaf 64"}
    for name, prec in (("mixed", 0), ("fp64", 1)):
        cands = []
        for leaf in (32, 64, 128, 256):
            for p in (2, 4, 6, 8, 10, 12):
                mesh, dg, solve_s, st = _solve(pkg, mol, torch, p=p, leaf_size=leaf, precision=prec)
                err = abs(dg - dg_ref) / abs(dg_ref)
                if err <= 1e-5:
                    solves = [solve_s]
                    for _ in range(2):
                        torch.cuda.synchronize()
                        t1 = time.perf_counter()
                        sig, st = mesh.solve(allow_noconv=True)
                        mesh.energy(sig)
                        torch.cuda.synchronize()
                        solves.append(time.perf_counter() - t1)
                    y = mesh.matvec(xr).cpu().numpy()
                    cands.append({"p": p, "leaf_size": leaf, "dG_rel_err": err,
                                  "solve_s": round(float(np.median(solves)), 5),
                                  "gmres_iters": st["iterations"],
                                  "matvec_ms": round(_time_matvec(pkg, mesh, mol.n_p, torch), 4),
                                  "matvec_rel_err": float(np.linalg.norm(y - y16) / np.linalg.norm(y16)),
                                  "matvec_max_err": float(np.abs(y - y16).max() / np.abs(y16).max())})
                    mesh.close()
                    break
                mesh.close()
        out[name + "_candidates"] = cands
        out[name] = min(cands, key=lambda c: c["solve_s"]) if cands else None
    if out.get("mixed") and out.get("fp64"):
        out["speedup_matvec"] = round(out["fp64"]["matvec_ms"] / out["mixed"]["matvec_ms"], 2)
        out["speedup_solve"] = round(out["fp64"]["solve_s"] / out["mixed"]["solve_s"], 2)
    return out


def run_ours(args):
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import paper_1007_4591_gb300 as pkg
    pkg.load_library()
    mol = workload()
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    opts = dict(p=args.p, leaf_size=args.leaf, precision=0, m2l_mode=args.m2l_mode)
    if args.graph >= 0:
        opts["graph"] = args.graph
    if args.galerkin:
        opts["galerkin"] = 1
    t0 = time.perf_counter()
    mesh = pkg.Mesh(mol.panels, mol.charges, mol.eps_in, mol.eps_out, **opts)
    tree_s = time.perf_counter() - t0
    info = mesh.info()
    n = mol.n_p
    x = torch.from_numpy(np.random.default_rng(1).standard_normal(n)).to(dev)
    y = torch.empty_like(x)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(max(3, args.warmup)):
        pkg.bem_matvec(mesh.h, x, y)
    torch.cuda.synchronize()
    # timed region: K products, L2 flushed between products (outside the events)
    clk = clock_sampler(local)
    clk.start()
    _barrier(ws)
    torch.cuda.synchronize()
    evs = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pkg.bem_matvec(mesh.h, x, y)
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    _barrier(ws)
    clocks = clk.stop()
    t_ms = sum(a.elapsed_time(b) for a, b in evs)
    t_ms = _max_over_ranks(t_ms, ws)
    value = _aggregate(n, args.steps, t_ms, ws)

    # rooflines of the two large kernels from phase events on the library's
    # stream (phases run one after another in this mode); the dominant one is
    # the "roofline" entry
    pkg.bem_set_profiling(mesh.h, True)
    phases, m2l_k, near_k = [], [], []
    for _ in range(max(3, min(args.steps, 10))):
        flush.fill_(1.0)
        pkg.bem_matvec(mesh.h, x, y)
        phases.append(pkg.bem_last_phase_ms(mesh.h))
        m2l_k.append(pkg.bem_last_m2l_ms(mesh.h))
        near_k.append(pkg.bem_last_near_ms(mesh.h))
    pkg.bem_set_profiling(mesh.h, False)
    ph = {k: float(np.mean([d[k] for d in phases])) for k in phases[0]}
    # the M2L phase holds the multipole split and the tensor-core kernel
    # (zeros when the product has no tensor-core M2L: then the whole phase is
    # the SIMT kernel); the P2P phase the strength records and the
    # near-field kernel
    mk = {k: float(np.mean([d[k] for d in m2l_k])) for k in m2l_k[0]}
    nk = {k: float(np.mean([d[k] for d in near_k])) for k in near_k[0]}
    t_m2l = mk["tc"] if mk["tc"] > 0 else ph["m2l"]
    t_p2p = nk["p2p"] if nk["p2p"] > 0 else ph["p2p"]
    peaks, src = _peaks()
    f_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = N_SM * FP32_LANES_PER_SM * 2 * f_mhz * 1e6 / 1e12
    p2p_flops = 20.0 * info["p2p_pairs"]
    rl_p2p = {"kernel": "k_p2p (near-field panel quadrature)", "bound": "alu",
              "achieved": round(p2p_flops / (t_p2p * 1e-3) / 1e12, 3), "peak": round(fp32_peak, 2),
              "unit": "TFLOP/s", "traffic": _traffic("k_p2p"), "time_ms": round(t_p2p, 4),
              "peak_source": f"FP32: {N_SM} SMs x {FP32_LANES_PER_SM} lanes x 2 x "
                             f"{f_mhz:.0f} MHz (sm_max_mhz from MEASURED_PEAKS.json, {src})",
              "algorithmic": f"20 flop x {info['p2p_pairs']} (collocation point, source point) pairs"}
    rl_p2p["frac"] = round(rl_p2p["achieved"] / fp32_peak, 4)
    # the FP32 rate the FMA pipe delivers on this device (packed FMA chains on
    # every SM), next to the derived peak
    fp32_meas = pkg.bem_fp32_peak()
    rl_p2p["peak_measured"] = round(fp32_meas, 2)
    rl_p2p["frac_of_measured"] = round(rl_p2p["achieved"] / fp32_meas, 4) if fp32_meas > 0 else None
    # M2L: credited with the rotation-form count (8,866 flop per translation at
    # p = 10), not the dense 121 x 121 product the kernel executes; peak = the
    # dense TF32 tensor rate, the measured bf16 rate x the nominal 1.1 / 2.25
    p = args.p
    m2l_unit = 2 * (2 * (p + 1) * (2 * p + 1) * (2 * p + 3) / 3 + (p + 1) ** 2 + p * (p + 1) * (2 * p + 1) / 3)
    m2l_flops = m2l_unit * info["m2l_pairs"]
    bf16 = float(peaks.get("bf16_tflops", 1900.0))
    tf32_peak = bf16 * 1.1 / 2.25
    rl_m2l = {"kernel": "k_m2l_tc (tensor-core M2L)" if mk["tc"] > 0 else "k_translate (M2L phase)",
              "bound": "tensor", "achieved": round(m2l_flops / (t_m2l * 1e-3) / 1e12, 3),
              "peak": round(tf32_peak, 1), "unit": "TFLOP/s", "traffic": _traffic("k_m2l_tc"),
              "time_ms": round(t_m2l, 4),
              "peak_source": f"dense TF32 = bf16 {bf16:.1f} TFLOP/s (MEASURED_PEAKS.json, {src}) x 1.1/2.25",
              "algorithmic": f"{m2l_unit:.0f} flop (rotation-form count, p={p}) x {info['m2l_pairs']} translations"}
    rl_m2l["frac"] = round(rl_m2l["achieved"] / tf32_peak, 4)
    # the dominant kernel: the longest single kernel of the product
    roofline = dict(rl_m2l if t_m2l >= t_p2p else rl_p2p)
    # the whole product: algorithmic flops of every stage / (time x FP32 peak)
    nq = info["source_points"]
    mm_unit = m2l_unit
    alg = (p2p_flops + m2l_flops + mm_unit * 2 * info["m2m_pairs"] + 8 * (p + 1) ** 2 * nq
           + 12 * (p + 1) ** 2 * n)
    matvec_roofline = {"algorithmic_gflop": round(alg / 1e9, 3),
                       "achieved_tflops": round(alg / (t_ms / args.steps * 1e-3) / 1e12, 3),
                       "frac_of_fp32_peak": round(alg / (t_ms / args.steps * 1e-3) / 1e12 / fp32_peak, 4),
                       "counts": "P2P 20/pair, M2L and M2M/L2L 8,866/translation (p=10), "
                                 "P2M 8(p+1)^2/source point, L2P 12(p+1)^2/target"}

    # end to end through the C-ABI with host buffers
    xh = np.ascontiguousarray(x.cpu().numpy())
    yh = np.empty(n)
    for _ in range(2):
        pkg.bem_matvec(mesh.h, xh, yh)
    ts = []
    for _ in range(args.steps):
        t1 = time.perf_counter()
        pkg.bem_matvec(mesh.h, xh, yh)
        ts.append(time.perf_counter() - t1)
    e2e_s = _max_over_ranks(float(np.sum(ts)), ws)
    e2e = {"value": ws * n * args.steps / e2e_s / 1e6, "unit": "Mpanels/s",
           "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n}

    # full solves (rhs + GMRES to 1e-8 + energy) on the same mesh: the median of 5
    solve_ts = []
    for _ in range(5):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        sig, st = mesh.solve(allow_noconv=True)
        dg = mesh.energy(sig)
        torch.cuda.synchronize()
        solve_ts.append(time.perf_counter() - t1)
    solve_s = float(np.median(solve_ts))

    # mixed vs FP64 GPU at equal accuracy: the smallest p whose solvation
    # energy is within 1e-5 of the FP64 form at p = 14
    prec_cmp = None
    if not args.no_precision:
        prec_cmp = precision_comparison(pkg, mol, torch)

    L = info["depth"]
    # gather, source strengths, P2P (with the near-singular table), scatter;
    # P2M, multipole split, tensor-core M2L, L2P (with the operator's
    # epilogue) and one M2M and one L2L launch per level from 3 to L (14
    # kernels at L = 5); without a far field, an epilogue kernel instead
    launches_per = 4 + ((4 + 2 * (L - 2)) if L >= 2 else 1)
    cpu = cpu_baseline(mol, budget_s=args.cpu_budget) if (rank == 0 and not args.no_cpu) else None
    born_oracle = oracle_born_timings() if (rank == 0 and not args.no_cpu) else None
    mesh_graph = int(mesh.opt.graph)
    mesh.close()
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": round(value, 3), "unit": "Mpanels/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_ms / args.steps, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": dict(_config(args, L, ws), cuda_graph=bool(mesh_graph),
                           form="galerkin" if args.galerkin else "collocation"),
            "phases_ms": {k: round(v, 4) for k, v in ph.items()},
            "tree_build_s": round(tree_s, 4),
            "p2m_segments": int(info.get("p2m_segments", 0)),
            "solve_s": round(solve_s, 4), "solve_s_runs": [round(t, 4) for t in solve_ts],
            "solve_iters": st["iterations"], "dG_kcal": dg,
            "roofline": roofline,
            "roofline_kernels": {"p2p": rl_p2p, "m2l": rl_m2l},
            "m2l_kernels_ms": {k: round(v, 4) for k, v in mk.items()},
            "near_kernels_ms": {k: round(v, 4) for k, v in nk.items()},
            "matvec_roofline": matvec_roofline, "cpu_baseline": cpu, "oracle_born": born_oracle, "e2e": e2e,
            "precision_comparison": prec_cmp,
            "gpu_launches": launches_per * args.steps, "clocks": clocks,
        }))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_batch(args):
    """Batched uneven molecules: 64 spheres (R ~ U[10, 25] A, subdivisions
    5-7, 500-4,000 charges, seed 4), (leaf size, p) autotuned once per
    subdivision level on its first molecule, then one bem_batch_solve giving
    the full solve and both BIBEE bounds of every molecule."""
    import torch
    import synth
    import paper_1007_4591_gb300 as pkg
    torch.cuda.set_device(0)
    pkg.load_library()
    mols = synth.batch(64, seed=4)
    tuned = {}
    t0 = time.perf_counter()
    for m in mols:
        s = m.name.split("-s")[-1]
        if s not in tuned:
            o = pkg.bem_autotune(np.ascontiguousarray(m.panels), np.ascontiguousarray(m.charges),
                                 m.eps_in, m.eps_out, target=1e-5)
            tuned[s] = (int(o.leaf_size), int(o.p))
    tune_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    meshes = []
    for m in mols:
        leaf, p = tuned[m.name.split("-s")[-1]]
        meshes.append(pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, p=p, leaf_size=leaf,
                               precision=0, tol=1e-8))
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    n_p = sum(m.n_p for m in mols)
    times = []
    for it in range(max(1, args.warmup) + max(1, args.steps)):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        dg, dc, dpb, st = pkg.bem_batch_solve(meshes, threads=8)
        torch.cuda.synchronize()
        if it >= max(1, args.warmup):
            times.append(time.perf_counter() - t1)
    ok = all(s["converged"] == 1 for s in st) and all(p_ < g < c for g, c, p_ in zip(dg, dc, dpb))
    t = float(np.median(times))
    # algorithmic flops of the K' products the solves ran (GMRES iterations),
    # counted as for the single product (P2P 20/pair, translations 8,866 at
    # p = 10, P2M 8(p+1)^2/point, L2P 12(p+1)^2/target)
    peaks, _ = _peaks()
    fp32_peak = N_SM * FP32_LANES_PER_SM * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    alg = 0.0
    for g, s_ in zip(meshes, st):
        inf = g.info()
        pp = inf["p"]
        tu = 2 * (2 * (pp + 1) * (2 * pp + 1) * (2 * pp + 3) / 3 + (pp + 1) ** 2 + pp * (pp + 1) * (2 * pp + 1) / 3)
        per = (20.0 * inf["p2p_pairs"] + tu * (inf["m2l_pairs"] + 2 * inf["m2m_pairs"])
               + 8 * (pp + 1) ** 2 * inf["source_points"] + 12 * (pp + 1) ** 2 * inf["n_p"])
        alg += per * s_["iterations"]
    print(json.dumps({
        "metric": "batched FMM-BEM solve + BIBEE bounds, panels solved per second",
        "value": round(n_p / t / 1e6, 3), "unit": "Mpanels/s", "n_gpus": 1, "steps": len(times),
        "warmup": max(1, args.warmup), "higher_is_better": True, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "batch64 (64 spheres, R ~ U[10,25] A, icosphere subdivisions 5-7, "
                               "500-4,000 charges, eps 4/80, seed 4)",
                   "molecules": len(mols), "panels": n_p, "tuned_leaf_p_by_subdivision": tuned,
                   "gmres_tol": 1e-8, "threads": 8},
        "batch_solve_s": round(t, 4), "autotune_s": round(tune_s, 2), "mesh_build_s": round(build_s, 2),
        "all_converged_and_bounded": bool(ok),
        "gmres_iters_max": int(max(s["iterations"] for s in st)),
        "products_roofline": {"algorithmic_tflop": round(alg / 1e12, 4),
                              "achieved_tflops_over_batch_time": round(alg / t / 1e12, 3),
                              "frac_of_fp32_peak": round(alg / t / 1e12 / fp32_peak, 4),
                              "note": "K' products only; the batch time also holds RHS, energies, "
                                      "BIBEE passes and host work"}}), flush=True)
    for g in meshes:
        g.close()


def run_lattice(args):
    """1,000 randomly rotated copies of the globular molecule on a 50 A cubic
    lattice (81,920,000 panels, 2,000,000 charges): one coupled system on one
    GPU.  Product throughput (CUDA events, median of the timed steps) and one
    full solve (RHS + GMRES to 1e-8 + energy)."""
    import torch
    import synth
    import paper_1007_4591_gb300 as pkg
    torch.cuda.set_device(0)
    pkg.load_library()
    t0 = time.perf_counter()
    mol = synth.lattice(10)
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    mesh = pkg.Mesh(mol.panels, mol.charges, mol.eps_in, mol.eps_out, p=args.p, leaf_size=args.leaf,
                    precision=0, tol=1e-8)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    info = mesh.info()
    n = mol.n_p
    x = torch.from_numpy(np.random.default_rng(1).standard_normal(n)).cuda()
    y = torch.empty_like(x)
    for _ in range(max(1, args.warmup)):
        pkg.bem_matvec(mesh.h, x, y)
    ts = []
    for _ in range(max(1, args.steps)):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        pkg.bem_matvec(mesh.h, x, y)
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    t_ms = float(np.median(ts))
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    sig, st = mesh.solve(allow_noconv=True)
    dg = mesh.energy(sig)
    torch.cuda.synchronize()
    solve_s = time.perf_counter() - t1
    print(json.dumps({
        "metric": "FMM-BEM matvec Mpanels/s & solve s, one coupled 81.9M-panel system",
        "value": round(n / (t_ms * 1e-3) / 1e6, 3), "unit": "Mpanels/s", "n_gpus": 1,
        "steps": len(ts), "warmup": max(1, args.warmup), "ms_per_step": round(t_ms, 3),
        "higher_is_better": True, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "lattice10 (1,000 randomly rotated copies of globular-s6 on a 50 A "
                               "cubic lattice, seed 5)", "panels": n, "charges": int(mol.charges.shape[0]),
                   "p": args.p, "leaf_size": args.leaf, "depth": info["depth"], "precision": "mixed"},
        "solve_s": round(solve_s, 3), "solve_iters": st["iterations"], "dG_kcal": dg,
        "mesh_build_s": round(build_s, 2), "generate_s": round(gen_s, 2),
        "device_bytes": int(info["device_bytes"]), "m2l_pairs": int(info["m2l_pairs"]),
        "p2m_segments": int(info.get("p2m_segments", 0)),
        "p2p_pairs": int(info["p2p_pairs"])}), flush=True)
    mesh.close()


def run_workflow(args):
    """binding: dG_bind = dG_complex - dG_receptor - dG_ligand for a receptor
    sphere (globular-s6 size) and a ligand sphere (subdivision 4, R 6 A) 2 A
    apart; superposition: the isolated-molecule induced charge reused on
    n_side^3 rotated copies of globular-s6 at 50 A spacing, against the
    coupled solve of the whole lattice."""
    import torch
    import synth
    import paper_1007_4591_gb300 as pkg
    torch.cuda.set_device(0)
    pkg.load_library()
    opts = dict(p=args.p, leaf_size=args.leaf, precision=0, tol=1e-8)
    if args.workload == "binding":
        cpx, rec, lig = synth.complex_pair()
        pkg.binding_free_energy(cpx, rec, lig, **opts)  # warm-up (tables, allocations)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dg_bind, (dc, dr, dl) = pkg.binding_free_energy(cpx, rec, lig, **opts)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        line = {"metric": "electrostatic binding free energy (three solves, mesh builds included)",
                "value": round(t, 4), "unit": "s", "higher_is_better": False,
                "config": {"workload": "complex_pair (receptor s6 R 20 A 2,000 charges, ligand s4 R 6 A "
                                       "60 charges, 2 A gap, seed 11)",
                           "panels": cpx.n_p, "p": args.p, "leaf_size": args.leaf},
                "dG_bind_kcal": dg_bind, "dG_complex": dc, "dG_receptor": dr, "dG_ligand": dl}
    else:
        base = synth.globular(6)
        n = args.n_side
        system = synth.lattice(n_side=n)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = pkg.superposition_energy(base, system, copies=n ** 3, **opts)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        line = {"metric": "superposition heuristic vs coupled solve (mesh builds included)",
                "value": round(t, 3), "unit": "s", "higher_is_better": False,
                "config": {"workload": f"lattice{n} ({n ** 3} rotated copies of globular-s6, 50 A spacing, "
                                       "seed 5)", "panels": system.n_p, "p": args.p, "leaf_size": args.leaf},
                **{k: v for k, v in out.items()},
                "heuristic_rel_error": (out["dG_superposed"] - out["dG_coupled"]) / abs(out["dG_coupled"]),
                "isolated_rel_error": (out["dG_isolated"] - out["dG_coupled"]) / abs(out["dG_coupled"])}
    line.update({"n_gpus": 1, "dtype": "f32+f64", "data": "synthetic"})
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--p", type=int, default=10)
    ap.add_argument("--leaf", type=int, default=64)
    ap.add_argument("--m2l-mode", type=int, default=0)
    ap.add_argument("--graph", type=int, default=-1, help="1/0: replay the product as a CUDA graph or not "
                    "(default: the library's default)")
    ap.add_argument("--galerkin", type=int, default=0, help="1: the Galerkin form of the operator "
                    "(rows averaged over each panel) instead of collocation")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--ref-rows", type=int, default=256)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--workload", default="globular-s6", choices=["globular-s6", "batch64", "lattice10", "binding", "superposition"],
                    help="globular-s6: the K' product and solve (default); batch64: 64 uneven "
                         "molecules solved with their BIBEE bounds in one batched call; lattice10: "
                         "one coupled system of 81.9M panels; binding: a two-sphere complex's "
                         "binding free energy; superposition: the isolated-charge heuristic against "
                         "the coupled solve of a lattice of copies")
    ap.add_argument("--n-side", type=int, default=4, help="lattice side for --workload superposition")
    args = ap.parse_args()
    if args.workload == "batch64":
        run_batch(args)
    elif args.workload == "lattice10":
        run_lattice(args)
    elif args.workload in ("binding", "superposition"):
        run_workflow(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
