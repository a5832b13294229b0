"""Benchmark: batched fast-spectral collision evaluations on GB300.

Workload (default): 3D velocity grid 32^3 on [-8,8]^3, hard spheres gamma = 1,
R = 8, N_rho = 32 Gauss-Legendre radial nodes x M = 38 sphere directions; a
rank-16 Hermite-Maxwellian basis (seed 2112) gives the 256 ordered pairs
Q(V_j, V_l) of one low-rank step plus the 16^3 projection <V_k, Q(V_j, V_l)>.
One step = spectra of the 16 basis functions + all 256 evaluations + the
projection, inputs already resident in HBM; metric = collision evaluations/s.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--config c2|c3|c1]

Prints one JSON line on rank 0.  --impl reference times the FP64 CPU oracle
on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CONFIGS = {
    # name: (N, d, L, R, gamma, N_rho, M, kind, size)
    "c2": (32, 3, 8.0, 8.0, 1.0, 32, 38, "pairs", 16),
    "c3": (32, 3, 8.0, 8.0, 1.0, 32, 38, "cells", 512),
    "c1": (32, 2, 8.0, 8.0, 0.0, 16, 16, "bkw", 1),
    "c4": (64, 3, 10.0, 10.0, 1.0, 32, 86, "pairs", 8),
    "c5": (0, 0, 8.0, 8.0, 0.0, 0, 0, "mixed", 0),
    "shock": (32, 2, 13.11, 13.11, 0.0, 16, 16, "shock", 1000),
}
# 1D normal shock (Sec. 5.2 set-up, Mach 1.4): x in [-30, 30] with 1000 cells
SHOCK = dict(L_x=30.0, mach=1.4, alpha=0.5, dt=0.004, r0=2, r_max=64, drop_tol=1e-6, c=0.2)
# mixed batch: (N, d, gamma, M, r); R = L = 8, N_rho = N, bases seeded 2114 + i
C5_GRIDS = [(24, 3, 0.0, 38, 32), (32, 3, 1.0, 38, 16), (48, 3, 0.0, 86, 8), (64, 3, 1.0, 86, 4),
            (64, 2, 0.0, 16, 16), (128, 2, 1.0, 16, 8)]
WORKLOAD_NAMES = {
    "c2": "lowrank pair batch: 3D 32^3 on [-8,8]^3, gamma=1, R=8, N_rho=32 x M=38, rank 16 -> 256 pairs Q(V_j,V_l) + r^3 projection",
    "c3": "full-tensor-grid batch: 512 normal-shock cells (Mach 3, d=3), 3D 32^3, gamma=1, R=8, N_rho=32 x M=38",
    "c1": "single homogeneous Q(f,f): 2D 32^2 on [-8,8]^2, Maxwell molecules, R=8, N_rho=16 x M=16, BKW t0=0.5",
    "c4": "precision-variant workload, FP32 path: 3D 64^3 on [-10,10]^3, gamma=1, R=10, N_rho=32 x M=86, rank 8 -> 64 pairs + r^3",
    "shock": "1D normal shock end to end (Mach 1.4, x in [-30,30], 1000 cells; 2D 32^2 on [-13.11,13.11]^2, Maxwell molecules, R=13.11, N_rho=16 x M=16): adaptive low-rank K-S-L steps vs full-tensor upwind steps from the same bimodal initial state, dt=0.004, drop_tol = 0.2 x the previous step's ||f^{n+1} - f^n|| (first step 1e-6)",
    "c5": "uneven mixed batch in one captured CUDA graph: 3D N=24 r=32 M=38 g=0 | 3D N=32 r=16 M=38 g=1 | 3D N=48 r=8 M=86 g=0 | 3D N=64 r=4 M=86 g=1 | 2D N=64 r=16 M=16 g=0 | 2D N=128 r=8 M=16 g=1; N_rho=N, R=L=8; spectra + all r^2 pairs + r^3 per grid",
}
METRIC = "collision evals/s at 32^3 (batch 256) & % roofline; fast form vs plain FP32"
SHOCK_METRIC = "1D normal shock time steps/s (adaptive low rank), with the full-tensor rate beside it"
L2_FLUSH_BYTES = 512 << 20
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "shift_kernel_traffic.json")


# ----------------------------------------------------------------------------- inputs

def make_inputs(cfg_name):
    from paper_2112_02695_gb300 import workloads as W
    N, d, L, R, gamma, n_rho, M, kind, size = CONFIGS[cfg_name]
    if kind == "pairs":
        fields = W.hermite_maxwellian_basis(N, d, L, size, seed=2113 if cfg_name == "c4" else 2112)
        pairs = [(j, l) for j in range(size) for l in range(size)]
    elif kind == "cells":
        fields, _ = W.shock_cells(N, d, L, n_cells=size)
        pairs = [(x, x) for x in range(size)]
    else:
        fields = W.bkw(N, d, L, 0.5)[None]
        pairs = [(0, 0)]
    return np.asarray(fields, dtype=np.float32), pairs


def flops_per_transform(n):
    """Nominal real transform of n points: 2.5 n log2 n."""
    return 2.5 * n * math.log2(n)


def algorithmic_flops(cfg_name, n_inputs, pairs):
    """Algorithmic FP32 work of one step, by step of the method."""
    N, d, L, R, gamma, n_rho, M, kind, size = CONFIGS[cfg_name]
    n = N ** d
    U = len({(min(a, b), max(a, b)) for a, b in pairs})
    ft = flops_per_transform(n)
    out = {
        "spectrum": n_inputs * (ft + 3 * n),
        "prep": 2 * n_inputs * (ft + 3 * n),
        "shift": n_rho * M * n_inputs * (ft + 3 * n),
        "contract": n_rho * M * (2 * U * n + n_inputs * n),
        "radial": n_rho * U * (ft + 2 * n),
        "output": U * ft + len(pairs) * 2 * n,
        "project": (2 * n_inputs ** 3 * n) if kind == "pairs" else 0,
    }
    return out


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.proc = None
        self.lines = []
        self.device_index = device_index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device_index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- oracle timing

def oracle_sample(cfg_name, r=4):
    """A bounded sample of the workload for the FP64 CPU oracle: the first r
    basis functions (r^2 of the 256 pairs) for the pair batch, 4 cells for the
    cell batch, the single evaluation for c1."""
    fields, pairs = make_inputs(cfg_name)
    N, d, L, R, gamma, n_rho, M, kind, size = CONFIGS[cfg_name]
    if kind == "pairs":
        return fields[:r], [(j, l) for j in range(r) for l in range(r)], f"rank-{r} subset: {r * r} of the {size * size} pairs"
    if kind == "cells":
        idx = [0, 200, 256, 511]
        return fields[idx], [(i, i) for i in range(4)], "4 of the 512 cells"
    return fields, pairs, "the single evaluation"


def shock_oracle_step():
    """The FP64 oracle's adaptive low-rank step of the shock workload from the
    rank-2 bimodal initial state (a bounded sample: one step, all 1000 cells)."""
    from oracle import collision as C
    from oracle import shock as SH
    N, d, L, R, gamma, n_rho, M, kind, size = CONFIGS["shock"]
    sp = SH.ShockProblem(vel=C.Problem(N=N, d=d, L=L, R=R, gamma=gamma, n_rho=n_rho, M=M), n_x=size,
                         L_x=SHOCK["L_x"], mach=SHOCK["mach"], alpha=SHOCK["alpha"])
    fL, fR = sp.boundary()
    s = (np.tanh(SHOCK["alpha"] * sp.x) + 1.0) / 2.0
    f0 = np.outer(1.0 - s, fL) + np.outer(s, fR)
    X, S, V = SH.factor(sp, f0, SHOCK["r0"])
    t0 = time.perf_counter()
    SH.lowrank_step(sp, X, S, V, SHOCK["dt"], SHOCK["drop_tol"], SH.random_xh(size))
    dt = time.perf_counter() - t0
    return 1.0 / dt, dt, "one adaptive low-rank step (rank 2 + 2 boundary directions, all 1000 cells)"


def time_oracle(cfg_name, r=4, results=None, max_items=None):
    """Times the oracle on the bounded sample (its first `max_items` pairs or
    cells when given); when `results` is a dict it receives the sample and the
    oracle's outputs (full evaluations only)."""
    from oracle import collision as C
    from oracle import quadrature as Qd
    N, d, L, R, gamma, n_rho, M, kind, size = CONFIGS[cfg_name]
    if kind == "shock":
        return shock_oracle_step()
    fields, pairs, desc = oracle_sample(cfg_name, r)
    if N >= 64:
        # one evaluation costs ~4 TFLOP of FP64 here: time one pair over the first radial
        # node only and scale by the node count (the oracle's cost is linear in N_rho)
        rho, w = Qd.radial_rule(n_rho, R)
        prob = C.Problem(N=N, d=d, L=L, R=R, gamma=gamma, rho=rho[:1], w_rho=w[:1], M=M)
        fields, pairs = fields[:2], [(0, 1)]
        t0 = time.perf_counter()
        C.collide_fields(prob, fields.astype(np.float64), pairs)
        dt = (time.perf_counter() - t0) * n_rho
        return 1.0 / dt, dt, f"one pair over 1 of the {n_rho} radial nodes, time x {n_rho}"
    if max_items is not None and kind in ("pairs", "cells") and len(pairs) > max_items:
        pairs = pairs[:max_items]
        desc = f"{len(pairs)} evaluation(s) of: {desc}"
    prob = C.Problem(N=N, d=d, L=L, R=R, gamma=gamma, n_rho=n_rho, M=M)
    t0 = time.perf_counter()
    Q, Qp, Qm = C.collide_fields(prob, fields.astype(np.float64), pairs, return_parts=True)
    dt = time.perf_counter() - t0
    if results is not None:
        results.update(fields=fields, pairs=pairs, Q=Q, scale=C.scale(Q, Qp, Qm))
    return len(pairs) / dt, dt, desc


def sample_errors(B, g, results, forms):
    """Relative L-infinity error of each form on the oracle's sample, per
    result normalised by s = max(max|Q|, max|Q+|, max|Q-|) of the oracle;
    reports the largest over the sample."""
    import torch
    f = torch.tensor(results["fields"], dtype=torch.float32, device="cuda")
    pj = [p[0] for p in results["pairs"]]
    pl = [p[1] for p in results["pairs"]]
    spec = B.boltz_spectrum(g, f)
    out = {}
    for name, form in forms.items():
        Qg = B.boltz_collide_batched(g, spec, pj, pl, form=form).cpu().numpy().astype(np.float64)
        ax = tuple(range(1, Qg.ndim))
        out[name] = float(np.max(np.max(np.abs(Qg - results["Q"]), axis=ax) / results["scale"]))
    B.boltz_sync_status(g)
    return out


def lowrank_consumers(B, T, Q, r, n_v, flush, dev, n_x=1000, reps=20):
    """Times the consumers of one pair batch on its own T and Q: K-step term
    over n_x cells (the paper's 1D shock runs use 1000 cells), L-step term,
    FP64 QR of K and of L, SVD truncation and the two rotations.  Each call
    is timed alone with CUDA events after an L2 flush."""
    import torch
    rng = np.random.default_rng(5)
    K = torch.tensor(rng.standard_normal((r, n_x)), dtype=torch.float32, device=dev)
    C = torch.tensor(rng.standard_normal((r, r, r)), dtype=torch.float32, device=dev)
    Kd = torch.tensor(rng.standard_normal((r, n_x)), dtype=torch.float64, device=dev)
    Ld = torch.tensor(rng.standard_normal((r, n_v)), dtype=torch.float64, device=dev)
    S = torch.tensor(rng.standard_normal((r, r)), dtype=torch.float64, device=dev)
    U, _, Qm, _, _ = B.boltz_svd_truncate_f64(S, 0.0)
    ops = {
        "kstep_collision": (lambda: B.boltz_kstep_collision(T, K), 2.0 * r ** 3 * n_x, 4.0 * (2 * r * n_x + r ** 3)),
        "coupling_and_sstep": (lambda: B.boltz_lowrank_coupling(C, C[0], T), 4.0 * r ** 4 + 2.0 * r ** 4,
                               4.0 * (3 * r ** 3 + r * r)),
        "lstep_collision": (lambda: B.boltz_lstep_collision(Q, C), 2.0 * r ** 3 * n_v, 4.0 * (r * r + r) * n_v),
        "qr_f64_K": (lambda: B.boltz_qr_f64(Kd, 0.06), 8.0 * r * r * n_x, 8.0 * 6 * r * n_x),
        "qr_f64_L": (lambda: B.boltz_qr_f64(Ld, 0.125), 8.0 * r * r * n_v, 8.0 * 6 * r * n_v),
        "svd_truncate_f64": (lambda: B.boltz_svd_truncate_f64(S, 1e-8), None, None),
        "rotate_f64_V": (lambda: B.boltz_basis_rotate_f64(Ld, Qm, r), 2.0 * r * r * n_v, 8.0 * 2 * r * n_v),
    }
    out = {"rank": r, "n_x": n_x, "n_v": n_v}
    for name, (fn, flops, nbytes) in ops.items():
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        us = 1e3 * float(np.median(ts))
        rec = {"us": us}
        if flops:
            rec["gflop_s"] = flops / (us * 1e-6) / 1e9
            rec["gb_s"] = nbytes / (us * 1e-6) / 1e9
        out[name] = rec
    return out


def other_workloads():
    """Short runs of the other workloads (each in its own process, 10 timed
    steps; the shock 100, since a rank change inside the timed steps costs a
    direct step and a graph capture), reported beside the headline so that
    their numbers come from the same run: value, time per step and each one's
    own roofline or rate."""
    out = {}
    runs = [("c3", []), ("c4", []), ("c5", []), ("shock", []), ("shock_carleman", ["--form", "carleman"])]
    for name, extra in runs:
        steps = "100" if name.startswith("shock") else "10"
        cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--config", name.split("_")[0], "--steps", steps,
               "--warmup", "3", "--no-cpu-baseline", "--no-plain", "--no-split", "--no-carleman", "--no-others"] + extra
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
            lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
            if r.returncode != 0 or not lines:
                out[name] = {"error": (r.stderr.strip().splitlines() or ["no output"])[-1][:200]}
                continue
            d = json.loads(lines[-1])
        except (subprocess.TimeoutExpired, ValueError) as exc:
            out[name] = {"error": str(exc)[:200]}
            continue
        keep = {k: d[k] for k in ("value", "unit", "ms_per_step", "steps") if k in d}
        keep["workload"] = d.get("config", {}).get("workload")
        if d.get("roofline"):
            keep["roofline_frac"] = d["roofline"].get("frac")
            keep["step_alu_frac"] = d["roofline"].get("step_alu_frac")
            keep["kernel"] = d["roofline"].get("kernel")
        for k in ("full_tensor", "speedup_lowrank_vs_full", "rank", "lowrank_vs_full", "mass_conservation"):
            if k in d:
                keep[k] = d[k]
        if "graph_kernels" in d.get("config", {}):
            keep["graph_kernels"] = d["config"]["graph_kernels"]
        keep["clocks"] = d.get("clocks")
        out[name] = keep
    return out


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


# ----------------------------------------------------------------------------- main

def run_mixed(args, world, rank, local_rank):
    """The mixed batch: all six grids' steps captured in one CUDA graph, replayed per step."""
    import torch
    from paper_2112_02695_gb300 import boltz as B
    from paper_2112_02695_gb300 import workloads as W
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    grids, items = [], []
    evals = 0
    for i, (N, d, gamma, M, r) in enumerate(C5_GRIDS):
        g = B.boltz_grid_init(N, d, 8.0, 8.0, gamma, N, M)
        grids.append(g)
        V = torch.tensor(np.asarray(W.hermite_maxwellian_basis(N, d, 8.0, r, seed=2114 + i), dtype=np.float32),
                         device=dev)
        pj = [j for j in range(r) for _ in range(r)]
        pl = [l for _ in range(r) for l in range(r)]
        items.append(dict(grid=g, fields=V, spectra=torch.empty((r,) + g.half_shape, dtype=torch.complex64, device=dev),
                          pair_j=pj, pair_l=pl, Q_out=torch.empty((r * r,) + g.shape, device=dev), V=V,
                          T_out=torch.empty((r, r, r), device=dev)))
        evals += r * r
    # each grid's schedule autotuned on its own item before the graph is captured
    for it in items:
        B.boltz_spectrum(it["grid"], it["fields"], out=it["spectra"])
        B.boltz_autotune(it["grid"], it["spectra"], it["pair_j"], it["pair_l"], Q_scratch=it["Q_out"],
                         cache_path=os.environ.get("BOLTZ_TUNE_CACHE"))
    torch.cuda.synchronize()
    batch = B.boltz_batch_plan(items)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        B.boltz_batch_run(batch)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local_rank) as clk:
        for e0, e1 in evs:
            flush.zero_()
            e0.record()
            B.boltz_batch_run(batch)
            e1.record()
        torch.cuda.synchronize()
    for g in grids:
        B.boltz_sync_status(g)
    total_ms = sum(e0.elapsed_time(e1) for e0, e1 in evs)
    kernels = B.boltz_batch_kernel_count(batch)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": evals * args.steps / (total_ms / 1e3), "unit": "evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAMES["c5"], "evals_per_step": evals, "graph_kernels": kernels,
                       "l2": "flushed between timed steps (512 MB write outside the timed events)"},
            "gpu_launches": kernels * args.steps, "clocks": clk.summary()}))
    batch.close()
    for g in grids:
        g.close()


def run_shock(args, world, rank, local_rank):
    """1D normal shock end to end: W + K adaptive low-rank steps and W + K
    full-tensor steps from the same bimodal state f0 = (1 - s) f_L + s f_R
    (exactly rank 2, so the initial factors come from two QRs on the device);
    the K timed steps of each are bracketed by CUDA events.  Reported: low-rank
    steps/s (value), full-tensor steps/s, the ranks, and the distance between
    the two solutions after the run."""
    import torch
    from paper_2112_02695_gb300 import boltz as B
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    N, d, L, R, gamma, n_rho, M, kind, n_x = CONFIGS["shock"]
    cfg = SHOCK
    if args.form == "carleman":
        # the Carleman (Mouhot-Pareschi) form of the paper's own experiments:
        # truncation R = 0.75 L (as in the 2D BKW workload), 32 directions
        form = B.BOLTZ_FORM_CARLEMAN
        g = B.boltz_grid_init(N, d, L, 0.75 * L, gamma, 1, 32)
    else:
        form = B.BOLTZ_FORM_BATCHED
        g = B.boltz_grid_init(N, d, L, R, gamma, n_rho, M)
    n_v = N ** d
    dv = 2.0 * L / N
    axis = -L + np.arange(N) * dv
    v1, v2 = np.meshgrid(axis, axis, indexing="ij")
    g_ = 1.0 + 2.0 / d
    m2 = cfg["mach"] ** 2
    rl, ul, tl = 1.0, cfg["mach"] * np.sqrt(g_), 1.0
    rr = rl * (d + 1.0) * m2 / (m2 + d)
    ur, tr = ul * (m2 + d) / ((d + 1.0) * m2), tl * ((d + 2.0) * m2 - 1.0) * (m2 + d) / ((d + 1.0) ** 2 * m2)
    maxw = lambda rho, u, T: (rho / (2 * np.pi * T) * np.exp(-((v1 - u) ** 2 + v2 ** 2) / (2 * T))).reshape(-1)
    fL, fR = maxw(rl, ul, tl), maxw(rr, ur, tr)
    sh = B.boltz_shock_create(g, n_x, cfg["L_x"], fL, fR, cfg["r_max"], form)
    dx = 2.0 * cfg["L_x"] / n_x
    x = -cfg["L_x"] + (np.arange(n_x) + 0.5) * dx
    s = (np.tanh(cfg["alpha"] * x) + 1.0) / 2.0
    rm = cfg["r_max"]
    Xd = torch.zeros((rm, n_x), dtype=torch.float64, device=dev)
    Vd = torch.zeros((rm, n_v), dtype=torch.float64, device=dev)
    Sd = torch.zeros(rm * rm, dtype=torch.float64, device=dev)
    Yx, Rx, ix = B.boltz_qr_f64(torch.tensor(np.stack([1.0 - s, s]), device=dev), dx)
    Yv, Rv, iv = B.boltz_qr_f64(torch.tensor(np.stack([fL, fR]), device=dev), dv ** d)
    Xd[:2] = Yx
    Vd[:2] = Yv
    Sd[:4] = (Rx @ Rv.T).reshape(-1)                  # f0 = sum_ij X_i (R_x R_v^T)_ij V_j
    r = 2
    f_full = torch.empty((n_x, n_v), dtype=torch.float64, device=dev)
    B.boltz_shock_reconstruct(sh, Xd, Sd, Vd, r, f_full)
    f0 = f_full.clone()
    dt, tol = cfg["dt"], cfg["drop_tol"]
    ranks, err = [], 0.0
    for _ in range(args.warmup):
        r, err = B.boltz_shock_lowrank_step(sh, Xd, Sd, Vd, r, dt, tol)
        tol = cfg["c"] * err                       # Sec. 5.1: drop_tol = c err
    B.boltz_shock_full_step(sh, f_full, args.warmup, dt)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    with ClockSampler(local_rank) as clk:
        e[0].record()
        for _ in range(args.steps):
            r, err = B.boltz_shock_lowrank_step(sh, Xd, Sd, Vd, r, dt, tol)
            tol = cfg["c"] * err
            ranks.append(r)
        e[1].record()
        e[2].record()
        B.boltz_shock_full_step(sh, f_full, args.steps, dt)
        e[3].record()
        torch.cuda.synchronize()
    lr_ms, full_ms = e[0].elapsed_time(e[1]), e[2].elapsed_time(e[3])
    f_lr = torch.empty_like(f_full)
    B.boltz_shock_reconstruct(sh, Xd, Sd, Vd, r, f_lr)
    torch.cuda.synchronize()
    diff = (f_lr - f_full).norm().item()
    rel_change = diff / max((f_full - f0).norm().item(), 1e-300)
    rel = diff / f_full.norm().item()
    rho_lr = f_lr.sum(dim=1) * dv ** d
    rho_full = f_full.sum(dim=1) * dv ** d
    cpu = None
    if not args.no_cpu_baseline:
        rate, tsec, desc = shock_oracle_step()
        cpu = {"value": rate, "unit": "steps/s", "cores": host_cores(), "kind": "oracle", "sample": desc}
    if rank == 0:
        print(json.dumps({
            "metric": SHOCK_METRIC,
            "value": args.steps / (lr_ms / 1e3), "unit": "steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": lr_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 factors, f32 collision batch", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAMES["shock"], "n_x": n_x, "n_v": n_v, "dt": dt, "last_drop_tol": tol,
                       "form": args.form,
                       "l2": "state larger than L2 is not the point here: steps run back to back"},
            "full_tensor": {"value": args.steps / (full_ms / 1e3), "unit": "steps/s",
                            "ms_per_step": full_ms / args.steps},
            "speedup_lowrank_vs_full": full_ms / lr_ms,
            "rank": {"first": ranks[0] if ranks else r, "last": r, "max": max(ranks) if ranks else r},
            "last_step_change": err,
            "lowrank_vs_full": {"rel_l2_f": rel, "rel_l2_of_the_change": rel_change,
                                "max_density_diff": (rho_lr - rho_full).abs().max().item()},
            "cpu_baseline": cpu, "clocks": clk.summary()}))
    sh.close()
    g.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c2", choices=sorted(CONFIGS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-split", action="store_true")
    ap.add_argument("--no-carleman", action="store_true")
    ap.add_argument("--no-others", action="store_true",
                    help="skip the short runs of the other workloads (c3, c4, c5, shock) reported beside c2")
    ap.add_argument("--form", default="batched", choices=["batched", "split", "carleman"],
                    help="form of the headline measurement (the other arms run only with the default)")
    ap.add_argument("--field-budget-mb", type=int, default=0,
                    help="fix the schedule instead of autotuning it (e.g. for profiling runs)")
    ap.add_argument("--schedule", default="auto", choices=["auto", "node-blocks"],
                    help="batched-form schedule: the library's choice (pipelined on 3D 32^3), "
                         "or the node-block launches for comparison")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    N, d, L, R, gamma, n_rho, M, kind, size = CONFIGS[args.config]

    if args.impl == "reference":
        if rank != 0:
            return
        # per-step sample sized so that the whole run takes about two minutes:
        # one evaluation timed first, then as many per step as the budget allows
        n_items = None
        if kind in ("pairs", "cells"):
            _, t_one, _ = time_oracle(args.config, r=3, max_items=1)
            n_items = int(max(1, min(9, (120.0 / (args.warmup + args.steps)) // max(t_one, 1e-9))))
        ev, items = [], 1
        for i in range(args.warmup + args.steps):
            rate, dt, desc = time_oracle(args.config, r=3, max_items=n_items)
            if i >= args.warmup:
                ev.append(dt)
                items = rate * dt
        if kind == "shock":
            desc = shock_oracle_step()[2]
            value, unit = len(ev) / sum(ev), "steps/s"
        else:
            value, unit = round(items) * len(ev) / sum(ev), "evals/s"
        cores = host_cores()
        print(json.dumps({
            "impl": "reference", "metric": SHOCK_METRIC if kind == "shock" else METRIC, "value": value,
            "unit": unit, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(ev) / len(ev),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD_NAMES[args.config], "sample": desc},
            "cpu_baseline": {"value": value, "unit": unit, "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }))
        return

    if kind == "mixed":
        run_mixed(args, world, rank, local_rank)
        return
    if kind == "shock":
        run_shock(args, world, rank, local_rank)
        return

    import torch
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    from paper_2112_02695_gb300 import boltz as B
    FORM = {"batched": B.BOLTZ_FORM_BATCHED, "split": B.BOLTZ_FORM_SPLIT_BF16,
            "carleman": B.BOLTZ_FORM_CARLEMAN}[args.form]

    fields, pairs = make_inputs(args.config)
    n_in = fields.shape[0]
    pj = [p[0] for p in pairs]
    pl = [p[1] for p in pairs]
    g = B.boltz_grid_init(N, d, L, R, gamma, n_rho, M, field_budget_mb=args.field_budget_mb,
                          schedule=B.BOLTZ_SCHEDULE_NODE_BLOCKS if args.schedule == "node-blocks"
                          else B.BOLTZ_SCHEDULE_AUTO)
    dev = torch.device("cuda", local_rank)
    f_dev = torch.tensor(fields, device=dev)
    spec = torch.empty((n_in,) + g.half_shape, dtype=torch.complex64, device=dev)
    Q = torch.empty((len(pairs),) + g.shape, dtype=torch.float32, device=dev)
    T = torch.empty((n_in, n_in, n_in), dtype=torch.float32, device=dev) if kind == "pairs" else None
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    # schedule autotuning (shifted-field budget per radial block), outside the timed region
    B.boltz_spectrum(g, f_dev, out=spec)
    if args.field_budget_mb > 0:
        tuned_mb = args.field_budget_mb
    else:
        tuned_mb = B.boltz_autotune(g, spec, pj, pl, Q_scratch=Q, form=FORM,
                                    cache_path=os.environ.get("BOLTZ_TUNE_CACHE"))

    def step():
        B.boltz_spectrum(g, f_dev, out=spec)
        B.boltz_collide_batched(g, spec, pj, pl, form=FORM, out=Q)
        if kind == "pairs":
            B.boltz_project(g, f_dev, Q, out=T)

    def timed(fn, steps):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for e0, e1 in evs:
            flush.zero_()                      # L2 flush between timed steps (outside the events)
            e0.record()
            fn()
            e1.record()
        torch.cuda.synchronize()
        return [e0.elapsed_time(e1) for e0, e1 in evs]

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    B.boltz_profile_read(g, reset=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        wall0 = time.perf_counter()
        times = timed(step, args.steps)
        wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    counts = B.boltz_profile_read(g, reset=True)
    gpu_launches = sum(c for c, _ in counts.values())
    total_ms = sum(times)
    if dist:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    evals = len(pairs) * args.steps * world
    value = evals / (total_ms / 1e3)
    ms_per_step = total_ms / args.steps

    # kernel-level timing: the same steps again with per-launch events on the launching stream
    B.boltz_profile_enable(g, True)
    timed(step, args.steps)
    prof = B.boltz_profile_read(g, reset=True)
    B.boltz_profile_enable(g, False)

    # end to end through the public C API from pinned host buffers
    e2e = None
    if kind == "pairs" and args.form == "batched":     # boltz_lowrank_step_host runs the batched form
        Vh = torch.tensor(fields).pin_memory()
        Qh = torch.empty((len(pairs),) + g.shape, dtype=torch.float32).pin_memory()
        Th = torch.empty((n_in, n_in, n_in), dtype=torch.float32).pin_memory()
        for _ in range(2):
            B.boltz_lowrank_step_host(g, Vh, Qh, Th)
        te = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            B.boltz_lowrank_step_host(g, Vh, Qh, Th)
            te.append(time.perf_counter() - t0)
        e2e = {"value": len(pairs) * len(te) / sum(te), "unit": "evals/s",
               "h2d_bytes_per_step": int(Vh.numel() * 4),
               "d2h_bytes_per_step": int(Qh.numel() * 4 + Th.numel() * 4)}

    # plain per-evaluation FP32 form on the same batch
    plain = None
    if not args.no_plain and args.form == "batched":
        Qp = torch.empty_like(Q)

        def step_plain():
            B.boltz_spectrum(g, f_dev, out=spec)
            B.boltz_collide_batched(g, spec, pj, pl, form=B.BOLTZ_FORM_PLAIN, out=Qp)
            if kind == "pairs":
                B.boltz_project(g, f_dev, Qp, out=T)
        step_plain()
        torch.cuda.synchronize()
        tp = timed(step_plain, max(2, min(5, args.steps // 4)))
        plain = {"value": len(pairs) * len(tp) / (sum(tp) / 1e3), "unit": "evals/s",
                 "ms_per_step": sum(tp) / len(tp)}
        plain["batched_speedup"] = value / world / plain["value"]
        B.boltz_profile_read(g, reset=True)

    # split-precision form (BF16x3 DFT-as-GEMM shifted fields on the tensor cores), same batch
    split = None
    split_ok = d == 3 and N in (32, 64)
    if split_ok and not args.no_split and args.form == "batched":
        Qs = torch.empty_like(Q)
        split_mb = args.field_budget_mb or B.boltz_autotune(g, spec, pj, pl, Q_scratch=Qs, form=B.BOLTZ_FORM_SPLIT_BF16,
                                                           cache_path=os.environ.get("BOLTZ_TUNE_CACHE"))

        def step_split():
            B.boltz_spectrum(g, f_dev, out=spec)
            B.boltz_collide_batched(g, spec, pj, pl, form=B.BOLTZ_FORM_SPLIT_BF16, out=Qs)
            if kind == "pairs":
                B.boltz_project(g, f_dev, Qs, out=T)
        for _ in range(args.warmup):
            step_split()
        torch.cuda.synchronize()
        B.boltz_profile_read(g, reset=True)
        ts = timed(step_split, args.steps)
        B.boltz_profile_read(g, reset=True)
        B.boltz_profile_enable(g, True)
        timed(step_split, max(3, args.steps // 4))
        prof_s = B.boltz_profile_read(g, reset=True)
        B.boltz_profile_enable(g, False)
        B.boltz_sync_status(g)
        ls, mss = prof_s["shift"]
        fields_per_launch = n_rho * M * n_in / (ls / max(3, args.steps // 4))
        # executed tensor work: 3 passes x (N^2/128 tiles, all CTAs) x (2N/16 K-steps) x 2*128*(2N)*16 per field
        tc_flops_field = 3 * (N * N // 128) * (2 * N // 16) * 2 * 128 * (2 * N) * 16
        tc_achieved = tc_flops_field * fields_per_launch / (mss / ls * 1e-3) / 1e12
        bf16_peak, peak_src = 1900.0, "fallback 1.9 PFLOP/s dense BF16 burst (no MEASURED_PEAKS.json)"
        try:
            with open(MEASURED_PEAKS) as fh:
                mp = json.load(fh)
            if mp.get("bf16_tflops"):
                bf16_peak, peak_src = float(mp["bf16_tflops"]), "MEASURED_PEAKS.json bf16_tflops (burst)"
        except (OSError, ValueError):
            pass
        split = {"value": len(pairs) * len(ts) / (sum(ts) / 1e3), "unit": "evals/s", "ms_per_step": sum(ts) / len(ts),
                 "dtype": "bf16x3 split (FP32 accumulate) for the shifted fields, f32 elsewhere",
                 "autotuned_field_budget_mb": split_mb,
                 "shift_kernel": {"kernel": "k_shift_split (tcgen05 kind::f16, 3 GEMM passes per field)",
                                  "tensor_tflops_executed": tc_achieved, "peak": bf16_peak,
                                  "frac": tc_achieved / bf16_peak, "peak_source": peak_src,
                                  "share_of_step": mss / max(sum(ms for _, ms in prof_s.values()), 1e-9)}}
        # the same kernel against the algorithmic (FFT) flops of the fields it makes,
        # at the pipe it runs on: how much of the BF16 peak the method's own work uses
        alg_field = flops_per_transform(N ** d) + 3 * N ** d
        alg_tflops = alg_field * fields_per_launch / (mss / ls * 1e-3) / 1e12
        split["shift_kernel"]["alg_tflops"] = alg_tflops
        split["shift_kernel"]["alg_frac_of_bf16_peak"] = alg_tflops / bf16_peak
        split["speedup_vs_fp32_batched"] = split["value"] / (value / world)

    # Carleman form (the paper's own fast method, gamma = d - 2 only) on the same batch
    carleman = None
    if (abs(gamma - (d - 2)) < 1e-12 and not (d == 2 and N == 128) and not args.no_carleman
            and args.form == "batched"):
        Qc = torch.empty_like(Q)

        def step_carleman():
            B.boltz_spectrum(g, f_dev, out=spec)
            B.boltz_collide_batched(g, spec, pj, pl, form=B.BOLTZ_FORM_CARLEMAN, out=Qc)
            if kind == "pairs":
                B.boltz_project(g, f_dev, Qc, out=T)
        for _ in range(args.warmup):
            step_carleman()
        torch.cuda.synchronize()
        B.boltz_profile_read(g, reset=True)
        tc = timed(step_carleman, args.steps)
        B.boltz_profile_read(g, reset=True)
        B.boltz_profile_enable(g, True)
        timed(step_carleman, max(3, args.steps // 4))
        prof_c = B.boltz_profile_read(g, reset=True)
        B.boltz_profile_enable(g, False)
        B.boltz_sync_status(g)
        tot_c = sum(ms for _, ms in prof_c.values())
        carleman = {"value": len(pairs) * len(tc) / (sum(tc) / 1e3), "unit": "evals/s",
                    "ms_per_step": sum(tc) / len(tc),
                    "method": f"Carleman form: {M // 2} half-sphere directions x 2 multipliers per input, "
                              "truncation |x|,|y| <= R, no radial quadrature and no forward transform",
                    "kernel_shares": {k: round(ms / tot_c, 4) for k, (_, ms) in prof_c.items() if ms > 0}}
        carleman["speedup_vs_separated_fp32"] = carleman["value"] / (value / world)

    # mass of every Q of the batch with the default (exact) loss and with the
    # mass-consistent loss option: |dv^d sum Q| / dv^d sum |Q|, worst pair, and the
    # option's step time
    mass = None
    if kind == "pairs" and args.form == "batched":
        def rel_mass(gg, QQ):
            mom = B.boltz_moments(gg, QQ)[:, 0]
            l1 = QQ.abs().reshape(QQ.shape[0], -1).sum(dim=1).double() * (2.0 * L / N) ** d
            return float((mom.abs() / l1).max().item())
        step()
        torch.cuda.synchronize()
        mass = {"exact_loss": rel_mass(g, Q)}
        gmc = B.boltz_grid_init(N, d, L, R, gamma, n_rho, M, loss=B.BOLTZ_LOSS_MASS_CONSISTENT)
        Qmc = torch.empty_like(Q)

        def step_mc():
            B.boltz_spectrum(gmc, f_dev, out=spec)
            B.boltz_collide_batched(gmc, spec, pj, pl, out=Qmc)
            B.boltz_project(gmc, f_dev, Qmc, out=T)
        for _ in range(args.warmup):
            step_mc()
        tm = timed(step_mc, max(3, args.steps // 4))
        B.boltz_sync_status(gmc)
        mass["mass_consistent_loss"] = rel_mass(gmc, Qmc)
        mass["mass_consistent_ms_per_step"] = sum(tm) / len(tm)
        mass["normalisation"] = "max over the batch of |int Q dv| / int |Q| dv (FP64 moment sums)"
        gmc.close()

    # low-rank step consumers of this batch (Sec. 2.4 K- and L-step collision terms,
    # FP64 QR of K and L, Sec. 3.2 SVD truncation and basis rotation), L2 flushed before each call
    lowrank = None
    if kind == "pairs" and args.form == "batched":
        lowrank = lowrank_consumers(B, T, Q, n_in, N ** d, flush, dev)
    mott = None
    if kind == "cells":
        # Sec. 4.2 closure of the same shock: alpha from the two cross evaluations of the end states
        from paper_2112_02695_gb300 import workloads as W
        (rL, uL, TL), (rR, uR, TR) = W.rankine_hugoniot(d, 3.0)
        fLR = torch.tensor(np.stack(W.shock_states_fields(N, d, L)), dtype=torch.float32, device=dev)
        specLR = B.boltz_spectrum(g, fLR)
        B.boltz_mott_smith(g, specLR, rL, uL, TL, TR)
        t0 = time.perf_counter()
        al, be, _ = B.boltz_mott_smith(g, specLR, rL, uL, TL, TR)
        mott = {"alpha": al, "beta": be, "ms": 1e3 * (time.perf_counter() - t0),
                "note": "two cross evaluations + FP64 v_1^2 moment, host-timed including the readback"}

    # roofline of the dominant kernel (the shifted-field inverse transforms)
    props = torch.cuda.get_device_properties(dev)
    clocks = clk.summary()
    max_mhz = clocks.get("sm_max_mhz") or 2070.0
    alu_peak = props.multi_processor_count * 128 * 2 * max_mhz * 1e6 / 1e12    # TFLOP/s FP32
    fl = algorithmic_flops(args.config, n_in, pairs)
    if args.form == "carleman":
        # M multiplier fields per input (one real multiply per mode), no radial step
        ft = flops_per_transform(N ** d)
        fl["shift"] = M * n_in * (ft + 2 * N ** d)
        fl["radial"] = 0
        fl["contract"] = (M // 2) * 2 * len(set(pairs)) * N ** d
    pipelined = prof.get("pipeline", (0, 0.0))[0] > 0
    if pipelined:
        # one persistent kernel per step does the shifted fields, the sigma-contraction
        # and the radial step of every node: its algorithmic work is the sum of the three
        launches_s, ms_s = prof["pipeline"]
        kernel_flops = fl["shift"] + fl["contract"] + fl["radial"]
    else:
        launches_s, ms_s = prof["shift"]
        kernel_flops = fl["shift"]
    kernel_launches_per_step = launches_s / args.steps
    avg_launch_ms = ms_s / max(launches_s, 1)
    flops_per_launch = kernel_flops / max(kernel_launches_per_step, 1e-9)
    achieved = flops_per_launch / (avg_launch_ms * 1e-3) / 1e12
    traffic = None
    try:
        with open(TRAFFIC_FILE) as fh:
            entries = json.load(fh)
        ksrc = open(os.path.join(ROOT, "paper_2112_02695_gb300", "csrc", "kernels.cuh"), "rb").read()
        if pipelined:
            ksrc += open(os.path.join(ROOT, "paper_2112_02695_gb300", "csrc", "pencil.cuh"), "rb").read()
        fsrc = open(os.path.join(ROOT, "paper_2112_02695_gb300", "csrc", "fft.cuh"), "rb").read()
        lsrc = open(os.path.join(ROOT, "paper_2112_02695_gb300", "csrc", "boltz.cu"), "rb").read()
        digest = hashlib.sha256(ksrc + fsrc + lsrc).hexdigest()
        for tr in entries:
            if (tr.get("source_sha256") == digest and tr.get("config") == args.config
                    and tr.get("form", "batched") == args.form
                    and (tr.get("field_budget_mb") == tuned_mb or (pipelined and tr.get("schedule") == "pipelined"))):
                traffic = tr["bytes_per_launch"]
    except (OSError, ValueError, KeyError):
        traffic = None
    total_ms_prof = sum(ms for _, ms in prof.values())
    shares = {k: round(ms / total_ms_prof, 4) for k, (_, ms) in prof.items() if ms > 0}
    step_flops = sum(fl.values())

    cpu = None
    errors = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res = {}
        rate, dt, desc = time_oracle(args.config, results=res)
        cpu = {"value": rate, "unit": "evals/s", "cores": host_cores(), "kind": "oracle",
               "sample": f"{desc}; {dt:.1f} s of FP64 numpy/BLAS on the host"}
        if res:
            forms = {"fp32_batched": B.BOLTZ_FORM_BATCHED, "fp32_plain": B.BOLTZ_FORM_PLAIN}
            if split_ok:
                forms["split_bf16"] = B.BOLTZ_FORM_SPLIT_BF16
            errors = sample_errors(B, g, res, forms)
            errors["normalisation"] = "max over the oracle sample of max|Q_gpu - Q_oracle| / max(|Q|,|Q+|,|Q-|)"
            errors["sample"] = desc
            if carleman is not None:
                from oracle import carleman as CMO
                from oracle import collision as COL
                pc = CMO.CarlemanProblem(N=N, d=d, L=L, R=R, M=M)
                Qo, Qop, Qom = CMO.collide_fields(pc, res["fields"].astype(np.float64), res["pairs"], return_parts=True)
                errors["carleman_vs_its_oracle"] = sample_errors(
                    B, g, dict(res, Q=Qo, scale=COL.scale(Qo, Qop, Qom)), {"carleman": B.BOLTZ_FORM_CARLEMAN})["carleman"]

    others = None
    if rank == 0 and world == 1 and not args.no_others and args.config == "c2" and args.form == "batched":
        others = other_workloads()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16x3+f32" if args.form == "split" else "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAMES[args.config], "evals_per_step": len(pairs),
                       "autotuned_field_budget_mb": tuned_mb, "form": args.form,
                       "schedule": "pipelined" if pipelined else "node blocks",
                       "l2": "flushed between timed steps (512 MB write outside the timed events)",
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                         "frac": achieved / alu_peak, "traffic": traffic,
                         "kernel": {"batched": ("k_pencil (pipelined schedule: shifted fields, sigma-contraction and "
                                                "radial step of every node; algorithmic flops of the three)")
                                    if pipelined else
                                    "k_synth (phase-weighted inverse 3D transforms of the shifted fields)",
                                    "carleman": "k_synth SYN_MULT (multiplier-weighted inverse 3D transforms)",
                                    "split": "k_shift_split (tensor cores; algorithmic FFT flops over its time)"}[args.form],
                         "peak_source": f"{props.multi_processor_count} SMs x 128 FP32 lanes x 2 x {max_mhz:.0f} MHz",
                         "step_alu_frac": (step_flops / (ms_per_step * 1e-3) / 1e12) / alu_peak},
            "kernel_shares": shares,
            "gpu_launches": gpu_launches,
            "clocks": clocks,
            "e2e": e2e,
            "plain_fp32": plain,
            "split_bf16": split,
            "carleman_form": carleman,
            "mass_conservation": mass,
            "lowrank_step_consumers": lowrank,
            "mott_smith": mott,
            "error_vs_oracle": errors,
            "cpu_baseline": cpu,
            "other_workloads": others,
            "wall_s_timed_region": wall,
        }
        print(json.dumps(line))
    g.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
