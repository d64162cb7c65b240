"""Benchmark: batched AIMx matvec throughput on one GB300 (one JSON line on stdout).

Workload (default): dielectric_sphere_61440 -- eps_r = 4 sphere, 30720 RWG /
61440 unknowns (two-region formulation), 64^3 grid padded to 128^3, order 2,
64 right-hand sides, FP32 matvec at 449.7 MHz.  One step = one batched
matvec y = A(k) x of all 64 right-hand sides (projection, zero-padded FFT
convolution with the kernel multiply, interpolation, near correction); the
grid-kernel spectra of the frequency are generated during warm-up.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (direct grid summation) on the
host cores on a bounded sample of the same workload: a few rows of one
matvec, reported in the same unit (full-matvec equivalents per second).
Under torchrun each rank runs an independent replica of the workload (weak
scaling, no data-path collective); rank 0 prints the line.
"""

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "AIMx matvecs/s"
UNIT = "RHS-matvecs/s"
C0 = 299792458.0
FALLBACK_HBM = 6800.0
L2_FLUSH_BYTES = 512 << 20


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM, "fallback"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def _barrier_max(value, ws, device=None):
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class Clocks:
    """nvidia-smi clock and throttle sampling during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.reader = None

    def start(self):
        """Start sampling every 100 ms and return once the first sample has arrived (the sampler is live)."""
        import threading
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        first = threading.Event()

        def read():
            for line in self.proc.stdout:
                self.lines.append(line)
                first.set()
            first.set()

        self.reader = threading.Thread(target=read, daemon=True)
        self.reader.start()
        first.wait(timeout=10)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            self.proc.wait()
        self.reader.join(timeout=5)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in list(self.lines):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _traffic_record(kernel, workload):
    """dram bytes per launch from the committed ncu summary, if its source hash matches."""
    path = os.path.join(ROOT, "profiles", "%s_%s.md" % (kernel, workload))
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    h = re.search(r"source_sha256:\s*([0-9a-f]+)", txt)
    if not m or not h:
        return None
    src = b""
    for f in ("fused.cu", "fftreg.cuh", "regfft.cuh"):   # the plane-fused kernels' sources
        src += open(os.path.join(ROOT, "paper_2009_02281_gb300", "csrc", f), "rb").read()
    if hashlib.sha256(src).hexdigest()[:16] != h.group(1)[:16]:
        return None
    return float(m.group(1))


def _algorithmic_bytes(info, wl, B):
    """Compulsory DRAM bytes per batched FP32 matvec and per launch of each fused stage."""
    nx, ny, nz = info["grid_n"]
    Mx, My, Mz = info["pad"]
    F = 8 if wl["formulation"] == "pmchwt" else 4
    nspec = 7 if F == 8 else 2
    oct_pts = (Mx // 2 + 1) * (My // 2 + 1) * (Mz // 2 + 1)
    half = nz * My * Mx                      # stored half-spectrum points per field
    N = info["n_basis"]
    nunk = info["n_unknowns"]
    nnz = info["near_nnz"]
    U = (info["order"] + 1) ** 3
    grid = 8.0 * Mx * My * Mz * (F + F) * B  # each field written and read once per direction
    kern = 8.0 * nspec * oct_pts
    weights = 2 * U * 4 * 4.0 * N
    near = nnz * (4.0 * (3 if F == 8 else 2) + 4.0)
    vec = 2 * 8.0 * nunk * B
    step = grid + kern + weights + near + vec
    stages = {
        "z_fft_mix_inverse": 2 * 8.0 * F * half * B + kern,
        "xy_fft_forward": 8.0 * F * nx * ny * nz * B + 8.0 * F * half * B,
        "xy_fft_inverse_interp": 8.0 * F * half * B + weights / 2,
        "gather_projection": 8.0 * F * nx * ny * nz * B + weights / 2 + 8.0 * nunk * B,
    }
    return step, stages


def measure_solves(ctx, wl, args):
    """Batched GMRES solves of the workload's plane-wave right-hand sides (seeded
    directions) to a true FP64 relative residual of args.solve_tol, with the
    diagonal preconditioner and with the learned one trained on this context and
    frequency (training reported as a one-time cost, like setup)."""
    import torch
    from synth import planewave_batch
    from paper_2009_02281_gb300 import Gnn, PRECOND_DIAG, PRECOND_LEARNED, F64
    freq, B = wl["freq"], wl["nrhs"]
    dirs, pols = planewave_batch(B, seed=0)
    b = ctx.rhs_planewave(freq, dirs, pols)

    def solve(pc, rhs=b, **kw):
        torch.cuda.synchronize()
        t = time.perf_counter()
        _, st, rc = ctx.solve(freq, rhs, tol=args.solve_tol, restart=100, max_iter=4000, precond=pc, **kw)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        it = [s["iterations"] for s in st]
        ok = sum(1 for s in st if s["rel_residual"] <= args.solve_tol)
        return {"solves_per_s": round(ok / dt, 3), "wall_s": round(dt, 3), "converged": ok, "rhs": rhs.shape[0],
                "iterations_mean": round(float(np.mean(it)), 1), "iterations_max": int(max(it)),
                "max_rel_residual": max(s["rel_residual"] for s in st)}

    out = {"tol": args.solve_tol, "restart": 100, "inner": "f32 products, f64 Arnoldi and refinement",
           "diag": solve(PRECOND_DIAG)}
    if args.gnn_steps > 0:
        net = Gnn(ctx.info["formulation"])
        net.init_params(0)
        torch.cuda.synchronize()
        t = time.perf_counter()
        losses = net.fit([(ctx, freq)], steps=args.gnn_steps, nprobe=8, lr=2e-3, clip=1.0, seed=1)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        ctx.gnn_attach(net)
        net.close()
        out["learned"] = solve(PRECOND_LEARNED)
        out["learned_training"] = {"steps": args.gnn_steps, "probes_per_step": 8, "wall_s": round(dt, 2),
                                   "ms_per_step": round(1e3 * dt / args.gnn_steps, 2),
                                   "loss_first": round(losses[0], 4),
                                   "loss_last": round(float(np.mean(losses[-20:])), 4)}
    # the plain FP64 cuFFT-based AIM solve on the same GPU (generic projection and interpolation,
    # cuFFT transforms of the full padded grids, FP64 products throughout, diagonal
    # preconditioner) on a bounded sample of the right-hand sides; solves/s per converged RHS
    if args.plain_rhs > 0:
        nb = min(args.plain_rhs, B)
        ctx.set_path(2)
        try:
            plain = solve(PRECOND_DIAG, rhs=b[:nb].contiguous(), inner_precision=F64)
        finally:
            ctx.set_path(args.path)
        plain["path"] = "generic + cuFFT, FP64 products, diagonal preconditioner"
        # per-RHS cost of its product at 4, 16 and 64 right-hand sides: the solve's cost is its
        # products, so this shows whether the per-RHS solve cost stays flat up to the full batch
        per_rhs = {}
        ctx.set_path(2)
        try:
            stream = torch.cuda.current_stream()
            for nb2 in (4, 16, 64):
                if nb2 > B:
                    continue
                xx = torch.ones((nb2, ctx.nunk), dtype=torch.complex128, device="cuda")
                yy = torch.empty_like(xx)
                ctx.matvec(freq, xx, yy)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(2):
                    ctx.matvec(freq, xx, yy)
                e1.record(stream)
                torch.cuda.synchronize()
                per_rhs[str(nb2)] = round(e0.elapsed_time(e1) / 2 / nb2, 3)
                del xx, yy
        finally:
            ctx.set_path(args.path)
        plain["product_ms_per_rhs"] = per_rhs
        out["plain_fp64_cufft"] = plain
        best = max(out["diag"]["solves_per_s"], out.get("learned", {}).get("solves_per_s", 0.0))
        if plain["solves_per_s"] > 0:
            out["speedup_vs_plain_fp64_cufft"] = round(best / plain["solves_per_s"], 2)
    return out


def measure_config1(args, ws):
    """The 1920-unknown PEC sphere in FP64 (latency-bound): one-RHS product latency and the
    plane-wave solve to 1e-6 (FP64 products inside GMRES), wall time per solve."""
    import torch
    from synth import workloads, planewave_batch
    from paper_2009_02281_gb300 import Context, EFIE, F32, F64
    wl = workloads.pec_sphere_1920()
    t0 = time.time()
    ctx = Context(wl["xyz"], wl["tri"], wl["grid_n"], order=wl["order"], formulation=EFIE, near_radius=wl["radius"])
    torch.cuda.synchronize()
    setup_s = time.time() - t0
    f = wl["freq"]
    stream = torch.cuda.current_stream()
    x = torch.ones((1, ctx.nunk), dtype=torch.complex128, device="cuda")
    y = torch.empty_like(x)
    for _ in range(5):
        ctx.matvec(f, x, y)
    torch.cuda.synchronize()
    reps = 50
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        ctx.matvec(f, x, y)
    e1.record(stream)
    torch.cuda.synchronize()
    us = 1e3 * e0.elapsed_time(e1) / reps
    b = ctx.rhs_planewave(f, [[0.0, 0.0, 1.0]], [[1.0, 0.0, 0.0]])
    ctx.solve(f, b, tol=1e-6, inner_precision=F64)     # warm-up
    # the sweep: 100 frequencies from ka = 1 to ka = pi (50-150 MHz), static data reused,
    # kernel spectra regenerated per frequency, warm start from the previous frequency
    freqs = np.linspace(C0 / (2 * np.pi), C0 / 2, 100)
    torch.cuda.synchronize()
    t = time.perf_counter()
    _, sst, src = ctx.sweep(freqs, [[0.0, 0.0, 1.0]], [[1.0, 0.0, 0.0]], tol=1e-6, inner_precision=F64)
    torch.cuda.synchronize()
    sweep_s = time.perf_counter() - t
    sweep = {"frequencies": len(freqs), "f_range_hz": [float(freqs[0]), float(freqs[-1])], "rhs": 1,
             "wall_s": round(sweep_s, 3), "solves_per_s": round(ws * len(freqs) / sweep_s, 2),
             "converged": sum(1 for q in sst if q["status"] == 0),
             "iterations_mean": round(float(np.mean([q["iterations"] for q in sst])), 1), "status": src}
    # the same sweep with FP32 products inside the FP64 refinement loop (the library's default
    # precision pattern; the configuration above is specified in FP64 throughout)
    torch.cuda.synchronize()
    t = time.perf_counter()
    _, mst, mrc = ctx.sweep(freqs, [[0.0, 0.0, 1.0]], [[1.0, 0.0, 0.0]], tol=1e-6)
    torch.cuda.synchronize()
    mixed_s = time.perf_counter() - t
    sweep["fp32_products_in_fp64_refinement"] = {
        "wall_s": round(mixed_s, 3), "solves_per_s": round(ws * len(freqs) / mixed_s, 2),
        "converged": sum(1 for q in mst if q["status"] == 0),
        "iterations_mean": round(float(np.mean([q["iterations"] for q in mst])), 1),
        "max_rel_residual": max(q["rel_residual"] for q in mst), "status": mrc}
    # the batched sweep: all 100 frequencies in one call (device-side GMRES, one CUDA graph per
    # cycle, one product per Arnoldi step for every open system); right-hand sides included
    batched = {}
    for label, inner, mb, warm in (("fp64", F64, 0, False), ("fp32_products_in_fp64_refinement", F32, 0, False),
                                   ("fp64_warm_half_batch", F64, 50, True),
                                   ("fp32_warm_half_batch", F32, 50, True)):
        torch.cuda.synchronize()
        t = time.perf_counter()
        Bb = torch.stack([ctx.rhs_planewave(fq, [[0.0, 0.0, 1.0]], [[1.0, 0.0, 0.0]]) for fq in freqs])
        _, bst, brc, cnt = ctx.sweep_batched(freqs, Bb, tol=1e-6, inner_precision=inner, max_iter=3000,
                                             max_batch=mb, warm_start=warm)
        torch.cuda.synchronize()
        bs_s = time.perf_counter() - t
        flat = [q for row in bst for q in row]
        batched[label] = {"wall_s": round(bs_s, 3), "solves_per_s": round(ws * len(freqs) / bs_s, 2),
                          "max_iter": 3000, "max_batch": mb or len(freqs),
                          "initial_guess": "converged neighbour frequency" if warm else "zero",
                          "converged": sum(1 for q in flat if q["status"] == 0),
                          "iterations_mean": round(float(np.mean([q["iterations"] for q in flat])), 1),
                          "max_rel_residual": max(q["rel_residual"] for q in flat), "status": brc,
                          "cycles": cnt[0], "graphs_captured": cnt[1], "batched_products": cnt[2]}
    sweep["batched"] = batched
    best64 = min(batched["fp64"]["wall_s"], batched["fp64_warm_half_batch"]["wall_s"])
    best32 = min(batched["fp32_products_in_fp64_refinement"]["wall_s"], batched["fp32_warm_half_batch"]["wall_s"])
    sweep["batched"]["speedup_over_per_frequency_fp64"] = round(sweep_s / best64, 2)
    sweep["batched"]["speedup_over_per_frequency_fp32"] = round(mixed_s / best32, 2)
    # the same sweep with the conventional AIM (Sec. II-B): the near entries are integrated
    # directly and precorrected again at every frequency (the paper's per-frequency matrix fill)
    aim_cmp = None
    if not args.no_aim:
        ctx.set_conventional_aim(True)
        ctx.profile(True)
        ctx.profile_read()
        torch.cuda.synchronize()
        t = time.perf_counter()
        _, ast, arc = ctx.sweep(freqs, [[0.0, 0.0, 1.0]], [[1.0, 0.0, 0.0]], tol=1e-6, inner_precision=F64)
        torch.cuda.synchronize()
        aim_s = time.perf_counter() - t
        fill = ctx.profile_read().get("aim_near_fill", (0.0, 0))
        ctx.profile(False)
        ctx.set_conventional_aim(False)
        aim_cmp = {"aim_sweep_s": round(aim_s, 3), "aimx_sweep_s": round(sweep_s, 3),
                   "speedup_aimx_over_aim": round(aim_s / sweep_s, 2),
                   "aim_fill_ms_per_frequency": round(fill[0] / max(fill[1], 1), 2), "aim_fills": fill[1],
                   "aimx_one_time_static_fill_s": round(setup_s, 3), "near_pairs": ctx.info["near_nnz"],
                   "aim_converged": sum(1 for q in ast if q["status"] == 0),
                   "aim_iterations_mean": round(float(np.mean([q["iterations"] for q in ast])), 1),
                   "status": arc}
    # the same sweep with the AIMx CFIE (Sec. III-B): the closed sphere passes through its first
    # interior resonance (ka ~ 2.74) inside the band, where the EFIE's iteration count peaks
    cfie_cmp = None
    if not args.no_cfie:
        from paper_2009_02281_gb300 import CFIE
        cc = Context(wl["xyz"], wl["tri"], wl["grid_n"], order=wl["order"], formulation=CFIE,
                     near_radius=wl["radius"])
        cc.solve(f, cc.rhs_planewave(f, [[0.0, 0.0, 1.0]], [[1.0, 0.0, 0.0]]), tol=1e-6, inner_precision=F64)
        torch.cuda.synchronize()
        t = time.perf_counter()
        _, cst, crc = cc.sweep(freqs, [[0.0, 0.0, 1.0]], [[1.0, 0.0, 0.0]], tol=1e-6, inner_precision=F64)
        torch.cuda.synchronize()
        cfie_s = time.perf_counter() - t
        cc.close()
        it_e = [q["iterations"] for q in sst]
        it_c = [q["iterations"] for q in cst]
        cfie_cmp = {"sweep_s": round(cfie_s, 3), "solves_per_s": round(ws * len(freqs) / cfie_s, 2),
                    "converged": sum(1 for q in cst if q["status"] == 0), "status": crc,
                    "iterations_mean": round(float(np.mean(it_c)), 1), "iterations_max": int(max(it_c)),
                    "efie_iterations_max": int(max(it_e)),
                    "efie_peak_ka": round(float(freqs[int(np.argmax(it_e))] * 2 * np.pi / C0), 3),
                    "path": "generic (8 grid fields per RHS)", "alpha": 0.5}
    torch.cuda.synchronize()
    t = time.perf_counter()
    nsol = 5
    for _ in range(nsol):
        _, st, rc = ctx.solve(f, b, tol=1e-6, inner_precision=F64)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t) / nsol
    ctx.close()
    return {"workload": "pec_sphere_1920", "setup_s": round(setup_s, 3), "fp64_matvec_us": round(us, 1),
            "solve_ms": round(1e3 * dt, 2), "solves_per_s": round(ws / dt, 2), "iterations": st[0]["iterations"],
            "rel_residual": st[0]["rel_residual"], "status": rc, "sweep": sweep, "conventional_aim": aim_cmp,
            "cfie_sweep": cfie_cmp}


def measure_config3(args, ws):
    """The copper-bar sweep workload (8 bars, SIBC, eps_r 3.5 background): setup and the FP32
    product of its 8 port right-hand sides at three frequencies of the sweep, on the
    autotuned schedule.  Solves are not timed here: plain-EFIE GMRES stalls on this mesh."""
    import torch
    from synth import workloads, random_complex
    from paper_2009_02281_gb300 import Context, EFIE
    wl = workloads.conductor_bars()
    t0 = time.time()
    ctx = Context(wl["xyz"], wl["tri"], wl["grid_n"], order=wl["order"], formulation=EFIE, eps_out=wl["eps_out"],
                  near_radius=wl["radius"], sigma=wl["sigma"])
    torch.cuda.synchronize()
    setup_s = time.time() - t0
    nrhs = len(wl["ports"])
    x = torch.tensor(random_complex((nrhs, ctx.nunk), seed=33).astype(np.complex64), device="cuda")
    y = torch.empty_like(x)
    freqs = [float(wl["freqs"][k]) for k in (0, 50, 99)]
    tune = ctx.autotune(freqs[-1], nrhs) if not args.no_autotune else None
    stream = torch.cuda.current_stream()
    per = []
    for f in freqs:
        ctx.matvec(f, x, y)                  # spectra for this frequency
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(5):
            ctx.matvec(f, x, y)
        e1.record(stream)
        torch.cuda.synchronize()
        per.append(e0.elapsed_time(e1) / 5)
    ms = float(np.median(per))
    info = ctx.info
    # the sweep itself: the charge-form scalar potential (the RWG form stalls near 3e-2 on these
    # bars), the 8 unit-voltage port excitations, every tenth frequency of the 100-point log sweep,
    # all systems in one batched solve (FP64 inner products: the FP32 ones level off at ~1.2e-5)
    sweep = None
    if not args.no_config3_sweep:
        from paper_2009_02281_gb300 import Port, F64
        ports = [Port.make(*p) for p in wl["ports"]]
        t = time.time()
        ctx.set_charge_form(True)
        torch.cuda.synchronize()
        charge_setup_s = time.time() - t
        fs = np.asarray(wl["freqs"])[::10]
        torch.cuda.synchronize()
        t = time.perf_counter()
        b1 = ctx.rhs_ports(ports)
        Bb = b1.unsqueeze(0).repeat(len(fs), 1, 1).contiguous()
        X, bst, brc, cnt = ctx.sweep_batched(fs, Bb, tol=1e-5, restart=100, max_iter=args.config3_max_iter,
                                             inner_precision=F64)
        torch.cuda.synchronize()
        sw_s = time.perf_counter() - t
        Y = np.stack([ctx.port_currents(ports, X[i]) for i in range(len(fs))])   # [f][excited][measured]
        conv_f = [i for i in range(len(fs)) if all(q["status"] == 0 for q in bst[i])]
        asym = [float(np.linalg.norm(Y[i] - Y[i].T) / np.linalg.norm(Y[i])) for i in conv_f]
        nconv = sum(1 for row in bst for q in row if q["status"] == 0)
        sweep = {"formulation": "EFIE, charge-form scalar potential, surface impedance", "ports": len(ports),
                 "frequencies_hz": [float(v) for v in fs], "systems": len(fs) * len(ports),
                 "tol": 1e-5, "max_iter": args.config3_max_iter, "wall_s": round(sw_s, 2),
                 "converged": nconv, "sweep_solves_per_s": round(ws * nconv / sw_s, 3),
                 "converged_frequencies_hz": [float(fs[i]) for i in conv_f],
                 "iterations_per_frequency": [int(np.mean([q["iterations"] for q in row])) for row in bst],
                 "max_rel_residual_per_frequency": [float("%.3g" % max(q["rel_residual"] for q in row))
                                                    for row in bst],
                 "y_reciprocity_max": max(asym) if asym else None,
                 "charge_setup_s": round(charge_setup_s, 2), "cycles": cnt[0], "graphs_captured": cnt[1],
                 "status": brc}
    ctx.close()
    return {"workload": wl["name"], "n_unknowns": info["n_unknowns"], "near_nnz": info["near_nnz"],
            "grid": list(info["grid_n"]), "padded": list(info["pad"]), "setup_s": round(setup_s, 2),
            "rhs": nrhs, "ms_per_product": round(ms, 3), "value": round(ws * nrhs / (ms * 1e-3), 2), "unit": UNIT,
            "freqs_hz": freqs, "schedule": tune["best"] if tune else None, "sweep": sweep}


def learned_eval(args):
    """Learned preconditioner trained on seeded small copper-block layouts (10 mm
    region, 1-4 mm blocks, several frequencies) and evaluated on held-out larger
    layouts (20 mm region, up to 12 blocks of 1-6 mm) at held-out frequencies:
    GMRES iterations and wall time against the diagonal preconditioner."""
    import torch
    from synth import workloads, planewave_batch
    from paper_2009_02281_gb300 import Context, EFIE, Gnn, PRECOND_DIAG, PRECOND_LEARNED

    charge = args.learned_form == "charge"

    def make(w):
        c = Context(w["xyz"], w["tri"], w["grid_n"], order=2, formulation=EFIE, eps_out=1.0, sigma=w["sigma"])
        if charge:
            c.set_charge_form(True)
        return c

    train_w = [workloads.copper_blocks(s, region=10e-3, footprint=(1e-3, 4e-3)) for s in range(8)]
    train = [make(w) for w in train_w]
    samples = [(c, f) for c in train for f in (10e9, 25e9, 40e9)]
    net = Gnn(EFIE)
    net.init_params(0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = net.fit(samples, steps=args.gnn_eval_steps, nprobe=8, lr=2e-3, clip=1.0, seed=1)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    out = {"scalar_potential": "charge form (D^T Pt D)" if charge else "RWG form",
           "train_layouts": len(train), "train_unknowns": [c.nunk for c in train], "train_freqs_ghz": [10, 25, 40],
           "steps": args.gnn_eval_steps, "train_s": round(train_s, 2), "loss_first": round(losses[0], 4),
           "loss_last": round(float(np.mean(losses[-50:])), 4), "eval": []}
    dirs, pols = planewave_batch(8, seed=5)
    for seed in (100, 101):
        w = workloads.copper_blocks(seed, nblocks=12, region=20e-3)
        ctx = make(w)
        ctx.gnn_attach(net)
        for f in (15e9, 30e9, 45e9):
            b = ctx.rhs_planewave(f, dirs, pols)
            row = {"layout": seed, "unknowns": ctx.nunk, "freq_ghz": f / 1e9}
            for name, pc in (("diag", PRECOND_DIAG), ("learned", PRECOND_LEARNED)):
                torch.cuda.synchronize()
                t = time.perf_counter()
                _, st, rc = ctx.solve(f, b, tol=1e-5, restart=100, max_iter=4000, precond=pc)
                torch.cuda.synchronize()
                row[name] = {"iterations_mean": float(np.mean([s["iterations"] for s in st])),
                             "wall_s": round(time.perf_counter() - t, 3), "status": rc}
            out["eval"].append(row)
        ctx.close()
    for c in train:
        c.close()
    net.close()
    return out


def measure_batch(args, ws):
    """The first args.batch_members members of the seeded uneven batch (spheres, boxes,
    tori; PEC and dielectric; 4 RHS each): one captured graph per call versus the
    same products issued one member after another on one stream."""
    import torch
    from synth import workloads, random_complex
    from paper_2009_02281_gb300 import Batch, Context, PMCHWT, EFIE
    members = workloads.uneven_batch(n=args.batch_members)
    t0 = time.time()
    ctxs = [Context(m["xyz"], m["tri"], m["grid_n"], order=m["order"],
                    formulation=PMCHWT if m["formulation"] == "pmchwt" else EFIE,
                    eps_out=m["eps_out"], eps_in=m["eps_in"] or 1.0, near_radius=m["radius"]) for m in members]
    torch.cuda.synchronize()
    setup_s = time.time() - t0
    xs = [torch.tensor(random_complex((m["nrhs"], c.nunk), seed=700 + i).astype(np.complex64), device="cuda")
          for i, (m, c) in enumerate(zip(members, ctxs))]
    ys = [torch.empty_like(x) for x in xs]
    freqs = [m["freq"] for m in members]
    stream = torch.cuda.current_stream()
    batch = Batch(ctxs)
    batch.matvec(freqs, xs, ys)              # capture
    for _ in range(2):
        batch.matvec(freqs, xs, ys)
        for c, f, x, y in zip(ctxs, freqs, xs, ys):
            c.matvec(f, x, y)
    torch.cuda.synchronize()
    reps = 5
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record(stream)
    for _ in range(reps):
        batch.matvec(freqs, xs, ys)
    e[1].record(stream)
    for _ in range(reps):
        for c, f, x, y in zip(ctxs, freqs, xs, ys):
            c.matvec(f, x, y)
    e[2].record(stream)
    torch.cuda.synchronize()
    ms_graph = _barrier_max(e[0].elapsed_time(e[1]) / reps, ws, device="cuda")
    ms_seq = _barrier_max(e[1].elapsed_time(e[2]) / reps, ws, device="cuda")
    # per-member schedules from the autotuner (one cache for the batch: members of the same
    # shape reuse the first one's choice), then the same graph timing again
    tuned = None
    if not args.no_autotune:
        import tempfile
        fd, cache = tempfile.mkstemp(prefix="aimx_tune_", suffix=".txt")
        os.close(fd)
        t0 = time.time()
        picks = {}
        hits = 0
        for c, f, m in zip(ctxs, freqs, members):
            r = c.autotune(f, m["nrhs"], cache_path=cache)
            hits += 0 if r["tried"] else 1
            k = "variant%d_pass%d" % (r["best"]["variant"], r["best"]["pass"])
            picks[k] = picks.get(k, 0) + 1
        tune_s = time.time() - t0
        os.remove(cache)
        batch.matvec(freqs, xs, ys)          # recapture with the tuned schedules
        for _ in range(2):
            batch.matvec(freqs, xs, ys)
        torch.cuda.synchronize()
        e[2].record(stream)
        for _ in range(reps):
            batch.matvec(freqs, xs, ys)
        e[3].record(stream)
        torch.cuda.synchronize()
        ms_tuned = _barrier_max(e[2].elapsed_time(e[3]) / reps, ws, device="cuda")
        # members are tuned alone; inside the concurrent graph keep their choices only if the
        # whole call got faster
        kept = ms_tuned < ms_graph
        if not kept:
            for c in ctxs:
                c.set_schedule(0, 0)
        tuned = {"ms_per_call": round(ms_tuned, 3), "speedup_vs_default": round(ms_graph / ms_tuned, 3),
                 "tune_s": round(tune_s, 2), "cache_hits": hits, "schedules": picks,
                 "kept": bool(kept)}
    rhs = sum(m["nrhs"] for m in members)
    step_bytes = 0.0
    bins = {}
    for m, c in zip(members, ctxs):
        b, _ = _algorithmic_bytes(c.info, m, m["nrhs"])
        step_bytes += b
        key = "<5k" if c.nunk < 5000 else ("5k-20k" if c.nunk < 20000 else ">=20k")
        d = bins.setdefault(key, {"members": 0, "unknowns": 0})
        d["members"] += 1
        d["unknowns"] += c.nunk
    hbm, peak_kind = _peaks()
    ach = step_bytes / (ms_graph * 1e-3) / 1e9
    out = {"members": len(members), "rhs_per_call": rhs, "unknowns_total": int(sum(c.nunk for c in ctxs)),
           "value": round(ws * rhs / (ms_graph * 1e-3), 2), "unit": UNIT, "ms_per_call": round(ms_graph, 3),
           "sequential_ms_per_call": round(ms_seq, 3), "speedup_vs_sequential": round(ms_seq / ms_graph, 3),
           "graph_nodes": batch.graph_nodes, "setup_s": round(setup_s, 2),
           "roofline": {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
                        "frac": round(ach / hbm, 4), "peak_kind": "of " + peak_kind,
                        "algorithmic_bytes_per_call": step_bytes},
           "size_bins": bins, "autotuned": tuned}
    batch.close()
    for c in ctxs:
        c.close()
    return out


def run_ours(args):
    import torch
    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from synth import workloads, random_complex
    from paper_2009_02281_gb300 import Context, build, PMCHWT, EFIE, F32
    build.build()
    wl = workloads.WORKLOADS[args.workload]() if args.nrhs is None else \
        workloads.WORKLOADS[args.workload](nrhs=args.nrhs)
    B = wl["nrhs"]
    t0 = time.time()
    ctx = Context(wl["xyz"], wl["tri"], wl["grid_n"], order=wl["order"],
                  formulation=PMCHWT if wl["formulation"] == "pmchwt" else EFIE,
                  eps_out=wl["eps_out"], eps_in=wl["eps_in"] or 1.0, near_radius=wl["radius"])
    torch.cuda.synchronize()
    setup_s = time.time() - t0
    ctx.set_path(args.path)
    info = ctx.info
    x_np = random_complex((B, ctx.nunk), seed=100 + rank).astype(np.complex64)
    x = torch.tensor(x_np, device="cuda")
    y = torch.empty_like(x)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    freq = wl["freq"]
    # kernel generation for this frequency, timed once
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    ctx.matvec(freq, x, y)
    ev1.record(stream)
    torch.cuda.synchronize()
    first_ms = ev0.elapsed_time(ev1)
    # product schedule for this workload (kernel variant x RHS per pass), timed on the GPU
    tune = None
    if not args.no_autotune and args.path == 0:
        t0 = time.time()
        tune = ctx.autotune(freq, B)
        tune["tune_s"] = round(time.time() - t0, 2)
    for _ in range(args.warmup):
        flush.fill_(1.0)
        ctx.matvec(freq, x, y)
    torch.cuda.synchronize()
    # timed region
    clocks = Clocks(local)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ctx.profile(True)
    ctx.profile_read()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for k in range(args.steps):
        flush.fill_(1.0)                      # evict L2 between steps (not timed)
        starts[k].record(stream)
        ctx.matvec(freq, x, y)
        ends[k].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    prof = ctx.profile_read()
    ctx.profile(False)
    total_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    total_ms = _barrier_max(total_ms, ws, device="cuda")
    launches = sum(c for _, c in prof.values())

    # end-to-end through the public host-buffer call (pinned host memory, copies inside)
    xh = torch.tensor(x_np).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    for _ in range(2):
        ctx.matvec_host_ptr(freq, B, xh.data_ptr(), yh.data_ptr(), F32, stream)
    torch.cuda.synchronize()
    e2e_steps = max(1, min(args.steps, 10))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ctx.matvec_host_ptr(freq, B, xh.data_ptr(), yh.data_ptr(), F32, stream)
    torch.cuda.synchronize()
    e2e_s = _barrier_max(time.perf_counter() - t0, ws, device="cuda")

    # FP64 products (generic radix-2 path, the precision of the paper's solver) on a sub-batch
    fp64 = None
    if not args.no_fp64:
        nb64 = min(B, 8)
        x64 = torch.tensor(x_np[:nb64].astype(np.complex128), device="cuda")
        y64 = torch.empty_like(x64)
        ctx.matvec(freq, x64, y64)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 3
        e0.record(stream)
        for _ in range(reps):
            ctx.matvec(freq, x64, y64)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1) / reps
        fp64 = {"value": round(ws * nb64 / (ms64 * 1e-3), 2), "unit": UNIT, "rhs_per_call": nb64,
                "ms_per_call": round(ms64, 3), "path": "generic FP64, shared-memory line FFTs on the 128^3 pad (kernel spectra FP64)"}
        del x64, y64

    # the plain comparison path on the same GPU: generic projection / interpolation with cuFFT
    # transforms of the full padded grids, FP32 and FP64, on a sub-batch
    plain = None
    if not args.no_fp64:
        plain = {}
        nbp = min(B, 8)
        ctx.set_path(2)
        for name, dt in (("fp32", torch.complex64), ("fp64", torch.complex128)):
            xp = torch.tensor(x_np[:nbp], dtype=dt, device="cuda")
            yp = torch.empty_like(xp)
            ctx.matvec(freq, xp, yp)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(3):
                ctx.matvec(freq, xp, yp)
            e1.record(stream)
            torch.cuda.synchronize()
            msp = e0.elapsed_time(e1) / 3
            plain[name] = {"value": round(ws * nbp / (msp * 1e-3), 2), "unit": UNIT, "rhs_per_call": nbp,
                           "ms_per_call": round(msp, 3)}
            del xp, yp
        ctx.set_path(args.path)
        plain["path"] = "generic projection/interpolation + cuFFT full 3-D transforms (comparison only)"
        plain["fused_fp32_speedup"] = round((ws * B / (total_ms / args.steps * 1e-3)) / plain["fp32"]["value"], 2)

    # the linear-term modification (Sec. III-A-3) on the same product: its one-time build and
    # the product time with the term on (L2 flushed between steps like the timed region)
    linterm = None
    if not args.no_linear_term:
        t0 = time.time()
        ctx.set_linear_term(True)
        build_s = time.time() - t0
        nl = len(ctx.export_linear_term()["cols"])
        ctx.matvec(freq, x, y)
        reps = max(3, min(args.steps, 10))
        st = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
        en = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
        for k in range(reps):
            flush.fill_(1.0)
            st[k].record(stream)
            ctx.matvec(freq, x, y)
            en[k].record(stream)
        torch.cuda.synchronize()
        ms_on = sum(a.elapsed_time(b) for a, b in zip(st, en)) / reps
        ctx.set_linear_term(False)
        linterm = {"value": round(ws * B / (ms_on * 1e-3), 2), "unit": UNIT, "ms_per_step": round(ms_on, 4),
                   "overhead_vs_off": round(ms_on / (total_ms / args.steps) - 1.0, 4),
                   "overlapping_pairs": nl, "build_s": round(build_s, 3)}

    hbm, peak_kind = _peaks()
    step_bytes, stage_bytes = _algorithmic_bytes(info, wl, B)
    dom = max(prof.items(), key=lambda kv: kv[1][0])[0] if prof else None
    roof = None
    if dom in stage_bytes:
        avg_ms = prof[dom][0] / prof[dom][1]
        ach = stage_bytes[dom] / (avg_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(ach / hbm, 4), "peak_kind": "of " + peak_kind,
                "traffic": _traffic_record(dom, args.workload),
                "algorithmic_bytes_per_launch": stage_bytes[dom], "avg_launch_ms": round(avg_ms, 4)}
    ms_per_step = total_ms / args.steps
    step_gbs = step_bytes / (ms_per_step * 1e-3) / 1e9
    value = ws * B * args.steps / (total_ms * 1e-3)
    out = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64 (f32)", "data": "synthetic",
        "config": {"workload": args.workload, "n_unknowns": ctx.nunk, "n_basis": ctx.N,
                   "rhs_per_step": B, "grid": list(info["grid_n"]), "padded": list(info["pad"]),
                   "order": info["order"], "near_nnz": info["near_nnz"], "freq_hz": freq,
                   "formulation": wl["formulation"], "l2": "flushed between steps (512 MiB write)",
                   "path": "plane-fused" if ctx.matvec_path(F32) == 0 else "generic",
                   "parallelism": "replicas" if ws > 1 else "single"},
        "roofline": roof,
        "step_roofline": {"algorithmic_bytes": step_bytes, "achieved_gbs": round(step_gbs, 1),
                          "frac": round(step_gbs / hbm, 4)},
        "stages_ms": {k: [round(v[0] / args.steps, 4), v[1]] for k, v in prof.items()},
        "e2e": {"value": round(ws * B * e2e_steps / e2e_s, 2), "unit": UNIT,
                "h2d_bytes_per_step": int(x_np.nbytes), "d2h_bytes_per_step": int(x_np.nbytes)},
        "gpu_launches": launches,
        "fp64": fp64,
        "plain_cufft": plain,
        "linear_term": linterm,
        "autotune": tune,
        "clocks": clk,
        "setup_s": round(setup_s, 3),
        "first_call_ms_incl_kernel_generation": round(first_ms, 3),
    }
    if not args.no_solves:
        out["solves"] = measure_solves(ctx, wl, args)
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(wl, args.cpu_rows, ctx, args.path)
    if args.batch_members > 0:
        ctx.close()
        out["uneven_batch"] = measure_batch(args, ws)
    if not args.no_config1:
        out["pec_sphere_1920"] = measure_config1(args, ws)
    if not args.no_config3:
        out["conductor_bars"] = measure_config3(args, ws)
    if not args.no_learned_eval:
        out["learned_generalisation"] = learned_eval(args)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if args.batch_members <= 0:
        ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


class OracleSample:
    """The FP64 oracle (direct grid summation) on sampled rows of one matvec of the workload."""

    def __init__(self, wl, rows):
        from oracle import operator as op
        from synth import random_complex
        self.op = op
        self.wl = wl
        nb = len(wl["tri"]) * 3 // 2
        self.rows = (np.arange(rows) * 997 + 13) % nb
        self.prob = op.setup(wl["xyz"], wl["tri"], wl["order"], wl["grid_n"], radius=wl["radius"],
                             near_rows=self.rows)
        self.x = random_complex(self.prob["N"] * (2 if wl["formulation"] == "pmchwt" else 1), seed=5)

    def run(self, rows):
        """Time the oracle on the given subset of sampled basis rows; returns (output rows, seconds)."""
        wl, op = self.wl, self.op
        t0 = time.perf_counter()
        if wl["formulation"] == "pmchwt":
            y = op.matvec_pmchwt(self.prob, wl["freq"], self.x, wl["eps_out"], wl["eps_in"], rows=rows)
            nout = 2 * len(rows)
        else:
            y = op.matvec_efie(self.prob, wl["freq"], self.x, wl["eps_out"], rows=rows)
            nout = len(rows)
        self.y = y
        return nout, time.perf_counter() - t0

    def sampled(self, y_full):
        """The sampled rows of a full product vector, in the oracle's output order."""
        if self.wl["formulation"] == "pmchwt":
            n = len(y_full) // 2
            return np.concatenate([y_full[self.rows], y_full[n + self.rows]])
        return y_full[self.rows]


def cpu_baseline(wl, rows, ctx=None, path=0):
    """The oracle timed on sampled rows; with ctx, also the GPU products' errors on those rows
    (the timed FP32 product, and FP32 / FP64 on the generic and cuFFT comparison paths; the
    context is returned to product path ``path``)."""
    s = OracleSample(wl, rows)
    nout, dt = s.run(s.rows)
    nunk = len(s.x)
    out = {"value": nout / nunk / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
           "sample": "%d of %d output rows of one matvec (%s) by direct grid summation, %.1f s, numpy "
                     "default threading; value = rows/s divided by rows per matvec" % (nout, nunk, wl["name"], dt)}
    if ctx is not None:
        import torch
        from paper_2009_02281_gb300 import F32
        x32 = torch.tensor(s.x[None].astype(np.complex64), device="cuda")
        x64 = torch.tensor(s.x[None].astype(np.complex128), device="cuda")

        def err(x):
            y = ctx.matvec(wl["freq"], x).cpu().numpy()[0].astype(np.complex128)
            return float(np.linalg.norm(s.sampled(y) - s.y) / np.linalg.norm(s.y))

        out["gpu_fp32_rel_err_on_sample"] = err(x32)
        errs = {("fp32_plane_fused" if ctx.matvec_path(F32) == 0 else "fp32_generic"): out["gpu_fp32_rel_err_on_sample"]}
        ctx.set_path(1)
        errs["fp32_generic"] = err(x32)
        errs["fp64_generic"] = err(x64)
        ctx.set_path(2)
        errs["fp32_cufft"] = err(x32)
        errs["fp64_cufft"] = err(x64)
        ctx.set_path(path)
        out["gpu_rel_err_on_sample_by_path"] = errs
    out["host"] = host_cpu()
    out["single_thread"] = oracle_single_thread(wl, max(2, rows // 8))
    out["fast_cpu_reference"] = fast_cpu_reference(s)
    return out


def host_cpu():
    """Host CPU model and logical core count (lscpu, else /proc/cpuinfo)."""
    import platform
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None and os.path.exists("/proc/cpuinfo"):
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                model = line.split(":", 1)[1].strip()
                break
    return {"nproc": os.cpu_count(), "model": model, "machine": platform.machine()}


_SINGLE_THREAD_CHILD = """
import json, sys
import bench
from synth import workloads
wl = workloads.WORKLOADS[sys.argv[1]]()
s = bench.OracleSample(wl, int(sys.argv[2]))
nout, dt = s.run(s.rows)
print(json.dumps({"nout": nout, "nunk": len(s.x), "s": dt}))
"""


def oracle_single_thread(wl, rows):
    """The oracle sample with one BLAS / OpenMP thread, in a fresh interpreter (thread pools are
    sized when numpy loads); returns {value, sample} or {error}."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               OMP_THREAD_LIMIT="1")
    try:
        r = subprocess.run([sys.executable, "-c", _SINGLE_THREAD_CHILD, wl["name"], str(rows)], env=env, cwd=ROOT,
                           capture_output=True, text=True, timeout=900)
        d = json.loads(r.stdout.strip().splitlines()[-1])
    except (OSError, subprocess.SubprocessError, ValueError, IndexError) as e:
        return {"error": "single-thread oracle run failed: %s" % str(e)[:200]}
    return {"value": d["nout"] / d["nunk"] / d["s"], "unit": UNIT, "cores": 1,
            "sample": "%d of %d output rows, %.1f s, one thread" % (d["nout"], d["nunk"], d["s"])}


class FastCpuAIMx:
    """An FP64 AIMx product on the host cores with NumPy and scipy.fft: a timing baseline for
    the GPU product (a reasonably fast CPU program), not the oracle and not a fallback.

    Projection by bincount onto the zero-padded (2N)^3 grid, forward FFTs of the projected
    fields, the kernel spectra of every region combined per output field in the spectral domain
    (scalar kernel for the vector and scalar potentials, the gradient kernel's cross product for
    K), inverse FFTs of the output fields, interpolation by gather (W = P^T).  Kernel tables are
    the oracle's (sampled G and grad G over all offsets, Eqs. Hmn and Hmm), embedded in the
    circulant grid at offset mod 2N; their spectra are computed once per frequency.

    The near correction is a CSR SpMV over the full near pattern with three value arrays (N^A,
    N^Phi, N^K).  Only the sampled rows' near values exist on the host (integrating all of them in
    Python would take far longer than the product), so the timed SpMV runs on placeholder values
    of the true pattern and the accuracy check uses the exact near rows of the sample."""

    def __init__(self, sample, workers):
        import scipy.fft as sfft
        import scipy.sparse as sp
        from oracle import greens, grid as gridmod
        self.sfft, self.workers = sfft, workers
        self.s = sample
        wl, prob = sample.wl, sample.prob
        self.pmchwt = wl["formulation"] == "pmchwt"
        g = prob["grid"]
        Nx, Ny, Nz = g["n"]
        self.M = (2 * Nz, 2 * Ny, 2 * Nx)
        off = gridmod.stencil_offsets(g["order"])
        node = prob["anc"][:, None, :] + off[None, :, :]
        self.flat = ((node[..., 2] * self.M[1] + node[..., 1]) * self.M[2] + node[..., 0]).ravel()
        self.lam = prob["lam"]
        self.N = prob["N"]
        w = 2.0 * np.pi * wl["freq"]
        self.w = w
        self.regions = sample.op.materials(wl["freq"], wl["eps_out"], wl["eps_in"] if self.pmchwt else None)[1]
        t0 = time.perf_counter()
        idx = [np.arange(-(n - 1), n) % m for n, m in zip((Nz, Ny, Nx), self.M)]
        self.spec = []
        for mu, eps, k in self.regions:
            H = np.zeros(self.M, dtype=np.complex128)
            H[np.ix_(*idx)] = greens.kernel_table(k, g["n"], g["h"])
            Hs = sfft.fftn(H, workers=workers)
            Gs = None
            if self.pmchwt:
                Gt = greens.grad_kernel_table(k, g["n"], g["h"])
                Gs = np.zeros((3,) + self.M, dtype=np.complex128)
                for a in range(3):
                    Gs[a][np.ix_(*idx)] = Gt[a]
                Gs = sfft.fftn(Gs, axes=(1, 2, 3), workers=workers)
            self.spec.append((mu, eps, k, Hs, Gs))
        self.spectra_s = time.perf_counter() - t0
        rng = np.random.default_rng(11)
        pat = (np.ones(len(prob["cols"])), prob["cols"], prob["row_ptr"])
        self.near_pattern = sp.csr_matrix(pat, shape=(self.N, self.N))
        self.near_vals = [rng.standard_normal(self.near_pattern.nnz) for _ in range(3)]

    def _project(self, x):
        size = self.M[0] * self.M[1] * self.M[2]
        g = np.empty((4,) + self.M, dtype=np.complex128)
        for f in range(4):
            wts = (self.lam[:, :, f] * x[:, None]).ravel()
            g[f] = (np.bincount(self.flat, weights=wts.real, minlength=size)
                    + 1j * np.bincount(self.flat, weights=wts.imag, minlength=size)).reshape(self.M)
        return self.sfft.fftn(g, axes=(1, 2, 3), workers=self.workers)

    def _interp(self, O):
        o = self.sfft.ifftn(O, axes=(1, 2, 3), workers=self.workers).reshape(4, -1)
        nu = self.lam.shape[1]
        return sum(np.einsum("nu,nu->n", self.lam[:, :, f], o[f][self.flat].reshape(-1, nu)) for f in range(4))

    @staticmethod
    def _cross(G, F):
        return np.stack([G[1] * F[2] - G[2] * F[1], G[2] * F[0] - G[0] * F[2], G[0] * F[1] - G[1] * F[0]])

    def far(self, x):
        """The grid part W H P x of every output row (E rows, then H rows for the two-region form)."""
        from oracle.constants import ETA0
        w, N = self.w, self.N
        if not self.pmchwt:
            mu, eps, k, Hs, _ = self.spec[0]
            FJ = self._project(x)
            O = np.empty_like(FJ)
            O[:3] = (1j * w * mu) * Hs * FJ[:3]
            O[3] = (-1j * w * mu / k ** 2) * Hs * FJ[3]
            return self._interp(O)
        FJ, FM = self._project(x[:N]), self._project(x[N:])
        OE = np.zeros_like(FJ)
        OH = np.zeros_like(FJ)
        for mu, eps, k, Hs, Gs in self.spec:
            OE[:3] += (1j * w * mu) * Hs * FJ[:3] + ETA0 * self._cross(Gs, FM[:3])
            OE[3] += (-1j * w * mu / k ** 2) * Hs * FJ[3]
            OH[:3] += (ETA0 ** 2 * 1j * w * eps) * Hs * FM[:3] - ETA0 * self._cross(Gs, FJ[:3])
            OH[3] += (-ETA0 ** 2 * 1j * w * eps / k ** 2) * Hs * FM[3]
        return np.concatenate([self._interp(OE), self._interp(OH)])

    def near_placeholder(self, x):
        """Cost stand-in for the near correction: three CSR products per input vector block."""
        A = self.near_pattern
        ys = []
        for xs in ((x,) if not self.pmchwt else (x[:self.N], x[self.N:])):
            for v in self.near_vals:
                A.data = v
                ys.append(A @ xs)
        return ys

    def near_exact_rows(self, x):
        """The exact near correction on the sampled rows (the oracle's integrals of those rows)."""
        from oracle.constants import ETA0
        op, prob, rows, w, N = self.s.op, self.s.prob, self.s.rows, self.w, self.N
        if not self.pmchwt:
            mu, eps, k, _, _ = self.spec[0]
            return 1j * w * mu * (op.near_apply(prob, "NA", x, rows) - op.near_apply(prob, "NP", x, rows) / k ** 2)
        nJ = {c: op.near_apply(prob, c, x[:N], rows) for c in ("NA", "NP", "NK")}
        nM = {c: op.near_apply(prob, c, x[N:], rows) for c in ("NA", "NP", "NK")}
        yE, yH = 0.0, 0.0
        for mu, eps, k, _, _ in self.spec:
            yE = yE + 1j * w * mu * (nJ["NA"] - nJ["NP"] / k ** 2) + ETA0 * nM["NK"]
            yH = yH - ETA0 * nJ["NK"] + ETA0 ** 2 * 1j * w * eps * (nM["NA"] - nM["NP"] / k ** 2)
        return np.concatenate([yE, yH])


def fast_cpu_reference(sample, reps=3):
    """Time FastCpuAIMx on the sample's workload and check it on the oracle's sampled rows."""
    workers = os.cpu_count() or 1
    t0 = time.perf_counter()
    fc = FastCpuAIMx(sample, workers)
    setup_s = time.perf_counter() - t0
    times = []
    for _ in range(reps):
        t = time.perf_counter()
        yf = fc.far(sample.x)
        fc.near_placeholder(sample.x)
        times.append(time.perf_counter() - t)
    y_rows = sample.sampled(yf) + fc.near_exact_rows(sample.x)
    err = float(np.linalg.norm(y_rows - sample.y) / np.linalg.norm(sample.y))
    ms = float(np.median(times))
    return {"value": 1.0 / ms, "unit": UNIT, "cores": workers, "kind": "numpy + scipy.fft FP64 timing baseline",
            "sample": "one full single-RHS product, median of %d; kernel spectra once per frequency "
                      "(%.2f s, not timed per product); near SpMV on placeholder values of the true "
                      "pattern (%d entries x 3)" % (reps, fc.spectra_s, len(fc.near_vals[0])),
            "ms_per_matvec": round(1e3 * ms, 1), "setup_s": round(setup_s, 2),
            "rel_err_vs_oracle_on_sample": err}


def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return
    from synth import workloads
    wl = workloads.WORKLOADS[args.workload]()
    samp = OracleSample(wl, max(1, args.steps))      # warm-up: oracle setup (not timed)
    nunk = len(samp.x)
    rates, t_all = [], 0.0
    for k in range(args.steps):
        nout, dt = samp.run(samp.rows[k:k + 1])      # one basis row per step
        rates.append(nout / nunk / dt)
        t_all += dt
    value = float(np.median(rates))
    sample = ("one basis row (%d output rows) of one matvec per step (%s), direct grid summation, numpy "
              "default threading; value = median rows/s divided by %d rows per matvec"
              % (2 if wl["formulation"] == "pmchwt" else 1, wl["name"], nunk))
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(1e3 * t_all / max(1, args.steps), 1), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "c128 (f64)", "data": "synthetic", "impl": "reference",
           "config": {"workload": args.workload},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                            "sample": sample, "host": host_cpu()},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="dielectric_sphere_61440")
    ap.add_argument("--nrhs", type=int, default=None)
    ap.add_argument("--cpu-rows", type=int, default=32)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solves", action="store_true", help="skip the batched solve measurement")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 product measurement")
    ap.add_argument("--no-config1", action="store_true", help="skip the 1920-unknown FP64 latency measurement")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default product schedules")
    ap.add_argument("--no-config3", action="store_true", help="skip the copper-bar product measurement")
    ap.add_argument("--no-config3-sweep", action="store_true", help="skip the copper-bar batched port sweep")
    ap.add_argument("--config3-max-iter", type=int, default=800,
                    help="GMRES iteration cap per system of the copper-bar sweep")
    ap.add_argument("--no-cfie", action="store_true", help="skip the CFIE sweep of the 1920-unknown sphere")
    ap.add_argument("--no-aim", action="store_true",
                    help="skip the conventional-AIM sweep of the 1920-unknown sphere")
    ap.add_argument("--no-linear-term", action="store_true",
                    help="skip the product timing with the linear-term modification on")
    ap.add_argument("--no-learned-eval", action="store_true",
                    help="skip training on small copper layouts and evaluating on held-out larger ones")
    ap.add_argument("--gnn-eval-steps", type=int, default=1500, help="training steps of the generalisation study")
    ap.add_argument("--learned-form", default="charge", choices=["charge", "rwg"],
                    help="scalar-potential form of the generalisation study's contexts")
    ap.add_argument("--batch-members", type=int, default=48,
                    help="members of the seeded uneven batch to time (0 = skip; 48 = the full batch)")
    ap.add_argument("--path", type=int, default=0, choices=[0, 1], help="product path for the timed steps (aimx_set_path)")
    ap.add_argument("--solve-tol", type=float, default=1e-5)
    ap.add_argument("--plain-rhs", type=int, default=4,
                    help="right-hand sides of the plain FP64 cuFFT solve comparison (0 skips it)")
    ap.add_argument("--gnn-steps", type=int, default=600, help="training steps of the learned preconditioner")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
