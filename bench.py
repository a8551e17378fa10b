"""Benchmark of the domain-wall multigrid hot path on one GB300 (or N replicas).

Prints ONE JSON line (rank 0).  Metric: fine D_DW HBM bandwidth (algorithmic
GB/s, % of the measured HBM peak), with the time to a 1e-10 true residual of
the mixed-precision MG solve versus FP64 CGNE on the 256x256 x Ls=16 workload
reported alongside.

  value        fine D_DW apply (FP32 spinors, FP16 links) on the 1024x1024 x Ls=16
               U(1) lattice (537 MB of algorithmic traffic per apply, larger than
               L2), whole-job GB/s over N ranks; L2 flushed before every timed apply
  e2e          the same apply through the C ABI from pinned host buffers: H2D of
               psi and links, apply, D2H of the result, all inside the timed region
  roofline     the apply kernel: algorithmic bytes / CUDA-event duration vs the
               measured HBM copy bandwidth
  solve        256x256 x Ls=16 (sigma 0.7, M5 1, m 0.005; and the paper-like sigma 0.214):
               FP64 CGNE, BiCGStab-6, the two-level and the deflated three-level
               K-cycle, each to ||b - D x|| / ||b|| <= 1e-10, wall time on the same GPU
  cpu_baseline the FP64 oracle's CSR apply on the host cores, bounded sample

--impl reference times the FP64 CPU oracle (the only reference this method
has) on the same metric and prints the same line with "impl": "reference".
"""
from __future__ import annotations

import argparse
import hashlib
import ctypes
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "D_dw HBM GB/s (% peak); MG vs CGNE time to 1e-10 residual, same GPU"
APPLY_WL = synth.SCHWINGER_1024
SOLVE_WL = synth.SCHWINGER_256
# Wilson setup mass near the critical mass of the synthetic fields: minus the
# smallest real part of spec D_W(U, 0), estimated once offline on 64^2 samples
# of each link-angle width (0.31-0.39 for sigma 0.7, 0.19-0.20 for 0.5).
SETUP_MASS = {0.7: -0.3, 0.5: -0.19, 0.214: -0.035}
# 4-d SU(3), eps 0.3: the smallest real part of spec D_W(U, 0) is 0.443 (scipy on 6^4 and 8^4
# samples of the same ensemble), so the setup relaxes at m_s = -0.42, just above critical
SETUP_MASS_SU3 = -0.42
E2E_CHUNKS = (1, 4, 16)   # s-chunk counts of dwf_apply_host tried; the fastest is the e2e figure
# algorithmic bytes per 5-d site of the FP32-spinor / FP16-link 2-d apply:
# read psi (2 complex64 = 16 B) + write out (16 B) + 2 links x 4 B shared by Ls slices
def apply_bytes(V, Ls, spinor_b=16, link_b=4):
    return V * Ls * 2 * spinor_b + 2 * V * link_b


def env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


class Ranks:
    """Process-group plumbing of the benchmark: one process per GPU (replicas),
    launched by torchrun.  barrier() + device sync brackets every timed region,
    max() takes the slowest rank's time, and only rank 0 prints."""

    def __init__(self, backend="nccl", device=None):
        self.world = env_int("WORLD_SIZE", 1)
        self.rank = env_int("RANK", 0)
        self.local = env_int("LOCAL_RANK", 0)
        self.device = device
        self.dist = None
        if self.world > 1:
            import torch.distributed as dist
            kw = {"device_id": device} if (backend == "nccl" and device is not None) else {}
            dist.init_process_group(backend, **kw)
            self.dist = dist

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()
        if self.device is not None and self.device.type == "cuda":
            import torch
            torch.cuda.synchronize(self.device)

    def max(self, x: float) -> float:
        if self.dist is None:
            return float(x)
        import torch
        dev = self.device if self.device is not None else torch.device("cpu")
        t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def whole_job_rate(self, units_per_rank: float, seconds_this_rank: float) -> float:
        """Units processed by all ranks / the slowest rank's time (weak scaling)."""
        return self.world * units_per_rank / self.max(seconds_this_rank)

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def kernel_traffic():
    """Per-launch DRAM traffic of the apply kernel from the committed ncu summary,
    or None if the kernel source changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "k_dwf2d_f32l16_1024x1024_Ls16.md")
    src = os.path.join(ROOT, "paper_2004_07732_gb300", "csrc", "dwf_fine.cu")
    try:
        txt = open(path).read()
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    vals = {}
    for line in txt.splitlines():
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_source_sha256_16") != sha:
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


_ORACLE_CACHE = {}


def cpu_oracle_apply(budget_s=12.0):
    """Time the FP64 oracle's CSR apply of D_DW on the host (bounded sample)."""
    from oracle import dirac
    wl = SOLVE_WL
    if "D" not in _ORACLE_CACHE:
        U, srcs = wl.draw(1)
        _ORACLE_CACHE["D"] = dirac.dwf_matrix(U, wl.dims, wl.Ls, wl.M5, wl.mf)
        _ORACLE_CACHE["b"] = srcs[0].reshape(-1)
    D, b = _ORACLE_CACHE["D"], _ORACLE_CACHE["b"]
    D @ b
    reps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        D @ b
        reps += 1
    t = (time.perf_counter() - t0) / reps
    gbs = apply_bytes(wl.V, wl.Ls, 32, 16) / t / 1e9
    return {"value": gbs, "unit": "GB/s", "cores": 1, "kind": "oracle", "precision": "f64",
            "sample": f"scipy CSR matvec (single-threaded) of the FP64 D_DW on {wl.dims[0]}x{wl.dims[1]}xLs{wl.Ls} "
                      f"(1/16 of the bench lattice), {reps} reps in {budget_s:.0f} s, charged the FP64 algorithmic "
                      f"bytes per 5-d site (32 B in, 32 B out, 2 x 16 B links / Ls)",
            "seconds_per_apply": t, "seconds_per_site_apply": t / (wl.V * wl.Ls), "host_cpus": os.cpu_count()}


def run_reference(args):
    rank = env_int("RANK", 0)
    if rank != 0:
        return
    per = []
    base = None
    for i in range(args.warmup + args.steps):
        r = cpu_oracle_apply(budget_s=4.0 if i >= args.warmup else 1.0)
        if i >= args.warmup:
            per.append(r["seconds_per_apply"])
            base = r
    t = float(np.mean(per))
    v = apply_bytes(SOLVE_WL.V, SOLVE_WL.Ls, 32, 16) / t / 1e9
    base["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{APPLY_WL.name} D_DW apply (oracle sample {SOLVE_WL.name})",
                       "l2": "oracle runs on the host"},
            "cpu_baseline": base,
            "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import paper_2004_07732_gb300 as dw

    world = env_int("WORLD_SIZE", 1)
    local = env_int("LOCAL_RANK", 0)
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    ranks = Ranks("nccl", dev)
    rank = ranks.rank
    dw.lib()
    stream = torch.cuda.current_stream(dev)
    barrier = ranks.barrier
    max_over_ranks = ranks.max

    # ---------------- fine apply bandwidth (value) ----------------
    wl = APPLY_WL
    g = dw.make_geom(wl.dims, wl.Ls)
    U, srcs = wl.draw(1)
    U64 = torch.from_numpy(U.reshape(-1)).to(dev)
    Ud = dw.links_to(g, U64, "f32_l16")
    psi_h = torch.from_numpy(srcs[0].reshape(-1).astype(np.complex64)).pin_memory()
    psi = psi_h.to(dev)
    out = torch.empty_like(psi)
    del U64
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 512 MB > L2
    nbytes = apply_bytes(wl.V, wl.Ls)
    for _ in range(args.warmup):
        flush.fill_(1.0)
        dw.dwf_apply(g, Ud, psi, out, wl.M5, wl.mf, prec="f32_l16")
    barrier()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clk = ClockSampler(dev.index).__enter__()
    for a, b in evs:
        flush.fill_(1.0)
        a.record(stream)
        dw.dwf_apply(g, Ud, psi, out, wl.M5, wl.mf, prec="f32_l16")
        b.record(stream)
    barrier()
    times = [a.elapsed_time(b) * 1e-3 for a, b in evs]
    t_apply = max_over_ranks(float(np.mean(times)))
    value = world * nbytes / t_apply / 1e9
    launches = args.steps

    # ---------------- e2e through host buffers ----------------
    # dwf_apply_host: links and spinors from pinned host memory, result back to host memory,
    # the copies pipelined with the apply over s-chunks; each step ends with a synchronize
    out_h = torch.empty_like(psi_h).pin_memory()
    Ud_h = Ud.cpu().pin_memory()
    e2e_steps = max(3, args.steps // 4)

    def e2e_host_call(nchunks):
        def fn():
            dw.dwf_apply_host(g, Ud_h, psi_h, out_h, Ud, psi, out, wl.M5, wl.mf, prec="f32_l16", nchunks=nchunks)
            torch.cuda.synchronize(dev)
        return fn

    def e2e_serial():
        Ud.copy_(Ud_h, non_blocking=True)
        psi.copy_(psi_h, non_blocking=True)
        dw.dwf_apply(g, Ud, psi, out, wl.M5, wl.mf, prec="f32_l16")
        out_h.copy_(out, non_blocking=True)
        torch.cuda.synchronize(dev)

    t_e2e_by = {}
    for name, fn in [("serial", e2e_serial)] + [(f"host_call_{c}", e2e_host_call(c)) for c in E2E_CHUNKS]:
        for _ in range(max(1, args.warmup // 2)):
            fn()
        barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            fn()
        t_e2e_by[name] = max_over_ranks((time.perf_counter() - t0) / e2e_steps)
    e2e_best = min(E2E_CHUNKS, key=lambda c: t_e2e_by[f"host_call_{c}"])
    t_e2e = t_e2e_by[f"host_call_{e2e_best}"]
    h2d = psi_h.numel() * psi_h.element_size() + Ud_h.numel() * Ud_h.element_size()
    d2h = out_h.numel() * out_h.element_size()
    del flush, out_h, Ud_h, psi, out, Ud, psi_h

    # ---------------- 4-d SU(3) apply (16^3 x 32 x Ls=16), same method ----------------
    su3 = None
    if not args.skip_su3:
        su3 = time_su3_apply(dw, dev, stream, args)
    su3_solve = None
    if not args.skip_su3 and not args.skip_solve and not args.skip_mg:
        su3_solve = time_su3_solves(dw, dev)

    # ---------------- batched multi-RHS apply: 64 sources, mixed lattices ----------------
    batched = None
    if not args.skip_batched:
        batched = time_batched_apply(dw, dev, stream, args)

    # ---------------- batched MG solve of the 64-source mixed batch ----------------
    batched_solve = None
    if not args.skip_mg and not args.skip_batched:
        batched_solve = time_batched_solve(dw, dev, args)

    # ---------------- tensor-core coarse operator on 64 right-hand sides ----------------
    coarse_multi = None
    if not args.skip_coarse:
        coarse_multi = time_coarse_multi(dw, dev)

    # ---------------- time to solution on the 256^2 workloads ----------------
    solve = smooth = None
    if not args.skip_solve:
        solve = time_solves(dw, dev, args)
        smooth = time_solves(dw, dev, args, synth.SCHWINGER_256_SMOOTH)

    # ---------------- small FP64 workload, FP64 apply, differentiation ----------------
    cfg1 = fp64_apply = grad = ls_sweep = None
    if not args.skip_solve:
        cfg1 = time_config1(dw, dev, stream)
        grad = time_gradient(dw, dev)
        if not args.skip_mg:
            ls_sweep = time_ls_sweep(dw, dev)
    if not args.skip_fp64:
        fp64_apply = time_fp64_apply(dw, dev, stream, args)

    clk.__exit__(None, None, None)
    peaks, peak_kind = measured_peaks()
    hbm_peak = float(peaks["hbm_gbs"])
    achieved = nbytes / float(np.mean(times)) / 1e9
    traffic = kernel_traffic()
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": traffic,
                "kernel": "k_dwf2d<LinkH16,float> (fine D_DW apply)",
                "algorithmic_bytes_per_launch": nbytes, "peak_kind": f"{peak_kind} hbm_gbs (burst copy)"}
    cpu = cpu_oracle_apply() if (rank == 0 and world == 1 and not args.skip_cpu) else None
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_apply * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32 (fp16 links)", "data": "synthetic",
                "config": {"workload": f"{wl.name}: fine D_DW(m) apply, U(1) 2-d, sigma {wl.sigma}, "
                                       f"M5 {wl.M5}, m {wl.mf}",
                           "solve_workload": SOLVE_WL.name, "parallelism": f"replicas x{world}",
                           "l2": "flushed (512 MB write) before every timed apply; the apply moves 537 MB"},
                "pct_of_hbm_peak": 100.0 * achieved / hbm_peak,
                "e2e": {"value": world * nbytes / t_e2e / 1e9, "unit": "GB/s", "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h, "ms_per_step": t_e2e * 1e3,
                        "call": f"dwf_apply_host, {e2e_best} s-chunk(s) (fastest of {list(E2E_CHUNKS)})",
                        "ms_per_step_by_chunks": {c: t_e2e_by[f"host_call_{c}"] * 1e3 for c in E2E_CHUNKS},
                        "serial_copies_ms_per_step": t_e2e_by["serial"] * 1e3},
                "roofline": roofline, "cpu_baseline": cpu, "clocks": clk.summary(),
                "gpu_launches": launches, "su3_apply": su3, "su3_solve": su3_solve, "batched_apply": batched,
                "solve": solve, "solve_smooth_sigma0214": smooth, "config1_fp64": cfg1, "fp64_apply": fp64_apply,
                "gradient": grad, "coarse_Ls_sweep": ls_sweep,
                "batched_solve": batched_solve, "coarse_multi_rhs": coarse_multi}
        print(json.dumps(line), flush=True)
    ranks.close()


def time_su3_solves(dw, dev):
    """16^3 x 32 x Ls=16 SU(3) (eps 0.3, M5 1.8, m 0.01) to 1e-10: the two-level MG
    (2^4 aggregates, Nvec = 24, FP16 coarse blocks, 16 post-smoothing steps, coarse tolerance
    0.4) against FP64 CGNE, same source."""
    import torch
    wl = synth.SU3_16x32
    U, srcs = wl.draw(1)
    g = dw.make_geom(wl.dims, wl.Ls, group="su3")
    U64 = torch.from_numpy(U.reshape(-1)).to(dev)
    b = torch.from_numpy(srcs[0].reshape(-1)).to(dev)
    x = torch.empty_like(b)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    st, status = dw.cgne_solve(g, U64, b, x, wl.M5, wl.mf, tol=1e-10, maxiter=200000, raise_noconv=False)
    torch.cuda.synchronize(dev)
    t_cg = time.perf_counter() - t0
    nvec = 24
    rng = synth.rng_for(wl.seed + 7000)
    starts = np.stack([synth.gaussian_complex(rng, (wl.V * 12,)) for _ in range(nvec)])
    # 16 post-smoothing steps and a 0.4 coarse tolerance: the best of a sweep on this workload
    # (the paper's 8 / 0.25 are for its 2-d runs; they take 121 outer iterations here, these 50)
    params = {"nvec": nvec, "block": [2, 2, 2, 2], "setup_mass": SETUP_MASS_SU3, "post_smooth": 16, "coarse_tol": 0.4}
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    mg = dw.mg_setup(g, U64, wl.M5, wl.mf, params, torch.from_numpy(starts.reshape(-1)).to(dev))
    torch.cuda.synchronize(dev)
    t_setup = time.perf_counter() - t0
    y = torch.empty_like(b)
    dw.mg_solve(mg, b, y, tol=1e-10, maxiter=2, raise_noconv=False)      # warm (workspace, graphs)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    sm, mstatus = dw.mg_solve(mg, b, y, tol=1e-10, raise_noconv=False)
    torch.cuda.synchronize(dev)
    t_mg = time.perf_counter() - t0
    dw.mg_destroy(mg)
    return {"workload": f"{wl.name}: D_DW x = b to 1e-10, M5 {wl.M5}, m {wl.mf}",
            "cgne_fp64": {"seconds": t_cg, "iterations": st["iterations"], "true_residual": st["true_residual"],
                          "status": status},
            "mg": {"seconds": t_mg, "setup_seconds": t_setup, "outer_iterations": sm["iterations"],
                   "fine_applies": sm["fine_applies"], "coarse_avg_iters": sm["coarse_avg_iters"],
                   "true_residual": sm["true_residual"], "status": mstatus},
            "mg_speedup_vs_cgne": t_cg / t_mg if t_mg > 0 else None}


def time_su3_apply(dw, dev, stream, args):
    """FP32/FP16-link 4-d SU(3) apply on 16^3 x 32 x Ls=16 (421 MB per apply), in the canonical layout
    and in the packed layout (blocks of 32 sites, each piece of a spinor a 512-byte plane)."""
    import torch
    wl = synth.SU3_16x32
    U, srcs = wl.draw(1)
    g = dw.make_geom(wl.dims, wl.Ls, group="su3")
    U64 = torch.from_numpy(U.reshape(-1)).to(dev)
    Ud = dw.links_to(g, U64, "f32_l16")
    Up = dw.pack_links(g, U64, "f32_l16")
    psi = torch.from_numpy(srcs[0].reshape(-1).astype(np.complex64)).to(dev)
    out = torch.empty_like(psi)
    psi_p = dw.pack_spinor(g, psi)
    out_p = torch.empty_like(psi_p)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    nbytes = wl.V * wl.Ls * 2 * 96 + 4 * wl.V * 36

    def timed(fn):
        for _ in range(args.warmup):
            flush.fill_(1.0)
            fn()
        torch.cuda.synchronize(dev)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for a, b in evs:
            flush.fill_(1.0)
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize(dev)
        return float(np.mean([a.elapsed_time(b) * 1e-3 for a, b in evs]))

    t = timed(lambda: dw.dwf_apply(g, Ud, psi, out, wl.M5, wl.mf, prec="f32_l16"))
    tp = timed(lambda: dw.dwf_apply_packed(g, Up, psi_p, out_p, wl.M5, wl.mf, prec="f32_l16"))
    tc = timed(lambda: dw.pack_spinor(g, psi, psi_p))
    diff = float((dw.unpack_spinor(g, out_p) - out).abs().max() / out.abs().max())
    peaks, _ = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    return {"workload": f"{wl.name}: 4-d SU(3) D_DW(m) apply, FP32 spinors, FP16 links, M5 {wl.M5}, m {wl.mf}",
            "algorithmic_bytes_per_launch": nbytes, "ms": t * 1e3, "GBps": nbytes / t / 1e9,
            "frac_of_hbm": nbytes / t / 1e9 / hbm,
            "packed": {"ms": tp * 1e3, "GBps": nbytes / tp / 1e9, "frac_of_hbm": nbytes / tp / 1e9 / hbm,
                       "pack_ms": tc * 1e3, "max_rel_diff_vs_canonical": diff}}


def time_batched_apply(dw, dev, stream, args):
    """The 64-source batch over {64^2, 128^2, 256^2} x Ls=16 in one launch, vs one launch per source."""
    import torch
    geoms, Us, psis, outs = [], [], [], []
    nbytes = 0
    for wl, nsrc in synth.batched_classes():
        U, srcs = wl.draw(nsrc)
        g = dw.make_geom(wl.dims, wl.Ls)
        Ud = dw.links_to(g, torch.from_numpy(U.reshape(-1)).to(dev), "f32_l16")
        for src in srcs:
            geoms.append(g)
            Us.append(Ud)
            psis.append(torch.from_numpy(src.reshape(-1).astype(np.complex64)).to(dev))
            outs.append(torch.empty_like(psis[-1]))
            nbytes += apply_bytes(wl.V, wl.Ls)
    M5, mf = synth.batched_classes()[0][0].M5, synth.batched_classes()[0][0].mf
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def timed(fn):
        for _ in range(args.warmup):
            flush.fill_(1.0)
            fn()
        torch.cuda.synchronize(dev)
        ts = []
        for _ in range(max(5, args.steps // 5)):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b) * 1e-3)
        return float(np.mean(ts))

    # the argument arrays are marshalled once (BatchedApply), so the timed region holds one C call;
    # the per-source comparison calls the C entry point with pre-built arguments as well
    plan = dw.BatchedApply(geoms, Us, psis, outs, prec="f32_l16")
    t_batched = timed(lambda: plan(M5, mf))
    t_call = timed(lambda: dw.dwf_apply_batched(geoms, Us, psis, outs, M5, mf, prec="f32_l16"))
    lib = dw.lib()
    st = ctypes.c_void_p(stream.cuda_stream)
    single_args = [(ctypes.byref(g), ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(p.data_ptr()),
                    ctypes.c_void_p(o.data_ptr()), float(M5), float(mf), 0, dw.PREC["f32_l16"], st)
                   for g, U, p, o in zip(geoms, Us, psis, outs)]

    def singles():
        for a in single_args:
            if lib.dwf_apply(*a) != 0:
                raise RuntimeError("dwf_apply failed")
    t_single = timed(singles)
    peaks, _ = measured_peaks()
    return {"workload": "64 sources, lattices (64, 128, 256)^2 [i mod 3] x Ls=16, FP32 spinors, FP16 links",
            "algorithmic_bytes": nbytes, "one_launch_ms": t_batched * 1e3, "one_launch_GBps": nbytes / t_batched / 1e9,
            "frac_of_hbm": nbytes / t_batched / 1e9 / float(peaks["hbm_gbs"]),
            "per_source_launches_ms": t_single * 1e3, "per_source_launches_GBps": nbytes / t_single / 1e9,
            "with_marshalling_ms": t_call * 1e3,
            "timing": "CUDA events around one prepared call (BatchedApply); with_marshalling_ms times "
                      "dwf_apply_batched building its 64-entry argument arrays inside the timed region"}


def time_batched_solve(dw, dev, args, cgne_per_class=2):
    """The 64 sources over {64^2, 128^2, 256^2} x Ls=16 (sigma 0.7, m 0.005) to 1e-10: one batched
    K-cycle per lattice class, the three classes concurrently (mg_solve_groups), against FP64 CGNE.
    CGNE is timed on `cgne_per_class` sources of each class and scaled to the class size."""
    import torch
    hs, Bs, Xs, ns, setup_s, cg_s, cg_it = [], [], [], [], 0.0, 0.0, []
    for wl, nsrc in synth.batched_classes():
        U, srcs = wl.draw(nsrc)
        g = dw.make_geom(wl.dims, wl.Ls)
        U64 = torch.from_numpy(U.reshape(-1)).to(dev)
        B = torch.from_numpy(np.stack([x.reshape(-1) for x in srcs])).to(dev)
        params = dw.mg_default_params()
        params["setup_mass"] = SETUP_MASS[wl.sigma]
        rng = synth.rng_for(wl.seed + 7000)
        starts = np.stack([synth.gaussian_complex(rng, (wl.V * 2,)) for _ in range(params["nvec"])])
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        hs.append(dw.mg_setup(g, U64, wl.M5, wl.mf, params, torch.from_numpy(starts.reshape(-1)).to(dev)))
        torch.cuda.synchronize(dev)
        setup_s += time.perf_counter() - t0
        Bs.append(B.reshape(-1))
        Xs.append(torch.empty_like(Bs[-1]))
        ns.append(nsrc)
        x = torch.empty(B.shape[1], dtype=torch.complex128, device=dev)
        t_c = 0.0
        for r in range(cgne_per_class):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            st, _ = dw.cgne_solve(g, U64, B[r], x, wl.M5, wl.mf, tol=1e-10, maxiter=200000, raise_noconv=False)
            torch.cuda.synchronize(dev)
            t_c += time.perf_counter() - t0
            cg_it.append(st["iterations"])
        cg_s += t_c / cgne_per_class * nsrc
    # warm run: workspaces and graph capture (two outer iterations)
    dw.mg_solve_groups(hs, Bs, Xs, ns, tol=1e-10, maxiter=2, raise_noconv=False)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    stats, status = dw.mg_solve_groups(hs, Bs, Xs, ns, tol=1e-10, raise_noconv=False)
    torch.cuda.synchronize(dev)
    t_mg = time.perf_counter() - t0
    for h in hs:
        dw.mg_destroy(h)
    flat = [s for st in stats for s in st]
    return {"workload": "64 sources, lattices (64, 128, 256)^2 [i mod 3] x Ls=16, sigma 0.7, M5 1, m 0.005, to 1e-10",
            "mg_batched_seconds": t_mg, "status": status, "setup_seconds_3_hierarchies": setup_s,
            "outer_iterations_max_per_class": [max(s["iterations"] for s in st) for st in stats],
            "worst_true_residual": max(s["true_residual"] for s in flat),
            "cgne_fp64_seconds_scaled": cg_s, "cgne_sample": f"{cgne_per_class} sources per class, scaled to 64",
            "cgne_iterations_sampled": cg_it, "speedup_vs_cgne": cg_s / t_mg if t_mg > 0 else None}


def time_solves(dw, dev, args, wl=SOLVE_WL):
    """One workload to a true residual of 1e-10 on the same GPU: FP64 CGNE, BiCGStab-6 on
    D_PV^dag D_DW (FP32 / FP16-link inner solves, FP64 reliable updates), the two-level K-cycle and
    the paper's three-level K-cycle with 128 deflated coarsest modes (Table kcycle, Table
    zerospacing).  MG times are given without and with the setup."""
    import torch
    U, srcs = wl.draw(1)
    g = dw.make_geom(wl.dims, wl.Ls)
    U64 = torch.from_numpy(U.reshape(-1)).to(dev)
    b = torch.from_numpy(srcs[0].reshape(-1)).to(dev)
    x = torch.empty_like(b)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    st, status = dw.cgne_solve(g, U64, b, x, wl.M5, wl.mf, tol=1e-10, maxiter=200000, raise_noconv=False)
    torch.cuda.synchronize(dev)
    t_cg = time.perf_counter() - t0
    res = {"workload": f"{wl.name} (sigma {wl.sigma}, M5 {wl.M5}, m {wl.mf})", "tol": 1e-10,
           "cgne_fp64": {"seconds": t_cg, "iterations": st["iterations"], "fine_applies": st["fine_applies"],
                         "true_residual": st["true_residual"], "status": status}}
    dw.bicgstab_solve(g, U64, b, x, wl.M5, wl.mf, ell=6, tol=1e-10, maxiter=12, raise_noconv=False)   # warm
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    sb, bstatus = dw.bicgstab_solve(g, U64, b, x, wl.M5, wl.mf, ell=6, tol=1e-10, raise_noconv=False)
    torch.cuda.synchronize(dev)
    t_bs = time.perf_counter() - t0
    res["bicgstab6"] = {"seconds": t_bs, "bicg_steps": sb["iterations"], "fine_applies": sb["fine_applies"],
                        "reliable_updates": sb["restarts"], "true_residual": sb["true_residual"], "status": bstatus,
                        "speedup_vs_cgne": t_cg / t_bs if t_bs > 0 else None}
    if hasattr(dw, "mg_setup") and not args.skip_mg:
        res["mg"] = time_mg(dw, dev, wl, U64, b, g, t_cg, levels=2)
        res["mg3_deflated"] = time_mg(dw, dev, wl, U64, b, g, t_cg, levels=3)
        res["mg3_deflated_gcr"] = time_mg(dw, dev, wl, U64, b, g, t_cg, levels=3, coarsest_solver=1)
        res["mg_speedup_vs_cgne"] = res["mg"]["speedup_vs_cgne"]
    return res


def time_mg(dw, dev, wl, U64, b, g, t_cg, levels=2, coarsest_solver=0):
    """Two-level K-cycle (Table kcycle defaults), or three levels with 128 deflated coarsest
    eigenvectors: coarsest_solver 0 = CGNR (the paper's), 1 = GCR(8)."""
    import torch
    params = dw.mg_default_params()
    params["setup_mass"] = SETUP_MASS[wl.sigma]
    rng = synth.rng_for(wl.seed + 7000)
    nvec = params["nvec"]
    starts = np.stack([synth.gaussian_complex(rng, (wl.V * 2,)) for _ in range(nvec)])
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    mg = dw.mg_setup(g, U64, wl.M5, wl.mf, params, torch.from_numpy(starts.reshape(-1)).to(dev))
    if levels == 3:
        Vc = wl.V // 16
        lp = dw.mg_default_level_params()
        s2 = np.stack([synth.gaussian_complex(rng, (Vc * 16,)) for _ in range(lp["nvec"])])
        ls = synth.gaussian_complex(rng, ((Vc // 4) * lp["Ls_c"] * 2 * lp["nvec"],))
        dw.mg_add_level(mg, {"setup_mass": SETUP_MASS[wl.sigma], "coarsest_solver": coarsest_solver},
                        torch.from_numpy(s2.reshape(-1)).to(dev),
                        torch.from_numpy(ls).to(dev))
    torch.cuda.synchronize(dev)
    t_setup = time.perf_counter() - t0
    x = torch.empty_like(b)
    dw.mg_solve(mg, b, x, tol=1e-10, maxiter=2, raise_noconv=False)     # warm run (allocations, graphs)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    st, status = dw.mg_solve(mg, b, x, tol=1e-10, raise_noconv=False)
    torch.cuda.synchronize(dev)
    t_mg = time.perf_counter() - t0
    dw.mg_destroy(mg)
    out = {"levels": levels, "seconds": t_mg, "setup_seconds": t_setup, "seconds_with_setup": t_mg + t_setup,
           "outer_iterations": st["iterations"], "fine_applies": st["fine_applies"],
           "coarse_avg_iters": st["coarse_avg_iters"], "true_residual": st["true_residual"], "status": status,
           "speedup_vs_cgne": t_cg / t_mg if t_mg > 0 else None,
           "speedup_vs_cgne_with_setup": t_cg / (t_mg + t_setup) if t_mg > 0 else None}
    if levels == 3:
        out["coarsest_avg_iters"] = st["coarsest_avg_iters"]
        out["deflated_modes"] = 128
        out["coarsest_solver"] = "GCR(8)" if coarsest_solver else "CGNR"
    return out


def time_ls_sweep(dw, dev):
    """The coarse-Ls study of the paper's discussion: 128^2 x Ls 32 (sigma 0.214, m 0.01), two-level
    K-cycle with the coarse Lhat_s reduced to 4, 8, 16 and kept at 32 (wall transfer), and the bulk
    transfer at Lhat_s = 32; fine applications and wall time to 1e-10 for each."""
    import torch
    wl = synth.SCHWINGER_128_LS32
    U, srcs = wl.draw(1)
    g = dw.make_geom(wl.dims, wl.Ls)
    U64 = torch.from_numpy(U.reshape(-1)).to(dev)
    b = torch.from_numpy(srcs[0].reshape(-1)).to(dev)
    x = torch.empty_like(b)
    rng = synth.rng_for(wl.seed + 7000)
    starts = torch.from_numpy(np.stack([synth.gaussian_complex(rng, (wl.V * 2,)) for _ in range(8)]).reshape(-1)).to(dev)
    out = {"workload": f"{wl.name}: Ls {wl.Ls}, sigma {wl.sigma}, M5 {wl.M5}, m {wl.mf}, to 1e-10", "runs": []}
    for Ls_c, transfer in ((4, 0), (8, 0), (16, 0), (32, 0), (32, 1)):
        mg = dw.mg_setup(g, U64, wl.M5, wl.mf, {"setup_mass": SETUP_MASS[wl.sigma], "Ls_c": Ls_c,
                                                "transfer": transfer}, starts)
        dw.mg_solve(mg, b, x, tol=1e-10, maxiter=2, raise_noconv=False)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        st, status = dw.mg_solve(mg, b, x, tol=1e-10, raise_noconv=False)
        torch.cuda.synchronize(dev)
        out["runs"].append({"Ls_c": Ls_c, "transfer": "bulk" if transfer else "walls",
                            "seconds": time.perf_counter() - t0, "fine_applies": st["fine_applies"],
                            "outer_iterations": st["iterations"], "coarse_avg_iters": st["coarse_avg_iters"],
                            "true_residual": st["true_residual"], "status": status})
        dw.mg_destroy(mg)
    return out


def time_config1(dw, dev, stream, reps=200):
    """The 32^2 x Ls 8 FP64 workload (sigma 0.5, m 0.01): one D_DW apply (latency; it is far too small
    to reach HBM bandwidth) and FP64 CGNE to 1e-10."""
    import torch
    wl = synth.SCHWINGER_32
    U, srcs = wl.draw(1)
    g = dw.make_geom(wl.dims, wl.Ls)
    U64 = torch.from_numpy(U.reshape(-1)).to(dev)
    b = torch.from_numpy(srcs[0].reshape(-1)).to(dev)
    out = torch.empty_like(b)
    for _ in range(10):
        dw.dwf_apply(g, U64, b, out, wl.M5, wl.mf)
    torch.cuda.synchronize(dev)
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        dw.dwf_apply(g, U64, b, out, wl.M5, wl.mf)
    e.record(stream)
    e.synchronize()
    t_apply = a.elapsed_time(e) * 1e-3 / reps
    x = torch.empty_like(b)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    st, status = dw.cgne_solve(g, U64, b, x, wl.M5, wl.mf, tol=1e-10, raise_noconv=False)
    torch.cuda.synchronize(dev)
    return {"workload": f"{wl.name}: FP64, sigma {wl.sigma}, M5 {wl.M5}, m {wl.mf}",
            "apply_us": t_apply * 1e6, "apply_GBps": apply_bytes(wl.V, wl.Ls, 32, 16) / t_apply / 1e9,
            "cgne_fp64": {"seconds": time.perf_counter() - t0, "iterations": st["iterations"],
                          "true_residual": st["true_residual"], "status": status}}


def time_fp64_apply(dw, dev, stream, args):
    """FP64 D_DW on the 1024^2 x Ls 16 lattice against the FP64 rate cuBLAS DGEMM reaches on the same
    GPU (the FP64 apply is bound by the FP64 units, not HBM)."""
    import torch
    wl = APPLY_WL
    U, srcs = wl.draw(1)
    g = dw.make_geom(wl.dims, wl.Ls)
    U64 = torch.from_numpy(U.reshape(-1)).to(dev)
    psi = torch.from_numpy(srcs[0].reshape(-1)).to(dev)
    out = torch.empty_like(psi)
    for _ in range(3):
        dw.dwf_apply(g, U64, psi, out, wl.M5, wl.mf)
    torch.cuda.synchronize(dev)
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = max(5, args.steps // 5)
    a.record(stream)
    for _ in range(n):
        dw.dwf_apply(g, U64, psi, out, wl.M5, wl.mf)
    e.record(stream)
    e.synchronize()
    t = a.elapsed_time(e) * 1e-3 / n
    del psi, out, U64
    # measured FP64 rate: cuBLAS DGEMM 8192^3 (2 N^3 flops), best of 5
    N = 8192
    A = torch.randn(N, N, dtype=torch.float64, device=dev)
    B = torch.randn(N, N, dtype=torch.float64, device=dev)
    torch.matmul(A, B)
    best = 1e30
    for _ in range(5):
        a.record(stream)
        torch.matmul(A, B)
        e.record(stream)
        e.synchronize()
        best = min(best, a.elapsed_time(e) * 1e-3)
    dgemm = 2.0 * N ** 3 / best / 1e12
    del A, B
    sites = wl.V * wl.Ls
    # per 5-d site: 2 directions x (project 2 + complex multiply 6 + reconstruct 4) x 2 hops, diagonal
    # and s-hops: 60 real flops (the counting convention of the 2-d kernel)
    flops = 60.0 * sites
    return {"workload": f"{wl.name}: FP64 spinors and links", "ms": t * 1e3,
            "GBps": apply_bytes(wl.V, wl.Ls, 32, 16) / t / 1e9, "TFLOPs": flops / t / 1e12,
            "dgemm_TFLOPs_measured": dgemm, "frac_of_dgemm": flops / t / 1e12 / dgemm,
            "flops_per_site": 60}


def time_gradient(dw, dev):
    """The 128^2 x Ls 12 workload (sigma 0.7, m 0.005): x = D^-1 b with FP64 CGNE (tol 1e-12), loss |x|^2,
    backward = one adjoint solve and the link force; forward and backward wall times."""
    import torch
    wl = synth.SCHWINGER_128_GRAD
    theta, rng = wl.angles()
    b = torch.from_numpy(synth.gaussian_spinor(rng, wl.dims, wl.Ls).reshape(-1)).to(dev)
    g = dw.make_geom(wl.dims, wl.Ls)
    th = torch.from_numpy(theta.reshape(-1)).to(dev).requires_grad_(True)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    x = dw.solve(th, b, g, wl.M5, wl.mf, tol=1e-12)
    loss = (x.abs() ** 2).sum()
    torch.cuda.synchronize(dev)
    t_fwd = time.perf_counter() - t0
    t0 = time.perf_counter()
    loss.backward()
    torch.cuda.synchronize(dev)
    t_bwd = time.perf_counter() - t0
    return {"workload": f"{wl.name}: d|x|^2/dtheta, FP64 CGNE solves to 1e-12", "forward_seconds": t_fwd,
            "backward_seconds": t_bwd, "angles": int(th.numel())}


FORM_NAMES = {1: "mma.sync, 1 tile/warp", 2: "mma.sync, 2 tiles/warp", 4: "mma.sync, 4 tiles/warp",
              256: "tcgen05, one item per CTA", 257: "tcgen05, persistent warp-specialised",
              258: "tcgen05, data operand in tensor memory"}


def time_coarse_multi(dw, dev, nrhs=64, reps=20):
    """The Galerkin coarse operator of the 256^2 solve's hierarchy on nrhs vectors: one
    tensor-core launch (mg_coarse_apply_multi) against nrhs launches of the one-vector stencil."""
    import torch
    wl = SOLVE_WL
    mf = wl.mf
    U, _ = wl.draw(1)
    g = dw.make_geom(wl.dims, wl.Ls)
    params = dw.mg_default_params()
    params["setup_mass"] = SETUP_MASS[wl.sigma]
    rng = synth.rng_for(wl.seed + 7000)
    starts = np.stack([synth.gaussian_complex(rng, (wl.V * 2,)) for _ in range(params["nvec"])])
    mg = dw.mg_setup(g, torch.from_numpy(U.reshape(-1)).to(dev), wl.M5, wl.mf, params,
                     torch.from_numpy(starts.reshape(-1)).to(dev))
    nc = mg.coarse_size
    vin = torch.randn(nrhs, nc, dtype=torch.complex64, device=dev)
    vout = torch.empty_like(vin)
    Vc, Ls_c, ncd = mg.Vc, mg.coarse_geom.Ls, mg.ncdof
    ndir = 1 + 2 * mg.coarse_geom.nd
    flops = 8.0 * ndir * ncd * ncd * Vc * Ls_c * nrhs
    nbytes = 8.0 * (ndir * ncd * ncd * Vc + 2 * nrhs * nc)

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        b.synchronize()
        return a.elapsed_time(b) * 1e-3 / reps

    t_tc = timed(lambda: dw.mg_coarse_apply_multi(mg, vin, vout, nrhs, mf))
    form = dw.mg_coarse_tc_form(mg, nrhs)
    t_sm = timed(lambda: dw.mg_coarse_apply_multi(mg, vin, vout, nrhs, mf, layout="site_major"))
    form_sm = dw.mg_coarse_tc_form(mg, nrhs, layout="site_major")

    def singles():
        for r in range(nrhs):
            dw.mg_coarse_apply(mg, vin[r], vout[r], mf)
    t_one = timed(singles)
    dw.mg_destroy(mg)
    return {"workload": f"{wl.name} hierarchy (default FP16 blocks), coarse D_DW(m) on {nrhs} vectors",
            "nrhs": nrhs, "coarse_sites": Vc, "Ls_c": Ls_c, "useful_flops": flops, "algorithmic_bytes": nbytes,
            "autotuned_form": FORM_NAMES.get(form, str(form)),
            "tensor_core_ms": t_tc * 1e3, "tensor_core_TFLOPs": flops / t_tc / 1e12,
            "tensor_core_GBps": nbytes / t_tc / 1e9, "frac_of_hbm": nbytes / t_tc / 1e9 / measured_peaks()[0]["hbm_gbs"],
            "site_major_layout": {"ms": t_sm * 1e3, "autotuned_form": FORM_NAMES.get(form_sm, str(form_sm))},
            "per_vector_launches_ms": t_one * 1e3, "speedup": t_one / t_tc}


def profile_solve(which):
    """One MG solve inside the NVTX range "solve", for an ncu launch list (no JSON line): the
    hierarchy is set up as in the timed legs, a warm call builds the workspaces and graphs, then
    the solve runs.  which: "solve2d" (256^2 x 16), "solve4d" (16^3 x 32 x 16) or "batched256"
    (the 21 sources of the 64-source batch's 256^2 class, one batched K-cycle)."""
    import torch
    import paper_2004_07732_gb300 as dw
    dev = torch.device("cuda", 0)
    if which == "solve4d":
        wl = synth.SU3_16x32
        U, srcs = wl.draw(1)
        g = dw.make_geom(wl.dims, wl.Ls, group="su3")
        nvec = 24
        rng = synth.rng_for(wl.seed + 7000)
        starts = np.stack([synth.gaussian_complex(rng, (wl.V * 12,)) for _ in range(nvec)])
        params = {"nvec": nvec, "block": [2, 2, 2, 2], "setup_mass": SETUP_MASS_SU3, "post_smooth": 16,
                  "coarse_tol": 0.4}
        nrhs = 1
    else:
        if which == "batched256":
            wl, nrhs = synth.batched_classes()[2]
        else:
            wl, nrhs = SOLVE_WL, 1
        U, srcs = wl.draw(nrhs)
        g = dw.make_geom(wl.dims, wl.Ls)
        params = dw.mg_default_params()
        params["setup_mass"] = SETUP_MASS[wl.sigma]
        rng = synth.rng_for(wl.seed + 7000)
        starts = np.stack([synth.gaussian_complex(rng, (wl.V * 2,)) for _ in range(params["nvec"])])
    U64 = torch.from_numpy(U.reshape(-1)).to(dev)
    b = torch.from_numpy(np.stack([x.reshape(-1) for x in srcs[:nrhs]]).reshape(-1)).to(dev)
    mg = dw.mg_setup(g, U64, wl.M5, wl.mf, params, torch.from_numpy(starts.reshape(-1)).to(dev))
    x = torch.empty_like(b)
    dw.mg_solve_batched(mg, b, x, nrhs, tol=1e-10, maxiter=2, raise_noconv=False)
    torch.cuda.synchronize(dev)
    torch.cuda.nvtx.range_push("solve")
    t0 = time.perf_counter()
    st, status = dw.mg_solve_batched(mg, b, x, nrhs, tol=1e-10, raise_noconv=False)
    torch.cuda.synchronize(dev)
    t = time.perf_counter() - t0
    torch.cuda.nvtx.range_pop()
    dw.mg_destroy(mg)
    print(json.dumps({"profile": which, "seconds": t, "status": status,
                      "outer_iterations_max": max(s["iterations"] for s in st)}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--skip-solve", action="store_true")
    ap.add_argument("--skip-mg", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-su3", action="store_true")
    ap.add_argument("--skip-batched", action="store_true")
    ap.add_argument("--skip-coarse", action="store_true")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--profile", choices=["solve2d", "solve4d", "batched256"], default=None,
                    help="run one MG solve inside the NVTX range 'solve' for an ncu launch list, print no bench line")
    args = ap.parse_args()
    if args.profile:
        profile_solve(args.profile)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
