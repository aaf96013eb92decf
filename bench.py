"""Benchmark: (H2O)64-like exact-exchange applications per second on GB300.

One step = one pass of the whole path on one synthetic configuration
(the headline is the chosen form, mixed precision; plain FP64 is timed in
the same run and reported beside it):
sea_apply_vxx (domain boxes, pair selection, per-pair Poisson CG with
multipole boundaries, far field, accumulation of V_xx phi and E_xx),
sea_build_ace (M, Cholesky, L^-1) and sea_apply_ace on 256 trial vectors.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

``value``: steps/s with inputs resident in HBM (CUDA events on the
library's stream).  ``e2e``: the same through the C ABI with pinned host
buffers, host<->device copies inside the timed region.  ``--impl
reference`` times the CPU oracle (the plain FP64 reference of the method)
on the host cores.  For N > 1 (torchrun) every rank runs an independent
replica of the workload (the path has no exchange step between
configurations); value = all ranks' steps / max time.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "(H2O)64 V_xx applications/s, plain FP64 vs chosen form, same |dExx| bound"
UNIT = "applications/s"
CONFIG = "h2o64_96"
N_TRIAL = 256
WORKLOAD = ("(H2O)64-like, 256 localized orbitals, L=12.42 A, 96^3 grid, eps=10^-3.5, "
            "delta=1e-3, CG tol 1e-8, l_max=6, O(h^12) stencil; ACE build + apply to "
            "256 trial vectors")
FORMS = {"plain": "plain FP64",
         "mixed": "mixed: FP32 CG sweeps/vectors inside iterative refinement (true residual and "
                  "solution in double-float at tol >= 1e-10, FP64 below; FP64 E_xx); "
                  "double-float multipoles and Cholesky; ACE contractions on the tensor cores "
                  "from exact digit splits of FP64 values"}

# Algorithmic FP64 flops per CG unknown and iteration: the symmetric 37-point
# stencil as 18 pair sums, 18 multiply-adds and the centre product (55), plus
# two dot products and three vector updates (10).
CG_FLOPS_PER_UNKNOWN_ITER = 65
# FP64 peak from the part's unit counts and clock: 152 SMs x 2 FP64 FMA/clk x
# 2 flop x 2.07 GHz (the nominal 1.25 TFLOP/s FP64 figure).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _clock_sampler(path):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        return subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                 "-lms", "200"], stdout=open(path, "w"),
                                stderr=subprocess.DEVNULL)
    except (OSError, FileNotFoundError):
        return None


def _clock_summary(path, index):
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    try:
        for line in open(path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9 or not f[0].isdigit() or int(f[0]) != index:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
    except OSError:
        pass
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons)}


def max_over_ranks(values, ws, device=None):
    """Element-wise maximum of per-rank timings over all ranks (the job's
    time is its slowest replica); identity for a single rank."""
    if ws <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def job_value(steps, ws, t_ms_max):
    """Whole-job throughput: every rank runs `steps` applications of its own
    replica; the job takes the slowest rank's time."""
    return ws * steps / (t_ms_max / 1e3)


# DRAM traffic per launch at the benchmark size (dram__bytes_read.sum +
# dram__bytes_write.sum), captured with the current kernels on this workload
# by a one-pass ncu run (the two counters and the duration only).  None: not
# captured.
DRAM_BYTES_PER_LAUNCH = {
    "k_cg_mixed": 25.6e6,
    "k_gram_tc": 2.026e9,
    "k_expand_tc": 1.934e9,
}


def _tiles_with_support(w, torch):
    """Number of 8 x 4 x 4 grid tiles on which some row of W is nonzero (the
    tiles the contraction with W reads A on)."""
    n, nz, ny, nx = w.shape
    pz, py, px = (-nz) % 4, (-ny) % 4, (-nx) % 8
    nzmask = (w != 0).any(dim=0).to(torch.float32)
    if pz or py or px:
        nzmask = torch.nn.functional.pad(nzmask, (0, px, 0, py, 0, pz))
    t = nzmask.reshape((nz + pz) // 4, 4, (ny + py) // 4, 4, (nx + px) // 8, 8)
    return int((t.sum(dim=(1, 3, 5)) > 0).sum().item())


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def _time_form(args, sea, s, psi, vxx, y, stream, precision, barrier, torch, rank, local,
               sample_clocks):
    """W warm-up + K timed steps of one form; per-stage and per-kernel times."""
    ctx = sea.Context(s.cell, s.grid, stream=stream.cuda_stream, precision=precision)
    phi = torch.from_numpy(s.phi).to(vxx.device)
    ctx.set_orbitals(phi)
    del phi
    for _ in range(args.warmup):
        ctx.apply_vxx(vxx)
        ctx.build_ace()
        ctx.apply_ace(psi, y)
    stream.synchronize()
    clk_path = os.path.join(tempfile.gettempdir(), f"sea_clocks_{os.getpid()}_{precision}.csv")
    sampler = _clock_sampler(clk_path) if (rank == 0 and sample_clocks) else None
    time.sleep(0.5 if sampler else 0)
    st0 = ctx.stats()
    keys = ["ms_plan", "ms_setup", "ms_cg", "ms_accumulate", "ms_ace_build", "ms_gram_build",
            "ms_ace_apply", "ms_gram_apply", "ms_expand_apply"]
    acc = {k: 0.0 for k in keys}
    cg_work = 0
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        ctx.apply_vxx(vxx)
        ctx.build_ace()
        ctx.apply_ace(psi, y)
        stream.synchronize()
        st = ctx.stats()
        for k in keys:
            acc[k] += st[k]
        cg_work += st["cg_unknown_iters"]
    e1.record(stream)
    barrier()
    t_ms = e0.elapsed_time(e1)
    st1 = ctx.stats()
    if sampler:
        sampler.terminate()
        sampler.wait()
    clocks = _clock_summary(clk_path, local) if sampler else None
    K = args.steps
    out = {"ctx": ctx, "t_ms": t_ms, "clocks": clocks, "launches": st1["n_launches"] - st0["n_launches"],
           "stage_ms": {k[3:]: v / K for k, v in acc.items()}, "cg_unknown_iters": cg_work / K,
           "stats": st1}
    return out


def run_ours(args, ws, rank, local):
    import torch

    from paper_2208_06097_gb300 import build as B
    from paper_2208_06097_gb300 import sea, synth

    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    s = synth.make_config(args.config)
    psi_h = synth.random_trial_vectors(N_TRIAL, s.grid, 2024)
    stream = torch.cuda.Stream(device=dev)
    psi = torch.from_numpy(psi_h).to(dev)
    vxx = torch.empty(s.phi.shape, dtype=torch.float64, device=dev)
    y = torch.empty_like(psi)
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    forms = ["plain", "mixed"] if args.form == "both" else [args.form]
    chosen = "mixed" if "mixed" in forms else forms[0]
    res = {}
    results = {}  # each form's V_xx phi (host copy, outside the timed region) and E_xx
    for f in forms:
        res[f] = _time_form(args, sea, s, psi, vxx, y, stream, 1 if f == "mixed" else 0, barrier,
                            torch, rank, local, sample_clocks=(f == chosen))
        if rank == 0 and ws == 1 and not args.no_cpu_baseline:
            results[f] = (vxx.cpu().numpy(), res[f]["stats"]["exx"])
        if f != chosen:
            res[f]["ctx"].close()
    R = res[chosen]
    ctx = R["ctx"]
    nnz_w = int((vxx != 0).sum().item())  # exact support of W (outside the timed region)
    tiles_w = _tiles_with_support(vxx, torch)

    # e2e: host buffers through the C ABI, copies inside the timed region
    phi_pin = torch.from_numpy(s.phi).pin_memory().numpy()
    psi_pin = torch.from_numpy(psi_h).pin_memory().numpy()
    out_pin = torch.empty(s.phi.shape, dtype=torch.float64).pin_memory().numpy()
    y_pin = torch.empty(psi_h.shape, dtype=torch.float64).pin_memory().numpy()
    e2e_steps = 0 if args.no_e2e else max(1, min(args.steps, 5))

    e2e_calls = {"set_orbitals": 0.0, "apply_vxx": 0.0, "build_ace": 0.0, "apply_ace": 0.0}

    def step_host():
        t = [time.perf_counter()]
        ctx.set_orbitals(phi_pin)
        t.append(time.perf_counter())
        ctx.apply_vxx(out_pin)
        t.append(time.perf_counter())
        ctx.build_ace()
        t.append(time.perf_counter())
        ctx.apply_ace(psi_pin, y_pin)
        t.append(time.perf_counter())
        for k, key in enumerate(e2e_calls):
            e2e_calls[key] += (t[k + 1] - t[k]) * 1e3

    if e2e_steps:
        step_host()
        for key in e2e_calls:
            e2e_calls[key] = 0.0
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        step_host()
    barrier()
    t_e2e = time.perf_counter() - t0

    agg = max_over_ranks([R["t_ms"], t_e2e] + [res[f]["t_ms"] for f in forms], ws, dev)
    t_ms, t_e2e = agg[0], agg[1]
    form_ms = {f: agg[2 + k] for k, f in enumerate(forms)}
    if rank != 0:
        ctx.close()
        return None

    K = args.steps
    value = job_value(K, ws, t_ms)
    e2e_value = ws * e2e_steps / t_e2e if e2e_steps else None
    st = R["stats"]
    sm = R["stage_ms"]
    n = s.n_orb
    # candidate kernels: (name, ms per launch, launches per step, work per
    # launch, peak, bound, note); work in the peak's unit (flop or FP32 op)
    cand = []
    gram_ms = (sm["gram_build"] + sm["gram_apply"]) / 2
    if chosen == "plain":
        note = ("FP64 ALU from unit counts: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz; "
                "algorithmic flops: CG 65/unknown/iteration, ACE 2 x rows x nonzeros of W")
        cand.append(("k_cg (persistent FP64 CG)", sm["cg"], 1,
                     CG_FLOPS_PER_UNKNOWN_ITER * R["cg_unknown_iters"], FP64_PEAK_TFLOPS, "alu",
                     note))
        cand.append(("k_gram_partial (FP64 M = Phi^T W and W^T psi over W's tiles)", gram_ms, 2,
                     2.0 * n * nnz_w, FP64_PEAK_TFLOPS, "alu", note))
        cand.append(("k_tile_expand (FP64 W H over W's tiles)", sm["expand_apply"], 1,
                     2.0 * N_TRIAL * nnz_w, FP64_PEAK_TFLOPS, "alu", note))
    else:
        hbm = float(_peaks().get("hbm_gbs", 6800.0))  # GB/s, measured copy
        note_cg = ("HBM of measured (copy, MEASURED_PEAKS.json); effective model bytes: 11 vector "
                   "passes x 4 B per unknown and FP32 inner iteration (the pair vectors stay "
                   "on chip, so DRAM traffic is lower)")
        cand.append(("k_cg_mixed (FP32 CG sweeps inside FP64 refinement)", sm["cg"], 1,
                     44.0 * R["cg_unknown_iters"], hbm, "hbm", note_cg))
        # the CG's own roof: shared memory (37 four-byte stencil loads per
        # unknown and inner iteration) against 152 SMs x 128 B/clk at the
        # sampled SM clock
        sm_mhz = (R["clocks"] or {}).get("sm_mhz") or 2070.0
        smem_peak = 152 * 128 * sm_mhz * 1e6 / 1e9  # GB/s
        cand.append(("k_cg_mixed [shared-memory roof]", sm["cg"], 1,
                     37 * 4.0 * R["cg_unknown_iters"], smem_peak, "smem",
                     "shared-memory bandwidth from unit counts: 152 SMs x 128 B/clk x the "
                     "sampled SM clock; algorithmic bytes: the 37 stencil loads (4 B) per "
                     "unknown and inner FP32 iteration"))
        note_gt = ("HBM of measured (copy); algorithmic bytes: the A rows on the tiles where W is "
                   "nonzero (8 B per point), W's FP16 digit planes (1536 B per tile slot and "
                   "128-row block), the FP64 partials written")
        slots = st["ace_support_points"] / 128  # total W list length over the tiles
        gram_bytes = (n * 128 * 8.0 * tiles_w + 1536.0 * slots * ((n + 127) // 128) +
                      8.0 * slots * n)
        cand.append(("k_gram_tc (tensor-core M = Phi^T W and W^T psi, exact FP16 digits)",
                     gram_ms, 2, gram_bytes, hbm, "hbm", note_gt))
        note_x = ("HBM of measured (copy); algorithmic bytes: the FP64 output (8 B per grid "
                  "point and vector) and W's per-tile BF16 digit image (24 KB per tile with "
                  "support and K step of 16 W rows)")
        ng = float(np.prod(s.grid))
        expand_bytes = 8.0 * N_TRIAL * ng + 24576.0 * tiles_w
        cand.append(("k_expand_tc (tensor-core W H, exact FP16 digits)", sm["expand_apply"], 1,
                     expand_bytes, hbm, "hbm", note_x))
    def _rate(c):  # work per launch / time: flop -> TFLOP/s, bytes -> GB/s
        return c[3] / (c[1] / 1e3) / (1e9 if c[5] in ("hbm", "smem") else 1e12) if c[1] > 0 else 0.0

    top = max((c for c in cand if c[5] != "smem"), key=lambda c: c[1] * c[2])
    name, kms, nl, flops, peak, bound, peak_note = top
    achieved = _rate(top)
    others = [{"kernel": c[0], "bound": c[5], "ms_per_step": c[1] * c[2], "achieved": _rate(c),
               "peak": c[4], "unit": "GB/s" if c[5] in ("hbm", "smem") else "TFLOP/s",
               "frac": _rate(c) / c[4]} for c in cand if c is not top]
    cpu, oracle_res = (cpu_baseline(s, psi_h) if (ws == 1 and not args.no_cpu_baseline)
                       else (None, None))
    # the metric's bound: each form's error against the oracle on this input
    n_mol = s.n_orb // 4
    errors = None
    if oracle_res is not None and results:
        vref = oracle_res["vxx"]
        vmax = float(np.abs(vref).max())
        errors = {f: {"exx": e, "exx_oracle": float(oracle_res["exx"]),
                      "exx_err_per_molecule": abs(e - float(oracle_res["exx"])) / n_mol,
                      "max_abs_dvxx": float(np.abs(v - vref).max()),
                      "max_abs_dvxx_rel": float(np.abs(v - vref).max()) / vmax,
                      "bound_exx_per_molecule": 1e-6}
                  for f, (v, e) in results.items()}
    batched = run_batched(args, sea, torch, dev) if (ws == 1 and not args.no_batched) else None
    warm = run_warm_start(args, sea, synth, torch, dev, s) if (ws == 1 and not args.no_warm_start) else None
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "plain_value": ws * K / (form_ms["plain"] / 1e3) if "plain" in form_ms else None,
        "exx_err_per_molecule": errors[chosen]["exx_err_per_molecule"] if errors else None,
        "max_abs_dvxx": errors[chosen]["max_abs_dvxx"] if errors else None,
        "n_gpus": ws,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": t_ms / K,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if chosen == "plain" else "f64+f32",
        "data": "synthetic (seeded water-like localized orbitals, see synth.py)",
        "config": {
            "workload": WORKLOAD if args.config == CONFIG else
                        f"{args.config} (profiling case: {s.n_orb} orbitals, {s.grid} grid)",
            "form": FORMS[chosen],
            "forms_applications_per_s": {f: ws * K / (form_ms[f] / 1e3) for f in forms},
            "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
            "l2": "inputs larger than L2 (Phi and psi 1.81 GB each)",
            "n_pairs": st["n_pairs"],
            "cg_unknowns": st["n_unknowns"],
            "cg_iters_mean": st["cg_iters_mean"],
            "cg_unknown_iters": R["cg_unknown_iters"],
            "w_nonzeros": nnz_w,
            "ace_tile_points": st["ace_support_points"],
            "stage_ms": sm,
            "stage_ms_plain": res["plain"]["stage_ms"] if "plain" in res else None,
            "errors_vs_oracle": errors,
            "batched_form": batched,
            "warm_start": warm,
        },
        "e2e": {
            "value": e2e_value,
            "unit": UNIT,
            "h2d_bytes_per_step": int(s.phi.nbytes + psi_h.nbytes),
            "d2h_bytes_per_step": int(s.phi.nbytes + psi_h.nbytes + 8),
            "call_ms": {k: v / e2e_steps for k, v in e2e_calls.items()} if e2e_steps else None,
        },
        "gpu_launches": int(R["launches"]),
        "roofline": {
            "kernel": name,
            "bound": bound,
            "achieved": achieved,
            "peak": peak,
            "unit": "GB/s" if bound == "hbm" else "TFLOP/s",
            "frac": achieved / peak,
            "traffic": DRAM_BYTES_PER_LAUNCH.get(name.split(" ")[0]) if args.config == "h2o64_96" else None,
            "traffic_unit": "bytes per launch (DRAM read + write, ncu)",
            "peak_note": peak_note,
            "other_kernels": others,
        },
        "clocks": R["clocks"],
    }
    if cpu:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    ctx.close()
    return line


def batched_workload(n_cfg=64, seed=3000):
    """The batched form's workload: n_cfg independent configurations (H2O)n,
    n ~ U{32..128}, density ~ U[0.4, 1.7] g/cm^3, grid spacing ~0.13 A
    (0.2457 bohr).  Returns (n_mol, L in angstrom, grid points per axis,
    seed) per configuration."""
    from paper_2208_06097_gb300 import synth
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_cfg):
        n_mol = int(rng.integers(32, 129))
        dens = float(rng.uniform(0.4, 1.7))
        L = (n_mol * 18.015 / 0.60221408 / dens) ** (1.0 / 3.0)  # angstrom
        grid = max(16, int(round(L * synth.ANGSTROM / 0.2457)))
        out.append((n_mol, L, grid, seed + 1 + k))
    return out


def _groups(work, budget_bytes):
    """Consecutive groups of configurations whose device arrays (the
    context's orbitals and W, the output: 3 x n_orb x grid^3 doubles) fit the
    budget."""
    groups, cur, used = [], [], 0
    for w in work:
        b = 3 * 4 * w[0] * w[2] ** 3 * 8
        if cur and used + b > budget_bytes:
            groups.append(cur)
            cur, used = [], 0
        cur.append(w)
        used += b
    if cur:
        groups.append(cur)
    return groups


def run_batched(args, sea, torch, dev, budget_gb=140.0):
    """Batched form vs one call per configuration, V_xx application only, on
    the 64-configuration workload; orbitals generated on the device.  The
    configurations go through sea_apply_vxx_batch in groups that fit the
    device (each group one batched call: autotuned, graph-captured, then
    replayed); the times of the groups add up."""
    from paper_2208_06097_gb300 import synth
    work = batched_workload()
    groups = _groups(work, budget_gb * 1e9)
    stream = torch.cuda.Stream(device=dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        stream.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / args.steps

    t_batch = t_seq = t_gen = 0.0
    pairs = orbitals = 0
    tuned = []
    for grp in groups:
        tg = time.perf_counter()
        ctxs, outs = [], []
        for n_mol, L, g, seed in grp:
            phi, cell, grid = synth.make_waters_device(n_mol, L, g, seed, dev)
            c = sea.Context(cell, grid, stream=stream.cuda_stream, precision=1)
            c.set_orbitals(phi)
            del phi
            torch.cuda.empty_cache()  # the generator's blocks back to the driver
            ctxs.append(c)
            outs.append(torch.empty((4 * n_mol, g, g, g), dtype=torch.float64, device=dev))
        torch.cuda.synchronize()
        t_gen += time.perf_counter() - tg
        t_batch += timed(lambda: sea.apply_vxx_batch(ctxs, outs))
        st0 = ctxs[0].stats()
        tuned.append({"configurations": len(grp), "order": st0["batch_order"],
                      "ctas_per_sm": st0["batch_ctas_per_sm"]})
        t_seq += timed(lambda: [c.apply_vxx(o) for c, o in zip(ctxs, outs)])
        pairs += sum(c.stats()["n_pairs"] for c in ctxs)
        orbitals += sum(c.n_orb for c in ctxs)
        for c in ctxs:
            c.close()
        del ctxs, outs
        torch.cuda.empty_cache()
    n = len(work)
    return {"configurations": n, "orbitals_total": orbitals, "pairs_total": pairs,
            "groups": len(groups), "tuned": tuned,
            "ms_batched": t_batch, "ms_one_by_one": t_seq,
            "configs_per_s_batched": n / (t_batch / 1e3),
            "configs_per_s_one_by_one": n / (t_seq / 1e3),
            "generation_s": t_gen,
            "workload": "64 configurations (H2O)32-128, 0.4-1.7 g/cm^3, h = 0.13 A (BASELINE "
                        "config 4), mixed form, V_xx application only; in groups of at most "
                        f"{budget_gb:.0f} GB of device arrays, one batched call per group"}


def _eval_warm(net, sea, torch, phi, cell, grid, out):
    """CG work and apply_vxx time with and without the learned warm start,
    both forms, on the orbitals phi (device tensor): one warm-up call and one
    timed call per case."""
    res = {}
    for name, prec in (("plain", 0), ("mixed", 1)):
        row = {}
        for mode in (0, 1):
            ctx = sea.Context(cell, grid, precision=prec, warm_start=mode)
            if mode:
                net.attach(ctx)
            ctx.set_orbitals(phi)
            ctx.apply_vxx(out)  # warm-up
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            e = ctx.apply_vxx(out)
            ev1.record()
            torch.cuda.synchronize()
            st = ctx.stats()
            key = "warm" if mode else "cold"
            row[key] = {"cg_iters_mean": st["cg_iters_mean"], "cg_unknown_iters": st["cg_unknown_iters"],
                        "ms_apply_vxx": ev0.elapsed_time(ev1), "ms_setup": st["ms_setup"],
                        "ms_cg": st["ms_cg"], "exx": e, "n_pairs": st["n_pairs"]}
            if mode:
                sea.WarmStartNet.detach(ctx)
            ctx.close()
        row["cg_work_saved_frac"] = 1.0 - row["warm"]["cg_unknown_iters"] / max(row["cold"]["cg_unknown_iters"], 1.0)
        row["ms_cg_saved"] = row["cold"]["ms_cg"] - row["warm"]["ms_cg"]
        row["ms_network"] = row["warm"]["ms_setup"] - row["cold"]["ms_setup"]
        row["exx_rel_diff"] = abs(row["warm"]["exx"] - row["cold"]["exx"]) / abs(row["cold"]["exx"])
        res[name] = row
    return res


def run_warm_start(args, sea, synth, torch, dev, s, width=16, train_seeds=(2001, 2002), steps=400,
                   batch=8, large=True):
    """The learned warm start: a width-16 U-Net trained on the pair solves of
    two other seeded (H2O)64-like systems (plain CG), then CG iterations and
    apply_vxx time with and without it on the benchmark system and on the
    (H2O)256-like system (1024 orbitals, L = 24.84 A, 192^3, seed 1005,
    generated on the device) (outside the timed region)."""
    t0 = time.perf_counter()
    net = sea.WarmStartNet(width=width, seed=11)
    for seed in train_seeds:
        sys_t = synth.make_waters(64, s.cell[0] / synth.ANGSTROM, s.grid[0], seed)
        ctx = sea.Context(sys_t.cell, sys_t.grid)
        phi = torch.from_numpy(sys_t.phi).to(dev)
        ctx.set_orbitals(phi)
        ctx.apply_vxx(torch.empty_like(phi))
        net.collect(ctx)
        ctx.close()
        del phi
    n_samples = int(sea.lib().sea_unet_num_samples(net.handle))
    loss0 = net.train(1, batch=batch, lr=1e-3, seed=1)
    loss1 = net.train(steps, batch=batch, lr=1e-3, seed=2)
    t_train = time.perf_counter() - t0
    phi = torch.from_numpy(s.phi).to(dev)
    out = torch.empty_like(phi)
    res = {"width": width, "train_systems": [f"(H2O)64-like seed {k}" for k in train_seeds],
           "train_samples": n_samples, "train_steps": steps + 1, "batch": batch,
           "loss_first": loss0, "loss_last": loss1, "train_s": t_train,
           "eval": "the benchmark system (not in the training set), cg_tol 1e-8"}
    res.update(_eval_warm(net, sea, torch, phi, s.cell, s.grid, out))
    del phi, out
    if large:
        phi = out = None
        try:
            t1 = time.perf_counter()
            phi, cell, grid = synth.make_waters_device(256, 24.84, 192, 1005, dev)
            torch.cuda.synchronize()
            t_gen = time.perf_counter() - t1
            torch.cuda.empty_cache()
            out = torch.empty_like(phi)
            big = _eval_warm(net, sea, torch, phi, cell, grid, out)
            big["generation_s"] = t_gen
        except (RuntimeError, sea.SeaError) as exc:  # device memory: reported, not fatal
            big = {"error": str(exc)[:300]}
        big["system"] = ("(H2O)256-like, 1024 orbitals, L = 24.84 A, 192^3 grid, seed 1005 "
                         "(generated on the device), cg_tol 1e-8")
        res["h2o256_192"] = big
        del phi, out
        torch.cuda.empty_cache()
    net.close()
    return res


def oracle_step(s, psi_h):
    """One full step of the CPU oracle (test infrastructure, timed only)."""
    from oracle import ace as OA
    from oracle import oracle as O
    r = O.apply_vxx(s.phi, s.cell, O.Params())
    F = s.phi.reshape(s.n_orb, -1)
    a = OA.build_ace(F, r["vxx"].reshape(s.n_orb, -1), s.dV)
    OA.apply_ace(a["Xi"], psi_h.reshape(psi_h.shape[0], -1), s.dV)
    return r


def cpu_baseline(s, psi_h):
    """The oracle as it stands, timed on the host cores: one full step of the
    same workload (a few seconds on the GPU machine's host).  Returns the timing
    record and the oracle's result (V_xx phi, E_xx) on this input."""
    from oracle import oracle as O
    O.build()
    t0 = time.perf_counter()
    r = oracle_step(s, psi_h)
    dt = time.perf_counter() - t0
    return ({"value": 1.0 / dt, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
             "sample": "one full step (V_xx + ACE build + ACE apply to 256 vectors) of the "
                       "same (H2O)64-like 96^3 workload; C oracle with OpenMP over pairs, "
                       "numpy/BLAS ACE"}, r)


def run_reference(args, ws, rank):
    if rank != 0:
        return None
    from oracle import oracle as O
    from paper_2208_06097_gb300 import synth
    O.build()
    s = synth.make_config(CONFIG)
    psi_h = synth.random_trial_vectors(N_TRIAL, s.grid, 2024)
    for _ in range(min(args.warmup, 1)):
        oracle_step(s, psi_h)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_step(s, psi_h)
    dt = time.perf_counter() - t0
    v = args.steps / dt
    line = {
        "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": min(args.warmup, 1), "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded water-like localized orbitals, see synth.py)",
        "config": {"workload": WORKLOAD,
                   "form": "CPU oracle (plain FP64 reference of the method)"},
        "impl": "reference",
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                         "sample": "full steps of the same workload on the host cores"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--config", default=CONFIG, help="workload name in synth.CONFIGS "
                    "(default: the (H2O)64 96^3 benchmark workload; smaller ones for profiling)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer pass")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-form section")
    ap.add_argument("--no-warm-start", action="store_true",
                    help="skip the learned warm-start section")
    ap.add_argument("--form", choices=["plain", "mixed", "both"], default="both",
                    help="plain FP64, the mixed form, or both (headline: mixed)")
    args = ap.parse_args()
    ws, rank, local = _dist()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
