"""Benchmark of the DEC conduction hot path on GB300.

One step = the whole path on one synthetic workload, through the C ABI:
mesh_upload (edge list, CSR structure) -> hodge_assemble (*1) ->
laplacian_build (L, b, FSAI factor) -> solve (PCG to rel. residual 1e-10)
-> k_eff.  Inputs are resident in HBM when a step starts; L2 is flushed
(a 512 MiB write) between timed steps, outside the timed events.

Prints ONE JSON line (rank 0).  Default workload: the largest single-GPU
configuration, the 192^3 jittered Delaunay cube with lognormal conductivity
(sigma = 1.5) and 5000 penny cracks, 8 Dirichlet value sets solved together
by the batched mixed-precision PCG (FP32 CG, BF16 FSAI factor, FP64 residual
replacement, one persistent launch); FP64 PCG of each set in turn on the same
inputs is timed next to it (`other_mode`).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the CPU oracle (the plain FP64 reference of the
method) on a complete small instance of the same workload recipe, each phase
scaled to the full workload by the oracle's own cost law.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MAX_ITER = 20000
DATA = {
    "kuhn9": "Kuhn lattice of the unit cube, k = 1",
    "lognormal64": "jittered-lattice Delaunay cube, lognormal k (sigma 1) per tet",
    "cracked128": "jittered-lattice Delaunay cube, k = 1, 2000 penny cracks",
    "growth96": "jittered-lattice Delaunay cube, k = 1, 1500 penny cracks at 64 radius scales",
    "hetero192": "jittered-lattice Delaunay cube, lognormal k (sigma 1.5), 5000 penny cracks, "
                 "8 Dirichlet value sets",
}
METRIC = "PCG time to rel-res 1e-10 & SpMV HBM GB/s: mixed/batched vs FP64, 1 GB300"
L2_FLUSH = 512 << 20


def sync_ranks(world, device):
    """Device synchronize, then a barrier across ranks: brackets the timed
    region on both sides."""
    import torch
    if device is not None and torch.device(device).type == "cuda":
        torch.cuda.synchronize(device)
    if world > 1:
        torch.distributed.barrier()


def max_over_ranks(x, world, device="cpu"):
    """The largest value of x over all ranks (the slowest rank's time)."""
    if world <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def rank_instances(B, rank, world):
    """Global ids of the instances rank `rank` solves when each of `world`
    ranks solves B of them (weak scaling: the work per GPU is fixed, the job
    solves B * world instances; instances are independent, so the ranks
    exchange nothing but the k_eff results)."""
    return list(range(rank * B, (rank + 1) * B))


def gather_instances(values, world, device="cpu"):
    """Every rank's per-instance values, concatenated in global instance
    order (rank 0's first), on every rank."""
    v = np.asarray(values, dtype=np.float64)
    if world <= 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor(v, dtype=torch.float64, device=device)
    parts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(parts, t)
    return np.concatenate([p.cpu().numpy() for p in parts])


def _log(msg):
    print(f"[bench] {msg}", file=sys.stderr, flush=True)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,"
              "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None

    def __enter__(self):
        import threading
        self.lines = []
        first = threading.Event()
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device),
                 f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return self

        def reader():
            for line in self.proc.stdout:
                self.lines.append(line)
                first.set()
            first.set()
        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()
        # nvidia-smi's start-up (driver queries) must not overlap the timed
        # region: wait for its first sample
        first.wait(timeout=10.0)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.thread.join(timeout=5)
        self.out = "".join(getattr(self, "lines", []))

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [],
                    "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------- GPU arm
def gpu_arm(args, rank, world):
    import torch
    from dec_inputs import make_workload
    from paper_2104_05999_gb300 import abi, _build

    dev_id = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev_id)
    dev = torch.device("cuda", dev_id)
    _build.build()
    t0 = time.time()
    wl = make_workload(args.workload, N=args.N)
    B_rank = wl.batch
    if world > 1 and wl.scales is None and wl.T0.shape[0] > 1:
        # Dirichlet value sets: rank r solves sets r*B .. r*B + B - 1 of one
        # recipe drawn for all ranks (set 0, the paper's problem, on rank 0)
        allw = make_workload(args.workload, N=args.N, n_sets=B_rank * world)
        wl.T0 = np.ascontiguousarray(allw.T0[rank_instances(B_rank, rank, world)])
    _log(f"inputs {wl.name}: n={wl.n} m={wl.m} in {time.time() - t0:.1f} s")
    stream = torch.cuda.Stream(device=dev)
    ctx = abi.Context(device=dev_id, stream=stream.cuda_stream)
    t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    d_xyz, d_tets, d_tags, d_T0 = t(wl.xyz), t(wl.tets), t(wl.tags), t(wl.T0)
    d_k, d_discs = t(wl.k), t(wl.discs)
    d_scales = t(wl.scales)
    flush = torch.empty(L2_FLUSH, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    want = wl.mode if args.mode == "auto" else args.mode
    modes = {"fp64": abi.DEC_MODE_FP64, "mixed": abi.DEC_MODE_MIXED,
             "mixed_phased": abi.DEC_MODE_MIXED_PHASED,
             "batched": abi.DEC_MODE_MIXED_BATCHED}
    mode64 = modes[want]
    # comparison: FP64 per instance for the mixed and batched modes, mixed for FP64
    other = abi.DEC_MODE_MIXED if want == "fp64" else abi.DEC_MODE_FP64

    def precond_for(mode):
        if mode == abi.DEC_MODE_MIXED_BATCHED:
            return abi.DEC_PRECOND_FSAI_SHARED
        return abi.DEC_PRECOND_FSAI if wl.precond == "fsai" else abi.DEC_PRECOND_JACOBI
    rtol = wl.rtol

    # pinned host copies for the end-to-end measurement
    pin = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
    h_xyz, h_tets, h_tags, h_T0 = pin(wl.xyz), pin(wl.tets), pin(wl.tags), pin(wl.T0)
    h_k, h_discs, h_scales = pin(wl.k), pin(wl.discs), pin(wl.scales)

    def step(mode, host=False, T_out=None):
        src = wl if host else None
        pc = precond_for(mode)
        if host:
            ctx.dec_mesh_upload(h_xyz, h_tets, h_tags)
            ctx.dec_hodge_assemble(h_k, h_discs, h_scales)
            ctx.dec_laplacian_build(h_T0, pc)
        else:
            ctx.dec_mesh_upload(d_xyz, d_tets, d_tags)
            ctx.dec_hodge_assemble(d_k, d_discs, d_scales)
            ctx.dec_laplacian_build(d_T0, pc)
        st, iters, relres = ctx.dec_solve(rtol, MAX_ITER, mode, T_out)
        q_in, q_out, en = ctx.dec_k_eff()
        del src
        return iters, relres, q_in

    def timed(mode, steps, warmup, host=False, bracket=False):
        T_out = None
        if host:
            T_out = torch.empty((wl.batch, wl.n), dtype=torch.float64).pin_memory()
        for _ in range(warmup):
            step(mode, host, T_out)
        if bracket:
            sync_ranks(world, dev)
        times = []
        launches0 = ctx.dec_get_launch_count()
        res = None
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush.fill_(1)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            res = step(mode, host, T_out)
            with torch.cuda.stream(stream):
                e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            if mode == abi.DEC_MODE_MIXED_BATCHED:
                # device time of the batched kernel's launch in this step
                # (CUDA events on the context's stream, around the launch)
                kernel_ms.append(ctx.dec_get_batch_kernel_ms())
        launches = (ctx.dec_get_launch_count() - launches0) / max(steps, 1)
        if bracket:
            sync_ranks(world, dev)
        return times, res, launches

    kernel_ms = []


    with ClockSampler(dev_id) as clk:
        times, (iters, relres, q_in), launches = timed(mode64, args.steps, args.warmup,
                                                       bracket=True)
    batch_kernel_ms = list(kernel_ms)
    _log(f"timed steps: {[round(t, 3) for t in times]} ms")
    ms = max_over_ranks(statistics.mean(times), world, dev)

    # the other precision on the same inputs (comparison, fewer steps)
    o_times, (o_iters, o_relres, o_q), _ = timed(other, max(2, args.steps // 2), 1)
    _log(f"other mode: {[round(t, 3) for t in o_times]} ms")
    # end to end through host buffers (H2D of the inputs, D2H of T and k_eff)
    e_times, _, _ = timed(mode64, max(2, args.steps // 2), 1, host=True)
    h2d = (wl.xyz.nbytes + wl.tets.nbytes + wl.tags.nbytes + wl.T0.nbytes +
           (wl.k.nbytes if wl.k is not None else 0) +
           (wl.discs.nbytes if wl.discs is not None else 0))
    d2h = wl.batch * wl.n * 8 + 3 * 8 * wl.batch

    # per-phase breakdown of one (untimed) device-resident step
    import torch as _t
    ev = [_t.cuda.Event(enable_timing=True) for _ in range(6)]
    pc = precond_for(mode64)
    with _t.cuda.stream(stream):
        flush.fill_(1)
        ev[0].record(stream)
    ctx.dec_mesh_upload(d_xyz, d_tets, d_tags)
    ev[1].record(stream)
    ctx.dec_hodge_assemble(d_k, d_discs, d_scales)
    ev[2].record(stream)
    ctx.dec_laplacian_build(d_T0, pc)
    ev[3].record(stream)
    ctx.dec_solve(rtol, MAX_ITER, mode64, None)
    ev[4].record(stream)
    ctx.dec_k_eff()
    ev[5].record(stream)
    ev[5].synchronize()
    phases = {name: round(ev[i].elapsed_time(ev[i + 1]), 4) for i, name in enumerate(
        ("mesh_upload", "hodge_assemble", "laplacian_build", "solve", "k_eff"))}
    _log(f"phases ms: {phases}")

    # the same step with FP32 geometry for well-shaped tets (DEC_GEOM_MIXED):
    # Hodge time, tets kept in FP64 and the change of k_eff (untimed step)
    ev2 = [_t.cuda.Event(enable_timing=True) for _ in range(2)]
    ctx.dec_set_geom_precision(abi.DEC_GEOM_MIXED)
    ctx.dec_mesh_upload(d_xyz, d_tets, d_tags)
    with _t.cuda.stream(stream):
        flush.fill_(1)
        ev2[0].record(stream)
    ctx.dec_hodge_assemble(d_k, d_discs, d_scales)
    ev2[1].record(stream)
    ev2[1].synchronize()
    n_fp64_tets = ctx.dec_get_geom_fp64_tets()
    ctx.dec_laplacian_build(d_T0, pc)
    ctx.dec_solve(rtol, MAX_ITER, mode64, None)
    q_geo = ctx.dec_k_eff()[0]
    ctx.dec_set_geom_precision(abi.DEC_GEOM_FP64)
    geom_mixed = {"hodge_assemble_ms": round(ev2[0].elapsed_time(ev2[1]), 4),
                  "hodge_assemble_ms_fp64_geometry": phases["hodge_assemble"],
                  "fp64_tets": int(n_fp64_tets), "tets": int(wl.m),
                  "k_eff_rel_diff": float(np.max(np.abs(q_geo - q_in)) / np.max(np.abs(q_in)))}
    _log(f"FP32 geometry: {geom_mixed}")

    # solve-only timing: time dec_solve alone (assembly already done)
    step(mode64)
    s_times = []
    for _ in range(3):
        with torch.cuda.stream(stream):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        ctx.dec_solve(rtol, MAX_ITER, mode64, None)
        with torch.cuda.stream(stream):
            e1.record(stream)
        e1.synchronize()
        s_times.append(e0.elapsed_time(e1))

    # roofline of the dominant kernel: cold-L2 launches of the CSR SpMV
    n, m, ne, nnz, B = ctx.sizes()
    spmv_ms = ctx.dec_time_kernel(abi.DEC_KERNEL_SPMV_F64, reps=20)
    spmv32_ms = ctx.dec_time_kernel(abi.DEC_KERNEL_SPMV_F32, reps=20)
    fsai_ms = fsai16_ms = None
    if precond_for(mode64) != abi.DEC_PRECOND_JACOBI:
        fsai_ms = ctx.dec_time_kernel(abi.DEC_KERNEL_FSAI_F64, reps=20)
        fsai16_ms = ctx.dec_time_kernel(abi.DEC_KERNEL_FSAI_BF16, reps=20)
    bytes64 = 12 * nnz + 4 * (n + 1) + 16 * n
    bytes32 = 8 * nnz + 4 * (n + 1) + 8 * n
    nnz_g = (nnz + n) // 2
    fsai_bytes64 = 2 * (12 * nnz_g + 4 * (n + 1) + 16 * n) + 8 * n
    fsai_bytes16 = 2 * (6 * nnz_g + 4 * (n + 1) + 8 * n) + 4 * n
    peak, peak_kind = _peaks()
    solve_ms = statistics.mean(s_times)
    # the dominant kernel of the timed mode: the FP64 SpMV (FP64 mode), the
    # FP32 SpMV (mixed modes) or the batched persistent PCG, whose figure is
    # per iteration: algorithmic bytes of one iteration over the solve time
    # per iteration of the slowest instance
    roof_kernel = "spmv_pq_kernel<double,double> (SELL-32 SpMV + p.q, FP64)"
    roof_bytes, roof_ms = bytes64, spmv_ms
    if want in ("mixed", "mixed_phased"):
        roof_kernel = "spmv_pq_kernel<float,float> (SELL-32 SpMV + p.q, FP32)"
        roof_bytes, roof_ms = bytes32, spmv32_ms
    elif want == "batched":
        BS = 8
        while BS < B:
            BS *= 2
        per_inst_g = wl.scales is not None and len(wl.scales) > 1
        vec = 4 * n * BS
        # algorithmic bytes of one launch (the whole batched solve): the
        # shared structure once per iteration of the slowest instance, the
        # [n][BS] FP32 vectors per iteration (15 passes) for the mean
        # iteration count
        struct = 9 * nnz + 2 * nnz_g * (4 + 2 * (BS if per_inst_g else 1))
        roof_bytes = (struct * int(np.max(iters)) +
                      vec * 15 * float(np.mean(iters)))
        roof_ms = statistics.mean(batch_kernel_ms)
        roof_kernel = ("pcg_batched_persistent (one launch = the whole solve of "
                       "%d instances; mean of the timed steps' launches)" % B)
    roof_gbs = roof_bytes / (roof_ms * 1e-3) / 1e9
    # DRAM traffic of the dominant kernel from an ncu capture stored in
    # profiles/traffic.json, scaled to this launch by the units it processes;
    # null when the kernel's source file has changed since the capture
    traffic = None
    if want == "batched":
        traffic = stored_traffic("pcg_batched_persistent",
                                 n * int(np.max(iters)), B)
    clocks = clk.summary()
    # k_eff of every rank's instances, in global order
    q_all = gather_instances(q_in, world, dev)

    out = {
        "metric": METRIC, "value": round(ms, 4), "unit": "ms",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms, 4), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if want == "fp64" else "f32 (bf16 FSAI values; f64 residual and k_eff)",
        "data": "synthetic, seeded: " + DATA.get(wl.name.split("@")[0], "jittered-lattice Delaunay cube"),
        "config": {"workload": wl.name, "n_nodes": n, "n_tets": m,
                   "n_edges": ne, "nnz": nnz, "instances": B * world,
                   "instances_per_gpu": B,
                   "precond": wl.precond,
                   "mode": want,
                   "rtol": rtol, "l2": "flushed (512 MiB write) between steps",
                   "step": "mesh_upload+hodge+laplacian+FSAI+PCG+k_eff"},
        "iters": int(iters[0]), "relres": float(np.max(relres)),
        "k_eff": float(q_in[0]),
        "iters_per_instance": [int(v) for v in iters] if len(iters) > 1 else None,
        "k_eff_per_instance": [float(v) for v in q_all] if len(q_all) > 1 else None,
        "solve_ms": round(solve_ms, 4),
        "phases_ms": phases,
        "other_mode": {"mode": "mixed" if other == abi.DEC_MODE_MIXED else "fp64 per instance",
                       "ms_per_step": round(statistics.mean(o_times), 4),
                       "iters": int(o_iters[0]), "relres": float(o_relres[0]),
                       # largest k_eff difference over the largest |k_eff|
                       # (Dirichlet value sets can have fluxes near 0)
                       "k_eff_rel_diff": float(np.max(np.abs(o_q - q_in)) / np.max(np.abs(q_in)))},
        "kernels_ms": {"spmv_f64": spmv_ms, "spmv_f32": spmv32_ms,
                       "fsai_apply_f64": fsai_ms, "fsai_apply_bf16": fsai16_ms},
        "kernels_gbs": {
            "spmv_f64": round(bytes64 / (spmv_ms * 1e-3) / 1e9, 1),
            "spmv_f32": round(bytes32 / (spmv32_ms * 1e-3) / 1e9, 1),
            "fsai_apply_f64": round(fsai_bytes64 / (fsai_ms * 1e-3) / 1e9, 1) if fsai_ms else None,
            "fsai_apply_bf16": round(fsai_bytes16 / (fsai16_ms * 1e-3) / 1e9, 1) if fsai16_ms else None},
        "roofline": {"kernel": roof_kernel,
                     "bound": "hbm", "achieved": round(roof_gbs, 1),
                     "peak": peak, "unit": "GB/s", "frac": round(roof_gbs / peak, 4),
                     "peak_kind": f"{peak_kind} burst copy",
                     "traffic": traffic,
                     "algorithmic_bytes": int(roof_bytes),
                     "duration_ms": round(roof_ms, 5)},
        "e2e": {"value": round(statistics.mean(e_times), 4), "unit": "ms",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(round(launches)),
        "geom_mixed": geom_mixed,
        # launch shapes the single-instance autotuner picked (L, FSAI halves)
        "sell_shapes": {"fp64": list(ctx.dec_get_sell_variant(0)),
                        "fp32": list(ctx.dec_get_sell_variant(1))},
        "batch_variant": ctx.dec_get_batch_variant() if want == "batched" else None,
        "batch_phase_ms": ([round(float(x), 4) for x in ctx.dec_get_batch_phase_ms()]
                           if want == "batched" else None),
        "clocks": clocks,
    }
    ctx.close()
    return out


def stored_traffic(kernel, units, instances):
    """Bytes per launch from profiles/traffic.json: the measured DRAM bytes
    per unit times ``units``, if the entry was taken with ``instances``
    instances and the SHA-256 of its source file still matches."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            entry = json.load(f)[kernel]
        with open(os.path.join(ROOT, entry["source"]), "rb") as f:
            digest = hashlib.sha256(f.read()).hexdigest()
    except (OSError, KeyError, ValueError):
        return None
    if digest != entry["sha256"] or entry["instances"] != instances:
        return None
    return int(entry["bytes_per_unit"] * units)


def crack_growth_measure(max_steps=600, oracle_steps=3, paths=64, path_steps=200):
    """Crack growth on a mesh of the size of the paper's crack study (a 15^3
    jittered Delaunay cube, 3,375 nodes, k = 1):
      * max-flux rule (Sec. 3.3): GPU time per step (crack + update + solve +
        k_eff) with row updates and warm starts, and with a full rebuild and
        a cold start per step, over up to max_steps steps; CG iterations;
      * Monte-Carlo paths (Sec. 3.4): `paths` random orders cracked together
        as one batch, time per path-step over `path_steps` steps;
      * the oracle's time per step over a few steps on the host."""
    import oracle as O
    from dec_inputs import make_workload
    from paper_2104_05999_gb300 import abi
    wl = make_workload("lognormal64", N=15)
    dev = int(os.environ.get("LOCAL_RANK", 0))
    out = {"mesh": f"15^3 jittered Delaunay cube, k = 1 ({wl.n} nodes, {wl.m} tets)",
           "rule": "max_flux"}
    for rebuild in (False, True):
        ctx = abi.Context(device=dev)
        ctx.dec_mesh_upload(wl.xyz, wl.tets, wl.tags)
        ctx.dec_hodge_assemble(None)
        ctx.dec_laplacian_build(wl.T0[:1], abi.DEC_PRECOND_FSAI)
        rule = abi.DEC_CRACK_MAX_FLUX | (abi.DEC_CRACK_REBUILD if rebuild else 0)
        t0 = time.perf_counter()
        _, cracked, keff = ctx.dec_crack_evolve(rule, max_steps, rtol=1e-10)
        dt = time.perf_counter() - t0
        its = ctx.dec_get_crack_iterations()
        ctx.close()
        key = "rebuild_cold_start" if rebuild else "row_update_warm_start"
        out[key] = {"steps": int(len(cracked)),
                    "ms_per_step": round(1000 * dt / max(1, len(cracked)), 3),
                    "cg_iters_per_step": round(its / max(1, len(cracked)), 1),
                    "k_eff_after_first": float(keff[0]), "k_eff_last": float(keff[-1])}
    out["ms_per_step"] = out["row_update_warm_start"]["ms_per_step"]
    # Monte-Carlo paths, batched
    E, t2e = O.edge_list(wl.tets)
    w = O.hodge_star1(wl.xyz, wl.tets, E, t2e, None)
    cand = np.flatnonzero(O.crackable_edges(w))
    orders = np.stack([np.random.default_rng(500 + b).permutation(cand)[:path_steps]
                       for b in range(paths)]).astype(np.int32)
    ctx = abi.Context(device=dev)
    ctx.dec_mesh_upload(wl.xyz, wl.tets, wl.tags)
    ctx.dec_hodge_assemble(None)
    ctx.dec_laplacian_build(wl.T0[:1], abi.DEC_PRECOND_FSAI)
    t0 = time.perf_counter()
    _, keffs, steps = ctx.dec_crack_paths(orders, rtol=1e-10)
    dt = time.perf_counter() - t0
    its = ctx.dec_get_crack_iterations()
    ctx.close()
    done = int(np.sum(steps))
    out["monte_carlo_paths"] = {
        "paths": paths, "steps_per_path": path_steps,
        "ms_per_path_step": round(1000 * dt / max(1, done), 4),
        "ms_per_batched_step": round(1000 * dt / max(1, int(np.max(steps))), 3),
        "cg_iters_per_path_step": round(its / max(1, done), 1),
        "k_eff_last_mean": float(np.mean([k[-1] for k in keffs]))}
    t0 = time.perf_counter()
    O.crack_evolution(wl.xyz, wl.tets, wl.tags, wl.T0[0], k=None,
                      max_steps=oracle_steps, rtol=1e-10)
    ot = (time.perf_counter() - t0) / (oracle_steps + 1)   # + the first solve
    out["oracle_ms_per_step"] = round(1000 * ot, 1)
    out["oracle"] = "oracle.crack_evolution, numpy/scipy FP64, 1 thread"
    return out


def fields_measure(n_fields=16, N=64):
    """Many conductivity fields on one mesh (Sec. 1, Sec. 2.1): `n_fields`
    lognormal fields (sigma 1) on the 64^3 jittered Delaunay cube, solved as
    one batch (mixed precision) and one field at a time in FP64; step = Hodge
    star of every field + L + preconditioners + solve + k_eff."""
    import torch
    from dec_inputs import make_fields, make_workload
    from paper_2104_05999_gb300 import abi
    dev = int(os.environ.get("LOCAL_RANK", 0))
    wl = make_workload("lognormal64", N=N)
    k = make_fields(wl, n_fields, sigma=1.0)
    d = torch.device("cuda", dev)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(d)  # noqa: E731
    xyz, tets, tags, T0, kk = t(wl.xyz), t(wl.tets), t(wl.tags), t(wl.T0), t(k)
    res = {}
    for name, pc, mode in (("batched", abi.DEC_PRECOND_FSAI_SHARED, abi.DEC_MODE_MIXED_BATCHED),
                           ("fp64_per_field", abi.DEC_PRECOND_FSAI, abi.DEC_MODE_FP64)):
        ctx = abi.Context(device=dev)
        ctx.dec_mesh_upload(xyz, tets, tags)
        times = []
        for rep in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.dec_hodge_assemble_fields(kk)
            ctx.dec_laplacian_build(T0, pc)
            _, iters, _ = ctx.dec_solve(1e-10, MAX_ITER, mode)
            q, _, _ = ctx.dec_k_eff()
            times.append(1000 * (time.perf_counter() - t0))
        ctx.close()
        res[name] = (min(times[1:]), q, iters)
    qb, q64 = res["batched"][1], res["fp64_per_field"][1]
    return {"mesh": f"64^3 jittered Delaunay cube ({wl.n} nodes, {wl.m} tets)",
            "fields": n_fields,
            "batched_ms": round(res["batched"][0], 2),
            "fp64_per_field_ms": round(res["fp64_per_field"][0], 2),
            "iters_batched_max": int(np.max(res["batched"][2])),
            "iters_fp64_max": int(np.max(res["fp64_per_field"][2])),
            "k_eff_max_rel_diff": float(np.max(np.abs(qb - q64) / np.abs(q64)))}


def tet_measure(N=64):
    """The paper's own tet-centred form (Sec. 2.3 Eq. 11-13 with the flux
    block eliminated, Sec. 3.1 limiter): faces of the 64^3 jittered Delaunay
    cube, then the two-point operator solved by FP64 Jacobi PCG to 1e-10 with
    k = 1; q_in should be 1 (a linear field) where nothing is limited."""
    import torch
    from dec_inputs import make_workload
    from paper_2104_05999_gb300 import abi
    dev = int(os.environ.get("LOCAL_RANK", 0))
    wl = make_workload("lognormal64", N=N)
    d = torch.device("cuda", dev)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(d)  # noqa: E731
    xyz, tets, tags, T0 = t(wl.xyz), t(wl.tets), t(wl.tags), t(wl.T0[0])
    ctx = abi.Context(device=dev)
    ctx.dec_mesh_upload(xyz, tets, tags)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nf = len(ctx.dec_tet_get_faces()[0])
    faces_ms = 1000 * (time.perf_counter() - t0)
    times = []
    for rep in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = ctx.dec_tet_solve(T0, kappa=1.0, limiter=1e-8, rtol=1e-10)
        times.append(1000 * (time.perf_counter() - t0))
    ctx.close()
    return {"mesh": f"{N}^3 jittered Delaunay cube ({wl.n} nodes, {wl.m} tets, {nf} faces)",
            "faces_ms": round(faces_ms, 2), "solve_ms": round(min(times[1:]), 2),
            "iters": int(res["iters"]), "relres": float(res["relres"]),
            "limited": int(res["limited"]), "q_in": float(res["q_in"]),
            "q_out": float(res["q_out"]),
            "note": "faces_ms includes copying the faces to the host; solve_ms is the whole "
                    "dec_tet_solve call (face weights, rows, PCG, k_eff)"}


# ------------------------------------------------------------- CPU oracle
def oracle_phases(name, N_s):
    """Run the oracle's whole path, phase by phase, on the complete instance
    of workload ``name`` at lattice size ``N_s`` (same recipe: jitter, k,
    discs scaled to the lattice, every Dirichlet set or crack state solved to
    the workload's tolerance).  Returns the small instance's counts and the
    seconds of each phase."""
    import oracle as O
    from dec_inputs import make_workload
    wl = make_workload(name, N=N_s)
    T0 = np.atleast_2d(wl.T0)
    t = {}
    c = time.perf_counter()
    E, t2e = O.edge_list(wl.tets)
    t["edges"] = time.perf_counter() - c
    first = None
    t["crack_fixed"] = t["crack_discs"] = 0.0
    if wl.discs is not None:
        # the crack test's cost has a part per sub-triangle (the dual-face
        # points) and a part per (sub-triangle, disc) pair: time it without
        # discs, then with all of them
        c = time.perf_counter()
        O.edge_crack_state(wl.xyz, wl.tets, E, t2e, wl.discs[:0], wl.scales)
        t["crack_fixed"] = time.perf_counter() - c
        c = time.perf_counter()
        first = O.edge_crack_state(wl.xyz, wl.tets, E, t2e, wl.discs, wl.scales)
        t["crack_discs"] = max(0.0, time.perf_counter() - c - t["crack_fixed"])
    c = time.perf_counter()
    w0 = O.hodge_star1(wl.xyz, wl.tets, E, t2e, wl.k)
    t["hodge"] = time.perf_counter() - c
    if wl.scales is not None:
        inst = [(np.where(first <= b, 0.0, w0), T0[0]) for b in range(len(wl.scales))]
    else:
        w = w0 if first is None else np.where(first == 0, 0.0, w0)
        inst = [(w, T0[s]) for s in range(T0.shape[0])]
    t["laplacian"] = t["precond"] = t["pcg"] = t["k_eff"] = 0.0
    iters, nnz = [], 0
    dirich = wl.tags == O.DIRICHLET
    for w, t0 in inst:
        c = time.perf_counter()
        L, b, _ = O.laplacian(wl.n, E, w, wl.tags, t0)
        t["laplacian"] += time.perf_counter() - c
        nnz = L.nnz
        c = time.perf_counter()
        if wl.precond == "fsai":
            G = O.fsai_factor(L)
            Gt = G.T.tocsr()
            M = lambda r, G=G, Gt=Gt: Gt @ (G @ r)  # noqa: E731
        else:
            d = O.jacobi(L)
            M = lambda r, d=d: d * r  # noqa: E731
        t["precond"] += time.perf_counter() - c
        c = time.perf_counter()
        u, it, _ = O.pcg(L, b[0], M, wl.rtol)
        t["pcg"] += time.perf_counter() - c
        iters.append(int(it))
        c = time.perf_counter()
        O.k_eff(wl.xyz, E, w, u + np.where(dirich, t0, 0.0), wl.tags)
        t["k_eff"] += time.perf_counter() - c
    nd = 0 if wl.discs is None else len(wl.discs)
    return dict(N=N_s, n=wl.n, m=wl.m, nnz=nnz, nd=nd, inst=len(inst),
                iters=iters, sec=t)


def oracle_scaled(name, small, full):
    """Scale the oracle's measured phases on the small instance to the full
    workload by the oracle's own cost laws: edge list, Hodge star, L and
    preconditioner set-up grow with the number of tets; the crack test has a
    part per sub-triangle (tets) and a brute force over every (sub-triangle,
    disc) pair (tets x discs); PCG grows with matrix entries x iterations, and FSAI-PCG
    iterations on these cubes grow in proportion to the lattice size (about
    3.8 per lattice spacing on the 16^3, 24^3 and 32^3 instances of the
    heterogeneous cracked cube).  ``full`` holds N, n, m, nnz, nd (counts
    of the full workload; m and nnz may come from lattice scaling).
    Returns (ms per step, description, detail dict)."""
    sec = small["sec"]
    fm = full["m"] / small["m"]
    fcr = fm * (max(full["nd"], 1) / max(small["nd"], 1))
    fit = (full["N"] - 1) / (small["N"] - 1)
    fpcg = full["nnz"] / small["nnz"] * fit
    scaled = {"edges": sec["edges"] * fm, "crack_fixed": sec["crack_fixed"] * fm,
              "crack_discs": sec["crack_discs"] * fcr,
              "hodge": sec["hodge"] * fm, "laplacian": sec["laplacian"] * fm,
              "precond": sec["precond"] * fm, "pcg": sec["pcg"] * fpcg,
              "k_eff": sec["k_eff"] * fm}
    ms = 1e3 * sum(scaled.values())
    # crack_fixed is measured once more inside the full crack test: count it
    # once
    measured_ms = 1e3 * (sum(sec.values()) - sec["crack_fixed"])
    desc = (f"oracle (numpy/scipy FP64, 1 thread), whole path on the complete "
            f"{name}@{small['N']} instance ({small['n']} nodes, {small['m']} tets, "
            f"{small['nd']} discs, {small['inst']} instances solved to the "
            f"workload's tolerance in {min(small['iters'])}-{max(small['iters'])} "
            f"iterations): {measured_ms:.0f} ms measured; each phase scaled to the "
            f"full workload by the oracle's cost law (tets; crack test tets x "
            f"discs; PCG entries x iterations, iterations in proportion to the "
            f"lattice size)")
    detail = {"measured_ms": round(measured_ms, 1),
              "measured_instance": f"{name}@{small['N']}",
              "measured_phases_ms": {k: round(1e3 * v, 1) for k, v in sec.items()},
              "scaled_phases_ms": {k: round(1e3 * v, 1) for k, v in scaled.items()},
              "iterations_measured": small["iters"],
              "iterations_scaled": int(round(np.mean(small["iters"]) * fit))}
    return ms, desc, detail


def full_counts(name, N, small, exact=None):
    """Counts of the full workload: exact when the GPU arm has them, else
    scaled from the small instance by the lattice's cell count."""
    from dec_inputs.workloads import WORKLOADS
    N0 = WORKLOADS[name][1] if N is None else N
    nd0 = WORKLOADS[name][4]
    if exact is not None:
        n, m, nnz = exact
    else:
        f = ((N0 - 1) / (small["N"] - 1)) ** 3
        n, m, nnz = N0 ** 3, small["m"] * f, small["nnz"] * f
    nd = nd0 if N is None else max(1, int(round(nd0 * (N / WORKLOADS[name][1]) ** 3)))
    return {"N": N0, "n": n, "m": m, "nnz": nnz, "nd": nd if nd0 else 0}


def reference_arm(args):
    times = []
    desc, detail = "", {}
    N_s = args.ref_N
    for i in range(args.warmup + args.steps):
        small = oracle_phases(args.workload, N_s)
        full = full_counts(args.workload, args.N, small)
        ms, desc, detail = oracle_scaled(args.workload, small, full)
        if i >= args.warmup:
            times.append(ms)
    ms = statistics.mean(times)
    from dec_inputs.workloads import WORKLOADS
    mode = WORKLOADS[args.workload][10]
    return {
        "metric": METRIC, "value": round(ms, 2), "unit": "ms", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 2),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": args.workload if args.N is None else f"{args.workload}@{args.N}",
                   "precond": "fsai", "mode": mode, "rtol": 1e-10},
        "cpu_baseline": {"value": round(ms, 2), "unit": "ms", "cores": 1,
                         "kind": "oracle", "sample": desc, **detail},
        "e2e": {"value": round(ms, 2), "unit": "ms", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="hetero192")
    # another lattice size of the same workload recipe (small profiling cases)
    ap.add_argument("--N", type=int, default=None)
    ap.add_argument("--mode", default="auto",
                    choices=["auto", "fp64", "mixed", "mixed_phased", "batched"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tet-only", action="store_true",
                    help="only the tet-centred form's measurement (lattice --N, default 64)")
    # lattice size of the complete small instance the oracle runs: per
    # reference-arm step, and for the GPU arm's cpu_baseline
    ap.add_argument("--ref-N", type=int, default=14)
    ap.add_argument("--baseline-N", type=int, default=24)
    args = ap.parse_args()
    if args.tet_only:
        from paper_2104_05999_gb300 import _build
        _build.build()
        print(json.dumps(tet_measure(N=args.N or 64)), flush=True)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(reference_arm(args)), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    out = gpu_arm(args, rank, world)
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:
            small = oracle_phases(args.workload, args.baseline_N)
            c = out["config"]
            full = full_counts(args.workload, args.N, small,
                               exact=(c["n_nodes"], c["n_tets"], c["nnz"]))
            ms, desc, detail = oracle_scaled(args.workload, small, full)
            out["cpu_baseline"] = {"value": round(ms, 1), "unit": "ms",
                                   "cores": 1, "kind": "oracle",
                                   "sample": desc, **detail}
            out["crack_growth"] = crack_growth_measure()
            out["conductivity_fields"] = fields_measure()
            out["tet_centred"] = tet_measure()
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
