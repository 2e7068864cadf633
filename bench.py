"""Benchmark of the NOLSM hot path on one GB300 (prints one JSON line).

A step is one pass of the whole hot path over the synthetic system: nolsm_build_submatrices (a0),
nolsm_find_mu (a1-a7 for every submatrix at every bisection point, a9) and nolsm_scatter_density
(a8). value = submatrices / s = molecules / step time, device-timed with CUDA events, inputs resident
in HBM. e2e is the same step through the same public calls with the block-CSR inputs copied from
pinned host memory each step and D copied back. The sign-iteration kernel's achieved tensor rate is
taken from the library's own CUDA-event timers (same stream) and its algorithmic flop count.

--impl reference times the FP64 CPU oracle on the host cores: each step runs the oracle's bisection
for mu on a bounded sample of the same system's submatrices (electron count of the sample).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "batched_uneven": ("spec_batched_uneven",
                       "water-like lattice, 32768 molecules (32x32x32), 6 functions each, +-20% local "
                       "length-scale field, 6 A cutoff"),
    "small_fp64": ("spec_small_fp64", "water-like lattice, 64 molecules (4x4x4), 6 functions each, 6 A cutoff"),
    "uneven_4096": ("spec_batched_uneven_4096",
                    "water-like lattice, 4096 molecules (16x16x16), 6 functions each, +-20% local length-scale "
                    "field, 6 A cutoff (profiling size)"),
    "streamed_bf16": ("spec_streamed_bf16",
                      "water-like lattice, 262144 molecules (64x64x64), 6 functions each, 6 A cutoff"),
    "split_valence": ("spec_split_valence",
                      "water-like lattice, 16384 molecules (32x32x16), 23 functions each (split-valence-like), "
                      "6 A cutoff"),
    "mixed": ("spec_mixed",
              "water-like lattice, 65536 molecules (64x32x32), 6 or 23 functions per molecule (50/50), 6 A cutoff"),
}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": d.get("hbm_gbs"), "bf16": d.get("bf16_tflops"),
                "bf16_sustained": d.get("bf16_tflops_sustained"), "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16": 1900.0, "bf16_sustained": 1700.0, "source": "fallback"}


# the metric both arms report (the reference arm on a bounded sample of the same workload)
METRIC = "submatrices/s (NOLSM step: plan, mu bisection, write-back) and sign-iteration TFLOP/s"

# FP32 SIMT peak from the unit counts: 152 SMs x 128 FP32 lanes x 2 flops (FMA) x 2.07 GHz maximum SM clock
FP32_ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def _src_sha(rel):
    import hashlib
    with open(os.path.join(ROOT, rel), "rb") as f:
        return hashlib.sha1(f.read()).hexdigest()


def kernel_traffic(kernel, units_per_launch):
    """DRAM bytes per launch of a kernel from the committed ncu summary (profiles/traffic.json), scaled
    by the units (submatrices) one launch processes; None when the kernel's source changed since the
    counters were taken or no capture exists."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f).get(kernel)
    if not d or _src_sha(d["source"]) != d["source_sha1"]:
        return None
    return d["dram_bytes"] / d["units"] * units_per_launch


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
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
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------ oracle (CPU)

_ORC = {}


def _oracle_init(spec_name, spec_kw):
    import synth
    from oracle import nolsm_oracle as orc
    sysm = synth.make_system(getattr(synth, spec_name)(**spec_kw))
    _ORC["sys"] = sysm
    _ORC["plan"] = orc.build_plan(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.H.row_ptr, sysm.H.col_idx)


def _oracle_solve(args):
    from oracle import nolsm_oracle as orc
    subs, mu = args
    r = orc.solve(_ORC["sys"], mu, subs=subs, plan=_ORC["plan"])
    return {J: (s.D_cols, s.t_S, s.t_H) for J, s in r.subs.items()}


def _oracle_gersh(subs):
    """Spectral interval of A_J for the listed submatrices (for the reference arm's bracket)."""
    import numpy as np
    from oracle import nolsm_oracle as orc
    sysm, plan = _ORC["sys"], _ORC["plan"]
    lo, hi = np.inf, -np.inf
    for J in subs:
        S = orc.gather(plan, J, sysm.S.row_ptr, sysm.S.col_idx, sysm.S.blk_off, sysm.S.vals)
        H = orc.gather(plan, J, sysm.H.row_ptr, sysm.H.col_idx, sysm.H.blk_off, sysm.H.vals)
        A = orc.overlap_inverse(S) @ H
        d = np.diag(A)
        R = np.sum(np.abs(A), axis=1) - np.abs(d)
        lo, hi = min(lo, float(np.min(d - R))), max(hi, float(np.max(d + R)))
    return lo, hi


def oracle_pool(spec_name, spec_kw, workers):
    import multiprocessing as mp
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    ctx = mp.get_context("spawn")
    return ctx.Pool(workers, initializer=_oracle_init, initargs=(spec_name, spec_kw))


def run_oracle(pool, subs, mu, workers):
    chunks = [subs[i::workers] for i in range(workers)]
    t0 = time.perf_counter()
    parts = pool.map(_oracle_solve, [(c, mu) for c in chunks if c])
    dt = time.perf_counter() - t0
    out = {}
    for p in parts:
        out.update(p)
    return out, dt


# ------------------------------------------------------------------------------------ reference arm

def reference_arm(args, spec_name, desc):
    import numpy as np
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    workers = max(1, os.cpu_count() or 1)
    pool = oracle_pool(spec_name, {}, workers)
    import synth
    n_mol = getattr(synth, spec_name)().n_mol
    rng = np.random.default_rng(7)
    sample = sorted(int(j) for j in rng.choice(n_mol, size=min(n_mol, args.ref_sample), replace=False))
    chunks = [sample[i::workers] for i in range(workers)]
    bounds = pool.map(_oracle_gersh, [c for c in chunks if c])
    lo, hi = min(b[0] for b in bounds), max(b[1] for b in bounds)
    n_occ = 4.0 * len(sample)

    def step():
        from oracle import nolsm_oracle as orc
        evals = []

        def count(mu):
            res, _ = run_oracle(pool, sample, mu, workers)
            evals.append(mu)
            return sum(v[1] for v in res.values())
        r = orc.find_mu(count, n_occ, lo, hi, tol_n=1e-5 * n_occ)
        return r, len(evals)

    for _ in range(args.warmup):
        step()
    times = []
    nev = 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        _, nev = step()
        times.append(time.perf_counter() - t0)
    pool.close()
    ms = 1e3 * statistics.mean(times)
    value = len(sample) / (ms / 1e3)
    line = {"impl": "reference", "metric": METRIC,
            "value": value, "unit": "submatrices/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "precision": "fp64 CPU oracle", "molecules": n_mol,
                       "molecules_per_gpu": n_mol, "bracket": "Gershgorin interval of the sampled submatrices",
                       "sample": f"{len(sample)} submatrices, their own electron count, {nev} bisection points"},
            "cpu_baseline": {"value": value, "unit": "submatrices/s", "cores": workers, "kind": "oracle",
                             "sample": f"oracle bisection on {len(sample)} sampled submatrices per step"},
            "e2e": {"value": value, "unit": "submatrices/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------ bound sources

def bound_sources_leg(nl, synth, spec_name, dsys, mu_star, precision, dev):
    """a4/a10: the learned predictor trained on samples the method produces on this system (power
    interval and step counts at three chemical potentials around mu*), then Gershgorin, power and
    learned bounds compared on a fresh system of the same kind (another seed) at mu*."""
    import dataclasses

    import torch
    o = nl.options(precision)
    plan = nl.nolsm_build_submatrices(dsys)
    t0 = time.perf_counter()
    xs, ts = [], []
    for dmu in (-0.05, 0.0, 0.05):
        x, t = nl.nolsm_training_data(plan, mu_star + dmu, o)
        xs.append(x)
        ts.append(t)
    x, t = torch.cat(xs), torch.cat(ts)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    plan.close()
    mlp = nl.Mlp(seed=11)
    t0 = time.perf_counter()
    losses = mlp.train(x, t, epochs=30, batch=1024, lr=2e-3)
    t_train = time.perf_counter() - t0
    spec = getattr(synth, spec_name)()
    fresh = synth.make_system(dataclasses.replace(spec, seed=spec.seed + 1000))
    p2 = nl.nolsm_build_submatrices(nl.DeviceSystem(fresh, dev))
    nl.nolsm_plan_set_mlp(p2, mlp)
    out = {"training_samples": int(x.shape[0]), "epochs": 30, "batch": 1024,
           "loss_first_last": [losses[0], losses[-1]], "s_training_data": t_data, "s_training": t_train,
           "evaluated_on": f"fresh system of the same workload (seed {spec.seed + 1000}), mu*"}
    ref = None
    for name, b in (("gershgorin", nl.BOUND_GERSHGORIN), ("power", nl.BOUND_POWER), ("mlp", nl.BOUND_MLP)):
        ob = nl.options(precision, bound_source=b)
        nl.nolsm_solve_batch(p2, mu_star, ob, check=False)          # geometry caches, power bounds
        p2.stats_reset()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = nl.nolsm_solve_batch(p2, mu_star, ob, check=False)
        dt = time.perf_counter() - t0
        s2 = p2.stats()
        D = p2.scatter()
        if ref is None:
            ref = D.clone()
        out[name] = {"mean_ns_steps": float(r.iters.float().mean()), "ms_sign": s2["ms_sign"],
                     "ms_solve_call": dt * 1e3, "submatrices_per_s_one_mu": fresh.n_mol / dt,
                     "reruns": int(s2["reruns"]), "status": int(r.status),
                     "not_converged": int((r.sub_status != 0).sum()),
                     "max_abs_dD_vs_gershgorin": float((D - ref).abs().max())}
    p2.close()
    return out


# ------------------------------------------------------------------------------------ our arm

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16x3")
    ap.add_argument("--workload", default="batched_uneven", choices=list(WORKLOADS))
    ap.add_argument("--sample", type=int, default=640, help="oracle submatrices for accuracy and CPU baseline")
    ap.add_argument("--ref-sample", type=int, default=96, help="submatrices per reference-arm step")
    ap.add_argument("--no-extra", action="store_true", help="skip the per-precision side measurements")
    ap.add_argument("--no-oracle", action="store_true", help="skip the CPU oracle (profiling runs)")
    args = ap.parse_args()
    spec_name, desc = WORKLOADS[args.workload]
    if args.impl == "reference":
        return reference_arm(args, spec_name, desc)

    import numpy as np
    import torch

    import paper_2104_08245_gb300 as nl
    import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    # weak scaling: with N ranks the lattice is N times longer along x and rank r owns the r-th slab of
    # the one-GPU workload's size (molecule index runs fastest along z, slowest along x)
    spec = getattr(synth, spec_name)()
    if world > 1:
        import dataclasses
        spec = dataclasses.replace(spec, nx=spec.nx * world)
    sysm = synth.make_system(spec)
    n_mol = sysm.n_mol
    n_occ = sysm.n_occ
    peaks = measured_peaks()
    opts = nl.options(args.precision)

    # host copies (pinned) for the e2e leg; device copies for the resident leg
    host = {"nbf": torch.from_numpy(sysm.nbf).pin_memory(),
            "s_row_ptr": torch.from_numpy(sysm.S.row_ptr).pin_memory(),
            "s_col_idx": torch.from_numpy(sysm.S.col_idx).pin_memory(),
            "s_vals": torch.from_numpy(sysm.S.vals).pin_memory(),
            "h_row_ptr": torch.from_numpy(sysm.H.row_ptr).pin_memory(),
            "h_col_idx": torch.from_numpy(sysm.H.col_idx).pin_memory(),
            "h_vals": torch.from_numpy(sysm.H.vals).pin_memory()}
    dsys = nl.DeviceSystem(sysm, dev)
    stream = torch.cuda.current_stream(dev)

    # shard molecules over ranks (independent submatrices; one scalar all-reduce per bisection point)
    j0 = (n_mol * rank) // world
    j1 = (n_mol * (rank + 1)) // world
    opts.sub_begin, opts.sub_end = j0, j1

    def find_mu(plan):
        if world == 1:
            return plan.find_mu(n_occ, 0.0, 0.0, opts)
        from paper_2104_08245_gb300.sharded import sharded_find_mu
        return sharded_find_mu(plan, n_occ, opts)

    def step(dsys_, d_out):
        plan = nl.nolsm_build_submatrices(dsys_)
        r = find_mu(plan)
        plan.scatter(d_out)
        stats = plan.stats()
        plan.close()
        return r, stats

    info_plan = nl.nolsm_build_submatrices(dsys)
    info = info_plan.info()
    info_plan.close()
    D = torch.zeros(info.d_nvals, dtype=torch.float64, device=dev)

    for _ in range(args.warmup):
        r0, _ = step(dsys, D)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    stats_all = []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            r, st = step(dsys, D)
            stats_all.append(st)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms_step = ev0.elapsed_time(ev1) / args.steps
    if world > 1:
        t = torch.tensor([ms_step], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_step = float(t.item())
    mu_star = r.mu
    value = n_mol / (ms_step / 1e3)

    # e2e: inputs from pinned host memory, D back to host, same public calls
    d_host = torch.empty(info.d_nvals, dtype=torch.float64).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in host.values())
    d2h = d_host.numel() * 8

    class _Sys:  # DeviceSystem built from already-copied device tensors
        pass

    def e2e_step():
        e = _Sys()
        for k, t in host.items():
            setattr(e, k, t.to(dev, non_blocking=True))
        e.n_mol, e.n_occ = n_mol, n_occ
        e.struct = lambda: nl.DeviceSystem.struct(e)
        plan = nl.nolsm_build_submatrices(e)
        r_ = find_mu(plan)
        plan.scatter(D)
        plan.close()
        d_host.copy_(D, non_blocking=True)
        return r_

    e2e_step()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = ev0.elapsed_time(ev1) / args.steps

    if rank != 0:
        return 0

    st = stats_all[-1]
    launches = int(np.mean([s["launches"] for s in stats_all]))
    ms_sign = statistics.mean(s["ms_sign"] for s in stats_all)
    ms_factor = statistics.mean(s["ms_factor"] for s in stats_all)
    fl_fp32 = statistics.mean(s["flops_fp32"] for s in stats_all)
    fl_tensor = statistics.mean(s["flops_tensor"] for s in stats_all)
    fl_paper = statistics.mean(s["flops_paper"] for s in stats_all)
    fl_padded = statistics.mean(s["flops_tensor_padded"] for s in stats_all)
    evals = st["solves"]
    fp64_path = args.precision == "fp64"
    achieved = fl_tensor / (ms_sign / 1e3) / 1e12 if ms_sign > 0 else 0.0
    peak = peaks["bf16_sustained"]
    # launches of the factorisation kernel per step: one per preparation chunk
    chunks = max(1, int(st["factor_launches"]))
    roof_sign = {"bound": "tensor" if not fp64_path else "alu", "kernel": "k_ns_tc (sign iteration)",
                 "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak if peak else None,
                 "traffic": kernel_traffic("k_ns_tc", n_mol),
                 "peak_source": peaks["source"] + " bf16 sustained (kernel timed inside a long step)",
                 "algorithmic": "tensor flops the products need: (1 or 3 terms) x 2 n^3 per product, "
                                "2 products per Newton-Schulz step, unpadded n"}
    if not fp64_path and ms_factor > ms_sign:
        ach_f = fl_fp32 / (ms_factor / 1e3) / 1e12 if ms_factor > 0 else 0.0
        roofline = {"bound": "alu", "kernel": "k_prepare_mixed (FP32 factorisation and solves, double-FP32 refinement of Q)",
                    "achieved": ach_f, "peak": FP32_ALU_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": ach_f / FP32_ALU_PEAK_TFLOPS,
                    "traffic": kernel_traffic("k_prepare_mixed", n_mol / chunks), "launches_per_step": chunks,
                    "peak_source": "FP32 SIMT peak from unit counts (152 SMs x 128 lanes x 2 x 2.07 GHz)",
                    "algorithmic": "FP32 flops 2 (n^3/3 + n^3 + 3 n^2 b) per submatrix: Cholesky, the two "
                                   "triangular solves for A, the Q solve, its residual and correction"}
    else:
        roofline = roof_sign

    extra = {"mu": mu_star, "trace_DS": r.trace_DS, "n_occ": n_occ, "bisection_points": evals,
             "ms_phases": {k: statistics.mean(s[k] for s in stats_all)
                           for k in ("ms_plan", "ms_prepare", "ms_gather", "ms_factor", "ms_sign", "ms_reduce",
                                     "ms_scatter")},
             "sign_tflops_paper_convention": fl_paper / (ms_sign / 1e3) / 1e12 if ms_sign > 0 else 0.0,
             "sign_tflops_tensor_padded": fl_padded / (ms_sign / 1e3) / 1e12 if ms_sign > 0 else 0.0,
             "ns_steps_per_submatrix": st["ns_steps"] / max(1, st["sub_solves"]),
             "submatrix_n": [info.min_n, info.max_n]}

    # side measurements: one solve at mu* per precision (whole system; FP64 on a range), accuracy
    paths = {}
    if not args.no_extra:
        plan = nl.nolsm_build_submatrices(dsys)
        for prec in ["fp32", "bf16x3", "fp16", "bf16", "fp8e4m3", "fp64"]:
            o = nl.options(prec)
            if prec == "fp64":
                o.sub_begin, o.sub_end = 0, min(n_mol, 2 * 152 * 4)
            nl.nolsm_solve_batch(plan, mu_star, o, check=False)      # prepares the geometry caches
            plan.stats_reset()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rr = nl.nolsm_solve_batch(plan, mu_star, o, check=False)
            dt = time.perf_counter() - t0
            s2 = plan.stats()
            cnt = (o.sub_end or n_mol) - o.sub_begin
            paths[prec] = {"submatrices_per_s_one_mu": cnt / dt, "ms_sign": s2["ms_sign"], "status": rr.status,
                           "sign_tflops_paper": s2["flops_paper"] / (s2["ms_sign"] / 1e3) / 1e12,
                           "tensor_tflops": (s2["flops_tensor"] / (s2["ms_sign"] / 1e3) / 1e12
                                             if prec != "fp64" else None),
                           "_Dc": {}}
            paths[prec]["_D"] = plan.scatter().cpu().numpy()
        plan.close()

    # energy-weighted density matrix T_J(W) = T_J(D) T_J(H0) T_J(D) at mu* (once per geometry, after the
    # bisection; not part of the timed step): the kernel alone, timed by the library's CUDA events
    energy_weighted = {}
    if not args.no_extra and not fp64_path:
        plan = nl.nolsm_build_submatrices(dsys)
        nl.nolsm_solve_batch(plan, mu_star, opts, check=False)
        W = torch.zeros(info.d_nvals, dtype=torch.float64, device=dev)
        plan.energy_weighted(W)
        plan.stats_reset()
        reps = 5
        for _ in range(reps):
            _, tw = plan.energy_weighted(W)
        ms_ew = plan.stats()["ms_energy_weighted"] / reps
        sub_n = plan.maps()["sub_n"].cpu().numpy().astype(np.float64)[j0:j1]
        nbf = sysm.nbf.astype(np.float64)[j0:j1]
        bytes_ew = float(np.sum(sub_n * sub_n * 4.0 + 3.0 * sub_n * nbf * 8.0))
        ach_ew = bytes_ew / (ms_ew / 1e3) / 1e9 if ms_ew > 0 else 0.0
        energy_weighted = {
            "ms_kernel": ms_ew, "trace_WS": tw,
            "roofline": {"bound": "hbm", "kernel": "k_energy_weighted (W_c = A_J D_c)", "achieved": ach_ew,
                         "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": ach_ew / peaks["hbm_gbs"] if peaks["hbm_gbs"] else None,
                         "traffic": kernel_traffic("k_energy_weighted", j1 - j0),
                         "peak_source": peaks["source"] + " HBM copy bandwidth",
                         "algorithmic": "FP32 A_J read once (n^2 x 4 B), D_c and the centre columns of "
                                        "T_J(S) read and W_c written (3 n b x 8 B) per submatrix"}}
        plan.close()

    # submatrix combination heuristic (host planning step, Eq. combination_criterion) on an atom-resolved
    # pattern of the kind the paper applies it to (its water benchmark runs without it)
    combination = {}
    if not args.no_extra:
        sp = synth.make_site_pattern(synth.spec_ions_in_water())
        t0 = time.perf_counter()
        cr = nl.nolsm_combine_submatrices(sp.nbf, sp.nb_ptr, sp.nb_idx)
        dt_c = time.perf_counter() - t0
        combination = {"workload": "atom-resolved water lattice 16x16x16 with 2 % ions (O 4, H 2, ion 4 functions; "
                                   "6 / 10 Angstrom interaction radii)",
                       "sites": sp.n_sites, "groups": cr.n_groups, "sweeps": cr.sweeps,
                       "sum_n3_reduction": cr.sum_n3_before / cr.sum_n3_after,
                       "sum_n2_reduction": cr.sum_n2_before / cr.sum_n2_after,
                       "host_s": dt_c, "host_threads": os.cpu_count()}

    bounds = {}
    if not args.no_extra and not fp64_path:
        bounds = bound_sources_leg(nl, synth, spec_name, dsys, mu_star, args.precision, dev)

    # oracle: accuracy on a sample at mu* and the CPU baseline
    workers = max(1, os.cpu_count() or 1)
    rng = np.random.default_rng(7)
    sample = sorted(int(j) for j in rng.choice(n_mol, size=min(n_mol, args.sample), replace=False))
    ref, cpu_subs_per_s = {}, None
    if not args.no_oracle:
        pool = oracle_pool(spec_name, {}, workers)
        pool.map(_oracle_gersh, [[0]] * workers)   # warm the workers (system generation) before timing
        ref, dt_cpu = run_oracle(pool, sample, mu_star, workers)
        pool.close()
        cpu_subs_per_s = len(sample) / dt_cpu / max(1, evals)

    if paths and ref:
        from oracle import nolsm_oracle as orc
        po = orc.build_plan(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.H.row_ptr, sysm.H.col_idx)
        off = orc.d_block_offsets(po)
        acc_sample = sample[:64]
        for prec, pth in paths.items():
            Dn = pth["_D"]
            lim = (0, 2 * 152 * 4) if prec == "fp64" else (0, n_mol)
            err, rel_tH = 0.0, 0.0
            subs = [J for J in acc_sample if lim[0] <= J < lim[1]] or [J for J in range(lim[1]) if J in ref][:8]
            for J in subs:
                if J not in ref:
                    continue
                cols, tS_ref, tH_ref = ref[J]
                for p in range(po.nb_ptr[J], po.nb_ptr[J + 1]):
                    I = int(po.nb_idx[p])
                    q = po.nb_ptr[I] + int(np.nonzero(po.nb_idx[po.nb_ptr[I]:po.nb_ptr[I + 1]] == J)[0][0])
                    got = Dn[off[q]:off[q + 1]].reshape(6, 6)
                    err = max(err, float(np.max(np.abs(got - cols[po.nb_off[p]:po.nb_off[p] + 6, :]))))
            pth["max_abs_dD_sampled"] = err
            pth["sampled_submatrices"] = len(subs)
    if paths:
        fp64_rate = paths["fp64"]["submatrices_per_s_one_mu"]
        for prec, pth in paths.items():
            pth["speedup_vs_fp64_path"] = pth["submatrices_per_s_one_mu"] / fp64_rate

    for pth in paths.values():
        pth.pop("_D", None)
        pth.pop("_Dc", None)
    line = {
        "metric": METRIC,
        "value": value, "unit": "submatrices/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "fp16x3", "bf16x3": "bf16x3", "bf16": "bf16", "fp16": "fp16"}.get(args.precision,
                                                                                           args.precision),
        "data": "synthetic",
        "config": {"workload": desc if world == 1 else f"{desc}; lattice {world}x longer along x, one slab per GPU",
                   "precision": args.precision, "molecules": n_mol, "molecules_per_gpu": n_mol // world,
                   "l2": "inputs larger than L2 (block-CSR S and H, %.0f MB each)" % (sysm.S.vals.nbytes / 1e6),
                   "bracket": "Gershgorin interval of all submatrices"},
        "e2e": {"value": n_mol / (ms_e2e / 1e3), "unit": "submatrices/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches * args.steps,
        "roofline": roofline,
        "roofline_sign": roof_sign,
        "cpu_baseline": {"value": cpu_subs_per_s, "unit": "submatrices/s", "cores": workers, "kind": "oracle",
                         "sample": f"{len(sample)} submatrices solved once at the final mu, divided by the "
                                   f"{evals} bisection points of a step"},
        "clocks": clk.summary(),
        "extra": extra,
        "paths_one_mu": paths,
        "bound_sources": bounds,
        "energy_weighted": energy_weighted,
        "combination": combination,
    }
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
