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
    "streamed_4096": ("spec_streamed_4096",
                      "water-like lattice, 4096 molecules (16x16x16), 6 functions each, 6 A cutoff (profiling size of "
                      "the 262144-molecule workload)"),
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
# The main process builds the oracle's plan and writes it with the block-CSR system to a temporary
# directory; spawned workers map those files read-only (one copy in the page cache), gather their
# submatrices (Sec. "The Submatrix Method", step (i)) and solve them one by one with the FP64 oracle.

_ORC = {}
_FIELDS = ("row_ptr", "col_idx", "blk_off", "vals")
_PLAN_FIELDS = ("nb_ptr", "nb_idx", "nb_off", "sub_n", "sub_c0", "nbf")


def _oracle_init(path):
    import numpy as np
    from oracle import nolsm_oracle as orc
    ld = lambda k: np.load(os.path.join(path, k + ".npy"), mmap_mode="r")
    _ORC["S"] = tuple(ld("S_" + k) for k in _FIELDS)
    _ORC["H"] = tuple(ld("H_" + k) for k in _FIELDS)
    _ORC["plan"] = orc.OraclePlan(*(np.asarray(ld("P_" + k)) for k in _PLAN_FIELDS))


def _oracle_gather(J):
    from oracle import nolsm_oracle as orc
    p = _ORC["plan"]
    return orc.gather(p, J, *_ORC["S"]), orc.gather(p, J, *_ORC["H"])


def _oracle_sub(item):
    from oracle import nolsm_oracle as orc
    J, mu = item
    S_sub, H_sub = _oracle_gather(J)
    p = _ORC["plan"]
    r = orc.submatrix_density(S_sub, H_sub, mu, int(p.sub_c0[J]), int(p.nbf[J]))
    return J, (r.D_cols, r.t_S, r.t_H)


def _oracle_gersh(J):
    """Gershgorin interval of A = T_J(S)^-1 T_J(H0) (reference arm's bracket)."""
    import numpy as np
    from oracle import nolsm_oracle as orc
    S_sub, H_sub = _oracle_gather(J)
    A = orc.overlap_inverse(S_sub) @ H_sub
    d = np.diag(A)
    R = np.sum(np.abs(A), axis=1) - np.abs(d)
    return float(np.min(d - R)), float(np.max(d + R))


class OracleSample:
    """The oracle's plan of a system and a pool of spawned workers that solve sampled submatrices."""

    def __init__(self, sysm, workers):
        import multiprocessing as mp
        import tempfile

        import numpy as np
        from oracle import nolsm_oracle as orc
        os.environ.setdefault("OMP_NUM_THREADS", "1")
        os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
        self.plan = orc.build_plan(sysm.nbf, sysm.S.row_ptr, sysm.S.col_idx, sysm.H.row_ptr, sysm.H.col_idx)
        self.dir = tempfile.mkdtemp(prefix="nolsm_oracle_")
        for name, m in (("S", sysm.S), ("H", sysm.H)):
            for k in _FIELDS:
                np.save(os.path.join(self.dir, f"{name}_{k}.npy"), getattr(m, k))
        for k in _PLAN_FIELDS:
            np.save(os.path.join(self.dir, f"P_{k}.npy"), getattr(self.plan, k))
        self.workers = workers
        self.pool = mp.get_context("spawn").Pool(workers, initializer=_oracle_init, initargs=(self.dir,))
        self.pool.map(_oracle_gersh, [0] * workers)   # start every worker before anything is timed

    def solve(self, subs, mu):
        """({J: (D_cols, t_S, t_H)}, seconds) for the listed submatrices at mu, gathers included."""
        t0 = time.perf_counter()
        out = dict(self.pool.map(_oracle_sub, [(J, mu) for J in subs],
                                 chunksize=max(1, len(subs) // (4 * self.workers))))
        return out, time.perf_counter() - t0

    def bracket(self, subs):
        b = self.pool.map(_oracle_gersh, list(subs))
        return min(x[0] for x in b), max(x[1] for x in b)

    def close(self):
        import shutil
        self.pool.close()
        self.pool.join()
        shutil.rmtree(self.dir, ignore_errors=True)


# ------------------------------------------------------------------------------------ reference arm

def reference_arm(args, spec_name, desc):
    import numpy as np
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import synth
    from oracle import nolsm_oracle as orc
    sysm = synth.make_system(getattr(synth, spec_name)())
    n_mol = sysm.n_mol
    workers = max(1, os.cpu_count() or 1)
    ora = OracleSample(sysm, workers)
    rng = np.random.default_rng(7)
    sample = sorted(int(j) for j in rng.choice(n_mol, size=min(n_mol, args.ref_sample), replace=False))
    lo, hi = ora.bracket(sample)
    n_occ = float(np.sum(sysm.occ[sample]))   # the sample's own electron count

    def step():
        evals = []

        def count(mu):
            res, _ = ora.solve(sample, mu)
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
    ora.close()
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

def d_elements(po, subs):
    """Element indices into D (merged pattern, the oracle's block offsets) of every block (I, J), I in N(J),
    of the listed submatrices, with the matching (row, column) of J's centre columns."""
    import numpy as np
    from oracle import nolsm_oracle as orc
    off = orc.d_block_offsets(po)
    idx, where = [], {}
    pos = 0
    for J in subs:
        bJ = int(po.nbf[J])
        parts = []
        for p in range(po.nb_ptr[J], po.nb_ptr[J + 1]):
            I = int(po.nb_idx[p])
            bI = int(po.nbf[I])
            q = po.nb_ptr[I] + int(np.nonzero(po.nb_idx[po.nb_ptr[I]:po.nb_ptr[I + 1]] == J)[0][0])
            parts.append((int(po.nb_off[p]), bI, int(off[q])))
            idx.append(np.arange(off[q], off[q] + bI * bJ, dtype=np.int64))
        n = sum(bI for _, bI, _ in parts)
        where[J] = (pos, parts, bJ)
        pos += n * bJ
    return np.concatenate(idx), where


def sampled_errors(D_dev, po, subs, ref):
    """{J: max|dD|} over the blocks (I, J), I in N(J), of the listed submatrices: the device D (merged
    pattern) against the oracle's centre columns ref[J][0]."""
    import numpy as np
    import torch
    idx, where = d_elements(po, subs)
    got = D_dev.index_select(0, torch.from_numpy(idx).to(D_dev.device)).cpu().numpy()
    out = {}
    for J in subs:
        pos, parts, bJ = where[J]
        cols = ref[J][0]
        err = 0.0
        for r0, bI, _ in parts:
            blk = got[pos:pos + bI * bJ].reshape(bI, bJ)
            pos += bI * bJ
            err = max(err, float(np.max(np.abs(blk - cols[r0:r0 + bI, :]))))
        out[J] = err
    return out


def learned_bounds_leg(nl, synth, dsys, plan_sub_range, mu_star, precision, dev, ora_factory):
    """a4/a10, the learned spectral-bound experiment: the network is trained on samples the method produces
    on 100,000 submatrices of this system (power-iteration interval and step counts, three chemical
    potentials around mu*), then Gershgorin, power and learned bounds are compared on a fresh system of
    65,536 molecules with 6 or 23 functions (50/50) at mu*: Newton-Schulz steps, sign time, reruns, and the
    error of D against the FP64 oracle on sampled submatrices."""
    import numpy as np
    import torch
    o = nl.options(precision)
    n_train = min(100000, plan_sub_range)
    plan = nl.nolsm_build_submatrices(dsys)
    t0 = time.perf_counter()
    xs, ts = [], []
    thirds = [(k * n_train // 3, (k + 1) * n_train // 3) for k in range(3)]
    for dmu, (a, b) in zip((-0.05, 0.0, 0.05), thirds):
        ob = nl.options(precision, sub_begin=a, sub_end=b)
        x, t = nl.nolsm_training_data(plan, mu_star + dmu, ob)
        xs.append(x[a:b])
        ts.append(t[a:b])
    x, t = torch.cat(xs), torch.cat(ts)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    plan.close()
    mlp = nl.Mlp(seed=11)
    t0 = time.perf_counter()
    losses = mlp.train(x, t, epochs=30, batch=1024, lr=2e-3)
    t_train = time.perf_counter() - t0
    fresh = synth.make_system(synth.spec_mixed())
    p2 = nl.nolsm_build_submatrices(nl.DeviceSystem(fresh, dev))
    nl.nolsm_plan_set_mlp(p2, mlp)
    out = {"training_submatrices": int(x.shape[0]), "trained_on": "the benchmark system, submatrices 0..%d, "
           "power-iteration targets at mu* - 0.05, mu*, mu* + 0.05 (a third each)" % n_train,
           "epochs": 30, "batch": 1024, "loss_first_last": [losses[0], losses[-1]], "s_training_data": t_data,
           "s_training": t_train,
           "evaluated_on": "fresh water-like lattice, 65536 molecules (64x32x32), 6 or 23 functions (50/50), "
                           "seed %d, at mu*" % synth.spec_mixed().seed}
    ora = ora_factory(fresh)
    rng = np.random.default_rng(5)
    subs = sorted(int(j) for j in rng.choice(fresh.n_mol, size=48, replace=False))
    ref, _ = ora.solve(subs, mu_star)
    ora.close()
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
        errs = sampled_errors(D, ora.plan, subs, ref)
        out[name] = {"mean_ns_steps": float(r.iters.float().mean()), "ms_sign": s2["ms_sign"],
                     "ms_solve_call": dt * 1e3, "submatrices_per_s_one_mu": fresh.n_mol / dt,
                     "reruns": int(s2["reruns"]), "status": int(r.status),
                     "not_converged": int((r.sub_status != 0).sum()),
                     "max_abs_dD_vs_oracle_sampled": max(errs.values())}
    # what each interval costs to obtain for the whole system: Gershgorin comes with the preparation; the
    # power iteration is one kernel per geometry; the predictor is the features kernel and the network's
    # forward pass per chemical potential (each timed alone with CUDA events, after one untimed call)
    ob = nl.options(precision)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    costs = {}
    for rep in range(2):
        torch.cuda.synchronize()
        e0.record()
        mlp.forward(nl.nolsm_features(p2, mu_star, ob))
        e1.record()
        torch.cuda.synchronize()
    costs["mlp"] = e0.elapsed_time(e1)
    p2.close()
    # the power intervals are kept per geometry: their cost is that of their first computation, on a fresh
    # plan of the same system whose preparation is done
    p3 = nl.nolsm_build_submatrices(nl.DeviceSystem(fresh, dev))
    nl.nolsm_solve_batch(p3, mu_star, ob, check=False)
    torch.cuda.synchronize()
    e0.record()
    nl.nolsm_power_bounds(p3, ob)
    e1.record()
    torch.cuda.synchronize()
    costs["power"] = e0.elapsed_time(e1)
    p3.close()
    out["gershgorin"]["ms_bounds"] = 0.0
    for name in ("power", "mlp"):
        out[name]["ms_bounds"] = costs[name]
    for name in ("gershgorin", "power", "mlp"):
        out[name]["ms_bounds_plus_sign"] = out[name]["ms_bounds"] + out[name]["ms_sign"]
    out["steps_saved_vs_power"] = out["power"]["mean_ns_steps"] - out["mlp"]["mean_ns_steps"]
    out["steps_saved_vs_gershgorin"] = out["gershgorin"]["mean_ns_steps"] - out["mlp"]["mean_ns_steps"]
    return out


# ------------------------------------------------------------------------------------ our arm

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16x3")
    ap.add_argument("--workload", default="streamed_bf16", choices=list(WORKLOADS))
    ap.add_argument("--inverse", default="ns", choices=["cholesky", "ns"],
                    help="preparation of A_J: the tensor-core Newton-Schulz inverse square root (Eqs. inv1-inv3), "
                         "or the FP32 Cholesky factor")
    ap.add_argument("--batches", type=int, default=8, help="molecule batches the errors are reported for")
    ap.add_argument("--sample", type=int, default=640, help="oracle submatrices (errors and CPU baseline)")
    ap.add_argument("--ref-sample", type=int, default=96, help="submatrices per reference-arm step")
    ap.add_argument("--no-extra", action="store_true", help="skip the per-precision and learned-bound legs")
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

    # weak scaling: with N ranks the lattice is N times longer along x and rank r owns the r-th slab of
    # the one-GPU workload's size (molecule index runs fastest along z, slowest along x)
    spec = getattr(synth, spec_name)()
    if world > 1:
        import dataclasses
        spec = dataclasses.replace(spec, nx=spec.nx * world)
    sysm = synth.make_system(spec)
    n_mol = sysm.n_mol
    n_occ = sysm.n_occ
    workers = max(1, os.cpu_count() or 1)
    if world > 1:   # the side measurements and the oracle's accuracy check are single-GPU legs
        args.no_extra = args.no_oracle = True
    # the oracle's worker pool (spawned) and plan, before the first GPU call
    ora = OracleSample(sysm, workers) if (rank == 0 and not args.no_oracle) else None

    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    peaks = measured_peaks()
    inverse = nl._abi.INVERSE_NEWTON_SCHULZ if args.inverse == "ns" else nl._abi.INVERSE_CHOLESKY
    opts = nl.options(args.precision, inverse=inverse)

    # shard molecules over ranks (independent submatrices; one scalar all-reduce per bisection point); with
    # several ranks each holds only its halo: the block rows of its molecules' neighbourhoods
    j0 = (n_mol * rank) // world
    j1 = (n_mol * (rank + 1)) // world
    full = sysm
    if world > 1:
        from paper_2104_08245_gb300.sharded import extract_halo
        halo = extract_halo(sysm, j0, j1)
        sysm = halo.system
        opts.sub_begin, opts.sub_end = halo.l0, halo.l1
    else:
        opts.sub_begin, opts.sub_end = j0, j1

    # host copies (pinned) for the e2e leg; device copies for the resident leg
    host = {"nbf": torch.from_numpy(sysm.nbf).pin_memory(),
            "s_row_ptr": torch.from_numpy(sysm.S.row_ptr).pin_memory(),
            "s_col_idx": torch.from_numpy(sysm.S.col_idx).pin_memory(),
            "s_vals": torch.from_numpy(sysm.S.vals).pin_memory(),
            "h_row_ptr": torch.from_numpy(sysm.H.row_ptr).pin_memory(),
            "h_col_idx": torch.from_numpy(sysm.H.col_idx).pin_memory(),
            "h_vals": torch.from_numpy(sysm.H.vals).pin_memory()}
    dsys = nl.DeviceSystem(sysm, dev)
    n_local = dsys.n_mol      # molecules this rank holds (its halo with several ranks)
    stream = torch.cuda.current_stream(dev)


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
    D_e2e = torch.zeros_like(D)

    class _Sys:  # DeviceSystem built from already-copied device tensors
        pass

    def e2e_step():
        e = _Sys()
        for k, t in host.items():
            setattr(e, k, t.to(dev, non_blocking=True))
        e.n_mol, e.n_occ = n_local, n_occ
        e.struct = lambda: nl.DeviceSystem.struct(e)
        plan = nl.nolsm_build_submatrices(e)
        r_ = find_mu(plan)
        plan.scatter(D_e2e)
        plan.close()
        d_host.copy_(D_e2e, non_blocking=True)
        return r_

    e2e_step()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = ev0.elapsed_time(ev1) / args.steps

    # the same end to end with the elements generated on the device from the geometry (Sec. "Minimization of
    # Communication"): per step only the block patterns, positions and on-site energies go to the device
    mdl = nl.ElementModel(sysm, dev)
    host_g = {k: host[k] for k in ("nbf", "s_row_ptr", "s_col_idx", "h_row_ptr", "h_col_idx")}
    host_g["pos"] = mdl.pos.cpu().pin_memory()
    host_g["onsite"] = mdl.onsite.cpu().pin_memory()
    h2d_g = sum(t.numel() * t.element_size() for t in host_g.values())

    def e2e_gen_step():
        e = _Sys()
        dv = {k: t.to(dev, non_blocking=True) for k, t in host_g.items()}
        for k in ("nbf", "s_row_ptr", "s_col_idx", "h_row_ptr", "h_col_idx"):
            setattr(e, k, dv[k])
        e.s_vals = e.h_vals = None
        e.n_mol, e.n_occ = n_local, n_occ
        e.struct = lambda: nl.DeviceSystem.struct(e)
        m = nl.ElementModel.__new__(nl.ElementModel)
        m.pos, m.onsite, m.dirs, m.cell, m.params = dv["pos"], dv["onsite"], mdl.dirs, mdl.cell, mdl.params
        plan = nl.nolsm_build_submatrices(e)
        nl.nolsm_plan_set_elements(plan, m)
        r_ = find_mu(plan)
        plan.scatter(D_e2e)
        plan.close()
        d_host.copy_(D_e2e, non_blocking=True)
        return r_

    e2e_gen_step()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        rg = e2e_gen_step()
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_e2e_gen = ev0.elapsed_time(ev1) / args.steps
    gen_mu_diff = abs(rg.mu - r0.mu)

    if rank != 0:
        return 0

    st = stats_all[-1]
    launches = int(np.mean([s["launches"] for s in stats_all]))
    mean = lambda k: statistics.mean(s[k] for s in stats_all)
    ms_sign, ms_factor = mean("ms_sign"), mean("ms_factor")
    fl_paper, fl_tensor, fl_padded, fl_fp32 = (mean("flops_paper"), mean("flops_tensor"),
                                               mean("flops_tensor_padded"), mean("flops_fp32"))
    evals = st["solves"]
    fp64_path = args.precision == "fp64"
    tf = lambda fl, ms: fl / (ms / 1e3) / 1e12 if ms > 0 else 0.0
    peak = peaks["bf16_sustained"]
    chunks = max(1, int(st["factor_launches"]))
    roof_sign = {"bound": "tensor" if not fp64_path else "alu", "kernel": "k_ns_tc (sign iteration)",
                 "achieved": tf(fl_paper, ms_sign), "peak": peak, "unit": "TFLOP/s",
                 "frac": tf(fl_paper, ms_sign) / peak if peak else None,
                 "traffic": kernel_traffic("k_ns_tc", j1 - j0),
                 "peak_source": peaks["source"] + " bf16 sustained (kernel timed inside a long step)",
                 "algorithmic": "4 k n^3 flops per submatrix (2 n^3 per product, 2 products per Newton-Schulz "
                                "step, k steps, unpadded n; Sec. 'FLOPs in the NOLSM method'), k counted per "
                                "submatrix, summed over the step's bisection points",
                 "achieved_tensor_issued": tf(fl_tensor, ms_sign),
                 "achieved_tensor_issued_note": "the products the arithmetic needs: x3 for three-term split "
                                                "steps, unpadded n",
                 "achieved_padded": tf(fl_padded, ms_sign),
                 "achieved_padded_note": "split products on the padded tiles the kernel executes"}
    roof_prep = None
    ms_prep_kernel = 0.0
    if not fp64_path and args.inverse == "ns":
        ms_prep_kernel = mean("ms_prep_tensor")
        fl_prep = mean("flops_prep_tensor")
        roof_prep = {"bound": "tensor", "kernel": "k_ns_tc<1> (inverse square root of T_J(S), Eqs. inv1-inv3, "
                                                  "and A_J)",
                     "achieved": tf(fl_prep, ms_prep_kernel), "peak": peak, "unit": "TFLOP/s",
                     "frac": tf(fl_prep, ms_prep_kernel) / peak if peak else None,
                     "traffic": kernel_traffic("k_ns_tc_inv", (j1 - j0) / chunks), "launches_per_step": chunks,
                     "peak_source": peaks["source"] + " bf16 sustained (FP16 operands run at the BF16 rate)",
                     "algorithmic": "2 n^3 flops per product on the unpadded n, 3 k - 1 products per submatrix "
                                    "(k coupled steps: step 0 one product since Z_0 = I, the middle ones "
                                    "three, the last two as it needs no Y update; then T_J(S)^-1 = Z^2 / c "
                                    "and A_J = T_J(S)^-1 T_J(H0))",
                     "achieved_tensor_issued": tf(mean("flops_prep_tensor_issued"), ms_prep_kernel),
                     "achieved_tensor_issued_note": "x3 for the three-term FP16 split"}
    elif not fp64_path:
        ms_prep_kernel = ms_factor
        ach_f = tf(fl_fp32, ms_factor)
        roof_prep = {"bound": "alu", "kernel": "k_prepare_mixed (FP32 factorisation and solves, double-FP32 "
                                               "refinement of Q)",
                     "achieved": ach_f, "peak": FP32_ALU_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": ach_f / FP32_ALU_PEAK_TFLOPS,
                     "traffic": kernel_traffic("k_prepare_mixed", (j1 - j0) / chunks), "launches_per_step": chunks,
                     "peak_source": "FP32 SIMT peak from unit counts (152 SMs x 128 lanes x 2 x 2.07 GHz)",
                     "algorithmic": "FP32 flops 2 (n^3/3 + n^3 + 3 n^2 b) per submatrix: Cholesky, the two "
                                    "triangular solves for A, the Q solve, its residual and correction"}
    # the headline roofline is the step's dominant kernel
    roofline = roof_prep if (roof_prep is not None and ms_prep_kernel > ms_sign) else roof_sign

    extra = {"mu": mu_star, "trace_DS": r.trace_DS, "n_occ": n_occ, "bisection_points": evals,
             "ms_phases": {k: mean(k) for k in ("ms_plan", "ms_prepare", "ms_gather", "ms_factor", "ms_prep_tensor",
                                                 "ms_sign", "ms_reduce", "ms_scatter")},
             "ns_steps_per_submatrix": st["ns_steps"] / max(1, st["sub_solves"]),
             "submatrix_n": [info.min_n, info.max_n]}

    # accuracy of the headline result (the D of the last timed step) against the FP64 oracle, batch by
    # batch (contiguous molecule ranges), and the CPU baseline on the same sample
    nb = max(1, args.batches)
    rng = np.random.default_rng(7)
    per = max(1, min(n_mol // nb, args.sample // nb))
    batches = [(b * n_mol // nb, (b + 1) * n_mol // nb) for b in range(nb)]
    sample = sorted({int(j) for a, b in batches for j in rng.choice(np.arange(a, b), size=per, replace=False)})
    ref, cpu_subs_per_s, errors = {}, None, None
    if ora is not None:
        ref, dt_cpu = ora.solve(sample, mu_star)
        cpu_subs_per_s = len(sample) / dt_cpu / max(1, evals)
        # per-submatrix traces at mu* from the library (same mode), for the trace errors
        plan = nl.nolsm_build_submatrices(dsys)
        rr = nl.nolsm_solve_batch(plan, mu_star, opts, check=False)
        tS_gpu, tH_gpu = rr.sub_t_S.cpu().numpy(), rr.sub_t_H.cpu().numpy()
        plan.close()
        errs = sampled_errors(D, ora.plan, sample, ref)
        errors = []
        for b, (a, e) in enumerate(batches):
            js = [J for J in sample if a <= J < e]
            sS = sum(ref[J][1] for J in js)
            sH = sum(ref[J][2] for J in js)
            errors.append({"batch": b, "molecules": [a, e], "sampled": len(js),
                           "max_abs_dD": max(errs[J] for J in js),
                           "rel_err_tr_DH": abs(sum(tH_gpu[J] for J in js) - sH) / abs(sH),
                           "rel_err_tr_DS": abs(sum(tS_gpu[J] for J in js) - sS) / abs(sS),
                           "max_rel_err_t_H": max(abs(tH_gpu[J] - ref[J][2]) / abs(ref[J][2]) for J in js)})
        extra["errors_per_batch"] = errors
        extra["errors_worst"] = {k: max(x[k] for x in errors) for k in
                                 ("max_abs_dD", "rel_err_tr_DH", "rel_err_tr_DS", "max_rel_err_t_H")}

    # side measurements: one solve at mu* per precision (whole system; FP64 on a range), accuracy
    paths = {}
    if not args.no_extra:
        plan = nl.nolsm_build_submatrices(dsys)
        fp64_range = (0, min(n_mol, 2 * 152 * 4))
        for prec in ["fp32", "bf16x3", "fp16", "bf16", "fp8e4m3", "fp64"]:
            # the FP32 mode's 1e-6 target is the Cholesky preparation's; the other modes use the bench's
            o = nl.options(prec, inverse=nl._abi.INVERSE_CHOLESKY if prec == "fp32" else inverse)
            if prec == "fp64":
                o.sub_begin, o.sub_end = fp64_range
            nl.nolsm_solve_batch(plan, mu_star, o, check=False)      # prepares the geometry caches
            plan.stats_reset()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rr = nl.nolsm_solve_batch(plan, mu_star, o, check=False)
            dt = time.perf_counter() - t0
            s2 = plan.stats()
            cnt = (o.sub_end or n_mol) - o.sub_begin
            pth = {"submatrices_per_s_one_mu": cnt / dt, "ms_sign": s2["ms_sign"], "status": rr.status,
                   "inverse": "cholesky" if o.inverse == nl._abi.INVERSE_CHOLESKY else "ns",
                   "sign_tflops_paper": tf(s2["flops_paper"], s2["ms_sign"]),
                   "tensor_tflops_issued": tf(s2["flops_tensor"], s2["ms_sign"]) if prec != "fp64" else None}
            if ref:
                Dp = plan.scatter()
                subs = [J for J in sample if (prec != "fp64" or J < fp64_range[1])][:96]
                if subs:
                    pth["max_abs_dD_sampled"] = max(sampled_errors(Dp, ora.plan, subs, ref).values())
                    pth["sampled_submatrices"] = len(subs)
                del Dp
            paths[prec] = pth
        plan.close()
        fp64_rate = paths["fp64"]["submatrices_per_s_one_mu"]
        for pth in paths.values():
            pth["speedup_vs_fp64_path"] = pth["submatrices_per_s_one_mu"] / fp64_rate

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
        del W
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
        # the merged submatrices solved on the device: a step (plan, one solve at the per-site mu*, write-back)
        # with one submatrix per site against one per group
        ssys = synth.site_system(sp)
        dss = nl.DeviceSystem(ssys, dev)
        o_s = nl.options(args.precision, inverse=inverse)
        mp = nl.nolsm_build_submatrices(dss)
        mu_s = mp.find_mu(float(np.sum(ssys.occ)), 0.0, 0.0, o_s).mu
        Ds = torch.zeros(mp.info().d_nvals, dtype=torch.float64, device=dev)
        mp.close()

        def site_step(grouped):
            p_ = nl.nolsm_build_submatrices(dss)
            q_ = nl.nolsm_build_grouped(p_, cr.group_of) if grouped else p_
            r_ = nl.nolsm_solve_batch(q_, mu_s, o_s, check=False)
            q_.scatter(Ds)
            st_ = q_.stats()
            if grouped:
                q_.close()
            p_.close()
            return r_, st_

        timing = {}
        for grouped in (False, True):
            site_step(grouped)
            torch.cuda.synchronize()
            ev0.record(stream)
            for _ in range(3):
                r_s, st_s = site_step(grouped)
            ev1.record(stream)
            torch.cuda.synchronize()
            timing["grouped" if grouped else "per_site"] = {
                "ms_step": ev0.elapsed_time(ev1) / 3, "ms_prepare": st_s["ms_prepare"], "ms_sign": st_s["ms_sign"],
                "status": r_s.status, "trace_DS": r_s.trace_DS}
        combination["device_solve"] = {
            **timing, "mu": mu_s, "precision": args.precision,
            "step_time_ratio": timing["per_site"]["ms_step"] / timing["grouped"]["ms_step"],
            "note": "step = plan (plus the grouped plan's host construction), preparation and one solve at the "
                    "per-site plan's mu*, and the write-back into the per-site pattern of D"}

    bounds = {}
    if not args.no_extra and not fp64_path and ora is not None:
        bounds = learned_bounds_leg(nl, synth, dsys, j1 - j0, mu_star, args.precision, dev,
                                    lambda s_: OracleSample(s_, workers))
    if ora is not None:
        ora.close()

    line = {
        "metric": METRIC,
        "value": value, "unit": "submatrices/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "fp16x3", "bf16x3": "bf16x3", "bf16": "bf16", "fp16": "fp16"}.get(args.precision,
                                                                                           args.precision),
        "data": "synthetic",
        "config": {"workload": desc if world == 1 else f"{desc}; lattice {world}x longer along x, one slab per GPU",
                   "precision": args.precision, "inverse": args.inverse, "molecules": n_mol, "molecules_per_gpu": n_mol // world,
                   "l2": "inputs larger than L2 (block-CSR S and H, %.0f MB each)" % (sysm.S.vals.nbytes / 1e6),
                   "bracket": "Gershgorin interval of all submatrices",
                   "batches": f"{nb} contiguous molecule ranges, errors reported per range"},
        "e2e": {"value": n_mol / (ms_e2e / 1e3), "unit": "submatrices/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "e2e_generated": {"value": n_mol / (ms_e2e_gen / 1e3), "unit": "submatrices/s", "h2d_bytes_per_step": h2d_g,
                          "d2h_bytes_per_step": d2h, "mu_difference_to_stored_elements": gen_mu_diff,
                          "note": "elements of T_J(S), T_J(H0) generated on the device from positions and on-site "
                                  "energies; per step the block patterns, positions and on-site energies are "
                                  "copied instead of the block-CSR values"},
        "gpu_launches": launches * args.steps,
        "roofline": roofline,
        "roofline_sign": roof_sign,
        "roofline_prep": roof_prep,
        "cpu_baseline": {"value": cpu_subs_per_s, "unit": "submatrices/s", "cores": workers, "kind": "oracle",
                         "sample": f"{len(sample)} submatrices ({per} per batch) gathered and solved once at the "
                                   f"final mu, divided by the {evals} bisection points of a step"},
        "clocks": clk.summary(),
        "extra": extra,
        "paths_one_mu": paths,
        "learned_bounds": bounds,
        "tuned_shapes": {f"{k} bucket {b}": nl.nolsm_tc_shape(k, args.precision if k == "sign" else "fp16", b)
                         for k in ("sign", "inverse") for b in (0, 1)},
        "energy_weighted": energy_weighted,
        "combination": combination,
    }
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
