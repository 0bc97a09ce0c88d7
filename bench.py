"""Benchmark: factor + PCG seconds to relative residual 1e-8.

Workload: 7-point finite-volume diffusion on a 96^3 grid (884,736 unknowns) with
cell conductivity exp(g), g a seeded Gaussian random field (sigma 2, correlation
length 8 cells); compression tolerance 1e-2, 16-column Gaussian samples, PCG to
||r||/||b|| <= 1e-8.  One step = rsc_factor + rsc_solve_device (b resident on the
device); its time is the sum of the two calls' device times (CUDA events on the
library's stream).  The default form (BF16 Schur updates on tcgen05 tensor cores with
FP32 accumulation, FP32 factor storage, diagonal Cholesky and sampling, FP64 PCG) is
timed for K steps; the FP32 form and the plain FP64 form are timed once beside it.  L2
is flushed between steps (the factor storage is also larger than L2).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec bf16|fp32|fp64] [--side 96]
  python bench.py --impl reference ...   # the CPU oracle on a bounded sample

For N > 1 (torchrun) every rank solves its own replica (replicas only: the method
has no data-parallel exchange step at this size); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "factor+PCG seconds to rel. residual 1e-8"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="bf16")
    ap.add_argument("--side", type=int, default=None,
                    help="grid side: 96 (diffusion cells) or 40 (elasticity elements) by default")
    ap.add_argument("--tol", type=float, default=None, help="compression tolerance: 0.1 (poisson) or 0.01")
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--workload", default="diffusion",
                    choices=["diffusion", "elasticity", "poisson", "batch", "autograd"])
    ap.add_argument("--systems", type=int, default=256)
    ap.add_argument("--nrhs", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-others", action="store_true",
                    help="skip the compact runs of the other configurations (C1, C3, C4, C5)")
    a = ap.parse_args()
    if a.side is None:
        a.side = {"elasticity": 40, "poisson": 32, "autograd": 64}.get(a.workload, 96)
    if a.tol is None:
        a.tol = 0.1 if a.workload == "poisson" else 1e-2
    return a


def _elasticity_incl(ne):
    """The stiff inclusion of an ne^3-element block: the central (ne/4)^3 elements."""
    return (3 * ne // 8, 3 * ne // 8 + ne // 4)


def _workload_name(side, tol, workload="diffusion"):
    if workload == "poisson":
        return (f"poisson7_{side}^3 ({side ** 3:,} unknowns, Dirichlet), b ~ U[-1,1] seed 0, compression tol "
                f"{tol:g}, 16-col Gaussian samples, PCG rtol 1e-8")
    if workload == "elasticity":
        n = 3 * side * (side + 1) ** 2
        return (f"q1_elasticity_{side}^3 elements ({n:,} unknowns, 3 DOF per node kept together), x = 0 face "
                f"clamped, E = 1, nu = 0.3, stiff inclusion E = 1e3 on the central {side // 4}^3 elements, "
                f"body force; compression tol {tol:g}, 16-col Gaussian samples, PCG rtol 1e-8")
    return (f"fv_diffusion_grf_{side}^3 ({side ** 3:,} unknowns), conductivity exp(GRF sigma 2, corr len 8), "
            f"compression tol {tol:g}, 16-col Gaussian samples, PCG rtol 1e-8")


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- CPU oracle leg
_ORACLE_CODE = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
import workloads as W
from oracle import factor as F
c = {crop}
if {kind!r} == "elasticity":
    p = W.elasticity_q1(c, incl={incl})
elif {kind!r} == "poisson":
    p = W.poisson7(c)
else:
    g = W.grf(({side}, {side}, {side}), 2.0, 8.0, 0)
    p = W.fv_diffusion(np.exp(g[:c, :c, :c]), 0)
t0 = time.perf_counter()
an = F.analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, F.Options(dof_per_node=p.dof_per_node))
t1 = time.perf_counter()
f = F.factor(an, {tol})
t2 = time.perf_counter()
x, it, rr, ok = F.solve(an, f, p.b, {rtol}, 2000)
t3 = time.perf_counter()
print(json.dumps(dict(n=p.n, analyze=t1 - t0, factor=t2 - t1, solve=t3 - t2, iters=it, relres=rr, ok=bool(ok))))
"""


def run_oracle_sample(side, crop, tol, rtol, workload="diffusion", threads=1):
    """The oracle, as it stands, on a crop of the same conductivity field, or on a smaller
    elasticity block of the same shape (numpy with `threads` BLAS threads)."""
    t = str(threads)
    env = dict(os.environ, OMP_NUM_THREADS=t, OPENBLAS_NUM_THREADS=t, MKL_NUM_THREADS=t)
    code = _ORACLE_CODE.format(root=ROOT, side=side, crop=crop, tol=tol, rtol=rtol, kind=workload,
                               incl=_elasticity_incl(crop))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def cpu_baseline(side, tol, rtol, crop=32, workload="diffusion", n_full=None, threads=1):
    if workload == "elasticity":
        crop = 12
    elif workload == "poisson":
        crop = side          # the whole problem: seconds for the oracle
    r = run_oracle_sample(side, crop, tol, rtol, workload, threads)
    secs = r["factor"] + r["solve"]
    scale = (n_full or side ** 3) / r["n"]
    what = {"elasticity": f"a {crop}^3-element block of the same elasticity problem",
            "poisson": "the whole problem"}.get(workload, f"the {crop}^3 corner crop of the same conductivity field")
    return {"value": secs * scale, "unit": "s", "cores": threads, "kind": "oracle",
            "sample": (f"oracle factor+PCG on {what} "
                       f"({r['n']:,} unknowns, tol {tol:g}, {r['iters']} iterations, measured {secs:.2f} s, "
                       f"{threads} BLAS thread{'s' if threads > 1 else ''} of nproc = {os.cpu_count()}), "
                       f"scaled linearly by unknowns x{scale:.1f} (a lower bound: the method is superlinear)")}


def _oracle_code(code, threads=1, timeout=900):
    t = str(threads)
    env = dict(os.environ, OMP_NUM_THREADS=t, OPENBLAS_NUM_THREADS=t, MKL_NUM_THREADS=t)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=timeout)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


_ORACLE_BATCH = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import workloads as W
from oracle import factor as F
p = W.diffusion_lognormal({side}, 1.0, seed=0)
t0 = time.perf_counter()
an = F.analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, F.Options())
f = F.factor(an, {tol})
t1 = time.perf_counter()
its = [F.solve(an, f, W.rhs_uniform(p.n, seed=c), {rtol}, 2000)[1] for c in range({nrhs})]
t2 = time.perf_counter()
print(json.dumps(dict(n=p.n, factor=t1 - t0, solve=t2 - t1, iters=max(its))))
"""

_ORACLE_ADJOINT = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
import workloads as W
from oracle import factor as F
c = {crop}
theta = np.random.default_rng(0).standard_normal(({side}, {side}, {side}))[:c, :c, :c]
p = W.fv_diffusion(np.exp(theta), 2)
t0 = time.perf_counter()
an = F.analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, F.Options())
f = F.factor(an, {tol})
x, it, rr, ok = F.solve(an, f, p.b, {rtol}, 2000)
t1 = time.perf_counter()
lam, it2, rr2, ok2 = F.solve(an, f, x, {rtol}, 2000)
t2 = time.perf_counter()
print(json.dumps(dict(n=p.n, forward=t1 - t0, backward=t2 - t1, iters=it)))
"""


def _sub_bench(args, timeout=900):
    """One compact run of bench.py for another configuration; its JSON line, or the failure."""
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--no-others"] + args
    try:
        out = subprocess.run(cmd, capture_output=True, text=True, timeout=timeout)
        for ln in reversed(out.stdout.strip().splitlines()):
            if ln.startswith("{"):
                return json.loads(ln)
        return {"failed": (out.stderr or out.stdout)[-400:]}
    except Exception as e:
        return {"failed": str(e)[:400]}


def _compact(d, keys):
    if not d or "failed" in d:
        return d
    return {k: d.get(k) for k in keys if k in d}


def other_configs(a):
    """C1 (Poisson 32^3, all FP64), C3 (elasticity 40^3, TF32 Schur updates), C4 (256 systems x 8
    right-hand sides, BF16), C5 (differentiation 64^3, FP32 factor): value, iterations, the plain
    FP64 GPU path beside and the oracle baseline, 3 timed steps each after 3 warm-up steps (a
    handle's first factorizations still grow its workspaces)."""
    base = ["--steps", "3", "--warmup", "3"]
    keys = ["value", "factor_s", "solve_s", "iters", "relres", "factor_bytes", "restarts", "factor_tflops",
            "cpu_baseline", "plain_fp64", "fp32_form", "roofline", "dtype", "config", "form", "e2e", "gpu_launches"]
    out = {}
    c1 = _sub_bench(["--workload", "poisson", "--prec", "fp64"] + base)
    c1_32 = _sub_bench(["--workload", "poisson", "--prec", "fp32", "--no-cpu-baseline"] + base)
    out["C1_poisson32_fp64"] = _compact(c1, keys)
    if c1_32 and "failed" not in c1_32:
        out["C1_poisson32_fp64"]["fp32_form"] = _compact(c1_32, ["value", "factor_s", "solve_s", "iters"])
    out["C3_elasticity40_tf32"] = _compact(_sub_bench(["--workload", "elasticity", "--prec", "tf32"] + base), keys)
    bkeys = ["value", "factor_s", "solve_s", "iters_max", "iters_mean", "relres_max", "factor_bytes", "restarts",
             "config", "dtype", "cpu_baseline", "gpu_launches"]
    c4 = _compact(_sub_bench(["--workload", "batch"] + base), bkeys)
    c4_64 = _sub_bench(["--workload", "batch", "--prec", "fp64", "--no-cpu-baseline", "--steps", "1", "--warmup", "2"])
    if c4 and "failed" not in c4:
        c4["plain_fp64"] = _compact(c4_64, ["value", "factor_s", "solve_s", "iters_max", "factor_bytes"])
    out["C4_batch256x8_bf16"] = c4
    akeys = ["value", "forward_s", "backward_s", "last_iters", "factor_bytes", "restarts", "config", "dtype",
             "cpu_baseline", "gpu_launches"]
    c5 = _compact(_sub_bench(["--workload", "autograd", "--prec", "fp32"] + base), akeys)
    c5_64 = _sub_bench(["--workload", "autograd", "--prec", "fp64", "--no-cpu-baseline"] + base)
    if c5 and "failed" not in c5:
        c5["plain_fp64"] = _compact(c5_64, ["value", "forward_s", "backward_s", "last_iters"])
    out["C5_autograd64_fp32"] = c5
    return out


# ----------------------------------------------------------------------------- reference arm
FORMS = {"bf16": "BF16 Schur updates on tcgen05 (FP32 accumulation), FP32 factor, diagonal Cholesky and "
                 "sampling, FP64 PCG",
         "tf32": "TF32 Schur updates on tcgen05 (FP32 accumulation), FP32 factor, diagonal Cholesky and "
                 "sampling, FP64 PCG",
         "fp32": "FP32 factor, Schur updates, diagonal Cholesky and sampling; FP64 PCG",
         "fp64": "all FP64"}

# ncu dram__bytes_read.sum + dram__bytes_write.sum per launch at 96^3, by kernel class, for the
# code as it stands (profiles/); a class whose kernel changed after its capture has none
NCU_TRAFFIC = {}

# SIMT peaks measured on this machine's GB300 with an FMA loop; the HBM and
# BF16 tensor peaks come from MEASURED_PEAKS.json.  TF32 tensor: the BF16 peak times the nominal
# TF32 / BF16 ratio (1.1 / 2.25 PFLOP/s dense).
FP64_SIMT_TFLOPS = 1.00
FP32_SIMT_TFLOPS = 67.7


def _peaks():
    try:
        pk = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return {"hbm": pk.get("hbm_gbs", 6766.4), "bf16": pk.get("bf16_tflops", 1884.3), "src": "of measured"}
    except Exception:
        return {"hbm": 6800.0, "bf16": 1900.0, "src": "of fallback"}


# which compute roof bounds a kernel class: tensor-core classes against the tensor peak of their
# operand type, the rest (diagonal Cholesky tiles included) against SIMT of the storage type
TENSOR_CLASSES = {"push_tc", "tn_tc", "nn_tc"}


def roofline_entry(name, k, prec, source):
    """Roofline of one kernel class from its launches: achieved algorithmic bytes and flops per
    launch / average launch time; the bound is the roof the class's arithmetic intensity reaches
    first (ridge = compute peak / HBM peak)."""
    pk = _peaks()
    if not k or k.get("launches", 0) == 0 or k.get("ms", 0) <= 0:
        return None
    sec = k["ms"] * 1e-3
    gbs = k["bytes"] / sec / 1e9 if k.get("bytes") else 0.0
    tfs = k["flops"] / sec / 1e12 if k.get("flops") else 0.0
    if name in TENSOR_CLASSES:
        cpk = pk["bf16"] * (1.1 / 2.25 if prec == "tf32" else 1.0)
        cunit, csrc = f"{'TF32' if prec == 'tf32' else 'BF16'} tensor", pk["src"]
    elif prec == "fp64":
        cpk, cunit, csrc = FP64_SIMT_TFLOPS, "FP64 SIMT", "of builder-measured (DFMA loop)"
    else:
        cpk, cunit, csrc = FP32_SIMT_TFLOPS, "FP32 SIMT", "of builder-measured (FFMA loop)"
    ridge = cpk * 1e12 / (pk["hbm"] * 1e9)
    ai = (k["flops"] / k["bytes"]) if k.get("bytes") else float("inf")
    if k.get("bytes") and ai < ridge:
        ent = {"bound": "hbm", "achieved": gbs, "peak": pk["hbm"], "unit": "GB/s", "frac": gbs / pk["hbm"],
               "peak_src": pk["src"]}
    else:
        ent = {"bound": "tensor" if name in TENSOR_CLASSES else "alu", "achieved": tfs, "peak": cpk,
               "unit": "TFLOP/s", "frac": tfs / cpk, "peak_src": f"{cunit} {csrc}"}
    ent.update({"kernel": name, "launches": k["launches"], "avg_launch_us": k["ms"] / k["launches"] * 1e3,
                "achieved_gbs": gbs, "achieved_tflops": tfs, "intensity_flop_per_byte": None if ai == float("inf")
                else ai, "source": source})
    return ent


def max_over_ranks(t_local, dist, device):
    """Whole-job step time of N replicas: the slowest rank's time (every rank gets it)."""
    import torch
    if dist is None:
        return t_local
    tt = torch.tensor([t_local], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def replica_seed(rank):
    """Each replica factors and solves its own system: the conductivity field and b of rank r use seed r."""
    return rank


def reference_arm(a, rank, world):
    if rank != 0:
        return
    elastic = a.workload == "elasticity"
    n_full = 3 * a.side * (a.side + 1) ** 2 if elastic else a.side ** 3
    vals, secs = [], []
    rec = None
    for i in range(a.warmup + a.steps):
        if elastic:
            crop = 10 if i < a.warmup else 12
        elif a.workload == "poisson":
            crop = a.side
        else:
            crop = 24 if i < a.warmup else 32
        r = run_oracle_sample(a.side, crop, a.tol, a.rtol, a.workload)
        if i >= a.warmup:
            vals.append((r["factor"] + r["solve"]) * n_full / r["n"])
            secs.append(r["factor"] + r["solve"])
            rec = r
    v = sum(vals) / len(vals)
    t_sample = sum(secs) / len(secs)
    what = {"elasticity": "a 12^3-element block of the same elasticity problem",
            "poisson": "the whole problem"}.get(a.workload, "the 32^3 corner crop of the same conductivity field")
    sample = (f"oracle (numpy FP64, 1 thread) factor+PCG on {what} "
              f"({rec['n']:,} unknowns, {rec['iters']} iterations), scaled linearly by unknowns to the full problem")
    # value: the sample's time scaled to the whole workload (the metric); ms_per_step: the time a
    # timed step took (one bounded sample)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": t_sample * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": _workload_name(a.side, a.tol, a.workload)}, "form": "cpu oracle (FP64)",
            "value_basis": f"sample time x {n_full / rec['n']:.1f} (unknowns of the workload / of the sample)",
            "cpu_baseline": {"value": v, "unit": "s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- batch workload
def batch_workload(a):
    """Many independent systems: 7-point FV diffusion with iid log-normal conductivity
    (sigma 1), cube sides ~ U{12..40} (numpy Philox, seed 0), each system's right-hand
    sides ~ U[-1,1] (seed = system id * 100 + rhs), stacked block-diagonally and solved
    as one forest: factor + batched PCG to 1e-8 for every (system, right-hand side)."""
    import numpy as np
    import scipy.sparse as sp
    import torch

    import paper_1507_05593_gb300 as R
    import workloads as W

    torch.cuda.set_device(0)
    sides = np.random.Generator(np.random.Philox(0)).integers(12, 41, a.systems)
    ps = [W.diffusion_lognormal(int(sd), 1.0, seed=i) for i, sd in enumerate(sides)]
    A = sp.block_diag([p.scipy() for p in ps]).tocsr()
    A.sort_indices()
    coords, off = [], 0
    for p in ps:
        c = p.coords.copy()
        c[:, 0] += off
        off = int(c[:, 0].max()) + 4      # systems side by side along x, 3 empty planes apart
        coords.append(c)
    coords = np.vstack(coords)
    n = A.shape[0]
    B = np.zeros((a.nrhs, n))
    o = 0
    for i, p in enumerate(ps):
        for c in range(a.nrhs):
            B[c, o:o + p.n] = W.rhs_uniform(p.n, seed=100 * i + c)
        o += p.n
    dB = torch.tensor(B, device="cuda")
    dX = torch.empty_like(dB)
    t0 = time.perf_counter()
    h = R.rsc_analyze(n, A.indptr, A.indices, A.data, coords, R.rsc_options_default(precision=a.prec))
    t_an = time.perf_counter() - t0
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    res = []
    for i in range(a.warmup + a.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        R.rsc_factor(h, a.tol)
        its, rr = R.rsc_solve_batch_device(h, dB, dX, a.rtol, 2000)
        st = R.rsc_get_stats(h)
        if i >= a.warmup:
            res.append((st["factor_seconds"], st["solve_seconds"], its, rr, st))
    fs = sum(r[0] for r in res) / len(res)
    ss = sum(r[1] for r in res) / len(res)
    its, rr, st = res[-1][2], res[-1][3], res[-1][4]
    cpu = None
    if not a.no_cpu_baseline:
        try:   # the oracle on system 0 (all its right-hand sides), scaled by unknowns
            r = _oracle_code(_ORACLE_BATCH.format(root=ROOT, side=int(sides[0]), tol=a.tol, rtol=a.rtol,
                                                  nrhs=a.nrhs))
            secs = r["factor"] + r["solve"]
            cpu = {"value": secs * n / r["n"], "unit": "s", "cores": 1, "kind": "oracle",
                   "sample": (f"oracle factor + {a.nrhs} PCG solves of system 0 ({r['n']:,} unknowns, side "
                              f"{int(sides[0])}, measured {secs:.2f} s), scaled linearly by unknowns x{n / r['n']:.1f}")}
        except Exception as e:
            cpu = {"value": None, "sample": f"failed: {e}"[:300]}
    line = {"metric": "batched factor+PCG seconds (all systems x right-hand sides to rel. residual 1e-8)",
            "value": fs + ss, "unit": "s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
            "higher_is_better": False, "dtype": {"bf16": "bf16", "fp32": "f32"}.get(a.prec, "f64"),
            "data": "synthetic",
            "config": {"workload": f"{a.systems} FV diffusion systems, sides U{{12..40}}, log-normal sigma 1, "
                                   f"{a.nrhs} right-hand sides each, tol {a.tol:g}", "unknowns": n,
                       "form": FORMS.get(a.prec, a.prec)},
            "factor_s": fs, "solve_s": ss, "iters_max": int(its.max()), "iters_mean": float(its.mean()),
            "relres_max": float(rr.max()), "analyze_s": t_an, "factor_bytes": st["factor_bytes"],
            "gpu_launches": st["gpu_launches"], "n_supernodes": st["n_supernodes"], "n_levels": st["n_levels"],
            "restarts": st["restarts"], "cpu_baseline": cpu,
            "step_factor_s": [r[0] for r in res], "step_solve_s": [r[1] for r in res]}
    print(json.dumps(line), flush=True)


def autograd_workload(a):
    """Differentiation form: loss 0.5 ||x(theta) - x*||^2 for the 7-point FV diffusion operator
    on a side^3 grid with per-cell log-conductivity theta ~ N(0, 1) (seed 0), x* solved from
    theta + 0.1 N(0, 1) (seed 1), b ~ U[-1, 1] (seed 2).  Forward = refactor with the new values
    + PCG; backward = the adjoint PCG with the kept factor + the pattern contraction, then
    autograd through the values to theta.  Timed with CUDA events around each, after warm-up."""
    import numpy as np
    import torch

    import paper_1507_05593_gb300 as R
    import workloads as W
    from paper_1507_05593_gb300.autograd import sparse_spd_solve

    torch.cuda.set_device(0)
    shape = (a.side,) * 3
    fv = W.FVValues(shape)
    theta = np.random.default_rng(0).standard_normal(shape)
    theta_star = theta + 0.1 * np.random.default_rng(1).standard_normal(shape)
    b = torch.tensor(np.random.default_rng(2).uniform(-1, 1, fv.n), device="cuda")
    h = R.rsc_analyze(fv.n, fv.row_ptr, fv.col_idx, fv(torch.tensor(theta)).numpy(), fv.coords,
                      R.rsc_options_default(precision=a.prec))
    with torch.no_grad():
        xs = sparse_spd_solve(fv(torch.tensor(theta_star, device="cuda")), b, h, tol=a.tol, rtol=a.rtol)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    fw, bw = [], []
    for i in range(a.warmup + a.steps):
        flush.fill_(1.0)
        th = torch.tensor(theta, device="cuda", requires_grad=True)
        torch.cuda.synchronize()
        ev[0].record()
        x = sparse_spd_solve(fv(th), b, h, tol=a.tol, rtol=a.rtol)
        loss = 0.5 * ((x - xs) ** 2).sum()
        ev[1].record()
        loss.backward()
        ev[2].record()
        torch.cuda.synchronize()
        if i >= a.warmup:
            fw.append(ev[0].elapsed_time(ev[1]) * 1e-3)
            bw.append(ev[1].elapsed_time(ev[2]) * 1e-3)
    st = R.rsc_get_stats(h)
    f, g = sum(fw) / len(fw), sum(bw) / len(bw)
    cpu = None
    if not a.no_cpu_baseline:
        try:   # the oracle's factor + forward PCG and adjoint PCG on a 24^3 corner of theta, scaled
            crop = min(24, a.side)
            r = _oracle_code(_ORACLE_ADJOINT.format(root=ROOT, side=a.side, crop=crop, tol=a.tol, rtol=a.rtol))
            secs = r["forward"] + r["backward"]
            cpu = {"value": secs * fv.n / r["n"], "unit": "s", "cores": 1, "kind": "oracle",
                   "sample": (f"oracle factor + PCG + adjoint PCG on the {crop}^3 corner of theta ({r['n']:,} "
                              f"unknowns, measured {secs:.2f} s), scaled linearly by unknowns x{fv.n / r['n']:.1f}")}
        except Exception as e:
            cpu = {"value": None, "sample": f"failed: {e}"[:300]}
    line = {"metric": "loss forward (factor + PCG) + backward (adjoint PCG, kept factor) seconds",
            "value": f + g, "unit": "s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
            "higher_is_better": False, "dtype": {"bf16": "bf16", "tf32": "tf32", "fp32": "f32"}.get(a.prec, "f64"),
            "data": "synthetic",
            "config": {"workload": f"FV diffusion {a.side}^3, per-cell log-conductivity theta ~ N(0,1), "
                                   f"loss 0.5||x(theta) - x*||^2, tol {a.tol:g}, PCG rtol {a.rtol:g}",
                       "form": FORMS.get(a.prec, a.prec)},
            "forward_s": f, "backward_s": g, "grad_norm": float(th.grad.norm()), "loss": float(loss),
            "last_iters": st["last_iters"], "factor_bytes": st["factor_bytes"], "restarts": st["restarts"],
            "gpu_launches": st["gpu_launches"], "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- our arm
def main():
    a = _args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if a.impl == "reference":
        reference_arm(a, rank, world)
        return
    if a.workload == "batch":
        if rank == 0:
            batch_workload(a)
        return
    if a.workload == "autograd":
        if rank == 0:
            autograd_workload(a)
        return
    # the other configurations first, each in its own process while this one holds no CUDA
    # context yet: the batched configuration's solve ran 3x slower next to the live handles of
    # this process
    others = None
    if world == 1 and not a.no_others and a.workload == "diffusion" and a.side == 96:
        others = other_configs(a)
    import numpy as np
    import torch

    import paper_1507_05593_gb300 as R
    import workloads as W

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    # cpu baseline first (host cores; a separate process) so it does not overlap the GPU timing
    elastic = a.workload == "elasticity"
    if elastic:
        p = W.elasticity_q1(a.side, incl=_elasticity_incl(a.side))
    elif a.workload == "poisson":
        p = W.poisson7(a.side)
    else:
        p = W.diffusion_grf(a.side, 2.0, 8.0, seed=replica_seed(rank))
    cpu = None
    if rank == 0 and not a.no_cpu_baseline:
        try:
            cpu = cpu_baseline(a.side, a.tol, a.rtol, workload=a.workload, n_full=p.n)
        except Exception as e:  # reported, not fatal
            cpu = {"value": None, "unit": "s", "cores": 1, "kind": "oracle", "sample": f"failed: {e}"[:300]}

    d_b = torch.tensor(p.b, device="cuda")
    d_x = torch.empty_like(d_b)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def make(prec, power_iters=0, interior_blocks=0):
        t = time.perf_counter()
        o = R.rsc_options_default(precision=prec, power_iters=power_iters, dof_per_node=p.dof_per_node,
                                  interior_blocks=interior_blocks)
        h = R.rsc_analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, o)
        return h, time.perf_counter() - t

    def step(h, fixed_rank=False):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        if fixed_rank:   # Section 5.2 ranks: alpha^O = alpha^D = 0.5, p = 8
            R.rsc_factor_fixed_rank(h, 0.5, 0.5, 8)
        else:
            R.rsc_factor(h, a.tol)
        it, rr = R.rsc_solve_device(h, d_b, d_x, a.rtol, 2000)
        st = R.rsc_get_stats(h)
        return st["factor_seconds"] + st["solve_seconds"], it, rr, st

    h, t_an = make(a.prec)
    # untimed: the first factorization of a BF16 / TF32 handle times both kernel variants of the
    # thin products and keeps the faster per size (rsc_get_autotune); the profile is taken after it
    step(h)
    # untimed profiling pass: find the dominant kernel class
    R.rsc_profile(h, True)
    step(h)
    prof_all = R.rsc_get_kernel_profile(h)
    # kernel classes only (profile mode also reports host phases, idle gaps and k_rf_pass phases)
    kern = {k: v for k, v in prof_all.items() if not k.startswith(("wall_", "h_", "gap>", "rfp_", "host_"))}
    dom = max(kern.items(), key=lambda kv: kv[1]["ms"])[0] if kern else None
    R.rsc_profile(h, False)
    for _ in range(max(a.warmup - 1, 0)):
        step(h)
    if dom:
        R.rsc_profile(h, True, dom)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    times, walls, iters, rrs, st = [], [], [], [], None
    for _ in range(a.steps):
        tw = time.perf_counter()
        t, it, rr, st = step(h)
        walls.append(time.perf_counter() - tw)
        times.append(t)
        iters.append(it)
        rrs.append(rr)
    torch.cuda.synchronize()
    clk = clocks.stop()
    kprof = R.rsc_get_kernel_profile(h) if dom else {}
    R.rsc_profile(h, False)
    t_step = sum(times) / len(times)
    t_step = max_over_ranks(t_step, dist, "cuda")
    # end to end through the public host API: values and b copied in, x copied out
    # (one untimed call first, then the mean of `steps` calls, like the device-timed steps)
    def e2e_once():
        t0 = time.perf_counter()
        R.rsc_factor(h, a.tol)
        t1 = time.perf_counter()
        xx, ii, rr_ = R.rsc_solve(h, p.b, a.rtol, 2000)
        return time.perf_counter() - t0, t1 - t0, xx

    e2e_once()
    e2e_runs = [e2e_once() for _ in range(a.steps)]
    t_e2e = sum(r[0] for r in e2e_runs) / len(e2e_runs)
    t_f = sum(r[1] for r in e2e_runs) / len(e2e_runs)
    x = e2e_runs[-1][2]
    res = np.linalg.norm(p.b - p.scipy() @ x) / np.linalg.norm(p.b)
    # the other forms over the same number of timed steps (after one untimed step); the paper's
    # own rank rule over min(steps, 3)
    def side_form(prec, power_iters=0, fixed_rank=False, nsteps=None, interior_blocks=0):
        hs, _ = make(prec, power_iters, interior_blocks)
        step(hs, fixed_rank)   # untimed (and the kernel-variant tuning of the BF16 / TF32 forms)
        runs = [step(hs, fixed_rank) for _ in range(nsteps or a.steps)]
        sts = runs[-1][3]
        secs = sum(r[0] for r in runs) / len(runs)
        fsec = sum(r[3]["factor_seconds"] for r in runs) / len(runs)
        return {"seconds": secs, "steps": len(runs), "factor_s": fsec, "solve_s": secs - fsec,
                "iters": runs[-1][1], "relres": runs[-1][2], "factor_bytes": sts["factor_bytes"],
                "restarts": sts["restarts"], "factor_tflops": sts["factor_flops"] / fsec / 1e12}
    st_main_bytes = R.rsc_get_stats(h)["factor_bytes"]
    fp64 = side_form("fp64") if not a.no_fp64 and a.prec != "fp64" else None
    fp32 = side_form("fp32") if not a.no_fp64 and a.prec in ("bf16", "tf32") else None
    # the paper's own rank rule (Section 5.2) in the same form: RSC0 and RSC1 (one power iteration)
    fixed = None
    if not a.no_fp64 and a.workload == "diffusion":
        fixed = {f"rsc{q}": side_form(a.prec, q, True, min(a.steps, 3)) for q in (0, 1)}
        for q, v in enumerate(fixed.values()):
            v.update({"alpha_O": 0.5, "alpha_D": 0.5, "p": 8, "power_iters": q})
    # Section 5.1's time-memory trade: the same form with interior blocks (their off-diagonal
    # factor blocks never stored), over min(steps, 3) steps
    interior = None
    if not a.no_fp64:
        interior = side_form(a.prec, 0, False, min(a.steps, 3), 1)
        interior["factor_bytes_saved"] = st_main_bytes - interior["factor_bytes"]
    # roofline of the dominant class, timed live over the K timed steps
    roof = None
    if dom and dom in kprof and kprof[dom]["ms"] > 0:
        roof = roofline_entry(dom, kprof[dom], a.prec, "CUDA events on the library's stream around every launch "
                                                        "of the class during the timed steps")
        if roof:
            roof["traffic"] = NCU_TRAFFIC.get(dom) if a.side == 96 and a.workload == "diffusion" else None
            roof["launches_timed"] = roof.pop("launches")
            roof["note"] = "algorithmic bytes (flops) per launch / CUDA-event launch time"
    # every hot class and the preconditioner apply, from the untimed profiled step
    top = sorted(kern.items(), key=lambda kv: -kv[1]["ms"])[:8]
    rooflines = [e for e in (roofline_entry(n, v, a.prec, "untimed profiled step (CUDA events per launch)")
                             for n, v in top) if e]
    if "apply" in kern and all(e["kernel"] != "apply" for e in rooflines):
        e = roofline_entry("apply", kern["apply"], a.prec, "untimed profiled step (one graph launch per apply)")
        if e:
            rooflines.append(e)
    if world > 1 and rank == 0 and not a.no_others and a.workload == "diffusion" and a.side == 96:
        others = other_configs(a)
    cpu_all = None
    if rank == 0 and cpu is not None and not a.no_cpu_baseline:
        try:
            cpu_all = cpu_baseline(a.side, a.tol, a.rtol, workload=a.workload, n_full=p.n, threads=os.cpu_count())
        except Exception as e:
            cpu_all = {"value": None, "sample": f"failed: {e}"[:300]}
    line = {
        "metric": METRIC, "value": t_step, "unit": "s", "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": t_step * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "step_times_s": times,
        "dtype": {"bf16": "bf16", "tf32": "tf32", "fp32": "f32"}.get(a.prec, "f64"), "data": "synthetic",
        "config": {"workload": _workload_name(a.side, a.tol, a.workload)},
        "form": FORMS.get(a.prec, a.prec), "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
        "l2": "L2 flushed (256 MB write) before each step; factor storage larger than L2",
        "iters": iters[-1], "relres": rrs[-1], "true_relres_check": res,
        "factor_s": st["factor_seconds"], "solve_s": st["solve_seconds"],
        "factor_tflops": st["factor_flops"] / st["factor_seconds"] / 1e12, "factor_gflop": st["factor_flops"] / 1e9,
        "factor_bytes": st["factor_bytes"], "analyze_s": t_an, "restarts": st["restarts"],
        "gpu_launches": st["gpu_launches"], "plain_fp64": fp64, "fp32_form": fp32,
        "fixed_rank_form": fixed, "interior_blocks_form": interior, "roofline": roof, "rooflines": rooflines,
        "autotune": R.rsc_get_autotune(h),
        "kernel_profile_untimed": prof_all,
        "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all, "clocks": clk, "other_configs": others,
        "step_wall_s": sum(walls) / len(walls),
        "e2e": {"value": t_e2e, "unit": "s", "factor_wall_s": t_f, "solve_wall_s": t_e2e - t_f,
                "h2d_bytes_per_step": int(8 * (p.nnz + p.n)),
                "d2h_bytes_per_step": int(8 * p.n)},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
