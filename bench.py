"""Throughput of the sparse SCF hot path on one GB300 (or N replicas).

One step = one SCC iteration through the C-ABI (sscf_step: Fock build,
C^T H C transform, pair selection, rotation sweep, one occupied
orthonormalisation pass, density / Mulliken charges / energy, mixing) on the
synthetic water-like cluster of 4096 molecules (16^3 lattice, 12288 atoms,
24576 AOs), mixed precision (FP32 storage, FP64 angles, norms, overlaps and
charge / energy accumulation), cut-off 1e-5.

Input state (untimed): per-molecule guess, full orthonormalisation at the
loose threshold 1e-3 (the paper's first SCF stage), charges of that state;
then W warm-up iterations at the user threshold. That state (C and the
charges) is checkpointed, and every one of the K timed steps restarts from
it before it runs (outside the timed region): all K steps time the same
iteration W + 1, so the result does not depend on K. C (>1 GB) is larger
than the 129 MB L2, so no L2 flush is needed between steps.

Beside the mixed-precision number the line reports the FP64 path on the same
checkpoint (ms per iteration and the energy difference of that iteration),
the converged accuracy of both paths on the 32-molecule cluster against the
dense FP64 oracle, and the end-to-end rate through the C-ABI with the
checkpoint and the charges copied in from page-locked host memory and the
charges copied out, every step.

``--impl reference`` times the FP64 CPU oracle (the same SCC iteration,
step by step) on a bounded sample of the same workload: a 6^3 sub-cube of
the lattice, per iteration, on the host cores.
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
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

L2_BYTES = 129_000_000   # GB300 L2
METRIC = "SCF iter/s & atom·iter/s (mixed vs FP64 GPU), |ΔE|/atom vs oracle, HBM GB/s"
UNIT = "atom*iter/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sscf", choices=["sscf", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--n-mol", type=int, default=4096)
    ap.add_argument("--eps", type=float, default=1e-5)
    ap.add_argument("--prep-eps", type=float, default=1e-3)
    ap.add_argument("--prep-passes", type=int, default=200)
    ap.add_argument("--sample-mol", type=int, default=216,
                    help="molecules of the sub-cube the oracle is timed on (CPU baseline and reference arm)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--clusters", type=int, default=0,
                    help="batched workload: the first K clusters of the seed-7 size draw U[200, 3000] in one context")
    ap.add_argument("--wave", type=int, default=0,
                    help="batched workload: clusters per context, contexts run one after another (0: all in one)")
    ap.add_argument("--cap-tiles", type=int, default=0, help="tiles per row of C (0: the largest cluster's tiles)")
    ap.add_argument("--cap-y", type=int, default=0, help="row blocks per tile of Y (0: the largest cluster)")
    ap.add_argument("--closure-mode", type=int, default=0,
                    help="0: structural fill once per sweep; k >= 1: once per k colours (bounded rows, large clusters)")
    ap.add_argument("--graph", action="store_true", help="replay each SCC iteration as one CUDA graph")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default transform launch shape")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 path on the same checkpoint")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the converged 32-molecule accuracy check")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (very large single clusters)")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batch leg (the first wave of the 256-cluster batch, graph-replayed steps)")
    ap.add_argument("--batch-clusters", type=int, default=32, help="clusters in the batch leg")
    return ap.parse_args()


def oracle_rate_one_core(n_mol: int, eps: float):
    """The oracle's iteration rate with one BLAS thread, in a child process (thread counts are read at import)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import json, bench; r = bench.oracle_iteration_rate(%d, %r, 1); print(json.dumps(r[:2]))"
            % (n_mol, eps))
    try:
        out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                             timeout=600)
        return tuple(json.loads(out.stdout.strip().splitlines()[-1]))
    except (subprocess.SubprocessError, ValueError, IndexError):
        return None


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


# ---------------------------------------------------------------------------
# oracle timing (CPU baseline and the reference arm)
# ---------------------------------------------------------------------------
def oracle_iteration_rate(n_mol: int, eps: float, steps: int, warmup: int = 0):
    """Atom*iter/s of oracle B's SCC iteration on a sub-cube of n_mol molecules."""
    from oracle import sparse
    from synth import default_params, lattice_water
    p = default_params()
    s = lattice_water(n_mol, seed=0)
    scf = sparse.SparseSCF(s, p)
    st = scf.start(1e-3)
    for _ in range(warmup):
        scf.step(st, eps)
    t0 = time.perf_counter()
    for _ in range(steps):
        scf.step(st, eps)
    dt = time.perf_counter() - t0
    return s.n_atoms * steps / dt, dt, s.n_atoms


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
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
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
def shard(items, rank: int, world: int):
    """Independent units (clusters) of rank `rank` out of `world`: every `world`-th, starting at `rank`."""
    return list(items)[rank::world]


def aggregate(local_atoms: float, local_ms: float, dist=None, device=None):
    """Whole-job atoms (sum over ranks) and the slowest rank's time (max over ranks)."""
    if dist is None:
        return float(local_atoms), float(local_ms)
    import torch
    a = torch.tensor([float(local_atoms)], dtype=torch.float64, device=device)
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(a, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(a.item()), float(t.item())


# ---------------------------------------------------------------------------
def kernel_code_digest(path: str) -> str:
    """SHA-256 of the sweep kernels' source (k_rotate.cu: kernels and launchers)
    and of the shared header beside it (sscf_internal.h: argument structs,
    constants, layout), without comments and white space."""
    parts = []
    for f in (path, os.path.join(os.path.dirname(path), "sscf_internal.h")):
        with open(f) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        parts.append(re.sub(r"\s+", "", src))
    return hashlib.sha256("\0".join(parts).encode()).hexdigest()


def measured_traffic(name: str, workload: str, root: str = ROOT):
    """DRAM bytes per call of a launcher from a committed ncu capture
    (profiles/dram_traffic_<name>_water4096_mixed.md), or None when the kernel
    code or the workload differs from the captured one."""
    path = os.path.join(root, "profiles", f"dram_traffic_{name}_water4096_mixed.md")
    try:
        with open(path) as f:
            line = next(l for l in f if l.startswith(f"traffic: {name} "))
        digest = kernel_code_digest(os.path.join(root, "paper_1402_2880_gb300", "csrc", "k_rotate.cu"))
    except (OSError, StopIteration, ValueError):
        return None
    fields = dict(kv.split("=", 1) for kv in line.split()[2:])
    if fields.get("kernel_code_sha256") != digest or fields.get("workload") != workload:
        return None
    return float(fields["bytes_per_call"])


def pinned_copy(a):
    """A page-locked host copy of a numpy array (the end-to-end leg's inputs)."""
    import numpy as np
    import torch
    t = torch.empty(a.shape, dtype=getattr(torch, str(a.dtype)), pin_memory=True)
    out = t.numpy()
    np.copyto(out, a)
    return out


def accuracy_config1(p):
    """Converged 32-molecule cluster (4x4x2, eps 1e-6, converged to 1e-7 e and
    1e-10 Ha so that the SCF criterion stays below the tolerances): |dE| per
    atom and the largest charge difference of the mixed and the FP64 path
    against the dense FP64 oracle's converged state, stored by
    tests/golden/make_config1_dense.py (this leg runs no oracle code)."""
    import numpy as np

    from paper_1402_2880_gb300 import SSCF_FP64, SSCF_MIXED, Context
    from synth import lattice_water
    with open(os.path.join(ROOT, "tests", "golden", "config1_dense.json")) as f:
        ref = json.load(f)
    s = lattice_water(32, seed=0)
    pt = dict(p, dq_tol=1e-7, e_tol=1e-10)
    out = {}
    for name, prec in (("mixed", SSCF_MIXED), ("fp64", SSCF_FP64)):
        ctx = Context.from_system(s, pt, precision=prec)
        r = ctx.run(allow_not_converged=True)
        q, _, _ = ctx.get_charges()
        ctx.close()
        out[name] = {"converged": bool(r["converged"]),
                     "abs_dE_per_atom": abs(r["energy"] - ref["energy"]) / s.n_atoms,
                     "max_abs_dq": float(np.abs(q - np.asarray(ref["q"])).max())}
    out["oracle"] = ref["what"]
    return out


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    n_gpus = max(args.gpus, world)

    if args.impl == "reference":
        if rank != 0:
            return
        K, W = max(args.steps, 1), args.warmup
        cores = host_cores()
        rate, dt, n_at = oracle_iteration_rate(args.sample_mol, args.eps, K, W)
        line = {
            "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": n_gpus,
            "steps": K, "warmup": W, "ms_per_step": 1e3 * dt / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"water lattice, {args.sample_mol}-molecule sub-cube of the "
                                   f"{args.n_mol}-molecule cluster, eps {args.eps:g}", "n_mol": args.n_mol,
                       "sample_mol": args.sample_mol},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{K} SCC iterations of oracle B on {args.sample_mol} molecules"},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }
        print(json.dumps(line), flush=True)
        return

    import numpy as np
    import torch

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count

    from paper_1402_2880_gb300 import SSCF_FP64, SSCF_MIXED, SSCF_ORTHO_ALL, Context, build
    from synth import default_params, lattice_water
    if rank == 0:
        build.build()
    if dist is not None:
        dist.barrier()
    build.build()

    p = default_params()
    if args.clusters > 0:
        # independent clusters: each rank converges its own share, no data-path collective
        from synth import cluster_sizes, concat_clusters
        if args.clusters < world:
            raise SystemExit(f"--clusters {args.clusters} gives some of the {world} ranks no cluster")
        mine = shard(enumerate(cluster_sizes()[:args.clusters]), rank, world)
        w = args.wave if args.wave > 0 else len(mine)
        systems = [concat_clusters([lattice_water(int(nm), seed=k) for k, nm in mine[i:i + w]])
                   for i in range(0, len(mine), w)]
    else:
        systems = [lattice_water(args.n_mol, seed=0)]
    stream = torch.cuda.Stream(dev) if args.graph else torch.cuda.current_stream(dev)
    prec = SSCF_MIXED if args.precision == "mixed" else SSCF_FP64
    K = args.steps
    flush = None

    def timed_steps(ctx, ck, n_steps, flushing, on=None):
        """n_steps replays of the checkpointed iteration: restore (untimed), then one
        sscf_step between CUDA events on the context's stream; returns (ms, infos)."""
        nonlocal flush
        st = stream if on is None else on
        if flushing and flush is None:
            flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(n_steps)]
        infos = []
        for k in range(n_steps):
            ctx.set_C_tiles(*ck[0])
            ctx.set_charges(*ck[1])
            if flushing:
                with torch.cuda.stream(st):
                    flush.zero_()
            ev[k][0].record(st)
            infos.append(ctx.step())
            ev[k][1].record(st)
        torch.cuda.synchronize(dev)
        return sum(a.elapsed_time(b_) for a, b_ in ev), infos

    def run_one(s, fp64_leg: bool):
        """Prepare one context (untimed), warm up, checkpoint, time K replays of the
        next iteration, then K end-to-end replays; optionally the FP64 path on the
        same checkpoint."""
        ctx = Context.from_system(s, p, precision=prec, stream=stream.cuda_stream, cap_tiles=args.cap_tiles,
                                  cap_y=args.cap_y, closure_mode=args.closure_mode)
        ctx.set_thresholds(args.prep_eps, 10 * args.prep_eps, 1e-8)
        ctx.guess()
        prep = ctx.orthonormalise(SSCF_ORTHO_ALL, max_pass=args.prep_passes)
        ctx.set_thresholds(args.eps, 10 * args.eps, 1e-6)
        ctx.reset_charges()
        # warm-up: eager steps, then the launch-shape autotuner on the state of
        # the last warm-up step (the closest to the replayed one), which that step
        # runs with (graph-captured when asked, so that no capture falls in the
        # timed region)
        warm = None
        tuned = None
        for w in range(max(args.warmup, 0)):
            if w == max(args.warmup - 1, 0):
                if not args.no_autotune:
                    tuned = ctx.autotune()
                if args.graph:
                    ctx.enable_graph(True)
            warm = ctx.step()
        torch.cuda.synchronize(dev)
        ck = (ctx.get_C_tiles(), ctx.get_charges())
        n_stored = int(ck[0][1].size)
        c_bytes = (4 if prec == SSCF_MIXED else 8) * n_stored * 96
        flushing = c_bytes < 2 * L2_BYTES
        # one untimed replay: the graph (if any) is captured for the restored buffer parity
        ctx.set_C_tiles(*ck[0])
        ctx.set_charges(*ck[1])
        ctx.step()
        ctx.profile(True)
        ms, infos = timed_steps(ctx, ck, K, flushing)
        prof = ctx.profile_read()
        ctx.profile(False)
        # end to end through the C-ABI: the checkpoint (C and charges) in from
        # page-locked host memory, one SCC iteration, the charges out, every step
        e2e_dt, h2d, d2h = None, 0, 0
        if not args.no_e2e:
            pin_ck = tuple(pinned_copy(a) for a in ck[0])
            pin_q = [pinned_copy(a) for a in ck[1]]
            pin_out = [pinned_copy(a) for a in ck[1]]
            h2d = sum(a.nbytes for a in pin_ck) + sum(a.nbytes for a in pin_q)
            d2h = sum(a.nbytes for a in pin_out)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            for _ in range(K):
                ctx.set_C_tiles(*pin_ck)
                ctx.set_charges(*pin_q)
                ctx.step()
                ctx.get_charges(out=pin_out)
            torch.cuda.synchronize(dev)
            e2e_dt = time.perf_counter() - t0
        n_mo = ctx.n_mo
        ctx.close()
        fp64 = None
        if fp64_leg and prec == SSCF_MIXED:
            # the FP64 path on the same checkpoint (the FP32 values widen exactly)
            c64 = Context.from_system(s, p, precision=SSCF_FP64, stream=stream.cuda_stream,
                                      cap_tiles=args.cap_tiles, cap_y=args.cap_y, closure_mode=args.closure_mode)
            c64.set_thresholds(args.eps, 10 * args.eps, 1e-6)
            if not args.no_autotune:
                c64.set_C_tiles(*ck[0])
                c64.set_charges(*ck[1])
                c64.autotune()
            n64 = 2
            ms64, inf64 = timed_steps(c64, ck, n64, flushing)
            c64.close()
            e_mixed = float(np.mean([inf["energy"] for inf in infos]))
            fp64 = {"ms_per_step": ms64 / n64, "steps": n64, "energy": inf64[-1]["energy"],
                    "energy_mixed": e_mixed,
                    "abs_dE_per_atom_mixed_vs_fp64": abs(e_mixed - inf64[-1]["energy"]) / s.n_atoms,
                    "n_rot": inf64[-1]["n_rot"], "n_combo": inf64[-1]["n_combo"]}
        return dict(ms=ms, infos=infos, prof=prof, e2e_dt=e2e_dt, prep=prep, c_bytes=c_bytes,
                    flushing=flushing, n_mo=n_mo, tuned=tuned, h2d=h2d, d2h=d2h, fp64=fp64,
                    same_iteration=len({round(inf["energy"], 9) for inf in infos}) == 1)

    sampler = ClockSampler(local_rank)
    sampler.start()
    if dist is not None:
        dist.barrier()
    runs = [run_one(s, fp64_leg=(rank == 0 and i == 0 and not args.no_fp64)) for i, s in enumerate(systems)]
    if dist is not None:
        dist.barrier()
    clocks = sampler.stop()
    n_atoms_local = sum(s.n_atoms for s in systems)
    n_mol_local = sum(s.n_mol for s in systems)
    ms = sum(r["ms"] for r in runs)
    job_atoms, t_max = aggregate(n_atoms_local, ms, dist, dev)
    value = job_atoms * K / (t_max / 1e3)
    e2e_value = None
    if not args.no_e2e:
        _, e2e_t = aggregate(n_atoms_local, sum(r["e2e_dt"] for r in runs), dist, dev)
        e2e_value = job_atoms * K / e2e_t
    infos = [inf for r in runs for inf in r["infos"]]
    prof = {}
    for r in runs:
        for k_, (t_, n_) in r["prof"].items():
            t0_, n0_ = prof.get(k_, (0.0, 0))
            prof[k_] = (t0_ + t_, n0_ + n_)
    prep_passes, prep_eta = runs[0]["prep"]
    c_bytes = max(r["c_bytes"] for r in runs)
    flushed = any(r["flushing"] for r in runs)
    n_mo_local = sum(r["n_mo"] for r in runs)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    # roofline of the dominant launcher: algorithmic HBM bytes per call / mean call time
    tsz = 4 if prec == SSCF_MIXED else 8
    # per-step quantities summed over the waves
    mean = lambda k: float(np.mean([inf[k] for inf in infos])) * len(runs)  # noqa: E731
    nnz_c, nnz_o = mean("nnz_c"), mean("nnz_occ")
    n_rot, n_combo = mean("n_rot"), mean("n_combo")
    algo_bytes = {
        "apply_rot": 2 * tsz * nnz_c + 24 * n_rot,           # read + write C once, pair records
        "apply_ortho": 2 * tsz * nnz_o + 16 * n_combo,        # read + write C_occ once, pair records
        "xc_h": 2 * tsz * nnz_c,                              # read C, write Y = H C
        "xc_s": 2 * tsz * nnz_o,
        "transform_ov": 2 * tsz * nnz_c,                      # read C and Y once
        "transform_ss": 2 * tsz * nnz_o,
        "density": tsz * nnz_o + 8 * n_atoms_local,
        "closure": 2 * tsz * nnz_c,
        "compact": 2 * tsz * nnz_c,
    }
    per_step = {k: v[0] / K for k, v in prof.items() if v[1] > 0}
    dominant = max(per_step, key=per_step.get) if per_step else None
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in peaks else "fallback 6800 GB/s"

    # FP32 (or FP64) ALU peak from unit counts and the maximum SM clock:
    # SMs (read from the device) x 128 FP32 lanes x 2 flops x max clock; FP64 at 1/64 of it
    sm_clk = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    alu_peak = n_sm * 128 * 2 * sm_clk / 1e12 * (1.0 if prec == SSCF_MIXED else 1.0 / 64)
    upd = {"apply_rot": mean("upd_rot"), "apply_ortho": mean("upd_combo")}
    workload_key = (f"n_mol:{args.n_mol},eps:{args.eps:g},precision:{args.precision},"
                    f"clusters:{max(args.clusters, 1)},replayed_iteration:{args.warmup + 1}")

    def roof(name):
        """HBM roofline of one launcher (the headline: algorithmic bytes / time
        against the measured copy bandwidth); the sweeps also get the ALU view."""
        calls = prof[name][1] / K
        t_call = prof[name][0] / max(prof[name][1], 1) / 1e3
        b = algo_bytes.get(name)
        if b is None:
            return None
        achieved = b / max(calls, 1) / t_call / 1e9
        r = {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
             "frac": achieved / hbm_peak, "traffic": measured_traffic(name, workload_key),
             "peak_source": peak_src, "algorithmic_bytes_per_call": b / max(calls, 1),
             "ms_per_step": per_step[name]}
        if name in upd:
            # 2x2 updates: 2 FMAs (4 flops) per AO row and pair
            a_alu = 4.0 * upd[name] / max(calls, 1) / t_call / 1e12
            r["alu_view"] = {"achieved": a_alu, "peak": alu_peak, "unit": "TFLOP/s", "frac": a_alu / alu_peak,
                             "peak_source": f"derived: {n_sm} SMs x 128 FP32 lanes x 2 flops x max SM clock "
                                            f"{sm_clk / 1e6:.0f} MHz"}
        return r

    # graph replays are not seen by the per-launcher events: no per-kernel split then
    roofline = roof(dominant) if dominant else None
    kernels = {k: {"ms_per_step": round(v, 3), "calls_per_step": prof[k][1] / K} for k, v in per_step.items()}
    for name in ("apply_rot", "apply_ortho", "transform_ov", "transform_ss", "density", "xc_h", "xc_s"):
        if name in per_step and name != dominant:
            kernels[name]["roofline"] = roof(name)

    cpu = None
    if not args.no_cpu_baseline:
        rate, dt, n_at = oracle_iteration_rate(args.sample_mol, args.eps, 3)
        cpu = {"value": rate, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
               "sample": f"3 SCC iterations of oracle B (FP64, numpy) on a {args.sample_mol}-molecule "
                         f"sub-cube of the same lattice ({n_at} atoms), {dt:.1f} s; its per-atom rate falls "
                         f"as the cluster grows (dense N^3 products), so the rate on the full cluster is lower"}
        one = oracle_rate_one_core(args.sample_mol, args.eps)
        if one is not None:
            cpu["one_core"] = {"value": one[0], "unit": UNIT, "cores": 1,
                               "sample": f"1 SCC iteration of the same sample with one BLAS thread, {one[1]:.1f} s"}

    accuracy = None
    if not args.no_accuracy:
        accuracy = accuracy_config1(p)

    def batch_leg(n_clusters: int, n_steps: int = 2, warmup: int = 3):
        """The first n_clusters of the 256-cluster batch (sizes U[200, 3000], seed 7)
        in one context, mixed, eps 1e-5: every SCC iteration of all of them is one
        CUDA-graph replay on a side stream; iteration warmup + 1 replayed from a
        checkpoint n_steps times between CUDA events, as the main leg."""
        from synth import cluster_sizes, concat_clusters
        sizes = cluster_sizes()[:n_clusters]
        sb = concat_clusters([lattice_water(int(nm), seed=k) for k, nm in enumerate(sizes)])
        st = torch.cuda.Stream(dev)
        ctx = Context.from_system(sb, p, precision=SSCF_MIXED, stream=st.cuda_stream)
        ctx.set_thresholds(args.prep_eps, 10 * args.prep_eps, 1e-8)
        ctx.guess()
        ctx.orthonormalise(SSCF_ORTHO_ALL, max_pass=args.prep_passes)
        ctx.set_thresholds(1e-5, 1e-4, 1e-6)
        ctx.reset_charges()
        for w in range(warmup):
            if w == 1:
                ctx.autotune()
                ctx.enable_graph(True)
            ctx.step()
        torch.cuda.synchronize(dev)
        ckb = (ctx.get_C_tiles(), ctx.get_charges())
        ctx.set_C_tiles(*ckb[0])
        ctx.set_charges(*ckb[1])
        ctx.step()   # untimed replay
        samp = ClockSampler(local_rank)
        samp.start()
        msb, infb = timed_steps(ctx, ckb, n_steps, False, on=st)
        clk = samp.stop()
        n_mo_b = ctx.n_mo
        ctx.close()
        t = msb / n_steps / 1e3
        return {"workload": f"the first {n_clusters} clusters of the 256-cluster batch ({sb.n_mol} molecules, "
                            f"{sb.n_atoms} atoms) in one context, mixed, eps 1e-05; each SCC iteration of all "
                            f"of them is one CUDA-graph replay; iteration {warmup + 1} replayed {n_steps} times "
                            "from a checkpoint",
                "clusters": n_clusters, "n_mol": sb.n_mol, "n_atoms": sb.n_atoms,
                "ms_per_step": msb / n_steps, "cluster_iter_per_s": n_clusters / t,
                "atom_iter_per_s": sb.n_atoms / t, "graph": True,
                "nnz_per_mo": float(np.mean([inf["nnz_c"] for inf in infb])) / n_mo_b,
                "same_iteration_every_step": len({round(inf["energy"], 9) for inf in infb}) == 1,
                "clocks": clk}

    batch = None
    if not args.no_batch and args.clusters == 0 and args.precision == "mixed":
        batch = batch_leg(args.batch_clusters)

    launches = int(round(mean("launches")))
    fp64 = runs[0]["fp64"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": n_gpus, "steps": K, "warmup": args.warmup,
        "ms_per_step": t_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if prec == SSCF_MIXED else "f64", "data": "synthetic",
        "config": {"workload": (f"batch of {args.clusters} independent water-lattice clusters "
                                f"({n_mol_local} molecules, {n_atoms_local} atoms"
                                + (f", {len(runs)} waves of {args.wave}" if len(runs) > 1 else "") + "), "
                                if args.clusters > 0 else
                                f"water lattice {args.n_mol} molecules ({n_atoms_local} atoms, {6 * args.n_mol} AOs), ")
                               + f"{args.precision}, eps {args.eps:g}; every step replays SCC iteration "
                               + f"{args.warmup + 1} from a checkpoint of C and the charges (restored before "
                               + "each step, outside the timed region)"
                               + (", CUDA graph" if args.graph else ""),
                   "n_mol": n_mol_local, "eps": args.eps, "precision": args.precision, "clusters": max(args.clusters, 1),
                   "replayed_iteration": args.warmup + 1,
                   "closure": f"per {args.closure_mode} colours" if args.closure_mode > 0 else "per sweep",
                   "cap_tiles": args.cap_tiles, "cap_y": args.cap_y,
                   "nnz_per_mo": nnz_c / n_mo_local,
                   "parallelism": ("clusters sharded over ranks" if args.clusters > 0 else "replicas")
                                  if n_gpus > 1 else "single",
                   "l2": (f"C holds {c_bytes / 1e6:.0f} MB, " + ("L2 flushed (256 MB write) before every timed step"
                                                                   if flushed else
                                                                   "more than twice the 129 MB L2: no flush")),
                   "prep": {"eps": args.prep_eps, "ortho_passes": prep_passes, "eta": prep_eta},
                   "autotune": {"transform_ctas_per_tile": sorted({r["tuned"] % 16 for r in runs if r["tuned"]}),
                                "transform_regs_cut_for_4_ctas": sorted({r["tuned"] >= 16 for r in runs
                                                                         if r["tuned"]})}},
        "scf_iter_per_s": n_gpus * K / (t_max / 1e3),
        "cluster_iter_per_s": (max(args.clusters, 1) if args.clusters > 0 else n_gpus) * K / (t_max / 1e3),
        "clocks": clocks,
        "e2e": None if e2e_value is None else {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": sum(r["h2d"] for r in runs),
                "d2h_bytes_per_step": sum(r["d2h"] for r in runs),
                "what": "per step through the C-ABI: sscf_set_C_tiles (checkpoint of C, FP64 tiles) and "
                        "sscf_set_charges from page-locked host memory, sscf_step, sscf_get_charges"},
        "gpu_launches": launches * K,
        "roofline": roofline,
        "kernels": kernels,
        "cpu_baseline": cpu,
        "fp64": fp64,
        "mixed_speedup_vs_fp64": (fp64["ms_per_step"] / (t_max / K)) if fp64 else None,
        "accuracy": accuracy,
        "batch": batch,
        "state": {"energy": infos[-1]["energy"], "dq_max": infos[-1]["dq_max"], "n_rot": n_rot,
                  "n_combo": n_combo, "nnz_per_mo": nnz_c / n_mo_local,
                  "same_iteration_every_step": all(r["same_iteration"] for r in runs)},
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
