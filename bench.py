"""Benchmark: butterfly Legendre stage of the SHT at l = 1024 on one GB300.

One step = one synthesis (beta -> G at the 2l Gauss-Legendre nodes, all
orders m) plus one analysis (G -> beta, the transposed butterfly) of one
synthetic field, through the C ABI, with the float64 butterfly (eps_id =
1e-12).  value = Legendre-stage transforms per second (a synthesis and an
analysis each count as one transform), whole job over all ranks.

Prints ONE JSON line (rank 0).  Launch: python bench.py [--gpus N --steps K
--warmup W]; for N > 1 under torch.distributed.run (one process per GPU,
each rank transforms its own field: weak scaling, no collective on the data
path).  --impl reference times the float64 oracle on the host cores instead.
"""

import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

HBM_FALLBACK_GBS = 6800.0
# float64 FMA peak of a GB300 from its unit counts and clock: 2 DFMA
# thread-ops / clock / SM (ncu sm__sass_thread_inst_executed_op_dfma_pred_on
# .peak_sustained) x 152 SMs x 2.07 GHz x 2 flops.  The library's DFMA loop
# (sht_measure_fp64_fma: eight independent chains per thread, 2048 threads
# per SM) reaches about 99.8 % of it; the bench reports both fractions.
FP64_PEAK_TFLOPS = 2 * 152 * 2.07e9 * 2 / 1e12
METRIC = "SHT/s at l=1024, butterfly vs direct FP64 on GPU (Legendre-stage transforms per second)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--l", type=int, default=1024)
    ap.add_argument("--leaf-cols", type=int, default=32)
    ap.add_argument("--page-bytes", type=int, default=0, help="record chunk bytes (0: the plan default)")
    ap.add_argument("--consumer-warps", type=int, default=0)
    ap.add_argument("--eps", type=float, default=1e-12)
    ap.add_argument("--no-extras", action="store_true", help="skip every leg beside the float64 headline")
    ap.add_argument("--paths", default="split32,split32acc64,fp32,direct,full,batched,autograd,device_build,"
                                       "gauss_jacobi",
                    help="comma-separated legs to run beside the headline (also: trace, the sweep's "
                         "per-op trace shares)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the cpu_baseline leg")
    ap.add_argument("--cpu-all-cores", type=int, default=1,
                    help="also time the oracle over all orders on every host core (0: skip)")
    ap.add_argument("--batch-fields", type=int, default=96,
                    help="fields of the batched leg (bandlimits drawn from 64..1024); 0 skips it")
    ap.add_argument("--cpu-stride", type=int, default=8, help="oracle samples every stride-th order")
    return ap.parse_args()


# DRAM traffic of the float64 sweep, from a small capture: dram__bytes_read.sum
# + dram__bytes_write.sum of one synthesis and one analysis launch at l = 512
# (leaf_cols 32, the default record chunk), both per launch, beside that
# plan's float64 stream bytes.  A launch at another l is credited with the
# same bytes per stream byte (traffic scales with the stream: every value is
# read once, beta and G are under 1 % of it).  Valid only for the kernel and
# stream-format sources the capture was taken with (sources_sha); None when
# no capture matches.
SWEEP_TRAFFIC_CAPTURE = {"l": 512, "leaf_cols": 32, "page_bytes": 0, "stream_bytes": 1087871856,
                         "dram_bytes_syn": 1.098007e9 + 20.198400e6, "dram_bytes_ana": 1.093494e9 + 12.580608e6,
                         "sources_sha": "d3e72f6c3621d35e"}


def sweep_sources_sha():
    """Hash of the kernel, stream-format and encoder sources, comments and
    blank lines left out (they change no launch)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for name in ("sweep.cu", "sht_stream.h", "plan_build.cpp", "kernels.h"):
        with open(os.path.join(ROOT, "paper_0910_5435_gb300", "csrc", name)) as f:
            text = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
        code = [ln.split("//")[0].rstrip() for ln in text.splitlines()]
        h.update(name.encode() + "\n".join(ln for ln in code if ln).encode())
    return h.hexdigest()[:16]


def device_build_leg(args, sht, torch, dev, stream, plan, st, beta):
    """The same plan with its factorizations built on the GPU: build time
    beside the host build's, rank statistics, and the two plans' float64
    syntheses of the bench field compared."""
    l = plan.l
    t0 = time.perf_counter()
    pd = sht.Plan(l, args.eps, leaf_cols=args.leaf_cols, page_bytes=args.page_bytes,
                  consumer_warps=args.consumer_warps, device_build=True)
    t_plan = time.perf_counter() - t0
    sd = pd.stats()
    gh = torch.empty((2 * l, 2 * l), dtype=torch.complex128, device=dev)
    gd = torch.empty_like(gh)
    sht.sht_legendre_synthesize(plan, sht.SHT_FP64, beta, gh, stream)
    sht.sht_legendre_synthesize(pd, sht.SHT_FP64, beta, gd, stream)
    torch.cuda.synchronize()
    out = {"t_plan_s": t_plan, "t_comp": sd["t_comp"], "t_factor": sd["t_factor"],
           "t_factor_kernel": sd["t_factor_kernel"], "host_t_comp": st["t_comp"], "host_t_factor": st["t_factor"],
           "factor_speedup_vs_host": st["t_factor"] / max(1e-9, sd["t_factor"]),
           "factor_flops": sd["factor_flops"],
           "factor_kernel_tflops": sd["factor_flops"] / max(1e-9, sd["t_factor_kernel"]) / 1e12,
           "factor_kernel_frac_of_fp64_peak": sd["factor_flops"] / max(1e-9, sd["t_factor_kernel"]) / 1e12
                                              / FP64_PEAK_TFLOPS,
           "k_avg": sd["k_avg"], "k_max": sd["k_max"], "factor_values": sd["factor_values"],
           "host_factor_values": st["factor_values"],
           "rel_synthesis_vs_host_plan": float(torch.linalg.vector_norm(gd - gh) / torch.linalg.vector_norm(gh)),
           "device_status": int(sht.sht_last_device_status(pd))}
    pd.close()
    return out


def gauss_jacobi_leg(args, sht, torch, dev, stream):
    """The paper's own matrices (Section 4, eq. transform; Tables evens_time /
    evens_pre at m = n): one single-block plan per n (C = 60, IDs to 1e-15 as
    the paper's "nearly machine precision"), the forward and inverse
    transforms of two unit-norm U(-1, 1) vectors on the GPU (float64),
    timed with CUDA events over 20 calls each, and eps_inv (forward then
    inverse, largest entry error).  Parity against the oracle is in the
    test suite."""
    out = []
    for n in (1250, 2500, 5000, 10000):
        t0 = time.perf_counter()
        P = sht.GJPlan(n, n, 0, eps_id=1e-15, leaf_cols=60)
        t_plan = time.perf_counter() - t0
        st = P.stats()
        rng = np.random.default_rng(n)
        v = rng.uniform(-1, 1, (n, 2))
        v /= np.linalg.norm(v, axis=0)
        x = torch.from_numpy(v[:, 0] + 1j * v[:, 1]).to(dev)
        y = torch.empty_like(x)
        z = torch.empty_like(x)

        def timed(fn, reps=20):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps

        ms_f = timed(lambda: sht.sht_gj_forward(P, sht.SHT_FP64, x, y, stream))
        ms_i = timed(lambda: sht.sht_gj_inverse(P, sht.SHT_FP64, y, z, stream))
        torch.cuda.synchronize()
        out.append({"n": n, "m": n, "parity": 0, "t_fwd_s": ms_f / 1e3, "t_inv_s": ms_i / 1e3,
                    "launches": [P.launches(0, 0), P.launches(0, 1)], "t_quad_s": st["t_quad"],
                    "t_comp_s": st["t_comp"], "t_plan_s": t_plan, "k_max": st["k_max"], "k_avg": st["k_avg"],
                    "eps_inv": float((z - x).abs().max()), "device_status": sht.sht_last_device_status(P, stream)})
        P.close()
    return out


TRACE_KEYS = ("exec_gemv", "exec_control", "wait_dep", "wait_values", "wait_records", "wait_barrier", "complete")


def trace_leg(args, sht, torch, dev, stream, plan, beta):
    """Per-op trace of the sweep (sht_trace_enable): for float64, split and
    float32, one traced synthesis and one traced analysis after the timed
    ones, as shares of the warps' cycles (executing compute ops, control ops,
    waiting for other warps, for staged values, for record chunks, at the
    item barrier, publishing) and the mean cycles per compute op."""
    l = args.l
    out = {}
    for name, prec, cdt in (("fp64", sht.SHT_FP64, torch.complex128), ("split32", sht.SHT_SPLIT32, torch.complex128),
                            ("fp32", sht.SHT_FP32, torch.complex64)):
        plan.prepare(prec)
        b = beta.to(cdt)
        g = torch.empty((2 * l, 2 * l), dtype=cdt, device=dev)
        bk = torch.empty_like(b)
        res = {}
        for direction, fn in (("synthesis", lambda: sht.sht_legendre_synthesize(plan, prec, b, g, stream)),
                              ("analysis", lambda: sht.sht_legendre_analyze(plan, prec, g, bk, stream))):
            for _ in range(3):
                fn()
            torch.cuda.synchronize(dev)
            sht.sht_trace_enable(plan, True)
            try:
                sht.sht_trace_read(plan, reset=True)
                fn()
                torch.cuda.synchronize(dev)
                t = sht.sht_trace_read(plan, reset=True)
            finally:
                sht.sht_trace_enable(plan, False)
            tot = sum(t[k] for k in TRACE_KEYS)
            res[direction] = {"share": {k: t[k] / tot for k in TRACE_KEYS},
                              "compute_ops": int(t["n_gemv"]), "control_ops": int(t["n_control"]),
                              "cycles_per_compute_op": t["exec_gemv"] / max(1, t["n_gemv"])}
        out[name] = res
    return out


def shard_fields(ls, rank, world):
    """Fields of a batch assigned to one rank: longest-processing-time order
    with the cost of a field taken as l^2 log l (the butterfly's work), each
    field to the currently least loaded rank; ties go to the lower rank.
    Every rank computes the same assignment, so no exchange is needed."""
    import math
    order = sorted(range(len(ls)), key=lambda f: (-ls[f] ** 2 * math.log2(max(2, ls[f])), f))
    load = [0.0] * world
    mine = []
    for f in order:
        r = min(range(world), key=lambda q: (load[q], q))
        load[r] += ls[f] ** 2 * math.log2(max(2, ls[f]))
        if r == rank:
            mine.append(f)
    return sorted(mine)


def max_over_ranks(value, world, dist, device=None):
    """The largest value over all ranks (the job's time is its slowest
    rank's); the value itself when there is one rank."""
    if world <= 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
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
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_leg(l, stride, seed, outputs_path=None, err_stride=64):
    """Runs the float64 oracle (one thread, in a subprocess) on the middle
    order of every run of stride orders, m = stride/2, 3*stride/2, ..., and
    returns its timing.  An order's cost falls about linearly in m, so the
    middle order stands for its run without the bias of the first one.  If
    GPU outputs are given (npz with <path>_G and <path>_beta arrays), also
    returns, on the orders m = 0, err_stride, ..., the relative l2 error of
    each path's synthesis against the oracle synthesis of the same beta, and
    of its analysis against the oracle analysis of that path's own G."""
    code = r"""
import json, sys, time, os
import numpy as np
sys.path.insert(0, sys.argv[1])
import oracle
from paper_0910_5435_gb300 import inputs
l, stride, seed, err_stride = int(sys.argv[2]), int(sys.argv[3]), int(sys.argv[4]), int(sys.argv[6])
ms = list(range(stride // 2, 2 * l, stride))
assert ms, "empty order sample"
beta = inputs.random_beta(l, seed=seed, decay=True)
tn = time.perf_counter()
oracle.gl_nodes_weights(2 * l)
t0 = time.perf_counter()
Go = oracle.legendre_synthesis(beta, l, orders=ms)
t1 = time.perf_counter()
bo = oracle.legendre_analysis(Go, l, orders=ms)
t2 = time.perf_counter()
out = {"orders": len(ms), "t_nodes": t0 - tn, "t_synth": t1 - t0, "t_analysis": t2 - t1}
path = sys.argv[5]
if path != "-":
    d = np.load(path)
    me = list(range(0, 2 * l, err_stride))
    Ge = oracle.legendre_synthesis(beta, l, orders=me)  # untimed: the scored orders
    off = oracle.triangle_offsets(l)
    sel = np.concatenate([np.arange(off[m], off[m + 1]) for m in me])
    def score(tag, G, b, lf, bf):
        mf = list(range(0, 2 * lf, err_stride))
        Gf = Ge if bf is None else oracle.legendre_synthesis(bf, lf, orders=mf)
        of = oracle.triangle_offsets(lf)
        sf = np.concatenate([np.arange(of[m], of[m + 1]) for m in mf])
        out["rel_synth_" + tag] = float(np.linalg.norm(G[mf] - Gf[mf]) / np.linalg.norm(Gf[mf]))
        ba = oracle.legendre_analysis(G, lf, orders=mf)
        out["rel_analysis_" + tag] = float(np.linalg.norm(b[sf] - ba[sf]) / np.linalg.norm(ba[sf]))
    names = sorted({k.rsplit("_", 1)[0] for k in d.files})
    for name in names:
        if name.startswith("bt_"):  # one field of the batched leg: bt_<l>_<seed>
            _, lf, sd = name.split("_")
            lf, sd = int(lf), int(sd)
            score("batched_l%d" % lf, d[name + "_G"], d[name + "_beta"], lf,
                  inputs.random_beta(lf, seed=sd, decay=True))
        elif name.startswith("ag_"):  # autograd gradient of field 0: ag_<path>_<l>
            _, pname, lf = name.split("_")
            lf = int(lf)
            gr = d[name + "_grad"]
            mf = list(range(0, 2 * lf, err_stride))
            of = oracle.triangle_offsets(lf)
            sf = np.concatenate([np.arange(of[m], of[m + 1]) for m in mf])
            db = inputs.random_beta(lf, seed=5000, decay=True) - inputs.random_beta(lf, seed=6000, decay=True)
            ref = 2.0 * oracle.legendre_adjoint(oracle.legendre_synthesis(db, lf, orders=mf), lf, orders=mf)
            out["rel_grad_" + pname] = float(np.linalg.norm(gr[sf] - ref[sf]) / np.linalg.norm(ref[sf]))
        else:
            score(name, d[name + "_G"], d[name + "_beta"], l, None)
print(json.dumps(out))
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code, ROOT, str(l), str(stride), str(seed),
                        outputs_path or "-", str(err_stride)],
                       stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError("oracle leg failed: " + r.stderr[-2000:])
    res = json.loads(r.stdout.strip().splitlines()[-1])
    # stratified estimate of the full transform: each call computes the
    # nodes and weights once (t_nodes, timed alone), then its orders; every
    # sampled order stands for the run of stride orders around it
    tn = res["t_nodes"]
    per_order = max(0.0, res["t_synth"] - tn) + max(0.0, res["t_analysis"] - tn)
    res["t_full_est"] = 2 * tn + per_order * (2 * l) / res["orders"]
    return res


def workload_config(args, world=1):
    """The config of the bench line, the same for both arms."""
    return {"workload": f"Legendre stage, one field per GPU: synthesis + analysis at l={args.l} "
                        f"(2l={2 * args.l} GL nodes, orders m=0..{2 * args.l - 1}), FP64 butterfly "
                        f"eps_id={args.eps}, leaf_cols={args.leaf_cols}, beta ~ N(0,1)/(k+1)",
            "l": args.l, "eps_id": args.eps, "parallelism": f"replicas x{world}",
            "l2": "no flush: every launch streams the whole factor stream (6.3 GB at l=1024), "
                  "far larger than the 129 MB L2"}


def cpu_oracle_all_cores(l, seed, nproc):
    """The same float64 oracle over every order of the field, split
    round-robin over nproc single-threaded processes (one per host core);
    returns the wall time of one synthesis plus one analysis of the whole
    field, process start-up included."""
    code = r"""
import sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import oracle
from paper_0910_5435_gb300 import inputs
l, seed, r, n = (int(x) for x in sys.argv[2:6])
ms = list(range(r, 2 * l, n))
beta = inputs.random_beta(l, seed=seed, decay=True)
Go = oracle.legendre_synthesis(beta, l, orders=ms)
oracle.legendre_analysis(Go, l, orders=ms)
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    t0 = time.perf_counter()
    procs = [subprocess.Popen([sys.executable, "-c", code, ROOT, str(l), str(seed), str(r), str(nproc)],
                              stdout=subprocess.DEVNULL, stderr=subprocess.PIPE, env=env) for r in range(nproc)]
    errs = [p.communicate()[1] for p in procs]
    wall = time.perf_counter() - t0
    for p, e in zip(procs, errs):
        if p.returncode != 0:
            raise RuntimeError("oracle leg failed: " + e.decode(errors="replace")[-2000:])
    return wall


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    stride = max(1, min(args.cpu_stride * 8, 2 * args.l))  # at least one order in the sample
    res = None
    for _ in range(args.warmup):
        cpu_oracle_leg(args.l, stride, 3)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        res = cpu_oracle_leg(args.l, stride, 3)
    wall = time.perf_counter() - t0
    value = 2.0 / res["t_full_est"]
    line = {
        "impl": "reference", "metric": METRIC,
        "value": value, "unit": "transforms/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * wall / max(1, args.steps), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(args),
        "cpu_baseline": {"value": value, "unit": "transforms/s", "cores": 1, "kind": "oracle",
                         "sample": f"each step: orders m = {stride // 2}, {stride // 2 + stride}, ... of l={args.l} "
                                   "(synthesis + analysis), the middle of every run of "
                                   f"{stride} orders; the per-order time scaled to all 2l orders, "
                                   "the nodes and weights (computed once per call) timed alone and added once"},
        "e2e": {"value": value, "unit": "transforms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": wall,
    }
    print(json.dumps(line), flush=True)


def batched_leg(args, sht, inputs, torch, dev, stream, plan, rank=0, world=1, dist=None):
    """Many fields of mixed bandlimits (l drawn uniformly from 64..1024, seed
    4; beta ~ N(0,1)/(k+1), seed 1000 + f) through one batched launch per
    direction, split float32, launch shape autotuned, replayed from a CUDA
    graph; against a loop of per-field launches on the same buffers.  With
    several ranks the fields are sharded (shard_fields) and the times are the
    slowest rank's: the total work is fixed (strong scaling)."""
    all_ls = [int(x) for x in np.random.default_rng(4).choice([64, 128, 256, 512, 1024], size=args.batch_fields)]
    mine = shard_fields(all_ls, rank, world)
    ls = [all_ls[f] for f in mine]
    def run_local():
        plans = {}
        t0 = time.perf_counter()
        for l in sorted(set(ls)):
            plans[l] = plan if l == args.l else sht.Plan(l, args.eps, leaf_cols=args.leaf_cols, page_bytes=args.page_bytes,
                                                         consumer_warps=args.consumer_warps)
            plans[l].prepare(sht.SHT_SPLIT32)
        t_plans = time.perf_counter() - t0
        betas = [torch.from_numpy(inputs.random_beta(all_ls[f], seed=1000 + f, decay=True)).to(dev) for f in mine]
        Gs = [torch.empty((2 * l, 2 * l), dtype=torch.complex128, device=dev) for l in ls]
        backs = [torch.empty_like(b) for b in betas]
        B = sht.Batch([plans[l] for l in ls], sht.SHT_SPLIT32)
        bp, gp, kp = sht.pointer_array(betas), sht.pointer_array(Gs), sht.pointer_array(backs)
        cfg_syn = sht.sht_batch_autotune(B, 0, bp, gp, reps=2, stream=stream)
        cfg_ana = sht.sht_batch_autotune(B, 1, gp, kp, reps=2, stream=stream)
        graph = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream(dev)
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            with torch.cuda.graph(graph, stream=side):
                sht.sht_batch_synthesize(B, bp, gp, side)
                sht.sht_batch_analyze(B, gp, kp, side)
        torch.cuda.synchronize()

        def timed(fn, steps):
            for _ in range(2):
                fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / steps

        steps = max(3, args.steps // 2)
        ms_batch = timed(graph.replay, steps)
        status = sht.sht_batch_last_device_status(B, stream)
        Gb = [g.clone() for g in Gs]
        kb = [k.clone() for k in backs]

        def loop():
            for l, b, g in zip(ls, betas, Gs):
                sht.sht_legendre_synthesize(plans[l], sht.SHT_SPLIT32, b, g, stream)
            for l, g, k in zip(ls, Gs, backs):
                sht.sht_legendre_analyze(plans[l], sht.SHT_SPLIT32, g, k, stream)

        ms_loop = timed(loop, steps)
        same = all(torch.equal(a, b) for a, b in zip(Gb, Gs)) and all(torch.equal(a, b) for a, b in zip(kb, backs))
        eps_inv = max(float(torch.linalg.vector_norm(k - b) / torch.linalg.vector_norm(b)) for k, b in zip(kb, betas))
        first = {}
        for i, f in enumerate(mine):
            first.setdefault(all_ls[f], (i, f))
        for lf, (i, f) in first.items():
            samples[f"bt_{lf}_{1000 + f}_G"] = Gb[i].cpu().numpy()
            samples[f"bt_{lf}_{1000 + f}_beta"] = kb[i].cpu().numpy()
        groups = [B.groups(0), B.groups(1)]
        B.close()
        return ms_batch, ms_loop, eps_inv, same, status, cfg_syn, cfg_ana, t_plans, groups

    samples = {}
    if ls:
        ms_batch, ms_loop, eps_inv, same, status, cfg_syn, cfg_ana, t_plans, groups = run_local()
    else:  # more ranks than fields: this rank has nothing to do
        ms_batch, ms_loop, eps_inv, same, status, cfg_syn, cfg_ana, t_plans, groups = (
            0.0, 0.0, 0.0, True, 0, None, None, 0.0, None)
    ms_batch = max_over_ranks(ms_batch, world, dist, dev)
    ms_loop = max_over_ranks(ms_loop, world, dist, dev)
    eps_inv = max_over_ranks(eps_inv, world, dist, dev)
    same = max_over_ranks(0.0 if same else 1.0, world, dist, dev) == 0.0
    ls = all_ls
    return {
        "fields": len(ls), "ranks": world, "l_counts": {str(l): ls.count(l) for l in sorted(set(ls))},
        "field_transforms_per_s": 2.0 * len(ls) / (ms_batch / 1e3),
        "ms_batch_synthesis_plus_analysis": ms_batch, "ms_per_field_loop": ms_loop,
        "speedup_vs_loop": ms_loop / ms_batch, "batch_equals_loop": same, "max_eps_inv": eps_inv,
        "device_status": status, "autotuned": {"synthesis": cfg_syn, "analysis": cfg_ana},
        "launches": {"batched": 2, "loop": 2 * len(ls)}, "cuda_graph": True, "t_plans_s": t_plans,
        "field_groups": groups, "_samples": samples,
    }


def full_sht_leg(args, sht, inputs, torch, dev, stream, plan, beta, back):
    """The whole transform to and from the real grid ([2l][4l-1]: the float64
    butterfly Legendre stage with the phase fused into its unfold / fold,
    plus the length-(4l-1) cuFFT per node), and the phi stage alone."""
    l = args.l
    ws = torch.empty(sht.sht_workspace_bytes(plan, sht.SHT_FP64) // 8 + 1, dtype=torch.float64, device=dev)
    values = torch.empty((2 * l, 4 * l - 1), dtype=torch.float64, device=dev)
    G = torch.empty((2 * l, 2 * l), dtype=torch.complex128, device=dev)

    def timed(fn, steps):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    steps = max(3, args.steps // 2)
    ms_syn = timed(lambda: sht.sht_synthesize(plan, sht.SHT_FP64, beta, values, ws, stream), steps)
    ms_ana = timed(lambda: sht.sht_analyze(plan, sht.SHT_FP64, values, back, ws, stream), steps)
    sht.sht_legendre_synthesize(plan, sht.SHT_FP64, beta, G, stream)
    ms_phi_syn = timed(lambda: sht.sht_phi_synthesize(plan, sht.SHT_FP64, G, values, ws, stream), steps)
    ms_phi_ana = timed(lambda: sht.sht_phi_analyze(plan, sht.SHT_FP64, values, G, stream), steps)
    sht.sht_synthesize(plan, sht.SHT_FP64, beta, values, ws, stream)
    sht.sht_analyze(plan, sht.SHT_FP64, values, back, ws, stream)
    torch.cuda.synchronize()
    eps = float(torch.linalg.vector_norm(back - beta) / torch.linalg.vector_norm(beta))
    return {"grid": [2 * l, 4 * l - 1], "transforms_per_s": 2.0 / ((ms_syn + ms_ana) / 1e3),
            "ms_synthesis": ms_syn, "ms_analysis": ms_ana, "ms_phi_synthesis": ms_phi_syn,
            "ms_phi_analysis": ms_phi_ana, "eps_inv": eps,
            "device_status": sht.sht_last_device_status(plan, stream)}


def autograd_leg(args, sht, inputs, torch, dev, stream):
    """Differentiable Legendre stage: l = 512, a batch of 16 fields, loss
    ||synthesize(beta) - g||^2 with g the synthesis of an independent
    band-limited beta_g (seeds 5000 + f and 6000 + f); forward plus the
    hand-written backward (the transposed butterfly) timed for the float64
    and split float32 paths.  The gradient of field 0 is scored against the
    oracle's 2 S^T S (beta_5000 - beta_6000) on sampled orders (cpu leg)."""
    from paper_0910_5435_gb300 import autograd as ag
    l, nb = 512, 16
    P = sht.Plan(l, args.eps, leaf_cols=args.leaf_cols, page_bytes=args.page_bytes,
                 consumer_warps=args.consumer_warps)
    beta0 = torch.from_numpy(np.stack([inputs.random_beta(l, seed=5000 + f, decay=True) for f in range(nb)])).to(dev)
    beta_g = torch.from_numpy(np.stack([inputs.random_beta(l, seed=6000 + f, decay=True) for f in range(nb)])).to(dev)
    out = {"l": l, "batch": nb}
    grads = {}
    for name, prec in (("fp64", sht.SHT_FP64), ("split32", sht.SHT_SPLIT32)):
        P.prepare(prec)
        g = ag.legendre_synthesis(beta_g, P, prec).detach()

        def step():
            beta = beta0.clone().requires_grad_()
            loss = (ag.legendre_synthesis(beta, P, prec) - g).abs().pow(2).sum()
            loss.backward()
            return beta.grad

        for _ in range(2):
            step()
        torch.cuda.synchronize()
        steps = max(3, args.steps // 2)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            gr = step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        grads[name] = gr
        out[name] = {"ms_forward_backward": ms, "field_fwd_bwd_per_s": nb / (ms / 1e3)}
    out["rel_grad_split32_vs_fp64"] = float(torch.linalg.vector_norm(grads["split32"] - grads["fp64"])
                                            / torch.linalg.vector_norm(grads["fp64"]))
    out["_samples"] = {f"ag_{name}_{l}_grad": gr[0].cpu().numpy() for name, gr in grads.items()}
    P.close()
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__
    __graft_entry__.build()
    from paper_0910_5435_gb300 import inputs, sht

    l = args.l
    t0 = time.perf_counter()
    plan = sht.Plan(l, args.eps, leaf_cols=args.leaf_cols, page_bytes=args.page_bytes,
                    consumer_warps=args.consumer_warps)
    t_plan = time.perf_counter() - t0
    st = plan.stats()

    beta_h = inputs.random_beta(l, seed=3 + rank, decay=True)
    beta = torch.from_numpy(beta_h).to(dev)
    G = torch.empty((2 * l, 2 * l), dtype=torch.complex128, device=dev)
    back = torch.empty_like(beta)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            dist.barrier()

    pct = {}

    def time_path(prec, steps, warmup, b, g, bk, synth_fn=None, ana_fn=None):
        synth_fn = synth_fn or (lambda: sht.sht_legendre_synthesize(plan, prec, b, g, stream))
        ana_fn = ana_fn or (lambda: sht.sht_legendre_analyze(plan, prec, g, bk, stream))
        for _ in range(warmup):
            synth_fn()
            ana_fn()
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        start.record(stream)
        for i in range(steps):
            ev[i][0].record(stream)
            synth_fn()
            ev[i][1].record(stream)
            ana_fn()
            ev[i][2].record(stream)
        end.record(stream)
        torch.cuda.synchronize()
        barrier()
        total = start.elapsed_time(end)
        ts = [e[0].elapsed_time(e[1]) for e in ev]
        ta = [e[1].elapsed_time(e[2]) for e in ev]
        pct.update({"synthesis_ms_p10_p50_p90": [float(np.percentile(ts, q)) for q in (10, 50, 90)],
                    "analysis_ms_p10_p50_p90": [float(np.percentile(ta, q)) for q in (10, 50, 90)]})
        return total, float(np.mean(ts)), float(np.mean(ta))

    # ---- headline: float64 butterfly
    clocks = ClockSampler(local)
    for _ in range(args.warmup):
        sht.sht_legendre_synthesize(plan, sht.SHT_FP64, beta, G, stream)
        sht.sht_legendre_analyze(plan, sht.SHT_FP64, G, back, stream)
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    total_ms, ms_syn, ms_ana = time_path(sht.SHT_FP64, args.steps, 0, beta, G, back)
    step_percentiles = dict(pct)
    clk = clocks.stop()
    status = sht.sht_last_device_status(plan, stream)
    total_ms = max_over_ranks(total_ms, world, dist, dev)
    value = world * 2.0 * args.steps / (total_ms / 1e3)
    ms_per_step = total_ms / args.steps
    eps_inv64 = float(torch.linalg.vector_norm(back - beta) / torch.linalg.vector_norm(beta))
    G64 = G.cpu().numpy()
    back64 = back.cpu().numpy()

    # ---- end to end through the C ABI with pinned host buffers
    beta_pin = torch.from_numpy(beta_h).pin_memory()
    out_pin = torch.empty_like(beta_pin).pin_memory()

    def e2e_step():
        beta.copy_(beta_pin, non_blocking=True)
        sht.sht_legendre_synthesize(plan, sht.SHT_FP64, beta, G, stream)
        sht.sht_legendre_analyze(plan, sht.SHT_FP64, G, back, stream)
        out_pin.copy_(back, non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), world, dist, dev)
    e2e_value = world * 2.0 * args.steps / (e2e_ms / 1e3)
    nbytes = beta.numel() * beta.element_size()

    # ---- roofline of the dominant kernel (the float64 sweep)
    flops = 4.0 * st["factor_values"]  # 2 real right-hand sides x (mul + add) per stored value
    achieved = flops / (0.5 * (ms_syn + ms_ana) / 1e3) / 1e12
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs") if peaks else None
    stream_gbs = st["stream_bytes_fp64"] / (0.5 * (ms_syn + ms_ana) / 1e3) / 1e9
    traffic = None
    cap = SWEEP_TRAFFIC_CAPTURE
    if (cap["sources_sha"] is not None and sweep_sources_sha() == cap["sources_sha"]
            and args.leaf_cols == cap["leaf_cols"] and args.page_bytes == cap["page_bytes"]):
        traffic = 0.5 * (cap["dram_bytes_syn"] + cap["dram_bytes_ana"]) / cap["stream_bytes"] * st["stream_bytes_fp64"]
    # this device's float64 FMA loop (after the timed region): the reachable ceiling
    dfma_loop = sht.measure_fp64_fma()
    # and its float64 tensor-core (warp MMA) loop: whether block GEMMs over
    # several right-hand sides could beat the FMA pipe on this part
    dmma_loop = sht.measure_fp64_mma()
    roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic,
                "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum at l=512, "
                                "scaled by the float64 stream size)",
                "algorithmic_bytes_per_launch": st["stream_bytes_fp64"] + nbytes + G.numel() * G.element_size(),
                "kernel": "bfly_sweep_kernel<TF64>",
                "peak_source": "derived: 2 DFMA/clk/SM x 152 SMs x 2.07 GHz x 2 flops",
                "dfma_loop_tflops": dfma_loop,
                "frac_of_dfma_loop": achieved / dfma_loop if dfma_loop > 0 else None,
                "dmma_loop_tflops": dmma_loop,
                "hbm_view": {"stream_bytes_per_launch": st["stream_bytes_fp64"], "achieved_gbs": stream_gbs,
                             "peak_gbs": hbm or HBM_FALLBACK_GBS,
                             "frac": stream_gbs / (hbm or HBM_FALLBACK_GBS),
                             "peak_source": "measured" if hbm else "fallback"}}

    extras = {}
    legs = set() if args.no_extras else {s.strip() for s in args.paths.split(",") if s.strip()}
    if rank == 0:
        for name, prec, cdt in (("split32", sht.SHT_SPLIT32, torch.complex128),
                                ("split32acc64", sht.SHT_SPLIT32_ACC64, torch.complex128),
                                ("fp32", sht.SHT_FP32, torch.complex64)):
            if name not in legs:
                continue
            t0 = time.perf_counter()
            plan.prepare(prec)
            tprep = time.perf_counter() - t0
            b = beta.to(cdt)
            g = torch.empty((2 * l, 2 * l), dtype=cdt, device=dev)
            bk = torch.empty_like(b)
            tot, s_ms, a_ms = time_path(prec, args.steps, 2, b, g, bk)
            st2 = plan.stats()
            sb = st2["stream_bytes_fp32" if name == "fp32" else "stream_bytes_split32"]
            extras[name] = {
                "transforms_per_s": 2.0 * args.steps / (tot / 1e3), "ms_synthesis": s_ms, "ms_analysis": a_ms,
                "stream_bytes": sb, "achieved_gbs": sb / (0.5 * (s_ms + a_ms) / 1e3) / 1e9,
                "hbm_frac": sb / (0.5 * (s_ms + a_ms) / 1e3) / 1e9 / (hbm or HBM_FALLBACK_GBS),
                "eps_inv": float(torch.linalg.vector_norm((bk - b).to(torch.complex128))
                                 / torch.linalg.vector_norm(b.to(torch.complex128))),
                "prepare_s": tprep,
            }
            extras[name + "_G"] = g.to(torch.complex128).cpu().numpy()
            extras[name + "_beta"] = bk.to(torch.complex128).cpu().numpy()
    if rank == 0 and "direct" in legs:
        # direct float64 baseline (dense operator in HBM)
        t0 = time.perf_counter()
        sht.sht_direct_prepare(plan)
        tprep = time.perf_counter() - t0
        g = torch.empty_like(G)
        bk = torch.empty_like(beta)
        tot, s_ms, a_ms = time_path(
            None, max(2, args.steps // 2), 1, beta, g, bk,
            synth_fn=lambda: sht.sht_direct_synthesize(plan, beta, g, stream),
            ana_fn=lambda: sht.sht_direct_analyze(plan, g, bk, stream))
        extras["direct_fp64"] = {
            "transforms_per_s": 2.0 * max(2, args.steps // 2) / (tot / 1e3), "ms_synthesis": s_ms,
            "ms_analysis": a_ms, "prepare_s": tprep,
            "eps_inv": float(torch.linalg.vector_norm(bk - beta) / torch.linalg.vector_norm(beta)),
        }
        extras["direct_G"] = g.cpu().numpy()
        extras["direct_beta"] = bk.cpu().numpy()

    if rank == 0 and "full" in legs:
        extras["full_sht_fp64"] = full_sht_leg(args, sht, inputs, torch, dev, stream, plan, beta, back)
    if "batched" in legs and args.batch_fields > 0:
        extras["batched_split32"] = batched_leg(args, sht, inputs, torch, dev, stream, plan, rank, world, dist)
    if rank == 0 and "autograd" in legs:
        extras["autograd_l512_b16"] = autograd_leg(args, sht, inputs, torch, dev, stream)
    if rank == 0 and "gauss_jacobi" in legs:
        extras["gauss_jacobi_m_eq_n"] = gauss_jacobi_leg(args, sht, torch, dev, stream)
    if rank == 0 and "device_build" in legs:
        extras["plan_device_build"] = device_build_leg(args, sht, torch, dev, stream, plan, st, beta)
    if rank == 0 and "trace" in legs:
        extras["sweep_trace"] = trace_leg(args, sht, torch, dev, stream, plan, beta)

    cpu = None
    cpu_all = None
    rel = {}
    if rank == 0 and world == 1 and not args.no_cpu:
        with tempfile.TemporaryDirectory() as td:
            op = os.path.join(td, "outputs.npz")
            arrays = {"fp64_G": G64, "fp64_beta": back64}
            for k in ("split32", "split32acc64", "fp32", "direct"):
                if k + "_G" in extras:
                    arrays[k + "_G"] = extras[k + "_G"]
                    arrays[k + "_beta"] = extras[k + "_beta"]
            for leg in extras.values():
                if isinstance(leg, dict):
                    arrays.update(leg.get("_samples", {}))
            np.savez(op, **arrays)
            res = cpu_oracle_leg(l, args.cpu_stride, 3, op)
        cpu = {"value": 2.0 / res["t_full_est"], "unit": "transforms/s", "cores": 1, "kind": "oracle",
               "sample": f"{res['orders']} of {2 * l} orders (m = {args.cpu_stride // 2}, "
                         f"{args.cpu_stride // 2 + args.cpu_stride}, ...), synthesis + analysis, "
                         f"scaled by the stride; {res['t_synth'] + res['t_analysis']:.1f} s of CPU"}
        rel = {k: v for k, v in res.items() if k.startswith("rel_")}
        if args.cpu_all_cores:
            ncores = os.cpu_count() or 1
            wall = cpu_oracle_all_cores(l, 3, ncores)
            cpu_all = {"value": 2.0 / wall, "unit": "transforms/s", "cores": ncores, "kind": "oracle",
                       "sample": f"all {2 * l} orders, synthesis + analysis, one single-threaded process "
                                 f"per core; {wall:.1f} s wall including process start-up"}
    for k in list(extras):
        if k.endswith("_G") or k.endswith("_beta"):
            extras.pop(k)
    for leg in extras.values():
        if isinstance(leg, dict):
            leg.pop("_samples", None)
    # each leg carries its own scores against the oracle
    rel_main = {k: v for k, v in rel.items() if "batched_l" not in k and not k.startswith("rel_grad_")}
    if "batched_split32" in extras and rel:
        extras["batched_split32"]["rel_l2_vs_oracle_sampled"] = {
            k: v for k, v in rel.items() if "batched_l" in k}
    if "autograd_l512_b16" in extras and rel:
        extras["autograd_l512_b16"]["rel_l2_vs_oracle_sampled"] = {
            k: v for k, v in rel.items() if k.startswith("rel_grad_")}

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": value, "unit": "transforms/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, world),
            "ms_synthesis": ms_syn, "ms_analysis": ms_ana, "step_ms_percentiles": step_percentiles,
            "eps_inv": eps_inv64, "rel_l2_vs_oracle_sampled": rel_main,
            "roofline": roofline, "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all,
            "e2e": {"value": e2e_value, "unit": "transforms/s", "h2d_bytes_per_step": nbytes,
                    "d2h_bytes_per_step": nbytes},
            "gpu_launches": 2 * args.steps, "clocks": clk, "device_status": status,
            "plan": {"t_plan_s": t_plan, "k_max": st["k_max"], "k_avg": st["k_avg"], "k_sigma": st["k_sigma"],
                     "factor_values": st["factor_values"], "dense_values": st["dense_values"],
                     "rows_kept_frac": st["rows_kept"] / max(1, st["rows_total"]),
                     "levels": st["max_levels"], "t_comp": st["t_comp"], "t_factor": st["t_factor"]},
            "paths": extras,
        }
        if "direct_fp64" in extras:
            line["butterfly_vs_direct_fp64"] = value / extras["direct_fp64"]["transforms_per_s"]
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
