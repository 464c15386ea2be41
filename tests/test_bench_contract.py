"""The reference arm of bench.py (the float64 oracle timed on the host) runs
on the CPU: its one JSON line carries the keys of the bench contract, with
the same metric and config as the GPU arm."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--l", "64",
                        "--steps", "1", "--warmup", "1", "--cpu-stride", "4"],
                       stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    sys.path.insert(0, ROOT)
    import bench
    assert d["metric"] == bench.METRIC
    assert d["config"]["l"] == 64 and "workload" in d["config"] and "l2" in d["config"]


def test_reference_arm_under_torchrun_prints_once():
    """Launched as the multi-GPU bench is (one process per rank), the
    reference arm runs on rank 0 alone: one JSON line, every rank exits 0."""
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(port),
                        os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "1", "--cpu-stride", "512"],
                       stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0


def test_oracle_leg_scores_outputs_against_the_oracle(tmp_path):
    """The CPU leg that times the oracle also scores a path's outputs: given
    the oracle's own synthesis and analysis as that path's outputs, both
    errors are at rounding level, and the timing sample has one order per
    stride."""
    sys.path.insert(0, ROOT)
    import numpy as np

    import bench
    import oracle
    from paper_0910_5435_gb300 import inputs
    l = 16
    beta = inputs.random_beta(l, seed=3, decay=True)
    G = oracle.legendre_synthesis(beta, l)
    path = str(tmp_path / "outs.npz")
    np.savez(path, fp64_G=G, fp64_beta=oracle.legendre_analysis(G, l))
    res = bench.cpu_oracle_leg(l, 4, 3, path, err_stride=3)
    assert res["orders"] == 2 * l // 4
    assert res["rel_synth_fp64"] < 1e-15 and res["rel_analysis_fp64"] < 1e-15
    assert res["t_full_est"] > 0


def test_oracle_leg_scores_batched_fields_and_gradients(tmp_path):
    """The batched and autograd legs' samples are scored too: a field of the
    batch at the headline's own bandlimit and one at another, and the
    gradient 2 S^T S (beta_5000 - beta_6000) of field 0.  Exact oracle
    outputs score at rounding level, a planted error in one node row of one
    field shows in that field's score only."""
    sys.path.insert(0, ROOT)
    import numpy as np

    import bench
    import oracle
    from paper_0910_5435_gb300 import inputs
    l = 16
    beta = inputs.random_beta(l, seed=3, decay=True)
    G = oracle.legendre_synthesis(beta, l)
    arrays = {"fp64_G": G, "fp64_beta": oracle.legendre_analysis(G, l)}
    for lf, seed in ((16, 1004), (8, 1007)):
        bf = inputs.random_beta(lf, seed=seed, decay=True)
        Gf = oracle.legendre_synthesis(bf, lf)
        if lf == 8:
            Gf[2] *= 1.01  # planted: one order's node row off by 1 %
        arrays[f"bt_{lf}_{seed}_G"] = Gf
        arrays[f"bt_{lf}_{seed}_beta"] = oracle.legendre_analysis(Gf, lf)
    db = inputs.random_beta(8, seed=5000, decay=True) - inputs.random_beta(8, seed=6000, decay=True)
    arrays["ag_fp64_8_grad"] = 2 * oracle.legendre_adjoint(oracle.legendre_synthesis(db, 8), 8)
    path = str(tmp_path / "outs.npz")
    np.savez(path, **arrays)
    res = bench.cpu_oracle_leg(l, 4, 3, path, err_stride=1)
    assert res["rel_synth_fp64"] < 1e-15
    assert res["rel_synth_batched_l16"] < 1e-15 and res["rel_analysis_batched_l16"] < 1e-15
    assert res["rel_synth_batched_l8"] > 1e-4 and res["rel_analysis_batched_l8"] < 1e-15
    assert res["rel_grad_fp64"] < 1e-15
