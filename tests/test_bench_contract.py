"""bench.py's reference arm (the FP64 oracle on host cores) keeps the benchmark's JSON
contract, alone and under torchrun with two ranks (rank 0 alone works and prints; the other
rank exits 0).  CPU only: a tiny oracle sample stands in for the timed one."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ARGS = ["--impl", "reference", "--steps", "1", "--warmup", "0", "--cpu-sample-M", "128"]


def _json_lines(out):
    return [json.loads(l) for l in out.splitlines() if l.strip().startswith("{")]


def _check_line(line, n_gpus):
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference"
    assert line["n_gpus"] == n_gpus and line["steps"] == 1 and line["warmup"] == 0
    assert line["higher_is_better"] is False and line["unit"] == "s"
    assert line["value"] > 0 and abs(line["ms_per_step"] - 1e3 * line["value"]) <= 1e-9 * line["ms_per_step"]
    assert "workload" in line["config"] and line["config"]["M"] == 32768
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and "128" in cb["sample"]
    # the M = 32768 figure is a c M^3 fit of the timed samples, and says so
    assert line["extrapolated"] is True and cb["extrapolated"] is True and line["config"]["sampled_M"] == [128]
    assert abs(cb["c_s_per_M3"] * 32768.0 ** 3 - line["value"]) <= 1e-9 * line["value"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_single_process():
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "bench.py"] + ARGS, cwd=ROOT, capture_output=True, text=True,
                       timeout=300, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    _check_line(lines[0], 1)


def test_reference_arm_under_torchrun_two_ranks():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--gpus", "2"] + ARGS
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    _check_line(lines[0], 2)


def _bench_module():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    return bench


def test_stage_rooflines_counts_the_method_not_the_gpu_path():
    """The per-stage roofline block uses the method's algorithmic flop counts: the two-stage
    back-transformation is 4 M^3 (2 M^3 for 1-stage), the lowest-n route shrinks S3 and R3 by
    n / M, the Cholesky-free reducer's stages are named for Eq. 7-9, and every rate is those
    flops over the stage time (36 plane products per FP64-equivalent flop for the BF16 ratio)."""
    b = _bench_module()
    M = 1000
    m3 = float(M) ** 3
    stages = [1.0, 2.0, 4.0, 3.0, 5.0, 1.0, 0.0]
    f64 = {"fp64_dgemm_tflops_sustained": 1.0}
    full = b.stage_rooflines(M, stages, [3.0, 1.0], True, "2stage", 64, 1000.0, f64)
    assert full["stages"]["S3_back_q"]["alg_flops"] == 4.0 * m3
    assert full["stages"]["R3_backsub"]["alg_flops"] == m3
    r1 = full["stages"]["R1_cholesky"]
    assert abs(r1["fp64_equiv_tflops"] - (m3 / 3) / 1e-3 / 1e12) < 1e-12
    assert abs(r1["frac_of_bf16_sustained_36_planes"] - r1["fp64_equiv_tflops"] * 36 / 1000.0) < 1e-12
    one = b.stage_rooflines(M, stages, None, True, "1stage", 0, 1000.0, f64)
    assert one["stages"]["S3_back_q"]["alg_flops"] == 2.0 * m3
    half = b.stage_rooflines(M, stages, [3.0, 1.0], True, "2stage", 64, 1000.0, f64, n=M // 2)
    assert half["stages"]["S3_back_q"]["alg_flops"] == 2.0 * m3
    assert half["stages"]["R3_backsub"]["alg_flops"] == 0.5 * m3
    ee = b.stage_rooflines(M, stages, [3.0, 1.0], True, "2stage", 64, 1000.0, f64, reducer="eigenexa")
    assert set(ee["stages"]) >= {"E7_sep_of_B", "E8_A_prime", "E9_Y_is_XZ", "S3_back_q"}
    assert ee["stages"]["E8_A_prime"]["alg_flops"] == 3.0 * m3
    vals = b.stage_rooflines(M, stages, [3.0, 1.0], False, "2stage", 64, 1000.0, f64)
    assert "S3_back_q" not in vals["stages"] and "R3_backsub" not in vals["stages"]


def test_cm3_fit_recovers_a_cubic_law():
    b = _bench_module()
    samples = [(m, 2e-9 * m ** 3) for m in (100, 200, 300)]
    v, c = b.cm3_fit(samples, 1000)
    assert abs(c - 2e-9) < 1e-18 and abs(v - 2.0) < 1e-9
