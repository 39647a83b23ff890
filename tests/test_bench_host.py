"""Host-side checks of bench.py's accounting (CPU only): the algorithmic bytes and FP64 flops
per point-step behind the roofline, the rule that a committed ncu traffic figure is used only
while the kernel source it was taken on is unchanged, and the oracle baseline's report."""

import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402
from paper_2507_23613_gb300 import inputs  # noqa: E402


def test_bytes_and_flops_per_point_step():
    # homogeneous: read W^n, W^{n-1}, q_1..8; write W^{n+1}, q_1..8 (8-byte words)
    assert bench.bytes_per_point_step(8, False) == (3 + 2 * 8) * 8 == 152
    # forced adds the 8 forcing grids
    assert bench.bytes_per_point_step(8, True) == (3 + 3 * 8) * 8 == 216
    # FP64 flops: 3 leapfrog FMAs and 2 neighbour adds in 2D (4 and 3 in 3D); forcing FMAs if
    # forced (the float-pair split and the filter updates are not FP64 work)
    assert bench.flops_per_point_step(8, False) == 8
    assert bench.flops_per_point_step(8, True) == 24
    assert bench.flops_per_point_step(4, False, dim=3) == 11
    # a blocked launch reads and writes both levels and the 8 float-pair sums once, whatever
    # its depth; forced launches read the 8 forcing grids once
    assert bench.blocked_bytes_per_point_launch(8, False) == (4 + 2 * 8) * 8 == 160
    assert bench.blocked_bytes_per_point_launch(8, True) == (4 + 3 * 8) * 8 == 224


def test_traffic_only_for_the_kernel_it_was_taken_on(tmp_path, monkeypatch):
    key = bench.kernel_source_key()
    assert len(key) == 16 and key == bench.kernel_source_key()
    assert len(bench.blocked_kernel_source_key()) == 16 and bench.blocked_kernel_source_key() != key
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "k.txt").write_text("# comment: 1\nsource_sha256: %s\ndram_bytes_per_launch: 123.5\n"
                                % key)
    (prof / "old.txt").write_text("source_sha256: 0000000000000000\ndram_bytes_per_launch: 9\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_traffic("k.txt", key) == 123.5
    assert bench.kernel_traffic("old.txt", key) is None
    assert bench.kernel_traffic("missing.txt", key) is None


def test_committed_fp64_blocked_profile_matches_its_kernel():
    """The FP64 pipelined blocked kernel's ncu summary carries the hash of the source it was
    taken on (bench.py uses its DRAM bytes only while that holds)."""
    assert bench.kernel_traffic("k_tb2d_pipe_square1025_nf8.txt",
                                bench.blocked_kernel_source_key()) is not None


def test_committed_fp32_profile_matches_its_kernel():
    """The FP32 blocked kernel's ncu summary carries the hash of the source it was taken on."""
    assert bench.kernel_traffic("k_tb2d32_square1025_nf8.txt", bench.fp32_kernel_source_key()) \
        is not None


def test_cpu_baseline_report():
    info = bench.cpu_baseline(("square_small", {}), budget_s=0.2, workers=1)
    assert info["kind"] == "oracle" and info["cores"] == 1 and info["unit"] == "Gpts/s"
    assert info["value"] > 0 and "65x65" in info["sample"]


def test_cpu_baseline_on_several_cores():
    """Two spawned processes time the same sample together; the rate counts both."""
    rig = bench.OracleRig(("square_small", {}), budget_s=0.2, workers=2)
    try:
        one = rig.run()
        two = rig.run()
    finally:
        rig.close()
    assert one["cores"] == 2 and two["cores"] == 2 and "2 process(es)" in one["sample"]
    assert one["value"] > 0 and two["value"] > 0


@pytest.mark.parametrize("argv,flag", [(["--small"], "small"),
                                       (["--implicit-scaling", "--cube"], "implicit_scaling"),
                                       (["--impl", "reference", "--oracle-timings"],
                                        "oracle_timings")])
def test_modes_parse(argv, flag, monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"] + argv)
    args = bench.parse()
    assert getattr(args, flag)
    assert args.steps == 3 and args.warmup == 3 and args.gpus == 1


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` (the oracle timed on the host) prints one JSON line with
    the keys the benchmark contract asks for."""
    import json
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                       timeout=300, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["higher_is_better"] is True and d["n_gpus"] == 1
    assert d["value"] > 0 and d["unit"] == "Gpts/s" and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["config"]["workload"].startswith("square1025x1025_nf8")


def test_reference_arm_under_torchrun_prints_once():
    """Launched as the benchmark contract launches N > 1 runs (torch.distributed.run, two
    ranks, rendezvous on 127.0.0.1), the reference arm runs on rank 0 alone and prints one
    line; the other rank exits 0 without work."""
    import json
    import socket
    import subprocess
    pytest.importorskip("torch")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                        "--nproc-per-node", "2", "--master-addr", "127.0.0.1",
                        "--master-port", str(port), os.path.join(root, "bench.py"),
                        "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
