"""Host logic of bench.py on CPU: the multi-rank path with two gloo ranks (no GPU, no data-path
collective; the replicas only agree on the slowest time), the reference arm (rank > 0 doing no
work, rank 0 printing the contract's line), and the roofline traffic taken from the committed ncu
summary."""
import argparse
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        # each replica measured its own step and apply times; the job reports the slowest of each
        got = bench.max_over_ranks([10.0 + rank, 3.0 - rank], world, "cpu")
        out.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0] == res[1] == [11.0, 3.0]


def test_whole_job_value_and_single_rank():
    import bench
    assert bench.max_over_ranks([1.5, 2.5], 1, "cpu") == [1.5, 2.5]
    # 4 replicas of m = 7 matvecs of 1e6 coefficients in 10 ms each: 2.8 Gcoeff/s for the job
    assert bench.whole_job_gcoeff_s(7, 1_000_000, 4, 0.010) == pytest.approx(2.8)


def test_reference_arm_other_ranks_do_nothing():
    import bench
    args = argparse.Namespace(workload="hh2_b32", steps=1, warmup=0, gpus=2)
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args, rank=1)
    assert buf.getvalue() == ""


def test_reference_arm_line(oracle):
    """Rank 0 of the reference arm times the oracle's full matvec and prints one JSON line with the
    contract's keys (on a tiny workload here; the default workload takes seconds per step)."""
    import json
    import bench
    args = argparse.Namespace(workload="hh2_b32", steps=3, warmup=1, gpus=1)
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args, rank=0)
    lines = [x for x in buf.getvalue().splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "Galerkin matvecs: Gcoeff/s" and d["unit"] == "Gcoeff/s"
    assert d["steps"] == 3 and d["warmup"] == 1 and d["higher_is_better"] is True and d["value"] > 0
    assert d["config"]["workload"] == "hh2_b32" and d["config"]["size"] == 119
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "Gcoeff/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["value"] == pytest.approx(119 / (d["ms_per_step"] * 1e-3) / 1e9)


def test_profiled_traffic_tracks_kernel_source(tmp_path, monkeypatch):
    """roofline.traffic comes from the committed ncu summary only while the kernel sources are the
    ones that summary names."""
    import bench
    src = tmp_path / "paper_1403_3511_gb300" / "csrc"
    src.mkdir(parents=True)
    for name in bench.KERNEL_SOURCES:
        (src / name).write_text(name + " v1\n")
    prof = tmp_path / "profiles"
    prof.mkdir()
    h = bench.kernel_source_hash(str(tmp_path))
    (prof / "apply_kernel_w_c64.md").write_text(f"kernel sources sha256 {h}\ntraffic_bytes_per_launch: 1234\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("w", "c64") == 1234
    assert bench.profiled_traffic("w", "c128") is None
    (src / "hx_stencil.cuh").write_text("changed\n")
    assert bench.profiled_traffic("w", "c64") is None


def test_issue_roofline_and_profiled_values(tmp_path, monkeypatch):
    """The product's issue roofline: warp instructions from the committed summary (same source
    check as the traffic) over the launch time, against 4 instructions per SM and cycle."""
    import bench
    src = tmp_path / "paper_1403_3511_gb300" / "csrc"
    src.mkdir(parents=True)
    for name in bench.KERNEL_SOURCES:
        (src / name).write_text(name + " v1\n")
    prof = tmp_path / "profiles"
    prof.mkdir()
    h = bench.kernel_source_hash(str(tmp_path))
    (prof / "apply_kernel_w_c64.md").write_text(
        f"kernel sources sha256 {h}\ntraffic_bytes_per_launch: 1234\nwarp_instructions_per_launch: 608000000\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    w = bench.profiled_value("w", "c64", "apply_kernel", "warp_instructions_per_launch")
    assert w == 608000000
    r = bench.issue_roofline(w, 1.0, 2000.0, 152)
    assert r["peak"] == 152 * 4 * 2000e6
    assert abs(r["achieved"] - 6.08e11) < 1.0 and abs(r["frac"] - 6.08e11 / r["peak"]) < 1e-12
    (src / "hx_jit.cu").write_text("changed\n")
    assert bench.profiled_value("w", "c64", "apply_kernel", "warp_instructions_per_launch") is None


def test_step_bytes_per_coefficient():
    """Algorithmic bytes of one complex64 step at m = 7: start 24, products 7 x 16, sweeps
    8 (4 + 5 + ... + 10) = 392, recombination 7 x 8 + 16 = 72: 600 B per coefficient."""
    import bench
    assert bench.step_bytes_per_coef(7, 8) == 24 + 7 * 16 + 8 * sum(range(4, 11)) + 7 * 8 + 16 == 600
    assert bench.step_bytes_per_coef(1, 8) == 24 + 16 + 8 * 4 + 8 + 16
