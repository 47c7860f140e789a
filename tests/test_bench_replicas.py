"""The multi-GPU bench path (one independent replica per rank) on CPU with gloo, world size 2:
max-over-ranks timing, the whole-job rate, and the reference arm running on rank 0 only."""
import io
import os
import sys
from contextlib import redirect_stdout

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [12.5, 30.25][rank]
        ms = bench.max_over_ranks(local_ms, world, device="cpu")
        rate = bench.job_rate(world, 256**3, 10, ms / 1e3)
        # the reference arm: only rank 0 runs and prints; the others return without work
        buf = io.StringIO()
        args = type("A", (), dict(steps=1, warmup=0, gpus=world, config="cavity32"))()
        called = []
        orig = bench.cpu_oracle_rate
        bench.cpu_oracle_rate = lambda cfg, steps, warmup: (called.append(1) or (1.0e4, 0.5))
        with redirect_stdout(buf):
            bench.run_reference(args, bench.CONFIGS["cavity32"])
        bench.cpu_oracle_rate = orig
        q.put((rank, ms, rate, len(called), buf.getvalue()))
    finally:
        dist.destroy_process_group()


def test_replicas_max_over_ranks_and_job_rate():
    port = 29500 + (os.getpid() % 2000)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res = {r: (ms, rate, called, text) for r, ms, rate, called, text in out}
    for r in (0, 1):
        assert res[r][0] == 30.25  # the slowest rank's time
        assert res[r][1] == pytest.approx(2 * 256**3 * 10 / 30.25e-3)
    assert res[0][2] == 1 and '"impl": "reference"' in res[0][3]
    assert res[1][2] == 0 and res[1][3] == ""


def test_dram_traffic_record_follows_its_source_file(tmp_path, monkeypatch):
    """roofline.traffic comes from the committed small-case ncu record, scaled by the cell count,
    and only while the kernel's source file still hashes to the record's prefix."""
    import hashlib

    import bench

    src = tmp_path / "k.cu"
    src.write_text("kernel source\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    (tmp_path / "profiles").mkdir()
    rec = tmp_path / "profiles" / "dram_traffic_small_case.txt"
    rec.write_text(f"# comment\nk_x    1000    10    k.cu    {sha}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.dram_traffic("k_x", 40) == pytest.approx(4000.0)
    assert bench.dram_traffic("k_other", 40) is None
    src.write_text("kernel source, changed\n")
    assert bench.dram_traffic("k_x", 40) is None
    # the committed record parses; it counts while the sweep kernel's file is the one captured
    monkeypatch.setattr(bench, "ROOT", ROOT)
    t = bench.dram_traffic("k_rbgs_sweep(mac,level0)", 256**3)
    assert t is None or 0.5 * 16 * 256**3 < t < 1.5 * 16 * 256**3


def test_step_byte_model_counts_the_schedule():
    """The whole-step byte model: 24 words per V-cycle of 6 passes, scaled by the passes the
    schedule makes (2 + 2 MAC sweeps and 2 + 1 FE sweeps: 6 and 5 passes)."""
    import bench

    A = type("A", (), dict(mac_sweeps=2, fe_pre=2, fe_post=2, mg_cycles_mac=5, mg_cycles_fe=4))
    assert bench.step_model_words(A()) == pytest.approx(55 + 24 * 9 * 8 / 7)
    A.fe_post = 1
    assert bench.step_model_words(A()) == pytest.approx(55 + 24 * (5 + 4 * 5 / 6) * 8 / 7)
    assert bench.step_model_words(A()) * 4 == pytest.approx(1134.2857, rel=1e-6)
