"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

Replicas share no data-path collective; the only exchange is the max of the timed
region over ranks, and the whole-job rate is every rank's frames over that max.
"""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    try:
        got = bench.max_over_ranks(10.0 * (rank + 1))
        env = bench.dist_env()
        # the reference arm runs on rank 0 alone: other ranks return without output
        out = io.StringIO()
        if rank != 0:
            with redirect_stdout(out):
                bench.run_reference(None)
        dist.barrier()
        q.put((rank, got, env, out.getvalue()))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [20.0, 20.0]  # both ranks see the slowest rank's time
    assert [r[2] for r in res] == [(0, 2, 0), (1, 2, 1)]
    assert res[1][3] == ""


def test_whole_job_rate_and_single_rank():
    import bench
    # 2 replicas x 100 frames, slowest rank 50 ms -> 4000 frames/s for the whole job
    assert bench.whole_job_rate(2, 100, 50.0) == pytest.approx(4000.0)
    assert bench.whole_job_rate(1, 100, 50.0) == pytest.approx(2000.0)
    if not dist.is_initialized():
        assert bench.max_over_ranks(3.5) == 3.5


def test_frame_algorithmic_bytes():
    import bench
    T, V, W, H, Tv, C = 4096000, 2048400, 1920, 1080, 262158, 36112
    edge = bench.frame_algorithmic_bytes(T, V, W, H, Tv, C, 0)
    vert = bench.frame_algorithmic_bytes(T, V, W, H, Tv, C, 1)
    assert edge - vert == 12 * T  # adjacency is read in edge mode only
    assert 0.15e9 < edge < 0.21e9


def test_every_frame_kernel_has_compulsory_bytes():
    import bench
    T, V, W, H, Tv, C = 4096000, 2048400, 1920, 1080, 262158, 36112
    work = {"survivors": 509772, "clip_records": 0, "big_entries": 9483, "big_tiles": 15205,
            "visible_tiles": 811}
    kernels = [k for ks in bench.STAGES.values() for k in ks]
    assert len(kernels) == len(set(kernels)) == 16  # the 15 of a frame, and the tile-depth pass
    for k in kernels:
        b = bench.algorithmic_bytes(k, T, V, W, H, Tv, C, work)
        assert b is not None and b > 0, k
    # the front end reads the mesh once and clears the per-frame buffers
    assert bench.algorithmic_bytes("k_raster_front", T, V, W, H, Tv, C, work) == \
        12 * T + 12 * V + 4 * W * H + (T + 31) // 32 * 4 + 4 * T


def test_host_info():
    import bench
    h = bench.host_info()
    assert h["nproc"] >= 1 and isinstance(h["cpu"], str)


def test_reference_arm_line():
    """The reference arm times the oracle on the host and prints one contract line
    (small scene here: 10 spheres, 204,800 triangles)."""
    import json
    import subprocess
    import bench
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1", "--spheres", "10"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "frames/s"
    assert d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["config"]["workload"].startswith("icospheres10_") and d["config"]["triangles"] == 10 * 20480
    assert d["value"] > 0 and d["ms_per_step"] == pytest.approx(1e3 / d["value"])
    cb, e2e = d["cpu_baseline"], d["e2e"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and cb["sample"]
    assert e2e == {"value": d["value"], "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_traffic_table_round_trip(tmp_path, monkeypatch):
    """bench.py --write-traffic: every per-frame kernel has a source file; the table
    written from an ncu CSV log (thousands separators, scaled units, other metrics)
    is read back for the workload it was captured on while the sources are unchanged."""
    import bench
    for k in [k for ks in bench.STAGES.values() for k in ks]:
        assert bench.kernel_source(k) is not None, k
    log = tmp_path / "traffic.csv"
    hdr = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size",'
           '"Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"')
    rows = [("0", "void fa::(anonymous namespace)::k_raster_front<false>(RasterArgs)", "dram__bytes_read.sum",
             "byte", "73,751,296"),
            ("0", "void fa::(anonymous namespace)::k_raster_front<false>(RasterArgs)", "dram__bytes_write.sum",
             "Mbyte", "26.0"),
            ("1", "k_uv<false>", "gpu__time_duration.sum", "usecond", "18.5"),
            ("1", "k_uv<false>", "dram__bytes_read.sum", "Kbyte", "1,500")]
    body = "\n".join(",".join(f'"{x}"' for x in (i, "1", "python", "h", k, "1", "7", "(1,1,1)", "(1,1,1)", "0",
                                                  "10.3", "s", m, u, v)) for i, k, m, u, v in rows)
    log.write_text("==PROF== Connected\n" + hdr + "\n" + body + "\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "profiles").mkdir()
    real = __import__("os").path.dirname(bench.__file__)
    (tmp_path / "paper_2502_17712_gb300").symlink_to(__import__("os").path.join(real, "paper_2502_17712_gb300"))
    bench.write_traffic(str(log), "frame_a")
    assert bench.measured_traffic("k_raster_front", "frame_a") == 73751296 + 26000000
    assert bench.measured_traffic("k_uv", "frame_a") == 1500000
    assert bench.measured_traffic("k_pack_push", "frame_a") is None
    assert bench.measured_traffic("k_uv", "frame_b") is None
