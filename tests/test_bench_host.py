"""Host-side logic of bench.py on CPU: the whole-job throughput of N ranks is
the sum of their units over the slowest rank's time (2 gloo ranks)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    value, t = bench.job_throughput(1.0 + rank, 100.0 * (rank + 1))
    q.put((rank, value, t))
    dist.destroy_process_group()


def test_job_throughput_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(2))
    for _, value, t in res:
        assert t == 2.0                     # slowest rank
        assert value == pytest.approx(300.0 / 2.0)


def test_job_throughput_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_throughput(2.0, 10.0) == (5.0, 2.0)


def _args(argv, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py"] + argv)
    return bench, bench.parse()


def test_oracle_cycle_counts_for_the_bench_lines(monkeypatch):
    """The CPU baseline of each bench line scales by the oracle's own count
    for that line (oracle/bench_cycles.json): the stand-alone cycle, FGMRES
    around Jacobi cycles, FGMRES around the GMRES(3) cycle."""
    bench, a = _args([], monkeypatch)
    assert (a.smoother, a.nu, a.krylov, a.transfer) == ("gmres3", 2, 0, "bezier")
    assert bench._cycles_from_cache(a) == 43
    bench, a = _args(["--krylov", "20", "--smoother", "jacobi", "--nu", "1"], monkeypatch)
    assert abs(a.beta2 - 0.7) < 1e-15
    assert bench._cycles_from_cache(a) == 417
    bench, a = _args(["--krylov", "10"], monkeypatch)
    assert bench._cycles_from_cache(a) == 63
    bench, a = _args(["--transfer", "linear"], monkeypatch)
    assert bench._cycles_from_cache(a) is None      # no oracle count stored: the line says so


def test_workload_config_names_the_outer_loop_and_transfer(monkeypatch):
    bench, a = _args(["--krylov", "20", "--smoother", "jacobi", "--nu", "1"], monkeypatch)
    c = bench.workload_config(a)
    assert "FGMRES(20)" in c["outer"] and c["cycle"] == "V(1,1)" and c["smoother"] == "jacobi"
    assert c["transfer"].startswith("Eq. (xex)")
    bench, a = _args(["--transfer", "linear"], monkeypatch)
    c = bench.workload_config(a)
    assert c["outer"] == "stand-alone cycle iteration" and "linear" in c["transfer"]


def test_step_traffic_only_for_the_captured_sources(monkeypatch, tmp_path):
    """roofline.traffic comes from the committed ncu record only while the
    kernel sources it hashes are unchanged, and only for the captured
    workload (n = 1024, cycle precision complex64, FGMRES restart length m)."""
    import json
    import shutil
    bench, a = _args([], monkeypatch)
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic_gmres_step_level0.json")))
    assert bench.step_traffic(a, 4) == rec["dram_bytes_per_rhs"] * a.batch
    bench, a64 = _args(["--precision", "fp64"], monkeypatch)
    assert bench.step_traffic(a64, 4) is None
    bench, a5 = _args(["--krylov", "20", "--smoother", "jacobi", "--nu", "1"], monkeypatch)
    fg = json.load(open(os.path.join(ROOT, "profiles", "traffic_fgmres_step_level0.json")))
    assert fg["m"] == 20 and bench.step_traffic(a5, 5) == fg["dram_bytes_per_rhs"] * a5.batch
    bench, a10 = _args(["--krylov", "10"], monkeypatch)
    assert bench.step_traffic(a10, 5) is None      # captured with m = 20
    # a copy of the tree in which one hashed source differs by a byte
    for d in ("profiles",):
        shutil.copytree(os.path.join(ROOT, d), tmp_path / d)
    for f in rec["sources"]:
        os.makedirs(tmp_path / os.path.dirname(f), exist_ok=True)
        shutil.copy(os.path.join(ROOT, f), tmp_path / f)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.step_traffic(a, 4) == rec["dram_bytes_per_rhs"] * a.batch
    with open(tmp_path / rec["sources"][0], "a") as fh:
        fh.write("\n")
    assert bench.step_traffic(a, 4) is None
