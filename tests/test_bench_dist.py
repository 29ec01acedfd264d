"""The bench's multi-rank plumbing on CPU: two gloo ranks agree on the
maximum step time and pass the barrier; the reference arm's non-zero ranks
exit without work; the whole-job figure counts every rank's strings."""

import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.multiprocessing as mp

from conftest import ROOT

sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    r, w, local = bench.dist_env()
    assert (r, w, local) == (rank, world, rank)
    bench.dist_init(w, local, backend="gloo")
    bench.barrier(w)
    slowest = bench.max_over_ranks(10.0 + rank, w, torch.device("cpu"))
    with open(os.path.join(out_dir, f"rank{rank}"), "w") as f:
        f.write(repr(slowest))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    got = [float(open(tmp_path / f"rank{r}").read()) for r in range(world)]
    assert got == [11.0, 11.0]


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.5, 1, torch.device("cpu")) == 3.5
    bench.barrier(1)   # no-op


def test_job_throughput_counts_every_rank():
    # 1e7 strings per rank, 4 ranks, slowest rank 2 ms: 4e7 strings in 2 ms
    assert bench.job_throughput(10_000_000, 4, 2.0) == pytest.approx(20_000.0)
    assert bench.job_throughput(10_000_000, 1, 2.0) == pytest.approx(5_000.0)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1", "--workload", "random_lower_1e5"],
                       capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_profile_traffic_lookup(tmp_path, monkeypatch):
    """roofline.traffic comes from profiles/traffic.json under the key
    '<kernel>_kernel/<workload>' while the sources digest matches, else None."""
    import json
    import bench
    (tmp_path / "profiles").mkdir()
    entry = {"dram_bytes_per_launch": 123, "sources_sha256": bench.sources_digest()}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"onesweep_kernel/w": entry}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "sources_digest", lambda paths=None: entry["sources_sha256"])
    assert bench.profile_traffic("onesweep_kernel/w") == 123
    assert bench.profile_traffic("onesweep/w") is None
    monkeypatch.setattr(bench, "sources_digest", lambda paths=None: "other")
    assert bench.profile_traffic("onesweep_kernel/w") is None


def test_reference_arm_json_line():
    """bench.py --impl reference on one rank: the oracle timed on the host
    cores prints one JSON line with the contract's keys, its cpu_baseline
    and an e2e with no transfers."""
    import json
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1", "--workload", "random_lower_1e5", "--scale", "0.1"],
                       capture_output=True, text=True, timeout=300,
                       env={k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 1
    assert d["higher_is_better"] is True and d["unit"] == "M keys/s" and d["value"] > 0
    assert d["config"]["workload"] == "random_lower_1e5@0.1" and d["config"]["n"] == 10_000
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
