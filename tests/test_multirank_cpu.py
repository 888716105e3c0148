"""The N > 1 path of bench.py on CPU: two gloo ranks run independent
replicas; the whole-job step time is the slowest rank's and the value counts
every rank's samples; each replica draws its own random streams (graph id =
rank); the reference arm prints from rank 0 only."""
import json
import os
import subprocess
import sys

import pytest

from conftest import ROOT

torch = pytest.importorskip("torch")


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
    rate = bench.whole_job_rate(1000, world, ms / 1000.0)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms, rate))


def test_two_rank_timing_is_the_slowest_rank():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    for _, ms, rate in out:
        assert ms == 15.0                      # max over ranks
        assert rate == pytest.approx(2 * 1000 / 0.015)


def test_replicas_draw_their_own_streams():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2008_07799_gb300 import build
    build.build()
    import paper_2008_07799_gb300 as drg

    class A:
        mode, precision, seed, substeps, coarsen, level_tables, perplexity, row_cap = "hogwild", "fp32", 0, None, "hem", False, 0.0, 0
    wl = bench.WORKLOADS["dcsbm1m"]
    gids = [bench.make_params(drg, wl, A, gid=r).gid for r in range(3)]
    assert gids == [0, 1, 2]


def test_reference_arm_prints_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--workload", "grid32", "--cpu-budget", "1"], capture_output=True,
                       text=True, env=env, timeout=600)
    assert r.returncode == 0
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "updates/s"


def test_traffic_record_only_for_its_configuration(tmp_path):
    # a DRAM-traffic record of the level kernel feeds the bench's roofline
    # only for the configuration and kernel source it was taken on
    sys.path.insert(0, ROOT)
    import bench
    cfg = {"workload": "dcsbm1m", "k": 2, "coarsen": "hem", "mode": "hogwild", "precision": "fp32",
           "multilevel": True}
    (tmp_path / "profiles").mkdir()
    rec = {"kernel": "k_hogwild", "kernel_hash": bench.kernel_hash(), "dram_bytes_per_sample": 100.0, "config": cfg}
    (tmp_path / "profiles" / "k_hogwild_traffic.json").write_text(json.dumps(rec))
    assert bench.ncu_traffic_per_sample("k_hogwild", cfg, root=str(tmp_path)) == 100.0
    for key, other in (("coarsen", "star"), ("workload", "ba100k"), ("k", 3), ("mode", "sync"), ("multilevel", False),
                       ("precision", "bf16")):
        assert bench.ncu_traffic_per_sample("k_hogwild", dict(cfg, **{key: other}), root=str(tmp_path)) is None
    assert bench.ncu_traffic_per_sample("k_no_such_kernel", cfg, root=str(tmp_path)) is None
    # a record taken on other kernel source is not used
    (tmp_path / "profiles" / "k_hogwild_traffic.json").write_text(json.dumps(dict(rec, kernel_hash="0" * 16)))
    assert bench.ncu_traffic_per_sample("k_hogwild", cfg, root=str(tmp_path)) is None
