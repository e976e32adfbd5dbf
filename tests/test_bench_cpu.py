"""bench.py's multi-rank bookkeeping on CPU: two gloo ranks (spawned) agree on
the slowest rank's time and the whole-job rate, and the reference arm does
its work on rank 0 only."""
import io
import os
import sys
import contextlib

import pytest

from conftest import ROOT

torch = pytest.importorskip("torch")
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 + 50.0 * rank            # rank 1 is the slow one
    mx = bench.max_over_ranks(ms, dist, "cpu")
    units = 1024 * 30                   # particles x timed generations per rank
    out.put((rank, mx, bench.job_throughput(units, world, mx)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_time_and_job_rate():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [150.0, 150.0]
    # both ranks' units over the slowest rank's time
    assert got[0][2] == got[1][2] == pytest.approx(2 * 1024 * 30 / 0.150)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.job_throughput(100, 1, 1000.0) == pytest.approx(100.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        rc = bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0",
                         "--workload", "tiny"])
    assert rc == 0 and buf.getvalue() == ""


def test_reference_arm_line(monkeypatch):
    import json
    monkeypatch.setenv("RANK", "0")
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        rc = bench.main(["--impl", "reference", "--steps", "2", "--warmup", "0",
                         "--workload", "tiny"])
    line = json.loads(buf.getvalue())
    assert rc == 0 and line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["cpu_baseline"]["cores"] == bench.cpu_cores()
    assert line["e2e"]["h2d_bytes_per_step"] == 0
    # the workload's config, plus the oracle sample's real swarm size
    assert line["config"]["workload"] == "tiny-30vp-32p" and line["config"]["swarm"] == 32
    assert line["config"]["sample_swarm"] == bench.reference_swarm(30, bench.cpu_cores())


def test_default_workload_is_the_bridge():
    import argparse
    assert bench.DEFAULT_STEPS["bridge"] * 2.5 < 120      # about a minute of timed work
    # parse the defaults without running anything
    captured = {}

    def fake_line(args):
        captured.update(vars(args))
        return None
    orig = bench.gpu_line
    bench.gpu_line = fake_line
    try:
        bench.main([])
    finally:
        bench.gpu_line = orig
    assert captured["workload"] == "bridge" and captured["steps"] == 20
    assert captured["warmup"] >= 3
    assert isinstance(argparse.Namespace(**captured), argparse.Namespace)


def _shard_rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1706_04399_gb300 import inputs
    mine = [inst.name for inst in bench.shard(inputs.batched(count=10), rank, world)]
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    out.put((rank, gathered))
    dist.destroy_process_group()


def test_instance_sharding_covers_every_instance_once():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = 30500 + os.getpid() % 1000
    procs = [ctx.Process(target=_shard_rank, args=(r, 3, port, q)) for r in range(3)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    views = [g for _, g in got]
    assert all(v == views[0] for v in views)          # every rank sees the same split
    names = [n for part in views[0] for n in part]
    assert sorted(names) == sorted(f"batched{i}" for i in range(10))  # each exactly once
    assert [len(part) for part in views[0]] == [4, 3, 3]


def test_oracle_sample_is_bounded_by_instance_size():
    # the bridge-sized oracle sample is one generation of one particle per
    # host thread (each particle's exchange on its own thread)
    assert bench.cpu_sample_shape(400, 16) == (128, 4)
    assert bench.cpu_sample_shape(400, 16, node_swap=True) == (128, 2)
    s, g = bench.cpu_sample_shape(1992, 16)
    assert (s, g) == (16, 1)
    assert bench.reference_swarm(1992, 16) == 16


def test_clock_samples_are_kept_only_inside_the_timed_window(tmp_path):
    # samples before and after the marked window (a slow start-up, an idle
    # tail) must not enter the reported clocks or throttle reasons
    import datetime
    cs = bench.ClockSampler(None)
    cs.proc = object()                 # as if nvidia-smi had run
    cs.out = str(tmp_path / "clocks.csv")
    t = 1_800_000_000.0

    def stamp(x):
        return datetime.datetime.fromtimestamp(x).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    rows = [(-1.0, 900, "Active"), (0.02, 2070, "Not Active"), (0.1, 2040, "Not Active"),
            (2.0, 800, "Active")]
    with open(cs.out, "w") as fh:
        for dt, mhz, slow in rows:
            fh.write(f"{stamp(t + dt)}, {mhz}, 2070, 900.0, {slow}, Not Active, Not Active, "
                     "Not Active, 99\n")
    cs.window = [t, t + 0.2]
    got = cs.summary()
    assert got["samples"] == 2 and got["samples_all"] == 4
    assert got["sm_mhz"] == 2055.0 and got["reasons"] == []


def test_every_global_name_the_bench_uses_exists():
    # the GPU legs only run where a GPU is present: a name they use that the
    # module does not define must still fail here
    import builtins
    import dis
    import types

    def globals_of(code):
        for ins in dis.get_instructions(code):
            if ins.opname == "LOAD_GLOBAL":
                yield ins.argval
        for const in code.co_consts:
            if isinstance(const, types.CodeType):
                yield from globals_of(const)
    missing = sorted({name for name in globals_of(compile(open(bench.__file__).read(),
                                                          bench.__file__, "exec"))
                      if not hasattr(bench, name) and not hasattr(builtins, name)})
    assert not missing, missing
