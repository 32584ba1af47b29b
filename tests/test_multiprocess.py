"""The N > 1 host logic of bench.py on CPU ranks (gloo, world size 2): the
path does not partition a solve (replicas), so the only cross-rank steps are
the barrier around the timed region and the max over ranks of the step time
that gives the whole-job throughput."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _members_rank(rank: int, world: int, port: int, out):
    """A rank of the batched workload's split: solves nothing, but returns
    per-member values computed from the member index, which the gather must
    put back in member order on every rank."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    w, r, local, pg = bench.dist_init("gloo")
    try:
        sizes = [(i * 37) % 11 + 1 for i in range(20)]
        parts = bench.split_members(sizes, w)
        mine = parts[r]
        vals = [1e-9 * (i + 1) for i in mine]
        full = bench.gather_members(pg, w, mine, vals, len(sizes))
        out.put((r, mine, full))
    finally:
        pg.destroy_process_group()


def test_two_ranks_split_the_members_and_gather_their_residuals():
    """World size 2 on gloo: the two ranks take disjoint parts of the members
    that together cover all of them, and both reassemble the per-member
    values in member order."""
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_members_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, f0), (r1, m1, f1) = res
    assert (r0, r1) == (0, 1)
    assert sorted(m0 + m1) == list(range(20)) and not set(m0) & set(m1)
    want = [1e-9 * (i + 1) for i in range(20)]
    assert f0 == want and f1 == want


def _rank(rank: int, world: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    w, r, local, pg = bench.dist_init("gloo")
    try:
        bench.barrier(pg)
        ms_local = 100.0 + 50.0 * r  # rank 1 is the slow one
        ms, value = bench.job_value(pg, ms_local, w, torch.device("cpu"))
        bench.barrier(pg)
        out.put((r, w, ms, value))
    finally:
        pg.destroy_process_group()


def test_two_cpu_ranks_time_by_the_slowest_rank():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, *_ in res] == [0, 1]
    for _, w, ms, value in res:
        assert w == 2 and ms == 150.0 and value == pytest.approx(2 * 1000.0 / 150.0)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    os.environ.pop("WORLD_SIZE", None)
    w, r, local, pg = bench.dist_init()
    assert (w, r, pg) == (1, 0, None)
    assert bench.job_value(pg, 80.0, 1, torch.device("cpu")) == (80.0, 12.5)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    """bench.py --impl reference under torchrun: ranks other than 0 print
    nothing and do no work."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(bench, "_oracle_sample", lambda *a, **k: pytest.fail("rank 1 must not run the oracle"))
    bench.run_reference(type("A", (), {"workload": "tube_large", "warmup": 1, "steps": 1, "gpus": 2})())
    assert capsys.readouterr().out == ""


def test_bench_describes_each_workload_from_its_preset():
    """The bench line names its workload by the preset's geometry."""
    import bench
    assert bench.describe_workload("tube_large") == "straight tube 96x(11+5)x400"
    assert bench.describe_workload("stenosis") == "stenosed tube 160x(13+7)x600"
    assert bench.describe_workload("bifurcation").startswith("bifurcation, O-grid core 40x40, (24+5) rings")


def test_member_split_is_balanced_and_complete():
    """Independent problems split over ranks: every member on exactly one
    rank, largest first to the least-loaded rank, so no rank carries more
    than the lightest rank plus the largest member."""
    import bench
    sizes = [5, 80, 17, 17, 40, 3, 60, 22, 9, 31]
    for world in (1, 2, 3, 4):
        parts = bench.split_members(sizes, world)
        assert sorted(i for p in parts for i in p) == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(sizes)
        assert all(p == sorted(p) for p in parts)
    assert bench.split_members([10, 10], 2) == [[0], [1]]
    assert bench.split_members([4, 3, 3], 2) == [[0], [1, 2]]
