"""Host-side logic of bench.py that needs no GPU: the replica timing
collectives (world size 2 over gloo), the clock-record parser and the cost
model it reports with."""
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    r, w, lr = bench.dist_env()
    d = bench.Dist(w, "gloo")
    d.barrier()
    m = d.max(1.5 * (rank + 1))
    q.put((r, w, lr, m))
    d.close()


def test_replica_max_over_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == [(0, 2, 0, 3.0), (1, 2, 1, 3.0)]


def test_clock_summary_parsing():
    sys.path.insert(0, ROOT)
    import bench
    cs = bench.ClockSampler(0)
    cs.lines = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1995, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage",
    ]
    s = cs.summary()
    assert s["sm_mhz"] == 2070 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 3
    assert bench.ClockSampler(0).summary()["reasons"] == ["unavailable"]
