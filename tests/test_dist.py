"""Multi-rank plumbing of the benchmark on CPU: two gloo ranks, replicas only.
The job time is the maximum over ranks and the work is the sum over ranks; there
is no collective on the data path."""
import os
import socket
import subprocess
import sys
import textwrap

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_two_gloo_ranks_reduce_time_and_work(tmp_path):
    script = tmp_path / "rank.py"
    script.write_text(textwrap.dedent("""
        import json, os, sys
        sys.path.insert(0, %r)
        from paper_2604_02755_gb300 import dist
        d = dist.init("gloo")
        rank, ws, _ = dist.world()
        dist.barrier(d)
        t, w = dist.reduce_time_and_work(d, 1.0 + rank, 100.0 * (rank + 1))
        print(json.dumps({"rank": rank, "ws": ws, "t": t, "w": w}))
        dist.finalize(d)
    """ % ROOT))
    port = free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, str(script)], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=120)
        assert p.returncode == 0, e
        outs.append(o.strip().splitlines()[-1])
    import json
    res = [json.loads(o) for o in outs]
    for r in res:
        assert r["ws"] == 2
        assert r["t"] == 2.0   # max over ranks
        assert r["w"] == 300.0  # sum over ranks


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    from paper_2604_02755_gb300 import dist
    assert dist.reduce_time_and_work(None, 3.0, 7.0) == (3.0, 7.0)
