"""The multi-rank host logic of bench.py on CPU: two gloo ranks (one process
each), launched the way torchrun sets the environment.  Each rank takes its
own incidence (replicas, no data-path collective), the job's time is the
maximum over ranks on every rank, and in the reference arm only rank 0
works and prints."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    w, r, local = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    inc = bench.rank_incidence(r)
    ms = bench.max_over_ranks(10.0 + 5.0 * r, dist, "cpu")
    dist.barrier()
    # reference arm: ranks other than 0 return at once and print nothing
    buf = io.StringIO()
    if r != 0:
        with redirect_stdout(buf):
            bench.run_reference(None, w, r)
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
        json.dump({"ws": w, "rank": r, "local": local, "theta_i": float(inc[0, 0]), "ms": ms,
                   "ref_out": buf.getvalue()}, f)
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    ws = 2
    mp.start_processes(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(ws)]
    assert [x["rank"] for x in res] == [0, 1] and all(x["ws"] == ws for x in res)
    assert res[0]["theta_i"] != res[1]["theta_i"]           # each rank its own incidence
    assert all(x["ms"] == 15.0 for x in res)                 # max over ranks, seen by every rank
    assert res[1]["ref_out"] == ""
