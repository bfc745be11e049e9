"""The N > 1 path of bench.py on the CPU: two gloo ranks on 127.0.0.1.

The path does not shard (replicas only): under torchrun every rank steps its
own seeded system, timings are reduced to the slowest rank's, the job's
value counts every rank's bands, and the reference arm runs on rank 0 alone
(the other ranks exit without work).  No GPU is involved."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, outdir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    slowest = bench.max_over_ranks(10.0 + rank, w, device="cpu")
    cfg = bench.replica_config("tiny-16", r)
    value = bench.aggregate_value(6, 4, w, slowest)
    args = SimpleNamespace(workload="tiny-16", warmup=0, steps=1, gpus=w)
    buf = io.StringIO()
    with redirect_stdout(buf):
        rc = bench.run_reference(args)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(outdir, f"rank{rank}.json"), "w") as f:
        json.dump({"rank": r, "world": w, "local": local, "slowest": slowest, "value": value, "rc": rc,
                   "printed": buf.getvalue(), "atom0": list(cfg["atoms"][0]["pos"])}, f)


def test_two_gloo_ranks(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    out = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for r, o in enumerate(out):
        assert (o["rank"], o["world"], o["local"]) == (r, 2, r)
        assert o["slowest"] == 11.0                    # the slower rank's time on every rank
        assert o["value"] == pytest.approx(6 * 4 * 2 / 0.011)
        assert o["rc"] == 0
    # rank 0 alone prints the reference arm's line; rank 1 does no work
    line = json.loads(out[0]["printed"].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert out[1]["printed"] == ""
    # each replica steps its own seeded system
    assert out[0]["atom0"] != out[1]["atom0"]
