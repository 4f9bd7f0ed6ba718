"""The multi-GPU benchmark path on CPU: two gloo ranks on 127.0.0.1 check the
cross-rank pieces of bench.py (replica seeds, max-over-ranks timing, rank 0
alone printing the reference arm)."""
import json
import os
import socket
import subprocess
import sys


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    got = bench.max_over_ranks([1.0 + rank, 10.0 - rank, 0.5 * rank], world)
    seed = bench.replica_seed(7, rank)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got, seed))


def test_two_gloo_ranks_take_the_max_and_distinct_seeds():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    by = {r: (g, s) for r, g, s in out}
    for r in (0, 1):
        assert by[r][0] == [2.0, 10.0, 0.5]
    assert by[0][1] != by[1][1]


def test_reference_arm_under_two_ranks_prints_once():
    # torchrun-style environment: rank 1 must exit quietly, rank 0 prints the
    # oracle's line (a tiny grid keeps the CPU work short)
    outs = []
    for rank in (0, 1):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
        r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                            "--steps", "1", "--warmup", "0", "--n", "256"],
                           capture_output=True, text=True, env=env, timeout=300)
        assert r.returncode == 0, r.stderr
        outs.append(r.stdout.strip())
    line = json.loads(outs[0].splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["n_gpus"] == 2
    assert outs[1] == ""
