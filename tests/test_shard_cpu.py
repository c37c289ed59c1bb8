"""Frame sharding (host logic, CPU): the frame partition, and the gradient
sum over processes that a sharded fit takes between its backward and its
update, on two gloo ranks."""
import os
import socket
import sys

import pytest
import torch
import torch.multiprocessing as mp

from paper_2505_05356_gb300 import shard

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("n,world", [(16, 1), (16, 2), (16, 3), (60, 8), (3, 5), (0, 2)])
def test_frame_range_partitions_the_batch(n, world):
    ranges = [shard.frame_range(n, world, r) for r in range(world)]
    covered = [f for a, b in ranges for f in range(a, b)]
    assert covered == list(range(n))  # every frame once, in order
    sizes = [b - a for a, b in ranges]
    assert max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)


def test_frame_range_rejects_bad_requests():
    for args in ((4, 0, 0), (4, 2, 2), (4, 2, -1), (-1, 2, 0)):
        with pytest.raises(ValueError):
            shard.frame_range(*args)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2505_05356_gb300 import shard as sh
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # a rank's "gradients": groups of different shapes, rank-dependent values
    g = {"means": torch.full((5, 3), 1.0 + rank), "opacity": torch.arange(4.0) * (rank + 1),
         "empty": torch.zeros(0)}
    sh.allreduce_sum_(g.values())
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, {k: v.tolist() for k, v in g.items()}))


def test_allreduce_sum_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, g in res:  # every rank holds the sum
        assert g["means"] == [[3.0] * 3] * 5
        assert g["opacity"] == [0.0, 3.0, 6.0, 9.0]
        assert g["empty"] == []


@pytest.mark.parametrize("offset,total", [(-1, 4), (3, 4), (0, 1)])
def test_fit_loop_rejects_a_shard_outside_its_batch(offset, total):
    """A loop over 2 frames at frame_offset in a batch of total_frames: the
    range must lie inside the batch (checked before anything touches a GPU)."""
    from paper_2505_05356_gb300 import fit
    params = {"means": torch.zeros((10, 3))}
    targets = torch.zeros((2, 5, 4, 4))
    with pytest.raises(ValueError):
        fit.FitLoop(params, [None, None], None, None, targets, frame_offset=offset,
                    total_frames=total)
