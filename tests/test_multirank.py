"""The N > 1 path of the benchmark on CPU (gloo, world size 2): frames are
sharded by rank with no data-path collective (each rank's streams equal the
streams one process makes of the same frames), the job time is the maximum
over ranks, and the job throughput counts every rank's frames."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from oracle import oracle as orc
    from paper_2606_05650_gb300 import synthetic as syn
    frames = bench.make_frames(rank, 2, n=1500)
    sizes = []
    for pos, attr in frames:
        bs = orc.encode_frame(pos, attr, 10, syn.gs_channel_groups(), syn.GS_BASE_STEPS, 0.5, 512)["bitstream"]
        sizes.append(np.asarray(bs, dtype=np.uint8))
    gathered = [None] * world
    dist.all_gather_object(gathered, [s.tobytes() for s in sizes])  # test-only check, not the data path
    t = bench.max_over_ranks(10.0 * (rank + 1), world, dist)
    v = bench.job_throughput(world, 2, 5, t)
    if rank == 0:
        np.save(os.path.join(out_dir, "res.npy"), np.array([t, v]))
        with open(os.path.join(out_dir, "streams.bin"), "wb") as f:
            for per_rank in gathered:
                for b in per_rank:
                    f.write(len(b).to_bytes(8, "little"))
                    f.write(b)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_frames_and_reduce_time(tmp_path):
    import torch.multiprocessing as mp
    import sys
    sys.path.insert(0, ROOT)
    import bench
    from oracle import oracle as orc
    from paper_2606_05650_gb300 import synthetic as syn
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    t, v = np.load(tmp_path / "res.npy")
    assert t == 20.0  # the slower rank's time
    assert np.isclose(v, 2 * 2 * 5 / 0.020)
    # each rank's streams equal the streams of the same frames coded in one process
    data = (tmp_path / "streams.bin").read_bytes()
    got, i = [], 0
    while i < len(data):
        n = int.from_bytes(data[i:i + 8], "little")
        got.append(data[i + 8:i + 8 + n])
        i += 8 + n
    want = []
    for r in range(world):
        for pos, attr in bench.make_frames(r, 2, n=1500):
            bs = orc.encode_frame(pos, attr, 10, syn.gs_channel_groups(), syn.GS_BASE_STEPS, 0.5, 512)["bitstream"]
            want.append(np.asarray(bs, dtype=np.uint8).tobytes())
    assert got == want
    assert got[0] != got[2]  # ranks code different frames


def test_single_rank_needs_no_collective():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1, None) == 12.5
    assert bench.job_throughput(1, 8, 80, 1000.0) == 640.0
