"""Multi-rank logic of bench.py on CPU (gloo, world size 2): each rank draws
its own field (independent units, no data-path collective) and the step time
reported is the maximum over ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        x = bench.make_field(16, rank, "cpu")
        np.save(os.path.join(out_dir, f"field{rank}.npy"), x)
        m = bench.reduce_max(1.5 + rank, "cpu")
        np.save(os.path.join(out_dir, f"max{rank}.npy"), np.array([m]))
    finally:
        tdist.destroy_process_group()


def test_two_ranks_own_fields_and_max_time(tmp_path):
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn")
    f0 = np.load(tmp_path / "field0.npy")
    f1 = np.load(tmp_path / "field1.npy")
    assert f0.shape == f1.shape == (16, 16, 16) and not np.array_equal(f0, f1)
    assert np.load(tmp_path / "max0.npy")[0] == 2.5 and np.load(tmp_path / "max1.npy")[0] == 2.5


def test_single_rank_max_is_identity():
    import bench

    assert bench.reduce_max(3.25, "cpu") == 3.25
