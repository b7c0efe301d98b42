"""The benchmark's replica logic on two gloo ranks (CPU): each rank gets its
own right-hand sides, the slowest rank's time is shared by every rank, and
the whole-job value counts every rank's right-hand sides."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    from paper_1907_04417_gb300.hostsetup import inputs
    import torch.distributed as dist
    w, r, _ = bench.dist_init(backend="gloo")
    P = inputs.anisotropic(N=16, nrhs=1, levels=2)
    B = bench.rhs_block(P, 4, r)
    bench.barrier(w)
    m = bench.max_over_ranks(10.0 + r, w)
    val = bench.whole_job_ms_per_rhs(m, 2, 4, w)
    np.save(os.path.join(out, f"rank{r}.npy"), np.concatenate([[m, val], B.ravel()]))
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    ws, port = 2, _free_port()
    mp.start_processes(_rank_main, args=(ws, port, str(tmp_path)), nprocs=ws, start_method="spawn")
    r0 = np.load(tmp_path / "rank0.npy")
    r1 = np.load(tmp_path / "rank1.npy")
    assert r0[0] == r1[0] == 11.0
    assert r0[1] == r1[1] == 11.0 / 2 / (4 * 2)
    assert not np.array_equal(r0[2:], r1[2:])
