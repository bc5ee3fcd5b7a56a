"""The multi-rank path on CPUs (gloo, world size 2): walk ids are sharded by rank with no data exchange,
and the whole-job figures are the slowest rank's time and the sum of the ranks' work."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import bench
    import labs_inputs as inp
    import oracle

    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    L, p, n = 37, 6, 6
    pre = inp.distinct_prefixes(8, p, seed=3)
    begin, count = bench.shard(rank, n)
    cand, st = oracle.walk_search(L, True, p, pre, count, 400, 60, seed=11, R=4, walk_begin=begin)
    gathered = [None] * world
    dist.all_gather_object(gathered, (begin, cand.tobytes(), st.tobytes()))
    from paper_2409_07222_gb300.merge import merge_across_ranks

    top = merge_across_ranks(cand, 9)
    if rank == 0:
        np.save(os.path.join(out_dir, "top.npy"), top)
    else:
        assert top is None
    t, u = bench.reduce_over_ranks(10.0 + rank, 100 * (rank + 1), "cpu")
    np.save(os.path.join(out_dir, "rank%d.npy" % rank), np.array([t, u], dtype=np.float64))
    if rank == 0:
        parts = sorted(gathered)
        with open(os.path.join(out_dir, "walks.bin"), "wb") as f:
            for _, c, s in parts:
                f.write(c)
        with open(os.path.join(out_dir, "stats.bin"), "wb") as f:
            for _, c, s in parts:
                f.write(s)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_walks_and_reduce(tmp_path):
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn")
    import labs_inputs as inp
    import oracle

    L, p, n = 37, 6, 6
    pre = inp.distinct_prefixes(8, p, seed=3)
    cand, st = oracle.walk_search(L, True, p, pre, 2 * n, 400, 60, seed=11, R=4)
    assert (tmp_path / "walks.bin").read_bytes() == cand.tobytes()
    assert (tmp_path / "stats.bin").read_bytes() == st.tobytes()
    for r in range(2):
        t, u = np.load(tmp_path / ("rank%d.npy" % r))
        assert t == 11.0 and u == 300  # slowest rank's time, all ranks' work
    # the merged step-2 seeds equal the K best distinct states of the single-process run
    from paper_2409_07222_gb300.merge import topk_candidates

    top = np.load(tmp_path / "top.npy")
    want = topk_candidates(cand, 9)
    assert top.tobytes() == want.tobytes()
    assert len(np.unique(top["fp"])) == len(top) and np.all(np.diff(top["E"]) >= 0)


def test_topk_keeps_first_record_of_each_state():
    """K smallest distinct (E, fp), first (walk, step) record of each, empty slots dropped -- written out
    on a hand-made record set."""
    sys.path.insert(0, ROOT)
    from paper_2409_07222_gb300 import CANDIDATE_DTYPE
    from paper_2409_07222_gb300.merge import topk_candidates

    rows = [(5, 3, 9, 11), (5, 1, 4, 11), (2, 7, 1, 20), (5, 0, 8, 10), (2**31 - 1, 0, 0, 2**64 - 1), (9, 2, 2, 1)]
    c = np.zeros(len(rows), dtype=CANDIDATE_DTYPE)
    for i, (E, w, st, fp) in enumerate(rows):
        c[i]["E"], c[i]["walk"], c[i]["step"], c[i]["fp"] = E, w, st, fp
    got = topk_candidates(c, 3)
    assert [(int(r["E"]), int(r["fp"]), int(r["walk"]), int(r["step"])) for r in got] == \
        [(2, 20, 7, 1), (5, 10, 0, 8), (5, 11, 1, 4)]


def test_single_process_reduction_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.reduce_over_ranks(5.5, 42, "cpu") == (5.5, 42)
    assert bench.shard(3, 100) == (300, 100)
