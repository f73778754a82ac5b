"""The multi-process path of bench.py, on CPU: two ranks over gloo.

Galaxies are independent, so under torchrun every rank fits its own batch (weak
scaling) and the only collectives are host scalars: the max over ranks of the
timed region and the sum of the work done.  These tests run bench.py's own
helpers in two spawned processes (127.0.0.1 rendezvous): the environment parse,
the process-group set-up, both reductions, the per-rank batch seeds (same recipe
and shapes, different galaxies), and the reference arm, which runs on rank 0 only
while the other ranks leave it without work or output."""
import json
import os
import socket

import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out_dir: str):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import contextlib
    import io

    import bench
    from paper_2404_07780_b300 import synth

    w, r, local = bench.dist_env()
    dist = bench.dist_init(w, "gloo")
    res = {"env": [w, r, local], "initialized": dist.is_initialized(),
           "ms_max": bench.reduce_max(10.0 + 5.0 * r, w),      # per-rank timed region
           "units": bench.reduce_sum(100.0 + r, w),           # per-rank converged galaxies
           "seed": bench.rank_seed(r)}
    b = synth.draw_sdss(seed=bench.rank_seed(r), G=2)
    res["shape"] = list(b.truth.shape) + [b.H, b.W, b.K]
    res["truth0"] = b.truth[0].tolist()
    buf = io.StringIO()
    if r != 0:
        with contextlib.redirect_stdout(buf):
            res["ref_rc"] = bench.run_reference(None, w, r)
    res["ref_out"] = buf.getvalue()
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
        json.dump(res, f)


@pytest.mark.timeout(300)
def test_two_gloo_ranks_reduce_timing_and_work_and_draw_their_own_batches(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r, x in enumerate(res):
        assert x["env"] == [world, r, r] and x["initialized"]
        assert x["ms_max"] == 15.0           # max over ranks, not the local value
        assert x["units"] == 201.0           # whole-job work: 100 + 101
    # value = units of all ranks / max time: what rank 0 prints
    assert res[0]["units"] / (res[0]["ms_max"] / 1e3) == pytest.approx(201.0 / 0.015)
    # weak scaling: the same recipe and shapes on every rank, different galaxies
    assert res[0]["seed"] != res[1]["seed"]
    assert res[0]["shape"] == res[1]["shape"]
    assert res[0]["truth0"] != res[1]["truth0"]
    # the reference arm: rank 1 exits 0 at once and prints nothing
    assert res[1]["ref_rc"] == 0 and res[1]["ref_out"] == ""


def test_single_process_reductions_are_the_identity():
    import bench
    assert bench.reduce_max(12.5, 1) == 12.5
    assert bench.reduce_sum(7.0, 1) == 7.0
