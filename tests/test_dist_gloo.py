"""Element-partitioned operator and Jacobi-PCG (paper_2109_04996_b300/dist.py)
on 2 and 3 CPU ranks over gloo, the local element operator being the FP64
oracle: the assembled apply equals the one-process oracle apply on every
rank's nodes, the distributed PCG takes the one-process iteration count
(within 1) to the same solution, and the owned nodes partition the mesh."""
import multiprocessing as mp
import os
import tempfile

import pytest

from _dist_worker import run_rank


def _run(world, case, expect_errors=False):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    with tempfile.TemporaryDirectory() as td:
        init = os.path.join(td, "pg_init")
        procs = [ctx.Process(target=run_rank, args=(r, world, init, case, q)) for r in range(world)]
        for p in procs:
            p.start()
        res = {}
        try:
            for _ in range(world):
                r, d = q.get(timeout=240)
                res[r] = d
        finally:
            for p in procs:
                p.join(timeout=30)
                if p.is_alive():
                    p.kill()
    if not expect_errors:
        for r, d in res.items():
            assert "error" not in d, (r, d)
    return res


@pytest.mark.parametrize("world,case", [
    (2, dict(n=4, p=3, seed=5)),
    (3, dict(n=4, p=2, seed=6, random_part=True)),
    (2, dict(n=3, p=2, seed=7, ncomp=3)),
    (3, dict(n=3, p=3, seed=8, mass=True)),
])
def test_partitioned_apply_and_pcg_match_one_process(world, case):
    res = _run(world, case)
    for r, d in res.items():
        assert d["apply_err"] <= 1e-13, (r, d)
        assert abs(d["iters"] - d["ref_iters"]) <= 1, (r, d)
        assert d["sol_err"] <= 1e-8, (r, d)
        assert d["neighbours"] >= 1
    assert sum(d["owned"] for d in res.values()) == res[0]["global_N"]


def test_a_failed_rank_ends_its_peers_with_an_error_not_a_hang():
    # rank 1 raises before the first exchange; rank 0's exchange or
    # all-reduce must fail (peer gone / process-group timeout) and report it
    res = _run(2, dict(n=3, p=2, seed=9, fail_rank=1, timeout=10), expect_errors=True)
    assert "injected failure" in res[1].get("error", "")
    assert "error" in res[0], res[0]
