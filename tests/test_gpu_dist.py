"""The element-partitioned operator and Jacobi-PCG with the library's GPU
operator (fem_pcg_dist) on two and three ranks: gloo processes that all use
cuda:0, interface sums staged through host memory, so no kernel waits on
another rank.  The assembled apply on every rank's nodes must equal the
one-process FP64 oracle (1e-12), and the distributed PCG must take the
oracle PCG's iteration count (within 1) to the same solution (1e-8)."""
import multiprocessing as mp
import os
import tempfile

import pytest

from _dist_worker import run_rank_gpu

pytestmark = pytest.mark.gpu


def _run(world, case):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    with tempfile.TemporaryDirectory() as td:
        init = os.path.join(td, "pg_init")
        procs = [ctx.Process(target=run_rank_gpu, args=(r, world, init, case, q))
                 for r in range(world)]
        for p in procs:
            p.start()
        res = {}
        try:
            for _ in range(world):
                r, d = q.get(timeout=300)
                res[r] = d
        finally:
            for p in procs:
                p.join(timeout=60)
                if p.is_alive():
                    p.kill()
    for r, d in res.items():
        assert "error" not in d, (r, d)
    return res


@pytest.mark.parametrize("world,case", [
    (2, dict(n=4, p=3, seed=5)),
    (3, dict(n=4, p=2, seed=6, random_part=True)),
    (2, dict(n=3, p=4, seed=7, name="BP6")),
    (2, dict(n=4, p=5, seed=8, name="BP5")),
])
def test_partitioned_gpu_apply_and_pcg_match_one_process_oracle(world, case):
    res = _run(world, case)
    for r, d in res.items():
        assert d["apply_err"] <= 1e-12, (r, d)
        assert d["status"] == "FEM_OK", (r, d)
        assert abs(d["iters"] - d["ref_iters"]) <= 1, (r, d)
        assert d["sol_err"] <= 1e-8, (r, d)
        assert d["neighbours"] >= 1
    assert len({d["iters"] for d in res.values()}) == 1     # the ranks agree
