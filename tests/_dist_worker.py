"""Rank body of the multi-rank CPU tests (gloo): one rank of an element-
partitioned apply and Jacobi-PCG, with the FP64 oracle as the local element
operator.  Results go back through a multiprocessing queue."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def run_rank(rank, world, init_file, case, queue):
    import numpy as np
    import torch
    import torch.distributed as dist
    from datetime import timedelta
    import fem_inputs
    import oracle
    from paper_2109_04996_b300 import dist as fdist
    try:
        dist.init_process_group("gloo", init_method="file://" + init_file, rank=rank,
                                world_size=world, timeout=timedelta(seconds=case.get("timeout", 60)))
        if case.get("fail_rank") == rank:
            # a rank that fails between steps, before the interface exchange
            raise RuntimeError("injected failure on the host")
        m = fem_inputs.box_mesh(case["n"], case["p"], perturb=0.1, seed=case["seed"])
        part = None
        if case.get("random_part"):
            part = np.random.default_rng(case["seed"]).integers(0, world, m["E"])
        nc = case.get("ncomp", 1)
        sh = fdist.Shard(m, rank, world, part=part, ncomp=nc)
        kind = oracle.MASS if case.get("mass") else oracle.DIFFUSION
        orc = oracle.Operator(sh.local_mesh, kind, oracle.GAUSS, case["p"] + 2, ncomp=nc)
        glob = oracle.Operator(m, kind, oracle.GAUSS, case["p"] + 2, ncomp=nc)

        def local_apply(x):
            return torch.from_numpy(orc.apply(x.numpy()))

        xg = np.random.default_rng(1).uniform(-1, 1, nc * m["N"])
        y = sh.apply(local_apply, sh.scatter(torch.from_numpy(xg))).numpy()
        ref = sh.scatter(torch.from_numpy(glob.apply(xg))).numpy()
        apply_err = float(np.abs(y - ref).max() / np.abs(ref).max())
        bg = fem_inputs.rhs_uniform(m["N"], m["dirichlet"], seed=2, ncomp=nc)
        x, k = sh.pcg(local_apply, torch.from_numpy(orc.diagonal()), sh.scatter(torch.from_numpy(bg)),
                      rtol=1e-10)
        xr, kr, _ = oracle.pcg(glob, bg, m["dirichlet"], rtol=1e-10)
        xr = sh.scatter(torch.from_numpy(xr)).numpy()
        sol_err = float(np.linalg.norm(x.numpy() - xr) / np.linalg.norm(xr))
        owned = int(sh.owned.sum().item())
        queue.put((rank, dict(apply_err=apply_err, iters=k, ref_iters=kr, sol_err=sol_err,
                              owned=owned, nodes=sh.N, neighbours=len(sh.neighbours),
                              global_N=nc * m["N"])))
        dist.destroy_process_group()
    except Exception as e:  # reported to the parent, which fails the test
        queue.put((rank, {"error": repr(e)}))
