"""Rank body of the multi-rank CPU tests (gloo): one rank of an element-
partitioned apply and Jacobi-PCG, with the FP64 oracle as the local element
operator.  Results go back through a multiprocessing queue."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def reference_pcg(sh, local_apply, local_diag, b, rtol=1e-10, maxit=10000):
    """Distributed Jacobi-PCG written out in torch on one rank (the test's
    reference for the partition and the exchange; the library's own
    distributed solver is fem_pcg_dist): the interface sum assembles every
    apply and the diagonal, dot products sum over owned nodes and
    all-reduce."""
    import torch
    import torch.distributed as dist

    def dot(u, v):
        s = torch.sum(torch.where(sh.owned, u * v, torch.zeros((), dtype=u.dtype)))
        s = s.reshape(1).to(torch.float64)
        dist.all_reduce(s)
        return s.item()

    inner = sh.inner
    zero = torch.zeros((), dtype=b.dtype)
    d = sh.sum_interfaces(local_diag.clone())
    dinv = torch.where(inner, 1.0 / torch.where(inner, d, torch.ones_like(d)), zero)
    b = torch.where(inner, b, zero)
    x = torch.zeros_like(b)
    r = b.clone()
    z = dinv * r
    p = z.clone()
    rz = dot(r, z)
    bn = dot(b, b) ** 0.5
    k = 0
    while k < maxit and dot(r, r) ** 0.5 > rtol * bn:
        Ap = torch.where(inner, sh.apply(local_apply, torch.where(inner, p, zero)), zero)
        alpha = rz / dot(p, Ap)
        x += alpha * p
        r -= alpha * Ap
        z = dinv * r
        rz_new = dot(r, z)
        p = z + (rz_new / rz) * p
        rz = rz_new
        k += 1
    return x, k


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
        x, k = reference_pcg(sh, local_apply, torch.from_numpy(orc.diagonal()),
                             sh.scatter(torch.from_numpy(bg)), rtol=1e-10)
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


def run_rank_gpu(rank, world, init_file, case, queue):
    """One rank of the element-partitioned solve on the GPU: the library's
    operator on this rank's local mesh, the interface sums over gloo (staged
    through host memory), the library's distributed PCG (fem_pcg_dist).
    Every rank uses cuda:0; no kernel waits on another rank."""
    import numpy as np
    import torch
    import torch.distributed as dist
    from datetime import timedelta
    import fem_inputs
    import oracle
    import paper_2109_04996_b300 as fem
    from paper_2109_04996_b300 import dist as fdist
    try:
        torch.cuda.set_device(0)
        dist.init_process_group("gloo", init_method="file://" + init_file, rank=rank,
                                world_size=world, timeout=timedelta(seconds=120))
        m = fem_inputs.box_mesh(case["n"], case["p"], perturb=0.1, seed=case["seed"])
        part = None
        if case.get("random_part"):
            part = np.random.default_rng(case["seed"]).integers(0, world, m["E"])
        name = case.get("name", "BP3")
        kind, nc, quad, dq = fem.BAKE_OFF[name]
        sh = fdist.Shard(m, rank, world, part=part, device="cuda", ncomp=nc)
        gm = fem.Mesh(sh.local_mesh)
        op = fem.Operator(gm, kind, quad, case["p"] + dq, ncomp=nc)
        glob = oracle.Operator(m, kind, quad, case["p"] + dq, ncomp=nc)
        xg = np.random.default_rng(1).uniform(-1, 1, nc * m["N"])
        y = sh.apply(op.apply, sh.scatter(torch.from_numpy(xg)).cuda()).cpu().numpy()
        ref = sh.scatter(torch.from_numpy(glob.apply(xg))).cpu().numpy()
        apply_err = float(np.linalg.norm(y - ref) / np.linalg.norm(ref))
        bg = fem_inputs.rhs_uniform(m["N"], m["dirichlet"], seed=2, ncomp=nc)
        b = sh.scatter(torch.from_numpy(bg)).cuda()
        x = torch.zeros_like(b)
        st = sh.pcg(op, b, x, rtol=1e-10)
        xr, kr, _ = oracle.pcg(glob, bg, m["dirichlet"], rtol=1e-10)
        xr = sh.scatter(torch.from_numpy(xr)).cpu().numpy()
        sol_err = float(np.linalg.norm(x.cpu().numpy() - xr) / np.linalg.norm(xr))
        queue.put((rank, dict(apply_err=apply_err, iters=st["iterations"], ref_iters=kr,
                              status=st["status"], sol_err=sol_err,
                              neighbours=len(sh.neighbours))))
        dist.destroy_process_group()
    except Exception as e:  # reported to the parent, which fails the test
        import traceback
        queue.put((rank, {"error": repr(e) + traceback.format_exc()[-800:]}))
