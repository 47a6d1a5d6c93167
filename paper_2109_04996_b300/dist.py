"""Element-partitioned (multi-rank) form of the operator and of Jacobi-PCG.

The paper's parallel setting (sections "libCEED" and "Nek and MFEM"): the
global operator is A = P^T G^T B^T D B G P, where P maps the global vector to
each process's subdomain vector, G restricts to elements; the action of P^T
is a sum over the processes that share an interface node (gslib's
gather-scatter), and CG's dot products are global sums (all-reduce).

Here each rank owns a set of elements and the nodes they touch (local
numbering).  This module holds the partition and the communication only:
`Shard.sum_interfaces` adds the neighbouring ranks' contributions on shared
nodes by point-to-point exchange (staged through host memory when the
backend is gloo), and `Shard.pcg` runs the library's element-partitioned
Jacobi-PCG (`fem_pcg_dist`), whose applies, vector updates and dot products
are the library's kernels, handing it the interface sum and the scalar
all-reduce as callbacks.  A node is owned by the lowest rank that touches
it; dot products sum over owned nodes.  Communication goes through
torch.distributed (gloo on CPU, NCCL on GPUs).
"""
import numpy as np
import torch
import torch.distributed as dist


def contiguous_partition(E, world):
    """Element -> rank map with contiguous, near-equal element blocks."""
    bounds = np.linspace(0, E, world + 1).round().astype(np.int64)
    part = np.empty(E, dtype=np.int64)
    for r in range(world):
        part[bounds[r]:bounds[r + 1]] = r
    return part


class Shard:
    """Rank `rank`'s part of a global mesh dict (as from fem_inputs.box_mesh
    or mesh_connectivity): `local_mesh` is a mesh dict of its elements with
    local node ids (sorted by global id), `gnodes` the global ids of its
    nodes, `neighbours` a list of (rank, local indices of the shared nodes in
    ascending global order), `owned` a bool mask of the nodes it owns."""

    def __init__(self, mesh, rank, world, part=None, device="cpu", ncomp=1):
        E = mesh["E"]
        part = contiguous_partition(E, world) if part is None else np.asarray(part)
        if part.shape != (E,) or part.min() < 0 or part.max() >= world:
            raise ValueError("partition must give every element a rank in [0, world)")
        self.rank, self.world, self.device, self.ncomp = rank, world, device, ncomp
        en_all = np.asarray(mesh["elem_nodes"])
        self.elems = np.flatnonzero(part == rank)
        en = en_all[self.elems]
        self.gnodes = np.unique(en)
        local_en = np.searchsorted(self.gnodes, en).astype(np.int32)
        self.N = self.gnodes.size
        dirichlet = np.asarray(mesh["dirichlet"])[self.gnodes]
        self.local_mesh = dict(vert_xyz=mesh["vert_xyz"],
                               elem_verts=np.ascontiguousarray(np.asarray(mesh["elem_verts"])[self.elems]),
                               elem_nodes=np.ascontiguousarray(local_en), dirichlet=dirichlet,
                               p=mesh["p"], N=self.N, E=self.elems.size, n=None, M=None,
                               perm=np.arange(self.elems.size, dtype=np.int64))
        # ranks touching each of this rank's nodes (from the global element map)
        lowest = np.full(mesh["N"], world, dtype=np.int64)
        self.neighbours = []
        for q in range(world):
            nodes_q = np.unique(en_all[part == q])
            lowest[nodes_q] = np.minimum(lowest[nodes_q], q)
            if q == rank:
                continue
            shared = np.intersect1d(self.gnodes, nodes_q, assume_unique=True)
            if shared.size:
                self.neighbours.append((q, torch.from_numpy(np.searchsorted(self.gnodes, shared)).to(device)))
        self.owned = torch.from_numpy(np.tile(lowest[self.gnodes] == rank, ncomp)).to(device)
        self.inner = torch.from_numpy(np.tile(dirichlet == 0, ncomp)).to(device)

    # -- communication
    def sum_interfaces(self, y):
        """y (local, unassembled) += the neighbours' contributions on shared
        nodes; every component [ncomp][N] is exchanged together.  With the
        gloo backend CUDA buffers are staged through host memory."""
        N = self.N
        yv = y.view(self.ncomp, N)
        stage = y.is_cuda and dist.get_backend() == "gloo"
        sends, recvs, reqs = [], [], []
        for q, idx in self.neighbours:
            idx_y = idx.to(y.device) if idx.device != y.device else idx
            buf = yv[:, idx_y].contiguous()
            if stage:
                buf = buf.cpu()
            out = torch.empty_like(buf)
            sends.append(buf)
            recvs.append((idx_y, out))
            reqs.append(dist.isend(buf, q))
            reqs.append(dist.irecv(out, q))
        for r in reqs:
            r.wait()
        for idx_y, out in recvs:
            yv[:, idx_y] += out.to(y.device) if stage else out
        return y

    # -- operator
    def apply(self, local_apply, x):
        """Assembled y = A x on this rank's nodes: local element operator,
        then the interface sum."""
        return self.sum_interfaces(local_apply(x))

    def scatter(self, xg):
        """This rank's entries of a global vector [ncomp * N_global]."""
        xg = torch.as_tensor(xg)
        Ng = xg.numel() // self.ncomp
        idx = torch.from_numpy(self.gnodes).to(xg.device)
        return torch.cat([xg[c * Ng + idx] for c in range(self.ncomp)]).to(self.device)

    def owned_nodes(self, device="cuda"):
        """[N] uint8: 1 on the local nodes this rank owns."""
        return self.owned[:self.N].to(torch.uint8).to(device)

    def pcg(self, op, b, x, precond=None, rtol=1e-10, maxit=10000, zero_guess=True):
        """Jacobi-PCG (or plain CG, precond=PC_NONE) on the Dirichlet-
        constrained global system through the library (fem_pcg_dist): op is
        this rank's fem.Operator on local_mesh, b this rank's entries of the
        assembled right-hand side, x its entries of the solution (in place).
        Returns the library's statistics."""
        import ctypes
        import paper_2109_04996_b300 as fem
        y = torch.zeros_like(b)
        owned = self.owned_nodes(b.device)
        errors = []

        def cb_sum(ctx, ptr):
            try:
                self.sum_interfaces(y)
                return 0
            except Exception as e:  # noqa: BLE001 -- reported after the call
                errors.append(e)
                return 1

        def cb_reduce(ctx, vals, count):
            try:
                t = torch.tensor([vals[i] for i in range(count)], dtype=torch.float64)
                if dist.get_backend() != "gloo":
                    t = t.to(b.device)
                dist.all_reduce(t)
                for i, v in enumerate(t.cpu().tolist()):
                    vals[i] = v
                return 0
            except Exception as e:  # noqa: BLE001
                errors.append(e)
                return 1

        st = fem.pcg_dist(op, owned, b, x, y, fem._CommSum(cb_sum), fem._CommReduce(cb_reduce),
                          precond=fem.PC_JACOBI if precond is None else precond, rtol=rtol,
                          maxit=maxit, zero_guess=zero_guess)
        if errors:
            raise errors[0]
        return st
