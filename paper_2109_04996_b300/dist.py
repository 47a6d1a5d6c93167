"""Element-partitioned (multi-rank) form of the operator and of Jacobi-PCG.

The paper's parallel setting (sections "libCEED" and "Nek and MFEM"): the
global operator is A = P^T G^T B^T D B G P, where P maps the global vector to
each process's subdomain vector, G restricts to elements; the action of P^T
is a sum over the processes that share an interface node (gslib's
gather-scatter), and CG's dot products are global sums (all-reduce).

Here each rank owns a set of elements and the nodes they touch (local
numbering); `Shard.apply` runs the local element operator (any callable on
the local vector: the library's GPU operator in production, the FP64 oracle
in the CPU tests) and then `Shard.sum_interfaces` adds the neighbouring
ranks' contributions on shared nodes by point-to-point exchange, so every
rank holds the assembled values of its nodes.  A node is owned by the lowest
rank that touches it; dot products sum over owned nodes and all-reduce.
Communication goes through torch.distributed (gloo on CPU, NCCL on GPUs).
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
        nodes; every component [ncomp][N] is exchanged together."""
        N = self.N
        yv = y.view(self.ncomp, N)
        sends, recvs, reqs = [], [], []
        for q, idx in self.neighbours:
            buf = yv[:, idx].contiguous()
            out = torch.empty_like(buf)
            sends.append(buf)
            recvs.append((idx, out))
            reqs.append(dist.isend(buf, q))
            reqs.append(dist.irecv(out, q))
        for r in reqs:
            r.wait()
        for idx, out in recvs:
            yv[:, idx] += out
        return y

    def dot(self, u, v):
        s = torch.sum(torch.where(self.owned, u * v, torch.zeros((), dtype=u.dtype, device=u.device)))
        s = s.reshape(1).to(torch.float64)
        dist.all_reduce(s)
        return s.item()

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

    def pcg(self, local_apply, local_diag, b, rtol=1e-10, maxit=10000):
        """Jacobi-PCG on the Dirichlet-constrained global system, distributed:
        b is this rank's part of the right-hand side (assembled values);
        local_diag the local (unassembled) diagonal, summed here.  Returns
        (x, iterations) with x this rank's part of the solution."""
        inner = self.inner
        zero = torch.zeros((), dtype=b.dtype, device=b.device)
        d = self.sum_interfaces(local_diag.clone())
        dinv = torch.where(inner, 1.0 / torch.where(inner, d, torch.ones_like(d)), zero)
        b = torch.where(inner, b, zero)
        x = torch.zeros_like(b)
        r = b.clone()
        z = dinv * r
        p = z.clone()
        rz = self.dot(r, z)
        bn = self.dot(b, b) ** 0.5
        k = 0
        while k < maxit and self.dot(r, r) ** 0.5 > rtol * bn:
            Ap = torch.where(inner, self.apply(local_apply, torch.where(inner, p, zero)), zero)
            alpha = rz / self.dot(p, Ap)
            x += alpha * p
            r -= alpha * Ap
            z = dinv * r
            rz_new = self.dot(r, z)
            p = z + (rz_new / rz) * p
            rz = rz_new
            k += 1
        return x, k
