"""p-multigrid oracle (TEST INFRASTRUCTURE: only tests/, __graft_entry__ and
the CPU-baseline leg of bench.py may import it).  Plain FP64 numpy around the
brute-force operators of `oracle.Operator`; it shares no code with the CUDA
library.

The paper (section "Ecosystem", matrix-free preconditioning) names
p-multigrid -- a hierarchy of polynomial degrees on one mesh, with
matrix-free smoothers -- without fixing its parts.  The readings taken here:

  * levels: orders p_0 > p_1 > ... > p_L on the same elements, Gauss-Lobatto
    nodes, every level its own discretization (oracle.Operator of that order);
  * prolongation P_l (level l+1 -> l): on each element the coarse nodal values
    are interpolated at the fine element's nodes with the 1D coarse Lagrange
    basis in each direction; a fine node shared by several elements gets the
    average of their values (weight 1 / multiplicity).  Restriction is the
    transpose, R_l = P_l^T;
  * smoother: the Chebyshev iteration of Saad (2003), Algorithm 12.1, applied
    to D^-1 A (D = diag A) on [lo * lmax, hi * lmax], m steps from zero;
    lmax from power iterations on D^-1 A with the Rayleigh quotient
    v^T A v / v^T D v, started from the SplitMix64 vector below;
  * coarsest level: k_c Jacobi-PCG iterations from zero;
  * V-cycle: z = S(r); z += P (V(R (r - A z))); z += S(r - A z).
Dirichlet: every vector of level l vanishes on that level's boundary nodes
and A_l stands for M A M + (I - M) (the form the solvers use).
"""
import numpy as np

from . import Operator, DIFFUSION, GAUSS, gauss_lobatto, lagrange_1d

GOLDEN_GAMMA = 0x9E3779B97F4A7C15


def splitmix64(n, seed):
    """The first n outputs of a SplitMix64 generator (Steele, Lea & Flood
    2014) whose state starts at `seed`: state += gamma; z = state;
    z = (z ^ z >> 30) * 0xBF58476D1CE4E5B9; z = (z ^ z >> 27) * 0x94D049BB133111EB;
    out = z ^ z >> 31 (all mod 2^64).  Python integers, one at a time."""
    mask = (1 << 64) - 1
    out = np.zeros(n, dtype=np.uint64)
    state = seed & mask
    for i in range(n):
        state = (state + GOLDEN_GAMMA) & mask
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        out[i] = z ^ (z >> 31)
    return out


def start_vector(n, seed=0):
    """Power-iteration start: u_i = (splitmix64 output i >> 11) * 2^-53 - 1/2."""
    u = splitmix64(n, seed)
    return np.array([(int(v) >> 11) * 2.0 ** -53 - 0.5 for v in u])


def interpolation_1d(pc, pf):
    """I[i, j] = l_j(z_i): coarse Gauss-Lobatto Lagrange basis of order pc at
    the fine Gauss-Lobatto nodes of order pf ([pf+1, pc+1])."""
    zf, _ = gauss_lobatto(pf + 1)
    v, _ = lagrange_1d(pc, zf)
    return v


class Level:
    """One level: its mesh (fem_inputs.box_mesh dict) and operator (Gauss
    rule of q points per direction, q = p + 2 unless given)."""

    def __init__(self, mesh, kind=DIFFUSION, rff=None, q=None):
        p = mesh["p"]
        self.mesh = mesh
        self.p = p
        self.N = mesh["N"]
        self.op = Operator(mesh, kind, GAUSS, p + 2 if q is None else q, rff=rff)
        self.inner = mesh["dirichlet"] == 0
        d = self.op.diagonal()
        self.diag = np.where(self.inner, d, 0.0)
        self.dinv = np.where(self.inner, 1.0 / np.where(self.inner, d, 1.0), 0.0)
        mult = np.bincount(mesh["elem_nodes"].ravel(), minlength=self.N).astype(float)
        self.w = 1.0 / mult

    def A(self, v):
        """M A M v for v vanishing on the boundary."""
        return np.where(self.inner, self.op.apply(np.where(self.inner, v, 0.0)), 0.0)


def prolong(fine, coarse, xc, masked=True):
    """x_f = P x_c (see the module docstring); masked: input and output
    restricted to the levels' interior nodes (M_f P M_c, the transpose of
    `restrict`), else the plain interpolation of the coarse function."""
    Pf, Pc = fine.p + 1, coarse.p + 1
    if masked:
        xc = np.where(coarse.inner, xc, 0.0)
    I = interpolation_1d(coarse.p, fine.p)
    E = fine.mesh["E"]
    enc = coarse.mesh["elem_nodes"].reshape(E, Pc, Pc, Pc)   # [e][c][b][a]
    enf = fine.mesh["elem_nodes"].reshape(E, Pf * Pf * Pf)
    u = xc[enc]                                              # coarse element values
    u = np.einsum("ia,ecba->ecbi", I, u)                     # direction a (x)
    u = np.einsum("jb,ecbi->ecji", I, u)                     # direction b (y)
    u = np.einsum("kc,ecji->ekji", I, u)                     # direction c (z)
    u = u.reshape(E, -1)
    xf = np.zeros(fine.N)
    np.add.at(xf, enf, u * fine.w[enf])
    return np.where(fine.inner, xf, 0.0) if masked else xf


def restrict(fine, coarse, rf):
    """r_c = P^T r_f (the transpose of `prolong`, built from its steps)."""
    Pf, Pc = fine.p + 1, coarse.p + 1
    I = interpolation_1d(coarse.p, fine.p)
    E = fine.mesh["E"]
    enc = coarse.mesh["elem_nodes"].reshape(E, Pc * Pc * Pc)
    enf = fine.mesh["elem_nodes"].reshape(E, Pf, Pf, Pf)
    rf = np.where(fine.inner, rf, 0.0)
    u = rf[enf] * fine.w[enf]                                # [e][k][j][i]
    u = np.einsum("kc,ekji->ecji", I, u)
    u = np.einsum("jb,ecji->ecbi", I, u)
    u = np.einsum("ia,ecbi->ecba", I, u)
    rc = np.zeros(coarse.N)
    np.add.at(rc, enc, u.reshape(E, -1))
    return np.where(coarse.inner, rc, 0.0)


def power_lmax(level, its, seed=0):
    """Estimate of the largest eigenvalue of D^-1 A: `its` power steps
    v <- D^-1 A v / ||D^-1 A v|| from the SplitMix64 start, then the Rayleigh
    quotient v^T A v / v^T D v of the last v."""
    v = np.where(level.inner, start_vector(level.N, seed), 0.0)
    for _ in range(its):
        v = level.dinv * level.A(v)
        v = v / np.linalg.norm(v)
    return float(v @ level.A(v)) / float(v @ (level.diag * v))


def chebyshev(level, r, lmax, degree, lo=0.1, hi=1.1):
    """m = degree steps of the Chebyshev iteration (Saad 2003, Alg. 12.1) for
    A z = r from z = 0 with preconditioner D: interval [a, b] = [lo, hi] *
    lmax, theta = (a + b)/2, delta = (b - a)/2, sigma = theta/delta;
    rho_0 = 1/sigma, d_0 = D^-1 r / theta; then for k >= 1
    r_k = r_{k-1} - A d_{k-1}, rho_k = 1 / (2 sigma - rho_{k-1}),
    d_k = rho_k rho_{k-1} d_{k-1} + (2 rho_k / delta) D^-1 r_k; z = sum d_k."""
    a, b = lo * lmax, hi * lmax
    theta, delta = 0.5 * (a + b), 0.5 * (b - a)
    sigma = theta / delta
    rho = 1.0 / sigma
    rk = r.copy()
    d = level.dinv * rk / theta
    z = d.copy()
    for _ in range(1, degree):
        rk = rk - level.A(d)
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * level.dinv * rk
        z = z + d
        rho = rho_new
    return z


def coarse_pcg(level, r, its):
    """`its` Jacobi-PCG iterations on A z = r from z = 0 (no stopping test;
    an exactly zero residual ends early)."""
    z = np.zeros_like(r)
    res = r.copy()
    s = level.dinv * res
    p = s.copy()
    rs = res @ s
    for _ in range(its):
        if rs == 0.0:
            break
        Ap = level.A(p)
        alpha = rs / (p @ Ap)
        z += alpha * p
        res -= alpha * Ap
        s = level.dinv * res
        rs_new = res @ s
        p = s + (rs_new / rs) * p
        rs = rs_new
    return z


def vcycle(levels, lmax, r, degree=3, coarse_its=20, lo=0.1, hi=1.1, l=0, coarse_exact=None):
    """z = B r, one V-cycle from level l down.  `lmax[l]` bounds the spectrum
    of D^-1 A on level l; `coarse_exact` (a dense matrix of the coarsest
    level) replaces the coarse PCG by a direct solve."""
    lev = levels[l]
    if l == len(levels) - 1:
        if coarse_exact is not None:
            z = np.zeros_like(r)
            m = lev.inner
            z[m] = np.linalg.solve(coarse_exact[np.ix_(m, m)], r[m])
            return z
        return coarse_pcg(lev, r, coarse_its)
    z = chebyshev(lev, r, lmax[l], degree, lo, hi)
    rc = restrict(lev, levels[l + 1], r - lev.A(z))
    zc = vcycle(levels, lmax, rc, degree, coarse_its, lo, hi, l + 1, coarse_exact)
    z = z + prolong(lev, levels[l + 1], zc)
    z = z + chebyshev(lev, r - lev.A(z), lmax[l], degree, lo, hi)
    return z


def fcg(level, b, precond, rtol=1e-10, maxit=1000):
    """Flexible CG with one stored direction (Notay 2000) on A x = b:
    p_k = z_k - (z_k^T A p_{k-1} / p_{k-1}^T A p_{k-1}) p_{k-1},
    alpha_k = p_k^T r_k / p_k^T A p_k.  Returns (x, iterations)."""
    b = np.where(level.inner, b, 0.0)
    x = np.zeros_like(b)
    r = b.copy()
    bn = np.linalg.norm(b)
    p_old = Ap_old = None
    k = 0
    while k < maxit and np.linalg.norm(r) > rtol * bn:
        z = precond(r)
        p = z if p_old is None else z - (z @ Ap_old) / (p_old @ Ap_old) * p_old
        Ap = level.A(p)
        alpha = (p @ r) / (p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        p_old, Ap_old = p, Ap
        k += 1
    return x, k
