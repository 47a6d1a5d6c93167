/*
 * fem.h -- C ABI of a B300-native (sm_103a) library for matrix-free,
 * partially assembled high-order finite element operators on hexahedral
 * meshes:  y = G^T B^T D B G x  (Kolev et al., "Efficient Exascale
 * Discretizations: High-Order Finite Element Methods", section "libCEED",
 * finite element operator decomposition), applied inside conjugate gradients
 * for the bake-off problems BP1-BP6 (section "Benchmarks").
 *
 *   G  element restriction: gather of global (L-vector) values into element
 *      (E-vector) values, and its transpose, a scatter-add;
 *   B  tensor-product basis: interpolation / gradients from the (p+1)^3
 *      Gauss-Lobatto nodes of an element to its q^3 quadrature points,
 *      evaluated by sum factorization (section "Benchmarks");
 *   D  pointwise data at quadrature points: w det J (mass, BP1/BP2) or the
 *      symmetric w det J J^{-1} J^{-T} (diffusion, BP3-BP6), times an optional
 *      coefficient kappa(x).
 *
 * Conventions shared by every call:
 *  - Every function returns fem_status; FEM_OK == 0.  On failure the
 *    message of the calling thread's last error is fem_last_error().  No call
 *    aborts, exits or throws across the ABI.
 *  - Arguments named *_host are host pointers and are copied before the call
 *    returns.  All other array arguments are DEVICE pointers owned by the
 *    caller; the library never frees them and keeps no reference after the
 *    call returns (unless stated).
 *  - Work is ordered on the CUDA stream given to fem_op_create (NULL = the
 *    legacy default stream).  Calls return without synchronizing the host
 *    unless stated (fem_cg_solve and fem_solve_refined copy their statistics
 *    back and therefore synchronize).
 *  - Vectors are contiguous float64 (float32 where stated) of length
 *    ncomp * N, component-major: entry c*N + i is component c of node i.
 *  - Local node (a, b, c) of an element (a fastest) is entry a + P b + P^2 c of
 *    its row of elem_nodes, P = p + 1; vertex v = vi + 2 vj + 4 vk of a brick
 *    likewise (lexicographic tensor order).
 *  - Supported orders: 1 <= p <= 8.  Quadrature: FEM_GAUSS with q = p + 2
 *    (BP1-BP4) or q = p + 1, FEM_LOBATTO with q = p + 1 (BP5/BP6,
 *    collocated).
 *  - Handles are not thread safe: one host thread at a time per handle.
 */
#ifndef FEM_H
#define FEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int fem_status;
enum {
  FEM_OK = 0,
  FEM_EINVAL = 1,      /* bad argument: order, quadrature, sizes, null pointer */
  FEM_ENOMEM = 2,      /* device or host allocation failed */
  FEM_ECUDA = 3,       /* a CUDA runtime call failed */
  FEM_EBREAKDOWN = 4,  /* CG breakdown: p^T A p <= 0 or a non-finite scalar */
  FEM_ENOCONV = 5,     /* iteration limit reached before the tolerance */
  FEM_ETIMEOUT = 6,    /* a bounded device-side wait expired */
  FEM_EDEVICE = 7      /* a kernel raised its device error word (bad index) */
};

enum { FEM_MASS = 0, FEM_DIFFUSION = 1 };      /* D: B_ij or A_ij (section "Benchmarks") */
enum { FEM_GAUSS = 0, FEM_LOBATTO = 1 };       /* quadrature family */
enum { FEM_F64 = 0, FEM_F32 = 1 };             /* arithmetic of the apply */
enum { FEM_PC_NONE = 0, FEM_PC_JACOBI = 1, FEM_PC_LEARNED = 2 };

typedef struct fem_mesh fem_mesh;
typedef struct fem_op fem_op;

/* Message of the calling thread's most recent failure ("" if none). */
const char *fem_last_error(void);
/* Library version as 10000*major + 100*minor + patch. */
int fem_version(void);

/* ---------------------------------------------------------------- tables */

/* 1D tables of the tensor basis (section "Benchmarks": Gauss-Legendre q = p+2
 * for BP1-BP4, Gauss-Lobatto-Legendre q = p+1 for BP5/BP6), host output:
 *   nodes_host[P]     Gauss-Lobatto nodes of the Lagrange basis on [-1, 1]
 *   qpts_host[q], qwts_host[q]   quadrature points and weights
 *   interp_host[q*P]  l_a(r_k) at row k, column a
 *   grad_host[q*P]    l_a'(r_k)
 * Any output pointer may be NULL.  FEM_EINVAL for p or q out of range. */
fem_status fem_basis_tables(int p, int q, int quad, double *nodes_host,
                            double *qpts_host, double *qwts_host,
                            double *interp_host, double *grad_host);

/* ---------------------------------------------------------------- mesh */

/* Coordinates of the Q_p nodes of trilinear bricks (host, setup only): node
 * (a,b,c) of element e is the trilinear map of the element's 8 vertices at
 * the tensor Gauss-Lobatto point (z_a, z_b, z_c) (the isoparametric bricks of
 * section "Benchmarks").  vert_xyz_host [nvert][3], elem_verts_host [E][8],
 * elem_nodes_host [E][P^3]; writes node_xyz_host [N][3]. */
fem_status fem_mesh_nodes_from_vertices(int p, int64_t E, int64_t nvert,
                                        const double *vert_xyz_host,
                                        const int32_t *elem_verts_host,
                                        const int32_t *elem_nodes_host,
                                        int64_t N, double *node_xyz_host);

/* Upload a Q_p mesh: connectivity elem_nodes_host [E][P^3] (global node ids in
 * [0, N)), node coordinates node_xyz_host [N][3] and the Dirichlet marker
 * dirichlet_host [N] (1 = constrained node; NULL = none).  The element
 * restriction G is this connectivity (section "libCEED").  Indices are
 * checked on the host (FEM_EINVAL if out of range).  stream: cudaStream_t or
 * NULL. */
fem_status fem_mesh_create(int p, int64_t N, int64_t E,
                           const int32_t *elem_nodes_host,
                           const double *node_xyz_host,
                           const uint8_t *dirichlet_host, void *stream,
                           fem_mesh **out);
/* Same as fem_mesh_create, with the node coordinates computed on the GPU
 * from trilinear bricks (the map of fem_mesh_nodes_from_vertices):
 * vert_xyz_host [nvert][3], elem_verts_host [E][8]. */
fem_status fem_mesh_create_vertices(int p, int64_t N, int64_t E,
                                    const int32_t *elem_nodes_host, int64_t nvert,
                                    const double *vert_xyz_host,
                                    const int32_t *elem_verts_host,
                                    const uint8_t *dirichlet_host, void *stream,
                                    fem_mesh **out);
/* Q_p connectivity of an unstructured hexahedral mesh given by its
 * elements' vertices (host, no GPU): elem_verts_host [E][8] in local order
 * i + 2j + 4k (any orientation per element, right-handed); the element-node
 * table [E][(p+1)^3] (local a + P b + P^2 c) is written with one global id per
 * node of the C^0 Q_p space: vertices, then edge nodes ordered from the
 * edge's lower vertex id, face nodes in a frame anchored at the face's lowest
 * vertex id, interior nodes; ids in order of first use.  dirichlet_host (may
 * be NULL; room for E*(p+1)^3 bytes) gets 1 on every node of a face that
 * belongs to one element only.  *N_out = number of nodes.  FEM_EINVAL for
 * vertex ids out of [0, nvert), an element repeating a vertex, a face of
 * more than two elements, or more than 2^31-1 nodes. */
fem_status fem_mesh_connectivity(int p, int64_t nvert, int64_t E, const int32_t *elem_verts_host,
                                 int32_t *elem_nodes_host, uint8_t *dirichlet_host, int64_t *N_out);
/* Generator of the bake-off meshes (section "Benchmarks": the BPs on brick
 * meshes of the unit cube): nx*ny*nz trilinear bricks of [0,1]^3 with Q_p
 * nodes, built on the host and uploaded like fem_mesh_create_vertices.
 *  - vertex (i,j,k) = i + (nx+1)(j + (ny+1)k) sits at (i/nx, j/ny, k/nz); each
 *    coordinate d of a vertex not on a face normal to d is moved by
 *    perturb * h_d * (2u - 1), u = (SplitMix64 output 3v + d of `seed`) >> 11
 *    times 2^-53 (Steele, Lea & Flood 2014), h_d the element size along d;
 *    coordinates on the cube's faces stay, so the domain is exactly [0,1]^3;
 *  - element (ex,ey,ez) = ex + nx(ey + ny ez), its local vertex t at offset
 *    (t & 1, t >> 1 & 1, t >> 2 & 1);
 *  - node (I,J,K) = I + Mx(J + My K), Mx = p nx + 1 (likewise My, Mz); local
 *    node (a,b,c) of element (ex,ey,ez) is (p ex + a, p ey + b, p ez + c);
 *  - Dirichlet marker 1 on every node of the cube's surface.
 * With perturb = 0 the mesh is the Cartesian one.  FEM_EINVAL for p outside
 * [1, 8], a size < 1, perturb outside [0, 0.5) or more than 2^31-1 nodes.
 * The mesh (nodes, connectivity) is the caller's to destroy. */
fem_status fem_mesh_box(int p, int nx, int ny, int nz, double perturb, uint64_t seed,
                        void *stream, fem_mesh **out);
/* Node coordinates [N][3] of a mesh, copied to host (synchronizes). */
fem_status fem_mesh_node_coords(const fem_mesh *mesh, double *xyz_host);
fem_status fem_mesh_destroy(fem_mesh *mesh);

/* ---------------------------------------------------------------- operator */

/* Create an operator on a mesh and compute its pointwise data D (qdata) and
 * the diagonal of the assembled matrix on the GPU in FP64:
 *   kind   FEM_MASS (B_ij = int phi_i phi_j) or FEM_DIFFUSION
 *          (A_ij = int grad phi_i . grad phi_j), section "Benchmarks";
 *   quad, q  see "Supported orders" above;
 *   ncomp  1 (BP1/BP3/BP5) or 3 (BP2/BP4/BP6), the same scalar operator on
 *          each component;
 *   prec   FEM_F64: the apply computes in FP64 with FP64 qdata;
 *          FEM_F32: an additional FP32 copy of the qdata is kept and
 *          fem_op_apply_f32 becomes available (fem_op_apply stays FP64);
 *   rff_host  NULL (kappa = 1) or the [M][4] rows (w_x, w_y, w_z, b) of
 *          kappa(x) = exp(sigma sqrt(2/M) sum_m cos(w_m . x + b_m)), a random
 *          Fourier feature draw of a Gaussian random field; the data D is
 *          multiplied by kappa at each physical quadrature point.
 * Diffusion with a non-collocated rule at p = 1 and 2 also assembles the
 * element matrices K_e = sum_q grad phi_a^T D grad phi_b in FP64 (and an
 * FP32 copy with FEM_F32) for the element-matrix body: (P^3)(P^3 + 1)/2
 * values per element, 36 at p = 1 and 378 at p = 2.
 * The mesh must outlive the operator.  Work goes to the mesh's stream. */
fem_status fem_op_create(const fem_mesh *mesh, int kind, int quad, int q,
                         int ncomp, int prec, const double *rff_host, int M,
                         double sigma, fem_op **out);
fem_status fem_op_destroy(fem_op *op);

/* Sizes: N nodes, E elements, ncomp, P = p+1, q, and the device bytes held. */
fem_status fem_op_sizes(const fem_op *op, int64_t *N, int64_t *E, int *ncomp,
                        int *P, int *q, int64_t *device_bytes);

/* y = G^T B^T D B G x, the unconstrained operator (no Dirichlet rows),
 * FP64, one fused kernel: gather, sum-factorized interpolation / gradients,
 * pointwise D, transposes and an atomic scatter-add (section "libCEED",
 * fused single-kernel operator).  x, y: device [ncomp*N]; y is overwritten;
 * x and y must not alias. */
fem_status fem_op_apply(fem_op *op, const double *x, double *y);

/* Same in FP32 arithmetic with FP32 qdata (operator created with FEM_F32). */
fem_status fem_op_apply_f32(fem_op *op, const float *x, float *y);

/* y = sum over the listed elements of G_e^T B^T D B G_e x (FP64): the operator
 * restricted to a subset of elements.  elems: device int32 [n]; y overwritten. */
fem_status fem_op_apply_elements(fem_op *op, const int32_t *elems, int64_t n,
                                 const double *x, double *y);

/* diag(A): device [ncomp*N] FP64 diagonal of the assembled operator
 * (computed at create by sum factorization of squared 1D tables). */
fem_status fem_op_diagonal(fem_op *op, double *d);

/* Copy the FP64 qdata of element e to host: mass [q^3] = w det J kappa;
 * diffusion [6][q^3] = (11, 22, 33, 23, 13, 12) entries of
 * w det J kappa J^{-1} J^{-T}; quadrature point (i,j,k) at i + q j + q^2 k. */
fem_status fem_op_qdata_host(fem_op *op, int64_t e, double *out_host);

/* Manufactured load b_i = int phi_i f dV on the GPU (same quadrature as the
 * operator): which = 0: f = sin(pi x) sin(pi y) sin(pi z) (BP1/BP2);
 * which = 1: f = 3 pi^2 sin sin sin (Poisson load of u = sin sin sin).
 * b: device [N] (scalar). */
fem_status fem_op_rhs(fem_op *op, int which, double *b);

/* ---------------------------------------------------------------- autotuning */

/* Launch shape of the fused apply.  epb_choice selects the element body and
 * the elements per block: 0, 1, 2 = the line-based body with even-odd split
 * 1D operators and about 256, 128 or 512 threads per block, 3, 4, 5 = the
 * slab body (one thread per quadrature column) with the same three sizes,
 * 6 = the trilinear body (one thread per element; Gauss diffusion at p = 1
 * only), 7 = the element-matrix body (one thread per element with the
 * operator's assembled element matrices; diffusion with a non-collocated
 * rule at p = 1 and 2 only).  The collocated mass operator (pointwise) has
 * choice 0 only.  FP64 only, the double-word bodies: every product and sum
 * in double-word arithmetic (pairs of FP32 numbers, ~48 bits) on the FP32
 * pipe, with FP64 vectors and FP64 atomic scatter: 8, 9, 10 = the line-based
 * body with the three sizes, 11 = the element-matrix body (where 7 exists),
 * 12, 13, 14 = 8, 9, 10 with the next element group's x gather carried one
 * group ahead (scalar whole-mesh launches; otherwise as 8, 9, 10), 15, 16,
 * 17 = 8, 9, 10 with the even and odd halves of every 1D contraction
 * carried together in packed FP32x2 instructions (the same arithmetic,
 * bit for bit, in half the issue slots), 18, 19, 20 = 15, 16, 17 with an L2
 * bulk prefetch of the next element group's qdata and node ids, 21, 22,
 * 23 = 18, 19, 20 with the pipelined gather of 12, 13, 14 (same results as
 * 15, 16, 17 up to the order of the atomic additions), 24 = the globally
 * assembled operator of p = 1 Gauss diffusion on a lattice mesh (the
 * n x n x n brick with lexicographic nodes and elements, E = n^3 and
 * N = (n+1)^3, checked at operator creation): a 27-point stencil of
 * double-word coefficients assembled from the element matrices, applied
 * one row per thread without atomics (whole-mesh scalar applies; element
 * lists take 11's body); the default where it exists.  Their
 * error against exact FP64 arithmetic: ~5e-14 relative l2 for random x; for
 * diffusion each element's x_e is shifted by its node-0 value first (A_e
 * annihilates constants), which keeps the smoothest fields within ~1e-12 at
 * 8e6 DOFs; x values below 2^-74 in magnitude lose the low word (FP32's
 * exponent range).  blocks_per_sm: resident blocks per SM (0 = the occupancy
 * maximum).  Defaults: the fastest choice of a sweep at 8e6 DOFs per order
 * and operator type (BP3 FP64 at 5e7 DOFs); FP64: the double-word bodies; FP32: 7 for Gauss
 * diffusion at p = 1, the line body elsewhere. */
typedef struct {
  int epb_choice;
  int blocks_per_sm;
  double us;          /* measured time of one apply of this operator, us */
  int from_cache;     /* 1 if read from the cache file, 0 if timed now */
  int candidates;     /* shapes timed */
} fem_tune_result;

/* Set the launch shape used by this operator's apply of precision prec
 * (FEM_F64 or FEM_F32).  Every shape computes the same result up to the
 * order of the atomic additions.  FEM_EINVAL for an invalid choice. */
fem_status fem_op_set_launch_shape(fem_op *op, int prec, int epb_choice,
                                   int blocks_per_sm);

/* Autotuner (the paper specializes kernels on the order by just-in-time
 * compilation, sections "Ecosystem" and "libCEED"; here the variants are
 * precompiled and timed): time every valid launch shape of the apply of
 * precision prec on this operator's mesh with CUDA events (2 warm-up + 5
 * timed launches each), keep the fastest for the operator.  cache_path: NULL,
 * or a JSON file keyed by (GPU architecture, P, q, kind, collocation, ncomp,
 * precision, log2 E); a hit skips the timing, a miss adds the entry.
 * Allocates two temporary vectors; synchronizes. */
fem_status fem_op_autotune(fem_op *op, int prec, const char *cache_path,
                           fem_tune_result *result);

/* ---------------------------------------------------------------- solvers */

typedef struct {
  int precond;        /* FEM_PC_NONE, FEM_PC_JACOBI or FEM_PC_LEARNED */
  int maxit;          /* iteration cap (inner iterations for refinement) */
  double rtol;        /* stop when ||r||_2 <= rtol ||b||_2; 0 = run maxit */
  int use_graph;      /* 1: device-side loop in one CUDA graph (conditional
                         WHILE node); 0: one host launch sequence per step */
  double inner_rtol;  /* fem_solve_refined: relative tolerance of each inner
                         FP32 solve */
  int max_outer;      /* fem_solve_refined: outer FP64 refinement steps cap */
  int zero_guess;     /* fem_cg_solve: 1 = start from x = 0 (x's entries on
                         entry are ignored; the initial residual is b and no
                         apply is spent on it), 0 = x is the initial guess */
} fem_cg_opts;

typedef struct {
  int iterations;     /* CG iterations (total inner iterations if refined) */
  int outer;          /* refinement steps taken (0 for fem_cg_solve) */
  int status;         /* FEM_OK, FEM_ENOCONV or FEM_EBREAKDOWN */
  double rnorm;       /* final ||r||_2 of the recursive residual */
  double bnorm;       /* ||b||_2 over the unconstrained nodes */
  double true_rel;    /* refined: ||b - A_64 x|| / ||b|| in FP64 at exit */
  int fallback;       /* fem_fcg_solve: 1 if the learned part was switched off
                         (stagnation) and the solve finished with Jacobi */
} fem_cg_stats;

/* Preconditioned CG (section "Benchmarks": CG on the BP systems; diagonal
 * preconditioner as in Nekbone, section "Miniapps") on the Dirichlet-
 * constrained system  (M A M + (I - M)) x = b,  M = interior mask, FP64 apply.
 * b, x: device [ncomp*N]; x is the initial guess on entry (its Dirichlet
 * entries are set to 0; opts->zero_guess = 1 starts from 0 instead) and the
 * solution on exit.  Scalars stay on the
 * device; with use_graph = 1 the whole loop is one graph launch.  Copies the
 * statistics back (synchronizes).  Returns FEM_OK, FEM_ENOCONV (maxit reached
 * with rtol > 0) or FEM_EBREAKDOWN. */
fem_status fem_cg_solve(fem_op *op, const double *b, double *x,
                        const fem_cg_opts *opts, fem_cg_stats *stats);

/* Checkpoint and resume of a CG solve (fem_cg_solve) that stopped at its
 * iteration cap (status FEM_ENOCONV, or maxit reached with rtol = 0).  The
 * operator keeps that solve's state: r_k, z_k = M^-1 r_k, the previous
 * direction and the scalars (r^T z, beta, ||b||^2, iterations); x_k is the
 * caller's vector.
 *  fem_cg_checkpoint_size: bytes of the state (a header, the scalars, three
 *    ncomp*N FP64 vectors).
 *  fem_cg_checkpoint: copy the state to host memory of that size
 *    (synchronizes).  FEM_EINVAL if the operator has run no CG solve.
 *  fem_cg_restore: load a state into an operator of the same size (another
 *    process, or after the solve's workspace was reused); allocates the CG
 *    workspace if needed.  FEM_EINVAL for a buffer that is no checkpoint of
 *    that size.
 *  fem_cg_resume: continue from the state with x = x_k (device [ncomp*N])
 *    for at most opts->maxit further iterations to opts->rtol (relative to
 *    the original ||b||); opts->precond must be the interrupted solve's.  The
 *    iterates are those of the uninterrupted solve up to the order of the
 *    apply's atomic additions; stats->iterations counts from the original
 *    start.  Host-driven launches (no CUDA graph); synchronizes.  FEM_EINVAL
 *    when the last solve did not stop at its cap. */
fem_status fem_cg_checkpoint_size(const fem_op *op, int64_t *bytes);
fem_status fem_cg_checkpoint(fem_op *op, void *state_host);
fem_status fem_cg_restore(fem_op *op, const void *state_host);
fem_status fem_cg_resume(fem_op *op, const double *b, double *x,
                         const fem_cg_opts *opts, fem_cg_stats *stats);

/* ---------------------------------------------------------------- element-partitioned solve */

/* Host callbacks through which fem_pcg_dist exchanges data with the other
 * ranks (MPI, torch.distributed, ...).  Both return 0 on success; any other
 * value ends the solve with FEM_EINVAL.
 *  sum_interfaces(ctx, y): y is the caller's device work vector (the `y`
 *    argument of fem_pcg_dist, ncomp*N local entries); add to every entry
 *    of a node shared with other ranks their values of that node -- the
 *    action of the subdomain restriction's transpose P^T (section "libCEED";
 *    gslib's gather-scatter, section "Nek and MFEM").  The library has
 *    synchronized its stream before the call.
 *  allreduce(ctx, vals, count): vals is host memory; replace each of the
 *    count values by its sum over all ranks. */
typedef struct {
  void *ctx;
  int (*sum_interfaces)(void *ctx, double *y_dev);
  int (*allreduce)(void *ctx, double *vals_host, int count);
} fem_comm;

/* One rank's part of Jacobi-PCG (opts->precond FEM_PC_JACOBI) or plain CG
 * (FEM_PC_NONE) on an element-partitioned system: op is this rank's
 * operator on its local mesh (its elements, local node ids), the global
 * operator is the sum of the ranks' element operators.  owned: device [N]
 * bytes, 1 on the local nodes this rank owns (every global node owned by
 * exactly one rank); dot products sum over owned nodes and all-reduce.
 * b, x: device [ncomp*N] local entries of the assembled right-hand side and
 * of the solution (x is the initial guess unless opts->zero_guess);
 * y: device [ncomp*N] work vector handed to sum_interfaces.  Dirichlet
 * constraint and stopping test as fem_cg_solve (rtol relative to the global
 * ||b||).  The applies and vector updates are the library's kernels; each
 * iteration synchronizes the stream for one interface sum and two
 * all-reduces.  Allocates 4 ncomp*N work vectors for the call. */
fem_status fem_pcg_dist(fem_op *op, const uint8_t *owned, const double *b, double *x,
                        double *y, const fem_cg_opts *opts, const fem_comm *comm,
                        fem_cg_stats *stats);

/* Mixed-precision solve of the same constrained system: FP64 iterative
 * refinement (classical; the paper fixes only the operator and CG) around an
 * inner Jacobi-PCG (or plain CG) that runs the FP32 apply on FP32 vectors
 * with FP64 dot products and scalars.  Outer step: r = b - A_64 x (FP64
 * apply); stop when ||r|| <= rtol ||b||; else solve A_32 d = r to
 * inner_rtol (at most maxit inner iterations) and set x += d.  The operator
 * must have been created with FEM_F32.  Each outer step is one CUDA graph
 * launch; the host reads one status word per step (synchronizes).
 * stats: iterations = inner iterations in total, outer = corrections,
 * true_rel = ||b - A_64 x|| / ||b|| of the returned x.  Returns FEM_OK,
 * FEM_ENOCONV (max_outer reached) or FEM_EBREAKDOWN. */
fem_status fem_solve_refined(fem_op *op, const double *b, double *x,
                             const fem_cg_opts *opts, fem_cg_stats *stats);

/* Dirichlet-masked FP64 residual r = M (b - A x) (0 on constrained entries).
 * b, x, r: device [ncomp*N]; r must not alias b or x. */
fem_status fem_op_residual(fem_op *op, const double *b, const double *x,
                           double *r);

/* ---------------------------------------------------------------- learned preconditioner */

/* A per-element multilayer perceptron and its training (the paper has none;
 * its preconditioning material is the section "Ecosystem").  Network:
 *   h1 = relu(x W1^T + b1), h2 = relu(h1 W2^T + b2), y = h2 W3^T + b3,
 * x in R^n_in, hidden width n_h, y in R^n_out (all multiples of 32).
 * Parameters: one FP32 array in the order W1 [n_h][n_in], b1, W2 [n_h][n_h],
 * b2, W3 [n_out][n_h], b3 (FP32 masters, Adam moments on the device).
 * mode 0: GEMMs in bf16 on the tensor cores (tcgen05) with FP32
 * accumulation, activations in bf16; mode 1: all FP32 (reference/debug).
 * Row inputs X are bf16 (mode 0) or FP32 (mode 1), row-major [rows][n_in]. */
typedef struct fem_mlp fem_mlp;
fem_status fem_mlp_create(int n_in, int n_h, int n_out, int mode,
                          const float *params_host, void *stream, fem_mlp **out);
fem_status fem_mlp_destroy(fem_mlp *mlp);
/* Current parameters to host (params_host may be NULL) and their count. */
fem_status fem_mlp_params(fem_mlp *mlp, float *params_host, int64_t *count);
/* Save the network's state to a file: sizes, mode, the Adam step count,
 * the FP32 parameters and both Adam moment arrays (the format is the
 * library's own: an 8-byte tag, six int32, int64 count, 3 * count FP32).
 * fem_mlp_load creates a network from such a file on `stream`; training
 * continues from the saved step as if it had not stopped.  FEM_EINVAL when
 * the file cannot be opened or is not a saved network. */
fem_status fem_mlp_save(fem_mlp *mlp, const char *path);
fem_status fem_mlp_load(const char *path, void *stream, fem_mlp **out);
/* Y [rows][n_out] FP32 = network(X). */
fem_status fem_mlp_forward(fem_mlp *mlp, const void *X, int64_t rows, float *Y);
/* One Adam step (lr; b1 = 0.9, b2 = 0.999, eps = 1e-8) on the loss
 * (1/S) sum_rows ||y[:valid] - T[:valid]||^2 over S rows (a multiple of 32).
 * grad_host != NULL: copy the FP32 gradient out and do NOT update.
 * loss_host: the loss before the step.  Synchronizes. */
fem_status fem_mlp_train_step(fem_mlp *mlp, const void *X, const float *T,
                              int64_t S, int valid, float lr, float *grad_host,
                              double *loss_host);
/* Minibatch training: `epochs` passes over S rows in seeded random order,
 * floor(S/batch) Adam steps each; loss_host[epochs] = mean loss per epoch. */
fem_status fem_mlp_train(fem_mlp *mlp, const void *X, const float *T, int64_t S,
                         int valid, int epochs, int batch, float lr,
                         uint64_t seed, double *loss_host);

/* fem_mlp_train in chunks of `chunk` epochs (a fresh permutation seed per
 * chunk) until a chunk's mean loss is not below (1 - rel_tol) times the
 * previous chunk's, or max_epochs have run.  loss_host[max_epochs] receives
 * the mean loss of every epoch run, *epochs_run their number. */
fem_status fem_mlp_train_plateau(fem_mlp *mlp, const void *X, const float *T, int64_t S,
                                 int valid, int max_epochs, int chunk, double rel_tol,
                                 int batch, float lr, uint64_t seed, double *loss_host,
                                 int *epochs_run);

/* The learned preconditioner of a scalar FEM_F32 operator:
 *   z = dinv * r + sum_e G_e^T ( w * ||r_e|| * net([r_e / ||r_e||, g_e]) )
 * g_e: 32 element features (the 8 corner nodes' offsets from the centroid
 * divided by the element size, then log kappa at the corners); w = 1 / node
 * multiplicity.  mlp == NULL gives the Jacobi part alone.  The network needs
 * n_in >= (p+1)^3 + 32 and n_out >= (p+1)^3; both must outlive the
 * preconditioner. */
typedef struct fem_precond fem_precond;
fem_status fem_precond_create(fem_op *op, fem_mlp *mlp, fem_precond **out);
fem_status fem_precond_destroy(fem_precond *pc);
/* Element features [E][32] to host. */
fem_status fem_precond_features(fem_precond *pc, float *feat_host);
/* Training rows (E of them) from an iterate x_k of the plain solver for the
 * right-hand side b whose solution is x_star (device FP64 [N] each): with
 * r = M (b - A x_k) and e = x_star - x_k, per element
 * X = [r_e / ||r_e||, g_e, 0...] (network input type) and
 * T = [e_e / ||r_e||, 0...] (FP32, n_out wide). */
fem_status fem_precond_samples(fem_precond *pc, const double *b,
                               const double *x_star, const double *x_k,
                               void *X, float *T);
/* Weight gamma >= 0 of the learned correction in B (default 1; 0 = Jacobi
 * alone, the network is then skipped). */
fem_status fem_precond_set_gamma(fem_precond *pc, double gamma);
/* Pick gamma among gammas[0..n): for each candidate run probe_iters
 * flexible-CG iterations (one refinement step) on right-hand side b from
 * x = 0 (x: device [N] work vector, overwritten) and keep the candidate with
 * the smallest true residual; a candidate whose solve switched the learned
 * part off (fallback) never wins.  Include 0 among the candidates to let
 * Jacobi alone win.  Sets the preconditioner's gamma to the winner and
 * returns it in *best_gamma.  Synchronizes. */
fem_status fem_precond_calibrate(fem_precond *pc, const double *b, double *x,
                                 const double *gammas, int n, int probe_iters,
                                 double *best_gamma);
/* z = B(r) (device FP32 [N] each). */
fem_status fem_precond_apply(fem_precond *pc, const float *r, float *z);
/* Flexible CG (Notay 2000, one stored direction) with preconditioner B as
 * the inner FP32 solve of FP64 iterative refinement (as fem_solve_refined).
 * Each outer step is one CUDA graph; the learned correction sits in a
 * conditional IF node.  The direction carries over between outer steps with
 * its preconditioned-residual part replaced (p += z_new - z_old), so with the
 * Jacobi part alone the iteration counts track fem_solve_refined.  Fallback: every 64 inner iterations the residual
 * must have dropped 4x, else the learned part is switched off for the rest
 * of the solve (stats->fallback = 1), which then is Jacobi-PCG.  opts: rtol,
 * inner_rtol, maxit, max_outer (precond is implied).  Synchronizes. */
fem_status fem_fcg_solve(fem_precond *pc, const double *b, double *x,
                         const fem_cg_opts *opts, fem_cg_stats *stats);

/* ---------------------------------------------------------------- batches */

typedef struct fem_batch fem_batch;

/* A batch of independent problems solved together (no counterpart in the
 * paper beyond batching small products across elements, section
 * "Ecosystem").  ops: n operators (1 <= n <= 1024), each a diffusion
 * operator with Gauss q = p+2 (BP3/BP4 type, any order and size) created
 * with FEM_F32, all on one stream.  The batch keeps pointers to the
 * operators (they must outlive it) and allocates the per-problem inner
 * vectors.  fem_batch_create_split: problems with ncomp*N >= solo_dofs are
 * not put in the persistent kernel but solved one after another by
 * fem_solve_refined, whose order-specialized kernels run a large problem
 * faster than the persistent kernel's all-orders body; solo_dofs <= 0 puts
 * every problem in the persistent kernel.  fem_batch_create uses
 * FEM_BATCH_SOLO_DOFS. */
#define FEM_BATCH_SOLO_DOFS (1LL << 21)
fem_status fem_batch_create(fem_op *const *ops, int n, fem_batch **out);
fem_status fem_batch_create_split(fem_op *const *ops, int n, int64_t solo_dofs,
                                  fem_batch **out);
fem_status fem_batch_destroy(fem_batch *batch);

/* Solve every problem i: (M A_i M + (I - M)) x_i = b_i with the method of
 * fem_solve_refined (FP64 refinement, FP32 inner Jacobi-PCG, FP64 dots), all
 * problems in lockstep outer steps; the inner iterations of all problems of
 * one outer step run in ONE persistent cooperative kernel (work items:
 * (problem, element group) and (problem, vector chunk); grid barriers with a
 * wall-clock limit).  The outer loop runs as one CUDA graph (conditional
 * WHILE node over the refinement steps, captured at the first solve and
 * re-captured when the options or the launch shape change); where the runtime
 * refuses to capture the cooperative launch, the steps are launched from the
 * host instead (fem_batch_graph_state).  Problems split off at creation are
 * solved first, one after another.  b, x: host arrays of n device pointers.  opts: precond
 * must be FEM_PC_JACOBI; rtol, inner_rtol, maxit (inner cap per step),
 * max_outer as in fem_solve_refined.  stats: host array of n (or NULL).
 * Returns the first non-OK problem status, or FEM_ETIMEOUT if a barrier ran
 * out (the batch stays usable).  Synchronizes. */
fem_status fem_batch_solve(fem_batch *batch, const double *const *b,
                           double *const *x, const fem_cg_opts *opts,
                           fem_cg_stats *stats);
/* How the persistent part's refinement loop runs: 1 = one captured CUDA graph,
 * 0 = not captured yet (no solve so far, or nothing in the persistent
 * kernel), -1 = capture refused by the runtime, host-launched steps. */
fem_status fem_batch_graph_state(const fem_batch *batch, int *state);

/* Launch shape of the persistent kernel: block size choice (0: 128, 1: 256,
 * 2: 512 threads), blocks per SM (0 = occupancy maximum) and the barrier
 * wall-clock limit in ms.  (A batch whose problems are all split off has
 * no persistent kernel: set_shape and autotune then do nothing.) */
fem_status fem_batch_set_shape(fem_batch *batch, int nt_choice,
                               int blocks_per_sm, double timeout_ms);

/* Autotuner of the batch: time `iters` inner iterations of the persistent
 * kernel for every (block size, blocks per SM) candidate from the same start
 * state (b, x as in fem_batch_solve; x is not modified), keep the fastest.
 * result->epb_choice holds the block size choice, result->us the time of one
 * inner iteration of the whole batch. */
fem_status fem_batch_autotune(fem_batch *batch, const double *const *b,
                              double *const *x, int iters,
                              fem_tune_result *result);

/* Self-test of the bounded grid barrier: launches the persistent kernel with
 * one arrival that never comes; the first barrier runs out after timeout_ms
 * and the call returns FEM_ETIMEOUT with the batch still usable.  Requires a
 * previous fem_batch_solve (it reuses the bound vectors). */
fem_status fem_batch_barrier_selftest(fem_batch *batch, double timeout_ms);

/* ---------------------------------------------------------------- p-multigrid */
/* p-multigrid preconditioner (section "Ecosystem": multigrid on a hierarchy
 * of polynomial degrees of one mesh, with matrix-free smoothers) and flexible
 * CG around it.  The paper fixes no details; this library's choices:
 *  - levels[0] is the finest operator, levels[nlevels-1] the coarsest; all
 *    on meshes of the same elements in the same order (Gauss-Lobatto nodes,
 *    element-local node order a + P b + P^2 c), with the kind, ncomp and
 *    stream of level 0 and strictly decreasing orders; each level is its own
 *    discretization (its own quadrature).  The hierarchy does not own them.
 *  - prolongation level l+1 -> l: coarse element values interpolated at the
 *    fine element's nodes (1D coarse Lagrange basis per direction), averaged
 *    on shared nodes (weight 1 / multiplicity); restriction = its transpose;
 *    both act on Dirichlet-masked vectors (zero on the levels' boundary).
 *  - smoother: cheb_degree steps of the Chebyshev iteration (Saad 2003,
 *    Alg. 12.1) on D^-1 A over [cheb_lo, cheb_hi] * lmax; lmax of each
 *    smoothed level from power_its power iterations (FP64, at create) from
 *    the SplitMix64 vector u_i = (splitmix64_i(seed 0) >> 11) 2^-53 - 1/2,
 *    with the Rayleigh quotient v^T A v / v^T D v.
 *  - coarsest level: coarse_its Jacobi-PCG iterations from zero.
 *  - V-cycle: z = S(r); z += P V(R(r - A z)); z += S(r - A z), in FP64 or,
 *    with prec = FEM_F32, on the levels' FP32 operators and vectors with
 *    FP64 dot products (the levels must then be created with FEM_F32).
 * Vectors are device [ncomp*N] FP64 of the level they belong to. */
typedef struct fem_pmg fem_pmg;
typedef struct {
  int cheb_degree;    /* Chebyshev steps per smoothing, >= 1 (default 4) */
  double cheb_lo;     /* smoothing interval [cheb_lo, cheb_hi] * lmax */
  double cheb_hi;     /*   (defaults 0.1 and 1.1) */
  int power_its;      /* power iterations for lmax, >= 1 (default 20) */
  int coarse_its;     /* coarsest-level Jacobi-PCG iterations, >= 1 (30) */
  int prec;           /* FEM_F64 or FEM_F32: precision of the V-cycle */
} fem_pmg_opts;

/* opts may be NULL (the defaults).  FEM_EINVAL for an inconsistent
 * hierarchy, FEM_ENOMEM, FEM_EBREAKDOWN if a power iteration degenerates.
 * Synchronizes the levels' stream. */
fem_status fem_pmg_create(fem_op *const *levels, int nlevels, const fem_pmg_opts *opts,
                          fem_pmg **out);
fem_status fem_pmg_destroy(fem_pmg *pmg);
/* lmax of a level (0 for the coarsest, which is not smoothed). */
fem_status fem_pmg_get_lmax(const fem_pmg *pmg, int level, double *lmax);
/* Override lmax of a smoothed level (lmax > 0). */
fem_status fem_pmg_set_lmax(fem_pmg *pmg, int level, double lmax);
/* xf = P xc, level+1 -> level (xf overwritten); FP64. */
fem_status fem_pmg_prolong(fem_pmg *pmg, int level, const double *xc, double *xf);
/* rc = R rf, level -> level+1 (rc overwritten); FP64. */
fem_status fem_pmg_restrict(fem_pmg *pmg, int level, const double *rf, double *rc);
/* z = B r, one V-cycle (r, z: level 0, FP64; r is only read).  The V-cycle
 * is one CUDA graph, captured at the first call. */
fem_status fem_pmg_vcycle(fem_pmg *pmg, const double *r, double *z);
/* Flexible CG (Notay 2000, one stored direction) in FP64 on the constrained
 * level-0 system with z = B r; x is the initial guess (its Dirichlet entries
 * are kept).  opts: rtol (on the recursive residual, ||r|| <= rtol ||b||)
 * and maxit; the rest is ignored.  One CUDA graph with a conditional WHILE
 * node; synchronizes.  stats: iterations, rnorm, bnorm, true_rel = rnorm /
 * bnorm.  FEM_OK, FEM_ENOCONV or FEM_EBREAKDOWN. */
fem_status fem_pmg_solve(fem_pmg *pmg, const double *b, double *x, const fem_cg_opts *opts,
                         fem_cg_stats *stats);
/* The V-cycle as the preconditioner of fem_fcg_solve: B(r) = V(r), one FP32
 * V-cycle (the hierarchy must have prec = FEM_F32 and a scalar finest level;
 * it must outlive the preconditioner).  fem_fcg_solve then runs flexible CG
 * in FP32 with FP64 iterative refinement around it: the FP64 operator is
 * applied once per refinement step instead of once per iteration as in
 * fem_pmg_solve.  fem_precond_apply gives z = V(r); set_gamma, features and
 * samples do not apply. */
fem_status fem_precond_create_pmg(fem_pmg *pmg, fem_precond **out);

/* ------------------------------------------------------- allocation-free solve */

/* Largest ncomp*N accepted by fem_cg_solve_noalloc. */
#define FEM_NOALLOC_MAX_N 131072

/* The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory while they solve: code that works inside
 * a device-memory budget fixed at start-up, or a real-time loop in which
 * cudaMalloc's implicit device-wide synchronization is not acceptable.
 *
 * Same arguments, arithmetic and results as fem_cg_solve (FEM_PC_NONE or
 * FEM_PC_JACOBI; opts->zero_guess is honoured as there; launches are
 * host-driven, no CUDA graph, so opts->use_graph is ignored), but the CG
 * workspace (five vectors, reduction partials, scalars) lives in one fixed
 * file-scope device array of the library instead of cudaMalloc'd buffers, so
 * the call allocates nothing.  The array holds 5 * FEM_NOALLOC_MAX_N doubles
 * plus about 260 KB and is held on every GPU that loads the library until the
 * process exits.
 *  - ncomp*N > FEM_NOALLOC_MAX_N: FEM_EINVAL with a message naming the limit.
 *  - The first call on a device looks up the array's device address (with
 *    that device current); make that first call before any stream capture.
 *  - Every call shares the array and it keeps the previous call's contents;
 *    each call rewrites what it reads first.  Calls that overlap on the GPU
 *    (other streams, other host threads) race on it and give wrong results.
 *  - The operator itself was allocated by fem_op_create; b and x are the
 *    caller's device buffers.  Synchronizes the operator's stream. */
fem_status fem_cg_solve_noalloc(fem_op *op, const double *b, double *x,
                                const fem_cg_opts *opts, fem_cg_stats *stats);

#ifdef __cplusplus
}
#endif
#endif /* FEM_H */
