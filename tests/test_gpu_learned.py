"""GPU tests of the learned preconditioner: the network's forward and
backward against the FP64 CPU oracle (oracle/mlp.c), training, the element
features and samples, and flexible CG with the trained network (final error
judged by the FP64 oracle)."""
import numpy as np
import pytest
import torch

import fem_inputs
import oracle
import paper_2109_04996_b300 as fem
from paper_2109_04996_b300 import build as fembuild

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    fembuild.build()
    assert torch.cuda.is_available()


def rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300)


DIMS = (96, 64, 64)


def _data(S, seed=0):
    rng = np.random.default_rng(seed)
    x = rng.normal(0, 1, (S, DIMS[0]))
    t = rng.normal(0, 0.3, (S, DIMS[2]))
    return x, t


@pytest.mark.parametrize("mode,tol", [(1, 1e-5), (0, 2e-2)])
def test_forward_matches_oracle(mode, tol):
    p = fem_inputs.mlp_init(*DIMS, seed=1, out_scale=1.0)
    net = fem.Mlp(*DIMS, p, mode=mode)
    x, _ = _data(200)
    X = torch.from_numpy(x).to(net.input_dtype).cuda()
    y = net.forward(X).double().cpu().numpy()
    xin = X.double().cpu().numpy()           # the rounded input the GPU saw
    yr, _, _ = oracle.mlp_forward(DIMS, p.astype(np.float64), xin)
    assert rel(y, yr) <= tol


@pytest.mark.parametrize("dims,S", [((160, 256, 128), 1000), ((256, 256, 256), 389), ((32, 128, 32), 129)])
def test_tensor_core_forward_matches_oracle(dims, S):
    # mode 0: the forward products run on tcgen05 (bf16 in, FP32 in tensor
    # memory); the hidden activations are stored in bf16 between layers
    p = fem_inputs.mlp_init(*dims, seed=4, out_scale=1.0)
    net = fem.Mlp(*dims, p, mode=0)
    x = np.random.default_rng(5).normal(0, 1, (S, dims[0]))
    X = torch.from_numpy(x).to(net.input_dtype).cuda()
    y = net.forward(X).double().cpu().numpy()
    yr, _, _ = oracle.mlp_forward(dims, p.astype(np.float64), X.double().cpu().numpy())
    assert rel(y, yr) <= 2e-2


def _bf16(a):
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).double().numpy()


@pytest.mark.parametrize("mode,tol,seed", [(1, 1e-5, 2), (0, 1e-2, 2), (0, 1e-2, 3), (0, 1e-2, 4)])
def test_gradient_matches_oracle(mode, tol, seed):
    """Mode 1 (FP32): the FP64 oracle's gradient to 1e-5.  Mode 0: the tensor
    cores multiply the bf16 roundings of the FP32 master weights (and of the
    bf16 input rows), so the oracle differentiates that network -- the FP32
    masters rounded to bf16 -- and the remaining differences are the bf16
    storage of the hidden activations and FP32 accumulation: 1e-2 relative
    (measured 2.9e-3 .. 5.8e-3 over these seeds)."""
    p = fem_inputs.mlp_init(*DIMS, seed=seed, out_scale=1.0)
    net = fem.Mlp(*DIMS, p, mode=mode)
    x, t = _data(256, seed=seed + 1)
    valid = 50
    t[:, valid:] = 0.0
    X = torch.from_numpy(x).to(net.input_dtype).cuda()
    T = torch.from_numpy(t).float().cuda()
    L, g = net.gradient(X, T, valid)
    xin = X.double().cpu().numpy()
    # the oracle's loss over the first `valid` outputs: zero the other outputs' rows of W3, b3
    n_in, n_h, n_out = DIMS
    pv = (p.astype(np.float64) if mode == 1 else _bf16(p)).copy()
    off3 = n_h * n_in + n_h + n_h * n_h + n_h
    W3 = pv[off3:off3 + n_out * n_h].reshape(n_out, n_h)
    W3[valid:] = 0.0
    pv[off3 + n_out * n_h + valid:] = 0.0
    Lr, gr = oracle.mlp_loss_grad(DIMS, pv, xin, np.where(np.arange(n_out) < valid, t, 0.0))
    gm = g.astype(np.float64)
    keep = np.ones_like(gm, dtype=bool)    # outputs >= valid carry no gradient on the GPU side
    keep[off3:off3 + n_out * n_h] = (np.arange(n_out)[:, None] < valid).repeat(n_h, 1).ravel()
    keep[off3 + n_out * n_h:] = np.arange(n_out) < valid
    assert abs(L - Lr) <= tol * Lr
    assert rel(gm[keep], gr[keep]) <= tol


def test_adam_step_matches_oracle():
    p = fem_inputs.mlp_init(*DIMS, seed=4, out_scale=1.0)
    net = fem.Mlp(*DIMS, p, mode=1)
    x, t = _data(128, seed=5)
    X = torch.from_numpy(x).float().cuda()
    T = torch.from_numpy(t).float().cuda()
    _, g = net.gradient(X, T, DIMS[2])
    net.step(X, T, DIMS[2], 1e-3)
    q = p.astype(np.float64).copy()
    m = np.zeros_like(q); v = np.zeros_like(q)
    oracle.adam_step(q, g.astype(np.float64), m, v, 1, lr=1e-3)
    assert rel(net.params(), q) <= 1e-6


@pytest.mark.parametrize("mode", [1, 0])
def test_save_load_resumes_training(mode, tmp_path):
    """Train 6 Adam steps, save, load into a new network: parameters and both
    moments come back exactly, and 4 more steps on both networks give the
    same parameters (a network that lost its Adam moments or step count
    takes a different step: checked with a fresh-moment copy)."""
    x, t = _data(512, seed=11)
    p0 = fem_inputs.mlp_init(*DIMS, seed=12, out_scale=1.0)
    net = fem.Mlp(*DIMS, p0, mode=mode)
    X = torch.from_numpy(x).to(net.input_dtype).cuda()
    T = torch.from_numpy(t).float().cuda()
    for _ in range(6):
        net.step(X, T, DIMS[2], 1e-3)
    path = str(tmp_path / "net.bin")
    net.save(path)
    net2 = fem.Mlp.load(path)
    assert (net2.n_in, net2.n_h, net2.n_out, net2.mode) == DIMS + (mode,)
    assert np.array_equal(net2.params(), net.params())
    fresh = fem.Mlp(*DIMS, net.params(), mode=mode)      # same weights, no Adam state
    for _ in range(4):
        net.step(X, T, DIMS[2], 1e-3)
        net2.step(X, T, DIMS[2], 1e-3)
        fresh.step(X, T, DIMS[2], 1e-3)
    a, b, c = net.params(), net2.params(), fresh.params()
    assert rel(b, a) <= 1e-6
    assert rel(c, a) > 1e-4
    with open(path, "r+b") as f:                          # a damaged file is refused
        f.write(b"NOTANMLP")
    with pytest.raises(fem.FemError):
        fem.Mlp.load(path)


@pytest.mark.parametrize("mode", [0, 1])
def test_training_reduces_the_loss(mode):
    # a learnable map: t = tanh(x A) for a fixed random A
    rng = np.random.default_rng(7)
    A = rng.normal(0, 0.2, (DIMS[0], DIMS[2]))
    x = rng.normal(0, 1, (8192, DIMS[0]))
    t = np.tanh(x @ A)
    net = fem.Mlp(*DIMS, fem_inputs.mlp_init(*DIMS, seed=8), mode=mode)
    X = torch.from_numpy(x).to(net.input_dtype).cuda()
    T = torch.from_numpy(t).float().cuda()
    losses = net.train(X, T, DIMS[2], epochs=15, batch=512, lr=2e-3, seed=1)
    assert losses[-1] < 0.5 * losses[0], losses
    assert all(b < a for a, b in zip(losses[:-1], losses[1:]))


def _kappa_problem(n=4, p=4, seed=11):
    rff = fem_inputs.rff_params(128, 0.1, seed=seed)
    m = fem_inputs.box_mesh(n, p, perturb=0.1, seed=seed)
    gm = fem.Mesh(m)
    op = fem.Operator.bake_off(gm, "BP3", prec=fem.F32, rff=rff)
    return m, gm, op, rff


def test_features_and_samples():
    m, gm, op, rff = _kappa_problem(n=3, p=2)
    n_in = 64 if 27 + 32 <= 64 else 96
    net = fem.Mlp(n_in, 64, 32, fem_inputs.mlp_init(n_in, 64, 32), mode=1)
    pc = fem.Precond(op, net)
    f = pc.features()
    # corners of element e are its trilinear vertices; h = side of the cube
    orc = oracle.Operator(m, oracle.DIFFUSION, oracle.GAUSS, 4, rff=rff)
    V = m["vert_xyz"][m["elem_verts"]]                  # [E, 8, 3]
    cen = V.mean(1, keepdims=True)
    h = 2 / np.sqrt(3) * np.sqrt(((V - cen) ** 2).sum((1, 2)) / 8)
    np.testing.assert_allclose(f[:, :24], ((V - cen) / h[:, None, None]).reshape(-1, 24), atol=1e-5)
    lk = np.array([[np.log(orc.kappa(V[e, v])) for v in range(8)] for e in range(m["E"])])
    np.testing.assert_allclose(f[:, 24:], lk, atol=1e-5)
    # samples: X = [r_e/|r_e|, g_e, 0], T = [e_e/|r_e|, 0]
    b = torch.from_numpy(fem_inputs.rhs_uniform(m["N"], m["dirichlet"], seed=1)).cuda()
    xs = torch.from_numpy(np.random.default_rng(2).uniform(-1, 1, m["N"])).cuda()
    xk = torch.from_numpy(np.random.default_rng(3).uniform(-1, 1, m["N"])).cuda()
    X = torch.zeros(m["E"], n_in, dtype=torch.float32, device="cuda")
    T = torch.zeros(m["E"], 32, dtype=torch.float32, device="cuda")
    pc.samples(b, xs, xk, X, T)
    inner = m["dirichlet"] == 0
    r = np.where(inner, b.cpu().numpy() - orc.apply(xk.cpu().numpy()), 0.0)
    err = xs.cpu().numpy() - xk.cpu().numpy()
    en = m["elem_nodes"]
    nr = np.linalg.norm(r[en], axis=1)
    np.testing.assert_allclose(X.cpu().numpy()[:, :27], r[en] / nr[:, None], atol=2e-6)
    np.testing.assert_allclose(X.cpu().numpy()[:, 27:59], f, atol=0)
    np.testing.assert_allclose(T.cpu().numpy()[:, :27], err[en] / nr[:, None], rtol=1e-5, atol=1e-5)


@pytest.mark.parametrize("mode,tol", [(1, 1e-5), (0, 2e-2)])
@pytest.mark.parametrize("gamma", [1.0, 0.37])
def test_precond_apply_matches_oracle(mode, tol, gamma):
    """z = B(r) element-wise against oracle/learned.py on a kappa mesh with
    shuffled elements (27 elements: a ragged warp and block tail).  Mode 1
    (FP32 network): 1e-5.  Mode 0 (bf16 inputs, weights and hidden
    activations on the tensor cores): the forward's bf16 bound, 2e-2 relative
    on the learned correction (the Jacobi part is exact in FP32)."""
    from oracle import learned
    rff = fem_inputs.rff_params(128, 0.1, seed=17)
    m = fem_inputs.box_mesh(3, 2, perturb=0.1, seed=17, shuffle_seed=4)
    gm = fem.Mesh(m)
    op = fem.Operator.bake_off(gm, "BP3", prec=fem.F32, rff=rff)
    dims = (64, 64, 32)
    params = fem_inputs.mlp_init(*dims, seed=6, out_scale=1.0)
    net = fem.Mlp(*dims, params, mode=mode)
    pc = fem.Precond(op, net)
    pc.set_gamma(gamma)
    orc = oracle.Operator(m, oracle.DIFFUSION, oracle.GAUSS, 4, rff=rff)
    diag = orc.diagonal()
    feat = learned.features(m, rff=rff)
    # a residual with element norms over several decades
    rng = np.random.default_rng(8)
    r = rng.uniform(-1, 1, m["N"]) * np.exp(rng.uniform(-4, 2, m["N"]))
    r = np.where(m["dirichlet"] == 0, r, 0.0).astype(np.float32).astype(np.float64)
    z = pc.apply(torch.from_numpy(r).float().cuda()).double().cpu().numpy()
    zo = learned.precond_apply(m, diag, dims, params.astype(np.float64), r, gamma, feat)
    z0 = learned.precond_apply(m, diag, dims, params.astype(np.float64), r, 0.0, feat)
    assert np.linalg.norm(zo - z0) > 0.1 * np.linalg.norm(z0)   # the network part matters
    assert rel(z - z0, zo - z0) <= tol
    assert rel(z, zo) <= tol
    assert np.all(z[m["dirichlet"] == 1] == 0.0)


def test_fcg_jacobi_only_converges_like_pcg():
    m, gm, op, rff = _kappa_problem(n=5, p=3)
    b = torch.from_numpy(fem_inputs.rhs_uniform(m["N"], m["dirichlet"], seed=3)).cuda()
    pc = fem.Precond(op, None)
    x = torch.zeros_like(b)
    st = pc.fcg(b, x, rtol=1e-10)
    assert st["status"] == "FEM_OK" and st["true_rel"] <= 1e-10
    x2 = torch.zeros_like(b)
    st2 = op.solve_refined(b, x2, rtol=1e-10, inner_rtol=0.1)
    # with a fixed SPD preconditioner flexible CG is CG in exact arithmetic,
    # and both keep their direction across the FP64 residual replacements:
    # the counts differ only by FP32 rounding (beta formulas differ)
    assert abs(st["iterations"] - st2["iterations"]) <= max(8, 0.2 * st2["iterations"])
    assert rel(x.cpu().numpy(), x2.cpu().numpy()) <= 1e-8


def _train_learned(op, m, nrhs=6, ks=(2, 5, 10, 20, 40, 80), epochs=40, mode=0, seed=0):
    P3 = (m["p"] + 1) ** 3
    n_in = ((P3 + 32 + 31) // 32) * 32
    n_out = ((P3 + 31) // 32) * 32
    net = fem.Mlp(n_in, 256, n_out, fem_inputs.mlp_init(n_in, 256, n_out, seed=seed), mode=mode)
    pc = fem.Precond(op, net)
    rows = nrhs * len(ks) * m["E"]
    X = torch.zeros(rows, n_in, dtype=net.input_dtype, device="cuda")
    T = torch.zeros(rows, n_out, dtype=torch.float32, device="cuda")
    r0 = 0
    for j in range(nrhs):
        b = torch.from_numpy(fem_inputs.rhs_uniform(m["N"], m["dirichlet"], seed=100 + j)).cuda()
        xs = torch.zeros_like(b)
        op.solve_refined(b, xs, rtol=1e-12, inner_rtol=1e-5)
        for k in ks:
            xk = torch.zeros_like(b)
            op.cg(b, xk, maxit=k, rtol=0.0)
            pc.samples(b, xs, xk, X[r0:r0 + m["E"]], T[r0:r0 + m["E"]])
            r0 += m["E"]
    batch = max(32, min(1024, (rows // 8) // 32 * 32))
    scale = torch.sqrt(torch.mean(T[:, :P3].double() ** 2)).item()
    T /= scale
    losses = net.train_plateau(X, T, P3, max_epochs=epochs, chunk=4, rel_tol=0.01, batch=batch,
                               lr=1e-3, seed=seed)
    return net, pc, losses, scale


def test_learned_fcg_reaches_fp64_accuracy_and_reports_its_gain():
    m, gm, op, rff = _kappa_problem(n=6, p=4)
    net, pc, losses, scale = _train_learned(op, m)
    # normalized targets (unit RMS over the P^3 outputs): predicting zero
    # scores P^3 = 125; the network must explain a good part of that, and
    # training stops at a plateau (or the epoch cap)
    P3 = (m["p"] + 1) ** 3
    assert losses[0] < 1.2 * P3 and losses[-1] < 0.8 * losses[0]
    # the chunked training stopped at its plateau rule or at the 40-epoch cap
    assert len(losses) == 40 or losses[-4:].mean() >= 0.99 * losses[-8:-4].mean()
    bval = torch.from_numpy(fem_inputs.rhs_uniform(m["N"], m["dirichlet"], seed=998)).cuda()
    gammas = [scale * g for g in (2.0, 1.0, 0.5, 0.25, 0.1)] + [0.0]
    gamma = pc.calibrate(bval, gammas=gammas)
    assert gamma in gammas
    b = torch.from_numpy(fem_inputs.rhs_uniform(m["N"], m["dirichlet"], seed=999)).cuda()
    x = torch.zeros_like(b)
    st = pc.fcg(b, x, rtol=1e-10)
    assert st["status"] == "FEM_OK" and st["true_rel"] <= 1e-10
    orc = oracle.Operator(m, oracle.DIFFUSION, oracle.GAUSS, 6, rff=rff)
    inner = m["dirichlet"] == 0
    bn = b.cpu().numpy()
    res = np.where(inner, bn - orc.apply(x.cpu().numpy()), 0.0)
    assert np.linalg.norm(res) <= 1.05e-10 * np.linalg.norm(bn)
    # the method without the network on the same system
    x0 = torch.zeros_like(b)
    st0 = fem.Precond(op, None).fcg(b, x0, rtol=1e-10)
    gain = st0["iterations"] / st["iterations"]
    print("\nlearned FCG: gamma %.2f, %d iterations (fallback %d) vs Jacobi %d: gain %.2fx;"
          " training loss %.3g -> %.3g" % (gamma, st["iterations"], st["fallback"],
                                          st0["iterations"], gain, losses[0], losses[-1]))
    # what the bench reports: the calibrated preconditioner never loses to
    # Jacobi-FCG beyond the iteration noise of FP32 inner solves
    assert st["iterations"] <= 1.02 * st0["iterations"] + 2, (gamma, st, st0)


def test_bad_network_falls_back_to_jacobi_and_still_converges():
    m, gm, op, rff = _kappa_problem(n=5, p=3)
    P3 = 64
    net = fem.Mlp(96, 64, 64, fem_inputs.mlp_init(96, 64, 64, seed=3, out_scale=30.0), mode=0)
    pc = fem.Precond(op, net)
    pc.set_gamma(1.0)
    b = torch.from_numpy(fem_inputs.rhs_uniform(m["N"], m["dirichlet"], seed=5)).cuda()
    x = torch.zeros_like(b)
    st = pc.fcg(b, x, rtol=1e-10)
    assert st["status"] == "FEM_OK" and st["true_rel"] <= 1e-10
    assert st["fallback"] == 1
    # gamma = 0 is the Jacobi method (no network work at all)
    pc.set_gamma(0.0)
    x0 = torch.zeros_like(b)
    st0 = pc.fcg(b, x0, rtol=1e-10)
    assert st0["fallback"] == 0 and st0["true_rel"] <= 1e-10
