"""GPU parity of the wavelet-domain deblurring solver (Section 4.3; FISTA-W / FISTA-WP of the
appendix on deblurring algorithms) and of its building blocks -- the adjoint product, the
Jacobi diagonal diag(Theta^T Theta) and the power iteration -- against the FP64 oracle run on
the oracle's own Theta (restricted to the pattern)."""
import numpy as np
import pytest

import oracle
import pc_inputs as P
from helpers import dense_theta_pattern, make_gpu_op

pytestmark = pytest.mark.gpu

CASES = [("small-1d", {}), ("small-2d", {"n": 32, "levels": 3}), ("small-2d", {"n": 32, "levels": 3, "order": 1}),
         ("small-2d", {"n": 64, "levels": 4, "delta": 3}), ("op1", {"n": 32, "levels": 3})]


@pytest.fixture(scope="module")
def pw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_09870_gb300 as m
    return m


def _setup(pw, name, kw, prec):
    op = P.workload(name, **kw)
    g = make_gpu_op(pw, op, precision=prec)
    g.assemble()
    return op, g, dense_theta_pattern(op)


def _problem(op, T, seed):
    """Sparse wavelet coefficients seen through Theta plus 1% noise, and seeded weights."""
    N = op.N
    zt = P.normal(seed, N) * (P.uniform(seed + 1, N) < 0.1)
    z0 = T @ zt + 0.01 * P.normal(seed + 2, N)
    w = 0.02 * (0.5 + P.uniform(seed + 3, N))
    return z0, w


@pytest.mark.parametrize("name,kw", CASES)
@pytest.mark.parametrize("nrhs", [1, 5, 16])
@pytest.mark.parametrize("prec", [0, 1])
def test_adjoint_matches_oracle(pw, name, kw, nrhs, prec):
    import torch
    op, g, T = _setup(pw, name, kw, prec)
    dt = torch.float64 if prec else torch.float32
    x = P.normal(P.BASE_SEED + 71, op.N * nrhs).reshape(op.N, nrhs)
    y = g.apply_adjoint(torch.tensor(x, dtype=dt, device="cuda"))
    g.sync()
    ref = T.T @ x
    rel = np.linalg.norm(y.double().cpu().numpy() - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert rel.max() <= (1e-12 if prec else 1e-5), rel


@pytest.mark.parametrize("name,kw", CASES)
@pytest.mark.parametrize("prec", [0, 1])
def test_jacobi_and_power_norm(pw, name, kw, prec):
    op, g, T = _setup(pw, name, kw, prec)
    J = g.jacobi()
    g.sync()
    Jo = oracle.jacobi(T)
    # FP32 stored values carry up to 1e-5 of the largest entry; squaring doubles that
    tol = 1e-12 if prec else 2e-5
    assert np.abs(J.double().cpu().numpy() - Jo).max() <= tol * Jo.max()
    for iters, sigma in ((1, None), (20, None), (20, 1.0 / Jo)):
        s_d = None
        if sigma is not None:
            import torch
            s_d = torch.tensor(sigma, dtype=g.dtype, device="cuda")
        got = g.power_norm(sigma=s_d, iters=iters)
        want = oracle.power_norm(T, iters, sigma=sigma)
        # eigenvalues of Theta^T Theta move by up to twice the relative value error
        assert abs(got - want) <= (1e-11 if prec else 4e-5) * want, (iters, got, want)


@pytest.mark.parametrize("name,kw", CASES)
@pytest.mark.parametrize("precond", [False, True])
@pytest.mark.parametrize("prec", [0, 1])
def test_fista_matches_oracle(pw, name, kw, precond, prec):
    import torch
    op, g, T = _setup(pw, name, kw, prec)
    z0, w = _problem(op, T, P.BASE_SEED + 90)
    sigma = 1.0 / oracle.jacobi(T) if precond else None
    tau = 0.95 / oracle.power_norm(T, 100, sigma=sigma)
    dt = g.dtype
    iters = 40
    want = oracle.fista(T, z0, w, iters, tau, sigma=sigma)
    z = g.fista(torch.tensor(z0, dtype=dt, device="cuda"), torch.tensor(w, dtype=dt, device="cuda"), iters, tau,
                sigma=None if sigma is None else torch.tensor(sigma, dtype=dt, device="cuda"))
    g.sync()
    got = z.double().cpu().numpy()
    scale = np.abs(want).max()
    assert np.abs(got - want).max() <= (1e-10 if prec else 2e-4) * scale
    # the support (entries kept by the threshold) agrees wherever the oracle is clear of it
    clear = np.abs(want) > 1e-3 * scale
    assert np.all(got[clear] != 0)


def test_fista_zero_iterations_and_warm_start(pw):
    """iters = 0 leaves z; k iterations then m more from the result equal k + m only when the
    momentum restarts, so a warm start is compared with the oracle's warm start."""
    import torch
    op, g, T = _setup(pw, "small-2d", {"n": 32, "levels": 3}, 0)
    z0, w = _problem(op, T, P.BASE_SEED + 95)
    tau = 0.9 / oracle.power_norm(T, 50)
    zi = P.normal(P.BASE_SEED + 96, op.N)
    z = torch.tensor(zi, dtype=torch.float32, device="cuda")
    zd, wd = torch.tensor(z0, dtype=torch.float32, device="cuda"), torch.tensor(w, dtype=torch.float32, device="cuda")
    pw.pc_fista(g.h, zd, wd, None, z, 0, tau)
    g.sync()
    assert np.array_equal(z.cpu().numpy(), zi.astype(np.float32))
    pw.pc_fista(g.h, zd, wd, None, z, 7, tau)
    pw.pc_fista(g.h, zd, wd, None, z, 5, tau)
    g.sync()
    want = oracle.fista(T, z0, w, 5, tau, z_init=oracle.fista(T, z0, w, 7, tau, z_init=zi))
    assert np.abs(z.double().cpu().numpy() - want).max() <= 1e-4 * np.abs(want).max()


def test_solver_errors(pw):
    import torch
    op = P.workload("small-1d")
    g = make_gpu_op(pw, op)
    x = torch.zeros(op.N, dtype=torch.float32, device="cuda")
    for call in (lambda: pw.pc_fista(g.h, x, x, None, x, 3, 0.1), lambda: pw.pc_jacobi(g.h, x),
                 lambda: pw.pc_power_norm(g.h, None, 3), lambda: pw.pc_apply_adjoint(g.h, x, x)):
        with pytest.raises(pw.PCError) as e:
            call()
        assert e.value.status == pw.PC_ERR_NOT_ASSEMBLED
    g.assemble()
    for bad in (dict(iters=-1, tau=0.1), dict(iters=3, tau=0.0), dict(iters=3, tau=-1.0)):
        with pytest.raises(pw.PCError) as e:
            pw.pc_fista(g.h, x, x, None, x, bad["iters"], bad["tau"])
        assert e.value.status == pw.PC_ERR_INVALID_ARG
    with pytest.raises(pw.PCError):
        pw.pc_fista(g.h, None, x, None, x, 3, 0.1)
    with pytest.raises(pw.PCError):
        pw.pc_power_norm(g.h, None, 0)
    g.close()


def test_full_size_adjoint_and_first_iteration(pw):
    """The 256^2, db4, L=4, m=16 workload: sampled entries of Theta^T x and of the first FISTA
    iterate from zero, soft(tau Theta^T z0, tau w), against oracle columns of Theta."""
    import torch
    op = P.workload("c2")
    g = make_gpu_op(pw, op)
    g.assemble()
    x = P.normal(P.BASE_SEED + 77, op.N)
    w = 0.02 * (0.5 + P.uniform(P.BASE_SEED + 78, op.N))
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    y = g.apply_adjoint(xd)
    tau = 0.5
    z1 = g.fista(xd, torch.tensor(w, dtype=torch.float32, device="cuda"), 1, tau)
    g.sync()
    rng = np.random.default_rng(12)
    n, L = op.n, op.levels
    starts = [(0, (n >> L) ** 2)] + [((n >> j) ** 2 * (1 + t), (n >> j) ** 2) for j in range(L, 0, -1) for t in range(3)]
    cols = np.array([0, op.N - 1] + [off + int(rng.integers(0, size)) for off, size in starts], dtype=np.int64)
    Tc = oracle.theta_columns(op, cols)
    for c, lam in enumerate(cols):
        col = Tc[c] * oracle.pattern_column(op, lam)
        ref = float(col @ x)
        assert abs(float(y[lam]) - ref) <= 1e-5 * np.sqrt(np.sum(col * col) * op.N) + 1e-6, lam
        a = tau * ref
        want = np.sign(a) * max(abs(a) - tau * w[lam], 0.0)
        assert abs(float(z1[lam]) - want) <= 1e-5 * np.sqrt(np.sum(col * col) * op.N) * tau + 1e-6, lam
    g.close()


@pytest.mark.parametrize("order", [0, 1])
def test_solver_follows_reassembly(pw, order):
    """The solver's transposed copy of Theta is rebuilt after every assembly: parameters
    alternate between two operators through pc_set_params, assembled by pc_assemble, by the
    two stages and by the batched path, each followed by FISTA against the oracle."""
    import dataclasses
    import torch
    op1 = P.workload("small-2d", n=32, levels=3, order=order)
    op2 = dataclasses.replace(op1, u=op1.u[::-1].copy() * 0.8, v=np.roll(op1.v, 5, axis=1))
    g = make_gpu_op(pw, op1)
    z0 = torch.tensor(P.normal(P.BASE_SEED + 97, op1.N), dtype=torch.float32, device="cuda")
    w = torch.full((op1.N,), 0.01, dtype=torch.float32, device="cuda")
    want = {}
    for k, o in (("op1", op1), ("op2", op2)):
        want[k] = oracle.fista(dense_theta_pattern(o), z0.double().cpu().numpy(), w.double().cpu().numpy(), 10, 0.5)
    for how in ("assemble", "stages", "batch"):
        for k, o in (("op1", op1), ("op2", op2)):
            pw.pc_set_params(g.h, torch.tensor(o.u, dtype=torch.float32, device="cuda"),
                             torch.tensor(o.v, dtype=torch.float32, device="cuda"))
            if how == "assemble":
                g.assemble()
            elif how == "stages":
                pw.pc_assemble_stage(g.h, 0)
                pw.pc_assemble_stage(g.h, 1)
            else:
                pw.pc_batch_assemble([g.h])
            z = g.fista(z0, w, 10, 0.5)
            g.sync()
            got = z.double().cpu().numpy()
            assert np.abs(got - want[k]).max() <= 2e-4 * np.abs(want[k]).max(), (how, k)
    g.close()
