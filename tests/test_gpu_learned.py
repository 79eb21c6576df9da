"""GPU parity of the learned preconditioner correction against the oracle
(oracle/learned.py), through the C ABI: gates, forward pass, loss gradient,
the corrected preconditioner T(r), training pairs, the PCG solve of
Op e = r, and a short training run.  FP32 kernels: tolerances relative to the
largest entry, 2e-5 for fields and 2e-4 for parameter gradients (sums over
N^3 voxels and 27 taps in FP32)."""
import numpy as np
import pytest

import workloads as wl
from oracle import fourier, learned, penalty, permittivity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pcx():
    from paper_2511_17107_gb300 import build, pcx as binding
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return binding


def _params(seed, scale=0.25):
    rng = np.random.default_rng(seed)
    p = {name: (rng.standard_normal(shape) * scale).astype(np.float32).astype(np.float64)
         for name, shape in learned.param_shapes()}
    return p


def _case(pcx, n, seed=3):
    s = wl.random_inclusions(seed)
    f = learned.features(permittivity.cell_blocks(s, n))
    ctx = pcx.setup_structure(s, n)
    return s, f, ctx


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a).astype(dtype)).cuda()


def _close(got, want, tol):
    err = np.abs(got - want).max() / np.abs(want).max()
    assert err <= tol, err
    return err


@pytest.mark.parametrize("n", [8, 32])
def test_gates_and_forward_match_oracle(pcx, n):
    s, f, ctx = _case(pcx, n)
    p = _params(1)
    P = _dev(learned.pack(p), np.float32)
    G = torch.empty(2 * learned.HIDDEN * n ** 3, dtype=torch.float32, device="cuda")
    pcx.pcx_cnn_gates(ctx, P, G)
    g1, g2 = learned.gates(p, f)
    _close(G.cpu().numpy()[: learned.HIDDEN * n ** 3].reshape(g1.shape), g1, 1e-5)
    _close(G.cpu().numpy()[learned.HIDDEN * n ** 3:].reshape(g2.shape), g2, 1e-5)
    U = wl.random_block(2, n, seed=7)
    Y = torch.empty((2, 3, n, n, n), dtype=torch.complex64, device="cuda")
    pcx.pcx_cnn_forward(ctx, P, G, _dev(U, np.complex64), Y)
    _close(Y.cpu().numpy(), learned.forward(p, f, U.astype(np.complex64).astype(np.complex128)), 2e-5)


def test_gradient_matches_oracle(pcx):
    n, nv = 8, 2
    s, f, ctx = _case(pcx, n, seed=4)
    p = _params(2)
    U = wl.random_block(nv, n, seed=8).astype(np.complex64).astype(np.complex128)
    T = wl.random_block(nv, n, seed=9).astype(np.complex64).astype(np.complex128)
    w = np.array([0.8, 1.7])
    want_loss, want = learned.loss_and_grad(p, f, U, T, w)
    P = _dev(learned.pack(p), np.float32)
    grad = torch.zeros(pcx.PCX_CNN_NPARAMS, dtype=torch.float32, device="cuda")
    loss = pcx.pcx_cnn_grad(ctx, P, _dev(U, np.complex64), _dev(T, np.complex64), w, grad)
    assert abs(loss - want_loss) <= 1e-5 * want_loss
    got = learned.unpack(grad.cpu().numpy().astype(np.float64))
    for name, _ in learned.param_shapes():
        _close(got[name], want[name], 2e-4)
    # accumulate = 1 adds a second gradient on top
    pcx.pcx_cnn_grad(ctx, P, _dev(U, np.complex64), _dev(T, np.complex64), w, grad, accumulate=True)
    _close(grad.cpu().numpy().astype(np.float64), 2 * learned.pack(want), 2e-4)


@pytest.mark.parametrize("n", [16, 64])
def test_learned_preconditioner_matches_oracle(pcx, n):
    s, f, ctx = _case(pcx, n, seed=7)
    k = np.array([0.6, -1.1, 2.0])
    g = penalty.gamma_practical(k)
    kap = fourier.kappa(n, s.lattice, k)
    p = _params(3, 0.2)
    P = _dev(learned.pack(p), np.float32)
    G = torch.empty(2 * learned.HIDDEN * n ** 3, dtype=torch.float32, device="cuda")
    pcx.pcx_cnn_gates(ctx, P, G)
    nv = 2 if n == 16 else 1
    R = wl.random_block(nv, n, seed=12).astype(np.complex64)
    W = torch.empty((nv, 3, n, n, n), dtype=torch.complex64, device="cuda")
    pcx.pcx_cnn_precond(ctx, k, P, G, _dev(R, np.complex64), W)
    blocks = permittivity.cell_blocks(s, n)
    want = np.stack([learned.precondition(p, f, R[v].astype(np.complex128), kap, g, blocks) for v in range(nv)])
    _close(W.cpu().numpy(), want, 2e-5)


SANDWICH_CASES = [(16, np.complex128, 1e-12), (16, np.complex64, 2e-5), (64, np.complex64, 2e-5),
                  (32, np.complex128, 1e-12)]


@pytest.mark.parametrize("n,dtype,tol", SANDWICH_CASES)
def test_sandwich_preconditioner_matches_oracle(pcx, n, dtype, tol):
    s = wl.random_inclusions(8)
    blocks = permittivity.cell_blocks(s, n)
    k = np.array([-0.8, 1.9, 0.3])
    g = penalty.gamma_practical(k)
    kap = fourier.kappa(n, s.lattice, k)
    ctx = pcx.setup_structure(s, n)
    R = wl.random_block(2, n, seed=40).astype(dtype)
    W = torch.empty((2, 3, n, n, n), dtype=torch.complex64 if dtype == np.complex64 else torch.complex128,
                    device="cuda")
    pcx.pcx_sandwich_precond(ctx, k, _dev(R, dtype), W)
    want = learned.sandwich_precondition(R.astype(np.complex128), kap, blocks, g)
    _close(W.cpu().numpy(), want, tol)
    # in place, W = T0 W
    X = _dev(R, dtype)
    pcx.pcx_sandwich_precond(ctx, k, X, X)
    _close(X.cpu().numpy(), want, tol)


def test_training_pairs_match_oracle(pcx):
    n = 16
    s, f, ctx = _case(pcx, n, seed=6)
    k = np.array([1.3, 0.2, -0.7])
    g = penalty.gamma_practical(k)
    kap = fourier.kappa(n, s.lattice, k)
    R = wl.random_block(2, n, seed=14).astype(np.complex64)
    E = wl.random_block(2, n, seed=15).astype(np.complex64)
    U = torch.empty((2, 3, n, n, n), dtype=torch.complex64, device="cuda")
    T = torch.empty_like(U)
    en2 = pcx.pcx_cnn_pairs(ctx, k, _dev(R, np.complex64), _dev(E, np.complex64), U, T)
    wu, wt, wen2 = learned.training_pair(R.astype(np.complex128), E.astype(np.complex128), kap, g,
                                         permittivity.cell_blocks(s, n))
    _close(U.cpu().numpy(), wu, 2e-5)
    _close(T.cpu().numpy(), wt, 2e-5)
    np.testing.assert_allclose(en2, wen2, rtol=1e-5)


def test_cg_solve_inverts_the_operator(pcx):
    """E = Op^{-1} R: the true residual ||Op E - R|| / ||R||, with Op the
    oracle's symbol form of the compensated operator, is at the requested
    tolerance (FP32 vectors)."""
    n = 16
    s = wl.random_inclusions(2)
    blocks = permittivity.cell_blocks(s, n)
    k = np.array([0.9, 0.4, -1.2])
    g = penalty.gamma_practical(k)
    kap = fourier.kappa(n, s.lattice, k)
    ctx = pcx.setup_structure(s, n)
    R = wl.random_block(3, n, seed=21).astype(np.complex64)
    E = torch.empty((3, 3, n, n, n), dtype=torch.complex64, device="cuda")
    its, rel = pcx.pcx_cg_solve(ctx, k, _dev(R, np.complex64), E, tol=1e-4, maxit=300)
    assert np.all(rel <= 1e-4) and its < 300
    e = E.cpu().numpy().astype(np.complex128)
    ope = fourier.apply_symbols(e, kap, lambda x: permittivity.apply_m(blocks, x), g)
    true = np.linalg.norm((ope - R).reshape(3, -1), axis=1) / np.linalg.norm(R.reshape(3, -1), axis=1)
    assert np.all(true <= 5e-4), true


def test_training_lowers_the_loss(pcx):
    """Targets e = Op^{-1} r from the PCG solve, 60 Adam steps on one
    structure: the relative error of T against e must fall well below that
    of K_P^{-1} alone."""
    n, nv = 32, 4
    s = wl.random_inclusions(11)
    ctx = pcx.setup_structure(s, n)
    k = np.array([1.0, 0.5, 0.25]) * np.pi
    R = _dev(wl.random_block(nv, n, seed=30), np.complex64)
    E = torch.empty_like(R)
    pcx.pcx_cg_solve(ctx, k, R, E, tol=1e-4, maxit=300)
    U = torch.empty_like(R)
    T = torch.empty_like(R)
    en2 = pcx.pcx_cnn_pairs(ctx, k, R, E, U, T)
    w = 1.0 / (nv * en2)
    P = torch.empty(pcx.PCX_CNN_NPARAMS, dtype=torch.float32, device="cuda")
    pcx.pcx_cnn_init(5, P)
    m = torch.zeros_like(P)
    v = torch.zeros_like(P)
    grad = torch.zeros_like(P)
    losses = []
    for step in range(1, 61):
        losses.append(pcx.pcx_cnn_grad(ctx, P, U, T, w, grad))
        pcx.pcx_cnn_adam(P, grad, m, v, step, 3e-3)
    assert losses[-1] < 0.6 * losses[0], (losses[0], losses[-1])


def test_learned_gain_on_held_out_structures(pcx, capsys):
    """What the trained correction gains over its base: 6 random training
    structures at 32^3 (residual dump of the mixed solve, PCG targets, 300
    Adam steps; Hermitian form, BF16 weights), 3 held-out structures solved
    to 1e-8 (12 bands, mixed precision) with K_P^{-1}, with the
    curl-sandwich T0 and with the learned T = T0 + correction (fallback to T0
    after 3 iterations without a 10% drop).  Every variant must reach the same
    eigenvalues and T0 must need fewer iterations than K_P^{-1}.  Against T0,
    its base, the measured outcome is that the learned T does not gain: the
    training loss falls, but the held-out iteration counts are T0's or more
    (one structure needed about twice T0's count).  The test asserts that
    outcome -- no gain of 10% or more over T0 -- so that a correction that
    starts to gain shows up here; the counts are printed."""
    from paper_2511_17107_gb300 import learned as lrn
    n = 32
    rng = np.random.default_rng(0)
    samples, seed = [], 100
    while len(samples) < 6:
        s = wl.random_inclusions(seed)
        seed += 1
        try:
            ctx = pcx.setup_structure(s, n)
        except pcx.PcxError:
            continue
        smp = lrn.collect(ctx, rng.uniform(-np.pi, np.pi, 3), n_pairs=16, seed=seed)
        if smp is not None:
            samples.append(smp)
    P, losses = lrn.train(samples, steps=300, lr=3e-3)
    P0 = torch.empty_like(P)
    pcx.pcx_cnn_init(1, P0)
    assert lrn.relative_error(samples, P) < lrn.relative_error(samples, P0)
    its = {"K_P": [], "T0": [], "learned": []}
    seed = 5000
    while len(its["K_P"]) < 3:
        s = wl.random_inclusions(seed)
        seed += 1
        try:
            ctx = pcx.setup_structure(s, n)
        except pcx.PcxError:
            continue
        k = rng.uniform(-np.pi, np.pi, 3)
        pcx.pcx_set_cnn_form(ctx, lrn.FORM)
        ev = {}
        for name, cp, kind in (("K_P", None, 0), ("T0", None, 1), ("learned", P, 1)):
            e, r, it, st = pcx.pcx_solve(ctx, [k], 12, 1e-8, block=16, precision=pcx.PCX_FP32, cnn_params=cp,
                                         precond_kind=kind)
            assert st == pcx.PCX_OK
            ev[name] = e[0]
            its[name].append(int(it[0]))
        for name in ("T0", "learned"):
            np.testing.assert_allclose(ev[name], ev["K_P"], rtol=1e-6)
    with capsys.disabled():
        print("\nlearned-correction gain, iterations per held-out structure:", its)
    assert np.mean(its["T0"]) < np.mean(its["K_P"])
    assert np.mean(its["learned"]) > 0.9 * np.mean(its["T0"])


FORMS = [("hermitian", 1), ("bf16", 2), ("hermitian-bf16", 3)]


def _oracle_params(p, flags):
    return learned.rounded(p) if flags & 2 else p


@pytest.mark.parametrize("name,flags", FORMS, ids=[f[0] for f in FORMS])
def test_forms_forward_and_gradient_match_oracle(pcx, name, flags):
    """The Hermitian form g_s = (g + g^T) / 2 and the BF16 weights, against
    the oracle's symmetric form on bfloat16-rounded weights: gates and
    forward 2e-5, loss 1e-5, gradient 2e-4 (the gradient of the rounded
    network, applied to the FP32 parameters)."""
    n, nv = 8, 2
    s, f, ctx = _case(pcx, n, seed=4)
    pcx.pcx_set_cnn_form(ctx, flags)
    p = _params(2)
    po = _oracle_params(p, flags)
    herm = bool(flags & 1)
    P = _dev(learned.pack(p), np.float32)
    G = torch.empty(2 * learned.HIDDEN * n ** 3, dtype=torch.float32, device="cuda")
    pcx.pcx_cnn_gates(ctx, P, G)
    g1, _ = learned.gates(po, f)
    _close(G.cpu().numpy()[: learned.HIDDEN * n ** 3].reshape(g1.shape), g1, 1e-5)
    U = wl.random_block(nv, n, seed=8).astype(np.complex64).astype(np.complex128)
    Y = torch.empty((nv, 3, n, n, n), dtype=torch.complex64, device="cuda")
    pcx.pcx_cnn_forward(ctx, P, G, _dev(U, np.complex64), Y)
    _close(Y.cpu().numpy(), learned.forward(po, f, U, symmetric=herm), 2e-5)
    T = wl.random_block(nv, n, seed=9).astype(np.complex64).astype(np.complex128)
    w = np.array([0.8, 1.7])
    want_loss, want = learned.loss_and_grad(po, f, U, T, w, symmetric=herm)
    grad = torch.zeros(pcx.PCX_CNN_NPARAMS, dtype=torch.float32, device="cuda")
    loss = pcx.pcx_cnn_grad(ctx, P, _dev(U, np.complex64), _dev(T, np.complex64), w, grad)
    assert abs(loss - want_loss) <= 1e-5 * want_loss
    got = learned.unpack(grad.cpu().numpy().astype(np.float64))
    for pname, _ in learned.param_shapes():
        _close(got[pname], want[pname], 2e-4)


def test_hermitian_form_preconditioner_matches_oracle_and_is_hermitian(pcx):
    n = 16
    s, f, ctx = _case(pcx, n, seed=7)
    pcx.pcx_set_cnn_form(ctx, 3)
    k = np.array([0.6, -1.1, 2.0])
    g = penalty.gamma_practical(k)
    kap = fourier.kappa(n, s.lattice, k)
    p = _params(3, 0.2)
    P = _dev(learned.pack(p), np.float32)
    G = torch.empty(2 * learned.HIDDEN * n ** 3, dtype=torch.float32, device="cuda")
    pcx.pcx_cnn_gates(ctx, P, G)
    R = wl.random_block(2, n, seed=12).astype(np.complex64)
    W = torch.empty((2, 3, n, n, n), dtype=torch.complex64, device="cuda")
    pcx.pcx_cnn_precond(ctx, k, P, G, _dev(R, np.complex64), W)
    blocks = permittivity.cell_blocks(s, n)
    po = learned.rounded(p)
    want = np.stack([learned.precondition(po, f, R[v].astype(np.complex128), kap, g, blocks, symmetric=True)
                     for v in range(2)])
    got = W.cpu().numpy().astype(np.complex128)
    _close(got, want, 2e-5)
    # <x, T y> = conj <y, T x> on the GPU's own outputs
    x, y = R[0].astype(np.complex128), R[1].astype(np.complex128)
    lhs, rhs = np.vdot(x, got[1]), np.conj(np.vdot(y, got[0]))
    assert abs(lhs - rhs) <= 1e-4 * abs(lhs)
