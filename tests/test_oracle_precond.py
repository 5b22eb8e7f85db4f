"""Pins of the learned-preconditioner oracle (oracle/precond.py), CPU only.

Each pin checks the oracle against something other than itself: the Wilson
operator of the C oracle (a special choice of weights), gauge covariance,
the adjoint identity, central finite differences of the loss, the closed form
of Adam under a constant gradient, and flexible CG against plain CG (identity
preconditioner) and against the exact inverse (one iteration).
"""

import numpy as np
import pytest

from oracle import _clib
from oracle import dwf as orc
from oracle import precond as pc
from paper_2602_14454_gb300 import inputs

DIMS = (4, 2, 2, 4)
BC = (1, 1, 1, -1)


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


def cfield(C, dims, seed):
    g = np.random.default_rng(seed)
    shape = (C,) + tuple(reversed(dims)) + (4, 3)
    return g.normal(size=shape) + 1j * g.normal(size=shape)


def cweights(L, C, seed, scale=0.3):
    g = np.random.default_rng(seed)
    shape = (L, pc.NHOP, 2, C, C)
    return scale * (g.normal(size=shape) + 1j * g.normal(size=shape))


def gauge_transform(U, g):
    Ug = np.empty_like(U)
    for mu in range(4):
        gfwd = np.roll(g, -1, axis=(3, 2, 1, 0)[mu])
        Ug[mu] = g @ U[mu] @ np.swapaxes(gfwd.conj(), -1, -2)
    return Ug


@pytest.mark.parametrize("bc", [(1, 1, 1, -1), (-1, 1, -1, 1)])
def test_layer_with_wilson_weights_is_the_wilson_operator(bc):
    """W_0 = (4 - M0) A, W_{+-mu} = -1/2 A for a channel matrix A: the layer is
    A (x) D_W(-M0), D_W from the C oracle (eq. Wilson_matrix)."""
    M0 = 1.3
    C = 3
    U = inputs.random_links(DIMS, 0.6, 31)
    A = np.random.default_rng(32).normal(size=(C, C)) + 1j * np.random.default_rng(33).normal(size=(C, C))
    W = np.zeros((pc.NHOP, 2, C, C), dtype=np.complex128)
    W[0] = (4 - M0) * A
    W[1:] = -0.5 * A
    psi = cfield(C, DIMS, 34)
    got = pc.layer(U, W, psi, bc)
    dw = _clib.wilson(U, DIMS, bc, M0, psi, False)
    want = np.einsum("ij,j...->i...", A, dw)
    assert rel(got, want) < 1e-13


def test_layer_chirality_weights():
    """Hop weights on P_+ outputs only: out = P_+ D_W psi + (4 - M0) P_- psi."""
    M0 = 1.8
    U = inputs.random_links(DIMS, 0.6, 35)
    W = np.zeros((pc.NHOP, 2, 1, 1), dtype=np.complex128)
    W[0, :] = 4 - M0
    W[1:, 0] = -0.5
    psi = cfield(1, DIMS, 36)
    got = pc.layer(U, W, psi, BC)
    dw = _clib.wilson(U, DIMS, BC, M0, psi, False)
    want = orc.spin(orc.P_PLUS, dw) + (4 - M0) * orc.spin(orc.P_MINUS, psi)
    assert rel(got, want) < 1e-13


def test_layer_gauge_covariance():
    C = 2
    U = inputs.random_links(DIMS, 0.6, 37)
    g = inputs.random_gauge_transform(DIMS, 38)
    Ug = gauge_transform(U, g)
    W = cweights(1, C, 39)[0]
    psi = cfield(C, DIMS, 40)
    gpsi = np.einsum("...ab,c...ib->c...ia", g, psi)
    lhs = pc.layer(Ug, W, gpsi, BC)
    rhs = np.einsum("...ab,c...ib->c...ia", g, pc.layer(U, W, psi, BC))
    assert rel(lhs, rhs) < 1e-13


def test_net_gauge_covariance_and_linearity():
    Ls = 3
    U = inputs.random_links(DIMS, 0.6, 41)
    g = inputs.random_gauge_transform(DIMS, 42)
    W = cweights(3, Ls, 43)
    net, netg = pc.Net(U, DIMS, BC, W), pc.Net(gauge_transform(U, g), DIMS, BC, W)
    r1 = cfield(Ls, DIMS, 44).reshape(Ls, -1, 4, 3)[:, net.even]
    r2 = cfield(Ls, DIMS, 45).reshape(Ls, -1, 4, 3)[:, net.even]
    ge = g.reshape(-1, 3, 3)[net.even]
    lhs = netg.forward(np.einsum("vab,svib->svia", ge, r1))
    rhs = np.einsum("vab,svib->svia", ge, net.forward(r1))
    assert rel(lhs, rhs) < 1e-13
    a, b = 0.7 - 0.2j, -1.1 + 0.4j
    assert rel(net.forward(a * r1 + b * r2), a * net.forward(r1) + b * net.forward(r2)) < 1e-13


def test_identity_weights_give_the_identity():
    Ls = 4
    U = inputs.random_links(DIMS, 0.6, 46)
    W = np.zeros((3, pc.NHOP, 2, Ls, Ls), dtype=np.complex128)
    W[:, 0, :] = np.eye(Ls)
    net = pc.Net(U, DIMS, BC, W)
    r = cfield(Ls, DIMS, 47).reshape(Ls, -1, 4, 3)[:, net.even]
    assert np.array_equal(net.forward(r), r)


@pytest.mark.parametrize("bc", [(1, 1, 1, -1), (1, -1, 1, -1)])
def test_layer_adjoint_identity(bc):
    """<y, L psi> = <L^dag y, psi> with L^dag y the input gradient of Re<y, L psi>."""
    C = 3
    U = inputs.random_links(DIMS, 0.6, 48)
    W = cweights(1, C, 49)[0]
    psi, y = cfield(C, DIMS, 50), cfield(C, DIMS, 51)
    _, ldag_y = pc.layer_backward(U, W, psi, y, bc)
    lhs = np.vdot(y.ravel(), pc.layer(U, W, psi, bc).ravel())
    rhs = np.vdot(ldag_y.ravel(), psi.ravel())
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_net_adjoint_and_preconditioner_hermiticity():
    """<y, N r> = <N^dag y, r>; M = N N^dag is Hermitian and positive."""
    Ls = 3
    U = inputs.random_links(DIMS, 0.6, 57)
    net = pc.Net(U, DIMS, BC, cweights(3, Ls, 58))
    r = cfield(Ls, DIMS, 59).reshape(Ls, -1, 4, 3)[:, net.even]
    y = cfield(Ls, DIMS, 60).reshape(Ls, -1, 4, 3)[:, net.even]
    lhs = np.vdot(y.ravel(), net.forward(r).ravel())
    rhs = np.vdot(net.adjoint(y).ravel(), r.ravel())
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    a = np.vdot(y.ravel(), net.precondition(r).ravel())
    b = np.vdot(net.precondition(y).ravel(), r.ravel())
    assert abs(a - b) < 1e-12 * abs(a)
    q = np.vdot(r.ravel(), net.precondition(r).ravel())
    assert abs(q.imag) < 1e-12 * abs(q) and q.real > 0


def test_loss_gradient_against_finite_differences():
    Ls = 2
    dims = (2, 2, 2, 4)
    U = inputs.random_links(dims, 0.6, 52)
    W = cweights(3, Ls, 53, scale=0.4)
    net = pc.Net(U, dims, BC, W)
    g = np.random.default_rng(54)
    pairs = []
    for k in range(2):
        b = g.normal(size=(Ls, 16, 4, 3)) + 1j * g.normal(size=(Ls, 16, 4, 3))
        x = g.normal(size=(Ls, 16, 4, 3)) + 1j * g.normal(size=(Ls, 16, 4, 3))
        pairs.append((b, x))
    L0, gW = net.loss_and_grad(pairs)
    h = 1e-6
    picks = [tuple(g.integers(0, n) for n in W.shape) for _ in range(12)]
    for idx in picks:
        for part in (1.0, 1j):
            Wp, Wm = W.copy(), W.copy()
            Wp[idx] += h * part
            Wm[idx] -= h * part
            Lp, _ = pc.Net(U, dims, BC, Wp).loss_and_grad(pairs)
            Lm, _ = pc.Net(U, dims, BC, Wm).loss_and_grad(pairs)
            fd = (Lp - Lm) / (2 * h)
            an = gW[idx].real if part == 1.0 else gW[idx].imag
            assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3 * np.abs(gW).max()), (idx, part, fd, an)


def test_adam_constant_gradient_closed_form():
    """With a constant gradient g the bias-corrected moments are exactly g and g^2,
    so every step moves each real parameter by -lr g / (|g| + eps)."""
    g = np.array([0.3 - 2.0j, -1e-3 + 4.0j])
    th = np.array([1.0 + 1.0j, -2.0 + 0.5j])
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    lr, eps = 0.01, 1e-8
    th0 = th.copy()
    for t in range(1, 6):
        th, m, v = pc.adam_step(th, g, m, v, t, lr, eps=eps)
    want = th0 - 5 * lr * (g.real / (np.abs(g.real) + eps) + 1j * g.imag / (np.abs(g.imag) + eps))
    assert np.abs(th - want).max() < 1e-12


def test_adam_minimises_a_quadratic():
    th = np.array([3.0 - 1.0j])
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    target = np.array([0.5 + 0.25j])
    for t in range(1, 3001):
        th, m, v = pc.adam_step(th, 2 * (th - target), m, v, t, 0.01)
    assert abs(th[0] - target[0]) < 1e-3


def _small_system():
    dims, Ls = (2, 2, 2, 4), 4
    U = inputs.random_links(dims, 0.5, 55)
    ref = orc.DWF(U, dims, Ls, 1.8, 0.1, 1.5, 0.5, form="neff", alpha=0.5)
    bt = ref.to_eo(inputs.gaussian_5d(dims, Ls, 56), 0)
    A = lambda v: ref.d_pc(ref.d_pc(v), dag=True)  # noqa: E731
    return ref, bt, A


def test_fcg_with_identity_is_cg():
    """Identity preconditioner: flexible CG on D^dag D x = D^dag b~ takes the same
    iterates as CGNR on D x = b~ (the oracle's cgnr)."""
    ref, bt, A = _small_system()
    b = ref.d_pc(bt, dag=True)
    for K in (5, 20):
        x1, _ = pc.fcg(A, lambda r: r, b, tol=0.0, maxiter=K)
        x2, _ = orc.cgnr(ref.d_pc, lambda v: ref.d_pc(v, dag=True), bt, tol=0.0, maxiter=K)
        assert rel(x1, x2) < 1e-10


def test_fcg_with_exact_inverse_takes_one_iteration():
    ref, bt, A = _small_system()
    n = bt.size
    cols = []
    for k in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[k] = 1
        cols.append(A(e.reshape(bt.shape)).ravel())
    Ainv = np.linalg.inv(np.array(cols).T)
    b = ref.d_pc(bt, dag=True)
    x, info = pc.fcg(A, lambda r: (Ainv @ r.ravel()).reshape(r.shape), b, tol=1e-12)
    assert info["iterations"] == 1
    assert info["true_residual"] < 1e-12


def test_training_lowers_the_loss():
    """A few Adam steps on pairs (b = D x, x) lower the loss from the identity start."""
    ref, bt, A = _small_system()
    Ls = ref.Ls
    W = np.zeros((3, pc.NHOP, 2, Ls, Ls), dtype=np.complex128)
    W[:, 0, :] = np.eye(Ls)
    net = pc.Net(ref.U, (2, 2, 2, 4), BC, W)
    pairs = []
    for k in range(3):
        x = ref.to_eo(inputs.gaussian_5d((2, 2, 2, 4), Ls, 60 + k), 0)
        pairs.append((ref.d_pc(x), x))
    L0, _ = net.loss_and_grad(pairs)
    m = np.zeros_like(W)
    v = np.zeros_like(W)
    for t in range(1, 31):
        _, g = net.loss_and_grad(pairs)
        net.W, m, v = pc.adam_step(net.W, g, m, v, t, 0.01)
    L1, _ = net.loss_and_grad(pairs)
    assert L1 < 0.8 * L0
