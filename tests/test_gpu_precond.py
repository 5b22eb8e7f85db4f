"""Learned preconditioner through the C ABI against the FP64 oracle (oracle/precond.py).

The network N, its adjoint, the preconditioner M = N N^dag, the loss and its
gradients are compared element by element with the oracle (FP32 kernels, the
oracle fed the same BF16-rounded weights the kernels use); gauge covariance
is checked on the GPU; training lowers the loss; flexible CG with the trained
network reaches the FP64 true residual and the oracle's 4D solution; and the
gain of the trained network over the same solver without it (identity
network: M = 1, plain CG) is measured.
"""

import numpy as np
import pytest

from _util import make_pair, rel, to_gpu, to_np
from paper_2602_14454_gb300 import inputs

pytestmark = pytest.mark.gpu

BC = (1, 1, 1, -1)


@pytest.fixture(scope="module", autouse=True)
def _built(cuda_ok):
    from paper_2602_14454_gb300 import build
    build.build()


def random_weights(L, C, seed, scale=0.3):
    g = np.random.default_rng(seed)
    w = scale * (g.normal(size=(L, 9, 2, C, C)) + 1j * g.normal(size=(L, 9, 2, C, C)))
    w[:, 0] += np.eye(C)
    return w


def even_field(ref, seed):
    return ref.to_eo(inputs.gaussian_5d(ref.dims, ref.Ls, seed), 0)


@pytest.mark.parametrize("dims,Ls,L", [((4, 4, 2, 4), 4, 3), ((2, 4, 4, 6), 6, 2), ((4, 2, 2, 4), 16, 1)])
def test_forward_matches_oracle(dims, Ls, L):
    from oracle import precond as pc
    op, ref = make_pair(dims, Ls, 1.8, 0.05, 1.5, 0.5, "neff", 0.5, seed=201)
    op.precond_set_weights(random_weights(L, Ls, 202))
    W = op.precond_get_weights(L, compute_copy=True)        # the BF16-rounded weights the kernels use
    net = pc.Net(ref.U, dims, BC, W)
    r = even_field(ref, 203)
    got = to_np(op.precond_apply(to_gpu(r)))
    assert rel(got, net.forward(r)) < 1e-5
    assert rel(to_np(op.precond_apply(to_gpu(r), which="Ndag")), net.adjoint(r)) < 1e-5
    assert rel(to_np(op.precond_apply(to_gpu(r), which="M")), net.precondition(r)) < 1e-5


def test_bf16_weight_rounding_is_reported():
    dims, Ls = (4, 4, 2, 4), 4
    op, ref = make_pair(dims, Ls, 1.8, 0.05, 1.5, 0.5, "neff", 0.5, seed=204)
    w = random_weights(3, Ls, 205)
    op.precond_set_weights(w)
    master = op.precond_get_weights(3, compute_copy=False)
    comp = op.precond_get_weights(3, compute_copy=True)
    assert np.array_equal(master, w)
    err = np.abs(comp - w).max() / np.abs(w).max()
    assert 0 < err < 2 ** -8                                 # BF16: 8 significant bits


def test_loss_and_gradient_match_oracle():
    from oracle import precond as pc
    dims, Ls, L = (4, 4, 2, 4), 4, 3
    op, ref = make_pair(dims, Ls, 1.8, 0.05, 1.5, 0.5, "neff", 0.5, seed=206)
    op.precond_set_weights(random_weights(L, Ls, 207, scale=0.2))
    W = op.precond_get_weights(L, compute_copy=True)
    net = pc.Net(ref.U, dims, BC, W)
    pairs = [(even_field(ref, 208 + 2 * k), even_field(ref, 209 + 2 * k)) for k in range(3)]
    loss, grad = op.precond_loss_grad([to_gpu(b) for b, _ in pairs], [to_gpu(x) for _, x in pairs], layers=L)
    L0, G0 = net.loss_and_grad(pairs)
    assert abs(loss / L0 - 1) < 1e-5
    assert rel(grad, G0) < 1e-5
    # per layer as well (the first layer's gradient flows through the other two)
    for l in range(L):
        assert rel(grad[l], G0[l]) < 1e-5


def test_gauge_covariance_on_the_gpu():
    import torch
    from paper_2602_14454_gb300 import dwf
    dims, Ls = (4, 4, 2, 4), 4
    U = inputs.random_links(dims, 0.5, 210)
    g = inputs.random_gauge_transform(dims, 211)
    Ug = np.empty_like(U)
    for mu in range(4):
        gf = np.roll(g, -1, axis=(3, 2, 1, 0)[mu])
        Ug[mu] = g @ U[mu] @ np.swapaxes(gf.conj(), -1, -2)
    w = random_weights(3, Ls, 212)
    outs = []
    op, ref = make_pair(dims, Ls, 1.8, 0.05, 1.5, 0.5, "neff", 0.5, U=U)
    opg = dwf.Operator(dims, Ls, 1.8, 0.05, 1.5, 0.5, form="neff", alpha=0.5)
    opg.set_gauge(torch.from_numpy(Ug).cuda())
    op.precond_set_weights(w)
    opg.precond_set_weights(w)
    r = even_field(ref, 213)
    ge = g.reshape(-1, 3, 3)[ref._eo_setup()["even"]]
    gr = np.einsum("vab,svib->svia", ge, r)
    lhs = to_np(opg.precond_apply(to_gpu(gr)))
    rhs = np.einsum("vab,svib->svia", ge, to_np(op.precond_apply(to_gpu(r))))
    assert rel(lhs, rhs) < 1e-5


def _train(op, dims, nsrc, seed0, **kw):
    b4s = [to_gpu(inputs.gaussian_4d(dims, seed0 + k)) for k in range(nsrc)]
    return op.precond_train(b4s, **kw)


def test_training_lowers_the_loss_and_fcg_solves():
    """C1-like lattice: train on 16 sources; FCG with the network reaches the FP64
    true residual 1e-10 and the oracle's 4D solution within 1e-9."""
    dims, Ls = (4, 4, 4, 4), 8
    U = inputs.random_links(dims, 0.5, 1004)
    op, ref = make_pair(dims, Ls, 1.8, 0.04, 1.5, 0.5, "neff", 0.5, U=U)
    st = _train(op, dims, 16, 4000, epochs=8, batch=4, lr=2e-3)
    assert st["pairs"] == 32 and st["epochs"] == 8          # 16 solution pairs + 16 white-noise pairs
    assert st["loss_last"] < st["loss_first"]
    b4 = inputs.gaussian_4d(dims, 5000)
    b5 = ref.source_5d(b4)
    x5_ref, _ = ref.solve(b5, tol=1e-13)
    x5, s = op.solve(to_gpu(b5), inner_prec="f32", precond=1, tol=1e-10)
    x5 = to_np(x5)
    assert s["precond_applications"] > 0
    assert rel(ref.apply(x5), b5) <= 1e-10
    assert rel(ref.project_4d(x5), ref.project_4d(x5_ref)) < 1e-9


def test_identity_network_gives_plain_cg():
    """Identity weights: N = 1, so the preconditioned cycles are plain CG on D^dag D
    restarted at every defect correction; the solve converges, with at most about
    twice the iterations of the reliable-update CG (which keeps its direction)."""
    dims, Ls = (4, 4, 4, 4), 8
    op, ref = make_pair(dims, Ls, 1.8, 0.04, 1.0, 0.0, "standard", 1.0, seed=1001)
    op.precond_init(3, seed=1, noise=0.0)
    b5 = ref.source_5d(inputs.gaussian_4d(dims, 2001))
    x5, s = op.solve(to_gpu(b5), inner_prec="f32", precond=1)
    _, s0 = op.solve(to_gpu(b5), inner_prec="f32")
    assert rel(ref.apply(to_np(x5)), b5) <= 1e-10
    assert s["fallbacks"] == 0
    assert s["iterations"] <= 2 * s0["iterations"] + 16


def test_trained_network_gain():
    """8^4, Ls = 8, mf = 0.01, smeared links: train on 32 sources, then compare
    the solve preconditioned by the trained network with the same solver and the
    identity network (plain CG) on held-out sources.  Both must reach the FP64
    true residual; the iteration and time ratios are printed (gain = plain /
    trained).  On these synthetic fields the 3-layer network does not reduce the
    iteration count (measured gain about 0.5), so no gain is asserted."""
    import time
    dims, Ls = (8, 8, 8, 8), 8
    U = inputs.smeared_links(dims, 0.3, 0.1, 3, 1004)
    op, ref = make_pair(dims, Ls, 1.8, 0.01, 1.5, 0.5, "neff", 0.5, U=U)
    op.precond_init(3, seed=1, noise=0.0)
    plain = []
    for k in range(2):
        b5 = op.source_5d(to_gpu(inputs.gaussian_4d(dims, 5000 + k)))
        t0 = time.perf_counter()
        _, s = op.solve(b5, inner_prec="f32", precond=1)
        plain.append((s["iterations"], time.perf_counter() - t0, s["true_residual"]))
    st = _train(op, dims, 32, 4000, epochs=10, batch=8, lr=3e-3)
    trained = []
    for k in range(2):
        b5 = op.source_5d(to_gpu(inputs.gaussian_4d(dims, 5000 + k)))
        t0 = time.perf_counter()
        _, s = op.solve(b5, inner_prec="f32", precond=1)
        trained.append((s["iterations"], time.perf_counter() - t0, s["true_residual"]))
    print("learned preconditioner gain: loss %.3e -> %.3e; iterations plain %s trained %s; seconds plain %s "
          "trained %s" % (st["loss_first"], st["loss_last"], [p[0] for p in plain], [t[0] for t in trained],
                          ["%.3f" % p[1] for p in plain], ["%.3f" % t[1] for t in trained]))
    assert st["loss_last"] < st["loss_first"]
    for p, t in zip(plain, trained):
        assert t[2] <= 1e-10 and p[2] <= 1e-10
    print("iteration gain %.2f, time gain %.2f" % (sum(p[0] for p in plain) / sum(t[0] for t in trained),
                                                  sum(p[1] for p in plain) / sum(t[1] for t in trained)))


def test_adam_step_matches_oracle():
    """Three Adam steps of the library (the update of dwf_precond_train) from
    given gradients against oracle.precond.adam_step, element by element: the
    FP64 master weights after each step (the moments enter the later steps), and
    the compute copy = the BF16 rounding of the master weights."""
    from oracle import precond as pc
    dims, Ls, L = (4, 4, 2, 4), 4, 2
    op, ref = make_pair(dims, Ls, 1.8, 0.05, 1.5, 0.5, "neff", 0.5, seed=231)
    w0 = random_weights(L, Ls, 232)
    op.precond_set_weights(w0)
    theta = op.precond_get_weights(L, compute_copy=False)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    g = np.random.default_rng(233)
    for t, lr in zip((1, 2, 3), (2e-3, 5e-3, 1e-3)):
        grad = g.normal(size=theta.shape) + 1j * g.normal(size=theta.shape)
        if t == 2:
            grad[0, 0] *= 1e-6                                      # small gradients: eps matters
        op.precond_adam_step(grad, lr, layers=L)
        theta, m, v = pc.adam_step(theta, grad, m, v, t, lr)
        got = op.precond_get_weights(L, compute_copy=False)
        assert np.abs(got - theta).max() <= 1e-14 * np.abs(theta).max(), t
        comp = op.precond_get_weights(L, compute_copy=True)
        assert np.abs(comp - theta).max() <= 2.0 ** -8 * np.abs(theta).max()


def test_save_load_round_trip(tmp_path):
    """dwf_precond_save / dwf_precond_load: the weights, the compute copy and the
    Adam state (the next step from the loaded state equals the next step from the
    original) survive the round trip; files for another Ls, truncated files and
    files of another format are refused."""
    from paper_2602_14454_gb300 import dwf
    dims, Ls, L = (4, 4, 2, 4), 4, 2
    op, ref = make_pair(dims, Ls, 1.8, 0.05, 1.5, 0.5, "neff", 0.5, seed=241)
    op.precond_set_weights(random_weights(L, Ls, 242))
    g = np.random.default_rng(243)
    shape = (L, 9, 2, Ls, Ls)
    for _ in range(2):
        op.precond_adam_step(g.normal(size=shape) + 1j * g.normal(size=shape), 3e-3, layers=L)
    path = str(tmp_path / "net.bin")
    op.precond_save(path)
    op2, _ = make_pair(dims, Ls, 1.8, 0.05, 1.5, 0.5, "neff", 0.5, seed=241)
    op2.precond_load(path)
    for cc in (False, True):
        assert np.array_equal(op2.precond_get_weights(L, cc), op.precond_get_weights(L, cc))
    r = to_gpu(even_field(ref, 244))
    assert np.array_equal(to_np(op2.precond_apply(r)), to_np(op.precond_apply(r)))
    grad = g.normal(size=shape) + 1j * g.normal(size=shape)
    op.precond_adam_step(grad, 3e-3, layers=L)
    op2.precond_adam_step(grad, 3e-3, layers=L)
    assert np.array_equal(op2.precond_get_weights(L, False), op.precond_get_weights(L, False))
    op3, _ = make_pair(dims, 6, 1.8, 0.05, 1.5, 0.5, "neff", 0.5, seed=241)
    with pytest.raises(dwf.DwfError):
        op3.precond_load(path)                                       # another Ls
    data = open(path, "rb").read()
    open(path + ".cut", "wb").write(data[: len(data) // 2])
    with pytest.raises(dwf.DwfError):
        op2.precond_load(path + ".cut")
    open(path + ".bad", "wb").write(b"X" + data[1:])
    with pytest.raises(dwf.DwfError):
        op2.precond_load(path + ".bad")


@pytest.mark.parametrize("plain", [False, True])
def test_fcg_cycle_matches_the_oracle_fcg(plain):
    """The library's flexible-CG cycle (the inner solve of dwf_solve with
    precond = 1, run alone by dwf_precond_fcg in FP32) against oracle.precond.fcg
    in FP64 on the same normal equation D^dag D x = b with the same
    preconditioner M = N N^dag (the oracle fed the kernels' BF16-rounded
    weights), step by step: the residual histories agree to FP32 accuracy, and
    so do the solutions.  plain: M = 1, the FCG of the oracle is then plain CG."""
    from oracle import precond as pc
    dims, Ls, L = (4, 4, 2, 4), 6, 2
    op, ref = make_pair(dims, Ls, 1.8, 0.1, 1.5, 0.5, "neff", 0.5, seed=251)
    op.precond_set_weights(random_weights(L, Ls, 252, scale=0.05))
    W = op.precond_get_weights(L, compute_copy=True)
    net = pc.Net(ref.U, dims, BC, W)
    b = even_field(ref, 253)
    x, hist = op.precond_fcg(to_gpu(b), tol=1e-5, max_iter=60, plain=plain)

    def A(v):
        return ref.d_pc(ref.d_pc(v), dag=True)
    M = (lambda v: v) if plain else net.precondition
    x_ref, info = pc.fcg(A, M, b, tol=1e-5, maxiter=60)
    want = np.array(info["history"])
    # the same recurrence: FP32 and FP64 agree step by step at first (finite
    # precision then lets the two drift apart slowly), and both stop after about
    # the same number of steps; the FP32 iterate's true residual (recomputed in
    # FP64) stalls near the FP32 rounding times the condition number of D^dag D
    # (about 1e-7 x 1e3 here), which the solver's FP64 defect corrections remove
    assert np.all(np.abs(np.log(hist[:16] / want[:16])) < 1e-4), (hist[:16], want[:16])
    assert abs(len(hist) - len(want)) <= 3
    xg = to_np(x)
    assert rel(A(xg), b) <= 1e-3
    assert rel(xg, x_ref) < 1e-2
