"""The 5D even-odd split (Sec. 2.3's alternative to the 4D split) on the GPU:
its Schur complement and adjoint against the oracle's, and the solve through
it against the oracle's residual and the 4D route's solution."""

import numpy as np
import pytest

from _util import TOL, make_pair, maxrel, rel, to_gpu, to_np
from paper_2602_14454_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built(cuda_ok):
    from paper_2602_14454_gb300 import build
    build.build()


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("b,Ls,dims", [(1.0, 8, (4, 4, 2, 4)), (1.5, 4, (2, 4, 4, 6)), (1.2, 16, (4, 2, 2, 4))])
def test_eo5_schur_complement(prec, b, Ls, dims):
    op, ref = make_pair(dims, Ls, 1.8, 0.03, b, 0.0, "standard", 1.0, seed=91)
    par = ref.parity5()
    x = np.where(par == 0, inputs.gaussian_5d(dims, Ls, 92), 0)
    for dag in (False, True):
        got = to_np(op.apply(to_gpu(x), op="eo5", prec=prec, dag=dag))
        want = ref.d_pc5(x, dag=dag)
        assert rel(got, want) < TOL[prec], (dag, rel(got, want))
        assert maxrel(got[np.broadcast_to(par == 0, got.shape)], want[np.broadcast_to(par == 0, want.shape)]) < 10 * TOL[prec]
        assert not np.any(got[np.broadcast_to(par == 1, got.shape)])


def test_eo5_refused_where_the_blocks_are_not_diagonal():
    from paper_2602_14454_gb300 import dwf
    dims = (2, 2, 2, 4)
    for Ls, c, form in ((8, 0.5, "standard"), (5, 0.0, "standard"), (8, 0.0, "neff")):
        op, ref = make_pair(dims, Ls, 1.8, 0.03, 1.0, c, form, 0.5, seed=93)
        with pytest.raises(dwf.DwfError):
            op.apply(to_gpu(inputs.gaussian_5d(dims, Ls, 94)), op="eo5")


@pytest.mark.parametrize("b", [1.0, 1.5])
def test_eo5_solve_matches_oracle_and_4d_route(b):
    """FP64 CGNR through the 5D split: the oracle recomputes ||b5 - D x5|| <=
    1e-10 ||b5||, the solution equals the 4D route's (dwf_solve, FP64), and the
    residual history follows the oracle's CGNR on the 5D Schur complement."""
    dims, Ls = (4, 4, 2, 4), 8
    op, ref = make_pair(dims, Ls, 1.8, 0.05, b, 0.0, "standard", 1.0, seed=95)
    b5 = inputs.gaussian_5d(dims, Ls, 96)
    x5, hist = op.solve_eo5(to_gpu(b5), tol=1e-10, max_iter=3000)
    x5 = to_np(x5)
    assert rel(ref.apply(x5), b5) <= 1e-10
    x4d, st = op.solve(to_gpu(b5), inner_prec="f64", tol=1e-11)
    assert rel(x5, to_np(x4d)) < 1e-8
    _, info = ref.solve_eo5(b5, tol=1e-10)
    k = min(20, len(hist), len(info["history"]))
    assert np.allclose(np.log(hist[:k]), np.log(info["history"][:k]), atol=1e-6)
    print("iterations: 5D split %d, 4D split %d" % (len(hist) - 1, st["iterations"]))
