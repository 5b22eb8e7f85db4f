"""s-dependent coefficients (b_i, c_i) of eq. (domainwall_general) through the
C ABI (dwf_create_s) against the FP64 oracle: the whole 5D matrix, the even-odd
matrix, the source and the mixed-precision solve with its 4D solution.

The newest component: this file is collected last, so that a failure here
leaves every other test already run."""

import numpy as np
import pytest

from _util import TOL, make_pair, rel, to_gpu, to_np
from paper_2602_14454_gb300 import inputs

pytestmark = pytest.mark.gpu

W8 = np.array([0.35, 0.7, 1.1, 1.6, 1.9, 1.4, 0.9, 0.5])
CASES = [
    # dims, Ls, M0, mf, b_s, c_s
    ((4, 4, 4, 4), 8, 1.8, 0.04, tuple((W8 + 1) / 2), tuple((W8 - 1) / 2)),   # b_s - c_s = 1 (Mobius-like)
    ((4, 2, 6, 4), 8, 1.4, 0.02, tuple(W8), tuple(W8)),                       # b_s = c_s (Chiu's choice)
    ((2, 4, 4, 6), 6, 1.8, 0.1, (1.2, 0.7, 1.9, 1.1, 0.9, 1.4), (0.3, 0.6, 0.2, 0.8, 0.1, 0.5)),
]
IDS = ["mobius_like", "chiu_like", "general"]


@pytest.fixture(scope="module", autouse=True)
def _built(cuda_ok):
    from paper_2602_14454_gb300 import build
    build.build()


@pytest.mark.parametrize("case", CASES, ids=IDS)
@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
def test_full5d_and_eo_apply(case, prec):
    dims, Ls, M0, mf, b, c = case
    op, ref = make_pair(dims, Ls, M0, mf, b, c, "standard", 1.0, seed=51)
    x = inputs.gaussian_5d(dims, Ls, 52)
    xe = ref.to_eo(x, 0)
    for dag in (False, True):
        got = to_np(op.apply(to_gpu(x), op="full", prec=prec, dag=dag))
        assert rel(got, ref.apply(x, dag=dag)) < TOL[prec], dag
        got = to_np(op.apply(to_gpu(xe), op="eo", prec=prec, dag=dag))
        assert rel(got, ref.d_pc(xe, dag=dag)) < TOL[prec], dag


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_source_uses_the_end_coefficients(case):
    dims, Ls, M0, mf, b, c = case
    op, ref = make_pair(dims, Ls, M0, mf, b, c, "standard", 1.0, seed=53)
    b4 = inputs.gaussian_4d(dims, 54)
    assert rel(to_np(op.source_5d(to_gpu(b4))), ref.source_5d(b4)) < 1e-13
    assert op.mix_mode("f64") == 0   # the structured FP64 form assumes constant coefficients


@pytest.mark.parametrize("case", CASES[:2], ids=IDS[:2])
@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
def test_solve_and_4d_solution(case, prec):
    dims, Ls, M0, mf, b, c = case
    op, ref = make_pair(dims, Ls, M0, mf, b, c, "standard", 1.0, seed=55)
    b4 = inputs.gaussian_4d(dims, 56)
    b5 = ref.source_5d(b4)
    x5, st = op.solve(to_gpu(b5), inner_prec=prec, tol=1e-10)
    x5 = to_np(x5)
    assert rel(ref.apply(x5), b5) <= 1e-10
    x5_ref, _ = ref.solve(b5, tol=1e-13)
    assert rel(ref.project_4d(x5), ref.project_4d(x5_ref)) < 1e-9
