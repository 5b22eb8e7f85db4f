"""Pins of the oracle with s-dependent coefficients (b_i, c_i) of eq.
(domainwall_general), Sec. 2.2: row i of the 5D matrix holds D_+^(i) = b_i D_W + 1
and D_-^(i) = c_i D_W - 1 (Chiu's optimal domain-wall fermion chooses b_i = c_i
depending on i).

Checked against a closed form: with b_i - c_i = d independent of i, the 4D
solution from the 5D solve is (D_eff^-1 - 1) b4 / (1 - m) with
D_eff = (1+m)/2 + (1-m)/2 gamma5 eps(H), H = gamma5 D_W [2 + d D_W]^-1 and
eps(H) = [prod_i (1 + w_i H) - prod_i (1 - w_i H)] [prod_i (1 + w_i H) + prod_i (1 - w_i H)]^-1,
w_i = b_i + c_i (every factor is a function of the same H, so they commute).
Also: constant sequences reproduce the scalar operator, the dense adjoint,
and the Neff form refuses s-dependent coefficients.
"""

import numpy as np
import pytest

from oracle import dwf
from paper_2602_14454_gb300 import inputs

TINY = (2, 2, 2, 4)


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300)


def dense_dw(op):
    V = int(np.prod(op.dims))
    n4 = V * 12
    E = np.eye(n4).reshape((n4,) + op.site_shape + (4, 3))
    return op.dw(E).reshape(n4, n4).T


def g5_4d(V):
    return np.kron(np.eye(V), np.kron(dwf.GAMMA5, np.eye(3)))


@pytest.mark.parametrize("d", [0.0, 1.0])
def test_s_dependent_effective_operator(d):
    Ls, m, M0 = 5, 0.1, 1.8
    w = np.array([0.35, 0.9, 1.7, 0.6, 1.2])          # b_i + c_i, s-dependent
    bs, cs = (w + d) / 2, (w - d) / 2
    U = inputs.random_links(TINY, 0.5, 7)
    op = dwf.DWF(U, TINY, Ls, M0, m, bs, cs)
    DW = dense_dw(op)
    n4 = DW.shape[0]
    I = np.eye(n4)
    g5 = g5_4d(32)
    H = g5 @ DW @ np.linalg.inv(2 * I + d * DW)
    Tp, Tm = I.copy(), I.copy()
    for wi in w:
        Tp = Tp @ (I + wi * H)
        Tm = Tm @ (I - wi * H)
    Deff = (1 + m) / 2 * I + (1 - m) / 2 * g5 @ (Tp - Tm) @ np.linalg.inv(Tp + Tm)
    b4 = inputs.gaussian_4d(TINY, 3)
    x4_closed = ((np.linalg.inv(Deff) - I) @ b4.ravel()) / (1 - m)
    b5 = op.source_5d(b4)
    x5 = np.linalg.solve(op.dense(), b5.ravel()).reshape(b5.shape)
    assert rel(op.project_4d(x5).ravel(), x4_closed) < 1e-11


def test_constant_sequences_reproduce_the_scalar_operator():
    U = inputs.random_links(TINY, 0.5, 8)
    a = dwf.DWF(U, TINY, 4, 1.8, 0.05, 1.5, 0.5)
    b = dwf.DWF(U, TINY, 4, 1.8, 0.05, [1.5] * 4, [0.5] * 4)
    x = inputs.gaussian_5d(TINY, 4, 9)
    assert np.array_equal(a.apply(x), b.apply(x))
    assert np.array_equal(a.source_5d(x[0]), b.source_5d(x[0]))


def test_s_dependent_adjoint_and_source():
    Ls = 4
    bs, cs = [1.2, 0.7, 1.9, 1.1], [0.3, 0.6, 0.2, 0.8]
    U = inputs.random_links(TINY, 0.5, 10)
    op = dwf.DWF(U, TINY, Ls, 1.8, 0.05, bs, cs)
    g = np.random.default_rng(11)
    shape = (Ls,) + op.site_shape + (4, 3)
    x = g.normal(size=shape) + 1j * g.normal(size=shape)
    y = g.normal(size=shape) + 1j * g.normal(size=shape)
    assert abs(np.vdot(y, op.apply(x)) - np.vdot(op.apply(y, dag=True), x)) < 1e-11 * np.abs(np.vdot(y, op.apply(x)))
    # b5 = (-D_-) P^dag (0, .., b4): slice 1 is (1 - c_1 D_W) P_+ b4, slice Ls is (1 - c_Ls D_W) P_- b4
    b4 = inputs.gaussian_4d(TINY, 12)
    b5 = op.source_5d(b4)
    pp, pm = dwf.spin(dwf.P_PLUS, b4), dwf.spin(dwf.P_MINUS, b4)
    assert rel(b5[0], pp - cs[0] * op.dw(pp)) < 1e-14
    assert rel(b5[Ls - 1], pm - cs[Ls - 1] * op.dw(pm)) < 1e-14
    assert np.abs(b5[1:Ls - 1]).max() == 0


def test_neff_form_refuses_s_dependent_coefficients():
    U = inputs.random_links(TINY, 0.5, 13)
    with pytest.raises(ValueError):
        dwf.DWF(U, TINY, 4, 1.8, 0.05, [1.0, 1.1, 1.0, 1.0], 0.0, form="neff", alpha=0.5)
