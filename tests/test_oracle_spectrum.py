"""Pins of the oracle's spectrum of D^dag D (oracle/spectrum.py, Sec. 3.2).

Each test checks the dense-matrix route against something other than itself:
Rayleigh quotients and eigenvector residuals computed with DWF.d_pc (the
operator the solver tests already pin), the Neff form at alpha = 1 against the
standard form, and the similarity D^(alpha) = R^-1 D R of Sec. 2.3 (the
eigenvalues of D are independent of alpha while those of D^dag D are not,
which is the paper's premise).
"""

import numpy as np
import pytest

from oracle import dwf, spectrum
from paper_2602_14454_gb300 import inputs

TINY = (2, 2, 2, 4)
LS = 4


def make(form, alpha, b=1.5, c=0.5, mf=0.05, seed=311):
    U = inputs.random_links(TINY, 0.5, seed)
    return dwf.DWF(U, TINY, LS, 1.8, mf, b, c, form=form, alpha=alpha)


@pytest.fixture(scope="module")
def neff05():
    op = make("neff", 0.5)
    D = spectrum.d_pc_dense(op)
    return op, D


def test_rayleigh_quotients_lie_in_the_spectrum(neff05):
    op, D = neff05
    ev, vec = np.linalg.eigh(D.conj().T @ D)
    g = np.random.default_rng(5)
    shape = (op.Ls, len(op._eo_setup()["even"]), 4, 3)
    for _ in range(10):
        x = g.normal(size=shape) + 1j * g.normal(size=shape)
        q = np.vdot(op.d_pc(x), op.d_pc(x)).real / np.vdot(x, x).real
        assert ev[0] * (1 - 1e-12) <= q <= ev[-1] * (1 + 1e-12)
    # the extremal eigenvectors: |D v|^2 = lambda and D^dag D v = lambda v through d_pc
    for j in (0, -1):
        v = vec[:, j].reshape(shape)
        Dv = op.d_pc(v)
        assert abs(np.vdot(Dv, Dv).real - ev[j]) <= 1e-11 * ev[-1]
        r = op.d_pc(Dv, dag=True) - ev[j] * v
        assert np.linalg.norm(r) <= 1e-10 * ev[-1]


def test_dense_columns_match_the_operator(neff05):
    op, D = neff05
    g = np.random.default_rng(6)
    shape = (op.Ls, len(op._eo_setup()["even"]), 4, 3)
    x = g.normal(size=shape) + 1j * g.normal(size=shape)
    assert np.allclose(D @ x.ravel(), op.d_pc(x).ravel(), rtol=0, atol=1e-12 * np.abs(D).max() * np.abs(x).sum())
    assert np.allclose(D.conj().T @ x.ravel(), op.d_pc(x, dag=True).ravel(), rtol=0,
                       atol=1e-12 * np.abs(D).max() * np.abs(x).sum())


def test_neff_alpha_one_is_the_standard_form():
    a = spectrum.normal_spectrum(make("neff", 1.0))
    b = spectrum.normal_spectrum(make("standard", 1.0))
    assert np.allclose(a, b, rtol=1e-11, atol=1e-13 * b[-1])


def test_alpha_changes_the_normal_spectrum_not_the_spectrum_of_d(neff05):
    op, D05 = neff05
    D10 = spectrum.d_pc_dense(make("standard", 1.0))
    e05 = np.linalg.eigvals(D05)
    e10 = np.linalg.eigvals(D10)
    # the same multiset of eigenvalues of D (similarity by R): match greedily
    rest = list(e10)
    scale = np.abs(e10).max()
    for z in e05:
        k = int(np.argmin(np.abs(np.array(rest) - z)))
        assert abs(rest[k] - z) <= 1e-8 * scale
        rest.pop(k)
    # while D^dag D differs (the condition number depends on alpha)
    s05 = np.linalg.eigvalsh(D05.conj().T @ D05)
    s10 = np.linalg.eigvalsh(D10.conj().T @ D10)
    assert abs(s05[-1] / s05[0] - s10[-1] / s10[0]) > 1e-3 * (s10[-1] / s10[0])


def test_condition_number_is_the_ratio():
    lo, hi, k = spectrum.condition_number(make("standard", 1.0, b=1.0, c=0.0))
    assert 0 < lo < hi and k == pytest.approx(hi / lo, rel=1e-15)


def test_second_even_odd_form_is_similar_to_d_and_alpha_free(neff05):
    """D' = 1 - D_eo D_oo^-1 D_oe D_ee^-1 = D_ee D D_ee^-1 (same eigenvalues as D), and,
    as Sec. 2.3 argues, the Neff factor cancels in it: D'^dag D' is the same for
    every alpha."""
    op, D05 = neff05
    A05 = spectrum.alt_dense(op)
    e_d = np.linalg.eigvals(D05)
    e_a = np.linalg.eigvals(A05)
    rest = list(e_a)
    scale = np.abs(e_a).max()
    for z in e_d:
        k = int(np.argmin(np.abs(np.array(rest) - z)))
        assert abs(rest[k] - z) <= 1e-8 * scale
        rest.pop(k)
    s05 = np.linalg.eigvalsh(A05.conj().T @ A05)
    s10 = spectrum.normal_spectrum(make("standard", 1.0), eo_form=1)
    s03 = spectrum.normal_spectrum(make("neff", 0.3), eo_form=1)
    assert np.allclose(s05, s10, rtol=1e-10, atol=1e-12 * s10[-1])
    assert np.allclose(s03, s10, rtol=1e-10, atol=1e-12 * s10[-1])
    # and it is not the spectrum of D^dag D (the forms differ by the non-unitary D_ee)
    s_d = np.linalg.eigvalsh(D05.conj().T @ D05)
    assert abs(s_d[-1] / s_d[0] - s05[-1] / s05[0]) > 1e-3 * (s05[-1] / s05[0])
