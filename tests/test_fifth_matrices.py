"""Host-built fifth-direction matrices (dwf_fifth_matrix_host, no device) against
the oracle and the algebra of Sec. 2.3.

The kernels apply per-chirality Ls x Ls matrices built on the host; these tests
run on the CPU.  D_ee = A5 R is compared with the oracle's site-local block of
the full operator (built independently, block by block, from eq.
domainwall_general / domainwall_neff); the Neff factor R with the oracle's
D_ee^(alpha) = D_ee^(1) R; the remaining matrices with their definitions
(products, inverses, transposes, scalings) and the cyclic-tridiagonal flags
with their nonzero patterns.
"""

import numpy as np
import pytest

from oracle import dwf as orc
from paper_2602_14454_gb300 import dwf, inputs

PARAMS = [(8, 1.8, 0.04, 1.0, 0.0, "standard", 1.0), (16, 1.8, 0.01, 1.5, 0.5, "neff", 0.5),
          (12, 1.0, 0.05, 1.0, 1.0, "neff", 0.3), (6, 1.8, 0.1, 1.5, 0.5, "standard", 1.0),
          # s-dependent coefficients (rows of eq. domainwall_general), standard form
          (6, 1.8, 0.05, (1.2, 0.7, 1.9, 1.1, 0.9, 1.4), (0.3, 0.6, 0.2, 0.8, 0.1, 0.5), "standard", 1.0),
          (8, 1.4, 0.02, (0.4, 0.9, 1.3, 1.7, 1.7, 1.3, 0.9, 0.4), (0.4, 0.9, 1.3, 1.7, 1.7, 1.3, 0.9, 0.4),
           "standard", 1.0)]


def host(p, which, chi):
    Ls, M0, mf, b, c, form, alpha = p
    return dwf.fifth_matrix_host(Ls, M0, mf, b, c, form, alpha, which, chi)


def oracle_dee(p, form=None, alpha=None):
    Ls, M0, mf, b, c, f, a = p
    U = inputs.random_links((2, 2, 2, 2), 0.5, 1)
    op = orc.DWF(U, (2, 2, 2, 2), Ls, M0, mf, b, c, form=form or f, alpha=a if alpha is None else alpha)
    return op.site_matrix()   # (4 Ls x 4 Ls) over (s, spin)


def chirality_block(L, chi, spin_in_block=0):
    sp = 2 * chi + spin_in_block
    return L[sp::4, sp::4]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2602_14454_gb300 import build
    build.build()   # host code only below: no device is touched


@pytest.mark.parametrize("p", PARAMS)
def test_dee_matches_the_oracle_site_block(p):
    L = oracle_dee(p)
    for chi in (0, 1):
        A5R, band = host(p, "A5R", chi)
        for s in (0, 1):
            assert np.allclose(chirality_block(L, chi, s), A5R, rtol=0, atol=1e-13)
        # D_ee does not mix chiralities
        other = L[2 * chi::4, 2 * (1 - chi)::4]
        assert np.abs(other).max() == 0.0
        assert np.allclose(host(p, 0, chi)[0] @ host(p, 3, chi)[0], A5R, rtol=0, atol=1e-13)


@pytest.mark.parametrize("p", PARAMS)
def test_neff_factor_matches_the_oracle(p):
    Ls, M0, mf, b, c, form, alpha = p
    L1 = oracle_dee(p, form="standard", alpha=1.0)
    La = oracle_dee(p)
    for chi in (0, 1):
        R = host(p, 3, chi)[0]
        want = np.linalg.solve(chirality_block(L1, chi), chirality_block(La, chi))
        assert np.allclose(R, want, rtol=0, atol=1e-12)
        if form == "standard":
            assert np.array_equal(R, np.eye(Ls))


@pytest.mark.parametrize("p", PARAMS)
def test_kernel_matrices_follow_their_definitions(p):
    Ls = p[0]
    I = np.eye(Ls)
    for chi in (0, 1):
        A5, A5i, B, R = (host(p, k, chi)[0] for k in range(4))
        m = {k: host(p, k, chi)[0] for k in dwf.KERNEL_MATRICES}
        tol = dict(rtol=0, atol=1e-12)
        assert np.allclose(A5 @ A5i, I, **tol)
        assert np.allclose(m["P"], B @ R, **tol)
        assert np.allclose(m["Q"] @ m["A5R"], I, **tol)          # Q = D_ee^-1
        assert np.allclose(m["M"], B @ A5i, **tol)
        for k in ("P", "Q", "M", "A5R"):
            t = {"P": "PT", "Q": "QT", "M": "MT", "A5R": "RA5T"}[k]
            assert np.array_equal(m[t], m[k].T)
        assert np.allclose(m["NQ4"], -0.25 * m["Q"], **tol)
        assert np.allclose(m["HALF_Q"], 0.5 * m["Q"], **tol)
        assert np.allclose(m["NPT4"], -0.25 * m["P"].T, **tol)
        assert np.allclose(m["NHALF_RBT"], -0.5 * R @ B.T, **tol)
        assert np.array_equal(m["ID"], I) and np.array_equal(m["NHALF"], -0.5 * I)
        Ls_, M0, mf, b, c = p[:5]
        cs = np.broadcast_to(np.asarray(c, dtype=float), (Ls,))
        assert np.allclose(m["SRC_POST"], np.diag(0.5 * cs), **tol)
        assert np.allclose(m["SRC_Y"], np.diag(1 - cs * (4 - M0)), **tol)


@pytest.mark.parametrize("p", PARAMS)
def test_fifth_direction_hop_matches_the_oracle_blocks(p):
    """B = b + c K (per row s: b_s, c_s) against the D_W coefficients of the
    oracle's printed blocks, projected on each chirality; for the Neff form the
    oracle's blocks are those of D^(alpha) = D (P A P^dag), i.e. B R."""
    Ls, M0, mf, b, c, form, alpha = p
    U = inputs.random_links((2, 2, 2, 2), 0.5, 1)
    op = orc.DWF(U, (2, 2, 2, 2), Ls, M0, mf, b, c, form=form, alpha=alpha)
    for chi in (0, 1):
        sp = 2 * chi
        W = np.zeros((Ls, Ls))
        for bl in op.blocks():
            W[bl.s, bl.t] += (bl.cw * bl.S[sp, sp]).real
        B, R = host(p, 2, chi)[0], host(p, 3, chi)[0]
        assert np.allclose(W, B @ R, rtol=0, atol=1e-13)


@pytest.mark.parametrize("p", PARAMS)
def test_banded_flags_match_the_nonzero_pattern(p):
    Ls = p[0]
    s, t = np.meshgrid(np.arange(Ls), np.arange(Ls), indexing="ij")
    off_band = ~np.isin((t - s) % Ls, [0, 1, Ls - 1])
    for k in dwf.KERNEL_MATRICES:
        mats = [host(p, k, chi) for chi in (0, 1)]
        banded = all(np.all(M[off_band] == 0) for M, _ in mats)
        assert mats[0][1] == mats[1][1] == banded, k
    # the fifth-direction hop and D_ee are cyclic tridiagonal, their inverses are dense
    for k in ("P", "PT", "A5R", "RA5T"):
        assert host(p, k, 0)[1]
    for k in ("Q", "M"):
        assert not host(p, k, 0)[1]


def test_bad_arguments():
    with pytest.raises(dwf.DwfError):
        dwf.fifth_matrix_host(1, 1.8, 0.1, 1.0, 0.0, "standard", 1.0, 0, 0)
    with pytest.raises(dwf.DwfError):
        dwf.fifth_matrix_host(8, 1.8, 0.1, 1.0, 0.0, "standard", 1.0, 5, 0)
    with pytest.raises(dwf.DwfError):
        dwf.fifth_matrix_host(8, 1.8, 0.1, 1.0, 0.0, "neff", 0.0, 0, 0)
    with pytest.raises(dwf.DwfError):
        dwf.fifth_matrix_host(8, 1.8, 0.1, 1.0, 0.0, "standard", 1.0, 0, 2)
    with pytest.raises(dwf.DwfError):   # the Neff form takes constant coefficients
        dwf.fifth_matrix_host(4, 1.8, 0.1, (1.0, 1.1, 1.0, 1.0), 0.0, "neff", 0.5, 0, 0)
