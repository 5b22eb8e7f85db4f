"""Spectrum of D^dag D for the even-odd matrix (test infrastructure only).

Sec. 3.2 ("Condition number"): the paper measures the smallest and largest
eigenvalues of D^dag D, D the even-odd preconditioned matrix of Sec. 2.3 in
the standard or Neff form, and takes their ratio as the condition number that
governs CG.  Here the dense matrix of D is built column by column from
DWF.d_pc applied to unit vectors of the even half field, and numpy's Hermitian
eigenvalue routine gives every eigenvalue of D^dag D.  Tiny lattices only
(the dense matrix has (Ls * Vh * 12)^2 entries).

The second even-odd form of Sec. 2.3, eq. (another_even-odd_linear_equation),
D' = 1 - D_eo D_oo^-1 D_oe D_ee^-1, is built the same way from the blocks of
the full operator (DWF.D_block, DWF.Dinv_site); the paper notes that alpha
cancels in it.

Pinned in tests/test_oracle_spectrum.py by Rayleigh quotients computed with
DWF.d_pc itself, by the alpha = 1 Neff form equalling the standard form, by
the similarity D^(alpha) = R^-1 D R of Sec. 2.3 (the eigenvalues of D do not
depend on alpha, those of D^dag D do), and for D' by its similarity to D
(D' = D_ee D D_ee^-1) and its independence of alpha.
"""

from __future__ import annotations

import numpy as np


def d_pc_dense(op) -> np.ndarray:
    """Dense matrix of the even-odd operator D: column k = D e_k, the unit vectors
    e_k of the even half field (Ls, Vh, 4, 3) in C order."""
    eo = op._eo_setup()
    shape = (op.Ls, len(eo["even"]), 4, 3)
    n = int(np.prod(shape))
    D = np.empty((n, n), dtype=np.complex128)
    e = np.zeros(shape, dtype=np.complex128)
    for k in range(n):
        e.flat[k] = 1.0
        D[:, k] = op.d_pc(e).ravel()
        e.flat[k] = 0.0
    return D


def alt_apply(op, y):
    """D' y = y - D_eo D_oo^-1 D_oe D_ee^-1 y, eq. (another_even-odd_linear_equation)."""
    return y - op.D_block(0, 1, op.Dinv_site(op.D_block(1, 0, op.Dinv_site(y))))


def alt_dense(op) -> np.ndarray:
    """Dense matrix of D' (columns from unit vectors, as d_pc_dense)."""
    eo = op._eo_setup()
    shape = (op.Ls, len(eo["even"]), 4, 3)
    n = int(np.prod(shape))
    D = np.empty((n, n), dtype=np.complex128)
    e = np.zeros(shape, dtype=np.complex128)
    for k in range(n):
        e.flat[k] = 1.0
        D[:, k] = alt_apply(op, e).ravel()
        e.flat[k] = 0.0
    return D


def normal_spectrum(op, eo_form=0) -> np.ndarray:
    """All eigenvalues of D^dag D in ascending order (eo_form 1: of D'^dag D')."""
    D = d_pc_dense(op) if eo_form == 0 else alt_dense(op)
    return np.linalg.eigvalsh(D.conj().T @ D)


def condition_number(op, eo_form=0):
    """(lambda_min, lambda_max, lambda_max / lambda_min) of D^dag D (Sec. 3.2)."""
    ev = normal_spectrum(op, eo_form)
    return ev[0], ev[-1], ev[-1] / ev[0]
