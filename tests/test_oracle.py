"""Pins of the FP64 oracle against facts fixed by the paper and by the mathematics.

Each test checks the oracle against something other than itself: closed forms
(free-field momentum space, the Mobius/overlap effective operator), identities
printed in Sec. 2.3, structural invariants (gauge covariance, adjointness,
Gamma-hermiticity), brute force on tiny lattices (dense matrices), and the
paper's own claims (4D solution independent of alpha, the second even-odd form
independent of alpha).
"""

import numpy as np
import pytest

from oracle import _clib, dwf
from paper_2602_14454_gb300 import inputs

TINY = (2, 2, 2, 4)
BC_SETS = [(1, 1, 1, -1), (1, 1, 1, 1), (-1, 1, 1, -1)]
BCS_PARAMS = [(1.0, 0.0), (1.5, 0.5), (1.0, 1.0)]


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300)


def dense_dw(op):
    V = int(np.prod(op.dims))
    n4 = V * 12
    E = np.eye(n4).reshape((n4,) + op.site_shape + (4, 3))
    return op.dw(E).reshape(n4, n4).T, op.dw(E, dag=True).reshape(n4, n4).T


def g5_4d(V):
    return np.kron(np.eye(V), np.kron(dwf.GAMMA5, np.eye(3)))


# ------------------------------------------------------------------ spin algebra
def test_gamma_algebra():
    G = dwf.GAMMA
    for mu in range(4):
        assert np.allclose(G[mu], G[mu].conj().T)
        assert np.array_equal(_clib.gamma_table(mu), G[mu])  # C table == Python construction
        for nu in range(4):
            ac = G[mu] @ G[nu] + G[nu] @ G[mu]
            assert np.allclose(ac, 2.0 * (mu == nu) * np.eye(4), atol=1e-15)
    # gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 (Sec. 2.1) is diag(1,1,-1,-1) in this basis
    assert np.allclose(dwf.GAMMA5, np.diag([1, 1, -1, -1]))
    for P in (dwf.P_PLUS, dwf.P_MINUS):
        assert np.allclose(P @ P, P)
    assert np.allclose(dwf.P_PLUS @ dwf.P_MINUS, 0)


# --------------------------------------------------------------- Wilson operator
@pytest.mark.parametrize("bc", BC_SETS)
def test_wilson_free_field_plane_waves(bc):
    """D_W e^{ipx} v = e^{ipx} [sum_mu (1 - cos p_mu) - M0 + i sum_mu gamma_mu sin p_mu] v."""
    dims = (4, 2, 6, 4)
    M0 = 1.3
    op = dwf.DWF(inputs.unit_links(dims), dims, 4, M0, 0.1, 1.0, 0.0, bc=bc)
    g = np.random.default_rng(5)
    Lx, Ly, Lz, Lt = dims
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    coords = (x, y, z, t)
    for trial in range(6):
        n = [g.integers(0, L) for L in dims]
        p = [(2 * np.pi * n[mu] + (np.pi if bc[mu] == -1 else 0.0)) / dims[mu] for mu in range(4)]
        phase = np.exp(1j * sum(p[mu] * coords[mu] for mu in range(4)))
        v = g.normal(size=(4, 3)) + 1j * g.normal(size=(4, 3))
        psi = phase[..., None, None] * v
        Dp = (sum(1 - np.cos(p[mu]) for mu in range(4)) - M0) * np.eye(4) \
            + 1j * sum(dwf.GAMMA[mu] * np.sin(p[mu]) for mu in range(4))
        want = phase[..., None, None] * (Dp @ v)
        assert rel(op.dw(psi), want) < 1e-13
        want_dag = phase[..., None, None] * (Dp.conj().T @ v)
        assert rel(op.dw(psi, dag=True), want_dag) < 1e-13


def test_wilson_dense_adjoint_and_gamma5_hermiticity():
    U = inputs.random_links(TINY, 0.6, 11)
    op = dwf.DWF(U, TINY, 4, 1.8, 0.1, 1.0, 0.0)
    DW, DWd = dense_dw(op)
    assert np.abs(DWd - DW.conj().T).max() < 1e-14       # explicit adjoint == conjugate transpose
    g5 = g5_4d(32)
    assert np.abs(g5 @ DW @ g5 - DW.conj().T).max() < 1e-14


def gauge_transform(U, g):
    Ug = np.empty_like(U)
    for mu in range(4):
        gfwd = np.roll(g, -1, axis=(3, 2, 1, 0)[mu])
        Ug[mu] = g @ U[mu] @ np.swapaxes(gfwd.conj(), -1, -2)
    return Ug


def test_gauge_covariance_wilson_and_dwf():
    dims = (4, 2, 2, 4)
    U = inputs.random_links(dims, 0.7, 21)
    g = inputs.random_gauge_transform(dims, 22)
    Ug = gauge_transform(U, g)
    for form in ("standard", "neff"):
        op = dwf.DWF(U, dims, 5, 1.8, 0.07, 1.5, 0.5, form=form, alpha=0.6)
        opg = dwf.DWF(Ug, dims, 5, 1.8, 0.07, 1.5, 0.5, form=form, alpha=0.6)
        x = inputs.gaussian_5d(dims, 5, 23)
        gx = np.einsum("...ab,s...ib->s...ia", g, x)
        for dag in (False, True):
            lhs = opg.apply(gx, dag=dag)
            rhs = np.einsum("...ab,s...ib->s...ia", g, op.apply(x, dag=dag))
            assert rel(lhs, rhs) < 1e-13


# ------------------------------------------------------------ 5D operator pins
@pytest.mark.parametrize("bcp", BCS_PARAMS)
@pytest.mark.parametrize("form,alpha", [("standard", 1.0), ("neff", 0.45)])
def test_overlap_effective_operator(bcp, form, alpha):
    """4D solution from the 5D solve equals (D_eff^-1 - 1) b4 / (1 - m), with the
    Mobius effective operator D_eff = (1+m)/2 + (1-m)/2 gamma5 eps(H_M),
    H_M = gamma5 (b+c) D_W [2 + (b-c) D_W]^-1,
    eps(H) = [(1+H)^Ls - (1-H)^Ls] [(1+H)^Ls + (1-H)^Ls]^-1.
    This pins the printed 5D matrices, the mass corners, the source and the projection."""
    b, c = bcp
    Ls, m, M0 = 4, 0.1, 1.8
    U = inputs.random_links(TINY, 0.5, 7)
    op = dwf.DWF(U, TINY, Ls, M0, m, b, c, form=form, alpha=alpha)
    DW, _ = dense_dw(op)
    n4 = DW.shape[0]
    I = np.eye(n4)
    g5 = g5_4d(32)
    H = g5 @ ((b + c) * DW) @ np.linalg.inv(2 * I + (b - c) * DW)
    Tp, Tm = np.linalg.matrix_power(I + H, Ls), np.linalg.matrix_power(I - H, Ls)
    Deff = (1 + m) / 2 * I + (1 - m) / 2 * g5 @ (Tp - Tm) @ np.linalg.inv(Tp + Tm)
    b4 = inputs.gaussian_4d(TINY, 3)
    x4_closed = ((np.linalg.inv(Deff) - I) @ b4.ravel()) / (1 - m)
    D5 = op.dense()
    b5 = op.source_5d(b4)
    x5 = np.linalg.solve(D5, b5.ravel()).reshape(b5.shape)
    assert rel(op.project_4d(x5).ravel(), x4_closed) < 1e-12


def test_free_field_zero_momentum_mass():
    """Free field, zero momentum, Shamir (b=1, c=0) at M0 = 1: the transfer-matrix
    kernel is h = -M0/(2-M0) = -1, so eps(h) = -1 for every Ls and D_eff = m exactly.
    A constant source b4 then has the 4D solution b4/m, for both forms."""
    dims = (2, 2, 2, 2)
    m = 0.05
    for Ls in (3, 6):
        for form in ("standard", "neff"):
            op = dwf.DWF(inputs.unit_links(dims), dims, Ls, 1.0, m, 1.0, 0.0, bc=(1, 1, 1, 1),
                         form=form, alpha=0.4)
            v = np.random.default_rng(1).normal(size=(4, 3)) + 0j
            b4 = np.broadcast_to(v, op.site_shape + (4, 3)).copy()
            x5 = np.linalg.solve(op.dense(), op.source_5d(b4).ravel()).reshape((Ls,) + b4.shape)
            assert rel(op.project_4d(x5), b4 / m) < 1e-12


@pytest.mark.parametrize("form", ["standard", "neff"])
def test_adjoint_identity_5d(form):
    dims = (4, 2, 2, 4)
    U = inputs.random_links(dims, 0.5, 31)
    for (b, c) in BCS_PARAMS:
        op = dwf.DWF(U, dims, 6, 1.8, 0.02, b, c, form=form, alpha=0.55)
        x = inputs.gaussian_5d(dims, 6, 32)
        y = inputs.gaussian_5d(dims, 6, 33)
        lhs = dwf.inner(y, op.apply(x))
        rhs = dwf.inner(op.apply(y, dag=True), x)
        assert abs(lhs - rhs) / abs(lhs) < 1e-13
        xe, ye = op.to_eo(x, 0), op.to_eo(y, 0)
        lhs = dwf.inner(ye, op.d_pc(xe))
        rhs = dwf.inner(op.d_pc(ye, dag=True), xe)
        assert abs(lhs - rhs) / abs(lhs) < 1e-13


def test_neff_relation_and_P_unitary():
    """D^(alpha) P = D^(alpha=1) P A  and  P P^dag = P^dag P = 1 (Sec. 2.3)."""
    dims = (2, 2, 2, 4)
    U = inputs.random_links(dims, 0.5, 41)
    for (b, c) in BCS_PARAMS:
        for alpha in (0.3, 0.7, 1.6):
            st = dwf.DWF(U, dims, 5, 1.8, 0.03, b, c)
            nf = dwf.DWF(U, dims, 5, 1.8, 0.03, b, c, form="neff", alpha=alpha)
            x = inputs.gaussian_5d(dims, 5, 42)
            assert rel(nf.apply(nf.P(x)), st.apply(st.P(nf.A(x)))) < 1e-14
            assert rel(nf.P(nf.P(x, dag=True)), x) < 1e-15
            assert rel(nf.P(nf.P(x), dag=True), x) < 1e-15
    st = dwf.DWF(U, dims, 5, 1.8, 0.03, 1.5, 0.5)
    one = dwf.DWF(U, dims, 5, 1.8, 0.03, 1.5, 0.5, form="neff", alpha=1.0)
    x = inputs.gaussian_5d(dims, 5, 43)
    assert rel(one.apply(x), st.apply(x)) == 0.0


def test_gamma_hermiticity():
    """Gamma = gamma5 R5: Gamma D_-^-1 D is Hermitian; for Neff, R Gamma D_-^-1 D^(alpha)
    with R = P A P^dag is Hermitian."""
    dims = (2, 2, 2, 2)
    Ls = 4
    U = inputs.random_links(dims, 0.5, 51)
    V = 16
    for (b, c) in BCS_PARAMS:
        for form in ("standard", "neff"):
            op = dwf.DWF(U, dims, Ls, 1.8, 0.05, b, c, form=form, alpha=0.6)
            D5 = op.dense()
            DW, _ = dense_dw(op)
            Dm = c * DW - np.eye(V * 12)
            Dm5 = np.kron(np.eye(Ls), Dm)
            R5 = np.fliplr(np.eye(Ls))
            Gam = np.kron(R5, g5_4d(V))
            X = Gam @ np.linalg.solve(Dm5, D5)
            if form == "neff":
                n = D5.shape[0]
                Rm = np.zeros((n, n), dtype=complex)
                for j in range(n):
                    e = np.zeros(n, dtype=complex)
                    e[j] = 1
                    Rm[:, j] = op.P(op.A(op.P(e.reshape((Ls,) + op.site_shape + (4, 3)), dag=True))).ravel()
                X = Rm @ X
            assert np.abs(X - X.conj().T).max() / np.abs(X).max() < 1e-13


# -------------------------------------------------------------- even-odd route
def test_site_matrix_is_masked_operator():
    dims = (2, 2, 2, 4)
    op = dwf.DWF(inputs.random_links(dims, 0.5, 61), dims, 5, 1.8, 0.04, 1.5, 0.5, form="neff", alpha=0.5)
    x = inputs.gaussian_5d(dims, 5, 62)
    for par in (0, 1):
        xp = op.to_eo(x, par)
        assert rel(op.D_block(par, par, xp), op.site_apply(op.site_matrix(), xp)) < 1e-14
        assert rel(op.Dinv_site(op.site_apply(op.site_matrix(), xp)), xp) < 1e-13


@pytest.mark.parametrize("form", ["standard", "neff"])
def test_eo_route_equals_dense_solve(form):
    dims = (2, 2, 2, 4)
    op = dwf.DWF(inputs.random_links(dims, 0.5, 71), dims, 4, 1.8, 0.05, 1.5, 0.5, form=form, alpha=0.5)
    b5 = inputs.gaussian_5d(dims, 4, 72)
    x_dense = np.linalg.solve(op.dense(), b5.ravel()).reshape(b5.shape)
    x_eo, info = op.solve(b5, tol=1e-14)
    assert rel(x_eo, x_dense) < 1e-11
    assert rel(op.apply(x_eo), b5) < 1e-12


def test_eo_similarity_and_alternative_form():
    """D_pc^(alpha) = R^-1 D_pc R: same eigenvalues, different singular values;
    the second even-odd form (1 - D_eo D_oo^-1 D_oe D_ee^-1) does not depend on alpha."""
    dims = (2, 2, 2, 2)
    U = inputs.random_links(dims, 0.5, 81)
    st = dwf.DWF(U, dims, 4, 1.8, 0.05, 1.5, 0.5)
    nf = dwf.DWF(U, dims, 4, 1.8, 0.05, 1.5, 0.5, form="neff", alpha=0.5)
    n = 4 * 8 * 12

    def dense_eo(f):
        M = np.zeros((n, n), dtype=complex)
        for j in range(n):
            e = np.zeros(n, dtype=complex)
            e[j] = 1
            M[:, j] = f(e.reshape(4, 8, 4, 3)).ravel()
        return M

    A1 = dense_eo(st.d_pc)
    Aa = dense_eo(nf.d_pc)
    ev1 = np.linalg.eigvals(A1)
    eva = np.linalg.eigvals(Aa)
    dist = np.abs(ev1[:, None] - eva[None, :])
    assert dist.min(axis=1).max() < 1e-9 and dist.min(axis=0).max() < 1e-9
    s1 = np.linalg.svd(A1, compute_uv=False)
    sa = np.linalg.svd(Aa, compute_uv=False)
    assert abs(s1.max() / s1.min() - sa.max() / sa.min()) > 1e-3

    def alt(op):
        return lambda v: v - op.D_block(0, 1, op.Dinv_site(op.D_block(1, 0, op.Dinv_site(v))))
    assert np.abs(dense_eo(alt(st)) - dense_eo(alt(nf))).max() < 1e-13


def test_4d_solution_independent_of_alpha():
    """Sec. 2.3: the standard and Neff 5D equations give the same 4D solution."""
    dims = (4, 2, 2, 4)
    U = inputs.random_links(dims, 0.5, 91)
    b4 = inputs.gaussian_4d(dims, 92)
    ref = None
    for alpha in (1.0, 0.3, 0.5, 0.8):
        form = "standard" if alpha == 1.0 else "neff"
        op = dwf.DWF(U, dims, 6, 1.8, 0.04, 1.5, 0.5, form=form, alpha=alpha)
        x5, info = op.solve(op.source_5d(b4), tol=1e-13)
        x4 = op.project_4d(x5)
        if ref is None:
            ref = x4
        else:
            assert rel(x4, ref) < 1e-11


def test_cgnr_matches_dense_and_reaches_tolerance():
    dims = (2, 2, 2, 4)
    op = dwf.DWF(inputs.random_links(dims, 0.5, 101), dims, 4, 1.8, 0.04, 1.0, 0.0)
    b5 = inputs.gaussian_5d(dims, 4, 102)
    bt = op.b_tilde(b5)
    xe, info = dwf.cgnr(op.d_pc, lambda v: op.d_pc(v, dag=True), bt, tol=1e-13)
    assert info["true_residual"] < 1e-12
    n = bt.size
    M = np.zeros((n, n), dtype=complex)
    for j in range(n):
        e = np.zeros(n, dtype=complex)
        e[j] = 1
        M[:, j] = op.d_pc(e.reshape(bt.shape)).ravel()
    x_lu = np.linalg.solve(M, bt.ravel())
    assert rel(xe.ravel(), x_lu) < 1e-11


def test_free_field_5d_spectrum():
    """Unit links: the eigenvalues of the dense 5D matrix are the union over lattice
    momenta of those of the 4Ls x 4Ls momentum-space matrix (each 3 times, colour)."""
    dims = (2, 2, 2, 4)
    Ls = 3
    for form in ("standard", "neff"):
        op = dwf.DWF(inputs.unit_links(dims), dims, Ls, 1.8, 0.1, 1.5, 0.5, form=form, alpha=0.6)
        ev = np.linalg.eigvals(op.dense())
        want = []
        for n in np.ndindex(*dims):
            p = [(2 * np.pi * n[mu] + (np.pi if op.bc[mu] == -1 else 0.0)) / dims[mu] for mu in range(4)]
            Dp = (sum(1 - np.cos(q) for q in p) - op.M0) * np.eye(4) \
                + 1j * sum(dwf.GAMMA[mu] * np.sin(p[mu]) for mu in range(4))
            M = np.zeros((4 * Ls, 4 * Ls), dtype=complex)
            for bl in op.blocks():
                M[4 * bl.s:4 * bl.s + 4, 4 * bl.t:4 * bl.t + 4] += (bl.cw * Dp + bl.c1 * np.eye(4)) @ bl.S
            want += list(np.linalg.eigvals(M)) * 3
        want = np.array(want)
        dist = np.abs(ev[:, None] - want[None, :])
        assert dist.min(axis=1).max() < 1e-8 and dist.min(axis=0).max() < 1e-8
        assert abs(ev.sum() - want.sum()) < 1e-9 * len(ev)
        assert abs((ev ** 2).sum() - (want ** 2).sum()) < 1e-8 * len(ev)


# ------------------------------------------------------------------- smearing
def test_smearing_su3_covariance_identity():
    dims = (4, 2, 2, 4)
    U = inputs.random_links(dims, 0.5, 111)
    Us = inputs.smear_stout(U, 0.1, 2)
    I3 = np.eye(3)
    assert np.abs(np.swapaxes(Us.conj(), -1, -2) @ Us - I3).max() < 1e-13
    assert np.abs(np.linalg.det(Us) - 1).max() < 1e-13
    assert np.abs(inputs.smear_stout(U, 0.0, 3) - U).max() < 1e-13
    g = inputs.random_gauge_transform(dims, 112)
    Ug = gauge_transform(U, g)
    assert np.abs(inputs.smear_stout(Ug, 0.1, 2, reunit=False)
                  - gauge_transform(inputs.smear_stout(U, 0.1, 2, reunit=False), g)).max() < 1e-12
    # a smearing step raises the average plaquette of a rough field
    assert plaquette(Us) > plaquette(U)


def plaquette(U):
    tot = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            Ux = np.roll(U[nu], -1, axis=(3, 2, 1, 0)[mu])
            Uy = np.roll(U[mu], -1, axis=(3, 2, 1, 0)[nu])
            P = U[mu] @ Ux @ np.swapaxes(Uy.conj(), -1, -2) @ np.swapaxes(U[nu].conj(), -1, -2)
            tot += np.trace(P, axis1=-2, axis2=-1).real.mean() / 3
    return tot / 6


def test_links_are_su3():
    U = inputs.random_links((4, 4, 2, 2), 0.5, 1)
    assert np.abs(np.swapaxes(U.conj(), -1, -2) @ U - np.eye(3)).max() < 1e-13
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-13


def test_expi_hermitian_against_eigendecomposition():
    """The link generator's exp(i eps H) (scaling and squaring of a Taylor
    polynomial) against the closed form V diag(exp(i eps w)) V^dag from numpy's
    eigendecomposition."""
    g = np.random.default_rng(5)
    G = g.normal(size=(500, 3, 3)) + 1j * g.normal(size=(500, 3, 3))
    H = 0.5 * (G + np.swapaxes(G.conj(), -1, -2))
    w, v = np.linalg.eigh(H)
    for eps in (0.3, 0.5, 2.0):
        want = np.einsum("...ij,...j,...kj->...ik", v, np.exp(1j * eps * w), v.conj())
        assert np.abs(inputs._expi_hermitian(H, eps) - want).max() < 1e-13


@pytest.mark.parametrize("form,alpha,b,c", [("standard", 1.0, 1.5, 0.5), ("neff", 0.5, 1.5, 0.5),
                                            ("neff", 0.7, 1.0, 1.0)])
def test_row_apply_and_residual_match_apply(form, alpha, b, c):
    """apply_row (the large-lattice residual check) reproduces apply() row by row,
    and residual_norm equals the norm of b5 - apply(x5)."""
    dims, Ls = (4, 2, 2, 4), 6
    U = inputs.random_links(dims, 0.5, 131)
    ref = dwf.DWF(U, dims, Ls, 1.8, 0.03, b, c, form=form, alpha=alpha)
    x = inputs.gaussian_5d(dims, Ls, 132)
    y = ref.apply(x)
    for s in range(Ls):
        assert np.abs(ref.apply_row(x, s) - y[s]).max() < 1e-13
    bvec = inputs.gaussian_5d(dims, Ls, 133)
    want = np.linalg.norm((bvec - y).ravel()) / np.linalg.norm(bvec.ravel())
    assert abs(ref.residual_norm(bvec, x) - want) < 1e-14 * want
    # the source row by row, and the residual of a solve from a 4D source
    b4 = inputs.gaussian_4d(dims, 134)
    b5 = ref.source_5d(b4)
    for s in range(Ls):
        assert np.abs(ref.source_row(b4, s) - b5[s]).max() < 1e-14
    want = np.linalg.norm((b5 - y).ravel()) / np.linalg.norm(b5.ravel())
    assert abs(ref.residual_norm(lambda s: ref.source_row(b4, s), x) - want) < 1e-14 * want


# ---------------------------------------------------------------- 5D even-odd split
@pytest.mark.parametrize("b", [1.0, 1.5])
def test_eo5_route_solves_the_5d_system(b):
    """The 5D even-odd route (sites with x+y+z+t+s even; Sec. 2.3's alternative
    split) gives the same x5 as the dense solve of the printed matrix and as the
    4D route, and its Schur complement passes the adjoint identity."""
    dims, Ls = (2, 2, 2, 4), 4
    U = inputs.random_links(dims, 0.5, 71)
    d = dwf.DWF(U, dims, Ls, 1.8, 0.1, b, 0.0)
    assert d.eo5_available()
    b5 = inputs.gaussian_5d(dims, Ls, 72)
    x5, info = d.solve_eo5(b5, tol=1e-13)
    xd = np.linalg.solve(d.dense(), b5.reshape(-1)).reshape(b5.shape)
    assert np.linalg.norm(x5 - xd) / np.linalg.norm(xd) < 1e-10
    x4r, _ = d.solve(b5, tol=1e-13)
    assert np.linalg.norm(x5 - x4r) / np.linalg.norm(x4r) < 1e-10
    par = d.parity5()
    g = np.random.default_rng(73)
    xe = np.where(par == 0, inputs.gaussian_5d(dims, Ls, 74), 0)
    ye = np.where(par == 0, inputs.gaussian_5d(dims, Ls, 75), 0)
    lhs = np.vdot(ye, d.d_pc5(xe))
    rhs = np.vdot(d.d_pc5(ye, dag=True), xe)
    assert abs(lhs - rhs) / abs(lhs) < 1e-13
    assert not np.any(d.d_pc5(xe)[np.broadcast_to(par == 1, xe.shape)])   # stays on the even sites
    del g


def test_eo5_needs_diagonal_blocks():
    """c != 0 puts 4D hops into the fifth-direction couplings (D_ee is no longer
    on-site) and odd Ls puts the mass corner inside one parity: both refused."""
    dims = (2, 2, 2, 2)
    U = inputs.random_links(dims, 0.5, 76)
    for Ls, c, form in ((4, 0.5, "standard"), (5, 0.0, "standard"), (4, 0.0, "neff")):
        d = dwf.DWF(U, dims, Ls, 1.8, 0.1, 1.0, c, form=form, alpha=0.5)
        assert not d.eo5_available()
        with pytest.raises(ValueError):
            d.d_pc5(inputs.gaussian_5d(dims, Ls, 77))
