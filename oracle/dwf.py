"""FP64 oracle of the domain-wall operators and of the solve (test infrastructure only).

Everything here follows Sec. 2 of the paper literally:
  * the domain-wall matrix, eq. (domainwall_general), applied block by block;
  * Neff's matrix, eq. (domainwall_neff), applied block by block;
  * the maps P and A of eq. (relation_to_alpha=1);
  * the 5D source b5 = (-D_-) P^dag (0,...,0,b4)^T and the 4D solution
    x4 = [P^dag x5]_{s=1} (Sec. 2.3, with eq. (4d_quark_field));
  * the even-odd Schur route, eq. (even-odd_linear_equation) and the two
    equations after it, built by masking the full operator;
  * CG on the normal equation (CGNR, Hestenes-Stiefel form), Sec. 2.3.
No shortcut of the CUDA path is used: no spin projection, no closed-form
fifth-direction inverse, no folding of the Neff factor into mixing matrices.

Readings where the paper is silent:
  * gamma basis: chiral, gamma_5 = diag(1,1,-1,-1) (wilson.c);
  * fermion boundary phases bc[mu], default periodic in x,y,z and
    antiperiodic in t;
  * rows 2..Ls-1 of the printed Neff matrix are all scaled by alpha (its text);
  * even sites: (x+y+z+t) even; 4D even-odd split as the paper chooses.

Array shapes: 4D field (Lt,Lz,Ly,Lx,4,3); 5D field (Ls,Lt,Lz,Ly,Lx,4,3);
even-odd half field (Ls,Vh,4,3) with the sites of one parity in
lexicographic order.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import _clib

# ---------------------------------------------------------------------------
# spin algebra (Sec. 2.1): chiral basis, built from the Pauli matrices
# ---------------------------------------------------------------------------
_S1 = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_S2 = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_S3 = np.array([[1, 0], [0, -1]], dtype=np.complex128)
_Z2 = np.zeros((2, 2), dtype=np.complex128)
_I2 = np.eye(2, dtype=np.complex128)


def gammas():
    """gamma_1..gamma_4 (chiral basis) as a (4,4,4) array."""
    g = [np.block([[_Z2, -1j * s], [1j * s, _Z2]]) for s in (_S1, _S2, _S3)]
    g.append(np.block([[_Z2, _I2], [_I2, _Z2]]))
    return np.array(g)


GAMMA = gammas()
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
ONE4 = np.eye(4, dtype=np.complex128)
P_PLUS = 0.5 * (ONE4 + GAMMA5)
P_MINUS = 0.5 * (ONE4 - GAMMA5)


def spin(S: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Apply a 4x4 spin matrix to the spin index (second-last axis)."""
    return np.einsum("ij,...jc->...ic", S, v)


def inner(a: np.ndarray, b: np.ndarray) -> complex:
    return complex(np.vdot(a.ravel(), b.ravel()))


def norm(a: np.ndarray) -> float:
    return float(np.linalg.norm(a.ravel()))


@dataclass
class Block:
    """One nonzero block (row s, column t) = (cw * D_W + c1) * S, S a spin matrix."""
    s: int
    t: int
    cw: float
    c1: float
    S: np.ndarray


@dataclass
class DWF:
    """Domain-wall fermion operator on one gauge field.

    form = "standard": eq. (domainwall_general); b and c are numbers, or
                       sequences of Ls numbers b_i, c_i (row i of the matrix
                       holds D_+^(i) = b_i D_W + 1 and D_-^(i) = c_i D_W - 1).
    form = "neff":     eq. (domainwall_neff) with parameter alpha (constant b, c:
                       the form is printed for coefficients independent of i).
    """
    U: np.ndarray
    dims: tuple
    Ls: int
    M0: float
    mf: float
    b: float
    c: float
    form: str = "standard"
    alpha: float = 1.0
    bc: tuple = (1, 1, 1, -1)
    _blocks: list = field(default=None, repr=False)

    def __post_init__(self):
        self.dims = tuple(int(d) for d in self.dims)
        self.U = np.ascontiguousarray(self.U, dtype=np.complex128)
        if self.form not in ("standard", "neff"):
            raise ValueError(self.form)
        # per-row coefficients b_i, c_i (Sec. 2.2)
        self._bs = np.broadcast_to(np.asarray(self.b, dtype=np.float64), (self.Ls,)).copy()
        self._cs = np.broadcast_to(np.asarray(self.c, dtype=np.float64), (self.Ls,)).copy()
        if self.form == "neff" and (np.ptp(self._bs) != 0 or np.ptp(self._cs) != 0):
            raise ValueError("the Neff form takes coefficients independent of s")
        self._blocks = self.blocks()
        self._eo = None

    # --------------------------------------------------------------- 4D part
    def dw(self, v: np.ndarray, dag: bool = False) -> np.ndarray:
        """D_W(-M0) of eq. (Wilson_matrix), or its adjoint, on stacked 4D fields."""
        return _clib.wilson(self.U, self.dims, self.bc, self.M0, v, dag)

    @property
    def site_shape(self):
        Lx, Ly, Lz, Lt = self.dims
        return (Lt, Lz, Ly, Lx)

    # ----------------------------------------------------- 5D block matrices
    def blocks(self):
        """Nonzero blocks of the printed 5D matrix, 0-based s, t.

        D_+ = b D_W + 1, D_- = c D_W - 1 (Sec. 2.2); row s takes b_s, c_s.
        standard, eq. (domainwall_general):
          (s,s)     D_+            (s,s+1) D_- P_-        (s,s-1) D_- P_+
          (1,Ls)   -m D_- P_+      (Ls,1)  -m D_- P_-
        Neff, eq. (domainwall_neff): the same blocks times alpha, except the
        corners: (1,1) = D_+ (P_- + alpha P_+), (Ls,Ls) = D_+ (P_+ + alpha P_-),
        (1,Ls) and (Ls,1) unchanged.
        Blocks that land on the same position (Ls = 2) are summed.
        """
        Ls, m = self.Ls, self.mf
        a = self.alpha if self.form == "neff" else 1.0
        out = []
        for s in range(Ls):
            b, c = float(self._bs[s]), float(self._cs[s])
            if self.form == "neff" and s == 0:
                out.append(Block(s, s, b, 1.0, P_MINUS + a * P_PLUS))
            elif self.form == "neff" and s == Ls - 1:
                out.append(Block(s, s, b, 1.0, P_PLUS + a * P_MINUS))
            else:
                out.append(Block(s, s, a * b, a * 1.0, ONE4))
            if s + 1 < Ls:
                out.append(Block(s, s + 1, a * c, -a * 1.0, P_MINUS))
            if s - 1 >= 0:
                out.append(Block(s, s - 1, a * c, -a * 1.0, P_PLUS))
        out.append(Block(0, Ls - 1, -m * float(self._cs[0]), m, P_PLUS))
        out.append(Block(Ls - 1, 0, -m * float(self._cs[Ls - 1]), m, P_MINUS))
        return out

    def apply(self, x5: np.ndarray, dag: bool = False) -> np.ndarray:
        """y = D x (row by row over the blocks) or y = D^dag x.

        Adjoint: block (t,s) of D^dag is [(cw D_W + c1) S]^dag = S^dag (cw D_W^dag + c1).
        """
        assert x5.shape[0] == self.Ls
        y = np.zeros_like(x5, dtype=np.complex128)
        if not dag:
            proj = np.stack([spin(bl.S, x5[bl.t]) for bl in self._blocks])
            wproj = self.dw(proj)
            for k, bl in enumerate(self._blocks):
                y[bl.s] += bl.cw * wproj[k] + bl.c1 * proj[k]
        else:
            wx = self.dw(x5, dag=True)
            for bl in self._blocks:
                y[bl.t] += spin(bl.S.conj().T, bl.cw * wx[bl.s] + bl.c1 * x5[bl.s])
        return y

    def apply_row(self, x5: np.ndarray, s: int) -> np.ndarray:
        """Row s of y = D x: sum over the blocks (s, t) of (cw D_W + c1) S x[t].

        The same block formula as apply(), one row at a time, for lattices whose
        stacked block fields do not fit in memory: D_W is linear, so the blocks
        of a row are summed before it is applied (one D_W per row).
        """
        inner = np.zeros_like(x5[0], dtype=np.complex128)
        local = np.zeros_like(x5[0], dtype=np.complex128)
        for bl in self._blocks:
            if bl.s != s:
                continue
            sx = spin(bl.S, x5[bl.t])
            inner += bl.cw * sx
            local += bl.c1 * sx
        return self.dw(inner) + local

    def residual_norm(self, b5, x5: np.ndarray) -> float:
        """||b5 - D x5|| / ||b5||, accumulated row by row (apply_row); b5 is a
        5D array or a function of s giving row s."""
        row = b5.__getitem__ if isinstance(b5, np.ndarray) else b5
        num = den = 0.0
        for s in range(self.Ls):
            bs = row(s)
            r = (bs - self.apply_row(x5, s)).ravel()
            num += float(np.vdot(r, r).real)
            den += float(np.vdot(bs.ravel(), bs.ravel()).real)
        return float(np.sqrt(num / den))

    def dense(self) -> np.ndarray:
        """Dense matrix of the full 5D operator (tiny lattices only)."""
        n = self.Ls * int(np.prod(self.dims)) * 12
        shp = (self.Ls,) + self.site_shape + (4, 3)
        M = np.zeros((n, n), dtype=np.complex128)
        e = np.zeros(n, dtype=np.complex128)
        for j in range(n):
            e[:] = 0
            e[j] = 1
            M[:, j] = self.apply(e.reshape(shp)).ravel()
        return M

    # --------------------------------------- P and A, eq. (relation_to_alpha=1)
    def _p_blocks(self):
        """Blocks of P: row s has P_- at column s and P_+ at column s+1;
        the last row has P_+ at column 1 and P_- at column Ls."""
        Ls = self.Ls
        out = []
        for s in range(Ls - 1):
            out += [(s, s, P_MINUS), (s, s + 1, P_PLUS)]
        out += [(Ls - 1, 0, P_PLUS), (Ls - 1, Ls - 1, P_MINUS)]
        return out

    def P(self, x5, dag=False):
        y = np.zeros_like(x5, dtype=np.complex128)
        for (s, t, S) in self._p_blocks():
            if not dag:
                y[s] += spin(S, x5[t])
            else:
                y[t] += spin(S.conj().T, x5[s])
        return y

    def A(self, x5, inverse=False):
        """A = diag(1, alpha, ..., alpha) in the fifth direction."""
        a = self.alpha
        y = np.array(x5, dtype=np.complex128, copy=True)
        y[1:] *= (1.0 / a) if inverse else a
        return y

    # ------------------------------------------------- 4D source / 4D solution
    def d_minus(self, x5, dag=False):
        """D_- = diag_s(c_s D_W - 1)."""
        cs = self._cs.reshape((self.Ls,) + (1,) * (x5.ndim - 1))
        return cs * self.dw(x5, dag=dag) - x5

    def source_5d(self, b4: np.ndarray) -> np.ndarray:
        """b5 = (-D_-) P^dag (0, ..., 0, b4)^T (Sec. 2.3)."""
        v = np.zeros((self.Ls,) + b4.shape, dtype=np.complex128)
        v[self.Ls - 1] = b4
        return -self.d_minus(self.P(v, dag=True))

    def source_row(self, b4: np.ndarray, s: int) -> np.ndarray:
        """Row s of source_5d(b4), from the rows of P^dag that (0, ..., 0, b4)
        reaches: [P^dag v]_s = sum over the blocks (Ls-1, s) of P of S^dag b4,
        then -D_- of that row (c_s D_W - 1 for row s)."""
        Ls = self.Ls
        v = np.zeros_like(b4, dtype=np.complex128)
        for (r, t, S) in self._p_blocks():
            if r == Ls - 1 and t == s:
                v += spin(S.conj().T, b4)
        if not np.any(v):
            return v
        return -(float(self._cs[s]) * self.dw(v) - v)

    def project_4d(self, x5: np.ndarray) -> np.ndarray:
        """x4 = [P^dag x5]_{s=1} (Sec. 2.3)."""
        return self.P(x5, dag=True)[0]

    # ---------------------------------------------------------- even-odd split
    def _eo_setup(self):
        if self._eo is not None:
            return self._eo
        Lx, Ly, Lz, Lt = self.dims
        t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx),
                                 indexing="ij")
        par = ((x + y + z + t) % 2).ravel()
        even = np.nonzero(par == 0)[0]
        odd = np.nonzero(par == 1)[0]
        L = self.site_matrix()
        Linv = np.linalg.inv(L)
        self._eo = dict(even=even, odd=odd, L=L, Linv=Linv)
        return self._eo

    def site_matrix(self) -> np.ndarray:
        """Site-local block D_ee = D_oo as a (4Ls x 4Ls) matrix over (s, spin).

        The diagonal of D_W(-M0) is (4 - M0) times the identity (eq. (Wilson_matrix)),
        so each block (cw D_W + c1) S contributes (cw (4-M0) + c1) S on the diagonal
        of the 4D lattice; the colour index is untouched.
        """
        Ls = self.Ls
        L = np.zeros((4 * Ls, 4 * Ls), dtype=np.complex128)
        for bl in self._blocks:
            L[4 * bl.s:4 * bl.s + 4, 4 * bl.t:4 * bl.t + 4] += (bl.cw * (4.0 - self.M0) + bl.c1) * bl.S
        return L

    def to_eo(self, x5, parity):
        eo = self._eo_setup()
        idx = eo["even"] if parity == 0 else eo["odd"]
        flat = x5.reshape((self.Ls, -1, 4, 3))
        return np.ascontiguousarray(flat[:, idx])

    def from_eo(self, xe=None, xo=None):
        eo = self._eo_setup()
        V = int(np.prod(self.dims))
        ref = xe if xe is not None else xo
        out = np.zeros((self.Ls, V, 4, 3), dtype=np.complex128)
        if xe is not None:
            out[:, eo["even"]] = xe
        if xo is not None:
            out[:, eo["odd"]] = xo
        return out.reshape((self.Ls,) + self.site_shape + (4, 3))

    def site_apply(self, Mat, v):
        """Apply a (4Ls x 4Ls) site-local matrix to a half field (Ls,Vh,4,3)."""
        Ls = self.Ls
        w = v.transpose(0, 2, 1, 3).reshape(4 * Ls, -1, 3)
        r = np.einsum("ij,jka->ika", Mat, w)
        return np.ascontiguousarray(r.reshape(Ls, 4, -1, 3).transpose(0, 2, 1, 3))

    def D_block(self, out_par, in_par, v, dag=False):
        """D_{out,in} v by masking the full operator (or (D^dag)_{out,in} v)."""
        full = self.from_eo(xe=v) if in_par == 0 else self.from_eo(xo=v)
        return self.to_eo(self.apply(full, dag=dag), out_par)

    def Dinv_site(self, v, dag=False):
        eo = self._eo_setup()
        Mat = eo["Linv"].conj().T if dag else eo["Linv"]
        return self.site_apply(Mat, v)

    def d_pc(self, xe, dag=False):
        """D x_e = (1 - D_ee^-1 D_eo D_oo^-1 D_oe) x_e, eq. (even-odd_linear_equation);
        dag: D^dag x_e = x_e - D_oe^dag D_oo^-dag D_eo^dag D_ee^-dag x_e."""
        if not dag:
            t = self.Dinv_site(self.D_block(1, 0, xe))
            return xe - self.Dinv_site(self.D_block(0, 1, t))
        t = self.D_block(1, 0, self.Dinv_site(xe, dag=True), dag=True)
        return xe - self.D_block(0, 1, self.Dinv_site(t, dag=True), dag=True)

    def b_tilde(self, b5):
        """b~_e = D_ee^-1 (b_e - D_eo D_oo^-1 b_o)."""
        be, bo = self.to_eo(b5, 0), self.to_eo(b5, 1)
        return self.Dinv_site(be - self.D_block(0, 1, self.Dinv_site(bo)))

    def x_odd(self, b5, xe):
        """x_o = D_oo^-1 (b_o - D_oe x_e)."""
        bo = self.to_eo(b5, 1)
        return self.Dinv_site(bo - self.D_block(1, 0, xe))

    # ------------------------------------------- 5D even-odd preconditioning
    # The alternative split of Sec. 2.3: sites (x, s) even when x+y+z+t+s is
    # even.  D_ee and D_oo are then the on-site diagonal a0_s = b_s (4 - M0) + 1
    # only when c_s = 0 (no 4D hop in the fifth-direction couplings) and Ls is
    # even (the mass corners join s = 1 and s = Ls, of opposite parity), in the
    # standard form; the Schur route is then the same as in 4D:
    #   D5 x_e = x_e - D_ee^-1 D_eo D_oo^-1 D_oe x_e = b'_e,
    #   b'_e = D_ee^-1 (b_e - D_eo D_oo^-1 b_o),  x_o = D_oo^-1 (b_o - D_oe x_e).
    # Fields stay full 5D arrays; the sites of the other parity are zero.
    def eo5_available(self):
        return self.form == "standard" and bool(np.all(self._cs == 0)) and self.Ls % 2 == 0

    def parity5(self):
        """(x+y+z+t+s) mod 2 for every 5D site, shape (Ls,)+site_shape+(1, 1)."""
        Lt, Lz, Ly, Lx = self.site_shape
        s, t, z, y, x = np.meshgrid(np.arange(self.Ls), np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx),
                                    indexing="ij")
        return ((s + t + z + y + x) % 2)[..., None, None]

    def _a0(self):
        return (self._bs * (4.0 - self.M0) + 1.0).reshape((self.Ls,) + (1,) * 6)

    def d_pc5(self, x5, dag=False):
        """(1 - D_ee^-1 D_eo D_oo^-1 D_oe) x_e of the 5D split, or its adjoint
        (1 - D_oe^dag D_oo^-1 D_eo^dag D_ee^-1) x_e; x5's odd sites are ignored."""
        if not self.eo5_available():
            raise ValueError("5D even-odd preconditioning needs the standard form, c = 0 and even Ls")
        par = self.parity5()
        ev, od = (par == 0), (par == 1)
        a0 = self._a0()
        x = np.where(ev, x5, 0)
        if not dag:
            t = np.where(od, self.apply(x), 0) / a0           # D_oo^-1 D_oe x
            return x - np.where(ev, self.apply(t), 0) / a0    # x - D_ee^-1 D_eo t
        u = x / a0                                            # D_ee^-1 x
        t = np.where(od, self.apply(u, dag=True), 0) / a0     # D_oo^-1 D_eo^dag u
        return x - np.where(ev, self.apply(t, dag=True), 0)   # x - D_oe^dag t

    def solve_eo5(self, b5, tol=1e-12, maxiter=20000):
        """x5 = D^-1 b5 through the 5D even-odd route and CGNR on its Schur complement."""
        par = self.parity5()
        ev, od = (par == 0), (par == 1)
        a0 = self._a0()
        be, bo = np.where(ev, b5, 0), np.where(od, b5, 0)
        bp = (be - np.where(ev, self.apply(bo / a0), 0)) / a0
        xe, info = cgnr(lambda v: self.d_pc5(v), lambda v: self.d_pc5(v, dag=True), bp, tol=tol, maxiter=maxiter)
        xo = (bo - np.where(od, self.apply(xe), 0)) / a0
        return np.where(ev, xe, 0) + xo, info

    # ------------------------------------------------------------------ solve
    def solve(self, b5, tol=1e-12, maxiter=20000, x0=None):
        """x5 = D^-1 b5 through the even-odd route and CGNR on D x_e = b~_e."""
        bt = self.b_tilde(b5)
        xe, info = cgnr(lambda v: self.d_pc(v), lambda v: self.d_pc(v, dag=True), bt,
                        tol=tol, maxiter=maxiter, x0=x0)
        xo = self.x_odd(b5, xe)
        return self.from_eo(xe, xo), info


def cgnr(A, Adag, b, tol=1e-12, maxiter=20000, x0=None):
    """Conjugate gradient on A^dag A x = A^dag b (Hestenes-Stiefel CGNR), FP64.

    Stops when ||b - A x|| <= tol ||b|| (the true residual of A x = b, tracked
    by the recursion and recomputed at the end).
    """
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128, copy=True)
    r = b - A(x)
    z = Adag(r)
    p = z.copy()
    gamma = inner(z, z).real
    bn = norm(b)
    hist = [norm(r) / bn]
    it = 0
    while hist[-1] > tol and it < maxiter:
        w = A(p)
        alpha = gamma / inner(w, w).real
        x += alpha * p
        r -= alpha * w
        z = Adag(r)
        gnew = inner(z, z).real
        p = z + (gnew / gamma) * p
        gamma = gnew
        it += 1
        hist.append(norm(r) / bn)
    true_res = norm(b - A(x)) / bn
    return x, dict(iterations=it, history=hist, true_residual=true_res)


def random_su3(g: np.random.Generator, shape) -> np.ndarray:
    """Helper for tests: Haar-like SU(3) matrices (QR of complex normal)."""
    G = g.normal(size=shape + (3, 3)) + 1j * g.normal(size=shape + (3, 3))
    q, r = np.linalg.qr(G)
    d = np.diagonal(r, axis1=-2, axis2=-1)
    q = q * (d / np.abs(d))[..., None, :]
    det = np.linalg.det(q)
    return q * (det ** (-1.0 / 3.0))[..., None, None]
