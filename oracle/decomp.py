"""Domain-decomposed FP64 oracle of the even-odd domain-wall operator and its
CG solve, on CPU ranks of a torch.distributed process group (gloo).

TEST INFRASTRUCTURE ONLY: it emulates, on host processes, the 4D domain
decomposition of one solve over several GPUs -- the lattice cut into slabs of
the time direction, one slab per rank -- and is compared in the tests with the
unsplit oracle (oracle/dwf.py).  Nothing in the library imports it.

What it computes is the operator of oracle/dwf.py, split:
  * every rank owns the sites with t in [t0, t0 + Tl) (Tl even, so the parity
    (x+y+z+t) of a site is the same in local and global coordinates) and the
    links U_mu(x) of those sites;
  * D_W of eq. (Wilson_matrix) needs, at the slab's last slice, the forward
    neighbour psi(x+t) of the next rank and, at its first slice, the backward
    term U_t(x-t)^dag psi(x-t) of the previous rank.  The projector
    (1 -+ gamma_t) has rank 2, so each rank sends only the two-spin half spinor
    h = E^dag (1 -+ gamma_t) v (E an orthonormal basis of the projector's
    range): 6 complex numbers per site and fifth-dimension slice; the
    receiver rebuilds (1 -+ gamma_t) v = E h.  The sender applies U_t^dag to
    its own last slice before projecting (it owns those links); the boundary
    phase bc[t] is applied where the global boundary is crossed;
  * the domain-wall blocks, the site-local D_ee, D_oo and the even-odd Schur
    form are those of oracle/dwf.py (no communication);
  * CG on the normal equation (Hestenes-Stiefel CGNR, as oracle.dwf.cgnr) with
    every inner product summed over the ranks by one all-reduce.
"""

from __future__ import annotations

import numpy as np

from . import dwf as orc


def _range_basis(Pm: np.ndarray) -> np.ndarray:
    """Orthonormal basis (4 x 2) of the range of a rank-2 spin matrix."""
    u, sv, _ = np.linalg.svd(Pm)
    assert sv[2] < 1e-12 and sv[1] > 1e-12
    return u[:, :2]


class SplitDWF:
    """The domain-wall operator of one form on this rank's time slab."""

    def __init__(self, U_global, dims, Ls, M0, mf, b, c, form="standard", alpha=1.0, bc=(1, 1, 1, -1),
                 group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.size = dist.get_world_size(group)
        Lx, Ly, Lz, Lt = (int(d) for d in dims)
        if Lt % self.size or (Lt // self.size) % 2:
            raise ValueError("Lt must split into slabs of even length")
        self.dims = (Lx, Ly, Lz, Lt)
        self.Tl = Lt // self.size
        self.t0 = self.rank * self.Tl
        self.Ls, self.M0, self.bc = Ls, M0, tuple(bc)
        # the full-lattice operator defines the blocks and the site matrix (no lattice sum)
        self.full = orc.DWF(U_global, dims, Ls, M0, mf, b, c, form=form, alpha=alpha, bc=bc)
        self.U = np.ascontiguousarray(U_global[:, self.t0:self.t0 + self.Tl])
        g = orc.GAMMA
        self.Sm = [orc.ONE4 - g[m] for m in range(4)]   # (1 - gamma_mu)
        self.Sp = [orc.ONE4 + g[m] for m in range(4)]   # (1 + gamma_mu)
        self.Em = _range_basis(self.Sm[3])
        self.Ep = _range_basis(self.Sp[3])
        t, z, y, x = np.meshgrid(np.arange(self.t0, self.t0 + self.Tl), np.arange(Lz), np.arange(Ly),
                                 np.arange(Lx), indexing="ij")
        par = ((x + y + z + t) % 2).ravel()
        self.even = np.nonzero(par == 0)[0]
        self.odd = np.nonzero(par == 1)[0]
        self.Linv = np.linalg.inv(self.full.site_matrix())
        self.halo_bytes = 0

    # ------------------------------------------------------------ exchange
    def _sendrecv(self, send: np.ndarray, to: int, frm: int) -> np.ndarray:
        import torch
        sbuf = torch.from_numpy(np.ascontiguousarray(send).view(np.float64).copy())
        rbuf = torch.empty_like(sbuf)
        reqs = [self.dist.isend(sbuf, to, group=self.group), self.dist.irecv(rbuf, frm, group=self.group)]
        for r in reqs:
            r.wait()
        self.halo_bytes += sbuf.numel() * 8
        return rbuf.numpy().view(np.complex128).reshape(send.shape)

    def _halos(self, v: np.ndarray, sgn: int):
        """(forward, backward) terms of the slab's boundary slices, received from
        the neighbouring ranks: (1 - s gamma_t) v(x + t) at the last slice and
        (1 + s gamma_t) U_t(x - t)^dag v(x - t) at the first (s = sgn; -1 for
        the adjoint), as full spinors rebuilt from the half spinors."""
        nxt, prv = (self.rank + 1) % self.size, (self.rank - 1) % self.size
        Sm = orc.ONE4 - sgn * orc.GAMMA[3]
        Sp = orc.ONE4 + sgn * orc.GAMMA[3]
        Em = self.Em if sgn > 0 else self.Ep
        Ep = self.Ep if sgn > 0 else self.Em
        # to the previous rank: my first slice, projected
        first = orc.spin(Em.conj().T @ Sm, v[:, 0])
        h_fwd = self._sendrecv(first, prv, nxt)
        fwd = orc.spin(Em, h_fwd)
        # to the next rank: U_t^dag v at my last slice, projected
        Ul = self.U[3, self.Tl - 1]
        Uv = np.einsum("...ba,...sb->...sa", Ul.conj(), v[:, self.Tl - 1])
        last = orc.spin(Ep.conj().T @ Sp, Uv)
        h_bwd = self._sendrecv(last, nxt, prv)
        bwd = orc.spin(Ep, h_bwd)
        # the global time boundary
        if self.rank == self.size - 1:
            fwd = fwd * self.bc[3]
        if self.rank == 0:
            bwd = bwd * self.bc[3]
        return fwd, bwd

    # ------------------------------------------------------------- operator
    def dw(self, v: np.ndarray, dag: bool = False) -> np.ndarray:
        """D_W(-M0) (or its adjoint) on a stack of slab fields (nf, Tl, Lz, Ly, Lx, 4, 3):
        the adjoint is the same sum with gamma_mu -> -gamma_mu (gamma_mu Hermitian)."""
        sgn = -1 if dag else 1
        out = (4.0 - self.M0) * v
        axis = {0: 4, 1: 3, 2: 2}           # mu -> axis of the stacked array (x, y, z)
        for mu in range(3):
            ax = axis[mu]
            U = self.U[mu]
            Sm = orc.ONE4 - sgn * orc.GAMMA[mu]
            Sp = orc.ONE4 + sgn * orc.GAMMA[mu]
            L = v.shape[ax]
            # forward: U_mu(x) v(x + mu), phase across the boundary
            vf = np.roll(v, -1, axis=ax)
            if self.bc[mu] != 1:
                idx = [slice(None)] * v.ndim
                idx[ax] = L - 1
                vf[tuple(idx)] *= self.bc[mu]
            Uvf = np.einsum("...ab,n...sb->n...sa", U, vf)
            out = out - 0.5 * orc.spin(Sm, Uvf)
            # backward: U_mu(x - mu)^dag v(x - mu)
            Ub = np.roll(U, 1, axis=ax - 1)
            vb = np.roll(v, 1, axis=ax)
            if self.bc[mu] != 1:
                idx = [slice(None)] * v.ndim
                idx[ax] = 0
                vb[tuple(idx)] *= self.bc[mu]
            Uvb = np.einsum("...ba,n...sb->n...sa", Ub.conj(), vb)
            out = out - 0.5 * orc.spin(Sp, Uvb)
        # time direction: inside the slab, then the halos at its two faces
        Ut = self.U[3]
        Sm = orc.ONE4 - sgn * orc.GAMMA[3]
        Sp = orc.ONE4 + sgn * orc.GAMMA[3]
        fwd, bwd = self._halos(v, sgn)
        tf = np.zeros_like(v)
        tf[:, :-1] = orc.spin(Sm, np.einsum("...ab,n...sb->n...sa", Ut[:-1], v[:, 1:]))
        tf[:, -1] = np.einsum("...ab,n...sb->n...sa", Ut[-1], fwd)
        tb = np.zeros_like(v)
        tb[:, 1:] = orc.spin(Sp, np.einsum("...ba,n...sb->n...sa", Ut[:-1].conj(), v[:, :-1]))
        tb[:, 0] = bwd
        return out - 0.5 * (tf + tb)

    def apply(self, x5: np.ndarray, dag: bool = False) -> np.ndarray:
        """The 5D matrix on this slab, block by block as oracle.dwf.DWF.apply."""
        y = np.zeros_like(x5, dtype=np.complex128)
        blocks = self.full._blocks
        if not dag:
            proj = np.stack([orc.spin(bl.S, x5[bl.t]) for bl in blocks])
            wproj = self.dw(proj)
            for k, bl in enumerate(blocks):
                y[bl.s] += bl.cw * wproj[k] + bl.c1 * proj[k]
        else:
            wx = self.dw(x5, dag=True)
            for bl in blocks:
                y[bl.t] += orc.spin(bl.S.conj().T, bl.cw * wx[bl.s] + bl.c1 * x5[bl.s])
        return y

    # ------------------------------------------------------------ even-odd
    @property
    def slab_shape(self):
        Lx, Ly, Lz, _ = self.dims
        return (self.Tl, Lz, Ly, Lx)

    def to_eo(self, x5_slab, parity):
        idx = self.even if parity == 0 else self.odd
        return np.ascontiguousarray(x5_slab.reshape((self.Ls, -1, 4, 3))[:, idx])

    def from_eo(self, xe=None, xo=None):
        out = np.zeros((self.Ls, int(np.prod(self.slab_shape)), 4, 3), dtype=np.complex128)
        if xe is not None:
            out[:, self.even] = xe
        if xo is not None:
            out[:, self.odd] = xo
        return out.reshape((self.Ls,) + self.slab_shape + (4, 3))

    def D_block(self, out_par, in_par, v, dag=False):
        full = self.from_eo(xe=v) if in_par == 0 else self.from_eo(xo=v)
        return self.to_eo(self.apply(full, dag=dag), out_par)

    def Dinv_site(self, v, dag=False):
        Mat = self.Linv.conj().T if dag else self.Linv
        return self.full.site_apply(Mat, v)

    def d_pc(self, xe, dag=False):
        """eq. (even-odd_linear_equation) on this rank's even sites, or its adjoint."""
        if not dag:
            t = self.Dinv_site(self.D_block(1, 0, xe))
            return xe - self.Dinv_site(self.D_block(0, 1, t))
        t = self.D_block(1, 0, self.Dinv_site(xe, dag=True), dag=True)
        return xe - self.D_block(0, 1, self.Dinv_site(t, dag=True), dag=True)

    # ----------------------------------------------------------------- CG
    def inner(self, a, b) -> complex:
        import torch
        loc = np.vdot(a.ravel(), b.ravel())
        t = torch.tensor([loc.real, loc.imag], dtype=torch.float64)
        self.dist.all_reduce(t, group=self.group)
        return complex(t[0].item(), t[1].item())

    def norm(self, a) -> float:
        return float(np.sqrt(self.inner(a, a).real))

    def cgnr(self, b, tol=1e-12, maxiter=20000):
        """CGNR on D_pc x = b over the ranks (each holds its slab's even sites)."""
        x = np.zeros_like(b)
        r = b.copy()
        z = self.d_pc(r, dag=True)
        p = z.copy()
        gamma = self.inner(z, z).real
        bn = self.norm(b)
        res = 1.0
        it = 0
        while res > tol and it < maxiter:
            w = self.d_pc(p)
            alpha = gamma / self.inner(w, w).real
            x += alpha * p
            r -= alpha * w
            z = self.d_pc(r, dag=True)
            gnew = self.inner(z, z).real
            p = z + (gnew / gamma) * p
            gamma = gnew
            it += 1
            res = self.norm(r) / bn
        true_res = self.norm(b - self.d_pc(x)) / bn
        return x, dict(iterations=it, true_residual=true_res)
