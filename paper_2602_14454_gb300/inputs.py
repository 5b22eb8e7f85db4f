"""Seeded synthetic inputs shared by the CUDA path, the tests and the benchmark.

This module only makes data: SU(3) link fields, link smearing (a set-up step
of Sec. 3.1, not part of the solver), Gaussian and point sources.  It holds
none of the solver's arithmetic (no Wilson or domain-wall operator, no even-odd
algebra, no Krylov method), so both the CUDA path and the FP64 oracle may take
their inputs from here.

Canonical layouts (complex128, C order, x fastest):
  links       U[mu][t][z][y][x][a][b]        mu = 0..3 for the x, y, z, t directions
  4D fermion  psi[t][z][y][x][spin][colour]
  5D fermion  psi[s][t][z][y][x][spin][colour]
``dims`` is always (Lx, Ly, Lz, Lt).
"""

from __future__ import annotations

import numpy as np

# axis of the (Lt, Lz, Ly, Lx) site array that moves along direction mu
_AXIS = (3, 2, 1, 0)


def rng(seed: int) -> np.random.Generator:
    """numpy PCG64 stream for one seed."""
    return np.random.Generator(np.random.PCG64(int(seed)))


def site_shape(dims) -> tuple:
    Lx, Ly, Lz, Lt = (int(d) for d in dims)
    return (Lt, Lz, Ly, Lx)


def _complex_normal(g: np.random.Generator, shape) -> np.ndarray:
    """i.i.d. complex normal entries with Re, Im ~ N(0, 1/2)."""
    s = np.sqrt(0.5)
    return g.normal(0.0, s, shape) + 1j * g.normal(0.0, s, shape)


def _expi_hermitian(H: np.ndarray, eps: float) -> np.ndarray:
    """exp(i*eps*H) for a batch of Hermitian 3x3 matrices (eigendecomposition)."""
    w, v = np.linalg.eigh(H)
    ph = np.exp(1j * eps * w)
    return np.einsum("...ij,...j,...kj->...ik", v, ph, v.conj())


def random_links(dims, eps: float, seed: int) -> np.ndarray:
    """U = exp(i*eps*H), H = (G+G^dag)/2 - tr(...)/3 with G complex normal.

    The result is unitary with det 1 (H traceless), i.e. in SU(3).
    """
    g = rng(seed)
    shp = (4,) + site_shape(dims) + (3, 3)
    G = _complex_normal(g, shp)
    H = 0.5 * (G + np.swapaxes(G.conj(), -1, -2))
    tr = np.trace(H, axis1=-2, axis2=-1)
    H = H - (tr / 3.0)[..., None, None] * np.eye(3)
    return np.ascontiguousarray(_expi_hermitian(H, eps))


def unit_links(dims) -> np.ndarray:
    shp = (4,) + site_shape(dims) + (3, 3)
    U = np.zeros(shp, dtype=np.complex128)
    U[...] = np.eye(3)
    return U


def _dag(A):
    return np.swapaxes(A.conj(), -1, -2)


def _shift(A, mu: int, k: int):
    """B(x) = A(x + k*mu_hat), periodic; A has site axes (Lt,Lz,Ly,Lx) first."""
    return np.roll(A, -k, axis=_AXIS[mu])


def reunitarise(U: np.ndarray) -> np.ndarray:
    """Nearest SU(3) matrix: polar factor (SVD) with the determinant phase removed."""
    u, _, vh = np.linalg.svd(U)
    W = u @ vh
    det = np.linalg.det(W)
    return W * (det ** (-1.0 / 3.0))[..., None, None]


def smear_stout(U: np.ndarray, rho: float, nsteps: int, reunit: bool = True) -> np.ndarray:
    """Stout projection of APE staples, eq. (stout_smearing) of Sec. 2.2, repeated.

    C_mu(x) = rho * sum_{nu != mu} [ U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag
                                     + U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) ]
    U'_mu(x) = exp([C_mu(x) U_mu(x)^dag]_AT) U_mu(x),
    [W]_AT = (W - W^dag)/2 - tr(W - W^dag)/6.
    All directions are updated together from the previous step's links.  The
    optional re-unitarisation only removes rounding drift.
    """
    U = np.array(U, dtype=np.complex128, copy=True)
    for _ in range(nsteps):
        Unew = np.empty_like(U)
        for mu in range(4):
            C = np.zeros_like(U[mu])
            for nu in range(4):
                if nu == mu:
                    continue
                up = U[nu] @ _shift(U[mu], nu, 1) @ _dag(_shift(U[nu], mu, 1))
                Unu_m = _shift(U[nu], nu, -1)
                dn = _dag(Unu_m) @ _shift(U[mu], nu, -1) @ _shift(_shift(U[nu], nu, -1), mu, 1)
                C += up + dn
            C *= rho
            W = C @ _dag(U[mu])
            A = 0.5 * (W - _dag(W))
            tr = np.trace(A, axis1=-2, axis2=-1)
            A = A - (tr / 3.0)[..., None, None] * np.eye(3)
            # A is anti-Hermitian and traceless: A = i*Hm with Hm Hermitian
            Hm = -1j * A
            Hm = 0.5 * (Hm + _dag(Hm))
            Unew[mu] = _expi_hermitian(Hm, 1.0) @ U[mu]
        U = reunitarise(Unew) if reunit else Unew
    return np.ascontiguousarray(U)


def smeared_links(dims, eps: float, rho: float, nsteps: int, seed: int) -> np.ndarray:
    """Random SU(3) links followed by ``nsteps`` stout/APE smearing steps."""
    return smear_stout(random_links(dims, eps, seed), rho, nsteps)


def random_gauge_transform(dims, seed: int) -> np.ndarray:
    """g(x) in SU(3) per site, shape (Lt,Lz,Ly,Lx,3,3)."""
    g = rng(seed)
    G = _complex_normal(g, site_shape(dims) + (3, 3))
    q, r = np.linalg.qr(G)
    d = np.diagonal(r, axis1=-2, axis2=-1)
    q = q * (d / np.abs(d))[..., None, :]
    det = np.linalg.det(q)
    return np.ascontiguousarray(q * (det ** (-1.0 / 3.0))[..., None, None])


def gaussian_4d(dims, seed: int) -> np.ndarray:
    return np.ascontiguousarray(_complex_normal(rng(seed), site_shape(dims) + (4, 3)))


def gaussian_5d(dims, Ls: int, seed: int) -> np.ndarray:
    return np.ascontiguousarray(_complex_normal(rng(seed), (Ls,) + site_shape(dims) + (4, 3)))


def point_source(dims, spin: int, colour: int, site=(0, 0, 0, 0)) -> np.ndarray:
    """delta_{x,site} delta_{spin} delta_{colour}; ``site`` is (x, y, z, t)."""
    b = np.zeros(site_shape(dims) + (4, 3), dtype=np.complex128)
    x, y, z, t = site
    b[t, z, y, x, spin, colour] = 1.0
    return b


# ---------------------------------------------------------------------------
# Named workloads.  Lattice shapes, parameters and seeds of the five
# configurations the library is measured on.
# ---------------------------------------------------------------------------

WORKLOADS = {
    # plain method, FP64: Shamir, unsmeared, eps 0.5
    "c1_4^4_ls8_shamir": dict(dims=(4, 4, 4, 4), Ls=8, M0=1.8, mf=0.04, b=1.0, c=0.0,
                              eps=0.5, smear=0, gauge_seed=1001, src_seed=2001, alpha=0.5),
    # 16^3x32 Mobius, 3 smearing steps
    "c2_16^3x32_ls16_mobius": dict(dims=(16, 16, 16, 32), Ls=16, M0=1.8, mf=0.01, b=1.5, c=0.5,
                                   eps=0.3, smear=3, gauge_seed=1002, src_seed=2002, alpha=0.5),
    # batched 24^3x48: 12 point sources x 3 masses x Ls in {8,12,16}
    "c3_24^3x48_batched": dict(dims=(24, 24, 24, 48), Ls_list=(8, 12, 16), M0=1.8,
                               mf_list=(0.005, 0.02, 0.05), b=1.5, c=0.5,
                               eps=0.3, smear=3, gauge_seed=1003, alpha=1.0),
    # learned preconditioner: 16^4, Neff form
    "c4_16^4_ls16_neff": dict(dims=(16, 16, 16, 16), Ls=16, M0=1.8, mf=0.01, b=1.5, c=0.5,
                              eps=0.3, smear=3, gauge_seed=1004, alpha=0.5,
                              train_seeds=range(4000, 4256), test_seeds=range(5000, 5016)),
    # large 32^3x64 Mobius
    "c5_32^3x64_ls16_mobius": dict(dims=(32, 32, 32, 64), Ls=16, M0=1.8, mf=0.005, b=1.5, c=0.5,
                                   eps=0.3, smear=3, gauge_seed=1005, src_seed=2005, alpha=0.5),
}


def workload_links(w: dict) -> np.ndarray:
    if w["smear"]:
        return smeared_links(w["dims"], w["eps"], 0.1, w["smear"], w["gauge_seed"])
    return random_links(w["dims"], w["eps"], w["gauge_seed"])
