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


# The link algebra below runs on torch tensors, on the CPU or (device="cuda")
# on a GPU, so that the 32^3x64 fields are made in seconds; every function
# returns numpy arrays.  The random numbers always come from numpy's PCG64
# stream on the host, so a seed names the same field on every device (up to
# the rounding of the device's arithmetic).
def _torch():
    import torch
    return torch


def _dev(device):
    return "cpu" if device is None else device


def _tdag(A):
    return A.conj().transpose(-1, -2)


def _texpm(A):
    """exp(A) for a batch of 3x3 complex matrices: scaling and squaring with a
    Taylor polynomial of degree 16 (|A| / 2^k <= 1/2 for every matrix, so the
    truncation error is below 1e-18 relative)."""
    torch = _torch()
    nrm = float(torch.linalg.matrix_norm(A, ord="fro").max()) if A.numel() else 0.0
    k = 0
    while nrm / (1 << k) > 0.5:
        k += 1
    X = A / float(1 << k)
    eye = torch.eye(3, dtype=A.dtype, device=A.device)
    E = eye.expand_as(X).clone()
    T = eye.expand_as(X).clone()
    for n in range(1, 17):
        T = (T @ X) / float(n)
        E = E + T
    for _ in range(k):
        E = E @ E
    return E


def _tdet(W):
    return (W[..., 0, 0] * (W[..., 1, 1] * W[..., 2, 2] - W[..., 1, 2] * W[..., 2, 1])
            - W[..., 0, 1] * (W[..., 1, 0] * W[..., 2, 2] - W[..., 1, 2] * W[..., 2, 0])
            + W[..., 0, 2] * (W[..., 1, 0] * W[..., 2, 1] - W[..., 1, 1] * W[..., 2, 0]))


def _treunitarise(U):
    """Nearest SU(3) matrix of an almost unitary U: its polar factor by two
    Newton-Schulz steps X <- X (3 - X^dag X) / 2 (quadratic convergence from
    |1 - U^dag U| << 1), then the determinant phase removed."""
    torch = _torch()
    eye = torch.eye(3, dtype=U.dtype, device=U.device)
    X = U
    for _ in range(2):
        X = X @ (3.0 * eye - _tdag(X) @ X) * 0.5
    det = _tdet(X)
    return X * (det ** (-1.0 / 3.0))[..., None, None]


def _expi_hermitian(H: np.ndarray, eps: float, device=None) -> np.ndarray:
    """exp(i*eps*H) for a batch of Hermitian 3x3 matrices."""
    torch = _torch()
    Ht = torch.from_numpy(np.ascontiguousarray(H, dtype=np.complex128)).to(_dev(device))
    return _texpm(1j * eps * Ht).cpu().numpy()


def _random_links_t(dims, eps: float, seed: int, device):
    torch = _torch()
    g = rng(seed)
    shp = (4,) + site_shape(dims) + (3, 3)
    G = torch.from_numpy(_complex_normal(g, shp)).to(_dev(device))
    H = 0.5 * (G + _tdag(G))
    tr = torch.diagonal(H, dim1=-2, dim2=-1).sum(-1)
    H = H - (tr / 3.0)[..., None, None] * torch.eye(3, dtype=H.dtype, device=H.device)
    return _treunitarise(_texpm(1j * eps * H))


def random_links(dims, eps: float, seed: int, device=None) -> np.ndarray:
    """U = exp(i*eps*H), H = (G+G^dag)/2 - tr(...)/3 with G complex normal.

    The result is unitary with det 1 (H traceless), i.e. in SU(3).
    """
    return np.ascontiguousarray(_random_links_t(dims, eps, seed, device).cpu().numpy())


def unit_links(dims) -> np.ndarray:
    shp = (4,) + site_shape(dims) + (3, 3)
    U = np.zeros(shp, dtype=np.complex128)
    U[...] = np.eye(3)
    return U


def reunitarise(U: np.ndarray, device=None) -> np.ndarray:
    """Nearest SU(3) matrix (polar factor with the determinant phase removed) of
    an almost unitary U."""
    torch = _torch()
    Ut = torch.from_numpy(np.ascontiguousarray(U, dtype=np.complex128)).to(_dev(device))
    return _treunitarise(Ut).cpu().numpy()


def _smear_t(U, rho: float, nsteps: int, reunit: bool):
    torch = _torch()
    eye = torch.eye(3, dtype=U.dtype, device=U.device)

    def shift(A, mu, k):
        """B(x) = A(x + k*mu_hat), periodic; A has site axes (Lt,Lz,Ly,Lx) first."""
        return torch.roll(A, shifts=-k, dims=_AXIS[mu])

    for _ in range(nsteps):
        Unew = torch.empty_like(U)
        for mu in range(4):
            C = torch.zeros_like(U[mu])
            for nu in range(4):
                if nu == mu:
                    continue
                up = U[nu] @ shift(U[mu], nu, 1) @ _tdag(shift(U[nu], mu, 1))
                Unu_m = shift(U[nu], nu, -1)
                dn = _tdag(Unu_m) @ shift(U[mu], nu, -1) @ shift(Unu_m, mu, 1)
                C += up + dn
            C *= rho
            W = C @ _tdag(U[mu])
            A = 0.5 * (W - _tdag(W))
            tr = torch.diagonal(A, dim1=-2, dim2=-1).sum(-1)
            A = A - (tr / 3.0)[..., None, None] * eye
            Unew[mu] = _texpm(A) @ U[mu]
        U = _treunitarise(Unew) if reunit else Unew
    return U


def smear_stout(U: np.ndarray, rho: float, nsteps: int, reunit: bool = True, device=None) -> np.ndarray:
    """Stout projection of APE staples, eq. (stout_smearing) of Sec. 2.2, repeated.

    C_mu(x) = rho * sum_{nu != mu} [ U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag
                                     + U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) ]
    U'_mu(x) = exp([C_mu(x) U_mu(x)^dag]_AT) U_mu(x),
    [W]_AT = (W - W^dag)/2 - tr(W - W^dag)/6.
    All directions are updated together from the previous step's links.  The
    optional re-unitarisation only removes rounding drift.
    """
    torch = _torch()
    Ut = torch.from_numpy(np.array(U, dtype=np.complex128, copy=True)).to(_dev(device))
    return np.ascontiguousarray(_smear_t(Ut, rho, nsteps, reunit).cpu().numpy())


def smeared_links(dims, eps: float, rho: float, nsteps: int, seed: int, device=None) -> np.ndarray:
    """Random SU(3) links followed by ``nsteps`` stout/APE smearing steps."""
    U = _random_links_t(dims, eps, seed, device)
    return np.ascontiguousarray(_smear_t(U, rho, nsteps, True).cpu().numpy())


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


def workload_links(w: dict, device=None) -> np.ndarray:
    """The workload's link field; device selects where the link algebra runs
    (None: the host; "cuda" for the large lattices)."""
    if w["smear"]:
        return smeared_links(w["dims"], w["eps"], 0.1, w["smear"], w["gauge_seed"], device=device)
    return random_links(w["dims"], w["eps"], w["gauge_seed"], device=device)
