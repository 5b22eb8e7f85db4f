"""FP64 oracle of the learned preconditioner and of flexible CG (test infrastructure only).

The paper has no learned part; this restates the network that the library
trains, in plain NumPy, so that the CUDA forward, backward and optimiser
kernels can be checked element by element.  Only tests/, the smoke check and
the benchmark's CPU legs may import it.

Network (a gauge-covariant linear stencil net after the parallel-transport
convolutions of Lehner and Wettig, 2023).  A field psi has C channels of 4D
spinors: shape (C, Lt, Lz, Ly, Lx, 4, 3).  One layer with weights
W[p, chi, c, c'] (complex; p = 0 self, 1 + 2 mu the hop from x + mu,
2 + 2 mu the hop from x - mu; chi = 0 for the output spins 0, 1 (P_+),
1 for spins 2, 3 (P_-)) computes

    out(c, x)_alpha = sum_p sum_c' W[p, chi(alpha), c, c'] T_p(c', x)_alpha,
    T_0(x)      = psi(x),
    T_{+mu}(x)  = (1 - gamma_mu) U_mu(x)          psi(x + mu),
    T_{-mu}(x)  = (1 + gamma_mu) U_mu(x - mu)^dag psi(x - mu),

with the fermion boundary phases bc[mu] on hops across the boundary: the
spin and colour structure of the Wilson hop of eq. (Wilson_matrix), so that
C = 1, W_0 = 4 - M0, W_{+-mu} = -1/2 is D_W(-M0) itself (pinned by a test
against the C oracle of D_W).  Gauge transformations act on colour only and
W on channels and chirality only, so every layer is gauge covariant.

The network N acts on even-site 5D fields r (Ls, Vh, 4, 3) of the even-odd
system: the Ls slices are the C = Ls channels, the field is put on the even
sites of the full lattice (zero on odd sites), the layers are applied, and
the even sites of the result are N(r).  N is linear in r and is trained to
approximate D^-1, D the even-odd matrix; the preconditioner of CG on the
normal equation D^dag D is M = N N^dag (Hermitian, positive semi-definite).

Training loss over pairs (b_k, x_k) with D x_k = b_k:
L = (1/K) sum_k |N(b_k) - x_k|^2 / |x_k|^2.
Gradients use the convention grad(z) = dL/dRe z + i dL/dIm z, under which
y = w t gives grad(w) = sum grad(y) conj(t) and grad(t) = sum grad(y) conj(w).
"""

from __future__ import annotations

import numpy as np

from .dwf import GAMMA, ONE4, norm

NHOP = 9


def site_axis(mu: int) -> int:
    """Axis of direction mu (0 = x .. 3 = t) in a (C, Lt, Lz, Ly, Lx, 4, 3) field."""
    return 4 - mu


def shift(psi: np.ndarray, mu: int, k: int, bc) -> np.ndarray:
    """psi(x + k mu) for k = +1 / -1, with the boundary phase bc[mu] on the wrapped sites."""
    ax = site_axis(mu)
    out = np.roll(psi, -k, axis=ax)
    L = psi.shape[ax]
    edge = [slice(None)] * psi.ndim
    edge[ax] = L - 1 if k == 1 else 0
    out[tuple(edge)] *= bc[mu]
    return out


def link(U: np.ndarray, mu: int) -> np.ndarray:
    """U_mu(x) as (Lt, Lz, Ly, Lx, 3, 3)."""
    return U[mu]


def colour(Um: np.ndarray, psi: np.ndarray, dag: bool = False) -> np.ndarray:
    """Apply the site's colour matrix (or its adjoint) to every channel and spin."""
    if dag:
        return np.einsum("tzyxba,ctzyxsb->ctzyxsa", Um.conj(), psi)
    return np.einsum("tzyxab,ctzyxsb->ctzyxsa", Um, psi)


def spinm(S: np.ndarray, psi: np.ndarray) -> np.ndarray:
    return np.einsum("ij,...jc->...ic", S, psi)


def transports(U: np.ndarray, psi: np.ndarray, bc) -> list:
    """[T_0, T_{+x}, T_{-x}, T_{+y}, ...] of the layer definition above."""
    T = [psi]
    for mu in range(4):
        fwd = spinm(ONE4 - GAMMA[mu], colour(link(U, mu), shift(psi, mu, +1, bc)))
        # U_mu(x - mu)^dag psi(x - mu) = [U_mu^dag psi](x - mu)
        bwd = spinm(ONE4 + GAMMA[mu], shift(colour(link(U, mu), psi, dag=True), mu, -1, bc))
        T += [fwd, bwd]
    return T


def chirality_mix(W: np.ndarray, T: np.ndarray) -> np.ndarray:
    """sum_c' W[chi(alpha), c, c'] T(c')_alpha for one hop (W: (2, C, C))."""
    out = np.empty_like(T)
    out[..., 0:2, :] = np.einsum("ij,jtzyxsa->itzyxsa", W[0], T[..., 0:2, :])
    out[..., 2:4, :] = np.einsum("ij,jtzyxsa->itzyxsa", W[1], T[..., 2:4, :])
    return out


def layer(U: np.ndarray, W: np.ndarray, psi: np.ndarray, bc) -> np.ndarray:
    """One layer: W of shape (9, 2, C, C), psi of shape (C, Lt, Lz, Ly, Lx, 4, 3)."""
    T = transports(U, psi, bc)
    out = np.zeros_like(psi)
    for p in range(NHOP):
        out += chirality_mix(W[p], T[p])
    return out


def layer_backward(U: np.ndarray, W: np.ndarray, psi: np.ndarray, G: np.ndarray, bc):
    """Given grad of the layer output G, return (grad W, grad psi).

    grad W[p, chi, c, c'] = sum_{x, alpha in chi, a} G(c, x)_alpha,a conj(T_p(c', x)_alpha,a);
    grad psi = layer_adjoint(G).
    """
    T = transports(U, psi, bc)
    C = psi.shape[0]
    gW = np.zeros((NHOP, 2, C, C), dtype=np.complex128)
    for p in range(NHOP):
        for chi, sp in ((0, slice(0, 2)), (1, slice(2, 4))):
            gW[p, chi] = np.einsum("ctzyxsa,dtzyxsa->cd", G[..., sp, :], T[p][..., sp, :].conj())
    return gW, layer_adjoint(U, W, G, bc)


def layer_adjoint(U: np.ndarray, W: np.ndarray, G: np.ndarray, bc) -> np.ndarray:
    """The adjoint of the layer (as a linear map of its input) applied to G:
    grad T_p = W^H G per chirality, then the adjoint of each transport, written
    out hop by hop (not derived from the forward)."""
    gpsi = np.zeros_like(G)
    for p in range(NHOP):
        # grad T_p(c') = sum_c conj(W[p, chi, c, c']) G(c)
        gT = np.empty_like(G)
        gT[..., 0:2, :] = np.einsum("ij,itzyxsa->jtzyxsa", W[p, 0].conj(), G[..., 0:2, :])
        gT[..., 2:4, :] = np.einsum("ij,itzyxsa->jtzyxsa", W[p, 1].conj(), G[..., 2:4, :])
        if p == 0:
            gpsi += gT
            continue
        mu, fwd = (p - 1) // 2, (p - 1) % 2 == 0
        if fwd:
            # T(x) = S U_mu(x) psi(x+mu)  =>  grad psi(y) += U_mu(y-mu)^dag S^dag gT(y-mu)
            h = colour(link(U, mu), spinm((ONE4 - GAMMA[mu]).conj().T, gT), dag=True)
            gpsi += shift(h, mu, -1, bc)
        else:
            # T(x) = S U_mu(x-mu)^dag psi(x-mu)  =>  grad psi(y) += U_mu(y) S^dag gT(y+mu)
            h = shift(spinm((ONE4 + GAMMA[mu]).conj().T, gT), mu, +1, bc)
            gpsi += colour(link(U, mu), h)
    return gpsi


class Net:
    """The network N: weights (L, 9, 2, C, C) complex, on the even-odd system of
    a lattice with the parity split of the oracle (even: x+y+z+t even)."""

    def __init__(self, U, dims, bc, weights: np.ndarray):
        self.U = np.asarray(U)
        self.dims = tuple(dims)
        self.bc = tuple(bc)
        self.W = np.array(weights, dtype=np.complex128)
        Lx, Ly, Lz, Lt = dims
        t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
        par = ((x + y + z + t) % 2).ravel()
        self.even = np.nonzero(par == 0)[0]

    @property
    def C(self):
        return self.W.shape[-1]

    def embed(self, r: np.ndarray) -> np.ndarray:
        """(Ls, Vh, 4, 3) even-site field -> (C, Lt, Lz, Ly, Lx, 4, 3), zero on odd sites."""
        Lx, Ly, Lz, Lt = self.dims
        full = np.zeros((r.shape[0], Lx * Ly * Lz * Lt, 4, 3), dtype=np.complex128)
        full[:, self.even] = r
        return full.reshape((r.shape[0], Lt, Lz, Ly, Lx, 4, 3))

    def restrict(self, psi: np.ndarray) -> np.ndarray:
        return np.ascontiguousarray(psi.reshape((psi.shape[0], -1, 4, 3))[:, self.even])

    def forward(self, r: np.ndarray, keep: bool = False):
        acts = [self.embed(r)]
        for l in range(self.W.shape[0]):
            acts.append(layer(self.U, self.W[l], acts[-1], self.bc))
        out = self.restrict(acts[-1])
        return (out, acts) if keep else out

    def adjoint(self, r: np.ndarray) -> np.ndarray:
        """N^dag r: the adjoint layers in reverse order between the same embedding
        and restriction (their adjoints are each other)."""
        G = self.embed(r)
        for l in range(self.W.shape[0] - 1, -1, -1):
            G = layer_adjoint(self.U, self.W[l], G, self.bc)
        return self.restrict(G)

    def precondition(self, r: np.ndarray) -> np.ndarray:
        """M r = N N^dag r: Hermitian positive semi-definite by construction, the
        preconditioner of CG on D^dag D when N approximates D^-1."""
        return self.forward(self.adjoint(r))

    def loss_and_grad(self, pairs):
        """L = (1/K) sum |M b - x|^2/|x|^2 and its gradient with respect to W."""
        K = len(pairs)
        gW = np.zeros_like(self.W)
        L = 0.0
        for b, x in pairs:
            y, acts = self.forward(b, keep=True)
            xn2 = norm(x) ** 2
            L += norm(y - x) ** 2 / xn2 / K
            G = self.embed(2.0 * (y - x) / xn2 / K)
            for l in range(self.W.shape[0] - 1, -1, -1):
                g, G = layer_backward(self.U, self.W[l], acts[l], G, self.bc)
                gW[l] += g
        return L, gW


def adam_step(theta: np.ndarray, g: np.ndarray, m: np.ndarray, v: np.ndarray, t: int, lr: float,
              beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam step (Kingma and Ba, 2015) on the real and imaginary parts of a
    complex parameter array separately; t counts steps from 1.  Returns the new
    (theta, m, v); m and v hold the moments of (Re g, Im g) as complex numbers
    (first moment) and as a complex number of the two second moments."""
    gr, gi = g.real, g.imag
    m = complex(beta1) * m + (1 - beta1) * g
    v = beta2 * v.real + (1 - beta2) * gr ** 2 + 1j * (beta2 * v.imag + (1 - beta2) * gi ** 2)
    mh = m / (1 - beta1 ** t)
    vr = v.real / (1 - beta2 ** t)
    vi = v.imag / (1 - beta2 ** t)
    step = mh.real / (np.sqrt(vr) + eps) + 1j * mh.imag / (np.sqrt(vi) + eps)
    return theta - lr * step, m, v


def fcg(A, M, b, tol=1e-12, maxiter=10000, x0=None):
    """Flexible CG (Notay 2000) on the Hermitian positive definite A x = b with a
    possibly varying preconditioner M: beta by the Polak-Ribiere formula
    (z_new, r_new - r_old) / (z_old, r_old).  Stops when |r| <= tol |b|."""
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128, copy=True)
    r = b - A(x)
    z = M(r)
    p = z.copy()
    rz = np.vdot(r.ravel(), z.ravel()).real
    bn = norm(b)
    hist = [norm(r) / bn]
    it = 0
    while hist[-1] > tol and it < maxiter:
        q = A(p)
        alpha = rz / np.vdot(p.ravel(), q.ravel()).real
        x = x + alpha * p
        rn = r - alpha * q
        zn = M(rn)
        beta = np.vdot(zn.ravel(), (rn - r).ravel()).real / rz
        rz = np.vdot(rn.ravel(), zn.ravel()).real
        p = zn + beta * p
        r, z = rn, zn
        it += 1
        hist.append(norm(r) / bn)
    return x, dict(iterations=it, history=hist, true_residual=norm(b - A(x)) / bn)
