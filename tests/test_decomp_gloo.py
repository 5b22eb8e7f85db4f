"""The 4D domain decomposition of one solve, emulated on two CPU ranks (gloo):
the lattice is cut into two slabs of the time direction, each rank applies the
even-odd operator on its slab with halos of spin-projected half spinors from
its neighbour (oracle/decomp.py), and CG on the normal equation sums its inner
products over the ranks.  The split operator, its adjoint and the split solve
must equal the unsplit oracle (oracle/dwf.py)."""

import os
import socket

import numpy as np
import pytest

DIMS, LS = (4, 2, 2, 8), 6
PARAMS = dict(M0=1.8, mf=0.05, b=1.5, c=0.5, form="neff", alpha=0.5, bc=(1, -1, 1, -1))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _inputs():
    from oracle import dwf as orc
    from paper_2602_14454_gb300 import inputs
    U = inputs.random_links(DIMS, 0.5, 141)
    ref = orc.DWF(U, DIMS, LS, PARAMS["M0"], PARAMS["mf"], PARAMS["b"], PARAMS["c"], form=PARAMS["form"],
                  alpha=PARAMS["alpha"], bc=PARAMS["bc"])
    xe = ref.to_eo(inputs.gaussian_5d(DIMS, LS, 142), 0)
    b5 = ref.source_5d(inputs.gaussian_4d(DIMS, 143))
    return U, ref, xe, b5


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import decomp
    U, ref, xe, b5 = _inputs()
    sp = decomp.SplitDWF(U, DIMS, LS, PARAMS["M0"], PARAMS["mf"], PARAMS["b"], PARAMS["c"], form=PARAMS["form"],
                         alpha=PARAMS["alpha"], bc=PARAMS["bc"])
    nloc = len(sp.even)
    mine = slice(rank * nloc, (rank + 1) * nloc)   # this slab's even sites in the global even order
    y = sp.d_pc(xe[:, mine])
    yd = sp.d_pc(xe[:, mine], dag=True)
    bt = ref.b_tilde(b5)
    x, info = sp.cgnr(bt[:, mine], tol=1e-12)
    out.put((rank, y, yd, x, info, sp.halo_bytes))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_split_operator_and_solve_equal_the_unsplit_oracle(world):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    U, ref, xe, b5 = _inputs()
    y = np.concatenate([r[1] for r in res], axis=1)
    yd = np.concatenate([r[2] for r in res], axis=1)
    want, wantd = ref.d_pc(xe), ref.d_pc(xe, dag=True)
    assert np.abs(y - want).max() <= 1e-14 * np.abs(want).max()
    assert np.abs(yd - wantd).max() <= 1e-14 * np.abs(wantd).max()
    # the split solve: the same iterate as the unsplit CGNR up to the order of the sums
    x = np.concatenate([r[3] for r in res], axis=1)
    assert all(r[4]["iterations"] == res[0][4]["iterations"] for r in res)
    bt = ref.b_tilde(b5)
    from oracle import dwf as orc
    x_ref, info = orc.cgnr(ref.d_pc, lambda v: ref.d_pc(v, dag=True), bt, tol=1e-12)
    assert abs(res[0][4]["iterations"] - info["iterations"]) <= 2
    assert np.linalg.norm((x - x_ref).ravel()) <= 1e-9 * np.linalg.norm(x_ref.ravel())
    assert np.linalg.norm((bt - ref.d_pc(x)).ravel()) <= 1e-11 * np.linalg.norm(bt.ravel())
    # every hop exchanged half spinors only: 6 complex numbers per boundary site and slice
    assert res[0][5] > 0 and res[0][5] % (6 * 16) == 0


def test_half_spinor_basis_rebuilds_the_projection():
    """The two-spin basis of the range of 1 -+ gamma_t reproduces (1 -+ gamma_t) v
    for any spinor v (what makes 6 complex numbers per site enough)."""
    from oracle import decomp, dwf as orc
    g = np.random.default_rng(3)
    v = g.normal(size=(5, 4, 3)) + 1j * g.normal(size=(5, 4, 3))
    for S in (orc.ONE4 - orc.GAMMA[3], orc.ONE4 + orc.GAMMA[3]):
        E = decomp._range_basis(S)
        assert E.shape == (4, 2)
        pv = orc.spin(S, v)
        assert np.abs(orc.spin(E @ E.conj().T, pv) - pv).max() < 1e-14
