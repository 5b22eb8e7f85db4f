"""4D domain decomposition in time on one GPU: a ring of slab handles, each
with the ghost faces of its neighbours, applies the even-odd matrix of
eq. even-odd_linear_equation in three stages with face exchanges; the result
equals the unsplit operator (library and oracle) on the whole lattice."""

import numpy as np
import pytest

from _util import TOL, make_pair, maxrel, rel, to_gpu, to_np
from paper_2602_14454_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built(cuda_ok):
    from paper_2602_14454_gb300 import build
    build.build()


def _ring(gdims, nt, Ls, U, form, alpha):
    import torch
    from paper_2602_14454_gb300 import dwf
    slabs = []
    for t0 in range(0, gdims[3], nt):
        sl = dwf.Slab(gdims, t0, nt, Ls, 1.8, 0.02, 1.5, 0.5, form=form, alpha=alpha, bc=(1, 1, 1, -1))
        sl.set_gauge(torch.from_numpy(U).cuda())
        slabs.append(sl)
    return slabs


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("nslab,nt", [(2, 4), (3, 2), (2, 2)])
@pytest.mark.parametrize("dag", [False, True])
def test_slab_ring_equals_unsplit(prec, nslab, nt, dag):
    from paper_2602_14454_gb300 import dwf
    gdims, Ls = (4, 2, 4, nslab * nt), 8
    U = inputs.random_links(gdims, 0.5, 1031)
    op, ref = make_pair(gdims, Ls, 1.8, 0.02, 1.5, 0.5, "neff", 0.5, U=U)
    x = ref.to_eo(inputs.gaussian_5d(gdims, Ls, 1032), 0)
    want_lib = to_np(op.apply(to_gpu(x), op="eo", prec=prec, dag=dag))
    want = ref.d_pc(x, dag=dag)
    slabs = _ring(gdims, nt, Ls, U, "neff", 0.5)
    per = x.shape[1] // nslab   # the slab's even sites: a contiguous range of the even-odd index
    xs = [to_gpu(np.ascontiguousarray(x[:, k * per:(k + 1) * per])) for k in range(nslab)]
    outs = dwf.slab_apply_eo(slabs, xs, prec=prec, dag=dag)
    got = np.concatenate([to_np(o) for o in outs], axis=1)
    assert rel(got, want_lib) < (1e-15 if prec == "f64" else 1e-7), rel(got, want_lib)
    assert rel(got, want) < TOL[prec]
    assert maxrel(got, want) < 10 * TOL[prec]
    for sl in slabs:
        sl.device_status()


def test_slab_faces_and_checks():
    from paper_2602_14454_gb300 import dwf
    gdims, Ls = (4, 2, 4, 8), 4
    U = inputs.random_links(gdims, 0.5, 1033)
    a, b = _ring(gdims, 4, Ls, U, "standard", 1.0)
    f = a.faces("f32", 0)
    A3 = 4 * 2 * 4 // 2
    assert f["bytes"] == A3 * Ls * 24 * 4
    assert f["send_hi"] - f["send_lo"] == 3 * f["bytes"]     # the last of 4 slices
    assert f["recv_lo"] - f["send_lo"] == 4 * f["bytes"]     # ghost rows after Vh = 4 A3
    assert f["recv_hi"] - f["recv_lo"] == f["bytes"]
    x = to_gpu(np.zeros(a.shape_eo(), dtype=np.complex128))
    with pytest.raises(dwf.DwfError):
        a.apply(x, op="eo")                                 # a slab applies only through the stages
    with pytest.raises(dwf.DwfError):
        a.apply_eo_stage(0, x=x, prec="f16")               # FP64 and FP32 only
    with pytest.raises(dwf.DwfError):
        dwf.slab_exchange_ring([b, a, b], "f64", 0)         # not consecutive
    for t0, nt in ((1, 4), (0, 3), (0, 8)):
        with pytest.raises(dwf.DwfError):
            dwf.Slab(gdims, t0, nt, Ls, 1.8, 0.02, 1.0, 0.0)


@pytest.mark.parametrize("nslab,nt", [(2, 4), (3, 2)])
def test_slab_cgnr_ring_matches_oracle(nslab, nt):
    """The decomposed FP64 CGNR over a ring of slabs: the oracle recomputes
    ||b - D x|| <= 1e-10 ||b|| on the joined solution, and the residual history
    follows the oracle's unsplit CGNR step by step (the same Krylov iteration)."""
    from oracle import dwf as orc
    from paper_2602_14454_gb300 import dwf
    gdims, Ls = (4, 2, 4, nslab * nt), 8
    U = inputs.random_links(gdims, 0.5, 1034)
    ref = orc.DWF(U, gdims, Ls, 1.8, 0.05, 1.5, 0.5, form="neff", alpha=0.5)
    b = ref.to_eo(inputs.gaussian_5d(gdims, Ls, 1035), 0)
    import torch
    slabs = []
    for t0 in range(0, gdims[3], nt):
        sl = dwf.Slab(gdims, t0, nt, Ls, 1.8, 0.05, 1.5, 0.5, form="neff", alpha=0.5)
        sl.set_gauge(torch.from_numpy(U).cuda())
        slabs.append(sl)
    per = b.shape[1] // nslab
    bs = [to_gpu(np.ascontiguousarray(b[:, k * per:(k + 1) * per])) for k in range(nslab)]
    xs, hist = dwf.slab_cgnr_ring(slabs, bs, tol=1e-10, max_iter=2000)
    x = np.concatenate([to_np(v) for v in xs], axis=1)
    assert rel(ref.d_pc(x), b) <= 1e-10
    x_ref, info = orc.cgnr(ref.d_pc, lambda v: ref.d_pc(v, dag=True), b, tol=1e-10)
    assert rel(x, x_ref) < 1e-8
    h_ref = info["history"]
    k = min(20, len(h_ref), len(hist))
    assert np.allclose(np.log(hist[:k]), np.log(h_ref[:k]), atol=1e-6)
    assert abs(len(hist) - len(h_ref)) <= 1
