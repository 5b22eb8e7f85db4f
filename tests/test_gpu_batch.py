"""Batched multi-system solve (dwf_solve_batch) against the FP64 oracle.

Systems of one lattice with different Ls, quark masses, forms and sources run
in lock step in shared launches; each 4D solution must match the oracle's
solve of its own system within 1e-9 (relative 2-norm), whatever the wave
split, the inner precision or the order in which the systems converge.
"""

import numpy as np
import pytest

from _util import rel, to_gpu, to_np
from paper_2602_14454_gb300 import inputs

pytestmark = pytest.mark.gpu

DIMS = (4, 4, 4, 4)


@pytest.fixture(scope="module", autouse=True)
def _built(cuda_ok):
    from paper_2602_14454_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def systems():
    """12 systems: Ls in {4, 6, 8} x m in {0.02, 0.1} x {point source, Gaussian source},
    Mobius (1.5, 0.5) Neff alpha 0.5 for even Ls, Shamir standard for Ls = 6."""
    import torch
    from oracle import dwf as orc
    from paper_2602_14454_gb300 import dwf
    U = inputs.random_links(DIMS, 0.5, 1003)
    Ut = torch.from_numpy(U).cuda()
    ops, refs, b4s, want = [], [], [], []
    handles = {}
    for Ls in (4, 6, 8):
        for mf in (0.02, 0.1):
            if Ls == 6:
                kw = dict(b=1.0, c=0.0, form="standard", alpha=1.0)
            else:
                kw = dict(b=1.5, c=0.5, form="neff", alpha=0.5)
            op = dwf.Operator(DIMS, Ls, 1.8, mf, kw["b"], kw["c"], form=kw["form"], alpha=kw["alpha"])
            op.set_gauge(Ut)
            ref = orc.DWF(U, DIMS, Ls, 1.8, mf, kw["b"], kw["c"], form=kw["form"], alpha=kw["alpha"])
            handles[(Ls, mf)] = (op, ref)
    k = 0
    for (Ls, mf), (op, ref) in handles.items():
        for src in ("point", "gauss"):
            b4 = (inputs.point_source(DIMS, spin=k % 4, colour=k % 3) if src == "point"
                  else inputs.gaussian_4d(DIMS, 3000 + k))
            x5, _ = ref.solve(ref.source_5d(b4), tol=1e-13)
            ops.append(op)
            refs.append(ref)
            b4s.append(b4)
            want.append(ref.project_4d(x5))
            k += 1
    return ops, refs, b4s, want


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
def test_batch_matches_oracle(systems, prec):
    from paper_2602_14454_gb300 import dwf
    ops, refs, b4s, want = systems
    x4s, stats = dwf.solve_batch(ops, [to_gpu(b) for b in b4s], inner_prec=prec, tol=1e-10)
    for i, (x4, w, s) in enumerate(zip(x4s, want, stats)):
        assert s["status"] == "DWF_OK", i
        assert s["true_residual"] <= 1e-10, i
        assert rel(to_np(x4), w) < 1e-9, i
        assert s["waves"] == 1 and s["iterations"] > 0


def test_batch_waves_give_the_same_solutions(systems):
    from paper_2602_14454_gb300 import dwf
    ops, refs, b4s, want = systems
    x4a, sa = dwf.solve_batch(ops, [to_gpu(b) for b in b4s], inner_prec="f32", tol=1e-10)
    x4b, sb = dwf.solve_batch(ops, [to_gpu(b) for b in b4s], inner_prec="f32", tol=1e-10, batch_wave=5)
    assert all(s["waves"] == 3 for s in sb)
    for i in range(len(ops)):
        assert rel(to_np(x4b[i]), want[i]) < 1e-9
        # same arithmetic per system whatever the wave it ran in
        assert sa[i]["iterations"] == sb[i]["iterations"]
        assert np.array_equal(to_np(x4a[i]), to_np(x4b[i]))


def test_batch_matches_single_solves(systems):
    """A batched system follows the iteration of dwf_solve on the same system."""
    from paper_2602_14454_gb300 import dwf
    ops, refs, b4s, want = systems
    idx = [0, 5, 9]
    x4s, st = dwf.solve_batch([ops[i] for i in idx], [to_gpu(b4s[i]) for i in idx], inner_prec="f32")
    for j, i in enumerate(idx):
        b5 = ops[i].source_5d(to_gpu(b4s[i]))
        x5, s1 = ops[i].solve(b5, inner_prec="f32")
        assert abs(s1["iterations"] - st[j]["iterations"]) <= 16   # one convergence-check interval
        assert rel(to_np(x4s[j]), to_np(ops[i].project_4d(x5))) < 1e-9


def test_batch_zero_source_and_empty(systems):
    import torch
    from paper_2602_14454_gb300 import dwf
    ops, refs, b4s, want = systems
    z = torch.zeros_like(to_gpu(b4s[0]))
    x4s, st = dwf.solve_batch([ops[0], ops[1]], [z, to_gpu(b4s[1])])
    assert float(torch.abs(x4s[0]).max()) == 0.0
    assert rel(to_np(x4s[1]), want[1]) < 1e-9
    x4s, st = dwf.solve_batch([], [])
    assert x4s == [] and st == []


def test_batch_rejects_mixed_lattices(systems):
    import torch
    from paper_2602_14454_gb300 import dwf
    ops, refs, b4s, want = systems
    other = dwf.Operator((4, 4, 4, 6), 4, 1.8, 0.1, 1.5, 0.5, form="neff", alpha=0.5)
    other.set_gauge(torch.from_numpy(inputs.random_links((4, 4, 4, 6), 0.5, 1)).cuda())
    with pytest.raises(dwf.DwfError):
        dwf.solve_batch([ops[0], other], [to_gpu(b4s[0]), to_gpu(inputs.gaussian_4d((4, 4, 4, 6), 1))])


def test_batch_medium_lattice_alpha_invariance():
    """8^3x16, Ls in {8, 12, 16}, three masses, two forms, two point sources: 72 systems in one
    batch; the Neff and standard forms of each system give the same 4D solution
    (Sec. 2.3), and each agrees with a separate dwf_solve."""
    import torch
    from paper_2602_14454_gb300 import dwf
    dims = (8, 8, 8, 16)
    U = torch.from_numpy(inputs.smeared_links(dims, 0.3, 0.1, 3, 1003)).cuda()
    ops, b4s = [], []
    for Ls in (8, 12, 16):
        for mf in (0.005, 0.02, 0.05):
            for form, alpha in (("standard", 1.0), ("neff", 0.5)):
                op = dwf.Operator(dims, Ls, 1.8, mf, 1.5, 0.5, form=form, alpha=alpha)
                op.set_gauge(U)
                for sc in ((0, 0), (2, 1)):
                    ops.append(op)
                    b4s.append(to_gpu(inputs.point_source(dims, spin=sc[0], colour=sc[1])))
    x4s, st = dwf.solve_batch(ops, b4s, inner_prec="f16", tol=1e-10)
    assert all(s["status"] == "DWF_OK" and s["true_residual"] <= 1e-10 for s in st)
    assert len({s["iterations"] for s in st}) > 1      # the systems left the lock step at different times
    for i in range(0, len(ops), 4):   # (standard, src0), (standard, src1), (neff, src0), (neff, src1)
        for k in (0, 1):
            assert rel(to_np(x4s[i + 2 + k]), to_np(x4s[i + k])) < 1e-9
    b5 = ops[-1].source_5d(b4s[-1])
    x5, _ = ops[-1].solve(b5, inner_prec="f32")
    assert rel(to_np(x4s[-1]), to_np(ops[-1].project_4d(x5))) < 1e-9
