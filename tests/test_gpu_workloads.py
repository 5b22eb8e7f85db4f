"""The solver on the full-size workloads, checked by the FP64 oracle.

* 32^3x64, Ls 16, Mobius (1.5, 0.5), M0 1.8, m 0.005 (the benchmark's
  workload): FP32 and FP16 inner CG with FP64 reliable updates, Neff's form
  (alpha 0.5) and the standard form.  The oracle builds b5 from b4 and
  recomputes ||b5 - D x5|| / ||b5|| of the full 5D system row by row
  (oracle.DWF.residual_norm); the 4D solutions of the two forms agree
  (Sec. 2.3: x4 does not depend on alpha).
* 24^3x48 batched wave: Ls 8, 12 and 16 with m 0.005, 0.02 and 0.05 and
  point sources in one dwf_solve_batch call; every 4D solution equals the one
  of the same system solved alone, whose 5D residual the oracle recomputes.
* 16^4, Ls 16, Neff alpha 0.5, m 0.01: a network trained on the method's own
  solves preconditions the solve; the oracle recomputes its residual and its
  4D solution equals the plain solve's.
"""

import numpy as np
import pytest

from _util import rel, to_gpu, to_np
from paper_2602_14454_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built(cuda_ok):
    from paper_2602_14454_gb300 import build
    build.build()


def _pair(w, U, Ut, Ls, mf, form, alpha):
    from oracle import dwf as orc
    from paper_2602_14454_gb300 import dwf
    op = dwf.Operator(w["dims"], Ls, w["M0"], mf, w["b"], w["c"], form=form, alpha=alpha)
    op.set_gauge(Ut)
    ref = orc.DWF(U, w["dims"], Ls, w["M0"], mf, w["b"], w["c"], form=form, alpha=alpha)
    return op, ref


def test_c5_32c64_mixed_precision_solves():
    import torch
    w = inputs.WORKLOADS["c5_32^3x64_ls16_mobius"]
    U = inputs.workload_links(w, device="cuda")
    Ut = torch.from_numpy(U).cuda()
    b4 = inputs.gaussian_4d(w["dims"], w["src_seed"])
    ops = {f: _pair(w, U, Ut, w["Ls"], w["mf"], f, a) for f, a in (("neff", 0.5), ("standard", 1.0))}
    op, ref = ops["neff"]
    b5 = op.source_5d(to_gpu(b4))
    # the source (the same for both forms), row by row against the oracle's
    b5h = to_np(b5)
    num = den = 0.0
    for s in range(w["Ls"]):
        want = ref.source_row(b4, s)
        num += np.linalg.norm((b5h[s] - want).ravel()) ** 2
        den += np.linalg.norm(want.ravel()) ** 2
    del b5h
    assert np.sqrt(num / den) < 1e-13
    x4 = {}
    for form, prec, oracle_check in (("neff", "f32", True), ("standard", "f16", True), ("neff", "f16", False)):
        op, ref = ops[form]
        x5, st = op.solve(b5, inner_prec=prec, tol=1e-10)
        assert st["true_residual"] <= 1e-10, (form, prec)
        if oracle_check:
            r = ref.residual_norm(lambda s: ref.source_row(b4, s), to_np(x5))
            print("32^3x64 %s %s: %d iterations, oracle residual %.3e" % (form, prec, st["iterations"], r))
            assert r <= 1e-10, (form, prec, r)
        x4[(form, prec)] = to_np(op.project_4d(x5))
        del x5
    keys = list(x4)
    for k in keys[1:]:
        assert rel(x4[k], x4[keys[0]]) < 1e-9, k


def test_c3_24c48_batched_wave_mixed_ls():
    import torch
    from paper_2602_14454_gb300 import dwf
    w = inputs.WORKLOADS["c3_24^3x48_batched"]
    U = inputs.workload_links(w, device="cuda")
    Ut = torch.from_numpy(U).cuda()
    systems = [(8, 0.005, 0, 0), (12, 0.02, 1, 1), (16, 0.05, 2, 2)]   # (Ls, m, spin, colour)
    pairs = [_pair(w, U, Ut, Ls, mf, "standard", 1.0) for Ls, mf, _, _ in systems]
    b4s = [inputs.point_source(w["dims"], spin=sp, colour=co) for _, _, sp, co in systems]
    x4_batch, stats = dwf.solve_batch([p[0] for p in pairs], [to_gpu(b) for b in b4s], inner_prec="f32",
                                      tol=1e-10)
    for (op, ref), b4, xb, sb in zip(pairs, b4s, x4_batch, stats):
        b5 = op.source_5d(to_gpu(b4))
        x5, st = op.solve(b5, inner_prec="f32", tol=1e-10)
        r = ref.residual_norm(lambda s: ref.source_row(b4, s), to_np(x5))
        assert r <= 1e-10, (op.Ls, r)
        assert sb["true_residual"] <= 1e-10
        assert rel(to_np(xb), to_np(op.project_4d(x5))) < 1e-9, op.Ls


def test_c4_16c4_learned_preconditioner_solve():
    import torch
    w = inputs.WORKLOADS["c4_16^4_ls16_neff"]
    U = inputs.workload_links(w, device="cuda")
    Ut = torch.from_numpy(U).cuda()
    op, ref = _pair(w, U, Ut, w["Ls"], w["mf"], "neff", w["alpha"])
    srcs = [to_gpu(inputs.gaussian_4d(w["dims"], s)) for s in list(w["train_seeds"])[:8]]
    st = op.precond_train(srcs, epochs=3, batch=8, lr=2e-3, solve_inner_prec="f32")
    assert st["loss_last"] < st["loss_first"]
    b4 = inputs.gaussian_4d(w["dims"], list(w["test_seeds"])[0])
    b5 = op.source_5d(to_gpu(b4))
    x5, s = op.solve(b5, inner_prec="f32", precond=1, tol=1e-10)
    x5p, s0 = op.solve(b5, inner_prec="f32", tol=1e-10)
    assert s["precond_applications"] > 0
    r = ref.residual_norm(lambda s: ref.source_row(b4, s), to_np(x5))
    print("16^4 learned: %d iterations (plain %d), oracle residual %.3e" % (s["iterations"], s0["iterations"], r))
    assert r <= 1e-10
    assert rel(to_np(op.project_4d(x5)), to_np(op.project_4d(x5p))) < 1e-9
