"""Parity of the CUDA operators with the FP64 oracle, through the C ABI.

FULL5D: the whole 5D matrix (eq. domainwall_general / domainwall_neff) and its
adjoint; EO_PREC: the even-odd matrix of eq. even-odd_linear_equation and its
adjoint; the 5D source and the 4D projection of Sec. 2.3.  Element-wise
comparison on the same seeded inputs, in FP64 (1e-12), FP32 (1e-5) and
FP16-with-scales (3e-3).
"""

import numpy as np
import pytest

from _util import TOL, make_pair, maxrel, rel, to_gpu, to_np
from paper_2602_14454_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built(cuda_ok):
    from paper_2602_14454_gb300 import build
    build.build()


CASES = [
    # dims, Ls, M0, mf, b, c, form, alpha
    ((4, 4, 4, 4), 8, 1.8, 0.04, 1.0, 0.0, "standard", 1.0),
    ((4, 4, 4, 4), 8, 1.8, 0.04, 1.0, 0.0, "neff", 0.5),
    ((4, 2, 6, 4), 12, 1.8, 0.01, 1.5, 0.5, "neff", 0.4),
    ((6, 2, 2, 4), 16, 1.8, 0.01, 1.5, 0.5, "standard", 1.0),
    ((2, 4, 4, 6), 4, 1.0, 0.1, 1.0, 1.0, "neff", 0.7),
    ((4, 4, 2, 2), 2, 1.8, 0.2, 1.5, 0.5, "neff", 0.6),
    ((2, 2, 2, 4), 32, 1.8, 0.005, 1.5, 0.5, "neff", 0.5),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "L%s_Ls%d_%s" % ("x".join(map(str, c[0])), c[1], c[6]))
@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
def test_full5d_apply_and_dag(case, prec):
    dims, Ls, M0, mf, b, c, form, alpha = case
    op, ref = make_pair(dims, Ls, M0, mf, b, c, form, alpha, seed=11)
    x = inputs.gaussian_5d(dims, Ls, 12)
    for dag in (False, True):
        want = ref.apply(x, dag=dag)
        got = to_np(op.apply(to_gpu(x), op="full", prec=prec, dag=dag))
        assert rel(got, want) < TOL[prec], (dag, rel(got, want))
        assert maxrel(got, want) < 10 * TOL[prec]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "L%s_Ls%d_%s" % ("x".join(map(str, c[0])), c[1], c[6]))
@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
def test_eo_prec_apply_and_dag(case, prec):
    dims, Ls, M0, mf, b, c, form, alpha = case
    op, ref = make_pair(dims, Ls, M0, mf, b, c, form, alpha, seed=21)
    x = ref.to_eo(inputs.gaussian_5d(dims, Ls, 22), 0)
    for dag in (False, True):
        want = ref.d_pc(x, dag=dag)
        got = to_np(op.apply(to_gpu(x), op="eo", prec=prec, dag=dag))
        assert rel(got, want) < TOL[prec], (dag, rel(got, want))
        assert maxrel(got, want) < 10 * TOL[prec], (dag, maxrel(got, want))


@pytest.mark.parametrize("bc", [(1, 1, 1, -1), (1, 1, 1, 1), (-1, 1, -1, 1)])
def test_boundary_phases(bc):
    dims = (4, 2, 2, 4)
    op, ref = make_pair(dims, 6, 1.8, 0.03, 1.5, 0.5, "neff", 0.5, seed=31, bc=bc)
    x = inputs.gaussian_5d(dims, 6, 32)
    assert rel(to_np(op.apply(to_gpu(x), op="full", prec="f64")), ref.apply(x)) < 1e-12


@pytest.mark.parametrize("form", ["standard", "neff"])
def test_source_and_projection(form):
    dims = (4, 4, 2, 4)
    op, ref = make_pair(dims, 8, 1.8, 0.02, 1.5, 0.5, form, 0.5, seed=41)
    b4 = inputs.gaussian_4d(dims, 42)
    b5 = op.source_5d(to_gpu(b4))
    assert rel(to_np(b5), ref.source_5d(b4)) < 1e-13
    x5 = inputs.gaussian_5d(dims, 8, 43)
    assert rel(to_np(op.project_4d(to_gpu(x5))), ref.project_4d(x5)) == 0.0


def test_fifth_matrices_against_closed_form():
    """A5^-1 per chirality equals the closed form of the bidiagonal-plus-corner inverse:
    with kappa = -beta0/alpha0, on P_+ components
    x_Ls = (sum_t kappa^(Ls-t) z_t / alpha0) / (1 + m kappa^Ls),
    x_s = sum_{t<=s} kappa^(s-t) z_t / alpha0 - m kappa^s x_Ls."""
    from paper_2602_14454_gb300 import dwf
    for (Ls, M0, m, b, c) in [(8, 1.8, 0.04, 1.0, 0.0), (16, 1.8, 0.01, 1.5, 0.5), (12, 1.0, 0.1, 1.0, 1.0)]:
        op = dwf.Operator((2, 2, 2, 2), Ls, M0, m, b, c)
        a0, b0 = b * (4 - M0) + 1, c * (4 - M0) - 1
        k = -b0 / a0
        Ainv = op.fifth_matrix(1, 0)
        for t in range(Ls):
            z = np.zeros(Ls)
            z[t] = 1.0
            xl = sum(k ** (Ls - 1 - u) * z[u] / a0 for u in range(Ls)) / (1 + m * k ** Ls)
            x = np.array([sum(k ** (s - u) * z[u] / a0 for u in range(s + 1)) - m * k ** (s + 1) * xl
                          for s in range(Ls)])
            assert np.abs(Ainv[:, t] - x).max() < 1e-13
        A = op.fifth_matrix(0, 0)
        assert np.abs(A @ Ainv - np.eye(Ls)).max() < 1e-13
        Am = op.fifth_matrix(0, 1)
        assert np.abs(Am @ op.fifth_matrix(1, 1) - np.eye(Ls)).max() < 1e-13
        op.close()


def test_adjoint_identity_full_size_f32():
    """<y, D x> = <D^dag y, x> on the 16^3x32, Ls=16 workload (no oracle needed)."""
    dims = (16, 16, 16, 32)
    U = inputs.random_links(dims, 0.3, 1002)
    op, _ = make_pair(dims, 16, 1.8, 0.01, 1.5, 0.5, "neff", 0.5, U=U)
    import torch
    g = torch.Generator(device="cuda").manual_seed(5)
    shp = (16, 65536, 4, 3)
    x = torch.randn(shp, dtype=torch.complex128, device="cuda", generator=g)
    y = torch.randn(shp, dtype=torch.complex128, device="cuda", generator=g)
    for prec, tol in (("f64", 1e-13), ("f32", 1e-6)):
        lhs = torch.vdot(y.flatten(), op.apply(x, op="eo", prec=prec).flatten())
        rhs = torch.vdot(op.apply(y, op="eo", prec=prec, dag=True).flatten(), x.flatten())
        assert abs((lhs - rhs) / lhs) < tol


def test_full_size_eo_parity():
    """EO_PREC at the full 16^3x32, Ls=16 size against the oracle (FP64 and FP32)."""
    from oracle import dwf as orc
    dims = (16, 16, 16, 32)
    U = inputs.random_links(dims, 0.3, 1002)
    op, ref = make_pair(dims, 16, 1.8, 0.01, 1.5, 0.5, "neff", 0.5, U=U)
    x = ref.to_eo(inputs.gaussian_5d(dims, 16, 7), 0)
    want = ref.d_pc(x)
    for prec in ("f64", "f32"):
        got = to_np(op.apply(to_gpu(x), op="eo", prec=prec))
        assert rel(got, want) < TOL[prec]


HOP_CONFIGS = [(4, 1, 4), (4, 2, 6), (4, 1, 12), (4, 2, 16), (4, 1, 5), (3, 1, 3), (3, 2, 8), (3, 1, 8), (0, 1, 3),
               (0, 2, 5), (0, 1, 16), (0, 2, 1), (5, 1, 8), (5, 2, 5), (5, 4, 3), (5, 4, 16), (7, 1, 1), (7, 1, 5),
               (7, 0, 16), (9, 1, 4), (9, 2, 2), (9, 0, 1), (9, 2, 3), (10, 0, 0)]


@pytest.mark.parametrize("cfg", HOP_CONFIGS, ids=lambda c: "var%d_ns%d_sb%d" % c)
@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
@pytest.mark.parametrize("Ls", [8, 12])
def test_hop_configurations_ragged_tiles(cfg, prec, Ls):
    """Every hop variant and tiling gives the same operator; the lattice has
    Vh = 48 sites so most CTA sizes leave a ragged last tile."""
    var, ns, sb = cfg
    dims = (6, 2, 2, 4)
    op, ref = make_pair(dims, Ls, 1.8, 0.02, 1.5, 0.5, "neff", 0.6, seed=51)
    if var >= 7 and prec == "f64":
        return                      # variants 7 and 9 have no FP64 form (FP64 falls back to variant 0)
    op.set_hop_config(prec, var, ns, sb)
    assert op.hop_config(prec)[0] == var
    x = ref.to_eo(inputs.gaussian_5d(dims, Ls, 52), 0)
    for dag in (False, True):
        got = to_np(op.apply(to_gpu(x), op="eo", prec=prec, dag=dag))
        assert rel(got, ref.d_pc(x, dag=dag)) < TOL[prec]
    xf = inputs.gaussian_5d(dims, Ls, 53)
    got = to_np(op.apply(to_gpu(xf), op="full", prec=prec))
    assert rel(got, ref.apply(xf)) < TOL[prec]
    op.device_status()


MIX_CASES = [
    ((4, 2, 6, 4), 12, 1.8, 0.01, 1.5, 0.5, "neff", 0.4),    # Mobius, kappa = -0.023
    ((4, 4, 2, 4), 8, 1.8, 0.04, 1.0, 0.0, "standard", 1.0),  # Shamir, kappa = 0.3125
    ((4, 4, 2, 4), 16, 1.8, 0.02, 1.0, 1.0, "neff", 0.6),     # Borici, kappa = -0.375
    ((2, 2, 4, 4), 32, 1.0, 0.1, 1.0, 1.0, "neff", 0.5),      # Borici M0 = 1, kappa = -0.5, Ls = 32
    ((2, 2, 2, 4), 3, 1.8, 0.3, 1.5, 0.5, "neff", 1.7),       # odd Ls, alpha > 1
]


@pytest.mark.parametrize("case", MIX_CASES, ids=lambda c: "Ls%d_b%g_c%g_%s" % (c[1], c[4], c[5], c[6]))
@pytest.mark.parametrize("mix", [0, 1, 2])
@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
def test_dense_and_structured_mixing(case, mix, prec):
    """The dense Ls x Ls mixing, its structured (recurrence) form and the tensor-core
    product give the same operators."""
    from paper_2602_14454_gb300 import dwf
    dims, Ls, M0, mf, b, c, form, alpha = case
    op, ref = make_pair(dims, Ls, M0, mf, b, c, form, alpha, seed=71)
    if mix == 2 and prec == "f64":
        with pytest.raises(dwf.DwfError):
            op.set_mix_mode(prec, mix)
        return
    op.set_mix_mode(prec, mix)
    assert op.mix_mode(prec) == mix
    x = ref.to_eo(inputs.gaussian_5d(dims, Ls, 72), 0)
    for dag in (False, True):
        assert rel(to_np(op.apply(to_gpu(x), op="eo", prec=prec, dag=dag)), ref.d_pc(x, dag=dag)) < TOL[prec]
    xf = inputs.gaussian_5d(dims, Ls, 73)
    for dag in (False, True):
        assert rel(to_np(op.apply(to_gpu(xf), op="full", prec=prec, dag=dag)), ref.apply(xf, dag=dag)) < TOL[prec]


@pytest.mark.parametrize("ns,sb", [(1, 1), (1, 3), (1, 5), (1, 7), (1, 16), (2, 5), (2, 11)])
@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_tensor_core_mixing_tile_shapes(prec, ns, sb):
    """Tensor-core mixing for CTAs of fewer than 32 threads (dense fallback), with a
    partial last warp, and with a ragged last tile (Vh = 96 sites)."""
    dims, Ls = (4, 4, 2, 6), 12
    op, ref = make_pair(dims, Ls, 1.8, 0.02, 1.5, 0.5, "neff", 0.5, seed=75)
    op.set_mix_mode(prec, 2)
    op.set_hop_config(prec, 0, ns, sb)
    x = ref.to_eo(inputs.gaussian_5d(dims, Ls, 76), 0)
    for dag in (False, True):
        assert rel(to_np(op.apply(to_gpu(x), op="eo", prec=prec, dag=dag)), ref.d_pc(x, dag=dag)) < TOL[prec]
    op.device_status()


def test_tensor_core_mixing_full_size():
    """16^3x32, Ls = 16: the tensor-core mixing against the dense mixing (FP32 fields
    with the split product agree to FP32 rounding)."""
    dims, Ls = (16, 16, 16, 32), 16
    U = inputs.random_links(dims, 0.3, 1002)
    op, ref = make_pair(dims, Ls, 1.8, 0.01, 1.5, 0.5, "neff", 0.5, seed=77, U=U)
    x = to_gpu(ref.to_eo(inputs.gaussian_5d(dims, Ls, 78), 0))
    for prec, tol in (("f32", 5e-6), ("f16", 2e-3)):
        want = [to_np(op.apply(x, op="eo", prec=prec, dag=d)) for d in (False, True)]
        op.set_mix_mode(prec, 2)
        for d, w in zip((False, True), want):
            assert rel(to_np(op.apply(x, op="eo", prec=prec, dag=d)), w) < tol
        op.set_mix_mode(prec, 0)


def test_structured_mixing_refused_when_unstable():
    from paper_2602_14454_gb300 import dwf
    # b = 0.1, c = 1: alpha0 = 0.1*2.2 + 1 = 1.22, beta0 = 1.2 -> |kappa| = 0.98
    op, ref = make_pair((2, 2, 2, 4), 8, 1.8, 0.05, 0.1, 1.0, "standard", 1.0, seed=81)
    assert op.mix_mode("f64") == 0   # dense is the default; the structured form is refused
    with pytest.raises(dwf.DwfError):
        op.set_mix_mode("f64", 1)
    x = ref.to_eo(inputs.gaussian_5d((2, 2, 2, 4), 8, 82), 0)
    assert rel(to_np(op.apply(to_gpu(x), op="eo", prec="f64")), ref.d_pc(x)) < 1e-12


def test_autotuner_picks_a_valid_configuration(tmp_path):
    from paper_2602_14454_gb300 import dwf
    dims = (8, 8, 4, 4)
    op, ref = make_pair(dims, 16, 1.8, 0.01, 1.5, 0.5, "standard", 1.0, seed=61)
    cache = str(tmp_path / "tune.txt")
    cfg = op.autotune("f32", cache)
    assert (cfg[0] in (0, 3, 4, 7, 9) and cfg[1] in (1, 2) and cfg[2] >= 1) or cfg == (10, 0, 0)
    c16 = op.autotune("f16")
    assert c16[0] in (0, 3, 4, 5, 7, 9) and c16[1] in (1, 2, 4) and c16[2] >= 1
    x = ref.to_eo(inputs.gaussian_5d(dims, 16, 63), 0)
    assert rel(to_np(op.apply(to_gpu(x), op="eo", prec="f16")), ref.d_pc(x)) < TOL["f16"]
    op2, _ = make_pair(dims, 16, 1.8, 0.01, 1.5, 0.5, "standard", 1.0, seed=61)
    assert op2.autotune("f32", cache) == cfg          # cache hit
    x = ref.to_eo(inputs.gaussian_5d(dims, 16, 62), 0)
    assert rel(to_np(op.apply(to_gpu(x), op="eo", prec="f32")), ref.d_pc(x)) < TOL["f32"]


def test_errors():
    import torch
    from paper_2602_14454_gb300 import dwf
    with pytest.raises(dwf.DwfError) as e:
        dwf.Operator((3, 4, 4, 4), 8, 1.8, 0.1, 1, 0)
    assert e.value.status == 1
    with pytest.raises(dwf.DwfError):
        dwf.Operator((4, 4, 4, 4), 33, 1.8, 0.1, 1, 0)
    with pytest.raises(dwf.DwfError):
        dwf.Operator((4, 4, 4, 4), 8, 1.8, 0.1, 1, 0, form="neff", alpha=0.0)
    op = dwf.Operator((4, 4, 4, 4), 8, 1.8, 0.1, 1, 0)
    x = torch.zeros((8, 4, 4, 4, 4, 4, 3), dtype=torch.complex128, device="cuda")
    with pytest.raises(dwf.DwfError) as e:
        op.apply(x)
    assert e.value.status == 8


@pytest.mark.parametrize("Ls,dims", [(16, (4, 2, 6, 4)), (4, (2, 4, 4, 6)), (32, (2, 2, 2, 4)), (8, (8, 4, 4, 4)),
                                     (12, (4, 2, 2, 6))])
@pytest.mark.parametrize("prec", ["f32", "f16"])
@pytest.mark.parametrize("var,ns,sb", [(7, 1, 1), (7, 1, 3), (7, 0, 8), (9, 1, 1), (9, 1, 3), (9, 2, 4), (9, 2, 2),
                                       (10, 0, 0)])
def test_persistent_hop_variants(Ls, dims, prec, var, ns, sb):
    """Variant 7 (links staged per CTA tile of sb sites, padded mixing tile,
    mixing by half of the threads) and variant 9 (warp tiles with their own links
    and mixing tile, sb warps per CTA, ns the register budget) give the even-odd
    operator, its adjoint and the full 5D operator of the oracle; Ls = 4, 8, 16
    and 32 put 8, 4, 2 and 1 sites in a warp tile (Ls 12 takes variant 9's
    fallback).  Variant 10 (variant 9 with the mixings on the tensor cores) runs
    for FP32 at Ls 8 and 16 and falls back to variant 9 elsewhere."""
    op, ref = make_pair(dims, Ls, 1.8, 0.02, 1.5, 0.5, "neff", 0.5, seed=81)
    op.set_hop_config(prec, var, ns, sb)
    x = ref.to_eo(inputs.gaussian_5d(dims, Ls, 82), 0)
    for dag in (False, True):
        got = to_np(op.apply(to_gpu(x), op="eo", prec=prec, dag=dag))
        want = ref.d_pc(x, dag=dag)
        assert rel(got, want) < TOL[prec], (dag, rel(got, want))
        assert maxrel(got, want) < 10 * TOL[prec]
    xf = inputs.gaussian_5d(dims, Ls, 83)
    assert rel(to_np(op.apply(to_gpu(xf), op="full", prec=prec)), ref.apply(xf)) < TOL[prec]
    op.device_status()


@pytest.mark.parametrize("var", [7, 9, 10])
def test_persistent_hop_variants_full_size(var):
    """16^3x32, Ls 16: variants 7 and 9 against variant 0 (FP32) and variant 5 (FP16)
    on the same input: the same operator to the precision's rounding."""
    dims, Ls = (16, 16, 16, 32), 16
    U = inputs.random_links(dims, 0.3, 1002)
    op, ref = make_pair(dims, Ls, 1.8, 0.01, 1.5, 0.5, "neff", 0.5, seed=84, U=U)
    x = to_gpu(ref.to_eo(inputs.gaussian_5d(dims, Ls, 85), 0))
    for prec, base, tol in (("f32", 0, 2e-6), ("f16", 5, 2e-3)):
        for dag in (False, True):
            op.set_hop_config(prec, base, 1, 0)
            want = to_np(op.apply(x, op="eo", prec=prec, dag=dag))
            op.set_hop_config(prec, var, 0 if var == 10 else 1, 0)
            got = to_np(op.apply(x, op="eo", prec=prec, dag=dag))
            assert rel(got, want) < tol, (prec, dag, rel(got, want))
    op.device_status()


@pytest.mark.parametrize("prec,var,ns,sb", [("f32", 9, 2, 4), ("f32", 0, 1, 0), ("f16", 5, 1, 0), ("f16", 9, 1, 3),
                                            ("f64", 0, 1, 0)])
@pytest.mark.parametrize("zblock", [1, 2, 4])
def test_sweep_order_columns(prec, var, ns, sb, zblock):
    """The hops swept in columns of zblock z-planes (dwf_set_sweep) give the
    oracle's even-odd operator and adjoint."""
    dims, Ls = (8, 8, 8, 6), 8     # A = 32 sites of one parity per z-plane
    op, ref = make_pair(dims, Ls, 1.8, 0.02, 1.5, 0.5, "neff", 0.5, seed=86)
    op.set_hop_config(prec, var, ns, sb)
    op.set_sweep(prec, zblock)
    assert op.sweep(prec) == zblock
    x = ref.to_eo(inputs.gaussian_5d(dims, Ls, 87), 0)
    for dag in (False, True):
        got = to_np(op.apply(to_gpu(x), op="eo", prec=prec, dag=dag))
        want = ref.d_pc(x, dag=dag)
        assert rel(got, want) < TOL[prec], (dag, rel(got, want))
        assert maxrel(got, want) < 10 * TOL[prec]
    op.device_status()


def test_sweep_argument_checks():
    from paper_2602_14454_gb300 import dwf
    op = dwf.Operator((8, 8, 8, 6), 8, 1.8, 0.02, 1.5, 0.5)
    assert op.sweep("f32") == 0           # a whole t-slice fits the column budget: index order
    for bad in (-3, 3, 8, 16):            # 3 does not divide Lz, 8 is Lz
        with pytest.raises(dwf.DwfError):
            op.set_sweep("f32", bad)
    op2 = dwf.Operator((4, 2, 4, 4), 4, 1.8, 0.02, 1.5, 0.5)
    with pytest.raises(dwf.DwfError):     # 1 z-plane = 4 sites: not a multiple of 32
        op2.set_sweep("f32", 1)
    op.set_sweep("f32", -1)
    assert op.sweep("f32") == 0
    op.set_sweep("f32", -2)               # automatic: a t-slice of this lattice fits the budget
    assert op.sweep("f32") == 0
    w = (32, 32, 32, 8)
    op3 = dwf.Operator(w, 16, 1.8, 0.02, 1.5, 0.5)
    op3.set_sweep("f32", -2)              # a z-plane pair of 32x32 at Ls 16 in FP32: 1.9 MB
    assert op3.sweep("f32") == 8
    assert op3.sweep("f16") == 0


@pytest.mark.parametrize("limit_ns", [0, 1000, 200000])
def test_bounded_wait_that_runs_out_is_reported(limit_ns):
    """A bounded device wait on a flag that nothing sets (dwf_wait_probe) gives
    up after its limit and records it like every bounded wait of the library:
    the next status check reports DWF_ETIMEOUT once, and the context stays
    usable (the operator still matches the oracle)."""
    from paper_2602_14454_gb300 import dwf
    dims, Ls = (2, 2, 2, 4), 4
    op, ref = make_pair(dims, Ls, 1.8, 0.1, 1.0, 0.0, "standard", 1.0, seed=97)
    op.device_status()
    op.wait_probe(limit_ns)
    with pytest.raises(dwf.DwfError) as e:
        op.device_status()
    assert e.value.status == 6
    op.device_status()   # the report cleared the flag
    x = inputs.gaussian_5d(dims, Ls, 98)
    assert rel(to_np(op.apply(to_gpu(x), op="full", prec="f64")), ref.apply(x)) < 1e-12
    with pytest.raises(dwf.DwfError):
        op.wait_probe(-1)
