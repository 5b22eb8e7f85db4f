"""dwf_spectrum_bounds (FP64 Lanczos on the GPU) against the oracle's dense
spectrum of D^dag D (oracle/spectrum.py, Sec. 3.2 condition number)."""

import numpy as np
import pytest

from _util import make_pair
from paper_2602_14454_gb300 import inputs

pytestmark = pytest.mark.gpu

TINY = (2, 2, 2, 4)


@pytest.fixture(scope="module", autouse=True)
def _built(cuda_ok):
    from paper_2602_14454_gb300 import build
    build.build()


@pytest.mark.parametrize("form,alpha,b,c", [("standard", 1.0, 1.5, 0.5), ("neff", 0.5, 1.5, 0.5),
                                            ("neff", 0.3, 1.0, 1.0), ("standard", 1.0, 1.0, 0.0)])
def test_extremal_eigenvalues_match_the_dense_oracle(form, alpha, b, c):
    from oracle import spectrum
    U = inputs.random_links(TINY, 0.5, 311)
    op, ref = make_pair(TINY, 4, 1.8, 0.05, b, c, form, alpha, U=U)
    lo_ref, hi_ref, _ = spectrum.condition_number(ref)
    lo, hi, steps = op.spectrum_bounds(max_steps=1500, rtol=1e-13, seed=7)
    assert 20 <= steps <= 1500
    assert abs(lo / lo_ref - 1) < 1e-8
    assert abs(hi / hi_ref - 1) < 1e-8


@pytest.mark.parametrize("form,alpha", [("standard", 1.0), ("neff", 0.5), ("neff", 0.3)])
def test_second_even_odd_form_matches_the_dense_oracle(form, alpha):
    """eo_form 1 (eq. another_even-odd_linear_equation): the oracle's spectrum, which
    does not depend on alpha."""
    from oracle import spectrum
    U = inputs.random_links(TINY, 0.5, 311)
    op, ref = make_pair(TINY, 4, 1.8, 0.05, 1.5, 0.5, form, alpha, U=U)
    lo_ref, hi_ref, _ = spectrum.condition_number(ref, eo_form=1)
    lo, hi, steps = op.spectrum_bounds(max_steps=1500, rtol=1e-13, seed=7, eo_form=1)
    assert abs(lo / lo_ref - 1) < 1e-8
    assert abs(hi / hi_ref - 1) < 1e-8


def test_bounds_do_not_depend_on_the_start_vector():
    dims, Ls = (4, 4, 4, 4), 8
    op, ref = make_pair(dims, Ls, 1.8, 0.04, 1.5, 0.5, "neff", 0.5, seed=1001)
    a = op.spectrum_bounds(max_steps=3000, rtol=1e-10, seed=1)
    b = op.spectrum_bounds(max_steps=3000, rtol=1e-10, seed=2)
    assert abs(a[0] / b[0] - 1) < 1e-6 and abs(a[1] / b[1] - 1) < 1e-6
    assert 0 < a[0] < a[1]


def test_bad_arguments():
    from paper_2602_14454_gb300 import dwf
    op, ref = make_pair(TINY, 4, 1.8, 0.05, 1.0, 0.0, "standard", 1.0)
    with pytest.raises(dwf.DwfError) as e:
        op.spectrum_bounds(max_steps=1)
    assert e.value.status == 1
    with pytest.raises(dwf.DwfError):
        op.spectrum_bounds(rtol=0.0)
    with pytest.raises(dwf.DwfError):
        op.spectrum_bounds(eo_form=2)
