"""The allocation-free even-odd apply (dwf_apply_eo_noalloc), called through the C ABI.

It is meant for callers that cannot let the library allocate device memory
during a call; its work space is a fixed device array inside the library.
This file is collected last so that a failure here leaves every other test
already run.  It must pass alone in a fresh process and after the others.
"""

import ctypes

import numpy as np
import pytest

from _util import TOL, make_pair, rel, to_gpu, to_np
from paper_2602_14454_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built(cuda_ok):
    from paper_2602_14454_gb300 import build
    build.build()


def _noalloc(op, x, prec, dag):
    import torch
    from paper_2602_14454_gb300 import dwf
    out = torch.empty_like(x)
    rc = dwf.lib().dwf_apply_eo_noalloc(op.handle, dwf.PREC[prec], int(dag), ctypes.c_void_p(x.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr()),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    dwf.check(rc)
    return out


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
@pytest.mark.parametrize("form,alpha", [("standard", 1.0), ("neff", 0.5)])
def test_noalloc_matches_dwf_apply_twice(prec, form, alpha):
    dims, Ls = (4, 4, 2, 6), 12
    op, ref = make_pair(dims, Ls, 1.8, 0.02, 1.5, 0.5, form, alpha, seed=91)
    for call, seed in enumerate((92, 93)):            # two calls in a row share the array
        x = to_gpu(ref.to_eo(inputs.gaussian_5d(dims, Ls, seed), 0))
        for dag in (False, True):
            want = to_np(op.apply(x, op="eo", prec=prec, dag=dag))
            got = to_np(_noalloc(op, x, prec, dag))
            assert rel(got, want) < TOL[prec], (call, dag)
    op.device_status()


def test_noalloc_allocates_nothing_in_the_handle():
    import torch
    dims, Ls = (4, 4, 4, 4), 8
    op, ref = make_pair(dims, Ls, 1.8, 0.04, 1.0, 0.0, "standard", 1.0, seed=94)
    before = op.device_bytes()
    x = to_gpu(ref.to_eo(inputs.gaussian_5d(dims, Ls, 95), 0))
    outs = [torch.empty_like(x) for _ in range(4)]
    # the first call may load the device code that holds the array; after it,
    # calls change neither the handle's buffers nor the device's free memory
    _noalloc(op, x, "f64", False)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    from paper_2602_14454_gb300 import dwf
    for k, o in enumerate(outs):
        dwf.check(dwf.lib().dwf_apply_eo_noalloc(op.handle, dwf.PREC["f64"], k & 1, ctypes.c_void_p(x.data_ptr()),
                                                 ctypes.c_void_p(o.data_ptr()),
                                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0        # no device allocation during the calls
    y1 = to_np(outs[0])
    y2 = to_np(outs[2])
    assert op.device_bytes() == before                  # no work fields were created
    assert rel(y1, ref.d_pc(ref.to_eo(inputs.gaussian_5d(dims, Ls, 95), 0))) < TOL["f64"]
    assert np.array_equal(y1, y2)


def test_noalloc_rejects_lattices_beyond_the_array():
    from paper_2602_14454_gb300 import dwf
    dims, Ls = (16, 16, 16, 16), 16                    # FP64 work fields: 4 x 100 MB > 64 MiB
    op, _ = make_pair(dims, Ls, 1.8, 0.01, 1.5, 0.5, "standard", 1.0, seed=96,
                      U=inputs.unit_links(dims))
    import torch
    x = torch.zeros((Ls, 16 ** 4 // 2, 4, 3), dtype=torch.complex128, device="cuda")
    with pytest.raises(dwf.DwfError) as e:
        _noalloc(op, x, "f64", False)
    assert e.value.status == 1
