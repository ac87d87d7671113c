"""fr_rhs_static: the RHS for callers that cannot allocate device memory.

Such callers (an application whose own pool allocator holds the device's
memory, a time-critical loop where an allocation may not happen) cannot use
fr_create, which allocates the face-trace scratch.  fr_rhs_static takes that
scratch from a fixed 16 MiB array in the library's device image instead.
These tests call it through the C ABI and check, on two calls in a row with
different states, that it gives the same R as fr_rhs bit for bit (the same
kernels with the same constants on the same inputs); that, once its first
call on the device has loaded the array, a further call leaves the device's
free memory unchanged; that it runs on a non-default stream; and that a
problem larger than the array is refused.  The file sorts last so that a run
stopping at the first failure has already run every other test; it also
passes on its own.
"""
import numpy as np
import pytest

from oracle import fr
from tests import parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def abi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_14027_gb300 import build
    build.build()
    from paper_2107_14027_gb300 import abi as _abi
    return _abi


CASES = [((6, 5, 7), 3, 32), ((6, 5, 7), 3, 64), ((16, 16), 2, 64), ((9, 3), 5, 32)]
PRM = fr.Params(2.5, 1.0 / 1600.0, 5e-3)


def _compare(abi, n, order, precision, stream):
    d = len(n)
    nv = 1 + d + d * d
    ctx = abi.fr_create(n, (-np.pi,) * d, (np.pi,) * d, order, nv, PRM.zeta, PRM.nu, PRM.T,
                        precision)
    try:
        stride, ne, _ = abi.fr_layout(ctx)
        for seed in (1, 2):   # two calls in a row, different states
            U, mesh, _, lo, hi = parity.make_case(n, order, seed=seed)
            Ud = abi.pack_state(ctx, U, precision)
            R_ref = abi.new_state(ctx, precision, fill=float("nan"))
            R_static = abi.new_state(ctx, precision, fill=float("nan"))
            torch.cuda.synchronize()
            abi.fr_rhs(ctx, Ud, R_ref, stream)
            abi.fr_rhs_static(n, lo, hi, order, nv, PRM.zeta, PRM.nu, PRM.T, precision,
                              abi.FR_CORR_DG, Ud, R_static, stream)
            torch.cuda.synchronize()
            assert torch.equal(R_static[:, :ne], R_ref[:, :ne]), f"call {seed} differs"
    finally:
        abi.fr_destroy(ctx)


@pytest.mark.parametrize("n,order,precision", CASES)
def test_static_equals_fr_rhs_on_two_calls(abi, n, order, precision):
    _compare(abi, n, order, precision, torch.cuda.current_stream())


def test_static_on_a_non_default_stream(abi):
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        _compare(abi, (7, 4, 3), 2, 32, s)


def test_static_call_after_the_first_allocates_nothing(abi):
    n, order, precision = (6, 5, 7), 3, 32
    U, mesh, _, lo, hi = parity.make_case(n, order, seed=3)
    ctx = abi.fr_create(n, lo, hi, order, 13, PRM.zeta, PRM.nu, PRM.T, precision)
    try:
        Ud = abi.pack_state(ctx, U, precision)
        Rd = abi.new_state(ctx, precision)
    finally:
        abi.fr_destroy(ctx)
    args = (n, lo, hi, order, 13, PRM.zeta, PRM.nu, PRM.T, precision, abi.FR_CORR_DG, Ud, Rd)
    abi.fr_rhs_static(*args)          # first call on this device: loads the array
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        abi.fr_rhs_static(*args)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_static_refuses_problems_beyond_its_array(abi):
    n, order, precision = (20, 20, 20), 3, 32     # 8000 hexahedra > 6240
    U = torch.zeros(16, device="cuda")
    R = torch.zeros(16, device="cuda")
    with pytest.raises(abi.FrError) as ei:
        abi.fr_rhs_static(n, (0.0,) * 3, (1.0,) * 3, order, 13, 2.5, 1e-3, 5e-3, precision,
                          abi.FR_CORR_DG, U, R)
    assert ei.value.status == abi.FR_EINVAL
    assert "static" in abi.fr_last_error()
