"""fr_rhs_host: the host-buffer RHS, pipelined over element slabs (copies in
both directions and the kernels on three streams), gives the same R as
fr_rhs on device buffers, bit for bit, through the C ABI."""
import numpy as np
import pytest

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


# slab counts 2, 3 and 4; ragged element counts; both precisions; a mesh
# too small to pipeline (one slab)
CASES = [((64, 4), 2, 32), ((64, 5), 2, 64), ((9, 8, 7), 1, 32), ((97, 40), 3, 32),
         ((20, 6, 30), 2, 32), ((16, 16, 16), 3, 64), ((5, 4, 3), 3, 32)]


@pytest.mark.parametrize("n,order,precision", CASES)
def test_host_buffer_rhs_equals_device_rhs(abi, n, order, precision):
    d = len(n)
    nv = 1 + d + d * d
    U, mesh, prm, lo, hi = parity.make_case(n, order)
    ctx = abi.fr_create(n, lo, hi, order, nv, prm.zeta, prm.nu, prm.T, precision, 0)
    try:
        Ud = abi.pack_state(ctx, U, precision)
        Rd = abi.new_state(ctx, precision, fill=float("nan"))
        abi.fr_rhs(ctx, Ud, Rd)
        Uh = Ud.cpu().pin_memory()
        Rh = torch.full_like(Uh, float("nan")).pin_memory()
        for _ in range(2):                 # the second call reuses the pipeline
            abi.fr_rhs_host(ctx, Uh, Rh)
        torch.cuda.synchronize()
        stride, ne, _ = abi.fr_layout(ctx)
        assert torch.equal(Rh[:, :ne], Rd[:, :ne].cpu())
    finally:
        abi.fr_destroy(ctx)
