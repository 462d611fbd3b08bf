"""The log-determinant entry point that allocates nothing.

stiles_logdet_tiles_noalloc serves callers that cannot allocate device
memory (a process whose HBM budget is owned by its own pool, or code where a
cudaMalloc would block the device or is not allowed).  It reads factor tiles
the caller already holds and reduces into a fixed static array inside the
library.  This test calls it through the C ABI twice in a row and compares
each result with stiles_logdet on the same factor.
"""
import ctypes
import math

import numpy as np
import pytest

from paper_2501_02483_b300 import build, inputs
from paper_2501_02483_b300 import stiles as st

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def _noalloc():
    L = st.lib()
    fn = L.stiles_logdet_tiles_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                   ctypes.c_void_p]
    fn.restype = ctypes.c_int32
    return fn


@pytest.mark.parametrize("maker,T", [(lambda: inputs.config_small(0), 64),
                                     (lambda: inputs.band_arrow(6000, 25, 40, 0.3, 3), 32)])
def test_noalloc_logdet_matches_stiles_logdet_twice(maker, T):
    build.build_library()
    fn = _noalloc()
    m = maker()
    plan = st.Plan.from_matrix(m, tile=T)
    f = st.Factor(plan)
    f.factorize(torch.from_numpy(m["values"]).cuda())
    ref = f.logdet()
    info = plan.info()
    tiles = torch.empty((info["nnzt"], T, T), dtype=torch.float64, device="cuda")
    f.tiles(out=tiles)
    tc, _ = plan.tilemap()
    tcol = torch.from_numpy(tc).cuda()
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        out.fill_(math.nan)
        status = fn(tiles.data_ptr(), tcol.data_ptr(), m["n"], T, out.data_ptr(), stream)
        assert status == 0
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - ref) <= 1e-12 * abs(ref), (got, ref)


def test_noalloc_rejects_more_tile_columns_than_its_scratch():
    fn = _noalloc()
    buf = torch.zeros(4, dtype=torch.float64, device="cuda")
    idx = torch.zeros(2, dtype=torch.int64, device="cuda")
    # ceil(n / T) = 65,537 > 65,536 partial sums
    status = fn(buf.data_ptr(), idx.data_ptr(), 65537, 1, buf.data_ptr(), None)
    assert status == 1  # STILES_ERR_INVALID, checked on the host before any launch
    assert np.all(buf.cpu().numpy() == 0)
