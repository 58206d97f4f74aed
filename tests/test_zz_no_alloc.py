"""The allocation-free H-matrix product (fifa_matvec_static) against the
regular one (fifa_matvec), through the C ABI, on two calls in a row.

fifa_matvec_static serves callers that cannot allocate device memory
themselves (a plug-in whose host framework owns the device memory, a process
whose memory a pooling allocator has fully reserved, a loop that must not enter
the allocator).  Its scratch is a static device array shared by all calls, so
the second call also checks that leftovers of the first do not leak into it.
This file is collected last so that a failure here does not stop the rest of
the suite.
"""
import numpy as np
import pytest

from paper_2006_06537_gb300.inputs import uniform_sine
from tests.gpu_util import build_lib, dev, host, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

build_lib()
from paper_2006_06537_gb300 import fifa  # noqa: E402


def test_static_scratch_matvec_matches_regular_matvec():
    n, B = 2048, 64
    x, _ = uniform_sine(n, 0)
    ctx = fifa.Context(leaf_size=B, aca_tol=1e-12, rank_cap=32, arena_bytes=512 << 20)
    C = fifa.fifa_assemble(ctx.h, dev(x, torch), n, fifa.fifa_hyper(0, 1.0, 0.1, 1.0, 1e-8))
    M = fifa.fifa_shift_scale(ctx.h, C, 250.0)
    g = np.random.default_rng(12)
    for A, nrhs in ((C, 2), (M, 1)):  # two calls in a row, different operators and widths
        v = dev(g.standard_normal((nrhs, n)), torch)
        ref = torch.empty_like(v)
        got = torch.full_like(v, float("nan"))
        fifa.fifa_matvec(ctx.h, A, v, ref, nrhs)
        fifa.fifa_matvec_static(ctx.h, A, v, got, nrhs)
        torch.cuda.synchronize()
        assert rel(host(got), host(ref)) <= 1e-13


def test_static_scratch_rejects_sizes_beyond_its_maximum():
    n, B = 1 << 18, 32  # 13 levels: partial sums exceed the 2^20-double array
    x, _ = uniform_sine(n, 1)
    ctx = fifa.Context(leaf_size=B, aca_tol=1e-10, rank_cap=32, arena_bytes=2 << 30)
    C = fifa.fifa_assemble(ctx.h, dev(x, torch), n, fifa.fifa_hyper(0, 1.0, 0.1, 1.0, 1e-6))
    v = torch.zeros(n, dtype=torch.float64, device="cuda")
    out = torch.empty_like(v)
    code = fifa.fifa_matvec_static(ctx.h, C, v, out, 1, allow=(fifa.FIFA_ERR_UNSUPPORTED,))
    assert code == fifa.FIFA_ERR_UNSUPPORTED
