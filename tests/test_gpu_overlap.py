"""Chains with overlap_proposal = 1 (the proposal's assembly and factorization
on a second stream beside Algorithm 1's draw) against the same chain in serial
order.

The overlapped iteration launches the same kernels with the same sizes on the
same data (W'^-1 f, for q', may run as two launches with the one-launch
arithmetic); only their order across the streams differs, and no kernel of
one stream reads what another writes before they are joined.  So every trace field
(sigma2, tau2, rho, log alpha, acceptances, residuals), the draw f and the
posterior mean must agree bit for bit with the serial chain, in FP64 and in
mixed precision, for a size with CTA groups at the top levels (grouped ACA and
grouped level kernels run outside the overlapped window) and a size without.
fifa_chain_bytes counts the second scratch area exactly.
"""
import math

import numpy as np
import pytest

from paper_2006_06537_gb300.inputs import clustered, uniform_sine
from tests.gpu_util import build_lib, dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

build_lib()
from paper_2006_06537_gb300 import fifa  # noqa: E402


def _chain(x, y, leaf, prec, overlap, rho0, nugget, arena=4 << 30, indep=0):
    ctx = fifa.Context(leaf_size=leaf, aca_tol=1e-10, rank_cap=32, prec=prec, refine_max=8, refine_tol=1e-12,
                       arena_bytes=arena, stream=torch.cuda.Stream(), independent_ctas=indep,
                       overlap_proposal=overlap)
    vy = float(np.var(y))
    pr = fifa.fifa_prior(1.0, 1.0, 1.0, 1.0, math.log(rho0), 1.0, 0.2)
    xd, yd = dev(x, torch), dev(y, torch)
    ch = fifa.fifa_chain_create(ctx.h, xd, yd, len(x), fifa.fifa_hyper(0, vy, rho0, 0.5 * vy, nugget), pr, 5, 3)
    return ctx, ch


def _run(x, y, leaf, prec, overlap, rho0, nugget, iters, indep=0):
    ctx, ch = _chain(x, y, leaf, prec, overlap, rho0, nugget, indep=indep)
    tr = np.zeros((iters, fifa.FIFA_TRACE_FIELDS))
    fifa.fifa_gibbs_step(ctx.h, ch, iters, tr)
    n = len(x)
    f = torch.empty(n, dtype=torch.float64, device="cuda")
    mean = torch.empty(n, dtype=torch.float64, device="cuda")
    fifa.fifa_chain_get(ctx.h, ch, f, mean)
    kn = fifa.fifa_chain_kernel_nodes(ch)
    out = (tr, f.cpu().numpy(), mean.cpu().numpy(), kn)
    fifa.fifa_destroy_chain(ctx.h, ch)
    ctx.close()
    return out


CASES = [
    # clustered recipe with CTA groups at the top levels (ACA and level kernels)
    ("clustered", 65536, 32, 0.01, 1e-6),
    # uniform sine, small: no grouped level, no grouped ACA
    ("sine", 3000, 64, 0.1, 1e-6),
]


@pytest.mark.parametrize("prec", [fifa.FIFA_FP64, fifa.FIFA_MIXED])
@pytest.mark.parametrize("recipe,n,leaf,rho0,nugget", CASES)
def test_overlap_matches_serial_bitwise(recipe, n, leaf, rho0, nugget, prec):
    x, y = clustered(n) if recipe == "clustered" else uniform_sine(n, 4)
    iters = 6
    a = _run(x, y, leaf, prec, 0, rho0, nugget, iters)
    b = _run(x, y, leaf, prec, 1, rho0, nugget, iters)
    assert np.array_equal(a[0].view(np.uint64), b[0].view(np.uint64)), (a[0] - b[0])
    assert np.array_equal(a[1].view(np.uint64), b[1].view(np.uint64))
    assert np.array_equal(a[2].view(np.uint64), b[2].view(np.uint64))
    assert np.all(np.isfinite(b[0]))
    # the overlapped graph has the serial graph's kernels (the propose kernel
    # moved, nothing dropped), plus one where W'^-1 f is split around the
    # grouped levels (two launches of the one-launch sweep's arithmetic)
    assert a[3] > 0 and b[3] in (a[3], a[3] + 1)


def test_overlap_with_independent_ctas():
    """independent_ctas = 1 has no grouped launch at all: the whole proposal runs beside the draw."""
    x, y = uniform_sine(20000, 6)
    a = _run(x, y, 64, fifa.FIFA_FP64, 0, 0.1, 1e-6, 4, indep=1)
    b = _run(x, y, 64, fifa.FIFA_FP64, 1, 0.1, 1e-6, 4, indep=1)
    assert np.array_equal(a[0].view(np.uint64), b[0].view(np.uint64))
    assert np.array_equal(a[1].view(np.uint64), b[1].view(np.uint64))


@pytest.mark.parametrize("prec", [fifa.FIFA_FP64, fifa.FIFA_MIXED])
def test_overlap_chain_bytes_is_exact(prec):
    n = 40000
    x, y = uniform_sine(n, 2)
    o = fifa.fifa_opts(32, 1e-10, 32, prec, 1e-12, 8, 0, 0, 0, 1)
    need = fifa.fifa_chain_bytes(o, n)
    vy = float(np.var(y))
    hy = fifa.fifa_hyper(0, vy, 0.1, 0.5 * vy, 1e-6)
    pr = fifa.fifa_prior(1.0, 1.0, 1.0, 1.0, math.log(0.1), 1.0, 0.2)
    for size, ok in ((need, True), (need - 256, False)):
        ctx = fifa.Context(leaf_size=32, aca_tol=1e-10, rank_cap=32, prec=prec, refine_max=8, refine_tol=1e-12,
                           arena_bytes=size, stream=torch.cuda.Stream(), overlap_proposal=1)
        xd, yd = dev(x, torch), dev(y, torch)
        if ok:
            ch = fifa.fifa_chain_create(ctx.h, xd, yd, n, hy, pr, 0, 0)
            fifa.fifa_gibbs_step(ctx.h, ch, 2)
            fifa.fifa_destroy_chain(ctx.h, ch)
        else:
            with pytest.raises(fifa.FifaError) as e:
                fifa.fifa_chain_create(ctx.h, xd, yd, n, hy, pr, 0, 0)
            assert e.value.code == fifa.FIFA_ERR_OOM
        ctx.close()


def test_overlap_matches_serial_at_full_size():
    """The benchmark's configuration: clustered SE n = 2^20, leaf 32, mixed precision."""
    n = 1 << 20
    x, y = clustered(n, 2, noise=0.05)
    outs = []
    for overlap in (0, 1):
        ctx, ch = _chain(x, y, 32, fifa.FIFA_MIXED, overlap, 0.01, 1e-6, arena=40 << 30)
        tr = np.zeros((3, fifa.FIFA_TRACE_FIELDS))
        fifa.fifa_gibbs_step(ctx.h, ch, 3, tr)
        f = torch.empty(n, dtype=torch.float64, device="cuda")
        fifa.fifa_chain_get(ctx.h, ch, f, None)
        outs.append((tr, f.cpu().numpy()))
        fifa.fifa_destroy_chain(ctx.h, ch)
        ctx.close()
        del ctx
        torch.cuda.empty_cache()
    assert np.array_equal(outs[0][0].view(np.uint64), outs[1][0].view(np.uint64))
    assert np.array_equal(outs[0][1].view(np.uint64), outs[1][1].view(np.uint64))
