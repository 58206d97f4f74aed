"""Bounded device waits: a CTA waiting for the rest of its group gives up after
fifa_opts.wait_polls polls, records FIFA_ERR_TIMEOUT in the object's status,
raises the launch's abort flag so every other CTA of the launch returns too,
and the host reads the status at the next synchronizing call.  Here a context
with a one-poll limit assembles and factors a problem whose top levels run in
CTA groups (n = 2^17), so the first CTA of a group to reach a barrier gives up
almost at once: the calls must report TIMEOUT, nothing may hang or fault, and
the GPU and the library stay usable (a default context then reproduces the
reference results bit for bit).
"""
import numpy as np
import pytest

from paper_2006_06537_gb300.inputs import clustered
from tests.gpu_util import build_lib, dev, host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

build_lib()
from paper_2006_06537_gb300 import fifa  # noqa: E402

N = 1 << 17


def _assemble_factor(ctx, xd):
    H = fifa.fifa_assemble(ctx.h, xd, N, fifa.fifa_hyper(0, 1.0, 0.01, 1.0, 1e-6))
    F = fifa.fifa_factor(ctx.h, H)
    ld, code_f = fifa.fifa_logdet(ctx.h, F, allow=(fifa.FIFA_ERR_TIMEOUT, fifa.FIFA_ERR_NOT_SPD))
    code_h = fifa.fifa_hmat_export(ctx.h, H, allow=(fifa.FIFA_ERR_TIMEOUT, fifa.FIFA_ERR_RANK_CAP), bases=False,
                                   leaves=False)["status"]
    return H, F, ld, code_h, code_f


def test_group_wait_gives_up_and_reports_timeout():
    x, _ = clustered(N, 2, noise=0.05)
    xd = dev(x, torch)
    ref = fifa.Context(leaf_size=32, aca_tol=1e-10, rank_cap=32, arena_bytes=4 << 30)
    _, _, ld_ref, ch, cf = _assemble_factor(ref, xd)
    assert ch == fifa.FIFA_OK and cf == fifa.FIFA_OK
    # one poll: a group barrier that is not already complete gives up at once
    short = fifa.Context(leaf_size=32, aca_tol=1e-10, rank_cap=32, arena_bytes=4 << 30, wait_polls=1)
    _, _, _, ch, cf = _assemble_factor(short, xd)
    assert fifa.FIFA_ERR_TIMEOUT in (ch, cf), (ch, cf)
    torch.cuda.synchronize()  # no fault, nothing left running
    # the timed-out context still runs kernels correctly
    v = torch.linspace(-5.0, 0.0, 1000, dtype=torch.float64, device="cuda")
    out = torch.empty_like(v)
    fifa.fifa_det_exp(short.h, v, out, 1000)
    torch.cuda.synchronize()
    assert np.allclose(host(out), np.exp(host(v)), rtol=1e-15, atol=0)
    short.close()
    # and a default context reproduces the reference bit for bit
    again = fifa.Context(leaf_size=32, aca_tol=1e-10, rank_cap=32, arena_bytes=4 << 30)
    _, _, ld2, ch, cf = _assemble_factor(again, xd)
    assert ch == fifa.FIFA_OK and cf == fifa.FIFA_OK and ld2 == ld_ref
    again.close()
    ref.close()
