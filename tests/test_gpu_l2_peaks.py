"""The L2 ceilings that the transport kernel's L2 roofline is reported against
(dpm_diag_l2_peaks): argument checks and physically plausible magnitudes."""
import numpy as np
import pytest

from paper_0910_0329_gb300 import dpm

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("ws", [0, 1 << 19, (1 << 20) + 8, 1 << 27])
def test_rejects_bad_sizes(tables_ctx, ws):
    with pytest.raises(dpm.DpmError):
        dpm.dpm_diag_l2_peaks(tables_ctx.ctx, ws)


def test_plausible_and_repeatable(tables_ctx):
    a1, r1 = dpm.dpm_diag_l2_peaks(tables_ctx.ctx, 16 << 20)
    a2, r2 = dpm.dpm_diag_l2_peaks(tables_ctx.ctx, 16 << 20)
    # one 64-bit atomic per L2 slice and clock is of order 1e11/s on a GPU
    # of this size; an L2 sweep runs at several TB/s
    for a in (a1, a2):
        assert 1e9 < a < 1e13
    for r in (r1, r2):
        assert 1e11 < r < 1e15
    assert abs(a1 - a2) / a1 < 0.25 and abs(r1 - r2) / r1 < 0.25
    # the context stays usable
    dpm.dpm_sync(tables_ctx.ctx)


def test_atomic_replay_arguments_and_contention(tables_ctx):
    ctx = tables_ctx.ctx
    with pytest.raises(dpm.DpmError):
        dpm.dpm_diag_atomic_replay(ctx, np.array([5], np.uint32), 5)  # id out of range
    with pytest.raises(dpm.DpmError):
        dpm.dpm_diag_atomic_replay(ctx, np.zeros(0, np.uint32), 5)
    n = 1 << 22
    spread = dpm.dpm_diag_atomic_replay(ctx, np.random.default_rng(1).integers(0, 1 << 20, n, dtype=np.uint32), 1 << 20)
    hot = dpm.dpm_diag_atomic_replay(ctx, np.full(n, 7, np.uint32), 1 << 20)
    # one address serialises at its L2 slice: far below the scattered rate
    assert 1e9 < spread < 1e13 and hot < 0.5 * spread
