"""Tomographic abundance matching on the GPU against the FP64 oracle, through the C ABI.

The oracle takes the GPU's own FP32 intensities for each interval, so the
comparison isolates the masking, ranking, matching and per-interval
acceptance; z_re may then differ by > 1e-3 in at most 1e-4 of the cells.
"""
import numpy as np
import pytest
import torch

from oracle import amber_oracle as O
from paper_2109_10375_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import __graft_entry__ as g
    g.build()
    from paper_2109_10375_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def ctx(B):
    c = B.Context(64 ** 3)
    yield c
    c.close()


def test_one_source_in_every_interval_is_the_plain_solve(ctx, B):
    # exact fixed-point prefix sums: ranking the ionized cells first, in any
    # order, changes no later cell's cumulative mass
    n, box = 64, 100.0
    S, m = synth.realisation(n, box, 0, device="cuda")
    h = B.history(8.0, 4.0, 3.0)
    plain = ctx.solve(S, m, box, 3.0, h)
    plain_passes = ctx.sort_passes()
    z = ctx.solve_tomographic([S, S, S], [20.0, 9.0, 7.5, 5.0], m, box, 3.0, h)
    assert ctx.sync_status() == 0
    assert torch.equal(z, plain)
    # the ionized cells' intensity (one float above the interval's largest)
    # widens the key range by one key: the last ranking needs no extra digit pass
    assert ctx.sort_passes() == plain_passes


def test_tomographic_vs_oracle(ctx, B):
    n, box, l = 64, 100.0, 3.0
    S0, m = synth.realisation(n, box, 0, device="cuda")
    S1, _ = synth.realisation(n, box, 1, device="cuda")
    # sources that drift from one interval to the next
    srcs = [S0, (0.6 * S0 + 0.4 * S1).contiguous(), (0.2 * S0 + 0.8 * S1).contiguous()]
    bounds = [20.0, 8.6, 7.2, 5.0]
    h = B.history(8.0, 4.0, 3.0)
    z = ctx.solve_tomographic(srcs, bounds, m, box, l, h)
    assert ctx.sync_status() == 0
    Js = [ctx.radiation_field(s, box, l).cpu().numpy().reshape(-1).astype(np.float64) for s in srcs]
    t = O.history_table(8.0, 4.0, 3.0)
    mo = m.cpu().numpy().reshape(-1).astype(np.float64)
    zo = O.assign_zre_tomographic(Js, bounds, mo, t)
    d = np.abs(z.cpu().numpy().reshape(-1).astype(np.float64) - zo)
    assert np.mean(d > 1e-3) <= 1e-4, (np.mean(d > 1e-3), d.max())
    assert not np.any(np.isnan(z.cpu().numpy()))


def test_tomographic_rejects_bad_bounds(ctx, B):
    S = torch.ones((16, 16, 16), device="cuda")
    h = B.history(8.0, 4.0, 3.0)
    for bounds in ([20.0, 20.0, 5.0], [5.0, 20.0, 7.0], [20.0, 5.0, 7.0, 1.0]):
        with pytest.raises(B.AmberError):
            ctx.solve_tomographic([S, S], bounds, S, 10.0, 1.0, h)
