"""Source-field pipeline on the GPU (Sec. 3.2, 3.2.1, 3.3) against the FP64 oracle, through the C ABI.

Tolerances: FP32 transforms (relative ~1e-6 of the field's scale per pass,
a few passes deep) and FP32 atomics on the mesh, so fields are compared to
~1e-4 of their own scale; NGP cases keep every particle away from a cell
boundary, where FP32 and FP64 positions could pick different mesh points.
"""
import math

import numpy as np
import pytest
import torch

from oracle import amber_oracle as O

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


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _close(got, ref, rel=1e-4):
    got = np.asarray(got, dtype=np.float64)
    scale = max(np.max(np.abs(ref)), 1e-30)
    assert np.max(np.abs(got - ref)) <= rel * scale, (np.max(np.abs(got - ref)), scale)


@pytest.mark.parametrize("n", [8, 16, 32])
def test_lpt_displacement_vs_oracle(ctx, B, n):
    g = np.random.default_rng(n)
    box = 1.3 * n
    d = g.normal(scale=0.3, size=(n, n, n))
    D1 = 0.9
    D2 = -3.0 / 7.0 * D1 ** 2
    got = ctx.lpt_displacement(_t(d), box, D1, D2)
    assert ctx.sync_status() == 0
    ref = O.lpt_displacement(d.astype(np.float32).astype(np.float64), box, D1, D2)
    for a in range(3):
        _close(got[a].cpu().numpy(), ref[a])


def test_lpt_two_waves_closed_form(ctx, B):
    n, box, A, Bm, D1 = 64, 50.0, 0.4, 0.25, 1.3
    D2 = -3.0 / 7.0 * D1 ** 2
    x = np.arange(n) * box / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    k1, k2 = 2 * np.pi * 2 / box, 2 * np.pi * 5 / box
    got = ctx.lpt_displacement(_t(A * np.cos(k1 * X) + Bm * np.cos(k2 * Y)), box, D1, D2)
    c = A * Bm / (k1 ** 2 + k2 ** 2)
    _close(got[0].cpu().numpy(), -D1 * A * np.sin(k1 * X) / k1 + D2 * c * k1 * np.sin(k1 * X) * np.cos(k2 * Y), 2e-5)
    _close(got[1].cpu().numpy(), -D1 * Bm * np.sin(k2 * Y) / k2 + D2 * c * k2 * np.cos(k1 * X) * np.sin(k2 * Y), 2e-5)
    assert float(got[2].abs().max()) < 1e-5


@pytest.mark.parametrize("order", [1, 2, 3])
@pytest.mark.parametrize("interlace", [False, True])
@pytest.mark.parametrize("weighted", [False, True])
def test_mesh_density_vs_oracle(ctx, B, order, interlace, weighted):
    n, box = 16, 24.0
    g = np.random.default_rng(order * 10 + interlace)
    dx = box / n
    # NGP: displacements in [0.05, 0.45] cells, so no particle of either mesh
    # sits on a cell boundary; CIC and TSC windows are continuous there
    lo, hi = (0.05, 0.45) if order == 1 else (-1.4, 1.4)
    psi = [(g.uniform(lo, hi, (n, n, n)) * dx).astype(np.float32) for _ in range(3)]
    mass = g.uniform(0.2, 3.0, (n, n, n)).astype(np.float32) if weighted else None
    got = ctx.mesh_density(tuple(_t(p) for p in psi), box, order, interlace, mass=_t(mass) if weighted else None)
    assert ctx.sync_status() == 0
    p64 = [p.astype(np.float64) for p in psi]
    m64 = None if mass is None else mass.astype(np.float64)
    r1 = O.mesh_assign(p64, m64, box, order)
    ref = O.interlace_deconvolve(r1, O.mesh_assign(p64, m64, box, order, 0.5), box, order) if interlace else r1
    _close(got.cpu().numpy(), ref, 2e-5)


@pytest.mark.parametrize("order,interlace", [(2, False), (3, True)])
def test_mesh_density_blocks_vs_oracle_64(ctx, B, order, interlace):
    # 64^3: particles whose windows cross the periodic edge and overlap their
    # neighbours' (displacements up to 2.5 cells)
    n, box = 64, 64.0
    g = np.random.default_rng(order + 40)
    psi = [g.uniform(-2.5, 2.5, (n, n, n)).astype(np.float32) for _ in range(3)]
    got = ctx.mesh_density(tuple(_t(p) for p in psi), box, order, interlace)
    assert ctx.sync_status() == 0
    p64 = [p.astype(np.float64) for p in psi]
    r1 = O.mesh_assign(p64, None, box, order)
    ref = O.interlace_deconvolve(r1, O.mesh_assign(p64, None, box, order, 0.5), box, order) if interlace else r1
    _close(got.cpu().numpy(), ref, 2e-5)


@pytest.mark.parametrize("order", [2, 3])
def test_mesh_density_wide_spread_vs_oracle(ctx, B, order):
    # displacements up to 7.5 cells: particles far from their lattice points,
    # windows wrapping the periodic edge, weighted
    n, box = 16, 24.0
    g = np.random.default_rng(order + 50)
    dx = box / n
    psi = [(g.uniform(-7.5, 7.5, (n, n, n)) * dx).astype(np.float32) for _ in range(3)]
    mass = g.uniform(0.2, 3.0, (n, n, n)).astype(np.float32)
    got = ctx.mesh_density(tuple(_t(p) for p in psi), box, order, False, mass=_t(mass))
    assert ctx.sync_status() == 0
    ref = O.mesh_assign([p.astype(np.float64) for p in psi], mass.astype(np.float64), box, order)
    _close(got.cpu().numpy(), ref, 2e-5)


@pytest.mark.parametrize("order", [1, 2, 3])
def test_mesh_density_uniform_lattice_256(B, order):
    # no displacement: every window, with or without interlacing, gives 1
    n = 256
    with B.Context(n ** 3) as c:
        zero = torch.zeros((n, n, n), device="cuda")
        for il in (False, True):
            rho = c.mesh_density((zero, zero, zero), 300.0, order, il)
            assert c.sync_status() == 0
            assert float((rho - 1).abs().max()) < 1e-5


@pytest.mark.parametrize("filt", ["sharpk", "tophat"])
def test_esf_fcoll_vs_oracle(ctx, B, filt):
    n, box = 32, 40.0
    d = np.random.default_rng(7).normal(scale=1.0, size=(n, n, n))
    R, dc, ds2 = 2.1, 1.5, 0.6
    got = ctx.esf_fcoll(_t(d), box, R, dc, ds2, filt)
    assert ctx.sync_status() == 0
    ref = O.fcoll_esf(O.filter_field(d.astype(np.float32).astype(np.float64), box, R, filt), dc, ds2)
    assert np.max(np.abs(got.cpu().numpy() - ref)) < 2e-5


def test_esf_l_halo_density_chain(ctx, B):
    # ESF-L (Sec. 3.3): f_coll in Lagrangian space, the particles carry
    # f_coll m_p to their 2LPT positions, CIC with interlacing
    n = 16
    box = 0.8 * n
    g = np.random.default_rng(11)
    d = g.normal(scale=0.5, size=(n, n, n)).astype(np.float32)
    D1 = 0.1
    D2 = -3.0 / 7.0 * D1 ** 2
    td = _t(d)
    psi = ctx.lpt_displacement(td, box, D1, D2)
    f = ctx.esf_fcoll(td, box, 1.0, 1.686 / D1, 2.0, "sharpk")
    rho_h = ctx.mesh_density(psi, box, 2, True, mass=f)
    assert ctx.sync_status() == 0
    d64 = d.astype(np.float64)
    po = O.lpt_displacement(d64, box, D1, D2)
    fo = O.fcoll_esf(O.filter_field(d64, box, 1.0, "sharpk"), 1.686 / D1, 2.0)
    ref = O.interlace_deconvolve(O.mesh_assign(po, fo, box, 2), O.mesh_assign(po, fo, box, 2, 0.5), box, 2)
    _close(rho_h.cpu().numpy(), ref, 5e-4)


def test_source_pipeline_rejects_bad_arguments(ctx, B):
    z = torch.zeros((8, 8, 8), device="cuda")
    with pytest.raises(B.AmberError):
        ctx.mesh_density((z, z, z), 10.0, 4, True)
    with pytest.raises(B.AmberError):
        ctx.esf_fcoll(z, 10.0, -1.0, 1.0, 1.0)
    with pytest.raises(B.AmberError):
        ctx.lpt_displacement(torch.zeros((128, 128, 128), device="cuda"), 10.0, 1.0, 0.0)  # over capacity
