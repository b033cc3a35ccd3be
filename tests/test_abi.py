"""Host-side checks of libamber (no GPU): symbols, the Weibull solve, argument errors."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def B():
    import __graft_entry__ as g
    g.build()
    from paper_2109_10375_gb300 import binding
    return binding


def _declared():
    src = open(os.path.join(ROOT, "include", "amber.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(amber_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(B):
    names = _declared()
    assert len(names) >= 18
    for name in names:
        assert hasattr(B.lib, name), name
    assert set(names) == set(B.EXPORTED)


def test_host_weibull_matches_table1(B):
    with open(os.path.join(ROOT, "tests", "golden", "weibull_table1.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for name, *v in rows:
        z_mid, dz, Az, a_w, b_w, c_w = map(float, v)
        a, b, c = B.history_coeffs(B.history(z_mid, dz, Az))
        assert abs(a - a_w) <= 0.01 and abs(b - b_w) <= 0.01 and abs(c - c_w) <= 0.01, name


@pytest.mark.parametrize("p", [(8, 4, 3), (7.5, 4, 3), (6.5, 6, 1.5), (9, 2, 5), (8, 4, 14), (8, 2, 2)])
def test_host_history_table_matches_oracle(B, p):
    from oracle import amber_oracle as o
    z, x = B.history_table(B.history(*p))
    t = o.history_table(*p)
    np.testing.assert_allclose(z, t.z, rtol=0, atol=1e-12)
    np.testing.assert_allclose(x, t.x, rtol=0, atol=1e-12)
    a, b, c = B.history_coeffs(B.history(*p))
    assert abs(a - t.a_w) < 1e-10 and abs(b - t.b_w) < 1e-10 and abs(c - t.c_w) < 1e-10


def test_host_history_rejects_bad_arguments(B):
    h = B.history(8, 4, 3)
    h.x_ear, h.x_mid = 0.6, 0.5
    out = (C.c_double * 3)()
    assert B.lib.amber_history_coeffs(C.byref(h), out) == B.AMBER_ERR_INVALID_ARG
    h = B.history(8, -4, 3)
    assert B.lib.amber_history_coeffs(C.byref(h), out) == B.AMBER_ERR_INVALID_ARG
    h = B.history(8, 4, 3, n_table=1)
    assert B.lib.amber_history_coeffs(C.byref(h), out) == B.AMBER_ERR_INVALID_ARG


def test_entry_points_reject_null_context(B):
    vp = C.c_void_p
    assert B.lib.amber_radiation_field(None, vp(16), 64, 1.0, 1.0, vp(16), None) == B.AMBER_ERR_INVALID_ARG
    assert B.lib.amber_rank(None, vp(16), 10, vp(16), None) == B.AMBER_ERR_INVALID_ARG
    assert B.lib.amber_sync_status(None, None) == B.AMBER_ERR_INVALID_ARG
    assert B.status_string(B.AMBER_ERR_NONFINITE) == "non-finite intensity"


def test_workspace_plan(B):
    # 1024^3: half spectrum (4 B/cell), six 4 B/cell sort buffers, two
    # 9-bit look-back regions (1 B/cell) and the bucket table, allocated once
    wb = B.workspace_bytes(1 << 30)
    assert 29e9 < wb < 33e9
    with pytest.raises(B.AmberError):
        B.workspace_bytes((1 << 30) + 1)


def test_create_without_gpu_reports_cuda_error(B):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    assert B.lib.amber_create(C.byref(h), 0, 4096) == B.AMBER_ERR_CUDA


def test_sigma2_tophat_host_matches_oracle():
    # Eq. variance on a tabulated power law (host FP64, no GPU)
    import numpy as np
    from oracle import amber_oracle as O
    from paper_2109_10375_gb300 import binding as B
    k = np.geomspace(1e-3, 1e3, 4001)
    D2 = 0.3 * (k / 1.0) ** 1.5 * np.exp(-k / 50.0)
    for R in (0.2, 0.5, 2.0):
        assert abs(B.sigma2_tophat(k, D2, R) / O.sigma2_tophat(k, D2, R) - 1.0) < 1e-9


def test_noalloc_rejects_pointers_off_their_element_size(B):
    # the argument checks run before any CUDA call, so nothing is enqueued and
    # no device is needed: a float array must start on a multiple of 4 bytes
    vp = C.c_void_p
    assert B.lib.amber_rank_noalloc(vp(0x1002), 64, vp(0x2000), None, None) == B.AMBER_ERR_INVALID_ARG
    assert B.lib.amber_rank_noalloc(vp(0x1000), 64, vp(0x2001), None, None) == B.AMBER_ERR_INVALID_ARG
    assert B.lib.amber_rank_noalloc(vp(0x1000), 64, vp(0x2000), vp(0x3002), None) == B.AMBER_ERR_INVALID_ARG
    assert B.lib.amber_rank_noalloc(vp(0x1000), 0, vp(0x2000), None, None) == B.AMBER_ERR_INVALID_ARG


def test_binding_rejects_non_contiguous_tensors(B):
    import torch
    t = torch.zeros(8, 8)[:, ::2]
    with pytest.raises(ValueError):
        B._ptr(t)
    assert B._ptr(torch.zeros(4)) is not None and B._ptr(None) is None


def test_ctypes_structs_match_the_compiled_layout(B):
    # the binding's copies of the public structs against sizeof and offsetof
    # as the library was compiled (host-only call: no CUDA, no context)
    import ctypes as C
    for which, cls in enumerate([B.amber_history_t, B.amber_params_t, B.amber_tuning_t, B.amber_batch_item]):
        size, count = C.c_size_t(), C.c_int()
        offs = (C.c_size_t * 16)()
        assert B.lib.amber_struct_layout(which, C.byref(size), offs, 16, C.byref(count)) == 0
        fields = [f[0] for f in cls._fields_]
        assert size.value == C.sizeof(cls), cls.__name__
        assert count.value == len(fields), cls.__name__
        assert list(offs[:count.value]) == [getattr(cls, f).offset for f in fields], cls.__name__
    size, count = C.c_size_t(), C.c_int()
    assert B.lib.amber_struct_layout(4, C.byref(size), None, 0, C.byref(count)) != 0
    assert B.lib.amber_struct_layout(0, None, None, 0, C.byref(count)) != 0
