"""The C ABI library loads on a CPU-only host and exports every entry point
that include/gcdf.h declares; the Python binding declares the same set."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gcdf.h")).read()
    return sorted(set(re.findall(r"GCDF_API\s+[\w\s\*]+?\b(gcdf_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("gcdf_create_net", "gcdf_destroy_net", "gcdf_query", "gcdf_collision_cost",
                 "gcdf_last_error", "gcdf_weight_count"):
        assert must in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2601_18548_gb300 import _lib
    lib = ctypes.CDLL(_lib.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert sorted(_lib.SIGNATURES) == declared_functions()


def test_weight_count_and_argument_errors_without_gpu():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2601_18548_gb300 as g
    import synth
    for (n, H, L) in ((9, 256, 4), (10, 512, 5), (3, 64, 2)):
        assert g.weight_count(n, H, L) == synth.NetShape(n, H, L).n_params()
    lib = g._lib.load()
    # invalid shapes are rejected before any CUDA call
    d = g._lib.NetDesc(2, 256, 4, 0)
    assert lib.gcdf_weight_count(ctypes.byref(d)) == 0
    out = ctypes.c_void_p()
    rc = lib.gcdf_create_net(ctypes.byref(d), None, 0, ctypes.byref(out))
    assert rc == g._lib.GCDF_EINVAL
    assert "n_dof" in g.last_error()
    rc = lib.gcdf_query(None, None, 1, None, 1, None, None, 0, None, None, None, None)
    assert rc == g._lib.GCDF_EINVAL


def test_fit_argument_errors_without_gpu():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2601_18548_gb300 as g
    lib = g._lib.load()
    # precision other than FP32 / BF16, bad shapes and a negative batch are
    # rejected before any CUDA call
    for desc in ((9, 256, 4, g._lib.GCDF_FP8), (9, 256, 4, 7), (2, 256, 4, 0), (9, 0, 4, 1), (9, 256, 17, 1)):
        d = g._lib.FitDesc(*desc)
        assert lib.gcdf_fit_forward(ctypes.byref(d), None, None, None, 0, None, None) == g._lib.GCDF_EINVAL
        assert lib.gcdf_fit_vjp2(ctypes.byref(d), None, None, None, 0, None, None, None, None) == g._lib.GCDF_EINVAL
    d = g._lib.FitDesc(9, 256, 4, g._lib.GCDF_BF16)
    assert lib.gcdf_fit_value_grad(ctypes.byref(d), None, None, None, -1, None, None, None) == g._lib.GCDF_EINVAL
    assert lib.gcdf_fit_device_status(None) == g._lib.GCDF_EINVAL
    with pytest.raises(ValueError):
        g._fit_desc((9, 256, 4), "fp16")
    # the tape: BF16 only, a size output, an aligned and large enough buffer
    n = ctypes.c_size_t(0)
    fp32 = g._lib.FitDesc(9, 256, 4, g._lib.GCDF_FP32)
    assert lib.gcdf_fit_tape_bytes(ctypes.byref(fp32), 1000, ctypes.byref(n)) == g._lib.GCDF_EINVAL
    assert lib.gcdf_fit_tape_bytes(ctypes.byref(d), 1000, None) == g._lib.GCDF_EINVAL
    assert lib.gcdf_fit_tape_bytes(ctypes.byref(d), 1000, ctypes.byref(n)) == g._lib.GCDF_OK
    # transposed images of v (d_in = 19 rows) and h_1..h_3 (row length: the batch padded to a
    # multiple of 8), s' of 4 layers and h_L, each part rounded up to 256 bytes
    expect = sum(((b + 255) // 256) * 256 for b in [19 * 1000 * 2] + [256 * 1000 * 2] * 3 + [1000 * 256 * 4] * 5)
    assert n.value == expect
    assert lib.gcdf_fit_tape_bytes(ctypes.byref(d), 0, ctypes.byref(n)) == g._lib.GCDF_OK and n.value == 0
    fake = ctypes.c_void_p(1 << 20)  # aligned, never dereferenced
    rc = lib.gcdf_fit_forward_tape(ctypes.byref(d), fake, fake, fake, 1000, fake, None, 1 << 30, None)
    assert rc == g._lib.GCDF_EINVAL and "tape" in g.last_error()
    rc = lib.gcdf_fit_forward_tape(ctypes.byref(d), fake, fake, fake, 1000, fake, fake, 100, None)
    assert rc == g._lib.GCDF_EINVAL and "needed" in g.last_error()
    rc = lib.gcdf_fit_vjp_tape(ctypes.byref(fp32), fake, fake, fake, 1000, fake, fake, 1 << 30, fake, None, None)
    assert rc == g._lib.GCDF_EINVAL


def test_host_side_argument_checks_without_gpu():
    """Every entry point rejects bad arguments before any CUDA call (the fake
    pointers below are non-NULL and aligned but never dereferenced)."""
    import __graft_entry__
    __graft_entry__.build()
    import paper_2601_18548_gb300 as g
    L = g._lib
    lib = L.load()
    fake = ctypes.c_void_p(1 << 20)
    # partition: negative or NaN radius, negative sizes, NULL / misaligned pointers
    for r in (-1.0, float("nan")):
        assert lib.gcdf_partition_offsets(fake, 4, fake, 4, r, fake, None) == L.GCDF_EINVAL
    assert lib.gcdf_partition_offsets(fake, -1, fake, 4, 1.0, fake, None) == L.GCDF_EINVAL
    assert lib.gcdf_partition_offsets(None, 4, fake, 4, 1.0, fake, None) == L.GCDF_EINVAL
    assert lib.gcdf_partition_indices(fake, 4, ctypes.c_void_p((1 << 20) + 4), 4, 1.0, fake, fake,
                                      None) == L.GCDF_EINVAL
    # Jacobian scatter: n_dof outside 1..12, negative sizes, 2 N n past 2^31 - 1
    for (N, n, P) in ((4, 0, 4), (4, 13, 4), (-1, 9, 4), (4, 9, -1), (1 << 30, 9, 1)):
        assert lib.gcdf_jacobian_scatter(fake, N, n, None, 4, P, fake, fake, fake, None) == L.GCDF_EINVAL
    # planner and server
    prm = L.PlanParams(0.1, 1.0, 0.5, 100.0, 1.0, 0.05, 1.0, 1e-6, 1e8, 50, 0.0)
    assert lib.gcdf_plan_solve(None, None, 0, ctypes.byref(prm), fake, None, None, None) == L.GCDF_EINVAL
    out = ctypes.c_void_p()
    assert lib.gcdf_server_create(None, ctypes.byref(out)) == L.GCDF_EINVAL
    for bad in (dict(dt=0.0), dict(iterations=-1), dict(partition_radius=-1.0), dict(lambda_max=1e-9),
                dict(delta=float("nan"))):
        p2 = L.PlanParams(0.1, 1.0, 0.5, 100.0, 1.0, 0.05, 1.0, 1e-6, 1e8, 50, 0.0)
        for k, v in bad.items():
            setattr(p2, k, v)
        d = L.ServerDesc(1 << 30, 4, 16, p2)
        assert lib.gcdf_server_create(ctypes.byref(d), ctypes.byref(out)) == L.GCDF_EINVAL, bad
    for (budget, act, queued) in ((0, 4, 16), (1 << 30, 0, 16), (1 << 30, 4, -1)):
        d = L.ServerDesc(budget, act, queued, prm)
        assert lib.gcdf_server_create(ctypes.byref(d), ctypes.byref(out)) == L.GCDF_EINVAL
    t = ctypes.c_uint64()
    assert lib.gcdf_plan_submit(None, None, ctypes.byref(t)) == L.GCDF_EINVAL
    assert lib.gcdf_plan_poll(None, 1, None) == L.GCDF_EINVAL
    assert lib.gcdf_plan_request_bytes(None, 10, 10) == 0
    assert lib.gcdf_server_destroy(None) == L.GCDF_OK
    assert lib.gcdf_project(None, fake, 1, fake, 1, None, None, 0, None, None, fake, None) == L.GCDF_EINVAL


def test_diagnostic_entry_points_check_their_arguments_without_gpu():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2601_18548_gb300 as g
    lib = g._lib.load()
    seen = (ctypes.c_int * 3)()
    assert lib.gcdf_selftest_wait_expiry(None, 100000, seen) == g._lib.GCDF_EINVAL
    assert lib.gcdf_diag_fp32_fma(0, 256, 10, None, None) == -g._lib.GCDF_EINVAL
    assert lib.gcdf_diag_fp32_fma(4, 100, 10, None, None) == -g._lib.GCDF_EINVAL
    assert "FMA" in g.last_error()
