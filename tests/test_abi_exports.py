"""The C-ABI library builds, loads without a GPU, and exports every declared symbol."""
import ctypes

from tests import _util


def test_every_declared_symbol_is_exported():
    nv = _util.native()
    names = _util.declared_functions()
    assert len(names) >= 8
    lib = nv.lib()
    for name in names:
        assert hasattr(lib, name), name
        assert name in nv.SIGNATURES, f"binding lacks {name}"


def test_binding_names_are_declared():
    nv = _util.native()
    declared = set(_util.declared_functions())
    for name in nv.SIGNATURES:
        assert name in declared, f"binding exports undeclared {name}"


def test_argument_errors_need_no_gpu():
    nv = _util.native()
    lib = nv.lib()
    assert lib.zkvc_version() >= 100
    assert lib.zkvc_ntt(None, 4, 0, None) == nv.ZKVC_EINVAL
    assert b"null" in lib.zkvc_last_error()
    assert lib.zkvc_ntt(ctypes.c_void_p(16), 4, 9, None) == nv.ZKVC_EINVAL
    assert lib.zkvc_fr_mul(None, None, None, 4, None) == nv.ZKVC_EINVAL
    assert lib.zkvc_fr_inv(None, None, 4, None) == nv.ZKVC_EINVAL
    assert lib.zkvc_fp_inv(None, None, 4, None) == nv.ZKVC_EINVAL
    assert lib.zkvc_fp_inv(None, None, 0, None) == nv.ZKVC_OK  # n = 0: nothing to do
    t0, t1 = ctypes.c_double(), ctypes.c_double()
    assert lib.zkvc_profile_span(-1, ctypes.byref(t0), ctypes.byref(t1)) == nv.ZKVC_EINVAL
    assert lib.zkvc_profile_span(1 << 20, None, None) == nv.ZKVC_EINVAL
    assert lib.zkvc_profile_span(0, ctypes.byref(t0), ctypes.byref(t1)) == nv.ZKVC_OK
    out = (ctypes.c_uint8 * 64)()
    assert lib.zkvc_msm_g1(None, None, 0, None, 0, out, None) == nv.ZKVC_OK   # n = 0: infinity
    assert bytes(out) == bytes(64)
    assert lib.zkvc_msm_workspace_bytes(1000, 1) > 1000 * 64
    assert lib.zkvc_msm_workspace_bytes(1000, 2) > lib.zkvc_msm_workspace_bytes(1000, 1)


def test_msm_plans_fit_on_the_host():
    """The variable-base MSM's planner runs on the host alone (zkvc_msm_workspace_bytes):
    from 1 to 2^24 points the workspace holds at least the 2n endomorphism-split bases
    (64 bytes each in G1, 128 in G2) and their 16-byte half scalars, grows with n, and at
    the allocation-free entry's largest n fits its fixed 8 MiB scratch (the host has no
    occupancy data, so its chunks are the planner's smallest and this bound is the loose
    one)."""
    nv = _util.native()
    lib = nv.lib()
    prev = {1: 0, 2: 0}
    for lg in range(0, 25, 2):
        n = 1 << lg
        for group, pt in ((1, 64), (2, 128)):
            b = lib.zkvc_msm_workspace_bytes(n, group)
            assert b >= 2 * n * (pt + 16), (n, group, b)
            assert b >= prev[group], (n, group, b, prev[group])
            prev[group] = b
    assert lib.zkvc_msm_workspace_bytes(nv.ZKVC_MSM_NOALLOC_MAX_POINTS, 1) <= 8 << 20


def test_msm_size_limit():
    """Up to ZKVC_MSM_MAX_POINTS (2^27) the planner sizes a workspace; one point more is
    rejected before any device work: the workspace query answers 0 and the call
    ZKVC_EINVAL (the 16 n window digits of the split scalars would pass 2^31)."""
    nv = _util.native()
    lib = nv.lib()
    m = nv.ZKVC_MSM_MAX_POINTS
    assert m == 1 << 27
    for group, pt in ((1, 64), (2, 128)):
        assert lib.zkvc_msm_workspace_bytes(m, group) >= 2 * m * (pt + 16 + 8)
        assert lib.zkvc_msm_workspace_bytes(m + 1, group) == 0
    out = (ctypes.c_uint8 * 128)()
    for fn in (lib.zkvc_msm_g1, lib.zkvc_msm_g2):
        assert fn(ctypes.c_void_p(256), ctypes.c_void_p(256), m + 1, ctypes.c_void_p(256), 1 << 40, out,
                  None) == nv.ZKVC_EINVAL
        assert b"above" in lib.zkvc_last_error()
