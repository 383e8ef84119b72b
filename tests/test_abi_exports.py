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
