"""Thin ctypes binding of libzkvc.so: the C ABI of ``include/zkvc.h`` under the same names.

Only argument marshalling happens here: device tensors become raw pointers, the current
torch CUDA stream becomes the ``stream`` argument, and non-zero status codes become
``ZkvcError``.  Every computation runs in the library's CUDA kernels; there is no
fallback.  If ``libzkvc.so`` has not been built, loading raises immediately.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libzkvc.so")

ZKVC_OK = 0
ZKVC_EINVAL = -1
ZKVC_ENOMEM = -2
ZKVC_ECUDA = -3
ZKVC_ETIMEOUT = -4
ZKVC_EUNSAT = -5
ZKVC_EIO = -6

ZKVC_NTT_FORWARD = 0
ZKVC_NTT_INVERSE = 1
ZKVC_NTT_COSET_FORWARD = 2
ZKVC_NTT_COSET_INVERSE = 3

_c_p = ctypes.c_void_p
_c_sz = ctypes.c_size_t
_c_int = ctypes.c_int
_c_u32 = ctypes.c_uint32

# name -> (restype, argtypes)
SIGNATURES = {
    "zkvc_last_error": (ctypes.c_char_p, []),
    "zkvc_version": (_c_int, []),
    "zkvc_kernel_launches": (ctypes.c_uint64, []),
    "zkvc_profile_enable": (None, [_c_int]),
    "zkvc_profile_span": (_c_int, [_c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "zkvc_profile_read": (_c_int, [_c_int, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
    "zkvc_imad_rate": (_c_int, [_c_int, _c_u32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(_c_int), _c_p]),
    "zkvc_fr_mul": (_c_int, [_c_p, _c_p, _c_p, _c_sz, _c_p]),
    "zkvc_fp_mul": (_c_int, [_c_p, _c_p, _c_p, _c_sz, _c_p]),
    "zkvc_fp2_mul": (_c_int, [_c_p, _c_p, _c_p, _c_sz, _c_p]),
    "zkvc_fr_inv": (_c_int, [_c_p, _c_p, _c_sz, _c_p]),
    "zkvc_glv_split": (_c_int, [_c_p, _c_p]),
    "zkvc_fp_inv": (_c_int, [_c_p, _c_p, _c_sz, _c_p]),
    "zkvc_ntt": (_c_int, [_c_p, _c_u32, _c_int, _c_p]),
    "zkvc_matmul_i8": (_c_int, [_c_p, _c_p, _c_p, _c_int, _c_int, _c_int, _c_p]),
    "zkvc_msm_workspace_bytes": (_c_sz, [_c_sz, _c_int]),
    "zkvc_msm_g1": (_c_int, [_c_p, _c_p, _c_sz, _c_p, _c_sz, _c_p, _c_p]),
    "zkvc_msm_g2": (_c_int, [_c_p, _c_p, _c_sz, _c_p, _c_sz, _c_p, _c_p]),
    "zkvc_msm_g1_noalloc": (_c_int, [_c_p, _c_p, _c_sz, _c_p, _c_p]),
    "zkvc_generator_mul_workspace_bytes": (_c_sz, [_c_sz, _c_int]),
    "zkvc_g1_generator_mul": (_c_int, [_c_p, _c_sz, _c_p, _c_p, _c_sz, _c_p]),
    "zkvc_g2_generator_mul": (_c_int, [_c_p, _c_sz, _c_p, _c_p, _c_sz, _c_p]),
    "zkvc_setup": (_c_int, [_c_int, _c_int, _c_int, _c_p, _c_p, ctypes.POINTER(_c_p), ctypes.POINTER(_c_p)]),
    "zkvc_pk_free": (None, [_c_p]),
    "zkvc_vk_free": (None, [_c_p]),
    "zkvc_pk_info": (_c_int, [_c_p, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int), ctypes.POINTER(_c_int),
                              ctypes.POINTER(_c_u32), ctypes.POINTER(_c_sz), ctypes.POINTER(_c_sz)]),
    "zkvc_pk_export": (_c_int, [_c_p, _c_int, _c_sz, _c_sz, _c_p]),
    "zkvc_vk_export": (_c_int, [_c_p, _c_int, _c_sz, _c_sz, _c_p]),
    "zkvc_vk_info": (_c_int, [_c_p, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int), ctypes.POINTER(_c_int)]),
    "zkvc_vk_import": (_c_int, [_c_int, _c_int, _c_int, _c_p, _c_p, _c_p, _c_p, _c_p, _c_sz, ctypes.POINTER(_c_p)]),
    "zkvc_verify": (_c_int, [_c_p, _c_p, _c_p, _c_p, ctypes.POINTER(_c_int)]),
    "zkvc_pk_save": (_c_int, [_c_p, ctypes.c_char_p]),
    "zkvc_pk_load": (_c_int, [ctypes.c_char_p, _c_p, ctypes.POINTER(_c_p)]),
    "zkvc_vk_save": (_c_int, [_c_p, ctypes.c_char_p]),
    "zkvc_vk_load": (_c_int, [ctypes.c_char_p, ctypes.POINTER(_c_p)]),
    "zkvc_prove_workspace_bytes": (_c_sz, [_c_p]),
    "zkvc_prove": (_c_int, [_c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_sz, _c_p, _c_p]),
    "zkvc_prove_workspace_bytes_mode": (_c_sz, [_c_p, _c_int]),
    "zkvc_pk_autotune": (_c_int, [_c_p, _c_int, _c_p, _c_p, _c_p, _c_p, _c_p]),
    "zkvc_tune_cache_save": (_c_int, [ctypes.c_char_p]),
    "zkvc_tune_cache_load": (_c_int, [ctypes.c_char_p]),
    "zkvc_tune_cache_clear": (_c_int, []),
    "zkvc_pk_set_tuning": (_c_int, [_c_p, _c_p]),
    "zkvc_pk_get_tuning": (_c_int, [_c_p, _c_p]),
    "zkvc_setup_circuit": (_c_int, [_c_int, _c_int, _c_int, _c_int, _c_int, _c_p, _c_p, ctypes.POINTER(_c_p),
                                    ctypes.POINTER(_c_p)]),
    "zkvc_pk_circuit": (_c_int, [_c_p, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int), ctypes.POINTER(ctypes.c_uint64),
                                 ctypes.POINTER(ctypes.c_uint64)]),
    "zkvc_prove_mode": (_c_int, [_c_p, _c_int, _c_p, _c_p, _c_p, _c_p, _c_p, _c_sz, _c_p, _c_p]),
    "zkvc_batch_create": (_c_int, [_c_p, _c_int, _c_int, ctypes.POINTER(_c_p)]),
    "zkvc_batch_free": (None, [_c_p]),
    "zkvc_batch_info": (_c_int, [_c_p, ctypes.POINTER(_c_int), ctypes.POINTER(_c_sz), ctypes.POINTER(ctypes.c_uint64)]),
    "zkvc_batch_get_tuning": (_c_int, [_c_p, _c_p, _c_int]),
    "zkvc_batch_terms": (_c_int, [_c_p, _c_p]),
    "zkvc_batch_set_tuning": (_c_int, [_c_p, _c_p, _c_int]),
    "zkvc_batch_prove": (_c_int, [_c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p]),
    "zkvc_prove_batch": (_c_int, [_c_p, _c_p, _c_p, _c_p, _c_int, _c_p, _c_p, _c_p, _c_p]),
    "zkvc_set_wait_timeout_ms": (_c_int, [_c_int]),
    "zkvc_set_device_wait_limit_ns": (_c_int, [ctypes.c_uint64]),
    "zkvc_prove_claimed": (_c_int, [_c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_sz, _c_p, _c_p]),
    "zkvc_verify_batch": (_c_int, [_c_p, _c_p, _c_p, _c_p, _c_int, _c_p, _c_p]),
    "zkvc_pairing": (_c_int, [_c_p, _c_p, _c_sz, _c_p, _c_p]),
    "zkvc_server_create": (_c_int, [_c_p, _c_int, _c_int, _c_sz, _c_int, ctypes.POINTER(_c_p)]),
    "zkvc_server_free": (None, [_c_p]),
    "zkvc_server_submit": (_c_int, [_c_p, _c_int, _c_p, _c_p, _c_p, ctypes.POINTER(ctypes.c_uint64)]),
    "zkvc_server_wait": (_c_int, [_c_p, ctypes.c_uint64, _c_int, _c_p, _c_p, _c_p, ctypes.POINTER(_c_int)]),
    "zkvc_server_stats": (_c_int, [_c_p, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(_c_int),
                                   ctypes.POINTER(_c_int), ctypes.POINTER(_c_sz), ctypes.POINTER(_c_sz),
                                   ctypes.POINTER(ctypes.c_uint64)]),
    "zkvc_server_request_bytes": (_c_sz, [_c_p, _c_int]),
    "zkvc_server_merge_stats": (_c_int, [_c_p, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
}

ZKVC_Q_A, ZKVC_Q_B1, ZKVC_Q_B2, ZKVC_Q_L, ZKVC_Q_H = 0, 1, 2, 3, 4
ZKVC_Q_ALPHA1, ZKVC_Q_BETA1, ZKVC_Q_BETA2, ZKVC_Q_DELTA1, ZKVC_Q_DELTA2 = 5, 6, 7, 8, 9
ZKVC_VK_IC, ZKVC_VK_ALPHA1, ZKVC_VK_BETA2, ZKVC_VK_GAMMA2, ZKVC_VK_DELTA2 = 0, 1, 2, 3, 4
_G2_QUERIES = {ZKVC_Q_B2, ZKVC_Q_BETA2, ZKVC_Q_DELTA2}
_G2_VK = {ZKVC_VK_BETA2, ZKVC_VK_GAMMA2, ZKVC_VK_DELTA2}


class ZkvcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"zkvc status {code}: {msg}")
        self.code = code


_lib = None


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2504_12217_gb300.build.build()")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def check(rc):
    if rc != ZKVC_OK:
        raise ZkvcError(rc, lib().zkvc_last_error().decode())
    return rc


def _torch():
    import torch
    return torch


def _dev_ptr(t):
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _u8(t, width):
    torch = _torch()
    if t.dtype != torch.uint8 or t.dim() != 2 or t.shape[1] != width:
        raise ValueError(f"expected a uint8 tensor of shape [n, {width}]")
    return t


# ------------------------------------------------------------------ kernel layer
def zkvc_version():
    return lib().zkvc_version()


def zkvc_kernel_launches():
    return lib().zkvc_kernel_launches()


def zkvc_profile_enable(on):
    lib().zkvc_profile_enable(1 if on else 0)


def zkvc_profile_read():
    """{stage name: {"ms": total ms, "calls": n, "units": accumulated units, "start_ms": mean
    begin offset, "end_ms": mean end offset (both from the witness stage's begin)}}"""
    out = {}
    stage = 0
    while True:
        name, ms = ctypes.c_char_p(), ctypes.c_double()
        calls, units = ctypes.c_uint64(), ctypes.c_uint64()
        rc = lib().zkvc_profile_read(stage, ctypes.byref(name), ctypes.byref(ms), ctypes.byref(calls),
                                     ctypes.byref(units))
        if rc != ZKVC_OK:
            return out
        t0, t1 = ctypes.c_double(), ctypes.c_double()
        check(lib().zkvc_profile_span(stage, ctypes.byref(t0), ctypes.byref(t1)))
        out[name.value.decode()] = {"ms": ms.value, "calls": calls.value, "units": units.value,
                                    "start_ms": t0.value, "end_ms": t1.value}
        stage += 1


def zkvc_imad_rate(form=1, iters=1 << 14):
    """The integer-pipe microbenchmark: {"imad_per_s", "ms", "sms"} (form 0: independent
    mad.lo chains; 1: the field code's CIOS carry-chain row; 2: independent mad.hi; 3:
    independent mad.wide (two IMADs each); 4: mad.lo carry chains)."""
    rate, ms, sms = ctypes.c_double(), ctypes.c_double(), _c_int()
    check(lib().zkvc_imad_rate(form, iters, ctypes.byref(rate), ctypes.byref(ms), ctypes.byref(sms), _stream()))
    return {"imad_per_s": rate.value, "ms": ms.value, "sms": sms.value}


def zkvc_fr_mul(a, b, out=None):
    """Elementwise a * b mod r of [n, 32] canonical uint8 CUDA tensors."""
    return _field_mul("zkvc_fr_mul", a, b, out, 32)


def zkvc_fp_mul(a, b, out=None):
    return _field_mul("zkvc_fp_mul", a, b, out, 32)


def zkvc_fp2_mul(a, b, out=None):
    return _field_mul("zkvc_fp2_mul", a, b, out, 64)


def zkvc_glv_split(k):
    """(k1, k2) as signed Python ints with k = k1 + k2 lambda (mod r), for 0 <= k < r."""
    kb = ctypes.create_string_buffer(int(k).to_bytes(32, "little"), 32)
    out = ctypes.create_string_buffer(34)
    check(lib().zkvc_glv_split(kb, out))
    raw = out.raw
    halves = []
    for h in range(2):
        mag = int.from_bytes(raw[17 * h:17 * h + 16], "little")
        halves.append(-mag if raw[17 * h + 16] else mag)
    return tuple(halves)


def zkvc_fr_inv(a, out=None):
    """Elementwise a^-1 mod r (0 -> 0) of a [n, 32] canonical uint8 CUDA tensor."""
    return _field_inv("zkvc_fr_inv", a, out)


def zkvc_fp_inv(a, out=None):
    """Elementwise a^-1 mod p (0 -> 0) of a [n, 32] canonical uint8 CUDA tensor."""
    return _field_inv("zkvc_fp_inv", a, out)


def _field_inv(name, a, out):
    _u8(a, 32)
    if out is None:
        out = _torch().empty_like(a)
    check(getattr(lib(), name)(_dev_ptr(a), _dev_ptr(out), a.shape[0], _stream()))
    return out


def _field_mul(name, a, b, out, width):
    _u8(a, width)
    _u8(b, width)
    if out is None:
        out = _torch().empty_like(a)
    check(getattr(lib(), name)(_dev_ptr(a), _dev_ptr(b), _dev_ptr(out), a.shape[0], _stream()))
    return out


def zkvc_matmul_i8(X, W):
    """Y = X W for int8 CUDA tensors X [a, n] and W [n, b] (contiguous), exactly, on the
    tensor cores; returns int32 Y [a, b] (a CUDA tensor)."""
    import torch
    if X.dtype != torch.int8 or W.dtype != torch.int8 or X.dim() != 2 or W.dim() != 2:
        raise ValueError("X and W must be 2-D int8 tensors")
    if not (X.is_cuda and W.is_cuda and X.is_contiguous() and W.is_contiguous()):
        raise ValueError("X and W must be contiguous CUDA tensors")
    a, n = X.shape
    n2, b = W.shape
    if n != n2:
        raise ValueError("inner dimensions differ")
    Y = torch.empty((a, b), dtype=torch.int32, device=X.device)
    check(lib().zkvc_matmul_i8(_dev_ptr(X), _dev_ptr(W), _dev_ptr(Y), a, n, b, _stream()))
    return Y


def zkvc_ntt(data, kind):
    """In-place NTT of a [2^k, 32] canonical Fr CUDA tensor (kind: ZKVC_NTT_*)."""
    _u8(data, 32)
    n = data.shape[0]
    log_n = n.bit_length() - 1
    if n != 1 << log_n:
        raise ValueError("length must be a power of two")
    check(lib().zkvc_ntt(_dev_ptr(data), log_n, kind, _stream()))
    return data


ZKVC_MSM_MAX_POINTS = 1 << 27


def zkvc_msm_workspace_bytes(n, group):
    return lib().zkvc_msm_workspace_bytes(n, group)


def _msm(name, group, points, scalars, workspace=None):
    torch = _torch()
    width = 64 if group == 1 else 128
    _u8(points, width)
    _u8(scalars, 32)
    n = points.shape[0]
    if scalars.shape[0] != n:
        raise ValueError("points and scalars differ in length")
    need = zkvc_msm_workspace_bytes(n, group)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device=points.device)
    out = (ctypes.c_uint8 * width)()
    check(getattr(lib(), name)(_dev_ptr(points), _dev_ptr(scalars), n, _dev_ptr(workspace),
                               workspace.numel(), out, _stream()))
    return bytes(out)


def zkvc_msm_g1(points, scalars, workspace=None):
    """sum_i s_i P_i over G1: points [n, 64], scalars [n, 32]; returns 64 bytes."""
    return _msm("zkvc_msm_g1", 1, points, scalars, workspace)


def zkvc_msm_g2(points, scalars, workspace=None):
    """sum_i s_i Q_i over G2: points [n, 128], scalars [n, 32]; returns 128 bytes."""
    return _msm("zkvc_msm_g2", 2, points, scalars, workspace)


def _generator_mul(name, group, scalars):
    torch = _torch()
    _u8(scalars, 32)
    n = scalars.shape[0]
    width = 64 if group == 1 else 128
    out = torch.empty((n, width), dtype=torch.uint8, device=scalars.device)
    if n == 0:
        return out
    ws = torch.empty(lib().zkvc_generator_mul_workspace_bytes(n, group), dtype=torch.uint8, device=scalars.device)
    check(getattr(lib(), name)(_dev_ptr(scalars), n, _dev_ptr(out), _dev_ptr(ws), ws.numel(), _stream()))
    return out


def zkvc_g1_generator_mul(scalars):
    """[k_i] G1 for [n, 32] canonical scalars; returns [n, 64] canonical affine points."""
    return _generator_mul("zkvc_g1_generator_mul", 1, scalars)


def zkvc_g2_generator_mul(scalars):
    """[k_i] G2 for [n, 32] canonical scalars; returns [n, 128] canonical affine points."""
    return _generator_mul("zkvc_g2_generator_mul", 2, scalars)


ZKVC_MSM_NOALLOC_MAX_POINTS = 4096


def zkvc_msm_g1_noalloc(points, scalars):
    """sum_i s_i P_i over G1 for n <= ZKVC_MSM_NOALLOC_MAX_POINTS without any device
    allocation (the library's built-in scratch array is used); returns 64 bytes."""
    _u8(points, 64)
    _u8(scalars, 32)
    n = points.shape[0]
    if scalars.shape[0] != n:
        raise ValueError("points and scalars differ in length")
    out = (ctypes.c_uint8 * 64)()
    check(lib().zkvc_msm_g1_noalloc(_dev_ptr(points) if n else None, _dev_ptr(scalars) if n else None, n, out,
                                    _stream()))
    return bytes(out)


# ------------------------------------------------------------------ Groth16 layer
class ProvingKey:
    """Owns a zkvc_pk handle (device-resident proving key); freed with the object."""

    def __init__(self, handle):
        self.handle = handle
        info = zkvc_pk_info(self)
        self.shape = (info["a"], info["n"], info["b"])
        self.log_domain = info["log_domain"]

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.zkvc_pk_free(self.handle)
            self.handle = None


class VerifyingKey:
    """Owns a zkvc_vk handle (host memory)."""

    def __init__(self, handle, shape):
        self.handle = handle
        self.shape = shape

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.zkvc_vk_free(self.handle)
            self.handle = None


def zkvc_setup(a, n, b, toxic):
    """Gen for the (a, n, b) matmul circuit; toxic: 192 bytes (tau, alpha, beta, gamma,
    delta, z canonical little-endian).  Returns (ProvingKey, VerifyingKey)."""
    if len(toxic) != 192:
        raise ValueError("toxic must be 192 bytes")
    pk, vk = _c_p(), _c_p()
    buf = ctypes.create_string_buffer(bytes(toxic), 192)
    check(lib().zkvc_setup(a, n, b, buf, _stream(), ctypes.byref(pk), ctypes.byref(vk)))
    return ProvingKey(pk), VerifyingKey(vk, (a, n, b))


ZKVC_CIRCUIT_CRPC_PSQ, ZKVC_CIRCUIT_CRPC, ZKVC_CIRCUIT_PSQ, ZKVC_CIRCUIT_VANILLA = 0, 1, 2, 3
ZKVC_PUBLIC_XY, ZKVC_PUBLIC_NONE = 0, 1
CIRCUIT_NAMES = {"crpc_psq": 0, "crpc": 1, "psq": 2, "vanilla": 3, "crpc_psq_softmax": 4, "crpc_psq_gelu": 5}
PUBLIC_NAMES = {"xy": 0, "none": 1}


def zkvc_setup_circuit(a, n, b, circuit, public_io, toxic):
    """Gen for one of the ablation circuits (ZKVC_CIRCUIT_* or its name) with X and Y
    public or private (ZKVC_PUBLIC_* or "xy" / "none").  Returns (ProvingKey, VerifyingKey)."""
    circuit = CIRCUIT_NAMES.get(circuit, circuit)
    public_io = PUBLIC_NAMES.get(public_io, public_io)
    if len(toxic) != 192:
        raise ValueError("toxic must be 192 bytes")
    pk, vk = _c_p(), _c_p()
    buf = ctypes.create_string_buffer(bytes(toxic), 192)
    check(lib().zkvc_setup_circuit(a, n, b, circuit, public_io, buf, _stream(), ctypes.byref(pk), ctypes.byref(vk)))
    out_vk = VerifyingKey(vk, (a, n, b))
    out_vk.public_io = public_io
    return ProvingKey(pk), out_vk


def zkvc_pk_circuit(pk):
    c, p, r, v = _c_int(), _c_int(), ctypes.c_uint64(), ctypes.c_uint64()
    check(lib().zkvc_pk_circuit(pk.handle, ctypes.byref(c), ctypes.byref(p), ctypes.byref(r), ctypes.byref(v)))
    return {"circuit": c.value, "public_io": p.value, "rows": r.value, "vars": v.value}


def zkvc_pk_info(pk):
    a, n, b = _c_int(), _c_int(), _c_int()
    logd, g1, g2 = _c_u32(), _c_sz(), _c_sz()
    check(lib().zkvc_pk_info(pk.handle, ctypes.byref(a), ctypes.byref(n), ctypes.byref(b), ctypes.byref(logd),
                             ctypes.byref(g1), ctypes.byref(g2)))
    return {"a": a.value, "n": n.value, "b": b.value, "log_domain": logd.value, "g1_bases": g1.value,
            "g2_bases": g2.value}


def zkvc_pk_export(pk, query, start, count):
    width = 128 if query in _G2_QUERIES else 64
    out = ctypes.create_string_buffer(max(1, width * count))
    check(lib().zkvc_pk_export(pk.handle, query, start, count, out))
    return out.raw[: width * count]


def zkvc_vk_export(vk, query, start, count):
    width = 128 if query in _G2_VK else 64
    out = ctypes.create_string_buffer(max(1, width * count))
    check(lib().zkvc_vk_export(vk.handle, query, start, count, out))
    return out.raw[: width * count]


def zkvc_vk_import(a, n, b, alpha1, beta2, gamma2, delta2, ic):
    """VerifyingKey from canonical encodings (bytes); ic holds l + 1 points of 64 bytes."""
    if len(ic) % 64:
        raise ValueError("ic must be a multiple of 64 bytes")
    vk = _c_p()
    check(lib().zkvc_vk_import(a, n, b, bytes(alpha1), bytes(beta2), bytes(gamma2), bytes(delta2), bytes(ic),
                               len(ic) // 64, ctypes.byref(vk)))
    return VerifyingKey(vk, (a, n, b))


def zkvc_verify(vk, X, Y, proof):
    """Host-side verification; X: int8 [a, n], Y: int32 [a, b] (numpy or CPU tensors), or
    None for both with a key that has no public inputs."""
    import numpy as np
    a, n, b = vk.shape
    if len(proof) != 256:
        raise ValueError("proof must be 256 bytes")
    ok = _c_int(0)
    if X is None and Y is None:
        check(lib().zkvc_verify(vk.handle, None, None, bytes(proof), ctypes.byref(ok)))
        return bool(ok.value)
    Xn = np.ascontiguousarray(np.asarray(X, dtype=np.int8).reshape(a, n))
    Yn = np.ascontiguousarray(np.asarray(Y, dtype=np.int32).reshape(a, b))
    check(lib().zkvc_verify(vk.handle, Xn.ctypes.data_as(_c_p), Yn.ctypes.data_as(_c_p), bytes(proof),
                            ctypes.byref(ok)))
    return bool(ok.value)


def zkvc_pk_save(pk, path):
    check(lib().zkvc_pk_save(pk.handle, os.fsencode(path)))


def zkvc_pk_load(path):
    pk = _c_p()
    check(lib().zkvc_pk_load(os.fsencode(path), _stream(), ctypes.byref(pk)))
    return ProvingKey(pk)


def zkvc_vk_save(vk, path):
    check(lib().zkvc_vk_save(vk.handle, os.fsencode(path)))


def zkvc_vk_load(path):
    vk = _c_p()
    check(lib().zkvc_vk_load(os.fsencode(path), ctypes.byref(vk)))
    a, n, b = _c_int(), _c_int(), _c_int()
    check(lib().zkvc_vk_info(vk, ctypes.byref(a), ctypes.byref(n), ctypes.byref(b)))
    return VerifyingKey(vk, (a.value, n.value, b.value))


def zkvc_prove_workspace_bytes(pk):
    return lib().zkvc_prove_workspace_bytes(pk.handle)


ZKVC_PROVE_FOLD = 0
ZKVC_PROVE_CHAIN = 1
ZKVC_PROVE_AUTO = 2


ZKVC_PK_TUNING_LEN = 10


ZKVC_TUNE_FRESH = 0x10


def zkvc_pk_autotune(pk, X, W, rs, mode=0, fresh=False):
    """Tune the key's launch shape for one-proof latency on these inputs; returns the
    chosen [small, rest, h, g2 chunk terms, NTT log2 elements per block, side-MSM start,
    prover mode, G2-MSM start, H-run quads, small-run quads].  mode: ZKVC_PROVE_FOLD,
    ZKVC_PROVE_CHAIN or ZKVC_PROVE_AUTO (both).  A cached result for the same shape, mode
    and GPU is applied without timing unless fresh=True."""
    arr = (ctypes.c_uint32 * ZKVC_PK_TUNING_LEN)()
    rsb = ctypes.create_string_buffer(bytes(rs), 64)
    m = mode | (ZKVC_TUNE_FRESH if fresh else 0)
    check(lib().zkvc_pk_autotune(pk.handle, m, _dev_ptr(X), _dev_ptr(W), rsb, _stream(), arr))
    return list(arr)


def zkvc_tune_cache_save(path):
    check(lib().zkvc_tune_cache_save(os.fsencode(path)))


def zkvc_tune_cache_load(path):
    check(lib().zkvc_tune_cache_load(os.fsencode(path)))


def zkvc_tune_cache_clear():
    check(lib().zkvc_tune_cache_clear())


def zkvc_pk_set_tuning(pk, tuning):
    arr = (ctypes.c_uint32 * ZKVC_PK_TUNING_LEN)(*tuning)
    check(lib().zkvc_pk_set_tuning(pk.handle, arr))


def zkvc_pk_get_tuning(pk):
    arr = (ctypes.c_uint32 * ZKVC_PK_TUNING_LEN)()
    check(lib().zkvc_pk_get_tuning(pk.handle, arr))
    return list(arr)


def zkvc_prove_workspace_bytes_mode(pk, mode):
    return lib().zkvc_prove_workspace_bytes_mode(pk.handle, mode)


def zkvc_prove_mode(pk, mode, X, W, rs, Y=None, workspace=None):
    """zkvc_prove with an explicit mode (ZKVC_PROVE_FOLD or ZKVC_PROVE_CHAIN)."""
    torch = _torch()
    a, n, b = pk.shape
    if X.dtype != torch.int8 or tuple(X.shape) != (a, n) or W.dtype != torch.int8 or tuple(W.shape) != (n, b):
        raise ValueError(f"expected X int8 [{a}, {n}] and W int8 [{n}, {b}]")
    if len(rs) != 64:
        raise ValueError("rs must be 64 bytes")
    if Y is None:
        Y = torch.empty((a, b), dtype=torch.int32, device=X.device)
    need = zkvc_prove_workspace_bytes_mode(pk, mode)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device=X.device)
    proof = ctypes.create_string_buffer(256)
    rsb = ctypes.create_string_buffer(bytes(rs), 64)
    check(lib().zkvc_prove_mode(pk.handle, mode, _dev_ptr(X), _dev_ptr(W), rsb, _dev_ptr(Y), _dev_ptr(workspace),
                                workspace.numel(), proof, _stream()))
    return proof.raw, Y


def zkvc_prove(pk, X, W, rs, Y=None, workspace=None):
    """Prove Y = X W.  X: [a, n] int8 CUDA tensor, W: [n, b] int8, rs: 64 bytes (r || s).
    Returns (proof bytes, Y as an [a, b] int32 CUDA tensor)."""
    torch = _torch()
    a, n, b = pk.shape
    if X.dtype != torch.int8 or tuple(X.shape) != (a, n) or W.dtype != torch.int8 or tuple(W.shape) != (n, b):
        raise ValueError(f"expected X int8 [{a}, {n}] and W int8 [{n}, {b}]")
    if len(rs) != 64:
        raise ValueError("rs must be 64 bytes")
    if Y is None:
        Y = torch.empty((a, b), dtype=torch.int32, device=X.device)
    need = zkvc_prove_workspace_bytes(pk)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=X.device)
    proof = ctypes.create_string_buffer(256)
    rsb = ctypes.create_string_buffer(bytes(rs), 64)
    check(lib().zkvc_prove(pk.handle, _dev_ptr(X), _dev_ptr(W), rsb, _dev_ptr(Y), _dev_ptr(workspace),
                           workspace.numel(), proof, _stream()))
    return proof.raw, Y


def zkvc_prove_claimed(pk, X, W, Y_claimed, rs, workspace=None):
    """Prove a claimed product: Y_claimed ([a, b] int32 CUDA tensor) enters the witness as
    it is; raises ZkvcError(ZKVC_EUNSAT) if it is not X W.  Returns the proof bytes."""
    torch = _torch()
    a, n, b = pk.shape
    if X.dtype != torch.int8 or tuple(X.shape) != (a, n) or W.dtype != torch.int8 or tuple(W.shape) != (n, b):
        raise ValueError(f"expected X int8 [{a}, {n}] and W int8 [{n}, {b}]")
    if Y_claimed.dtype != torch.int32 or tuple(Y_claimed.shape) != (a, b):
        raise ValueError(f"expected Y int32 [{a}, {b}]")
    if len(rs) != 64:
        raise ValueError("rs must be 64 bytes")
    need = zkvc_prove_workspace_bytes(pk)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=X.device)
    proof = ctypes.create_string_buffer(256)
    rsb = ctypes.create_string_buffer(bytes(rs), 64)
    check(lib().zkvc_prove_claimed(pk.handle, _dev_ptr(X), _dev_ptr(W), _dev_ptr(Y_claimed), rsb, _dev_ptr(workspace),
                                   workspace.numel(), proof, _stream()))
    return proof.raw


# ------------------------------------------------------------------ batched proving
ZKVC_BATCH_AUTOTUNE = 1
ZKVC_BATCH_EAGER = 2
ZKVC_BATCH_TUNING_LEN = 7
TUNING_NAMES = ("small_chunk", "small_accum_threads", "main_chunk", "main_accum_threads",
                "g2_chunk", "g2_accum_threads", "ntt_log_elems_per_block")


def zkvc_set_wait_timeout_ms(ms):
    check(lib().zkvc_set_wait_timeout_ms(int(ms)))


def zkvc_set_device_wait_limit_ns(ns):
    """Limit of the tensor-core matmul's first waits (0: give up at once; default 200 ms)."""
    check(lib().zkvc_set_device_wait_limit_ns(int(ns)))


def _ptr_array(ptrs):
    arr = (_c_p * len(ptrs))()
    for i, p in enumerate(ptrs):
        arr[i] = p
    return arr


class Batch:
    """Owns a zkvc_batch handle: one proof per listed proving key per prove() call, in one
    captured launch sequence.  Keeps the keys alive."""

    def __init__(self, pks, flags=0):
        self.pks = list(pks)
        h = _c_p()
        keys = _ptr_array([pk.handle for pk in self.pks])
        check(lib().zkvc_batch_create(keys, len(self.pks), flags, ctypes.byref(h)))
        self.handle = h

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.zkvc_batch_free(self.handle)
            self.handle = None

    def info(self):
        count, nbytes, launches = _c_int(), _c_sz(), ctypes.c_uint64()
        check(lib().zkvc_batch_info(self.handle, ctypes.byref(count), ctypes.byref(nbytes), ctypes.byref(launches)))
        return {"count": count.value, "device_bytes": nbytes.value, "graph_launches": launches.value}

    def terms(self):
        """{"small": n, "main": n, "g2": n}: bucket terms of the last call's MSM runs."""
        arr = (ctypes.c_uint64 * 3)()
        check(lib().zkvc_batch_terms(self.handle, arr))
        return {"small": arr[0], "main": arr[1], "g2": arr[2]}

    def get_tuning(self):
        arr = (ctypes.c_int32 * ZKVC_BATCH_TUNING_LEN)()
        check(lib().zkvc_batch_get_tuning(self.handle, arr, ZKVC_BATCH_TUNING_LEN))
        return dict(zip(TUNING_NAMES, list(arr)))

    def set_tuning(self, tuning):
        vals = [tuning[k] for k in TUNING_NAMES] if isinstance(tuning, dict) else list(tuning)
        arr = (ctypes.c_int32 * ZKVC_BATCH_TUNING_LEN)(*vals)
        check(lib().zkvc_batch_set_tuning(self.handle, arr, ZKVC_BATCH_TUNING_LEN))

    def prove(self, Xs, Ws, rs_list, Ys=None, with_status=False):
        """Xs[i], Ws[i]: int8 CUDA tensors of key i's shape; rs_list[i]: 64 bytes.
        Returns (list of 256-byte proofs, list of Y tensors[, per-instance status])."""
        torch = _torch()
        n = len(self.pks)
        if not (len(Xs) == len(Ws) == len(rs_list) == n):
            raise ValueError(f"expected {n} instances")
        if Ys is None:
            Ys = [torch.empty((pk.shape[0], pk.shape[2]), dtype=torch.int32, device=Xs[0].device) for pk in self.pks]
        for pk, X, W, Y in zip(self.pks, Xs, Ws, Ys):
            a, nn, b = pk.shape
            if X.dtype != torch.int8 or tuple(X.shape) != (a, nn) or W.dtype != torch.int8 or tuple(W.shape) != (nn, b):
                raise ValueError(f"expected X int8 [{a}, {nn}] and W int8 [{nn}, {b}]")
            if Y.dtype != torch.int32 or tuple(Y.shape) != (a, b):
                raise ValueError(f"expected Y int32 [{a}, {b}]")
        if any(len(r) != 64 for r in rs_list):
            raise ValueError("each rs must be 64 bytes")
        xs = _ptr_array([_dev_ptr(X).value for X in Xs])
        ws = _ptr_array([_dev_ptr(W).value for W in Ws])
        ys = _ptr_array([_dev_ptr(Y).value for Y in Ys])
        rsb = ctypes.create_string_buffer(b"".join(bytes(r) for r in rs_list), 64 * n)
        proofs = ctypes.create_string_buffer(256 * n)
        status = (_c_int * n)()
        rc = lib().zkvc_batch_prove(self.handle, xs, ws, rsb, ys, proofs, status, _stream())
        st = list(status)
        if rc != ZKVC_OK and not (with_status and rc in (ZKVC_EINVAL, ZKVC_EUNSAT) and any(st)):
            check(rc)
        out = [proofs.raw[256 * i: 256 * (i + 1)] for i in range(n)]
        return (out, Ys, st) if with_status else (out, Ys)


def zkvc_prove_batch(pks, Xs, Ws, rs_list):
    """One-shot batched prove (eager launches); returns (proofs, Ys)."""
    torch = _torch()
    n = len(pks)
    Ys = [torch.empty((pk.shape[0], pk.shape[2]), dtype=torch.int32, device=Xs[0].device) for pk in pks]
    keys = _ptr_array([pk.handle for pk in pks])
    xs = _ptr_array([_dev_ptr(X).value for X in Xs])
    ws = _ptr_array([_dev_ptr(W).value for W in Ws])
    ys = _ptr_array([_dev_ptr(Y).value for Y in Ys])
    rsb = ctypes.create_string_buffer(b"".join(bytes(r) for r in rs_list), 64 * n)
    proofs = ctypes.create_string_buffer(256 * n)
    check(lib().zkvc_prove_batch(keys, xs, ws, rsb, n, ys, proofs, None, _stream()))
    return [proofs.raw[256 * i: 256 * (i + 1)] for i in range(n)], Ys


# ------------------------------------------------------------------ proof server
ZKVC_SERVER_ADAPTIVE = 0
ZKVC_SERVER_FOLD = 1
ZKVC_SERVER_CHAIN = 2
ZKVC_SERVER_MERGE = 3


def zkvc_server_request_bytes(pk, mode):
    return lib().zkvc_server_request_bytes(pk.handle, mode)


class Server:
    """Owns a zkvc_server handle: continuous batching of proof requests over resident
    keys.  submit() returns a ticket; wait() returns the result."""

    def __init__(self, pks, slots=4, mem_budget=8 << 30, policy=ZKVC_SERVER_ADAPTIVE):
        self.pks = list(pks)
        h = _c_p()
        keys = _ptr_array([pk.handle for pk in self.pks])
        check(lib().zkvc_server_create(keys, len(self.pks), slots, mem_budget, policy, ctypes.byref(h)))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.zkvc_server_free(self.handle)
            self.handle = None

    def __del__(self):
        self.close()

    def submit(self, key, X, W, rs):
        """X, W: int8 numpy arrays (host) of key `key`'s shape; rs: 64 bytes."""
        import numpy as np
        Xn = np.ascontiguousarray(np.asarray(X, dtype=np.int8))
        Wn = np.ascontiguousarray(np.asarray(W, dtype=np.int8))
        if 0 <= key < len(self.pks):  # the library rejects other key indices itself
            a, n, b = self.pks[key].shape
            Xn, Wn = Xn.reshape(a, n), Wn.reshape(n, b)
        if len(rs) != 64:
            raise ValueError("rs must be 64 bytes")
        t = ctypes.c_uint64()
        check(lib().zkvc_server_submit(self.handle, key, Xn.ctypes.data_as(_c_p), Wn.ctypes.data_as(_c_p), bytes(rs),
                                       ctypes.byref(t)))
        return t.value

    def wait(self, ticket, key, timeout_ms=60000):
        """(status, proof bytes or None, Y numpy int32 or None, {queue_ms, prove_ms, total_ms});
        raises ZkvcError(ZKVC_ETIMEOUT) if the request is not done in time."""
        import numpy as np
        a, n, b = self.pks[key].shape if 0 <= key < len(self.pks) else (1, 1, 1)
        proof = ctypes.create_string_buffer(256)
        Y = np.empty((a, b), dtype=np.int32)
        times = (ctypes.c_double * 3)()
        status = _c_int()
        check(lib().zkvc_server_wait(self.handle, ticket, int(timeout_ms), proof, Y.ctypes.data_as(_c_p), times,
                                     ctypes.byref(status)))
        t = {"queue_ms": times[0], "prove_ms": times[1], "total_ms": times[2]}
        if status.value != ZKVC_OK:
            return status.value, None, None, t
        return ZKVC_OK, proof.raw, Y, t

    def stats(self):
        c, f, q, u, p, ch = ctypes.c_uint64(), _c_int(), _c_int(), _c_sz(), _c_sz(), ctypes.c_uint64()
        check(lib().zkvc_server_stats(self.handle, ctypes.byref(c), ctypes.byref(f), ctypes.byref(q), ctypes.byref(u),
                                      ctypes.byref(p), ctypes.byref(ch)))
        mr, nb = ctypes.c_uint64(), ctypes.c_uint64()
        check(lib().zkvc_server_merge_stats(self.handle, ctypes.byref(mr), ctypes.byref(nb)))
        return {"completed": c.value, "in_flight": f.value, "queued": q.value, "bytes_in_use": u.value,
                "peak_bytes": p.value, "chain_mode": ch.value, "merged_requests": mr.value, "merged_batches": nb.value}


# ------------------------------------------------------------------ GPU verification
def zkvc_verify_batch(vks, Xs, Ys, proofs):
    """Verify proofs[i] against vks[i] with public inputs Xs[i] (int8 [a, n]) and Ys[i]
    (int32 [a, b]) on the GPU (None for keys without public inputs).  Returns a list of
    booleans."""
    import numpy as np
    n = len(proofs)
    keep = []
    xs = (_c_p * max(1, n))()
    ys = (_c_p * max(1, n))()
    for i in range(n):
        if Xs is not None and Xs[i] is not None:
            a, nn, b = vks[i].shape
            Xn = np.ascontiguousarray(np.asarray(Xs[i], dtype=np.int8).reshape(a, nn))
            Yn = np.ascontiguousarray(np.asarray(Ys[i], dtype=np.int32).reshape(a, b))
            keep += [Xn, Yn]
            xs[i] = Xn.ctypes.data
            ys[i] = Yn.ctypes.data
    vka = _ptr_array([vk.handle for vk in vks]) if n else (_c_p * 1)()
    pb = ctypes.create_string_buffer(b"".join(bytes(p) for p in proofs), max(1, 256 * n))
    ok = (_c_int * max(1, n))()
    check(lib().zkvc_verify_batch(vka, xs, ys, pb, n, ok, _stream()))
    return [bool(ok[i]) for i in range(n)]


def zkvc_pairing(P, Q):
    """e(P_i, Q_i) on the GPU: P uint8 [n, 64], Q uint8 [n, 128] canonical CUDA tensors;
    returns a uint8 [n, 384] CUDA tensor (tower-basis coefficients)."""
    torch = _torch()
    _u8(P, 64)
    _u8(Q, 128)
    out = torch.empty((P.shape[0], 384), dtype=torch.uint8, device=P.device)
    check(lib().zkvc_pairing(_dev_ptr(P), _dev_ptr(Q), P.shape[0], _dev_ptr(out), _stream()))
    return out
