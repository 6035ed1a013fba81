"""Python binding of libfhe_gb300 (include/fhe.h): the non-RNS CKKS hot path on a GB300.

Argument marshalling only.  Every homomorphic step runs in the library's CUDA
kernels; PyTorch provides device memory (the context's allocator callbacks
and the caller's tensors) and the current CUDA stream.  The module-level
functions carry the C ABI's names and signatures with tensors in place of raw
pointers; ``Context`` bundles them for convenience.

Layouts (see include/fhe.h): a ciphertext batch is a CUDA int32 tensor of
shape (cnum, 2, L, N) holding uint32 limbs (poly 0 = b, poly 1 = a), least
significant limb first, L = ceil(logQ / 32).  Plaintexts are (cnum, L, N).

Importing the package loads the shared library and raises ImportError if it
has not been built (``python -c "import __graft_entry__ as g; g.build()"``):
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfhe_gb300.so")

FHE_OK = 0
FHE_EINVAL = -1
FHE_ENOMEM = -2
FHE_ELEVEL = -3
FHE_ENOKEY = -4
FHE_ECUDA = -5
FHE_ETIMEOUT = -6
FHE_EWORKSPACE = -7
FHE_SCHEME_CKKS = 0
FHE_SCHEME_BGV = 1
FHE_CRT_DIRECT = 0
FHE_CRT_GARNER = 1
FHE_CRT_DIRECT_INT = 2
FHE_CRT_DIRECT_CVT = 3
FHE_OP_MULT = 1
FHE_OP_ROTATE = 2
FHE_OP_ENCRYPT = 3
FHE_OP_DECRYPT = 4
FHE_OP_KEYGEN = 5
FHE_OP_RING_MUL = 6
FHE_OP_MULT_RAGGED = 7
FHE_OP_MULT_PLAIN = 8
FHE_OP_ENCODE = 9
FHE_LIFT_AUTO = 0
FHE_LIFT_INT = 1
FHE_LIFT_TC = 2
FHE_NTT_FUSED = 0
FHE_NTT_SPLIT = 1
FHE_NTT_FUSED_GROUPS = 2
FHE_SAMPLE_UNIFORM = 0
FHE_SAMPLE_TERNARY = 1
FHE_SAMPLE_HWT = 2
FHE_SAMPLE_GAUSSIAN = 3


class FheParams(ctypes.Structure):
    _fields_ = [("scheme", ctypes.c_int32), ("logN", ctypes.c_int32), ("logQ", ctypes.c_int32),
                ("logP", ctypes.c_int32), ("crt", ctypes.c_int32), ("bgv_levels", ctypes.c_int32),
                ("t", ctypes.c_uint32), ("bgv_q0", ctypes.c_uint64), ("bgv_r", ctypes.c_uint64),
                ("hamming_weight", ctypes.c_int32), ("sigma", ctypes.c_double)]


class FheCt(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("cnum", ctypes.c_int32), ("logQ", ctypes.c_int32),
                ("level", ctypes.c_int32), ("log_scale", ctypes.c_double)]


class FheBatchGroup(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("a", ctypes.c_void_p), ("b", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("item_logQ", ctypes.c_void_p), ("cnum", ctypes.c_int32), ("L_pad", ctypes.c_int32),
                ("logQ_max", ctypes.c_int32), ("ws", ctypes.c_void_p), ("ws_bytes", ctypes.c_size_t)]


class FheBatchSched(ctypes.Structure):
    _fields_ = [("col_ctas_per_sm", ctypes.c_int32), ("row_ctas_per_sm", ctypes.c_int32),
                ("col_unit_rows", ctypes.c_int32)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)

_P = ctypes.c_void_p
_I = ctypes.c_int
_SZ = ctypes.c_size_t

# name -> (restype, argtypes); mirrors include/fhe.h one to one
SIGNATURES = {
    "fhe_ctx_create": (_I, [ctypes.POINTER(FheParams), ALLOC_FN, FREE_FN, _P, ctypes.POINTER(_P)]),
    "fhe_ctx_destroy": (_I, [_P]),
    "fhe_last_error": (ctypes.c_char_p, []),
    "fhe_sync": (_I, [_P]),
    "fhe_ct_bytes": (_SZ, [_I, _I, _I]),
    "fhe_workspace_bytes": (_SZ, [_P, _I, _I, _I]),
    "fhe_keygen": (_I, [_P, ctypes.c_uint64, _P, _I]),
    "fhe_keygen_inject": (_I, [_P, _P, _P, _P, _P, _P]),
    "fhe_keygen_rotation": (_I, [_P, _I, _P, _P]),
    "fhe_keygen_conjugation": (_I, [_P, _P, _P]),
    "fhe_encrypt": (_I, [_P, _P, ctypes.c_uint64, ctypes.POINTER(FheCt), _P, _SZ, _P]),
    "fhe_encrypt_inject": (_I, [_P, _P, _P, _P, _P, ctypes.POINTER(FheCt), _P, _SZ, _P]),
    "fhe_sample": (_I, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, _I, _I, _I, ctypes.c_double, _P]),
    "fhe_decrypt": (_I, [_P, ctypes.POINTER(FheCt), _P, _P, _SZ, _P]),
    "fhe_mult_relin": (_I, [_P, ctypes.POINTER(FheCt), ctypes.POINTER(FheCt), ctypes.POINTER(FheCt), _P, _SZ, _P]),
    "fhe_mult_relin_rescale": (_I, [_P, ctypes.POINTER(FheCt), ctypes.POINTER(FheCt), _I, ctypes.POINTER(FheCt), _P,
                                    _SZ, _P]),
    "fhe_rescale": (_I, [_P, ctypes.POINTER(FheCt), _I, ctypes.POINTER(FheCt), _P]),
    "fhe_mult_relin_rescale_ragged": (_I, [_P, _P, _P, _P, _I, _I, _P, _I, _I, _P, _SZ, _P]),
    "fhe_mult_relin_rescale_batch": (_I, [ctypes.POINTER(FheBatchGroup), _I, _I, ctypes.POINTER(FheBatchSched), _P]),
    "fhe_moddown": (_I, [_P, ctypes.POINTER(FheCt), ctypes.POINTER(FheCt), _P]),
    "fhe_rotate": (_I, [_P, ctypes.POINTER(FheCt), _I, ctypes.POINTER(FheCt), _P, _SZ, _P]),
    "fhe_rotate_hoisted": (_I, [_P, ctypes.POINTER(FheCt), _P, _I, _P, _P, _SZ, _P]),
    "fhe_conjugate": (_I, [_P, ctypes.POINTER(FheCt), ctypes.POINTER(FheCt), _P, _SZ, _P]),
    "fhe_add": (_I, [_P, ctypes.POINTER(FheCt), ctypes.POINTER(FheCt), ctypes.POINTER(FheCt), _P]),
    "fhe_sub": (_I, [_P, ctypes.POINTER(FheCt), ctypes.POINTER(FheCt), ctypes.POINTER(FheCt), _P]),
    "fhe_negate": (_I, [_P, ctypes.POINTER(FheCt), ctypes.POINTER(FheCt), _P]),
    "fhe_mult_const": (_I, [_P, ctypes.POINTER(FheCt), ctypes.c_int32, ctypes.POINTER(FheCt), _P]),
    "fhe_ring_mul": (_I, [_P, _P, _I, _P, _I, _I, _P, _I, _P, _SZ, _P]),
    "fhe_add_const": (_I, [_P, ctypes.POINTER(FheCt), ctypes.c_int64, _I, ctypes.POINTER(FheCt), _P]),
    "fhe_add_const_vec": (_I, [_P, ctypes.POINTER(FheCt), _P, _I, ctypes.POINTER(FheCt), _P]),
    "fhe_imult": (_I, [_P, ctypes.POINTER(FheCt), ctypes.POINTER(FheCt), _P]),
    "fhe_mult_plain": (_I, [_P, ctypes.POINTER(FheCt), _P, _I, ctypes.c_double, ctypes.POINTER(FheCt), _P, _SZ, _P]),
    "fhe_primes_for_bound": (_I, [_I]),
    "fhe_selftest_wait_timeout": (_I, [_I, _P]),
    "fhe_ckks_encode": (_I, [_P, _P, _I, _I, _I, _P, _P, _SZ, _P]),
    "fhe_ckks_decode": (_I, [_P, _P, _I, _I, ctypes.c_double, _P, _P, _SZ, _P]),
    "fhe_bgv_encode": (_I, [_P, _P, _I, _P, _SZ, _P]),
    "fhe_bgv_decode": (_I, [_P, _P, _SZ, _I, _P, _P]),
    "fhe_mult_relin_rescale_noalloc": (_I, [_P, ctypes.POINTER(FheCt), ctypes.POINTER(FheCt), _I,
                                            ctypes.POINTER(FheCt), _P]),
    "fhe_set_forms": (_I, [_P, _I, _I, _I]),
    "fhe_profile_reset": (_I, [_P, _I]),
    "fhe_profile_read": (_I, [_P, _I, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)]),
}

KERNEL_CLASSES = ("lift", "ntt_fwd", "ntt_inv", "pointwise", "crt", "limb", "ntt_pw")


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() (no CPU fallback exists)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


class FheError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = lib.fhe_last_error().decode(errors="replace")
        super().__init__(f"{where} failed with {code}: {msg}")
        self.code = code


def _check(rc: int, where: str) -> None:
    if rc != FHE_OK:
        raise FheError(rc, where)


def limbs(bits: int) -> int:
    return (int(bits) + 31) // 32


@dataclass
class Ciphertext:
    """A CipherTensor: data (cnum, 2, L, N) int32 CUDA tensor of uint32 limbs.

    CKKS: modulus 2^logQ.  BGV: modulus Q_level = q0 r^level of logQ bits.
    """

    data: "object"
    logQ: int
    level: int = 0
    log_scale: float = 0.0

    @property
    def cnum(self) -> int:
        return int(self.data.shape[0])

    def c(self) -> FheCt:
        if not self.data.is_contiguous():
            raise ValueError("ciphertext tensor must be contiguous (the C ABI reads a dense [cnum][2][L][N] block)")
        return FheCt(self.data.data_ptr(), self.cnum, self.logQ, self.level, float(self.log_scale))


def _stream():
    import torch

    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _host(arr, dtype) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(arr), dtype=dtype)
    return a


class Context:
    """One ring size and modulus chain; owns tables and keys (allocated through torch)."""

    def __init__(self, logN: int, logQ: int, logP: int, crt: int = FHE_CRT_DIRECT, scheme: int = FHE_SCHEME_CKKS,
                 t: int = 0, bgv_q0: int = 0, bgv_r: int = 0, bgv_levels: int = 0, hamming_weight: int = 0,
                 sigma: float = 0.0):
        import torch

        self.logN, self.logQ, self.logP = int(logN), int(logQ), int(logP)
        self.N = 1 << self.logN
        self.device = torch.device("cuda", torch.cuda.current_device())
        self._torch = torch

        def _alloc(nbytes, user):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), self.device.index)
            except Exception:  # out of memory -> NULL, the library reports FHE_ENOMEM
                return None

        def _free(ptr, nbytes, user):
            torch.cuda.caching_allocator_delete(ptr)

        self._alloc_cb = ALLOC_FN(_alloc)
        self._free_cb = FREE_FN(_free)
        prm = FheParams(int(scheme), self.logN, self.logQ, self.logP, int(crt), int(bgv_levels), int(t), int(bgv_q0),
                        int(bgv_r), int(hamming_weight), float(sigma))
        self.crt = int(crt)
        self.scheme = int(scheme)
        self.t, self.bgv_q0, self.bgv_r, self.bgv_levels = int(t), int(bgv_q0), int(bgv_r), int(bgv_levels)
        h = ctypes.c_void_p()
        _check(lib.fhe_ctx_create(ctypes.byref(prm), self._alloc_cb, self._free_cb, None, ctypes.byref(h)),
               "fhe_ctx_create")
        self.handle = h
        self._ws = {}

    def close(self) -> None:
        if getattr(self, "handle", None):
            lib.fhe_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- memory
    def workspace(self, op: int, logQ: int, cnum: int):
        """A cached device workspace large enough for `op` at (logQ, cnum), one per stream: calls
        on different streams may run concurrently only with different workspaces."""
        nbytes = lib.fhe_workspace_bytes(self.handle, op, int(logQ), int(cnum))
        if nbytes == 0:
            raise FheError(FHE_EINVAL, "fhe_workspace_bytes")
        stream = self._torch.cuda.current_stream()
        key = (op, stream.cuda_stream)
        cur = self._ws.get(key)
        if cur is None or cur.numel() < nbytes:
            if cur is not None:
                cur.record_stream(stream)  # the old buffer may still be in use by queued work
            cur = self._torch.empty(int(nbytes), dtype=self._torch.uint8, device=self.device)
            self._ws[key] = cur
        return cur

    def bgv_bits(self, level: int) -> int:
        """Bit length of Q_level = q0 r^level (BGV)."""
        return (self.bgv_q0 * self.bgv_r ** int(level)).bit_length()

    def empty_ct(self, cnum: int, logQ: int, level: int = 0, log_scale: float = 0.0) -> Ciphertext:
        t = self._torch.empty((int(cnum), 2, limbs(logQ), self.N), dtype=self._torch.int32, device=self.device)
        return Ciphertext(t, int(logQ), int(level), float(log_scale))

    def empty_level(self, cnum: int, level: int) -> Ciphertext:
        """An uninitialised BGV ciphertext batch at `level`."""
        return self.empty_ct(cnum, self.bgv_bits(level), level)

    # ------------------------------------------------------------------ keys
    def keygen(self, seed: int, rot_steps=()) -> None:
        fhe_keygen(self, seed, rot_steps)

    def keygen_inject(self, s, a_pk, e_pk, a_ev, e_ev) -> None:
        fhe_keygen_inject(self, s, a_pk, e_pk, a_ev, e_ev)

    def keygen_rotation(self, step: int, a, e) -> None:
        fhe_keygen_rotation(self, step, a, e)

    def keygen_conjugation(self, a, e) -> None:
        fhe_keygen_conjugation(self, a, e)

    # ------------------------------------------------------------ operations
    def _enc_out(self, cnum, logQ, level, log_scale):
        if self.scheme == FHE_SCHEME_BGV:
            lv = self.bgv_levels if level is None else int(level)
            return self.empty_level(cnum, lv)
        return self.empty_ct(cnum, self.logQ if logQ is None else logQ, log_scale=log_scale)

    def encrypt(self, pt, seed: int, logQ: int | None = None, level: int | None = None,
                log_scale: float = 0.0) -> Ciphertext:
        out = self._enc_out(pt.shape[0], logQ, level, log_scale)
        fhe_encrypt(self, pt, seed, out)
        return out

    def encrypt_inject(self, pt, v, e0, e1, logQ: int | None = None, level: int | None = None,
                       log_scale: float = 0.0) -> Ciphertext:
        out = self._enc_out(pt.shape[0], logQ, level, log_scale)
        fhe_encrypt_inject(self, pt, v, e0, e1, out)
        return out

    def decrypt(self, ct: Ciphertext):
        """CKKS: (cnum, L, N) centred two's-complement limbs.  BGV: (cnum, N) plaintext coefficients mod t."""
        if self.scheme == FHE_SCHEME_BGV:
            out = self._torch.empty((ct.cnum, self.N), dtype=self._torch.int32, device=self.device)
        else:
            out = self._torch.empty((ct.cnum, limbs(ct.logQ), self.N), dtype=self._torch.int32, device=self.device)
        fhe_decrypt(self, ct, out)
        return out

    def mult_relin(self, a: Ciphertext, b: Ciphertext) -> Ciphertext:
        out = self.empty_ct(a.cnum, a.logQ, a.level)
        fhe_mult_relin(self, a, b, out)
        return out

    def mod_switch(self, ct: Ciphertext) -> Ciphertext:
        """BGV modulus switch to level - 1 (fhe_moddown)."""
        out = self.empty_level(ct.cnum, ct.level - 1)
        fhe_moddown(self, ct, out)
        return out

    def mult_relin_rescale(self, a: Ciphertext, b: Ciphertext, k: int) -> Ciphertext:
        out = self.empty_ct(a.cnum, a.logQ - k)
        fhe_mult_relin_rescale(self, a, b, k, out)
        return out

    def rescale(self, ct: Ciphertext, k: int) -> Ciphertext:
        out = self.empty_ct(ct.cnum, ct.logQ - k)
        fhe_rescale(self, ct, k, out)
        return out

    def moddown(self, ct: Ciphertext, logQ: int) -> Ciphertext:
        out = self.empty_ct(ct.cnum, logQ)
        fhe_moddown(self, ct, out)
        return out

    def rotate(self, ct: Ciphertext, step: int) -> Ciphertext:
        out = self.empty_ct(ct.cnum, ct.logQ)
        fhe_rotate(self, ct, step, out)
        return out

    def rotate_hoisted(self, ct: Ciphertext, steps) -> list:
        outs = [self.empty_ct(ct.cnum, ct.logQ) for _ in steps]
        fhe_rotate_hoisted(self, ct, steps, outs)
        return outs

    def conjugate(self, ct: Ciphertext) -> Ciphertext:
        out = self.empty_ct(ct.cnum, ct.logQ)
        fhe_conjugate(self, ct, out)
        return out

    def add(self, a: Ciphertext, b: Ciphertext) -> Ciphertext:
        out = self.empty_ct(a.cnum, a.logQ, a.level)
        fhe_add(self, a, b, out)
        return out

    def sub(self, a: Ciphertext, b: Ciphertext) -> Ciphertext:
        out = self.empty_ct(a.cnum, a.logQ, a.level)
        fhe_sub(self, a, b, out)
        return out

    def negate(self, a: Ciphertext) -> Ciphertext:
        out = self.empty_ct(a.cnum, a.logQ, a.level)
        fhe_negate(self, a, out)
        return out

    def mult_const(self, a: Ciphertext, c: int) -> Ciphertext:
        out = self.empty_ct(a.cnum, a.logQ)
        fhe_mult_const(self, a, c, out)
        return out

    def imult(self, a: Ciphertext) -> Ciphertext:
        out = self.empty_ct(a.cnum, a.logQ)
        fhe_imult(self, a, out)
        return out

    def mult_plain(self, a: Ciphertext, pt, pt_log_scale: float = 0.0) -> Ciphertext:
        out = self.empty_ct(a.cnum, a.logQ)
        fhe_mult_plain(self, a, pt, pt_log_scale, out)
        return out

    def add_const_vec(self, a: Ciphertext, values, shift: int) -> Ciphertext:
        out = self.empty_ct(a.cnum, a.logQ)
        fhe_add_const_vec(self, a, values, shift, out)
        return out

    def ring_mul(self, a, b, logOut: int):
        cnum = a.shape[0]
        out = self._torch.empty((cnum, limbs(logOut), self.N), dtype=self._torch.int32, device=self.device)
        fhe_ring_mul(self, a, b, logOut, out)
        return out


# ------------------------------------------------ C-ABI-named thin wrappers
def fhe_keygen(ctx: Context, seed: int, rot_steps=()) -> None:
    steps = np.ascontiguousarray(np.asarray(list(rot_steps), dtype=np.int32))
    _check(lib.fhe_keygen(ctx.handle, int(seed) & (2 ** 64 - 1), steps.ctypes.data if steps.size else None,
                          int(steps.size)), "fhe_keygen")


def fhe_keygen_inject(ctx: Context, s, a_pk, e_pk, a_ev, e_ev) -> None:
    N = ctx.N
    s = _host(s, np.int8).reshape(N)
    a_pk = _host(a_pk, np.uint32).reshape(limbs(ctx.logQ), N)
    e_pk = _host(e_pk, np.int32).reshape(N)
    a_ev = _host(a_ev, np.uint32).reshape(limbs(ctx.logQ + ctx.logP), N)
    e_ev = _host(e_ev, np.int32).reshape(N)
    _check(lib.fhe_keygen_inject(ctx.handle, s.ctypes.data, a_pk.ctypes.data, e_pk.ctypes.data, a_ev.ctypes.data,
                                 e_ev.ctypes.data), "fhe_keygen_inject")


def fhe_keygen_rotation(ctx: Context, step: int, a, e) -> None:
    N = ctx.N
    a = _host(a, np.uint32).reshape(limbs(ctx.logQ + ctx.logP), N)
    e = _host(e, np.int32).reshape(N)
    _check(lib.fhe_keygen_rotation(ctx.handle, int(step), a.ctypes.data, e.ctypes.data), "fhe_keygen_rotation")


def fhe_keygen_conjugation(ctx: Context, a, e) -> None:
    N = ctx.N
    a = _host(a, np.uint32).reshape(limbs(ctx.logQ + ctx.logP), N)
    e = _host(e, np.int32).reshape(N)
    _check(lib.fhe_keygen_conjugation(ctx.handle, a.ctypes.data, e.ctypes.data), "fhe_keygen_conjugation")


def fhe_sample(seed: int, tag0: int, tag1: int, kind: int, n: int, param: int = 0, sigma: float = 3.2) -> np.ndarray:
    """The library's host sampler (see include/fhe.h): uniform limbs (L, n) uint32, ternary / HWT int8 (n,),
    Gaussian int32 (n,)."""
    if kind == FHE_SAMPLE_UNIFORM:
        out = np.zeros((limbs(param), n), dtype=np.uint32)
    elif kind in (FHE_SAMPLE_TERNARY, FHE_SAMPLE_HWT):
        out = np.zeros(n, dtype=np.int8)
    else:
        out = np.zeros(n, dtype=np.int32)
    _check(lib.fhe_sample(int(seed) & (2 ** 64 - 1), int(tag0), int(tag1), int(kind), int(n), int(param),
                          float(sigma), out.ctypes.data), "fhe_sample")
    return out


def _dev(t, dtype, shape):
    import torch

    assert t.is_cuda and t.dtype == dtype and t.is_contiguous() and tuple(t.shape) == tuple(shape), \
        (t.dtype, tuple(t.shape), shape)
    return t.data_ptr()


def fhe_encrypt(ctx: Context, pt, seed: int, out: Ciphertext) -> None:
    import torch

    cnum, L, N = out.cnum, limbs(out.logQ), ctx.N
    ws = ctx.workspace(FHE_OP_ENCRYPT, ctx.logQ, cnum)
    oc = out.c()
    _check(lib.fhe_encrypt(ctx.handle, _dev(pt, torch.int32, (cnum, L, N)), int(seed) & (2 ** 64 - 1),
                           ctypes.byref(oc), ws.data_ptr(), ws.numel(), _stream()), "fhe_encrypt")


def fhe_encrypt_inject(ctx: Context, pt, v, e0, e1, out: Ciphertext) -> None:
    import torch

    cnum, L, N = out.cnum, limbs(out.logQ), ctx.N
    ws = ctx.workspace(FHE_OP_ENCRYPT, ctx.logQ, cnum)
    oc = out.c()
    _check(lib.fhe_encrypt_inject(ctx.handle, _dev(pt, torch.int32, (cnum, L, N)), _dev(v, torch.int8, (cnum, N)),
                                  _dev(e0, torch.int32, (cnum, N)), _dev(e1, torch.int32, (cnum, N)),
                                  ctypes.byref(oc), ws.data_ptr(), ws.numel(), _stream()), "fhe_encrypt_inject")


def fhe_decrypt(ctx: Context, ct: Ciphertext, out) -> None:
    import torch

    ws = ctx.workspace(FHE_OP_DECRYPT, ct.logQ, ct.cnum)
    c = ct.c()
    shape = (ct.cnum, ctx.N) if ctx.scheme == FHE_SCHEME_BGV else (ct.cnum, limbs(ct.logQ), ctx.N)
    _check(lib.fhe_decrypt(ctx.handle, ctypes.byref(c), _dev(out, torch.int32, shape), ws.data_ptr(), ws.numel(),
                           _stream()), "fhe_decrypt")


def fhe_mult_relin(ctx: Context, a: Ciphertext, b: Ciphertext, out: Ciphertext) -> None:
    ws = ctx.workspace(FHE_OP_MULT, a.logQ, a.cnum)
    ca, cb, co = a.c(), b.c(), out.c()
    _check(lib.fhe_mult_relin(ctx.handle, ctypes.byref(ca), ctypes.byref(cb), ctypes.byref(co), ws.data_ptr(),
                              ws.numel(), _stream()), "fhe_mult_relin")
    out.log_scale = co.log_scale


def fhe_mult_relin_rescale(ctx: Context, a: Ciphertext, b: Ciphertext, k: int, out: Ciphertext) -> None:
    ws = ctx.workspace(FHE_OP_MULT, a.logQ, a.cnum)
    ca, cb, co = a.c(), b.c(), out.c()
    _check(lib.fhe_mult_relin_rescale(ctx.handle, ctypes.byref(ca), ctypes.byref(cb), int(k), ctypes.byref(co),
                                      ws.data_ptr(), ws.numel(), _stream()), "fhe_mult_relin_rescale")
    out.log_scale = co.log_scale


def fhe_mult_relin_rescale_noalloc(ctx: Context, a: Ciphertext, b: Ciphertext, k: int, out: Ciphertext) -> None:
    """fhe_mult_relin_rescale without a workspace, for callers that cannot allocate (static 32 MiB scratch)."""
    ca, cb, co = a.c(), b.c(), out.c()
    _check(lib.fhe_mult_relin_rescale_noalloc(ctx.handle, ctypes.byref(ca), ctypes.byref(cb), int(k),
                                              ctypes.byref(co), _stream()), "fhe_mult_relin_rescale_noalloc")
    out.log_scale = co.log_scale


def fhe_mult_relin_rescale_ragged(ctx: Context, a, b, out, item_logQ, logQ_max: int, k: int, ws=None) -> None:
    """Pairs at different levels in one batch: a, b, out (cnum, 2, L_pad, N) int32 CUDA tensors,
    item_logQ a CUDA int32 tensor (cnum,).  `ws`: optional caller workspace (uint8 CUDA tensor)."""
    import torch

    cnum, two, L_pad, N = a.shape
    if ws is None:
        ws = ctx.workspace(FHE_OP_MULT_RAGGED, logQ_max, cnum)
    _check(lib.fhe_mult_relin_rescale_ragged(
        ctx.handle, _dev(a, torch.int32, (cnum, 2, L_pad, N)), _dev(b, torch.int32, (cnum, 2, L_pad, N)),
        _dev(out, torch.int32, (cnum, 2, L_pad, N)), int(cnum), int(L_pad), _dev(item_logQ, torch.int32, (cnum,)),
        int(logQ_max), int(k), ws.data_ptr(), ws.numel(), _stream()), "fhe_mult_relin_rescale_ragged")


def fhe_mult_relin_rescale_batch(groups, k: int, sched=None) -> None:
    """Ragged batches of several ring sizes in one call, the transform stages of all of them as single
    work-table launches.  groups: sequence of (ctx, a, b, out, item_logQ, logQ_max, ws) with the tensors of
    fhe_mult_relin_rescale_ragged and a distinct workspace per group (uint8 CUDA tensor of at least
    fhe_workspace_bytes(FHE_OP_MULT_RAGGED, logQ_max, cnum)); sched: (col_ctas_per_sm, row_ctas_per_sm,
    col_unit_rows) or None for the library's default."""
    import torch

    arr = (FheBatchGroup * len(groups))()
    for i, (ctx, a, b, out, item_logQ, logQ_max, ws) in enumerate(groups):
        cnum, two, L_pad, N = a.shape
        shape = (cnum, 2, L_pad, N)
        arr[i] = FheBatchGroup(ctx.handle, _dev(a, torch.int32, shape), _dev(b, torch.int32, shape),
                               _dev(out, torch.int32, shape), _dev(item_logQ, torch.int32, (cnum,)), int(cnum),
                               int(L_pad), int(logQ_max), ws.data_ptr(), ws.numel())
    sp = ctypes.byref(FheBatchSched(*[int(x) for x in sched])) if sched is not None else None
    _check(lib.fhe_mult_relin_rescale_batch(arr, len(groups), int(k), sp, _stream()),
           "fhe_mult_relin_rescale_batch")


def fhe_rescale(ctx: Context, ct: Ciphertext, k: int, out: Ciphertext) -> None:
    ci, co = ct.c(), out.c()
    _check(lib.fhe_rescale(ctx.handle, ctypes.byref(ci), int(k), ctypes.byref(co), _stream()), "fhe_rescale")
    out.log_scale = co.log_scale


def fhe_moddown(ctx: Context, ct: Ciphertext, out: Ciphertext) -> None:
    ci, co = ct.c(), out.c()
    _check(lib.fhe_moddown(ctx.handle, ctypes.byref(ci), ctypes.byref(co), _stream()), "fhe_moddown")
    out.log_scale = co.log_scale


def fhe_rotate(ctx: Context, ct: Ciphertext, step: int, out: Ciphertext, ws=None) -> None:
    if ws is None:
        ws = ctx.workspace(FHE_OP_ROTATE, ct.logQ, ct.cnum)
    ci, co = ct.c(), out.c()
    _check(lib.fhe_rotate(ctx.handle, ctypes.byref(ci), int(step), ctypes.byref(co), ws.data_ptr(), ws.numel(),
                          _stream()), "fhe_rotate")
    out.log_scale = co.log_scale


def fhe_rotate_hoisted(ctx: Context, ct: Ciphertext, steps, outs, ws=None) -> None:
    if ws is None:
        ws = ctx.workspace(FHE_OP_ROTATE, ct.logQ, ct.cnum)
    st = np.ascontiguousarray(np.asarray(list(steps), dtype=np.int32))
    cs = [o.c() for o in outs]
    arr = (ctypes.POINTER(FheCt) * len(cs))(*[ctypes.pointer(c) for c in cs])
    ci = ct.c()
    _check(lib.fhe_rotate_hoisted(ctx.handle, ctypes.byref(ci), st.ctypes.data, int(st.size), arr, ws.data_ptr(),
                                  ws.numel(), _stream()), "fhe_rotate_hoisted")
    for o, c in zip(outs, cs):
        o.log_scale = c.log_scale


def fhe_conjugate(ctx: Context, ct: Ciphertext, out: Ciphertext, ws=None) -> None:
    if ws is None:
        ws = ctx.workspace(FHE_OP_ROTATE, ct.logQ, ct.cnum)
    ci, co = ct.c(), out.c()
    _check(lib.fhe_conjugate(ctx.handle, ctypes.byref(ci), ctypes.byref(co), ws.data_ptr(), ws.numel(), _stream()),
           "fhe_conjugate")
    out.log_scale = co.log_scale


def fhe_add(ctx: Context, a: Ciphertext, b: Ciphertext, out: Ciphertext) -> None:
    ca, cb, co = a.c(), b.c(), out.c()
    _check(lib.fhe_add(ctx.handle, ctypes.byref(ca), ctypes.byref(cb), ctypes.byref(co), _stream()), "fhe_add")
    out.log_scale = co.log_scale


def fhe_sub(ctx: Context, a: Ciphertext, b: Ciphertext, out: Ciphertext) -> None:
    ca, cb, co = a.c(), b.c(), out.c()
    _check(lib.fhe_sub(ctx.handle, ctypes.byref(ca), ctypes.byref(cb), ctypes.byref(co), _stream()), "fhe_sub")
    out.log_scale = co.log_scale


def fhe_negate(ctx: Context, a: Ciphertext, out: Ciphertext) -> None:
    ca, co = a.c(), out.c()
    _check(lib.fhe_negate(ctx.handle, ctypes.byref(ca), ctypes.byref(co), _stream()), "fhe_negate")
    out.log_scale = co.log_scale


def fhe_mult_const(ctx: Context, a: Ciphertext, c: int, out: Ciphertext) -> None:
    ca, co = a.c(), out.c()
    _check(lib.fhe_mult_const(ctx.handle, ctypes.byref(ca), int(c), ctypes.byref(co), _stream()), "fhe_mult_const")
    out.log_scale = co.log_scale


def fhe_add_const(ctx: Context, a: Ciphertext, value: int, shift: int, out: Ciphertext) -> None:
    ca, co = a.c(), out.c()
    _check(lib.fhe_add_const(ctx.handle, ctypes.byref(ca), int(value), int(shift), ctypes.byref(co), _stream()),
           "fhe_add_const")
    out.log_scale = co.log_scale


def fhe_add_const_vec(ctx: Context, a: Ciphertext, values, shift: int, out: Ciphertext) -> None:
    """values: a CUDA int64 tensor (cnum,)."""
    import torch

    ca, co = a.c(), out.c()
    _check(lib.fhe_add_const_vec(ctx.handle, ctypes.byref(ca), _dev(values, torch.int64, (a.cnum,)), int(shift),
                                 ctypes.byref(co), _stream()), "fhe_add_const_vec")
    out.log_scale = co.log_scale


def fhe_imult(ctx: Context, a: Ciphertext, out: Ciphertext) -> None:
    ca, co = a.c(), out.c()
    _check(lib.fhe_imult(ctx.handle, ctypes.byref(ca), ctypes.byref(co), _stream()), "fhe_imult")
    out.log_scale = co.log_scale


def fhe_mult_plain(ctx: Context, a: Ciphertext, pt, pt_log_scale: float, out: Ciphertext) -> None:
    """pt: a CUDA int32 tensor (pt_cnum, L, N) of uint32 limbs, pt_cnum = cnum or 1 (broadcast)."""
    import torch

    pc = int(pt.shape[0])
    ws = ctx.workspace(FHE_OP_MULT_PLAIN, a.logQ, a.cnum)
    ca, co = a.c(), out.c()
    _check(lib.fhe_mult_plain(ctx.handle, ctypes.byref(ca), _dev(pt, torch.int32, (pc, limbs(a.logQ), ctx.N)), pc,
                              float(pt_log_scale), ctypes.byref(co), ws.data_ptr(), ws.numel(), _stream()),
           "fhe_mult_plain")
    out.log_scale = co.log_scale


def fhe_ring_mul(ctx: Context, a, b, logOut: int, out) -> None:
    import torch

    cnum, La, N = a.shape
    Lb = b.shape[1]
    ws = ctx.workspace(FHE_OP_RING_MUL, 32 * max(La, Lb), cnum)
    _check(lib.fhe_ring_mul(ctx.handle, _dev(a, torch.int32, (cnum, La, N)), int(La),
                            _dev(b, torch.int32, (cnum, Lb, N)), int(Lb), int(logOut),
                            _dev(out, torch.int32, (cnum, limbs(logOut), N)), int(cnum), ws.data_ptr(), ws.numel(),
                            _stream()), "fhe_ring_mul")


def fhe_ckks_encode(ctx: Context, z, log_scale: int, logQ: int):
    """z: CUDA complex128 tensor (cnum, N/2) -> plaintext limbs (cnum, ceil(logQ/32), N) int32."""
    import torch

    cnum = int(z.shape[0])
    pt = torch.empty((cnum, limbs(logQ), ctx.N), dtype=torch.int32, device=ctx.device)
    ws = ctx.workspace(FHE_OP_ENCODE, 1, cnum)
    _check(lib.fhe_ckks_encode(ctx.handle, _dev(z, torch.complex128, (cnum, ctx.N // 2)), cnum, int(log_scale),
                               int(logQ), pt.data_ptr(), ws.data_ptr(), ws.numel(), _stream()), "fhe_ckks_encode")
    return pt


def fhe_ckks_decode(ctx: Context, pt, logQ: int, log_scale: float):
    """pt: CUDA int32 tensor (cnum, ceil(logQ/32), N) of signed two's-complement limbs -> complex128 (cnum, N/2)."""
    import torch

    cnum = int(pt.shape[0])
    z = torch.empty((cnum, ctx.N // 2), dtype=torch.complex128, device=ctx.device)
    ws = ctx.workspace(FHE_OP_ENCODE, 1, cnum)
    _check(lib.fhe_ckks_decode(ctx.handle, _dev(pt, torch.int32, (cnum, limbs(logQ), ctx.N)), cnum, int(logQ),
                               float(log_scale), z.data_ptr(), ws.data_ptr(), ws.numel(), _stream()),
           "fhe_ckks_decode")
    return z


def fhe_bgv_encode(ctx: Context, slots, logQ: int):
    """slots: CUDA int32 tensor (cnum, N) of values mod t -> an encryption input (cnum, ceil(logQ/32), N)."""
    import torch

    cnum = int(slots.shape[0])
    L = limbs(logQ)
    pt = torch.zeros((cnum, L, ctx.N), dtype=torch.int32, device=ctx.device)
    _check(lib.fhe_bgv_encode(ctx.handle, _dev(slots, torch.int32, (cnum, ctx.N)), cnum, pt.data_ptr(), L * ctx.N,
                              _stream()), "fhe_bgv_encode")
    return pt


def fhe_bgv_decode(ctx: Context, coeffs):
    """coeffs: CUDA int32 tensor (cnum, N) of plaintext coefficients mod t (fhe_decrypt's BGV output) -> slots."""
    import torch

    cnum = int(coeffs.shape[0])
    slots = torch.empty((cnum, ctx.N), dtype=torch.int32, device=ctx.device)
    _check(lib.fhe_bgv_decode(ctx.handle, _dev(coeffs, torch.int32, (cnum, ctx.N)), ctx.N, cnum, slots.data_ptr(),
                              _stream()), "fhe_bgv_decode")
    return slots


def fhe_primes_for_bound(bound_bits: int) -> int:
    return int(lib.fhe_primes_for_bound(int(bound_bits)))


def fhe_set_forms(ctx: Context, crt: int, lift: int = FHE_LIFT_AUTO, ntt: int = FHE_NTT_FUSED) -> None:
    _check(lib.fhe_set_forms(ctx.handle, int(crt), int(lift), int(ntt)), "fhe_set_forms")
    ctx.crt = int(crt)


def fhe_profile_reset(ctx: Context, enable: bool) -> None:
    _check(lib.fhe_profile_reset(ctx.handle, 1 if enable else 0), "fhe_profile_reset")


def fhe_profile_read(ctx: Context) -> dict:
    """{class name: (launches, milliseconds)} since the last reset."""
    out = {}
    for k, name in enumerate(KERNEL_CLASSES):
        n = ctypes.c_int64()
        ms = ctypes.c_double()
        _check(lib.fhe_profile_read(ctx.handle, k, ctypes.byref(n), ctypes.byref(ms)), "fhe_profile_read")
        out[name] = (int(n.value), float(ms.value))
    return out


def fhe_sync(ctx: Context) -> None:
    _check(lib.fhe_sync(ctx.handle), "fhe_sync")
