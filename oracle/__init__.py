"""CPU oracle of the chaotic video cipher (arXiv 2302.07411), test infrastructure.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product (the CUDA library and its
Python binding) never does: it shares no code with this oracle.

The arithmetic lives in ``vc_oracle.c`` (plain C, single thread, binary64 with
FMA contraction off); this module compiles it with gcc and wraps it with ctypes.
Each wrapper names the paper passage it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vc_oracle.c")
_HDR = os.path.join(_HERE, "vc_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

PLCM, DLASM, LOGISTIC = 0, 1, 2
PRBG_PLCM_PAIR, PRBG_LASM_PAIR, PRBG_LASM_SINGLE, PRBG_LOGI_PAIR = 0, 1, 2, 3

# gcc flags: one IEEE rounding per operation, no contraction into fma, no
# fast-math reassociation.
CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
          "-Wall", "-Wextra", "-Wno-unused-parameter"]


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (idempotent)."""
    with _lock:
        stale = (not os.path.exists(_LIB) or
                 os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
        if force or stale:
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


class _Prbg(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pos", C.c_int32), ("len", C.c_int32),
                ("buf", C.c_uint8 * 12), ("s", C.c_double * 6)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        d, i32, i64, u64, p = C.c_double, C.c_int, C.c_int64, C.c_uint64, C.c_void_p
        sig = {
            "orc_csin": (d, [d]),
            "orc_sin_coef": (d, [i32]),
            "orc_cos_coef": (d, [i32]),
            "orc_constants": (None, [p]),
            "orc_plcm_step": (d, [d, d]),
            "orc_lasm_step": (None, [p, p, d]),
            "orc_logistic_step": (d, [d, d]),
            "orc_mantissa_bytes": (None, [d, p]),
            "orc_prbg_init": (None, [p, i32, p]),
            "orc_prbg_bytes": (None, [p, p, u64]),
            "orc_key_valid": (i32, [i32, p]),
            "orc_layout_valid": (i32, [i32, i32, i32, i32, i32]),
            "orc_ctx_size": (C.c_size_t, [i32]),
            "orc_ctx_init": (i32, [p, i32, p, i32, i32, i32, i32, i32]),
            "orc_sub_params": (None, [p, i32, p]),
            "orc_set_sub_params": (None, [p, i32, p]),
            "orc_next_sc": (i64, [p]),
            "orc_ktable": (None, [i32, i64, p]),
            "orc_confuse": (None, [i32, i32, i32, p, p, p]),
            "orc_unconfuse": (None, [i32, i32, i32, p, p, p]),
            "orc_diffuse": (None, [i32, i32, i32, i32, p, p, p]),
            "orc_undiffuse": (None, [i32, i32, i32, i32, p, p, p]),
            "orc_diffuse_pc": (None, [i32, i32, i32, i32, p, p, p]),
            "orc_undiffuse_pc": (None, [i32, i32, i32, i32, p, p, p]),
            "orc_ctx_set_chains": (i32, [p, i32]),
            "orc_encrypt_frame": (i32, [p, p, p, p]),
            "orc_decrypt_frame": (i32, [p, p, p, p]),
            "orc_frame_keystream": (i32, [p, p, p]),
            "orc_save_state": (None, [p, p]),
            "orc_load_state": (None, [p, p]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


# ---------------------------------------------------------------- primitives

def csin(t: float) -> float:
    """The cipher's sine (reading of 'sin' in Eq. 1 and Eq. 6)."""
    return lib().orc_csin(float(t))


def sin_coef(k: int) -> float:
    return lib().orc_sin_coef(k)


def cos_coef(k: int) -> float:
    return lib().orc_cos_coef(k)


def constants() -> dict:
    out = np.zeros(5, dtype=np.float64)
    lib().orc_constants(_ptr(out))
    return dict(zip(["PI", "TWO_PI", "TWO_OVER_PI", "PIO2_HI", "PIO2_LO"], map(float, out)))


def plcm_step(x: float, p: float) -> float:
    """Eq. 5."""
    return lib().orc_plcm_step(float(x), float(p))


def lasm_step(x: float, y: float, mu: float) -> tuple[float, float]:
    """Eq. 6."""
    xs, ys = C.c_double(x), C.c_double(y)
    lib().orc_lasm_step(C.byref(xs), C.byref(ys), float(mu))
    return xs.value, ys.value


def logistic_step(x: float, r: float) -> float:
    """The logistic map x' = (r x)(1 - x), the third map of the strategy
    (Sec. 7, advantage iii)."""
    return lib().orc_logistic_step(float(x), float(r))


def mantissa_bytes(v: float) -> bytes:
    """Sec. 3: six bytes of the mantissa of an iterate (low 48 bits, LSB first)."""
    out = (C.c_uint8 * 6)()
    lib().orc_mantissa_bytes(float(v), out)
    return bytes(out)


def prbg_bytes(kind: int, params, nbytes: int, chunks=None) -> bytes:
    """Sec. 3 byte stream of a PRBG with the given map parameters; ``chunks``
    optionally splits the request into pieces (the stream must not care)."""
    g = _Prbg()
    prm = np.zeros(6, dtype=np.float64)
    prm[: len(params)] = params
    lib().orc_prbg_init(C.byref(g), kind, _ptr(prm))
    out = np.zeros(nbytes, dtype=np.uint8)
    sizes = [nbytes] if chunks is None else list(chunks)
    assert sum(sizes) == nbytes
    off = 0
    for s in sizes:
        lib().orc_prbg_bytes(C.byref(g), C.c_void_p(out.ctypes.data + off), s)
        off += s
    return out.tobytes()


def key_valid(kind: int, key) -> bool:
    k = np.zeros(4, dtype=np.float64)
    k[: len(key)] = key
    return bool(lib().orc_key_valid(kind, _ptr(k)))


def layout_valid(H, W, C_, n, rounds=5) -> bool:
    return bool(lib().orc_layout_valid(H, W, C_, n, rounds))


def subframe_bounds(H: int, W: int, C_: int, n: int) -> np.ndarray:
    """Byte offsets C*pi_i, pi_i = floor(i*P/n), i = 0..n (subframe reading)."""
    P = H * W
    return np.array([C_ * ((i * P) // n) for i in range(n + 1)], dtype=np.int64)


def ktable(H: int, sc: int) -> np.ndarray:
    """Eq. 1 shift table k(alpha) = floor(s_c * sin(2*pi*alpha/H))."""
    k = np.zeros(H, dtype=np.int64)
    lib().orc_ktable(H, int(sc), _ptr(k))
    return k


def confuse(X: np.ndarray, k: np.ndarray) -> np.ndarray:
    """Eq. 1 on an H x W x C frame."""
    X = np.ascontiguousarray(X, dtype=np.uint8)
    H, W, Cc = X.shape
    k = np.ascontiguousarray(k, dtype=np.int64)
    Y = np.empty_like(X)
    lib().orc_confuse(H, W, Cc, _ptr(k), _ptr(X), _ptr(Y))
    return Y


def unconfuse(Y: np.ndarray, k: np.ndarray) -> np.ndarray:
    """Eq. 2."""
    Y = np.ascontiguousarray(Y, dtype=np.uint8)
    H, W, Cc = Y.shape
    k = np.ascontiguousarray(k, dtype=np.int64)
    X = np.empty_like(Y)
    lib().orc_unconfuse(H, W, Cc, _ptr(k), _ptr(Y), _ptr(X))
    return X


def _ks_ptrs(ks_list):
    arrs = [np.ascontiguousarray(np.frombuffer(bytes(b), dtype=np.uint8)) if not isinstance(b, np.ndarray)
            else np.ascontiguousarray(b, dtype=np.uint8) for b in ks_list]
    ptrs = (C.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])
    return arrs, ptrs


def diffuse(Y: np.ndarray, ks_list, n: int) -> np.ndarray:
    """Eq. 3 over all n subframes of one round; ks_list[i] = subframe i's bytes."""
    Y = np.ascontiguousarray(Y, dtype=np.uint8)
    H, W, Cc = Y.shape
    keep, ptrs = _ks_ptrs(ks_list)
    out = np.empty_like(Y)
    lib().orc_diffuse(H, W, Cc, n, ptrs, _ptr(Y), _ptr(out))
    return out


def undiffuse(Xc: np.ndarray, ks_list, n: int) -> np.ndarray:
    """Eq. 4."""
    Xc = np.ascontiguousarray(Xc, dtype=np.uint8)
    H, W, Cc = Xc.shape
    keep, ptrs = _ks_ptrs(ks_list)
    out = np.empty_like(Xc)
    lib().orc_undiffuse(H, W, Cc, n, ptrs, _ptr(Xc), _ptr(out))
    return out


def diffuse_pc(Y: np.ndarray, ks_list, n: int) -> np.ndarray:
    """Eq. 3 with one chain per colour channel (the alternative reading)."""
    Y = np.ascontiguousarray(Y, dtype=np.uint8)
    H, W, Cc = Y.shape
    keep, ptrs = _ks_ptrs(ks_list)
    out = np.empty_like(Y)
    lib().orc_diffuse_pc(H, W, Cc, n, ptrs, _ptr(Y), _ptr(out))
    return out


def undiffuse_pc(Xc: np.ndarray, ks_list, n: int) -> np.ndarray:
    """Eq. 4 with one chain per colour channel."""
    Xc = np.ascontiguousarray(Xc, dtype=np.uint8)
    H, W, Cc = Xc.shape
    keep, ptrs = _ks_ptrs(ks_list)
    out = np.empty_like(Xc)
    lib().orc_undiffuse_pc(H, W, Cc, n, ptrs, _ptr(Xc), _ptr(out))
    return out


# ---------------------------------------------------------------- the cipher

class OracleCipher:
    """One video stream of the cipher (Alg. 1 + Alg. 2, executed serially).

    kind: PLCM (key = x0^1, p^1, x0^2, p^2), DLASM (key = x0, mu, y0) or
    LOGISTIC (key = x0^1, r^1, x0^2, r^2).  per_channel selects one diffusion
    chain per colour channel instead of the byte chain (reading R4).
    Frames are H x W x C uint8 arrays; state advances one frame per call.
    """

    def __init__(self, kind: int, key, H: int, W: int, C_: int = 3, n: int = 4, rounds: int = 5,
                 per_channel: bool = False):
        self.kind, self.H, self.W, self.C, self.n, self.rounds = kind, H, W, C_, n, rounds
        self._buf = np.zeros(lib().orc_ctx_size(n), dtype=np.uint8)
        k = np.zeros(4, dtype=np.float64)
        k[: len(key)] = key
        rc = lib().orc_ctx_init(_ptr(self._buf), kind, _ptr(k), H, W, C_, n, rounds)
        if rc == 1:
            raise ValueError("key outside the valid ranges of Eq. 5 / Eq. 6")
        if rc == 2:
            raise ValueError("invalid layout")
        if per_channel and lib().orc_ctx_set_chains(_ptr(self._buf), 1) != 0:
            raise ValueError("per-channel chains need at least 2 pixels per subframe")
        self.N = H * W * C_
        self.last_sc = None

    @property
    def ptr(self):
        return _ptr(self._buf)

    def sub_params(self, i: int) -> np.ndarray:
        out = np.zeros(6, dtype=np.float64)
        lib().orc_sub_params(self.ptr, i, _ptr(out))
        return out

    def set_sub_params(self, i: int, params) -> None:
        """Test hook: restart subframe i's PRBG (Alg. 2) from these map
        parameters, e.g. an orbit a test can compute exactly."""
        prm = np.zeros(6, dtype=np.float64)
        prm[: len(params)] = params
        lib().orc_set_sub_params(self.ptr, i, _ptr(prm))

    def _run(self, fn, frames: np.ndarray) -> np.ndarray:
        frames = np.ascontiguousarray(frames, dtype=np.uint8)
        single = frames.ndim == 3
        if single:
            frames = frames[None]
        assert frames.shape[1:] == (self.H, self.W, self.C), frames.shape
        out = np.empty_like(frames)
        sc = C.c_int64(0)
        for f in range(frames.shape[0]):
            rc = fn(self.ptr, C.c_void_p(frames.ctypes.data + f * self.N),
                    C.c_void_p(out.ctypes.data + f * self.N), C.byref(sc))
            if rc != 0:
                raise MemoryError("oracle allocation failed")
            self.last_sc = sc.value
        return out[0] if single else out

    def encrypt(self, frames: np.ndarray) -> np.ndarray:
        return self._run(lib().orc_encrypt_frame, frames)

    def decrypt(self, frames: np.ndarray) -> np.ndarray:
        return self._run(lib().orc_decrypt_frame, frames)

    def frame_keystream(self):
        """(concatenated r*S_i bytes of every subframe, s_c) of the next frame."""
        out = np.zeros(self.N * self.rounds, dtype=np.uint8)
        sc = C.c_int64(0)
        lib().orc_frame_keystream(self.ptr, _ptr(out), C.byref(sc))
        return out, sc.value

    def save_state(self) -> bytes:
        out = np.zeros_like(self._buf)
        lib().orc_save_state(self.ptr, _ptr(out))
        return out.tobytes()

    def load_state(self, state: bytes) -> None:
        src = np.frombuffer(state, dtype=np.uint8).copy()
        lib().orc_load_state(self.ptr, _ptr(src))
