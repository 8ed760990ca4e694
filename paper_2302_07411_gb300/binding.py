"""Thin Python binding of the C ABI in include/vcrypt.h (ctypes).

Argument marshalling only: every step of the cipher runs in libvcrypt.so's
CUDA kernels.  PyTorch supplies device memory (tensors) and the current CUDA
stream.  The functions carry the C names; ``Cipher`` wraps a context.
If the library is not built this module raises instead of falling back.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvcrypt.so")
_lib = None

VC_OK = 0
VC_PLCM, VC_2DLASM, VC_LOGISTIC = 0, 1, 2
VC_OPT_CHUNK, VC_OPT_PLCM_INT, VC_OPT_KS_LANES, VC_OPT_OVERLAP, VC_OPT_TILE_ROWS, VC_OPT_KS_SM_WARPS = 1, 2, 3, 4, 5, 6
VC_OPT_RUNAHEAD_CALLS, VC_OPT_DIFFUSION = 7, 8
VC_BOPT_GRAPH, VC_BOPT_CTAS_PER_SM, VC_BOPT_RUNAHEAD, VC_BOPT_SINE, VC_BOPT_SPLIT, VC_BOPT_KS_PLACE = 1, 2, 3, 4, 5, 6
VC_BOPT_KS_PRIORITY, VC_BOPT_KS_URGENT = 7, 8
VC_SOPT_QUEUED_TICKS, VC_SOPT_LANES = 100, 101
ERRORS = {1: "VC_ERR_ARG", 2: "VC_ERR_KEY_RANGE", 3: "VC_ERR_LAYOUT", 4: "VC_ERR_CUDA", 5: "VC_ERR_OOM",
          6: "VC_ERR_TIMEOUT", 7: "VC_ERR_SEQUENCE", 8: "VC_ERR_STATE", 9: "VC_ERR_UNSUPPORTED"}


class VcError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = lib().vc_last_error().decode(errors="replace") if _lib is not None else ""
        super().__init__(f"{where}: {ERRORS.get(code, code)} ({msg})")


class vc_key(C.Structure):
    _fields_ = [("kind", C.c_int32), ("k", C.c_double * 4)]


class vc_job(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("direction", C.c_int32), ("d_in", C.c_void_p), ("d_out", C.c_void_p),
                ("nframes", C.c_int32)]


class vc_layout(C.Structure):
    _fields_ = [("height", C.c_int32), ("width", C.c_int32), ("channels", C.c_int32),
                ("n_subframes", C.c_int32), ("rounds", C.c_int32)]


def lib():
    """Load libvcrypt.so (built by paper_2302_07411_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() (no CPU fallback exists)")
        L = C.CDLL(LIB_PATH)
        p, i32, i64, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t
        sig = {
            "enc_init": (C.c_int, [p, p, p]),
            "encrypt_frames": (C.c_int, [p, p, p, i32, p]),
            "decrypt_frames": (C.c_int, [p, p, p, i32, p]),
            "crypt_frames_host": (C.c_int, [p, i32, p, p, i32, p]),
            "crypt_frames_host_async": (C.c_int, [p, i32, p, p, i32, p, p]),
            "encrypt_frames_pitched": (C.c_int, [p, p, p, i32, sz, p]),
            "decrypt_frames_pitched": (C.c_int, [p, p, p, i32, sz, p]),
            "vc_dbg_call_plan": (C.c_int, [p, i32, p, i32, p]),
            "vc_dbg_batch_split": (C.c_int, [p]),
            "vc_dbg_fp64_peak": (C.c_int, [C.POINTER(C.c_double), p]),
            "vc_dbg_imad_peak": (C.c_int, [C.POINTER(C.c_double), p]),
            "vc_dbg_plcm_latency": (C.c_int, [C.c_double, C.c_double, i32, C.POINTER(C.c_double), p]),
            "encrypt_frames_static": (C.c_int, [p, p, p, i32, p]),
            "vc_batcher_create": (C.c_int, [p]),
            "vc_batch_submit": (C.c_int, [p, p, i32, p]),
            "vc_batcher_set_option": (C.c_int, [p, i32, i64]),
            "vc_batcher_destroy": (None, [p]),
            "vc_batch_prefetch": (C.c_int, [p, p, i32]),
            "vc_batch_ready": (C.c_int, [p, p, i32]),
            "enc_state_size": (sz, [p]),
            "enc_save_state": (C.c_int, [p, p, C.POINTER(C.c_size_t)]),
            "enc_load_state": (C.c_int, [p, p, sz]),
            "enc_frame_index": (i64, [p]),
            "enc_sync_status": (C.c_int, [p]),
            "enc_set_chunk": (C.c_int, [p, i32]),
            "enc_destroy": (None, [p]),
            "enc_join": (C.c_int, [p, p]),
            "enc_destroy_async": (None, [p]),
            "enc_profile_enable": (C.c_int, [p, i32]),
            "enc_profile_read": (C.c_int, [p, p, p]),
            "vc_strerror": (C.c_char_p, [C.c_int]),
            "vc_last_error": (C.c_char_p, []),
            "vc_dbg_csin": (C.c_int, [p, p, i64, i32, p]),
            "vc_dbg_plcm": (C.c_int, [p, p, p, i64, i32, p]),
            "enc_set_option": (C.c_int, [p, i32, i64]),
            "enc_get_option": (C.c_int, [p, i32, C.POINTER(C.c_int64)]),
            "vc_dbg_lasm": (C.c_int, [p, p, i64, p]),
            "vc_dbg_keystream": (C.c_int, [p, p, p, i32, p]),
            "vc_dbg_layout": (C.c_int, [p, p]),
            "vc_server_create": (C.c_int, [i32, i32, p, p]),
            "vc_server_add": (C.c_int, [p, p, i32, i64, p, i32, p, i32, C.c_double, C.c_double, i64,
                                        C.POINTER(C.c_int32)]),
            "vc_server_tick": (C.c_int, [p, C.c_double, C.POINTER(C.c_int32)]),
            "vc_server_drain": (C.c_int, [p, i32, i32, p, p, p, p, C.POINTER(C.c_int32)]),
            "vc_server_stream_done": (C.c_int, [p, i32]),
            "vc_server_remove": (C.c_int, [p, i32]),
            "vc_server_inflight": (i32, [p]),
            "vc_server_set_option": (C.c_int, [p, i32, i64]),
            "vc_server_destroy": (None, [p]),
            "vc_dbg_server_stats": (C.c_int, [p, p, p]),
            "vc_dbg_server_record": (C.c_int, [p, i32]),
            "vc_dbg_server_take": (C.c_int, [p, i32, i32, p, p]),
            "vc_stats_histogram": (C.c_int, [p, i32, i32, i32, i32, p, p, p, p, p]),
            "vc_stats_correlation": (C.c_int, [p, i32, i32, i32, i32, i32, p, i64, p, p, p]),
            "vc_stats_local_entropy": (C.c_int, [p, i32, i32, i32, i32, i32, p, i32, i32, p, p, p]),
            "vc_stats_npcr_uaci": (C.c_int, [p, p, i32, i32, i32, i32, p, p, p, p]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc: int, where: str):
    if rc != VC_OK:
        raise VcError(rc, where)


def _stream(stream):
    if stream is None:
        import torch

        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _dptr(t):
    if t.device.type != "cuda":
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _dbase(t):
    """Base address of a CUDA tensor that may be a strided view (pitched frames)."""
    if t.device.type != "cuda":
        raise ValueError("expected a CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _hptr(a):
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("expected a contiguous array")
        return C.c_void_p(a.ctypes.data)
    if a.device.type != "cpu" or not a.is_contiguous():
        raise ValueError("expected a contiguous host tensor")
    return C.c_void_p(a.data_ptr())


# ---- C names ---------------------------------------------------------------

def enc_init(kind: int, key, height: int, width: int, channels: int = 3, n_subframes: int = 4,
             rounds: int = 5) -> C.c_void_p:
    k = vc_key(kind, (C.c_double * 4)(*([float(v) for v in key] + [0.0] * (4 - len(key)))))
    lay = vc_layout(height, width, channels, n_subframes, rounds)
    ctx = C.c_void_p()
    _check(lib().enc_init(C.byref(k), C.byref(lay), C.byref(ctx)), "enc_init")
    return ctx


def encrypt_frames(ctx, d_in, d_out, nframes: int, stream=None) -> None:
    _check(lib().encrypt_frames(ctx, _dptr(d_in), _dptr(d_out), nframes, _stream(stream)), "encrypt_frames")


def decrypt_frames(ctx, d_in, d_out, nframes: int, stream=None) -> None:
    _check(lib().decrypt_frames(ctx, _dptr(d_in), _dptr(d_out), nframes, _stream(stream)), "decrypt_frames")


def encrypt_frames_pitched(ctx, d_in, d_out, nframes: int, frame_pitch: int, stream=None) -> None:
    """encrypt_frames on frames frame_pitch bytes apart (0 = packed)."""
    _check(lib().encrypt_frames_pitched(ctx, _dbase(d_in), _dbase(d_out), nframes,
                                        frame_pitch, _stream(stream)), "encrypt_frames_pitched")


def decrypt_frames_pitched(ctx, d_in, d_out, nframes: int, frame_pitch: int, stream=None) -> None:
    _check(lib().decrypt_frames_pitched(ctx, _dbase(d_in), _dbase(d_out), nframes,
                                        frame_pitch, _stream(stream)), "decrypt_frames_pitched")


def encrypt_frames_static(ctx, d_in, d_out, nframes: int, stream=None) -> None:
    """encrypt_frames without any device allocation (scratch in a static device array)."""
    _check(lib().encrypt_frames_static(ctx, _dptr(d_in), _dptr(d_out), nframes, _stream(stream)),
           "encrypt_frames_static")


def crypt_frames_host(ctx, direction: int, h_in, h_out, nframes: int, stream=None) -> None:
    _check(lib().crypt_frames_host(ctx, direction, _hptr(h_in), _hptr(h_out), nframes, _stream(stream)),
           "crypt_frames_host")


def crypt_frames_host_async(ctx, direction: int, h_in, h_out, nframes: int, stream=None, done_event=None) -> None:
    """crypt_frames_host without the wait; done_event: a torch.cuda.Event recorded after the last download."""
    ev = C.c_void_p(done_event.cuda_event) if done_event is not None else None
    _check(lib().crypt_frames_host_async(ctx, direction, _hptr(h_in), _hptr(h_out), nframes, _stream(stream), ev),
           "crypt_frames_host_async")


def enc_save_state(ctx) -> bytes:
    n = lib().enc_state_size(ctx)
    buf = (C.c_uint8 * n)()
    ln = C.c_size_t(n)
    _check(lib().enc_save_state(ctx, buf, C.byref(ln)), "enc_save_state")
    return bytes(buf)


def enc_load_state(ctx, state: bytes) -> None:
    buf = (C.c_uint8 * len(state)).from_buffer_copy(state)
    _check(lib().enc_load_state(ctx, buf, len(state)), "enc_load_state")


def enc_frame_index(ctx) -> int:
    return lib().enc_frame_index(ctx)


def enc_sync_status(ctx) -> None:
    _check(lib().enc_sync_status(ctx), "enc_sync_status")


def enc_set_chunk(ctx, frames: int) -> None:
    _check(lib().enc_set_chunk(ctx, frames), "enc_set_chunk")


def enc_profile_enable(ctx, enable: bool) -> None:
    _check(lib().enc_profile_enable(ctx, 1 if enable else 0), "enc_profile_enable")


def enc_profile_read(ctx) -> dict:
    ms = (C.c_double * 3)()
    ln = (C.c_int64 * 3)()
    _check(lib().enc_profile_read(ctx, ms, ln), "enc_profile_read")
    names = ("schedule", "keystream", "rounds")
    return {nm: {"ms": ms[i], "launches": ln[i]} for i, nm in enumerate(names)}


def enc_join(ctx, stream=None) -> None:
    """`stream` waits on the device for the context's internal streams."""
    _check(lib().enc_join(ctx, _stream(stream)), "enc_join")


def enc_destroy(ctx) -> None:
    lib().enc_destroy(ctx)


def enc_destroy_async(ctx) -> None:
    lib().enc_destroy_async(ctx)


def vc_dbg_csin(d_t, d_out, variant: int = 1, stream=None) -> None:
    _check(lib().vc_dbg_csin(_dptr(d_t), _dptr(d_out), d_t.numel(), variant, _stream(stream)), "vc_dbg_csin")


def vc_dbg_plcm(d_x, d_p, d_out, variant: int = 0, stream=None) -> None:
    _check(lib().vc_dbg_plcm(_dptr(d_x), _dptr(d_p), _dptr(d_out), d_x.numel(), variant, _stream(stream)),
           "vc_dbg_plcm")


def enc_set_option(ctx, option: int, value: int) -> None:
    _check(lib().enc_set_option(ctx, option, value), "enc_set_option")


def enc_get_option(ctx, option: int) -> int:
    v = C.c_int64()
    _check(lib().enc_get_option(ctx, option, C.byref(v)), "enc_get_option")
    return v.value


def vc_dbg_lasm(d_xymu, d_out, stream=None) -> None:
    _check(lib().vc_dbg_lasm(_dptr(d_xymu), _dptr(d_out), d_xymu.numel() // 3, _stream(stream)), "vc_dbg_lasm")


def vc_dbg_keystream(ctx, d_ks, d_sc, nframes: int, stream=None) -> None:
    _check(lib().vc_dbg_keystream(ctx, _dptr(d_ks), _dptr(d_sc), nframes, _stream(stream)), "vc_dbg_keystream")


def vc_dbg_call_plan(ctx, nframes: int) -> dict:
    """The passes the next call of nframes frames would run (diagnostic)."""
    cap = 4096
    plan = (C.c_int32 * cap)()
    info = (C.c_int32 * 4)()
    _check(lib().vc_dbg_call_plan(ctx, nframes, plan, cap, info), "vc_dbg_call_plan")
    return {"passes": list(plan[: min(info[0], cap)]), "first_runahead": bool(info[1]),
            "runahead_next": info[2], "ks_sm_warps": info[3]}


def vc_dbg_peaks(stream=None) -> dict:
    """Measured binary64 FMA and 32-bit IMAD rates (operations/s) of this GPU and
    the cycles of one dependent PLCM step (the keystream roofline's
    denominators)."""
    fp, im, cyc = C.c_double(), C.c_double(), C.c_double()
    _check(lib().vc_dbg_fp64_peak(C.byref(fp), _stream(stream)), "vc_dbg_fp64_peak")
    _check(lib().vc_dbg_imad_peak(C.byref(im), _stream(stream)), "vc_dbg_imad_peak")
    _check(lib().vc_dbg_plcm_latency(0.3141592653589793, 0.2718281828459045, 20000, C.byref(cyc), _stream(stream)),
           "vc_dbg_plcm_latency")
    return {"fp64_ops_per_s": fp.value, "imad_ops_per_s": im.value, "plcm_step_cycles": cyc.value}


def vc_dbg_layout(ctx) -> dict:
    out = (C.c_int32 * 8)()
    _check(lib().vc_dbg_layout(ctx, out), "vc_dbg_layout")
    return dict(zip(["T", "NT", "Npad", "N", "P", "cap", "chunk", "smem"], list(out)))


# ---- convenience wrapper -----------------------------------------------------

class Cipher:
    """One video stream: key, layout and device-resident chaotic state."""

    def __init__(self, kind: int, key, height: int, width: int, channels: int = 3, n_subframes: int = 4,
                 rounds: int = 5):
        self.kind, self.H, self.W, self.C = kind, height, width, channels
        self.n, self.rounds = n_subframes, rounds
        self.N = height * width * channels
        self.ctx = enc_init(kind, key, height, width, channels, n_subframes, rounds)

    def encrypt(self, d_in, d_out=None, stream=None):
        """Encrypt a (F, H, W, C) uint8 CUDA tensor; returns the ciphertext tensor."""
        import torch

        if d_out is None:
            d_out = torch.empty_like(d_in)
        nframes = d_in.numel() // self.N
        assert d_in.numel() == nframes * self.N and d_in.dtype == torch.uint8
        encrypt_frames(self.ctx, d_in, d_out, nframes, stream)
        return d_out

    def decrypt(self, d_in, d_out=None, stream=None):
        import torch

        if d_out is None:
            d_out = torch.empty_like(d_in)
        nframes = d_in.numel() // self.N
        assert d_in.numel() == nframes * self.N and d_in.dtype == torch.uint8
        decrypt_frames(self.ctx, d_in, d_out, nframes, stream)
        return d_out

    def crypt_host(self, direction: int, h_in, h_out, stream=None) -> None:
        nframes = (h_in.size if isinstance(h_in, np.ndarray) else h_in.numel()) // self.N
        crypt_frames_host(self.ctx, direction, h_in, h_out, nframes, stream)

    def crypt_host_async(self, direction: int, h_in, h_out, stream=None, done_event=None) -> None:
        nframes = (h_in.size if isinstance(h_in, np.ndarray) else h_in.numel()) // self.N
        crypt_frames_host_async(self.ctx, direction, h_in, h_out, nframes, stream, done_event)

    def save_state(self) -> bytes:
        return enc_save_state(self.ctx)

    def load_state(self, state: bytes) -> None:
        enc_load_state(self.ctx, state)

    @property
    def frame_index(self) -> int:
        return enc_frame_index(self.ctx)

    def sync(self) -> None:
        enc_sync_status(self.ctx)

    def set_chunk(self, frames: int) -> None:
        enc_set_chunk(self.ctx, frames)

    def set_option(self, option: int, value: int) -> None:
        enc_set_option(self.ctx, option, value)

    def get_option(self, option: int) -> int:
        return enc_get_option(self.ctx, option)

    def layout_info(self) -> dict:
        return vc_dbg_layout(self.ctx)

    def close(self, wait: bool = True) -> None:
        """Release the context: after its work (wait), or with its memory given
        back in stream order after that work (enc_destroy_async: the caller
        keeps the frames that work uses alive until it is complete)."""
        if getattr(self, "ctx", None):
            (enc_destroy if wait else enc_destroy_async)(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- ragged batches -------------------------------------------------------------

def vc_batcher_create() -> C.c_void_p:
    b = C.c_void_p()
    _check(lib().vc_batcher_create(C.byref(b)), "vc_batcher_create")
    return b


def vc_batch_submit(batcher, jobs, stream=None) -> None:
    """jobs: sequence of (Cipher or ctx, direction, d_in tensor, d_out tensor, nframes)."""
    arr = (vc_job * max(1, len(jobs)))()
    for k, (ctx, direction, d_in, d_out, nframes) in enumerate(jobs):
        c = ctx.ctx if isinstance(ctx, Cipher) else ctx
        arr[k] = vc_job(c, direction, _dptr(d_in).value, _dptr(d_out).value, nframes)
    _check(lib().vc_batch_submit(batcher, arr, len(jobs), _stream(stream)), "vc_batch_submit")


def vc_batcher_set_option(batcher, option: int, value: int) -> None:
    _check(lib().vc_batcher_set_option(batcher, option, value), "vc_batcher_set_option")


def vc_batcher_destroy(batcher) -> None:
    lib().vc_batcher_destroy(batcher)


class Batcher:
    """Runs frames of many streams per launch (one CUDA graph replay per batch)."""

    def __init__(self, graph: bool = True, ctas_per_sm: int = 0, runahead: int = 0):
        self.b = vc_batcher_create()
        vc_batcher_set_option(self.b, VC_BOPT_GRAPH, 1 if graph else 0)
        if ctas_per_sm:
            vc_batcher_set_option(self.b, VC_BOPT_CTAS_PER_SM, ctas_per_sm)
        if runahead:
            vc_batcher_set_option(self.b, VC_BOPT_RUNAHEAD, runahead)

    def submit(self, jobs, stream=None) -> None:
        vc_batch_submit(self.b, jobs, stream)

    def prefetch(self, ciphers) -> None:
        """Start producing the next run-ahead frames of keystream of these streams."""
        arr = (C.c_void_p * max(1, len(ciphers)))(*[c.ctx.value for c in ciphers])
        _check(lib().vc_batch_prefetch(self.b, arr, len(ciphers)), "vc_batch_prefetch")

    def ready(self, cipher, nframes: int) -> bool:
        """True if the keystream of the stream's next nframes frames exists on the device."""
        r = lib().vc_batch_ready(self.b, cipher.ctx, nframes)
        if r < 0:
            raise VcError(-r, "vc_batch_ready")
        return r == 1

    def close(self) -> None:
        if getattr(self, "b", None):
            vc_batcher_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class NativeServer:
    """Per-tick work of the serving loop in libvcrypt (vc_server_*): mode 0
    batches every ready frame of every stream into one submission per tick,
    mode 1 makes one encrypt/decrypt call per frame."""

    def __init__(self, mode: int, max_frames_per_tick: int, stream):
        import numpy as np

        self._np = np
        h = C.c_void_p()
        _check(lib().vc_server_create(mode, max_frames_per_tick, _stream(stream), C.byref(h)), "vc_server_create")
        self.s = h
        self._cap = 4096
        self._ids = np.empty(self._cap, dtype=np.int32)
        self._frames = np.empty(self._cap, dtype=np.int64)
        self._arr = np.empty(self._cap, dtype=np.float64)
        self._lat = np.empty(self._cap, dtype=np.float64)

    def add(self, cipher, direction: int, frame_bytes: int, d_src, src_period: int, d_ring, ring_frames: int,
            fps: float, t_arrival: float, frames_total: int) -> int:
        i = C.c_int32()
        _check(lib().vc_server_add(self.s, cipher.ctx, direction, frame_bytes, _dptr(d_src), src_period, _dptr(d_ring),
                                   ring_frames, fps, t_arrival, frames_total, C.byref(i)), "vc_server_add")
        return i.value

    def tick(self, now: float) -> int:
        n = C.c_int32()
        _check(lib().vc_server_tick(self.s, now, C.byref(n)), "vc_server_tick")
        return n.value

    def drain(self, block: bool = False):
        """(ids, frame indices, arrival s, latency ms) of completed frames."""
        np = self._np
        out = [], [], [], []
        while True:
            n = C.c_int32()
            _check(lib().vc_server_drain(self.s, 1 if block else 0, self._cap, self._ids.ctypes.data,
                                         self._frames.ctypes.data, self._arr.ctypes.data, self._lat.ctypes.data,
                                         C.byref(n)), "vc_server_drain")
            k = n.value
            for dst, src in zip(out, (self._ids, self._frames, self._arr, self._lat)):
                dst.append(src[:k].copy())
            if k < self._cap or not block and k == 0:
                break
        return tuple(np.concatenate(x) if x else np.empty(0) for x in out)

    def stream_done(self, i: int) -> bool:
        r = lib().vc_server_stream_done(self.s, i)
        if r < 0:
            raise VcError(-r, "vc_server_stream_done")
        return r == 1

    def remove(self, i: int) -> None:
        _check(lib().vc_server_remove(self.s, i), "vc_server_remove")

    def inflight(self) -> int:
        return lib().vc_server_inflight(self.s)

    def set_option(self, option: int, value: int) -> None:
        """A batcher option (VC_BOPT_*) of a batching server."""
        _check(lib().vc_server_set_option(self.s, option, value), "vc_server_set_option")

    def host_stats(self) -> dict:
        """Host ms per part of the ticks since the last call (vc_dbg_server_stats)."""
        ms = (C.c_double * 6)()
        t = C.c_int64()
        _check(lib().vc_dbg_server_stats(self.s, ms, C.byref(t)), "vc_dbg_server_stats")
        return {"ticks": t.value, "clocks_ms": ms[0], "prefetch_ms": ms[1], "submit_ms": ms[2], "event_ms": ms[3],
                "gpu_ms_per_tick": ms[4] / ms[5] if ms[5] else 0.0}

    def record(self, enable: bool = True) -> None:
        """Keep per-frame and per-tick latency records (vc_dbg_server_record)."""
        _check(lib().vc_dbg_server_record(self.s, 1 if enable else 0), "vc_dbg_server_record")

    def take_records(self):
        """(frames [k, 4]: stream, arrival, submission, completion; ticks [m, 4]:
        submission, device start, device end, frame count), seconds."""
        np = self._np
        out = []
        for which in (0, 1):
            parts = []
            while True:
                buf = np.empty((4096, 4), dtype=np.float64)
                n = C.c_int32()
                _check(lib().vc_dbg_server_take(self.s, which, 4096, buf.ctypes.data, C.byref(n)), "vc_dbg_server_take")
                parts.append(buf[:n.value].copy())
                if n.value < 4096:
                    break
            out.append(np.concatenate(parts))
        return tuple(out)

    def close(self) -> None:
        if getattr(self, "s", None):
            lib().vc_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- statistical measures of Sec. 4 and Sec. 5 on the device -----------------

def _frames_shape(t):
    if t.dim() == 3:
        t = t.unsqueeze(0)
    F, H, W, Cc = t.shape
    return t, F, H, W, Cc


def stats_histogram(frames, stream=None):
    """(counts [F, C, 256] uint32 as int32, chi^2 [F, C], variance [F, C],
    entropy [F, C]) of device HWC uint8 frames."""
    import torch

    t, F, H, W, Cc = _frames_shape(frames)
    hist = torch.empty((F, Cc, 256), dtype=torch.int32, device=t.device)
    chi2, var, ent = (torch.empty((F, Cc), dtype=torch.float64, device=t.device) for _ in range(3))
    _check(lib().vc_stats_histogram(_dptr(t), F, H, W, Cc, _dptr(hist), _dptr(chi2), _dptr(var), _dptr(ent),
                                    _stream(stream)), "vc_stats_histogram")
    return hist, chi2, var, ent


def stats_correlation(frames, direction: int, pairs=None, stream=None):
    """Adjacent-pixel correlation [F, C]; direction 0 H, 1 V, 2 D; pairs: device
    int32 first-pixel indices, or None for every pair."""
    import torch

    t, F, H, W, Cc = _frames_shape(frames)
    sums = torch.empty((F, Cc, 6), dtype=torch.int64, device=t.device)
    r = torch.empty((F, Cc), dtype=torch.float64, device=t.device)
    n = 0 if pairs is None else pairs.numel()
    _check(lib().vc_stats_correlation(_dptr(t), F, H, W, Cc, direction, _dptr(pairs) if pairs is not None else None,
                                      n, _dptr(sums), _dptr(r), _stream(stream)), "vc_stats_correlation")
    return r


def stats_local_entropy(frames, channel: int, blocks, side: int, stream=None):
    """(block entropies [F, k], means [F]) of one channel; blocks: device int32
    [k, 2] top-left (row, column) corners."""
    import torch

    t, F, H, W, Cc = _frames_shape(frames)
    k = blocks.shape[0]
    be = torch.empty((F, k), dtype=torch.float64, device=t.device)
    mean = torch.empty((F,), dtype=torch.float64, device=t.device)
    _check(lib().vc_stats_local_entropy(_dptr(t), F, H, W, Cc, channel, _dptr(blocks), k, side, _dptr(be), _dptr(mean),
                                        _stream(stream)), "vc_stats_local_entropy")
    return be, mean


def stats_npcr_uaci(a, b, stream=None):
    """(NPCR [F, C], UACI [F, C]) in percent between device frames a and b."""
    import torch

    ta, F, H, W, Cc = _frames_shape(a)
    tb, *_ = _frames_shape(b)
    sums = torch.empty((F, Cc, 2), dtype=torch.int64, device=ta.device)
    npcr = torch.empty((F, Cc), dtype=torch.float64, device=ta.device)
    uaci = torch.empty((F, Cc), dtype=torch.float64, device=ta.device)
    _check(lib().vc_stats_npcr_uaci(_dptr(ta), _dptr(tb), F, H, W, Cc, _dptr(sums), _dptr(npcr), _dptr(uaci),
                                    _stream(stream)), "vc_stats_npcr_uaci")
    return npcr, uaci
