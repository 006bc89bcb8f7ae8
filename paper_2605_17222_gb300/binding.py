"""Python binding of the C ABI in include/ckks_lt.h (ctypes; argument
marshalling only).  Device memory for ciphertexts and step buffers is held in
torch tensors (int64 storage, read as uint64 residues by the library) and the
stream is torch's current CUDA stream unless one is given.  Every step runs in
the library's CUDA kernels; there is no CPU path: if the library cannot be
built or loaded, or there is no GPU, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import re
from dataclasses import dataclass

import numpy as np

from . import build as _build

LT_DIAG, LT_BSGS, LT_DH_BSGS, LT_TH_BSGS = 0, 1, 2, 3
ALGOS = {"diag": LT_DIAG, "bsgs": LT_BSGS, "dh": LT_DH_BSGS, "th": LT_TH_BSGS}
HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "ckks_lt.h")


class CkksError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"ckks status {status}: {msg}")
        self.status = status


class Split(ctypes.Structure):
    _fields_ = [("n1", ctypes.c_uint32), ("n2", ctypes.c_uint32), ("n3", ctypes.c_uint32)]

    def tuple(self):
        return (self.n1, self.n2, self.n3)


_lib = None


def declared_functions() -> list:
    """Names of the functions include/ckks_lt.h declares."""
    with open(HEADER) as f:
        text = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n.startswith(("ckks_", "lt_"))))


def lib():
    """Load the library, building it first if the sources are newer
    (CKKS_LT_LIBRARY names a prebuilt copy to load instead)."""
    global _lib
    if _lib is not None:
        return _lib
    path = os.environ.get("CKKS_LT_LIBRARY") or _build.build()
    L = ctypes.CDLL(path)
    P, U32, I32, SZ, I = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int32, ctypes.c_size_t, ctypes.c_int
    PP = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "ckks_ctx_create": [PP, U32, P, U32, P, U32, U32, I],
        "ckks_ctx_destroy": [P],
        "ckks_upload_rotation_key": [P, I32, P, SZ],
        "ckks_upload_rotation_key_device": [P, I32, P, SZ, P],
        "ckks_upload_diagonals": [P, PP, U32, I32, I32, U32, P, SZ],
        "ckks_upload_diagonals_device": [P, PP, U32, I32, I32, U32, P, SZ, P],
        "ckks_free_diags": [P],
        "ckks_diags_create": [P, PP, U32, I32, I32, U32],
        "ckks_diags_write_device": [P, U32, U32, P, SZ, P],
        "ckks_ct_create": [P, PP, U32],
        "ckks_ct_upload": [P, PP, U32, P],
        "ckks_ct_wrap_device": [P, PP, U32, P],
        "ckks_ct_h2d_async": [P, P, SZ, P],
        "ckks_ct_d2h_async": [P, P, SZ, P],
        "ckks_ct_download": [P, P, SZ],
        "ckks_free_ct": [P],
        "lt_eval": [P, P, P, I, P, P, P, P],
        "lt_eval_batch": [P, U32, P, P, P, P, P, P],
        "lt_eval_chain": [P, P, U32, P, P, P, P, P, P],
        "lt_choose_split": [P, I, U32, U32, P],
        "lt_autotune": [P, I, P, P, U32, P, P],
        "lt_autotune_batch": [P, I, U32, P, P, U32, P, P],
        "ckks_poly_ntt": [P, P, U32, I, I, P],
        "ckks_decompose": [P, U32, P, I32, P, P],
        "ckks_ks_inner": [P, U32, P, I32, I32, P, I, P, P, I, P],
        "ckks_moddown": [P, U32, P, P, P],
        "ckks_moddown_noalloc": [P, U32, P, P, P],
        "ckks_moddown_rescale": [P, U32, P, P, P],
        "ckks_rescale": [P, U32, P, P, P],
        "ckks_automorphism": [P, U32, P, I32, P, P],
        "ckks_device_status": [P],
        "lt_graph_create": [P, U32, P, P, P, P, P, PP],
        "lt_graph_launch": [P, P],
        "lt_graph_begin": [P, P],
        "lt_graph_end": [P, P, PP],
        "lt_graph_destroy": [P],
        "ckks_selftest_bounded_wait": [P, U32, P],
        "ckks_debug_diag_mac_waits": [P, ctypes.c_uint64, U32],
        "ckks_debug_diag_mac_tile": [P, U32, U32],
        "ckks_profile_enable": [ctypes.c_char_p, I],
        "ckks_profile_read": [ctypes.c_char_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint64)],
        "ckks_profile_work": [ctypes.c_char_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
        "ckks_probe_int_rates": [I, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
        "lt_model_estimate": [P, I, U32, U32, P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    L.ckks_last_error.restype = ctypes.c_char_p
    L.ckks_device_bytes_in_use.argtypes = [P]
    L.ckks_device_bytes_in_use.restype = SZ
    L.ckks_kernel_launch_count.restype = ctypes.c_uint64
    L.ckks_has_rotation_key.argtypes = [P, I32]
    L.ckks_has_rotation_key.restype = I
    L.lt_required_rotations.argtypes = [P, I, P, U32, I32, I32, P, U32]
    L.lt_required_rotations.restype = I32
    L.ckks_ct_level.argtypes = [P]
    L.ckks_ct_level.restype = U32
    L.ckks_ct_device_ptr.argtypes = [P]
    L.ckks_ct_device_ptr.restype = P
    L.lt_tuned_tile.argtypes = [P, I, P, U32, P, P]
    L.lt_tuned_tile.restype = I32
    L.lt_dh_schedule.argtypes = [P, P, U32, P]
    L.lt_dh_schedule.restype = I32
    L.lt_candidate_splits.argtypes = [P, I, U32, U32, P, U32]
    L.lt_candidate_splits.restype = I32
    L.ckks_profile_reset.restype = None
    _lib = L
    return L


def check(st: int) -> None:
    if st != 0:
        raise CkksError(st, lib().ckks_last_error().decode())


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("the CKKS LT library needs a CUDA GPU")
    return torch


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(_torch().cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _ptr(t) -> ctypes.c_void_p:
    if t is None:
        return ctypes.c_void_p(0)
    if isinstance(t, np.ndarray):
        assert t.dtype == np.uint64 and t.flags.c_contiguous
        return ctypes.c_void_p(t.ctypes.data)
    assert t.is_contiguous() and t.is_cuda and t.element_size() == 8
    return ctypes.c_void_p(t.data_ptr())


def to_device(a: np.ndarray, device=None):
    """Host uint64 array -> device int64 tensor with the same bits."""
    torch = _torch()
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64))
    return t.to(device or "cuda", non_blocking=False)


def to_host(t) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint64)


@dataclass
class Ciphertext:
    handle: ctypes.c_void_p
    level: int
    tensor: object  # backing torch tensor [2][level][N] (None if library-owned)
    ctx: "Context"

    def numpy(self) -> np.ndarray:
        if self.tensor is not None:
            _torch().cuda.synchronize()
            return to_host(self.tensor)
        out = np.empty((2, self.level, self.ctx.N), dtype=np.uint64)
        check(lib().ckks_ct_download(self.handle, _ptr(out), out.size))
        return out

    def free(self):
        if self.handle:
            check(lib().ckks_free_ct(self.handle))
            self.handle = None

    def __del__(self):
        try:
            if self.handle and _lib is not None:
                _lib.ckks_free_ct(self.handle)
        except Exception:
            pass


class Diagonals:
    """Encoded diagonals on the device; offsets offset0 + stride * t, t < n_diag."""

    def __init__(self, ctx, handle, n_diag, stride, level, offset0=0):
        self.ctx, self.handle, self.n_diag, self.stride, self.level = ctx, handle, n_diag, stride, level
        self.offset0 = offset0

    def free(self):
        if self.handle:
            check(lib().ckks_free_diags(self.handle))
            self.handle = None


class RecordedBatch:
    """A replayable recording of LT calls (lt_graph_create, or lt_graph_begin/end)."""

    def __init__(self, handle, outs, keep):
        self.h, self.outs, self._keep = handle, outs, keep

    def launch(self, stream=None):
        check(lib().lt_graph_launch(self.h, _stream(stream)))
        return self.outs

    def close(self):
        if self.h:
            check(lib().lt_graph_destroy(self.h))
            self.h = None


class Context:
    """An RNS-CKKS context on one GPU (ckks_ctx_create)."""

    def __init__(self, log_n: int, q, p, dnum: int, device: int = 0):
        _torch()
        L = lib()
        self.log_n, self.N = log_n, 1 << log_n
        self.q, self.p = [int(v) for v in q], [int(v) for v in p]
        self.L, self.k, self.dnum = len(self.q), len(self.p), dnum
        self.alpha = -(-self.L // dnum)
        self.beta_max = -(-self.L // self.alpha)
        self.device = device
        qa = np.array(self.q, dtype=np.uint64)
        pa = np.array(self.p, dtype=np.uint64)
        h = ctypes.c_void_p()
        check(L.ckks_ctx_create(ctypes.byref(h), log_n, _ptr(qa), len(qa), _ptr(pa), len(pa), dnum, device))
        self.h = h

    @classmethod
    def from_params(cls, ps, device: int = 0):
        return cls(ps.log_n, ps.q, ps.p, ps.dnum, device)

    def close(self):
        if getattr(self, "h", None):
            check(lib().ckks_ctx_destroy(self.h))
            self.h = None

    def beta(self, level: int) -> int:
        return -(-level // self.alpha)

    def device_status(self) -> None:
        """Raise CkksError(CKKS_ETIMEOUT) if a bounded device-side wait gave up."""
        check(lib().ckks_device_status(self.h))

    def selftest_bounded_wait(self, limit_ms: int = 200, stream=None) -> None:
        check(lib().ckks_selftest_bounded_wait(self.h, limit_ms, _stream(stream)))

    def debug_diag_mac_waits(self, wait_limit_ns: int = 0, starve_step: int = 0xFFFFFFFF) -> None:
        """Failure-detection test hook (ckks_debug_diag_mac_waits); (0, 0xFFFFFFFF) resets it."""
        check(lib().ckks_debug_diag_mac_waits(self.h, int(wait_limit_ns), int(starve_step)))

    def debug_diag_mac_tile(self, outer_per_cta: int = 0, positions_per_cta: int = 0) -> None:
        """Test hook (ckks_debug_diag_mac_tile): force the diagonal kernel's tile; (0, 0) resets."""
        check(lib().ckks_debug_diag_mac_tile(self.h, int(outer_per_cta), int(positions_per_cta)))

    def bytes_in_use(self) -> int:
        return lib().ckks_device_bytes_in_use(self.h)

    # ----------------------------------------------------------- keys / diagonals
    def upload_rotation_key(self, r: int, key: np.ndarray) -> None:
        key = np.ascontiguousarray(key, dtype=np.uint64)
        check(lib().ckks_upload_rotation_key(self.h, int(r), _ptr(key), key.size))

    def upload_rotation_key_device(self, r: int, key_t, stream=None) -> None:
        check(lib().ckks_upload_rotation_key_device(self.h, int(r), _ptr(key_t), key_t.numel(), _stream(stream)))

    def has_key(self, r: int) -> bool:
        return bool(lib().ckks_has_rotation_key(self.h, int(r)))

    def upload_diagonals(self, diags: np.ndarray, stride: int = 1, level: int | None = None,
                         offset0: int = 0) -> Diagonals:
        diags = np.ascontiguousarray(diags, dtype=np.uint64)
        level = level if level is not None else diags.shape[1] - self.k
        h = ctypes.c_void_p()
        check(lib().ckks_upload_diagonals(self.h, ctypes.byref(h), diags.shape[0], offset0, stride, level,
                                          _ptr(diags), diags.size))
        return Diagonals(self, h, diags.shape[0], stride, level, offset0)

    def upload_diagonals_device(self, diags_t, stride: int = 1, level: int | None = None, stream=None,
                                offset0: int = 0) -> Diagonals:
        """diags_t: device tensor [n_diag][level + k][N] (copied by the library)."""
        level = level if level is not None else diags_t.shape[1] - self.k
        h = ctypes.c_void_p()
        check(lib().ckks_upload_diagonals_device(self.h, ctypes.byref(h), diags_t.shape[0], offset0, stride, level,
                                                 _ptr(diags_t), diags_t.numel(), _stream(stream)))
        return Diagonals(self, h, diags_t.shape[0], stride, level, offset0)

    def diags_create(self, n_diag: int, stride: int = 1, level: int | None = None, offset0: int = 0) -> Diagonals:
        level = level if level is not None else self.L
        h = ctypes.c_void_p()
        check(lib().ckks_diags_create(self.h, ctypes.byref(h), n_diag, offset0, stride, level))
        return Diagonals(self, h, n_diag, stride, level, offset0)

    def diags_write(self, f: Diagonals, first: int, chunk_t, stream=None) -> None:
        check(lib().ckks_diags_write_device(f.handle, first, chunk_t.shape[0], _ptr(chunk_t), chunk_t.numel(),
                                            _stream(stream)))

    def required_rotations(self, algo: str, split, n_diag: int, stride: int = 1, offset0: int = 0) -> list:
        sp = Split(*(tuple(split) + (0,) * (3 - len(split)))) if split else None
        buf = (ctypes.c_int32 * 4096)()
        n = lib().lt_required_rotations(self.h, ALGOS[algo], ctypes.byref(sp) if sp else None, n_diag, offset0,
                                        stride, buf, 4096)
        if n < 0:
            raise CkksError(1, "bad split")
        return list(buf[:n])

    def autotune(self, algo: str, sample: "Ciphertext", diags: "Diagonals", max_candidates: int = 6):
        """Time the model's best candidate splits on `sample` and keep the fastest."""
        sp, ms = Split(), ctypes.c_double()
        check(lib().lt_autotune(self.h, ALGOS[algo], sample.handle, diags.handle, max_candidates, ctypes.byref(sp),
                                ctypes.byref(ms)))
        return sp.tuple(), ms.value

    def autotune_batch(self, algo: str, samples, diags: "Diagonals", max_candidates: int = 6):
        """Time the model's best candidate splits as one lt_eval_batch over `samples`
        (one level); returns (fastest split, ms per batch)."""
        n = len(samples)
        arr = (ctypes.c_void_p * n)(*[c.handle for c in samples])
        sp, ms = Split(), ctypes.c_double()
        check(lib().lt_autotune_batch(self.h, ALGOS[algo], n, arr, diags.handle, max_candidates, ctypes.byref(sp),
                                      ctypes.byref(ms)))
        return sp.tuple(), ms.value

    def candidate_splits(self, algo: str, level: int, n_diag: int, count: int):
        """The cost model's `count` best splits, fastest first (lt_candidate_splits)."""
        buf = (Split * count)()
        n = lib().lt_candidate_splits(self.h, ALGOS[algo], level, n_diag, buf, count)
        if n < 0:
            raise CkksError(1, "bad arguments")
        return [buf[i].tuple() for i in range(n)]

    def tuned_tile(self, algo: str, diags: "Diagonals", level: int):
        """(outer indices per CTA, positions per CTA) lt_autotune measured for the
        shape (0 = default), or None if the shape was not tuned (lt_tuned_tile)."""
        k3, run = ctypes.c_uint32(), ctypes.c_uint32()
        r = lib().lt_tuned_tile(self.h, ALGOS[algo], diags.handle, level, ctypes.byref(k3), ctypes.byref(run))
        if r < 0:
            raise CkksError(1, "bad arguments")
        return (k3.value, run.value) if r == 1 else None

    def dh_schedule(self, diags: "Diagonals", level: int, split) -> str:
        """'fused' (baby steps inside the diagonal kernel, TH(1, n1, n2)) or 'baby'
        (Algorithm 1's materialised baby steps) for DH-BSGS with `split` (lt_dh_schedule)."""
        sp = Split(split[0], split[1], 1)
        r = lib().lt_dh_schedule(self.h, diags.handle, level, ctypes.byref(sp))
        if r < 0:
            raise CkksError(1, "bad arguments")
        return "fused" if r == 1 else "baby"

    def model_estimate(self, algo: str, level: int, n_diag: int, split):
        """(DRAM bytes, seconds) the split-selection cost model assigns to one LT (lt_model_estimate)."""
        sp = Split(*(tuple(split) + (1,) * (3 - len(split))))
        b, t = ctypes.c_double(), ctypes.c_double()
        check(lib().lt_model_estimate(self.h, ALGOS[algo], level, n_diag, ctypes.byref(sp), ctypes.byref(b),
                                      ctypes.byref(t)))
        return b.value, t.value

    def choose_split(self, algo: str, level: int, n_diag: int):
        sp = Split()
        check(lib().lt_choose_split(self.h, ALGOS[algo], level, n_diag, ctypes.byref(sp)))
        return sp.tuple()

    # ----------------------------------------------------------- ciphertexts
    def ct_empty(self, level: int) -> Ciphertext:
        torch = _torch()
        t = torch.empty((2, level, self.N), dtype=torch.int64, device=f"cuda:{self.device}")
        return self.ct_wrap(t, level)

    def ct_wrap(self, tensor, level: int) -> Ciphertext:
        h = ctypes.c_void_p()
        check(lib().ckks_ct_wrap_device(self.h, ctypes.byref(h), level, _ptr(tensor)))
        return Ciphertext(h, level, tensor, self)

    def ct_from_host(self, c: np.ndarray) -> Ciphertext:
        c = np.ascontiguousarray(c, dtype=np.uint64)
        return self.ct_wrap(to_device(c, f"cuda:{self.device}"), c.shape[1])

    def ct_upload(self, c: np.ndarray) -> Ciphertext:
        """Library-owned device copy (ckks_ct_upload)."""
        c = np.ascontiguousarray(c, dtype=np.uint64)
        h = ctypes.c_void_p()
        check(lib().ckks_ct_upload(self.h, ctypes.byref(h), c.shape[1], _ptr(c)))
        return Ciphertext(h, c.shape[1], None, self)

    def ct_create(self, level: int) -> Ciphertext:
        h = ctypes.c_void_p()
        check(lib().ckks_ct_create(self.h, ctypes.byref(h), level))
        return Ciphertext(h, level, None, self)

    def h2d_async(self, ct: Ciphertext, host: np.ndarray, stream=None) -> None:
        check(lib().ckks_ct_h2d_async(ct.handle, _ptr(host), host.size, _stream(stream)))

    def d2h_async(self, ct: Ciphertext, host: np.ndarray, stream=None) -> None:
        check(lib().ckks_ct_d2h_async(ct.handle, _ptr(host), host.size, _stream(stream)))

    # ----------------------------------------------------------- the LT
    def lt_eval(self, ct: Ciphertext, diags: Diagonals, algo: str = "th", split=None, out: Ciphertext | None = None,
                stream=None):
        out = out or self.ct_empty(ct.level - 1)
        sp = Split(*(tuple(split) + (1,) * (3 - len(split)))) if split else Split(0, 0, 0)
        chosen = Split()
        check(lib().lt_eval(self.h, ct.handle, diags.handle, ALGOS[algo], ctypes.byref(sp), out.handle,
                            _stream(stream), ctypes.byref(chosen)))
        return out, chosen.tuple()

    def lt_eval_batch(self, cts, diags, algos=None, splits=None, outs=None, stream=None):
        n = len(cts)
        outs = outs or [self.ct_empty(c.level - 1) for c in cts]
        arr = lambda xs: (ctypes.c_void_p * n)(*[x.handle for x in xs])
        al = (ctypes.c_int * n)(*[ALGOS[a] for a in algos]) if algos else None
        sp = None
        if splits:
            sp = (Split * n)(*[Split(*(tuple(s) + (1,) * (3 - len(s)))) for s in splits])
        check(lib().lt_eval_batch(self.h, n, arr(cts), arr(diags), al, sp, arr(outs), _stream(stream)))
        return outs

    def lt_eval_chain(self, ct, stages, algos=None, splits=None, out=None, stream=None):
        """A chain of LTs (lt_eval_chain): stage i applies stages[i] at level
        ct.level - i; returns (output at ct.level - len(stages), chosen splits)."""
        n = len(stages)
        out = out or self.ct_empty(ct.level - n)
        fs = (ctypes.c_void_p * n)(*[f.handle for f in stages])
        al = (ctypes.c_int * n)(*[ALGOS[a] for a in algos]) if algos else None
        sp = (Split * n)(*[Split(*(tuple(x) + (1,) * (3 - len(x)))) for x in splits]) if splits else None
        chosen = (Split * n)()
        check(lib().lt_eval_chain(self.h, ct.handle, n, fs, al, sp, out.handle, _stream(stream), chosen))
        return out, [c.tuple() for c in chosen]

    def lt_graph(self, cts, diags, algos=None, splits=None, outs=None):
        """Record one lt_eval_batch into a replayable graph (see lt_graph_create)."""
        n = len(cts)
        outs = outs or [self.ct_empty(c.level - 1) for c in cts]
        arr = lambda xs: (ctypes.c_void_p * n)(*[x.handle for x in xs])
        al = (ctypes.c_int * n)(*[ALGOS[a] for a in algos]) if algos else None
        sp = (Split * n)(*[Split(*(tuple(s) + (1,) * (3 - len(s)))) for s in splits]) if splits else None
        h = ctypes.c_void_p()
        check(lib().lt_graph_create(self.h, n, arr(cts), arr(diags), al, sp, arr(outs), ctypes.byref(h)))
        return RecordedBatch(h, outs, (cts, diags))

    def graph_begin(self, stream) -> None:
        """Start recording the LT calls queued on `stream` (a torch.cuda.Stream)."""
        check(lib().lt_graph_begin(self.h, _stream(stream)))

    def graph_end(self, stream, keep=()) -> "RecordedBatch":
        """Stop recording `stream`; the recorded calls as one replayable graph.
        `keep` holds the objects the graph reads or writes alive with it."""
        h = ctypes.c_void_p()
        check(lib().lt_graph_end(self.h, _stream(stream), ctypes.byref(h)))
        return RecordedBatch(h, None, tuple(keep))

    # ----------------------------------------------------------- steps (device tensors)
    def ntt(self, poly, level: int, ext: bool, inverse: bool, stream=None):
        check(lib().ckks_poly_ntt(self.h, _ptr(poly), level, int(ext), int(inverse), _stream(stream)))

    def decompose(self, c, level: int, rot: int = 0, digits=None, stream=None):
        torch = _torch()
        if digits is None:
            digits = torch.empty((self.beta(level), level + self.k, self.N), dtype=torch.int64, device=c.device)
        check(lib().ckks_decompose(self.h, level, _ptr(c), rot, _ptr(digits), _stream(stream)))
        return digits

    def ks_inner(self, level: int, digits, key_rot: int, rot: int, x0=None, lift_x0: bool = False,
                 out0=None, out1=None, accumulate: bool = False, stream=None):
        torch = _torch()
        shape = (level + self.k, self.N)
        out0 = out0 if out0 is not None else torch.empty(shape, dtype=torch.int64, device=digits.device)
        out1 = out1 if out1 is not None else torch.empty(shape, dtype=torch.int64, device=digits.device)
        check(lib().ckks_ks_inner(self.h, level, _ptr(digits), key_rot, rot, _ptr(x0), int(lift_x0), _ptr(out0),
                                  _ptr(out1), int(accumulate), _stream(stream)))
        return out0, out1

    def moddown(self, x, level: int, out=None, stream=None):
        torch = _torch()
        out = out if out is not None else torch.empty((level, self.N), dtype=torch.int64, device=x.device)
        check(lib().ckks_moddown(self.h, level, _ptr(x), _ptr(out), _stream(stream)))
        return out

    def moddown_noalloc(self, x, level: int, out, stream=None):
        """ModDown into caller-provided `out` through ckks_moddown_noalloc (no device allocation)."""
        check(lib().ckks_moddown_noalloc(self.h, level, _ptr(x), _ptr(out), _stream(stream)))
        return out

    def moddown_rescale(self, x, level: int, out=None, stream=None):
        torch = _torch()
        out = out if out is not None else torch.empty((level - 1, self.N), dtype=torch.int64, device=x.device)
        check(lib().ckks_moddown_rescale(self.h, level, _ptr(x), _ptr(out), _stream(stream)))
        return out

    def rescale(self, x, level: int, out=None, stream=None):
        torch = _torch()
        out = out if out is not None else torch.empty((level - 1, self.N), dtype=torch.int64, device=x.device)
        check(lib().ckks_rescale(self.h, level, _ptr(x), _ptr(out), _stream(stream)))
        return out

    def automorphism(self, x, rot: int, out=None, stream=None):
        torch = _torch()
        out = out if out is not None else torch.empty_like(x)
        check(lib().ckks_automorphism(self.h, x.numel() // self.N, _ptr(x), rot, _ptr(out), _stream(stream)))
        return out


def kernel_launches() -> int:
    return int(lib().ckks_kernel_launch_count())


def profile_enable(kernel_class: str, on: bool = True) -> None:
    check(lib().ckks_profile_enable(kernel_class.encode(), int(on)))


def profile_read(kernel_class: str):
    """(total device ms, launches) of a kernel class since the last reset."""
    ms, n = ctypes.c_double(), ctypes.c_uint64()
    check(lib().ckks_profile_read(kernel_class.encode(), ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def profile_reset() -> None:
    lib().ckks_profile_reset()


def profile_work(kernel_class: str):
    """(128-bit multiply-accumulates, NTT butterflies) of the profiled launches
    of a kernel class since the last reset."""
    macs, bfly = ctypes.c_double(), ctypes.c_double()
    check(lib().ckks_profile_work(kernel_class.encode(), ctypes.byref(macs), ctypes.byref(bfly)))
    return macs.value, bfly.value


def probe_int_rates(device: int = 0):
    """(multiply-accumulates per s, butterflies per s) of the library's own
    arithmetic in register-only loops on `device`: the integer-ALU peaks."""
    macs, bfly = ctypes.c_double(), ctypes.c_double()
    check(lib().ckks_probe_int_rates(int(device), ctypes.byref(macs), ctypes.byref(bfly)))
    return macs.value, bfly.value


KERNEL_CLASSES = ["diag_mac", "ks_inner", "ntt_fwd_cols", "ntt_fwd_rows", "ntt_inv_rows", "ntt_inv_cols",
                  "automorphism", "add_gather"]
