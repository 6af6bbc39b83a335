"""pulda: Polya-urn partially collapsed LDA on one GB300 (sm_103a).

A thin Python binding of the C ABI in include/pulda.h.  Each function has the
C name and only marshals arguments: every step of the sampler runs in the
CUDA kernels of ``_build/libpulda.so``.  There is no CPU fallback -- if the
library has not been built (``paper_1704_03581_gb300.build.build()``), loading
fails loudly.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# PULDA_LIB selects another build of the same library (e.g. one compiled
# with different tile constants); by default the in-tree build is used.
LIB_PATH = os.environ.get("PULDA_LIB") or os.path.join(_PKG, "_build", "libpulda.so")

PULDA_OK = 0
STATUS = {0: "PULDA_OK", -1: "PULDA_ERR_INVALID", -2: "PULDA_ERR_OOM", -3: "PULDA_ERR_CUDA",
          -4: "PULDA_ERR_TIMEOUT", -5: "PULDA_ERR_DEGENERATE", -6: "PULDA_ERR_BUSY"}

EXPORTED = ["pulda_init", "pulda_sweep", "pulda_phi_step", "pulda_z_step", "pulda_sync", "pulda_sync_timeout",
            "pulda_get_z",
            "pulda_get_z_dev", "pulda_set_z", "pulda_get_counts", "pulda_log_posterior", "pulda_get_phi",
            "pulda_get_word_tables",
            "pulda_infer", "pulda_infer_noalloc", "pulda_stats", "pulda_z_layout", "pulda_last_error", "pulda_free",
            "pulda_batch_init", "pulda_batch_sweep", "pulda_batch_sync", "pulda_batch_get_z", "pulda_batch_stats",
            "pulda_batch_tuning", "pulda_batch_last_error", "pulda_batch_free", "pulda_barrier_selftest",
            "pulda_serve_open", "pulda_serve_submit", "pulda_serve_poll", "pulda_serve_pending", "pulda_serve_stats",
            "pulda_serve_close"]


class PuldaError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


# pulda_options' device-allocator callbacks: alloc(bytes, stream, ctx) -> pointer or NULL,
# free(ptr, stream, ctx)
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class Options(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_void_p), ("zstep_path", ctypes.c_int32), ("warps_per_block", ctypes.c_int32),
                ("docs_per_warp", ctypes.c_int32), ("phi_mode", ctypes.c_int32),
                ("slice_len", ctypes.c_int32), ("coop_min_len", ctypes.c_int32), ("count_path", ctypes.c_int32),
                ("batch_form", ctypes.c_int32), ("alias_layout", ctypes.c_int32),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", ctypes.c_void_p)]


def allocator_callbacks(allocator) -> tuple:
    """C callbacks for an object with ``alloc(nbytes, stream) -> int`` (a
    device pointer, 0 when it cannot) and ``free(ptr, stream)``.  Keep the
    returned pair alive while the library may call it (until the handle,
    server or batch is freed)."""
    def _alloc(nbytes, stream, ctx):
        try:
            return int(allocator.alloc(int(nbytes), stream)) or None
        except Exception:
            return None

    def _free(ptr, stream, ctx):
        allocator.free(int(ptr), stream)

    return ALLOC_FN(_alloc), FREE_FN(_free)


class SweepStats(ctypes.Structure):
    _fields_ = [("tokens", ctypes.c_int64), ("a_branch", ctypes.c_int64), ("sum_min", ctypes.c_int64),
                ("zero_mass", ctypes.c_int64), ("dead_rows", ctypes.c_int64), ("nnz_phi", ctypes.c_int64),
                ("sweep", ctypes.c_int64), ("cum_tokens", ctypes.c_int64), ("cum_a_branch", ctypes.c_int64),
                ("cum_sum_min", ctypes.c_int64), ("cum_zero_mass", ctypes.c_int64), ("sum_inter", ctypes.c_int64),
                ("docside", ctypes.c_int64), ("cum_sum_inter", ctypes.c_int64), ("cum_docside", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {f[0]: int(getattr(self, f[0])) for f in self._fields_}


_lib = None


def lib() -> ctypes.CDLL:
    """Load the CUDA library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1704_03581_gb300.build.build() "
                               "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        P, i32, i64, u64, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_float
        sig = {
            "pulda_init": [P, P, P, i64, i32, i32, P, f32, u64, P],
            "pulda_sweep": [P, i32],
            "pulda_phi_step": [P],
            "pulda_z_step": [P],
            "pulda_sync": [P],
            "pulda_sync_timeout": [P, ctypes.c_int32],
            "pulda_get_z": [P, P],
            "pulda_get_z_dev": [P, P],
            "pulda_set_z": [P, P, i64],
            "pulda_get_counts": [P, P, P],
            "pulda_log_posterior": [P, P],
            "pulda_get_phi": [P, P, P, P, P],
            "pulda_get_word_tables": [P, P, P, P, P, P, P, P, P, P],
            "pulda_infer": [P, P, P, i64, i32, u64, P, P],
            "pulda_infer_noalloc": [P, P, P, i64, i64, i32, u64, P],
            "pulda_stats": [P, P],
            "pulda_z_layout": [P, P, P, P],
        }
        sig.update({
            "pulda_batch_init": [P, P, i32, P],
            "pulda_batch_sweep": [P, i32],
            "pulda_batch_sync": [P],
            "pulda_batch_get_z": [P, i32, P],
            "pulda_batch_stats": [P, i32, P],
            "pulda_batch_tuning": [P, P, P, P, P, P],
            "pulda_barrier_selftest": [i32, i32, i32, P],
            "pulda_serve_open": [P, i64, i32, i64, P],
            "pulda_serve_submit": [P, u64, u64, P, i32, i32, P],
            "pulda_serve_poll": [P, P, i32, P, i32],
            "pulda_serve_pending": [P, P, P, P],
            "pulda_serve_stats": [P, P],
            "pulda_serve_close": [P],
        })
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.pulda_last_error.argtypes = [P]
        L.pulda_last_error.restype = ctypes.c_char_p
        L.pulda_free.argtypes = [P]
        L.pulda_free.restype = None
        L.pulda_batch_last_error.argtypes = [P]
        L.pulda_batch_last_error.restype = ctypes.c_char_p
        L.pulda_batch_free.argtypes = [P]
        L.pulda_batch_free.restype = None
        _lib = L
    return _lib


def _ptr(a) -> int | None:
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    return int(a.data_ptr())          # a torch tensor


def _check(h, status: int):
    if status != PULDA_OK:
        msg = lib().pulda_last_error(h)
        raise PuldaError(status, msg.decode() if msg else "")


# ----------------------------------------------------------- C-named calls

def pulda_init(word_ids, doc_offsets, K: int, V: int, alpha, beta: float, seed: int, stream=None,
               zstep_path: int = 0, warps_per_block: int = 0, docs_per_warp: int = 0, phi_mode: int = 0,
               slice_len: int = 0, coop_min_len: int = 0, callbacks: tuple | None = None,
               count_path: int = 0, alias_layout: int = 0) -> int:
    """``callbacks`` = allocator_callbacks(...) routes the handle's device memory through them."""
    w = np.ascontiguousarray(word_ids, dtype=np.int32)
    off = np.ascontiguousarray(doc_offsets, dtype=np.int64)
    a = np.ascontiguousarray(np.broadcast_to(np.asarray(alpha, dtype=np.float32), (K,)))
    opt = Options()
    opt.stream = stream
    opt.zstep_path = zstep_path
    opt.warps_per_block = warps_per_block
    opt.docs_per_warp = docs_per_warp
    opt.phi_mode = phi_mode
    opt.slice_len = slice_len
    opt.coop_min_len = coop_min_len
    opt.count_path = count_path
    opt.alias_layout = alias_layout
    if callbacks is not None:
        opt.alloc, opt.free = callbacks
    h = ctypes.c_void_p()
    st = lib().pulda_init(ctypes.byref(h), _ptr(w), _ptr(off), off.shape[0] - 1, K, V, _ptr(a), float(beta),
                          int(seed) & (2 ** 64 - 1), ctypes.byref(opt))
    _check(None, st)
    return h.value


def pulda_sweep(h, n_sweeps: int = 1):
    _check(h, lib().pulda_sweep(h, n_sweeps))


def pulda_phi_step(h):
    _check(h, lib().pulda_phi_step(h))


def pulda_z_step(h):
    _check(h, lib().pulda_z_step(h))


def pulda_sync(h):
    _check(h, lib().pulda_sync(h))


def pulda_sync_timeout(h, timeout_ms: int) -> bool:
    """True when the handle's work finished within timeout_ms, False on PULDA_ERR_TIMEOUT."""
    st = lib().pulda_sync_timeout(h, int(timeout_ms))
    if st == -4:
        return False
    _check(h, st)
    return True


def pulda_get_z(h, out: np.ndarray):
    _check(h, lib().pulda_get_z(h, _ptr(out)))
    return out


def pulda_get_z_dev(h, out_tensor):
    _check(h, lib().pulda_get_z_dev(h, _ptr(out_tensor)))
    return out_tensor


def pulda_set_z(h, z: np.ndarray, sweep: int):
    z = np.ascontiguousarray(z, dtype=np.int16)
    _check(h, lib().pulda_set_z(h, _ptr(z), sweep))


def pulda_get_counts(h, n_kv: np.ndarray | None, m_dk: np.ndarray | None):
    _check(h, lib().pulda_get_counts(h, _ptr(n_kv), _ptr(m_dk)))


def pulda_log_posterior(h) -> np.ndarray:
    """[total, document sum, topic sum] of log p(w, z | alpha, beta) for the current z."""
    out = np.zeros(3, np.float64)
    _check(h, lib().pulda_log_posterior(h, _ptr(out)))
    return out


def pulda_get_phi(h, V: int):
    nnz = ctypes.c_int64(0)
    _check(h, lib().pulda_get_phi(h, None, None, None, ctypes.byref(nnz)))
    col = np.zeros(V + 1, np.int64)
    top = np.zeros(max(nnz.value, 1), np.int16)
    phi = np.zeros(max(nnz.value, 1), np.float32)
    _check(h, lib().pulda_get_phi(h, _ptr(col), _ptr(top), _ptr(phi), ctypes.byref(nnz)))
    return col, top[:nnz.value], phi[:nnz.value]


def pulda_get_word_tables(h, K: int, V: int) -> dict:
    nnz = ctypes.c_int64(0)
    _check(h, lib().pulda_get_word_tables(h, None, None, None, None, None, None, None, None, ctypes.byref(nnz)))
    n = max(nnz.value, 1)
    out = dict(col_ptr=np.zeros(V + 1, np.int64), topic=np.zeros(n, np.int16), c=np.zeros(n, np.uint32),
               S=np.zeros(K, np.int64), q=np.zeros(n, np.uint32), A=np.zeros(V, np.uint64),
               athr=np.zeros(n, np.uint32), atopic=np.zeros(n, np.int16))
    _check(h, lib().pulda_get_word_tables(h, *[_ptr(out[k]) for k in
                                               ("col_ptr", "topic", "c", "S", "q", "A", "athr", "atopic")],
                                          ctypes.byref(nnz)))
    for k in ("topic", "c", "q", "athr", "atopic"):
        out[k] = out[k][:nnz.value]
    return out


def pulda_infer(h, word_ids, doc_offsets, n_sweeps: int, seed: int, K: int, want_m: bool = False):
    w = np.ascontiguousarray(word_ids, dtype=np.int32)
    off = np.ascontiguousarray(doc_offsets, dtype=np.int64)
    D = off.shape[0] - 1
    z = np.zeros(max(w.shape[0], 1), np.int16)
    m = np.zeros((D, K), np.int32) if want_m else None
    _check(h, lib().pulda_infer(h, _ptr(w), _ptr(off), D, n_sweeps, int(seed) & (2 ** 64 - 1), _ptr(z), _ptr(m)))
    return (z[:w.shape[0]], m) if want_m else z[:w.shape[0]]


def _check_noalloc_tensors(word_ids_dev, doc_offsets_dev, z_out_dev) -> tuple[int, int]:
    """(D, N) of pulda_infer_noalloc's device tensors, or ValueError: the C
    call trusts the sizes it is given, so a wrong dtype, a strided view or a
    short output would make its kernels read or write past a buffer."""
    want = (("word_ids_dev", word_ids_dev, "int32"), ("doc_offsets_dev", doc_offsets_dev, "int64"),
            ("z_out_dev", z_out_dev, "int16"))
    for name, t, dt in want:
        if not hasattr(t, "data_ptr") or not hasattr(t, "is_cuda"):
            raise ValueError(f"{name} must be a torch tensor")
        if str(t.dtype) != f"torch.{dt}":
            raise ValueError(f"{name} must be {dt} (got {t.dtype})")
        if t.dim() != 1:
            raise ValueError(f"{name} must be one-dimensional (got shape {tuple(t.shape)})")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    D = int(doc_offsets_dev.shape[0]) - 1
    N = int(word_ids_dev.shape[0])
    if D < 0:
        raise ValueError("doc_offsets_dev needs at least one entry (D + 1 offsets)")
    if int(z_out_dev.shape[0]) < N:
        raise ValueError(f"z_out_dev holds {int(z_out_dev.shape[0])} topics, fewer than the {N} word ids")
    for name, t, _ in want:
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
    devs = {t.device.index for _, t, _ in want}
    if len(devs) != 1:
        raise ValueError(f"the three tensors must be on one device (got {sorted(devs)})")
    return D, N


def pulda_infer_noalloc(h, word_ids_dev, doc_offsets_dev, n_sweeps: int, seed: int, z_out_dev):
    """Device tensors in and out; nothing is allocated (see include/pulda.h).
    word_ids_dev int32[N], doc_offsets_dev int64[D+1], z_out_dev int16[>= N],
    contiguous CUDA tensors on the handle's device (the library checks the
    device; the values of ids and offsets are checked on the GPU)."""
    D, N = _check_noalloc_tensors(word_ids_dev, doc_offsets_dev, z_out_dev)
    _check(h, lib().pulda_infer_noalloc(h, _ptr(word_ids_dev), _ptr(doc_offsets_dev), D, N, n_sweeps,
                                        int(seed) & (2 ** 64 - 1), _ptr(z_out_dev)))
    return z_out_dev


def pulda_stats(h) -> dict:
    s = SweepStats()
    _check(h, lib().pulda_stats(h, ctypes.byref(s)))
    return s.as_dict()


def pulda_z_layout(h) -> dict:
    """The corpus z-step's launch layout: documents per warp of the main kernel,
    documents on cooperative CTAs, documents one per warp beside them."""
    d, c, o = ctypes.c_int32(0), ctypes.c_int64(0), ctypes.c_int64(0)
    _check(h, lib().pulda_z_layout(h, ctypes.byref(d), ctypes.byref(c), ctypes.byref(o)))
    return {"docs_per_warp": d.value, "coop_docs": c.value, "one_warp_docs": o.value}


def pulda_last_error(h) -> str:
    m = lib().pulda_last_error(h)
    return m.decode() if m else ""


def pulda_free(h):
    if h:
        lib().pulda_free(h)


class Sampler:
    """One chain: ``Sampler(w, doc_off, K, V, alpha, beta, seed).sweep(n)``."""

    def __init__(self, word_ids, doc_offsets, K: int, V: int, alpha=0.1, beta: float = 0.01, seed: int = 0,
                 stream=None, zstep_path: int = 0, warps_per_block: int = 0, docs_per_warp: int = 0,
                 phi_mode: int = 0, slice_len: int = 0, coop_min_len: int = 0, allocator=None,
                 count_path: int = 0, alias_layout: int = 0):
        """phi_mode 0: Poisson Polya urn (Algorithm 2); 1: Dirichlet Phi (Algorithm 1).
        slice_len > 0: documents longer than it resampled in concurrent stale-count slices (not the paper's).
        coop_min_len: documents at least this long resampled by a whole CTA (0 = automatic, -1 = never);
        the topics are the same either way.  allocator: an object with alloc(nbytes, stream) -> device
        pointer (0 if it cannot) and free(ptr, stream) that supplies every device buffer of the handle,
        its temporaries and its servers (see pulda_options in include/pulda.h).  alias_layout 2: the
        z-step reads packed alias slots (0 or 1: threshold and topic arrays); results are identical."""
        self.K, self.V = K, V
        self.phi_mode = phi_mode
        self.N = int(np.asarray(doc_offsets)[-1])
        self.D = int(np.asarray(doc_offsets).shape[0] - 1)
        self.h = None
        self._callbacks = allocator_callbacks(allocator) if allocator is not None else None
        self.h = pulda_init(word_ids, doc_offsets, K, V, alpha, beta, seed, stream, zstep_path, warps_per_block,
                            docs_per_warp, phi_mode, slice_len, coop_min_len, self._callbacks, count_path,
                            alias_layout)

    def close(self):
        if self.h:
            pulda_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sweep(self, n: int = 1):
        pulda_sweep(self.h, n)
        return self

    def phi_step(self):
        pulda_phi_step(self.h)
        return self

    def z_step(self):
        pulda_z_step(self.h)
        return self

    def sync(self):
        pulda_sync(self.h)

    def z(self) -> np.ndarray:
        return pulda_get_z(self.h, np.zeros(max(self.N, 1), np.int16))[:self.N]

    def set_z(self, z, sweep: int):
        pulda_set_z(self.h, z, sweep)

    def n(self) -> np.ndarray:
        out = np.zeros((self.K, self.V), np.int32)
        pulda_get_counts(self.h, out, None)
        return out

    def m(self) -> np.ndarray:
        out = np.zeros((self.D, self.K), np.int32)
        pulda_get_counts(self.h, None, out)
        return out

    def log_posterior(self) -> np.ndarray:
        return pulda_log_posterior(self.h)

    def phi(self):
        return pulda_get_phi(self.h, self.V)

    def word_tables(self) -> dict:
        return pulda_get_word_tables(self.h, self.K, self.V)

    def infer(self, word_ids, doc_offsets, n_sweeps: int, seed: int, want_m: bool = False):
        return pulda_infer(self.h, word_ids, doc_offsets, n_sweeps, seed, self.K, want_m)

    def stats(self) -> dict:
        return pulda_stats(self.h)

    def z_layout(self) -> dict:
        return pulda_z_layout(self.h)


# ------------------------------------------------------------------ batches

class ChainDesc(ctypes.Structure):
    _fields_ = [("word_ids_host", ctypes.c_void_p), ("doc_offsets_host", ctypes.c_void_p), ("D", ctypes.c_int64),
                ("K", ctypes.c_int32), ("V", ctypes.c_int32), ("alpha_host", ctypes.c_void_p),
                ("beta", ctypes.c_float), ("seed", ctypes.c_uint64)]


def _bcheck(b, status: int):
    if status != PULDA_OK:
        msg = lib().pulda_batch_last_error(b)
        raise PuldaError(status, msg.decode() if msg else "")


def pulda_batch_init(chains: list[dict], stream=None, warps_per_block: int = 0, coop_min_len: int = 0,
                     callbacks: tuple | None = None, batch_form: int = 0, alias_layout: int = 0):
    """chains: dicts with w, doc_off, K, V, alpha, beta, seed.  coop_min_len: 0 tuned, -1 never, > 0 fixed.
    alias_layout: 0 tuned, 1 threshold and topic arrays, 2 packed slots.
    callbacks = allocator_callbacks(...) routes every device buffer of the batch through them."""
    keep = []
    arr = (ChainDesc * len(chains))()
    for i, c in enumerate(chains):
        w = np.ascontiguousarray(c["w"], dtype=np.int32)
        off = np.ascontiguousarray(c["doc_off"], dtype=np.int64)
        a = np.ascontiguousarray(np.broadcast_to(np.asarray(c.get("alpha", 0.1), np.float32), (c["K"],)))
        keep += [w, off, a]
        arr[i] = ChainDesc(_ptr(w), _ptr(off), off.shape[0] - 1, c["K"], c["V"], _ptr(a), float(c.get("beta", 0.01)),
                           int(c.get("seed", 0)) & (2 ** 64 - 1))
    opt = Options()
    opt.stream = stream
    opt.warps_per_block = warps_per_block
    opt.coop_min_len = coop_min_len
    opt.batch_form = batch_form
    opt.alias_layout = alias_layout
    if callbacks is not None:
        opt.alloc, opt.free = callbacks
    b = ctypes.c_void_p()
    _bcheck(None, lib().pulda_batch_init(ctypes.byref(b), arr, len(chains), ctypes.byref(opt)))
    return b.value


def pulda_batch_sweep(b, n_sweeps: int = 1):
    _bcheck(b, lib().pulda_batch_sweep(b, n_sweeps))


def pulda_batch_sync(b):
    _bcheck(b, lib().pulda_batch_sync(b))


def pulda_batch_get_z(b, chain: int, out: np.ndarray):
    _bcheck(b, lib().pulda_batch_get_z(b, chain, _ptr(out)))
    return out


def pulda_batch_stats(b, chain: int) -> dict:
    s = SweepStats()
    _bcheck(b, lib().pulda_batch_stats(b, chain, ctypes.byref(s)))
    return s.as_dict()


def pulda_batch_tuning(b) -> tuple[int, int, bool, bool, int]:
    """(z-step warps per CTA, cooperative threshold or -1, tuning over, one persistent launch per sweep,
    alias layout: 1 arrays, 2 packed slots)."""
    w, c, t, o, al = (ctypes.c_int32(0) for _ in range(5))
    _bcheck(b, lib().pulda_batch_tuning(b, ctypes.byref(w), ctypes.byref(c), ctypes.byref(t), ctypes.byref(o),
                                        ctypes.byref(al)))
    return w.value, c.value, bool(t.value), bool(o.value), al.value


def pulda_barrier_selftest(blocks: int, missing: int, rounds: int = 4) -> tuple[int, int]:
    """(status, barriers passed) of the one-launch form's grid barrier self-test."""
    n = ctypes.c_int32(0)
    st = lib().pulda_barrier_selftest(blocks, missing, rounds, ctypes.byref(n))
    return st, n.value


def pulda_batch_last_error(b) -> str:
    m = lib().pulda_batch_last_error(b)
    return m.decode() if m else ""


def pulda_batch_free(b):
    if b:
        lib().pulda_batch_free(b)


class Batch:
    """Many chains advanced together: ``Batch(chains).sweep(n)``."""

    def __init__(self, chains: list[dict], stream=None, warps_per_block: int = 0, coop_min_len: int = 0,
                 allocator=None, batch_form: int = 0, alias_layout: int = 0):
        """batch_form 0: the launch form is tuned; 1: six launches per sweep; 2: one persistent launch.
        alias_layout 0: tuned; 1: threshold and topic arrays; 2: packed slots."""
        self.sizes = [int(np.asarray(c["doc_off"])[-1]) for c in chains]
        self.b = None
        self._callbacks = allocator_callbacks(allocator) if allocator is not None else None
        self.b = pulda_batch_init(chains, stream, warps_per_block, coop_min_len, self._callbacks, batch_form,
                                  alias_layout)

    def close(self):
        if self.b:
            pulda_batch_free(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sweep(self, n: int = 1):
        pulda_batch_sweep(self.b, n)
        return self

    def sync(self):
        pulda_batch_sync(self.b)

    def z(self, chain: int) -> np.ndarray:
        n = self.sizes[chain]
        return pulda_batch_get_z(self.b, chain, np.zeros(max(n, 1), np.int16))[:n]

    def stats(self, chain: int) -> dict:
        return pulda_batch_stats(self.b, chain)

    def tuning(self):
        return pulda_batch_tuning(self.b)


# ------------------------------------------------------------------ serving

class ServeResult(ctypes.Structure):
    _fields_ = [("req_id", ctypes.c_uint64), ("status", ctypes.c_int32), ("len", ctypes.c_int32),
                ("submit_ns", ctypes.c_int64), ("done_ns", ctypes.c_int64)]


def pulda_serve_open(h, token_budget: int, max_slots: int, slice_tokens: int) -> int:
    s = ctypes.c_void_p()
    _check(h, lib().pulda_serve_open(h, token_budget, max_slots, slice_tokens, ctypes.byref(s)))
    return s.value


def pulda_serve_submit(s, req_id: int, seed: int, words: np.ndarray, n_sweeps: int, z_out: np.ndarray):
    st = lib().pulda_serve_submit(s, req_id, int(seed) & (2 ** 64 - 1), _ptr(words), int(words.shape[0]), n_sweeps,
                                  _ptr(z_out))
    if st != PULDA_OK:
        raise PuldaError(st, "submit rejected")


def pulda_serve_poll(s, max_results: int = 1024, timeout_ms: int = 100) -> list[dict]:
    buf = (ServeResult * max_results)()
    n = ctypes.c_int32(0)
    st = lib().pulda_serve_poll(s, buf, max_results, ctypes.byref(n), timeout_ms)
    if st == -4:          # PULDA_ERR_TIMEOUT
        return []
    if st != PULDA_OK:
        raise PuldaError(st, "serving failed")
    return [dict(req_id=int(r.req_id), status=int(r.status), len=int(r.len), submit_ns=int(r.submit_ns),
                 done_ns=int(r.done_ns)) for r in buf[:n.value]]


def pulda_serve_pending(s) -> tuple[int, int, int]:
    a, b, c = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
    st = lib().pulda_serve_pending(s, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
    if st != PULDA_OK:
        raise PuldaError(st, "serve_pending failed")
    return a.value, b.value, c.value


def pulda_serve_stats(s) -> dict:
    out = np.zeros(8, np.int64)
    st = lib().pulda_serve_stats(s, _ptr(out))
    if st != PULDA_OK:
        raise PuldaError(st, "serve_stats failed")
    keys = ["launches", "completed", "token_steps", "kernel_ns", "slice", "max_active", "waiting", "running"]
    return {k: int(v) for k, v in zip(keys, out)}


def pulda_serve_close(s):
    st = lib().pulda_serve_close(s)
    if st != PULDA_OK:
        raise PuldaError(st, "server reported an error")


class Server:
    """Continuous-batching fold-in against a sampler's current Phi."""

    def __init__(self, sampler: Sampler, token_budget: int = 1 << 24, max_slots: int = 4096,
                 slice_tokens: int = 4096):
        self.s = pulda_serve_open(sampler.h, token_budget, max_slots, slice_tokens)
        self._keep = {}

    def submit(self, req_id: int, seed: int, words, n_sweeps: int) -> np.ndarray:
        w = np.ascontiguousarray(words, dtype=np.int32)
        z = np.zeros(w.shape[0], np.int16)
        self._keep[req_id] = (w, z)
        pulda_serve_submit(self.s, req_id, seed, w, n_sweeps, z)
        return z

    def poll(self, max_results: int = 1024, timeout_ms: int = 100) -> list[dict]:
        out = pulda_serve_poll(self.s, max_results, timeout_ms)
        for r in out:
            r["z"] = self._keep.pop(r["req_id"])[1]
        return out

    def pending(self):
        return pulda_serve_pending(self.s)

    def stats(self) -> dict:
        return pulda_serve_stats(self.s)

    def close(self):
        if self.s:
            pulda_serve_close(self.s)
            self.s = None
