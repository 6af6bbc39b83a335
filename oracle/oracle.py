"""Python wrapper of the CPU oracle (test infrastructure only).

Builds ``pulda_oracle.c`` with gcc into ``oracle/_build/`` and exposes its
functions on numpy arrays.  Only the tests, the smoke check and the CPU
baseline of the benchmark use this module; the CUDA library never does.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle.so")
SRC = [os.path.join(HERE, "pulda_oracle.c")]

L = 100
LG = 1024
GAUSS_CELLS = 65536
FRAC_BITS = 16
TAG_INIT, TAG_POIS, TAG_BETA, TAG_REDRAW_POIS, TAG_REDRAW_BETA, TAG_Z = 1, 2, 3, 4, 5, 6


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, no FMA contraction) if it is missing or stale."""
    os.makedirs(BUILD, exist_ok=True)
    deps = SRC + [os.path.join(HERE, "pulda_oracle.h")]
    if not force and os.path.exists(LIB) and all(os.path.getmtime(LIB) >= os.path.getmtime(s) for s in deps):
        return LIB
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
           "-pthread", *SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64, u32, u64, f32, f64 = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64,
                                        ctypes.c_float, ctypes.c_double)
        sig = {
            "or_philox": (None, [P, P, P]),
            "or_vose": (u64, [P, i32, P, P]),
            "or_pois_weights": (i32, [f64, i32, i32, P, P]),
            "or_norm_quantile": (f64, [f64]),
            "or_gauss_table": (None, [P]),
            "or_geo_table": (None, [f64, P]),
            "or_ctx_new": (P, [f32]),
            "or_ctx_free": (None, [P]),
            "or_ctx_table": (i32, [P, i32, P, P, P]),
            "or_ctx_geo": (None, [P, P]),
            "or_ctx_gauss": (None, [P, P]),
            "or_gauss_draw": (f64, [P, u32, u32]),
            "or_draw_entry": (u32, [P, i64, u32, u32]),
            "or_init_z": (None, [i64, i32, u64, i64, P]),
            "or_count_n": (None, [i64, P, P, i32, i32, P]),
            "or_doc_topic": (None, [P, i64, P, i32, P]),
            "or_phi_draw": (i32, [P, P, i32, i32, u64, u32, P, P, P]),
            "or_word_tables": (None, [P, P, P, i32, i32, P, P, P, P, P, P, P]),
            "or_z_step": (i32, [P, i64, P, P, i32, i32, P, P, P, P, P, P, u64, u32, i64, P]),
            "or_z_step_sliced": (i32, [P, i64, P, P, i32, i32, P, P, P, P, P, P, u64, u32, i64, i64, P]),
            "or_log_posterior": (i32, [P, i64, P, P, i32, i32, P, f64, P]),
            "or_logf": (f32, [f32]),
            "or_expf": (f32, [f32]),
            "or_gamma_draw": (f32, [P, f32, u64, u32, u32, u32, P]),
            "or_phi_draw_dir": (i32, [P, P, i32, i32, u64, u32, P, P]),
            "or_word_tables_dir": (None, [P, P, P, i32, i32, P, P, P, P, P, P, P]),
            "or_count_n_mt": (None, [i64, P, P, i32, i32, P, i32]),
            "or_phi_draw_mt": (i32, [P, P, i32, i32, u64, u32, P, P, P, i32]),
            "or_word_tables_mt": (None, [P, P, P, i32, i32, P, P, P, P, P, P, P, i32]),
            "or_z_step_mt": (i32, [P, i64, P, P, i32, i32, P, P, P, P, P, P, u64, u32, i64, P, i32]),
        }
        for name, (res, args) in sig.items():
            f = getattr(_lib, name)
            f.restype = res
            f.argtypes = args
    return _lib


def _p(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be contiguous"
    return a.ctypes.data


# ---------------------------------------------------------------- primitives

def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().or_philox(_p(c), _p(k), _p(o))
    return o


def vose(W) -> tuple[np.ndarray, np.ndarray, int]:
    W = np.ascontiguousarray(W, dtype=np.uint64)
    n = W.shape[0]
    thr = np.zeros(n, dtype=np.uint32)
    alias = np.zeros(n, dtype=np.int32)
    T = lib().or_vose(_p(W), n, _p(thr), _p(alias))
    return thr, alias, int(T)


def pois_weights(lam: float, jmin: int = 0, cap: int = 100000) -> tuple[int, np.ndarray]:
    W = np.zeros(cap, dtype=np.uint64)
    lo = np.zeros(1, dtype=np.int64)
    n = lib().or_pois_weights(float(lam), jmin, cap, _p(lo), _p(W))
    if n < 0:
        raise ValueError("capacity too small")
    return int(lo[0]), W[:n].copy()


def norm_quantile(p: float) -> float:
    return lib().or_norm_quantile(float(p))


def geo_table(beta: float) -> np.ndarray:
    t = np.zeros(LG, dtype=np.uint32)
    lib().or_geo_table(float(beta), _p(t))
    return t


class Ctx:
    """Tables for one beta (Poisson alias tables, geometric gaps, Gaussian)."""

    def __init__(self, beta: float):
        self.beta = float(np.float32(beta))
        self.h = lib().or_ctx_new(float(beta))
        if not self.h:
            raise RuntimeError("oracle table construction failed")

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.or_ctx_free(self.h)
            self.h = None

    def table(self, which: int) -> tuple[int, np.ndarray, np.ndarray]:
        """``which`` = l in 1..L for Pois(beta + l), 0 for zero-truncated Pois(beta)."""
        n = lib().or_ctx_table(self.h, which, None, None, None)
        thr = np.zeros(n, dtype=np.uint32)
        alias = np.zeros(n, dtype=np.int32)
        lo = np.zeros(1, dtype=np.int64)
        lib().or_ctx_table(self.h, which, _p(lo), _p(thr), _p(alias))
        return int(lo[0]), thr, alias

    def geo(self) -> np.ndarray:
        t = np.zeros(LG, dtype=np.uint32)
        lib().or_ctx_geo(self.h, _p(t))
        return t

    def gauss(self) -> np.ndarray:
        q = np.zeros(GAUSS_CELLS + 1, dtype=np.float64)
        lib().or_ctx_gauss(self.h, _p(q))
        return q

    def gauss_draw(self, x0: int, x1: int) -> float:
        return lib().or_gauss_draw(self.h, int(x0), int(x1))

    def draw_entry(self, l: int, x0: int, x1: int) -> int:
        return int(lib().or_draw_entry(self.h, int(l), int(x0), int(x1)))


# ------------------------------------------------------------------ the method

def init_z(N: int, K: int, seed: int, index_base: int = 0) -> np.ndarray:
    z = np.zeros(N, dtype=np.int16)
    lib().or_init_z(N, K, seed, index_base, _p(z))
    return z


def host_threads() -> int:
    """The host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def count_n(w: np.ndarray, z: np.ndarray, K: int, V: int, threads: int = 1) -> np.ndarray:
    """Dense n, word-major: ``n[v, k]``."""
    if threads > 1:
        w = np.ascontiguousarray(w, dtype=np.int32)
        z = np.ascontiguousarray(z, dtype=np.int16)
        n = np.empty((V, K), dtype=np.int32)
        lib().or_count_n_mt(w.shape[0], _p(w), _p(z), K, V, _p(n), threads)
        return n
    n = np.zeros((V, K), dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.int32)
    z = np.ascontiguousarray(z, dtype=np.int16)
    lib().or_count_n(w.shape[0], _p(w), _p(z), K, V, _p(n))
    return n


def doc_topic(doc_off: np.ndarray, z: np.ndarray, K: int) -> np.ndarray:
    D = doc_off.shape[0] - 1
    m = np.zeros((D, K), dtype=np.int32)
    doc_off = np.ascontiguousarray(doc_off, dtype=np.int64)
    z = np.ascontiguousarray(z, dtype=np.int16)
    lib().or_doc_topic(_p(doc_off), D, _p(z), K, _p(m))
    return m


def log_posterior(doc_off, w, z, K: int, V: int, alpha, beta: float) -> np.ndarray:
    """[total, document part, topic part] of the collapsed log p(w, z | alpha, beta)
    (the log-posterior diagnostic of Section 5)."""
    doc_off = np.ascontiguousarray(doc_off, dtype=np.int64)
    w = np.ascontiguousarray(w, dtype=np.int32)
    z = np.ascontiguousarray(z, dtype=np.int16)
    a = np.ascontiguousarray(np.broadcast_to(np.asarray(alpha, dtype=np.float32), (K,)))
    out = np.zeros(3, dtype=np.float64)
    if lib().or_log_posterior(_p(doc_off), doc_off.shape[0] - 1, _p(w), _p(z), K, V, _p(a), float(beta), _p(out)):
        raise MemoryError("oracle log posterior: out of memory")
    return out


def phi_draw(ctx: Ctx, n_vk: np.ndarray, seed: int, sweep: int,
             threads: int = 1) -> tuple[np.ndarray, np.ndarray, int]:
    """c[v, k] ~ Pois(beta + n[v, k]); S[k] = sum_v c[v, k]."""
    V, K = n_vk.shape
    n_vk = np.ascontiguousarray(n_vk, dtype=np.int32)
    c = np.zeros((V, K), dtype=np.uint32)
    S = np.zeros(K, dtype=np.int64)
    dead = np.zeros(1, dtype=np.int32)
    if threads > 1:
        rc = lib().or_phi_draw_mt(ctx.h, _p(n_vk), K, V, seed, sweep, _p(c), _p(S), _p(dead), threads)
    else:
        rc = lib().or_phi_draw(ctx.h, _p(n_vk), K, V, seed, sweep, _p(c), _p(S), _p(dead))
    if rc != 0:
        raise RuntimeError("dead-row redraw did not terminate")
    return c, S, int(dead[0])


def logf(x: float) -> float:
    """The oracle's own float natural log (R-GAMMA)."""
    return lib().or_logf(float(x))


def expf(x: float) -> float:
    """The oracle's own float exponential (R-GAMMA)."""
    return lib().or_expf(float(x))


def gamma_draw(ctx: Ctx, a: float, seed: int, v: int, k: int, sweep: int) -> float:
    """One G(a, 1) draw keyed by (v, k, sweep) (R-GAMMA)."""
    err = np.zeros(1, dtype=np.int32)
    g = lib().or_gamma_draw(ctx.h, float(np.float32(a)), seed, v, k, sweep, _p(err))
    if err[0]:
        raise RuntimeError("Gamma draw did not accept")
    return g


def phi_draw_dir(ctx: Ctx, n_vk: np.ndarray, seed: int, sweep: int) -> tuple[np.ndarray, np.ndarray]:
    """Algorithm 1: gamma[v, k] ~ G(beta + n[v, k], 1); S[k] = sum_v gamma[v, k] (R-DIRSUM)."""
    V, K = n_vk.shape
    n_vk = np.ascontiguousarray(n_vk, dtype=np.int32)
    g = np.zeros((V, K), dtype=np.float32)
    S = np.zeros(K, dtype=np.float64)
    if lib().or_phi_draw_dir(ctx.h, _p(n_vk), K, V, seed, sweep, _p(g), _p(S)) != 0:
        raise RuntimeError("Gamma draw did not accept")
    return g, S


class WordTables:
    """Per-word z-step tables, dense [V, K] with the first ncol[v] entries valid.
    From Polya-urn counts c (uint32) and row sums S (int64), or, with
    ``dirichlet=True``, from Gamma draws (float32) and row sums S (float64)."""

    def __init__(self, c_vk: np.ndarray, S: np.ndarray, alpha: np.ndarray, dirichlet: bool = False,
                 threads: int = 1):
        V, K = c_vk.shape
        self.V, self.K = V, K
        self.ncol = np.zeros(V, dtype=np.int32)
        self.topic = np.zeros((V, K), dtype=np.int16)
        self.q = np.zeros((V, K), dtype=np.uint32)
        self.A = np.zeros(V, dtype=np.uint64)
        self.athr = np.zeros((V, K), dtype=np.uint32)
        self.atopic = np.zeros((V, K), dtype=np.int16)
        self.phi32 = np.zeros((V, K), dtype=np.float32)
        alpha = np.ascontiguousarray(alpha, dtype=np.float32)
        if dirichlet:
            g = np.ascontiguousarray(c_vk, dtype=np.float32)
            S = np.ascontiguousarray(S, dtype=np.float64)
            fn = lib().or_word_tables_dir
        else:
            g = np.ascontiguousarray(c_vk, dtype=np.uint32)
            S = np.ascontiguousarray(S, dtype=np.int64)
            fn = lib().or_word_tables
        args = [_p(g), _p(S), _p(alpha), K, V, _p(self.ncol), _p(self.topic), _p(self.q),
                _p(self.A), _p(self.athr), _p(self.atopic), _p(self.phi32)]
        if threads > 1 and not dirichlet:
            lib().or_word_tables_mt(*args, threads)
        else:
            fn(*args)

    def column(self, v: int):
        n = int(self.ncol[v])
        return self.topic[v, :n], self.q[v, :n], self.athr[v, :n], self.atopic[v, :n], self.phi32[v, :n]

    def phi_dense(self) -> np.ndarray:
        """Phi as a dense K x V float32 matrix."""
        out = np.zeros((self.K, self.V), dtype=np.float32)
        for v in range(self.V):
            t, _, _, _, p = self.column(v)
            out[t.astype(np.int64), v] = p
        return out


def z_step(doc_off: np.ndarray, w: np.ndarray, z: np.ndarray, tables: WordTables, seed: int, sweep: int,
           index_base: int = 0, slice_len: int = 0, threads: int = 1) -> tuple[np.ndarray, np.ndarray]:
    """One z-step; returns (new z, stats[tokens, a_branch, sum_min, zero_mass, sum_inter, docside]).
    slice_len > 0 splits longer documents into concurrent slices with stale counts (not Algorithm 2);
    threads > 1 resamples whole documents on that many host threads (the same results)."""
    z = np.array(z, dtype=np.int16, copy=True)
    doc_off = np.ascontiguousarray(doc_off, dtype=np.int64)
    w = np.ascontiguousarray(w, dtype=np.int32)
    stats = np.zeros(6, dtype=np.int64)
    t = tables
    if threads > 1 and slice_len == 0:
        rc = lib().or_z_step_mt(_p(doc_off), doc_off.shape[0] - 1, _p(w), _p(z), t.K, t.V, _p(t.ncol), _p(t.topic),
                                _p(t.q), _p(t.A), _p(t.athr), _p(t.atopic), seed, sweep, index_base, _p(stats),
                                threads)
        if rc != 0:
            raise RuntimeError("z-step failed")
        return z, stats
    rc = lib().or_z_step_sliced(_p(doc_off), doc_off.shape[0] - 1, _p(w), _p(z), t.K, t.V, _p(t.ncol), _p(t.topic),
                                _p(t.q), _p(t.A), _p(t.athr), _p(t.atopic), seed, sweep, index_base, slice_len,
                                _p(stats))
    if rc != 0:
        raise RuntimeError("z-step failed")
    return z, stats


class Chain:
    """The Polya-urn partially collapsed sampler (Algorithm 2) on the CPU.

    Each sweep: rebuild n from z, draw Phi (Polya urn), build the per-word
    tables, then resample every z.  Sweep s uses RNG counter s; the initial
    topics use counter 0.
    """

    def __init__(self, w, doc_off, K: int, V: int, alpha, beta: float, seed: int, z=None, sweep: int = 0,
                 dirichlet: bool = False, slice_len: int = 0, threads: int = 1):
        self.w = np.ascontiguousarray(w, dtype=np.int32)
        self.doc_off = np.ascontiguousarray(doc_off, dtype=np.int64)
        self.K, self.V, self.seed = K, V, int(seed)
        self.alpha = np.broadcast_to(np.asarray(alpha, dtype=np.float32), (K,)).copy()
        self.beta = float(np.float32(beta))
        self.ctx = Ctx(beta)
        self.z = init_z(self.w.shape[0], K, self.seed) if z is None else np.array(z, dtype=np.int16)
        self.sweep_index = sweep
        self.tables: WordTables | None = None
        self.S = None
        self.c = None
        self.stats = np.zeros(6, dtype=np.int64)
        self.dead_rows = 0
        self.dirichlet = dirichlet      # Algorithm 1's Dirichlet Phi instead of the Polya urn
        self.slice_len = slice_len      # > 0: long documents in concurrent slices with stale counts
        self.threads = threads          # host threads of the Polya-urn steps (results are the same)

    def phi_step(self, sweep: int):
        n = count_n(self.w, self.z, self.K, self.V, threads=self.threads)
        if self.dirichlet:
            self.c, self.S = phi_draw_dir(self.ctx, n, self.seed, sweep)
            self.dead_rows = 0
        else:
            self.c, self.S, self.dead_rows = phi_draw(self.ctx, n, self.seed, sweep, threads=self.threads)
        self.tables = WordTables(self.c, self.S, self.alpha, dirichlet=self.dirichlet, threads=self.threads)

    def sweep(self, n_sweeps: int = 1):
        for _ in range(n_sweeps):
            self.sweep_index += 1
            self.phi_step(self.sweep_index)
            self.z, self.stats = z_step(self.doc_off, self.w, self.z, self.tables, self.seed, self.sweep_index,
                                        slice_len=self.slice_len, threads=self.threads)
        return self

    def n(self) -> np.ndarray:
        return count_n(self.w, self.z, self.K, self.V)

    def m(self) -> np.ndarray:
        return doc_topic(self.doc_off, self.z, self.K)


def infer(tables: WordTables, w, doc_off, n_sweeps: int, seed: int, index_base: int = 0) -> np.ndarray:
    """Fold-in of new documents against fixed per-word tables: topics start
    uniform (counter 0) and take ``n_sweeps`` z-steps (counters 1..n)."""
    w = np.ascontiguousarray(w, dtype=np.int32)
    z = init_z(w.shape[0], tables.K, seed, index_base)
    for s in range(1, n_sweeps + 1):
        z, _ = z_step(doc_off, w, z, tables, seed, s, index_base)
    return z
