"""Helpers shared by the GPU parity tests: run the CUDA path and the CPU
oracle side by side on the same seeded corpus and compare every output.

Everything the sampler decides is integer (topics, Poisson counts, alias
tables, fixed-point weights) or an IEEE-rounded fp32 quotient (phi), so the
bar is bit-exact equality."""
from __future__ import annotations

import numpy as np

import paper_1704_03581_gb300 as P
from oracle import oracle as O


def oracle_tables_flat(t: O.WordTables) -> dict:
    """The oracle's dense per-word tables in the CUDA path's CSC layout."""
    mask = np.arange(t.K)[None, :] < t.ncol[:, None]
    col_ptr = np.zeros(t.V + 1, np.int64)
    np.cumsum(t.ncol, out=col_ptr[1:])
    return dict(col_ptr=col_ptr, topic=t.topic[mask], q=t.q[mask], athr=t.athr[mask], atopic=t.atopic[mask],
                A=t.A.copy(), phi=t.phi32[mask])


def compare_tables(gpu: dict, ch: O.Chain, where: str = ""):
    """Bitwise: in Dirichlet mode S is compared as the bits of the double row sums and c
    as the bits of the float Gamma draws of the kept entries."""
    o = oracle_tables_flat(ch.tables)
    dirichlet = getattr(ch, "dirichlet", False)
    if dirichlet:
        bad = np.nonzero(gpu["S"] != ch.S.view(np.int64))[0]
        assert bad.size == 0, f"{where}: row sums S differ at {bad[:10]} (gpu {gpu['S'][bad[:3]].view(np.float64)} " \
            f"oracle {ch.S[bad[:3]]})"
    else:
        assert np.array_equal(gpu["S"], ch.S), f"{where}: row sums S differ"
    assert np.array_equal(gpu["col_ptr"], o["col_ptr"]), f"{where}: Phi sparsity (column sizes) differs " \
        f"at words {np.nonzero(np.diff(gpu['col_ptr']) != np.diff(o['col_ptr']))[0][:10]}"
    mask = np.arange(ch.K)[None, :] < ch.tables.ncol[:, None]
    assert np.array_equal(gpu["topic"], o["topic"]), f"{where}: Phi topic ids differ"
    want_c = ch.c[np.arange(ch.V)[:, None], ch.tables.topic.astype(np.int64)][mask]
    if dirichlet:
        want_c = want_c.view(np.uint32)
    what = "Gamma draws" if dirichlet else "Poisson counts c"
    assert np.array_equal(gpu["c"], want_c), f"{where}: {what} differ"
    for k in ("q", "athr", "atopic", "A"):
        bad = np.nonzero(gpu[k] != o[k])[0]
        assert bad.size == 0, f"{where}: {k} differs at {bad[:10]} (gpu {gpu[k][bad[:5]]} oracle {o[k][bad[:5]]})"


def first_mismatch(z_gpu: np.ndarray, z_or: np.ndarray, doc_off: np.ndarray) -> str:
    bad = np.nonzero(z_gpu != z_or)[0]
    if bad.size == 0:
        return ""
    i = int(bad[0])
    d = int(np.searchsorted(doc_off, i, side="right") - 1)
    return f"{bad.size} tokens differ; first at token {i} (doc {d}, position {i - doc_off[d]}): " \
           f"gpu {z_gpu[i]} oracle {z_or[i]}"


def lockstep(w, doc_off, K: int, V: int, alpha, beta: float, seed: int, sweeps: int, path: int = 0,
             check_tables: bool = True, check_counts_every: int = 0, docs_per_warp: int = 0, phi_mode: int = 0,
             slice_len: int = 0, coop_min_len: int = 0, count_path: int = 0, alias_layout: int = 0):
    """Run both sides for `sweeps` sweeps, comparing after each half-sweep.
    phi_mode 1 runs both in Algorithm 1's Dirichlet mode; slice_len > 0 both in stale-count slices;
    coop_min_len sets which documents the GPU resamples with a whole CTA (the oracle has one way);
    alias_layout 2 has the GPU's z-step read packed alias slots (the oracle has one layout)."""
    s = P.Sampler(w, doc_off, K, V, alpha, beta, seed, zstep_path=path, docs_per_warp=docs_per_warp,
                  phi_mode=phi_mode, slice_len=slice_len, coop_min_len=coop_min_len, count_path=count_path,
                  alias_layout=alias_layout)
    ch = O.Chain(w, doc_off, K, V, alpha, beta, seed, dirichlet=phi_mode == 1, slice_len=slice_len)
    try:
        zg = s.z()
        assert np.array_equal(zg, ch.z), "initial topics differ: " + first_mismatch(zg, ch.z, doc_off)
        for it in range(1, sweeps + 1):
            s.phi_step()
            ch.sweep_index += 1
            ch.phi_step(ch.sweep_index)
            if check_tables:
                compare_tables(s.word_tables(), ch, f"sweep {it}")
            s.z_step()
            ch.z, ch.stats = O.z_step(ch.doc_off, ch.w, ch.z, ch.tables, ch.seed, ch.sweep_index,
                                      slice_len=slice_len)
            zg = s.z()
            msg = first_mismatch(zg, ch.z, doc_off)
            assert not msg, f"sweep {it}: " + msg
            st = s.stats()
            assert st["tokens"] == ch.stats[0] and st["a_branch"] == ch.stats[1] and \
                st["sum_min"] == ch.stats[2] and st["zero_mass"] == ch.stats[3] and \
                st["sum_inter"] == ch.stats[4] and st["docside"] == ch.stats[5], f"sweep {it}: stats {st} vs {ch.stats}"
            assert st["dead_rows"] == ch.dead_rows, f"sweep {it}: dead rows {st['dead_rows']} vs {ch.dead_rows}"
            if check_counts_every and it % check_counts_every == 0:
                assert np.array_equal(s.n(), ch.n().T), f"sweep {it}: n differs"
                assert np.array_equal(s.m(), ch.m()), f"sweep {it}: m differs"
        return s, ch
    except BaseException:
        s.close()
        raise
