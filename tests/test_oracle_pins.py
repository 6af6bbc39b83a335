"""Pins of the CPU oracle against things other than itself: published test
vectors, textbook distributions, closed forms, brute force and exact
enumeration of the stationary law.  No GPU is used here."""
import math
import os

import numpy as np
import pytest
from scipy import special, stats

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox

def test_philox_known_answers():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(x, 16) for x in line.split()])
    assert len(rows) == 3
    for r in rows:
        out = O.philox(r[0:4], r[4:6])
        assert [int(x) for x in out] == r[6:10]


# ------------------------------------------------------ alias tables (Vose)

def alias_masses(thr, alias, n_out=None):
    """Probability of each outcome implied by an alias table (exact up to the
    2^-32 threshold grid)."""
    n = thr.shape[0]
    n_out = n if n_out is None else n_out
    keep = thr.astype(np.float64) / 2.0 ** 32
    mass = np.zeros(n_out)
    np.add.at(mass, np.arange(n), keep / n)
    np.add.at(mass, alias, (1.0 - keep) / n)
    return mass


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_vose_reconstructs_weights(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 300))
    W = rng.integers(0, 2 ** 40, size=n).astype(np.uint64)
    W[rng.random(n) < 0.2] = 0
    if W.sum() == 0:
        W[0] = 1
    thr, alias, T = O.vose(W)
    assert T == int(W.astype(object).sum())
    mass = alias_masses(thr, alias)
    assert np.abs(mass - W.astype(np.float64) / T).max() <= 2.0 / 2 ** 32
    # zero-weight outcomes can never be drawn
    assert np.all(thr[W == 0] == 0)


def test_vose_uniform_weights_are_all_full():
    thr, alias, _ = O.vose(np.full(17, 5, dtype=np.uint64))
    assert np.all(thr == 0xFFFFFFFF) and np.all(alias == np.arange(17))


# ------------------------------------------ Poisson tables ("Efficient sampling of Phi")

@pytest.mark.parametrize("lam", [0.01 + 1, 0.01 + 5, 0.01 + 37, 0.01 + 100, 3.7])
def test_poisson_weights_are_the_pmf(lam):
    lo, W = O.pois_weights(lam)
    j = np.arange(lo, lo + W.shape[0])
    pmf = stats.poisson.pmf(j, lam)
    assert np.abs(W / W.sum() - pmf / pmf.sum()).max() < 1e-11
    # the support keeps everything above 2^-40 of the mode and loses < 2^-35 of the mass
    assert pmf.sum() > 1 - 2.0 ** -35
    mode = stats.poisson.pmf(math.floor(lam), lam)
    assert stats.poisson.pmf(lo - 1, lam) < mode * 2.0 ** -40 or lo == 0
    assert stats.poisson.pmf(j[-1] + 1, lam) < mode * 2.0 ** -40


def test_zero_truncated_weights():
    lo, W = O.pois_weights(0.01, jmin=1)
    assert lo == 1
    j = np.arange(1, 1 + W.shape[0])
    pmf = stats.poisson.pmf(j, 0.01)
    assert np.abs(W / W.sum() - pmf / pmf.sum()).max() < 1e-11


@pytest.mark.parametrize("l", [1, 2, 9, 50, 100])
def test_context_alias_tables_give_poisson(l):
    ctx = O.Ctx(0.01)
    lo, thr, alias = ctx.table(l)
    mass = alias_masses(thr, alias)
    j = np.arange(lo, lo + thr.shape[0])
    lam = float(np.float32(0.01)) + l
    pmf = stats.poisson.pmf(j, lam)
    assert np.abs(mass - pmf).max() < 3.0 * thr.shape[0] / 2 ** 32 + 1e-12


# ------------------------------------------------ geometric gaps and Gaussian

def test_geometric_gap_table_closed_form():
    beta = float(np.float32(0.01))
    thr = O.geo_table(beta)
    g = np.arange(O.LG)
    cdf = 1.0 - np.exp(-beta * (g + 1))
    assert np.all(np.abs(thr / 2.0 ** 32 - cdf) <= 2.0 ** -32)
    assert np.all(np.diff(thr.astype(np.int64)) >= 0)


def test_gaussian_table_is_the_normal_quantile():
    ctx = O.Ctx(0.01)
    Q = ctx.gauss()
    i = np.arange(1, O.GAUSS_CELLS // 2)
    assert np.abs(Q[1:O.GAUSS_CELLS // 2] - special.ndtri(i / O.GAUSS_CELLS)).max() < 1e-12
    assert abs(Q[0] - special.ndtri(2.0 ** -24)) < 1e-12
    assert np.array_equal(Q[::-1], -Q)                      # the normal law is symmetric
    assert np.all(np.diff(Q) > 0)


def test_gaussian_draw_moments():
    ctx = O.Ctx(0.01)
    rng = np.random.default_rng(7)
    x = rng.integers(0, 2 ** 32, size=(200000, 2), dtype=np.uint64)
    g = np.array([ctx.gauss_draw(a, b) for a, b in x])
    assert abs(g.mean()) < 0.01 and abs(g.var() - 1) < 0.01
    assert stats.kstest(g, "norm").pvalue > 1e-3


# --------------------------------------------------------------- the Phi-step

def _phi_samples(n_vk, beta, sweeps, seed=11):
    ctx = O.Ctx(beta)
    out = []
    for s in range(1, sweeps + 1):
        c, S, _ = O.phi_draw(ctx, n_vk, seed, s)
        out.append(c)
    return np.stack(out)


def _chi2_counts(sample, pmf_fn, min_exp=5.0):
    vals, cnt = np.unique(sample, return_counts=True)
    hi = int(vals.max()) + 1
    obs = np.bincount(sample, minlength=hi).astype(np.float64)
    exp = pmf_fn(np.arange(hi)) * sample.shape[0]
    tail = 1.0 - exp.sum() / sample.shape[0]
    # pool small cells into their neighbours from the left
    o, e = [], []
    acc_o = acc_e = 0.0
    for a, b in zip(obs, exp):
        acc_o += a
        acc_e += b
        if acc_e >= min_exp:
            o.append(acc_o); e.append(acc_e); acc_o = acc_e = 0.0
    if e:
        o[-1] += acc_o
        e[-1] += acc_e + tail * sample.shape[0]
    o, e = np.array(o), np.array(e)
    chi = ((o - e) ** 2 / e).sum()
    return stats.chi2.sf(chi, len(o) - 1)


def test_phi_entries_follow_poisson_beta_plus_n():
    """Eq. (9): c_{k,v} ~ Pois(beta + n_{k,v}), independently; rounded Gaussian above L."""
    beta = 0.01
    V, K = 120, 40
    n = np.zeros((V, K), dtype=np.int32)   # n[v, k]
    n[0:20, :] = 5          # every topic has mass, so no row is ever redrawn
    n[20:40, :] = 3
    n[40:60, :] = 150       # above L = 100: rounded Gaussian
    n[60:70, :] = 1
    c = _phi_samples(n, beta, 60)
    b = float(np.float32(beta))
    assert _chi2_counts(c[:, 20:40].ravel(), lambda j: stats.poisson.pmf(j, b + 3)) > 1e-4
    assert _chi2_counts(c[:, 0:20].ravel(), lambda j: stats.poisson.pmf(j, b + 5)) > 1e-4
    assert _chi2_counts(c[:, 60:70].ravel(), lambda j: stats.poisson.pmf(j, b + 1)) > 1e-4
    mu = b + 150
    rg = lambda j: stats.norm.cdf((j + 0.5 - mu) / math.sqrt(mu)) - stats.norm.cdf((j - 0.5 - mu) / math.sqrt(mu))
    assert _chi2_counts(c[:, 40:60].ravel(), rg) > 1e-4
    # beta-only entries: Pois(beta), so P(c > 0) = 1 - e^-beta and the values are ZTP
    zero = c[:, 70:].ravel()
    p_hit = 1 - math.exp(-b)
    hits = int((zero > 0).sum())
    assert stats.binomtest(hits, zero.shape[0], p_hit).pvalue > 1e-4
    assert _chi2_counts(zero, lambda j: stats.poisson.pmf(j, b)) > 1e-4


def _geo_pmf(j, p):
    return p * (1.0 - p) ** j


def test_beta_field_chains_past_the_gap_table():
    """Eq. (9) with n = 0: every entry is an independent Pois(beta), so the
    positions of the nonzero ones are i.i.d. Bernoulli(1 - e^-beta).  At
    beta = 0.001 a gap exceeds the 1024-entry table of the skip-ahead walk
    with probability e^-1.02 ~ 0.36, so the walk's chaining past the table
    (a run of 1024 misses, then a fresh gap) is taken in about a third of the
    gaps, often several times in a row.  Pinned three ways: the number of
    hits (binomial), the gaps between hits (chi-square against
    Geometric(1 - e^-beta), gaps of 1023/1024 and 2047/2048 binned alone so an
    off-by-one in the chaining shows), and the hit rate at every position
    (flat; the positions where chained runs end are binned alone)."""
    beta, K, V, sweeps = 0.001, 4096, 1000, 50
    b = float(np.float32(beta))
    p = -math.expm1(-b)
    n = np.zeros((V, K), dtype=np.int32)
    n[0, :] = 100           # word 0 keeps every row alive; words 1.. are pure beta-field walks
    ctx = O.Ctx(beta)
    G = 3072                # gaps of at least G are binned together (censoring)
    edges = [0, 64, 256, 512, 768, 1000, 1023, 1024, 1025, 1100, 1500, 2047, 2048, 2049, 2600, G]
    gap_obs = np.zeros(len(edges), np.float64)      # bins [e_i, e_{i+1}) and [G, inf)
    pos_hits = np.zeros(K, np.int64)
    hits = ones = 0
    cols = 0
    for s in range(1, sweeps + 1):
        c, S, dead = O.phi_draw(ctx, n, 41, s)
        assert dead == 0
        f = c[1:, :]
        cols += f.shape[0]
        nz = f > 0
        pos_hits += nz.sum(axis=0)
        hits += int(nz.sum())
        ones += int((f == 1).sum())
        for row in nz:
            h = np.flatnonzero(row)
            # starts: the walk's origin (-1) and every hit early enough that a
            # gap of G fits before the end (a stopping time: the next gap is
            # Geometric, independent of the past)
            starts = np.concatenate([[-1], h[h <= K - 1 - G]])
            nxt = np.searchsorted(h, starts, side="right")
            if h.size == 0:
                g = np.full(starts.shape, G)
            else:
                g = np.where(nxt < h.size, h[np.minimum(nxt, h.size - 1)] - starts - 1, G)
            g = np.minimum(g, G)
            gap_obs += np.bincount(np.searchsorted(edges, g, side="right") - 1, minlength=len(edges))
    # 1. number of hits
    assert stats.binomtest(hits, cols * K, p).pvalue > 1e-4
    # values at hits are zero-truncated Pois(beta): P(c = 1 | c > 0) = beta e^-beta / (1 - e^-beta)
    assert stats.binomtest(ones, hits, b * math.exp(-b) / p).pvalue > 1e-4
    # 2. gaps
    tot = gap_obs.sum()
    cdf = lambda j: 1.0 - (1.0 - p) ** j           # P(gap < j)
    probs = np.array([cdf(edges[i + 1]) - cdf(edges[i]) for i in range(len(edges) - 1)] + [(1.0 - p) ** G])
    assert abs(probs.sum() - 1.0) < 1e-12
    exp = probs * tot
    assert gap_obs[-1] > 1000 and gap_obs[edges.index(1024)] > 10      # the chained branch is exercised
    chi = ((gap_obs - exp) ** 2 / exp).sum()
    assert stats.chi2.sf(chi, len(exp) - 1) > 1e-4, (gap_obs, exp)
    # 3. hit rate by position: single positions around the ends of chained runs
    singles = [1022, 1023, 1024, 1025, 2046, 2047, 2048, 2049, 3070, 3071, 3072, 3073]
    o, e = [], []
    mask = np.ones(K, bool)
    for j in singles:
        o.append(pos_hits[j]); e.append(cols * p); mask[j] = False
    for lo in range(0, K, 256):
        sel = np.flatnonzero(mask[lo:lo + 256]) + lo
        o.append(pos_hits[sel].sum()); e.append(cols * p * sel.size)
    o, e = np.array(o, np.float64), np.array(e)
    chi = ((o - e) ** 2 / e).sum()
    assert stats.chi2.sf(chi, len(o) - 1) > 1e-4


def test_dead_row_redraw_walk_chains_past_the_gap_table():
    """A redrawn row walks the beta field across V words with the same
    skip-ahead; with V = 6000 and beta = 0.0002 its gaps pass the table in most
    rows.  Given S_k > 0 the hit positions are i.i.d. Bernoulli(1 - e^-beta)
    conditioned on at least one hit, so every position has the same hit rate
    and the number of hits is a zero-truncated binomial."""
    beta, V, K, sweeps = 0.0002, 6000, 40, 60
    b = float(np.float32(beta))
    p = -math.expm1(-b)
    n = np.zeros((V, K), dtype=np.int32)
    ctx = O.Ctx(beta)
    pos_hits = np.zeros(V, np.int64)
    counts = []
    dead_total = 0
    for s in range(1, sweeps + 1):
        c, S, dead = O.phi_draw(ctx, n, 43, s)
        dead_total += dead
        assert (S > 0).all()
        nz = c > 0                      # [V, K]
        pos_hits += nz.sum(axis=1)
        counts.extend(nz.sum(axis=0).tolist())
    rows = sweeps * K
    assert dead_total > rows // 4                   # P(S_k = 0) = e^{-V beta} ~ 0.30
    q0 = (1.0 - p) ** V
    # hits per row: Binomial(V, p) given >= 1
    counts = np.array(counts)
    kk = np.arange(1, 8)
    pmf = stats.binom.pmf(kk, V, p) / (1 - q0)
    o = np.append(np.bincount(counts, minlength=9)[1:8], (counts >= 8).sum()).astype(np.float64)
    e = np.append(pmf, 1 - pmf.sum()) * rows
    chi = ((o - e) ** 2 / e).sum()
    assert stats.chi2.sf(chi, len(o) - 1) > 1e-4
    # every position equally likely: E[hits at v] = rows * p / (1 - q0)
    rate = rows * p / (1 - q0)
    singles = [1022, 1023, 1024, 1025, 2046, 2047, 2048, 2049]
    mask = np.ones(V, bool)
    o, e = [], []
    for j in singles:
        o.append(pos_hits[j]); e.append(rate); mask[j] = False
    for lo in range(0, V, 500):
        sel = np.flatnonzero(mask[lo:lo + 500]) + lo
        o.append(pos_hits[sel].sum()); e.append(rate * sel.size)
    o, e = np.array(o, np.float64), np.array(e)
    chi = ((o - e) ** 2 / e).sum()
    assert stats.chi2.sf(chi, len(o) - 1) > 1e-4


def test_phi_row_sums_and_normalisation():
    beta = 0.01
    rng = np.random.default_rng(3)
    V, K = 300, 25
    n = rng.poisson(2.0, size=(V, K)).astype(np.int32)
    ctx = O.Ctx(beta)
    c, S, _ = O.phi_draw(ctx, n, 5, 1)
    assert np.array_equal(S, c.sum(axis=0).astype(np.int64))
    t = O.WordTables(c, S, np.full(K, 0.1, np.float32))
    phi = t.phi_dense().astype(np.float64)
    assert np.abs(phi.sum(axis=1) - 1).max() < 1e-6          # rows of Phi are distributions
    nz = c.T > 0
    assert np.array_equal(phi > 0, nz)                      # sparsity pattern of Phi = that of c
    ref = (c.T.astype(np.float64) / S[:, None])
    assert np.array_equal(phi[nz].astype(np.float32), ref[nz].astype(np.float32))


def test_dead_rows_are_conditioned_on_nonzero_sum():
    """Definition "Poisson Polya Urn": the normalisation needs a nonzero sum;
    the hierarchical representation (Eq. 8) draws the total from Pois+.  A row
    with S_k = 0 is redrawn, so its law is the Poisson law given S_k > 0."""
    beta = 0.3
    V, K = 3, 1
    n = np.zeros((V, K), dtype=np.int32)
    ctx = O.Ctx(beta)
    b = float(np.float32(beta))
    samples = []
    dead_total = 0
    for s in range(1, 6001):
        c, S, dead = O.phi_draw(ctx, n, 21, s)
        assert S[0] > 0
        dead_total += dead
        samples.append(tuple(int(x) for x in c[:, 0]))
    assert dead_total > 1000                                 # P(S=0) = e^{-0.9} ~ 0.41
    # exact conditional law over the states seen, pooled beyond total 3
    p0 = math.exp(-3 * b)
    def pmf(state):
        return np.prod([stats.poisson.pmf(x, b) for x in state]) / (1 - p0)
    keys = sorted(set(samples))
    obs = np.array([samples.count(k) for k in keys], dtype=np.float64)
    exp = np.array([pmf(k) for k in keys]) * len(samples)
    big = exp < 5
    o = np.append(obs[~big], obs[big].sum())
    e = np.append(exp[~big], len(samples) - exp[~big].sum())
    chi = ((o - e) ** 2 / e).sum()
    assert stats.chi2.sf(chi, len(o) - 1) > 1e-4


# ----------------------------------------------------- per-word z-step tables

def test_word_tables_reproduce_the_conditional():
    """The fixed-point weights give p(k) proportional to phi_{k,v}(alpha_k + m_k)
    ("Efficient sampling of z") to within 2^-20 relative."""
    rng = np.random.default_rng(5)
    V, K = 50, 64
    c = (rng.poisson(0.7, size=(V, K)) * rng.integers(1, 900, size=(V, K))).astype(np.uint32)
    c[0] = 0
    S = c.sum(axis=0).astype(np.int64)
    S[S == 0] = 1
    alpha = rng.uniform(0.05, 2.0, size=K).astype(np.float32)
    t = O.WordTables(c, S, alpha)
    for v in range(V):
        top, q, athr, atop, phi32 = t.column(v)
        assert top.shape[0] == int((c[v] > 0).sum())
        if top.shape[0] == 0:
            assert t.A[v] == 0
            continue
        assert np.all(np.diff(top) > 0)
        assert 2 ** 23 <= q.max() <= 2 ** 24 and q.min() >= 1
        m = rng.integers(0, 40, size=K)
        phi = c[v, top].astype(np.float64) / S[top]
        p = phi * (alpha[top].astype(np.float64) + m[top])
        p /= p.sum()
        a = np.floor(q.astype(np.float64) * alpha[top] * 2 ** 16 + 0.5)
        w = a + q.astype(np.float64) * m[top] * 2 ** 16
        assert int(a.sum()) == int(t.A[v])
        # rounding q to an integer moves an entry by at most half a unit;
        # the shared normalisation moves every entry by at most ~n 2^-24
        rel = np.abs(w / w.sum() - p) / p
        assert np.all(rel <= 0.5 / q + 2.0 ** -17)
        assert rel[q >= 2 ** 20].max() < 2.0 ** -17
        # the alias table draws topic top[j] with probability a_j / A
        mass = alias_masses(athr, np.searchsorted(top, atop))
        assert np.abs(mass - a / a.sum()).max() <= 2.0 * top.shape[0] / 2 ** 32


# ----------------------------------------------------------------- the z-step

def _tables_from_phi(phi_kv, alpha, scale=10 ** 6):
    """Word tables whose phi equals phi_kv (given as exact ratios c/S)."""
    K, V = phi_kv.shape
    c = np.rint(phi_kv * scale).astype(np.uint32).T.copy()
    S = np.full(K, scale, dtype=np.int64)
    return O.WordTables(c, S, np.asarray(alpha, np.float32)), c.T.astype(np.float64) / scale


def test_z_conditional_chi_square():
    """p(z_i = k) proportional to phi_{k,v(i)} (alpha_k + m^{-i}_{d,k}) (Algorithm 2)."""
    K, V = 6, 3
    phi = np.array([[0.5, 0.2, 0.3],
                    [0.1, 0.6, 0.3],
                    [0.25, 0.25, 0.5],
                    [0.7, 0.1, 0.2],
                    [0.0, 0.5, 0.5],
                    [0.3, 0.3, 0.4]])
    alpha = np.array([0.1, 0.5, 0.2, 0.1, 0.3, 0.05], np.float32)
    t, phi_x = _tables_from_phi(phi, alpha)
    # token 0 (word 0, topic 1) first, then other tokens that define m^{-0}
    w = np.array([0, 1, 2, 0, 0, 1, 2, 2], np.int32)
    z0 = np.array([1, 3, 3, 0, 3, 5, 2, 0], np.int16)
    doc_off = np.array([0, 8], np.int64)
    m = np.bincount(z0[1:], minlength=K).astype(np.float64)  # m^{-0}; topic 1 has only token 0
    p = phi_x[:, 0] * (alpha.astype(np.float64) + m)
    p /= p.sum()
    draws = np.array([O.z_step(doc_off, w, z0, t, 99, s)[0][0] for s in range(1, 40001)])
    obs = np.bincount(draws, minlength=K)
    assert obs[4] == 0                                      # phi_{4,0} = 0: never drawn
    keep = p > 0
    chi = ((obs[keep] - p[keep] * draws.shape[0]) ** 2 / (p[keep] * draws.shape[0])).sum()
    assert stats.chi2.sf(chi, keep.sum() - 1) > 1e-4
    # the removal of token i matters here: without it topic 1 would carry
    # phi(alpha+1) instead of phi*alpha, far outside the statistical tolerance
    assert obs[1] < 0.5 * draws.shape[0] * phi_x[1, 0] * (alpha[1] + 1) / (phi_x[:, 0] * (alpha + m + np.eye(K)[1])).sum()


def test_z_step_stationary_law_by_enumeration():
    """With Phi fixed, the z-step's stationary law is
    p(z | Phi, w) proportional to prod_i phi_{z_i, w_i} prod_{d,k} Gamma(alpha_k + m_{d,k}),
    the partially collapsed target of Algorithm 2 (theta integrated out).
    2 topics, 3 words, 4 documents, 6 tokens: 64 states, enumerated exactly."""
    K = 2
    phi = np.array([[0.6, 0.3, 0.1],
                    [0.1, 0.3, 0.6]])
    alpha = np.array([0.5, 0.5], np.float32)
    t, phi_x = _tables_from_phi(phi, alpha)
    w = np.array([0, 2, 1, 0, 2, 1], np.int32)
    doc_off = np.array([0, 2, 3, 5, 6], np.int64)
    N = w.shape[0]
    states = np.array([[(s >> i) & 1 for i in range(N)] for s in range(2 ** N)])
    logp = np.zeros(2 ** N)
    for si, zz in enumerate(states):
        lp = np.log(phi_x[zz, w]).sum()
        for d in range(4):
            mm = np.bincount(zz[doc_off[d]:doc_off[d + 1]], minlength=K)
            lp += special.gammaln(alpha.astype(np.float64) + mm).sum()
        logp[si] = lp
    p = np.exp(logp - logp.max())
    p /= p.sum()
    z = np.zeros(N, np.int16)
    counts = np.zeros(2 ** N)
    weights = 1 << np.arange(N)
    n_sweeps = 300000
    for s in range(1, n_sweeps + 1):
        z, _ = O.z_step(doc_off, w, z, t, 7, s)
        counts[int((z.astype(np.int64) * weights).sum())] += 1
    tv = 0.5 * np.abs(counts / n_sweeps - p).sum()
    assert tv < 0.015, tv
    # a sampler that forgot alpha's Gamma terms (independent tokens) has a
    # different law; the test can tell them apart
    q = np.exp(np.array([np.log(phi_x[zz, w]).sum() for zz in states]))
    q /= q.sum()
    assert 0.5 * np.abs(q - p).sum() > 0.1


# -------------------------------------------------------- counts and init

def test_counts_brute_force():
    rng = np.random.default_rng(8)
    K, V, N = 7, 11, 500
    w = rng.integers(0, V, N).astype(np.int32)
    z = rng.integers(0, K, N).astype(np.int16)
    n = O.count_n(w, z, K, V)
    ref = np.zeros((V, K), np.int32)
    for a, b in zip(w, z):
        ref[a, b] += 1
    assert np.array_equal(n, ref)
    doc_off = np.array([0, 0, 100, 101, 400, 500], np.int64)   # includes an empty document
    m = O.doc_topic(doc_off, z, K)
    for d in range(5):
        assert np.array_equal(m[d], np.bincount(z[doc_off[d]:doc_off[d + 1]], minlength=K))


def test_init_is_uniform():
    K = 37
    z = O.init_z(200000, K, 3)
    obs = np.bincount(z, minlength=K)
    assert stats.chisquare(obs).pvalue > 1e-4


def test_chain_invariants_tiny_corpus():
    from paper_1704_03581_gb300 import synth
    c = synth.tiny()
    ch = O.Chain(c.w, c.doc_off, 20, c.V, 0.1, 0.01, seed=0).sweep(3)
    m = ch.m()
    assert np.array_equal(m.sum(axis=1), np.diff(c.doc_off))           # sum_k m_{d,k} = N_d
    n = ch.n()
    assert n.sum() == c.N                                              # sum n = N
    assert np.array_equal(n.sum(axis=0), np.bincount(ch.z, minlength=20))
    assert ch.z.min() >= 0 and ch.z.max() < 20
    assert np.abs(ch.tables.phi_dense().astype(np.float64).sum(axis=1) - 1).max() < 1e-6
    assert ch.stats[0] == c.N


# ---------------------------------------------------------------- log posterior
# The diagnostic of Section 5 is the collapsed log joint log p(w, z | alpha, beta)
# of Dirichlet-multinomial LDA.  It is pinned by what the model itself fixes:
# a probability law over every (w, z) of a given shape sums to one; its ratios
# are the collapsed Gibbs conditional; a one-token corpus has a closed form.

@pytest.mark.parametrize("K,V,alpha,beta,k", [(2, 3, [0.25, 0.75], 0.5, 1), (5, 7, [0.125] * 5, 0.03125, 3),
                                               (1, 1, [2.0], 1.5, 0)])
def test_log_posterior_single_token_closed_form(K, V, alpha, beta, k):
    """One document of one token, word 0, topic k: p(z=k) = alpha_k / sum(alpha), p(w | z) = 1/V."""
    out = O.log_posterior(np.array([0, 1]), np.array([0]), np.array([k]), K, V, alpha, beta)
    want = math.log(alpha[k] / sum(alpha)) - math.log(V)
    assert abs(out[0] - want) < 1e-12
    assert abs(out[0] - out[1] - out[2]) < 1e-12


@pytest.mark.parametrize("lengths,K,V,alpha,beta", [((2, 1), 2, 2, [0.25, 1.75], 0.375),
                                                     ((1, 0, 2), 3, 2, [0.5, 0.125, 1.0], 0.75),
                                                     ((4,), 2, 3, [0.5, 0.5], 0.0625)])
def test_log_posterior_sums_to_one_over_every_corpus(lengths, K, V, alpha, beta):
    """sum over all words w in V^N and topics z in K^N of p(w, z | alpha, beta) = 1
    for fixed document lengths (an empty document contributes a factor 1)."""
    import itertools
    doc_off = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    N = int(doc_off[-1])
    total = 0.0
    for w in itertools.product(range(V), repeat=N):
        for z in itertools.product(range(K), repeat=N):
            total += math.exp(O.log_posterior(doc_off, np.array(w), np.array(z), K, V, alpha, beta)[0])
    assert abs(total - 1.0) < 1e-12


def test_log_posterior_ratios_are_the_collapsed_gibbs_conditional():
    """exp(LP(z_i = k) - LP(z_i = k0)) = f(k) / f(k0) with
    f(k) = (m^-i_{d,k} + alpha_k) (n^-i_{k,w_i} + beta) / (n^-i_k + V beta)  (Griffiths and Steyvers, 2004)."""
    rng = np.random.default_rng(11)
    K, V, beta = 4, 6, 0.2
    alpha = np.array([0.1, 0.5, 0.25, 1.5], dtype=np.float32)
    doc_off = np.array([0, 5, 9, 16], np.int64)
    N = int(doc_off[-1])
    w = rng.integers(0, V, N).astype(np.int32)
    z = rng.integers(0, K, N).astype(np.int16)
    for i in (0, 4, 7, 15):
        d = int(np.searchsorted(doc_off, i, side="right") - 1)
        keep = np.arange(N) != i
        zi = z[keep]
        m = np.bincount(z[doc_off[d]:doc_off[d + 1]][np.arange(doc_off[d], doc_off[d + 1]) != i], minlength=K)
        n_kv = np.zeros((K, V))
        np.add.at(n_kv, (zi, w[keep]), 1)
        f = (m + alpha.astype(np.float64)) * (n_kv[:, w[i]] + beta) / (n_kv.sum(1) + V * beta)
        lp = []
        for k in range(K):
            zz = z.copy()
            zz[i] = k
            lp.append(O.log_posterior(doc_off, w, zz, K, V, alpha, beta)[0])
        got = np.exp(np.array(lp) - lp[0])
        assert np.allclose(got, f / f[0], rtol=1e-11, atol=0), (i, got, f / f[0])


# ------------------------------------------------------- Dirichlet Phi (Algorithm 1)
# phi_k ~ Dir(n_k + beta) through Gamma draws (Marsaglia and Tsang), with the
# oracle's own float log and exp.  Pinned to libm, to scipy's Gamma and Beta
# laws, and to the z conditional.

def _ulps(a, b):
    ia = int(np.array(np.float32(a)).view(np.int32))
    ib = int(np.array(np.float32(b)).view(np.int32))
    return abs(ia - ib)


def test_own_logf_expf_within_two_ulps():
    """Against the double-precision library result rounded to float, over normal and subnormal
    arguments of log and the arguments exp takes (|x| <= 104; subnormal results included)."""
    rng = np.random.default_rng(21)
    xs = np.concatenate([rng.uniform(0, 1, 3000), np.exp(rng.uniform(-100, 88, 3000)),
                         np.float32(2.0) ** rng.integers(-149, -126, 100) * rng.uniform(1, 2, 100),
                         [1.0, 0.5, 2.0, 1.41421354, 1.4142137, 1e-45]]).astype(np.float32)
    for x in xs[xs > 0]:
        assert _ulps(O.logf(x), np.log(np.float64(x))) <= 2, x
    for t in np.concatenate([rng.uniform(-104, 0, 3000), rng.uniform(-1, 1, 1000), rng.uniform(0, 88, 1000)]):
        t = np.float32(t)
        assert _ulps(O.expf(t), np.exp(np.float64(t))) <= 2, t
    assert O.expf(-104.5) == 0.0


@pytest.mark.parametrize("a", [0.01, 0.1, 0.5, 1.0, 3.7, 40.0, 1500.0])
def test_gamma_draws_follow_the_gamma_law(a):
    """20,000 keyed draws against G(a, 1): KS test, and the mean.  At a = 0.01 about
    36% of the law lies below the smallest float, where draws underflow to 0; there
    a chi-square over logarithmic bins (the first holding the zeros) replaces KS."""
    ctx = O.Ctx(0.01)
    n = 20000
    g = np.array([O.gamma_draw(ctx, a, 77, 3, k, 5) for k in range(n)], dtype=np.float64)
    assert np.all(g >= 0)
    a32 = float(np.float32(a))
    law = stats.gamma(a32)
    if a32 < 0.05:
        edges = np.array([0.0, 1e-40, 1e-30, 1e-20, 1e-10, 1e-5, 1e-3, 1e-2, 0.1, np.inf])
        obs = np.histogram(g, bins=edges)[0]
        exp = n * np.diff(law.cdf(edges))
        assert stats.chisquare(obs, exp).pvalue > 1e-4, (obs, exp)
    else:
        assert stats.kstest(g, law.cdf).pvalue > 1e-4
    assert abs(g.mean() - a32) < 5 * math.sqrt(a32 / n)


def test_dirichlet_phi_marginals_are_beta():
    """Algorithm 1: phi_{k,.} ~ Dir(n_{k,.} + beta), so phi_{k,v} ~ Beta(n_{k,v} + beta, sum_v (n + beta) - (n_{k,v} + beta)).
    KS over 3,000 sweeps of the keyed draws; every row sums to 1."""
    beta = 0.5
    ctx = O.Ctx(beta)
    n_vk = np.array([[0, 3, 1], [2, 0, 0], [5, 1, 0], [0, 0, 0], [1, 7, 2]], dtype=np.int32)    # V=5, K=3
    V, K = n_vk.shape
    phis = []
    for sw in range(1, 3001):
        g, S = O.phi_draw_dir(ctx, n_vk, 9, sw)
        phi = g.astype(np.float64) / S
        assert np.allclose(phi.sum(axis=0), 1.0, atol=1e-6)
        phis.append(phi)
    phis = np.array(phis)
    tot = n_vk.sum(axis=0) + V * beta
    for v, k in [(0, 0), (0, 1), (2, 0), (3, 2), (4, 1)]:
        a = n_vk[v, k] + beta
        assert stats.kstest(phis[:, v, k], stats.beta(a, tot[k] - a).cdf).pvalue > 1e-4, (v, k)


def test_dirichlet_row_sums_are_the_row_totals():
    """S_k is the sum of row k of the Gamma draws, to within V eps S_k of the exact sum."""
    rng = np.random.default_rng(4)
    ctx = O.Ctx(0.01)
    n_vk = rng.integers(0, 3, size=(700, 6)).astype(np.int32)
    g, S = O.phi_draw_dir(ctx, n_vk, 3, 2)
    for k in range(6):
        exact = math.fsum(g[:, k].astype(np.float64))
        assert abs(S[k] - exact) <= 700 * 2.0 ** -53 * exact


def test_dirichlet_word_tables_reproduce_the_conditional():
    """Weights from Gamma draws give p(k) proportional to phi_{k,v}(alpha_k + m_k) to within
    0.5/(q - 0.5) + 2^-17 for kept entries; dropped entries have phi below 2^-24 of the column maximum."""
    rng = np.random.default_rng(6)
    ctx = O.Ctx(0.01)
    V, K = 40, 96
    n_vk = (rng.poisson(0.5, size=(V, K)) * rng.integers(1, 50, size=(V, K))).astype(np.int32)
    g, S = O.phi_draw_dir(ctx, n_vk, 11, 3)
    alpha = rng.uniform(0.05, 2.0, size=K).astype(np.float32)
    t = O.WordTables(g, S, alpha, dirichlet=True)
    for v in range(V):
        top, q, athr, atop, phi32 = t.column(v)
        phi_all = g[v].astype(np.float64) * (1.0 / S)
        keep = np.zeros(K, bool)
        keep[top] = True
        assert np.all(np.diff(top) > 0)
        # kept iff phi >= 2^(e-25), the column maximum being in [2^(e-1), 2^e)
        e = math.frexp(phi_all.max())[1]
        assert np.all(phi_all[~keep] < 2.0 ** (e - 25)) and np.all(phi_all[keep] >= 2.0 ** (e - 25) * (1 - 2.0 ** -30))
        assert np.all(phi_all[~keep] < 2.0 ** -24 * phi_all.max())
        assert 2 ** 23 <= q.max() <= 2 ** 24 and q.min() >= 1
        m = rng.integers(0, 40, size=K)
        p = phi_all[top] * (alpha[top].astype(np.float64) + m[top])
        p /= p.sum()
        a = np.floor(q.astype(np.float64) * alpha[top] * 2 ** 16 + 0.5)
        w = a + q.astype(np.float64) * m[top] * 2 ** 16
        assert int(a.sum()) == int(t.A[v])
        rel = np.abs(w / w.sum() - p) / p
        assert np.all(rel <= 0.5 / (q - 0.5) + 2.0 ** -17)   # round to nearest: x >= q - 1/2
        mass = alias_masses(athr, np.searchsorted(top, atop))
        assert np.abs(mass - a / a.sum()).max() <= 2.0 * top.shape[0] / 2 ** 32


def test_dirichlet_chain_invariants():
    """The oracle chain in Dirichlet mode keeps its counts consistent and its topics in range."""
    rng = np.random.default_rng(8)
    lengths = rng.integers(1, 40, size=30)
    off = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    w = rng.integers(0, 25, int(off[-1])).astype(np.int32)
    ch = O.Chain(w, off, 7, 25, 0.3, 0.05, seed=4, dirichlet=True)
    ch.sweep(3)
    assert ch.z.min() >= 0 and ch.z.max() < 7
    assert ch.m().sum(axis=1).tolist() == lengths.tolist()
    assert ch.n().sum() == off[-1]


# ------------------------------------------------- stale-count slices (outside the paper)
# Long documents cut into slices that start from the pass-start counts m0 and
# update only their own copy.  Pinned to Algorithm 2 (one slice per document)
# and to the stale conditional p(k) ~ phi_{k,v}(alpha_k + m0_k - [k = z_i]).

def test_sliced_z_step_with_whole_documents_is_algorithm_2():
    rng = np.random.default_rng(31)
    K, V = 7, 30
    c = (rng.poisson(0.6, size=(V, K)) * rng.integers(1, 200, size=(V, K))).astype(np.uint32)
    S = np.maximum(c.sum(axis=0).astype(np.int64), 1)
    t = O.WordTables(c, S, rng.uniform(0.05, 1.0, K).astype(np.float32))
    lengths = rng.integers(0, 60, size=25)
    off = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    w = rng.integers(0, V, int(off[-1])).astype(np.int32)
    z = rng.integers(0, K, int(off[-1])).astype(np.int16)
    exact = O.z_step(off, w, z, t, 5, 3)
    for L in (0, int(lengths.max()), 10 ** 6):
        got = O.z_step(off, w, z, t, 5, 3, slice_len=L)
        assert np.array_equal(got[0], exact[0]) and np.array_equal(got[1], exact[1])
    # shorter slices change the chain but keep every count consistent
    got = O.z_step(off, w, z, t, 5, 3, slice_len=7)
    assert got[1][0] == off[-1] and got[0].min() >= 0 and got[0].max() < K


def test_sliced_z_step_uses_the_pass_start_counts():
    """One-token slices: token 5 of a six-token document draws from phi(alpha + m0 - e_{z_5}) whatever
    tokens 0-4 draw.  Phi strongly prefers topic 1 while every token starts in topic 0, so the
    exact sampler (which sees tokens 0-4 move) gives a clearly different law."""
    K = 2
    phi = np.array([[0.1], [0.9]])
    alpha = np.array([0.5, 0.5], np.float32)
    t, phi_x = _tables_from_phi(phi, alpha)
    w = np.zeros(6, np.int32)
    z0 = np.zeros(6, np.int16)
    off = np.array([0, 6], np.int64)
    m0 = np.array([5.0, 0.0])                       # pass-start counts without token 5
    p = phi_x[:, 0] * (alpha.astype(np.float64) + m0)
    p /= p.sum()
    n = 20000
    sliced = np.array([O.z_step(off, w, z0, t, 7, s, slice_len=1)[0][5] for s in range(1, n + 1)])
    obs = np.bincount(sliced, minlength=K)
    chi = ((obs - p * n) ** 2 / (p * n)).sum()
    assert stats.chi2.sf(chi, K - 1) > 1e-4
    exact = np.array([O.z_step(off, w, z0, t, 7, s)[0][5] for s in range(1, n + 1)])
    assert abs(np.mean(exact == 1) - p[1]) > 0.1     # the exact law is far from the stale one


# ------------------------------------------------- the oracle on many threads

def test_threaded_oracle_equals_the_single_threaded_one():
    """The document- and word-parallel oracle (Algorithm 2's documents are
    independent given Phi; each word's Phi entries are independent) gives the
    single-threaded results bit for bit: topics, counts, Poisson counts, row
    sums, dead rows, tables and every z-step counter, on a corpus whose
    small V and beta kill rows (so the parallel redraw runs too)."""
    from paper_1704_03581_gb300 import synth
    c = synth.tiny()
    rng = np.random.default_rng(9)
    cases = [(c.w, c.doc_off, 20, c.V, 0.1, 0.01),
             (rng.integers(0, 40, size=1500).astype(np.int32), np.arange(0, 1501, 30, dtype=np.int64), 2000, 40,
              0.2, 0.002)]
    for w, off, K, V, alpha, beta in cases:
        a = O.Chain(w, off, K, V, alpha, beta, seed=4)
        b = O.Chain(w, off, K, V, alpha, beta, seed=4, threads=5)
        dead = 0
        for _ in range(3):
            a.sweep(1)
            b.sweep(1)
            assert np.array_equal(a.z, b.z) and np.array_equal(a.stats, b.stats)
            assert np.array_equal(a.c, b.c) and np.array_equal(a.S, b.S) and a.dead_rows == b.dead_rows
            for k in ("ncol", "topic", "q", "A", "athr", "atopic", "phi32"):
                assert np.array_equal(getattr(a.tables, k), getattr(b.tables, k)), k
            assert np.array_equal(O.count_n(a.w, a.z, K, V), O.count_n(b.w, b.z, K, V, threads=3))
            dead += a.dead_rows
        if beta < 0.01:
            assert dead > 0
