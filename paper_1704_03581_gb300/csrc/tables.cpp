// Host construction of the fixed tables the Phi-step draws from.
//
// "Efficient sampling of Phi" (Section 3) draws Pois(beta + l) from
// precomputed Walker alias tables for l <= L = 100 and from a rounded
// Gaussian above.  Entries whose count n_{k,v} is zero have rate beta alone;
// they are drawn by skipping ahead over Geometric(1 - e^-beta) gaps, with a
// zero-truncated Pois(beta) value at each hit (the same law, entry by entry).
//
// All tables are exact-integer alias tables (Vose's construction in 64-bit
// integers) or IEEE double values from basic operations and the C library's
// expm1/erfc, so the device draws are reproducible bit for bit.
#include <cmath>
#include <cstring>
#include <mutex>
#include <thread>

#include "pulda_internal.h"

namespace pulda {
namespace {

constexpr double kTrunc = 9.094947017729282e-13;   // 2^-40: support cut-off relative to the mode
constexpr double kTwo40 = 1099511627776.0;          // 2^40: integer scale of the alias weights

// Poisson(lam) weights relative to the mode over j >= jmin, truncated where
// they fall below 2^-40.  Uses pmf(j+1)/pmf(j) = lam/(j+1) in both
// directions from the mode, so no exponential is evaluated.
bool poisson_weights(double lam, int jmin, int &lo, std::vector<uint64_t> &W) {
    long mode = static_cast<long>(std::floor(lam));
    if (mode < jmin) mode = jmin;
    std::vector<double> below;          // pmf(mode-1), pmf(mode-2), ... relative to pmf(mode)
    double w = 1.0;
    for (long j = mode; j > jmin; --j) {
        double next = w * static_cast<double>(j) / lam;
        if (next < kTrunc) break;
        below.push_back(next);
        w = next;
    }
    std::vector<double> rel(below.rbegin(), below.rend());
    rel.push_back(1.0);
    w = 1.0;
    for (long j = mode;; ++j) {
        double next = w * lam / static_cast<double>(j + 1);
        if (next < kTrunc) break;
        rel.push_back(next);
        w = next;
        if (rel.size() > 60000) return false;
    }
    lo = static_cast<int>(mode - static_cast<long>(below.size()));
    W.resize(rel.size());
    for (size_t j = 0; j < rel.size(); ++j) W[j] = static_cast<uint64_t>(std::floor(rel[j] * kTwo40 + 0.5));
    return true;
}

// Walker alias table by Vose's method with exact integer masses: slot s keeps
// outcome s when a uniform 32-bit word is below thr[s], else yields alias[s].
// Worklists are stacks filled in increasing index order.
void vose_build(const std::vector<uint64_t> &W, std::vector<uint32_t> &thr, std::vector<uint32_t> &alias) {
    const size_t n = W.size();
    thr.assign(n, 0xFFFFFFFFu);
    alias.resize(n);
    for (size_t j = 0; j < n; ++j) alias[j] = static_cast<uint32_t>(j);
    uint64_t total = 0;
    for (uint64_t x : W) total += x;
    if (total == 0) return;
    std::vector<uint64_t> mass(n);
    std::vector<uint32_t> small, large;
    for (size_t j = 0; j < n; ++j) {
        mass[j] = W[j] * static_cast<uint64_t>(n);
        (mass[j] < total ? small : large).push_back(static_cast<uint32_t>(j));
    }
    while (!small.empty() && !large.empty()) {
        uint32_t s = small.back(); small.pop_back();
        uint32_t l = large.back(); large.pop_back();
        thr[s] = static_cast<uint32_t>((static_cast<unsigned __int128>(mass[s]) << 32) / total);
        alias[s] = l;
        mass[l] -= total - mass[s];
        (mass[l] < total ? small : large).push_back(l);
    }
    // whatever is left holds exactly one slot of mass: keep it
}

double normal_cdf(double x) { return 0.5 * std::erfc(-x * 0.70710678118654752440); }

// Bisection for the normal quantile: the smallest point of the bisection
// with CDF >= p.
double normal_quantile(double p) {
    double a = -40.0, b = 40.0;
    for (int it = 0; it < 2000; ++it) {
        double mid = 0.5 * (a + b);
        if (mid == a || mid == b) break;
        if (normal_cdf(mid) < p) a = mid; else b = mid;
    }
    return b;
}

// Equiprobable inverse-normal nodes: node i is the (i / 2^16) quantile; the
// outer nodes are the 2^-24 and 1 - 2^-24 quantiles; the upper half mirrors
// the lower half.  Independent of beta, so built once per process.
const std::vector<double> &gauss_nodes() {
    static std::vector<double> nodes;
    static std::once_flag once;
    std::call_once(once, [] {
        const int half = kGaussCells / 2;
        nodes.assign(kGaussCells + 1, 0.0);
        nodes[0] = normal_quantile(5.9604644775390625e-08);
        // every node is its own bisection: split over host threads
        const int nt = static_cast<int>(std::max(1u, std::min(16u, std::thread::hardware_concurrency())));
        auto fill = [&](int t) {
            for (int i = 1 + t; i < half; i += nt) nodes[i] = normal_quantile(static_cast<double>(i) / kGaussCells);
        };
        std::vector<std::thread> th;
        for (int t = 1; t < nt; ++t) th.emplace_back(fill, t);
        fill(0);
        for (auto &x : th) x.join();
        nodes[half] = 0.0;
        for (int i = 0; i < half; ++i) nodes[kGaussCells - i] = -nodes[i];
    });
    return nodes;
}

}  // namespace

int build_host_tables(float beta_f, HostTables *out) {
    const double beta = static_cast<double>(beta_f);
    out->thr.clear(); out->alias.clear();
    out->off.assign(kL + 1, 0); out->lo.assign(kL + 1, 0); out->n.assign(kL + 1, 0);
    for (int t = 0; t <= kL; ++t) {
        int lo = 0;
        std::vector<uint64_t> W;
        // t = 0: zero-truncated Pois(beta) for the skip-ahead hits; t = l: Pois(beta + l)
        bool ok = t == 0 ? poisson_weights(beta, 1, lo, W) : poisson_weights(beta + static_cast<double>(t), 0, lo, W);
        if (!ok || W.empty() || W.size() > 65535) return -1;
        std::vector<uint32_t> thr, alias;
        vose_build(W, thr, alias);
        out->off[t] = static_cast<int32_t>(out->thr.size());
        out->lo[t] = lo;
        out->n[t] = static_cast<int32_t>(W.size());
        for (size_t j = 0; j < W.size(); ++j) {
            out->thr.push_back(thr[j]);
            out->alias.push_back(static_cast<uint16_t>(alias[j]));
        }
    }
    out->geo.resize(kGeoLen);
    for (int g = 0; g < kGeoLen; ++g) {
        double cdf = -std::expm1(-beta * static_cast<double>(g + 1));   // P(gap <= g)
        double t = std::floor(cdf * 4294967296.0);
        out->geo[g] = t >= 4294967295.0 ? 0xFFFFFFFFu : static_cast<uint32_t>(t);
    }
    out->gauss = gauss_nodes();
    return 0;
}

}  // namespace pulda
