"""Host checks of the z-step kernels' index arithmetic, for every K the
library accepts: each one-warp lane's bitmap words lie inside its word's
bitmap row, each count index (the leading zero, a lane's slots, the gap word
before a lane's slots that an empty gather slot reads) inside the warp's count
area for both count widths, the token records 16-byte aligned after it, and
the cooperative kernel's slots inside the row and its count area.  A small
host program compiled with nvcc against the library's own headers prints any
violation; no GPU is used."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1704_03581_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <cstdint>
#include "pulda_internal.h"
#include "zstep.cuh"
using namespace pulda;

static int bad = 0;
#define CHECK(cond, ...) do { if (!(cond)) { if (bad < 20) { std::printf(__VA_ARGS__); std::printf("\n"); } ++bad; } } while (0)

// topic k's count slot in units of the count type, from the start of the
// warp's region: a leading zero, then lane l's TPL topics at (TPL + 1) l + b
static long slot(int k, int tpl, int lead) { return lead + k + k / tpl; }

template <typename CT>
static void one_warp(int K) {
    const int tpl = z_lane_topics(K);
    const int lead = 4 / static_cast<int>(sizeof(CT));
    const long cap = static_cast<long>(z_count_words<CT>(K)) * lead;   // count slots of the area
    const int KW = (K + 31) / 32;
    const int nl = tpl == 32 ? KW : (K + tpl - 1) / tpl;                 // lanes that own topics
    CHECK(nl >= 1 && (K > kMaxKBitmap || nl <= 32), "K=%d: %d lanes own topics", K, nl);
    CHECK(slot(K - 1, tpl, lead) < cap, "K=%d CT%zu: last count slot %ld of %ld", K, sizeof(CT), slot(K - 1, tpl, lead), cap);
    CHECK(lead - 1 >= 0, "K=%d: no leading zero", K);
    for (int l = 0; l < nl; ++l) {
        const long before = lead + static_cast<long>(tpl + 1) * l - 1;   // an empty slot's read
        CHECK(before >= 0 && before < cap, "K=%d: lane %d reads %ld", K, l, before);
        if (l + 1 < nl) {
            const long gap = lead + static_cast<long>(tpl + 1) * l + tpl;
            CHECK(gap < cap, "K=%d: lane %d gap %ld", K, l, gap);
            // the gap is no topic's slot
            CHECK(gap != slot(tpl * (l + 1), tpl, lead) && gap != slot(tpl * l + tpl - 1, tpl, lead),
                  "K=%d: lane %d gap collides", K, l);
        }
    }
    CHECK(z_count_words<CT>(K) % 4 == 0, "K=%d: records not 16-byte aligned", K);
    CHECK((z_count_words<CT>(K) + 32 * kTokRecWords) % 2 == 0, "K=%d: counters not 8-byte aligned", K);
    if (K <= kMaxKBitmap) {
        const int KWp = bitmap_row_words(K);
        CHECK(KWp >= KW && KWp % 8 == 0, "K=%d: row of %d words", K, KWp);
        const int l = nl - 1;                                            // the last owning lane
        const int last_word = tpl == 64 ? 2 * l + 1 : tpl == 32 ? l : (l * tpl) >> 5;
        CHECK(last_word < KWp, "K=%d: lane %d reads word %d of %d", K, l, last_word, KWp);
        CHECK(32 * tpl >= K, "K=%d: %d lanes of %d topics do not cover K", K, 32, tpl);
    }
}

static void coop(int K) {
    const int KW = (K + 31) / 32;
    const int slots = 128;
    int R = 1;
    while (32 * KW > R * slots) R <<= 1;
    const long cap = z_m_words(K);
    CHECK(1 + mi(K - 1) < cap, "coop K=%d: last count %d of %ld", K, 1 + mi(K - 1), cap);
    if (K <= kMaxKBitmap) {
        CHECK(R <= 32, "coop K=%d: R=%d", K, R);
        const int owners = 32 * KW / R;
        CHECK(owners <= slots, "coop K=%d: %d owning slots", K, owners);
        const int wi = ((owners - 1) * R) >> 5;
        CHECK(wi < KW && wi < bitmap_row_words(K), "coop K=%d: slot word %d", K, wi);
    }
}

int main() {
    for (int K = 1; K <= kMaxK; ++K) {
        one_warp<uint32_t>(K);
        one_warp<uint16_t>(K);
        coop(K);
        if (K <= kMaxKGrouped) {
            const int wpl = bitmap_row_words(K) / 8;
            CHECK(wpl == 1 || wpl == 2 || wpl == 4, "grouped K=%d: %d words per lane", K, wpl);
        }
    }
    std::printf("violations %d\n", bad);
    return bad != 0;
}
"""


def test_z_step_indices_stay_inside_their_buffers(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    src = tmp_path / "layout.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "layout"
    r = subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-I", CSRC,
                        "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and "violations 0" in out.stdout, out.stdout + out.stderr
