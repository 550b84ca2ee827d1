"""Host logic of the search kernel: the per-query shared-memory layout.

A small host program built with nvcc evaluates make_layout over the whole
supported parameter grid and checks that every region is 16-byte aligned,
that regions follow one another without overlap, that the shared region
holds each of its users (walk lists, radix counters, bridge window, staged
rows), that the heap and visited set hold a budget's entries, and that one
query fits the shared memory of a CTA.  No GPU is needed."""
from __future__ import annotations

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r'''
#include "ann_search_dev.cuh"
#include <cstdio>
using namespace ann;
static long bad = 0, checked = 0;
#define CHECK(c) do { if (!(c)) { if (bad < 10) printf("violated: %s  dtype=%d d=%d P=%d n=%d T=%d kmax=%d R=%d b=%d grp=%d stg=%d\n", #c, dtype, d, P, n, capT, kmax, R, b, (int)grouped, (int)stage); bad++; } } while (0)
int main() {
    const int Ds[] = {64, 96, 128, 384, 512};
    for (int dtype = 0; dtype < 2; dtype++) for (int d : Ds) for (int P = 2; P <= 4; P++) {
        if (d % P || (dtype == ANN_U8 && d % 16) || (dtype == ANN_F32 && d % 4)) continue;
        const int PA = P - 1 < 2 ? P - 1 : 2;
        for (int n : {8, 16, 64, 128, 256}) for (int capT = 32; capT <= 8192; capT *= 2)
        for (int kmax : {1, 10, 100, 128}) for (int R : {8, 16, 20, 32}) for (int b : {1, 5, 8})
        for (bool grouped : {false, true}) for (bool stage : {false, true}) {
            const int bcap = capT >= 1024 ? 128 : 64;
            const WarpLayout L = make_layout(dtype, d, P, n, PA, capT, kmax, bcap, b, R, stage, grouped);
            const uint32_t s = dtype == ANN_U8 ? 1 : 4, wb = 32u * b, cn = wb > 32 ? wb : 32;
            checked++;
            const uint32_t offs[] = {L.q, L.tabD, L.rank, L.sc, L.heap, L.hash, L.rbuf, L.bkey, L.bidx, L.cand,
                                     L.ckey, L.pref, L.nodes, L.glist, L.wref, L.wkey, L.stage, L.misc, L.total};
            for (uint32_t o : offs) CHECK(o % 16 == 0);
            CHECK(L.q + d * s <= L.tabD);
            CHECK(L.tabD + 4u * P * n <= L.rank);
            CHECK(L.rank + (uint32_t)P * n <= L.sc);
            CHECK(L.sc + (uint32_t)PA * n <= L.heap);
            CHECK(L.heap_cap >= (uint32_t)capT && L.heap + 8u * L.heap_cap <= L.hash);
            CHECK((1u << L.hash_log) >= 2u * capT && L.hash + 4u * (1u << L.hash_log) <= L.rbuf);
            CHECK(L.rbuf + 8u * kmax <= L.bkey);
            CHECK(L.bkey + 8u * bcap <= L.bidx && L.bidx + 4u * bcap <= L.cand);
            CHECK(L.cand + 4u * cn <= L.ckey && L.ckey + 4u * cn <= L.pref);
            // the shared region [pref, misc) and its users
            CHECK(L.pref + 4u * (n + 1) <= L.nodes);
            CHECK(L.nodes + 16u * L.ncap <= L.glist && L.glist + 20u * L.gcap <= L.misc);
            CHECK(L.nodes + 1024u <= L.misc);  // 256 radix counters of the windowed refill
            CHECK(L.wref + 4u * wb <= L.wkey && L.wkey + 4u * wb <= L.misc);
            CHECK(L.stage + L.stage_rows * L.stage_stride <= L.misc);
            CHECK(!stage || L.stage_rows == 0 || (L.stage_rows == (uint32_t)R && L.stage_stride >= d * s));
            CHECK(L.ncap >= 32 && (!grouped || L.gcap >= 32));
            CHECK(L.misc + 64 <= L.total);
            CHECK(L.total <= 227u * 1024u);  // one query per CTA always fits
        }
    }
    printf("%ld layouts, %ld violations\n", checked, bad);
    return bad != 0;
}
'''


def test_search_layout_over_the_parameter_grid(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "layout.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "layout"
    cmd = [nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
           "-I" + os.path.join(ROOT, "include"), "-I" + os.path.join(ROOT, "paper_1312_3062_gb300", "csrc"),
           str(src), "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout[-3000:]
    assert " 0 violations" in out.stdout
