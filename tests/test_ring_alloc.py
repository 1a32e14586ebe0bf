"""The serving loop's arena allocator (csrc/lg_ring.h, host C++): contiguous
ranges of a circular buffer, allocated in admission order and released in the
same order.  A random sequence of allocations, rollbacks and releases, checked
against a brute-force occupancy map: every live range lies inside the buffer,
no two overlap, a request that fits in the free space at the end or at the
start is placed, and releasing everything empties the ring."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROG = r"""
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "lg_ring.h"
using lg::RingAlloc;
static unsigned long long st = 88172645463325252ull;
static unsigned rnd() { st ^= st << 13; st ^= st >> 7; st ^= st << 17; return (unsigned)st; }
int main() {
    for (int trial = 0; trial < 200; ++trial) {
        const size_t cap = 1 + rnd() % 200;
        RingAlloc ra;
        ra.reset(cap);
        std::vector<std::pair<size_t, size_t>> live;  // (start, n) as handed out, in order
        for (int step = 0; step < 2000; ++step) {
            const unsigned op = rnd() % 10;
            if (op < 6) {
                const size_t n = rnd() % (cap / 2 + 2);
                const RingAlloc::Mark m = ra.mark();
                size_t at = 0;
                std::vector<char> occ(cap, 0);
                for (auto &p : live)
                    for (size_t i = 0; i < p.second; ++i) occ[p.first + i] = 1;
                if (ra.alloc(n, &at)) {
                    if (at + n > cap) { printf("out of range %zu+%zu > %zu\n", at, n, cap); return 1; }
                    for (size_t i = 0; i < n; ++i)
                        if (occ[at + i]) { printf("overlap at %zu\n", at + i); return 1; }
                    if (rnd() % 4 == 0) { ra.rollback(m); continue; }
                    live.emplace_back(at, n);
                } else {
                    // refused: then neither the space after the last range nor
                    // (when wrapping) the space before the first holds n
                    if (live.empty() && n <= cap) { printf("refused on an empty ring\n"); return 1; }
                    if (!live.empty()) {
                        const size_t b = live.front().first, e = live.back().first + live.back().second;
                        const bool wrapped = e <= b && !(e == b && ra.used == 0);
                        if (wrapped ? (b - e >= n) : (cap - e >= n || (n <= b))) {
                            printf("refused %zu with room (b=%zu e=%zu cap=%zu)\n", n, b, e, cap);
                            return 1;
                        }
                    }
                }
            } else if (!live.empty()) {
                ra.release_front();
                live.erase(live.begin());
            }
        }
        while (!live.empty()) { ra.release_front(); live.erase(live.begin()); }
        if (ra.used != 0 || !ra.live.empty()) { printf("not empty after releasing all\n"); return 1; }
    }
    printf("ok\n");
    return 0;
}
"""


def test_ring_allocator_against_an_occupancy_map(tmp_path):
    src = tmp_path / "ring.cc"
    src.write_text(PROG)
    exe = tmp_path / "ring"
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_2110_11644_gb300", "csrc"),
                           str(src), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
