"""The streaming service's device-memory arena (csrc/arena.h, host C++)
compiled with g++ and driven by random allocation and release sequences
against a reference model of 256-byte units: every offset is 256-aligned,
live blocks never overlap and stay inside the budget, the used count is
exact, a request fails only when no free run is long enough, the block
chosen is the first free run that fits (so freed neighbours must have been
merged), and releasing everything leaves the whole budget free."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

DRIVER = r"""
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>
#include "arena.h"

using mmf::Arena;

int main() {
    std::mt19937_64 rng(12345);
    for (int trial = 0; trial < 200; ++trial) {
        const size_t units = 1 + rng() % 300;            // budget in 256-byte units
        const size_t size = units * 256 - (rng() % 2 ? 0 : rng() % 200);  // sometimes not a multiple
        Arena a;
        a.init(size);
        const size_t cap = size / 256;                   // whole units usable at most
        std::vector<char> taken(units + 1, 0);           // model: unit in use
        struct Blk { int64_t off; size_t bytes; };
        std::vector<Blk> live;
        for (int step = 0; step < 2000; ++step) {
            if (live.empty() || rng() % 3) {
                const size_t bytes = rng() % 4 == 0 ? 0 : 1 + rng() % (256 * 12);
                const size_t need = Arena::round(bytes) / 256;
                // model's first fit over maximal free runs of whole units
                int64_t want = -1;
                for (size_t u = 0, run = 0; u < cap; ++u) {
                    run = taken[u] ? 0 : run + 1;
                    if (run == need) { want = (int64_t)(u + 1 - need) * 256; break; }
                }
                const int64_t off = a.alloc(bytes);
                if (off != want) { printf("trial %d step %d: got %lld want %lld\n", trial, step,
                                          (long long)off, (long long)want); return 1; }
                if (off >= 0) {
                    if (off % 256) return 2;
                    for (size_t u = off / 256; u < off / 256 + need; ++u) {
                        if (u >= cap || taken[u]) return 3;
                        taken[u] = 1;
                    }
                    live.push_back({off, bytes});
                }
            } else {
                const size_t k = rng() % live.size();
                const Blk b = live[k];
                a.release(b.off, b.bytes);
                for (size_t u = b.off / 256; u < b.off / 256 + Arena::round(b.bytes) / 256; ++u) taken[u] = 0;
                live[k] = live.back();
                live.pop_back();
            }
            size_t used = 0;
            for (const Blk &b : live) used += Arena::round(b.bytes);
            if (a.used() != used) return 4;
        }
        for (const Blk &b : live) a.release(b.off, b.bytes);
        if (a.used() != 0) return 5;
        if (cap > 0 && a.alloc(cap * 256) != 0) return 6;  // one block again
    }
    printf("ok\n");
    return 0;
}
"""


def test_arena_against_unit_model(tmp_path):
    if shutil.which("g++") is None:
        pytest.skip("no C++ compiler")
    drv = tmp_path / "arena_drive.cpp"
    drv.write_text(DRIVER)
    exe = tmp_path / "arena_drive"
    inc = os.path.join(ROOT, "paper_cs_0610046_gb300", "csrc")
    subprocess.run(["g++", "-std=c++17", "-O1", "-g", "-fsanitize=address,undefined", "-I", inc, str(drv),
                    "-o", str(exe)], check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.strip() == "ok", (out.returncode, out.stdout, out.stderr[-2000:])
