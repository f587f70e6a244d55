"""The serving worker's device-memory arena (host code, csrc/fw_arena.h),
compiled with the host C++ compiler and driven directly: fixed cases for
each placement rule and a seeded fuzz of mixed requests that checks no two
live ranges overlap, the used count, and full coalescing once all is freed."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_2512_00705_gb300", "csrc", "fw_arena.h")

HARNESS = r"""
#include <cstdio>
#include <random>
#include <utility>
#include <vector>
#include "fw_arena.h"
using fw::Arena;
#define CHECK(c) do { if (!(c)) { std::printf("FAIL line %d: %s\n", __LINE__, #c); return 1; } } while (0)

int main() {
  {  // first fit from the bottom, last fit from the top, coalescing
    Arena a(1000);
    size_t r1, r2, t1;
    CHECK(a.alloc(100, &r1) && r1 == 0);
    CHECK(a.alloc(200, &r2) && r2 == 100);
    CHECK(a.alloc_top(50, &t1) && t1 == 950);
    CHECK(a.used() == 350);
    a.release(r1, 100);
    size_t r3;
    CHECK(a.alloc(80, &r3) && r3 == 0);     // the hole at the bottom
    CHECK(a.alloc(30, &r3) && r3 == 300);   // 20 bytes left below 100 do not fit
    a.release(0, 80);
    a.release(100, 200);
    a.release(300, 30);
    a.release(950, 50);
    CHECK(a.used() == 0);
    size_t all;
    CHECK(a.alloc(1000, &all) && all == 0);  // everything coalesced into one range
  }
  {  // next fit: alloc_at succeeds exactly where a free range holds the request
    Arena a(1000);
    size_t r;
    CHECK(a.alloc_at(0, 100));
    CHECK(a.alloc_at(100, 100));             // right after the previous one
    CHECK(!a.alloc_at(150, 10));             // inside a taken range
    CHECK(!a.alloc_at(950, 100));            // runs past the end
    CHECK(a.alloc_at(500, 100));             // splits a free range in two
    CHECK(a.alloc(300, &r) && r == 200);     // the lower part of the split
    CHECK(a.used() == 600);
    CHECK(!a.alloc(401, &r));
    CHECK(a.alloc(400, &r) && r == 600);
  }
  {  // zero-byte requests take nothing
    Arena a(64);
    size_t r = 7;
    CHECK(a.alloc(0, &r) && a.used() == 0);
    CHECK(a.alloc_top(0, &r) && a.used() == 0);
    CHECK(a.alloc_at(5, 0) && a.used() == 0);
    a.release(r, 0);
    CHECK(a.alloc(64, &r) && r == 0);
  }
  // fuzz: rows next-fit from a cursor, starts from the top, random releases
  std::mt19937_64 rng(12345);
  for (int trial = 0; trial < 300; ++trial) {
    const size_t size = 4096 + (rng() % 200000) * 4;
    Arena a(size);
    std::vector<std::pair<size_t, size_t>> live;
    size_t cursor = 0, used = 0;
    for (int op = 0; op < 3000; ++op) {
      if (live.empty() || rng() % 3) {
        const size_t b = (rng() % (size / 16 + 1)) * 4;
        size_t off = 0;
        bool ok;
        if (rng() % 2) {
          off = cursor;
          ok = a.alloc_at(off, b) || a.alloc(b, &off);
        } else {
          ok = a.alloc_top(b, &off);
        }
        if (!ok || b == 0) continue;
        CHECK(off + b <= size);
        for (auto& x : live) CHECK(off + b <= x.first || x.first + x.second <= off);
        live.push_back({off, b});
        used += b;
        cursor = off + b;
      } else {
        const size_t i = rng() % live.size();
        a.release(live[i].first, live[i].second);
        used -= live[i].second;
        live.erase(live.begin() + (long)i);
      }
      CHECK(a.used() == used);
    }
    for (auto& x : live) a.release(x.first, x.second);
    size_t off = 1;
    CHECK(a.used() == 0 && a.alloc(size, &off) && off == 0);
  }
  std::printf("ok\n");
  return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("arena")
    src = d / "arena_test.cpp"
    src.write_text(HARNESS)
    exe = d / "arena_test"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    return str(exe)


def test_arena_placement_rules_and_fuzz(harness):
    r = subprocess.run([harness], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
