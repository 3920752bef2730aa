"""Host-only policy of the lattice server (csrc/serve_sched.h), compiled with g++ and driven by
seeded scenarios: first-fit arena invariants, admission caps and order for both policies, the
chunk cut, and a random job stream run to completion."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2408_15654_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>
#include <set>
#include "serve_sched.h"
using namespace lbm_serve;

#define CHECK(c) do { if (!(c)) { std::printf("FAIL line %d: %s\n", __LINE__, #c); std::exit(1); } } while (0)

// every used block inside the arena, no two blocks overlap, free blocks never adjacent, the
// lengths add up to the arena size
static void arena_invariants(const Arena& a) {
    std::map<size_t, std::pair<size_t, int>> all;
    for (auto& kv : a.used_list()) all[kv.first] = {kv.second, 1};
    for (auto& kv : a.free_list()) { CHECK(!all.count(kv.first)); all[kv.first] = {kv.second, 0}; }
    size_t pos = 0; int prev_free = 0;
    for (auto& kv : all) {
        CHECK(kv.first == pos);
        CHECK(kv.second.first > 0 && kv.second.first % 256 == 0);
        if (!kv.second.second) { CHECK(!prev_free); }
        prev_free = !kv.second.second;
        pos += kv.second.first;
    }
    CHECK(pos == a.size());
}

static void arena_random() {
    std::mt19937_64 rng(7);
    Arena a(1 << 24);
    std::vector<int64_t> live;
    for (int it = 0; it < 20000; ++it) {
        if (live.empty() || rng() % 3 != 0) {
            const size_t bytes = 1 + rng() % (1 << 18);
            // expected first fit: the lowest free block that can hold the rounded size
            const size_t need = (bytes + 255) / 256 * 256;
            int64_t expect = -1;
            for (auto& kv : a.free_list()) if (kv.second >= need) { expect = (int64_t)kv.first; break; }
            const int64_t off = a.alloc(bytes);
            CHECK(off == expect);
            if (off >= 0) live.push_back(off);
        } else {
            const size_t k = rng() % live.size();
            CHECK(a.release(live[k]));
            CHECK(!a.release(live[k]));  // double free is refused
            live.erase(live.begin() + k);
        }
        if (it % 97 == 0) arena_invariants(a);
    }
    for (int64_t off : live) CHECK(a.release(off));
    arena_invariants(a);
    CHECK(a.used_bytes() == 0 && a.free_blocks() == 1 && a.largest_free() == a.size());
    std::printf("arena ok\n");
}

static JobSpec job(int64_t id, int64_t cells, int64_t steps, size_t bytes = 1024) {
    return JobSpec{id, cells, (cells + 255) / 256, steps, bytes};
}

static void fcfs_order() {
    Scheduler s(kFCFS, 3, 1000, 1 << 20, 1 << 20);
    CHECK(s.submit(job(1, 400, 50)));
    CHECK(s.submit(job(2, 500, 10)));
    CHECK(s.submit(job(3, 300, 30)));   // does not fit beside 1 and 2 (1200 > 1000): blocks 4
    CHECK(s.submit(job(4, 50, 5)));
    auto a = s.admit();
    CHECK(a.size() == 2 && a[0].id == 1 && a[1].id == 2);
    CHECK(s.active_cells() == 900 && s.queued() == 2);
    CHECK(s.next_chunk(100) == 10);     // cut at job 2's end
    auto f = s.advance(10);
    CHECK(f.size() == 1 && f[0] == 2);
    a = s.admit();                      // 3 (300) and then 4 (50): 750 <= 1000, 3 jobs
    CHECK(a.size() == 2 && a[0].id == 3 && a[1].id == 4);
    CHECK(s.next_chunk(100) == 5);
    f = s.advance(5);
    CHECK(f.size() == 1 && f[0] == 4);
    CHECK(s.steps_done(1) == 15 && s.steps_done(3) == 5);
    CHECK(!s.submit(job(9, 10, 0)));          // no steps
    CHECK(!s.submit(job(9, 10, 5, 2 << 20)));  // larger than the arena
    // a job larger than max_cells runs alone once the server is idle
    Scheduler t(kFCFS, 4, 100, 1 << 20, 1 << 20);
    CHECK(t.submit(job(1, 50, 10)));
    CHECK(t.submit(job(2, 500, 10)));
    a = t.admit();
    CHECK(a.size() == 1 && a[0].id == 1);
    t.advance(10);
    a = t.admit();
    CHECK(a.size() == 1 && a[0].id == 2 && t.active_cells() == 500);
    std::printf("fcfs ok\n");
}

static void shortest_first_order() {
    Scheduler s(kShortestFirst, 2, 1 << 30, 1 << 20, 1 << 20);
    CHECK(s.submit(job(1, 100, 1000)));  // work 1e5
    CHECK(s.submit(job(2, 10, 100)));    // 1e3
    CHECK(s.submit(job(3, 50, 100)));    // 5e3
    auto a = s.admit();
    CHECK(a.size() == 2 && a[0].id == 2 && a[1].id == 3);
    s.advance(100);
    a = s.admit();
    CHECK(a.size() == 1 && a[0].id == 1);
    // jobs that do not fit are skipped, not blocking
    Scheduler t(kShortestFirst, 4, 100, 1 << 20, 1 << 20);
    CHECK(t.submit(job(1, 80, 10)));
    a = t.admit();
    CHECK(a.size() == 1);
    CHECK(t.submit(job(2, 50, 1)));      // smallest work but does not fit beside job 1
    CHECK(t.submit(job(3, 20, 100)));
    a = t.admit();
    CHECK(a.size() == 1 && a[0].id == 3);
    std::printf("sjf ok\n");
}

static void random_stream(Policy pol) {
    std::mt19937_64 rng(pol == kFCFS ? 11 : 12);
    const int64_t max_cells = 5000, max_tiles = 40;
    Scheduler s(pol, 6, max_cells, max_tiles, 1 << 22);
    std::map<int64_t, int64_t> want, got;
    int64_t next = 1, chunk = 37;
    for (int round = 0; round < 4000; ++round) {
        if (next <= 300 && rng() % 2 == 0) {
            const int64_t cells = 1 + rng() % 3000, steps = 1 + rng() % 500;
            const size_t bytes = 256 + rng() % (1 << 20);
            CHECK(s.submit(JobSpec{next, cells, (cells + 255) / 256, steps, bytes}));
            want[next] = steps;
            next++;
        }
        s.admit();
        CHECK((int)s.active_count() <= 6);
        CHECK(s.active_count() <= 1 || (s.active_cells() <= max_cells && s.active_tiles() <= max_tiles));
        const int64_t n = s.next_chunk(chunk);
        if (s.idle()) { CHECK(n == 0); continue; }
        CHECK(n >= 1 && n <= chunk);
        for (int64_t id : s.active_ids()) { CHECK(s.steps_done(id) + n <= want[id]); got[id] += n; }
        for (int64_t id : s.advance(n)) CHECK(got[id] == want[id]);
    }
    while (!s.idle() || s.queued()) {
        s.admit();
        const int64_t n = s.next_chunk(chunk);
        for (int64_t id : s.active_ids()) got[id] += n;
        s.advance(n);
    }
    CHECK(got == want);
    CHECK(s.arena().used_bytes() == 0 && s.arena().free_blocks() == 1);
    std::printf("stream %d ok %zu jobs\n", (int)pol, want.size());
}

int main(int argc, char** argv) {
    const char* w = argc > 1 ? argv[1] : "";
    if (!std::strcmp(w, "arena")) arena_random();
    else if (!std::strcmp(w, "fcfs")) fcfs_order();
    else if (!std::strcmp(w, "sjf")) shortest_first_order();
    else if (!std::strcmp(w, "stream")) { random_stream(kFCFS); random_stream(kShortestFirst); }
    else return 2;
    return 0;
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    d = tmp_path_factory.mktemp("sched")
    src = d / "driver.cpp"
    src.write_text(DRIVER)
    exe = d / "driver"
    subprocess.run(["g++", "-std=c++17", "-O1", "-Wall", "-I", CSRC, "-o", str(exe), str(src)], check=True)
    return str(exe)


@pytest.mark.parametrize("scenario", ["arena", "fcfs", "sjf", "stream"])
def test_serving_policy(driver, scenario):
    r = subprocess.run([driver, scenario], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "ok" in r.stdout
