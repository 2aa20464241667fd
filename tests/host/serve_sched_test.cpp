// Host tests of the request server's arena allocator and step planner
// (paper_2403_06777_gb300/csrc/serve_sched.h).  Prints "ok" and exits 0.
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <map>
#include <random>
#include <vector>

#include "serve_sched.h"

using namespace zxp;

#define CHECK(c)                                                          \
    do {                                                                  \
        if (!(c)) {                                                       \
            fprintf(stderr, "%s:%d: check failed: %s\n", __FILE__, __LINE__, #c); \
            exit(1);                                                      \
        }                                                                 \
    } while (0)

// Arena against a byte-map model: live blocks never overlap, stay inside
// the capacity and aligned, and freeing everything restores one free block.
static void test_arena_random() {
    std::mt19937_64 rng(7);
    for (int round = 0; round < 20; round++) {
        const uint64_t align = 1ull << (rng() % 10);
        const uint64_t cap = align * (1 + rng() % 4000);
        Arena a(cap, align);
        CHECK(a.capacity() == cap);
        std::map<uint64_t, uint64_t> live;   // off -> requested bytes
        for (int op = 0; op < 4000; op++) {
            if (live.empty() || rng() % 3) {
                const uint64_t want = 1 + rng() % (cap / 8 + 1);
                uint64_t off = ~0ull;
                const bool ok = a.alloc(want, &off);
                if (ok) {
                    CHECK(off % align == 0);
                    CHECK(off + want <= cap);
                    auto nx = live.lower_bound(off);
                    if (nx != live.end()) CHECK(off + want <= nx->first);
                    if (nx != live.begin()) {
                        auto pv = std::prev(nx);
                        CHECK(pv->first + pv->second <= off);
                    }
                    live[off] = want;
                } else {
                    // first fit fails only if no free block is large enough
                    CHECK(a.largest_free() < (want + align - 1) / align * align);
                }
            } else {
                auto it = live.begin();
                std::advance(it, rng() % live.size());
                CHECK(a.release(it->first));
                if (!live.count(it->first + 1)) CHECK(!a.release(it->first + 1));   // not a block
                live.erase(it);
            }
            CHECK(a.live_blocks() == live.size());
            CHECK(a.used() <= cap && a.peak() <= cap);
        }
        for (auto& b : live) CHECK(a.release(b.first));
        CHECK(a.used() == 0 && a.free_blocks() == 1 && a.largest_free() == cap);
    }
}

static void test_arena_edges() {
    Arena a(4096, 512);
    uint64_t o0, o1, o2, o3;
    CHECK(a.alloc(1, &o0) && o0 == 0);
    CHECK(a.alloc(512, &o1) && o1 == 512);
    CHECK(a.alloc(513, &o2) && o2 == 1024);
    CHECK(!a.alloc(4096, &o3));
    CHECK(a.fits_at_all(4096) && !a.fits_at_all(4097));
    CHECK(a.release(o1));
    CHECK(!a.release(o1));                 // double free refused
    CHECK(a.alloc(300, &o3) && o3 == 512); // first fit reuses the hole
    CHECK(a.release(o0) && a.release(o3) && a.release(o2));
    CHECK(a.free_blocks() == 1 && a.used() == 0 && a.peak() == 2048);
    Arena z(100, 512);                     // capacity below one block
    CHECK(z.capacity() == 0 && !z.alloc(1, &o0) && !z.fits_at_all(1));
}

// Plan steps until every item is done: every term is planned exactly once,
// chunk starts are multiples of 8, chunks are at most 2^clog, a step stays
// within its budget (a single whole small item may overrun it), and small
// items are taken whole, fewest terms first.
static void run_plan(std::vector<WorkItem> items, uint64_t budget, uint32_t clog, uint64_t small,
                     uint64_t seed) {
    std::mt19937_64 rng(seed);
    std::vector<std::vector<char>> seen(items.size());
    for (size_t i = 0; i < items.size(); i++) seen[i].assign(items[i].total, 0);
    std::vector<PlannedChunk> out;
    int steps = 0;
    for (;;) {
        std::vector<uint64_t> before;
        for (auto& w : items) before.push_back(w.next);
        bool work = false;
        for (auto& w : items) work |= w.next < w.total;
        plan_step(items, budget, clog, small, &out);
        if (!work) { CHECK(out.empty()); break; }
        CHECK(!out.empty());
        steps++;
        CHECK(steps < 1000000);
        uint64_t used = 0, small_whole = 0;
        size_t small_items = 0;
        std::map<size_t, uint64_t> per_item;
        for (auto& c : out) {
            CHECK(c.item < items.size());
            CHECK(c.count >= 1 && c.count <= (1ull << clog));
            CHECK(c.first % 8 == 0);
            for (uint64_t t = c.first; t < c.first + c.count; t++) {
                CHECK(t < items[c.item].total);
                CHECK(!seen[c.item][t]);
                seen[c.item][t] = 1;
            }
            used += c.count;
            per_item[c.item] += c.count;
        }
        for (auto& p : per_item) {
            const uint64_t left = items[p.first].total - before[p.first];
            CHECK(items[p.first].next == before[p.first] + p.second);
            if (left <= small) {
                CHECK(p.second == left);   // small items run whole
                small_whole = std::max(small_whole, left);
                small_items++;
            } else if (p.second < left) {
                CHECK(p.second % 8 == 0);  // an unfinished share keeps starts aligned
            }
        }
        CHECK(used <= std::max<uint64_t>(budget, 8) + small_whole);
        // a small item left out has at least as many terms as every small item taken
        for (size_t i = 0; i < items.size(); i++) {
            const uint64_t left = items[i].total - before[i];
            if (!left || left > small || per_item.count(i)) continue;
            for (auto& p : per_item) {
                const uint64_t lp = items[p.first].total - before[p.first];
                if (lp <= small) CHECK(lp <= left);
            }
        }
        (void)rng;
    }
    for (size_t i = 0; i < items.size(); i++) {
        CHECK(items[i].next == items[i].total);
        for (char c : seen[i]) CHECK(c);
    }
}

static void test_plan_random() {
    std::mt19937_64 rng(11);
    for (int round = 0; round < 60; round++) {
        std::vector<WorkItem> items(1 + rng() % 12);
        for (size_t i = 0; i < items.size(); i++) {
            items[i].total = 1ull << (rng() % 15);
            items[i].order = rng() % 5;
        }
        const uint64_t budget = 8 + rng() % 3000;
        const uint32_t clog = 3 + rng() % 8;
        const uint64_t small = rng() % 600;
        run_plan(items, budget, clog, small, rng());
    }
}

// A large item keeps progressing while small ones keep arriving, and small
// items that fit the budget finish in the step that first sees them.
static void test_plan_progress() {
    std::vector<WorkItem> items(1);
    items[0].total = 1ull << 21;
    items[0].order = 0;
    std::vector<PlannedChunk> out;
    uint64_t order = 1;
    for (int step = 0; step < 64; step++) {
        for (int j = 0; j < 3; j++) {
            WorkItem w;
            w.total = 1ull << (step % 10);
            w.order = order++;
            items.push_back(w);
        }
        const uint64_t large_before = items[0].next;
        plan_step(items, 1 << 16, 12, 1 << 12, &out);
        const uint64_t left = items[0].total - large_before;
        CHECK(items[0].next - large_before >= std::min<uint64_t>(left, (1 << 16) / 4));   // its quarter
        for (size_t i = 1; i < items.size(); i++) CHECK(items[i].next == items[i].total);
        std::vector<WorkItem> keep(1, items[0]);
        items.swap(keep);
    }
    CHECK(items[0].next == items[0].total);   // 64 steps of nearly the whole budget
    // with the budget at 8 the planner still makes progress one chunk at a time
    std::vector<WorkItem> one(1);
    one[0].total = 100;
    run_plan(one, 8, 3, 0, 3);
}

int main() {
    test_arena_edges();
    test_arena_random();
    test_plan_random();
    test_plan_progress();
    printf("ok\n");
    return 0;
}
