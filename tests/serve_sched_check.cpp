// Host-only checks of the serving loop's bookkeeping (serve_sched.h): the
// arena allocator and the scheduler's admission, packing and release rules.
// Built with g++ by tests/test_serve_sched.py; prints "PASS <name>" per check
// and exits non-zero on the first failure.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <set>
#include <vector>

#include "serve_sched.h"

using namespace lya::serve;

#define CHECK(cond)                                                              \
    do {                                                                         \
        if (!(cond)) {                                                           \
            std::printf("FAIL %s:%d %s\n", __FILE__, __LINE__, #cond);          \
            std::exit(1);                                                        \
        }                                                                        \
    } while (0)

static Request req(uint64_t t, int64_t rows, int n_pix, int shift = 0, double row_cost = 1.0)
{
    Request r;
    r.ticket = t;
    r.n_rows = rows;
    r.n_pix = n_pix;
    r.shift = shift;
    r.row_cost = row_cost;
    r.task_key = row_cost * (1 << shift);
    return r;
}

static void arena_random()
{
    std::mt19937_64 rng(7);
    Arena a(1 << 24, 256);
    std::vector<size_t> live;
    for (int it = 0; it < 20000; ++it) {
        if (live.empty() || rng() % 3 != 0) {
            const size_t bytes = 1 + rng() % 200000;
            const size_t off = a.alloc(bytes);
            if (off != kNoOffset) {
                CHECK(off % 256 == 0);
                CHECK(off + bytes <= a.capacity());
                live.push_back(off);
            }
        } else {
            const size_t k = rng() % live.size();
            CHECK(a.release(live[k]));
            live.erase(live.begin() + (long)k);
        }
        if (it % 97 == 0) CHECK(a.consistent());
    }
    CHECK(!a.release(12345));                // not a block
    for (size_t off : live) CHECK(a.release(off));
    CHECK(a.consistent());
    CHECK(a.used() == 0);
    CHECK(a.largest_free() == a.capacity());  // everything merged back
    std::printf("PASS arena_random\n");
}

static void budget_and_fifo()
{
    Limits L;
    L.budget = 1 << 20;                      // 1 MiB
    L.max_slots = 4;
    Scheduler s(L);
    CHECK(!s.enqueue(req(1, 1024, 1024)));  // 8 MiB: never fits
    CHECK(s.enqueue(req(2, 64, 1024)));     // 512 KiB
    CHECK(s.enqueue(req(3, 96, 1024)));     // 768 KiB: waits for 2
    CHECK(s.enqueue(req(4, 8, 1024)));      // small, but behind 3 (arrival order)
    auto a = s.admit();
    CHECK(a.size() == 1 && a[0] == 2);
    CHECK(s.queued() == 2);
    // run 2 to the end of its root-find, release it: 3 and then 4 fit
    StepPlan p = s.plan();
    CHECK(p.items.size() == 64 && p.rf.size() == 1 && p.rf[0].init == 1);
    s.finish(2);
    CHECK(s.arena().used() == 256 * 1024);  // F of 2 still held
    a = s.admit();
    CHECK(a.empty());                        // 3 needs 768 KiB, only 768 KiB free but F holds 256
    CHECK(s.release(2));
    a = s.admit();
    CHECK(a.size() == 2 && a[0] == 3 && a[1] == 4);   // then 4 fits beside 3
    CHECK(!s.release(3));                    // not finished
    std::printf("PASS budget_and_fifo\n");
}

static void slots()
{
    Limits L;
    L.budget = 1 << 26;
    L.max_slots = 2;
    Scheduler s(L);
    for (uint64_t t = 1; t <= 5; ++t) CHECK(s.enqueue(req(t, 4, 512)));
    auto a = s.admit();
    CHECK(a.size() == 2);
    s.plan();
    s.finish(a[0]);
    a = s.admit();
    CHECK(a.size() == 1 && a[0] == 3);
    std::printf("PASS slots\n");
}

// A long request is spread over steps by the quota; one that arrives later
// gets its skewers in the next step and finishes while the long one runs.
static void quota_interleave()
{
    Limits L;
    L.budget = (size_t)1 << 34;
    L.max_slots = 8;
    L.step_quota_ns = 1000.0;
    Scheduler s(L);
    CHECK(s.enqueue(req(1, 4096, 8192, 0, 10.0)));   // 40,960 ns of work: ~41 steps
    s.admit();
    StepPlan p1 = s.plan();
    CHECK(p1.items.size() == 100);
    CHECK(p1.rf.empty());
    CHECK(s.enqueue(req(2, 5, 512, 2, 1.0)));
    s.admit();
    StepPlan p2 = s.plan();
    int rows2 = 0;
    for (const auto& it : p2.items) rows2 += it.slot == s.find(2)->slot;
    CHECK(rows2 == 5);                                 // all of the short one
    CHECK(p2.rf.size() == 1 && p2.rf[0].slot == s.find(2)->slot);
    // tasks of the short request come in groups of 4 (shift 2): 4 + 1
    int t4 = 0, t1 = 0;
    for (const auto& t : p2.tasks)
        if (t.slot == s.find(2)->slot) (t.n_items == 4 ? t4 : t1) += 1;
    CHECK(t4 == 1 && t1 == 1);
    // every row of the long one is planned exactly once, in order
    std::vector<int> seen(4096, 0);
    for (const auto& it : p1.items) seen[it.row]++;
    for (const auto& it : p2.items)
        if (it.slot == s.find(1)->slot) seen[it.row]++;
    int64_t planned = s.find(1)->rows_planned;
    for (int k = 0; k < 4096; ++k) CHECK(seen[k] == (k < planned ? 1 : 0));
    std::printf("PASS quota_interleave\n");
}

static void units_cover()
{
    Limits L;
    L.budget = (size_t)1 << 34;
    L.max_slots = 8;
    L.max_units = 64;
    L.unit_pix = 1000;                 // rounded up to a multiple of 4
    L.max_units_per_request = 40;
    Scheduler s(L);
    CHECK(s.enqueue(req(1, 7, 1234)));        // 8,638 px -> 9 units of 1,000
    CHECK(s.enqueue(req(2, 100, 4000)));      // 400,000 px -> 40 units of 10,000
    CHECK(s.enqueue(req(3, 100, 4000)));      // deferred: would exceed 64 units
    s.admit();
    StepPlan p = s.plan();
    CHECK(p.rf.size() == 2);
    CHECK((int64_t)p.units.size() <= L.max_units);
    for (size_t r = 0; r < p.rf.size(); ++r) {
        const auto& f = p.rf[r];
        const Request* q = s.find(s.ticket_of_slot(f.slot));
        int64_t pos = 0;
        for (int u = f.unit_first; u < f.unit_first + f.unit_count; ++u) {
            CHECK(p.units[u].rf == (int)r);
            CHECK(p.units[u].begin == pos && p.units[u].begin % 4 == 0);
            CHECK(p.units[u].end > p.units[u].begin);
            pos = p.units[u].end;
        }
        CHECK(pos == q->pixels());
        CHECK(f.init == 1);
    }
    StepPlan p2 = s.plan();                    // 1 and 2 go on first; 3 still does not fit
    int inits = 0, conts = 0;
    for (const auto& f : p2.rf) (f.init ? inits : conts) += 1;
    CHECK(inits == 0 && conts == 2);
    s.finish(1);
    s.finish(2);
    StepPlan p3 = s.plan();                    // now the deferred one starts
    CHECK(p3.rf.size() == 1 && p3.rf[0].init == 1 && p3.rf[0].unit_count == 40);
    std::printf("PASS units_cover\n");
}

// Random arrivals through admit/plan/finish/release: memory stays within the
// budget, every row is planned once, every request ends, and everything is
// freed at the end.
static void random_loop()
{
    std::mt19937_64 rng(11);
    Limits L;
    L.budget = 64ull << 20;
    L.max_slots = 16;
    L.step_quota_ns = 5000.0;
    L.max_items = 512;
    L.max_units = 256;
    Scheduler s(L);
    std::vector<std::vector<int>> seen(1);
    std::set<uint64_t> open, finished;
    std::vector<int> rf_steps(1, 0);
    uint64_t next = 1;
    for (int step = 0; step < 4000; ++step) {
        if (next <= 600 && rng() % 2 == 0) {
            const int npix = 512 << (rng() % 5);
            const int64_t rows = 1 + (int64_t)(rng() % 300);
            Request r = req(next, rows, npix, (int)(rng() % 4), 1.0 + (rng() % 100));
            if (s.enqueue(r)) {
                open.insert(next);
                seen.push_back(std::vector<int>((size_t)rows, 0));
            } else {
                seen.push_back({});
            }
            rf_steps.push_back(0);
            ++next;
        }
        s.admit();
        StepPlan p = s.plan();
        CHECK(s.arena().used() <= L.budget);
        CHECK((int64_t)p.items.size() <= L.max_items);
        for (const auto& it : p.items) {
            const uint64_t t = s.ticket_of_slot(it.slot);
            CHECK(t != 0);
            seen[t][(size_t)it.row]++;
        }
        for (const auto& f : p.rf) {
            const uint64_t t = s.ticket_of_slot(f.slot);
            // a request's root-find takes one to three steps
            if (++rf_steps[t] >= 1 + (int)(t % 3)) {
                s.finish(t);
                finished.insert(t);
            }
        }
        for (auto it = finished.begin(); it != finished.end();) {
            if (rng() % 4 == 0) {
                CHECK(s.release(*it));
                open.erase(*it);
                it = finished.erase(it);
            } else {
                ++it;
            }
        }
        CHECK(s.arena().consistent());
    }
    for (uint64_t t : finished) {
        CHECK(s.release(t));
        open.erase(t);
    }
    CHECK(open.empty());
    for (size_t t = 1; t < seen.size(); ++t)
        for (int c : seen[t]) CHECK(c == 1);
    CHECK(s.arena().used() == 0);
    std::printf("PASS random_loop\n");
}

int main()
{
    arena_random();
    budget_and_fifo();
    slots();
    quota_interleave();
    units_cover();
    random_loop();
    return 0;
}
