// Host-only checks of the serving scheduler core (no CUDA): pool allocator,
// admission by footprint and slots, round-robin step building under a tile
// budget, completion and latency bookkeeping.  Prints "ok <name>" per check
// and exits non-zero on the first failure.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <set>

#include "fcfs_sched.h"

using fcfs::sched::Pool;
using fcfs::sched::Request;
using fcfs::sched::Scheduler;
using fcfs::sched::Step;

#define CHECK(c)                                                          \
    do {                                                                  \
        if (!(c)) {                                                       \
            std::printf("FAIL %s:%d %s\n", __FILE__, __LINE__, #c);       \
            std::exit(1);                                                 \
        }                                                                 \
    } while (0)

static Request req(uint64_t id, long long tiles, size_t bytes, double t = 0) {
    Request r;
    r.id = id;
    r.tiles = tiles;
    r.out_bytes = bytes;
    r.arrival = t;
    r.out_pixels = 1;
    return r;
}

static void pool_basics() {
    Pool p(4096);
    const size_t a = p.alloc(100), b = p.alloc(300), c = p.alloc(256);
    CHECK(a == 0 && b == 256 && c == 768);
    CHECK(p.used() == 256 + 512 + 256);
    p.release(b, 300);
    CHECK(p.alloc(600) == 1024);            // the 512-byte hole is too small
    CHECK(p.alloc(500) == 256);             // first fit reuses the hole
    p.release(a, 100);
    p.release(256, 500);
    p.release(c, 256);
    p.release(1024, 600);
    CHECK(p.used() == 0 && p.largest_free() == 4096);  // everything coalesced
    CHECK(p.alloc(5000) == SIZE_MAX);
    std::printf("ok pool_basics\n");
}

static void admission_by_footprint() {
    Scheduler S(1024, 8, 100);
    CHECK(S.submit(req(1, 4, 600)));
    CHECK(S.submit(req(2, 4, 600)));
    CHECK(!S.submit(req(3, 4, 2000)));     // can never fit: rejected
    auto a = S.admit(0.0);
    CHECK(a.size() == 1 && a[0]->id == 1);  // the second waits for memory
    CHECK(S.deferred() == 1);
    S.admit(0.0);
    CHECK(S.deferred() == 1);               // a deferral is counted once
    Step st = S.next_step();
    CHECK(st.tiles == 4);
    auto done = S.finish(st, 1.0, true);
    CHECK(done.size() == 1 && done[0].id == 1);
    a = S.admit(1.0);
    CHECK(a.size() == 1 && a[0]->id == 2);  // memory freed by completion
    std::printf("ok admission_by_footprint\n");
}

static void slots_limit_inflight() {
    Scheduler S(0, 2, 100);
    for (int i = 1; i <= 3; ++i) CHECK(S.submit(req(i, 2, 0)));
    CHECK(S.admit(0).size() == 2);
    CHECK(S.active() == 2 && S.queued() == 1);
    Step st = S.next_step();
    CHECK(st.tiles == 4);
    S.finish(st, 1, true);
    CHECK(S.admit(1).size() == 1 && S.max_inflight_seen() == 2);
    std::printf("ok slots_limit_inflight\n");
}

static void steps_round_robin_and_chunking() {
    Scheduler S(0, 8, 10);
    S.submit(req(1, 25, 0));
    S.submit(req(2, 3, 0));
    S.admit(0);
    Step a = S.next_step();
    CHECK(a.tiles == 10);
    long long t1 = 0, t2 = 0;
    for (auto& p : a.pieces) (p.id == 1 ? t1 : t2) += p.count;
    CHECK(t2 == 3 && t1 == 7);              // the small request is not starved
    S.submit(req(3, 7, 0));                 // arrives while step a is on the GPU
    S.admit(0.5);
    Step b = S.next_step();                 // and joins the next step
    bool has3 = false;
    for (auto& p : b.pieces) has3 |= p.id == 3;
    CHECK(has3 && b.tiles == 10);
    auto d = S.finish(a, 1.0, true);
    CHECK(d.size() == 1 && d[0].id == 2);   // request 2 finished in step a
    std::printf("ok steps_round_robin_and_chunking\n");
}

static void latency_and_percentiles() {
    Scheduler S(0, 4, 100);
    S.submit(req(1, 1, 0, 10.0));
    S.admit(10.0);
    auto d = S.finish(S.next_step(), 10.25, true);
    CHECK(d.size() == 1 && S.latencies().size() == 1 && S.latencies()[0] == 0.25);
    std::vector<double> v = {1, 2, 3, 4, 5, 6, 7, 8, 9, 10};
    CHECK(Scheduler::percentile(v, 50) == 5.5);
    CHECK(Scheduler::percentile(v, 100) == 10.0 && Scheduler::percentile(v, 0) == 1.0);
    std::printf("ok latency_and_percentiles\n");
}

static void randomized_invariants() {
    std::mt19937_64 rng(42);
    const size_t pool = 1 << 20;
    Scheduler S(pool, 16, 37);
    std::uniform_int_distribution<int> tiles(1, 60), bytes(1, 200000);
    std::map<uint64_t, long long> want;
    std::map<uint64_t, std::set<long long>> seen;
    uint64_t next = 1;
    int submitted = 0;
    std::vector<Step> inflight;
    double now = 0;
    while (submitted < 2000 || !S.idle()) {
        if (submitted < 2000 && rng() % 3 == 0) {
            Request r = req(next, tiles(rng), bytes(rng), now);
            want[next] = r.tiles;
            CHECK(S.submit(r));
            ++next;
            ++submitted;
        }
        S.admit(now);
        CHECK(S.pool().used() <= pool);
        if (inflight.size() < 2) {
            Step st = S.next_step();
            CHECK(st.tiles <= 37);
            for (auto& p : st.pieces)
                for (long long t = p.first; t < p.first + p.count; ++t) CHECK(seen[p.id].insert(t).second);
            if (st.tiles) inflight.push_back(st);
        }
        if (!inflight.empty() && rng() % 2 == 0) {
            S.finish(inflight.front(), now, true);
            inflight.erase(inflight.begin());
        }
        now += 1e-3;
    }
    CHECK(S.completed() == 2000);
    for (auto& kv : want) CHECK((long long)seen[kv.first].size() == kv.second);  // every tile exactly once
    CHECK(S.pool().used() == 0);
    std::printf("ok randomized_invariants\n");
}

// Cancellation (a client that abandons its requests): queued ones leave at once,
// admitted ones stop receiving tiles and finish when their launched tiles do,
// uncounted in the latency and throughput totals; slots and pool memory return.
static void cancel_requests() {
    Scheduler S(1 << 20, 2, 8);
    for (uint64_t id = 1; id <= 4; ++id) CHECK(S.submit(req(id, 10, 4096)));
    CHECK(S.admit(0.0).size() == 2);  // 1 and 2 admitted, 3 and 4 queued
    Request out;
    CHECK(S.cancel(3, true, &out) == 1 && out.id == 3 && out.canceled);
    CHECK(S.queued() == 1);
    CHECK(S.cancel(99, true, &out) == -1);
    // request 1 has tiles in flight: it stops receiving tiles and finishes with them
    Step st = S.next_step();
    CHECK(st.tiles == 8);
    CHECK(S.cancel(1, true, &out) == 0);
    auto done = S.finish(st, 1.0, true);
    CHECK(done.size() == 1 && done[0].id == 1 && done[0].canceled);
    CHECK(S.canceled() == 2 && S.completed() == 0 && S.latencies().empty());
    // request 2 (4 tiles launched, 6 left) is not scheduled again after its cancel
    CHECK(S.cancel(2, true, &out) == 1 && out.id == 2);
    CHECK(S.admit(2.0).size() == 1);  // the freed slots admit request 4
    Step s2 = S.next_step();
    for (auto& p : s2.pieces) CHECK(p.id == 4);
    while (!S.idle()) {
        Step sn = s2.tiles ? s2 : S.next_step();
        S.finish(sn, 3.0, true);
        s2 = Step();
    }
    CHECK(S.completed() == 1 && S.canceled() == 3 && S.latencies().size() == 1);
    std::printf("ok cancel_requests\n");
}

int main() {
    pool_basics();
    admission_by_footprint();
    slots_limit_inflight();
    steps_round_robin_and_chunking();
    latency_and_percentiles();
    randomized_invariants();
    cancel_requests();
    return 0;
}
