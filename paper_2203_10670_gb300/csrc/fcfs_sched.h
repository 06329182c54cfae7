// Host-side core of the FCFS serving loop: the device-memory pool, admission
// by footprint, step building under a tile budget, and latency statistics.
// Plain C++ with no CUDA calls, so its logic is testable without a GPU.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <deque>
#include <map>
#include <vector>

namespace fcfs {
namespace sched {

// First-fit allocator over [0, size) with 256-byte granules.  Offsets only;
// the caller adds its device base address.
class Pool {
   public:
    explicit Pool(size_t size = 0) { reset(size); }
    void reset(size_t size) {
        size_ = size / kAlign * kAlign;
        free_.clear();
        if (size_) free_[0] = size_;
        used_ = 0;
    }
    static size_t round(size_t n) { return (n + kAlign - 1) / kAlign * kAlign; }
    // offset of a block of n bytes, or SIZE_MAX when no free block is large enough
    size_t alloc(size_t n) {
        n = round(std::max<size_t>(n, 1));
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            const size_t off = it->first, len = it->second;
            free_.erase(it);
            if (len > n) free_[off + n] = len - n;
            used_ += n;
            return off;
        }
        return SIZE_MAX;
    }
    void release(size_t off, size_t n) {
        n = round(std::max<size_t>(n, 1));
        used_ -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t size() const { return size_; }
    size_t used() const { return used_; }
    size_t largest_free() const {
        size_t m = 0;
        for (auto& f : free_) m = std::max(m, f.second);
        return m;
    }

   private:
    static constexpr size_t kAlign = 256;
    size_t size_ = 0, used_ = 0;
    std::map<size_t, size_t> free_;  // offset -> length
};

struct Request {
    uint64_t id = 0;
    double arrival = 0;       // seconds, steady clock
    long long tiles = 0;      // tiles of the whole request
    long long next_tile = 0;  // first tile not yet launched
    long long done_tiles = 0;
    size_t out_bytes = 0;     // pool bytes (0 when the caller owns y)
    size_t pool_off = SIZE_MAX;
    int slot = -1;            // device parameter slot
    double out_pixels = 0;
    double bytes = 0;         // algorithmic bytes (input + output)
    double admitted = 0;
    bool deferred_counted = false;
    bool canceled = false;    // no further tiles; completes when its launched tiles finish
};

// One launch: the tile ranges it covers, per request slot.
struct Piece {
    int slot;
    uint64_t id;
    long long first, count;
};

struct Step {
    std::vector<Piece> pieces;
    long long tiles = 0;
};

class Scheduler {
   public:
    Scheduler(size_t pool_bytes, int max_inflight, long long tile_budget)
        : pool_(pool_bytes), max_inflight_(std::max(1, max_inflight)), budget_(std::max(1LL, tile_budget)) {
        for (int s = max_inflight_ - 1; s >= 0; --s) free_slots_.push_back(s);
    }

    // queue a request; false when its output could never fit the pool
    bool submit(const Request& r) {
        if (r.out_bytes > 0 && Pool::round(r.out_bytes) > pool_.size()) return false;
        queue_.push_back(r);
        ++submitted_;
        return true;
    }

    // Move queued requests into the active set while a slot and pool memory
    // are free (arrival order; the head of the queue blocks the rest so large
    // requests are not starved).  Returns the newly admitted requests.
    std::vector<Request*> admit(double now) {
        std::vector<Request*> out;
        while (!queue_.empty() && !free_slots_.empty()) {
            Request& q = queue_.front();
            size_t off = SIZE_MAX;
            if (q.out_bytes > 0) {
                off = pool_.alloc(q.out_bytes);
                if (off == SIZE_MAX) {
                    if (!q.deferred_counted) {
                        ++deferred_;
                        q.deferred_counted = true;
                    }
                    break;
                }
            }
            Request r = q;
            queue_.pop_front();
            r.pool_off = off;
            r.slot = free_slots_.back();
            free_slots_.pop_back();
            r.admitted = now;
            active_[r.id] = r;
            out.push_back(&active_[r.id]);
            max_inflight_seen_ = std::max(max_inflight_seen_, (int)active_.size());
        }
        return out;
    }

    // Build the next launch: up to `budget` tiles, shared round-robin among the
    // active requests that still have tiles (requests admitted later join the
    // next step; a large request is chunked across steps).
    Step next_step() {
        Step st;
        std::vector<Request*> pending;
        for (auto& kv : active_)
            if (kv.second.next_tile < kv.second.tiles) pending.push_back(&kv.second);
        if (pending.empty()) return st;
        std::sort(pending.begin(), pending.end(), [](Request* a, Request* b) { return a->id < b->id; });
        long long left = budget_;
        // fair share, at least one tile each, leftover to the oldest
        const long long share = std::max(1LL, budget_ / (long long)pending.size());
        for (int pass = 0; pass < 2 && left > 0; ++pass) {
            for (Request* r : pending) {
                if (left <= 0) break;
                const long long remain = r->tiles - r->next_tile;
                if (remain <= 0) continue;
                const long long take = std::min(remain, pass == 0 ? std::min(share, left) : left);
                if (take <= 0) continue;
                bool merged = false;
                for (auto& p : st.pieces)
                    if (p.slot == r->slot && p.first + p.count == r->next_tile) {
                        p.count += take;
                        merged = true;
                    }
                if (!merged) st.pieces.push_back(Piece{r->slot, r->id, r->next_tile, take});
                r->next_tile += take;
                st.tiles += take;
                left -= take;
            }
        }
        return st;
    }

    // The tiles of a launched step have finished; returns the requests that
    // are now complete (removed from the active set, slot and pool returned).
    std::vector<Request> finish(const Step& st, double now, bool release_pool) {
        std::vector<Request> done;
        for (auto& p : st.pieces) {
            auto it = active_.find(p.id);
            if (it == active_.end()) continue;
            Request& r = it->second;
            r.done_tiles += p.count;
            if (r.done_tiles >= r.tiles) {
                if (r.canceled) {
                    ++canceled_;
                } else {
                    latencies_.push_back(now - r.arrival);
                    out_pixels_ += r.out_pixels;
                    bytes_ += r.bytes;
                    ++completed_;
                }
                if (release_pool && r.pool_off != SIZE_MAX) {
                    pool_.release(r.pool_off, r.out_bytes);
                    r.pool_off = SIZE_MAX;
                }
                free_slots_.push_back(r.slot);
                done.push_back(r);
                active_.erase(it);
            }
        }
        return done;
    }

    // return the pool block of a completed request kept for the caller
    // Cancel a request.  Queued: removed at once.  Admitted with none of its tiles in flight:
    // finished at once (slot and pool memory returned).  Otherwise no further tile is launched and
    // it finishes, uncounted in the latency and throughput totals, when its launched tiles
    // complete.  Returns 1 when the request is finished now (*out holds it), 0 when it finishes
    // later, -1 when the id is neither queued nor active.
    int cancel(uint64_t id, bool release_pool, Request* out) {
        for (auto it = queue_.begin(); it != queue_.end(); ++it)
            if (it->id == id) {
                *out = *it;
                out->canceled = true;
                queue_.erase(it);
                ++canceled_;
                return 1;
            }
        auto it = active_.find(id);
        if (it == active_.end()) return -1;
        Request& r = it->second;
        r.canceled = true;
        r.tiles = r.next_tile;  // nothing more is scheduled
        if (r.done_tiles < r.tiles) return 0;
        if (release_pool && r.pool_off != SIZE_MAX) {
            pool_.release(r.pool_off, r.out_bytes);
            r.pool_off = SIZE_MAX;
        }
        free_slots_.push_back(r.slot);
        *out = r;
        active_.erase(it);
        ++canceled_;
        return 1;
    }

    void release_output(size_t off, size_t bytes) {
        if (off != SIZE_MAX) pool_.release(off, bytes);
    }

    static double percentile(std::vector<double> v, double p) {
        if (v.empty()) return 0;
        std::sort(v.begin(), v.end());
        const double k = p / 100.0 * (v.size() - 1);
        const size_t lo = (size_t)std::floor(k), hi = (size_t)std::ceil(k);
        return v[lo] + (v[hi] - v[lo]) * (k - lo);
    }

    size_t queued() const { return queue_.size(); }
    size_t active() const { return active_.size(); }
    long long submitted() const { return submitted_; }
    long long completed() const { return completed_; }
    long long canceled() const { return canceled_; }
    long long deferred() const { return deferred_; }
    int max_inflight_seen() const { return max_inflight_seen_; }
    const std::vector<double>& latencies() const { return latencies_; }
    double out_pixels() const { return out_pixels_; }
    double bytes() const { return bytes_; }
    const Pool& pool() const { return pool_; }
    bool idle() const { return queue_.empty() && active_.empty(); }
    std::map<uint64_t, Request>& active_map() { return active_; }

   private:
    Pool pool_;
    int max_inflight_;
    long long budget_;
    std::deque<Request> queue_;
    std::map<uint64_t, Request> active_;
    std::vector<int> free_slots_;
    std::vector<double> latencies_;
    long long submitted_ = 0, completed_ = 0, deferred_ = 0, canceled_ = 0;
    int max_inflight_seen_ = 0;
    double out_pixels_ = 0, bytes_ = 0;
};

}  // namespace sched
}  // namespace fcfs
