// serve_sched.h -- host-side bookkeeping of the serving loop: the device
// memory arena and the plan of each step.  Plain C++17 without CUDA, so the
// admission, packing and memory rules can be exercised on any host.
//
// A request goes QUEUED -> EXTRACT (its skewers are spread over one or more
// steps) -> ROOT (its mean-flux root-find runs, one or more steps) -> DONE.
// It holds a slot from admission to the end of its root-find, and two arena
// blocks: tau (freed when the root-find ends) and F (freed on release).
#pragma once

#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <deque>
#include <map>
#include <unordered_map>
#include <vector>

namespace lya {
namespace serve {

constexpr size_t kNoOffset = SIZE_MAX;

// First-fit allocator over the byte range [0, capacity).  Blocks are rounded
// up to `align` bytes; a freed block merges with free neighbours.
class Arena {
public:
    explicit Arena(size_t capacity, size_t align = 256) : cap_(capacity - capacity % align), align_(align)
    {
        if (cap_ > 0) free_[0] = cap_;
    }

    size_t alloc(size_t bytes)
    {
        if (bytes == 0) bytes = 1;
        const size_t need = (bytes + align_ - 1) / align_ * align_;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < need) continue;
            const size_t off = it->first, left = it->second - need;
            free_.erase(it);
            if (left) free_[off + need] = left;
            used_[off] = need;
            in_use_ += need;
            peak_ = std::max(peak_, in_use_);
            return off;
        }
        return kNoOffset;
    }

    bool release(size_t off)
    {
        auto u = used_.find(off);
        if (u == used_.end()) return false;
        size_t start = off, size = u->second;
        in_use_ -= size;
        used_.erase(u);
        auto next = free_.lower_bound(start);
        if (next != free_.end() && next->first == start + size) {
            size += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == start) {
                start = prev->first;
                size += prev->second;
                free_.erase(prev);
            }
        }
        free_[start] = size;
        return true;
    }

    size_t rounded(size_t bytes) const { return (std::max<size_t>(bytes, 1) + align_ - 1) / align_ * align_; }
    size_t capacity() const { return cap_; }
    size_t used() const { return in_use_; }
    size_t peak() const { return peak_; }
    size_t largest_free() const
    {
        size_t m = 0;
        for (const auto& f : free_) m = std::max(m, f.second);
        return m;
    }

    // Free and used blocks tile [0, capacity) without overlap, free blocks
    // are never adjacent, and the in-use count matches.
    bool consistent() const
    {
        std::map<size_t, std::pair<size_t, bool>> all;
        for (const auto& f : free_) all[f.first] = {f.second, true};
        for (const auto& u : used_) {
            if (all.count(u.first)) return false;
            all[u.first] = {u.second, false};
        }
        size_t pos = 0, used = 0;
        bool prev_free = false;
        for (const auto& b : all) {
            if (b.first != pos || b.second.first == 0 || b.second.first % align_) return false;
            if (b.second.second && prev_free) return false;
            prev_free = b.second.second;
            if (!b.second.second) used += b.second.first;
            pos += b.second.first;
        }
        return pos == cap_ && used == in_use_;
    }

private:
    size_t cap_, align_;
    size_t in_use_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_, used_;
};

enum class Phase { kQueued, kExtract, kRoot, kDone };

struct Request {
    uint64_t ticket = 0;
    int64_t n_rows = 0;       // skewers
    int n_pix = 0;
    int shift = 0;            // log2(skewers per optical-depth task)
    double row_cost = 1.0;    // estimated optical-depth time per skewer (ns)
    double task_key = 0.0;    // order of tasks within a step (larger first)
    // scheduler state
    Phase phase = Phase::kQueued;
    int slot = -1;
    size_t tau_off = kNoOffset, flux_off = kNoOffset;
    int64_t rows_planned = 0;     // skewers handed to steps so far
    bool rf_started = false;      // root-find state initialised on the device
    int64_t admit_seq = 0;

    int64_t pixels() const { return n_rows * (int64_t)n_pix; }
    size_t block_bytes() const { return (size_t)pixels() * sizeof(float); }
};

struct StepPlan {
    struct Task { int slot; int first_item; int n_items; int shift; };
    struct Item { int slot; int64_t row; };
    struct Rf { int slot; int init; int unit_first; int unit_count; int64_t unit_pix; };
    struct Unit { int rf; int64_t begin, end; };
    std::vector<int> tau_slots;     // slots with optical-depth work this step
    std::vector<Task> tasks;        // items [first_item, first_item + n_items), larger first
    std::vector<Item> items;
    std::vector<Rf> rf;             // root-find participants
    std::vector<Unit> units;        // root-find work units, grouped by participant
    bool empty() const { return tasks.empty() && rf.empty(); }
};

struct Limits {
    size_t budget = 0;            // arena bytes
    int max_slots = 1;
    double step_quota_ns = 2e6;   // optical-depth work per step (estimated)
    int64_t max_items = 1 << 16;  // skewers per step
    int64_t max_units = 1 << 16;  // root-find units per step
    int64_t unit_pix = 16384;     // pixels per root-find unit (minimum)
    int64_t max_units_per_request = 4096;
};

class Scheduler {
public:
    explicit Scheduler(const Limits& lim) : lim_(lim), arena_(lim.budget), slot_used_(lim.max_slots, 0) {}

    // Bytes a request holds in the arena (tau + F).
    size_t request_bytes(const Request& r) const { return 2 * arena_.rounded(r.block_bytes()); }

    // Queue a request; false if it could never fit the arena.
    bool enqueue(const Request& r)
    {
        if (request_bytes(r) > arena_.capacity() || r.n_rows <= 0 || r.n_pix <= 0) return false;
        reqs_[r.ticket] = r;
        reqs_[r.ticket].phase = Phase::kQueued;
        queue_.push_back(r.ticket);
        return true;
    }

    // Admit from the head of the queue, in order, while a slot and memory
    // are free; returns the tickets admitted.
    std::vector<uint64_t> admit()
    {
        std::vector<uint64_t> out;
        while (!queue_.empty()) {
            Request& r = reqs_.at(queue_.front());
            const int slot = free_slot();
            if (slot < 0) break;
            const size_t tau = arena_.alloc(r.block_bytes());
            if (tau == kNoOffset) break;
            const size_t flux = arena_.alloc(r.block_bytes());
            if (flux == kNoOffset) {
                arena_.release(tau);
                break;
            }
            r.tau_off = tau;
            r.flux_off = flux;
            r.slot = slot;
            slot_used_[slot] = 1;
            r.phase = Phase::kExtract;
            r.rows_planned = 0;
            r.rf_started = false;
            r.admit_seq = seq_++;
            active_.push_back(r.ticket);
            out.push_back(r.ticket);
            queue_.pop_front();
        }
        return out;
    }

    // The next step: skewers of extracting requests (oldest first; each gets
    // at least one task, then the rest of the quota in order), and the
    // root-find of every request whose skewers are all planned.
    StepPlan plan()
    {
        StepPlan p;
        double quota = lim_.step_quota_ns;
        // pass 1: one task per extracting request; pass 2: the quota
        for (int pass = 0; pass < 2; ++pass) {
            for (uint64_t t : active_) {
                Request& r = reqs_.at(t);
                if (r.phase != Phase::kExtract) continue;
                const int64_t left = r.n_rows - r.rows_planned;
                if (left <= 0) continue;
                const int64_t g = (int64_t)1 << r.shift;
                int64_t rows;
                if (pass == 0) {
                    rows = std::min(left, g);
                } else {
                    const double fit = quota / std::max(r.row_cost, 1e-9);
                    rows = std::min<int64_t>(left, (int64_t)fit / g * g);
                }
                rows = std::min<int64_t>(rows, lim_.max_items - (int64_t)p.items.size());
                if (rows <= 0) continue;
                add_rows(p, r, rows);
                quota -= rows * r.row_cost;
            }
        }
        // tasks: larger first (the work list is taken in order by the CTAs)
        std::stable_sort(p.tasks.begin(), p.tasks.end(), [&](const StepPlan::Task& a, const StepPlan::Task& b) {
            return key_of_slot(a.slot) > key_of_slot(b.slot);
        });
        // root-find participants
        for (uint64_t t : active_) {
            Request& r = reqs_.at(t);
            if (r.phase == Phase::kExtract && r.rows_planned == r.n_rows) r.phase = Phase::kRoot;
            if (r.phase != Phase::kRoot) continue;
            const int64_t n = r.pixels();
            int64_t upix = std::max(lim_.unit_pix, (n + lim_.max_units_per_request - 1) / lim_.max_units_per_request);
            upix = (upix + 3) / 4 * 4;                       // units start 16-byte aligned
            const int64_t cnt = (n + upix - 1) / upix;
            if (!p.rf.empty() && (int64_t)p.units.size() + cnt > lim_.max_units) continue;   // next step
            StepPlan::Rf f{r.slot, r.rf_started ? 0 : 1, (int)p.units.size(), (int)cnt, upix};
            const int rf_index = (int)p.rf.size();
            for (int64_t u = 0; u < cnt; ++u)
                p.units.push_back(StepPlan::Unit{rf_index, u * upix, std::min(n, (u + 1) * upix)});
            p.rf.push_back(f);
            r.rf_started = true;
        }
        return p;
    }

    // A request's root-find has ended (result read back): frees its slot and
    // tau block; F stays until release().
    void finish(uint64_t ticket)
    {
        Request& r = reqs_.at(ticket);
        if (r.phase == Phase::kDone) return;
        r.phase = Phase::kDone;
        if (r.slot >= 0) slot_used_[r.slot] = 0;
        r.slot = -1;
        if (r.tau_off != kNoOffset) arena_.release(r.tau_off);
        r.tau_off = kNoOffset;
        active_.erase(std::remove(active_.begin(), active_.end(), ticket), active_.end());
    }

    // Fail a request wherever it is (queued or active); frees what it holds
    // except F, which release() frees.
    void fail(uint64_t ticket)
    {
        Request& r = reqs_.at(ticket);
        if (r.phase == Phase::kQueued) {
            queue_.erase(std::remove(queue_.begin(), queue_.end(), ticket), queue_.end());
            r.phase = Phase::kDone;
            return;
        }
        finish(ticket);
    }

    // Forget a finished request and free its F.
    bool release(uint64_t ticket)
    {
        auto it = reqs_.find(ticket);
        if (it == reqs_.end() || it->second.phase != Phase::kDone) return false;
        if (it->second.flux_off != kNoOffset) arena_.release(it->second.flux_off);
        reqs_.erase(it);
        return true;
    }

    Request* find(uint64_t ticket)
    {
        auto it = reqs_.find(ticket);
        return it == reqs_.end() ? nullptr : &it->second;
    }

    int slot_ticket_count() const { return (int)active_.size(); }
    bool has_work() const { return !active_.empty() || (!queue_.empty() && can_admit_head()); }
    size_t queued() const { return queue_.size(); }
    const std::vector<uint64_t>& active() const { return active_; }
    const Arena& arena() const { return arena_; }
    const Limits& limits() const { return lim_; }
    uint64_t ticket_of_slot(int slot) const
    {
        for (uint64_t t : active_)
            if (reqs_.at(t).slot == slot) return t;
        return 0;
    }

private:
    int free_slot() const
    {
        for (int s = 0; s < (int)slot_used_.size(); ++s)
            if (!slot_used_[s]) return s;
        return -1;
    }

    bool can_admit_head() const
    {
        if (queue_.empty() || free_slot() < 0) return false;
        const Request& r = reqs_.at(queue_.front());
        const size_t b = arena_.rounded(r.block_bytes());
        if (arena_.largest_free() < b) return false;
        return true;   // a precise two-block fit is checked by admit()
    }

    double key_of_slot(int slot) const
    {
        for (uint64_t t : active_) {
            const Request& r = reqs_.at(t);
            if (r.slot == slot) return r.task_key;
        }
        return 0.0;
    }

    void add_rows(StepPlan& p, Request& r, int64_t rows)
    {
        const int g = 1 << r.shift;
        if (std::find(p.tau_slots.begin(), p.tau_slots.end(), r.slot) == p.tau_slots.end())
            p.tau_slots.push_back(r.slot);
        for (int64_t k = 0; k < rows; k += g) {
            const int n = (int)std::min<int64_t>(g, rows - k);
            p.tasks.push_back(StepPlan::Task{r.slot, (int)p.items.size(), n, r.shift});
            for (int i = 0; i < n; ++i) p.items.push_back(StepPlan::Item{r.slot, r.rows_planned + k + i});
        }
        r.rows_planned += rows;
    }

    Limits lim_;
    Arena arena_;
    std::vector<char> slot_used_;
    std::unordered_map<uint64_t, Request> reqs_;
    std::deque<uint64_t> queue_;
    std::vector<uint64_t> active_;   // admitted, not finished, in admission order
    int64_t seq_ = 0;
};

}  // namespace serve
}  // namespace lya
