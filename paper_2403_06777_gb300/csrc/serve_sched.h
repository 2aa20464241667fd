// serve_sched.h -- host-side pieces of the request server (no CUDA): the
// allocator of the device arena that holds resident tables, and the planner
// that cuts the resident requests' ranges into one step's chunks.
#pragma once
#include <stddef.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <vector>

namespace zxp {

// First-fit allocator over offsets [0, capacity), blocks aligned to `align`
// bytes; freeing coalesces with both neighbours.
class Arena {
  public:
    explicit Arena(uint64_t capacity = 0, uint64_t align = 512) { reset(capacity, align); }

    void reset(uint64_t capacity, uint64_t align = 512) {
        align_ = align ? align : 1;
        cap_ = capacity / align_ * align_;
        free_.clear();
        live_.clear();
        used_ = peak_ = 0;
        if (cap_) free_[0] = cap_;
    }

    bool alloc(uint64_t bytes, uint64_t* off) {
        if (!bytes) bytes = 1;
        const uint64_t sz = (bytes + align_ - 1) / align_ * align_;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < sz) continue;
            const uint64_t o = it->first, rest = it->second - sz;
            free_.erase(it);
            if (rest) free_[o + sz] = rest;
            live_[o] = sz;
            used_ += sz;
            peak_ = std::max(peak_, used_);
            *off = o;
            return true;
        }
        return false;
    }

    // Returns false (and changes nothing) if off is not a live block.
    bool release(uint64_t off) {
        auto it = live_.find(off);
        if (it == live_.end()) return false;
        uint64_t o = off, sz = it->second;
        live_.erase(it);
        used_ -= sz;
        auto nx = free_.lower_bound(o);
        if (nx != free_.end() && nx->first == o + sz) {
            sz += nx->second;
            nx = free_.erase(nx);
        }
        if (nx != free_.begin()) {
            auto pv = std::prev(nx);
            if (pv->first + pv->second == o) {
                o = pv->first;
                sz += pv->second;
                free_.erase(pv);
            }
        }
        free_[o] = sz;
        return true;
    }

    uint64_t capacity() const { return cap_; }
    uint64_t used() const { return used_; }
    uint64_t peak() const { return peak_; }
    size_t live_blocks() const { return live_.size(); }
    size_t free_blocks() const { return free_.size(); }
    uint64_t largest_free() const {
        uint64_t m = 0;
        for (auto& f : free_) m = std::max(m, f.second);
        return m;
    }
    // Would a block of `bytes` ever fit (empty arena)?
    bool fits_at_all(uint64_t bytes) const {
        return (std::max<uint64_t>(bytes, 1) + align_ - 1) / align_ * align_ <= cap_;
    }

  private:
    std::map<uint64_t, uint64_t> free_;   // offset -> size
    std::map<uint64_t, uint64_t> live_;   // offset -> size
    uint64_t cap_ = 0, align_ = 512, used_ = 0, peak_ = 0;
};

// The unplanned part [next, total) of one resident request's range.
struct WorkItem {
    uint64_t total = 0;     // 2^k terms
    uint64_t next = 0;      // first term not yet given to a step
    uint64_t order = 0;     // admission order: smaller is older
};

struct PlannedChunk {
    size_t item;            // index into the items vector
    uint64_t first, count;
};

// Plan one step of at most `budget` terms (at least one chunk when any work
// remains, so every step makes progress):
//   * items with at most `small` terms left are taken whole, fewest first
//     (ties: oldest first), while the small share of the budget lasts;
//   * when larger items exist, a quarter of the budget is kept for them and
//     whatever the small items leave is added; they are served oldest first.
// A share is cut into chunks of at most 2^chunk_log2 terms.  Every share but
// an item's last is a multiple of 8 terms, so chunk starts stay multiples of
// 8.  items[i].next advances by what was planned.
inline void plan_step(std::vector<WorkItem>& items, uint64_t budget, uint32_t chunk_log2,
                      uint64_t small, std::vector<PlannedChunk>* out) {
    out->clear();
    const uint64_t clen = 1ull << std::min<uint32_t>(std::max<uint32_t>(chunk_log2, 3), 62);
    budget = std::max<uint64_t>(budget, 8);
    std::vector<size_t> sm, lg;
    for (size_t i = 0; i < items.size(); i++) {
        const uint64_t left = items[i].total - items[i].next;
        if (!left) continue;
        (left <= small ? sm : lg).push_back(i);
    }
    auto left_of = [&](size_t i) { return items[i].total - items[i].next; };
    std::stable_sort(sm.begin(), sm.end(), [&](size_t a, size_t b) {
        const uint64_t la = left_of(a), lb = left_of(b);
        return la != lb ? la < lb : items[a].order < items[b].order;
    });
    std::stable_sort(lg.begin(), lg.end(), [&](size_t a, size_t b) { return items[a].order < items[b].order; });

    auto emit = [&](size_t i, uint64_t n) {
        WorkItem& w = items[i];
        for (uint64_t f = w.next, end = w.next + n; f < end; f += clen)
            out->push_back(PlannedChunk{i, f, std::min(clen, end - f)});
        w.next += n;
    };
    uint64_t used = 0;
    const uint64_t small_budget = lg.empty() ? budget : budget - budget / 4;
    for (size_t i : sm) {
        const uint64_t n = left_of(i);
        if (used + n > small_budget && !out->empty()) break;
        emit(i, n);
        used += n;
    }
    for (size_t i : lg) {
        const uint64_t room = budget > used ? budget - used : 0;
        if (room < 8 && !out->empty()) break;
        uint64_t n = left_of(i);
        if (n > room) n = std::min(n, std::max<uint64_t>(room / 8 * 8, 8));   // a multiple of 8, or all
        emit(i, n);
        used += n;
    }
}

}  // namespace zxp
