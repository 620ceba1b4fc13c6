// rcg_admission.h -- admission bookkeeping of the serving engine (host code,
// no CUDA): which submitted requests may start now.
//
// A request has an arrival time, an HBM footprint and one or two device byte
// extents [lo, hi) it reads or writes.  admit(now) examines the arrived
// requests in submission order and admits each one whose extents overlap
// neither an admitted (not yet retired) request nor an earlier request that
// is still waiting; a request that does overlap waits, and the ones behind it
// that do not go ahead.  Admission stops at the first request that would
// exceed the in-flight count or the HBM budget.  So requests on the same
// bytes start in submission order and never run at the same time.
//
// Cost: a waiting request is examined again only after something retires
// (nothing else can free it); conflicts are found first by the exact extent
// (one hash lookup -- the common case, requests on the same stripe), then by
// ordered maps of disjoint intervals.
#pragma once

#include <stdint.h>

#include <algorithm>
#include <deque>
#include <iterator>
#include <map>
#include <unordered_map>
#include <vector>

namespace rcg {

// A device byte range [lo, hi) a request reads or writes.
struct Extent {
    uintptr_t lo = 0, hi = 0;
};

class Admission {
public:
    struct Item {
        uint64_t arrival_ns = 0;
        uint64_t footprint = 0;
        Extent ext[2];
        uint32_t n_ext = 0;
    };

    Admission(uint64_t budget_bytes, uint32_t max_inflight) : budget_(budget_bytes), max_inflight_(max_inflight) {}

    // Queue a request; ids are 0, 1, 2, ... in submission order.  Its two
    // extents are merged into one when they overlap or touch, so the extents
    // of admitted requests stay disjoint; empty extents are dropped.
    uint64_t add(Item it) {
        uint32_t n = 0;
        for (uint32_t k = 0; k < it.n_ext && k < 2; ++k)
            if (it.ext[k].hi > it.ext[k].lo) it.ext[n++] = it.ext[k];
        if (n == 2 && it.ext[1].lo <= it.ext[0].hi && it.ext[0].lo <= it.ext[1].hi) {
            it.ext[0].lo = std::min(it.ext[0].lo, it.ext[1].lo);
            it.ext[0].hi = std::max(it.ext[0].hi, it.ext[1].hi);
            n = 1;
        }
        it.n_ext = n;
        items_.push_back(it);
        pending_.push_back(items_.size() - 1);
        return items_.size() - 1;
    }

    // An admitted request has completed: free its extents, budget and slot.
    void retire(uint64_t id) {
        const Item &r = items_[id];
        budget_used_ -= r.footprint;
        --inflight_;
        for (uint32_t k = 0; k < r.n_ext; ++k) {
            busy_.erase(r.ext[k].lo);
            busy_exact_.erase(r.ext[k].lo);
        }
        freed_ = true;
    }

    // Admit the requests that may start at `now`; admitted(id) is called for
    // each, in submission order.  Returns how many were admitted.
    template <class F>
    uint32_t admit(uint64_t now, F &&admitted) {
        // waiting requests move only once something has retired: then they are
        // examined again, ahead of the later arrivals, and the union of waiting
        // extents is rebuilt as they are
        if (freed_ && !blocked_.empty()) {
            pending_.insert(pending_.begin(), blocked_.begin(), blocked_.end());
            blocked_.clear();
            waiting_.clear();
            waiting_exact_.clear();
        }
        freed_ = false;
        uint32_t n = 0;
        while (!pending_.empty()) {
            const uint64_t id = pending_.front();
            const Item &r = items_[id];
            if (r.arrival_ns > now) break;
            if (inflight_ >= max_inflight_) break;
            if (budget_used_ + r.footprint > budget_) break;
            bool conflict = false;
            for (uint32_t k = 0; k < r.n_ext && !conflict; ++k) {
                const Extent &e = r.ext[k];
                // two extents with the same first byte overlap
                conflict = busy_exact_.count(e.lo) || waiting_exact_.count(e.lo) || overlaps(busy_, e) ||
                           overlaps(waiting_, e);
            }
            pending_.pop_front();
            if (conflict) {
                for (uint32_t k = 0; k < r.n_ext; ++k) {
                    const Extent &e = r.ext[k];
                    // an extent identical to a busy or waiting one is covered already
                    auto b = busy_exact_.find(e.lo);
                    auto w = waiting_exact_.find(e.lo);
                    const bool known = (b != busy_exact_.end() && b->second == e.hi) ||
                                       (w != waiting_exact_.end() && w->second == e.hi);
                    if (!known) {
                        insert_merged(waiting_, e);
                        if (w == waiting_exact_.end() || w->second < e.hi) waiting_exact_[e.lo] = e.hi;
                    }
                }
                ++conflict_waits_;
                blocked_.push_back(id);
                continue;
            }
            for (uint32_t k = 0; k < r.n_ext; ++k) {
                busy_[r.ext[k].lo] = r.ext[k].hi;
                busy_exact_[r.ext[k].lo] = r.ext[k].hi;
            }
            budget_used_ += r.footprint;
            ++inflight_;
            max_inflight_seen_ = std::max(max_inflight_seen_, inflight_);
            ++n;
            admitted(id);
        }
        return n;
    }

    uint32_t inflight() const { return inflight_; }
    uint32_t max_inflight_seen() const { return max_inflight_seen_; }
    uint64_t conflict_waits() const { return conflict_waits_; }
    uint64_t budget_used() const { return budget_used_; }

private:
    // Does [e.lo, e.hi) overlap a range of the disjoint, sorted map?
    static bool overlaps(const std::map<uintptr_t, uintptr_t> &m, const Extent &e) {
        auto it = m.upper_bound(e.lo);
        if (it != m.begin() && std::prev(it)->second > e.lo) return true;
        return it != m.end() && it->first < e.hi;
    }

    // Add [e.lo, e.hi) to a disjoint, sorted map, merging the ranges it touches.
    static void insert_merged(std::map<uintptr_t, uintptr_t> &m, Extent e) {
        auto it = m.upper_bound(e.lo);
        if (it != m.begin() && std::prev(it)->second >= e.lo) --it;
        while (it != m.end() && it->first <= e.hi) {
            e.lo = std::min(e.lo, it->first);
            e.hi = std::max(e.hi, it->second);
            it = m.erase(it);
        }
        m[e.lo] = e.hi;
    }

    std::vector<Item> items_;
    std::deque<uint64_t> pending_;  // submitted, not yet examined (submission order)
    std::deque<uint64_t> blocked_;  // examined, waiting on an overlapping request
    std::map<uintptr_t, uintptr_t> busy_;     // extents of admitted requests, lo -> hi (disjoint)
    std::map<uintptr_t, uintptr_t> waiting_;  // union of the blocked requests' extents (merged)
    std::unordered_map<uintptr_t, uintptr_t> busy_exact_, waiting_exact_;
    uint64_t budget_ = 0, budget_used_ = 0, conflict_waits_ = 0;
    uint32_t max_inflight_ = 0, inflight_ = 0, max_inflight_seen_ = 0;
    bool freed_ = false;
};

}  // namespace rcg
