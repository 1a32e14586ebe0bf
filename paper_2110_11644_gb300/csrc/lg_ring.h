// Ring allocator of the serving loop's arenas (host code, no CUDA): contiguous
// ranges of a circular buffer, allocated in order and released in the same
// order.  Kept in a header of its own so that it can be tested on the CPU.
#pragma once

#include <cstddef>
#include <deque>
#include <utility>

namespace lg {

// Contiguous allocations in a circular range, released in the order made.
// The live allocations cover [beg, end), wrapping past the end of the range
// (a gap left at the end is counted with the allocation before it).
struct RingAlloc {
    size_t cap = 0, beg = 0, end = 0, used = 0;
    std::deque<std::pair<size_t, size_t>> live;  // (start, length including a gap after it)
    struct Mark {
        size_t beg, end, used, nlive, back_len;
    };
    void reset(size_t c) {
        cap = c;
        beg = end = used = 0;
        live.clear();
    }
    Mark mark() const { return {beg, end, used, live.size(), live.empty() ? 0 : live.back().second}; }
    void rollback(const Mark &m) {
        while (live.size() > m.nlive) live.pop_back();
        if (!live.empty()) live.back().second = m.back_len;
        beg = m.beg;
        end = m.end;
        used = m.used;
    }
    bool alloc(size_t n, size_t *at) {
        if (live.empty()) beg = end = used = 0;
        if (n > cap) return false;
        const bool wrapped = !live.empty() && (end < beg || (end == beg && used > 0));
        if (wrapped) {  // the free range is [end, beg)
            if (beg - end < n) return false;
        } else if (cap - end < n) {  // no room before the end of the range: wrap if [0, beg) holds it
            if (live.empty() || beg < n) return false;
            live.back().second += cap - end;
            used += cap - end;
            end = 0;
        }
        *at = end;
        live.emplace_back(end, n);
        end += n;
        used += n;
        return true;
    }
    void release_front() {
        used -= live.front().second;
        live.pop_front();
        if (live.empty()) beg = end = used = 0;
        else beg = live.front().first;
    }
};

}  // namespace lg
