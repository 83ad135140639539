// ranges.h -- first-fit allocator of index ranges (a server's record space),
// host code.
#pragma once
#include <cstdint>
#include <utility>
#include <vector>

namespace lpp {

// Free ranges (start, length), sorted by start and never adjacent: take()
// returns the lowest start of a free range long enough (first fit) or -1;
// give() returns a range and merges it with its free neighbours.
struct Ranges {
    std::vector<std::pair<int32_t, int32_t>> free_;
    void init(int32_t cap) { free_.assign(1, {0, cap}); }
    int32_t take(int32_t len) {
        if (len == 0) return 0;
        for (size_t k = 0; k < free_.size(); k++)
            if (free_[k].second >= len) {
                const int32_t s = free_[k].first;
                free_[k].first += len;
                free_[k].second -= len;
                if (free_[k].second == 0) free_.erase(free_.begin() + (long)k);
                return s;
            }
        return -1;
    }
    void give(int32_t s, int32_t len) {
        if (len == 0) return;
        auto it = free_.begin();
        while (it != free_.end() && it->first < s) ++it;
        it = free_.insert(it, {s, len});
        if (it + 1 != free_.end() && it->first + it->second == (it + 1)->first) {
            it->second += (it + 1)->second;
            free_.erase(it + 1);
        }
        if (it != free_.begin() && (it - 1)->first + (it - 1)->second == it->first) {
            (it - 1)->second += it->second;
            free_.erase(it);
        }
    }
};

}  // namespace lpp
