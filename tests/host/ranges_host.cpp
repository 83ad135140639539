// Host build of the server's record-space allocator (ranges.h) for its CPU
// test: a handle-based C interface over lpp::Ranges.
#include <cstdint>

#include "../../paper_2609_16182_gb300/csrc/ranges.h"

extern "C" {
void *ranges_new(int32_t cap) {
    auto *r = new lpp::Ranges();
    r->init(cap);
    return r;
}
void ranges_free(void *r) { delete static_cast<lpp::Ranges *>(r); }
int32_t ranges_take(void *r, int32_t len) { return static_cast<lpp::Ranges *>(r)->take(len); }
void ranges_give(void *r, int32_t s, int32_t len) { static_cast<lpp::Ranges *>(r)->give(s, len); }
// the free list: up to cap (start, length) pairs into out, returns its size
int32_t ranges_list(void *r, int32_t *out, int32_t cap) {
    const auto &f = static_cast<lpp::Ranges *>(r)->free_;
    for (int32_t k = 0; k < (int32_t)f.size() && k < cap; k++) {
        out[2 * k] = f[k].first;
        out[2 * k + 1] = f[k].second;
    }
    return (int32_t)f.size();
}
}
