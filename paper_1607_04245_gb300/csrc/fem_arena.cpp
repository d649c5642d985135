// fem_arena.cpp -- host-side first-fit sub-allocator over one caller-owned device
// buffer, used by the serving loop to admit requests by their HBM footprint.
//
// The arena only manages offsets: it never touches device memory and makes no CUDA
// call. Free ranges are kept sorted by offset and merged with their neighbours on
// release, so the largest free range is what a new request can get.
#include <cstdint>
#include <iterator>
#include <map>
#include <mutex>
#include <new>
#include <unordered_map>

#include "../../include/fem.h"

namespace fem {
fem_status fail(fem_status st, const char *fmt, ...);
}

struct fem_arena {
    int64_t capacity = 0;
    int64_t alignment = 256;
    std::map<int64_t, int64_t> free_ranges;       // offset -> size, disjoint, non-adjacent
    std::unordered_map<int64_t, int64_t> in_use;  // offset -> size
    int64_t free_bytes = 0;
    std::mutex mu;
};

using fem::fail;

extern "C" fem_status fem_arena_create(int64_t capacity, int64_t alignment, fem_arena **out) {
    if (!out) return fail(FEM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (capacity < 0) return fail(FEM_ERR_ARG, "negative capacity");
    if (alignment <= 0 || (alignment & (alignment - 1)) != 0) return fail(FEM_ERR_ARG, "alignment must be a power of 2");
    fem_arena *a = new (std::nothrow) fem_arena;
    if (!a) return fail(FEM_ERR_OOM, "host allocation failed");
    a->capacity = capacity - capacity % alignment;
    a->alignment = alignment;
    if (a->capacity > 0) a->free_ranges.emplace(0, a->capacity);
    a->free_bytes = a->capacity;
    *out = a;
    return FEM_OK;
}

extern "C" void fem_arena_destroy(fem_arena *a) { delete a; }

extern "C" fem_status fem_arena_alloc(fem_arena *a, int64_t bytes, int64_t *offset) {
    if (!a || !offset) return fail(FEM_ERR_ARG, "NULL arena or offset");
    if (bytes < 0) return fail(FEM_ERR_ARG, "negative size");
    const int64_t need = bytes == 0 ? a->alignment : (bytes + a->alignment - 1) / a->alignment * a->alignment;
    std::lock_guard<std::mutex> lk(a->mu);
    for (auto it = a->free_ranges.begin(); it != a->free_ranges.end(); ++it) {
        if (it->second >= need) {
            const int64_t off = it->first, rest = it->second - need;
            a->free_ranges.erase(it);
            if (rest > 0) a->free_ranges.emplace(off + need, rest);
            a->in_use.emplace(off, need);
            a->free_bytes -= need;
            *offset = off;
            return FEM_OK;
        }
    }
    return fail(FEM_ERR_OOM, "no free range of %lld bytes (free %lld)", static_cast<long long>(need),
                static_cast<long long>(a->free_bytes));
}

extern "C" fem_status fem_arena_free(fem_arena *a, int64_t offset) {
    if (!a) return fail(FEM_ERR_ARG, "NULL arena");
    std::lock_guard<std::mutex> lk(a->mu);
    auto u = a->in_use.find(offset);
    if (u == a->in_use.end()) return fail(FEM_ERR_ARG, "offset %lld is not allocated", static_cast<long long>(offset));
    int64_t off = offset, size = u->second;
    a->in_use.erase(u);
    a->free_bytes += size;
    auto next = a->free_ranges.lower_bound(off);
    if (next != a->free_ranges.begin()) {
        auto prev = std::prev(next);
        if (prev->first + prev->second == off) {
            off = prev->first;
            size += prev->second;
            a->free_ranges.erase(prev);
        }
    }
    if (next != a->free_ranges.end() && off + size == next->first) {
        size += next->second;
        a->free_ranges.erase(next);
    }
    a->free_ranges.emplace(off, size);
    return FEM_OK;
}

extern "C" int64_t fem_arena_free_bytes(fem_arena *a) {
    if (!a) return 0;
    std::lock_guard<std::mutex> lk(a->mu);
    return a->free_bytes;
}

extern "C" int64_t fem_arena_largest_free(fem_arena *a) {
    if (!a) return 0;
    std::lock_guard<std::mutex> lk(a->mu);
    int64_t m = 0;
    for (const auto &r : a->free_ranges) m = r.second > m ? r.second : m;
    return m;
}

extern "C" int64_t fem_arena_capacity(fem_arena *a) { return a ? a->capacity : 0; }
