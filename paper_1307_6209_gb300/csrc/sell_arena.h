// sell_arena.h -- the serving loop's sub-allocator of its device arena
// (host-only C++, no CUDA): offsets into one buffer allocated once, so the
// requests in flight can never exceed the budget the arena was sized for.
#ifndef SELL_ARENA_H
#define SELL_ARENA_H

#include <cstddef>
#include <iterator>
#include <map>

namespace sell {

inline size_t round256(size_t x) { return (x + 255) / 256 * 256; }

// Arena bytes of one region of n bytes (empty regions still take one block, so
// that every request owns distinct addresses).
inline size_t region(size_t n) { return round256(n ? n : 1); }

// First-fit sub-allocator of one device buffer; blocks are 256-byte aligned
// and freed blocks merge with their free neighbours, so the free list always
// holds maximal free ranges in offset order.
class Arena {
   public:
    void reset(size_t size) {
        free_.clear();
        if (size) free_[0] = size;
    }
    bool alloc(size_t n, size_t *off) {
        n = round256(n);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            *off = it->first;
            const size_t rest = it->second - n, o = it->first;
            free_.erase(it);
            if (rest) free_[o + n] = rest;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t n) {
        n = round256(n);
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
    // free ranges (offset -> bytes), for inspection
    const std::map<size_t, size_t> &free_ranges() const { return free_; }

   private:
    std::map<size_t, size_t> free_;
};

}  // namespace sell

#endif  // SELL_ARENA_H
