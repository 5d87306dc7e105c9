// Test harness: exposes the serving loop's arena (sell_arena.h) through a C
// interface so that a CPU test can drive it.  Built with g++ by the test.
#include <cstddef>

#include "sell_arena.h"

static sell::Arena g_arena;

extern "C" {
void arena_reset(size_t bytes) { g_arena.reset(bytes); }
int arena_alloc(size_t bytes, size_t *off) { return g_arena.alloc(bytes, off) ? 1 : 0; }
void arena_release(size_t off, size_t bytes) { g_arena.release(off, bytes); }
size_t arena_region(size_t bytes) { return sell::region(bytes); }
size_t arena_free_ranges(size_t *offs, size_t *lens, size_t cap) {
    size_t n = 0;
    for (const auto &kv : g_arena.free_ranges()) {
        if (n < cap) {
            offs[n] = kv.first;
            lens[n] = kv.second;
        }
        ++n;
    }
    return n;
}
}
