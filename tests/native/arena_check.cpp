// Host check of the engine's arena allocator (compiled with g++ by tests/test_arena_cpu.py).
// A seeded sequence of allocations and releases against an independent byte map: every
// allocation is aligned, inside the arena and disjoint from every live one; first fit takes
// the lowest hole that fits; after everything is released the arena is one free block again.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "fwi_arena.h"

#define CHECK(c)                                                            \
    do {                                                                    \
        if (!(c)) {                                                         \
            std::printf("FAIL line %d: %s\n", __LINE__, #c);                \
            return 1;                                                       \
        }                                                                   \
    } while (0)

int main()
{
    const size_t A = 256, N = 1 << 16;        // 64 KiB arena, 256 cells of 256 B
    fwi::Arena ar(A);
    ar.init(N + 100);                         // the unaligned tail is dropped
    CHECK(ar.largest() == N && ar.used() == 0 && ar.free_blocks() == 1);
    std::vector<int> owner(N / A, -1);       // independent map: cell -> live allocation
    struct Live { size_t off, bytes; };
    std::vector<Live> live;
    std::mt19937_64 rng(12345);
    for (int step = 0; step < 20000; ++step) {
        const bool take = live.empty() || rng() % 3 != 0;
        if (take) {
            const size_t bytes = 1 + rng() % (8 * A);
            const size_t cells = (bytes + A - 1) / A;
            // what first fit must return: the lowest run of `cells` free cells
            long expect = -1;
            for (size_t c = 0, run = 0; c < owner.size(); ++c) {
                run = owner[c] < 0 ? run + 1 : 0;
                if (run == cells) { expect = (long)(c + 1 - cells); break; }
            }
            size_t off = 0;
            const bool ok = ar.alloc(bytes, off);
            CHECK(ok == (expect >= 0));
            if (!ok) continue;
            CHECK(off % A == 0 && off + cells * A <= N);
            CHECK((long)(off / A) == expect);
            for (size_t c = off / A; c < off / A + cells; ++c) {
                CHECK(owner[c] < 0);
                owner[c] = (int)live.size();
            }
            live.push_back({off, bytes});
        } else {
            const size_t k = rng() % live.size();
            const Live l = live[k];
            ar.release(l.off, l.bytes);
            for (size_t c = l.off / A; c < l.off / A + (l.bytes + A - 1) / A; ++c) owner[c] = -1;
            live[k] = live.back();
            live.pop_back();
            for (size_t c = 0; c < owner.size(); ++c)   // renumber the moved allocation
                if (owner[c] == (int)live.size()) owner[c] = (int)k;
        }
        size_t used = 0;
        for (const Live &l : live) used += (l.bytes + A - 1) / A * A;
        CHECK(ar.used() == used);
    }
    for (const Live &l : live) ar.release(l.off, l.bytes);
    CHECK(ar.used() == 0 && ar.free_blocks() == 1 && ar.largest() == N);
    std::printf("arena ok\n");
    return 0;
}
