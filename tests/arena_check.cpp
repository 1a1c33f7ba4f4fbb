// Randomized check of the serving arena's first-fit allocator against a
// byte-map model: blocks never overlap, stay inside the capacity, are
// aligned, the used count matches, the allocator refuses only when no free
// run of the rounded size exists, and freeing everything leaves one block.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "arena.h"

int main(int argc, char** argv)
{
    const unsigned seed = argc > 1 ? (unsigned)atoi(argv[1]) : 1u;
    srand(seed);
    const size_t cap = 256 * 1024;
    const size_t A = glcm_arena::Arena::kAlign;
    glcm_arena::Arena ar;
    ar.reset(cap);
    std::vector<unsigned char> owner(cap / A, 0);  // 1 = in use, per 256-byte unit
    struct Blk { size_t off, bytes; };
    std::vector<Blk> live;
    size_t used = 0;
    for (int step = 0; step < 20000; ++step) {
        if (!live.empty() && (rand() % 100) < 45) {
            const size_t k = rand() % live.size();
            const Blk b = live[k];
            live[k] = live.back();
            live.pop_back();
            const size_t units = glcm_arena::Arena::round_up(b.bytes) / A;
            for (size_t u = 0; u < units; ++u)
                owner[b.off / A + u] = 0;
            used -= units * A;
            ar.release(b.off, b.bytes);
        } else {
            const size_t bytes = 1 + (size_t)(rand() % 20000);
            const size_t units = glcm_arena::Arena::round_up(bytes) / A;
            // First free run of `units` in the model.
            size_t run = 0, first = (size_t)-1;
            for (size_t u = 0; u < owner.size(); ++u) {
                run = owner[u] ? 0 : run + 1;
                if (run == units) {
                    first = u + 1 - units;
                    break;
                }
            }
            size_t off = 0;
            const bool ok = ar.alloc(bytes, &off);
            if (ok != (first != (size_t)-1)) {
                printf("FAIL step %d: alloc(%zu) returned %d, model says %d\n", step, bytes, (int)ok,
                       (int)(first != (size_t)-1));
                return 1;
            }
            if (!ok)
                continue;
            if (off != first * A || off % A || off + units * A > cap) {
                printf("FAIL step %d: offset %zu, first fit %zu\n", step, off, first * A);
                return 1;
            }
            for (size_t u = 0; u < units; ++u)
                owner[off / A + u] = 1;
            used += units * A;
            live.push_back({off, bytes});
        }
        if (ar.used() != used) {
            printf("FAIL step %d: used %zu, model %zu\n", step, ar.used(), used);
            return 1;
        }
    }
    for (const Blk& b : live)
        ar.release(b.off, b.bytes);
    if (ar.used() != 0 || ar.free_blocks() != 1 || ar.largest_free() != cap) {
        printf("FAIL: after freeing all, used %zu, %zu free blocks, largest %zu\n", ar.used(), ar.free_blocks(),
               ar.largest_free());
        return 1;
    }
    printf("OK peak %zu\n", ar.peak());
    return 0;
}
