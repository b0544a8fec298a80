// Host check of the bracket histogram's bin layout (binmap.cuh): over many
// random brackets (half of them crossing key 0), the bins tile [p1, p2] in
// order without gaps, every key maps to the bin whose range holds it, the
// crossing layout starts a bin at key 0, and "the keys G below and above
// share a bin" is the same test as "G away from both edges of the bin"; the
// same for the aligned layout of the 32-bit selection (BinMapA), whose test
// may only be more cautious than the edges.
#include <cstdio>
#include <cstdint>

#include "../../paper_2402_16712_gb300/csrc/binmap.cuh"

using l1l::BinMap;
using l1l::CK0;

static uint64_t rng_state = 0x9E3779B97F4A7C15ull;
static uint32_t next32() {  // xorshift64*
    rng_state ^= rng_state >> 12;
    rng_state ^= rng_state << 25;
    rng_state ^= rng_state >> 27;
    return (uint32_t)((rng_state * 0x2545F4914F6CDD1Dull) >> 32);
}

static int check(uint32_t p1, uint32_t p2) {
    BinMap bm;
    bm.init(p1, p2, 64);
    const int nb = bm.nbins();
    if (nb < 1 || nb > 64) return 1;
    uint64_t prev = (uint64_t)p1 - 1;  // p1 = 0: 2^64 - 1, and prev + 1 wraps to 0
    for (int b = 0; b < nb; ++b) {
        const uint32_t lo = bm.lower(b), hi = bm.upper(b);
        if (lo > hi) return 2;
        if ((uint64_t)lo != prev + 1) return 3;
        prev = hi;
        const uint32_t probes[3] = {lo, hi, lo + (hi - lo) / 2};
        for (uint32_t kk : probes)
            if (bm.bin(kk) != b) return 4;
    }
    if (prev != p2) return 5;
    if (bm.cross && (bm.lower(bm.n0) != CK0 || bm.upper(bm.n0 - 1) != CK0 - 1u)) return 6;
    const uint32_t G = 8;
    for (int t = 0; t < 16; ++t) {
        if (p2 - p1 < 2 * G + 1) break;
        const uint32_t kk = p1 + G + next32() % (p2 - p1 - 2 * G + 1);
        const int b = bm.bin(kk);
        const bool edges = kk - bm.lower(b) >= G && bm.upper(b) - kk >= G;
        const bool same = bm.bin(kk - G) == bm.bin(kk + G);
        if (edges != same) return 7;
    }
    return 0;
}

// The aligned layout of the 32-bit selection (BinMapA): the same tiling
// checks, and same() never calls a key clear that sits within G of an edge
// (it may call a key next to a non-edge multiple of 2^21 unclear).
static int check_a(uint32_t p1, uint32_t p2) {
    l1l::BinMapA bm;
    bm.init(p1, p2);
    const int nb = bm.nbins();
    if (nb < 1 || nb > 64) return 11;
    uint64_t prev = (uint64_t)p1 - 1;
    for (int b = 0; b < nb; ++b) {
        const uint32_t lo = bm.lower(b), hi = bm.upper(b);
        if (lo > hi) return 12;
        if ((uint64_t)lo != prev + 1) return 13;
        prev = hi;
        const uint32_t probes[3] = {lo, hi, lo + (hi - lo) / 2};
        for (uint32_t kk : probes)
            if (bm.bin(kk) != b) return 14;
    }
    if (prev != p2) return 15;
    if (bm.cross && (bm.lower(bm.nneg) != CK0 || bm.upper(bm.nneg - 1) != CK0 - 1u)) return 16;
    const uint32_t G = 8;
    for (int t = 0; t < 24; ++t) {
        if (p2 - p1 < 2 * G + 1) break;
        uint32_t kk = p1 + G + next32() % (p2 - p1 - 2 * G + 1);
        if (t & 1) {  // next to a bin edge
            const int b = (int)(next32() % (uint32_t)nb);
            kk = bm.lower(b) + (next32() % (2 * G + 1)) - G;
            if (kk < p1 + G || kk > p2 - G) continue;
        }
        const int b = bm.bin(kk);
        const bool edges = kk - bm.lower(b) >= G && bm.upper(b) - kk >= G;
        if (bm.same(kk, G) && !edges) return 17;
        if (!bm.cross && bm.same(kk, G) != edges) return 18;
    }
    return 0;
}

int main() {
    int crossing = 0, bad = 0;
    const uint32_t fixed[][2] = {{0u, 0xFFFFFFFEu}, {CK0 - 5u, CK0}, {CK0 - 1u, CK0 + 1u},
                                 {CK0 - (200u << 23), CK0 + (180u << 23)},
                                 {CK0 - (40u << 21), CK0 + (40u << 21)},
                                 {CK0 - (70u << 21), CK0}, {CK0 - 1u, CK0 + (70u << 21)},
                                 {5u, 5u}, {CK0, CK0}};
    for (const auto &f : fixed) {
        const int r = check(f[0], f[1]) | check_a(f[0], f[1]);
        if (r) {
            std::printf("FAIL %d at [%08x, %08x]\n", r, f[0], f[1]);
            ++bad;
        }
    }
    for (int t = 0; t < 200000; ++t) {
        uint32_t a = next32(), b = next32();
        if (t & 1) {  // a bracket around key 0
            a = next32() % CK0;
            b = CK0 + next32() % (0xFFFFFFFFu - CK0);
        }
        const uint32_t p1 = a < b ? a : b, p2 = a < b ? b : a;
        BinMap bm;
        bm.init(p1, p2, 64);
        crossing += bm.cross ? 1 : 0;
        int r = check(p1, p2);
        if (!r) r = check_a(p1, p2);
        if (r) {
            if (bad < 10) std::printf("FAIL %d at [%08x, %08x]\n", r, p1, p2);
            ++bad;
        }
    }
    std::printf("brackets 200009 crossing %d failures %d\n", crossing, bad);
    return bad ? 1 : 0;
}
