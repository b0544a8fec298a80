// select32.cuh -- the weighted median of one (jhat, k) pair for float input on
// 32-bit fixed-point weights (Lemma 1, decided exactly).
//
// Same plan as the 64-bit selection in pairs.cuh (sample bracket, one pass
// over the rows, exact histogram of the bracket, list levels, final rank
// test), with a cheaper inner loop:
//   * weights are q32_i = floor(|x_ijhat| 2^s32) with the column total below
//     2^32 (ColInfo::Q32), so every partial sum is one 32-bit add and a bin of
//     the bracket histogram takes one 32-bit shared atomic;
//   * a lane owns four consecutive rows per 128-row group: x_ik, 1/x_ijhat
//     and q32 arrive with one 128-bit load each;
//   * rows are classified by float compares of the approximate ratio against
//     bounds G keys outside the pivots (no key arithmetic per row), and a
//     candidate is stored as one 8-byte entry (ratio bits, row) by a pointer
//     that advances only for candidates.
// Truncating the weights to 32 bits widens the certainty band of the exact
// test (Decide, e = n_inexact32); a decision inside the band, a lane whose
// candidate quota overflows, or a bracket that keeps missing returns SEL_W64,
// and the caller repeats the pair on 64-bit weights.
#pragma once
#include <cstdint>

#include "binmap.cuh"
#include "checks.cuh"
#include "common.cuh"

// Unroll factors of the level-0 row loop and of the candidate-list loops,
// set per launch shape by the file that instantiates the kernels (measured:
// unrolling the level-0 loop by two helps the 64- and 80-register shapes and
// hurts the 128-register one, unrolling the list loops the reverse).
#ifndef L1L_L0_UNROLL
#define L1L_L0_UNROLL 1
#endif
#ifndef L1L_LIST_UNROLL
#define L1L_LIST_UNROLL 1
#endif
// Lane balancing of the candidate lists after each level-0 pass
// (list32_balance), chosen per launch shape like the unroll factors.
#ifndef L1L_BALANCE
#define L1L_BALANCE 0
#endif
// Warps of a CTA take their pairs from a shared counter (pairs_unit); 0: a
// fixed share per warp.
#ifndef L1L_DYNAMIC_K
#define L1L_DYNAMIC_K 1
#endif
#define L1L_PRAGMA(x) _Pragma(#x)
#define L1L_UNROLL(n) L1L_PRAGMA(unroll n)

namespace l1l {

// Candidate entry: x = float bits of the approximate ratio, or (KEYED) its
// coarse key; y = row | flags.  EXACT: the key is the coarse key of the
// correctly rounded ratio.
constexpr uint32_t E32_EXACT = 1u << 31;
constexpr uint32_t E32_KEYED = 1u << 30;
constexpr uint32_t E32_PEND = 1u << 29;  // histogram pass A: exact key still needed
constexpr uint32_t E32_ROW = (1u << 29) - 1u;
constexpr int XB32 = 64;                 // bins of the 32-bit bracket histogram
constexpr int SEL_W64 = 16;              // repeat this pair on 64-bit weights

// Float value of a key of akey's order (-0 just below +0).
__device__ __forceinline__ float akey_value(uint32_t k) {
    const uint32_t u = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
    return __uint_as_float(u);
}
// r < key_lo_bound(k)  implies  akey(r) < k   (NaN r: false)
__device__ __forceinline__ float key_lo_bound(uint32_t k) {
    return k <= 0x007FFFFFu ? -__int_as_float(0x7F800000) : akey_value(k);
}
// r > key_hi_bound(k)  implies  akey(r) > k   (NaN r: false)
__device__ __forceinline__ float key_hi_bound(uint32_t k) {
    return k >= 0xFF800000u ? __int_as_float(0x7F800000) : akey_value(k);
}

// Shared-memory accesses by 32-bit shared-window address, so that they stay
// shared-memory instructions (not generic ones) whatever the inlining.
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void st_shared_v2_if(bool ok, uint32_t addr, uint32_t a, uint32_t b) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %0, 0;\n\t@p st.shared.v2.u32 [%1], {%2, %3};\n\t}" ::
            "r"((int)ok),
        "r"(addr), "r"(a), "r"(b)
        : "memory");
}
__device__ __forceinline__ void st_shared_v2(uint32_t addr, uint32_t a, uint32_t b) {
    asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(addr), "r"(a), "r"(b) : "memory");
}
__device__ __forceinline__ void st_shared_u32(uint32_t addr, uint32_t a) {
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(addr), "r"(a) : "memory");
}
__device__ __forceinline__ uint2 ld_shared_v2(uint32_t addr) {
    uint2 v;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_shared_u32(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ float ld_shared_f32(uint32_t addr) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ float4 ld_shared_v4f(uint32_t addr) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(addr)
                 : "memory");
    return v;
}
__device__ __forceinline__ uint4 ld_shared_v4u(uint32_t addr) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(addr)
                 : "memory");
    return v;
}
__device__ __forceinline__ void red_shared_add(uint32_t addr, uint32_t v) {
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void red_shared_add_if(bool ok, uint32_t addr, uint32_t v) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %0, 0;\n\t@p red.shared.add.u32 [%1], %2;\n\t}" ::"r"(
            (int)ok),
        "r"(addr), "r"(v)
        : "memory");
}
__device__ __forceinline__ void st_shared_u32_if(bool ok, uint32_t addr, uint32_t v) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %0, 0;\n\t@p st.shared.u32 [%1], %2;\n\t}" ::"r"(
            (int)ok),
        "r"(addr), "r"(v)
        : "memory");
}
// One row of the level-0 pass: r = x * (1/x_ijhat); below (r < fb): add the
// row's weight to Sb; candidate (fb <= r <= fa): store (r, row) at the lane's
// next slot sp while sp < lend, and advance sp by one slot row (256 bytes)
// either way, so that an overflow shows in the count.  NaN r (x_ijhat = 0, a
// padding row) is neither.  Nine predicated instructions, no branch.
__device__ __forceinline__ void level0_row(float x, float iv, uint32_t q, uint32_t row, float fb,
                                           float fa, uint32_t lend, uint32_t &Sb, uint32_t &sp) {
    asm volatile(
        "{\n\t"
        ".reg .pred pb, pc, po;\n\t"
        ".reg .f32 r;\n\t"
        ".reg .b32 rb;\n\t"
        "mul.rn.f32 r, %2, %3;\n\t"
        "setp.lt.f32 pb, r, %4;\n\t"
        "setp.ge.f32 pc, r, %4;\n\t"
        "setp.le.and.f32 pc, r, %5, pc;\n\t"
        "@pb add.u32 %0, %0, %6;\n\t"
        "setp.lt.and.u32 po, %1, %7, pc;\n\t"
        "mov.b32 rb, r;\n\t"
        "@po st.shared.v2.b32 [%1], {rb, %8};\n\t"
        "@pc add.u32 %1, %1, 256;\n\t"
        "}"
        : "+r"(Sb), "+r"(sp)
        : "f"(x), "f"(iv), "f"(fb), "f"(fa), "r"(q), "r"(lend), "r"(row)
        : "memory");
}

// One 128-row group of the level-0 pass for this lane's four consecutive rows
// i0 .. i0+3 (x: their x_ik): the staged 1/x_ijhat and q32 of the four rows
// come with one 128-bit shared load each (ainv, aq: their shared addresses),
// then each row as in level0_row: below (r < fb) adds q to Sb; a candidate
// (not below, r <= fa, so not NaN) is stored at sp while sp < lend and
// advances sp by one slot row.
__device__ __forceinline__ void level0_group(float4 x, uint32_t ainv, uint32_t aq, uint32_t i0,
                                             float fb, float fa, uint32_t lend, uint32_t &Sb,
                                             uint32_t &sp) {
    asm volatile(
        "{\n\t"
        ".reg .pred pb, pc, po;\n\t"
        ".reg .f32 r, v0, v1, v2, v3;\n\t"
        ".reg .b32 q0, q1, q2, q3, rb, rid;\n\t"
        "ld.shared.v4.f32 {v0, v1, v2, v3}, [%2];\n\t"
        "ld.shared.v4.u32 {q0, q1, q2, q3}, [%3];\n\t"
        // row 0
        "mul.rn.f32 r, %4, v0;\n\t"
        "setp.lt.f32 pb, r, %8;\n\t"
        "setp.le.and.f32 pc, r, %9, !pb;\n\t"
        "@pb add.u32 %0, %0, q0;\n\t"
        "setp.lt.and.u32 po, %1, %10, pc;\n\t"
        "mov.b32 rb, r;\n\t"
        "@po st.shared.v2.b32 [%1], {rb, %11};\n\t"
        "@pc add.u32 %1, %1, 256;\n\t"
        // row 1
        "mul.rn.f32 r, %5, v1;\n\t"
        "setp.lt.f32 pb, r, %8;\n\t"
        "setp.le.and.f32 pc, r, %9, !pb;\n\t"
        "@pb add.u32 %0, %0, q1;\n\t"
        "setp.lt.and.u32 po, %1, %10, pc;\n\t"
        "mov.b32 rb, r;\n\t"
        "add.u32 rid, %11, 1;\n\t"
        "@po st.shared.v2.b32 [%1], {rb, rid};\n\t"
        "@pc add.u32 %1, %1, 256;\n\t"
        // row 2
        "mul.rn.f32 r, %6, v2;\n\t"
        "setp.lt.f32 pb, r, %8;\n\t"
        "setp.le.and.f32 pc, r, %9, !pb;\n\t"
        "@pb add.u32 %0, %0, q2;\n\t"
        "setp.lt.and.u32 po, %1, %10, pc;\n\t"
        "mov.b32 rb, r;\n\t"
        "add.u32 rid, %11, 2;\n\t"
        "@po st.shared.v2.b32 [%1], {rb, rid};\n\t"
        "@pc add.u32 %1, %1, 256;\n\t"
        // row 3
        "mul.rn.f32 r, %7, v3;\n\t"
        "setp.lt.f32 pb, r, %8;\n\t"
        "setp.le.and.f32 pc, r, %9, !pb;\n\t"
        "@pb add.u32 %0, %0, q3;\n\t"
        "setp.lt.and.u32 po, %1, %10, pc;\n\t"
        "mov.b32 rb, r;\n\t"
        "add.u32 rid, %11, 3;\n\t"
        "@po st.shared.v2.b32 [%1], {rb, rid};\n\t"
        "@pc add.u32 %1, %1, 256;\n\t"
        "}"
        : "+r"(Sb), "+r"(sp)
        : "r"(ainv), "r"(aq), "f"(x.x), "f"(x.y), "f"(x.z), "f"(x.w), "f"(fb), "f"(fa),
          "r"(lend), "r"(i0)
        : "memory");
}

// Read-only global loads (the column copies do not change during a launch).
__device__ __forceinline__ float4 ldg_f4(const float *p) {
    return __ldg(reinterpret_cast<const float4 *>(p));
}

// One slot of the candidate histogram's pass A (select_w32; G: the guard
// band in keys), zero-crossing bin layout (BinMapA, cross: bins of 2^21
// keys): entry (ratio bits, row) at eaddr; act: the slot holds a
// candidate of this lane.  A candidate whose approximate key lies G inside
// [g1 - G, g2 + G] and G inside its bin's edges adds its weight q32[row] to
// its bin; any other candidate is flagged pending.  pend |= 1 for a pending
// candidate.  Branch-free, about 30 instructions.
template <uint32_t G>
__device__ __forceinline__ void passa_slot_cross(uint32_t eaddr, int act, uint32_t g1, uint32_t g2,
                                                 int tp1, int tp2, int nneg1, int npos1, int nb1,
                                                 uint32_t aq, uint32_t ahist, int &pend) {
    asm volatile(
        "{\n\t"
        ".reg .pred pa, pc, pj, pn;\n\t"
        ".reg .b32 ex, ey, s, kk, a, b, t, dn, dp, bn, q, qa, ha, ey2, row;\n\t"
        "setp.ne.b32 pa, %1, 0;\n\t"
        "ld.shared.v2.u32 {ex, ey}, [%2];\n\t"
        "shr.s32 s, ex, 31;\n\t"
        "or.b32 s, s, 0x80000000;\n\t"
        "xor.b32 kk, ex, s;\n\t"
        "setp.ge.and.u32 pc, kk, %3, pa;\n\t"
        "setp.le.and.u32 pc, kk, %4, pc;\n\t"
        "sub.u32 a, kk, %12;\n\t"
        "add.u32 b, kk, %12;\n\t"
        "shr.u32 a, a, 21;\n\t"
        "shr.u32 b, b, 21;\n\t"
        "setp.eq.and.u32 pc, a, b, pc;\n\t"
        "shr.u32 t, kk, 21;\n\t"
        "sub.s32 dn, t, %5;\n\t"
        "min.s32 dn, dn, %7;\n\t"
        "sub.s32 dp, %6, t;\n\t"
        "min.s32 dp, dp, %8;\n\t"
        "sub.s32 bn, %9, dp;\n\t"
        "setp.lt.u32 pn, kk, 0x80000000;\n\t"
        "selp.b32 bn, dn, bn, pn;\n\t"
        "selp.b32 row, ey, 0, pa;\n\t"
        "shl.b32 qa, row, 2;\n\t"
        "add.u32 qa, qa, %10;\n\t"
        "ld.shared.u32 q, [qa];\n\t"
        "shl.b32 ha, bn, 2;\n\t"
        "add.u32 ha, ha, %11;\n\t"
        "@pc red.shared.add.u32 [ha], q;\n\t"
        "not.pred pj, pc;\n\t"
        "and.pred pj, pj, pa;\n\t"
        "or.b32 ey2, ey, 0x20000000;\n\t"
        "@pj st.shared.u32 [%2+4], ey2;\n\t"
        "selp.b32 s, 1, 0, pj;\n\t"
        "or.b32 %0, %0, s;\n\t"
        "}"
        : "+r"(pend)
        : "r"(act), "r"(eaddr), "r"(g1), "r"(g2), "r"(tp1), "r"(tp2), "r"(nneg1), "r"(npos1),
          "r"(nb1), "r"(aq), "r"(ahist), "n"(G)
        : "memory");
}

// The same for the uniform layout: bin (kk - base) >> sh.
template <uint32_t G>
__device__ __forceinline__ void passa_slot_unif(uint32_t eaddr, int act, uint32_t g1, uint32_t g2,
                                                uint32_t base, uint32_t sh, uint32_t aq,
                                                uint32_t ahist, int &pend) {
    asm volatile(
        "{\n\t"
        ".reg .pred pa, pc, pj;\n\t"
        ".reg .b32 ex, ey, s, kk, a, b, d, q, qa, ha, ey2, row;\n\t"
        "setp.ne.b32 pa, %1, 0;\n\t"
        "ld.shared.v2.u32 {ex, ey}, [%2];\n\t"
        "shr.s32 s, ex, 31;\n\t"
        "or.b32 s, s, 0x80000000;\n\t"
        "xor.b32 kk, ex, s;\n\t"
        "setp.ge.and.u32 pc, kk, %3, pa;\n\t"
        "setp.le.and.u32 pc, kk, %4, pc;\n\t"
        "sub.u32 d, kk, %5;\n\t"
        "sub.u32 a, d, %9;\n\t"
        "add.u32 b, d, %9;\n\t"
        "shr.u32 a, a, %6;\n\t"
        "shr.u32 b, b, %6;\n\t"
        "setp.eq.and.u32 pc, a, b, pc;\n\t"
        "shr.u32 d, d, %6;\n\t"
        "selp.b32 row, ey, 0, pa;\n\t"
        "shl.b32 qa, row, 2;\n\t"
        "add.u32 qa, qa, %7;\n\t"
        "ld.shared.u32 q, [qa];\n\t"
        "shl.b32 ha, d, 2;\n\t"
        "add.u32 ha, ha, %8;\n\t"
        "@pc red.shared.add.u32 [ha], q;\n\t"
        "not.pred pj, pc;\n\t"
        "and.pred pj, pj, pa;\n\t"
        "or.b32 ey2, ey, 0x20000000;\n\t"
        "@pj st.shared.u32 [%2+4], ey2;\n\t"
        "selp.b32 s, 1, 0, pj;\n\t"
        "or.b32 %0, %0, s;\n\t"
        "}"
        : "+r"(pend)
        : "r"(act), "r"(eaddr), "r"(g1), "r"(g2), "r"(base), "r"(sh), "r"(aq), "r"(ahist),
          "n"(G)
        : "memory");
}

// First bin of [base, top] (bins of 2^sh keys) whose upper key passes the
// exact test with S = Sbase + weight of bins <= b, over 32-bit bins.
// Returns the bin (-1: none passes, -2: undecidable) and the weight below it.
__device__ __forceinline__ int hist32_cross(const uint32_t *h, const BinMapA *bm, int nbins,
                                            uint32_t base, uint32_t top, int sh, int64_t Sbase,
                                            const Decide &dc, int64_t *below, int lane) {
    const unsigned FULL = 0xFFFFFFFFu;
    const int b0 = 2 * lane, b1 = 2 * lane + 1;
    const uint32_t s0 = b0 < nbins ? h[L1L_CHK(b0, XB32)] : 0u;
    const uint32_t s1 = b1 < nbins ? h[L1L_CHK(b1, XB32)] : 0u;
    uint32_t incl = s0 + s1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
    }
    const int64_t ex = (int64_t)(incl - s0 - s1);
    auto bhi = [&](int b) -> uint32_t {
        if (bm) return bm->upper(b);
        const uint64_t v = (uint64_t)base + ((uint64_t)(b + 1) << sh) - 1;
        return v > top ? top : (uint32_t)v;
    };
    const int c0 = b0 < nbins ? dc.cond(Sbase + ex + s0, bhi(b0) >= CK0) : 0;
    const int c1 = b1 < nbins ? dc.cond(Sbase + ex + s0 + s1, bhi(b1) >= CK0) : 0;
    const unsigned m0 = __ballot_sync(FULL, c0 != 0), m1 = __ballot_sync(FULL, c1 != 0);
    const unsigned any = m0 | m1;
    if (!any) return -1;
    const int ln = __ffs(any) - 1;
    const bool first_is_b0 = (m0 >> ln) & 1u;
    const int csel = __shfl_sync(FULL, first_is_b0 ? c0 : c1, ln);
    const int64_t bel = __shfl_sync(FULL, first_is_b0 ? ex : ex + (int64_t)s0, ln);
    if (csel < 0) return -2;
    *below = Sbase + bel;
    return 2 * ln + (first_is_b0 ? 0 : 1);
}

// Keeps, lane-locally and in place, the entries whose key lies in [K1, K2]
// (every entry is KEYED afterwards); returns this lane's new count.
__device__ __forceinline__ int list32_keep(uint2 *__restrict__ lst, int cnt, uint32_t K1,
                                           uint32_t K2, int lane, int nslot) {
    // every lane runs to the warp's largest count (no divergent loop exit);
    // slots past a lane's own count are read but not used
    const int cmax = __reduce_max_sync(0xFFFFFFFFu, (unsigned)cnt);
    const uint32_t base = smem_addr(lst) + 8u * (uint32_t)lane;
    int w = 0;
    L1L_UNROLL(L1L_LIST_UNROLL)
    for (int j = 0; j < cmax; ++j) {
        const bool act = j < cnt;
        const uint2 e = lst[L1L_CHK(j * 32 + lane, nslot)];
        const uint32_t kk = (e.y & E32_KEYED) ? e.x : akey(__uint_as_float(e.x));
        st_shared_v2_if(act, base + 256u * (uint32_t)L1L_CHK(w, nslot / 32), kk,
                        e.y | E32_KEYED);  // w <= j
        w += (act & (kk >= K1) & (kk <= K2)) ? 1 : 0;
    }
    return w;
}

// Evens out the lanes' candidate counts in place after a level-0 pass.  The
// rows fall to the lanes by position, so one lane often holds nearly twice
// the warp's mean; pass A, pass B and the keep loop run to the busiest
// lane's count.  With C candidates in the warp and T = ceil(C / 32), a lane
// holding more than T hands its last entries to lanes holding fewer: excess
// entry e (numbered across the lanes in lane order) fills hole e (the free
// slots below T, numbered the same way), so every lane then holds at most T.
// Holes lie below slot T and handed entries at or above it, so no slot is
// both read and written.  tab (XB32 words, free at this point) maps a hole
// to its slot; at most XB32 entries move (the rest stay where they are).
// The order of a lane's entries carries no meaning.  Returns the lane's new
// count.
__device__ __forceinline__ int list32_balance(uint2 *__restrict__ lst, uint32_t *__restrict__ tab,
                                              int cnt, int lane, int nslot) {
    const unsigned FULL = 0xFFFFFFFFu;
    const int C = (int)__reduce_add_sync(FULL, (unsigned)cnt);
    const int T = (C + 31) >> 5;
    const int E = max(cnt - T, 0), D = max(T - cnt, 0);
    // excess in the high half, holes in the low half: both sums stay below
    // 2^16 (at most 32 qt slots)
    const uint32_t pk = ((uint32_t)E << 16) | (uint32_t)D;
    const uint32_t inc = warp_scan_add(pk, lane);
    const int M = min((int)(__shfl_sync(FULL, inc, 31) >> 16), XB32);  // entries that move
    if (M == 0) return cnt;
    const uint32_t ex = inc - pk;
    const int Epre = (int)(ex >> 16), Dpre = (int)(ex & 0xFFFFu);
    const int got = min(max(M - Dpre, 0), D);   // holes of this lane that are filled
    const int gave = min(max(M - Epre, 0), E);  // entries this lane hands over
    for (int u = 0; u < got; ++u)
        tab[L1L_CHK(Dpre + u, XB32)] = (uint32_t)((cnt + u) * 32 + lane);
    __syncwarp();
    for (int t = 0; t < gave; ++t) {
        const uint32_t dst = tab[L1L_CHK(Epre + t, XB32)];
        lst[L1L_CHK((int)dst, nslot)] = lst[L1L_CHK((cnt - 1 - t) * 32 + lane, nslot)];
    }
    __syncwarp();
    return cnt + got - gave;
}

// Weighted median of pair (jhat, k).  xf: column k as float (global, rows
// padded to a multiple of 128 with zeros; the column itself for float input,
// its float copy for double input), read for the approximate keys; xk, colb:
// column k and x_ijhat in the input type (colb shared or global), read for
// the exact divisions; inv, q32: the staged column jhat (shared, padded; inv
// NaN where x_ijhat = 0 and on padding rows, q32 0 there); lst: this warp's
// candidate list (qt entries per lane, lane l's j-th entry at j*32 + l); hist:
// XB32 words.  Keys up to the final step are coarse keys (of the ratio
// rounded to float; the exact key for float input).  Returns SEL_OK with the
// exact key of v_k in tstar, SEL_INTERNAL, or SEL_W64.
template <typename T>
__device__ __forceinline__ int select_w32(const float *__restrict__ xf, const T *__restrict__ xk,
                                          const T *__restrict__ colb,
                                          const float *__restrict__ inv,
                                          const uint32_t *__restrict__ q32,
                                          const uint16_t *__restrict__ samp,
                                          uint2 *__restrict__ lst, uint32_t *__restrict__ hist,
                                          int qt, int n, int d0, const Decide &dc,
                                          typename Traits<T>::K &tstar, int lane) {
    using Tr = Traits<T>;
    using K = typename Tr::K;
    constexpr uint32_t G = Approx<T>::G;  // guard band of the approximate keys
    const unsigned FULL = 0xFFFFFFFFu;
    // exact coarse key of row i
    auto exact_ck = [&](uint32_t i) -> uint32_t {
        return Approx<T>::exact_ck(__ldg(xk + i), colb[i]);
    };
    const float Qf = (float)dc.Q;
    const float hneg0 = 0.5f * (Qf + (float)dc.Lf), hpos0 = 0.5f * (Qf - (float)dc.Lc);
    const int ng = (n + 127) >> 7;  // 128-row groups (rows are padded to them)
    const int nrow = ng * 128;      // rows every staged or copied column holds
    const int nslot = qt * 32;      // candidate slots of this warp's list
    (void)nrow;                     // read by the bounds checks only
    (void)nslot;

    // ---------------- sample bracket ------------------------------------
    uint32_t sk[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int i = L1L_CHK((int)samp[e * 32 + lane], nrow);
        sk[e] = akey(__fmul_rn(__ldg(xf + i), inv[i]));
    }
    warp_sort64(sk, lane);
    int jx;
    {
        const float unit = Qf * (1.0f / 64.0f);
        const bool c0 = (float)(lane + 1) * unit > target_for(sk[0], hneg0, hpos0);
        const bool c1 = (float)(lane + 33) * unit > target_for(sk[1], hneg0, hpos0);
        const unsigned m0 = __ballot_sync(FULL, c0), m1 = __ballot_sync(FULL, c1);
        jx = m0 ? __ffs(m0) - 1 : (m1 ? 32 + __ffs(m1) - 1 : 63);
    }
    auto sample_key = [&](int g) -> uint32_t {
        const uint32_t a0 = __shfl_sync(FULL, sk[0], g & 31);
        const uint32_t a1 = __shfl_sync(FULL, sk[1], g & 31);
        return g < 32 ? a0 : a1;
    };
    uint32_t lo0 = 0, hi0 = CKMAX;  // the median's coarse key lies in [lo0, hi0]
    auto pick = [&](int g, uint32_t dflt) -> uint32_t {
        uint32_t kk = (g < 0 || g > 63) ? dflt : sample_key(g);
        if (kk > CKMAX) kk = dflt;
        return min(max(kk, lo0), hi0);
    };
    // The pivots sit 2G + 1 keys outside the sample keys: a sample row (or any
    // row tied with it) then lies clear of the bracket's guard bands instead of
    // always needing an exact division.
    auto sample_bracket = [&](int d, uint32_t &Q1, uint32_t &Q2) {
        Q1 = max(sat_sub(pick(jx - d, lo0), 2 * G + 1), lo0);
        Q2 = min(sat_add(pick(jx + d, hi0), 2 * G + 1), hi0);
        if (Q1 > Q2) Q1 = Q2;
    };
    uint32_t P1, P2;
    sample_bracket(d0, P1, P2);
    bool sampled = true;
    int dcur = d0;  // half-width of the current sample bracket

    const uint32_t lbase = smem_addr(lst) + (uint32_t)lane * 8u;
    const uint32_t lend = lbase + (uint32_t)qt * 256u;
    const float4 *xk4 = reinterpret_cast<const float4 *>(xf);
    const uint32_t ainv0 = smem_addr(inv) + 16u * (uint32_t)lane;
    const uint32_t aq0 = smem_addr(q32) + 16u * (uint32_t)lane;

    int64_t L = 0;  // exact weight (q32 units) of rows with key < lo
    uint32_t lo = 0, hi = CKMAX;
    int cnt = 0;
    bool placed = false;
    for (int attempt = 0; attempt < 12 && !placed; ++attempt) {
        // ---- one pass over all rows: weight certainly below P1, candidates
        const float fb = key_lo_bound(sat_sub(P1, G));
        const float fa = key_hi_bound(min(sat_add(P2, G), CKMAX));
        uint32_t Sb = 0;
        uint32_t sp = lbase;
        const float4 *xp = xk4 + lane;
        uint32_t ainv = ainv0, aq = aq0, i0 = 4u * (uint32_t)lane;
        float4 xn = __ldg(xp);
        L1L_UNROLL(L1L_L0_UNROLL)
        for (int g = 0; g < ng; ++g) {
            const float4 xc = xn;
            xp += 32;
            if (g + 1 < ng) xn = __ldg(xp);
            level0_group(xc, ainv, aq, i0, fb, fa, lend, Sb, sp);
            ainv += 512u;
            aq += 512u;
            i0 += 128u;
        }
        cnt = (int)((sp - lbase) >> 8);
        Sb = __reduce_add_sync(FULL, Sb);  // < Q32 < 2^32
        __syncwarp();
        if (__any_sync(FULL, cnt > qt)) {
            // a lane overflowed its quota: the bracket holds more rows than its
            // weight share suggests (light rows); halve it around the sample
            // estimate and pass again (the list keeps nothing of this pass)
            if (!sampled || dcur <= 1) return SEL_W64;
            dcur >>= 1;
            sample_bracket(dcur, P1, P2);
            continue;
        }
#if L1L_BALANCE
        cnt = list32_balance(lst, hist, cnt, lane, nslot);
#endif

        // ---- exact histogram of the candidates over the bins of [P1, P2].
        // Pass A: a candidate whose approximate key is at least G inside P1,
        // P2 and its bin's edges has its exact key in that bin: add its weight.
        // The others are marked pending.  Pass B (only when some lane has
        // one): divide them exactly and add them where they fall.
        BinMapA bm;
        bm.init(P1, P2);
        const uint32_t g1 = sat_add(P1, G), g2 = sat_sub(P2, G);
        const uint32_t ahist = smem_addr(hist);
        hist[lane] = 0u;
        hist[lane + 32] = 0u;
        __syncwarp();
        bool pend = false;
        {
            // branch-free body over the warp's largest count (slots past a
            // lane's own count are read but not used, their row clamped to 0)
            const int cmax = __reduce_max_sync(FULL, (unsigned)cnt);
            const uint32_t ebase = smem_addr(lst) + 8u * (uint32_t)lane;
#if L1L_CHECKS
            // the bounds-checked build keeps the loop in C++, where every index is checked
            const int nb1 = bm.nneg + bm.npos - 1, nneg1 = bm.nneg - 1, npos1 = bm.npos - 1;
            L1L_UNROLL(L1L_LIST_UNROLL)
            for (int j = 0; j < cmax; ++j) {
                const bool act = j < cnt;
                const uint2 e = lst[L1L_CHK(j * 32 + lane, nslot)];  // fresh: (ratio bits, row)
                const uint32_t kk = akey(__uint_as_float(e.x));
                const bool clear = act & (kk >= g1) & (kk <= g2) &
                                   (((kk - G - bm.base) >> bm.sh) == ((kk + G - bm.base) >> bm.sh));
                const int t = (int)(kk >> BinMapA::QSH);
                const int dn = min(t - bm.tp1, nneg1), dp = min(bm.tp2 - t, npos1);
                const int bx = kk < CK0 ? dn : nb1 - dp;
                const int bu = (int)((kk - bm.base) >> bm.sh);
                const int b = bm.cross ? bx : bu;
                const uint32_t q = q32[act ? L1L_CHK(e.y, (uint32_t)nrow) : 0u];
                red_shared_add_if(clear, ahist + 4u * (uint32_t)L1L_CHK(clear ? b : 0, XB32), q);
                const bool pj = act & !clear;
                st_shared_u32_if(pj, ebase + 256u * (uint32_t)j + 4u, e.y | E32_PEND);
                pend |= pj;
            }
#else
            // one predicated PTX block per slot (measured 2.8% faster than the same loop in C++)
            static_assert(BinMapA::QSH == 21, "the PTX blocks hold bins of 2^21 keys");
            const uint32_t aq = smem_addr(q32);
            int pendi = 0;
            if (bm.cross) {
                const int nb1 = bm.nneg + bm.npos - 1, nneg1 = bm.nneg - 1, npos1 = bm.npos - 1;
                L1L_UNROLL(L1L_LIST_UNROLL)
                for (int j = 0; j < cmax; ++j)
                    passa_slot_cross<G>(ebase + 256u * (uint32_t)j, j < cnt, g1, g2, bm.tp1, bm.tp2,
                                     nneg1, npos1, nb1, aq, ahist, pendi);
            } else {
                L1L_UNROLL(L1L_LIST_UNROLL)
                for (int j = 0; j < cmax; ++j)
                    passa_slot_unif<G>(ebase + 256u * (uint32_t)j, j < cnt, g1, g2, bm.base,
                                    (uint32_t)bm.sh, aq, ahist, pendi);
            }
            pend = pendi != 0;
#endif
        }
        uint32_t Sb2 = 0;
        if (__any_sync(FULL, pend)) {
            for (int j = 0; j < cnt; ++j) {
                const uint2 e = lst[L1L_CHK(j * 32 + lane, nslot)];
                if (e.y & E32_PEND) {
                    const uint32_t id = L1L_CHK(e.y & E32_ROW, (uint32_t)nrow);
                    const uint32_t kk = exact_ck(id);
                    lst[j * 32 + lane] = make_uint2(kk, id | E32_EXACT | E32_KEYED);
                    const uint32_t q = q32[id];
                    if (kk < P1)
                        Sb2 += q;
                    else if (kk <= P2)
                        red_shared_add(ahist + 4u * (uint32_t)L1L_CHK(bm.bin(kk), XB32), q);
                }
            }
        }
        const int64_t Sbt = (int64_t)Sb + (int64_t)__reduce_add_sync(FULL, Sb2);
        __syncwarp();
        const int r1 = P1 == lo0 ? 0 : dc.cond(Sbt, (P1 - 1) >= CK0);
        if (r1 < 0) return SEL_W64;
        if (r1 == 1) {  // median below P1: retry under P1
            hi0 = P1 - 1;
            P2 = hi0;
            P1 = sampled ? max(sat_sub(pick(jx - 3 * max(dcur, 1) - 1, lo0), 2 * G + 1), lo0) : lo0;
            if (P1 > P2) P1 = lo0;
            continue;
        }
        int64_t below = 0;
        const int bs = hist32_cross(hist, &bm, bm.nbins(), 0, 0, 0, Sbt, dc, &below, lane);
        __syncwarp();
        if (bs == -2) return SEL_W64;
        if (bs < 0) {  // median above P2: retry over P2
            if (P2 >= hi0) return SEL_INTERNAL;
            lo0 = P2 + 1;
            P1 = lo0;
            P2 = sampled ? min(sat_add(pick(jx + 3 * max(dcur, 1) + 1, hi0), 2 * G + 1), hi0) : hi0;
            if (P2 < P1) P2 = hi0;
            continue;
        }
        const uint32_t K1 = bm.lower(bs), K2 = bm.upper(bs);
        cnt = list32_keep(lst, cnt, K1, K2, lane, nslot);
        __syncwarp();
        L = below;
        lo = K1;
        hi = K2;
        placed = true;
        sampled = false;
    }
    if (!placed) return SEL_W64;

    // ---------------- list levels: exact histograms of the survivors -------
    int c = __reduce_add_sync(FULL, cnt);
    for (int level = 0; c > 31 && lo < hi; ++level) {
        if (level >= 8) return SEL_W64;
        const uint32_t span = hi - lo;
        const int sh = span >= (uint32_t)XB32 ? (32 - __clz((int)span)) - 6 : 0;
        const uint32_t bmask = (1u << sh) - 1u;
        const int nbins = (int)(span >> sh) + 1;
        const uint32_t ahist = smem_addr(hist);
        hist[lane] = 0u;
        hist[lane + 32] = 0u;
        __syncwarp();
#pragma unroll 2
        for (int j = 0; j < cnt; ++j) {
            uint2 e = lst[L1L_CHK(j * 32 + lane, nslot)];  // KEYED
            const uint32_t id = L1L_CHK(e.y & E32_ROW, (uint32_t)nrow);
            uint32_t kk = e.x;
            const uint32_t off = (kk - lo) & bmask;
            if (!(e.y & E32_EXACT) && (off < G || off + G > bmask)) {
                kk = exact_ck(id);
                lst[j * 32 + lane] = make_uint2(kk, id | E32_EXACT | E32_KEYED);
            }
            red_shared_add(ahist + 4u * L1L_CHK((kk - lo) >> sh, (uint32_t)XB32), q32[id]);
        }
        __syncwarp();
        int64_t below = 0;
        const int bs = hist32_cross(hist, nullptr, nbins, lo, hi, sh, L, dc, &below, lane);
        __syncwarp();
        if (bs == -2) return SEL_W64;
        if (bs < 0) return SEL_INTERNAL;
        const uint32_t K1 = lo + ((uint32_t)bs << sh);
        const uint32_t K2 = min(hi, K1 + bmask);
        cnt = list32_keep(lst, cnt, K1, K2, lane, nslot);
        __syncwarp();
        L = below;
        lo = K1;
        hi = K2;
        c = __reduce_add_sync(FULL, cnt);
    }

    // ---------------- final: exact keys of the <= 31 candidates -----------
    if constexpr (sizeof(T) == 4) {
        if (lo == hi) {  // coarse keys are the exact keys for float input
            tstar = lo;
            return SEL_OK;
        }
    }
    if (c > 31) {
        // float: lo < hi and the levels stopped, which cannot happen; double:
        // more than 31 rows share one coarse key (the 64-bit selection sorts
        // them out)
        return sizeof(T) == 4 ? SEL_INTERNAL : SEL_W64;
    }
    {
        const int excl = warp_scan_add(cnt, lane) - cnt;
        uint32_t *stage = hist;
        for (int j = 0; j < cnt; ++j)
            stage[L1L_CHK(excl + j, 31)] = lst[L1L_CHK(j * 32 + lane, nslot)].y & E32_ROW;
    }
    __syncwarp();
    const bool zero_in = lo <= CK0 && CK0 <= hi;
    K fk = Tr::NONE;
    uint32_t fq = 0;
    if (lane < c) {
        const uint32_t row = L1L_CHK(hist[lane], (uint32_t)nrow);
        fk = Tr::key(Tr::div_rn(__ldg(xk + row), colb[row]));
        fq = q32[row];
    } else if (lane == c && zero_in) {
        fk = Tr::KEY0;  // the penalty point (0, lambda); lambda sits in the test
    }
    __syncwarp();
    // each candidate's cumulative weight: the weight of candidates with a key
    // at or below its own (equal keys alike); the smallest key that passes
    const int nv = c + (zero_in ? 1 : 0);
    uint32_t S = 0;
    for (int u = 0; u < nv; ++u) {
        const K ku = __shfl_sync(FULL, fk, u);
        const uint32_t qu = __shfl_sync(FULL, fq, u);
        S += ku <= fk ? qu : 0u;
    }
    int r = 0;
    if (lane < nv) r = dc.cond(L + (int64_t)S, fk >= Tr::KEY0);
    K kmin = r != 0 ? fk : Tr::NONE;
    if constexpr (sizeof(T) == 4) {
        kmin = __reduce_min_sync(FULL, kmin);
    } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const K y = __shfl_xor_sync(FULL, kmin, o);
            kmin = y < kmin ? y : kmin;
        }
    }
    if (kmin == Tr::NONE) return SEL_INTERNAL;
    if (__any_sync(FULL, r == -1 && fk == kmin)) return SEL_W64;
    tstar = kmin;
    return SEL_OK;
}

// Residual sum_i |x_ik - v x_ijhat| over the padded rows (padding rows are 0
// in both columns), float input, four consecutive rows per lane per 128-row
// group and four groups per step: the step's sixteen loads are in flight
// together (column k comes from L2, so the pass is bound by load latency, not
// arithmetic); xj in shared memory when XS, else in global memory.
template <bool XS>
__device__ __forceinline__ float warp_residual_f4(const float *__restrict__ xk,
                                                  const float *__restrict__ xj, int n, float v,
                                                  int lane) {
    const int ng = (n + 127) >> 7;
    const float4 *a4 = reinterpret_cast<const float4 *>(xk) + lane;
    const float4 *b4 = reinterpret_cast<const float4 *>(xj) + lane;
    auto ldb = [&](int g) -> float4 {
        if constexpr (XS)
            return b4[g * 32];
        else
            return __ldg(b4 + g * 32);
    };
    float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
    auto add4 = [&](const float4 &a, const float4 &b) {
        acc0 += fabsf(fmaf(-v, b.x, a.x));
        acc1 += fabsf(fmaf(-v, b.y, a.y));
        acc2 += fabsf(fmaf(-v, b.z, a.z));
        acc3 += fabsf(fmaf(-v, b.w, a.w));
    };
    int g = 0;
    for (; g + 3 < ng; g += 4) {
        float4 a[4], b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) a[u] = __ldg(a4 + (g + u) * 32);
#pragma unroll
        for (int u = 0; u < 4; ++u) b[u] = ldb(g + u);
#pragma unroll
        for (int u = 0; u < 4; ++u) add4(a[u], b[u]);
    }
    for (; g < ng; ++g) add4(__ldg(a4 + g * 32), ldb(g));
    float s = (acc0 + acc1) + (acc2 + acc3);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    return s;
}

}  // namespace l1l
