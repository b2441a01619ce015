// pt_philox.cuh -- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) for the kernels.
//
// philox10() is the generator as published: 10 rounds, each two 32x32->64
// multiplies (M0 on word 0, M1 on word 2) whose high halves are xor-ed with the
// other two words and the round key, the key advancing by the Weyl constants
// W0, W1 between rounds.
//
// The Metropolis draws use counter (sweep, run << 16 | slot, group, 0): within
// one sweep a thread keeps its group and walks over slots, so only word 1
// changes.  philox_pre()/philox_slot() split the same computation so that every
// product whose inputs do not depend on the slot is formed once per sweep:
// round 0 needs no multiply per slot, rounds 1 and 2 one each.  The output is
// identical to philox10() (checked on the host against the plain form).
#pragma once
#include <cstdint>

namespace ptg {

constexpr uint32_t PHILOX_M0 = 0xD2511F53u;
constexpr uint32_t PHILOX_M1 = 0xCD9E8D57u;
constexpr uint32_t PHILOX_W0 = 0x9E3779B9u;
constexpr uint32_t PHILOX_W1 = 0xBB67AE85u;

__host__ __device__ __forceinline__ uint4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                   uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)PHILOX_M0 * c0;
        const uint64_t p1 = (uint64_t)PHILOX_M1 * c2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        c1 = (uint32_t)p1;
        c3 = (uint32_t)p0;
        c0 = n0;
        c2 = n2;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    return make_uint4(c0, c1, c2, c3);
}

// Slot-independent part of the counter (s, *, g, 0) under key (k0, k1).
struct PhiloxPre {
    uint32_t x0b;   // round-0 output word 0 without the slot word
    uint32_t y2x;   // round-1 term xor-ed into word 2
    uint32_t y1k;   // round-2 term xor-ed into word 0
    uint32_t z2x;   // round-2 term xor-ed into word 2
    uint32_t z3;    // round-2 output word 3
};

__host__ __device__ __forceinline__ PhiloxPre philox_pre(uint32_t s, uint32_t g, uint32_t k0, uint32_t k1)
{
    const uint64_t A = (uint64_t)PHILOX_M0 * s;            // round 0, word 0
    const uint64_t B = (uint64_t)PHILOX_M1 * g;            // round 0, word 2
    const uint32_t x1 = (uint32_t)B;
    const uint32_t x2 = (uint32_t)(A >> 32) ^ k1;          // word 3 of the counter is 0
    const uint32_t x3 = (uint32_t)A;
    const uint64_t D = (uint64_t)PHILOX_M1 * x2;           // round 1, word 2
    const uint32_t y0 = (uint32_t)(D >> 32) ^ x1 ^ (k0 + PHILOX_W0);
    const uint32_t y1 = (uint32_t)D;
    const uint64_t E = (uint64_t)PHILOX_M0 * y0;           // round 2, word 0
    PhiloxPre p;
    p.x0b = (uint32_t)(B >> 32) ^ k0;
    p.y2x = x3 ^ (k1 + PHILOX_W1);
    p.y1k = y1 ^ (k0 + 2u * PHILOX_W0);
    p.z2x = (uint32_t)(E >> 32) ^ (k1 + 2u * PHILOX_W1);
    p.z3 = (uint32_t)E;
    return p;
}

// Output of philox10(s, c1, g, 0, k0, k1) given philox_pre(s, g, k0, k1).
__host__ __device__ __forceinline__ uint4 philox_slot(const PhiloxPre& p, uint32_t c1, uint32_t k0,
                                                      uint32_t k1)
{
    const uint32_t x0 = p.x0b ^ c1;
    const uint64_t C = (uint64_t)PHILOX_M0 * x0;           // round 1, word 0
    const uint32_t y2 = (uint32_t)(C >> 32) ^ p.y2x;
    const uint32_t y3 = (uint32_t)C;
    const uint64_t F = (uint64_t)PHILOX_M1 * y2;           // round 2, word 2
    uint32_t a0 = (uint32_t)(F >> 32) ^ p.y1k;
    uint32_t a1 = (uint32_t)F;
    uint32_t a2 = p.z2x ^ y3;
    uint32_t a3 = p.z3;
    k0 += 3u * PHILOX_W0;
    k1 += 3u * PHILOX_W1;
#pragma unroll
    for (int r = 3; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)PHILOX_M0 * a0;
        const uint64_t p1 = (uint64_t)PHILOX_M1 * a2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ a1 ^ k0;
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ a3 ^ k1;
        a1 = (uint32_t)p1;
        a3 = (uint32_t)p0;
        a0 = n0;
        a2 = n2;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    return make_uint4(a0, a1, a2, a3);
}

// The same counter (s, c1, g, 0) when a thread keeps the slot word c1 and
// walks over groups g: the products of round 0 word 0 and round 1 word 2
// depend on neither g nor c1 and are formed once per sweep; round 0's word-2
// product depends on g alone and comes from the caller.
struct PhiloxSweep {
    uint32_t y0k;   // round-1 high product of word 2, xor round-1 key word 0
    uint32_t y1;    // round-1 low product of word 2
    uint32_t x3k;   // round-0 low product of word 0, xor round-1 key word 1
};

__host__ __device__ __forceinline__ PhiloxSweep philox_sweep_pre(uint32_t s, uint32_t k0, uint32_t k1)
{
    const uint64_t A = (uint64_t)PHILOX_M0 * s;            // round 0, word 0
    const uint32_t x2 = (uint32_t)(A >> 32) ^ k1;          // counter word 3 is 0
    const uint64_t D = (uint64_t)PHILOX_M1 * x2;           // round 1, word 2
    PhiloxSweep p;
    p.y0k = (uint32_t)(D >> 32) ^ (k0 + PHILOX_W0);
    p.y1 = (uint32_t)D;
    p.x3k = (uint32_t)A ^ (k1 + PHILOX_W1);
    return p;
}

// Output of philox10(s, c1, g, 0, k0, k1) given philox_sweep_pre(s, k0, k1) and
// round 0's word-2 product M1 * g as its high and low halves (bh, bl): a
// thread that visits the same groups every sweep can keep that product.
__host__ __device__ __forceinline__ uint4 philox_group_prod(const PhiloxSweep& p, uint32_t c1, uint32_t bh,
                                                            uint32_t bl, uint32_t k0, uint32_t k1)
{
    const uint32_t x0 = bh ^ c1 ^ k0;
    const uint64_t C = (uint64_t)PHILOX_M0 * x0;           // round 1, word 0
    uint32_t a0 = p.y0k ^ bl;
    uint32_t a1 = p.y1;
    uint32_t a2 = (uint32_t)(C >> 32) ^ p.x3k;
    uint32_t a3 = (uint32_t)C;
    k0 += 2u * PHILOX_W0;
    k1 += 2u * PHILOX_W1;
#pragma unroll
    for (int r = 2; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)PHILOX_M0 * a0;
        const uint64_t p1 = (uint64_t)PHILOX_M1 * a2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ a1 ^ k0;
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ a3 ^ k1;
        a1 = (uint32_t)p1;
        a3 = (uint32_t)p0;
        a0 = n0;
        a2 = n2;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    return make_uint4(a0, a1, a2, a3);
}

}  // namespace ptg
