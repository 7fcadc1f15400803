// rs_rng.cuh -- counter-based randomness on the device.
//
// Every random decision is keyed by the subtree it belongs to, so no node
// waits for another (Sec. 3.2: the t-th deviate of subproblem j..k is a hash
// of (j, k, t), a PE's local generator is seeded by its number).  Here the
// keyed source is Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11):
// key = (seed lo, seed hi), counter = (block t, tag, node id lo, node id hi).
#pragma once
#include "rs_common.cuh"

namespace rs {

struct Key2 { uint32_t k0, k1; };

RS_HD Key2 make_key(uint64_t seed) { return Key2{(uint32_t)seed, (uint32_t)(seed >> 32)}; }

// One Philox4x32-10 block: ten rounds of two 32x32->64 multiplies and xors,
// the key bumped by the Weyl constants between rounds.
RS_DEV uint4 philox_block(uint32_t t, uint32_t tag, uint64_t id, Key2 key) {
    uint32_t x0 = t, x1 = tag, x2 = (uint32_t)id, x3 = (uint32_t)(id >> 32);
    uint32_t k0 = key.k0, k1 = key.k1;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        // one 32x32 -> 64 product per multiplier gives both halves
        const uint64_t p0 = (uint64_t)0xD2511F53u * x0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * x2;
        const uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        const uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        x0 = y0; x1 = (uint32_t)p1; x2 = y2; x3 = (uint32_t)p0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return make_uint4(x0, x1, x2, x3);
}

// The same generator with its ten round keys worked out in advance.  A
// kernel whose key is the same for every thread takes them as a kernel
// parameter (__grid_constant__): each round then reads its key from the
// parameter bank instead of bumping two registers.
struct RoundKeys {
    uint32_t k[20];   // round r: k[2r] = k0 + r 0x9E3779B9, k[2r+1] = k1 + r 0xBB67AE85 (mod 2^32)
    RS_HD static RoundKeys of(uint64_t seed) {
        RoundKeys rk;
        const Key2 key = make_key(seed);
        for (int r = 0; r < 10; ++r) {
            rk.k[2 * r] = key.k0 + (uint32_t)r * 0x9E3779B9u;
            rk.k[2 * r + 1] = key.k1 + (uint32_t)r * 0xBB67AE85u;
        }
        return rk;
    }
    RS_HD operator Key2() const { return Key2{k[0], k[1]}; }
};

RS_DEV uint4 philox_block(uint32_t t, uint32_t tag, uint64_t id, const RoundKeys& rk) {
    uint32_t x0 = t, x1 = tag, x2 = (uint32_t)id, x3 = (uint32_t)(id >> 32);
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * x0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * x2;
        const uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ rk.k[2 * r];
        const uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ rk.k[2 * r + 1];
        x0 = y0; x1 = (uint32_t)p1; x2 = y2; x3 = (uint32_t)p0;
    }
    return make_uint4(x0, x1, x2, x3);
}

// 64-bit value j of a stream: words 2j and 2j+1 (low, high), block j/2.
RS_DEV uint64_t stream_value(Key2 key, uint32_t tag, uint64_t id, uint64_t j) {
    uint4 b = philox_block((uint32_t)(j >> 1), tag, id, key);
    return (j & 1) ? (((uint64_t)b.w << 32) | b.z) : (((uint64_t)b.y << 32) | b.x);
}

// Uniforms from a 64-bit value, exact: U in (0,1], V in [0,1).
RS_DEV double u_open(uint64_t x) { return (double)((x >> 11) + 1) * (1.0 / 9007199254740992.0); }
RS_DEV double v_closed(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }

// Lemire's multiply-and-reject for a range of s <= 2^32 values, one 32-bit
// word per candidate; a rejected ("void") candidate still consumes its word.
// thr = (2^32 - s) mod s.
struct Bounded32 {
    uint64_t s;
    uint32_t thr;
    RS_DEV bool draw(uint32_t w, uint32_t& v) const {
        const uint64_t prod = (uint64_t)w * s;
        v = (uint32_t)(prod >> 32);
        return (uint32_t)prod >= thr;
    }
};

// Same for s > 2^32 with one 64-bit value per candidate; thr = (2^64 - s) mod s.
struct Bounded64 {
    uint64_t s;
    uint64_t thr;
    RS_DEV bool draw(uint64_t x, uint64_t& v) const {
        v = __umul64hi(x, s);
        return x * s >= thr;
    }
};

// Host helpers for the rejection thresholds.
inline uint32_t bounded32_threshold(uint64_t s) { return (uint32_t)(((1ull << 32) - s) % s); }
inline uint64_t bounded64_threshold(uint64_t s) { return (0ull - s) % s; }

}  // namespace rs
