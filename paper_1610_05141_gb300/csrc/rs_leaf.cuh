// rs_leaf.cuh -- candidate draws and the monotone bucket map of the general
// (global-memory) leaf path, rs_big_leaf.cuh.
//
// A leaf's candidates are Lemire draws from its stream (one 32-bit word per
// candidate when the leaf has at most 2^32 positions, one 64-bit value
// otherwise); a rejected draw is void but consumed.  Buckets are addressed
// by the top bits of the value through a monotone map, so that a counting
// sort by bucket followed by ordering each bucket gives sorted output
// (Sec. 4.1).
#pragma once
#include "rs_block.cuh"
#include "rs_internal.h"
#include "rs_rng.cuh"

namespace rs {

constexpr uint32_t kInvalid = 0xFFFFFFFFu;

// Candidate draws of one Philox block: CPB = 4 candidates of 32-bit words
// (s <= 2^32) or CPB = 2 candidates of 64-bit values (s > 2^32).
template <int CPB>
struct Draw;

template <>
struct Draw<4> {
    Bounded32 b;
    template <typename KeyT>
    RS_DEV bool operator()(const uint4& w, int c, KeyT& out) const {
        const uint32_t x = c == 0 ? w.x : c == 1 ? w.y : c == 2 ? w.z : w.w;
        uint32_t v;
        const bool ok = b.draw(x, v);
        out = (KeyT)v;
        return ok;
    }
};

template <>
struct Draw<2> {
    Bounded64 b;
    template <typename KeyT>
    RS_DEV bool operator()(const uint4& w, int c, KeyT& out) const {
        const uint64_t x = c == 0 ? (((uint64_t)w.y << 32) | w.x) : (((uint64_t)w.w << 32) | w.z);
        uint64_t v;
        const bool ok = b.draw(x, v);
        out = (KeyT)v;
        return ok;
    }
};

// Monotone bucket map into [0, T): floor(v * mult / 2^width), with
// mult <= T 2^width / s so that v < s gives a bucket < T.
RS_DEV uint32_t bucket_of(uint32_t v, uint64_t mult) { return __umulhi(v, (uint32_t)mult); }
RS_DEV uint32_t bucket_of(uint64_t v, uint64_t mult) { return (uint32_t)__umul64hi(v, mult); }

template <typename KeyT>
RS_DEV uint64_t bucket_mult(uint64_t s, uint32_t T) {
    if (sizeof(KeyT) == 4) {
        const uint64_t m = ((uint64_t)T << 32) / s;
        return m > 0xFFFFFFFFull ? 0xFFFFFFFFull : m;
    }
    if ((uint64_t)T >= s) return ~0ull;
    return (uint64_t)(((unsigned __int128)T << 64) / s);
}

}  // namespace rs
