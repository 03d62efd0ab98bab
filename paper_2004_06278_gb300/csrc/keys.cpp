// "Different digits" keys (Section 3 of arXiv:2004.06278), host side.
//
// The paper asks for keys with an irregular bit pattern, roughly half ones,
// whose upper 8 digits are mutually different and whose lower 8 digits are
// too, the digits chosen randomly. This implementation fixes the points the
// paper leaves open: digits are hexadecimal nibbles drawn from 1..15, most
// significant first, each the top four bits of a splitmix64 draw (Steele,
// Lea, Flood 2014), redrawn while zero or already present in its half; the
// least significant digit is also redrawn while even, which makes every key
// odd and ctr*key a full-period Weyl sequence over 2^64 counters; a key
// equal to an earlier one is discarded and drawn again.
#include <cstdint>
#include <vector>

#include "internal.h"

namespace sq {
namespace {

class SplitMix64 {
  public:
    explicit SplitMix64(uint64_t seed) : s_(seed) {}
    uint64_t next() {
        s_ += 0x9E3779B97F4A7C15ull;
        uint64_t v = s_;
        v = (v ^ (v >> 30)) * 0xBF58476D1CE4E5B9ull;
        v = (v ^ (v >> 27)) * 0x94D049BB133111EBull;
        return v ^ (v >> 31);
    }
    unsigned nibble() { return static_cast<unsigned>(next() >> 60); }

  private:
    uint64_t s_;
};

uint64_t draw_half(SplitMix64 &g, bool odd_last) {
    uint64_t half = 0;
    unsigned seen = 0;
    for (int i = 0; i < 8; ++i) {
        const bool last = odd_last && i == 7;
        unsigned d = g.nibble();
        while (d == 0 || ((seen >> d) & 1u) || (last && (d & 1u) == 0)) d = g.nibble();
        seen |= 1u << d;
        half = (half << 4) | d;
    }
    return half;
}

// Open-addressing set of non-zero 64-bit keys.
class KeySet {
  public:
    explicit KeySet(size_t n) {
        size_t cap = 16;
        while (cap < 2 * n) cap <<= 1;
        slots_.assign(cap, 0);
        mask_ = cap - 1;
    }
    bool insert(uint64_t k) {
        size_t i = static_cast<size_t>((k ^ (k >> 29)) * 0xD6E8FEB86659FD93ull) & mask_;
        while (slots_[i] != 0) {
            if (slots_[i] == k) return false;
            i = (i + 1) & mask_;
        }
        slots_[i] = k;
        return true;
    }

  private:
    std::vector<uint64_t> slots_;
    size_t mask_;
};

}  // namespace

int make_keys(uint64_t seed, size_t n, uint64_t *keys) {
    SplitMix64 g(seed);
    KeySet set(n);
    for (size_t i = 0; i < n;) {
        const uint64_t upper = draw_half(g, false);
        const uint64_t lower = draw_half(g, true);
        const uint64_t k = (upper << 32) | lower;
        if (set.insert(k)) keys[i++] = k;
    }
    return SQ_OK;
}

}  // namespace sq
