/* squares32 (Section 2) and squares64 (Section 5) re-derived with 128-bit
 * integers, for pinning the oracle. TEST INFRASTRUCTURE ONLY.
 *
 * Each round forms the full 128-bit product x*x, reduces it modulo 2^64 by
 * masking, adds the Weyl term with a 128-bit sum reduced the same way, and
 * exchanges the 32-bit halves of the 64-bit result by shifting a 128-bit
 * value that holds two copies of it. The Weyl terms are the 128-bit
 * products ctr*key and (ctr+1)*key reduced modulo 2^64. Nothing here is
 * shared with the oracle or the CUDA path. */
#include <stdint.h>

typedef unsigned __int128 u128;

static u128 mask64(void) { return (((u128)1) << 64) - 1; }

/* (x*x + w) mod 2^64 from the full 128-bit square. */
static uint64_t square_plus(uint64_t x, uint64_t w) {
    const u128 sq = (u128)x * (u128)x;
    return (uint64_t)(((sq & mask64()) + (u128)w) & mask64());
}

/* Halves exchanged: bits 32..95 of the 128-bit value v:v. */
static uint64_t halves_exchanged(uint64_t v) {
    const u128 twice = ((u128)v << 64) | (u128)v;
    return (uint64_t)((twice >> 32) & mask64());
}

static void weyl(uint64_t ctr, uint64_t key, uint64_t *y, uint64_t *z) {
    *y = (uint64_t)(((u128)ctr * (u128)key) & mask64());
    *z = (uint64_t)((((u128)ctr + 1) * (u128)key) & mask64());
}

uint32_t r128_squares32(uint64_t ctr, uint64_t key) {
    uint64_t y, z, x;
    weyl(ctr, key, &y, &z);
    x = halves_exchanged(square_plus(y, y));
    x = halves_exchanged(square_plus(x, z));
    x = halves_exchanged(square_plus(x, y));
    return (uint32_t)(square_plus(x, z) >> 32);
}

uint64_t r128_squares64(uint64_t ctr, uint64_t key) {
    uint64_t y, z, x, t;
    weyl(ctr, key, &y, &z);
    x = halves_exchanged(square_plus(y, y));
    x = halves_exchanged(square_plus(x, z));
    x = halves_exchanged(square_plus(x, y));
    t = square_plus(x, z);
    x = halves_exchanged(t);
    return t ^ (square_plus(x, y) >> 32);
}
