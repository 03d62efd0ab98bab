/*
 * Oracle for the Squares counter-based generator
 * (B. Widynski, "Squares: A Fast Counter-Based RNG", arXiv:2004.06278).
 *
 * TEST INFRASTRUCTURE. This file is the slow, obviously correct CPU statement
 * of what the GPU path computes. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it. It shares no code, header, table
 * or helper with the CUDA library, and the library never calls it.
 *
 * Every integer step below is unsigned 64-bit C arithmetic, which wraps
 * modulo 2^64 exactly as the paper's uint64_t code does (Section 2).
 * Floating-point outputs of the distribution transforms are computed in
 * double precision (FP64) from the same integers.
 *
 * Pins (what ties this file to something other than itself) live in
 * tests/test_oracle_pins.py: hand-derived worked examples, the squares32 /
 * squares64 high-half identity, the even-key period, key = 0, a route through
 * arbitrary-precision integers that rotates by multiplication modulo
 * 2^64 - 1, exhaustive reduced-width brute force, and chi-square smoke tests.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* The generator (Section 2, Section 5).                                     */
/* ------------------------------------------------------------------------ */

/* Circular shift by 32 bits: moves the middle of the square into the low
 * half (Section 3, second paragraph). */
static uint64_t swap_halves(uint64_t v) { return (v << 32) | (v >> 32); }

/* One middle-square round of Section 2: square modulo 2^64, add the Weyl
 * term w (either ctr*key or (ctr+1)*key), then rotate by 32 bits. */
static uint64_t middle_square_round(uint64_t x, uint64_t w) {
    return swap_halves(x * x + w);
}

/* squares32, Section 2: four rounds; rounds 1..4 add y, z, y, z where
 * y = ctr*key and z = (ctr+1)*key = y + key (Section 3, "For keys generated
 * by the key utility ..."). The fourth round is not rotated: its upper
 * 32 bits are the output. */
uint32_t oracle_squares32(uint64_t ctr, uint64_t key) {
    const uint64_t y = ctr * key;
    const uint64_t z = y + key;
    uint64_t x = y;
    x = middle_square_round(x, y);
    x = middle_square_round(x, z);
    x = middle_square_round(x, y);
    const uint64_t last = x * x + z;
    return (uint32_t)(last >> 32);
}

/* squares64, Section 5: rounds 1..3 as in squares32; the fourth round value
 * t (before its rotation) is kept whole; a fifth round squares rotate(t),
 * adds y, and its upper 32 bits are xored into t. */
uint64_t oracle_squares64(uint64_t ctr, uint64_t key) {
    const uint64_t y = ctr * key;
    const uint64_t z = y + key;
    uint64_t x = y;
    x = middle_square_round(x, y);
    x = middle_square_round(x, z);
    x = middle_square_round(x, y);
    const uint64_t t = x * x + z;
    x = swap_halves(t);
    const uint64_t fifth = x * x + y;
    return t ^ (fifth >> 32);
}

/* Reduced-width analogue of the same construction, for exhaustive tests.
 * The state is w bits (w even, 8 <= w <= 64); every operation is taken
 * modulo 2^w and the rotation is by w/2. With w = 64, rounds = 4 this is
 * squares32 and with rounds = 5, wide = 1 it is squares64. use_z = 0 adds y
 * in every round instead of alternating y and z: that is the variant the
 * paper's acknowledgements describe as non-uniform ("too many zeros")
 * before (ctr+1)*key was introduced. rounds = 3 is the variant reported to
 * fail a statistical test. Output: the upper w/2 bits of the last square
 * (wide = 0), or the squares64-style wide output (wide = 1). */
uint64_t oracle_squares_w(uint64_t ctr, uint64_t key, unsigned w,
                          unsigned rounds, int use_z, int wide) {
    const uint64_t mask = (w >= 64) ? ~(uint64_t)0 : (((uint64_t)1 << w) - 1);
    const unsigned half = w / 2;
    const uint64_t y = (ctr * key) & mask;
    const uint64_t z = use_z ? ((y + key) & mask) : y;
    uint64_t x = y;
    unsigned r;
    /* Every round but the last is rotated; the wide output also keeps the
     * value of the next-to-last round before its rotation. */
    const unsigned rotated = rounds - 1;
    uint64_t t = 0;
    for (r = 1; r <= rotated; ++r) {
        const uint64_t w_r = (r % 2 == 1) ? y : z;
        const uint64_t s = (x * x + w_r) & mask;
        if (wide && r == rotated) t = s;
        x = ((s >> half) | (s << half)) & mask;
    }
    {
        const uint64_t w_last = (rounds % 2 == 1) ? y : z;
        const uint64_t s = (x * x + w_last) & mask;
        if (wide) return t ^ (s >> half);
        return s >> half;
    }
}

/* Adds to hist (2^(w/2) bins) the reduced-width narrow outputs of the
 * counters c0 .. c1 - 1 for one key. */
void oracle_hist_w_range(uint64_t key, unsigned w, unsigned rounds, int use_z,
                         uint64_t c0, uint64_t c1, uint64_t *hist) {
    uint64_t c;
    for (c = c0; c < c1; ++c) hist[oracle_squares_w(c, key, w, rounds, use_z, 0)] += 1;
}

/* Exhaustive histogram of the reduced-width narrow output over every
 * counter 0 .. 2^w - 1 for one key; hist has 2^(w/2) bins. */
void oracle_hist_w(uint64_t key, unsigned w, unsigned rounds, int use_z,
                   uint64_t *hist) {
    memset(hist, 0, sizeof(uint64_t) * ((size_t)1 << (w / 2)));
    oracle_hist_w_range(key, w, rounds, use_z, 0, (uint64_t)1 << w, hist);
}

/* ------------------------------------------------------------------------ */
/* Array forms.                                                              */
/* ------------------------------------------------------------------------ */

/* out[i] = squares32(base + i mod 2^64, key), i < n. */
void oracle_fill32(uint64_t key, uint64_t base, uint64_t n, uint32_t *out) {
    uint64_t i;
    for (i = 0; i < n; ++i) out[i] = oracle_squares32(base + i, key);
}

/* out[i] = squares64(base + i mod 2^64, key), i < n. */
void oracle_fill64(uint64_t key, uint64_t base, uint64_t n, uint64_t *out) {
    uint64_t i;
    for (i = 0; i < n; ++i) out[i] = oracle_squares64(base + i, key);
}

/* Strided counters (Section 4's "increments other than one"):
 * out[i] = squares32(base + i*stride mod 2^64, key). */
void oracle_fill32_strided(uint64_t key, uint64_t base, uint64_t stride, uint64_t n,
                           uint32_t *out) {
    uint64_t i;
    for (i = 0; i < n; ++i) out[i] = oracle_squares32(base + i * stride, key);
}

void oracle_fill64_strided(uint64_t key, uint64_t base, uint64_t stride, uint64_t n,
                           uint64_t *out) {
    uint64_t i;
    for (i = 0; i < n; ++i) out[i] = oracle_squares64(base + i * stride, key);
}

/* Per-element (counter, key) pairs, for sampled checks and Section 4's
 * key-counter mode (one counter, many keys). */
void oracle_pairs32(const uint64_t *ctrs, const uint64_t *keys, uint64_t n,
                    uint32_t *out) {
    uint64_t i;
    for (i = 0; i < n; ++i) out[i] = oracle_squares32(ctrs[i], keys[i]);
}

void oracle_pairs64(const uint64_t *ctrs, const uint64_t *keys, uint64_t n,
                    uint64_t *out) {
    uint64_t i;
    for (i = 0; i < n; ++i) out[i] = oracle_squares64(ctrs[i], keys[i]);
}

/* Batched ragged form: stream s owns out[offsets[s] .. offsets[s] +
 * lengths[s]) and element i of it is squares32(bases[s] + i mod 2^64,
 * keys[s]). Positions owned by no stream are not written. */
void oracle_batch32(const uint64_t *keys, const uint64_t *bases,
                    const int64_t *lengths, const int64_t *offsets,
                    uint64_t nstreams, uint32_t *out) {
    uint64_t s;
    int64_t i;
    for (s = 0; s < nstreams; ++s)
        for (i = 0; i < lengths[s]; ++i)
            out[offsets[s] + i] = oracle_squares32(bases[s] + (uint64_t)i, keys[s]);
}

/* ------------------------------------------------------------------------ */
/* Distribution transforms, in FP64.                                         */
/* ------------------------------------------------------------------------ */

/* Uniform on [0, 1) from the upper 24 bits of the squares32 output:
 * floor(u / 2^8) / 2^24. The value has at most 24 significant bits, so the
 * conversion to float is exact. */
void oracle_uniform_f32(uint64_t key, uint64_t base, uint64_t n, float *out) {
    uint64_t i;
    for (i = 0; i < n; ++i) {
        const uint32_t u = oracle_squares32(base + i, key);
        const double v = (double)(u >> 8) / 16777216.0;
        out[i] = (float)v;
    }
}

/* The same uniform, rounded toward zero to bfloat16 (8 significant bits),
 * returned as the bfloat16 bit pattern. Computed from the value, not from
 * float bits: v = m * 2^e with m in [0.5, 1), keep floor(m * 256) / 256. */
void oracle_uniform_bf16(uint64_t key, uint64_t base, uint64_t n,
                         uint16_t *out) {
    uint64_t i;
    for (i = 0; i < n; ++i) {
        const uint32_t u = oracle_squares32(base + i, key);
        const double v = (double)(u >> 8) / 16777216.0;
        if (v == 0.0) {
            out[i] = 0;
        } else {
            int e;
            const double m = frexp(v, &e);         /* v = m * 2^e, m in [0.5,1) */
            const int q = (int)floor(m * 256.0);   /* 128 .. 255 */
            const int biased = (e - 1) + 127;      /* v in [2^(e-1), 2^e) */
            out[i] = (uint16_t)((biased << 7) | (q - 128));
        }
    }
}

/* Two uniforms per squares64 output (Section 5: the 64 bits split into two
 * 32-bit halves): output j = squares64(base + j, key) supplies
 * out[2j] = floor(hi / 2^8) / 2^24 and out[2j+1] = floor(lo / 2^8) / 2^24,
 * hi and lo its upper and lower 32 bits. An odd n drops the last one. */
void oracle_uniform2_f32(uint64_t key, uint64_t base, uint64_t n, float *out) {
    uint64_t j;
    for (j = 0; 2 * j < n; ++j) {
        const uint64_t v = oracle_squares64(base + j, key);
        out[2 * j] = (float)((double)((v >> 32) >> 8) / 16777216.0);
        if (2 * j + 1 < n) out[2 * j + 1] = (float)((double)((v & 0xffffffffu) >> 8) / 16777216.0);
    }
}

/* 53-bit double uniforms (Section 5): floor(squares64 / 2^11) / 2^53, exact
 * in double precision. */
void oracle_uniform_f64(uint64_t key, uint64_t base, uint64_t n, double *out) {
    uint64_t i;
    for (i = 0; i < n; ++i) {
        const uint64_t v = oracle_squares64(base + i, key);
        out[i] = (double)(v >> 11) / 9007199254740992.0;
    }
}

/* The 53-bit double uniform of given 64-bit values: floor(v / 2^11) / 2^53. */
void oracle_uniform53_of(const uint64_t *v, uint64_t n, double *out) {
    uint64_t i;
    for (i = 0; i < n; ++i) out[i] = (double)(v[i] >> 11) / 9007199254740992.0;
}

/* The Box-Muller pair from the two 32-bit halves of one squares64 output:
 *   u1 = (hi + 1) / 2^32 in (0, 1],  theta = 2 pi lo / 2^32,
 *   r  = sqrt(-2 ln u1),  z0 = r cos theta,  z1 = r sin theta.
 * All in double precision. */
static void box_muller_pair(uint32_t hi, uint32_t lo, double *z0, double *z1) {
    const double two_pi = 6.283185307179586476925286766559;
    const double u1 = ((double)hi + 1.0) / 4294967296.0;
    const double theta = two_pi * ((double)lo / 4294967296.0);
    const double r = sqrt(-2.0 * log(u1));
    *z0 = r * cos(theta);
    *z1 = r * sin(theta);
}

/* Standard normals by the Box-Muller transform from squares64 outputs.
 * Output j = squares64(base + j, key) supplies the pair (2j, 2j+1) from
 * hi = its upper 32 bits and lo = its lower 32 bits (box_muller_pair).
 * An odd n drops the last sine. */
void oracle_normal_f64(uint64_t key, uint64_t base, uint64_t n, double *out) {
    uint64_t j;
    for (j = 0; 2 * j < n; ++j) {
        const uint64_t v = oracle_squares64(base + j, key);
        double z0, z1;
        box_muller_pair((uint32_t)(v >> 32), (uint32_t)v, &z0, &z1);
        out[2 * j] = z0;
        if (2 * j + 1 < n) out[2 * j + 1] = z1;
    }
}

/* The same pair for given halves: out[2i], out[2i+1] from (hi[i], lo[i]). */
void oracle_box_muller_f64(const uint32_t *hi, const uint32_t *lo, uint64_t n, double *out) {
    uint64_t i;
    for (i = 0; i < n; ++i) box_muller_pair(hi[i], lo[i], &out[2 * i], &out[2 * i + 1]);
}

/* ------------------------------------------------------------------------ */
/* Generation-only statistics.                                               */
/* ------------------------------------------------------------------------ */

/* For each stream s, the counters bases[s] + i (i < ctrs_per_stream):
 *   xor_out[s] = XOR of the squares32 outputs,
 *   sum_out[s] = sum of their top bytes (output >> 24),
 * and hist[b] (256 bins, over all streams) counts outputs with top byte b. */
void oracle_fused_stats(const uint64_t *keys, const uint64_t *bases,
                        uint64_t nstreams, uint64_t ctrs_per_stream,
                        uint32_t *xor_out, uint64_t *sum_out, uint64_t *hist) {
    uint64_t s, i;
    memset(hist, 0, 256 * sizeof(uint64_t));
    for (s = 0; s < nstreams; ++s) {
        uint32_t acc_xor = 0;
        uint64_t acc_sum = 0;
        for (i = 0; i < ctrs_per_stream; ++i) {
            const uint32_t u = oracle_squares32(bases[s] + i, keys[s]);
            acc_xor ^= u;
            acc_sum += u >> 24;
            hist[u >> 24] += 1;
        }
        xor_out[s] = acc_xor;
        sum_out[s] = acc_sum;
    }
}

/* ------------------------------------------------------------------------ */
/* Keys with "different digits" (Section 3).                                 */
/* ------------------------------------------------------------------------ */

/* splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): a Weyl state advanced by the golden-ratio
 * increment, passed through a 64-bit finaliser. Only the digit draws use it. */
typedef struct { uint64_t state; } oracle_splitmix;

static uint64_t splitmix_next(oracle_splitmix *g) {
    uint64_t v;
    g->state += 0x9E3779B97F4A7C15ull;
    v = g->state;
    v = (v ^ (v >> 30)) * 0xBF58476D1CE4E5B9ull;
    v = (v ^ (v >> 27)) * 0x94D049BB133111EBull;
    return v ^ (v >> 31);
}

/* One hexadecimal digit: the top four bits of the next draw. */
static unsigned draw_digit(oracle_splitmix *g) {
    return (unsigned)(splitmix_next(g) >> 60);
}

/* A key whose upper eight hex digits are non-zero and mutually different,
 * whose lower eight are too, and whose last digit is odd (Section 3, with
 * the readings: digits are nibbles, drawn from 1..15, most significant
 * first, by rejection; the lowest digit is drawn from the odd digits not
 * yet used in the lower half so that ctr*key has full period 2^64). */
static uint64_t draw_key(oracle_splitmix *g) {
    uint64_t key = 0;
    int pos;
    unsigned used = 0;
    for (pos = 15; pos >= 8; --pos) {
        unsigned d;
        do { d = draw_digit(g); } while (d == 0 || (used >> d) & 1u);
        used |= 1u << d;
        key |= (uint64_t)d << (4 * pos);
    }
    used = 0;
    for (pos = 7; pos >= 0; --pos) {
        unsigned d;
        if (pos > 0) {
            do { d = draw_digit(g); } while (d == 0 || (used >> d) & 1u);
        } else {
            do { d = draw_digit(g); } while (d % 2 == 0 || (used >> d) & 1u);
        }
        used |= 1u << d;
        key |= (uint64_t)d << (4 * pos);
    }
    return key;
}

/* n distinct keys from one seed; a key equal to an earlier one is redrawn.
 * Deterministic in the seed, and the first m keys do not depend on n.
 * Returns 0 on success, -1 if the table cannot be allocated. */
int oracle_make_keys(uint64_t seed, uint64_t n, uint64_t *keys) {
    oracle_splitmix g;
    uint64_t cap = 16, i;
    uint64_t *table;
    g.state = seed;
    while (cap < 2 * n) cap *= 2;
    table = (uint64_t *)calloc(cap, sizeof(uint64_t)); /* 0 = empty slot */
    if (!table) return -1;
    for (i = 0; i < n;) {
        const uint64_t k = draw_key(&g);
        uint64_t h = (k * 0x9E3779B97F4A7C15ull) & (cap - 1);
        int seen = 0;
        while (table[h] != 0) {
            if (table[h] == k) { seen = 1; break; }
            h = (h + 1) & (cap - 1);
        }
        if (seen) continue;
        table[h] = k;
        keys[i++] = k;
    }
    free(table);
    return 0;
}

/* The digit source alone, exposed for property tests. */
void oracle_splitmix64(uint64_t seed, uint64_t n, uint64_t *out) {
    oracle_splitmix g;
    uint64_t i;
    g.state = seed;
    for (i = 0; i < n; ++i) out[i] = splitmix_next(&g);
}
