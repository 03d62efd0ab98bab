/*
 * squares.h -- C ABI of the GB300 (sm_103a) implementation of the Squares
 * counter-based random number generator (B. Widynski, "Squares: A Fast
 * Counter-Based RNG", arXiv:2004.06278).
 *
 * The generator is a pure function out = f(ctr, key) of a 64-bit counter and
 * a 64-bit key (Section 1, Section 6): squares32 (Section 2) runs four rounds
 * of "square modulo 2^64, add ctr*key or (ctr+1)*key, swap the 32-bit halves"
 * and returns 32 bits; squares64 (Section 5) adds a fifth round and returns
 * 64 bits.
 *
 * Conventions shared by every entry point:
 *   - Return value: SQ_OK (0) or a negative status below. After a failure,
 *     sq_last_error() returns a message for the calling thread.
 *   - Device calls are asynchronous on `stream` (a cudaStream_t passed as
 *     void*; NULL is the legacy default stream). Errors that happen while a
 *     kernel runs surface at the caller's next synchronisation. Every launch
 *     is legal inside CUDA stream capture.
 *   - Pointers marked [device] must be device (or managed) memory on the
 *     current device; [host] pointers are ordinary host memory. Output
 *     pointers of the generating calls (sq_u32 ... sq_uniform_f64 and
 *     sq_batch) may also be host memory the device can write (pinned, or
 *     system memory on a coherent host link): the kernels then store
 *     straight across the link, with the 32-byte-per-lane store variant
 *     whatever variant is configured for device memory, since it fills each
 *     128-byte line in one warp store.
 *   - The caller owns every buffer. No entry point allocates device memory
 *     except sq_autotune (a temporary buffer it frees before returning) and
 *     sq_batch_validate / sq_batch_graph_create (documented there).
 *   - n = 0 is valid and launches nothing. Counters wrap modulo 2^64, as the
 *     paper's uint64_t arithmetic does (Section 2); that is not an error.
 *   - Output pointers need only the natural alignment of their element type;
 *     unaligned heads and tails are handled inside the kernels.
 */
#ifndef SQUARES_H_
#define SQUARES_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SQ_OK 0
#define SQ_EINVAL (-1) /* null pointer with n > 0, misaligned pointer, bad id */
#define SQ_ECUDA (-2)  /* a CUDA call or kernel launch failed */
#define SQ_ERANGE (-3) /* a size beyond the documented maximum */

typedef void *sq_stream_t; /* cudaStream_t */

/* Message describing the calling thread's most recent failure ("" if none).
 * The pointer stays valid until that thread's next call into the library. */
const char *sq_last_error(void);

/* Version of this ABI: 100 * major + minor. */
int sq_abi_version(void);

/* Identifier of the kernel code this library was built from: 16 hex digits
 * of a hash of the kernel sources' code (comments and whitespace excluded),
 * or "unknown" when built without it. A tuned launch table is keyed by it
 * (see sq_autotune_save). Static storage; never NULL. No counterpart in the
 * paper. */
const char *sq_build_id(void);

/* Test hook: the next call of the named entry point (e.g. "sq_u32") on the
 * calling thread fails with SQ_ECUDA after its argument checks and before it
 * touches the GPU, as a failed launch would; NULL or "" disarms. Lets a
 * caller exercise its error handling without faulting a device. No
 * counterpart in the paper. */
int sq_debug_fail_next(const char *entry_point);

/* ------------------------------------------------------------------------
 * Keys (Section 3, "different digits"; Section 4, keys.h).
 * Writes n distinct keys to keys[0..n) [host]. Each key's upper eight hex
 * digits are non-zero and mutually different, as are its lower eight; the
 * least significant digit is odd, so that ctr*key runs through all 2^64
 * values (the Weyl argument of Section 2). Digits are drawn with splitmix64
 * (Steele, Lea, Flood 2014) seeded by `seed`: most significant first, each
 * as the top four bits of a draw, redrawn while zero or already used in its
 * half (the last digit also while even); a key equal to an earlier one is
 * redrawn. The output is deterministic in `seed`, and the first m keys do
 * not depend on n. Host only, no GPU needed. SQ_ERANGE if n > 2^31;
 * SQ_EINVAL if keys is NULL with n > 0.
 * ---------------------------------------------------------------------- */
int sq_make_keys(uint64_t seed, size_t n, uint64_t *keys);

/* ------------------------------------------------------------------------
 * Plain streams, one key.
 * sq_u32 (Section 2):  out[i] = squares32(ctr_base + i mod 2^64, key), i < n.
 * sq_u64 (Section 5):  out[i] = squares64(ctr_base + i mod 2^64, key), i < n.
 * out [device], uint32_t / uint64_t aligned. SQ_EINVAL for a NULL or
 * misaligned out with n > 0; SQ_ERANGE if n > 2^62.
 * ---------------------------------------------------------------------- */
int sq_u32(uint64_t key, uint64_t ctr_base, size_t n, uint32_t *out, sq_stream_t stream);
int sq_u64(uint64_t key, uint64_t ctr_base, size_t n, uint64_t *out, sq_stream_t stream);

/* ------------------------------------------------------------------------
 * Strided counters (Section 4: counter increments other than one).
 * sq_u32_strided: out[i] = squares32(ctr_base + i*stride mod 2^64, key).
 * sq_u64_strided: out[i] = squares64(ctr_base + i*stride mod 2^64, key).
 * Any stride is valid, including 0 (every element the same). out [device].
 * Errors as for sq_u32.
 * ---------------------------------------------------------------------- */
int sq_u32_strided(uint64_t key, uint64_t ctr_base, uint64_t stride, size_t n, uint32_t *out,
                   sq_stream_t stream);
int sq_u64_strided(uint64_t key, uint64_t ctr_base, uint64_t stride, size_t n, uint64_t *out,
                   sq_stream_t stream);

/* ------------------------------------------------------------------------
 * Key-counter mode (Section 4: the counter fixed, the key varying).
 * sq_keys_u32: out[i] = squares32(ctr, keys[i]);  sq_keys_u64: squares64.
 * keys [device, uint64_t[nkeys]], out [device]. SQ_EINVAL for NULL or
 * misaligned arrays with nkeys > 0; SQ_ERANGE if nkeys > 2^62.
 * ---------------------------------------------------------------------- */
int sq_keys_u32(const uint64_t *keys, size_t nkeys, uint64_t ctr, uint32_t *out,
                sq_stream_t stream);
int sq_keys_u64(const uint64_t *keys, size_t nkeys, uint64_t ctr, uint64_t *out,
                sq_stream_t stream);

/* ------------------------------------------------------------------------
 * Ragged batch of squares32 streams in one persistent launch (Section 3:
 * many keys, each with its own 2^64 counter space).
 * For every stream s < nstreams and i < lengths[s]:
 *   out[offsets[s] + i] = squares32(ctr_bases[s] + i mod 2^64, keys[s]).
 * keys, ctr_bases [device, uint64_t[nstreams]]; lengths, offsets [device,
 * int64_t[nstreams]]; out [device, uint32_t[offsets[S-1] + lengths[S-1]]].
 * Requirements (not checked by this call, which never reads device memory
 * on the host; see sq_batch_validate): lengths[s] >= 0, offsets[0] >= 0,
 * offsets[s] + lengths[s] <= offsets[s+1]. Positions of out that no stream
 * covers are left untouched. Whatever the inputs, no launch variant writes
 * outside [0, offsets[S-1] + lengths[S-1]). That extent is read on the
 * device, so the call can be captured once and replayed with new lengths.
 * SQ_EINVAL for NULL arrays with nstreams > 0 or a misaligned pointer;
 * SQ_ERANGE if nstreams > 2^31.
 * ---------------------------------------------------------------------- */
int sq_batch(const uint64_t *keys, const uint64_t *ctr_bases, const int64_t *lengths,
             const int64_t *offsets, size_t nstreams, uint32_t *out, sq_stream_t stream);

/* Synchronous debug check of sq_batch's requirements: copies lengths and
 * offsets to the host (through a temporary host buffer) after synchronising
 * `stream`. SQ_OK if they hold, SQ_EINVAL (with the first bad index in the
 * message) otherwise. Not capturable. */
int sq_batch_validate(const int64_t *lengths, const int64_t *offsets, size_t nstreams,
                      sq_stream_t stream);

/* ------------------------------------------------------------------------
 * Distribution transforms (floating-point conversion, Section 5).
 * sq_uniform_f32:  out[i] = floor(squares32(ctr_base+i, key) / 2^8) * 2^-24,
 *                  a float in [0, 1), exact (24 significant bits).
 * sq_uniform_bf16: the same value rounded toward zero to bfloat16 (so it
 *                  stays below 1), stored as its 16-bit pattern.
 * sq_normal_f32:   standard normals by the Box-Muller transform. With
 *                  v = squares64(ctr_base + j, key), hi = v >> 32,
 *                  lo = v mod 2^32: u1 = (hi + 1) 2^-32 in (0, 1],
 *                  theta = 2 pi lo 2^-32, r = sqrt(-2 ln u1),
 *                  out[2j] = r cos theta, out[2j+1] = r sin theta; an odd n
 *                  drops the last sine. Computed in FP32 without branches
 *                  and without CUDA math-library calls: with
 *                  hi + 1 = 2^E (1 + f), 1 + f in [1/sqrt2, sqrt2),
 *                  ln u1 = (E - 32) ln 2 + 2 atanh(s), s = D / (hi + 1 + 2^E)
 *                  where D = hi + 1 - 2^E is formed exactly in 32-bit
 *                  integers (so s keeps its relative accuracy as u1 -> 1),
 *                  atanh by a fitted polynomial of degree 5; the angle is
 *                  split into an exact quadrant of lo and a remainder whose
 *                  sine and cosine come from polynomials of degree 7 and 6
 *                  (all three fitted by least squares on Chebyshev nodes,
 *                  csrc/fit_box_muller.py); r from the
 *                  hardware reciprocal square root (r^2 times rsqrt(r^2)).
 *                  Error against the FP64 values, measured over all 2^32
 *                  values of each half: at most 1.2e-6 absolute where
 *                  |z| < 5 and 2.1e-7 relative beyond (bound stated for
 *                  callers: 2e-6 absolute, 1e-5 relative).
 *                  A pointer 4-byte but not 8-byte aligned still gets vector
 *                  stores: chunks then start at a pair's second element and
 *                  compute one pair more than they store.
 * out [device], naturally aligned. Errors as for sq_u32.
 * ---------------------------------------------------------------------- */
int sq_uniform_f32(uint64_t key, uint64_t ctr_base, size_t n, float *out, sq_stream_t stream);
int sq_uniform_bf16(uint64_t key, uint64_t ctr_base, size_t n, uint16_t *out,
                    sq_stream_t stream);
int sq_normal_f32(uint64_t key, uint64_t ctr_base, size_t n, float *out, sq_stream_t stream);

/* Section 5's 64-bit output used for floating point:
 * sq_uniform2_f32: two floats per squares64 output v = squares64(ctr_base+j):
 *                  out[2j] = floor(hi/2^8) 2^-24, out[2j+1] = floor(lo/2^8)
 *                  2^-24 (hi, lo the upper and lower 32 bits); an odd n drops
 *                  the last one. Exact. Like sq_normal_f32, a pointer 4-byte
 *                  but not 8-byte aligned still gets vector stores.
 * sq_uniform_f64:  out[i] = floor(squares64(ctr_base+i) / 2^11) 2^-53, a
 *                  53-bit double in [0, 1), exact; built from integer
 *                  operations (no FP64 arithmetic on the GPU).
 * out [device], naturally aligned. Errors as for sq_u32. */
int sq_uniform2_f32(uint64_t key, uint64_t ctr_base, size_t n, float *out, sq_stream_t stream);
int sq_uniform_f64(uint64_t key, uint64_t ctr_base, size_t n, double *out, sq_stream_t stream);

/* ------------------------------------------------------------------------
 * Generation-only statistics: squares32 values consumed in registers, never
 * stored. For each stream s < nstreams over the counters ctr_bases[s] + i,
 * i < ctrs_per_stream (mod 2^64), with key keys[s]:
 *   xor_out[s] = XOR of the outputs,
 *   sum_top[s] = sum of the outputs' top bytes (output >> 24),
 * and hist256[b] = number of outputs, over all streams, whose top byte is b.
 * keys, ctr_bases [device, uint64_t[nstreams]]; xor_out [device,
 * uint32_t[nstreams]]; sum_top [device, uint64_t[nstreams]]; hist256
 * [device, uint64_t[256]]. The call clears the three outputs on `stream`
 * before accumulating into them. SQ_ERANGE if nstreams > 2^31 or
 * ctrs_per_stream > 2^40.
 * ---------------------------------------------------------------------- */
int sq_fused_stats(const uint64_t *keys, const uint64_t *ctr_bases, size_t nstreams,
                   uint64_t ctrs_per_stream, uint32_t *xor_out, uint64_t *sum_top,
                   uint64_t *hist256, sq_stream_t stream);

/* ------------------------------------------------------------------------
 * Launch configuration and autotuning. Each kernel family has a table of
 * launch configurations indexed by a size bucket (floor(log2(n))): n is the
 * number of output elements for the plain generators, the total number of
 * counters for SQ_KERNEL_FUSED, and the number of streams for
 * SQ_KERNEL_BATCH (so a batch of a few long streams and one of millions of
 * short ones keep separate choices). The default entry is a fixed choice
 * for GB300. All variants compute identical results; only the speed
 * differs.
 * ---------------------------------------------------------------------- */
#define SQ_KERNEL_U32 0
#define SQ_KERNEL_U64 1
#define SQ_KERNEL_BATCH 2
#define SQ_KERNEL_UNIFORM_F32 3
#define SQ_KERNEL_UNIFORM_BF16 4
#define SQ_KERNEL_NORMAL_F32 5
#define SQ_KERNEL_FUSED 6
#define SQ_KERNEL_UNIFORM2_F32 7
#define SQ_KERNEL_UNIFORM_F64 8
#define SQ_NUM_KERNELS 9

typedef struct {
    int32_t variant;     /* kernel body: store width / cache policy, see sq_variant_name;
                          * for SQ_KERNEL_BATCH 0-3 tile the packed output, 4-8 give each
                          * stream to 32, 8, 16, 4 or 1 lanes, 9 lays 32 streams end to
                          * end per warp, one position per lane, 10-12 give each lane
                          * an aligned segment of 4, 8 or 16 values of one of a warp's
                          * 32 streams (4-12 are for many short streams); for
                          * SQ_KERNEL_FUSED 0 gives each stream part to a CTA, 1 to a
                          * warp */
    int32_t block;       /* threads per CTA: 128, 256 or 512 (SQ_KERNEL_BATCH also 64) */
    int32_t ctas_per_sm; /* persistent grid = SMs * ctas_per_sm; 0 = max resident, except
                          * for the SQ_KERNEL_BATCH flattened-warp variants (9-12),
                          * where 0 launches one warp per 32 streams */
    int32_t reserved;
} sq_launch_config;

/* Number of body variants of a kernel family, and a short name for one. */
int sq_num_variants(int kernel_id);
const char *sq_variant_name(int kernel_id, int variant);

/* Read / override the configuration used for problems of size n. Setting
 * applies to every size bucket when n == 0. SQ_EINVAL for a bad id or an
 * invalid configuration. */
int sq_get_config(int kernel_id, size_t n, sq_launch_config *cfg);
int sq_set_config(int kernel_id, size_t n, const sq_launch_config *cfg);

/* Time every candidate configuration on a problem of size n_hint (in output
 * elements; for SQ_KERNEL_FUSED, total counters) and keep the fastest for
 * that size bucket. For SQ_KERNEL_BATCH the candidates are the tile
 * variants on a synthetic batch of 64 long streams holding n_hint elements,
 * and the pick becomes the entry of every stream-count bucket (calls of
 * sq_autotune_batch afterwards refine single buckets). Synchronous;
 * allocates and frees a temporary device buffer of at most 2 GiB; must not
 * run during stream capture. */
int sq_autotune(int kernel_id, size_t n_hint);

/* Tune the ragged-batch kernel on the caller's own batch: candidate
 * configurations are launched on these device arrays (each launch writes the
 * same, correct outputs into out) and the fastest becomes the one sq_batch
 * uses for batches in the same stream-count bucket (floor(log2(nstreams))).
 * The streams-to-lanes and flattened-warp variants are candidates
 * only when the mean stream length (read back from the batch extent) is at
 * most 8192, and a variant whose probe (block 256, ctas_per_sm 0)
 * takes over 3x the best time so far is not timed in its other
 * configurations. sq_autotune(SQ_KERNEL_BATCH, n) times the tile variants
 * only. Synchronous; allocates no device memory; must not run during stream
 * capture. Arguments and errors as for sq_batch. */
int sq_autotune_batch(const uint64_t *keys, const uint64_t *ctr_bases, const int64_t *lengths,
                      const int64_t *offsets, size_t nstreams, uint32_t *out);

/* Persist / restore the tuned table as a small text file keyed by the
 * device name and by sq_build_id(). Loading a table saved on another
 * device name is a no-op (SQ_OK). Loading a table saved by a library built
 * from other kernel code (or a file of format 1, which records no code
 * identifier) leaves the table unchanged and returns SQ_EINVAL; the message
 * names both identifiers. If the environment variable SQ_TUNE_FILE names a
 * file, it is loaded the same way on the library's first use of the table
 * (a file that does not apply is ignored silently there). */
int sq_autotune_save(const char *path);
int sq_autotune_load(const char *path);

/* Store ceiling: writes `value` to out[0..n) with the store path of the
 * plain generators (the same head / vector-chunk / tail split, persistent
 * grid and store variant) and no generator arithmetic, so its rate is the
 * write bandwidth those kernels are held against, for device memory or,
 * given host memory the device can write, for the host link. cfg selects
 * the variant, block and CTAs per SM as for SQ_KERNEL_U32 (NULL: the entry
 * sq_u32 would use for n). pause_ns > 0 makes every thread pause that long
 * (__nanosleep) after each chunk it stores: a paced store stream, like a
 * generator's, can reach more DRAM write bandwidth than one that floods
 * the memory system. out [device or device-writable host], 4-byte aligned.
 * Errors as for sq_u32, and SQ_EINVAL for an invalid cfg. No counterpart
 * in the paper: a measurement kernel. */
int sq_fill_u32(uint32_t value, size_t n, uint32_t *out, const sq_launch_config *cfg,
                uint32_t pause_ns, sq_stream_t stream);

/* ------------------------------------------------------------------------
 * CUDA graph of one sq_batch launch, for callers without a graph API of
 * their own. Capture happens once, on an internal stream; the graph reads
 * the same device arrays at every replay, so new lengths / offsets / bases
 * written there between replays take effect without re-capture.
 * ---------------------------------------------------------------------- */
typedef struct sq_graph_s *sq_graph_t;
int sq_batch_graph_create(const uint64_t *keys, const uint64_t *ctr_bases,
                          const int64_t *lengths, const int64_t *offsets, size_t nstreams,
                          uint32_t *out, sq_graph_t *graph);
int sq_graph_launch(sq_graph_t graph, sq_stream_t stream);
int sq_graph_destroy(sq_graph_t graph);

#ifdef __cplusplus
}
#endif

#endif /* SQUARES_H_ */
