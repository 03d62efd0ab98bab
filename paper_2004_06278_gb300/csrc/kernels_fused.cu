// Generation-only statistics: squares32 values are consumed in registers.
//
// Work is split into items (stream s, part p). Variant 0 gives an item to a
// whole CTA: every thread walks a contiguous run of the item's counters by
// Weyl addition, round 1 carried by accumulation (walk_stats). Variant 1
// gives an item to a warp. In both, the top-byte histogram is kept per warp in shared memory and
// flushed to the global 256-bin histogram at the end, or earlier if a warp's
// 32-bit bins could overflow. A lane keeps only its XOR in registers. The
// item's top-byte sum is read off the warp's histogram: sum over bins of
// b * h[b] grows by exactly that sum while the warp walks the item, so per
// value the loop pays for the histogram increment alone. The warp combines
// the XORs with shuffles and lane 0 merges XOR and sum into the stream's
// outputs with one atomic each (the outputs were cleared on the stream
// beforehand, so the result does not depend on how streams are split into
// parts). Nothing but the statistics is written to global memory.
#include <cuda_runtime.h>

#include "internal.h"
#include "squares_device.cuh"
#include "stores.cuh"

namespace sq {
namespace {

constexpr uint64_t kFlushEvery = 1ull << 31;  // counters per warp between flushes

__device__ __forceinline__ void flush_hist(uint32_t *h, uint64_t *__restrict__ hist, int lane) {
    __syncwarp();
    for (int b = lane; b < 256; b += 32) {
        const uint32_t v = h[b];
        if (v) {
            atomicAdd(reinterpret_cast<unsigned long long *>(hist + b), static_cast<unsigned long long>(v));
            h[b] = 0;
        }
    }
    __syncwarp();
}

// Sum over the warp's bins of b * h[b], in every lane. Bins hold < 2^32
// each (flushes come every 2^31 counters at most), so 64 bits are exact.
__device__ __forceinline__ uint64_t weighted_bins(const uint32_t *h, int lane) {
    __syncwarp();
    uint64_t w = 0;
#pragma unroll
    for (int b = lane; b < 256; b += 32) w += static_cast<uint64_t>(h[b]) * static_cast<uint32_t>(b);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xFFFFFFFFu, w, o);
    return w;
}

// Folds a warp's item into the stream's outputs: XOR by shuffles, the
// top-byte sum as the change of the warp's weighted bins; then flushes the
// histogram when the warp's bins could next overflow.
__device__ __forceinline__ void finish_item(uint32_t x, uint32_t *h, int lane, uint64_t s,
                                            uint64_t item_len, uint64_t &weighted,
                                            uint64_t &since_flush, uint32_t *__restrict__ xor_out,
                                            uint64_t *__restrict__ sum_top, uint64_t *__restrict__ hist) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x ^= __shfl_xor_sync(0xFFFFFFFFu, x, o);
    const uint64_t now = weighted_bins(h, lane);
    if (lane == 0) {
        atomicXor(xor_out + s, x);
        atomicAdd(reinterpret_cast<unsigned long long *>(sum_top + s),
                  static_cast<unsigned long long>(now - weighted));
    }
    weighted = now;
    since_flush += item_len;
    if (since_flush >= kFlushEvery) {
        flush_hist(h, hist, lane);
        since_flush = 0;
        weighted = 0;
    }
}

// Walks cnt consecutive counters of one key from Weyl term y: XOR of the
// values into x, top-byte counts into the warp's histogram h. Round 1 is
// carried by accumulation (t += e, e += c2: two additions per counter, no
// per-block constants), B values per unrolled block.
template <int B>
__device__ __forceinline__ void walk_stats(uint64_t y, uint64_t key, uint64_t cnt, uint32_t &x, uint32_t *h) {
    const uint64_t c2 = (key * key) << 1;
    uint64_t t = round1_value(y);
    uint64_t er = round1_delta(y, key);
    uint64_t i = 0;
    for (; i + B <= cnt; i += B) {
#pragma unroll
        for (int j = 0; j < B; ++j) {
            const uint64_t yn = add64(y, key);
            const uint32_t u = squares32_tyz(t, y, yn);
            y = yn;
            t = add64(t, er);
            er = add64(er, c2);
            x ^= u;
            atomicAdd(h + (u >> 24), 1u);
        }
    }
    for (; i < cnt; ++i) {
        const uint64_t yn = add64(y, key);
        const uint32_t u = squares32_tyz(t, y, yn);
        y = yn;
        t = add64(t, er);
        er = add64(er, c2);
        x ^= u;
        atomicAdd(h + (u >> 24), 1u);
    }
}

// Variant 0: CTA items. Thread i of the block walks counters
// [a + i * m, a + (i + 1) * m) of item [a, b), m = ceil((b - a) / block).
// Two instantiations by block size (register targets for up to 256 and for
// 512 threads).
template <int B, int MAXB, int MINB>
__global__ void __launch_bounds__(MAXB, MINB)
    fused_cta_kernel(const uint64_t *__restrict__ keys, const uint64_t *__restrict__ bases, uint64_t S,
                     uint64_t C, uint64_t parts, uint64_t part_len, uint32_t *__restrict__ xor_out,
                     uint64_t *__restrict__ sum_top, uint64_t *__restrict__ hist) {
    extern __shared__ uint32_t sh_hist[];
    const int lane = threadIdx.x & 31;
    uint32_t *h = sh_hist + (threadIdx.x >> 5) * 256;
    for (int b = lane; b < 256; b += 32) h[b] = 0;
    __syncwarp();
    const uint64_t items = S * parts;
    uint64_t since_flush = 0;
    uint64_t weighted = 0;  // weighted_bins(h) as of the last item's end
    for (uint64_t w = blockIdx.x; w < items; w += gridDim.x) {
        const uint64_t s = w / parts;
        const uint64_t a = (w - s * parts) * part_len;
        const uint64_t b = (a + part_len < C) ? a + part_len : C;
        const uint64_t per_thread = (b - a + blockDim.x - 1) / blockDim.x;
        const uint64_t la = a + threadIdx.x * per_thread;
        const uint64_t lb = (la + per_thread < b) ? la + per_thread : b;
        const uint64_t key = keys[s];
        uint32_t x = 0;
        walk_stats<B>((bases[s] + la) * key, key, (lb > la) ? lb - la : 0, x, h);
        finish_item(x, h, lane, s, b - a, weighted, since_flush, xor_out, sum_top, hist);
    }
    flush_hist(h, hist, lane);
}

// Variant 1: warp items (each lane a contiguous run of the warp's item).
__global__ void __launch_bounds__(512)
    fused_kernel(const uint64_t *__restrict__ keys, const uint64_t *__restrict__ bases, uint64_t S,
                 uint64_t C, uint64_t parts, uint64_t part_len, uint32_t *__restrict__ xor_out,
                 uint64_t *__restrict__ sum_top, uint64_t *__restrict__ hist) {
    extern __shared__ uint32_t sh_hist[];
    const int lane = threadIdx.x & 31;
    uint32_t *h = sh_hist + (threadIdx.x >> 5) * 256;
    for (int b = lane; b < 256; b += 32) h[b] = 0;
    __syncwarp();

    const uint64_t gwarp = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
    const uint64_t items = S * parts;
    uint64_t since_flush = 0;
    uint64_t weighted = 0;  // weighted_bins(h) as of the last item's end
    for (uint64_t w = gwarp; w < items; w += nwarps) {
        const uint64_t s = w / parts;
        const uint64_t a = (w - s * parts) * part_len;
        const uint64_t b = (a + part_len < C) ? a + part_len : C;
        const uint64_t per_lane = (b - a + 31) / 32;
        const uint64_t la = a + lane * per_lane;
        const uint64_t lb = (la + per_lane < b) ? la + per_lane : b;
        const uint64_t key = __ldg(keys + s);
        uint32_t x = 0;
        walk_stats<8>((__ldg(bases + s) + la) * key, key, (lb > la) ? lb - la : 0, x, h);
        finish_item(x, h, lane, s, b - a, weighted, since_flush, xor_out, sum_top, hist);
    }
    flush_hist(h, hist, lane);
}

}  // namespace

int fused_num_variants() { return 2; }

const char *fused_variant_name(int variant) {
    return variant == 0 ? "cta-item" : (variant == 1 ? "warp-item" : nullptr);
}

namespace {
const void *fused_fn(int variant, int block) {
    if (variant == 1) return reinterpret_cast<const void *>(&fused_kernel);
    return block <= 256 ? reinterpret_cast<const void *>(&fused_cta_kernel<32, 256, 0>)
                        : reinterpret_cast<const void *>(&fused_cta_kernel<32, 512, 2>);
}
}  // namespace

int fused_max_ctas_per_sm(int variant, int block) {
    const size_t smem = static_cast<size_t>(block / 32) * 256 * sizeof(uint32_t);
    return occupancy(fused_fn(variant, block), block, smem);
}

cudaError_t launch_fused(const Cfg &cfg, const uint64_t *keys, const uint64_t *bases,
                         size_t nstreams, uint64_t ctrs_per_stream, uint32_t *xor_out,
                         uint64_t *sum_top, uint64_t *hist256, cudaStream_t stream) {
    cudaError_t err = cudaMemsetAsync(hist256, 0, 256 * sizeof(uint64_t), stream);
    if (err != cudaSuccess) return err;
    if (nstreams == 0) return cudaSuccess;
    err = cudaMemsetAsync(xor_out, 0, nstreams * sizeof(uint32_t), stream);
    if (err != cudaSuccess) return err;
    err = cudaMemsetAsync(sum_top, 0, nstreams * sizeof(uint64_t), stream);
    if (err != cudaSuccess) return err;
    if (ctrs_per_stream == 0) return cudaSuccess;

    const int ctas = cfg.ctas_per_sm > 0 ? cfg.ctas_per_sm : fused_max_ctas_per_sm(cfg.variant, cfg.block);
    const uint64_t grid = static_cast<uint64_t>(current_sm_count()) * ctas;
    // the units that take items: CTAs (variant 0) or warps (variant 1)
    const uint64_t units = cfg.variant == 1 ? grid * (cfg.block / 32) : grid;
    // Parts per stream: each item at most 2^29 counters (so a warp's 32-bit
    // bins stay below 2^32 between flushes), and at least ~4 items per unit
    // when there are few streams, but never parts shorter than 1024 counters.
    uint64_t parts = (ctrs_per_stream + (1ull << 29) - 1) >> 29;
    const uint64_t want = (4 * units + nstreams - 1) / nstreams;
    const uint64_t max_parts = (ctrs_per_stream + 1023) / 1024;
    if (want > parts) parts = want < max_parts ? want : max_parts;
    if (parts == 0) parts = 1;
    const uint64_t part_len = (ctrs_per_stream + parts - 1) / parts;
    parts = (ctrs_per_stream + part_len - 1) / part_len;
    const size_t smem = static_cast<size_t>(cfg.block / 32) * 256 * sizeof(uint32_t);
    if (cfg.variant == 1)
        fused_kernel<<<static_cast<unsigned>(grid), cfg.block, smem, stream>>>(
            keys, bases, nstreams, ctrs_per_stream, parts, part_len, xor_out, sum_top, hist256);
    else if (cfg.block <= 256)
        fused_cta_kernel<32, 256, 0><<<static_cast<unsigned>(grid), cfg.block, smem, stream>>>(
            keys, bases, nstreams, ctrs_per_stream, parts, part_len, xor_out, sum_top, hist256);
    else
        fused_cta_kernel<32, 512, 2><<<static_cast<unsigned>(grid), cfg.block, smem, stream>>>(
            keys, bases, nstreams, ctrs_per_stream, parts, part_len, xor_out, sum_top, hist256);
    return cudaGetLastError();
}

}  // namespace sq
