// Ragged batch of squares32 streams in one persistent launch.
//
// The packed output index space is cut into tiles of blockDim * 8 elements
// (one 32-byte chunk per thread), aligned to the output's 32-byte boundary.
// CTA c of the persistent grid owns one contiguous run of tiles, so as it
// walks its run the stream index only grows: one binary search over the
// offsets at the start, then a forward step whenever a tile crosses into
// the next stream. A run of whole tiles inside one stream is generated like
// the plain kernel (Weyl stepping by tile * key, 32-byte vector stores);
// a tile that touches a stream boundary, a gap or the end of the batch is
// written element by element, each element finding its stream by binary
// search. The batch extent offsets[S-1] + lengths[S-1] is read on the
// device, so the launch needs no host-side knowledge of the lengths and can
// be captured in a CUDA graph. There are no spin-waits and no inter-CTA
// communication.
#include <cuda_runtime.h>

#include "internal.h"
#include "squares_core.cuh"

namespace sq {
namespace {

constexpr uint32_t kNoStream = 0xFFFFFFFFu;

// Largest s in [from, S) with offsets[s] <= e, given offsets[from] <= e.
__device__ __forceinline__ uint32_t find_stream(const int64_t *__restrict__ offsets, uint32_t S,
                                                uint32_t from, int64_t e) {
    uint32_t lo = from, hi = S;
    while (hi - lo > 1) {
        const uint32_t mid = lo + (hi - lo) / 2;
        if (__ldg(offsets + mid) <= e) lo = mid; else hi = mid;
    }
    return lo;
}

// Writes out[e] if some stream covers position e (and e < end).
__device__ __forceinline__ void batch_single(const uint64_t *__restrict__ keys,
                                             const uint64_t *__restrict__ bases,
                                             const int64_t *__restrict__ lengths,
                                             const int64_t *__restrict__ offsets, uint32_t S,
                                             uint32_t from, int64_t e, int64_t end,
                                             uint32_t *__restrict__ out) {
    if (e >= end) return;
    if (from == kNoStream) {
        if (__ldg(offsets) > e) return;
        from = 0;
    }
    const uint32_t s = find_stream(offsets, S, from, e);
    const int64_t off = __ldg(offsets + s);
    if (e >= off + __ldg(lengths + s)) return;
    out[e] = squares32(__ldg(bases + s) + static_cast<uint64_t>(e - off), __ldg(keys + s));
}

template <bool CS>
__global__ void __launch_bounds__(512)
    batch_kernel(const uint64_t *__restrict__ keys, const uint64_t *__restrict__ bases,
                 const int64_t *__restrict__ lengths, const int64_t *__restrict__ offsets,
                 uint32_t S, uint32_t *__restrict__ out, uint32_t head) {
    constexpr int EPV = 8;  // 32-byte chunks of uint32_t
    const int tile = blockDim.x * EPV;  // a power of two
    const int shift = __ffs(tile) - 1;
    if (S == 0) return;
    const int64_t start = __ldg(offsets);
    const int64_t end = __ldg(offsets + S - 1) + __ldg(lengths + S - 1);

    // Elements before the first 32-byte boundary.
    if (blockIdx.x == 0 && threadIdx.x < head)
        batch_single(keys, bases, lengths, offsets, S, kNoStream, threadIdx.x, end, out);
    if (end <= static_cast<int64_t>(head)) return;

    const int64_t first = start > static_cast<int64_t>(head) ? start : head;
    const int64_t t_begin = (first - head) >> shift;
    const int64_t t_end = (end - head + tile - 1) >> shift;
    const int64_t per = (t_end - t_begin + gridDim.x - 1) / gridDim.x;
    int64_t t = t_begin + static_cast<int64_t>(blockIdx.x) * per;
    const int64_t t_stop = (t + per < t_end) ? t + per : t_end;
    if (t >= t_stop) return;

    int64_t lo = head + (t << shift);
    uint32_t s = (start <= lo) ? find_stream(offsets, S, 0, lo) : kNoStream;
    while (t < t_stop) {
        lo = head + (t << shift);
        if (s == kNoStream) {
            if (start <= lo) s = find_stream(offsets, S, 0, lo);
        } else if (s + 1 < S && __ldg(offsets + s + 1) <= lo) {
            s = find_stream(offsets, S, s + 1, lo);
        }
        int64_t k = 0;
        int64_t seg_lo = 0;
        if (s != kNoStream) {
            seg_lo = __ldg(offsets + s);
            const int64_t seg_hi = seg_lo + __ldg(lengths + s);
            if (lo + tile <= seg_hi) {
                k = (seg_hi - lo) >> shift;
                if (k > t_stop - t) k = t_stop - t;
            }
        }
        if (k > 0) {
            // Whole tiles inside stream s.
            const uint64_t key = __ldg(keys + s);
            const int64_t e = lo + threadIdx.x * EPV;
            uint64_t y = (__ldg(bases + s) + static_cast<uint64_t>(e - seg_lo)) * key;
            const uint64_t ystep = key << shift;
            uint32_t *p = out + e;
            for (int64_t i = 0; i < k; ++i) {
                uint64_t ys[EPV + 1];
                ys[0] = y;
#pragma unroll
                for (int j = 0; j < EPV; ++j) ys[j + 1] = add64(ys[j], key);
                uint32_t w[EPV];
#pragma unroll
                for (int j = 0; j < EPV; ++j) w[j] = squares32_yz(ys[j], ys[j + 1]);
                store32B<CS>(p, w);
                y = add64(y, ystep);
                p += tile;
            }
            t += k;
        } else {
            // A tile at a stream boundary, in a gap, or at the end.
            const int64_t e0 = lo + threadIdx.x * EPV;
#pragma unroll 1
            for (int j = 0; j < EPV; ++j)
                batch_single(keys, bases, lengths, offsets, S, s, e0 + j, end, out);
            t += 1;
        }
    }
}

constexpr int kBatchVariants = 2;
const char *kBatchVariantNames[kBatchVariants] = {"st32", "st32.cs"};

const void *batch_fn(int variant) {
    return variant == 1 ? reinterpret_cast<const void *>(&batch_kernel<true>)
                        : reinterpret_cast<const void *>(&batch_kernel<false>);
}

}  // namespace

int batch_num_variants() { return kBatchVariants; }

const char *batch_variant_name(int variant) {
    return (variant >= 0 && variant < kBatchVariants) ? kBatchVariantNames[variant] : nullptr;
}

int batch_max_ctas_per_sm(int variant, int block) {
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, batch_fn(variant), block, 0) !=
        cudaSuccess)
        return 1;
    return blocks > 0 ? blocks : 1;
}

cudaError_t launch_batch(const Cfg &cfg, const uint64_t *keys, const uint64_t *bases,
                         const int64_t *lengths, const int64_t *offsets, size_t nstreams,
                         uint32_t *out, cudaStream_t stream) {
    if (nstreams == 0) return cudaSuccess;
    const int ctas = cfg.ctas_per_sm > 0 ? cfg.ctas_per_sm : batch_max_ctas_per_sm(cfg.variant, cfg.block);
    const unsigned grid = static_cast<unsigned>(current_sm_count()) * static_cast<unsigned>(ctas);
    const uintptr_t addr = reinterpret_cast<uintptr_t>(out);
    const uint32_t head = static_cast<uint32_t>(((32 - (addr % 32)) % 32) / 4);
    const uint32_t S = static_cast<uint32_t>(nstreams);
    if (cfg.variant == 1)
        batch_kernel<true><<<grid, cfg.block, 0, stream>>>(keys, bases, lengths, offsets, S, out, head);
    else
        batch_kernel<false><<<grid, cfg.block, 0, stream>>>(keys, bases, lengths, offsets, S, out, head);
    return cudaGetLastError();
}

}  // namespace sq
