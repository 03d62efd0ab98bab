// Plain generators: one key, consecutive counters ctr_base + i.
//
// Layout: the output is split into a head (elements before the first
// 32- or 16-byte aligned address), a vector region of whole chunks, and a
// tail. In the vector region thread t of a persistent grid of T threads
// handles chunks t, t + T, t + 2T, ...; a chunk is one vector store of
// BYTES bytes, i.e. BYTES / sizeof(element) consecutive outputs. Adjacent
// threads write adjacent chunks, so each warp store covers 32 * BYTES
// contiguous bytes. The thread computes y = ctr*key once and then only adds:
// within a chunk y_{j+1} = y_j + key, and z_j = y_{j+1}; between chunks
// y += T * (counters per chunk) * key (Section 2's Weyl equivalence).
// Nothing is read from memory.
#include <cuda_runtime.h>

#include "internal.h"
#include "squares_core.cuh"

namespace sq {
namespace {

// Every op maps a chunk of consecutive counters to BYTES/4 32-bit words.
// CPC = counters per chunk, EPC = output elements per counter.

struct OpU32 {
    using T = uint32_t;
    static constexpr int EPC = 1;
    template <int W>
    __device__ static void chunk(uint64_t y, uint64_t key, uint32_t (&w)[W]) {
        uint64_t ys[W + 1];
        ys[0] = y;
#pragma unroll
        for (int j = 0; j < W; ++j) ys[j + 1] = add64(ys[j], key);
#pragma unroll
        for (int j = 0; j < W; ++j) w[j] = squares32_yz(ys[j], ys[j + 1]);
    }
    __device__ static T single(uint64_t ctr0, uint64_t key, uint64_t e) {
        return squares32(ctr0 + e, key);
    }
};

struct OpU64 {
    using T = uint64_t;
    static constexpr int EPC = 1;
    template <int W>
    __device__ static void chunk(uint64_t y, uint64_t key, uint32_t (&w)[W]) {
        constexpr int C = W / 2;
        uint64_t ys[C + 1];
        ys[0] = y;
#pragma unroll
        for (int j = 0; j < C; ++j) ys[j + 1] = add64(ys[j], key);
#pragma unroll
        for (int j = 0; j < C; ++j) {
            const uint64_t v = squares64_yz(ys[j], ys[j + 1]);
            w[2 * j] = lo32(v);
            w[2 * j + 1] = hi32(v);
        }
    }
    __device__ static T single(uint64_t ctr0, uint64_t key, uint64_t e) {
        return squares64(ctr0 + e, key);
    }
};

struct OpUniformF32 {
    using T = float;
    static constexpr int EPC = 1;
    template <int W>
    __device__ static void chunk(uint64_t y, uint64_t key, uint32_t (&w)[W]) {
        uint64_t ys[W + 1];
        ys[0] = y;
#pragma unroll
        for (int j = 0; j < W; ++j) ys[j + 1] = add64(ys[j], key);
#pragma unroll
        for (int j = 0; j < W; ++j) w[j] = __float_as_uint(uniform24(squares32_yz(ys[j], ys[j + 1])));
    }
    __device__ static T single(uint64_t ctr0, uint64_t key, uint64_t e) {
        return uniform24(squares32(ctr0 + e, key));
    }
};

struct OpUniformBF16 {
    using T = uint16_t;
    static constexpr int EPC = 1;
    template <int W>
    __device__ static void chunk(uint64_t y, uint64_t key, uint32_t (&w)[W]) {
        constexpr int C = 2 * W;
        uint64_t ys[C + 1];
        ys[0] = y;
#pragma unroll
        for (int j = 0; j < C; ++j) ys[j + 1] = add64(ys[j], key);
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const float a = uniform24(squares32_yz(ys[2 * j], ys[2 * j + 1]));
            const float b = uniform24(squares32_yz(ys[2 * j + 1], ys[2 * j + 2]));
            w[j] = pack_bf16_rz(a, b);
        }
    }
    __device__ static T single(uint64_t ctr0, uint64_t key, uint64_t e) {
        return static_cast<T>(bf16_bits_rz(uniform24(squares32(ctr0 + e, key))));
    }
};

struct OpNormalF32 {
    using T = float;
    static constexpr int EPC = 2;
    template <int W>
    __device__ static void chunk(uint64_t y, uint64_t key, uint32_t (&w)[W]) {
        constexpr int C = W / 2;
        uint64_t ys[C + 1];
        ys[0] = y;
#pragma unroll
        for (int j = 0; j < C; ++j) ys[j + 1] = add64(ys[j], key);
#pragma unroll
        for (int j = 0; j < C; ++j) {
            const uint64_t v = squares64_yz(ys[j], ys[j + 1]);
            const float2 z = box_muller(hi32(v), lo32(v));
            w[2 * j] = __float_as_uint(z.x);
            w[2 * j + 1] = __float_as_uint(z.y);
        }
    }
    __device__ static T single(uint64_t ctr0, uint64_t key, uint64_t e) {
        const uint64_t v = squares64(ctr0 + e / 2, key);
        const float2 z = box_muller(hi32(v), lo32(v));
        return (e & 1) ? z.y : z.x;
    }
};

template <int BYTES, bool CS>
__device__ __forceinline__ void store_chunk(void *p, const uint32_t (&w)[BYTES / 4]) {
    if constexpr (BYTES == 32) {
        store32B<CS>(p, w);
    } else {
        store16B<CS>(p, w[0], w[1], w[2], w[3]);
    }
}

// head: elements [0, head) and tail: [head + nvec*EPV, n) are written one
// element per thread; the vector region in between by whole chunks.
template <class Op, int BYTES, bool CS>
__global__ void __launch_bounds__(512)
    plain_kernel(uint64_t key, uint64_t ctr0, typename Op::T *__restrict__ out, uint64_t n,
                 uint64_t head, uint64_t nvec) {
    using T = typename Op::T;
    constexpr int W = BYTES / 4;
    constexpr int EPV = BYTES / sizeof(T);  // elements per chunk
    constexpr int CPV = EPV / Op::EPC;      // counters per chunk
    const uint64_t tid = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const uint64_t nthreads = static_cast<uint64_t>(gridDim.x) * blockDim.x;

    const uint64_t tail0 = head + nvec * EPV;
    for (uint64_t e = tid; e < head; e += nthreads) out[e] = Op::single(ctr0, key, e);
    for (uint64_t e = tail0 + tid; e < n; e += nthreads) out[e] = Op::single(ctr0, key, e);
    if (tid >= nvec) return;

    // Counter of the first element of chunk `tid` (head is a multiple of EPC).
    uint64_t y = (ctr0 + (head + tid * EPV) / Op::EPC) * key;
    const uint64_t ystep = nthreads * CPV * key;
    char *p = reinterpret_cast<char *>(out + head) + tid * BYTES;
    const uint64_t pstep = nthreads * BYTES;
    for (uint64_t it = (nvec - tid + nthreads - 1) / nthreads; it != 0; --it) {
        uint32_t w[W];
        Op::template chunk<W>(y, key, w);
        store_chunk<BYTES, CS>(p, w);
        y = add64(y, ystep);
        p += pstep;
    }
}

// Variants: 0 = 32 B stores, 1 = 32 B streaming stores, 2 = 16 B stores,
// 3 = 16 B streaming stores.
constexpr int kPlainVariants = 4;
const char *kPlainVariantNames[kPlainVariants] = {"st32", "st32.cs", "st16", "st16.cs"};

template <class Op>
const void *plain_fn(int variant) {
    switch (variant) {
        case 0: return reinterpret_cast<const void *>(&plain_kernel<Op, 32, false>);
        case 1: return reinterpret_cast<const void *>(&plain_kernel<Op, 32, true>);
        case 2: return reinterpret_cast<const void *>(&plain_kernel<Op, 16, false>);
        default: return reinterpret_cast<const void *>(&plain_kernel<Op, 16, true>);
    }
}

const void *plain_fn_for(int kernel_id, int variant) {
    switch (kernel_id) {
        case SQ_KERNEL_U32: return plain_fn<OpU32>(variant);
        case SQ_KERNEL_U64: return plain_fn<OpU64>(variant);
        case SQ_KERNEL_UNIFORM_F32: return plain_fn<OpUniformF32>(variant);
        case SQ_KERNEL_UNIFORM_BF16: return plain_fn<OpUniformBF16>(variant);
        case SQ_KERNEL_NORMAL_F32: return plain_fn<OpNormalF32>(variant);
        default: return nullptr;
    }
}

template <class Op>
cudaError_t launch_op(const Cfg &cfg, uint64_t key, uint64_t ctr0, size_t n, void *out,
                      cudaStream_t stream, int max_ctas) {
    using T = typename Op::T;
    const int bytes = (cfg.variant < 2) ? 32 : 16;
    const size_t epv = bytes / sizeof(T);
    const uintptr_t addr = reinterpret_cast<uintptr_t>(out);
    size_t head = ((bytes - (addr % bytes)) % bytes) / sizeof(T);
    if (head > n) head = n;
    if (head % Op::EPC != 0) head = n;  // pairs would straddle chunks: all singles
    const size_t nvec = (n - head) / epv;
    const int ctas = cfg.ctas_per_sm > 0 ? cfg.ctas_per_sm : max_ctas;
    uint64_t grid = static_cast<uint64_t>(current_sm_count()) * (ctas > 0 ? ctas : 1);
    // Never launch more threads than there are chunks to fill (small n).
    const uint64_t need = (nvec + cfg.block - 1) / cfg.block;
    const uint64_t need_single = (head + (n - head - nvec * epv) + cfg.block - 1) / cfg.block;
    const uint64_t want = need > need_single ? need : need_single;
    if (grid > want) grid = want > 0 ? want : 1;
    T *o = static_cast<T *>(out);
    switch (cfg.variant) {
        case 0: plain_kernel<Op, 32, false><<<grid, cfg.block, 0, stream>>>(key, ctr0, o, n, head, nvec); break;
        case 1: plain_kernel<Op, 32, true><<<grid, cfg.block, 0, stream>>>(key, ctr0, o, n, head, nvec); break;
        case 2: plain_kernel<Op, 16, false><<<grid, cfg.block, 0, stream>>>(key, ctr0, o, n, head, nvec); break;
        default: plain_kernel<Op, 16, true><<<grid, cfg.block, 0, stream>>>(key, ctr0, o, n, head, nvec); break;
    }
    return cudaGetLastError();
}

}  // namespace

int plain_num_variants() { return kPlainVariants; }

const char *plain_variant_name(int variant) {
    return (variant >= 0 && variant < kPlainVariants) ? kPlainVariantNames[variant] : nullptr;
}

int plain_max_ctas_per_sm(int kernel_id, int variant, int block) {
    const void *fn = plain_fn_for(kernel_id, variant);
    int blocks = 0;
    if (!fn || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, block, 0) != cudaSuccess)
        return 1;
    return blocks > 0 ? blocks : 1;
}

cudaError_t launch_plain(int kernel_id, const Cfg &cfg, uint64_t key, uint64_t ctr_base, size_t n,
                         void *out, cudaStream_t stream) {
    if (n == 0) return cudaSuccess;
    const int max_ctas = cfg.ctas_per_sm > 0 ? cfg.ctas_per_sm
                                             : plain_max_ctas_per_sm(kernel_id, cfg.variant, cfg.block);
    switch (kernel_id) {
        case SQ_KERNEL_U32: return launch_op<OpU32>(cfg, key, ctr_base, n, out, stream, max_ctas);
        case SQ_KERNEL_U64: return launch_op<OpU64>(cfg, key, ctr_base, n, out, stream, max_ctas);
        case SQ_KERNEL_UNIFORM_F32:
            return launch_op<OpUniformF32>(cfg, key, ctr_base, n, out, stream, max_ctas);
        case SQ_KERNEL_UNIFORM_BF16:
            return launch_op<OpUniformBF16>(cfg, key, ctr_base, n, out, stream, max_ctas);
        case SQ_KERNEL_NORMAL_F32:
            return launch_op<OpNormalF32>(cfg, key, ctr_base, n, out, stream, max_ctas);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sq
