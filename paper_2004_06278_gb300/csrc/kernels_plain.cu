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
// y += T * (counters per chunk) * key (Section 2's Weyl equivalence). Round
// 1 squares y itself, and its value for consecutive counters follows a
// second-order recurrence (see walk), so it costs additions, not multiplies.
// Nothing is read from memory.
#include <cuda_runtime.h>

#include <type_traits>

#include "internal.h"
#include "squares_device.cuh"
#include "stores.cuh"

namespace sq {
namespace {

// Calls f(j, t, y, z) for the C consecutive counters of a chunk, where y and
// z are the counter's Weyl terms and t its round-1 value. y starts at the
// chunk's first counter, e = t(ctr+1) - t(ctr) there, c2 = 2*key^2: after
// one squaring for t, counter j+1 follows from counter j by y += key and
// t += e + j*c2 (one three-input addition; j*c2 is the same for every thread
// of the launch, since the key is) before rounds 2.. of the generator.
template <int C, class F>
__device__ __forceinline__ void walk(uint64_t y, uint64_t e, uint64_t key, uint64_t c2, F &&f) {
    uint64_t t = round1_value(y);
#pragma unroll
    for (int j = 0; j < C; ++j) {
        const uint64_t z = add64(y, key);
        f(j, t, y, z);
        y = z;
        t = add64x3(t, e, c2 * static_cast<uint64_t>(j));
    }
}

// Every op maps a chunk of consecutive counters to W 32-bit words.
// EPC = output elements per counter.

struct OpU32 {
    static constexpr int kHeadParity = 0;
    using T = uint32_t;
    static constexpr int EPC = 1;
    template <int W>
    __device__ static void chunk(uint64_t y, uint64_t e, uint64_t key, uint64_t c2, uint32_t (&w)[W]) {
        walk<W>(y, e, key, c2, [&](int j, uint64_t t, uint64_t yy, uint64_t z) {
            w[j] = squares32_tyz(t, yy, z);
        });
    }
    __device__ static T single(uint64_t ctr0, uint64_t key, uint64_t e) {
        return squares32(ctr0 + e, key);
    }
};

struct OpU64 {
    static constexpr int kHeadParity = 0;
    using T = uint64_t;
    static constexpr int EPC = 1;
    template <int W>
    __device__ static void chunk(uint64_t y, uint64_t e, uint64_t key, uint64_t c2, uint32_t (&w)[W]) {
        walk<W / 2>(y, e, key, c2, [&](int j, uint64_t t, uint64_t yy, uint64_t z) {
            const uint64_t v = squares64_tyz(t, yy, z);
            w[2 * j] = lo32(v);
            w[2 * j + 1] = hi32(v);
        });
    }
    __device__ static T single(uint64_t ctr0, uint64_t key, uint64_t e) {
        return squares64(ctr0 + e, key);
    }
};

struct OpUniformF32 {
    static constexpr int kHeadParity = 0;
    using T = float;
    static constexpr int EPC = 1;
    template <int W>
    __device__ static void chunk(uint64_t y, uint64_t e, uint64_t key, uint64_t c2, uint32_t (&w)[W]) {
        walk<W>(y, e, key, c2, [&](int j, uint64_t t, uint64_t yy, uint64_t z) {
            w[j] = __float_as_uint(uniform24(squares32_tyz(t, yy, z)));
        });
    }
    __device__ static T single(uint64_t ctr0, uint64_t key, uint64_t e) {
        return uniform24(squares32(ctr0 + e, key));
    }
};

struct OpUniformBF16 {
    static constexpr int kHeadParity = 0;
    using T = uint16_t;
    static constexpr int EPC = 1;
    template <int W>
    __device__ static void chunk(uint64_t y, uint64_t e, uint64_t key, uint64_t c2, uint32_t (&w)[W]) {
        float f[2 * W];
        walk<2 * W>(y, e, key, c2, [&](int j, uint64_t t, uint64_t yy, uint64_t z) {
            f[j] = uniform24(squares32_tyz(t, yy, z));
        });
#pragma unroll
        for (int j = 0; j < W; ++j) w[j] = pack_bf16_rz(f[2 * j], f[2 * j + 1]);
    }
    __device__ static T single(uint64_t ctr0, uint64_t key, uint64_t e) {
        return static_cast<T>(bf16_bits_rz(uniform24(squares32(ctr0 + e, key))));
    }
};

struct OpNormalF32 {
    static constexpr int kHeadParity = 0;
    using T = float;
    static constexpr int EPC = 2;
    // the two elements of one counter
    __device__ static uint2 pair(uint64_t t, uint64_t y, uint64_t z) {
        const uint64_t v = squares64_tyz(t, y, z);
        const float2 n = box_muller(hi32(v), lo32(v));
        return make_uint2(__float_as_uint(n.x), __float_as_uint(n.y));
    }
    template <int W>
    __device__ static void chunk(uint64_t y, uint64_t e, uint64_t key, uint64_t c2, uint32_t (&w)[W]) {
        walk<W / 2>(y, e, key, c2, [&](int j, uint64_t t, uint64_t yy, uint64_t z) {
            const uint2 v = pair(t, yy, z);
            w[2 * j] = v.x;
            w[2 * j + 1] = v.y;
        });
    }
    __device__ static T single(uint64_t ctr0, uint64_t key, uint64_t e) {
        const uint64_t v = squares64(ctr0 + e / 2, key);
        const float2 z = box_muller(hi32(v), lo32(v));
        return (e & 1) ? z.y : z.x;
    }
};

// Two floats per squares64 output: the upper 32 bits, then the lower
// (Section 5's split into halves), each as floor(half / 2^8) * 2^-24.
struct OpUniform2F32 {
    static constexpr int kHeadParity = 0;
    using T = float;
    static constexpr int EPC = 2;
    __device__ static uint2 pair(uint64_t t, uint64_t y, uint64_t z) {
        const uint64_t v = squares64_tyz(t, y, z);
        return make_uint2(__float_as_uint(uniform24(hi32(v))), __float_as_uint(uniform24(lo32(v))));
    }
    template <int W>
    __device__ static void chunk(uint64_t y, uint64_t e, uint64_t key, uint64_t c2, uint32_t (&w)[W]) {
        walk<W / 2>(y, e, key, c2, [&](int j, uint64_t t, uint64_t yy, uint64_t z) {
            const uint2 v = pair(t, yy, z);
            w[2 * j] = v.x;
            w[2 * j + 1] = v.y;
        });
    }
    __device__ static T single(uint64_t ctr0, uint64_t key, uint64_t e) {
        const uint64_t v = squares64(ctr0 + e / 2, key);
        return uniform24((e & 1) ? lo32(v) : hi32(v));
    }
};

// A two-elements-per-counter op whose chunks start at the second element of
// a counter's pair: an output pointer that is 4-byte but not 8-byte aligned
// puts the 16- and 32-byte boundaries at odd element indices. A chunk of W
// elements then spans W/2 + 1 counters: the first contributes its second
// element, the last its first, so each chunk computes one pair more than it
// stores (W/2 + 1 for W/2), and the vector stores stay aligned.
template <class Op>
struct OddPairs {
    static constexpr int kHeadParity = 1;
    using T = typename Op::T;
    static constexpr int EPC = 2;
    template <int W>
    __device__ static void chunk(uint64_t y, uint64_t e, uint64_t key, uint64_t c2, uint32_t (&w)[W]) {
        walk<W / 2 + 1>(y, e, key, c2, [&](int j, uint64_t t, uint64_t yy, uint64_t z) {
            const uint2 v = Op::pair(t, yy, z);
            if (j > 0) w[2 * j - 1] = v.x;
            if (j < W / 2) w[2 * j] = v.y;
        });
    }
    __device__ static T single(uint64_t ctr0, uint64_t key, uint64_t e) { return Op::single(ctr0, key, e); }
};

// Store ceiling: the plain kernels' chunking, grid and store path with no
// generator arithmetic; every element is the 32-bit value passed in place
// of the key, and the counter-base argument carries a pause in nanoseconds
// that each thread takes after each chunk (paced writers: a store stream
// that saturates the memory system runs slower than one that leaves gaps).
struct OpFill {
    static constexpr int kHeadParity = 0;
    using T = uint32_t;
    static constexpr int EPC = 1;
    template <int W>
    __device__ static void chunk(uint64_t, uint64_t, uint64_t key, uint64_t, uint32_t (&w)[W]) {
#pragma unroll
        for (int j = 0; j < W; ++j) w[j] = static_cast<uint32_t>(key);
    }
    __device__ static T single(uint64_t, uint64_t key, uint64_t) { return static_cast<uint32_t>(key); }
};

// 53-bit double uniforms floor(squares64 / 2^11) * 2^-53, built with
// integer operations only (see uniform53_bits).
// 53-bit doubles. Per value the chunk takes the conversion's common path,
// exact whenever v >= 2^43 (the upper word of v >> 11 is non-zero), and
// flags the other values (probability 2^-21 each); when any active lane of
// the warp flagged one, the flagged values are recomputed with the full
// conversion. Keeping the rare path out of the per-value code matters: with
// it inline, the compiler predicated it into every value (37.1 against 33.1
// warp instructions per warp of outputs, 12 % slower).
__device__ __forceinline__ uint64_t uniform53_bits_common(uint64_t v) {
    const uint32_t kh = static_cast<uint32_t>(v >> 43);
    const uint32_t kl = static_cast<uint32_t>(v >> 11);
    const uint32_t pos = 31 - __clz(static_cast<int>(kh));  // 0..20 when kh != 0
    const uint32_t sh = 20 - pos;
    const uint32_t mhi = __funnelshift_l(kl, kh, sh);
    const uint32_t mlo = kl << sh;
    return (static_cast<uint64_t>(((1001u + pos) << 20) + mhi) << 32) | mlo;
}

struct OpUniformF64 {
    static constexpr int kHeadParity = 0;
    using T = double;
    static constexpr int EPC = 1;
    template <int W>
    __device__ static void chunk(uint64_t y, uint64_t e, uint64_t key, uint64_t c2, uint32_t (&w)[W]) {
        uint32_t rare = 0;
        walk<W / 2>(y, e, key, c2, [&](int j, uint64_t t, uint64_t yy, uint64_t z) {
            const uint64_t v = squares64_tyz(t, yy, z);
            const uint64_t b = uniform53_bits_common(v);
            rare |= static_cast<uint32_t>(v < (uint64_t{1} << 43)) << j;
            w[2 * j] = lo32(b);
            w[2 * j + 1] = hi32(b);
        });
        // The vote covers the lanes still walking chunks (at the end of the
        // vector region some lanes of a warp have finished theirs).
        if (__any_sync(__activemask(), rare != 0u)) {
#pragma unroll
            for (int j = 0; j < W / 2; ++j) {
                if (rare & (1u << j)) {
                    const uint64_t yy = y + static_cast<uint64_t>(j) * key;
                    const uint64_t b = uniform53_bits(squares64_yz(yy, add64(yy, key)));
                    w[2 * j] = lo32(b);
                    w[2 * j + 1] = hi32(b);
                }
            }
        }
    }
    __device__ static T single(uint64_t ctr0, uint64_t key, uint64_t e) {
        return __longlong_as_double(static_cast<long long>(uniform53_bits(squares64(ctr0 + e, key))));
    }
};

template <int BYTES, bool CS>
__device__ __forceinline__ void store_chunk(void *p, const uint32_t (&w)[BYTES / 4]) {
    if constexpr (BYTES == 64) {
        store32B<CS>(p, *reinterpret_cast<const uint32_t(*)[8]>(&w[0]));
        store32B<CS>(static_cast<char *>(p) + 32, *reinterpret_cast<const uint32_t(*)[8]>(&w[8]));
    } else if constexpr (BYTES == 32) {
        store32B<CS>(p, w);
    } else {
        store16B<CS>(p, w[0], w[1], w[2], w[3]);
    }
}

// After each chunk: a pause for the store-ceiling kernel (ctr0 carries its
// length in nanoseconds), nothing for the generators.
template <class Op>
__device__ __forceinline__ void pace(uint64_t ctr0) {
    if constexpr (std::is_same<Op, OpFill>::value) {
        if (ctr0 != 0) __nanosleep(static_cast<unsigned>(ctr0));
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
    const uint64_t c2 = (key * key) << 1;
    uint64_t e = round1_delta(y, key);
    // Between chunks the counter jumps by nthreads*CPV: y by that many keys,
    // e (linear in the counter) by that many c2.
    const uint64_t ystep = nthreads * CPV * key;
    const uint64_t estep = nthreads * CPV * c2;
    char *p = reinterpret_cast<char *>(out + head) + tid * BYTES;
    const uint64_t pstep = nthreads * BYTES;
    for (uint64_t it = (nvec - tid + nthreads - 1) / nthreads; it != 0; --it) {
        uint32_t w[W];
        Op::template chunk<W>(y, e, key, c2, w);
        store_chunk<BYTES, CS>(p, w);
        pace<Op>(ctr0);
        y = add64(y, ystep);
        e = add64(e, estep);
        p += pstep;
    }
}

// TMA bulk-store body: each warp stages 32 lanes x 64 bytes (2 KiB of
// consecutive output) in shared memory, double-buffered, and one lane hands
// each full buffer to the copy engine with cp.async.bulk (shared -> global).
// The lane waits with cp.async.bulk.wait_group.read until the copy issued
// two steps earlier has finished reading a buffer before the warp refills
// it, and waits for all of its copies before the CTA exits. The warp
// chunks cover [head, head + nwc * 2 KiB / sizeof(T)); the rest is written
// element by element.
constexpr int kBulkLaneBytes = 64;
constexpr int kBulkWarpBytes = 32 * kBulkLaneBytes;

template <class Op>
__global__ void __launch_bounds__(512)
    plain_bulk_kernel(uint64_t key, uint64_t ctr0, typename Op::T *__restrict__ out, uint64_t n,
                      uint64_t head, uint64_t nwc) {
    using T = typename Op::T;
    constexpr int W = kBulkLaneBytes / 4;
    constexpr int EPV = kBulkLaneBytes / sizeof(T);
    constexpr int CPV = EPV / Op::EPC;
    constexpr int WC_ELEMS = 32 * EPV;
    extern __shared__ __align__(128) unsigned char stage_all[];
    const int lane = threadIdx.x & 31;
    const uint64_t tid = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const uint64_t nthreads = static_cast<uint64_t>(gridDim.x) * blockDim.x;

    const uint64_t tail0 = head + nwc * WC_ELEMS;
    for (uint64_t e = tid; e < head; e += nthreads) out[e] = Op::single(ctr0, key, e);
    for (uint64_t e = tail0 + tid; e < n; e += nthreads) out[e] = Op::single(ctr0, key, e);

    const uint64_t gwarp = tid >> 5;
    const uint64_t nwarps = nthreads >> 5;
    if (gwarp >= nwc) return;  // uniform across the warp

    const uint32_t stage = static_cast<uint32_t>(__cvta_generic_to_shared(
        stage_all + (threadIdx.x >> 5) * 2 * kBulkWarpBytes));
    uint64_t y = (ctr0 + (head + gwarp * WC_ELEMS + lane * EPV) / Op::EPC) * key;
    const uint64_t c2 = (key * key) << 1;
    uint64_t e = round1_delta(y, key);
    const uint64_t ystep = nwarps * 32 * CPV * key;
    const uint64_t estep = nwarps * 32 * CPV * c2;
    char *gp = reinterpret_cast<char *>(out + head) + gwarp * kBulkWarpBytes;
    const uint64_t gstep = nwarps * kBulkWarpBytes;
    uint32_t buf = 0;
    for (uint64_t c = gwarp; c < nwc; c += nwarps) {
        if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
        __syncwarp();
        uint32_t w[W];
        Op::template chunk<W>(y, e, key, c2, w);
        const uint32_t s = stage + buf * kBulkWarpBytes + lane * kBulkLaneBytes;
#pragma unroll
        for (int q = 0; q < W / 4; ++q)
            asm volatile("st.shared.v4.b32 [%0], {%1,%2,%3,%4};" ::"r"(s + 16 * q), "r"(w[4 * q]),
                         "r"(w[4 * q + 1]), "r"(w[4 * q + 2]), "r"(w[4 * q + 3])
                         : "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
            asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gp),
                         "r"(stage + buf * kBulkWarpBytes), "n"(kBulkWarpBytes)
                         : "memory");
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        }
        pace<Op>(ctr0);
        y = add64(y, ystep);
        e = add64(e, estep);
        gp += gstep;
        buf ^= 1u;
    }
    if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Variants (bytes written per thread per step, cache policy):
// 0 = 32 B, 1 = 32 B streaming, 2 = 16 B, 3 = 16 B streaming,
// 4 = 64 B (two adjacent 32 B stores), 5 = 64 B streaming,
// 6 = 64 B per lane staged in shared memory, TMA bulk store per warp.
constexpr int kPlainVariants = 7;
constexpr int kBulkVariant = 6;
const char *kPlainVariantNames[kPlainVariants] = {"st32", "st32.cs", "st16", "st16.cs",
                                                  "st32x2", "st32x2.cs", "bulk64"};

constexpr int variant_bytes(int v) { return v < 2 ? 32 : (v < 4 ? 16 : 64); }

size_t bulk_smem(int block) { return static_cast<size_t>(block / 32) * 2 * kBulkWarpBytes; }

template <class Op>
const void *plain_fn(int variant) {
    switch (variant) {
        case 0: return reinterpret_cast<const void *>(&plain_kernel<Op, 32, false>);
        case 1: return reinterpret_cast<const void *>(&plain_kernel<Op, 32, true>);
        case 2: return reinterpret_cast<const void *>(&plain_kernel<Op, 16, false>);
        case 3: return reinterpret_cast<const void *>(&plain_kernel<Op, 16, true>);
        case 4: return reinterpret_cast<const void *>(&plain_kernel<Op, 64, false>);
        case 5: return reinterpret_cast<const void *>(&plain_kernel<Op, 64, true>);
        default: return reinterpret_cast<const void *>(&plain_bulk_kernel<Op>);
    }
}

// The bulk body needs up to 64 KiB of dynamic shared memory (block 512):
// opt in once per instantiation.
template <class Op>
cudaError_t prepare_bulk() {
    static cudaError_t status = cudaFuncSetAttribute(
        reinterpret_cast<const void *>(&plain_bulk_kernel<Op>),
        cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bulk_smem(512)));
    return status;
}

const void *plain_fn_for(int kernel_id, int variant) {
    switch (kernel_id) {
        case SQ_KERNEL_U32: return plain_fn<OpU32>(variant);
        case SQ_KERNEL_U64: return plain_fn<OpU64>(variant);
        case SQ_KERNEL_UNIFORM_F32: return plain_fn<OpUniformF32>(variant);
        case SQ_KERNEL_UNIFORM_BF16: return plain_fn<OpUniformBF16>(variant);
        case SQ_KERNEL_NORMAL_F32: return plain_fn<OpNormalF32>(variant);
        case SQ_KERNEL_UNIFORM2_F32: return plain_fn<OpUniform2F32>(variant);
        case SQ_KERNEL_UNIFORM_F64: return plain_fn<OpUniformF64>(variant);
        case kFillKernelId: return plain_fn<OpFill>(variant);
        default: return nullptr;
    }
}

template <class Op>
cudaError_t launch_bulk(const Cfg &cfg, uint64_t key, uint64_t ctr0, size_t n, void *out,
                        cudaStream_t stream, int max_ctas) {
    using T = typename Op::T;
    const cudaError_t prep = prepare_bulk<Op>();
    if (prep != cudaSuccess) return prep;
    const size_t wc_elems = 32 * kBulkLaneBytes / sizeof(T);
    const uintptr_t addr = reinterpret_cast<uintptr_t>(out);
    size_t head = ((32 - (addr % 32)) % 32) / sizeof(T);
    if (head > n) head = n;
    if (head % Op::EPC != Op::kHeadParity) head = n;  // chunk form of the other parity: all singles
    const size_t nwc = (n - head) / wc_elems;
    const int ctas = cfg.ctas_per_sm > 0 ? cfg.ctas_per_sm : max_ctas;
    uint64_t grid = static_cast<uint64_t>(current_sm_count()) * (ctas > 0 ? ctas : 1);
    const uint64_t warps_per_cta = cfg.block / 32;
    const uint64_t need = (nwc + warps_per_cta - 1) / warps_per_cta;
    const uint64_t need_single = (head + (n - head - nwc * wc_elems) + cfg.block - 1) / cfg.block;
    const uint64_t want = need > need_single ? need : need_single;
    if (grid > want) grid = want > 0 ? want : 1;
    plain_bulk_kernel<Op><<<grid, cfg.block, bulk_smem(cfg.block), stream>>>(
        key, ctr0, static_cast<T *>(out), n, head, nwc);
    return cudaGetLastError();
}

template <class Op>
cudaError_t launch_op(const Cfg &cfg, uint64_t key, uint64_t ctr0, size_t n, void *out,
                      cudaStream_t stream, int max_ctas) {
    using T = typename Op::T;
    if (cfg.variant == kBulkVariant) return launch_bulk<Op>(cfg, key, ctr0, n, out, stream, max_ctas);
    const int bytes = variant_bytes(cfg.variant);
    const int align = bytes > 32 ? 32 : bytes;  // each store is at most 32 B
    const size_t epv = bytes / sizeof(T);
    const uintptr_t addr = reinterpret_cast<uintptr_t>(out);
    size_t head = ((align - (addr % align)) % align) / sizeof(T);
    if (head > n) head = n;
    if (head % Op::EPC != Op::kHeadParity) head = n;  // chunk form of the other parity: all singles
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
        case 3: plain_kernel<Op, 16, true><<<grid, cfg.block, 0, stream>>>(key, ctr0, o, n, head, nvec); break;
        case 4: plain_kernel<Op, 64, false><<<grid, cfg.block, 0, stream>>>(key, ctr0, o, n, head, nvec); break;
        default: plain_kernel<Op, 64, true><<<grid, cfg.block, 0, stream>>>(key, ctr0, o, n, head, nvec); break;
    }
    return cudaGetLastError();
}

// Elements before the first aligned chunk for a variant: the bulk body and
// the 32- and 64-byte bodies start at a 32-byte boundary, the 16-byte ones at
// a 16-byte boundary.
size_t head_elems(int variant, const void *out, size_t elem, size_t n) {
    const size_t align = variant == kBulkVariant ? 32 : (variant_bytes(variant) > 32 ? 32 : variant_bytes(variant));
    const size_t head = ((align - (reinterpret_cast<uintptr_t>(out) % align)) % align) / elem;
    return head > n ? n : head;
}

template <class Op>
cudaError_t launch_kind(const Cfg &c, uint64_t key, uint64_t ctr_base, size_t n, void *out,
                        cudaStream_t stream) {
    if constexpr (Op::EPC == 2) {
        // An odd head (a 4-byte but not 8-byte aligned float pointer) takes
        // the chunk form that starts mid-pair.
        if (head_elems(c.variant, out, sizeof(typename Op::T), n) % 2 == 1) {
            using Odd = OddPairs<Op>;
            if (c.variant == kBulkVariant) prepare_bulk<Odd>();
            const int max_ctas = c.ctas_per_sm > 0
                                     ? c.ctas_per_sm
                                     : occupancy(plain_fn<Odd>(c.variant), c.block,
                                                 c.variant == kBulkVariant ? bulk_smem(c.block) : 0);
            return launch_op<Odd>(c, key, ctr_base, n, out, stream, max_ctas);
        }
    }
    if (c.variant == kBulkVariant) prepare_bulk<Op>();
    const int max_ctas = c.ctas_per_sm > 0
                             ? c.ctas_per_sm
                             : occupancy(plain_fn<Op>(c.variant), c.block,
                                         c.variant == kBulkVariant ? bulk_smem(c.block) : 0);
    return launch_op<Op>(c, key, ctr_base, n, out, stream, max_ctas);
}

}  // namespace

int plain_num_variants() { return kPlainVariants; }

const char *plain_variant_name(int variant) {
    return (variant >= 0 && variant < kPlainVariants) ? kPlainVariantNames[variant] : nullptr;
}

int plain_max_ctas_per_sm(int kernel_id, int variant, int block) {
    const void *fn = plain_fn_for(kernel_id, variant);
    if (!fn) return 1;
    const size_t smem = variant == kBulkVariant ? bulk_smem(block) : 0;
    if (variant == kBulkVariant) {
        // the opt-in must precede the occupancy query for > 48 KiB
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(bulk_smem(512)));
    }
    return occupancy(fn, block, smem);
}

cudaError_t launch_plain(int kernel_id, const Cfg &cfg, uint64_t key, uint64_t ctr_base, size_t n,
                         void *out, cudaStream_t stream) {
    if (n == 0) return cudaSuccess;
    Cfg c = cfg;
    // Outputs outside device memory (pinned or system host memory, written
    // over the host link) take the 32-byte-per-lane stores, where one warp
    // store fills a contiguous 1 KiB. The 64-byte-per-lane forms leave each
    // 128 B line half written per store, which halves the link's write rate,
    // and the bulk copy stages for device memory only.
    if (variant_bytes(c.variant) > 32 && !in_device_memory(out)) c.variant = c.variant == 5 ? 1 : 0;
    switch (kernel_id) {
        case SQ_KERNEL_U32: return launch_kind<OpU32>(c, key, ctr_base, n, out, stream);
        case SQ_KERNEL_U64: return launch_kind<OpU64>(c, key, ctr_base, n, out, stream);
        case SQ_KERNEL_UNIFORM_F32: return launch_kind<OpUniformF32>(c, key, ctr_base, n, out, stream);
        case SQ_KERNEL_UNIFORM_BF16: return launch_kind<OpUniformBF16>(c, key, ctr_base, n, out, stream);
        case SQ_KERNEL_NORMAL_F32: return launch_kind<OpNormalF32>(c, key, ctr_base, n, out, stream);
        case SQ_KERNEL_UNIFORM2_F32: return launch_kind<OpUniform2F32>(c, key, ctr_base, n, out, stream);
        case SQ_KERNEL_UNIFORM_F64: return launch_kind<OpUniformF64>(c, key, ctr_base, n, out, stream);
        case kFillKernelId: return launch_kind<OpFill>(c, key, ctr_base, n, out, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sq
