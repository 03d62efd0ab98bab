// Strided counters (Section 4's "increments other than one") and
// key-counter mode (Section 4: one counter, many keys). Neither is on the
// throughput path; both write one element per thread per step, coalesced
// (adjacent threads write adjacent elements).
#include <cuda_runtime.h>

#include "internal.h"
#include "squares_device.cuh"
#include "stores.cuh"

namespace sq {
namespace {

// out[e] = squares(ctr0 + e*stride, key): y advances by T*stride*key per
// step, and z = y + key as the definition asks for whatever the stride.
template <bool WIDE>
__global__ void __launch_bounds__(256)
    strided_kernel(uint64_t key, uint64_t ctr0, uint64_t stride, void *__restrict__ out, uint64_t n) {
    const uint64_t tid = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const uint64_t nt = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    if (tid >= n) return;
    uint64_t y = (ctr0 + tid * stride) * key;
    const uint64_t ystep = nt * stride * key;
    for (uint64_t e = tid; e < n; e += nt) {
        const uint64_t z = add64(y, key);
        if constexpr (WIDE)
            static_cast<uint64_t *>(out)[e] = squares64_yz(y, z);
        else
            static_cast<uint32_t *>(out)[e] = squares32_yz(y, z);
        y = add64(y, ystep);
    }
}

// out[e] = squares(ctr, keys[e]).
template <bool WIDE>
__global__ void __launch_bounds__(256)
    keys_kernel(const uint64_t *__restrict__ keys, uint64_t n, uint64_t ctr, void *__restrict__ out) {
    const uint64_t tid = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const uint64_t nt = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    for (uint64_t e = tid; e < n; e += nt) {
        const uint64_t k = __ldg(keys + e);
        const uint64_t y = ctr * k;
        const uint64_t z = add64(y, k);
        if constexpr (WIDE)
            static_cast<uint64_t *>(out)[e] = squares64_yz(y, z);
        else
            static_cast<uint32_t *>(out)[e] = squares32_yz(y, z);
    }
}

// squares32 with keys and out 16-byte aligned: a thread takes four keys per
// step (two 16-byte loads, one 16-byte store of the four values), so more
// loads are in flight per thread; the last n mod 4 keys are taken one per
// thread.
__global__ void __launch_bounds__(256)
    keys_kernel_x4(const uint64_t *__restrict__ keys, uint64_t n, uint64_t ctr, uint32_t *__restrict__ out) {
    const uint64_t tid = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const uint64_t nt = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    const uint64_t ng = n / 4;
    const ulonglong2 *kv = reinterpret_cast<const ulonglong2 *>(keys);
    for (uint64_t g = tid; g < ng; g += nt) {
        const ulonglong2 a = __ldg(kv + 2 * g);
        const ulonglong2 b = __ldg(kv + 2 * g + 1);
        const uint64_t k[4] = {a.x, a.y, b.x, b.y};
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint64_t y = ctr * k[j];
            w[j] = squares32_yz(y, add64(y, k[j]));
        }
        store16B<false>(out + 4 * g, w[0], w[1], w[2], w[3]);
    }
    for (uint64_t e = 4 * ng + tid; e < n; e += nt) {
        const uint64_t k = __ldg(keys + e);
        const uint64_t y = ctr * k;
        out[e] = squares32_yz(y, add64(y, k));
    }
}

unsigned grid_for(uint64_t n, const void *fn) {
    const int per_sm = occupancy(fn, 256, 0);
    const uint64_t full = static_cast<uint64_t>(current_sm_count()) * per_sm;
    const uint64_t need = (n + 255) / 256;
    return static_cast<unsigned>(need < full ? (need > 0 ? need : 1) : full);
}

}  // namespace

cudaError_t launch_strided(bool wide, uint64_t key, uint64_t ctr_base, uint64_t stride, size_t n,
                           void *out, cudaStream_t stream) {
    if (n == 0) return cudaSuccess;
    if (wide) {
        strided_kernel<true><<<grid_for(n, reinterpret_cast<const void *>(&strided_kernel<true>)), 256, 0,
                               stream>>>(key, ctr_base, stride, out, n);
    } else {
        strided_kernel<false><<<grid_for(n, reinterpret_cast<const void *>(&strided_kernel<false>)), 256, 0,
                                stream>>>(key, ctr_base, stride, out, n);
    }
    return cudaGetLastError();
}

cudaError_t launch_keys(bool wide, const uint64_t *keys, size_t n, uint64_t ctr, void *out,
                        cudaStream_t stream) {
    if (n == 0) return cudaSuccess;
    // Four keys per thread for squares32 (measured 0.56 against 0.43 Tkeys/s
    // one per thread); squares64, with twice the bytes out, gains nothing.
    const bool x4 = !wide && reinterpret_cast<uintptr_t>(keys) % 16 == 0 &&
                    reinterpret_cast<uintptr_t>(out) % 16 == 0;
    if (x4) {
        keys_kernel_x4<<<grid_for((n + 3) / 4, reinterpret_cast<const void *>(&keys_kernel_x4)), 256, 0,
                         stream>>>(keys, n, ctr, static_cast<uint32_t *>(out));
    } else if (wide) {
        keys_kernel<true><<<grid_for(n, reinterpret_cast<const void *>(&keys_kernel<true>)), 256, 0, stream>>>(
            keys, n, ctr, out);
    } else {
        keys_kernel<false><<<grid_for(n, reinterpret_cast<const void *>(&keys_kernel<false>)), 256, 0, stream>>>(
            keys, n, ctr, out);
    }
    return cudaGetLastError();
}

}  // namespace sq
