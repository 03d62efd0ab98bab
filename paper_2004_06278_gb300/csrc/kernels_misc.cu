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

// The same in chunks of 16 squares32 values (two adjacent 32-byte stores,
// 512-thread CTAs) or 4 squares64 values (one 32-byte store, 256-thread
// CTAs): elements before the first 32-byte boundary of out and after the
// last whole chunk are written one per thread; thread t of the grid writes
// chunks t, t + T, ... Inside a chunk y steps by S = stride*key and z = y +
// key; round 1 (t = y*y + y) advances by round1_delta(y, S) + j * 2S^2 for
// the chunk's j-th element (one three-input addition; the j * 2S^2 are the
// same in every thread), and between a thread's chunks y and that delta jump
// by T * (elements per chunk) steps. (Measured at stride 3: squares32 in
// chunks of 8 with 256 threads 7 % slower; squares64 in chunks of 8 with
// 512 threads no faster.)
template <bool WIDE>
constexpr int strided_block() {
    return WIDE ? 256 : 512;
}

template <bool WIDE>
__global__ void __launch_bounds__(strided_block<WIDE>())
    strided_vec_kernel(uint64_t key, uint64_t ctr0, uint64_t stride, void *__restrict__ out, uint64_t n,
                       uint64_t head, uint64_t nvec) {
    constexpr int EPV = WIDE ? 4 : 16;
    constexpr int CHUNK = WIDE ? 32 : 64;  // bytes
    const uint64_t tid = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const uint64_t nt = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    const uint64_t tail0 = head + nvec * EPV;
    auto single = [&](uint64_t e) {
        const uint64_t y = (ctr0 + e * stride) * key;
        if constexpr (WIDE)
            static_cast<uint64_t *>(out)[e] = squares64_yz(y, add64(y, key));
        else
            static_cast<uint32_t *>(out)[e] = squares32_yz(y, add64(y, key));
    };
    for (uint64_t e = tid; e < head; e += nt) single(e);
    for (uint64_t e = tail0 + tid; e < n; e += nt) single(e);
    if (tid >= nvec) return;
    const uint64_t S = stride * key;
    const uint64_t c2 = (S * S) << 1;
    uint64_t y = (ctr0 + (head + tid * EPV) * stride) * key;
    uint64_t e0 = round1_delta(y, S);
    const uint64_t ystep = nt * EPV * S;
    const uint64_t estep = nt * EPV * c2;
    char *p = reinterpret_cast<char *>(out) + head * (WIDE ? 8 : 4) + tid * CHUNK;
    const uint64_t pstep = nt * CHUNK;
    for (uint64_t it = (nvec - tid + nt - 1) / nt; it != 0; --it) {
        uint32_t w[16];
        uint64_t yy = y;
        uint64_t t = round1_value(y);
#pragma unroll
        for (int j = 0; j < EPV; ++j) {
            const uint64_t z = add64(yy, key);
            if constexpr (WIDE) {
                const uint64_t v = squares64_tyz(t, yy, z);
                w[2 * j] = lo32(v);
                w[2 * j + 1] = hi32(v);
            } else {
                w[j] = squares32_tyz(t, yy, z);
            }
            yy = add64(yy, S);
            t = add64x3(t, e0, c2 * static_cast<uint64_t>(j));
        }
        store32B<false>(p, *reinterpret_cast<const uint32_t(*)[8]>(&w[0]));
        if constexpr (!WIDE) store32B<false>(p + 32, *reinterpret_cast<const uint32_t(*)[8]>(&w[8]));
        y = add64(y, ystep);
        e0 = add64(e0, estep);
        p += pstep;
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

// squares64 with keys and out 16-byte aligned: two keys per thread per step
// (one 16-byte load, one 16-byte store of the two values); an odd last key is
// taken by one thread. (Measured on 2^27 keys: 0.40 against 0.36 Tkeys/s
// one key per thread; four keys per thread, two loads and two stores, no
// faster than one.)
__global__ void __launch_bounds__(256)
    keys64_kernel_x2(const uint64_t *__restrict__ keys, uint64_t n, uint64_t ctr, uint64_t *__restrict__ out) {
    const uint64_t tid = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const uint64_t nt = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    const uint64_t ng = n / 2;
    const ulonglong2 *kv = reinterpret_cast<const ulonglong2 *>(keys);
    ulonglong2 *ov = reinterpret_cast<ulonglong2 *>(out);
    for (uint64_t g = tid; g < ng; g += nt) {
        const ulonglong2 k = __ldg(kv + g);
        const uint64_t ya = ctr * k.x, yb = ctr * k.y;
        ov[g] = make_ulonglong2(squares64_yz(ya, add64(ya, k.x)), squares64_yz(yb, add64(yb, k.y)));
    }
    if (tid == 0 && (n & 1)) {
        const uint64_t k = __ldg(keys + n - 1);
        const uint64_t y = ctr * k;
        out[n - 1] = squares64_yz(y, add64(y, k));
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
    const size_t es = wide ? 8 : 4;
    const size_t epv = wide ? 4 : 16;
    const int block = wide ? strided_block<true>() : strided_block<false>();
    if (n >= 64 * epv) {
        // whole chunks from the first 32-byte boundary of out
        const uintptr_t addr = reinterpret_cast<uintptr_t>(out);
        const uint64_t head = ((32 - addr % 32) % 32) / es;
        const uint64_t nvec = (n - head) / epv;
        const void *fn = wide ? reinterpret_cast<const void *>(&strided_vec_kernel<true>)
                              : reinterpret_cast<const void *>(&strided_vec_kernel<false>);
        const uint64_t full = static_cast<uint64_t>(current_sm_count()) * occupancy(fn, block, 0);
        const uint64_t need = (nvec + block - 1) / block;
        const unsigned grid = static_cast<unsigned>(need < full ? need : full);
        if (wide)
            strided_vec_kernel<true><<<grid, block, 0, stream>>>(key, ctr_base, stride, out, n, head, nvec);
        else
            strided_vec_kernel<false><<<grid, block, 0, stream>>>(key, ctr_base, stride, out, n, head, nvec);
        return cudaGetLastError();
    }
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
    // one per thread), two for squares64 (0.40 against 0.36), given 16-byte
    // aligned keys and out.
    const bool a16 = reinterpret_cast<uintptr_t>(keys) % 16 == 0 && reinterpret_cast<uintptr_t>(out) % 16 == 0;
    if (a16 && !wide) {
        keys_kernel_x4<<<grid_for((n + 3) / 4, reinterpret_cast<const void *>(&keys_kernel_x4)), 256, 0,
                         stream>>>(keys, n, ctr, static_cast<uint32_t *>(out));
    } else if (a16 && wide) {
        keys64_kernel_x2<<<grid_for((n + 1) / 2, reinterpret_cast<const void *>(&keys64_kernel_x2)), 256, 0,
                           stream>>>(keys, n, ctr, static_cast<uint64_t *>(out));
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
