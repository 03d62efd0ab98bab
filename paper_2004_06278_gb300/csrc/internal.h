// Internal C++ interface between the C ABI (api.cpp) and the kernel
// translation units. Not installed; the public interface is squares.h.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "squares.h"

namespace sq {

struct Cfg {
    int variant;
    int block;
    int ctas_per_sm;  // 0 = as many as fit
};

// Streaming multiprocessors of the current device (cached per device).
int current_sm_count();

// Resident CTAs per SM for a kernel, block size and dynamic shared memory on
// the current device (cudaOccupancyMaxActiveBlocksPerMultiprocessor, cached;
// at least 1).
int occupancy(const void *kernel, int block, size_t smem);

// True when `p` is device memory of the current context. Pinned, registered
// or plain system host memory (written over the host link) gives false.
bool in_device_memory(const void *p);

// --- plain generators (sq_u32, sq_u64, uniform, bf16, normal) -------------
// kernel_id is one of SQ_KERNEL_U32, _U64, _UNIFORM_F32, _UNIFORM_BF16,
// _NORMAL_F32, _UNIFORM2_F32, _UNIFORM_F64, or kFillKernelId (the
// write-only store-ceiling kernel: uint32 elements, all equal to the low 32
// bits of `key`). `out` is the caller's buffer; element type per kernel.
constexpr int kFillKernelId = 100;
int plain_num_variants();
const char *plain_variant_name(int variant);
cudaError_t launch_plain(int kernel_id, const Cfg &cfg, uint64_t key, uint64_t ctr_base,
                         size_t n, void *out, cudaStream_t stream);
int plain_max_ctas_per_sm(int kernel_id, int variant, int block);

// --- ragged batch --------------------------------------------------------
int batch_num_variants();
const char *batch_variant_name(int variant);
cudaError_t launch_batch(const Cfg &cfg, const uint64_t *keys, const uint64_t *bases,
                         const int64_t *lengths, const int64_t *offsets, size_t nstreams,
                         uint32_t *out, cudaStream_t stream);
int batch_max_ctas_per_sm(int variant, int block);

// --- generation-only statistics -----------------------------------------
int fused_num_variants();
const char *fused_variant_name(int variant);
cudaError_t launch_fused(const Cfg &cfg, const uint64_t *keys, const uint64_t *bases,
                         size_t nstreams, uint64_t ctrs_per_stream, uint32_t *xor_out,
                         uint64_t *sum_top, uint64_t *hist256, cudaStream_t stream);
int fused_max_ctas_per_sm(int variant, int block);

// --- strided counters and key-counter mode -------------------------------
cudaError_t launch_strided(bool wide, uint64_t key, uint64_t ctr_base, uint64_t stride, size_t n,
                           void *out, cudaStream_t stream);
cudaError_t launch_keys(bool wide, const uint64_t *keys, size_t n, uint64_t ctr, void *out,
                        cudaStream_t stream);

// --- keys (host) ---------------------------------------------------------
int make_keys(uint64_t seed, size_t n, uint64_t *keys);

}  // namespace sq
