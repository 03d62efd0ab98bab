"""The public device header (include/squares_device.cuh) used by a kernel
outside the library: a consumer compiled here with nvcc draws squares32 /
squares64 values in registers -- by counter, and through WeylStream -- and
must equal the oracle bit for bit. This is how a fused consumer (dropout
mask, Monte Carlo path) gets the same numbers sq_u32 / sq_u64 would store."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2004_06278_gb300 import build as libbuild

pytestmark = pytest.mark.gpu

CONSUMER = r'''
#include <cstdint>
#include <cuda_runtime.h>
#include "squares_device.cuh"

__global__ void by_counter(uint64_t key, uint64_t ctr0, uint64_t n, uint32_t *o32, uint64_t *o64,
                           double *of64) {
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    o32[i] = sq::squares32(ctr0 + i, key);
    o64[i] = sq::squares64(ctr0 + i, key);
    of64[i] = __longlong_as_double((long long)sq::uniform53_bits(sq::squares64(ctr0 + i, key)));
}

__global__ void by_stream(uint64_t key, uint64_t ctr0, uint64_t per, uint64_t step, uint64_t nthreads,
                          uint32_t *o32, uint64_t *o64) {
    const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (t >= nthreads) return;
    sq::WeylStream a(ctr0 + t * per * step, key, step), b(ctr0 + t * per * step, key, step);
    for (uint64_t j = 0; j < per; ++j) {
        o32[t * per + j] = a.next32();
        o64[t * per + j] = b.next64();
    }
}

extern "C" int run_by_counter(uint64_t key, uint64_t ctr0, uint64_t n, uint32_t *o32, uint64_t *o64,
                              double *of64) {
    by_counter<<<(unsigned)((n + 255) / 256), 256>>>(key, ctr0, n, o32, o64, of64);
    return (int)cudaDeviceSynchronize();
}

extern "C" int run_by_stream(uint64_t key, uint64_t ctr0, uint64_t per, uint64_t step,
                             uint64_t nthreads, uint32_t *o32, uint64_t *o64) {
    by_stream<<<(unsigned)((nthreads + 127) / 128), 128>>>(key, ctr0, per, step, nthreads, o32, o64);
    return (int)cudaDeviceSynchronize();
}
'''


@pytest.fixture(scope="module")
def consumer(tmp_path_factory):
    d = tmp_path_factory.mktemp("consumer")
    src = d / "consumer.cu"
    src.write_text(CONSUMER)
    so = d / "libconsumer.so"
    subprocess.run([libbuild.nvcc(), *libbuild.ARCH, "-O3", "-std=c++17", "-shared", "-Xcompiler",
                    "-fPIC", "-I", libbuild.INCLUDE, str(src), "-o", str(so)], check=True)
    lib = ctypes.CDLL(str(so))
    u64, p = ctypes.c_uint64, ctypes.c_void_p
    lib.run_by_counter.argtypes = [u64, u64, u64, p, p, p]
    lib.run_by_stream.argtypes = [u64, u64, u64, u64, u64, p, p]
    return lib


def test_by_counter(gpu_lib, consumer):
    import torch

    key = int(gpu_lib.make_keys(31, 1)[0])
    base, n = (1 << 64) - 5000, 100_003
    o32 = torch.empty(n, dtype=torch.int32, device="cuda")
    o64 = torch.empty(n, dtype=torch.int64, device="cuda")
    of = torch.empty(n, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    assert consumer.run_by_counter(key, base, n, o32.data_ptr(), o64.data_ptr(), of.data_ptr()) == 0
    assert np.array_equal(o32.cpu().numpy().view(np.uint32), oracle.fill32(key, base, n))
    assert np.array_equal(o64.cpu().numpy().view(np.uint64), oracle.fill64(key, base, n))
    assert np.array_equal(of.cpu().numpy(), oracle.uniform_f64(key, base, n))


@pytest.mark.parametrize("step", [1, 3])
def test_weyl_stream(gpu_lib, consumer, step):
    import torch

    key = int(gpu_lib.make_keys(32, 1)[0])
    base, per, nth = 77, 1000, 333
    n = per * nth
    o32 = torch.empty(n, dtype=torch.int32, device="cuda")
    o64 = torch.empty(n, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    assert consumer.run_by_stream(key, base, per, step, nth, o32.data_ptr(), o64.data_ptr()) == 0
    assert np.array_equal(o32.cpu().numpy().view(np.uint32), oracle.fill32_strided(key, base, step, n))
    assert np.array_equal(o64.cpu().numpy().view(np.uint64), oracle.fill64_strided(key, base, step, n))
