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

__global__ void bm_pairs(const uint32_t *hi, const uint32_t *lo, uint64_t n, float2 *out) {
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = sq::box_muller(hi[i], lo[i]);
}

__global__ void u53(const uint64_t *v, uint64_t n, uint64_t *out) {
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = sq::uniform53_bits(v[i]);
}

extern "C" int run_u53(const uint64_t *v, uint64_t n, uint64_t *out) {
    u53<<<(unsigned)((n + 255) / 256), 256>>>(v, n, out);
    return (int)cudaDeviceSynchronize();
}

extern "C" int run_bm_pairs(const uint32_t *hi, const uint32_t *lo, uint64_t n, float2 *out) {
    bm_pairs<<<(unsigned)((n + 255) / 256), 256>>>(hi, lo, n, out);
    return (int)cudaDeviceSynchronize();
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
    lib.run_bm_pairs.argtypes = [p, p, u64, p]
    lib.run_u53.argtypes = [p, u64, p]
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


def _edge_halves(rng):
    """hi: both ends of the range, every power of two and every switch of
    the exponent split (2^E sqrt2), each +-64, plus random values; lo:
    every quadrant boundary (multiples of 2^29) +-64, plus random values."""
    M = 1 << 32
    his = [np.arange(0, 1 << 16), np.arange(M - (1 << 16), M)]
    for e in range(33):
        for c in (1 << e, int(round((1 << e) * np.sqrt(2)))):
            his.append(np.arange(c - 65, c + 64))  # k = hi + 1 in [c - 64, c + 64]
    his.append(rng.integers(0, M, 1 << 20))
    hi_edge = np.concatenate(his)
    hi_edge = hi_edge[(hi_edge >= 0) & (hi_edge < M)].astype(np.uint64).astype(np.uint32)
    lo_edge = np.concatenate([(np.arange(-64, 65) + (j << 29)) % M for j in range(8)]
                             + [rng.integers(0, M, 1 << 18)]).astype(np.uint64).astype(np.uint32)
    hi = np.concatenate([hi_edge, rng.integers(0, M, lo_edge.size).astype(np.uint32)])
    lo = np.concatenate([rng.integers(0, M, hi_edge.size).astype(np.uint32), lo_edge])
    return hi, lo


def test_box_muller_edges(gpu_lib, consumer):
    """sq::box_muller on the edges of its exponent split and quadrant
    reduction, against the oracle's double-precision pair: within 2e-6
    absolute where |z| < 5 and 1e-5 relative beyond."""
    import torch

    hi, lo = _edge_halves(np.random.default_rng(61))
    n = hi.size
    d_hi = torch.from_numpy(hi.view(np.int32)).cuda()
    d_lo = torch.from_numpy(lo.view(np.int32)).cuda()
    out = torch.empty((n, 2), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    assert consumer.run_bm_pairs(d_hi.data_ptr(), d_lo.data_ptr(), n, out.data_ptr()) == 0
    got = out.cpu().numpy().astype(np.float64)
    want = oracle.box_muller_f64(hi, lo)
    err = np.abs(got - want)
    small = np.abs(want) < 5
    assert err[small].max() <= 2e-6, err[small].max()
    if (~small).any():
        assert (err[~small] / np.abs(want[~small])).max() <= 1e-5
    assert np.all(np.isfinite(got))


def test_uniform53_edges(gpu_lib, consumer):
    """sq::uniform53_bits at every leading-one position of k = v >> 11
    (2^j - 1, 2^j, 2^j + 1 and a random value with that leading one),
    around the switch at k = 2^32, at 0 and all-ones, against the oracle."""
    import torch

    rng = np.random.default_rng(81)
    ks = [0, 1, 2, 3]
    for j in range(1, 53):
        ks += [(1 << j) - 1, 1 << j, (1 << j) + 1, (1 << j) | int(rng.integers(0, 1 << j))]
    ks = np.array([k for k in ks if k < (1 << 53)], dtype=np.uint64)
    low = rng.integers(0, 1 << 11, ks.size, dtype=np.uint64)  # bits dropped by >> 11
    v = np.concatenate([(ks << np.uint64(11)) | low, np.array([(1 << 64) - 1], dtype=np.uint64),
                        rng.integers(0, 1 << 64, 100_000, dtype=np.uint64)])
    d_v = torch.from_numpy(v.view(np.int64)).cuda()
    out = torch.empty(v.size, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    assert consumer.run_u53(d_v.data_ptr(), v.size, out.data_ptr()) == 0
    got = out.cpu().numpy().view(np.uint64)
    assert np.array_equal(got, oracle.uniform53_of(v).view(np.uint64))
