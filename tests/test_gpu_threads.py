"""Host threads calling the C ABI at once, each on its own CUDA stream with
its own key and counter base: every output matches the oracle, so launches
from different threads neither share state nor overwrite each other."""
import threading

import numpy as np
import pytest

import oracle
from paper_2004_06278_gb300 import _lib as C

pytestmark = pytest.mark.gpu


def test_concurrent_threads_own_streams(gpu_lib):
    import torch

    nthreads, n = 8, (1 << 22) + 13
    keys = gpu_lib.make_keys(91, nthreads)
    outs32 = [torch.empty(n, dtype=torch.int32, device="cuda") for _ in range(nthreads)]
    outs64 = [torch.empty(n, dtype=torch.int64, device="cuda") for _ in range(nthreads)]
    streams = [torch.cuda.Stream() for _ in range(nthreads)]
    errors = []
    go = threading.Barrier(nthreads)

    def work(i):
        try:
            go.wait()
            h = int(streams[i].cuda_stream)
            for rep in range(3):
                C.sq_u32(int(keys[i]), 1000 * i + rep, n, outs32[i].data_ptr(), h)
                C.sq_u64(int(keys[i]), 1000 * i + rep, n, outs64[i].data_ptr(), h)
            streams[i].synchronize()
        except Exception as e:  # reported after join
            errors.append((i, e))

    ts = [threading.Thread(target=work, args=(i,)) for i in range(nthreads)]
    for t in ts:
        t.start()
    for t in ts:
        t.join(120)
    assert not errors, errors
    torch.cuda.synchronize()
    for i in range(nthreads):
        base = 1000 * i + 2  # the last repetition
        assert np.array_equal(outs32[i].cpu().numpy().view(np.uint32), oracle.fill32(int(keys[i]), base, n)), i
        assert np.array_equal(outs64[i].cpu().numpy().view(np.uint64), oracle.fill64(int(keys[i]), base, n)), i
