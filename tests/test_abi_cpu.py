"""The C-ABI library without a GPU: it loads, exports every symbol that
include/squares.h declares, makes the same keys as the oracle, and rejects
bad arguments on the host before touching CUDA. No kernel is launched."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
import paper_2004_06278_gb300 as sq
from paper_2004_06278_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "squares.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2004_06278_gb300 import build

    build.build()
    return sq.load()


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sq_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    declared = header_functions()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(_lib.declared_symbols()) == declared


def test_abi_version(lib):
    assert sq.sq_abi_version() == 100


def test_make_keys_matches_oracle(lib):
    for seed, n in [(1, 1), (7, 4096), (13, 1 << 16), (0, 5), ((1 << 64) - 1, 100)]:
        assert np.array_equal(sq.make_keys(seed, n), oracle.make_keys(seed, n)), (seed, n)


def test_make_keys_errors(lib):
    sq.sq_make_keys(1, 0, 0)  # n = 0 is fine, even with NULL
    with pytest.raises(sq.SquaresError) as e:
        sq.sq_make_keys(1, 5, 0)
    assert e.value.status == sq.SQ_EINVAL
    with pytest.raises(sq.SquaresError) as e:
        sq.sq_make_keys(1, (1 << 31) + 1, 0)
    assert e.value.status == sq.SQ_ERANGE


@pytest.mark.parametrize("fn,elem", [(sq.sq_u32, 4), (sq.sq_u64, 8), (sq.sq_uniform_f32, 4),
                                     (sq.sq_uniform_bf16, 2), (sq.sq_normal_f32, 4),
                                     (sq.sq_uniform2_f32, 4), (sq.sq_uniform_f64, 8)])
def test_plain_argument_checks(lib, fn, elem):
    fn(1, 0, 0, 0)  # n = 0: no launch, OK
    with pytest.raises(sq.SquaresError) as e:
        fn(1, 0, 10, 0)
    assert e.value.status == sq.SQ_EINVAL and "NULL" in e.value.message
    if elem > 1:
        with pytest.raises(sq.SquaresError) as e:
            fn(1, 0, 10, 0x1000 + 1)
        assert e.value.status == sq.SQ_EINVAL and "aligned" in e.value.message
    with pytest.raises(sq.SquaresError) as e:
        fn(1, 0, (1 << 62) + 1, 0x1000)
    assert e.value.status == sq.SQ_ERANGE


def test_strided_and_keys_argument_checks(lib):
    for fn, elem in ((sq.sq_u32_strided, 4), (sq.sq_u64_strided, 8)):
        fn(1, 0, 3, 0, 0)
        with pytest.raises(sq.SquaresError) as e:
            fn(1, 0, 3, 10, 0)
        assert e.value.status == sq.SQ_EINVAL
        with pytest.raises(sq.SquaresError) as e:
            fn(1, 0, 3, 10, 0x1000 + elem // 2)
        assert e.value.status == sq.SQ_EINVAL
    for fn in (sq.sq_keys_u32, sq.sq_keys_u64):
        fn(0, 0, 5, 0)
        with pytest.raises(sq.SquaresError) as e:
            fn(0, 4, 5, 0x1000)
        assert e.value.status == sq.SQ_EINVAL
        with pytest.raises(sq.SquaresError) as e:
            fn(0x1004, 4, 5, 0x1000)
        assert e.value.status == sq.SQ_EINVAL


def test_fill_argument_checks(lib):
    """The store-ceiling kernel's entry point checks its arguments on the
    host like the generators: n = 0 is a no-op, NULL or misaligned output
    and invalid launch configurations are refused before any CUDA call."""
    sq.sq_fill_u32(7, 0, 0)
    with pytest.raises(sq.SquaresError) as e:
        sq.sq_fill_u32(7, 10, 0)
    assert e.value.status == sq.SQ_EINVAL
    with pytest.raises(sq.SquaresError) as e:
        sq.sq_fill_u32(7, 10, 0x1002)
    assert e.value.status == sq.SQ_EINVAL
    with pytest.raises(sq.SquaresError) as e:
        sq.sq_fill_u32(7, 10, 0x1000, (0, 100, 0))
    assert e.value.status == sq.SQ_EINVAL and "configuration" in e.value.message
    with pytest.raises(sq.SquaresError) as e:
        sq.sq_fill_u32(7, (1 << 62) + 1, 0x1000)
    assert e.value.status == sq.SQ_ERANGE
    sq.sq_debug_fail_next("sq_fill_u32")
    with pytest.raises(sq.SquaresError) as e:
        sq.sq_fill_u32(7, 16, 0x1000, (1, 256, 0), 50)
    assert e.value.status == sq.SQ_ECUDA and "injected" in e.value.message


def test_batch_and_fused_argument_checks(lib):
    sq.sq_batch(0, 0, 0, 0, 0, 0)  # empty batch
    with pytest.raises(sq.SquaresError) as e:
        sq.sq_batch(0, 0x1000, 0x1000, 0x1000, 3, 0x1000)
    assert e.value.status == sq.SQ_EINVAL
    with pytest.raises(sq.SquaresError) as e:
        sq.sq_batch(0x1000, 0x1000, 0x1004, 0x1000, 3, 0x1000)
    assert e.value.status == sq.SQ_EINVAL and "misaligned" in e.value.message
    with pytest.raises(sq.SquaresError) as e:
        sq.sq_batch(0x1000, 0x1000, 0x1000, 0x1000, (1 << 31) + 1, 0x1000)
    assert e.value.status == sq.SQ_ERANGE
    with pytest.raises(sq.SquaresError) as e:
        sq.sq_fused_stats(0x1000, 0x1000, 4, 16, 0x1000, 0x1000, 0)
    assert e.value.status == sq.SQ_EINVAL
    with pytest.raises(sq.SquaresError) as e:
        sq.sq_fused_stats(0x1000, 0x1000, 4, (1 << 40) + 1, 0x1000, 0x1000, 0x1000)
    assert e.value.status == sq.SQ_ERANGE
    with pytest.raises(sq.SquaresError):
        sq.sq_graph_launch(0)
    sq.sq_graph_destroy(0)


def test_config_table(lib):
    assert sq.sq_num_variants(sq.SQ_KERNEL_U32) == 7
    assert sq.sq_variant_name(sq.SQ_KERNEL_U32, 6) == "bulk64"
    assert sq.sq_num_variants(sq.SQ_KERNEL_BATCH) == 13
    assert sq.sq_variant_name(sq.SQ_KERNEL_BATCH, 9) == "flat-warp"
    assert [sq.sq_variant_name(sq.SQ_KERNEL_BATCH, v) for v in (10, 11, 12)] == [
        "flat-seg4", "flat-seg8", "flat-seg16"]
    assert sq.sq_num_variants(sq.SQ_KERNEL_FUSED) == 2
    assert sq.sq_variant_name(sq.SQ_KERNEL_FUSED, 0) == "cta-item"
    assert sq.sq_variant_name(sq.SQ_KERNEL_FUSED, 1) == "warp-item"
    assert sq.sq_variant_name(sq.SQ_KERNEL_BATCH, 4) == "warp-stream"
    assert sq.sq_variant_name(sq.SQ_KERNEL_BATCH, 5) == "lane8-stream"
    assert sq.sq_variant_name(sq.SQ_KERNEL_BATCH, 6) == "lane16-stream"
    assert sq.sq_variant_name(sq.SQ_KERNEL_U32, 0) == "st32"
    assert sq.sq_variant_name(sq.SQ_KERNEL_U32, 99) is None
    cfg = sq.sq_get_config(sq.SQ_KERNEL_U64, 1 << 20)
    assert (cfg.variant, cfg.block) == (0, 256)
    sq.sq_set_config(sq.SQ_KERNEL_U64, 1 << 20, 1, 512, 2)
    got = sq.sq_get_config(sq.SQ_KERNEL_U64, (1 << 20) + 5)  # same size bucket
    assert (got.variant, got.block, got.ctas_per_sm) == (1, 512, 2)
    other = sq.sq_get_config(sq.SQ_KERNEL_U64, 1 << 10)
    assert (other.variant, other.block) == (0, 256)
    sq.sq_set_config(sq.SQ_KERNEL_U64, 0, 0, 256, 0)  # all buckets back
    with pytest.raises(sq.SquaresError):
        sq.sq_set_config(sq.SQ_KERNEL_U64, 0, 9, 256, 0)
    with pytest.raises(sq.SquaresError):
        sq.sq_set_config(sq.SQ_KERNEL_U64, 0, 0, 100, 0)
    with pytest.raises(sq.SquaresError):
        sq.sq_set_config(sq.SQ_KERNEL_U64, 0, 0, 64, 0)  # 64-thread CTAs: batch kernel only
    sq.sq_set_config(sq.SQ_KERNEL_BATCH, 0, 1, 64, 0)
    assert sq.sq_get_config(sq.SQ_KERNEL_BATCH, 0).block == 64
    sq.sq_set_config(sq.SQ_KERNEL_BATCH, 0, 0, 256, 0)
    # the batch table is keyed by stream count: a pick for a batch of 2^20
    # short streams leaves batches of a few thousand long ones alone
    sq.sq_set_config(sq.SQ_KERNEL_BATCH, 1 << 20, 9, 512, 0)
    assert sq.sq_get_config(sq.SQ_KERNEL_BATCH, (1 << 20) + 100).variant == 9
    assert sq.sq_get_config(sq.SQ_KERNEL_BATCH, 4096).variant == 0
    sq.sq_set_config(sq.SQ_KERNEL_BATCH, 0, 0, 256, 0)
    with pytest.raises(sq.SquaresError):
        sq.sq_get_config(42, 0)
    with pytest.raises(sq.SquaresError):
        sq.sq_num_variants(-1)


def test_autotune_file_errors(lib, tmp_path):
    with pytest.raises(sq.SquaresError):
        sq.sq_autotune_load(str(tmp_path / "missing.txt"))
    bad = tmp_path / "bad.txt"
    bad.write_text("not a tune file\n")
    with pytest.raises(sq.SquaresError):
        sq.sq_autotune_load(str(bad))


def _device_name():
    import torch

    return torch.cuda.get_device_name(0) if torch.cuda.is_available() else "unknown"


def test_build_id_is_the_kernel_code_hash(lib):
    """The library reports the hash of the kernel sources' code it was built
    from (the identifier a tuned table is keyed by)."""
    from paper_2004_06278_gb300 import build as libbuild

    bid = sq.sq_build_id()
    assert len(bid) == 16 and int(bid, 16) >= 0
    assert bid == libbuild.build_id()


def test_tuned_table_from_other_kernel_code_is_ignored(lib, tmp_path):
    """A table saved by a library built from other kernel code is not
    applied: the load fails with a message naming both code identifiers and
    the table keeps its entries. A file of format 1 (no code identifier) is
    refused the same way; the same rows under this library's identifier are
    applied."""
    dev = _device_name()
    rows = "0 20 4 512 2\n"
    sq.sq_set_config(sq.SQ_KERNEL_U32, 0, 0, 256, 0)
    try:
        other = tmp_path / "other_code.txt"
        other.write_text(f"squares-autotune 2\ndevice {dev}\ncode 0123456789abcdef\n{rows}")
        with pytest.raises(sq.SquaresError) as e:
            sq.sq_autotune_load(str(other))
        assert e.value.status == sq.SQ_EINVAL
        assert "0123456789abcdef" in e.value.message and sq.sq_build_id() in e.value.message
        assert "0123456789abcdef" in sq.sq_last_error()
        c = sq.sq_get_config(sq.SQ_KERNEL_U32, 1 << 20)
        assert (c.variant, c.block, c.ctas_per_sm) == (0, 256, 0)
        old = tmp_path / "format1.txt"
        old.write_text(f"squares-autotune 1\ndevice {dev}\n{rows}")
        with pytest.raises(sq.SquaresError) as e:
            sq.sq_autotune_load(str(old))
        assert "none" in e.value.message
        assert sq.sq_get_config(sq.SQ_KERNEL_U32, 1 << 20).variant == 0
        good = tmp_path / "this_code.txt"
        good.write_text(f"squares-autotune 2\ndevice {dev}\ncode {sq.sq_build_id()}\n{rows}")
        sq.sq_autotune_load(str(good))
        c = sq.sq_get_config(sq.SQ_KERNEL_U32, 1 << 20)
        assert (c.variant, c.block, c.ctas_per_sm) == (4, 512, 2)
    finally:
        sq.sq_set_config(sq.SQ_KERNEL_U32, 0, 0, 256, 0)


def test_autotune_save_round_trip(lib, tmp_path):
    """sq_autotune_save writes format 2 with the device name and the build
    identifier; loading it back restores every entry."""
    sq.sq_set_config(sq.SQ_KERNEL_U64, 1 << 24, 5, 512, 1)
    sq.sq_set_config(sq.SQ_KERNEL_BATCH, 1 << 20, 9, 512, 0)
    try:
        path = tmp_path / "saved.txt"
        sq.sq_autotune_save(str(path))
        lines = path.read_text().splitlines()
        assert lines[0] == "squares-autotune 2"
        assert lines[1] == f"device {_device_name()}"
        assert lines[2] == f"code {sq.sq_build_id()}"
        sq.sq_set_config(sq.SQ_KERNEL_U64, 0, 0, 256, 0)
        sq.sq_set_config(sq.SQ_KERNEL_BATCH, 0, 0, 256, 0)
        sq.sq_autotune_load(str(path))
        c = sq.sq_get_config(sq.SQ_KERNEL_U64, 1 << 24)
        assert (c.variant, c.block, c.ctas_per_sm) == (5, 512, 1)
        b = sq.sq_get_config(sq.SQ_KERNEL_BATCH, (1 << 20) + 7)
        assert (b.variant, b.block) == (9, 512)
        assert sq.sq_get_config(sq.SQ_KERNEL_BATCH, 4096).variant == 0
    finally:
        sq.sq_set_config(sq.SQ_KERNEL_U64, 0, 0, 256, 0)
        sq.sq_set_config(sq.SQ_KERNEL_BATCH, 0, 0, 256, 0)


def test_last_error_is_per_call(lib):
    with pytest.raises(sq.SquaresError):
        sq.sq_u32(1, 0, 10, 0)
    assert "NULL" in sq.sq_last_error()
    sq.sq_u32(1, 0, 0, 0)
    assert sq.sq_last_error() == ""


def test_injected_launch_failure_reaches_the_caller(lib):
    """A failed launch surfaces as SQ_ECUDA with a message, through the C ABI
    and the binding; made on the host (no GPU is touched: the armed entry
    point fails after its argument checks and before any CUDA call)."""
    calls = [("sq_u32", lambda: sq.sq_u32(1, 0, 16, 0x1000)),
             ("sq_u64_strided", lambda: sq.sq_u64_strided(1, 0, 3, 16, 0x1000)),
             ("sq_keys_u32", lambda: sq.sq_keys_u32(0x1000, 4, 0, 0x2000)),
             ("sq_batch", lambda: sq.sq_batch(0x1000, 0x1000, 0x1000, 0x1000, 3, 0x1000)),
             ("sq_fused_stats", lambda: sq.sq_fused_stats(0x1000, 0x1000, 4, 16, 0x1000, 0x1000, 0x1000)),
             ("sq_graph_launch", lambda: sq.sq_graph_launch(0x1000))]
    for name, call in calls:
        sq.sq_debug_fail_next(name)
        with pytest.raises(sq.SquaresError) as e:
            call()
        assert e.value.status == sq.SQ_ECUDA and "injected" in e.value.message, name
    # one-shot: the next bad-argument call reports its own error again
    sq.sq_debug_fail_next("sq_u32")
    sq.sq_debug_fail_next(None)
    with pytest.raises(sq.SquaresError) as e:
        sq.sq_u32(1, 0, 10, 0)
    assert e.value.status == sq.SQ_EINVAL


def test_tune_file_from_environment(lib, tmp_path):
    """SQ_TUNE_FILE: the table is loaded from that file on first use (checked
    in a fresh process; a table for another device name, or saved by a
    library built from other kernel code, is ignored)."""
    import subprocess
    import sys

    import torch

    name = torch.cuda.get_device_name(0) if torch.cuda.is_available() else "unknown"
    bid = sq.sq_build_id()
    good = tmp_path / "tune.txt"
    good.write_text(f"squares-autotune 2\ndevice {name}\ncode {bid}\n0 20 4 512 2\n")
    other = tmp_path / "other.txt"
    other.write_text(f"squares-autotune 2\ndevice some other GPU\ncode {bid}\n0 20 4 512 2\n")
    stale = tmp_path / "stale.txt"
    stale.write_text(f"squares-autotune 2\ndevice {name}\ncode ffffffffffffffff\n0 20 4 512 2\n")
    code = ("import paper_2004_06278_gb300 as sq; c = sq.sq_get_config(0, 1 << 20); "
            "print(c.variant, c.block, c.ctas_per_sm)")
    for path, want in ((good, "4 512 2"), (other, "0 256 0"), (stale, "0 256 0")):
        env = dict(os.environ, SQ_TUNE_FILE=str(path))
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT,
                           env=env, timeout=120)
        assert r.returncode == 0, r.stderr
        assert r.stdout.strip() == want, (path, r.stdout)


def test_last_error_is_per_thread(lib):
    """Each host thread sees its own last error: a failing call in one
    thread leaves another thread's message untouched."""
    import threading

    seen = {}
    started = threading.Barrier(2)
    failed = threading.Event()

    def failing():
        started.wait()
        with pytest.raises(sq.SquaresError):
            sq.sq_u64(1, 0, 10, 0)
        seen["failing"] = sq.sq_last_error()
        failed.set()

    def clean():
        started.wait()
        sq.sq_u32(1, 0, 0, 0)  # n = 0: succeeds, clears this thread's message
        failed.wait(10)
        seen["clean"] = sq.sq_last_error()

    ts = [threading.Thread(target=failing), threading.Thread(target=clean)]
    for t in ts:
        t.start()
    for t in ts:
        t.join(30)
    assert "NULL" in seen["failing"]
    assert seen["clean"] == ""


def test_device_header_compiles_in_a_consumer(tmp_path):
    """The public device header builds, for sm_103a, inside a kernel outside
    the library: the consumer the GPU test runs (squares32 / squares64 by
    counter and through WeylStream, Box-Muller pairs, 53-bit doubles),
    compiled here with nvcc without launching anything."""
    from paper_2004_06278_gb300 import build as libbuild
    from tests.test_gpu_device_header import CONSUMER

    try:
        nvcc = libbuild.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    src = tmp_path / "consumer.cu"
    src.write_text(CONSUMER)
    r = subprocess.run([nvcc, *libbuild.ARCH, "-O3", "-std=c++17", "-I", libbuild.INCLUDE, "-c",
                        str(src), "-o", str(tmp_path / "consumer.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
