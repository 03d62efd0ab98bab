"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle
checks. This module holds none of the generator's arithmetic: it returns
seeds, counter bases, stream lengths and offsets. Keys are not made here;
each side derives them from a seed with its own key construction.

Workloads (sizes of the benchmark configurations):
  single      one key (seed 1), counters 0 .. 2^24-1 -> uint32[2^24]
  throughput  one key (seed 2), counter base uniform in [0, 2^64) (numpy
              default_rng(3)), squares64 -> uint64[2^30] and squares32 ->
              uint32[2^32]
  batched     4096 keys (seed 7); lengths floor(exp(U)), U ~ Uniform[ln 1e3,
              ln 1e7) (default_rng(7)); bases uniform 64-bit; streams
              s = 0 mod 64 start at 2^64 - d, d uniform in [1, min(1e6,
              len-1)], so they wrap; offsets are the exclusive prefix sum
  transforms  one key (seed 11), base 0, 2^30 outputs each
  fused       2^20 keys (seed 13), base 0, 2^18 counters per stream
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

M64 = (1 << 64) - 1


@dataclass
class Batch:
    key_seed: int
    bases: np.ndarray    # uint64[S]
    lengths: np.ndarray  # int64[S]
    offsets: np.ndarray  # int64[S]

    @property
    def nstreams(self) -> int:
        return int(self.lengths.size)

    @property
    def total(self) -> int:
        return int(self.offsets[-1] + self.lengths[-1]) if self.lengths.size else 0


def throughput_base(seed: int = 3) -> int:
    """Counter base drawn uniformly from [0, 2^64)."""
    return int(np.random.default_rng(seed).integers(0, 1 << 64, dtype=np.uint64))


def ragged_batch(nstreams: int = 4096, seed: int = 7, lo: float = 1e3, hi: float = 1e7,
                 wrap_every: int = 64, wrap_window: int = 1_000_000, gap_max: int = 0) -> Batch:
    """Log-uniform ragged stream lengths with wrapping counter bases.

    gap_max > 0 leaves a random gap of 0..gap_max positions before each
    stream (positions no stream covers)."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(np.log(lo), np.log(hi), nstreams)
    lengths = np.floor(np.exp(u)).astype(np.int64)
    bases = rng.integers(0, 1 << 64, nstreams, dtype=np.uint64)
    for s in range(0, nstreams, wrap_every):
        top = int(min(wrap_window, max(1, lengths[s] - 1)))
        d = int(rng.integers(1, top + 1))
        bases[s] = np.uint64((1 << 64) - d)
    gaps = rng.integers(0, gap_max + 1, nstreams).astype(np.int64) if gap_max else np.zeros(
        nstreams, dtype=np.int64)
    ends = np.cumsum(lengths + gaps)
    offsets = (ends - lengths).astype(np.int64)
    return Batch(key_seed=seed, bases=bases, lengths=lengths, offsets=offsets)


def small_ragged_batch(nstreams: int, seed: int, max_len: int, gap_max: int = 3,
                       wrap_every: int = 4) -> Batch:
    """A batch small enough for the oracle: lengths uniform in [0, max_len],
    including empty streams, with gaps and wrapping bases."""
    rng = np.random.default_rng(seed)
    lengths = rng.integers(0, max_len + 1, nstreams).astype(np.int64)
    lengths[rng.integers(0, nstreams)] = 0
    bases = rng.integers(0, 1 << 64, nstreams, dtype=np.uint64)
    for s in range(0, nstreams, wrap_every):
        d = int(rng.integers(1, max(2, int(lengths[s]) + 1)))
        bases[s] = np.uint64((1 << 64) - d)
    gaps = rng.integers(0, gap_max + 1, nstreams).astype(np.int64)
    ends = np.cumsum(lengths + gaps)
    offsets = (ends - lengths).astype(np.int64)
    return Batch(key_seed=seed, bases=bases, lengths=lengths, offsets=offsets)


def key_counter_batch(nstreams: int, seed: int) -> Batch:
    """Section 4's key-counter mode: every stream has length 1 at counter 0."""
    return Batch(key_seed=seed, bases=np.zeros(nstreams, dtype=np.uint64),
                 lengths=np.ones(nstreams, dtype=np.int64),
                 offsets=np.arange(nstreams, dtype=np.int64))


def sample_positions(n: int, count: int, seed: int) -> np.ndarray:
    """Sorted unique sample indices in [0, n), always including both ends."""
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, n, count, dtype=np.int64)
    idx = np.concatenate([idx, [0, n - 1], np.arange(min(n, 64)), np.arange(max(0, n - 64), n)])
    return np.unique(idx)
