"""Models of the index arithmetic of the ragged-batch kernels in
paper_2004_06278_gb300/csrc/kernels_batch.cu, run on the CPU.

Each model follows one kernel's walk step by step in Python integers: the
tile kernel (variants 0-3: per-CTA runs of tiles, the galloping stream
search, boundary chunks, the extent clamp), the streams-to-lanes kernel
(variants 4-8) and the flattened-warp kernel (variant 9: the warp scan of
the lengths, the table of non-empty streams, the per-step window masks and
owner lookup, in 32-bit and 64-bit positions). They record which (stream,
index) each output position receives; the values themselves are the GPU
parity tests' business. The models use small blocks and grids so that
every path (heads, whole-tile runs, boundary tiles, empty streams, gaps,
wrapping counters, partial last steps) is met on batches of a few thousand
elements.

On batches that meet sq_batch's requirements every element of every stream
must be written exactly once, at offsets[s] + i; on metadata that breaks
them (unsorted or overlapping streams, negative offsets, an early stream
far past the last one's end) every write must stay inside the extent
[0, offsets[S-1] + lengths[S-1]) and no position may be written twice by
the tile kernel. The models are kept in step with the CUDA code by hand; the segment
walk (variants 10-12) has a model of its own below.
"""
import numpy as np
import pytest

from paper_2004_06278_gb300 import workloads

M32 = (1 << 32) - 1
M64 = (1 << 64) - 1


def _s64(x: int) -> int:
    x &= M64
    return x - (1 << 64) if x >> 63 else x


def _popc(x: int) -> int:
    return bin(x & M32).count("1")


# --- tile kernel (variants 0-3) -------------------------------------------

def _find_stream(off, S, frm, e):
    lo, step = frm, 1
    while step <= S - 1 - lo and off[lo + step] <= e:
        lo += step
        step <<= 1
    hi = lo + step if step <= S - lo else S
    while hi - lo > 1:
        mid = lo + (hi - lo) // 2
        if off[mid] <= e:
            lo = mid
        else:
            hi = mid
    return lo


def _stream_at(off, S, frm, e):
    if frm is None:
        if off[0] > e:
            return None
        frm = 0
    return _find_stream(off, S, frm, e)


def tile_writes(off, ln, head, block, EPV, grid, nelem):
    """Positions written by batch_kernel<CS, EPV> with `block` threads per CTA
    and `grid` CTAs, for an output whose first 32-byte boundary is `head`
    elements in: {position: (stream, index)}."""
    S = len(off)
    writes = {}

    def w(e, s, i):
        assert 0 <= e < nelem, ("outside the buffer", e)
        assert e not in writes, ("written twice", e)
        writes[e] = (s, i)

    tile = block * EPV
    shift = tile.bit_length() - 1
    start, end = off[0], off[S - 1] + ln[S - 1]
    for e in range(0, min(head, end)):  # the unaligned head, CTA 0
        s = _stream_at(off, S, None, e)
        if s is not None and e < off[s] + ln[s]:
            w(e, s, e - off[s])
    if end <= head:
        return writes
    first = max(start, head)
    t_begin = (first - head) >> shift
    t_end = (end - head + tile - 1) >> shift
    per = (t_end - t_begin + grid - 1) // grid
    for c in range(grid):
        t = t_begin + c * per
        t_stop = min(t + per, t_end)
        if t >= t_stop:
            continue
        s = _stream_at(off, S, None, head + (t << shift))
        while t < t_stop:
            lo = head + (t << shift)
            if s is None or (s + 1 < S and off[s + 1] <= lo):
                s = _stream_at(off, S, s, lo)
            k = 0
            seg_lo = 0
            if s is not None:
                seg_lo = off[s]
                seg_hi = min(seg_lo + ln[s], end)
                if lo + tile <= seg_hi:
                    k = min((seg_hi - lo) >> shift, t_stop - t)
            if k > 0:  # whole tiles inside stream s
                for i in range(k):
                    for tid in range(block):
                        e = lo + i * tile + tid * EPV
                        for j in range(EPV):
                            w(e + j, s, e + j - seg_lo)
                t += k
                continue
            for tid in range(block):  # a boundary tile: each chunk on its own
                e0 = lo + tid * EPV
                if e0 >= end:
                    continue
                ss = _stream_at(off, S, s, e0)
                if ss is None:
                    ss = 0
                slo = off[ss]
                shi = slo + ln[ss]
                if slo <= e0 and e0 + EPV <= shi and e0 + EPV <= end:
                    for j in range(EPV):
                        w(e0 + j, ss, e0 + j - slo)
                    continue
                for j in range(EPV):
                    e = e0 + j
                    if e >= end:
                        break
                    if e >= shi and ss + 1 < S:
                        ss = _find_stream(off, S, ss, e)
                        slo = off[ss]
                        shi = slo + ln[ss]
                    if e < slo or e >= shi:
                        continue
                    w(e, ss, e - slo)
            t += 1
    return writes


# --- streams to lanes (variants 4-8) ---------------------------------------

def stream_writes(off, ln, LPS, groups):
    """Positions written by batch_stream_kernel<LPS> with `groups` lane
    groups: {position: [(stream, index), ...]} (overlapping streams may
    write a position more than once; the last writer is not modelled)."""
    S = len(off)
    end = off[S - 1] + ln[S - 1]
    writes = {}
    for g in range(groups):
        for s in range(g, S, groups):
            length = min(ln[s], end - off[s])
            if off[s] < 0:
                continue
            for j in range(LPS):
                for i in range(j, length, LPS):
                    writes.setdefault(off[s] + i, []).append((s, i))
    return writes


# --- flattened warps (variant 9) -------------------------------------------

def flat_writes(keys, bases, off, ln, force64=False, end_override=None):
    """Positions written by batch_flat_kernel, with the Weyl term y the
    kernel forms for each: [(position, stream, index, y)]. force64 takes the
    64-bit position walk whatever the group's total (the kernel takes it
    from 2^31 values on)."""
    S = len(off)
    end = _s64(off[S - 1] + ln[S - 1]) if end_override is None else end_override
    out = []
    for g in range(0, S, 32):
        L, O, K, B = [0] * 32, [0] * 32, [0] * 32, [0] * 32
        for lane in range(32):
            s = g + lane
            if s < S:
                L[lane], O[lane], K[lane], B[lane] = ln[s], off[s], keys[s], bases[s]
            n, o = L[lane], O[lane]
            if o < 0:
                n = 0
            elif n > _s64(end - o):
                n = _s64(end - o)
            n = min(max(n, 0), 1 << 57)
            L[lane] = n
        inc, acc = [], 0
        for lane in range(32):
            acc = _s64(acc + L[lane])
            inc.append(acc)
        P = [_s64(inc[i] - L[i]) for i in range(32)]
        T = inc[31]
        nonempty = sum(1 << i for i in range(32) if L[i] > 0)
        table = [None] * 32
        for i in range(32):
            if L[i] > 0:
                table[_popc(nonempty & ((1 << i) - 1))] = (
                    ((B[i] - P[i]) * K[i]) & M64, _s64(O[i] - P[i]), K[i], g + i, P[i])
        if T < (1 << 31) and not force64:
            MW, sentinel = M32, 0xC0000000
        else:
            MW, sentinel = M64, 0xC000000000000000
        Pe = [(P[i] & MW) if L[i] > 0 else sentinel for i in range(32)]
        before = M32  # streams started before the step, minus 1
        b = 0
        while b < T:
            starts = 0
            for i in range(32):
                r = (Pe[i] - b) & MW
                if r < 32:
                    starts |= 1 << r
            for t in range(32):
                p = b + t
                k = (before + _popc(starts & (M32 >> (31 - t)))) & M32
                if p < T:
                    assert 0 <= k < 32 and table[k] is not None, ("no owner", p)
                    y0, dst, key, s, ps = table[k]
                    out.append((_s64(dst + p), s, p - ps, (y0 + p * key) & M64))
            before = (before + _popc(starts)) & M32
            b += 32
    return out


# --- flattened warps over aligned segments (variants 10-12) ---------------

SEG_LEN_CAP = 1 << 26


def _clamped_group(keys, bases, off, ln, g, end):
    S = len(off)
    L, O, K, B = [0] * 32, [0] * 32, [0] * 32, [0] * 32
    for lane in range(32):
        s = g + lane
        if s < S:
            L[lane], O[lane], K[lane], B[lane] = ln[s], off[s], keys[s], bases[s]
        n, o = L[lane], O[lane]
        if o < 0:
            n = 0
        elif n > _s64(end - o):
            n = _s64(end - o)
        L[lane] = min(max(n, 0), 1 << 57)
    return L, O, K, B


def seg_writes(keys, bases, off, ln, C, out_elem=0, cap=SEG_LEN_CAP):
    """Positions written by batch_seg_kernel<C>, with the Weyl term y formed
    for each: [(position, stream, index, y)]. out_elem is the output
    pointer's address in elements (its value modulo C places the block
    cuts). A group with a clamped length of `cap` or more takes the
    per-position walk (flat_writes on the group alone); the kernel's cap is
    2^26, smaller ones exercise the switch on small batches. Follows the two
    passes: whole segments (scan, compacted table, window-bit owner, strides
    of one segment) and each lane's pieces."""
    S = len(off)
    end = _s64(off[S - 1] + ln[S - 1])
    a = out_elem % C
    out = []
    for g in range(0, S, 32):
        L, O, K, B = _clamped_group(keys, bases, off, ln, g, end)
        if any(x >= cap for x in L):
            sub = range(g, min(g + 32, S))
            for e, s, i, y in flat_writes([keys[x] for x in sub], [bases[x] for x in sub],
                                          [off[x] for x in sub], [ln[x] for x in sub],
                                          end_override=end):
                out.append((e, g + s, i, y))
            continue
        lo = [((O[i] & M64) + a) % C for i in range(32)]
        hi = [lo[i] + L[i] for i in range(32)]
        assert all(h < (1 << 32) for h in hi)
        # whole segments
        ws = [1 if lo[i] else 0 for i in range(32)]
        we = [hi[i] // C for i in range(32)]
        nw = [we[i] - ws[i] if L[i] > 0 and we[i] > ws[i] else 0 for i in range(32)]
        Q, acc = [], 0
        for i in range(32):
            Q.append(acc)
            acc += nw[i]
        R = acc
        assert R < (1 << 30)
        with_ = [i for i in range(32) if nw[i] > 0]
        tab = []
        for i in with_:
            first = ws[i] * C - lo[i]
            y = ((B[i] + first) * K[i]) & M64
            tab.append((y, K[i], O[i] + first, Q[i], g + i, first))
        Pe = [Q[i] if nw[i] > 0 else 0xC0000000 for i in range(32)]
        before = M32
        for b in range(0, R, 32):
            starts = 0
            for i in range(32):
                r = (Pe[i] - b) & M32
                if r < 32:
                    starts |= 1 << r
            for t in range(32):
                k = (before + _popc(starts & (M32 >> (31 - t)))) & M32
                r = b + t
                if r >= R:
                    continue
                assert k < len(tab), ("no owner", r)
                y0, key, dst, Qk, s, first = tab[k]
                j = r - Qk
                assert 0 <= j, ("owner after the segment", r)
                p0 = dst + j * C
                assert (out_elem + p0) % C == 0, "misaligned vector store"
                for i in range(C):
                    idx = first + j * C + i
                    assert idx < L[s - g], ("whole segment past the stream", r)
                    out.append((p0 + i, s, idx, (y0 + (j * C + i) * key) & M64))
            before = (before + _popc(starts)) & M32
        # pieces, one lane per stream
        for i in range(32):
            if L[i] <= 0:
                continue
            nseg = (hi[i] + C - 1) // C
            head = lo[i] != 0 or hi[i] < C
            tail = hi[i] % C != 0 and nseg > 1
            for piece, act in ((0, head), (1, tail)):
                if not act:
                    continue
                b0 = 0 if piece == 0 else (nseg - 1) * C
                p_lo = lo[i] if piece == 0 else b0
                p_hi = min(hi[i], b0 + C)
                y = ((B[i] - lo[i] + b0) * K[i]) & M64
                for c in range(C):
                    if p_lo <= b0 + c < p_hi:
                        idx = b0 + c - lo[i]
                        out.append((O[i] + idx, g + i, idx, (y + c * K[i]) & M64))
    return out


# --- batches ---------------------------------------------------------------

def _valid_batch(rng, trial):
    S = int(rng.integers(1, 70))
    max_len = int(rng.choice([1, 3, 11, 50, 300]))
    b = workloads.small_ragged_batch(S, seed=1000 + trial, max_len=max_len,
                                     gap_max=int(rng.choice([0, 3, 40])))
    lead = int(rng.choice([0, 0, 37]))
    off = [int(x) + lead for x in b.offsets]
    ln = [int(x) for x in b.lengths]
    keys = [int(k) | 1 for k in rng.integers(0, 1 << 63, S, dtype=np.uint64)]
    bases = [int(x) for x in b.bases]
    return off, ln, keys, bases


def _invalid_batch(rng, kind):
    """Metadata that breaks sq_batch's requirements in one of four ways."""
    S = int(rng.integers(1, 40))
    ln = [int(x) for x in rng.integers(0, 300, S)]
    if kind == 0:  # unsorted offsets
        off = [int(x) for x in rng.integers(0, 2000, S)]
    elif kind == 1:  # sorted, but streams run past the next ones
        off = sorted(int(x) for x in rng.integers(0, 1500, S))
        ln = [int(x) for x in rng.integers(0, 3000, S)]
    elif kind == 2:  # negative offsets sprinkled in
        off = [int(x) for x in rng.integers(-400, 1500, S)]
    else:  # an early stream far past the last one's end
        off = sorted(int(x) for x in rng.integers(0, 400, S))
        ln = [int(x) for x in rng.integers(0, 40, S)]
        ln[0] = 100_000
    keys = [int(k) | 1 for k in rng.integers(0, 1 << 63, S, dtype=np.uint64)]
    bases = [int(x) for x in rng.integers(0, 1 << 63, S, dtype=np.uint64)]
    return off, ln, keys, bases


def _expected(off, ln):
    return {off[s] + i: (s, i) for s in range(len(off)) for i in range(ln[s])}


TILE_SHAPES = [(8, 8, 0, 1), (8, 8, 3, 3), (16, 16, 7, 7), (4, 8, 5, 2), (4, 8, 0, 7)]


def test_tile_model_valid_batches():
    rng = np.random.default_rng(0)
    for trial in range(300):
        off, ln, _, _ = _valid_batch(rng, trial)
        nelem = off[-1] + ln[-1] + 40
        want = _expected(off, ln)
        for block, EPV, head, grid in TILE_SHAPES:
            assert tile_writes(off, ln, head, block, EPV, grid, nelem) == want, (trial, block, EPV,
                                                                                 head, grid)


def test_tile_model_invalid_metadata_stays_inside_the_extent():
    rng = np.random.default_rng(1)
    for trial in range(300):
        off, ln, _, _ = _invalid_batch(rng, trial % 4)
        end = off[-1] + ln[-1]
        for block, EPV, head, grid in TILE_SHAPES:
            tile_writes(off, ln, head, block, EPV, grid, max(end, 0))  # asserts inside


@pytest.mark.parametrize("LPS", [32, 16, 8, 4, 1])
def test_stream_model(LPS):
    rng = np.random.default_rng(2)
    for trial in range(40):
        off, ln, _, _ = _valid_batch(rng, trial)
        got = stream_writes(off, ln, LPS, groups=int(rng.integers(1, 9)))
        assert {e: v[0] for e, v in got.items()} == _expected(off, ln)
        assert all(len(v) == 1 for v in got.values())
        off, ln, _, _ = _invalid_batch(rng, trial % 4)
        end = off[-1] + ln[-1]
        assert all(0 <= e < end for e in stream_writes(off, ln, LPS, groups=3))


def test_flat_model_valid_batches():
    rng = np.random.default_rng(3)
    for trial in range(400):
        off, ln, keys, bases = _valid_batch(rng, trial)
        got = flat_writes(keys, bases, off, ln, force64=bool(trial % 3 == 0))
        positions = [e for e, _, _, _ in got]
        assert len(positions) == len(set(positions)), trial
        assert {e: (s, i) for e, s, i, _ in got} == _expected(off, ln), trial
        for e, s, i, y in got:
            assert y == ((bases[s] + i) * keys[s]) & M64, (trial, e)


def test_flat_model_invalid_metadata_stays_inside_the_extent():
    rng = np.random.default_rng(4)
    for trial in range(300):
        off, ln, keys, bases = _invalid_batch(rng, trial % 4)
        end = off[-1] + ln[-1]
        for e, s, i, _ in flat_writes(keys, bases, off, ln, force64=bool(trial % 2)):
            assert 0 <= e < end, (trial, e, end)
            assert off[s] <= e < off[s] + ln[s]  # inside its own stream as well


def test_flat_model_huge_lengths_are_capped():
    """Lengths near 2^62 on contract-violating metadata: the 2^57 cap keeps
    the scan from overflowing; a small extent still bounds every write."""
    off = [0, 5, 10]
    ln = [(1 << 62), (1 << 62) - 7, 6]
    keys, bases = [3, 5, 7], [0, 0, 0]
    for e, s, i, _ in flat_writes(keys, bases, off, ln):
        assert 0 <= e < 16


SEG_CS = [4, 8, 16]


@pytest.mark.parametrize("C", SEG_CS)
def test_seg_model_valid_batches(C):
    """Flattened warps over aligned segments: every element written once
    with its own stream's Weyl term, on batches with and without gaps, for
    every placement of the output pointer modulo C; every whole segment's
    vector store aligned."""
    rng = np.random.default_rng(31 + C)
    for trial in range(300):
        off, ln, keys, bases = _valid_batch(rng, trial)
        out_elem = int(rng.integers(0, 64))
        got = seg_writes(keys, bases, off, ln, C, out_elem)
        positions = [e for e, _, _, _ in got]
        assert len(positions) == len(set(positions)), trial
        assert {e: (s, i) for e, s, i, _ in got} == _expected(off, ln), trial
        for e, s, i, y in got:
            assert y == ((bases[s] + i) * keys[s]) & M64, (trial, e)


@pytest.mark.parametrize("C", SEG_CS)
def test_seg_model_recipe_batches(C):
    """The benchmark's short-stream length ranges (packed, with empty
    streams), and the switch to the per-position walk for a group holding a
    stream at or above the length cap (a small cap in the model)."""
    rng = np.random.default_rng(41 + C)
    for trial in range(60):
        S = int(rng.integers(1, 100))
        lo, hi = [(3, 30), (30, 300), (1, 4)][trial % 3]
        ln = [int(x) for x in rng.integers(lo, hi, S)]
        for s in rng.integers(0, S, 3):
            ln[int(s)] = 0
        lead = int(rng.integers(0, 9))
        off = [int(x) + lead for x in np.concatenate([[0], np.cumsum(ln)[:-1]])]
        keys = [int(k) | 1 for k in rng.integers(0, 1 << 63, S, dtype=np.uint64)]
        bases = [int(x) for x in rng.integers(0, 1 << 64, S, dtype=np.uint64)]
        for cap in (SEG_LEN_CAP, hi // 2):
            got = seg_writes(keys, bases, off, ln, C, int(rng.integers(0, 32)), cap=cap)
            assert {e: (s, i) for e, s, i, _ in got} == _expected(off, ln), (trial, cap)
            assert len(got) == sum(ln)
            for e, s, i, y in got:
                assert y == ((bases[s] + i) * keys[s]) & M64, (trial, e)


@pytest.mark.parametrize("C", SEG_CS)
def test_seg_model_invalid_metadata_stays_inside_the_extent(C):
    rng = np.random.default_rng(51 + C)
    for trial in range(300):
        off, ln, keys, bases = _invalid_batch(rng, trial % 4)
        end = off[-1] + ln[-1]
        for e, s, i, _ in seg_writes(keys, bases, off, ln, C, int(rng.integers(0, 32)),
                                     cap=int(rng.choice([SEG_LEN_CAP, 200]))):
            assert 0 <= e < end, (trial, e, end)
            assert off[s] <= e < off[s] + ln[s]


@pytest.mark.parametrize("C", SEG_CS)
def test_seg_index_widths(C):
    """Below the cap every whole-segment index and count of a group, and every
    in-stream element index, fits the kernel's 32-bit arithmetic, and the
    total stays below the 0xC0000000 sentinel that streams without whole
    segments take: 32 streams of 2^26 - 1 values, each starting C - 1
    elements past a cut."""
    hi = (C - 1) + SEG_LEN_CAP - 1
    nw = hi // C - 1
    R = 32 * nw
    assert hi < (1 << 32)
    assert R + 31 < (1 << 30)
    assert 0xC0000000 - R > 32
    assert (nw - 1) * C + C - 1 < (1 << 32)
