// Ragged batch of squares32 streams in one persistent launch.
//
// The packed output index space is cut into tiles of blockDim * EPV elements
// (EPV = 8 or 16 consecutive outputs per thread), aligned to the output's
// 32-byte boundary.
// CTA c of the persistent grid owns one contiguous run of tiles, so as it
// walks its run the stream index only grows: one binary search over the
// offsets at the start, then a forward step whenever a tile crosses into
// the next stream. A run of whole tiles inside one stream is generated like
// the plain kernel (Weyl stepping by tile * key, 32-byte vector stores). In
// a tile that touches a stream boundary, a gap or the end of the batch each
// thread finds the stream of its own chunk by a galloping search forward;
// chunks inside one stream still take the vector path and only chunks that
// straddle a boundary are written element by element. The batch extent
// offsets[S-1] + lengths[S-1] is read on the device, so the launch needs no
// host-side knowledge of the lengths and can be captured in a CUDA graph;
// no write lands outside it, whatever the other streams' offsets. There are
// no spin-waits and no inter-CTA communication. Batches of many short
// streams are better served by the streams-to-lanes kernels (variants 4-8)
// and the flattened-warp kernels (variants 9-12) further down, which the
// batch autotuner picks when they win.
#include <cuda_runtime.h>

#include "internal.h"
#include "squares_device.cuh"
#include "stores.cuh"

namespace sq {
namespace {

constexpr uint32_t kNoStream = 0xFFFFFFFFu;

// Largest s in [from, S) with offsets[s] <= e, given offsets[from] <= e:
// gallop forward (from+1, from+2, from+4, ...) then bisect, so a stream d
// positions ahead costs about 2 log2(d) loads -- one or two at a boundary.
__device__ __forceinline__ uint32_t find_stream(const int64_t *__restrict__ offsets, uint32_t S,
                                                uint32_t from, int64_t e) {
    uint32_t lo = from, step = 1;
    while (step <= S - 1 - lo && __ldg(offsets + lo + step) <= e) {
        lo += step;
        step <<= 1;
    }
    uint32_t hi = (step <= S - lo) ? lo + step : S;
    while (hi - lo > 1) {
        const uint32_t mid = lo + (hi - lo) / 2;
        if (__ldg(offsets + mid) <= e) lo = mid; else hi = mid;
    }
    return lo;
}

// squares32 of C consecutive counters from y = ctr*key, e = t(ctr+1) - t(ctr)
// and c2 = 2*key^2: one squaring for round 1, then additions (the
// recurrence of round1_delta): t_{j+1} = t_j + e + j*c2, one three-input
// addition per counter with e fixed for the chunk. (In the tile kernel the
// key is fixed over a run of whole tiles; carrying e by accumulation
// instead, as the segment walk does, measured 5 % slower there.)
template <int C>
__device__ __forceinline__ void run32(uint64_t y, uint64_t e, uint64_t key, uint64_t c2, uint32_t (&w)[C]) {
    uint64_t t = round1_value(y);
#pragma unroll
    for (int j = 0; j < C; ++j) {
        const uint64_t z = add64(y, key);
        w[j] = squares32_tyz(t, y, z);
        y = z;
        t = add64x3(t, e, c2 * static_cast<uint64_t>(j));
    }
}

// Stream containing or preceding position e, searching forward from `from`
// (kNoStream: nothing found yet). kNoStream if e precedes the first stream.
__device__ __forceinline__ uint32_t stream_at(const int64_t *__restrict__ offsets, uint32_t S,
                                              uint32_t from, int64_t e) {
    if (from == kNoStream) {
        if (__ldg(offsets) > e) return kNoStream;
        from = 0;
    }
    return find_stream(offsets, S, from, e);
}

// Writes the EPV consecutive positions [e0, e0 + EPV) of a tile that touches
// a stream boundary, a gap or the end of the batch: a chunk that lies inside
// one stream is generated and stored like a whole tile; otherwise element by
// element, walking forward across stream boundaries (Weyl steps inside each
// stream) and skipping positions that no stream covers.
template <bool CS, int EPV>
__device__ __forceinline__ void boundary_chunk(const uint64_t *__restrict__ keys,
                                               const uint64_t *__restrict__ bases,
                                               const int64_t *__restrict__ lengths,
                                               const int64_t *__restrict__ offsets, uint32_t S,
                                               uint32_t from, int64_t e0, int64_t end,
                                               uint32_t *__restrict__ out) {
    if (e0 >= end) return;
    uint32_t s = stream_at(offsets, S, from, e0);
    if (s == kNoStream) {  // e0 precedes the first stream: start at stream 0
        s = 0;
    }
    int64_t seg_lo = __ldg(offsets + s);
    int64_t seg_hi = seg_lo + __ldg(lengths + s);
    if (seg_lo <= e0 && e0 + EPV <= seg_hi && e0 + EPV <= end) {
        const uint64_t key = __ldg(keys + s);
        const uint64_t y = (__ldg(bases + s) + static_cast<uint64_t>(e0 - seg_lo)) * key;
        uint32_t w[EPV];
        run32<EPV>(y, round1_delta(y, key), key, (key * key) << 1, w);
        store32B<CS>(out + e0, *reinterpret_cast<const uint32_t(*)[8]>(&w[0]));
        if constexpr (EPV == 16)
            store32B<CS>(out + e0 + 8, *reinterpret_cast<const uint32_t(*)[8]>(&w[8]));
        return;
    }
    uint64_t key = __ldg(keys + s);
    uint64_t y = 0;
    bool have_y = false;
#pragma unroll 1
    for (int j = 0; j < EPV; ++j) {
        const int64_t e = e0 + j;
        if (e >= end) break;
        if (e >= seg_hi && s + 1 < S) {  // next stream(s); empty ones are skipped
            s = find_stream(offsets, S, s, e);
            seg_lo = __ldg(offsets + s);
            seg_hi = seg_lo + __ldg(lengths + s);
            key = __ldg(keys + s);
            have_y = false;
        }
        if (e < seg_lo || e >= seg_hi) continue;  // a gap
        if (!have_y) {
            y = (__ldg(bases + s) + static_cast<uint64_t>(e - seg_lo)) * key;
            have_y = true;
        }
        const uint64_t z = add64(y, key);
        out[e] = squares32_yz(y, z);
        y = z;
    }
}

// EPV consecutive outputs per thread per tile: 8 (one 32-byte store) or 16
// (two adjacent 32-byte stores). Register targets by chunk size (measured on
// a 4096-stream batch of mean length 10^6 and a 2^14-stream batch of mean
// 11,800): 16-value chunks gain 2 % with room for 3 CTAs of 512 threads per
// SM (42 registers) rather than 4; 8-value chunks lose 4 % with it.
template <bool CS, int EPV>
__global__ void __launch_bounds__(512, EPV == 16 ? 3 : 4)
    batch_kernel(const uint64_t *__restrict__ keys, const uint64_t *__restrict__ bases,
                 const int64_t *__restrict__ lengths, const int64_t *__restrict__ offsets,
                 uint32_t S, uint32_t *__restrict__ out, uint32_t head) {
    const int tile = blockDim.x * EPV;  // a power of two
    const int shift = __ffs(tile) - 1;
    if (S == 0) return;
    const int64_t start = __ldg(offsets);
    const int64_t end = __ldg(offsets + S - 1) + __ldg(lengths + S - 1);

    // Elements before the first 32-byte boundary (fewer than 8), by CTA 0.
    if (blockIdx.x == 0) {
        for (int64_t e = threadIdx.x; e < static_cast<int64_t>(head) && e < end; e += blockDim.x) {
            const uint32_t s = stream_at(offsets, S, kNoStream, e);
            if (s != kNoStream) {
                const int64_t off = __ldg(offsets + s);
                if (e < off + __ldg(lengths + s))
                    out[e] = squares32(__ldg(bases + s) + static_cast<uint64_t>(e - off), __ldg(keys + s));
            }
        }
    }
    if (end <= static_cast<int64_t>(head)) return;

    const int64_t first = start > static_cast<int64_t>(head) ? start : head;
    const int64_t t_begin = (first - head) >> shift;
    const int64_t t_end = (end - head + tile - 1) >> shift;
    const int64_t per = (t_end - t_begin + gridDim.x - 1) / gridDim.x;
    int64_t t = t_begin + static_cast<int64_t>(blockIdx.x) * per;
    const int64_t t_stop = (t + per < t_end) ? t + per : t_end;
    if (t >= t_stop) return;

    uint32_t s = stream_at(offsets, S, kNoStream, head + (t << shift));
    while (t < t_stop) {
        const int64_t lo = head + (t << shift);
        if (s == kNoStream || (s + 1 < S && __ldg(offsets + s + 1) <= lo)) s = stream_at(offsets, S, s, lo);
        int64_t k = 0;
        int64_t seg_lo = 0;
        if (s != kNoStream) {
            seg_lo = __ldg(offsets + s);
            int64_t seg_hi = seg_lo + __ldg(lengths + s);
            if (seg_hi > end) seg_hi = end;  // only met when the offsets break the requirements
            if (lo + tile <= seg_hi) {
                k = (seg_hi - lo) >> shift;
                if (k > t_stop - t) k = t_stop - t;
            }
        }
        if (k > 0) {
            // Whole tiles inside stream s.
            const uint64_t key = __ldg(keys + s);
            const int64_t e = lo + threadIdx.x * EPV;
            uint64_t y = (__ldg(bases + s) + static_cast<uint64_t>(e - seg_lo)) * key;
            const uint64_t c2 = (key * key) << 1;
            uint64_t er = round1_delta(y, key);
            const uint64_t ystep = key << shift;  // one tile of counters
            const uint64_t estep = c2 << shift;
            uint32_t *p = out + e;
            for (int64_t i = 0; i < k; ++i) {
                uint32_t w[EPV];
                run32<EPV>(y, er, key, c2, w);
                store32B<CS>(p, *reinterpret_cast<const uint32_t(*)[8]>(&w[0]));
                if constexpr (EPV == 16)
                    store32B<CS>(p + 8, *reinterpret_cast<const uint32_t(*)[8]>(&w[8]));
                y = add64(y, ystep);
                er = add64(er, estep);
                p += tile;
            }
            t += k;
        } else {
            boundary_chunk<CS, EPV>(keys, bases, lengths, offsets, S, s, lo + threadIdx.x * EPV, end, out);
            t += 1;
        }
    }
}

// Streams to lanes, for batches of many short streams: a group of LPS
// consecutive lanes (32, 16, 8, 4 or 1) takes stream s, s + G, ... (G groups
// in the grid); lane j of the group writes elements j, j + LPS, ... of the
// stream, so a group's store covers LPS consecutive outputs. The lane's
// counters are LPS apart and y steps by d = LPS * key. With 32 or 16 lanes
// per stream round 1 is carried by round1_delta(y, d), which grows by 2d^2
// per step, four values per loop iteration; with 8 or fewer lanes per stream
// (meant for streams of a few dozen values or fewer, a few per lane) round 1
// is squared for each value, since the recurrence's setup would cost more
// (both choices measured). A stream's metadata loads are the same address
// for every lane of the group and are issued one stream ahead. Any offsets
// are accepted, gaps are untouched, and no stream lookup is needed.
template <int LPS>
__global__ void __launch_bounds__(512)
    batch_stream_kernel(const uint64_t *__restrict__ keys, const uint64_t *__restrict__ bases,
                        const int64_t *__restrict__ lengths, const int64_t *__restrict__ offsets,
                        uint32_t S, uint32_t *__restrict__ out) {
    const uint64_t gt = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const uint32_t j = static_cast<uint32_t>(gt % LPS);
    const uint64_t groups = (static_cast<uint64_t>(gridDim.x) * blockDim.x) / LPS;
    // Like the tile kernels, write nothing outside [0, end), end the extent
    // offsets[S-1] + lengths[S-1], whatever the other streams' offsets are.
    const int64_t end = __ldg(offsets + S - 1) + __ldg(lengths + S - 1);
    // The next stream's metadata is loaded while the current one is written.
    uint64_t s = gt / LPS;
    int64_t n_len = 0, n_off = 0;
    uint64_t n_key = 0, n_base = 0;
    if (s < S) {
        n_len = __ldg(lengths + s);
        n_off = __ldg(offsets + s);
        n_key = __ldg(keys + s);
        n_base = __ldg(bases + s);
    }
    for (; s < S; s += groups) {
        const int64_t off = n_off;
        const int64_t len = (n_len < end - off) ? n_len : end - off;
        const uint64_t key = n_key;
        const uint64_t base = n_base;
        if (s + groups < S) {
            n_len = __ldg(lengths + s + groups);
            n_off = __ldg(offsets + s + groups);
            n_key = __ldg(keys + s + groups);
            n_base = __ldg(bases + s + groups);
        }
        if (off < 0 || len <= static_cast<int64_t>(j)) continue;
        uint32_t *o = out + off;
        uint64_t y = (base + j) * key;
        const uint64_t d = key * LPS;
        if constexpr (LPS >= 16) {
            uint64_t t = round1_value(y);
            uint64_t dt = round1_delta(y, d);
            const uint64_t ddt = (d * d) << 1;
            const uint64_t ddt2 = ddt << 1, ddt3 = ddt2 + ddt, ddt4 = ddt << 2;
            int64_t i = j;
            // four values per step: t advances by dt + m*ddt for the m-th
            // (one three-input addition each), dt by 4*ddt per step
            for (; i + 3 * LPS < len; i += 4 * LPS) {
                uint64_t z = add64(y, key);
                o[i] = squares32_tyz(t, y, z);
                y = add64(y, d);
                t = add64(t, dt);
                z = add64(y, key);
                o[i + LPS] = squares32_tyz(t, y, z);
                y = add64(y, d);
                t = add64x3(t, dt, ddt);
                z = add64(y, key);
                o[i + 2 * LPS] = squares32_tyz(t, y, z);
                y = add64(y, d);
                t = add64x3(t, dt, ddt2);
                z = add64(y, key);
                o[i + 3 * LPS] = squares32_tyz(t, y, z);
                y = add64(y, d);
                t = add64x3(t, dt, ddt3);
                dt = add64(dt, ddt4);
            }
            for (; i < len; i += LPS) {
                o[i] = squares32_tyz(t, y, add64(y, key));
                y = add64(y, d);
                t = add64(t, dt);
                dt = add64(dt, ddt);
            }
        } else {
            for (int64_t i = j; i < len; i += LPS) {
                o[i] = squares32_yz(y, add64(y, key));
                y = add64(y, d);
            }
        }
    }
}

// One entry of a warp's stream table, for a stream that starts at position
// P of the warp's value sequence: y0 = (base - P) * key, so that position p
// has Weyl term y = y0 + p * key; the address of the output of position 0
// (out + offset - P, as an integer: it may lie before out); the key.
struct alignas(16) FlatEntry {
    uint64_t y0;
    uint64_t dst;
    uint64_t key;
    uint64_t pad;
};

// 1 << r for r < 32, else 0 (shl.b32 clamps the shift amount at 32).
__device__ __forceinline__ uint32_t window_bit(uint32_t r) {
    uint32_t v;
    asm("shl.b32 %0, 1, %1;" : "=r"(v) : "r"(r));
    return v;
}
__device__ __forceinline__ uint32_t window_bit(uint64_t r) {
    return r < 32 ? window_bit(static_cast<uint32_t>(r)) : 0u;
}

// The walk of a warp's value sequence, 32 positions per step; Pos is
// uint32_t when the sequence has fewer than 2^31 values, else uint64_t. Pe
// is the lane's stream start P, or a sentinel that no window reaches when
// its stream is empty.
template <typename Pos>
__device__ __forceinline__ void flat_walk(const FlatEntry *table, Pos Pe, Pos T, uint32_t lane) {
    const uint32_t le = 0xFFFFFFFFu >> (31u - lane);
    uint32_t before = 0xFFFFFFFFu;  // streams started before the window, minus 1
    for (Pos b = 0; b < T; b += 32) {
        const uint32_t starts = __reduce_or_sync(0xFFFFFFFFu, window_bit(static_cast<Pos>(Pe - b)));
        const Pos p = b + lane;
        const uint32_t k = before + __popc(starts & le);
        before += __popc(starts);
        if (p < T) {
            const FlatEntry &e = table[k];
            const uint64_t y = e.y0 + static_cast<uint64_t>(p) * e.key;
            uint32_t *dst = reinterpret_cast<uint32_t *>(e.dst) + p;
            *dst = squares32_yz(y, add64(y, e.key));
        }
    }
}

// Flattened warps, for batches of streams of a few values to a few hundred:
// warp w takes streams 32g .. 32g + 31 for g = w, w + W, ... (W warps in the
// grid). Lane L loads stream 32g + L's metadata (coalesced loads), clamps
// its length to the extent, and a warp scan of the lengths lays the 32
// streams' values end to end: stream L owns positions P_L .. P_L + len_L - 1
// of a sequence of T values. The non-empty streams' entries (FlatEntry) go,
// in order, to a 32-entry table of the warp in shared memory. The warp then
// walks the sequence 32 positions per step, lane t taking position
// p = b + t: each stream that starts inside the step sets one bit (an OR
// across the warp), so the owner of p is entry (streams started before the
// step) + (bits set at or below t) - 1, and p's output is squares32 of
// y = y0 + p * key, stored at dst + p. Every lane of a step does the same
// work whatever the lengths, and consecutive positions of a stream are
// consecutive outputs, so the stores stay coalesced; round 1 is squared for
// each value. Positions are 32-bit unless the 32 streams hold 2^31 values or
// more. A clamped length is also capped at 2^57 so that the 64-bit scan
// cannot overflow; every write then lies inside its owner's clamped range,
// whatever the metadata.
// Lane L's stream s = g + L of a flattened warp's group: its metadata, with
// the length clamped to the batch extent (0 for a negative offset or s past
// the last stream, at most 2^57).
struct StreamMeta {
    int64_t len, off;
    uint64_t key, base;
};

__device__ __forceinline__ StreamMeta stream_meta(const uint64_t *__restrict__ keys,
                                                  const uint64_t *__restrict__ bases,
                                                  const int64_t *__restrict__ lengths,
                                                  const int64_t *__restrict__ offsets, uint32_t S,
                                                  int64_t end, uint64_t s) {
    constexpr int64_t kLenCap = int64_t{1} << 57;
    StreamMeta m{0, 0, 0, 0};
    if (s < S) {
        m.len = __ldg(lengths + s);
        m.off = __ldg(offsets + s);
        m.key = __ldg(keys + s);
        m.base = __ldg(bases + s);
    }
    if (m.off < 0) m.len = 0;
    else if (m.len > end - m.off) m.len = end - m.off;
    if (m.len < 0) m.len = 0;
    if (m.len > kLenCap) m.len = kLenCap;
    return m;
}

// One group of 32 streams of a flattened warp: lane L's stream and its first
// position P in the warp's value sequence (exclusive scan of the clamped
// lengths; T values in all).
struct FlatGroup {
    int64_t len, off, P, T;
    uint64_t key, base;
    uint32_t nonempty;  // lanes with len > 0
};

// The scan runs in 32-bit words when every length is below 2^26 (so that
// the 32 lengths sum below 2^31), else in 64-bit words.
__device__ __forceinline__ FlatGroup flat_group(const StreamMeta &m, uint32_t lane) {
    FlatGroup fg{m.len, m.off, 0, 0, m.key, m.base, 0};
    if (__any_sync(0xFFFFFFFFu, fg.len >= (int64_t{1} << 26))) {
        int64_t inc = fg.len;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t o = __shfl_up_sync(0xFFFFFFFFu, inc, d);
            if (lane >= static_cast<uint32_t>(d)) inc += o;
        }
        fg.P = inc - fg.len;
        fg.T = __shfl_sync(0xFFFFFFFFu, inc, 31);
    } else {
        const uint32_t len = static_cast<uint32_t>(fg.len);
        uint32_t inc = len;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, inc, d);
            if (lane >= static_cast<uint32_t>(d)) inc += o;
        }
        fg.P = static_cast<int64_t>(inc - len);
        fg.T = static_cast<int64_t>(__shfl_sync(0xFFFFFFFFu, inc, 31));
    }
    fg.nonempty = __ballot_sync(0xFFFFFFFFu, fg.len > 0);
    return fg;
}

// The group's walk one position per lane per step (see flat_walk): the
// non-empty streams' entries go, in order, to the warp's table.
__device__ __forceinline__ void flat_positions(FlatEntry *table, const FlatGroup &fg,
                                               uint32_t *__restrict__ out, uint32_t lane) {
    if (fg.len > 0) {
        FlatEntry &e = table[__popc(fg.nonempty & ((1u << lane) - 1u))];
        e.y0 = (fg.base - static_cast<uint64_t>(fg.P)) * fg.key;
        e.dst = reinterpret_cast<uint64_t>(out) + static_cast<uint64_t>(fg.off - fg.P) * 4u;
        e.key = fg.key;
    }
    __syncwarp();
    if (fg.T < (int64_t{1} << 31))
        flat_walk<uint32_t>(table, fg.len > 0 ? static_cast<uint32_t>(fg.P) : 0xC0000000u,
                            static_cast<uint32_t>(fg.T), lane);
    else
        flat_walk<uint64_t>(table, fg.len > 0 ? static_cast<uint64_t>(fg.P) : 0xC000000000000000ull,
                            static_cast<uint64_t>(fg.T), lane);
    __syncwarp();
}

__global__ void __launch_bounds__(512)
    batch_flat_kernel(const uint64_t *__restrict__ keys, const uint64_t *__restrict__ bases,
                      const int64_t *__restrict__ lengths, const int64_t *__restrict__ offsets,
                      uint32_t S, uint32_t *__restrict__ out) {
    extern __shared__ FlatEntry flat_tables[];
    FlatEntry *table = flat_tables + (threadIdx.x & ~31u);
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warp = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const uint64_t stride = ((static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5) * 32;
    const int64_t end = __ldg(offsets + S - 1) + __ldg(lengths + S - 1);
    for (uint64_t g = warp * 32; g < S; g += stride)
        flat_positions(table, flat_group(stream_meta(keys, bases, lengths, offsets, S, end, g + lane), lane), out,
                       lane);
}

// Flattened warps over aligned segments (variants 10-12, C = 4, 8 or 16),
// for the same batches and any offsets. The output is cut at every C-element
// boundary of its address (4C bytes); a stream's outputs fall into whole
// segments (aligned blocks of C outputs of the stream) and at most two
// pieces (the shorter runs at its start and end, or one run when the stream
// lies inside one block). A warp takes 32 streams at a time, in two passes:
//
// * Whole segments. The streams' whole segments are laid end to end (an
//   exclusive scan of the counts, one per lane) and walked 32 per step, one
//   segment per lane, owner found as in flat_walk (one bit per stream start
//   in the step, a warp OR and a population count) over a table of the
//   streams that have whole segments. The table holds each stream's Weyl
//   term, round-1 step and output address at its first whole segment, and
//   the per-segment strides, so segment j of the stream starts from
//   y + j * (C * key), e + j * (C * c2) and dst + j * C: every lane generates
//   C consecutive counters of one stream (round 1 squared once, then carried
//   by additions) and writes them with one aligned vector store.
// * Pieces. Each lane writes its own stream's pieces, element by element:
//   C counters from the piece's block start, stored where they fall inside
//   the stream.
//
// The key differs from lane to lane, so round 1's step is carried by
// accumulation (t += e, e += c2: additions only) rather than by the
// launch-uniform j * c2 terms the plain kernels use. Nothing is written
// outside the owner's clamped range. A group holding a stream of 2^26
// values or more takes batch_flat_kernel's walk instead, so that segment
// counts and in-stream positions stay 32-bit.

// squares32 of C consecutive counters of one key from y, e = t(ctr+1) -
// t(ctr) and c2 = 2*key^2, round 1 carried by two additions per counter.
template <int C>
__device__ __forceinline__ void run32_lane(uint64_t y, uint64_t e, uint64_t key, uint64_t c2, uint32_t (&w)[C]) {
    uint64_t t = round1_value(y);
#pragma unroll
    for (int j = 0; j < C; ++j) {
        const uint64_t z = add64(y, key);
        w[j] = squares32_tyz(t, y, z);
        y = z;
        t = add64(t, e);
        e = add64(e, c2);
    }
}

// One stream of a warp's whole-segment table: at its first whole segment the
// Weyl term y, the round-1 step e and the output address dst (4C-byte
// aligned); key and c2 = 2*key^2; the strides of one segment, C*key and
// C*c2; Q, the stream's first whole segment in the warp's sequence.
struct alignas(16) SegEntry {
    uint64_t y, key, e, c2, kc, c2c, dst;
    uint32_t Q, pad;
};
static_assert(sizeof(SegEntry) >= sizeof(FlatEntry), "the flat walk's table fits a segment table's slots");

constexpr int64_t kSegLenCap = int64_t{1} << 26;

template <int C>
__device__ __forceinline__ void seg_store(uint32_t *p, const uint32_t (&w)[C]) {
    if constexpr (C == 4) {
        store16B<false>(p, w[0], w[1], w[2], w[3]);
    } else {
        store32B<false>(p, *reinterpret_cast<const uint32_t(*)[8]>(&w[0]));
        if constexpr (C == 16) store32B<false>(p + 8, *reinterpret_cast<const uint32_t(*)[8]>(&w[8]));
    }
}

// The whole-segment pass. The stream's first output lies lo elements past a
// block start; its outputs are elements lo .. hi - 1 counted from there, and
// its whole segments the blocks ws .. we - 1 (ws = 1 if lo > 0, we = hi / C).
template <int C, int LC>
__device__ __forceinline__ void seg_whole(SegEntry *tab, const StreamMeta &m, uint32_t lo, uint32_t hi,
                                          uint32_t *__restrict__ out, uint32_t lane) {
    const uint32_t le = 0xFFFFFFFFu >> (31u - lane);
    const uint32_t ws = lo != 0u;
    const uint32_t we = hi >> LC;
    const uint32_t nw = (m.len > 0 && we > ws) ? we - ws : 0u;
    uint32_t inc = nw;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, inc, d);
        if (lane >= static_cast<uint32_t>(d)) inc += o;
    }
    const uint32_t Q = inc - nw;
    const uint32_t R = __shfl_sync(0xFFFFFFFFu, inc, 31);
    const uint32_t with = __ballot_sync(0xFFFFFFFFu, nw > 0u);
    if (nw > 0u) {
        const uint64_t K = m.key;
        const uint64_t first = (static_cast<uint64_t>(ws) << LC) - lo;  // first whole element, from the stream's
        const uint64_t y = (m.base + first) * K;
        const uint64_t c2 = (K * K) << 1;
        tab[__popc(with & (le >> 1))] =
            SegEntry{y, K, round1_delta(y, K), c2, K << LC, c2 << LC,
                     reinterpret_cast<uint64_t>(out) + (static_cast<uint64_t>(m.off) + first) * 4u, Q, 0u};
    }
    __syncwarp();
    // Streams without whole segments set no bit: their start never falls in
    // a window (R < 2^30 below the 0xC0000000 sentinel).
    const uint32_t Pe = nw > 0u ? Q : 0xC0000000u;
    uint32_t before = 0xFFFFFFFFu;  // table entries started before the step, minus 1
    for (uint32_t b = 0; b < R; b += 32) {
        const uint32_t starts = __reduce_or_sync(0xFFFFFFFFu, window_bit(Pe - b));
        const uint32_t k = before + __popc(starts & le);
        before += __popc(starts);
        const uint32_t r = b + lane;
        if (r < R) {
            const SegEntry &e = tab[k];
            const uint32_t j = r - e.Q;
            uint32_t w[C];
            run32_lane<C>(e.y + static_cast<uint64_t>(j) * e.kc, e.e + static_cast<uint64_t>(j) * e.c2c, e.key, e.c2,
                          w);
            seg_store<C>(reinterpret_cast<uint32_t *>(e.dst) + (static_cast<size_t>(j) << LC), w);
        }
    }
}

// The pieces pass: block 0 when the stream starts inside it or ends before
// its end (elements lo .. min(hi, C) - 1), and the last block nseg - 1 when
// it is another block and the stream ends inside it (elements (nseg-1)*C ..
// hi - 1). Each is C counters from the block start, stored element by
// element where they fall inside the stream.
template <int C, int LC>
__device__ __forceinline__ void seg_pieces(const StreamMeta &m, uint32_t lo, uint32_t hi,
                                           uint32_t *__restrict__ out) {
    const bool has = m.len > 0;
    const uint32_t nseg = (hi + C - 1) >> LC;
    const bool head = has && (lo != 0u || hi < static_cast<uint32_t>(C));
    const bool tail = has && (hi & (C - 1)) != 0u && nseg > 1u;
#pragma unroll 1
    for (int piece = 0; piece < 2; ++piece) {
        if (piece == 0 ? head : tail) {
            const uint32_t b0 = piece == 0 ? 0u : (nseg - 1u) << LC;  // block start, from the block origin
            const uint32_t p_lo = piece == 0 ? lo : b0;
            const uint32_t p_hi = hi < b0 + C ? hi : b0 + C;
            const uint64_t K = m.key;
            const uint64_t y = (m.base - lo + b0) * K;
            uint32_t w[C];
            run32_lane<C>(y, round1_delta(y, K), K, (K * K) << 1, w);
            // the block's first output, before out + off when lo > off
            uint32_t *p = reinterpret_cast<uint32_t *>(reinterpret_cast<uint64_t>(out) +
                                                       (static_cast<uint64_t>(m.off) - lo + b0) * 4u);
#pragma unroll
            for (int i = 0; i < C; ++i)
                if (b0 + i >= p_lo && b0 + i < p_hi) p[i] = w[i];
        }
    }
}

template <int C>
__global__ void __launch_bounds__(512)
    batch_seg_kernel(const uint64_t *__restrict__ keys, const uint64_t *__restrict__ bases,
                     const int64_t *__restrict__ lengths, const int64_t *__restrict__ offsets,
                     uint32_t S, uint32_t *__restrict__ out) {
    constexpr int LC = C == 4 ? 2 : C == 8 ? 3 : 4;
    static_assert(C == 1 << LC, "C is 4, 8 or 16");
    extern __shared__ SegEntry seg_tables[];
    SegEntry *tab = seg_tables + (threadIdx.x & ~31u);
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warp = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const uint64_t stride = ((static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5) * 32;
    const int64_t end = __ldg(offsets + S - 1) + __ldg(lengths + S - 1);
    // the output's distance past a C-element boundary of its address
    const uint32_t a = static_cast<uint32_t>((reinterpret_cast<uintptr_t>(out) >> 2) & (C - 1));
    for (uint64_t g = warp * 32; g < S; g += stride) {
        const StreamMeta m = stream_meta(keys, bases, lengths, offsets, S, end, g + lane);
        if (__any_sync(0xFFFFFFFFu, m.len >= kSegLenCap)) {
            flat_positions(reinterpret_cast<FlatEntry *>(tab), flat_group(m, lane), out, lane);
            continue;
        }
        const uint32_t lo = static_cast<uint32_t>((static_cast<uint64_t>(m.off) + a) & (C - 1));
        const uint32_t hi = lo + static_cast<uint32_t>(m.len);
        seg_whole<C, LC>(tab, m, lo, hi, out, lane);
        seg_pieces<C, LC>(m, lo, hi, out);
        __syncwarp();  // the table is rewritten for the next group
    }
}

// Variants 0-3: tiles (8 or 16 elements per thread, default or streaming
// stores); 4-8: streams to lanes (32, 8, 16, 4 or 1 lanes per stream);
// 9: flattened warps, one position per lane; 10-12: flattened warps over
// aligned segments of 4, 8 or 16 values.
constexpr int kBatchVariants = 13;
const char *kBatchVariantNames[kBatchVariants] = {
    "st32",          "st32.cs",      "st32x2",       "st32x2.cs",    "warp-stream", "lane8-stream",
    "lane16-stream", "lane4-stream", "lane1-stream", "flat-warp",    "flat-seg4",   "flat-seg8",
    "flat-seg16"};

size_t batch_smem(int variant, int block) {
    if (variant == 9) return static_cast<size_t>(block) * sizeof(FlatEntry);
    return variant >= 10 ? static_cast<size_t>(block) * sizeof(SegEntry) : 0;
}

const void *batch_fn(int variant) {
    switch (variant) {
        case 0: return reinterpret_cast<const void *>(&batch_kernel<false, 8>);
        case 1: return reinterpret_cast<const void *>(&batch_kernel<true, 8>);
        case 2: return reinterpret_cast<const void *>(&batch_kernel<false, 16>);
        case 3: return reinterpret_cast<const void *>(&batch_kernel<true, 16>);
        case 4: return reinterpret_cast<const void *>(&batch_stream_kernel<32>);
        case 5: return reinterpret_cast<const void *>(&batch_stream_kernel<8>);
        case 6: return reinterpret_cast<const void *>(&batch_stream_kernel<16>);
        case 7: return reinterpret_cast<const void *>(&batch_stream_kernel<4>);
        case 8: return reinterpret_cast<const void *>(&batch_stream_kernel<1>);
        case 9: return reinterpret_cast<const void *>(&batch_flat_kernel);
        case 10: return reinterpret_cast<const void *>(&batch_seg_kernel<4>);
        case 11: return reinterpret_cast<const void *>(&batch_seg_kernel<8>);
        default: return reinterpret_cast<const void *>(&batch_seg_kernel<16>);
    }
}

}  // namespace

int batch_num_variants() { return kBatchVariants; }

const char *batch_variant_name(int variant) {
    return (variant >= 0 && variant < kBatchVariants) ? kBatchVariantNames[variant] : nullptr;
}

int batch_max_ctas_per_sm(int variant, int block) {
    return occupancy(batch_fn(variant), block, batch_smem(variant, block));
}

cudaError_t launch_batch(const Cfg &cfg, const uint64_t *keys, const uint64_t *bases,
                         const int64_t *lengths, const int64_t *offsets, size_t nstreams,
                         uint32_t *out, cudaStream_t stream) {
    if (nstreams == 0) return cudaSuccess;
    Cfg c = cfg;
    // Host-resident outputs: contiguous 1 KiB warp stores (see launch_plain).
    if ((c.variant == 2 || c.variant == 3) && !in_device_memory(out)) c.variant -= 2;
    const int ctas = c.ctas_per_sm > 0 ? c.ctas_per_sm : batch_max_ctas_per_sm(c.variant, c.block);
    const unsigned grid = static_cast<unsigned>(current_sm_count()) * static_cast<unsigned>(ctas);
    const uintptr_t addr = reinterpret_cast<uintptr_t>(out);
    const uint32_t head = static_cast<uint32_t>(((32 - (addr % 32)) % 32) / 4);
    const uint32_t S = static_cast<uint32_t>(nstreams);
    if (c.variant >= 9) {
        // Flattened warps: with ctas_per_sm = 0, one group of 32 streams per
        // warp (the block scheduler balances groups of unequal work);
        // otherwise a persistent grid of ctas_per_sm CTAs per SM.
        const uint64_t groups_grid = (static_cast<uint64_t>(S) + c.block - 1) / c.block;
        const unsigned fgrid = c.ctas_per_sm > 0 ? grid : static_cast<unsigned>(groups_grid);
        const size_t smem = batch_smem(c.variant, c.block);
        if (c.variant == 9)
            batch_flat_kernel<<<fgrid, c.block, smem, stream>>>(keys, bases, lengths, offsets, S, out);
        else if (c.variant == 10)
            batch_seg_kernel<4><<<fgrid, c.block, smem, stream>>>(keys, bases, lengths, offsets, S, out);
        else if (c.variant == 11)
            batch_seg_kernel<8><<<fgrid, c.block, smem, stream>>>(keys, bases, lengths, offsets, S, out);
        else
            batch_seg_kernel<16><<<fgrid, c.block, smem, stream>>>(keys, bases, lengths, offsets, S, out);
        return cudaGetLastError();
    }
    if (c.variant >= 4) {
        if (c.variant == 4)
            batch_stream_kernel<32><<<grid, cfg.block, 0, stream>>>(keys, bases, lengths, offsets, S, out);
        else if (c.variant == 5)
            batch_stream_kernel<8><<<grid, cfg.block, 0, stream>>>(keys, bases, lengths, offsets, S, out);
        else if (c.variant == 6)
            batch_stream_kernel<16><<<grid, cfg.block, 0, stream>>>(keys, bases, lengths, offsets, S, out);
        else if (c.variant == 7)
            batch_stream_kernel<4><<<grid, cfg.block, 0, stream>>>(keys, bases, lengths, offsets, S, out);
        else
            batch_stream_kernel<1><<<grid, cfg.block, 0, stream>>>(keys, bases, lengths, offsets, S, out);
        return cudaGetLastError();
    }
    switch (c.variant) {
        case 0: batch_kernel<false, 8><<<grid, cfg.block, 0, stream>>>(keys, bases, lengths, offsets, S, out, head); break;
        case 1: batch_kernel<true, 8><<<grid, cfg.block, 0, stream>>>(keys, bases, lengths, offsets, S, out, head); break;
        case 2: batch_kernel<false, 16><<<grid, cfg.block, 0, stream>>>(keys, bases, lengths, offsets, S, out, head); break;
        default: batch_kernel<true, 16><<<grid, cfg.block, 0, stream>>>(keys, bases, lengths, offsets, S, out, head); break;
    }
    return cudaGetLastError();
}

}  // namespace sq
