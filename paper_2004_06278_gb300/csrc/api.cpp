// C ABI of the Squares library (declared in include/squares.h): argument
// checks, error reporting, launch-configuration table, autotuner, graph
// helper. Every device computation happens in the kernel translation units.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <vector>

#include "internal.h"
#include "squares.h"

#ifndef SQ_BUILD_ID
#define SQ_BUILD_ID "unknown"  // build.py passes the hash of the kernel sources' code
#endif

namespace {

thread_local std::string g_error;
thread_local std::string g_fail_next;  // armed by sq_debug_fail_next

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *where) {
    return fail(SQ_ECUDA, "%s: %s (%s)", where, cudaGetErrorString(e), cudaGetErrorName(e));
}

int ok() {
    g_error.clear();
    return SQ_OK;
}

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// True once if sq_debug_fail_next armed a failure for this entry point.
bool injected(const char *name) {
    if (g_fail_next.empty() || g_fail_next != name) return false;
    g_fail_next.clear();
    return true;
}

int injected_fail(const char *name) {
    return fail(SQ_ECUDA, "%s: injected launch failure (sq_debug_fail_next)", name);
}

constexpr size_t kMaxElems = size_t(1) << 62;
constexpr size_t kMaxStreams = size_t(1) << 31;
constexpr int kBuckets = 64;

int bucket_of(size_t n) {
    int b = 0;
    while (n > 1 && b < kBuckets - 1) {
        n >>= 1;
        ++b;
    }
    return b;
}

bool valid_kernel(int kid) { return kid >= 0 && kid < SQ_NUM_KERNELS; }

bool is_plain(int kid) {
    return kid == SQ_KERNEL_U32 || kid == SQ_KERNEL_U64 || kid == SQ_KERNEL_UNIFORM_F32 ||
           kid == SQ_KERNEL_UNIFORM_BF16 || kid == SQ_KERNEL_NORMAL_F32 ||
           kid == SQ_KERNEL_UNIFORM2_F32 || kid == SQ_KERNEL_UNIFORM_F64;
}

int num_variants(int kid) {
    if (is_plain(kid)) return sq::plain_num_variants();
    if (kid == SQ_KERNEL_BATCH) return sq::batch_num_variants();
    if (kid == SQ_KERNEL_FUSED) return sq::fused_num_variants();
    return 0;
}

int max_ctas(int kid, int variant, int block) {
    if (is_plain(kid)) return sq::plain_max_ctas_per_sm(kid, variant, block);
    if (kid == SQ_KERNEL_BATCH) return sq::batch_max_ctas_per_sm(variant, block);
    return sq::fused_max_ctas_per_sm(variant, block);
}

bool valid_cfg(int kid, const sq::Cfg &c) {
    return c.variant >= 0 && c.variant < num_variants(kid) &&
           (c.block == 128 || c.block == 256 || c.block == 512 || (kid == SQ_KERNEL_BATCH && c.block == 64)) &&
           c.ctas_per_sm >= 0 &&
           c.ctas_per_sm <= 32;
}

struct ConfigTable {
    std::mutex m;
    sq::Cfg cfg[SQ_NUM_KERNELS][kBuckets];
    ConfigTable() {
        for (auto &row : cfg)
            for (auto &c : row) c = sq::Cfg{0, 256, 0};
    }
    sq::Cfg get(int kid, size_t n) {
        std::lock_guard<std::mutex> g(m);
        return cfg[kid][bucket_of(n)];
    }
    void set(int kid, size_t n, const sq::Cfg &c) {
        std::lock_guard<std::mutex> g(m);
        if (n == 0) {
            for (auto &e : cfg[kid]) e = c;
        } else {
            cfg[kid][bucket_of(n)] = c;
        }
    }
};

std::string device_name() {
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess)
        return prop.name;
    cudaGetLastError();
    return "unknown";
}

ConfigTable &raw_table() {
    static ConfigTable t;
    return t;
}

// Reads a table written by sq_autotune_save into the configuration table.
// Entries tuned for another device name are ignored (SQ_OK). A table saved
// by a library built from other kernel code (another sq_build_id, or a
// version-1 file, which records none) is ignored too, with SQ_EINVAL and a
// message naming both identifiers: its timings belong to other kernels.
int load_table_file(const char *path, std::string *err) {
    FILE *f = fopen(path, "r");
    if (!f) {
        *err = std::string("cannot open ") + path;
        return SQ_EINVAL;
    }
    char line[512];
    int version = 0;
    if (!fgets(line, sizeof line, f) || sscanf(line, "squares-autotune %d", &version) != 1 ||
        (version != 1 && version != 2)) {
        fclose(f);
        *err = std::string(path) + " is not an autotune file";
        return SQ_EINVAL;
    }
    std::string file_dev;
    if (fgets(line, sizeof line, f) && strncmp(line, "device ", 7) == 0) {
        file_dev = line + 7;
        while (!file_dev.empty() && (file_dev.back() == '\n' || file_dev.back() == '\r')) file_dev.pop_back();
    }
    std::string file_code = "none";
    if (version == 2 && fgets(line, sizeof line, f) && strncmp(line, "code ", 5) == 0) {
        file_code = line + 5;
        while (!file_code.empty() && (file_code.back() == '\n' || file_code.back() == '\r')) file_code.pop_back();
    }
    if (file_dev != device_name()) {
        fclose(f);
        return SQ_OK;  // tuned for another device: keep the defaults
    }
    if (file_code != SQ_BUILD_ID) {
        fclose(f);
        *err = std::string(path) + " was tuned on kernel code " + file_code + ", this library's is " +
               SQ_BUILD_ID + ": table ignored";
        return SQ_EINVAL;
    }
    int k, b, v, bl, c;
    std::vector<std::pair<std::pair<int, int>, sq::Cfg>> rows;
    while (fgets(line, sizeof line, f)) {
        if (sscanf(line, "%d %d %d %d %d", &k, &b, &v, &bl, &c) != 5) continue;
        const sq::Cfg cfg{v, bl, c};
        if (!valid_kernel(k) || b < 0 || b >= kBuckets || !valid_cfg(k, cfg)) {
            fclose(f);
            *err = std::string("bad entry '") + line + "'";
            return SQ_EINVAL;
        }
        rows.push_back({{k, b}, cfg});
    }
    fclose(f);
    ConfigTable &t = raw_table();
    std::lock_guard<std::mutex> g(t.m);
    for (auto &r : rows) t.cfg[r.first.first][r.first.second] = r.second;
    return SQ_OK;
}

// The configuration table; on first use it is filled from the file named by
// the environment variable SQ_TUNE_FILE, if that is set, readable and was
// saved by a library with this build identifier (otherwise the defaults
// stay).
ConfigTable &table() {
    static std::once_flag once;
    std::call_once(once, [] {
        const char *path = getenv("SQ_TUNE_FILE");
        std::string err;
        if (path && *path) load_table_file(path, &err);
    });
    return raw_table();
}

int plain_entry(int kid, uint64_t key, uint64_t base, size_t n, void *out, size_t elem,
                sq_stream_t stream, const char *name) {
    if (n == 0) return ok();
    if (out == nullptr) return fail(SQ_EINVAL, "%s: out is NULL with n = %zu", name, n);
    if (!aligned(out, elem)) return fail(SQ_EINVAL, "%s: out is not %zu-byte aligned", name, elem);
    if (n > kMaxElems) return fail(SQ_ERANGE, "%s: n = %zu exceeds 2^62", name, n);
    if (injected(name)) return injected_fail(name);
    const sq::Cfg cfg = table().get(kid, n);
    const cudaError_t e = sq::launch_plain(kid, cfg, key, base, n, out, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, name);
    return ok();
}

int batch_checks(const uint64_t *keys, const uint64_t *bases, const int64_t *lengths,
                 const int64_t *offsets, size_t nstreams, const uint32_t *out, const char *name) {
    if (nstreams > kMaxStreams) return fail(SQ_ERANGE, "%s: nstreams = %zu exceeds 2^31", name, nstreams);
    if (!keys || !bases || !lengths || !offsets || !out)
        return fail(SQ_EINVAL, "%s: NULL array with nstreams = %zu", name, nstreams);
    if (!aligned(keys, 8) || !aligned(bases, 8) || !aligned(lengths, 8) || !aligned(offsets, 8) ||
        !aligned(out, 4))
        return fail(SQ_EINVAL, "%s: misaligned array", name);
    return SQ_OK;
}

}  // namespace

namespace sq {

bool in_device_memory(const void *p) {
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice;
}

int current_sm_count() {
    static std::array<std::atomic<int>, 64> cache{};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) dev = 0;
    const int slot = dev & 63;
    int v = cache[slot].load(std::memory_order_relaxed);
    if (v > 0) return v;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        sms = 1;
    cache[slot].store(sms, std::memory_order_relaxed);
    return sms;
}

int occupancy(const void *kernel, int block, size_t smem) {
    static std::mutex m;
    static std::map<std::tuple<int, const void *, int, size_t>, int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    const auto k = std::make_tuple(dev, kernel, block, smem);
    {
        std::lock_guard<std::mutex> g(m);
        const auto it = cache.find(k);
        if (it != cache.end()) return it->second;
    }
    int blocks = 0;
    if (!kernel || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernel, block, smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;  // not cached: the query may succeed later
    }
    if (blocks < 1) blocks = 1;
    std::lock_guard<std::mutex> g(m);
    cache[k] = blocks;
    return blocks;
}

}  // namespace sq

// ---------------------------------------------------------------------------
// C ABI

extern "C" {

const char *sq_last_error(void) { return g_error.c_str(); }

int sq_abi_version(void) { return 100; }

const char *sq_build_id(void) { return SQ_BUILD_ID; }

int sq_debug_fail_next(const char *entry_point) {
    g_fail_next = entry_point ? entry_point : "";
    return ok();
}

int sq_make_keys(uint64_t seed, size_t n, uint64_t *keys) {
    if (n > kMaxStreams) return fail(SQ_ERANGE, "sq_make_keys: n = %zu exceeds 2^31", n);
    if (n == 0) return ok();
    if (keys == nullptr) return fail(SQ_EINVAL, "sq_make_keys: keys is NULL with n = %zu", n);
    try {
        sq::make_keys(seed, n, keys);
    } catch (const std::bad_alloc &) {
        return fail(SQ_ERANGE, "sq_make_keys: cannot allocate the duplicate table for n = %zu", n);
    }
    return ok();
}

int sq_u32(uint64_t key, uint64_t ctr_base, size_t n, uint32_t *out, sq_stream_t stream) {
    return plain_entry(SQ_KERNEL_U32, key, ctr_base, n, out, 4, stream, "sq_u32");
}

int sq_u64(uint64_t key, uint64_t ctr_base, size_t n, uint64_t *out, sq_stream_t stream) {
    return plain_entry(SQ_KERNEL_U64, key, ctr_base, n, out, 8, stream, "sq_u64");
}

int sq_uniform_f32(uint64_t key, uint64_t ctr_base, size_t n, float *out, sq_stream_t stream) {
    return plain_entry(SQ_KERNEL_UNIFORM_F32, key, ctr_base, n, out, 4, stream, "sq_uniform_f32");
}

int sq_uniform_bf16(uint64_t key, uint64_t ctr_base, size_t n, uint16_t *out, sq_stream_t stream) {
    return plain_entry(SQ_KERNEL_UNIFORM_BF16, key, ctr_base, n, out, 2, stream, "sq_uniform_bf16");
}

int sq_normal_f32(uint64_t key, uint64_t ctr_base, size_t n, float *out, sq_stream_t stream) {
    return plain_entry(SQ_KERNEL_NORMAL_F32, key, ctr_base, n, out, 4, stream, "sq_normal_f32");
}

int sq_uniform2_f32(uint64_t key, uint64_t ctr_base, size_t n, float *out, sq_stream_t stream) {
    return plain_entry(SQ_KERNEL_UNIFORM2_F32, key, ctr_base, n, out, 4, stream, "sq_uniform2_f32");
}

int sq_uniform_f64(uint64_t key, uint64_t ctr_base, size_t n, double *out, sq_stream_t stream) {
    return plain_entry(SQ_KERNEL_UNIFORM_F64, key, ctr_base, n, out, 8, stream, "sq_uniform_f64");
}

int sq_fill_u32(uint32_t value, size_t n, uint32_t *out, const sq_launch_config *cfg,
                uint32_t pause_ns, sq_stream_t stream) {
    if (n == 0) return ok();
    if (out == nullptr) return fail(SQ_EINVAL, "sq_fill_u32: out is NULL with n = %zu", n);
    if (!aligned(out, 4)) return fail(SQ_EINVAL, "sq_fill_u32: out is not 4-byte aligned");
    if (n > kMaxElems) return fail(SQ_ERANGE, "sq_fill_u32: n = %zu exceeds 2^62", n);
    sq::Cfg c = table().get(SQ_KERNEL_U32, n);
    if (cfg) {
        c = sq::Cfg{cfg->variant, cfg->block, cfg->ctas_per_sm};
        if (!valid_cfg(SQ_KERNEL_U32, c))
            return fail(SQ_EINVAL, "sq_fill_u32: invalid configuration (variant %d, block %d, ctas %d)",
                        c.variant, c.block, c.ctas_per_sm);
    }
    if (injected("sq_fill_u32")) return injected_fail("sq_fill_u32");
    const cudaError_t e = sq::launch_plain(sq::kFillKernelId, c, value, pause_ns, n, out,
                                           static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "sq_fill_u32");
    return ok();
}

static int strided_entry(bool wide, uint64_t key, uint64_t base, uint64_t stride, size_t n, void *out,
                         sq_stream_t stream, const char *name) {
    const size_t elem = wide ? 8 : 4;
    if (n == 0) return ok();
    if (out == nullptr) return fail(SQ_EINVAL, "%s: out is NULL with n = %zu", name, n);
    if (!aligned(out, elem)) return fail(SQ_EINVAL, "%s: out is not %zu-byte aligned", name, elem);
    if (n > kMaxElems) return fail(SQ_ERANGE, "%s: n = %zu exceeds 2^62", name, n);
    if (injected(name)) return injected_fail(name);
    const cudaError_t e = sq::launch_strided(wide, key, base, stride, n, out, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, name);
    return ok();
}

int sq_u32_strided(uint64_t key, uint64_t ctr_base, uint64_t stride, size_t n, uint32_t *out,
                   sq_stream_t stream) {
    return strided_entry(false, key, ctr_base, stride, n, out, stream, "sq_u32_strided");
}

int sq_u64_strided(uint64_t key, uint64_t ctr_base, uint64_t stride, size_t n, uint64_t *out,
                   sq_stream_t stream) {
    return strided_entry(true, key, ctr_base, stride, n, out, stream, "sq_u64_strided");
}

static int keys_entry(bool wide, const uint64_t *keys, size_t n, uint64_t ctr, void *out,
                      sq_stream_t stream, const char *name) {
    const size_t elem = wide ? 8 : 4;
    if (n == 0) return ok();
    if (!keys || !out) return fail(SQ_EINVAL, "%s: NULL array with nkeys = %zu", name, n);
    if (!aligned(keys, 8) || !aligned(out, elem)) return fail(SQ_EINVAL, "%s: misaligned array", name);
    if (n > kMaxElems) return fail(SQ_ERANGE, "%s: nkeys = %zu exceeds 2^62", name, n);
    if (injected(name)) return injected_fail(name);
    const cudaError_t e = sq::launch_keys(wide, keys, n, ctr, out, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, name);
    return ok();
}

int sq_keys_u32(const uint64_t *keys, size_t nkeys, uint64_t ctr, uint32_t *out, sq_stream_t stream) {
    return keys_entry(false, keys, nkeys, ctr, out, stream, "sq_keys_u32");
}

int sq_keys_u64(const uint64_t *keys, size_t nkeys, uint64_t ctr, uint64_t *out, sq_stream_t stream) {
    return keys_entry(true, keys, nkeys, ctr, out, stream, "sq_keys_u64");
}

int sq_batch(const uint64_t *keys, const uint64_t *ctr_bases, const int64_t *lengths,
             const int64_t *offsets, size_t nstreams, uint32_t *out, sq_stream_t stream) {
    if (nstreams == 0) return ok();
    const int rc = batch_checks(keys, ctr_bases, lengths, offsets, nstreams, out, "sq_batch");
    if (rc != SQ_OK) return rc;
    if (injected("sq_batch")) return injected_fail("sq_batch");
    const sq::Cfg cfg = table().get(SQ_KERNEL_BATCH, nstreams);
    const cudaError_t e = sq::launch_batch(cfg, keys, ctr_bases, lengths, offsets, nstreams, out,
                                           static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "sq_batch");
    return ok();
}

int sq_batch_validate(const int64_t *lengths, const int64_t *offsets, size_t nstreams,
                      sq_stream_t stream) {
    if (nstreams == 0) return ok();
    if (nstreams > kMaxStreams) return fail(SQ_ERANGE, "sq_batch_validate: nstreams exceeds 2^31");
    if (!lengths || !offsets) return fail(SQ_EINVAL, "sq_batch_validate: NULL array");
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "sq_batch_validate");
    std::vector<int64_t> len(nstreams), off(nstreams);
    e = cudaMemcpy(len.data(), lengths, nstreams * sizeof(int64_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = cudaMemcpy(off.data(), offsets, nstreams * sizeof(int64_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "sq_batch_validate");
    if (off[0] < 0) return fail(SQ_EINVAL, "sq_batch_validate: offsets[0] = %lld < 0", (long long)off[0]);
    for (size_t s = 0; s < nstreams; ++s) {
        if (len[s] < 0) return fail(SQ_EINVAL, "sq_batch_validate: lengths[%zu] < 0", s);
        if (off[s] > INT64_MAX - len[s])
            return fail(SQ_EINVAL, "sq_batch_validate: offsets[%zu] + lengths[%zu] overflows", s, s);
        if (s + 1 < nstreams && off[s] + len[s] > off[s + 1])
            return fail(SQ_EINVAL, "sq_batch_validate: stream %zu overlaps stream %zu", s, s + 1);
    }
    return ok();
}

int sq_fused_stats(const uint64_t *keys, const uint64_t *ctr_bases, size_t nstreams,
                   uint64_t ctrs_per_stream, uint32_t *xor_out, uint64_t *sum_top,
                   uint64_t *hist256, sq_stream_t stream) {
    if (nstreams > kMaxStreams) return fail(SQ_ERANGE, "sq_fused_stats: nstreams exceeds 2^31");
    if (ctrs_per_stream > (uint64_t(1) << 40))
        return fail(SQ_ERANGE, "sq_fused_stats: ctrs_per_stream exceeds 2^40");
    if (!hist256) return fail(SQ_EINVAL, "sq_fused_stats: hist256 is NULL");
    if (nstreams > 0 && (!keys || !ctr_bases || !xor_out || !sum_top))
        return fail(SQ_EINVAL, "sq_fused_stats: NULL array with nstreams = %zu", nstreams);
    if (!aligned(hist256, 8) || (nstreams > 0 && (!aligned(keys, 8) || !aligned(ctr_bases, 8) ||
                                                  !aligned(xor_out, 4) || !aligned(sum_top, 8))))
        return fail(SQ_EINVAL, "sq_fused_stats: misaligned array");
    if (injected("sq_fused_stats")) return injected_fail("sq_fused_stats");
    const sq::Cfg cfg = table().get(SQ_KERNEL_FUSED, nstreams * ctrs_per_stream);
    const cudaError_t e = sq::launch_fused(cfg, keys, ctr_bases, nstreams, ctrs_per_stream, xor_out,
                                           sum_top, hist256, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "sq_fused_stats");
    return ok();
}

int sq_num_variants(int kernel_id) {
    if (!valid_kernel(kernel_id)) return fail(SQ_EINVAL, "sq_num_variants: bad kernel id %d", kernel_id);
    return num_variants(kernel_id);
}

const char *sq_variant_name(int kernel_id, int variant) {
    if (!valid_kernel(kernel_id)) return nullptr;
    if (is_plain(kernel_id)) return sq::plain_variant_name(variant);
    if (kernel_id == SQ_KERNEL_BATCH) return sq::batch_variant_name(variant);
    return sq::fused_variant_name(variant);
}

int sq_get_config(int kernel_id, size_t n, sq_launch_config *cfg) {
    if (!valid_kernel(kernel_id) || !cfg) return fail(SQ_EINVAL, "sq_get_config: bad arguments");
    const sq::Cfg c = table().get(kernel_id, n);
    cfg->variant = c.variant;
    cfg->block = c.block;
    cfg->ctas_per_sm = c.ctas_per_sm;
    cfg->reserved = 0;
    return ok();
}

int sq_set_config(int kernel_id, size_t n, const sq_launch_config *cfg) {
    if (!valid_kernel(kernel_id) || !cfg) return fail(SQ_EINVAL, "sq_set_config: bad arguments");
    const sq::Cfg c{cfg->variant, cfg->block, cfg->ctas_per_sm};
    if (!valid_cfg(kernel_id, c))
        return fail(SQ_EINVAL, "sq_set_config: invalid configuration (variant %d, block %d, ctas %d)",
                    c.variant, c.block, c.ctas_per_sm);
    table().set(kernel_id, n, c);
    return ok();
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Autotuner

namespace {

struct DevBuf {
    void *p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
};

// Average milliseconds of `reps` launches of `run` after two warm-up runs.
template <class F>
cudaError_t time_it(cudaStream_t st, int reps, F run, float *ms) {
    cudaEvent_t a, b;
    cudaError_t e = cudaEventCreate(&a);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&b);
    if (e != cudaSuccess) {
        cudaEventDestroy(a);
        return e;
    }
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = run();
    if (e == cudaSuccess) e = cudaEventRecord(a, st);
    for (int i = 0; i < reps && e == cudaSuccess; ++i) e = run();
    if (e == cudaSuccess) e = cudaEventRecord(b, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
    *ms = t / reps;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return e;
}

size_t elem_size(int kid) {
    switch (kid) {
        case SQ_KERNEL_U64: return 8;
        case SQ_KERNEL_UNIFORM_F64: return 8;
        case SQ_KERNEL_UNIFORM_BF16: return 2;
        default: return 4;
    }
}

}  // namespace

extern "C" {

int sq_autotune(int kernel_id, size_t n_hint) {
    if (!valid_kernel(kernel_id)) return fail(SQ_EINVAL, "sq_autotune: bad kernel id %d", kernel_id);
    if (n_hint == 0) return fail(SQ_EINVAL, "sq_autotune: n_hint is 0");
    cudaStream_t st;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "sq_autotune");
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamDestroy(s); }
    } guard{st};

    const size_t cap_bytes = size_t(1) << 31;
    DevBuf out, aux;
    std::vector<sq::Cfg> cands;
    const int blocks[3] = {128, 256, 512};
    const int ctas_opts[4] = {1, 2, 4, 0};
    // The batch kernel is tuned here on 64 long streams, where only its tile
    // variants (0-3) can win; sq_autotune_batch tunes on real batches.
    const int nv = (kernel_id == SQ_KERNEL_BATCH) ? 4 : num_variants(kernel_id);
    for (int v = 0; v < nv; ++v)
        for (int b : blocks) {
            const int mx = max_ctas(kernel_id, v, b);
            for (int c : ctas_opts)
                if (c <= mx) cands.push_back(sq::Cfg{v, b, c});
        }

    size_t n = n_hint;
    // Synthetic batch / fused inputs live in `aux`.
    uint64_t *keys = nullptr, *bases = nullptr, *sums = nullptr, *hist = nullptr;
    int64_t *lengths = nullptr, *offsets = nullptr;
    uint32_t *xors = nullptr;
    size_t S = 0;
    uint64_t cps = 0;
    if (is_plain(kernel_id) || kernel_id == SQ_KERNEL_BATCH) {
        const size_t es = (kernel_id == SQ_KERNEL_BATCH) ? 4 : elem_size(kernel_id);
        n = std::min(n_hint, cap_bytes / es);
        e = cudaMalloc(&out.p, n * es);
        if (e != cudaSuccess) return cuda_fail(e, "sq_autotune: cudaMalloc");
    }
    if (kernel_id == SQ_KERNEL_BATCH) {
        // 64 ragged streams covering [0, n): lengths vary by a factor ~3.
        S = 64;
        std::vector<uint64_t> hk(S), hb(S);
        std::vector<int64_t> hl(S), ho(S);
        sq::make_keys(1, S, hk.data());
        uint64_t acc = 0;
        for (size_t s = 0; s < S; ++s) hl[s] = int64_t(1 + (s * 2654435761u) % 3);
        for (size_t s = 0; s < S; ++s) acc += hl[s];
        int64_t off = 0;
        for (size_t s = 0; s < S; ++s) {
            ho[s] = off;
            hl[s] = (s + 1 == S) ? int64_t(n) - off : int64_t(double(hl[s]) / acc * n);
            off += hl[s];
            hb[s] = 0x9E3779B97F4A7C15ull * (s + 1);
        }
        e = cudaMalloc(&aux.p, S * 32);
        if (e != cudaSuccess) return cuda_fail(e, "sq_autotune: cudaMalloc");
        keys = static_cast<uint64_t *>(aux.p);
        bases = keys + S;
        lengths = reinterpret_cast<int64_t *>(bases + S);
        offsets = lengths + S;
        cudaMemcpy(keys, hk.data(), S * 8, cudaMemcpyHostToDevice);
        cudaMemcpy(bases, hb.data(), S * 8, cudaMemcpyHostToDevice);
        cudaMemcpy(lengths, hl.data(), S * 8, cudaMemcpyHostToDevice);
        e = cudaMemcpy(offsets, ho.data(), S * 8, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "sq_autotune: cudaMemcpy");
    }
    if (kernel_id == SQ_KERNEL_FUSED) {
        cps = std::min<uint64_t>(n_hint, uint64_t(1) << 18);
        S = std::max<size_t>(1, std::min<size_t>(n_hint / cps, size_t(1) << 20));
        e = cudaMalloc(&aux.p, S * (8 + 8 + 4 + 8) + 256 * 8 + 64);
        if (e != cudaSuccess) return cuda_fail(e, "sq_autotune: cudaMalloc");
        keys = static_cast<uint64_t *>(aux.p);
        bases = keys + S;
        sums = bases + S;
        hist = sums + S;
        xors = reinterpret_cast<uint32_t *>(hist + 256);
        std::vector<uint64_t> hk(S);
        sq::make_keys(13, S, hk.data());
        cudaMemcpy(keys, hk.data(), S * 8, cudaMemcpyHostToDevice);
        e = cudaMemset(bases, 0, S * 8);
        if (e != cudaSuccess) return cuda_fail(e, "sq_autotune: cudaMemset");
    }

    float best = 1e30f;
    sq::Cfg best_cfg = table().get(kernel_id, n_hint);
    for (const sq::Cfg &c : cands) {
        auto launch = [&]() -> cudaError_t {
            if (is_plain(kernel_id))
                return sq::launch_plain(kernel_id, c, 0x8B5CA2F1E3D6479Bull, 12345, n, out.p, st);
            if (kernel_id == SQ_KERNEL_BATCH)
                return sq::launch_batch(c, keys, bases, lengths, offsets, S, static_cast<uint32_t *>(out.p), st);
            return sq::launch_fused(c, keys, bases, S, cps, xors, sums, hist, st);
        };
        float ms = 0.f;
        e = time_it(st, 10, launch, &ms);
        if (e != cudaSuccess) return cuda_fail(e, "sq_autotune: candidate launch");
        if (ms < best) {
            best = ms;
            best_cfg = c;
        }
    }
    // The batch table is indexed by stream count; the synthetic 64-stream
    // pick (tile variants only) becomes the default for every count.
    table().set(kernel_id, kernel_id == SQ_KERNEL_BATCH ? 0 : n_hint, best_cfg);
    return ok();
}

int sq_autotune_batch(const uint64_t *keys, const uint64_t *ctr_bases, const int64_t *lengths,
                      const int64_t *offsets, size_t nstreams, uint32_t *out) {
    if (nstreams == 0) return ok();
    int rc = batch_checks(keys, ctr_bases, lengths, offsets, nstreams, out, "sq_autotune_batch");
    if (rc != SQ_OK) return rc;
    cudaError_t e = cudaDeviceSynchronize();  // inputs may come from any stream
    if (e != cudaSuccess) return cuda_fail(e, "sq_autotune_batch");
    cudaStream_t st;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "sq_autotune_batch");
    // Mean stream length from the batch extent (two values read back). The
    // streams-to-lanes and flattened-warp variants (4 and up) are candidates
    // only for streams of at most 8192 values on average: on longer ones a
    // lane group or a warp walks a whole stream alone and cannot win. Each
    // variant is first timed at block 256 with ctas_per_sm 0 (as many CTAs
    // as fit; one warp per 32 streams for the flattened-warp variants); if
    // that takes over 3x the best time so far, its other configurations are
    // not timed.
    int64_t last_off = 0, last_len = 0;
    e = cudaMemcpy(&last_off, offsets + nstreams - 1, sizeof(int64_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = cudaMemcpy(&last_len, lengths + nstreams - 1, sizeof(int64_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        cudaStreamDestroy(st);
        return cuda_fail(e, "sq_autotune_batch: reading the batch extent");
    }
    const double extent = static_cast<double>(last_off) + static_cast<double>(last_len);
    const bool short_streams = extent > 0 && extent / static_cast<double>(nstreams) <= 8192.0;
    float best = 1e30f;
    sq::Cfg best_cfg = table().get(SQ_KERNEL_BATCH, nstreams);
    const int blocks[4] = {64, 128, 256, 512};
    const int ctas_opts[4] = {1, 2, 4, 0};
    const int nv = short_streams ? sq::batch_num_variants() : 4;
    auto time_cfg = [&](const sq::Cfg &cfg, float *ms) {
        return time_it(st, 5, [&]() {
            return sq::launch_batch(cfg, keys, ctr_bases, lengths, offsets, nstreams, out, st);
        }, ms);
    };
    for (int v = 0; v < nv && e == cudaSuccess; ++v) {
        // probe: block 256, ctas_per_sm 0
        const sq::Cfg probe{v, 256, 0};
        float ms = 0.f;
        e = time_cfg(probe, &ms);
        if (e != cudaSuccess) break;
        if (ms < best) {
            best = ms;
            best_cfg = probe;
        }
        if (ms > 3.f * best) continue;
        for (int b : blocks) {
            const int mx = sq::batch_max_ctas_per_sm(v, b);
            for (int c : ctas_opts) {
                if (c > mx || (b == 256 && c == 0)) continue;
                const sq::Cfg cfg{v, b, c};
                e = time_cfg(cfg, &ms);
                if (e != cudaSuccess) break;
                if (ms < best) {
                    best = ms;
                    best_cfg = cfg;
                }
            }
            if (e != cudaSuccess) break;
        }
    }
    cudaStreamDestroy(st);
    if (e != cudaSuccess) return cuda_fail(e, "sq_autotune_batch: candidate launch");
    table().set(SQ_KERNEL_BATCH, nstreams, best_cfg);
    return ok();
}

int sq_autotune_save(const char *path) {
    if (!path) return fail(SQ_EINVAL, "sq_autotune_save: path is NULL");
    const std::string name = device_name();
    FILE *f = fopen(path, "w");
    if (!f) return fail(SQ_EINVAL, "sq_autotune_save: cannot open %s", path);
    fprintf(f, "squares-autotune 2\ndevice %s\ncode %s\n", name.c_str(), SQ_BUILD_ID);
    ConfigTable &t = table();
    {
        std::lock_guard<std::mutex> g(t.m);
        for (int k = 0; k < SQ_NUM_KERNELS; ++k)
            for (int b = 0; b < kBuckets; ++b) {
                const sq::Cfg &c = t.cfg[k][b];
                fprintf(f, "%d %d %d %d %d\n", k, b, c.variant, c.block, c.ctas_per_sm);
            }
    }
    fclose(f);
    return ok();
}

int sq_autotune_load(const char *path) {
    if (!path) return fail(SQ_EINVAL, "sq_autotune_load: path is NULL");
    std::string err;
    const int rc = load_table_file(path, &err);
    if (rc != SQ_OK) return fail(rc, "sq_autotune_load: %s", err.c_str());
    return ok();
}

// ---------------------------------------------------------------------------
// Graph helper

struct sq_graph_s {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

int sq_batch_graph_create(const uint64_t *keys, const uint64_t *ctr_bases, const int64_t *lengths,
                          const int64_t *offsets, size_t nstreams, uint32_t *out, sq_graph_t *graph) {
    if (!graph) return fail(SQ_EINVAL, "sq_batch_graph_create: graph is NULL");
    *graph = nullptr;
    if (nstreams > 0) {
        const int rc = batch_checks(keys, ctr_bases, lengths, offsets, nstreams, out, "sq_batch_graph_create");
        if (rc != SQ_OK) return rc;
    }
    cudaStream_t st;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "sq_batch_graph_create");
    sq_graph_s *g = new sq_graph_s;
    e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        const cudaError_t le = sq::launch_batch(table().get(SQ_KERNEL_BATCH, nstreams), keys, ctr_bases,
                                                lengths, offsets, nstreams, out, st);
        e = cudaStreamEndCapture(st, &g->graph);
        if (le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    cudaStreamDestroy(st);
    if (e != cudaSuccess) {
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
        return cuda_fail(e, "sq_batch_graph_create");
    }
    *graph = g;
    return ok();
}

int sq_graph_launch(sq_graph_t graph, sq_stream_t stream) {
    if (!graph) return fail(SQ_EINVAL, "sq_graph_launch: graph is NULL");
    if (injected("sq_graph_launch")) return injected_fail("sq_graph_launch");
    const cudaError_t e = cudaGraphLaunch(graph->exec, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "sq_graph_launch");
    return ok();
}

int sq_graph_destroy(sq_graph_t graph) {
    if (!graph) return ok();
    if (graph->exec) cudaGraphExecDestroy(graph->exec);
    if (graph->graph) cudaGraphDestroy(graph->graph);
    delete graph;
    return ok();
}

}  // extern "C"
