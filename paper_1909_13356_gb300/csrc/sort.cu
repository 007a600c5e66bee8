// sort.cu -- stable LSD radix sort of (key, value) pairs and stable stream
// compaction.  Used to order sources and targets along a Morton curve (so
// tiles and target blocks are spatially compact) and to drop converged chart
// nodes from the Newton active set (Sec. 5: converged targets leave the
// target list of later evaluations).
#include "lsm_internal.cuh"

namespace lsm {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortChunk = kSortThreads * kSortItems;  // elements per block
constexpr int kScanThreads = 1024;

__global__ void k_digit_hist(const uint32_t* __restrict__ keys, int n, int shift, int nb,
                             uint32_t* __restrict__ cnt)
{
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int base = blockIdx.x * kSortChunk;
    for (int r = 0; r < kSortItems; r++) {
        int i = base + r * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    cnt[threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of a[0..len) in place with one block; also writes the total.
__global__ void k_scan_exclusive(uint32_t* a, int64_t len, uint32_t* total)
{
    __shared__ uint32_t wsum[kScanThreads / 32];
    const int64_t per = (len + kScanThreads - 1) / kScanThreads;
    const int64_t lo = threadIdx.x * per;
    const int64_t hi = lo + per < len ? lo + per : len;
    uint32_t s = 0;
    for (int64_t i = lo; i < hi; i++) s += a[i];
    // block-wide exclusive scan of s
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t v = s;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) wsum[w] = v;
    __syncthreads();
    if (w == 0) {
        uint32_t x = wsum[lane];
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += t;
        }
        wsum[lane] = x;  // inclusive
    }
    __syncthreads();
    uint32_t run = v - s + (w > 0 ? wsum[w - 1] : 0u);
    for (int64_t i = lo; i < hi; i++) {
        uint32_t x = a[i];
        a[i] = run;
        run += x;
    }
    if (total != nullptr && threadIdx.x == kScanThreads - 1) *total = run;
}

__global__ void k_digit_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, int n,
                                int shift, int nb, const uint32_t* __restrict__ cnt)
{
    constexpr int W = kSortThreads / 32;
    __shared__ uint32_t running[256];
    __shared__ uint32_t wc[W][256];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    running[tid] = cnt[tid * nb + blockIdx.x];
    for (int k = 0; k < W; k++) wc[k][tid] = 0;
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    const int base = blockIdx.x * kSortChunk;
    for (int r = 0; r < kSortItems; r++) {
        const int i = base + r * kSortThreads + tid;
        const bool ok = i < n;
        uint32_t key = ok ? kin[i] : 0u;
        uint32_t val = ok ? vin[i] : 0u;
        uint32_t d = ok ? ((key >> shift) & 255u) : 256u;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int rank = __popc(peers & lt);
        if (ok && rank == 0) wc[w][d] = __popc(peers);
        __syncthreads();
        if (ok) {
            uint32_t off = running[d] + rank;
            for (int k = 0; k < w; k++) off += wc[k][d];
            kout[off] = key;
            vout[off] = val;
        }
        __syncthreads();
        uint32_t add = 0;
        for (int k = 0; k < W; k++) {
            add += wc[k][tid];
            wc[k][tid] = 0;
        }
        running[tid] += add;
        __syncthreads();
    }
}

constexpr int kCompThreads = 256;
constexpr int kCompItems = 4;
constexpr int kCompChunk = kCompThreads * kCompItems;

__global__ void k_flag_count(const int32_t* __restrict__ flags, int want, int n, uint32_t* bc)
{
    __shared__ uint32_t ws[kCompThreads / 32];
    const int base = blockIdx.x * kCompChunk + threadIdx.x * kCompItems;
    uint32_t c = 0;
    for (int k = 0; k < kCompItems; k++) {
        int i = base + k;
        if (i < n && flags[i] == want) c++;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int k = 0; k < kCompThreads / 32; k++) t += ws[k];
        bc[blockIdx.x] = t;
    }
}

__global__ void k_flag_scatter(const int32_t* __restrict__ flags, int want,
                               const int32_t* __restrict__ in, int n,
                               const uint32_t* __restrict__ bc, int32_t* __restrict__ out)
{
    __shared__ uint32_t ws[kCompThreads / 32];
    const int base = blockIdx.x * kCompChunk + threadIdx.x * kCompItems;
    uint32_t c = 0;
    for (int k = 0; k < kCompItems; k++) {
        int i = base + k;
        if (i < n && flags[i] == want) c++;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t v = c;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) ws[w] = v;
    __syncthreads();
    uint32_t off = bc[blockIdx.x] + v - c;
    for (int k = 0; k < w; k++) off += ws[k];
    for (int k = 0; k < kCompItems; k++) {
        int i = base + k;
        if (i < n && flags[i] == want) out[off++] = in ? in[i] : i;
    }
}

// Same as k_flag_count / k_flag_scatter with the length read on the device.
__global__ void k_flag_count_dev(const int32_t* __restrict__ flags, int want, const int* __restrict__ n_dev,
                                 uint32_t* bc)
{
    __shared__ uint32_t ws[kCompThreads / 32];
    const int n = *n_dev;
    const int base = blockIdx.x * kCompChunk + threadIdx.x * kCompItems;
    uint32_t c = 0;
    for (int k = 0; k < kCompItems; k++) {
        int i = base + k;
        if (i < n && flags[i] == want) c++;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int k = 0; k < kCompThreads / 32; k++) t += ws[k];
        bc[blockIdx.x] = t;
    }
}

__global__ void k_flag_scatter_dev(const int32_t* __restrict__ flags, int want, const int32_t* __restrict__ in,
                                   const int* __restrict__ n_dev, const uint32_t* __restrict__ bc,
                                   int32_t* __restrict__ out)
{
    __shared__ uint32_t ws[kCompThreads / 32];
    const int n = *n_dev;
    const int base = blockIdx.x * kCompChunk + threadIdx.x * kCompItems;
    uint32_t c = 0;
    for (int k = 0; k < kCompItems; k++) {
        int i = base + k;
        if (i < n && flags[i] == want) c++;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t v = c;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) ws[w] = v;
    __syncthreads();
    uint32_t off = bc[blockIdx.x] + v - c;
    for (int k = 0; k < w; k++) off += ws[k];
    for (int k = 0; k < kCompItems; k++) {
        int i = base + k;
        if (i < n && flags[i] == want) out[off++] = in ? in[i] : i;
    }
}

}  // namespace

// Sorts (keys, vals) by the low key_bits bits of keys, stably, in place.
int radix_sort_pairs(Ctx* ctx, uint32_t* keys, uint32_t* vals, int n, int key_bits,
                     cudaStream_t st)
{
    if (n <= 1) return LSM_OK;
    Scratch s(st);
    const int nb = (n + kSortChunk - 1) / kSortChunk;
    uint32_t *k2, *v2, *cnt;
    LSM_CUDA_TRY(ctx, s.get(&k2, n));
    LSM_CUDA_TRY(ctx, s.get(&v2, n));
    LSM_CUDA_TRY(ctx, s.get(&cnt, (size_t)256 * nb));
    uint32_t *ka = keys, *va = vals, *kb = k2, *vb = v2;
    const int passes = (key_bits + 7) / 8;
    for (int p = 0; p < passes; p++) {
        const int shift = 8 * p;
        k_digit_hist<<<nb, kSortThreads, 0, st>>>(ka, n, shift, nb, cnt);
        LSM_LAUNCHED(ctx);
        k_scan_exclusive<<<1, kScanThreads, 0, st>>>(cnt, (int64_t)256 * nb, nullptr);
        LSM_LAUNCHED(ctx);
        k_digit_scatter<<<nb, kSortThreads, 0, st>>>(ka, va, kb, vb, n, shift, nb, cnt);
        LSM_LAUNCHED(ctx);
        uint32_t* t = ka; ka = kb; kb = t;
        t = va; va = vb; vb = t;
    }
    if (ka != keys) {
        LSM_CUDA_TRY(ctx, cudaMemcpyAsync(keys, ka, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st));
        LSM_CUDA_TRY(ctx, cudaMemcpyAsync(vals, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st));
    }
    return LSM_OK;
}

// out = [in[i] (or i when in == NULL) for i with flags[i] == want], in order;
// *d_count (device) = its length.
int compact_flags(Ctx* ctx, const int32_t* flags, int want, const int32_t* in, int n,
                  int32_t* out, int32_t* d_count, cudaStream_t st)
{
    if (n <= 0) {
        LSM_CUDA_TRY(ctx, cudaMemsetAsync(d_count, 0, sizeof(int32_t), st));
        return LSM_OK;
    }
    Scratch s(st);
    const int nb = (n + kCompChunk - 1) / kCompChunk;
    uint32_t* bc;
    LSM_CUDA_TRY(ctx, s.get(&bc, nb));
    k_flag_count<<<nb, kCompThreads, 0, st>>>(flags, want, n, bc);
    LSM_LAUNCHED(ctx);
    k_scan_exclusive<<<1, kScanThreads, 0, st>>>(bc, nb, reinterpret_cast<uint32_t*>(d_count));
    LSM_LAUNCHED(ctx);
    k_flag_scatter<<<nb, kCompThreads, 0, st>>>(flags, want, in, n, bc, out);
    LSM_LAUNCHED(ctx);
    return LSM_OK;
}

// Exclusive scan of a[0..len) in place; *total (device, may be NULL) = sum.
int scan_exclusive(Ctx* ctx, uint32_t* a, int64_t len, uint32_t* total, cudaStream_t st)
{
    k_scan_exclusive<<<1, kScanThreads, 0, st>>>(a, len, total);
    LSM_LAUNCHED(ctx);
    return LSM_OK;
}

// compact_flags with the input length read on the device (*n_dev <= n_max);
// `bc` is caller scratch of compact_blocks(n_max) words.  Launch shapes
// depend on n_max only, so the sequence can be captured in a CUDA graph.
int compact_blocks(int n_max) { return (n_max + kCompChunk - 1) / kCompChunk; }
int compact_flags_dev(Ctx* ctx, const int32_t* flags, int want, const int32_t* in, const int* n_dev, int n_max,
                      int32_t* out, int32_t* d_count, uint32_t* bc, cudaStream_t st)
{
    const int nb = compact_blocks(n_max);
    if (nb <= 0) return LSM_OK;
    k_flag_count_dev<<<nb, kCompThreads, 0, st>>>(flags, want, n_dev, bc);
    LSM_LAUNCHED(ctx);
    k_scan_exclusive<<<1, kScanThreads, 0, st>>>(bc, nb, reinterpret_cast<uint32_t*>(d_count));
    LSM_LAUNCHED(ctx);
    k_flag_scatter_dev<<<nb, kCompThreads, 0, st>>>(flags, want, in, n_dev, bc, out);
    LSM_LAUNCHED(ctx);
    return LSM_OK;
}

}  // namespace lsm
