// Device-wide building blocks of the tree construction: an exclusive prefix scan of int32
// counts into int64 offsets, and a stable least-significant-digit radix sort of
// (uint32 key, int32 value) pairs.  Both are plain HBM-bound passes; the sort orders the
// particles by the first slot of their leaf, which (because the scan over the input runs in
// original index order and every pass is stable) keeps particles of one leaf in their
// original relative order, as the refinement of Sec. 3 does.
#include "sts_internal.cuh"

namespace sts {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kScanThreads = 512;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

// Exclusive scan across a block of NT threads; returns the calling thread's exclusive
// prefix and writes the block total to *total.  sh holds NT / 32 values.
template <int NT>
__device__ int64_t block_excl_scan(int64_t v, int64_t* sh, int64_t* total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        int64_t t = lane < NT / 32 ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(kFull, t, o);
            if (lane >= o) t += y;
        }
        if (lane < NT / 32) sh[lane] = t;
    }
    __syncthreads();
    const int64_t woff = w ? sh[w - 1] : 0;
    *total = sh[NT / 32 - 1];
    __syncthreads();
    return woff + x - v;
}

__global__ void k_scan_reduce(const int32_t* __restrict__ in, int64_t n, const int64_t* __restrict__ nd,
                              int64_t* __restrict__ part)
{
    __shared__ int64_t sh[kScanThreads / 32];
    if (nd) n = min(*nd, n);
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++)
        if (base + i < n) s += in[base + i];
    int64_t tot;
    block_excl_scan<kScanThreads>(s, sh, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// Single block: exclusive scan of part[0, nb) in place; part[nb] = total.
__global__ void k_scan_top(int64_t* part, int64_t nb)
{
    __shared__ int64_t sh[1024 / 32];
    int64_t carry = 0;
    for (int64_t s0 = 0; s0 < nb; s0 += 1024) {
        const int64_t i = s0 + threadIdx.x;
        const int64_t v = i < nb ? part[i] : 0;
        int64_t tot;
        const int64_t ex = block_excl_scan<1024>(v, sh, &tot);
        if (i < nb) part[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) part[nb] = carry;
}

__global__ void k_scan_down(const int32_t* __restrict__ in, int64_t n, const int64_t* __restrict__ nd,
                            const int64_t* __restrict__ part, int64_t nb, int64_t* __restrict__ out)
{
    if (nd) n = min(*nd, n);
    __shared__ int64_t sh[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        v[i] = base + i < n ? in[base + i] : 0;
        s += v[i];
    }
    int64_t tot;
    int64_t run = part[blockIdx.x] + block_excl_scan<kScanThreads>(s, sh, &tot);
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = part[nb];
}

// ---------------------------------------------------------------------------- radix sort
constexpr int kRadixWarps = 8;
constexpr int kRadixRounds = 8;
constexpr int kRadixTile = kRadixWarps * kRadixRounds * 32;  // 2048 items per block

__global__ void k_radix_hist(const uint32_t* __restrict__ key, int64_t n, const int64_t* __restrict__ n_dev,
                             int shift, int64_t nb, int32_t* __restrict__ hist)
{
    if (n_dev) n = min(*n_dev, n);
    __shared__ int32_t h[256];
    for (int d = threadIdx.x; d < 256; d += blockDim.x) h[d] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
    for (int i = threadIdx.x; i < kRadixTile; i += blockDim.x) {
        const int64_t k = base + i;
        if (k < n) atomicAdd(&h[(key[k] >> shift) & 255u], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[(int64_t)d * nb + blockIdx.x] = h[d];
}

// Scatter with ranks that are stable inside the block: warp w owns items
// [w * 256, (w + 1) * 256) of the tile and walks them in rounds of 32 consecutive items.
__global__ void __launch_bounds__(kRadixWarps * 32)
k_radix_scatter(const uint32_t* __restrict__ key, const int32_t* __restrict__ val, int64_t n,
                const int64_t* __restrict__ n_dev, int shift, int64_t nb, const int64_t* __restrict__ scanned,
                uint32_t* __restrict__ key_out, int32_t* __restrict__ val_out)
{
    if (n_dev) n = min(*n_dev, n);
    __shared__ int32_t wcount[kRadixWarps][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = lane; d < 256; d += 32) wcount[w][d] = 0;
    __syncwarp();
    const unsigned lt = (1u << lane) - 1u;
    const int64_t base = (int64_t)blockIdx.x * kRadixTile + (int64_t)w * (kRadixRounds * 32);
    uint32_t kk[kRadixRounds];
    int32_t vv[kRadixRounds];
    int32_t rank[kRadixRounds];
#pragma unroll
    for (int r = 0; r < kRadixRounds; r++) {
        const int64_t idx = base + r * 32 + lane;
        const bool valid = idx < n;
        kk[r] = valid ? key[idx] : 0u;
        vv[r] = valid ? val[idx] : 0;
        const int d = valid ? (int)((kk[r] >> shift) & 255u) : 256 + lane;
        const unsigned peers = __match_any_sync(kFull, d);
        const int rk = __popc(peers & lt);
        const int cnt = __popc(peers);
        const int prior = valid ? wcount[w][d] : 0;
        __syncwarp();
        if (valid && rk == cnt - 1) wcount[w][d] = prior + cnt;
        __syncwarp();
        rank[r] = prior + rk;
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x) {
        int64_t run = scanned[(int64_t)d * nb + blockIdx.x];
        for (int ww = 0; ww < kRadixWarps; ww++) {
            const int32_t c = wcount[ww][d];
            wcount[ww][d] = (int32_t)run;  // positions are < 2^31
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRadixRounds; r++) {
        const int64_t idx = base + r * 32 + lane;
        if (idx < n) {
            const int d = (int)((kk[r] >> shift) & 255u);
            const int64_t dst = (int64_t)wcount[w][d] + rank[r];
            key_out[dst] = kk[r];
            val_out[dst] = vv[r];
        }
    }
}

}  // namespace

int64_t scan_scratch(int64_t n) { return (n + kScanTile - 1) / kScanTile + 2; }

// Whole scan in one block, tile by tile with a running carry, for n <= kSingleMax (the
// per-level node scans and other small scans: one launch instead of three).
constexpr int64_t kSingleMax = 16 * kScanTile;

__global__ void k_scan_single(const int32_t* __restrict__ in, int64_t n, const int64_t* __restrict__ nd,
                              int64_t* __restrict__ out)
{
    if (nd) n = min(*nd, n);
    __shared__ int64_t sh[kScanThreads / 32];
    int64_t carry = 0;
    for (int64_t t0 = 0; t0 < n; t0 += kScanTile) {
        const int64_t base = t0 + (int64_t)threadIdx.x * kScanItems;
        int64_t v[kScanItems];
        int64_t sum = 0;
#pragma unroll
        for (int i = 0; i < kScanItems; i++) {
            v[i] = base + i < n ? in[base + i] : 0;
            sum += v[i];
        }
        int64_t tot;
        int64_t run = carry + block_excl_scan<kScanThreads>(sum, sh, &tot);
#pragma unroll
        for (int i = 0; i < kScanItems; i++) {
            if (base + i < n) out[base + i] = run;
            run += v[i];
        }
        carry += tot;
    }
    if (threadIdx.x == 0) out[n] = carry;
}

void exclusive_scan_i32(const int32_t* in, int64_t* out, int64_t n, int64_t* scratch, cudaStream_t s,
                        const int64_t* n_dev)
{
    // with n_dev, n is only a capacity: the kernels read the count from the device
    if (n <= kSingleMax) {
        (k_scan_single<<<1, kScanThreads, 0, s>>>(in, n, n_dev, out), note_launch());
        return;
    }
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    (k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, n_dev, scratch), note_launch());
    (k_scan_top<<<1, 1024, 0, s>>>(scratch, nb), note_launch());
    (k_scan_down<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, n_dev, scratch, nb, out), note_launch());
}

int64_t radix_hist_size(int64_t n) { return 256 * ((n + kRadixTile - 1) / kRadixTile) + 1; }

void radix_sort_pairs(uint32_t* key, int32_t* val, uint32_t* key_tmp, int32_t* val_tmp, int64_t n,
                      int bits, uint32_t* hist, int64_t* scan_out, int64_t* scan_scratch_buf,
                      cudaStream_t s, const int64_t* n_dev)
{
    if (n <= 1) return;
    const int64_t nb = (n + kRadixTile - 1) / kRadixTile;
    const int passes = bits <= 0 ? 0 : (bits + 7) / 8;
    uint32_t *ka = key, *kb = key_tmp;
    int32_t *va = val, *vb = val_tmp;
    for (int p = 0; p < passes; p++) {
        const int shift = 8 * p;
        (k_radix_hist<<<(unsigned)nb, 256, 0, s>>>(ka, n, n_dev, shift, nb, (int32_t*)hist), note_launch());
        exclusive_scan_i32((const int32_t*)hist, scan_out, 256 * nb, scan_scratch_buf, s);
        (k_radix_scatter<<<(unsigned)nb, kRadixWarps * 32, 0, s>>>(ka, va, n, n_dev, shift, nb, scan_out, kb, vb),
         note_launch());
        uint32_t* tk = ka;
        ka = kb;
        kb = tk;
        int32_t* tv = va;
        va = vb;
        vb = tv;
    }
    if (ka != key) {
        cudaMemcpyAsync(key, ka, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(val, va, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    }
}

}  // namespace sts
