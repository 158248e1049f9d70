// Device-wide building blocks of the tree construction: an exclusive prefix scan of int32
// counts into int64 offsets, and a stable least-significant-digit radix sort of
// (uint32 key, int32 value) pairs.  Both are plain HBM-bound passes; the sort orders the
// particles by the first slot of their leaf, which (because the scan over the input runs in
// original index order and every pass is stable) keeps particles of one leaf in their
// original relative order, as the refinement of Sec. 3 does.
#include <algorithm>

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

// Single-pass exclusive scan (decoupled look-back).  Tiles are numbered in the order their
// CTAs start (a ticket counter), so every tile a CTA waits for belongs to a CTA that already
// runs; tile t publishes its aggregate, then its inclusive prefix, and adds the aggregates of
// tiles t - 1, t - 2, ... until it meets an inclusive prefix.  The tile state carries the
// scan's generation (a device counter advanced by the last CTA to finish), so the state of
// an earlier scan, or of an earlier replay of a recorded graph, never matches and no reset
// pass is needed.  Every wait is bounded: a wait that gives up flags STS_ERR_TIMEOUT.
//
// state (int64, zero when allocated): [0] ticket, [1] CTAs finished, [2] generation, then
// per tile: aggregate, inclusive prefix, and the generation + 1 at which each was published.
constexpr int kLookbackSpins = 1 << 22;

__device__ __forceinline__ int64_t ld_volatile(const int64_t* p) { return *(const volatile int64_t*)p; }

__global__ void __launch_bounds__(kScanThreads)
k_scan_onepass(const int32_t* __restrict__ in, int64_t n, const int64_t* __restrict__ nd, int64_t* __restrict__ out,
               int64_t* __restrict__ st, int64_t tcap, int* __restrict__ status)
{
    __shared__ int64_t sh[kScanThreads / 32];
    __shared__ int64_t s_tile, s_gen, s_prefix;
    if (nd) n = min(*nd, n);
    if (n > tcap * kScanTile) {  // more tiles than the state holds: flag it, scan what fits
        if (threadIdx.x == 0 && blockIdx.x == 0) atomicOr(status, kStatusCapacity);
        n = tcap * kScanTile;
    }
    const int64_t T = (n + kScanTile - 1) / kScanTile;
    if (threadIdx.x == 0) {
        s_tile = (int64_t)atomicAdd((unsigned long long*)&st[0], 1ull);
        s_gen = ld_volatile(&st[2]) + 1;
    }
    __syncthreads();
    const int64_t tile = s_tile, g = s_gen;
    int64_t* agg = st + 3;
    int64_t* inc = agg + tcap;
    int64_t* fa = inc + tcap;
    int64_t* fp = fa + tcap;
    if (tile < T) {
        const int64_t base = tile * kScanTile + (int64_t)threadIdx.x * kScanItems;
        int64_t v[kScanItems];
        int64_t sum = 0;
#pragma unroll
        for (int i = 0; i < kScanItems; i++) {
            v[i] = base + i < n ? in[base + i] : 0;
            sum += v[i];
        }
        int64_t tot;
        const int64_t local = block_excl_scan<kScanThreads>(sum, sh, &tot);
        // warp 0 publishes and looks back 32 tiles at a time: lane j reads tile hi - j; the
        // nearest tile with an inclusive prefix ends the walk, the ones before it give their
        // aggregates
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            int64_t excl = 0;
            if (lane == 0) {
                if (tile == 0) {
                    inc[0] = tot;
                    __threadfence();
                    *(volatile int64_t*)&fp[0] = g;
                } else {
                    agg[tile] = tot;
                    __threadfence();
                    *(volatile int64_t*)&fa[tile] = g;
                }
            }
            bool ok = true;
            for (int64_t hi = tile - 1; hi >= 0 && ok;) {
                const int64_t q = hi - lane;
                int state = q < 0 ? 3 : 0;  // 3: before tile 0 (adds nothing)
                int64_t val = 0;
                for (int spins = 0;; spins++) {
                    if (state == 0) {
                        if (ld_volatile(&fp[q]) == g) {
                            __threadfence();
                            val = ld_volatile(&inc[q]);
                            state = 2;
                        } else if (ld_volatile(&fa[q]) == g) {
                            __threadfence();
                            val = ld_volatile(&agg[q]);
                            state = 1;
                        }
                    }
                    if (!__any_sync(kFull, state == 0)) break;
                    if (spins > kLookbackSpins) {
                        if (lane == 0) atomicOr(status, kStatusTimeout);
                        ok = false;
                        break;
                    }
                }
                const unsigned pm = __ballot_sync(kFull, state == 2);
                const int stop = pm ? __ffs(pm) - 1 : 32;  // lanes up to stop contribute
                int64_t c = lane <= stop ? val : 0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
                excl += c;
                if (pm) break;
                hi -= 32;
            }
            if (lane == 0) {
                if (tile > 0) {
                    inc[tile] = excl + tot;
                    __threadfence();
                    *(volatile int64_t*)&fp[tile] = g;
                }
                s_prefix = excl;
                if (tile == T - 1) out[n] = excl + tot;
            }
        }
        __syncthreads();
        int64_t run = s_prefix + local;
#pragma unroll
        for (int i = 0; i < kScanItems; i++) {
            if (base + i < n) out[base + i] = run;
            run += v[i];
        }
    } else if (T == 0 && tile == 0 && threadIdx.x == 0) {
        out[0] = 0;
    }
    // the last CTA to finish rearms the state for the next scan
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned long long done = atomicAdd((unsigned long long*)&st[1], 1ull);
        if (done == (unsigned long long)gridDim.x - 1) {
            st[0] = 0;
            st[1] = 0;
            __threadfence();
            *(volatile int64_t*)&st[2] = g;
        }
    }
}

int64_t scan_state_size(int64_t n) { return 3 + 4 * ((n + kScanTile - 1) / kScanTile + 1); }

int scan_state_reserve(DevBuf<int64_t>& b, int64_t n, cudaStream_t s)
{
    const int64_t need = scan_state_size(n);
    if ((int64_t)b.cap >= need) return STS_OK;
    STS_CUDA(b.reserve(need));
    STS_CUDA(cudaMemsetAsync(b.p, 0, b.cap * sizeof(int64_t), s));  // generation 0, nothing published
    return STS_OK;
}

void exclusive_scan_i32(const int32_t* in, int64_t* out, int64_t n, DevBuf<int64_t>& state, cudaStream_t s,
                        const int* status, const int64_t* n_dev)
{
    // with n_dev, n is only a capacity: the kernel reads the count from the device
    const int64_t nb = std::max<int64_t>(1, (n + kScanTile - 1) / kScanTile);
    const int64_t tcap = ((int64_t)state.cap - 3) / 4;
    (k_scan_onepass<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, n_dev, out, state.p, tcap, (int*)status),
     note_launch());
}

int64_t radix_hist_size(int64_t n) { return 256 * ((n + kRadixTile - 1) / kRadixTile) + 1; }

void radix_sort_pairs(uint32_t* key, int32_t* val, uint32_t* key_tmp, int32_t* val_tmp, int64_t n,
                      int bits, uint32_t* hist, int64_t* scan_out, DevBuf<int64_t>& state, const int* status,
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
        exclusive_scan_i32((const int32_t*)hist, scan_out, 256 * nb, state, s, status);
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
