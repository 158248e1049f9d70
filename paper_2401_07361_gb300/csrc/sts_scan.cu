// Device-wide exclusive prefix scan of int32 counts into int64 offsets (list, cluster and
// task offsets): a plain HBM-bound pass.
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

}  // namespace sts
