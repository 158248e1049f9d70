// Proxy-point weights of the upward pass (Sec. 3.3.2) on the tensor cores.
//
// Each cluster's weights are W = diag(rho^d) V_ref^-T omega (the proxy-weight form of the PC
// interaction, with omega_k = sum_j B_k(b_j) zeta_j A_j the SBB moments of Sec. 3.2).  The
// contraction W'_m = sum_k omega_k Vinv[k][m] over a batch of R clusters is a dense
// [R, M] x [M, M] product (R <= 128), run here as tcgen05.mma (kind::f16, BF16 operands, FP32
// accumulators in tensor memory).  V_ref^-1 has entries up to ~5e4 of alternating sign at d = 8
// (cond(V_ref) ~ 3.5e5), so a plain FP32 or TF32 product loses the weights; the product is
// instead made exact by splitting both operands into balanced 8-bit integer digits (the idea of
// Ozaki's error-free splitting of a matrix product):
//   omega_k 2^E[k] = 2^G sum_{a=1..4} s_a,k 2^-8a          (32 bits of the row's largest)
//   Vinv[k][m] 2^-E[k] = 2^F_m sum_{b=1..7} v_b,km 2^-8b    (every FP64 bit)
// with |s|, |v| <= 128, exact in BF16.  2^E[k] (a power of two, so nothing rounds) is the
// reciprocal of basis function k's integral over the simplex: it brings the moments, which
// span several decades, to comparable sizes, so that the 32 bits kept of the largest hold
// every moment's leading bits.  A product of digit matrices has integer entries of at most
// 80 * 128^2 < 2^21, and the (at most four) products of one level L = a + b accumulate below
// 2^24 in their own tensor-memory columns, so every FP32 sum is exact; the epilogue adds the
// levels with TwoSum and scales:  W'_m = 2^(G + F_m) sum_L 2^-8L D_L[m].
//
// Layout: persistent CTAs of 8 warps, one per SM, looping over batches of rows (the MMA's 128
// rows; the upward pass fills 32 of them, so that its FP64 sums of the moments spread over
// ~125 SMs, a row with many partial sums split over all eight warps; the interpolation
// coefficients 126: 42 clusters x 3 components).  Operands in shared
// memory in the no-swizzle K-major layout of 8 x 8 core matrices (K-adjacent core matrices 128
// bytes apart, row groups Kp * 16 bytes apart); the digit table of V_ref^-1 is precomputed on
// the host in that layout.  The row maxima and the digits are taken from the bits of the FP64
// values with integer arithmetic (FP64 runs at 1/64 of the FP32 rate here).  One thread issues
// the MMAs and commits them to an mbarrier; the wait is bounded.  Warps w and w + 4 read
// tensor-memory lanes 32 (w % 4) .. 32 (w % 4) + 31 and leave the level sums in shared memory;
// all threads then write the outputs, coalesced.  Every CTA holds all 512 tensor-memory
// columns: a second CTA on the same SM waits in tcgen05.alloc until the first releases them
// (the holder waits on nothing of the other, so the wait always ends).
#include <algorithm>

#include "sts_internal.cuh"

namespace sts {
namespace {

constexpr int kTcRows = 128;                 // rows of the MMA (M)
constexpr int kTcUp = 32;                    // rows of a batch of the upward pass (rows 32 .. 127
                                             // stay zero): its FP64 moment sums spread over more SMs
constexpr int kTcThreads = 256;              // 8 warps
constexpr int kTcWarps = kTcThreads / 32;
constexpr int kTcCols = 512;                 // tensor-memory columns held by a CTA
constexpr int kTcASlices = 4;                // digits of omega
constexpr int kTcLevels = kTcASlices + kTcSlices - 1;  // L = 2 .. 11
constexpr int kTcMaxKp = 80;                 // M <= 80 (degree <= 11): the operands fit shared memory
constexpr int kTcWaitSpins = 1 << 20;
constexpr int kTcHeavy = 32;                 // a row with more partial sums is summed by all warps

__device__ __forceinline__ unsigned su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of tcgen05: start address, leading (K) and stride (M/N)
// byte offsets, all >> 4; bit 46 the descriptor version; no swizzle, base offset 0.
__device__ __forceinline__ uint64_t tc_desc(unsigned saddr, unsigned lbo, unsigned sbo)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A and B BF16 (bits
// 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ uint32_t tc_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int accum)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ bool tc_try_wait(uint64_t* bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool tc_wait(uint64_t* bar, unsigned parity)
{
    for (int k = 0; k < kTcWaitSpins; k++)
        if (tc_try_wait(bar, parity)) return true;
    return false;
}

// A digit (an integer in [-128, 128]) as the bit pattern of the (exact) BF16 value.
__device__ __forceinline__ uint16_t bf16_of_digit(float v) { return (uint16_t)(__float_as_uint(v) >> 16); }

// 2^e as a double (e in the normal range), built from its bits: no FP64 instruction.
__device__ __forceinline__ double pow2d(int e) { return __longlong_as_double((long long)(e + 1023) << 52); }
// Knuth's TwoSum in FP32: hi + lo += x with the add's rounding error kept in lo.
__device__ __forceinline__ void tc_two_sum(float& hi, float& lo, float x)
{
    const float s = hi + x;
    const float bp = s - hi;
    lo += (hi - (s - bp)) + (x - bp);
    hi = s;
}

// The two contractions run by the kernel below.  MODE 0, the upward pass: row = cluster,
// A = the moments omega_k (summed from the moment pass's partial sums, scaled by 2^E[k]),
// B = the columns of V_ref^-1, out W'[cluster, m] (FP64), turned into the proxy points and
// weights W2 = 2 rho_m^d W'_m in the epilogue.  MODE 1, the dual traversal's
// interpolation coefficients (c = V_ref^-1 diag(rho^d) U_T, Sec. 3.3 CP / CC): row = (cluster,
// velocity component), A = rho_m^d U_m (the kernel sum at the proxy points, comparable values:
// no scaling), B = the rows of V_ref^-1, out c[cluster, k] as FP32 (x, y, z, -) per k.
struct TcArgs {
    int M, Kp, R;  // R: rows of a batch (at most 128)
    const uint4* tcB;
    const int32_t* tcF;
    const int32_t* tcE;
    const int64_t* nclu;
    int* status;
    // MODE 0: the moments' partial sums in, the proxy points and weights out (as the upward
    // pass's FP64 path forms them: y~_m, rho_m^d, W2 = 2 rho_m^d W'_m)
    const int32_t* cnode;
    const int64_t* toff;
    const double* part;
    const double* geom;
    const double* beta;
    int d;
    double4* prx64;
    float4* prx32;
    double* prx_rd;
    // MODE 1
    const uint8_t* has;
    const double* rd;
    const double* cvel;
    float* coef32;
};

// Round-half-even of x 2^s to an integer, from the bits of x (integer arithmetic: FP64
// instructions are scarce on this part).  Equal to __double2ll_rn(x * 2^s) whenever x 2^s is
// below 2^62 in magnitude.
__device__ __forceinline__ long long round_scaled(double x, int s)
{
    const long long b = __double_as_longlong(x);
    int e = (int)((b >> 52) & 0x7FF);
    unsigned long long mant = (unsigned long long)b & 0xFFFFFFFFFFFFFull;
    if (e == 0) {
        if (mant == 0) return 0;
        e = 1;  // subnormal: no implicit bit
    } else {
        mant |= 1ull << 52;
    }
    const int sh = 1075 - e - s;  // |x| 2^s = mant 2^-sh
    unsigned long long q;
    if (sh <= 0) {
        q = mant << (-sh);
    } else if (sh >= 64) {
        q = 0;  // below 2^-11: rounds to zero
    } else {
        q = mant >> sh;
        const unsigned long long rem = mant & ((1ull << sh) - 1), half = 1ull << (sh - 1);
        if (rem > half || (rem == half && (q & 1))) q++;
    }
    return b < 0 ? -(long long)q : (long long)q;
}

template <int MODE>
__global__ void __launch_bounds__(kTcThreads, 1) k_tc_contract(const TcArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const int M = a.M, Kp = a.Kp, R = a.R;
    const uint4* __restrict__ tcB = a.tcB;
    const int32_t* __restrict__ tcF = a.tcF;
    int* status = a.status;
    const int64_t ncl = *a.nclu;
    // MODE 0: row r of batch b = cluster b + r nb.  MODE 1: rows 3j .. 3j + 2 of batch b = the
    // three components of cluster b + j nb (j < R / 3).  Strided so that the few large clusters
    // of the top levels spread over the batches.
    const int per = MODE == 0 ? R : R / 3;
    const int64_t nb = (ncl + per - 1) / per;
    if ((int64_t)blockIdx.x >= nb) return;  // the whole CTA: no batch for it
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int Np = Kp;
    const unsigned aBytes = (unsigned)(kTcRows * Kp * 2), bBytes = (unsigned)(Np * Kp * 2);
    unsigned char* A = smem;                        // kTcASlices digit matrices [128, Kp]
    unsigned char* B = smem + kTcASlices * aBytes;  // kTcSlices digit matrices [Np, Kp]
    double* om = reinterpret_cast<double*>(B + kTcSlices * bBytes);  // [R, Kp] the rows (FP64)
    float* hs = reinterpret_cast<float*>(om);       // [Np, R + 1] the level sums (aliases om),
    float* ls = hs + Np * (R + 1);                  // hi and lo of TwoSum
    double* part8 = om + (size_t)Kp * (R + 1);                      // [8, Kp] warps' partial sums
    int* gexp = reinterpret_cast<int*>(part8 + (size_t)kTcWarps * Kp);  // [R] row exponents
    uint64_t* bar = reinterpret_cast<uint64_t*>(gexp + R);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // operand B: the digit table, already in the MMA layout
    const int nB = (int)(kTcSlices * bBytes / 16);
    for (int i = tid; i < nB; i += kTcThreads) reinterpret_cast<uint4*>(B)[i] = tcB[i];
    // A's rows past the batch's R stay zero
    const int nA = (int)(kTcASlices * aBytes / 16);
    for (int i = tid; i < nA; i += kTcThreads) reinterpret_cast<uint4*>(A)[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    const uint32_t tmem = *tslot;
    const uint32_t idesc = tc_idesc(kTcRows, Np);
    const unsigned aBase = su32(A), bBase = su32(B), sbo = (unsigned)(Kp * 16);
    const int perRound = kTcCols / Np;
    unsigned phase = 0;
    // persistent CTAs: batches blockIdx.x, blockIdx.x + gridDim.x, ...
    for (int64_t bt = blockIdx.x; bt < nb; bt += gridDim.x) {
        if (MODE == 0) {
            // the moments, each from its partial sums, scaled by 2^E[k] (exactly): warp w sums
            // the rows w, w + 8, ... with at most kTcHeavy partial sums (lanes over k, two k per
            // lane, four interleaved sums each); the few larger rows (the top levels' clusters)
            // come next, each split over all warps
            for (int r = warp; r < R; r += kTcWarps) {
                const int64_t c = bt + (int64_t)r * nb;
                int64_t q0 = 0, q1 = 0;
                if (c < ncl) {
                    q0 = a.toff[a.cnode[c]];
                    q1 = a.toff[a.cnode[c] + 1];
                    if (q1 - q0 > kTcHeavy) continue;  // below
                }
                for (int k0 = 0; k0 < Kp; k0 += 64) {
                    const int ka = k0 + lane, kb = k0 + 32 + lane;
                    const bool va = c < ncl && ka < M, vb = c < ncl && kb < M;
                    double sa[4] = {0.0, 0.0, 0.0, 0.0}, sb[4] = {0.0, 0.0, 0.0, 0.0};
                    int64_t q = q0;
                    for (; q + 4 <= q1; q += 4) {
#pragma unroll
                        for (int u = 0; u < 4; u++) {
                            if (va) sa[u] += a.part[(q + u) * M + ka];
                            if (vb) sb[u] += a.part[(q + u) * M + kb];
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 3; u++) {
                        if (q + u < q1) {
                            if (va) sa[u] += a.part[(q + u) * M + ka];
                            if (vb) sb[u] += a.part[(q + u) * M + kb];
                        }
                    }
                    if (ka < Kp) om[r * Kp + ka] = va ? ((sa[0] + sa[1]) + (sa[2] + sa[3])) * pow2d(a.tcE[ka]) : 0.0;
                    if (kb < Kp) om[r * Kp + kb] = vb ? ((sb[0] + sb[1]) + (sb[2] + sb[3])) * pow2d(a.tcE[kb]) : 0.0;
                }
            }
            for (int r = 0; r < R; r++) {  // the same branch in every thread
                const int64_t c = bt + (int64_t)r * nb;
                if (c >= ncl) continue;
                const int64_t q0 = a.toff[a.cnode[c]], q1 = a.toff[a.cnode[c] + 1];
                if (q1 - q0 <= kTcHeavy) continue;
                // warp w: partial sums q0 + w, q0 + w + 8, ... (four interleaved), then the eight
                // warps' sums added in warp order
                for (int k0 = 0; k0 < Kp; k0 += 64) {
                    const int ka = k0 + lane, kb = k0 + 32 + lane;
                    const bool va = ka < M, vb = kb < M;
                    double sa[4] = {0.0, 0.0, 0.0, 0.0}, sb[4] = {0.0, 0.0, 0.0, 0.0};
                    int64_t q = q0 + warp;
                    for (; q + 3 * kTcWarps < q1; q += 4 * kTcWarps) {
#pragma unroll
                        for (int u = 0; u < 4; u++) {
                            if (va) sa[u] += a.part[(q + u * kTcWarps) * M + ka];
                            if (vb) sb[u] += a.part[(q + u * kTcWarps) * M + kb];
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 3; u++) {
                        if (q + u * kTcWarps < q1) {
                            if (va) sa[u] += a.part[(q + u * kTcWarps) * M + ka];
                            if (vb) sb[u] += a.part[(q + u * kTcWarps) * M + kb];
                        }
                    }
                    if (ka < Kp) part8[warp * Kp + ka] = (sa[0] + sa[1]) + (sa[2] + sa[3]);
                    if (kb < Kp) part8[warp * Kp + kb] = (sb[0] + sb[1]) + (sb[2] + sb[3]);
                }
                __syncthreads();
                for (int k = tid; k < Kp; k += kTcThreads) {
                    double v = 0.0;
                    for (int w8 = 0; w8 < kTcWarps; w8++) v += part8[w8 * Kp + k];
                    om[r * Kp + k] = k < M ? v * pow2d(a.tcE[k]) : 0.0;
                }
                __syncthreads();
            }
        } else {
            // rho_m^d (kept by the upward pass) times the kernel sum at proxy point m, the three
            // components at once (rows 3j .. 3j + 2)
            const int nj = R / 3;
            for (int e = tid; e < nj * Kp; e += kTcThreads) {
                const int j = e / Kp, m = e - j * Kp;
                const int64_t cs = bt + (int64_t)j * nb;
                double v0 = 0.0, v1 = 0.0, v2 = 0.0;
                if (m < M && cs < ncl && a.has[cs]) {
                    const int64_t o = cs * M + m;
                    const double rd = a.rd[o];
                    v0 = rd * a.cvel[3 * o];
                    v1 = rd * a.cvel[3 * o + 1];
                    v2 = rd * a.cvel[3 * o + 2];
                }
                om[(3 * j) * Kp + m] = v0;
                om[(3 * j + 1) * Kp + m] = v1;
                om[(3 * j + 2) * Kp + m] = v2;
            }
            for (int e = 3 * nj * Kp + tid; e < R * Kp; e += kTcThreads) om[e] = 0.0;
        }
        __syncthreads();
        // each row's largest magnitude (compared as bits: no FP64 instruction); every scaled
        // value below 2^(G - 1), so the leading digit stays in [-128, 128]
        for (int r = warp; r < R; r += kTcWarps) {
            unsigned long long mx = 0;
            for (int k = lane; k < Kp; k += 32)
                mx = max(mx, (unsigned long long)__double_as_longlong(om[r * Kp + k]) & 0x7FFFFFFFFFFFFFFFull);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (lane == 0) gexp[r] = mx != 0 ? (int)(mx >> 52) - 1021 : 0;
        }
        __syncthreads();
        // operand A: 32 bits of each row value as four balanced base-256 digits
        for (int e = tid; e < R * Kp; e += kTcThreads) {
            const int r = e / Kp, k = e - r * Kp;
            long long T = round_scaled(om[e], 32 - gexp[r]);  // |T| <= 2^31
            const long long s1 = (T + (1ll << 23)) >> 24;     // floor division: round to nearest
            T -= s1 * (1ll << 24);
            const long long s2 = (T + (1ll << 15)) >> 16;
            T -= s2 * (1ll << 16);
            const long long s3 = (T + (1ll << 7)) >> 8;
            const long long s4 = T - s3 * (1ll << 8);
            const unsigned off = tc_kmajor_offset(r, k, Kp);
            *reinterpret_cast<uint16_t*>(A + off) = bf16_of_digit((float)s1);
            *reinterpret_cast<uint16_t*>(A + aBytes + off) = bf16_of_digit((float)s2);
            *reinterpret_cast<uint16_t*>(A + 2 * aBytes + off) = bf16_of_digit((float)s3);
            *reinterpret_cast<uint16_t*>(A + 3 * aBytes + off) = bf16_of_digit((float)s4);
        }
        // the operands' generic writes before the tensor cores read them (async proxy); om is
        // dead from here (hs / ls take its place)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        for (int l0 = 0; l0 < kTcLevels; l0 += perRound) {
            const int l1 = min(kTcLevels, l0 + perRound);
            if (tid == 0) {
                for (int li = l0; li < l1; li++) {
                    const int L = li + 2;
                    const uint32_t dcol = tmem + (uint32_t)((li - l0) * Np);
                    int acc = 0;
                    for (int sa = 1; sa <= kTcASlices; sa++) {
                        const int sb = L - sa;
                        if (sb < 1 || sb > kTcSlices) continue;
                        for (int kk = 0; kk < Kp / 16; kk++) {
                            const uint64_t ad = tc_desc(aBase + (unsigned)(sa - 1) * aBytes + 256u * kk, 128u, sbo);
                            const uint64_t bd = tc_desc(bBase + (unsigned)(sb - 1) * bBytes + 256u * kk, 128u, sbo);
                            tc_mma(dcol, ad, bd, idesc, acc);
                            acc = 1;
                        }
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 su32(bar))
                             : "memory");
            }
            if (!tc_wait(bar, phase)) {
                // give the products a bounded time to land, flag the timeout, free the columns
                if (tid == 0) atomicOr(status, kStatusTimeout);
                tc_wait(bar, phase);
                tc_fence_before();
                __syncthreads();
                if (warp == 0)
                    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols)
                                 : "memory");
                return;
            }
            phase ^= 1u;
            tc_fence_after();
            // epilogue, first half: warps w and w + 4 read tensor-memory lanes 32 (w % 4) ..
            // (rows of the batch), each half of the 16-column chunks, and add the levels in FP32
            // with TwoSum (each D_L an exact integer below 2^24, scaled exactly by 2^-8L),
            // carrying hi / lo over the rounds in shared memory
            const int quarter = warp & 3, r = 32 * quarter + lane;
            if (32 * quarter < R) {
                const uint32_t tlane = tmem + ((uint32_t)(32 * quarter) << 16);
                for (int m0 = 16 * (warp >> 2); m0 < Np; m0 += 32) {
                    float h[16], l[16];
#pragma unroll
                    for (int j = 0; j < 16; j++) {
                        h[j] = (l0 > 0 && r < R) ? hs[(m0 + j) * (R + 1) + r] : 0.f;
                        l[j] = (l0 > 0 && r < R) ? ls[(m0 + j) * (R + 1) + r] : 0.f;
                    }
                    for (int li = l0; li < l1; li++) {
                        uint32_t v[16];
                        asm volatile(
                            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
                            "%12, %13, %14, %15}, [%16];"
                            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                              "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                              "=r"(v[14]), "=r"(v[15])
                            : "r"(tlane + (uint32_t)((li - l0) * Np + m0)));
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                        const float sc = __uint_as_float((uint32_t)(127 - 8 * (li + 2)) << 23);  // 2^-8L
#pragma unroll
                        for (int j = 0; j < 16; j++) tc_two_sum(h[j], l[j], __uint_as_float(v[j]) * sc);
                    }
                    if (r < R) {
#pragma unroll
                        for (int j = 0; j < 16; j++) {
                            hs[(m0 + j) * (R + 1) + r] = h[j];
                            ls[(m0 + j) * (R + 1) + r] = l[j];
                        }
                    }
                }
            }
            // the loads of these columns (and the products' reads of A) come before the next
            // round's products and the next batch's operand writes; hs / ls complete
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
        }
        // epilogue, second half (every thread, coalesced over m): the value 2^(G + F_m) (hi + lo)
        if (MODE == 0) {
            // W' in FP64, then proxy point m of the cluster: y~_m = unit(beta_m . corners),
            // rho_m = |beta_m . corners|, W2 = 2 rho_m^d W'_m (the FP32 copy relative to the centre)
            for (int e = tid; e < R * M; e += kTcThreads) {
                const int r = e / M, m = e - r * M;
                const int64_t c = bt + (int64_t)r * nb;
                if (c < ncl) {
                    const int o = m * (R + 1) + r;
                    const double wv = ((double)hs[o] + (double)ls[o]) * pow2d(gexp[r] + tcF[m]);
                    const double* g = a.geom + 13 * (int64_t)a.cnode[c];
                    const double b1 = a.beta[3 * m], b2 = a.beta[3 * m + 1], b3 = a.beta[3 * m + 2];
                    const double sx = (b1 * g[0] + b2 * g[3]) + b3 * g[6];
                    const double sy = (b1 * g[1] + b2 * g[4]) + b3 * g[7];
                    const double sz = (b1 * g[2] + b2 * g[5]) + b3 * g[8];
                    const double ss = (sx * sx + sy * sy) + sz * sz;
                    const double ri = rsqrt(ss);
                    const double yx = sx * ri, yy = sy * ri, yz = sz * ri, rho = ss * ri;
                    double rd = 1.0;
                    for (int q = 0; q < a.d; q++) rd *= rho;
                    const double W2 = 2.0 * (rd * wv);
                    const int64_t i = c * M + m;
                    a.prx_rd[i] = rd;
                    a.prx64[i] = make_double4(yx, yy, yz, W2);
                    a.prx32[i] = make_float4((float)(yx - g[9]), (float)(yy - g[10]), (float)(yz - g[11]), (float)W2);
                }
            }
        } else {
            // the coefficients in FP32: hi + lo rounded once, then scaled exactly
            const int nj = R / 3;
            for (int e = tid; e < nj * M; e += kTcThreads) {
                const int j = e / M, m = e - j * M;
                const int64_t cs = bt + (int64_t)j * nb;
                if (cs < ncl && a.has[cs]) {
                    float* o = a.coef32 + 4 * (cs * M + m);
#pragma unroll
                    for (int comp = 0; comp < 3; comp++) {
                        const int r = 3 * j + comp, i = m * (R + 1) + r;
                        o[comp] = ldexpf(hs[i] + ls[i], gexp[r] + tcF[m]);
                    }
                }
            }
        }
        // hs / ls read before the next batch's rows overwrite them
        __syncthreads();
    }
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols) : "memory");
}

}  // namespace

bool proxy_weights_tc_supported(int degree) { return (nbasis(degree) + 15) / 16 * 16 <= kTcMaxKp; }

namespace {

// Shared memory of a CTA with batches of R rows: the digit matrices, then the rows (FP64) /
// level sums (hi, lo), then R row exponents, the mbarrier and the tensor-memory address.
size_t tc_smem(int Kp, int R)
{
    return (size_t)kTcASlices * kTcRows * Kp * 2 + (size_t)kTcSlices * Kp * Kp * 2 + (size_t)Kp * (R + 1) * 8 +
           (size_t)kTcWarps * Kp * 8 + (size_t)R * 4 + 16;
}

template <int MODE>
int launch_tc(sts_ctx* c, TcArgs a, int64_t nclu_cap, cudaStream_t s)
{
    const int Kp = a.Kp;
    if (MODE == 0) {
        a.R = kTcUp;
    } else {
        // the largest batch the shared memory holds (three rows per cluster)
        int optin = 0;
        STS_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
        a.R = 126;
        while (a.R > 3 && tc_smem(Kp, a.R) > (size_t)optin) a.R -= 30;
    }
    const size_t sm = tc_smem(Kp, a.R);
    if (!c->capturing)
        STS_CUDA(cudaFuncSetAttribute(k_tc_contract<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    // persistent: at most one CTA per SM, each looping over its batches
    const int per = MODE == 0 ? a.R : a.R / 3;
    const int64_t batches = (nclu_cap + per - 1) / per;
    const unsigned g = (unsigned)std::min<int64_t>(batches, c->num_sms);
    if (g == 0) return STS_OK;
    (k_tc_contract<MODE><<<g, kTcThreads, sm, s>>>(a), note_launch());
    STS_LAUNCH_CHECK();
    return STS_OK;
}

}  // namespace

int proxy_weights_tc(sts_ctx* c, const RefTable* ref, int degree, int64_t nclu, cudaStream_t s)
{
    TcArgs a{};
    a.M = ref->M;
    a.Kp = ref->tcKp;
    a.tcB = reinterpret_cast<const uint4*>(ref->d_tcB.p);
    a.tcF = ref->d_tcF.p;
    a.tcE = ref->d_tcE.p;
    a.nclu = c->dc.p + kDcClusters;
    a.status = c->d_status;
    a.cnode = c->cluster_node.p;
    a.toff = c->up_toff.p;
    a.part = c->up_part.p;
    a.geom = c->nd_geom.p;
    a.beta = ref->d_beta.p;
    a.d = degree;
    a.prx64 = c->prx64.p;
    a.prx32 = c->prx32.p;
    a.prx_rd = c->prx_rd.p;
    return launch_tc<0>(c, a, nclu, s);
}

int cluster_coef_tc(sts_ctx* c, const RefTable* ref, int degree, int64_t nclu, const double* cvel, float* coef32,
                    cudaStream_t s)
{
    TcArgs a{};
    a.M = ref->M;
    a.Kp = ref->tcKp;
    a.tcB = reinterpret_cast<const uint4*>(ref->d_tcBr.p);
    a.tcF = ref->d_tcFr.p;
    a.nclu = c->dc.p + kDcClusters;
    a.status = c->d_status;
    a.cnode = c->cluster_node.p;
    a.has = c->chas.p;
    a.rd = c->prx_rd.p;
    a.cvel = cvel;
    a.coef32 = coef32;
    return launch_tc<1>(c, a, nclu, s);
}

}  // namespace sts
