// Proxy-point weights of the upward pass (Sec. 3.3.2) on the tensor cores.
//
// Each cluster's weights are W = diag(rho^d) V_ref^-T omega (the proxy-weight form of the PC
// interaction, with omega_k = sum_j B_k(b_j) zeta_j A_j the SBB moments of Sec. 3.2).  The
// contraction W'_m = sum_k omega_k Vinv[k][m] over a batch of 128 clusters is a dense
// [128, M] x [M, M] product, run here as tcgen05.mma (kind::f16, BF16 operands, FP32
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
// 2^24 in their own tensor-memory columns, so every FP32 sum is exact; the FP64 epilogue adds
// the levels:  W'_m = 2^(G + F_m) sum_L 2^-8L D_L[m].
//
// Layout: batches of 32 clusters (the MMA's 128 rows, the last 96 zero: the FP64 sums of the
// moments then spread over ~125 SMs), batch b = clusters b, b + nb, b + 2 nb, ... of the nb
// batches; persistent CTAs of 4 warps, one per SM; warp 0 reads the accumulators
// (tensor-memory lanes 0 .. 31).  Operands in shared memory in the no-swizzle K-major layout of
// 8 x 8 core matrices (K-adjacent core matrices 128 bytes apart, row groups Kp * 16 bytes
// apart); the digit table of V_ref^-1 is precomputed on the host in that layout.  One thread
// issues the MMAs and commits them to an mbarrier; the wait is bounded.  Every CTA holds all
// 512 tensor-memory columns: a second CTA on the same SM waits in tcgen05.alloc until the first
// releases them (the holder waits on nothing of the other, so the wait always ends).
#include <algorithm>

#include "sts_internal.cuh"

namespace sts {
namespace {

constexpr int kTcRows = 128;                 // rows of the MMA (M)
constexpr int kTcUsed = 32;                  // clusters per CTA (rows 32 .. 127 stay zero): the
                                             // FP64 moment sums spread over more SMs
constexpr int kTcThreads = 128;              // 4 warps
constexpr int kTcCols = 512;                 // tensor-memory columns held by a CTA
constexpr int kTcASlices = 4;                // digits of omega
constexpr int kTcLevels = kTcASlices + kTcSlices - 1;  // L = 2 .. 11
constexpr int kTcMaxKp = 80;                 // M <= 80 (degree <= 11): the operands fit shared memory
constexpr int kTcWaitSpins = 1 << 20;

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
// The exponent e of frexp (x = f 2^e, 0.5 <= f < 1) of a normal double x != 0, from its bits.
__device__ __forceinline__ int frexp_exp(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7FF) - 1022; }

// Knuth's TwoSum in FP32: hi + lo += x with the add's rounding error kept in lo.
__device__ __forceinline__ void tc_two_sum(float& hi, float& lo, float x)
{
    const float s = hi + x;
    const float bp = s - hi;
    lo += (hi - (s - bp)) + (x - bp);
    hi = s;
}

__global__ void __launch_bounds__(kTcThreads, 1)
k_proxy_weights_tc(const int32_t* __restrict__ cnode, const int64_t* __restrict__ toff,
                   const double* __restrict__ part, int M, int Kp, const uint4* __restrict__ tcB,
                   const int32_t* __restrict__ tcF, const int32_t* __restrict__ tcE, double* __restrict__ wout,
                   const int64_t* __restrict__ nclu, int* __restrict__ status)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const int64_t ncl = *nclu;
    // batch b holds clusters b, b + nb, b + 2 nb, ... (nb batches): the few large clusters of
    // the top levels, whose moments come in many partial sums, spread over the batches
    const int64_t nb = (ncl + kTcUsed - 1) / kTcUsed;
    if ((int64_t)blockIdx.x >= nb) return;  // the whole CTA: no batch for it
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int Np = Kp;
    const unsigned aBytes = (unsigned)(kTcRows * Kp * 2), bBytes = (unsigned)(Np * Kp * 2);
    unsigned char* A = smem;                        // kTcASlices digit matrices [128, Kp]
    unsigned char* B = smem + kTcASlices * aBytes;  // kTcSlices digit matrices [Np, Kp]
    double* om = reinterpret_cast<double*>(B + kTcSlices * bBytes);  // [kTcUsed, Kp] scaled moments
    int* gexp = reinterpret_cast<int*>(om + kTcUsed * Kp);           // [kTcUsed] row exponents
    uint64_t* bar = reinterpret_cast<uint64_t*>(gexp + kTcUsed);
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
    // A's rows past the batch's clusters stay zero
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
        // the moments: warp w sums rows w, w + 4, ... (lanes over k, coalesced over the partial
        // sums), scales moment k by 2^E[k] and keeps the row's largest magnitude's exponent
        for (int r = warp; r < kTcUsed; r += kTcThreads / 32) {
            const int64_t c = bt + (int64_t)r * nb;
            double mx = 0.0;
            if (c < ncl) {
                const int64_t q0 = toff[cnode[c]], q1 = toff[cnode[c] + 1];
                for (int k = lane; k < Kp; k += 32) {
                    double v = 0.0;
                    if (k < M) {
                        // four interleaved sums (their loads overlap), added in a fixed order
                        double v4[4] = {0.0, 0.0, 0.0, 0.0};
                        int64_t q = q0;
                        for (; q + 4 <= q1; q += 4) {
#pragma unroll
                            for (int u = 0; u < 4; u++) v4[u] += part[(q + u) * M + k];
                        }
                        for (int u = 0; q + u < q1; u++) v4[u] += part[(q + u) * M + k];
                        v = ((v4[0] + v4[1]) + (v4[2] + v4[3])) * pow2d(tcE[k]);  // the scaling is exact
                    }
                    om[r * Kp + k] = v;
                    mx = fmax(mx, fabs(v));
                }
            } else {
                for (int k = lane; k < Kp; k += 32) om[r * Kp + k] = 0.0;
            }
    #pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            // every scaled moment below 2^(G - 1): the leading digit stays in [-128, 128]
            if (lane == 0) gexp[r] = mx > 0.0 ? frexp_exp(mx) + 1 : 0;
        }
        __syncthreads();
        // operand A: 32 bits of each scaled moment as four balanced base-256 digits
        for (int e = tid; e < kTcUsed * Kp; e += kTcThreads) {
            const int r = e / Kp, k = e - r * Kp;
            long long T = __double2ll_rn(om[e] * pow2d(32 - gexp[r]));  // |T| <= 2^31, exact scaling
            const long long s1 = (T + (1ll << 23)) >> 24;  // floor division: round to nearest
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
        // the operands' generic writes before the tensor cores read them (async proxy)
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
                    for (int a = 1; a <= kTcASlices; a++) {
                        const int b = L - a;
                        if (b < 1 || b > kTcSlices) continue;
                        for (int kk = 0; kk < Kp / 16; kk++) {
                            const uint64_t ad = tc_desc(aBase + (unsigned)(a - 1) * aBytes + 256u * kk, 128u, sbo);
                            const uint64_t bd = tc_desc(bBase + (unsigned)(b - 1) * bBytes + 256u * kk, 128u, sbo);
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
            // epilogue, warp 0 (tensor-memory lanes 0 .. 31 hold the CTA's clusters): the levels
            // added in FP32 with TwoSum (each D_L is an exact integer below 2^24, scaled exactly by
            // 2^-8L), then W' = (hi + lo) 2^(G + F_m) in FP64
            if (warp == 0) {
                const int64_t c = bt + (int64_t)lane * nb;
                for (int m0 = 0; m0 < Np; m0 += 16) {
                    float hs[16], ls[16];
    #pragma unroll
                    for (int j = 0; j < 16; j++) hs[j] = ls[j] = 0.f;
                    for (int li = l0; li < l1; li++) {
                        uint32_t v[16];
                        asm volatile(
                            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
                            "%12, %13, %14, %15}, [%16];"
                            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                              "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                              "=r"(v[14]), "=r"(v[15])
                            : "r"(tmem + (uint32_t)((li - l0) * Np + m0)));
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                        const float sc = __uint_as_float((uint32_t)(127 - 8 * (li + 2)) << 23);  // 2^-8L
    #pragma unroll
                        for (int j = 0; j < 16; j++) tc_two_sum(hs[j], ls[j], __uint_as_float(v[j]) * sc);
                    }
                    if (c < ncl) {
    #pragma unroll
                        for (int j = 0; j < 16; j++) {
                            const int m = m0 + j;
                            if (m >= M) break;
                            const int64_t o = c * M + m;
                            const double w = ((double)hs[j] + (double)ls[j]) * pow2d(gexp[lane] + tcF[m]);
                            wout[o] = l0 > 0 ? wout[o] + w : w;
                        }
                    }
                }
            }
            // the loads of these columns (and the products' reads of A) come before the next
            // round's products and the next batch's operand writes
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
        }
    }
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols) : "memory");
}

}  // namespace

bool proxy_weights_tc_supported(int degree) { return (nbasis(degree) + 15) / 16 * 16 <= kTcMaxKp; }

int proxy_weights_tc(sts_ctx* c, const RefTable* ref, int64_t nclu, double* wout, cudaStream_t s)
{
    const int Kp = ref->tcKp;
    const size_t need = (size_t)kTcASlices * kTcRows * Kp * 2 + (size_t)kTcSlices * Kp * Kp * 2 +
                        (size_t)kTcUsed * Kp * 8 + kTcUsed * 4 + 64;
    const size_t sm = need;
    if (!c->capturing)
        STS_CUDA(cudaFuncSetAttribute(k_proxy_weights_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    // persistent: at most one CTA per SM, each looping over batches of 32 clusters (batch b:
    // clusters b, b + nb, ...)
    const int64_t batches = (nclu + kTcUsed - 1) / kTcUsed;
    const unsigned g = (unsigned)std::min<int64_t>(batches, c->num_sms);
    if (g == 0) return STS_OK;
    (k_proxy_weights_tc<<<g, kTcThreads, sm, s>>>(c->cluster_node.p, c->up_toff.p, c->up_part.p, ref->M, Kp,
                                                  reinterpret_cast<const uint4*>(ref->d_tcB.p), ref->d_tcF.p,
                                                  ref->d_tcE.p, wout, c->dc.p + kDcClusters, c->d_status),
     note_launch());
    STS_LAUNCH_CHECK();
    return STS_OK;
}

}  // namespace sts
