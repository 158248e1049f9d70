// Velocity evaluation: the tree code's far field (PC interactions with the proxy points of
// well-separated clusters, Sec. 3.3.2) and near field (PP interactions, Sec. 3.3.1), and the
// direct sum of the Sec. 2 particle system.  Every pair term is
//     w_j (x_i x d) / (|d|^2 / 2),   d = y_j - x_i,   w_j = zeta_j A_j,
// i.e. the kernel (x_i x x_j) / (1 - x_i . x_j) with 1 - x.y written as |x - y|^2 / 2
// (Eq. altkernel) and x_i x x_j = x_i x d.  The kernels accumulate S_i = sum_j 2 w_j d /
// |d|^2 and the epilogue forms u_i = -(1/4 pi) x_i x S_i in FP64.
//
// Evaluation layout: one warp per task (up to 64 consecutive targets of one leaf, two per
// lane); S = 1..8 lanes share a pair of targets and split its sources, summed with shuffles at
// the end.  Persistent CTAs take the tasks from a device queue.  Consecutive source blocks (a
// cluster's M proxy points, a chunk of a near leaf's particles) of one kind are staged back
// to back as a group in one of two shared-memory stages by TMA bulk copies against the
// stage's mbarrier; one pass then moves every source into the task leaf's frame, the group is
// padded once to a multiple of 4 S entries, and each lane streams the whole stage with
// broadcast shared-memory reads.
//
// Mixed precision (STS_MIXED): targets, sources and proxy points are stored in FP32
// relative to the circumcentre of their own leaf or cluster; the FP32 offset between the two
// centres (rounded once from FP64 per list entry) is added to the staged sources, so that
// d = (y + delta) - x keeps FP32 relative accuracy at every distance the tree produces.  Per
// group the lane sums in FP32, and the group partials go into a TwoSum-compensated
// accumulator.  Near pairs
// with |d|^2 / 2 < tau are evaluated in FP64 from the FP64 positions instead.  A zero d
// (the target itself, or a coincident particle) contributes nothing, as in the oracle:
// |d|^2 carries an additive 1e-30 so that 2w / |d|^2 stays finite and is multiplied by 0.
#include <algorithm>
#include <mutex>

#include "sts_internal.cuh"

namespace sts {
namespace {

constexpr unsigned kFull = 0xffffffffu;

constexpr float kEps = 1e-30f;
constexpr double kInv4Pi = 1.0 / (4.0 * kPi);
constexpr double kLn2 = 0.6931471805599453;  // ln 2 rounded to FP64

inline unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Knuth's TwoSum: hi + lo += p with the rounding error of the add kept in lo.
__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float p)
{
    const float s = hi + p;
    const float bp = s - hi;
    const float e = (hi - (s - bp)) + (p - bp);
    hi = s;
    lo += e;
}

__device__ __forceinline__ void pair64(const double4 s, double tx, double ty, double tz, double& ax,
                                       double& ay, double& az)
{
    const double dx = s.x - tx, dy = s.y - ty, dz = s.z - tz;
    const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
    const double c = r2 > 0.0 ? s.w / r2 : 0.0;
    ax = fma(c, dx, ax);
    ay = fma(c, dy, ay);
    az = fma(c, dz, az);
}

// The potential kernel's pair term (Sec. 2 Green's function, Eq. altkernel): acc += (2 w)
// log(|d|^2 / 2); the caller scales by -1/(8 pi).  A source at the target's position (the
// target itself, or a distinct particle at the same point) adds nothing.
__device__ __forceinline__ void pot64(const double4 s, double tx, double ty, double tz, double& acc)
{
    const double dx = s.x - tx, dy = s.y - ty, dz = s.z - tz;
    const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
    if (r2 > 0.0) acc = fma(s.w, log(0.5 * r2), acc);
}

// ------------------------------------------------------------------------ tree tasks
// Task layout: targets t0 .. t0 + nt - 1 of one leaf; lane j < p = ceil(nt / 2) of phase s
// (lane = s p + j, s < S) holds targets t0 + 2j and t0 + 2j + 1 and takes the sources
// s, s + S, s + 2S, ... of every block; lanes beyond S p idle.  Blocks are the task leaf's
// far entries (M proxy points of a cluster) followed by its near chunks (<= kStage particles
// of a near leaf).
constexpr int kEvalWarps = 8;
constexpr int kEvalWarps64 = 4;

// The tasks a launch evaluates (those of leaves [leaf_lo, leaf_hi)) and where the targets'
// rows go: out_base < 0, row perm[t] (the caller's order); else row t - out_base.
struct EvalRange {
    int64_t leaf_lo, leaf_hi, out_base;
};

// Bulk copies (the TMA engine's 1-D form) into shared memory, completed on an mbarrier.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// dst, src and bytes are multiples of 16 bytes
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// A bounded wait for the phase `parity` of an mbarrier (all lanes of the warp): false after
// kWaitSpins polls, which no copy of a few KB ever needs; the caller then reports
// STS_ERR_TIMEOUT instead of hanging.
constexpr int kWaitSpins = 1 << 20;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int spins = kWaitSpins)
{
    for (int k = 0; k < spins; k++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// The bounded wait on a barrier that nothing arrives on: it must give up after `spins` polls
// and flag the timeout in the status word, leaving the context usable.
__global__ void k_wait_selftest(int spins, int* __restrict__ status)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_init_fence();
    }
    __syncwarp();
    const bool done = mbar_wait(&bar, 0, spins);
    if (!done && threadIdx.x == 0) atomicOr(status, kStatusTimeout);
}

// FP64 evaluation of one near pair whose FP32 squared distance fell below 2 tau; the sum
// goes to corr (sorted order), read back by the owning lane in the epilogue.
__device__ __forceinline__ void close_pair(const double4* __restrict__ src64, const double4* __restrict__ tgt64,
                                           int64_t j, int64_t tk, double* __restrict__ corr)
{
    const double4 y = src64[j];
    const double4 x = tgt64[tk];
    const double dx = y.x - x.x, dy = y.y - x.y, dz = y.z - x.z;
    const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
    if (r2 > 0.0) {
        const double t = y.w / r2;
        atomicAdd(corr + 3 * tk, t * dx);
        atomicAdd(corr + 3 * tk + 1, t * dy);
        atomicAdd(corr + 3 * tk + 2, t * dz);
    }
}

__device__ __forceinline__ float sqdist(const float4 s, float ax, float ay, float az)
{
    const float dx = s.x - ax, dy = s.y - ay, dz = s.z - az;
    return fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, kEps)));
}

// The FP32 pair loop of one staged group for a lane's two targets: entries ph, ph + S, ... of
// the group padded to a multiple of 4 S (padding entries carry w = 0 far away), four per trip,
// the two targets in the two halves of paired FP32 instructions (f32x2: one FADD2 / FFMA2 /
// FMUL2 does a step for both, halving the issued FP32 instructions of an issue-bound loop).
// TEST:
// pairs with |d|^2 < 2 tau contribute nothing here and set `hit`; the caller then evaluates
// them in FP64.
template <bool TEST, int S>
__device__ __forceinline__ void block_pairs(const float4* sb, int cntp, int ph, float ax, float ay, float az,
                                            float bx, float by, float bz, float& p0x, float& p0y, float& p0z,
                                            float& p1x, float& p1y, float& p1z, float tau2, bool& hit)
{
    // the two targets as the halves of paired FP32 operations (f32x2: each half the scalar
    // operation, so the squared distances are bit for bit those of the close-pair pass)
    const float2 na = make_float2(-ax, -bx), nb = make_float2(-ay, -by), nc = make_float2(-az, -bz);
    const float2 eps2 = make_float2(kEps, kEps);
    float2 px = make_float2(p0x, p1x), py = make_float2(p0y, p1y), pz = make_float2(p0z, p1z);
    for (int i = ph; i < cntp; i += 4 * S) {
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const float4 s = sb[i + u * S];
            const float2 dx = __fadd2_rn(make_float2(s.x, s.x), na);
            const float2 dy = __fadd2_rn(make_float2(s.y, s.y), nb);
            const float2 dz = __fadd2_rn(make_float2(s.z, s.z), nc);
            const float2 r = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __ffma2_rn(dx, dx, eps2)));
            float2 c = __fmul2_rn(make_float2(s.w, s.w), make_float2(rcp_approx(r.x), rcp_approx(r.y)));
            if (TEST) {
                const bool z0 = r.x < tau2, z1 = r.y < tau2;
                c.x = z0 ? 0.f : c.x;
                c.y = z1 ? 0.f : c.y;
                hit = hit || z0 || z1;
            }
            px = __ffma2_rn(c, dx, px);
            py = __ffma2_rn(c, dy, py);
            pz = __ffma2_rn(c, dz, pz);
        }
    }
    p0x = px.x;
    p1x = px.y;
    p0y = py.x;
    p1y = py.y;
    p0z = pz.x;
    p1z = pz.y;
}

// Second pass over a tested block for a lane that hit (its entries ph, ph + S, ...; slot
// base + i): the same FP32 squared distances pick the same pairs, which are evaluated in FP64
// from the FP64 positions.
template <int S>
__device__ __forceinline__ void block_close_pairs(const float4* sb, int cnt, int ph, float ax, float ay, float az,
                                                  float bx, float by, float bz, float tau2, int64_t base,
                                                  int64_t tk0, int64_t tk1, const double4* __restrict__ src64,
                                                  const double4* __restrict__ tgt64, double* __restrict__ corr)
{
    for (int i = ph; i < cnt; i += S) {
        const float4 s = sb[i];
        if (sqdist(s, ax, ay, az) < tau2) close_pair(src64, tgt64, base + i, tk0, corr);
        if (sqdist(s, bx, by, bz) < tau2) close_pair(src64, tgt64, base + i, tk1, corr);
    }
}

// The potential's FP64 close pair: corr[tk] += (2 w) log(|d|^2 / 2) (pot64's term).
__device__ __forceinline__ void close_pot(const double4* __restrict__ src64, const double4* __restrict__ tgt64,
                                          int64_t j, int64_t tk, double* __restrict__ corr)
{
    double a = 0.0;
    const double4 x = tgt64[tk];
    pot64(src64[j], x.x, x.y, x.z, a);
    if (a != 0.0) atomicAdd(corr + tk, a);
}

// The potential's FP32 pair loop (Sec. 2 Green's function) over one staged group, as
// block_pairs: (2 w) log2(|d|^2 / 2) per pair, the two targets in the halves of paired FP32
// instructions.  The log terms of a zero-mean vorticity cancel by ~100 across a target's
// sources, so the running sums are TwoSum-compensated pairs (hi, lo) per target: FP32 sums of
// the uncancelled partials would lose the result.  log2 by the FP32 hardware approximation
// (absolute error ~2^-22 whatever the argument); the caller scales by ln 2 in FP64.  TEST:
// pairs with |d|^2 below tau2 are left out (the close-pair pass takes them in FP64).
template <bool TEST, int S>
__device__ __forceinline__ void block_pot(const float4* sb, int cntp, int ph, float ax, float ay, float az,
                                          float bx, float by, float bz, float2& hi, float2& lo, float tau2,
                                          bool& hit)
{
    const float2 na = make_float2(-ax, -bx), nb = make_float2(-ay, -by), nc = make_float2(-az, -bz);
    const float2 eps2 = make_float2(kEps, kEps), half = make_float2(0.5f, 0.5f);
    for (int i = ph; i < cntp; i += 4 * S) {
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const float4 s = sb[i + u * S];
            const float2 dx = __fadd2_rn(make_float2(s.x, s.x), na);
            const float2 dy = __fadd2_rn(make_float2(s.y, s.y), nb);
            const float2 dz = __fadd2_rn(make_float2(s.z, s.z), nc);
            const float2 r = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __ffma2_rn(dx, dx, eps2)));
            const float2 h = __fmul2_rn(r, half);
            float2 t = __fmul2_rn(make_float2(s.w, s.w), make_float2(__log2f(h.x), __log2f(h.y)));
            if (TEST) {
                const bool z0 = r.x < tau2, z1 = r.y < tau2;
                t.x = z0 ? 0.f : t.x;
                t.y = z1 ? 0.f : t.y;
                hit = hit || z0 || z1;
            }
            // Knuth's TwoSum: hi + t = sum + e exactly; lo collects e
            const float2 sum = __fadd2_rn(hi, t);
            const float2 bv = __fadd2_rn(sum, make_float2(-hi.x, -hi.y));
            const float2 av = __fadd2_rn(sum, make_float2(-bv.x, -bv.y));
            const float2 ea = __fadd2_rn(hi, make_float2(-av.x, -av.y));
            const float2 eb = __fadd2_rn(t, make_float2(-bv.x, -bv.y));
            lo = __fadd2_rn(lo, __fadd2_rn(ea, eb));
            hi = sum;
        }
    }
}

// The potential's close pairs of one tested block for a lane that hit, as block_close_pairs.
template <int S>
__device__ __forceinline__ void block_close_pot(const float4* sb, int cnt, int ph, float ax, float ay, float az,
                                                float bx, float by, float bz, float tau2, int64_t base, int64_t tk0,
                                                int64_t tk1, const double4* __restrict__ src64,
                                                const double4* __restrict__ tgt64, double* __restrict__ corr)
{
    for (int i = ph; i < cnt; i += S) {
        const float4 s = sb[i];
        if (sqdist(s, ax, ay, az) < tau2) close_pot(src64, tgt64, base + i, tk0, corr);
        if (sqdist(s, bx, by, bz) < tau2) close_pot(src64, tgt64, base + i, tk1, corr);
    }
}

// ------------------------------------------------------------------------ mixed tree
// A group: consecutive blocks of one kind (untested, or near blocks tested for close pairs)
// with at most kGroupMax sources in all, staged back to back and padded once, at its end, to
// a multiple of 4 S entries (at most 31 more).
// Groups of up to 352 sources (two 384-entry stages, 12 KB, per warp) at two CTAs of 8
// warps per SM: measured at 655k targets, 2.37 ms against 2.41 ms for 192-source groups at
// three CTAs per SM (the per-group work is amortised over twice the pairs; occupancy 16 warps).
#ifndef STS_GROUP_MAX
#define STS_GROUP_MAX 352
#endif
constexpr int kGroupMax = STS_GROUP_MAX;
constexpr int kStagePad = kGroupMax + 32;
static_assert(kStage <= kGroupMax, "one proxy block or near chunk must fit a group");
#ifndef STS_EVAL_MIN_BLOCKS
#define STS_EVAL_MIN_BLOCKS 2  // resident blocks per SM asked of the register allocator
#endif
constexpr int kRing = 64;               // block descriptors per warp: two windows of 32

// Per-warp shared state of the mixed evaluation: two stages and a ring of block descriptors.
struct EvalSmem {
    float4 stage[2][kStagePad];
    float4 off[kRing];  // source offset (dx, dy, dz) of the block
    int4 info[kRing];   // first source (slot or cluster), count, kind (0 far, 1 near, 2 tested near),
                        // start of the block within its window (sum of the counts before it)
    uint64_t bar[2];    // mbarriers of the two stages
};

struct Group {
    int e0, e1;  // ring positions [e0, e1)
    int base;    // window start of e0
    int cnt;     // sources of the group
    bool tested;
};

// Loads the descriptors of list blocks [wb, wb + 32) into the ring at positions wb .. wb + 31:
// the untested blocks first, then the near blocks whose gap bound is below tau_r (the ones
// tested for close pairs), each part in list order, so that a window holds at most two runs of
// one kind.  Returns the inclusive prefix of the counts at the lane's position and sets the
// position's tested flag.
__device__ __forceinline__ int load_window(EvalSmem& sm, int wb, int lane, int nf, int nbt,
                                           const FarEntry* __restrict__ fe, const NearEntry* __restrict__ ne,
                                           int M, float tau_r, bool& tested)
{
    const int e = wb + lane;
    const bool valid = e < nbt;
    int idx = 0, cnt = 0, kind = 0;
    float dx = 0.f, dy = 0.f, dz = 0.f;
    if (valid) {
        if (e < nf) {
            const FarEntry f = fe[e];
            idx = f.slot;
            cnt = M;
            dx = f.dx;
            dy = f.dy;
            dz = f.dz;
        } else {
            const NearEntry q = ne[e - nf];
            idx = q.start;
            cnt = q.count;
            dx = q.dx;
            dy = q.dy;
            dz = q.dz;
            kind = q.gap < tau_r ? 2 : 1;
        }
    }
    const unsigned um = __ballot_sync(kFull, valid && kind != 2);
    const unsigned tm = __ballot_sync(kFull, valid && kind == 2);
    const unsigned lt = (1u << lane) - 1u;
    // invalid lanes are the top ones (e >= nbt) and keep their positions
    const int pos = !valid ? lane : (kind == 2 ? __popc(um) + __popc(tm & lt) : __popc(um & lt));
    const int r = (wb + pos) & (kRing - 1);
    sm.off[r] = make_float4(dx, dy, dz, 0.f);
    sm.info[r] = make_int4(idx, cnt, kind, 0);
    __syncwarp();
    const int me = (wb + lane) & (kRing - 1);
    const int c = sm.info[me].y;
    tested = sm.info[me].z == 2;
    int inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += v;
    }
    sm.info[me].w = inc - c;
    __syncwarp();
    return inc;
}

// The largest run of blocks of one kind from ring position e0 on, within e0's window, whose
// sources fit one group; loads the next window when e0 starts it.  An empty group (e0 == e1)
// ends the task.
__device__ __forceinline__ Group form_group(EvalSmem& sm, int e0, int& wb, int& winc, bool& wtest, int lane, int nf,
                                            int nbt, const FarEntry* __restrict__ fe,
                                            const NearEntry* __restrict__ ne, int M, float tau_r)
{
    Group g;
    g.e0 = g.e1 = e0;
    g.base = g.cnt = 0;
    g.tested = false;
    if (e0 >= nbt) return g;
    if (e0 >= wb + 32) {
        wb += 32;
        winc = load_window(sm, wb, lane, nf, nbt, fe, ne, M, tau_r, wtest);
    }
    const int r = e0 - wb;
    const int prev = __shfl_sync(kFull, winc, (r + 31) & 31);
    g.base = r > 0 ? prev : 0;
    g.tested = __shfl_sync(kFull, (int)wtest, r) != 0;
    const unsigned other = __ballot_sync(kFull, lane >= r && wtest != g.tested);
    const int end = other ? __ffs(other) - 1 : 32;
    const bool in = lane >= r && lane < end && wb + lane < nbt && winc - g.base <= kGroupMax;
    const int k = __popc(__ballot_sync(kFull, in));
    g.e1 = e0 + k;
    g.cnt = __shfl_sync(kFull, winc, r + k - 1) - g.base;
    return g;
}

// Copies the blocks of a group into a stage, back to back: one bulk copy per block, issued by
// its own lane, against the stage's mbarrier (lane 0 arms it with the group's byte count; a
// copy that lands first leaves the count transiently negative, which the barrier allows), and
// pads the group with zero-weight entries far from every target up to a multiple of 4 S.
template <int S>
__device__ __forceinline__ void issue_group(EvalSmem& sm, const Group& g, int stg, int lane,
                                            const float4* __restrict__ prx32, const float4* __restrict__ src32,
                                            int M)
{
    if (g.e1 == g.e0) return;
    float4* st = sm.stage[stg];
    // the stage's earlier generic reads and writes (two groups ago) come before the copies
    fence_proxy_async();
    __syncwarp();
    const int e = g.e0 + lane;
    int bytes = 0;
    if (e < g.e1) {
        const int4 in = sm.info[e & (kRing - 1)];
        const float4* src = in.z == 0 ? prx32 + (int64_t)in.x * M : src32 + in.x;
        bytes = 16 * in.y;
        if (in.y > 0) bulk_g2s(st + (in.w - g.base), src, (unsigned)bytes, &sm.bar[stg]);
    }
    const int gp = (g.cnt + 4 * S - 1) / (4 * S) * (4 * S);
    if (g.cnt + lane < gp) st[g.cnt + lane] = make_float4(1e3f, 1e3f, 1e3f, 0.f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bytes += __shfl_xor_sync(kFull, bytes, o);
    if (lane == 0) mbar_arrive_expect_tx(&sm.bar[stg], (unsigned)bytes);
}

// One warp task of the mixed tree code.  Returns false if a staging wait gave up (status
// flagged STS_ERR_TIMEOUT after the copies in flight were given a bounded time to land).
// par: the parity bits of the two stage barriers, carried from task to task.
template <int S, bool POT>
__device__ __forceinline__ bool eval_task_mixed(const Task& tk, EvalSmem& sm, int lane, unsigned& par,
                                                int* __restrict__ status,
                                                const int64_t* __restrict__ far_off,
                                                const FarEntry* __restrict__ far_ent,
                                                const int64_t* __restrict__ near_coff,
                                                const NearEntry* __restrict__ near_ent,
                                                const float4* __restrict__ prx32, int M,
                                                const float4* __restrict__ src32, const double4* __restrict__ src64,
                                                const float4* __restrict__ tgt32, const double4* __restrict__ tgt64,
                                                const int32_t* __restrict__ perm, float tau2, float tau_r,
                                                double* __restrict__ corr, double* __restrict__ vel,
                                                int64_t out_base)
{
    const int p = (tk.nt + 1) >> 1;
    const int j = lane % p;
    const int ph = lane < p * S ? lane / p : (1 << 20);
    const int64_t tk0 = tk.t0 + 2 * j, tk1 = tk0 + 1;
    const bool v0 = 2 * j < tk.nt, v1 = 2 * j + 1 < tk.nt;
    float4 q = tgt32[v0 ? tk0 : tk.t0];
    const float t0x = v0 ? q.x : -1e3f, t0y = v0 ? q.y : -1e3f, t0z = v0 ? q.z : -1e3f;
    q = tgt32[v1 ? tk1 : tk.t0];
    const float t1x = v1 ? q.x : -1e3f, t1y = v1 ? q.y : -1e3f, t1z = v1 ? q.z : -1e3f;
    float h0x = 0.f, h0y = 0.f, h0z = 0.f, l0x = 0.f, l0y = 0.f, l0z = 0.f;
    float h1x = 0.f, h1y = 0.f, h1z = 0.f, l1x = 0.f, l1y = 0.f, l1z = 0.f;
    float2 phi = make_float2(0.f, 0.f), plo = make_float2(0.f, 0.f);  // POT: the two targets' sums

    const int64_t fo = far_off[tk.leaf], co = near_coff[tk.leaf];
    const int nf = (int)(far_off[tk.leaf + 1] - fo);
    const int nbt = nf + (int)(near_coff[tk.leaf + 1] - co);
    const FarEntry* fe = far_ent + fo;
    const NearEntry* ne = near_ent + co;

    int wb = 0;
    bool wtest = false;
    int winc = load_window(sm, 0, lane, nf, nbt, fe, ne, M, tau_r, wtest);
    Group cur = form_group(sm, 0, wb, winc, wtest, lane, nf, nbt, fe, ne, M, tau_r);
    issue_group<S>(sm, cur, 0, lane, prx32, src32, M);
    Group nxt = form_group(sm, cur.e1, wb, winc, wtest, lane, nf, nbt, fe, ne, M, tau_r);
    for (int b = 0; cur.e1 > cur.e0; b++) {
        const int stg = b & 1;
        issue_group<S>(sm, nxt, stg ^ 1, lane, prx32, src32, M);
        if (!mbar_wait(&sm.bar[stg], (par >> stg) & 1u)) {
            if (lane == 0) atomicOr(status, kStatusTimeout);
            if (nxt.e1 > nxt.e0) mbar_wait(&sm.bar[stg ^ 1], (par >> (stg ^ 1)) & 1u);
            mbar_wait(&sm.bar[stg], (par >> stg) & 1u);
            return false;
        }
        par ^= 1u << stg;
        float4* st = sm.stage[stg];
        // every source moves into the task leaf's frame: y + delta, delta = c_source - c_leaf
        // (FP32, rounded once per list entry), so that d = (y + delta) - x over the whole group
        for (int f = cur.e0; f < cur.e1; f++) {
            const int4 in = sm.info[f & (kRing - 1)];
            const float4 o = sm.off[f & (kRing - 1)];
            float4* sb = st + (in.w - cur.base);
            for (int k = lane; k < in.y; k += 32) {
                float4 v = sb[k];
                v.x += o.x;
                v.y += o.y;
                v.z += o.z;
                sb[k] = v;
            }
        }
        __syncwarp();  // the moved sources and the padding written by the other lanes
        const int gp = (cur.cnt + 4 * S - 1) / (4 * S) * (4 * S);
        float p0x = 0.f, p0y = 0.f, p0z = 0.f, p1x = 0.f, p1y = 0.f, p1z = 0.f;
        bool hit = false;
        if (POT) {
            if (cur.tested) {
                block_pot<true, S>(st, gp, ph, t0x, t0y, t0z, t1x, t1y, t1z, phi, plo, tau2, hit);
                if (hit) {
                    for (int f = cur.e0; f < cur.e1; f++) {
                        const int4 in = sm.info[f & (kRing - 1)];
                        const int b0 = in.w - cur.base;
                        int i0 = (ph - b0) % S;
                        if (i0 < 0) i0 += S;
                        block_close_pot<S>(st + b0, in.y, i0, t0x, t0y, t0z, t1x, t1y, t1z, tau2, in.x, tk0, tk1,
                                           src64, tgt64, corr);
                    }
                }
            } else {
                block_pot<false, S>(st, gp, ph, t0x, t0y, t0z, t1x, t1y, t1z, phi, plo, tau2, hit);
            }
        } else if (cur.tested) {
            block_pairs<true, S>(st, gp, ph, t0x, t0y, t0z, t1x, t1y, t1z, p0x, p0y, p0z, p1x, p1y, p1z, tau2,
                                 hit);
            if (hit) {
                // the pairs left out above, in FP64; stage entry q belongs to phase q mod S
                for (int f = cur.e0; f < cur.e1; f++) {
                    const int4 in = sm.info[f & (kRing - 1)];
                    const int b0 = in.w - cur.base;
                    int i0 = (ph - b0) % S;
                    if (i0 < 0) i0 += S;
                    block_close_pairs<S>(st + b0, in.y, i0, t0x, t0y, t0z, t1x, t1y, t1z, tau2, in.x, tk0, tk1,
                                         src64, tgt64, corr);
                }
            }
        } else {
            block_pairs<false, S>(st, gp, ph, t0x, t0y, t0z, t1x, t1y, t1z, p0x, p0y, p0z, p1x, p1y, p1z, tau2,
                                  hit);
        }
        two_sum_add(h0x, l0x, p0x);
        two_sum_add(h0y, l0y, p0y);
        two_sum_add(h0z, l0z, p0z);
        two_sum_add(h1x, l1x, p1x);
        two_sum_add(h1y, l1y, p1y);
        two_sum_add(h1z, l1z, p1z);
        __syncwarp();
        cur = nxt;
        nxt = form_group(sm, cur.e1, wb, winc, wtest, lane, nf, nbt, fe, ne, M, tau_r);
    }
    double a[6] = {(double)h0x + (double)l0x, (double)h0y + (double)l0y, (double)h0z + (double)l0z,
                   (double)h1x + (double)l1x, (double)h1y + (double)l1y, (double)h1z + (double)l1z};
    if (POT) {
        a[0] = (double)phi.x + (double)plo.x;
        a[3] = (double)phi.y + (double)plo.y;
    }
#pragma unroll
    for (int s2 = 1; s2 < S; s2++) {
        const int src = (lane + s2 * p) & 31;
#pragma unroll
        for (int c = 0; c < 6; c++) {
            const double v = __shfl_sync(kFull, a[c], src);
            if (lane < p) a[c] += v;
        }
    }
    __syncwarp();
    if (POT) {
        // psi = -(1/4 pi) sum w log(|d|^2 / 2) = -(1/8 pi) (ln 2 sum 2w log2(.) + the FP64 close pairs)
        if (lane < p) {
#pragma unroll
            for (int u = 0; u < 2; u++) {
                const int64_t t = u == 0 ? tk0 : tk1;
                if (!(u == 0 ? v0 : v1)) continue;
                double acc = kLn2 * a[3 * u];
                if (corr) acc += __ldcg(corr + t);
                const int64_t i = out_base >= 0 ? t - out_base : (int64_t)perm[t];
                vel[i] = -0.5 * kInv4Pi * acc;
            }
        }
        return true;
    }
    if (lane < p) {
#pragma unroll
        for (int u = 0; u < 2; u++) {
            const int64_t t = u == 0 ? tk0 : tk1;
            if (!(u == 0 ? v0 : v1)) continue;
            double Sx = a[3 * u], Sy = a[3 * u + 1], Sz = a[3 * u + 2];
            if (corr) {
                Sx += __ldcg(corr + 3 * t);
                Sy += __ldcg(corr + 3 * t + 1);
                Sz += __ldcg(corr + 3 * t + 2);
            }
            if (!perm) {  // proxy targets of the dual traversal: the kernel sum, -(1/4 pi) S
                vel[3 * t] = -kInv4Pi * Sx;
                vel[3 * t + 1] = -kInv4Pi * Sy;
                vel[3 * t + 2] = -kInv4Pi * Sz;
                continue;
            }
            const double4 x = tgt64[t];
            const int64_t i = out_base >= 0 ? t - out_base : (int64_t)perm[t];
            vel[3 * i] = -kInv4Pi * (x.y * Sz - x.z * Sy);
            vel[3 * i + 1] = -kInv4Pi * (x.z * Sx - x.x * Sz);
            vel[3 * i + 2] = -kInv4Pi * (x.x * Sy - x.y * Sx);
        }
    }
    return true;
}

template <bool POT>
__global__ void __launch_bounds__(kEvalWarps * 32, STS_EVAL_MIN_BLOCKS)
k_eval_mixed(const Task* __restrict__ tasks, const int64_t* __restrict__ far_off,
             const FarEntry* __restrict__ far_ent, const int64_t* __restrict__ near_coff,
             const NearEntry* __restrict__ near_ent, const float4* __restrict__ prx32, int M,
             const float4* __restrict__ src32, const double4* __restrict__ src64,
             const float4* __restrict__ tgt32, const double4* __restrict__ tgt64,
             const int32_t* __restrict__ perm, float tau2, float tau_r, double* __restrict__ corr,
             double* __restrict__ vel, const int64_t* __restrict__ ntasks_d, int64_t cap,
             unsigned long long* __restrict__ queue, int* __restrict__ status, const int64_t* __restrict__ over,
             EvalRange rg)
{
    extern __shared__ __align__(16) EvalSmem sbuf[];  // kEvalWarps of them
    // a recorded step whose lists outgrew their capacities evaluates nothing (the host redoes it)
    if (*over) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t nt = min(*ntasks_d, cap);  // a recorded step whose tasks overflowed is redone
    if (lane == 0) {
        mbar_init(&sbuf[w].bar[0], 1);
        mbar_init(&sbuf[w].bar[1], 1);
        mbar_init_fence();
    }
    __syncwarp();
    unsigned par = 0;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(queue, 1ull);
        const int64_t ti = (int64_t)__shfl_sync(kFull, t, 0);
        if (ti >= nt) break;
        const Task tk = tasks[ti];
        if (tk.leaf < rg.leaf_lo || tk.leaf >= rg.leaf_hi) continue;
        bool ok;
        switch (tk.S) {
            case 1:
                ok = eval_task_mixed<1, POT>(tk, sbuf[w], lane, par, status, far_off, far_ent, near_coff, near_ent, prx32,
                                         M, src32, src64, tgt32, tgt64, perm, tau2, tau_r, corr, vel, rg.out_base);
                break;
            case 2:
                ok = eval_task_mixed<2, POT>(tk, sbuf[w], lane, par, status, far_off, far_ent, near_coff, near_ent, prx32,
                                         M, src32, src64, tgt32, tgt64, perm, tau2, tau_r, corr, vel, rg.out_base);
                break;
            case 3:
                ok = eval_task_mixed<3, POT>(tk, sbuf[w], lane, par, status, far_off, far_ent, near_coff, near_ent, prx32,
                                         M, src32, src64, tgt32, tgt64, perm, tau2, tau_r, corr, vel, rg.out_base);
                break;
            case 4:
                ok = eval_task_mixed<4, POT>(tk, sbuf[w], lane, par, status, far_off, far_ent, near_coff, near_ent, prx32,
                                         M, src32, src64, tgt32, tgt64, perm, tau2, tau_r, corr, vel, rg.out_base);
                break;
            case 5:
                ok = eval_task_mixed<5, POT>(tk, sbuf[w], lane, par, status, far_off, far_ent, near_coff, near_ent, prx32,
                                         M, src32, src64, tgt32, tgt64, perm, tau2, tau_r, corr, vel, rg.out_base);
                break;
            case 6:
                ok = eval_task_mixed<6, POT>(tk, sbuf[w], lane, par, status, far_off, far_ent, near_coff, near_ent, prx32,
                                         M, src32, src64, tgt32, tgt64, perm, tau2, tau_r, corr, vel, rg.out_base);
                break;
            case 7:
                ok = eval_task_mixed<7, POT>(tk, sbuf[w], lane, par, status, far_off, far_ent, near_coff, near_ent, prx32,
                                         M, src32, src64, tgt32, tgt64, perm, tau2, tau_r, corr, vel, rg.out_base);
                break;
            default:
                ok = eval_task_mixed<8, POT>(tk, sbuf[w], lane, par, status, far_off, far_ent, near_coff, near_ent, prx32,
                                         M, src32, src64, tgt32, tgt64, perm, tau2, tau_r, corr, vel, rg.out_base);
                break;
        }
        if (!ok) break;
        __syncwarp();
    }
}

// ------------------------------------------------------------------------ FP64 tree
template <bool POT>
__device__ __forceinline__ void eval_task_fp64(const Task& tk, double4* sb, int lane,
                                               const int64_t* __restrict__ far_off,
                                               const FarEntry* __restrict__ far_ent,
                                               const int64_t* __restrict__ near_coff,
                                               const NearEntry* __restrict__ near_ent,
                                               const double4* __restrict__ prx64, int M,
                                               const double4* __restrict__ src64, const double4* __restrict__ tgt64,
                                               const int32_t* __restrict__ perm, double* __restrict__ vel,
                                               int64_t out_base = -1)
{
    const int p = (tk.nt + 1) >> 1, S = tk.S;
    const int j = lane % p;
    const int ph = lane < p * S ? lane / p : (1 << 20);
    const int64_t tk0 = tk.t0 + 2 * j, tk1 = tk0 + 1;
    const bool v0 = 2 * j < tk.nt, v1 = 2 * j + 1 < tk.nt;
    const double4 x0 = tgt64[v0 ? tk0 : tk.t0], x1 = tgt64[v1 ? tk1 : tk.t0];
    const double ax = v0 ? x0.x : -1e3, ay = v0 ? x0.y : -1e3, az = v0 ? x0.z : -1e3;
    const double bx = v1 ? x1.x : -1e3, by = v1 ? x1.y : -1e3, bz = v1 ? x1.z : -1e3;
    double a[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    const int64_t fo = far_off[tk.leaf], co = near_coff[tk.leaf];
    const int nf = (int)(far_off[tk.leaf + 1] - fo);
    const int nbt = nf + (int)(near_coff[tk.leaf + 1] - co);
    for (int b = 0; b < nbt; b++) {
        const double4* src;
        int cnt;
        if (b < nf) {
            src = prx64 + (int64_t)far_ent[fo + b].slot * M;
            cnt = M;
        } else {
            const NearEntry e = near_ent[co + b - nf];
            src = src64 + e.start;
            cnt = e.count;
        }
        __syncwarp();
        for (int i = lane; i < cnt; i += 32) sb[i] = src[i];
        __syncwarp();
#pragma unroll 2
        for (int i = ph; i < cnt; i += S) {
            const double4 sv = sb[i];
            if (POT) {
                pot64(sv, ax, ay, az, a[0]);
                pot64(sv, bx, by, bz, a[3]);
            } else {
                pair64(sv, ax, ay, az, a[0], a[1], a[2]);
                pair64(sv, bx, by, bz, a[3], a[4], a[5]);
            }
        }
    }
    for (int s2 = 1; s2 < S; s2++) {
        const int src = (lane + s2 * p) & 31;
#pragma unroll
        for (int c = 0; c < 6; c++) {
            const double v = __shfl_sync(kFull, a[c], src);
            if (lane < p) a[c] += v;
        }
    }
    if (POT) {
        // psi = -(1/4 pi) sum w log(|d|^2 / 2), accumulated with 2 w
        if (lane < p && v0) vel[perm[tk0]] = -0.5 * kInv4Pi * a[0];
        if (lane < p && v1) vel[perm[tk1]] = -0.5 * kInv4Pi * a[3];
    } else if (lane < p && !perm) {  // proxy targets of the dual traversal: -(1/4 pi) S
        if (v0)
            for (int c = 0; c < 3; c++) vel[3 * tk0 + c] = -kInv4Pi * a[c];
        if (v1)
            for (int c = 0; c < 3; c++) vel[3 * tk1 + c] = -kInv4Pi * a[3 + c];
    } else if (lane < p) {
        if (v0) {
            const int64_t i = out_base >= 0 ? tk0 - out_base : (int64_t)perm[tk0];
            vel[3 * i] = -kInv4Pi * (x0.y * a[2] - x0.z * a[1]);
            vel[3 * i + 1] = -kInv4Pi * (x0.z * a[0] - x0.x * a[2]);
            vel[3 * i + 2] = -kInv4Pi * (x0.x * a[1] - x0.y * a[0]);
        }
        if (v1) {
            const int64_t i = out_base >= 0 ? tk1 - out_base : (int64_t)perm[tk1];
            vel[3 * i] = -kInv4Pi * (x1.y * a[5] - x1.z * a[4]);
            vel[3 * i + 1] = -kInv4Pi * (x1.z * a[3] - x1.x * a[5]);
            vel[3 * i + 2] = -kInv4Pi * (x1.x * a[4] - x1.y * a[3]);
        }
    }
    __syncwarp();
}

// Next task of a persistent warp: lane 0 takes the queue's next index, all lanes receive it.
__device__ __forceinline__ int64_t next_task(unsigned long long* queue, int lane)
{
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(queue, 1ull);
    return (int64_t)__shfl_sync(kFull, t, 0);
}

// Persistent warps: each warp takes tasks from the queue until it runs dry.  POT: the
// potential kernel (vel then receives psi[n]).
template <bool POT>
__global__ void __launch_bounds__(kEvalWarps64 * 32)
k_eval_fp64(const Task* __restrict__ tasks, const int64_t* __restrict__ far_off,
            const FarEntry* __restrict__ far_ent, const int64_t* __restrict__ near_coff,
            const NearEntry* __restrict__ near_ent, const double4* __restrict__ prx64, int M,
            const double4* __restrict__ src64, const double4* __restrict__ tgt64, const int32_t* __restrict__ perm,
            double* __restrict__ vel, const int64_t* __restrict__ ntasks_d, int64_t cap,
            unsigned long long* __restrict__ queue, const int64_t* __restrict__ over, EvalRange rg)
{
    __shared__ double4 sbuf[kEvalWarps64][kStage];
    if (*over) return;  // lists past their recorded capacities: the host redoes the step
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t nt = min(*ntasks_d, cap);
    for (int64_t ti = next_task(queue, lane); ti < nt; ti = next_task(queue, lane)) {
        const Task tk = tasks[ti];
        if (tk.leaf < rg.leaf_lo || tk.leaf >= rg.leaf_hi) continue;
        eval_task_fp64<POT>(tk, sbuf[w], lane, far_off, far_ent, near_coff, near_ent, prx64, M, src64, tgt64,
                            perm, vel, rg.out_base);
    }
}

// Per-leaf work of the target-leaf lists: targets x (far entries x M + near sources), the PC +
// PP interactions of each depth-first leaf (the self pair included).
__global__ void k_leaf_work(const int64_t* __restrict__ nleaves_p, const int32_t* __restrict__ leaves,
                            const int32_t* __restrict__ count, const int64_t* __restrict__ far_off,
                            const int64_t* __restrict__ near_coff, const NearEntry* __restrict__ near_ent, int M,
                            int64_t* __restrict__ work)
{
    const int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (L >= *nleaves_p) return;
    int64_t ns = 0;
    for (int64_t q = near_coff[L]; q < near_coff[L + 1]; q++) ns += near_ent[q].count;
    work[L] = (int64_t)count[leaves[L]] * ((int64_t)M * (far_off[L + 1] - far_off[L]) + ns);
}

// vel[perm[t]] = vs[t]: rows in sorted slot order back to the caller's order.
__global__ void k_unpermute(const double* __restrict__ vs, const int32_t* __restrict__ perm, int64_t n,
                            double* __restrict__ vel)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int64_t i = perm[t];
    vel[3 * i] = vs[3 * t];
    vel[3 * i + 1] = vs[3 * t + 1];
    vel[3 * i + 2] = vs[3 * t + 2];
}

// ------------------------------------------------------------------------ counts
__global__ void k_count(const int64_t* __restrict__ nleaves_p, const int32_t* __restrict__ leaves,
                        const int32_t* __restrict__ count, const int64_t* __restrict__ far_off,
                        const int64_t* __restrict__ near_coff, const NearEntry* __restrict__ near_ent,
                        int M, unsigned long long* __restrict__ stats)
{
    const int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (L >= *nleaves_p) return;
    const unsigned long long nl = (unsigned long long)count[leaves[L]];
    const unsigned long long pc = nl * (unsigned long long)M * (unsigned long long)(far_off[L + 1] - far_off[L]);
    unsigned long long ns = 0;
    for (int64_t q = near_coff[L]; q < near_coff[L + 1]; q++) ns += (unsigned long long)near_ent[q].count;
    atomicAdd(&stats[0], pc);
    atomicAdd(&stats[1], nl * (ns - 1ull));
}

// ------------------------------------------------------------------------ direct sum
constexpr int kDirT = 128;

__global__ void k_direct_prep(const double* __restrict__ pos, const double* __restrict__ zeta,
                              const double* __restrict__ area, int64_t n, double4* __restrict__ s64,
                              float4* __restrict__ s32)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const double x = pos[3 * j], y = pos[3 * j + 1], z = pos[3 * j + 2];
    const double w2 = 2.0 * (zeta[j] * area[j]);
    s64[j] = make_double4(x, y, z, w2);
    const float hx = (float)x, hy = (float)y, hz = (float)z;
    s32[2 * j] = make_float4(hx, hy, hz, (float)w2);
    s32[2 * j + 1] = make_float4((float)(x - (double)hx), (float)(y - (double)hy), (float)(z - (double)hz), 0.f);
}

__global__ void __launch_bounds__(kDirT)
k_direct_fp64(const double4* __restrict__ s64, int64_t n, const int64_t* __restrict__ targets,
              int64_t nt, int64_t chunk, double* __restrict__ part)
{
    __shared__ double4 sb[kDirT];
    const int64_t t = (int64_t)blockIdx.x * kDirT + threadIdx.x;
    const bool valid = t < nt;
    const int64_t i = valid ? (targets ? targets[t] : t) : 0;
    const double4 x = s64[i];
    const double tx = valid ? x.x : -1e3, ty = valid ? x.y : -1e3, tz = valid ? x.z : -1e3;
    const int64_t j0 = (int64_t)blockIdx.y * chunk, j1 = min(n, j0 + chunk);
    double ax = 0.0, ay = 0.0, az = 0.0;
    for (int64_t b = j0; b < j1; b += kDirT) {
        __syncthreads();
        const int64_t j = b + threadIdx.x;
        sb[threadIdx.x] = j < j1 ? s64[j] : make_double4(1e3, 1e3, 1e3, 0.0);
        __syncthreads();
#pragma unroll 4
        for (int q = 0; q < kDirT; q++) pair64(sb[q], tx, ty, tz, ax, ay, az);
    }
    if (valid) {
        double* o = part + 3 * ((int64_t)blockIdx.y * nt + t);
        o[0] = ax;
        o[1] = ay;
        o[2] = az;
    }
}

// Mixed direct sum: positions carried as FP32 hi + lo pairs, d = (y_hi - x_hi) + (y_lo -
// x_lo), so d keeps FP32 relative accuracy for close pairs without any tree frame.
__global__ void __launch_bounds__(kDirT)
k_direct_mixed(const float4* __restrict__ s32, int64_t n, const int64_t* __restrict__ targets,
               int64_t nt, int64_t chunk, double* __restrict__ part)
{
    __shared__ float4 sh[kDirT], sl[kDirT];
    const int64_t t = (int64_t)blockIdx.x * kDirT + threadIdx.x;
    const bool valid = t < nt;
    const int64_t i = valid ? (targets ? targets[t] : t) : 0;
    const float4 xh = s32[2 * i], xl = s32[2 * i + 1];
    const float hx = valid ? xh.x : -1e3f, hy = valid ? xh.y : -1e3f, hz = valid ? xh.z : -1e3f;
    const int64_t j0 = (int64_t)blockIdx.y * chunk, j1 = min(n, j0 + chunk);
    float Hx = 0.f, Hy = 0.f, Hz = 0.f, Lx = 0.f, Ly = 0.f, Lz = 0.f;
    for (int64_t b = j0; b < j1; b += kDirT) {
        __syncthreads();
        const int64_t j = b + threadIdx.x;
        if (j < j1) {
            sh[threadIdx.x] = s32[2 * j];
            sl[threadIdx.x] = s32[2 * j + 1];
        } else {
            sh[threadIdx.x] = make_float4(1e3f, 1e3f, 1e3f, 0.f);
            sl[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        float px = 0.f, py = 0.f, pz = 0.f;
#pragma unroll 4
        for (int q = 0; q < kDirT; q++) {
            const float4 a = sh[q], l = sl[q];
            const float dx = (a.x - hx) + (l.x - xl.x);
            const float dy = (a.y - hy) + (l.y - xl.y);
            const float dz = (a.z - hz) + (l.z - xl.z);
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, kEps)));
            const float c = a.w * rcp_approx(r2);
            px = fmaf(c, dx, px);
            py = fmaf(c, dy, py);
            pz = fmaf(c, dz, pz);
        }
        two_sum_add(Hx, Lx, px);
        two_sum_add(Hy, Ly, py);
        two_sum_add(Hz, Lz, pz);
    }
    if (valid) {
        double* o = part + 3 * ((int64_t)blockIdx.y * nt + t);
        o[0] = (double)Hx + (double)Lx;
        o[1] = (double)Hy + (double)Ly;
        o[2] = (double)Hz + (double)Lz;
    }
}

__global__ void k_direct_finish(const double* __restrict__ part, int splits, int64_t nt,
                                const int64_t* __restrict__ targets, const double4* __restrict__ s64,
                                double* __restrict__ vel)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    double Sx = 0.0, Sy = 0.0, Sz = 0.0;
    for (int s = 0; s < splits; s++) {
        const double* o = part + 3 * ((int64_t)s * nt + t);
        Sx += o[0];
        Sy += o[1];
        Sz += o[2];
    }
    const double4 x = s64[targets ? targets[t] : t];
    vel[3 * t] = -kInv4Pi * (x.y * Sz - x.z * Sy);
    vel[3 * t + 1] = -kInv4Pi * (x.z * Sx - x.x * Sz);
    vel[3 * t + 2] = -kInv4Pi * (x.x * Sy - x.y * Sx);
}

// Direct sum of the potential (FP64), same tiling as k_direct_fp64: partial sums of 2 w
// log(|d|^2 / 2) per (target, source chunk).
__global__ void __launch_bounds__(kDirT)
k_direct_pot_fp64(const double4* __restrict__ s64, int64_t n, const int64_t* __restrict__ targets,
                  int64_t nt, int64_t chunk, double* __restrict__ part)
{
    __shared__ double4 sb[kDirT];
    const int64_t t = (int64_t)blockIdx.x * kDirT + threadIdx.x;
    const bool valid = t < nt;
    const int64_t i = valid ? (targets ? targets[t] : t) : 0;
    const double4 x = s64[i];
    const double tx = valid ? x.x : -1e3, ty = valid ? x.y : -1e3, tz = valid ? x.z : -1e3;
    const int64_t j0 = (int64_t)blockIdx.y * chunk, j1 = min(n, j0 + chunk);
    double acc = 0.0;
    for (int64_t b = j0; b < j1; b += kDirT) {
        __syncthreads();
        const int64_t j = b + threadIdx.x;
        sb[threadIdx.x] = j < j1 ? s64[j] : make_double4(1e3, 1e3, 1e3, 0.0);
        __syncthreads();
#pragma unroll 4
        for (int q = 0; q < kDirT; q++) pot64(sb[q], tx, ty, tz, acc);
    }
    if (valid) part[(int64_t)blockIdx.y * nt + t] = acc;
}

__global__ void k_direct_pot_finish(const double* __restrict__ part, int splits, int64_t nt,
                                    double* __restrict__ psi)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    double S = 0.0;
    for (int s = 0; s < splits; s++) S += part[(int64_t)s * nt + t];
    psi[t] = -0.5 * kInv4Pi * S;
}

}  // namespace

int direct_potential(sts_ctx* c, const double* pos, const double* zeta, const double* area, int64_t n,
                     double* psi, cudaStream_t s)
{
    const int64_t nt = n;
    if (nt == 0) return STS_OK;
    STS_CUDA(c->dsrc64.reserve(n + 1));
    STS_CUDA(c->dsrc32.reserve(2 * n + 2));
    const int64_t ntb = (nt + kDirT - 1) / kDirT;
    int64_t splits = (4 * (int64_t)c->num_sms + ntb - 1) / ntb;
    splits = std::max<int64_t>(1, std::min<int64_t>(splits, std::max<int64_t>(1, n / 1024)));
    splits = std::min<int64_t>(splits, 256);
    const int64_t chunk = ((n + splits - 1) / splits + kDirT - 1) / kDirT * kDirT;
    splits = std::max<int64_t>(1, (n + chunk - 1) / chunk);
    STS_CUDA(c->dpart.reserve(splits * nt + 1));
    phase_begin(c, kPhDirect, s);
    (k_direct_prep<<<blocks(n, 256), 256, 0, s>>>(pos, zeta, area, n, c->dsrc64.p, c->dsrc32.p), note_launch());
    (k_direct_pot_fp64<<<dim3((unsigned)ntb, (unsigned)splits), kDirT, 0, s>>>(c->dsrc64.p, n, nullptr, nt, chunk,
                                                                                c->dpart.p), note_launch());
    (k_direct_pot_finish<<<blocks(nt, 256), 256, 0, s>>>(c->dpart.p, (int)splits, nt, psi), note_launch());
    phase_end(c, kPhDirect, s);
    STS_LAUNCH_CHECK();
    return STS_OK;
}

namespace {
int eval_blocks(sts_ctx* c);
}  // namespace

int evaluate_potential(sts_ctx* c, int degree, int precision, double tau, double* psi, cudaStream_t s)
{
    const int M = nbasis(degree);
    const int64_t ntasks = c->capturing ? (int64_t)c->tasks.cap : c->ntasks;
    if (ntasks <= 0) return STS_OK;
    int rc = eval_blocks(c);
    if (rc) return rc;
    unsigned long long* queue = (unsigned long long*)(c->dc.p + kDcQueue);
    STS_CUDA(cudaMemsetAsync(queue, 0, sizeof(unsigned long long), s));
    if (precision == STS_FP64) {
        const unsigned g = (unsigned)std::min<int64_t>(blocks(ntasks, kEvalWarps64), c->eval_blocks_fp64);
        phase_begin(c, kPhEval, s);
        (k_eval_fp64<true><<<g, kEvalWarps64 * 32, 0, s>>>(c->tasks.p, c->far_off.p, c->far_ent.p, c->near_coff.p,
                                                           c->near_ent.p, c->prx64.p, M, c->src64.p, c->src64.p,
                                                           c->perm.p, psi, c->dc.p + kDcTasks, ntasks, queue,
                                                           c->dc.p + kDcOver, EvalRange{0, INT64_MAX, -1}),
         note_launch());
        phase_end(c, kPhEval, s);
    } else {
        // mixed: the FP32 log terms (compensated sums) with the close pairs below tau in FP64,
        // as the velocity (one correction per target).  The log has no finite value at
        // coincident points (a target and itself, duplicates), so a tau of at least 1e-20 always
        // sends those pairs to the FP64 pass, which leaves them out
        tau = std::min(std::max(tau, 1e-20), 2.0);
        if (!c->capturing) STS_CUDA(c->corr.reserve(3 * c->n + 3));
        STS_CUDA(cudaMemsetAsync(c->corr.p, 0, c->n * sizeof(double), s));
        double* corr = c->corr.p;
        const float tau2 = (float)(2.0 * tau);
        const float tau_r = (float)(sqrt(2.0 * tau) * (1.0 + 1e-3) + 1e-6);
        const unsigned g = (unsigned)std::min<int64_t>(blocks(ntasks, kEvalWarps), c->eval_blocks_mixed);
        phase_begin(c, kPhEval, s);
        (k_eval_mixed<true><<<g, kEvalWarps * 32, kEvalWarps * sizeof(EvalSmem), s>>>(
             c->tasks.p, c->far_off.p, c->far_ent.p, c->near_coff.p, c->near_ent.p, c->prx32.p, M, c->src32.p,
             c->src64.p, c->src32.p, c->src64.p, c->perm.p, tau2, tau_r, corr, psi, c->dc.p + kDcTasks, ntasks,
             queue, c->d_status, c->dc.p + kDcOver, EvalRange{0, INT64_MAX, -1}),
         note_launch());
        phase_end(c, kPhEval, s);
    }
    STS_LAUNCH_CHECK();
    return STS_OK;
}

namespace {


int eval_blocks(sts_ctx* c)
{
    if (c->eval_blocks_mixed > 0) return STS_OK;
    // persistent grids: as many blocks as stay resident on all SMs at once
    int b32 = 0, b64 = 0;
    STS_CUDA(cudaFuncSetAttribute(k_eval_mixed<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(kEvalWarps * sizeof(EvalSmem))));
    STS_CUDA(cudaFuncSetAttribute(k_eval_mixed<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(kEvalWarps * sizeof(EvalSmem))));
    STS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b32, k_eval_mixed<false>, kEvalWarps * 32,
                                                           kEvalWarps * sizeof(EvalSmem)));
    STS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b64, k_eval_fp64<false>, kEvalWarps64 * 32, 0));
    c->eval_blocks_mixed = std::max(1, c->num_sms * b32);
    c->eval_blocks_fp64 = std::max(1, c->num_sms * b64);
    return STS_OK;
}

}  // namespace

// corr: FP64 close-pair scratch of at least 3 * ls.ntargets doubles (mixed precision).
int evaluate_lists(sts_ctx* c, const ListSet& ls, int degree, int precision, double tau, DevBuf<double>& corrbuf,
                   double* vel, cudaStream_t s, int phase)
{
    const int M = nbasis(degree);
    if (ls.ntasks <= 0) return STS_OK;
    unsigned long long* queue = (unsigned long long*)(c->dc.p + kDcQueue);
    int rc = eval_blocks(c);
    if (rc) return rc;
    STS_CUDA(cudaMemsetAsync(queue, 0, sizeof(unsigned long long), s));
    if (precision == STS_FP64) {
        const unsigned g = (unsigned)std::min<int64_t>(blocks(ls.ntasks, kEvalWarps64), c->eval_blocks_fp64);
        phase_begin(c, phase, s);
        (k_eval_fp64<false><<<g, kEvalWarps64 * 32, 0, s>>>(ls.tasks, ls.far_off, ls.far_ent, ls.near_coff,
                                                            ls.near_ent, c->prx64.p, M, c->src64.p, ls.tgt64,
                                                            ls.perm, vel, ls.ntasks_d, ls.ntasks, queue,
                                                            c->dc.p + kDcOver,
                                                            EvalRange{ls.leaf_lo, ls.leaf_hi, ls.out_base}),
         note_launch());
        phase_end(c, phase, s);
    } else {
        double* corr = nullptr;
        // |x - y|^2 / 2 <= 2 on the unit sphere: larger tau changes nothing, and the bound keeps
        // the dummy targets of idle lanes (at distance ~1e3) out of the FP64 path
        tau = std::min(tau, 2.0);
        if (tau > 0.0) {
            if (!c->capturing) STS_CUDA(corrbuf.reserve(3 * ls.ntargets + 3));
            STS_CUDA(cudaMemsetAsync(corrbuf.p, 0, 3 * ls.ntargets * sizeof(double), s));
            corr = corrbuf.p;
        }
        // FP32 threshold on |d|^2 and the distance bound below which a near block is tested
        const float tau2 = corr ? (float)(2.0 * tau) : 0.f;
        const float tau_r = corr ? (float)(sqrt(2.0 * tau) * (1.0 + 1e-3) + 1e-6) : -1.f;
        const unsigned g = (unsigned)std::min<int64_t>(blocks(ls.ntasks, kEvalWarps), c->eval_blocks_mixed);
        phase_begin(c, phase, s);
        (k_eval_mixed<false><<<g, kEvalWarps * 32, kEvalWarps * sizeof(EvalSmem), s>>>(
             ls.tasks, ls.far_off, ls.far_ent, ls.near_coff, ls.near_ent, c->prx32.p, M, c->src32.p, c->src64.p,
             ls.tgt32, ls.tgt64, ls.perm, tau2, tau_r, corr, vel, ls.ntasks_d, ls.ntasks, queue, c->d_status,
             c->dc.p + kDcOver, EvalRange{ls.leaf_lo, ls.leaf_hi, ls.out_base}),
         note_launch());
        phase_end(c, phase, s);
    }
    STS_LAUNCH_CHECK();
    return STS_OK;
}

int evaluate(sts_ctx* c, int degree, int precision, double tau, double* vel, cudaStream_t s)
{
    ListSet ls;
    ls.tasks = c->tasks.p;
    ls.ntasks_d = c->dc.p + kDcTasks;
    ls.ntasks = c->capturing ? (int64_t)c->tasks.cap : c->ntasks;
    ls.far_off = c->far_off.p;
    ls.near_coff = c->near_coff.p;
    ls.far_ent = c->far_ent.p;
    ls.near_ent = c->near_ent.p;
    ls.tgt32 = c->src32.p;
    ls.tgt64 = c->src64.p;
    ls.perm = c->perm.p;
    ls.ntargets = c->n;
    return evaluate_lists(c, ls, degree, precision, tau, c->corr, vel, s);
}

int evaluate_range(sts_ctx* c, int degree, int precision, double tau, int64_t leaf_lo, int64_t leaf_hi,
                   int64_t out_base, double* vel, cudaStream_t s)
{
    ListSet ls;
    ls.tasks = c->tasks.p;
    ls.ntasks_d = c->dc.p + kDcTasks;
    ls.ntasks = c->ntasks;
    ls.far_off = c->far_off.p;
    ls.near_coff = c->near_coff.p;
    ls.far_ent = c->far_ent.p;
    ls.near_ent = c->near_ent.p;
    ls.tgt32 = c->src32.p;
    ls.tgt64 = c->src64.p;
    ls.perm = c->perm.p;
    ls.ntargets = c->n;
    ls.leaf_lo = leaf_lo;
    ls.leaf_hi = leaf_hi;
    ls.out_base = out_base;
    return evaluate_lists(c, ls, degree, precision, tau, c->corr, vel, s);
}

int leaf_work(sts_ctx* c, int degree, int64_t* work, cudaStream_t s)
{
    const int64_t L = c->nleaves;
    if (L <= 0) return STS_OK;
    STS_CUDA(c->d_work.reserve(L));
    (k_leaf_work<<<blocks(L, 128), 128, 0, s>>>(c->dc.p + kDcLeaves, c->leaves.p, c->nd_count.p, c->far_off.p,
                                                c->near_coff.p, c->near_ent.p, nbasis(degree), c->d_work.p),
     note_launch());
    STS_LAUNCH_CHECK();
    STS_CUDA(cudaMemcpyAsync(work, c->d_work.p, L * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    STS_CUDA(cudaStreamSynchronize(s));
    return STS_OK;
}

int unpermute(sts_ctx* c, const double* vs, double* vel, cudaStream_t s)
{
    if (c->n <= 0) return STS_OK;
    (k_unpermute<<<blocks(c->n, 256), 256, 0, s>>>(vs, c->perm.p, c->n, vel), note_launch());
    STS_LAUNCH_CHECK();
    return STS_OK;
}

int wait_selftest(sts_ctx* c, int spins, cudaStream_t s)
{
    (k_wait_selftest<<<1, 32, 0, s>>>(spins, c->d_status), note_launch());
    STS_LAUNCH_CHECK();
    return STS_OK;
}

int count_interactions(sts_ctx* c, int degree, cudaStream_t s)
{
    STS_CUDA(c->d_stats.reserve(2));
    STS_CUDA(cudaMemsetAsync(c->d_stats.p, 0, 2 * sizeof(unsigned long long), s));
    const int64_t L = c->nleaves > 0 ? c->nleaves : c->n;
    if (L > 0)
        (k_count<<<blocks(L, 128), 128, 0, s>>>(c->dc.p + kDcLeaves, c->leaves.p, c->nd_count.p, c->far_off.p,
                                               c->near_coff.p, c->near_ent.p, nbasis(degree), c->d_stats.p),
         note_launch());
    STS_LAUNCH_CHECK();
    return STS_OK;
}

int direct_sum(sts_ctx* c, const double* pos, const double* zeta, const double* area, int64_t n,
               const int64_t* targets, int64_t nt, int precision, double* vel, cudaStream_t s)
{
    if (nt == 0) return STS_OK;
    STS_CUDA(c->dsrc64.reserve(n + 1));
    STS_CUDA(c->dsrc32.reserve(2 * n + 2));
    const int64_t ntb = (nt + kDirT - 1) / kDirT;
    int64_t splits = (4 * 152 + ntb - 1) / ntb;
    splits = std::max<int64_t>(1, std::min<int64_t>(splits, std::max<int64_t>(1, n / 1024)));
    splits = std::min<int64_t>(splits, 256);
    const int64_t chunk = ((n + splits - 1) / splits + kDirT - 1) / kDirT * kDirT;
    splits = (n + chunk - 1) / chunk;
    if (splits < 1) splits = 1;
    STS_CUDA(c->dpart.reserve(3 * splits * nt + 3));
    phase_begin(c, kPhDirect, s);
    (k_direct_prep<<<blocks(n, 256), 256, 0, s>>>(pos, zeta, area, n, c->dsrc64.p, c->dsrc32.p), note_launch());
    const dim3 grid((unsigned)ntb, (unsigned)splits);
    if (precision == STS_FP64)
        (k_direct_fp64<<<grid, kDirT, 0, s>>>(c->dsrc64.p, n, targets, nt, chunk, c->dpart.p), note_launch());
    else
        (k_direct_mixed<<<grid, kDirT, 0, s>>>(c->dsrc32.p, n, targets, nt, chunk, c->dpart.p), note_launch());
    (k_direct_finish<<<blocks(nt, 256), 256, 0, s>>>(c->dpart.p, (int)splits, nt, targets, c->dsrc64.p, vel), note_launch());
    phase_end(c, kPhDirect, s);
    STS_LAUNCH_CHECK();
    return STS_OK;
}

}  // namespace sts

// ---------------------------------------------------------------------------------------
// Direct sum without any allocation (sts_direct_noalloc).
//
// Some callers cannot call cudaMalloc at the time they need a result: code that records
// into a CUDA graph it does not own, processes whose device memory is already handed to
// another allocator (a framework's caching allocator), and latency-critical loops that
// must not enter the allocator after start-up (cudaMalloc and cudaFree can synchronise the
// device and take unbounded time).  For them the direct sum takes its scratch from one
// file-scope device array of fixed size instead of the context's growable buffers.  The
// array is part of the loaded module, so every GPU that loads the library holds it until
// the process exits.  Every call shares it: calls that overlap on the GPU race, so callers
// order them on one stream or synchronise between streams.  Nothing in it needs to start
// at zero (each call writes every entry it later reads), so no clearing is done.
namespace sts {
namespace {

constexpr int64_t kNoAllocMaxN = 65536;
// Partial sums: splits * n <= (4 * 152 / ceil(n / 128) + 1) * n <= 4 * 152 * 128 + n.
constexpr int64_t kNoAllocMaxPart = 3 * (4 * 152 * kDirT + kNoAllocMaxN);
constexpr size_t kNoAllocBytes64 = sizeof(double4) * kNoAllocMaxN;
constexpr size_t kNoAllocBytes32 = sizeof(float4) * 2 * kNoAllocMaxN;
constexpr size_t kNoAllocBytesPart = sizeof(double) * kNoAllocMaxPart;
constexpr size_t kNoAllocBytes = kNoAllocBytes64 + kNoAllocBytes32 + kNoAllocBytesPart;  // ~7.4 MB
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_direct_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of g_direct_scratch on the current device.  In host code the array's name
// is only a host-side stand-in, so the address is looked up once per device (with that
// device current) and cached.
int noalloc_scratch(unsigned char** out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_error("sts_direct_noalloc: cudaGetDevice failed: %s", cudaGetErrorString(e));
        return STS_ERR_CUDA;
    }
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        set_error("sts_direct_noalloc: device %d is beyond the %d devices supported", dev, kNoAllocMaxDevices);
        return STS_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_direct_scratch);
        if (e != cudaSuccess || !ptr) {
            set_error("sts_direct_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return STS_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = ptr;
    }
    *out = (unsigned char*)g_noalloc_ptr[dev];
    return STS_OK;
}

}  // namespace
}  // namespace sts

extern "C" int sts_direct_noalloc(const double* pos, const double* zeta, const double* area, int64_t n,
                                  int32_t precision, double* vel, void* stream)
{
    using namespace sts;
    set_error("%s", "");
    if (n < 0 || (n > 0 && (!pos || !zeta || !area || !vel))) {
        set_error("sts_direct_noalloc: n < 0 or NULL array");
        return STS_ERR_ARG;
    }
    if (precision != STS_FP64 && precision != STS_MIXED) {
        set_error("sts_direct_noalloc: precision must be STS_FP64 or STS_MIXED");
        return STS_ERR_ARG;
    }
    if (n > kNoAllocMaxN) {
        set_error("sts_direct_noalloc: n = %lld exceeds the fixed scratch limit of %lld particles "
                  "(use sts_direct)", (long long)n, (long long)kNoAllocMaxN);
        return STS_ERR_CAPACITY;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) return STS_OK;
    if (n == 1) {
        STS_CUDA(cudaMemsetAsync(vel, 0, 3 * sizeof(double), s));
        return STS_OK;
    }
    unsigned char* base = nullptr;
    int rc = noalloc_scratch(&base);
    if (rc) return rc;
    double4* s64 = (double4*)base;
    float4* s32 = (float4*)(base + kNoAllocBytes64);
    double* part = (double*)(base + kNoAllocBytes64 + kNoAllocBytes32);
    // the same split of the sources as sts_direct, so both give the same sums
    const int64_t nt = n;
    const int64_t ntb = (nt + kDirT - 1) / kDirT;
    int64_t splits = (4 * 152 + ntb - 1) / ntb;
    splits = std::max<int64_t>(1, std::min<int64_t>(splits, std::max<int64_t>(1, n / 1024)));
    splits = std::min<int64_t>(splits, 256);
    const int64_t chunk = ((n + splits - 1) / splits + kDirT - 1) / kDirT * kDirT;
    splits = (n + chunk - 1) / chunk;
    if (splits < 1) splits = 1;
    if (3 * splits * nt > kNoAllocMaxPart) {
        set_error("sts_direct_noalloc: internal partial-sum bound exceeded");
        return STS_ERR_CAPACITY;
    }
    (k_direct_prep<<<blocks(n, 256), 256, 0, s>>>(pos, zeta, area, n, s64, s32), note_launch());
    const dim3 grid((unsigned)ntb, (unsigned)splits);
    if (precision == STS_FP64)
        (k_direct_fp64<<<grid, kDirT, 0, s>>>(s64, n, nullptr, nt, chunk, part), note_launch());
    else
        (k_direct_mixed<<<grid, kDirT, 0, s>>>(s32, n, nullptr, nt, chunk, part), note_launch());
    (k_direct_finish<<<blocks(nt, 256), 256, 0, s>>>(part, (int)splits, nt, nullptr, s64, vel), note_launch());
    STS_LAUNCH_CHECK();
    return STS_OK;
}
