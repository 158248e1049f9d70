// Icosahedral triangle tree (Sec. 3, "Grids on a Sphere": the 20 faces of an icosahedron,
// each refined into four children) and the MAC-driven interaction lists of the tree
// traversal (Sec. 3.4), built on the device.
//
// Every floating-point decision here (face of a particle, child digit, MAC) must come out
// exactly as in an IEEE FP64 evaluation of the same expressions in the same order, so this
// translation unit is compiled with --fmad=false and spells every FP64 operation on a
// decision path with a round-to-nearest intrinsic (no contraction, no reassociation).
//
// Readings fixed here (the paper gives no orientation, numbering or tie rule):
//   face      first face f maximising x . C_f over the 20 face centres C_f (the centres'
//             spherical Voronoi cells are exactly the faces of the regular icosahedron);
//   children  of (v1, v2, v3), with m_ab = unit(v_a + v_b): 0 = (v1, m12, m31),
//             1 = (m12, v2, m23), 2 = (m31, m23, v3), 3 = (m12, m23, m31); digit of x is 0
//             if (m12 x m31) . x >= 0, else 1 if (m23 x m12) . x >= 0, else 2 if
//             (m31 x m23) . x >= 0, else 3;
//   split     a triangle with more than N_T particles below the depth limit has children;
//   geometry  circumcentre c = unit((v2 - v1) x (v3 - v1)), chord radius r = |c - v1|;
//   MAC       (r_t + r_s) < theta |c_t - c_s| (strict; coincident centres never pass).
//
// Build, level by level, with the particles left in their original order:
//   level 0   face of every particle (warp-aggregated counts); root nodes in face order.
//   level l   split flags and child-digit normals per node; child digit per particle and
//             child counts; child nodes numbered in key order (scan); particles move to
//             their child.  All levels run in one cooperative launch with grid-wide
//             barriers between the passes; the host reads the counts once, at the end.
//   sort      a stable radix sort by the first slot of each particle's leaf gives the
//             sorted order (leaves depth first, original order inside a leaf), in the same
//             launch; then the leaf list in slot order.
#include <stdio.h>

#include <algorithm>
#include <utility>

#include "sts_internal.cuh"

namespace sts {
namespace {

constexpr unsigned kFull = 0xffffffffu;

struct g3 {
    double x, y, z;
};
__device__ __forceinline__ g3 gmk(double x, double y, double z) { return g3{x, y, z}; }
__device__ __forceinline__ g3 gadd(g3 a, g3 b)
{
    return gmk(__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y), __dadd_rn(a.z, b.z));
}
__device__ __forceinline__ g3 gsub(g3 a, g3 b)
{
    return gmk(__dsub_rn(a.x, b.x), __dsub_rn(a.y, b.y), __dsub_rn(a.z, b.z));
}
// (a.x b.x + a.y b.y) + a.z b.z
__device__ __forceinline__ double gdot(g3 a, g3 b)
{
    return __dadd_rn(__dadd_rn(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y)), __dmul_rn(a.z, b.z));
}
__device__ __forceinline__ g3 gcross(g3 a, g3 b)
{
    return gmk(__dsub_rn(__dmul_rn(a.y, b.z), __dmul_rn(a.z, b.y)),
               __dsub_rn(__dmul_rn(a.z, b.x), __dmul_rn(a.x, b.z)),
               __dsub_rn(__dmul_rn(a.x, b.y), __dmul_rn(a.y, b.x)));
}
// s / |s|, |s| = sqrt of the dot above, three divisions
__device__ __forceinline__ g3 gunit(g3 s)
{
    const double n = __dsqrt_rn(gdot(s, s));
    return gmk(__ddiv_rn(s.x, n), __ddiv_rn(s.y, n), __ddiv_rn(s.z, n));
}
__device__ __forceinline__ g3 gld(const double* p) { return gmk(p[0], p[1], p[2]); }
__device__ __forceinline__ void gst(double* p, g3 a)
{
    p[0] = a.x;
    p[1] = a.y;
    p[2] = a.z;
}

__constant__ double c_fc[20][3];     // face centres
__constant__ double c_fv[20][3][3];  // face vertices (counter-clockwise seen from outside)
__constant__ float c_fc32[20][3];    // face centres rounded to FP32 (pre-filter only)

// FP32 pre-filters.  A decision is taken from FP32 values only when the FP32 result is
// farther from the decision boundary than its worst-case rounding error (inputs rounded to
// FP32, three products and two sums: below 3.1e-7 times the sum of |products| for points of
// norm <= 1); otherwise the exact FP64 expression decides.  So every decision equals the
// FP64 one bit for bit, and FP64 runs only for points within ~1e-6 of a boundary.
__device__ __forceinline__ float fdot(float ax, float ay, float az, float bx, float by, float bz)
{
    return fmaf(az, bz, fmaf(ay, by, ax * bx));
}

// x rounded to the nearest FP32 value (ties to even), from its bits with integer arithmetic
// (conversions run on GB300's narrow FP64 path); zero, and values outside FP32's normal range,
// take the conversion instruction.
__device__ __forceinline__ float f32_rn(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FF);
    if (e < 1023 - 126 || e > 1023 + 127) return (float)x;
    const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    unsigned q = (unsigned)(m >> 29);
    const unsigned long long r = m & ((1ull << 29) - 1), half = 1ull << 28;
    q += (r > half || (r == half && (q & 1u))) ? 1u : 0u;  // a carry into the exponent is exact
    return __uint_as_float(((unsigned)(b >> 32) & 0x80000000u) + ((unsigned)(e - 1023 + 127) << 23) + q);
}

__device__ void node_geometry(double* g, g3 v1, g3 v2, g3 v3)
{
    gst(g, v1);
    gst(g + 3, v2);
    gst(g + 6, v3);
    const g3 c = gunit(gcross(gsub(v2, v1), gsub(v3, v1)));
    gst(g + 9, c);
    const g3 e = gsub(c, v1);
    g[12] = __dsqrt_rn(gdot(e, e));
}

// Warp-aggregated atomicAdd of 1 to ctr[key] (keys may differ across lanes).
__device__ __forceinline__ void agg_inc(int32_t* ctr, int key, bool active)
{
    const unsigned m = __ballot_sync(kFull, active);
    if (!active) return;
    const unsigned peers = __match_any_sync(m, key);
    const int leader = __ffs(peers) - 1;
    if ((int)(threadIdx.x & 31) == leader) atomicAdd(&ctr[key], __popc(peers));
}

// ------------------------------------------------------------------------- level 0
// Root key of a particle: instance b (from the instance offsets, b = 0 without them) times 20
// plus its face (the first face maximising x . C_f).  The dots are taken in FP32; the FP32
// winner stands when it leads by more than twice the FP32 error, else FP64 decides among the
// faces within that margin of the FP32 maximum (any other face is below the FP64 maximum, so
// the first FP64 maximiser is the same as over all 20).
__device__ int root_key(const double* __restrict__ pos, int64_t i, const int64_t* __restrict__ inst_off, int ninst,
                        float4* __restrict__ posf, int* __restrict__ status)
{
    const g3 x = gld(pos + 3 * i);
    if (!isfinite(x.x) || !isfinite(x.y) || !isfinite(x.z)) atomicOr(status, kStatusNonfinite);
    const float fx = f32_rn(x.x), fy = f32_rn(x.y), fz = f32_rn(x.z);
    posf[i] = make_float4(fx, fy, fz, 0.f);
    float df[20];
#pragma unroll
    for (int f = 0; f < 20; f++) df[f] = fdot(fx, fy, fz, c_fc32[f][0], c_fc32[f][1], c_fc32[f][2]);
    float b1 = df[0], b2 = -3.f;
    int fb = 0, best = 0;
#pragma unroll
    for (int f = 1; f < 20; f++) {
        if (df[f] > b1) {
            b2 = b1;
            b1 = df[f];
            fb = f;
        } else if (df[f] > b2) {
            b2 = df[f];
        }
    }
    const float scale = fmaxf(1.f, fmaxf(fabsf(fx), fmaxf(fabsf(fy), fabsf(fz))));
    const float margin = 4e-6f * scale;
    if (b1 - b2 > margin) {
        best = fb;
    } else {
        double bd = 0.0;
        bool any = false;
#pragma unroll
        for (int f = 0; f < 20; f++) {
            if (!(df[f] >= b1 - margin)) continue;
            const double d = gdot(x, gmk(c_fc[f][0], c_fc[f][1], c_fc[f][2]));
            if (!any || d > bd) {
                bd = d;
                best = f;
                any = true;
            }
        }
    }
    int b = 0;
    if (inst_off) {  // largest b with inst_off[b] <= i
        int lo = 0, hi = ninst - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (inst_off[mid] <= i)
                lo = mid;
            else
                hi = mid - 1;
        }
        b = lo;
    }
    return 20 * b + best;
}

// ------------------------------------------------------------------------- levels
// All levels below the roots in one cooperative launch (every CTA resident): per level l,
// with nodes [lb, le) = [lvl[l], lvl[l + 1]),
//   nodes      split flags, edge midpoints and child-digit normals (four lanes per node);
//   particles  the move of level l - 1 and the child digit at level l, counted per (node,
//              digit);
//   totals     the number of children of each CTA's contiguous share of the nodes;
//   children   numbered in key order (the CTA's offset from the totals before it, a block scan
//              inside), with vertices, start and count; lvl[l + 2] = end of level l + 1;
// with a grid-wide barrier after each.  Every CTA computes the level's total itself, so all
// of them see the same next range and stop at the same level: after a level that adds no
// node, or after nlev levels (while recording: the planned depth plus one that must come out
// empty).  The arithmetic of every decision is that of the per-level passes it replaces.
constexpr int kBuildThreads = 256;
constexpr int kBuildWarps = kBuildThreads / 32;
constexpr int kPrivNodes = 256;       // levels with at most this many nodes count in shared memory
constexpr int kBarSpins = 1 << 22;    // x 64 ns sleeps: a barrier gives up after ~0.3 s
constexpr int kCcRep = 8;             // copies of the (node, digit) counters: CTA b adds to copy
                                      // b % 8, so that each counter takes 8x fewer same-address
                                      // atomics (they serialise in L2)

struct BuildArgs {
    int64_t* lvl;
    const int64_t* inst_off;  // instance offsets (NULL: one instance)
    int ninst;
    int32_t* face_count;      // [20 ninst] particles per root key, zeroed before the launch
    int32_t* face_node;       // [20 ninst] root node of each key, or -1
    int nlev, leaf_size, max_level;
    int64_t cap;  // node capacity
    const double* pos_in;  // the caller's positions, copied into pos by the faces pass
    double* pos;
    float4* posf;  // [n] the positions rounded to FP32 (written with the faces, read by the levels)
    int64_t n;
    int32_t* nodeof;
    uint8_t* digit;
    int32_t *level, *parent, *first_child, *nchild, *start, *count, *leaf, *child;
    int32_t* cc;        // kCcRep copies of [cap, 4], cc_stride apart
    int64_t cc_stride;  // 4 cap
    uint64_t* key;
    double *geom, *norm, *mid;
    float4 *norm32, *c32;
    int64_t *over, *nnodes, *tot;  // tot: [2 CTAs] per-CTA totals
    unsigned* bar;   // arrival counter, zeroed before the launch
    unsigned* bar2;  // the sort launch's arrival counter, zeroed by the tree launch
    int32_t* mark;   // [n] scratch: node + 1 at each leaf's first slot, else 0
    int* status;
    // the sorted order
    int sort_passes;             // 8-bit digits of the slot keys
    int32_t *perm, *perm_tmp;    // sorted position -> particle
    uint32_t *skey, *skey_tmp;   // keys between passes
    int32_t* hist;               // [256 CTAs + 256] digit counts per CTA, then per digit
    int32_t *leaves, *slot_leaf;
    int64_t* nleaves;
    // clusters (nodes with more than N_T particles) and the moment pass's tasks
    int32_t *cluster_slot, *cluster_node;
    int64_t* up_toff;  // [nodes + 1] first task of each node
    int2* up_tasks;    // (cluster, first particle of the chunk)
    int64_t up_cap;
    double* up_frame;
    float* up_frame32;
    int64_t *nclusters, *nuptasks;
};

// Frame of cluster cl (node p) for the spherical barycentric coordinates of Sec. 3.2 (y =
// b1 v1 + b2 v2 + b3 v3, Cramer's rule): rows n_i / D with n1 = v2 x v3, n2 = v3 x v1,
// n3 = v1 x v2, D = v1 . n1, and b(c) = (n_i / D) . c at the circumcentre; frame32: the
// frame in FP32 and the centre as an FP32 hi/lo pair (18 floats).
__device__ void cluster_frame(const BuildArgs& a, int64_t cl, int32_t p)
{
    const double* g = a.geom + 13 * (int64_t)p;
    const double v1x = g[0], v1y = g[1], v1z = g[2], v2x = g[3], v2y = g[4], v2z = g[5];
    const double v3x = g[6], v3y = g[7], v3z = g[8];
    const double n[9] = {v2y * v3z - v2z * v3y, v2z * v3x - v2x * v3z, v2x * v3y - v2y * v3x,
                         v3y * v1z - v3z * v1y, v3z * v1x - v3x * v1z, v3x * v1y - v3y * v1x,
                         v1y * v2z - v1z * v2y, v1z * v2x - v1x * v2z, v1x * v2y - v1y * v2x};
    const double D = v1x * n[0] + v1y * n[1] + v1z * n[2];
    double* f = a.up_frame + 12 * cl;
    for (int q = 0; q < 9; q++) f[q] = n[q] / D;
    for (int q = 0; q < 3; q++) f[9 + q] = f[3 * q] * g[9] + f[3 * q + 1] * g[10] + f[3 * q + 2] * g[11];
    float* h = a.up_frame32 + 18 * cl;
    for (int q = 0; q < 12; q++) h[q] = (float)f[q];
    for (int q = 0; q < 3; q++) {
        const float hi = (float)g[9 + q];
        h[12 + q] = hi;
        h[15 + q] = (float)(g[9 + q] - (double)hi);
    }
}

// Grid-wide barrier of a cooperative launch: barrier k of the launch ends when the arrival
// counter reaches k G.  A CTA that waits too long flags the timeout and sets the counter's top
// bit, which releases every CTA, now and at later barriers; all of them then return.
__device__ bool grid_sync(unsigned* cnt, unsigned& k, int* status, int* s_ok)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        k++;
        const unsigned target = k * gridDim.x;
        __threadfence();  // this CTA's writes before its arrival
        unsigned v = atomicAdd(cnt, 1u) + 1u;
        for (int spins = 0; v < target; spins++) {
            if (spins > kBarSpins) {
                atomicOr(status, kStatusTimeout);
                v = atomicOr(cnt, 0x80000000u) | 0x80000000u;
                break;
            }
            __nanosleep(64);
            v = *(volatile unsigned*)cnt;
        }
        __threadfence();  // the others' writes after the release
        *s_ok = (v & 0x80000000u) ? 0 : 1;
    }
    __syncthreads();
    return *s_ok != 0;
}

// Level nodes.  The FP64 square roots and divisions are long dependent chains, so the work of
// a node is spread over lanes: in the first ceil(nl / 10) warps, lanes 3 j + a (j < 10, a < 3)
// form the edge midpoint m_a of node 10 w + j and its child-digit normal n_a = m_a x
// m_(a+2 mod 3); in the next ceil(nl / 32) warps, lane j sets the split flag and clears the
// counters of node 32 w + j (leaves get norm32.w = -1).  Circumcentres and radii, which no
// later level needs, are left to one pass over all nodes after the last level.
__device__ void level_nodes(const BuildArgs& a, int32_t lb, int32_t le, int64_t gt, int64_t gs)
{
    const int32_t nl = le - lb;
    const int64_t wm = (nl + 9) / 10, wc = (nl + 31) / 32;
    const int lane = threadIdx.x & 31;
    for (int64_t w = gt >> 5; w < wm + wc; w += gs >> 5) {
        if (w < wm) {
            const int j = lane / 3, q = lane - 3 * j;
            const int32_t p = lb + (int32_t)(10 * w) + j;
            const bool valid = lane < 30 && p < le;
            const bool split = valid && a.count[p] > a.leaf_size && a.level[p] < a.max_level;
            g3 m = gmk(0.0, 0.0, 0.0);
            if (split) {
                // m_0 = unit(v1 + v2), m_1 = unit(v2 + v3), m_2 = unit(v3 + v1)
                const double* g = a.geom + 13 * (int64_t)p;
                const g3 va = gld(g + 3 * q), vb = gld(g + 3 * (q == 2 ? 0 : q + 1));
                m = gunit(gadd(va, vb));
                gst(a.mid + 9 * (int64_t)p + 3 * q, m);
            }
            // m_(a+2 mod 3) from lane 3 j + 2 (a = 0) or 3 j + a - 1 (a = 1, 2)
            const int src = 3 * j + (q == 0 ? 2 : q - 1);
            const g3 mp =
                gmk(__shfl_sync(kFull, m.x, src), __shfl_sync(kFull, m.y, src), __shfl_sync(kFull, m.z, src));
            if (split) {
                const g3 nv = gcross(m, mp);
                gst(a.norm + 9 * (int64_t)p + 3 * q, nv);
                const float thr = 1e-6f * (float)(fabs(nv.x) + fabs(nv.y) + fabs(nv.z));
                a.norm32[3 * (int64_t)p + q] = make_float4((float)nv.x, (float)nv.y, (float)nv.z, thr);
            }
        } else {
            const int32_t p = lb + (int32_t)(32 * (w - wm)) + lane;
            if (p < le) {
                const bool split = a.count[p] > a.leaf_size && a.level[p] < a.max_level;
                a.leaf[p] = split ? 0 : 1;
                if (split) {
                    for (int r = 0; r < kCcRep; r++)
                        *reinterpret_cast<int4*>(a.cc + r * a.cc_stride + 4 * (int64_t)p) = make_int4(0, 0, 0, 0);
                } else {
                    a.norm32[3 * (int64_t)p] = make_float4(0.f, 0.f, 0.f, -1.f);  // w < 0: a leaf
                }
            }
        }
    }
}

// Per particle: first the move of level l - 1 (a particle of a node of level l - 1 goes to
// the child its digit names; a leaf's child table points at itself), then the digit of its
// node if that node of level l splits (norm32.w >= 0), counted per (node, digit) in cc.  The
// loads of one particle form two dependent rounds (node, then child and normals).  Levels with
// at most kPrivNodes nodes count in shared memory first (one global add per counter and
// CTA): there every counter takes thousands of increments, which serialise in L2.
__device__ void level_particles(const BuildArgs& a, int l, int32_t pb, int32_t lb, int32_t le, int64_t gt,
                                int64_t gs, int32_t* shc)
{
    const bool priv = le - lb <= kPrivNodes;
    int32_t* cc = a.cc + (blockIdx.x % kCcRep) * a.cc_stride;  // this CTA's copy of the counters
    if (priv) {
        for (int k = threadIdx.x; k < 4 * (le - lb); k += blockDim.x) shc[k] = 0;
        __syncthreads();
    }
    // kPU particles per thread and trip, their loads issued together round by round
    constexpr int kPU = 4;
    const int64_t n = a.n;
    const int64_t nr = (n + 31) & ~(int64_t)31;  // whole warps run every trip (warp-wide counting)
    for (int64_t i0 = gt; i0 < nr; i0 += kPU * gs) {
        int p[kPU], dg[kPU];
        float fx[kPU], fy[kPU], fz[kPU];
#pragma unroll
        for (int u = 0; u < kPU; u++) {
            const int64_t i = i0 + u * gs;
            p[u] = -1;
            dg[u] = 0;
            fx[u] = fy[u] = fz[u] = 0.f;
            if (i < n) {
                p[u] = a.nodeof[i];
                dg[u] = a.digit[i];
                const float4 q = a.posf[i];
                fx[u] = q.x;
                fy[u] = q.y;
                fz[u] = q.z;
            }
        }
#pragma unroll
        for (int u = 0; u < kPU; u++) {
            if (l == 0 && p[u] >= 0) {  // the root key becomes the root node
                p[u] = a.face_node[p[u]];
                a.nodeof[i0 + u * gs] = p[u];
            } else if (p[u] >= pb && p[u] < lb) {
                p[u] = a.child[4 * p[u] + dg[u]];
                a.nodeof[i0 + u * gs] = p[u];
            }
        }
        float4 q3[kPU][3];
#pragma unroll
        for (int u = 0; u < kPU; u++) {
            const int64_t pp = p[u] >= lb ? p[u] : 0;
#pragma unroll
            for (int q = 0; q < 3; q++) q3[u][q] = a.norm32[3 * pp + q];
        }
#pragma unroll
        for (int u = 0; u < kPU; u++) {
            const int64_t i = i0 + u * gs;
            const bool active = p[u] >= lb && p[u] < le && q3[u][0].w >= 0.f;
            int d = 0;
            if (active) {
                const float scale = fmaxf(1.f, fmaxf(fabsf(fx[u]), fmaxf(fabsf(fy[u]), fabsf(fz[u]))));
                // digit = first a with n_a . x >= 0, else 3; decided in FP32 while unambiguous
                d = -1;
#pragma unroll
                for (int q = 0; q < 3; q++) {
                    if (d != -1) continue;
                    const float t = fdot(q3[u][q].x, q3[u][q].y, q3[u][q].z, fx[u], fy[u], fz[u]);
                    const float thr = q3[u][q].w * scale;
                    if (t > thr)
                        d = q;
                    else if (!(t < -thr))
                        d = -2;  // too close to this boundary for FP32
                }
                if (d == -1) d = 3;
                if (d == -2) {
                    const g3 x = gld(a.pos + 3 * i);
                    const double* nn = a.norm + 9 * (int64_t)p[u];
                    if (gdot(gld(nn), x) >= 0.0)
                        d = 0;
                    else if (gdot(gld(nn + 3), x) >= 0.0)
                        d = 1;
                    else if (gdot(gld(nn + 6), x) >= 0.0)
                        d = 2;
                    else
                        d = 3;
                }
                a.digit[i] = (uint8_t)d;
            }
            if (priv)
                agg_inc(shc, 4 * (p[u] - lb) + d, active);
            else
                agg_inc(cc, 4 * p[u] + d, active);
        }
    }
    if (priv) {
        __syncthreads();
        for (int k = threadIdx.x; k < 4 * (le - lb); k += blockDim.x)
            if (shc[k]) atomicAdd(&cc[4 * (int64_t)lb + k], shc[k]);
    }
}

// Particles of node p per child digit: the sum of the counter copies.
__device__ __forceinline__ int4 level_counts(const BuildArgs& a, int32_t p)
{
    int4 c = make_int4(0, 0, 0, 0);
#pragma unroll
    for (int r = 0; r < kCcRep; r++) {
        const int4 v = *reinterpret_cast<const int4*>(a.cc + r * a.cc_stride + 4 * (int64_t)p);
        c.x += v.x;
        c.y += v.y;
        c.z += v.z;
        c.w += v.w;
    }
    return c;
}

// Number of children of node p of the current level (0 for a leaf).
__device__ __forceinline__ int level_nch(const BuildArgs& a, int32_t p)
{
    if (a.leaf[p]) return 0;
    const int4 c = level_counts(a, p);
    return (c.x > 0) + (c.y > 0) + (c.z > 0) + (c.w > 0);
}

// The children of node p, numbered from id on in digit order.  A child beyond the node
// capacity is not created: its particles stay with the parent and the overflow bit is set, so
// a recorded build reports it instead of writing out of range.
__device__ void level_children(const BuildArgs& a, int32_t p, int64_t id64)
{
    if (a.leaf[p]) {
        a.first_child[p] = -1;
        a.nchild[p] = 0;
        a.child[4 * p] = a.child[4 * p + 1] = a.child[4 * p + 2] = a.child[4 * p + 3] = p;
        return;
    }
    const double* g = a.geom + 13 * (int64_t)p;
    const g3 v1 = gld(g), v2 = gld(g + 3), v3 = gld(g + 6);
    const double* mm = a.mid + 9 * (int64_t)p;
    const g3 m12 = gld(mm), m23 = gld(mm + 3), m31 = gld(mm + 6);
    const g3 cv[4][3] = {{v1, m12, m31}, {m12, v2, m23}, {m31, m23, v3}, {m12, m23, m31}};
    int32_t id = (int32_t)min(id64, a.cap);
    const int32_t first = id;
    int32_t st = a.start[p];
    const int32_t lv = a.level[p] + 1;
    const uint64_t kp = a.key[p];
    const int4 c4 = level_counts(a, p);
    const int32_t cd[4] = {c4.x, c4.y, c4.z, c4.w};
    int nc = 0;
    for (int d = 0; d < 4; d++) {
        const int32_t c = cd[d];
        if (c == 0) {
            a.child[4 * p + d] = -1;
            continue;
        }
        if (id >= a.cap) {
            a.child[4 * p + d] = p;
            atomicOr((unsigned long long*)a.over, 1ull);
            st += c;
            continue;
        }
        a.child[4 * p + d] = id;
        a.level[id] = lv;
        a.key[id] = kp * 4u + (uint64_t)d;
        a.parent[id] = p;
        a.first_child[id] = -1;
        a.nchild[id] = 0;
        a.start[id] = st;
        a.count[id] = c;
        a.leaf[id] = 0;
        double* gc = a.geom + 13 * (int64_t)id;  // vertices; centre and radius with the next level
        gst(gc, cv[d][0]);
        gst(gc + 3, cv[d][1]);
        gst(gc + 6, cv[d][2]);
        st += c;
        id++;
        nc++;
    }
    a.first_child[p] = nc ? first : -1;
    a.nchild[p] = nc;
}

// Exclusive scan of one value per thread over a CTA of kBuildThreads; *total = the CTA's sum.
__device__ int64_t build_block_scan(int64_t v, int64_t* sh, int64_t* total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    int64_t before = 0, all = 0;
#pragma unroll
    for (int k = 0; k < kBuildThreads / 32; k++) {
        const int64_t s = sh[k];
        if (k < w) before += s;
        all += s;
    }
    __syncthreads();
    *total = all;
    return before + x - v;
}

// The cluster table from the per-CTA totals in tot (clusters, tasks): cluster number and first
// task of every node of [q0, q1) (a block scan on top of the CTAs before), the node of every
// cluster, its tasks and its frame; totals into the device counters.
__device__ void cluster_table(const BuildArgs& a, int G, int32_t q0, int32_t q1, int32_t nn, int64_t* sh,
                              int64_t* s_cf, int64_t* s_tf, int64_t* s_ct)
{
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid < 32) {
        int64_t bf = 0, bt = 0, tf = 0, tt = 0;
        for (int b = lane; b < G; b += 32) {
            const int64_t f = a.tot[2 * b], t = a.tot[2 * b + 1];
            tf += f;
            tt += t;
            if (b < (int)blockIdx.x) {
                bf += f;
                bt += t;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            bf += __shfl_xor_sync(kFull, bf, o);
            bt += __shfl_xor_sync(kFull, bt, o);
            tf += __shfl_xor_sync(kFull, tf, o);
            tt += __shfl_xor_sync(kFull, tt, o);
        }
        if (lane == 0) {
            *s_cf = bf;
            *s_ct = bt;
            *s_tf = tf;
            if (blockIdx.x == 0) {
                *a.nclusters = tf;
                *a.nuptasks = tt;
                a.up_toff[nn] = tt;
            }
        }
    }
    __syncthreads();
    int64_t cf = *s_cf, ct = *s_ct;
    __syncthreads();
    for (int32_t r0 = q0; r0 < q1; r0 += blockDim.x) {
        const int32_t p = r0 + tid;
        const int32_t c = p < q1 ? a.count[p] : 0;
        const int f = c > a.leaf_size ? 1 : 0;
        const int nt = f ? (c + kUpChunk - 1) / kUpChunk : 0;
        int64_t rf, rt;
        const int64_t ef = build_block_scan(f, sh, &rf);
        const int64_t et = build_block_scan(nt, sh, &rt);
        if (p < q1) {
            const int64_t t0 = ct + et;
            a.up_toff[p] = t0;
            if (f) {
                const int64_t cl = cf + ef;
                a.cluster_slot[p] = (int32_t)cl;
                a.cluster_node[cl] = p;
                for (int j = 0; j < nt; j++) {
                    if (t0 + j < a.up_cap)
                        a.up_tasks[t0 + j] = make_int2((int)cl, j * kUpChunk);
                    else
                        atomicOr((unsigned long long*)a.over, 4ull);
                }
                cluster_frame(a, cl, p);
            } else {
                a.cluster_slot[p] = -1;
            }
        }
        cf += rf;
        ct += rt;
    }
}

__global__ void __launch_bounds__(kBuildThreads) k_build_levels(const BuildArgs a)
{
    __shared__ int32_t shc[4 * kPrivNodes];
    __shared__ int64_t sh[kBuildThreads / 32];
    __shared__ int64_t s_before, s_total, s_cbefore;
    __shared__ int s_ok;
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + tid, gs = (int64_t)gridDim.x * blockDim.x;
    const int G = (int)gridDim.x;
    unsigned bk = 0;
    if (blockIdx.x == 0 && tid == 0) *a.bar2 = 0;
    // faces: the root key of every particle (into nodeof) and the particles per key
    const int nkeys = 20 * a.ninst;
    {
        const bool priv = nkeys <= 4 * kPrivNodes;
        if (priv) {
            for (int k = tid; k < nkeys; k += blockDim.x) shc[k] = 0;
            __syncthreads();
        }
        const int64_t nr = (a.n + 31) & ~(int64_t)31;  // whole warps (warp-wide counting)
        for (int64_t i = gt; i < nr; i += gs) {
            const bool active = i < a.n;
            int rk = 0;
            if (active) {
                rk = root_key(a.pos_in, i, a.inst_off, a.ninst, a.posf, a.status);
                for (int q = 0; q < 3; q++) a.pos[3 * i + q] = a.pos_in[3 * i + q];
                a.nodeof[i] = rk;
                a.digit[i] = 0;  // a particle whose root is a leaf moves to child[4 p + 0] = p
                a.mark[i] = 0;
            }
            agg_inc(priv ? shc : a.face_count, rk, active);
        }
        if (priv) {
            __syncthreads();
            for (int k = tid; k < nkeys; k += blockDim.x)
                if (shc[k]) atomicAdd(&a.face_count[k], shc[k]);
        }
    }
    if (!grid_sync(a.bar, bk, a.status, &s_ok)) return;
    // roots: the non-empty keys in key order, numbered by a scan over the CTAs' shares of the
    // keys (id = non-empty keys before, start = particles before)
    const int kchunk = (nkeys + G - 1) / G;
    const int k0 = min(nkeys, (int)blockIdx.x * kchunk), k1 = min(nkeys, ((int)blockIdx.x + 1) * kchunk);
    {
        int64_t nf = 0, nc = 0;
        for (int k = k0 + tid; k < k1; k += blockDim.x) {
            const int c = a.face_count[k];
            nf += c > 0;
            nc += c;
        }
        int64_t tf, tc;
        build_block_scan(nf, sh, &tf);
        build_block_scan(nc, sh, &tc);
        if (tid == 0) {
            a.tot[2 * blockIdx.x] = tf;
            a.tot[2 * blockIdx.x + 1] = tc;
        }
    }
    if (!grid_sync(a.bar, bk, a.status, &s_ok)) return;
    int32_t pb = 0, lb = 0, le = 0;
    {
        if (tid < 32) {
            int64_t bf = 0, bc = 0, tf = 0;
            for (int b = lane; b < G; b += 32) {
                const int64_t f = a.tot[2 * b], c = a.tot[2 * b + 1];
                tf += f;
                if (b < (int)blockIdx.x) {
                    bf += f;
                    bc += c;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                bf += __shfl_xor_sync(kFull, bf, o);
                bc += __shfl_xor_sync(kFull, bc, o);
                tf += __shfl_xor_sync(kFull, tf, o);
            }
            if (lane == 0) {
                s_before = bf;
                s_total = tf;
                s_cbefore = bc;
            }
        }
        __syncthreads();
        int64_t cf = s_before, cc = s_cbefore;
        le = (int32_t)s_total;
        for (int r0 = k0; r0 < k1; r0 += blockDim.x) {
            const int rk = r0 + tid;
            const int c = rk < k1 ? a.face_count[rk] : 0;
            int64_t rf, rc;
            const int64_t ef = build_block_scan(c > 0, sh, &rf);
            const int64_t ec = build_block_scan(c, sh, &rc);
            if (rk < k1) {
                if (c == 0) {
                    a.face_node[rk] = -1;
                } else {
                    const int f = rk % 20;
                    const int32_t id = (int32_t)(cf + ef);
                    a.face_node[rk] = id;
                    a.level[id] = 0;
                    a.key[id] = (uint64_t)rk;
                    a.parent[id] = -1;
                    a.first_child[id] = -1;
                    a.nchild[id] = 0;
                    a.start[id] = (int32_t)(cc + ec);
                    a.count[id] = c;
                    a.leaf[id] = 0;
                    double* g = a.geom + 13 * (int64_t)id;  // vertices; centre and radius after the levels
                    for (int v = 0; v < 3; v++) gst(g + 3 * v, gmk(c_fv[f][v][0], c_fv[f][v][1], c_fv[f][v][2]));
                }
            }
            cf += rf;
            cc += rc;
        }
        if (blockIdx.x == 0 && tid == 0) {
            a.lvl[0] = 0;
            a.lvl[1] = le;
        }
    }
    if (!grid_sync(a.bar, bk, a.status, &s_ok)) return;
    bool stopped = false;  // a level added no node
    int32_t nn = 0;
    for (int l = 0; l < a.nlev; l++) {
        level_nodes(a, lb, le, gt, gs);
        if (!grid_sync(a.bar, bk, a.status, &s_ok)) return;
        level_particles(a, l, pb, lb, le, gt, gs, shc);
        if (!grid_sync(a.bar, bk, a.status, &s_ok)) return;
        // this CTA's share of the nodes and its number of children
        const int32_t nl = le - lb;
        const int32_t chunk = (nl + G - 1) / G;
        const int32_t c0 = lb + min(nl, (int32_t)blockIdx.x * chunk), c1 = lb + min(nl, ((int32_t)blockIdx.x + 1) * chunk);
        int64_t mine = 0;
        for (int32_t p = c0 + tid; p < c1; p += blockDim.x) mine += level_nch(a, p);
        int64_t cta_total;
        build_block_scan(mine, sh, &cta_total);
        if (tid == 0) a.tot[blockIdx.x] = cta_total;
        if (!grid_sync(a.bar, bk, a.status, &s_ok)) return;
        // the children before this CTA's share and in the whole level
        if (tid < 32) {
            int64_t before = 0, total = 0;
            for (int b = lane; b < G; b += 32) {
                const int64_t v = a.tot[b];
                total += v;
                if (b < (int)blockIdx.x) before += v;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                before += __shfl_xor_sync(kFull, before, o);
                total += __shfl_xor_sync(kFull, total, o);
            }
            if (lane == 0) {
                s_before = before;
                s_total = total;
            }
        }
        __syncthreads();
        const int32_t next = (int32_t)min((int64_t)le + s_total, a.cap);
        if (blockIdx.x == 0 && tid == 0) a.lvl[l + 2] = next;  // end of level l + 1
        int64_t carry = s_before;
        for (int32_t r0 = c0; r0 < c1; r0 += blockDim.x) {
            const int32_t p = r0 + tid;
            const int k = p < c1 ? level_nch(a, p) : 0;
            int64_t rtot;
            const int64_t ex = build_block_scan(k, sh, &rtot);
            if (p < c1) level_children(a, p, (int64_t)le + carry + ex);
            carry += rtot;
        }
        if (!grid_sync(a.bar, bk, a.status, &s_ok)) return;
        if (next == le) {
            stopped = true;
            nn = le;
            break;
        }
        pb = lb;
        lb = le;
        le = next;
    }
    // nodes = lvl[last level + 1]; a last planned level that still produced children means the
    // build ran out of levels (overflow): its new nodes are not part of the tree
    if (!stopped) nn = lb;
    if (blockIdx.x == 0 && tid == 0) {
        *a.nnodes = nn;
        if (!stopped && le > lb) atomicOr((unsigned long long*)a.over, 2ull);
    }
    // circumcentres and radii of all nodes, with their FP32 copies for the pre-filtered MAC
    for (int64_t p = gt; p < nn; p += gs) {
        double* g = a.geom + 13 * p;
        node_geometry(g, gld(g), gld(g + 3), gld(g + 6));
        a.c32[p] = make_float4((float)g[9], (float)g[10], (float)g[11], (float)g[12]);
    }

    // ---- clusters: this CTA's share [q0, q1) of the nodes, its clusters and their tasks (one
    // per kUpChunk particles), numbered in node order after the first sort barrier
    const int32_t qch = (nn + G - 1) / G;
    const int32_t q0 = min(nn, (int32_t)blockIdx.x * qch), q1 = min(nn, q0 + qch);
    {
        int64_t fc = 0, tc = 0;
        for (int32_t p = q0 + tid; p < q1; p += blockDim.x) {
            const int32_t c = a.count[p];
            if (c > a.leaf_size) {
                fc++;
                tc += (c + kUpChunk - 1) / kUpChunk;
            }
        }
        int64_t t1, t2;
        build_block_scan(fc, sh, &t1);
        build_block_scan(tc, sh, &t2);
        if (tid == 0) {
            a.tot[2 * blockIdx.x] = t1;
            a.tot[2 * blockIdx.x + 1] = t2;
        }
    }
    // the first slot of every leaf, marked with its node (+1): the leaf list in slot order
    // needs no particle sort
    for (int32_t p = q0 + tid; p < q1; p += blockDim.x)
        if (a.leaf[p]) a.mark[a.start[p]] = p + 1;
    if (!grid_sync(a.bar, bk, a.status, &s_ok)) return;
    cluster_table(a, G, q0, q1, nn, sh, &s_before, &s_total, &s_cbefore);
    // ---- the leaves in slot order; slot_leaf = index of the slot's leaf (a scan over the
    // CTAs' shares of the slots)
    const int64_t n = a.n;
    const int64_t ich = (n + G - 1) / G;
    const int64_t i0 = min(n, (int64_t)blockIdx.x * ich), i1 = min(n, i0 + ich);
    {
        int64_t mine = 0;
        for (int64_t k = i0 + tid; k < i1; k += blockDim.x) mine += a.mark[k] != 0;
        int64_t t;
        build_block_scan(mine, sh, &t);
        if (tid == 0) a.tot[2 * G + blockIdx.x] = t;
    }
    if (!grid_sync(a.bar, bk, a.status, &s_ok)) return;
    if (tid < 32) {
        int64_t before = 0, total = 0;
        for (int b = lane; b < G; b += 32) {
            const int64_t v = a.tot[2 * G + b];
            total += v;
            if (b < (int)blockIdx.x) before += v;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            before += __shfl_xor_sync(kFull, before, o);
            total += __shfl_xor_sync(kFull, total, o);
        }
        if (lane == 0) {
            s_before = before;
            s_total = total;
        }
    }
    __syncthreads();
    int64_t carry = s_before;
    for (int64_t r0 = i0; r0 < i1; r0 += blockDim.x) {
        const int64_t k = r0 + tid;
        const int32_t mk = k < i1 ? a.mark[k] : 0;
        const int f = mk != 0;
        int64_t rt;
        const int64_t ex = build_block_scan(f, sh, &rt);
        if (k < i1) {
            const int64_t li = carry + ex + f - 1;
            a.slot_leaf[k] = (int32_t)li;
            if (f) a.leaves[li] = mk - 1;
        }
        carry += rt;
    }
    if (blockIdx.x == 0 && tid == 0) *a.nleaves = s_total;
}

// The sorted order, a second cooperative launch after the tree (the interaction lists, which
// need only the tree, start beside it on the side stream): a stable LSD radix sort (8-bit
// digits) of the particles by the first slot of their leaf, which keeps the particles of a
// leaf in their original order.  CTA b owns items [i0, i1) of every pass, its warp w the w-th
// part of them, so the rank of an item among equal digits follows (CTA, warp, round, lane),
// i.e. the item order.  Its barrier counter (bar2) is cleared by the tree launch.
__global__ void __launch_bounds__(kBuildThreads) k_build_sort(const BuildArgs a)
{
    __shared__ int32_t hw[kBuildWarps * 256];  // per-warp digit counts, then positions
    __shared__ int64_t sh[kBuildThreads / 32];
    __shared__ int s_ok;
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + tid;
    const int G = (int)gridDim.x;
    unsigned bk = 0;
    const int64_t n = a.n;
    const int64_t ich = (n + G - 1) / G;
    const int64_t i0 = min(n, (int64_t)blockIdx.x * ich), i1 = min(n, i0 + ich);
    const int w = tid >> 5;
    const int64_t wch = (i1 - i0 + kBuildWarps - 1) / kBuildWarps;
    const int64_t w0 = min(i1, i0 + w * wch), w1 = min(i1, w0 + wch);
    const int P = a.sort_passes;
    const unsigned lt = (1u << lane) - 1u;
    if (P == 0) {  // a single particle
        if (gt < n) a.perm[gt] = (int32_t)gt;
    }
    for (int pass = 0; pass < P; pass++) {
        const int shift = 8 * pass;
        // pass p writes the main buffers when P - 1 - p is even, so the last one ends there;
        // pass 0 takes its keys from the tree
        uint32_t* kout = ((P - 1 - pass) & 1) ? a.skey_tmp : a.skey;
        int32_t* vout = ((P - 1 - pass) & 1) ? a.perm_tmp : a.perm;
        const uint32_t* kin = ((P - pass) & 1) ? a.skey_tmp : a.skey;
        const int32_t* vin = ((P - pass) & 1) ? a.perm_tmp : a.perm;
        // digit counts per warp; this CTA's entry of every digit's row
        for (int k = tid; k < kBuildWarps * 256; k += blockDim.x) hw[k] = 0;
        __syncthreads();
        for (int64_t i = w0 + lane; i < w1; i += 32) {
            const uint32_t key = pass == 0 ? (uint32_t)a.start[a.nodeof[i]] : kin[i];
            atomicAdd(&hw[w * 256 + (int)((key >> shift) & 255u)], 1);
        }
        __syncthreads();
        for (int d = tid; d < 256; d += blockDim.x) {
            int t = 0;
            for (int ww = 0; ww < kBuildWarps; ww++) t += hw[ww * 256 + d];
            a.hist[d * G + blockIdx.x] = t;
        }
        if (!grid_sync(a.bar2, bk, a.status, &s_ok)) return;
        // rows d = b, b + G, ...: exclusive offsets along the row (over the CTAs), row totals
        for (int d = blockIdx.x; d < 256; d += G) {
            int64_t carry = 0;
            for (int r0 = 0; r0 < G; r0 += blockDim.x) {
                const int j = r0 + tid;
                const int v = j < G ? a.hist[d * G + j] : 0;
                int64_t rt;
                const int64_t ex = build_block_scan(v, sh, &rt);
                if (j < G) a.hist[d * G + j] = (int32_t)(carry + ex);
                carry += rt;
            }
            if (tid == 0) a.hist[256 * G + d] = (int32_t)carry;
        }
        if (!grid_sync(a.bar2, bk, a.status, &s_ok)) return;
        // the first position of each (digit, warp): digit base + CTA offset + earlier warps
        for (int d0 = 0; d0 < 256; d0 += blockDim.x) {
            const int d = d0 + tid;
            int64_t tot;
            const int64_t base = build_block_scan(d < 256 ? a.hist[256 * G + d] : 0, sh, &tot);
            if (d < 256) {
                int run = (int)base + a.hist[d * G + blockIdx.x];
                for (int ww = 0; ww < kBuildWarps; ww++) {
                    const int c = hw[ww * 256 + d];
                    hw[ww * 256 + d] = run;
                    run += c;
                }
            }
        }
        __syncthreads();
        // scatter, 32 consecutive items per round: rank among equal digits of the round
        const bool lastp = pass == P - 1;
        for (int64_t i = w0; i < w1; i += 32) {
            const int64_t ii = i + lane;
            const bool valid = ii < w1;
            uint32_t key = 0;
            int32_t val = 0;
            if (valid) {
                if (pass == 0) {
                    key = (uint32_t)a.start[a.nodeof[ii]];
                    val = (int32_t)ii;
                } else {
                    key = kin[ii];
                    val = vin[ii];
                }
            }
            const int d = valid ? (int)((key >> shift) & 255u) : 256 + lane;
            const unsigned peers = __match_any_sync(kFull, d);
            const int rk = __popc(peers & lt), cnt = __popc(peers);
            const int prior = valid ? hw[w * 256 + d] : 0;
            __syncwarp();
            if (valid && rk == cnt - 1) hw[w * 256 + d] = prior + cnt;
            __syncwarp();
            if (valid) {
                if (!lastp) kout[prior + rk] = key;
                vout[prior + rk] = val;
            }
        }
        if (!grid_sync(a.bar2, bk, a.status, &s_ok)) return;
    }
}



// ------------------------------------------------------------------------- lists
constexpr int kStack = 128;

__device__ __forceinline__ bool mac(const double* gt, const double* gs, double theta)
{
    const g3 e = gsub(gld(gt + 9), gld(gs + 9));
    const double R = __dsqrt_rn(gdot(e, e));
    return __dadd_rn(gt[12], gs[12]) < __dmul_rn(theta, R);
}

// MAC with the FP32 pre-filter: |(r_t + r_s) - theta R| is decided in FP32 when it exceeds
// the FP32 rounding bound (2.1e-7 + 5e-7 R + 2e-7 (r_t + r_s) for centres of norm 1),
// otherwise by the exact FP64 expression above.
__device__ __forceinline__ bool mac_filtered(float4 ct, float4 cs, float theta32, const double* gt,
                                             const double* gs, double theta)
{
    const float ex = ct.x - cs.x, ey = ct.y - cs.y, ez = ct.z - cs.z;
    const float R = sqrtf(fdot(ex, ey, ez, ex, ey, ez));
    const float lhs = ct.w + cs.w, rhs = theta32 * R;
    const float m = 1e-6f * (1.f + lhs + R);
    if (lhs < rhs - m) return true;
    if (lhs > rhs + m) return false;
    return mac(gt, gs, theta);
}

// A lower bound on the distance between any point of leaf t and any point of leaf s (their
// circumcircles' gap), in FP32: the centre difference and its squared length are FP64, the
// square root and the radii FP32, and a margin of 1e-6 of the sum covers every FP32 rounding
// (about 6 units of 2^-24 of it).  The evaluator only compares it with the close-pair radius to
// decide whether a near block needs the close-pair test, so a bound that is a little low costs
// a test and never changes a result.
__device__ __forceinline__ float near_gap(const double* gt, const double* gs)
{
    const g3 e3 = gsub(gld(gt + 9), gld(gs + 9));
    const float dist = sqrtf((float)gdot(e3, e3));
    const float rt = (float)gt[12], rs = (float)gs[12];
    return dist - rt - rs - 1e-6f * (dist + rt + rs);
}

// Target-leaf traversal of Sec. 3.4 (PC + PP), one thread per target leaf: from the roots of
// the leaf's instance in face order, a source node that passes the MAC is far (a cluster,
// more than N_T particles) or near; one that fails is near if it is a leaf, else its
// children are visited in digit order.  fill = 0 counts far nodes, near nodes and near
// chunks per leaf; fill = 1 writes them at the scanned offsets.
__global__ void k_lists(int fill, const int64_t* __restrict__ nleaves_p, const int32_t* __restrict__ leaves,
                        const int32_t* __restrict__ face_node, const uint64_t* __restrict__ key,
                        const int32_t* __restrict__ level, double theta, int leaf_size,
                        const double* __restrict__ geom, const float4* __restrict__ c32,
                        const int32_t* __restrict__ leaf,
                        const int32_t* __restrict__ first_child, const int32_t* __restrict__ nchild,
                        const int32_t* __restrict__ start, const int32_t* __restrict__ count,
                        const int32_t* __restrict__ cluster_slot, int32_t* __restrict__ cnt,
                        const int64_t* __restrict__ far_po, const int64_t* __restrict__ near_po,
                        const int64_t* __restrict__ chunk_po,
                        int32_t* __restrict__ far_idx, int32_t* __restrict__ near_idx,
                        FarEntry* __restrict__ far_ent, NearEntry* __restrict__ near_ent,
                        int64_t far_cap, int64_t near_cap, int64_t chunk_cap, int64_t ldc,
                        const uint8_t* __restrict__ only, int* __restrict__ status, int64_t* __restrict__ over)
{
    const int64_t nleaves = min(*nleaves_p, ldc);
    const int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (L >= nleaves) return;
    if (only && !only[L]) return;  // the warp traversal handled this leaf
    if (fill && (far_po[L + 1] > far_cap || near_po[L + 1] > near_cap || chunk_po[L + 1] > chunk_cap)) {
        atomicOr((unsigned long long*)over, 4ull);  // recorded capacities too small
        return;
    }
    const int32_t t = leaves[L];
    // roots of the target leaf's own instance: root key (instance * 20 + face) of the leaf
    const uint64_t rk = key[t] >> (2 * level[t]);
    const int32_t* roots = face_node + (int64_t)(rk / 20) * 20;
    const double* gt = geom + 13 * (int64_t)t;
    const float4 ct = c32[t];
    const float theta32 = (float)theta;
    int32_t stk[kStack];
    int sp = 0;
    for (int f = 19; f >= 0; f--)
        if (roots[f] >= 0) stk[sp++] = roots[f];
    int64_t nf = 0, nn = 0, nch = 0;
    const int64_t fo = fill ? far_po[L] : 0, no = fill ? near_po[L] : 0, co = fill ? chunk_po[L] : 0;
    while (sp > 0) {
        const int32_t s = stk[--sp];
        const double* gs = geom + 13 * (int64_t)s;
        bool is_far = false, is_near = false;
        if (mac_filtered(ct, c32[s], theta32, gt, gs, theta)) {
            if (count[s] > leaf_size)
                is_far = true;
            else
                is_near = true;
        } else if (leaf[s]) {
            is_near = true;
        } else {
            const int32_t fc = first_child[s], nc = nchild[s];
            if (sp + nc > kStack) {
                atomicOr(status, kStatusCapacity);
                break;
            }
            for (int c = nc - 1; c >= 0; c--) stk[sp++] = fc + c;
        }
        if (is_far) {
            if (fill) {
                const int64_t q = fo + nf;
                far_idx[q] = s;
                FarEntry e;
                e.slot = cluster_slot[s];
                e.dx = (float)__dsub_rn(gs[9], gt[9]);
                e.dy = (float)__dsub_rn(gs[10], gt[10]);
                e.dz = (float)__dsub_rn(gs[11], gt[11]);
                far_ent[q] = e;
            }
            nf++;
        } else if (is_near) {
            const int32_t st = start[s], ct2 = count[s];
            if (fill) {
                near_idx[no + nn] = s;
                const float gap = near_gap(gt, gs);
                NearEntry e;
                e.dx = (float)__dsub_rn(gs[9], gt[9]);
                e.dy = (float)__dsub_rn(gs[10], gt[10]);
                e.dz = (float)__dsub_rn(gs[11], gt[11]);
                e.gap = gap;
                e.pad[0] = e.pad[1] = 0;
                for (int32_t c0 = 0; c0 < ct2; c0 += kStage) {
                    e.start = st + c0;
                    e.count = min(kStage, ct2 - c0);
                    near_ent[co + nch] = e;
                    nch++;
                }
            } else {
                nch += (ct2 + kStage - 1) / kStage;
            }
            nn++;
        }
    }
    if (!fill) {
        cnt[L] = (int32_t)nf;
        cnt[ldc + L] = (int32_t)nn;
        cnt[2 * ldc + L] = (int32_t)nch;
    }
}

// ------------------------------------------------------------------------- lists, warp form
// One warp per target leaf: the traversal of k_lists, expanded breadth first (32 source
// nodes decided per round), then the terminal nodes (far and near entries) sorted into the
// depth-first order of the roots by a left-aligned key, which is the order the per-thread
// traversal emits.  Frontier and terminals live in shared memory; a leaf whose traversal
// does not fit sets `wover` and is left to k_lists.
constexpr int kLwWarps = 4;
// CAP: frontier nodes per level and far + near nodes per leaf that one warp holds in shared
// memory (256 for theta >= 0.6, whose lists stay well below it; 512 below, at half the
// occupancy).  A leaf that needs more goes to the per-thread traversal.

__device__ __forceinline__ uint64_t dfs_key(uint64_t key, int lv)
{
    const uint64_t low = key & ((1ull << (2 * lv)) - 1ull);
    const uint64_t face = (key >> (2 * lv)) % 20ull;
    return ((face << (2 * lv)) | low) << (2 * (kMaxLevel - lv));
}

__device__ __forceinline__ int warp_sum(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ int warp_excl_scan(int v, int lane, int* total)
{
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    *total = __shfl_sync(kFull, x, 31);
    return x - v;
}

// Count pass of the warp traversal, one warp per target leaf: breadth-first from the roots of
// the leaf's instance (frontier in shared memory), MAC as in k_lists; the terminals (far
// nodes flagged by the sign bit) go unsorted to terms[L * CAP ...] for the fill pass, the
// counts to cnt.  A leaf whose frontier or terminal list exceeds CAP is marked in wover and
// left to the per-thread traversal.
template <int CAP>
__global__ void __launch_bounds__(kLwWarps * 32)
k_lists_count(const int64_t* __restrict__ nleaves_p, const int32_t* __restrict__ leaves,
              const int32_t* __restrict__ face_node, const uint64_t* __restrict__ key,
              const int32_t* __restrict__ level, double theta, int leaf_size, const double* __restrict__ geom,
              const float4* __restrict__ c32, const int32_t* __restrict__ leaf,
              const int32_t* __restrict__ first_child, const int32_t* __restrict__ nchild,
              const int32_t* __restrict__ count, int32_t* __restrict__ cnt, int32_t* __restrict__ terms,
              int64_t ldc, uint8_t* __restrict__ wover)
{
    __shared__ int32_t front[kLwWarps][2][CAP];
    __shared__ int32_t tnode[kLwWarps][CAP];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t L = (int64_t)blockIdx.x * kLwWarps + w;
    if (L >= min(*nleaves_p, ldc)) return;
    const int32_t t = leaves[L];
    const double* gt = geom + 13 * (int64_t)t;
    const float4 ct = c32[t];
    const float theta32 = (float)theta;
    const uint64_t rk = key[t] >> (2 * level[t]);
    const int32_t* roots = face_node + (int64_t)(rk / 20) * 20;
    int32_t* fr[2] = {front[w][0], front[w][1]};
    // roots of the leaf's instance, in face order
    {
        const int32_t r = lane < 20 ? roots[lane] : -1;
        const unsigned m = __ballot_sync(kFull, r >= 0);
        if (r >= 0) fr[0][__popc(m & ((1u << lane) - 1u))] = r;
    }
    int nfront = __popc(__ballot_sync(kFull, lane < 20 && roots[lane < 20 ? lane : 0] >= 0));
    int cur = 0, nterm = 0;
    bool bad = false;
    __syncwarp();
    while (nfront > 0 && !bad) {
        int nnext = 0;
        for (int b0 = 0; b0 < nfront; b0 += 32) {
            const int i = b0 + lane;
            int32_t s = -1;
            int kind = 0;  // 1 far, 2 near, 3 expand
            if (i < nfront) {
                s = fr[cur][i];
                const double* gs = geom + 13 * (int64_t)s;
                if (mac_filtered(ct, c32[s], theta32, gt, gs, theta))
                    kind = count[s] > leaf_size ? 1 : 2;
                else
                    kind = leaf[s] ? 2 : 3;
            }
            const int nc = kind == 3 ? nchild[s] : 0;
            int ctot;
            const int coff = warp_excl_scan(nc, lane, &ctot);
            if (nnext + ctot > CAP) {
                bad = true;
                break;
            }
            for (int c = 0; c < nc; c++) fr[cur ^ 1][nnext + coff + c] = first_child[s] + c;
            nnext += ctot;
            const bool term = kind == 1 || kind == 2;
            const unsigned tm = __ballot_sync(kFull, term);
            if (nterm + __popc(tm) > CAP) {
                bad = true;
                break;
            }
            if (term) tnode[w][nterm + __popc(tm & ((1u << lane) - 1u))] = s | (kind == 1 ? (int32_t)0x80000000 : 0);
            nterm += __popc(tm);
        }
        __syncwarp();
        cur ^= 1;
        nfront = nnext;
    }
    if (bad) {
        if (lane == 0) wover[L] = 1;
        return;
    }
    int nf = 0, nn = 0, nch = 0;
    int32_t* out = terms + L * CAP;
    for (int i = lane; i < nterm; i += 32) {
        const int32_t tn = tnode[w][i];
        out[i] = tn;
        if (tn < 0) {
            nf++;
        } else {
            nn++;
            nch += (count[tn] + kStage - 1) / kStage;
        }
    }
    nf = warp_sum(nf);
    nn = warp_sum(nn);
    nch = warp_sum(nch);
    if (lane == 0) {
        wover[L] = 0;
        cnt[L] = nf;
        cnt[ldc + L] = nn;
        cnt[2 * ldc + L] = nch;
    }
}

// Fill pass of the warp traversal: the leaf's terminals from terms, sorted by depth-first key
// (bitonic sort in shared memory), written at the scanned offsets: far clusters with their
// FP32 centre offsets, near leaves split into chunks of at most kStage particles.
template <int CAP>
__global__ void __launch_bounds__(kLwWarps * 32)
k_lists_fill(const int64_t* __restrict__ nleaves_p, const int32_t* __restrict__ leaves,
             const uint64_t* __restrict__ key, const int32_t* __restrict__ level, const double* __restrict__ geom,
             const int32_t* __restrict__ start, const int32_t* __restrict__ count,
             const int32_t* __restrict__ cluster_slot, const int32_t* __restrict__ terms,
             const int64_t* __restrict__ far_po, const int64_t* __restrict__ near_po,
             const int64_t* __restrict__ chunk_po, int32_t* __restrict__ far_idx, int32_t* __restrict__ near_idx,
             FarEntry* __restrict__ far_ent, NearEntry* __restrict__ near_ent, int64_t far_cap,
             int64_t near_cap, int64_t chunk_cap, int64_t ldc, const uint8_t* __restrict__ wover,
             int64_t* __restrict__ over)
{
    __shared__ uint64_t tkey[kLwWarps][CAP];
    __shared__ int32_t tnode[kLwWarps][CAP];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t L = (int64_t)blockIdx.x * kLwWarps + w;
    if (L >= min(*nleaves_p, ldc)) return;
    if (wover[L]) return;  // done by k_lists
    if (far_po[L + 1] > far_cap || near_po[L + 1] > near_cap || chunk_po[L + 1] > chunk_cap) {
        if (lane == 0) atomicOr((unsigned long long*)over, 4ull);
        return;
    }
    const int32_t t = leaves[L];
    const double* gt = geom + 13 * (int64_t)t;
    const int nterm = (int)((far_po[L + 1] - far_po[L]) + (near_po[L + 1] - near_po[L]));
    const int32_t* in = terms + L * CAP;
    int P = 1;
    while (P < nterm) P <<= 1;
    for (int i = lane; i < P; i += 32) {
        uint64_t k = ~0ull;  // padding keys sort last
        if (i < nterm) {
            const int32_t tn = in[i];
            const int32_t s = tn & 0x7fffffff;
            tnode[w][i] = tn;
            k = dfs_key(key[s], level[s]);
        }
        tkey[w][i] = k;
    }
    __syncwarp();
    for (int k = 2; k <= P; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = lane; i < P; i += 32) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const uint64_t a = tkey[w][i], b = tkey[w][ixj];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) {
                        tkey[w][i] = b;
                        tkey[w][ixj] = a;
                        const int32_t tn = tnode[w][i];
                        tnode[w][i] = tnode[w][ixj];
                        tnode[w][ixj] = tn;
                    }
                }
            }
            __syncwarp();
        }
    // emit in order: far, near and near chunks get their ranks by warp scans
    int64_t nf = 0, nn = 0, nch = 0;
    const int64_t fo = far_po[L], no = near_po[L], co = chunk_po[L];
    for (int b0 = 0; b0 < nterm; b0 += 32) {
        const int i = b0 + lane;
        int32_t s = -1;
        bool isfar = false;
        int chunks = 0;
        if (i < nterm) {
            const int32_t tn = tnode[w][i];
            isfar = tn < 0;
            s = tn & 0x7fffffff;
            if (!isfar) chunks = (count[s] + kStage - 1) / kStage;
        }
        const bool valid = i < nterm;
        const unsigned fm = __ballot_sync(kFull, valid && isfar);
        const unsigned nm = __ballot_sync(kFull, valid && !isfar);
        int chtot;
        const int choff = warp_excl_scan(chunks, lane, &chtot);
        if (valid) {
            const double* gs = geom + 13 * (int64_t)s;
            const float dx = (float)__dsub_rn(gs[9], gt[9]);
            const float dy = (float)__dsub_rn(gs[10], gt[10]);
            const float dz = (float)__dsub_rn(gs[11], gt[11]);
            if (isfar) {
                const int64_t q = fo + nf + __popc(fm & ((1u << lane) - 1u));
                far_idx[q] = s;
                FarEntry e;
                e.slot = cluster_slot[s];
                e.dx = dx;
                e.dy = dy;
                e.dz = dz;
                far_ent[q] = e;
            } else {
                near_idx[no + nn + __popc(nm & ((1u << lane) - 1u))] = s;
                const float gap = near_gap(gt, gs);
                NearEntry e;
                e.dx = dx;
                e.dy = dy;
                e.dz = dz;
                e.gap = gap;
                e.pad[0] = e.pad[1] = 0;
                const int32_t st = start[s], ct2 = count[s];
                int64_t q = co + nch + choff;
                for (int32_t c0 = 0; c0 < ct2; c0 += kStage) {
                    e.start = st + c0;
                    e.count = min(kStage, ct2 - c0);
                    near_ent[q++] = e;
                }
            }
        }
        nf += __popc(fm);
        nn += __popc(nm);
        nch += chtot;
    }
}

// List and task totals (scanned offsets read at index nleaves) into the device counters.
__global__ void k_list_totals(int64_t* __restrict__ dc, const int64_t* __restrict__ far_off,
                              const int64_t* __restrict__ near_off, const int64_t* __restrict__ chunk_off,
                              int64_t ldc)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (dc[kDcLeaves] > ldc) atomicOr((unsigned long long*)(dc + kDcOver), 4ull);  // recorded leaf bound
    const int64_t L = min(dc[kDcLeaves], ldc);
    dc[kDcFar] = far_off[L];
    dc[kDcNear] = near_off[L];
    dc[kDcChunks] = chunk_off[L];
    int64_t t = 0;
    for (int q = 0; q < 8; q++) t += dc[kDcClass + q];
    dc[kDcTasks] = t;
}


// Lanes sharing a pair of targets: the largest S <= 8 with S * pairs <= 32.
__device__ __forceinline__ int lanes_per_pair(int pairs) { return min(8, 32 / pairs); }

// Splits a leaf of nt targets into k warp tasks of nearly equal size, at most tmax targets
// each, two targets per lane and S lanes per pair of targets.  k maximises the fraction of
// useful interactions per warp step, nt S / (64 k) (ties go to the smaller k).
__device__ int task_split(int nt, int tmax)
{
    const int kmin = max(1, (nt + tmax - 1) / tmax);
    int best = kmin;
    float be = -1.f;
    for (int k = kmin; k <= kmin + 3; k++) {
        const int m = (nt + k - 1) / k;
        const int p = (m + 1) / 2;
        const int S = lanes_per_pair(p);
        const float e = (float)nt * (float)S / (64.f * (float)k);
        if (e > be * (1.f + 1e-6f)) {
            be = e;
            best = k;
        }
    }
    return best;
}

// Counts the warp tasks of every leaf by lane class (S = 1 .. 8) into cls[0..7].
__global__ void k_task_count(const int64_t* __restrict__ nleaves, int64_t ldc, const int32_t* __restrict__ leaves,
                             const int32_t* __restrict__ count, int tmax, unsigned long long* __restrict__ cls)
{
    const int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (L >= min(*nleaves, ldc)) return;
    const int32_t c = count[leaves[L]];
    const int k = task_split(c, tmax);
    for (int i = 0; i < k; i++) atomicAdd(cls + lanes_per_pair((c / k + (i < c % k ? 1 : 0) + 1) / 2) - 1, 1ull);
}

// Writes the warp tasks grouped by lane class, S = 1 first: a task's run time grows with the
// sources each lane visits (list length / S), so the task queue hands out the longest tasks
// first and the persistent evaluation kernel ends with short ones.  The order within a class
// is arbitrary; every task writes only its own targets, so the results do not depend on it.
__global__ void k_task_fill(const int64_t* __restrict__ nleaves, int64_t ldc, const int32_t* __restrict__ leaves,
                            const int32_t* __restrict__ start, const int32_t* __restrict__ count,
                            int tmax, const int64_t* __restrict__ cls, unsigned long long* __restrict__ fill,
                            int64_t cap, Task* __restrict__ tasks, int64_t* __restrict__ over)
{
    const int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (L >= min(*nleaves, ldc)) return;
    int64_t base[8];
    base[0] = 0;
#pragma unroll
    for (int q = 1; q < 8; q++) base[q] = base[q - 1] + cls[q - 1];
    const int32_t id = leaves[L];
    const int32_t st = start[id], c = count[id];
    const int k = task_split(c, tmax);
    int32_t t0 = 0;
    for (int i = 0; i < k; i++) {
        const int32_t m = c / k + (i < c % k ? 1 : 0);
        Task tk;
        tk.leaf = (int32_t)L;
        tk.t0 = st + t0;
        tk.nt = m;
        tk.S = lanes_per_pair((m + 1) / 2);
        const int q = tk.S - 1;
        const int64_t pos = base[q] + (int64_t)atomicAdd(fill + q, 1ull);
        if (pos < cap)
            tasks[pos] = tk;
        else
            atomicOr((unsigned long long*)over, 4ull);
        t0 += m;
    }
}

// Copies up to four device int64 values and the status word into out[0..4] so that the host
// reads them with one copy.
__global__ void k_gather(const int64_t* a, const int64_t* b, const int64_t* c, const int64_t* d,
                         const int* status, int64_t* out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    out[0] = a ? *a : 0;
    out[1] = b ? *b : 0;
    out[2] = c ? *c : 0;
    out[3] = d ? *d : 0;
    out[4] = *status;
}

// ------------------------------------------------------------------------- dual traversal
// Dual tree traversal of Sec. 3.4 over pairs (target node, source node), level-synchronous:
// every pair of the current frontier is decided at once.  A pair that passes the MAC is a
// terminal of its kind by the two particle counts against N_T (PP both at most N_T, PC only
// the source above, CP only the target above, CC both above); a failing pair of two leaves
// is PP; otherwise the triangle with more particles (the target on a tie; never a leaf) is
// replaced by its children, which form the next frontier's pairs.  Terminals are appended in
// any order and sorted afterwards (by kind, target, source), so nothing depends on the
// schedule.  Every count stays on the device: a fixed number of level launches (enough for
// the tree's depth) reads its frontier size from the counters, and a write past a capacity
// is dropped and flagged, after which the host grows the buffers and runs the traversal again.
enum { kPP = 0, kPC = 1, kCP = 2, kCC = 3 };

// dual_cnt layout (int64)
constexpr int kDuTerms = 0;      // terminal pairs found (every attempt counted)
constexpr int kDuP = 1;          // terminal pairs kept: min(found, capacity)
constexpr int kDuStart = 2;      // [2 .. 6]: first sorted pair of each kind, then the end
constexpr int kDuChunks = 8;     // [8] near chunks of PP, [9] of CP
constexpr int kDuFrontMax = 10;  // largest frontier asked for
constexpr int kDuOver = 11;      // overflow bits (eager runs)
constexpr int kDuCTasks = 12;    // evaluation tasks of the target clusters
constexpr int kDuFront = 16;     // [16 + l]: pairs entering level l
constexpr int kDuMaxLevels = 2 * kMaxLevel + 8;
constexpr int kDuSize = kDuFront + kDuMaxLevels + 1;

__device__ __forceinline__ bool near_kind(int k) { return k == kPP || k == kCP; }
__device__ __forceinline__ bool leaf_kind(int k) { return k == kPP || k == kPC; }

// The 20 x 20 root pairs of every instance (a target interacts with its own instance only).
__global__ void k_dual_roots(const int32_t* __restrict__ face_node, int ninst, int32_t* __restrict__ ft,
                             int32_t* __restrict__ fs, int64_t fcap, int64_t* __restrict__ du,
                             unsigned long long* __restrict__ over)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)ninst * 400) return;
    const int64_t b = i / 400;
    const int f1 = (int)(i % 400) / 20, f2 = (int)(i % 20);
    const int32_t t = face_node[20 * b + f1], s = face_node[20 * b + f2];
    if (t < 0 || s < 0) return;
    const int64_t q = (int64_t)atomicAdd((unsigned long long*)(du + kDuFront), 1ull);
    if (q < fcap) {
        ft[q] = t;
        fs[q] = s;
    } else {
        atomicOr(over, 4ull);
    }
}

// Level l of the traversal: the pairs of frontier l (ft, fs) decided; terminals appended to
// (tt, ts, tk), refined pairs to frontier l + 1 (gt, gs).  Appends are warp-aggregated: one
// atomic per warp reserves the warp's terminals, one its refined pairs.
__global__ void k_dual_level(int l, const int32_t* __restrict__ ft, const int32_t* __restrict__ fs,
                             int32_t* __restrict__ gt, int32_t* __restrict__ gs, int64_t fcap, double theta,
                             int leaf_size, const double* __restrict__ geom, const float4* __restrict__ c32,
                             const int32_t* __restrict__ leaf, const int32_t* __restrict__ first_child,
                             const int32_t* __restrict__ nchild, const int32_t* __restrict__ count,
                             int32_t* __restrict__ tt, int32_t* __restrict__ ts, uint8_t* __restrict__ tk,
                             int64_t tcap, int64_t* __restrict__ du, unsigned long long* __restrict__ over)
{
    const int64_t nf = min(du[kDuFront + l], fcap);
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x;
    if (i0 >= nf) return;  // whole warps below (the warp scans need every lane)
    const int64_t i = i0 + threadIdx.x;
    const int lane = threadIdx.x & 31;
    int32_t t = -1, s = -1, fc = 0, nc = 0;
    int kind = -1;
    bool split_t = false;
    if (i < nf) {
        t = ft[i];
        s = fs[i];
        const int32_t ct = count[t], cs = count[s];
        const bool lt = leaf[t] != 0, ls = leaf[s] != 0;
        if (mac_filtered(c32[t], c32[s], (float)theta, geom + 13 * (int64_t)t, geom + 13 * (int64_t)s, theta)) {
            const bool tc = ct > leaf_size, sc = cs > leaf_size;
            kind = tc ? (sc ? kCC : kCP) : (sc ? kPC : kPP);
        } else if (lt && ls) {
            kind = kPP;
        } else {
            split_t = !lt && (ls || ct >= cs);
            const int32_t p = split_t ? t : s;
            fc = first_child[p];
            nc = nchild[p];
        }
    }
    // terminals: one reservation per warp
    const unsigned tm = __ballot_sync(kFull, kind >= 0);
    if (tm) {
        unsigned long long base = 0;
        if (lane == __ffs(tm) - 1) base = atomicAdd((unsigned long long*)(du + kDuTerms), (unsigned long long)__popc(tm));
        base = __shfl_sync(kFull, base, __ffs(tm) - 1);
        if (kind >= 0) {
            const int64_t q = (int64_t)base + __popc(tm & ((1u << lane) - 1u));
            if (q < tcap) {
                tt[q] = t;
                ts[q] = s;
                tk[q] = (uint8_t)kind;
            } else {
                atomicOr(over, 4ull);
            }
        }
    }
    // refined pairs: a warp scan of the child counts, one reservation per warp
    int tot;
    const int off = warp_excl_scan(nc, lane, &tot);
    if (tot > 0) {
        unsigned long long base = 0;
        if (lane == 0) {
            base = atomicAdd((unsigned long long*)(du + kDuFront + l + 1), (unsigned long long)tot);
            atomicMax((unsigned long long*)(du + kDuFrontMax), base + (unsigned long long)tot);
        }
        base = __shfl_sync(kFull, base, 0);
        const int64_t q = (int64_t)base + off;
        if (nc > 0 && q + nc > fcap) atomicOr(over, 4ull);
        // every slot below the capacity is written (the next level reads min(count, fcap) pairs),
        // also those of a refinement that does not fit whole
        for (int32_t c = 0; c < nc && q + c < fcap; c++) {
            gt[q + c] = split_t ? fc + c : t;
            gs[q + c] = split_t ? s : fc + c;
        }
    }
}

// After the last level: the traversal must have ended (an empty frontier), and the pairs kept
// are the found ones up to the capacity.
__global__ void k_dual_close(int levels, int64_t tcap, int64_t* __restrict__ du, unsigned long long* __restrict__ over)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (du[kDuFront + levels] > 0) atomicOr(over, 4ull);  // deeper than the levels launched
    du[kDuP] = min(du[kDuTerms], tcap);
}

// The pairs are put in the order of the lists, (kind, target key, source node), by a counting
// sort on the bucket (kind, target key) followed by ranking within each bucket: the target key
// is the depth-first leaf index of a leaf target and the cluster slot of a cluster target, and
// the sources of one target are distinct (ties would go by the pair's index).  Buckets are
// small (the pairs of one target), so the ranking is a count over the bucket.
__global__ void k_dual_bucket(const int32_t* __restrict__ tt, const uint8_t* __restrict__ tk,
                              const int64_t* __restrict__ du, int64_t cap, int64_t KT,
                              const int32_t* __restrict__ start, const int32_t* __restrict__ slot_leaf,
                              const int32_t* __restrict__ cluster_slot, int32_t* __restrict__ bucket,
                              int32_t* __restrict__ bcnt, int32_t* __restrict__ arrive)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= min(du[kDuP], cap)) return;
    const int32_t t = tt[i];
    const int k = tk[i];
    const int64_t tkey = leaf_kind(k) ? slot_leaf[start[t]] : cluster_slot[t];
    const int32_t b = (int32_t)(k * KT + tkey);
    bucket[i] = b;
    arrive[i] = atomicAdd(bcnt + b, 1);
}

// Each pair at its arrival slot in its bucket: its source and index, for the ranking.
__global__ void k_dual_scatter(const int64_t* __restrict__ du, int64_t cap, const int32_t* __restrict__ bucket,
                               const int32_t* __restrict__ arrive, const int64_t* __restrict__ boff,
                               const int32_t* __restrict__ ts, uint32_t* __restrict__ bsrc, int32_t* __restrict__ bidx)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= min(du[kDuP], cap)) return;
    const int64_t q = boff[bucket[i]] + arrive[i];
    bsrc[q] = (uint32_t)ts[i];
    bidx[q] = (int32_t)i;
}

// The pair's place in the sorted order: its bucket's start plus the number of pairs of the
// bucket before it by (source, index); key = kind << bits_t | target key, perm = pair index.
__global__ void k_dual_rank(const int64_t* __restrict__ du, int64_t cap, int64_t KT, int bits_t,
                            const int32_t* __restrict__ bucket, const int64_t* __restrict__ boff,
                            const int32_t* __restrict__ bcnt, const int32_t* __restrict__ ts,
                            const uint32_t* __restrict__ bsrc, const int32_t* __restrict__ bidx,
                            uint32_t* __restrict__ key, int32_t* __restrict__ perm)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= min(du[kDuP], cap)) return;
    const int32_t b = bucket[i];
    const int64_t lo = boff[b];
    const int n = bcnt[b];
    const uint32_t s = (uint32_t)ts[i];
    int r = 0;
    for (int j = 0; j < n; j++) {
        const uint32_t sj = bsrc[lo + j];
        r += (sj < s || (sj == s && bidx[lo + j] < (int32_t)i)) ? 1 : 0;
    }
    const int64_t kind = b / KT;
    key[lo + r] = ((uint32_t)kind << bits_t) | (uint32_t)(b - kind * KT);
    perm[lo + r] = (int32_t)i;
}

// Sorted pairs, and the near chunks of every pair (0 for far kinds).
__global__ void k_dual_gather(const int32_t* __restrict__ tt, const int32_t* __restrict__ ts,
                              const int32_t* __restrict__ perm, const uint32_t* __restrict__ key, int bits_t,
                              const int64_t* __restrict__ du, int64_t cap, const int32_t* __restrict__ count,
                              int32_t* __restrict__ st, int32_t* __restrict__ ss, int32_t* __restrict__ chunks)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= min(du[kDuP], cap)) return;
    const int32_t q = perm[i], s = ts[q];
    st[i] = tt[q];
    ss[i] = s;
    chunks[i] = near_kind((int)(key[i] >> bits_t)) ? (count[s] + kStage - 1) / kStage : 0;
}

__device__ __forceinline__ int64_t lower_bound_u32(const uint32_t* __restrict__ key, int64_t n, uint32_t v)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (key[mid] < v)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// CSR offsets of the four kinds (blockIdx.y = kind): off[j] = first pair of target key j
// within its kind, j = 0 .. K (leaves for PP / PC, clusters for CP / CC); near kinds also the
// chunk offsets.  Thread 0 of each kind records the kind's first pair and its chunk total.
struct DualCsr {
    int64_t* off[4];
    int64_t* coff[4];
};

__global__ void k_dual_csr(const uint32_t* __restrict__ key, const int64_t* __restrict__ scan, int bits_t,
                           const int64_t* __restrict__ dc, int64_t lcap, int64_t ccap, DualCsr out,
                           int64_t* __restrict__ du)
{
    const int k = blockIdx.y;
    const int64_t K = leaf_kind(k) ? min(dc[kDcLeaves], lcap) : min(dc[kDcClusters], ccap);
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j > K) return;
    const int64_t P = du[kDuP];
    const uint32_t base = (uint32_t)k << bits_t;
    const int64_t ks = lower_bound_u32(key, P, base);
    const int64_t o = lower_bound_u32(key, P, base + (uint32_t)j);
    out.off[k][j] = o - ks;
    if (near_kind(k)) out.coff[k][j] = scan[o] - scan[ks];
    if (j == 0) {
        du[kDuStart + k] = ks;
        if (k == kCC) du[kDuStart + 4] = P;
        if (near_kind(k)) {
            const int64_t ke = lower_bound_u32(key, P, (uint32_t)(k + 1) << bits_t);  // k + 1 <= kCC
            du[kDuChunks + (k == kPP ? 0 : 1)] = scan[ke] - scan[ks];
        }
    }
}

// List entries of the sorted pairs: far (a source cluster's proxy block) or near (a source leaf
// in chunks of at most kStage particles), with the FP32 centre offset c_s - c_t and, for near
// entries, the lower bound on the distance between the two triangles' points.  Entries of kind
// k go to its arrays at (pair index - the kind's first pair), chunks at their scanned offsets.
struct DualFill {
    FarEntry* far[2];     // PC, CC
    NearEntry* near[2];   // PP, CP
    int32_t* idx[2];      // source node ids: PP (near_idx), PC (far_idx)
    int64_t far_cap[2], near_cap[2], idx_cap[2];
};

__global__ void k_dual_fill(const uint32_t* __restrict__ key, const int32_t* __restrict__ st,
                            const int32_t* __restrict__ ss, const int64_t* __restrict__ scan, int bits_t,
                            const int64_t* __restrict__ du, int64_t cap, const double* __restrict__ geom,
                            const int32_t* __restrict__ start, const int32_t* __restrict__ count,
                            const int32_t* __restrict__ cluster_slot, DualFill out,
                            unsigned long long* __restrict__ over)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= min(du[kDuP], cap)) return;
    const int k = (int)(key[i] >> bits_t);
    const int64_t ks = du[kDuStart + k], local = i - ks;
    const int32_t t = st[i], s = ss[i];
    const double* gt = geom + 13 * (int64_t)t;
    const double* gs = geom + 13 * (int64_t)s;
    const float dx = (float)__dsub_rn(gs[9], gt[9]);
    const float dy = (float)__dsub_rn(gs[10], gt[10]);
    const float dz = (float)__dsub_rn(gs[11], gt[11]);
    if (leaf_kind(k)) {
        const int a = k == kPP ? 0 : 1;
        if (local < out.idx_cap[a])
            out.idx[a][local] = s;
        else
            atomicOr(over, 4ull);
    }
    if (!near_kind(k)) {
        const int a = k == kPC ? 0 : 1;
        if (local >= out.far_cap[a]) {
            atomicOr(over, 4ull);
            return;
        }
        FarEntry e;
        e.slot = cluster_slot[s];
        e.dx = dx;
        e.dy = dy;
        e.dz = dz;
        out.far[a][local] = e;
        return;
    }
    const int a = k == kPP ? 0 : 1;
    NearEntry e;
    e.dx = dx;
    e.dy = dy;
    e.dz = dz;
    e.gap = near_gap(gt, gs);
    e.pad[0] = e.pad[1] = 0;
    const int32_t s0 = start[s], ct = count[s];
    int64_t q = scan[i] - scan[ks];
    if (q + (ct + kStage - 1) / kStage > out.near_cap[a]) {
        atomicOr(over, 4ull);
        return;
    }
    for (int32_t c0 = 0; c0 < ct; c0 += kStage) {
        e.start = s0 + c0;
        e.count = min(kStage, ct - c0);
        out.near[a][q++] = e;
    }
}

// Evaluation tasks of the target clusters (targets: the M proxy points of cluster slot c,
// rows c M .. c M + M - 1); has[c] = the cluster is the target of a CP or CC pair.
__global__ void k_cluster_tasks(const int64_t* __restrict__ dc, int64_t ccap, const int64_t* __restrict__ cfar_off,
                                const int64_t* __restrict__ cnear_off, int M, uint8_t* __restrict__ has,
                                Task* __restrict__ tasks, int64_t cap, int64_t* __restrict__ du,
                                unsigned long long* __restrict__ over)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= min(dc[kDcClusters], ccap)) return;
    const bool h = cfar_off[c + 1] > cfar_off[c] || cnear_off[c + 1] > cnear_off[c];
    has[c] = h ? 1 : 0;
    if (!h) return;
    const int k = task_split(M, kTaskTargets);
    const int64_t base = (int64_t)atomicAdd((unsigned long long*)(du + kDuCTasks), (unsigned long long)k);
    int32_t t0 = 0;
    for (int i = 0; i < k; i++) {
        const int32_t m = M / k + (i < M % k ? 1 : 0);
        Task tk;
        tk.leaf = (int32_t)c;
        tk.t0 = (int32_t)(c * M) + t0;
        tk.nt = m;
        tk.S = lanes_per_pair((m + 1) / 2);
        if (base + i < cap)
            tasks[base + i] = tk;
        else
            atomicOr(over, 4ull);
        t0 += m;
    }
}

// Interaction counts of the sorted dual pairs: st[kind] += PP pairs (j != i), PC target x
// proxy, CP proxy x source, CC proxy x proxy; launched over clusters with kind = 4: downward
// particle x M over the clusters in has.
__global__ void k_dual_count(int kind, const int32_t* __restrict__ tgt, const int32_t* __restrict__ src,
                             int64_t first, int64_t n, const int32_t* __restrict__ count,
                             const uint8_t* __restrict__ has, int M, unsigned long long* __restrict__ st)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long v = 0;
    if (i < n) {
        const unsigned long long mm = (unsigned long long)M;
        if (kind == 4) {
            v = has[i] ? (unsigned long long)count[tgt[i]] * mm : 0ull;  // tgt: cluster nodes
        } else {
            const int32_t t = tgt[first + i], s = src[first + i];
            const unsigned long long ct = (unsigned long long)count[t], cs = (unsigned long long)count[s];
            if (kind == kPP)
                v = ct * cs - (t == s ? ct : 0ull);
            else if (kind == kPC)
                v = ct * mm;
            else if (kind == kCP)
                v = mm * cs;
            else
                v = mm * mm;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(st + kind, v);
}

inline unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

int read_i64(sts_ctx* ctx, const int64_t* dptr, int64_t* out, cudaStream_t s)
{
    STS_CUDA(cudaMemcpyAsync(ctx->h_pinned, dptr, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    STS_CUDA(cudaStreamSynchronize(s));
    *out = ctx->h_pinned[0];
    return STS_OK;
}

int grow_nodes(sts_ctx* c, int64_t need, int64_t keep, cudaStream_t s)
{
    STS_CUDA(c->nd_level.grow(need, keep, s));
    STS_CUDA(c->nd_parent.grow(need, keep, s));
    STS_CUDA(c->nd_first_child.grow(need, keep, s));
    STS_CUDA(c->nd_nchild.grow(need, keep, s));
    STS_CUDA(c->nd_start.grow(need, keep, s));
    STS_CUDA(c->nd_count.grow(need, keep, s));
    STS_CUDA(c->nd_leaf.grow(need, keep, s));
    STS_CUDA(c->nd_key.grow(need, keep, s));
    STS_CUDA(c->nd_geom.grow(13 * need, 13 * keep, s));
    STS_CUDA(c->nd_norm.grow(9 * need, 9 * keep, s));
    STS_CUDA(c->nd_norm32.grow(3 * need, 3 * keep, s));
    STS_CUDA(c->nd_c32.grow(need, keep, s));
    STS_CUDA(c->nd_mid.grow(9 * need, 9 * keep, s));
    STS_CUDA(c->nd_cc.grow((size_t)kCcRep * 4 * c->nd_level.cap, 0, s));  // copies 4 cap apart
    STS_CUDA(c->nd_child.grow(4 * need, 4 * keep, s));
    return STS_OK;
}

}  // namespace

int reserve_tree_nodes(sts_ctx* c, int64_t nodes, cudaStream_t s) { return grow_nodes(c, nodes, 0, s); }

void gather_values(const int64_t* a, const int64_t* b, const int64_t* c, const int64_t* d, const int* status,
                   int64_t* out, cudaStream_t s)
{
    (k_gather<<<1, 32, 0, s>>>(a, b, c, d, status, out), note_launch());
}

// Nodes a tree can have: the roots plus four children of every split node, where a level
// holds at most n / (N_T + 1) split nodes (disjoint, each with more than N_T particles) and at
// most 20 instances 4^l nodes.  Without `full`, the bound is capped at 12 n / (N_T + 1) more
// than the roots (a first guess several times the node count of uniform data).
static int64_t tree_node_bound(int64_t n, int ninst, int leaf_size, int max_level, bool full)
{
    const int64_t roots = 20 * (int64_t)ninst, per = n / ((int64_t)leaf_size + 1);
    int64_t b = roots, w = roots;
    for (int l = 0; l < max_level; l++) {
        b += 4 * std::min(w, per);
        w = std::min(w * 4, per + 1);
    }
    return full ? b + 64 : std::min(b, roots + 12 * per) + 64;
}

int tree_build(sts_ctx* c, const double* pos, int64_t n, const int64_t* inst_off, int ninst, int leaf_size,
               int max_level, cudaStream_t s)
{
    c->have_tree = false;
    c->have_lists = false;
    c->have_dual = false;
    c->up_degree = -1;
    c->n = n;
    c->leaf_size = leaf_size;
    c->max_level = max_level;
    c->level_begin.clear();
    c->nnodes = c->nleaves = c->deepest = 0;
    if (n == 0) {
        c->level_begin.push_back(0);
        c->have_tree = true;
        return STS_OK;
    }
    if (!c->consts_ok) {  // the icosahedron tables, uploaded once (never while recording)
        c->consts_ok = true;
        double V[12][3], C[20][3], FV[20][3][3];
        int F[20][3];
        icosahedron(V, F, C);
        for (int f = 0; f < 20; f++)
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) FV[f][a][b] = V[F[f][a]][b];
        STS_CUDA(cudaMemcpyToSymbolAsync(c_fc, C, sizeof(C), 0, cudaMemcpyHostToDevice, s));
        STS_CUDA(cudaMemcpyToSymbolAsync(c_fv, FV, sizeof(FV), 0, cudaMemcpyHostToDevice, s));
        float C32[20][3];
        for (int f = 0; f < 20; f++)
            for (int a = 0; a < 3; a++) C32[f][a] = (float)C[f][a];
        STS_CUDA(cudaMemcpyToSymbolAsync(c_fc32, C32, sizeof(C32), 0, cudaMemcpyHostToDevice, s));
    }
    STS_CUDA(c->pos.reserve(3 * n));
    STS_CUDA(c->nodeof.reserve(n));
    STS_CUDA(c->posf.reserve(n));
    STS_CUDA(c->digit.reserve(n));
    STS_CUDA(c->perm.reserve(n));
    STS_CUDA(c->perm_tmp.reserve(n));
    STS_CUDA(c->skey.reserve(n));
    STS_CUDA(c->skey_tmp.reserve(n));
    STS_CUDA(c->flags.reserve(n + 1));
    STS_CUDA(c->offs.reserve(n + 1));
    STS_CUDA(c->slot_leaf.reserve(n));
    STS_CUDA(c->leaves.reserve(n + 1));
    STS_CUDA(c->counters.reserve(64));
    STS_CUDA(c->small.reserve(16));
    const int32_t nkeys = 20 * ninst;
    // node capacity: while recording, the planned one; eagerly an estimate, raised to the
    // proven bound (and the build redone) if a level runs out of it
    if (grow_nodes(c, c->capturing ? nkeys + 80 : std::max(c->node_hint, tree_node_bound(n, ninst, leaf_size, max_level, false)), 0, s))
        return STS_ERR_CUDA;
    STS_CUDA(c->root_cnt.reserve(nkeys + 2));
    STS_CUDA(c->face_node.reserve(nkeys + 1));
    c->ninst = ninst;

    const int T = 256;
    // the per-key counts and, right after them, the tree launch's grid-barrier counter: one
    // memset (the sort launch's counter, next, is cleared by the tree launch)
    STS_CUDA(cudaMemsetAsync(c->root_cnt.p, 0, (nkeys + 1) * sizeof(int32_t), s));
    int64_t* dc = c->dc.p;
    const bool cap = c->capturing;  // recording a graph: no host reads, planned capacities
    if (!cap) STS_CUDA(cudaMemsetAsync(dc + kDcOver, 0, sizeof(int64_t), s));
    // faces, roots and levels: one cooperative launch (its CTAs wait on one another at grid-wide
    // barriers)
    if (c->build_grid == 0) {  // both launches co-resident at this grid
        int per_sm = 0, per_sm2 = 0;
        STS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_build_levels, kBuildThreads, 0));
        STS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, k_build_sort, kBuildThreads, 0));
        c->build_grid = std::max(1, std::min(std::min(per_sm, per_sm2), 4)) * c->num_sms;
    }
    STS_CUDA(c->bld_tot.reserve(3 * (size_t)c->build_grid));
    if (!cap) {  // the cluster table for every node the capacity allows; the moment tasks for
                 // the largest count possible: a cluster holds more than N_T particles of one
                 // level, so there are at most (levels) n / kUpChunk + (clusters) tasks
        const int64_t nc = (int64_t)c->nd_level.cap;
        STS_CUDA(c->cluster_slot.reserve(nc + 1));
        STS_CUDA(c->cluster_node.reserve(nc + 1));
        STS_CUDA(c->up_toff.reserve(nc + 2));
        STS_CUDA(c->up_frame.reserve(12 * nc + 12));
        STS_CUDA(c->up_frame32.reserve(18 * nc + 18));
        STS_CUDA(c->up_tasks.reserve((int64_t)(max_level + 1) * (n / kUpChunk + 1) + nc + 1));
    }
    STS_CUDA(c->hist.reserve(256 * (size_t)c->build_grid + 256));
    BuildArgs a;
    a.lvl = dc + kDcLevel;
    a.inst_off = inst_off;
    a.ninst = ninst;
    a.face_count = c->root_cnt.p;
    a.face_node = c->face_node.p;
    // eagerly every level up to the depth limit (the last one never splits); while recording,
    // the planned number of levels plus one that must come out empty
    a.nlev = cap ? std::min(c->plan.depth + 2, max_level + 1) : max_level + 1;
    a.leaf_size = leaf_size;
    a.max_level = max_level;
    // nodes the node table and every node-indexed buffer of the cluster table can hold
    // (while recording, also the recorded node count the later kernels are sized for)
    a.cap = std::min<int64_t>({(int64_t)c->nd_level.cap, (int64_t)c->cluster_slot.cap - 1,
                               (int64_t)c->cluster_node.cap - 1, (int64_t)c->up_toff.cap - 2,
                               (int64_t)c->up_frame.cap / 12 - 1, (int64_t)c->up_frame32.cap / 18 - 1,
                               cap ? c->nodes_rec : INT64_MAX});
    a.pos_in = pos;
    a.pos = c->pos.p;
    a.posf = c->posf.p;
    a.n = n;
    a.nodeof = c->nodeof.p;
    a.digit = c->digit.p;
    a.level = c->nd_level.p;
    a.parent = c->nd_parent.p;
    a.first_child = c->nd_first_child.p;
    a.nchild = c->nd_nchild.p;
    a.start = c->nd_start.p;
    a.count = c->nd_count.p;
    a.leaf = c->nd_leaf.p;
    a.cc = c->nd_cc.p;
    a.cc_stride = 4 * (int64_t)c->nd_level.cap;
    a.child = c->nd_child.p;
    a.key = c->nd_key.p;
    a.geom = c->nd_geom.p;
    a.norm = c->nd_norm.p;
    a.mid = c->nd_mid.p;
    a.norm32 = c->nd_norm32.p;
    a.c32 = c->nd_c32.p;
    a.over = dc + kDcOver;
    a.nnodes = dc + kDcNodes;
    a.tot = c->bld_tot.p;
    a.bar = reinterpret_cast<unsigned*>(c->root_cnt.p + nkeys);
    a.bar2 = reinterpret_cast<unsigned*>(c->root_cnt.p + nkeys + 1);
    a.mark = reinterpret_cast<int32_t*>(c->skey_tmp.p);  // free until the sort launch
    a.status = c->d_status;
    int bits = 0;
    while (bits < 32 && ((int64_t)1 << bits) < n) bits++;
    a.sort_passes = (bits + 7) / 8;
    a.perm = c->perm.p;
    a.perm_tmp = c->perm_tmp.p;
    a.skey = c->skey.p;
    a.skey_tmp = c->skey_tmp.p;
    a.hist = (int32_t*)c->hist.p;
    a.leaves = c->leaves.p;
    a.slot_leaf = c->slot_leaf.p;
    a.nleaves = dc + kDcLeaves;
    a.cluster_slot = c->cluster_slot.p;
    a.cluster_node = c->cluster_node.p;
    a.up_toff = c->up_toff.p;
    a.up_tasks = reinterpret_cast<int2*>(c->up_tasks.p);
    // while recording, the tasks the upward pass's grid covers; eagerly, the whole buffer
    a.up_cap = cap ? std::min<int64_t>((int64_t)c->up_tasks.cap, c->up_tasks_rec) : (int64_t)c->up_tasks.cap;
    a.up_frame = c->up_frame.p;
    a.up_frame32 = c->up_frame32.p;
    a.nclusters = dc + kDcClusters;
    a.nuptasks = dc + kDcUpTasks;
    {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)c->build_grid);
        cfg.blockDim = dim3(kBuildThreads);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeCooperative;
        at[0].val.cooperative = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        STS_CUDA(cudaLaunchKernelEx(&cfg, k_build_levels, a));
        note_launch();
        // the tree is complete here: the interaction lists may start (sources_and_lists)
        STS_CUDA(cudaEventRecord(c->ev_tree, s));
        c->tree_event = true;
        STS_CUDA(cudaLaunchKernelEx(&cfg, k_build_sort, a));
        note_launch();
    }
    if (!cap) {
        // one read of the counters: errors, node overflow (redo with the proven bound), levels
        STS_CUDA(cudaMemcpyAsync(c->h_pinned, dc, kDcSize * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        STS_CUDA(cudaMemcpyAsync(c->h_pinned + kDcSize, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
        STS_CUDA(cudaStreamSynchronize(s));
        const int64_t* h = c->h_pinned;
        const int st = ((const int32_t*)(h + kDcSize))[0];
        if (st & (kStatusNonfinite | kStatusTimeout)) {
            STS_CUDA(cudaMemsetAsync(c->d_status, 0, sizeof(int), s));
            if (st & kStatusNonfinite) {
                set_error("sts_tree_build: non-finite position");
                return STS_ERR_NONFINITE;
            }
            set_error("sts_tree_build: a grid-wide barrier of the level build gave up");
            return STS_ERR_TIMEOUT;
        }
        if (h[kDcOver] & 1) {
            const int64_t bound = tree_node_bound(n, ninst, leaf_size, max_level, true);
            if (c->node_hint >= bound) {
                set_error("sts_tree_build: node capacity %lld exhausted", (long long)bound);
                return STS_ERR_CUDA;
            }
            c->node_hint = bound;
            return tree_build(c, pos, n, inst_off, ninst, leaf_size, max_level, s);
        }
        if (h[kDcOver] & 4) {  // the moment tasks are sized by a proven bound: not expected
            set_error("sts_tree_build: moment task capacity %lld exhausted", (long long)c->up_tasks.cap);
            return STS_ERR_CAPACITY;
        }
        c->nnodes = h[kDcNodes];
        c->nleaves = h[kDcLeaves];
        c->nclusters = h[kDcClusters];
        c->n_up_tasks = h[kDcUpTasks];
        c->plan.clusters = std::max(c->plan.clusters, c->nclusters);
        c->plan.leaves = std::max(c->plan.leaves, c->nleaves);
        c->plan.up_tasks = std::max(c->plan.up_tasks, c->n_up_tasks);
        c->level_begin.assign(1, 0);
        c->deepest = 0;
        for (int l = 1; l <= kMaxLevel + 2 && h[kDcLevel + l] > h[kDcLevel + l - 1]; l++) {
            c->level_begin.push_back(h[kDcLevel + l]);
            c->deepest = l - 1;
        }
        c->plan.nodes = std::max(c->plan.nodes, c->nnodes);
        c->plan.depth = std::max(c->plan.depth, (int)c->deepest);
    } else {
        c->nnodes = -1;  // known after the graph runs
        c->deepest = -1;
        c->nclusters = c->n_up_tasks = c->nleaves = -1;
    }

    c->have_tree = true;
    return STS_OK;
}

// Targets per warp task: kTaskTargets, or fewer for small problems, where tasks of 64 targets
// would leave most of the evaluation kernel's resident warps (16 per SM) idle: about two tasks
// per resident warp, at least 8 targets per task (four pairs of eight lanes), a multiple of 8.
static int task_targets(const sts_ctx* c)
{
    const int64_t warps = 16 * (int64_t)c->num_sms;
    const int64_t want = (c->n + 2 * warps - 1) / (2 * warps);
    return (int)std::min<int64_t>(kTaskTargets, std::max<int64_t>(8, (want + 7) / 8 * 8));
}

int build_lists(sts_ctx* c, double theta, cudaStream_t s)
{
    c->have_lists = false;
    c->have_dual = false;  // the leaf lists no longer hold the dual traversal's PP / PC pairs
    const bool cap = c->capturing;
    // leaf count, or while recording its planned bound (a replay with more leaves sets the
    // overflow bit in k_list_totals and is redone)
    const int64_t L = cap ? std::min<int64_t>(c->n, c->plan.leaves + c->plan.leaves / 4 + 64) : c->nleaves;
    const int lcap = theta >= 0.6 ? 256 : 512;  // terminals per leaf held by the warp traversal
    const int T = 128;
    int64_t* dc = c->dc.p;
    if (!cap) {
        STS_CUDA(c->list_cnt.reserve(3 * L + 3));
        STS_CUDA(c->far_off.reserve(L + 1));
        STS_CUDA(c->near_off.reserve(L + 1));
        STS_CUDA(c->near_coff.reserve(L + 1));
        STS_CUDA(c->flags.reserve(L + 1));
        STS_CUDA(c->offs.reserve(L + 1));
        STS_CUDA(c->scan_tmp.reserve(scan_scratch(L + 1) + 8));
        if (scan_state_reserve(c->scan_state_side, std::max<int64_t>(c->n, L) + 1, s)) return STS_ERR_CUDA;
    }
    int64_t* far_po = c->far_off.p;
    int64_t* near_po = c->near_off.p;
    int64_t* chunk_po = c->near_coff.p;
    STS_CUDA(c->wover.reserve(L + 1));
    STS_CUDA(c->lw_terms.reserve(L * lcap + 1));
    const unsigned g = blocks(std::max<int64_t>(L, 1), T);
    const unsigned gw = blocks(std::max<int64_t>(L, 1), kLwWarps);
    // counts: one warp per leaf; leaves whose traversal overflows the warp's shared memory are
    // counted (and later filled) by the per-thread traversal
    (lcap == 256 ? k_lists_count<256> : k_lists_count<512>)<<<gw, kLwWarps * 32, 0, s>>>(
        dc + kDcLeaves, c->leaves.p, c->face_node.p, c->nd_key.p, c->nd_level.p, theta, c->leaf_size, c->nd_geom.p,
        c->nd_c32.p, c->nd_leaf.p, c->nd_first_child.p, c->nd_nchild.p, c->nd_count.p, c->list_cnt.p,
        c->lw_terms.p, L, c->wover.p);
    note_launch();
    (k_lists<<<g, T, 0, s>>>(0, dc + kDcLeaves, c->leaves.p, c->face_node.p, c->nd_key.p, c->nd_level.p, theta,
                             c->leaf_size, c->nd_geom.p, c->nd_c32.p, c->nd_leaf.p, c->nd_first_child.p,
                             c->nd_nchild.p, c->nd_start.p, c->nd_count.p, c->cluster_slot.p, c->list_cnt.p, nullptr,
                             nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0, 0, 0, L, c->wover.p,
                             c->d_status, dc + kDcOver), note_launch());  // list_cnt: three rows of stride L
    exclusive_scan_i32(c->list_cnt.p, far_po, L, c->scan_state_side, s, c->d_status, dc + kDcLeaves);
    exclusive_scan_i32(c->list_cnt.p + L, near_po, L, c->scan_state_side, s, c->d_status, dc + kDcLeaves);
    exclusive_scan_i32(c->list_cnt.p + 2 * L, chunk_po, L, c->scan_state_side, s, c->d_status, dc + kDcLeaves);
    // evaluation tasks: each leaf's targets split into warp tasks
    STS_CUDA(cudaMemsetAsync(dc + kDcClass, 0, 16 * sizeof(int64_t), s));
    (k_task_count<<<g, T, 0, s>>>(dc + kDcLeaves, L, c->leaves.p, c->nd_count.p, task_targets(c),
                                  (unsigned long long*)(dc + kDcClass)), note_launch());
    (k_list_totals<<<1, 32, 0, s>>>(dc, far_po, near_po, chunk_po, L), note_launch());
    STS_LAUNCH_CHECK();
    if (!cap) {
        STS_CUDA(cudaMemcpyAsync(c->h_pinned, dc, 16 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        STS_CUDA(cudaMemcpyAsync(c->h_pinned + 16, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
        STS_CUDA(cudaStreamSynchronize(s));
        if (((int32_t*)(c->h_pinned + 16))[0] & kStatusCapacity) {
            STS_CUDA(cudaMemsetAsync(c->d_status, 0, sizeof(int), s));
            set_error("interaction lists: traversal stack overflow");
            return STS_ERR_CAPACITY;
        }
        c->nfar = c->h_pinned[kDcFar];
        c->nnear = c->h_pinned[kDcNear];
        c->nnear_chunks = c->h_pinned[kDcChunks];
        c->ntasks = c->h_pinned[kDcTasks];
        c->plan.far = std::max(c->plan.far, c->nfar);
        c->plan.near = std::max(c->plan.near, c->nnear);
        c->plan.chunks = std::max(c->plan.chunks, c->nnear_chunks);
        c->plan.tasks = std::max(c->plan.tasks, c->ntasks);
        STS_CUDA(c->far_idx.reserve(c->nfar + 1));
        STS_CUDA(c->near_idx.reserve(c->nnear + 1));
        STS_CUDA(c->far_ent.reserve(c->nfar + 1));
        STS_CUDA(c->near_ent.reserve(c->nnear_chunks + 1));
        STS_CUDA(c->tasks.reserve(c->ntasks + 1));
    } else {
        c->nfar = c->nnear = c->nnear_chunks = c->ntasks = -1;
    }
    (lcap == 256 ? k_lists_fill<256> : k_lists_fill<512>)<<<gw, kLwWarps * 32, 0, s>>>(
        dc + kDcLeaves, c->leaves.p, c->nd_key.p, c->nd_level.p, c->nd_geom.p, c->nd_start.p, c->nd_count.p,
        c->cluster_slot.p, c->lw_terms.p, far_po, near_po, chunk_po, c->far_idx.p, c->near_idx.p, c->far_ent.p,
        c->near_ent.p, (int64_t)c->far_ent.cap, (int64_t)c->near_idx.cap, (int64_t)c->near_ent.cap, L, c->wover.p,
        dc + kDcOver);
    note_launch();
    (k_lists<<<g, T, 0, s>>>(1, dc + kDcLeaves, c->leaves.p, c->face_node.p, c->nd_key.p, c->nd_level.p, theta,
                             c->leaf_size, c->nd_geom.p, c->nd_c32.p, c->nd_leaf.p, c->nd_first_child.p,
                             c->nd_nchild.p, c->nd_start.p, c->nd_count.p, c->cluster_slot.p, nullptr, far_po, near_po,
                             chunk_po, c->far_idx.p, c->near_idx.p, c->far_ent.p, c->near_ent.p,
                             (int64_t)c->far_ent.cap, (int64_t)c->near_idx.cap, (int64_t)c->near_ent.cap, L,
                             c->wover.p, c->d_status, dc + kDcOver), note_launch());
    (k_task_fill<<<g, T, 0, s>>>(dc + kDcLeaves, L, c->leaves.p, c->nd_start.p, c->nd_count.p, task_targets(c),
                                 dc + kDcClass, (unsigned long long*)(dc + kDcClassFill), (int64_t)c->tasks.cap,
                                 c->tasks.p, dc + kDcOver), note_launch());
    STS_LAUNCH_CHECK();
    c->list_theta = theta;
    c->have_lists = true;
    return STS_OK;
}

// Capacities of the dual traversal's buffers.
struct DualCaps {
    int64_t front, terms, pc, pp, pp_chunks, cc, cp, cp_chunks;
    int levels;
};

static int bits_for(int64_t n)
{
    int b = 0;
    while (b < 31 && ((int64_t)1 << b) < n) b++;
    return b;
}

// Capacities from the plan (the largest sizes seen by eager runs), with slack; eager runs
// start from estimates and grow on overflow.
static DualCaps dual_caps(const sts_ctx* c, int64_t L, int64_t C, int64_t nodes)
{
    auto g = [](int64_t v, int64_t add) { return v + v / 4 + add; };
    const Plan& pl = c->plan;
    DualCaps k;
    k.front = std::max(g(pl.dual_front, 1024), 400 * (int64_t)c->ninst + 4 * nodes);
    k.terms = std::max(g(pl.dual_terms, 1024), 40 * L + 16 * C + 1024);
    k.pp = std::max(g(pl.dual_pairs[kPP], 256), k.terms / 2);
    k.pc = std::max(g(pl.dual_pairs[kPC], 256), 8 * L + 256);
    k.cp = std::max(g(pl.dual_pairs[kCP], 256), 16 * C + 256);
    k.cc = std::max(g(pl.dual_pairs[kCC], 256), 16 * C + 256);
    k.pp_chunks = std::max(g(pl.dual_chunks[0], 256), k.pp);
    k.cp_chunks = std::max(g(pl.dual_chunks[1], 256), k.cp);
    k.levels = 0;
    return k;
}

static int reserve_dual(sts_ctx* c, const DualCaps& k, int64_t L, int64_t C, int64_t nodes)
{
    STS_CUDA(c->dual_cnt.reserve(kDuSize + 8));
    STS_CUDA(c->dual_ft.reserve(k.front));
    STS_CUDA(c->dual_fs.reserve(k.front));
    STS_CUDA(c->dual_gt.reserve(k.front));
    STS_CUDA(c->dual_gs.reserve(k.front));
    STS_CUDA(c->dual_tt.reserve(k.terms));
    STS_CUDA(c->dual_ts.reserve(k.terms));
    STS_CUDA(c->dual_tk.reserve(k.terms));
    STS_CUDA(c->dual_t.reserve(k.terms));
    STS_CUDA(c->dual_s.reserve(k.terms));
    STS_CUDA(c->dual_key.reserve(k.terms));
    STS_CUDA(c->dual_ktmp.reserve(k.terms));
    STS_CUDA(c->dual_perm.reserve(k.terms));
    STS_CUDA(c->dual_ptmp.reserve(k.terms));
    STS_CUDA(c->dual_chunk.reserve(k.terms));
    STS_CUDA(c->dual_scan.reserve(k.terms + 1));
    const int64_t KT = std::max<int64_t>(std::max(L, C), 1);
    STS_CUDA(c->dual_bkt.reserve(k.terms));
    STS_CUDA(c->dual_bcnt.reserve(4 * KT + 1));
    STS_CUDA(c->dual_boff.reserve(4 * KT + 2));
    STS_CUDA(c->scan_tmp.reserve(scan_scratch(4 * KT + 1) + scan_scratch(k.terms + 1) + scan_scratch(nodes + 1) + 64));
    // the traversal's scans run on the side stream: its state, zeroed there
    if (scan_state_reserve(c->scan_state_side, std::max<int64_t>(4 * KT, k.terms) + 1, c->side)) return STS_ERR_CUDA;
    STS_CUDA(c->far_off.reserve(L + 1));
    STS_CUDA(c->near_off.reserve(L + 1));
    STS_CUDA(c->near_coff.reserve(L + 1));
    STS_CUDA(c->far_idx.reserve(k.pc));
    STS_CUDA(c->far_ent.reserve(k.pc));
    STS_CUDA(c->near_idx.reserve(k.pp));
    STS_CUDA(c->near_ent.reserve(k.pp_chunks));
    STS_CUDA(c->cfar_off.reserve(C + 1));
    STS_CUDA(c->cnear_off.reserve(C + 1));
    STS_CUDA(c->cnear_coff.reserve(C + 1));
    STS_CUDA(c->cfar_ent.reserve(k.cc));
    STS_CUDA(c->cnear_ent.reserve(k.cp_chunks));
    STS_CUDA(c->tasks.reserve(c->n / task_targets(c) + 4 * L + 64));  // task_split's bound per leaf
    STS_CUDA(c->chas.reserve(C + 1));
    return STS_OK;
}

// Every launch of the traversal, sort and list construction; no host access.
// k: the capacities reserve_dual sized the buffers for (every buffer holds at least that many).
static int launch_dual(sts_ctx* c, double theta, int levels, int64_t L, int64_t C, int64_t nodes,
                       const DualCaps& k, unsigned long long* over, cudaStream_t s)
{
    const int T = 256;
    int64_t* du = c->dual_cnt.p;
    int64_t* dc = c->dc.p;
    const int64_t fcap = k.front, tcap = k.terms;
    STS_CUDA(cudaMemsetAsync(du, 0, kDuSize * sizeof(int64_t), s));
    (k_dual_roots<<<blocks(400 * (int64_t)c->ninst, T), T, 0, s>>>(c->face_node.p, c->ninst, c->dual_ft.p,
                                                                  c->dual_fs.p, fcap, du, over), note_launch());
    const unsigned gf = blocks(fcap, T);
    for (int l = 0; l < levels; l++) {
        const bool even = (l & 1) == 0;
        (k_dual_level<<<gf, T, 0, s>>>(l, even ? c->dual_ft.p : c->dual_gt.p, even ? c->dual_fs.p : c->dual_gs.p,
                                       even ? c->dual_gt.p : c->dual_ft.p, even ? c->dual_gs.p : c->dual_fs.p, fcap,
                                       theta, c->leaf_size, c->nd_geom.p, c->nd_c32.p, c->nd_leaf.p,
                                       c->nd_first_child.p, c->nd_nchild.p, c->nd_count.p, c->dual_tt.p, c->dual_ts.p,
                                       c->dual_tk.p, tcap, du, over),
         note_launch());
    }
    (k_dual_close<<<1, 32, 0, s>>>(levels, tcap, du, over), note_launch());
    // sort by (kind, target key, source): counting sort on (kind, target key), then the rank
    // of each pair within its bucket by source
    const int64_t KT = std::max<int64_t>(std::max(L, C), 1);
    const int bits_t = bits_for(KT);
    const unsigned gt = blocks(tcap, T);
    STS_CUDA(cudaMemsetAsync(c->dual_bcnt.p, 0, 4 * KT * sizeof(int32_t), s));
    (k_dual_bucket<<<gt, T, 0, s>>>(c->dual_tt.p, c->dual_tk.p, du, tcap, KT, c->nd_start.p, c->slot_leaf.p,
                                    c->cluster_slot.p, c->dual_bkt.p, c->dual_bcnt.p, c->dual_ptmp.p),
     note_launch());
    exclusive_scan_i32(c->dual_bcnt.p, c->dual_boff.p, 4 * KT, c->scan_state_side, s, c->d_status);
    (k_dual_scatter<<<gt, T, 0, s>>>(du, tcap, c->dual_bkt.p, c->dual_ptmp.p, c->dual_boff.p, c->dual_ts.p,
                                     c->dual_ktmp.p, c->dual_chunk.p),
     note_launch());
    (k_dual_rank<<<gt, T, 0, s>>>(du, tcap, KT, bits_t, c->dual_bkt.p, c->dual_boff.p, c->dual_bcnt.p, c->dual_ts.p,
                                  c->dual_ktmp.p, c->dual_chunk.p, c->dual_key.p, c->dual_perm.p),
     note_launch());
    (k_dual_gather<<<gt, T, 0, s>>>(c->dual_tt.p, c->dual_ts.p, c->dual_perm.p, c->dual_key.p, bits_t, du, tcap,
                                    c->nd_count.p, c->dual_t.p, c->dual_s.p, c->dual_chunk.p), note_launch());
    exclusive_scan_i32(c->dual_chunk.p, c->dual_scan.p, tcap, c->scan_state_side, s, c->d_status, du + kDuP);
    // CSR per kind, then the entries
    DualCsr csr;
    csr.off[kPP] = c->near_off.p;
    csr.coff[kPP] = c->near_coff.p;
    csr.off[kPC] = c->far_off.p;
    csr.coff[kPC] = nullptr;
    csr.off[kCP] = c->cnear_off.p;
    csr.coff[kCP] = c->cnear_coff.p;
    csr.off[kCC] = c->cfar_off.p;
    csr.coff[kCC] = nullptr;
    const dim3 gc(blocks(std::max(L, C) + 1, T), 4);
    (k_dual_csr<<<gc, T, 0, s>>>(c->dual_key.p, c->dual_scan.p, bits_t, dc, L, C, csr, du), note_launch());
    DualFill fo;
    fo.far[0] = c->far_ent.p;
    fo.far[1] = c->cfar_ent.p;
    fo.near[0] = c->near_ent.p;
    fo.near[1] = c->cnear_ent.p;
    fo.idx[0] = c->near_idx.p;
    fo.idx[1] = c->far_idx.p;
    fo.far_cap[0] = (int64_t)c->far_ent.cap;
    fo.far_cap[1] = (int64_t)c->cfar_ent.cap;
    fo.near_cap[0] = (int64_t)c->near_ent.cap;
    fo.near_cap[1] = (int64_t)c->cnear_ent.cap;
    fo.idx_cap[0] = (int64_t)c->near_idx.cap;
    fo.idx_cap[1] = (int64_t)c->far_idx.cap;
    (k_dual_fill<<<gt, T, 0, s>>>(c->dual_key.p, c->dual_t.p, c->dual_s.p, c->dual_scan.p, bits_t, du, tcap,
                                  c->nd_geom.p, c->nd_start.p, c->nd_count.p, c->cluster_slot.p, fo, over),
     note_launch());
    // evaluation tasks of the target leaves (as for the leaf lists) and the list totals
    const unsigned g = blocks(std::max<int64_t>(L, 1), 128);
    STS_CUDA(cudaMemsetAsync(dc + kDcClass, 0, 16 * sizeof(int64_t), s));
    (k_task_count<<<g, 128, 0, s>>>(dc + kDcLeaves, L, c->leaves.p, c->nd_count.p, task_targets(c),
                                    (unsigned long long*)(dc + kDcClass)), note_launch());
    (k_list_totals<<<1, 32, 0, s>>>(dc, c->far_off.p, c->near_off.p, c->near_coff.p, L), note_launch());
    (k_task_fill<<<g, 128, 0, s>>>(dc + kDcLeaves, L, c->leaves.p, c->nd_start.p, c->nd_count.p, task_targets(c),
                                   dc + kDcClass, (unsigned long long*)(dc + kDcClassFill), (int64_t)c->tasks.cap,
                                   c->tasks.p, dc + kDcOver), note_launch());
    STS_LAUNCH_CHECK();
    return STS_OK;
}

int build_dual(sts_ctx* c, double theta, cudaStream_t s)
{
    c->have_dual = false;
    c->have_lists = false;  // the leaf lists are replaced by the PP / PC pairs
    for (int k = 0; k < 4; k++) c->dual_n[k] = -1;
    const bool cap = c->capturing;
    // leaf, cluster and node counts, or while recording their planned bounds (a replay that
    // exceeds them sets the overflow bit and is redone)
    const int64_t L = cap ? std::min<int64_t>(c->n, c->plan.leaves + c->plan.leaves / 4 + 64) : c->nleaves;
    const int64_t C = cap ? c->nodes_rec : c->nclusters;
    const int64_t nodes = cap ? c->nodes_rec : c->nnodes;
    const int depth = cap ? c->plan.depth : (int)c->deepest;
    // a pair's two levels each grow by one per refinement, up to the deepest level: at most
    // 2 depth + 1 levels, the last of which only has terminals
    const int levels = std::min(2 * depth + 2, kDuMaxLevels);
    if (cap) {
        const int rc = launch_dual(c, theta, levels, L, C, nodes, dual_caps(c, L, C, nodes),
                                   (unsigned long long*)(c->dc.p + kDcOver), s);
        if (rc) return rc;
        c->nfar = c->nnear = c->nnear_chunks = c->ntasks = -1;
        c->dual_theta = theta;
        c->have_dual = true;
        return STS_OK;
    }
    DualCaps k = dual_caps(c, L, C, nodes);
    for (int attempt = 0;; attempt++) {
        int rc = reserve_dual(c, k, L, C, nodes);
        if (rc) return rc;
        unsigned long long* over = (unsigned long long*)(c->dual_cnt.p + kDuOver);
        if ((rc = launch_dual(c, theta, levels, L, C, nodes, k, over, s))) return rc;
        int64_t* h = c->h_pinned;
        STS_CUDA(cudaMemcpyAsync(h, c->dual_cnt.p, 16 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        STS_CUDA(cudaMemcpyAsync(h + 16, c->dc.p, 16 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        STS_CUDA(cudaStreamSynchronize(s));
        const int64_t P = h[kDuP];
        int64_t n4[4];
        for (int q = 0; q < 4; q++) n4[q] = h[kDuStart + q + 1] - h[kDuStart + q];
        const bool over_hit = h[kDuOver] != 0 || (h[16 + kDcOver] & 4) != 0;
        if (!over_hit) {
            for (int q = 0; q < 4; q++) c->dual_n[q] = n4[q];
            Plan& pl = c->plan;
            pl.dual_front = std::max(pl.dual_front, h[kDuFrontMax]);
            pl.dual_terms = std::max(pl.dual_terms, P);
            for (int q = 0; q < 4; q++) pl.dual_pairs[q] = std::max(pl.dual_pairs[q], n4[q]);
            pl.dual_chunks[0] = std::max(pl.dual_chunks[0], h[kDuChunks]);
            pl.dual_chunks[1] = std::max(pl.dual_chunks[1], h[kDuChunks + 1]);
            c->nfar = h[16 + kDcFar];
            c->nnear = h[16 + kDcNear];
            c->nnear_chunks = h[16 + kDcChunks];
            c->ntasks = h[16 + kDcTasks];
            pl.far = std::max(pl.far, c->nfar);
            pl.near = std::max(pl.near, c->nnear);
            pl.chunks = std::max(pl.chunks, c->nnear_chunks);
            pl.tasks = std::max(pl.tasks, c->ntasks);
            break;
        }
        if (attempt >= 8) {
            set_error("dual traversal: buffers keep overflowing");
            return STS_ERR_CAPACITY;
        }
        // grow what overflowed (the counters saw every attempted write) and run it again
        STS_CUDA(cudaMemsetAsync(c->dc.p + kDcOver, 0, sizeof(int64_t), s));
        auto g = [](int64_t v) { return v + v / 2 + 1024; };
        k.front = std::max(k.front, g(h[kDuFrontMax]));
        k.terms = std::max(k.terms, g(h[kDuTerms]));
        if (P == h[kDuTerms]) {  // the sort ran on every pair: the kind counts are exact
            k.pp = std::max(k.pp, g(n4[kPP]));
            k.pc = std::max(k.pc, g(n4[kPC]));
            k.cp = std::max(k.cp, g(n4[kCP]));
            k.cc = std::max(k.cc, g(n4[kCC]));
            k.pp_chunks = std::max(k.pp_chunks, g(h[kDuChunks]));
            k.cp_chunks = std::max(k.cp_chunks, g(h[kDuChunks + 1]));
        }
    }
    c->dual_theta = theta;
    c->have_dual = true;
    return STS_OK;
}

int reserve_dual_for_capture(sts_ctx* c, int degree, cudaStream_t s)
{
    (void)s;
    const int64_t L = std::min<int64_t>(c->n, c->plan.leaves + c->plan.leaves / 4 + 64);
    const int64_t C = c->nodes_rec, nodes = c->nodes_rec;
    int rc = reserve_dual(c, dual_caps(c, L, C, nodes), L, C, nodes);
    if (rc) return rc;
    const int M = (degree + 1) * (degree + 2) / 2;
    STS_CUDA(c->ctasks.reserve(C * ((M + kTaskTargets - 1) / kTaskTargets + 3) + 1));
    STS_CUDA(c->cvel.reserve(3 * C * M + 3));
    STS_CUDA(c->cdown.reserve(3 * C * M + 3));
    STS_CUDA(c->cdown32.reserve(4 * C * M + 4));
    STS_CUDA(c->ccorr.reserve(3 * C * M + 3));
    STS_CUDA(c->cacc.reserve(C + 1));
    STS_CUDA(c->leaf_anc.reserve(L * (c->plan.depth + 2) + 1));
    return STS_OK;
}

int refresh_dual_counts(sts_ctx* c, cudaStream_t s)
{
    if (!c->have_dual || c->dual_n[0] >= 0) return STS_OK;
    STS_CUDA(cudaMemcpyAsync(c->h_pinned, c->dual_cnt.p, 16 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    STS_CUDA(cudaStreamSynchronize(s));
    for (int q = 0; q < 4; q++) c->dual_n[q] = c->h_pinned[kDuStart + q + 1] - c->h_pinned[kDuStart + q];
    return STS_OK;
}

int cluster_tasks(sts_ctx* c, int M, cudaStream_t s)
{
    const bool cap = c->capturing;
    const int64_t C = cap ? c->nodes_rec : c->nclusters;
    if (!cap) {
        STS_CUDA(c->chas.reserve(C + 1));
        STS_CUDA(c->ctasks.reserve(C * ((M + kTaskTargets - 1) / kTaskTargets + 3) + 1));
    }
    // task_split's bound: at most ceil(M / 64) + 3 tasks per cluster
    c->nctasks = std::min<int64_t>((int64_t)c->ctasks.cap, C * ((M + kTaskTargets - 1) / kTaskTargets + 3));
    STS_CUDA(cudaMemsetAsync(c->dual_cnt.p + kDuCTasks, 0, sizeof(int64_t), s));
    if (C > 0)
        (k_cluster_tasks<<<blocks(C, 128), 128, 0, s>>>(c->dc.p, C, c->cfar_off.p, c->cnear_off.p, M, c->chas.p,
                                                        c->ctasks.p, c->nctasks, c->dual_cnt.p,
                                                        (unsigned long long*)(c->dc.p + kDcOver)),
         note_launch());
    STS_LAUNCH_CHECK();
    return STS_OK;
}

const int64_t* cluster_task_count(sts_ctx* c) { return c->dual_cnt.p + kDuCTasks; }

int dual_stats(sts_ctx* c, int degree, int64_t* stats, cudaStream_t s)
{
    for (int k = 0; k < 5; k++) stats[k] = 0;
    if (!c->have_dual) return STS_OK;
    int rc = refresh_dual_counts(c, s);
    if (rc) return rc;
    STS_CUDA(cudaMemcpyAsync(c->h_pinned, c->dual_cnt.p, 16 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    STS_CUDA(cudaStreamSynchronize(s));
    int64_t first[4];
    for (int q = 0; q < 4; q++) first[q] = c->h_pinned[kDuStart + q];
    const int M = (degree + 1) * (degree + 2) / 2;
    STS_CUDA(c->d_stats.reserve(8));
    STS_CUDA(cudaMemsetAsync(c->d_stats.p, 0, 8 * sizeof(unsigned long long), s));
    const int T = 256;
    for (int k = 0; k < 4; k++)
        if (c->dual_n[k] > 0)
            (k_dual_count<<<blocks(c->dual_n[k], T), T, 0, s>>>(k, c->dual_t.p, c->dual_s.p, first[k], c->dual_n[k],
                                                                c->nd_count.p, nullptr, M, c->d_stats.p),
             note_launch());
    if (c->nclusters > 0) {
        // the clusters that are targets of CP or CC pairs (as the dual evaluation marks them)
        if ((rc = cluster_tasks(c, M, s))) return rc;
        (k_dual_count<<<blocks(c->nclusters, T), T, 0, s>>>(4, c->cluster_node.p, nullptr, 0, c->nclusters,
                                                            c->nd_count.p, c->chas.p, M, c->d_stats.p),
         note_launch());
    }
    STS_LAUNCH_CHECK();
    STS_CUDA(cudaMemcpyAsync(c->h_pinned, c->d_stats.p, 5 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    STS_CUDA(cudaStreamSynchronize(s));
    for (int k = 0; k < 5; k++) stats[k] = c->h_pinned[k];
    return STS_OK;
}

int dual_export(sts_ctx* c, int kind, int64_t* npairs, int32_t* tgt, int32_t* src, cudaStream_t s)
{
    int rc = refresh_dual_counts(c, s);
    if (rc) return rc;
    STS_CUDA(cudaMemcpyAsync(c->h_pinned, c->dual_cnt.p, 16 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    STS_CUDA(cudaStreamSynchronize(s));
    const int64_t first = c->h_pinned[kDuStart + kind], P = c->dual_n[kind];
    if (npairs) *npairs = P;
    if (tgt && P)
        STS_CUDA(cudaMemcpyAsync(tgt, c->dual_t.p + first, P * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    if (src && P)
        STS_CUDA(cudaMemcpyAsync(src, c->dual_s.p + first, P * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    STS_CUDA(cudaStreamSynchronize(s));
    return STS_OK;
}

}  // namespace sts
