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
//             their child.  The host reads the number of new nodes once per level.
//   sort      a stable radix sort by the first slot of each particle's leaf gives the
//             sorted order (leaves depth first, original order inside a leaf).
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
// Root key of every particle: instance b (from the instance offsets, b = 0 without them) times
// 20 plus its face; counts per root key.  The key goes to rkey[i].
__global__ void k_faces(const double* __restrict__ pos, int64_t n, const int64_t* __restrict__ inst_off,
                        int32_t ninst, int32_t* __restrict__ rkey, int32_t* __restrict__ face_count,
                        int* __restrict__ status)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = i < n;
    int best = 0, rk = 0;
    if (active) {
        const g3 x = gld(pos + 3 * i);
        if (!isfinite(x.x) || !isfinite(x.y) || !isfinite(x.z)) atomicOr(status, kStatusNonfinite);
        const float fx = (float)x.x, fy = (float)x.y, fz = (float)x.z;
        float b1 = fdot(fx, fy, fz, c_fc32[0][0], c_fc32[0][1], c_fc32[0][2]), b2 = -3.f;
        int fb = 0;
#pragma unroll 4
        for (int f = 1; f < 20; f++) {
            const float d = fdot(fx, fy, fz, c_fc32[f][0], c_fc32[f][1], c_fc32[f][2]);
            if (d > b1) {
                b2 = b1;
                b1 = d;
                fb = f;
            } else if (d > b2) {
                b2 = d;
            }
        }
        const float scale = fmaxf(1.f, fmaxf(fabsf(fx), fmaxf(fabsf(fy), fabsf(fz))));
        if (b1 - b2 > 4e-6f * scale) {
            best = fb;  // the FP32 winner leads by more than twice the FP32 error
        } else {
            double bd = gdot(x, gmk(c_fc[0][0], c_fc[0][1], c_fc[0][2]));
            for (int f = 1; f < 20; f++) {
                const double d = gdot(x, gmk(c_fc[f][0], c_fc[f][1], c_fc[f][2]));
                if (d > bd) {
                    bd = d;
                    best = f;
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
        rk = 20 * b + best;
        rkey[i] = rk;
    }
    agg_inc(face_count, rk, active);
}

// Root nodes for the non-empty (instance, face) keys in key order, one thread per key:
// id = number of non-empty keys before it, start = number of particles before it.
// face_node[key] = node id or -1.
__global__ void k_roots(int32_t nkeys, const int32_t* __restrict__ face_count, const int64_t* __restrict__ rid,
                        const int64_t* __restrict__ rstart, int32_t* __restrict__ face_node, int32_t* level,
                        uint64_t* key, int32_t* parent, int32_t* first_child, int32_t* nchild, int32_t* start,
                        int32_t* count, int32_t* leaf, double* geom)
{
    const int rk = blockIdx.x * blockDim.x + threadIdx.x;
    if (rk >= nkeys) return;
    const int c = face_count[rk];
    if (c == 0) {
        face_node[rk] = -1;
        return;
    }
    const int f = rk % 20;
    const int32_t id = (int32_t)rid[rk];
    face_node[rk] = id;
    level[id] = 0;
    key[id] = (uint64_t)rk;
    parent[id] = -1;
    first_child[id] = -1;
    nchild[id] = 0;
    start[id] = (int32_t)rstart[rk];
    count[id] = c;
    leaf[id] = 0;
    node_geometry(geom + 13 * (int64_t)id, gmk(c_fv[f][0][0], c_fv[f][0][1], c_fv[f][0][2]),
                  gmk(c_fv[f][1][0], c_fv[f][1][1], c_fv[f][1][2]),
                  gmk(c_fv[f][2][0], c_fv[f][2][1], c_fv[f][2][2]));
}

__global__ void k_root_flags(int32_t nkeys, const int32_t* __restrict__ face_count, int32_t* __restrict__ flags)
{
    const int rk = blockIdx.x * blockDim.x + threadIdx.x;
    if (rk < nkeys) flags[rk] = face_count[rk] > 0 ? 1 : 0;
}

__global__ void k_assign_roots(int64_t n, const int32_t* __restrict__ face_node, int32_t* __restrict__ nodeof)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) nodeof[i] = face_node[nodeof[i]];
}

// ------------------------------------------------------------------------- level l
// The level kernels read the node range of level l from the device array lvl: level l holds
// nodes [lvl[l], lvl[l + 1]).  Node kernels stride over that range, so any grid size works
// and the launches need no host-side count (the whole build can be captured in a graph).
//
// Level nodes, four lanes per node (the FP64 square roots and divisions are long dependent
// chains, so the work of one node is spread): lane a < 3 forms the edge midpoint m_a and the
// child-digit normal n_a = m_a x m_(a+2 mod 3); lane 3 the circumcentre and radius (levels
// below the roots).  Leaves get norm32.w = -1 (no digits).
__global__ void k_level_nodes(const int64_t* __restrict__ lvl, int l, int leaf_size, int max_level,
                              const int32_t* __restrict__ level, const int32_t* __restrict__ count,
                              double* __restrict__ geom, int32_t* __restrict__ leaf,
                              double* __restrict__ norm, float4* __restrict__ norm32, int32_t* __restrict__ cc,
                              double* __restrict__ mid)
{
    const int32_t lb = (int32_t)lvl[l], le = (int32_t)lvl[l + 1];
    const int64_t nt = ((int64_t)4 * (le - lb) + 31) & ~(int64_t)31;  // whole warps (shuffles below)
    const int lane = threadIdx.x & 31;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = lb + (int32_t)(t >> 2);
        const int a = (int)(t & 3);
        const bool valid = p < le;
        bool split = false;
        g3 m = gmk(0.0, 0.0, 0.0);
        if (valid) {
            double* g = geom + 13 * (int64_t)p;
            split = count[p] > leaf_size && level[p] < max_level;
            if (a == 3) {
                if (l > 0) node_geometry(g, gld(g), gld(g + 3), gld(g + 6));  // roots: k_roots
                leaf[p] = split ? 0 : 1;
                if (split)
                    cc[4 * p] = cc[4 * p + 1] = cc[4 * p + 2] = cc[4 * p + 3] = 0;
                else
                    norm32[3 * (int64_t)p] = make_float4(0.f, 0.f, 0.f, -1.f);  // w < 0: a leaf
            } else if (split) {
                // m_0 = unit(v1 + v2), m_1 = unit(v2 + v3), m_2 = unit(v3 + v1)
                const g3 va = gld(g + 3 * a), vb = gld(g + 3 * (a == 2 ? 0 : a + 1));
                m = gunit(gadd(va, vb));
                gst(mid + 9 * (int64_t)p + 3 * a, m);
            }
        }
        // m_(a+2 mod 3) from lane a + 2 (a = 0) or a - 1 (a = 1, 2) of the same node
        const int src = (lane & ~3) + (a == 0 ? 2 : a - 1);
        const g3 mp = gmk(__shfl_sync(kFull, m.x, src), __shfl_sync(kFull, m.y, src), __shfl_sync(kFull, m.z, src));
        if (valid && split && a < 3) {
            const g3 nv = gcross(m, mp);
            gst(norm + 9 * (int64_t)p + 3 * a, nv);
            const float thr = 1e-6f * (float)(fabs(nv.x) + fabs(nv.y) + fabs(nv.z));
            norm32[3 * (int64_t)p + a] = make_float4((float)nv.x, (float)nv.y, (float)nv.z, thr);
        }
    }
}

// Per particle: first the move of level l - 1 (a particle of a node of level l - 1 goes to
// the child its digit names; a leaf's child table points at itself), then the digit of its
// node if that node of level l splits (norm32.w >= 0), counted per (node, digit) in cc.  The
// loads of one particle form two dependent rounds (node, then child and normals).  Levels with
// at most kPrivNodes nodes count in shared memory first (one global add per counter and
// block): there every counter takes thousands of increments, which serialise in L2.
constexpr int kPrivNodes = 256;

__global__ void k_level_particles(const int64_t* __restrict__ lvl, int l, const double* __restrict__ pos,
                                  int64_t n, int32_t* __restrict__ nodeof, const double* __restrict__ norm,
                                  const float4* __restrict__ norm32, const int32_t* __restrict__ child,
                                  uint8_t* __restrict__ digit, int32_t* __restrict__ cc)
{
    __shared__ int32_t shc[4 * kPrivNodes];
    const int32_t lb = (int32_t)lvl[l], le = (int32_t)lvl[l + 1];
    const int32_t pb = l > 0 ? (int32_t)lvl[l - 1] : 0;
    const bool priv = le - lb <= kPrivNodes;
    if (priv) {
        for (int k = threadIdx.x; k < 4 * (le - lb); k += blockDim.x) shc[k] = 0;
        __syncthreads();
    }
    // kPU particles per thread and trip, their loads issued together round by round
    constexpr int kPU = 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t nr = (n + 31) & ~(int64_t)31;  // whole warps run every trip (warp-wide counting)
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < nr; i0 += kPU * stride) {
        int p[kPU], dg[kPU];
        float fx[kPU], fy[kPU], fz[kPU];
#pragma unroll
        for (int u = 0; u < kPU; u++) {
            const int64_t i = i0 + u * stride;
            p[u] = -1;
            dg[u] = 0;
            fx[u] = fy[u] = fz[u] = 0.f;
            if (i < n) {
                p[u] = nodeof[i];
                dg[u] = digit[i];
                fx[u] = (float)pos[3 * i];
                fy[u] = (float)pos[3 * i + 1];
                fz[u] = (float)pos[3 * i + 2];
            }
        }
#pragma unroll
        for (int u = 0; u < kPU; u++) {
            if (p[u] >= pb && p[u] < lb) {
                p[u] = child[4 * p[u] + dg[u]];
                nodeof[i0 + u * stride] = p[u];
            }
        }
        float4 q3[kPU][3];
#pragma unroll
        for (int u = 0; u < kPU; u++) {
            const int64_t pp = p[u] >= lb ? p[u] : 0;
#pragma unroll
            for (int a = 0; a < 3; a++) q3[u][a] = norm32[3 * pp + a];
        }
#pragma unroll
        for (int u = 0; u < kPU; u++) {
            const int64_t i = i0 + u * stride;
            const bool active = p[u] >= lb && q3[u][0].w >= 0.f;
            int d = 0;
            if (active) {
                const float scale = fmaxf(1.f, fmaxf(fabsf(fx[u]), fmaxf(fabsf(fy[u]), fabsf(fz[u]))));
                // digit = first a with n_a . x >= 0, else 3; decided in FP32 while unambiguous
                d = -1;
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    if (d != -1) continue;
                    const float t = fdot(q3[u][a].x, q3[u][a].y, q3[u][a].z, fx[u], fy[u], fz[u]);
                    const float thr = q3[u][a].w * scale;
                    if (t > thr)
                        d = a;
                    else if (!(t < -thr))
                        d = -2;  // too close to this boundary for FP32
                }
                if (d == -1) d = 3;
                if (d == -2) {
                    const g3 x = gld(pos + 3 * i);
                    const double* nn = norm + 9 * (int64_t)p[u];
                    if (gdot(gld(nn), x) >= 0.0)
                        d = 0;
                    else if (gdot(gld(nn + 3), x) >= 0.0)
                        d = 1;
                    else if (gdot(gld(nn + 6), x) >= 0.0)
                        d = 2;
                    else
                        d = 3;
                }
                digit[i] = (uint8_t)d;
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

// Number of children of every node of level l (0 for leaves) into nch[p - lb]; nl = nodes.
__global__ void k_level_nch(const int64_t* __restrict__ lvl, int l, const int32_t* __restrict__ leaf,
                            const int32_t* __restrict__ cc, int32_t* __restrict__ nch, int64_t* __restrict__ nl)
{
    const int32_t lb = (int32_t)lvl[l], le = (int32_t)lvl[l + 1];
    if (blockIdx.x == 0 && threadIdx.x == 0) *nl = le - lb;
    for (int32_t p = lb + (int32_t)(blockIdx.x * blockDim.x + threadIdx.x); p < le;
         p += (int32_t)(gridDim.x * blockDim.x)) {
        int c = 0;
        if (!leaf[p])
            for (int d = 0; d < 4; d++) c += cc[4 * p + d] > 0;
        nch[p - lb] = c;
    }
}

// Children of level l numbered in key order from le = lvl[l + 1] on (off = scan of nch).
// A child beyond the node capacity is not created: its particles stay with the parent and
// the overflow bit is set, so a captured build reports it instead of writing out of range.
__global__ void k_level_children(int64_t* __restrict__ lvl, int l, const int64_t* __restrict__ off,
                                 const int64_t* __restrict__ nl, int64_t cap, const int32_t* __restrict__ cc, int32_t* level, uint64_t* key,
                                 int32_t* parent, int32_t* first_child, int32_t* nchild, int32_t* start,
                                 int32_t* count, int32_t* leaf, double* geom, int32_t* __restrict__ child,
                                 int64_t* __restrict__ over, const double* __restrict__ mid)
{
    const int32_t lb = (int32_t)lvl[l], le = (int32_t)lvl[l + 1];
    if (blockIdx.x == 0 && threadIdx.x == 0) lvl[l + 2] = min((int64_t)le + off[*nl], cap);  // end of level l + 1
    for (int32_t p = lb + (int32_t)(blockIdx.x * blockDim.x + threadIdx.x); p < le;
         p += (int32_t)(gridDim.x * blockDim.x)) {
        if (leaf[p]) {
            first_child[p] = -1;
            nchild[p] = 0;
            child[4 * p] = child[4 * p + 1] = child[4 * p + 2] = child[4 * p + 3] = p;
            continue;
        }
        const double* g = geom + 13 * (int64_t)p;
        const g3 v1 = gld(g), v2 = gld(g + 3), v3 = gld(g + 6);
        const double* mm = mid + 9 * (int64_t)p;
        const g3 m12 = gld(mm), m23 = gld(mm + 3), m31 = gld(mm + 6);
        const g3 cv[4][3] = {{v1, m12, m31}, {m12, v2, m23}, {m31, m23, v3}, {m12, m23, m31}};
        int32_t id = le + (int32_t)off[p - lb];
        const int32_t first = id;
        int32_t st = start[p];
        const int32_t lv = level[p] + 1;
        const uint64_t kp = key[p];
        int nc = 0;
        for (int d = 0; d < 4; d++) {
            const int32_t c = cc[4 * p + d];
            if (c == 0) {
                child[4 * p + d] = -1;
                continue;
            }
            if (id >= cap) {
                child[4 * p + d] = p;
                atomicOr((unsigned long long*)over, 1ull);
                st += c;
                continue;
            }
            child[4 * p + d] = id;
            level[id] = lv;
            key[id] = kp * 4u + (uint64_t)d;
            parent[id] = p;
            first_child[id] = -1;
            nchild[id] = 0;
            start[id] = st;
            count[id] = c;
            leaf[id] = 0;
            double* gc = geom + 13 * (int64_t)id;  // vertices; centre and radius in k_level_nodes
            gst(gc, cv[d][0]);
            gst(gc + 3, cv[d][1]);
            gst(gc + 6, cv[d][2]);
            st += c;
            id++;
            nc++;
        }
        first_child[p] = nc ? first : -1;
        nchild[p] = nc;
    }
}

// After the level loop: nodes = lvl[last]; a last level that still produced children means
// the build ran out of planned levels (overflow).
__global__ void k_levels_done(const int64_t* __restrict__ lvl, int last, int64_t* __restrict__ nnodes,
                              int64_t* __restrict__ over)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    *nnodes = lvl[last];
    if (lvl[last + 1] > lvl[last]) atomicOr((unsigned long long*)over, 2ull);
}

// Level range of the roots: lvl[0] = 0, lvl[1] = number of roots.
__global__ void k_level0(int64_t* __restrict__ lvl, const int64_t* __restrict__ nroots)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        lvl[0] = 0;
        lvl[1] = *nroots;
    }
}

// ------------------------------------------------------------------------- sorting
__global__ void k_sort_keys(const int32_t* __restrict__ nodeof, int64_t n,
                            const int32_t* __restrict__ start, uint32_t* __restrict__ skey,
                            int32_t* __restrict__ perm)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    skey[i] = (uint32_t)start[nodeof[i]];
    perm[i] = (int32_t)i;
}

__global__ void k_leaf_flags(const int32_t* __restrict__ perm, const int32_t* __restrict__ nodeof,
                             const int32_t* __restrict__ start, int64_t n, int32_t* __restrict__ flags)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    flags[k] = start[nodeof[perm[k]]] == (int32_t)k ? 1 : 0;
}

__global__ void k_leaf_list(const int32_t* __restrict__ perm, const int32_t* __restrict__ nodeof,
                            const int32_t* __restrict__ flags, const int64_t* __restrict__ off,
                            int64_t n, int32_t* __restrict__ leaves, int32_t* __restrict__ slot_leaf)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t li = off[k] + flags[k] - 1;
    slot_leaf[k] = (int32_t)li;
    if (flags[k]) leaves[li] = nodeof[perm[k]];
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

__global__ void k_copy_count(const int64_t* __restrict__ src, int64_t* __restrict__ dst)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *dst = *src;
}

// FP32 copies of the node centres and radii for the pre-filtered MAC.
__global__ void k_node_f32(const int64_t* __restrict__ nnodes, const double* __restrict__ geom,
                           float4* __restrict__ c32)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= *nnodes) return;
    const double* g = geom + 13 * p;
    c32[p] = make_float4((float)g[9], (float)g[10], (float)g[11], (float)g[12]);
}

// Lanes sharing a pair of targets: the largest S <= 8 with S * pairs <= 32.
__device__ __forceinline__ int lanes_per_pair(int pairs) { return min(8, 32 / pairs); }

// Splits a leaf of nt targets into k warp tasks of nearly equal size, two targets per lane
// and S lanes per pair of targets.  k maximises the fraction of useful interactions per warp
// step, nt S / (64 k) (ties go to the smaller k).
__device__ int task_split(int nt)
{
    const int kmin = max(1, (nt + kTaskTargets - 1) / kTaskTargets);
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
                             const int32_t* __restrict__ count, unsigned long long* __restrict__ cls)
{
    const int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (L >= min(*nleaves, ldc)) return;
    const int32_t c = count[leaves[L]];
    const int k = task_split(c);
    for (int i = 0; i < k; i++) atomicAdd(cls + lanes_per_pair((c / k + (i < c % k ? 1 : 0) + 1) / 2) - 1, 1ull);
}

// Writes the warp tasks grouped by lane class, S = 1 first: a task's run time grows with the
// sources each lane visits (list length / S), so the task queue hands out the longest tasks
// first and the persistent evaluation kernel ends with short ones.  The order within a class
// is arbitrary; every task writes only its own targets, so the results do not depend on it.
__global__ void k_task_fill(const int64_t* __restrict__ nleaves, int64_t ldc, const int32_t* __restrict__ leaves,
                            const int32_t* __restrict__ start, const int32_t* __restrict__ count,
                            const int64_t* __restrict__ cls, unsigned long long* __restrict__ fill, int64_t cap,
                            Task* __restrict__ tasks, int64_t* __restrict__ over)
{
    const int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (L >= min(*nleaves, ldc)) return;
    int64_t base[8];
    base[0] = 0;
#pragma unroll
    for (int q = 1; q < 8; q++) base[q] = base[q - 1] + cls[q - 1];
    const int32_t id = leaves[L];
    const int32_t st = start[id], c = count[id];
    const int k = task_split(c);
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
// replaced by its children, which form the next frontier's pairs.  The terminals are
// appended in any order and sorted afterwards, so the lists do not depend on the schedule.
enum { kPP = 0, kPC = 1, kCP = 2, kCC = 3 };

struct DualOut {
    int32_t* t[4];
    int32_t* s[4];
    int64_t cap[4];
};

// The 20 x 20 root pairs of every instance (a target interacts with its own instance only).
__global__ void k_dual_roots(const int32_t* __restrict__ face_node, int ninst, int32_t* __restrict__ ft,
                             int32_t* __restrict__ fs, unsigned long long* __restrict__ cnt)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)ninst * 400) return;
    const int64_t b = i / 400;
    const int f1 = (int)(i % 400) / 20, f2 = (int)(i % 20);
    const int32_t t = face_node[20 * b + f1], s = face_node[20 * b + f2];
    if (t < 0 || s < 0) return;
    const unsigned long long q = atomicAdd(cnt + 4, 1ull);
    ft[q] = t;
    fs[q] = s;
}

// One level of the traversal: cnt[0..3] count the terminals per kind, cnt[4] the next
// frontier.  Writes past a capacity are dropped; the host sees the counts, grows the buffers
// and runs the level again from the same frontier.
__global__ void k_dual_step(const int32_t* __restrict__ ft, const int32_t* __restrict__ fs, int64_t nf,
                            double theta, int leaf_size, const double* __restrict__ geom,
                            const float4* __restrict__ c32, const int32_t* __restrict__ leaf,
                            const int32_t* __restrict__ first_child, const int32_t* __restrict__ nchild,
                            const int32_t* __restrict__ count, int32_t* __restrict__ gt, int32_t* __restrict__ gs,
                            int64_t gcap, DualOut out, unsigned long long* __restrict__ cnt)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    const int32_t t = ft[i], s = fs[i];
    const int32_t ct = count[t], cs = count[s];
    const bool lt = leaf[t] != 0, ls = leaf[s] != 0;
    int kind = -1;
    if (mac_filtered(c32[t], c32[s], (float)theta, geom + 13 * (int64_t)t, geom + 13 * (int64_t)s, theta)) {
        const bool tc = ct > leaf_size, sc = cs > leaf_size;
        kind = tc ? (sc ? kCC : kCP) : (sc ? kPC : kPP);
    } else if (lt && ls) {
        kind = kPP;
    }
    if (kind >= 0) {
        const unsigned long long q = atomicAdd(cnt + kind, 1ull);
        if ((int64_t)q < out.cap[kind]) {
            out.t[kind][q] = t;
            out.s[kind][q] = s;
        }
        return;
    }
    const bool split_t = !lt && (ls || ct >= cs);
    const int32_t p = split_t ? t : s;
    const int32_t fc = first_child[p], nc = nchild[p];
    const int64_t q = (int64_t)atomicAdd(cnt + 4, (unsigned long long)nc);
    if (q + nc > gcap) return;
    for (int32_t c = 0; c < nc; c++) {
        gt[q + c] = split_t ? fc + c : t;
        gs[q + c] = split_t ? s : fc + c;
    }
}

// Sorting a kind's pairs by (target key, source): key = source, then (after a stable sort)
// the target's key with the sources as values.  Target key: the depth-first leaf index for
// leaf targets (PP, PC), the cluster slot for cluster targets (CP, CC).
__global__ void k_dual_key_src(const int32_t* __restrict__ src, int64_t n, uint32_t* __restrict__ key)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) key[i] = (uint32_t)src[i];
}

__global__ void k_dual_key_tgt(uint32_t* __restrict__ key, const int32_t* __restrict__ tgt, int64_t n,
                               const int32_t* __restrict__ start, const int32_t* __restrict__ slot_leaf,
                               const int32_t* __restrict__ cluster_slot, int32_t* __restrict__ src)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    src[i] = (int32_t)key[i];
    const int32_t t = tgt[i];
    key[i] = (uint32_t)(cluster_slot ? cluster_slot[t] : slot_leaf[start[t]]);
}

__global__ void k_dual_key_back(const uint32_t* __restrict__ key, int64_t n, const int32_t* __restrict__ node_of,
                                int32_t* __restrict__ tgt)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) tgt[i] = node_of[key[i]];
}

// off[k] = first pair whose key is >= k, for k in [0, K] (binary search in the sorted keys).
__global__ void k_dual_offsets(const uint32_t* __restrict__ key, int64_t n, int64_t K, int64_t* __restrict__ off)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k > K) return;
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((int64_t)key[mid] < k)
            lo = mid + 1;
        else
            hi = mid;
    }
    off[k] = lo;
}

__global__ void k_dual_chunks(const int32_t* __restrict__ src, int64_t n, const int32_t* __restrict__ count,
                              int32_t* __restrict__ chunks)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) chunks[i] = (count[src[i]] + kStage - 1) / kStage;
}

__global__ void k_dual_coff(const int64_t* __restrict__ off, int64_t K, const int64_t* __restrict__ scan,
                            int64_t* __restrict__ coff)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k <= K) coff[k] = scan[off[k]];
}

// List entries of sorted pairs: far (a source cluster's proxy block) or near (a source leaf in
// chunks of at most kStage particles), with the FP32 centre offset c_s - c_t and, for near
// entries, the lower bound on the distance between the two triangles' points.
__global__ void k_dual_fill(bool is_far, const uint32_t* __restrict__ key, const int32_t* __restrict__ src,
                            int64_t n, const int32_t* __restrict__ node_of, const double* __restrict__ geom,
                            const int32_t* __restrict__ start, const int32_t* __restrict__ count,
                            const int32_t* __restrict__ cluster_slot, const int64_t* __restrict__ chunk_scan,
                            int32_t* __restrict__ idx, FarEntry* __restrict__ far_ent,
                            NearEntry* __restrict__ near_ent)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t t = node_of[key[i]], s = src[i];
    const double* gt = geom + 13 * (int64_t)t;
    const double* gs = geom + 13 * (int64_t)s;
    const float dx = (float)__dsub_rn(gs[9], gt[9]);
    const float dy = (float)__dsub_rn(gs[10], gt[10]);
    const float dz = (float)__dsub_rn(gs[11], gt[11]);
    if (idx) idx[i] = s;
    if (is_far) {
        FarEntry e;
        e.slot = cluster_slot[s];
        e.dx = dx;
        e.dy = dy;
        e.dz = dz;
        far_ent[i] = e;
        return;
    }
    NearEntry e;
    e.dx = dx;
    e.dy = dy;
    e.dz = dz;
    e.gap = near_gap(gt, gs);
    e.pad[0] = e.pad[1] = 0;
    const int32_t st = start[s], ct = count[s];
    int64_t q = chunk_scan[i];
    for (int32_t c0 = 0; c0 < ct; c0 += kStage) {
        e.start = st + c0;
        e.count = min(kStage, ct - c0);
        near_ent[q++] = e;
    }
}

// Evaluation tasks of the target clusters (targets: the M proxy points of cluster slot c,
// rows c M .. c M + M - 1); has[c] = the cluster is the target of a CP or CC pair.
__global__ void k_cluster_tasks(int64_t nclu, const int64_t* __restrict__ cfar_off,
                                const int64_t* __restrict__ cnear_off, int M, uint8_t* __restrict__ has,
                                Task* __restrict__ tasks, int64_t cap, unsigned long long* __restrict__ ntask,
                                int* __restrict__ status)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nclu) return;
    const bool h = cfar_off[c + 1] > cfar_off[c] || cnear_off[c + 1] > cnear_off[c];
    has[c] = h ? 1 : 0;
    if (!h) return;
    const int k = task_split(M);
    const int64_t base = (int64_t)atomicAdd(ntask, (unsigned long long)k);
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
            atomicOr(status, kStatusCapacity);
        t0 += m;
    }
}

// Interaction counts of the dual lists: st[0] PP pairs (j != i), st[1] PC target x proxy,
// st[2] CP proxy x source, st[3] CC proxy x proxy; st[4] downward particle x M over the
// clusters in has (launched over clusters with kind = 4).
__global__ void k_dual_count(int kind, const int32_t* __restrict__ tgt, const int32_t* __restrict__ src, int64_t n,
                             const int32_t* __restrict__ count, const uint8_t* __restrict__ has, int M,
                             unsigned long long* __restrict__ st)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long v = 0;
    if (i < n) {
        const unsigned long long mm = (unsigned long long)M;
        if (kind == 4) {
            v = has[i] ? (unsigned long long)count[tgt[i]] * mm : 0ull;  // tgt: cluster nodes
        } else {
            const int32_t t = tgt[i], s = src[i];
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
    STS_CUDA(c->nd_cc.grow(4 * need, 4 * keep, s));
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
    STS_CUDA(cudaMemcpyAsync(c->pos.p, pos, 3 * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    STS_CUDA(c->nodeof.reserve(n));
    STS_CUDA(c->digit.reserve(n));
    STS_CUDA(c->perm.reserve(n));
    STS_CUDA(c->perm_tmp.reserve(n));
    STS_CUDA(c->skey.reserve(n));
    STS_CUDA(c->skey_tmp.reserve(n));
    STS_CUDA(c->flags.reserve(n + 1));
    STS_CUDA(c->offs.reserve(n + 1));
    STS_CUDA(c->slot_leaf.reserve(n));
    const int64_t hs = radix_hist_size(n);
    STS_CUDA(c->hist.reserve(hs));
    STS_CUDA(c->scan_tmp.reserve(hs + 1 + scan_scratch(hs) + scan_scratch(n + 1)));
    STS_CUDA(c->counters.reserve(64));
    STS_CUDA(c->small.reserve(16));
    const int32_t nkeys = 20 * ninst;
    if (grow_nodes(c, nkeys + 80, 0, s)) return STS_ERR_CUDA;
    STS_CUDA(c->root_cnt.reserve(nkeys + 1));
    STS_CUDA(c->root_flag.reserve(nkeys + 1));
    STS_CUDA(c->face_node.reserve(nkeys + 1));
    STS_CUDA(c->root_id.reserve(nkeys + 1));
    STS_CUDA(c->root_start.reserve(nkeys + 1));
    STS_CUDA(c->scan_tmp.reserve(hs + 1 + scan_scratch(hs) + scan_scratch(n + 1) + scan_scratch(nkeys + 1)));
    c->ninst = ninst;

    const int T = 256;
    int32_t* face_count = c->root_cnt.p;  // [20 * instances]
    STS_CUDA(cudaMemsetAsync(face_count, 0, nkeys * sizeof(int32_t), s));
    (k_faces<<<blocks(n, T), T, 0, s>>>(c->pos.p, n, inst_off, ninst, c->nodeof.p, face_count, c->d_status),
     note_launch());
    (k_root_flags<<<blocks(nkeys, T), T, 0, s>>>(nkeys, face_count, c->root_flag.p), note_launch());
    exclusive_scan_i32(c->root_flag.p, c->root_id.p, nkeys, c->scan_tmp.p, s);
    exclusive_scan_i32(face_count, c->root_start.p, nkeys, c->scan_tmp.p, s);
    (k_roots<<<blocks(nkeys, T), T, 0, s>>>(nkeys, face_count, c->root_id.p, c->root_start.p, c->face_node.p,
                                            c->nd_level.p, c->nd_key.p, c->nd_parent.p, c->nd_first_child.p,
                                            c->nd_nchild.p, c->nd_start.p, c->nd_count.p, c->nd_leaf.p,
                                            c->nd_geom.p), note_launch());
    STS_LAUNCH_CHECK();
    (k_assign_roots<<<blocks(n, T), T, 0, s>>>(n, c->face_node.p, c->nodeof.p), note_launch());
    int64_t* dc = c->dc.p;
    int64_t* lvl = dc + kDcLevel;
    const bool cap = c->capturing;  // recording a graph: no host reads, planned capacities
    if (!cap) STS_CUDA(cudaMemsetAsync(dc + kDcOver, 0, sizeof(int64_t), s));
    (k_level0<<<1, 32, 0, s>>>(lvl, c->root_id.p + nkeys), note_launch());
    int64_t lb = 0, le = 0;
    if (!cap) {
        (k_gather<<<1, 32, 0, s>>>(c->root_id.p + nkeys, nullptr, nullptr, nullptr, c->d_status, c->small.p),
         note_launch());
        STS_CUDA(cudaMemcpyAsync(c->h_pinned, c->small.p, 5 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        STS_CUDA(cudaStreamSynchronize(s));
        le = c->h_pinned[0];
        if (c->h_pinned[4] & kStatusNonfinite) {
            STS_CUDA(cudaMemsetAsync(c->d_status, 0, sizeof(int), s));
            set_error("sts_tree_build: non-finite position");
            return STS_ERR_NONFINITE;
        }
    }
    // levels: eagerly until a level adds no node (one host read per level), or, while
    // recording, the planned number of levels plus one that must come out empty
    const int nlev = cap ? std::min(c->plan.depth + 2, max_level + 1) : max_level + 1;
    const int64_t node_cap = cap ? (int64_t)c->nd_level.cap : 0;
    const unsigned gnode = cap ? (unsigned)std::min<int64_t>(4096, (node_cap + T - 1) / T) : 0;
    int level = 0, last = 0;
    c->level_begin.assign(1, 0);
    // particle passes: a few resident blocks per SM, each striding over many particles
    const unsigned gpart = (unsigned)std::min<int64_t>(blocks(n, 4 * T), 4 * (int64_t)c->num_sms);
    for (level = 0; level < nlev; level++) {
        int64_t capn;
        unsigned g;
        if (!cap) {
            c->level_begin.push_back(le);
            const int64_t nl = le - lb;
            if (grow_nodes(c, le + 4 * nl, le, s)) return STS_ERR_CUDA;
            capn = (int64_t)c->nd_level.cap;
            g = blocks(std::max<int64_t>(nl, 1), T);
        } else {
            capn = node_cap;
            g = gnode;
        }
        (k_level_nodes<<<cap ? gnode : blocks(4 * std::max<int64_t>(le - lb, 1), T), T, 0, s>>>(
             lvl, level, leaf_size, max_level, c->nd_level.p, c->nd_count.p, c->nd_geom.p, c->nd_leaf.p,
             c->nd_norm.p, c->nd_norm32.p, c->nd_cc.p, c->nd_mid.p), note_launch());
        (k_level_particles<<<gpart, T, 0, s>>>(lvl, level, c->pos.p, n, c->nodeof.p, c->nd_norm.p,
                                                      c->nd_norm32.p, c->nd_child.p, c->digit.p, c->nd_cc.p),
         note_launch());
        (k_level_nch<<<g, T, 0, s>>>(lvl, level, c->nd_leaf.p, c->nd_cc.p, c->flags.p, dc + kDcTmp),
         note_launch());
        exclusive_scan_i32(c->flags.p, c->offs.p, cap ? std::min<int64_t>(capn, n) : le - lb, c->scan_tmp.p, s,
                           dc + kDcTmp);
        (k_level_children<<<g, T, 0, s>>>(lvl, level, c->offs.p, dc + kDcTmp, capn, c->nd_cc.p, c->nd_level.p,
                                          c->nd_key.p, c->nd_parent.p, c->nd_first_child.p, c->nd_nchild.p,
                                          c->nd_start.p, c->nd_count.p, c->nd_leaf.p, c->nd_geom.p, c->nd_child.p,
                                          dc + kDcOver, c->nd_mid.p), note_launch());
        STS_LAUNCH_CHECK();
        if (!cap) {
            int64_t next = 0;
            if (read_i64(c, lvl + level + 2, &next, s)) return STS_ERR_CUDA;
            if (next == le) break;
            lb = le;
            le = next;
        }
    }
    last = cap ? nlev : level + 1;
    (k_levels_done<<<1, 32, 0, s>>>(lvl, last, dc + kDcNodes, dc + kDcOver), note_launch());
    if (!cap) {
        c->nnodes = le;
        c->deepest = level;
        c->plan.nodes = std::max(c->plan.nodes, le);
        c->plan.depth = std::max(c->plan.depth, level);
    } else {
        c->nnodes = -1;  // known after the graph runs
        c->deepest = -1;
    }
    const int64_t nodes_grid = cap ? node_cap : c->nnodes;
    (k_node_f32<<<blocks(std::max<int64_t>(nodes_grid, 1), T), T, 0, s>>>(dc + kDcNodes, c->nd_geom.p, c->nd_c32.p),
     note_launch());

    phase_begin(c, kPhSort, s);
    (k_sort_keys<<<blocks(n, T), T, 0, s>>>(c->nodeof.p, n, c->nd_start.p, c->skey.p, c->perm.p), note_launch());
    int bits = 0;
    while (bits < 32 && ((int64_t)1 << bits) < n) bits++;
    int64_t* scan_out = c->scan_tmp.p;
    int64_t* scan_scr = c->scan_tmp.p + hs + 1;
    radix_sort_pairs(c->skey.p, c->perm.p, c->skey_tmp.p, c->perm_tmp.p, n, bits, c->hist.p,
                     scan_out, scan_scr, s);
    (k_leaf_flags<<<blocks(n, T), T, 0, s>>>(c->perm.p, c->nodeof.p, c->nd_start.p, n, c->flags.p), note_launch());
    exclusive_scan_i32(c->flags.p, c->offs.p, n, c->scan_tmp.p, s);
    (k_copy_count<<<1, 32, 0, s>>>(c->offs.p + n, c->dc.p + kDcLeaves), note_launch());
    STS_CUDA(c->leaves.reserve(n + 1));
    (k_leaf_list<<<blocks(n, T), T, 0, s>>>(c->perm.p, c->nodeof.p, c->flags.p, c->offs.p, n,
                                           c->leaves.p, c->slot_leaf.p), note_launch());
    STS_LAUNCH_CHECK();
    phase_end(c, kPhSort, s);
    c->nleaves = -1;  // set by build_clusters
    c->have_tree = true;
    return STS_OK;
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
    exclusive_scan_i32(c->list_cnt.p, far_po, L, c->scan_tmp.p, s, dc + kDcLeaves);
    exclusive_scan_i32(c->list_cnt.p + L, near_po, L, c->scan_tmp.p, s, dc + kDcLeaves);
    exclusive_scan_i32(c->list_cnt.p + 2 * L, chunk_po, L, c->scan_tmp.p, s, dc + kDcLeaves);
    // evaluation tasks: each leaf's targets split into warp tasks
    STS_CUDA(cudaMemsetAsync(dc + kDcClass, 0, 16 * sizeof(int64_t), s));
    (k_task_count<<<g, T, 0, s>>>(dc + kDcLeaves, L, c->leaves.p, c->nd_count.p,
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
    (k_task_fill<<<g, T, 0, s>>>(dc + kDcLeaves, L, c->leaves.p, c->nd_start.p, c->nd_count.p, dc + kDcClass,
                                 (unsigned long long*)(dc + kDcClassFill), (int64_t)c->tasks.cap, c->tasks.p,
                                 dc + kDcOver), note_launch());
    STS_LAUNCH_CHECK();
    c->list_theta = theta;
    c->have_lists = true;
    return STS_OK;
}

// Sorts the pairs of one kind by (target key, source); afterwards c->dual_key holds the sorted
// target keys and dual_t / dual_s the pairs.  leaf_targets: key = depth-first leaf index,
// else the cluster slot.
static int sort_dual_kind(sts_ctx* c, int kind, bool leaf_targets, cudaStream_t s)
{
    const int64_t P = c->dual_n[kind];
    if (P == 0) return STS_OK;
    const int T = 256;
    const int64_t hs = radix_hist_size(P);
    int64_t* scan_out = c->scan_tmp.p;
    int64_t* scan_scr = c->scan_tmp.p + hs + 1;
    int bits_node = 0, bits_key = 0;
    while (bits_node < 32 && ((int64_t)1 << bits_node) < c->nnodes) bits_node++;
    const int64_t K = leaf_targets ? c->nleaves : c->nclusters;
    while (bits_key < 32 && ((int64_t)1 << bits_key) < K) bits_key++;
    (k_dual_key_src<<<blocks(P, T), T, 0, s>>>(c->dual_s[kind].p, P, c->dual_key.p), note_launch());
    radix_sort_pairs(c->dual_key.p, c->dual_t[kind].p, c->dual_ktmp.p, c->dual_vtmp.p, P, bits_node, c->hist.p,
                     scan_out, scan_scr, s);
    (k_dual_key_tgt<<<blocks(P, T), T, 0, s>>>(c->dual_key.p, c->dual_t[kind].p, P, c->nd_start.p, c->slot_leaf.p,
                                               leaf_targets ? nullptr : c->cluster_slot.p, c->dual_s[kind].p),
     note_launch());
    radix_sort_pairs(c->dual_key.p, c->dual_s[kind].p, c->dual_ktmp.p, c->dual_vtmp.p, P, bits_key, c->hist.p,
                     scan_out, scan_scr, s);
    (k_dual_key_back<<<blocks(P, T), T, 0, s>>>(c->dual_key.p, P,
                                                leaf_targets ? c->leaves.p : c->cluster_node.p, c->dual_t[kind].p),
     note_launch());
    STS_LAUNCH_CHECK();
    return STS_OK;
}

// CSR of one sorted kind over K target keys: off[K + 1] (pairs); for near kinds also the chunk
// offsets coff[K + 1] and the chunked entries.  Reads the chunk total back (synchronises s).
static int fill_dual_kind(sts_ctx* c, int kind, int64_t K, bool is_far, int64_t* off, int64_t* coff,
                          int32_t* idx, DevBuf<FarEntry>* far_ent, DevBuf<NearEntry>* near_ent, int64_t* chunks,
                          cudaStream_t s)
{
    const int64_t P = c->dual_n[kind];
    const int T = 256;
    const int32_t* node_of = (kind == kPP || kind == kPC) ? c->leaves.p : c->cluster_node.p;
    (k_dual_offsets<<<blocks(K + 1, T), T, 0, s>>>(c->dual_key.p, P, K, off), note_launch());
    if (is_far) {
        STS_CUDA(far_ent->reserve(P + 1));
        if (P > 0)
            (k_dual_fill<<<blocks(P, T), T, 0, s>>>(true, c->dual_key.p, c->dual_s[kind].p, P, node_of, c->nd_geom.p,
                                                    c->nd_start.p, c->nd_count.p, c->cluster_slot.p, nullptr, idx,
                                                    far_ent->p, nullptr),
             note_launch());
        STS_LAUNCH_CHECK();
        return STS_OK;
    }
    // chunk counts per pair (in the radix scratch, free after the sort), their scan, and the
    // chunk offset of every key
    if (P > 0)
        (k_dual_chunks<<<blocks(P, T), T, 0, s>>>(c->dual_s[kind].p, P, c->nd_count.p, c->dual_vtmp.p),
         note_launch());
    exclusive_scan_i32(c->dual_vtmp.p, c->dual_scan.p, P, c->scan_tmp.p, s);
    (k_dual_coff<<<blocks(K + 1, T), T, 0, s>>>(off, K, c->dual_scan.p, coff), note_launch());
    STS_LAUNCH_CHECK();
    STS_CUDA(cudaMemcpyAsync(c->h_pinned, c->dual_scan.p + P, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    STS_CUDA(cudaStreamSynchronize(s));
    *chunks = c->h_pinned[0];
    STS_CUDA(near_ent->reserve(*chunks + 1));
    if (P > 0)
        (k_dual_fill<<<blocks(P, T), T, 0, s>>>(false, c->dual_key.p, c->dual_s[kind].p, P, node_of, c->nd_geom.p,
                                                c->nd_start.p, c->nd_count.p, c->cluster_slot.p, c->dual_scan.p, idx,
                                                nullptr, near_ent->p),
         note_launch());
    STS_LAUNCH_CHECK();
    return STS_OK;
}

int build_dual(sts_ctx* c, double theta, cudaStream_t s)
{
    c->have_dual = false;
    c->have_lists = false;  // the leaf lists are replaced by the PP / PC pairs
    if (c->capturing) {
        set_error("dual traversal: not available while recording a graph");
        return STS_ERR_STATE;
    }
    const int T = 256;
    const int64_t nn = c->nnodes, L = c->nleaves, C = c->nclusters;
    STS_CUDA(c->dual_cnt.reserve(8));
    unsigned long long* cnt = (unsigned long long*)c->dual_cnt.p;
    int64_t fcap = std::max<int64_t>(400 * (int64_t)c->ninst, 8 * nn + 64);
    STS_CUDA(c->dual_ft.reserve(fcap));
    STS_CUDA(c->dual_fs.reserve(fcap));
    STS_CUDA(c->dual_gt.reserve(fcap));
    STS_CUDA(c->dual_gs.reserve(fcap));
    const int64_t init_cap[4] = {48 * L + 64, 48 * L + 64, 16 * C + 64, 16 * C + 64};
    for (int k = 0; k < 4; k++) {
        STS_CUDA(c->dual_t[k].reserve(init_cap[k]));
        STS_CUDA(c->dual_s[k].reserve(init_cap[k]));
    }
    STS_CUDA(cudaMemsetAsync(c->dual_cnt.p, 0, 8 * sizeof(int64_t), s));
    (k_dual_roots<<<blocks(400 * (int64_t)c->ninst, T), T, 0, s>>>(c->face_node.p, c->ninst, c->dual_ft.p,
                                                                  c->dual_fs.p, cnt), note_launch());
    STS_LAUNCH_CHECK();
    STS_CUDA(cudaMemcpyAsync(c->h_pinned, c->dual_cnt.p, 8 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    STS_CUDA(cudaStreamSynchronize(s));
    int64_t nf = c->h_pinned[4];
    int64_t done[4] = {0, 0, 0, 0};
    // each level refines one side of a pair, so the traversal ends within 2 (depth + 1) levels;
    // every retry grows a buffer
    for (int it = 0; nf > 0; it++) {
        if (it > 4 * (kMaxLevel + 2) + 64) {
            set_error("dual traversal: no progress");
            return STS_ERR_CAPACITY;
        }
        for (int k = 0; k < 4; k++) c->h_pinned[k] = done[k];
        c->h_pinned[4] = 0;
        STS_CUDA(cudaMemcpyAsync(c->dual_cnt.p, c->h_pinned, 5 * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        DualOut out;
        for (int k = 0; k < 4; k++) {
            out.t[k] = c->dual_t[k].p;
            out.s[k] = c->dual_s[k].p;
            out.cap[k] = (int64_t)std::min(c->dual_t[k].cap, c->dual_s[k].cap);
        }
        const int64_t gcap = (int64_t)std::min(c->dual_gt.cap, c->dual_gs.cap);
        (k_dual_step<<<blocks(nf, T), T, 0, s>>>(c->dual_ft.p, c->dual_fs.p, nf, theta, c->leaf_size, c->nd_geom.p,
                                                 c->nd_c32.p, c->nd_leaf.p, c->nd_first_child.p, c->nd_nchild.p,
                                                 c->nd_count.p, c->dual_gt.p, c->dual_gs.p, gcap, out, cnt),
         note_launch());
        STS_LAUNCH_CHECK();
        STS_CUDA(cudaMemcpyAsync(c->h_pinned, c->dual_cnt.p, 5 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        STS_CUDA(cudaStreamSynchronize(s));
        bool redo = false;
        for (int k = 0; k < 4; k++)
            if (c->h_pinned[k] > out.cap[k]) {
                const int64_t need = c->h_pinned[k];
                STS_CUDA(c->dual_t[k].grow(need, done[k], s));
                STS_CUDA(c->dual_s[k].grow(need, done[k], s));
                redo = true;
            }
        const int64_t ng = c->h_pinned[4];
        if (ng > gcap) {
            STS_CUDA(c->dual_gt.reserve(ng));
            STS_CUDA(c->dual_gs.reserve(ng));
            redo = true;
        }
        if (redo) continue;  // the same frontier again, with room for every write
        for (int k = 0; k < 4; k++) done[k] = c->h_pinned[k];
        nf = ng;
        std::swap(c->dual_ft, c->dual_gt);
        std::swap(c->dual_fs, c->dual_gs);
    }
    int64_t pmax = 1;
    for (int k = 0; k < 4; k++) {
        c->dual_n[k] = done[k];
        pmax = std::max(pmax, done[k]);
    }
    // sort every kind by (target, source)
    const int64_t hs = radix_hist_size(pmax);
    STS_CUDA(c->dual_key.reserve(pmax + 1));
    STS_CUDA(c->dual_ktmp.reserve(pmax + 1));
    STS_CUDA(c->dual_vtmp.reserve(pmax + 1));
    STS_CUDA(c->dual_scan.reserve(pmax + 1));
    STS_CUDA(c->hist.reserve(hs));
    STS_CUDA(c->scan_tmp.reserve(hs + 1 + scan_scratch(hs) + scan_scratch(pmax + 1) + scan_scratch(nn + 1) + 64));
    // leaf lists: PC far, PP near (per depth-first leaf); cluster lists: CC far, CP near
    STS_CUDA(c->far_off.reserve(L + 1));
    STS_CUDA(c->near_off.reserve(L + 1));
    STS_CUDA(c->near_coff.reserve(L + 1));
    STS_CUDA(c->far_idx.reserve(c->dual_n[kPC] + 1));
    STS_CUDA(c->near_idx.reserve(c->dual_n[kPP] + 1));
    STS_CUDA(c->cfar_off.reserve(C + 1));
    STS_CUDA(c->cnear_off.reserve(C + 1));
    STS_CUDA(c->cnear_coff.reserve(C + 1));
    int rc;
    int64_t chunks = 0, cchunks = 0;
    if ((rc = sort_dual_kind(c, kPC, true, s))) return rc;
    if ((rc = fill_dual_kind(c, kPC, L, true, c->far_off.p, nullptr, c->far_idx.p, &c->far_ent, nullptr, nullptr, s)))
        return rc;
    if ((rc = sort_dual_kind(c, kPP, true, s))) return rc;
    if ((rc = fill_dual_kind(c, kPP, L, false, c->near_off.p, c->near_coff.p, c->near_idx.p, nullptr, &c->near_ent,
                             &chunks, s)))
        return rc;
    if ((rc = sort_dual_kind(c, kCC, false, s))) return rc;
    if ((rc = fill_dual_kind(c, kCC, C, true, c->cfar_off.p, nullptr, nullptr, &c->cfar_ent, nullptr, nullptr, s)))
        return rc;
    if ((rc = sort_dual_kind(c, kCP, false, s))) return rc;
    if ((rc = fill_dual_kind(c, kCP, C, false, c->cnear_off.p, c->cnear_coff.p, nullptr, nullptr, &c->cnear_ent,
                             &cchunks, s)))
        return rc;
    // the sorted target keys are no longer needed; the pairs stay for export (targets: node ids)
    int64_t* dc = c->dc.p;
    const unsigned g = blocks(std::max<int64_t>(L, 1), 128);
    STS_CUDA(cudaMemsetAsync(dc + kDcClass, 0, 16 * sizeof(int64_t), s));
    (k_task_count<<<g, 128, 0, s>>>(dc + kDcLeaves, L, c->leaves.p, c->nd_count.p,
                                    (unsigned long long*)(dc + kDcClass)), note_launch());
    (k_list_totals<<<1, 32, 0, s>>>(dc, c->far_off.p, c->near_off.p, c->near_coff.p, L), note_launch());
    STS_LAUNCH_CHECK();
    STS_CUDA(cudaMemcpyAsync(c->h_pinned, dc, 16 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    STS_CUDA(cudaStreamSynchronize(s));
    c->nfar = c->h_pinned[kDcFar];
    c->nnear = c->h_pinned[kDcNear];
    c->nnear_chunks = c->h_pinned[kDcChunks];
    c->ntasks = c->h_pinned[kDcTasks];
    c->ncnear_chunks = cchunks;
    STS_CUDA(c->tasks.reserve(c->ntasks + 1));
    (k_task_fill<<<g, 128, 0, s>>>(dc + kDcLeaves, L, c->leaves.p, c->nd_start.p, c->nd_count.p, dc + kDcClass,
                                   (unsigned long long*)(dc + kDcClassFill), (int64_t)c->tasks.cap, c->tasks.p,
                                   dc + kDcOver), note_launch());
    STS_LAUNCH_CHECK();
    c->dual_theta = theta;
    c->have_dual = true;
    return STS_OK;
}

int cluster_tasks(sts_ctx* c, int M, cudaStream_t s)
{
    const int64_t C = c->nclusters;
    c->nctasks = 0;
    STS_CUDA(c->chas.reserve(C + 1));
    if (C == 0) return STS_OK;
    const int64_t cap = C * ((M + kTaskTargets - 1) / kTaskTargets + 3);
    STS_CUDA(c->ctasks.reserve(cap + 1));
    STS_CUDA(cudaMemsetAsync(c->dual_cnt.p + 5, 0, sizeof(int64_t), s));
    (k_cluster_tasks<<<blocks(C, 128), 128, 0, s>>>(C, c->cfar_off.p, c->cnear_off.p, M, c->chas.p, c->ctasks.p, cap,
                                                    (unsigned long long*)(c->dual_cnt.p + 5), c->d_status),
     note_launch());
    STS_LAUNCH_CHECK();
    c->nctasks = cap;  // a bound: the kernels read the count from dual_cnt[5]
    return STS_OK;
}

int dual_stats(sts_ctx* c, int degree, int64_t* stats, cudaStream_t s)
{
    for (int k = 0; k < 5; k++) stats[k] = 0;
    if (!c->have_dual) return STS_OK;
    const int M = (degree + 1) * (degree + 2) / 2;
    STS_CUDA(c->d_stats.reserve(8));
    STS_CUDA(cudaMemsetAsync(c->d_stats.p, 0, 8 * sizeof(unsigned long long), s));
    const int T = 256;
    for (int k = 0; k < 4; k++)
        if (c->dual_n[k] > 0)
            (k_dual_count<<<blocks(c->dual_n[k], T), T, 0, s>>>(k, c->dual_t[k].p, c->dual_s[k].p, c->dual_n[k],
                                                                c->nd_count.p, nullptr, M, c->d_stats.p),
             note_launch());
    if (c->nclusters > 0) {
        // the clusters that are targets of CP or CC pairs (as the dual evaluation marks them)
        int rc = cluster_tasks(c, M, s);
        if (rc) return rc;
        (k_dual_count<<<blocks(c->nclusters, T), T, 0, s>>>(4, c->cluster_node.p, nullptr, c->nclusters,
                                                            c->nd_count.p, c->chas.p, M, c->d_stats.p),
         note_launch());
    }
    STS_LAUNCH_CHECK();
    STS_CUDA(cudaMemcpyAsync(c->h_pinned, c->d_stats.p, 5 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    STS_CUDA(cudaStreamSynchronize(s));
    for (int k = 0; k < 5; k++) stats[k] = c->h_pinned[k];
    return STS_OK;
}

}  // namespace sts
