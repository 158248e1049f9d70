// The dual traversal's CP and CC interactions and the downward pass (Sec. 3.3, 3.4): the
// evaluation kernel run over the cluster lists (targets: the proxy points of the target
// clusters), the interpolating polynomial of every target cluster formed from those values,
// and the polynomials evaluated at the particles below the clusters.  The PP and PC pairs of
// the dual traversal sit in the leaf lists and go through the evaluation of sts_eval.cu.
#include <algorithm>

#include "sts_internal.cuh"

namespace sts {
namespace {

inline unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// The interpolating polynomial of a cluster (degree D, M = (D+1)(D+2)/2 coefficients
// cf[M][3]) at a point with spherical barycentric coordinates b in the cluster's triangle
// (Sec. 3.2, x = b1 v1 + b2 v2 + b3 v3): sum_k B_k(b) c_k with B_k(b) = b1^a b2^b b3^c in the
// order a = D..0, b = D - a..0, summed per a and then over a.  D is a template parameter so
// that the powers stay in registers.  FP64 (the FP64 path).
template <int D>
__device__ __forceinline__ void eval_poly(double b1, double b2, double b3, const double* __restrict__ cf, double& ax,
                                          double& ay, double& az)
{
    double p1[D + 1], p2[D + 1], p3[D + 1];
    p1[0] = p2[0] = p3[0] = 1.0;
#pragma unroll
    for (int e = 1; e <= D; e++) {
        p1[e] = p1[e - 1] * b1;
        p2[e] = p2[e - 1] * b2;
        p3[e] = p3[e - 1] * b3;
    }
    int k = 0;
#pragma unroll
    for (int ea = D; ea >= 0; ea--) {
        double sx = 0.0, sy = 0.0, sz = 0.0;
#pragma unroll
        for (int eb = D - ea; eb >= 0; eb--, k++) {
            const double B = p2[eb] * p3[D - ea - eb];
            sx += B * cf[3 * k];
            sy += B * cf[3 * k + 1];
            sz += B * cf[3 * k + 2];
        }
        ax += p1[ea] * sx;
        ay += p1[ea] * sy;
        az += p1[ea] * sz;
    }
}

// The same sum in FP32 for the particles of the mixed path, each basis function's three
// coefficients in one float4 (x, y, z, unused): one 16-byte load per coefficient instead of
// three 4-byte ones.  The coefficients come from the FP64 contraction and describe a smooth
// interpolant, so the evaluation carries none of the contraction's cancellation (its error is
// eps32 times the Bernstein coefficients, which track the interpolated values).
template <int D>
__device__ __forceinline__ void eval_poly4(float b1, float b2, float b3, const float4* __restrict__ cf, float& ax,
                                           float& ay, float& az)
{
    float p1[D + 1], p2[D + 1], p3[D + 1];
    p1[0] = p2[0] = p3[0] = 1.f;
#pragma unroll
    for (int e = 1; e <= D; e++) {
        p1[e] = p1[e - 1] * b1;
        p2[e] = p2[e - 1] * b2;
        p3[e] = p3[e - 1] * b3;
    }
    int k = 0;
#pragma unroll
    for (int ea = D; ea >= 0; ea--) {
        float sx = 0.f, sy = 0.f, sz = 0.f;
#pragma unroll
        for (int eb = D - ea; eb >= 0; eb--, k++) {
            const float B = p2[eb] * p3[D - ea - eb];
            const float4 q = cf[k];
            sx += B * q.x;
            sy += B * q.y;
            sz += B * q.z;
        }
        ax += p1[ea] * sx;
        ay += p1[ea] * sy;
        az += p1[ea] * sz;
    }
}

// Barycentric coordinates from the FP64 frame (rows n_i / D of Cramer's rule: n1 = v2 x v3,
// n2 = v3 x v1, n3 = v1 x v2, D = v1 . n1) ...
__device__ __forceinline__ void bary64(const double* __restrict__ f, double x, double y, double z, double& b1,
                                       double& b2, double& b3)
{
    b1 = f[0] * x + f[1] * y + f[2] * z;
    b2 = f[3] * x + f[4] * y + f[5] * z;
    b3 = f[6] * x + f[7] * y + f[8] * z;
}

// ... and from the FP32 frame about the centre: b = b(c) + (n_i / D) . (x - c), with x - c
// already formed accurately (hi/lo pairs or an FP64 difference).
__device__ __forceinline__ void bary32(const float* __restrict__ h, float dx, float dy, float dz, float& b1,
                                       float& b2, float& b3)
{
    b1 = h[9] + (h[0] * dx + h[1] * dy + h[2] * dz);
    b2 = h[10] + (h[3] * dx + h[4] * dy + h[5] * dz);
    b3 = h[11] + (h[6] * dx + h[7] * dy + h[8] * dz);
}

// FP64 precision: interpolants of the clusters of level l (Sec. 3.3, CP and CC: the kernel sum
// -(1/4 pi) S at the target cluster's proxy points, interpolated over the cluster; the velocity
// at a particle x is then x x the interpolant, tangent to the sphere), passed down the tree.
// U_T = the sum of T's own CP and CC pairs at its proxy points (cvel; zero without such pairs)
// plus the interpolant of its parent, which already holds every ancestor's, evaluated there.  A
// degree-d polynomial in one triangle's barycentric coordinates is one in any other's (both are
// the homogeneous degree-d polynomials in x), so interpolating the parent's at T's M proxy
// points reproduces it exactly: a particle then evaluates its lowest cluster's interpolant only,
// which equals the sum of all its ancestors' interpolants.  Coefficients: with proxy points
// x~_m = s_m / rho_m, s_m = sum_i beta_mi v_i, rho_m = |s_m|, the barycentric coordinates of
// x~_m are beta_m / rho_m, so V_T = diag(rho^-d) V_ref and c = V_ref^-1 diag(rho^d) U.
// acc[c]: cluster c holds an interpolant.  One CTA per cluster of the level.
template <int D>
__global__ void k_down_level(const int64_t* __restrict__ lvl, int l, const int32_t* __restrict__ parent,
                             const int32_t* __restrict__ cluster_slot, const uint8_t* __restrict__ has,
                             uint8_t* __restrict__ acc, const double* __restrict__ geom,
                             const double* __restrict__ frame, const double4* __restrict__ prx64,
                             const double* __restrict__ beta, const double* __restrict__ vinvT,
                             const double* __restrict__ cvel, double* __restrict__ coef)
{
    constexpr int d = D, M = (D + 1) * (D + 2) / 2;
    __shared__ double u[3 * kMaxM];
    const int64_t lb = lvl[l], le = lvl[l + 1];
    for (int64_t p = lb + blockIdx.x; p < le; p += gridDim.x) {
        const int32_t cs = cluster_slot[p];
        if (cs < 0) continue;
        const int32_t par = parent[p];
        const int32_t ps = par >= 0 ? cluster_slot[par] : -1;
        const bool from_parent = ps >= 0 && acc[ps];
        const bool own = has[cs] != 0;
        if (threadIdx.x == 0) acc[cs] = (own || from_parent) ? 1 : 0;
        if (!own && !from_parent) continue;
        const double* g = geom + 13 * p;
        __syncthreads();  // u of the previous cluster is no longer read
        for (int m = threadIdx.x; m < M; m += blockDim.x) {
            double vx = 0.0, vy = 0.0, vz = 0.0;
            if (own) {
                const double* v = cvel + 3 * ((int64_t)cs * M + m);
                vx = v[0];
                vy = v[1];
                vz = v[2];
            }
            if (from_parent) {
                const double4 x = prx64[(int64_t)cs * M + m];
                double b1, b2, b3;
                bary64(frame + 12 * (int64_t)ps, x.x, x.y, x.z, b1, b2, b3);
                eval_poly<D>(b1, b2, b3, coef + 3 * (int64_t)ps * M, vx, vy, vz);
            }
            const double b1 = beta[3 * m], b2 = beta[3 * m + 1], b3 = beta[3 * m + 2];
            const double sx = (b1 * g[0] + b2 * g[3]) + b3 * g[6];
            const double sy = (b1 * g[1] + b2 * g[4]) + b3 * g[7];
            const double sz = (b1 * g[2] + b2 * g[5]) + b3 * g[8];
            const double rho = sqrt((sx * sx + sy * sy) + sz * sz);
            double rd = 1.0;
            for (int e = 0; e < d; e++) rd *= rho;
            u[3 * m] = rd * vx;
            u[3 * m + 1] = rd * vy;
            u[3 * m + 2] = rd * vz;
        }
        __syncthreads();
        for (int k = threadIdx.x; k < M; k += blockDim.x) {
            double ax = 0.0, ay = 0.0, az = 0.0;
            for (int m = 0; m < M; m++) {
                const double w = vinvT[m * M + k];
                ax += w * u[3 * m];
                ay += w * u[3 * m + 1];
                az += w * u[3 * m + 2];
            }
            double* o = coef + 3 * ((int64_t)cs * M + k);
            o[0] = ax;
            o[1] = ay;
            o[2] = az;
        }
    }
}

// FP64 precision: adds to every particle x (sorted slot) x crossed with the interpolant of its
// lowest cluster: its leaf when that is a cluster (at the depth limit), else the leaf's parent.
template <int D>
__global__ void k_downward(int64_t n, const int32_t* __restrict__ slot_leaf, const int32_t* __restrict__ leaves,
                           const int32_t* __restrict__ parent, const int32_t* __restrict__ cluster_slot,
                           const uint8_t* __restrict__ acc, const double* __restrict__ frame,
                           const double4* __restrict__ src64, const int32_t* __restrict__ perm,
                           const double* __restrict__ coef, double* __restrict__ vel)
{
    constexpr int M = (D + 1) * (D + 2) / 2;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int32_t a = leaves[slot_leaf[j]];
    if (cluster_slot[a] < 0) a = parent[a];
    if (a < 0) return;  // a root leaf: no cluster above it
    const int32_t cs = cluster_slot[a];
    if (cs < 0 || !acc[cs]) return;
    const double4 x = src64[j];
    double ax = 0.0, ay = 0.0, az = 0.0;  // the interpolated -(1/4 pi) S
    double b1, b2, b3;
    bary64(frame + 12 * (int64_t)cs, x.x, x.y, x.z, b1, b2, b3);
    eval_poly<D>(b1, b2, b3, coef + 3 * (int64_t)cs * M, ax, ay, az);
    const int64_t i = perm[j];
    vel[3 * i] += x.y * az - x.z * ay;
    vel[3 * i + 1] += x.z * ax - x.x * az;
    vel[3 * i + 2] += x.x * ay - x.y * ax;
}

// Mixed precision: the interpolant of every cluster with CP or CC pairs (Sec. 3.3), each from
// its own U_T only: c = V_ref^-1 diag(rho^d) U_T in FP64 (V_ref^-1 carries cond(V_ref), so
// FP32 would lose the coefficients), rounded to FP32 once for the particles.  The clusters are
// independent (no parent's interpolant is carried down), so one launch takes all of them: a
// fixed grid strides over the clusters, whose count is on the device.  A CTA of 3M threads
// (rounded up to whole warps) takes one cluster, a thread one (coefficient, component): the
// FP64 pipe is the bound, so the lanes are kept busy rather than the loads shared.
template <int D>
constexpr int coef_threads()
{
    return (3 * ((D + 1) * (D + 2) / 2) + 31) / 32 * 32;
}

template <int D>
__global__ void __launch_bounds__(coef_threads<D>()) k_cluster_coef(const int64_t* __restrict__ nclu, const int32_t* __restrict__ cnode,
                               const uint8_t* __restrict__ has, const double* __restrict__ geom,
                               const double* __restrict__ beta, const double* __restrict__ vinvT,
                               const double* __restrict__ cvel, float* __restrict__ coef32)
{
    constexpr int d = D, M = (D + 1) * (D + 2) / 2;
    __shared__ double u[3 * kMaxM];
    const int64_t ncl = *nclu;
    for (int64_t cs = blockIdx.x; cs < ncl; cs += gridDim.x) {
        if (!has[cs]) continue;
        const double* g = geom + 13 * (int64_t)cnode[cs];
        __syncthreads();  // u of the previous cluster is no longer read
        for (int m = threadIdx.x; m < M; m += blockDim.x) {
            const double b1 = beta[3 * m], b2 = beta[3 * m + 1], b3 = beta[3 * m + 2];
            const double sx = (b1 * g[0] + b2 * g[3]) + b3 * g[6];
            const double sy = (b1 * g[1] + b2 * g[4]) + b3 * g[7];
            const double sz = (b1 * g[2] + b2 * g[5]) + b3 * g[8];
            const double rho = sqrt((sx * sx + sy * sy) + sz * sz);
            double rd = 1.0;
            for (int e = 0; e < d; e++) rd *= rho;
            const double* v = cvel + 3 * (cs * M + m);
            u[3 * m] = rd * v[0];
            u[3 * m + 1] = rd * v[1];
            u[3 * m + 2] = rd * v[2];
        }
        __syncthreads();
        const int t = threadIdx.x;
        if (t < 3 * M) {
            const int k = t / 3, comp = t - 3 * k;
            double acc = 0.0;
            for (int m = 0; m < M; m++) acc += vinvT[m * M + k] * u[3 * m + comp];
            coef32[4 * (cs * M + k) + comp] = (float)acc;  // float4 per coefficient, w unused
        }
    }
}

// Mixed precision: the ancestor clusters with CP or CC pairs of every leaf, its own node
// included when it is one, from the leaf up: anc[L * A] = their count (at most A - 1),
// anc[L * A + 1 + i] = their cluster slots.  One thread per leaf, so that the particles read
// their leaf's list instead of each walking the parent chain.
__global__ void k_leaf_anc(const int64_t* __restrict__ nleaves, int64_t lcap, const int32_t* __restrict__ leaves,
                           const int32_t* __restrict__ parent, const int32_t* __restrict__ cluster_slot,
                           const uint8_t* __restrict__ has, int A, int32_t* __restrict__ anc)
{
    const int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (L >= min(*nleaves, lcap)) return;
    int32_t* o = anc + L * A;
    int k = 0;
    for (int32_t a = leaves[L]; a >= 0 && k < A - 1; a = parent[a]) {
        const int32_t cs = cluster_slot[a];
        if (cs >= 0 && has[cs]) o[1 + k++] = cs;
    }
    o[0] = k;
}

// Mixed precision: adds to every particle x (sorted slot) x crossed with the sum of the
// interpolants of its ancestor clusters that have CP or CC pairs (its leaf included when that is
// such a cluster), each evaluated in FP32 (Sec. 3.3: each target cluster's polynomial at every
// particle below it).  One CTA per leaf: its clusters' coefficients and frames are staged in
// shared memory by all threads at once (one round of independent loads), then each thread
// takes particles of the leaf.  Barycentric coordinates come from the FP32 frame about the
// cluster centre and x - c formed from the hi/lo pairs, so they carry no cancellation; the
// coefficients describe a smooth interpolant in a basis that is non-negative on the triangle,
// so the evaluation carries none of the contraction's.
constexpr int kFrame32 = 18;  // floats per FP32 cluster frame

template <int D>
__global__ void __launch_bounds__(128) k_downward32(const int64_t* __restrict__ nleaves, int64_t lcap,
                                                    const int32_t* __restrict__ leaves,
                                                    const int32_t* __restrict__ start,
                                                    const int32_t* __restrict__ count,
                                                    const int32_t* __restrict__ anc, int A,
                                                    const float* __restrict__ frame32,
                                                    const double4* __restrict__ src64,
                                                    const float4* __restrict__ src_hl,
                                                    const int32_t* __restrict__ perm,
                                                    const float4* __restrict__ coef4, double* __restrict__ vel)
{
    constexpr int M = (D + 1) * (D + 2) / 2;
    extern __shared__ float4 sh[];  // [A - 1][M] coefficients, then [A - 1][18] frame floats
    float* fr = reinterpret_cast<float*>(sh + (int64_t)(A - 1) * M);
    const int64_t nl = min(*nleaves, lcap);  // a recorded step with more leaves is redone
    for (int64_t L = blockIdx.x; L < nl; L += gridDim.x) {
        const int32_t* o = anc + L * A;
        const int na = o[0];
        if (na == 0) continue;
        const int32_t node = leaves[L];
        const int32_t st = start[node], cnt = count[node];
        __syncthreads();  // the previous leaf's staged clusters are no longer read
        for (int t = threadIdx.x; t < na * M; t += blockDim.x) {
            const int i = t / M;
            sh[t] = coef4[(int64_t)o[1 + i] * M + (t - i * M)];
        }
        for (int t = threadIdx.x; t < na * kFrame32; t += blockDim.x) {
            const int i = t / kFrame32;
            fr[t] = frame32[(int64_t)o[1 + i] * kFrame32 + (t - i * kFrame32)];
        }
        __syncthreads();
        for (int64_t j = st + threadIdx.x; j < (int64_t)st + cnt; j += blockDim.x) {
            const float4 hi = src_hl[2 * j], lo = src_hl[2 * j + 1];
            float fx = 0.f, fy = 0.f, fz = 0.f;  // the interpolated -(1/4 pi) S
            for (int i = 0; i < na; i++) {
                const float* h = fr + kFrame32 * i;
                float b1, b2, b3;
                bary32(h, (hi.x - h[12]) + (lo.x - h[15]), (hi.y - h[13]) + (lo.y - h[16]),
                       (hi.z - h[14]) + (lo.z - h[17]), b1, b2, b3);
                eval_poly4<D>(b1, b2, b3, sh + i * M, fx, fy, fz);
            }
            const double4 x = src64[j];
            const double ax = fx, ay = fy, az = fz;
            const int64_t r = perm[j];
            vel[3 * r] += x.y * az - x.z * ay;
            vel[3 * r + 1] += x.z * ax - x.x * az;
            vel[3 * r + 2] += x.x * ay - x.y * ax;
        }
    }
}

template <int D>
constexpr int M_of()
{
    return (D + 1) * (D + 2) / 2;
}

template <int D>
int launch_down(sts_ctx* c, const RefTable* ref, int levels, int64_t C, int64_t lcap, double* vel, bool mixed,
                cudaStream_t s)
{
    const unsigned gl = (unsigned)std::min<int64_t>(C, 16 * (int64_t)c->num_sms);
    if (mixed) {
        const int A = levels + 1;  // a leaf has at most `levels` ancestors (itself included)
        if (proxy_weights_tc_supported(D)) {
            // on the tensor cores (exact digit products, sts_tc.cu)
            const int rc = cluster_coef_tc(c, ref, D, C, c->cvel.p, c->cdown32.p, s);
            if (rc) return rc;
        } else {
            (k_cluster_coef<D><<<gl, coef_threads<D>(), 0, s>>>(c->dc.p + kDcClusters, c->cluster_node.p, c->chas.p,
                                                                 c->nd_geom.p, ref->d_beta.p, ref->d_vinvT.p,
                                                                 c->cvel.p, c->cdown32.p),
             note_launch());
        }
        if (lcap > 0)
            (k_leaf_anc<<<blocks(lcap, 128), 128, 0, s>>>(c->dc.p + kDcLeaves, lcap, c->leaves.p, c->nd_parent.p,
                                                          c->cluster_slot.p, c->chas.p, A, c->leaf_anc.p),
             note_launch());
        const size_t smem = (size_t)(A - 1) * (M_of<D>() * sizeof(float4) + kFrame32 * sizeof(float));
        if (!c->capturing) {  // the largest a recording can ask for: every level of the deepest tree
            const size_t smax = (size_t)(kMaxLevel + 2) * (M_of<D>() * sizeof(float4) + kFrame32 * sizeof(float));
            STS_CUDA(cudaFuncSetAttribute(k_downward32<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax));
        }
        if (lcap > 0)
            (k_downward32<D><<<(unsigned)std::min<int64_t>(lcap, 1 << 30), 128, smem, s>>>(
                 c->dc.p + kDcLeaves, lcap, c->leaves.p, c->nd_start.p, c->nd_count.p, c->leaf_anc.p, A,
                 c->up_frame32.p, c->src64.p, c->src_hl.p, c->perm.p,
                 reinterpret_cast<const float4*>(c->cdown32.p), vel),
             note_launch());
        return STS_OK;
    }
    for (int l = 0; l < levels; l++)
        (k_down_level<D><<<gl, 64, 0, s>>>(c->dc.p + kDcLevel, l, c->nd_parent.p, c->cluster_slot.p, c->chas.p,
                                           c->cacc.p, c->nd_geom.p, c->up_frame.p, c->prx64.p, ref->d_beta.p,
                                           ref->d_vinvT.p, c->cvel.p, c->cdown.p),
         note_launch());
    (k_downward<D><<<blocks(c->n, 128), 128, 0, s>>>(c->n, c->slot_leaf.p, c->leaves.p, c->nd_parent.p,
                                                      c->cluster_slot.p, c->cacc.p, c->up_frame.p, c->src64.p,
                                                      c->perm.p, c->cdown.p, vel),
     note_launch());
    return STS_OK;
}

}  // namespace

int evaluate_dual(sts_ctx* c, int degree, int precision, double tau, double* vel, cudaStream_t s)
{
    // PP and PC: the leaf lists hold the dual traversal's pairs of the target leaves
    int rc = evaluate(c, degree, precision, tau, vel, s);
    if (rc) return rc;
    const bool cap = c->capturing;
    const int64_t C = cap ? c->nodes_rec : c->nclusters;
    if (C == 0 || c->n < 2) return STS_OK;
    if (!cap && c->dual_n[2] == 0 && c->dual_n[3] == 0) return STS_OK;  // no CP or CC pairs
    RefTable* ref = get_ref(c, degree);
    if (!ref) return STS_ERR_CUDA;
    const int M = ref->M;
    if ((rc = cluster_tasks(c, M, s))) return rc;
    if (!cap) {
        STS_CUDA(c->cvel.reserve(3 * C * M + 3));
        STS_CUDA(c->cdown.reserve(3 * C * M + 3));
        STS_CUDA(c->cdown32.reserve(4 * C * M + 4));
        STS_CUDA(c->cacc.reserve(C + 1));
    }
    // CP and CC: the velocity at the proxy points of the target clusters
    ListSet ls;
    ls.tasks = c->ctasks.p;
    ls.ntasks_d = cluster_task_count(c);
    ls.ntasks = c->nctasks;
    ls.far_off = c->cfar_off.p;
    ls.near_coff = c->cnear_coff.p;
    ls.far_ent = c->cfar_ent.p;
    ls.near_ent = c->cnear_ent.p;
    ls.tgt32 = c->prx32.p;
    ls.tgt64 = c->prx64.p;
    ls.perm = nullptr;
    ls.ntargets = C * M;
    phase_begin(c, kPhCluster, s);
    if ((rc = evaluate_lists(c, ls, degree, precision, tau, c->ccorr, c->cvel.p, s, -1))) return rc;
    // the interpolants (FP64: passed down level by level; mixed: one per cluster, every
    // ancestor's evaluated at each particle), then evaluated at the particles
    const int levels = (cap ? c->plan.depth : (int)c->deepest) + 1;
    const bool mixed = precision != STS_FP64;
    // leaves held by the per-leaf ancestor lists: all of them, or while recording the lists'
    // planned bound (a replay with more leaves sets the overflow bit and is redone)
    const int64_t lcap = cap ? std::min<int64_t>(c->n, c->plan.leaves + c->plan.leaves / 4 + 64) : c->nleaves;
    if (!cap && mixed) STS_CUDA(c->leaf_anc.reserve(lcap * (levels + 1) + 1));
    switch (degree) {
        case 1: rc = launch_down<1>(c, ref, levels, C, lcap, vel, mixed, s); break;
        case 2: rc = launch_down<2>(c, ref, levels, C, lcap, vel, mixed, s); break;
        case 3: rc = launch_down<3>(c, ref, levels, C, lcap, vel, mixed, s); break;
        case 4: rc = launch_down<4>(c, ref, levels, C, lcap, vel, mixed, s); break;
        case 5: rc = launch_down<5>(c, ref, levels, C, lcap, vel, mixed, s); break;
        case 6: rc = launch_down<6>(c, ref, levels, C, lcap, vel, mixed, s); break;
        case 7: rc = launch_down<7>(c, ref, levels, C, lcap, vel, mixed, s); break;
        case 8: rc = launch_down<8>(c, ref, levels, C, lcap, vel, mixed, s); break;
        case 9: rc = launch_down<9>(c, ref, levels, C, lcap, vel, mixed, s); break;
        case 10: rc = launch_down<10>(c, ref, levels, C, lcap, vel, mixed, s); break;
        case 11: rc = launch_down<11>(c, ref, levels, C, lcap, vel, mixed, s); break;
        case 12: rc = launch_down<12>(c, ref, levels, C, lcap, vel, mixed, s); break;
        case 13: rc = launch_down<13>(c, ref, levels, C, lcap, vel, mixed, s); break;
        case 14: rc = launch_down<14>(c, ref, levels, C, lcap, vel, mixed, s); break;
        case 15: rc = launch_down<15>(c, ref, levels, C, lcap, vel, mixed, s); break;
        default: rc = launch_down<16>(c, ref, levels, C, lcap, vel, mixed, s); break;
    }
    if (rc) return rc;
    phase_end(c, kPhCluster, s);
    STS_LAUNCH_CHECK();
    return STS_OK;
}

}  // namespace sts
