// Sorted source data and the upward pass of the tree code (Sec. 3.3.2, PC interaction):
// for every cluster (a triangle holding more than N_T particles) the SBB moments
//     omega_k = sum_j B_k(b(y_j)) w_j,   B_k(b) = b1^a b2^b b3^c,  a + b + c = d,
// with b(y) the spherical barycentric coordinates of y in the triangle (y = b1 v1 + b2 v2 +
// b3 v3), are folded into proxy-point weights
//     W_m = rho_m^d sum_k (V_ref^{-1})[k][m] omega_k,   y~_m = unit(sum_i beta_mi v_i),
//     rho_m = |sum_i beta_mi v_i|,
// so that the PC interaction sum_k alpha_k(x) omega_k of Sec. 3.3.2 equals
// sum_m G(x, y~_m) W_m for every target x (V_s = diag(rho^-d) V_ref because B_k is
// homogeneous of degree d and b(y~_m) = beta_m / rho_m).
//
// Moments: one CTA per (cluster, 128-particle chunk).  Each thread tabulates the powers
// b^0..b^d of its particle in shared memory; thread k then sums w_j B_k(b_j) over the chunk.
// The mixed path computes b = b(c) + T^{-1} (y - c) in FP32 from the FP64 offset y - c to
// the cluster centre c, so b keeps FP32 relative accuracy however small the triangle.
// Weights: one CTA per cluster sums the chunk partials in FP64 in a fixed order and applies
// V_ref^{-1} in FP64; in mixed precision (degree <= 11) the contraction runs exactly on the
// tensor cores instead (sts_tc.cu) and this kernel only forms the proxy points.  The SBB
// monomial basis is badly conditioned (cond(V_ref) ~ 3.5e5 at d = 8), so the contraction is
// never rounded to FP32 (or TF32): that would put errors of eps * |V_ref^{-1}| |omega| into W.
// Rounding the moments themselves to FP32 is benign: it perturbs W only along directions the
// interpolant maps back with norm ~1.  The cluster table (numbers, moment tasks, barycentric
// frames) comes with the tree build.
#include <algorithm>

#include "sts_internal.cuh"

namespace sts {
namespace {

inline unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Sorted copies: src64[k] = (x, y, z, 2 zeta A) of particle perm[k]; src32[k] = the same
// relative to the circumcentre of its leaf, rounded to FP32.
__global__ void k_prepare(const double* __restrict__ pos, const double* __restrict__ zeta,
                          const double* __restrict__ area, const int32_t* __restrict__ perm,
                          const int32_t* __restrict__ slot_leaf, const int32_t* __restrict__ leaves,
                          const double* __restrict__ geom, int64_t n, double4* __restrict__ src64,
                          float4* __restrict__ src32, float4* __restrict__ src_hl)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t i = perm[k];
    const double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
    const double zw = zeta[i] * area[i];
    const double w2 = 2.0 * zw;
    src64[k] = make_double4(x, y, z, w2);
    // x = hi + lo to about 2^-48 |x|: FP32 differences of these pairs keep FP32 relative accuracy
    const float hx = (float)x, hy = (float)y, hz = (float)z;
    src_hl[2 * k] = make_float4(hx, hy, hz, (float)zw);
    src_hl[2 * k + 1] = make_float4((float)(x - (double)hx), (float)(y - (double)hy), (float)(z - (double)hz), 0.f);
    const double* c = geom + 13 * (int64_t)leaves[slot_leaf[k]] + 9;
    src32[k] = make_float4((float)(x - c[0]), (float)(y - c[1]), (float)(z - c[2]), (float)w2);
}

// Exponents (a, b, c) of SBB function k of degree d: a = d..0, then b = d - a..0.
__device__ __forceinline__ void sbb_exponents(int d, int k, int& a, int& b, int& c)
{
    int q = 0;
    while ((q + 1) * (q + 2) / 2 <= k) q++;
    const int r = k - q * (q + 1) / 2;
    a = d - q;
    b = q - r;
    c = r;
}

// Moments of one (cluster, chunk) task.  T = float (mixed) or double (FP64).  Each thread
// tabulates the powers of its particle's barycentric coordinates; then G = 128 / M groups
// of M threads (thread = basis function k) each sum a share of the chunk's particles, and
// the group sums are added in a fixed order.
template <class T>
__global__ void __launch_bounds__(kUpChunk)
k_upward(const int2* __restrict__ tasks, const int32_t* __restrict__ cnode,
         const int32_t* __restrict__ start, const int32_t* __restrict__ count,
         const double* __restrict__ geom, const double* __restrict__ frame, const float* __restrict__ frame32,
         const double4* __restrict__ src64, const float4* __restrict__ src_hl, int d, int M,
         double* __restrict__ part, const int64_t* __restrict__ ntasks)
{
    if (blockIdx.x >= *ntasks) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* P = reinterpret_cast<T*>(smem_raw);  // [3][d+1][kUpChunk + 1]
    constexpr int LD = kUpChunk + 1;
    T* Wt = P + 3 * (d + 1) * LD;           // [kUpChunk]
    T* G2 = Wt + kUpChunk;                  // [kUpChunk] group partial sums

    const int2 tk = tasks[blockIdx.x];
    const int32_t node = cnode[tk.x];
    const double* f = frame + 12 * (int64_t)tk.x;
    const int t = threadIdx.x;
    const int64_t j = (int64_t)start[node] + tk.y + t;
    const int nv = min(kUpChunk, count[node] - tk.y);
    const bool valid = t < nv;
    T b[3] = {T(0), T(0), T(0)};
    T w = T(0);
    if (valid) {
        if (sizeof(T) == sizeof(double)) {
            const double4 y = src64[j];
            w = T(0.5 * y.w);
            for (int a = 0; a < 3; a++) b[a] = T(f[3 * a] * y.x + f[3 * a + 1] * y.y + f[3 * a + 2] * y.z);
        } else {
            // all-FP32: y - c from the hi/lo pairs, then the frame about the centre
            const float4 hi = src_hl[2 * j], lo = src_hl[2 * j + 1];
            const float* h = frame32 + 18 * (int64_t)tk.x;
            const float dx = (hi.x - h[12]) + (lo.x - h[15]);
            const float dy = (hi.y - h[13]) + (lo.y - h[16]);
            const float dz = (hi.z - h[14]) + (lo.z - h[17]);
            w = T(hi.w);
            for (int a = 0; a < 3; a++) b[a] = h[9 + a] + (h[3 * a] * dx + h[3 * a + 1] * dy + h[3 * a + 2] * dz);
        }
    }
    for (int a = 0; a < 3; a++) {
        T pw = T(1);
        P[(a * (d + 1) + 0) * LD + t] = pw;
        for (int e = 1; e <= d; e++) {
            pw = pw * b[a];
            P[(a * (d + 1) + e) * LD + t] = pw;
        }
    }
    Wt[t] = w;
    __syncthreads();
    const int G = max(1, kUpChunk / M);
    for (int k0 = 0; k0 < M; k0 += kUpChunk / G) {
        // thread t: basis k = k0 + t % (128 / G) ... in groups of M threads
        const int per = M < kUpChunk ? M : kUpChunk;
        const int grp = t / per, k = k0 + t % per;
        T acc = T(0);
        if (grp < G && k < M) {
            int ea, eb, ec;
            sbb_exponents(d, k, ea, eb, ec);
            const T* p1 = P + (0 * (d + 1) + ea) * LD;
            const T* p2 = P + (1 * (d + 1) + eb) * LD;
            const T* p3 = P + (2 * (d + 1) + ec) * LD;
            for (int q = grp; q < nv; q += G) acc += ((p1[q] * p2[q]) * p3[q]) * Wt[q];
        }
        if (grp < G && k < M) G2[t] = acc;
        __syncthreads();
        if (t < per && k0 + t < M) {
            double sum = 0.0;
            for (int gg = 0; gg < G; gg++) sum += (double)G2[gg * per + t];
            part[(int64_t)blockIdx.x * M + k0 + t] = sum;
        }
        __syncthreads();
        if (G > 1) break;  // with G > 1 groups, M < 128 and one pass covers every k
    }
}

// Proxy points and weights of one cluster (one CTA per cluster).  The contraction with
// V_ref^-T stays FP64 in both precisions: its entries alternate in sign and reach ~1e5 at
// d = 8, so FP32 rounding of the products would put errors ~1e-5 into the far field.  Four
// interleaved partial sums shorten the dependent FP64 chain.  MIXED: the proxy points are
// normalised with a reciprocal square root (FP32 copies only need the FP64 point to an ulp or
// so).  A fixed grid strides over the clusters (their count is on the device).  Used in FP64
// precision, and in mixed precision above the tensor-core tables' degree; otherwise the
// tensor-core contraction (sts_tc.cu) forms the weights and places the proxy points itself.
template <bool MIXED>
__global__ void k_contract(const int32_t* __restrict__ cnode, const int64_t* __restrict__ toff,
                           const double* __restrict__ part, const double* __restrict__ geom,
                           const double* __restrict__ beta, const double* __restrict__ vinv, int d,
                           int M, double4* __restrict__ prx64, float4* __restrict__ prx32,
                           const int64_t* __restrict__ nclu, double* __restrict__ prx_rd)
{
    __shared__ double om[kMaxM + 3];
    const int64_t ncl = *nclu;
    for (int64_t c = blockIdx.x; c < ncl; c += gridDim.x) {
        {
            const int64_t q0 = toff[cnode[c]], q1 = toff[cnode[c] + 1];
            __syncthreads();  // om of the previous cluster is no longer read
            for (int k = threadIdx.x; k < M + 3; k += blockDim.x) {
                double s = 0.0;
                if (k < M)
                    for (int64_t q = q0; q < q1; q++) s += part[q * M + k];
                om[k] = s;  // om[M .. M + 2] = 0 pads the four-way split below
            }
            __syncthreads();
        }
        const double* g = geom + 13 * (int64_t)cnode[c];
        for (int m = threadIdx.x; m < M; m += blockDim.x) {
            double a4[4] = {0.0, 0.0, 0.0, 0.0};
            for (int k = 0; k < M; k += 4) {
#pragma unroll
                for (int u = 0; u < 4; u++)
                    if (k + u < M) a4[u] += vinv[(k + u) * M + m] * om[k + u];
            }
            const double acc = (a4[0] + a4[1]) + (a4[2] + a4[3]);
            const double b1 = beta[3 * m], b2 = beta[3 * m + 1], b3 = beta[3 * m + 2];
            const double sx = (b1 * g[0] + b2 * g[3]) + b3 * g[6];
            const double sy = (b1 * g[1] + b2 * g[4]) + b3 * g[7];
            const double sz = (b1 * g[2] + b2 * g[5]) + b3 * g[8];
            const double ss = (sx * sx + sy * sy) + sz * sz;
            double yx, yy, yz, rho;
            if (MIXED) {
                const double ri = rsqrt(ss);
                yx = sx * ri;
                yy = sy * ri;
                yz = sz * ri;
                rho = ss * ri;
            } else {
                rho = sqrt(ss);
                yx = sx / rho;
                yy = sy / rho;
                yz = sz / rho;
            }
            double rd = 1.0;
            for (int e = 0; e < d; e++) rd *= rho;
            prx_rd[c * M + m] = rd;
            const double W2 = 2.0 * (rd * acc);
            prx64[c * M + m] = make_double4(yx, yy, yz, W2);
            prx32[c * M + m] = make_float4((float)(yx - g[9]), (float)(yy - g[10]), (float)(yz - g[11]), (float)W2);
        }
    }
}

}  // namespace

int prepare_sources(sts_ctx* c, const double* zeta, const double* area, cudaStream_t s)
{
    const int64_t n = c->n;
    STS_CUDA(c->src64.reserve(n + 1));
    STS_CUDA(c->src32.reserve(n + 1));
    STS_CUDA(c->src_hl.reserve(2 * n + 2));
    if (n > 0)
        (k_prepare<<<blocks(n, 256), 256, 0, s>>>(c->pos.p, zeta, area, c->perm.p, c->slot_leaf.p, c->leaves.p,
                                                 c->nd_geom.p, n, c->src64.p, c->src32.p, c->src_hl.p),
         note_launch());
    STS_LAUNCH_CHECK();
    return STS_OK;
}

int upward_pass(sts_ctx* c, int degree, int precision, cudaStream_t s)
{
    RefTable* ref = get_ref(c, degree);
    if (!ref) return STS_ERR_CUDA;
    const int M = ref->M;
    const bool cap = c->capturing;
    const int64_t nclu = cap ? c->nodes_rec : c->nclusters;
    const int64_t nupt = cap ? c->up_tasks_rec : c->n_up_tasks;
    if (!cap) {
        STS_CUDA(c->prx64.reserve(nclu * M + 1));
        STS_CUDA(c->prx32.reserve(nclu * M + 1));
        STS_CUDA(c->prx_rd.reserve(nclu * M + 1));
        STS_CUDA(c->up_part.reserve(nupt * M + 1));
    }
    if (nclu == 0 || nupt == 0) {
        c->up_degree = degree;
        c->up_precision = precision;
        return STS_OK;
    }
    int64_t* dc = c->dc.p;
    const int LD = kUpChunk + 1;
    if (precision == STS_FP64) {
        const size_t sm = (3 * (degree + 1) * LD + 2 * kUpChunk) * sizeof(double);
        if (!cap) STS_CUDA(cudaFuncSetAttribute(k_upward<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        (k_upward<double><<<(unsigned)nupt, kUpChunk, sm, s>>>(
            c->up_tasks.p, c->cluster_node.p, c->nd_start.p, c->nd_count.p, c->nd_geom.p, c->up_frame.p,
            c->up_frame32.p, c->src64.p, c->src_hl.p, degree, M, c->up_part.p, dc + kDcUpTasks), note_launch());
    } else {
        const size_t sm = (3 * (degree + 1) * LD + 2 * kUpChunk) * sizeof(float);
        if (!cap) STS_CUDA(cudaFuncSetAttribute(k_upward<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        (k_upward<float><<<(unsigned)nupt, kUpChunk, sm, s>>>(
            c->up_tasks.p, c->cluster_node.p, c->nd_start.p, c->nd_count.p, c->nd_geom.p, c->up_frame.p,
            c->up_frame32.p, c->src64.p, c->src_hl.p, degree, M, c->up_part.p, dc + kDcUpTasks), note_launch());
    }
    if (precision == STS_MIXED && proxy_weights_tc_supported(degree)) {
        // mixed precision: the contraction on the tensor cores (exact digit products,
        // sts_tc.cu), which also places the proxy points
        int rc = proxy_weights_tc(c, ref, degree, nclu, s);
        if (rc) return rc;
    } else {
        (precision == STS_FP64 ? k_contract<false> : k_contract<true>)<<<
            (unsigned)std::min<int64_t>(nclu, 16 * (int64_t)c->num_sms), 64, 0, s>>>(
            c->cluster_node.p, c->up_toff.p, c->up_part.p, c->nd_geom.p, ref->d_beta.p, ref->d_vinv.p, degree, M,
            c->prx64.p, c->prx32.p, dc + kDcClusters, c->prx_rd.p);
        note_launch();
    }
    STS_LAUNCH_CHECK();
    c->up_degree = degree;
    c->up_precision = precision;
    return STS_OK;
}

}  // namespace sts
