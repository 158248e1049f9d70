// Host-side tables of the tree code: the icosahedron whose faces are the 20 root
// triangles (Sec. 3, "Grids on a Sphere"), and per degree d the reference interpolation
// data of Sec. 3.2 / 3.3.2: approximate Fekete points on the reference simplex and the
// inverse of the SBB Vandermonde matrix at those points.
//
// Compiled without FMA contraction (-ffp-contract=off): the icosahedron values decide
// which face owns each particle, so every operation below is a plain IEEE double op in
// the order written.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "sts_internal.cuh"

namespace sts {

namespace {

struct h3 {
    double x, y, z;
};
h3 hmk(double x, double y, double z) { return h3{x, y, z}; }
h3 hadd(h3 a, h3 b) { return hmk(a.x + b.x, a.y + b.y, a.z + b.z); }
h3 hsub(h3 a, h3 b) { return hmk(a.x - b.x, a.y - b.y, a.z - b.z); }
double hdot(h3 a, h3 b) { return (a.x * b.x + a.y * b.y) + a.z * b.z; }
h3 hcross(h3 a, h3 b)
{
    return hmk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
h3 hunit(h3 s)
{
    double n = sqrt(hdot(s, s));
    return hmk(s.x / n, s.y / n, s.z / n);
}

}  // namespace

// The icosahedron, in the orientation and numbering this library fixes (the paper gives
// none): vertices are the cyclic families (0, +-1, +-g), (+-1, +-g, 0), (+-g, 0, +-1)
// (g = golden ratio; families in that order, sign pairs (+,+), (+,-), (-,+), (-,-)) scaled
// to unit length; faces are the vertex triples at unscaled pairwise squared distance 4,
// in lexicographic order, each stored counter-clockwise seen from outside; the face
// centre is the unit vector along the sum of its three vertices.
void icosahedron(double V[12][3], int F[20][3], double C[20][3])
{
    const double g = (1.0 + sqrt(5.0)) / 2.0;
    const double sgn[4][2] = {{1.0, 1.0}, {1.0, -1.0}, {-1.0, 1.0}, {-1.0, -1.0}};
    h3 raw[12], u[12];
    int n = 0;
    for (int fam = 0; fam < 3; fam++)
        for (int s = 0; s < 4; s++) {
            const double a = sgn[s][0], b = sgn[s][1];
            if (fam == 0)
                raw[n] = hmk(0.0, a * 1.0, b * g);
            else if (fam == 1)
                raw[n] = hmk(a * 1.0, b * g, 0.0);
            else
                raw[n] = hmk(a * g, 0.0, b * 1.0);
            n++;
        }
    for (int i = 0; i < 12; i++) {
        u[i] = hunit(raw[i]);
        V[i][0] = u[i].x;
        V[i][1] = u[i].y;
        V[i][2] = u[i].z;
    }
    int nf = 0;
    for (int i = 0; i < 12; i++)
        for (int j = i + 1; j < 12; j++)
            for (int k = j + 1; k < 12; k++) {
                h3 eij = hsub(raw[i], raw[j]), eik = hsub(raw[i], raw[k]), ejk = hsub(raw[j], raw[k]);
                if (fabs(hdot(eij, eij) - 4.0) > 1e-9 || fabs(hdot(eik, eik) - 4.0) > 1e-9 ||
                    fabs(hdot(ejk, ejk) - 4.0) > 1e-9)
                    continue;
                const bool ccw = hdot(u[i], hcross(u[j], u[k])) > 0.0;
                F[nf][0] = i;
                F[nf][1] = ccw ? j : k;
                F[nf][2] = ccw ? k : j;
                nf++;
            }
    for (int f = 0; f < 20; f++) {
        h3 c = hunit(hadd(hadd(u[F[f][0]], u[F[f][1]]), u[F[f][2]]));
        C[f][0] = c.x;
        C[f][1] = c.y;
        C[f][2] = c.z;
    }
}

// Bernstein-monomial row of degree d at barycentric b (Sec. 3.2: B_ijk = b1^i b2^j b3^k,
// i + j + k = d), in the order i = d..0, then j = d - i..0.
static void sbb_row(int d, const double b[3], double* out)
{
    double p[3][kMaxDegree + 1];
    for (int a = 0; a < 3; a++) {
        p[a][0] = 1.0;
        for (int e = 1; e <= d; e++) p[a][e] = p[a][e - 1] * b[a];
    }
    int k = 0;
    for (int i = d; i >= 0; i--)
        for (int j = d - i; j >= 0; j--) out[k++] = (p[0][i] * p[1][j]) * p[2][d - i - j];
}

// Approximate Fekete points: greedy column pivoting on the matrix whose columns are the
// SBB rows of candidate points (the barycentric lattice of resolution 3d, enumerated
// p = 3d..0, q = 3d - p..0).  At each step the candidate whose column has the largest
// component orthogonal to the columns already chosen is taken (ties within a relative
// 1e-9 go to the lowest candidate index).  Implemented with modified Gram-Schmidt on
// the residual columns.  Then V_ref[m][k] = B_k(beta_m) is inverted by LU with partial
// pivoting.
int build_ref_table(int d, RefTable* t)
{
    if (d < 1 || d > kMaxDegree) return STS_ERR_ARG;
    const int M = (d + 1) * (d + 2) / 2, R = 3 * d, K = (R + 1) * (R + 2) / 2;
    std::vector<double> cand(3 * (size_t)K), res((size_t)K * M), q(M);
    std::vector<char> taken(K, 0);
    int c = 0;
    for (int p = R; p >= 0; p--)
        for (int qq = R - p; qq >= 0; qq--) {
            double b[3] = {(double)p / (double)R, (double)qq / (double)R,
                           (double)(R - p - qq) / (double)R};
            memcpy(&cand[3 * (size_t)c], b, sizeof(b));
            sbb_row(d, b, &res[(size_t)c * M]);
            c++;
        }
    t->degree = d;
    t->M = M;
    t->beta.assign(3 * (size_t)M, 0.0);
    for (int s = 0; s < M; s++) {
        double best = -1.0;
        std::vector<double> nrm(K, 0.0);
        for (c = 0; c < K; c++) {
            if (taken[c]) continue;
            const double* r = &res[(size_t)c * M];
            double a = 0.0;
            for (int k = 0; k < M; k++) a += r[k] * r[k];
            nrm[c] = a;
            if (a > best) best = a;
        }
        int pick = -1;
        for (c = 0; c < K; c++)
            if (!taken[c] && nrm[c] >= best * (1.0 - 1e-9)) {
                pick = c;
                break;
            }
        if (pick < 0 || !(best > 0.0)) return STS_ERR_ARG;
        taken[pick] = 1;
        memcpy(&t->beta[3 * (size_t)s], &cand[3 * (size_t)pick], 3 * sizeof(double));
        const double inv = 1.0 / sqrt(nrm[pick]);
        for (int k = 0; k < M; k++) q[k] = res[(size_t)pick * M + k] * inv;
        for (c = 0; c < K; c++) {
            if (taken[c]) continue;
            double* r = &res[(size_t)c * M];
            double a = 0.0;
            for (int k = 0; k < M; k++) a += q[k] * r[k];
            for (int k = 0; k < M; k++) r[k] -= a * q[k];
        }
    }
    // LU with partial pivoting of V, then V^{-1} column by column.
    std::vector<double> lu((size_t)M * M);
    std::vector<int> piv(M);
    for (int m = 0; m < M; m++) sbb_row(d, &t->beta[3 * (size_t)m], &lu[(size_t)m * M]);
    for (int k = 0; k < M; k++) {
        int p = k;
        for (int i = k + 1; i < M; i++)
            if (fabs(lu[(size_t)i * M + k]) > fabs(lu[(size_t)p * M + k])) p = i;
        if (lu[(size_t)p * M + k] == 0.0) return STS_ERR_ARG;
        piv[k] = p;
        if (p != k)
            for (int j = 0; j < M; j++) {
                double tmp = lu[(size_t)k * M + j];
                lu[(size_t)k * M + j] = lu[(size_t)p * M + j];
                lu[(size_t)p * M + j] = tmp;
            }
        for (int i = k + 1; i < M; i++) {
            double f = lu[(size_t)i * M + k] / lu[(size_t)k * M + k];
            lu[(size_t)i * M + k] = f;
            for (int j = k + 1; j < M; j++) lu[(size_t)i * M + j] -= f * lu[(size_t)k * M + j];
        }
    }
    t->vinv.assign((size_t)M * M, 0.0);
    std::vector<double> x(M);
    for (int col = 0; col < M; col++) {
        for (int i = 0; i < M; i++) x[i] = (i == col) ? 1.0 : 0.0;
        for (int k = 0; k < M; k++) {
            double tmp = x[k];
            x[k] = x[piv[k]];
            x[piv[k]] = tmp;
        }
        for (int i = 0; i < M; i++)
            for (int j = 0; j < i; j++) x[i] -= lu[(size_t)i * M + j] * x[j];
        for (int i = M - 1; i >= 0; i--) {
            for (int j = i + 1; j < M; j++) x[i] -= lu[(size_t)i * M + j] * x[j];
            x[i] /= lu[(size_t)i * M + i];
        }
        for (int k = 0; k < M; k++) t->vinv[(size_t)k * M + col] = x[k];
    }
    return STS_OK;
}

RefTable* get_ref(sts_ctx* ctx, int d)
{
    if ((int)ctx->refs.size() <= d) ctx->refs.resize(d + 1, nullptr);
    if (ctx->refs[d]) return ctx->refs[d];
    RefTable* t = new RefTable();
    if (build_ref_table(d, t) != STS_OK) {
        delete t;
        set_error("proxy reference table for degree %d failed", d);
        return nullptr;
    }
    std::vector<double> vt(t->vinv.size());
    for (int k = 0; k < t->M; k++)
        for (int m = 0; m < t->M; m++) vt[(size_t)m * t->M + k] = t->vinv[(size_t)k * t->M + m];
    if (t->d_beta.reserve(t->beta.size()) != cudaSuccess ||
        t->d_vinv.reserve(t->vinv.size()) != cudaSuccess ||
        t->d_vinvT.reserve(vt.size()) != cudaSuccess ||
        cudaMemcpy(t->d_beta.p, t->beta.data(), t->beta.size() * sizeof(double),
                   cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(t->d_vinv.p, t->vinv.data(), t->vinv.size() * sizeof(double),
                   cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(t->d_vinvT.p, vt.data(), vt.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
        t->d_beta.release();
        t->d_vinv.release();
        t->d_vinvT.release();
        delete t;
        set_error("uploading the degree-%d proxy table failed", d);
        return nullptr;
    }
    // operand B of the tensor-core contraction.  Row k of V_ref^-1 is divided by 2^E[k], E[k]
    // the power of two nearest the integral of basis function k over the reference simplex
    // (a! b! c! 2 / (d + 2)!), by which the kernel multiplies moment k: the moments then have
    // comparable sizes, so 32 bits of the largest keep every moment's leading bits.  Column m
    // is then scaled into (-1/2, 1/2) by 2^-F[m] and cut into kTcSlices balanced base-256
    // digits (each in [-128, 128]; every exact operation, the last remainder below 2^-57 of
    // the column's largest entry).
    const int M = t->M;
    t->tcKp = (M + 15) / 16 * 16;
    t->tcNp = t->tcKp;
    std::vector<uint16_t> B((size_t)kTcSlices * t->tcNp * t->tcKp, 0);
    std::vector<int32_t> F((size_t)t->tcNp, 0), Ek((size_t)t->tcKp, 0);
    {
        double fact[2 * kMaxDegree + 3];
        fact[0] = 1.0;
        for (int i = 1; i <= 2 * kMaxDegree + 2; i++) fact[i] = fact[i - 1] * i;
        int k = 0;
        for (int i = d; i >= 0; i--)
            for (int j = d - i; j >= 0; j--) {
                const double mono = fact[i] * fact[j] * fact[d - i - j] * 2.0 / fact[d + 2];
                Ek[k++] = -(int32_t)std::lround(std::log2(mono));
            }
    }
    for (int m = 0; m < M; m++) {
        double mx = 0.0;
        for (int k = 0; k < M; k++) mx = std::max(mx, std::fabs(std::ldexp(t->vinv[(size_t)k * M + m], -Ek[k])));
        int e = 0;
        if (mx > 0.0) std::frexp(mx, &e);  // mx < 2^e
        F[m] = e + 1;                      // entries below 2^(F - 1) = 1/2 of 2^F
        for (int k = 0; k < M; k++) {
            double x = std::ldexp(t->vinv[(size_t)k * M + m], -Ek[k] - F[m]);  // |x| < 1/2, exact
            for (int b = 0; b < kTcSlices; b++) {
                x *= 256.0;                       // exact
                const double dg = std::nearbyint(x);  // |dg| <= 128
                x -= dg;                          // exact, |x| <= 1/2
                const float f = (float)dg;
                uint32_t u;
                std::memcpy(&u, &f, 4);
                const size_t off = (size_t)b * t->tcNp * t->tcKp * 2 + tc_kmajor_offset(m, k, t->tcKp);
                B[off / 2] = (uint16_t)(u >> 16);  // an integer of at most 8 bits: exact in bf16
            }
        }
    }
    // operand B of the coefficient contraction: row k of V_ref^-1 scaled by 2^-Fr[k] into
    // (-1/2, 1/2), the same balanced digits, stored as [Np rows k, Kp columns m]
    std::vector<uint16_t> Br((size_t)kTcSlices * t->tcNp * t->tcKp, 0);
    std::vector<int32_t> Fr((size_t)t->tcNp, 0);
    for (int k = 0; k < M; k++) {
        double mx = 0.0;
        for (int m = 0; m < M; m++) mx = std::max(mx, std::fabs(t->vinv[(size_t)k * M + m]));
        int e = 0;
        if (mx > 0.0) std::frexp(mx, &e);
        Fr[k] = e + 1;
        for (int m = 0; m < M; m++) {
            double x = std::ldexp(t->vinv[(size_t)k * M + m], -Fr[k]);
            for (int b = 0; b < kTcSlices; b++) {
                x *= 256.0;
                const double dg = std::nearbyint(x);
                x -= dg;
                const float f = (float)dg;
                uint32_t u;
                std::memcpy(&u, &f, 4);
                const size_t off = (size_t)b * t->tcNp * t->tcKp * 2 + tc_kmajor_offset(k, m, t->tcKp);
                Br[off / 2] = (uint16_t)(u >> 16);
            }
        }
    }
    if (t->d_tcB.reserve(B.size()) != cudaSuccess || t->d_tcF.reserve(F.size()) != cudaSuccess ||
        t->d_tcBr.reserve(Br.size()) != cudaSuccess || t->d_tcFr.reserve(Fr.size()) != cudaSuccess ||
        cudaMemcpy(t->d_tcBr.p, Br.data(), Br.size() * sizeof(uint16_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(t->d_tcFr.p, Fr.data(), Fr.size() * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        t->d_tcE.reserve(Ek.size()) != cudaSuccess ||
        cudaMemcpy(t->d_tcB.p, B.data(), B.size() * sizeof(uint16_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(t->d_tcF.p, F.data(), F.size() * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(t->d_tcE.p, Ek.data(), Ek.size() * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess) {
        t->d_beta.release();
        t->d_vinv.release();
        t->d_vinvT.release();
        t->d_tcB.release();
        t->d_tcF.release();
        t->d_tcE.release();
        t->d_tcBr.release();
        t->d_tcFr.release();
        delete t;
        set_error("uploading the degree-%d tensor-core table failed", d);
        return nullptr;
    }
    ctx->refs[d] = t;
    return t;
}

}  // namespace sts
