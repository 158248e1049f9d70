// Adaptive mesh refinement of the particle triangulation (Appendix A): leaf triangles split
// into four when their circulation or vorticity variation is large, at most `levels` levels
// below the base mesh, and merge back when neither criterion holds.
//
// The base triangles (faces over the base particles) come from the caller.  Every triangle and
// vertex the refinement can ever create is numbered once on the host: level by level, each
// triangle of the previous level in order gives the midpoints of its edges (v1 v2), (v2 v3),
// (v3 v1), numbered when first met (a shared edge shares its midpoint), and the children
// (v1, m12, m31), (m12, v2, m23), (m31, m23, v3), (m12, m23, m31).  A pass then only flips
// per-triangle states and per-vertex flags on the device: midpoints are found by table, not
// by search.
//
// Readings (the appendix gives the criteria and the limits, not the bookkeeping):
//   area      A = 2 atan2(|a . (b x c)|, 1 + a.b + b.c + c.a), the spherical excess of the
//             triangle of the three current corner positions;
//   criteria  split a leaf when |A (z1 + z2 + z3) / 3| >= eps1 or max z - min z >= eps2 (below
//             the level limit); merge four leaf children when neither holds on the parent's
//             corners and none of them splits; all decisions on the state at the start of
//             the pass;
//   new vertex  a midpoint not alive yet is placed at unit(p_a + p_b) of its edge ends' current
//             positions, with vorticity (z_a + z_b) / 2;
//   particles the vertices that are corners of leaf triangles, weighted by the sum of A / 3
//             over those triangles.
//
// Compiled with --fmad=false: positions and decisions come out as a plain IEEE evaluation of
// the expressions below (the atan2 of the area is the one library function in them).
#include <algorithm>
#include <unordered_map>
#include <vector>

#include "sts_internal.cuh"

namespace sts {

struct AmrState {
    int64_t n0 = 0, nv = 0, t0 = 0, nt = 0;
    int levels = 0;
    DevBuf<int32_t> tv, tparent, tchild, vparent;
    DevBuf<int8_t> tlevel;
    DevBuf<uint8_t> tstate, valive, valive0, split, merge;
    DevBuf<double> pos, zeta, area;
    DevBuf<int32_t> flags;   // [nv] alive as int32 for the scan
    DevBuf<int64_t> scan;    // [nv + 1]
    DevBuf<int64_t> cnt;     // [4] splits, merges, alive, leaves
    int64_t nalive = 0;
};

namespace {

inline unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

__device__ __forceinline__ double tri_area(const double* __restrict__ pos, const int32_t* __restrict__ tv)
{
    const double* a = pos + 3 * (int64_t)tv[0];
    const double* b = pos + 3 * (int64_t)tv[1];
    const double* c = pos + 3 * (int64_t)tv[2];
    const double bcx = b[1] * c[2] - b[2] * c[1];
    const double bcy = b[2] * c[0] - b[0] * c[2];
    const double bcz = b[0] * c[1] - b[1] * c[0];
    const double det = (a[0] * bcx + a[1] * bcy) + a[2] * bcz;
    const double ab = (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2];
    const double bc = (b[0] * c[0] + b[1] * c[1]) + b[2] * c[2];
    const double ca = (c[0] * a[0] + c[1] * a[1]) + c[2] * a[2];
    const double den = ((1.0 + ab) + bc) + ca;
    return 2.0 * atan2(fabs(det), den);
}

__device__ __forceinline__ bool crit(const int32_t* __restrict__ tv, const double* __restrict__ pos,
                                     const double* __restrict__ zeta, double eps1, double eps2)
{
    const double z1 = zeta[tv[0]], z2 = zeta[tv[1]], z3 = zeta[tv[2]];
    const double A = tri_area(pos, tv);
    const double circ = A * (((z1 + z2) + z3) / 3.0);
    double zmax = z1, zmin = z1;
    if (z2 > zmax) zmax = z2;
    if (z3 > zmax) zmax = z3;
    if (z2 < zmin) zmin = z2;
    if (z3 < zmin) zmin = z3;
    return fabs(circ) >= eps1 || zmax - zmin >= eps2;
}

// Splits: every leaf below the level limit that meets a criterion.
__global__ void k_amr_split(int64_t nt, const uint8_t* __restrict__ state, const int8_t* __restrict__ level,
                            int levels, const int32_t* __restrict__ tv, const double* __restrict__ pos,
                            const double* __restrict__ zeta, double eps1, double eps2, uint8_t* __restrict__ split)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    split[t] = (state[t] == 1 && level[t] < levels && crit(tv + 3 * t, pos, zeta, eps1, eps2)) ? 1 : 0;
}

// Merges: a split triangle whose four children are leaves, none splitting, and whose own
// corners meet neither criterion.
__global__ void k_amr_merge(int64_t nt, const uint8_t* __restrict__ state, const int32_t* __restrict__ child,
                            const uint8_t* __restrict__ split, const int32_t* __restrict__ tv,
                            const double* __restrict__ pos, const double* __restrict__ zeta, double eps1,
                            double eps2, uint8_t* __restrict__ merge)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    bool m = false;
    if (state[t] == 2) {
        const int32_t c0 = child[t];
        bool ok = true;
        for (int c = 0; c < 4; c++) ok = ok && state[c0 + c] == 1 && !split[c0 + c];
        m = ok && !crit(tv + 3 * t, pos, zeta, eps1, eps2);
    }
    merge[t] = m ? 1 : 0;
}

// Applies merges and splits (disjoint sets of triangles: merges act on split triangles,
// splits on leaves), and places the new midpoint vertices.  Two triangles that share an edge
// write the same values to its midpoint (both read the same, unchanged, edge ends).
__global__ void k_amr_apply(int64_t nt, uint8_t* __restrict__ state, const int32_t* __restrict__ child,
                            const int32_t* __restrict__ tv, const int32_t* __restrict__ vparent,
                            const uint8_t* __restrict__ split, const uint8_t* __restrict__ merge,
                            const uint8_t* __restrict__ alive0, double* __restrict__ pos, double* __restrict__ zeta,
                            unsigned long long* __restrict__ cnt)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    if (merge[t]) {
        state[t] = 1;
        for (int c = 0; c < 4; c++) state[child[t] + c] = 0;
        atomicAdd(cnt + 1, 1ull);
    }
    if (!split[t]) return;
    state[t] = 2;
    const int32_t c0 = child[t];
    for (int c = 0; c < 4; c++) state[c0 + c] = 1;
    for (int a = 0; a < 3; a++) {
        const int32_t v = tv[3 * (int64_t)(c0 + 3) + a];  // the centre child's corners: m12, m23, m31
        if (alive0[v]) continue;
        const int32_t pa = vparent[2 * (int64_t)v], pb = vparent[2 * (int64_t)v + 1];
        const double sx = pos[3 * (int64_t)pa] + pos[3 * (int64_t)pb];
        const double sy = pos[3 * (int64_t)pa + 1] + pos[3 * (int64_t)pb + 1];
        const double sz = pos[3 * (int64_t)pa + 2] + pos[3 * (int64_t)pb + 2];
        const double r = sqrt((sx * sx + sy * sy) + sz * sz);
        pos[3 * (int64_t)v] = sx / r;
        pos[3 * (int64_t)v + 1] = sy / r;
        pos[3 * (int64_t)v + 2] = sz / r;
        zeta[v] = (zeta[pa] + zeta[pb]) * 0.5;
    }
    atomicAdd(cnt, 1ull);
}

// Alive vertices: the corners of leaf triangles (alive cleared beforehand).
__global__ void k_amr_alive(int64_t nt, const uint8_t* __restrict__ state, const int32_t* __restrict__ tv,
                            uint8_t* __restrict__ alive, unsigned long long* __restrict__ cnt)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt || state[t] != 1) return;
    for (int a = 0; a < 3; a++) alive[tv[3 * t + a]] = 1;
    atomicAdd(cnt + 3, 1ull);
}

// Vertices that are no particles hold zeros; the alive flags as int32 for the scan.
__global__ void k_amr_clear(int64_t nv, const uint8_t* __restrict__ alive, double* __restrict__ pos,
                            double* __restrict__ zeta, double* __restrict__ area, int32_t* __restrict__ flags)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    flags[v] = alive[v];
    area[v] = 0.0;
    if (alive[v]) return;
    pos[3 * v] = pos[3 * v + 1] = pos[3 * v + 2] = 0.0;
    zeta[v] = 0.0;
}

// Particle weights: A / 3 of every leaf triangle added to its corners.
__global__ void k_amr_area(int64_t nt, const uint8_t* __restrict__ state, const int32_t* __restrict__ tv,
                           const double* __restrict__ pos, double* __restrict__ area)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt || state[t] != 1) return;
    const double w = tri_area(pos, tv + 3 * t) / 3.0;
    for (int a = 0; a < 3; a++) atomicAdd(area + tv[3 * t + a], w);
}

__global__ void k_amr_gather(int64_t nv, const uint8_t* __restrict__ alive, const int64_t* __restrict__ scan,
                             const double* __restrict__ pos, const double* __restrict__ zeta,
                             const double* __restrict__ area, double* __restrict__ opos, double* __restrict__ ozeta,
                             double* __restrict__ oarea, int64_t* __restrict__ oids)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv || !alive[v]) return;
    const int64_t i = scan[v];
    if (opos) {
        opos[3 * i] = pos[3 * v];
        opos[3 * i + 1] = pos[3 * v + 1];
        opos[3 * i + 2] = pos[3 * v + 2];
    }
    if (ozeta) ozeta[i] = zeta[v];
    if (oarea) oarea[i] = area[v];
    if (oids) oids[i] = v;
}

__global__ void k_amr_scatter(int64_t nv, const uint8_t* __restrict__ alive, const int64_t* __restrict__ scan,
                              const double* __restrict__ ipos, const double* __restrict__ izeta,
                              double* __restrict__ pos, double* __restrict__ zeta)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv || !alive[v]) return;
    const int64_t i = scan[v];
    pos[3 * v] = ipos[3 * i];
    pos[3 * v + 1] = ipos[3 * i + 1];
    pos[3 * v + 2] = ipos[3 * i + 2];
    zeta[v] = izeta[i];
}

// Liveness, cleared state, compaction offsets and weights after a change of the mesh or of
// the positions; nalive read back (synchronises s).
int refresh(sts_ctx* c, AmrState* m, cudaStream_t s)
{
    const int T = 256;
    STS_CUDA(cudaMemsetAsync(m->valive.p, 0, m->nv, s));
    STS_CUDA(cudaMemsetAsync(m->cnt.p + 3, 0, sizeof(int64_t), s));
    (k_amr_alive<<<blocks(m->nt, T), T, 0, s>>>(m->nt, m->tstate.p, m->tv.p, m->valive.p,
                                                (unsigned long long*)m->cnt.p), note_launch());
    (k_amr_clear<<<blocks(m->nv, T), T, 0, s>>>(m->nv, m->valive.p, m->pos.p, m->zeta.p, m->area.p, m->flags.p),
     note_launch());
    (k_amr_area<<<blocks(m->nt, T), T, 0, s>>>(m->nt, m->tstate.p, m->tv.p, m->pos.p, m->area.p), note_launch());
    if (scan_state_reserve(c->scan_state, m->nv + 1, s)) return STS_ERR_CUDA;
    exclusive_scan_i32(m->flags.p, m->scan.p, m->nv, c->scan_state, s, c->d_status);
    STS_LAUNCH_CHECK();
    STS_CUDA(cudaMemcpyAsync(c->h_pinned, m->scan.p + m->nv, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    STS_CUDA(cudaStreamSynchronize(s));
    m->nalive = c->h_pinned[0];
    return STS_OK;
}

}  // namespace

void amr_free(AmrState* m)
{
    m->tv.release(); m->tparent.release(); m->tchild.release(); m->vparent.release(); m->tlevel.release();
    m->tstate.release(); m->valive.release(); m->valive0.release(); m->split.release(); m->merge.release();
    m->pos.release(); m->zeta.release(); m->area.release(); m->flags.release(); m->scan.release();
    m->cnt.release();
    delete m;
}

int amr_init(sts_ctx* c, const int32_t* faces, int64_t t0, int64_t n0, const double* pos0, const double* zeta0,
             int levels, cudaStream_t s)
{
    // the possible triangles and vertices, numbered on the host
    std::vector<int32_t> tv(3 * (size_t)t0), tparent((size_t)t0, -1), tchild, vparent(2 * (size_t)n0, -1);
    std::vector<int8_t> tlevel((size_t)t0, 0);
    for (int64_t q = 0; q < 3 * t0; q++) {
        if (faces[q] < 0 || faces[q] >= n0) {
            set_error("sts_amr_init: face %lld names vertex %d, outside [0, %lld)", (long long)(q / 3), faces[q],
                      (long long)n0);
            return STS_ERR_ARG;
        }
        tv[(size_t)q] = faces[q];
    }
    int64_t nv = n0, lb = 0, le = t0;
    for (int l = 1; l <= levels; l++) {
        std::unordered_map<uint64_t, int32_t> mid;
        mid.reserve((size_t)(3 * (le - lb)));
        tchild.resize((size_t)le, -1);
        for (int64_t t = lb; t < le; t++) {
            int32_t mm[3];
            for (int e = 0; e < 3; e++) {
                const int32_t a = tv[3 * (size_t)t + e], b = tv[3 * (size_t)t + (e + 1) % 3];
                const uint64_t key = ((uint64_t)(uint32_t)std::min(a, b) << 32) | (uint32_t)std::max(a, b);
                auto it = mid.find(key);
                if (it == mid.end()) {
                    it = mid.emplace(key, (int32_t)nv).first;
                    vparent.push_back(a);
                    vparent.push_back(b);
                    nv++;
                }
                mm[e] = it->second;
            }
            const int32_t v1 = tv[3 * (size_t)t], v2 = tv[3 * (size_t)t + 1], v3 = tv[3 * (size_t)t + 2];
            const int32_t ch[4][3] = {{v1, mm[0], mm[2]}, {mm[0], v2, mm[1]}, {mm[2], mm[1], v3}, {mm[0], mm[1], mm[2]}};
            tchild[(size_t)t] = (int32_t)(tv.size() / 3);
            for (int k = 0; k < 4; k++) {
                for (int a = 0; a < 3; a++) tv.push_back(ch[k][a]);
                tparent.push_back((int32_t)t);
                tlevel.push_back((int8_t)l);
            }
        }
        lb = le;
        le = (int64_t)(tv.size() / 3);
    }
    tchild.resize((size_t)le, -1);
    if (nv > ((int64_t)1 << 31) - 2 || le > ((int64_t)1 << 31) - 2) {
        set_error("sts_amr_init: %lld vertices or %lld triangles exceed int32 ids", (long long)nv, (long long)le);
        return STS_ERR_ARG;
    }
    if (!c->amr) c->amr = new AmrState();
    AmrState* m = c->amr;
    m->n0 = n0;
    m->nv = nv;
    m->t0 = t0;
    m->nt = le;
    m->levels = levels;
    const int64_t nt = le;
    STS_CUDA(m->tv.reserve(3 * nt));
    STS_CUDA(m->tparent.reserve(nt));
    STS_CUDA(m->tchild.reserve(nt));
    STS_CUDA(m->tlevel.reserve(nt));
    STS_CUDA(m->vparent.reserve(2 * nv));
    STS_CUDA(m->tstate.reserve(nt));
    STS_CUDA(m->split.reserve(nt));
    STS_CUDA(m->merge.reserve(nt));
    STS_CUDA(m->valive.reserve(nv));
    STS_CUDA(m->valive0.reserve(nv));
    STS_CUDA(m->pos.reserve(3 * nv));
    STS_CUDA(m->zeta.reserve(nv));
    STS_CUDA(m->area.reserve(nv));
    STS_CUDA(m->flags.reserve(nv + 1));
    STS_CUDA(m->scan.reserve(nv + 1));
    STS_CUDA(m->cnt.reserve(8));
    STS_CUDA(c->scan_tmp.reserve(scan_scratch(nv + 1) + 8));
    STS_CUDA(cudaMemcpyAsync(m->tv.p, tv.data(), 3 * nt * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    STS_CUDA(cudaMemcpyAsync(m->tparent.p, tparent.data(), nt * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    STS_CUDA(cudaMemcpyAsync(m->tchild.p, tchild.data(), nt * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    STS_CUDA(cudaMemcpyAsync(m->tlevel.p, tlevel.data(), nt * sizeof(int8_t), cudaMemcpyHostToDevice, s));
    STS_CUDA(cudaMemcpyAsync(m->vparent.p, vparent.data(), 2 * nv * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    STS_CUDA(cudaMemsetAsync(m->tstate.p, 0, nt, s));
    STS_CUDA(cudaMemsetAsync(m->tstate.p, 1, t0, s));
    STS_CUDA(cudaMemsetAsync(m->pos.p, 0, 3 * nv * sizeof(double), s));
    STS_CUDA(cudaMemsetAsync(m->zeta.p, 0, nv * sizeof(double), s));
    STS_CUDA(cudaMemcpyAsync(m->pos.p, pos0, 3 * n0 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    STS_CUDA(cudaMemcpyAsync(m->zeta.p, zeta0, n0 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    // the host tables must stay alive until the copies are done
    STS_CUDA(cudaStreamSynchronize(s));
    return refresh(c, m, s);
}

int amr_step(sts_ctx* c, double eps1, double eps2, int64_t* counts, cudaStream_t s)
{
    AmrState* m = c->amr;
    const int T = 256;
    STS_CUDA(cudaMemsetAsync(m->cnt.p, 0, 4 * sizeof(int64_t), s));
    STS_CUDA(cudaMemcpyAsync(m->valive0.p, m->valive.p, m->nv, cudaMemcpyDeviceToDevice, s));
    const unsigned g = blocks(m->nt, T);
    (k_amr_split<<<g, T, 0, s>>>(m->nt, m->tstate.p, m->tlevel.p, m->levels, m->tv.p, m->pos.p, m->zeta.p, eps1,
                                 eps2, m->split.p), note_launch());
    (k_amr_merge<<<g, T, 0, s>>>(m->nt, m->tstate.p, m->tchild.p, m->split.p, m->tv.p, m->pos.p, m->zeta.p, eps1,
                                 eps2, m->merge.p), note_launch());
    (k_amr_apply<<<g, T, 0, s>>>(m->nt, m->tstate.p, m->tchild.p, m->tv.p, m->vparent.p, m->split.p, m->merge.p,
                                 m->valive0.p, m->pos.p, m->zeta.p, (unsigned long long*)m->cnt.p), note_launch());
    STS_LAUNCH_CHECK();
    int rc = refresh(c, m, s);
    if (rc) return rc;
    if (counts) {
        STS_CUDA(cudaMemcpyAsync(c->h_pinned, m->cnt.p, 4 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        STS_CUDA(cudaStreamSynchronize(s));
        counts[0] = c->h_pinned[0];
        counts[1] = c->h_pinned[1];
        counts[2] = m->nalive;
        counts[3] = c->h_pinned[3];
    }
    return STS_OK;
}

int amr_gather(sts_ctx* c, double* pos, double* zeta, double* area, int64_t* ids, cudaStream_t s)
{
    AmrState* m = c->amr;
    (k_amr_gather<<<blocks(m->nv, 256), 256, 0, s>>>(m->nv, m->valive.p, m->scan.p, m->pos.p, m->zeta.p, m->area.p,
                                                      pos, zeta, area, ids), note_launch());
    STS_LAUNCH_CHECK();
    return STS_OK;
}

int amr_scatter(sts_ctx* c, const double* pos, const double* zeta, cudaStream_t s)
{
    AmrState* m = c->amr;
    (k_amr_scatter<<<blocks(m->nv, 256), 256, 0, s>>>(m->nv, m->valive.p, m->scan.p, pos, zeta, m->pos.p, m->zeta.p),
     note_launch());
    STS_LAUNCH_CHECK();
    // the weights follow the moved particles
    return refresh(c, m, s);
}

int amr_info(sts_ctx* c, int64_t* info)
{
    AmrState* m = c->amr;
    info[0] = m->n0;
    info[1] = m->nv;
    info[2] = m->t0;
    info[3] = m->nt;
    info[4] = m->nalive;
    return STS_OK;
}

int amr_export(sts_ctx* c, int32_t* tv, int32_t* tparent, int32_t* tchild, int8_t* tlevel, int32_t* vparent,
               uint8_t* tstate, uint8_t* valive, double* pos, double* zeta, double* area, cudaStream_t s)
{
    AmrState* m = c->amr;
    const int64_t nt = m->nt, nv = m->nv;
    auto cp = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
        return dst ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s) : cudaSuccess;
    };
    STS_CUDA(cp(tv, m->tv.p, 3 * nt * sizeof(int32_t)));
    STS_CUDA(cp(tparent, m->tparent.p, nt * sizeof(int32_t)));
    STS_CUDA(cp(tchild, m->tchild.p, nt * sizeof(int32_t)));
    STS_CUDA(cp(tlevel, m->tlevel.p, nt * sizeof(int8_t)));
    STS_CUDA(cp(vparent, m->vparent.p, 2 * nv * sizeof(int32_t)));
    STS_CUDA(cp(tstate, m->tstate.p, nt));
    STS_CUDA(cp(valive, m->valive.p, nv));
    STS_CUDA(cp(pos, m->pos.p, 3 * nv * sizeof(double)));
    STS_CUDA(cp(zeta, m->zeta.p, nv * sizeof(double)));
    STS_CUDA(cp(area, m->area.p, nv * sizeof(double)));
    STS_CUDA(cudaStreamSynchronize(s));
    return STS_OK;
}

}  // namespace sts
