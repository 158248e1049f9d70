// The extern "C" entry points of libsts (declared in include/sts.h): argument checks, the
// context and its scratch, phase timing, and the order in which the device stages run.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <vector>

#include "sts_internal.cuh"

namespace sts {

static thread_local char g_err[512];
static std::atomic<long long> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void set_error(const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void phase_begin(sts_ctx* c, int ph, cudaStream_t s)
{
    if (!c->timing || ph < 0) return;  // ph < 0: inside a phase the caller times
    if (c->capturing) {  // an event record node of the graph (external: it records at replay)
        cudaEventRecordWithFlags(c->ev[ph][0], s, cudaEventRecordExternal);
        return;
    }
    if (c->phase_open[ph]) {
        float ms = 0.f;
        if (cudaEventSynchronize(c->ev[ph][1]) == cudaSuccess &&
            cudaEventElapsedTime(&ms, c->ev[ph][0], c->ev[ph][1]) == cudaSuccess) {
            c->phase_ms[ph] += ms;
            c->phase_count[ph] += 1;
        }
        c->phase_open[ph] = false;
    }
    cudaEventRecord(c->ev[ph][0], s);
}

void phase_end(sts_ctx* c, int ph, cudaStream_t s)
{
    if (!c->timing || ph < 0) return;
    if (c->capturing) {
        cudaEventRecordWithFlags(c->ev[ph][1], s, cudaEventRecordExternal);
        c->phase_in_graph[ph] = true;
    } else {
        cudaEventRecord(c->ev[ph][1], s);
        c->phase_open[ph] = true;
    }
}

// After a replay has completed: add the phases recorded inside the graph.
void phase_harvest_graph(sts_ctx* c)
{
    if (!c->timing) return;
    for (int ph = 0; ph < kNumPhases; ph++) {
        if (!c->phase_in_graph[ph]) continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->ev[ph][0], c->ev[ph][1]) == cudaSuccess) {
            c->phase_ms[ph] += ms;
            c->phase_count[ph] += 1;
        } else {
            (void)cudaGetLastError();  // timing is best effort; do not leave the error pending
        }
    }
}

}  // namespace sts

using namespace sts;

sts_ctx::~sts_ctx()
{
    pos.release(); nodeof.release(); digit.release(); perm.release(); perm_tmp.release();
    skey.release(); skey_tmp.release(); scan_tmp.release(); hist.release(); flags.release();
    offs.release(); nd_level.release(); nd_parent.release(); nd_first_child.release();
    nd_nchild.release(); nd_start.release(); nd_count.release(); nd_leaf.release();
    nd_key.release(); nd_geom.release(); nd_norm.release(); nd_mid.release(); nd_norm32.release(); nd_c32.release(); posf.release(); nd_cc.release(); nd_child.release();
    counters.release(); small.release(); dc.release(); inst_off.release(); root_cnt.release();
    face_node.release(); leaves.release(); slot_leaf.release(); cluster_slot.release();
    cluster_node.release(); up_toff.release(); up_tasks.release(); up_part.release(); up_frame.release();
    up_frame32.release(); src_hl.release(); lw_terms.release(); rk_zf.release();
    prx64.release(); prx32.release(); src64.release(); src32.release(); far_off.release(); near_coff.release(); corr.release();
    near_off.release(); far_idx.release(); near_idx.release(); far_ent.release();
    near_ent.release(); list_cnt.release(); wover.release(); tasks.release(); dsrc64.release(); dsrc32.release();
    dpart.release(); rk_x0.release(); rk_z0.release(); rk_xs.release(); rk_zs.release();
    rk_k.release(); rk_ksum.release(); d_stats.release(); d_work.release(); prx_rd.release(); scan_state.release(); scan_state_side.release(); bld_tot.release();
    dual_ft.release(); dual_fs.release(); dual_gt.release(); dual_gs.release(); dual_tt.release();
    dual_ts.release(); dual_tk.release(); dual_t.release(); dual_s.release(); dual_key.release();
    dual_ktmp.release(); dual_perm.release(); dual_ptmp.release(); dual_chunk.release(); dual_cnt.release();
    dual_bkt.release(); dual_bcnt.release(); dual_boff.release();
    dual_scan.release(); cfar_off.release(); cnear_off.release(); cnear_coff.release(); cfar_ent.release();
    cnear_ent.release(); ctasks.release(); cvel.release(); ccorr.release(); cdown.release(); cdown32.release();
    chas.release();
    cacc.release(); leaf_anc.release();
    if (amr) amr_free(amr);
    for (RefTable* t : refs)
        if (t) {
            t->d_beta.release();
            t->d_vinv.release();
            t->d_vinvT.release();
            t->d_tcB.release();
            t->d_tcF.release();
            t->d_tcE.release();
            t->d_tcBr.release();
            t->d_tcFr.release();
            delete t;
        }
    for (int p = 0; p < kNumPhases; p++)
        for (int q = 0; q < 2; q++)
            if (ev[p][q]) cudaEventDestroy(ev[p][q]);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (ev_tree) cudaEventDestroy(ev_tree);
    if (side) cudaStreamDestroy(side);
    if (rk_exec) cudaGraphExecDestroy(rk_exec);
    if (ev_exec) cudaGraphExecDestroy(ev_exec);
    if (d_status) cudaFree(d_status);
    if (h_pinned) cudaFreeHost(h_pinned);
}

namespace {

cudaStream_t S(void* s) { return (cudaStream_t)s; }

int check_ctx(sts_ctx* c, const char* fn)
{
    g_err[0] = 0;
    if (!c) {
        set_error("%s: NULL context", fn);
        return STS_ERR_ARG;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != c->device) {
        if (cudaSetDevice(c->device) != cudaSuccess) {
            set_error("%s: cannot select the context's device %d", fn, c->device);
            return STS_ERR_CUDA;
        }
    }
    return STS_OK;
}

int check_params(const sts_params* p, const char* fn)
{
    if (!p) {
        set_error("%s: NULL params", fn);
        return STS_ERR_ARG;
    }
    if (!(p->theta > 0.0 && p->theta < 1.0)) {
        set_error("%s: theta must be in (0, 1), got %g", fn, p->theta);
        return STS_ERR_ARG;
    }
    if (p->degree < 1 || p->degree > kMaxDegree) {
        set_error("%s: degree must be in [1, %d], got %d", fn, kMaxDegree, p->degree);
        return STS_ERR_ARG;
    }
    if (p->leaf_size < 1) {
        set_error("%s: leaf_size must be >= 1, got %d", fn, p->leaf_size);
        return STS_ERR_ARG;
    }
    if (p->max_level < 0 || p->max_level > kMaxLevel) {
        set_error("%s: max_level must be in [0, %d], got %d", fn, kMaxLevel, p->max_level);
        return STS_ERR_ARG;
    }
    if (p->precision != STS_FP64 && p->precision != STS_MIXED) {
        set_error("%s: precision must be STS_FP64 or STS_MIXED, got %d", fn, p->precision);
        return STS_ERR_ARG;
    }
    if (!(p->near_fp64_tau >= 0.0) || !isfinite(p->near_fp64_tau)) {
        set_error("%s: near_fp64_tau must be finite and >= 0", fn);
        return STS_ERR_ARG;
    }
    return STS_OK;
}

int check_n(int64_t n, const char* fn)
{
    if (n < 0 || n > ((int64_t)1 << 31) - 2) {
        set_error("%s: n must be in [0, 2^31 - 2], got %lld", fn, (long long)n);
        return STS_ERR_ARG;
    }
    return STS_OK;
}

int velocity_dual_impl(sts_ctx* c, const double* zeta, const double* area, const sts_params* p, double* vel,
                       cudaStream_t s);

// The sorted sources and the proxy weights (upward pass) on s, and, when the tree or theta
// changed, the interaction lists (target-leaf lists or the dual traversal's pairs) on the
// side stream: both read only the tree (the cluster table and the upward tasks are made with
// it), write disjoint buffers and device counters, and meet again before the evaluation.  The
// sources and weights are issued first, so that an eager list build, which reads its counts
// on the host, overlaps them too.  The side stream is joined back to s on every return.
int sources_and_lists(sts_ctx* c, const double* zeta, const double* area, const sts_params* p,
                      int up_precision, bool dual, cudaStream_t s)
{
    const bool lists = dual ? (!c->have_dual || c->dual_theta != p->theta)
                            : (!c->have_lists || c->list_theta != p->theta);
    if (lists) {
        if (c->tree_event) {
            // a tree built just before: the lists need only the tree, so they start when it is
            // complete, beside the particle sort that follows it on s
            STS_CUDA(cudaStreamWaitEvent(c->side, c->ev_tree, 0));
        } else {
            STS_CUDA(cudaEventRecord(c->ev_fork, s));
            STS_CUDA(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
        }
    }
    c->tree_event = false;
    int rc;
    phase_begin(c, kPhPrep, s);
    rc = prepare_sources(c, zeta, area, s);
    phase_end(c, kPhPrep, s);
    if (rc == STS_OK) {
        phase_begin(c, kPhUpward, s);
        rc = upward_pass(c, p->degree, up_precision, s);
        phase_end(c, kPhUpward, s);
    }
    if (lists) {
        int rl = STS_OK;
        if (rc == STS_OK) {
            phase_begin(c, kPhLists, c->side);
            rl = dual ? build_dual(c, p->theta, c->side) : build_lists(c, p->theta, c->side);
            phase_end(c, kPhLists, c->side);
        }
        const cudaError_t e1 = cudaEventRecord(c->ev_join, c->side);
        const cudaError_t e2 = cudaStreamWaitEvent(s, c->ev_join, 0);
        if (rc == STS_OK) rc = rl;
        if (rc == STS_OK && (e1 != cudaSuccess || e2 != cudaSuccess)) {
            set_error("joining the lists' stream: %s", cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
            rc = STS_ERR_CUDA;
        }
    }
    return rc;
}

int velocity_impl(sts_ctx* c, const double* zeta, const double* area, const sts_params* p,
                  double* vel, cudaStream_t s)
{
    if (c->use_dual) return velocity_dual_impl(c, zeta, area, p, vel, s);
    const int64_t n = c->n;
    if (n == 0) return STS_OK;
    if (n == 1) {
        STS_CUDA(cudaMemsetAsync(vel, 0, 3 * sizeof(double), s));
        return STS_OK;
    }
    int rc;
    if ((rc = sources_and_lists(c, zeta, area, p, p->precision, false, s))) return rc;
    if ((rc = evaluate(c, p->degree, p->precision, p->near_fp64_tau, vel, s))) return rc;
    c->list_degree = p->degree;
    return STS_OK;
}

// The stream function on the current tree: the FP64 sources, lists, FP64 proxy weights (the
// upward pass does not depend on the kernel) and the potential evaluation.
int potential_impl(sts_ctx* c, const double* zeta, const double* area, const sts_params* p, double* psi,
                   cudaStream_t s)
{
    const int64_t n = c->n;
    if (n == 0) return STS_OK;
    if (n == 1) {
        STS_CUDA(cudaMemsetAsync(psi, 0, sizeof(double), s));
        return STS_OK;
    }
    int rc;
    if ((rc = sources_and_lists(c, zeta, area, p, p->precision, false, s))) return rc;
    if ((rc = evaluate_potential(c, p->degree, p->precision, p->near_fp64_tau, psi, s))) return rc;
    c->list_degree = p->degree;
    return STS_OK;
}

// Dual-traversal velocity on the current tree: sources, the four pair lists (rebuilt when theta
// or the tree changed, or after the target-leaf lists replaced them), proxy weights and the
// evaluation with the downward interpolation.
int velocity_dual_impl(sts_ctx* c, const double* zeta, const double* area, const sts_params* p, double* vel,
                       cudaStream_t s)
{
    const int64_t n = c->n;
    if (n == 0) return STS_OK;
    if (n == 1) {
        STS_CUDA(cudaMemsetAsync(vel, 0, 3 * sizeof(double), s));
        return STS_OK;
    }
    int rc;
    if ((rc = sources_and_lists(c, zeta, area, p, p->precision, true, s))) return rc;
    if ((rc = evaluate_dual(c, p->degree, p->precision, p->near_fp64_tau, vel, s))) return rc;
    c->list_degree = p->degree;
    return STS_OK;
}

int build_impl(sts_ctx* c, const double* pos, int64_t n, const int64_t* inst_off, int ninst, const sts_params* p,
               cudaStream_t s)
{
    phase_begin(c, kPhBuild, s);
    int rc = tree_build(c, pos, n, inst_off, ninst, p->leaf_size, p->max_level, s);
    phase_end(c, kPhBuild, s);
    return rc;
}

int upload_offsets(sts_ctx* c, const int64_t* offsets, int32_t ninst, const int64_t** d_off, int64_t* n,
                   const char* fn, cudaStream_t s)
{
    if (!offsets || ninst < 1 || ninst > (1 << 24)) {
        set_error("%s: offsets must be a host array of ninst + 1 values, 1 <= ninst <= 2^24", fn);
        return STS_ERR_ARG;
    }
    if (offsets[0] != 0) {
        set_error("%s: offsets[0] must be 0", fn);
        return STS_ERR_ARG;
    }
    for (int32_t b = 0; b < ninst; b++)
        if (offsets[b + 1] < offsets[b]) {
            set_error("%s: offsets must be non-decreasing (offsets[%d] > offsets[%d])", fn, b, b + 1);
            return STS_ERR_ARG;
        }
    int rc = check_n(offsets[ninst], fn);
    if (rc) return rc;
    STS_CUDA(c->inst_off.reserve(ninst + 1));
    STS_CUDA(cudaMemcpyAsync(c->inst_off.p, offsets, (ninst + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    STS_CUDA(cudaStreamSynchronize(s));  // the host array may be pageable and reused by the caller
    *d_off = c->inst_off.p;
    *n = offsets[ninst];
    return STS_OK;
}

// One RK4 step of the whole forest (one instance when inst_off is NULL).
int rk4_impl(sts_ctx* ctx, double* pos, double* zeta, const double* area, int64_t n, const int64_t* inst_off,
             int ninst, double dt, double Omega, const sts_params* p, cudaStream_t s,
             const sts_forcing* forcing = nullptr, double t = 0.0)
{
    int rc;
    if (!isfinite(dt) || !isfinite(Omega)) {
        set_error("bve_rk4_step: dt and Omega must be finite");
        return STS_ERR_ARG;
    }
    if (n > 0 && (!pos || !zeta || !area)) {
        set_error("bve_rk4_step: NULL array");
        return STS_ERR_ARG;
    }
    if (n == 0) return STS_OK;
    sts_ctx* c = ctx;
    STS_CUDA(c->rk_x0.reserve(3 * n));
    STS_CUDA(c->rk_z0.reserve(n));
    STS_CUDA(c->rk_xs.reserve(3 * n));
    STS_CUDA(c->rk_zs.reserve(n));
    STS_CUDA(c->rk_k.reserve(3 * n));
    STS_CUDA(c->rk_ksum.reserve(3 * n));
    STS_CUDA(cudaMemcpyAsync(c->rk_x0.p, pos, 3 * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    STS_CUDA(cudaMemcpyAsync(c->rk_z0.p, zeta, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    const double cst[3] = {0.5, 0.5, 1.0};
    const double bst[3] = {1.0, 2.0, 2.0};
    const double tst[4] = {0.0, 0.5, 0.5, 1.0};  // stage times t + tst dt (forced system)
    if (forcing) STS_CUDA(c->rk_zf.reserve(n));
    const double* xs = c->rk_x0.p;
    const double* zs = c->rk_z0.p;
    for (int st = 0; st < 4; st++) {
        if ((rc = build_impl(c, xs, n, inst_off, ninst, p, s))) return rc;
        const double* src = zs;
        if (forcing) {
            forced_source(xs, zs, n, forcing, t + tst[st] * dt, c->rk_zf.p, s);
            src = c->rk_zf.p;
        }
        if ((rc = velocity_impl(c, src, area, p, c->rk_k.p, s))) return rc;
        if (st < 3) {
            rk4_stage(c->rk_x0.p, c->rk_z0.p, c->rk_k.p, cst[st] * dt, Omega, c->rk_xs.p, c->rk_zs.p,
                      c->rk_ksum.p, bst[st], st == 0, n, s);
            xs = c->rk_xs.p;
            zs = c->rk_zs.p;
        } else {
            rk4_final(pos, zeta, c->rk_x0.p, c->rk_z0.p, c->rk_ksum.p, c->rk_k.p, dt, Omega, n, s);
        }
        STS_LAUNCH_CHECK();
    }
    return STS_OK;
}

// Host copies of the device counters after a recorded step ran (they are not read while
// recording).
int refresh_counts(sts_ctx* c, cudaStream_t s)
{
    if (!c->have_tree || c->nnodes >= 0) return STS_OK;
    STS_CUDA(cudaMemcpyAsync(c->h_pinned, c->dc.p, kDcSize * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    STS_CUDA(cudaStreamSynchronize(s));
    const int64_t* h = c->h_pinned;
    c->nnodes = h[kDcNodes];
    c->nleaves = h[kDcLeaves];
    c->nclusters = h[kDcClusters];
    c->n_up_tasks = h[kDcUpTasks];
    c->nfar = h[kDcFar];
    c->nnear = h[kDcNear];
    c->nnear_chunks = h[kDcChunks];
    c->ntasks = h[kDcTasks];
    c->level_begin.assign(1, 0);
    c->deepest = 0;
    for (int l = 1; l <= kMaxLevel + 2 && h[kDcLevel + l] > h[kDcLevel + l - 1]; l++) {
        c->level_begin.push_back(h[kDcLevel + l]);
        c->deepest = l - 1;
    }
    return STS_OK;
}

// Buffers for recording a step: the plan's sizes (maxima over the eager step) with slack.
int reserve_for_capture(sts_ctx* c, const sts_params* p, int ninst, cudaStream_t s)
{
    const int64_t n = c->n;
    auto grow = [](int64_t v, int64_t add) { return v + v / 4 + add; };
    const int64_t nodes = grow(c->plan.nodes, 64 + 20 * (int64_t)ninst);
    c->nodes_rec = nodes;  // the node count a recorded step provides for
    const int M = nbasis(p->degree);
    const int64_t upt = grow(c->plan.up_tasks, 64);
    int rc = reserve_tree_nodes(c, nodes, s);
    if (rc) return rc;
    const int64_t big = std::max(n, nodes) + 2;
    STS_CUDA(c->cluster_slot.reserve(nodes + 1));
    STS_CUDA(c->cluster_node.reserve(nodes + 1));
    STS_CUDA(c->flags.reserve(big));
    STS_CUDA(c->offs.reserve(big));
    STS_CUDA(c->up_toff.reserve(nodes + 2));
    STS_CUDA(c->list_cnt.reserve(std::max(3 * n + 3, nodes + 1)));
    STS_CUDA(c->up_frame.reserve(12 * nodes + 12));
    STS_CUDA(c->up_frame32.reserve(18 * nodes + 18));
    STS_CUDA(c->src_hl.reserve(2 * n + 2));
    STS_CUDA(c->up_tasks.reserve(upt));
    c->up_tasks_rec = upt;  // the recorded moment tasks: grid of the upward pass, overflow bound
    STS_CUDA(c->prx64.reserve(nodes * M + 1));
    STS_CUDA(c->prx32.reserve(nodes * M + 1));
    STS_CUDA(c->prx_rd.reserve(nodes * M + 1));
    STS_CUDA(c->up_part.reserve(upt * M + 1));
    STS_CUDA(c->far_idx.reserve(grow(c->plan.far, 1024)));
    STS_CUDA(c->far_ent.reserve(grow(c->plan.far, 1024)));
    STS_CUDA(c->near_idx.reserve(grow(c->plan.near, 1024)));
    STS_CUDA(c->near_ent.reserve(grow(c->plan.chunks, 1024)));
    STS_CUDA(c->tasks.reserve(grow(c->plan.tasks, 1024)));
    // the leaf bound of build_lists while recording, times the larger traversal capacity
    STS_CUDA(c->lw_terms.reserve(std::min<int64_t>(n, grow(c->plan.leaves, 64)) * 512 + 1));
    STS_CUDA(c->far_off.reserve(n + 1));
    STS_CUDA(c->near_off.reserve(n + 1));
    STS_CUDA(c->near_coff.reserve(n + 1));
    STS_CUDA(c->leaves.reserve(n + 1));
    STS_CUDA(c->wover.reserve(n + 1));
    STS_CUDA(c->corr.reserve(3 * n + 3));
    STS_CUDA(c->scan_tmp.reserve(2 * scan_scratch(big) + 64));
    // every scan a recorded step runs (capacities included) fits its stream's state
    if (scan_state_reserve(c->scan_state, big + 1, s) ||
        scan_state_reserve(c->scan_state_side, big + 1, s))
        return STS_ERR_CUDA;
    if (c->use_dual && (rc = reserve_dual_for_capture(c, p->degree, s))) return rc;
    return STS_OK;
}

// After a replay the lists of the recorded traversal are in place (host counts refreshed on
// demand).
void mark_replayed_lists(sts_ctx* c, double theta)
{
    c->have_lists = !c->use_dual;
    c->have_dual = c->use_dual;
    c->list_theta = c->dual_theta = theta;
    for (int k = 0; k < 4; k++) c->dual_n[k] = -1;
}

// One RK4 step through a recorded graph: the first call (or a call with other arguments)
// runs the step eagerly, which plans the capacities, then records the step; later calls
// replay it.  A replay that ran out of a recorded capacity or level count is undone from
// the saved start state and redone eagerly (and recorded again).
int rk4_graph(sts_ctx* c, double* pos, double* zeta, const double* area, int64_t n, const int64_t* inst_off,
              const int64_t* off_host, int ninst, double dt, double Omega, const sts_params* p, cudaStream_t s)
{
    std::vector<double> key = {(double)n, (double)ninst, dt, Omega, p->theta, (double)p->degree,
                               (double)p->leaf_size, (double)p->max_level, (double)p->precision, p->near_fp64_tau,
                               (double)c->use_dual};
    std::vector<int64_t> okey = {(int64_t)(uintptr_t)pos, (int64_t)(uintptr_t)zeta, (int64_t)(uintptr_t)area,
                                 (int64_t)(uintptr_t)s};
    if (off_host) okey.insert(okey.end(), off_host, off_host + ninst + 1);
    int rc;
    if (c->rk_exec && key == c->rk_key && okey == c->rk_off_key && c->rk_epoch == g_alloc_epoch.load()) {
        STS_CUDA(cudaGraphLaunch(c->rk_exec, s));
        g_launches.fetch_add(c->rk_kernels, std::memory_order_relaxed);
        STS_CUDA(cudaMemcpyAsync(c->h_pinned, c->dc.p + kDcOver, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        STS_CUDA(cudaMemcpyAsync(c->h_pinned + 1, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
        STS_CUDA(cudaStreamSynchronize(s));
        phase_harvest_graph(c);
        const int64_t over = c->h_pinned[0];
        const int st = ((int32_t*)(c->h_pinned + 1))[0];
        if (st & kStatusNonfinite) {
            STS_CUDA(cudaMemsetAsync(c->d_status, 0, sizeof(int), s));
            set_error("bve_rk4_step: non-finite position");
            return STS_ERR_NONFINITE;
        }
        if (st & kStatusTimeout) {
            STS_CUDA(cudaMemsetAsync(c->d_status, 0, sizeof(int), s));
            set_error("bve_rk4_step: a device-side wait for staged sources gave up");
            return STS_ERR_TIMEOUT;
        }
        c->have_tree = true;
        mark_replayed_lists(c, p->theta);
        c->nnodes = -1;  // host counts refreshed on demand
        if (over == 0) return STS_OK;
        // undo the step and redo it eagerly below
        STS_CUDA(cudaMemcpyAsync(pos, c->rk_x0.p, 3 * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        STS_CUDA(cudaMemcpyAsync(zeta, c->rk_z0.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        STS_CUDA(cudaGraphExecDestroy(c->rk_exec));
        c->rk_exec = nullptr;
    }
    c->plan = Plan();
    if ((rc = rk4_impl(c, pos, zeta, area, n, inst_off, ninst, dt, Omega, p, s))) return rc;
    if ((rc = reserve_for_capture(c, p, ninst, s))) return rc;
    STS_CUDA(cudaStreamSynchronize(s));
    c->have_tree = c->have_lists = false;  // buffers may have moved; the replay rebuilds them
    c->have_dual = false;
    if (c->rk_exec) {
        cudaGraphExecDestroy(c->rk_exec);
        c->rk_exec = nullptr;
    }
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        set_error("bve_rk4_step: cannot record on this stream (%s); use a non-default stream",
                  cudaGetErrorString(e));
        return STS_ERR_CUDA;
    }
    for (int ph = 0; ph < kNumPhases; ph++) c->phase_in_graph[ph] = false;
    c->capturing = true;
    const long long l0 = g_launches.load();
    e = cudaMemsetAsync(c->dc.p + kDcOver, 0, sizeof(int64_t), s);
    rc = e == cudaSuccess ? rk4_impl(c, pos, zeta, area, n, inst_off, ninst, dt, Omega, p, s) : STS_ERR_CUDA;
    c->capturing = false;
    c->rk_kernels = g_launches.load() - l0;  // recorded, not launched: counted per replay
    g_launches.fetch_sub(c->rk_kernels);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(s, &g);
    if (rc == STS_OK && e2 != cudaSuccess) {
        set_error("bve_rk4_step: recording failed: %s", cudaGetErrorString(e2));
        rc = STS_ERR_CUDA;
    }
    if (rc == STS_OK) {
        const cudaError_t e3 = cudaGraphInstantiate(&c->rk_exec, g, 0);
        if (e3 != cudaSuccess) {
            set_error("bve_rk4_step: graph instantiation failed: %s", cudaGetErrorString(e3));
            c->rk_exec = nullptr;
            rc = STS_ERR_CUDA;
        }
    }
    if (g) cudaGraphDestroy(g);
    if (rc == STS_OK) {
        c->rk_key = key;
        c->rk_off_key = okey;
        c->rk_epoch = g_alloc_epoch.load();
    }
    return rc;
}

// Tree build + velocity through a recorded graph (same scheme as rk4_graph): record on the
// first call or when the arguments change, replay afterwards, redo eagerly on overflow.
int eval_graph(sts_ctx* c, const double* pos, const double* zeta, const double* area, int64_t n,
               const int64_t* inst_off, const int64_t* off_host, int ninst, const sts_params* p, double* vel,
               cudaStream_t s)
{
    std::vector<double> key = {-1.0, (double)n, (double)ninst, p->theta, (double)p->degree, (double)p->leaf_size,
                               (double)p->max_level, (double)p->precision, p->near_fp64_tau, (double)c->use_dual};
    std::vector<int64_t> okey = {(int64_t)(uintptr_t)pos, (int64_t)(uintptr_t)zeta, (int64_t)(uintptr_t)area,
                                 (int64_t)(uintptr_t)vel, (int64_t)(uintptr_t)s};
    if (off_host) okey.insert(okey.end(), off_host, off_host + ninst + 1);
    int rc;
    if (c->ev_exec && key == c->ev_key && okey == c->ev_off_key && c->ev_epoch == g_alloc_epoch.load()) {
        STS_CUDA(cudaGraphLaunch(c->ev_exec, s));
        g_launches.fetch_add(c->ev_kernels, std::memory_order_relaxed);
        STS_CUDA(cudaMemcpyAsync(c->h_pinned, c->dc.p + kDcOver, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        STS_CUDA(cudaMemcpyAsync(c->h_pinned + 1, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
        STS_CUDA(cudaStreamSynchronize(s));
        phase_harvest_graph(c);
        const int64_t over = c->h_pinned[0];
        const int st = ((int32_t*)(c->h_pinned + 1))[0];
        if (st & kStatusNonfinite) {
            STS_CUDA(cudaMemsetAsync(c->d_status, 0, sizeof(int), s));
            set_error("sts_tree_velocity: non-finite position");
            return STS_ERR_NONFINITE;
        }
        if (st & kStatusTimeout) {
            STS_CUDA(cudaMemsetAsync(c->d_status, 0, sizeof(int), s));
            set_error("sts_tree_velocity: a device-side wait for staged sources gave up");
            return STS_ERR_TIMEOUT;
        }
        c->have_tree = true;
        mark_replayed_lists(c, p->theta);
        c->nnodes = -1;
        if (over == 0) return STS_OK;
        STS_CUDA(cudaGraphExecDestroy(c->ev_exec));
        c->ev_exec = nullptr;
    }
    c->plan = Plan();
    if ((rc = build_impl(c, pos, n, inst_off, ninst, p, s))) return rc;
    if ((rc = velocity_impl(c, zeta, area, p, vel, s))) return rc;
    if (n < 2) return STS_OK;
    if ((rc = reserve_for_capture(c, p, ninst, s))) return rc;
    STS_CUDA(cudaStreamSynchronize(s));
    // the eager result is in vel; the recording below is not run now
    std::vector<double> keep;
    if (c->ev_exec) {
        cudaGraphExecDestroy(c->ev_exec);
        c->ev_exec = nullptr;
    }
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        set_error("sts_tree_velocity: cannot record on this stream (%s); use a non-default stream",
                  cudaGetErrorString(e));
        c->have_tree = c->have_lists = false;
        c->have_dual = false;
        return STS_ERR_CUDA;
    }
    for (int ph = 0; ph < kNumPhases; ph++) c->phase_in_graph[ph] = false;
    c->capturing = true;
    const long long l0 = g_launches.load();
    e = cudaMemsetAsync(c->dc.p + kDcOver, 0, sizeof(int64_t), s);
    rc = e == cudaSuccess ? build_impl(c, pos, n, inst_off, ninst, p, s) : STS_ERR_CUDA;
    if (rc == STS_OK) rc = velocity_impl(c, zeta, area, p, vel, s);
    c->capturing = false;
    c->ev_kernels = g_launches.load() - l0;  // recorded, not launched: counted per replay
    g_launches.fetch_sub(c->ev_kernels);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(s, &g);
    if (rc == STS_OK && e2 != cudaSuccess) {
        set_error("sts_tree_velocity: recording failed: %s", cudaGetErrorString(e2));
        rc = STS_ERR_CUDA;
    }
    if (rc == STS_OK && cudaGraphInstantiate(&c->ev_exec, g, 0) != cudaSuccess) {
        set_error("sts_tree_velocity: graph instantiation failed");
        c->ev_exec = nullptr;
        rc = STS_ERR_CUDA;
    }
    if (g) cudaGraphDestroy(g);
    c->have_tree = c->have_lists = false;  // the recording reused the buffers; the next call replays
    c->have_dual = false;
    if (rc == STS_OK) {
        c->ev_key = key;
        c->ev_off_key = okey;
        c->ev_epoch = g_alloc_epoch.load();
    }
    return rc;
}

}  // namespace

namespace {
template <class D, class H>
int copy_out(H* host, const D* dev, int64_t n, cudaStream_t s)
{
    if (!host || n <= 0) return STS_OK;
    std::vector<D> tmp((size_t)n);
    STS_CUDA(cudaMemcpyAsync(tmp.data(), dev, n * sizeof(D), cudaMemcpyDeviceToHost, s));
    STS_CUDA(cudaStreamSynchronize(s));
    for (int64_t i = 0; i < n; i++) host[i] = (H)tmp[(size_t)i];
    return STS_OK;
}

// Sorted slots [slot_lo, slot_hi) of the targets of depth-first leaves [leaf_lo, leaf_hi)
// (leaves hold consecutive slots in depth-first order); synchronises `s`.
int leaf_range_slots(sts_ctx* c, int64_t leaf_lo, int64_t leaf_hi, int64_t* slot_lo, int64_t* slot_hi,
                     cudaStream_t s)
{
    *slot_lo = *slot_hi = 0;
    if (leaf_hi <= leaf_lo) {
        if (leaf_lo < c->nleaves) {
            int32_t node = 0, st = 0;
            int rc = copy_out(&node, c->leaves.p + leaf_lo, 1, s);
            if (rc || (rc = copy_out(&st, c->nd_start.p + node, 1, s))) return rc;
            *slot_lo = *slot_hi = st;
        } else {
            *slot_lo = *slot_hi = c->n;
        }
        return STS_OK;
    }
    int32_t a = 0, b = 0, sa = 0, sb = 0, cb = 0;
    int rc = copy_out(&a, c->leaves.p + leaf_lo, 1, s);
    if (rc || (rc = copy_out(&b, c->leaves.p + leaf_hi - 1, 1, s))) return rc;
    if ((rc = copy_out(&sa, c->nd_start.p + a, 1, s)) || (rc = copy_out(&sb, c->nd_start.p + b, 1, s)) ||
        (rc = copy_out(&cb, c->nd_count.p + b, 1, s)))
        return rc;
    *slot_lo = sa;
    *slot_hi = (int64_t)sb + cb;
    return STS_OK;
}

}  // namespace

extern "C" {

int sts_create(sts_ctx** out)
{
    g_err[0] = 0;
    if (!out) {
        set_error("sts_create: NULL out");
        return STS_ERR_ARG;
    }
    sts_ctx* c = new (std::nothrow) sts_ctx();
    if (!c) {
        set_error("sts_create: out of host memory");
        return STS_ERR_ARG;
    }
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&c->h_pinned, (kDcSize + 16) * sizeof(int64_t));
    if (e == cudaSuccess) e = c->dc.reserve(sts::kDcSize);
    if (e == cudaSuccess) e = cudaMemset(c->dc.p, 0, sts::kDcSize * sizeof(int64_t));
    // inspection counters and the dual traversal's counters: allocated once here, so that
    // inspecting a context between graph replays moves no buffer the recordings use
    if (e == cudaSuccess) e = c->d_stats.reserve(8);
    if (e == cudaSuccess) e = c->dual_cnt.reserve(128);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_tree, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        set_error("sts_create: %s", cudaGetErrorString(e));
        delete c;
        return STS_ERR_CUDA;
    }
    *out = c;
    return STS_OK;
}

void sts_destroy(sts_ctx* ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    delete ctx;
}

const char* sts_last_error(void) { return g_err; }

int sts_status(sts_ctx* ctx, void* stream)
{
    int rc = check_ctx(ctx, "sts_status");
    if (rc) return rc;
    STS_CUDA(cudaMemcpyAsync(ctx->h_pinned, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, S(stream)));
    STS_CUDA(cudaStreamSynchronize(S(stream)));
    const int st = ((int32_t*)ctx->h_pinned)[0];
    STS_CUDA(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), S(stream)));
    if (st & kStatusCapacity) {
        set_error("device capacity exceeded");
        return STS_ERR_CAPACITY;
    }
    if (st & kStatusNonfinite) {
        set_error("non-finite position");
        return STS_ERR_NONFINITE;
    }
    if (st & kStatusTimeout) {
        set_error("a device-side wait for staged sources gave up; results of that launch are incomplete");
        return STS_ERR_TIMEOUT;
    }
    return STS_OK;
}

int sts_selftest_wait(sts_ctx* ctx, int32_t spins, void* stream)
{
    int rc = check_ctx(ctx, "sts_selftest_wait");
    if (rc) return rc;
    if (spins < 1 || spins > (1 << 20)) {
        set_error("sts_selftest_wait: spins must be in [1, 2^20]");
        return STS_ERR_ARG;
    }
    if ((rc = wait_selftest(ctx, spins, S(stream)))) return rc;
    return sts_status(ctx, stream);
}

int sts_potential(sts_ctx* ctx, const double* zeta, const double* area, const sts_params* p, double* psi,
                  void* stream)
{
    int rc = check_ctx(ctx, "sts_potential");
    if (rc || (rc = check_params(p, "sts_potential"))) return rc;
    if (!ctx->have_tree) {
        set_error("sts_potential: no tree (call sts_tree_build first)");
        return STS_ERR_STATE;
    }
    if (ctx->n > 0 && (!zeta || !area || !psi)) {
        set_error("sts_potential: NULL array");
        return STS_ERR_ARG;
    }
    return potential_impl(ctx, zeta, area, p, psi, S(stream));
}

int sts_direct_potential(sts_ctx* ctx, const double* pos, const double* zeta, const double* area, int64_t n,
                         int32_t precision, double* psi, void* stream)
{
    int rc = check_ctx(ctx, "sts_direct_potential");
    if (rc || (rc = check_n(n, "sts_direct_potential"))) return rc;
    if (precision != STS_FP64) {
        set_error("sts_direct_potential: only precision STS_FP64 is implemented");
        return STS_ERR_ARG;
    }
    if (n > 0 && (!pos || !zeta || !area || !psi)) {
        set_error("sts_direct_potential: NULL array");
        return STS_ERR_ARG;
    }
    if (n == 0) return STS_OK;
    if (n == 1) {
        STS_CUDA(cudaMemsetAsync(psi, 0, sizeof(double), S(stream)));
        return STS_OK;
    }
    return direct_potential(ctx, pos, zeta, area, n, psi, S(stream));
}

int sts_direct(sts_ctx* ctx, const double* pos, const double* zeta, const double* area, int64_t n,
               int32_t precision, double* vel, void* stream)
{
    int rc = check_ctx(ctx, "sts_direct");
    if (rc || (rc = check_n(n, "sts_direct"))) return rc;
    if (precision != STS_FP64 && precision != STS_MIXED) {
        set_error("sts_direct: precision must be STS_FP64 or STS_MIXED");
        return STS_ERR_ARG;
    }
    if (n > 0 && (!pos || !zeta || !area || !vel)) {
        set_error("sts_direct: NULL array");
        return STS_ERR_ARG;
    }
    if (n == 0) return STS_OK;
    if (n == 1) {
        STS_CUDA(cudaMemsetAsync(vel, 0, 3 * sizeof(double), S(stream)));
        return STS_OK;
    }
    return direct_sum(ctx, pos, zeta, area, n, nullptr, n, precision, vel, S(stream));
}

int sts_direct_targets(sts_ctx* ctx, const double* pos, const double* zeta, const double* area,
                       int64_t n, const int64_t* targets, int64_t nt, int32_t precision, double* vel,
                       void* stream)
{
    int rc = check_ctx(ctx, "sts_direct_targets");
    if (rc || (rc = check_n(n, "sts_direct_targets"))) return rc;
    if (precision != STS_FP64 && precision != STS_MIXED) {
        set_error("sts_direct_targets: precision must be STS_FP64 or STS_MIXED");
        return STS_ERR_ARG;
    }
    if (nt < 0 || (nt > 0 && (n < 1 || !targets || !vel || !pos || !zeta || !area))) {
        set_error("sts_direct_targets: bad targets or NULL array");
        return STS_ERR_ARG;
    }
    if (nt == 0) return STS_OK;
    return direct_sum(ctx, pos, zeta, area, n, targets, nt, precision, vel, S(stream));
}

int sts_tree_build(sts_ctx* ctx, const double* pos, int64_t n, const sts_params* p, void* stream)
{
    int rc = check_ctx(ctx, "sts_tree_build");
    if (rc || (rc = check_n(n, "sts_tree_build")) || (rc = check_params(p, "sts_tree_build"))) return rc;
    if (n > 0 && !pos) {
        set_error("sts_tree_build: NULL pos");
        return STS_ERR_ARG;
    }
    return build_impl(ctx, pos, n, nullptr, 1, p, S(stream));
}

int sts_velocity(sts_ctx* ctx, const double* zeta, const double* area, const sts_params* p, double* vel,
                 void* stream)
{
    int rc = check_ctx(ctx, "sts_velocity");
    if (rc || (rc = check_params(p, "sts_velocity"))) return rc;
    if (!ctx->have_tree) {
        set_error("sts_velocity: no tree (call sts_tree_build first)");
        return STS_ERR_STATE;
    }
    if (ctx->n > 0 && (!zeta || !area || !vel)) {
        set_error("sts_velocity: NULL array");
        return STS_ERR_ARG;
    }
    return velocity_impl(ctx, zeta, area, p, vel, S(stream));
}

int sts_velocity_dual(sts_ctx* ctx, const double* zeta, const double* area, const sts_params* p, double* vel,
                      void* stream)
{
    int rc = check_ctx(ctx, "sts_velocity_dual");
    if (rc || (rc = check_params(p, "sts_velocity_dual"))) return rc;
    if (!ctx->have_tree) {
        set_error("sts_velocity_dual: no tree (call sts_tree_build first)");
        return STS_ERR_STATE;
    }
    if (ctx->capturing) {
        set_error("sts_velocity_dual: not available while recording");
        return STS_ERR_STATE;
    }
    if (ctx->n > 0 && (!zeta || !area || !vel)) {
        set_error("sts_velocity_dual: NULL array");
        return STS_ERR_ARG;
    }
    return velocity_dual_impl(ctx, zeta, area, p, vel, S(stream));
}

int sts_velocity_range(sts_ctx* ctx, const double* zeta, const double* area, const sts_params* p,
                       int64_t leaf_begin, int64_t leaf_end, int32_t out_sorted, double* vel, void* stream)
{
    int rc = check_ctx(ctx, "sts_velocity_range");
    if (rc || (rc = check_params(p, "sts_velocity_range"))) return rc;
    if (!ctx->have_tree) {
        set_error("sts_velocity_range: no tree (call sts_tree_build first)");
        return STS_ERR_STATE;
    }
    if (ctx->capturing || ctx->use_dual) {
        set_error("sts_velocity_range: needs eager calls on the target-leaf lists (traversal 0)");
        return STS_ERR_STATE;
    }
    if (ctx->n > 0 && (!zeta || !area || (!vel && leaf_end > leaf_begin))) {
        set_error("sts_velocity_range: NULL array");
        return STS_ERR_ARG;
    }
    cudaStream_t s = S(stream);
    const int64_t n = ctx->n;
    if (n < 2) {
        if (leaf_begin < 0 || leaf_end < leaf_begin || leaf_end > (n > 0 ? 1 : 0)) {
            set_error("sts_velocity_range: leaf range [%lld, %lld) outside [0, %lld)", (long long)leaf_begin,
                      (long long)leaf_end, (long long)(n > 0 ? 1 : 0));
            return STS_ERR_ARG;
        }
        if (n == 1 && leaf_end > leaf_begin) STS_CUDA(cudaMemsetAsync(vel, 0, 3 * sizeof(double), s));
        return STS_OK;
    }
    if ((rc = sources_and_lists(ctx, zeta, area, p, p->precision, false, s))) return rc;
    ctx->list_degree = p->degree;
    if ((rc = refresh_counts(ctx, s))) return rc;
    if (leaf_begin < 0 || leaf_end < leaf_begin || leaf_end > ctx->nleaves) {
        set_error("sts_velocity_range: leaf range [%lld, %lld) outside [0, %lld)", (long long)leaf_begin,
                  (long long)leaf_end, (long long)ctx->nleaves);
        return STS_ERR_ARG;
    }
    int64_t base = -1;
    if (out_sorted) {
        int64_t hi = 0;
        if ((rc = leaf_range_slots(ctx, leaf_begin, leaf_end, &base, &hi, s))) return rc;
    }
    if (leaf_end == leaf_begin) return STS_OK;
    return evaluate_range(ctx, p->degree, p->precision, p->near_fp64_tau, leaf_begin, leaf_end, base, vel, s);
}

int sts_leaf_work(sts_ctx* ctx, int32_t degree, int64_t* work, void* stream)
{
    int rc = check_ctx(ctx, "sts_leaf_work");
    if (rc) return rc;
    if ((rc = refresh_counts(ctx, S(stream)))) return rc;
    if (!ctx->have_lists) {
        set_error("sts_leaf_work: no target-leaf lists (call sts_velocity first)");
        return STS_ERR_STATE;
    }
    if (degree < 1 || degree > kMaxDegree || (!work && ctx->nleaves > 0)) {
        set_error("sts_leaf_work: degree must be in [1, %d] and work non-NULL", kMaxDegree);
        return STS_ERR_ARG;
    }
    return leaf_work(ctx, degree, work, S(stream));
}

int sts_leaf_range(sts_ctx* ctx, int64_t leaf_begin, int64_t leaf_end, int64_t* slot_begin, int64_t* slot_end,
                   void* stream)
{
    int rc = check_ctx(ctx, "sts_leaf_range");
    if (rc) return rc;
    if ((rc = refresh_counts(ctx, S(stream)))) return rc;
    if (!ctx->have_tree || !slot_begin || !slot_end) {
        set_error("sts_leaf_range: no tree, or NULL output");
        return ctx->have_tree ? STS_ERR_ARG : STS_ERR_STATE;
    }
    const int64_t L = ctx->n < 2 ? (ctx->n > 0 ? 1 : 0) : ctx->nleaves;
    if (leaf_begin < 0 || leaf_end < leaf_begin || leaf_end > L) {
        set_error("sts_leaf_range: leaf range [%lld, %lld) outside [0, %lld)", (long long)leaf_begin,
                  (long long)leaf_end, (long long)L);
        return STS_ERR_ARG;
    }
    if (ctx->n < 2) {
        *slot_begin = leaf_begin;
        *slot_end = leaf_end;
        return STS_OK;
    }
    return leaf_range_slots(ctx, leaf_begin, leaf_end, slot_begin, slot_end, S(stream));
}

int sts_unpermute(sts_ctx* ctx, const double* vel_sorted, double* vel, void* stream)
{
    int rc = check_ctx(ctx, "sts_unpermute");
    if (rc) return rc;
    if (!ctx->have_tree) {
        set_error("sts_unpermute: no tree (call sts_tree_build first)");
        return STS_ERR_STATE;
    }
    if (ctx->n > 0 && (!vel_sorted || !vel)) {
        set_error("sts_unpermute: NULL array");
        return STS_ERR_ARG;
    }
    if (ctx->n == 1) {
        STS_CUDA(cudaMemcpyAsync(vel, vel_sorted, 3 * sizeof(double), cudaMemcpyDeviceToDevice, S(stream)));
        return STS_OK;
    }
    return unpermute(ctx, vel_sorted, vel, S(stream));
}

int sts_dual_export(sts_ctx* ctx, int32_t kind, int64_t* npairs, int32_t* tgt, int32_t* src, void* stream)
{
    int rc = check_ctx(ctx, "sts_dual_export");
    if (rc) return rc;
    if (kind < 0 || kind > 3) {
        set_error("sts_dual_export: kind must be 0 (PP), 1 (PC), 2 (CP) or 3 (CC), got %d", kind);
        return STS_ERR_ARG;
    }
    if (!ctx->have_dual) {
        set_error("sts_dual_export: no dual lists (call sts_velocity_dual first)");
        return STS_ERR_STATE;
    }
    if ((rc = refresh_counts(ctx, S(stream)))) return rc;
    return dual_export(ctx, kind, npairs, tgt, src, S(stream));
}

int sts_amr_init(sts_ctx* ctx, const int32_t* faces, int64_t nfaces, int64_t n0, const double* pos0,
                 const double* zeta0, int32_t levels, void* stream)
{
    int rc = check_ctx(ctx, "sts_amr_init");
    if (rc) return rc;
    if (!faces || !pos0 || !zeta0 || nfaces < 1 || n0 < 3 || levels < 0 || levels > 6) {
        set_error("sts_amr_init: need faces, pos0, zeta0, nfaces >= 1, n0 >= 3 and 0 <= levels <= 6");
        return STS_ERR_ARG;
    }
    if ((rc = check_n(n0, "sts_amr_init"))) return rc;
    return amr_init(ctx, faces, nfaces, n0, pos0, zeta0, levels, S(stream));
}

int sts_amr_step(sts_ctx* ctx, double eps1, double eps2, int64_t* counts, void* stream)
{
    int rc = check_ctx(ctx, "sts_amr_step");
    if (rc) return rc;
    if (!ctx->amr) {
        set_error("sts_amr_step: no mesh (call sts_amr_init first)");
        return STS_ERR_STATE;
    }
    if (std::isnan(eps1) || std::isnan(eps2)) {
        set_error("sts_amr_step: eps1 and eps2 must not be NaN");
        return STS_ERR_ARG;
    }
    return amr_step(ctx, eps1, eps2, counts, S(stream));
}

int sts_amr_info(sts_ctx* ctx, int64_t* info)
{
    int rc = check_ctx(ctx, "sts_amr_info");
    if (rc) return rc;
    if (!ctx->amr || !info) {
        set_error("sts_amr_info: no mesh or NULL info");
        return ctx->amr ? STS_ERR_ARG : STS_ERR_STATE;
    }
    return amr_info(ctx, info);
}

int sts_amr_gather(sts_ctx* ctx, double* pos, double* zeta, double* area, int64_t* ids, void* stream)
{
    int rc = check_ctx(ctx, "sts_amr_gather");
    if (rc) return rc;
    if (!ctx->amr) {
        set_error("sts_amr_gather: no mesh (call sts_amr_init first)");
        return STS_ERR_STATE;
    }
    return amr_gather(ctx, pos, zeta, area, ids, S(stream));
}

int sts_amr_scatter(sts_ctx* ctx, const double* pos, const double* zeta, void* stream)
{
    int rc = check_ctx(ctx, "sts_amr_scatter");
    if (rc) return rc;
    if (!ctx->amr || !pos || !zeta) {
        set_error("sts_amr_scatter: no mesh or NULL array");
        return ctx->amr ? STS_ERR_ARG : STS_ERR_STATE;
    }
    return amr_scatter(ctx, pos, zeta, S(stream));
}

int sts_amr_export(sts_ctx* ctx, int32_t* tv, int32_t* tparent, int32_t* tchild, int8_t* tlevel,
                   int32_t* vparent, uint8_t* tstate, uint8_t* valive, double* pos, double* zeta, double* area,
                   void* stream)
{
    int rc = check_ctx(ctx, "sts_amr_export");
    if (rc) return rc;
    if (!ctx->amr) {
        set_error("sts_amr_export: no mesh (call sts_amr_init first)");
        return STS_ERR_STATE;
    }
    return amr_export(ctx, tv, tparent, tchild, tlevel, vparent, tstate, valive, pos, zeta, area, S(stream));
}

int sts_set_traversal(sts_ctx* ctx, int32_t dual)
{
    int rc = check_ctx(ctx, "sts_set_traversal");
    if (rc) return rc;
    if (dual != 0 && dual != 1) {
        set_error("sts_set_traversal: dual must be 0 (target-leaf lists) or 1 (dual traversal), got %d", dual);
        return STS_ERR_ARG;
    }
    ctx->use_dual = dual != 0;
    return STS_OK;
}

int sts_dual_stats(sts_ctx* ctx, int32_t degree, int64_t* stats, void* stream)
{
    int rc = check_ctx(ctx, "sts_dual_stats");
    if (rc) return rc;
    if (!stats || degree < 1 || degree > kMaxDegree) {
        set_error("sts_dual_stats: stats must be non-NULL and 1 <= degree <= %d", kMaxDegree);
        return STS_ERR_ARG;
    }
    if (!ctx->have_dual) {
        set_error("sts_dual_stats: no dual lists (call sts_velocity_dual first)");
        return STS_ERR_STATE;
    }
    if ((rc = refresh_counts(ctx, S(stream)))) return rc;
    return dual_stats(ctx, degree, stats, S(stream));
}

int sts_tree_build_batched(sts_ctx* ctx, const double* pos, const int64_t* offsets, int32_t ninst,
                           const sts_params* p, void* stream)
{
    int rc = check_ctx(ctx, "sts_tree_build_batched");
    if (rc || (rc = check_params(p, "sts_tree_build_batched"))) return rc;
    const int64_t* d_off = nullptr;
    int64_t n = 0;
    if ((rc = upload_offsets(ctx, offsets, ninst, &d_off, &n, "sts_tree_build_batched", S(stream)))) return rc;
    if (n > 0 && !pos) {
        set_error("sts_tree_build_batched: NULL pos");
        return STS_ERR_ARG;
    }
    return build_impl(ctx, pos, n, d_off, ninst, p, S(stream));
}

int bve_rk4_step(sts_ctx* ctx, double* pos, double* zeta, const double* area, int64_t n, double dt,
                 double Omega, const sts_params* p, void* stream)
{
    int rc = check_ctx(ctx, "bve_rk4_step");
    if (rc || (rc = check_n(n, "bve_rk4_step")) || (rc = check_params(p, "bve_rk4_step"))) return rc;
    if (ctx->graph_on) return rk4_graph(ctx, pos, zeta, area, n, nullptr, nullptr, 1, dt, Omega, p, S(stream));
    return rk4_impl(ctx, pos, zeta, area, n, nullptr, 1, dt, Omega, p, S(stream));
}

int bve_rk4_step_forced(sts_ctx* ctx, double* pos, double* zeta, const double* area, int64_t n, double t,
                        double dt, double Omega, const sts_forcing* f, const sts_params* p, void* stream)
{
    int rc = check_ctx(ctx, "bve_rk4_step_forced");
    if (rc || (rc = check_params(p, "bve_rk4_step_forced")) || (rc = check_n(n, "bve_rk4_step_forced"))) return rc;
    if (!f || f->k < 1 || !(f->Tp > 0.0) || !(f->Tf >= 2.0 * f->Tp) || !(f->theta1 > 0.0) ||
        !(f->theta1 < 1.5707963267948966) || !isfinite(f->amplitude) || !isfinite(f->Tf) || !isfinite(t)) {
        set_error("bve_rk4_step_forced: forcing needs k >= 1, Tp > 0, Tf >= 2 Tp, 0 < theta1 < pi/2, finite values");
        return STS_ERR_ARG;
    }
    return rk4_impl(ctx, pos, zeta, area, n, nullptr, 1, dt, Omega, p, S(stream), f, t);
}

int bve_rk4_step_batched(sts_ctx* ctx, double* pos, double* zeta, const double* area, const int64_t* offsets,
                         int32_t ninst, double dt, double Omega, const sts_params* p, void* stream)
{
    int rc = check_ctx(ctx, "bve_rk4_step_batched");
    if (rc || (rc = check_params(p, "bve_rk4_step_batched"))) return rc;
    const int64_t* d_off = nullptr;
    int64_t n = 0;
    if ((rc = upload_offsets(ctx, offsets, ninst, &d_off, &n, "bve_rk4_step_batched", S(stream)))) return rc;
    if (ctx->graph_on) return rk4_graph(ctx, pos, zeta, area, n, d_off, offsets, ninst, dt, Omega, p, S(stream));
    return rk4_impl(ctx, pos, zeta, area, n, d_off, ninst, dt, Omega, p, S(stream));
}

int sts_tree_info(sts_ctx* ctx, int64_t* info, void* stream)
{
    int rc = check_ctx(ctx, "sts_tree_info");
    if (rc) return rc;
    if ((rc = refresh_counts(ctx, S(stream)))) return rc;
    if (!info) {
        set_error("sts_tree_info: NULL info");
        return STS_ERR_ARG;
    }
    STS_CUDA(cudaStreamSynchronize(S(stream)));
    info[0] = ctx->have_tree ? ctx->n : 0;
    info[1] = ctx->nnodes;
    info[2] = ctx->nleaves;
    info[3] = ctx->deepest;
    const bool lists = ctx->have_lists || ctx->have_dual;  // leaf lists (the dual's PP / PC)
    info[4] = lists ? ctx->nfar : 0;
    info[5] = lists ? ctx->nnear : 0;
    info[6] = ctx->nclusters;
    info[7] = lists ? ctx->ntasks : 0;
    return STS_OK;
}

int sts_tree_export(sts_ctx* ctx, int64_t* perm, int32_t* level, uint64_t* key, int32_t* parent,
                    int32_t* first_child, int32_t* nchild, int64_t* start, int64_t* count, int32_t* leaf,
                    int32_t* leaves, double* geom, void* stream)
{
    int rc = check_ctx(ctx, "sts_tree_export");
    if (rc) return rc;
    if ((rc = refresh_counts(ctx, S(stream)))) return rc;
    if (!ctx->have_tree) {
        set_error("sts_tree_export: no tree");
        return STS_ERR_STATE;
    }
    cudaStream_t s = S(stream);
    const int64_t nn = ctx->nnodes;
    if ((rc = copy_out(perm, ctx->perm.p, ctx->n, s)) || (rc = copy_out(level, ctx->nd_level.p, nn, s)) ||
        (rc = copy_out(key, ctx->nd_key.p, nn, s)) || (rc = copy_out(parent, ctx->nd_parent.p, nn, s)) ||
        (rc = copy_out(first_child, ctx->nd_first_child.p, nn, s)) ||
        (rc = copy_out(nchild, ctx->nd_nchild.p, nn, s)) || (rc = copy_out(start, ctx->nd_start.p, nn, s)) ||
        (rc = copy_out(count, ctx->nd_count.p, nn, s)) || (rc = copy_out(leaf, ctx->nd_leaf.p, nn, s)) ||
        (rc = copy_out(leaves, ctx->leaves.p, ctx->nleaves, s)) ||
        (rc = copy_out(geom, ctx->nd_geom.p, 13 * nn, s)))
        return rc;
    return STS_OK;
}

int sts_lists_export(sts_ctx* ctx, int64_t* far_off, int32_t* far_idx, int64_t* near_off, int32_t* near_idx,
                     void* stream)
{
    int rc = check_ctx(ctx, "sts_lists_export");
    if (rc) return rc;
    if ((rc = refresh_counts(ctx, S(stream)))) return rc;
    if (!ctx->have_lists) {
        set_error("sts_lists_export: no lists (call sts_velocity first)");
        return STS_ERR_STATE;
    }
    cudaStream_t s = S(stream);
    const int64_t L = ctx->nleaves;
    if ((rc = copy_out(far_off, ctx->far_off.p, L + 1, s)) || (rc = copy_out(near_off, ctx->near_off.p, L + 1, s)) ||
        (rc = copy_out(far_idx, ctx->far_idx.p, ctx->nfar, s)) ||
        (rc = copy_out(near_idx, ctx->near_idx.p, ctx->nnear, s)))
        return rc;
    return STS_OK;
}

int sts_clusters_export(sts_ctx* ctx, int32_t* node_ids, double* yt, double* W, void* stream)
{
    int rc = check_ctx(ctx, "sts_clusters_export");
    if (rc) return rc;
    if ((rc = refresh_counts(ctx, S(stream)))) return rc;
    if (ctx->up_degree < 0) {
        set_error("sts_clusters_export: no proxy weights (call sts_velocity first)");
        return STS_ERR_STATE;
    }
    cudaStream_t s = S(stream);
    const int64_t C = ctx->nclusters;
    const int M = nbasis(ctx->up_degree);
    if ((rc = copy_out(node_ids, ctx->cluster_node.p, C, s))) return rc;
    if ((yt || W) && C > 0) {
        std::vector<double4> tmp((size_t)(C * M));
        STS_CUDA(cudaMemcpyAsync(tmp.data(), ctx->prx64.p, C * M * sizeof(double4), cudaMemcpyDeviceToHost, s));
        STS_CUDA(cudaStreamSynchronize(s));
        for (int64_t q = 0; q < C * M; q++) {
            if (yt) {
                yt[3 * q] = tmp[(size_t)q].x;
                yt[3 * q + 1] = tmp[(size_t)q].y;
                yt[3 * q + 2] = tmp[(size_t)q].z;
            }
            if (W) W[q] = 0.5 * tmp[(size_t)q].w;
        }
    }
    return STS_OK;
}

int sts_proxy_reference(int32_t degree, double* beta, double* vinv)
{
    g_err[0] = 0;
    if (degree < 1 || degree > kMaxDegree) {
        set_error("sts_proxy_reference: degree must be in [1, %d]", kMaxDegree);
        return STS_ERR_ARG;
    }
    RefTable t;
    if (build_ref_table(degree, &t) != STS_OK) {
        set_error("sts_proxy_reference: degree %d table failed", degree);
        return STS_ERR_ARG;
    }
    if (beta) memcpy(beta, t.beta.data(), t.beta.size() * sizeof(double));
    if (vinv) memcpy(vinv, t.vinv.data(), t.vinv.size() * sizeof(double));
    return STS_OK;
}

int sts_stats(sts_ctx* ctx, int64_t* stats, void* stream)
{
    int rc = check_ctx(ctx, "sts_stats");
    if (rc) return rc;
    if ((rc = refresh_counts(ctx, S(stream)))) return rc;
    if (!stats) {
        set_error("sts_stats: NULL stats");
        return STS_ERR_ARG;
    }
    if (!ctx->have_lists || ctx->list_degree < 0) {
        set_error("sts_stats: no lists (call sts_velocity first)");
        return STS_ERR_STATE;
    }
    cudaStream_t s = S(stream);
    if ((rc = count_interactions(ctx, ctx->list_degree, s))) return rc;
    unsigned long long h[2];
    STS_CUDA(cudaMemcpyAsync(h, ctx->d_stats.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    STS_CUDA(cudaStreamSynchronize(s));
    stats[0] = (int64_t)h[0];
    stats[1] = (int64_t)h[1];
    return STS_OK;
}

int sts_set_timing(sts_ctx* ctx, int32_t on)
{
    int rc = check_ctx(ctx, "sts_set_timing");
    if (rc) return rc;
    if (on) {
        for (int p = 0; p < kNumPhases; p++)
            for (int q = 0; q < 2; q++)
                if (!ctx->ev[p][q]) STS_CUDA(cudaEventCreate(&ctx->ev[p][q]));
    }
    for (int p = 0; p < kNumPhases; p++) {
        ctx->phase_ms[p] = 0.f;
        ctx->phase_count[p] = 0;
        ctx->phase_open[p] = false;
    }
    ctx->timing = on != 0;
    return STS_OK;
}

int sts_phase_times(sts_ctx* ctx, double* ms, int32_t* count, int32_t nph)
{
    int rc = check_ctx(ctx, "sts_phase_times");
    if (rc) return rc;
    if (nph < 0 || nph > kNumPhases) {
        set_error("sts_phase_times: nph must be in [0, %d]", kNumPhases);
        return STS_ERR_ARG;
    }
    for (int p = 0; p < nph; p++) {
        if (ctx->phase_open[p]) {
            float m = 0.f;
            STS_CUDA(cudaEventSynchronize(ctx->ev[p][1]));
            STS_CUDA(cudaEventElapsedTime(&m, ctx->ev[p][0], ctx->ev[p][1]));
            ctx->phase_ms[p] += m;
            ctx->phase_count[p] += 1;
            ctx->phase_open[p] = false;
        }
        if (ms) ms[p] = ctx->phase_ms[p];
        if (count) count[p] = ctx->phase_count[p];
    }
    return STS_OK;
}

int sts_launch_count(int64_t* out)
{
    g_err[0] = 0;
    if (!out) {
        set_error("sts_launch_count: NULL out");
        return STS_ERR_ARG;
    }
    *out = (int64_t)g_launches.load(std::memory_order_relaxed);
    return STS_OK;
}

int sts_set_graph(sts_ctx* ctx, int32_t on)
{
    int rc = check_ctx(ctx, "sts_set_graph");
    if (rc) return rc;
    ctx->graph_on = on != 0;
    if (!ctx->graph_on && ctx->rk_exec) {
        cudaGraphExecDestroy(ctx->rk_exec);
        ctx->rk_exec = nullptr;
    }
    if (!ctx->graph_on && ctx->ev_exec) {
        cudaGraphExecDestroy(ctx->ev_exec);
        ctx->ev_exec = nullptr;
    }
    return STS_OK;
}

int sts_tree_velocity(sts_ctx* ctx, const double* pos, const double* zeta, const double* area,
                      const int64_t* offsets, int32_t ninst, const sts_params* p, double* vel, void* stream)
{
    int rc = check_ctx(ctx, "sts_tree_velocity");
    if (rc || (rc = check_params(p, "sts_tree_velocity"))) return rc;
    const int64_t* d_off = nullptr;
    int64_t n = 0;
    if ((rc = upload_offsets(ctx, offsets, ninst, &d_off, &n, "sts_tree_velocity", S(stream)))) return rc;
    if (n > 0 && (!pos || !zeta || !area || !vel)) {
        set_error("sts_tree_velocity: NULL array");
        return STS_ERR_ARG;
    }
    if (ninst == 1) d_off = nullptr;
    if (ctx->graph_on && n >= 2)
        return eval_graph(ctx, pos, zeta, area, n, d_off, ninst > 1 ? offsets : nullptr, ninst, p, vel, S(stream));
    if ((rc = build_impl(ctx, pos, n, d_off, ninst, p, S(stream)))) return rc;
    return velocity_impl(ctx, zeta, area, p, vel, S(stream));
}

}  // extern "C"
