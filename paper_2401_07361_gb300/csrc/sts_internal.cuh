// Internal declarations shared by the translation units of libsts (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <vector>

#include "../../include/sts.h"

namespace sts {

constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxDegree = 16;
constexpr int kMaxM = (kMaxDegree + 1) * (kMaxDegree + 2) / 2;  // 153
constexpr int kMaxLevel = 24;

// Device status word bits (ORed by kernels, read and cleared by sts_status).
constexpr int kStatusCapacity = 1;
constexpr int kStatusNonfinite = 2;
constexpr int kStatusTimeout = 4;  // a bounded device-side wait gave up

// Evaluation tasks: one warp evaluates up to kTaskTargets consecutive targets of a leaf, two
// per lane.
constexpr int kTaskTargets = 64;
// Source blocks (a cluster's proxy points, a chunk of a near leaf) hold at most kStage
// entries, so that one block fits the shared-memory stage; kStage >= the largest M.
constexpr int kStage = 160;
// Upward pass: one CTA folds kUpChunk particles of one cluster into SBB moments.
constexpr int kUpChunk = 128;

void set_error(const char* fmt, ...);
// Counts kernel launches of the library (reported by sts_launch_count).
void note_launch();

// Count of device (re)allocations made by any DevBuf.  A recorded graph holds buffer addresses,
// so it is replayed only while this count equals the one seen when it was recorded.
inline std::atomic<unsigned long long> g_alloc_epoch{0};

// A device buffer that only grows.  reserve() drops the old contents; grow() keeps them.
// cudaMalloc / cudaFree happen outside any stream capture.
template <class T>
struct DevBuf {
    T* p = nullptr;
    size_t cap = 0;  // elements
    cudaError_t reserve(size_t n)
    {
        if (n <= cap) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        size_t want = n + n / 8 + 16;
        g_alloc_epoch.fetch_add(1);
        cudaError_t e = cudaMalloc((void**)&p, want * sizeof(T));
        if (e == cudaSuccess) cap = want;
        return e;
    }
    cudaError_t grow(size_t n, size_t keep, cudaStream_t s)
    {
        if (n <= cap) return cudaSuccess;
        size_t want = n + n / 2 + 16;
        T* q = nullptr;
        cudaError_t e = cudaMalloc((void**)&q, want * sizeof(T));
        if (e != cudaSuccess) return e;
        if (p && keep) {
            e = cudaMemcpyAsync(q, p, keep * sizeof(T), cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) {
                cudaFree(q);
                return e;
            }
            e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) {
                cudaFree(q);
                return e;
            }
        }
        if (p) cudaFree(p);
        p = q;
        cap = want;
        g_alloc_epoch.fetch_add(1);
        return cudaSuccess;
    }
    void release()
    {
        if (p) g_alloc_epoch.fetch_add(1);
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
};

// Reference interpolation data for one degree (host computed, copied to the device).
struct RefTable {
    int degree = 0, M = 0;
    std::vector<double> beta;  // [M,3] barycentric proxy points on the reference simplex
    std::vector<double> vinv;  // [M,M], vinv[k*M+m] = (V_ref^{-1})[k][m]
    DevBuf<double> d_beta, d_vinv;
    DevBuf<double> d_vinvT;    // [M,M], d_vinvT[m*M+k] = (V_ref^{-1})[k][m] (threads over k read rows)
    // The tensor-core contraction's operand B: V_ref^{-1} with row k scaled by 2^-E[k] and
    // column m by 2^-F[m] (into (-1/2, 1/2)), split into kTcSlices balanced base-256 digits,
    // slice b (1-based) = digit b; each slice is an [Np, Kp] bf16 matrix (row n = proxy point
    // m, K = basis index k, zero padded) in the tcgen05 no-swizzle K-major layout (8 x 8 core
    // matrices, K-adjacent ones 128 bytes apart, row groups Kp * 16 bytes apart).
    int tcKp = 0, tcNp = 0;
    DevBuf<uint16_t> d_tcB;    // [kTcSlices][Np * Kp]
    DevBuf<int32_t> d_tcF;     // [Np]
    DevBuf<int32_t> d_tcE;     // [Kp] moment scales (powers of two)
    // The same for the dual traversal's coefficients c = V_ref^{-1} u: operand B holds the rows
    // of V_ref^{-1} (row n = coefficient k, K = proxy point m), row k scaled by 2^-Fr[k].
    DevBuf<uint16_t> d_tcBr;   // [kTcSlices][Np * Kp]
    DevBuf<int32_t> d_tcFr;    // [Np]
};
// Digits of the tensor-core contraction: kTcSlices x 8 bits hold every bit of an FP64 entry
// (below 2^-57 of its column's largest).
constexpr int kTcSlices = 7;
// Byte offset of element (r, k) of a K-major [rows, Kp] bf16 matrix in the no-swizzle layout.
__host__ __device__ inline unsigned tc_kmajor_offset(int r, int k, int Kp)
{
    return (unsigned)((r >> 3) * (Kp * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Far-field list entry as the evaluation kernel reads it: proxy block of cluster `slot`
// and the offset c_cluster - c_target_leaf rounded to FP32 (mixed precision).
struct FarEntry {
    int32_t slot;
    float dx, dy, dz;
};
// Near-field list entry: a chunk of at most kStage particles [start, start + count) of a
// source leaf, the offset c_source_leaf - c_target_leaf rounded to FP32, and a lower bound
// on the chord distance between any point of the target leaf and any of the source leaf
// (|c_t - c_s| - r_t - r_s, rounded down), which tells whether a pair can fall below tau.
struct NearEntry {
    int32_t start, count;
    float dx, dy, dz;
    float gap;
    int32_t pad[2];
};
// Evaluation task: targets [t0, t0 + nt) (sorted slots) of leaf `leaf` (depth-first index);
// S lanes share each pair of targets and split the sources between them.
struct Task {
    int32_t leaf, t0, nt, S;
};

enum Phase { kPhBuild = 0, kPhSort, kPhLists, kPhPrep, kPhUpward, kPhEval, kPhDirect, kPhCluster, kNumPhases };

// Device counters (ctx->dc, int64): every kernel reads its element counts from here, so no
// launch depends on a host-side count and a whole RK4 step can be recorded as a graph.
enum DevCount {
    kDcRoots = 0, kDcLeaves, kDcClusters, kDcUpTasks, kDcFar, kDcNear, kDcChunks, kDcTasks, kDcNodes,
    kDcOver,   // overflow bits: 1 node capacity, 2 levels, 4 list or task capacity
    kDcTmp,
    kDcLevel = 16,  // level_begin[0 .. kMaxLevel + 3]
    kDcClass = 44,      // evaluation tasks per lane class S = 1 .. 8 (8 counters)
    kDcClassFill = 52,  // tasks placed so far per class (8 counters)
    kDcQueue = 60,      // next task of the persistent evaluation kernels
    kDcSize = 64
};

// Sizes seen by the last eager build (maxima over a step), used as capacities when recording.
struct Plan {
    int64_t n = -1;
    int ninst = 0, leaf_size = 0, max_level = 0, depth = 0;
    int64_t nodes = 0, up_tasks = 0, far = 0, near = 0, chunks = 0, tasks = 0, clusters = 0, leaves = 0;
    // dual traversal: largest frontier, terminal pairs, and per kind pairs and near chunks
    int64_t dual_front = 0, dual_terms = 0, dual_pairs[4] = {0, 0, 0, 0}, dual_chunks[2] = {0, 0};
};

struct AmrState;  // adaptive mesh refinement of the particle triangulation (sts_amr.cu)

}  // namespace sts

struct sts_ctx {
    int device = 0;
    int* d_status = nullptr;  // device status word
    int64_t* h_pinned = nullptr;  // small pinned host staging buffer [kDcSize + 16]

    // ---- tree over the current positions -------------------------------------------
    int64_t n = 0;
    int leaf_size = 0, max_level = 0;
    bool have_tree = false;
    sts::DevBuf<double> pos;             // [n,3] copy of the positions (caller order)
    sts::DevBuf<int32_t> nodeof;         // [n] original index -> deepest node so far
    sts::DevBuf<uint8_t> digit;          // [n] child digit at the current level
    sts::DevBuf<int32_t> perm, perm_tmp; // [n] sorted slot -> original index
    sts::DevBuf<uint32_t> skey, skey_tmp;// [n] sort keys
    sts::DevBuf<int64_t> scan_tmp;       // scan scratch
    sts::DevBuf<uint32_t> hist;          // digit counts of the sort inside the tree build
    sts::DevBuf<int32_t> flags;          // [n + 1] scratch
    sts::DevBuf<int64_t> offs;           // [n + 1] scratch
    // node table (level by level, key order within a level)
    int64_t nnodes = 0, nleaves = 0, deepest = 0;
    std::vector<int64_t> level_begin;    // first node id of each level, plus the end
    sts::DevBuf<int32_t> nd_level, nd_parent, nd_first_child, nd_nchild, nd_start, nd_count,
        nd_leaf;
    sts::DevBuf<uint64_t> nd_key;
    sts::DevBuf<double> nd_geom;         // [nodes,13]: v1, v2, v3, c, r
    sts::DevBuf<double> nd_norm;         // [nodes,9]: child-digit normals of split nodes
    sts::DevBuf<float4> nd_norm32;       // [nodes,3]: the normals in FP32 + pre-filter margin
    sts::DevBuf<double> nd_mid;          // [nodes,9]: edge midpoints m12, m23, m31 of split nodes
    int num_sms = 1;                                  // SMs of the context's device (sts_create)
    int eval_blocks_mixed = 0, eval_blocks_fp64 = 0;  // resident blocks of the persistent eval kernels
    sts::DevBuf<float4> nd_c32;          // [nodes]: circumcentre and chord radius in FP32
    sts::DevBuf<float4> posf;            // [n]: positions rounded to FP32 (tree build)
    sts::DevBuf<int32_t> nd_cc;          // [nodes,4]: child counts by digit (scratch)
    sts::DevBuf<int32_t> nd_child;       // [nodes,4]: child id by digit (scratch)
    sts::DevBuf<int32_t> counters;       // small device counters
    int ninst = 1;                       // instances in the forest
    sts::DevBuf<int64_t> inst_off;       // [ninst + 1] instance offsets (batched builds)
    sts::DevBuf<int32_t> root_cnt, face_node;  // [20 * ninst] per (instance, face); root_cnt[20 * ninst]
                                               // is the tree build's grid-barrier counter
    sts::DevBuf<int64_t> small;          // [16] values gathered for one host read
    sts::DevBuf<int64_t> dc;             // [kDcSize] device counters
    bool capturing = false;              // recording a graph: no host reads or allocations
    bool consts_ok = false;              // icosahedron tables uploaded
    sts::Plan plan;
    // RK4 step recorded as a CUDA graph (sts_set_graph) and the arguments it was recorded for
    bool graph_on = false;
    cudaGraphExec_t rk_exec = nullptr;
    std::vector<double> rk_key;
    std::vector<int64_t> rk_off_key;
    cudaGraphExec_t ev_exec = nullptr;   // tree build + velocity recorded (sts_tree_velocity)
    unsigned long long rk_epoch = 0, ev_epoch = 0;  // g_alloc_epoch when each was recorded
    long long ev_kernels = 0, rk_kernels = 0;  // kernels per replay of each recording
    std::vector<double> ev_key;
    std::vector<int64_t> ev_off_key;
    sts::DevBuf<int32_t> leaves;         // leaf node ids in depth-first order
    sts::DevBuf<int32_t> slot_leaf;      // [n] sorted slot -> depth-first leaf index

    // ---- clusters, proxy weights ---------------------------------------------------
    int64_t nclusters = 0;
    int up_degree = -1, up_precision = -1;
    sts::DevBuf<int32_t> cluster_slot;   // per node: cluster index or -1
    sts::DevBuf<int32_t> cluster_node;   // per cluster: node id
    sts::DevBuf<int64_t> up_toff;        // [C+1] first upward task of each cluster
    sts::DevBuf<int2> up_tasks;          // (cluster, chunk start)
    int64_t n_up_tasks = 0;
    sts::DevBuf<double> up_part;         // [tasks, M] partial moments
    sts::DevBuf<double> up_frame;        // [C,12] barycentric frame of each cluster
    sts::DevBuf<float> up_frame32;       // [C,18] the frame in FP32 and the centre as FP32 hi, lo
    sts::DevBuf<double4> prx64;          // [C,M] (proxy point, 2 W)
    sts::DevBuf<float4> prx32;           // [C,M] (proxy point - c_cluster, 2 W)

    // ---- sorted particle data --------------------------------------------------------
    sts::DevBuf<double4> src64;          // [n] sorted (x, y, z, 2 w)
    sts::DevBuf<float4> src32;           // [n] sorted (x - c_leaf, 2 w)
    sts::DevBuf<int32_t> lw_terms;       // [leaves, 256 or 512] unsorted terminals of the warp traversal
    sts::DevBuf<float4> src_hl;          // [2n] sorted: hi (x, y, z, w), lo (x, y, z, 0) with x = hi + lo

    // ---- interaction lists (per leaf in depth-first order) --------------------------
    bool have_lists = false;
    double list_theta = 0.0;
    int64_t nfar = 0, nnear = 0;
    sts::DevBuf<int64_t> far_off, near_off, near_coff;  // near_coff: chunk offsets per leaf
    int64_t nnear_chunks = 0;
    sts::DevBuf<double> corr;            // [n,3] FP64 close-pair sums (sorted order)
    sts::DevBuf<int32_t> far_idx, near_idx;
    sts::DevBuf<sts::FarEntry> far_ent;
    sts::DevBuf<sts::NearEntry> near_ent;
    sts::DevBuf<int32_t> list_cnt;       // [3 * leaves * roots] scratch
    sts::DevBuf<uint8_t> wover;          // [leaves] lists left to the per-thread traversal
    sts::DevBuf<sts::Task> tasks;
    int64_t ntasks = 0;
    int list_degree = -1;                // degree the far entries' slots refer to

    // ---- dual traversal (Sec. 3.4) ---------------------------------------------------
    // Pairs (target node, source node) of the four kinds PP, PC, CP, CC, sorted by kind, target
    // key (depth-first leaf index for PP / PC, cluster slot for CP / CC), then source.  While
    // have_dual holds, the leaf lists above hold the PP (near) and PC (far) pairs of the target
    // leaves; the cluster lists below hold the CP (near) and CC (far) pairs of the target
    // clusters, whose targets are the clusters' proxy points.  Every count lives on the device
    // (dual_cnt), so the whole traversal can be recorded in a graph.
    bool have_dual = false;
    bool use_dual = false;               // sts_set_traversal: tree-code velocities by the dual traversal
    double dual_theta = 0.0;
    int64_t dual_n[4] = {-1, -1, -1, -1};  // host copies of the pair counts (-1: on the device only)
    sts::DevBuf<int32_t> dual_ft, dual_fs, dual_gt, dual_gs;  // pair frontiers (ping-pong)
    sts::DevBuf<int32_t> dual_tt, dual_ts;  // terminal pairs as found
    sts::DevBuf<uint8_t> dual_tk;           // their kinds
    sts::DevBuf<int32_t> dual_t, dual_s;    // terminal pairs sorted
    sts::DevBuf<uint32_t> dual_key, dual_ktmp;
    sts::DevBuf<int32_t> dual_perm, dual_ptmp, dual_chunk;
    sts::DevBuf<int32_t> dual_bkt, dual_bcnt;  // per pair: bucket (kind, target key); per bucket: pairs
    sts::DevBuf<int64_t> dual_boff;            // per bucket: first pair in the sorted order
    sts::DevBuf<int64_t> dual_cnt;       // counters of the traversal (layout in sts_tree.cu)
    sts::DevBuf<int64_t> dual_scan;      // chunk offsets of the sorted pairs
    sts::DevBuf<int64_t> cfar_off, cnear_off, cnear_coff;  // [C + 1] per target cluster slot
    sts::DevBuf<sts::FarEntry> cfar_ent;
    sts::DevBuf<sts::NearEntry> cnear_ent;
    sts::DevBuf<sts::Task> ctasks;
    int64_t nctasks = 0;
    sts::DevBuf<double> cvel;            // [C, M, 3] velocity at the proxy points of target clusters
    sts::DevBuf<double> ccorr;           // [C, M, 3] FP64 close-pair sums of the proxy targets
    sts::DevBuf<double> cdown;           // [C, M, 3] coefficients of the interpolating polynomials
    sts::DevBuf<float> cdown32;          // [C, M, 4] FP32 coefficients, one float4 per basis function (mixed)
    sts::DevBuf<uint8_t> chas;           // [C] the cluster is the target of CP or CC pairs
    sts::DevBuf<uint8_t> cacc;           // [C] the cluster holds an interpolant (its own or an ancestor's)
    sts::DevBuf<int32_t> leaf_anc;       // [L, A] per leaf: count, then its ancestor clusters with CP / CC pairs

    // ---- adaptive mesh refinement (Appendix A) -----------------------------------------
    sts::AmrState* amr = nullptr;

    // ---- direct sum scratch ------------------------------------------------------------
    sts::DevBuf<double4> dsrc64;
    sts::DevBuf<float4> dsrc32;          // [2n]: hi (x, y, z, 2w), lo (x, y, z, 0)
    sts::DevBuf<double> dpart;           // [splits, nt, 3]

    // ---- RK4 scratch -------------------------------------------------------------------
    sts::DevBuf<double> rk_x0, rk_z0, rk_xs, rk_zs, rk_k, rk_ksum;
    sts::DevBuf<double> rk_zf;           // [n] forced source vorticity zeta - F_R (Sec. 4.4)

    // ---- stats and phase timing -------------------------------------------------------
    sts::DevBuf<unsigned long long> d_stats;  // [2] PC, PP interactions
    sts::DevBuf<int64_t> d_work;              // [nleaves] per-leaf interactions (sts_leaf_work)
    sts::DevBuf<double> prx_rd;               // [clusters, M] rho_m^d of each proxy point
    sts::DevBuf<int64_t> scan_state;          // single-pass scan state of the main stream
    sts::DevBuf<int64_t> scan_state_side;     // ... of the side stream (lists)
    sts::DevBuf<int64_t> bld_tot;             // [CTAs] children per CTA of the level build
    int build_grid = 0;                       // CTAs of the level build (all resident)
    int64_t node_hint = 0;                    // node capacity that an eager build starts from
    int64_t up_tasks_rec = 0;                 // moment tasks a recorded step provides for
    int64_t nodes_rec = 0;                    // nodes (and clusters) a recorded step provides for
    bool timing = false;
    cudaEvent_t ev[sts::kNumPhases][2] = {};
    float phase_ms[sts::kNumPhases] = {};
    int phase_count[sts::kNumPhases] = {};
    bool phase_open[sts::kNumPhases] = {};
    bool phase_in_graph[sts::kNumPhases] = {};  // phases recorded inside the current graphs

    std::vector<sts::RefTable*> refs;    // by degree

    // ---- the lists' side stream --------------------------------------------------------
    // The interaction lists and the sources / proxy weights depend only on the tree, so the
    // lists are built on a stream of their own, forked from and joined back to the caller's
    // stream by events (graph recordings included).
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaEvent_t ev_tree = nullptr;  // recorded when the tree (not yet the sorted order) is built
    bool tree_event = false;        // ev_tree recorded by the last build, not yet waited on
    ~sts_ctx();
};

namespace sts {

// ---- host tables (sts_tables.cu) --------------------------------------------------
void icosahedron(double V[12][3], int F[20][3], double C[20][3]);
int build_ref_table(int d, RefTable* t);
RefTable* get_ref(sts_ctx* ctx, int d);
// The contraction sum_k omega_k Vinv[k][m] of the upward pass on the tensor cores, for the
// clusters of the current tree (counted on the device, at most nclu) into wout[cluster, M].
bool proxy_weights_tc_supported(int degree);
int proxy_weights_tc(sts_ctx* c, const RefTable* ref, int degree, int64_t nclu, cudaStream_t s);
// The dual traversal's mixed-precision interpolation coefficients c = V_ref^-1 diag(rho^d) U on
// the tensor cores, for the clusters with CP / CC pairs (chas), cvel[cluster, M, 3] ->
// coef32[cluster, M] as float4 (x, y, z, unused).
int cluster_coef_tc(sts_ctx* c, const RefTable* ref, int degree, int64_t nclu, const double* cvel, float* coef32,
                    cudaStream_t s);

// ---- scans (sts_scan.cu) ----------------------------------------------------------
int64_t scan_scratch(int64_t n);
// out[i] = sum_{j < i} in[j] for i in [0, n]; out[n] is the total: one single-pass launch.
// state: the scan state of the stream it runs on (scans on one state run one after another),
// at least scan_state_size(n) int64 and zero when allocated (scan_state_reserve); a
// look-back that gives up sets STS_ERR_TIMEOUT in *status.  n_dev: optional device count
// (then n is its upper bound, used to size the grid).
int64_t scan_state_size(int64_t n);
int scan_state_reserve(DevBuf<int64_t>& state, int64_t n, cudaStream_t s);
void exclusive_scan_i32(const int32_t* in, int64_t* out, int64_t n, DevBuf<int64_t>& state, cudaStream_t s,
                        const int* status, const int64_t* n_dev = nullptr);

// ---- tree and lists (sts_tree.cu) ----------------------------------------------------
// inst_off: device offsets [ninst + 1] of the instances (NULL: one instance)
int tree_build(sts_ctx* ctx, const double* pos, int64_t n, const int64_t* inst_off, int ninst,
               int leaf_size, int max_level, cudaStream_t s);
int build_lists(sts_ctx* ctx, double theta, cudaStream_t s);
// Dual traversal (Sec. 3.4): the four pair lists, the leaf lists of PP and PC pairs with the
// leaves' evaluation tasks, and the cluster lists of CP and CC pairs.  Eager: synchronises `s`
// once (counts and overflow; buffers grown and the traversal redone on overflow).  Recording:
// no host access; an overflow sets bit 4 of the device overflow word.
int build_dual(sts_ctx* ctx, double theta, cudaStream_t s);
// Buffers of the dual traversal for recording it (the plan's sizes with slack).
int reserve_dual_for_capture(sts_ctx* ctx, int degree, cudaStream_t s);
// Host copies of the dual pair counts after a recorded step ran.
int refresh_dual_counts(sts_ctx* ctx, cudaStream_t s);

// ---- adaptive mesh refinement (sts_amr.cu) -------------------------------------------------
void amr_free(AmrState* m);
int amr_init(sts_ctx* c, const int32_t* faces, int64_t t0, int64_t n0, const double* pos0, const double* zeta0,
             int levels, cudaStream_t s);
int amr_step(sts_ctx* c, double eps1, double eps2, int64_t* counts, cudaStream_t s);
int amr_gather(sts_ctx* c, double* pos, double* zeta, double* area, int64_t* ids, cudaStream_t s);
int amr_scatter(sts_ctx* c, const double* pos, const double* zeta, cudaStream_t s);
int amr_info(sts_ctx* c, int64_t* info);
int amr_export(sts_ctx* c, int32_t* tv, int32_t* tparent, int32_t* tchild, int8_t* tlevel, int32_t* vparent,
               uint8_t* tstate, uint8_t* valive, double* pos, double* zeta, double* area, cudaStream_t s);
// Pair counts of the dual lists: stats[0..3] = PP pairs (j != i), PC, CP, CC interactions.
int dual_stats(sts_ctx* ctx, int degree, int64_t* stats, cudaStream_t s);
// Evaluation tasks of the clusters that are targets of CP or CC pairs, and their has flags;
// cluster_task_count: the device count of those tasks.
int cluster_tasks(sts_ctx* ctx, int M, cudaStream_t s);
const int64_t* cluster_task_count(sts_ctx* ctx);
// Sorted pairs of one kind (0 PP, 1 PC, 2 CP, 3 CC) to host arrays (either may be NULL).
int dual_export(sts_ctx* ctx, int kind, int64_t* npairs, int32_t* tgt, int32_t* src, cudaStream_t s);
// node-table capacity (contents are not kept)
int reserve_tree_nodes(sts_ctx* ctx, int64_t nodes, cudaStream_t s);
// out[0..3] = *a, *b, *c, *d (0 for NULL), out[4] = status word: one host read for all.
void gather_values(const int64_t* a, const int64_t* b, const int64_t* c, const int64_t* d,
                   const int* status, int64_t* out, cudaStream_t s);

// ---- sorted sources and upward pass (sts_upward.cu; the cluster table, its moment tasks
// and frames are made by tree_build) ---------------------------------------------------
int prepare_sources(sts_ctx* ctx, const double* zeta, const double* area, cudaStream_t s);
int upward_pass(sts_ctx* ctx, int degree, int precision, cudaStream_t s);
int fill_far_slots(sts_ctx* ctx, cudaStream_t s);

// ---- evaluation (sts_eval.cu) ---------------------------------------------------------
int evaluate(sts_ctx* ctx, int degree, int precision, double tau, double* vel, cudaStream_t s);
// One list set for the evaluation kernels: the leaf lists (targets: the sorted particles,
// results to vel in the caller's order) or the cluster lists of the dual traversal (targets:
// the proxy points of the target clusters, results in proxy order).
struct ListSet {
    const Task* tasks;
    const int64_t* ntasks_d;
    int64_t ntasks;
    const int64_t *far_off, *near_coff;
    const FarEntry* far_ent;
    const NearEntry* near_ent;
    const float4* tgt32;
    const double4* tgt64;
    const int32_t* perm;  // target slot -> output row, or nullptr for the identity
    int64_t ntargets;     // rows of corr
    // only the tasks of leaves [leaf_lo, leaf_hi); out_base >= 0: target slot t goes to output
    // row t - out_base (sorted order) instead of perm[t]
    int64_t leaf_lo = 0, leaf_hi = INT64_MAX, out_base = -1;
};
// The mixed or FP64 evaluation kernel over one list set; corrbuf: the FP64 close-pair scratch
// (grown to 3 * ls.ntargets doubles eagerly); phase: the timed phase (-1: inside the caller's).
int evaluate_lists(sts_ctx* ctx, const ListSet& ls, int degree, int precision, double tau, DevBuf<double>& corrbuf,
                   double* vel, cudaStream_t s, int phase = kPhEval);

int direct_potential(sts_ctx* c, const double* pos, const double* zeta, const double* area, int64_t n,
                     double* psi, cudaStream_t s);
int evaluate_potential(sts_ctx* c, int degree, int precision, double tau, double* psi, cudaStream_t s);
int wait_selftest(sts_ctx* c, int spins, cudaStream_t s);
// The evaluation of the targets of depth-first leaves [leaf_lo, leaf_hi) only (lists, sources
// and proxy weights already in place); out_base >= 0: sorted-slot rows t - out_base.
int evaluate_range(sts_ctx* c, int degree, int precision, double tau, int64_t leaf_lo, int64_t leaf_hi,
                   int64_t out_base, double* vel, cudaStream_t s);
// Per-leaf PC + PP interactions of the current lists into host work[nleaves] (synchronises).
int leaf_work(sts_ctx* c, int degree, int64_t* work, cudaStream_t s);
// vel[perm[t]] = vs[t] for every sorted slot t.
int unpermute(sts_ctx* c, const double* vs, double* vel, cudaStream_t s);
int count_interactions(sts_ctx* ctx, int degree, cudaStream_t s);
int direct_sum(sts_ctx* ctx, const double* pos, const double* zeta, const double* area,
               int64_t n, const int64_t* targets, int64_t nt, int precision, double* vel,
               cudaStream_t s);


// ---- dual traversal: CP / CC evaluation and the downward pass (sts_down.cu) -----------
// Dual-traversal velocity: PP and PC at the particles of the target leaves, CP and CC at the
// proxy points of the target clusters, then the interpolating polynomial of every target
// cluster evaluated at its particles and added (Sec. 3.3, 3.4).
int evaluate_dual(sts_ctx* ctx, int degree, int precision, double tau, double* vel, cudaStream_t s);

// ---- RK4 (sts_rk4.cu) -----------------------------------------------------------------
double forcing_ramp(double t, double Tp, double Tf);
void forced_source(const double* xs, const double* zs, int64_t n, const sts_forcing* f, double t, double* zf,
                   cudaStream_t s);
void rk4_stage(const double* x0, const double* z0, const double* k, double cdt, double Omega,
               double* xs, double* zs, double* ksum, double b, int first, int64_t n,
               cudaStream_t s);
void rk4_final(double* x, double* z, const double* x0, const double* z0, const double* ksum,
               const double* k4, double dt, double Omega, int64_t n, cudaStream_t s);

// ---- phase timing (sts_api.cu) -----------------------------------------------------------
void phase_begin(sts_ctx* ctx, int ph, cudaStream_t s);
void phase_end(sts_ctx* ctx, int ph, cudaStream_t s);

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }
inline int nbasis(int d) { return (d + 1) * (d + 2) / 2; }

}  // namespace sts

#define STS_CUDA(call)                                                                    \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            sts::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),        \
                           __FILE__, __LINE__);                                           \
            return STS_ERR_CUDA;                                                          \
        }                                                                                 \
    } while (0)

#define STS_LAUNCH_CHECK()                                                                \
    do {                                                                                  \
        cudaError_t e_ = cudaGetLastError();                                              \
        if (e_ != cudaSuccess) {                                                          \
            sts::set_error("kernel launch failed: %s (%s:%d)", cudaGetErrorString(e_),    \
                           __FILE__, __LINE__);                                           \
            return STS_ERR_CUDA;                                                          \
        }                                                                                 \
    } while (0)
