/*
 * sts.h -- C ABI of the GB300 spherical tree summation library (libsts.so).
 *
 * The library evaluates the velocity of the Lagrangian barotropic-vorticity particle system
 * of Chen & Jablonowski, "Fast Summation on the Sphere with Applications to the Barotropic
 * Vorticity Equation" (arXiv 2401.07361), Sec. 2 (midpoint-rule discretisation):
 *
 *     u(x_i) = -(1/4pi) sum_{j != i} (x_i x x_j) zeta_j A_j / (1 - x_i . x_j)
 *
 * with 1 - x.y evaluated as |x - y|^2 / 2 (Sec. 2, Eq. altkernel), either directly (O(N^2))
 * or with the spherical tree code of Sec. 3: an icosahedral triangle tree, SBB
 * interpolation at approximate Fekete proxy points (Sec. 3.2, 3.3.2) and the MAC
 * (r_t + r_s) / R < theta (Sec. 3.4).  bve_rk4_step advances the particles with classical
 * RK4 (Sec. 4), dzeta_i/dt = -2 Omega u_z,i.
 *
 * Conventions shared by every entry point:
 *   - Array arguments are DEVICE pointers owned by the caller, contiguous, FP64 unless
 *     stated (the export calls take HOST pointers, as stated there).  Positions are
 *     row-major [n, 3] (x, y, z of particle i at 3i .. 3i+2), points on the unit sphere.
 *     Velocities are written row-major [n, 3] in the caller's particle order.  The library
 *     never frees or retains caller memory beyond the call.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Work is
 *     enqueued on it.  Calls that say "synchronises" wait for `stream` before returning.
 *   - Return value: STS_OK (0) or a negative STS_ERR_* code; sts_last_error() then holds a
 *     one-line message for the calling thread.  No exception crosses the ABI.  Arguments
 *     are checked on the host before anything is enqueued.
 *   - A context (sts_ctx) owns every scratch buffer (tree, lists, proxy weights, staging
 *     copies) on the device that was current at sts_create; it grows them with cudaMalloc
 *     on demand and frees them in sts_destroy.  One context must not be used by two host
 *     threads at once, and calls on one context must not overlap on the GPU (different
 *     streams without ordering race on its scratch).
 *   - n is limited to 2^31 - 2 particles.
 */
#ifndef STS_H
#define STS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define STS_OK 0
#define STS_ERR_ARG (-1)       /* invalid argument (checked on the host before launch)  */
#define STS_ERR_CUDA (-2)      /* a CUDA runtime call or kernel launch failed          */
#define STS_ERR_CAPACITY (-3)  /* a device-side capacity was exceeded                  */
#define STS_ERR_TIMEOUT (-4)   /* a bounded device-side wait gave up                   */
#define STS_ERR_NONFINITE (-5) /* non-finite position                                  */
#define STS_ERR_STATE (-6)     /* call order violated (e.g. velocity before a tree)    */

#define STS_FP64 0  /* every pair term in FP64                                          */
#define STS_MIXED 1 /* FP32 pair terms on leaf-local coordinates with compensated sums;
                       FP64 positions, tree geometry, proxy contraction and near pairs
                       with |x - y|^2 / 2 < near_fp64_tau                                */

/* Tree-code parameters (Sec. 3.4): theta in (0, 1) is the MAC parameter; degree in [1, 16]
 * the SBB interpolation degree d (M = (d + 1)(d + 2) / 2 proxy points per cluster);
 * leaf_size >= 1 the threshold N_T (a triangle with more than N_T particles is refined, and
 * a source triangle with more than N_T particles that passes the MAC is a cluster);
 * max_level in [0, 24] the depth limit; precision STS_FP64 or STS_MIXED;
 * near_fp64_tau >= 0 (STS_MIXED only): near pairs with |x - y|^2 / 2 < tau are evaluated in
 * FP64 (0 disables).                                                                       */
typedef struct sts_params {
    double theta;
    int32_t degree;
    int32_t leaf_size;
    int32_t max_level;
    int32_t precision;
    double near_fp64_tau;
} sts_params;

/* Vorticity forcing of Sec. 4.4 (the polar-vortex experiment): the Biot-Savart source of
 * every RK4 stage becomes (zeta - F_R(x, t)) A with
 *   F_R = amplitude k^2 A(t) B(theta) cos(k phi),
 *   A(t) = half-cosine ramp up over [0, Tp), 1 until Tf - Tp, ramp down until Tf, 0 after,
 *   B(theta) = r exp(1 - r), r = tan^2 theta1 / tan^2 theta for latitude theta > 0, else 0,
 * phi the longitude.  The paper's values: amplitude = (3/5) Omega, Tp = 4, Tf = 15 (days),
 * theta1 = pi / 3, k = 1 or 2.  The particle vorticity itself still follows
 * dzeta/dt = -2 Omega dz/dt. */
typedef struct {
    int32_t k;        /* zonal wavenumber, >= 1 */
    int32_t reserved; /* 0 */
    double amplitude; /* factor in front of k^2 A(t) B cos(k phi) */
    double Tp, Tf;    /* ramp length and end of the forcing, in the time unit of dt */
    double theta1;    /* latitude of maximum forcing (radians, in (0, pi/2)) */
} sts_forcing;

typedef struct sts_ctx sts_ctx;

/* Creates an empty context on the current device.  *out is set only on success. */
int sts_create(sts_ctx** out);
/* Synchronises the device and frees every buffer of the context.  NULL is a no-op. */
void sts_destroy(sts_ctx* ctx);
/* Message of the calling thread's last error ("" if none).  Never NULL. */
const char* sts_last_error(void);
/* Synchronises `stream`, returns STS_OK or the error recorded in the context's device
 * status word (STS_ERR_CAPACITY, STS_ERR_NONFINITE, STS_ERR_TIMEOUT: the mixed evaluation
 * gave up waiting for a staged source block, so that launch's velocities are incomplete),
 * and clears the word. */
int sts_status(sts_ctx* ctx, void* stream);
/* Self-test of the bounded device-side wait that the mixed evaluation uses while its sources
 * are staged: one warp waits on a shared-memory mbarrier that nothing arrives on, polling it
 * `spins` times (1 <= spins <= 2^20; the evaluation polls 2^20 times), then flags a timeout.
 * Returns STS_ERR_TIMEOUT (the expected result, from sts_status on `stream`) and leaves the
 * context usable; STS_ERR_ARG for spins out of range.  The paper has no counterpart: this
 * exists so that the timeout path can be exercised without faulting or hanging the GPU. */
int sts_selftest_wait(sts_ctx* ctx, int32_t spins, void* stream);

/* Direct summation of the Sec. 2 system (the O(N^2) sum of Sec. 4.1).
 * pos[n,3], zeta[n], area[n] in; vel[n,3] out (u_i at every particle; j = i and any other
 * particle at exactly the same position contribute nothing).  precision: STS_FP64, or
 * STS_MIXED (FP32 pair terms on positions carried as FP32 hi + lo pairs, compensated
 * sums).  n = 0 writes nothing; n = 1 writes zeros. */
int sts_direct(sts_ctx* ctx, const double* pos, const double* zeta, const double* area,
               int64_t n, int32_t precision, double* vel, void* stream);

/* Direct summation of the stream function psi_i = -(1/4 pi) sum_{j != i} log(|x_i - x_j|^2
 * / 2) zeta_j A_j (Sec. 2 Green's function, Sec. 3 convolution sum): pos[n,3], zeta[n],
 * area[n] in, psi[n] out; a distinct particle at the same position adds nothing.  Only
 * precision = STS_FP64 is implemented (STS_ERR_ARG otherwise).  Asynchronous on `stream`. */
int sts_direct_potential(sts_ctx* ctx, const double* pos, const double* zeta, const double* area,
                         int64_t n, int32_t precision, double* psi, void* stream);

/* Direct summation at nt targets: targets[nt] (device, int64 original indices in [0, n)),
 * vel[nt,3] out (row t = velocity of particle targets[t]).  Same arithmetic as
 * sts_direct.  Target indices are not range-checked on the device: the caller keeps them
 * in [0, n). */
int sts_direct_targets(sts_ctx* ctx, const double* pos, const double* zeta,
                       const double* area, int64_t n, const int64_t* targets, int64_t nt,
                       int32_t precision, double* vel, void* stream);

/* Direct sum like sts_direct, for callers that cannot allocate device memory when they
 * need the result: code recording into a CUDA graph it does not own, processes whose device
 * memory belongs to another allocator, and loops that must not enter cudaMalloc/cudaFree
 * (which can synchronise the device and take unbounded time) after start-up.  The paper has
 * no counterpart; this is a library facility.  Takes no context and allocates nothing: its
 * scratch is one fixed device array of about 7.4 MB inside the library, held on every GPU
 * that loads the library until the process exits.  n is limited to 65536 (larger n returns
 * STS_ERR_CAPACITY without touching the GPU).  The first call on a device looks up that
 * array's device address, so make it before any stream capture; the address is then kept
 * for the life of the process, so after a cudaDeviceReset (or any other teardown of the
 * device's primary context) this entry point must not be called again in that process.
 * All calls share the array: calls that overlap on the GPU race; order them on one stream.
 * Results equal sts_direct's bit for bit for the same inputs and precision (same source
 * split, same kernels). */
int sts_direct_noalloc(const double* pos, const double* zeta, const double* area, int64_t n,
                       int32_t precision, double* vel, void* stream);

/* Builds the icosahedral triangle tree of Sec. 3 over pos[n,3] (copied into the context):
 * each particle is assigned to one of the 20 faces, and every triangle holding more than
 * p->leaf_size particles below p->max_level is split into its four children.  Particles
 * keep their original relative order inside every leaf.  Uses p->leaf_size and
 * p->max_level; the other fields are checked but not used.  Synchronises `stream` once (it
 * reads the node, leaf and cluster counts after the build, which runs as one cooperative
 * launch; if the node table it started with ran out, it is enlarged to the proven bound and
 * the build redone).  STS_ERR_TIMEOUT if a grid-wide barrier of that launch gave up.
 * Replaces any previous tree of the context. */
int sts_tree_build(sts_ctx* ctx, const double* pos, int64_t n, const sts_params* p,
                   void* stream);

/* Batched build: ninst independent instances (separate particle sets on the unit sphere,
 * each with its own icosahedral tree of Sec. 3.1) concatenated in pos[n,3], instance b
 * holding particles offsets[b] .. offsets[b+1] - 1 (offsets: HOST array of ninst + 1
 * non-decreasing values, offsets[0] = 0, n = offsets[ninst]; empty instances allowed).  The
 * trees form one forest whose roots are keyed (instance, face) = 20 b + f; every level of
 * every instance is built by the same launches, and sts_velocity then evaluates all
 * instances in one launch over their combined leaf tasks, each target interacting only with
 * its own instance.  Each instance's velocities are those of sts_tree_build + sts_velocity
 * on that instance alone.  Synchronises `stream`. */
int sts_tree_build_batched(sts_ctx* ctx, const double* pos, const int64_t* offsets,
                           int32_t ninst, const sts_params* p, void* stream);

/* Tree-code velocity (Sec. 3.3 PC + PP interactions over MAC interaction lists, Sec. 3.4)
 * for the tree last built in ctx: zeta[n], area[n] in, vel[n,3] out in the caller's
 * order.  Uses p->theta, p->degree, p->precision and p->near_fp64_tau; the tree's own
 * leaf_size and max_level apply.  Builds the proxy weights (upward pass) on every call and
 * the interaction lists when theta or the tree changed; synchronises `stream` in that
 * case (list sizes are read back).  STS_ERR_STATE without a tree. */
int sts_velocity(sts_ctx* ctx, const double* zeta, const double* area, const sts_params* p,
                 double* vel, void* stream);

/* Tree-code stream function (the convolution of Sec. 3 with the Green's function of Sec. 2,
 * G(x, y) = -(1/4 pi) log(1 - x.y), written as -(1/4 pi) log(|x - y|^2 / 2)):
 * psi_i = sum_{j != i} G(x_i, x_j) zeta_j A_j over the same PC + PP lists and proxy weights as
 * sts_velocity (the weights do not depend on the kernel).  zeta[n], area[n] in, psi[n] out in
 * the caller's order; a distinct particle at a target's position adds nothing.  With this G,
 * u = grad psi x x is the velocity of sts_velocity and Lap psi = -zeta for zero-mean zeta.
 * p->precision: STS_FP64, or STS_MIXED: FP32 log terms (log2 of |d|^2 / 2 on leaf-local
 * coordinates, as the velocity's pair terms) summed per target in TwoSum-compensated FP32
 * pairs, the pairs closer than p->near_fp64_tau in FP64, ln 2 and the sum scaled in FP64 (the
 * log terms of a zero-mean vorticity cancel by ~100, which plain FP32 sums would not
 * survive).  STS_ERR_STATE without a tree.  Synchronises `stream` when the lists are
 * (re)built. */
int sts_potential(sts_ctx* ctx, const double* zeta, const double* area, const sts_params* p,
                  double* psi, void* stream);

/* Tree-code velocity by the dual tree traversal of Sec. 3.4 with all four interactions of
 * Sec. 3.3, for the tree last built in ctx: zeta[n], area[n] in, vel[n,3] out in the caller's
 * order.  From every pair of roots of an instance, a pair of triangles (T_t, T_s) that passes
 * the MAC interacts by its particle counts against N_T = leaf_size: PP (both at most N_T, the
 * particle sum), PC (only the source above: the target particles against the source's proxy
 * points and weights), CP (only the target above: the source particles summed at the target's
 * proxy points), CC (both above: proxy points against proxy points).  A pair that fails the
 * MAC is PP when both are leaves; otherwise the triangle holding more particles (the target
 * on a tie; a leaf never) is replaced by its children.  CP and CC give the kernel sum S (the
 * velocity is -(1/4 pi) x x S) at the target cluster's proxy points; the polynomial of degree
 * d interpolating it over the cluster (solve V_T c = U_T, V_T[m][k] = B_k(b(x~_m))) is
 * evaluated at every particle x below it, and -(1/4 pi) x x (that value) is added, so the
 * velocity stays tangent to the sphere.  Uses p->theta, p->degree, p->precision and
 * p->near_fp64_tau.  Mixed precision: the pair sums in FP32 as in sts_velocity, the
 * coefficients c in FP64, rounded to FP32 for the evaluation at the particles.  Builds the pair lists when
 * theta or the tree changed (synchronises `stream` once), which replaces the lists of
 * sts_velocity (the next sts_velocity rebuilds them).  STS_ERR_STATE without a tree. */
int sts_velocity_dual(sts_ctx* ctx, const double* zeta, const double* area, const sts_params* p,
                      double* vel, void* stream);

/* One GPU's share of a sharded tree-code velocity (Sec. 4.1 spreads the same convolution over
 * MPI ranks; here each GPU builds the whole tree and evaluates a contiguous range of target
 * leaves).  Evaluates sts_velocity's PC + PP sums (Sec. 3.3, lists of Sec. 3.4; same sources,
 * proxy weights, lists and arithmetic, so every row written is bit-identical to
 * sts_velocity's) for the targets of depth-first leaves [leaf_begin, leaf_end) only, 0 <=
 * leaf_begin <= leaf_end <= the tree's leaf count (sts_tree_info info[2]).  out_sorted = 0:
 * rows vel[i,3] in the caller's order, rows of other targets left untouched; out_sorted = 1:
 * vel[(slot_end - slot_begin), 3], row r = the target in sorted slot slot_begin + r
 * (sts_leaf_range), the compact block that GPUs all-gather and sts_unpermute puts back in
 * order.  Uses the target-leaf lists only (STS_ERR_STATE after sts_set_traversal(ctx, 1) or
 * while recording); builds the lists when theta or the tree changed (an empty range with
 * vel = NULL only builds them).  Synchronises `stream` (it reads the leaf count, and the slot
 * range when out_sorted = 1). */
int sts_velocity_range(sts_ctx* ctx, const double* zeta, const double* area, const sts_params* p,
                       int64_t leaf_begin, int64_t leaf_end, int32_t out_sorted, double* vel,
                       void* stream);

/* Work of each depth-first target leaf under the current target-leaf lists: work[nleaves]
 * (HOST int64 array, nleaves = sts_tree_info info[2]) = the leaf's targets x (its far
 * clusters x M + the particles of its near leaves), i.e. its PC + PP interactions at degree
 * `degree` (M = (d + 1)(d + 2) / 2), the cost a partition of the leaves between GPUs
 * balances.  STS_ERR_STATE without lists (call sts_velocity or sts_velocity_range first).
 * Synchronises `stream`. */
int sts_leaf_work(sts_ctx* ctx, int32_t degree, int64_t* work, void* stream);

/* The sorted slots [*slot_begin, *slot_end) holding the targets of depth-first leaves
 * [leaf_begin, leaf_end) (leaves own consecutive slots in depth-first order).  Synchronises
 * `stream`.  STS_ERR_ARG for a range outside [0, leaf count]. */
int sts_leaf_range(sts_ctx* ctx, int64_t leaf_begin, int64_t leaf_end, int64_t* slot_begin,
                   int64_t* slot_end, void* stream);

/* Puts rows in sorted slot order back into the caller's order: vel[perm[t], :] =
 * vel_sorted[t, :] for t < n (device arrays [n,3]; perm the current tree's slot -> particle
 * map).  Asynchronous on `stream`.  STS_ERR_STATE without a tree. */
int sts_unpermute(sts_ctx* ctx, const double* vel_sorted, double* vel, void* stream);

/* One classical RK4 step (Sec. 4) of the Sec. 2 system dx_i/dt = u_i,
 * dzeta_i/dt = -2 Omega u_z,i, in place on pos[n,3] and zeta[n]; area[n] is constant.
 * Every stage evaluates the tree-code velocity (parameters p, tree rebuilt) at the stage
 * positions (projected to the unit sphere) with the stage vorticities; the new positions
 * are projected to the sphere.  Leaves the tree of the last stage in ctx.  Synchronises
 * `stream`. */
int bve_rk4_step(sts_ctx* ctx, double* pos, double* zeta, const double* area, int64_t n,
                 double dt, double Omega, const sts_params* p, void* stream);

/* bve_rk4_step of the forced system of Sec. 4.4: the step starts at time t; stage k of the
 * step sees the forcing at t, t + dt/2, t + dt/2, t + dt.  The step runs eagerly (it is not
 * recorded as a graph: its stage times change from step to step).  STS_ERR_ARG for a NULL
 * forcing, k < 1, Tp <= 0, Tf < 2 Tp, theta1 outside (0, pi/2) or non-finite values. */
int bve_rk4_step_forced(sts_ctx* ctx, double* pos, double* zeta, const double* area, int64_t n, double t,
                        double dt, double Omega, const sts_forcing* forcing, const sts_params* p,
                        void* stream);

/* ---- adaptive mesh refinement (Appendix A) -------------------------------------------- */
/* The particles are the vertices of a triangulation of the sphere (the refined icosahedron):
 * faces[nfaces,3] (HOST, vertex indices in [0, n0)) over the base particles pos0[n0,3],
 * zeta0[n0] (device).  A leaf triangle splits into four (v1, m12, m31), (m12, v2, m23),
 * (m31, m23, v3), (m12, m23, m31) when the magnitude of its circulation |A (z1 + z2 + z3) / 3|
 * >= eps1 or its vorticity variation max z - min z >= eps2, at most `levels` (<= 6) times
 * below the base mesh; four leaf children merge back when neither criterion holds on their
 * parent's corners and none of them splits.  A is the spherical area of the triangle of the
 * current corner positions.  Every triangle and vertex the refinement can create is numbered
 * once here: level by level, each triangle of the previous level in order gives the midpoints
 * of its edges (v1 v2), (v2 v3), (v3 v1), numbered when first met.  Vertex v < n0 is base
 * particle v.  A new midpoint is placed at unit(p_a + p_b) of its edge ends' current positions
 * with vorticity (z_a + z_b) / 2.  The particles are the corners of leaf triangles, weighted by
 * the sum of A / 3 over them.  Synchronises `stream`.  The mesh lives in ctx until the next
 * sts_amr_init or sts_destroy. */
int sts_amr_init(sts_ctx* ctx, const int32_t* faces, int64_t nfaces, int64_t n0, const double* pos0,
                 const double* zeta0, int32_t levels, void* stream);
/* One refinement pass (every decision on the state at the start of the pass).  counts (HOST,
 * may be NULL) [4] = {splits, merges, particles, leaf triangles}.  Synchronises `stream`. */
int sts_amr_step(sts_ctx* ctx, double eps1, double eps2, int64_t* counts, void* stream);
/* info (HOST) [5] = {base vertices, possible vertices, base triangles, possible triangles,
 * particles}. */
int sts_amr_info(sts_ctx* ctx, int64_t* info);
/* The particles in vertex order (device outputs, any may be NULL): pos[np,3], zeta[np],
 * area[np] (the weights) and ids[np] (their vertex numbers), np = info[4]. */
int sts_amr_gather(sts_ctx* ctx, double* pos, double* zeta, double* area, int64_t* ids, void* stream);
/* Writes back the particles' positions and vorticities (device, in the order of
 * sts_amr_gather) and recomputes the weights.  Synchronises `stream`. */
int sts_amr_scatter(sts_ctx* ctx, const double* pos, const double* zeta, void* stream);
/* The whole mesh (HOST outputs, any may be NULL): per possible triangle corners tv[nt,3],
 * parent, first child (-1 at the deepest level), level (0 = base), state (0 absent, 1 leaf,
 * 2 split); per possible vertex the edge ends vparent[nv,2] (-1 for base vertices), alive
 * flag, pos[nv,3], zeta[nv], area[nv] (zeros where not alive). */
int sts_amr_export(sts_ctx* ctx, int32_t* tv, int32_t* tparent, int32_t* tchild, int8_t* tlevel,
                   int32_t* vparent, uint8_t* tstate, uint8_t* valive, double* pos, double* zeta,
                   double* area, void* stream);

/* One RK4 step of ninst independent instances (offsets as in sts_tree_build_batched), in
 * place on pos[n,3] and zeta[n]; every stage builds the forest and evaluates all instances
 * together.  Synchronises `stream`. */
int bve_rk4_step_batched(sts_ctx* ctx, double* pos, double* zeta, const double* area,
                         const int64_t* offsets, int32_t ninst, double dt, double Omega,
                         const sts_params* p, void* stream);

/* Tree build and tree-code velocity in one call (sts_tree_build_batched + sts_velocity):
 * pos[n,3], zeta[n], area[n], HOST offsets[ninst + 1] of the instances (ninst = 1 and
 * offsets = {0, n} for one instance), vel[n,3] out.  With sts_set_graph(ctx, 1) the call is
 * recorded as one CUDA graph and replayed on later calls with the same arguments, with the
 * same capacity planning and eager redo on overflow as the RK4 step. */
int sts_tree_velocity(sts_ctx* ctx, const double* pos, const double* zeta, const double* area,
                      const int64_t* offsets, int32_t ninst, const sts_params* p, double* vel,
                      void* stream);

/* on != 0: bve_rk4_step, bve_rk4_step_batched and sts_tree_velocity run as recorded CUDA
 * graphs.  For the RK4 step:
 * The first step (and any step whose arguments -- array pointers, n, offsets, dt, Omega,
 * parameters, stream -- differ from the recorded ones) runs eagerly, which sizes the
 * buffers (the largest tree, lists and task counts of its four stages, plus 25%), and then
 * records one step without running it; the next calls replay the recording with no host
 * synchronisation inside the step.  After a replay the host reads one overflow word: if the
 * tree needed more levels or any list outgrew its recorded capacity, the step is undone
 * from its saved start state and redone eagerly, and a new recording is made.  Recording
 * needs a non-default stream.  on = 0 drops the recording. */
int sts_set_graph(sts_ctx* ctx, int32_t on);

/* ---- inspection (HOST output buffers; every call synchronises `stream`) -------------- */
/* info[8] = {n, nodes, leaves, deepest level, far entries, near entries, clusters,
 * evaluation tasks}; the list counts are 0 before the first sts_velocity. */
int sts_tree_info(sts_ctx* ctx, int64_t* info, void* stream);
/* Node table in node order (level by level, key order within a level).  Any pointer may
 * be NULL.  perm[n]: sorted slot -> original index; per node: level, key (face index, then
 * two bits per level), parent (-1 for roots), first_child (-1 if none), nchild, start and
 * count (slot range), leaf flag, geom[13] = v1, v2, v3, circumcentre c, chord radius r;
 * leaves[leaves]: leaf node ids in depth-first order. */
int sts_tree_export(sts_ctx* ctx, int64_t* perm, int32_t* level, uint64_t* key,
                    int32_t* parent, int32_t* first_child, int32_t* nchild, int64_t* start,
                    int64_t* count, int32_t* leaf, int32_t* leaves, double* geom,
                    void* stream);
/* Interaction lists of the last sts_velocity, per leaf in depth-first order (CSR):
 * far_off[leaves+1], far_idx[far entries] (cluster node ids), near_off[leaves+1],
 * near_idx[near entries] (source node ids).  Any pointer may be NULL. */
int sts_lists_export(sts_ctx* ctx, int64_t* far_off, int32_t* far_idx, int64_t* near_off,
                     int32_t* near_idx, void* stream);
/* Clusters of the last sts_velocity in node order: node_ids[C], proxy points yt[C,M,3] and
 * proxy weights W[C,M] (FP64 values as the evaluation uses them).  Any pointer may be NULL. */
int sts_clusters_export(sts_ctx* ctx, int32_t* node_ids, double* yt, double* W, void* stream);
/* dual != 0: sts_velocity, sts_tree_velocity and the RK4 steps compute the tree-code
 * velocity by the dual traversal of sts_velocity_dual (all four interactions); 0 (the default):
 * by the target-leaf lists (PC + PP).  Graph recordings are keyed by this choice.  sts_potential
 * always uses the target-leaf lists. */
int sts_set_traversal(sts_ctx* ctx, int32_t dual);
/* Pairs of the last dual traversal (sts_velocity_dual) of one kind: 0 PP, 1 PC, 2 CP, 3 CC.
 * *npairs (HOST) receives the count; tgt[npairs] and src[npairs] (HOST, may be NULL) the
 * target and source node ids, sorted by target (depth-first leaf order for PP and PC, cluster
 * order for CP and CC), then source node id.  STS_ERR_STATE without dual lists. */
int sts_dual_export(sts_ctx* ctx, int32_t kind, int64_t* npairs, int32_t* tgt, int32_t* src,
                    void* stream);
/* Interaction counts of the dual lists at degree d (M = (d+1)(d+2)/2): stats[0] PP particle
 * pairs (j != i), stats[1] PC target x proxy, stats[2] CP proxy x source, stats[3] CC
 * proxy x proxy, stats[4] downward particle x M (clusters that are CP or CC targets). */
int sts_dual_stats(sts_ctx* ctx, int32_t degree, int64_t* stats, void* stream);
/* Proxy reference data of degree d, computed on the host: beta[M,3] (barycentric proxy
 * points on the reference simplex, in selection order) and vinv[M,M] (inverse of
 * V_ref[m][k] = B_k(beta_m), row k, column m).  Either pointer may be NULL.  Needs no GPU. */
int sts_proxy_reference(int32_t degree, double* beta, double* vinv);
/* Interaction counts of the last sts_velocity: stats[0] = PC interactions (targets x proxy
 * points), stats[1] = PP pairs (j != i). */
int sts_stats(sts_ctx* ctx, int64_t* stats, void* stream);

/* ---- phase timing (CUDA events recorded on the launching stream) ------------------- */
#define STS_PHASE_BUILD 0  /* sts_tree_build, whole call                                */
#define STS_PHASE_SORT 1   /* radix sort and leaf list inside the build                 */
#define STS_PHASE_LISTS 2  /* interaction lists and evaluation tasks                    */
#define STS_PHASE_PREP 3   /* sorted source copies                                      */
#define STS_PHASE_UPWARD 4 /* SBB moments and proxy weights                             */
#define STS_PHASE_EVAL 5   /* the far + near evaluation kernel (PP + PC of the dual too)  */
#define STS_PHASE_DIRECT 6 /* direct sum (all its kernels)                              */
#define STS_PHASE_CLUSTER 7 /* dual traversal: CP + CC at the target proxies, downward  */
#define STS_NUM_PHASES 8
/* on != 0 starts recording per-phase events and resets the totals; 0 stops. */
int sts_set_timing(sts_ctx* ctx, int32_t on);
/* Total milliseconds and number of timed occurrences per phase since sts_set_timing(1);
 * ms[nph], count[nph] (host), nph <= STS_NUM_PHASES.  Synchronises the recorded events. */
int sts_phase_times(sts_ctx* ctx, double* ms, int32_t* count, int32_t nph);

/* Number of kernels this library has launched in the process so far (all contexts). */
int sts_launch_count(int64_t* out);

#ifdef __cplusplus
}
#endif
#endif /* STS_H */
