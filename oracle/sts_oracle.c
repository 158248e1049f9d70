/*
 * Plain, slow FP64 CPU oracle for the spherical Biot-Savart velocity sum and the spherical
 * tree code of Chen & Jablonowski, "Fast Summation on the Sphere with Applications to the
 * Barotropic Vorticity Equation" (arXiv 2401.07361).
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the CPU-baseline legs of the
 * benchmark call it; the product (the CUDA library and its binding) never does.  It shares
 * no code, header, table or constant generator with the CUDA library.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC.  No FMA contraction, no fast
 * math: every floating-point decision (face, child, MAC) is taken by the IEEE-754 double
 * operations written out below, in the order written (sums left to right).
 *
 * What each part follows:
 *   bs_term / or_direct   the midpoint-rule particle system (Sec. 2, the discrete dx_i/dt),
 *                         with 1 - x.y written as |x - y|^2 / 2 (Eq. altkernel) and
 *                         x_i x x_j = x_i x (x_j - x_i).
 *   ico_build             the icosahedron whose faces are refined into the tree (Sec. 3,
 *                         "Grids on a Sphere").  Orientation and vertex order are not given
 *                         in the paper; the reading used is stated at the function.
 *   or_tree_build         iterative 4-way refinement of the faces (Sec. 3); a triangle is a
 *                         leaf when it holds at most N_T particles or sits at the depth limit.
 *   mac                   (r_t + r_s)/R < theta (Sec. 3.4, "Dual Tree Traversal").
 *   or_tree_lists         target-leaf traversal from the 20 roots (Sec. 3.4), PC + PP only.
 *   afp_points            approximate Fekete points (Sec. 3.2); construction not given in the
 *                         paper, read as greedy column-pivoted QR on a barycentric lattice.
 *   sbb                   the SBB basis B_ijk = b1^i b2^j b3^k, i+j+k = d (Sec. 3.2).
 *   cluster_weights       omega_k = sum_j B_k(y_j) q_j A_j and the proxy-point form of the PC
 *                         interaction (Sec. 3.3.2): W = V_s^{-T} omega.
 *   pc_literal            the PC interaction exactly as printed: solve V alpha = G(x, y~),
 *                         then sum_k alpha_k omega_k (Sec. 3.3.2).
 *   dual / or_dual_lists / or_tree_velocity_dual
 *                         the dual tree traversal of Sec. 3.4 with all four interactions
 *                         (PP, PC, CP, CC of Sec. 3.3); CP and CC give the velocity at the
 *                         target cluster's proxy points, interpolated to its particles.
 *   pot_term / or_direct_potential / or_tree_potential
 *                         the stream function: the same sums with the Green's function
 *                         G = -(1/4pi) log(1 - x.y) of Sec. 2 as the kernel (the convolution
 *                         of Sec. 3 with that G); pc_literal_pot is its printed PC form.
 *   or_amr_*              the adaptive mesh refinement of Appendix A (split and merge of the
 *                         particle triangulation by the circulation and vorticity-variation
 *                         criteria, at most `levels` levels below the base mesh).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_ERR_ARG (-1)
#define OR_ERR_MEM (-2)
#define OR_PI 3.14159265358979323846

typedef struct { double x, y, z; } v3;

static v3 mk(double x, double y, double z) { v3 r; r.x = x; r.y = y; r.z = z; return r; }
static v3 vadd(v3 a, v3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 vsub(v3 a, v3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static double vdot(v3 a, v3 b) { return (a.x * b.x + a.y * b.y) + a.z * b.z; }
static v3 vcross(v3 a, v3 b)
{
    return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
/* s / |s| with |s| = sqrt((sx^2 + sy^2) + sz^2) and three divisions. */
static v3 vunit(v3 s)
{
    double n = sqrt(vdot(s, s));
    return mk(s.x / n, s.y / n, s.z / n);
}
static v3 ld3(const double* p, int64_t i) { return mk(p[3 * i], p[3 * i + 1], p[3 * i + 2]); }

/* ------------------------------------------------------------------------------------- */
/* The kernel.  Sec. 2: dx_i/dt = -(1/4pi) sum_{j != i} (x_i x x_j) zeta_j A_j / (1 - x_i.x_j).
 * Eq. altkernel replaces 1 - x.y by |x - y|^2 / 2; x_i x x_j equals x_i x (x_j - x_i).
 * bs_term adds w (x x d) / (|d|^2 / 2), d = y - x, to *acc.  A distinct particle at the
 * same position (d = 0) adds nothing: the cross product vanishes with it.                 */
static void bs_term(v3 x, v3 y, double w, v3* acc)
{
    v3 d = vsub(y, x);
    double h = 0.5 * vdot(d, d);
    if (h == 0.0) return;
    double t = w / h;
    v3 c = vcross(x, d);
    acc->x += c.x * t;
    acc->y += c.y * t;
    acc->z += c.z * t;
}

/* The vector sum S of the velocity kernel: acc += w (y - x) / (|y - x|^2 / 2), so that the
 * velocity is -(1/4pi) x x S (the x x factor taken out of bs_term; x x (y - x) = x x y).     */
static void bs_sum(v3 x, v3 y, double w, v3* acc)
{
    v3 d = vsub(y, x);
    double h = 0.5 * vdot(d, d);
    if (h == 0.0) return;
    double t = w / h;
    acc->x += d.x * t;
    acc->y += d.y * t;
    acc->z += d.z * t;
}

/* The potential kernel: G(x, y) = -(1/4pi) log(1 - x.y) (Sec. 2), the Green's function of
 * the spherical Laplacian, so that psi_i = sum_{j != i} G(x_i, x_j) zeta_j A_j is the stream
 * function of the particle system (Delta psi = zeta).  With Eq. altkernel 1 - x.y =
 * |x - y|^2 / 2.  pot_term adds w log(|d|^2 / 2) to *acc; a distinct particle at the same
 * position adds nothing, as in bs_term (the kernel is singular there; the paper defines no
 * value).                                                                                  */
static void pot_term(v3 x, v3 y, double w, double* acc)
{
    v3 d = vsub(y, x);
    double h = 0.5 * vdot(d, d);
    if (h == 0.0) return;
    *acc += w * log(h);
}

static int set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
    return nthreads;
#else
    (void)nthreads;
    return 1;
#endif
}

/* Direct summation (Sec. 2 particle system; Sec. 4.1 "direct summation").
 * pos[n,3], zeta[n], area[n]; targets: NULL for all n targets, else nt original indices.
 * vel[nt,3] receives u at each target.  OpenMP splits targets only, so every target's sum
 * runs in the same order whatever the thread count.                                     */
int or_direct(int64_t n, const double* pos, const double* zeta, const double* area,
              int64_t nt, const int64_t* targets, double* vel, int nthreads)
{
    if (n < 0 || nt < 0 || (n > 0 && (!pos || !zeta || !area)) || (nt > 0 && !vel))
        return OR_ERR_ARG;
    if (!targets) nt = n;
    double* w = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!w) return OR_ERR_MEM;
    for (int64_t j = 0; j < n; j++) w[j] = zeta[j] * area[j];
    const double f = -1.0 / (4.0 * OR_PI);
    int nth = set_threads(nthreads);
    (void)nth;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nth)
    for (int64_t k = 0; k < nt; k++) {
        int64_t i = targets ? targets[k] : k;
        v3 x = ld3(pos, i);
        v3 acc = mk(0.0, 0.0, 0.0);
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            bs_term(x, ld3(pos, j), w[j], &acc);
        }
        vel[3 * k] = f * acc.x;
        vel[3 * k + 1] = f * acc.y;
        vel[3 * k + 2] = f * acc.z;
    }
    free(w);
    return OR_OK;
}

/* Direct summation of the stream function psi_i = -(1/4pi) sum_{j != i} log(1 - x_i.x_j)
 * zeta_j A_j (Sec. 2 Green's function, Sec. 3 convolution sum).  Arguments as or_direct;
 * psi[nt] receives psi at each target.                                                    */
int or_direct_potential(int64_t n, const double* pos, const double* zeta, const double* area,
                        int64_t nt, const int64_t* targets, double* psi, int nthreads)
{
    if (n < 0 || nt < 0 || (n > 0 && (!pos || !zeta || !area)) || (nt > 0 && !psi))
        return OR_ERR_ARG;
    if (!targets) nt = n;
    double* w = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!w) return OR_ERR_MEM;
    for (int64_t j = 0; j < n; j++) w[j] = zeta[j] * area[j];
    const double f = -1.0 / (4.0 * OR_PI);
    int nth = set_threads(nthreads);
    (void)nth;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nth)
    for (int64_t k = 0; k < nt; k++) {
        int64_t i = targets ? targets[k] : k;
        v3 x = ld3(pos, i);
        double acc = 0.0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            pot_term(x, ld3(pos, j), w[j], &acc);
        }
        psi[k] = f * acc;
    }
    free(w);
    return OR_OK;
}

/* ------------------------------------------------------------------------------------- */
/* Icosahedron (Sec. 3: "We start with an icosahedron and refine its faces").  The paper
 * gives no orientation or numbering, so this reading fixes one:
 *   vertices: the cyclic families (0, +-1, +-g), (+-1, +-g, 0), (+-g, 0, +-1), g the golden
 *             ratio, families in that order, sign pairs in the order (+,+), (+,-), (-,+),
 *             (-,-); each scaled to unit length by vunit;
 *   faces:    every i < j < k whose unscaled pairwise squared distances are all 4, in
 *             lexicographic order of (i, j, k), stored as (i, j, k) when
 *             det(v_i, v_j, v_k) > 0 and as (i, k, j) otherwise (counter-clockwise seen
 *             from outside).                                                               */
static void ico_build(v3 V[12], int F[20][3])
{
    const double g = (1.0 + sqrt(5.0)) / 2.0;
    const double sg[4][2] = {{1.0, 1.0}, {1.0, -1.0}, {-1.0, 1.0}, {-1.0, -1.0}};
    v3 raw[12];
    int n = 0;
    for (int fam = 0; fam < 3; fam++)
        for (int s = 0; s < 4; s++) {
            double a = sg[s][0], b = sg[s][1];
            if (fam == 0) raw[n++] = mk(0.0, a * 1.0, b * g);
            else if (fam == 1) raw[n++] = mk(a * 1.0, b * g, 0.0);
            else raw[n++] = mk(a * g, 0.0, b * 1.0);
        }
    for (int i = 0; i < 12; i++) V[i] = vunit(raw[i]);
    int nf = 0;
    for (int i = 0; i < 12; i++)
        for (int j = i + 1; j < 12; j++)
            for (int k = j + 1; k < 12; k++) {
                v3 a = vsub(raw[i], raw[j]), b = vsub(raw[i], raw[k]), c = vsub(raw[j], raw[k]);
                if (fabs(vdot(a, a) - 4.0) > 1e-9 || fabs(vdot(b, b) - 4.0) > 1e-9 ||
                    fabs(vdot(c, c) - 4.0) > 1e-9)
                    continue;
                double det = vdot(V[i], vcross(V[j], V[k]));
                F[nf][0] = i;
                F[nf][1] = det > 0.0 ? j : k;
                F[nf][2] = det > 0.0 ? k : j;
                nf++;
            }
}

/* ------------------------------------------------------------------------------------- */
/* Tree.  Node numbering: level by level (roots first), and within a level in key order;
 * only non-empty triangles are nodes.  key = face index, then two bits per level (the
 * child digit).  Children of (v1, v2, v3), with m_ab = vunit(v_a + v_b):
 *   0 = (v1, m12, m31), 1 = (m12, v2, m23), 2 = (m31, m23, v3), 3 = (m12, m23, m31).       */
typedef struct {
    int32_t level, parent, first_child, nchild, leaf;
    uint64_t key;
    int64_t start, count;
    v3 v[3];
    v3 c;     /* circumcentre direction: vunit((v2 - v1) x (v3 - v1)) */
    double r; /* chord radius |c - v1|                                 */
} onode;

typedef struct or_tree {
    int64_t n;
    int leaf_size, max_level, maxdepth;
    int64_t nnodes, cap;
    onode* nodes;
    int64_t nleaves;
    int32_t* leaves;  /* leaf node ids in depth-first order            */
    int64_t* perm;    /* sorted position -> original particle index     */
    double* pos;      /* copy of the positions, original order          */
    /* interaction lists for one theta, per leaf in depth-first order */
    double theta;
    int has_lists;
    int64_t *far_off, *near_off;
    int32_t *far_idx, *near_idx;
    /* dual-traversal pairs (target node, source node) for one theta, per kind PP, PC, CP, CC,
     * in traversal order */
    double dual_theta;
    int has_dual;
    int32_t* dual_t[4];
    int32_t* dual_s[4];
    int64_t dual_n[4];
} or_tree;

static int push_node(or_tree* t, const onode* nd)
{
    if (t->nnodes == t->cap) {
        int64_t nc = t->cap ? 2 * t->cap : 1024;
        onode* p = (onode*)realloc(t->nodes, sizeof(onode) * (size_t)nc);
        if (!p) return OR_ERR_MEM;
        t->nodes = p;
        t->cap = nc;
    }
    t->nodes[t->nnodes++] = *nd;
    return OR_OK;
}

static void node_geometry(onode* nd)
{
    nd->c = vunit(vcross(vsub(nd->v[1], nd->v[0]), vsub(nd->v[2], nd->v[0])));
    v3 e = vsub(nd->c, nd->v[0]);
    nd->r = sqrt(vdot(e, e));
}

/* Face of a particle: the first face f maximising x . c_f over the 20 face centres
 * c_f = vunit((v_a + v_b) + v_c).  For the regular icosahedron the centres' spherical
 * Voronoi cells are exactly the faces, so this is face containment with no gaps.          */
static int face_of(v3 x, const v3 C[20])
{
    int best = 0;
    double bd = vdot(x, C[0]);
    for (int f = 1; f < 20; f++) {
        double d = vdot(x, C[f]);
        if (d > bd) {
            bd = d;
            best = f;
        }
    }
    return best;
}

/* Child digit of x inside a triangle with edge midpoints m12, m23, m31:
 * (m12 x m31).x >= 0 -> 0, else (m23 x m12).x >= 0 -> 1, else (m31 x m23).x >= 0 -> 2,
 * else 3 (the centre triangle).                                                          */
static int child_digit(v3 x, v3 n0, v3 n1, v3 n2)
{
    if (vdot(n0, x) >= 0.0) return 0;
    if (vdot(n1, x) >= 0.0) return 1;
    if (vdot(n2, x) >= 0.0) return 2;
    return 3;
}

void or_tree_free(or_tree* t)
{
    if (!t) return;
    free(t->nodes);
    free(t->leaves);
    free(t->perm);
    free(t->pos);
    free(t->far_off);
    free(t->near_off);
    free(t->far_idx);
    free(t->near_idx);
    for (int k = 0; k < 4; k++) {
        free(t->dual_t[k]);
        free(t->dual_s[k]);
    }
    free(t);
}

static void dfs_leaves(or_tree* t, int32_t id, int64_t* k)
{
    onode* nd = &t->nodes[id];
    if (nd->leaf) {
        t->leaves[(*k)++] = id;
        return;
    }
    for (int c = 0; c < nd->nchild; c++) dfs_leaves(t, nd->first_child + c, k);
}

/* Builds the triangle tree of Sec. 3 over pos[n,3]: refine every triangle holding more
 * than leaf_size particles, up to level max_level.  Within a triangle particles keep
 * their original relative order, so the sorted order is the depth-first order of leaves
 * with ties broken by original index.                                                    */
or_tree* or_tree_build(int64_t n, const double* pos, int leaf_size, int max_level)
{
    if (n < 0 || (n > 0 && !pos) || leaf_size < 1 || max_level < 0 || max_level > 29) return NULL;
    or_tree* t = (or_tree*)calloc(1, sizeof(or_tree));
    if (!t) return NULL;
    t->n = n;
    t->leaf_size = leaf_size;
    t->max_level = max_level;
    size_t nn = (size_t)(n > 0 ? n : 1);
    t->pos = (double*)malloc(sizeof(double) * 3 * nn);
    t->perm = (int64_t*)malloc(sizeof(int64_t) * nn);
    int64_t* cur = (int64_t*)malloc(sizeof(int64_t) * nn);  /* particles grouped by node  */
    int64_t* nxt = (int64_t*)malloc(sizeof(int64_t) * nn);
    int64_t* seg = NULL;  /* per node: offset of its particles in cur (this level) */
    int* dig = (int*)malloc(sizeof(int) * nn);
    if (!t->pos || !t->perm || !cur || !nxt || !dig) goto fail;
    if (n > 0) memcpy(t->pos, pos, sizeof(double) * 3 * (size_t)n);

    v3 V[12];
    int F[20][3];
    ico_build(V, F);
    v3 C[20];
    for (int f = 0; f < 20; f++) C[f] = vunit(vadd(vadd(V[F[f][0]], V[F[f][1]]), V[F[f][2]]));

    /* level 0: faces */
    int64_t fcount[20] = {0};
    for (int64_t i = 0; i < n; i++) {
        dig[i] = face_of(ld3(pos, i), C);
        fcount[dig[i]]++;
    }
    int64_t foff[20], acc = 0;
    for (int f = 0; f < 20; f++) {
        foff[f] = acc;
        acc += fcount[f];
    }
    {
        int64_t fill[20];
        memcpy(fill, foff, sizeof(fill));
        for (int64_t i = 0; i < n; i++) cur[fill[dig[i]]++] = i;
    }
    int64_t level_first = 0;
    for (int f = 0; f < 20; f++) {
        if (fcount[f] == 0) continue;
        onode nd;
        memset(&nd, 0, sizeof(nd));
        nd.level = 0;
        nd.parent = -1;
        nd.first_child = -1;
        nd.key = (uint64_t)f;
        nd.start = foff[f];
        nd.count = fcount[f];
        for (int a = 0; a < 3; a++) nd.v[a] = V[F[f][a]];
        node_geometry(&nd);
        if (push_node(t, &nd)) goto fail;
    }
    /* seg offsets at level 0 equal the starts (faces are contiguous in cur) */
    int64_t level_end = t->nnodes;
    seg = (int64_t*)malloc(sizeof(int64_t) * (size_t)(level_end > 0 ? level_end : 1));
    if (!seg) goto fail;
    for (int64_t id = 0; id < level_end; id++) seg[id] = t->nodes[id].start;

    for (int level = 0;; level++) {
        int64_t nxt_fill = 0;
        int64_t new_first = t->nnodes;
        for (int64_t id = level_first; id < level_end; id++) {
            onode nd = t->nodes[id];
            const int64_t* mine = cur + seg[id - level_first];
            if (nd.count <= leaf_size || nd.level >= max_level) {
                t->nodes[id].leaf = 1;
                for (int64_t r = 0; r < nd.count; r++) t->perm[nd.start + r] = mine[r];
                continue;
            }
            v3 v1 = nd.v[0], v2 = nd.v[1], v3_ = nd.v[2];
            v3 m12 = vunit(vadd(v1, v2)), m23 = vunit(vadd(v2, v3_)), m31 = vunit(vadd(v3_, v1));
            v3 n0 = vcross(m12, m31), n1 = vcross(m23, m12), n2 = vcross(m31, m23);
            int64_t cc[4] = {0, 0, 0, 0};
            for (int64_t r = 0; r < nd.count; r++) {
                dig[r] = child_digit(ld3(pos, mine[r]), n0, n1, n2);
                cc[dig[r]]++;
            }
            int64_t coff[4], a2 = 0;
            for (int c = 0; c < 4; c++) {
                coff[c] = a2;
                a2 += cc[c];
            }
            int64_t fill[4];
            for (int c = 0; c < 4; c++) fill[c] = nxt_fill + coff[c];
            for (int64_t r = 0; r < nd.count; r++) nxt[fill[dig[r]]++] = mine[r];
            v3 cv[4][3] = {{v1, m12, m31}, {m12, v2, m23}, {m31, m23, v3_}, {m12, m23, m31}};
            t->nodes[id].first_child = (int32_t)t->nnodes;
            int nchild = 0;
            for (int c = 0; c < 4; c++) {
                if (cc[c] == 0) continue;
                onode ch;
                memset(&ch, 0, sizeof(ch));
                ch.level = nd.level + 1;
                ch.parent = (int32_t)id;
                ch.first_child = -1;
                ch.key = nd.key * 4u + (uint64_t)c;
                ch.start = nd.start + coff[c];
                ch.count = cc[c];
                for (int a = 0; a < 3; a++) ch.v[a] = cv[c][a];
                node_geometry(&ch);
                if (push_node(t, &ch)) goto fail;
                nchild++;
            }
            t->nodes[id].nchild = nchild;
            nxt_fill += nd.count;
        }
        int64_t new_end = t->nnodes;
        if (new_end == new_first) break;
        /* children are contiguous in nxt in node order: their seg offsets are cumulative */
        free(seg);
        seg = (int64_t*)malloc(sizeof(int64_t) * (size_t)(new_end - new_first));
        if (!seg) goto fail;
        int64_t off = 0;
        for (int64_t id = new_first; id < new_end; id++) {
            seg[id - new_first] = off;
            off += t->nodes[id].count;
        }
        int64_t* tmp = cur;
        cur = nxt;
        nxt = tmp;
        level_first = new_first;
        level_end = new_end;
        t->maxdepth = level + 1;
    }

    t->nleaves = 0;
    for (int64_t id = 0; id < t->nnodes; id++) t->nleaves += t->nodes[id].leaf;
    t->leaves = (int32_t*)malloc(sizeof(int32_t) * (size_t)(t->nleaves > 0 ? t->nleaves : 1));
    if (!t->leaves) goto fail;
    {
        int64_t k = 0;
        for (int64_t id = 0; id < t->nnodes && t->nodes[id].level == 0; id++) dfs_leaves(t, (int32_t)id, &k);
    }
    free(cur);
    free(nxt);
    free(seg);
    free(dig);
    return t;
fail:
    free(cur);
    free(nxt);
    free(seg);
    free(dig);
    or_tree_free(t);
    return NULL;
}

/* info: [0] n, [1] nodes, [2] leaves, [3] deepest level, [4] far list length,
 *       [5] near list length (the last two are 0 before or_tree_lists).                  */
int or_tree_info(const or_tree* t, int64_t* info)
{
    if (!t || !info) return OR_ERR_ARG;
    info[0] = t->n;
    info[1] = t->nnodes;
    info[2] = t->nleaves;
    info[3] = t->maxdepth;
    info[4] = t->has_lists ? t->far_off[t->nleaves] : 0;
    info[5] = t->has_lists ? t->near_off[t->nleaves] : 0;
    return OR_OK;
}

/* Copies the tree out.  Any pointer may be NULL.  geom[nodes,13] = v1, v2, v3, c, r.     */
int or_tree_export(const or_tree* t, int64_t* perm, int32_t* level, uint64_t* key, int32_t* parent,
                   int32_t* first_child, int32_t* nchild, int64_t* start, int64_t* count,
                   int32_t* leaf, int32_t* leaves, double* geom)
{
    if (!t) return OR_ERR_ARG;
    if (perm) memcpy(perm, t->perm, sizeof(int64_t) * (size_t)t->n);
    if (leaves) memcpy(leaves, t->leaves, sizeof(int32_t) * (size_t)t->nleaves);
    for (int64_t id = 0; id < t->nnodes; id++) {
        const onode* nd = &t->nodes[id];
        if (level) level[id] = nd->level;
        if (key) key[id] = nd->key;
        if (parent) parent[id] = nd->parent;
        if (first_child) first_child[id] = nd->first_child;
        if (nchild) nchild[id] = nd->nchild;
        if (start) start[id] = nd->start;
        if (count) count[id] = nd->count;
        if (leaf) leaf[id] = nd->leaf;
        if (geom) {
            double* g = geom + 13 * id;
            for (int a = 0; a < 3; a++) {
                g[3 * a] = nd->v[a].x;
                g[3 * a + 1] = nd->v[a].y;
                g[3 * a + 2] = nd->v[a].z;
            }
            g[9] = nd->c.x;
            g[10] = nd->c.y;
            g[11] = nd->c.z;
            g[12] = nd->r;
        }
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------------------- */
/* MAC of Sec. 3.4: well separated iff (r_t + r_s) / R < theta, written without the
 * division as (r_t + r_s) < theta * R, R = |c_t - c_s| (chord).  R = 0 never separates.  */
static int mac(const onode* a, const onode* b, double theta)
{
    v3 e = vsub(a->c, b->c);
    double R = sqrt(vdot(e, e));
    return (a->r + b->r) < theta * R;
}

typedef struct {
    int32_t* p;
    int64_t n, cap;
} ivec;

static int ivec_push(ivec* v, int32_t x)
{
    if (v->n == v->cap) {
        int64_t nc = v->cap ? 2 * v->cap : 4096;
        int32_t* q = (int32_t*)realloc(v->p, sizeof(int32_t) * (size_t)nc);
        if (!q) return OR_ERR_MEM;
        v->p = q;
        v->cap = nc;
    }
    v->p[v->n++] = x;
    return OR_OK;
}

/* Traversal of Sec. 3.4 for one target leaf t over source node s (preorder):
 *   MAC passes:  s holds more than N_T particles -> far (PC); else -> near (PP);
 *   MAC fails:   s is a leaf -> near (PP); else descend into s's children in digit order. */
static int traverse(const or_tree* tr, const onode* t, int32_t s, double theta, ivec* far, ivec* near)
{
    const onode* sn = &tr->nodes[s];
    if (mac(t, sn, theta)) {
        if (sn->count > tr->leaf_size) return ivec_push(far, s);
        return ivec_push(near, s);
    }
    if (sn->leaf) return ivec_push(near, s);
    for (int c = 0; c < sn->nchild; c++)
        if (traverse(tr, t, sn->first_child + c, theta, far, near)) return OR_ERR_MEM;
    return OR_OK;
}

int or_tree_lists(or_tree* tr, double theta)
{
    if (!tr || !(theta > 0.0) || !(theta < 1.0)) return OR_ERR_ARG;
    free(tr->far_off);
    free(tr->near_off);
    free(tr->far_idx);
    free(tr->near_idx);
    tr->far_off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(tr->nleaves + 1));
    tr->near_off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(tr->nleaves + 1));
    tr->far_idx = tr->near_idx = NULL;
    tr->has_lists = 0;
    if (!tr->far_off || !tr->near_off) return OR_ERR_MEM;
    ivec far = {0}, near = {0};
    tr->far_off[0] = tr->near_off[0] = 0;
    for (int64_t L = 0; L < tr->nleaves; L++) {
        const onode* t = &tr->nodes[tr->leaves[L]];
        for (int64_t id = 0; id < tr->nnodes && tr->nodes[id].level == 0; id++)
            if (traverse(tr, t, (int32_t)id, theta, &far, &near)) {
                free(far.p);
                free(near.p);
                return OR_ERR_MEM;
            }
        tr->far_off[L + 1] = far.n;
        tr->near_off[L + 1] = near.n;
    }
    tr->far_idx = far.p ? far.p : (int32_t*)malloc(sizeof(int32_t));
    tr->near_idx = near.p ? near.p : (int32_t*)malloc(sizeof(int32_t));
    tr->theta = theta;
    tr->has_lists = 1;
    return OR_OK;
}

int or_lists_export(const or_tree* tr, int64_t* far_off, int32_t* far_idx, int64_t* near_off,
                    int32_t* near_idx)
{
    if (!tr || !tr->has_lists) return OR_ERR_ARG;
    int64_t L = tr->nleaves;
    if (far_off) memcpy(far_off, tr->far_off, sizeof(int64_t) * (size_t)(L + 1));
    if (near_off) memcpy(near_off, tr->near_off, sizeof(int64_t) * (size_t)(L + 1));
    if (far_idx) memcpy(far_idx, tr->far_idx, sizeof(int32_t) * (size_t)tr->far_off[L]);
    if (near_idx) memcpy(near_idx, tr->near_idx, sizeof(int32_t) * (size_t)tr->near_off[L]);
    return OR_OK;
}

/* ------------------------------------------------------------------------------------- */
/* Dual tree traversal (Sec. 3.4) with the four interactions of Sec. 3.3.  From the 20 x 20
 * pairs of roots, a pair (T_t, T_s) that passes the MAC interacts by its particle counts
 * against N_T: PP when both hold at most N_T, PC when only the source holds more, CP when
 * only the target does, CC when both do.  A pair that fails the MAC interacts directly (PP)
 * when both triangles are leaves; otherwise the triangle with more particles is refined (its
 * children paired with the other, in digit order).  Reading (the paper's sentence is garbled
 * there): a leaf is never refined, so a failing pair with one leaf refines the other; on equal
 * counts the target is refined.  A node "holds more than N_T" exactly when it is a cluster
 * (count > N_T), so the targets of PC and PP are leaves and the targets of CP and CC are
 * clusters, possibly leaves at the depth limit.                                           */
enum { KPP = 0, KPC = 1, KCP = 2, KCC = 3 };

static int dual(const or_tree* tr, int32_t t, int32_t s, double theta, ivec* pt, ivec* ps)
{
    const onode *tn = &tr->nodes[t], *sn = &tr->nodes[s];
    const int tc = tn->count > tr->leaf_size, sc = sn->count > tr->leaf_size;
    int kind = -1;
    if (mac(tn, sn, theta))
        kind = tc ? (sc ? KCC : KCP) : (sc ? KPC : KPP);
    else if (tn->leaf && sn->leaf)
        kind = KPP;
    if (kind >= 0) {
        if (ivec_push(&pt[kind], t) || ivec_push(&ps[kind], s)) return OR_ERR_MEM;
        return OR_OK;
    }
    if (!tn->leaf && (sn->leaf || tn->count >= sn->count)) {
        for (int c = 0; c < tn->nchild; c++)
            if (dual(tr, tn->first_child + c, s, theta, pt, ps)) return OR_ERR_MEM;
    } else {
        for (int c = 0; c < sn->nchild; c++)
            if (dual(tr, t, sn->first_child + c, theta, pt, ps)) return OR_ERR_MEM;
    }
    return OR_OK;
}

int or_dual_lists(or_tree* tr, double theta, int64_t* counts)
{
    if (!tr || !(theta > 0.0) || !(theta < 1.0)) return OR_ERR_ARG;
    for (int k = 0; k < 4; k++) {
        free(tr->dual_t[k]);
        free(tr->dual_s[k]);
        tr->dual_t[k] = tr->dual_s[k] = NULL;
        tr->dual_n[k] = 0;
    }
    tr->has_dual = 0;
    ivec pt[4] = {{0}}, ps[4] = {{0}};
    int rc = OR_OK;
    for (int64_t a = 0; a < tr->nnodes && tr->nodes[a].level == 0 && rc == OR_OK; a++)
        for (int64_t b = 0; b < tr->nnodes && tr->nodes[b].level == 0 && rc == OR_OK; b++)
            rc = dual(tr, (int32_t)a, (int32_t)b, theta, pt, ps);
    for (int k = 0; k < 4; k++) {
        tr->dual_t[k] = pt[k].p;
        tr->dual_s[k] = ps[k].p;
        tr->dual_n[k] = pt[k].n;
        if (counts) counts[k] = pt[k].n;
    }
    if (rc != OR_OK) return rc;
    tr->dual_theta = theta;
    tr->has_dual = 1;
    return OR_OK;
}

int or_dual_export(const or_tree* tr, int kind, int32_t* tgt, int32_t* src)
{
    if (!tr || !tr->has_dual || kind < 0 || kind > 3) return OR_ERR_ARG;
    if (tgt && tr->dual_n[kind]) memcpy(tgt, tr->dual_t[kind], sizeof(int32_t) * (size_t)tr->dual_n[kind]);
    if (src && tr->dual_n[kind]) memcpy(src, tr->dual_s[kind], sizeof(int32_t) * (size_t)tr->dual_n[kind]);
    return OR_OK;
}

/* ------------------------------------------------------------------------------------- */
/* SBB basis of degree d (Sec. 3.2): B_k(b) = b1^a b2^b b3^c, a + b + c = d, enumerated as
 * a = d..0, then b = d - a..0 (c = d - a - b).  M = (d + 1)(d + 2) / 2 functions.        */
static int nbasis(int d) { return (d + 1) * (d + 2) / 2; }

static void sbb(int d, double b1, double b2, double b3, double* B)
{
    double p1[33], p2[33], p3[33];
    p1[0] = p2[0] = p3[0] = 1.0;
    for (int e = 1; e <= d; e++) {
        p1[e] = p1[e - 1] * b1;
        p2[e] = p2[e - 1] * b2;
        p3[e] = p3[e - 1] * b3;
    }
    int k = 0;
    for (int a = d; a >= 0; a--)
        for (int b = d - a; b >= 0; b--) {
            int c = d - a - b;
            B[k++] = (p1[a] * p2[b]) * p3[c];
        }
}

/* Spherical barycentric coordinates of y in the triangle (v1, v2, v3) (Sec. 3.2:
 * y = b1 v1 + b2 v2 + b3 v3), by Cramer's rule with D = v1 . (v2 x v3).                  */
static void sph_bary(v3 y, v3 v1, v3 v2, v3 v3_, double* b)
{
    double D = vdot(v1, vcross(v2, v3_));
    b[0] = vdot(y, vcross(v2, v3_)) / D;
    b[1] = vdot(y, vcross(v3_, v1)) / D;
    b[2] = vdot(y, vcross(v1, v2)) / D;
}

/* Approximate Fekete points of degree d on the planar reference simplex (Sec. 3.2 names
 * them and cites their construction; the construction itself is not printed).  Reading:
 * greedy column-pivoted Householder QR of A[k][c] = B_k(candidate c) over the barycentric
 * lattice of resolution 3d (candidates (p, q, 3d - p - q) / 3d, p = 3d..0, q = 3d - p..0).
 * At each step the candidate with the largest remaining column norm is taken; norms within
 * a relative 1e-9 of the largest count as equal and the lowest candidate index wins.
 * Writes beta[M,3] (in selection order) and the chosen candidate indices.                 */
int or_proxy_reference(int d, double* beta, int32_t* cand)
{
    if (d < 1 || d > 16 || !beta) return OR_ERR_ARG;
    const int M = nbasis(d), R = 3 * d, K = (R + 1) * (R + 2) / 2;
    double* cb = (double*)malloc(sizeof(double) * 3 * (size_t)K);
    double* A = (double*)malloc(sizeof(double) * (size_t)M * (size_t)K);
    double* nrm = (double*)malloc(sizeof(double) * (size_t)K);
    double* v = (double*)malloc(sizeof(double) * (size_t)M);
    char* chosen = (char*)calloc((size_t)K, 1);
    double* B = (double*)malloc(sizeof(double) * (size_t)M);
    if (!cb || !A || !nrm || !v || !chosen || !B) {
        free(cb); free(A); free(nrm); free(v); free(chosen); free(B);
        return OR_ERR_MEM;
    }
    int c = 0;
    for (int p = R; p >= 0; p--)
        for (int q = R - p; q >= 0; q--) {
            cb[3 * c] = (double)p / (double)R;
            cb[3 * c + 1] = (double)q / (double)R;
            cb[3 * c + 2] = (double)(R - p - q) / (double)R;
            sbb(d, cb[3 * c], cb[3 * c + 1], cb[3 * c + 2], B);
            for (int k = 0; k < M; k++) A[(size_t)k * K + c] = B[k];
            c++;
        }
    for (int s = 0; s < M; s++) {
        double mx = -1.0;
        for (c = 0; c < K; c++) {
            if (chosen[c]) continue;
            double acc = 0.0;
            for (int k = s; k < M; k++) acc += A[(size_t)k * K + c] * A[(size_t)k * K + c];
            nrm[c] = acc;
            if (acc > mx) mx = acc;
        }
        int pick = -1;
        for (c = 0; c < K; c++)
            if (!chosen[c] && nrm[c] >= mx * (1.0 - 1e-9)) {
                pick = c;
                break;
            }
        chosen[pick] = 1;
        if (cand) cand[s] = pick;
        beta[3 * s] = cb[3 * pick];
        beta[3 * s + 1] = cb[3 * pick + 1];
        beta[3 * s + 2] = cb[3 * pick + 2];
        /* Householder reflection zeroing rows s+1.. of the picked column */
        double sigma = sqrt(nrm[pick]);
        double a0 = A[(size_t)s * K + pick];
        double alpha = a0 > 0.0 ? -sigma : sigma;
        double vn = 0.0;
        for (int k = s; k < M; k++) v[k] = A[(size_t)k * K + pick];
        v[s] = v[s] - alpha;
        for (int k = s; k < M; k++) vn += v[k] * v[k];
        if (vn > 0.0)
            for (c = 0; c < K; c++) {
                if (chosen[c] && c != pick) continue;
                double tt = 0.0;
                for (int k = s; k < M; k++) tt += v[k] * A[(size_t)k * K + c];
                double f = 2.0 * tt / vn;
                for (int k = s; k < M; k++) A[(size_t)k * K + c] -= f * v[k];
            }
    }
    free(cb); free(A); free(nrm); free(v); free(chosen); free(B);
    return OR_OK;
}

/* Gauss-Jordan inverse with partial pivoting, a[n,n] row-major -> inv[n,n].             */
static int invert(int n, const double* a, double* inv)
{
    double* m = (double*)malloc(sizeof(double) * (size_t)n * (size_t)(2 * n));
    if (!m) return OR_ERR_MEM;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < 2 * n; j++)
            m[(size_t)i * 2 * n + j] = j < n ? a[(size_t)i * n + j] : (j - n == i ? 1.0 : 0.0);
    for (int col = 0; col < n; col++) {
        int piv = col;
        for (int i = col + 1; i < n; i++)
            if (fabs(m[(size_t)i * 2 * n + col]) > fabs(m[(size_t)piv * 2 * n + col])) piv = i;
        if (m[(size_t)piv * 2 * n + col] == 0.0) {
            free(m);
            return OR_ERR_ARG;
        }
        if (piv != col)
            for (int j = 0; j < 2 * n; j++) {
                double tmp = m[(size_t)col * 2 * n + j];
                m[(size_t)col * 2 * n + j] = m[(size_t)piv * 2 * n + j];
                m[(size_t)piv * 2 * n + j] = tmp;
            }
        double p = m[(size_t)col * 2 * n + col];
        for (int j = 0; j < 2 * n; j++) m[(size_t)col * 2 * n + j] /= p;
        for (int i = 0; i < n; i++) {
            if (i == col) continue;
            double f = m[(size_t)i * 2 * n + col];
            if (f == 0.0) continue;
            for (int j = 0; j < 2 * n; j++) m[(size_t)i * 2 * n + j] -= f * m[(size_t)col * 2 * n + j];
        }
    }
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) inv[(size_t)i * n + j] = m[(size_t)i * 2 * n + n + j];
    free(m);
    return OR_OK;
}

/* Solves a[n,n] x = b (Gaussian elimination, partial pivoting); b is overwritten by x.   */
static int solve(int n, double* a, double* b, int nrhs)
{
    for (int col = 0; col < n; col++) {
        int piv = col;
        for (int i = col + 1; i < n; i++)
            if (fabs(a[(size_t)i * n + col]) > fabs(a[(size_t)piv * n + col])) piv = i;
        if (a[(size_t)piv * n + col] == 0.0) return OR_ERR_ARG;
        if (piv != col) {
            for (int j = 0; j < n; j++) {
                double tmp = a[(size_t)col * n + j];
                a[(size_t)col * n + j] = a[(size_t)piv * n + j];
                a[(size_t)piv * n + j] = tmp;
            }
            for (int r = 0; r < nrhs; r++) {
                double tmp = b[(size_t)col * nrhs + r];
                b[(size_t)col * nrhs + r] = b[(size_t)piv * nrhs + r];
                b[(size_t)piv * nrhs + r] = tmp;
            }
        }
        for (int i = col + 1; i < n; i++) {
            double f = a[(size_t)i * n + col] / a[(size_t)col * n + col];
            if (f == 0.0) continue;
            for (int j = col; j < n; j++) a[(size_t)i * n + j] -= f * a[(size_t)col * n + j];
            for (int r = 0; r < nrhs; r++) b[(size_t)i * nrhs + r] -= f * b[(size_t)col * nrhs + r];
        }
    }
    for (int i = n - 1; i >= 0; i--)
        for (int r = 0; r < nrhs; r++) {
            double acc = b[(size_t)i * nrhs + r];
            for (int j = i + 1; j < n; j++) acc -= a[(size_t)i * n + j] * b[(size_t)j * nrhs + r];
            b[(size_t)i * nrhs + r] = acc / a[(size_t)i * n + i];
        }
    return OR_OK;
}

/* Reference interpolation data for degree d: beta[M,3] and V_ref^{-1}[M,M], where
 * V_ref[m][k] = B_k(beta_m).                                                              */
typedef struct {
    int d, M;
    double* beta;
    double* vinv;
} refdata;

static int ref_make(int d, refdata* r)
{
    r->d = d;
    r->M = nbasis(d);
    r->beta = (double*)malloc(sizeof(double) * 3 * (size_t)r->M);
    r->vinv = (double*)malloc(sizeof(double) * (size_t)r->M * (size_t)r->M);
    double* V = (double*)malloc(sizeof(double) * (size_t)r->M * (size_t)r->M);
    if (!r->beta || !r->vinv || !V) {
        free(V);
        return OR_ERR_MEM;
    }
    int rc = or_proxy_reference(d, r->beta, NULL);
    for (int m = 0; m < r->M && rc == OR_OK; m++)
        sbb(d, r->beta[3 * m], r->beta[3 * m + 1], r->beta[3 * m + 2], V + (size_t)m * r->M);
    if (rc == OR_OK) rc = invert(r->M, V, r->vinv);
    free(V);
    return rc;
}

static void ref_free(refdata* r)
{
    free(r->beta);
    free(r->vinv);
}

/* V_ref^{-1} for degree d (exported for the tests).                                     */
int or_vref_inverse(int d, double* vinv)
{
    if (d < 1 || d > 16 || !vinv) return OR_ERR_ARG;
    refdata r;
    int rc = ref_make(d, &r);
    if (rc == OR_OK) memcpy(vinv, r.vinv, sizeof(double) * (size_t)r.M * (size_t)r.M);
    ref_free(&r);
    return rc;
}

/* Proxy points of a source triangle: y~_m = vunit(b_m1 v1 + b_m2 v2 + b_m3 v3) (the sums
 * left to right), with rho_m = |b_m1 v1 + b_m2 v2 + b_m3 v3|.                            */
static void proxies(const refdata* r, const v3* v, v3* yt, double* rho)
{
    for (int m = 0; m < r->M; m++) {
        const double* b = r->beta + 3 * m;
        v3 s = mk((b[0] * v[0].x + b[1] * v[1].x) + b[2] * v[2].x,
                  (b[0] * v[0].y + b[1] * v[1].y) + b[2] * v[2].y,
                  (b[0] * v[0].z + b[1] * v[1].z) + b[2] * v[2].z);
        double n = sqrt(vdot(s, s));
        if (rho) rho[m] = n;
        yt[m] = mk(s.x / n, s.y / n, s.z / n);
    }
}

/* Proxy weights of one source triangle (Sec. 3.3.2).  omega_k = sum_j B_k(b(y_j)) w_j with
 * b(.) the spherical barycentric coordinates in the triangle, then W = V_s^{-T} omega with
 * V_s[m][k] = B_k(b(y~_m)).  Because B_k is homogeneous of degree d and b(y~_m) = beta_m /
 * rho_m, V_s = diag(rho^-d) V_ref and W_m = rho_m^d sum_k V_ref^{-1}[k][m] omega_k, so that
 * sum_k alpha_k(x) omega_k = sum_m G(x, y~_m) W_m for every x.                           */
static void cluster_weights(const refdata* r, const v3* v, int64_t ns, const v3* ys, const double* ws,
                            v3* yt, double* W, double* omega)
{
    const int M = r->M, d = r->d;
    double B[153], rho[153];
    for (int k = 0; k < M; k++) omega[k] = 0.0;
    for (int64_t j = 0; j < ns; j++) {
        double b[3];
        sph_bary(ys[j], v[0], v[1], v[2], b);
        sbb(d, b[0], b[1], b[2], B);
        for (int k = 0; k < M; k++) omega[k] += B[k] * ws[j];
    }
    proxies(r, v, yt, rho);
    for (int m = 0; m < M; m++) {
        double acc = 0.0;
        for (int k = 0; k < M; k++) acc += r->vinv[(size_t)k * M + m] * omega[k];
        double rd = 1.0;
        for (int e = 0; e < d; e++) rd *= rho[m];
        W[m] = rd * acc;
    }
}

/* One source triangle (verts[9] = v1, v2, v3), its sources ys[ns,3] with strengths
 * ws[ns]: writes the proxy points yt[M,3], proxy weights W[M] and moments omega[M].      */
int or_cluster(const double* verts, int d, int64_t ns, const double* ys, const double* ws, double* yt,
               double* W, double* omega)
{
    if (!verts || d < 1 || d > 16 || ns < 0 || !yt || !W || !omega) return OR_ERR_ARG;
    refdata r;
    int rc = ref_make(d, &r);
    if (rc != OR_OK) {
        ref_free(&r);
        return rc;
    }
    v3 v[3] = {ld3(verts, 0), ld3(verts, 1), ld3(verts, 2)};
    v3* y = (v3*)malloc(sizeof(v3) * (size_t)(ns > 0 ? ns : 1));
    v3 ytv[153];
    for (int64_t j = 0; j < ns; j++) y[j] = ld3(ys, j);
    cluster_weights(&r, v, ns, y, ws, ytv, W, omega);
    for (int m = 0; m < r.M; m++) {
        yt[3 * m] = ytv[m].x;
        yt[3 * m + 1] = ytv[m].y;
        yt[3 * m + 2] = ytv[m].z;
    }
    free(y);
    ref_free(&r);
    return OR_OK;
}

/* The PC interaction as printed (Sec. 3.3.2): for each velocity component c solve
 * V_s alpha = (K_c(x, y~_1), ..., K_c(x, y~_M)) and return sum_k alpha_k omega_k, where
 * K(x, y) = (x x y) / (|x - y|^2 / 2) is the kernel without the -1/4pi.                  */
static int pc_literal(const refdata* r, const v3* v, const v3* yt, const double* omega, v3 x, v3* out)
{
    const int M = r->M, d = r->d;
    double* Vs = (double*)malloc(sizeof(double) * (size_t)M * M);
    double* g = (double*)malloc(sizeof(double) * (size_t)M * 3);
    if (!Vs || !g) {
        free(Vs);
        free(g);
        return OR_ERR_MEM;
    }
    for (int m = 0; m < M; m++) {
        double b[3];
        sph_bary(yt[m], v[0], v[1], v[2], b);
        sbb(d, b[0], b[1], b[2], Vs + (size_t)m * M);
        v3 k = mk(0.0, 0.0, 0.0);
        bs_term(x, yt[m], 1.0, &k);
        g[3 * m] = k.x;
        g[3 * m + 1] = k.y;
        g[3 * m + 2] = k.z;
    }
    int rc = solve(M, Vs, g, 3);
    if (rc == OR_OK) {
        v3 acc = mk(0.0, 0.0, 0.0);
        for (int k = 0; k < M; k++) {
            acc.x += g[3 * k] * omega[k];
            acc.y += g[3 * k + 1] * omega[k];
            acc.z += g[3 * k + 2] * omega[k];
        }
        *out = acc;
    }
    free(Vs);
    free(g);
    return rc;
}

/* PC interaction of one target x[3] with one source triangle, both ways: the literal
 * alpha-solve (lit[3]) and the proxy-point form (prx[3]); both without the -1/4pi.       */
int or_pc_pair(const double* verts, int d, int64_t ns, const double* ys, const double* ws,
               const double* x, double* lit, double* prx)
{
    if (!verts || d < 1 || d > 16 || ns < 0 || !x || !lit || !prx) return OR_ERR_ARG;
    refdata r;
    int rc = ref_make(d, &r);
    if (rc != OR_OK) {
        ref_free(&r);
        return rc;
    }
    v3 v[3] = {ld3(verts, 0), ld3(verts, 1), ld3(verts, 2)};
    v3* y = (v3*)malloc(sizeof(v3) * (size_t)(ns > 0 ? ns : 1));
    for (int64_t j = 0; j < ns; j++) y[j] = ld3(ys, j);
    v3 yt[153];
    double W[153], om[153];
    cluster_weights(&r, v, ns, y, ws, yt, W, om);
    v3 xx = ld3(x, 0), a = mk(0.0, 0.0, 0.0), b;
    for (int m = 0; m < r.M; m++) bs_term(xx, yt[m], W[m], &a);
    rc = pc_literal(&r, v, yt, om, xx, &b);
    prx[0] = a.x; prx[1] = a.y; prx[2] = a.z;
    lit[0] = b.x; lit[1] = b.y; lit[2] = b.z;
    free(y);
    ref_free(&r);
    return rc;
}

/* The PC interaction of the potential as printed (Sec. 3.3.2): solve V_s alpha =
 * (log h(x, y~_1), ..., log h(x, y~_M)), h = |x - y|^2 / 2, and return sum_k alpha_k omega_k
 * (the kernel without the -1/4pi).                                                        */
static int pc_literal_pot(const refdata* r, const v3* v, const v3* yt, const double* omega, v3 x, double* out)
{
    const int M = r->M, d = r->d;
    double* Vs = (double*)malloc(sizeof(double) * (size_t)M * M);
    double* g = (double*)malloc(sizeof(double) * (size_t)M);
    if (!Vs || !g) {
        free(Vs);
        free(g);
        return OR_ERR_MEM;
    }
    for (int m = 0; m < M; m++) {
        double b[3];
        sph_bary(yt[m], v[0], v[1], v[2], b);
        sbb(d, b[0], b[1], b[2], Vs + (size_t)m * M);
        g[m] = 0.0;
        pot_term(x, yt[m], 1.0, &g[m]);
    }
    int rc = solve(M, Vs, g, 1);
    if (rc == OR_OK) {
        double acc = 0.0;
        for (int k = 0; k < M; k++) acc += g[k] * omega[k];
        *out = acc;
    }
    free(Vs);
    free(g);
    return rc;
}

/* The potential's PC interaction of one target with one source triangle, both ways (the
 * literal alpha-solve *lit, the proxy-point form *prx), without the -1/4pi.              */
int or_pc_pair_potential(const double* verts, int d, int64_t ns, const double* ys, const double* ws,
                         const double* x, double* lit, double* prx)
{
    if (!verts || d < 1 || d > 16 || ns < 0 || !x || !lit || !prx) return OR_ERR_ARG;
    refdata r;
    int rc = ref_make(d, &r);
    if (rc != OR_OK) {
        ref_free(&r);
        return rc;
    }
    v3 v[3] = {ld3(verts, 0), ld3(verts, 1), ld3(verts, 2)};
    v3* y = (v3*)malloc(sizeof(v3) * (size_t)(ns > 0 ? ns : 1));
    for (int64_t j = 0; j < ns; j++) y[j] = ld3(ys, j);
    v3 yt[153];
    double W[153], om[153];
    cluster_weights(&r, v, ns, y, ws, yt, W, om);
    v3 xx = ld3(x, 0);
    double a = 0.0, b = 0.0;
    for (int m = 0; m < r.M; m++) pot_term(xx, yt[m], W[m], &a);
    rc = pc_literal_pot(&r, v, yt, om, xx, &b);
    *prx = a;
    *lit = b;
    free(y);
    ref_free(&r);
    return rc;
}

/* ------------------------------------------------------------------------------------- */
/* Tree-code velocity (Sec. 3): PC interactions with the far triangles of each target
 * leaf's list, PP interactions with its near triangles, j = i excluded.  literal != 0 uses
 * the alpha-solve for every PC interaction (tiny n only).  vel[n,3] in original order.
 * stats[0] = PC interactions (targets x proxy points), stats[1] = PP interactions
 * (target, source) pairs with j != i.                                                    */
static int tree_sum(or_tree* tr, const double* zeta, const double* area, double theta, int d, int literal,
                    int pot, double* out, int64_t* stats, int nthreads)
{
    if (!tr || d < 1 || d > 16 || !(theta > 0.0) || !(theta < 1.0) || !out) return OR_ERR_ARG;
    if (tr->n > 0 && (!zeta || !area)) return OR_ERR_ARG;
    if (!tr->has_lists || tr->theta != theta) {
        int rc = or_tree_lists(tr, theta);
        if (rc) return rc;
    }
    const int64_t n = tr->n;
    refdata r;
    int rc = ref_make(d, &r);
    if (rc != OR_OK) {
        ref_free(&r);
        return rc;
    }
    const int M = r.M;
    size_t nn = (size_t)(n > 0 ? n : 1);
    /* sorted copies: ys[k] = x_{perm[k]}, ws[k] = zeta A at perm[k] */
    v3* ys = (v3*)malloc(sizeof(v3) * nn);
    double* ws = (double*)malloc(sizeof(double) * nn);
    int32_t* slot = (int32_t*)malloc(sizeof(int32_t) * (size_t)(tr->nnodes > 0 ? tr->nnodes : 1));
    if (!ys || !ws || !slot) {
        free(ys); free(ws); free(slot); ref_free(&r);
        return OR_ERR_MEM;
    }
    for (int64_t k = 0; k < n; k++) {
        int64_t i = tr->perm[k];
        ys[k] = ld3(tr->pos, i);
        ws[k] = zeta[i] * area[i];
    }
    int64_t nclu = 0;
    for (int64_t id = 0; id < tr->nnodes; id++) slot[id] = tr->nodes[id].count > tr->leaf_size ? (int32_t)nclu++ : -1;
    v3* yt = (v3*)malloc(sizeof(v3) * (size_t)(nclu > 0 ? nclu : 1) * M);
    double* W = (double*)malloc(sizeof(double) * (size_t)(nclu > 0 ? nclu : 1) * M);
    double* om = (double*)malloc(sizeof(double) * (size_t)(nclu > 0 ? nclu : 1) * M);
    if (!yt || !W || !om) {
        free(ys); free(ws); free(slot); free(yt); free(W); free(om); ref_free(&r);
        return OR_ERR_MEM;
    }
    for (int64_t id = 0; id < tr->nnodes; id++) {
        if (slot[id] < 0) continue;
        const onode* nd = &tr->nodes[id];
        cluster_weights(&r, nd->v, nd->count, ys + nd->start, ws + nd->start, yt + (size_t)slot[id] * M,
                        W + (size_t)slot[id] * M, om + (size_t)slot[id] * M);
    }
    const double f = -1.0 / (4.0 * OR_PI);
    int64_t npc = 0, npp = 0;
    int err = 0;
    int nth = set_threads(nthreads);
    (void)nth;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nth) reduction(+ : npc, npp) reduction(| : err)
    for (int64_t L = 0; L < tr->nleaves; L++) {
        const onode* t = &tr->nodes[tr->leaves[L]];
        for (int64_t k = t->start; k < t->start + t->count; k++) {
            v3 x = ys[k];
            v3 acc = mk(0.0, 0.0, 0.0);  /* velocity */
            double ph = 0.0;             /* potential */
            for (int64_t q = tr->far_off[L]; q < tr->far_off[L + 1]; q++) {
                int32_t s = tr->far_idx[q];
                const v3* y = yt + (size_t)slot[s] * M;
                const double* Wm = W + (size_t)slot[s] * M;
                if (literal) {
                    if (pot) {
                        double b;
                        if (pc_literal_pot(&r, tr->nodes[s].v, y, om + (size_t)slot[s] * M, x, &b)) err = 1;
                        ph += b;
                    } else {
                        v3 b;
                        if (pc_literal(&r, tr->nodes[s].v, y, om + (size_t)slot[s] * M, x, &b)) err = 1;
                        acc.x += b.x;
                        acc.y += b.y;
                        acc.z += b.z;
                    }
                } else if (pot) {
                    for (int m = 0; m < M; m++) pot_term(x, y[m], Wm[m], &ph);
                } else {
                    for (int m = 0; m < M; m++) bs_term(x, y[m], Wm[m], &acc);
                }
                npc += M;
            }
            for (int64_t q = tr->near_off[L]; q < tr->near_off[L + 1]; q++) {
                const onode* s = &tr->nodes[tr->near_idx[q]];
                for (int64_t j = s->start; j < s->start + s->count; j++) {
                    if (j == k) continue;
                    if (pot)
                        pot_term(x, ys[j], ws[j], &ph);
                    else
                        bs_term(x, ys[j], ws[j], &acc);
                    npp++;
                }
            }
            int64_t i = tr->perm[k];
            if (pot) {
                out[i] = f * ph;
            } else {
                out[3 * i] = f * acc.x;
                out[3 * i + 1] = f * acc.y;
                out[3 * i + 2] = f * acc.z;
            }
        }
    }
    if (stats) {
        stats[0] = npc;
        stats[1] = npp;
    }
    free(ys); free(ws); free(slot); free(yt); free(W); free(om);
    ref_free(&r);
    return err ? OR_ERR_ARG : OR_OK;
}

int or_tree_velocity(or_tree* tr, const double* zeta, const double* area, double theta, int d,
                     int literal, double* vel, int64_t* stats, int nthreads)
{
    return tree_sum(tr, zeta, area, theta, d, literal, 0, vel, stats, nthreads);
}

/* Tree-code stream function (Sec. 3 applied to the potential kernel G of Sec. 2): the same
 * lists, proxy points and proxy weights as or_tree_velocity (the weights do not depend on
 * the kernel), PC as sum_m G(x, y~_m) W_m and PP as sum_j G(x, y_j) zeta_j A_j, j = i
 * excluded.  psi[n] in original order; literal and stats as for the velocity.             */
int or_tree_potential(or_tree* tr, const double* zeta, const double* area, double theta, int d,
                      int literal, double* psi, int64_t* stats, int nthreads)
{
    return tree_sum(tr, zeta, area, theta, d, literal, 1, psi, stats, nthreads);
}

/* Tree-code velocity by the dual traversal (Sec. 3.3, 3.4): PP and PC at the target leaves as
 * in tree_sum; CP and CC accumulate the kernel sum U_T = S at the proxy points of each target
 * cluster T (bs_sum: the velocity is -(1/4pi) x x S, so the interpolated field keeps the
 * velocity tangent to the sphere), from the source particles, resp. the source proxies with
 * their weights W; then the interpolating polynomial of U_T over T (solve V_T c = U_T,
 * V_T[m][k] = B_k(b(x~_m)), the SBB basis in T's barycentric coordinates) is evaluated at every
 * particle below T.  A particle's velocity sums its leaf's PP and PC pairs in traversal order,
 * plus x crossed with the sum of the interpolants of its cluster ancestors from the root down
 * (its own leaf last when that is a cluster at the depth limit).  stats[0..4]: PP (target, source) particle pairs with j != i,
 * PC target x proxy, CP proxy x source, CC proxy x proxy, downward particle x M.            */
static int64_t* group_by(const int32_t* key, int64_t n, int64_t nkeys, int64_t** order)
{
    int64_t* off = (int64_t*)calloc((size_t)nkeys + 1, sizeof(int64_t));
    int64_t* ord = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!off || !ord) {
        free(off);
        free(ord);
        return NULL;
    }
    for (int64_t q = 0; q < n; q++) off[key[q] + 1]++;
    for (int64_t k = 0; k < nkeys; k++) off[k + 1] += off[k];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nkeys > 0 ? nkeys : 1));
    if (!fill) {
        free(off);
        free(ord);
        return NULL;
    }
    memcpy(fill, off, sizeof(int64_t) * (size_t)nkeys);
    for (int64_t q = 0; q < n; q++) ord[fill[key[q]]++] = q;  /* stable: traversal order kept */
    free(fill);
    *order = ord;
    return off;
}

int or_tree_velocity_dual(or_tree* tr, const double* zeta, const double* area, double theta, int d,
                          double* vel, int64_t* stats, int nthreads)
{
    if (!tr || d < 1 || d > 16 || !(theta > 0.0) || !(theta < 1.0) || !vel) return OR_ERR_ARG;
    if (tr->n > 0 && (!zeta || !area)) return OR_ERR_ARG;
    if (!tr->has_dual || tr->dual_theta != theta) {
        int rc = or_dual_lists(tr, theta, NULL);
        if (rc) return rc;
    }
    const int64_t n = tr->n, nn = tr->nnodes;
    refdata r;
    int rc = ref_make(d, &r);
    if (rc != OR_OK) {
        ref_free(&r);
        return rc;
    }
    const int M = r.M;
    size_t n1 = (size_t)(n > 0 ? n : 1);
    v3* ys = (v3*)malloc(sizeof(v3) * n1);
    double* ws = (double*)malloc(sizeof(double) * n1);
    int32_t* slot = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nn > 0 ? nn : 1));
    if (!ys || !ws || !slot) {
        free(ys); free(ws); free(slot); ref_free(&r);
        return OR_ERR_MEM;
    }
    for (int64_t k = 0; k < n; k++) {
        int64_t i = tr->perm[k];
        ys[k] = ld3(tr->pos, i);
        ws[k] = zeta[i] * area[i];
    }
    int64_t nclu = 0;
    for (int64_t id = 0; id < nn; id++) slot[id] = tr->nodes[id].count > tr->leaf_size ? (int32_t)nclu++ : -1;
    size_t c1 = (size_t)(nclu > 0 ? nclu : 1) * M;
    v3* yt = (v3*)malloc(sizeof(v3) * c1);
    double* W = (double*)malloc(sizeof(double) * c1);
    double* om = (double*)malloc(sizeof(double) * c1);
    v3* U = (v3*)calloc(c1, sizeof(v3));
    v3* cf = (v3*)calloc(c1, sizeof(v3));
    char* has = (char*)calloc((size_t)(nclu > 0 ? nclu : 1), 1);
    int64_t *offs[4] = {NULL, NULL, NULL, NULL}, *ords[4] = {NULL, NULL, NULL, NULL};
    int err = !yt || !W || !om || !U || !cf || !has;
    for (int k = 0; k < 4 && !err; k++)
        if (!(offs[k] = group_by(tr->dual_t[k], tr->dual_n[k], nn, &ords[k]))) err = 1;
    if (!err) {
        for (int64_t id = 0; id < nn; id++) {
            if (slot[id] < 0) continue;
            const onode* nd = &tr->nodes[id];
            cluster_weights(&r, nd->v, nd->count, ys + nd->start, ws + nd->start, yt + (size_t)slot[id] * M,
                            W + (size_t)slot[id] * M, om + (size_t)slot[id] * M);
        }
    }
    int64_t nst[5] = {0, 0, 0, 0, 0};
    int nth = set_threads(nthreads);
    (void)nth;
    /* CP and CC: velocity at the proxy points of every target cluster */
    if (!err) {
        int64_t ncp = 0, ncc = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nth) reduction(+ : ncp, ncc) reduction(| : err)
        for (int64_t T = 0; T < nn; T++) {
            if (slot[T] < 0) continue;
            const int64_t b0 = offs[KCP][T], b1 = offs[KCP][T + 1], c0 = offs[KCC][T], c1e = offs[KCC][T + 1];
            if (b0 == b1 && c0 == c1e) continue;
            has[slot[T]] = 1;
            const v3* xt = yt + (size_t)slot[T] * M;
            v3* Ut = U + (size_t)slot[T] * M;
            for (int m = 0; m < M; m++) {
                v3 acc = mk(0.0, 0.0, 0.0);
                for (int64_t q = b0; q < b1; q++) {
                    const onode* sn = &tr->nodes[tr->dual_s[KCP][ords[KCP][q]]];
                    for (int64_t j = sn->start; j < sn->start + sn->count; j++) bs_sum(xt[m], ys[j], ws[j], &acc);
                    ncp += sn->count;
                }
                for (int64_t q = c0; q < c1e; q++) {
                    const int32_t sid = tr->dual_s[KCC][ords[KCC][q]];
                    const v3* y = yt + (size_t)slot[sid] * M;
                    const double* Wm = W + (size_t)slot[sid] * M;
                    for (int mm = 0; mm < M; mm++) bs_sum(xt[m], y[mm], Wm[mm], &acc);
                    ncc += M;
                }
                Ut[m] = acc;
            }
            /* interpolating polynomial over T: V_T c = U_T, three right-hand sides */
            double* V = (double*)malloc(sizeof(double) * (size_t)M * M);
            double* rhs = (double*)malloc(sizeof(double) * (size_t)M * 3);
            if (!V || !rhs) {
                free(V);
                free(rhs);
                err = 1;
                continue;
            }
            const onode* tn = &tr->nodes[T];
            for (int m = 0; m < M; m++) {
                double b[3];
                sph_bary(xt[m], tn->v[0], tn->v[1], tn->v[2], b);
                sbb(d, b[0], b[1], b[2], V + (size_t)m * M);
                rhs[3 * m] = Ut[m].x;
                rhs[3 * m + 1] = Ut[m].y;
                rhs[3 * m + 2] = Ut[m].z;
            }
            if (solve(M, V, rhs, 3) != OR_OK) err = 1;
            v3* ct = cf + (size_t)slot[T] * M;
            for (int k = 0; k < M; k++) ct[k] = mk(rhs[3 * k], rhs[3 * k + 1], rhs[3 * k + 2]);
            free(V);
            free(rhs);
        }
        nst[2] = ncp;
        nst[3] = ncc;
    }
    /* PP and PC at the target leaves, then the interpolants of the cluster ancestors */
    if (!err) {
        const double f = -1.0 / (4.0 * OR_PI);
        int64_t npp = 0, npc = 0, ndn = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nth) reduction(+ : npp, npc, ndn)
        for (int64_t L = 0; L < tr->nleaves; L++) {
            const int32_t lid = tr->leaves[L];
            const onode* t = &tr->nodes[lid];
            int32_t chain[64];
            int nch = 0;
            for (int32_t a = lid; a >= 0 && nch < 64; a = tr->nodes[a].parent)
                if (slot[a] >= 0 && has[slot[a]]) chain[nch++] = a;
            double B[153];
            for (int64_t k = t->start; k < t->start + t->count; k++) {
                v3 x = ys[k];
                v3 acc = mk(0.0, 0.0, 0.0);
                for (int64_t q = offs[KPP][lid]; q < offs[KPP][lid + 1]; q++) {
                    const onode* sn = &tr->nodes[tr->dual_s[KPP][ords[KPP][q]]];
                    for (int64_t j = sn->start; j < sn->start + sn->count; j++) {
                        if (j == k) continue;
                        bs_term(x, ys[j], ws[j], &acc);
                        npp++;
                    }
                }
                for (int64_t q = offs[KPC][lid]; q < offs[KPC][lid + 1]; q++) {
                    const int32_t sid = tr->dual_s[KPC][ords[KPC][q]];
                    const v3* y = yt + (size_t)slot[sid] * M;
                    const double* Wm = W + (size_t)slot[sid] * M;
                    for (int m = 0; m < M; m++) bs_term(x, y[m], Wm[m], &acc);
                    npc += M;
                }
                v3 sacc = mk(0.0, 0.0, 0.0);  /* interpolated kernel sums, root down */
                for (int c = nch - 1; c >= 0; c--) {
                    const onode* an = &tr->nodes[chain[c]];
                    double b[3];
                    sph_bary(x, an->v[0], an->v[1], an->v[2], b);
                    sbb(d, b[0], b[1], b[2], B);
                    const v3* ct = cf + (size_t)slot[chain[c]] * M;
                    for (int kk = 0; kk < M; kk++) {
                        sacc.x += B[kk] * ct[kk].x;
                        sacc.y += B[kk] * ct[kk].y;
                        sacc.z += B[kk] * ct[kk].z;
                    }
                    ndn += M;
                }
                const v3 xs = vcross(x, sacc);
                int64_t i = tr->perm[k];
                vel[3 * i] = f * (acc.x + xs.x);
                vel[3 * i + 1] = f * (acc.y + xs.y);
                vel[3 * i + 2] = f * (acc.z + xs.z);
            }
        }
        nst[0] = npp;
        nst[1] = npc;
        nst[4] = ndn;
    }
    if (stats)
        for (int k = 0; k < 5; k++) stats[k] = nst[k];
    for (int k = 0; k < 4; k++) {
        free(offs[k]);
        free(ords[k]);
    }
    free(ys); free(ws); free(slot); free(yt); free(W); free(om); free(U); free(cf); free(has);
    ref_free(&r);
    return err ? OR_ERR_MEM : OR_OK;
}

/* Proxy points and weights of every node with more than N_T particles (the clusters), in
 * node order: yt[C,M,3], W[C,M].  Returns C through *nclu.  Needs the same zeta, area as
 * or_tree_velocity.                                                                       */
int or_tree_clusters(const or_tree* tr, const double* zeta, const double* area, int d, int64_t* nclu,
                     int32_t* node_ids, double* yt_out, double* W_out)
{
    if (!tr || d < 1 || d > 16 || !nclu) return OR_ERR_ARG;
    int64_t c = 0;
    for (int64_t id = 0; id < tr->nnodes; id++) c += tr->nodes[id].count > tr->leaf_size;
    *nclu = c;
    if (!yt_out && !W_out && !node_ids) return OR_OK;
    refdata r;
    int rc = ref_make(d, &r);
    if (rc != OR_OK) {
        ref_free(&r);
        return rc;
    }
    const int M = r.M;
    const int64_t n = tr->n;
    v3* ys = (v3*)malloc(sizeof(v3) * (size_t)(n > 0 ? n : 1));
    double* ws = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int64_t k = 0; k < n; k++) {
        int64_t i = tr->perm[k];
        ys[k] = ld3(tr->pos, i);
        ws[k] = zeta[i] * area[i];
    }
    int64_t q = 0;
    for (int64_t id = 0; id < tr->nnodes; id++) {
        const onode* nd = &tr->nodes[id];
        if (nd->count <= tr->leaf_size) continue;
        v3 yt[153];
        double W[153], om[153];
        cluster_weights(&r, nd->v, nd->count, ys + nd->start, ws + nd->start, yt, W, om);
        if (node_ids) node_ids[q] = (int32_t)id;
        for (int m = 0; m < M; m++) {
            if (yt_out) {
                yt_out[((size_t)q * M + m) * 3] = yt[m].x;
                yt_out[((size_t)q * M + m) * 3 + 1] = yt[m].y;
                yt_out[((size_t)q * M + m) * 3 + 2] = yt[m].z;
            }
            if (W_out) W_out[(size_t)q * M + m] = W[m];
        }
        q++;
    }
    free(ys);
    free(ws);
    ref_free(&r);
    return OR_OK;
}

/* Icosahedron of the tree (exported for the tests): V[12,3], F[20,3].                   */
int or_icosahedron(double* V, int32_t* F)
{
    v3 v[12];
    int f[20][3];
    ico_build(v, f);
    for (int i = 0; i < 12; i++) {
        V[3 * i] = v[i].x;
        V[3 * i + 1] = v[i].y;
        V[3 * i + 2] = v[i].z;
    }
    for (int i = 0; i < 20; i++)
        for (int a = 0; a < 3; a++) F[3 * i + a] = f[i][a];
    return OR_OK;
}

/* ------------------------------------------------------------------------------------- */
/* Adaptive mesh refinement of Appendix A.  The particles are the vertices of a triangulation
 * of the sphere (the refined icosahedron) with a tree structure: each leaf triangle may be
 * split into four, up to `levels` times below the base mesh, and merged back.
 *
 * Readings (the appendix gives the criteria and the limits, not the bookkeeping):
 *   mesh      the base triangles come from the caller (faces of the base particles); the
 *             possible refinements are numbered once: level by level, every triangle of the
 *             previous level in order gives the midpoint vertices of its edges (v1 v2),
 *             (v2 v3), (v3 v1), each numbered when first met (shared edges share it), and the
 *             children (v1, m12, m31), (m12, v2, m23), (m31, m23, v3), (m12, m23, m31).
 *   area      A = the spherical excess 2 atan2(|a . (b x c)|, 1 + a.b + b.c + c.a) of the
 *             triangle of the three current corner positions.
 *   criteria  refine a leaf when |A (z1 + z2 + z3) / 3| >= eps1 (the magnitude of its
 *             circulation) or max z - min z >= eps2, below the level limit; merge the four
 *             leaf children of a triangle when neither criterion holds on the parent's corners
 *             and no child is to be refined.  One pass per call: every decision is taken on
 *             the state at the start of the pass, then merges and splits are applied.
 *   new vertex  at a split, a midpoint not alive yet is placed at unit(p_a + p_b) of the
 *             current positions of its edge's ends, with vorticity (z_a + z_b) / 2.
 *   alive     a vertex is a particle when it is a corner of a leaf triangle; its weight is the
 *             sum of A / 3 over the leaf triangles it is a corner of.                       */
typedef struct or_amr {
    int64_t n0, nv;      /* base vertices, all possible vertices */
    int64_t t0, nt;      /* base triangles, all possible triangles */
    int levels;
    int32_t* tv;         /* [nt][3] corners */
    int32_t* tparent;    /* [nt] parent or -1 */
    int32_t* tchild;     /* [nt] first of the four children or -1 (deepest level) */
    int8_t* tlevel;      /* [nt] 0 = base */
    int32_t* vparent;    /* [nv][2] edge ends of a midpoint vertex (-1 for base vertices) */
    uint8_t* tstate;     /* [nt] 0 absent, 1 leaf, 2 split */
    uint8_t* valive;     /* [nv] */
    double *pos, *zeta, *area; /* [nv][3], [nv], [nv] */
} or_amr;

void or_amr_free(or_amr* m)
{
    if (!m) return;
    free(m->tv); free(m->tparent); free(m->tchild); free(m->tlevel); free(m->vparent);
    free(m->tstate); free(m->valive); free(m->pos); free(m->zeta); free(m->area);
    free(m);
}

int or_amr_create(const int32_t* faces, int64_t t0, int64_t n0, int levels, or_amr** out)
{
    if (!faces || !out || t0 < 1 || n0 < 3 || levels < 0 || levels > 6) return OR_ERR_ARG;
    int64_t nt = 0, per = t0;
    for (int l = 0; l <= levels; l++, per *= 4) nt += per;
    /* vertices: at most 3 new ones per triangle that has children (all but the deepest
     * level, t0 4^levels = per / 4 triangles) */
    const int64_t nvmax = n0 + 3 * (nt - per / 4);
    or_amr* m = (or_amr*)calloc(1, sizeof(or_amr));
    if (!m) return OR_ERR_MEM;
    m->n0 = n0; m->t0 = t0; m->nt = nt; m->levels = levels;
    m->tv = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)nt);
    m->tparent = (int32_t*)malloc(sizeof(int32_t) * (size_t)nt);
    m->tchild = (int32_t*)malloc(sizeof(int32_t) * (size_t)nt);
    m->tlevel = (int8_t*)malloc((size_t)nt);
    m->vparent = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)nvmax);
    if (!m->tv || !m->tparent || !m->tchild || !m->tlevel || !m->vparent) {
        or_amr_free(m);
        return OR_ERR_MEM;
    }
    for (int64_t t = 0; t < t0; t++) {
        for (int a = 0; a < 3; a++) {
            if (faces[3 * t + a] < 0 || faces[3 * t + a] >= n0) {
                or_amr_free(m);
                return OR_ERR_ARG;
            }
            m->tv[3 * t + a] = faces[3 * t + a];
        }
        m->tparent[t] = -1;
        m->tlevel[t] = 0;
    }
    for (int64_t v = 0; v < n0; v++) m->vparent[2 * v] = m->vparent[2 * v + 1] = -1;
    int64_t nv = n0, lb = 0, le = t0;
    /* edge -> midpoint map of one level: open addressing on the key lo * nvmax + hi */
    for (int l = 1; l <= levels; l++) {
        const int64_t ntl = le - lb, cap = 8 * ntl + 16;
        int64_t* hk = (int64_t*)malloc(sizeof(int64_t) * (size_t)cap);
        int32_t* hv = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
        if (!hk || !hv) {
            free(hk); free(hv); or_amr_free(m);
            return OR_ERR_MEM;
        }
        for (int64_t q = 0; q < cap; q++) hk[q] = -1;
        int64_t nc = le;
        for (int64_t t = lb; t < le; t++) {
            int32_t mid[3];
            for (int e = 0; e < 3; e++) {
                const int32_t a = m->tv[3 * t + e], b = m->tv[3 * t + (e + 1) % 3];
                const int64_t lo = a < b ? a : b, hi = a < b ? b : a, key = lo * nvmax + hi;
                int64_t q = (int64_t)((uint64_t)key * 0x9E3779B97F4A7C15ull % (uint64_t)cap);
                while (hk[q] != -1 && hk[q] != key) q = (q + 1) % cap;
                if (hk[q] == -1) {
                    hk[q] = key;
                    hv[q] = (int32_t)nv;
                    m->vparent[2 * nv] = a;
                    m->vparent[2 * nv + 1] = b;
                    nv++;
                }
                mid[e] = hv[q];
            }
            const int32_t v1 = m->tv[3 * t], v2 = m->tv[3 * t + 1], v3 = m->tv[3 * t + 2];
            const int32_t m12 = mid[0], m23 = mid[1], m31 = mid[2];
            const int32_t ch[4][3] = {{v1, m12, m31}, {m12, v2, m23}, {m31, m23, v3}, {m12, m23, m31}};
            m->tchild[t] = (int32_t)nc;
            for (int c = 0; c < 4; c++, nc++) {
                for (int a = 0; a < 3; a++) m->tv[3 * nc + a] = ch[c][a];
                m->tparent[nc] = (int32_t)t;
                m->tlevel[nc] = (int8_t)l;
            }
        }
        free(hk);
        free(hv);
        lb = le;
        le = nc;
    }
    for (int64_t t = lb; t < le; t++) m->tchild[t] = -1;
    m->nv = nv;
    m->tstate = (uint8_t*)calloc((size_t)nt, 1);
    m->valive = (uint8_t*)calloc((size_t)nv, 1);
    m->pos = (double*)calloc(3 * (size_t)nv, sizeof(double));
    m->zeta = (double*)calloc((size_t)nv, sizeof(double));
    m->area = (double*)calloc((size_t)nv, sizeof(double));
    if (!m->tstate || !m->valive || !m->pos || !m->zeta || !m->area) {
        or_amr_free(m);
        return OR_ERR_MEM;
    }
    for (int64_t t = 0; t < t0; t++) m->tstate[t] = 1;
    for (int64_t v = 0; v < n0; v++) m->valive[v] = 1;
    *out = m;
    return OR_OK;
}

static double amr_area(const double* pos, const int32_t* tv)
{
    const v3 a = ld3(pos, tv[0]), b = ld3(pos, tv[1]), c = ld3(pos, tv[2]);
    const double det = vdot(a, vcross(b, c));
    const double den = ((1.0 + vdot(a, b)) + vdot(b, c)) + vdot(c, a);
    return 2.0 * atan2(fabs(det), den);
}

static int amr_crit(const or_amr* m, int64_t t, double eps1, double eps2)
{
    const int32_t* tv = m->tv + 3 * t;
    const double z1 = m->zeta[tv[0]], z2 = m->zeta[tv[1]], z3 = m->zeta[tv[2]];
    const double A = amr_area(m->pos, tv);
    const double circ = A * (((z1 + z2) + z3) / 3.0);
    double zmax = z1, zmin = z1;
    if (z2 > zmax) zmax = z2;
    if (z3 > zmax) zmax = z3;
    if (z2 < zmin) zmin = z2;
    if (z3 < zmin) zmin = z3;
    return fabs(circ) >= eps1 || zmax - zmin >= eps2;
}

/* Particle weights: sum of A / 3 over the leaf triangles of each alive vertex (triangles in
 * index order). */
static void amr_areas(or_amr* m)
{
    for (int64_t v = 0; v < m->nv; v++) m->area[v] = 0.0;
    for (int64_t t = 0; t < m->nt; t++) {
        if (m->tstate[t] != 1) continue;
        const double w = amr_area(m->pos, m->tv + 3 * t) / 3.0;
        for (int a = 0; a < 3; a++) m->area[m->tv[3 * t + a]] += w;
    }
}

int or_amr_set(or_amr* m, const double* pos0, const double* zeta0)
{
    if (!m || !pos0 || !zeta0) return OR_ERR_ARG;
    for (int64_t v = 0; v < m->n0; v++) {
        for (int a = 0; a < 3; a++) m->pos[3 * v + a] = pos0[3 * v + a];
        m->zeta[v] = zeta0[v];
    }
    amr_areas(m);
    return OR_OK;
}

int or_amr_step(or_amr* m, double eps1, double eps2, int64_t* counts)
{
    if (!m) return OR_ERR_ARG;
    uint8_t* refine = (uint8_t*)calloc((size_t)m->nt, 1);
    uint8_t* merge = (uint8_t*)calloc((size_t)m->nt, 1);
    uint8_t* alive0 = (uint8_t*)malloc((size_t)m->nv);
    if (!refine || !merge || !alive0) {
        free(refine); free(merge); free(alive0);
        return OR_ERR_MEM;
    }
    memcpy(alive0, m->valive, (size_t)m->nv);
    int64_t nref = 0, nmerge = 0;
    for (int64_t t = 0; t < m->nt; t++)
        if (m->tstate[t] == 1 && m->tlevel[t] < m->levels && amr_crit(m, t, eps1, eps2)) refine[t] = 1;
    for (int64_t t = 0; t < m->nt; t++) {
        if (m->tstate[t] != 2) continue;
        const int32_t c0 = m->tchild[t];
        int ok = 1;
        for (int c = 0; c < 4; c++) ok = ok && m->tstate[c0 + c] == 1 && !refine[c0 + c];
        if (ok && !amr_crit(m, t, eps1, eps2)) merge[t] = 1;
    }
    for (int64_t t = 0; t < m->nt; t++) {
        if (merge[t]) {
            m->tstate[t] = 1;
            for (int c = 0; c < 4; c++) m->tstate[m->tchild[t] + c] = 0;
            nmerge++;
        }
        if (refine[t]) {
            m->tstate[t] = 2;
            const int32_t c0 = m->tchild[t];
            for (int c = 0; c < 4; c++) m->tstate[c0 + c] = 1;
            /* midpoints: the corners of the centre child (m12, m23, m31) */
            for (int a = 0; a < 3; a++) {
                const int32_t v = m->tv[3 * (c0 + 3) + a];
                if (alive0[v]) continue;
                const int32_t pa = m->vparent[2 * v], pb = m->vparent[2 * v + 1];
                const double sx = m->pos[3 * pa] + m->pos[3 * pb];
                const double sy = m->pos[3 * pa + 1] + m->pos[3 * pb + 1];
                const double sz = m->pos[3 * pa + 2] + m->pos[3 * pb + 2];
                const double r = sqrt((sx * sx + sy * sy) + sz * sz);
                m->pos[3 * v] = sx / r;
                m->pos[3 * v + 1] = sy / r;
                m->pos[3 * v + 2] = sz / r;
                m->zeta[v] = (m->zeta[pa] + m->zeta[pb]) * 0.5;
            }
            nref++;
        }
    }
    /* alive vertices: the corners of leaf triangles; a removed vertex's state is cleared */
    memset(m->valive, 0, (size_t)m->nv);
    for (int64_t t = 0; t < m->nt; t++)
        if (m->tstate[t] == 1)
            for (int a = 0; a < 3; a++) m->valive[m->tv[3 * t + a]] = 1;
    for (int64_t v = 0; v < m->nv; v++)
        if (!m->valive[v]) {
            m->pos[3 * v] = m->pos[3 * v + 1] = m->pos[3 * v + 2] = 0.0;
            m->zeta[v] = 0.0;
        }
    amr_areas(m);
    if (counts) {
        int64_t na = 0, nl = 0;
        for (int64_t v = 0; v < m->nv; v++) na += m->valive[v];
        for (int64_t t = 0; t < m->nt; t++) nl += m->tstate[t] == 1;
        counts[0] = nref;
        counts[1] = nmerge;
        counts[2] = na;
        counts[3] = nl;
    }
    free(refine);
    free(merge);
    free(alive0);
    return OR_OK;
}

int or_amr_info(const or_amr* m, int64_t* info)
{
    if (!m || !info) return OR_ERR_ARG;
    info[0] = m->n0;
    info[1] = m->nv;
    info[2] = m->t0;
    info[3] = m->nt;
    return OR_OK;
}

/* Full state: tables (any pointer may be NULL) and per-vertex / per-triangle state. */
int or_amr_export(const or_amr* m, int32_t* tv, int32_t* tparent, int32_t* tchild, int8_t* tlevel,
                  int32_t* vparent, uint8_t* tstate, uint8_t* valive, double* pos, double* zeta, double* area)
{
    if (!m) return OR_ERR_ARG;
    if (tv) memcpy(tv, m->tv, sizeof(int32_t) * 3 * (size_t)m->nt);
    if (tparent) memcpy(tparent, m->tparent, sizeof(int32_t) * (size_t)m->nt);
    if (tchild) memcpy(tchild, m->tchild, sizeof(int32_t) * (size_t)m->nt);
    if (tlevel) memcpy(tlevel, m->tlevel, (size_t)m->nt);
    if (vparent) memcpy(vparent, m->vparent, sizeof(int32_t) * 2 * (size_t)m->nv);
    if (tstate) memcpy(tstate, m->tstate, (size_t)m->nt);
    if (valive) memcpy(valive, m->valive, (size_t)m->nv);
    if (pos) memcpy(pos, m->pos, sizeof(double) * 3 * (size_t)m->nv);
    if (zeta) memcpy(zeta, m->zeta, sizeof(double) * (size_t)m->nv);
    if (area) memcpy(area, m->area, sizeof(double) * (size_t)m->nv);
    return OR_OK;
}

/* Writes positions and vorticities of the alive vertices (e.g. after a time step): pos[nv,3],
 * zeta[nv] indexed by vertex; entries of vertices that are not alive are ignored. */
int or_amr_update(or_amr* m, const double* pos, const double* zeta)
{
    if (!m || !pos || !zeta) return OR_ERR_ARG;
    for (int64_t v = 0; v < m->nv; v++)
        if (m->valive[v]) {
            for (int a = 0; a < 3; a++) m->pos[3 * v + a] = pos[3 * v + a];
            m->zeta[v] = zeta[v];
        }
    amr_areas(m);
    return OR_OK;
}
