/*
 * Plain FP64 CPU oracle of the Voronoi particle-merging algorithm
 * (Luu, Tueckmantel & Pukhov, "Voronoi particle merging algorithm for PIC
 * codes", Sec. 3 "Algorithm", Steps 1-7).
 *
 * TEST INFRASTRUCTURE ONLY.  The test-suite, the smoke check and the
 * benchmark's CPU-baseline leg are the only users of this file.  It shares no
 * code, header, table or helper with the CUDA library; the two are compared,
 * never combined.
 *
 * The code follows the paper's steps literally and in order, one subset at a
 * time, with a two-pass (mean first, then squared deviations) weighted
 * variance.  Readings of points the paper leaves open:
 *   - L in Delta_x = sigma/L (Eq. cv_x) is the grid-cell size on that axis.
 *   - Delta_p = sigma/|P| (Eq. cv_p): the absolute value of the mean momentum;
 *     sigma == 0 gives Delta = 0, sigma > 0 with P == 0 gives +infinity.
 *   - sigma_l is exactly 0 when every particle of the subset has the same
 *     value on axis l (the exact-arithmetic value; rounding cannot split a
 *     set of identical values).
 *   - Step 3 stops when every Delta is less than or equal to its tolerance.
 *   - Step 4 takes the axis with the largest raw Delta, ties to the lowest
 *     axis in the order x, y, z, p_x, p_y, p_z.
 *   - Step 5: V1 = {q <= Q}, V2 = {q > Q}; Step 6 recurses on V1 then V2, so
 *     the leaves of a cell come out in V1-before-V2 depth-first order.
 *   - Step 7: a leaf becomes (W, X, P); a one-particle leaf is copied
 *     verbatim.  Cells with N <= N_min are copied verbatim (Sec. 3, "Input").
 *   - A cut whose rounded centroid leaves one side empty (possible only when
 *     the exact centroid lies within rounding of an extreme value) ends the
 *     recursion there (leaf) and raises the cut near-tie flag.
 * Near-tie flags, recorded per cell (bit 0 stop test, bit 1 argmax, bit 2
 * cut): some |Delta_l - T_l| <= 1e-9 T_l; the top two Delta within 1e-9
 * relative; some |q_i - Q| <= 64 m eps (sum w|q|)/W on the cut axis.
 *
 * Two optional decision variants (bits of `variant`), off by default:
 *   ORC_VAR_NORMALIZED  Step 4 takes the axis of the largest Delta_l / T_l
 *                       (T_l = T_X or T_P; with T_l = 0 the ratio is +inf
 *                       for Delta_l > 0 and 0 for Delta_l = 0).
 *   ORC_VAR_PNORM       Delta_p uses the length of the mean momentum vector,
 *                       Delta_l = sigma_l / |P| with |P| = sqrt(sum_l P_l^2)
 *                       over the momentum axes, instead of |P_l|.
 * The near-tie flags then refer to the values that the variant compares.
 *
 * Optional energy-conserving replacement (ORC_VAR_CONSERVE_ENERGY; the paper
 * only names the idea of merging into two particles, Sec. 3, remark on
 * energy; the rule below is derived here from the conservation laws): a
 * final set of m >= 3 particles becomes two particles of weight W/2 at the
 * centroid X with momenta P + d and P - d.  They keep W, W P and the total
 * energy E = sum w sqrt(1 + |p|^2) when |P + d| = |P - d| = sqrt(g^2 - 1),
 * g = E / W: d orthogonal to P with |d|^2 = g^2 - 1 - |P|^2, which is >= 0
 * because sqrt(1 + |p|^2) is convex.  Its direction is the momentum axis e_k
 * with the largest sigma_k^2 (1 - Phat_k^2) (Phat = P / |P|, 0 for P = 0),
 * made orthogonal to P; when every such value is 0, the axis with the
 * smallest |P_k|.  With one momentum axis d is along P instead: P +- u with
 * u^2 = g^2 (g^2 - 1 - P^2) / (g^2 - P^2) (from sqrt(1 + (P + u)^2) +
 * sqrt(1 + (P - u)^2) = 2 g).  Sets of one or two particles are copied
 * verbatim (a pair in ascending input index); the members of a larger set
 * map to its first output.
 */
#include <float.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_INPUT 2
#define ORC_ERR_NOMEM 3

#define ORC_NEAR_STOP 1u
#define ORC_NEAR_ARGMAX 2u
#define ORC_NEAR_CUT 4u

#define ORC_MAXD 6
#define ORC_NEAR_REL 1e-9

#define ORC_VAR_NORMALIZED 2u
#define ORC_VAR_PNORM 4u
#define ORC_VAR_CONSERVE_ENERGY 8u

typedef struct {
    int dx, dp, D;
    const double *q[ORC_MAXD]; /* q[l][i]: positions (l < dx) then momenta */
    const double *w;
    double L[3];
    double tol_x, tol_p;
    unsigned variant;
} orc_problem;

typedef struct {
    double W;
    double Q[ORC_MAXD];
    double sigma[ORC_MAXD];
    double delta[ORC_MAXD];
} orc_moments;

typedef struct {
    int64_t n_in, n_out;
    int64_t cells_merged, cells_passthrough;
    int64_t splits, leaves;
    int64_t depth_sum, max_depth;
    int64_t near_stop, near_argmax, near_cut, degenerate_cuts;
    double energy_in, energy_out;
} orc_stats;

/* Steps 1-2: centroid (W, X, P), standard deviations and CVs of one subset. */
static void subset_moments(const orc_problem *P, const int64_t *idx, int64_t m,
                           orc_moments *M)
{
    double W = 0.0;
    for (int64_t i = 0; i < m; ++i)
        W += P->w[idx[i]];
    M->W = W;
    for (int l = 0; l < P->D; ++l) {
        const double *q = P->q[l];
        double s = 0.0;
        for (int64_t i = 0; i < m; ++i)
            s += P->w[idx[i]] * q[idx[i]];
        double Q = s / W;
        double v = 0.0, qmin = q[idx[0]], qmax = q[idx[0]];
        for (int64_t i = 0; i < m; ++i) {
            double d = q[idx[i]] - Q;
            v += P->w[idx[i]] * (d * d);
            if (q[idx[i]] < qmin) qmin = q[idx[i]];
            if (q[idx[i]] > qmax) qmax = q[idx[i]];
        }
        double sigma = (qmin == qmax) ? 0.0 : sqrt(v / W);
        M->Q[l] = Q;
        M->sigma[l] = sigma;
    }
    /* the momentum scale of Eq. cv_p: |P_l|, or |P| for ORC_VAR_PNORM */
    double pnorm = 0.0;
    if (P->variant & ORC_VAR_PNORM) {
        double s2 = 0.0;
        for (int l = P->dx; l < P->D; ++l)
            s2 += M->Q[l] * M->Q[l];
        pnorm = sqrt(s2);
    }
    for (int l = 0; l < P->D; ++l) {
        double sigma = M->sigma[l], delta;
        double scale = (P->variant & ORC_VAR_PNORM) ? pnorm : fabs(M->Q[l]);
        if (l < P->dx)
            delta = sigma / P->L[l];
        else if (sigma == 0.0)
            delta = 0.0;
        else if (scale == 0.0)
            delta = INFINITY;
        else
            delta = sigma / scale;
        M->delta[l] = delta;
    }
}

/* Step 3: stop test, with the near-tie record of the comparison. */
static int stop_test(const orc_problem *P, const orc_moments *M, unsigned *near)
{
    int stop = 1;
    for (int l = 0; l < P->D; ++l) {
        double T = (l < P->dx) ? P->tol_x : P->tol_p;
        if (!(M->delta[l] <= T))
            stop = 0;
        if (T > 0.0 && fabs(M->delta[l] - T) <= ORC_NEAR_REL * T)
            *near |= ORC_NEAR_STOP;
    }
    return stop;
}

/* The value Step 4 maximises on axis l: Delta_l, or Delta_l / T_l. */
static double axis_score(const orc_problem *P, const orc_moments *M, int l)
{
    double d = M->delta[l];
    if (!(P->variant & ORC_VAR_NORMALIZED))
        return d;
    double T = (l < P->dx) ? P->tol_x : P->tol_p;
    if (T == 0.0)
        return d > 0.0 ? INFINITY : 0.0;
    return d / T;
}

/* Step 4: axis of the largest CV. */
static int split_axis(const orc_problem *P, const orc_moments *M, unsigned *near)
{
    double score[ORC_MAXD];
    for (int l = 0; l < P->D; ++l)
        score[l] = axis_score(P, M, l);
    int k = 0;
    for (int l = 1; l < P->D; ++l)
        if (score[l] > score[k])
            k = l;
    double top = score[k];
    for (int l = 0; l < P->D; ++l) {
        if (l == k) continue;
        double d = score[l];
        if (isinf(top) ? isinf(d) : (d >= top * (1.0 - ORC_NEAR_REL)))
            *near |= ORC_NEAR_ARGMAX;
    }
    return k;
}

typedef struct {
    int64_t begin, end; /* range in the cell's index list */
    int64_t depth;
} orc_range;

typedef struct {
    double W;
    double c[ORC_MAXD]; /* X then P */
} orc_leaf;

/* Per-thread scratch. */
typedef struct {
    int64_t *tmp;
    orc_range *stack;
    int64_t cap;
} orc_scratch;

/* Trace record of one node (for invariant tests). */
typedef struct {
    int64_t begin, end, depth;
    int32_t axis; /* -1 for a leaf */
    double Q;
} orc_node;

/*
 * Steps 2-7 on one cell.  idx[0..m) holds the cell's particle ids in
 * ascending input order; it is permuted in place so that every subset stays a
 * contiguous range with V1 before V2.  leaf_of[i] receives the local leaf
 * number of idx[i] (after permutation); leaves[] the centroids in order.
 * Returns the number of leaves.
 */
static int64_t split_cell(const orc_problem *P, int64_t *idx, int64_t m,
                          int64_t *leaf_of, orc_leaf *leaves, orc_scratch *S,
                          unsigned *near_flags, orc_stats *st,
                          orc_node *trace, int64_t *n_trace)
{
    int64_t n_leaves = 0, sp = 0;
    S->stack[sp++] = (orc_range){0, m, 0};
    while (sp > 0) {
        orc_range r = S->stack[--sp];
        int64_t *sub = idx + r.begin;
        int64_t ms = r.end - r.begin;
        orc_moments M;
        subset_moments(P, sub, ms, &M);
        unsigned near = 0;
        int leaf = stop_test(P, &M, &near);
        int k = -1;
        double Qk = 0.0;
        int64_t n1 = 0;
        if (!leaf) {
            k = split_axis(P, &M, &near);
            Qk = M.Q[k];
            const double *q = P->q[k];
            /* cut near-tie scale: bound on the rounding of Q across orders */
            double aq = 0.0;
            for (int64_t i = 0; i < ms; ++i)
                aq += P->w[sub[i]] * fabs(q[sub[i]]);
            double tau = 64.0 * (double)ms * DBL_EPSILON * (aq / M.W);
            for (int64_t i = 0; i < ms; ++i) {
                if (fabs(q[sub[i]] - Qk) <= tau)
                    near |= ORC_NEAR_CUT;
                if (q[sub[i]] <= Qk)
                    ++n1;
            }
            if (n1 == 0 || n1 == ms) {
                leaf = 1;
                near |= ORC_NEAR_CUT;
                if (st) st->degenerate_cuts++;
            }
        }
        if (near_flags) *near_flags |= near;
        if (st) {
            if (near & ORC_NEAR_STOP) st->near_stop++;
            if (near & ORC_NEAR_ARGMAX) st->near_argmax++;
            if (near & ORC_NEAR_CUT) st->near_cut++;
        }
        if (trace) {
            trace[*n_trace] = (orc_node){r.begin, r.end, r.depth,
                                         leaf ? -1 : k, leaf ? 0.0 : Qk};
            ++*n_trace;
        }
        if (leaf) {
            orc_leaf *L = &leaves[n_leaves];
            if (ms == 1) {
                L->W = P->w[sub[0]];
                for (int l = 0; l < P->D; ++l)
                    L->c[l] = P->q[l][sub[0]];
            } else {
                L->W = M.W;
                for (int l = 0; l < P->D; ++l)
                    L->c[l] = M.Q[l];
            }
            for (int64_t i = r.begin; i < r.end; ++i)
                leaf_of[i] = n_leaves;
            ++n_leaves;
            if (st) {
                st->leaves++;
                st->depth_sum += r.depth * ms;
                if (r.depth > st->max_depth) st->max_depth = r.depth;
            }
            continue;
        }
        if (st) st->splits++;
        /* Steps 5-6: stable partition into V1 = {q <= Q} then V2 = {q > Q} */
        const double *q = P->q[k];
        int64_t a = 0, b = n1;
        for (int64_t i = 0; i < ms; ++i) {
            if (q[sub[i]] <= Qk)
                S->tmp[a++] = sub[i];
            else
                S->tmp[b++] = sub[i];
        }
        memcpy(sub, S->tmp, (size_t)ms * sizeof(int64_t));
        /* V2 is pushed first so that V1 is processed first */
        S->stack[sp++] = (orc_range){r.begin + n1, r.end, r.depth + 1};
        S->stack[sp++] = (orc_range){r.begin, r.begin + n1, r.depth + 1};
    }
    return n_leaves;
}

static int setup_problem(orc_problem *P, int dx, int dp, const double *pos,
                         const double *mom, int64_t stride, const double *w,
                         const double *cell_size, double tol_x, double tol_p,
                         unsigned variant)
{
    if (dx < 1 || dx > 3 || dp < 1 || dp > 3)
        return ORC_ERR_ARG;
    if (variant & ~(ORC_VAR_NORMALIZED | ORC_VAR_PNORM | ORC_VAR_CONSERVE_ENERGY))
        return ORC_ERR_ARG;
    P->variant = variant;
    if (!(tol_x >= 0.0) || !(tol_p >= 0.0) || isinf(tol_x) || isinf(tol_p))
        return ORC_ERR_ARG;
    P->dx = dx;
    P->dp = dp;
    P->D = dx + dp;
    for (int l = 0; l < dx; ++l) {
        P->q[l] = pos + (int64_t)l * stride;
        P->L[l] = cell_size[l];
        if (!(cell_size[l] > 0.0) || isinf(cell_size[l]))
            return ORC_ERR_ARG;
    }
    for (int l = 0; l < dp; ++l)
        P->q[dx + l] = mom + (int64_t)l * stride;
    P->w = w;
    P->tol_x = tol_x;
    P->tol_p = tol_p;
    return ORC_OK;
}

/* ---- exported helpers ------------------------------------------------- */

/* Steps 1-2 for one subset (idx NULL = all m particles).  Outputs W, then
 * Q, sigma and Delta, each of length dx+dp. */
int pma_oracle_subset_moments(int64_t m, int dx, int dp, const double *pos,
                              const double *mom, int64_t stride, const double *w,
                              const int64_t *idx, const double *cell_size,
                              double *W, double *Q, double *sigma, double *delta,
                              unsigned variant)
{
    orc_problem P;
    int rc = setup_problem(&P, dx, dp, pos, mom, stride, w, cell_size, 0.0, 0.0, variant);
    if (rc) return rc;
    if (m < 1) return ORC_ERR_ARG;
    int64_t *all = NULL;
    if (!idx) {
        all = (int64_t *)malloc((size_t)m * sizeof(int64_t));
        if (!all) return ORC_ERR_NOMEM;
        for (int64_t i = 0; i < m; ++i) all[i] = i;
        idx = all;
    }
    orc_moments M;
    subset_moments(&P, idx, m, &M);
    *W = M.W;
    for (int l = 0; l < P.D; ++l) {
        Q[l] = M.Q[l];
        sigma[l] = M.sigma[l];
        delta[l] = M.delta[l];
    }
    free(all);
    return ORC_OK;
}

/* The whole recursion on one particle set, with its tree: perm[m] is the
 * final order (each node a contiguous range), nodes[] the nodes in
 * depth-first (V1 first) preorder; capacity 2m.  Returns the node count in
 * *n_nodes and the near-tie bits in *near. */
int pma_oracle_trace(int64_t m, int dx, int dp, const double *pos,
                     const double *mom, const double *w, const double *cell_size,
                     double tol_x, double tol_p, int64_t *perm,
                     int64_t *node_begin, int64_t *node_end, int64_t *node_depth,
                     int32_t *node_axis, double *node_Q, int64_t *n_nodes,
                     uint32_t *near, unsigned variant)
{
    orc_problem P;
    int rc = setup_problem(&P, dx, dp, pos, mom, m, w, cell_size, tol_x, tol_p, variant);
    if (rc) return rc;
    if (m < 1) return ORC_ERR_ARG;
    orc_scratch S;
    S.tmp = (int64_t *)malloc((size_t)m * sizeof(int64_t));
    S.stack = (orc_range *)malloc((size_t)(m + 1) * sizeof(orc_range));
    int64_t *leaf_of = (int64_t *)malloc((size_t)m * sizeof(int64_t));
    orc_leaf *leaves = (orc_leaf *)malloc((size_t)m * sizeof(orc_leaf));
    orc_node *tr = (orc_node *)malloc((size_t)(2 * m) * sizeof(orc_node));
    if (!S.tmp || !S.stack || !leaf_of || !leaves || !tr) {
        free(S.tmp); free(S.stack); free(leaf_of); free(leaves); free(tr);
        return ORC_ERR_NOMEM;
    }
    for (int64_t i = 0; i < m; ++i) perm[i] = i;
    int64_t nt = 0;
    unsigned nf = 0;
    split_cell(&P, perm, m, leaf_of, leaves, &S, &nf, NULL, tr, &nt);
    for (int64_t j = 0; j < nt; ++j) {
        node_begin[j] = tr[j].begin;
        node_end[j] = tr[j].end;
        node_depth[j] = tr[j].depth;
        node_axis[j] = tr[j].axis;
        node_Q[j] = tr[j].Q;
    }
    *n_nodes = nt;
    *near = nf;
    free(S.tmp); free(S.stack); free(leaf_of); free(leaves); free(tr);
    return ORC_OK;
}

/* ---- full merge over all cells ---------------------------------------- */

typedef struct {
    const orc_problem *P;
    const int64_t *cell_begin; /* [n_cells + 1] into order[] */
    int64_t *order;            /* particle ids grouped by cell */
    int64_t *leaf_of;          /* [n] local leaf id per order[] position */
    orc_leaf *leaves;          /* [n] leaf records at the cell's begin */
    int64_t *n_leaves;         /* [n_cells] */
    uint8_t *flags;            /* [n_cells] or NULL */
    int64_t n_cells;
    int n_min;
    int64_t next;              /* atomic work counter */
    int64_t max_cell;
    orc_stats *thread_stats;
    int fail;
} orc_job;

typedef struct {
    orc_job *job;
    int tid;
} orc_worker_arg;

static void *worker(void *arg_)
{
    orc_worker_arg *arg = (orc_worker_arg *)arg_;
    orc_job *J = arg->job;
    orc_stats *st = &J->thread_stats[arg->tid];
    orc_scratch S;
    S.cap = J->max_cell;
    S.tmp = (int64_t *)malloc((size_t)(S.cap + 1) * sizeof(int64_t));
    S.stack = (orc_range *)malloc((size_t)(S.cap + 2) * sizeof(orc_range));
    if (!S.tmp || !S.stack) {
        __atomic_store_n(&J->fail, 1, __ATOMIC_SEQ_CST);
        free(S.tmp); free(S.stack);
        return NULL;
    }
    const int64_t chunk = 16;
    for (;;) {
        int64_t c0 = __atomic_fetch_add(&J->next, chunk, __ATOMIC_RELAXED);
        if (c0 >= J->n_cells) break;
        int64_t c1 = c0 + chunk < J->n_cells ? c0 + chunk : J->n_cells;
        for (int64_t c = c0; c < c1; ++c) {
            int64_t b = J->cell_begin[c], m = J->cell_begin[c + 1] - b;
            if (m == 0) { J->n_leaves[c] = 0; continue; }
            if (m <= J->n_min || m == 1) {
                /* Input: N <= N_min, or a single particle: copied verbatim */
                for (int64_t i = 0; i < m; ++i) {
                    int64_t id = J->order[b + i];
                    orc_leaf *L = &J->leaves[b + i];
                    L->W = J->P->w[id];
                    for (int l = 0; l < J->P->D; ++l)
                        L->c[l] = J->P->q[l][id];
                    J->leaf_of[b + i] = i;
                }
                J->n_leaves[c] = m;
                st->cells_passthrough++;
                continue;
            }
            unsigned nf = 0;
            J->n_leaves[c] = split_cell(J->P, J->order + b, m, J->leaf_of + b,
                                        J->leaves + b, &S, &nf, st, NULL, NULL);
            if (J->flags) J->flags[c] = (uint8_t)nf;
            st->cells_merged++;
        }
    }
    free(S.tmp);
    free(S.stack);
    return NULL;
}

static double kinetic(const orc_problem *P, int64_t i, const double *const *mom)
{
    double p2 = 0.0;
    for (int l = 0; l < P->dp; ++l)
        p2 += mom[l][i] * mom[l][i];
    return sqrt(1.0 + p2) - 1.0;
}

/* ORC_VAR_CONSERVE_ENERGY: the two momenta a, b that replace the set ids[ms]
 * (ms >= 3) with weight W and centroid momentum Pm (see the header). */
static void energy_pair(const orc_problem *P, const int64_t *ids, int64_t ms, double W,
                        const double *Pm, double *a, double *b)
{
    const int dp = P->dp, dx = P->dx;
    double E = 0.0;
    for (int64_t i = 0; i < ms; ++i) {
        double p2 = 0.0;
        for (int l = 0; l < dp; ++l)
            p2 += P->q[dx + l][ids[i]] * P->q[dx + l][ids[i]];
        E += P->w[ids[i]] * sqrt(1.0 + p2);
    }
    double g = E / W;
    double P2 = 0.0;
    for (int l = 0; l < dp; ++l)
        P2 += Pm[l] * Pm[l];
    if (dp == 1) {
        double u2 = g * g * (g * g - 1.0 - P2) / (g * g - P2);
        double u = sqrt(u2 > 0.0 ? u2 : 0.0);
        a[0] = Pm[0] + u;
        b[0] = Pm[0] - u;
        return;
    }
    double nP = sqrt(P2), ph[3] = {0.0, 0.0, 0.0};
    if (nP > 0.0)
        for (int l = 0; l < dp; ++l)
            ph[l] = Pm[l] / nP;
    /* sigma_k^2, two-pass about the centroid */
    int k = -1;
    double best = 0.0;
    for (int l = 0; l < dp; ++l) {
        double v = 0.0;
        for (int64_t i = 0; i < ms; ++i) {
            double d = P->q[dx + l][ids[i]] - Pm[l];
            v += P->w[ids[i]] * d * d;
        }
        double score = (v / W) * (1.0 - ph[l] * ph[l]);
        if (score > best) {
            best = score;
            k = l;
        }
    }
    if (k < 0) {
        k = 0;
        for (int l = 1; l < dp; ++l)
            if (fabs(Pm[l]) < fabs(Pm[k]))
                k = l;
    }
    /* e_k minus its component along P, normalised */
    double dir[3], n2 = 0.0;
    for (int l = 0; l < dp; ++l) {
        dir[l] = (l == k ? 1.0 : 0.0) - ph[k] * ph[l];
        n2 += dir[l] * dir[l];
    }
    double d2 = g * g - 1.0 - P2;
    double s = sqrt(d2 > 0.0 ? d2 : 0.0) / sqrt(n2);
    for (int l = 0; l < dp; ++l) {
        a[l] = Pm[l] + s * dir[l];
        b[l] = Pm[l] - s * dir[l];
    }
}

/*
 * Merge every cell.  Inputs: n particles, cell[n] in [0, n_cells), SoA
 * pos[dx][n], mom[dp][n] and w[n] (w > 0, all finite), cell_size[dx],
 * n_min, tol_x, tol_p.  Outputs (capacity n, stride n): out_cell, out_pos,
 * out_mom, out_w in canonical order (cells ascending, leaves in V1-first
 * depth-first order); out_index[i] = output slot of particle i (may be
 * NULL); cell_flags[n_cells] near-tie bits (may be NULL); *out_count = M.
 */
int pma_oracle_merge(int64_t n, const int32_t *cell, int dx, int dp,
                     const double *pos, const double *mom, const double *w,
                     int64_t n_cells, const double *cell_size, int32_t n_min,
                     double tol_x, double tol_p, int n_threads,
                     int32_t *out_cell, double *out_pos, double *out_mom,
                     double *out_w, int32_t *out_index, uint8_t *cell_flags,
                     int64_t *out_count, orc_stats *stats, unsigned variant)
{
    if (n < 0 || n_cells < 1 || n_min < 0 || !out_count)
        return ORC_ERR_ARG;
    orc_problem P;
    int rc = setup_problem(&P, dx, dp, pos, mom, n, w, cell_size, tol_x, tol_p, variant);
    if (rc) return rc;
    for (int64_t i = 0; i < n; ++i) {
        if (cell[i] < 0 || (int64_t)cell[i] >= n_cells) return ORC_ERR_INPUT;
        if (!(w[i] > 0.0) || isinf(w[i])) return ORC_ERR_INPUT;
        for (int l = 0; l < P.D; ++l)
            if (!isfinite(P.q[l][i])) return ORC_ERR_INPUT;
    }
    /* Step 1: collect each cell's particles, ascending input order */
    int64_t *cell_begin = (int64_t *)calloc((size_t)n_cells + 1, sizeof(int64_t));
    int64_t *order = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    int64_t *leaf_of = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    orc_leaf *leaves = (orc_leaf *)malloc((size_t)(n ? n : 1) * sizeof(orc_leaf));
    int64_t *n_leaves = (int64_t *)calloc((size_t)n_cells, sizeof(int64_t));
    int64_t *fill = (int64_t *)calloc((size_t)n_cells, sizeof(int64_t));
    if (!cell_begin || !order || !leaf_of || !leaves || !n_leaves || !fill) {
        free(cell_begin); free(order); free(leaf_of); free(leaves);
        free(n_leaves); free(fill);
        return ORC_ERR_NOMEM;
    }
    for (int64_t i = 0; i < n; ++i)
        cell_begin[cell[i] + 1]++;
    int64_t max_cell = 1;
    for (int64_t c = 0; c < n_cells; ++c) {
        if (cell_begin[c + 1] > max_cell) max_cell = cell_begin[c + 1];
        cell_begin[c + 1] += cell_begin[c];
    }
    for (int64_t i = 0; i < n; ++i) {
        int64_t c = cell[i];
        order[cell_begin[c] + fill[c]++] = i;
    }
    free(fill);
    if (cell_flags) memset(cell_flags, 0, (size_t)n_cells);

    if (n_threads < 1) n_threads = 1;
    orc_stats *ts = (orc_stats *)calloc((size_t)n_threads, sizeof(orc_stats));
    pthread_t *th = (pthread_t *)malloc((size_t)n_threads * sizeof(pthread_t));
    orc_worker_arg *args = (orc_worker_arg *)malloc((size_t)n_threads * sizeof(orc_worker_arg));
    orc_job J = {&P, cell_begin, order, leaf_of, leaves, n_leaves, cell_flags,
                 n_cells, n_min, 0, max_cell, ts, 0};
    if (!ts || !th || !args) {
        J.fail = 1;
    } else if (n_threads == 1) {
        args[0] = (orc_worker_arg){&J, 0};
        worker(&args[0]);
    } else {
        int started = 0;
        for (int t = 0; t < n_threads; ++t) {
            args[t] = (orc_worker_arg){&J, t};
            if (pthread_create(&th[t], NULL, worker, &args[t]) != 0) break;
            ++started;
        }
        if (started == 0) { args[0] = (orc_worker_arg){&J, 0}; worker(&args[0]); }
        for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    }
    if (J.fail) {
        free(cell_begin); free(order); free(leaf_of); free(leaves);
        free(n_leaves); free(ts); free(th); free(args);
        return ORC_ERR_NOMEM;
    }
    /* Step 7: replace each cell's particles by its centroids, compacted */
    int64_t M = 0;
    const double *momp[3] = {mom, mom + n, mom + 2 * n};
    double e_in = 0.0, e_out = 0.0;
    const int ec = (variant & ORC_VAR_CONSERVE_ENERGY) != 0;
    for (int64_t c = 0; c < n_cells; ++c) {
        int64_t b = cell_begin[c], m = cell_begin[c + 1] - b;
        int64_t i0 = 0;  /* the leaves' members are consecutive in order[] */
        for (int64_t j = 0; j < n_leaves[c]; ++j) {
            const orc_leaf *L = &leaves[b + j];
            int64_t i1 = i0;
            while (i1 < m && leaf_of[b + i1] == j)
                ++i1;
            const int64_t ms = i1 - i0;
            /* the outputs of this leaf: 1, or 2 with ORC_VAR_CONSERVE_ENERGY */
            double ow[2], oc[2][ORC_MAXD];
            int nout = 1;
            ow[0] = L->W;
            for (int l = 0; l < P.D; ++l)
                oc[0][l] = L->c[l];
            if (ec && ms == 2) {
                nout = 2;
                int64_t lo = order[b + i0], hi = order[b + i0 + 1];
                if (hi < lo) { int64_t tmp = lo; lo = hi; hi = tmp; }
                for (int t = 0; t < 2; ++t) {
                    int64_t id = t == 0 ? lo : hi;
                    ow[t] = w[id];
                    for (int l = 0; l < P.D; ++l)
                        oc[t][l] = P.q[l][id];
                }
            } else if (ec && ms >= 3) {
                nout = 2;
                ow[0] = ow[1] = 0.5 * L->W;
                for (int l = 0; l < dx; ++l)
                    oc[1][l] = L->c[l];
                energy_pair(&P, order + b + i0, ms, L->W, L->c + dx, oc[0] + dx, oc[1] + dx);
            }
            for (int t = 0; t < nout; ++t) {
                if (out_cell) out_cell[M + t] = (int32_t)c;
                if (out_w) out_w[M + t] = ow[t];
                for (int l = 0; l < dx; ++l)
                    if (out_pos) out_pos[(int64_t)l * n + M + t] = oc[t][l];
                double p2 = 0.0;
                for (int l = 0; l < dp; ++l) {
                    if (out_mom) out_mom[(int64_t)l * n + M + t] = oc[t][dx + l];
                    p2 += oc[t][dx + l] * oc[t][dx + l];
                }
                e_out += ow[t] * (sqrt(1.0 + p2) - 1.0);
            }
            for (int64_t i = i0; i < i1; ++i) {
                int64_t id = order[b + i];
                /* a verbatim pair keeps one output per member, the lower
                   input index first */
                int64_t other = order[b + (i == i0 ? i0 + 1 : i0)];
                int64_t slot = (ec && ms == 2) ? M + (id > other ? 1 : 0) : M;
                if (out_index) out_index[id] = (int32_t)slot;
                e_in += w[id] * kinetic(&P, id, momp);
            }
            M += nout;
            i0 = i1;
        }
    }
    *out_count = M;
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        for (int t = 0; t < n_threads; ++t) {
            stats->cells_merged += ts[t].cells_merged;
            stats->cells_passthrough += ts[t].cells_passthrough;
            stats->splits += ts[t].splits;
            stats->leaves += ts[t].leaves;
            stats->depth_sum += ts[t].depth_sum;
            if (ts[t].max_depth > stats->max_depth) stats->max_depth = ts[t].max_depth;
            stats->near_stop += ts[t].near_stop;
            stats->near_argmax += ts[t].near_argmax;
            stats->near_cut += ts[t].near_cut;
            stats->degenerate_cuts += ts[t].degenerate_cuts;
        }
        stats->n_in = n;
        stats->n_out = M;
        stats->energy_in = e_in;
        stats->energy_out = e_out;
    }
    free(cell_begin); free(order); free(leaf_of); free(leaves);
    free(n_leaves); free(ts); free(th); free(args);
    return ORC_OK;
}
