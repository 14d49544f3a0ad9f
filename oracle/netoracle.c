/*
 * netoracle.c -- plain FP64 CPU oracle for the Kirchhoff network solve.
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline / reference leg may load this library.  The CUDA
 * solver never calls it and shares no code with it.
 *
 * What it computes (Dashtian & Sahimi, arXiv:1908.03301):
 *   * Sec. II: a square (2D) or cubic (3D) bond network; bond ij has
 *     conductance g_ij and carries flow q_ij = g_ij (P_j - P_i).
 *   * Eq. 3:   mass balance sum_j q_ij = 0 at every interior node gives the
 *     linear system G P = b; b collects the bonds to the fixed-pressure faces.
 *   * Sec. II: a fixed pressure drop along one axis (faces x_f = 0 at p_in and
 *     x_f = n_f-1 at p_out).  Each transverse boundary is either no-flow (the
 *     plane has no bond beyond the last node) or periodic, as the paper
 *     states (the last layer's bonds connect to the first layer).
 *   * Eq. 4:   K = (Q/S)(mu L / dP) with Q the total inlet flow, in lattice
 *     units mu = 1, L = n_f - 1, S = product of the transverse node counts.
 *   * Sec. II / IV: G P = b solved by conjugate gradients; the preconditioner
 *     is Jacobi (z = D^-1 r), the textbook preconditioned CG.
 *
 * Clusters (the paper is silent; this is the reading used throughout): nodes
 * joined by open bonds (g > 0) among interior nodes form clusters.  A cluster
 * with open bonds to both faces is "spanning" and is the only part solved.
 * A cluster touching only the inlet face has P = p_in, only the outlet face
 * P = p_out (no current flows in either), an isolated cluster P = 0.  The
 * canonical cluster label is the smallest linear node index in the cluster;
 * inlet-face nodes carry label -1 and outlet-face nodes -2.
 *
 * Layout: node (x,y,z) has linear index x + nx*(y + ny*z).  Bond plane d holds
 * the bond from node c to c + e_d; its extents are the node extents with n_d
 * reduced by one (n_d itself for a periodic axis, whose last layer holds the
 * bonds that wrap to the first), indexed the same way.
 *
 * Sums over nodes use a fixed split into ORC_NCHUNK pieces added in order, so
 * results do not depend on the OpenMP thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_NCHUNK 64

typedef struct {
    int ndim;          /* 2 or 3 */
    int64_t n[3];      /* node extents; n[2] = 1 in 2D */
    int flow_axis;     /* axis of the imposed pressure drop */
    double p_in, p_out;
    unsigned periodic; /* bit d: axis d is periodic (never the flow axis) */
} or_desc;

typedef struct {
    double g_eff;         /* Q_in / (p_in - p_out) */
    double k_eff;         /* Eq. 4 in lattice units */
    double q_in, q_out;   /* total flow through the inlet / outlet faces */
    double rel_residual;  /* ||b - G P||_2 / ||b||_2 (true residual) */
    double max_imbalance; /* max_i |b - G P|_i over solved nodes */
    double energy_g;      /* sum_bonds g dP_b^2 / (p_in - p_out)^2 */
    int64_t n_active;     /* nodes of the spanning cluster(s) */
    int64_t iters;        /* CG iterations */
    int status;           /* 0 ok, 1 not converged, -1 invalid input */
} or_result;

enum { CLS_ISOLATED = 0, CLS_INLET = 1, CLS_OUTLET = 2, CLS_SPANNING = 3,
       CLS_FACE_IN = 4, CLS_FACE_OUT = 5 };

/* ------------------------------------------------------------------ */
/* lattice helpers                                                     */
/* ------------------------------------------------------------------ */
static int64_t n_nodes(const or_desc *d) { return d->n[0] * d->n[1] * d->n[2]; }

static void coords(const or_desc *d, int64_t i, int64_t c[3]) {
    c[0] = i % d->n[0];
    c[1] = (i / d->n[0]) % d->n[1];
    c[2] = i / (d->n[0] * d->n[1]);
}

static int64_t node_index(const or_desc *d, const int64_t c[3]) {
    return c[0] + d->n[0] * (c[1] + d->n[1] * c[2]);
}

static int periodic(const or_desc *d, int dir) { return (d->periodic >> dir) & 1u; }

/* Extent of bond plane dir along axis a: one bond fewer than nodes along dir,
 * unless dir is periodic (the last layer's bonds wrap to the first layer). */
static int64_t plane_extent(const or_desc *d, int dir, int a) {
    return d->n[a] - (a == dir && !periodic(d, dir));
}

/* Conductance of the bond from node c to c + e_dir (the bond must exist). */
static double bond(const or_desc *d, const double *const g[3], int dir, const int64_t c[3]) {
    int64_t m0 = plane_extent(d, dir, 0), m1 = plane_extent(d, dir, 1);
    return g[dir][c[0] + m0 * (c[1] + m1 * c[2])];
}

/* 0 = interior unknown, 1 = inlet face, 2 = outlet face */
static int node_kind(const or_desc *d, const int64_t c[3]) {
    int64_t cf = c[d->flow_axis];
    if (cf == 0) return 1;
    if (cf == d->n[d->flow_axis] - 1) return 2;
    return 0;
}

/*
 * Enumerate the (up to 2*ndim) neighbours of node c.  For k in [0, 2*ndim):
 * direction k/2, sign + for even k.  Returns 0 if that neighbour does not
 * exist, else 1 with *j its index and *gij the bond conductance.
 */
static int neighbour(const or_desc *d, const double *const g[3], const int64_t c[3], int k,
                     int64_t *j, double *gij) {
    int dir = k / 2;
    int64_t cc[3] = {c[0], c[1], c[2]};
    if ((k & 1) == 0) {
        if (c[dir] + 1 >= d->n[dir] && !periodic(d, dir)) return 0;
        *gij = bond(d, g, dir, c);
        cc[dir] = (c[dir] + 1) % d->n[dir];
    } else {
        if (c[dir] == 0 && !periodic(d, dir)) return 0;
        cc[dir] = (c[dir] + d->n[dir] - 1) % d->n[dir];
        *gij = bond(d, g, dir, cc);
    }
    *j = node_index(d, cc);
    return 1;
}

static int validate(const or_desc *d, const double *const g[3]) {
    if (!d || (d->ndim != 2 && d->ndim != 3)) return -1;
    for (int a = 0; a < 3; a++)
        if (d->n[a] < 1) return -1;
    if (d->ndim == 2 && d->n[2] != 1) return -1;
    if (d->flow_axis < 0 || d->flow_axis >= d->ndim) return -1;
    if (d->n[d->flow_axis] < 3) return -1;
    if (d->periodic >> d->ndim) return -1;
    if (periodic(d, d->flow_axis)) return -1;
    for (int dir = 0; dir < d->ndim; dir++)
        if (periodic(d, dir) && d->n[dir] < 3) return -1;
    if (!isfinite(d->p_in) || !isfinite(d->p_out)) return -1;
    if (n_nodes(d) >= ((int64_t)1 << 31)) return -1;
    for (int dir = 0; dir < d->ndim; dir++) {
        int64_t m = 1;
        for (int a = 0; a < 3; a++) m *= plane_extent(d, dir, a);
        for (int64_t b = 0; b < m; b++) {
            double v = g[dir][b];
            if (!(v >= 0.0) || !isfinite(v)) return -1;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* cluster labels                                                      */
/* ------------------------------------------------------------------ */
static int64_t uf_find(int64_t *parent, int64_t i) {
    while (parent[i] != i) {
        parent[i] = parent[parent[i]];
        i = parent[i];
    }
    return i;
}

/* The root of a merged set is the smaller of the two roots, so every root is
 * the smallest index of its set. */
static void uf_union(int64_t *parent, int64_t a, int64_t b) {
    int64_t ra = uf_find(parent, a), rb = uf_find(parent, b);
    if (ra == rb) return;
    if (ra < rb) parent[rb] = ra;
    else parent[ra] = rb;
}

/*
 * Cluster labels and classes.  label[i]: smallest node index of i's cluster
 * (interior nodes), -1 (inlet face), -2 (outlet face).  cls[i]: bit 0 = the
 * cluster has an open bond to the inlet face, bit 1 = to the outlet face;
 * face nodes get CLS_FACE_IN / CLS_FACE_OUT.  Returns 0, or -1 on bad input.
 */
int or_labels(const or_desc *d, const double *const g[3], int32_t *label, uint8_t *cls) {
    if (validate(d, g)) return -1;
    int64_t N = n_nodes(d);
    int64_t *parent = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    uint8_t *flags = (uint8_t *)calloc((size_t)N, 1);
    if (!parent || !flags) {
        free(parent);
        free(flags);
        return -1;
    }
    for (int64_t i = 0; i < N; i++) parent[i] = i;
    int64_t c[3], j;
    double gij;
    for (int64_t i = 0; i < N; i++) {
        coords(d, i, c);
        if (node_kind(d, c) != 0) continue;
        for (int k = 0; k < 2 * d->ndim; k += 2) { /* + neighbours only: each bond once */
            if (!neighbour(d, g, c, k, &j, &gij) || !(gij > 0.0)) continue;
            int64_t cj[3];
            coords(d, j, cj);
            if (node_kind(d, cj) == 0) uf_union(parent, i, j);
        }
    }
    for (int64_t i = 0; i < N; i++) {
        coords(d, i, c);
        int kind = node_kind(d, c);
        if (kind == 1) { label[i] = -1; continue; }
        if (kind == 2) { label[i] = -2; continue; }
        int64_t r = uf_find(parent, i);
        label[i] = (int32_t)r;
        for (int k = 0; k < 2 * d->ndim; k++) {
            if (!neighbour(d, g, c, k, &j, &gij) || !(gij > 0.0)) continue;
            int64_t cj[3];
            coords(d, j, cj);
            int kj = node_kind(d, cj);
            if (kj == 1) flags[r] |= 1;
            if (kj == 2) flags[r] |= 2;
        }
    }
    for (int64_t i = 0; i < N; i++) {
        if (label[i] == -1) cls[i] = CLS_FACE_IN;
        else if (label[i] == -2) cls[i] = CLS_FACE_OUT;
        else cls[i] = flags[label[i]];
    }
    free(parent);
    free(flags);
    return 0;
}

/*
 * Backbone of the spanning clusters: the nodes that remain when dead-end
 * trees are stripped.  A spanning interior node with at most one open bond
 * to nodes still present (face nodes always count as present) carries no
 * current: its only bond has no flow, so its pressure is that of its single
 * neighbour.  Removing such nodes one at a time until none is left gives a
 * unique set (the part of each spanning cluster in which every interior node
 * keeps at least two links, the two faces never removed).  This follows that
 * definition directly with a work list of removable nodes.
 * backbone[i] = 1 for spanning nodes that remain, 0 for every other node.
 * Returns 0, or -1 on bad input.
 */
int or_backbone(const or_desc *d, const double *const g[3], uint8_t *backbone) {
    if (validate(d, g)) return -1;
    const int64_t N = n_nodes(d);
    int32_t *label = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    uint8_t *cls = (uint8_t *)malloc((size_t)N);
    int32_t *deg = (int32_t *)calloc((size_t)N, sizeof(int32_t));
    int64_t *work = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    int rc = -1;
    if (!label || !cls || !deg || !work) goto out;
    if (or_labels(d, g, label, cls)) goto out;
    int64_t c[3], j, top = 0;
    double gij;
    /* present = spanning interior nodes and all face nodes */
    for (int64_t i = 0; i < N; i++) backbone[i] = cls[i] == CLS_SPANNING;
    for (int64_t i = 0; i < N; i++) {
        if (!backbone[i]) continue;
        coords(d, i, c);
        for (int k = 0; k < 2 * d->ndim; k++) {
            if (!neighbour(d, g, c, k, &j, &gij) || !(gij > 0.0)) continue;
            if (backbone[j] || cls[j] == CLS_FACE_IN || cls[j] == CLS_FACE_OUT) deg[i]++;
        }
        if (deg[i] <= 1) work[top++] = i;
    }
    while (top > 0) {
        const int64_t i = work[--top];
        if (!backbone[i]) continue;
        backbone[i] = 0;
        coords(d, i, c);
        for (int k = 0; k < 2 * d->ndim; k++) {
            if (!neighbour(d, g, c, k, &j, &gij) || !(gij > 0.0) || !backbone[j]) continue;
            if (--deg[j] == 1) work[top++] = j;  /* reaches 1 once: pushed once */
        }
    }
    rc = 0;
out:
    free(label);
    free(cls);
    free(deg);
    free(work);
    return rc;
}

/*
 * Current-carrying backbone (Sec. V and VI.B: near the percolation threshold
 * most of the spanning cluster carries no flow).  The graph: the interior
 * nodes joined by their open bonds; all inlet-face nodes taken together as
 * one vertex A and all outlet-face nodes as one vertex B (each face is at one
 * pressure, so it acts as one node); and one extra edge joining A and B.
 * For generic conductances a bond carries current exactly when it lies on a
 * path from A to B that visits no vertex twice, which is exactly when it
 * belongs to the same biconnected component (block) as the extra edge A-B.
 * Every other part of a spanning cluster hangs from that block by a single
 * node (a dead-end tree, or a dead-end loop), or by one face.
 *
 * The blocks come from one depth-first search (Hopcroft and Tarjan 1973):
 * disc[v] is v's discovery time, low[v] the smallest discovery time reachable
 * from v's subtree by one edge that is not a tree edge; edges are pushed on a
 * stack as they are met, and when the search returns from a child w of v with
 * low[w] >= disc[v] the edges above (v, w) on the stack, (v, w) included, are
 * one block.  The lattice has no parallel edges (periodic axes have at least
 * three nodes, and n_f >= 3 keeps the faces apart), so the tree edge to a
 * node's parent is recognised by the parent vertex.
 *
 * backbone[i] = 1 for the interior nodes that are an end of an edge of the
 * block of A-B, 0 for every other node.  Returns 0, or -1 on bad input.
 */
static int faces_kind(const or_desc *d, int64_t j) {
    int64_t c[3];
    coords(d, j, c);
    return node_kind(d, c);
}

int or_backbone_blocks(const or_desc *d, const double *const g[3], uint8_t *backbone) {
    if (validate(d, g)) return -1;
    const int64_t N = n_nodes(d), A = N, B = N + 1, V = N + 2;
    const int nk = 2 * d->ndim;
    int64_t *disc = (int64_t *)calloc((size_t)V, sizeof(int64_t));
    int64_t *low = (int64_t *)malloc(sizeof(int64_t) * (size_t)V);
    int64_t *par = (int64_t *)malloc(sizeof(int64_t) * (size_t)V);
    int64_t *nxt = (int64_t *)calloc((size_t)V, sizeof(int64_t));   /* next neighbour slot */
    int64_t *adjA = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N + 1));
    int64_t *adjB = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N + 1));
    int64_t *dstack = (int64_t *)malloc(sizeof(int64_t) * (size_t)V); /* DFS path */
    int64_t ne_max = (int64_t)d->ndim * N + 2 * N + 1;
    int64_t *eu = (int64_t *)malloc(sizeof(int64_t) * (size_t)ne_max);  /* edge stack */
    int64_t *ew = (int64_t *)malloc(sizeof(int64_t) * (size_t)ne_max);
    int rc = -1;
    if (!disc || !low || !par || !nxt || !adjA || !adjB || !dstack || !eu || !ew) goto out;
    memset(backbone, 0, (size_t)N);

    /* neighbours of the two face vertices: the interior nodes with an open
     * bond to that face, in index order (slot 0 of each is the other face) */
    int64_t nA = 0, nB = 0;
    for (int64_t i = 0; i < N; i++) {
        int64_t c[3], j;
        double gij;
        coords(d, i, c);
        if (node_kind(d, c) != 0) continue;
        for (int k = 0; k < nk; k++) {
            if (!neighbour(d, g, c, k, &j, &gij) || !(gij > 0.0)) continue;
            int kj = faces_kind(d, j);
            if (kj == 1) adjA[nA++] = i;
            if (kj == 2) adjB[nB++] = i;
        }
    }

    int64_t time = 0, top = 0, etop = 0;
    disc[A] = low[A] = ++time;
    par[A] = -1;
    dstack[top++] = A;
    while (top > 0) {
        const int64_t v = dstack[top - 1];
        /* next neighbour w of v, or -1 when v is done */
        int64_t w = -1;
        while (w < 0) {
            const int64_t slot = nxt[v]++;
            if (v == A || v == B) {
                const int64_t *adj = v == A ? adjA : adjB;
                const int64_t na = v == A ? nA : nB;
                if (slot == 0) w = v == A ? B : A;
                else if (slot <= na) w = adj[slot - 1];
                else break;
            } else {
                if (slot >= nk) break;
                int64_t c[3], j;
                double gij;
                coords(d, v, c);
                if (!neighbour(d, g, c, (int)slot, &j, &gij) || !(gij > 0.0)) continue;
                int kj = faces_kind(d, j);
                w = kj == 1 ? A : kj == 2 ? B : j;
            }
        }
        if (w >= 0) {
            if (w == par[v]) continue;
            if (disc[w] == 0) {             /* tree edge: descend */
                eu[etop] = v; ew[etop] = w; etop++;
                par[w] = v;
                disc[w] = low[w] = ++time;
                dstack[top++] = w;
            } else if (disc[w] < disc[v]) { /* edge back to an ancestor */
                eu[etop] = v; ew[etop] = w; etop++;
                if (disc[w] < low[v]) low[v] = disc[w];
            }
            continue;
        }
        /* v is finished: return to its parent u */
        top--;
        const int64_t u = par[v];
        if (u < 0) break;
        if (low[v] < low[u]) low[u] = low[v];
        if (low[v] >= disc[u]) {
            /* the edges above (u, v) on the stack form one block */
            int64_t e = etop;
            int has_ab = 0;
            do {
                e--;
                if ((eu[e] == A && ew[e] == B) || (eu[e] == B && ew[e] == A)) has_ab = 1;
            } while (!(eu[e] == u && ew[e] == v));
            if (has_ab)
                for (int64_t k = e; k < etop; k++) {
                    if (eu[k] < N) backbone[eu[k]] = 1;
                    if (ew[k] < N) backbone[ew[k]] = 1;
                }
            etop = e;
        }
    }
    rc = 0;
out:
    free(disc); free(low); free(par); free(nxt); free(adjA); free(adjB);
    free(dstack); free(eu); free(ew);
    return rc;
}

/* ------------------------------------------------------------------ */
/* vector helpers (fixed-order sums)                                   */
/* ------------------------------------------------------------------ */
static double dot(const double *a, const double *b, int64_t n) {
    double part[ORC_NCHUNK];
#pragma omp parallel for schedule(static)
    for (int ch = 0; ch < ORC_NCHUNK; ch++) {
        int64_t lo = n * ch / ORC_NCHUNK, hi = n * (ch + 1) / ORC_NCHUNK;
        double s = 0.0;
        for (int64_t i = lo; i < hi; i++) s += a[i] * b[i];
        part[ch] = s;
    }
    double s = 0.0;
    for (int ch = 0; ch < ORC_NCHUNK; ch++) s += part[ch];
    return s;
}

/*
 * Nodal current imbalance of a full pressure field P (face nodes included):
 * out_i = sum_{open j} g_ij (P_j - P_i) for interior nodes, 0 on the faces.
 * This is (b - G P)_i of Eq. 3 once P holds the face pressures.
 */
int or_residual(const or_desc *d, const double *const g[3], const double *P, double *out) {
    if (validate(d, g)) return -1;
    int64_t N = n_nodes(d);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; i++) {
        int64_t c[3], j;
        double gij, s = 0.0;
        coords(d, i, c);
        if (node_kind(d, c) != 0) { out[i] = 0.0; continue; }
        for (int k = 0; k < 2 * d->ndim; k++)
            if (neighbour(d, g, c, k, &j, &gij)) s += gij * (P[j] - P[i]);
        out[i] = s;
    }
    return 0;
}

/*
 * y = G v restricted to the solved (active) nodes: for active i,
 * y_i = D_i v_i - sum_{active j} g_ij v_j, with D_i the sum of all open bonds at
 * i (bonds to face nodes included).  y_i = 0 elsewhere.
 */
static void apply_G(const or_desc *d, const double *const g[3], const uint8_t *active,
                    const double *D, const double *v, double *y) {
    int64_t N = n_nodes(d);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; i++) {
        if (!active[i]) { y[i] = 0.0; continue; }
        int64_t c[3], j;
        double gij, s = D[i] * v[i];
        coords(d, i, c);
        for (int k = 0; k < 2 * d->ndim; k++)
            if (neighbour(d, g, c, k, &j, &gij) && active[j]) s -= gij * v[j];
        y[i] = s;
    }
}

/* ------------------------------------------------------------------ */
/* the solve                                                           */
/* ------------------------------------------------------------------ */
/*
 * Solve Eq. 3 on the spanning cluster with Jacobi-preconditioned CG to
 * ||b - G P||_2 <= tol ||b||_2, starting from the linear pressure profile
 * along the flow axis; then the flows and Eq. 4.
 *
 *   P     [out] N pressures (faces and non-spanning clusters included).
 *   label [out, optional] N cluster labels; cls [out, optional] N classes.
 * nthreads <= 0 keeps the OpenMP default.  Returns res->status.
 */
int or_solve(const or_desc *d, const double *const g[3], double tol, int64_t max_iter,
             int nthreads, double *P, int32_t *label_out, uint8_t *cls_out, or_result *res) {
    memset(res, 0, sizeof(*res));
    if (validate(d, g)) { res->status = -1; return -1; }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    int64_t N = n_nodes(d);
    int f = d->flow_axis;
    double dP = d->p_in - d->p_out;
    int32_t *label = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    uint8_t *cls = (uint8_t *)malloc((size_t)N);
    uint8_t *active = (uint8_t *)malloc((size_t)N);
    double *D = (double *)calloc((size_t)N, sizeof(double));
    double *b = (double *)calloc((size_t)N, sizeof(double));
    double *x = (double *)calloc((size_t)N, sizeof(double));
    double *r = (double *)calloc((size_t)N, sizeof(double));
    double *z = (double *)calloc((size_t)N, sizeof(double));
    double *p = (double *)calloc((size_t)N, sizeof(double));
    double *q = (double *)calloc((size_t)N, sizeof(double));
    if (!label || !cls || !active || !D || !b || !x || !r || !z || !p || !q) {
        res->status = -1;
        goto done;
    }
    or_labels(d, g, label, cls);

    /* initial pressures: faces, linear profile on the spanning cluster,
     * face pressure on one-sided clusters, 0 on isolated ones */
    int64_t n_active = 0;
    for (int64_t i = 0; i < N; i++) {
        int64_t c[3];
        coords(d, i, c);
        active[i] = (cls[i] == CLS_SPANNING);
        n_active += active[i];
        switch (cls[i]) {
        case CLS_FACE_IN: case CLS_INLET: P[i] = d->p_in; break;
        case CLS_FACE_OUT: case CLS_OUTLET: P[i] = d->p_out; break;
        case CLS_SPANNING:
            P[i] = d->p_in - dP * (double)c[f] / (double)(d->n[f] - 1);
            break;
        default: P[i] = 0.0;
        }
    }
    res->n_active = n_active;

    /* diagonal D and right-hand side b of Eq. 3 */
    for (int64_t i = 0; i < N; i++) {
        if (!active[i]) continue;
        int64_t c[3], j;
        double gij;
        coords(d, i, c);
        for (int k = 0; k < 2 * d->ndim; k++) {
            if (!neighbour(d, g, c, k, &j, &gij)) continue;
            D[i] += gij;
            if (!active[j]) b[i] += gij * P[j]; /* an open bond from an active
                                                   node leads only to the
                                                   cluster or to a face */
        }
        x[i] = P[i];
    }

    double bnorm = sqrt(dot(b, b, N));
    /* Jacobi-preconditioned CG */
    apply_G(d, g, active, D, x, q);
    for (int64_t i = 0; i < N; i++) r[i] = active[i] ? b[i] - q[i] : 0.0;
    for (int64_t i = 0; i < N; i++) z[i] = active[i] ? r[i] / D[i] : 0.0;
    memcpy(p, z, sizeof(double) * (size_t)N);
    double rz = dot(r, z, N);
    int64_t it = 0;
    int converged = (bnorm == 0.0);
    while (!converged && it < max_iter) {
        if (sqrt(dot(r, r, N)) <= tol * bnorm) { converged = 1; break; }
        apply_G(d, g, active, D, p, q);
        double alpha = rz / dot(p, q, N);
        for (int64_t i = 0; i < N; i++) {
            x[i] += alpha * p[i];
            r[i] -= alpha * q[i];
            z[i] = active[i] ? r[i] / D[i] : 0.0;
        }
        double rz_new = dot(r, z, N);
        double beta = rz_new / rz;
        rz = rz_new;
        for (int64_t i = 0; i < N; i++) p[i] = z[i] + beta * p[i];
        it++;
    }
    if (!converged && sqrt(dot(r, r, N)) <= tol * bnorm) converged = 1;
    res->iters = it;
    for (int64_t i = 0; i < N; i++)
        if (active[i]) P[i] = x[i];

    /* true residual of Eq. 3 on the solved nodes */
    or_residual(d, g, P, r);
    double rr = 0.0, rmax = 0.0;
    for (int64_t i = 0; i < N; i++) {
        if (!active[i]) continue;
        rr += r[i] * r[i];
        if (fabs(r[i]) > rmax) rmax = fabs(r[i]);
    }
    res->rel_residual = bnorm > 0.0 ? sqrt(rr) / bnorm : 0.0;
    res->max_imbalance = rmax;

    /* flows through the faces (Eq. 4's Q) and the dissipated power */
    double qin = 0.0, qout = 0.0, energy = 0.0;
    for (int64_t i = 0; i < N; i++) {
        int64_t c[3], j;
        double gij;
        coords(d, i, c);
        int ki = node_kind(d, c);
        for (int k = 0; k < 2 * d->ndim; k++) {
            if (!neighbour(d, g, c, k, &j, &gij)) continue;
            int64_t cj[3];
            coords(d, j, cj);
            int kj = node_kind(d, cj);
            if (ki == 0 && kj == 1) qin += gij * (P[j] - P[i]);
            if (ki == 0 && kj == 2) qout += gij * (P[i] - P[j]);
            if ((k & 1) == 0) energy += gij * (P[i] - P[j]) * (P[i] - P[j]);
        }
    }
    double S = 1.0;
    for (int a = 0; a < d->ndim; a++)
        if (a != f) S *= (double)d->n[a];
    res->q_in = qin;
    res->q_out = qout;
    res->g_eff = qin / dP;
    res->k_eff = res->g_eff * (double)(d->n[f] - 1) / S;
    res->energy_g = energy / (dP * dP);
    res->status = converged ? 0 : 1;
    if (label_out) memcpy(label_out, label, sizeof(int32_t) * (size_t)N);
    if (cls_out) memcpy(cls_out, cls, (size_t)N);
done:
    free(label); free(cls); free(active); free(D); free(b);
    free(x); free(r); free(z); free(p); free(q);
    return res->status;
}

int or_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
