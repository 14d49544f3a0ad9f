// kernels.h -- host-side launchers of the solver kernels (internal).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace netsolve {

// ---- set-up (kernels_setup.cu) --------------------------------------------
// Copy user bond plane d (compact layout, dtype src_f32 ? float : double,
// device memory) into the padded plane dst (dtype dst_f32 ? float : double);
// sets *bad if a value is negative, NaN or infinite.
cudaError_t launch_pack_bonds(const Geom &g, int d, const void *src, int src_f32, void *dst,
                              int dst_f32, unsigned int *bad, cudaStream_t st);
// Cluster labelling (union-find, min-index roots) and classes.
cudaError_t launch_labels(const Geom &g, const void *const graw[3], int f32, int *parent,
                          unsigned int *flags, uint8_t *cls, cudaStream_t st);
// Dead-end stripping (see kernels_setup.cu): one round over the lattice
// (nodes removed in it get pr = round and their anchor; *count += removed),
// then mark them CLS_DANGLING and resolve anchors to roots by `passes`
// pointer-jumping passes (root aliases the anchor array).
cudaError_t launch_prune_round(const Geom &g, const void *const graw[3], int f32, const uint8_t *cls,
                               unsigned int *pr, int *anchor, unsigned int round, unsigned int *count,
                               cudaStream_t st);
cudaError_t launch_prune_finish(const Geom &g, uint8_t *cls, const unsigned int *pr, int *root,
                                int passes, cudaStream_t st);
// Dead-end loops (blocks.cu): the spanning nodes still CLS_SPANNING that lie
// outside the biconnected component of the extra inlet-outlet edge become
// CLS_DANGLING with root = the node their part hangs from; roots of earlier
// dead-end nodes are re-resolved.  root: L ints, -1 where not removed;
// vmap: L ints of scratch.  *removed: nodes marked; *internal_err != 0 if a
// consistency check failed (nothing was marked).  Allocates its other
// scratch (about 4 (2d + 25) bytes per spanning node) on the stream and
// returns after the work has finished.
cudaError_t strip_dead_loops(const Geom &g, const void *const graw[3], int f32, uint8_t *cls, int *root,
                             int *vmap, long long *removed, int *internal_err, cudaStream_t st);
// x at every dead-end node := x at its root (root[i] = -1 elsewhere).
cudaError_t launch_fill_dangling(const Geom &g, const int *root, double *x, cudaStream_t st);
// Compact uint8 mask of the backbone (spanning nodes left in the system).
cudaError_t launch_backbone(const Geom &g, const uint8_t *cls, uint8_t *out, cudaStream_t st);
// Diagonal scaling, initial pressures, ||b||^2 and the active count.
cudaError_t launch_build_system(const Geom &g, const void *const graw[3], int f32,
                                const uint8_t *cls, double *dis, double *x, SetupScal *ss,
                                double *partials, cudaStream_t st);
// Scaled bonds ghat_d = g_d D_i^-1/2 D_j^-1/2 (0 unless both ends are solved).
cudaError_t launch_build_scaled(const Geom &g, const void *const graw[3], int f32,
                                const double *dis, void *const gs[3], int gs_f32,
                                cudaStream_t st);
// Overwrite solved pressures with a caller's initial guess (compact, device).
cudaError_t launch_apply_x0(const Geom &g, const uint8_t *cls, const double *x0c, double *x,
                            cudaStream_t st);
// Padded -> compact copies for output.
cudaError_t launch_unpack_x(const Geom &g, const double *x, double *dst, cudaStream_t st);
cudaError_t launch_unpack_labels(const Geom &g, const int *parent, const uint8_t *cls,
                                 int *label, uint8_t *cls_out, cudaStream_t st);

// ---- inner CG vectors of a lattice network (one set per inner precision) ---
struct InnerArgs {
    Geom g;
    const void *gs[3];  // scaled bonds (T)
    void *y;              // inner solution (T)
    void *r[2], *p[2], *q[2];  // double-buffered inner vectors (T)
    InnerScal *s;
    double *partials;
};

// ---- whole inner solve of a 2D network in one launch (cg_persist.cu) ------
struct PersistArgs {
    Geom g;
    const float *gx, *gy;      // scaled bonds
    float *y, *r, *p, *q;      // inner vectors, updated in place
    InnerScal *s;              // armed state in, final state out
    float *hb;                 // halo copies [2][grid][2][3][px]
    float *pb;                 // per-CTA sums as pairs [2][grid][hi 4, lo 4]
    unsigned *bar_count;       // grid barrier: arrivals (zeroed at launch)
    int *err;                  // set when a bounded wait gave up (cleared at launch)
    unsigned long long wait_ns;  // give up a grid-barrier wait after this long
    int skip_cta;              // testing: this CTA withholds its first arrival (-1: none)
};
bool persist_applies(const Geom &g, int f32);
int persist_grid(const Geom &g);
cudaError_t persist_prepare();
cudaError_t launch_persist(const PersistArgs &a, int grid, cudaStream_t st);

// ---- inner solve over a compacted list of unknowns (cg_compact.cu) --------
struct CompactArgs {
    long long n;            // unknowns
    void *y, *r, *p, *q;    // compact vectors (T), n + 1 entries each
    const int *cidx;        // lattice index of each unknown
    const void *val;        // scaled +e_d bonds [ndim][n + 1] (T; 0: none)
    const int *nbr;         // list indices of the +-e_d neighbours, d = y[, z]:
                            // [2 (ndim - 1)][n]; none: k (+e_d), ~k (-e_d)
    InnerScal *s;           // armed state in, final state out
    double *pb;             // per-CTA partial sums [2][grid][4]
    unsigned *bar;          // grid barrier: arrivals, generation
    int *err;               // set when a bounded wait gave up (cleared at launch)
    unsigned long long wait_ns;  // give up a grid-barrier wait after this long
    int skip_cta;           // testing: this CTA withholds its first arrival (-1: none)
    int jc;                 // cooperative solve: list chunks (grid x CTA threads entries each)
                            // whose table rows each CTA keeps in shared memory (set at launch)
};
int compact_grid(int ndim, int f32);
// List the unknowns (cls == CLS_SPANNING) in lattice order and build their
// ELL rows from the scaled lattice bonds gs (T).  cmap: L-entry scratch.
cudaError_t compact_build(const Geom &g, const uint8_t *cls, long long U, int f32, const void *const gs[3],
                          int *cmap, int *cidx, int *nbr, void *val, cudaStream_t st);
// x[cidx[k]] += D^-1/2 (y[k] (+ alpha p[k] when the pass ended with stop 6))
cudaError_t launch_compact_correct(const CompactArgs &a, const double *dis, double *x, int f32, cudaStream_t st);
cudaError_t launch_compact_cg(const CompactArgs &a, int ndim, int f32, int grid, cudaStream_t st);
// Compacted networks inside a batch: every running network's list is cut
// into segments (one CTA each); one CG iteration of all of them is a launch
// of phase A then a launch of phase B (the network's last segment reduces
// the part[] slots in order and runs finish_iteration).
struct CompactInst {
    CompactArgs a;   // the network's compact vectors, table and CG state (a.s)
    double *part;    // 4 partial sums per segment, in slot order
    int nseg;        // segments of this network in the current plan
};
struct CompactSeg {
    int inst;        // network
    int u0, u1;      // list range
    int slot;        // partial-sum slot within the network
};
constexpr int COMPACT_SEG = 4096;  // list entries per segment
cudaError_t launch_compact_batch(int ndim, int f32, const CompactInst *insts, const CompactSeg *segs, int nseg,
                                 cudaStream_t st);

// ---- persistent sweep over segmented networks (sweep.cu) -------------------
struct SweepInst;
struct SweepSeg;
int sweep_max_width(int ndim, int f32);
int sweep_vt(int f32);
int sweep_consumers();
// Rows a 2D segment stages per pipeline step (1 in 3D).
int sweep_rows_per_stage(int ndim, int f32, int w, int px, int x0);
// Whether a 3D patch of w columns x h rows (plus its halo) fits one stage slot.
bool sweep_patch_fits(int f32, int w, int h);
cudaError_t sweep_prepare(int ndim, int f32);
cudaError_t launch_sweep(int ndim, int f32, int grid, const SweepInst *insts, const SweepSeg *segs,
                         const int *cta_begin, cudaStream_t st);


struct OuterArgs {
    Geom g;
    const void *graw[3];  // raw bonds (double or float)
    int raw_f32;
    const double *dis;
    double *x;
    const void *y;        // inner correction (T), read when apply_corr
    void *r_buf[2];       // inner residual buffers (T) of the armed precision;
                          // r_buf[1] == r_buf[0] for in-place inner kernels
    const void *p_buf[2]; // search directions (T) of the correction's precision
    int inner_f32;
    int apply_corr;       // first apply x += D^-1/2 y (separate kernel)
    int corr_f32;         // dtype of y
    OuterScal *os;
    InnerScal *is;        // inner scalars to arm for the next inner solve
    const InnerScal *is_corr;  // scalars of the pass that produced y (apply_corr)
    int reliable;         // arm the next pass in reliable mode
    int allow_cont;       // continue the recursion if the last pass ended with
                          // stop 6 (same precision, correction applied)
    double delta2;        // reliable-update threshold (squared) for the next pass
    double tol_floor;     // smallest relative reduction asked of the inner solve
    double tol_rel;       // outer tolerance (relative 2-norm residual)
    double tol_geff;      // outer tolerance on the estimated relative error of G_eff
    double bnorm;         // ||b||_2
    long long max_inner, stag_window;
    double *partials;
    const int *root;      // dead-end nodes' roots (NULL: none); their x is
                          // refreshed before the residual pass
};
int outer_grid_blocks(const Geom &g);
cudaError_t launch_outer(const OuterArgs &a, cudaStream_t st);
// The residual pass of a network solved on its list of U unknowns (cidx:
// list -> lattice index): dead-end pressures filled, then the sums over the
// listed nodes only, the scaled residual written to r_list (inner precision).
// a.apply_corr must be 0 (the list's correction is its own launch).
cudaError_t launch_outer_list(const OuterArgs &a, const int *cidx, long long U, void *r_list, cudaStream_t st);
// Before a persistent-kernel launch that continues a recursion (iter > 0):
// refresh the halo copies of r, q, p that the first sweep reads (r was
// replaced by the refinement pass).  Does nothing when iter == 0.
cudaError_t launch_persist_resume(const PersistArgs &a, int grid, cudaStream_t st);

}  // namespace netsolve
