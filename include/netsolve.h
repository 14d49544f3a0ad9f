/*
 * netsolve.h -- C ABI of the GB300 Kirchhoff network solver.
 *
 * The solver computes the steady flow through a 2D square or 3D cubic bond
 * network (pore network / random-resistor network) with one conductance per
 * bond, following Dashtian & Sahimi, arXiv:1908.03301:
 *
 *   Sec. II   each bond ij carries q_ij = g_ij (P_j - P_i);
 *   Eq. 3     mass balance sum_j q_ij = 0 at every interior node: G P = b;
 *   Sec. II   a fixed pressure drop along one axis: the face x_f = 0 is held
 *             at p_in and the face x_f = n_f - 1 at p_out; each transverse
 *             boundary is no-flow (the default) or periodic, the paper's
 *             stated choice (periodic_mask; y and z only);
 *   Eq. 4     K = (Q / S)(mu L / dP), with Q the total flow through the inlet
 *             face, L = n_f - 1, S = product of the transverse node counts
 *             and mu = 1 (lattice units);
 *   Sec. IV   G P = b solved by conjugate gradients with single-precision
 *             inner iterations inside a double-precision iterative
 *             refinement loop.
 *
 * Before the solve every network is split into clusters of nodes joined by
 * open bonds (g > 0).  Only clusters with open bonds to both faces carry
 * flow; the others are removed from the linear system (their pressure is
 * p_in for clusters touching only the inlet, p_out for clusters touching
 * only the outlet, 0 for isolated ones).  Labels are canonical: the smallest
 * linear node index of the cluster, -1 on the inlet face, -2 on the outlet.
 *
 * Layout of every node array: node (x, y, z) has linear index
 * x + nx * (y + ny * z), x fastest.  Bond plane d (0 = x, 1 = y, 2 = z) holds
 * the bond from node c to node c + e_d; its extents are the node extents with
 * n_d reduced by one, indexed the same way (x fastest).  Along a periodic
 * axis n_d is not reduced: the last layer holds the bonds from layer n_d - 1
 * back to layer 0.  A plane of extent 0 (e.g. ny = 1) may be NULL.
 *
 * Errors: every call returns a net_status; nothing aborts or throws across
 * this boundary.  net_last_error() gives a thread-local message for the last
 * failing call on the calling thread.  Any call accepts a NULL handle and
 * returns NET_EINVAL.
 *
 * Threads: a net_t may be used by one thread at a time.  A netq_t may be used
 * from any number of threads.
 *
 * Device: the library runs on the CUDA device that is current on the calling
 * thread at net_create / netq_create time and keeps all state resident there.
 *
 * Bounded waits: the inner-solve kernels whose CTAs wait for one another at
 * a grid barrier give up after 2 s of device time (NETSOLVE_WAIT_NS, in
 * nanoseconds, overrides it); the solve then returns NET_ETIMEOUT and the
 * device stays usable.  NETSOLVE_WITHHOLD_ARRIVAL=c (testing only) makes CTA
 * c skip its first arrival so that a test can see the waits run out.
 */
#ifndef NETSOLVE_H
#define NETSOLVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct net_s net_t;    /* one resident network (opaque) */
typedef struct netq_s netq_t;  /* a continuous-batching request queue (opaque) */

typedef enum {
    NET_OK = 0,
    NET_EINVAL = 1,         /* bad argument or bad network (see net_create) */
    NET_ENOMEM = 2,         /* device or host allocation failed */
    NET_EBUDGET = 3,        /* request larger than the queue's memory budget */
    NET_ENOTCONVERGED = 4,  /* iteration caps reached above the tolerance */
    NET_ETIMEOUT = 5,       /* a bounded wait gave up (device or host) */
    NET_ECUDA = 6,          /* a CUDA runtime call failed */
    NET_ECANCELLED = 7,     /* request cancelled / queue shut down */
    NET_EBUSY = 8           /* result not ready yet (netq_poll) */
} net_status;

enum { NET_F64 = 0, NET_F32 = 1 };      /* bond conductance dtype */
enum { NET_MIXED = 0, NET_FP64 = 1 };   /* solver precision */
/* Refinement scheme (net_opts.refine).  Both keep x and the true residual in
 * FP64 and run CG on the correction equation in the inner precision.
 *   NET_REFINE_RELIABLE  after each refinement pass the inner CG continues
 *                        along its current search direction, with the true
 *                        residual put in place of the recursive one
 *                        ("reliable update"); it restarts only after
 *                        stagnation, a cap or a breakdown.
 *   NET_REFINE_RESTART   classical iterative refinement: every inner solve
 *                        starts from a zero correction and p = r. */
enum { NET_REFINE_RELIABLE = 0, NET_REFINE_RESTART = 1 };

/* Cluster classes returned by net_get_labels. */
enum {
    NET_CLS_ISOLATED = 0,  /* no open bond to either face: P = 0 */
    NET_CLS_INLET = 1,     /* open bonds to the inlet face only: P = p_in */
    NET_CLS_OUTLET = 2,    /* open bonds to the outlet face only: P = p_out */
    NET_CLS_SPANNING = 3,  /* open bonds to both faces: solved */
    NET_CLS_FACE_IN = 4,   /* node on the inlet face (fixed p_in) */
    NET_CLS_FACE_OUT = 5   /* node on the outlet face (fixed p_out) */
};

/* Network description (Sec. II; boundary conditions as stated above). */
typedef struct {
    int ndim;                /* 2 or 3 */
    int64_t n[3];            /* node extents (nx, ny, nz); n[2] = 1 in 2D */
    int flow_axis;           /* axis of the pressure drop, 0 <= flow_axis < ndim;
                                n[flow_axis] >= 3 */
    unsigned periodic_mask;  /* bit d set: axis d is periodic (Sec. II); only
                                y (bit 1) and z (bit 2), never the flow axis,
                                each with n[d] >= 3.  0: no-flow boundaries.
                                Periodic networks are solved on their list
                                of unknowns (whose table holds the wrap
                                bonds) or, dense 2D ones alone, by the
                                persistent kernel; net_solve, net_solve_batch
                                and netq_* take them, net_autotune (which
                                tunes the lattice sweep) and
                                net_labels_noalloc reject them with
                                NET_EINVAL. */
    double p_in, p_out;      /* face pressures, finite, p_in != p_out */
    int bond_dtype;          /* NET_F64 or NET_F32 */
    int on_device;           /* 1: bond pointers are device pointers on the
                                current device; 0: host pointers */
    void *stream;            /* cudaStream_t for set-up work; NULL = the
                                library's own stream for this network */
} net_desc;

/* Solver options.  net_opts_default() fills the defaults listed here. */
typedef struct {
    int precision;           /* NET_MIXED (default) or NET_FP64 */
    double tol_rel;          /* outer stop: ||b - G P||_2 <= tol_rel ||b||_2
                                (and see tol_geff); default 1e-11 */
    double tol_inner;        /* NET_REFINE_RESTART: deepest relative reduction
                                asked of one FP32 inner solve; default 1e-4 */
    int max_outer;           /* refinement passes (true-residual
                                evaluations); default 200 */
    int64_t max_inner;       /* CG iterations per inner solve; default 200000 */
    int check_every;         /* inner iterations per device-flag check;
                                0 = choose automatically */
    const double *x0;        /* optional initial pressures (N doubles, node
                                layout; entries on faces are ignored); NULL =
                                linear profile along the flow axis */
    int x0_on_device;        /* x0 is a device pointer */
    void *stream;            /* cudaStream_t to run on; NULL = network's own */
    double tol_geff;         /* outer stop also needs the estimated relative
                                error of g_eff below this; default 1e-9.  The
                                estimate is first order: by the symmetry of
                                Eq. 3, Q_in's sensitivity to the nodal
                                residual r is the pressure field scaled to
                                (p_in, p_out) = (1, 0), so the error of Q_in is
                                sum_i (P_i - p_out) r_i / (p_in - p_out). */
    int refine;              /* NET_REFINE_RELIABLE (default) or
                                NET_REFINE_RESTART */
    double update_delta;     /* NET_REFINE_RELIABLE with an FP32 inner loop:
                                a refinement pass is taken once the recursive
                                residual norm has fallen to update_delta times
                                its largest value since the last pass (or the
                                outer targets are reached); default 1e-3,
                                in (0, 1) */
} net_opts;

/* Per-solve result and diagnostics. */
typedef struct {
    double g_eff;            /* effective conductance Q_in / (p_in - p_out) */
    double k_eff;            /* Eq. 4: g_eff * (n_f - 1) / S */
    double q_in, q_out;      /* total flow through the inlet / outlet face */
    double rel_residual;     /* ||b - G P||_2 / ||b||_2, FP64 true residual */
    double max_imbalance;    /* max nodal current imbalance |b - G P|_inf */
    double energy_g;         /* sum_bonds g dP_b^2 / (p_in - p_out)^2 */
    int64_t n_active;        /* nodes of spanning clusters */
    int outer_iters;         /* refinement steps taken */
    int64_t inner_iters;     /* CG iterations summed over refinement steps */
    int fp64_fallback;       /* 1 if the inner solve was switched to FP64 */
    float ms;                /* wall time of the solve on its stream */
    float inner_ms;          /* device time spent in the inner CG loop */
    int64_t inner_launches;  /* inner CG kernel launches (incl. no-op tails) */
    net_status status;
    double g_eff_err;        /* estimated relative error of g_eff (see tol_geff) */
    int64_t n_solved;        /* unknowns of the linear system: n_active less the
                                dead-end nodes (see net_get_backbone) */
    double queue_ms;         /* netq_* only: time from netq_submit to admission
                                onto the device (0 for net_solve / batches) */
    int64_t co_running;      /* netq_* only: requests already running on the
                                device when this one was admitted */
} net_result;

/* Fill *opts with the defaults listed in net_opts. */
void net_opts_default(net_opts *opts);

/*
 * Create a network: copy the bond planes to the device, label clusters,
 * build the scaled system (diagonal, right-hand side, initial pressures).
 *   desc   network description (read during the call only).
 *   g[d]   bond plane d for d < ndim, dtype desc->bond_dtype, host or device
 *          per desc->on_device; copied, the caller keeps ownership.  Planes
 *          with zero entries may be NULL.
 *   out    receives the handle; the library owns its device state until
 *          net_destroy.
 * Errors: NET_EINVAL for ndim not 2/3, an extent < 1, n_f < 3, more than
 * 2^31 - 1 padded nodes, a periodic_mask with bit 0, the flow axis or an
 * axis beyond ndim set, or a periodic extent < 3, non-finite or equal pressures,
 * or a conductance that is negative, NaN or infinite (checked on the
 * device); NET_ENOMEM / NET_ECUDA otherwise.  A network without a spanning
 * cluster is valid and solves to g_eff = 0.  The call returns after the
 * set-up work has completed on the device.
 */
net_status net_create(const net_desc *desc, const void *const g[3], net_t **out);

/*
 * Solve Eq. 3 for the network (Sec. IV: CG, single-precision inner loop in a
 * double-precision refinement loop; NET_FP64 runs the inner loop in FP64).
 * The preconditioner is Jacobi, applied as the symmetric scaling
 * D^-1/2 G D^-1/2.  Pressures stay on the device (net_get_pressure).
 *   opts   NULL = defaults.   out   receives the result (required).
 * Returns out->status: NET_OK, NET_ENOTCONVERGED (caps reached; the result
 * holds the best pressures reached), NET_ETIMEOUT (a bounded device wait
 * gave up; see "Bounded waits" above), NET_ECUDA, NET_EINVAL.
 */
net_status net_solve(net_t *net, const net_opts *opts, net_result *out);

/*
 * Flows of the last solve (Eq. 4): total flow into the inlet face, out of the
 * outlet face, and the effective conductance q_in / (p_in - p_out).  Any
 * output pointer may be NULL.  NET_EINVAL before the first solve.
 */
net_status net_flux(net_t *net, double *q_in, double *q_out, double *g_eff);

/*
 * Copy the N = nx*ny*nz node pressures (FP64, node layout) to dst, a host or
 * device buffer of at least n doubles (n >= N, else NET_EINVAL).  Face nodes
 * hold p_in / p_out; removed clusters hold their fixed pressure.
 */
net_status net_get_pressure(net_t *net, double *dst, int64_t n, int dst_on_device);

/*
 * Copy the cluster labels (int32) and classes (uint8, NET_CLS_*) of the N
 * nodes into host buffers of at least n entries.  Either pointer may be NULL.
 */
net_status net_get_labels(net_t *net, int32_t *label, uint8_t *cls, int64_t n);

/*
 * Current-carrying backbone of the spanning clusters: backbone[i] = 1 for the
 * spanning nodes left in the linear system, 0 for every other node (host
 * buffer of at least n >= N entries, node layout).
 *
 * Take every inlet-face node as one vertex A, every outlet-face node as one
 * vertex B, and join A and B by one extra edge.  A bond carries current (for
 * generic conductances) exactly when it lies on a path from A to B that
 * visits no vertex twice, i.e. when it belongs to the biconnected component
 * of the extra edge; every other part of a spanning cluster -- a dead-end
 * tree, or a dead-end loop -- hangs from that component by a single node and
 * carries no current, so its pressure equals that node's.  net_create finds
 * the component on the device (Tarjan and Vishkin's parallel biconnectivity
 * method) and removes the rest: the removed nodes keep their cluster label
 * and class NET_CLS_SPANNING, but leave the linear system of Eq. 3 (the
 * diagonal and the CG iterations cover the backbone only), and each takes
 * the pressure of the node its part hangs from before every residual pass.
 * This is exact (the paper solves the whole cluster; it says that near the
 * percolation threshold much of it carries no flow).  The environment
 * variable NETSOLVE_PRUNE selects less: "trees" removes only the nodes left
 * with at most one link in rounds (dead-end trees), "0" keeps every spanning
 * node in the system.
 */
net_status net_get_backbone(net_t *net, uint8_t *backbone, int64_t n);

/* Release the network's device state.  NULL is accepted. */
net_status net_destroy(net_t *net);

/*
 * Cluster labels without any memory allocation.  (The paper has no
 * counterpart; this serves callers that cannot allocate device memory when
 * they need labels: code inside a framework whose pool owns all device memory,
 * or a latency-critical loop where cudaMalloc / cudaFree, which may block the
 * host and synchronise the device, are not acceptable.)
 *
 * Computes the same labels and classes as net_create + net_get_labels.
 *   desc    as for net_create; desc->on_device must be 1; desc->stream is
 *           the stream the work runs on (NULL = the default stream).
 *   g[d]    device bond planes (compact layout, desc->bond_dtype).
 *   label   device output, N int32 (may be NULL); cls: device output, N uint8
 *           (may be NULL).  N = nx*ny*nz.
 * The union-find scratch is a fixed array inside the library's device image,
 * sized for NET_NOALLOC_MAX_NODES nodes (8 MiB); once the library's device
 * code is loaded on a GPU, that GPU holds it until the process exits.  N
 * above that limit returns NET_EINVAL.  The first call on each device looks
 * up the array's device address (cudaGetSymbolAddress) with that device
 * current.  Under lazy module loading (the CUDA default) that lookup is also
 * what loads the device code and so creates the array: the first call on a
 * device may allocate those 8 MiB and block.  A caller that must not allocate
 * later makes one call at start-up (any small network will do), before its
 * own memory pool reserves the device and before any stream capture.  All calls on a device share the array, so
 * calls that overlap on the GPU (other streams or threads) race: keep them
 * ordered.  The call returns after the work on desc->stream has finished;
 * NET_EINVAL also for a negative, NaN or infinite conductance.
 */
#define NET_NOALLOC_MAX_NODES (1LL << 20)
net_status net_labels_noalloc(const net_desc *desc, const void *const g[3], int32_t *label,
                              uint8_t *cls);

/*
 * Correlated percolation by sorted removal (Sec. VI.B): of the M bonds of
 * the planes g[0..ndim-1] (taken in plane order, each x fastest), close (set
 * to 0) the floor(q * M) of smallest conductance, q * M computed in double.
 * Equal conductances close in that position order, so the closed set is
 * unique; 0 and -0 count as equal.  Unlike i.i.d. percolation this keeps the
 * field's correlations in the open bonds.
 *   desc   as for net_create (its dims, bond_dtype and periodic_mask fix the
 *          plane sizes); desc->on_device must be 1; the work runs on
 *          desc->stream (NULL = the default stream) and the call returns
 *          after it has finished.
 *   g[d]   device bond planes, modified in place; the caller keeps ownership.
 *   q      fraction to close, 0 <= q <= 1.
 * Device scratch (a few KB, plus 12 bytes per 4096 bonds when equal
 * conductances straddle the cut) is allocated and freed on the stream.
 * Errors: NET_EINVAL for a bad descriptor, q outside [0, 1], a NULL plane,
 * or a negative, NaN or infinite conductance (then nothing is written);
 * NET_ECUDA otherwise.
 */
net_status net_close_smallest(const net_desc *desc, void *const g[3], double q);

/*
 * Fractional Brownian motion field by spectral filtering (Eq. 1, Eq. 2), the
 * generator of the paper's correlated networks.  The random draws are an
 * input: complex white noise, one value per node.  Each Fourier mode is
 * weighted by sqrt(S(w)), S(w) = (sum_a beta_a w_a^2)^-(H + d/2) (d = ndim;
 * Eq. 1 is d = 2 with beta = 1, Eq. 2 the anisotropic case), with w_a the
 * discrete frequency in cycles per node (0, 1, .., ceil(n/2)-1, -floor(n/2),
 * .., -1 over n) and the zero mode dropped; the field is the real part of the
 * inverse FFT, shifted and scaled to zero mean and unit variance.
 *   d       extents, H, per-axis beta (> 0, finite) and the stream (NULL =
 *           the default stream); read during the call only.
 *   noise   device array of N complex values (real, imaginary interleaved;
 *           double, or float with fft_f32), node order x fastest; overwritten
 *           (it holds the transform).
 *   field   device array of N doubles, the field (output).
 * N = nx*ny*nz < 2^31.  The FFT is cuFFT's (loaded on first use; NET_ECUDA
 * if it cannot be loaded), with its plan and workspace allocated and freed
 * in the call.  Returns after the work has finished.  NET_EINVAL for bad
 * extents, a non-finite H or a bad beta.
 */
typedef struct {
    int ndim;          /* 2 or 3 */
    int64_t n[3];      /* node extents (nx, ny, nz); n[2] = 1 in 2D */
    double hurst;      /* Hurst exponent H */
    double beta[3];    /* anisotropy per axis (x, y, z); all 1 for Eq. 1 */
    int fft_f32;       /* 0: noise is complex double and the transform FP64;
                          1: complex float noise and an FP32 transform (GB300
                          runs FP64 arithmetic at 1/64 of the FP32 rate) */
    void *stream;      /* cudaStream_t; NULL = the default stream */
} net_fbm_desc;
net_status net_fbm_field(const net_fbm_desc *d, void *noise, double *field);

/*
 * Conductances from a field B (device, N doubles, node order x fastest):
 * g = exp(sigma * (B_i + B_j) / 2) for the bond between nodes i and j,
 * written into the bond planes g[d] (device, desc->bond_dtype, the layout of
 * net_create including periodic planes).  desc as for net_create with
 * on_device = 1; the work runs on desc->stream and has finished when the
 * call returns.  NET_EINVAL for a bad descriptor, a NULL plane or a
 * non-finite sigma.
 */
net_status net_fbm_bonds(const net_desc *desc, const double *field, double sigma, void *const g[3]);

/*
 * Solve `count` independent networks together.  Every sweep of the CG loop
 * (Sec. IV) is one launch of a kernel with one CTA per SM that walks all
 * running networks' segments; each network keeps its own CG scalars and its
 * own convergence mask, and networks drop out as they converge while the
 * rest continue.  Networks whose unknowns are under 35 % of their lattice
 * (near-critical percolation after dead-end stripping) and periodic networks
 * are solved on their lists of unknowns instead: one launch per phase of the
 * iteration for all of them, the lists cut into segments.  The sweeps run as
 * CUDA-graph chunks of opts->check_every iterations (0 = 16).  res[i] receives network i's result; each result
 * matches the network's stand-alone net_solve within the solver tolerance.
 * All networks must live on the current device.  opts NULL = defaults (one
 * opts for all; x0 is ignored).  Returns NET_OK if every network converged,
 * else the first non-OK status (each res[i].status says which).
 */
net_status net_solve_batch(net_t *const *nets, int count, const net_opts *opts,
                           net_result *res);

/*
 * Autotuner of the CG sweep's tile shape.  Sec. IV picks its launch shape
 * (64 blocks of 256 threads, a loop over rows per thread) once, by hand, for
 * the device it used; here the shape is measured on the GPU at hand.
 *
 * The sweep kernel (used for 3D networks, FP64 inner loops, 2D networks wider
 * than 2048 nodes and every batched or queued solve) cuts each network into
 * segments: blocks of columns (x), in 3D bands of rows (y), each marched
 * along the last axis.  net_autotune times every candidate shape (column
 * block width, row band height, segments per SM) with a few CUDA-graph
 * replays of CG sweeps over the given networks, keeps the fastest in a
 * process-wide table keyed by (device, dimension, inner precision, size
 * class = floor(log2(lattice nodes of the set))) and returns it.  Solves of
 * that key then plan with it.  Solves also tune by themselves the first time
 * they meet an untuned key (set NETSOLVE_AUTOTUNE=0 to disable; the default
 * shape is then used), so calling this is optional: it lets a caller tune
 * ahead of a latency-sensitive run, or re-tune.
 *   nets    count >= 1 networks on the current device, all 2D or all 3D.
 *   opts    precision selects the inner loop to tune (NULL = NET_MIXED).
 *   out     the chosen shape and times (may be NULL).
 * The networks' inner CG state is overwritten (their pressures are not);
 * every later net_solve / net_solve_batch starts afresh as always.
 * NET_EINVAL for mixed dimensions, a NULL network or another device.
 */
typedef struct {
    int col_block;        /* widest column block (nodes along x) */
    int row_band;         /* tallest row band in 3D (nodes along y); 1 in 2D */
    int seg_per_sm;       /* segments per SM the march ranges are cut into */
    int size_class;       /* floor(log2(lattice nodes)) of the key */
    int candidates;       /* shapes timed */
    double us_per_sweep;  /* one CG iteration over the set, chosen shape */
    double us_default;    /* the same with the default shape */
} net_tune;
net_status net_autotune(net_t *const *nets, int count, const net_opts *opts, net_tune *out);
/* Forget every tuned shape (all devices); later solves tune again. */
void net_tune_clear(void);

/*
 * Continuous-batching queue.  Requests are admitted while their device
 * footprint fits in mem_budget_bytes and a slot among max_slots is free;
 * admitted requests are solved together with those already running, and
 * finished ones leave at once, freeing memory and a slot for the next.
 * A background host thread drives the device.  opts applies to every request
 * (NULL = defaults).
 */
net_status netq_create(size_t mem_budget_bytes, int max_slots, const net_opts *opts,
                       netq_t **out);

/*
 * Submit a network (arguments as for net_create; host bond pointers only,
 * copied before the call returns).  *ticket identifies the request.
 * NET_EBUDGET if the request's estimated device footprint alone exceeds the
 * memory budget; NET_EINVAL for a bad descriptor.  Conductance errors found
 * on the device are reported through the request's result status.
 */
net_status netq_submit(netq_t *q, const net_desc *desc, const void *const g[3],
                       uint64_t *ticket);

/* Non-blocking: NET_EBUSY while the request is queued or running, else its
 * final status with *out filled; a finished ticket can be read once. */
net_status netq_poll(netq_t *q, uint64_t ticket, net_result *out);

/* Block up to timeout_ms (< 0: no limit) for the request; NET_ETIMEOUT if it
 * is still pending. */
net_status netq_wait(netq_t *q, uint64_t ticket, int timeout_ms, net_result *out);

/* Cancel a queued (not yet admitted) request: its status becomes
 * NET_ECANCELLED.  NET_EBUSY if it is already running. */
net_status netq_cancel(netq_t *q, uint64_t ticket);

/* Latency statistics over finished requests (arrival to result, ms). */
net_status netq_stats(netq_t *q, double *p50_ms, double *p99_ms, uint64_t *completed);

/* Stop the worker (pending requests finish as NET_ECANCELLED) and free. */
net_status netq_destroy(netq_t *q);

/* Thread-local message describing the last failing call on this thread. */
const char *net_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
