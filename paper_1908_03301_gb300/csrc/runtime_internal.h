// runtime_internal.h -- the network object behind net_t (internal).
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "../../include/netsolve.h"
#include "kernels.h"
#include "plan.h"
#include "sweep.cuh"

namespace netsolve {

// Device copy of a sweep plan (segments, per-CTA offsets, network record).
struct SweepDev {
    SweepSeg *segs = nullptr;
    int *cta = nullptr;
    double *part = nullptr;
    SweepInst *inst = nullptr;
    int grid = 0;
    PlanShape shape;  // tile shape the plan was built with
};
inline bool same_shape(const PlanShape &a, const PlanShape &b) {
    return a.wcap == b.wcap && a.hcap == b.hcap && a.seg_per_sm == b.seg_per_sm;
}

// Compacted inner solve of one precision (cg_compact.cu).
struct CompactDev {
    long long U = 0;          // unknowns
    int *cidx = nullptr;      // list index -> padded lattice index
    int *nbr = nullptr;       // [2 (ndim - 1)][U] y/z neighbour list indices
    void *val = nullptr;      // [ndim][U + 1] scaled +e_d bonds
    void *vec = nullptr;      // y, r, p, q, each U + 1 entries
    double *pb = nullptr;     // partial sums [2][grid][4]
    unsigned *bar = nullptr;  // barrier words
    int *err = nullptr;
    int grid = 0;
};

// Device-resident scalars of one network (one allocation).
struct DevScal {
    InnerScal in[2];  // [0] FP32 inner solve, [1] FP64 inner solve
    OuterScal os;
    SetupScal ss;
    int perr;  // host mirror of the persistent kernel's error word
};

}  // namespace netsolve

struct net_s {
    int device = 0;
    netsolve::Geom g{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int raw_f32 = 0;
    void *graw[3] = {nullptr, nullptr, nullptr};  // padded raw bonds
    int *parent = nullptr;                         // union-find roots (padded index)
    int *proot = nullptr;                          // dead-end node -> its root (-1 elsewhere);
                                                   // NULL when nothing was stripped
    int prune_rounds = 0;
    long long loop_nodes = 0;  // nodes removed as parts of dead-end loops
    uint8_t *cls = nullptr;                        // cluster classes
    double *dis = nullptr;                         // D^-1/2 on solved nodes, else 0
    double *x = nullptr;                           // FP64 pressures
    void *gs[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};  // scaled bonds [f32, f64]
    void *vec[2] = {nullptr, nullptr};            // y, r0, r1, p0, p1, q0, q1 per precision
    double *partials = nullptr;
    netsolve::DevScal *dsc = nullptr;              // device scalars
    netsolve::DevScal *hsc = nullptr;              // pinned host mirror
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    netsolve::SweepDev sw[2];                      // sweep plan per precision
    netsolve::CompactDev cp[2];                    // compacted solve per precision
    // whole-solve persistent kernel (2D, FP32): halo rows, partials, grid
    // barrier words, error word
    float *ps_hb = nullptr;
    float *ps_pb = nullptr;
    unsigned *ps_bar = nullptr;
    int *ps_err = nullptr;
    int ps_grid = 0;
    int gk[2] = {0, 0};
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    net_result last{};
    bool solved = false;
    double bnorm = 0.0;
    long long n_active = 0;   // nodes of spanning clusters
    long long n_solved = 0;   // of them, unknowns of the linear system
};

namespace netsolve {
template <typename T>
inline cudaError_t dalloc(T **p, size_t bytes, cudaStream_t st) {
    void *q = nullptr;
    cudaError_t e = cudaMallocAsync(&q, bytes ? bytes : 16, st);
    if (e != cudaSuccess) return e;
    *p = (T *)q;
    return cudaMemsetAsync(q, 0, bytes ? bytes : 16, st);
}
inline void dfree(void *p, cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
}
// Outer stopping measure: max(rel / tol_rel, g_err / tol_geff); converged
// when <= 1.  g_err is the first-order relative error of G_eff estimated by
// the last outer pass (see net_opts.tol_geff).
inline double eff_tol_geff(const net_opts &o) { return o.tol_geff > 0.0 ? o.tol_geff : 1e-9; }
inline double geff_err(const net_t *n) {
    const double dP = n->g.p_in - n->g.p_out;
    const double G = n->hsc->os.qin / dP;
    return G != 0.0 ? std::fabs(n->hsc->os.ez) / (dP * dP) / std::fabs(G) : 0.0;
}
inline double outer_dist(const net_t *n, const net_opts &o, double rel) {
    return std::fmax(rel / o.tol_rel, geff_err(n) / eff_tol_geff(o));
}
// Progress of the FP32 refinement passes.  A pass that halves neither the
// best relative residual nor the best G_eff error estimate so far is a stall;
// FP32 has reached its limit after `limit` stalls in a row (3 when the CG
// recursion is kept across passes, whose residual may rise between them; 1
// for restarted passes).  Then the inner loop continues in FP64.
struct Progress {
    double best_rel = 0.0, best_gerr = 0.0;
    int stall = 0;
    void start(double rel, double gerr) {
        best_rel = rel;
        best_gerr = gerr;
        stall = 0;
    }
    bool stalled(double rel, double gerr, int limit) {
        const bool gain = rel < 0.5 * best_rel || gerr < 0.5 * best_gerr;
        best_rel = std::fmin(best_rel, rel);
        best_gerr = std::fmin(best_gerr, gerr);
        stall = gain ? 0 : stall + 1;
        return stall >= limit;
    }
};
inline int stall_limit(const net_opts &o) { return o.refine == NET_REFINE_RESTART ? 1 : 3; }
// Options check shared by every solve entry point.
bool opts_valid(const net_opts &o);

// One line per refinement step on stderr when NETSOLVE_TRACE is set.
bool trace_on();
void trace_outer(const net_t *n, const char *who, int outer, int f32, int stop, long long iters,
                 double rel);
// Scaled bonds and inner vectors of one precision (allocated on first use).
net_status ensure_precision(net_t *n, int f32, cudaStream_t st);
void set_error(const char *fmt, ...);
const char *last_error();
net_status cuda_fail(cudaError_t e, const char *what);
net_status make_geom(const net_desc *d, Geom *g);
long long plane_elems(const Geom &g, int d);
size_t net_footprint_bytes(const Geom &g, int raw_f32);
InnerArgs inner_args(net_t *n, int f32);
OuterArgs outer_args(net_t *n, int f32, int apply_corr, int corr_f32, const net_opts &op,
                     int inplace = 0);
net_status setup_network(net_t *n, const void *const g[3], int on_device);
// NETSOLVE_PRUNE=0 keeps dead-end trees in the linear system (diagnostics).
bool prune_enabled();
net_status prune_dead_ends(net_t *n, const void *const gr[3], unsigned int *pr);
void release_network(net_t *n);
net_status create_network(const net_desc *desc, const void *const g[3], net_t **out);
net_status solve_impl(net_t *n, const net_opts *o, net_result *r);
// Arm a network's inner state of one precision for timing sweeps: a fresh CG
// from the current pressures that stops only on an exactly zero residual.
// The next solve (or batch add) re-arms it for real.
net_status arm_for_tuning(net_t *n, int f32, cudaStream_t st);
// Sweep record of one network for a plan (part / nseg filled by the planner).
SweepInst sweep_inst_of(net_t *n, int f32);
// Networks whose unknowns are a small part of the lattice (and periodic
// ones) are solved on their list of unknowns, in batches too.
bool batch_takes_compact(const net_t *n, int f32);
// List of unknowns and table of one inner precision (built on first use).
net_status prepare_compact(net_t *n, int f32, cudaStream_t st);
CompactArgs compact_args_of(net_t *n, int f32);
// Refinement pass of a network solved on its list (correction, FP64
// residual, gather of the new scaled residual).
net_status outer_pass_compact(net_t *n, int f32, int apply_corr, const net_opts &o, cudaStream_t st);
int device_sm_count(int dev);
// Tune the sweep tile shape over these networks (same dimension, inner
// precision f32) and store the winner under their key.  Their inner state is
// left armed for tuning.  *def_us gets the default shape's time.
net_status autotune_nets(const std::vector<net_t *> &nets, int f32, int default_seg, cudaStream_t st,
                         PlanShape *best, double *best_us, double *def_us, int *ncand);
}  // namespace netsolve
