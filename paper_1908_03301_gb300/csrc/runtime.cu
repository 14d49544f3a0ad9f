// runtime.cu -- the C ABI of include/netsolve.h: network set-up, the
// iterative-refinement driver around the CG kernels, result read-back.
//
// Iterative refinement (Sec. IV, "mixed-precision method"): the FP64 outer
// loop recomputes the true residual r = b - G x on the device, the inner CG
// solves D^-1/2 G D^-1/2 y = D^-1/2 r in FP32 to a relative reduction
// tol_inner, and the outer pass applies x += D^-1/2 y.  The inner iterations
// run as CUDA-graph chunks of `check_every` fused iteration kernels; the host
// reads one device flag per chunk.  Nothing is summed on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/netsolve.h"
#include "kernels.h"
#include "plan.h"
#include "runtime_internal.h"
#include "tune.h"

using namespace netsolve;

namespace {
thread_local std::string g_err;
}

namespace netsolve {

void set_error(const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
}

const char *last_error() { return g_err.c_str(); }

bool opts_valid(const net_opts &o) {
    if (o.precision != NET_MIXED && o.precision != NET_FP64) {
        set_error("bad precision");
        return false;
    }
    if (!(o.tol_rel > 0.0) || !(o.tol_inner > 0.0) || o.max_outer < 1 || o.max_inner < 1) {
        set_error("bad tolerances or caps");
        return false;
    }
    if (o.refine != NET_REFINE_RELIABLE && o.refine != NET_REFINE_RESTART) {
        set_error("bad refine mode");
        return false;
    }
    if (!(o.update_delta >= 0.0 && o.update_delta < 1.0)) {  // 0 = default
        set_error("update_delta must be in (0, 1)");
        return false;
    }
    return true;
}

bool trace_on() { return getenv("NETSOLVE_TRACE") != nullptr; }

void trace_outer(const net_t *n, const char *who, int outer, int f32, int stop, long long iters,
                 double rel) {
    if (!trace_on()) return;
    fprintf(stderr, "[trace %s %p %lldx%lldx%lld] step %d %s stop %d iters %lld rel %.3e gerr %.3e\n", who,
            (const void *)n, (long long)n->g.nx, (long long)n->g.ny, (long long)n->g.nz, outer,
            f32 ? "f32" : "f64", stop, iters, rel, geff_err(n));
}

net_status cuda_fail(cudaError_t e, const char *what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return NET_ECUDA;
}

static long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }

net_status make_geom(const net_desc *d, Geom *g) {
    if (!d) { set_error("desc is NULL"); return NET_EINVAL; }
    if (d->ndim != 2 && d->ndim != 3) { set_error("ndim must be 2 or 3"); return NET_EINVAL; }
    for (int a = 0; a < 3; a++)
        if (d->n[a] < 1 || d->n[a] > (1LL << 30)) { set_error("extent n[%d] out of range", a); return NET_EINVAL; }
    if (d->ndim == 2 && d->n[2] != 1) { set_error("2D network needs n[2] == 1"); return NET_EINVAL; }
    if (d->flow_axis < 0 || d->flow_axis >= d->ndim) { set_error("flow_axis out of range"); return NET_EINVAL; }
    if (d->n[d->flow_axis] < 3) { set_error("need at least 3 nodes along the flow axis"); return NET_EINVAL; }
    if (d->periodic_mask >> d->ndim) { set_error("periodic_mask names an axis beyond ndim"); return NET_EINVAL; }
    if ((d->periodic_mask >> d->flow_axis) & 1u) { set_error("the flow axis cannot be periodic"); return NET_EINVAL; }
    if (d->periodic_mask & 1u) {
        // the compacted solve finds an x neighbour as the adjacent list entry
        set_error("periodic x is not supported: put the flow along x, periodic y/z");
        return NET_EINVAL;
    }
    for (int a = 1; a < d->ndim; a++)
        if (((d->periodic_mask >> a) & 1u) && d->n[a] < 3) {
            set_error("a periodic axis needs at least 3 nodes");
            return NET_EINVAL;
        }
    if (!std::isfinite(d->p_in) || !std::isfinite(d->p_out) || d->p_in == d->p_out) {
        set_error("face pressures must be finite and differ");
        return NET_EINVAL;
    }
    if (d->bond_dtype != NET_F64 && d->bond_dtype != NET_F32) { set_error("bad bond_dtype"); return NET_EINVAL; }
    Geom G{};
    G.ndim = d->ndim;
    G.f = d->flow_axis;
    G.nx = (int)d->n[0];
    G.ny = (int)d->n[1];
    G.nz = (int)d->n[2];
    G.px = (int)round_up(G.nx, 4);
    G.nf = (int)d->n[d->flow_axis];
    G.plane = (long long)G.px * G.ny;
    // zeros before and after the grid: one plane (3D) or row (2D) for the
    // stencil, plus a row and 16 bytes for the halo rows the sweep copies
    G.pad = round_up((d->ndim == 3 ? G.plane : (long long)G.px) + G.px + 64, 64);
    G.len = G.pad + G.plane * G.nz + G.pad;
    G.p_in = d->p_in;
    G.p_out = d->p_out;
    G.per = d->periodic_mask;
    if (G.len >= (1LL << 31)) { set_error("network too large (padded nodes >= 2^31)"); return NET_EINVAL; }
    *g = G;
    return NET_OK;
}

long long plane_elems(const Geom &g, int d) {
    long long m[3] = {g.nx, g.ny, g.nz};
    if (!g.periodic(d)) m[d] -= 1;  // a periodic plane has a bond per node
    return m[0] * m[1] * m[2];
}

size_t net_footprint_bytes(const Geom &g, int raw_f32) {
    const size_t L = (size_t)g.len, nd = (size_t)g.ndim;
    size_t b = nd * L * (raw_f32 ? 4 : 8);  // raw bonds
    b += L * (4 + 1 + 8 + 8);                // parent, cls, dis, x
    b += nd * L * 4;                         // scaled FP32 bonds
    b += 7 * L * 4;                          // FP32 inner vectors
    b += L * 4;                              // label flags (set-up only)
    b += L * 4;                              // dead-end roots (percolated networks)
    b += L * 4 * (2 * nd + 25);              // set-up only: dead-end loop pass (spanning nodes <= L)
    // list of unknowns and table when solved on the list: at most 35 % of
    // the lattice, or all of it for periodic networks (48 B per unknown in
    // FP32, 76 B in FP64)
    b += g.per ? L * 80 : L * 20;
    return b;
}

}  // namespace netsolve

// ---------------------------------------------------------------------------
namespace {

#define CK(call)                                                  \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);       \
    } while (0)

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DevGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

int netsolve::device_sm_count(int dev) {
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
        nsm = 152;
    return nsm;
}

net_status netsolve::ensure_precision(net_t *n, int f32, cudaStream_t st) {
    const int k = f32 ? 0 : 1;
    const size_t L = (size_t)n->g.len;
    const size_t es = f32 ? 4 : 8;
    if (!n->gs[k][0]) {
        for (int d = 0; d < n->g.ndim; d++) CK(dalloc(&n->gs[k][d], L * es, st));
        void *gs3[3] = {n->gs[k][0], n->gs[k][1], n->gs[k][2]};
        const void *gr[3] = {n->graw[0], n->graw[1], n->graw[2]};
        CK(launch_build_scaled(n->g, gr, n->raw_f32, n->dis, gs3, f32, st));
    }
    if (!n->vec[k]) CK(dalloc(&n->vec[k], 7 * L * es, st));
    return NET_OK;
}

namespace {

// The compacted solve replaces the lattice kernels when the unknowns are a
// small part of the lattice (its list traffic is about twice a lattice
// sweep's per node): below 35 % of the lattice nodes, or always with
// NETSOLVE_KERNEL=compact.  Of the lattice kernels only the persistent 2D
// one follows a periodic (y) boundary; periodic networks it does not take
// (3D, FP64 inner loop, wider than its rows) take the compacted solve, whose
// neighbour table holds the wrap bonds.
bool use_compact_kernel(const net_t *n, int f32) {
    if (n->n_solved <= 0) return false;
    const char *e = getenv("NETSOLVE_KERNEL");
    const bool forced = e && strcmp(e, "compact") == 0;
    const long long lattice = (long long)n->g.nx * n->g.ny * n->g.nz;
    const bool sparse = 100 * n->n_solved < 35 * lattice;
    if (n->g.per) return forced || sparse || !persist_applies(n->g, f32);
    if (forced) return true;
    if (e && *e) return false;
    return sparse;
}

bool use_persist_kernel(const net_t *n, int f32) {
    if (use_compact_kernel(n, f32)) return false;
    if (n->g.per) return persist_applies(n->g, f32);
    const char *e = getenv("NETSOLVE_KERNEL");
    if (e && (strcmp(e, "sweep") == 0 || strcmp(e, "compact") == 0)) return false;
    return persist_applies(n->g, f32);
}

net_status ensure_compact(net_t *n, int f32, cudaStream_t st) {
    const int k = f32 ? 0 : 1;
    CompactDev &cd = n->cp[k];
    if (cd.cidx) return NET_OK;
    net_status s = ensure_precision(n, f32, st);
    if (s != NET_OK) return s;
    const Geom &G = n->g;
    const long long U = n->n_solved;
    const size_t es = f32 ? 4 : 8, nd = (size_t)G.ndim;
    int *cmap = nullptr;
    CK(dalloc(&cmap, sizeof(int) * (size_t)G.len, st));
    CK(cudaMemsetAsync(cmap, 0xFF, sizeof(int) * (size_t)G.len, st));  // -1: not an unknown
    CK(dalloc(&cd.cidx, sizeof(int) * (size_t)U, st));
    CK(dalloc(&cd.nbr, sizeof(int) * 2 * (nd - 1) * (size_t)U, st));
    CK(dalloc(&cd.val, es * nd * (size_t)(U + 1), st));
    CK(dalloc(&cd.vec, es * 4 * (size_t)(U + 1), st));
    cd.grid = compact_grid(G.ndim, f32);
    CK(dalloc(&cd.pb, sizeof(double) * 2 * 4 * (size_t)cd.grid, st));
    CK(dalloc(&cd.bar, sizeof(unsigned) * 2, st));
    CK(dalloc(&cd.err, sizeof(int), st));
    const void *gs[3] = {n->gs[k][0], n->gs[k][1], n->gs[k][2] ? n->gs[k][2] : n->gs[k][0]};
    CK(compact_build(G, n->cls, U, f32, gs, cmap, cd.cidx, cd.nbr, cd.val, st));
    dfree(cmap, st);
    cd.U = U;
    CK(cudaStreamSynchronize(st));
    return NET_OK;
}

// Limit of a grid-barrier wait in the cooperative kernels: NETSOLVE_WAIT_NS
// (device nanoseconds), default 2 s.  A wait that gives up ends the solve
// with NET_ETIMEOUT.
unsigned long long grid_wait_ns() {
    const char *e = getenv("NETSOLVE_WAIT_NS");
    if (e && *e) {
        const long long v = atoll(e);
        if (v > 0) return (unsigned long long)v;
    }
    return 2000000000ULL;
}

// Testing aid: NETSOLVE_WITHHOLD_ARRIVAL=c makes CTA c of the cooperative
// kernels skip its first grid-barrier arrival, so that every other CTA's
// bounded wait runs out (the way a failure detection test makes it happen
// without faulting the GPU).  Unset: -1, no CTA withholds.
int withheld_arrival_cta() {
    const char *e = getenv("NETSOLVE_WITHHOLD_ARRIVAL");
    return (e && *e) ? atoi(e) : -1;
}

CompactArgs compact_args(net_t *n, int f32) {
    const int k = f32 ? 0 : 1;
    CompactDev &cd = n->cp[k];
    const size_t es = f32 ? 4 : 8, V = (size_t)(cd.U + 1);
    char *v = (char *)cd.vec;
    CompactArgs a{};
    a.n = cd.U;
    a.y = v;
    a.r = v + 1 * V * es;
    a.p = v + 2 * V * es;
    a.q = v + 3 * V * es;
    a.cidx = cd.cidx;
    a.val = cd.val;
    a.nbr = cd.nbr;
    a.s = &n->dsc->in[k];
    a.pb = cd.pb;
    a.bar = cd.bar;
    a.err = cd.err;
    a.wait_ns = grid_wait_ns();
    a.skip_cta = withheld_arrival_cta();
    return a;
}

net_status ensure_persist(net_t *n) {
    if (n->ps_hb) return NET_OK;
    cudaStream_t st = n->stream;
    const int grid = persist_grid(n->g);
    // halo copies: [sweep parity][CTA][first/last row][r, q, p][px]
    CK(dalloc(&n->ps_hb, sizeof(float) * 2 * 2 * 3 * (size_t)grid * n->g.px, st));
    CK(dalloc(&n->ps_pb, sizeof(float) * 2 * 8 * (size_t)grid, st));
    CK(dalloc(&n->ps_bar, sizeof(unsigned) * 2, st));
    CK(dalloc(&n->ps_err, sizeof(int), st));
    CK(persist_prepare());
    n->ps_grid = grid;
    return NET_OK;
}

// Plan the sweep for this one network with a tile shape and upload it (per
// precision); an existing plan of another shape is replaced.
net_status ensure_sweep_plan(net_t *n, int f32, const PlanShape &shape) {
    const int k = f32 ? 0 : 1;
    SweepDev &sd = n->sw[k];
    if (sd.segs && same_shape(sd.shape, shape)) return NET_OK;
    cudaStream_t st = n->stream;
    if (sd.segs) {
        dfree(sd.segs, st);
        dfree(sd.cta, st);
        dfree(sd.part, st);
        dfree(sd.inst, st);
        sd = SweepDev{};
    }
    HostPlan hp;
    std::vector<PlanNet> nets{PlanNet{n->g, true}};
    build_plan(nets, n->g.ndim, f32, device_sm_count(n->device), shape, hp);
    sd.grid = hp.grid;
    sd.shape = shape;
    CK(dalloc(&sd.segs, sizeof(SweepSeg) * hp.segs.size(), st));
    CK(dalloc(&sd.cta, sizeof(int) * hp.cta_begin.size(), st));
    CK(dalloc(&sd.part, sizeof(double) * 4 * (size_t)std::max(1, hp.nseg[0]), st));
    CK(dalloc(&sd.inst, sizeof(SweepInst), st));
    SweepInst si = sweep_inst_of(n, f32);
    si.part = sd.part;
    si.nseg = hp.nseg[0];
    CK(cudaMemcpyAsync(sd.segs, hp.segs.data(), sizeof(SweepSeg) * hp.segs.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(sd.cta, hp.cta_begin.data(), sizeof(int) * hp.cta_begin.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(sd.inst, &si, sizeof(SweepInst), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    return NET_OK;
}

// Tile shape for a single network's sweep plan: the tuned entry of its key,
// else tune now (before the solve arms its state), else the default.
net_status sweep_shape_for(net_t *n, int f32, PlanShape *shape) {
    *shape = PlanShape{};
    const Geom &G = n->g;
    if (tune_forced(G.ndim, f32, shape)) return NET_OK;
    const TuneKey key = tune_key(n->device, G.ndim, f32, (long long)G.px * G.ny * G.nz);
    TuneEntry te;
    if (tune_lookup(key, &te)) {
        *shape = te.shape;
        return NET_OK;
    }
    if (!tune_enabled() || n->n_active == 0) return NET_OK;
    double best_us = 0, def_us = 0;
    int nc = 0;
    std::vector<net_t *> one{n};
    return autotune_nets(one, f32, 1, n->stream, shape, &best_us, &def_us, &nc);
}

net_status ensure_graph(net_t *n, int f32, int K) {
    const int k = f32 ? 0 : 1;
    PlanShape shape;
    net_status s = sweep_shape_for(n, f32, &shape);
    if (s != NET_OK) return s;
    if (n->gexec[k] && n->gk[k] == K && n->sw[k].segs && same_shape(n->sw[k].shape, shape))
        return NET_OK;
    if (n->gexec[k]) {
        cudaGraphExecDestroy(n->gexec[k]);
        n->gexec[k] = nullptr;
    }
    s = ensure_sweep_plan(n, f32, shape);
    if (s != NET_OK) return s;
    CK(sweep_prepare(n->g.ndim, f32));
    const SweepDev &sd = n->sw[k];
    cudaStream_t cs;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    for (int i = 0; e == cudaSuccess && i < K; i++)
        e = launch_sweep(n->g.ndim, f32, sd.grid, sd.inst, sd.segs, sd.cta, cs);
    cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&n->gexec[k], graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return cuda_fail(e, "inner graph");
    n->gk[k] = K;
    return NET_OK;
}

}  // namespace

namespace netsolve {

InnerArgs inner_args(net_t *n, int f32) {
    const int k = f32 ? 0 : 1;
    const size_t L = (size_t)n->g.len, es = f32 ? 4 : 8;
    char *v = (char *)n->vec[k];
    InnerArgs a{};
    a.g = n->g;
    for (int d = 0; d < 3; d++) a.gs[d] = n->gs[k][d] ? n->gs[k][d] : n->gs[k][0];
    a.y = v;
    a.r[0] = v + 1 * L * es;
    a.r[1] = v + 2 * L * es;
    a.p[0] = v + 3 * L * es;
    a.p[1] = v + 4 * L * es;
    a.q[0] = v + 5 * L * es;
    a.q[1] = v + 6 * L * es;
    a.s = &n->dsc->in[k];
    a.partials = n->partials;
    return a;
}

OuterArgs outer_args(net_t *n, int f32, int apply_corr, int corr_f32, const net_opts &op, int inplace) {
    const int k = f32 ? 0 : 1, kc = corr_f32 ? 0 : 1;
    OuterArgs o{};
    o.g = n->g;
    for (int d = 0; d < 3; d++) o.graw[d] = n->graw[d] ? n->graw[d] : n->graw[0];
    o.raw_f32 = n->raw_f32;
    o.dis = n->dis;
    o.x = n->x;
    // the correction comes from the inner precision used last
    o.y = n->vec[kc];
    o.apply_corr = apply_corr && n->vec[kc] != nullptr;
    o.corr_f32 = corr_f32;
    // inner vectors: y, r0, r1, p0, p1, q0, q1 (in-place kernels use r0, p0, q0)
    const size_t L = (size_t)n->g.len, es = f32 ? 4 : 8, esc = corr_f32 ? 4 : 8;
    char *v = (char *)n->vec[k];
    o.r_buf[0] = v + 1 * L * es;
    o.r_buf[1] = inplace ? o.r_buf[0] : v + 2 * L * es;
    const char *vc = (const char *)n->vec[kc];
    o.p_buf[0] = vc ? vc + 3 * L * esc : nullptr;
    o.p_buf[1] = vc ? (inplace ? o.p_buf[0] : vc + 4 * L * esc) : nullptr;
    o.inner_f32 = f32;
    o.os = &n->dsc->os;
    o.is = &n->dsc->in[k];
    o.is_corr = &n->dsc->in[kc];
    const bool rel_mode = op.refine != NET_REFINE_RESTART;
    o.reliable = rel_mode;
    o.allow_cont = rel_mode && o.apply_corr && k == kc;
    const double dl = op.update_delta > 0.0 && op.update_delta < 1.0 ? op.update_delta : 1e-3;
    o.delta2 = rel_mode && f32 ? dl * dl : 0.0;
    o.tol_floor = f32 && !rel_mode ? op.tol_inner : 0.0;
    o.tol_rel = op.tol_rel;
    o.tol_geff = op.tol_geff > 0.0 ? op.tol_geff : 1e-9;
    o.bnorm = n->bnorm;
    o.max_inner = op.max_inner;
    // An inner loop that has not halved its residual norm for this many
    // iterations ends its pass, and the next pass restarts CG.  On
    // near-critical networks the residual plateaus for hundreds of iterations
    // between drops, and a restart throws away the Krylov space, so the window
    // is long unless FP32 passes restart anyway (restart mode), where a stall
    // is more likely the FP32 precision floor.  (In reliable mode that floor
    // shows at the pass boundaries, in the true residual.)
    const long long side = std::max(n->g.nx, std::max(n->g.ny, n->g.nz));
    o.stag_window = f32 && !rel_mode ? std::max(400LL, 8LL * side) : std::max(4000LL, 64LL * side);
    o.partials = n->partials;
    o.root = n->proot;
    return o;
}

SweepInst sweep_inst_of(net_t *n, int f32) {
    InnerArgs a = inner_args(n, f32);
    SweepInst si{};
    si.g = n->g;
    for (int d = 0; d < 3; d++) si.gs[d] = a.gs[d];
    si.y = a.y;
    for (int j = 0; j < 2; j++) {
        si.r[j] = a.r[j];
        si.p[j] = a.p[j];
        si.q[j] = a.q[j];
    }
    si.s = a.s;
    si.part = nullptr;
    si.nseg = 0;
    return si;
}

net_status arm_for_tuning(net_t *n, int f32, cudaStream_t st) {
    net_opts o;
    net_opts_default(&o);
    o.refine = NET_REFINE_RESTART;
    OuterArgs oa = outer_args(n, f32, 0, f32, o, 0);
    oa.tol_rel = 0.0;
    oa.tol_geff = 0.0;
    oa.tol_floor = 0.0;
    oa.reliable = 0;
    oa.allow_cont = 0;
    oa.delta2 = 0.0;
    CK(launch_outer(oa, st));
    return NET_OK;
}

net_status autotune_nets(const std::vector<net_t *> &nets, int f32, int default_seg, cudaStream_t st,
                         PlanShape *best, double *best_us, double *def_us, int *ncand) {
    *best = PlanShape{};
    best->seg_per_sm = default_seg;
    *best_us = *def_us = 0.0;
    *ncand = 0;
    if (nets.empty()) return NET_OK;
    const int ndim = nets[0]->g.ndim, dev = nets[0]->device;
    long long nodes = 0;
    std::vector<PlanNet> pn;
    std::vector<SweepInst> si;
    for (net_t *n : nets) {
        if (n->g.ndim != ndim || n->device != dev) {
            set_error("autotune: networks differ in dimension or device");
            return NET_EINVAL;
        }
        if (n->stream != st) {  // the network's own stream may still hold its set-up work
            CK(cudaEventRecord(n->ev[3], n->stream));
            CK(cudaStreamWaitEvent(st, n->ev[3], 0));
        }
        net_status s = ensure_precision(n, f32, st);
        if (s != NET_OK) return s;
        nodes += (long long)n->g.px * n->g.ny * n->g.nz;
        pn.push_back(PlanNet{n->g, true});
        si.push_back(sweep_inst_of(n, f32));
    }
    const std::vector<PlanShape> cands = tune_candidates(ndim, f32, default_seg);
    const int nsm = device_sm_count(dev);
    // 8 sweeps per graph, 3 timed replays after one warm replay: every
    // candidate starts from the same freshly armed state
    const int K = 8, R = 3;
    double bu = -1.0;
    for (size_t c = 0; c < cands.size(); c++) {
        for (net_t *n : nets) {
            net_status s = arm_for_tuning(n, f32, st);
            if (s != NET_OK) return s;
        }
        const double us = tune_time_shape(pn, si, ndim, f32, nsm, cands[c], K, R, st);
        if (us < 0.0) return NET_ECUDA;
        if (c == 0) *def_us = us;
        // a candidate must beat the best so far by 2 % (timing noise)
        if (bu < 0.0 || us < 0.98 * bu) {
            bu = us;
            *best = cands[c];
        }
    }
    *best_us = bu;
    *ncand = (int)cands.size();
    TuneEntry te;
    te.shape = *best;
    te.us_per_sweep = bu;
    te.candidates = *ncand;
    tune_store(tune_key(dev, ndim, f32, nodes), te);
    if (trace_on())
        fprintf(stderr, "[trace autotune] %dD %s nets %zu nodes %lld: wcap %d hcap %d seg %d %.2f us (default %.2f)\n",
                ndim, f32 ? "f32" : "f64", nets.size(), nodes, best->wcap, best->hcap, best->seg_per_sm, bu,
                *def_us);
    return NET_OK;
}

// Outer correction with y of one precision but the residual written for
// another needs both inner buffers; outer_kernel reads y as the *target*
// precision's type, so a switch of precision first re-arms with no correction
// pending (see solve_impl).

// NETSOLVE_PRUNE: "0" keeps every spanning node in the linear system,
// "trees" strips dead-end trees only, anything else (the default) strips
// dead-end trees and then dead-end loops (the current-carrying backbone).
int prune_level() {
    const char *e = getenv("NETSOLVE_PRUNE");
    if (e && strcmp(e, "0") == 0) return 0;
    if (e && strcmp(e, "trees") == 0) return 1;
    return 2;
}
bool prune_enabled() { return prune_level() > 0; }

// Strip the parts of the spanning clusters that carry no current.  Level 1
// (NETSOLVE_PRUNE=trees): rounds of removing nodes with at most one link left
// (see prune_round_kernel), then every removed node resolved to the backbone
// or face node its tree hangs from; the removed set is exact at any point, so
// stopping after kMaxRounds only leaves deeper trees in the system.  Level 2
// (the default): the biconnectivity pass of blocks.cu, which removes trees
// and dead-end loops alike.  `pr` is a zeroable L-word scratch buffer.
net_status prune_dead_ends(net_t *n, const void *const gr[3], unsigned int *pr) {
    constexpr unsigned int kChunk = 16, kMaxRounds = 1u << 14;
    cudaStream_t st = n->stream;
    const Geom &G = n->g;
    const size_t L = (size_t)G.len;
    CK(cudaMemsetAsync(pr, 0, L * 4, st));
    CK(dalloc(&n->proot, L * 4, st));
    CK(cudaMemsetAsync(n->proot, 0xFF, L * 4, st));  // -1: not removed
    unsigned int round = 0;
    unsigned long long total = 0;
    // The biconnectivity pass removes dead-end trees too (no tree node lies on
    // a path between the faces), in one pass instead of a lattice sweep per
    // tree generation: the rounds run only when trees alone are stripped.
    while (prune_level() == 1 && round < kMaxRounds) {
        CK(cudaMemsetAsync(&n->dsc->ss.pruned, 0, sizeof(unsigned int), st));
        for (unsigned int k = 0; k < kChunk; k++)
            CK(launch_prune_round(G, gr, n->raw_f32, n->cls, pr, n->proot, ++round, &n->dsc->ss.pruned, st));
        CK(cudaMemcpyAsync(&n->hsc->ss.pruned, &n->dsc->ss.pruned, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        total += n->hsc->ss.pruned;
        if (n->hsc->ss.pruned == 0) break;
    }
    if (total > 0) {
        int passes = 1;
        while ((1u << passes) <= round) passes++;
        CK(launch_prune_finish(G, n->cls, pr, n->proot, passes + 1, st));
        n->prune_rounds = (int)round;
    }
    long long loops = 0;
    if (prune_level() >= 2) {
        int bad = 0;
        CK(strip_dead_loops(G, gr, n->raw_f32, n->cls, n->proot, (int *)pr, &loops, &bad, st));
        if (bad) {
            set_error("dead-end loop stripping: internal consistency check %d failed", bad);
            return NET_ECUDA;
        }
        n->loop_nodes = loops;
    }
    if (total == 0 && loops == 0) {
        dfree(n->proot, st);
        n->proot = nullptr;
    }
    return NET_OK;
}

net_status setup_network(net_t *n, const void *const g[3], int on_device) {
    cudaStream_t st = n->stream;
    const Geom &G = n->g;
    const size_t L = (size_t)G.len, rs = n->raw_f32 ? 4 : 8;
    for (int d = 0; d < G.ndim; d++) CK(dalloc(&n->graw[d], L * rs, st));
    CK(dalloc(&n->parent, L * 4, st));
    CK(dalloc(&n->cls, L, st));
    CK(dalloc(&n->dis, L * 8, st));
    CK(dalloc(&n->x, L * 8, st));
    const long long nb = std::max<long long>(
        {(long long)outer_grid_blocks(G), 152LL * 16});
    CK(dalloc(&n->partials, (size_t)nb * 8 * sizeof(double), st));
    CK(dalloc(&n->dsc, sizeof(DevScal), st));
    unsigned int *flags = nullptr;
    CK(dalloc(&flags, L * 4, st));
    void *stage = nullptr;
    for (int d = 0; d < G.ndim; d++) {
        const long long m = plane_elems(G, d);
        if (m == 0) continue;  // plane of extent 0: nothing to copy
        if (!g || !g[d]) { dfree(flags, st); set_error("bond plane %d is NULL", d); return NET_EINVAL; }
        const void *src = g[d];
        if (!on_device) {
            if (!stage) CK(dalloc(&stage, (size_t)std::max({plane_elems(G, 0), plane_elems(G, 1),
                                                           G.ndim == 3 ? plane_elems(G, 2) : 0LL}) * rs, st));
            CK(cudaMemcpyAsync(stage, g[d], (size_t)m * rs, cudaMemcpyHostToDevice, st));
            src = stage;
        }
        CK(launch_pack_bonds(G, d, src, n->raw_f32, n->graw[d], n->raw_f32, &n->dsc->ss.bad, st));
    }
    const void *gr[3] = {n->graw[0], n->graw[1], G.ndim == 3 ? n->graw[2] : n->graw[0]};
    CK(launch_labels(G, gr, n->raw_f32, n->parent, flags, n->cls, st));
    if (prune_enabled()) {
        net_status ps = prune_dead_ends(n, gr, flags);
        if (ps != NET_OK) { dfree(flags, st); dfree(stage, st); return ps; }
    }
    CK(launch_build_system(G, gr, n->raw_f32, n->cls, n->dis, n->x, &n->dsc->ss, n->partials, st));
    dfree(flags, st);
    dfree(stage, st);
    CK(cudaMemcpyAsync(n->hsc, n->dsc, sizeof(DevScal), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (n->hsc->ss.bad) {
        set_error("a conductance is negative, NaN or infinite");
        return NET_EINVAL;
    }
    n->bnorm = std::sqrt(n->hsc->ss.bb);
    n->n_active = (long long)n->hsc->ss.n_active;
    n->n_solved = (long long)n->hsc->ss.n_solved;
    return NET_OK;
}

void release_network(net_t *n) {
    if (!n) return;
    cudaStream_t st = n->stream;
    for (int k = 0; k < 2; k++) {
        CompactDev &cd = n->cp[k];
        dfree(cd.cidx, st);
        dfree(cd.nbr, st);
        dfree(cd.val, st);
        dfree(cd.vec, st);
        dfree(cd.pb, st);
        dfree(cd.bar, st);
        dfree(cd.err, st);
        if (n->gexec[k]) cudaGraphExecDestroy(n->gexec[k]);
        dfree(n->sw[k].segs, st);
        dfree(n->sw[k].cta, st);
        dfree(n->sw[k].part, st);
        dfree(n->sw[k].inst, st);
        for (int d = 0; d < 3; d++) dfree(n->gs[k][d], st);
        dfree(n->vec[k], st);
    }
    for (int d = 0; d < 3; d++) dfree(n->graw[d], st);
    dfree(n->ps_hb, st);
    dfree(n->ps_pb, st);
    dfree(n->ps_bar, st);
    dfree(n->ps_err, st);
    dfree(n->parent, st);
    dfree(n->proot, st);
    dfree(n->cls, st);
    dfree(n->dis, st);
    dfree(n->x, st);
    dfree(n->partials, st);
    dfree(n->dsc, st);
    cudaStreamSynchronize(st);
    if (n->hsc) cudaFreeHost(n->hsc);
    if (n->ev[0]) for (int i = 0; i < 4; i++) cudaEventDestroy(n->ev[i]);
    if (n->own_stream) cudaStreamDestroy(n->stream);
    delete n;
}

net_status create_network(const net_desc *desc, const void *const g[3], net_t **out) {
    if (!out) { set_error("out is NULL"); return NET_EINVAL; }
    *out = nullptr;
    Geom G;
    net_status s = make_geom(desc, &G);
    if (s != NET_OK) return s;
    net_t *n = new net_t();
    n->g = G;
    n->raw_f32 = desc->bond_dtype == NET_F32;
    cudaGetDevice(&n->device);
    cudaError_t e;
    if (desc->stream) {
        n->stream = (cudaStream_t)desc->stream;
        n->own_stream = false;
    } else {
        e = cudaStreamCreateWithFlags(&n->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete n; return cuda_fail(e, "stream"); }
        n->own_stream = true;
    }
    e = cudaMallocHost(&n->hsc, sizeof(DevScal));
    if (e == cudaSuccess)
        for (int i = 0; i < 4 && e == cudaSuccess; i++) e = cudaEventCreate(&n->ev[i]);
    if (e != cudaSuccess) { release_network(n); return cuda_fail(e, "host state"); }
    s = setup_network(n, g, desc->on_device);
    if (s != NET_OK) {
        std::string keep = g_err;
        release_network(n);
        g_err = keep;
        return s;
    }
    *out = n;
    return NET_OK;
}

// L2 set-aside for the persistent kernel's vectors (see cg_persist.cu): a
// per-context limit, set for the duration of one solve and put back to 0
// (with the persisting lines reset) before the solve returns, so nothing of
// it outlasts the call and later work sees the whole L2 again.
// NETSOLVE_L2_KEEP=0 leaves the limit alone.
struct L2Keep {
    bool on = false;
    void begin(const net_t *n) {
        const char *e = getenv("NETSOLVE_L2_KEEP");
        if (e && strcmp(e, "0") == 0) return;
        int maxp = 0;
        if (cudaDeviceGetAttribute(&maxp, cudaDevAttrMaxPersistingL2CacheSize, n->device) != cudaSuccess ||
            maxp <= 0)
            return;
        size_t want = (size_t)4 * (size_t)n->g.len * sizeof(float);  // y, r, p, q
        if (want > (size_t)maxp) want = (size_t)maxp;
        on = cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want) == cudaSuccess;
    }
    void end() {
        if (!on) return;
        cudaCtxResetPersistingL2Cache();
        cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, 0);
        on = false;
    }
    ~L2Keep() { end(); }
};

// One refinement pass of the single-network driver: the correction (if
// apply_corr), the FP64 residual and flows, and the next inner solve armed.
// For the compacted solve the correction is applied on the list, and the new
// scaled residual is gathered from the lattice into the list.
net_status outer_pass_single(net_t *n, int f32, int apply_corr, const net_opts &o, cudaStream_t st) {
    if (use_compact_kernel(n, f32)) return outer_pass_compact(n, f32, apply_corr, o, st);
    OuterArgs oa = outer_args(n, f32, apply_corr, f32, o, use_persist_kernel(n, f32));
    CK(launch_outer(oa, st));
    return NET_OK;
}

// The refinement pass of a network solved on its list of unknowns: the
// correction applied on the list, the FP64 residual on the lattice, the new
// scaled residual gathered into the list.
net_status outer_pass_compact(net_t *n, int f32, int apply_corr, const net_opts &o, cudaStream_t st) {
    net_status s = ensure_compact(n, f32, st);
    if (s != NET_OK) return s;
    const CompactArgs ca = compact_args(n, f32);
    if (apply_corr) CK(launch_compact_correct(ca, n->dis, n->x, f32, st));
    OuterArgs oa = outer_args(n, f32, 0, f32, o, 1);
    oa.allow_cont = o.refine != NET_REFINE_RESTART && apply_corr;  // correction applied above
    // residual over the listed nodes only, written straight to the list
    // (256^3 percolation: 1.11 M of 16.8 M nodes)
    CK(launch_outer_list(oa, ca.cidx, ca.n, ca.r, st));
    return NET_OK;
}

// In a batch the list path's launches are shared by all its members, so it
// may pay at a higher density than for a network solved alone:
// NETSOLVE_BATCH_COMPACT_BELOW (a fraction of the lattice) overrides the
// 35 % of use_compact_kernel for batch members.
bool batch_takes_compact(const net_t *n, int f32) {
    if (n->g.per != 0) return true;
    const char *e = getenv("NETSOLVE_BATCH_COMPACT_BELOW");
    if (e && *e && n->n_solved > 0) {
        const double frac = atof(e);
        const long long lattice = (long long)n->g.nx * n->g.ny * n->g.nz;
        return (double)n->n_solved < frac * (double)lattice;
    }
    return use_compact_kernel(n, f32);
}

net_status prepare_compact(net_t *n, int f32, cudaStream_t st) { return ensure_compact(n, f32, st); }

CompactArgs compact_args_of(net_t *n, int f32) { return compact_args(n, f32); }

// One solve.  Returns the status and fills *r.
net_status solve_impl(net_t *n, const net_opts *o_in, net_result *r) {
    net_opts o;
    net_opts_default(&o);
    if (o_in) o = *o_in;
    memset(r, 0, sizeof(*r));
    if (!opts_valid(o)) return r->status = NET_EINVAL;
    cudaStream_t st = o.stream ? (cudaStream_t)o.stream : n->stream;
    const Geom &G = n->g;
    const double dP = G.p_in - G.p_out;
    int f32 = o.precision == NET_MIXED;
    const int K = o.check_every > 0 ? o.check_every : 32;
    if (st != n->stream) {
        // make the caller's stream wait for the network's set-up work
        CK(cudaEventRecord(n->ev[3], n->stream));
        CK(cudaStreamWaitEvent(st, n->ev[3], 0));
    }
    net_status s = ensure_precision(n, f32, st);
    if (s != NET_OK) return r->status = s;
    if (use_compact_kernel(n, f32)) {
        s = ensure_compact(n, f32, st);
        if (s != NET_OK) return r->status = s;
    } else if (!use_persist_kernel(n, f32) && !G.per) {
        // (a periodic network without unknowns runs no inner solve)
        s = ensure_graph(n, f32, K);
        if (s != NET_OK) return r->status = s;
    }

    CK(cudaEventRecord(n->ev[0], st));
    // fresh start: initial pressures, then the caller's guess
    {
        const void *gr[3] = {n->graw[0], n->graw[1], G.ndim == 3 ? n->graw[2] : n->graw[0]};
        CK(launch_build_system(G, gr, n->raw_f32, n->cls, n->dis, n->x, &n->dsc->ss, n->partials, st));
        if (o.x0) {
            const double *x0d = o.x0;
            double *tmp = nullptr;
            const size_t nb = sizeof(double) * (size_t)G.nx * G.ny * G.nz;
            if (!o.x0_on_device) {
                CK(dalloc(&tmp, nb, st));
                CK(cudaMemcpyAsync(tmp, o.x0, nb, cudaMemcpyHostToDevice, st));
                x0d = tmp;
            }
            CK(launch_apply_x0(G, n->cls, x0d, n->x, st));
            dfree(tmp, st);
        }
    }
    // first residual pass (no correction pending)
    s = outer_pass_single(n, f32, 0, o, st);
    if (s != NET_OK) return r->status = s;
    CK(cudaMemcpyAsync(&n->hsc->os, &n->dsc->os, sizeof(OuterScal), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const double bn = n->bnorm;
    double rel = bn > 0.0 ? std::sqrt(n->hsc->os.rr) / bn : 0.0;
    double dist = outer_dist(n, o, rel);
    int outer = 0;
    long long inner_total = 0, launches = 0;
    float inner_ms = 0.f;
    int fallback = 0;
    net_status status = NET_OK;
    Progress prog;
    prog.start(rel, geff_err(n));
    L2Keep l2keep;
    if (use_persist_kernel(n, f32) && dist > 1.0 && bn != 0.0) l2keep.begin(n);
    while (true) {
        if (dist <= 1.0 || bn == 0.0) break;
        if (outer >= o.max_outer) { status = NET_ENOTCONVERGED; break; }
        CK(cudaEventRecord(n->ev[1], st));
        long long chunks = 0;
        InnerScal *hs = &n->hsc->in[f32 ? 0 : 1];
        InnerScal *ds = &n->dsc->in[f32 ? 0 : 1];
        const int k = f32 ? 0 : 1;
        if (use_compact_kernel(n, f32)) {
            // the whole inner solve over the listed unknowns, one cooperative launch
            const CompactArgs ca = compact_args(n, f32);
            CK(launch_compact_cg(ca, G.ndim, f32, n->cp[k].grid, st));
            launches += 1;
            CK(cudaMemcpyAsync(&n->hsc->perr, ca.err, sizeof(int), cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(hs, ds, sizeof(InnerScal), cudaMemcpyDeviceToHost, st));
            CK(cudaEventRecord(n->ev[2], st));
            CK(cudaEventSynchronize(n->ev[2]));
            if (n->hsc->perr) {
                set_error("a bounded device wait in the compacted CG kernel gave up");
                return r->status = NET_ETIMEOUT;
            }
        } else if (use_persist_kernel(n, f32)) {
            // the whole inner solve in one cooperative launch
            s = ensure_persist(n);
            if (s != NET_OK) return r->status = s;
            InnerArgs ia = inner_args(n, 1);
            PersistArgs pa{};
            pa.g = G;
            pa.gx = (const float *)ia.gs[0];
            pa.gy = (const float *)ia.gs[1];
            pa.y = (float *)ia.y;
            pa.r = (float *)ia.r[0];
            pa.p = (float *)ia.p[0];
            pa.q = (float *)ia.q[0];
            pa.s = ds;
            pa.hb = n->ps_hb;
            pa.pb = n->ps_pb;
            pa.bar_count = n->ps_bar;
            pa.err = n->ps_err;
            pa.wait_ns = grid_wait_ns();
            pa.skip_cta = withheld_arrival_cta();
            CK(launch_persist_resume(pa, n->ps_grid, st));
            CK(launch_persist(pa, n->ps_grid, st));
            chunks = 0;
            launches += 1;
            CK(cudaMemcpyAsync(&n->hsc->perr, n->ps_err, sizeof(int), cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(hs, ds, sizeof(InnerScal), cudaMemcpyDeviceToHost, st));
            CK(cudaEventRecord(n->ev[2], st));
            CK(cudaEventSynchronize(n->ev[2]));
            if (n->hsc->perr) {
                set_error("a bounded device wait in the persistent CG kernel gave up");
                return r->status = NET_ETIMEOUT;
            }
        } else {
        // keep one chunk in flight ahead of the flag read
        CK(cudaGraphLaunch(n->gexec[k], st));
        chunks++;
        while (true) {
            CK(cudaMemcpyAsync(hs, ds, sizeof(InnerScal), cudaMemcpyDeviceToHost, st));
            CK(cudaEventRecord(n->ev[2], st));
            CK(cudaGraphLaunch(n->gexec[k], st));
            chunks++;
            CK(cudaEventSynchronize(n->ev[2]));
            if (hs->stop) break;
            if ((chunks - 2) * (long long)n->gk[k] > o.max_inner) {
                // the device cap should have stopped the loop by now
                set_error("inner loop did not stop after %lld launches", chunks * (long long)n->gk[k]);
                return r->status = NET_ETIMEOUT;
            }
        }
        CK(cudaEventRecord(n->ev[2], st));
        CK(cudaEventSynchronize(n->ev[2]));
        CK(cudaMemcpyAsync(hs, ds, sizeof(InnerScal), cudaMemcpyDeviceToHost, st));
        }
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, n->ev[1], n->ev[2]));
        CK(cudaStreamSynchronize(st));
        inner_ms += ms;
        launches += chunks * n->gk[k];
        inner_total += hs->iter - hs->iter0;
        if (hs->stop == 5) {
            set_error("a bounded device wait in the CG kernel gave up");
            return r->status = NET_ETIMEOUT;
        }
        outer++;
        // apply the correction, new residual; arm the same precision again
        s = outer_pass_single(n, f32, 1, o, st);
        if (s != NET_OK) return r->status = s;
        CK(cudaMemcpyAsync(&n->hsc->os, &n->dsc->os, sizeof(OuterScal), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        rel = std::sqrt(n->hsc->os.rr) / bn;
        dist = outer_dist(n, o, rel);
        trace_outer(n, "solve", outer, f32, hs->stop, hs->iter - hs->iter0, rel);
        // FP32 passes that stopped making progress: continue in FP64
        if (prog.stalled(rel, geff_err(n), stall_limit(o)) && f32 && dist > 1.0) {
            f32 = 0;
            fallback = 1;
            s = ensure_precision(n, 0, st);
            if (s != NET_OK) return r->status = s;
            if (!use_persist_kernel(n, 0) && !use_compact_kernel(n, 0) && !G.per) {
                s = ensure_graph(n, 0, K);
                if (s != NET_OK) return r->status = s;
            }
            // re-arm the FP64 inner solve from the current x (no correction pending)
            s = outer_pass_single(n, 0, 0, o, st);
            if (s != NET_OK) return r->status = s;
            CK(cudaMemcpyAsync(&n->hsc->os, &n->dsc->os, sizeof(OuterScal), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            rel = std::sqrt(n->hsc->os.rr) / bn;
            dist = outer_dist(n, o, rel);
            prog.start(rel, geff_err(n));
        }
    }
    CK(cudaEventRecord(n->ev[2], st));
    CK(cudaEventSynchronize(n->ev[2]));
    l2keep.end();
    float total_ms = 0.f;
    CK(cudaEventElapsedTime(&total_ms, n->ev[0], n->ev[2]));
    const OuterScal &os = n->hsc->os;
    r->q_in = os.qin;
    r->q_out = os.qout;
    r->g_eff = os.qin / dP;
    double S = 1.0;
    const long long ext[3] = {G.nx, G.ny, G.nz};
    for (int a = 0; a < G.ndim; a++)
        if (a != G.f) S *= (double)ext[a];
    r->k_eff = r->g_eff * (double)(G.nf - 1) / S;
    r->rel_residual = rel;
    r->max_imbalance = os.rmax;
    r->energy_g = os.energy / (dP * dP);
    r->n_active = n->n_active;
    r->outer_iters = outer;
    r->inner_iters = inner_total;
    r->fp64_fallback = fallback;
    r->ms = total_ms;
    r->inner_ms = inner_ms;
    r->inner_launches = launches;
    r->g_eff_err = geff_err(n);
    r->n_solved = n->n_solved;
    r->status = status;
    n->last = *r;
    n->solved = true;
    if (status != NET_OK) set_error("not converged: relative residual %.3e after %d refinement steps", rel, outer);
    return status;
}

}  // namespace netsolve

// ---------------------------------------------------------------------------
// exported C ABI
// ---------------------------------------------------------------------------
#define NET_API extern "C" __attribute__((visibility("default")))

NET_API void net_opts_default(net_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->precision = NET_MIXED;
    o->tol_rel = 1e-11;
    o->tol_inner = 1e-4;
    o->max_outer = 200;
    o->max_inner = 200000;
    o->check_every = 0;
    o->tol_geff = 1e-9;
    o->refine = NET_REFINE_RELIABLE;
    o->update_delta = 1e-3;
}

NET_API net_status net_autotune(net_t *const *nets, int count, const net_opts *opts, net_tune *out) {
    if (count < 1 || !nets) {
        set_error("net_autotune: no networks");
        return NET_EINVAL;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    std::vector<net_t *> v;
    for (int i = 0; i < count; i++) {
        if (!nets[i] || nets[i]->device != dev) {
            set_error("net_autotune: network %d is NULL or on another device", i);
            return NET_EINVAL;
        }
        if (nets[i]->g.ndim != nets[0]->g.ndim) {
            set_error("net_autotune: networks mix 2D and 3D");
            return NET_EINVAL;
        }
        if (nets[i]->g.per) {
            set_error("net_autotune: network %d is periodic (it takes the compacted solve)", i);
            return NET_EINVAL;
        }
        v.push_back(nets[i]);
    }
    const int f32 = !opts || opts->precision == NET_MIXED;
    cudaStream_t st = opts && opts->stream ? (cudaStream_t)opts->stream : nets[0]->stream;
    PlanShape best;
    double bu = 0, du = 0;
    int nc = 0;
    // a set of one network is planned as net_solve plans it (one segment per
    // SM by default), a larger set as net_solve_batch does (two)
    net_status s = autotune_nets(v, f32, count == 1 ? 1 : 2, st, &best, &bu, &du, &nc);
    if (s != NET_OK) return s;
    if (out) {
        long long nodes = 0;
        for (net_t *n : v) nodes += (long long)n->g.px * n->g.ny * n->g.nz;
        const int ndim = v[0]->g.ndim;
        const int wmax = sweep_max_width(ndim, f32);
        const int w = best.wcap > 0 ? best.wcap : wmax;
        const int cap = sweep_consumers() * sweep_vt(f32);
        out->col_block = w;
        out->row_band = ndim == 3 ? std::min(best.hcap > 0 ? best.hcap : 32, cap / w) : 1;
        out->seg_per_sm = best.seg_per_sm;
        out->size_class = tune_key(dev, ndim, f32, nodes).size_class;
        out->candidates = nc;
        out->us_per_sweep = bu;
        out->us_default = du;
    }
    return NET_OK;
}

NET_API void net_tune_clear(void) { tune_clear(); }

NET_API net_status net_create(const net_desc *desc, const void *const g[3], net_t **out) {
    return create_network(desc, g, out);
}

NET_API net_status net_solve(net_t *net, const net_opts *opts, net_result *out) {
    if (!net || !out) { set_error("net_solve: NULL argument"); return NET_EINVAL; }
    DevGuard dg(net->device);
    return solve_impl(net, opts, out);
}

NET_API net_status net_flux(net_t *net, double *q_in, double *q_out, double *g_eff) {
    if (!net) { set_error("net_flux: NULL handle"); return NET_EINVAL; }
    if (!net->solved) { set_error("net_flux: no solve yet"); return NET_EINVAL; }
    if (q_in) *q_in = net->last.q_in;
    if (q_out) *q_out = net->last.q_out;
    if (g_eff) *g_eff = net->last.g_eff;
    return NET_OK;
}

NET_API net_status net_get_pressure(net_t *net, double *dst, int64_t n, int dst_on_device) {
    if (!net || !dst) { set_error("net_get_pressure: NULL argument"); return NET_EINVAL; }
    const Geom &G = net->g;
    const long long N = (long long)G.nx * G.ny * G.nz;
    if (n < N) { set_error("net_get_pressure: buffer holds %lld < %lld", (long long)n, N); return NET_EINVAL; }
    DevGuard dg(net->device);
    cudaStream_t st = net->stream;
    if (dst_on_device) {
        CK(launch_unpack_x(G, net->x, dst, st));
        CK(cudaStreamSynchronize(st));
        return NET_OK;
    }
    double *tmp = nullptr;
    CK(dalloc(&tmp, sizeof(double) * (size_t)N, st));
    CK(launch_unpack_x(G, net->x, tmp, st));
    CK(cudaMemcpyAsync(dst, tmp, sizeof(double) * (size_t)N, cudaMemcpyDeviceToHost, st));
    dfree(tmp, st);
    CK(cudaStreamSynchronize(st));
    return NET_OK;
}

NET_API net_status net_get_labels(net_t *net, int32_t *label, uint8_t *cls, int64_t n) {
    if (!net) { set_error("net_get_labels: NULL handle"); return NET_EINVAL; }
    const Geom &G = net->g;
    const long long N = (long long)G.nx * G.ny * G.nz;
    if (n < N) { set_error("net_get_labels: buffer holds %lld < %lld", (long long)n, N); return NET_EINVAL; }
    DevGuard dg(net->device);
    cudaStream_t st = net->stream;
    int *dl = nullptr;
    uint8_t *dc = nullptr;
    CK(dalloc(&dl, sizeof(int) * (size_t)N, st));
    CK(dalloc(&dc, (size_t)N, st));
    CK(launch_unpack_labels(G, net->parent, net->cls, dl, dc, st));
    if (label) CK(cudaMemcpyAsync(label, dl, sizeof(int) * (size_t)N, cudaMemcpyDeviceToHost, st));
    if (cls) CK(cudaMemcpyAsync(cls, dc, (size_t)N, cudaMemcpyDeviceToHost, st));
    dfree(dl, st);
    dfree(dc, st);
    CK(cudaStreamSynchronize(st));
    return NET_OK;
}

NET_API net_status net_get_backbone(net_t *net, uint8_t *backbone, int64_t n) {
    if (!net || !backbone) { set_error("net_get_backbone: NULL argument"); return NET_EINVAL; }
    const Geom &G = net->g;
    const long long N = (long long)G.nx * G.ny * G.nz;
    if (n < N) { set_error("net_get_backbone: buffer holds %lld < %lld", (long long)n, N); return NET_EINVAL; }
    DevGuard dg(net->device);
    cudaStream_t st = net->stream;
    uint8_t *db = nullptr;
    CK(dalloc(&db, (size_t)N, st));
    CK(launch_backbone(G, net->cls, db, st));
    CK(cudaMemcpyAsync(backbone, db, (size_t)N, cudaMemcpyDeviceToHost, st));
    dfree(db, st);
    CK(cudaStreamSynchronize(st));
    return NET_OK;
}

NET_API net_status net_destroy(net_t *net) {
    if (!net) return NET_OK;
    DevGuard dg(net->device);
    release_network(net);
    return NET_OK;
}

NET_API const char *net_last_error(void) { return last_error(); }
