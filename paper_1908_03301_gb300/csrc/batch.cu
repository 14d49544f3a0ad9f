// batch.cu -- the batch engine and net_solve_batch.
//
// Many independent networks share every sweep launch (sweep_kernel walks all
// running networks' segments, each network with its own CG scalars), so the
// GPU stays full even when each network alone is small.  See batch.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "../../include/netsolve.h"
#include "batch.h"
#include "kernels.h"
#include "plan.h"
#include "sweep.cuh"
#include "tune.h"

namespace netsolve {
namespace {

__global__ void gather_status_kernel(const InnerScal *const *s, int n, int *stop, long long *iter) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        stop[i] = s[i]->stop;
        iter[i] = s[i]->iter - s[i]->iter0;  // iterations of this pass
    }
}

__global__ void set_stop_kernel(InnerScal *s, int v) { s->stop = v; }

__global__ void retire_kernel(SweepInst *inst, int idx, InnerScal *dead) { inst[idx].s = dead; }
__global__ void retire_compact_kernel(CompactInst *inst, int idx, InnerScal *dead) { inst[idx].a.s = dead; }

#define CKB(call)                                                \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);      \
    } while (0)

template <typename T>
cudaError_t grow(T **p, size_t *cap, size_t need, cudaStream_t st) {
    if (*cap >= need && *p) return cudaSuccess;
    if (*p) cudaFreeAsync(*p, st);
    *p = nullptr;
    size_t n = std::max(need, (size_t)16);
    n = n + n / 2;
    cudaError_t e = cudaMallocAsync((void **)p, n * sizeof(T), st);
    if (e == cudaSuccess) *cap = n;
    return e;
}

}  // namespace

BatchEngine::BatchEngine(int device, cudaStream_t stream) : device_(device), st_(stream) {
    nsm_ = 0;
    if (cudaDeviceGetAttribute(&nsm_, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || nsm_ <= 0)
        nsm_ = 152;
    for (int c = 0; c < 2; c++)
        for (int d = 0; d < 2; d++)
            for (int f = 0; f < 2; f++) {
                groups_[c][d][f].ndim = d + 2;
                groups_[c][d][f].f32 = f;
                groups_[c][d][f].compact = c == 1;
            }
    InnerScal dead{};
    dead.stop = 1;
    if (cudaMallocAsync((void **)&dead_, sizeof(InnerScal), st_) == cudaSuccess)
        cudaMemcpyAsync(dead_, &dead, sizeof(InnerScal), cudaMemcpyHostToDevice, st_);
    cudaStreamSynchronize(st_);
}

void BatchEngine::retire(Group &g, BatchItem *it) {
    for (size_t k = 0; k < g.planned.size(); k++)
        if (g.planned[k] == it) {
            if (g.compact)
                retire_compact_kernel<<<1, 1, 0, st_>>>(g.d_cinst, (int)k, dead_);
            else
                retire_kernel<<<1, 1, 0, st_>>>(g.d_inst, (int)k, dead_);
            g.planned[k] = nullptr;
        }
}

BatchEngine::~BatchEngine() {
    for (int c = 0; c < 2; c++)
        for (int d = 0; d < 2; d++)
            for (int f = 0; f < 2; f++) {
                Group &g = groups_[c][d][f];
                if (g.exec) cudaGraphExecDestroy(g.exec);
                dfree(g.d_inst, st_);
                dfree(g.d_segs, st_);
                dfree(g.d_cta, st_);
                dfree(g.d_part, st_);
                dfree(g.d_cinst, st_);
                dfree(g.d_csegs, st_);
            }
    dfree((void *)d_sptr_, st_);
    dfree(d_stop_, st_);
    dfree(d_iter_, st_);
    dfree(dead_, st_);
    cudaStreamSynchronize(st_);
}

net_status BatchEngine::outer_pass(BatchItem *it, int apply_corr, int corr_f32) {
    if (it->compact) return outer_pass_compact(it->net, it->f32, apply_corr, it->opts, st_);
    OuterArgs oa = outer_args(it->net, it->f32, apply_corr, corr_f32, it->opts);
    CKB(launch_outer(oa, st_));
    return NET_OK;
}

void BatchEngine::finish(BatchItem *it, net_status st) {
    net_t *n = it->net;
    const Geom &G = n->g;
    const OuterScal &os = n->hsc->os;
    const double dP = G.p_in - G.p_out;
    net_result &r = it->res;
    memset(&r, 0, sizeof(r));
    r.q_in = os.qin;
    r.q_out = os.qout;
    r.g_eff = os.qin / dP;
    double S = 1.0;
    const long long ext[3] = {G.nx, G.ny, G.nz};
    for (int a = 0; a < G.ndim; a++)
        if (a != G.f) S *= (double)ext[a];
    r.k_eff = r.g_eff * (double)(G.nf - 1) / S;
    r.rel_residual = it->rel;
    r.max_imbalance = os.rmax;
    r.energy_g = os.energy / (dP * dP);
    r.n_active = n->n_active;
    r.outer_iters = it->outer;
    r.inner_iters = it->inner_total;
    r.fp64_fallback = it->fallback;
    r.g_eff_err = geff_err(n);
    r.n_solved = n->n_solved;
    r.ms = (float)std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - it->t_start).count();
    r.status = st;
    if (st != NET_OK) it->err = last_error();
    n->last = r;
    n->solved = true;
    // no more sweeps for this network, whatever plan it is still part of
    set_stop_kernel<<<1, 1, 0, st_>>>(&n->dsc->in[0], 1);
    set_stop_kernel<<<1, 1, 0, st_>>>(&n->dsc->in[1], 1);
    for (int c = 0; c < 2; c++)
        for (int d = 0; d < 2; d++)
            for (int f = 0; f < 2; f++) retire(groups_[c][d][f], it);
    it->done = true;
    done_.push_back(it);
}

net_status BatchEngine::add(const std::vector<BatchItem *> &items) {
    std::vector<BatchItem *> ok;
    for (BatchItem *it : items) {
        it->t_start = std::chrono::steady_clock::now();
        it->done = false;
        it->outer = 0;
        it->inner_total = 0;
        it->fallback = 0;
        net_opts o;
        net_opts_default(&o);
        if (it->opts.tol_rel > 0.0) o = it->opts;
        o.x0 = nullptr;
        o.stream = nullptr;
        it->opts = o;
        it->f32 = o.precision == NET_MIXED;
        net_t *n = it->net;
        if (!n || n->device != device_) {
            set_error("batch: network is not on the engine's device");
            it->err = last_error();
            it->res.status = NET_EINVAL;
            it->done = true;
            done_.push_back(it);
            continue;
        }
        // the network's own stream may still hold its set-up work
        CKB(cudaEventRecord(n->ev[3], n->stream));
        CKB(cudaStreamWaitEvent(st_, n->ev[3], 0));
        net_status s = ensure_precision(n, it->f32, st_);
        if (s != NET_OK) return s;
        it->compact = batch_takes_compact(n, it->f32);
        if (it->compact) {
            s = prepare_compact(n, it->f32, st_);
            if (s != NET_OK) return s;
        }
        const void *gr[3] = {n->graw[0], n->graw[1], n->g.ndim == 3 ? n->graw[2] : n->graw[0]};
        CKB(launch_build_system(n->g, gr, n->raw_f32, n->cls, n->dis, n->x, &n->dsc->ss, n->partials, st_));
        s = outer_pass(it, 0, it->f32);
        if (s != NET_OK) return s;
        CKB(cudaMemcpyAsync(&n->hsc->os, &n->dsc->os, sizeof(OuterScal), cudaMemcpyDeviceToHost, st_));
        ok.push_back(it);
    }
    CKB(cudaStreamSynchronize(st_));
    for (BatchItem *it : ok) {
        net_t *n = it->net;
        it->rel = n->bnorm > 0.0 ? std::sqrt(n->hsc->os.rr) / n->bnorm : 0.0;
        it->prog.start(it->rel, geff_err(n));
        if (n->bnorm == 0.0 || outer_dist(n, it->opts, it->rel) <= 1.0) {
            finish(it, NET_OK);
            continue;
        }
        Group &g = group_of(n->g.ndim, it->f32, it->compact);
        g.items.push_back(it);
        g.dirty = true;
        nrun_++;
    }
    return NET_OK;
}

net_status BatchEngine::choose_shape(Group &g, PlanShape *shape) {
    constexpr int kDefaultSeg = 2;
    *shape = PlanShape{};
    shape->seg_per_sm = kDefaultSeg;
    if (tune_forced(g.ndim, g.f32, shape)) return NET_OK;
    long long nodes = 0;
    for (BatchItem *it : g.items) nodes += (long long)it->net->g.px * it->net->g.ny * it->net->g.nz;
    const TuneKey key = tune_key(device_, g.ndim, g.f32, nodes);
    TuneEntry te;
    if (tune_lookup(key, &te)) {
        *shape = te.shape;
        return NET_OK;
    }
    if (tune_enabled() && !g.swept) {
        std::vector<net_t *> nets;
        for (BatchItem *it : g.items) nets.push_back(it->net);
        double bu = 0, du = 0;
        int nc = 0;
        net_status s = autotune_nets(nets, g.f32, kDefaultSeg, st_, shape, &bu, &du, &nc);
        if (s != NET_OK) return s;
        // the timing sweeps advanced the CG state: arm every network again
        // from its (unchanged) pressures, exactly as add() did
        for (BatchItem *it : g.items) {
            s = outer_pass(it, 0, it->f32);
            if (s != NET_OK) return s;
        }
        return NET_OK;
    }
    if (tune_nearest(key, &te)) *shape = te.shape;
    return NET_OK;
}

net_status BatchEngine::rebuild(Group &g, int K) {
    if (g.exec) {
        cudaGraphExecDestroy(g.exec);
        g.exec = nullptr;
    }
    PlanShape shape;
    net_status s0 = choose_shape(g, &shape);
    if (s0 != NET_OK) return s0;
    std::vector<PlanNet> nets;
    for (BatchItem *it : g.items) nets.push_back(PlanNet{it->net->g, true});
    HostPlan hp;
    build_plan(nets, g.ndim, g.f32, nsm_, shape, hp);
    size_t tot_part = 0;
    std::vector<SweepInst> si(g.items.size());
    std::vector<size_t> off(g.items.size());
    for (size_t k = 0; k < g.items.size(); k++) {
        off[k] = tot_part;
        tot_part += (size_t)std::max(1, hp.nseg[k]) * 4;
    }
    CKB(grow(&g.d_inst, &g.cap_inst, si.size(), st_));
    CKB(grow(&g.d_segs, &g.cap_segs, hp.segs.size(), st_));
    size_t cap_cta = 0;
    int *new_cta = nullptr;
    CKB(grow(&new_cta, &cap_cta, hp.cta_begin.size(), st_));
    dfree(g.d_cta, st_);
    g.d_cta = new_cta;
    CKB(grow(&g.d_part, &g.cap_part, tot_part, st_));
    for (size_t k = 0; k < g.items.size(); k++) {
        si[k] = sweep_inst_of(g.items[k]->net, g.f32);
        si[k].part = g.d_part + off[k];
        si[k].nseg = hp.nseg[k];
    }
    CKB(cudaMemcpyAsync(g.d_inst, si.data(), sizeof(SweepInst) * si.size(), cudaMemcpyHostToDevice, st_));
    CKB(cudaMemcpyAsync(g.d_segs, hp.segs.data(), sizeof(SweepSeg) * hp.segs.size(), cudaMemcpyHostToDevice, st_));
    CKB(cudaMemcpyAsync(g.d_cta, hp.cta_begin.data(), sizeof(int) * hp.cta_begin.size(), cudaMemcpyHostToDevice, st_));
    CKB(sweep_prepare(g.ndim, g.f32));
    // capture K sweeps
    cudaStream_t cs;
    CKB(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    for (int i = 0; e == cudaSuccess && i < K; i++)
        e = launch_sweep(g.ndim, g.f32, hp.grid, g.d_inst, g.d_segs, g.d_cta, cs);
    cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return cuda_fail(e, "batch graph");
    // the uploads above must land before the graph's first replay
    CKB(cudaStreamSynchronize(st_));
    g.grid = hp.grid;
    g.K = K;
    g.dirty = false;
    g.planned = g.items;
    g.shape = shape;
    return NET_OK;
}

net_status BatchEngine::rebuild_compact(Group &g, int K) {
    if (g.exec) {
        cudaGraphExecDestroy(g.exec);
        g.exec = nullptr;
    }
    std::vector<CompactInst> ci(g.items.size());
    std::vector<CompactSeg> segs;
    size_t tot_part = 0;
    std::vector<size_t> off(g.items.size());
    for (size_t k = 0; k < g.items.size(); k++) {
        const long long U = compact_args_of(g.items[k]->net, g.f32).n;
        const int ns = (int)std::max(1LL, (U + COMPACT_SEG - 1) / COMPACT_SEG);
        off[k] = tot_part;
        tot_part += (size_t)ns * 4;
        for (int j = 0; j < ns; j++)
            segs.push_back(CompactSeg{(int)k, (int)(U * j / ns), (int)(U * (j + 1) / ns), j});
        ci[k].nseg = ns;
    }
    CKB(grow(&g.d_cinst, &g.cap_cinst, ci.size(), st_));
    CKB(grow(&g.d_csegs, &g.cap_csegs, segs.size(), st_));
    CKB(grow(&g.d_part, &g.cap_part, tot_part, st_));
    for (size_t k = 0; k < g.items.size(); k++) {
        ci[k].a = compact_args_of(g.items[k]->net, g.f32);
        ci[k].part = g.d_part + off[k];
    }
    CKB(cudaMemcpyAsync(g.d_cinst, ci.data(), sizeof(CompactInst) * ci.size(), cudaMemcpyHostToDevice, st_));
    CKB(cudaMemcpyAsync(g.d_csegs, segs.data(), sizeof(CompactSeg) * segs.size(), cudaMemcpyHostToDevice, st_));
    cudaStream_t cs;
    CKB(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    for (int i = 0; e == cudaSuccess && i < K; i++)
        e = launch_compact_batch(g.ndim, g.f32, g.d_cinst, g.d_csegs, (int)segs.size(), cs);
    cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return cuda_fail(e, "batch graph (compacted)");
    CKB(cudaStreamSynchronize(st_));
    g.nseg = (int)segs.size();
    g.K = K;
    g.dirty = false;
    g.planned = g.items;
    return NET_OK;
}

net_status BatchEngine::step(int K) {
    if (nrun_ == 0) return NET_OK;
    const bool tr = trace_on();
    const auto t0 = std::chrono::steady_clock::now();
    if (tr) {
        // running networks and unknowns per group before this step
        for (int c = 0; c < 2; c++)
            for (int d = 0; d < 2; d++)
                for (int f = 0; f < 2; f++) {
                    const Group &g = groups_[c][d][f];
                    if (g.items.empty()) continue;
                    long long u = 0;
                    for (const BatchItem *it : g.items) u += it->net->n_solved;
                    fprintf(stderr, "[trace batch-step %dD %s %s] running %zu unknowns %lld K %d\n", d + 2,
                            f ? "f32" : "f64", c ? "list" : "lattice", g.items.size(), u, K);
                }
    }
    for (int c = 0; c < 2; c++)
        for (int d = 0; d < 2; d++)
            for (int f = 0; f < 2; f++) {
                Group &g = groups_[c][d][f];
                if (g.items.empty()) continue;
                if (g.dirty || g.K != K || !g.exec) {
                    net_status s = g.compact ? rebuild_compact(g, K) : rebuild(g, K);
                    if (s != NET_OK) return s;
                }
                CKB(cudaGraphLaunch(g.exec, st_));
                g.swept = true;
            }
    // one read of every running network's stop flag and iteration count
    std::vector<BatchItem *> run;
    std::vector<const InnerScal *> ptrs;
    for (int c = 0; c < 2; c++)
        for (int d = 0; d < 2; d++)
            for (int f = 0; f < 2; f++)
                for (BatchItem *it : groups_[c][d][f].items) {
                    run.push_back(it);
                    ptrs.push_back(&it->net->dsc->in[it->f32 ? 0 : 1]);
                }
    const size_t n = run.size();
    if (cap_g_ < n) {
        dfree((void *)d_sptr_, st_);
        dfree(d_stop_, st_);
        dfree(d_iter_, st_);
        cap_g_ = n + n / 2 + 16;
        CKB(dalloc(&d_sptr_, sizeof(void *) * cap_g_, st_));
        CKB(dalloc(&d_stop_, sizeof(int) * cap_g_, st_));
        CKB(dalloc(&d_iter_, sizeof(long long) * cap_g_, st_));
    }
    std::vector<int> stop(n);
    std::vector<long long> iters(n);
    CKB(cudaMemcpyAsync((void *)d_sptr_, ptrs.data(), sizeof(void *) * n, cudaMemcpyHostToDevice, st_));
    gather_status_kernel<<<(int)std::min<size_t>((n + 255) / 256, 1024), 256, 0, st_>>>(d_sptr_, (int)n, d_stop_, d_iter_);
    CKB(cudaGetLastError());
    CKB(cudaMemcpyAsync(stop.data(), d_stop_, sizeof(int) * n, cudaMemcpyDeviceToHost, st_));
    CKB(cudaMemcpyAsync(iters.data(), d_iter_, sizeof(long long) * n, cudaMemcpyDeviceToHost, st_));
    CKB(cudaStreamSynchronize(st_));
    if (tr)
        fprintf(stderr, "[trace batch-step] sweeps %.3f ms\n",
                std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count());
    // outer passes of every network whose inner solve stopped
    std::vector<BatchItem *> stopped;
    std::vector<int> stop_code, stop_iter;
    for (size_t i = 0; i < n; i++) {
        if (!stop[i]) continue;
        BatchItem *it = run[i];
        it->inner_total += iters[i];
        if (stop[i] == 5) {
            set_error("batch: a bounded device wait gave up");
            finish(it, NET_ETIMEOUT);
            continue;
        }
        net_status s = outer_pass(it, 1, it->f32);
        if (s != NET_OK) return s;
        CKB(cudaMemcpyAsync(&it->net->hsc->os, &it->net->dsc->os, sizeof(OuterScal), cudaMemcpyDeviceToHost, st_));
        stopped.push_back(it);
        stop_code.push_back(stop[i]);
        stop_iter.push_back((int)iters[i]);
    }
    CKB(cudaStreamSynchronize(st_));
    std::vector<BatchItem *> to_fp64;
    for (size_t j = 0; j < stopped.size(); j++) {
        BatchItem *it = stopped[j];
        net_t *nt = it->net;
        it->outer++;
        it->rel = std::sqrt(nt->hsc->os.rr) / nt->bnorm;
        const double dist = outer_dist(nt, it->opts, it->rel);
        const bool stalled = it->prog.stalled(it->rel, geff_err(nt), stall_limit(it->opts));
        trace_outer(nt, "batch", it->outer, it->f32, stop_code[j], stop_iter[j], it->rel);
        if (dist <= 1.0) {
            finish(it, NET_OK);
        } else if (it->outer >= it->opts.max_outer) {
            set_error("batch: not converged after %d refinement steps", it->outer);
            finish(it, NET_ENOTCONVERGED);
        } else if (it->f32 && stalled) {
            to_fp64.push_back(it);
        }
    }
    for (BatchItem *it : to_fp64) {
        // FP32 passes that stopped making progress: continue in FP64
        net_t *nt = it->net;
        set_stop_kernel<<<1, 1, 0, st_>>>(&nt->dsc->in[0], 1);
        net_status s = ensure_precision(nt, 0, st_);
        if (s != NET_OK) return s;
        Group &g32 = group_of(nt->g.ndim, 1, it->compact);
        g32.items.erase(std::remove(g32.items.begin(), g32.items.end(), it), g32.items.end());
        retire(g32, it);
        g32.dirty = true;
        it->f32 = 0;
        it->fallback = 1;
        it->compact = batch_takes_compact(nt, 0);
        if (it->compact) {
            s = prepare_compact(nt, 0, st_);
            if (s != NET_OK) return s;
        }
        s = outer_pass(it, 0, 0);
        if (s != NET_OK) return s;
        it->prog.start(it->rel, geff_err(nt));
        Group &g64 = group_of(nt->g.ndim, 0, it->compact);
        g64.items.push_back(it);
        g64.dirty = true;
    }
    // drop finished networks and replan the group: a sweep lasts as long as
    // its busiest CTA, and the CTAs that held a finished network's segments
    // would otherwise idle while the rest keep their full share.  A replan
    // (host cut, upload, graph instantiation) costs far less than a step.
    for (int c = 0; c < 2; c++)
        for (int d = 0; d < 2; d++)
            for (int f = 0; f < 2; f++) {
                Group &g = groups_[c][d][f];
                const size_t before = g.items.size();
                g.items.erase(std::remove_if(g.items.begin(), g.items.end(), [](BatchItem *it) { return it->done; }),
                              g.items.end());
                if (before != g.items.size()) g.dirty = true;
                if (g.items.empty()) g.swept = false;
            }
    nrun_ = 0;
    for (int c = 0; c < 2; c++)
        for (int d = 0; d < 2; d++)
            for (int f = 0; f < 2; f++) nrun_ += groups_[c][d][f].items.size();
    return NET_OK;
}

std::vector<BatchItem *> BatchEngine::take_done() {
    std::vector<BatchItem *> v;
    v.swap(done_);
    return v;
}

}  // namespace netsolve

// ---------------------------------------------------------------------------
#define NET_API extern "C" __attribute__((visibility("default")))

using namespace netsolve;

NET_API net_status net_solve_batch(net_t *const *nets, int count, const net_opts *opts,
                                   net_result *res) {
    if (count < 0 || (count > 0 && (!nets || !res))) {
        set_error("net_solve_batch: bad arguments");
        return NET_EINVAL;
    }
    if (count == 0) return NET_OK;
    int dev = 0;
    cudaGetDevice(&dev);
    for (int i = 0; i < count; i++) {
        if (!nets[i] || nets[i]->device != dev) {
            set_error("net_solve_batch: network %d is NULL or on another device", i);
            return NET_EINVAL;
        }
    }
    net_opts o;
    net_opts_default(&o);
    if (opts) o = *opts;
    if (!opts_valid(o)) {
        set_error("net_solve_batch: %s", std::string(last_error()).c_str());
        return NET_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)o.stream;
    bool own = false;
    if (!st) {
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            set_error("net_solve_batch: stream");
            return NET_ECUDA;
        }
        own = true;
    }
    net_status status = NET_OK;
    {
        BatchEngine eng(dev, st);
        std::vector<BatchItem> items(count);
        std::vector<BatchItem *> ptr(count);
        for (int i = 0; i < count; i++) {
            items[i].net = nets[i];
            items[i].opts = o;
            items[i].user = (uint64_t)i;
            ptr[i] = &items[i];
        }
        status = eng.add(ptr);
        const int K = o.check_every > 0 ? o.check_every : 16;
        while (status == NET_OK && eng.running() > 0) status = eng.step(K);
        eng.take_done();
        for (int i = 0; i < count; i++) {
            res[i] = items[i].res;
            if (status == NET_OK && items[i].res.status != NET_OK) status = items[i].res.status;
        }
        if (status != NET_OK && status != NET_ENOTCONVERGED && status != NET_ETIMEOUT && status != NET_EINVAL)
            for (int i = 0; i < count; i++)
                if (!items[i].done) res[i].status = status;
    }
    if (own) cudaStreamDestroy(st);
    return status;
}
