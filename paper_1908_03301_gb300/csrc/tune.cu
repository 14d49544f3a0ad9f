// tune.cu -- autotuner of the sweep kernel's tile shape.  See tune.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "kernels.h"
#include "runtime_internal.h"
#include "tune.h"

namespace netsolve {

bool TuneKey::operator<(const TuneKey &o) const {
    return std::tie(device, ndim, f32, size_class) < std::tie(o.device, o.ndim, o.f32, o.size_class);
}

namespace {
std::mutex g_mu;
std::map<TuneKey, TuneEntry> g_table;
}  // namespace

TuneKey tune_key(int device, int ndim, int f32, long long lattice_nodes) {
    TuneKey k;
    k.device = device;
    k.ndim = ndim;
    k.f32 = f32 ? 1 : 0;
    int c = 0;
    while (c < 62 && (2LL << c) <= lattice_nodes) c++;
    k.size_class = c;
    return k;
}

std::vector<PlanShape> tune_candidates(int ndim, int f32, int default_seg_per_sm) {
    std::vector<PlanShape> out;
    PlanShape def;
    def.seg_per_sm = default_seg_per_sm;
    out.push_back(def);
    const int wmax = sweep_max_width(ndim, f32);
    const int cap = sweep_consumers() * sweep_vt(f32);
    for (int seg : {1, 2, 4}) {
        for (int div : {1, 2, 4}) {
            PlanShape s;
            s.wcap = wmax / div;
            s.hcap = ndim == 3 ? std::min(32, cap / s.wcap) : 0;
            s.seg_per_sm = seg;
            if (s.wcap < 4 || !plan_shape_valid(ndim, f32, s)) continue;
            // skip the default's twin (wcap = wmax, hcap = cap / wmax)
            if (div == 1 && seg == default_seg_per_sm) continue;
            out.push_back(s);
        }
    }
    return out;
}

bool tune_lookup(const TuneKey &k, TuneEntry *out) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_table.find(k);
    if (it == g_table.end()) return false;
    *out = it->second;
    return true;
}

bool tune_nearest(const TuneKey &k, TuneEntry *out) {
    std::lock_guard<std::mutex> lk(g_mu);
    int best = 1 << 30;
    for (const auto &kv : g_table) {
        const TuneKey &t = kv.first;
        if (t.device != k.device || t.ndim != k.ndim || t.f32 != k.f32) continue;
        const int d = std::abs(t.size_class - k.size_class);
        if (d < best) {
            best = d;
            *out = kv.second;
        }
    }
    return best != (1 << 30);
}

void tune_store(const TuneKey &k, const TuneEntry &e) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_table[k] = e;
}

bool tune_enabled() {
    const char *e = getenv("NETSOLVE_AUTOTUNE");
    return !(e && strcmp(e, "0") == 0);
}

bool tune_forced(int ndim, int f32, PlanShape *s) {
    const char *e = getenv("NETSOLVE_SWEEP_SHAPE");
    if (!e || !*e) return false;
    PlanShape t;
    if (sscanf(e, "%d,%d,%d", &t.wcap, &t.hcap, &t.seg_per_sm) != 3) return false;
    if (!plan_shape_valid(ndim, f32, t)) return false;
    *s = t;
    return true;
}

size_t tune_table_size() {
    std::lock_guard<std::mutex> lk(g_mu);
    return g_table.size();
}

void tune_clear() {
    std::lock_guard<std::mutex> lk(g_mu);
    g_table.clear();
}

double tune_time_shape(const std::vector<PlanNet> &nets, const std::vector<SweepInst> &insts_in,
                       int ndim, int f32, int nsm, const PlanShape &shape, int K, int replays,
                       cudaStream_t st) {
    HostPlan hp;
    build_plan(nets, ndim, f32, nsm, shape, hp);
    std::vector<SweepInst> insts = insts_in;
    size_t tot_part = 0;
    std::vector<size_t> off(insts.size());
    for (size_t k = 0; k < insts.size(); k++) {
        off[k] = tot_part;
        tot_part += (size_t)std::max(1, hp.nseg[k]) * 4;
    }
    SweepInst *d_inst = nullptr;
    SweepSeg *d_segs = nullptr;
    int *d_cta = nullptr;
    double *d_part = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double us = -1.0;
    cudaError_t e = dalloc(&d_inst, sizeof(SweepInst) * std::max<size_t>(1, insts.size()), st);
    if (e == cudaSuccess) e = dalloc(&d_segs, sizeof(SweepSeg) * std::max<size_t>(1, hp.segs.size()), st);
    if (e == cudaSuccess) e = dalloc(&d_cta, sizeof(int) * hp.cta_begin.size(), st);
    if (e == cudaSuccess) e = dalloc(&d_part, sizeof(double) * std::max<size_t>(1, tot_part), st);
    if (e == cudaSuccess) {
        for (size_t k = 0; k < insts.size(); k++) {
            insts[k].part = d_part + off[k];
            insts[k].nseg = hp.nseg[k];
        }
        e = cudaMemcpyAsync(d_inst, insts.data(), sizeof(SweepInst) * insts.size(), cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_segs, hp.segs.data(), sizeof(SweepSeg) * hp.segs.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_cta, hp.cta_begin.data(), sizeof(int) * hp.cta_begin.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = sweep_prepare(ndim, f32);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) {
        cudaStream_t cs;
        e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e == cudaSuccess) {
            cudaGraph_t graph = nullptr;
            e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            for (int i = 0; e == cudaSuccess && i < K; i++)
                e = launch_sweep(ndim, f32, hp.grid, d_inst, d_segs, d_cta, cs);
            cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
            if (e == cudaSuccess) e = e2;
            if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            cudaStreamDestroy(cs);
        }
    }
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, st);  // warm: caches, clocks
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    for (int i = 0; e == cudaSuccess && i < replays; i++) e = cudaGraphLaunch(exec, st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) us = 1e3 * (double)ms / ((double)K * replays);
    if (exec) cudaGraphExecDestroy(exec);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dfree(d_inst, st);
    dfree(d_segs, st);
    dfree(d_cta, st);
    dfree(d_part, st);
    cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cuda_fail(e, "autotune");
        return -1.0;
    }
    return us;
}

}  // namespace netsolve
