// batch.h -- many networks solved together (internal).
//
// The engine keeps a set of networks whose refinement loops are in flight.
// Networks are grouped by (path, dimension, inner precision).  On the lattice
// path each group has one sweep plan (all its running networks' segments
// dealt over the SMs) and a CUDA graph of K sweep launches; on the compacted
// path (networks whose unknowns are a small part of the lattice, and periodic
// networks) a group's networks are cut into list segments and its graph holds
// K pairs of phase launches over all of them.  step() replays every group's graph once,
// gathers all stop flags with one small kernel and one read, and runs the
// FP64 outer pass of every network whose inner solve stopped; those
// networks then continue, switch to FP64, or finish.  Finished networks
// leave at once, so the others' sweeps get cheaper.
#pragma once
#include <chrono>
#include <cstdint>
#include <string>
#include <vector>

#include "plan.h"
#include "runtime_internal.h"

namespace netsolve {

struct BatchItem {
    net_t *net = nullptr;
    net_opts opts{};
    int f32 = 1;             // inner precision in use
    bool compact = false;    // solved on its list of unknowns
    int outer = 0;
    long long inner_total = 0;
    double rel = 0.0;
    Progress prog;           // FP32 progress watch (switch to FP64)
    int fallback = 0;
    bool done = false;
    net_result res{};
    std::string err;         // message of a non-OK finish
    uint64_t user = 0;       // caller's tag (queue ticket)
    std::chrono::steady_clock::time_point t_start;
};

class BatchEngine {
public:
    BatchEngine(int device, cudaStream_t stream);
    ~BatchEngine();
    // Start the refinement loops of these networks (set-up launches for all,
    // one synchronisation).  Items that need no iteration finish here.
    net_status add(const std::vector<BatchItem *> &items);
    // K sweeps for every running network, then the outer passes of those
    // whose inner solve stopped.
    net_status step(int K);
    // Finished items since the last call.
    std::vector<BatchItem *> take_done();
    size_t running() const { return nrun_; }

private:
    struct Group {
        int ndim = 2, f32 = 1;
        bool compact = false;              // the compacted path
        CompactInst *d_cinst = nullptr;    // compacted path: networks, segments
        CompactSeg *d_csegs = nullptr;
        size_t cap_cinst = 0, cap_csegs = 0;
        int nseg = 0;
        std::vector<BatchItem *> items;
        bool dirty = true;
        SweepInst *d_inst = nullptr;
        SweepSeg *d_segs = nullptr;
        int *d_cta = nullptr;
        double *d_part = nullptr;
        size_t cap_inst = 0, cap_segs = 0, cap_part = 0;
        int grid = 0, K = 0;
        cudaGraphExec_t exec = nullptr;
        std::vector<BatchItem *> planned;  // item order of d_inst
        bool swept = false;                // a sweep ran since the group was last empty
        PlanShape shape;                   // tile shape of the current plan
    };
    // A network leaving a group (finished or moved) must not be read by that
    // group's current plan again: its record is pointed at dead_ (stop = 1),
    // so the sweep skips it even if its memory is released before the next
    // replan.
    void retire(Group &g, BatchItem *it);
    net_status rebuild(Group &g, int K);
    net_status rebuild_compact(Group &g, int K);
    // Tile shape for the group's next plan: the tuned entry of its key; else,
    // while no sweep has run on the group (its state is freshly armed), tune
    // now and re-arm; else the nearest tuned size class; else the default.
    net_status choose_shape(Group &g, PlanShape *shape);
    net_status outer_pass(BatchItem *it, int apply_corr, int corr_f32);
    void finish(BatchItem *it, net_status st);
    Group &group_of(int ndim, int f32, bool compact) { return groups_[compact ? 1 : 0][ndim - 2][f32 ? 1 : 0]; }

    int device_;
    int nsm_;
    cudaStream_t st_;
    Group groups_[2][2][2];  // [compacted path][dimension - 2][FP32 inner]
    size_t nrun_ = 0;
    std::vector<BatchItem *> done_;
    // stop-flag gather
    const InnerScal **d_sptr_ = nullptr;
    int *d_stop_ = nullptr;
    long long *d_iter_ = nullptr;
    size_t cap_g_ = 0;
    InnerScal *dead_ = nullptr;  // always-stopped scalars
};

}  // namespace netsolve
