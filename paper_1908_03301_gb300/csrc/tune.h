// tune.h -- autotuner of the sweep kernel's tile shape (internal).
//
// The sweep kernel's speed depends on how networks are cut into segments:
// the column-block width (wide blocks read fewer halo columns, narrow ones
// give more segments to balance), the 3D row-band height (taller bands re-read
// fewer halo rows but cover fewer columns per march step) and how many
// segments each SM gets.  The best shape depends on the GPU, the dimension,
// the precision and the size of the set being swept, so it is measured: each
// candidate plan runs a few CUDA-graph replays of sweeps on the networks
// themselves, timed with events, and the fastest is kept in a table keyed by
// (device, dimension, inner precision, size class).  Later plans of the same
// key reuse it, so solves within one process stay bit-for-bit repeatable.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "plan.h"

namespace netsolve {

struct TuneKey {
    int device = 0;
    int ndim = 2;
    int f32 = 1;
    int size_class = 0;  // floor(log2(swept lattice nodes))
    bool operator<(const TuneKey &o) const;
};

struct TuneEntry {
    PlanShape shape;
    double us_per_sweep = 0.0;
    int candidates = 0;
};

// The key of a set of networks of one dimension and precision.
TuneKey tune_key(int device, int ndim, int f32, long long lattice_nodes);
// Candidate shapes for a dimension and precision (the default first).
std::vector<PlanShape> tune_candidates(int ndim, int f32, int default_seg_per_sm);
// Exact entry, if the key was tuned.
bool tune_lookup(const TuneKey &k, TuneEntry *out);
// Entry of the nearest size class of the same device/dimension/precision.
bool tune_nearest(const TuneKey &k, TuneEntry *out);
void tune_store(const TuneKey &k, const TuneEntry &e);
// NETSOLVE_AUTOTUNE=0 turns automatic tuning off (explicit net_autotune
// calls still tune).
bool tune_enabled();
// NETSOLVE_SWEEP_SHAPE="wcap,hcap,seg_per_sm" forces one shape for every plan
// (diagnostics and tests); true with *s set when it is given and valid.
bool tune_forced(int ndim, int f32, PlanShape *s);
size_t tune_table_size();
void tune_clear();

// Time `replays` replays of a graph of `K` sweeps over the plan built with
// `shape` for these sweep records (after one untimed replay).  Returns the
// microseconds per sweep, or a negative value on a CUDA error.  The records'
// CG state advances; callers re-arm it afterwards.
double tune_time_shape(const std::vector<PlanNet> &nets, const std::vector<SweepInst> &insts,
                       int ndim, int f32, int nsm, const PlanShape &shape, int K, int replays,
                       cudaStream_t st);

}  // namespace netsolve
