// plan.h -- host-side planning of the sweep kernel's work (internal).
#pragma once
#include <vector>

#include "kernels.h"
#include "sweep.cuh"

namespace netsolve {

struct PlanNet {
    Geom g;
    bool active;
};

struct HostPlan {
    std::vector<SweepSeg> segs;   // ordered by CTA
    std::vector<int> cta_begin;   // grid + 1 offsets into segs
    std::vector<int> nseg;        // segments per network
    int grid = 0;
};

// Segments of roughly total/(nsm*seg_per_sm) nodes, dealt longest-first.
void build_plan(const std::vector<PlanNet> &nets, int ndim, int f32, int nsm, int seg_per_sm,
                HostPlan &out);

}  // namespace netsolve
