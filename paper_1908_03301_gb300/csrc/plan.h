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

// Tile shape of a sweep plan: the widest column block (elements, a multiple
// of 4; 0 = the kernel's maximum), the tallest 3D row band (0 = as many rows
// as the consumer threads cover at that width, at most 32) and the number of
// segments per SM the march ranges are cut into.
struct PlanShape {
    int wcap = 0;
    int hcap = 0;
    int seg_per_sm = 1;
};

struct HostPlan {
    std::vector<SweepSeg> segs;   // ordered by CTA
    std::vector<int> cta_begin;   // grid + 1 offsets into segs
    std::vector<int> nseg;        // segments per network
    int grid = 0;
};

// Segments of roughly total/(nsm*seg_per_sm) nodes, dealt longest-first.
void build_plan(const std::vector<PlanNet> &nets, int ndim, int f32, int nsm, const PlanShape &shape,
                HostPlan &out);
// Whether a (width, rows) patch fits the sweep kernel's stage layout.
bool plan_shape_valid(int ndim, int f32, const PlanShape &shape);

}  // namespace netsolve
