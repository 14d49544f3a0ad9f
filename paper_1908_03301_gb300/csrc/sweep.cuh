// sweep.cuh -- work description of the persistent CG sweep kernel.
//
// A sweep is one CG iteration (Sec. IV, fused as in kernels_cg.cu) for every
// network of a set whose inner solve is still running.  Each network is cut
// into segments; a segment is a block of columns [x0, x0+w), for 3D a band of
// rows [y0, y0+h), and a range [m0, m1) along the march axis (y in 2D, z in
// 3D).  Every CTA walks the segments of its list in order, marching through
// each one; a network's last segment to finish reduces the network's sums and
// sets its next step lengths, so networks of any size and count progress
// independently (per-network convergence masks).
#pragma once
#include "common.cuh"

namespace netsolve {

struct SweepInst {
    Geom g;
    const void *gs[3];  // scaled bonds, inner precision
    void *y;
    void *r[2], *p[2], *q[2];
    InnerScal *s;       // this network's CG scalars (s->counter: segment arrivals)
    double *part;       // 4 partial sums per segment, in segment-slot order
    int nseg;           // segments of this network in the current plan
};

struct SweepSeg {
    int inst;
    int x0, w;   // column block
    int y0, h;   // 3D row band (2D: 0, 1)
    int m0, m1;  // march range
    int slot;    // partial-sum slot within the network
};

}  // namespace netsolve
