// plan_harness.cu -- prints the sweep plan the library builds for a set of
// networks (host code only; no CUDA call is made, so no GPU is needed).
//
// usage: plan_harness ndim f32 nsm wcap hcap seg_per_sm nx ny nz [nx ny nz ...]
// output: one line "grid P" then one line per segment in CTA order:
//         "cta inst x0 w y0 h m0 m1 slot", then "cap <elements per step>".
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../../paper_1908_03301_gb300/csrc/plan.h"

using namespace netsolve;

int main(int argc, char **argv) {
    if (argc < 10 || (argc - 7) % 3 != 0) {
        fprintf(stderr, "usage: %s ndim f32 nsm wcap hcap seg nx ny nz ...\n", argv[0]);
        return 2;
    }
    const int ndim = atoi(argv[1]), f32 = atoi(argv[2]), nsm = atoi(argv[3]);
    PlanShape shape;
    shape.wcap = atoi(argv[4]);
    shape.hcap = atoi(argv[5]);
    shape.seg_per_sm = atoi(argv[6]);
    if (!plan_shape_valid(ndim, f32, shape)) {
        printf("invalid\n");
        return 0;
    }
    std::vector<PlanNet> nets;
    for (int a = 7; a + 2 < argc; a += 3) {
        Geom g{};
        g.ndim = ndim;
        g.nx = atoi(argv[a]);
        g.ny = atoi(argv[a + 1]);
        g.nz = ndim == 3 ? atoi(argv[a + 2]) : 1;
        g.px = (g.nx + 3) / 4 * 4;
        nets.push_back(PlanNet{g, true});
    }
    HostPlan hp;
    build_plan(nets, ndim, f32, nsm, shape, hp);
    printf("grid %d %d\n", hp.grid, (int)hp.segs.size());
    for (int c = 0; c < hp.grid; c++)
        for (int i = hp.cta_begin[c]; i < hp.cta_begin[c + 1]; i++) {
            const SweepSeg &s = hp.segs[i];
            printf("%d %d %d %d %d %d %d %d %d\n", c, s.inst, s.x0, s.w, s.y0, s.h, s.m0, s.m1, s.slot);
        }
    for (size_t k = 0; k < nets.size(); k++) printf("nseg %zu %d\n", k, hp.nseg[k]);
    printf("cap %d wmax %d\n", sweep_consumers() * sweep_vt(f32), sweep_max_width(ndim, f32));
    return 0;
}
