// plan.cu -- host-side work planning for the sweep kernel.
//
// Cuts each network into segments (column block x row band x march range,
// see sweep.cuh) of roughly equal size and deals them to the CTAs (one per
// SM) longest-first onto the least-loaded CTA, so every SM streams about the
// same number of bytes per sweep.
#include <algorithm>
#include <cmath>
#include <queue>
#include <vector>

#include "plan.h"

namespace netsolve {

static std::vector<int> split4(int n, int parts) {
    // widths, multiples of 4, summing to n (n is a multiple of 4)
    std::vector<int> w(parts);
    const long long q = n / 4;
    for (int i = 0; i < parts; i++) w[i] = 4 * (int)((q * (i + 1)) / parts - (q * i) / parts);
    return w;
}

static std::vector<int> split(int n, int parts) {
    std::vector<int> w(parts);
    for (int i = 0; i < parts; i++) w[i] = (int)(((long long)n * (i + 1)) / parts - ((long long)n * i) / parts);
    return w;
}

void build_plan(const std::vector<PlanNet> &nets, int ndim, int f32, int nsm, int seg_per_sm,
                HostPlan &out) {
    out.segs.clear();
    out.nseg.assign(nets.size(), 0);
    const int wmax = sweep_max_width(ndim, f32);
    const int cap = sweep_consumers() * sweep_vt(f32);  // elements per step
    long long tot = 0;
    for (const PlanNet &pn : nets)
        if (pn.active) tot += (long long)pn.g.px * pn.g.ny * pn.g.nz;
    const double target = std::max(1.0, (double)tot / ((double)nsm * std::max(1, seg_per_sm)));
    std::vector<SweepSeg> all;
    std::vector<double> cost;
    for (size_t k = 0; k < nets.size(); k++) {
        const PlanNet &pn = nets[k];
        if (!pn.active) continue;
        const Geom &g = pn.g;
        const int kb = (g.px + wmax - 1) / wmax;
        const std::vector<int> ws = split4(g.px, kb);
        int x0 = 0;
        int slot = 0;
        for (int bx = 0; bx < kb; bx++) {
            const int w = ws[bx];
            std::vector<int> hs{1};
            std::vector<int> y0s{0};
            int nm = g.ny;
            if (ndim == 3) {
                const int hmax = std::max(1, std::min({32, cap / std::max(w, 1), g.ny}));
                const int yb = (g.ny + hmax - 1) / hmax;
                hs = split(g.ny, yb);
                y0s.assign(yb, 0);
                for (int j = 1; j < yb; j++) y0s[j] = y0s[j - 1] + hs[j - 1];
                nm = g.nz;
            }
            for (size_t j = 0; j < hs.size(); j++) {
                const double nodes = (double)w * hs[j] * nm;
                int R = (int)std::lround(nodes / target);
                R = std::max(1, std::min(R, std::max(1, nm / 4)));
                const std::vector<int> ms = split(nm, R);
                int m0 = 0;
                for (int rI = 0; rI < R; rI++) {
                    SweepSeg sg;
                    sg.inst = (int)k;
                    sg.x0 = x0;
                    sg.w = w;
                    sg.y0 = y0s[j];
                    sg.h = hs[j];
                    sg.m0 = m0;
                    sg.m1 = m0 + ms[rI];
                    sg.slot = slot++;
                    m0 = sg.m1;
                    all.push_back(sg);
                    cost.push_back((double)w * hs[j] * (ms[rI] + 2) + 2.0 * w * 2 * (ndim == 3 ? ms[rI] : 0));
                }
            }
            x0 += w;
        }
        out.nseg[k] = slot;
    }
    // longest first onto the least-loaded CTA
    const int grid = std::max(1, nsm);
    std::vector<int> order(all.size());
    for (size_t i = 0; i < order.size(); i++) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    using Item = std::pair<double, int>;
    std::priority_queue<Item, std::vector<Item>, std::greater<Item>> heap;
    for (int c = 0; c < grid; c++) heap.push({0.0, c});
    std::vector<std::vector<int>> lists(grid);
    for (int i : order) {
        Item it = heap.top();
        heap.pop();
        lists[it.second].push_back(i);
        it.first += cost[i];
        heap.push(it);
    }
    out.cta_begin.assign(grid + 1, 0);
    for (int c = 0; c < grid; c++) {
        std::sort(lists[c].begin(), lists[c].end());  // network-major order inside a CTA
        out.cta_begin[c + 1] = out.cta_begin[c] + (int)lists[c].size();
        for (int i : lists[c]) out.segs.push_back(all[i]);
    }
    out.grid = grid;
}

}  // namespace netsolve
