// plan.cu -- host-side work planning for the sweep kernel.
//
// Every network is cut into bands (column block, and in 3D row band) that
// are marched along the last axis.  The bands of all networks, in order, form
// one sequence of march steps; it is cut into equal-cost contiguous pieces,
// one (or seg_per_sm) per CTA, splitting a band's march range where a piece
// ends.  A sweep launch waits for its slowest CTA, so equal pieces are what
// matters: dealing whole, equal segments to CTAs leaves a remainder (e.g. 156
// segments on 152 SMs run in two rounds).  Each segment costs two extra
// pipeline-fill steps, which the cut counts.
#include <algorithm>
#include <cmath>
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

bool plan_shape_valid(int ndim, int f32, const PlanShape &shape) {
    const int wmax = sweep_max_width(ndim, f32);
    const int cap = sweep_consumers() * sweep_vt(f32);
    if (shape.seg_per_sm < 1 || shape.seg_per_sm > 64) return false;
    if (shape.wcap != 0 && (shape.wcap < 4 || shape.wcap % 4 || shape.wcap > wmax)) return false;
    if (shape.hcap < 0 || shape.hcap > 32) return false;
    if (ndim == 3 && shape.hcap > 0) {
        const int w = shape.wcap > 0 ? shape.wcap : wmax;
        if ((long long)w * shape.hcap > cap) return false;
        if (!sweep_patch_fits(f32, w, shape.hcap)) return false;
    }
    return true;
}

namespace {

// A band: one column block (and in 3D one row band) of one network, marched
// along the last axis; each march step touches w*h nodes.  `step` is the
// modelled cost of one march step in node-equivalents.
struct Band {
    int inst, x0, w, y0, h, nm;
    double step;
};

// A march step costs its nodes plus a fixed amount per bulk copy it issues
// (measured on GB300: about 0.1 us of the copy engine's time per copy, the
// time about 100 nodes' worth of bytes take at an SM's share of HBM
// bandwidth).  2D steps stage `rows` rows together: 6 copies per stage over
// whole rows, 6 per row otherwise; 3D steps over whole padded rows copy each
// array once (7 copies), narrower 3D patches copy row by row.  A 2D row also
// costs the consumer warps a fixed time whatever its width (they march the
// rows one by one, two columns per thread): batches of equal-sized square
// networks, 2.1 M nodes in all, swept in 86.5 / 46.2 / 33.7 / 25.2 / 21.0 us
// per iteration at sides 64 / 128 / 256 / 512 / 1024, i.e. about 7.9 ps per
// node plus 2.1 ns per row -- 270 nodes' worth per row, which the copies of
// narrow whole-row stages (several rows each) do not reach.
constexpr double kCopyCost = 100.0;
constexpr double kRowCost2D = 270.0;
inline double step_cost(int ndim, int w, int h, bool full_rows, int rows) {
    if (ndim == 2) {
        const double copies = full_rows ? 6.0 / rows : 6.0;
        return (double)w * h + std::max(kCopyCost * copies, kRowCost2D);
    }
    const double copies = full_rows ? 7.0 : 3.0 * (h + 2) + 4.0 * h + 1.0;
    return (double)w * h + kCopyCost * copies;
}

// Cost of a segment of L march steps of band b: its steps plus the two
// pipeline-fill steps that load the planes on either side.
inline double seg_cost(const Band &b, long long L) { return b.step * (double)(L + 2); }

// Greedy cut of the band sequence into pieces of cost <= T (a segment is
// never shorter than `min_steps` unless its band is).  Returns the number of
// pieces; fills `out` (piece index per segment) when non-null.
int greedy_cut(const std::vector<Band> &bands, double T, int min_steps, std::vector<SweepSeg> *segs,
               std::vector<int> *piece) {
    int np = 0;
    double load = 0.0;
    bool open = false;
    for (const Band &b : bands) {
        int m = 0;
        while (m < b.nm) {
            const int rem = b.nm - m;
            long long fit = (long long)((T - load) / b.step) - 2;
            int take;
            if (fit >= rem) {
                take = rem;
            } else if (fit >= min_steps || (!open && fit >= 1)) {
                take = (int)fit;
                if (rem - take < min_steps) take = std::max(1, rem - min_steps);  // no stub after it
            } else if (open) {
                np++;  // close the current piece, retry in a fresh one
                load = 0.0;
                open = false;
                continue;
            } else {
                take = std::min(rem, min_steps);  // a piece must make progress
            }
            if (segs) {
                SweepSeg sg;
                sg.inst = b.inst;
                sg.x0 = b.x0;
                sg.w = b.w;
                sg.y0 = b.y0;
                sg.h = b.h;
                sg.m0 = m;
                sg.m1 = m + take;
                sg.slot = 0;
                segs->push_back(sg);
                piece->push_back(np);
            }
            load += seg_cost(b, take);
            open = true;
            m += take;
            if (load >= T * 0.999) {
                np++;
                load = 0.0;
                open = false;
            }
        }
    }
    return np + (open ? 1 : 0);
}

}  // namespace

void build_plan(const std::vector<PlanNet> &nets, int ndim, int f32, int nsm, const PlanShape &shape,
                HostPlan &out) {
    out.segs.clear();
    out.nseg.assign(nets.size(), 0);
    const int wmax = shape.wcap > 0 ? std::min(shape.wcap, sweep_max_width(ndim, f32))
                                    : sweep_max_width(ndim, f32);
    const int hlim = shape.hcap > 0 ? shape.hcap : 32;
    const int cap = sweep_consumers() * sweep_vt(f32);  // elements per step
    const int grid = std::max(1, nsm);
    const int P = grid * std::max(1, shape.seg_per_sm);  // pieces
    // bands in network order
    std::vector<Band> bands;
    double total = 0.0, biggest = 0.0;
    for (size_t k = 0; k < nets.size(); k++) {
        const PlanNet &pn = nets[k];
        if (!pn.active) continue;
        const Geom &g = pn.g;
        const int kb = (g.px + wmax - 1) / wmax;
        const std::vector<int> ws = split4(g.px, kb);
        int x0 = 0;
        for (int bx = 0; bx < kb; bx++) {
            const int w = ws[bx];
            std::vector<int> hs{1}, y0s{0};
            int nm = g.ny;
            if (ndim == 3) {
                const int hmax = std::max(1, std::min({hlim, cap / std::max(w, 1), g.ny}));
                const int yb = (g.ny + hmax - 1) / hmax;
                hs = split(g.ny, yb);
                y0s.assign(yb, 0);
                for (int j = 1; j < yb; j++) y0s[j] = y0s[j - 1] + hs[j - 1];
                nm = g.nz;
            }
            for (size_t j = 0; j < hs.size(); j++) {
                const bool full_rows = kb == 1;
                const int rows = sweep_rows_per_stage(ndim, f32, w, g.px, x0);
                Band b{(int)k, x0, w, y0s[j], hs[j], nm, step_cost(ndim, w, hs[j], full_rows, rows)};
                bands.push_back(b);
                total += seg_cost(b, nm);
                biggest = std::max(biggest, b.step * 4.0);
            }
            x0 += w;
        }
    }
    // smallest bottleneck cost T with at most P pieces (binary search on T)
    const int min_steps = 4;
    double lo = std::max(total / P, biggest), hi = std::max(total, lo) * 1.01 + 1.0;
    for (int it = 0; it < 40 && hi - lo > 1e-4 * lo; it++) {
        const double mid = 0.5 * (lo + hi);
        if (greedy_cut(bands, mid, min_steps, nullptr, nullptr) <= P) hi = mid;
        else lo = mid;
    }
    std::vector<SweepSeg> all;
    std::vector<int> piece;
    greedy_cut(bands, hi, min_steps, &all, &piece);
    // slots: order of each network's segments
    for (SweepSeg &sg : all) sg.slot = out.nseg[sg.inst]++;
    // piece p -> CTA p % grid, pieces in order inside a CTA
    std::vector<std::vector<int>> lists(grid);
    for (size_t i = 0; i < all.size(); i++) lists[std::min(piece[i], P - 1) % grid].push_back((int)i);
    out.cta_begin.assign(grid + 1, 0);
    for (int c = 0; c < grid; c++) {
        out.cta_begin[c + 1] = out.cta_begin[c] + (int)lists[c].size();
        for (int i : lists[c]) out.segs.push_back(all[i]);
    }
    out.grid = grid;
}

}  // namespace netsolve
