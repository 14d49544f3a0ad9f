// kernels_cg.cu -- the FP64 side of the iterative refinement (Sec. IV): the
// correction update, the true-residual pass and the arming of the next inner
// CG solve.
//
// The inner CG iteration itself runs in cg_persist.cu (2D, FP32, one
// cooperative launch per inner solve), sweep.cu (one launch per iteration
// over a planned list of segments) and cg_compact.cu (listed unknowns).  All
// three apply Jacobi preconditioning as the symmetric scaling
// A = D^-1/2 G D^-1/2 (unit diagonal), so preconditioned CG on G becomes
// plain CG on A and the iteration reads no diagonal, and all three compute one
// iteration in one pass over the data:
//   1. finish iteration k-1 from its scalars alpha, beta:
//        r_k = r_{k-1} - alpha q_{k-1},  p_k = r_k + beta p_{k-1},
//        y_k = y_{k-1} + alpha p_{k-1};
//   2. q_k = A p_k (5- or 7-point stencil on the bond planes) and the four
//      sums <p,q>, <r,q>, <q,q>, <r,r>;
//   3. one grid-wide reduction, then
//        alpha_k = <r,r> / <p,q>,
//        beta_k  = <r_{k+1}, r_{k+1}> / <r,r>   with
//        <r_{k+1}, r_{k+1}> = <r,r> - 2 alpha_k <r,q> + alpha_k^2 <q,q>,
//      the expansion of ||r_k - alpha_k q_k||^2.
// The paper's three kernels per iteration with a host-side final sum
// (Sec. IV) become one pass with an on-device reduction.
//
// Outer loop (FP64, this file).  correct_kernel applies the previous
// correction x += D^-1/2 y; outer_kernel then recomputes the true residual
// r = b - G x = sum_j g_ij (x_j - x_i) at interior nodes with the raw bonds,
// writes the scaled residual D^-1/2 r as the next inner right-hand side, and
// reduces ||r||^2, max |r|, the face flows Q_in / Q_out (Eq. 4) and the
// dissipated power.  Its last CTA arms the next inner solve.
#include <cfloat>
#include <cmath>

#include "kernels.h"

namespace netsolve {
namespace {

constexpr int NT = 256;

// ---------------------------------------------------------------------------
// outer FP64 residual pass (scalar per node; runs a few times per solve)
// ---------------------------------------------------------------------------
template <int NDIM>
struct OTile {
    static constexpr int TW = NDIM == 3 ? 32 : 64;
    static constexpr int TH = NDIM == 3 ? 8 : 16;
    static constexpr int TD = NDIM == 3 ? 4 : 1;
    static constexpr int ZP = NDIM == 3 ? TD + 2 : 1;
    static constexpr int ZO = NDIM == 3 ? 1 : 0;
    static constexpr int SW = TW + 2, SH = TH + 2;
    __device__ static int sidx(int zz, int yy, int xx) { return (zz * SH + yy) * SW + xx + 1; }
};

// x += D^-1/2 y on every node (y = 0 and D^-1/2 = 0 off the solved set).
template <typename TI>
__global__ void __launch_bounds__(NT)
correct_kernel(Geom g, const double *__restrict__ dis, double *__restrict__ x,
               TI *__restrict__ yc, const TI *p0, const TI *p1, const InnerScal *is) {
    // A pass that ended with stop 6 still owes the step alpha_k p_k of the
    // recursion (Sec. IV refinement with the recursion kept): fold it in with
    // y and clear y, which the continuing recursion accumulates from zero.
    const bool owe = is->stop == 6;
    const double a = is->alpha;
    const TI *__restrict__ p = (is->iter & 1) ? p1 : p0;
    const long long n = (long long)g.px * g.ny * g.nz;
    for (long long t = blockIdx.x * (long long)NT + threadIdx.x; t < n;
         t += (long long)gridDim.x * NT) {
        const long long i = g.pad + t;
        double d = (double)yc[i];
        if (owe) {
            d = fma(a, (double)p[i], d);
            yc[i] = TI(0);
        }
        x[i] = fma(dis[i], d, x[i]);
    }
}

// Store the outer pass's sums and arm the inner scalars for the next inner
// solve (one thread, after the grid reduction): v = {rr, rmax, rh2, qin,
// qout, energy, ez}.
__device__ __forceinline__ void outer_arm(const Geom &g, const double (&v)[7], OuterScal *os, InnerScal *is,
                                          bool cont, long long it_prev, double rho_prev, int reliable,
                                          double delta2, double tol_floor, double tol_rel, double tol_geff,
                                          double bnorm, long long max_inner, long long stag_window) {
    os->rr = v[0];
    os->rmax = v[1];
    os->rh2 = v[2];
    os->qin = v[3];
    os->qout = v[4];
    os->energy = v[5];
    os->ez = v[6];
    is->alpha = 0.0;
    is->beta = 0.0;
    is->rho0 = v[2];
    is->rho = v[2];
    // Stop when the relative residual is below tol_rel and the first-order
    // error of G_eff is below tol_geff.  By the symmetry of Eq. 3 the
    // sensitivity of Q_in to the nodal residual r is the pressure field
    // normalised to (p_in, p_out) = (1, 0), so Q_in(x) - Q_in(exact) is
    // sum_i (x_i - p_out) r_i / dP to first order.
    // Inner target: reach both in this step if possible, but never ask the
    // inner loop for more than tol_floor (its precision limit).
    const double dP = g.p_in - g.p_out;
    const double rel = bnorm > 0.0 ? sqrt(v[0]) / bnorm : 0.0;
    const double G = v[3] / dP;
    const double gerr = G != 0.0 ? fabs(v[6]) / (dP * dP) / fabs(G) : 0.0;
    const bool done = !(rel > tol_rel) && !(gerr > tol_geff);
    double t = 1.0;
    if (rel > 0.0) t = fmin(t, 0.5 * tol_rel / rel);
    if (gerr > 0.0) t = fmin(t, 0.5 * tol_geff / gerr);
    t = fmin(0.5, fmax(t, tol_floor));
    is->tol2 = t * t;
    is->maxrr = v[2];
    is->delta2 = reliable ? delta2 : 0.0;
    is->reliable = reliable;
    if (cont) {
        // r_k is replaced by the true residual r^ and the step alpha_k was
        // folded into x, so the next iteration takes alpha = 0 and
        // p = r^ + beta p_k with beta = ||r^||^2 / ||r_k||^2.  A true residual
        // above the last recursive one means the recursion has drifted: its
        // direction is dropped (beta = 0), which restarts CG in place.
        is->beta = v[2] < rho_prev ? v[2] / rho_prev : 0.0;
        is->iter = it_prev;
    } else {
        is->beta = 0.0;
        is->iter = 0;
    }
    is->iter0 = is->iter;
    is->best = v[2];
    is->best_iter = is->iter;
    is->max_iter = is->iter + max_inner;
    is->stag_window = stag_window;
    is->err = 0;
    is->counter = 0u;
    // no inner solve when the outer tolerances are met (or nothing to solve)
    is->stop = (v[2] > 0.0 && !done) ? 0 : 1;
}

template <typename GT, typename TI, int NDIM>
__global__ void __launch_bounds__(NT)
outer_kernel(Geom g, const GT *__restrict__ g0, const GT *__restrict__ g1,
             const GT *__restrict__ g2, const double *__restrict__ dis, const double *__restrict__ x,
             TI *r_out0, TI *r_out1, OuterScal *os,
             InnerScal *is, int reliable, int allow_cont, double delta2, double tol_floor, double tol_rel,
             double tol_geff, double bnorm, long long max_inner, long long stag_window,
             double *partials) {
    using OT = OTile<NDIM>;
    constexpr int TW = OT::TW, TH = OT::TH, TD = OT::TD;
    __shared__ double sx[OT::ZP * OT::SH * OT::SW];
    const int x0 = blockIdx.x * TW, y0 = blockIdx.y * TH, z0 = blockIdx.z * TD;
    const GT *gp[3] = {g0, g1, g2};
    // Continue the recursion when the last pass asked for this refinement
    // (stop 6): the new residual goes where the next iteration reads r
    // (buffer iter & 1).  Otherwise restart: buffer 0, iteration 0.  The
    // scalars are read here, before the last CTA re-arms them.
    const bool cont = allow_cont && is->stop == 6;
    const long long it_prev = is->iter;
    const double rho_prev = is->rho;
    TI *__restrict__ r_out = (cont && (it_prev & 1)) ? r_out1 : r_out0;

    // stage x over the tile and its halo (x is read-only in this kernel; the
    // correction was applied by correct_kernel before it)
    constexpr int CELLS = OT::ZP * OT::SH * OT::SW;
    for (int c = threadIdx.x; c < CELLS; c += NT) {
        const int xx = c % OT::SW - 1, t = c / OT::SW, yy = t % OT::SH - 1, zz = t / OT::SH - OT::ZO;
        const int cx = x0 + xx, cy = y0 + yy, cz = z0 + zz;
        double xv = 0.0;
        if (cx >= 0 && cx < g.px && cy >= 0 && cy < g.ny && cz >= 0 && cz < g.nz)
            xv = x[g.idx(cx, cy, cz)];
        sx[c] = xv;
    }
    __syncthreads();

    double rr = 0.0, rmax = 0.0, rh2 = 0.0, qin = 0.0, qout = 0.0, en = 0.0, ez = 0.0;
    for (int c = threadIdx.x; c < TW * TH * TD; c += NT) {
        const int xx = c % TW, t = c / TW, yy = t % TH, zz = t / TH;
        const int cx = x0 + xx, cy = y0 + yy, cz = z0 + zz;
        if (!(cx < g.px && cy < g.ny && cz < g.nz)) continue;
        const long long i = g.idx(cx, cy, cz);
        const int s0 = OT::sidx(zz + OT::ZO, yy + 1, xx);
        const double xi = sx[s0];
        const int soff[3] = {1, OT::SW, OT::SH * OT::SW};
        double rs = 0.0;
#pragma unroll
        for (int d = 0; d < NDIM; d++) {
            double gmv = (double)gp[d][i - g.stride(d)];
            double xpv = sx[s0 + soff[d]], xmv = sx[s0 - soff[d]];
            if (g.periodic(d)) {
                // across a periodic boundary the neighbour is the opposite
                // layer, outside this tile's halo: read it directly
                const int cd = g.coord(d, cx, cy, cz);
                if (cd + 1 == g.extent(d)) xpv = x[g.up(i, d, cd)];
                if (cd == 0) {
                    const long long jm = g.down(i, d, cd);
                    xmv = x[jm];
                    gmv = (double)gp[d][jm];
                }
            }
            const double gpv = (double)gp[d][i];
            rs += gpv * (xpv - xi) + gmv * (xmv - xi);
            en += gpv * (xi - xpv) * (xi - xpv);
        }
        const int cf = g.coord(g.f, cx, cy, cz);
        const bool inner = cf > 0 && cf < g.nf - 1;
        const double rv = inner ? rs : 0.0;
        const double rh = dis[i] * rv;
        r_out[i] = (TI)rh;
        rr += rv * rv;
        rmax = fmax(rmax, fabs(rv));
        rh2 += rh * rh;
        ez += (xi - g.p_out) * rv;
        if (cf == 1) qin += (double)gp[g.f][i - g.stride(g.f)] * (g.p_in - xi);
        if (cf == g.nf - 2) qout += (double)gp[g.f][i] * (xi - g.p_out);
    }
    double v[7] = {rr, rmax, rh2, qin, qout, en, ez};
    const int ops[7] = {RED_SUM, RED_MAX, RED_SUM, RED_SUM, RED_SUM, RED_SUM, RED_SUM};
    if (!grid_reduce<7, NT>(v, ops, partials, &os->counter)) return;
    if (threadIdx.x != 0) return;
    outer_arm(g, v, os, is, cont, it_prev, rho_prev, reliable, delta2, tol_floor, tol_rel, tol_geff, bnorm,
              max_inner, stag_window);
}

// The same pass for a network solved on its list of unknowns (Eq. 3 residual
// in FP64 at the listed nodes only).  Every other node's residual, flux and
// energy is zero: a dead-end node holds its root's pressure
// (fill_dangling_kernel runs first), a node of a non-spanning cluster shares
// no open bond with the backbone, a face node is fixed.  So the sums run over
// the list: the residual at each unknown, the energy of its +e_d bonds plus,
// next to the inlet, of its bond to the inlet face (the only bond into the
// backbone no unknown counts as its +e_d bond), the fluxes of its face bonds.
// The scaled residual goes straight to the list vector r_list (what the
// lattice pass followed by a gather gives).  Same reduction and arming.
template <typename GT, typename TI, int NDIM>
__global__ void __launch_bounds__(NT)
outer_list_kernel(Geom g, const GT *__restrict__ g0, const GT *__restrict__ g1, const GT *__restrict__ g2,
                  const double *__restrict__ dis, const double *__restrict__ x, const int *__restrict__ cidx,
                  long long U, TI *__restrict__ r_list, OuterScal *os, InnerScal *is, int reliable,
                  int allow_cont, double delta2, double tol_floor, double tol_rel, double tol_geff, double bnorm,
                  long long max_inner, long long stag_window, double *partials) {
    const GT *gp[3] = {g0, g1, g2};
    const bool cont = allow_cont && is->stop == 6;
    const long long it_prev = is->iter;
    const double rho_prev = is->rho;
    double rr = 0.0, rmax = 0.0, rh2 = 0.0, qin = 0.0, qout = 0.0, en = 0.0, ez = 0.0;
    for (long long k = blockIdx.x * (long long)NT + threadIdx.x; k < U; k += (long long)gridDim.x * NT) {
        const long long i = cidx[k];
        const long long t = i - g.pad;
        const int cx = (int)(t % g.px);
        const int cy = (int)((t / g.px) % g.ny);
        const int cz = (int)(t / g.plane);
        const double xi = x[i];
        double rs = 0.0;
#pragma unroll
        for (int d = 0; d < NDIM; d++) {
            const int cd = g.coord(d, cx, cy, cz);
            const long long jp = g.up(i, d, cd), jm = g.down(i, d, cd);
            const double gpv = (double)gp[d][i], gmv = (double)gp[d][jm];
            const double xpv = x[jp], xmv = x[jm];
            rs += gpv * (xpv - xi) + gmv * (xmv - xi);
            en += gpv * (xi - xpv) * (xi - xpv);
        }
        const int cf = g.coord(g.f, cx, cy, cz);
        const double rv = rs;  // listed nodes are interior (0 < cf < nf - 1)
        const double rh = dis[i] * rv;
        r_list[k] = (TI)rh;
        rr += rv * rv;
        rmax = fmax(rmax, fabs(rv));
        rh2 += rh * rh;
        ez += (xi - g.p_out) * rv;
        if (cf == 1) {
            const double gin = (double)gp[g.f][i - g.stride(g.f)];
            qin += gin * (g.p_in - xi);
            en += gin * (g.p_in - xi) * (g.p_in - xi);
        }
        if (cf == g.nf - 2) qout += (double)gp[g.f][i] * (xi - g.p_out);
    }
    double v[7] = {rr, rmax, rh2, qin, qout, en, ez};
    const int ops[7] = {RED_SUM, RED_MAX, RED_SUM, RED_SUM, RED_SUM, RED_SUM, RED_SUM};
    if (!grid_reduce<7, NT>(v, ops, partials, &os->counter)) return;
    if (threadIdx.x != 0) return;
    outer_arm(g, v, os, is, cont, it_prev, rho_prev, reliable, delta2, tol_floor, tol_rel, tol_geff, bnorm,
              max_inner, stag_window);
}

template <int NDIM>
dim3 outer_grid(const Geom &g) {
    using OT = OTile<NDIM>;
    return dim3((g.px + OT::TW - 1) / OT::TW, (g.ny + OT::TH - 1) / OT::TH,
                NDIM == 3 ? (g.nz + OT::TD - 1) / OT::TD : 1);
}

template <typename GT, typename TI, int NDIM>
cudaError_t launch_outer_t(const OuterArgs &a, cudaStream_t st) {
    outer_kernel<GT, TI, NDIM><<<outer_grid<NDIM>(a.g), NT, 0, st>>>(
        a.g, (const GT *)a.graw[0], (const GT *)a.graw[1], (const GT *)a.graw[2], a.dis, a.x,
        (TI *)a.r_buf[0], (TI *)a.r_buf[1], a.os, a.is, a.reliable, a.allow_cont, a.delta2, a.tol_floor,
        a.tol_rel, a.tol_geff, a.bnorm, a.max_inner, a.stag_window, a.partials);
    return cudaGetLastError();
}

template <typename GT, typename TI, int NDIM>
cudaError_t launch_outer_list_t(const OuterArgs &a, const int *cidx, long long U, void *r_list, cudaStream_t st) {
    long long nb = (U + NT - 1) / NT;
    if (nb > 152LL * 16) nb = 152LL * 16;  // the partials array holds at least 152 x 16 blocks
    if (nb < 1) nb = 1;
    outer_list_kernel<GT, TI, NDIM><<<(int)nb, NT, 0, st>>>(
        a.g, (const GT *)a.graw[0], (const GT *)a.graw[1], (const GT *)a.graw[2], a.dis, a.x, cidx, U,
        (TI *)r_list, a.os, a.is, a.reliable, a.allow_cont, a.delta2, a.tol_floor, a.tol_rel, a.tol_geff, a.bnorm,
        a.max_inner, a.stag_window, a.partials);
    return cudaGetLastError();
}

inline long long nblocks(dim3 d) { return (long long)d.x * d.y * d.z; }

}  // namespace

int outer_grid_blocks(const Geom &g) {
    return (int)(g.ndim == 2 ? nblocks(outer_grid<2>(g)) : nblocks(outer_grid<3>(g)));
}

cudaError_t launch_outer_list(const OuterArgs &a, const int *cidx, long long U, void *r_list, cudaStream_t st) {
    if (a.root) {
        cudaError_t e = launch_fill_dangling(a.g, a.root, a.x, st);
        if (e != cudaSuccess) return e;
    }
    const bool r32 = a.raw_f32, i32 = a.inner_f32;
    if (a.g.ndim == 2) {
        if (r32) return i32 ? launch_outer_list_t<float, float, 2>(a, cidx, U, r_list, st)
                            : launch_outer_list_t<float, double, 2>(a, cidx, U, r_list, st);
        return i32 ? launch_outer_list_t<double, float, 2>(a, cidx, U, r_list, st)
                   : launch_outer_list_t<double, double, 2>(a, cidx, U, r_list, st);
    }
    if (r32) return i32 ? launch_outer_list_t<float, float, 3>(a, cidx, U, r_list, st)
                        : launch_outer_list_t<float, double, 3>(a, cidx, U, r_list, st);
    return i32 ? launch_outer_list_t<double, float, 3>(a, cidx, U, r_list, st)
               : launch_outer_list_t<double, double, 3>(a, cidx, U, r_list, st);
}

cudaError_t launch_outer(const OuterArgs &a, cudaStream_t st) {
    const bool r32 = a.raw_f32, i32 = a.inner_f32;
    if (a.apply_corr) {
        // the correction is applied in its own pass: the residual kernel reads
        // x at its neighbours' nodes, which must not change under it
        long long nb = ((long long)a.g.px * a.g.ny * a.g.nz + NT - 1) / NT;
        if (nb > 152LL * 16) nb = 152LL * 16;
        if (a.corr_f32)
            correct_kernel<float><<<(int)nb, NT, 0, st>>>(a.g, a.dis, a.x, (float *)a.y,
                                                          (const float *)a.p_buf[0],
                                                          (const float *)a.p_buf[1], a.is_corr);
        else
            correct_kernel<double><<<(int)nb, NT, 0, st>>>(a.g, a.dis, a.x, (double *)a.y,
                                                           (const double *)a.p_buf[0],
                                                           (const double *)a.p_buf[1], a.is_corr);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (a.root) {
        // dead-end nodes take their root's pressure (no current in a dead end)
        cudaError_t e = launch_fill_dangling(a.g, a.root, a.x, st);
        if (e != cudaSuccess) return e;
    }
    if (a.g.ndim == 2) {
        if (r32) return i32 ? launch_outer_t<float, float, 2>(a, st) : launch_outer_t<float, double, 2>(a, st);
        return i32 ? launch_outer_t<double, float, 2>(a, st) : launch_outer_t<double, double, 2>(a, st);
    }
    if (r32) return i32 ? launch_outer_t<float, float, 3>(a, st) : launch_outer_t<float, double, 3>(a, st);
    return i32 ? launch_outer_t<double, float, 3>(a, st) : launch_outer_t<double, double, 3>(a, st);
}

}  // namespace netsolve
