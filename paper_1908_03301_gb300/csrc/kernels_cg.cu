// kernels_cg.cu -- the conjugate-gradient hot loop (Sec. IV) and the FP64
// residual pass of the iterative refinement.
//
// Inner loop.  Jacobi preconditioning is applied as the symmetric scaling
// A = D^-1/2 G D^-1/2 (unit diagonal), so preconditioned CG on G becomes
// plain CG on A and the iteration reads no diagonal.  One kernel launch is
// one full CG iteration.  Launch k
//   1. finishes iteration k-1 from its scalars alpha, beta:
//        r_k = r_{k-1} - alpha q_{k-1},  p_k = r_k + beta p_{k-1},
//        y_k = y_{k-1} + alpha p_{k-1},
//      for its tile and (p only) a one-node halo, staged in shared memory;
//   2. computes q_k = A p_k from the staged p_k (5- or 7-point stencil on
//      the bond planes) and the four sums <p,q>, <r,q>, <q,q>, <r,r>;
//   3. the last CTA to finish reduces the sums (grid_reduce) and sets
//        alpha_k = <r,r> / <p,q>,
//        beta_k  = <r_{k+1}, r_{k+1}> / <r,r>   with
//        <r_{k+1}, r_{k+1}> = <r,r> - 2 alpha_k <r,q> + alpha_k^2 <q,q>,
//      the expansion of ||r_k - alpha_k q_k||^2, so one reduction per
//      iteration suffices.
// Every vector is read once and written once per iteration:
// y, r, p, q (4 + 4 accesses) plus one bond plane per dimension, the
// 32 + 4d bytes per unknown of the FP32 path.  r, p and q are double
// buffered (iteration k reads set k%2 and writes the other), so a CTA can
// read its neighbours' previous values for the halo while they write.  The paper's three kernels per
// iteration with a host-side final sum (Sec. IV) become one kernel with an
// on-device reduction.
//
// Outer loop (FP64).  One launch applies the previous correction
// x += D^-1/2 y (tile + halo), recomputes the true residual
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

// p_new = (r - alpha q) + beta p, identical on the owner and in every halo.
template <typename T>
__device__ __forceinline__ T rnew(T r, T q, T alpha) { return fma(-alpha, q, r); }
template <typename T>
__device__ __forceinline__ T pnew(T rn, T p, T beta) { return fma(beta, p, rn); }

template <typename T, int NDIM, int TW, int TH, int TD>
struct Tile {
    static constexpr int V = Vec<T>::N;
    static constexpr int TX = TW / V;                 // vector columns
    static constexpr int ZP = NDIM == 3 ? TD + 2 : 1; // staged planes
    static constexpr int ZO = NDIM == 3 ? 1 : 0;
    static constexpr int SH = TH + 2;
    static constexpr int SW = TW + 2 * V;             // staged row width
    static constexpr int ITEMS = TX * TH * TD / NT;
    static constexpr int HY = 2 * TD * TX;            // row-halo vectors
    static constexpr int HZ = NDIM == 3 ? 2 * TH * TX : 0;
    static constexpr int HX = 2 * TH * TD;            // column-halo scalars
    static_assert(TW % V == 0, "tile width");
    static_assert((TX * TH * TD) % NT == 0, "tile size must be a multiple of the CTA");
    static_assert(NDIM == 3 || TD == 1, "2D tiles are one plane");
    __device__ static int sidx(int zz, int yy, int xx) { return (zz * SH + yy) * SW + V + xx; }
};

template <typename T, int NDIM, int TW, int TH, int TD>
__global__ void __launch_bounds__(NT)
inner_iter_kernel(Geom g, const T *__restrict__ g0, const T *__restrict__ g1,
                  const T *__restrict__ g2, T *__restrict__ y, T *r0, T *r1, T *p0, T *p1,
                  T *q0, T *q1, InnerScal *s, double *partials) {
    using TL = Tile<T, NDIM, TW, TH, TD>;
    constexpr int V = TL::V;
    __shared__ __align__(16) T sp[TL::ZP * TL::SH * TL::SW];

    if (*(volatile int *)&s->stop) return;
    const long long iter = s->iter;
    const bool first = (iter == 0);
    const T alpha = (T)s->alpha, beta = (T)s->beta;
    // r, p, q are double-buffered: neighbours read the previous values as
    // halo while the owner writes the new ones.  Iteration k reads set k%2.
    const bool odd = iter & 1;
    const T *__restrict__ r = odd ? r1 : r0;
    const T *__restrict__ p = odd ? p1 : p0;
    const T *__restrict__ q = odd ? q1 : q0;
    T *__restrict__ ro = odd ? r0 : r1;
    T *__restrict__ po = odd ? p0 : p1;
    T *__restrict__ qo = odd ? q0 : q1;
    const int x0 = blockIdx.x * TW, y0 = blockIdx.y * TH, z0 = blockIdx.z * TD;

    // ---- 1. finish the previous iteration on the tile, stage p_k ----------
    Vec<T> rn[TL::ITEMS];
#pragma unroll
    for (int it = 0; it < TL::ITEMS; it++) {
        const int item = threadIdx.x + it * NT;
        const int vx = item % TL::TX, t = item / TL::TX, yy = t % TH, zz = t / TH;
        const int x = x0 + vx * V, yq = y0 + yy, z = z0 + zz;
        Vec<T> pn;
        if (x < g.px && yq < g.ny && z < g.nz) {
            const long long i = g.idx(x, yq, z);
            Vec<T> rv;
            rv.load(r + i);
            if (first) {
                rn[it] = rv;
                pn = rv;
                Vec<T> zv;
                zv.zero();
                zv.store(y + i);
                rv.store(ro + i);
            } else {
                Vec<T> qv, pv, yv;
                qv.load(q + i);
                pv.load(p + i);
                yv.load(y + i);
#pragma unroll
                for (int k = 0; k < V; k++) {
                    rn[it].v[k] = rnew(rv.v[k], qv.v[k], alpha);
                    pn.v[k] = pnew(rn[it].v[k], pv.v[k], beta);
                    yv.v[k] = fma(alpha, pv.v[k], yv.v[k]);
                }
                rn[it].store(ro + i);
                yv.store(y + i);
            }
            pn.store(po + i);
        } else {
            rn[it].zero();
            pn.zero();
        }
        pn.store(sp + TL::sidx(zz + TL::ZO, yy + 1, vx * V));
    }
    // halo rows (and planes in 3D): p only
    for (int item = threadIdx.x; item < TL::HY + TL::HZ; item += NT) {
        int vx, yy, zz;
        if (item < TL::HY) {
            vx = item % TL::TX;
            const int t = item / TL::TX;
            zz = t % TD;
            yy = (t / TD) ? TH : -1;
        } else {
            const int i2 = item - TL::HY;
            vx = i2 % TL::TX;
            const int t = i2 / TL::TX;
            yy = t % TH;
            zz = (t / TH) ? TD : -1;
        }
        const int x = x0 + vx * V, yq = y0 + yy, z = z0 + zz;
        Vec<T> pn;
        if (x < g.px && yq >= 0 && yq < g.ny && z >= 0 && z < g.nz) {
            const long long i = g.idx(x, yq, z);
            Vec<T> rv;
            rv.load(r + i);
            if (first) {
                pn = rv;
            } else {
                Vec<T> qv, pv;
                qv.load(q + i);
                pv.load(p + i);
#pragma unroll
                for (int k = 0; k < V; k++) pn.v[k] = pnew(rnew(rv.v[k], qv.v[k], alpha), pv.v[k], beta);
            }
        } else {
            pn.zero();
        }
        pn.store(sp + TL::sidx(zz + TL::ZO, yy + 1, vx * V));
    }
    // halo columns: scalars
    for (int item = threadIdx.x; item < TL::HX; item += NT) {
        const int side = item & 1, t = item >> 1, yy = t % TH, zz = t / TH;
        const int x = side ? x0 + TW : x0 - 1, yq = y0 + yy, z = z0 + zz;
        T pn = T(0);
        if (x >= 0 && x < g.px && yq < g.ny && z < g.nz) {
            const long long i = g.idx(x, yq, z);
            pn = first ? r[i] : pnew(rnew(r[i], q[i], alpha), p[i], beta);
        }
        sp[TL::sidx(zz + TL::ZO, yy + 1, side ? TW : -1)] = pn;
    }
    __syncthreads();

    // ---- 2. q = A p on the tile and the four sums -----------------------
    T a_pq = T(0), a_rq = T(0), a_qq = T(0), a_rr = T(0);
#pragma unroll
    for (int it = 0; it < TL::ITEMS; it++) {
        const int item = threadIdx.x + it * NT;
        const int vx = item % TL::TX, t = item / TL::TX, yy = t % TH, zz = t / TH;
        const int x = x0 + vx * V, yq = y0 + yy, z = z0 + zz;
        if (!(x < g.px && yq < g.ny && z < g.nz)) continue;
        const long long i = g.idx(x, yq, z);
        const T *row = sp + TL::sidx(zz + TL::ZO, yy + 1, vx * V);
        Vec<T> pc, pu, pd, gx, gy, gym, qv;
        pc.load(row);
        pu.load(row + TL::SW);
        pd.load(row - TL::SW);
        const T pl = row[-1], pr = row[V];
        gx.load(g0 + i);
        const T gxm = g0[i - 1];
        gy.load(g1 + i);
        gym.load(g1 + i - g.px);
        Vec<T> pf, pb, gz, gzm;
        if (NDIM == 3) {
            pf.load(row + TL::SH * TL::SW);
            pb.load(row - TL::SH * TL::SW);
            gz.load(g2 + i);
            gzm.load(g2 + i - g.plane);
        }
#pragma unroll
        for (int k = 0; k < V; k++) {
            const T left = k == 0 ? pl : pc.v[k - 1];
            const T right = k == V - 1 ? pr : pc.v[k + 1];
            const T gl = k == 0 ? gxm : gx.v[k - 1];
            T nb = gl * left;
            nb = fma(gx.v[k], right, nb);
            nb = fma(gym.v[k], pd.v[k], nb);
            nb = fma(gy.v[k], pu.v[k], nb);
            if (NDIM == 3) {
                nb = fma(gzm.v[k], pb.v[k], nb);
                nb = fma(gz.v[k], pf.v[k], nb);
            }
            const T qk = pc.v[k] - nb;
            qv.v[k] = qk;
            a_pq = fma(pc.v[k], qk, a_pq);
            a_rq = fma(rn[it].v[k], qk, a_rq);
            a_qq = fma(qk, qk, a_qq);
            a_rr = fma(rn[it].v[k], rn[it].v[k], a_rr);
        }
        qv.store(qo + i);
    }

    // ---- 3. one grid reduction; the last CTA sets the next step ----------
    double v[4] = {(double)a_pq, (double)a_rq, (double)a_qq, (double)a_rr};
    const int ops[4] = {RED_SUM, RED_SUM, RED_SUM, RED_SUM};
    if (!grid_reduce<4, NT>(v, ops, partials, &s->counter)) return;
    if (threadIdx.x == 0) finish_iteration(s, iter, v);
}

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

// ---------------------------------------------------------------------------
// tile configurations
// ---------------------------------------------------------------------------
template <typename T, int NDIM> struct InnerCfg;
template <> struct InnerCfg<float, 2> { static constexpr int TW = 256, TH = 16, TD = 1; };
template <> struct InnerCfg<double, 2> { static constexpr int TW = 128, TH = 16, TD = 1; };
template <> struct InnerCfg<float, 3> { static constexpr int TW = 64, TH = 8, TD = 8; };
template <> struct InnerCfg<double, 3> { static constexpr int TW = 32, TH = 8, TD = 8; };

template <typename T, int NDIM>
dim3 inner_grid(const Geom &g) {
    using C = InnerCfg<T, NDIM>;
    return dim3((g.px + C::TW - 1) / C::TW, (g.ny + C::TH - 1) / C::TH,
                NDIM == 3 ? (g.nz + C::TD - 1) / C::TD : 1);
}

template <typename T, int NDIM>
cudaError_t launch_inner_t(const InnerArgs &a, cudaStream_t st) {
    using C = InnerCfg<T, NDIM>;
    inner_iter_kernel<T, NDIM, C::TW, C::TH, C::TD><<<inner_grid<T, NDIM>(a.g), NT, 0, st>>>(
        a.g, (const T *)a.gs[0], (const T *)a.gs[1], (const T *)a.gs[2], (T *)a.y,
        (T *)a.r[0], (T *)a.r[1], (T *)a.p[0], (T *)a.p[1], (T *)a.q[0], (T *)a.q[1], a.s,
        a.partials);
    return cudaGetLastError();
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

inline long long nblocks(dim3 d) { return (long long)d.x * d.y * d.z; }

}  // namespace

int inner_grid_blocks(const Geom &g, int f32) {
    if (g.ndim == 2) return (int)nblocks(f32 ? inner_grid<float, 2>(g) : inner_grid<double, 2>(g));
    return (int)nblocks(f32 ? inner_grid<float, 3>(g) : inner_grid<double, 3>(g));
}

cudaError_t launch_inner_iter(const InnerArgs &a, int f32, cudaStream_t st) {
    if (a.g.ndim == 2) return f32 ? launch_inner_t<float, 2>(a, st) : launch_inner_t<double, 2>(a, st);
    return f32 ? launch_inner_t<float, 3>(a, st) : launch_inner_t<double, 3>(a, st);
}

int outer_grid_blocks(const Geom &g) {
    return (int)(g.ndim == 2 ? nblocks(outer_grid<2>(g)) : nblocks(outer_grid<3>(g)));
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
