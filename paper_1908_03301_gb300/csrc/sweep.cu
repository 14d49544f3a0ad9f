// sweep.cu -- persistent, warp-specialised CG sweep over segmented networks.
//
// One launch = one CG iteration (Sec. IV; the fused form of kernels_cg.cu:
// finish iteration k-1, stencil, four sums, last arrival sets alpha/beta) for
// every network in the plan whose inner solve is running.
//
// Organisation (GB300): one CTA per SM, 16 consumer warps + 1 producer warp.
//  * The producer walks the CTA's segments and, for every march step, issues
//    1D bulk copies (cp.async.bulk, TMA) of the rows the step needs into one
//    of S shared-memory stages, completing on that stage's "full" mbarrier;
//    it refills a stage once all consumer warps have arrived on its "empty"
//    mbarrier.  It runs ahead across segment boundaries, so the pipeline
//    never drains inside a CTA's list.
//  * Consumers, at step t of a segment (march index m = m0 + t):
//      - finish iteration k-1 on index m+1: r = r - a q, p = r + b p,
//        y = y + a p_old, for the segment's rows plus a one-node halo (p only),
//        into a 4-slot shared ring of p patches; owned values go to memory;
//      - named barrier;
//      - stencil q = A p on index m from the ring (x neighbours by warp
//        shuffle, y neighbours in the ring patch, march neighbours in the
//        adjacent ring slots) and the sums <p,q>, <r,q>, <q,q>, <r,r>.
//  * At the end of a segment its sums go to the network's slot; the network's
//    last segment to arrive reduces the slots in order (deterministic) and
//    runs finish_iteration.
// Every vector is read and written once per iteration plus one halo row /
// column per segment edge; r, p, q are double-buffered by iteration parity.
// All waits are bounded; a wait that gives up marks the network (err) and the
// CTA keeps the barrier protocol so that every issued copy is waited for.
#include <cfloat>
#include <cmath>
#include <type_traits>

#include "ffloat.cuh"
#include "kernels.h"
#include "sweep.cuh"
#include "tma.cuh"

namespace netsolve {
namespace {

constexpr int NC = 512;              // consumer threads
constexpr int NCW = NC / 32;         // consumer warps
constexpr int NTH = NC + 32;         // + one producer warp
constexpr uint32_t WAIT_LIMIT = 1u << 22;
constexpr uint32_t WAIT_LIMIT_AFTER_ERROR = 1u << 10;

template <typename T, int NDIM>
struct SW {
    static constexpr int V = 16 / (int)sizeof(T);   // elements per 16 bytes
    static constexpr int VT = 8 / (int)sizeof(T);   // elements per consumer thread
    static constexpr int HH = NDIM == 3 ? 1 : 0;    // halo rows above/below a patch
    static constexpr int NARR = NDIM == 3 ? 7 : 6;  // r q p y gx gy [gz]
    static constexpr int WMAX = NDIM == 3 ? 1024 / (int)sizeof(T) : NC * VT;
    // 2D: a slot holds one array's rows of a stage (up to two rows of the
    // widest block, more rows of narrower whole-row blocks)
    static constexpr int SLOT = NDIM == 3 ? 7296 : ((2 * NC * VT + 2 * V) * (int)sizeof(T) + 127) / 128 * 128;
    static constexpr int S = NDIM == 3 ? 3 : 4;     // stages
    static constexpr int BAR = 128;
    static constexpr int STAGE = NARR * SLOT;
    static constexpr int RING = NDIM == 3 ? 4 * SLOT : 0;  // 2D keeps p rows in registers
    static constexpr int BYTES = BAR + S * STAGE + RING;
    static_assert(2 * S * 8 <= BAR, "barrier area");
    static_assert(BYTES <= 227 * 1024, "shared memory");
};

enum { A_R = 0, A_Q = 1, A_P = 2, A_Y = 3, A_GX = 4, A_GY = 5, A_GZ = 6 };

// Rows of a 2D segment staged together.  A block spanning whole padded rows
// (x0 = 0, w = px) is contiguous in memory, so each array's rows of a stage
// are one bulk copy; other blocks copy row by row.  Fewer, larger copies: the
// copy engine spends a fixed time per copy (about 0.1 us on GB300).
constexpr int RMAX2 = 16;
template <typename T>
__host__ __device__ __forceinline__ int rows_per_stage_2d(int w, int px, bool fullrow) {
    using C = SW<T, 2>;
    constexpr int cap = C::SLOT / (int)sizeof(T);
    int R = fullrow ? (cap - 2 * C::V) / px : cap / (w + 2 * C::V);
    return R < 1 ? 1 : (R > RMAX2 ? RMAX2 : R);
}

template <typename T>
__device__ __forceinline__ T rnew(T r, T q, T a) { return fma(-a, q, r); }
template <typename T>
__device__ __forceinline__ T pnew(T rn, T p, T b) { return fma(b, p, rn); }

// 8-byte register vector of T
template <typename T> struct V8;
template <> struct V8<float> {
    float v[2];
    __device__ __forceinline__ void ld(const float *p) { float2 t = *reinterpret_cast<const float2 *>(p); v[0] = t.x; v[1] = t.y; }
    __device__ __forceinline__ void st(float *p) const { *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]); }
    __device__ __forceinline__ void zero() { v[0] = v[1] = 0.f; }
};
template <> struct V8<double> {
    double v[1];
    __device__ __forceinline__ void ld(const double *p) { v[0] = *p; }
    __device__ __forceinline__ void st(double *p) const { *p = v[0]; }
    __device__ __forceinline__ void zero() { v[0] = 0.0; }
};

__device__ __forceinline__ void cons_sync() { asm volatile("bar.sync 1, %0;" ::"n"(NC) : "memory"); }

template <int NDIM>
__device__ __forceinline__ long long gidx(const Geom &g, int x, int y, int m) {
    return NDIM == 2 ? g.idx(x, m, 0) : g.idx(x, y, m);
}

template <int NDIM>
__device__ __forceinline__ int march_extent(const Geom &g) { return NDIM == 2 ? g.ny : g.nz; }

template <typename T, int NDIM>
__device__ __forceinline__ T *stage_arr(unsigned char *smem, int b, int arr) {
    using C = SW<T, NDIM>;
    return reinterpret_cast<T *>(smem + C::BAR + b * C::STAGE + arr * C::SLOT);
}
template <typename T, int NDIM>
__device__ __forceinline__ T *ring_slot(unsigned char *smem, long long G) {
    using C = SW<T, NDIM>;
    return reinterpret_cast<T *>(smem + C::BAR + C::S * C::STAGE + (int)(G & 3) * C::SLOT);
}

struct SegView {
    int x0, w, y0, h, m0, m1, nv, nitems;
    bool first, odd;
};

__device__ __forceinline__ bool inst_stopped(const SweepInst &I) {
    return *(volatile int *)&I.s->stop != 0;
}

// ------------------------------------------------------------------ producer
// Per-segment constants of the producer (registers).
template <typename T>
struct ProdSeg {
    const T *r, *q, *p, *y, *gx, *gy, *gz;  // read set, at (x0 - V or x0, row y0)
    long long ms;                            // march stride (elements)
    long long rs;                            // row stride within a 3D patch
    int nm, m0, m1, w, h;
    int px;     // row pitch
    bool full;  // 3D patch spanning whole padded rows: its rows are contiguous
    bool first;
};

template <typename T, int NDIM>
__device__ __forceinline__ void produce_step(unsigned char *smem, uint64_t *full, int b,
                                             const ProdSeg<T> &ps, int t, int lane) {
    using C = SW<T, NDIM>;
    constexpr int V = C::V, HH = C::HH;
    const int me = ps.m0 + t + 1, mt = ps.m0 + t;
    const bool L = me >= 0 && me < ps.nm;
    const bool ownme = me >= ps.m0 && me < ps.m1;
    const bool bvalid = mt >= 0 && mt < ps.nm;
    const int h = ps.h, w = ps.w;
    const int rowsL = h + 2 * HH;
    const int nL = L ? (ps.first ? 1 : 3) : 0;
    const int nY = (L && ownme && !ps.first) ? h : 0;
    const int nGX = (t >= 0 && bvalid) ? h : 0;
    const int nGY = NDIM == 2 ? ((t >= -1 && bvalid) ? 1 : 0) : ((t >= 0 && bvalid) ? h + 1 : 0);
    const int nGZ = NDIM == 3 ? ((t >= -1 && bvalid) ? h : 0) : 0;
    const uint32_t bw = (uint32_t)(w + 2 * V) * sizeof(T), bn = (uint32_t)w * sizeof(T),
                   bx = (uint32_t)(w + V) * sizeof(T);
    const int total = nL * rowsL + nY + nGX + nGY + nGZ;
    const long long oe = (long long)me * ps.ms, ot = (long long)mt * ps.ms;
    // exactly one arrive.expect_tx per stage and step (the full barrier
    // counts one arrival): whole-row patches take their own branch
    if (NDIM == 3 && ps.full) {
        // whole rows: each array's rows are one contiguous run, so one copy
        // per array (the row ends' zero bonds stand in for halo columns)
        const int px = ps.px;
        if (lane == 0) {
            const uint32_t bytes = (uint32_t)nL * (uint32_t)(rowsL * px + 2 * V) * sizeof(T) +
                                   (uint32_t)(nY ? h * px : 0) * sizeof(T) +
                                   (uint32_t)(nGX ? h * px + V : 0) * sizeof(T) +
                                   (uint32_t)(nGY ? (h + 1) * px : 0) * sizeof(T) +
                                   (uint32_t)(nGZ ? h * px : 0) * sizeof(T);
            mbar_arrive_expect_tx(&full[b], bytes);
        }
        __syncwarp();
        if (lane < nL) {
            const T *src = lane == 0 ? ps.r : (lane == 1 ? ps.q : ps.p);
            bulk_load(stage_arr<T, NDIM>(smem, b, lane), src + oe - (long long)HH * ps.rs,
                      (uint32_t)(rowsL * px + 2 * V) * sizeof(T), &full[b]);
        } else if (lane == 4 && nY) {
            bulk_load(stage_arr<T, NDIM>(smem, b, A_Y), ps.y + oe, (uint32_t)(h * px) * sizeof(T), &full[b]);
        } else if (lane == 5 && nGX) {
            bulk_load(stage_arr<T, NDIM>(smem, b, A_GX), ps.gx + ot, (uint32_t)(h * px + V) * sizeof(T), &full[b]);
        } else if (lane == 6 && nGY) {
            bulk_load(stage_arr<T, NDIM>(smem, b, A_GY), ps.gy + ot - ps.rs, (uint32_t)((h + 1) * px) * sizeof(T),
                      &full[b]);
        } else if (lane == 7 && nGZ) {
            bulk_load(stage_arr<T, NDIM>(smem, b, A_GZ), ps.gz + ot, (uint32_t)(h * px) * sizeof(T), &full[b]);
        }
        return;
    }
    if (lane == 0) {
        const uint32_t bytes = (uint32_t)(nL * rowsL) * bw + (uint32_t)nY * bn + (uint32_t)nGX * bx +
                               (uint32_t)(nGY + nGZ) * bn;
        mbar_arrive_expect_tx(&full[b], bytes);
    }
    __syncwarp();
    for (int k = lane; k < total; k += 32) {
        int kk = k;
        if (kk < nL * rowsL) {
            const int a = kk / rowsL, rr = kk % rowsL - HH;
            const T *src = a == 0 ? ps.r : (a == 1 ? ps.q : ps.p);
            bulk_load(stage_arr<T, NDIM>(smem, b, a) + (rr + HH) * (w + 2 * V), src + oe + rr * ps.rs, bw,
                      &full[b]);
            continue;
        }
        kk -= nL * rowsL;
        if (kk < nY) {
            bulk_load(stage_arr<T, NDIM>(smem, b, A_Y) + kk * w, ps.y + oe + kk * ps.rs, bn, &full[b]);
            continue;
        }
        kk -= nY;
        if (kk < nGX) {
            bulk_load(stage_arr<T, NDIM>(smem, b, A_GX) + kk * (w + V), ps.gx + ot + kk * ps.rs, bx, &full[b]);
            continue;
        }
        kk -= nGX;
        if (kk < nGY) {
            const int rr = NDIM == 2 ? 0 : kk - 1;  // 3D: rows y0-1 .. y0+h-1
            bulk_load(stage_arr<T, NDIM>(smem, b, A_GY) + kk * w, ps.gy + ot + rr * ps.rs, bn, &full[b]);
            continue;
        }
        kk -= nGY;
        bulk_load(stage_arr<T, NDIM>(smem, b, A_GZ) + kk * w, ps.gz + ot + kk * ps.rs, bn, &full[b]);
    }
}

// Producer, 2D: the stage of march steps t0 .. t0+tn-1 (tn <= R rows).  Step
// t finishes row me = m0+t+1 (r, q, p; y when owned) and applies the stencil
// on row mt = m0+t (gx from t >= 0, gy from t >= -1).  Row j of a stage sits
// at j * pitch in each slot.
template <typename T>
__device__ __forceinline__ void produce_stage_2d(unsigned char *smem, uint64_t *full, int b,
                                                 const ProdSeg<T> &ps, int t0, int tn, bool fullrow,
                                                 int lane) {
    using C = SW<T, 2>;
    constexpr int V = C::V;
    const int w = ps.w, px = ps.px, nm = ps.nm;
    const int me_lo = ps.m0 + t0 + 1, mt_lo = ps.m0 + t0;
    const int jL0 = max(0, -me_lo), jL1 = min(tn, nm - me_lo);
    const int jY0 = ps.first ? 0 : max(jL0, ps.m0 - me_lo), jY1 = ps.first ? 0 : min(jL1, ps.m1 - me_lo);
    const int jX0 = max(max(0, -t0), -mt_lo), jX1 = min(tn, nm - mt_lo);
    const int jG0 = max(max(0, -1 - t0), -mt_lo), jG1 = jX1;
    const int nL = ps.first ? 1 : 3;
    const int rL = max(0, jL1 - jL0), rY = max(0, jY1 - jY0), rX = max(0, jX1 - jX0), rG = max(0, jG1 - jG0);
    const long long ms = ps.ms;
    if (fullrow) {
        if (lane == 0) {
            const uint32_t bytes = (uint32_t)sizeof(T) *
                ((rL ? (uint32_t)nL * (uint32_t)(rL * px + 2 * V) : 0u) + (uint32_t)(rY * px) +
                 (rX ? (uint32_t)(rX * px + V) : 0u) + (uint32_t)(rG * px));
            mbar_arrive_expect_tx(&full[b], bytes);
        }
        __syncwarp();
        if (lane < nL && rL) {
            const T *src = lane == 0 ? ps.r : (lane == 1 ? ps.q : ps.p);
            bulk_load(stage_arr<T, 2>(smem, b, lane) + jL0 * px, src + (long long)(me_lo + jL0) * ms,
                      (uint32_t)(rL * px + 2 * V) * sizeof(T), &full[b]);
        } else if (lane == 4 && rY) {
            bulk_load(stage_arr<T, 2>(smem, b, A_Y) + jY0 * px, ps.y + (long long)(me_lo + jY0) * ms,
                      (uint32_t)(rY * px) * sizeof(T), &full[b]);
        } else if (lane == 5 && rX) {
            bulk_load(stage_arr<T, 2>(smem, b, A_GX) + jX0 * px, ps.gx + (long long)(mt_lo + jX0) * ms,
                      (uint32_t)(rX * px + V) * sizeof(T), &full[b]);
        } else if (lane == 6 && rG) {
            bulk_load(stage_arr<T, 2>(smem, b, A_GY) + jG0 * px, ps.gy + (long long)(mt_lo + jG0) * ms,
                      (uint32_t)(rG * px) * sizeof(T), &full[b]);
        }
        return;
    }
    // row by row: pitches w + 2V (r q p), w (y, gy), w + V (gx)
    if (lane == 0) {
        const uint32_t bytes = (uint32_t)sizeof(T) *
            ((uint32_t)(nL * rL) * (uint32_t)(w + 2 * V) + (uint32_t)(rY * w) + (uint32_t)(rX * (w + V)) +
             (uint32_t)(rG * w));
        mbar_arrive_expect_tx(&full[b], bytes);
    }
    __syncwarp();
    const int total = nL * rL + rY + rX + rG;
    for (int k = lane; k < total; k += 32) {
        int kk = k;
        if (kk < nL * rL) {
            const int a = kk / rL, j = jL0 + kk % rL;
            const T *src = a == 0 ? ps.r : (a == 1 ? ps.q : ps.p);
            bulk_load(stage_arr<T, 2>(smem, b, a) + j * (w + 2 * V), src + (long long)(me_lo + j) * ms,
                      (uint32_t)(w + 2 * V) * sizeof(T), &full[b]);
            continue;
        }
        kk -= nL * rL;
        if (kk < rY) {
            const int j = jY0 + kk;
            bulk_load(stage_arr<T, 2>(smem, b, A_Y) + j * w, ps.y + (long long)(me_lo + j) * ms,
                      (uint32_t)w * sizeof(T), &full[b]);
            continue;
        }
        kk -= rY;
        if (kk < rX) {
            const int j = jX0 + kk;
            bulk_load(stage_arr<T, 2>(smem, b, A_GX) + j * (w + V), ps.gx + (long long)(mt_lo + j) * ms,
                      (uint32_t)(w + V) * sizeof(T), &full[b]);
            continue;
        }
        kk -= rX;
        const int j = jG0 + kk;
        bulk_load(stage_arr<T, 2>(smem, b, A_GY) + j * w, ps.gy + (long long)(mt_lo + j) * ms,
                  (uint32_t)w * sizeof(T), &full[b]);
    }
}

template <typename T, int NDIM>
__device__ SegView seg_view(const SweepSeg &sg, const SweepInst &I) {
    using C = SW<T, NDIM>;
    SegView v;
    v.x0 = sg.x0;
    v.w = sg.w;
    v.y0 = sg.y0;
    v.h = sg.h;
    v.m0 = sg.m0;
    v.m1 = sg.m1;
    v.nv = sg.w / C::VT;
    v.nitems = v.nv * sg.h;
    const long long it = I.s->iter;
    v.first = it == 0;
    v.odd = it & 1;
    return v;
}

// ------------------------------------------------------------------ 2D consumer
// 2D segments need no exchange between warps: warp k owns columns
// [64k, 64k+64) of the block (two per lane), the march neighbours (rows m-1,
// m, m+1) stay in registers, x neighbours come by shuffle and the strip-edge
// values are recomputed from the staged rows.  Warps meet only at the
// pipeline's mbarriers.
template <typename T>
__device__ void consume_segment_2d(unsigned char *smem, uint64_t *full, uint64_t *empty,
                                   const SweepInst &I, const SweepSeg &sg, long long &G,
                                   uint32_t &lim, int *s_err, T (&acc)[4]) {
    using C = SW<T, 2>;
    constexpr int V = C::V, VT = C::VT, S = C::S;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int px = I.g.px, nm = I.g.ny;
    const long long ms = px;
    const long long it = I.s->iter;
    const bool first = it == 0, odd = it & 1;
    const T alpha = (T)I.s->alpha, beta = (T)I.s->beta;
    const int w = sg.w, x0 = sg.x0, m0 = sg.m0, m1 = sg.m1;
    const int cx = warp * 32 * VT + lane * VT;  // first column (relative to x0)
    const bool act = cx < w;
    const bool need_l = lane == 0, need_r = lane == 31 || (act && cx + VT >= w);
    const long long base = I.g.pad + x0 + cx;
    T *ro = (T *)(odd ? I.r[0] : I.r[1]) + base;
    T *po = (T *)(odd ? I.p[0] : I.p[1]) + base;
    T *qo = (T *)(odd ? I.q[0] : I.q[1]) + base;
    T *yv = (T *)I.y + base;
    const bool lok = x0 + cx - 1 >= 0, rok = x0 + cx + VT < px;
    V8<T> pm1, p0, r_cur, r_next, mdown;
    pm1.zero(); p0.zero(); r_cur.zero(); r_next.zero(); mdown.zero();
    T h0l = T(0), h0r = T(0);  // p at row m, columns cx-1 and cx+VT (edge lanes)
    T a_pq = T(0), a_rq = T(0), a_qq = T(0), a_rr = T(0);
    // stages of R rows; row j of a stage at j * pitch in each slot
    const bool fullrow = x0 == 0 && w == px;
    const int R = rows_per_stage_2d<T>(w, px, fullrow);
    const int PL = fullrow ? px : w + 2 * V, PY = fullrow ? px : w, PGX = fullrow ? px : w + V;
    const int L = m1 - m0;
    for (int t0 = -2; t0 < L; t0 += R, G++) {
      const int b = (int)(G % S);
      if (!mbar_wait_bounded(&full[b], (uint32_t)(G / S) & 1u, lim)) {
          *s_err = 1;
          lim = WAIT_LIMIT_AFTER_ERROR;
      }
      const int tn = min(R, L - t0);
      for (int j = 0; j < tn; j++) {
        const int t = t0 + j;
        const int me = m0 + t + 1;
        const T *sr = stage_arr<T, 2>(smem, b, A_R) + j * PL + V + cx;
        const T *sq = stage_arr<T, 2>(smem, b, A_Q) + j * PL + V + cx;
        const T *sp = stage_arr<T, 2>(smem, b, A_P) + j * PL + V + cx;
        // ---- finish iteration k-1 on row me (registers) ----
        V8<T> pn;
        pn.zero();
        T h1l = T(0), h1r = T(0);
        if (me >= 0 && me < nm) {
            if (act) {
                V8<T> rv;
                rv.ld(sr);
                if (first) {
                    r_next = rv;
                    pn = rv;
                } else {
                    V8<T> qv, pv;
                    qv.ld(sq);
                    pv.ld(sp);
#pragma unroll
                    for (int k = 0; k < VT; k++) {
                        r_next.v[k] = rnew(rv.v[k], qv.v[k], alpha);
                        pn.v[k] = pnew(r_next.v[k], pv.v[k], beta);
                    }
                }
                if (me >= m0 && me < m1) {
                    const long long i = (long long)me * ms;
                    r_next.st(ro + i);
                    pn.st(po + i);
                    V8<T> yn;
                    if (first) {
                        yn.zero();
                    } else {
                        V8<T> pv;
                        pv.ld(sp);
                        yn.ld(stage_arr<T, 2>(smem, b, A_Y) + j * PY + cx);
#pragma unroll
                        for (int k = 0; k < VT; k++) yn.v[k] = fma(alpha, pv.v[k], yn.v[k]);
                    }
                    yn.st(yv + i);
                }
                if (need_l && lok) h1l = first ? sr[-1] : pnew(rnew(sr[-1], sq[-1], alpha), sp[-1], beta);
                if (need_r && rok) h1r = first ? sr[VT] : pnew(rnew(sr[VT], sq[VT], alpha), sp[VT], beta);
            }
        } else {
            r_next.zero();
        }
        // ---- stencil on row m = me - 1 ----
        if (t >= 0) {
            V8<T> gx, mup, qv;
            gx.zero();
            mup.zero();
            const T *sgx = stage_arr<T, 2>(smem, b, A_GX) + j * PGX + V + cx;
            if (act) {
                gx.ld(sgx);
                mup.ld(stage_arr<T, 2>(smem, b, A_GY) + j * PY + cx);
            }
            T left = __shfl_up_sync(0xffffffffu, p0.v[VT - 1], 1);
            T right = __shfl_down_sync(0xffffffffu, p0.v[0], 1);
            T gxm = __shfl_up_sync(0xffffffffu, gx.v[VT - 1], 1);
            if (act) {
                if (need_l) {
                    left = h0l;
                    gxm = sgx[-1];
                }
                if (need_r) right = h0r;
#pragma unroll
                for (int k = 0; k < VT; k++) {
                    const T lv = k == 0 ? left : p0.v[k - 1];
                    const T rv = k == VT - 1 ? right : p0.v[k + 1];
                    const T gl = k == 0 ? gxm : gx.v[k - 1];
                    T nb = gl * lv;
                    nb = fma(gx.v[k], rv, nb);
                    nb = fma(mdown.v[k], pm1.v[k], nb);
                    nb = fma(mup.v[k], pn.v[k], nb);
                    const T qk = p0.v[k] - nb;
                    qv.v[k] = qk;
                    a_pq = fma(p0.v[k], qk, a_pq);
                    a_rq = fma(r_cur.v[k], qk, a_rq);
                    a_qq = fma(qk, qk, a_qq);
                    a_rr = fma(r_cur.v[k], r_cur.v[k], a_rr);
                }
                qv.st(qo + (long long)(m0 + t) * ms);
            }
            mdown = mup;
        } else if (t == -1) {
            if (act && m0 - 1 >= 0) mdown.ld(stage_arr<T, 2>(smem, b, A_GY) + j * PY + cx);
        }
        pm1 = p0;
        p0 = pn;
        h0l = h1l;
        h0r = h1r;
        r_cur = r_next;
      }
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&empty[b])) : "memory");
    }
    acc[0] = a_pq;
    acc[1] = a_rq;
    acc[2] = a_qq;
    acc[3] = a_rr;
}

// ------------------------------------------------------------------ kernel
template <typename T, int NDIM>
__global__ void __launch_bounds__(NTH, 1)
sweep_kernel(const SweepInst *__restrict__ insts, const SweepSeg *__restrict__ segs,
             const int *__restrict__ cta_begin) {
    using C = SW<T, NDIM>;
    constexpr int V = C::V, VT = C::VT, HH = C::HH, S = C::S;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + S;
    __shared__ T s_red[NCW][4];
    __shared__ int s_last, s_err;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sb = cta_begin[blockIdx.x], se = cta_begin[blockIdx.x + 1];
    if (threadIdx.x == 0) {
        for (int i = 0; i < S; i++) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], NCW);
        }
        mbar_fence_init();
        s_err = 0;
    }
    __syncthreads();

    if (warp == NCW) {
        // ---------------- producer warp ----------------
        long long G = 0;
        uint32_t lim = WAIT_LIMIT;
        for (int si = sb; si < se; si++) {
            const SweepSeg sg = segs[si];
            const SweepInst &I = insts[sg.inst];
            if (inst_stopped(I)) continue;
            const SegView sv = seg_view<T, NDIM>(sg, I);
            const Geom g = I.g;
            ProdSeg<T> ps;
            const long long o0 = NDIM == 2 ? g.pad + sv.x0 : g.pad + sv.x0 + (long long)g.px * sv.y0;
            ps.r = (const T *)(sv.odd ? I.r[1] : I.r[0]) + o0 - V;
            ps.q = (const T *)(sv.odd ? I.q[1] : I.q[0]) + o0 - V;
            ps.p = (const T *)(sv.odd ? I.p[1] : I.p[0]) + o0 - V;
            ps.y = (const T *)I.y + o0;
            ps.gx = (const T *)I.gs[0] + o0 - V;
            ps.gy = (const T *)I.gs[1] + o0;
            ps.gz = (const T *)I.gs[2] + o0;
            ps.ms = NDIM == 2 ? (long long)g.px : g.plane;
            ps.rs = g.px;
            ps.nm = march_extent<NDIM>(g);
            ps.m0 = sv.m0;
            ps.m1 = sv.m1;
            ps.w = sv.w;
            ps.h = sv.h;
            ps.px = g.px;
            ps.full = NDIM == 3 && sv.x0 == 0 && sv.w == g.px;
            ps.first = sv.first;
            const bool fullrow = sv.x0 == 0 && sv.w == g.px;
            const int R = NDIM == 2 ? rows_per_stage_2d<T>(sv.w, g.px, fullrow) : 1;
            const int L = sv.m1 - sv.m0;
            for (int t = -2; t < L; t += R, G++) {
                const int b = (int)(G % S);
                if (G >= S) {
                    bool ok = true;
                    if (lane == 0) ok = mbar_wait_bounded(&empty[b], (uint32_t)((G / S) - 1) & 1u, lim);
                    ok = __shfl_sync(0xffffffffu, ok, 0);
                    if (!ok) lim = WAIT_LIMIT_AFTER_ERROR;
                    fence_proxy_async_smem();
                }
                if constexpr (NDIM == 2)
                    produce_stage_2d<T>(smem, full, b, ps, t, min(R, L - t), fullrow, lane);
                else
                    produce_step<T, NDIM>(smem, full, b, ps, t, lane);
            }
        }
        return;
    }

    // ---------------- consumer warps ----------------
    const int c = threadIdx.x;
    long long G = 0;
    uint32_t lim = WAIT_LIMIT;
    for (int si = sb; si < se; si++) {
        const SweepSeg sg = segs[si];
        const SweepInst &I = insts[sg.inst];
        if (inst_stopped(I)) continue;
        T v4[4];
        if constexpr (NDIM == 2) {
            consume_segment_2d<T>(smem, full, empty, I, sg, G, lim, &s_err, v4);
        } else {
        const SegView sv = seg_view<T, NDIM>(sg, I);
        const int px = I.g.px, ny = I.g.ny;
        const int nm = march_extent<NDIM>(I.g);
        const long long ms = NDIM == 2 ? (long long)px : I.g.plane;
        const T alpha = (T)I.s->alpha, beta = (T)I.s->beta;
        const bool first = sv.first;
        const int w = sv.w, h = sv.h, nv = sv.nv;
        // whole-row patches are staged as contiguous runs (row pitch px, the
        // halo columns are the neighbouring rows' ends, whose bonds are 0)
        const bool fullw = NDIM == 3 && sv.x0 == 0 && w == px;
        const int PW = fullw ? px : w + 2 * V;
        const int GXW = fullw ? px : w + V;
        const bool own = c < sv.nitems;
        const int rr = own ? c / nv : 0, vv = own ? c % nv : 0;
        // this thread's element at march index m is base + m * ms
        const long long base = I.g.pad + sv.x0 + vv * VT + (NDIM == 3 ? (long long)px * (sv.y0 + rr) : 0);
        T *ro = (T *)(sv.odd ? I.r[0] : I.r[1]) + base;
        T *po = (T *)(sv.odd ? I.p[0] : I.p[1]) + base;
        T *qo = (T *)(sv.odd ? I.q[0] : I.q[1]) + base;
        T *yv = (T *)I.y + base;
        const int o_own = (rr + HH) * PW + V + vv * VT;  // ring / r q p offset
        const int o_y = rr * w + vv * VT;
        const int o_gx = rr * GXW + V + vv * VT;
        const int o_gz = rr * w + vv * VT;
        const int y0 = sv.y0, x0 = sv.x0;
        V8<T> r_next, r_cur, mdown;
        r_next.zero();
        r_cur.zero();
        mdown.zero();
        T a_pq = T(0), a_rq = T(0), a_qq = T(0), a_rr = T(0);

        for (int t = -2; t < sv.m1 - sv.m0; t++, G++) {
            const int b = (int)(G % S);
            if (!mbar_wait_bounded(&full[b], (uint32_t)(G / S) & 1u, lim)) {
                s_err = 1;
                lim = WAIT_LIMIT_AFTER_ERROR;
            }
            const int me = sv.m0 + t + 1;
            T *ring = ring_slot<T, NDIM>(smem, G);
            const T *sr = stage_arr<T, NDIM>(smem, b, A_R);
            const T *sq = stage_arr<T, NDIM>(smem, b, A_Q);
            const T *sp = stage_arr<T, NDIM>(smem, b, A_P);
            // ---- finish iteration k-1 on march index me ----
            if (me >= 0 && me < nm) {
                const bool ownme = me >= sv.m0 && me < sv.m1;
                if (own) {
                    const int o = o_own;
                    V8<T> rv, pn;
                    rv.ld(sr + o);
                    if (first) {
                        r_next = rv;
                        pn = rv;
                    } else {
                        V8<T> qv, pv;
                        qv.ld(sq + o);
                        pv.ld(sp + o);
#pragma unroll
                        for (int k = 0; k < VT; k++) {
                            r_next.v[k] = rnew(rv.v[k], qv.v[k], alpha);
                            pn.v[k] = pnew(r_next.v[k], pv.v[k], beta);
                        }
                    }
                    pn.st(ring + o);
                    if (ownme) {
                        const long long i = (long long)me * ms;
                        r_next.st(ro + i);
                        pn.st(po + i);
                        V8<T> yn;
                        if (first) {
                            yn.zero();
                        } else {
                            V8<T> pv;
                            pv.ld(sp + o);
                            yn.ld(stage_arr<T, NDIM>(smem, b, A_Y) + o_y);
#pragma unroll
                            for (int k = 0; k < VT; k++) yn.v[k] = fma(alpha, pv.v[k], yn.v[k]);
                        }
                        yn.st(yv + i);
                    }
                }
                if (NDIM == 3) {  // halo rows y0-1 and y0+h: p only
                    for (int j = c; j < 2 * nv; j += NC) {
                        const int hr = j < nv ? -1 : h, hv = j % nv;
                        const int o = (hr + HH) * PW + V + hv * VT;
                        const int yrow = y0 + hr;
                        V8<T> pn;
                        if (yrow >= 0 && yrow < ny) {
                            V8<T> rv;
                            rv.ld(sr + o);
                            if (first) {
                                pn = rv;
                            } else {
                                V8<T> qv, pv;
                                qv.ld(sq + o);
                                pv.ld(sp + o);
#pragma unroll
                                for (int k = 0; k < VT; k++) pn.v[k] = pnew(rnew(rv.v[k], qv.v[k], alpha), pv.v[k], beta);
                            }
                        } else {
                            pn.zero();
                        }
                        pn.st(ring + o);
                    }
                }
                for (int j = c; !fullw && j < 2 * h; j += NC) {  // halo columns x0-1, x0+w
                    const int side = j & 1, hr = j >> 1;
                    const int col = side ? w : -1, x = x0 + col;
                    const int o = (hr + HH) * PW + V + col;
                    T pn = T(0);
                    if (x >= 0 && x < px)
                        pn = first ? sr[o] : pnew(rnew(sr[o], sq[o], alpha), sp[o], beta);
                    ring[o] = pn;
                }
            } else {
                if (own) {
                    V8<T> z;
                    z.zero();
                    z.st(ring + o_own);
                }
                if (NDIM == 3)
                    for (int j = c; j < 2 * nv; j += NC) {
                        V8<T> z;
                        z.zero();
                        z.st(ring + ((j < nv ? -1 : h) + HH) * PW + V + (j % nv) * VT);
                    }
                for (int j = c; !fullw && j < 2 * h; j += NC) ring[((j >> 1) + HH) * PW + V + ((j & 1) ? w : -1)] = T(0);
                r_next.zero();
            }
            cons_sync();
            // ---- stencil on march index m = m0 + t ----
            if (t >= 0) {
                const T *rc = ring_slot<T, NDIM>(smem, G - 1);
                const T *rup = ring_slot<T, NDIM>(smem, G);
                const T *rdn = ring_slot<T, NDIM>(smem, G - 2);
                const int o = o_own;
                V8<T> pc, pu, pd, gx, mup;
                pc.zero();
                gx.zero();
                if (own) {
                    pc.ld(rc + o);
                    gx.ld(stage_arr<T, NDIM>(smem, b, A_GX) + o_gx);
                }
                // x neighbours: shuffles within a row, shared memory at the edges
                T left = __shfl_up_sync(0xffffffffu, pc.v[VT - 1], 1);
                T right = __shfl_down_sync(0xffffffffu, pc.v[0], 1);
                T gxm = __shfl_up_sync(0xffffffffu, gx.v[VT - 1], 1);
                if (own) {
                    if (lane == 0 || vv == 0) {
                        left = rc[o - 1];
                        gxm = stage_arr<T, NDIM>(smem, b, A_GX)[o_gx - 1];
                    }
                    if (lane == 31 || vv == nv - 1) right = rc[o + VT];
                    pu.ld(rup + o);
                    pd.ld(rdn + o);
                    if (NDIM == 2) mup.ld(stage_arr<T, NDIM>(smem, b, A_GY) + vv * VT);
                    else mup.ld(stage_arr<T, NDIM>(smem, b, A_GZ) + o_gz);
                    V8<T> yu, yd, gyu, gyd, qv;
                    if (NDIM == 3) {
                        yu.ld(rc + o + PW);
                        yd.ld(rc + o - PW);
                        gyu.ld(stage_arr<T, NDIM>(smem, b, A_GY) + (rr + 1) * w + vv * VT);
                        gyd.ld(stage_arr<T, NDIM>(smem, b, A_GY) + rr * w + vv * VT);
                    }
#pragma unroll
                    for (int k = 0; k < VT; k++) {
                        const T lv = k == 0 ? left : pc.v[k - 1];
                        const T rv = k == VT - 1 ? right : pc.v[k + 1];
                        const T gl = k == 0 ? gxm : gx.v[k - 1];
                        T nb = gl * lv;
                        nb = fma(gx.v[k], rv, nb);
                        nb = fma(mdown.v[k], pd.v[k], nb);
                        nb = fma(mup.v[k], pu.v[k], nb);
                        if (NDIM == 3) {
                            nb = fma(gyd.v[k], yd.v[k], nb);
                            nb = fma(gyu.v[k], yu.v[k], nb);
                        }
                        const T qk = pc.v[k] - nb;
                        qv.v[k] = qk;
                        a_pq = fma(pc.v[k], qk, a_pq);
                        a_rq = fma(r_cur.v[k], qk, a_rq);
                        a_qq = fma(qk, qk, a_qq);
                        a_rr = fma(r_cur.v[k], r_cur.v[k], a_rr);
                    }
                    qv.st(qo + (long long)(sv.m0 + t) * ms);
                    mdown = mup;
                }
            } else if (t == -1 && own) {
                const int mt = sv.m0 - 1;
                if (mt >= 0) {
                    if (NDIM == 2) mdown.ld(stage_arr<T, NDIM>(smem, b, A_GY) + vv * VT);
                    else mdown.ld(stage_arr<T, NDIM>(smem, b, A_GZ) + o_gz);
                }
            }
            r_cur = r_next;
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&empty[b])) : "memory");
        }

        v4[0] = a_pq;
        v4[1] = a_rq;
        v4[2] = a_qq;
        v4[3] = a_rr;
        }
        // ---- segment sums -> the network's slot; last arrival finishes ----
        // Sums stay in T up to the warp; warp 0 combines the warps in a fixed
        // tree (FP32 path: into a float-float pair) -- GB300's FP64 rate makes
        // every FP64 instruction here cost ~64 cycles -- and the network's
        // last segment sums the slots in one warp.
#pragma unroll
        for (int k = 0; k < 4; k++)
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v4[k] += __shfl_xor_sync(0xffffffffu, v4[k], off);
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < 4; k++) s_red[warp][k] = v4[k];
        cons_sync();
        if (warp == 0) {
            typename std::conditional<sizeof(T) == 4, ff, double>::type t[4];
            warp_sum_rows<NCW>(s_red, t);
            if (lane == 0) {
                if (s_err) atomicExch(&I.s->err, 1);
                store_slot(I.part, sg.slot, t, s_err != 0);
                __threadfence();
                const unsigned int n = atomicAdd(&I.s->counter, 1u);
                s_last = (n == (unsigned)I.nseg - 1);
            }
        }
        cons_sync();
        if (s_last && warp == 0) {
            __threadfence();
            double tot[4];
            sum_slots(I.part, I.nseg, tot, T(0));
            if (lane == 0) {
                I.s->counter = 0u;
                finish_iteration(I.s, I.s->iter, tot);
            }
        }
        cons_sync();  // s_red / s_last reused by the next segment
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
int sweep_max_width(int ndim, int f32) {
    if (ndim == 2) return f32 ? SW<float, 2>::WMAX : SW<double, 2>::WMAX;
    return f32 ? SW<float, 3>::WMAX : SW<double, 3>::WMAX;
}
int sweep_vt(int f32) { return f32 ? 2 : 1; }
int sweep_rows_per_stage(int ndim, int f32, int w, int px, int x0) {
    if (ndim != 2) return 1;
    const bool fullrow = x0 == 0 && w == px;
    return f32 ? rows_per_stage_2d<float>(w, px, fullrow) : rows_per_stage_2d<double>(w, px, fullrow);
}
bool sweep_patch_fits(int f32, int w, int h) {
    const long long es = f32 ? 4 : 8, V = 16 / es;
    const long long need = (long long)(h + 2) * (w + 2 * V) * es;
    return need <= (f32 ? SW<float, 3>::SLOT : SW<double, 3>::SLOT);
}
int sweep_consumers() { return NC; }

cudaError_t sweep_prepare(int ndim, int f32) {
    if (ndim == 2)
        return f32 ? cudaFuncSetAttribute(sweep_kernel<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, SW<float, 2>::BYTES)
                   : cudaFuncSetAttribute(sweep_kernel<double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, SW<double, 2>::BYTES);
    return f32 ? cudaFuncSetAttribute(sweep_kernel<float, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, SW<float, 3>::BYTES)
               : cudaFuncSetAttribute(sweep_kernel<double, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, SW<double, 3>::BYTES);
}

cudaError_t launch_sweep(int ndim, int f32, int grid, const SweepInst *insts, const SweepSeg *segs,
                         const int *cta_begin, cudaStream_t st) {
    if (ndim == 2) {
        if (f32) sweep_kernel<float, 2><<<grid, NTH, SW<float, 2>::BYTES, st>>>(insts, segs, cta_begin);
        else sweep_kernel<double, 2><<<grid, NTH, SW<double, 2>::BYTES, st>>>(insts, segs, cta_begin);
    } else {
        if (f32) sweep_kernel<float, 3><<<grid, NTH, SW<float, 3>::BYTES, st>>>(insts, segs, cta_begin);
        else sweep_kernel<double, 3><<<grid, NTH, SW<double, 3>::BYTES, st>>>(insts, segs, cta_begin);
    }
    return cudaGetLastError();
}

}  // namespace netsolve
