// ffloat.cuh -- float-float ("double-word") scalars for the per-iteration
// work of the FP32 inner CG loops.
//
// GB300 runs FP64 at a small fraction of its FP32 rate: one FP64 warp
// instruction occupies the pipe for about 64 cycles whatever its active
// lanes, so a one-thread update of the CG scalars in FP64 (two divisions)
// costs ~2 300 cycles and one thread summing 16 warps' FP32 sums into FP64
// ~8 700 cycles.  The FP32 inner loops therefore keep their reductions and
// scalar updates in pairs of FP32 numbers (hi + lo, |lo| <= ulp(hi) / 2):
// about 48 significant bits, far more than the FP32 vectors the sums come
// from, at FP32 issue rates (~600 cycles for the update).
//
// The building blocks are the classical error-free transformations:
//   two_sum       Knuth's TwoSum (The Art of Computer Programming, vol. 2,
//                 sec. 4.2.2): s + e == a + b exactly, any a, b;
//   fast_two_sum  Dekker's Fast2Sum (Numer. Math. 18, 1971): the same for
//                 |a| >= |b|;
//   two_prod      the exact product error through one FMA (as in Ogita, Rump
//                 and Oishi, SIAM J. Sci. Comput. 26, 2005).
// Sum, product and quotient of two pairs follow the usual double-word
// constructions (Joldes, Muller and Popescu, ACM TOMS 44, 2017: the
// "accurate" sum, a product with the cross terms folded into the error, a
// quotient refined by one Newton-like correction).  Every operation is an
// explicitly rounded intrinsic so that no contraction or reassociation can
// change the results: every CTA that runs the same sequence on the same
// inputs gets the same bits.
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace netsolve {

struct ff {
    float h, l;
};

__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    ff s = two_sum(a.h, b.h);
    const ff t = two_sum(a.l, b.l);
    s = fast_two_sum(s.h, __fadd_rn(s.l, t.h));
    return fast_two_sum(s.h, __fadd_rn(s.l, t.l));
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.h, -a.l}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }
// Accumulate one FP32 value: the pair stays normalised.
__device__ __forceinline__ ff ff_add_f(ff a, float b) {
    const ff s = two_sum(a.h, b);
    return fast_two_sum(s.h, __fadd_rn(s.l, a.l));
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ ff ff_div(ff a, ff b) {
    const float q1 = __fdiv_rn(a.h, b.h);
    const ff r = ff_sub(a, ff_mul({q1, 0.f}, b));
    const float q2 = __fdiv_rn(r.h, b.h);
    return fast_two_sum(q1, q2);
}
// Exact scaling by 2 (no rounding for normal numbers).
__device__ __forceinline__ ff ff_twice(ff a) { return {__fmul_rn(2.f, a.h), __fmul_rn(2.f, a.l)}; }
__device__ __forceinline__ bool ff_le(ff a, ff b) { return a.h < b.h || (a.h == b.h && a.l <= b.l); }
__device__ __forceinline__ bool ff_lt(ff a, ff b) { return a.h < b.h || (a.h == b.h && a.l < b.l); }
__device__ __forceinline__ ff ff_of(double d) {
    const float h = __double2float_rn(d);
    return {h, isfinite(h) ? __double2float_rn(d - (double)h) : 0.f};
}
__device__ __forceinline__ double ff_to_double(ff a) { return isfinite(a.h) ? (double)a.h + (double)a.l : (double)a.h; }

// Sum of G per-CTA pairs of four sums by one warp: pair i is the float4s
// {hi[4]} at part[2 i] and {lo[4]} at part[2 i + 1].  Lane-strided, DEPTH
// CTAs per lane in flight (5: a grid of one CTA per SM, 152, is read in one
// round of loads), then a butterfly; the same inputs give the same bits in
// every lane and every CTA.
template <int PAIR_DEPTH = 4>
__device__ __forceinline__ void warp_sum_pairs(const float4 *part, int G, ff (&tot)[4]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < 4; k++) tot[k] = {0.f, 0.f};
    for (int i0 = lane; i0 < G; i0 += 32 * PAIR_DEPTH) {
        float4 h[PAIR_DEPTH], l[PAIR_DEPTH];
#pragma unroll
        for (int m = 0; m < PAIR_DEPTH; m++) {
            const int i = i0 + 32 * m;
            h[m] = i < G ? __ldcg(part + 2 * i) : make_float4(0.f, 0.f, 0.f, 0.f);
            l[m] = i < G ? __ldcg(part + 2 * i + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int m = 0; m < PAIR_DEPTH; m++) {
            tot[0] = ff_add(tot[0], {h[m].x, l[m].x});
            tot[1] = ff_add(tot[1], {h[m].y, l[m].y});
            tot[2] = ff_add(tot[2], {h[m].z, l[m].z});
            tot[3] = ff_add(tot[3], {h[m].w, l[m].w});
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < 4; k++)
            tot[k] = ff_add(tot[k], {__shfl_xor_sync(0xffffffffu, tot[k].h, o), __shfl_xor_sync(0xffffffffu, tot[k].l, o)});
}

// The four sums of NR rows (one row per warp of a CTA), combined by one warp
// in a fixed tree: FP32 rows into pairs, FP64 rows in FP64.  NR is a power of
// two <= 32; every lane ends with the same result.
template <int NR>
__device__ __forceinline__ void warp_sum_rows(const float (*rows)[4], ff (&t)[4]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < 4; k++) t[k] = {rows[lane & (NR - 1)][k], 0.f};
#pragma unroll
    for (int o = NR / 2; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < 4; k++)
            t[k] = ff_add(t[k], {__shfl_xor_sync(0xffffffffu, t[k].h, o), __shfl_xor_sync(0xffffffffu, t[k].l, o)});
}
template <int NR>
__device__ __forceinline__ void warp_sum_rows(const double (*rows)[4], double (&t)[4]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < 4; k++) t[k] = rows[lane & (NR - 1)][k];
#pragma unroll
    for (int o = NR / 2; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < 4; k++) t[k] += __shfl_xor_sync(0xffffffffu, t[k], o);
}

// Per-segment slots of the batched kernels: 32 bytes each, four FP64 sums or
// (FP32 path) one pair {hi[4]}, {lo[4]} of float4s.  `zero`: store zeros.
__device__ __forceinline__ void store_slot(double *part, long long slot, const ff (&t)[4], bool zero) {
    float4 *d = reinterpret_cast<float4 *>(part) + 2 * slot;
    d[0] = zero ? make_float4(0.f, 0.f, 0.f, 0.f) : make_float4(t[0].h, t[1].h, t[2].h, t[3].h);
    d[1] = zero ? make_float4(0.f, 0.f, 0.f, 0.f) : make_float4(t[0].l, t[1].l, t[2].l, t[3].l);
}
__device__ __forceinline__ void store_slot(double *part, long long slot, const double (&t)[4], bool zero) {
#pragma unroll
    for (int k = 0; k < 4; k++) part[slot * 4 + k] = zero ? 0.0 : t[k];
}
// A network's total over its nseg slots, by one warp, as FP64 for
// finish_iteration (the FP32 path sums the pairs and converts the four
// totals once).
__device__ __forceinline__ void sum_slots(const double *part, int nseg, double (&tot)[4], float /*FP32 path*/) {
    ff t[4];
    warp_sum_pairs(reinterpret_cast<const float4 *>(part), nseg, t);
#pragma unroll
    for (int k = 0; k < 4; k++) tot[k] = ff_to_double(t[k]);
}
__device__ __forceinline__ void sum_slots(const double *part, int nseg, double (&tot)[4], double /*FP64 path*/) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < 4; k++) tot[k] = 0.0;
    for (int i = lane; i < nseg; i += 32)
#pragma unroll
        for (int k = 0; k < 4; k++) tot[k] += __ldcg(part + (long long)i * 4 + k);
#pragma unroll
    for (int k = 0; k < 4; k++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tot[k] += __shfl_xor_sync(0xffffffffu, tot[k], o);
}

// The floating fields of InnerScal that one CG iteration reads and writes,
// as pairs; thr = tol2 * rho0 (fixed while a launch runs).
struct InnerScalF {
    ff alpha, beta, rho, best, maxrr, thr, delta2;
    long long best_iter, iter, max_iter, stag_window;
    int stop, err, reliable;
};

__device__ __forceinline__ void scal_to_ff(const InnerScal &s, InnerScalF &f) {
    f.alpha = ff_of(s.alpha);
    f.beta = ff_of(s.beta);
    f.rho = ff_of(s.rho);
    f.best = ff_of(s.best);
    f.maxrr = ff_of(s.maxrr);
    f.thr = ff_of(s.tol2 * s.rho0);
    f.delta2 = ff_of(s.delta2);
    f.best_iter = s.best_iter;
    f.iter = s.iter;
    f.max_iter = s.max_iter;
    f.stag_window = s.stag_window;
    f.stop = s.stop;
    f.err = s.err;
    f.reliable = s.reliable;
}
__device__ __forceinline__ void scal_from_ff(const InnerScalF &f, InnerScal &s) {
    s.alpha = ff_to_double(f.alpha);
    s.beta = ff_to_double(f.beta);
    s.rho = ff_to_double(f.rho);
    s.best = ff_to_double(f.best);
    s.maxrr = ff_to_double(f.maxrr);
    s.best_iter = f.best_iter;
    s.iter = f.iter;
    s.stop = f.stop;
    s.err = f.err;
}

// finish_iteration (common.cuh) in float-float: the same tests in the same
// order on v = {<p,q>, <r,q>, <q,q>, <r,r>} of iteration k.
__device__ __forceinline__ void finish_iteration_ff(InnerScalF *s, long long k, const ff (&v)[4]) {
    const ff pq = v[0], rq = v[1], qq = v[2], rr = v[3];
    s->rho = rr;
    s->iter = k + 1;
    if (s->err) {
        s->stop = 5;
        return;
    }
    if (rr.h == 0.f || (!s->reliable && ff_le(rr, s->thr))) {
        s->stop = 1;
        return;
    }
    if (!(pq.h > 0.f) || !isfinite(pq.h) || !isfinite(rr.h)) {
        s->stop = 4;
        return;
    }
    const ff a = ff_div(rr, pq);
    ff rn1 = ff_add(ff_sub(rr, ff_mul(ff_twice(a), rq)), ff_mul(ff_mul(a, a), qq));
    if (!(rn1.h > 0.f)) rn1 = {0.f, 0.f};  // cancellation: restart along the residual
    s->alpha = a;
    s->beta = ff_div(rn1, rr);
    if (s->reliable) {
        if (ff_lt(s->maxrr, rr)) s->maxrr = rr;
        if (ff_le(rn1, s->thr) || ff_le(rn1, ff_mul(s->delta2, s->maxrr))) {
            s->stop = 6;
            return;
        }
    }
    if (ff_lt(rr, {__fmul_rn(0.25f, s->best.h), __fmul_rn(0.25f, s->best.l)})) {
        s->best = rr;
        s->best_iter = k;
    }
    if (k + 1 >= s->max_iter) s->stop = 2;
    else if (k - s->best_iter > s->stag_window) s->stop = 3;
}

}  // namespace netsolve
