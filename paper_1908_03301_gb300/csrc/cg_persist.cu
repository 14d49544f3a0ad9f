// cg_persist.cu -- the whole inner CG solve of a 2D network in one launch.
//
// The arithmetic is that of the fused iteration (Sec. IV; see kernels_cg.cu):
// sweep k finishes iteration k-1 (r, p, y), applies the scaled 5-point
// operator (q = A p) and forms <p,q>, <r,q>, <q,q>, <r,r>, from which alpha_k
// and beta_k follow.  Organisation for GB300:
//  * cooperative launch, one CTA per SM; CTA c owns full-width rows
//    [row0, row1) for the whole solve;
//  * y, r, p, q are updated in place (one copy each), so a 2048^2 network
//    (about 100 MB with its two bond planes) can stay in the 126 MB L2;
//  * a CTA reads no row another CTA writes during the same sweep: while it
//    marches, each CTA copies r, p and q of its first and last rows into a
//    halo buffer indexed by sweep parity; in the next sweep the neighbours
//    fetch those rows and rebuild p there themselves;
//  * a producer warp streams the CTA's rows through a TMA (cp.async.bulk)
//    pipeline and starts the next sweep's rows before the grid barrier,
//    then waits for the barrier itself and starts the next sweep's halo
//    copies while warp 0 sums the partials;
//    16 consumer warps own column strips and keep the march neighbours in
//    registers, meeting only at the pipeline's mbarriers;
//  * one grid barrier per sweep (arrivals counted, every CTA polls the
//    count); afterwards every CTA sums all CTAs' partials in the same fixed
//    order and advances its own copy of the CG state -- identical everywhere.
//    The sums and the state are float-float pairs (ffloat.cuh): GB300's FP64
//    rate would put microseconds of FP64 on every sweep's critical path.
//    CTA 0 writes the final state back.
// Every wait is bounded; a wait that gives up ends the solve with stop code
// 5 and sets *err.
#include <cfloat>
#include <cmath>

#include "ffloat.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace netsolve {
namespace {

constexpr int NC = 512;
constexpr int NCW = NC / 32;
constexpr int NTH = NC + 32;
constexpr int VT = 4;                  // floats per consumer thread
constexpr int WMAX = NC * VT;          // widest row (2048 floats)
constexpr int S = 3;                   // row-pipeline stages
constexpr int ROWB = WMAX * 4;         // bytes per staged row
constexpr int NARR = 6;                // r q p y gx gy
constexpr int BAR = 128;
constexpr int HALO = S * NARR * ROWB;  // offset of the halo rows (after BAR)
constexpr int SMEM = BAR + HALO + 6 * ROWB;
constexpr uint32_t WAIT_LIMIT = 1u << 22;
static_assert(SMEM <= 227 * 1024, "shared memory");

enum { A_R = 0, A_Q = 1, A_P = 2, A_Y = 3, A_GX = 4, A_GY = 5 };
// halo buffer rows per (parity, CTA, edge): r, q, p
enum { H_R = 0, H_Q = 1, H_P = 2 };

__device__ __forceinline__ float *stg(unsigned char *smem, int b, int a) {
    return reinterpret_cast<float *>(smem + BAR + (b * NARR + a) * ROWB);
}
// top (e = 0) and bottom (e = 1) halo rows r, q, p
__device__ __forceinline__ float *hrow(unsigned char *smem, int e, int a) {
    return reinterpret_cast<float *>(smem + BAR + HALO + (e * 3 + a) * ROWB);
}


__device__ __forceinline__ float rnew(float r, float q, float a) { return fmaf(-a, q, r); }
__device__ __forceinline__ float pnew(float rn, float p, float b) { return fmaf(b, p, rn); }

struct F4 {
    float v[4];
    __device__ __forceinline__ void ld(const float *p) {
        float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
    __device__ __forceinline__ void st(float *p) const {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
    __device__ __forceinline__ void zero() { v[0] = v[1] = v[2] = v[3] = 0.f; }
    __device__ __forceinline__ void st_keep(float *p, uint64_t pol) const {
        st_hint_f4(p, v[0], v[1], v[2], v[3], pol);
    }
};

// halo buffer row (parity, cta, edge, array) in global memory
__device__ __forceinline__ float *hb_row(const PersistArgs &a, int par, int cta, int e, int arr,
                                         int G, int px) {
    return a.hb + ((((long long)par * G + cta) * 2 + e) * 3 + arr) * px;
}

// Producer: issue the row stage of step t (t = -1 .. n-1) of a sweep.  The
// vectors y, r, p, q are read and written every iteration (67 MB at 2048^2):
// they are loaded and stored with an evict-last L2 policy, which keeps them in
// the persisting part of L2 that the host sets aside for the solve; the bond
// planes (read only) stream.  With a periodic y axis the bond row below row 0
// is the wrap row ny-1.
__device__ __forceinline__ void issue_row_stage(unsigned char *smem, uint64_t *full, int b, int t,
                                                int row0, int row1, int px, bool first,
                                                const PersistArgs &a, int lane, uint64_t pol) {
    const uint32_t rb = (uint32_t)px * 4u;
    const bool wrap = a.g.periodic(1);
    const int me = row0 + t + 1, mt = row0 + t >= 0 ? row0 + t : a.g.ny - 1;
    const int nl = me < row1 ? (first ? 1 : 4) : 0;                   // r [q p y] of row me
    const int nb = (row0 + t >= 0 || wrap) ? (t >= 0 ? 2 : 1) : 0;  // [gx] gy of row mt
    if (lane == 0) mbar_arrive_expect_tx(&full[b], (uint32_t)(nl + nb) * rb);
    __syncwarp();
    const long long base = a.g.pad;
    if (lane < nl) {
        const float *src = lane == 0 ? a.r : (lane == 1 ? a.q : (lane == 2 ? a.p : a.y));
        bulk_load_hint(stg(smem, b, lane), src + base + (long long)me * px, rb, &full[b], pol);
    } else if (lane >= 8 && lane < 8 + nb) {
        const int which = nb == 1 ? A_GY : (lane == 8 ? A_GX : A_GY);
        bulk_load(stg(smem, b, which), (which == A_GX ? a.gx : a.gy) + base + (long long)mt * px, rb,
                  &full[b]);
    }
}

__global__ void __launch_bounds__(NTH, 1) cg_persist_kernel(PersistArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + S;
    uint64_t *hfull = empty + S;  // halo rows of the current sweep
    __shared__ InnerScal st;
    __shared__ InnerScalF sf;  // the running state, as pairs
    __shared__ float s_red[NCW][4];
    __shared__ int s_bad;

    const int G = gridDim.x, c = blockIdx.x;
    const int px = a.g.px, ny = a.g.ny;
    const bool wrap = a.g.periodic(1);  // periodic y: row ny-1 joins row 0
    const int row0 = (int)((long long)c * ny / G), row1 = (int)((long long)(c + 1) * ny / G);
    const int n = row1 - row0;  // >= 1
    const int steps = n + 1;    // row stages per sweep: t = -1 .. n-1
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long base = a.g.pad;

    if (threadIdx.x == 0) {
        for (int i = 0; i < S; i++) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], NCW);
        }
        mbar_init(hfull, 1);
        mbar_fence_init();
        st = *a.s;
        scal_to_ff(st, sf);
        s_bad = 0;
    }
    __syncthreads();

    const uint64_t keep = l2_policy_keep();
    // producer state
    long long P_step = 0;  // row stages issued (all sweeps)
    int pre = 0;           // stages of the coming sweep already issued
    uint32_t plim = WAIT_LIMIT;
    // consumer state
    long long C_step = 0;
    uint32_t clim = WAIT_LIMIT;

    auto producer_issue = [&](int t, bool first) {
        const int b = (int)(P_step % S);
        if (P_step >= S) {
            bool ok = true;
            if (lane == 0) ok = mbar_wait_bounded(&empty[b], (uint32_t)((P_step / S) - 1) & 1u, plim);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) plim = 1024;
            fence_proxy_async_smem();
        }
        issue_row_stage(smem, full, b, t, row0, row1, px, first, a, lane, keep);
        P_step++;
    };

    if (warp == NCW) {  // first sweep's leading stages
        asm volatile("fence.proxy.async.global;" ::: "memory");
        const bool first = st.iter == 0;
        if (!st.stop)
            for (; pre < S && pre < steps; pre++) producer_issue(pre - 1, first);
    }

    // Halo rows of a sweep (producer lane 0): r (first sweep: from the
    // vectors, whose values the first sweep leaves unchanged) or r, q, p
    // copied by the neighbours during the previous sweep (parity ppar_).
    // Neighbours across a periodic y boundary: the last CTA's last row above
    // row 0, the first CTA's first row below ny-1.
    auto issue_halo = [&](bool first_, int ppar_) {
        const uint32_t rb = (uint32_t)px * 4u;
        const bool top = c > 0 || wrap, bot = c + 1 < G || wrap;
        const int ct = c > 0 ? c - 1 : G - 1, cb = c + 1 < G ? c + 1 : 0;
        const int rt = row0 > 0 ? row0 - 1 : ny - 1, rbm = row1 < ny ? row1 : 0;
        const uint32_t per = first_ ? rb : 3u * rb;
        mbar_arrive_expect_tx(hfull, (top ? per : 0u) + (bot ? per : 0u));
        if (first_) {
            if (top) bulk_load(hrow(smem, 0, H_R), a.r + base + (long long)rt * px, rb, hfull);
            if (bot) bulk_load(hrow(smem, 1, H_R), a.r + base + (long long)rbm * px, rb, hfull);
        } else {
            for (int arr = 0; arr < 3; arr++) {
                if (top) bulk_load(hrow(smem, 0, arr), hb_row(a, ppar_, ct, 1, arr, G, px), rb, hfull);
                if (bot) bulk_load(hrow(smem, 1, arr), hb_row(a, ppar_, cb, 0, arr, G, px), rb, hfull);
            }
        }
    };
    bool halo_early = false;  // the next sweep's halo copies are already in flight
    unsigned goal = 0;  // arrivals the next grid barrier waits for
    int sweep = 0;
    for (;; sweep++) {
        if (sf.stop) break;
        const bool first = sf.iter == 0;
        const float alpha = sf.alpha.h, beta = sf.beta.h;
        const int par = sweep & 1, ppar = par ^ 1;

        if (warp == NCW) {
            // ---------------- producer ----------------
            asm volatile("fence.proxy.async.global;" ::: "memory");
            // halo rows of this sweep, unless already issued right after the
            // last grid barrier
            if (lane == 0 && !halo_early) issue_halo(first, ppar);
            halo_early = false;
            __syncwarp();
            for (; pre < steps; pre++) producer_issue(pre - 1, first);
            pre = 0;
        } else {
            // ---------------- consumers ----------------
            const int cx = threadIdx.x * VT;
            const bool act = cx < px;
            const bool edge_l = lane == 0 && cx > 0 && act;
            const bool edge_r = lane == 31 && cx + VT < px;
            F4 pm1, p0, pn, r_cur, r_next, mdown;
            pm1.zero(); p0.zero(); r_cur.zero(); r_next.zero(); mdown.zero();
            float h0l = 0.f, h0r = 0.f;
            float a_pq = 0.f, a_rq = 0.f, a_qq = 0.f, a_rr = 0.f;
            if (!mbar_wait_bounded(hfull, (uint32_t)sweep & 1u, clim)) {
                s_bad = 1;
                clim = 1024;
            }
            // p of row row0-1 from the top halo rows
            pn.zero();
            if ((c > 0 || wrap) && act) {
                F4 rv;
                rv.ld(hrow(smem, 0, H_R) + cx);
                if (first) {
                    pn = rv;
                } else {
                    F4 qv, pv;
                    qv.ld(hrow(smem, 0, H_Q) + cx);
                    pv.ld(hrow(smem, 0, H_P) + cx);
#pragma unroll
                    for (int k = 0; k < VT; k++) pn.v[k] = pnew(rnew(rv.v[k], qv.v[k], alpha), pv.v[k], beta);
                }
            }
            p0 = pn;
            for (int t = -1; t < n; t++, C_step++) {
                const int b = (int)(C_step % S);
                if (!mbar_wait_bounded(&full[b], (uint32_t)(C_step / S) & 1u, clim)) {
                    s_bad = 1;
                    clim = 1024;
                }
                const int me = row0 + t + 1;
                pn.zero();
                float h1l = 0.f, h1r = 0.f;
                if (me < row1) {
                    const float *sr = stg(smem, b, A_R), *sq = stg(smem, b, A_Q), *sp = stg(smem, b, A_P);
                    if (act) {
                        F4 rv;
                        rv.ld(sr + cx);
                        const long long i = base + (long long)me * px + cx;
                        if (first) {
                            r_next = rv;
                            pn = rv;
                            F4 z;
                            z.zero();
                            z.st_keep(a.y + i, keep);
                        } else {
                            F4 qv, pv, yv;
                            qv.ld(sq + cx);
                            pv.ld(sp + cx);
                            yv.ld(stg(smem, b, A_Y) + cx);
#pragma unroll
                            for (int k = 0; k < VT; k++) {
                                r_next.v[k] = rnew(rv.v[k], qv.v[k], alpha);
                                pn.v[k] = pnew(r_next.v[k], pv.v[k], beta);
                                yv.v[k] = fmaf(alpha, pv.v[k], yv.v[k]);
                            }
                            yv.st_keep(a.y + i, keep);
                        }
                        r_next.st_keep(a.r + i, keep);
                        pn.st_keep(a.p + i, keep);
                        if (me == row0) {
                            r_next.st(hb_row(a, par, c, 0, H_R, G, px) + cx);
                            pn.st(hb_row(a, par, c, 0, H_P, G, px) + cx);
                        }
                        if (me == row1 - 1) {
                            r_next.st(hb_row(a, par, c, 1, H_R, G, px) + cx);
                            pn.st(hb_row(a, par, c, 1, H_P, G, px) + cx);
                        }
                    }
                    if (edge_l) {
                        const int j = cx - 1;
                        h1l = first ? sr[j] : pnew(rnew(sr[j], sq[j], alpha), sp[j], beta);
                    }
                    if (edge_r) {
                        const int j = cx + VT;
                        h1r = first ? sr[j] : pnew(rnew(sr[j], sq[j], alpha), sp[j], beta);
                    }
                } else {
                    // me == row1: p of the first row of the CTA below
                    r_next.zero();
                    if ((c + 1 < G || wrap) && act) {
                        F4 rv;
                        rv.ld(hrow(smem, 1, H_R) + cx);
                        if (first) {
                            pn = rv;
                        } else {
                            F4 qv, pv;
                            qv.ld(hrow(smem, 1, H_Q) + cx);
                            pv.ld(hrow(smem, 1, H_P) + cx);
#pragma unroll
                            for (int k = 0; k < VT; k++) pn.v[k] = pnew(rnew(rv.v[k], qv.v[k], alpha), pv.v[k], beta);
                        }
                    }
                }
                if (t >= 0) {
                    // stencil on row mt = row0 + t
                    const int mt = row0 + t;
                    F4 gx, gy, qv;
                    gx.zero();
                    gy.zero();
                    if (act) {
                        gx.ld(stg(smem, b, A_GX) + cx);
                        gy.ld(stg(smem, b, A_GY) + cx);
                    }
                    float left = __shfl_up_sync(0xffffffffu, p0.v[VT - 1], 1);
                    float right = __shfl_down_sync(0xffffffffu, p0.v[0], 1);
                    float gxm = __shfl_up_sync(0xffffffffu, gx.v[VT - 1], 1);
                    if (lane == 0) {
                        left = h0l;
                        gxm = edge_l ? stg(smem, b, A_GX)[cx - 1] : 0.f;
                    }
                    if (lane == 31) right = h0r;
                    if (act) {
#pragma unroll
                        for (int k = 0; k < VT; k++) {
                            const float lv = k == 0 ? left : p0.v[k - 1];
                            const float rv = k == VT - 1 ? right : p0.v[k + 1];
                            const float gl = k == 0 ? gxm : gx.v[k - 1];
                            float nb = gl * lv;
                            nb = fmaf(gx.v[k], rv, nb);
                            nb = fmaf(mdown.v[k], pm1.v[k], nb);
                            nb = fmaf(gy.v[k], pn.v[k], nb);
                            const float qk = p0.v[k] - nb;
                            qv.v[k] = qk;
                            a_pq = fmaf(p0.v[k], qk, a_pq);
                            a_rq = fmaf(r_cur.v[k], qk, a_rq);
                            a_qq = fmaf(qk, qk, a_qq);
                            a_rr = fmaf(r_cur.v[k], r_cur.v[k], a_rr);
                        }
                        qv.st_keep(a.q + base + (long long)mt * px + cx, keep);
                        if (mt == row0) qv.st(hb_row(a, par, c, 0, H_Q, G, px) + cx);
                        if (mt == row1 - 1) qv.st(hb_row(a, par, c, 1, H_Q, G, px) + cx);
                    }
                    mdown = gy;
                } else if (act && (row0 - 1 >= 0 || wrap)) {
                    // t == -1: bond row row0-1 (ny-1 across a periodic
                    // boundary) gives the down bonds of row0
                    mdown.ld(stg(smem, b, A_GY) + cx);
                }
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&empty[b])) : "memory");
                pm1 = p0;
                p0 = pn;
                h0l = h1l;
                h0r = h1r;
                r_cur = r_next;
            }
            // this CTA's sums: FP32 within each warp, then a float-float pair
            float v4[4] = {a_pq, a_rq, a_qq, a_rr};
#pragma unroll
            for (int k = 0; k < 4; k++)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v4[k] += __shfl_xor_sync(0xffffffffu, v4[k], o);
            if (lane == 0)
#pragma unroll
                for (int k = 0; k < 4; k++) s_red[warp][k] = v4[k];
            asm volatile("bar.sync 1, %0;" ::"n"(NC) : "memory");
            if (threadIdx.x == 0) {
                ff tot[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
                for (int wi = 0; wi < NCW; wi++)
#pragma unroll
                    for (int k = 0; k < 4; k++) tot[k] = ff_add_f(tot[k], s_red[wi][k]);
                if (s_bad) tot[3] = {NAN, 0.f};
                float4 *dst = reinterpret_cast<float4 *>(a.pb) + 2 * ((long long)par * G + c);
                dst[0] = make_float4(tot[0].h, tot[1].h, tot[2].h, tot[3].h);
                dst[1] = make_float4(tot[0].l, tot[1].l, tot[2].l, tot[3].l);
            }
        }
        __syncthreads();  // A: this CTA's rows, halo copies and sums are written
        goal += (unsigned)G;
        if (warp == NCW) {
            // start the next sweep's own rows (written by this CTA itself);
            // if the solve stops instead, they are drained below
            asm volatile("fence.proxy.async.global;" ::: "memory");
            for (; pre < S && pre < steps; pre++) producer_issue(pre - 1, false);
            // then wait for the grid barrier too and start the next sweep's
            // halo copies (the neighbours' edge rows of this sweep): their
            // addresses do not depend on the CG scalars, so their latency
            // overlaps warp 0's reduction and scalar step instead of
            // following it.  Drained below if the solve stops instead.
            int early = 0;
            if (lane == 0 && wait_count(a.bar_count, goal, a.wait_ns)) {
                asm volatile("fence.proxy.async.global;" ::: "memory");
                fence_proxy_async_smem();
                issue_halo(false, par);
                early = 1;
            }
            halo_early = __shfl_sync(0xffffffffu, early, 0) != 0;
        } else if (warp == 0) {
            // grid barrier (a CTA told to withhold its first arrival, for
            // tests of the bounded wait, does not arrive), then this CTA's own
            // sum of all partials and its own step of the CG state
            int ok = 0;
            if (lane == 0) {
                __threadfence();
                if (!(sweep == 0 && c == a.skip_cta)) arrive_release(a.bar_count);
                if (s_bad) atomicExch(a.err, 1);
                ok = wait_count(a.bar_count, goal, a.wait_ns);
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (ok) {
                ff tot[4];
                warp_sum_pairs(reinterpret_cast<const float4 *>(a.pb) + 2LL * par * G, G, tot);
                if (lane == 0) {
                    sf.err = 0;
                    finish_iteration_ff(&sf, sf.iter, tot);
                }
            } else if (lane == 0) {
                atomicExch(a.err, 1);
                sf.stop = 5;
            }
        }
        __syncthreads();  // C
    }
    if (warp == NCW) {
        // drain stages and halo copies issued for a sweep that did not run
        for (long long k = P_step - pre; k < P_step; k++)
            mbar_wait_bounded(&full[(int)(k % S)], (uint32_t)(k / S) & 1u, plim);
        if (halo_early) mbar_wait_bounded(hfull, (uint32_t)sweep & 1u, plim);
    }
    if (c == 0 && threadIdx.x == 0) {
        InnerScal out = st;
        if (sweep > 0) scal_from_ff(sf, out);  // untouched when no sweep ran
        out.counter = 0u;
        *a.s = out;
    }
}

// A launch that continues the recursion (iter > 0 after a refinement pass)
// starts with a non-first sweep, which reads its neighbours' edge rows of r,
// q, p from the halo copies of parity 1.  The refinement pass replaced r, so
// those copies are rewritten from the vectors here (one CTA per persistent
// CTA, same row partition).
__global__ void persist_resume_kernel(PersistArgs a) {
    if (a.s->iter == 0) return;
    const int G = gridDim.x, c = blockIdx.x;
    const int px = a.g.px, ny = a.g.ny;
    const int row0 = (int)((long long)c * ny / G), row1 = (int)((long long)(c + 1) * ny / G);
    const long long base = a.g.pad;
    const float *src[3];
    src[H_R] = a.r;
    src[H_Q] = a.q;
    src[H_P] = a.p;
    for (int e = 0; e < 2; e++) {
        const long long row = e == 0 ? row0 : row1 - 1;
        for (int arr = 0; arr < 3; arr++) {
            const float *from = src[arr] + base + row * px;
            float *to = hb_row(a, 1, c, e, arr, G, px);
            for (int i = threadIdx.x; i < px; i += blockDim.x) to[i] = from[i];
        }
    }
}

}  // namespace

cudaError_t launch_persist_resume(const PersistArgs &a, int grid, cudaStream_t st) {
    persist_resume_kernel<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

bool persist_applies(const Geom &g, int f32) {
    return f32 && g.ndim == 2 && g.px <= WMAX && g.ny >= 2;
}

int persist_grid(const Geom &g) {
    static int nsm = 0;
    if (!nsm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (nsm <= 0) nsm = 1;
    }
    return nsm < g.ny ? nsm : g.ny;
}

cudaError_t persist_prepare() {
    return cudaFuncSetAttribute(cg_persist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
}

cudaError_t launch_persist(const PersistArgs &a, int grid, cudaStream_t st) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cg_persist_kernel, NTH, SMEM);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    e = cudaMemsetAsync(a.bar_count, 0, sizeof(unsigned), st);  // arrivals
    if (e == cudaSuccess) e = cudaMemsetAsync(a.err, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    PersistArgs arg = a;
    void *params[] = {&arg};
    return cudaLaunchCooperativeKernel((const void *)cg_persist_kernel, dim3(grid), dim3(NTH), params,
                                       SMEM, st);
}

}  // namespace netsolve
