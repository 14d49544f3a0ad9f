// kernels_march.cu -- the 2D CG iteration as a persistent row march.
//
// Same arithmetic as inner_iter_kernel (one launch = one CG iteration of
// Sec. IV on the scaled system; see kernels_cg.cu), organised for HBM:
//   * one CTA per SM; CTA c owns a column block [x0, x0+w) (w <= W) and a
//     contiguous run of rows [row0, row1) of the padded grid, so every SM
//     gets the same amount of work and there is no partial last wave;
//   * the CTA walks its rows top to bottom.  Step s finishes iteration k-1
//     on row row0+s+1 (r, p, y updates; p also on the two halo columns) into
//     a 4-slot shared ring of p rows, then applies the stencil to row row0+s,
//     whose up / down neighbours are ring rows - each row of r, q, p is read
//     once, plus one halo row above and below the run;
//   * the row data arrive by 1D bulk copies (TMA, cp.async.bulk) into an
//     S-stage shared-memory pipeline issued S-1 steps ahead by one thread and
//     completed on mbarriers, so about (S-1) x 25 KB are in flight per SM.
// Stage for step s: r, q, p (with V halo elements each side) and y of row
// row0+s+1, gx (with V left halo) and gy of row row0+s.  The down bonds
// gy(row-1) are kept in registers from the previous step.
#include <cfloat>
#include <cmath>

#include "kernels.h"
#include "tma.cuh"

namespace netsolve {
namespace {

constexpr int NT = 256;
constexpr int S = 6;                   // pipeline stages
constexpr uint32_t WAIT_LIMIT = 1u << 22;

template <typename T> struct MarchW;
template <> struct MarchW<float> { static constexpr int W = 1024; };
template <> struct MarchW<double> { static constexpr int W = 512; };

template <typename T>
struct Layout {
    static constexpr int V = Vec<T>::N;     // elements per 16 bytes
    static constexpr int W = MarchW<T>::W;  // widest column block
    static constexpr int SLOT = ((W + 2 * V) * (int)sizeof(T) + 127) / 128 * 128;  // bytes
    static constexpr int STAGE = 6 * SLOT;  // r q p gx y gy
    static constexpr int BAR = 128;         // mbarriers
    static constexpr int RING = 4 * SLOT;
    static constexpr int BYTES = BAR + S * STAGE + RING;
    static_assert(W / V == NT, "one vector per thread per row");
};

template <typename T>
__device__ __forceinline__ T *slot_ptr(unsigned char *smem, int stage, int arr) {
    using L = Layout<T>;
    return reinterpret_cast<T *>(smem + L::BAR + stage * L::STAGE + arr * L::SLOT);
}
template <typename T>
__device__ __forceinline__ T *ring_ptr(unsigned char *smem, int row) {
    using L = Layout<T>;
    return reinterpret_cast<T *>(smem + L::BAR + S * L::STAGE + ((row + 4) & 3) * L::SLOT);
}

enum { A_R = 0, A_Q = 1, A_P = 2, A_GX = 3, A_Y = 4, A_GY = 5 };

template <typename T>
__device__ __forceinline__ T rnew(T r, T q, T a) { return fma(-a, q, r); }
template <typename T>
__device__ __forceinline__ T pnew(T rn, T p, T b) { return fma(b, p, rn); }

struct Plan {
    int kb;  // column blocks
    int rb;  // row blocks
};

// Issue the bulk copies of step t (rows row0+t+1 and row0+t) into its stage.
template <typename T>
__device__ void issue_step(unsigned char *smem, uint64_t *bars, const Geom &g, int t, int row0,
                           int row1, int x0, int w, const T *r, const T *q, const T *p,
                           const T *y, const T *g0, const T *g1) {
    using L = Layout<T>;
    constexpr int V = L::V;
    const int b = (t + 2) % S;
    const int lr = row0 + t + 1;  // elementwise row
    const int br = row0 + t;      // stencil / bond row
    uint32_t bytes = 0;
    const uint32_t wide = (uint32_t)(w + 2 * V) * sizeof(T);
    const uint32_t gxb = (uint32_t)(w + V) * sizeof(T);
    const uint32_t nb = (uint32_t)w * sizeof(T);
    const bool ld_l = lr >= 0 && lr < g.ny;
    const bool ld_y = lr >= row0 && lr < row1;
    const bool ld_b = t >= -1 && br >= 0 && br < g.ny;
    if (ld_l) bytes += 3 * wide;
    if (ld_y) bytes += nb;
    if (ld_b) bytes += gxb + nb;
    mbar_arrive_expect_tx(&bars[b], bytes);
    if (ld_l) {
        const long long o = g.idx(x0 - V, lr, 0);
        bulk_load(slot_ptr<T>(smem, b, A_R), r + o, wide, &bars[b]);
        bulk_load(slot_ptr<T>(smem, b, A_Q), q + o, wide, &bars[b]);
        bulk_load(slot_ptr<T>(smem, b, A_P), p + o, wide, &bars[b]);
    }
    if (ld_y) bulk_load(slot_ptr<T>(smem, b, A_Y), y + g.idx(x0, lr, 0), nb, &bars[b]);
    if (ld_b) {
        bulk_load(slot_ptr<T>(smem, b, A_GX), g0 + g.idx(x0 - V, br, 0), gxb, &bars[b]);
        bulk_load(slot_ptr<T>(smem, b, A_GY), g1 + g.idx(x0, br, 0), nb, &bars[b]);
    }
}

template <typename T>
__global__ void __launch_bounds__(NT, 1)
march2d_kernel(Geom g, Plan plan, const T *__restrict__ g0, const T *__restrict__ g1,
               T *__restrict__ y, T *r0, T *r1, T *p0, T *p1, T *q0, T *q1, InnerScal *s,
               double *partials) {
    using L = Layout<T>;
    constexpr int V = L::V;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    __shared__ int s_err;

    if (*(volatile int *)&s->stop) return;
    const long long iter = s->iter;
    const bool first = iter == 0;
    const T alpha = (T)s->alpha, beta = (T)s->beta;
    const bool odd = iter & 1;
    const T *__restrict__ r = odd ? r1 : r0;
    const T *__restrict__ p = odd ? p1 : p0;
    const T *__restrict__ q = odd ? q1 : q0;
    T *__restrict__ ro = odd ? r0 : r1;
    T *__restrict__ po = odd ? p0 : p1;
    T *__restrict__ qo = odd ? q0 : q1;

    const int cb = blockIdx.x % plan.kb, rb = blockIdx.x / plan.kb;
    const int x0 = cb * L::W;
    const int w = min(L::W, g.px - x0);
    const int row0 = (int)((long long)rb * g.ny / plan.rb);
    const int row1 = (int)((long long)(rb + 1) * g.ny / plan.rb);
    const int nrows = row1 - row0;
    const int tid = threadIdx.x;
    const bool act = tid * V < w;  // this thread's vector lies in the block

    int last_issued = -3, last_waited = -3;  // meaningful in thread 0
    if (tid == 0) {
        s_err = 0;
        for (int i = 0; i < S; i++) mbar_init(&bars[i], 1);
        mbar_fence_init();
        for (int t = -2; t <= min(S - 3, nrows - 1); t++) {
            issue_step<T>(smem, bars, g, t, row0, row1, x0, w, r, q, p, y, g0, g1);
            last_issued = t;
        }
    }
    __syncthreads();

    Vec<T> r_next, r_cur, gy_prev;
    r_next.zero();
    r_cur.zero();
    gy_prev.zero();
    T a_pq = T(0), a_rq = T(0), a_qq = T(0), a_rr = T(0);

    for (int st = -2; st <= nrows - 1; st++) {
        const int b = (st + 2) % S;
        const uint32_t par = (uint32_t)((st + 2) / S) & 1u;
        if (!mbar_wait_bounded(&bars[b], par, WAIT_LIMIT)) s_err = 1;
        else last_waited = st;
        const int lr = row0 + st + 1;
        T *ring_l = ring_ptr<T>(smem, st + 1);
        // ---- finish iteration k-1 on row lr, stage p -----------------------
        if (lr >= 0 && lr < g.ny) {
            const T *sr = slot_ptr<T>(smem, b, A_R);
            const T *sq = slot_ptr<T>(smem, b, A_Q);
            const T *sp = slot_ptr<T>(smem, b, A_P);
            const bool own = lr >= row0 && lr < row1;
            if (act) {
                Vec<T> rv, pn;
                rv.load(sr + V + tid * V);
                if (first) {
                    r_next = rv;
                    pn = rv;
                } else {
                    Vec<T> qv, pv;
                    qv.load(sq + V + tid * V);
                    pv.load(sp + V + tid * V);
#pragma unroll
                    for (int k = 0; k < V; k++) {
                        r_next.v[k] = rnew(rv.v[k], qv.v[k], alpha);
                        pn.v[k] = pnew(r_next.v[k], pv.v[k], beta);
                    }
                }
                pn.store(ring_l + V + tid * V);
                if (own) {
                    const long long i = g.idx(x0 + tid * V, lr, 0);
                    r_next.store(ro + i);
                    pn.store(po + i);
                    Vec<T> yv;
                    if (first) {
                        yv.zero();
                    } else {
                        Vec<T> pv;
                        pv.load(sp + V + tid * V);
                        yv.load(slot_ptr<T>(smem, b, A_Y) + tid * V);
#pragma unroll
                        for (int k = 0; k < V; k++) yv.v[k] = fma(alpha, pv.v[k], yv.v[k]);
                    }
                    yv.store(y + i);
                }
            }
            if (tid < 2) {  // halo columns x0-1 and x0+w
                const int c = tid == 0 ? V - 1 : V + w;
                ring_l[c] = first ? sr[c] : pnew(rnew(sr[c], sq[c], alpha), sp[c], beta);
            }
        } else {
            Vec<T> z;
            z.zero();
            if (act) z.store(ring_l + V + tid * V);
            if (tid < 2) ring_l[tid == 0 ? V - 1 : V + w] = T(0);
            r_next.zero();
        }
        __syncthreads();
        if (s_err) break;
        if (tid == 0 && st >= -1 && st + S - 1 <= nrows - 1) {
            fence_proxy_async_smem();
            issue_step<T>(smem, bars, g, st + S - 1, row0, row1, x0, w, r, q, p, y, g0, g1);
            last_issued = st + S - 1;
        }
        // ---- stencil on row row0+st --------------------------------------
        if (st >= 0 && act) {
            const T *pc_row = ring_ptr<T>(smem, st) + V + tid * V;
            const T *pu_row = ring_ptr<T>(smem, st + 1) + V + tid * V;
            const T *pd_row = ring_ptr<T>(smem, st - 1) + V + tid * V;
            const T *sgx = slot_ptr<T>(smem, b, A_GX) + V + tid * V;
            Vec<T> pc, pu, pd, gx, gy, qv;
            pc.load(pc_row);
            pu.load(pu_row);
            pd.load(pd_row);
            gx.load(sgx);
            gy.load(slot_ptr<T>(smem, b, A_GY) + tid * V);
            const T pl = pc_row[-1], pr = pc_row[V], gxm = sgx[-1];
#pragma unroll
            for (int k = 0; k < V; k++) {
                const T left = k == 0 ? pl : pc.v[k - 1];
                const T right = k == V - 1 ? pr : pc.v[k + 1];
                const T gl = k == 0 ? gxm : gx.v[k - 1];
                T nb = gl * left;
                nb = fma(gx.v[k], right, nb);
                nb = fma(gy_prev.v[k], pd.v[k], nb);
                nb = fma(gy.v[k], pu.v[k], nb);
                const T qk = pc.v[k] - nb;
                qv.v[k] = qk;
                a_pq = fma(pc.v[k], qk, a_pq);
                a_rq = fma(r_cur.v[k], qk, a_rq);
                a_qq = fma(qk, qk, a_qq);
                a_rr = fma(r_cur.v[k], r_cur.v[k], a_rr);
            }
            qv.store(qo + g.idx(x0 + tid * V, row0 + st, 0));
            gy_prev = gy;
        } else if (st == -1 && act) {
            const int br = row0 - 1;
            if (br >= 0) gy_prev.load(slot_ptr<T>(smem, b, A_GY) + tid * V);
        }
        r_cur = r_next;
    }
    if (s_err) {
        // drain: wait (bounded) for every copy this CTA issued and has not
        // consumed, then report through the iteration scalars
        if (tid == 0) {
            s->err = 1;
            for (int t = max(-2, last_waited + 1); t <= last_issued; t++)
                mbar_wait_bounded(&bars[(t + 2) % S], (uint32_t)((t + 2) / S) & 1u, WAIT_LIMIT);
        }
        a_pq = a_rq = a_qq = a_rr = T(0);
    }

    double v[4] = {(double)a_pq, (double)a_rq, (double)a_qq, (double)a_rr};
    const int ops[4] = {RED_SUM, RED_SUM, RED_SUM, RED_SUM};
    if (!grid_reduce<4, NT>(v, ops, partials, &s->counter)) return;
    if (threadIdx.x == 0) finish_iteration(s, iter, v);
}

}  // namespace

bool march_applies(const Geom &g) {
    return g.ndim == 2 && (long long)g.px * g.ny >= (1LL << 18);
}

static int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 152;
    }
    return n;
}

template <typename T>
static Plan make_plan(const Geom &g) {
    Plan pl;
    pl.kb = (g.px + MarchW<T>::W - 1) / MarchW<T>::W;
    pl.rb = sm_count() / pl.kb;
    if (pl.rb < 1) pl.rb = 1;
    if (pl.rb > g.ny) pl.rb = g.ny;
    return pl;
}

int march_blocks(const Geom &g, int f32) {
    const Plan pl = f32 ? make_plan<float>(g) : make_plan<double>(g);
    return pl.kb * pl.rb;
}

cudaError_t march_prepare(int f32) {
    if (f32)
        return cudaFuncSetAttribute(march2d_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    Layout<float>::BYTES);
    return cudaFuncSetAttribute(march2d_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                Layout<double>::BYTES);
}

template <typename T>
static cudaError_t launch_march_t(const InnerArgs &a, cudaStream_t st) {
    const Plan pl = make_plan<T>(a.g);
    march2d_kernel<T><<<pl.kb * pl.rb, NT, Layout<T>::BYTES, st>>>(
        a.g, pl, (const T *)a.gs[0], (const T *)a.gs[1], (T *)a.y, (T *)a.r[0], (T *)a.r[1],
        (T *)a.p[0], (T *)a.p[1], (T *)a.q[0], (T *)a.q[1], a.s, a.partials);
    return cudaGetLastError();
}

cudaError_t launch_march(const InnerArgs &a, int f32, cudaStream_t st) {
    return f32 ? launch_march_t<float>(a, st) : launch_march_t<double>(a, st);
}

}  // namespace netsolve
