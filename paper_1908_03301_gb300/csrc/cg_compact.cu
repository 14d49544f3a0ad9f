// cg_compact.cu -- the inner CG solve over a compacted list of unknowns.
//
// Near the percolation threshold the unknowns of the linear system (the
// spanning clusters less their dead-end trees) are a small part of the
// lattice: 13 % of a 256^3 network at p = 0.26.  A sweep over the lattice
// then moves mostly zeros.  Here the unknowns are listed row by row (in 3D,
// rows in blocks of 8 x 8; see lattice_index);
// each keeps its scaled bonds to the +e_d neighbours and the list indices of
// its y and z neighbours (x neighbours are the adjacent list entries); the
// table is stored direction-major, so a warp reads consecutive entries, and
// y, r, p, q are compact vectors.
//
// One cooperative launch runs a whole inner solve.  Iteration k (the same
// arithmetic as the lattice kernels, Sec. IV):
//   phase A, every unknown:  r -= alpha q;  y += alpha p;  p = r + beta p
//                            (iteration 0: p = r, y = 0)
//   grid barrier
//   phase B, every unknown:  q = p - sum_j ghat_j p_j  and the sums
//                            <p,q>, <r,q>, <q,q>, <r,r>
//   grid barrier; then every CTA sums all CTAs' partials in CTA order in
//   FP64 and advances its own copy of the CG state (finish_iteration): the
//   same inputs in the same order give the same state everywhere, with no
//   record to publish and read back.
// A thread owns the same unknowns in both phases and in every iteration, so
// its own entries need no cross-SM visibility; neighbours' p written by other
// CTAs are read through L2 (ld.global.cg).  Every wait is bounded.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "kernels.h"

namespace netsolve {
namespace {

constexpr int CT = 512;                 // threads per CTA (batched phases)
constexpr int CW = CT / 32;
constexpr int CTC = 512;                // threads per CTA of the cooperative solve (two per SM: one
constexpr int CWC = CTC / 32;           //   1024-thread CTA per SM measured slower, 28.7 against 26.5 us)
constexpr int UNR = 2;                  // unknowns a thread keeps in flight (FP64)
constexpr int UNR32 = 2;                // the same in FP32
constexpr int SCAN_CHUNK = 4096;        // lattice nodes per block in the compaction scan

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Order of the listed unknowns: whole padded rows (so the +x neighbour of an
// unknown, if listed, is the next entry), the rows of a 3D network taken in
// blocks of 8 x 8 (y, z) rows.  A z neighbour is then a few rows away in the
// list (8 inside a block) instead of a whole plane, so the gathers of the
// operator mostly stay within the lines a CTA reads anyway.  Scan position t
// in [0, px * ny * nz) -> padded lattice index; a bijection.
constexpr long long ROW_BY = 8, ROW_BZ = 8;
__device__ __forceinline__ long long lattice_index(const Geom &g, long long t) {
    if (g.ndim < 3) return g.pad + t;
    const long long rho = t / g.px;
    const int x = (int)(t - rho * g.px);
    const long long ny = g.ny, nz = g.nz;
    const long long zb = rho / (ROW_BZ * ny);
    const long long hz = nz - zb * ROW_BZ < ROW_BZ ? nz - zb * ROW_BZ : ROW_BZ;
    const long long r1 = rho - zb * ROW_BZ * ny;
    const long long yb = r1 / (hz * ROW_BY);
    const long long hy = ny - yb * ROW_BY < ROW_BY ? ny - yb * ROW_BY : ROW_BY;
    const long long r2 = r1 - yb * hz * ROW_BY;
    const long long zz = r2 / hy, yy = r2 - zz * hy;
    return g.idx(x, (int)(yb * ROW_BY + yy), (int)(zb * ROW_BZ + zz));
}

// ------------------------------------------------------------------ build
// Unknowns per chunk of the lattice.
__global__ void compact_count_kernel(Geom g, const uint8_t *__restrict__ cls, unsigned int *counts) {
    __shared__ unsigned int s;
    if (threadIdx.x == 0) s = 0;
    __syncthreads();
    const long long n = (long long)g.px * g.ny * g.nz;
    const long long t0 = (long long)blockIdx.x * SCAN_CHUNK;
    unsigned int mine = 0;
    for (int j = threadIdx.x; j < SCAN_CHUNK; j += blockDim.x) {
        const long long t = t0 + j;
        if (t < n && cls[lattice_index(g, t)] == CLS_SPANNING) mine++;
    }
    atomicAdd(&s, mine);
    __syncthreads();
    if (threadIdx.x == 0) counts[blockIdx.x] = s;
}

// List index of every unknown, in lattice order: block b starts at
// offsets[b]; inside a chunk, thread j takes nodes [8j, 8j+8) and a block
// scan orders the threads.  cmap[i] = list index or -1; cidx[k] = node.
__global__ void compact_index_kernel(Geom g, const uint8_t *__restrict__ cls,
                                     const unsigned int *__restrict__ offsets, int *cmap, int *cidx) {
    constexpr int PER = SCAN_CHUNK / CT;  // 8
    __shared__ unsigned int warp_tot[CW];
    const long long n = (long long)g.px * g.ny * g.nz;
    const long long t0 = (long long)blockIdx.x * SCAN_CHUNK + (long long)threadIdx.x * PER;
    unsigned int flags = 0, cnt = 0;
    for (int j = 0; j < PER; j++) {
        const long long t = t0 + j;
        if (t < n && cls[lattice_index(g, t)] == CLS_SPANNING) {
            flags |= 1u << j;
            cnt++;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned int incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    unsigned int before = 0;
    for (int w = 0; w < warp; w++) before += warp_tot[w];
    unsigned int k = offsets[blockIdx.x] + before + incl - cnt;
    for (int j = 0; j < PER; j++) {
        const long long t = t0 + j;
        if (t >= n) break;
        const long long i = lattice_index(g, t);
        if (flags & (1u << j)) {
            cmap[i] = (int)k;
            cidx[k] = (int)i;
            k++;
        } else {
            cmap[i] = -1;
        }
    }
}

// ELL row of every unknown.  In list order (whole rows) an unknown's +x neighbour, if
// it is an unknown, is the next entry of the list, so x needs no index (x is
// never periodic).  The y and z neighbours follow periodic boundaries.
//   val[d][k]  (d < ndim, stride U + 1): scaled bond to the +e_d neighbour if
//              that node is an unknown, else 0 (val[d][U] = 0);
//   nbr[2(d-1)][k], nbr[2(d-1)+1][k]  (d >= 1, stride U): list index of the
//              +e_d / -e_d neighbour.  A missing +e_d neighbour is k itself
//              (its bond is 0); a missing -e_d neighbour is ~k (negative):
//              the -e_d bond is read from that neighbour's val[d] entry.
// The -x bond of k is val[0][k-1]: non-zero only if entry k-1 is the -x node.
template <typename T>
__global__ void compact_ell_kernel(Geom g, long long U, const int *__restrict__ cidx,
                                   const int *__restrict__ cmap, const T *gs0, const T *gs1, const T *gs2,
                                   int *nbr, T *val) {
    const T *gs[3] = {gs0, gs1, gs2};
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < U;
         k += (long long)gridDim.x * blockDim.x) {
        const long long i = cidx[k];
        // coordinates matter only across a periodic (y / z) boundary
        int c[3] = {0, 0, 0};
        if (g.per) {
            const long long t = i - g.pad, r = t / g.px;
            c[1] = (int)(r % g.ny);
            c[2] = (int)(r / g.ny);
        }
        for (int d = 0; d < g.ndim; d++) {
            const long long jp = d == 0 ? i + 1 : g.up(i, d, c[d]);
            const T gp = gs[d][i];
            const int mp = cmap[jp];
            const bool lp = mp >= 0 && gp != T(0);
            val[(long long)d * (U + 1) + k] = lp ? gp : T(0);
            if (d == 0) continue;
            const long long jm = g.down(i, d, c[d]);
            const T gm = gs[d][jm];
            const int mm = cmap[jm];
            const bool lm = mm >= 0 && gm != T(0);
            nbr[(long long)(2 * (d - 1)) * U + k] = lp ? mp : (int)k;
            nbr[(long long)(2 * (d - 1) + 1) * U + k] = lm ? mm : ~(int)k;
        }
    }
}

// ------------------------------------------------------------------ refinement glue
template <typename T>
__global__ void compact_gather_kernel(long long U, const int *__restrict__ cidx, const T *__restrict__ src,
                                      T *dst) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < U;
         k += (long long)gridDim.x * blockDim.x)
        dst[k] = src[cidx[k]];
}

// x += D^-1/2 y on the unknowns; a pass that ended with stop 6 still owes
// alpha_k p_k (the recursion continues): fold it in and clear y.
template <typename T>
__global__ void compact_correct_kernel(long long U, const int *__restrict__ cidx, const double *__restrict__ dis,
                                       double *x, T *y, const T *__restrict__ p, const InnerScal *is) {
    const bool owe = is->stop == 6;
    const double a = is->alpha;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < U;
         k += (long long)gridDim.x * blockDim.x) {
        double d = (double)y[k];
        if (owe) {
            d = fma(a, (double)p[k], d);
            y[k] = T(0);
        }
        const long long i = cidx[k];
        x[i] = fma(dis[i], d, x[i]);
    }
}

// ------------------------------------------------------------------ the solve
// Grid barrier part 1: every CTA's writes are done; thread 0 arrives.
// Returns (to all threads) whether this CTA arrived last at barrier `target`.
// `withhold`: for tests of the bounded wait, this CTA does not arrive.
__device__ __forceinline__ bool barrier_arrive(unsigned *count, unsigned target, int G, bool withhold) {
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (withhold) {
            s_last = 0;
        } else {
            const unsigned arrived = atomicAdd(count, 1u) + 1u;
            s_last = arrived == (unsigned)G * target;
        }
    }
    __syncthreads();
    return s_last != 0;
}
// Grid barrier part 2 for the CTAs that did not arrive last (thread 0 waits
// for the release); returns false if the wait gave up (after wait_ns of
// device time).
__device__ __forceinline__ bool barrier_wait(const unsigned *gen, unsigned target, unsigned long long wait_ns) {
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        // poll with relaxed loads (an acquire per poll would order, and slow,
        // the memory traffic of the other CTA on this SM), then one acquire
        bool ok = false;
        const unsigned long long t0 = globaltimer_ns();
        for (uint32_t i = 0;; i++) {
            if (ld_relaxed_u32(gen) >= target) {
                ok = ld_acquire_u32(gen) >= target;
                break;
            }
            if ((i & 255u) == 255u && globaltimer_ns() - t0 > wait_ns) break;
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}
__device__ __forceinline__ void barrier_release(unsigned *gen, unsigned target) {
    __threadfence();
    st_release_u32(gen, target);
}

// Phase A of iteration k on the list entries k = kb, kb + st, ... < ke:
// finish iteration k-1 (r -= alpha q; y += alpha p; p = r + beta p), or at
// the first iteration p = r, y = 0.  UN entries in flight per thread.
template <typename T, int UN>
__device__ __forceinline__ void compact_phase_a(T *__restrict__ y, T *__restrict__ r, T *p, const T *__restrict__ q,
                                                int kb, int ke, int st, T alpha, T beta, bool first) {
    for (int k0 = kb; k0 < ke; k0 += UN * st) {
        T rk[UN], pk[UN], qk[UN], yk[UN];
#pragma unroll
        for (int u = 0; u < UN; u++) {
            const int k = k0 + u * st;
            if (k < ke) {
                rk[u] = r[k];
                if (!first) {
                    pk[u] = p[k];
                    qk[u] = q[k];
                    yk[u] = y[k];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < UN; u++) {
            const int k = k0 + u * st;
            if (k >= ke) continue;
            if (first) {
                p[k] = rk[u];
                y[k] = T(0);
            } else {
                const T rn = fma(-alpha, qk[u], rk[u]);
                r[k] = rn;
                y[k] = fma(alpha, pk[u], yk[u]);
                p[k] = fma(beta, pk[u], rn);
            }
        }
    }
}

// Phase B on the entries k = kb, kb + st, ... < ke of a list of U unknowns:
// q = A p (neighbours' p read through L2) and this thread's share of
// <p,q>, <r,q>, <q,q>, <r,r>.
template <typename T, int NDIM, int UN>
__device__ __forceinline__ void compact_phase_b(const T *__restrict__ r, const T *p, T *__restrict__ q,
                                                const T *__restrict__ val, const int *__restrict__ nbr, int U,
                                                int kb, int ke, int st, T &s_pq, T &s_rq, T &s_qq, T &s_rr) {
    const long long VS = U + 1;  // val slot stride
    for (int k0 = kb; k0 < ke; k0 += UN * st) {
        T wxp[UN], wxm[UN], wp[UN][NDIM - 1];
        int ip[UN][NDIM - 1], im[UN][NDIM - 1];
#pragma unroll
        for (int u = 0; u < UN; u++) {
            const int k = k0 + u * st;
            const bool ok = k < ke;
            const int kk = ok ? k : 0;
            wxp[u] = ok ? __ldg(val + kk) : T(0);
            wxm[u] = (ok && k > 0) ? __ldg(val + kk - 1) : T(0);
#pragma unroll
            for (int d = 1; d < NDIM; d++) {
                wp[u][d - 1] = ok ? __ldg(val + d * VS + kk) : T(0);
                ip[u][d - 1] = ok ? __ldg(nbr + (long long)(2 * (d - 1)) * U + kk) : (int)kk;
                im[u][d - 1] = ok ? __ldg(nbr + (long long)(2 * (d - 1) + 1) * U + kk) : ~(int)kk;
            }
        }
#pragma unroll
        for (int u = 0; u < UN; u++) {
            const int k = k0 + u * st;
            if (k >= ke) continue;
            const T pk = __ldcg(p + k);
            T nb = wxp[u] * __ldcg(p + k + 1);
            nb = fma(wxm[u], __ldcg(p + (k > 0 ? k - 1 : 0)), nb);
#pragma unroll
            for (int d = 1; d < NDIM; d++) {
                nb = fma(wp[u][d - 1], __ldcg(p + ip[u][d - 1]), nb);
                const int jm = im[u][d - 1];
                const int jj = jm >= 0 ? jm : ~jm;
                const T wm = jm >= 0 ? __ldg(val + d * VS + jj) : T(0);
                nb = fma(wm, __ldcg(p + jj), nb);
            }
            const T qk = pk - nb;
            q[k] = qk;
            const T rk = r[k];
            s_pq = fma(pk, qk, s_pq);
            s_rq = fma(rk, qk, s_rq);
            s_qq = fma(qk, qk, s_qq);
            s_rr = fma(rk, rk, s_rr);
        }
    }
}

template <typename T, int NDIM>
__global__ void __launch_bounds__(CTC, 2) compact_cg_kernel(CompactArgs a) {
    __shared__ InnerScal st;
    __shared__ T s_red[CWC][4];
    const int G = gridDim.x, c = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T *__restrict__ y = (T *)a.y;
    T *__restrict__ r = (T *)a.r;
    T *p = (T *)a.p;
    T *__restrict__ q = (T *)a.q;
    const T *__restrict__ val = (const T *)a.val;
    const int *__restrict__ nbr = a.nbr;
    unsigned *bar_count = a.bar, *bar_gen = a.bar + 1;
    if (threadIdx.x == 0) {
        const unsigned long long *src = reinterpret_cast<const unsigned long long *>(a.s);
        unsigned long long *dst = reinterpret_cast<unsigned long long *>(&st);
        for (int k = 0; k < (int)(sizeof(InnerScal) / 8); k++) dst[k] = src[k];
    }
    __syncthreads();
    // list indices fit in 32 bits (the table stores them as int)
    const int tid = c * CTC + (int)threadIdx.x, nth = G * CTC;
    const int U = (int)a.n;
    constexpr int UN = sizeof(T) == 4 ? UNR32 : UNR;
    unsigned target = 0;
    bool bad = false;
    while (st.stop == 0) {
        const bool first = st.iter == 0;
        const T alpha = (T)st.alpha, beta = (T)st.beta;
        // ---- phase A: finish iteration k-1 (UN unknowns in flight per thread) ----
        compact_phase_a<T, UN>(y, r, p, q, tid, U, nth, alpha, beta, first);
        ++target;
        if (barrier_arrive(bar_count, target, G, target == 1u && c == a.skip_cta)) {
            if (threadIdx.x == 0) barrier_release(bar_gen, target);
        } else if (!barrier_wait(bar_gen, target, a.wait_ns)) {
            bad = true;
        }
        __syncthreads();
        // ---- phase B: q = A p and the four sums ----
        T s_pq = T(0), s_rq = T(0), s_qq = T(0), s_rr = T(0);
        compact_phase_b<T, NDIM, UN>(r, p, q, val, nbr, U, tid, U, nth, s_pq, s_rq, s_qq, s_rr);
        T t4[4] = {s_pq, s_rq, s_qq, s_rr};
#pragma unroll
        for (int k = 0; k < 4; k++)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t4[k] += __shfl_xor_sync(0xffffffffu, t4[k], o);
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < 4; k++) s_red[warp][k] = t4[k];
        __syncthreads();
        const int par = (int)(st.iter & 1);
        if (threadIdx.x == 0) {
            double tot[4] = {0, 0, 0, 0};
            for (int w = 0; w < CWC; w++)
#pragma unroll
                for (int k = 0; k < 4; k++) tot[k] += (double)s_red[w][k];
            if (bad) tot[0] = tot[1] = tot[2] = tot[3] = NAN;
#pragma unroll
            for (int k = 0; k < 4; k++) a.pb[((long long)par * G + c) * 4 + k] = tot[k];
        }
        ++target;
        // grid barrier without a published state: after it every CTA sums all
        // CTAs' partials itself, in the same fixed order (FP64, one warp), and
        // advances its own copy of the CG state -- identical everywhere; one
        // fewer store and load on the critical path than a reduction by the
        // last CTA to arrive (7.7 against 8.8 us per barrier over 304 CTAs)
        bool ok = true, last = false;
        if (barrier_arrive(bar_count, target, G, false)) {
            last = true;
            if (threadIdx.x == 0) barrier_release(bar_gen, target);
        } else {
            ok = barrier_wait(bar_gen, target, a.wait_ns);
        }
        if (warp == 0 && ok) {
            if (last) __threadfence();  // the others' partials, seen through the arrival count
            double tot[4] = {0, 0, 0, 0};
            for (int i0 = lane; i0 < G; i0 += 128) {
                double v[4][4];
#pragma unroll
                for (int m = 0; m < 4; m++) {
                    const int i = i0 + 32 * m;
#pragma unroll
                    for (int k = 0; k < 4; k++) v[m][k] = i < G ? __ldcg(a.pb + ((long long)par * G + i) * 4 + k) : 0.0;
                }
#pragma unroll
                for (int m = 0; m < 4; m++)
#pragma unroll
                    for (int k = 0; k < 4; k++) tot[k] += v[m][k];
            }
#pragma unroll
            for (int k = 0; k < 4; k++)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) tot[k] += __shfl_xor_sync(0xffffffffu, tot[k], o);
            if (lane == 0) {
                st.err = 0;
                finish_iteration(&st, st.iter, tot);
            }
        }
        if (threadIdx.x == 0 && (bad || !ok)) {
            atomicExch(a.err, 1);
            st.stop = 5;
        }
        __syncthreads();
    }
    if (c == 0 && threadIdx.x == 0) {
        st.counter = 0u;
        const unsigned long long *src = reinterpret_cast<const unsigned long long *>(&st);
        unsigned long long *dst = reinterpret_cast<unsigned long long *>(a.s);
        for (int k = 0; k < (int)(sizeof(InnerScal) / 8); k++) dst[k] = src[k];
    }
}

// ------------------------------------------------------------------ batches
// Compacted networks inside a batch: one launch of each kernel per CG
// iteration for every running network of the group (the kernel boundary is
// the barrier between the phases), a network cut into segments of list
// entries, one segment per CTA.  A network's last segment to finish phase B
// sums the segments' partials in slot order (FP64) and runs finish_iteration,
// as the lattice sweep does; stopped networks are skipped.
template <typename T, int NDIM>
__global__ void __launch_bounds__(CT) compact_batch_a_kernel(const CompactInst *__restrict__ insts,
                                                             const CompactSeg *__restrict__ segs) {
    const CompactSeg sg = segs[blockIdx.x];
    const CompactInst &I = insts[sg.inst];
    const InnerScal *s = I.a.s;
    if (s->stop) return;
    constexpr int UN = sizeof(T) == 4 ? UNR32 : UNR;
    compact_phase_a<T, UN>((T *)I.a.y, (T *)I.a.r, (T *)I.a.p, (const T *)I.a.q, sg.u0 + (int)threadIdx.x, sg.u1,
                           CT, (T)s->alpha, (T)s->beta, s->iter == 0);
}

template <typename T, int NDIM>
__global__ void __launch_bounds__(CT) compact_batch_b_kernel(const CompactInst *__restrict__ insts,
                                                             const CompactSeg *__restrict__ segs) {
    __shared__ T s_red[CW][4];
    __shared__ int s_last;
    const CompactSeg sg = segs[blockIdx.x];
    const CompactInst &I = insts[sg.inst];
    InnerScal *s = I.a.s;
    if (s->stop) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int UN = sizeof(T) == 4 ? UNR32 : UNR;
    T s_pq = T(0), s_rq = T(0), s_qq = T(0), s_rr = T(0);
    compact_phase_b<T, NDIM, UN>((const T *)I.a.r, (const T *)I.a.p, (T *)I.a.q, (const T *)I.a.val, I.a.nbr,
                                 (int)I.a.n, sg.u0 + (int)threadIdx.x, sg.u1, CT, s_pq, s_rq, s_qq, s_rr);
    T t4[4] = {s_pq, s_rq, s_qq, s_rr};
#pragma unroll
    for (int k = 0; k < 4; k++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t4[k] += __shfl_xor_sync(0xffffffffu, t4[k], o);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 4; k++) s_red[warp][k] = t4[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot[4] = {0, 0, 0, 0};
        for (int w = 0; w < CW; w++)
#pragma unroll
            for (int k = 0; k < 4; k++) tot[k] += (double)s_red[w][k];
#pragma unroll
        for (int k = 0; k < 4; k++) I.part[(long long)sg.slot * 4 + k] = tot[k];
        __threadfence();
        const unsigned n = atomicAdd(&s->counter, 1u);
        s_last = n == (unsigned)I.nseg - 1u;
    }
    __syncthreads();
    if (s_last && warp == 0) {
        __threadfence();
        double tot[4] = {0, 0, 0, 0};
        for (int i = lane; i < I.nseg; i += 32)
#pragma unroll
            for (int k = 0; k < 4; k++) tot[k] += __ldcg(I.part + (long long)i * 4 + k);
#pragma unroll
        for (int k = 0; k < 4; k++)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) tot[k] += __shfl_xor_sync(0xffffffffu, tot[k], o);
        if (lane == 0) {
            s->counter = 0u;
            finish_iteration(s, s->iter, tot);
        }
    }
}

template <typename T, int NDIM>
cudaError_t launch_cg_t(const CompactArgs &a, int grid, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(a.bar, 0, sizeof(unsigned) * 2, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.err, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    CompactArgs arg = a;
    void *params[] = {&arg};
    return cudaLaunchCooperativeKernel((const void *)compact_cg_kernel<T, NDIM>, dim3(grid), dim3(CTC), params, 0,
                                       st);
}

template <typename T, int NDIM>
int grid_t() {
    int dev = 0, nsm = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, compact_cg_kernel<T, NDIM>, CTC, 0);
    if (nsm < 1) nsm = 1;
    if (per < 1) per = 1;
    return nsm * per;
}

inline int nb_for(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 152LL * 32 ? 152LL * 32 : b));
}

}  // namespace

int compact_grid(int ndim, int f32) {
    if (ndim == 2) return f32 ? grid_t<float, 2>() : grid_t<double, 2>();
    return f32 ? grid_t<float, 3>() : grid_t<double, 3>();
}

cudaError_t compact_build(const Geom &g, const uint8_t *cls, long long U, int f32, const void *const gs[3],
                          int *cmap, int *cidx, int *nbr, void *val, cudaStream_t st) {
    const long long n = (long long)g.px * g.ny * g.nz;
    const int nblk = (int)((n + SCAN_CHUNK - 1) / SCAN_CHUNK);
    unsigned int *d_cnt = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&d_cnt, sizeof(unsigned int) * (size_t)nblk, st);
    if (e != cudaSuccess) return e;
    std::vector<unsigned int> cnt((size_t)nblk);
    compact_count_kernel<<<nblk, 256, 0, st>>>(g, cls, d_cnt);
    e = cudaMemcpyAsync(cnt.data(), d_cnt, sizeof(unsigned int) * (size_t)nblk, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) {
        // exclusive scan of the chunk counts (host, fixed order)
        unsigned long long run = 0;
        for (int b = 0; b < nblk; b++) {
            const unsigned int c = cnt[(size_t)b];
            cnt[(size_t)b] = (unsigned int)run;
            run += c;
        }
        if ((long long)run != U) e = cudaErrorInvalidValue;  // set-up count disagrees
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_cnt, cnt.data(), sizeof(unsigned int) * (size_t)nblk, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        compact_index_kernel<<<nblk, CT, 0, st>>>(g, cls, d_cnt, cmap, cidx);
        if (f32)
            compact_ell_kernel<float><<<nb_for(U), 256, 0, st>>>(g, U, cidx, cmap, (const float *)gs[0],
                                                                  (const float *)gs[1], (const float *)gs[2], nbr,
                                                                  (float *)val);
        else
            compact_ell_kernel<double><<<nb_for(U), 256, 0, st>>>(g, U, cidx, cmap, (const double *)gs[0],
                                                                   (const double *)gs[1], (const double *)gs[2], nbr,
                                                                   (double *)val);
        e = cudaGetLastError();
    }
    cudaFreeAsync(d_cnt, st);
    return e;
}

cudaError_t launch_compact_gather(const CompactArgs &a, const void *src, int f32, cudaStream_t st) {
    const long long U = a.n;
    if (f32)
        compact_gather_kernel<float><<<nb_for(U), 256, 0, st>>>(U, a.cidx, (const float *)src, (float *)a.r);
    else
        compact_gather_kernel<double><<<nb_for(U), 256, 0, st>>>(U, a.cidx, (const double *)src, (double *)a.r);
    return cudaGetLastError();
}

cudaError_t launch_compact_correct(const CompactArgs &a, const double *dis, double *x, int f32, cudaStream_t st) {
    const long long U = a.n;
    if (f32)
        compact_correct_kernel<float><<<nb_for(U), 256, 0, st>>>(U, a.cidx, dis, x, (float *)a.y, (const float *)a.p,
                                                                 a.s);
    else
        compact_correct_kernel<double><<<nb_for(U), 256, 0, st>>>(U, a.cidx, dis, x, (double *)a.y,
                                                                  (const double *)a.p, a.s);
    return cudaGetLastError();
}

cudaError_t launch_compact_batch(int ndim, int f32, const CompactInst *insts, const CompactSeg *segs, int nseg,
                                 cudaStream_t st) {
    if (nseg < 1) return cudaSuccess;
#define NET_CB(T, D)                                                              \
    do {                                                                          \
        compact_batch_a_kernel<T, D><<<nseg, CT, 0, st>>>(insts, segs);           \
        compact_batch_b_kernel<T, D><<<nseg, CT, 0, st>>>(insts, segs);           \
    } while (0)
    if (ndim == 2) {
        if (f32) NET_CB(float, 2);
        else NET_CB(double, 2);
    } else {
        if (f32) NET_CB(float, 3);
        else NET_CB(double, 3);
    }
#undef NET_CB
    return cudaGetLastError();
}

cudaError_t launch_compact_cg(const CompactArgs &a, int ndim, int f32, int grid, cudaStream_t st) {
    if (ndim == 2) return f32 ? launch_cg_t<float, 2>(a, grid, st) : launch_cg_t<double, 2>(a, grid, st);
    return f32 ? launch_cg_t<float, 3>(a, grid, st) : launch_cg_t<double, 3>(a, grid, st);
}

}  // namespace netsolve
