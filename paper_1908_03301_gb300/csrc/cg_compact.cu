// cg_compact.cu -- the inner CG solve over a compacted list of unknowns.
//
// Near the percolation threshold the unknowns of the linear system (the
// current-carrying backbone: the spanning clusters less their dead-end trees
// and loops) are a small part of the lattice: 6.6 % of a 256^3 network at
// p = 0.26.  A sweep over the lattice then moves mostly zeros.  Here the unknowns are listed row by row (in 3D,
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
//   grid barrier; then every CTA sums all CTAs' partials in the same fixed
//   order and advances its own copy of the CG state: the same inputs in the
//   same order give the same state everywhere, with no record to publish and
//   read back.  The FP32 solve keeps its sums and scalars as float-float
//   pairs (ffloat.cuh; GB300's FP64 rate would put microseconds of FP64 on
//   every iteration), the FP64 solve in FP64.
// One 1024-thread CTA per SM; thread i of CTA c owns the entries
// c * 1024 + i + j * (grid * 1024), j = 0, 1, ..., the same in both phases and
// in every iteration, so its own entries need no cross-SM visibility;
// neighbours' p written by other CTAs are read through L2 (ld.global.cg).
// Each CTA copies the table rows of its first chunks into shared memory once
// per launch (phase B's dependent chain then starts with a shared load).
// Every wait is bounded.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "ffloat.cuh"
#include "kernels.h"

namespace netsolve {
namespace {

constexpr int CT = 512;                 // threads per CTA (batched phases)
constexpr int CW = CT / 32;
constexpr int CTC = 1024;               // threads per CTA of the cooperative solve, one CTA per SM
constexpr int CWC = CTC / 32;           //   (256^3: 16.6 us per iteration against 17.6 us with two
                                        //   512-thread CTAs per SM: half the barrier arrivals and
                                        //   partial sums)
constexpr int UNR = 1;                  // unknowns a thread keeps in flight (FP64; 256^3: 46.3
                                        //   us per iteration against 49.3 us with 2)
constexpr int UNR32 = 1;                // the same in FP32 (256^3: 17.9 us per iteration against
                                        //   18.9 / 20.2 / 22.8 us with 2 / 3 / 4)
constexpr int UNA = 2;                  // unknowns in flight per thread in phase A of the
                                        //   cooperative solve (vector updates only; 256^3:
                                        //   16.5 us per iteration against 16.75 / 16.8 with 1 / 4)
constexpr int UNB = 2;                  // unknowns in flight per thread in the batched phase
                                        //   launches (8 list entries per thread per launch)
constexpr int SCAN_CHUNK = 4096;        // lattice nodes per block in the compaction scan


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
// Grid barrier (arrive_release / wait_count): every CTA's writes are done,
// thread 0 arrives and waits; returns to all threads whether the wait ended
// in time.  `withhold`: for tests of the bounded wait, this CTA does not
// arrive.
__device__ __forceinline__ bool grid_barrier(unsigned *count, unsigned goal, unsigned long long wait_ns,
                                             bool withhold) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (!withhold) arrive_release(count);
        s_ok = wait_count(count, goal, wait_ns);
    }
    __syncthreads();
    return s_ok != 0;
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

// All G CTAs' FP64 partials of one parity, summed by one warp as
// warp_sum_pairs (ffloat.cuh) sums the FP32 solve's pairs.
__device__ __forceinline__ void grid_sums(const double *part, int G, double (&tot)[4]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < 4; k++) tot[k] = 0.0;
    for (int i0 = lane; i0 < G; i0 += 128) {
        double v[4][4];
#pragma unroll
        for (int m = 0; m < 4; m++) {
            const int i = i0 + 32 * m;
#pragma unroll
            for (int k = 0; k < 4; k++) v[m][k] = i < G ? __ldcg(part + (long long)i * 4 + k) : 0.0;
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
}

// Phase B of the cooperative solve (one unknown in flight per thread), with
// the table rows of this CTA's first jc chunks in shared memory: thread i of
// CTA c owns entries k = c CTC + i + j nth, j = 0, 1, ...; for j < jc its
// row's +e_d bonds are s_w[(j NDIM + d) CTC + i] and its neighbour indices
// s_i[(j 2 (NDIM - 1) + m) CTC + i] (copied once per launch), so the
// operator's dependent chain starts with a shared-memory load instead of an
// L2 round trip.  Later chunks read the table from global memory.
template <typename T, int NDIM>
__device__ __forceinline__ void compact_phase_b_coop(const T *__restrict__ r, const T *p, T *__restrict__ q,
                                                     const T *__restrict__ val, const int *__restrict__ nbr, int U,
                                                     int tid, int nth, const T *s_w, const int *s_i, int jc,
                                                     T &s_pq, T &s_rq, T &s_qq, T &s_rr) {
    constexpr int NI = 2 * (NDIM - 1);
    const long long VS = U + 1;
    const int i = threadIdx.x;
    int j = 0;
    for (int k = tid; k < U; k += nth, j++) {
        T wxp, wxm, wp[NDIM - 1];
        int ip[NDIM - 1], im[NDIM - 1];
        if (j < jc) {
            wxp = s_w[(j * NDIM) * CTC + i];
            wxm = i > 0 ? s_w[(j * NDIM) * CTC + i - 1] : (k > 0 ? __ldg(val + k - 1) : T(0));
#pragma unroll
            for (int d = 1; d < NDIM; d++) {
                wp[d - 1] = s_w[(j * NDIM + d) * CTC + i];
                ip[d - 1] = s_i[(j * NI + 2 * (d - 1)) * CTC + i];
                im[d - 1] = s_i[(j * NI + 2 * (d - 1) + 1) * CTC + i];
            }
        } else {
            wxp = __ldg(val + k);
            wxm = k > 0 ? __ldg(val + k - 1) : T(0);
#pragma unroll
            for (int d = 1; d < NDIM; d++) {
                wp[d - 1] = __ldg(val + d * VS + k);
                ip[d - 1] = __ldg(nbr + (long long)(2 * (d - 1)) * U + k);
                im[d - 1] = __ldg(nbr + (long long)(2 * (d - 1) + 1) * U + k);
            }
        }
        const T pk = __ldcg(p + k);
        T nb = wxp * __ldcg(p + k + 1);
        nb = fma(wxm, __ldcg(p + (k > 0 ? k - 1 : 0)), nb);
#pragma unroll
        for (int d = 1; d < NDIM; d++) {
            nb = fma(wp[d - 1], __ldcg(p + ip[d - 1]), nb);
            const int jm = im[d - 1];
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

// Shared memory the table may take per CTA; the rest of the SM's 256 KB
// stays L1 cache for the gathered bonds and the -e_d weights.  256^3
// percolation (8 chunks of 28 KB wanted): 17.3 / 16.8 / 16.6 / 16.4 / 17.8 us
// per iteration with 0 / 56 / 112 / 168 / 224 KB; 192^3: 11.8 -> 11.1 us.
constexpr int TAB_MAX_BYTES = 172032;
// Bytes of shared memory one cached list chunk takes.
template <typename T, int NDIM>
constexpr int chunk_bytes() {
    return CTC * (NDIM * (int)sizeof(T) + 2 * (NDIM - 1) * (int)sizeof(int));
}

// Scalars of the cooperative solve: the FP32 solve keeps them as float-float
// pairs (InnerScalF), the FP64 solve as InnerScal.
template <typename T> struct SolveScal;
template <> struct SolveScal<float> {
    InnerScalF f;
    __device__ __forceinline__ void load(const InnerScal &s) { scal_to_ff(s, f); }
    __device__ __forceinline__ void store(InnerScal &s) const { scal_from_ff(f, s); }
    __device__ __forceinline__ int stop() const { return f.stop; }
    __device__ __forceinline__ void set_stop(int v) { f.stop = v; }
    __device__ __forceinline__ long long iter() const { return f.iter; }
    __device__ __forceinline__ float alpha() const { return f.alpha.h; }
    __device__ __forceinline__ float beta() const { return f.beta.h; }
    __device__ __forceinline__ void finish(const ff (&v)[4]) {
        f.err = 0;
        finish_iteration_ff(&f, f.iter, v);
    }
};
template <> struct SolveScal<double> {
    InnerScal d;
    __device__ __forceinline__ void load(const InnerScal &s) { d = s; }
    __device__ __forceinline__ void store(InnerScal &s) const { s = d; }
    __device__ __forceinline__ int stop() const { return d.stop; }
    __device__ __forceinline__ void set_stop(int v) { d.stop = v; }
    __device__ __forceinline__ long long iter() const { return d.iter; }
    __device__ __forceinline__ double alpha() const { return d.alpha; }
    __device__ __forceinline__ double beta() const { return d.beta; }
    __device__ __forceinline__ void finish(const double (&v)[4]) {
        d.err = 0;
        finish_iteration(&d, d.iter, v);
    }
};

template <typename T, int NDIM>
__global__ void __launch_bounds__(CTC, 1) compact_cg_kernel(CompactArgs a) {
    // FP32: sums and scalars as float-float pairs; FP64: FP64
    using S = typename std::conditional<sizeof(T) == 4, ff, double>::type;
    __shared__ InnerScal st;
    __shared__ SolveScal<T> sc;
    __shared__ T s_red[CWC][4];
    const int G = gridDim.x, c = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T *__restrict__ y = (T *)a.y;
    T *__restrict__ r = (T *)a.r;
    T *p = (T *)a.p;
    T *__restrict__ q = (T *)a.q;
    const T *__restrict__ val = (const T *)a.val;
    const int *__restrict__ nbr = a.nbr;
    if (threadIdx.x == 0) {
        const unsigned long long *src = reinterpret_cast<const unsigned long long *>(a.s);
        unsigned long long *dst = reinterpret_cast<unsigned long long *>(&st);
        for (int k = 0; k < (int)(sizeof(InnerScal) / 8); k++) dst[k] = src[k];
        sc.load(st);
    }
    __syncthreads();
    // list indices fit in 32 bits (the table stores them as int)
    const int tid = c * CTC + (int)threadIdx.x, nth = G * CTC;
    const int U = (int)a.n;
    constexpr int UN = sizeof(T) == 4 ? UNR32 : UNR;
    // this CTA's table rows of its first jc chunks, copied once per launch
    extern __shared__ __align__(16) unsigned char s_tab[];
    constexpr int NI = 2 * (NDIM - 1);
    T *s_w = reinterpret_cast<T *>(s_tab);
    int *s_i = reinterpret_cast<int *>(s_tab + (size_t)a.jc * NDIM * CTC * sizeof(T));
    for (int j = 0; j < a.jc; j++) {
        const int k = tid + j * nth;
        const bool in = k < U;
        const long long VS = U + 1;
#pragma unroll
        for (int d = 0; d < NDIM; d++) s_w[(j * NDIM + d) * CTC + threadIdx.x] = in ? val[d * VS + k] : T(0);
#pragma unroll
        for (int m = 0; m < NI; m++) s_i[(j * NI + m) * CTC + threadIdx.x] = in ? nbr[(long long)m * U + k] : 0;
    }
    __syncthreads();
    unsigned goal = 0;  // arrivals the next barrier waits for (G per barrier, modulo 2^32)
    int nbar = 0;
    bool bad = false;
    while (sc.stop() == 0) {
        const bool first = sc.iter() == 0;
        const T alpha = (T)sc.alpha(), beta = (T)sc.beta();
        // ---- phase A: finish iteration k-1 (UN unknowns in flight per thread) ----
        compact_phase_a<T, UNA>(y, r, p, q, tid, U, nth, alpha, beta, first);
        goal += (unsigned)G;
        if (!grid_barrier(a.bar, goal, a.wait_ns, nbar++ == 0 && c == a.skip_cta)) bad = true;
        // ---- phase B: q = A p and the four sums ----
        T s_pq = T(0), s_rq = T(0), s_qq = T(0), s_rr = T(0);
        compact_phase_b_coop<T, NDIM>(r, p, q, val, nbr, U, tid, nth, s_w, s_i, a.jc, s_pq, s_rq, s_qq, s_rr);
        T t4[4] = {s_pq, s_rq, s_qq, s_rr};
#pragma unroll
        for (int k = 0; k < 4; k++)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t4[k] += __shfl_xor_sync(0xffffffffu, t4[k], o);
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < 4; k++) s_red[warp][k] = t4[k];
        __syncthreads();
        const int par = (int)(sc.iter() & 1);
        if (warp == 0) {
            S t[4];
            warp_sum_rows<CWC>(s_red, t);
            if (lane == 0) {
                if constexpr (sizeof(T) == 4) {
                    float4 *dst = reinterpret_cast<float4 *>(a.pb) + 2 * ((long long)par * G + c);
                    const float *tf = reinterpret_cast<const float *>(t);  // {h, l} x 4
                    dst[0] = bad ? make_float4(NAN, NAN, NAN, NAN) : make_float4(tf[0], tf[2], tf[4], tf[6]);
                    dst[1] = bad ? make_float4(0.f, 0.f, 0.f, 0.f) : make_float4(tf[1], tf[3], tf[5], tf[7]);
                } else {
                    const double *td = reinterpret_cast<const double *>(t);
#pragma unroll
                    for (int k = 0; k < 4; k++) a.pb[((long long)par * G + c) * 4 + k] = bad ? NAN : td[k];
                }
            }
        }
        // grid barrier without a published state: after it every CTA sums all
        // CTAs' partials itself, in the same fixed order, and advances its own
        // copy of the CG state -- identical everywhere
        goal += (unsigned)G;
        const bool ok = grid_barrier(a.bar, goal, a.wait_ns, false);
        nbar++;
        if (warp == 0 && ok) {
            S tot[4];
            if constexpr (sizeof(T) == 4)
                warp_sum_pairs<5>(reinterpret_cast<const float4 *>(a.pb) + 2LL * par * G, G, tot);
            else
                grid_sums(a.pb + 4LL * par * G, G, tot);
            if (lane == 0) sc.finish(tot);
        }
        if (threadIdx.x == 0 && (bad || !ok)) {
            atomicExch(a.err, 1);
            sc.set_stop(5);
        }
        __syncthreads();
    }
    if (c == 0 && threadIdx.x == 0) {
        if (nbar > 0) sc.store(st);  // untouched (no pair round trip) when no iteration ran
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
// sums the segments' partials (pairs in the FP32 path) in slot order and runs
// finish_iteration, as the lattice sweep does; stopped networks are skipped.
template <typename T, int NDIM>
__global__ void __launch_bounds__(CT) compact_batch_a_kernel(const CompactInst *__restrict__ insts,
                                                             const CompactSeg *__restrict__ segs) {
    const CompactSeg sg = segs[blockIdx.x];
    const CompactInst &I = insts[sg.inst];
    const InnerScal *s = I.a.s;
    if (s->stop) return;
    constexpr int UN = UNB;
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
    constexpr int UN = UNB;
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
    if (warp == 0) {
        typename std::conditional<sizeof(T) == 4, ff, double>::type t[4];
        warp_sum_rows<CW>(s_red, t);
        if (lane == 0) {
            store_slot(I.part, sg.slot, t, false);
            __threadfence();
            const unsigned n = atomicAdd(&s->counter, 1u);
            s_last = n == (unsigned)I.nseg - 1u;
        }
    }
    __syncthreads();
    if (s_last && warp == 0) {
        __threadfence();
        double tot[4];
        sum_slots(I.part, I.nseg, tot, T(0));
        if (lane == 0) {
            s->counter = 0u;
            finish_iteration(s, s->iter, tot);
        }
    }
}

template <typename T, int NDIM>
cudaError_t launch_cg_t(const CompactArgs &a, int grid, cudaStream_t st) {
    // shared memory for the table rows: as many of the CTA's chunks as fit
    // beside the kernel's static shared memory
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, compact_cg_kernel<T, NDIM>);
    if (e != cudaSuccess) return e;
    const long long per_round = (long long)grid * CTC;
    const long long chunks = (a.n + per_round - 1) / per_round;
    const long long room = std::min((long long)optin - (long long)fa.sharedSizeBytes, (long long)TAB_MAX_BYTES);
    const long long fit = room / chunk_bytes<T, NDIM>();
    CompactArgs arg = a;
    arg.jc = (int)std::max(0LL, std::min(chunks, fit));
    const size_t dyn = (size_t)arg.jc * chunk_bytes<T, NDIM>();
    // the attribute is the kernel's ceiling, the same for every launch, so
    // that solves launched from several host threads cannot undercut
    // each other's setting
    e = cudaFuncSetAttribute(compact_cg_kernel<T, NDIM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.bar, 0, sizeof(unsigned) * 2, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.err, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    void *params[] = {&arg};
    return cudaLaunchCooperativeKernel((const void *)compact_cg_kernel<T, NDIM>, dim3(grid), dim3(CTC), params, dyn,
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
