// common.cuh -- shared device-side definitions of the network solver.
//
// Internal layout ("padded grid"): node (x, y, z) lives at
//     idx = pad + x + px * (y + ny * z),   px = round_up(nx, 4),
// so every row starts on a 16-byte boundary for both float and double.
// Columns x in [nx, px) are ghost nodes: zero conductance, zero vectors.
// `pad` zero elements precede and follow the grid (pad >= the largest
// neighbour offset), so the stencil never indexes outside an allocation.
// Bond plane d over the padded grid holds at idx(c) the conductance of the
// bond c -> c + e_d, and 0 where that bond does not exist.  Along a periodic
// axis (y or z) the last layer's bonds lead back to layer 0; the set-up
// kernels, the FP64 residual pass, the persistent 2D kernel (periodic y) and
// the compacted solve (whose neighbour table holds the wrap) follow them, and
// periodic networks take only those two inner solves.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace netsolve {

struct Geom {
    int ndim;        // 2 or 3
    int f;           // flow axis
    int nx, ny, nz;  // node extents (nz = 1 in 2D)
    int px;          // row pitch
    int nf;          // extent along the flow axis
    long long plane; // px * ny
    long long pad;   // zero elements before (and after) the grid
    long long len;   // pad + plane * nz + pad
    double p_in, p_out;
    unsigned per;    // bit d: axis d is periodic (y or z, never the flow axis)

    __host__ __device__ long long idx(int x, int y, int z) const {
        return pad + x + (long long)px * (y + (long long)ny * z);
    }
    __host__ __device__ long long stride(int d) const {
        return d == 0 ? 1 : (d == 1 ? (long long)px : plane);
    }
    __host__ __device__ int coord(int d, int x, int y, int z) const {
        return d == 0 ? x : (d == 1 ? y : z);
    }
    __host__ __device__ int extent(int d) const {
        return d == 0 ? nx : (d == 1 ? ny : nz);
    }
    __host__ __device__ bool periodic(int d) const { return (per >> d) & 1u; }
    // Neighbour of node i (coordinate cd along d) one step along +e_d / -e_d.
    // Off a no-flow boundary this is i +- stride(d) as everywhere else (a
    // ghost or pad node with zero bonds and vectors); across a periodic
    // boundary it wraps to the opposite layer.
    __host__ __device__ long long up(long long i, int d, int cd) const {
        return (cd + 1 == extent(d) && periodic(d)) ? i - (long long)(extent(d) - 1) * stride(d)
                                                    : i + stride(d);
    }
    __host__ __device__ long long down(long long i, int d, int cd) const {
        return (cd == 0 && periodic(d)) ? i + (long long)(extent(d) - 1) * stride(d) : i - stride(d);
    }
};

// Cluster classes (same values as the NET_CLS_* constants of the C ABI).
// CLS_DANGLING is internal: a node of a spanning cluster on a dead-end tree,
// left out of the linear system (reported as CLS_SPANNING).
enum : uint8_t {
    CLS_ISOLATED = 0, CLS_INLET = 1, CLS_OUTLET = 2, CLS_SPANNING = 3,
    CLS_FACE_IN = 4, CLS_FACE_OUT = 5, CLS_DANGLING = 6, CLS_GHOST = 255
};

// Scalars of one inner CG solve, in device memory.  The fused iteration
// kernel reads alpha/beta/iter/stop at entry; the last CTA to finish writes
// the next values, after every other CTA has read them.
struct InnerScal {
    double alpha, beta;   // step lengths for the next iteration
    double rho0;          // ||r||^2 when this pass was armed
    double tol2;          // pass target: ||r||^2 <= tol2 * rho0
    double rho;           // last directly computed ||r||^2
    double best;          // smallest ||r||^2 seen (stagnation watch)
    double maxrr;         // largest ||r||^2 since the pass was armed
    double delta2;        // reliable update due at ||r||^2 <= delta2 * maxrr (0: off)
    long long best_iter;
    long long iter;       // iterations since the CG recursion (re)started
    long long iter0;      // iter when this pass was armed
    long long max_iter;
    long long stag_window;
    int stop;             // 0 run, 1 converged, 2 cap, 3 stagnated, 4 breakdown,
                          // 5 device wait timed out, 6 refinement pass due
                          // (alpha, beta of the next iteration still pending)
    int err;              // set by a CTA whose bounded wait gave up
    unsigned int counter; // CTA arrival counter of the running launch
    int reliable;         // passes continue the recursion (stop 6) instead of restarting
};
static_assert(sizeof(InnerScal) % 8 == 0, "InnerScal is copied as 64-bit words");

// Sums of one outer (FP64) residual pass.
struct OuterScal {
    double rr;       // sum r_i^2 over interior nodes
    double rmax;     // max |r_i|
    double rh2;      // sum (D^-1/2 r)_i^2
    double qin, qout, energy;
    double ez;       // sum (x_i - p_out) r_i: first-order error of Q_in
    unsigned int counter;
};

// Sums of the set-up pass.
struct SetupScal {
    double bb;             // ||b||^2
    unsigned long long n_active;  // nodes of spanning clusters
    unsigned long long n_solved;  // of them, unknowns of the linear system
    unsigned int counter;
    unsigned int bad;      // nonzero: a conductance was negative / NaN / inf
    unsigned int pruned;   // dead-end nodes removed by the last pruning rounds
    unsigned int pad_;
};

// ---------------------------------------------------------------------------
// deterministic reductions
// ---------------------------------------------------------------------------
enum { RED_SUM = 0, RED_MAX = 1 };

template <int OP>
__device__ __forceinline__ double red_op(double a, double b) {
    return OP == RED_SUM ? a + b : fmax(a, b);
}

// Block-wide reduction of NV values; every thread receives the result.
// Order is fixed by thread index, so the result is reproducible.
template <int NV, int NT>
__device__ __forceinline__ void block_reduce(double (&v)[NV], const int (&ops)[NV]) {
    __shared__ double s_red[NT / 32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            double t = __shfl_xor_sync(0xffffffffu, v[k], o);
            v[k] = ops[k] == RED_SUM ? v[k] + t : fmax(v[k], t);
        }
    }
    __syncthreads();  // s_red may still be read from a previous call
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) s_red[warp][k] = v[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; k++) {
        double a = s_red[0][k];
        for (int w = 1; w < NT / 32; w++) a = ops[k] == RED_SUM ? a + s_red[w][k] : fmax(a, s_red[w][k]);
        v[k] = a;
    }
}

// Grid-wide reduction through per-CTA partials and an arrival counter: the
// last CTA to arrive sums the partials in CTA order and returns true with
// the totals in v (all its threads).  Other CTAs return false.  The counter
// is reset by the last CTA so the same storage serves the next launch.
template <int NV, int NT>
__device__ __forceinline__ bool grid_reduce(double (&v)[NV], const int (&ops)[NV],
                                            double *partials, unsigned int *counter) {
    __shared__ bool s_last;
    block_reduce<NV, NT>(v, ops);
    const int nb = gridDim.x * gridDim.y * gridDim.z;
    const int b = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) partials[(long long)b * NV + k] = v[k];
        __threadfence();
        unsigned int t = atomicAdd(counter, 1u);
        s_last = (t == (unsigned)nb - 1);
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
#pragma unroll
    for (int k = 0; k < NV; k++) v[k] = ops[k] == RED_SUM ? 0.0 : -INFINITY;
    for (int i = threadIdx.x; i < nb; i += NT) {
#pragma unroll
        for (int k = 0; k < NV; k++) {
            double p = __ldcg(&partials[(long long)i * NV + k]);
            v[k] = ops[k] == RED_SUM ? v[k] + p : fmax(v[k], p);
        }
    }
    block_reduce<NV, NT>(v, ops);
    if (threadIdx.x == 0) *counter = 0u;
    return true;
}

// End of one fused CG iteration, run by one thread of the last CTA with the
// four reduced sums v = {<p,q>, <r,q>, <q,q>, <r,r>} of iteration k:
// alpha_k = <r,r>/<p,q>, beta_k = ||r - alpha q||^2 / <r,r> with the square
// expanded; convergence, cap, stagnation and breakdown tests.
//
// Restart mode ends the pass when ||r_k|| reaches the pass target (stop 1,
// y consistent with r_k).  Reliable mode first takes alpha_k, beta_k and
// ends the pass when the next residual ||r_k - alpha_k q_k|| reaches the
// target or has fallen to delta times its largest value since the pass was
// armed (stop 6): the refinement pass then folds y + alpha_k p_k into x,
// recomputes r in FP64 and the recursion continues from p_k.
__device__ __forceinline__ void finish_iteration(InnerScal *s, long long k, const double (&v)[4]) {
    const double pq = v[0], rq = v[1], qq = v[2], rr = v[3];
    s->rho = rr;
    s->iter = k + 1;
    if (s->err) {
        s->stop = 5;
        return;
    }
    if (rr == 0.0 || (!s->reliable && rr <= s->tol2 * s->rho0)) {
        s->stop = 1;
        return;
    }
    if (!(pq > 0.0) || !isfinite(pq) || !isfinite(rr)) {
        s->stop = 4;
        return;
    }
    const double a = rr / pq;
    double rn1 = rr - 2.0 * a * rq + a * a * qq;
    if (!(rn1 > 0.0)) rn1 = 0.0;  // cancellation: restart along the residual
    s->alpha = a;
    s->beta = rn1 / rr;
    if (s->reliable) {
        s->maxrr = fmax(s->maxrr, rr);
        if (rn1 <= s->tol2 * s->rho0 || rn1 <= s->delta2 * s->maxrr) {
            s->stop = 6;
            return;
        }
    }
    if (rr < 0.25 * s->best) {
        s->best = rr;
        s->best_iter = k;
    }
    if (k + 1 >= s->max_iter) s->stop = 2;
    else if (k - s->best_iter > s->stag_window) s->stop = 3;
}

// Device clock in nanoseconds (bounds the grid-barrier waits in time).
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid barrier of the cooperative kernels, one counter for the whole launch
// (zeroed before it): each CTA, its writes done, adds its arrival with
// release semantics and no value returned; barrier n is passed when the count
// reaches G n.  Every CTA polls the count itself: nobody has to arrive last
// and release the others, which saves an atomic round trip and a release
// store per barrier (2.08 against 2.96 us over 304 CTAs in a stand-alone
// probe).
__device__ __forceinline__ void arrive_release(unsigned *count) {
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(count) : "memory");
}
// Waits until *count has reached goal (compared modulo 2^32: the count is
// never more than G arrivals away from a goal being waited for).  Relaxed
// polls -- an acquire per poll would order, and slow, the memory traffic of
// the other CTA on the SM -- then one acquire.  Gives up, returning false,
// after wait_ns of device time.
__device__ __forceinline__ bool wait_count(const unsigned *count, unsigned goal, unsigned long long wait_ns) {
    const unsigned long long t0 = globaltimer_ns();
    for (unsigned i = 0;; i++) {
        unsigned v;
        asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
        if ((int)(v - goal) >= 0) {
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
            return (int)(v - goal) >= 0;
        }
        if ((i & 255u) == 255u && globaltimer_ns() - t0 > wait_ns) return false;
    }
}

// 16-byte vector of T (float4 / double2) with element access.
template <typename T> struct Vec;
template <> struct Vec<float> {
    static constexpr int N = 4;
    float v[4];
    __device__ __forceinline__ void load(const float *p) {
        float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
    __device__ __forceinline__ void store(float *p) const {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
    __device__ __forceinline__ void zero() { v[0] = v[1] = v[2] = v[3] = 0.f; }
};
template <> struct Vec<double> {
    static constexpr int N = 2;
    double v[2];
    __device__ __forceinline__ void load(const double *p) {
        double2 t = *reinterpret_cast<const double2 *>(p);
        v[0] = t.x; v[1] = t.y;
    }
    __device__ __forceinline__ void store(double *p) const {
        *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
    }
    __device__ __forceinline__ void zero() { v[0] = v[1] = 0.0; }
};

}  // namespace netsolve
