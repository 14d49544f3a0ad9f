// sorted_removal.cu -- correlated percolation by sorted removal (Sec. VI.B):
// close the floor(q M) bonds of smallest conductance among all M bonds of a
// network's planes, keeping the correlations of the field in the open bonds.
//
// Order: by conductance, equal conductances by position (plane d, then the
// bond's linear index in its plane, x fastest), so the closed set is unique.
//
// Selection on the device, in place, without sorting:
//   1. radix select, most significant digit first (8 bits per pass): a
//      non-negative float's bit pattern orders like its value (0 and -0 both
//      map to key 0), so a histogram of the next digit over the keys that
//      match the digits chosen so far finds the digit of the k-th smallest
//      key (one warp picks it on the device, so the passes run back to
//      back); after 4 (FP32) or 8 (FP64) passes the k-th smallest key T and
//      the number `need` of bonds equal to T that still have to close are
//      known;
//   2. every bond with key < T closes; of the bonds with key == T, the first
//      `need` in position order close: all of them when need equals their
//      count (the usual case for continuous values), otherwise a count per
//      chunk of positions, a host prefix sum and an in-chunk scan rank them.
// The first histogram pass also checks the conductances (negative, NaN or
// infinite: nothing is written and the call fails).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <vector>

#include "../../include/netsolve.h"
#include "runtime_internal.h"

namespace netsolve {
namespace {

constexpr int RT = 512;                 // threads per CTA
constexpr int CHUNK = 4096;             // positions per CTA in the tie passes
constexpr int PER = CHUNK / RT;         // 8 consecutive positions per thread

// The planes seen as one array of M positions.
struct Planes {
    void *p[3];
    long long off[4];  // off[d] = first position of plane d; off[3] = M
};

__device__ __forceinline__ int plane_of(const Planes &P, long long t) {
    return t >= P.off[1] ? (t >= P.off[2] ? 2 : 1) : 0;
}

template <typename T>
__device__ __forceinline__ T *elem(const Planes &P, long long t) {
    const int d = plane_of(P, t);
    return static_cast<T *>(P.p[d]) + (t - P.off[d]);
}

__device__ __forceinline__ uint32_t key_of(float v) { return v == 0.f ? 0u : __float_as_uint(v); }
__device__ __forceinline__ uint64_t key_of(double v) {
    return v == 0.0 ? 0ull : (uint64_t)__double_as_longlong(v);
}

// Selection state, in device memory between the passes: the digits of T
// chosen so far, the rank still to find among the keys that match them, and
// (after the last pass) how many keys equal T.
struct RsState {
    unsigned long long prefix, rem, count_T;
    unsigned bad, pad_;
};

// Histogram of digit (key >> shift) & 255 over the keys whose bits above
// shift + 8 equal the prefix chosen so far (all keys in the first pass).
template <typename T, typename K>
__global__ void __launch_bounds__(RT) rs_hist_kernel(Planes P, int shift, const RsState *state, int check,
                                                     unsigned long long *hist, unsigned *bad) {
    __shared__ unsigned h[256];
    for (int i = threadIdx.x; i < 256; i += RT) h[i] = 0u;
    __syncthreads();
    constexpr int BITS = 8 * sizeof(K);
    const bool all = shift + 8 >= BITS;
    const K prefix = (K)state->prefix;
    const long long M = P.off[3];
    const int lane = threadIdx.x & 31;
    unsigned mybad = 0;
    // The leading digits of a conductance field fall in a few bins, so the
    // lanes of a warp that share a bin add once (a warp-wide match); the
    // loop runs warp-uniformly so every lane takes part in the match.
    for (long long base = blockIdx.x * (long long)RT + (threadIdx.x & ~31); base < M;
         base += (long long)gridDim.x * RT) {
        const long long t = base + lane;
        int bin = -1;
        if (t < M) {
            const T v = *elem<T>(P, t);
            if (check && (!(v >= T(0)) || isinf(v))) mybad = 1u;
            const K k = key_of(v);
            if (all || (k >> (shift + 8)) == prefix) bin = (int)((unsigned)(k >> shift) & 255u);
        }
        const unsigned same = __match_any_sync(0xffffffffu, bin);
        if (bin >= 0 && lane == __ffs(same) - 1) atomicAdd(&h[bin], (unsigned)__popc(same));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += RT)
        if (h[i]) atomicAdd(&hist[i], (unsigned long long)h[i]);
    if (mybad) atomicOr(bad, 1u);
}

// One warp: the digit whose bin holds the rank still to find (lane l scans
// bins 8l .. 8l+7 after a warp prefix sum of the lanes' totals); the bins are
// cleared for the next pass.
__global__ void rs_select_kernel(unsigned long long *hist, RsState *state) {
    const int lane = threadIdx.x;
    unsigned long long c[8], own = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        c[j] = hist[lane * 8 + j];
        own += c[j];
    }
    unsigned long long incl = own;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const unsigned long long total = __shfl_sync(0xffffffffu, incl, 31);
    const unsigned long long want = state->rem;
    const unsigned long long excl = incl - own;
    // the lane holding the rank; the last lane if the counts fall short (the
    // bins then end the search at 255, as a sequential scan would)
    if ((excl < want && want <= incl) || (lane == 31 && want > total)) {
        unsigned long long rem = want - excl;
        int j = 0;
        while (j < 7 && c[j] < rem) rem -= c[j++];
        state->prefix = (state->prefix << 8) | (unsigned long long)(lane * 8 + j);
        state->rem = rem;
        state->count_T = c[j];
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 8; j++) hist[lane * 8 + j] = 0ull;
}

// Close every bond with key < T (and key == T when `with_equal`).
template <typename T, typename K>
__global__ void __launch_bounds__(RT) rs_close_kernel(Planes P, K Tk, int with_equal) {
    const long long M = P.off[3];
    for (long long t = blockIdx.x * (long long)RT + threadIdx.x; t < M; t += (long long)gridDim.x * RT) {
        T *e = elem<T>(P, t);
        const K k = key_of(*e);
        if (k < Tk || (with_equal && k == Tk)) *e = T(0);
    }
}

// Bonds with key == T in each chunk of CHUNK positions.
template <typename T, typename K>
__global__ void __launch_bounds__(RT) rs_tie_count_kernel(Planes P, K Tk, unsigned *counts) {
    __shared__ unsigned s;
    if (threadIdx.x == 0) s = 0u;
    __syncthreads();
    const long long M = P.off[3];
    const long long t0 = (long long)blockIdx.x * CHUNK + (long long)threadIdx.x * PER;
    unsigned c = 0;
    for (int j = 0; j < PER; j++) {
        const long long t = t0 + j;
        if (t < M && key_of(*elem<T>(P, t)) == Tk) c++;
    }
    if (c) atomicAdd(&s, c);
    __syncthreads();
    if (threadIdx.x == 0) counts[blockIdx.x] = s;
}

// Close key < T, and the bonds with key == T whose rank in position order
// (chunk offset + rank inside the chunk) is below `need`.
template <typename T, typename K>
__global__ void __launch_bounds__(RT) rs_tie_close_kernel(Planes P, K Tk, const unsigned long long *offsets,
                                                          unsigned long long need) {
    __shared__ unsigned warp_tot[RT / 32];
    const long long M = P.off[3];
    const long long t0 = (long long)blockIdx.x * CHUNK + (long long)threadIdx.x * PER;
    unsigned eq = 0, cnt = 0;
    for (int j = 0; j < PER; j++) {
        const long long t = t0 + j;
        if (t < M && key_of(*elem<T>(P, t)) == Tk) {
            eq |= 1u << j;
            cnt++;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    unsigned before = 0;
    for (int w = 0; w < warp; w++) before += warp_tot[w];
    unsigned long long rank = offsets[blockIdx.x] + before + incl - cnt;
    for (int j = 0; j < PER; j++) {
        const long long t = t0 + j;
        if (t >= M) break;
        T *e = elem<T>(P, t);
        if (eq & (1u << j)) {
            if (rank < need) *e = T(0);
            rank++;
        } else if (key_of(*e) < Tk) {
            *e = T(0);
        }
    }
}

int grid_for(long long M) {
    long long b = (M + RT - 1) / RT;
    if (b > 152LL * 4) b = 152LL * 4;
    return b < 1 ? 1 : (int)b;
}

#define RS_CK(call)                                              \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) {                                 \
            st_ = cuda_fail(e_, #call);                          \
            goto done;                                           \
        }                                                        \
    } while (0)

template <typename T, typename K>
net_status close_smallest(const Planes &P, long long k, cudaStream_t cs) {
    constexpr int BITS = 8 * sizeof(K);
    const long long M = P.off[3];
    const int nb = grid_for(M);
    net_status st_ = NET_OK;
    unsigned long long *hist = nullptr, *offs = nullptr;
    RsState *state = nullptr;
    unsigned *counts = nullptr;
    RsState hs{};
    std::vector<unsigned> hc;
    std::vector<unsigned long long> ho;
    long long nch = 0;
    // all passes run back to back on the stream (the digit choice is made on
    // the device); the host reads the state once, before anything is written
    RS_CK(cudaMallocAsync((void **)&hist, 256 * sizeof(unsigned long long), cs));
    RS_CK(cudaMallocAsync((void **)&state, sizeof(RsState), cs));
    RS_CK(cudaMemsetAsync(hist, 0, 256 * sizeof(unsigned long long), cs));
    hs.rem = (unsigned long long)k;
    RS_CK(cudaMemcpyAsync(state, &hs, sizeof(RsState), cudaMemcpyHostToDevice, cs));
    for (int shift = BITS - 8; shift >= 0; shift -= 8) {
        const int first = shift == BITS - 8;
        rs_hist_kernel<T, K><<<nb, RT, 0, cs>>>(P, shift, state, first, hist, &state->bad);
        RS_CK(cudaGetLastError());
        if (k == 0) break;  // only the conductance check
        rs_select_kernel<<<1, 32, 0, cs>>>(hist, state);
        RS_CK(cudaGetLastError());
    }
    RS_CK(cudaMemcpyAsync(&hs, state, sizeof(RsState), cudaMemcpyDeviceToHost, cs));
    RS_CK(cudaStreamSynchronize(cs));
    if (hs.bad) {
        set_error("net_close_smallest: a conductance is negative, NaN or infinite");
        st_ = NET_EINVAL;
        goto done;
    }
    if (k == 0) goto done;
    // T = hs.prefix, the k-th smallest key; hs.rem of the hs.count_T bonds
    // equal to T close
    if (hs.rem == hs.count_T) {
        rs_close_kernel<T, K><<<nb, RT, 0, cs>>>(P, (K)hs.prefix, 1);
        RS_CK(cudaGetLastError());
    } else {
        nch = (M + CHUNK - 1) / CHUNK;
        RS_CK(cudaMallocAsync((void **)&counts, sizeof(unsigned) * (size_t)nch, cs));
        RS_CK(cudaMallocAsync((void **)&offs, sizeof(unsigned long long) * (size_t)nch, cs));
        rs_tie_count_kernel<T, K><<<(unsigned)nch, RT, 0, cs>>>(P, (K)hs.prefix, counts);
        RS_CK(cudaGetLastError());
        hc.resize((size_t)nch);
        ho.resize((size_t)nch);
        RS_CK(cudaMemcpyAsync(hc.data(), counts, sizeof(unsigned) * (size_t)nch, cudaMemcpyDeviceToHost, cs));
        RS_CK(cudaStreamSynchronize(cs));
        unsigned long long run = 0;
        for (long long c = 0; c < nch; c++) {
            ho[(size_t)c] = run;
            run += hc[(size_t)c];
        }
        RS_CK(cudaMemcpyAsync(offs, ho.data(), sizeof(unsigned long long) * (size_t)nch, cudaMemcpyHostToDevice, cs));
        rs_tie_close_kernel<T, K><<<(unsigned)nch, RT, 0, cs>>>(P, (K)hs.prefix, offs, hs.rem);
        RS_CK(cudaGetLastError());
    }
    RS_CK(cudaStreamSynchronize(cs));
done:
    if (hist) cudaFreeAsync(hist, cs);
    if (state) cudaFreeAsync(state, cs);
    if (counts) cudaFreeAsync(counts, cs);
    if (offs) cudaFreeAsync(offs, cs);
    cudaStreamSynchronize(cs);
    return st_;
}

}  // namespace
}  // namespace netsolve

#define NET_API extern "C" __attribute__((visibility("default")))

NET_API net_status net_close_smallest(const net_desc *desc, void *const g[3], double q) {
    netsolve::Geom G;
    net_status s = netsolve::make_geom(desc, &G);
    if (s != NET_OK) return s;
    if (!desc->on_device) {
        netsolve::set_error("net_close_smallest: bond planes must be device pointers (on_device = 1)");
        return NET_EINVAL;
    }
    if (!(q >= 0.0 && q <= 1.0)) {
        netsolve::set_error("net_close_smallest: q must lie in [0, 1]");
        return NET_EINVAL;
    }
    netsolve::Planes P{};
    P.off[0] = 0;
    for (int d = 0; d < 3; d++) {
        const long long m = d < G.ndim ? netsolve::plane_elems(G, d) : 0;
        if (m > 0 && (!g || !g[d])) {
            netsolve::set_error("net_close_smallest: bond plane %d is NULL", d);
            return NET_EINVAL;
        }
        P.p[d] = m > 0 ? g[d] : nullptr;
        P.off[d + 1] = P.off[d] + m;
    }
    const long long M = P.off[3];
    if (M == 0) return NET_OK;
    // the same product and rounding as floor(q * M) in double anywhere else
    const long long k = (long long)std::floor(q * (double)M);
    cudaStream_t cs = (cudaStream_t)desc->stream;
    return desc->bond_dtype == NET_F32 ? netsolve::close_smallest<float, uint32_t>(P, k, cs)
                                       : netsolve::close_smallest<double, uint64_t>(P, k, cs);
}
