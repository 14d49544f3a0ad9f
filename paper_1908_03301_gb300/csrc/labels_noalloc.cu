// labels_noalloc.cu -- cluster labelling that allocates no memory.
//
// Some callers cannot allocate device memory at the moment they need the
// labels: code that runs inside another framework which owns every byte of
// device memory through its own pool, or a latency-critical loop in which
// cudaMalloc / cudaFree are not acceptable (they can block the host and
// synchronise the device).  net_labels_noalloc serves them: the caller passes
// the bond planes and the two output arrays, and the union-find scratch lives
// in one fixed array of device memory that is part of the library image.
//
// That array, g_scratch, is a static __device__ object of a fixed size: once
// the library's device code is loaded on a GPU, that GPU holds it until the
// process exits, and all calls on one device share it.  Under lazy module
// loading (the CUDA default) the device code, and with it the array, is
// loaded on its first use on a device, which here is the address lookup of
// the first call: that first call can therefore allocate the array's memory
// and block, so a caller that may not allocate later makes one call at
// start-up, before its own pool takes the device memory.  Host code cannot use
// the name g_scratch as a device address; the device address is looked up
// once per device with cudaGetSymbolAddress (on the first call made on that
// device) and passed to the kernels.  Calls that overlap on the GPU (two streams, or two threads)
// would race on the shared array; the entry point serialises nothing, so the
// caller must keep calls on one device ordered.
//
// The labels are the same as those of net_create / net_get_labels: canonical
// union-find roots (smallest node index of each cluster of open bonds between
// interior nodes), -1 / -2 on the inlet / outlet faces, and the cluster class
// from the open bonds to each face.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/netsolve.h"
#include "runtime_internal.h"

namespace {

constexpr int NT = 256;
constexpr long long MAX_NODES = NET_NOALLOC_MAX_NODES;
// parent[MAX_NODES] | flags[MAX_NODES] | one word: bad-conductance flag
constexpr long long SCRATCH_WORDS = 2 * MAX_NODES + 64;

static __device__ __align__(256) unsigned int g_scratch[SCRATCH_WORDS];

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mu;
unsigned int *g_scratch_addr[MAX_DEVICES] = {};

struct Shape {
    int ndim, f, nf;
    long long n[3];
    long long N;
};

__device__ __forceinline__ void coords(const Shape &s, long long i, long long c[3]) {
    c[0] = i % s.n[0];
    c[1] = (i / s.n[0]) % s.n[1];
    c[2] = i / (s.n[0] * s.n[1]);
}

// compact index of the bond from node c to c + e_d in plane d
__device__ __forceinline__ long long bidx(const Shape &s, int d, const long long c[3]) {
    const long long m0 = s.n[0] - (d == 0), m1 = s.n[1] - (d == 1);
    return c[0] + m0 * (c[1] + m1 * c[2]);
}

__device__ __forceinline__ double bval(const void *p, int f32, long long k) {
    return f32 ? (double)static_cast<const float *>(p)[k] : static_cast<const double *>(p)[k];
}

__device__ __forceinline__ bool is_interior(const Shape &s, const long long c[3]) {
    return c[s.f] > 0 && c[s.f] < s.nf - 1;
}

__device__ int find_root(const unsigned int *parent, int i) {
    int p = (int)__ldcg(parent + i);
    while (p != i) {
        i = p;
        p = (int)__ldcg(parent + i);
    }
    return i;
}

__device__ void join(unsigned int *parent, int a, int b) {
    while (true) {
        a = find_root(parent, a);
        b = find_root(parent, b);
        if (a == b) return;
        if (a < b) {
            const int t = a;
            a = b;
            b = t;
        }
        const unsigned int old = atomicCAS(parent + a, (unsigned)a, (unsigned)b);
        if ((int)old == a) return;
        a = (int)old;
    }
}

__global__ void na_init(Shape s, unsigned int *parent) {
    for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < s.N; i += (long long)gridDim.x * NT)
        parent[i] = (unsigned)i;
}

__global__ void na_link(Shape s, const void *g0, const void *g1, const void *g2, int f32,
                        unsigned int *parent, unsigned int *bad) {
    const void *gp[3] = {g0, g1, g2};
    for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < s.N; i += (long long)gridDim.x * NT) {
        long long c[3];
        coords(s, i, c);
        const bool in_i = is_interior(s, c);
        for (int d = 0; d < s.ndim; d++) {
            if (c[d] + 1 >= s.n[d]) continue;
            const double v = bval(gp[d], f32, bidx(s, d, c));
            if (!(v >= 0.0) || isinf(v)) atomicOr(bad, 1u);
            if (!(v > 0.0) || !in_i) continue;
            long long cj[3] = {c[0], c[1], c[2]};
            cj[d] += 1;
            if (!is_interior(s, cj)) continue;
            const long long st = d == 0 ? 1 : (d == 1 ? s.n[0] : s.n[0] * s.n[1]);
            join(parent, (int)i, (int)(i + st));
        }
    }
}

__global__ void na_compress(Shape s, unsigned int *parent) {
    for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < s.N; i += (long long)gridDim.x * NT) {
        long long c[3];
        coords(s, i, c);
        if (is_interior(s, c)) parent[i] = (unsigned)find_root(parent, (int)i);
    }
}

__global__ void na_flags(Shape s, const void *gf, int f32, const unsigned int *parent,
                         unsigned int *flags) {
    for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < s.N; i += (long long)gridDim.x * NT) {
        long long c[3];
        coords(s, i, c);
        if (!is_interior(s, c)) continue;
        unsigned int fl = 0;
        if (c[s.f] == 1) {
            long long cm[3] = {c[0], c[1], c[2]};
            cm[s.f] -= 1;
            if (bval(gf, f32, bidx(s, s.f, cm)) > 0.0) fl |= 1u;
        }
        if (c[s.f] == s.nf - 2 && bval(gf, f32, bidx(s, s.f, c)) > 0.0) fl |= 2u;
        if (fl) atomicOr(flags + parent[i], fl);
    }
}

__global__ void na_final(Shape s, const unsigned int *parent, const unsigned int *flags,
                         int *label, uint8_t *cls) {
    for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < s.N; i += (long long)gridDim.x * NT) {
        long long c[3];
        coords(s, i, c);
        int lab;
        uint8_t k;
        if (c[s.f] == 0) {
            lab = -1;
            k = NET_CLS_FACE_IN;
        } else if (c[s.f] == s.nf - 1) {
            lab = -2;
            k = NET_CLS_FACE_OUT;
        } else {
            lab = (int)parent[i];
            k = (uint8_t)flags[lab];
        }
        if (label) label[i] = lab;
        if (cls) cls[i] = k;
    }
}

// Device address of g_scratch on the current device (looked up once).
net_status scratch_for_current_device(unsigned int **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return netsolve::cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= MAX_DEVICES) {
        netsolve::set_error("net_labels_noalloc: device %d beyond the supported %d", dev, MAX_DEVICES);
        return NET_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return netsolve::cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        g_scratch_addr[dev] = (unsigned int *)p;
    }
    *out = g_scratch_addr[dev];
    return NET_OK;
}

}  // namespace

#define NET_API extern "C" __attribute__((visibility("default")))

NET_API net_status net_labels_noalloc(const net_desc *desc, const void *const g[3],
                                      int32_t *label, uint8_t *cls) {
    netsolve::Geom G;
    net_status st = netsolve::make_geom(desc, &G);
    if (st != NET_OK) return st;
    if (!desc->on_device) {
        netsolve::set_error("net_labels_noalloc: bond planes must be device pointers (on_device = 1)");
        return NET_EINVAL;
    }
    if (G.per) {
        netsolve::set_error("net_labels_noalloc: periodic networks are labelled by net_create");
        return NET_EINVAL;
    }
    Shape s{};
    s.ndim = desc->ndim;
    s.f = desc->flow_axis;
    for (int a = 0; a < 3; a++) s.n[a] = desc->n[a];
    s.nf = (int)desc->n[desc->flow_axis];
    s.N = s.n[0] * s.n[1] * s.n[2];
    if (s.N > MAX_NODES) {
        netsolve::set_error("net_labels_noalloc: %lld nodes exceed the fixed scratch of %lld nodes",
                            s.N, MAX_NODES);
        return NET_EINVAL;
    }
    const void *gp[3] = {nullptr, nullptr, nullptr};
    for (int d = 0; d < s.ndim; d++) {
        const long long m = netsolve::plane_elems(G, d);
        if (m > 0 && (!g || !g[d])) {
            netsolve::set_error("net_labels_noalloc: bond plane %d is NULL", d);
            return NET_EINVAL;
        }
        gp[d] = m > 0 ? g[d] : nullptr;
    }
    // planes of extent 0 are never read; give the kernels a valid pointer
    for (int d = 0; d < 3; d++)
        if (!gp[d]) gp[d] = gp[0] ? gp[0] : (gp[1] ? gp[1] : gp[2]);
    unsigned int *scratch = nullptr;
    st = scratch_for_current_device(&scratch);
    if (st != NET_OK) return st;
    unsigned int *parent = scratch;
    unsigned int *flags = scratch + MAX_NODES;
    unsigned int *bad = scratch + 2 * MAX_NODES;
    cudaStream_t cs = (cudaStream_t)desc->stream;
    const int f32 = desc->bond_dtype == NET_F32;
    long long nb = (s.N + NT - 1) / NT;
    if (nb > 152LL * 8) nb = 152LL * 8;
    // the array keeps the previous call's contents: clear what must start at 0
    cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(unsigned int) * (size_t)s.N, cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(unsigned int), cs);
    if (e != cudaSuccess) return netsolve::cuda_fail(e, "net_labels_noalloc: clear scratch");
    na_init<<<(int)nb, NT, 0, cs>>>(s, parent);
    na_link<<<(int)nb, NT, 0, cs>>>(s, gp[0], gp[1], gp[2], f32, parent, bad);
    na_compress<<<(int)nb, NT, 0, cs>>>(s, parent);
    na_flags<<<(int)nb, NT, 0, cs>>>(s, gp[s.f], f32, parent, flags);
    na_final<<<(int)nb, NT, 0, cs>>>(s, parent, flags, label, cls);
    e = cudaGetLastError();
    if (e != cudaSuccess) return netsolve::cuda_fail(e, "net_labels_noalloc: launch");
    unsigned int hbad = 0;
    e = cudaMemcpyAsync(&hbad, bad, sizeof(hbad), cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) return netsolve::cuda_fail(e, "net_labels_noalloc");
    if (hbad) {
        netsolve::set_error("net_labels_noalloc: a conductance is negative, NaN or infinite");
        return NET_EINVAL;
    }
    return NET_OK;
}
