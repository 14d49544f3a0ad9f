// fbm.cu -- fractional Brownian motion fields and their conductance map on
// the device (Eq. 1, Eq. 2): the generator the paper parallelises with MPI
// (Table I), here on one GPU.
//
// Field: the given complex white noise is weighted mode by mode with the
// square root of the spectral density, S(w) ~ (sum_a beta_a w_a^2)^-(H + d/2)
// (Eq. 1: d = 2, beta = 1; Eq. 2: anisotropic beta), w_a the discrete
// frequency in cycles per node ([0, 1, .., ceil(n/2)-1, -floor(n/2), .., -1]/n);
// the zero mode is dropped.  An inverse FFT (cuFFT, complex-to-complex, FP64,
// or FP32 on request: GB300 runs FP64 at 1/64 of the FP32 rate, and the
// FP64 transform is bound by it) follows; the field is its real part shifted
// and scaled to zero mean and unit variance.  The 1/N of the inverse
// transform cancels in that scaling.
// Mean and variance are two passes with per-CTA partials summed on the host
// in CTA order, so the result does not depend on scheduling.
//
// Conductances: g = exp(sigma * (B_i + B_j) / 2) for the bond between nodes i
// and j (the workloads' map), written straight into bond planes.
//
// cuFFT is loaded on first use (dlopen), so the solver library does not
// depend on it: a missing cuFFT makes these two calls fail with NET_ECUDA
// and leaves everything else working.
#include <cuda_runtime.h>
#include <cufft.h>
#include <dlfcn.h>

#include <cmath>
#include <mutex>
#include <vector>

#include "../../include/netsolve.h"
#include "runtime_internal.h"

namespace netsolve {
namespace {

constexpr int FT = 256;

struct Cufft {
    bool tried = false, ok = false;
    cufftResult (*plan2d)(cufftHandle *, int, int, cufftType) = nullptr;
    cufftResult (*plan3d)(cufftHandle *, int, int, int, cufftType) = nullptr;
    cufftResult (*set_stream)(cufftHandle, cudaStream_t) = nullptr;
    cufftResult (*exec_z2z)(cufftHandle, cufftDoubleComplex *, cufftDoubleComplex *, int) = nullptr;
    cufftResult (*exec_c2c)(cufftHandle, cufftComplex *, cufftComplex *, int) = nullptr;
    cufftResult (*destroy)(cufftHandle) = nullptr;
};

Cufft &cufft() {
    static Cufft c;
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    if (c.tried) return c;
    c.tried = true;
    const char *names[] = {"libcufft.so.12", "libcufft.so", "/usr/local/cuda/lib64/libcufft.so.12"};
    void *h = nullptr;
    for (const char *n : names)
        if ((h = dlopen(n, RTLD_NOW | RTLD_LOCAL)) != nullptr) break;
    if (!h) return c;
    c.plan2d = (decltype(c.plan2d))dlsym(h, "cufftPlan2d");
    c.plan3d = (decltype(c.plan3d))dlsym(h, "cufftPlan3d");
    c.set_stream = (decltype(c.set_stream))dlsym(h, "cufftSetStream");
    c.exec_z2z = (decltype(c.exec_z2z))dlsym(h, "cufftExecZ2Z");
    c.exec_c2c = (decltype(c.exec_c2c))dlsym(h, "cufftExecC2C");
    c.destroy = (decltype(c.destroy))dlsym(h, "cufftDestroy");
    c.ok = c.plan2d && c.plan3d && c.set_stream && c.exec_z2z && c.exec_c2c && c.destroy;
    return c;
}

struct FShape {
    long long n[3];
    long long N;
    int ndim;
};

// numpy.fft.fftfreq: i / n for i <= (n - 1) / 2, (i - n) / n above
template <typename R>
__device__ __forceinline__ R freq(long long i, long long n) {
    return (R)(i <= (n - 1) / 2 ? i : i - n) / (R)n;
}

__device__ __forceinline__ double amp_pow(double k2, double e) { return pow(k2, e); }
__device__ __forceinline__ float amp_pow(float k2, float e) { return powf(k2, e); }

// C2 = double2 (FP64 generator) or float2 (FP32 generator).  One row (fixed
// y, z) at a time per CTA, x across the threads: the row's y/z part of the
// spectral sum is formed once, and no thread divides a 64-bit index.
template <typename C2>
__global__ void fbm_filter_kernel(FShape s, C2 *a, double expo, double bx, double by, double bz) {
    using R = decltype(C2::x);
    const long long rows = s.n[1] * s.n[2];
    const int n0 = (int)s.n[0];
    for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
        const long long y = row % s.n[1], z = row / s.n[1];
        const R wy = freq<R>(y, s.n[1]), wz = freq<R>(z, s.n[2]);
        const R kyz = (R)by * wy * wy + (s.ndim == 3 ? (R)bz * wz * wz : R(0));
        C2 *ar = a + row * n0;
        for (int x = threadIdx.x; x < n0; x += FT) {
            const R wx = freq<R>(x, n0);
            const R k2 = (R)bx * wx * wx + kyz;
            const R amp = (row == 0 && x == 0) ? R(0) : amp_pow(k2, (R)expo);
            C2 v = ar[x];
            v.x *= amp;
            v.y *= amp;
            ar[x] = v;
        }
    }
}

// Per-CTA sums of Re(a) (centre = 0) or of (Re(a) - centre)^2: each thread
// accumulates in the transform's precision (GB300's FP64 rate would bound the
// FP32 generator here), the threads' sums are combined in FP64.
template <typename C2>
__global__ void fbm_sum_kernel(long long N, const C2 *a, int square, double centre, double *part) {
    using R = decltype(C2::x);
    __shared__ double sh[FT / 32];
    const R c = (R)centre;
    R racc = R(0);
    for (long long t = blockIdx.x * (long long)FT + threadIdx.x; t < N; t += (long long)gridDim.x * FT) {
        const R v = a[t].x - c;
        racc += square ? v * v : v;
    }
    double acc = (double)racc;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < FT / 32; w++) s += sh[w];
        part[blockIdx.x] = s;
    }
}

template <typename C2>
__global__ void fbm_normalise_kernel(long long N, const C2 *a, double mean, double inv_sd, double *field) {
    using R = decltype(C2::x);
    const R m = (R)mean, is = (R)inv_sd;
    for (long long t = blockIdx.x * (long long)FT + threadIdx.x; t < N; t += (long long)gridDim.x * FT)
        field[t] = (double)((a[t].x - m) * is);
}


// Bond plane d, one row (fixed y, z of the plane) at a time per CTA.
template <typename T>
__global__ void fbm_bond_kernel(FShape s, int d, int wrap, const double *__restrict__ B, double half_sigma,
                                T *g) {
    long long m[3] = {s.n[0], s.n[1], s.n[2]};
    if (!wrap) m[d] -= 1;
    const long long rows = m[1] * m[2];
    const int m0 = (int)m[0];
    const long long row_stride = s.n[0], plane_stride = s.n[0] * s.n[1];
    for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
        const long long y = row % m[1], z = row / m[1];
        const long long i0 = row_stride * (y + s.n[1] * z);
        long long j0 = i0;  // the neighbours' row (d = 1, 2) or the same row (d = 0)
        if (d == 1) j0 = y + 1 == s.n[1] ? i0 - (s.n[1] - 1) * row_stride : i0 + row_stride;
        if (d == 2) j0 = z + 1 == s.n[2] ? i0 - (s.n[2] - 1) * plane_stride : i0 + plane_stride;
        const int dx = d == 0 ? 1 : 0;
        T *gr = g + row * m0;
        for (int x = threadIdx.x; x < m0; x += FT) {
            if (sizeof(T) == 4) {  // FP32 planes: the argument in FP32 too
                const float v = (float)half_sigma * ((float)B[i0 + x] + (float)B[j0 + x + dx]);
                gr[x] = (T)expf(v);
            } else {
                gr[x] = (T)exp(half_sigma * (B[i0 + x] + B[j0 + x + dx]));
            }
        }
    }
}

int rgrid(long long rows) {
    return (int)(rows < 152LL * 16 ? (rows < 1 ? 1 : rows) : 152LL * 16);
}

int fgrid(long long n) {
    long long b = (n + FT - 1) / FT;
    if (b > 152LL * 8) b = 152LL * 8;
    return b < 1 ? 1 : (int)b;
}

net_status host_sum(const std::vector<double> &p, double *out) {
    double s = 0.0;
    for (double v : p) s += v;
    *out = s;
    return NET_OK;
}

template <typename C2>
net_status fbm_field_t(const net_fbm_desc *d, const FShape &s, Cufft &cf, C2 *a, double *field) {
    constexpr bool F32 = sizeof(C2) == 8;
    cudaStream_t st = (cudaStream_t)d->stream;
    const int nb = fgrid(s.N);
    const double expo = -(2.0 * d->hurst + d->ndim) / 4.0;
    fbm_filter_kernel<C2><<<rgrid(s.n[1] * s.n[2]), FT, 0, st>>>(s, a, expo, d->beta[0], d->beta[1],
                                                                  d->ndim == 3 ? d->beta[2] : 1.0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "fbm_filter_kernel");
    const cufftType type = F32 ? CUFFT_C2C : CUFFT_Z2Z;
    cufftHandle plan;
    cufftResult fr = d->ndim == 2 ? cf.plan2d(&plan, (int)s.n[1], (int)s.n[0], type)
                                  : cf.plan3d(&plan, (int)s.n[2], (int)s.n[1], (int)s.n[0], type);
    if (fr != CUFFT_SUCCESS) {
        set_error("net_fbm_field: cuFFT plan failed (%d)", (int)fr);
        return fr == CUFFT_ALLOC_FAILED ? NET_ENOMEM : NET_ECUDA;
    }
    fr = cf.set_stream(plan, st);
    if (fr == CUFFT_SUCCESS) {
        if (F32)
            fr = cf.exec_c2c(plan, (cufftComplex *)a, (cufftComplex *)a, CUFFT_INVERSE);
        else
            fr = cf.exec_z2z(plan, (cufftDoubleComplex *)a, (cufftDoubleComplex *)a, CUFFT_INVERSE);
    }
    cf.destroy(plan);
    if (fr != CUFFT_SUCCESS) {
        set_error("net_fbm_field: cuFFT execution failed (%d)", (int)fr);
        return NET_ECUDA;
    }
    double *part = nullptr;
    std::vector<double> hp((size_t)nb);
    double sum = 0.0, sq = 0.0;
    e = cudaMallocAsync((void **)&part, sizeof(double) * (size_t)nb, st);
    if (e != cudaSuccess) return cuda_fail(e, "net_fbm_field: partials");
    fbm_sum_kernel<C2><<<nb, FT, 0, st>>>(s.N, a, 0, 0.0, part);
    e = cudaMemcpyAsync(hp.data(), part, sizeof(double) * (size_t)nb, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) {
        host_sum(hp, &sum);
        const double mean = sum / (double)s.N;
        fbm_sum_kernel<C2><<<nb, FT, 0, st>>>(s.N, a, 1, mean, part);
        e = cudaMemcpyAsync(hp.data(), part, sizeof(double) * (size_t)nb, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) {
            host_sum(hp, &sq);
            const double sd = std::sqrt(sq / (double)s.N);
            fbm_normalise_kernel<C2><<<nb, FT, 0, st>>>(s.N, a, mean, sd > 0.0 ? 1.0 / sd : 1.0, field);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        }
    }
    cudaFreeAsync(part, st);
    if (e != cudaSuccess) return cuda_fail(e, "net_fbm_field");
    return NET_OK;
}

}  // namespace
}  // namespace netsolve

#define NET_API extern "C" __attribute__((visibility("default")))

using netsolve::FShape;

NET_API net_status net_fbm_field(const net_fbm_desc *d, void *noise, double *field) {
    using namespace netsolve;
    if (!d || !noise || !field) {
        set_error("net_fbm_field: NULL argument");
        return NET_EINVAL;
    }
    if (d->ndim != 2 && d->ndim != 3) {
        set_error("net_fbm_field: ndim must be 2 or 3");
        return NET_EINVAL;
    }
    FShape s{};
    s.ndim = d->ndim;
    s.N = 1;
    for (int a = 0; a < 3; a++) {
        s.n[a] = a < d->ndim ? d->n[a] : 1;
        if (s.n[a] < 1 || s.n[a] > (1LL << 30)) {
            set_error("net_fbm_field: extent n[%d] out of range", a);
            return NET_EINVAL;
        }
        s.N *= s.n[a];
    }
    if (d->ndim == 2 && d->n[2] != 1) {
        set_error("net_fbm_field: 2D field needs n[2] == 1");
        return NET_EINVAL;
    }
    if (s.N >= (1LL << 31)) {
        set_error("net_fbm_field: more than 2^31 - 1 nodes");
        return NET_EINVAL;
    }
    if (!std::isfinite(d->hurst)) {
        set_error("net_fbm_field: hurst must be finite");
        return NET_EINVAL;
    }
    for (int a = 0; a < d->ndim; a++)
        if (!(d->beta[a] > 0.0) || !std::isfinite(d->beta[a])) {
            set_error("net_fbm_field: beta[%d] must be positive and finite", a);
            return NET_EINVAL;
        }
    Cufft &cf = cufft();
    if (!cf.ok) {
        set_error("net_fbm_field: cuFFT (libcufft.so.12) could not be loaded");
        return NET_ECUDA;
    }
    return d->fft_f32 ? fbm_field_t<float2>(d, s, cf, (float2 *)noise, field)
                      : fbm_field_t<double2>(d, s, cf, (double2 *)noise, field);
}

NET_API net_status net_fbm_bonds(const net_desc *desc, const double *field, double sigma, void *const g[3]) {
    using namespace netsolve;
    Geom G;
    net_status s = make_geom(desc, &G);
    if (s != NET_OK) return s;
    if (!desc->on_device || !field || !g) {
        set_error("net_fbm_bonds: field and planes must be device pointers (on_device = 1)");
        return NET_EINVAL;
    }
    if (!std::isfinite(sigma)) {
        set_error("net_fbm_bonds: sigma must be finite");
        return NET_EINVAL;
    }
    FShape fs{};
    fs.ndim = desc->ndim;
    for (int a = 0; a < 3; a++) fs.n[a] = desc->n[a];
    fs.N = fs.n[0] * fs.n[1] * fs.n[2];
    cudaStream_t st = (cudaStream_t)desc->stream;
    for (int d = 0; d < desc->ndim; d++) {
        const long long m = plane_elems(G, d);
        if (m == 0) continue;
        if (!g[d]) {
            set_error("net_fbm_bonds: bond plane %d is NULL", d);
            return NET_EINVAL;
        }
        long long mm[3] = {fs.n[0], fs.n[1], fs.n[2]};
        if (!G.periodic(d)) mm[d] -= 1;
        const int nb = rgrid(mm[1] * mm[2]);
        if (desc->bond_dtype == NET_F32)
            fbm_bond_kernel<float><<<nb, FT, 0, st>>>(fs, d, G.periodic(d), field, 0.5 * sigma, (float *)g[d]);
        else
            fbm_bond_kernel<double><<<nb, FT, 0, st>>>(fs, d, G.periodic(d), field, 0.5 * sigma, (double *)g[d]);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "fbm_bond_kernel");
    }
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "net_fbm_bonds");
    return NET_OK;
}
