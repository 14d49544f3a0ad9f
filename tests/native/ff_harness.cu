// ff_harness.cu -- runs the library's float-float helpers (ffloat.cuh) on
// inputs from a file and writes the raw results, for tests that check them
// against exact rational arithmetic.
//
// usage: ff_harness in.bin out.bin
// in.bin:  int32 n_ops, int32 n_sum, int32 n_fin;
//          n_ops x {ah, al, bh, bl} float32;
//          n_sum x {hi[4], lo[4]} float32 (the per-CTA slots one warp sums);
//          n_fin x {pq, rq, qq, rr, tol2, rho0, delta2, maxrr, best} float64,
//                  then {reliable, iter, best_iter, max_iter, stag_window} int64
// out.bin: n_ops x 5 pairs (a+b, a-b, a*b, a/b, a+bh) and 2 pairs (b+a, b*a);
//          32 lanes x 4 pairs {h, l} of the warp sum, one row per lane, for
//          four and then five slots per lane in flight;
//          n_fin x {alpha, beta, rho, best, maxrr} float64 and {stop, best_iter}
//          int64 from finish_iteration_ff, then the same from finish_iteration.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../../paper_1908_03301_gb300/csrc/ffloat.cuh"

using namespace netsolve;

struct FinIn {
    double v[9];
    long long i[5];
};
struct FinOut {
    double d[5];
    long long i[2];
};

__global__ void ops_kernel(const float4 *in, int n, ff *out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float4 x = in[t];
    const ff a = {x.x, x.y}, b = {x.z, x.w};
    ff *o = out + (long long)t * 7;
    o[0] = ff_add(a, b);
    o[1] = ff_sub(a, b);
    o[2] = ff_mul(a, b);
    o[3] = ff_div(a, b);
    o[4] = ff_add_f(a, b.h);
    o[5] = ff_add(b, a);
    o[6] = ff_mul(b, a);
}

__global__ void sum_kernel(const float4 *slots, int n, ff *out) {
    ff tot[4], tot5[4];
    warp_sum_pairs(slots, n, tot);
    warp_sum_pairs<5>(slots, n, tot5);
#pragma unroll
    for (int k = 0; k < 4; k++) {
        out[threadIdx.x * 4 + k] = tot[k];
        out[128 + threadIdx.x * 4 + k] = tot5[k];
    }
}

__global__ void fin_kernel(const FinIn *in, int n, FinOut *out_ff, FinOut *out_d) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const FinIn x = in[t];
    InnerScal s{};
    s.alpha = 0.0;
    s.beta = 0.0;
    s.tol2 = x.v[4];
    s.rho0 = x.v[5];
    s.delta2 = x.v[6];
    s.maxrr = x.v[7];
    s.best = x.v[8];
    s.rho = 0.0;
    s.reliable = (int)x.i[0];
    s.iter = x.i[1];
    s.best_iter = x.i[2];
    s.max_iter = x.i[3];
    s.stag_window = x.i[4];
    s.stop = 0;
    s.err = 0;
    InnerScalF f;
    scal_to_ff(s, f);
    const ff v[4] = {ff_of(x.v[0]), ff_of(x.v[1]), ff_of(x.v[2]), ff_of(x.v[3])};
    finish_iteration_ff(&f, f.iter, v);
    InnerScal sf = s;
    scal_from_ff(f, sf);
    out_ff[t] = FinOut{{sf.alpha, sf.beta, sf.rho, sf.best, sf.maxrr}, {sf.stop, sf.best_iter}};
    const double vd[4] = {ff_to_double(v[0]), ff_to_double(v[1]), ff_to_double(v[2]), ff_to_double(v[3])};
    finish_iteration(&s, s.iter, vd);
    out_d[t] = FinOut{{s.alpha, s.beta, s.rho, s.best, s.maxrr}, {s.stop, s.best_iter}};
}

#define CK(x)                                                                      \
    do {                                                                           \
        cudaError_t e_ = (x);                                                      \
        if (e_ != cudaSuccess) {                                                   \
            fprintf(stderr, "%s: %s\n", #x, cudaGetErrorString(e_));               \
            return 1;                                                              \
        }                                                                          \
    } while (0)

int main(int argc, char **argv) {
    if (argc != 3) {
        fprintf(stderr, "usage: %s in.bin out.bin\n", argv[0]);
        return 2;
    }
    FILE *fi = fopen(argv[1], "rb");
    if (!fi) return 2;
    int hdr[3];
    if (fread(hdr, sizeof(int), 3, fi) != 3) return 2;
    const int n_ops = hdr[0], n_sum = hdr[1], n_fin = hdr[2];
    if (n_ops < 1 || n_sum < 1 || n_fin < 1) return 2;
    std::vector<float4> ops(n_ops);
    std::vector<float4> sums(2 * (size_t)n_sum);
    std::vector<FinIn> fin(n_fin);
    if (fread(ops.data(), sizeof(float4), n_ops, fi) != (size_t)n_ops) return 2;
    if (fread(sums.data(), sizeof(float4), sums.size(), fi) != sums.size()) return 2;
    if (fread(fin.data(), sizeof(FinIn), n_fin, fi) != (size_t)n_fin) return 2;
    fclose(fi);

    float4 *d_ops, *d_sums;
    ff *d_ops_out, *d_sum_out;
    FinIn *d_fin;
    FinOut *d_ff, *d_d;
    CK(cudaMalloc(&d_ops, sizeof(float4) * n_ops));
    CK(cudaMalloc(&d_ops_out, sizeof(ff) * 7 * n_ops));
    CK(cudaMalloc(&d_sums, sizeof(float4) * sums.size()));
    CK(cudaMalloc(&d_sum_out, sizeof(ff) * 32 * 4 * 2));
    CK(cudaMalloc(&d_fin, sizeof(FinIn) * n_fin));
    CK(cudaMalloc(&d_ff, sizeof(FinOut) * n_fin));
    CK(cudaMalloc(&d_d, sizeof(FinOut) * n_fin));
    CK(cudaMemcpy(d_ops, ops.data(), sizeof(float4) * n_ops, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_sums, sums.data(), sizeof(float4) * sums.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_fin, fin.data(), sizeof(FinIn) * n_fin, cudaMemcpyHostToDevice));
    ops_kernel<<<(n_ops + 127) / 128, 128>>>(d_ops, n_ops, d_ops_out);
    CK(cudaGetLastError());
    sum_kernel<<<1, 32>>>(d_sums, n_sum, d_sum_out);
    CK(cudaGetLastError());
    fin_kernel<<<(n_fin + 127) / 128, 128>>>(d_fin, n_fin, d_ff, d_d);
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());
    std::vector<ff> o_ops(7 * (size_t)n_ops), o_sum(32 * 4 * 2);
    std::vector<FinOut> o_ff(n_fin), o_d(n_fin);
    CK(cudaMemcpy(o_ops.data(), d_ops_out, sizeof(ff) * o_ops.size(), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(o_sum.data(), d_sum_out, sizeof(ff) * o_sum.size(), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(o_ff.data(), d_ff, sizeof(FinOut) * n_fin, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(o_d.data(), d_d, sizeof(FinOut) * n_fin, cudaMemcpyDeviceToHost));
    FILE *fo = fopen(argv[2], "wb");
    if (!fo) return 2;
    fwrite(o_ops.data(), sizeof(ff), o_ops.size(), fo);
    fwrite(o_sum.data(), sizeof(ff), o_sum.size(), fo);
    fwrite(o_ff.data(), sizeof(FinOut), n_fin, fo);
    fwrite(o_d.data(), sizeof(FinOut), n_fin, fo);
    fclose(fo);
    return 0;
}
