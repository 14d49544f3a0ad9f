// kernels_setup.cu -- network set-up on the device: bond packing and
// validation, cluster labelling, Jacobi scaling, initial pressures.
//
// Cluster labelling (the step that makes Eq. 3 nonsingular at percolation
// disorder, Sec. V): a lock-free union-find over the open bonds between
// interior nodes.  A union always hooks the larger root under the smaller,
// so every root is the smallest index of its cluster and the final labels do
// not depend on thread scheduling: the result is bit-exact.
#include <cfloat>
#include <cmath>

#include "kernels.h"

namespace netsolve {
namespace {

constexpr int NT = 256;

__host__ __device__ inline long long grid_nodes(const Geom &g) {
    return (long long)g.px * g.ny * g.nz;
}

// Linear padded-grid position t in [0, px*ny*nz) -> coordinates.
__device__ inline void unflatten(const Geom &g, long long t, int &x, int &y, int &z) {
    x = (int)(t % g.px);
    long long r = t / g.px;
    y = (int)(r % g.ny);
    z = (int)(r / g.ny);
}

inline int blocks_for(long long n) {
    long long b = (n + NT - 1) / NT;
    if (b > 152LL * 16) b = 152LL * 16;
    if (b < 1) b = 1;
    return (int)b;
}

template <typename T>
__device__ inline double ld_bond(const void *p, long long i) {
    return (double)static_cast<const T *>(p)[i];
}

__device__ inline double bond_at(const void *p, int f32, long long i) {
    return f32 ? ld_bond<float>(p, i) : ld_bond<double>(p, i);
}

// ------------------------------------------------------------------ packing
template <typename S, typename D>
__global__ void pack_kernel(Geom g, int d, const S *__restrict__ src, D *__restrict__ dst,
                            unsigned int *bad) {
    const long long n = grid_nodes(g);
    const int last = g.periodic(d) ? 0 : 1;  // a periodic plane has a bond per node
    const int mx = g.nx - (d == 0) * last, my = g.ny - (d == 1) * last;
    for (long long t = blockIdx.x * (long long)NT + threadIdx.x; t < n;
         t += (long long)gridDim.x * NT) {
        int x, y, z;
        unflatten(g, t, x, y, z);
        D v = D(0);
        const int c = g.coord(d, x, y, z);
        if (x < g.nx && c < g.extent(d) - last) {
            S s = src[x + (long long)mx * (y + (long long)my * z)];
            if (!(s >= S(0)) || isinf((double)s)) atomicOr(bad, 1u);
            v = (D)s;
        }
        dst[g.idx(x, y, z)] = v;
    }
}

// ------------------------------------------------------------------ labels
__device__ inline int uf_find(const int *parent, int i) {
    int p = __ldcg(parent + i);
    while (p != i) {
        i = p;
        p = __ldcg(parent + i);
    }
    return i;
}

__device__ inline void uf_union(int *parent, int a, int b) {
    while (true) {
        a = uf_find(parent, a);
        b = uf_find(parent, b);
        if (a == b) return;
        if (a < b) {
            int t = a;
            a = b;
            b = t;
        }
        const int old = atomicCAS(parent + a, a, b);
        if (old == a) return;
        a = old;  // a was hooked meanwhile: continue from its new parent
    }
}

__device__ inline bool interior(const Geom &g, int x, int y, int z) {
    const int cf = g.coord(g.f, x, y, z);
    return x < g.nx && cf > 0 && cf < g.nf - 1;
}

__global__ void lab_init(Geom g, int *parent) {
    const long long n = grid_nodes(g);
    for (long long t = blockIdx.x * (long long)NT + threadIdx.x; t < n;
         t += (long long)gridDim.x * NT) {
        int x, y, z;
        unflatten(g, t, x, y, z);
        const long long i = g.idx(x, y, z);
        parent[i] = (int)i;
    }
}

__global__ void lab_link(Geom g, const void *g0, const void *g1, const void *g2, int f32,
                         int *parent) {
    const long long n = grid_nodes(g);
    const void *gp[3] = {g0, g1, g2};
    for (long long t = blockIdx.x * (long long)NT + threadIdx.x; t < n;
         t += (long long)gridDim.x * NT) {
        int x, y, z;
        unflatten(g, t, x, y, z);
        if (!interior(g, x, y, z)) continue;
        const long long i = g.idx(x, y, z);
        for (int d = 0; d < g.ndim; d++) {
            if (!(bond_at(gp[d], f32, i) > 0.0)) continue;
            int c[3] = {x, y, z};
            // the bond exists, so the neighbour is inside the grid
            c[d] = c[d] + 1 == g.extent(d) ? 0 : c[d] + 1;
            if (!interior(g, c[0], c[1], c[2])) continue;
            uf_union(parent, (int)i, (int)g.idx(c[0], c[1], c[2]));
        }
    }
}

__global__ void lab_compress(Geom g, int *parent) {
    const long long n = grid_nodes(g);
    for (long long t = blockIdx.x * (long long)NT + threadIdx.x; t < n;
         t += (long long)gridDim.x * NT) {
        int x, y, z;
        unflatten(g, t, x, y, z);
        if (!interior(g, x, y, z)) continue;
        const long long i = g.idx(x, y, z);
        parent[i] = uf_find(parent, (int)i);
    }
}

__global__ void lab_flags(Geom g, const void *gf, int f32, const int *parent,
                          unsigned int *flags) {
    const long long n = grid_nodes(g);
    const long long sf = g.stride(g.f);
    for (long long t = blockIdx.x * (long long)NT + threadIdx.x; t < n;
         t += (long long)gridDim.x * NT) {
        int x, y, z;
        unflatten(g, t, x, y, z);
        if (!interior(g, x, y, z)) continue;
        const long long i = g.idx(x, y, z);
        const int cf = g.coord(g.f, x, y, z);
        unsigned int fl = 0;
        if (cf == 1 && bond_at(gf, f32, i - sf) > 0.0) fl |= 1u;
        if (cf == g.nf - 2 && bond_at(gf, f32, i) > 0.0) fl |= 2u;
        if (fl) atomicOr(flags + parent[i], fl);
    }
}

__global__ void lab_final(Geom g, const int *parent, const unsigned int *flags, uint8_t *cls) {
    const long long n = grid_nodes(g);
    for (long long t = blockIdx.x * (long long)NT + threadIdx.x; t < n;
         t += (long long)gridDim.x * NT) {
        int x, y, z;
        unflatten(g, t, x, y, z);
        const long long i = g.idx(x, y, z);
        const int cf = g.coord(g.f, x, y, z);
        uint8_t c;
        if (x >= g.nx) c = CLS_GHOST;
        else if (cf == 0) c = CLS_FACE_IN;
        else if (cf == g.nf - 1) c = CLS_FACE_OUT;
        else c = (uint8_t)flags[parent[i]];
        cls[i] = c;
    }
}

// ------------------------------------------------------------------ dead ends
// One round of stripping dead-end trees from the spanning clusters: a
// spanning node still present with at most one open bond to a present node
// (face nodes are always present) carries no current; it is removed in this
// round (pr = round) and remembers that neighbour (anchor) as the node whose
// pressure it takes.  Nodes removed in the same round still count as present
// for each other, so the result does not depend on thread order.
__global__ void prune_round_kernel(Geom g, const void *g0, const void *g1, const void *g2, int f32,
                                   const uint8_t *__restrict__ cls, unsigned int *pr, int *anchor,
                                   unsigned int round, unsigned int *count) {
    const long long n = grid_nodes(g);
    const void *gp[3] = {g0, g1, g2};
    unsigned int mine = 0;
    for (long long t = blockIdx.x * (long long)NT + threadIdx.x; t < n;
         t += (long long)gridDim.x * NT) {
        int x, y, z;
        unflatten(g, t, x, y, z);
        const long long i = g.idx(x, y, z);
        if (cls[i] != CLS_SPANNING || pr[i] != 0u) continue;
        int links = 0;
        long long last = -1;
        for (int d = 0; d < g.ndim; d++) {
            const int cd = g.coord(d, x, y, z);
            for (int side = 0; side < 2; side++) {
                const long long j = side ? g.down(i, d, cd) : g.up(i, d, cd);
                if (!(bond_at(gp[d], f32, side ? j : i) > 0.0)) continue;
                const uint8_t cj = cls[j];
                const unsigned int pj = *(volatile const unsigned int *)&pr[j];
                if (cj == CLS_FACE_IN || cj == CLS_FACE_OUT || (cj == CLS_SPANNING && (pj == 0u || pj == round))) {
                    links++;
                    last = j;
                }
            }
        }
        if (links <= 1) {
            pr[i] = round;
            anchor[i] = (int)last;
            mine++;
        }
    }
    if (mine) atomicAdd(count, mine);
}

// Mark the removed nodes CLS_DANGLING.
__global__ void prune_mark_kernel(Geom g, uint8_t *cls, const unsigned int *pr) {
    const long long n = grid_nodes(g);
    for (long long t = blockIdx.x * (long long)NT + threadIdx.x; t < n;
         t += (long long)gridDim.x * NT) {
        int x, y, z;
        unflatten(g, t, x, y, z);
        const long long i = g.idx(x, y, z);
        if (pr[i] != 0u) cls[i] = CLS_DANGLING;
    }
}

// Pointer jumping along the anchors: a removed node's anchor was present
// when it was removed (removed later, or never), so following anchors ends
// at a backbone or face node; each pass doubles the distance covered.
__global__ void prune_jump_kernel(Geom g, const unsigned int *pr, int *root) {
    const long long n = grid_nodes(g);
    for (long long t = blockIdx.x * (long long)NT + threadIdx.x; t < n;
         t += (long long)gridDim.x * NT) {
        int x, y, z;
        unflatten(g, t, x, y, z);
        const long long i = g.idx(x, y, z);
        if (pr[i] == 0u) continue;
        const int a = root[i];
        if (a >= 0 && pr[a] != 0u) root[i] = *(volatile const int *)&root[a];
    }
}

// A dead-end node's pressure is that of the node its tree hangs from.
__global__ void fill_dangling_kernel(Geom g, const int *__restrict__ root, double *x) {
    const long long n = grid_nodes(g);
    for (long long t = blockIdx.x * (long long)NT + threadIdx.x; t < n;
         t += (long long)gridDim.x * NT) {
        int cx, cy, cz;
        unflatten(g, t, cx, cy, cz);
        const long long i = g.idx(cx, cy, cz);
        const int r = root[i];
        if (r >= 0) x[i] = x[r];
    }
}

__global__ void backbone_kernel(Geom g, const uint8_t *cls, uint8_t *out) {
    const long long n = grid_nodes(g);
    for (long long t = blockIdx.x * (long long)NT + threadIdx.x; t < n;
         t += (long long)gridDim.x * NT) {
        int cx, cy, cz;
        unflatten(g, t, cx, cy, cz);
        if (cx >= g.nx) continue;
        out[cx + (long long)g.nx * (cy + (long long)g.ny * cz)] = cls[g.idx(cx, cy, cz)] == CLS_SPANNING;
    }
}

// ------------------------------------------------------------------ system
__global__ void build_system_kernel(Geom g, const void *g0, const void *g1, const void *g2,
                                    int f32, const uint8_t *__restrict__ cls,
                                    double *__restrict__ dis, double *__restrict__ x,
                                    SetupScal *ss, double *partials) {
    const long long n = grid_nodes(g);
    const void *gp[3] = {g0, g1, g2};
    const long long sf = g.stride(g.f);
    const double dP = g.p_in - g.p_out;
    double bb = 0.0, na = 0.0, ns = 0.0;
    for (long long t = blockIdx.x * (long long)NT + threadIdx.x; t < n;
         t += (long long)gridDim.x * NT) {
        int cx, cy, cz;
        unflatten(g, t, cx, cy, cz);
        const long long i = g.idx(cx, cy, cz);
        const uint8_t c = cls[i];
        const int cf = g.coord(g.f, cx, cy, cz);
        double xv = 0.0, dv = 0.0;
        switch (c) {
        case CLS_FACE_IN: case CLS_INLET: xv = g.p_in; break;
        case CLS_FACE_OUT: case CLS_OUTLET: xv = g.p_out; break;
        case CLS_SPANNING: case CLS_DANGLING: xv = g.p_in - dP * (double)cf / (double)(g.nf - 1); break;
        default: xv = 0.0;
        }
        if (c == CLS_DANGLING) na += 1.0;
        if (c == CLS_SPANNING) {
            // D_i over the bonds of the linear system: dead-end neighbours
            // are not part of it
            double D = 0.0;
            for (int d = 0; d < g.ndim; d++) {
                const int cd = g.coord(d, cx, cy, cz);
                const long long jp = g.up(i, d, cd), jm = g.down(i, d, cd);
                if (cls[jp] != CLS_DANGLING) D += bond_at(gp[d], f32, i);
                if (cls[jm] != CLS_DANGLING) D += bond_at(gp[d], f32, jm);
            }
            dv = 1.0 / sqrt(D);
            double b = 0.0;
            if (cf == 1) b += bond_at(gp[g.f], f32, i - sf) * g.p_in;
            if (cf == g.nf - 2) b += bond_at(gp[g.f], f32, i) * g.p_out;
            bb += b * b;
            na += 1.0;
            ns += 1.0;
        }
        x[i] = xv;
        dis[i] = dv;
    }
    double v[3] = {bb, na, ns};
    const int ops[3] = {RED_SUM, RED_SUM, RED_SUM};
    if (grid_reduce<3, NT>(v, ops, partials, &ss->counter) && threadIdx.x == 0) {
        ss->bb = v[0];
        ss->n_active = (unsigned long long)v[1];
        ss->n_solved = (unsigned long long)v[2];
    }
}

template <typename T>
__global__ void build_scaled_kernel(Geom g, const void *g0, const void *g1, const void *g2,
                                    int f32, const double *__restrict__ dis, T *s0, T *s1,
                                    T *s2) {
    const long long n = grid_nodes(g);
    const void *gp[3] = {g0, g1, g2};
    T *sp[3] = {s0, s1, s2};
    for (long long t = blockIdx.x * (long long)NT + threadIdx.x; t < n;
         t += (long long)gridDim.x * NT) {
        int x, y, z;
        unflatten(g, t, x, y, z);
        const long long i = g.idx(x, y, z);
        const double di = dis[i];
        for (int d = 0; d < g.ndim; d++) {
            const double dj = dis[g.up(i, d, g.coord(d, x, y, z))];
            const double gv = bond_at(gp[d], f32, i);
            sp[d][i] = (di > 0.0 && dj > 0.0) ? (T)(gv * di * dj) : T(0);
        }
    }
}

__global__ void apply_x0_kernel(Geom g, const uint8_t *cls, const double *x0c, double *x) {
    const long long n = grid_nodes(g);
    for (long long t = blockIdx.x * (long long)NT + threadIdx.x; t < n;
         t += (long long)gridDim.x * NT) {
        int cx, cy, cz;
        unflatten(g, t, cx, cy, cz);
        const long long i = g.idx(cx, cy, cz);
        if (cls[i] == CLS_SPANNING)
            x[i] = x0c[cx + (long long)g.nx * (cy + (long long)g.ny * cz)];
    }
}

__global__ void unpack_x_kernel(Geom g, const double *x, double *dst) {
    const long long n = grid_nodes(g);
    for (long long t = blockIdx.x * (long long)NT + threadIdx.x; t < n;
         t += (long long)gridDim.x * NT) {
        int cx, cy, cz;
        unflatten(g, t, cx, cy, cz);
        if (cx >= g.nx) continue;
        dst[cx + (long long)g.nx * (cy + (long long)g.ny * cz)] = x[g.idx(cx, cy, cz)];
    }
}

__global__ void unpack_labels_kernel(Geom g, const int *parent, const uint8_t *cls, int *label,
                                     uint8_t *cls_out) {
    const long long n = grid_nodes(g);
    for (long long t = blockIdx.x * (long long)NT + threadIdx.x; t < n;
         t += (long long)gridDim.x * NT) {
        int cx, cy, cz;
        unflatten(g, t, cx, cy, cz);
        if (cx >= g.nx) continue;
        const long long i = g.idx(cx, cy, cz);
        const long long o = cx + (long long)g.nx * (cy + (long long)g.ny * cz);
        const uint8_t c = cls[i];
        int lab;
        if (c == CLS_FACE_IN) lab = -1;
        else if (c == CLS_FACE_OUT) lab = -2;
        else {
            // padded root index -> compact node index
            const long long r = (long long)parent[i] - g.pad;
            const int rx = (int)(r % g.px);
            const long long ry = r / g.px;
            lab = (int)(rx + (long long)g.nx * ry);
        }
        if (label) label[o] = lab;
        if (cls_out) cls_out[o] = c == CLS_DANGLING ? (uint8_t)CLS_SPANNING : c;
    }
}

}  // namespace

cudaError_t launch_pack_bonds(const Geom &g, int d, const void *src, int src_f32, void *dst,
                              int dst_f32, unsigned int *bad, cudaStream_t st) {
    const int nb = blocks_for(grid_nodes(g));
    if (src_f32 && dst_f32)
        pack_kernel<float, float><<<nb, NT, 0, st>>>(g, d, (const float *)src, (float *)dst, bad);
    else if (src_f32)
        pack_kernel<float, double><<<nb, NT, 0, st>>>(g, d, (const float *)src, (double *)dst, bad);
    else if (dst_f32)
        pack_kernel<double, float><<<nb, NT, 0, st>>>(g, d, (const double *)src, (float *)dst, bad);
    else
        pack_kernel<double, double><<<nb, NT, 0, st>>>(g, d, (const double *)src, (double *)dst, bad);
    return cudaGetLastError();
}

cudaError_t launch_labels(const Geom &g, const void *const graw[3], int f32, int *parent,
                          unsigned int *flags, uint8_t *cls, cudaStream_t st) {
    const int nb = blocks_for(grid_nodes(g));
    lab_init<<<nb, NT, 0, st>>>(g, parent);
    lab_link<<<nb, NT, 0, st>>>(g, graw[0], graw[1], graw[2], f32, parent);
    lab_compress<<<nb, NT, 0, st>>>(g, parent);
    cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(unsigned int) * (size_t)g.len, st);
    if (e != cudaSuccess) return e;
    lab_flags<<<nb, NT, 0, st>>>(g, graw[g.f], f32, parent, flags);
    lab_final<<<nb, NT, 0, st>>>(g, parent, flags, cls);
    return cudaGetLastError();
}

cudaError_t launch_prune_round(const Geom &g, const void *const graw[3], int f32, const uint8_t *cls,
                               unsigned int *pr, int *anchor, unsigned int round, unsigned int *count,
                               cudaStream_t st) {
    prune_round_kernel<<<blocks_for(grid_nodes(g)), NT, 0, st>>>(g, graw[0], graw[1], graw[2], f32, cls, pr,
                                                                anchor, round, count);
    return cudaGetLastError();
}

cudaError_t launch_prune_finish(const Geom &g, uint8_t *cls, const unsigned int *pr, int *root,
                                int passes, cudaStream_t st) {
    const int nb = blocks_for(grid_nodes(g));
    prune_mark_kernel<<<nb, NT, 0, st>>>(g, cls, pr);
    for (int k = 0; k < passes; k++) prune_jump_kernel<<<nb, NT, 0, st>>>(g, pr, root);
    return cudaGetLastError();
}

cudaError_t launch_fill_dangling(const Geom &g, const int *root, double *x, cudaStream_t st) {
    long long nb = blocks_for(grid_nodes(g));
    fill_dangling_kernel<<<(int)nb, NT, 0, st>>>(g, root, x);
    return cudaGetLastError();
}

cudaError_t launch_backbone(const Geom &g, const uint8_t *cls, uint8_t *out, cudaStream_t st) {
    backbone_kernel<<<blocks_for(grid_nodes(g)), NT, 0, st>>>(g, cls, out);
    return cudaGetLastError();
}

cudaError_t launch_build_system(const Geom &g, const void *const graw[3], int f32,
                                const uint8_t *cls, double *dis, double *x, SetupScal *ss,
                                double *partials, cudaStream_t st) {
    const int nb = blocks_for(grid_nodes(g));
    build_system_kernel<<<nb, NT, 0, st>>>(g, graw[0], graw[1], graw[2], f32, cls, dis, x, ss,
                                            partials);
    return cudaGetLastError();
}

cudaError_t launch_build_scaled(const Geom &g, const void *const graw[3], int f32,
                                const double *dis, void *const gs[3], int gs_f32,
                                cudaStream_t st) {
    const int nb = blocks_for(grid_nodes(g));
    if (gs_f32)
        build_scaled_kernel<float><<<nb, NT, 0, st>>>(g, graw[0], graw[1], graw[2], f32, dis,
                                                      (float *)gs[0], (float *)gs[1],
                                                      (float *)gs[2]);
    else
        build_scaled_kernel<double><<<nb, NT, 0, st>>>(g, graw[0], graw[1], graw[2], f32, dis,
                                                       (double *)gs[0], (double *)gs[1],
                                                       (double *)gs[2]);
    return cudaGetLastError();
}

cudaError_t launch_apply_x0(const Geom &g, const uint8_t *cls, const double *x0c, double *x,
                            cudaStream_t st) {
    apply_x0_kernel<<<blocks_for(grid_nodes(g)), NT, 0, st>>>(g, cls, x0c, x);
    return cudaGetLastError();
}

cudaError_t launch_unpack_x(const Geom &g, const double *x, double *dst, cudaStream_t st) {
    unpack_x_kernel<<<blocks_for(grid_nodes(g)), NT, 0, st>>>(g, x, dst);
    return cudaGetLastError();
}

cudaError_t launch_unpack_labels(const Geom &g, const int *parent, const uint8_t *cls,
                                 int *label, uint8_t *cls_out, cudaStream_t st) {
    unpack_labels_kernel<<<blocks_for(grid_nodes(g)), NT, 0, st>>>(g, parent, cls, label,
                                                                   cls_out);
    return cudaGetLastError();
}

}  // namespace netsolve
