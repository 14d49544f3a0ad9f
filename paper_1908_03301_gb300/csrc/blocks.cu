// blocks.cu -- the current-carrying backbone of the spanning clusters on the
// device (Sec. V and VI.B: near the percolation threshold most of the
// spanning cluster carries no flow, and solving for it slows CG down).
//
// The graph: the spanning nodes still marked as unknowns ("core" nodes; all
// spanning nodes, as the round-based tree stripping does not run before this
// pass by default), joined by their open bonds; every inlet-face node taken
// together as one vertex A and every outlet-face node as one vertex B; and
// one extra edge A-B.  A bond carries current (for generic conductances) exactly when it lies
// on a path from A to B that visits no vertex twice, i.e. when it belongs to
// the biconnected component (block) of the extra edge.  Every other part of a
// spanning cluster hangs from that block by one node: a dead-end loop (or a
// tree growing from one).  Its pressure is that node's, and it leaves the
// linear system of Eq. 3 exactly as the dead-end trees do.
//
// The blocks follow Tarjan and Vishkin's parallel method (SIAM J. Comput.
// 14, 1985), written for the lattice:
//   1. a spanning tree: the edges whose union-find hook merged two sets
//      (every successful hook joins two different trees, so they form a
//      spanning tree of the connected graph); the extra edge A-B is hooked
//      first and so is always a tree edge;
//   2. an Euler tour of that tree, rooted at A and starting with A -> B: the
//      arcs leaving a lattice node are taken in direction order, those
//      leaving A or B in list order; list ranking by pointer jumping gives
//      every arc its position in the tour;
//   3. the preorder number pre(v) of every vertex (forward arcs counted by a
//      prefix sum) and its number of descendants nd(v), so the subtree of v
//      is the preorder range [pre(v), pre(v) + nd(v));
//   4. low(v) / high(v): the smallest / largest preorder number of a vertex
//      reached from v's subtree by one non-tree edge (or of the subtree
//      itself), a range minimum / maximum over that preorder range;
//   5. a union-find over the tree edges (each named by its child vertex):
//      a non-tree edge joins the tree edges of its two ends when neither end
//      is an ancestor of the other; the tree edge of w joins that of its
//      parent v (v not the root) when low(w) < pre(v) or
//      high(w) >= pre(v) + nd(v) -- w's subtree reaches around v;
//   6. the blocks are the resulting sets, a non-tree edge belonging to the
//      set of the tree edge of its end with the larger preorder number.  A
//      core node is in the backbone when its parent edge, one of its child
//      edges or one of its non-tree edges is in the set of A-B.
// Removed nodes take as their anchor the nearest backbone (or face) node on
// their tree path to A: the node their part hangs from.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "kernels.h"

namespace netsolve {
namespace {

constexpr int NT = 256;
constexpr int ST = 512;               // threads of the scan kernels
constexpr int SPER = 8;               // elements per thread in a scan block
constexpr int SCHUNK = ST * SPER;     // elements per scan block

inline int blocks_for(long long n) {
    long long b = (n + NT - 1) / NT;
    if (b > 152LL * 16) b = 152LL * 16;
    if (b < 1) b = 1;
    return (int)b;
}

#define GRID_LOOP(t, n) \
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (n); t += (long long)gridDim.x * blockDim.x)

__device__ inline double bond_at(const void *p, int f32, long long i) {
    return f32 ? (double)static_cast<const float *>(p)[i] : static_cast<const double *>(p)[i];
}

// ------------------------------------------------------------------ scan
// Exclusive prefix sum of n unsigned counts: block sums, one block scanning
// the block sums, then every block rescans its chunk.  out may alias in.
__device__ inline unsigned block_excl_scan(unsigned v, unsigned *total) {
    __shared__ unsigned wsum[ST / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    unsigned before = 0, all = 0;
    for (int w = 0; w < ST / 32; w++) {
        if (w < warp) before += wsum[w];
        all += wsum[w];
    }
    __syncthreads();
    if (total) *total = all;
    return before + incl - v;
}

__global__ void __launch_bounds__(ST) scan_sums_kernel(const unsigned *in, long long n, unsigned *bsum) {
    const long long base = (long long)blockIdx.x * SCHUNK + (long long)threadIdx.x * SPER;
    unsigned s = 0;
    for (int j = 0; j < SPER; j++)
        if (base + j < n) s += in[base + j];
    unsigned tot;
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(ST) scan_top_kernel(unsigned *bsum, int nb, unsigned *total) {
    __shared__ unsigned carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nb; b0 += ST) {
        const int b = b0 + threadIdx.x;
        const unsigned v = b < nb ? bsum[b] : 0u;
        unsigned tot;
        const unsigned ex = block_excl_scan(v, &tot);
        if (b < nb) bsum[b] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(ST) scan_apply_kernel(const unsigned *in, long long n, const unsigned *boff,
                                                        unsigned *out) {
    const long long base = (long long)blockIdx.x * SCHUNK + (long long)threadIdx.x * SPER;
    unsigned v[SPER], s = 0;
    for (int j = 0; j < SPER; j++) {
        v[j] = base + j < n ? in[base + j] : 0u;
        s += v[j];
    }
    unsigned run = boff[blockIdx.x] + block_excl_scan(s, nullptr);
    for (int j = 0; j < SPER; j++) {
        if (base + j < n) out[base + j] = run;
        run += v[j];
    }
}

// ------------------------------------------------------------------ union-find
__device__ inline int uf_find(const int *parent, int i) {
    int p = __ldcg(parent + i);
    while (p != i) {
        i = p;
        p = __ldcg(parent + i);
    }
    return i;
}

// Hooks the larger root under the smaller; true if this call merged two sets.
__device__ inline bool uf_union(int *parent, int a, int b) {
    while (true) {
        a = uf_find(parent, a);
        b = uf_find(parent, b);
        if (a == b) return false;
        if (a < b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicCAS(parent + a, a, b);
        if (old == a) return true;
        a = old;
    }
}

// ------------------------------------------------------------------ kernels
// Set when an existing bond touching an interior node is closed: without one,
// every interior node lies on a straight open path between the faces and the
// whole spanning set is the backbone.
__global__ void closed_bond_kernel(Geom g, const void *g0, const void *g1, const void *g2, int f32,
                                   const uint8_t *cls, unsigned *flag) {
    const void *gp[3] = {g0, g1, g2};
    const long long n = (long long)g.px * g.ny * g.nz;
    GRID_LOOP(t, n) {
        const long long i = g.pad + t;
        const uint8_t c = cls[i];
        if (c == CLS_GHOST || c == CLS_FACE_IN || c == CLS_FACE_OUT) continue;
        const int x = (int)(t % g.px);
        const long long r = t / g.px;
        const int y = (int)(r % g.ny), z = (int)(r / g.ny);
        bool closed = false;
        for (int d = 0; d < g.ndim; d++) {
            const int cd = g.coord(d, x, y, z);
            if (cd + 1 < g.extent(d) || g.periodic(d)) closed |= !(bond_at(gp[d], f32, i) > 0.0);
            if (cd > 0 || g.periodic(d)) closed |= !(bond_at(gp[d], f32, g.down(i, d, cd)) > 0.0);
        }
        if (closed) atomicOr(flag, 1u);
    }
}

__global__ void core_flag_kernel(Geom g, const uint8_t *cls, unsigned *flag) {
    const long long n = (long long)g.px * g.ny * g.nz;
    GRID_LOOP(t, n) flag[t] = cls[g.pad + t] == CLS_SPANNING ? 1u : 0u;
}

__global__ void core_index_kernel(Geom g, const uint8_t *cls, const unsigned *off, int *vmap, int *vlist) {
    const long long n = (long long)g.px * g.ny * g.nz;
    GRID_LOOP(t, n) {
        const long long i = g.pad + t;
        if (cls[i] == CLS_SPANNING) {
            vmap[i] = (int)off[t];
            vlist[off[t]] = (int)i;
        } else {
            vmap[i] = -1;
        }
    }
}

// nb[k][c] (k = 2d for +e_d, 2d+1 for -e_d): the vertex at the other end of
// an open bond -- a core node's index, A, B -- or -1.
__global__ void neighbour_kernel(Geom g, const void *g0, const void *g1, const void *g2, int f32,
                                 const uint8_t *cls, const int *vmap, const int *vlist, int V0, int *nb) {
    const void *gp[3] = {g0, g1, g2};
    const int A = V0, B = V0 + 1;
    GRID_LOOP(c, (long long)V0) {
        const long long i = vlist[c];
        const long long t = i - g.pad;
        const int x = (int)(t % g.px);
        const long long r = t / g.px;
        const int y = (int)(r % g.ny), z = (int)(r / g.ny);
        for (int d = 0; d < g.ndim; d++) {
            const int cd = g.coord(d, x, y, z);
            for (int side = 0; side < 2; side++) {
                int w = -1;
                const long long j = side ? g.down(i, d, cd) : g.up(i, d, cd);
                const bool exists = side ? (cd > 0 || g.periodic(d)) : (cd + 1 < g.extent(d) || g.periodic(d));
                if (exists && bond_at(gp[d], f32, side ? j : i) > 0.0) {
                    const uint8_t cj = cls[j];
                    w = cj == CLS_FACE_IN ? A : cj == CLS_FACE_OUT ? B : cj == CLS_SPANNING ? vmap[j] : -1;
                }
                nb[(long long)(2 * d + side) * V0 + c] = w;
            }
        }
    }
}

// hook_ab: the spanning-tree union-find starts with the extra edge A-B
// joined (B under A); the union-find over tree edges starts with every set
// alone.
__global__ void uf_init_kernel(int *uf, int V0, int hook_ab) {
    GRID_LOOP(v, (long long)V0 + 2) uf[v] = (hook_ab && v == V0 + 1) ? V0 : (int)v;
}

// Spanning tree: every lattice edge once (the +e_d side, or the side of the
// core node for a face edge); a hook that merged two sets makes it a tree
// edge (bit k of the node's tree mask, and the opposite bit of a core
// neighbour).
__global__ void tree_kernel(int V0, int K, const int *nb, int *uf, unsigned *tmask, unsigned *hooks) {
    unsigned mine = 0;
    GRID_LOOP(c, (long long)V0) {
        for (int k = 0; k < K; k++) {
            const int w = nb[(long long)k * V0 + c];
            if (w < 0 || (w < V0 && (k & 1))) continue;
            if (uf_union(uf, (int)c, w)) {
                mine++;
                atomicOr(&tmask[c], 1u << k);
                if (w < V0) atomicOr(&tmask[w], 1u << (k ^ 1));
            }
        }
    }
    if (mine) atomicAdd(hooks, mine);
}

// Face lists: flags of the core nodes whose tree edge in direction kf leads
// to the face vertex fv.
__global__ void face_flag_kernel(int V0, const int *nb, const unsigned *tmask, int kf, int fv, unsigned *flag) {
    GRID_LOOP(c, (long long)V0) flag[c] = ((tmask[c] >> kf) & 1u) && nb[(long long)kf * V0 + c] == fv ? 1u : 0u;
}

// L[0] = the other face; L[1 + off[c]] = c for flagged c; pos[c] = its slot.
__global__ void face_list_kernel(int V0, const unsigned *flag, const unsigned *off, int other, int *L, int *pos) {
    GRID_LOOP(c, (long long)V0) {
        if (flag[c]) {
            L[1 + off[c]] = (int)c;
            pos[c] = 1 + (int)off[c];
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) L[0] = other;
}

__global__ void popc_kernel(int V0, const unsigned *tmask, unsigned *cnt) {
    GRID_LOOP(c, (long long)V0) cnt[c] = __popc(tmask[c]);
}

struct Tour {
    int V0, K, f;
    const int *nb;
    const unsigned *tmask, *abase;
    const int *LA, *LB, *posA, *posB;
    int Tl, degA, degB;
    __device__ int arc(int c, int k) const {
        return (int)abase[c] + __popc(tmask[c] & ((1u << k) - 1u));
    }
    // the arc opposite to the arc leaving core node c in direction k
    __device__ int rev(int c, int k) const {
        const int w = nb[(long long)k * V0 + c];
        if (w == V0) return Tl + posA[c];
        if (w == V0 + 1) return Tl + degA + posB[c];
        return arc(w, k ^ 1);
    }
};

// succ(arc into v) = the arc leaving v after the reverse arc, cyclically.
__global__ void succ_core_kernel(Tour tr, int *succ) {
    GRID_LOOP(c, (long long)tr.V0) {
        const unsigned m = tr.tmask[c];
        for (int k = 0; k < tr.K; k++) {
            if (!((m >> k) & 1u)) continue;
            int k2 = k;
            for (int s = 1; s <= tr.K; s++) {
                const int kk = (k + s) % tr.K;
                if ((m >> kk) & 1u) {
                    k2 = kk;
                    break;
                }
            }
            succ[tr.rev((int)c, k)] = tr.arc((int)c, k2);
        }
    }
}

__global__ void succ_face_kernel(Tour tr, int *succ) {
    const int start = tr.Tl;  // A -> B
    GRID_LOOP(j, (long long)tr.degA) {
        const int r = j == 0 ? tr.Tl + tr.degA : tr.arc(tr.LA[j], 2 * tr.f + 1);
        const int nxt = tr.Tl + (int)((j + 1) % tr.degA);
        succ[r] = nxt == start ? -1 : nxt;  // the tour ends where it began
    }
    GRID_LOOP(j, (long long)tr.degB) {
        const int r = j == 0 ? tr.Tl : tr.arc(tr.LB[j], 2 * tr.f);
        succ[r] = tr.Tl + tr.degA + (int)((j + 1) % tr.degB);
    }
}

__global__ void rank_init_kernel(int T, const int *succ, int *nx, int *rk) {
    GRID_LOOP(a, (long long)T) {
        nx[a] = succ[a];
        rk[a] = succ[a] < 0 ? 0 : 1;
    }
}

__global__ void rank_jump_kernel(int T, const int *nx, const int *rk, int *nx2, int *rk2) {
    GRID_LOOP(a, (long long)T) {
        const int s = nx[a];
        if (s < 0) {
            nx2[a] = -1;
            rk2[a] = rk[a];
        } else {
            nx2[a] = nx[s];
            rk2[a] = rk[a] + rk[s];
        }
    }
}

// Parent of each core node: the tree neighbour whose arc into the node comes
// first in the tour.  F[pos] = 1 marks forward arcs (parent -> child).
__global__ void parent_kernel(Tour tr, int T, const int *rk, int *par, int *fpos, int *bpos, unsigned *F,
                              unsigned *bad) {
    GRID_LOOP(c, (long long)tr.V0) {
        const unsigned m = tr.tmask[c];
        int found = 0;
        for (int k = 0; k < tr.K; k++) {
            if (!((m >> k) & 1u)) continue;
            const int pa = T - 1 - rk[tr.arc((int)c, k)], pr = T - 1 - rk[tr.rev((int)c, k)];
            if (pa < 0 || pr < 0) {  // the arcs did not form one list: reported, nothing written
                found = -1;
                break;
            }
            if (pa > pr) {
                found++;
                par[c] = tr.nb[(long long)k * tr.V0 + c];
                fpos[c] = pr;
                bpos[c] = pa;
                F[pr] = 1u;
            }
        }
        if (found != 1) atomicOr(bad, 1u);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int B = tr.V0 + 1;
        par[B] = tr.V0;
        fpos[B] = 0;
        bpos[B] = T - 1 - rk[tr.Tl + tr.degA];
        F[0] = 1u;
        par[tr.V0] = -1;
    }
}

// pre(v) = number of forward arcs up to v's (exclusive scan + 1);
// nd(v) = half the tour positions between entering and leaving v, plus one.
__global__ void preorder_kernel(int V0, const unsigned *Fx, const int *fpos, const int *bpos, int *pre, int *nd) {
    GRID_LOOP(v, (long long)V0 + 2) {
        if (v == V0) {
            pre[v] = 0;
            nd[v] = V0 + 2;
        } else {
            pre[v] = (int)Fx[fpos[v]] + 1;
            nd[v] = (bpos[v] - fpos[v] + 1) / 2;
        }
    }
}

// Local low / high of every vertex, stored at its preorder number.
__global__ void local_kernel(int V0, int K, const int *nb, const unsigned *tmask, const int *pre, int *LO, int *HI) {
    GRID_LOOP(c, (long long)V0) {
        const int pc = pre[c];
        int lo = pc, hi = pc;
        const unsigned m = tmask[c];
        for (int k = 0; k < K; k++) {
            const int w = nb[(long long)k * V0 + c];
            if (w < 0 || ((m >> k) & 1u)) continue;
            const int pw = pre[w];
            lo = min(lo, pw);
            hi = max(hi, pw);
        }
        LO[pc] = lo;
        HI[pc] = hi;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        LO[0] = HI[0] = 0;  // A
        LO[1] = HI[1] = 1;  // B (never inside another vertex's range)
    }
}

// Sparse-table range minimum / maximum, one level at a time: cur holds the
// minima / maxima of the windows [i, i + 2^lev); vertices whose subtree
// length has floor(log2) = lev take their answer from this level.
__global__ void rmq_answer_kernel(int V, int lev, const int *pre, const int *nd, const int *curlo, const int *curhi,
                                  int *low, int *high) {
    GRID_LOOP(v, (long long)V) {
        const int L = nd[v];
        if (L < 1 || 31 - __clz(L) != lev) continue;
        const int l = pre[v], r = l + L - (1 << lev);
        if (l < 0 || (long long)l + L > V) continue;  // cannot happen for a valid tour
        low[v] = min(curlo[l], curlo[r]);
        high[v] = max(curhi[l], curhi[r]);
    }
}

__global__ void rmq_next_kernel(int V, int lev, const int *curlo, const int *curhi, int *nlo, int *nhi) {
    const int h = 1 << lev;
    GRID_LOOP(i, (long long)V) {
        if (i + h < V) {
            nlo[i] = min(curlo[i], curlo[i + h]);
            nhi[i] = max(curhi[i], curhi[i + h]);
        } else {
            nlo[i] = curlo[i];
            nhi[i] = curhi[i];
        }
    }
}

// Union-find over the tree edges (named by their child vertex).
__global__ void aux_kernel(int V0, int K, const int *nb, const unsigned *tmask, const int *par, const int *pre,
                           const int *nd, const int *low, const int *high, int *uf2) {
    const int A = V0;
    GRID_LOOP(c, (long long)V0) {
        const int v = par[c];
        if (v != A && (low[c] < pre[v] || high[c] >= pre[v] + nd[v])) uf_union(uf2, (int)c, v);
        const unsigned m = tmask[c];
        const int pc = pre[c], ec = pc + nd[c];
        for (int k = 0; k < K; k++) {
            const int w = nb[(long long)k * V0 + c];
            if (w < 0 || w == A || ((m >> k) & 1u)) continue;
            if (w < V0 && w < c) continue;  // each core-core edge once
            const int pw = pre[w];
            if (pw + nd[w] <= pc || ec <= pw) uf_union(uf2, (int)c, w);
        }
    }
}

__global__ void uf_compress_kernel(int V, int *uf) {
    GRID_LOOP(v, (long long)V) uf[v] = uf_find(uf, (int)v);
}

// Mark the core nodes outside the block of A-B as dead ends, anchored at
// their tree parent (a face node for A or B).
__global__ void mark_kernel(Geom g, int V0, int K, const int *nb, const unsigned *tmask, const int *par,
                            const int *pre, const int *uf2, const int *vlist, uint8_t *cls, int *root,
                            long long faceA, long long faceB, unsigned *removed) {
    const int target = uf2[V0 + 1];
    unsigned mine = 0;
    GRID_LOOP(c, (long long)V0) {
        bool in = uf2[c] == target;
        const unsigned m = tmask[c];
        for (int k = 0; k < K && !in; k++) {
            const int w = nb[(long long)k * V0 + c];
            if (w < 0) continue;
            if ((m >> k) & 1u) {
                if (w < V0 && par[w] == (int)c) in = uf2[w] == target;  // child edge
            } else {
                const int owner = pre[w] > pre[c] ? w : (int)c;
                in = uf2[owner] == target;
            }
        }
        if (!in) {
            const long long i = vlist[c];
            const int p = par[c];
            cls[i] = CLS_DANGLING;
            root[i] = (int)(p == V0 ? faceA : p == V0 + 1 ? faceB : vlist[p]);
            mine++;
        }
    }
    if (mine) atomicAdd(removed, mine);
}

// Anchors follow removed nodes until they reach a node still in the system
// (or a face); each pass at least halves every remaining chain.
__global__ void anchor_jump_kernel(Geom g, const uint8_t *cls, int *root) {
    const long long n = (long long)g.px * g.ny * g.nz;
    GRID_LOOP(t, n) {
        const long long i = g.pad + t;
        if (cls[i] != CLS_DANGLING) continue;
        const int a = root[i];
        if (a >= 0 && cls[a] == CLS_DANGLING) root[i] = *(volatile const int *)&root[a];
    }
}

// ------------------------------------------------------------------ host
struct Pool {
    cudaStream_t st;
    std::vector<void *> ptrs;
    cudaError_t err = cudaSuccess;
    template <typename T>
    T *get(long long n) {
        void *p = nullptr;
        if (err != cudaSuccess) return nullptr;
        err = cudaMallocAsync(&p, (size_t)(n < 1 ? 1 : n) * sizeof(T), st);
        if (err != cudaSuccess) return nullptr;
        ptrs.push_back(p);
        return (T *)p;
    }
    ~Pool() {
        for (void *p : ptrs) cudaFreeAsync(p, st);
    }
};

// Exclusive scan of n counts (in may equal out); *total_dev gets the sum.
cudaError_t scan(const unsigned *in, unsigned *out, long long n, unsigned *bsum, unsigned *total_dev, cudaStream_t st) {
    const int nb = (int)((n + SCHUNK - 1) / SCHUNK);
    if (nb < 1) return cudaMemsetAsync(total_dev, 0, sizeof(unsigned), st);
    scan_sums_kernel<<<nb, ST, 0, st>>>(in, n, bsum);
    scan_top_kernel<<<1, ST, 0, st>>>(bsum, nb, total_dev);
    scan_apply_kernel<<<nb, ST, 0, st>>>(in, n, bsum, out);
    return cudaGetLastError();
}

#define BK(x)                                   \
    do {                                        \
        cudaError_t e_ = (x);                   \
        if (e_ != cudaSuccess) return e_;       \
    } while (0)

}  // namespace

cudaError_t strip_dead_loops(const Geom &g, const void *const graw[3], int f32, uint8_t *cls, int *root,
                             int *vmap, long long *removed, int *internal_err, cudaStream_t st) {
    *removed = 0;
    *internal_err = 0;
    Pool pool{st};
    const long long n = (long long)g.px * g.ny * g.nz;
    const int nbk = blocks_for(n);
    // host-visible scalars: [0] closed-bond flag, [1] V0, [2] hooks, [3] degA-1,
    // [4] degB-1, [5] Tl, [6] parent check, [7] removed, [8..] scan totals
    unsigned *dsc = pool.get<unsigned>(16);
    unsigned hsc[16];
    BK(pool.err);
    BK(cudaMemsetAsync(dsc, 0, 16 * sizeof(unsigned), st));
    closed_bond_kernel<<<nbk, NT, 0, st>>>(g, graw[0], graw[1], graw[2], f32, cls, dsc + 0);
    unsigned *flag = pool.get<unsigned>(n);
    unsigned *bsum = pool.get<unsigned>((2 * n + 2) / SCHUNK + 2);  // scans of up to 2n + 2 entries
    BK(pool.err);
    core_flag_kernel<<<nbk, NT, 0, st>>>(g, cls, flag);
    BK(scan(flag, flag, n, bsum, dsc + 1, st));
    BK(cudaMemcpyAsync(hsc, dsc, 2 * sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    BK(cudaStreamSynchronize(st));
    const long long V0l = hsc[1];
    if (hsc[0] == 0u || V0l == 0) return cudaSuccess;   // nothing can hang off
    if (V0l > (1LL << 29)) return cudaSuccess;          // arc indices would not fit in int
    const int V0 = (int)V0l, V = V0 + 2, K = 2 * g.ndim;
    int *vlist = pool.get<int>(V0);
    int *nb = pool.get<int>((long long)K * V0);
    int *uf = pool.get<int>(V);
    unsigned *tmask = pool.get<unsigned>(V0);
    BK(pool.err);
    BK(cudaMemsetAsync(vmap, 0xFF, sizeof(int) * (size_t)g.len, st));
    core_index_kernel<<<nbk, NT, 0, st>>>(g, cls, flag, vmap, vlist);
    const int nbv = blocks_for(V0);
    neighbour_kernel<<<nbv, NT, 0, st>>>(g, graw[0], graw[1], graw[2], f32, cls, vmap, vlist, V0, nb);
    uf_init_kernel<<<blocks_for(V), NT, 0, st>>>(uf, V0, 1);
    BK(cudaMemsetAsync(tmask, 0, sizeof(unsigned) * (size_t)V0, st));
    tree_kernel<<<nbv, NT, 0, st>>>(V0, K, nb, uf, tmask, dsc + 2);
    // face lists (A: tree edges in direction -f, B: +f)
    const int kA = 2 * g.f + 1, kB = 2 * g.f;
    unsigned *fa = pool.get<unsigned>(V0);
    unsigned *fb = pool.get<unsigned>(V0);
    unsigned *cnt = pool.get<unsigned>(V0);
    int *posA = pool.get<int>(V0);
    int *posB = pool.get<int>(V0);
    BK(pool.err);
    face_flag_kernel<<<nbv, NT, 0, st>>>(V0, nb, tmask, kA, V0, fa);
    face_flag_kernel<<<nbv, NT, 0, st>>>(V0, nb, tmask, kB, V0 + 1, fb);
    popc_kernel<<<nbv, NT, 0, st>>>(V0, tmask, cnt);
    // the flags are kept for the list kernels: scan into the count buffers
    unsigned *offA = flag, *offB = flag + V0;  // the core flags are no longer needed
    if (n < 2LL * V0) {
        offA = pool.get<unsigned>(V0);
        offB = pool.get<unsigned>(V0);
        BK(pool.err);
    }
    BK(scan(fa, offA, V0, bsum, dsc + 3, st));
    BK(scan(fb, offB, V0, bsum, dsc + 4, st));
    BK(scan(cnt, cnt, V0, bsum, dsc + 5, st));
    BK(cudaMemcpyAsync(hsc, dsc, 8 * sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    BK(cudaStreamSynchronize(st));
    const int degA = (int)hsc[3] + 1, degB = (int)hsc[4] + 1, Tl = (int)hsc[5];
    const long long T = (long long)Tl + degA + degB;
    if ((long long)hsc[2] != V0 || T != 2LL * (V - 1)) {
        *internal_err = 1;  // the graph was not connected: not a set of spanning clusters
        return cudaSuccess;
    }
    int *LA = pool.get<int>(degA);
    int *LB = pool.get<int>(degB);
    BK(pool.err);
    face_list_kernel<<<nbv, NT, 0, st>>>(V0, fa, offA, V0 + 1, LA, posA);
    face_list_kernel<<<nbv, NT, 0, st>>>(V0, fb, offB, V0, LB, posB);
    Tour tr{V0, K, g.f, nb, tmask, cnt, LA, LB, posA, posB, Tl, degA, degB};
    const int Ti = (int)T;
    int *succ = pool.get<int>(T);
    int *nx = pool.get<int>(T), *rk = pool.get<int>(T), *nx2 = pool.get<int>(T), *rk2 = pool.get<int>(T);
    BK(pool.err);
    succ_core_kernel<<<nbv, NT, 0, st>>>(tr, succ);
    succ_face_kernel<<<blocks_for(std::max(degA, degB)), NT, 0, st>>>(tr, succ);
    const int nbt = blocks_for(T);
    rank_init_kernel<<<nbt, NT, 0, st>>>(Ti, succ, nx, rk);
    int rounds = 0;
    while ((1LL << rounds) < T) rounds++;
    for (int r = 0; r < rounds; r++) {
        rank_jump_kernel<<<nbt, NT, 0, st>>>(Ti, nx, rk, nx2, rk2);
        std::swap(nx, nx2);
        std::swap(rk, rk2);
    }
    // parents, forward arcs, preorder numbers and subtree sizes
    int *par = pool.get<int>(V), *fpos = pool.get<int>(V), *bpos = pool.get<int>(V);
    unsigned *F = (unsigned *)succ;  // succ is no longer needed
    int *pre = pool.get<int>(V), *ndv = pool.get<int>(V);
    BK(pool.err);
    BK(cudaMemsetAsync(F, 0, sizeof(unsigned) * (size_t)T, st));
    parent_kernel<<<nbv, NT, 0, st>>>(tr, Ti, rk, par, fpos, bpos, F, dsc + 6);
    BK(scan(F, F, T, bsum, dsc + 8, st));
    BK(cudaMemcpyAsync(hsc, dsc, 9 * sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    BK(cudaStreamSynchronize(st));
    if (hsc[6] || (long long)hsc[8] != V - 1) {
        *internal_err = 2;  // a core node without exactly one parent, or a broken tour
        return cudaSuccess;
    }
    preorder_kernel<<<blocks_for(V), NT, 0, st>>>(V0, F, fpos, bpos, pre, ndv);
    // low / high
    int *lo = nx, *hi = nx2, *lo2 = rk2, *hi2 = (int *)fpos;  // reuse the ranking buffers (T >= V)
    int *low = pool.get<int>(V), *high = pool.get<int>(V);
    BK(pool.err);
    local_kernel<<<nbv, NT, 0, st>>>(V0, K, nb, tmask, pre, lo, hi);
    const int nbV = blocks_for(V);
    for (int lev = 0; (1LL << lev) <= V; lev++) {
        rmq_answer_kernel<<<nbV, NT, 0, st>>>(V, lev, pre, ndv, lo, hi, low, high);
        if ((1LL << (lev + 1)) > V) break;
        rmq_next_kernel<<<nbV, NT, 0, st>>>(V, lev, lo, hi, lo2, hi2);
        std::swap(lo, lo2);
        std::swap(hi, hi2);
    }
    // blocks: union-find over the tree edges, then the nodes of A-B's set
    int *uf2 = uf;
    uf_init_kernel<<<blocks_for(V), NT, 0, st>>>(uf2, V0, 0);
    aux_kernel<<<nbv, NT, 0, st>>>(V0, K, nb, tmask, par, pre, ndv, low, high, uf2);
    uf_compress_kernel<<<blocks_for(V), NT, 0, st>>>(V, uf2);
    const long long faceA = g.idx(0, 0, 0);
    int cB[3] = {0, 0, 0};
    cB[g.f] = g.nf - 1;
    const long long faceB = g.idx(cB[0], cB[1], cB[2]);
    mark_kernel<<<nbv, NT, 0, st>>>(g, V0, K, nb, tmask, par, pre, uf2, vlist, cls, root, faceA, faceB, dsc + 7);
    int passes = 1;
    while ((1LL << passes) <= V) passes++;
    for (int p = 0; p < passes + 1; p++) anchor_jump_kernel<<<nbk, NT, 0, st>>>(g, cls, root);
    BK(cudaGetLastError());
    BK(cudaMemcpyAsync(hsc, dsc, 8 * sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    BK(cudaStreamSynchronize(st));
    *removed = hsc[7];
    return cudaSuccess;
}

}  // namespace netsolve
