// The odometry start's spanning forest and its rooting, on the device.
//
// The paper starts from a chordal initialisation it does not define; the
// start used here composes the relative measurements along a spanning
// forest: an edge joins the forest when it links two components, edges taken
// in input order (Kruskal with the edge index as the weight), and each
// component is rooted at its lowest vertex, which gets the identity pose.
//
// Forest.  With every weight distinct the minimum spanning forest is unique,
// so Boruvka's rounds find Kruskal's forest: each component picks its
// lowest-index edge to another component (atomicMin), hooks to that
// component (a pair that picked the same edge keeps the lower id as root),
// the hooks are flattened by pointer jumping, and the rounds repeat until no
// edge links two components.
//
// Rooting.  The Euler tour of each tree (arc u->v followed by the arc after
// v->u in v's cyclic list of arcs), cut just before the root's first arc, is
// ranked by pointer jumping (distance to the tour's end); a tree edge's arc
// that the tour walks first points from parent to child.  That gives every
// vertex its parent and the edge to it, which the composition kernels of
// pradmm_setup.cu turn into poses.  The endpoints come from the out-edge CSR
// (the tail of a slot is its row, the head its column).
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

#include "pradmm_internal.h"

namespace pradmm {
namespace {

inline int grid_for(int64_t work) {
    const int64_t want = (work + 255) / 256;
    return (int)(want < 152 * 8 ? (want > 0 ? want : 1) : 152 * 8);
}

#define GRID_STRIDE(i, count) \
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (count); i += (int64_t)gridDim.x * blockDim.x)

__global__ void __launch_bounds__(256) k_fill(int32_t* a, int64_t n, int32_t v) {
    GRID_STRIDE(i, n) a[i] = v;
}

__global__ void __launch_bounds__(256) k_iota32(int32_t* a, int64_t n) {
    GRID_STRIDE(i, n) a[i] = (int32_t)i;
}

// the input edges' endpoints from the out-edge CSR (owner = each slot's tail)
__global__ void __launch_bounds__(256) k_edge_ends(const int32_t* __restrict__ out_edge,
                                                   const int32_t* __restrict__ owner,
                                                   const int32_t* __restrict__ out_idx, int64_t m, int32_t* src,
                                                   int32_t* dst) {
    GRID_STRIDE(k, m) {
        const int32_t e = out_edge[k];
        src[e] = owner[k];
        dst[e] = out_idx[k];
    }
}

// best[c] = the lowest edge index between component c and another one
__global__ void __launch_bounds__(256) k_bor_min(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                                                 int64_t m, const int32_t* __restrict__ comp, int32_t* best) {
    GRID_STRIDE(e, m) {
        const int32_t a = comp[src[e]], b = comp[dst[e]];
        if (a != b) {
            atomicMin(best + a, (int32_t)e);
            atomicMin(best + b, (int32_t)e);
        }
    }
}

// Every component root c with an edge out hooks to the component at its
// other end (the lower of a mutual pair stays a root) and marks the edge;
// *added counts the hooks.
__global__ void __launch_bounds__(256) k_bor_hook(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                                                  const int32_t* __restrict__ comp, const int32_t* __restrict__ best,
                                                  int64_t n, int32_t* hook, int32_t* in_tree, int32_t* added) {
    GRID_STRIDE(c, n) {
        int32_t h = (int32_t)c;
        if (comp[c] == c && best[c] != INT_MAX) {
            const int32_t e = best[c];
            const int32_t a = comp[src[e]], b = comp[dst[e]];
            const int32_t other = a == c ? b : a;
            in_tree[e] = 1;
            if (!(best[other] == e && other > c)) h = other;
            atomicAdd(added, 1);
        }
        hook[c] = h;
    }
}

// one pointer-jumping step of the hooks (double buffered)
__global__ void __launch_bounds__(256) k_jump(const int32_t* __restrict__ in, int64_t n, int32_t* out) {
    GRID_STRIDE(c, n) out[c] = in[in[c]];
}

__global__ void __launch_bounds__(256) k_relabel(int32_t* comp, int64_t n, const int32_t* __restrict__ hook) {
    GRID_STRIDE(v, n) comp[v] = hook[comp[v]];
}

// lowest[c] = the lowest vertex of component c.  One big component would
// put every vertex's atomic on one word: the lanes of a warp that share a
// label send only their lowest vertex (the first such lane: v grows with
// the lane), and only while the word holds a higher one.
__global__ void __launch_bounds__(256) k_lowest(const int32_t* __restrict__ comp, int64_t n, int32_t* lowest) {
    GRID_STRIDE(v, n) {
        const int32_t c = comp[v];
        const unsigned same = __match_any_sync(__activemask(), c);
        if ((int)(threadIdx.x & 31) == __ffs(same) - 1 && *((volatile int32_t*)(lowest + c)) > (int32_t)v)
            atomicMin(lowest + c, (int32_t)v);
    }
}

// tree[k] = the k-th tree edge in edge order (pos = inclusive scan of in_tree)
__global__ void __launch_bounds__(256) k_compact(const int32_t* __restrict__ in_tree, const int32_t* __restrict__ pos,
                                                 int64_t m, int32_t* tree) {
    GRID_STRIDE(e, m) if (in_tree[e]) tree[pos[e] - 1] = (int32_t)e;
}

// Arcs of tree edge k = tree[k]: 2k from its tail to its head, 2k + 1 back.
__device__ __forceinline__ int32_t arc_source(const int32_t* src, const int32_t* dst, const int32_t* tree, int32_t a) {
    const int32_t e = tree[a >> 1];
    return (a & 1) ? dst[e] : src[e];
}

__global__ void __launch_bounds__(256) k_arc_degree(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                                                    const int32_t* __restrict__ tree, int64_t arcs, int32_t* cnt1) {
    GRID_STRIDE(a, arcs) atomicAdd(cnt1 + arc_source(src, dst, tree, (int32_t)a), 1);
}

__global__ void __launch_bounds__(256) k_arc_place(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                                                   const int32_t* __restrict__ tree, int64_t arcs,
                                                   const int32_t* __restrict__ ptr, int32_t* fill, int32_t* list,
                                                   int32_t* aslot) {
    GRID_STRIDE(a, arcs) {
        const int32_t u = arc_source(src, dst, tree, (int32_t)a);
        const int32_t s = ptr[u] + atomicAdd(fill + u, 1);
        list[s] = (int32_t)a;
        aslot[a] = s;
    }
}

// next(u->v) = the arc after v->u in v's cyclic list; the tour of each tree
// is cut before its root's first arc (next = -1 there)
__global__ void __launch_bounds__(256) k_arc_next(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                                                  const int32_t* __restrict__ tree, int64_t arcs,
                                                  const int32_t* __restrict__ ptr, const int32_t* __restrict__ list,
                                                  const int32_t* __restrict__ aslot, int32_t* next) {
    GRID_STRIDE(a, arcs) {
        const int32_t tw = (int32_t)a ^ 1;
        const int32_t v = arc_source(src, dst, tree, tw);
        const int32_t b = ptr[v], deg = ptr[v + 1] - b;
        const int32_t pos = aslot[tw] - b + 1;
        next[a] = list[b + (pos == deg ? 0 : pos)];
    }
}

__global__ void __launch_bounds__(256) k_arc_cut(const int32_t* __restrict__ comp, const int32_t* __restrict__ lowest,
                                                 int64_t n, const int32_t* __restrict__ ptr,
                                                 const int32_t* __restrict__ list, int32_t* next) {
    GRID_STRIDE(r, n) {
        if (lowest[comp[r]] != r) continue;
        const int32_t b = ptr[r], deg = ptr[r + 1] - b;
        if (deg > 0) next[list[b + deg - 1] ^ 1] = -1;
    }
}

__global__ void __launch_bounds__(256) k_rank_init(const int32_t* __restrict__ next, int64_t arcs, int32_t* rank) {
    GRID_STRIDE(a, arcs) rank[a] = next[a] < 0 ? 0 : 1;
}

// one list-ranking step: rank = distance (in arcs) to the tour's end
__global__ void __launch_bounds__(256) k_rank_jump(const int32_t* __restrict__ nx_in, const int32_t* __restrict__ rk_in,
                                                   int64_t arcs, int32_t* nx_out, int32_t* rk_out) {
    GRID_STRIDE(a, arcs) {
        const int32_t x = nx_in[a];
        if (x >= 0) {
            rk_out[a] = rk_in[a] + rk_in[x];
            nx_out[a] = nx_in[x];
        } else {
            rk_out[a] = rk_in[a];
            nx_out[a] = -1;
        }
    }
}

// the arc walked first (the larger distance to the end) points parent -> child
__global__ void __launch_bounds__(256) k_orient(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                                                const int32_t* __restrict__ tree, int64_t nt,
                                                const int32_t* __restrict__ rank, int32_t* par, int32_t* pedge) {
    GRID_STRIDE(k, nt) {
        const int32_t e = tree[k];
        if (rank[2 * k] > rank[2 * k + 1]) {  // tail -> head first: the head is the child
            par[dst[e]] = src[e];
            pedge[dst[e]] = e;
        } else {
            par[src[e]] = dst[e];
            pedge[src[e]] = -(e + 2);
        }
    }
}

inline int ceil_log2(int64_t x) {
    int r = 0;
    while (((int64_t)1 << r) < x) ++r;
    return r;
}

}  // namespace

size_t forest_scratch_ints(int64_t n, int64_t m) {
    return (size_t)(20 * n + 4 * m + 1) + (size_t)((n > m ? n : m) + 1023) / 1024 + 72;
}

cudaError_t launch_forest(const int32_t* out_ptr, const int32_t* out_idx, const int32_t* out_edge, int64_t n,
                          int64_t m, int32_t* scratch, int32_t* par, int32_t* pedge, cudaStream_t st) {
    cudaError_t err;
#define FQ(call)                                       \
    do {                                               \
        if ((err = (call)) != cudaSuccess) return err; \
    } while (0)
    int32_t* comp = scratch;          // n: component label (its current root)
    int32_t* hook = comp + n;         // n
    int32_t* hook2 = hook + n;        // n
    int32_t* best = hook2 + n;        // n
    int32_t* lowest = best + n;       // n
    int32_t* fill = lowest + n;       // n
    int32_t* aptr = fill + n;         // n + 1: arcs' CSR by source vertex
    int32_t* tree = aptr + n + 1;     // n: tree edges in edge order
    int32_t* list = tree + n;         // 2n: arcs by source vertex
    int32_t* aslot = list + 2 * n;    // 2n: slot of each arc in list
    int32_t* nx0 = aslot + 2 * n;     // 2n
    int32_t* nx1 = nx0 + 2 * n;       // 2n
    int32_t* rk0 = nx1 + 2 * n;       // 2n
    int32_t* rk1 = rk0 + 2 * n;       // 2n
    int32_t* in_tree = rk1 + 2 * n;   // m
    int32_t* pos = in_tree + m;       // m (first the slots' tails)
    int32_t* src = pos + m;           // m: tail of input edge e
    int32_t* dst = src + m;           // m: head of input edge e
    int32_t* cnt = dst + m;           // 64
    int32_t* sums = cnt + 64;         // (max(n, m) + 1023) / 1024
    const int gn = grid_for(n), gm = grid_for(m);
    k_iota32<<<gn, 256, 0, st>>>(comp, n);
    k_fill<<<gn, 256, 0, st>>>(par, n, -1);
    k_fill<<<gn, 256, 0, st>>>(pedge, n, -1);
    if (m == 0) return cudaGetLastError();
    FQ(launch_slot_owner(out_ptr, n, pos, st));
    k_edge_ends<<<gm, 256, 0, st>>>(out_edge, pos, out_idx, m, src, dst);
    FQ(cudaMemsetAsync(in_tree, 0, sizeof(int32_t) * m, st));
    // Boruvka rounds; the components at least halve every round
    const int jumps = ceil_log2(n) + 1;
    for (int round = 0;; ++round) {
        if (round > 64) return cudaErrorUnknown;
        k_fill<<<gn, 256, 0, st>>>(best, n, INT_MAX);
        FQ(cudaMemsetAsync(cnt, 0, sizeof(int32_t), st));
        k_bor_min<<<gm, 256, 0, st>>>(src, dst, m, comp, best);
        k_bor_hook<<<gn, 256, 0, st>>>(src, dst, comp, best, n, hook, in_tree, cnt);
        int32_t added = 0;
        FQ(cudaMemcpyAsync(&added, cnt, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        FQ(cudaStreamSynchronize(st));
        if (added == 0) break;
        int32_t *a = hook, *b = hook2;
        for (int j = 0; j < jumps; ++j) {
            k_jump<<<gn, 256, 0, st>>>(a, n, b);
            int32_t* t = a;
            a = b;
            b = t;
        }
        k_relabel<<<gn, 256, 0, st>>>(comp, n, a);
    }
    // the roots: the lowest vertex of every component
    k_fill<<<gn, 256, 0, st>>>(lowest, n, INT_MAX);
    k_lowest<<<gn, 256, 0, st>>>(comp, n, lowest);
    // the tree edges in edge order
    FQ(cudaMemcpyAsync(pos, in_tree, sizeof(int32_t) * m, cudaMemcpyDeviceToDevice, st));
    FQ(inclusive_scan_i32(pos, m, sums, st));
    int32_t nt = 0;
    FQ(cudaMemcpyAsync(&nt, pos + m - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    FQ(cudaStreamSynchronize(st));
    if (nt == 0) return cudaGetLastError();
    k_compact<<<gm, 256, 0, st>>>(in_tree, pos, m, tree);
    // the arcs' cyclic lists and the Euler tours, cut at the roots
    const int64_t arcs = 2 * (int64_t)nt;
    const int ga = grid_for(arcs);
    FQ(cudaMemsetAsync(aptr, 0, sizeof(int32_t) * (n + 1), st));
    FQ(cudaMemsetAsync(fill, 0, sizeof(int32_t) * n, st));
    k_arc_degree<<<ga, 256, 0, st>>>(src, dst, tree, arcs, aptr + 1);
    FQ(inclusive_scan_i32(aptr + 1, n, sums, st));
    k_arc_place<<<ga, 256, 0, st>>>(src, dst, tree, arcs, aptr, fill, list, aslot);
    k_arc_next<<<ga, 256, 0, st>>>(src, dst, tree, arcs, aptr, list, aslot, nx0);
    k_arc_cut<<<gn, 256, 0, st>>>(comp, lowest, n, aptr, list, nx0);
    // list ranking
    k_rank_init<<<ga, 256, 0, st>>>(nx0, arcs, rk0);
    int32_t *nxa = nx0, *nxb = nx1, *rka = rk0, *rkb = rk1;
    const int rj = ceil_log2(arcs) + 1;
    for (int j = 0; j < rj; ++j) {
        k_rank_jump<<<ga, 256, 0, st>>>(nxa, rka, arcs, nxb, rkb);
        int32_t* t = nxa;
        nxa = nxb;
        nxb = t;
        t = rka;
        rka = rkb;
        rkb = t;
    }
    k_orient<<<grid_for(nt), 256, 0, st>>>(src, dst, tree, nt, rka, par, pedge);
    return cudaGetLastError();
#undef FQ
}

}  // namespace pradmm
