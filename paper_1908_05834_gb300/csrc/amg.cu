// Aggregation multigrid preconditioner for the minimisation's linear system.
//
// The system (A-hat A-hat^T + W) y = F of the penalised minimisation is, after
// flipping the sign of the column unknowns (S = diag(1 rows, -1 columns)), the
// M-matrix L = [[D_r, -W], [-W^T, D_c]] + diag(w): a weighted graph Laplacian
// of the bipartite row/column graph (edge weights a_ij^2) plus a small
// positive shift.  Its conditioning is poor on two counts: mesh-scale smooth
// modes, and weak links (near-tangent ball overlaps give a_ij that are orders
// of magnitude below the row's main entries).  A cluster of nodes held to the
// rest only by weak links has a near-null mode (constant on the cluster); the
// coarse levels keep that mode only if no aggregate straddles the weak links.
// So the aggregation follows strong links alone:
//   - an edge is strong when its weight is at least kStrength sqrt(d_i d_j);
//   - each level pairs every node with its heaviest strong neighbour when the
//     choice is mutual (kHandshakes rounds, each among the nodes still
//     unpaired); a node left unpaired joins the aggregate of its heaviest
//     strong neighbour when that one is paired, else stays single;
//   - a node without any off-diagonal entry (a whole connected component
//     that has collapsed into one node, or an isolated row or column) leaves
//     the hierarchy: its equation is solved exactly by the smoother (weight 1
//     instead of kOmega) and it has no coarse counterpart;
//   - so does a node whose off-diagonal weights sum to at most kDominant of
//     its diagonal (a constraint held by its shift: in the minimisation's late
//     iterations, one priced by the linear part of the penalty, or one whose
//     entries all sit at a bound).  The smoother alone reduces its error by
//     about that ratio per sweep, and left in, such nodes stall the coarsening
//     (they have no strong neighbour, so every level keeps them as singletons
//     and the coarsest level stays large).  Its edges to the nodes that stay
//     are carried into their coarse shift, so the coarse operator is still the
//     Galerkin product;
//   - coarsening stops when a level would keep more than kStall of its
//     remaining nodes, or has at most kCoarsest of them;
//   - the coarse operator is the Galerkin product P^T L P for the piecewise-
//     constant P of the aggregates (coarse edge = sum of fine edges between
//     two aggregates).  Its diagonal is formed as the coarse node's excess
//     (the sum of its members' shifts) plus the sum of its coarse edge
//     weights, not as member diagonals minus internal edges: the shift is
//     ~1e-14 of the edge weights and the subtraction would cancel it away;
//   - a symmetric V-cycle (one damped-Jacobi sweep before and after the
//     coarse correction, Jacobi sweeps on the coarsest level) is applied as
//     the preconditioner of the conjugate gradients; per level it takes three
//     kernels (pre-smoothing fused with the residual, restriction,
//     prolongation fused with post-smoothing).
// Every sum runs in a fixed order, so the hierarchy and its application are
// deterministic.
#include <math.h>

#include "amg.cuh"
#include "device.cuh"

namespace bchar {

#define GRID_STRIDE(i, n)                                                                    \
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < (n); \
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)

constexpr int kCoarseCap = 384;       // neighbours a coarse node may collect before merging
constexpr int64_t kCoarsest = 128;    // stop coarsening at this many nodes
constexpr int64_t kOneBlock = 4096;   // levels up to this size are cycled by one block
constexpr int kMaxLevels = 40;
constexpr int kHandshakes = 4;        // matching rounds per level
constexpr double kStall = 0.9;        // stop coarsening when a level keeps this fraction of nodes
constexpr double kOmega = 0.9;        // Jacobi damping (rows with off-diagonal entries)
constexpr double kStrength = 0.1;     // strong edge: w_ij >= kStrength sqrt(d_i d_j)
constexpr double kAttach = 0.25;      // a leftover node follows an edge carrying this share of its diagonal
constexpr double kDominant = 0.25;    // a node leaves the hierarchy when its off-diagonal sum is this share of its diagonal
constexpr int kCoarsestSweeps = 40;   // sweeps of a one-block coarsest level
constexpr int64_t kFuseBelow = 1 << 19;  // levels smaller than this fuse prolongation with smoothing
constexpr int kLargeCoarsestSweeps = 20;
constexpr int kDominantSweeps = 4;

// ---------------------------------------------------------------- level 0

// Row node l < nc: its entries come from row l of A (columns nc + j);
// column node nc + j: from column j (rows i).  Values -a_ij^2.
__global__ void k_level0_ptr(int64_t nc, int64_t nnz, const int64_t *row_ptr, const int64_t *col_ptr,
                             int64_t *ptr0) {
    dep_enter();
    GRID_STRIDE(l, 2 * nc + 1) ptr0[l] = l <= nc ? row_ptr[l] : nnz + col_ptr[l - nc];
}

__global__ void k_level0_fill(int64_t nc, const int64_t *row_ptr, const int32_t *col, const int64_t *col_ptr,
                              const int32_t *csc_row, const double *a2, const double *a2c, const int64_t *ptr0,
                              int32_t *col0, double *val0) {
    dep_enter();
    GRID_STRIDE(l, 2 * nc) {
        int64_t dst = ptr0[l];
        if (l < nc) {
            for (int64_t e = row_ptr[l]; e < row_ptr[l + 1]; ++e, ++dst) {
                col0[dst] = static_cast<int32_t>(nc + col[e]);
                val0[dst] = -a2[e];
            }
        } else {
            const int64_t j = l - nc;
            for (int64_t p = col_ptr[j]; p < col_ptr[j + 1]; ++p, ++dst) {
                col0[dst] = csc_row[p];
                val0[dst] = -a2c[p];
            }
        }
    }
}

// ---------------------------------------------------------------- matching
//
// Neighbours are ranked by (weight class, edge hash): the class is the binary
// exponent of the weight, so weights within a factor of two rank equal and a
// symmetric hash of the edge decides between them.  Ranking by the exact
// weight fails on smooth flows: the weights then grow monotonically along the
// strong chains of the graph, every node points the same way and almost no
// choice is mutual (on a uniform 261^2 mesh one level kept 92 % of its nodes).
// Equal classes with hashed order put local maxima everywhere.

__device__ __forceinline__ uint32_t edge_hash(int64_t i, int64_t j) {
    const uint64_t a = static_cast<uint64_t>(i < j ? i : j), b = static_cast<uint64_t>(i < j ? j : i);
    uint64_t x = (a * 0x9E3779B1ull + b * 0x85EBCA77ull) & 0xFFFFFFFFull;
    x ^= x >> 16;
    x = (x * 0x7FEB352Dull) & 0xFFFFFFFFull;
    x ^= x >> 15;
    x = (x * 0x846CA68Bull) & 0xFFFFFFFFull;
    x ^= x >> 16;
    return static_cast<uint32_t>(x);
}

// Is neighbour j (weight w > 0) ranked above the current best (class bc, hash bh, index b)?
// The class is the exponent field of w's bits (monotone in w, read without
// the FP64 pipe).
__device__ __forceinline__ bool ranks_above(int64_t i, int32_t j, double w, int32_t b, int bc, uint32_t bh, int &cls,
                                            uint32_t &hs) {
    cls = static_cast<int>((__double_as_longlong(w) >> 52) & 0x7ff);
    hs = edge_hash(i, j);
    return b < 0 || cls > bc || (cls == bc && (hs > bh || (hs == bh && j < b)));
}

// leave[i] = 1 when node i leaves the hierarchy: no off-diagonal entry, or
// off-diagonal weights summing to at most kDominant d_i.
__global__ void k_leaving(int64_t n, const int64_t *ptr, const int32_t *col, const double *val, const double *diag,
                          int32_t *leave) {
    dep_enter();
    GRID_STRIDE(i, n) {
        double w = 0.0;
        for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e)
            if (col[e] != i) w -= val[e];
        leave[i] = (ptr[i + 1] == ptr[i] || w <= kDominant * diag[i]) ? 1 : 0;
    }
}

// Top-ranked strong neighbour (off-diagonal weight w_ij = -l_ij > 0 with
// w_ij >= kStrength sqrt(d_i d_j)) among the nodes that stay; with only_free,
// among neighbours that are still unpaired.
__global__ void k_heaviest(int64_t n, const int64_t *ptr, const int32_t *col, const double *val, const double *diag,
                           const int32_t *leave, const int32_t *partner, int only_free, int32_t *best) {
    dep_enter();
    GRID_STRIDE(i, n) {
        int32_t b = -1;
        int bc = 0;
        uint32_t bh = 0;
        if (!leave[i] && (!only_free || partner[i] < 0)) {
            const double di = diag[i];
            for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e) {
                const int32_t j = col[e];
                if (j == i || leave[j]) continue;
                if (only_free && partner[j] >= 0) continue;
                const double w = -val[e];
                // strong: w >= kStrength sqrt(d_i d_j), compared squared (no FP64 square root)
                if (!(w > 0.0) || !(w * w >= (kStrength * kStrength) * (di * diag[j]))) continue;
                int cls;
                uint32_t hs;
                if (ranks_above(i, j, w, b, bc, bh, cls, hs)) {
                    b = j;
                    bc = cls;
                    bh = hs;
                }
            }
        }
        best[i] = b;
    }
}

__global__ void k_handshake(int64_t n, const int32_t *best, int32_t *partner) {
    dep_enter();
    GRID_STRIDE(i, n) {
        if (partner[i] >= 0) continue;
        const int32_t b = best[i];
        if (b >= 0 && best[b] == i) partner[i] = b;
    }
}

// Attachment target of every node that stays: its top-ranked neighbour over
// all edges to nodes that stay when the node's heaviest such edge carries at
// least kAttach of its own diagonal, else -1.  The test is one-sided on
// purpose: a leaf hanging off a hub by an edge that is strong for the leaf
// (most of its diagonal) but weak for the hub should follow the hub.
__global__ void k_attach_target(int64_t n, const int64_t *ptr, const int32_t *col, const double *val,
                                const double *diag, const int32_t *leave, int32_t *att) {
    dep_enter();
    GRID_STRIDE(i, n) {
        int32_t b = -1;
        int bc = 0;
        uint32_t bh = 0;
        double wmax = 0.0;
        for (int64_t e = leave[i] ? ptr[i + 1] : ptr[i]; e < ptr[i + 1]; ++e) {
            const int32_t j = col[e];
            if (j == i || leave[j]) continue;
            const double w = -val[e];
            if (!(w > 0.0)) continue;
            wmax = fmax(wmax, w);
            int cls;
            uint32_t hs;
            if (ranks_above(i, j, w, b, bc, bh, cls, hs)) {
                b = j;
                bc = cls;
                bh = hs;
            }
        }
        att[i] = (b >= 0 && wmax >= kAttach * diag[i]) ? b : -1;
    }
}

// Leaders, first pass.  A node that leaves the hierarchy gets leader -1
// (no coarse node; counted in *isolated); a paired node, the smaller node of
// its pair; an unpaired node whose attachment target is paired joins that
// pair; every other node is left open (-2) for the second pass.
__global__ void k_leaders1(int64_t n, const int32_t *leave, const int32_t *partner, const int32_t *att,
                           int32_t *leader, int *isolated) {
    dep_enter();
    GRID_STRIDE(i, n) {
        int32_t lead = -2;
        if (leave[i]) {
            atomicAdd(isolated, 1);
            lead = -1;
        } else if (partner[i] >= 0) {
            const int32_t p = partner[i];
            lead = i < p ? static_cast<int32_t>(i) : p;
        } else {
            const int32_t t = att[i];
            if (t >= 0 && partner[t] >= 0) {
                const int32_t q = partner[t];
                lead = t < q ? t : q;
            }
        }
        leader[i] = lead;
    }
}

// want[i]: the attachment target of an open node when that target is open
// too, else -1.
__global__ void k_want(int64_t n, const int32_t *att, const int32_t *leader, int32_t *want) {
    dep_enter();
    GRID_STRIDE(i, n) {
        const int32_t t = att[i];
        want[i] = (leader[i] == -2 && t >= 0 && leader[t] == -2) ? t : -1;
    }
}

// Leaders, second pass over the open nodes: two nodes that want each other
// pair up (the smaller leads); a node that wants a node wanting nothing joins
// it; every other open node leads itself.  Each leader leads itself, so
// aggregates have no chains.  is_leader flags the leaders for the scan.
__global__ void k_leaders2(int64_t n, const int32_t *want, int32_t *leader, int32_t *is_leader) {
    dep_enter();
    GRID_STRIDE(i, n) {
        int32_t lead = leader[i];
        if (lead == -2) {
            const int32_t t = want[i];
            if (t < 0)
                lead = static_cast<int32_t>(i);
            else if (want[t] == i)
                lead = i < t ? static_cast<int32_t>(i) : t;
            else if (want[t] < 0)
                lead = t;
            else
                lead = static_cast<int32_t>(i);
            leader[i] = lead;
        }
        is_leader[i] = lead == i ? 1 : 0;
    }
}

__global__ void k_aggregates(int64_t n, const int32_t *leader, const int64_t *leader_pos, int32_t *agg,
                             int32_t *count) {
    dep_enter();
    GRID_STRIDE(i, n) {
        if (leader[i] < 0) {
            agg[i] = -1;
            continue;
        }
        const int32_t I = static_cast<int32_t>(leader_pos[leader[i]]);
        agg[i] = I;
        atomicAdd(&count[I], 1);
    }
}

__global__ void k_members_fill(int64_t n, const int32_t *agg, const int64_t *mptr, int32_t *fill, int32_t *mlist) {
    dep_enter();
    GRID_STRIDE(i, n) {
        const int32_t I = agg[i];
        if (I < 0) continue;
        mlist[mptr[I] + atomicAdd(&fill[I], 1)] = static_cast<int32_t>(i);
    }
}

// Members of each aggregate in increasing node order (small insertion sort).
__global__ void k_members_sort(int64_t nco, const int64_t *mptr, int32_t *mlist) {
    dep_enter();
    GRID_STRIDE(I, nco) {
        const int64_t b = mptr[I], e = mptr[I + 1];
        for (int64_t p = b + 1; p < e; ++p) {
            const int32_t v = mlist[p];
            int64_t q = p;
            while (q > b && mlist[q - 1] > v) {
                mlist[q] = mlist[q - 1];
                --q;
            }
            mlist[q] = v;
        }
    }
}

// ---------------------------------------------------------------- Galerkin coarse operator

// Collect, sort and merge the coarse neighbours of coarse node I (internal
// edges drop out of the Laplacian).  Returns the number of distinct
// neighbours (or -1 on overflow); *eI receives the coarse excess.
__device__ int coarse_row(int64_t I, const int64_t *mptr, const int32_t *mlist, const int64_t *ptr,
                          const int32_t *col, const double *val, const double *exc, const int32_t *agg, int32_t *cbuf,
                          double *vbuf, double *eI) {
    int cnt = 0;
    double e_sum = 0.0;
    for (int64_t k = mptr[I]; k < mptr[I + 1]; ++k) {
        const int32_t m = mlist[k];
        e_sum += exc[m];
        for (int64_t e = ptr[m]; e < ptr[m + 1]; ++e) {
            const int32_t J = agg[col[e]];
            if (J == I) continue;  // internal edge
            if (J < 0) {           // an edge to a node without coarse counterpart: part of the coarse shift
                e_sum -= val[e];
                continue;
            }
            // insertion into the sorted buffer, merging equal columns
            int pos = cnt;
            while (pos > 0 && cbuf[pos - 1] > J) --pos;
            if (pos > 0 && cbuf[pos - 1] == J) {
                vbuf[pos - 1] += val[e];
                continue;
            }
            if (cnt == kCoarseCap) return -1;
            for (int q = cnt; q > pos; --q) {
                cbuf[q] = cbuf[q - 1];
                vbuf[q] = vbuf[q - 1];
            }
            cbuf[pos] = J;
            vbuf[pos] = val[e];
            ++cnt;
        }
    }
    *eI = e_sum;
    return cnt;
}

// Short coarse rows (2D): one thread per coarse node, merging by insertion.
__global__ void k_coarse_count_thread(int64_t nco, const int64_t *mptr, const int32_t *mlist, const int64_t *ptr,
                                      const int32_t *col, const double *val, const double *exc, const int32_t *agg,
                                      int32_t *rowcnt, int *overflow) {
    dep_enter();
    int32_t cbuf[kCoarseCap];
    double vbuf[kCoarseCap];
    GRID_STRIDE(I, nco) {
        double e;
        const int c = coarse_row(I, mptr, mlist, ptr, col, val, exc, agg, cbuf, vbuf, &e);
        if (c < 0) {
            atomicOr(overflow, 1);
            rowcnt[I] = 0;
        } else {
            rowcnt[I] = c;
        }
    }
}

__global__ void k_coarse_fill_thread(int64_t nco, const int64_t *mptr, const int32_t *mlist, const int64_t *ptr,
                                     const int32_t *col, const double *val, const double *exc, const int32_t *agg,
                                     const int64_t *cptr, int32_t *ccol, double *cval, double *cdiag, double *cexc) {
    dep_enter();
    int32_t cbuf[kCoarseCap];
    double vbuf[kCoarseCap];
    GRID_STRIDE(I, nco) {
        double e;
        const int c = coarse_row(I, mptr, mlist, ptr, col, val, exc, agg, cbuf, vbuf, &e);
        const int64_t dst = cptr[I];
        double d = e;
        for (int k = 0; k < c; ++k) {
            ccol[dst + k] = cbuf[k];
            cval[dst + k] = vbuf[k];
            d -= vbuf[k];
        }
        cdiag[I] = d;
        cexc[I] = e;
    }
}

// The same rows built by one warp per coarse node I: the members' entries are
// gathered into shared memory in arrival order (members in order, then each
// member's entries), sorted by (J, arrival), and each run of equal J is summed
// by one lane in arrival order -- the order in which the insertion above adds
// them, so the coarse operator is the same bit for bit.  A row with more than
// kMergeCap raw entries is built by the warp's first lane with coarse_row.
constexpr int kMergeCap = 512;
constexpr int kMergeWarps = 4;  // warps per block
struct MergeSmem {
    int32_t key[kMergeCap];
    int32_t pos[kMergeCap];
    double val[kMergeCap];
};

// Gathers row I into sm; returns the raw entry count (> kMergeCap: not all
// gathered) and the coarse excess in *eI (valid in every lane).
__device__ int gather_row(int64_t I, const int64_t *mptr, const int32_t *mlist, const int64_t *ptr, const int32_t *col,
                          const double *val, const double *exc, const int32_t *agg, MergeSmem &sm, double *eI) {
    const int lane = threadIdx.x & 31;
    int n = 0;
    double e_sum = 0.0;
    for (int64_t k = mptr[I]; k < mptr[I + 1]; ++k) {
        const int32_t m = mlist[k];
        e_sum += exc[m];
        const int64_t b = ptr[m], e = ptr[m + 1];
        for (int64_t base = b; base < e; base += 32) {
            const int64_t idx = base + lane;
            const int32_t J = idx < e ? agg[col[idx]] : I;
            const bool keep = J != I && J >= 0;
            // edges to nodes without coarse counterpart join the shift, added in entry order
            // (the order of coarse_row)
            const double shift = J < 0 ? -val[idx] : 0.0;
            if (__any_sync(0xffffffffu, J < 0))
                for (int q = 0; q < 32; ++q) e_sum += __shfl_sync(0xffffffffu, shift, q);
            const unsigned mask = __ballot_sync(0xffffffffu, keep);
            const int at = n + __popc(mask & ((1u << lane) - 1u));
            if (keep && at < kMergeCap) {
                sm.key[at] = J;
                sm.pos[at] = at;
                sm.val[at] = val[idx];
            }
            n += __popc(mask);
        }
    }
    *eI = e_sum;
    __syncwarp();
    return n;
}

// Sorts the first n gathered entries by (key, pos) (bitonic, padded to a
// power of two with keys that sort last).
__device__ void sort_row(MergeSmem &sm, int n) {
    const int lane = threadIdx.x & 31;
    int P = 32;
    while (P < n) P <<= 1;
    for (int i = n + lane; i < P; i += 32) {
        sm.key[i] = 0x7fffffff;
        sm.pos[i] = 0x7fffffff;
        sm.val[i] = 0.0;
    }
    __syncwarp();
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = lane; i < P; i += 32) {
                const int l = i ^ j;
                if (l > i) {
                    const bool up = (i & k) == 0;
                    const bool greater = sm.key[i] > sm.key[l] || (sm.key[i] == sm.key[l] && sm.pos[i] > sm.pos[l]);
                    if (greater == up) {
                        const int32_t tk = sm.key[i], tp = sm.pos[i];
                        const double tv = sm.val[i];
                        sm.key[i] = sm.key[l];
                        sm.pos[i] = sm.pos[l];
                        sm.val[i] = sm.val[l];
                        sm.key[l] = tk;
                        sm.pos[l] = tp;
                        sm.val[l] = tv;
                    }
                }
            }
            __syncwarp();
        }
    }
}

// Runs of equal keys in the sorted entries: calls out(r, key, sum) once per
// run (r = run index, runs in key order; the sum in arrival order); returns
// the number of runs.
template <class F> __device__ int merge_runs(const MergeSmem &sm, int n, F out) {
    const int lane = threadIdx.x & 31;
    int runs = 0;
    for (int base = 0; base < n; base += 32) {
        const int i = base + lane;
        const bool start = i < n && (i == 0 || sm.key[i] != sm.key[i - 1]);
        const unsigned mask = __ballot_sync(0xffffffffu, start);
        if (start) {
            const int r = runs + __popc(mask & ((1u << lane) - 1u));
            double sum = sm.val[i];
            for (int q = i + 1; q < n && sm.key[q] == sm.key[i]; ++q) sum += sm.val[q];
            out(r, sm.key[i], sum);
        }
        runs += __popc(mask);
    }
    return runs;
}

__global__ void __launch_bounds__(32 * kMergeWarps) k_coarse_count(int64_t nco, const int64_t *mptr,
                                                                   const int32_t *mlist, const int64_t *ptr,
                                                                   const int32_t *col, const double *val,
                                                                   const double *exc, const int32_t *agg,
                                                                   int32_t *rowcnt, int *overflow) {
    dep_enter();
    __shared__ MergeSmem sm_all[kMergeWarps];
    MergeSmem &sm = sm_all[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = static_cast<int64_t>(gridDim.x) * kMergeWarps;
    for (int64_t I = blockIdx.x * static_cast<int64_t>(kMergeWarps) + (threadIdx.x >> 5); I < nco; I += nwarps) {
        double e;
        const int n = gather_row(I, mptr, mlist, ptr, col, val, exc, agg, sm, &e);
        int c;
        if (n == 0) {
            c = 0;
        } else if (n <= kMergeCap) {
            sort_row(sm, n);
            c = merge_runs(sm, n, [](int, int32_t, double) {});
        } else {
            c = 0;
            if (lane == 0) {
                int32_t cbuf[kCoarseCap];
                double vbuf[kCoarseCap];
                c = coarse_row(I, mptr, mlist, ptr, col, val, exc, agg, cbuf, vbuf, &e);
            }
            c = __shfl_sync(0xffffffffu, c, 0);
        }
        if (lane == 0) {
            if (c < 0) {
                atomicOr(overflow, 1);
                rowcnt[I] = 0;
            } else {
                rowcnt[I] = c;
            }
        }
        __syncwarp();
    }
}

__global__ void __launch_bounds__(32 * kMergeWarps) k_coarse_fill(int64_t nco, const int64_t *mptr,
                                                                  const int32_t *mlist, const int64_t *ptr,
                                                                  const int32_t *col, const double *val,
                                                                  const double *exc, const int32_t *agg,
                                                                  const int64_t *cptr, int32_t *ccol, double *cval,
                                                                  double *cdiag, double *cexc) {
    dep_enter();
    __shared__ MergeSmem sm_all[kMergeWarps];
    MergeSmem &sm = sm_all[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = static_cast<int64_t>(gridDim.x) * kMergeWarps;
    for (int64_t I = blockIdx.x * static_cast<int64_t>(kMergeWarps) + (threadIdx.x >> 5); I < nco; I += nwarps) {
        double e;
        const int n = gather_row(I, mptr, mlist, ptr, col, val, exc, agg, sm, &e);
        const int64_t dst = cptr[I];
        int c;
        if (n <= kMergeCap) {
            sort_row(sm, n);
            c = merge_runs(sm, n, [&](int r, int32_t J, double v) {
                ccol[dst + r] = J;
                cval[dst + r] = v;
            });
        } else {
            c = 0;
            if (lane == 0) {
                int32_t cbuf[kCoarseCap];
                double vbuf[kCoarseCap];
                c = coarse_row(I, mptr, mlist, ptr, col, val, exc, agg, cbuf, vbuf, &e);
                for (int k = 0; k < c; ++k) {
                    ccol[dst + k] = cbuf[k];
                    cval[dst + k] = vbuf[k];
                }
            }
            c = __shfl_sync(0xffffffffu, c, 0);
        }
        __syncwarp();
        if (lane == 0) {  // the diagonal from the merged entries, in their order
            double d = e;
            for (int k = 0; k < c; ++k) d -= cval[dst + k];
            cdiag[I] = d;
            cexc[I] = e;
        }
        __syncwarp();
    }
}

// The coarse operator of one level: warp per row where the finer level's rows
// are wide (the per-thread insertion then works in local memory), thread per
// row where they are short (a warp's sort would cost more than the merge).
static bool wide_rows(const AmgLevel &F) { return F.nnz > 8 * F.n; }

static void coarse_count(bchar_mesh_t m, const AmgLevel &F, const AmgLevel &C, int64_t ncoarse, const double *fexc,
                         int32_t *rowcnt, int *overflow) {
    AmgLevel &Fm = const_cast<AmgLevel &>(F);
    AmgLevel &Cm = const_cast<AmgLevel &>(C);
    if (wide_rows(F))
        launch_dep(k_coarse_count, blocks_for(ncoarse * 32, 32 * kMergeWarps), 32 * kMergeWarps, m->stream, 
            ncoarse, ptr<int64_t>(Cm.mptr), ptr<int32_t>(Cm.mlist), ptr<int64_t>(Fm.ptr), ptr<int32_t>(Fm.col),
            ptr<double>(Fm.val), fexc, ptr<int32_t>(Fm.agg), rowcnt, overflow);
    else
        launch_dep(k_coarse_count_thread, blocks_for(ncoarse, 128), 128, m->stream, 
            ncoarse, ptr<int64_t>(Cm.mptr), ptr<int32_t>(Cm.mlist), ptr<int64_t>(Fm.ptr), ptr<int32_t>(Fm.col),
            ptr<double>(Fm.val), fexc, ptr<int32_t>(Fm.agg), rowcnt, overflow);
    ++m->launches;
}

static void coarse_fill(bchar_mesh_t m, const AmgLevel &F, AmgLevel &C, int64_t ncoarse, const double *fexc) {
    AmgLevel &Fm = const_cast<AmgLevel &>(F);
    if (wide_rows(F))
        launch_dep(k_coarse_fill, blocks_for(ncoarse * 32, 32 * kMergeWarps), 32 * kMergeWarps, m->stream, 
            ncoarse, ptr<int64_t>(C.mptr), ptr<int32_t>(C.mlist), ptr<int64_t>(Fm.ptr), ptr<int32_t>(Fm.col),
            ptr<double>(Fm.val), fexc, ptr<int32_t>(Fm.agg), ptr<int64_t>(C.ptr), ptr<int32_t>(C.col),
            ptr<double>(C.val), ptr<double>(C.diag), ptr<double>(C.exc));
    else
        launch_dep(k_coarse_fill_thread, blocks_for(ncoarse, 128), 128, m->stream, 
            ncoarse, ptr<int64_t>(C.mptr), ptr<int32_t>(C.mlist), ptr<int64_t>(Fm.ptr), ptr<int32_t>(Fm.col),
            ptr<double>(Fm.val), fexc, ptr<int32_t>(Fm.agg), ptr<int64_t>(C.ptr), ptr<int32_t>(C.col),
            ptr<double>(C.val), ptr<double>(C.diag), ptr<double>(C.exc));
    ++m->launches;
}

// ---------------------------------------------------------------- V-cycle kernels
//
// The V-cycle runs in FP64 on a copy of each level's operator divided by a
// fixed scale (the square of the largest |K|_phi, so that the entries sit near
// 1).  An FP32 V-cycle costs less per application but loses the modes the
// preconditioner exists for: a cluster held by a shift ~1e-10 of its diagonal
// has a residual that cancels below FP32 rounding in b - L x, and the
// conjugate gradients then need more than twice the iterations (measured on
// the 1024^2 and 128^3 workloads), which costs more than FP64 saves.  The
// kernels are templates on the precision all the same.

template <class T> __global__ void k_scaled_copy(int64_t n, const double *in, T *out, double inv_scale) {
    dep_enter();
    GRID_STRIDE(i, n) out[i] = static_cast<T>(in[i] * inv_scale);
}

// Relaxation weight of row i: kOmega, or 1 for a row without off-diagonal
// entries (then one sweep solves its equation exactly).
__device__ __forceinline__ double row_weight(const int64_t *ptr, int64_t i) {
    return ptr[i + 1] == ptr[i] ? 1.0 : kOmega;
}

// w_i = omega_i / (diag_i / scale): kOmega, or 1 for a row without
// off-diagonal entries (one sweep then solves its equation exactly)
template <class T>
__global__ void k_scaled_inv(int64_t n, const int64_t *ptr, const double *diag, T *out, double inv_scale) {
    dep_enter();
    GRID_STRIDE(i, n) out[i] = static_cast<T>(row_weight(ptr, i) / (diag[i] * inv_scale));
}

// b = S res (S: +1 rows, -1 columns), in the V-cycle's precision
template <class T> __global__ void k_flip_in(int64_t nc, const double *res, T *b, const CgState *st) {
    dep_enter();
    if (st && st->converged) return;
    GRID_STRIDE(l, 2 * nc) b[l] = static_cast<T>(l < nc ? res[l] : -res[l]);
}

// z = S x / scale, in FP64
template <class T> __global__ void k_flip_out(int64_t nc, const T *x, double inv_scale, double *z, const CgState *st) {
    dep_enter();
    if (st && st->converged) return;
    GRID_STRIDE(l, 2 * nc) {
        const double v = static_cast<double>(x[l]) * inv_scale;
        z[l] = l < nc ? v : -v;
    }
}

// z = S x / scale, with the per-block partial sums of z.res and z.rp that
// the conjugate gradients need next (one pass instead of two)
template <class T>
__global__ void k_flip_out_dots(int64_t nc, const T *x, double inv_scale, double *z, const double *res,
                                const double *rp, double *pa, double *pb, const CgState *st) {
    dep_enter();
    if (st && st->converged) return;
    double a = 0.0, b = 0.0;
    GRID_STRIDE(l, 2 * nc) {
        const double v = static_cast<double>(x[l]) * inv_scale;
        const double zl = l < nc ? v : -v;
        z[l] = zl;
        a += zl * res[l];
        b += zl * rp[l];
    }
    a = block_sum(a);
    b = block_sum(b);
    if (threadIdx.x == 0) {
        pa[blockIdx.x] = a;
        pb[blockIdx.x] = b;
    }
}


// The smoothers multiply by w_i = omega_i / diag_i, formed once per build
// (k_scaled_inv): a division per node (and, in the pre-smoothing, per entry)
// would cost far more, in FP64 above all.

// x = w b
template <class T> __global__ void k_jacobi0(int64_t n, const T *dinv, const T *b, T *x, const CgState *st) {
    dep_enter();
    if (st && st->converged) return;
    GRID_STRIDE(i, n) x[i] = dinv[i] * b[i];
}

// x_out = x + w (b - L x)
template <class T>
__global__ void k_jacobi(int64_t n, const int64_t *ptr, const int32_t *col, const T *val, const T *diag,
                         const T *dinv, const T *x, const T *b, T *x_out, const CgState *st) {
    dep_enter();
    if (st && st->converged) return;
    GRID_STRIDE(i, n) {
        const int64_t e0 = ptr[i], e1 = ptr[i + 1];
        T s = diag[i] * x[i];
        for (int64_t e = e0; e < e1; ++e) s += val[e] * x[col[e]];
        x_out[i] = x[i] + dinv[i] * (b[i] - s);
    }
}

// Pre-smoothing from zero and the residual in one pass: x = w b, r = b - L x
// (a neighbour's x_j = w_j b_j is formed exactly as its owner forms it).
template <class T>
__global__ void k_presmooth_residual(int64_t n, const int64_t *ptr, const int32_t *col, const T *val, const T *diag,
                                     const T *dinv, const T *b, T *x, T *r, const CgState *st) {
    dep_enter();
    if (st && st->converged) return;
    GRID_STRIDE(i, n) {
        const int64_t e0 = ptr[i], e1 = ptr[i + 1];
        const T bi = b[i];
        const T xi = dinv[i] * bi;
        x[i] = xi;
        T s = diag[i] * xi;
        for (int64_t e = e0; e < e1; ++e) {
            const int32_t j = col[e];
            s += val[e] * (dinv[j] * b[j]);
        }
        r[i] = bi - s;
    }
}

// Prolongation and post-smoothing in one pass: with x' = x + xc[agg] (the
// coarse correction; nothing for a node without a coarse counterpart),
// x_out = x' + w (b - L x').  A neighbour's x'_j is formed as its owner forms it.
template <class T>
__global__ void k_prolong_smooth(int64_t n, const int64_t *ptr, const int32_t *col, const T *val, const T *diag,
                                 const T *dinv, const int32_t *agg, const T *xc, const T *x, const T *b, T *x_out,
                                 const CgState *st) {
    dep_enter();
    if (st && st->converged) return;
    GRID_STRIDE(i, n) {
        const int64_t e0 = ptr[i], e1 = ptr[i + 1];
        const int32_t I = agg[i];
        const T xi = I >= 0 ? x[i] + xc[I] : x[i];
        T s = diag[i] * xi;
        for (int64_t e = e0; e < e1; ++e) {
            const int32_t j = col[e];
            const int32_t J = agg[j];  // < 0: a neighbour that left the hierarchy
            s += val[e] * (J >= 0 ? x[j] + xc[J] : x[j]);
        }
        x_out[i] = xi + dinv[i] * (b[i] - s);
    }
}

template <class T>
__global__ void k_restrict(int64_t nco, const int64_t *mptr, const int32_t *mlist, const T *r, T *bc,
                           const CgState *st) {
    dep_enter();
    if (st && st->converged) return;
    GRID_STRIDE(I, nco) {
        T s = 0;
        for (int64_t k = mptr[I]; k < mptr[I + 1]; ++k) s += r[mlist[k]];
        bc[I] = s;
    }
}

template <class T> __global__ void k_prolong(int64_t n, const int32_t *agg, const T *xc, T *x, const CgState *st) {
    dep_enter();
    if (st && st->converged) return;
    GRID_STRIDE(i, n) {
        const int32_t I = agg[i];
        if (I >= 0) x[i] += xc[I];
    }
}

// The levels small enough for one block (n <= kOneBlock each), from the
// first of them down to the coarsest and back, in one launch: the same
// arithmetic per node as the per-level kernels above (pre-smoothing fused with
// the residual, restriction, kCoarsestSweeps sweeps on the coarsest level,
// prolongation fused with post-smoothing), with a block barrier between the
// passes instead of a kernel boundary.  On a fine mesh the hierarchy has a
// handful of such levels, each of which otherwise costs three launches of a
// few microseconds that do almost no work.
template <class T> struct SmallLevel {
    int64_t n;
    const int64_t *ptr;
    const int32_t *col;
    const T *val, *diag, *dinv;
    const int32_t *agg;    // node -> aggregate of the next level (levels above the coarsest)
    const int64_t *mptr;   // members (nodes of the previous level) of each node of this level
    const int32_t *mlist;
    T *x, *x2, *b, *r;
};

template <class T>
__global__ void __launch_bounds__(1024) k_small_cycle(const SmallLevel<T> *Ls, int nl, const CgState *st) {
    dep_enter();
    if (st && st->converged) return;
    for (int l = 0; l + 1 < nl; ++l) {  // down
        const SmallLevel<T> &L = Ls[l];
        for (int64_t i = threadIdx.x; i < L.n; i += blockDim.x) {
            const int64_t e0 = L.ptr[i], e1 = L.ptr[i + 1];
            const T bi = L.b[i];
            const T xi = L.dinv[i] * bi;
            L.x[i] = xi;
            T sum = L.diag[i] * xi;
            for (int64_t e = e0; e < e1; ++e) {
                const int32_t j = L.col[e];
                sum += L.val[e] * (L.dinv[j] * L.b[j]);
            }
            L.r[i] = bi - sum;
        }
        __syncthreads();
        const SmallLevel<T> &C = Ls[l + 1];
        for (int64_t I = threadIdx.x; I < C.n; I += blockDim.x) {
            T sum = 0;
            for (int64_t k = C.mptr[I]; k < C.mptr[I + 1]; ++k) sum += L.r[C.mlist[k]];
            C.b[I] = sum;
        }
        __syncthreads();
    }
    {  // coarsest
        const SmallLevel<T> &L = Ls[nl - 1];
        for (int64_t i = threadIdx.x; i < L.n; i += blockDim.x)
            L.x[i] = L.dinv[i] * L.b[i];
        __syncthreads();
        for (int k = 0; k < kCoarsestSweeps; ++k) {
            const T *xi = (k & 1) ? L.x2 : L.x;
            T *xo = (k & 1) ? L.x : L.x2;
            for (int64_t i = threadIdx.x; i < L.n; i += blockDim.x) {
                T sum = L.diag[i] * xi[i];
                for (int64_t e = L.ptr[i]; e < L.ptr[i + 1]; ++e) sum += L.val[e] * xi[L.col[e]];
                xo[i] = xi[i] + L.dinv[i] * (L.b[i] - sum);
            }
            __syncthreads();
        }
    }
    for (int l = nl - 2; l >= 0; --l) {  // up
        const SmallLevel<T> &L = Ls[l];
        const T *xc = l + 1 == nl - 1 ? Ls[l + 1].x : Ls[l + 1].x2;
        for (int64_t i = threadIdx.x; i < L.n; i += blockDim.x) {
            const int64_t e0 = L.ptr[i], e1 = L.ptr[i + 1];
            const int32_t I = L.agg[i];
            const T xi = I >= 0 ? L.x[i] + xc[I] : L.x[i];
            T sum = L.diag[i] * xi;
            for (int64_t e = e0; e < e1; ++e) {
                const int32_t j = L.col[e];
                const int32_t J = L.agg[j];
                sum += L.val[e] * (J >= 0 ? L.x[j] + xc[J] : L.x[j]);
            }
            L.x2[i] = xi + L.dinv[i] * (L.b[i] - sum);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- host side

void amg_release(Amg &amg) {
    for (AmgLevel &L : amg.levels) {
        Buf *all[] = {&L.ptr, &L.col, &L.val, &L.diag, &L.exc, &L.agg, &L.mptr, &L.mlist, &L.x, &L.x2, &L.b, &L.r,
                      &L.dval, &L.ddiag, &L.ddinv};
        for (Buf *b : all) release(*b);
    }
    amg.levels.clear();
    release(amg.tmp);
    release(amg.small_d);
}

static bool level_vectors(bchar_mesh_t m, AmgLevel &L) {
    // x holds n + 1 entries: it doubles as the int64 scan output while coarsening
    return ensure(m, L.x, sizeof(double) * (L.n + 1)) && ensure(m, L.x2, sizeof(double) * L.n) &&
           ensure(m, L.b, sizeof(double) * L.n) && ensure(m, L.r, sizeof(double) * L.n);
}

static bool amg_scaled_copies(bchar_mesh_t m, Amg &amg);

// The one-block levels: every level from the first with at most kOneBlock
// nodes down to the coarsest (levels shrink, so they are a suffix), when the
// coarsest is one of them.  Their descriptors go to the device once per build.
static bool small_descriptors(bchar_mesh_t m, Amg &amg) {
    int from = amg.nlev;
    while (from > 0 && amg.levels[from - 1].n <= kOneBlock) --from;
    amg.small_from = from;
    const int nl = amg.nlev - from;
    if (nl == 0) return true;
    std::vector<SmallLevel<double>> hd(nl);
    for (int k = 0; k < nl; ++k) {
        AmgLevel &L = amg.levels[from + k];
        const bool last = from + k == amg.nlev - 1;
        const bool first = k == 0;
        hd[k] = {L.n, ptr<int64_t>(L.ptr), ptr<int32_t>(L.col), ptr<double>(L.dval), ptr<double>(L.ddiag), ptr<double>(L.ddinv),
                 last ? nullptr : ptr<int32_t>(L.agg), first ? nullptr : ptr<int64_t>(L.mptr),
                 first ? nullptr : ptr<int32_t>(L.mlist), ptr<double>(L.x), ptr<double>(L.x2), ptr<double>(L.b),
                 ptr<double>(L.r)};
    }
    if (!ensure(m, amg.small_d, sizeof(SmallLevel<double>) * nl)) return false;
    // a pageable source: the copy has read it when the call returns
    cudaMemcpyAsync(amg.small_d.p, hd.data(), sizeof(SmallLevel<double>) * nl, cudaMemcpyHostToDevice, m->stream);
    return true;
}

bool amg_build(bchar_mesh_t m, Amg &amg) {
    cudaStream_t s = m->stream;
    const int64_t nc = m->nc, nnz = m->nnz;
    if (amg.levels.empty()) amg.levels.resize(1);
    amg.nlev = 1;
    amg.large_sweeps = kLargeCoarsestSweeps;
    AmgLevel &L0 = amg.levels[0];
    L0.n = 2 * nc;
    L0.nnz = 2 * nnz;
    if (!ensure(m, L0.ptr, sizeof(int64_t) * (L0.n + 1)) || !ensure(m, L0.col, sizeof(int32_t) * L0.nnz) ||
        !ensure(m, L0.val, sizeof(double) * L0.nnz) || !level_vectors(m, L0))
        return false;
    L0.diag_ext = ptr<double>(m->diag);
    L0.exc_ext = ptr<double>(m->qexc);
    launch_dep(k_level0_ptr, blocks_for(L0.n + 1), kThreads, s, nc, nnz, ptr<int64_t>(m->row_ptr), ptr<int64_t>(m->col_ptr),
                                                           ptr<int64_t>(L0.ptr));
    launch_dep(k_level0_fill, blocks_for(L0.n), kThreads, s, nc, ptr<int64_t>(m->row_ptr), ptr<int32_t>(m->col),
                                                        ptr<int64_t>(m->col_ptr), ptr<int32_t>(m->csc_row),
                                                        ptr<double>(m->a2), ptr<double>(m->a2c),
                                                        ptr<int64_t>(L0.ptr), ptr<int32_t>(L0.col),
                                                        ptr<double>(L0.val));
    m->launches += 2;
    while (amg.nlev < kMaxLevels) {
        AmgLevel &F = amg.levels[amg.nlev - 1];
        if (F.n <= kCoarsest) break;
        const double *fexc = F.exc_ext ? F.exc_ext : ptr<double>(F.exc);
        const double *fdg = F.diag_ext ? F.diag_ext : ptr<double>(F.diag);
        if (!ensure(m, amg.tmp, sizeof(int32_t) * 6 * F.n + 64) || !ensure(m, F.agg, sizeof(int32_t) * F.n))
            return false;
        int32_t *best = ptr<int32_t>(amg.tmp);
        int32_t *partner = best + F.n;
        int32_t *att = partner + F.n;     // attachment targets
        int32_t *want = att + F.n;
        int32_t *leader = want + F.n;
        int32_t *flag = leader + F.n;     // leader flags, later member counts / fill / row counts
        int *overflow = reinterpret_cast<int *>(flag + F.n);
        int *isolated = overflow + 1;
        const int bl = blocks_for(F.n);
        cudaMemsetAsync(partner, 0xff, sizeof(int32_t) * F.n, s);
        cudaMemsetAsync(overflow, 0, 2 * sizeof(int), s);
        // the want array holds the leave flags until k_want overwrites them
        launch_dep(k_leaving, bl, kThreads, s, F.n, ptr<int64_t>(F.ptr), ptr<int32_t>(F.col), ptr<double>(F.val), fdg,
                   want);
        ++m->launches;
        for (int round = 0; round < kHandshakes; ++round) {
            launch_dep(k_heaviest, bl, kThreads, s, F.n, ptr<int64_t>(F.ptr), ptr<int32_t>(F.col), ptr<double>(F.val),
                                               fdg, want, partner, round > 0, best);
            launch_dep(k_handshake, bl, kThreads, s, F.n, best, partner);
            m->launches += 2;
        }
        launch_dep(k_attach_target, bl, kThreads, s, F.n, ptr<int64_t>(F.ptr), ptr<int32_t>(F.col), ptr<double>(F.val), fdg,
                                                want, att);
        launch_dep(k_leaders1, bl, kThreads, s, F.n, want, partner, att, leader, isolated);
        launch_dep(k_want, bl, kThreads, s, F.n, att, leader, want);
        launch_dep(k_leaders2, bl, kThreads, s, F.n, want, leader, flag);
        m->launches += 4;
        // leader positions: scan of the leader flags (int32 -> int64), reuse the
        // per-level x buffer as int64 scratch (it holds n + 1 entries)
        int64_t *pos = reinterpret_cast<int64_t *>(ptr<double>(F.x));
        scan_i32_to_i64(m, flag, pos, F.n);
        // The coarse level is laid out for U = F.n coarse nodes, a bound on their
        // number nco, so that its members and row counts are formed before nco is
        // read back: nodes nco..U-1 have no members and empty rows.  One read-back
        // per level then returns nco, the isolated nodes and the coarse entries.
        if (static_cast<int>(amg.levels.size()) <= amg.nlev) amg.levels.resize(amg.nlev + 1);
        AmgLevel &Fr = amg.levels[amg.nlev - 1];  // re-fetch after resize
        AmgLevel &C = amg.levels[amg.nlev];
        const int64_t U = Fr.n;
        C.n = U;
        C.diag_ext = nullptr;
        C.exc_ext = nullptr;
        if (!ensure(m, C.mptr, sizeof(int64_t) * (U + 1)) || !ensure(m, C.mlist, sizeof(int32_t) * Fr.n) ||
            !ensure(m, C.ptr, sizeof(int64_t) * (U + 1)) || !ensure(m, C.diag, sizeof(double) * U) ||
            !ensure(m, C.exc, sizeof(double) * U) || !level_vectors(m, C))
            return false;
        // aggregates: map, member counts -> pointers, members sorted by node
        cudaMemsetAsync(flag, 0, sizeof(int32_t) * U, s);
        launch_dep(k_aggregates, bl, kThreads, s, Fr.n, leader, pos, ptr<int32_t>(Fr.agg), flag);
        scan_i32_to_i64(m, flag, ptr<int64_t>(C.mptr), U);
        cudaMemsetAsync(flag, 0, sizeof(int32_t) * U, s);
        launch_dep(k_members_fill, bl, kThreads, s, Fr.n, ptr<int32_t>(Fr.agg), ptr<int64_t>(C.mptr), flag,
                                               ptr<int32_t>(C.mlist));
        launch_dep(k_members_sort, blocks_for(U), kThreads, s, U, ptr<int64_t>(C.mptr), ptr<int32_t>(C.mlist));
        m->launches += 3;
        int32_t *rowcnt = flag;
        coarse_count(m, Fr, C, U, fexc, rowcnt, overflow);
        scan_i32_to_i64(m, rowcnt, ptr<int64_t>(C.ptr), U);
        int64_t nco = 0, cnnz = 0;
        int niso = 0, ovf = 0;
        cudaMemcpyAsync(&nco, pos + Fr.n, sizeof nco, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(&niso, isolated, sizeof niso, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(&cnnz, ptr<int64_t>(C.ptr) + U, sizeof cnnz, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(&ovf, overflow, sizeof ovf, cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) return false;
        m->launches += 1;
        const int64_t active = Fr.n - niso;  // nodes that would have a coarse counterpart
        // a coarsest level whose nodes have all left the hierarchy is diagonally
        // dominant (ratio <= kDominant): a few sweeps reduce its error enough
        amg.large_sweeps = active == 0 ? kDominantSweeps : kLargeCoarsestSweeps;
        if (active <= kCoarsest || nco >= active * kStall || nco < 1) break;  // Fr is the coarsest level
        if (ovf) break;  // a coarse row would be too wide: stop at the finer level
        C.n = nco;
        C.nnz = cnnz;
        if (!ensure(m, C.col, sizeof(int32_t) * (cnnz > 0 ? cnnz : 1)) ||
            !ensure(m, C.val, sizeof(double) * (cnnz > 0 ? cnnz : 1)))
            return false;
        coarse_fill(m, Fr, C, nco, fexc);
        ++amg.nlev;
    }
    return amg_scaled_copies(m, amg);
}

// The FP64 copy of every level's operator divided by a fixed scale (the
// square of the largest |K|_phi), and the smoother weights.
static bool amg_scaled_copies(bchar_mesh_t m, Amg &amg) {
    cudaStream_t s = m->stream;
    amg.scale = m->max_volphi * m->max_volphi;
    const double inv = 1.0 / amg.scale;
    for (int l = 0; l < amg.nlev; ++l) {
        AmgLevel &L = amg.levels[l];
        const int64_t nnzl = L.nnz > 0 ? L.nnz : 1;
        if (!ensure(m, L.dval, sizeof(double) * nnzl) || !ensure(m, L.ddiag, sizeof(double) * L.n) ||
            !ensure(m, L.ddinv, sizeof(double) * L.n))
            return false;
        const double *dg = L.diag_ext ? L.diag_ext : ptr<double>(L.diag);
        if (L.nnz > 0) {
            launch_dep(k_scaled_copy<double>, blocks_for(L.nnz), kThreads, s, L.nnz, ptr<double>(L.val),
                       ptr<double>(L.dval), inv);
            ++m->launches;
        }
        launch_dep(k_scaled_copy<double>, blocks_for(L.n), kThreads, s, L.n, dg, ptr<double>(L.ddiag), inv);
        launch_dep(k_scaled_inv<double>, blocks_for(L.n), kThreads, s, L.n, ptr<int64_t>(L.ptr), dg,
                   ptr<double>(L.ddinv), inv);
        m->launches += 2;
    }
    return small_descriptors(m, amg);
}

// Buffers of one level in the V-cycle's precision.
template <class T> struct LevelBufs;
template <> struct LevelBufs<double> {
    static double *val(AmgLevel &L) { return ptr<double>(L.dval); }
    static double *diag(AmgLevel &L) { return ptr<double>(L.ddiag); }
    static double *dinv(AmgLevel &L) { return ptr<double>(L.ddinv); }
    static double *x(AmgLevel &L) { return ptr<double>(L.x); }
    static double *x2(AmgLevel &L) { return ptr<double>(L.x2); }
    static double *b(AmgLevel &L) { return ptr<double>(L.b); }
    static double *r(AmgLevel &L) { return ptr<double>(L.r); }
    static void *small(Amg &a) { return a.small_d.p; }
};

// z = S V(S res) / scale: one V-cycle of the sign-flipped operator in precision T.
template <class T>
static void vcycle(bchar_mesh_t m, Amg &amg, const double *res, double *z, const CgState *st, bool b_ready,
                   const double *rp, double *pa, double *pb) {
    using B = LevelBufs<T>;
    cudaStream_t s = m->stream;
    const int64_t nc = m->nc;
    AmgLevel &L0 = amg.levels[0];
    if (!b_ready) {
        launch_dep(k_flip_in<T>, blocks_for(L0.n), kThreads, s, nc, res, B::b(L0), st);
        ++m->launches;
    }
    const int big = amg.small_from < amg.nlev ? amg.small_from : amg.nlev - 1;  // levels cycled kernel by kernel
    for (int l = 0; l < big; ++l) {  // down: pre-smooth from zero, residual, restrict
        AmgLevel &L = amg.levels[l];
        AmgLevel &C = amg.levels[l + 1];
        const int bl = blocks_for(L.n);
        launch_dep(k_presmooth_residual<T>, bl, kThreads, s, L.n, ptr<int64_t>(L.ptr), ptr<int32_t>(L.col), B::val(L),
                                                        B::diag(L), B::dinv(L), B::b(L), B::x(L), B::r(L), st);
        launch_dep(k_restrict<T>, blocks_for(C.n), kThreads, s, C.n, ptr<int64_t>(C.mptr), ptr<int32_t>(C.mlist), B::r(L),
                                                           B::b(C), st);
        m->launches += 2;
    }
    if (amg.small_from < amg.nlev) {  // the one-block levels down to the coarsest and back, one launch
        launch_dep(k_small_cycle<T>, 1, 1024, s, static_cast<const SmallLevel<T> *>(B::small(amg)),
                                             amg.nlev - amg.small_from, st);
        ++m->launches;
    } else {  // a coarsest level too large for one block: Jacobi sweeps from zero (even count: the result is in x)
        AmgLevel &L = amg.levels[amg.nlev - 1];
        const int bl = blocks_for(L.n);
        launch_dep(k_jacobi0<T>, bl, kThreads, s, L.n, B::dinv(L), B::b(L), B::x(L), st);
        for (int k = 0; k < amg.large_sweeps; ++k)
            launch_dep(k_jacobi<T>, bl, kThreads, s, L.n, ptr<int64_t>(L.ptr), ptr<int32_t>(L.col), B::val(L),
                                                B::diag(L), B::dinv(L), k & 1 ? B::x2(L) : B::x(L), B::b(L),
                                                k & 1 ? B::x(L) : B::x2(L), st);
        m->launches += 1 + amg.large_sweeps;
    }
    // up: prolong into x, post-smooth into x2 (the next finer level reads x2; the
    // coarsest level, and a one-block cycle of a single level, leave theirs in x)
    for (int l = big - 1; l >= 0; --l) {
        AmgLevel &L = amg.levels[l];
        AmgLevel &C = amg.levels[l + 1];
        const T *xc = l + 1 == amg.nlev - 1 ? B::x(C) : B::x2(C);
        if (L.n < kFuseBelow) {  // launch-bound levels: one kernel
            launch_dep(k_prolong_smooth<T>, blocks_for(L.n), kThreads, s, L.n, ptr<int64_t>(L.ptr), ptr<int32_t>(L.col),
                                                                     B::val(L), B::diag(L), B::dinv(L), ptr<int32_t>(L.agg), xc,
                                                                     B::x(L), B::b(L), B::x2(L), st);
            ++m->launches;
        } else {  // large levels: the sweep's neighbours read one array instead of three
            launch_dep(k_prolong<T>, blocks_for(L.n), kThreads, s, L.n, ptr<int32_t>(L.agg), xc, B::x(L), st);
            launch_dep(k_jacobi<T>, blocks_for(L.n), kThreads, s, L.n, ptr<int64_t>(L.ptr), ptr<int32_t>(L.col), B::val(L),
                                                             B::diag(L), B::dinv(L), B::x(L), B::b(L), B::x2(L), st);
            m->launches += 2;
        }
    }
    const T *x0 = amg.nlev > 1 ? B::x2(L0) : B::x(L0);
    if (pa)
        launch_dep(k_flip_out_dots<T>, kRedBlocks, kThreads, s, nc, x0, 1.0 / amg.scale, z, res, rp, pa, pb, st);
    else
        launch_dep(k_flip_out<T>, blocks_for(L0.n), kThreads, s, nc, x0, 1.0 / amg.scale, z, st);
    ++m->launches;
}

// One damped-Jacobi sweep on the finest level (for timing; on a large finest
// level this is the V-cycle's post-smoothing kernel).
void amg_smooth_once(bchar_mesh_t m, Amg &amg) {
    AmgLevel &L = amg.levels[0];
    k_jacobi<double><<<blocks_for(L.n), kThreads, 0, m->stream>>>(L.n, ptr<int64_t>(L.ptr), ptr<int32_t>(L.col),
                                                                   ptr<double>(L.dval), ptr<double>(L.ddiag),
                                                                   ptr<double>(L.ddinv), ptr<double>(L.x),
                                                                   ptr<double>(L.b), ptr<double>(L.x2), nullptr);
}

void amg_apply(bchar_mesh_t m, Amg &amg, const double *res, double *z, const CgState *st, bool b_ready,
               const double *rp, double *pa, double *pb) {
    vcycle<double>(m, amg, res, z, st, b_ready, rp, pa, pb);
}

double *amg_finest_rhs(Amg &amg) { return ptr<double>(amg.levels[0].b); }

}  // namespace bchar
