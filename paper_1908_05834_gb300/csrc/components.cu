// Consistent local targets (reading of Sec 3.2): the row targets |K_i|_phi
// of a connected block of rows and columns are multiplied by
// sum_cols |M_j|_phi / sum_rows |K_i|_phi when the two sums differ by more
// than 1e-12 relative, so that the constraints of eq. localmassconsMat and
// eq. globalmassconsMat can hold together.  Row i and column j are linked
// whenever a0_ij != 0: the components of A's pattern, on which both sums must
// equal the sum of the component's entries once the constraints hold.
//
// Components: lock-free union-find over the 2 n_c row/column nodes, always
// hooking the larger root under the smaller one, so every component ends with
// its smallest node as root whatever the order of the unions.
// Sums: |K|_phi is converted to an exact 52-bit fixed-point integer (scaled by
// a power of two fixed per mesh) split into two 26-bit limbs whose integer
// sums cannot overflow, so the per-component sums do not depend on the order
// of the atomic additions (the step stays bitwise reproducible).
#include <math.h>

#include "device.cuh"

namespace bchar {

#define GRID_STRIDE(i, n)                                                                    \
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < (n); \
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)

constexpr int kUnionRetries = 1 << 20;

__device__ __forceinline__ int32_t uf_find(int32_t *parent, int32_t x) {
    for (int it = 0; it < kUnionRetries; ++it) {
        const int32_t p = parent[x];
        if (p == x) return x;
        const int32_t g = parent[p];
        if (g != p) parent[x] = g;  // path halving; a stale value is still an ancestor
        x = g;
    }
    return x;
}

__global__ void k_uf_init(int64_t n2, int32_t *parent) {
    GRID_STRIDE(l, n2) parent[l] = static_cast<int32_t>(l);
}

__global__ void k_uf_union(int64_t nc, const int64_t *row_ptr, const int32_t *col, const double *a0,
                           int32_t *parent, DevInfo *info) {
    GRID_STRIDE(i, nc) {
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            if (a0[e] == 0.0) continue;
            int32_t a = static_cast<int32_t>(i), b = static_cast<int32_t>(nc + col[e]);
            int it = 0;
            for (; it < kUnionRetries; ++it) {
                int32_t ra = uf_find(parent, a), rb = uf_find(parent, b);
                if (ra == rb) break;
                if (ra < rb) {
                    const int32_t t = ra;
                    ra = rb;
                    rb = t;
                }
                if (atomicCAS(&parent[ra], ra, rb) == ra) break;
            }
            if (it == kUnionRetries) atomicOr(&info->err, kErrUnion);
        }
    }
}

__global__ void k_uf_label(int64_t n2, int32_t *parent, int32_t *label) {
    GRID_STRIDE(l, n2) label[l] = uf_find(parent, static_cast<int32_t>(l));
}

// Node l < n_c is row l, node n_c + j column j; both carry |.|_phi of their cell.
// The lanes of a warp that add into the same slot are summed first (integer
// limbs, so the order does not matter) and their leader adds once: one large
// component would otherwise serialise every node on the same two counters.
__global__ void k_comp_sums(int64_t nc, const int32_t *label, const double *volphi, int shift,
                            unsigned long long *acc) {
    GRID_STRIDE(l, 2 * nc) {
        const double b = volphi[l < nc ? l : l - nc];
        const unsigned long long q = static_cast<unsigned long long>(ldexp(b, shift));  // < 2^52, exact
        const long long slot = 4 * static_cast<long long>(label[l]) + (l < nc ? 0 : 2);
        const unsigned peers = __match_any_sync(__activemask(), slot);
        unsigned long long hi = 0, lo = 0;
        for (unsigned rest = peers; rest; rest &= rest - 1) {
            const int src = __ffs(rest) - 1;
            hi += __shfl_sync(peers, q >> 26, src);
            lo += __shfl_sync(peers, q & ((1ull << 26) - 1), src);
        }
        if ((threadIdx.x & 31) == __ffs(peers) - 1) {
            atomicAdd(&acc[slot], hi);
            atomicAdd(&acc[slot + 1], lo);
        }
    }
}

__device__ __forceinline__ double limbs(const unsigned long long *a, int shift) {
    return ldexp(ldexp(static_cast<double>(a[0]), 26) + static_cast<double>(a[1]), -shift);
}

__global__ void k_balance(int64_t nc, const int32_t *label, const double *volphi, const unsigned long long *acc,
                          int shift, double tol, double *bloc, DevInfo *info) {
    GRID_STRIDE(i, nc) {
        const int32_t r = label[i];
        const double sr = limbs(acc + 4 * static_cast<int64_t>(r), shift);
        const double sc = limbs(acc + 4 * static_cast<int64_t>(r) + 2, shift);
        double f = 1.0;
        if (fabs(sc - sr) > tol * sr) {
            f = sc / sr;
            if (r == i) atomicAdd(&info->unbalanced, 1);  // one count per component (its root row)
        }
        bloc[i] = volphi[i] * f;
    }
}

bool launch_balance(bchar_mesh_t m) {
    const int64_t nc = m->nc, n2 = 2 * nc;
    if (!ensure(m, m->uf_parent, sizeof(int32_t) * n2) || !ensure(m, m->uf_label, sizeof(int32_t) * n2) ||
        !ensure(m, m->comp_acc, sizeof(unsigned long long) * 4 * n2))
        return false;
    int32_t *parent = ptr<int32_t>(m->uf_parent), *label = ptr<int32_t>(m->uf_label);
    unsigned long long *acc = ptr<unsigned long long>(m->comp_acc);
    DevInfo *di = ptr<DevInfo>(m->dinfo);
    cudaStream_t s = m->stream;
    int e = 0;
    frexp(m->max_volphi, &e);                 // max |K|_phi < 2^e
    const int shift = 52 - e;                 // so every |K|_phi * 2^shift < 2^52
    cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * 4 * n2, s);
    k_uf_init<<<blocks_for(n2), kThreads, 0, s>>>(n2, parent);
    k_uf_union<<<blocks_for(nc), kThreads, 0, s>>>(nc, ptr<int64_t>(m->row_ptr), ptr<int32_t>(m->col),
                                                   ptr<double>(m->a0), parent, di);
    k_uf_label<<<blocks_for(n2), kThreads, 0, s>>>(n2, parent, label);
    k_comp_sums<<<blocks_for(n2), kThreads, 0, s>>>(nc, label, ptr<double>(m->volphi), shift, acc);
    k_balance<<<blocks_for(nc), kThreads, 0, s>>>(nc, label, ptr<double>(m->volphi), acc, shift, 1e-12,
                                                  ptr<double>(m->bloc), di);
    m->launches += 5;
    return true;
}

}  // namespace bchar
