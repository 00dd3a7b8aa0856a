// FP64 matrix stages of a B-char step:
//   - device-wide scans (row / column pointers),
//   - the column view of A (deterministic: columns sorted by row),
//   - N alternating column/row scalings (Sec 3.2, eq. volAdj), kept as
//     diagonal factors, A^(N) = diag(R) A^(0) diag(C),
//   - the mass-conservation minimisation (Sec 3.2, eq. opti_masscons) with
//     its bounds 0 <= 1 + x <= 2 inside the problem and an elastic penalty on
//     the relative violations of the mass constraints (quadratic, weight
//     1/eps^2, up to 1e-6; linear beyond), by a primal-dual interior-point
//     method whose normal equations (A-hat D A-hat^T + diag(exc)) are the
//     bipartite matrix [[D_r, W], [W^T, D_c]], W_ij = a_ij^2 D_ij, applied
//     through the row and column views of A without forming A-hat and solved
//     by conjugate gradients with an aggregation-multigrid preconditioner,
//   - a final column scaling (global mass to rounding), W_KM = a_KM / |K|_phi
//     and the update c^{n+1} = W c^n (eq. phys-inter-ELLAM) with FP64
//     accumulation.
// All sums run in a fixed order (no floating-point atomics), so a step is
// bitwise reproducible.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <time.h>

#include "amg.cuh"
#include "device.cuh"
#include "tiles.cuh"

namespace bchar {

#define GRID_STRIDE(i, n)                                                            \
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < (n); \
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)

// ---------------------------------------------------------------- scan

__global__ void k_scan_partial(const int32_t *in, int64_t n, int64_t *block_sums) {
    dep_enter();
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanChunk;
    int64_t s = 0;
    for (int i = threadIdx.x; i < kScanChunk; i += blockDim.x)
        if (base + i < n) s += in[base + i];
    __shared__ int64_t sh[kThreads];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) block_sums[blockIdx.x] = sh[0];
}

// One block: exclusive scan of nb block sums in place, total in sums[nb].
__global__ void k_scan_top(int64_t *sums, int nb) {
    dep_enter();
    __shared__ int64_t sh[1024];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += 1024) {
        int i = base + threadIdx.x;
        int64_t v = i < nb ? sums[i] : 0;
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {  // Hillis-Steele inclusive scan
            int64_t t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
            __syncthreads();
            sh[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < nb) sums[i] = carry + sh[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 0) carry += sh[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[nb] = carry;
}

__global__ void k_scan_final(const int32_t *in, int64_t n, const int64_t *block_off, int64_t *out, int nb) {
    dep_enter();
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanChunk;
    constexpr int per = kScanChunk / kThreads;
    const int64_t mine = base + static_cast<int64_t>(threadIdx.x) * per;
    int64_t local[per];
    int64_t s = 0;
    for (int k = 0; k < per; ++k) {
        local[k] = (mine + k < n) ? in[mine + k] : 0;
        s += local[k];
    }
    __shared__ int64_t sh[kThreads];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < kThreads; o <<= 1) {
        int64_t t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
    }
    int64_t run = block_off[blockIdx.x] + sh[threadIdx.x] - s;
    for (int k = 0; k < per; ++k) {
        if (mine + k < n) out[mine + k] = run;
        run += local[k];
    }
    if (blockIdx.x == nb - 1 && threadIdx.x == 0) out[n] = block_off[nb];
}

void scan_i32_to_i64(bchar_mesh_t m, const int32_t *in, int64_t *out, int64_t n) {
    const int nb = static_cast<int>((n + kScanChunk - 1) / kScanChunk);
    const int nbb = nb < 1 ? 1 : nb;
    ensure(m, m->scan_tmp, sizeof(int64_t) * (nbb + 1));
    int64_t *sums = ptr<int64_t>(m->scan_tmp);
    launch_dep(k_scan_partial, nbb, kThreads, m->stream, in, n, sums);
    launch_dep(k_scan_top, 1, 1024, m->stream, sums, nbb);
    launch_dep(k_scan_final, nbb, kThreads, m->stream, in, n, sums, out, nbb);
    m->launches += 3;
}

// ---------------------------------------------------------------- reductions

// Final reduction of per-block partial sums (fixed order) into *out.
__global__ void k_sum_partials(const double *partials, int n, double *out) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += partials[i];
    s = block_sum(s);
    if (threadIdx.x == 0) *out = s;
}

// ---------------------------------------------------------------- column view

__global__ void k_fill_columns(int64_t nc, const int64_t *row_ptr, const int32_t *col, const int64_t *col_ptr,
                               int32_t *fill, int32_t *csc_row, int32_t *csc_src) {
    GRID_STRIDE(i, nc) {
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            const int32_t j = col[e];
            const int64_t p = col_ptr[j] + atomicAdd(&fill[j], 1);
            csc_row[p] = static_cast<int32_t>(i);
            csc_src[p] = static_cast<int32_t>(e);
        }
    }
}

// Entries of each column in increasing row order (insertion sort; columns
// hold a few tens of entries at most).
__global__ void k_sort_columns(int64_t nc, const int64_t *col_ptr, int32_t *csc_row, int32_t *csc_src) {
    GRID_STRIDE(j, nc) {
        const int64_t b = col_ptr[j], e = col_ptr[j + 1];
        for (int64_t p = b + 1; p < e; ++p) {
            const int32_t r = csc_row[p], s = csc_src[p];
            int64_t q = p;
            while (q > b && csc_row[q - 1] > r) {
                csc_row[q] = csc_row[q - 1];
                csc_src[q] = csc_src[q - 1];
                --q;
            }
            csc_row[q] = r;
            csc_src[q] = s;
        }
    }
}

void launch_transpose(bchar_mesh_t m) {
    scan_i32_to_i64(m, ptr<int32_t>(m->colcnt), ptr<int64_t>(m->col_ptr), m->nc);
    cudaMemsetAsync(m->colfill.p, 0, sizeof(int32_t) * m->nc, m->stream);
    k_fill_columns<<<blocks_for(m->nc), kThreads, 0, m->stream>>>(m->nc, ptr<int64_t>(m->row_ptr), ptr<int32_t>(m->col),
                                                                  ptr<int64_t>(m->col_ptr), ptr<int32_t>(m->colfill),
                                                                  ptr<int32_t>(m->csc_row), ptr<int32_t>(m->csc_src));
    k_sort_columns<<<blocks_for(m->nc), kThreads, 0, m->stream>>>(m->nc, ptr<int64_t>(m->col_ptr),
                                                                  ptr<int32_t>(m->csc_row), ptr<int32_t>(m->csc_src));
    m->launches += 2;
}

// ---------------------------------------------------------------- sub-warp row walks
//
// The streaming stages (scalings, update) walk rows of a few to a few tens of
// entries: L lanes of a warp share one row (L a power of two sized to the mean
// row length), so consecutive lanes read consecutive entries and a warp reads
// 32 consecutive entries of neighbouring rows at once.  A row's partial sums
// are reduced by shuffles within its L lanes.  Every lane of a warp runs the
// same number of outer iterations (rows past the end contribute nothing), so
// the shuffles always see the whole warp.  The grid is persistent (a fixed
// multiple of the SM count), so the order of every sum is fixed.

template <int L> __device__ __forceinline__ double group_sum(double v) {
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Lanes per row for a mean of `mean` entries per row.
static int lanes_for(double mean) {
    int L = 2;
    while (L < 32 && L < mean) L <<= 1;
    return L;
}

#define DISPATCH_LANES(L, CALL)                 \
    switch (L) {                                \
    case 2: { constexpr int LL = 2; CALL; } break;   \
    case 4: { constexpr int LL = 4; CALL; } break;   \
    case 8: { constexpr int LL = 8; CALL; } break;   \
    case 16: { constexpr int LL = 16; CALL; } break; \
    default: { constexpr int LL = 32; CALL; } break; \
    }

constexpr int kStreamBlocks = 152 * 8;  // persistent grid of the streaming kernels (256 threads each)

// ---------------------------------------------------------------- tiles of the two views

template <class K> static void allow_tile_smem(K kernel) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kTileSmem));
}

__global__ void k_tile_bounds(int64_t n, const int64_t *ptr, int64_t ntile, int32_t *tile) {
    GRID_STRIDE(k, ntile + 1) {
        if (k == ntile) {
            tile[k] = static_cast<int32_t>(n);
        } else {
            const int64_t want = k * static_cast<int64_t>(kTileEntries);
            int64_t lo = 0, hi = n;  // the first l in [0, n] with ptr[l] >= want
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (ptr[mid] >= want) hi = mid;
                else lo = mid + 1;
            }
            tile[k] = static_cast<int32_t>(lo);
        }
    }
}

__global__ void k_scale_tiles(LineView V, const double *f, const double *tgt, double *out);
__global__ void k_scaled_col_error(LineView V, const double *R, const double *C, const double *volphi,
                                   unsigned long long *slot);
__global__ void k_cg_matvec(LineView Vr, LineView Vc, const double *diag, const double *p, double *q,
                            double *partials, const CgState *st);
template <class T> __global__ void k_spmv(LineView V, const double *volphi, const T *c_in, T *c_out, double *partials);

bool launch_tiles(bchar_mesh_t m) {
    static bool attrs = false;  // the shared-memory opt-in of the tile kernels (per process; harmless to repeat)
    if (!attrs) {
        allow_tile_smem(k_scale_tiles);
        allow_tile_smem(k_scaled_col_error);
        allow_tile_smem(k_cg_matvec);
        allow_tile_smem(k_spmv<float>);
        allow_tile_smem(k_spmv<double>);
        attrs = true;
    }
    m->ntile = tile_count(m->nnz);
    const size_t b = sizeof(int32_t) * (m->ntile + 1);
    if (!ensure(m, m->tile_r, b) || !ensure(m, m->tile_c, b)) return false;
    k_tile_bounds<<<blocks_for(m->ntile + 1), kThreads, 0, m->stream>>>(m->nc, ptr<int64_t>(m->row_ptr), m->ntile,
                                                                        ptr<int32_t>(m->tile_r));
    k_tile_bounds<<<blocks_for(m->ntile + 1), kThreads, 0, m->stream>>>(m->nc, ptr<int64_t>(m->col_ptr), m->ntile,
                                                                        ptr<int32_t>(m->tile_c));
    m->launches += 2;
    return true;
}

static LineView row_view(bchar_mesh_t m, const double *val) {
    return LineView{m->nc, ptr<int64_t>(m->row_ptr), ptr<int32_t>(m->col), val, ptr<int32_t>(m->tile_r), m->ntile};
}

static LineView col_view(bchar_mesh_t m, const double *val) {
    return LineView{m->nc, ptr<int64_t>(m->col_ptr), ptr<int32_t>(m->csc_row), val, ptr<int32_t>(m->tile_c), m->ntile};
}

static int tile_grid(int64_t ntiles) { return static_cast<int>(ntiles < kTileBlocks ? (ntiles > 0 ? ntiles : 1) : kTileBlocks); }

// ---------------------------------------------------------------- scaling (eq. volAdj)

__global__ void k_fill(double *v, int64_t n, double val) {
    GRID_STRIDE(i, n) v[i] = val;
}

// a0 in column order (a0c[p] = a0[csc_src[p]]), once per step, so that the
// column passes stream their values.
__global__ void k_gather_col_values(int64_t nnz, const int32_t *csc_src, const double *a0, double *a0c) {
    GRID_STRIDE(p, nnz) a0c[p] = a0[csc_src[p]];
}

// Line sums of one view: out_l = tgt_l / sum_k v_k f[idx_k] over line l (a
// column of the column view with f = R, or a row of the row view with f = C):
// a^{n+1/2}: C_j = |M_j|_phi / sum_i R_i a0_ij; a^{n+1}: R_i = b_i / sum_j a0_ij C_j.
struct ScaleEpi {
    const double *tgt;
    double *out;
    __device__ void operator()(int64_t l, double s) { out[l] = tgt[l] / s; }
};

struct NoEpi {
    __device__ void operator()(int64_t, double) {}
};

__global__ void __launch_bounds__(kTileThreads) k_scale_tiles(LineView V, const double *f, const double *tgt,
                                                              double *out) {
    extern __shared__ __align__(16) unsigned char smem[];
    ScaleEpi epi{tgt, out};
    NoEpi none;
    const LineView nov{0, nullptr, nullptr, nullptr, nullptr, 0};
    tile_loop(V, f, epi, nov, f, none, smem);
}

// aN = R a0 C per entry (row view)
template <int L>
__global__ void __launch_bounds__(256) k_apply_scaling(int64_t nc, const int64_t *row_ptr, const int32_t *col,
                                                       const double *a0, const double *R, const double *C,
                                                       double *aN) {
    constexpr int G = 256 / L;
    const int g = threadIdx.x / L, lane = threadIdx.x % L;
    for (int64_t base = static_cast<int64_t>(blockIdx.x) * G; base < nc; base += static_cast<int64_t>(gridDim.x) * G) {
        const int64_t i = base + g;
        if (i < nc) {
            const double ri = R[i];
            for (int64_t e = row_ptr[i] + lane; e < row_ptr[i + 1]; e += L) aN[e] = ri * a0[e] * C[col[e]];
        }
    }
}

// max_j |C_j sum_i R_i a0_ij - |M_j|_phi| / |M_j|_phi (the column sums of A^(N))
struct ColErrEpi {
    const double *C, *volphi;
    double mx;
    __device__ void operator()(int64_t j, double s) { mx = fmax(mx, fabs(C[j] * s - volphi[j]) / volphi[j]); }
};

__global__ void __launch_bounds__(kTileThreads) k_scaled_col_error(LineView V, const double *R, const double *C,
                                                                   const double *volphi, unsigned long long *slot) {
    extern __shared__ __align__(16) unsigned char smem[];
    ColErrEpi epi{C, volphi, 0.0};
    NoEpi none;
    const LineView nov{0, nullptr, nullptr, nullptr, nullptr, 0};
    tile_loop(V, R, epi, nov, R, none, smem);
    const double mx = block_max(epi.mx);
    if (threadIdx.x == 0) atomic_max_nonneg(slot, mx);
}

// max_j |sum_i a_ij - |M_j|_phi| / |M_j|_phi over the column view of a
__global__ void k_col_error(int64_t nc, const int64_t *col_ptr, const int32_t *csc_src, const double *a,
                            const double *volphi, unsigned long long *slot) {
    double mx = 0.0;
    GRID_STRIDE(j, nc) {
        double s = 0.0;
        for (int64_t p = col_ptr[j]; p < col_ptr[j + 1]; ++p) s += a[csc_src[p]];
        mx = fmax(mx, fabs(s - volphi[j]) / volphi[j]);
    }
    mx = block_max(mx);
    if (threadIdx.x == 0) atomic_max_nonneg(slot, mx);
}

static void scaling_pass(bchar_mesh_t m, bool col_pass, const double *a0c) {
    const int grid = tile_grid(m->ntile);
    if (col_pass)
        k_scale_tiles<<<grid, kTileThreads, kTileSmem, m->stream>>>(col_view(m, a0c), ptr<double>(m->R), ptr<double>(m->volphi),
                                                            ptr<double>(m->C));
    else
        k_scale_tiles<<<grid, kTileThreads, kTileSmem, m->stream>>>(row_view(m, ptr<double>(m->a0)), ptr<double>(m->C),
                                                            ptr<double>(m->bloc), ptr<double>(m->R));
    ++m->launches;
}

void launch_scaling(bchar_mesh_t m) {
    const int64_t nc = m->nc, nnz = m->nnz;
    const int L = lanes_for(static_cast<double>(nnz) / static_cast<double>(nc > 0 ? nc : 1));
    double *a0c = ptr<double>(m->a2c);  // scratch until the minimisation: A^(0) in column order
    k_gather_col_values<<<blocks_for(nnz), kThreads, 0, m->stream>>>(nnz, ptr<int32_t>(m->csc_src), ptr<double>(m->a0),
                                                                   a0c);
    k_fill<<<blocks_for(nc), kThreads, 0, m->stream>>>(ptr<double>(m->R), nc, 1.0);
    m->launches += 2;
    for (int it = 0; it < m->opt.n_scale; ++it) {
        scaling_pass(m, true, a0c);
        scaling_pass(m, false, a0c);
    }
    if (m->opt.n_scale == 0) {
        k_fill<<<blocks_for(nc), kThreads, 0, m->stream>>>(ptr<double>(m->C), nc, 1.0);
        ++m->launches;
    }
    DISPATCH_LANES(L, (k_apply_scaling<LL><<<kStreamBlocks, 256, 0, m->stream>>>(
                           nc, ptr<int64_t>(m->row_ptr), ptr<int32_t>(m->col), ptr<double>(m->a0), ptr<double>(m->R),
                           ptr<double>(m->C), ptr<double>(m->aN))));
    DevInfo *di = ptr<DevInfo>(m->dinfo);
    k_scaled_col_error<<<tile_grid(m->ntile), kTileThreads, kTileSmem, m->stream>>>(
        col_view(m, a0c), ptr<double>(m->R), ptr<double>(m->C), ptr<double>(m->volphi),
        reinterpret_cast<unsigned long long *>(&di->scale_err));
    m->launches += 2;
}

// One column and one row scaling (timing aid: the streaming stages of a step).
void launch_scaling_once(bchar_mesh_t m) {
    scaling_pass(m, true, ptr<double>(m->a2c));
    scaling_pass(m, false, ptr<double>(m->a2c));
}

// ---------------------------------------------------------------- minimisation
//
// eq. opti_masscons with the bounds 0 <= f = 1 + x <= 2 inside the problem and
// the 2 n_c mass constraints enforced by an elastic penalty on their relative
// violations v_l (see bchar_step in bchar.h): quadratic, weight 1/eps^2, up to
// |v| = 1e-6 and linear beyond, slope gamma = 1e-6 / eps^2.  Solved by a
// primal-dual interior-point method (Mehrotra predictor-corrector) with f, its
// upper slack u = 2 - f (carried separately: f near 2 would lose u to
// rounding), the bound multipliers zl, zh >= 0, the constraint multipliers y
// (node l < n_c: row l, node n_c + j: column j) and, per node, the violation
// beyond the quadratic zone split p - n with p, n >= 0 and multipliers zp, zn:
//     stationarity  rd_e = f_e - 1 - a_e (y_i + y_{n_c+j}) - zl_e + zh_e,
//                   gamma - b_l y_l - zp_l = 0,  gamma + b_l y_l - zn_l = 0
//     constraints   rp_l = b_l - (A-hat f)_l - eps^2 b_l^2 y_l - b_l (p_l - n_l)
//     slack         ru_e = 2 - f_e - u_e
// Each iteration solves the normal equations (A-hat D A-hat^T + diag(exc)) dy = r,
// D_e = 1 / (1 + zl_e / f_e + zh_e / u_e), exc_l = b_l^2 (eps^2 + p_l / zp_l +
// n_l / zn_l), twice with one preconditioner: the bipartite Laplacian of the
// step's pattern with edge weights a_e^2 D_e and that diagonal shift, by the
// conjugate gradients below with the aggregation multigrid.

__global__ void k_qp_gather_cols(int64_t nnz, const int32_t *csc_src, const double *a2, double *a2c) {
    GRID_STRIDE(p, nnz) a2c[p] = a2[csc_src[p]];
}

// Preconditioned conjugate gradients on (A-hat A-hat^T + W) d = F.  Every
// kernel returns at once when the solve has converged, so that batches of
// iterations can be queued without reading the state back each time.

__global__ void k_copy(int64_t n, const double *in, double *out, const CgState *st) {
    if (st && st->converged) return;
    GRID_STRIDE(i, n) out[i] = in[i];
}

// res = rhs - q (the residual of a starting guess whose product is q)
__global__ void k_residual(int64_t n, const double *rhs, const double *q, double *res) {
    GRID_STRIDE(i, n) res[i] = rhs[i] - q[i];
}

// Clears the converged flag a finished solve left, before a product that the
// next solve's start needs (the CG kernels return at once while it is set).
__global__ void k_cg_reopen(CgState *st) { st->converged = 0; }

// z = res / diag (Jacobi preconditioner)
__global__ void k_jacobi_precond(int64_t n, const double *diag, const double *res, double *z, const CgState *st) {
    dep_enter();
    if (st && st->converged) return;
    GRID_STRIDE(i, n) z[i] = res[i] / diag[i];
}

__global__ void k_dot(int64_t n, const double *a, const double *b, double *partials, const CgState *st) {
    if (st && st->converged) return;
    double acc = 0.0;
    GRID_STRIDE(i, n) acc += a[i] * b[i];
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// The target b_l of constraint node l: |K_l|_phi-balanced row target for a
// row node, |M_j|_phi for a column node.
__device__ __forceinline__ double ip_target(int64_t nc, int64_t l, const double *b_row, const double *volphi) {
    return l < nc ? b_row[l] : volphi[l - nc];
}

// Start of a solve: z.res of the initial residual, the two stopping targets
// (z.res <= target and max_l |res_l| / b_l <= target_res; the initial value of
// the latter is rhs_max).
__global__ void k_cg_start(const double *partials, int nparts, double target, double target_res, double rhs_max,
                           CgState *st) {
    double s = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += partials[i];
    s = block_sum(s);
    if (threadIdx.x == 0) {
        st->rz = s;
        st->target = target;
        st->target_res = target_res;
        st->res_max = rhs_max;
        st->converged = (s == 0.0) || (s <= target && rhs_max <= target_res);
        st->iters = 0;
    }
}

// q = (A-hat D A-hat^T + diag(exc)) p through the row view (node l < n_c:
// row l, its entries a2 = a^2 D against the column nodes) and the column view
// (node n_c + j: column j, its entries a2c against the row nodes), tile by
// tile (the row view's tiles first), and per-block partial sums of p.q.
struct MatvecEpi {
    const double *diag, *p;
    double *q;
    int64_t off;  // 0 for the rows, n_c for the columns
    double acc;
    __device__ void operator()(int64_t l, double s) {
        const int64_t node = off + l;
        const double v = s + diag[node] * p[node];
        q[node] = v;
        acc += p[node] * v;
    }
};

__global__ void __launch_bounds__(kTileThreads) k_cg_matvec(LineView Vr, LineView Vc, const double *diag,
                                                            const double *p, double *q, double *partials,
                                                            const CgState *st) {
    dep_enter();
    if (st->converged) return;
    extern __shared__ __align__(16) unsigned char smem[];
    const int64_t nc = Vr.n;
    MatvecEpi er{diag, p, q, 0, 0.0}, ec{diag, p, q, nc, 0.0};
    tile_loop(Vr, p + nc, er, Vc, p, ec, smem);
    const double acc = block_sum(er.acc + ec.acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

__global__ void k_cg_alpha(const double *partials, int nparts, CgState *st) {
    dep_enter();
    if (st->converged) return;
    double s = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += partials[i];
    s = block_sum(s);
    if (threadIdx.x == 0) {
        st->pq = s;
        st->alpha = s > 0.0 ? st->rz / s : 0.0;
    }
}

// d += alpha p, res -= alpha q (the previous residual kept in rp), per-block
// maxima of |res_l| / b_l (res is the constraint residual the direction leaves)
__global__ void k_cg_update(int64_t n2, const double *p, const double *q, double *d, double *res, double *rp,
                            const double *b_row, const double *volphi, double *partials, const CgState *st) {
    dep_enter();
    if (st->converged) return;
    const double alpha = st->alpha;
    const int64_t nc = n2 / 2;
    double mx = 0.0;
    GRID_STRIDE(l, n2) {
        d[l] += alpha * p[l];
        const double r0 = res[l];
        rp[l] = r0;
        const double r = r0 - alpha * q[l];
        res[l] = r;
        mx = fmax(mx, fabs(r) / ip_target(nc, l, b_row, volphi));
    }
    mx = block_max(mx);
    if (threadIdx.x == 0) partials[blockIdx.x] = mx;
}

// The same, also writing the next V-cycle's right-hand side b = S res in its
// precision T (S: +1 rows, -1 columns), so that the V-cycle needs no pass of
// its own over res.
template <class T>
__global__ void k_cg_update_b(int64_t nc, const double *p, const double *q, double *d, double *res, double *rp,
                              const double *b_row, const double *volphi, double *partials, T *b, const CgState *st) {
    dep_enter();
    if (st->converged) return;
    const double alpha = st->alpha;
    double mx = 0.0;
    GRID_STRIDE(l, 2 * nc) {
        d[l] += alpha * p[l];
        const double r0 = res[l];
        rp[l] = r0;
        const double r = r0 - alpha * q[l];
        res[l] = r;
        b[l] = static_cast<T>(l < nc ? r : -r);
        mx = fmax(mx, fabs(r) / ip_target(nc, l, b_row, volphi));
    }
    mx = block_max(mx);
    if (threadIdx.x == 0) partials[blockIdx.x] = mx;
}

// partial sums of z.res and z.rp (flexible, Polak-Ribiere form of beta: the
// preconditioner may differ slightly between applications)
__global__ void k_dot2(int64_t n, const double *z, const double *res, const double *rp, double *pa, double *pb,
                       const CgState *st) {
    dep_enter();
    if (st && st->converged) return;
    double a = 0.0, b = 0.0;
    GRID_STRIDE(i, n) {
        a += z[i] * res[i];
        b += z[i] * rp[i];
    }
    a = block_sum(a);
    b = block_sum(b);
    if (threadIdx.x == 0) {
        pa[blockIdx.x] = a;
        pb[blockIdx.x] = b;
    }
}

__global__ void k_cg_beta(const double *rz_parts, const double *zp_parts, const double *res_parts, int nparts,
                          CgState *st) {
    dep_enter();
    if (st->converged) return;
    double rz = 0.0, zp = 0.0, mx = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        rz += rz_parts[i];
        zp += zp_parts[i];
        mx = fmax(mx, res_parts[i]);
    }
    rz = block_sum(rz);
    zp = block_sum(zp);
    mx = block_max(mx);
    if (threadIdx.x == 0) {
        st->beta = st->rz > 0.0 ? fmax(0.0, (rz - zp) / st->rz) : 0.0;
        st->rz = rz;
        st->res_max = mx;
        st->iters += 1;
        if ((rz <= st->target && mx <= st->target_res) || !(st->pq > 0.0) || !(rz > 0.0)) st->converged = 1;
    }
}

__global__ void k_cg_pupdate(int64_t n2, const double *z, double *p, const CgState *st) {
    dep_enter();
    if (st->converged) return;
    const double beta = st->beta;
    GRID_STRIDE(l, n2) p[l] = z[l] + beta * p[l];
}

// Scalars of one interior-point iteration, reduced over blocks (kRedBlocks
// partial slots each) and read back once.
struct IpScalars {
    double rp_max;      // max_l |rp_l| / b_l (the scaled constraint residual)
    double rd_max;      // max_e |rd_e|
    double rpq_max;     // max_l of the stationarity residuals of p and n
    double dual_max;    // max(max_l |y_l| b_l, max zl, max zh)
    double comp;        // sum of the complementarity products of all pairs
    double rp_l1;       // sum_l |rp_l| (unscaled)
    double ap, ad;      // largest primal / dual step to the boundary (<= 1)
    double comp_aff;    // the same sum after the predictor's steps
};

constexpr int kIpSlots = 8;  // partial-sum slots per block in the reduction scratch

__device__ __forceinline__ double ip_rd(double f, double zl, double zh, double gty) { return f - 1.0 - gty - zl + zh; }

// Entry pass (thread per row): stationarity residuals rd and the entries'
// complementarity sum; slots 0 (max |rd|), 1 (max multiplier), 2 (sum).
__global__ void k_ip_entries(int64_t nc, const int64_t *row_ptr, const int32_t *col, const double *a,
                             const double *y, const double *f, const double *u, const double *zl, const double *zh,
                             double *part) {
    dep_enter();
    double rd_max = 0.0, comp = 0.0, zmax = 0.0;
    GRID_STRIDE(i, nc) {
        const double yi = y[i];
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            rd_max = fmax(rd_max, fabs(ip_rd(f[e], zl[e], zh[e], a[e] * (yi + y[nc + col[e]]))));
            comp += f[e] * zl[e] + u[e] * zh[e];
            zmax = fmax(zmax, fmax(zl[e], zh[e]));
        }
    }
    rd_max = block_max(rd_max);
    zmax = block_max(zmax);
    comp = block_sum(comp);
    if (threadIdx.x == 0) {
        double *pb = part + kIpSlots * blockIdx.x;
        pb[0] = rd_max;
        pb[1] = zmax;
        pb[2] = comp;
    }
}

// Node l: its constraint sum (row l by CSR, column l - n_c by CSC).
__device__ __forceinline__ double ip_node_sum(int64_t nc, int64_t l, const int64_t *row_ptr, const int64_t *col_ptr,
                                              const int32_t *csc_src, const double *a, const double *v) {
    double s = 0.0;
    if (l < nc) {
        for (int64_t e = row_ptr[l]; e < row_ptr[l + 1]; ++e) s += a[e] * v[e];
    } else {
        for (int64_t k = col_ptr[l - nc]; k < col_ptr[l - nc + 1]; ++k) {
            const int32_t e = csc_src[k];
            s += a[e] * v[e];
        }
    }
    return s;
}

// Node pass: constraint residual rp_l = b_l - (A-hat f)_l - eps^2 b_l^2 y_l - b_l (p_l - n_l),
// the stationarity residuals gamma -+ b y - z of p and n, their complementarity;
// slots 3 (max |rp| / b), 4 (max |rdp|, |rdn|), 5 (max |y| b), 6 (sum).
__global__ void k_ip_nodes(int64_t nc, const int64_t *row_ptr, const int64_t *col_ptr, const int32_t *csc_src,
                           const double *a, const double *b_row, const double *volphi, double eps2, double gamma,
                           const double *y, const double *f, const double *p, const double *n, const double *zp,
                           const double *zn, double *rp, double *part) {
    dep_enter();
    double rp_max = 0.0, rpq_max = 0.0, ymax = 0.0, comp = 0.0, rp_l1 = 0.0;
    GRID_STRIDE(l, 2 * nc) {
        const double bl = ip_target(nc, l, b_row, volphi);
        const double ys = y[l] * bl;
        const double r = bl - ip_node_sum(nc, l, row_ptr, col_ptr, csc_src, a, f) - eps2 * bl * ys - bl * (p[l] - n[l]);
        rp[l] = r;
        rp_l1 += fabs(r);
        rp_max = fmax(rp_max, fabs(r) / bl);
        rpq_max = fmax(rpq_max, fmax(fabs(gamma - ys - zp[l]), fabs(gamma + ys - zn[l])));
        ymax = fmax(ymax, fabs(ys));
        comp += p[l] * zp[l] + n[l] * zn[l];
    }
    rp_max = block_max(rp_max);
    rpq_max = block_max(rpq_max);
    ymax = block_max(ymax);
    comp = block_sum(comp);
    rp_l1 = block_sum(rp_l1);
    if (threadIdx.x == 0) {
        double *pb = part + kIpSlots * blockIdx.x;
        pb[3] = rp_max;
        pb[4] = rpq_max;
        pb[5] = ymax;
        pb[6] = comp;
        pb[7] = rp_l1;
    }
}

__global__ void k_ip_reduce_resid(const double *part, int nparts, IpScalars *st) {
    double rd = 0.0, rp = 0.0, rpq = 0.0, dm = 0.0, comp = 0.0, l1 = 0.0;
    for (int k = threadIdx.x; k < nparts; k += blockDim.x) {
        const double *pb = part + kIpSlots * k;
        l1 += pb[7];
        rd = fmax(rd, pb[0]);
        dm = fmax(dm, fmax(pb[1], pb[5]));
        comp += pb[2] + pb[6];
        rp = fmax(rp, pb[3]);
        rpq = fmax(rpq, pb[4]);
    }
    rd = block_max(rd);
    rp = block_max(rp);
    rpq = block_max(rpq);
    dm = block_max(dm);
    comp = block_sum(comp);
    l1 = block_sum(l1);
    if (threadIdx.x == 0) {
        st->rp_l1 = l1;
        st->rd_max = rd;
        st->rp_max = rp;
        st->rpq_max = rpq;
        st->dual_max = dm;
        st->comp = comp;
    }
}

// Normal-equation weights: D_e, a2_e = a_e^2 D_e, and per node
// exc_l = b_l^2 (eps^2 + p_l / zp_l + n_l / zn_l) and diag_l = sum a^2 D + exc_l.
__global__ void k_ip_weights(int64_t nc, const int64_t *row_ptr, const int64_t *col_ptr, const int32_t *csc_src,
                             const double *a, const double *b_row, const double *volphi, double eps2,
                             const double *f, const double *u, const double *zl, const double *zh, const double *p,
                             const double *n, const double *zp, const double *zn, double *D, double *a2, double *diag,
                             double *exc) {
    dep_enter();
    GRID_STRIDE(l, 2 * nc) {
        double d = 0.0;
        if (l < nc) {
            for (int64_t e = row_ptr[l]; e < row_ptr[l + 1]; ++e) {
                const double De = 1.0 / (1.0 + zl[e] / f[e] + zh[e] / u[e]);
                D[e] = De;
                a2[e] = a[e] * a[e] * De;
                d += a2[e];
            }
        } else {
            for (int64_t k = col_ptr[l - nc]; k < col_ptr[l - nc + 1]; ++k) {
                const int32_t e = csc_src[k];
                d += a[e] * a[e] / (1.0 + zl[e] / f[e] + zh[e] / u[e]);
            }
        }
        const double bl = ip_target(nc, l, b_row, volphi);
        const double x = bl * bl * (eps2 + p[l] / zp[l] + n[l] / zn[l]);
        diag[l] = d + x;
        exc[l] = x;
    }
}

// Reduced right-hand side per entry for the predictor (corrector = 0) or the
// corrector (sigma_mu = sigma * mu, with the predictor's direction in df..dzh):
//   cl = target of f zl, ch = target of u zh,
//   q = -rd + cl / f - ch / u + (zh / u) ru.
__global__ void k_ip_q(int64_t nc, const int64_t *row_ptr, const int32_t *col, const double *a, const double *y,
                       const double *f, const double *u, const double *zl, const double *zh, int corrector,
                       double sigma_mu, const double *df, const double *du, const double *dzl, const double *dzh,
                       double *cl, double *ch, double *q) {
    dep_enter();
    GRID_STRIDE(i, nc) {
        const double yi = y[i];
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            const double fe = f[e], ue = u[e], zle = zl[e], zhe = zh[e];
            const double rd = ip_rd(fe, zle, zhe, a[e] * (yi + y[nc + col[e]]));
            const double ru = 2.0 - fe - ue;
            double c_lo = -fe * zle, c_hi = -ue * zhe;
            if (corrector) {
                c_lo += sigma_mu - df[e] * dzl[e];
                c_hi += sigma_mu - du[e] * dzh[e];
            }
            cl[e] = c_lo;
            ch[e] = c_hi;
            q[e] = -rd + c_lo / fe - c_hi / ue + (zhe / ue) * ru;
        }
    }
}

// Per node: the targets of p zp and n zn, and
// rhs_l = rp_l - (A-hat (D q))_l - b_l (p/zp sp - n/zn sn),
// sp = -(gamma - b y - zp) + cp / p, sn = -(gamma + b y - zn) + cn / n.
__global__ void k_ip_rhs(int64_t nc, const int64_t *row_ptr, const int64_t *col_ptr, const int32_t *csc_src,
                         const double *a, const double *D, const double *q, const double *rp, const double *b_row,
                         const double *volphi, double gamma, const double *y, const double *p, const double *n,
                         const double *zp, const double *zn, int corrector, double sigma_mu, const double *dp,
                         const double *dn, const double *dzp, const double *dzn, double *cp, double *cn, double *rhs) {
    dep_enter();
    GRID_STRIDE(l, 2 * nc) {
        double s = 0.0;
        if (l < nc) {
            for (int64_t e = row_ptr[l]; e < row_ptr[l + 1]; ++e) s += a[e] * D[e] * q[e];
        } else {
            for (int64_t k = col_ptr[l - nc]; k < col_ptr[l - nc + 1]; ++k) {
                const int32_t e = csc_src[k];
                s += a[e] * D[e] * q[e];
            }
        }
        const double bl = ip_target(nc, l, b_row, volphi);
        const double ys = y[l] * bl;
        double c_p = -p[l] * zp[l], c_n = -n[l] * zn[l];
        if (corrector) {
            c_p += sigma_mu - dp[l] * dzp[l];
            c_n += sigma_mu - dn[l] * dzn[l];
        }
        cp[l] = c_p;
        cn[l] = c_n;
        const double sp = -(gamma - ys - zp[l]) + c_p / p[l];
        const double sn = -(gamma + ys - zn[l]) + c_n / n[l];
        rhs[l] = rp[l] - s - bl * (p[l] / zp[l] * sp - n[l] / zn[l] * sn);
    }
}

// Direction per entry from dy, and the ratio tests (largest steps <= 1 that
// keep f, u, zl, zh positive), reduced per block as their reciprocals
// max(1, -dv / v) into slots 0 (primal) and 1 (dual).
__global__ void k_ip_dir(int64_t nc, const int64_t *row_ptr, const int32_t *col, const double *a, const double *dy,
                         const double *f, const double *u, const double *zl, const double *zh, const double *D,
                         const double *q, const double *cl, const double *ch, double *df, double *du, double *dzl,
                         double *dzh, double *part) {
    dep_enter();
    double ap_inv = 1.0, ad_inv = 1.0;
    GRID_STRIDE(i, nc) {
        const double di = dy[i];
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            const double fe = f[e], ue = u[e];
            const double d_f = D[e] * (q[e] + a[e] * (di + dy[nc + col[e]]));
            const double ru = 2.0 - fe - ue;
            const double d_u = ru - d_f;
            const double d_zl = (cl[e] - zl[e] * d_f) / fe;
            const double d_zh = (ch[e] - zh[e] * d_u) / ue;
            df[e] = d_f;
            du[e] = d_u;
            dzl[e] = d_zl;
            dzh[e] = d_zh;
            ap_inv = fmax(ap_inv, fmax(-d_f / fe, -d_u / ue));
            ad_inv = fmax(ad_inv, fmax(-d_zl / zl[e], -d_zh / zh[e]));
        }
    }
    ap_inv = block_max(ap_inv);  // block_max pads with 0: only for non-negative values
    ad_inv = block_max(ad_inv);
    if (threadIdx.x == 0) {
        part[kIpSlots * blockIdx.x] = ap_inv;
        part[kIpSlots * blockIdx.x + 1] = ad_inv;
    }
}

// The same per node for p, n and their multipliers (dy scaled: b_l dy_l),
// into slots 2 (primal) and 3 (dual).
__global__ void k_ip_dir_nodes(int64_t nc, const double *b_row, const double *volphi, double gamma, const double *y,
                               const double *dy, const double *p, const double *n, const double *zp, const double *zn,
                               const double *cp, const double *cn, double *dp, double *dn, double *dzp, double *dzn,
                               double *part) {
    dep_enter();
    double ap_inv = 1.0, ad_inv = 1.0;
    GRID_STRIDE(l, 2 * nc) {
        const double bl = ip_target(nc, l, b_row, volphi);
        const double ys = y[l] * bl, dys = dy[l] * bl;
        const double sp = -(gamma - ys - zp[l]) + cp[l] / p[l];
        const double sn = -(gamma + ys - zn[l]) + cn[l] / n[l];
        const double d_p = p[l] / zp[l] * (sp + dys);
        const double d_n = n[l] / zn[l] * (sn - dys);
        const double d_zp = (cp[l] - zp[l] * d_p) / p[l];
        const double d_zn = (cn[l] - zn[l] * d_n) / n[l];
        dp[l] = d_p;
        dn[l] = d_n;
        dzp[l] = d_zp;
        dzn[l] = d_zn;
        ap_inv = fmax(ap_inv, fmax(-d_p / p[l], -d_n / n[l]));
        ad_inv = fmax(ad_inv, fmax(-d_zp / zp[l], -d_zn / zn[l]));
    }
    ap_inv = block_max(ap_inv);
    ad_inv = block_max(ad_inv);
    if (threadIdx.x == 0) {
        part[kIpSlots * blockIdx.x + 2] = ap_inv;
        part[kIpSlots * blockIdx.x + 3] = ad_inv;
    }
}

__global__ void k_ip_reduce_steps(const double *part, int nparts, IpScalars *st) {
    double ap_inv = 1.0, ad_inv = 1.0;
    for (int k = threadIdx.x; k < nparts; k += blockDim.x) {
        const double *pb = part + kIpSlots * k;
        ap_inv = fmax(ap_inv, fmax(pb[0], pb[2]));
        ad_inv = fmax(ad_inv, fmax(pb[1], pb[3]));
    }
    ap_inv = block_max(ap_inv);
    ad_inv = block_max(ad_inv);
    if (threadIdx.x == 0) {
        st->ap = 1.0 / ap_inv;
        st->ad = 1.0 / ad_inv;
    }
}

// Complementarity after the predictor's steps to the boundary: entries into
// slot 4, nodes into slot 5.
__global__ void k_ip_comp_aff(int64_t nnz, int64_t n2, const double *f, const double *u, const double *zl,
                              const double *zh, const double *df, const double *du, const double *dzl,
                              const double *dzh, const double *p, const double *n, const double *zp, const double *zn,
                              const double *dp, const double *dn, const double *dzp, const double *dzn,
                              const IpScalars *st, double *part) {
    dep_enter();
    const double ap = st->ap, ad = st->ad;
    double s = 0.0, t = 0.0;
    GRID_STRIDE(e, nnz > n2 ? nnz : n2) {
        if (e < nnz)
            s += (f[e] + ap * df[e]) * (zl[e] + ad * dzl[e]) + (u[e] + ap * du[e]) * (zh[e] + ad * dzh[e]);
        if (e < n2)
            t += (p[e] + ap * dp[e]) * (zp[e] + ad * dzp[e]) + (n[e] + ap * dn[e]) * (zn[e] + ad * dzn[e]);
    }
    s = block_sum(s);
    t = block_sum(t);
    if (threadIdx.x == 0) {
        part[kIpSlots * blockIdx.x + 4] = s;
        part[kIpSlots * blockIdx.x + 5] = t;
    }
}

__global__ void k_ip_reduce_comp_aff(const double *part, int nparts, IpScalars *st) {
    double s = 0.0;
    for (int k = threadIdx.x; k < nparts; k += blockDim.x) s += part[kIpSlots * k + 4] + part[kIpSlots * k + 5];
    s = block_sum(s);
    if (threadIdx.x == 0) st->comp_aff = s;
}

// Step with fraction 0.99 of the way to the boundary.
__global__ void k_ip_update(int64_t nnz, int64_t n2, const IpScalars *st, double frac, const double *df,
                            const double *du, const double *dzl, const double *dzh, const double *dy, const double *dp,
                            const double *dn, const double *dzp, const double *dzn, double *f, double *u, double *zl,
                            double *zh, double *y, double *p, double *n, double *zp, double *zn) {
    dep_enter();
    const double ap = frac * st->ap, ad = frac * st->ad;
    GRID_STRIDE(e, nnz > n2 ? nnz : n2) {
        if (e < nnz) {
            f[e] += ap * df[e];
            u[e] += ap * du[e];
            zl[e] += ad * dzl[e];
            zh[e] += ad * dzh[e];
        }
        if (e < n2) {
            y[e] += ad * dy[e];
            p[e] += ap * dp[e];
            n[e] += ap * dn[e];
            zp[e] += ad * dzp[e];
            zn[e] += ad * dzn[e];
        }
    }
}

__global__ void k_ip_init(int64_t nnz, int64_t n2, double z0, double p0, double zp0, double *f, double *u,
                          double *zl, double *zh, double *y, double *p, double *n, double *zp, double *zn) {
    GRID_STRIDE(e, nnz > n2 ? nnz : n2) {
        if (e < nnz) {
            f[e] = 1.0;
            u[e] = 1.0;
            zl[e] = z0;
            zh[e] = z0;
        }
        if (e < n2) {
            y[e] = 0.0;
            p[e] = p0;
            n[e] = p0;
            zp[e] = zp0;
            zn[e] = zp0;
        }
    }
}

// x_e = f_e - 1 (kept in qx for the bounds / column-fix stage) and the count
// of entries within 1e-9 of a bound.
__global__ void k_ip_finish(int64_t nnz, const double *f, double *qx, DevInfo *info) {
    int at = 0;
    GRID_STRIDE(e, nnz) {
        const double fe = fmin(fmax(f[e], 0.0), 2.0);
        qx[e] = fe - 1.0;
        if (fe < 1e-9 || fe > 2.0 - 1e-9) ++at;
    }
    if (at) atomicAdd(&info->n_at_bounds, at);
}

static void precondition(bchar_mesh_t m, bool amg, const double *res, double *z, const CgState *st,
                         bool b_ready = false, const double *rp = nullptr, double *pa = nullptr,
                         double *pb = nullptr) {
    if (amg) {
        amg_apply(m, m->amg, res, z, st, b_ready, rp, pa, pb);
    } else {
        k_jacobi_precond<<<blocks_for(2 * m->nc), kThreads, 0, m->stream>>>(2 * m->nc, ptr<double>(m->diag), res, z, st);
        ++m->launches;
    }
}

// A solve of the conjugate gradients stops when its residual has not dropped
// by 1 % for kStallIters iterations (it cannot improve further in FP64).
constexpr int kStallIters = 400;

// The conjugate gradients on (A-hat D A-hat^T + diag(exc)) d = rhs, from
// d = 0 (or, with warm, from the d already in place), until z.res <= target_rz
// (z the preconditioned residual: about the squared error of d in the norm of
// the matrix, which bounds the error of A-hat^T d where the interior-point
// direction needs it -- an L1 test alone would not bound the error along the
// nearly singular modes of weakly linked cells) and max_l |res_l| / b_l <=
// target_res (after a full step, res is the constraint residual, which the
// interior point measures in that norm).  One batch of iterations is captured
// into a CUDA graph per preconditioner build (*exec; destroyed by the caller)
// and replayed until the solve has converged (its kernels do nothing then);
// the host polls once per batch.  Returns the iterations done.
static int pcg_solve(bchar_mesh_t m, const double *rhs, double target_rz, double target_res, bool amg, bool warm,
                     int max_iter, cudaGraphExec_t *exec, int *graph_launches) {
    const int64_t nc = m->nc, n2 = 2 * nc;
    const int bl = blocks_for(n2);
    cudaStream_t s = m->stream;
    double *a2 = ptr<double>(m->a2), *a2c = ptr<double>(m->a2c), *diag = ptr<double>(m->diag);
    double *d = ptr<double>(m->cg_d), *res = ptr<double>(m->cg_r), *z = ptr<double>(m->cg_z);
    double *p = ptr<double>(m->cg_p), *q = ptr<double>(m->cg_q), *rp = ptr<double>(m->cg_rp);
    double *part = ptr<double>(m->partials);
    double *part_res = part + 152 * 64;
    const double *brow = ptr<double>(m->bloc), *volphi = ptr<double>(m->volphi);
    double *part_rz = part + 2 * 152 * 64;
    double *part_zp = part + 3 * 152 * 64;
    CgState *st = ptr<CgState>(m->cg);
    CgState *host_st = reinterpret_cast<CgState *>(static_cast<char *>(m->info_host.p) + sizeof(DevInfo));
    if (warm) {  // start from the d already in place: res = rhs - M d
        k_cg_reopen<<<1, 1, 0, s>>>(st);
        k_cg_matvec<<<tile_grid(2 * m->ntile), kTileThreads, kTileSmem, s>>>(
            row_view(m, a2), col_view(m, a2c), diag, d, q, part, st);
        k_residual<<<bl, kThreads, 0, s>>>(n2, rhs, q, res);
        m->launches += 3;
    } else {
        cudaMemsetAsync(d, 0, sizeof(double) * n2, s);
        k_copy<<<bl, kThreads, 0, s>>>(n2, rhs, res, nullptr);
        ++m->launches;
    }
    precondition(m, amg, res, z, nullptr);
    k_dot<<<kRedBlocks, kThreads, 0, s>>>(n2, res, z, part_rz, nullptr);
    // the right-hand side's residual norm is not formed: the first iteration checks it
    k_cg_start<<<1, 1024, 0, s>>>(part_rz, kRedBlocks, target_rz, target_res, INFINITY, st);
    k_copy<<<bl, kThreads, 0, s>>>(n2, z, p, nullptr);
    m->launches += 3;
    const int batch = amg ? 8 : 32;
    const int mv_grid = tile_grid(2 * m->ntile);  // <= kRedBlocks partial sums of p.q
    auto enqueue_batch = [&]() {
        for (int k = 0; k < batch; ++k) {
            launch_dep_smem(k_cg_matvec, mv_grid, kTileThreads, kTileSmem, s, row_view(m, a2), col_view(m, a2c), diag, p,
                            q, part, st);
            launch_dep(k_cg_alpha, 1, 1024, s, part, mv_grid, st);
            if (amg) {
                launch_dep(k_cg_update_b<double>, kRedBlocks, kThreads, s, nc, p, q, d, res, rp, brow, volphi, part_res,
                           amg_finest_rhs(m->amg), st);
                precondition(m, amg, res, z, st, true, rp, part_rz, part_zp);
                m->launches += 3;
            } else {
                launch_dep(k_cg_update, kRedBlocks, kThreads, s, n2, p, q, d, res, rp, brow, volphi, part_res, st);
                precondition(m, amg, res, z, st);
                launch_dep(k_dot2, kRedBlocks, kThreads, s, n2, z, res, rp, part_rz, part_zp, st);
                m->launches += 4;
            }
            launch_dep(k_cg_beta, 1, 1024, s, part_rz, part_zp, part_res, kRedBlocks, st);
            launch_dep(k_cg_pupdate, bl, kThreads, s, n2, z, p, st);
            m->launches += 2;
        }
    };
    if (!*exec) {
        const int before = m->launches;
        cudaGraph_t graph = nullptr;
        bool ok = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            enqueue_batch();
            ok = cudaStreamEndCapture(s, &graph) == cudaSuccess && graph;
        }
        if (ok) ok = cudaGraphInstantiate(exec, graph, 0) == cudaSuccess;
        if (graph) cudaGraphDestroy(graph);
        if (!ok) {  // capture unavailable (for instance, the caller is capturing): plain launches
            cudaGetLastError();
            *exec = nullptr;
        }
        *graph_launches = m->launches - before;
        m->launches = before;
    }
    double best = INFINITY;
    int best_at = 0;
    for (;;) {
        if (*exec) {
            cudaGraphLaunch(*exec, s);
            m->launches += *graph_launches;
        } else {
            enqueue_batch();
        }
        cudaMemcpyAsync(host_st, st, sizeof(CgState), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        if (host_st->converged || host_st->iters >= max_iter) break;
        if (host_st->res_max < 0.99 * best) {
            best = host_st->res_max;
            best_at = host_st->iters;
        } else if (host_st->iters - best_at >= kStallIters) {
            break;
        }
    }
    return host_st->iters;
}

// Host wall clock in milliseconds (for the diagnostic trace only).
static double trace_ms() {
    timespec t;
    clock_gettime(CLOCK_MONOTONIC, &t);
    return t.tv_sec * 1e3 + t.tv_nsec * 1e-6;
}

// The elastic penalty of the constraints is quadratic up to a relative
// violation kLinearFrom and linear beyond, with slope gamma = kLinearFrom / eps^2.
constexpr double kLinearFrom = 1e-6;
// The interior-point stopping rule: scaled constraint residual <= qp_tol,
// mean complementarity <= 1e-12, the stationarity residual of 1 + x <= 1e-12 of
// the largest dual value and those of the violation parts <= 1e-12 of gamma
// (y and the multipliers reach ~gamma where the problem is infeasible, and the
// residuals then carry that much rounding).
constexpr double kIpMuTol = 1e-12;
// The corrector's centring target never goes below kIpMuFloor: once the mean
// complementarity meets its tolerance, the iterations that are still needed to
// bring the constraint residual down hold it there instead of driving it
// towards zero (which makes the normal equations so badly conditioned that the
// inexact solves raise the constraint residual again).
constexpr double kIpMuFloor = 0.1 * kIpMuTol;
// Conjugate-gradient iterations per interior-point solve at most (the late
// normal equations are badly conditioned; an inexact direction is corrected by
// the next iteration).
constexpr int kIpCgPerSolve = 400;
constexpr double kIpRdRel = 1e-12;
constexpr double kIpStep = 0.99;
// The starting point: y = 0; the violation parts p = n = kIpStartViol with
// multipliers gamma, which satisfies their stationarity at y = 0; f = u = 1
// with multipliers kIpStartViol * gamma, so that every complementarity
// product starts equal (a centred point).  Multipliers 1 for the violation
// parts leave a dual residual of gamma = 1e8 for the first Newton step, after
// which the steps shrink to nothing on some small meshes; uncentred starts
// take up to twice the iterations on the 1024^2 workload.
constexpr double kIpStartViol = 0.1;

bool launch_minimise(bchar_mesh_t m, int *cg_iters, int *ip_iters) {
    const bool trace = getenv("BCHAR_TRACE") != nullptr;  // diagnostic: per-iteration scalars on stderr
    double t_start = 0.0;
    if (trace) {
        cudaStreamSynchronize(m->stream);
        t_start = trace_ms();
    }
    const int64_t nc = m->nc, n2 = 2 * nc, nnz = m->nnz;
    const size_t zb = sizeof(double) * (nnz > 0 ? nnz : 1), nb = sizeof(double) * n2;
    Buf *ent[] = {&m->ip_f, &m->ip_u, &m->ip_zl, &m->ip_zh, &m->ip_D, &m->ip_q, &m->ip_cl, &m->ip_ch,
                  &m->ip_df, &m->ip_du, &m->ip_dzl, &m->ip_dzh};
    for (Buf *b : ent)
        if (!ensure(m, *b, zb)) return false;
    Buf *nod[] = {&m->ip_p, &m->ip_n, &m->ip_zp, &m->ip_zn, &m->ip_cp, &m->ip_cn, &m->ip_dp, &m->ip_dn,
                  &m->ip_dzp, &m->ip_dzn};
    for (Buf *b : nod)
        if (!ensure(m, *b, nb)) return false;
    static_assert(kIpSlots * kRedBlocks <= 152 * 64, "interior-point partials fit the first scratch section");
    cudaStream_t s = m->stream;
    const double eps2 = m->opt.penalty * m->opt.penalty;
    const double gamma = kLinearFrom / eps2;
    const int64_t *row_ptr = ptr<int64_t>(m->row_ptr), *col_ptr = ptr<int64_t>(m->col_ptr);
    const int32_t *col = ptr<int32_t>(m->col), *csc_src = ptr<int32_t>(m->csc_src);
    const double *a = ptr<double>(m->aN), *brow = ptr<double>(m->bloc), *volphi = ptr<double>(m->volphi);
    double *f = ptr<double>(m->ip_f), *u = ptr<double>(m->ip_u), *zl = ptr<double>(m->ip_zl),
           *zh = ptr<double>(m->ip_zh), *D = ptr<double>(m->ip_D), *q = ptr<double>(m->ip_q),
           *cl = ptr<double>(m->ip_cl), *ch = ptr<double>(m->ip_ch), *df = ptr<double>(m->ip_df),
           *du = ptr<double>(m->ip_du), *dzl = ptr<double>(m->ip_dzl), *dzh = ptr<double>(m->ip_dzh);
    double *p = ptr<double>(m->ip_p), *n = ptr<double>(m->ip_n), *zp = ptr<double>(m->ip_zp),
           *zn = ptr<double>(m->ip_zn), *cp = ptr<double>(m->ip_cp), *cn = ptr<double>(m->ip_cn),
           *dp = ptr<double>(m->ip_dp), *dn = ptr<double>(m->ip_dn), *dzp = ptr<double>(m->ip_dzp),
           *dzn = ptr<double>(m->ip_dzn);
    double *y = ptr<double>(m->qy), *rp = ptr<double>(m->F), *rhs = ptr<double>(m->rhs), *dy = ptr<double>(m->cg_d);
    double *part = ptr<double>(m->partials);
    IpScalars *st = reinterpret_cast<IpScalars *>(ptr<CgState>(m->cg) + 1);
    static_assert(sizeof(CgState) + sizeof(IpScalars) <= 256, "both scalar blocks fit the cg buffer");
    IpScalars hs{};
    const int blr = kRedBlocks;  // the entry and node passes are grid-stride over kRedBlocks blocks
    const int bl2 = blocks_for(n2);
    const int blm = blocks_for(nnz > n2 ? nnz : n2);
    const double pairs = 2.0 * static_cast<double>(nnz) + 2.0 * static_cast<double>(n2);
    const bool use_amg = m->opt.qp_precond == 1;

    k_ip_init<<<blm, kThreads, 0, s>>>(nnz, n2, kIpStartViol * gamma, kIpStartViol, gamma, f, u, zl, zh, y, p, n, zp,
                                       zn);
    ++m->launches;
    int it = 0, total_cg = 0;
    bool converged = false;
    for (it = 0; it <= m->opt.qp_max_refine; ++it) {
        launch_dep(k_ip_entries, blr, kThreads, s, nc, row_ptr, col, a, y, f, u, zl, zh, part);
        launch_dep(k_ip_nodes, blr, kThreads, s, nc, row_ptr, col_ptr, csc_src, a, brow, volphi, eps2, gamma, y, f, p,
                   n, zp, zn, rp, part);
        k_ip_reduce_resid<<<1, 1024, 0, s>>>(part, blr, st);
        m->launches += 3;
        cudaMemcpyAsync(&hs, st, sizeof hs, cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) break;  // the caller reads the error
        const double mu = hs.comp / pairs;
        if (trace)
            fprintf(stderr, "[bchar] ip %d rp %.3e rd %.3e rpq %.3e mu %.3e dual %.3e ap %.3e ad %.3e cg %d (%.1f ms)\n",
                    it, hs.rp_max, hs.rd_max, hs.rpq_max, mu, hs.dual_max, hs.ap, hs.ad, total_cg,
                    trace_ms() - t_start);
        if (hs.rp_max <= m->opt.qp_tol && mu <= kIpMuTol && hs.rd_max <= kIpRdRel * (1.0 + hs.dual_max) &&
            hs.rpq_max <= kIpRdRel * (1.0 + gamma)) {
            converged = true;
            break;
        }
        if (it == m->opt.qp_max_refine || total_cg >= m->opt.qp_max_iter) break;
        // normal-equation matrix and its preconditioner; the weights change by orders of
        // magnitude between iterations, so the aggregates are built anew every time
        launch_dep(k_ip_weights, bl2, kThreads, s, nc, row_ptr, col_ptr, csc_src, a, brow, volphi, eps2, f, u, zl, zh, p,
                   n, zp, zn, D, ptr<double>(m->a2), ptr<double>(m->diag), ptr<double>(m->qexc));
        k_qp_gather_cols<<<blocks_for(nnz), kThreads, 0, s>>>(nnz, csc_src, ptr<double>(m->a2), ptr<double>(m->a2c));
        m->launches += 2;
        const bool amg = use_amg && amg_build(m, m->amg);
        // each direction solved until its squared energy-norm error is about <= 1e-2 mu (then
        // every entry's step error stays about <= 0.1 of its distance to the bound) and the
        // constraint residual it leaves is, relative to each target, <= 0.1 of the current
        // one (which the step then reduces), but not below half the stopping tolerance
        const double target_rz = 1e-2 * mu;
        const double target_res = fmax(0.1 * hs.rp_max, 0.5 * m->opt.qp_tol);
        cudaGraphExec_t exec = nullptr;
        int graph_launches = 0;
        for (int corr = 0; corr < 2; ++corr) {
            const double sigma_mu = corr ? fmax(fmin(1.0, pow(hs.comp_aff / hs.comp, 3.0)) * mu, kIpMuFloor) : 0.0;
            launch_dep(k_ip_q, blr, kThreads, s, nc, row_ptr, col, a, y, f, u, zl, zh, corr, sigma_mu, df, du, dzl,
                       dzh, cl, ch, q);
            launch_dep(k_ip_rhs, bl2, kThreads, s, nc, row_ptr, col_ptr, csc_src, a, D, q, rp, brow, volphi, gamma, y,
                       p, n, zp, zn, corr, sigma_mu, dp, dn, dzp, dzn, cp, cn, rhs);
            m->launches += 2;
            const int left = m->opt.qp_max_iter - total_cg;
            const int cap = left < kIpCgPerSolve ? left : kIpCgPerSolve;
            // the right-hand side's L1 norm: the node pass's |rp|_1 bounds it well enough for the start
            // the corrector's system differs from the predictor's only in its right-hand
            // side (the centring and second-order terms): its solve starts from the
            // predictor's direction
            const int done = pcg_solve(m, rhs, target_rz, target_res, amg, corr == 1, cap > 0 ? cap : 1,
                                       &exec, &graph_launches);
            total_cg += done;
            if (trace)
                fprintf(stderr, "[bchar]   solve %d: %d CG iterations, levels %d, coarsest %lld\n", corr, done,
                        amg ? m->amg.nlev : 0, amg ? static_cast<long long>(m->amg.levels[m->amg.nlev - 1].n) : 0LL);
            launch_dep(k_ip_dir, blr, kThreads, s, nc, row_ptr, col, a, dy, f, u, zl, zh, D, q, cl, ch, df, du, dzl,
                       dzh, part);
            launch_dep(k_ip_dir_nodes, blr, kThreads, s, nc, brow, volphi, gamma, y, dy, p, n, zp, zn, cp, cn, dp, dn,
                       dzp, dzn, part);
            k_ip_reduce_steps<<<1, 1024, 0, s>>>(part, blr, st);
            m->launches += 3;
            if (!corr) {
                launch_dep(k_ip_comp_aff, blr, kThreads, s, nnz, n2, f, u, zl, zh, df, du, dzl, dzh, p, n, zp, zn, dp,
                           dn, dzp, dzn, st, part);
                k_ip_reduce_comp_aff<<<1, 1024, 0, s>>>(part, blr, st);
                m->launches += 2;
                cudaMemcpyAsync(&hs, st, sizeof hs, cudaMemcpyDeviceToHost, s);
                cudaStreamSynchronize(s);
            }
        }
        if (exec) cudaGraphExecDestroy(exec);
        launch_dep(k_ip_update, blm, kThreads, s, nnz, n2, st, kIpStep, df, du, dzl, dzh, dy, dp, dn, dzp, dzn, f, u,
                   zl, zh, y, p, n, zp, zn);
        ++m->launches;
    }
    k_ip_finish<<<blocks_for(nnz), kThreads, 0, s>>>(nnz, f, ptr<double>(m->qx), ptr<DevInfo>(m->dinfo));
    ++m->launches;
    DevInfo *di = ptr<DevInfo>(m->dinfo);
    cudaMemcpyAsync(&di->kkt_l1, &st->rp_max, sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (trace) {
        cudaStreamSynchronize(s);
        fprintf(stderr, "[bchar] interior point: %d iterations, %d CG iterations, %s, %.3f ms\n", it, total_cg,
                converged ? "converged" : "not converged", trace_ms() - t_start);
    }
    m->ip_iters = it;
    m->ip_converged = converged;
    *cg_iters = total_cg;
    *ip_iters = it;
    m->amg_levels = use_amg ? m->amg.nlev : 0;
    m->amg_coarsest = use_amg && m->amg.nlev > 0 ? m->amg.levels[m->amg.nlev - 1].n : 0;
    return true;
}

void launch_cg_matvec_once(bchar_mesh_t m, CgState *st) {
    k_cg_matvec<<<tile_grid(2 * m->ntile), kTileThreads, kTileSmem, m->stream>>>(
        row_view(m, ptr<double>(m->a2)), col_view(m, ptr<double>(m->a2c)), ptr<double>(m->diag), ptr<double>(m->cg_p),
        ptr<double>(m->cg_q), ptr<double>(m->partials), st);
}

// ---------------------------------------------------------------- bounds, column fix, W

// a_q = a^(N) (1 + x), per row (1 + x is inside [0, 2] by construction).
__global__ void k_clip(int64_t nc, const int64_t *row_ptr, const double *aN, const double *qx, double *aq) {
    GRID_STRIDE(i, nc) {
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) aq[e] = aN[e] * fmin(fmax(1.0 + qx[e], 0.0), 2.0);
    }
}

// C2_j = |M_j|_phi / sum_i a_q,ij (first half of eq. volAdj).  A column whose
// entries all ended on the bound 0 keeps its A^(N) entries (dead[j] = 1).
__global__ void k_colfix(int64_t nc, const int64_t *col_ptr, const int32_t *csc_src, const double *aq,
                         const double *aN, const double *volphi, double *C2, int32_t *dead) {
    GRID_STRIDE(j, nc) {
        double s = 0.0;
        for (int64_t p = col_ptr[j]; p < col_ptr[j + 1]; ++p) s += aq[csc_src[p]];
        int d = 0;
        if (s == 0.0) {
            d = 1;
            for (int64_t p = col_ptr[j]; p < col_ptr[j + 1]; ++p) s += aN[csc_src[p]];
        }
        dead[j] = d;
        C2[j] = volphi[j] / s;
    }
}

// a_KM final, W_KM = a_KM / |K|_phi, and the relative row residual.
__global__ void k_weights(int64_t nc, const int64_t *row_ptr, const int32_t *col, const double *aq, const double *aN,
                          const int32_t *dead, const double *C2, const double *volphi, double *afin, double *wgt,
                          unsigned long long *row_res) {
    double mx = 0.0;
    GRID_STRIDE(i, nc) {
        double s = 0.0;
        const double vi = volphi[i];
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            const int32_t j = col[e];
            const double a = (dead[j] ? aN[e] : aq[e]) * C2[j];
            afin[e] = a;
            wgt[e] = a / vi;
            s += a;
        }
        mx = fmax(mx, fabs(s - vi) / vi);
    }
    mx = block_max(mx);
    if (threadIdx.x == 0) atomic_max_nonneg(row_res, mx);
}

void launch_finalise(bchar_mesh_t m) {
    const int64_t nc = m->nc;
    const int bl = blocks_for(nc);
    DevInfo *di = ptr<DevInfo>(m->dinfo);
    double *aq = ptr<double>(m->a2);  // reuse: a2 is no longer needed
    k_clip<<<bl, kThreads, 0, m->stream>>>(nc, ptr<int64_t>(m->row_ptr), ptr<double>(m->aN), ptr<double>(m->qx), aq);
    int32_t *dead = ptr<int32_t>(m->colfill);  // scratch: the column fill counters are no longer needed
    k_colfix<<<bl, kThreads, 0, m->stream>>>(nc, ptr<int64_t>(m->col_ptr), ptr<int32_t>(m->csc_src), aq,
                                             ptr<double>(m->aN), ptr<double>(m->volphi), ptr<double>(m->C), dead);
    k_weights<<<bl, kThreads, 0, m->stream>>>(nc, ptr<int64_t>(m->row_ptr), ptr<int32_t>(m->col), aq, ptr<double>(m->aN),
                                              dead, ptr<double>(m->C), ptr<double>(m->volphi), ptr<double>(m->afin),
                                              ptr<double>(m->wgt),
                                              reinterpret_cast<unsigned long long *>(&di->max_rel_row_res));
    k_col_error<<<bl, kThreads, 0, m->stream>>>(nc, ptr<int64_t>(m->col_ptr), ptr<int32_t>(m->csc_src),
                                                ptr<double>(m->afin), ptr<double>(m->volphi),
                                                reinterpret_cast<unsigned long long *>(&di->max_rel_col_res));
    m->launches += 4;
}

// ---------------------------------------------------------------- update (eq. phys-inter-ELLAM)

// c_out_i = sum_j W_ij c_in_j with FP64 accumulation, rounded once on store,
// tile by tile over the row view, and per-block partial sums of the three
// masses sum |K|_phi c (before, after the FP64 update, after the stored
// rounding), all in one pass.
template <class T> struct SpmvEpi {
    const double *volphi;
    const T *c_in;
    T *c_out;
    double mb, ma, ms;
    __device__ void operator()(int64_t i, double s) {
        const T stored = static_cast<T>(s);
        c_out[i] = stored;
        const double v = volphi[i];
        mb += v * static_cast<double>(c_in[i]);
        ma += v * s;
        ms += v * static_cast<double>(stored);
    }
};

template <class T>
__global__ void __launch_bounds__(kTileThreads) k_spmv(LineView V, const double *volphi, const T *c_in, T *c_out,
                                                       double *partials) {
    extern __shared__ __align__(16) unsigned char smem[];
    SpmvEpi<T> epi{volphi, c_in, c_out, 0.0, 0.0, 0.0};
    NoEpi none;
    const LineView nov{0, nullptr, nullptr, nullptr, nullptr, 0};
    tile_loop(V, c_in, epi, nov, c_in, none, smem);
    const double mb = block_sum(epi.mb);
    const double ma = block_sum(epi.ma);
    const double ms = block_sum(epi.ms);
    if (threadIdx.x == 0) {
        partials[3 * blockIdx.x] = mb;
        partials[3 * blockIdx.x + 1] = ma;
        partials[3 * blockIdx.x + 2] = ms;
    }
}

__global__ void k_mass_final(const double *partials, int n, DevInfo *info) {
    double mb = 0.0, ma = 0.0, ms = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        mb += partials[3 * i];
        ma += partials[3 * i + 1];
        ms += partials[3 * i + 2];
    }
    mb = block_sum(mb);
    ma = block_sum(ma);
    ms = block_sum(ms);
    if (threadIdx.x == 0) {
        info->mass_before = mb;
        info->mass_after = ma;
        info->mass_after_stored = ms;
    }
}

void launch_update(bchar_mesh_t m, const void *c_in, void *c_out, int c_dtype) {
    double *part = ptr<double>(m->partials);
    const int grid = tile_grid(m->ntile);
    static_assert(3 * kTileBlocks <= 4 * 152 * 64, "mass partials fit the scratch");
    const LineView V = row_view(m, ptr<double>(m->wgt));
    if (c_dtype == BCHAR_C_F32)
        k_spmv<float><<<grid, kTileThreads, kTileSmem, m->stream>>>(V, ptr<double>(m->volphi), static_cast<const float *>(c_in),
                                                            static_cast<float *>(c_out), part);
    else
        k_spmv<double><<<grid, kTileThreads, kTileSmem, m->stream>>>(V, ptr<double>(m->volphi),
                                                             static_cast<const double *>(c_in),
                                                             static_cast<double *>(c_out), part);
    k_mass_final<<<1, 1024, 0, m->stream>>>(part, grid, ptr<DevInfo>(m->dinfo));
    m->launches += 2;
}

}  // namespace bchar
