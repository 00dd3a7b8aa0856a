// FP64 matrix stages of a B-char step:
//   - device-wide scans (row / column pointers),
//   - the column view of A (deterministic: columns sorted by row),
//   - N alternating column/row scalings (Sec 3.2, eq. volAdj), kept as
//     diagonal factors, A^(N) = diag(R) A^(0) diag(C),
//   - the mass-conservation minimisation (Sec 3.2, eq. opti_masscons) in the
//     penalised form: the minimiser of 1/2 x.x + 1/2 sum_l (s_l/(eps b_l))^2,
//     s = b - A-hat (1 + x), i.e. x = A-hat^T y with
//     (A-hat A-hat^T + diag((eps b)^2)) y = b - A-hat 1.  A-hat A-hat^T is the
//     bipartite matrix [[D_r, W], [W^T, D_c]], W_ij = a_ij^2, applied through
//     the row and column views of A without forming A-hat; it is solved by
//     Jacobi-preconditioned conjugate gradients with iterative refinement
//     (x accumulated per entry, since y itself can grow very large),
//   - the bounds 0 <= 1 + x <= 2, a final column scaling (global mass to
//     rounding), W_KM = a_KM / |K|_phi and the update c^{n+1} = W c^n
//     (eq. phys-inter-ELLAM) with FP64 accumulation.
// All sums run in a fixed order (no floating-point atomics), so a step is
// bitwise reproducible.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <time.h>

#include "amg.cuh"
#include "device.cuh"

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

// ---------------------------------------------------------------- scaling (eq. volAdj)

__global__ void k_fill(double *v, int64_t n, double val) {
    GRID_STRIDE(i, n) v[i] = val;
}

// a^{n+1/2}: C_j = |M_j|_phi / sum_i R_i a0_ij
__global__ void k_colscale(int64_t nc, const int64_t *col_ptr, const int32_t *csc_row, const int32_t *csc_src,
                           const double *a0, const double *R, const double *volphi, double *C) {
    GRID_STRIDE(j, nc) {
        double s = 0.0;
        for (int64_t p = col_ptr[j]; p < col_ptr[j + 1]; ++p) s += R[csc_row[p]] * a0[csc_src[p]];
        C[j] = volphi[j] / s;
    }
}

// a^{n+1}: R_i = b_i / sum_j a0_ij C_j, b_i the (balanced) local target
__global__ void k_rowscale(int64_t nc, const int64_t *row_ptr, const int32_t *col, const double *a0,
                           const double *C, const double *brow, double *R) {
    GRID_STRIDE(i, nc) {
        double s = 0.0;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) s += a0[e] * C[col[e]];
        R[i] = brow[i] / s;
    }
}

__global__ void k_apply_scaling(int64_t nc, const int64_t *row_ptr, const int32_t *col, const double *a0,
                                const double *R, const double *C, double *aN) {
    GRID_STRIDE(i, nc) {
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) aN[e] = R[i] * a0[e] * C[col[e]];
    }
}

// max_j |sum_i a_ij - |M_j|_phi| / |M_j|_phi
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

void launch_scaling(bchar_mesh_t m) {
    const int64_t nc = m->nc;
    const int bl = blocks_for(nc);
    k_fill<<<bl, kThreads, 0, m->stream>>>(ptr<double>(m->R), nc, 1.0);
    ++m->launches;
    for (int it = 0; it < m->opt.n_scale; ++it) {
        k_colscale<<<bl, kThreads, 0, m->stream>>>(nc, ptr<int64_t>(m->col_ptr), ptr<int32_t>(m->csc_row),
                                                   ptr<int32_t>(m->csc_src), ptr<double>(m->a0), ptr<double>(m->R),
                                                   ptr<double>(m->volphi), ptr<double>(m->C));
        k_rowscale<<<bl, kThreads, 0, m->stream>>>(nc, ptr<int64_t>(m->row_ptr), ptr<int32_t>(m->col),
                                                   ptr<double>(m->a0), ptr<double>(m->C), ptr<double>(m->bloc),
                                                   ptr<double>(m->R));
        m->launches += 2;
    }
    if (m->opt.n_scale == 0) {
        k_fill<<<bl, kThreads, 0, m->stream>>>(ptr<double>(m->C), nc, 1.0);
        ++m->launches;
    }
    k_apply_scaling<<<bl, kThreads, 0, m->stream>>>(nc, ptr<int64_t>(m->row_ptr), ptr<int32_t>(m->col),
                                                    ptr<double>(m->a0), ptr<double>(m->R), ptr<double>(m->C),
                                                    ptr<double>(m->aN));
    DevInfo *di = ptr<DevInfo>(m->dinfo);
    k_col_error<<<bl, kThreads, 0, m->stream>>>(nc, ptr<int64_t>(m->col_ptr), ptr<int32_t>(m->csc_src),
                                                ptr<double>(m->aN), ptr<double>(m->volphi),
                                                reinterpret_cast<unsigned long long *>(&di->scale_err));
    m->launches += 2;
}

// ---------------------------------------------------------------- minimisation

// Node l < n: row l; node l >= n: column l - n.  b_l = |K|_phi resp. |M|_phi,
// w_l = (eps b_l)^2.
__global__ void k_qp_setup(int64_t nc, const int64_t *row_ptr, const int64_t *col_ptr, const int32_t *csc_src,
                           const double *aN, const double *brow, const double *volphi, double eps, double *a2,
                           double *diag, double *exc, double *rhs) {
    GRID_STRIDE(l, 2 * nc) {
        double d = 0.0, s = 0.0;
        if (l < nc) {
            for (int64_t e = row_ptr[l]; e < row_ptr[l + 1]; ++e) {
                const double a = aN[e];
                a2[e] = a * a;
                d += a * a;
                s += a;
            }
        } else {
            const int64_t j = l - nc;
            for (int64_t p = col_ptr[j]; p < col_ptr[j + 1]; ++p) {
                const double a = aN[csc_src[p]];
                d += a * a;
                s += a;
            }
        }
        const double b = l < nc ? brow[l] : volphi[l - nc];
        const double w = (eps * b) * (eps * b);
        diag[l] = d + w;
        exc[l] = w;
        rhs[l] = b - s;
    }
}

__global__ void k_qp_gather_cols(int64_t nnz, const int32_t *csc_src, const double *a2, double *a2c) {
    GRID_STRIDE(p, nnz) a2c[p] = a2[csc_src[p]];
}

// F = r - A-hat x - w y and per-block partial sums of |F|.
__global__ void k_qp_kkt(int64_t nc, const int64_t *row_ptr, const int64_t *col_ptr, const int32_t *csc_src,
                         const double *aN, const double *qx, const double *y, const double *rhs, const double *brow,
                         const double *volphi, double eps, double *F, double *partials) {
    double acc = 0.0;
    GRID_STRIDE(l, 2 * nc) {
        double s = 0.0;
        if (l < nc) {
            for (int64_t e = row_ptr[l]; e < row_ptr[l + 1]; ++e) s += aN[e] * qx[e];
        } else {
            const int64_t j = l - nc;
            for (int64_t p = col_ptr[j]; p < col_ptr[j + 1]; ++p) s += aN[csc_src[p]] * qx[csc_src[p]];
        }
        const double b = l < nc ? brow[l] : volphi[l - nc];
        const double f = rhs[l] - s - (eps * b) * (eps * b) * y[l];
        F[l] = f;
        acc += fabs(f);
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// Preconditioned conjugate gradients on (A-hat A-hat^T + W) d = F.  Every
// kernel returns at once when the solve has converged, so that batches of
// iterations can be queued without reading the state back each time.

__global__ void k_copy(int64_t n, const double *in, double *out, const CgState *st) {
    if (st && st->converged) return;
    GRID_STRIDE(i, n) out[i] = in[i];
}

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

__global__ void k_cg_start(const double *partials, int nparts, double target, CgState *st) {
    double s = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += partials[i];
    s = block_sum(s);
    if (threadIdx.x == 0) {
        st->rz = s;
        st->target = target;
        st->converged = (s == 0.0);
        st->iters = 0;
    }
}

__global__ void k_cg_matvec(int64_t nc, const int64_t *row_ptr, const int32_t *col, const int64_t *col_ptr,
                            const int32_t *csc_row, const double *a2, const double *a2c, const double *diag,
                            const double *p, double *q, double *partials, const CgState *st) {
    dep_enter();
    if (st->converged) return;
    double acc = 0.0;
    GRID_STRIDE(l, 2 * nc) {
        double s = diag[l] * p[l];
        if (l < nc) {
            for (int64_t e = row_ptr[l]; e < row_ptr[l + 1]; ++e) s += a2[e] * p[nc + col[e]];
        } else {
            const int64_t j = l - nc;
            for (int64_t k = col_ptr[j]; k < col_ptr[j + 1]; ++k) s += a2c[k] * p[csc_row[k]];
        }
        q[l] = s;
        acc += p[l] * s;
    }
    acc = block_sum(acc);
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

// d += alpha p, res -= alpha q (the previous residual kept in rp), partial
// sums of |res|
__global__ void k_cg_update(int64_t n2, const double *p, const double *q, double *d, double *res, double *rp,
                            double *partials, const CgState *st) {
    dep_enter();
    if (st->converged) return;
    const double alpha = st->alpha;
    double l1 = 0.0;
    GRID_STRIDE(l, n2) {
        d[l] += alpha * p[l];
        const double r0 = res[l];
        rp[l] = r0;
        const double r = r0 - alpha * q[l];
        res[l] = r;
        l1 += fabs(r);
    }
    l1 = block_sum(l1);
    if (threadIdx.x == 0) partials[blockIdx.x] = l1;
}

// The same, also writing the next V-cycle's right-hand side b = S res in its
// precision T (S: +1 rows, -1 columns), so that the V-cycle needs no pass of
// its own over res.
template <class T>
__global__ void k_cg_update_b(int64_t nc, const double *p, const double *q, double *d, double *res, double *rp,
                              double *partials, T *b, const CgState *st) {
    dep_enter();
    if (st->converged) return;
    const double alpha = st->alpha;
    double l1 = 0.0;
    GRID_STRIDE(l, 2 * nc) {
        d[l] += alpha * p[l];
        const double r0 = res[l];
        rp[l] = r0;
        const double r = r0 - alpha * q[l];
        res[l] = r;
        b[l] = static_cast<T>(l < nc ? r : -r);
        l1 += fabs(r);
    }
    l1 = block_sum(l1);
    if (threadIdx.x == 0) partials[blockIdx.x] = l1;
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

__global__ void k_cg_beta(const double *rz_parts, const double *zp_parts, const double *l1_parts, int nparts,
                          CgState *st) {
    dep_enter();
    if (st->converged) return;
    double rz = 0.0, zp = 0.0, l1 = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        rz += rz_parts[i];
        zp += zp_parts[i];
        l1 += l1_parts[i];
    }
    rz = block_sum(rz);
    zp = block_sum(zp);
    l1 = block_sum(l1);
    if (threadIdx.x == 0) {
        st->beta = st->rz > 0.0 ? fmax(0.0, (rz - zp) / st->rz) : 0.0;
        st->rz = rz;
        st->res_l1 = l1;
        st->iters += 1;
        if (l1 <= st->target || !(st->pq > 0.0) || !(rz > 0.0)) st->converged = 1;
    }
}

__global__ void k_cg_pupdate(int64_t n2, const double *z, double *p, const CgState *st) {
    dep_enter();
    if (st->converged) return;
    const double beta = st->beta;
    GRID_STRIDE(l, n2) p[l] = z[l] + beta * p[l];
}

// Warm start: x_e = a_e (y_i + y_{n+j}) from a dual y kept from the
// previous step (x = A-hat^T y on the new matrix).
__global__ void k_qp_warm(int64_t nc, const int64_t *row_ptr, const int32_t *col, const double *aN, const double *y,
                          double *qx) {
    GRID_STRIDE(i, nc) {
        const double yi = y[i];
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) qx[e] = aN[e] * (yi + y[nc + col[e]]);
    }
}

// x_e += a_e (d_i + d_{n+j}), y += d
__global__ void k_qp_accumulate(int64_t nc, const int64_t *row_ptr, const int32_t *col, const double *aN,
                                const double *d, double *qx, double *y) {
    GRID_STRIDE(l, 2 * nc) {
        if (l < nc)
            for (int64_t e = row_ptr[l]; e < row_ptr[l + 1]; ++e) qx[e] += aN[e] * (d[l] + d[nc + col[e]]);
        y[l] += d[l];
    }
}

static void precondition(bchar_mesh_t m, bool amg, bool fp32, const double *res, double *z, const CgState *st,
                         bool b_ready = false, const double *rp = nullptr, double *pa = nullptr,
                         double *pb = nullptr) {
    if (amg) {
        amg_apply(m, m->amg, res, z, st, fp32, b_ready, rp, pa, pb);
    } else {
        k_jacobi_precond<<<blocks_for(2 * m->nc), kThreads, 0, m->stream>>>(2 * m->nc, ptr<double>(m->diag), res, z, st);
        ++m->launches;
    }
}

#ifndef BCHAR_INNER_REDUCTION
#define BCHAR_INNER_REDUCTION 1e-4
#endif
constexpr double kInnerReduction = BCHAR_INNER_REDUCTION;
constexpr double kFp32Above = 1e-9;  // relative optimality residual above which the V-cycle runs in FP32
// A round of the conjugate gradients ends when its residual has not dropped
// by 1 % for kStallIters iterations; the refinement ends when a round that
// ended so improved the optimality residual by less than a factor of two.
// Below a floor of about 1e-9..1e-11 of sum |K|_phi (near-null components of
// the dual, which the operator hardly sees, accumulate in y) the iterations
// stop making progress, so a tolerance under that floor ends at the floor
// instead of at qp_max_iter; qp_converged reports whether qp_tol was met.
constexpr int kStallIters = 400;
// The warm start (see bchar_options.qp_warm_start) begins from zero every
// kWarmResetSteps steps, so that near-null components cannot pile up in the
// dual over many steps.
constexpr int kWarmResetSteps = 32;
// On 3D meshes the multigrid aggregation is kept for up to kAmgReuseSteps
// steps (only the level operators are rebuilt from the new matrix), and built
// anew earlier when a solve needs more than 1.5 times (+5) the iterations of
// the solve right after the last full build.  3D rows have many entries, the
// matching is a large part of the set-up, and kept aggregates solved in as
// few iterations (128^3 porous: 11.3 vs 11.7).  2D meshes build anew every
// step: their strong row-column pairs move between steps, and kept
// aggregates raised the iterations from 42 to 363 at 1024^2, while the 2D
// matching costs a few ms.
constexpr int kAmgReuseSteps = 8;

// Host wall clock in milliseconds (for the diagnostic trace only).
static double trace_ms() {
    timespec t;
    clock_gettime(CLOCK_MONOTONIC, &t);
    return t.tv_sec * 1e3 + t.tv_nsec * 1e-6;
}

void launch_minimise(bchar_mesh_t m, int *cg_iters, int *refines) {
    const bool trace = getenv("BCHAR_TRACE") != nullptr;  // diagnostic: residual history and phases on stderr
    double t_start = 0.0, t_setup = 0.0, t_graph = 0.0;
    if (trace) {
        cudaStreamSynchronize(m->stream);
        t_start = trace_ms();
    }
    const int64_t nc = m->nc, n2 = 2 * nc, nnz = m->nnz;
    const int bl = blocks_for(n2);
    const double eps = m->opt.penalty;
    cudaStream_t s = m->stream;
    double *a2 = ptr<double>(m->a2), *a2c = ptr<double>(m->a2c), *diag = ptr<double>(m->diag);
    double *rhs = ptr<double>(m->rhs), *qx = ptr<double>(m->qx), *y = ptr<double>(m->qy), *F = ptr<double>(m->F);
    double *d = ptr<double>(m->cg_d), *res = ptr<double>(m->cg_r), *z = ptr<double>(m->cg_z);
    double *p = ptr<double>(m->cg_p), *q = ptr<double>(m->cg_q);
    double *part = ptr<double>(m->partials);
    double *part_l1 = part + 152 * 64;
    double *part_rz = part + 2 * 152 * 64;
    double *part_zp = part + 3 * 152 * 64;
    double *rp = ptr<double>(m->cg_rp);
    DevInfo *di = ptr<DevInfo>(m->dinfo);
    CgState *st = ptr<CgState>(m->cg);
    CgState *host_st = reinterpret_cast<CgState *>(static_cast<char *>(m->info_host.p) + sizeof(DevInfo));

    k_qp_setup<<<bl, kThreads, 0, s>>>(nc, ptr<int64_t>(m->row_ptr), ptr<int64_t>(m->col_ptr), ptr<int32_t>(m->csc_src),
                                      ptr<double>(m->aN), ptr<double>(m->bloc), ptr<double>(m->volphi), eps, a2,
                                      diag, ptr<double>(m->qexc), rhs);
    k_qp_gather_cols<<<blocks_for(nnz), kThreads, 0, s>>>(nnz, ptr<int32_t>(m->csc_src), a2, a2c);
    if (m->opt.qp_warm_start && m->have_dual && m->warm_steps < kWarmResetSteps) {
        ++m->warm_steps;
        k_qp_warm<<<blocks_for(nc), kThreads, 0, s>>>(nc, ptr<int64_t>(m->row_ptr), ptr<int32_t>(m->col),
                                                     ptr<double>(m->aN), y, qx);
        ++m->launches;
    } else {
        cudaMemsetAsync(qx, 0, sizeof(double) * nnz, s);
        cudaMemsetAsync(y, 0, sizeof(double) * n2, s);
        m->warm_steps = 0;
    }
    m->have_dual = false;  // set again below once this solve has finished
    m->launches += 2;
    const bool reuse = m->dim == 3 && m->amg_age >= 0 && m->amg_age < kAmgReuseSteps &&
                       m->last_cg_iters <= 1.5 * m->amg_built_iters + 5;
    const bool amg = m->opt.qp_precond == 1 && amg_build(m, m->amg, reuse);
    m->amg_age = !amg ? -1 : (reuse ? m->amg_age + 1 : 0);
    if (trace) {
        cudaStreamSynchronize(m->stream);
        t_setup = trace_ms();
        fprintf(stderr, "[bchar] set-up and multigrid %.3f ms (%s)\n", t_setup - t_start, reuse ? "kept aggregates" : "built");
    }
    if (trace && amg) {
        fprintf(stderr, "[bchar] multigrid levels:");
        for (int l = 0; l < m->amg.nlev; ++l)
            fprintf(stderr, " %lld/%lld", static_cast<long long>(m->amg.levels[l].n),
                    static_cast<long long>(m->amg.levels[l].nnz));
        fprintf(stderr, "\n");
    }

    int iters = 0, rounds = 0;
    cudaGraphExec_t exec = nullptr;  // the captured batch, reused by the refinement rounds
    bool exec_fp32 = true;
    int graph_launches = 0;
    const double target_abs = m->opt.qp_tol * total_volphi(m);
    double kkt = 0.0, prev_kkt = INFINITY;
    bool stalled = false;
    for (rounds = 0; rounds <= m->opt.qp_max_refine; ++rounds) {
        k_qp_kkt<<<bl, kThreads, 0, s>>>(nc, ptr<int64_t>(m->row_ptr), ptr<int64_t>(m->col_ptr),
                                        ptr<int32_t>(m->csc_src), ptr<double>(m->aN), qx, y, rhs,
                                        ptr<double>(m->bloc), ptr<double>(m->volphi), eps, F, part);
        k_sum_partials<<<1, 1024, 0, s>>>(part, bl, &di->kkt_l1);
        m->launches += 2;
        cudaMemcpyAsync(&kkt, &di->kkt_l1, sizeof(double), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        if (trace) fprintf(stderr, "[bchar] round %d kkt_l1 %.3e (target %.3e)\n", rounds, kkt, target_abs);
        if (kkt <= target_abs || rounds == m->opt.qp_max_refine || iters >= m->opt.qp_max_iter) break;
        if (stalled && kkt > 0.5 * prev_kkt) break;  // the floor: rounds no longer improve
        prev_kkt = kkt;
        // restart the conjugate gradients from the true residual once it has
        // dropped by kInnerReduction: on these ill-conditioned systems short
        // cycles lose less to round-off than one long one
        const double inner = fmax(kInnerReduction * kkt, 0.75 * target_abs);
        cudaMemsetAsync(d, 0, sizeof(double) * n2, s);
        k_copy<<<bl, kThreads, 0, s>>>(n2, F, res, nullptr);
        // FP32 V-cycle while the optimality residual is large, FP64 for the last digits
        const bool fp32 = kkt > kFp32Above * total_volphi(m);
        if (exec && fp32 != exec_fp32) {
            cudaGraphExecDestroy(exec);
            exec = nullptr;
        }
        exec_fp32 = fp32;
        precondition(m, amg, fp32, res, z, nullptr);
        k_dot<<<kRedBlocks, kThreads, 0, s>>>(n2, res, z, part_rz, nullptr);
        k_cg_start<<<1, 1024, 0, s>>>(part_rz, kRedBlocks, inner, st);
        k_copy<<<bl, kThreads, 0, s>>>(n2, z, p, nullptr);
        m->launches += 4;
        // one batch of iterations is captured once into a CUDA graph and
        // replayed until the solve converges (its kernels do nothing then)
        const int batch = amg ? 8 : 32;
        auto enqueue_batch = [&]() {
            for (int k = 0; k < batch; ++k) {
                launch_dep(k_cg_matvec, kRedBlocks, kThreads, s, nc, ptr<int64_t>(m->row_ptr), ptr<int32_t>(m->col),
                                                           ptr<int64_t>(m->col_ptr), ptr<int32_t>(m->csc_row), a2,
                                                           a2c, diag, p, q, part, st);
                launch_dep(k_cg_alpha, 1, 1024, s, part, kRedBlocks, st);
                if (amg) {
                    // the update also writes the V-cycle's right-hand side; the
                    // V-cycle's last kernel also forms the two dot products
                    if (fp32)
                        launch_dep(k_cg_update_b<float>, kRedBlocks, kThreads, s, 
                            nc, p, q, d, res, rp, part_l1, static_cast<float *>(amg_finest_rhs(m->amg, true)), st);
                    else
                        launch_dep(k_cg_update_b<double>, kRedBlocks, kThreads, s, 
                            nc, p, q, d, res, rp, part_l1, static_cast<double *>(amg_finest_rhs(m->amg, false)), st);
                    precondition(m, amg, fp32, res, z, st, true, rp, part_rz, part_zp);
                    m->launches += 3;
                } else {
                    launch_dep(k_cg_update, kRedBlocks, kThreads, s, n2, p, q, d, res, rp, part_l1, st);
                    precondition(m, amg, fp32, res, z, st);
                    launch_dep(k_dot2, kRedBlocks, kThreads, s, n2, z, res, rp, part_rz, part_zp, st);
                    m->launches += 4;
                }
                launch_dep(k_cg_beta, 1, 1024, s, part_rz, part_zp, part_l1, kRedBlocks, st);
                launch_dep(k_cg_pupdate, bl, kThreads, s, n2, z, p, st);
                m->launches += 2;
            }
        };
        if (!exec) {
            const double t0 = trace ? trace_ms() : 0.0;
            const int before = m->launches;
            cudaGraph_t graph = nullptr;
            bool ok = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                enqueue_batch();
                ok = cudaStreamEndCapture(s, &graph) == cudaSuccess && graph;
            }
            if (ok) ok = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
            if (graph) cudaGraphDestroy(graph);
            if (!ok) {  // capture unavailable (for instance, the caller is capturing): plain launches
                cudaGetLastError();
                exec = nullptr;
            }
            graph_launches = m->launches - before;
            m->launches = before;
            if (trace) t_graph += trace_ms() - t0;
        }
        int done = 0;
        double best = INFINITY;
        int best_at = 0;
        stalled = false;
        while (!done) {
            if (exec) {
                cudaGraphLaunch(exec, s);
                m->launches += graph_launches;
            } else {
                enqueue_batch();
            }
            cudaMemcpyAsync(host_st, st, sizeof(CgState), cudaMemcpyDeviceToHost, s);
            cudaStreamSynchronize(s);
            if (trace && (host_st->iters % 512 < batch || host_st->converged))
                fprintf(stderr, "[bchar] round %d iter %d res_l1 %.3e target %.3e\n", rounds, host_st->iters,
                        host_st->res_l1, host_st->target);
            if (host_st->converged || iters + host_st->iters >= m->opt.qp_max_iter) done = 1;
            if (host_st->res_l1 < 0.99 * best) {
                best = host_st->res_l1;
                best_at = host_st->iters;
            } else if (host_st->iters - best_at >= kStallIters) {
                stalled = true;
                done = 1;
            }
        }
        iters += host_st->iters;
        k_qp_accumulate<<<bl, kThreads, 0, s>>>(nc, ptr<int64_t>(m->row_ptr), ptr<int32_t>(m->col),
                                               ptr<double>(m->aN), d, qx, y);
        ++m->launches;
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (trace) {
        cudaStreamSynchronize(m->stream);
        fprintf(stderr, "[bchar] capture+instantiate %.3f ms, total %.3f ms, %d iterations\n", t_graph,
                trace_ms() - t_start, iters);
    }
    m->have_dual = isfinite(kkt);
    if (m->amg_age == 0) m->amg_built_iters = iters;
    m->last_cg_iters = iters;
    *cg_iters = iters;
    *refines = rounds;
    m->amg_levels = amg ? m->amg.nlev : 0;
    m->amg_coarsest = amg ? m->amg.levels[m->amg.nlev - 1].n : 0;
}

void launch_cg_matvec_once(bchar_mesh_t m, CgState *st) {
    const int64_t nc = m->nc;
    k_cg_matvec<<<blocks_for(2 * nc), kThreads, 0, m->stream>>>(
        nc, ptr<int64_t>(m->row_ptr), ptr<int32_t>(m->col), ptr<int64_t>(m->col_ptr), ptr<int32_t>(m->csc_row),
        ptr<double>(m->a2), ptr<double>(m->a2c), ptr<double>(m->diag), ptr<double>(m->cg_p), ptr<double>(m->cg_q),
        ptr<double>(m->partials), st);
}

// ---------------------------------------------------------------- bounds, column fix, W

// a_q = a^(N) clip(1 + x, 0, 2), per row; counts entries outside the bounds.
__global__ void k_clip(int64_t nc, const int64_t *row_ptr, const double *aN, const double *qx, double *aq,
                       DevInfo *info) {
    int clipped = 0;
    GRID_STRIDE(i, nc) {
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            double f = 1.0 + qx[e];
            if (f < 0.0 || f > 2.0) ++clipped;
            f = fmin(fmax(f, 0.0), 2.0);
            aq[e] = aN[e] * f;
        }
    }
    if (clipped) atomicAdd(&info->n_clipped, clipped);
}

// C2_j = |M_j|_phi / sum_i a_q,ij (first half of eq. volAdj).  A column whose
// entries were all clipped to zero keeps its A^(N) entries (dead[j] = 1).
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
    k_clip<<<bl, kThreads, 0, m->stream>>>(nc, ptr<int64_t>(m->row_ptr), ptr<double>(m->aN), ptr<double>(m->qx), aq, di);
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

template <class T>
__global__ void k_spmv(int64_t nc, const int64_t *row_ptr, const int32_t *col, const double *wgt,
                       const double *volphi, const T *c_in, T *c_out, double *partials) {
    double mb = 0.0, ma = 0.0, ms = 0.0;
    GRID_STRIDE(i, nc) {
        double s = 0.0;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) s += wgt[e] * static_cast<double>(c_in[col[e]]);
        const T stored = static_cast<T>(s);
        c_out[i] = stored;
        const double v = volphi[i];
        mb += v * static_cast<double>(c_in[i]);
        ma += v * s;
        ms += v * static_cast<double>(stored);
    }
    mb = block_sum(mb);
    ma = block_sum(ma);
    ms = block_sum(ms);
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
    const int64_t nc = m->nc;
    const int bl = blocks_for(nc);
    double *part = ptr<double>(m->partials);
    if (c_dtype == BCHAR_C_F32)
        k_spmv<float><<<bl, kThreads, 0, m->stream>>>(nc, ptr<int64_t>(m->row_ptr), ptr<int32_t>(m->col),
                                                      ptr<double>(m->wgt), ptr<double>(m->volphi),
                                                      static_cast<const float *>(c_in), static_cast<float *>(c_out), part);
    else
        k_spmv<double><<<bl, kThreads, 0, m->stream>>>(nc, ptr<int64_t>(m->row_ptr), ptr<int32_t>(m->col),
                                                       ptr<double>(m->wgt), ptr<double>(m->volphi),
                                                       static_cast<const double *>(c_in), static_cast<double *>(c_out),
                                                       part);
    k_mass_final<<<1, 1024, 0, m->stream>>>(part, bl, ptr<DevInfo>(m->dinfo));
    m->launches += 2;
}

}  // namespace bchar
