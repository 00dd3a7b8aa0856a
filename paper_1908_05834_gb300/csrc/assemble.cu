// The initial weights V_{K,M} (Sec 3.1, eq. fracMaterial, eq. ball_int):
//
//   V_{K,M} = sum_s m_K * (sum_{m in M} w_{s,m}) / (sum_{all M', m} w_{s,m}),
//   w_{s,m} = rho_M phi_M |B_hat_{K,s} cap B_{M,m}|,  m_K = |K|_phi / n_K,
//
// (the mass of a tracked ball, rho_K phi_hat |B_hat| = rho_K phi_K |B| by
// eq. expPhiB).  One warp builds one row K: lane s owns tracked ball s (at most
// 32 per cell), finds the box of cells its ball can touch (every residing ball
// is inside its cell, so cells outside C_hat +- (r_hat + r_max) cannot) and
// sums its denominator; then the lanes sweep the union box of the cell, one
// residing cell M per lane, and the non-zero V_{K,M} (>= drop_tol |K|_phi)
// are compacted into the row with a warp ballot, in increasing column order.
// Rows are written to a slab of row_cap entries per row; a row with more
// entries records its length only, and a second pass over those rows alone
// writes them, at their exact length, to a spill area (offsets from a scan),
// so memory follows the number of non-zeros rather than the widest row.
// A tracked ball that meets no residing ball gives its whole mass to the cell
// holding its centre.
//
// Distances are formed relative to the tracked ball's own cell: the offset of
// a residing cell's corner is an FP64 difference of node coordinates, the rest
// is in the tracking precision, so FP32 keeps its relative precision at the
// scale of a ball.
#include <math.h>

#include "device.cuh"

namespace bchar {

// Circular segment of height s (sagitta) in a circle of radius r:
// r^2/2 (phi - sin phi), phi the central angle, with phi - sin phi from its
// Taylor series for small phi (no cancellation for thin segments).
template <class real> __device__ __forceinline__ real segment(real r, real s) {
    real h = sqrt(fmax(s * (real(2) * r - s), real(0)));
    real ph = real(2) * atan2(h, r - s);
    const real small = sizeof(real) == 4 ? real(1.0) : real(0.25);
    real f;
    if (ph < small) {
        real p2 = ph * ph;
        f = ph * p2 / real(6) *
            (real(1) - p2 / real(20) * (real(1) - p2 / real(42) * (real(1) - p2 / real(72) * (real(1) - p2 / real(110)))));
    } else {
        f = ph - sin(ph);
    }
    return real(0.5) * r * r * f;
}

// Area (2D) or volume (3D) of the intersection of two balls of radii r1, r2
// whose centres are d apart: the two segments / caps cut off by the common
// chord / plane, of heights s1 = (r1+r2-d)(d+r2-r1)/(2d) and
// s2 = (r1+r2-d)(d+r1-r2)/(2d).
template <class real> __device__ __forceinline__ real lens(int dim, real d, real r1, real r2) {
    const real pi = real(3.14159265358979323846);
    if (d >= r1 + r2) return real(0);
    real rmin = fmin(r1, r2);
    if (d <= fabs(r1 - r2)) return dim == 2 ? pi * rmin * rmin : real(4) / real(3) * pi * rmin * rmin * rmin;
    real t = r1 + r2 - d;
    real s1 = t * (d + r2 - r1) / (real(2) * d);
    real s2 = t * (d + r1 - r2) / (real(2) * d);
    if (dim == 2) return segment<real>(r1, s1) + segment<real>(r2, s2);
    return pi / real(3) * (s1 * s1 * (real(3) * r1 - s1) + s2 * s2 * (real(3) * r2 - s2));
}

template <class real> struct BallSmem {
    // (tracked ball, residing cell) pairs of one row held in shared memory
    static constexpr int kPairCap = sizeof(real) == 4 ? 512 : 256;
    int c[kMaxBallsPerCell][3];   // tracked cell, per axis
    int lo[kMaxBallsPerCell][3];  // candidate box of cells
    int hi[kMaxBallsPerCell][3];
    real p[kMaxBallsPerCell][3];  // tracked centre relative to the lower corner of its cell
    real rh[kMaxBallsPerCell];
    real den[kMaxBallsPerCell];
    int poff[kMaxBallsPerCell + 1];  // first pair of each ball
    real S[kPairCap];                // pair weights, ball by ball, each ball's box in (z, y, x) order
};

// Sum over the balls of residing cell M (cell coordinates mc) of
// rho_M phi_M |B_hat cap B_{M,m}| for a tracked ball of radius rh at position p
// relative to the corner of cell tc.
template <class real, int DIM>
__device__ __forceinline__ real ball_cell_weight(const MeshView &m, const int tc[3], const real p[3], real rh,
                                                 const int mc[3], int64_t M) {
    int cnt[3];
    unpack_counts(m.cnt[M], cnt);
    const real rM = Real<real>::rad(m, M);
    const real rp = Real<real>::rhophi(m, M);
    real o[3] = {real(0), real(0), real(0)}, wM[3] = {real(0), real(0), real(0)};
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        o[a] = static_cast<real>(m.x[a][mc[a]] - m.x[a][tc[a]]) - p[a];
        wM[a] = Real<real>::w(m, a)[mc[a]];
    }
    const real reach = rh + rM;
    // every residing ball lies inside its cell, so a cell farther than the
    // reach from the tracked centre holds no overlapping ball (the loop below
    // would return exactly 0); the margin keeps the test conservative
    real dist2 = real(0);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const real g = o[a] > real(0) ? o[a] : (o[a] + wM[a] < real(0) ? -(o[a] + wM[a]) : real(0));
        dist2 += g * g;
    }
    const real lim = reach * real(1.001);
    if (dist2 > lim * lim) return real(0);
    real sum = real(0);
    for (int sz = 0; sz < cnt[2]; ++sz) {
        real dz = DIM == 3 ? o[2] + (real(sz) + real(0.5)) * wM[2] / real(cnt[2]) : real(0);
        for (int sy = 0; sy < cnt[1]; ++sy) {
            real dy = o[1] + (real(sy) + real(0.5)) * wM[1] / real(cnt[1]);
            for (int sx = 0; sx < cnt[0]; ++sx) {
                real dx = o[0] + (real(sx) + real(0.5)) * wM[0] / real(cnt[0]);
                real d = sqrt(dx * dx + dy * dy + dz * dz);
                if (d < reach) sum += rp * lens<real>(DIM, d, rh, rM);
            }
        }
    }
    return sum;
}

// Local index of cell mc in the candidate box of ball s ((z, y, x) order).
template <class real>
__device__ __forceinline__ int box_index(const BallSmem<real> &sm, int s, const int mc[3]) {
    const int wx = sm.hi[s][0] - sm.lo[s][0] + 1, wy = sm.hi[s][1] - sm.lo[s][1] + 1;
    return ((mc[2] - sm.lo[s][2]) * wy + (mc[1] - sm.lo[s][1])) * wx + (mc[0] - sm.lo[s][0]);
}

template <class real, int DIM>
__global__ void __launch_bounds__(256, 3) k_assemble(MeshView m, const int32_t *t_cell, const real *t_xi,
                                                  const real *t_rhat, double drop_tol, int row_cap, int win_cap,
                                                  int32_t *slab_col, double *slab_val, int32_t *row_len,
                                                  const int64_t *spill_off, int32_t *spill_col, double *spill_val,
                                                  DevInfo *info) {
    const bool spill = spill_col != nullptr;  // second pass: only the rows wider than the slab
    __shared__ BallSmem<real> sm_all[256 / 32];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    BallSmem<real> &sm = sm_all[wib];
    const int64_t nwarps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
    const real r_max = static_cast<real>(m.r_max);
    for (int64_t K = blockIdx.x * static_cast<int64_t>(blockDim.x >> 5) + wib; K < m.nc; K += nwarps) {
        if (spill && row_len[K] <= row_cap) continue;  // warp-uniform
        const int64_t off = m.ball_off[K];
        const int nK = static_cast<int>(m.ball_off[K + 1] - off);
        if (nK > kMaxBallsPerCell) {  // warp-uniform
            if (lane == 0) {
                row_len[K] = 0;
                atomicOr(&info->err, kErrBallsPerCell);
            }
            continue;
        }
        // 1. each lane s < nK: its tracked ball's cell, centre, radius and box of candidate cells
        int box = 0;
        if (lane < nK) {
            const int64_t b = off + lane;
            int c[3];
            split_cell(m, t_cell[b], c);
            const real rh = t_rhat[b];
            const real reach = rh + r_max;
            real p[3] = {real(0), real(0), real(0)};
            for (int a = 0; a < 3; ++a) {
                sm.c[lane][a] = c[a];
                sm.lo[lane][a] = c[a];
                sm.hi[lane][a] = c[a];
            }
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                const real *w = Real<real>::w(m, a);
                p[a] = t_xi[3 * b + a] * w[c[a]];
                int lo = c[a];
                real rem = reach - p[a];
                while (lo > 0 && rem >= real(0)) {
                    --lo;
                    rem -= w[lo];
                }
                int hi = c[a];
                rem = reach - (w[c[a]] - p[a]);
                while (hi < m.n[a] - 1 && rem >= real(0)) {
                    ++hi;
                    rem -= w[hi];
                }
                sm.lo[lane][a] = lo;
                sm.hi[lane][a] = hi;
                sm.p[lane][a] = p[a];
            }
            sm.p[lane][2] = p[2];
            sm.rh[lane] = rh;
            box = (sm.hi[lane][0] - sm.lo[lane][0] + 1) * (sm.hi[lane][1] - sm.lo[lane][1] + 1) *
                  (sm.hi[lane][2] - sm.lo[lane][2] + 1);
        }
        // 2. pair offsets: exclusive scan of the box sizes over the lanes
        int incl = box;
        for (int d = 1; d < 32; d <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += t;
        }
        const int npairs = __shfl_sync(0xffffffffu, incl, 31);
        if (lane <= nK) sm.poff[lane] = incl - box;  // lane nK holds the total
        __syncwarp();
        const bool table = npairs <= BallSmem<real>::kPairCap;  // warp-uniform
        // 3. every pair's weight once, spread over all lanes; then each
        //    ball's denominator as the sum over its pairs in box order
        if (table) {
            for (int q = lane; q < npairs; q += 32) {
                int s = 0;
                while (s + 1 < nK && sm.poff[s + 1] <= q) ++s;
                const int t = q - sm.poff[s];
                const int wx = sm.hi[s][0] - sm.lo[s][0] + 1, wy = sm.hi[s][1] - sm.lo[s][1] + 1;
                int mc[3] = {sm.lo[s][0] + t % wx, sm.lo[s][1] + (t / wx) % wy, sm.lo[s][2] + t / (wx * wy)};
                sm.S[q] = ball_cell_weight<real, DIM>(m, sm.c[s], sm.p[s], sm.rh[s], mc, flat_cell(m, mc));
            }
            __syncwarp();
            if (lane < nK) {
                real den = real(0);
                for (int q = sm.poff[lane]; q < sm.poff[lane + 1]; ++q) den += sm.S[q];
                sm.den[lane] = den;
                if (den == real(0)) atomicAdd(&info->void_balls, 1);
            }
        } else if (lane < nK) {  // too many pairs for the table: the ball's lane sums its own box
            real den = real(0);
            int mc[3];
            for (mc[2] = sm.lo[lane][2]; mc[2] <= sm.hi[lane][2]; ++mc[2])
                for (mc[1] = sm.lo[lane][1]; mc[1] <= sm.hi[lane][1]; ++mc[1])
                    for (mc[0] = sm.lo[lane][0]; mc[0] <= sm.hi[lane][0]; ++mc[0])
                        den += ball_cell_weight<real, DIM>(m, sm.c[lane], sm.p[lane], sm.rh[lane], mc, flat_cell(m, mc));
            sm.den[lane] = den;
            if (den == real(0)) atomicAdd(&info->void_balls, 1);
        }
        __syncwarp();
        // 4. the union box of the row, one residing cell per lane
        int LO[3], HI[3];
        for (int a = 0; a < 3; ++a) {
            LO[a] = sm.lo[0][a];
            HI[a] = sm.hi[0][a];
            for (int s = 1; s < nK; ++s) {
                LO[a] = min(LO[a], sm.lo[s][a]);
                HI[a] = max(HI[a], sm.hi[s][a]);
            }
        }
        const int wx = HI[0] - LO[0] + 1, wy = HI[1] - LO[1] + 1, wz = HI[2] - LO[2] + 1;
        const int nW = wx * wy * wz;
        if (nW > win_cap) {
            if (lane == 0) {
                row_len[K] = 0;
                atomicOr(&info->err, kErrWindow);
            }
            __syncwarp();
            continue;
        }
        const double vK = m.volphi[K];
        const double mK = vK / nK;
        const double thr = drop_tol * vK;
        int count = 0;
        for (int base = 0; base < nW; base += 32) {
            const int t = base + lane;
            double V = 0.0;
            int64_t M = 0;
            if (t < nW) {
                int mc[3] = {LO[0] + t % wx, LO[1] + (t / wx) % wy, LO[2] + t / (wx * wy)};
                M = flat_cell(m, mc);
                for (int s = 0; s < nK; ++s) {
                    bool in = true;
#pragma unroll
                    for (int a = 0; a < DIM; ++a) in = in && mc[a] >= sm.lo[s][a] && mc[a] <= sm.hi[s][a];
                    if (!in) continue;
                    if (sm.den[s] > real(0)) {
                        const real S = table ? sm.S[sm.poff[s] + box_index(sm, s, mc)]
                                             : ball_cell_weight<real, DIM>(m, sm.c[s], sm.p[s], sm.rh[s], mc, M);
                        V += mK * static_cast<double>(S / sm.den[s]);
                    } else if (mc[0] == sm.c[s][0] && mc[1] == sm.c[s][1] && mc[2] == sm.c[s][2]) {
                        V += mK;
                    }
                }
            }
            const bool keep = t < nW && V > 0.0 && V >= thr;
            const unsigned mask = __ballot_sync(0xffffffffu, keep);
            const int pos = count + __popc(mask & ((1u << lane) - 1u));
            if (keep && spill) {
                spill_col[spill_off[K] + pos] = static_cast<int32_t>(M);
                spill_val[spill_off[K] + pos] = V;
            } else if (keep && pos < row_cap) {
                slab_col[K * row_cap + pos] = static_cast<int32_t>(M);
                slab_val[K * row_cap + pos] = V;
            }
            count += __popc(mask);
        }
        if (lane == 0 && !spill) {
            row_len[K] = count;  // the true length; rows wider than the slab are written by the spill pass
            atomicMax(&info->need_row_cap, count);
            if (count > row_cap) atomicAdd(&info->n_spill_rows, 1);
        }
        __syncwarp();
    }
}

MeshView full_view(bchar_mesh_t m);

template <class real, int DIM>
static void assemble_in(bchar_mesh_t m, const MeshView &mv, int win_cap, int blocks, bool spill) {
    k_assemble<real, DIM><<<blocks, 256, 0, m->stream>>>(
        mv, ptr<int32_t>(m->t_cell), ptr<real>(m->t_xi), ptr<real>(m->t_rhat), m->opt.drop_tol, m->row_cap, win_cap,
        ptr<int32_t>(m->slab_col), ptr<double>(m->slab_val), ptr<int32_t>(m->row_len),
        spill ? ptr<int64_t>(m->spill_off) : nullptr, spill ? ptr<int32_t>(m->spill_col) : nullptr,
        spill ? ptr<double>(m->spill_val) : nullptr, ptr<DevInfo>(m->dinfo));
}

static void assemble_pass(bchar_mesh_t m, bool spill) {
    MeshView mv = full_view(m);
    const int win_cap = m->dim == 2 ? 4096 : 32768;
    const int blocks = blocks_for(m->nc * 32, 256);
    const bool f32 = m->opt.precision == BCHAR_FP32_SPLIT;
    if (m->dim == 2) {
        if (f32)
            assemble_in<float, 2>(m, mv, win_cap, blocks, spill);
        else
            assemble_in<double, 2>(m, mv, win_cap, blocks, spill);
    } else {
        if (f32)
            assemble_in<float, 3>(m, mv, win_cap, blocks, spill);
        else
            assemble_in<double, 3>(m, mv, win_cap, blocks, spill);
    }
    ++m->launches;
}

void launch_assemble(bchar_mesh_t m) { assemble_pass(m, false); }

__global__ void k_spill_counts(int64_t nc, int row_cap, const int32_t *row_len, int32_t *cnt) {
    for (int64_t K = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; K < nc;
         K += static_cast<int64_t>(gridDim.x) * blockDim.x)
        cnt[K] = row_len[K] > row_cap ? row_len[K] : 0;
}

bool launch_assemble_spill(bchar_mesh_t m) {
    if (!ensure(m, m->spill_cnt, sizeof(int32_t) * m->nc) || !ensure(m, m->spill_off, sizeof(int64_t) * (m->nc + 1)))
        return false;
    k_spill_counts<<<blocks_for(m->nc), kThreads, 0, m->stream>>>(m->nc, m->row_cap, ptr<int32_t>(m->row_len),
                                                                  ptr<int32_t>(m->spill_cnt));
    ++m->launches;
    scan_i32_to_i64(m, ptr<int32_t>(m->spill_cnt), ptr<int64_t>(m->spill_off), m->nc);
    int64_t total = 0;
    cudaMemcpyAsync(&total, ptr<int64_t>(m->spill_off) + m->nc, sizeof total, cudaMemcpyDeviceToHost, m->stream);
    if (cudaStreamSynchronize(m->stream) != cudaSuccess) return true;  // the caller reads the error
    const size_t z = total > 0 ? static_cast<size_t>(total) : 1;
    if (!ensure(m, m->spill_col, sizeof(int32_t) * z) || !ensure(m, m->spill_val, sizeof(double) * z)) return false;
    assemble_pass(m, true);
    return true;
}

// Where row K's entries are: the slab, or the spill area when it is wider.
__device__ __forceinline__ int64_t row_src(int64_t K, int row_cap, int32_t len, const int64_t *spill_off) {
    return len > row_cap ? -1 - spill_off[K] : K * row_cap;
}

// ---------------------------------------------------------------- columns

__global__ void k_column_counts(int64_t nc, int row_cap, const int32_t *row_len, const int32_t *slab_col,
                                const int64_t *spill_off, const int32_t *spill_col, int32_t *colcnt) {
    for (int64_t K = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; K < nc;
         K += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int32_t len = row_len[K];
        const int64_t src = row_src(K, row_cap, len, spill_off);
        const int32_t *cols = src >= 0 ? slab_col + src : spill_col + (-1 - src);
        for (int e = 0; e < len; ++e) atomicAdd(&colcnt[cols[e]], 1);
    }
}

void launch_column_counts(bchar_mesh_t m) {
    cudaMemsetAsync(m->colcnt.p, 0, sizeof(int32_t) * m->nc, m->stream);
    const bool sp = m->spill_rows > 0;
    k_column_counts<<<blocks_for(m->nc), kThreads, 0, m->stream>>>(
        m->nc, m->row_cap, ptr<int32_t>(m->row_len), ptr<int32_t>(m->slab_col), sp ? ptr<int64_t>(m->spill_off) : nullptr,
        sp ? ptr<int32_t>(m->spill_col) : nullptr, ptr<int32_t>(m->colcnt));
    ++m->launches;
}

// One block sorts the seed keys (row << 32 | column) so that the result does
// not depend on the order in which the seeding threads ran (bitonic network
// over a power-of-two padded array in shared memory).
__global__ void k_sort_seeds(unsigned long long *seeds, int n) {
    __shared__ unsigned long long s[kMaxSeeds];
    int np = 1;
    while (np < n) np <<= 1;
    for (int i = threadIdx.x; i < np; i += blockDim.x) s[i] = i < n ? seeds[i] : ~0ull;
    __syncthreads();
    for (int k = 2; k <= np; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < np; i += blockDim.x) {
                int l = i ^ j;
                if (l > i) {
                    bool up = (i & k) == 0;
                    unsigned long long a = s[i], b = s[l];
                    if ((a > b) == up) {
                        s[i] = b;
                        s[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) seeds[i] = s[i];
}

// Rows receiving seeds merge them into their (column-sorted) slab entries;
// each seeded column then has exactly one entry.
__global__ void k_insert_seeds(int64_t nc, int row_cap, const unsigned long long *seeds, int nseeds,
                               const double *volphi, int32_t *row_len, int32_t *slab_col, double *slab_val,
                               int32_t *colcnt, DevInfo *info) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nseeds; i += gridDim.x * blockDim.x) {
        const int64_t row = static_cast<int64_t>(seeds[i] >> 32);
        if (i > 0 && static_cast<int64_t>(seeds[i - 1] >> 32) == row) continue;  // first seed of its row does the row
        int e = i;
        int len = row_len[row];  // a row in the spill area (len > row_cap) is refused below
        while (e < nseeds && static_cast<int64_t>(seeds[e] >> 32) == row) {
            const int32_t col = static_cast<int32_t>(seeds[e] & 0xffffffffull);
            if (len >= row_cap) {
                atomicOr(&info->err, kErrSeedCapacity);
                break;
            }
            int pos = len;
            while (pos > 0 && slab_col[row * row_cap + pos - 1] > col) {
                slab_col[row * row_cap + pos] = slab_col[row * row_cap + pos - 1];
                slab_val[row * row_cap + pos] = slab_val[row * row_cap + pos - 1];
                --pos;
            }
            slab_col[row * row_cap + pos] = col;
            slab_val[row * row_cap + pos] = volphi[col];
            colcnt[col] = 1;
            ++len;
            ++e;
        }
        row_len[row] = len;
    }
}

void launch_insert_seeds(bchar_mesh_t m, int nseeds) {
    k_sort_seeds<<<1, 1024, 0, m->stream>>>(ptr<unsigned long long>(m->seeds), nseeds);
    k_insert_seeds<<<blocks_for(nseeds), kThreads, 0, m->stream>>>(
        m->nc, m->row_cap, ptr<unsigned long long>(m->seeds), nseeds, ptr<double>(m->volphi), ptr<int32_t>(m->row_len),
        ptr<int32_t>(m->slab_col), ptr<double>(m->slab_val), ptr<int32_t>(m->colcnt), ptr<DevInfo>(m->dinfo));
    m->launches += 2;
}

// Slab and spill rows -> CSR (row_ptr from the scan of the row lengths).
__global__ void k_compact(int64_t nc, int row_cap, const int32_t *row_len, const int64_t *row_ptr,
                          const int32_t *slab_col, const double *slab_val, const int64_t *spill_off,
                          const int32_t *spill_col, const double *spill_val, int32_t *col, double *val) {
    for (int64_t K = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; K < nc;
         K += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t dst = row_ptr[K];
        const int32_t len = row_len[K];
        const int64_t src = row_src(K, row_cap, len, spill_off);
        const int32_t *cs = src >= 0 ? slab_col + src : spill_col + (-1 - src);
        const double *vs = src >= 0 ? slab_val + src : spill_val + (-1 - src);
        for (int e = 0; e < len; ++e) {
            col[dst + e] = cs[e];
            val[dst + e] = vs[e];
        }
    }
}

void launch_compact(bchar_mesh_t m) {
    const bool sp = m->spill_rows > 0;
    k_compact<<<blocks_for(m->nc), kThreads, 0, m->stream>>>(
        m->nc, m->row_cap, ptr<int32_t>(m->row_len), ptr<int64_t>(m->row_ptr), ptr<int32_t>(m->slab_col),
        ptr<double>(m->slab_val), sp ? ptr<int64_t>(m->spill_off) : nullptr, sp ? ptr<int32_t>(m->spill_col) : nullptr,
        sp ? ptr<double>(m->spill_val) : nullptr, ptr<int32_t>(m->col), ptr<double>(m->a0));
    ++m->launches;
}

}  // namespace bchar
