// Tracking the balls back along the flow (Sec 2 eq. charac; Sec 3).
//
// dp/dt = sign u(p) / phi(p) is integrated by classical RK4 with `substeps`
// equal steps; sign = -1 gives F_{-dt}(p), the foot of the characteristic.
// u is the lowest-order Raviart-Thomas field of the face velocities: in cell
// c, u_a = U_a(lower face) + xi_a (U_a(upper face) - U_a(lower face)), xi_a the
// local coordinate of p in [0, 1] along axis a.
//
// A point is kept as (cell index, local coordinate) per axis rather than as an
// absolute coordinate, so that FP32 tracking keeps FP32 relative precision
// inside the cell (an absolute FP32 coordinate near 1 would only resolve 6e-8,
// about 2.5e-4 of a ball radius on a 1024^2 mesh).  A point that leaves its
// cell is moved to the neighbour ("last node <= p": a point on an interior
// face belongs to the upper cell) and is clamped to the closed box at the
// boundary.  The first stage is evaluated in the ball's own cell, so the
// points on a ball's surface that touch a face use that cell's field.
//
// The tracked radius (Sec 3): r_hat = r_K when phi is constant
// (eq. ball_volChange); otherwise the 2 d points C +- r e_a are tracked too and
// r_hat is their mean distance to the tracked centre (eq. rTrackedBall, with
// the six axis points in 3D).
#include "device.cuh"

namespace bchar {

template <class real>
__device__ __forceinline__ void relocate(const MeshView &m, int a, int &c, real &xi) {
    const real *w = Real<real>::w(m, a);
    const int n = m.n[a];
#pragma unroll 1
    for (int it = 0; it < 64; ++it) {  // one face per stage under the substep rule
        if (xi >= real(1)) {
            if (c >= n - 1) {
                xi = real(1);
                return;
            }
            xi = (xi - real(1)) * w[c] / w[c + 1];
            ++c;
        } else if (xi < real(0)) {
            if (c <= 0) {
                xi = real(0);
                return;
            }
            xi = real(1) + xi * w[c] / w[c - 1];
            --c;
        } else {
            return;
        }
    }
    xi = xi < real(0) ? real(0) : (xi > real(1) ? real(1) : xi);
}

// Arithmetic of one stage in the tracking precision.  FP64 divides by phi and
// by the width (the operations of a plain evaluation of the RT0 field); FP32
// multiplies by 1 / phi and 1 / width, all read from the cell's record (and
// formed from FP64 values).  A substep's moves and its final update use the
// width terms of the point's cell at the start of the substep, loaded once.
template <class real> struct Stage;
template <> struct Stage<double> {
    // r[0..5]: lower/upper face velocity per axis, r[6]: phi; wr[0..2]: widths
    static __device__ __forceinline__ void load(const VelView &v, int64_t k, double r[7]) {
        const double2 *p = reinterpret_cast<const double2 *>(v.recd + kRecordLen * k);
        const double2 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2), d = __ldg(p + 3);
        r[0] = a.x, r[1] = a.y, r[2] = b.x, r[3] = b.y, r[4] = c.x, r[5] = c.y, r[6] = d.x;
    }
    static __device__ __forceinline__ void load_widths(const VelView &v, int64_t k, double wr[3]) {
        const double2 *p = reinterpret_cast<const double2 *>(v.recd + kRecordLen * k);
        const double2 e = __ldg(p + 4), f = __ldg(p + 5);
        wr[0] = e.x, wr[1] = e.y, wr[2] = f.x;
    }
    static __device__ __forceinline__ double per_phi(double u, double phi) { return u / phi; }
    // d over the width held in a record
    static __device__ __forceinline__ double by_width(double wr, double d) { return d / wr; }
};
template <> struct Stage<float> {
    // r[0..5]: lower/upper face velocity per axis, r[6]: 1 / phi; wr[0..2]: inverse widths
    static __device__ __forceinline__ void load(const VelView &v, int64_t k, float r[7]) {
        const float4 *p = reinterpret_cast<const float4 *>(v.recf + kRecordLen * k);
        const float4 a = __ldg(p), b = __ldg(p + 1);
        r[0] = a.x, r[1] = a.y, r[2] = a.z, r[3] = a.w, r[4] = b.x, r[5] = b.y, r[6] = b.z;
    }
    static __device__ __forceinline__ void load_widths(const VelView &v, int64_t k, float wr[3]) {
        const float4 c = __ldg(reinterpret_cast<const float4 *>(v.recf + kRecordLen * k) + 2);
        wr[0] = c.x, wr[1] = c.y, wr[2] = c.z;
    }
    static __device__ __forceinline__ float per_phi(float u, float inv_phi) { return u * inv_phi; }
    // d times the inverse width held in a record (the same value as m.wif)
    static __device__ __forceinline__ float by_width(float wr, float d) { return d * wr; }
};

// Flat index of a cell (32-bit: meshes hold fewer than 2^31 cells).
template <int DIM> __device__ __forceinline__ int64_t cell_of(const MeshView &m, const int (&c)[3]) {
    return DIM == 2 ? c[0] + m.n[0] * c[1] : c[0] + m.n[0] * (c[1] + m.n[1] * c[2]);
}

// f = sign u(p) / phi(p) at the point (c, xi): one record load.  The axis
// count is a template parameter so that every per-point array stays in
// registers (all loops unroll).
template <class real, int DIM>
__device__ __forceinline__ void flow(const MeshView &m, const VelView &v, const int (&c)[3], const real (&xi)[3],
                                     real sign, real (&f)[3]) {
    real r[7];
    Stage<real>::load(v, cell_of<DIM>(m, c), r);
    f[2] = real(0);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const real u = r[2 * a] + xi[a] * (r[2 * a + 1] - r[2 * a]);
        f[a] = sign * Stage<real>::per_phi(u, r[6]);
    }
}

// (c2, x2) = (c, xi) moved by the physical displacement s * k; wb holds the
// width terms of cell c (from its record).
template <class real, int DIM>
__device__ __forceinline__ void moved(const MeshView &m, const int (&c)[3], const real (&xi)[3], real s,
                                      const real (&k)[3], const real (&wb)[3], int (&c2)[3], real (&x2)[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        c2[a] = c[a];
        x2[a] = xi[a];
    }
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        x2[a] = xi[a] + Stage<real>::by_width(wb[a], s * k[a]);
        relocate<real>(m, a, c2[a], x2[a]);
    }
}

template <class real, int DIM, int P>
__device__ void rk4(const MeshView &m, const VelView &v, int (&c)[P][3], real (&xi)[P][3], real h, int substeps,
                    real sign) {
    const real half = real(0.5) * h;
    for (int st = 0; st < substeps; ++st) {
        real acc[P][3], k[P][3], x2[P][3], wb[P][3];
        int c2[P][3];
#pragma unroll
        for (int p = 0; p < P; ++p) {
            flow<real, DIM>(m, v, c[p], xi[p], sign, k[p]);
            Stage<real>::load_widths(v, cell_of<DIM>(m, c[p]), wb[p]);
        }
#pragma unroll
        for (int p = 0; p < P; ++p) {
#pragma unroll
            for (int a = 0; a < 3; ++a) acc[p][a] = k[p][a];
            moved<real, DIM>(m, c[p], xi[p], half, k[p], wb[p], c2[p], x2[p]);
        }
#pragma unroll
        for (int p = 0; p < P; ++p) flow<real, DIM>(m, v, c2[p], x2[p], sign, k[p]);
#pragma unroll
        for (int p = 0; p < P; ++p) {
#pragma unroll
            for (int a = 0; a < 3; ++a) acc[p][a] = acc[p][a] + real(2) * k[p][a];
            moved<real, DIM>(m, c[p], xi[p], half, k[p], wb[p], c2[p], x2[p]);
        }
#pragma unroll
        for (int p = 0; p < P; ++p) flow<real, DIM>(m, v, c2[p], x2[p], sign, k[p]);
#pragma unroll
        for (int p = 0; p < P; ++p) {
#pragma unroll
            for (int a = 0; a < 3; ++a) acc[p][a] = acc[p][a] + real(2) * k[p][a];
            moved<real, DIM>(m, c[p], xi[p], h, k[p], wb[p], c2[p], x2[p]);
        }
#pragma unroll
        for (int p = 0; p < P; ++p) flow<real, DIM>(m, v, c2[p], x2[p], sign, k[p]);
#pragma unroll
        for (int p = 0; p < P; ++p) {
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                const real d = h / real(6) * (acc[p][a] + k[p][a]);
                xi[p][a] = xi[p][a] + Stage<real>::by_width(wb[p][a], d);
                relocate<real>(m, a, c[p][a], xi[p][a]);
            }
        }
    }
}

// Absolute position of (c, xi) in FP64.
template <class real>
__device__ __forceinline__ double position(const MeshView &m, int a, int c, real xi) {
    return m.x[a][c] + static_cast<double>(xi) * m.wd[a][c];
}

// Start of ball b: its cell and the local coordinate of its centre.
template <class real, int DIM>
__device__ __forceinline__ void ball_start(const MeshView &m, int64_t b, int64_t &K, int (&c0)[3], real (&xi0)[3]) {
    K = m.ball_cell[b];
    const int s = static_cast<int>(b - m.ball_off[K]);
    int cnt[3];
    unpack_counts(m.cnt[K], cnt);
    split_cell(m, K, c0);
    const int sub[3] = {s % cnt[0], (s / cnt[0]) % cnt[1], s / (cnt[0] * cnt[1])};
    xi0[0] = xi0[1] = xi0[2] = real(0);
#pragma unroll
    for (int a = 0; a < DIM; ++a) xi0[a] = (real(sub[a]) + real(0.5)) / real(cnt[a]);
}

// phi constant: r_hat = r_K, only the centres move; each thread tracks
// kBallsPerThread balls side by side (the last group repeats its last ball).
constexpr int kBallsPerThread = 4;

template <class real, int DIM>
__global__ void k_track_centres(MeshView m, VelView v, real h, int substeps, int64_t nballs, int32_t *out_cell,
                                real *out_xi, real *out_rhat) {
    const int64_t ngroups = (nballs + kBallsPerThread - 1) / kBallsPerThread;
    for (int64_t g = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; g < ngroups;
         g += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        int c[kBallsPerThread][3];
        real xi[kBallsPerThread][3];
        int64_t Ks[kBallsPerThread];
#pragma unroll
        for (int p = 0; p < kBallsPerThread; ++p) {
            int64_t b = g * kBallsPerThread + p;
            if (b >= nballs) b = nballs - 1;
            ball_start<real, DIM>(m, b, Ks[p], c[p], xi[p]);
        }
        rk4<real, DIM, kBallsPerThread>(m, v, c, xi, h, substeps, real(-1));
#pragma unroll
        for (int p = 0; p < kBallsPerThread; ++p) {
            const int64_t b = g * kBallsPerThread + p;
            if (b >= nballs) break;
            out_cell[b] = static_cast<int32_t>(cell_of<DIM>(m, c[p]));
#pragma unroll
            for (int a = 0; a < 3; ++a) out_xi[3 * b + a] = xi[p][a];
            out_rhat[b] = Real<real>::rad(m, Ks[p]);
        }
    }
}

// phi varying: the centre and the 2 DIM axis points C +- r e_a of one ball
// are tracked by 1 + 2 DIM adjacent lanes, one point per lane (a small
// single-point RK4, so few registers and many warps per SM); the lanes then
// exchange positions by shuffles and the centre's lane forms r_hat, the mean
// distance, summing the axis points in order.
template <class real, int DIM>
__global__ void k_track_balls(MeshView m, VelView v, real h, int substeps, int64_t nballs, int32_t *out_cell,
                              real *out_xi, real *out_rhat) {
    constexpr int G = 1 + 2 * DIM;   // lanes (points) per ball
    constexpr int PER_WARP = 32 / G;  // balls per warp
    const int lane = threadIdx.x & 31;
    const int g = lane / G, p = lane % G;
    const int base = g * G;
    const int64_t warp = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
    const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    const int64_t nw_needed = (nballs + PER_WARP - 1) / PER_WARP;
    for (int64_t w = warp; w < nw_needed; w += nwarps) {  // warp-uniform loop
        int64_t b = w * PER_WARP + g;
        const bool valid = g < PER_WARP && b < nballs;
        if (!valid) b = nballs - 1;  // idle lanes track a copy and write nothing
        int64_t K;
        int c0[3];
        real xi0[3];
        ball_start<real, DIM>(m, b, K, c0, xi0);
        const real r = Real<real>::rad(m, K);
        int c[1][3] = {{c0[0], c0[1], c0[2]}};
        real xi[1][3] = {{xi0[0], xi0[1], xi0[2]}};
        {  // point p > 0: axis (p - 1) / 2, sign - for odd p, + for even p
            const real sg = (p & 1) ? real(-1) : real(1);
#pragma unroll
            for (int q = 0; q < DIM; ++q)
                if (p > 0 && (p - 1) / 2 == q) xi[0][q] = xi0[q] + sg * r / Real<real>::w(m, q)[c0[q]];
        }
        rk4<real, DIM, 1>(m, v, c, xi, h, substeps, real(-1));
        double pos[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int q = 0; q < DIM; ++q) pos[q] = position<real>(m, q, c[0][q], xi[0][q]);
        double cen[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int q = 0; q < DIM; ++q) cen[q] = __shfl_sync(0xffffffffu, pos[q], base < 32 ? base : 0);
        double dist = 0.0;
        {
            double d2 = 0.0;
#pragma unroll
            for (int q = 0; q < DIM; ++q) {
                const double dq = pos[q] - cen[q];
                d2 += dq * dq;
            }
            dist = sqrt(d2);
        }
        double sum = 0.0;
#pragma unroll
        for (int q = 1; q < G; ++q) {
            const int src = base + q < 32 ? base + q : 0;
            sum += __shfl_sync(0xffffffffu, dist, src);
        }
        if (valid && p == 0) {
            out_cell[b] = static_cast<int32_t>(cell_of<DIM>(m, c[0]));
#pragma unroll
            for (int a = 0; a < 3; ++a) out_xi[3 * b + a] = xi[0][a];
            out_rhat[b] = static_cast<real>(sum / (2.0 * DIM));
        }
    }
}

MeshView full_view(bchar_mesh_t m);
VelView vel_view(bchar_mesh_t m);

template <class real>
static void track_in(bchar_mesh_t m, real h, int substeps, int32_t *cell, real *xi, real *rhat) {
    MeshView mv = full_view(m);
    VelView vv = vel_view(m);
    if (m->phi_const) {
        const int64_t groups = (m->nballs + kBallsPerThread - 1) / kBallsPerThread;
        if (m->dim == 2)
            k_track_centres<real, 2><<<blocks_for(groups, 128), 128, 0, m->stream>>>(mv, vv, h, substeps, m->nballs,
                                                                                      cell, xi, rhat);
        else
            k_track_centres<real, 3><<<blocks_for(groups, 128), 128, 0, m->stream>>>(mv, vv, h, substeps, m->nballs,
                                                                                      cell, xi, rhat);
    } else if (m->dim == 2) {  // 6 balls per warp
        const int64_t threads = (m->nballs + 5) / 6 * 32;
        k_track_balls<real, 2><<<blocks_for(threads, 128), 128, 0, m->stream>>>(mv, vv, h, substeps, m->nballs, cell,
                                                                                  xi, rhat);
    } else {  // 4 balls per warp
        const int64_t threads = (m->nballs + 3) / 4 * 32;
        k_track_balls<real, 3><<<blocks_for(threads, 128), 128, 0, m->stream>>>(mv, vv, h, substeps, m->nballs, cell,
                                                                                  xi, rhat);
    }
    ++m->launches;
}

void launch_track(bchar_mesh_t m, double dt, int substeps) {
    if (m->opt.precision == BCHAR_FP32_SPLIT)
        track_in<float>(m, static_cast<float>(dt / substeps), substeps, ptr<int32_t>(m->t_cell), ptr<float>(m->t_xi),
                        ptr<float>(m->t_rhat));
    else
        track_in<double>(m, dt / substeps, substeps, ptr<int32_t>(m->t_cell), ptr<double>(m->t_xi),
                         ptr<double>(m->t_rhat));
}

// Residing cells that no tracked ball reached (Sec 3.2 assumes there are
// none): the centre of such a cell M_j is carried forward over dt (F_{+dt})
// and M_j's whole porous volume is assigned to the cell K_i it lands in,
// a_ij = |M_j|_phi.  Seeds are recorded as (i << 32 | j).
template <class real, int DIM>
__global__ void k_seed_columns(MeshView m, VelView v, real h, int substeps, const int32_t *colcnt,
                               unsigned long long *seeds, DevInfo *info) {
    for (int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; j < m.nc;
         j += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        if (colcnt[j] != 0) continue;
        int c[1][3];
        split_cell(m, j, c[0]);
        real xi[1][3] = {{real(0), real(0), real(0)}};
#pragma unroll
        for (int a = 0; a < DIM; ++a) xi[0][a] = real(0.5);
        rk4<real, DIM, 1>(m, v, c, xi, h, substeps, real(1));
        int slot = atomicAdd(&info->n_seeds, 1);
        if (slot < kMaxSeeds)
            seeds[slot] =
                (static_cast<unsigned long long>(flat_cell(m, c[0])) << 32) | static_cast<unsigned long long>(j);
        else
            atomicOr(&info->err, kErrSeeds);
    }
}

template <class real, int DIM>
static void seed_in(bchar_mesh_t m, real h, int substeps) {
    k_seed_columns<real, DIM><<<blocks_for(m->nc), kThreads, 0, m->stream>>>(
        full_view(m), vel_view(m), h, substeps, ptr<int32_t>(m->colcnt), ptr<unsigned long long>(m->seeds),
        ptr<DevInfo>(m->dinfo));
}

void launch_seed_columns(bchar_mesh_t m, double dt, int substeps) {
    const bool f32 = m->opt.precision == BCHAR_FP32_SPLIT;
    if (m->dim == 2) {
        if (f32)
            seed_in<float, 2>(m, static_cast<float>(dt / substeps), substeps);
        else
            seed_in<double, 2>(m, dt / substeps, substeps);
    } else {
        if (f32)
            seed_in<float, 3>(m, static_cast<float>(dt / substeps), substeps);
        else
            seed_in<double, 3>(m, dt / substeps, substeps);
    }
    ++m->launches;
}

// Tracked centres as absolute FP64 coordinates (for the parity tests).
template <class real>
__global__ void k_tracked_positions(MeshView m, int64_t nballs, const int32_t *t_cell, const real *t_xi,
                                    const real *t_rhat, double *pos, double *rhat) {
    for (int64_t b = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; b < nballs;
         b += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        int c[3];
        split_cell(m, t_cell[b], c);
        for (int a = 0; a < 3; ++a) pos[3 * b + a] = a < m.dim ? position<real>(m, a, c[a], t_xi[3 * b + a]) : 0.0;
        rhat[b] = static_cast<double>(t_rhat[b]);
    }
}

void launch_export_tracked(bchar_mesh_t m, double *pos, double *rhat) {
    MeshView mv = full_view(m);
    if (m->opt.precision == BCHAR_FP32_SPLIT)
        k_tracked_positions<float><<<blocks_for(m->nballs), kThreads, 0, m->stream>>>(
            mv, m->nballs, ptr<int32_t>(m->t_cell), ptr<float>(m->t_xi), ptr<float>(m->t_rhat), pos, rhat);
    else
        k_tracked_positions<double><<<blocks_for(m->nballs), kThreads, 0, m->stream>>>(
            mv, m->nballs, ptr<int32_t>(m->t_cell), ptr<double>(m->t_xi), ptr<double>(m->t_rhat), pos, rhat);
    ++m->launches;
}

}  // namespace bchar
