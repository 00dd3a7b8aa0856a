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

__device__ __forceinline__ int64_t face_idx(const MeshView &m, int a, const int c[3], int f) {
    int e[3] = {c[0], c[1], c[2]};
    int64_t len[3] = {m.n[0], m.n[1], m.n[2]};
    e[a] = f;
    len[a] += 1;
    return e[0] + len[0] * (e[1] + len[1] * static_cast<int64_t>(e[2]));
}

template <class real>
__device__ __forceinline__ void flow(const MeshView &m, const VelView &v, const int c[3], const real xi[3],
                                     real sign, real f[3]) {
    const real phi = Real<real>::phi(m, flat_cell(m, c));
    f[0] = f[1] = f[2] = real(0);
    for (int a = 0; a < m.dim; ++a) {
        const real *U = Real<real>::u(v, a);
        real lo = U[face_idx(m, a, c, c[a])];
        real hi = U[face_idx(m, a, c, c[a] + 1)];
        real u = lo + xi[a] * (hi - lo);
        f[a] = sign * u / phi;
    }
}

// (c2, x2) = (c, xi) moved by the physical displacement s * k.
template <class real>
__device__ __forceinline__ void moved(const MeshView &m, const int c[3], const real xi[3], real s, const real k[3],
                                      int c2[3], real x2[3]) {
    c2[0] = c[0], c2[1] = c[1], c2[2] = c[2];
    x2[0] = xi[0], x2[1] = xi[1], x2[2] = xi[2];
    for (int a = 0; a < m.dim; ++a) {
        x2[a] = xi[a] + (s * k[a]) / Real<real>::w(m, a)[c[a]];
        relocate<real>(m, a, c2[a], x2[a]);
    }
}

template <class real>
__device__ void rk4(const MeshView &m, const VelView &v, int c[3], real xi[3], real h, int substeps, real sign) {
    for (int st = 0; st < substeps; ++st) {
        real k1[3], k2[3], k3[3], k4[3];
        int c2[3];
        real x2[3];
        flow<real>(m, v, c, xi, sign, k1);
        moved<real>(m, c, xi, real(0.5) * h, k1, c2, x2);
        flow<real>(m, v, c2, x2, sign, k2);
        moved<real>(m, c, xi, real(0.5) * h, k2, c2, x2);
        flow<real>(m, v, c2, x2, sign, k3);
        moved<real>(m, c, xi, h, k3, c2, x2);
        flow<real>(m, v, c2, x2, sign, k4);
        for (int a = 0; a < m.dim; ++a) {
            real d = h / real(6) * (k1[a] + real(2) * k2[a] + real(2) * k3[a] + k4[a]);
            xi[a] = xi[a] + d / Real<real>::w(m, a)[c[a]];
            relocate<real>(m, a, c[a], xi[a]);
        }
    }
}

// Absolute position of (c, xi) in FP64.
template <class real>
__device__ __forceinline__ double position(const MeshView &m, int a, int c, real xi) {
    return m.x[a][c] + static_cast<double>(xi) * m.wd[a][c];
}

template <class real>
__global__ void k_track(MeshView m, VelView v, real h, int substeps, int phi_const, int64_t nballs,
                        int32_t *out_cell, real *out_xi, real *out_rhat) {
    for (int64_t b = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; b < nballs;
         b += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t K = m.ball_cell[b];
        const int s = static_cast<int>(b - m.ball_off[K]);
        int cnt[3], c0[3];
        unpack_counts(m.cnt[K], cnt);
        split_cell(m, K, c0);
        const int sub[3] = {s % cnt[0], (s / cnt[0]) % cnt[1], s / (cnt[0] * cnt[1])};
        real xi0[3] = {real(0), real(0), real(0)};
        for (int a = 0; a < m.dim; ++a) xi0[a] = (real(sub[a]) + real(0.5)) / real(cnt[a]);
        int c[3] = {c0[0], c0[1], c0[2]};
        real xi[3] = {xi0[0], xi0[1], xi0[2]};
        rk4<real>(m, v, c, xi, h, substeps, real(-1));
        out_cell[b] = static_cast<int32_t>(flat_cell(m, c));
        for (int a = 0; a < 3; ++a) out_xi[3 * b + a] = xi[a];
        const real r = Real<real>::rad(m, K);
        if (phi_const) {
            out_rhat[b] = r;
            continue;
        }
        double sum = 0.0;
        for (int a = 0; a < m.dim; ++a) {
            for (int sg = -1; sg <= 1; sg += 2) {
                int cc[3] = {c0[0], c0[1], c0[2]};
                real xx[3] = {xi0[0], xi0[1], xi0[2]};
                xx[a] = xi0[a] + real(sg) * r / Real<real>::w(m, a)[c0[a]];
                rk4<real>(m, v, cc, xx, h, substeps, real(-1));
                double d2 = 0.0;
                for (int q = 0; q < m.dim; ++q) {
                    double dq = position<real>(m, q, cc[q], xx[q]) - position<real>(m, q, c[q], xi[q]);
                    d2 += dq * dq;
                }
                sum += sqrt(d2);
            }
        }
        out_rhat[b] = static_cast<real>(sum / (2.0 * m.dim));
    }
}

MeshView full_view(bchar_mesh_t m);
VelView vel_view(bchar_mesh_t m);

void launch_track(bchar_mesh_t m, double dt, int substeps) {
    MeshView mv = full_view(m);
    VelView vv = vel_view(m);
    const int blocks = blocks_for(m->nballs, 128);
    if (m->opt.precision == BCHAR_FP32_SPLIT)
        k_track<float><<<blocks, 128, 0, m->stream>>>(mv, vv, static_cast<float>(dt / substeps), substeps,
                                                      m->phi_const, m->nballs, ptr<int32_t>(m->t_cell),
                                                      ptr<float>(m->t_xi), ptr<float>(m->t_rhat));
    else
        k_track<double><<<blocks, 128, 0, m->stream>>>(mv, vv, dt / substeps, substeps, m->phi_const, m->nballs,
                                                       ptr<int32_t>(m->t_cell), ptr<double>(m->t_xi),
                                                       ptr<double>(m->t_rhat));
    ++m->launches;
}

// Residing cells that no tracked ball reached (Sec 3.2 assumes there are
// none): the centre of such a cell M_j is carried forward over dt (F_{+dt})
// and M_j's whole porous volume is assigned to the cell K_i it lands in,
// a_ij = |M_j|_phi.  Seeds are recorded as (i << 32 | j).
template <class real>
__global__ void k_seed_columns(MeshView m, VelView v, real h, int substeps, const int32_t *colcnt,
                               unsigned long long *seeds, DevInfo *info) {
    for (int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; j < m.nc;
         j += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        if (colcnt[j] != 0) continue;
        int c[3];
        split_cell(m, j, c);
        real xi[3] = {real(0), real(0), real(0)};
        for (int a = 0; a < m.dim; ++a) xi[a] = real(0.5);
        rk4<real>(m, v, c, xi, h, substeps, real(1));
        int slot = atomicAdd(&info->n_seeds, 1);
        if (slot < kMaxSeeds)
            seeds[slot] = (static_cast<unsigned long long>(flat_cell(m, c)) << 32) | static_cast<unsigned long long>(j);
        else
            atomicOr(&info->err, kErrSeeds);
    }
}

void launch_seed_columns(bchar_mesh_t m, double dt, int substeps) {
    MeshView mv = full_view(m);
    VelView vv = vel_view(m);
    if (m->opt.precision == BCHAR_FP32_SPLIT)
        k_seed_columns<float><<<blocks_for(m->nc), kThreads, 0, m->stream>>>(
            mv, vv, static_cast<float>(dt / substeps), substeps, ptr<int32_t>(m->colcnt),
            ptr<unsigned long long>(m->seeds), ptr<DevInfo>(m->dinfo));
    else
        k_seed_columns<double><<<blocks_for(m->nc), kThreads, 0, m->stream>>>(
            mv, vv, dt / substeps, substeps, ptr<int32_t>(m->colcnt), ptr<unsigned long long>(m->seeds),
            ptr<DevInfo>(m->dinfo));
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
