// Mesh setup (once per mesh) and the per-step velocity checks.
//
// Balls (Sec 3): every cell K holds n_K equal balls of radius
// r_K = min width / (2 nb) (a quarter of the smallest face for nb = 2, Sec 3),
// n_a = max(nb, floor(nb w_a / w_min)) of them along axis a at the centres of
// an equal split, so that a stretched cell is packed as tightly as a cube (the
// remedy Sec 3.2 gives for residing cells that no tracked ball reaches).
// The porous density rho_K solves rho_K sum_s |B_{K,s}|_phi = |K|_phi
// (eq. def:porous.density), so rho_K phi_K = |K|_phi / (n_K |B_K|).
#include <math.h>

#include "device.cuh"

namespace bchar {

__global__ void k_widths(const double *x, double *wd, float *wf, float *wif, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double w = x[i + 1] - x[i];
        wd[i] = w;
        wf[i] = static_cast<float>(w);
        wif[i] = static_cast<float>(1.0 / w);
    }
}

__global__ void k_cells(MeshView m, int nb, double *volphi, double *rad, float *radf, double *rhophi,
                        float *rhophif, float *phif, int32_t *cnt, int32_t *nballs, DevInfo *info) {
    for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < m.nc;
         k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        int c[3];
        split_cell(m, k, c);
        double w[3] = {1.0, 1.0, 1.0};
        double vol = 1.0, wmin = 0.0;
        for (int a = 0; a < m.dim; ++a) {
            w[a] = m.wd[a][c[a]];
            vol *= w[a];
            wmin = (a == 0 || w[a] < wmin) ? w[a] : wmin;
        }
        int ca[3] = {1, 1, 1};
        for (int a = 0; a < m.dim; ++a) {
            int q = static_cast<int>(floor(nb * w[a] / wmin + 1e-9));
            ca[a] = q < nb ? nb : q;
        }
        int nk = ca[0] * ca[1] * ca[2];
        double r = wmin / (2.0 * nb);
        double bvol = m.dim == 2 ? M_PI * r * r : 4.0 / 3.0 * M_PI * r * r * r;
        double vp = m.phi[k] * vol;
        volphi[k] = vp;
        rad[k] = r;
        radf[k] = static_cast<float>(r);
        rhophi[k] = vp / (nk * bvol);
        rhophif[k] = static_cast<float>(vp / (nk * bvol));
        phif[k] = static_cast<float>(m.phi[k]);
        cnt[k] = ca[0] | (ca[1] << 8) | (ca[2] << 16);
        nballs[k] = nk;
        atomic_max_nonneg(&info->umax_bits, r);
        if (nk > kMaxBallsPerCell || ca[0] > 255 || ca[1] > 255 || ca[2] > 255) atomicOr(&info->err, kErrBallsPerCell);
    }
}

__global__ void k_ball_cells(MeshView m, const int64_t *off, int32_t *ball_cell) {
    for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < m.nc;
         k += static_cast<int64_t>(gridDim.x) * blockDim.x)
        for (int64_t b = off[k]; b < off[k + 1]; ++b) ball_cell[b] = static_cast<int32_t>(k);
}

static MeshView partial_view(bchar_mesh_t m) {
    MeshView v{};
    v.dim = m->dim;
    for (int a = 0; a < 3; ++a) {
        v.n[a] = static_cast<int>(m->n[a]);
        v.x[a] = ptr<double>(m->x[a]);
        v.wd[a] = ptr<double>(m->wd[a]);
        v.wf[a] = ptr<float>(m->wf[a]);
    }
    v.nc = m->nc;
    v.phi = ptr<double>(m->phi);
    return v;
}

void launch_mesh_setup(bchar_mesh_t m) {
    for (int a = 0; a < m->dim; ++a) {
        k_widths<<<blocks_for(m->n[a]), kThreads, 0, m->stream>>>(ptr<double>(m->x[a]), ptr<double>(m->wd[a]),
                                                                    ptr<float>(m->wf[a]), ptr<float>(m->wif[a]),
                                                                    static_cast<int>(m->n[a]));
        ++m->launches;
    }
    MeshView v = partial_view(m);
    int32_t *nballs = ptr<int32_t>(m->colcnt);  // scratch, n_c entries
    k_cells<<<blocks_for(m->nc), kThreads, 0, m->stream>>>(
        v, m->nb, ptr<double>(m->volphi), ptr<double>(m->rad), ptr<float>(m->radf), ptr<double>(m->rhophi),
        ptr<float>(m->rhophif), ptr<float>(m->phif), ptr<int32_t>(m->cnt), nballs, ptr<DevInfo>(m->dinfo));
    ++m->launches;
    scan_i32_to_i64(m, nballs, ptr<int64_t>(m->ball_off), m->nc);
}

void launch_ball_cells(bchar_mesh_t m) {
    MeshView v = partial_view(m);
    k_ball_cells<<<blocks_for(m->nc), kThreads, 0, m->stream>>>(v, ptr<int64_t>(m->ball_off),
                                                                ptr<int32_t>(m->ball_cell));
    ++m->launches;
}

// ---------------------------------------------------------------- velocity

__device__ __forceinline__ int64_t face_index(const MeshView &m, int a, const int c[3], int f) {
    int e[3] = {c[0], c[1], c[2]};
    int64_t len[3] = {m.n[0], m.n[1], m.n[2]};
    e[a] = f;
    len[a] += 1;
    return e[0] + len[0] * (e[1] + len[1] * static_cast<int64_t>(e[2]));
}

// Per cell: the largest |u|/phi_K over its faces (for the substep rule), the
// largest |u| and |u.n| on boundary faces (u.n = 0 on the boundary, Sec 1),
// and the net flux relative to the total flux through its faces
// (div u = 0, Sec 2.2).
// The four maxima are kept per thread, reduced per block and written with one
// atomic per block (per-cell atomics on four shared counters serialise).
__global__ void k_velocity_check(MeshView m, VelView v, DevInfo *info) {
    double t_vmax = 0.0, t_umax = 0.0, t_bflux = 0.0, t_div = 0.0;
    for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < m.nc;
         k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        int c[3];
        split_cell(m, k, c);
        double vol = 1.0;
        for (int a = 0; a < m.dim; ++a) vol *= m.wd[a][c[a]];
        double umax = 0.0, net = 0.0, tot = 0.0, bflux = 0.0;
        bool bad = false;
        for (int a = 0; a < m.dim; ++a) {
            double lo = v.u[a][face_index(m, a, c, c[a])];
            double hi = v.u[a][face_index(m, a, c, c[a] + 1)];
            if (!isfinite(lo) || !isfinite(hi)) bad = true;
            double area = vol / m.wd[a][c[a]];
            umax = fmax(umax, fmax(fabs(lo), fabs(hi)));
            net += (hi - lo) * area;
            tot += (fabs(hi) + fabs(lo)) * area;
            if (c[a] == 0) bflux = fmax(bflux, fabs(lo));
            if (c[a] == m.n[a] - 1) bflux = fmax(bflux, fabs(hi));
        }
        if (bad) {
            atomicOr(&info->nonfinite, 1);
            continue;
        }
        t_vmax = fmax(t_vmax, umax / m.phi[k]);
        t_umax = fmax(t_umax, umax);
        t_bflux = fmax(t_bflux, bflux);
        t_div = fmax(t_div, tot > 0.0 ? fabs(net) / tot : 0.0);
    }
    t_vmax = block_max(t_vmax);
    t_umax = block_max(t_umax);
    t_bflux = block_max(t_bflux);
    t_div = block_max(t_div);
    if (threadIdx.x == 0) {
        atomic_max_nonneg(&info->vmax_bits, t_vmax);
        atomic_max_nonneg(&info->umax_bits, t_umax);
        atomic_max_nonneg(&info->bflux_bits, t_bflux);
        atomic_max_nonneg(&info->div_bits, t_div);
    }
}

__global__ void k_to_float(const double *in, float *out, int64_t n) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        out[i] = static_cast<float>(in[i]);
}

__global__ void k_scale(double *v, int64_t n, double scale) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        v[i] *= scale;
}

void launch_scale_velocity(bchar_mesh_t m, double scale) {
    for (int a = 0; a < m->dim; ++a) {
        k_scale<<<blocks_for(m->nface[a]), kThreads, 0, m->stream>>>(ptr<double>(m->u[a]), m->nface[a], scale);
        ++m->launches;
    }
}

// Per-cell tracking records (see VelView): FP64 records hold phi, FP32
// records 1 / phi (formed in FP64), so that a FP32 stage multiplies.
template <class real>
__global__ void k_cell_records(MeshView m, VelView v, real *rec) {
    for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < m.nc;
         k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        int c[3];
        split_cell(m, k, c);
        real r[kRecordLen];
        for (int q = 0; q < kRecordLen; ++q) r[q] = real(0);
        for (int a = 0; a < m.dim; ++a) {
            int e[3] = {c[0], c[1], c[2]};
            int64_t len[3] = {m.n[0], m.n[1], m.n[2]};
            len[a] += 1;
            const int64_t lo = e[0] + len[0] * (e[1] + len[1] * static_cast<int64_t>(e[2]));
            e[a] += 1;
            const int64_t hi = e[0] + len[0] * (e[1] + len[1] * static_cast<int64_t>(e[2]));
            r[2 * a] = Real<real>::u(v, a)[lo];
            r[2 * a + 1] = Real<real>::u(v, a)[hi];
        }
        r[6] = sizeof(real) == 8 ? static_cast<real>(m.phi[k]) : static_cast<real>(1.0 / m.phi[k]);
        for (int a = 0; a < 3; ++a) {  // the cell's widths (FP64) or inverse widths (FP32); 1 for a missing axis
            const double w = a < m.dim ? m.wd[a][c[a]] : 1.0;
            r[8 + a] = sizeof(real) == 8 ? static_cast<real>(w) : static_cast<real>(1.0 / w);
        }
        for (int q = 0; q < kRecordLen; ++q) rec[kRecordLen * k + q] = r[q];
    }
}

MeshView full_view(bchar_mesh_t m);
VelView vel_view(bchar_mesh_t m);

void launch_cell_records(bchar_mesh_t m) {
    MeshView mv = full_view(m);
    VelView vv = vel_view(m);
    if (m->opt.precision == BCHAR_FP32_SPLIT)
        k_cell_records<float><<<blocks_for(m->nc), kThreads, 0, m->stream>>>(mv, vv, ptr<float>(m->rec));
    else
        k_cell_records<double><<<blocks_for(m->nc), kThreads, 0, m->stream>>>(mv, vv, ptr<double>(m->rec));
    ++m->launches;
}

void launch_velocity_check(bchar_mesh_t m) {
    MeshView mv = partial_view(m);
    VelView vv{};
    for (int a = 0; a < m->dim; ++a) {
        vv.u[a] = ptr<double>(m->u[a]);
        k_to_float<<<blocks_for(m->nface[a]), kThreads, 0, m->stream>>>(ptr<double>(m->u[a]), ptr<float>(m->uf[a]),
                                                                           m->nface[a]);
        ++m->launches;
    }
    k_velocity_check<<<blocks_for(m->nc), kThreads, 0, m->stream>>>(mv, vv, ptr<DevInfo>(m->dinfo));
    ++m->launches;
}

}  // namespace bchar
