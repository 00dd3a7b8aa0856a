// The C ABI of libbchar (include/bchar.h): argument checks, device memory
// owned by the handle, and the order of the kernels of one B-char step.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "amg.cuh"
#include "internal.cuh"

using namespace bchar;

namespace bchar {

bool ensure(bchar_mesh_t m, Buf &b, size_t bytes) {
    if (b.p && b.bytes >= bytes) return true;
    if (b.p) {
        cudaStreamSynchronize(m->stream);  // the old buffer may still be read by queued work
        release(b);
    }
    const size_t want = bytes < 256 ? 256 : bytes;
    if (cudaMalloc(&b.p, want) != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        char msg[128];
        snprintf(msg, sizeof msg, "device allocation of %zu bytes failed", want);
        m->err = msg;
        return false;
    }
    b.bytes = want;
    b.acct = &m->dev_bytes;
    m->dev_bytes += static_cast<int64_t>(want);
    if (m->dev_bytes > m->dev_bytes_peak) m->dev_bytes_peak = m->dev_bytes;
    return true;
}

void release(Buf &b) {
    if (b.p) cudaFree(b.p);
    if (b.p && b.acct) *b.acct -= static_cast<int64_t>(b.bytes);
    b.p = nullptr;
    b.bytes = 0;
    b.acct = nullptr;
}

MeshView full_view(bchar_mesh_t m) {
    MeshView v{};
    v.dim = m->dim;
    for (int a = 0; a < 3; ++a) {
        v.n[a] = static_cast<int>(m->n[a]);
        v.x[a] = ptr<double>(m->x[a]);
        v.wd[a] = ptr<double>(m->wd[a]);
        v.wf[a] = ptr<float>(m->wf[a]);
        v.wif[a] = ptr<float>(m->wif[a]);
    }
    v.nc = m->nc;
    v.phi = ptr<double>(m->phi);
    v.phif = ptr<float>(m->phif);
    v.volphi = ptr<double>(m->volphi);
    v.rad = ptr<double>(m->rad);
    v.radf = ptr<float>(m->radf);
    v.rhophi = ptr<double>(m->rhophi);
    v.rhophif = ptr<float>(m->rhophif);
    v.cnt = ptr<int32_t>(m->cnt);
    v.ball_off = ptr<int64_t>(m->ball_off);
    v.ball_cell = ptr<int32_t>(m->ball_cell);
    v.r_max = m->r_max;
    return v;
}

VelView vel_view(bchar_mesh_t m) {
    VelView v{};
    for (int a = 0; a < m->dim; ++a) {
        v.u[a] = ptr<double>(m->u[a]);
        v.uf[a] = ptr<float>(m->uf[a]);
    }
    v.recd = ptr<double>(m->rec);
    v.recf = ptr<float>(m->rec);
    return v;
}

static double bits_to_double(unsigned long long b) {
    double d;
    memcpy(&d, &b, sizeof d);
    return d;
}

}  // namespace bchar

namespace {

bchar_status fail(bchar_mesh_t m, bchar_status s, const char *msg) {
    if (m) m->err = msg;
    return s;
}

bchar_status cuda_check(bchar_mesh_t m) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        m->err = std::string("CUDA: ") + cudaGetErrorString(e);
        return BCHAR_ERR_CUDA;
    }
    return BCHAR_OK;
}

DevInfo *host_info(bchar_mesh_t m) { return static_cast<DevInfo *>(m->info_host.p); }

bchar_status read_info(bchar_mesh_t m) {
    cudaMemcpyAsync(m->info_host.p, m->dinfo.p, sizeof(DevInfo), cudaMemcpyDeviceToHost, m->stream);
    if (cudaStreamSynchronize(m->stream) != cudaSuccess) return cuda_check(m);
    return cuda_check(m);
}

bool options_valid(const bchar_options &o) {
    return o.balls_per_axis >= 1 && o.balls_per_axis <= 8 && o.n_scale >= 0 && o.n_scale <= 100000 &&
           (o.precision == BCHAR_FP64 || o.precision == BCHAR_FP32_SPLIT) && o.substeps >= 0 && o.cfl > 0.0 &&
           o.drop_tol >= 0.0 && o.drop_tol < 1.0 && o.penalty > 0.0 && o.qp_tol > 0.0 && o.qp_max_iter >= 0 &&
           o.qp_max_refine >= 0 && o.div_tol > 0.0 && (o.qp_precond == 0 || o.qp_precond == 1) &&
           (o.qp_warm_start == 0 || o.qp_warm_start == 1) && o.slab_width >= 0 && o.slab_width <= 4096;
}

}  // namespace

extern "C" {

void bchar_default_options(bchar_options *o) {
    if (!o) return;
    o->balls_per_axis = 2;
    o->n_scale = 10;
    o->precision = BCHAR_FP64;
    o->substeps = 0;
    o->cfl = 0.5;
    o->drop_tol = 1e-12;
    o->penalty = 1e-7;
    o->qp_tol = 1e-9;
    o->qp_max_iter = 200000;
    o->qp_max_refine = 300;
    o->div_tol = 1e-9;
    o->qp_precond = 1;
    o->qp_warm_start = 1;
    o->slab_width = 0;
}

const char *bchar_status_string(bchar_status s) {
    switch (s) {
    case BCHAR_OK: return "ok";
    case BCHAR_ERR_INVALID_ARG: return "invalid argument";
    case BCHAR_ERR_OUT_OF_MEMORY: return "out of device memory";
    case BCHAR_ERR_CUDA: return "CUDA error";
    case BCHAR_ERR_BOUNDARY_FLUX: return "velocity has a normal component on the boundary";
    case BCHAR_ERR_DIVERGENCE: return "velocity is not divergence free";
    case BCHAR_ERR_NONFINITE: return "non-finite input";
    case BCHAR_ERR_NO_VELOCITY: return "no velocity set";
    case BCHAR_ERR_CAPACITY: return "internal capacity exceeded";
    }
    return "unknown status";
}

const char *bchar_last_error(bchar_mesh_t m) { return m ? m->err.c_str() : ""; }

int64_t bchar_cell_count(bchar_mesh_t m) { return m ? m->nc : 0; }
int64_t bchar_ball_count(bchar_mesh_t m) { return m ? m->nballs : 0; }

void bchar_destroy(bchar_mesh_t m) {
    if (!m) return;
    cudaStreamSynchronize(m->stream);
    Buf *all[] = {&m->phi, &m->phif, &m->volphi, &m->rad, &m->radf, &m->rhophi, &m->rhophif, &m->cnt,
                  &m->ball_off, &m->ball_cell, &m->t_cell, &m->t_xi, &m->t_rhat, &m->slab_col, &m->slab_val,
                  &m->row_len, &m->colcnt, &m->colfill, &m->seeds, &m->seed_row_cnt, &m->row_ptr, &m->col_ptr,
                  &m->col, &m->a0, &m->aN, &m->afin, &m->wgt, &m->csc_row, &m->csc_src, &m->R, &m->C, &m->bloc, &m->tile_r, &m->tile_c, &m->uf_parent, &m->uf_label, &m->comp_acc, &m->a2,
                  &m->a2c, &m->diag, &m->qexc, &m->rhs, &m->qx, &m->qy, &m->F, &m->cg_d, &m->cg_r, &m->cg_z, &m->cg_p,
                  &m->cg_q, &m->cg_rp, &m->scan_tmp, &m->partials, &m->dinfo, &m->cg, &m->ip_f, &m->ip_u,
                  &m->ip_zl, &m->ip_zh, &m->ip_D, &m->ip_q, &m->ip_cl, &m->ip_ch, &m->ip_df, &m->ip_du,
                  &m->ip_dzl, &m->ip_dzh, &m->ip_p, &m->ip_n, &m->ip_zp, &m->ip_zn, &m->ip_cp, &m->ip_cn,
                  &m->ip_dp, &m->ip_dn, &m->ip_dzp, &m->ip_dzn};
    for (Buf *b : all) release(*b);
    for (int a = 0; a < 3; ++a) {
        release(m->x[a]);
        release(m->wd[a]);
        release(m->wf[a]);
        release(m->wif[a]);
        release(m->u[a]);
        release(m->uf[a]);
    }
    release(m->rec);
    for (cudaEvent_t e : m->stage_ev)
        if (e) cudaEventDestroy(e);
    if (m->info_host.p) cudaFreeHost(m->info_host.p);
    amg_release(m->amg);
    delete m;
}

bchar_status bchar_create_mesh(int dim, const int64_t *n_cells, const double *const *coords, const double *phi,
                               const bchar_options *opt, void *stream, bchar_mesh_t *out) {
    if (!out) return BCHAR_ERR_INVALID_ARG;
    *out = nullptr;
    if ((dim != 2 && dim != 3) || !n_cells || !coords || !phi) return BCHAR_ERR_INVALID_ARG;
    bchar_options o;
    bchar_default_options(&o);
    if (opt) o = *opt;
    if (!options_valid(o)) return BCHAR_ERR_INVALID_ARG;
    int64_t n[3] = {1, 1, 1}, nc = 1;
    for (int a = 0; a < dim; ++a) {
        if (n_cells[a] < 1 || n_cells[a] > (1 << 30) || !coords[a]) return BCHAR_ERR_INVALID_ARG;
        n[a] = n_cells[a];
        nc *= n[a];
        if (nc > 0x7fffffffLL) return BCHAR_ERR_INVALID_ARG;
    }
    double hmin = INFINITY, sum_vp = 0.0;
    for (int a = 0; a < dim; ++a)
        for (int64_t i = 0; i <= n[a]; ++i) {
            if (!isfinite(coords[a][i])) return BCHAR_ERR_NONFINITE;
            if (i > 0) {
                double w = coords[a][i] - coords[a][i - 1];
                if (!(w > 0.0)) return BCHAR_ERR_INVALID_ARG;
                hmin = w < hmin ? w : hmin;
            }
        }
    bool phi_const = true;
    for (int64_t k = 0; k < nc; ++k) {
        if (!isfinite(phi[k])) return BCHAR_ERR_NONFINITE;
        if (!(phi[k] > 0.0)) return BCHAR_ERR_INVALID_ARG;
        if (phi[k] != phi[0]) phi_const = false;
    }
    double max_vp = 0.0;
    for (int64_t k = 0; k < nc; ++k) {
        int64_t c[3] = {k % n[0], (k / n[0]) % n[1], k / (n[0] * n[1])};
        double v = phi[k];
        for (int a = 0; a < dim; ++a) v *= coords[a][c[a] + 1] - coords[a][c[a]];
        sum_vp += v;
        max_vp = v > max_vp ? v : max_vp;
    }

    bchar_mesh_t m = new bchar_mesh_s();
    if (cudaGetDevice(&m->device) != cudaSuccess) {
        cudaGetLastError();
        delete m;
        return BCHAR_ERR_CUDA;
    }
    m->dim = dim;
    m->nb = o.balls_per_axis;
    for (int a = 0; a < 3; ++a) m->n[a] = n[a];
    m->nc = nc;
    m->opt = o;
    m->stream = static_cast<cudaStream_t>(stream);
    m->phi_const = phi_const;
    m->hmin = hmin;
    m->sum_volphi = sum_vp;
    m->max_volphi = max_vp * (1.0 + 1e-12);  // a bound on the device's |K|_phi (same product, maybe another order)

    bool ok = true;
    for (int a = 0; a < dim; ++a) {
        ok = ok && ensure(m, m->x[a], sizeof(double) * (n[a] + 1)) && ensure(m, m->wd[a], sizeof(double) * n[a]) &&
             ensure(m, m->wf[a], sizeof(float) * n[a]) && ensure(m, m->wif[a], sizeof(float) * n[a]);
    }
    for (int a = dim; a < 3; ++a) {  // unit extent along the missing axis
        ok = ok && ensure(m, m->x[a], sizeof(double) * 2) && ensure(m, m->wd[a], sizeof(double)) &&
             ensure(m, m->wf[a], sizeof(float)) && ensure(m, m->wif[a], sizeof(float));
    }
    ok = ok && ensure(m, m->phi, sizeof(double) * nc) && ensure(m, m->phif, sizeof(float) * nc) &&
         ensure(m, m->volphi, sizeof(double) * nc) && ensure(m, m->rad, sizeof(double) * nc) &&
         ensure(m, m->radf, sizeof(float) * nc) && ensure(m, m->rhophi, sizeof(double) * nc) &&
         ensure(m, m->rhophif, sizeof(float) * nc) && ensure(m, m->cnt, sizeof(int32_t) * nc) &&
         ensure(m, m->ball_off, sizeof(int64_t) * (nc + 1)) && ensure(m, m->colcnt, sizeof(int32_t) * nc) &&
         ensure(m, m->colfill, sizeof(int32_t) * nc) && ensure(m, m->row_len, sizeof(int32_t) * nc) &&
         ensure(m, m->row_ptr, sizeof(int64_t) * (nc + 1)) && ensure(m, m->col_ptr, sizeof(int64_t) * (nc + 1)) &&
         ensure(m, m->R, sizeof(double) * nc) && ensure(m, m->C, sizeof(double) * nc) &&
         ensure(m, m->bloc, sizeof(double) * nc) &&
         ensure(m, m->seeds, sizeof(unsigned long long) * kMaxSeeds) &&
         ensure(m, m->diag, sizeof(double) * 2 * nc) && ensure(m, m->rhs, sizeof(double) * 2 * nc) &&
         ensure(m, m->qexc, sizeof(double) * 2 * nc) &&
         ensure(m, m->qy, sizeof(double) * 2 * nc) && ensure(m, m->F, sizeof(double) * 2 * nc) &&
         ensure(m, m->cg_d, sizeof(double) * 2 * nc) && ensure(m, m->cg_r, sizeof(double) * 2 * nc) &&
         ensure(m, m->cg_z, sizeof(double) * 2 * nc) && ensure(m, m->cg_p, sizeof(double) * 2 * nc) &&
         ensure(m, m->cg_q, sizeof(double) * 2 * nc) && ensure(m, m->cg_rp, sizeof(double) * 2 * nc) && ensure(m, m->partials, sizeof(double) * 4 * 152 * 64) &&
         ensure(m, m->dinfo, sizeof(DevInfo)) && ensure(m, m->cg, sizeof(CgState));
    if (ok && cudaMallocHost(&m->info_host.p, sizeof(DevInfo) + sizeof(CgState)) != cudaSuccess) {
        cudaGetLastError();
        m->info_host.p = nullptr;
        ok = false;
    }
    if (!ok) {
        bchar_destroy(m);
        return BCHAR_ERR_OUT_OF_MEMORY;
    }
    for (int a = 0; a < dim; ++a)
        cudaMemcpyAsync(m->x[a].p, coords[a], sizeof(double) * (n[a] + 1), cudaMemcpyHostToDevice, m->stream);
    const double unit[2] = {0.0, 1.0};
    for (int a = dim; a < 3; ++a) cudaMemcpyAsync(m->x[a].p, unit, sizeof unit, cudaMemcpyHostToDevice, m->stream);
    cudaMemcpyAsync(m->phi.p, phi, sizeof(double) * nc, cudaMemcpyHostToDevice, m->stream);
    cudaMemsetAsync(m->dinfo.p, 0, sizeof(DevInfo), m->stream);
    launch_mesh_setup(m);
    for (int a = dim; a < 3; ++a) {  // widths of the missing axis (launch_mesh_setup covers dim axes)
        const double one = 1.0;
        const float onef = 1.0f;
        cudaMemcpyAsync(m->wd[a].p, &one, sizeof one, cudaMemcpyHostToDevice, m->stream);
        cudaMemcpyAsync(m->wf[a].p, &onef, sizeof onef, cudaMemcpyHostToDevice, m->stream);
        cudaMemcpyAsync(m->wif[a].p, &onef, sizeof onef, cudaMemcpyHostToDevice, m->stream);
    }
    int64_t nballs = 0;
    cudaMemcpyAsync(&nballs, ptr<int64_t>(m->ball_off) + nc, sizeof nballs, cudaMemcpyDeviceToHost, m->stream);
    bchar_status st = read_info(m);
    if (st != BCHAR_OK) {
        bchar_destroy(m);
        return st;
    }
    if (host_info(m)->err & kErrBallsPerCell) {
        bchar_destroy(m);
        return BCHAR_ERR_CAPACITY;
    }
    m->nballs = nballs;
    m->r_max = bits_to_double(host_info(m)->umax_bits);
    const size_t rb = o.precision == BCHAR_FP32_SPLIT ? sizeof(float) : sizeof(double);
    ok = ensure(m, m->ball_cell, sizeof(int32_t) * nballs) && ensure(m, m->t_cell, sizeof(int32_t) * nballs) &&
         ensure(m, m->t_xi, rb * 3 * nballs) && ensure(m, m->t_rhat, rb * nballs);
    m->row_cap = o.slab_width > 0 ? o.slab_width : (dim == 2 ? 24 : 64);
    ok = ok && ensure(m, m->slab_col, sizeof(int32_t) * nc * m->row_cap) &&
         ensure(m, m->slab_val, sizeof(double) * nc * m->row_cap);
    if (!ok) {
        bchar_destroy(m);
        return BCHAR_ERR_OUT_OF_MEMORY;
    }
    launch_ball_cells(m);
    st = read_info(m);
    if (st != BCHAR_OK) {
        bchar_destroy(m);
        return st;
    }
    *out = m;
    return BCHAR_OK;
}

bchar_status bchar_set_velocity(bchar_mesh_t m, const double *const *face_u, int on_device) {
    return bchar_set_velocity_scaled(m, face_u, on_device, 1.0);
}

bchar_status bchar_set_velocity_scaled(bchar_mesh_t m, const double *const *face_u, int on_device, double scale) {
    if (!m) return BCHAR_ERR_INVALID_ARG;
    if (!isfinite(scale)) return fail(m, BCHAR_ERR_INVALID_ARG, "scale must be finite");
    m->err.clear();
    if (!face_u) return fail(m, BCHAR_ERR_INVALID_ARG, "face_u is NULL");
    m->has_velocity = false;
    for (int a = 0; a < m->dim; ++a) {
        if (!face_u[a]) return fail(m, BCHAR_ERR_INVALID_ARG, "a face velocity array is NULL");
        int64_t nf = 1;
        for (int b = 0; b < m->dim; ++b) nf *= m->n[b] + (b == a ? 1 : 0);
        m->nface[a] = nf;
        if (!ensure(m, m->u[a], sizeof(double) * nf) || !ensure(m, m->uf[a], sizeof(float) * nf))
            return BCHAR_ERR_OUT_OF_MEMORY;
        cudaMemcpyAsync(m->u[a].p, face_u[a], sizeof(double) * nf,
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, m->stream);
    }
    if (scale != 1.0) launch_scale_velocity(m, scale);
    cudaMemsetAsync(m->dinfo.p, 0, sizeof(DevInfo), m->stream);
    launch_velocity_check(m);
    bchar_status st = read_info(m);
    if (st != BCHAR_OK) return st;
    const DevInfo *h = host_info(m);
    if (h->nonfinite) return fail(m, BCHAR_ERR_NONFINITE, "non-finite face velocity");
    const double umax = bits_to_double(h->umax_bits);
    const double bflux = bits_to_double(h->bflux_bits);
    const double div = bits_to_double(h->div_bits);
    if (bflux > m->opt.div_tol * umax) {
        char msg[160];
        snprintf(msg, sizeof msg, "max |u.n| on the boundary %.3e exceeds div_tol * max|u| = %.3e", bflux,
                 m->opt.div_tol * umax);
        return fail(m, BCHAR_ERR_BOUNDARY_FLUX, msg);
    }
    if (div > m->opt.div_tol) {
        char msg[160];
        snprintf(msg, sizeof msg, "a cell's net flux is %.3e of its total face flux (div_tol %.1e)", div,
                 m->opt.div_tol);
        return fail(m, BCHAR_ERR_DIVERGENCE, msg);
    }
    m->vmax = bits_to_double(h->vmax_bits);
    const size_t rec_bytes =
        (m->opt.precision == BCHAR_FP32_SPLIT ? sizeof(float) : sizeof(double)) * kRecordLen * m->nc;
    if (!ensure(m, m->rec, rec_bytes)) return BCHAR_ERR_OUT_OF_MEMORY;
    launch_cell_records(m);
    m->has_velocity = true;
    return BCHAR_OK;
}

bchar_status bchar_step(bchar_mesh_t m, double dt, const void *c_in, void *c_out, int c_dtype,
                        bchar_step_info *info) {
    if (!m) return BCHAR_ERR_INVALID_ARG;
    m->err.clear();
    if (!(dt > 0.0) || !isfinite(dt)) return fail(m, BCHAR_ERR_INVALID_ARG, "dt must be finite and > 0");
    if (!c_in || !c_out || c_in == c_out) return fail(m, BCHAR_ERR_INVALID_ARG, "c_in / c_out NULL or aliased");
    if (c_dtype != BCHAR_C_F64 && c_dtype != BCHAR_C_F32) return fail(m, BCHAR_ERR_INVALID_ARG, "bad c_dtype");
    if (!m->has_velocity) return fail(m, BCHAR_ERR_NO_VELOCITY, "bchar_set_velocity first");
    m->launches = 0;
    if (!m->stage_ev[0])
        for (cudaEvent_t &e : m->stage_ev)
            if (cudaEventCreate(&e) != cudaSuccess) return cuda_check(m);
    cudaEvent_t *ev = m->stage_ev;
    cudaEventRecord(ev[0], m->stream);

    // substeps: the smallest s with dt * vmax / s <= cfl * hmin
    int substeps = m->opt.substeps;
    if (substeps <= 0) {
        double s = ceil(dt * m->vmax / (m->opt.cfl * m->hmin));
        if (!(s <= 1e6)) return fail(m, BCHAR_ERR_INVALID_ARG, "dt needs more than 1e6 RK4 substeps");
        substeps = s < 1.0 ? 1 : static_cast<int>(s);
    }
    cudaMemsetAsync(m->dinfo.p, 0, sizeof(DevInfo), m->stream);
    launch_track(m, dt, substeps);
    cudaEventRecord(ev[1], m->stream);

    // initial weights, row by row, into the slab; rows wider than the slab go to the spill area
    DevInfo *h = host_info(m);
    bchar_status st;
    launch_assemble(m);
    if ((st = read_info(m)) != BCHAR_OK) return st;
    m->spill_rows = h->n_spill_rows;
    if (m->spill_rows > 0 && !launch_assemble_spill(m)) return BCHAR_ERR_OUT_OF_MEMORY;
    launch_column_counts(m);
    launch_seed_columns(m, dt, substeps);
    if ((st = read_info(m)) != BCHAR_OK) return st;
    if (h->err) {
        char msg[96];
        snprintf(msg, sizeof msg, "capacity error bits 0x%x during assembly", h->err);
        return fail(m, BCHAR_ERR_CAPACITY, msg);
    }
    const int void_balls = h->void_balls;
    const int nseeds = h->n_seeds;
    if (nseeds > 0) {
        launch_insert_seeds(m, nseeds);
        if ((st = read_info(m)) != BCHAR_OK) return st;
        if (h->err) return fail(m, BCHAR_ERR_CAPACITY, "a seeded row overflowed its slab row");
    }

    cudaEventRecord(ev[2], m->stream);
    // CSR and its column view
    scan_i32_to_i64(m, ptr<int32_t>(m->row_len), ptr<int64_t>(m->row_ptr), m->nc);
    int64_t nnz = 0;
    cudaMemcpyAsync(&nnz, ptr<int64_t>(m->row_ptr) + m->nc, sizeof nnz, cudaMemcpyDeviceToHost, m->stream);
    if (cudaStreamSynchronize(m->stream) != cudaSuccess) return cuda_check(m);
    if (nnz >= 0x7fffffffLL) return fail(m, BCHAR_ERR_CAPACITY, "more than 2^31 - 1 non-zeros");
    m->nnz = nnz;
    const size_t z = nnz > 0 ? static_cast<size_t>(nnz) : 1;
    if (!ensure(m, m->col, sizeof(int32_t) * z) || !ensure(m, m->a0, sizeof(double) * z) ||
        !ensure(m, m->aN, sizeof(double) * z) || !ensure(m, m->afin, sizeof(double) * z) ||
        !ensure(m, m->wgt, sizeof(double) * z) || !ensure(m, m->qx, sizeof(double) * z) ||
        !ensure(m, m->a2, sizeof(double) * z) || !ensure(m, m->a2c, sizeof(double) * z) ||
        !ensure(m, m->csc_row, sizeof(int32_t) * z) || !ensure(m, m->csc_src, sizeof(int32_t) * z))
        return BCHAR_ERR_OUT_OF_MEMORY;
    launch_compact(m);
    launch_transpose(m);
    if (!launch_tiles(m)) return BCHAR_ERR_OUT_OF_MEMORY;
    if (!launch_balance(m)) return BCHAR_ERR_OUT_OF_MEMORY;
    cudaEventRecord(ev[3], m->stream);

    // N alternating scalings, the minimisation, bounds and column fix, update
    launch_scaling(m);
    cudaEventRecord(ev[4], m->stream);
    int cg_iters = 0, ip_iters = 0;
    if (!launch_minimise(m, &cg_iters, &ip_iters)) return BCHAR_ERR_OUT_OF_MEMORY;
    cudaEventRecord(ev[5], m->stream);
    launch_finalise(m);
    cudaEventRecord(ev[6], m->stream);
    launch_update(m, c_in, c_out, c_dtype);
    cudaEventRecord(ev[7], m->stream);
    if ((st = read_info(m)) != BCHAR_OK) return st;
    if (h->err) {
        char msg[96];
        snprintf(msg, sizeof msg, "capacity error bits 0x%x", h->err);
        return fail(m, BCHAR_ERR_CAPACITY, msg);
    }
    float ms_stage[8] = {};
    for (int k = 0; k < 7; ++k) cudaEventElapsedTime(&ms_stage[k], ev[k], ev[k + 1]);
    cudaEventElapsedTime(&ms_stage[7], ev[0], ev[7]);
    m->have_step = true;
    m->substeps = substeps;
    m->dt = dt;
    if (info) {
        memset(info, 0, sizeof *info);
        info->mass_before = h->mass_before;
        info->mass_after = h->mass_after;
        info->mass_after_stored = h->mass_after_stored;
        info->max_rel_row_res = h->max_rel_row_res;
        info->max_rel_col_res = h->max_rel_col_res;
        info->scale_err = h->scale_err;
        info->kkt_rel = h->kkt_l1;
        info->nnz = nnz;
        info->substeps = substeps;
        info->cg_iters = cg_iters;
        info->ip_iters = ip_iters;
        info->qp_converged = m->ip_converged;
        info->void_balls = void_balls;
        info->empty_cols = nseeds;
        info->n_at_bounds = h->n_at_bounds;
        info->kernel_launches = m->launches;
        info->amg_levels = m->amg_levels;
        info->amg_coarsest = static_cast<int32_t>(m->amg_coarsest);
        info->row_cap = m->row_cap;
        info->spill_rows = m->spill_rows;
        info->max_row_len = h->need_row_cap;
        info->unbalanced = h->unbalanced;
        for (int k = 0; k < 8; ++k) info->ms_stage[k] = ms_stage[k];
    }
    return BCHAR_OK;
}

bchar_status bchar_export_matrix(bchar_mesh_t m, int which, int64_t *row_ptr, int32_t *cols, double *vals,
                                 int64_t cap, int64_t *nnz_out) {
    if (!m) return BCHAR_ERR_INVALID_ARG;
    if (!m->have_step || which < 0 || which > 2 || !row_ptr || !cols || !vals)
        return fail(m, BCHAR_ERR_INVALID_ARG, "no step yet or bad arguments");
    if (nnz_out) *nnz_out = m->nnz;
    if (cap < m->nnz) return fail(m, BCHAR_ERR_CAPACITY, "cap < nnz");
    const Buf &src = which == 0 ? m->a0 : (which == 1 ? m->aN : m->afin);
    cudaMemcpyAsync(row_ptr, m->row_ptr.p, sizeof(int64_t) * (m->nc + 1), cudaMemcpyDeviceToHost, m->stream);
    cudaMemcpyAsync(cols, m->col.p, sizeof(int32_t) * m->nnz, cudaMemcpyDeviceToHost, m->stream);
    cudaMemcpyAsync(vals, src.p, sizeof(double) * m->nnz, cudaMemcpyDeviceToHost, m->stream);
    if (cudaStreamSynchronize(m->stream) != cudaSuccess) return cuda_check(m);
    return cuda_check(m);
}

bchar_status bchar_export_tracked(bchar_mesh_t m, double *pos, double *rhat, int64_t *ball_offset, int64_t cap) {
    if (!m) return BCHAR_ERR_INVALID_ARG;
    if (!m->have_step || !pos || !rhat || !ball_offset) return fail(m, BCHAR_ERR_INVALID_ARG, "no step yet");
    if (cap < m->nballs) return fail(m, BCHAR_ERR_CAPACITY, "cap < number of balls");
    Buf dpos, drh;
    if (!ensure(m, dpos, sizeof(double) * 3 * m->nballs) || !ensure(m, drh, sizeof(double) * m->nballs)) {
        release(dpos);
        release(drh);
        return BCHAR_ERR_OUT_OF_MEMORY;
    }
    launch_export_tracked(m, ptr<double>(dpos), ptr<double>(drh));
    cudaMemcpyAsync(pos, dpos.p, sizeof(double) * 3 * m->nballs, cudaMemcpyDeviceToHost, m->stream);
    cudaMemcpyAsync(rhat, drh.p, sizeof(double) * m->nballs, cudaMemcpyDeviceToHost, m->stream);
    cudaMemcpyAsync(ball_offset, m->ball_off.p, sizeof(int64_t) * (m->nc + 1), cudaMemcpyDeviceToHost, m->stream);
    cudaStreamSynchronize(m->stream);
    release(dpos);
    release(drh);
    return cuda_check(m);
}

bchar_status bchar_device_bytes(bchar_mesh_t m, int64_t *now, int64_t *peak) {
    if (!m || (!now && !peak)) return BCHAR_ERR_INVALID_ARG;
    if (now) *now = m->dev_bytes;
    if (peak) *peak = m->dev_bytes_peak;
    return BCHAR_OK;
}

bchar_status bchar_estimate_device_bytes(int dim, const int64_t *n_cells, const double *const *coords,
                                         const bchar_options *opt, int64_t *bytes) {
    if (!bytes || (dim != 2 && dim != 3) || !n_cells || !coords) return BCHAR_ERR_INVALID_ARG;
    *bytes = 0;
    bchar_options o;
    bchar_default_options(&o);
    if (opt) o = *opt;
    if (!options_valid(o)) return BCHAR_ERR_INVALID_ARG;
    int64_t n[3] = {1, 1, 1}, nc = 1;
    for (int a = 0; a < dim; ++a) {
        if (n_cells[a] < 1 || n_cells[a] > (1 << 30) || !coords[a]) return BCHAR_ERR_INVALID_ARG;
        n[a] = n_cells[a];
        nc *= n[a];
        if (nc > 0x7fffffffLL) return BCHAR_ERR_INVALID_ARG;
    }
    // balls: the tight packing of every cell (counted on the host from the widths)
    int64_t nballs = 0;
    for (int64_t k = 0; k < nc; ++k) {
        const int64_t c[3] = {k % n[0], (k / n[0]) % n[1], k / (n[0] * n[1])};
        double w[3] = {0, 0, 0}, wmin = INFINITY;
        for (int a = 0; a < dim; ++a) {
            w[a] = coords[a][c[a] + 1] - coords[a][c[a]];
            if (!(w[a] > 0.0)) return BCHAR_ERR_INVALID_ARG;
            wmin = w[a] < wmin ? w[a] : wmin;
        }
        int64_t cnt = 1;
        for (int a = 0; a < dim; ++a) {
            int64_t na = static_cast<int64_t>(floor(o.balls_per_axis * w[a] / wmin + 1e-9));
            cnt *= na > o.balls_per_axis ? na : o.balls_per_axis;
        }
        nballs += cnt;
    }
    // bytes per cell, per ball and per matrix entry of every buffer a step holds:
    // mesh and row arrays 116, minimisation vectors 2 x 11 x 8, union-find 80,
    // face velocities 12 d, tracking records kRecordLen x precision, row slab
    // 12 row_cap, matching scratch 48, multigrid level 0 144 and coarser levels
    // ~154, interior-point state of the 2 constraint nodes 2 x 10 x 8, spill
    // counts and offsets 12; per entry: CSR and column view 68, multigrid
    // level 0 48 and coarser ~50, interior-point state 12 x 8, spill area at
    // most 12; per ball 8 + 4 (3 + 1) x precision.
    const int row_cap = o.slab_width > 0 ? o.slab_width : (dim == 2 ? 24 : 64);
    const double rec = kRecordLen * (o.precision == BCHAR_FP32_SPLIT ? 4.0 : 8.0);
    const double per_cell = 116 + 176 + 80 + 12.0 * dim + rec + 12.0 * row_cap + 48 + 144 + 154 + 160 + 12;
    const double per_entry = 68 + 48 + 50 + 96 + 12;
    const double per_ball = 8 + 4.0 * (o.precision == BCHAR_FP32_SPLIT ? 4 : 8);
    const double nnz_bound = (dim == 2 ? 9.0 : 27.0) * nc;  // a 3^d neighbourhood per row
    const double fixed = 4.0 * 152 * 64 * 8 + 4096 * 8 + (1 << 20);
    *bytes = static_cast<int64_t>(1.1 * (per_cell * nc + per_entry * nnz_bound + per_ball * nballs + fixed));
    return BCHAR_OK;
}

bchar_status bchar_time_stage(bchar_mesh_t m, int stage, int reps, float *mean_ms) {
    if (!m) return BCHAR_ERR_INVALID_ARG;
    if (!m->have_step || reps < 1 || !mean_ms || stage < 0 || stage > 6 ||
        ((stage == BCHAR_STAGE_SMOOTH || stage == BCHAR_STAGE_VCYCLE) && m->amg_levels == 0))
        return fail(m, BCHAR_ERR_INVALID_ARG, "no step yet or bad arguments");
    Buf st, cin, cout;
    if (!ensure(m, st, sizeof(CgState)) || !ensure(m, cin, sizeof(double) * m->nc) ||
        !ensure(m, cout, sizeof(double) * m->nc)) {
        release(st);
        release(cin);
        release(cout);
        return BCHAR_ERR_OUT_OF_MEMORY;
    }
    cudaMemsetAsync(st.p, 0, sizeof(CgState), m->stream);
    cudaMemsetAsync(cin.p, 0, sizeof(double) * m->nc, m->stream);
    // the final weights are kept in wgt; the slab of the assembly is scratch
    auto once = [&]() {
        switch (stage) {
        case BCHAR_STAGE_CG_MATVEC: launch_cg_matvec_once(m, ptr<CgState>(st)); break;
        case BCHAR_STAGE_UPDATE: launch_update(m, cin.p, cout.p, BCHAR_C_F64); break;
        case BCHAR_STAGE_ASSEMBLE: launch_assemble(m); break;
        case BCHAR_STAGE_SMOOTH: amg_smooth_once(m, m->amg); break;
        case BCHAR_STAGE_VCYCLE:  // on the finest right-hand side left by the last solve; z is scratch after the step
            amg_apply(m, m->amg, nullptr, ptr<double>(m->cg_z), nullptr, true);
            break;
        case BCHAR_STAGE_SCALING: launch_scaling_once(m); break;
        default: launch_track(m, m->dt, m->substeps); break;
        }
    };
    once();  // warm-up
    // The short stages (tens of microseconds) are replayed from a CUDA graph
    // so that the host's launch rate does not bound the measurement; the
    // graph is captured on a private stream and launched on the handle's.
    cudaGraphExec_t exec = nullptr;
    if (stage == BCHAR_STAGE_CG_MATVEC || stage == BCHAR_STAGE_UPDATE || stage == BCHAR_STAGE_SMOOTH ||
        stage == BCHAR_STAGE_SCALING || stage == BCHAR_STAGE_VCYCLE) {
        cudaStream_t user = m->stream, cap = nullptr;
        cudaGraph_t graph = nullptr;
        bool ok = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) == cudaSuccess;
        if (ok) {
            cudaStreamSynchronize(user);
            m->stream = cap;
            ok = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                for (int r = 0; r < reps; ++r) once();
                ok = cudaStreamEndCapture(cap, &graph) == cudaSuccess;
            }
            m->stream = user;
            if (ok) ok = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
            if (graph) cudaGraphDestroy(graph);
            cudaStreamDestroy(cap);
        }
        if (ok) ok = cudaGraphLaunch(exec, m->stream) == cudaSuccess;  // warm-up of the graph
        if (!ok) {
            if (exec) cudaGraphExecDestroy(exec);
            release(st);
            release(cin);
            release(cout);
            cudaGetLastError();
            return fail(m, BCHAR_ERR_CUDA, "stage graph capture failed");
        }
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, m->stream);
    if (exec)
        cudaGraphLaunch(exec, m->stream);
    else
        for (int r = 0; r < reps; ++r) once();
    cudaEventRecord(e1, m->stream);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *mean_ms = ms / reps;
    if (exec) cudaGraphExecDestroy(exec);
    release(st);
    release(cin);
    release(cout);
    return cuda_check(m);
}

}  // extern "C"

namespace bchar {
double total_volphi(bchar_mesh_t m) { return m->sum_volphi; }
}  // namespace bchar
