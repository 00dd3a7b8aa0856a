// Internal declarations of libbchar: the state behind a bchar_mesh_t, the
// plain-old-data views handed to kernels, and the launch helpers shared by
// the kernel files.  Nothing here is part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "bchar.h"

namespace bchar {

constexpr int kThreads = 256;     // threads per block of the element-wise kernels
constexpr int kScanChunk = 4096;  // elements per block of the device-wide scan
constexpr int kMaxSeeds = 4096;   // empty columns handled per step
constexpr int kMaxBallsPerCell = 32;

// Device error word bits (BCHAR_ERR_CAPACITY causes).
enum : int {
    kErrBallsPerCell = 1,   // a cell has more than kMaxBallsPerCell balls
    kErrRowCapacity = 2,    // (unused: rows wider than the slab go to the spill area)
    kErrWindow = 4,         // a candidate window is larger than the window limit
    kErrSeeds = 8,          // more than kMaxSeeds empty columns
    kErrSeedCapacity = 16,  // a seeded row overflowed the slab row capacity
    kErrUnion = 32,         // the component search did not settle (never expected)
};

// Read-only mesh data passed by value to kernels.
struct MeshView {
    int dim;
    int n[3];               // cells per axis (n[2] = 1 in 2D)
    int64_t nc;
    const double *x[3];     // node coordinates per axis
    const double *wd[3];    // cell widths per axis, FP64
    const float *wf[3];     // cell widths per axis, FP32
    const float *wif[3];    // 1 / cell width per axis, FP32 (from the FP64 width)
    const double *phi;      // porosity per cell
    const float *phif;
    const double *volphi;   // |K|_phi
    const double *rad;      // ball radius r_K
    const float *radf;
    const double *rhophi;   // rho_K phi_K = |K|_phi / (n_K |B_K|)
    const float *rhophif;
    const int32_t *cnt;     // balls per axis, packed n_x | n_y << 8 | n_z << 16
    const int64_t *ball_off;  // first ball of each cell, n_c + 1
    const int32_t *ball_cell; // cell of each ball
    double r_max;
};

// Face velocities of the current step.
struct VelView {
    const double *u[3];
    const float *uf[3];
    // one record of kRecordLen values per cell: the lower and upper face
    // velocity of each axis (0 for a missing axis), phi (FP64 records) or
    // 1 / phi (FP32 records), 0, then the cell's width per axis (FP64) or
    // inverse width (FP32), 0; a tracking stage reads the first 8 values, the
    // first stage of a substep all 12
    const double *recd;
    const float *recf;
};

// Scalars produced on the device during a step, copied to the host once.
struct DevInfo {
    double mass_before, mass_after, mass_after_stored;
    double max_rel_row_res, max_rel_col_res, scale_err;
    double kkt_l1, f_l1;
    int n_at_bounds;    // entries with 1 + x within 1e-9 of 0 or 2 after the minimisation
    unsigned long long vmax_bits;   // max |u|/phi as the bits of a non-negative double
    unsigned long long umax_bits;   // max |u| over all faces
    unsigned long long bflux_bits;  // max |u.n| over boundary faces
    unsigned long long div_bits;    // max relative net flux of a cell
    int nonfinite;
    int err;            // capacity error bits
    int need_row_cap;   // largest row length seen
    int n_spill_rows;   // rows wider than the slab (written to the spill area)
    int void_balls;
    int n_seeds;
    int unbalanced;
    long long nnz;
};

// Conjugate-gradient scalars.
struct CgState {
    double rz, rz_new, pq, alpha, beta, res_max, target;
    double target_res;  // the solve also needs max_l |res_l| / b_l <= target_res (b_l: the constraint's target)
    int converged;
    int iters;
};

// A growable device buffer.
struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
    int64_t *acct = nullptr;  // the owning handle's byte counter
};

// One level of the multigrid hierarchy: a symmetric CSR operator (off-diagonal
// entries only) with its diagonal and excess, the map to the next coarser
// level, the members of each of its own nodes' aggregates (coarse levels),
// plus work vectors.
struct AmgLevel {
    int64_t n = 0, nnz = 0;
    Buf ptr, col, val, diag, exc, agg, mptr, mlist, x, x2, b, r;  // mptr/mlist: members of each aggregate
    Buf dval, ddiag;                   // the operator divided by the scale (work vectors: x, x2, b, r)
    Buf ddinv;                         // smoother weights omega_i / diag_i of the scaled copy
    const double *diag_ext = nullptr;  // level 0 shares the minimisation's diagonal
    const double *exc_ext = nullptr;   // and its excess (the penalty shift)
};

struct Amg {
    std::vector<AmgLevel> levels;
    int nlev = 0;
    Buf tmp;
    double scale = 1.0;  // the V-cycle's levels hold operator / scale
    int small_from = 0;        // levels small_from..nlev-1 are cycled by one block (nlev: none)
    int large_sweeps = 0;      // Jacobi sweeps of a coarsest level too large for one block
    Buf small_d;               // device descriptors of the small levels
};

}  // namespace bchar

struct bchar_mesh_s {
    int device = 0;               // CUDA device current at create
    int64_t dev_bytes = 0;        // device memory held now (every Buf of the handle)
    int64_t dev_bytes_peak = 0;
    int dim = 0;
    int nb = 2;
    int64_t n[3] = {1, 1, 1};
    int64_t nc = 0;
    int64_t nballs = 0;
    int max_balls = 0;
    bool phi_const = false;
    double hmin = 0.0;
    double r_max = 0.0;
    double sum_volphi = 0.0;
    double max_volphi = 0.0;
    bchar_options opt{};
    cudaStream_t stream = nullptr;
    std::string err;

    // persistent mesh data
    bchar::Buf x[3], wd[3], wf[3], wif[3], phi, phif, volphi, rad, radf, rhophi, rhophif, cnt, ball_off, ball_cell;
    // velocity
    bchar::Buf u[3], uf[3], rec;  // face velocities; per-cell tracking records
    cudaEvent_t stage_ev[8] = {};  // stage boundaries of bchar_step (created on first use)
    int64_t nface[3] = {0, 0, 0};
    bool has_velocity = false;
    double vmax = 0.0;

    // per-step buffers
    bchar::Buf t_cell, t_xi, t_rhat;                 // tracked balls
    bchar::Buf slab_col, slab_val, row_len;          // per-row assembly slab of row_cap entries per row
    bchar::Buf spill_cnt, spill_off, spill_col, spill_val;  // rows wider than the slab, at their exact length
    int row_cap = 0;
    int spill_rows = 0;
    bchar::Buf colcnt, colfill, seeds, seed_row_cnt; // columns, empty-column seeds
    bchar::Buf row_ptr, col_ptr;                     // CSR / CSC pointers
    bchar::Buf col, a0, aN, afin, wgt;               // CSR entries
    bchar::Buf csc_row, csc_src;                     // CSC: row and CSR index of each entry
    bchar::Buf R, C, bloc;                           // scaling factors, balanced row targets
    bchar::Buf tile_r, tile_c;                       // tiles of the row and column views (first line of each)
    int64_t ntile = 0;                               // tiles per view
    bchar::Buf uf_parent, uf_label, comp_acc;        // components of A's pattern
    bchar::Buf a2, a2c, diag, qexc, rhs, qx, qy, F, cg_d, cg_r, cg_z, cg_p, cg_q;  // minimisation
    // interior-point state per entry: 1 + x and its upper slack 2 - (1 + x), the bound multipliers,
    // the normal-equation weight, the reduced right-hand side, the complementarity targets, a direction
    bchar::Buf ip_f, ip_u, ip_zl, ip_zh, ip_D, ip_q, ip_cl, ip_ch, ip_df, ip_du, ip_dzl, ip_dzh;
    // per node (row or column constraint): the violation beyond the quadratic zone, split
    // p - q, their multipliers, complementarity targets and a direction
    bchar::Buf ip_p, ip_n, ip_zp, ip_zn, ip_cp, ip_cn, ip_dp, ip_dn, ip_dzp, ip_dzn;
    bchar::Buf scan_tmp, partials, dinfo, cg, cg_rp; // scratch (cg_rp: previous residual of the flexible CG)
    bchar::Buf info_host;                            // pinned DevInfo
    bchar::Amg amg;                                  // preconditioner of the minimisation
    int64_t nnz = 0;
    int substeps = 1;
    double dt = 0.0;
    int amg_levels = 0;
    int64_t amg_coarsest = 0;
    bool have_step = false;
    int ip_iters = 0;        // interior-point iterations of the last minimisation
    bool ip_converged = false;
    int launches = 0;
};

namespace bchar {

// ---- host helpers (capi.cu) ------------------------------------------------
bool ensure(bchar_mesh_t m, Buf &b, size_t bytes);
void release(Buf &b);
double total_volphi(bchar_mesh_t m);  // sum of |K|_phi over the mesh

template <class T> inline T *ptr(Buf &b) { return static_cast<T *>(b.p); }

constexpr int kRecordLen = 12;  // values per cell in the tracking records

// Blocks of the reduction kernels of the conjugate gradients (grid-stride;
// one partial sum per block).
constexpr int kRedBlocks = 152 * 8;

// Launch of a kernel that begins with dep_enter(): it may be scheduled while
// the previous kernel in the stream drains (programmatic dependent launch).
template <typename... P, typename... A>
inline void launch_dep(void (*kernel)(P...), int grid, int block, cudaStream_t s, A... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, static_cast<P>(args)...);
}

// The same with dynamic shared memory.
template <typename... P, typename... A>
inline void launch_dep_smem(void (*kernel)(P...), int grid, int block, size_t smem, cudaStream_t s, A... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, static_cast<P>(args)...);
}

inline int blocks_for(int64_t n, int threads = kThreads) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 64) b = 152 * 64;  // grid-stride beyond this
    return static_cast<int>(b);
}

// ---- kernels launched from capi.cu ------------------------------------------
// mesh.cu
void launch_mesh_setup(bchar_mesh_t m);
void launch_ball_cells(bchar_mesh_t m);
void launch_velocity_check(bchar_mesh_t m);
void launch_scale_velocity(bchar_mesh_t m, double scale);
void launch_cell_records(bchar_mesh_t m);
// track.cu
void launch_track(bchar_mesh_t m, double dt, int substeps);
void launch_seed_columns(bchar_mesh_t m, double dt, int substeps);
// assemble.cu
void launch_assemble(bchar_mesh_t m);
bool launch_assemble_spill(bchar_mesh_t m);  // rows wider than the slab, into the spill area (false: no memory)
void launch_column_counts(bchar_mesh_t m);
void launch_insert_seeds(bchar_mesh_t m, int nseeds);
void launch_compact(bchar_mesh_t m);
void launch_export_tracked(bchar_mesh_t m, double *pos, double *rhat);
MeshView full_view(bchar_mesh_t m);
VelView vel_view(bchar_mesh_t m);
// sparse.cu
void scan_i32_to_i64(bchar_mesh_t m, const int32_t *in, int64_t *out, int64_t n);  // out has n + 1 entries
void launch_transpose(bchar_mesh_t m);
bool launch_tiles(bchar_mesh_t m);  // tile boundaries of both views (false: out of memory)
bool launch_balance(bchar_mesh_t m);  // components.cu
void launch_scaling(bchar_mesh_t m);
void launch_scaling_once(bchar_mesh_t m);  // one column and one row scaling (timing aid)
bool launch_minimise(bchar_mesh_t m, int *cg_iters, int *ip_iters);  // false: out of memory
void launch_finalise(bchar_mesh_t m);
void launch_update(bchar_mesh_t m, const void *c_in, void *c_out, int c_dtype);
void launch_cg_matvec_once(bchar_mesh_t m, CgState *st);  // q = J p with the current p, for timing
int last_substeps(bchar_mesh_t m);

}  // namespace bchar
