/*
 * bchar_oracle.c -- plain FP64 CPU oracle for the per-step geometry of the
 * ball-approximated characteristics (B-char) method (Cheng & Droniou,
 * arXiv 1908.05834).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * CUDA path is checked against.  Only tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header,
 * table or helper with the CUDA library, and the CUDA library never loads it.
 *
 * Everything is double precision, serial, with no blocking or reordering
 * beyond what each definition states.  Positions are absolute coordinates.
 *
 * Contents (paper section / equation each part follows):
 *   - RT0 velocity evaluation on a tensor-product mesh          (Sec 1.2, hyp:un)
 *   - classical RK4 integration of the flow dF/dt = u/phi       (Sec 2, eq. charac)
 *   - tracked radius from cardinal points                       (Sec 3, eq. rTrackedBall)
 *   - ball-ball intersection measure (lens area / lens volume)  (Sec 3, "trivial" intersections)
 *   - the initial weights V_{K,M}                               (Sec 3.1, eq. fracMaterial, eq. ball_int)
 *
 * Readings where the paper is silent:
 *   - all balls of a cell have the radius r_K = min(width)/(2 nb) (a quarter of
 *     the smallest face for nb = 2); along axis a the cell holds
 *     n_a = max(nb, floor(nb w_a / w_min)) balls at the centres of an equal
 *     split, so the cell is tightly packed (nb^d balls on a cube, more along
 *     the long axes of a stretched cell);
 *   - a tracked point starts in the cell of its ball, and the first RK stage is
 *     evaluated there; every later point is located by "last node x_i <= p",
 *     clamped to the mesh, and every stage point is clamped into the closed box;
 *   - a tracked ball that meets no residing ball deposits its mass in the cell
 *     that contains its tracked centre;
 *   - V_{K,M} < drop_tol * |K|_phi is dropped.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int dim;              /* 2 or 3 */
    int nb;               /* balls per axis (nb^dim balls per cell) */
    int64_t n[3];         /* cells per axis; n[2] = 1 when dim = 2 */
    const double *x[3];   /* node coordinates per axis, n[a]+1 values, increasing */
    const double *phi;    /* porosity per cell, x index fastest */
    const double *u[3];   /* RT0 face-normal velocities per axis (see face_index) */
} orc_mesh;

/* ---------------------------------------------------------------- geometry */

static double width(const orc_mesh *m, int a, int64_t i) { return m->x[a][i + 1] - m->x[a][i]; }

static int64_t cell_flat(const orc_mesh *m, const int64_t c[3]) {
    return c[0] + m->n[0] * (c[1] + m->n[1] * c[2]);
}

static void cell_split(const orc_mesh *m, int64_t k, int64_t c[3]) {
    c[0] = k % m->n[0];
    c[1] = (k / m->n[0]) % m->n[1];
    c[2] = k / (m->n[0] * m->n[1]);
}

/* |K| */
double orc_cell_volume(const orc_mesh *m, int64_t k) {
    int64_t c[3];
    cell_split(m, k, c);
    double v = 1.0;
    for (int a = 0; a < m->dim; ++a) v *= width(m, a, c[a]);
    return v;
}

/* Ball radius of cell k: min width / (2 nb), so that the nb^d balls at the
 * sub-cell centres are disjoint and inside the cell (Sec 3, radius at most a
 * quarter of the smallest face for nb = 2). */
double orc_ball_radius(const orc_mesh *m, int64_t k) {
    int64_t c[3];
    cell_split(m, k, c);
    double w = width(m, 0, c[0]);
    for (int a = 1; a < m->dim; ++a) {
        double wa = width(m, a, c[a]);
        if (wa < w) w = wa;
    }
    return w / (2.0 * m->nb);
}

/* Balls along each axis of cell k: n_a = max(nb, floor(nb w_a / w_min)), so
 * that neighbouring balls are at least 2 r_K apart (disjoint) and at most
 * 2 r_K (nb+1)/nb apart (tightly packed); n_a = nb on a cube. */
void orc_ball_counts(const orc_mesh *m, int64_t k, int cnt[3]) {
    int64_t c[3];
    cell_split(m, k, c);
    double wmin = width(m, 0, c[0]);
    for (int a = 1; a < m->dim; ++a) {
        double wa = width(m, a, c[a]);
        if (wa < wmin) wmin = wa;
    }
    cnt[0] = cnt[1] = cnt[2] = 1;
    for (int a = 0; a < m->dim; ++a) {
        int q = (int)floor(m->nb * width(m, a, c[a]) / wmin + 1e-9);
        cnt[a] = q < m->nb ? m->nb : q;
    }
}

/* n_K, the number of balls of cell k. */
int orc_ball_total(const orc_mesh *m, int64_t k) {
    int cnt[3];
    orc_ball_counts(m, k, cnt);
    return cnt[0] * cnt[1] * cnt[2];
}

/* |B| for radius r in dimension dim. */
static double ball_measure(int dim, double r) {
    return dim == 2 ? M_PI * r * r : 4.0 / 3.0 * M_PI * r * r * r;
}

/* Centre of ball s (s = sx + nx*(sy + ny*sz), n_a the counts above) of cell k. */
void orc_ball_centre(const orc_mesh *m, int64_t k, int s, double p[3]) {
    int64_t c[3];
    cell_split(m, k, c);
    int cnt[3];
    orc_ball_counts(m, k, cnt);
    int sub[3] = {s % cnt[0], (s / cnt[0]) % cnt[1], s / (cnt[0] * cnt[1])};
    p[2] = 0.0;
    for (int a = 0; a < m->dim; ++a)
        p[a] = m->x[a][c[a]] + (sub[a] + 0.5) * width(m, a, c[a]) / cnt[a];
}

/* Last i with x[i] <= p, clamped to [0, n-1] (binary search). */
static int64_t locate_axis(const double *x, int64_t n, double p) {
    if (p <= x[0]) return 0;
    if (p >= x[n]) return n - 1;
    int64_t lo = 0, hi = n; /* invariant: x[lo] <= p < x[hi] */
    while (hi - lo > 1) {
        int64_t mid = lo + (hi - lo) / 2;
        if (x[mid] <= p) lo = mid; else hi = mid;
    }
    return lo;
}

int64_t orc_locate(const orc_mesh *m, const double p[3]) {
    int64_t c[3] = {0, 0, 0};
    for (int a = 0; a < m->dim; ++a) c[a] = locate_axis(m->x[a], m->n[a], p[a]);
    return cell_flat(m, c);
}

/* ------------------------------------------------------- RT0 velocity field */

/* Index of the face of axis a with face coordinate f (0..n[a]) and cell
 * coordinates c[b] for the other axes; x index fastest, the face axis has n[a]+1
 * entries. */
static int64_t face_index(const orc_mesh *m, int a, const int64_t c[3], int64_t f) {
    int64_t e[3] = {c[0], c[1], c[2]};
    int64_t len[3] = {m->n[0], m->n[1], m->n[2]};
    e[a] = f;
    len[a] += 1;
    return e[0] + len[0] * (e[1] + len[1] * e[2]);
}

/* Lowest-order Raviart-Thomas interpolant in cell c at point p: component a is
 * linear in x_a between the two a-faces of the cell and constant in the other
 * coordinates (Sec 1.2, u^{(n+1)} piecewise polynomial in H(div)). */
static void rt0_velocity(const orc_mesh *m, const int64_t c[3], const double p[3], double u[3]) {
    u[0] = u[1] = u[2] = 0.0;
    for (int a = 0; a < m->dim; ++a) {
        double lo = m->u[a][face_index(m, a, c, c[a])];
        double hi = m->u[a][face_index(m, a, c, c[a] + 1)];
        double t = (p[a] - m->x[a][c[a]]) / width(m, a, c[a]);
        u[a] = lo + t * (hi - lo);
    }
}

static void clamp_to_box(const orc_mesh *m, double p[3]) {
    for (int a = 0; a < m->dim; ++a) {
        if (p[a] < m->x[a][0]) p[a] = m->x[a][0];
        if (p[a] > m->x[a][m->n[a]]) p[a] = m->x[a][m->n[a]];
    }
}

/* Right-hand side of the flow, sign * u(p)/phi(p) (eq. charac).  When
 * forced_cell >= 0 that cell is used instead of locating p. */
static void flow_rhs(const orc_mesh *m, double sign, const double p[3], int64_t forced_cell, double f[3]) {
    int64_t k = forced_cell >= 0 ? forced_cell : orc_locate(m, p);
    int64_t c[3];
    cell_split(m, k, c);
    double u[3];
    rt0_velocity(m, c, p, u);
    double ph = m->phi[k];
    for (int a = 0; a < 3; ++a) f[a] = sign * u[a] / ph;
}

/* Classical RK4 with `substeps` equal steps over a time span tau, solving
 * dp/dt = sign * u(p)/phi(p) from p0 (sign = -1 tracks back along the flow,
 * giving F_{-tau}(p0); sign = +1 gives F_{tau}(p0)).  The first stage is
 * evaluated in start_cell. */
void orc_rk4(const orc_mesh *m, double sign, double tau, int substeps,
             const double p0[3], int64_t start_cell, double out[3]) {
    double p[3] = {p0[0], p0[1], p0[2]};
    double h = tau / substeps;
    for (int st = 0; st < substeps; ++st) {
        double k1[3], k2[3], k3[3], k4[3], q[3];
        flow_rhs(m, sign, p, st == 0 ? start_cell : -1, k1);
        for (int a = 0; a < 3; ++a) q[a] = p[a] + 0.5 * h * k1[a];
        clamp_to_box(m, q);
        flow_rhs(m, sign, q, -1, k2);
        for (int a = 0; a < 3; ++a) q[a] = p[a] + 0.5 * h * k2[a];
        clamp_to_box(m, q);
        flow_rhs(m, sign, q, -1, k3);
        for (int a = 0; a < 3; ++a) q[a] = p[a] + h * k3[a];
        clamp_to_box(m, q);
        flow_rhs(m, sign, q, -1, k4);
        for (int a = 0; a < 3; ++a) p[a] = p[a] + h / 6.0 * (k1[a] + 2.0 * k2[a] + 2.0 * k3[a] + k4[a]);
        clamp_to_box(m, p);
    }
    for (int a = 0; a < 3; ++a) out[a] = p[a];
}

/* Track many points: p0[i*3..], start cells cells[i]. */
void orc_rk4_many(const orc_mesh *m, double sign, double tau, int substeps, int64_t npts,
                  const double *p0, const int64_t *cells, double *out) {
    for (int64_t i = 0; i < npts; ++i) orc_rk4(m, sign, tau, substeps, p0 + 3 * i, cells[i], out + 3 * i);
}

/* Tracked centre and radius of every ball of the cells listed in rows.
 * If phi_const: only the centre is tracked and r_hat = r (eq. ball_volChange).
 * Otherwise the 2*dim points C +- r e_a are tracked too and r_hat is the mean
 * distance from the tracked centre to them (eq. rTrackedBall; the 3D analogue
 * uses the six points on the axes).
 * Ball b = offset[r] + s of listed row r (offset = running sum of n_K):
 * centres[3 b + a], rhat[b]. */
void orc_track_balls(const orc_mesh *m, double dt, int substeps, int phi_const,
                     int64_t nrows, const int64_t *rows, const int64_t *offset, double *centres, double *rhat) {
    for (int64_t r = 0; r < nrows; ++r) {
        int64_t k = rows[r];
        double rad = orc_ball_radius(m, k);
        int nballs = orc_ball_total(m, k);
        for (int s = 0; s < nballs; ++s) {
            int64_t b = offset[r] + s;
            double c0[3], c1[3];
            orc_ball_centre(m, k, s, c0);
            orc_rk4(m, -1.0, dt, substeps, c0, k, c1);
            double *dst = centres + 3 * b;
            for (int a = 0; a < 3; ++a) dst[a] = c1[a];
            if (phi_const) {
                rhat[b] = rad;
                continue;
            }
            double sum = 0.0;
            for (int a = 0; a < m->dim; ++a) {
                for (int sg = -1; sg <= 1; sg += 2) {
                    double q0[3] = {c0[0], c0[1], c0[2]}, q1[3];
                    q0[a] += sg * rad;
                    orc_rk4(m, -1.0, dt, substeps, q0, k, q1);
                    double d2 = 0.0;
                    for (int b = 0; b < m->dim; ++b) d2 += (q1[b] - c1[b]) * (q1[b] - c1[b]);
                    sum += sqrt(d2);
                }
            }
            rhat[b] = sum / (2.0 * m->dim);
        }
    }
}

/* ------------------------------------------------------ intersection measure */

/* Area of the intersection of two discs of radii r1, r2 whose centres are d
 * apart: the two circular sectors spanned by the common chord minus the kite
 * formed by the centres and the chord's end points, sector_i = r_i^2 theta_i,
 * kite = d h.  The half-chord h comes from the product (Heron) form and the
 * half-angles from atan2, which stay accurate for nearly tangent discs
 * (acos of a cosine near 1 would not). */
double orc_lens_area(double d, double r1, double r2) {
    if (d >= r1 + r2) return 0.0;
    double rmin = r1 < r2 ? r1 : r2;
    if (d <= fabs(r1 - r2)) return M_PI * rmin * rmin;
    double k = (-d + r1 + r2) * (d + r1 - r2) * (d - r1 + r2) * (d + r1 + r2);
    if (k < 0.0) k = 0.0;
    double h = sqrt(k) / (2.0 * d);
    double x1 = (d * d + r1 * r1 - r2 * r2) / (2.0 * d); /* centre 1 to the chord, signed */
    double x2 = d - x1;
    double area = r1 * r1 * atan2(h, x1) + r2 * r2 * atan2(h, x2) - d * h;
    return area > 0.0 ? area : 0.0;
}

/* Volume of the intersection of two balls of radii r1, r2 whose centres are d
 * apart (closed form of the lens volume). */
double orc_lens_volume(double d, double r1, double r2) {
    if (d >= r1 + r2) return 0.0;
    double rmin = r1 < r2 ? r1 : r2;
    if (d <= fabs(r1 - r2)) return 4.0 / 3.0 * M_PI * rmin * rmin * rmin;
    double t = r1 + r2 - d;
    return M_PI * t * t * (d * d + 2.0 * d * r1 + 2.0 * d * r2 - 3.0 * r1 * r1 - 3.0 * r2 * r2 + 6.0 * r1 * r2) /
           (12.0 * d);
}

static double lens(int dim, double d, double r1, double r2) {
    return dim == 2 ? orc_lens_area(d, r1, r2) : orc_lens_volume(d, r1, r2);
}

/* --------------------------------------------------------- initial weights */

/* The largest ball radius of the mesh. */
double orc_max_radius(const orc_mesh *m) {
    int64_t nc = m->n[0] * m->n[1] * m->n[2];
    double r = 0.0;
    for (int64_t k = 0; k < nc; ++k) {
        double rk = orc_ball_radius(m, k);
        if (rk > r) r = rk;
    }
    return r;
}

/* First and last index of the cells of axis a whose closed extent meets
 * [lo, hi]. */
static void axis_range(const orc_mesh *m, int a, double lo, double hi, int64_t *first, int64_t *last) {
    *first = locate_axis(m->x[a], m->n[a], lo);
    /* a cell whose upper node equals lo also meets the interval */
    while (*first > 0 && m->x[a][*first] >= lo) --*first;
    *last = locate_axis(m->x[a], m->n[a], hi);
}

typedef struct {
    int64_t col;
    double val;
} entry;

static int cmp_entry(const void *a, const void *b) {
    int64_t x = ((const entry *)a)->col, y = ((const entry *)b)->col;
    return (x > y) - (x < y);
}

/* Row K of A^(0): V_{K,M} for every residing cell M (eq. ball_int), from the
 * tracked centres and radii of K's balls.
 *
 * For every tracked ball s of K and every residing ball (M, m) with
 * |C_hat - C_{M,m}| < r_hat + r_M, w = rho_M phi_M |B_hat cap B_{M,m}| with
 * rho_M phi_M = |M|_phi / (n_M |B_M|) (eq. def:porous.density).  The mass of
 * tracked ball s is rho_K phi_hat |B_hat| = rho_K phi_K |B_K| = |K|_phi / n_K
 * (eq. expPhiB); it is split over the residing cells in the proportions
 * sum_{m in M} w / sum_all w (eq. fracMaterial).
 *
 * Residing balls are found by looking at every cell whose extent meets the
 * box C_hat +- (r_hat + r_max): a ball inside a cell outside that box is
 * farther than r_hat + r_max from C_hat.
 *
 * cols/vals receive the row (sorted by column) with up to cap entries;
 * returns the number of entries, or -1 if cap is too small.  *voids is
 * incremented for each tracked ball that meets no residing ball. */
int64_t orc_assemble_row(const orc_mesh *m, int64_t K, const double *centres, const double *rhat,
                         double r_max, double drop_tol, int64_t cap, int64_t *cols, double *vals,
                         int64_t *voids) {
    int nballs = orc_ball_total(m, K);
    double volphi_K = m->phi[K] * orc_cell_volume(m, K);
    double mass_ball = volphi_K / nballs;

    int64_t row_cap = 4096, row_n = 0;
    entry *row = (entry *)malloc(sizeof(entry) * row_cap);
    int64_t cand_cap = 4096;
    entry *cand = (entry *)malloc(sizeof(entry) * cand_cap); /* (cell M, w) per residing ball */

    for (int s = 0; s < nballs; ++s) {
        const double *p = centres + 3 * s;
        double rh = rhat[s];
        double reach = rh + r_max;
        int64_t lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
        for (int a = 0; a < m->dim; ++a) axis_range(m, a, p[a] - reach, p[a] + reach, &lo[a], &hi[a]);
        int64_t nc_cand = 0;
        for (int64_t cz = lo[2]; cz <= hi[2]; ++cz)
            for (int64_t cy = lo[1]; cy <= hi[1]; ++cy)
                for (int64_t cx = lo[0]; cx <= hi[0]; ++cx) {
                    int64_t cM[3] = {cx, cy, cz};
                    int64_t M = cell_flat(m, cM);
                    double rM = orc_ball_radius(m, M);
                    int nballs_M = orc_ball_total(m, M);
                    double rhophi_M = m->phi[M] * orc_cell_volume(m, M) / (nballs_M * ball_measure(m->dim, rM));
                    for (int sm = 0; sm < nballs_M; ++sm) {
                        double q[3];
                        orc_ball_centre(m, M, sm, q);
                        double d2 = 0.0;
                        for (int a = 0; a < m->dim; ++a) d2 += (p[a] - q[a]) * (p[a] - q[a]);
                        double d = sqrt(d2);
                        if (!(d < rh + rM)) continue;
                        double w = rhophi_M * lens(m->dim, d, rh, rM);
                        if (nc_cand == cand_cap) {
                            cand_cap *= 2;
                            cand = (entry *)realloc(cand, sizeof(entry) * cand_cap);
                        }
                        cand[nc_cand].col = M;
                        cand[nc_cand].val = w;
                        ++nc_cand;
                    }
                }
        double den = 0.0;
        for (int64_t c = 0; c < nc_cand; ++c) den += cand[c].val;
        if (den == 0.0) {
            /* void: the whole mass of the ball goes to the cell holding C_hat */
            ++*voids;
            if (row_n == row_cap) { row_cap *= 2; row = (entry *)realloc(row, sizeof(entry) * row_cap); }
            row[row_n].col = orc_locate(m, p);
            row[row_n].val = mass_ball;
            ++row_n;
            continue;
        }
        /* S_{s,M} = sum over the balls of M, then mass_ball * S / den */
        qsort(cand, nc_cand, sizeof(entry), cmp_entry);
        int64_t c = 0;
        while (c < nc_cand) {
            int64_t M = cand[c].col;
            double S = 0.0;
            while (c < nc_cand && cand[c].col == M) S += cand[c++].val;
            if (row_n == row_cap) { row_cap *= 2; row = (entry *)realloc(row, sizeof(entry) * row_cap); }
            row[row_n].col = M;
            row[row_n].val = mass_ball * (S / den);
            ++row_n;
        }
    }
    /* merge equal columns (sum over the tracked balls s), drop tiny entries */
    qsort(row, row_n, sizeof(entry), cmp_entry);
    int64_t out = 0, i = 0;
    int overflow = 0;
    while (i < row_n) {
        int64_t M = row[i].col;
        double V = 0.0;
        while (i < row_n && row[i].col == M) V += row[i++].val;
        if (V < drop_tol * volphi_K) continue;
        if (out == cap) { overflow = 1; break; }
        cols[out] = M;
        vals[out] = V;
        ++out;
    }
    free(row);
    free(cand);
    return overflow ? -1 : out;
}

/* All rows listed in rows[] (n_rows of them), with tracked data laid out as
 * produced by orc_track_balls (same offsets).  Rows are written one after another into
 * cols/vals (total capacity cap); row_len[r] receives each row's length.
 * Returns the total entry count, or -1 on overflow. */
int64_t orc_assemble_rows(const orc_mesh *m, int64_t nrows, const int64_t *rows, const int64_t *offset,
                          const double *centres, const double *rhat, double drop_tol, int64_t cap, int64_t *cols,
                          double *vals, int64_t *row_len, int64_t *voids) {
    double r_max = orc_max_radius(m);
    int64_t used = 0;
    for (int64_t r = 0; r < nrows; ++r) {
        int64_t len = orc_assemble_row(m, rows[r], centres + 3 * offset[r], rhat + offset[r], r_max,
                                       drop_tol, cap - used, cols + used, vals + used, voids);
        if (len < 0) return -1;
        row_len[r] = len;
        used += len;
    }
    return used;
}

/* n_K for each listed cell. */
void orc_ball_totals(const orc_mesh *m, int64_t nrows, const int64_t *rows, int64_t *out) {
    for (int64_t r = 0; r < nrows; ++r) out[r] = orc_ball_total(m, rows[r]);
}
