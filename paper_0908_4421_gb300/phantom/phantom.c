/*
 * Seeded synthetic prostate phantom and its dose-deposition matrix D.
 *
 * This is an INPUT generator. It stands in for the clinical prostate case of
 * the paper's Sec. 3.1 / Table 1, which is not available. It contains none of
 * the optimiser's arithmetic: no penalty, no normalisation, no gradient.
 * Both the CUDA library and the FP64 oracle consume what it writes.
 *
 * Geometry (all lengths in mm, isocentre at the grid centre):
 *   x = left-right, y = anterior(+) / posterior(-), z = superior(+).
 *   Body    : elliptic cylinder along z, semi-axes body_a (x) and body_b (y).
 *   PTV     : axis-aligned ellipsoid, radii ptv_r, centre ptv_c.
 *   Rectum  : cylinder along z, radius rect_r, axis at (0, rect_y), z in [rect_z0, rect_z1].
 *   Bladder : sphere, radius blad_r, centre blad_c.
 *   Beams   : coplanar, parallel (no divergence); gantry angle theta measured
 *             from anterior, source direction s = (sin t, cos t, 0), beam
 *             travels along d = -s. Beam's-eye axes: u = (cos t, -sin t, 0), v = z.
 *   Beamlets: square grid of pitch beamlet_mm in the (u, v) plane through the
 *             isocentre, centres at (k + 1/2) * pitch, k integer. A beamlet is
 *             kept when its centre lies inside the PTV projection with both
 *             semi-axes enlarged by margin_mm.
 *   D_ij    : exp(-mu * depth_j) * exp(-rho_ij^2 / (2 sigma^2)), where depth is
 *             the path length inside the body from the entry surface to voxel j
 *             along the beam, and rho is the distance of voxel j's centre from
 *             beamlet i's central ray. Entries below `cutoff` are dropped.
 *   Rows    : body voxels only, raster order (z slowest, then y, then x). With
 *             coarse_unspecified, voxels in no structure but the body are kept
 *             only where all three grid indices are even (the 2x coarser grid
 *             of the paper's Sec. 3.1 for unspecified tissue), at that voxel's
 *             centre.
 *   Columns : beam-major, then v row, then u, over kept beamlets; each row's
 *             columns come out strictly increasing.
 *
 * Built with -ffp-contract=off so that x86-64 and aarch64 builds round alike.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t nx, ny, nz;
    double spacing;
    double body_a, body_b;
    double ptv_r[3];
    double ptv_c[3];
    double rect_r, rect_y, rect_z0, rect_z1;
    double blad_r;
    double blad_c[3];
    int32_t n_beams;
    double angle0_deg;
    double beamlet_mm;
    double margin_mm;
    double mu_per_mm;
    double sigma_mm;
    double cutoff;
    int32_t coarse_unspecified; /* 1: tissue outside the PTV and organs only on the 2x coarser grid */
} phantom_spec;

#define BIT_PTV 1u
#define BIT_RECTUM 2u
#define BIT_BLADDER 4u
#define BIT_BODY 8u

static double coord(int32_t i, int32_t n, double h) { return ((double)i + 0.5 - 0.5 * (double)n) * h; }

static int in_body(const phantom_spec* s, double x, double y) {
    double a = x / s->body_a, b = y / s->body_b;
    return a * a + b * b <= 1.0;
}

static uint8_t structure_bits(const phantom_spec* s, double x, double y, double z) {
    uint8_t b = BIT_BODY;
    double px = (x - s->ptv_c[0]) / s->ptv_r[0];
    double py = (y - s->ptv_c[1]) / s->ptv_r[1];
    double pz = (z - s->ptv_c[2]) / s->ptv_r[2];
    if (px * px + py * py + pz * pz <= 1.0) b |= BIT_PTV;
    double ry = y - s->rect_y;
    if (x * x + ry * ry <= s->rect_r * s->rect_r && z >= s->rect_z0 && z <= s->rect_z1) b |= BIT_RECTUM;
    double bx = x - s->blad_c[0], by = y - s->blad_c[1], bz = z - s->blad_c[2];
    if (bx * bx + by * by + bz * bz <= s->blad_r * s->blad_r) b |= BIT_BLADDER;
    return b;
}

/* Whether grid voxel (ix, iy, iz) is a row of D. */
static int keep_voxel(const phantom_spec* s, int32_t ix, int32_t iy, int32_t iz) {
    double x = coord(ix, s->nx, s->spacing), y = coord(iy, s->ny, s->spacing), z = coord(iz, s->nz, s->spacing);
    if (!in_body(s, x, y)) return 0;
    if (!s->coarse_unspecified) return 1;
    if (structure_bits(s, x, y, z) != BIT_BODY) return 1;
    return (ix % 2 == 0) && (iy % 2 == 0) && (iz % 2 == 0);
}

int64_t phantom_count_body(const phantom_spec* s) {
    int64_t m = 0;
    for (int32_t iz = 0; iz < s->nz; ++iz)
        for (int32_t iy = 0; iy < s->ny; ++iy)
            for (int32_t ix = 0; ix < s->nx; ++ix)
                if (keep_voxel(s, ix, iy, iz)) ++m;
    return m;
}

/* Voxel centres (m x 3, mm) and structure bitmask (m). */
void phantom_fill_voxels(const phantom_spec* s, float* xyz, uint8_t* mask) {
    int64_t j = 0;
    for (int32_t iz = 0; iz < s->nz; ++iz) {
        double z = coord(iz, s->nz, s->spacing);
        for (int32_t iy = 0; iy < s->ny; ++iy) {
            double y = coord(iy, s->ny, s->spacing);
            for (int32_t ix = 0; ix < s->nx; ++ix) {
                double x = coord(ix, s->nx, s->spacing);
                if (!keep_voxel(s, ix, iy, iz)) continue;
                if (xyz) {
                    xyz[3 * j + 0] = (float)x;
                    xyz[3 * j + 1] = (float)y;
                    xyz[3 * j + 2] = (float)z;
                }
                mask[j] = structure_bits(s, x, y, z);
                ++j;
            }
        }
    }
}

/* Per-beam beamlet grid: half-counts, the kept-beamlet index map and geometry. */
typedef struct {
    double ct, st;   /* cos / sin of gantry angle */
    int32_t ku, kv;  /* grid spans k in [-ku, ku-1] x [-kv, kv-1] */
    int32_t* index;  /* (2kv) x (2ku), -1 where not kept */
} beam_grid;

static double deg2rad(double a) { return a * 3.14159265358979323846 / 180.0; }

/* Builds all beam grids; returns the number of kept beamlets. */
static int32_t build_grids(const phantom_spec* s, beam_grid* g) {
    int32_t next = 0;
    double h = s->beamlet_mm;
    for (int32_t b = 0; b < s->n_beams; ++b) {
        double th = deg2rad(s->angle0_deg + 360.0 * (double)b / (double)s->n_beams);
        double ct = cos(th), st = sin(th);
        g[b].ct = ct;
        g[b].st = st;
        /* support of the PTV ellipse along u = (cos t, -sin t) and along z */
        double hu = sqrt(s->ptv_r[0] * s->ptv_r[0] * ct * ct + s->ptv_r[1] * s->ptv_r[1] * st * st) + s->margin_mm;
        double hv = s->ptv_r[2] + s->margin_mm;
        double cu = s->ptv_c[0] * ct - s->ptv_c[1] * st; /* PTV centre in beam's-eye coordinates */
        double cv = s->ptv_c[2];
        int32_t ku = (int32_t)ceil((fabs(cu) + hu) / h) + 1;
        int32_t kv = (int32_t)ceil((fabs(cv) + hv) / h) + 1;
        g[b].ku = ku;
        g[b].kv = kv;
        g[b].index = (int32_t*)malloc(sizeof(int32_t) * (size_t)(4 * ku * kv));
        for (int32_t iv = 0; iv < 2 * kv; ++iv) {
            double v = ((double)(iv - kv) + 0.5) * h;
            for (int32_t iu = 0; iu < 2 * ku; ++iu) {
                double u = ((double)(iu - ku) + 0.5) * h;
                double a = (u - cu) / hu, c = (v - cv) / hv;
                g[b].index[iv * 2 * ku + iu] = (a * a + c * c <= 1.0) ? next++ : -1;
            }
        }
    }
    return next;
}

static void free_grids(const phantom_spec* s, beam_grid* g) {
    for (int32_t b = 0; b < s->n_beams; ++b) free(g[b].index);
}

int32_t phantom_count_beamlets(const phantom_spec* s) {
    beam_grid* g = (beam_grid*)calloc((size_t)s->n_beams, sizeof(beam_grid));
    int32_t n = build_grids(s, g);
    free_grids(s, g);
    free(g);
    return n;
}

/* Beamlet table (n x 3): beam index, u centre, v centre (mm). */
void phantom_fill_beamlets(const phantom_spec* s, float* info) {
    beam_grid* g = (beam_grid*)calloc((size_t)s->n_beams, sizeof(beam_grid));
    build_grids(s, g);
    double h = s->beamlet_mm;
    for (int32_t b = 0; b < s->n_beams; ++b)
        for (int32_t iv = 0; iv < 2 * g[b].kv; ++iv)
            for (int32_t iu = 0; iu < 2 * g[b].ku; ++iu) {
                int32_t id = g[b].index[iv * 2 * g[b].ku + iu];
                if (id < 0) continue;
                info[3 * id + 0] = (float)b;
                info[3 * id + 1] = (float)(((double)(iu - g[b].ku) + 0.5) * h);
                info[3 * id + 2] = (float)(((double)(iv - g[b].kv) + 0.5) * h);
            }
    free_grids(s, g);
    free(g);
}

/* Path length inside the body from the entry surface to p, along d = -(sin t, cos t). */
static double depth_in_body(const phantom_spec* s, double px, double py, double ct, double st) {
    double dx = -st, dy = -ct;
    double ia = 1.0 / (s->body_a * s->body_a), ib = 1.0 / (s->body_b * s->body_b);
    double A = dx * dx * ia + dy * dy * ib;
    double B = px * dx * ia + py * dy * ib;
    double C = px * px * ia + py * py * ib - 1.0;
    double disc = B * B - A * C;
    if (disc < 0.0) disc = 0.0;
    double t = (B + sqrt(disc)) / A; /* distance back toward the source to the surface */
    return t > 0.0 ? t : 0.0;
}

/* Visits every entry of voxel row j in column order. With cols == NULL it only counts. */
static int64_t row_entries(const phantom_spec* s, const beam_grid* g, double x, double y, double z, int32_t* cols,
                           float* vals) {
    int64_t cnt = 0;
    double h = s->beamlet_mm;
    double two_s2 = 2.0 * s->sigma_mm * s->sigma_mm;
    for (int32_t b = 0; b < s->n_beams; ++b) {
        double ct = g[b].ct, st = g[b].st;
        double u = x * ct - y * st;
        double v = z;
        double dep = depth_in_body(s, x, y, ct, st);
        double atten = exp(-s->mu_per_mm * dep);
        if (atten < s->cutoff) continue;
        double rmax2 = two_s2 * log(atten / s->cutoff);
        double rmax = sqrt(rmax2);
        int32_t ku = g[b].ku, kv = g[b].kv;
        int32_t iv0 = (int32_t)floor((v - rmax) / h - 0.5) + kv, iv1 = (int32_t)ceil((v + rmax) / h - 0.5) + kv;
        int32_t iu0 = (int32_t)floor((u - rmax) / h - 0.5) + ku, iu1 = (int32_t)ceil((u + rmax) / h - 0.5) + ku;
        if (iv0 < 0) iv0 = 0;
        if (iu0 < 0) iu0 = 0;
        if (iv1 > 2 * kv - 1) iv1 = 2 * kv - 1;
        if (iu1 > 2 * ku - 1) iu1 = 2 * ku - 1;
        double slack = rmax2 * 1e-9 + 1e-9;
        for (int32_t iv = iv0; iv <= iv1; ++iv) {
            double dv = v - ((double)(iv - kv) + 0.5) * h;
            double dv2 = dv * dv;
            if (dv2 > rmax2 + slack) continue;
            const int32_t* irow = g[b].index + (size_t)iv * 2 * ku;
            for (int32_t iu = iu0; iu <= iu1; ++iu) {
                int32_t id = irow[iu];
                if (id < 0) continue;
                double du = u - ((double)(iu - ku) + 0.5) * h;
                double r2 = du * du + dv2;
                if (r2 > rmax2 + slack) continue;
                double val = atten * exp(-r2 / two_s2);
                if (!(val >= s->cutoff)) continue;
                if (cols) {
                    cols[cnt] = id;
                    vals[cnt] = (float)val;
                }
                ++cnt;
            }
        }
    }
    return cnt;
}

/* Fills voxel centres for all body voxels (m x 3, double) used by the row passes. */
static double* body_centres(const phantom_spec* s, int64_t m) {
    double* c = (double*)malloc(sizeof(double) * (size_t)(3 * m));
    int64_t j = 0;
    for (int32_t iz = 0; iz < s->nz; ++iz)
        for (int32_t iy = 0; iy < s->ny; ++iy)
            for (int32_t ix = 0; ix < s->nx; ++ix) {
                if (!keep_voxel(s, ix, iy, iz)) continue;
                double x = coord(ix, s->nx, s->spacing), y = coord(iy, s->ny, s->spacing);
                c[3 * j + 0] = x;
                c[3 * j + 1] = y;
                c[3 * j + 2] = coord(iz, s->nz, s->spacing);
                ++j;
            }
    return c;
}

/* Pass 1: nonzeros per voxel row (m entries). */
void phantom_count_rows(const phantom_spec* s, int64_t m, int64_t* row_nnz) {
    beam_grid* g = (beam_grid*)calloc((size_t)s->n_beams, sizeof(beam_grid));
    build_grids(s, g);
    double* c = body_centres(s, m);
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t j = 0; j < m; ++j) row_nnz[j] = row_entries(s, g, c[3 * j], c[3 * j + 1], c[3 * j + 2], NULL, NULL);
    free(c);
    free_grids(s, g);
    free(g);
}

/* Pass 2: column indices and values, given row_ptr from pass 1. */
void phantom_fill_rows(const phantom_spec* s, int64_t m, const int64_t* row_ptr, int32_t* col, float* val) {
    beam_grid* g = (beam_grid*)calloc((size_t)s->n_beams, sizeof(beam_grid));
    build_grids(s, g);
    double* c = body_centres(s, m);
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t j = 0; j < m; ++j)
        row_entries(s, g, c[3 * j], c[3 * j + 1], c[3 * j + 2], col + row_ptr[j], val + row_ptr[j]);
    free(c);
    free_grids(s, g);
    free(g);
}
