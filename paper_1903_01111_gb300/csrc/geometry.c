/* Host-side geometry builder: solid mask and cut-link list with the wall
 * fraction q of each link (Sec. 3: fluid, solid and boundary nodes; q is the
 * distance from the boundary node x_f to the wall along the link, divided by
 * the link length).
 *
 * This file computes geometry only.  It holds none of the lattice-Boltzmann
 * arithmetic and is the one input generator that both the CUDA library's
 * tests and the CPU oracle read from.
 *
 * Bodies: closed balls (circles in 2-D, spheres in 3-D) and half-spaces.  A
 * node is solid iff it lies in a body (|x - c| <= R, or n.x >= d).  For a
 * fluid node x_f and a direction i' whose neighbour x_s = x_f + e_i' is solid,
 * q is the smallest t in (0, 1] at which x_f + t e_i' enters a body.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>

typedef struct {
  int32_t kind;      /* 0 = ball, 1 = half-space */
  int32_t force_id;  /* value stored in lbm_link.body, or -1 */
  int32_t bc;        /* value stored in lbm_link.bc (-1 = lattice default) */
  int32_t pad;
  double c[3];       /* ball centre, or half-space normal n (unit, into the solid) */
  double r;          /* ball radius, or half-space offset d */
  double vel[3];     /* translational velocity */
  double omega[3];   /* angular velocity about c (balls only) */
} geom_body;

typedef struct {
  int64_t node;
  int32_t dir;
  int16_t bc;
  int16_t body;
  double q;
  double uw[3];
} geom_link;

/* Velocity sets in the library's direction numbering. */
static const int E2[9][3] = {{0, 0, 0}, {1, 0, 0},  {0, 1, 0},   {-1, 0, 0}, {0, -1, 0},
                             {1, 1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
static const int E3[19][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},
                              {0, 0, 1},  {0, 0, -1}, {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},
                              {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1},  {-1, 0, 1},
                              {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

typedef struct {
  int nx, ny, nz;
  int periodic[3];
  int Q;
  const int (*e)[3];
  const geom_body* bodies;
  int nb;
  /* uniform cell grid over the lattice for ball lookup */
  int cs;            /* cell size */
  int gx, gy, gz;    /* cells per axis */
  int32_t* cell_start;
  int32_t* cell_items;
  int32_t* planes;   /* indices of half-spaces */
  int nplanes;
} ctx_t;

static double min_image(double d, int L, int periodic) {
  if (periodic) d -= L * floor(d / L + 0.5);
  return d;
}

/* displacement x - c of a ball, minimal image on periodic axes */
static void ball_disp(const ctx_t* g, const geom_body* b, const double x[3], double d[3]) {
  const int L[3] = {g->nx, g->ny, g->nz};
  for (int a = 0; a < 3; ++a) d[a] = min_image(x[a] - b->c[a], L[a], g->periodic[a]);
}

static int inside(const ctx_t* g, const geom_body* b, const double x[3]) {
  if (b->kind == 0) {
    double d[3];
    ball_disp(g, b, x, d);
    return d[0] * d[0] + d[1] * d[1] + d[2] * d[2] <= b->r * b->r;
  }
  return b->c[0] * x[0] + b->c[1] * x[1] + b->c[2] * x[2] >= b->r;
}

/* Entry parameter of x + t e into body b for t in (0, 1+eps]; returns -1 if
 * none.  x is outside b. */
static double entry(const ctx_t* g, const geom_body* b, const double x[3], const int e[3]) {
  if (b->kind == 0) {
    double d[3];
    ball_disp(g, b, x, d);
    const double A = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
    const double B = d[0] * e[0] + d[1] * e[1] + d[2] * e[2];
    const double C = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] - b->r * b->r;
    const double disc = B * B - A * C;
    if (disc < 0.0) return -1.0;
    /* smaller root, written to avoid cancellation when B < 0 */
    const double sq = sqrt(disc);
    double t;
    if (B <= 0.0)
      t = C / (-B + sq);
    else
      t = (-B - sq) / A;
    if (t <= 0.0) return -1.0;
    return t;
  }
  const double nd = b->c[0] * e[0] + b->c[1] * e[1] + b->c[2] * e[2];
  if (nd <= 0.0) return -1.0;
  const double t = (b->r - (b->c[0] * x[0] + b->c[1] * x[1] + b->c[2] * x[2])) / nd;
  return t > 0.0 ? t : -1.0;
}

static int wrap_idx(int v, int L) { return ((v % L) + L) % L; }

static int build_grid(ctx_t* g) {
  g->cs = 16;
  g->gx = (g->nx + g->cs - 1) / g->cs;
  g->gy = (g->ny + g->cs - 1) / g->cs;
  g->gz = (g->nz + g->cs - 1) / g->cs;
  const int64_t ncell = (int64_t)g->gx * g->gy * g->gz;
  g->cell_start = (int32_t*)calloc(ncell + 1, sizeof(int32_t));
  g->planes = (int32_t*)malloc(sizeof(int32_t) * (g->nb + 1));
  if (!g->cell_start || !g->planes) return -1;
  g->nplanes = 0;
  /* two passes: count then fill */
  for (int pass = 0; pass < 2; ++pass) {
    int32_t* fill = NULL;
    if (pass == 1) {
      for (int64_t k = 0; k < ncell; ++k) g->cell_start[k + 1] += g->cell_start[k];
      g->cell_items = (int32_t*)malloc(sizeof(int32_t) * (g->cell_start[ncell] + 1));
      fill = (int32_t*)calloc(ncell, sizeof(int32_t));
      if (!g->cell_items || !fill) return -1;
    }
    for (int bi = 0; bi < g->nb; ++bi) {
      const geom_body* b = &g->bodies[bi];
      if (b->kind != 0) {
        if (pass == 0) g->planes[g->nplanes++] = bi;
        continue;
      }
      /* cells touched by the ball's box (grown by 2), per axis, found by
       * wrapping lattice coordinates first so that lattice sizes that are
       * not multiples of the cell size wrap correctly */
      const int L[3] = {g->nx, g->ny, g->nz};
      int cells[3][64];
      int nc[3];
      for (int a = 0; a < 3; ++a) {
        int l = (int)floor(b->c[a] - b->r - 2.0), h = (int)ceil(b->c[a] + b->r + 2.0);
        if (!g->periodic[a]) {
          if (l < 0) l = 0;
          if (h > L[a] - 1) h = L[a] - 1;
        } else if (h - l + 1 > L[a]) {
          l = 0;
          h = L[a] - 1;
        }
        nc[a] = 0;
        for (int v = l; v <= h; ++v) {
          const int c = wrap_idx(v, L[a]) / g->cs;
          int seen = 0;
          for (int k = 0; k < nc[a]; ++k) seen |= cells[a][k] == c;
          if (!seen && nc[a] < 64) cells[a][nc[a]++] = c;
        }
      }
      for (int kz = 0; kz < nc[2]; ++kz)
        for (int ky = 0; ky < nc[1]; ++ky)
          for (int kx = 0; kx < nc[0]; ++kx) {
            const int64_t k = cells[0][kx] + (int64_t)g->gx * (cells[1][ky] + (int64_t)g->gy * cells[2][kz]);
            if (pass == 0)
              g->cell_start[k + 1]++;
            else
              g->cell_items[g->cell_start[k] + fill[k]++] = bi;
          }
    }
    if (pass == 1) free(fill);
  }
  return 0;
}

static void free_grid(ctx_t* g) {
  free(g->cell_start);
  free(g->cell_items);
  free(g->planes);
}

static int setup(ctx_t* g, int stencil, int nx, int ny, int nz, const int32_t* periodic, const geom_body* bodies,
                 int nb) {
  memset(g, 0, sizeof *g);
  g->nx = nx; g->ny = ny; g->nz = nz;
  for (int a = 0; a < 3; ++a) g->periodic[a] = periodic[a];
  g->Q = stencil == 0 ? 9 : 19;
  g->e = stencil == 0 ? E2 : E3;
  g->bodies = bodies;
  g->nb = nb;
  return build_grid(g);
}

/* Rasterise all bodies into mask (1 = solid).  Returns the number of solid
 * nodes, or -1 on allocation failure. */
int64_t geom_mask(int stencil, int nx, int ny, int nz, const int32_t* periodic, const geom_body* bodies, int nb,
                  uint8_t* mask) {
  ctx_t g;
  if (setup(&g, stencil, nx, ny, nz, periodic, bodies, nb) != 0) return -1;
  const int64_t N = (int64_t)nx * ny * nz;
  memset(mask, 0, (size_t)N);
  const int L[3] = {nx, ny, nz};
  for (int bi = 0; bi < nb; ++bi) {
    const geom_body* b = &bodies[bi];
    if (b->kind != 0) {
      for (int64_t n = 0; n < N; ++n) {
        const double x[3] = {(double)(n % nx), (double)((n / nx) % ny), (double)(n / ((int64_t)nx * ny))};
        if (inside(&g, b, x)) mask[n] = 1;
      }
      continue;
    }
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
      lo[a] = (int)floor(b->c[a] - b->r) - 1;
      hi[a] = (int)ceil(b->c[a] + b->r) + 1;
      if (!periodic[a]) {
        if (lo[a] < 0) lo[a] = 0;
        if (hi[a] > L[a] - 1) hi[a] = L[a] - 1;
      } else if (hi[a] - lo[a] + 1 > L[a]) {
        lo[a] = 0;
        hi[a] = L[a] - 1;
      }
    }
    for (int z = lo[2]; z <= hi[2]; ++z)
      for (int y = lo[1]; y <= hi[1]; ++y)
        for (int x = lo[0]; x <= hi[0]; ++x) {
          const int wx = wrap_idx(x, nx), wy = wrap_idx(y, ny), wz = wrap_idx(z, nz);
          const double p[3] = {(double)wx, (double)wy, (double)wz};
          if (inside(&g, b, p)) mask[wx + (int64_t)nx * (wy + (int64_t)ny * wz)] = 1;
        }
  }
  free_grid(&g);
  int64_t ns = 0;
  for (int64_t n = 0; n < N; ++n) ns += mask[n];
  return ns;
}

/* Add balls from (centres, radii) in order until the solid node count reaches
 * target_solid.  mask must hold the current solid mask.  Returns the number
 * of balls used (<= count) and updates *solid_count. */
int64_t geom_pack_add(int nx, int ny, int nz, const int32_t* periodic, const double* centres, const double* radii,
                      int64_t count, int64_t target_solid, uint8_t* mask, int64_t* solid_count) {
  const int L[3] = {nx, ny, nz};
  int64_t ns = *solid_count;
  int64_t k = 0;
  for (; k < count && ns < target_solid; ++k) {
    const double* c = centres + 3 * k;
    const double r = radii[k];
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
      lo[a] = (int)floor(c[a] - r) - 1;
      hi[a] = (int)ceil(c[a] + r) + 1;
      if (!periodic[a]) {
        if (lo[a] < 0) lo[a] = 0;
        if (hi[a] > L[a] - 1) hi[a] = L[a] - 1;
      }
    }
    for (int z = lo[2]; z <= hi[2]; ++z)
      for (int y = lo[1]; y <= hi[1]; ++y)
        for (int x = lo[0]; x <= hi[0]; ++x) {
          const int wx = wrap_idx(x, nx), wy = wrap_idx(y, ny), wz = wrap_idx(z, nz);
          double d[3] = {wx - c[0], wy - c[1], wz - c[2]};
          for (int a = 0; a < 3; ++a) d[a] = min_image(d[a], L[a], periodic[a]);
          if (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] <= r * r) {
            uint8_t* m = &mask[wx + (int64_t)nx * (wy + (int64_t)ny * wz)];
            if (!*m) {
              *m = 1;
              ++ns;
            }
          }
        }
  }
  *solid_count = ns;
  return k;
}

/* Links of one lattice row (y, z): count only (out == NULL) or fill.
 * Returns the count, or a negative error code with *err_node set. */
static int64_t row_links(const ctx_t* g, const uint8_t* mask, int open_lo, int open_hi, int64_t y, int64_t z,
                         geom_link* out, int64_t* err_node) {
  const int nx = g->nx, ny = g->ny, nz = g->nz;
  const int L[3] = {nx, ny, nz};
  int64_t count = 0;
  for (int x = 0; x < nx; ++x) {
    const int64_t n = x + (int64_t)nx * (y + (int64_t)ny * z);
    if (mask[n]) continue;
    if ((open_lo && x == 0) || (open_hi && x == nx - 1)) continue;
    const int xi[3] = {x, (int)y, (int)z};
    const double xf[3] = {(double)x, (double)y, (double)z};
    for (int d = 1; d < g->Q; ++d) {
      int s[3];
      int outside = 0;
      for (int a = 0; a < 3; ++a) {
        s[a] = xi[a] + g->e[d][a];
        if (s[a] < 0 || s[a] >= L[a]) {
          if (!g->periodic[a]) outside = 1;
          s[a] = wrap_idx(s[a], L[a]);
        }
      }
      if (outside) {
        /* allowed only when the neighbour face is an open boundary column */
        const int through_x_open = (xi[0] + g->e[d][0] < 0 && open_lo) || (xi[0] + g->e[d][0] >= nx && open_hi);
        if (through_x_open) continue;
        *err_node = n;
        return -2;
      }
      const int64_t sn = s[0] + (int64_t)nx * (s[1] + (int64_t)ny * s[2]);
      if (!mask[sn]) continue;
      if (out) {
        /* first wall crossing along x_f + t e_d */
        double best = 2.0;
        int bbest = -1;
        const int cx = s[0] / g->cs, cy = s[1] / g->cs, cz = s[2] / g->cs;
        const int64_t cell = cx + (int64_t)g->gx * (cy + (int64_t)g->gy * cz);
        for (int32_t k = g->cell_start[cell]; k < g->cell_start[cell + 1]; ++k) {
          const int bi = g->cell_items[k];
          const double t = entry(g, &g->bodies[bi], xf, g->e[d]);
          if (t > 0.0 && t < best) {
            best = t;
            bbest = bi;
          }
        }
        for (int k = 0; k < g->nplanes; ++k) {
          const int bi = g->planes[k];
          const double t = entry(g, &g->bodies[bi], xf, g->e[d]);
          if (t > 0.0 && t < best) {
            best = t;
            bbest = bi;
          }
        }
        if (bbest < 0 || best > 1.0 + 1e-9) {
          *err_node = n;
          return -3;
        }
        if (best > 1.0) best = 1.0;
        geom_link* lk = &out[count];
        const geom_body* b = &g->bodies[bbest];
        lk->node = n;
        lk->dir = d;
        lk->bc = (int16_t)b->bc;
        lk->body = (int16_t)b->force_id;
        lk->q = best;
        /* wall velocity at x_w = x_f + q e: U + omega x (x_w - c) */
        double uw[3] = {b->vel[0], b->vel[1], b->vel[2]};
        if (b->kind == 0) {
          const double xw[3] = {xf[0] + best * g->e[d][0], xf[1] + best * g->e[d][1], xf[2] + best * g->e[d][2]};
          double r[3];
          ball_disp(g, b, xw, r);
          uw[0] += b->omega[1] * r[2] - b->omega[2] * r[1];
          uw[1] += b->omega[2] * r[0] - b->omega[0] * r[2];
          uw[2] += b->omega[0] * r[1] - b->omega[1] * r[0];
        }
        lk->uw[0] = uw[0];
        lk->uw[1] = uw[1];
        lk->uw[2] = uw[2];
      }
      ++count;
    }
  }
  return count;
}

/* Cut links of all fluid nodes, sorted by (node, dir).  Fluid nodes in the
 * columns x = 0 (if open_lo) and x = nx-1 (if open_hi) are open-boundary nodes
 * and get no links.  out may be NULL to count only.  Returns the link count,
 * or a negative error code:
 *   -1 allocation failure, -2 a fluid node's neighbour leaves the lattice
 *   through a non-periodic face, -3 a solid neighbour has no wall crossing.
 * err_node receives the offending node (the smallest one) for -2/-3.
 * Rows are processed in parallel (OpenMP). */
int64_t geom_links(int stencil, int nx, int ny, int nz, const int32_t* periodic, const geom_body* bodies, int nb,
                   const uint8_t* mask, int open_lo, int open_hi, geom_link* out, int64_t* err_node) {
  ctx_t g;
  if (setup(&g, stencil, nx, ny, nz, periodic, bodies, nb) != 0) return -1;
  const int64_t rows = (int64_t)ny * nz;
  int64_t* start = (int64_t*)calloc(rows + 1, sizeof(int64_t));
  if (!start) {
    free_grid(&g);
    return -1;
  }
  int64_t err = 0, bad = INT64_MAX;
  /* pass 1: counts per row (no intersection work) */
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t r = 0; r < rows; ++r) {
    int64_t en = 0;
    const int64_t c = row_links(&g, mask, open_lo, open_hi, r % ny, r / ny, NULL, &en);
    if (c < 0) {
#pragma omp critical
      {
        if (en < bad) {
          bad = en;
          err = c;
        }
      }
    } else {
      start[r + 1] = c;
    }
  }
  if (err == 0) {
    for (int64_t r = 0; r < rows; ++r) start[r + 1] += start[r];
    if (out) {
      /* pass 2: fill each row's slice */
#pragma omp parallel for schedule(dynamic, 16)
      for (int64_t r = 0; r < rows; ++r) {
        int64_t en = 0;
        const int64_t c = row_links(&g, mask, open_lo, open_hi, r % ny, r / ny, out + start[r], &en);
        if (c < 0) {
#pragma omp critical
          {
            if (en < bad) {
              bad = en;
              err = c;
            }
          }
        }
      }
    }
  }
  const int64_t total = start[rows];
  free(start);
  free_grid(&g);
  if (err != 0) {
    if (err_node) *err_node = bad;
    return err;
  }
  return total;
}
