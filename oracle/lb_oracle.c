/*
 * FP64 CPU oracle for the D2Q9 free-energy multiple-relaxation-time lattice
 * Boltzmann method of Pooley, Kusumaatmaja & Yeomans, "Modelling capillary
 * filling dynamics using lattice Boltzmann simulations".
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark use this file.  It shares no code with the CUDA library: it
 * keeps its own velocity, weight and matrix tables, its own geometry array, its
 * own equilibrium and collision code.
 *
 * It is written to be checked against the paper by eye, not to be fast:
 *   - populations are stored per node (f[node*9 + i]) in double precision;
 *   - the collision is the full matrix product  f* = f - M^-1 S M (f - f^eq)
 *     of Eq. (latbolt) with M as printed in Appendix A and M^-1 obtained by
 *     Gauss-Jordan elimination at start-up;
 *   - the equilibria are Eq. (equilibrium), Eq. (feq0) and the g^eq formula of
 *     Appendix A, evaluated term by term with the weight tables of Appendix A;
 *   - the gradient and Laplacian are the stencils of Eq. (best), applied as
 *     3x3 weight tables;
 *   - streaming pushes every post-collision population to r + e_i in a second
 *     array, then the wall rule of Sec. 2.2 is applied (bounce-back, then
 *     boundary nodes set to rest).
 *
 * Readings of points the paper leaves open (each one is also listed in the
 * design notes):
 *   lambda  : lambda = lambda_scale * nu_local (Galilean-invariance correction).
 *   binary f^eq : Eq. (equilibrium) with p0 - kappa phi lap(phi) in place of
 *             p0 - kappa rho lap(rho) and the kappa gradient terms in phi (the
 *             binary pressure tensor of Sec. 3.1); the lambda term keeps rho.
 *   d_y     : the y-derivative stencil is the transpose of the printed d_x.
 *   nu(phi) : (phi + 1)/2 is clamped to [0, 1] so nu stays between the bulk
 *             values nu_g and nu_l.
 *   walls   : a population whose push target is solid returns to its own node
 *             in the opposite direction; afterwards every boundary node (a fluid
 *             node with at least one solid node among its 8 neighbours) has its
 *             momentum removed with f_i -= w_i e_i . j (density unchanged).  The
 *             g populations get the bounce-back only.  The initial state built
 *             from macroscopic fields obeys the same rest rule at boundary nodes.
 *   wetting : in the stencils a solid neighbour s = r + d of a fluid node r takes
 *             a ghost value: d = (dx, 0) -> v(r - (dx, 0)) (neutral mirror);
 *             d = (0, dy) -> v(r - (0, dy)) - 2h; diagonal -> v(r + (dx, -dy)) - 2h
 *             if that node is fluid, else v(r + (-dx, dy)).  h is the prescribed
 *             normal gradient d_n rho|_b (liquid-gas) or d_n phi|_b (binary); the
 *             binary rho field uses h = 0.
 *   l(t)    : distance from the tube inlet x0 to the first sign change, scanning
 *             from x0, of phi (binary) or rho - (rho_l + rho_g)/2 (liquid-gas)
 *             along the tube's middle row (mean of the two middle rows when H is
 *             even), linearly interpolated.
 *   table   : App. A keeps collision matrices for ~10^4 viscosities and uses the
 *             closest one; with nu_table = K >= 2 the K viscosities are spaced
 *             evenly over [nu_g, nu_l] and the nearest is used (0: exact nu).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- tables -- */

/* Lattice velocities, Sec. 2.1: e0 = 0, e1,2 = (+-1, 0), e3,4 = (0, +-1),
 * e5,6 = +-(1, 1), e7,8 = +-(-1, 1); the diagonal signs follow the jx and jy
 * rows of M in Appendix A. */
static const int EX[9] = {0, 1, -1, 0, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 0, 1, -1, 1, -1, 1, -1};
static const int OPP[9] = {0, 2, 1, 4, 3, 6, 5, 8, 7};

/* Appendix A weights: w_{1-4} = 1/3, w_{5-8} = 1/12 and the gradient weights. */
static const double WI[9] = {0.0, 1.0 / 3, 1.0 / 3, 1.0 / 3, 1.0 / 3,
                             1.0 / 12, 1.0 / 12, 1.0 / 12, 1.0 / 12};
static const double WXX[9] = {0.0, 1.0 / 3, 1.0 / 3, -1.0 / 6, -1.0 / 6,
                              -1.0 / 24, -1.0 / 24, -1.0 / 24, -1.0 / 24};
static const double WYY[9] = {0.0, -1.0 / 6, -1.0 / 6, 1.0 / 3, 1.0 / 3,
                              -1.0 / 24, -1.0 / 24, -1.0 / 24, -1.0 / 24};
static const double WXY[9] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.25, 0.25, -0.25, -0.25};

/* Change-of-basis matrix M, Appendix A, row by row as printed. */
static const double MP[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},
    {-4, -1, -1, -1, -1, 2, 2, 2, 2},
    {4, -2, -2, -2, -2, 1, 1, 1, 1},
    {0, 1, -1, 0, 0, 1, -1, -1, 1},
    {0, -2, 2, 0, 0, 1, -1, -1, 1},
    {0, 0, 0, 1, -1, 1, -1, 1, -1},
    {0, 0, 0, -2, 2, 1, -1, 1, -1},
    {0, 1, 1, -1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, 1, -1, -1},
};

/* Stencils of Eq. (best) as weight tables T[jy][jx], jy = dy + 1, jx = dx + 1.
 * The printed d_x is symmetric in y; d_y is its transpose. */
static const double SDX[3][3] = {{-1.0 / 12, 0.0, 1.0 / 12},
                                 {-4.0 / 12, 0.0, 4.0 / 12},
                                 {-1.0 / 12, 0.0, 1.0 / 12}};
static const double SDY[3][3] = {{-1.0 / 12, -4.0 / 12, -1.0 / 12},
                                 {0.0, 0.0, 0.0},
                                 {1.0 / 12, 4.0 / 12, 1.0 / 12}};
static const double SLAP[3][3] = {{1.0 / 6, 4.0 / 6, 1.0 / 6},
                                  {4.0 / 6, -20.0 / 6, 4.0 / 6},
                                  {1.0 / 6, 4.0 / 6, 1.0 / 6}};

/* ------------------------------------------------------------- structures -- */

typedef struct {
  int nx, ny, model; /* model 0 = liquid-gas (van der Waals), 1 = binary */
  int tube_x0, tube_len, tube_y0, tube_h;
  double wall_grad;
  double kappa, a, b, T;
  double A, M, nu_l, nu_g;
  double nu, lambda_scale;
  double rho_l, rho_g;
  int nu_table; /* 0: exact nu; K >= 2: nearest of K viscosities evenly spaced over [nu_g, nu_l] */
} orc_params;

typedef struct {
  orc_params p;
  int n;
  unsigned char *solid, *bnd;
  double *f, *g, *ft, *gt;                 /* per node, 9 each */
  double *rho, *ux, *uy, *phi;             /* macroscopic fields */
  double *rdx, *rdy, *rlap;                /* stencils of rho */
  double *pdx, *pdy, *plap;                /* stencils of phi */
  double Mm[9][9], Mi[9][9];
  long t;
} orc_state;

enum { ORC_OK = 0, ORC_ERR_ARG = -1, ORC_ERR_GEOM = -2, ORC_ERR_MEM = -3, ORC_ERR_MATH = -4 };

static int wrap(int v, int n) {
  int r = v % n;
  return r < 0 ? r + n : r;
}

static int is_solid_geom(const orc_params *p, int x, int y) {
  if (p->tube_len <= 0) return 0;
  int in_tube = wrap(x - p->tube_x0, p->nx) < p->tube_len;
  int in_band = wrap(y - p->tube_y0, p->ny) < p->tube_h;
  return in_tube && !in_band;
}

/* ----------------------------------------------------------- linear algebra */

/* Gauss-Jordan inverse with partial pivoting. */
static int invert9(const double a_in[9][9], double inv[9][9]) {
  double a[9][18];
  for (int r = 0; r < 9; ++r)
    for (int c = 0; c < 18; ++c) a[r][c] = c < 9 ? a_in[r][c] : (c - 9 == r ? 1.0 : 0.0);
  for (int c = 0; c < 9; ++c) {
    int piv = c;
    for (int r = c + 1; r < 9; ++r)
      if (fabs(a[r][c]) > fabs(a[piv][c])) piv = r;
    if (fabs(a[piv][c]) < 1e-12) return ORC_ERR_MATH;
    if (piv != c)
      for (int k = 0; k < 18; ++k) {
        double t = a[c][k];
        a[c][k] = a[piv][k];
        a[piv][k] = t;
      }
    double d = a[c][c];
    for (int k = 0; k < 18; ++k) a[c][k] /= d;
    for (int r = 0; r < 9; ++r) {
      if (r == c) continue;
      double m = a[r][c];
      if (m == 0.0) continue;
      for (int k = 0; k < 18; ++k) a[r][k] -= m * a[c][k];
    }
  }
  for (int r = 0; r < 9; ++r)
    for (int c = 0; c < 9; ++c) inv[r][c] = a[r][c + 9];
  return ORC_OK;
}

void orc_matrices(double *M, double *Minv) {
  double inv[9][9];
  invert9(MP, inv);
  for (int r = 0; r < 9; ++r)
    for (int c = 0; c < 9; ++c) {
      M[r * 9 + c] = MP[r][c];
      Minv[r * 9 + c] = inv[r][c];
    }
}

/* --------------------------------------------------- equilibria, collision -- */

/* Eq. (equilibrium) and Eq. (feq0), c = dt = dx = 1.
 *   P0     : the scalar p0 - kappa psi lap(psi)
 *   gpx,gpy: gradient of psi in the kappa terms (psi = rho or phi)
 *   grx,gry: gradient of rho in the lambda term. */
void orc_feq(double rho, double ux, double uy, double P0, double kappa,
             double gpx, double gpy, double grx, double gry, double lambda,
             double out[9]) {
  const double u[2] = {ux, uy};
  const double dr[2] = {grx, gry};
  const double udr = ux * grx + uy * gry;
  double Tm[2][2];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      Tm[a][b] = rho * u[a] * u[b] +
                 lambda * (u[a] * dr[b] + u[b] * dr[a] + (a == b ? udr : 0.0));
  double sum = 0.0;
  for (int i = 1; i < 9; ++i) {
    const double e[2] = {(double)EX[i], (double)EY[i]};
    double s = P0;
    for (int a = 0; a < 2; ++a) s += e[a] * rho * u[a];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b)
        s += 1.5 * (e[a] * e[b] - (a == b ? 1.0 / 3.0 : 0.0)) * Tm[a][b];
    out[i] = WI[i] * s +
             kappa * (WXX[i] * gpx * gpx + WYY[i] * gpy * gpy + WXY[i] * gpx * gpy);
    sum += out[i];
  }
  out[0] = rho - sum;
}

/* g^eq of Appendix A with dt = 1. */
void orc_geq(double phi, double ux, double uy, double mu, double Mob, double out[9]) {
  const double u[2] = {ux, uy};
  double sum = 0.0;
  for (int i = 1; i < 9; ++i) {
    const double e[2] = {(double)EX[i], (double)EY[i]};
    double s = 2.0 * Mob * mu;
    for (int a = 0; a < 2; ++a) s += e[a] * phi * u[a];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b)
        s += 1.5 * (e[a] * e[b] - (a == b ? 1.0 / 3.0 : 0.0)) * phi * u[a] * u[b];
    out[i] = WI[i] * s;
    sum += out[i];
  }
  out[0] = phi - sum;
}

/* Eq. (latbolt) right-hand side: f - M^-1 S M (f - f^eq), S = diag(0,1,1,0,1,0,1,w,w). */
static void collide_full(const double Mm[9][9], const double Mi[9][9], const double *f,
                         const double *feq, double omega, double *out) {
  const double S[9] = {0.0, 1.0, 1.0, 0.0, 1.0, 0.0, 1.0, omega, omega};
  double d[9], m[9], c[9];
  for (int i = 0; i < 9; ++i) d[i] = f[i] - feq[i];
  for (int k = 0; k < 9; ++k) {
    double s = 0.0;
    for (int i = 0; i < 9; ++i) s += Mm[k][i] * d[i];
    m[k] = S[k] * s;
  }
  for (int i = 0; i < 9; ++i) {
    double s = 0.0;
    for (int k = 0; k < 9; ++k) s += Mi[i][k] * m[k];
    c[i] = s;
  }
  for (int i = 0; i < 9; ++i) out[i] = f[i] - c[i];
}

void orc_collide(const double *f, const double *feq, double omega, double *out) {
  double inv[9][9];
  invert9(MP, inv);
  collide_full(MP, inv, f, feq, omega, out);
}

/* ------------------------------------------------------------- geometry ---- */

static int node_solid(const orc_state *s, int x, int y) {
  return s->solid[wrap(y, s->p.ny) * s->p.nx + wrap(x, s->p.nx)];
}

/* Gather the 3x3 neighbourhood of field v around fluid node (x, y), replacing
 * solid neighbours by their ghost values.  Returns ORC_ERR_GEOM when a ghost has
 * no fluid mirror node. */
static int neighbourhood(const orc_state *s, const double *v, double h, int x, int y,
                         double out[3][3]) {
  const int nx = s->p.nx;
  int sol[3][3];
  double raw[3][3];
  for (int jy = 0; jy < 3; ++jy)
    for (int jx = 0; jx < 3; ++jx) {
      int xx = wrap(x + jx - 1, nx), yy = wrap(y + jy - 1, s->p.ny);
      sol[jy][jx] = s->solid[yy * nx + xx];
      raw[jy][jx] = sol[jy][jx] ? 0.0 : v[yy * nx + xx];
    }
  for (int jy = 0; jy < 3; ++jy)
    for (int jx = 0; jx < 3; ++jx) {
      out[jy][jx] = raw[jy][jx];
      if (!sol[jy][jx]) continue;
      const int dx = jx - 1, dy = jy - 1;
      if (dy == 0) { /* x-facing end face of a wall block: neutral mirror */
        if (sol[1][1 - dx]) return ORC_ERR_GEOM;
        out[jy][jx] = raw[1][1 - dx];
      } else if (dx == 0) { /* y-facing wall: mirror with the wetting gradient */
        if (sol[1 - dy][1]) return ORC_ERR_GEOM;
        out[jy][jx] = raw[1 - dy][1] - 2.0 * h;
      } else if (!sol[1 - dy][1 + dx]) { /* diagonal: mirror in y if possible */
        out[jy][jx] = raw[1 - dy][1 + dx] - 2.0 * h;
      } else if (!sol[1 + dy][1 - dx]) { /* else mirror in x, neutral */
        out[jy][jx] = raw[1 + dy][1 - dx];
      } else {
        return ORC_ERR_GEOM;
      }
    }
  return ORC_OK;
}

static double apply3(const double T[3][3], const double v[3][3]) {
  double s = 0.0;
  for (int jy = 0; jy < 3; ++jy)
    for (int jx = 0; jx < 3; ++jx) s += T[jy][jx] * v[jy][jx];
  return s;
}

static int stencils(const orc_state *s, const double *v, double h, double *dx, double *dy,
                    double *lap) {
  const int nx = s->p.nx, ny = s->p.ny;
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const int k = y * nx + x;
      if (s->solid[k]) {
        dx[k] = dy[k] = lap[k] = 0.0;
        continue;
      }
      double nb[3][3];
      int rc = neighbourhood(s, v, h, x, y, nb);
      if (rc) return rc;
      dx[k] = apply3(SDX, nb);
      dy[k] = apply3(SDY, nb);
      lap[k] = apply3(SLAP, nb);
    }
  return ORC_OK;
}

/* ------------------------------------------------------------------ api ---- */

void orc_destroy(void *h) {
  orc_state *s = (orc_state *)h;
  if (!s) return;
  free(s->solid); free(s->bnd);
  free(s->f); free(s->g); free(s->ft); free(s->gt);
  free(s->rho); free(s->ux); free(s->uy); free(s->phi);
  free(s->rdx); free(s->rdy); free(s->rlap);
  free(s->pdx); free(s->pdy); free(s->plap);
  free(s);
}

int orc_create(const orc_params *p, void **out) {
  *out = NULL;
  if (p->nx < 3 || p->ny < 3 || (p->model != 0 && p->model != 1)) return ORC_ERR_ARG;
  if (p->tube_len < 0 || p->tube_len > p->nx) return ORC_ERR_ARG;
  if (p->tube_len > 0 && (p->tube_h < 2 || p->tube_h >= p->ny)) return ORC_ERR_ARG;
  if (p->tube_len > 0 && p->tube_len < p->nx && p->nx - p->tube_len < 2) return ORC_ERR_ARG;
  if (p->nu_table < 0 || p->nu_table == 1) return ORC_ERR_ARG;
  orc_state *s = (orc_state *)calloc(1, sizeof(orc_state));
  if (!s) return ORC_ERR_MEM;
  s->p = *p;
  s->n = p->nx * p->ny;
  const size_t n = (size_t)s->n;
  s->solid = (unsigned char *)calloc(n, 1);
  s->bnd = (unsigned char *)calloc(n, 1);
  s->f = (double *)calloc(9 * n, sizeof(double));
  s->g = (double *)calloc(9 * n, sizeof(double));
  s->ft = (double *)calloc(9 * n, sizeof(double));
  s->gt = (double *)calloc(9 * n, sizeof(double));
  double **fl[] = {&s->rho, &s->ux, &s->uy, &s->phi, &s->rdx, &s->rdy,
                   &s->rlap, &s->pdx, &s->pdy, &s->plap};
  for (size_t k = 0; k < sizeof(fl) / sizeof(fl[0]); ++k) *fl[k] = (double *)calloc(n, sizeof(double));
  if (!s->solid || !s->bnd || !s->f || !s->g || !s->ft || !s->gt || !s->plap) {
    orc_destroy(s);
    return ORC_ERR_MEM;
  }
  for (int y = 0; y < p->ny; ++y)
    for (int x = 0; x < p->nx; ++x) s->solid[y * p->nx + x] = (unsigned char)is_solid_geom(p, x, y);
  for (int y = 0; y < p->ny; ++y)
    for (int x = 0; x < p->nx; ++x) {
      const int k = y * p->nx + x;
      if (s->solid[k]) continue;
      for (int i = 1; i < 9; ++i)
        if (node_solid(s, x + EX[i], y + EY[i])) s->bnd[k] = 1;
    }
  for (int r = 0; r < 9; ++r)
    for (int c = 0; c < 9; ++c) s->Mm[r][c] = MP[r][c];
  if (invert9(MP, s->Mi)) {
    orc_destroy(s);
    return ORC_ERR_MATH;
  }
  /* validate that every ghost has a mirror node */
  int rc = stencils(s, s->rho, 0.0, s->rdx, s->rdy, s->rlap);
  if (rc) {
    orc_destroy(s);
    return rc;
  }
  *out = s;
  return ORC_OK;
}

/* Per-node thermodynamics: local nu (Eq. nu, clamped), omega = 2/(6 nu + 1). */
static double local_nu(const orc_params *p, double phi) {
  if (p->model == 0) return p->nu;
  double c = 0.5 * (phi + 1.0);
  if (c < 0.0) c = 0.0;
  if (c > 1.0) c = 1.0;
  /* App. A: a table of viscosities, the closest entry is used */
  if (p->nu_table >= 2) c = nearbyint(c * (p->nu_table - 1)) / (p->nu_table - 1);
  return p->nu_g + c * (p->nu_l - p->nu_g);
}

static void moments(orc_state *s) {
  for (int k = 0; k < s->n; ++k) {
    if (s->solid[k]) {
      s->rho[k] = s->ux[k] = s->uy[k] = s->phi[k] = 0.0;
      continue;
    }
    const double *fk = s->f + 9 * (size_t)k, *gk = s->g + 9 * (size_t)k;
    double r = 0.0, jx = 0.0, jy = 0.0, ph = 0.0;
    for (int i = 0; i < 9; ++i) {
      r += fk[i];
      jx += fk[i] * EX[i];
      jy += fk[i] * EY[i];
      ph += gk[i];
    }
    s->rho[k] = r;
    s->ux[k] = jx / r;
    s->uy[k] = jy / r;
    s->phi[k] = s->p.model == 1 ? ph : 0.0;
  }
}

static int all_stencils(orc_state *s) {
  const orc_params *p = &s->p;
  if (p->model == 0) return stencils(s, s->rho, p->wall_grad, s->rdx, s->rdy, s->rlap);
  int rc = stencils(s, s->rho, 0.0, s->rdx, s->rdy, s->rlap);
  if (rc) return rc;
  return stencils(s, s->phi, p->wall_grad, s->pdx, s->pdy, s->plap);
}

/* Equilibria at node k from the current fields and stencils. */
static void node_equilibria(const orc_state *s, int k, double feq[9], double geq[9], double *omega) {
  const orc_params *p = &s->p;
  const double r = s->rho[k], ux = s->ux[k], uy = s->uy[k];
  if (p->model == 0) {
    const double p0 = r * p->T / (1.0 - p->b * r) - p->a * r * r;           /* Sec. 2 */
    const double P0 = p0 - p->kappa * r * s->rlap[k];
    const double nu = local_nu(p, 0.0);
    orc_feq(r, ux, uy, P0, p->kappa, s->rdx[k], s->rdy[k], s->rdx[k], s->rdy[k],
            p->lambda_scale * nu, feq);
    *omega = 2.0 / (6.0 * nu + 1.0);                                         /* App. A */
  } else {
    const double ph = s->phi[k];
    const double p0 = r / 3.0 + p->A * (-0.5 * ph * ph + 0.75 * ph * ph * ph * ph); /* Sec. 3.1 */
    const double P0 = p0 - p->kappa * ph * s->plap[k];
    const double mu = p->A * (-ph + ph * ph * ph) - p->kappa * s->plap[k];  /* Eq. chempot */
    const double nu = local_nu(p, ph);
    orc_feq(r, ux, uy, P0, p->kappa, s->pdx[k], s->pdy[k], s->rdx[k], s->rdy[k],
            p->lambda_scale * nu, feq);
    orc_geq(ph, ux, uy, mu, p->M, geq);
    *omega = 2.0 / (6.0 * nu + 1.0);
  }
}

/* Sec. 2.2: boundary nodes set to rest after streaming, keeping the density. */
static void rest_node(double *fk) {
  double jx = 0.0, jy = 0.0;
  for (int i = 0; i < 9; ++i) {
    jx += fk[i] * EX[i];
    jy += fk[i] * EY[i];
  }
  for (int i = 1; i < 9; ++i) fk[i] -= WI[i] * (EX[i] * jx + EY[i] * jy);
}

int orc_init_fields(void *h, const double *rho, const double *ux, const double *uy,
                    const double *phi) {
  orc_state *s = (orc_state *)h;
  for (int k = 0; k < s->n; ++k) {
    const int sol = s->solid[k];
    s->rho[k] = sol ? 0.0 : rho[k];
    s->ux[k] = sol ? 0.0 : ux[k];
    s->uy[k] = sol ? 0.0 : uy[k];
    s->phi[k] = (sol || s->p.model == 0 || !phi) ? 0.0 : phi[k];
  }
  int rc = all_stencils(s);
  if (rc) return rc;
  for (int k = 0; k < s->n; ++k) {
    double *fk = s->f + 9 * (size_t)k, *gk = s->g + 9 * (size_t)k;
    if (s->solid[k]) {
      memset(fk, 0, 9 * sizeof(double));
      memset(gk, 0, 9 * sizeof(double));
      continue;
    }
    double om;
    double geq[9] = {0};
    node_equilibria(s, k, fk, geq, &om);
    memcpy(gk, geq, sizeof geq);
    if (s->bnd[k]) rest_node(fk); /* the initial state obeys the wall rule too */
  }
  s->t = 0;
  return ORC_OK;
}

int orc_step(void *h, long nsteps) {
  orc_state *s = (orc_state *)h;
  const orc_params *p = &s->p;
  const int nx = p->nx, ny = p->ny;
  for (long t = 0; t < nsteps; ++t) {
    moments(s);
    int rc = all_stencils(s);
    if (rc) return rc;
    memset(s->ft, 0, 9 * (size_t)s->n * sizeof(double));
    memset(s->gt, 0, 9 * (size_t)s->n * sizeof(double));
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const int k = y * nx + x;
        if (s->solid[k]) continue;
        double feq[9], geq[9] = {0}, fs[9], om;
        node_equilibria(s, k, feq, geq, &om);
        collide_full(s->Mm, s->Mi, s->f + 9 * (size_t)k, feq, om, fs); /* Eq. latbolt */
        for (int i = 0; i < 9; ++i) {                                  /* streaming */
          const int xd = wrap(x + EX[i], nx), yd = wrap(y + EY[i], ny);
          const int kd = yd * nx + xd;
          if (s->solid[kd]) {
            s->ft[9 * (size_t)k + OPP[i]] = fs[i];   /* bounce-back */
            s->gt[9 * (size_t)k + OPP[i]] = geq[i];
          } else {
            s->ft[9 * (size_t)kd + i] = fs[i];
            s->gt[9 * (size_t)kd + i] = geq[i];     /* Eq. latbolt2: g* = g^eq */
          }
        }
      }
    for (int k = 0; k < s->n; ++k)
      if (s->bnd[k]) rest_node(s->ft + 9 * (size_t)k);
    double *tmp = s->f; s->f = s->ft; s->ft = tmp;
    tmp = s->g; s->g = s->gt; s->gt = tmp;
    s->t++;
  }
  moments(s);
  return ORC_OK;
}

int orc_fields(void *h, double *rho, double *ux, double *uy, double *phi) {
  orc_state *s = (orc_state *)h;
  moments(s);
  for (int k = 0; k < s->n; ++k) {
    if (rho) rho[k] = s->rho[k];
    if (ux) ux[k] = s->ux[k];
    if (uy) uy[k] = s->uy[k];
    if (phi) phi[k] = s->phi[k];
  }
  return ORC_OK;
}

/* Populations in plane-major layout [9][ny][nx]. */
int orc_get_populations(void *h, double *f, double *g) {
  orc_state *s = (orc_state *)h;
  for (int i = 0; i < 9; ++i)
    for (int k = 0; k < s->n; ++k) {
      if (f) f[(size_t)i * s->n + k] = s->f[9 * (size_t)k + i];
      if (g) g[(size_t)i * s->n + k] = s->g[9 * (size_t)k + i];
    }
  return ORC_OK;
}

/* Load populations; with apply_rest the boundary-node rest rule is applied to f
 * (for a state saved before that rule). */
int orc_set_populations(void *h, const double *f, const double *g, int apply_rest) {
  orc_state *s = (orc_state *)h;
  for (int i = 0; i < 9; ++i)
    for (int k = 0; k < s->n; ++k) {
      s->f[9 * (size_t)k + i] = s->solid[k] ? 0.0 : f[(size_t)i * s->n + k];
      s->g[9 * (size_t)k + i] = (s->solid[k] || !g) ? 0.0 : g[(size_t)i * s->n + k];
    }
  if (apply_rest)
    for (int k = 0; k < s->n; ++k)
      if (s->bnd[k]) rest_node(s->f + 9 * (size_t)k);
  moments(s);
  return ORC_OK;
}

/* Node kinds: 0 fluid, 1 boundary (fluid with a solid neighbour), 2 solid. */
int orc_node_kinds(void *h, unsigned char *kinds) {
  orc_state *s = (orc_state *)h;
  for (int k = 0; k < s->n; ++k) kinds[k] = s->solid[k] ? 2 : (s->bnd[k] ? 1 : 0);
  return ORC_OK;
}

/* Stencils of an arbitrary field with the ghost rule (h = prescribed gradient). */
int orc_stencils(void *h, const double *v, double hw, double *dx, double *dy, double *lap) {
  return stencils((orc_state *)h, v, hw, dx, dy, lap);
}

/* Equilibria and omega at every fluid node for the current state (for moment
 * checks).  feq, geq are [9][ny][nx]. */
int orc_equilibria(void *h, double *feq, double *geq, double *omega) {
  orc_state *s = (orc_state *)h;
  moments(s);
  int rc = all_stencils(s);
  if (rc) return rc;
  for (int k = 0; k < s->n; ++k) {
    double fe[9] = {0}, ge[9] = {0}, om = 0.0;
    if (!s->solid[k]) node_equilibria(s, k, fe, ge, &om);
    for (int i = 0; i < 9; ++i) {
      if (feq) feq[(size_t)i * s->n + k] = fe[i];
      if (geq) geq[(size_t)i * s->n + k] = ge[i];
    }
    if (omega) omega[k] = om;
  }
  return ORC_OK;
}

/* Diagnostics: l(t) along the tube's middle row, the filled volume divided by
 * H, total mass and total phi over fluid nodes (Sec. 1 defines l; l_eff = l + H/2
 * is formed by the caller). */
int orc_filled_length(void *h, double *l_centre, double *l_vol, double *mass, double *phi_sum) {
  orc_state *s = (orc_state *)h;
  const orc_params *p = &s->p;
  const int nx = p->nx, ny = p->ny;
  moments(s);
  double m = 0.0, ps = 0.0;
  for (int k = 0; k < s->n; ++k)
    if (!s->solid[k]) {
      m += s->rho[k];
      ps += s->phi[k];
    }
  if (mass) *mass = m;
  if (phi_sum) *phi_sum = ps;
  if (p->tube_len <= 0) {
    if (l_centre) *l_centre = 0.0;
    if (l_vol) *l_vol = 0.0;
    return ORC_OK;
  }
  const double thr = p->model == 0 ? 0.5 * (p->rho_l + p->rho_g) : 0.0;
  const double *v = p->model == 0 ? s->rho : s->phi;
  int ya, yb;
  if (p->tube_h % 2) {
    ya = yb = wrap(p->tube_y0 + (p->tube_h - 1) / 2, ny);
  } else {
    ya = wrap(p->tube_y0 + p->tube_h / 2 - 1, ny);
    yb = wrap(p->tube_y0 + p->tube_h / 2, ny);
  }
  double l = -1.0;
  for (int k = 0; k < p->tube_len; ++k) {
    const int x = wrap(p->tube_x0 + k, nx);
    const double c0 = 0.5 * (v[ya * nx + x] + v[yb * nx + x]) - thr;
    if (k == 0 && c0 <= 0.0) {
      l = 0.0;
      break;
    }
    if (k + 1 >= p->tube_len) break;
    const int x1 = wrap(x + 1, nx);
    const double c1 = 0.5 * (v[ya * nx + x1] + v[yb * nx + x1]) - thr;
    if (c0 > 0.0 && c1 <= 0.0) {
      l = k + c0 / (c0 - c1);
      break;
    }
  }
  if (l < 0.0) l = (double)p->tube_len;
  double vol = 0.0;
  for (int k = 0; k < p->tube_len; ++k) {
    const int x = wrap(p->tube_x0 + k, nx);
    for (int j = 0; j < p->tube_h; ++j) {
      const int y = wrap(p->tube_y0 + j, ny);
      const double q = v[y * nx + x];
      vol += p->model == 0 ? (q - p->rho_g) / (p->rho_l - p->rho_g) : 0.5 * (q + 1.0);
    }
  }
  if (l_centre) *l_centre = l;
  if (l_vol) *l_vol = vol / p->tube_h;
  return ORC_OK;
}

long orc_time(void *h) { return ((orc_state *)h)->t; }
