/*
 * oracle.c -- plain FP64 CPU reference of the RZ electrostatic PIC-MCC step.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  Nothing here is tuned: one loop
 * per particle, the Poisson problem solved by a banded Cholesky factorisation
 * of the whole system, random numbers from a Philox4x64-10 written from its
 * published definition (Salmon, Moraes, Dror, Shaw, SC'11).
 *
 * Section references are to arXiv:2507.10727.  The paper gives the method's
 * ingredients (Section 2: EC-PIC / MC-PIC interpolation and the edge-centred
 * field; Section 3: field and particle boundaries, the external circuit,
 * secondary emission, MCC with reactions (1a)-(1c)) but not their equations;
 * comments marked "reading" state the equation taken where it is silent.
 */
#define _DEFAULT_SOURCE
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* CODATA 2018 */
#define QE 1.602176634e-19
#define ME 9.1093837015e-31
#define EPS0 8.8541878128e-12
#define KBOLTZ 1.380649e-23
#define PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon et al., SC'11): 10 rounds of a multiply-xor       */
/* S-box on four 64-bit words with a Weyl-sequence key schedule.            */
/* ------------------------------------------------------------------------ */
void orc_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
  uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += W0; k1 += W1; }
    unsigned __int128 p0 = (unsigned __int128)M0 * x0;
    unsigned __int128 p1 = (unsigned __int128)M1 * x2;
    uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
    uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
    uint64_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (the same paper): the 32-bit form, four 32-bit words,      */
/* multipliers 0xD2511F53 and 0xCD9E8D57, Weyl key increments 0x9E3779B9    */
/* and 0xBB67AE85.                                                          */
/* ------------------------------------------------------------------------ */
void orc_philox4x32(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += W0; k1 += W1; }
    uint64_t p0 = (uint64_t)M0 * x0, p1 = (uint64_t)M1 * x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* uniform on [0,1) from the top 53 bits */
static double u01(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }

/* Draw the four words of stream `k` for particle `id` at step `step` of a species. */
static void draws(const orc_config* c, int species, int64_t id, int64_t step, int k, double u[4]) {
  uint64_t ctr[4] = {(uint64_t)id, (uint64_t)step, (uint64_t)k, 0};
  uint64_t key[2] = {c->seed, (uint64_t)species};
  uint64_t w[4];
  orc_philox4x64(ctr, key, w);
  for (int j = 0; j < 4; ++j) u[j] = u01(w[j]);
}

/* The null-collision candidate draw of electron `id` at step `step`: the
 * first word of Philox4x32-10 with counter (id, step) as four 32-bit halves
 * (low half first) and key (seed low half, seed high half), as a uniform
 * U = word 2^-32 on [0,1) (exact in a double).  Reading: Section 3 draws one
 * uniform number per electron and step for the null-collision test and fixes
 * no generator; the test is the one draw made for every electron at every
 * step, so it takes the 32-bit form of the generator, whose 2^-32 resolution
 * is far below the collision probabilities of these runs, and the collision
 * itself draws from stream 0 of the 64-bit form. */
static double candidate_draw(const orc_config* c, int64_t id, int64_t step) {
  const uint64_t uid = (uint64_t)id, ust = (uint64_t)step;
  uint32_t ctr[4] = {(uint32_t)uid, (uint32_t)(uid >> 32), (uint32_t)ust, (uint32_t)(ust >> 32)};
  uint32_t key[2] = {(uint32_t)c->seed, (uint32_t)(c->seed >> 32)};
  uint32_t w[4];
  orc_philox4x32(ctr, key, w);
  return (double)w[0] * (1.0 / 4294967296.0);
}

/* ------------------------------------------------------------------------ */
/* Static magnetic field.  Section 3 computes B once from a magnet scalar  */
/* potential and hands it to the plasma solve; reading: the stand-in       */
/* potential A0 J0(kr) e^{-kz}, B = -grad, so                               */
/*   B_r = k A0 J1(kr) e^{-kz},  B_z = k A0 J0(kr) e^{-kz}.                 */
/* ------------------------------------------------------------------------ */
void orc_bfield(const orc_config* c, double r, double z, double* Br, double* Bz) {
  if (c->b_mode == 1) { *Br = c->B0r; *Bz = c->B0z; return; }
  double e = exp(-c->B_k * z);
  *Br = c->B_kA0 * j1(c->B_k * r) * e;
  *Bz = c->B_kA0 * j0(c->B_k * r) * e;
}

/* ------------------------------------------------------------------------ */
/* Grid geometry.  Nodes r_m = m dr (m = 0..nr), z_n = n dz (n = 0..nz);    */
/* phi and rho live on nodes (Section 2, last sentences).                   */
/* ------------------------------------------------------------------------ */
static int nidx(const orc_config* c, int m, int n) { return m * (c->nz + 1) + n; }
static double dr_of(const orc_config* c) { return c->R / c->nr; }
static double dz_of(const orc_config* c) { return c->L / c->nz; }

/* Area of the annulus belonging to radial node m (times dz gives the node's
 * control volume): 2 pi r_m dr inside, pi (dr/2)^2 on the axis, and the
 * half annulus pi (R^2 - (R - dr/2)^2) at r = R. */
static double node_area(const orc_config* c, int m) {
  double dr = dr_of(c);
  if (m == 0) return PI * 0.25 * dr * dr;
  if (m == c->nr) return PI * (c->R * c->R - (c->R - 0.5 * dr) * (c->R - 0.5 * dr));
  return 2.0 * PI * (m * dr) * dr;
}

/* Control volume of node (m,n); half volume on the z walls. */
double orc_node_volume(const orc_config* c, int m, int n) {
  double h = (n == 0 || n == c->nz) ? 0.5 : 1.0;
  return node_area(c, m) * dz_of(c) * h;
}

/* Cell containing coordinate x on a uniform axis of `ncell` cells of size d,
 * and the fractional offset in it.  The last cell is closed on the right. */
static void locate(double x, double d, int ncell, int* k, double* f) {
  int i = (int)floor(x / d);
  if (i > ncell - 1) i = ncell - 1;
  if (i < 0) i = 0;
  *k = i;
  *f = x / d - i;
}

/* Radial weight of node m+1 for a particle at r in cell m (the weight of node
 * m is one minus it).  Section 2: linear (tent) interpolation for the
 * deposit.  rweight 1 (reading of "volume-weighted in r"): linear in r^2,
 * S_{m+1} = (r^2 - r_m^2) / (r_{m+1}^2 - r_m^2). */
static double rweight_upper(const orc_config* c, double r, int m, double fr) {
  if (c->rweight == 0) return fr;
  double dr = dr_of(c);
  double rm = m * dr, rp = (m + 1) * dr;
  return (r * r - rm * rm) / (rp * rp - rm * rm);
}

/* ------------------------------------------------------------------------ */
/* Charge deposit: Q_mn += q w S^r_m(r) S^z_n(z) (Section 2: tent functions) */
/* ------------------------------------------------------------------------ */
void orc_deposit(const orc_config* c, int64_t np, const double* r, const double* z, double qw,
                 double* Q) {
  double dr = dr_of(c), dz = dz_of(c);
  for (int64_t p = 0; p < np; ++p) {
    int m, n;
    double fr, fz;
    locate(r[p], dr, c->nr, &m, &fr);
    locate(z[p], dz, c->nz, &n, &fz);
    double sr1 = rweight_upper(c, r[p], m, fr), sr0 = 1.0 - sr1;
    double sz1 = fz, sz0 = 1.0 - fz;
    Q[nidx(c, m, n)] += qw * sr0 * sz0;
    Q[nidx(c, m + 1, n)] += qw * sr1 * sz0;
    Q[nidx(c, m, n + 1)] += qw * sr0 * sz1;
    Q[nidx(c, m + 1, n + 1)] += qw * sr1 * sz1;
  }
}

/* ------------------------------------------------------------------------ */
/* Fields from phi.  Section 2: EC-PIC stores E on edges,                   */
/*   E_z at (r_m, z_{n+1/2}),  E_r at (r_{m+1/2}, z_n),                     */
/* and interpolates E_r NGP in r / linear in z, E_z linear in r / NGP in z. */
/* MC-PIC interpolates nodal E with the deposit's own stencil.              */
/* ------------------------------------------------------------------------ */
static double er_edge(const orc_config* c, const double* phi, int m, int n) {
  return -(phi[nidx(c, m + 1, n)] - phi[nidx(c, m, n)]) / dr_of(c);
}
static double ez_edge(const orc_config* c, const double* phi, int m, int n) {
  return -(phi[nidx(c, m, n + 1)] - phi[nidx(c, m, n)]) / dz_of(c);
}
/* Reading: nodal E is the mean of the two adjacent edge values, the single
 * adjacent edge on a conducting wall, zero normal component on an insulating
 * (Neumann) wall -- the boundary condition itself -- and E_r = 0 on the axis
 * by symmetry. */
static int cathode_node(const orc_config* c, int m);
static double er_node(const orc_config* c, const double* phi, int m, int n) {
  if (m == 0) return 0.0;
  if (m == c->nr) return c->wall_neumann ? 0.0 : er_edge(c, phi, m - 1, n);
  return 0.5 * (er_edge(c, phi, m - 1, n) + er_edge(c, phi, m, n));
}
static double ez_node(const orc_config* c, const double* phi, int m, int n) {
  if (n == 0) {
    int insulating = m == c->nr ? (c->gap_neumann && c->wall_neumann)
                                : (c->gap_neumann && !cathode_node(c, m));
    return insulating ? 0.0 : ez_edge(c, phi, m, 0);
  }
  if (n == c->nz) return ez_edge(c, phi, m, c->nz - 1);
  return 0.5 * (ez_edge(c, phi, m, n - 1) + ez_edge(c, phi, m, n));
}

void orc_efield_at(const orc_config* c, const double* phi, double r, double z, double* Er,
                   double* Ez) {
  double dr = dr_of(c), dz = dz_of(c);
  int m, n;
  double fr, fz;
  locate(r, dr, c->nr, &m, &fr);
  locate(z, dz, c->nz, &n, &fz);
  double sr1 = rweight_upper(c, r, m, fr), sr0 = 1.0 - sr1;
  double sz1 = fz, sz0 = 1.0 - fz;
  if (c->gather == 0) {
    /* EC-PIC: E = -sum phi_mn grad S_mn.  E_r: NGP in r (the edge of the cell
     * the particle is in), linear in z.  With volume weighting dS/dr carries
     * the factor r / r_{m+1/2}. */
    double er = sz0 * er_edge(c, phi, m, n) + sz1 * er_edge(c, phi, m, n + 1);
    if (c->rweight == 1) er *= r / ((m + 0.5) * dr);
    double ez = sr0 * ez_edge(c, phi, m, n) + sr1 * ez_edge(c, phi, m + 1, n);
    *Er = er;
    *Ez = ez;
  } else {
    /* MC-PIC: the deposit's stencil applied to nodal E. */
    *Er = sr0 * sz0 * er_node(c, phi, m, n) + sr1 * sz0 * er_node(c, phi, m + 1, n) +
          sr0 * sz1 * er_node(c, phi, m, n + 1) + sr1 * sz1 * er_node(c, phi, m + 1, n + 1);
    *Ez = sr0 * sz0 * ez_node(c, phi, m, n) + sr1 * sz0 * ez_node(c, phi, m + 1, n) +
          sr0 * sz1 * ez_node(c, phi, m, n + 1) + sr1 * sz1 * ez_node(c, phi, m + 1, n + 1);
  }
}

/* ------------------------------------------------------------------------ */
/* Poisson problem (Section 3: anode grounded, cathode at the circuit       */
/* voltage, the insulating "block" a Neumann boundary, Gauss's law on the   */
/* axis).  Reading: finite volumes on the nodes.  Node (m,n) owns the part  */
/* of the box [r_m -+ dr/2] x [z_n -+ dz/2] inside the domain (area(m) in r,*/
/* half height on z = 0 and z = L).  Integrating -div(eps0 grad phi) = rho  */
/* over it, with the flux through a face between two nodes approximated by  */
/* eps0 (face area) (phi_k - phi_j) / spacing and no flux through the       */
/* domain's outer surface, gives  sum_j a_kj (phi_k - phi_j) = V_k rho_k    */
/* with the symmetric couplings                                             */
/*   r-neighbours m, m+1:  a_r(m) h(n),  a_r(m) = eps0 2 pi r_{m+1/2} dz/dr, */
/*                         h = 1/2 on z = 0 and z = L, else 1              */
/*   z-neighbours n, n+1:  a_z(m) = eps0 area(m) / dz                       */
/* (on the axis the first line is Gauss's law on the disk r < dr/2).  Nodes */
/* on a conductor are Dirichlet (given values), the rest are unknowns; the  */
/* couplings to Dirichlet neighbours move to the right-hand side, so the    */
/* system is symmetric positive definite (the anode is always Dirichlet).   */
/* ------------------------------------------------------------------------ */
static double a_r(const orc_config* c, int m) {
  return EPS0 * 2.0 * PI * ((m + 0.5) * dr_of(c)) * dz_of(c) / dr_of(c);
}
static double a_z(const orc_config* c, int m) {
  return EPS0 * node_area(c, m) * dz_of(c) / (dz_of(c) * dz_of(c));
}
static double h_of(const orc_config* c, int n) { return (n == 0 || n == c->nz) ? 0.5 : 1.0; }

/* Cathode nodes: z = 0, r_m <= Rc, m < nr (Section 3 and Table 1's
 * benchmark geometry). */
static int cathode_node(const orc_config* c, int m) { return m * dr_of(c) <= c->Rc && m < c->nr; }

/* Unknown (not on a conductor).  Conductors: the anode z = L; the cathode;
 * the rest of z = 0 unless gap_neumann; the wall r = R unless wall_neumann. */
static int node_free(const orc_config* c, int m, int n) {
  if (n == c->nz) return 0;
  if (m == c->nr && !c->wall_neumann) return 0;
  if (n == 0) return c->gap_neumann && !cathode_node(c, m);
  return 1;
}

typedef struct chol {
  int nfree, bw;
  int* idx;  /* unknown number of node (m,n), -1 for Dirichlet nodes */
  double* L; /* L(k, k-j) at L[k*(bw+1) + j] */
} chol;

/* the four neighbours of a node and their couplings (0 outside the grid) */
static int neighbours(const orc_config* c, int m, int n, int nb[4][2], double a[4]) {
  int k = 0;
  if (m > 0) { nb[k][0] = m - 1; nb[k][1] = n; a[k++] = a_r(c, m - 1) * h_of(c, n); }
  if (m < c->nr) { nb[k][0] = m + 1; nb[k][1] = n; a[k++] = a_r(c, m) * h_of(c, n); }
  if (n > 0) { nb[k][0] = m; nb[k][1] = n - 1; a[k++] = a_z(c, m); }
  if (n < c->nz) { nb[k][0] = m; nb[k][1] = n + 1; a[k++] = a_z(c, m); }
  return k;
}

static int chol_build(const orc_config* c, chol* f) {
  size_t nn = (size_t)(c->nr + 1) * (c->nz + 1);
  f->idx = (int*)malloc(sizeof(int) * nn);
  int nfree = 0;
  for (int m = 0; m <= c->nr; ++m)
    for (int n = 0; n <= c->nz; ++n) f->idx[nidx(c, m, n)] = node_free(c, m, n) ? nfree++ : -1;
  /* unknowns are numbered m-major, so a neighbour is at most nz+1 away */
  int bw = c->nz + 1;
  f->nfree = nfree;
  f->bw = bw;
  f->L = (double*)calloc((size_t)(nfree > 0 ? nfree : 1) * (bw + 1), sizeof(double));
  if (!f->L || !f->idx) return -1;
  /* assemble the lower band of A */
  for (int m = 0; m <= c->nr; ++m)
    for (int n = 0; n <= c->nz; ++n) {
      int k = f->idx[nidx(c, m, n)];
      if (k < 0) continue;
      int nb[4][2];
      double a[4], diag = 0.0;
      int cnt = neighbours(c, m, n, nb, a);
      for (int j = 0; j < cnt; ++j) {
        diag += a[j];
        int kj = f->idx[nidx(c, nb[j][0], nb[j][1])];
        if (kj >= 0 && kj < k) f->L[(size_t)k * (bw + 1) + (k - kj)] = -a[j];
      }
      f->L[(size_t)k * (bw + 1) + 0] = diag;
    }
  /* in-place banded Cholesky A = L L^T */
  for (int k = 0; k < nfree; ++k) {
    int j0 = k - bw < 0 ? 0 : k - bw;
    for (int j = j0; j <= k; ++j) {
      double s = f->L[(size_t)k * (bw + 1) + (k - j)];
      int p0 = j0 > j - bw ? j0 : j - bw;
      for (int p = p0; p < j; ++p)
        s -= f->L[(size_t)k * (bw + 1) + (k - p)] * f->L[(size_t)j * (bw + 1) + (j - p)];
      if (j == k) {
        if (!(s > 0.0)) return -2;
        f->L[(size_t)k * (bw + 1)] = sqrt(s);
      } else {
        f->L[(size_t)k * (bw + 1) + (k - j)] = s / f->L[(size_t)j * (bw + 1)];
      }
    }
  }
  return 0;
}

static void chol_free(chol* f) {
  free(f->L);
  free(f->idx);
}

static void chol_solve(const chol* f, double* x /* in: b, out: solution */) {
  int bw = f->bw, N = f->nfree;
  for (int k = 0; k < N; ++k) {
    double s = x[k];
    int j0 = k - bw < 0 ? 0 : k - bw;
    for (int j = j0; j < k; ++j) s -= f->L[(size_t)k * (bw + 1) + (k - j)] * x[j];
    x[k] = s / f->L[(size_t)k * (bw + 1)];
  }
  for (int k = N - 1; k >= 0; --k) {
    double s = x[k];
    int i1 = k + bw > N - 1 ? N - 1 : k + bw;
    for (int i = k + 1; i <= i1; ++i) s -= f->L[(size_t)i * (bw + 1) + (i - k)] * x[i];
    x[k] = s / f->L[(size_t)k * (bw + 1)];
  }
}

/* Solve with the factor: rho on nodes, Dirichlet values taken from phi_bc on
 * the conductor nodes; result written to phi (all nodes). */
static void poisson_with(const orc_config* c, const chol* f, const double* rho,
                         const double* phi_bc, double* phi) {
  double* x = (double*)malloc(sizeof(double) * (size_t)(f->nfree > 0 ? f->nfree : 1));
  for (int m = 0; m <= c->nr; ++m)
    for (int n = 0; n <= c->nz; ++n) {
      int k = f->idx[nidx(c, m, n)];
      if (k < 0) continue;
      double b = orc_node_volume(c, m, n) * rho[nidx(c, m, n)];
      int nb[4][2];
      double a[4];
      int cnt = neighbours(c, m, n, nb, a);
      for (int j = 0; j < cnt; ++j)
        if (f->idx[nidx(c, nb[j][0], nb[j][1])] < 0) b += a[j] * phi_bc[nidx(c, nb[j][0], nb[j][1])];
      x[k] = b;
    }
  chol_solve(f, x);
  for (int m = 0; m <= c->nr; ++m)
    for (int n = 0; n <= c->nz; ++n) {
      int k = f->idx[nidx(c, m, n)];
      phi[nidx(c, m, n)] = k < 0 ? phi_bc[nidx(c, m, n)] : x[k];
    }
  free(x);
}

int orc_poisson(const orc_config* c, const double* rho, const double* phi_bc, double* phi) {
  chol f;
  int rc = chol_build(c, &f);
  if (rc == 0) poisson_with(c, &f, rho, phi_bc, phi);
  chol_free(&f);
  return rc;
}

/* Field energy 1/2 sum over edges a_e (delta phi)^2, i.e. eps0/2 sum E^2 times
 * the edge's volume; r-edges on the z walls carry half volume. */
double orc_field_energy(const orc_config* c, const double* phi) {
  double W = 0.0;
  for (int m = 0; m < c->nr; ++m)
    for (int n = 0; n <= c->nz; ++n) {
      double h = (n == 0 || n == c->nz) ? 0.5 : 1.0;
      double d = phi[nidx(c, m + 1, n)] - phi[nidx(c, m, n)];
      W += 0.5 * a_r(c, m) * h * d * d;
    }
  for (int m = 0; m <= c->nr; ++m)
    for (int n = 0; n < c->nz; ++n) {
      double d = phi[nidx(c, m, n + 1)] - phi[nidx(c, m, n)];
      W += 0.5 * a_z(c, m) * d * d;
    }
  return W;
}

/* ------------------------------------------------------------------------ */
/* Boris push in RZ (reading: the paper says only "explicit").  The particle */
/* is placed at (x, y, z) = (r, 0, z), so (v_r, v_theta, v_z) and (E_r, 0,  */
/* E_z), (B_r, 0, B_z) are Cartesian there.  Half kick, rotation, half kick,*/
/* straight move, then rotation of the frame back onto the new r axis.     */
/* ------------------------------------------------------------------------ */
/* Boris velocity update in the frame where the particle sits on the x axis:
 * returns the Cartesian v^{n+1/2} = (vx, vy, vz) of that frame. */
static void boris_velocity(double q_over_m, double dt, double Er, double Ez, double Br,
                           double Bz, double vr, double vt, double vz, double v[3]) {
  double h = 0.5 * q_over_m * dt;
  /* v- = v + h E */
  double ax = vr + h * Er, ay = vt, az = vz + h * Ez;
  /* t = h B, s = 2 t / (1 + t^2) */
  double tx = h * Br, ty = 0.0, tz = h * Bz;
  double t2 = tx * tx + ty * ty + tz * tz;
  double sx = 2.0 * tx / (1.0 + t2), sy = 2.0 * ty / (1.0 + t2), sz = 2.0 * tz / (1.0 + t2);
  /* v' = v- + v- x t */
  double px = ax + (ay * tz - az * ty);
  double py = ay + (az * tx - ax * tz);
  double pz = az + (ax * ty - ay * tx);
  /* v+ = v- + v' x s */
  double bx = ax + (py * sz - pz * sy);
  double by = ay + (pz * sx - px * sz);
  double bz = az + (px * sy - py * sx);
  /* v^{n+1/2} = v+ + h E */
  v[0] = bx + h * Er;
  v[1] = by;
  v[2] = bz + h * Ez;
}

/* Straight move from (r, 0, z) with Cartesian v, then rotation of the frame
 * so that the particle is back on the x axis: r' = sqrt(x'^2 + y'^2),
 * v_r = (x' vx + y' vy)/r', v_theta = (x' vy - y' vx)/r' (unchanged when
 * r' = 0).  Also returns the Cartesian end point (x', y'). */
static void move_rotate(double dt, const double v[3], double* r, double* z, double* vr,
                        double* vt, double* vz, double* x1_out, double* y1_out) {
  double x1 = *r + v[0] * dt, y1 = v[1] * dt, z1 = *z + v[2] * dt;
  double r1 = sqrt(x1 * x1 + y1 * y1);
  if (r1 > 0.0) {
    *vr = (x1 * v[0] + y1 * v[1]) / r1;
    *vt = (x1 * v[1] - y1 * v[0]) / r1;
  } else {
    *vr = v[0];
    *vt = v[1];
  }
  *vz = v[2];
  *r = r1;
  *z = z1;
  *x1_out = x1;
  *y1_out = y1;
}

void orc_boris_move(double q_over_m, double dt, double Er, double Ez, double Br, double Bz,
                    double* r, double* z, double* vr, double* vt, double* vz) {
  double v[3], x1, y1;
  boris_velocity(q_over_m, dt, Er, Ez, Br, Bz, *vr, *vt, *vz, v);
  move_rotate(dt, v, r, z, vr, vt, vz, &x1, &y1);
}

/* ------------------------------------------------------------------------ */
/* Cross sections (Section 3 takes them from QDB, unavailable; reading:     */
/* analytic stand-ins).  Elastic constant; excitation (1b) and ionization   */
/* (1c) of the form C ln(E/E_th) / (E E_th) above threshold.                */
/* ------------------------------------------------------------------------ */
void orc_sigma(const orc_config* c, double E, double out[3]) {
  out[0] = E > 0.0 ? c->sigma_el : 0.0;
  out[1] = E > c->exc_E ? c->exc_C * log(E / c->exc_E) / (E * c->exc_E) : 0.0;
  out[2] = E > c->ion_I ? c->ion_a * log(E / c->ion_I) / (E * c->ion_I) : 0.0;
}

/* Stepwise ionization from the metastable (1d), threshold 4.20 eV (Section 3);
 * same Lotz form as (1c), one outer-shell electron. */
double orc_sigma_meta(const orc_config* c, double E) {
  return E > c->meta_I ? c->meta_a * log(E / c->meta_I) / (E * c->meta_I) : 0.0;
}

/* Null-collision frequency (MCC [14]): nu_max = 1.001 max_E nu_T(E) with
 * nu_T = (n_g sigma_T(E) + n_meta sigma_1d(E)) v(E), over a log grid of 100001
 * energies in [1e-4 eV, E_cap]. */
double orc_nu_max(const orc_config* c) {
  double best = 0.0;
  for (int k = 0; k <= 100000; ++k) {
    double E = 1e-4 * pow(c->E_cap / 1e-4, k / 100000.0);
    if (k == 100000) E = c->E_cap;
    double s[3];
    orc_sigma(c, E, s);
    double v = sqrt(2.0 * E * QE / ME);
    double nu = (c->n_gas * (s[0] + s[1] + s[2]) + c->n_meta * orc_sigma_meta(c, E)) * v;
    if (nu > best) best = nu;
  }
  return 1.001 * best;
}

/* Rotate unit vector e by polar angle chi (cos given) and azimuth phi about
 * itself: e' = cos(chi) e + sin(chi) (cos(phi) u + sin(phi) w), with (u, w)
 * completing an orthonormal frame built from the coordinate axis along which
 * e has its smallest component. */
static void scatter_dir(const double e[3], double cos_chi, double phi, double out[3]) {
  int a = 0;
  if (fabs(e[1]) < fabs(e[a])) a = 1;
  if (fabs(e[2]) < fabs(e[a])) a = 2;
  double ax[3] = {0.0, 0.0, 0.0};
  ax[a] = 1.0;
  double u[3] = {ax[1] * e[2] - ax[2] * e[1], ax[2] * e[0] - ax[0] * e[2],
                 ax[0] * e[1] - ax[1] * e[0]};
  double un = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  u[0] /= un; u[1] /= un; u[2] /= un;
  double w[3] = {e[1] * u[2] - e[2] * u[1], e[2] * u[0] - e[0] * u[2], e[0] * u[1] - e[1] * u[0]};
  double sin_chi = sqrt(fmax(0.0, 1.0 - cos_chi * cos_chi));
  double cp = cos(phi), sp = sin(phi);
  for (int j = 0; j < 3; ++j) out[j] = cos_chi * e[j] + sin_chi * (cp * u[j] + sp * w[j]);
}

/* ------------------------------------------------------------------------ */
/* The simulation state                                                     */
/* ------------------------------------------------------------------------ */
typedef struct pstore {
  int64_t n, cap;
  double *r, *z, *vr, *vt, *vz;
  int64_t* id;
} pstore;

typedef struct birth {
  uint64_t key; /* (parent id << 2) | kind */
  double r, z, vr, vt, vz;
} birth;

typedef struct blist {
  int64_t n, cap;
  birth* b;
} blist;

struct orc_sim {
  orc_config c;
  int64_t step, next_id;
  pstore sp[2];
  double *phi, *rho, *Q, *Qs[2], *Bnr, *Bnz;
  chol f;
  double Vc;
  double* qhist;
  double nu_max, p_null;
  orc_diag d;
  /* region diagnostics */
  int64_t* ied;            /* ied_bins counts */
  int64_t ied_over;
  int64_t *rc_n[2];        /* per cell particle counts, summed over samples */
  double* rc_mom;          /* per cell electron sums: v_r, v_theta, v_z, |v|^2 */
  double* rc_phi;          /* per node potential, summed over samples */
  int64_t rc_samples;
};

static void ps_reserve(pstore* p, int64_t n) {
  if (n <= p->cap) return;
  int64_t cap = n + n / 2 + 16;
  p->r = (double*)realloc(p->r, sizeof(double) * cap);
  p->z = (double*)realloc(p->z, sizeof(double) * cap);
  p->vr = (double*)realloc(p->vr, sizeof(double) * cap);
  p->vt = (double*)realloc(p->vt, sizeof(double) * cap);
  p->vz = (double*)realloc(p->vz, sizeof(double) * cap);
  p->id = (int64_t*)realloc(p->id, sizeof(int64_t) * cap);
  p->cap = cap;
}

static void bl_push(blist* l, uint64_t key, double r, double z, double vr, double vt, double vz) {
  if (l->n == l->cap) {
    l->cap = l->cap * 2 + 64;
    l->b = (birth*)realloc(l->b, sizeof(birth) * l->cap);
  }
  birth* b = &l->b[l->n++];
  b->key = key; b->r = r; b->z = z; b->vr = vr; b->vt = vt; b->vz = vz;
}

static int cmp_birth(const void* a, const void* b) {
  uint64_t ka = ((const birth*)a)->key, kb = ((const birth*)b)->key;
  return ka < kb ? -1 : (ka > kb ? 1 : 0);
}

orc_sim* orc_create(const orc_config* c) {
  if (c->nr < 2 || c->nz < 2 || !(c->R > 0) || !(c->L > 0) || !(c->dt > 0)) return NULL;
  orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
  s->c = *c;
  size_t nn = (size_t)(c->nr + 1) * (c->nz + 1);
  s->phi = (double*)calloc(nn, sizeof(double));
  s->rho = (double*)calloc(nn, sizeof(double));
  s->Q = (double*)calloc(nn, sizeof(double));
  s->Qs[0] = (double*)calloc(nn, sizeof(double));
  s->Qs[1] = (double*)calloc(nn, sizeof(double));
  s->Bnr = (double*)calloc(nn, sizeof(double));
  s->Bnz = (double*)calloc(nn, sizeof(double));
  for (int m = 0; m <= c->nr; ++m)
    for (int n = 0; n <= c->nz; ++n)
      orc_bfield(c, m * dr_of(c), n * dz_of(c), &s->Bnr[nidx(c, m, n)], &s->Bnz[nidx(c, m, n)]);
  if (chol_build(c, &s->f) != 0) { orc_destroy(s); return NULL; }
  s->Vc = c->circuit_mode == 0 ? c->Vc_fixed : -c->Vs;
  s->qhist = (double*)calloc(c->n_avg > 0 ? c->n_avg : 1, sizeof(double));
  s->ied = (int64_t*)calloc(c->ied_bins > 0 ? c->ied_bins : 1, sizeof(int64_t));
  s->rc_n[0] = (int64_t*)calloc((size_t)c->nr * c->nz, sizeof(int64_t));
  s->rc_n[1] = (int64_t*)calloc((size_t)c->nr * c->nz, sizeof(int64_t));
  s->rc_mom = (double*)calloc((size_t)c->nr * c->nz * 4, sizeof(double));
  s->rc_phi = (double*)calloc(nn, sizeof(double));
  s->nu_max = orc_nu_max(c);
  s->p_null = -expm1(-s->nu_max * c->dt);
  return s;
}

void orc_destroy(orc_sim* s) {
  if (!s) return;
  for (int k = 0; k < 2; ++k) {
    free(s->sp[k].r); free(s->sp[k].z); free(s->sp[k].vr); free(s->sp[k].vt);
    free(s->sp[k].vz); free(s->sp[k].id); free(s->Qs[k]);
  }
  free(s->phi); free(s->rho); free(s->Q); free(s->Bnr); free(s->Bnz);
  chol_free(&s->f); free(s->qhist);
  free(s->ied); free(s->rc_n[0]); free(s->rc_n[1]); free(s->rc_mom); free(s->rc_phi);
  free(s);
}

int orc_set_particles(orc_sim* s, int sp, int64_t n, const double* r, const double* z,
                      const double* vr, const double* vt, const double* vz, const int64_t* id) {
  if (sp < 0 || sp > 1 || n < 0) return -1;
  pstore* p = &s->sp[sp];
  ps_reserve(p, n);
  p->n = n;
  for (int64_t k = 0; k < n; ++k) {
    p->r[k] = r[k]; p->z[k] = z[k]; p->vr[k] = vr[k]; p->vt[k] = vt[k]; p->vz[k] = vz[k];
    p->id[k] = id[k];
    if (id[k] + 1 > s->next_id) s->next_id = id[k] + 1;
  }
  return 0;
}

int64_t orc_count(const orc_sim* s, int sp) { return s->sp[sp].n; }

int orc_get_particles(const orc_sim* s, int sp, double* r, double* z, double* vr, double* vt,
                      double* vz, int64_t* id) {
  const pstore* p = &s->sp[sp];
  for (int64_t k = 0; k < p->n; ++k) {
    r[k] = p->r[k]; z[k] = p->z[k]; vr[k] = p->vr[k]; vt[k] = p->vt[k]; vz[k] = p->vz[k];
    id[k] = p->id[k];
  }
  return 0;
}

/* Deposit both species (electrons -e w, ions +e w) into Q and rho = Q / V. */
static void deposit_all(orc_sim* s) {
  const orc_config* c = &s->c;
  size_t nn = (size_t)(c->nr + 1) * (c->nz + 1);
  for (int k = 0; k < 2; ++k) {
    memset(s->Qs[k], 0, nn * sizeof(double));
    double qw = (k == 0 ? -QE : QE) * c->weight;
    orc_deposit(c, s->sp[k].n, s->sp[k].r, s->sp[k].z, qw, s->Qs[k]);
  }
  for (int m = 0; m <= c->nr; ++m)
    for (int n = 0; n <= c->nz; ++n) {
      int i = nidx(c, m, n);
      s->Q[i] = s->Qs[0][i] + s->Qs[1][i];
      s->rho[i] = s->Q[i] / orc_node_volume(c, m, n);
    }
}

/* Dirichlet data: the cathode (z = 0, r_m <= Rc) at V_c; the other
 * conductor nodes (anode z = L; the rest of z = 0 and the wall r = R unless
 * insulating) grounded (Section 3, with the cathode disk of the benchmark
 * configuration). */
static void solve_phi(orc_sim* s) {
  const orc_config* c = &s->c;
  size_t nn = (size_t)(c->nr + 1) * (c->nz + 1);
  double* bc = (double*)calloc(nn, sizeof(double));
  for (int m = 0; m <= c->nr; ++m)
    if (cathode_node(c, m)) bc[nidx(c, m, 0)] = s->Vc;
  poisson_with(c, &s->f, s->rho, bc, s->phi);
  free(bc);
}

int orc_solve_fields(orc_sim* s) {
  deposit_all(s);
  solve_phi(s);
  return 0;
}

void orc_set_phi(orc_sim* s, const double* phi) {
  size_t nn = (size_t)(s->c.nr + 1) * (s->c.nz + 1);
  memcpy(s->phi, phi, nn * sizeof(double));
}

void orc_get_fields(const orc_sim* s, double* phi, double* rho, double* Q) {
  size_t nn = (size_t)(s->c.nr + 1) * (s->c.nz + 1);
  if (phi) memcpy(phi, s->phi, nn * sizeof(double));
  if (rho) memcpy(rho, s->rho, nn * sizeof(double));
  if (Q) memcpy(Q, s->Q, nn * sizeof(double));
}

void orc_get_species_charge(const orc_sim* s, int species, double* Q) {
  size_t nn = (size_t)(s->c.nr + 1) * (s->c.nz + 1);
  memcpy(Q, s->Qs[species == 0 ? 0 : 1], nn * sizeof(double));
}

void orc_set_circuit(orc_sim* s, double Vc, int64_t step, const double* qhist, int n) {
  s->Vc = Vc;
  s->step = step;
  for (int k = 0; k < s->c.n_avg && k < n; ++k) s->qhist[k] = qhist[k];
}

void orc_set_next_id(orc_sim* s, int64_t next_id) { s->next_id = next_id; }
int64_t orc_get_next_id(const orc_sim* s) { return s->next_id; }
int64_t orc_get_step(const orc_sim* s) { return s->step; }

/* Particle re-weighting (Section 6, the large-grid EC/MC runs): when the
 * particles per cell grow too large, two thirds of the particles are removed
 * and the weight of the rest is tripled.  Reading: the paper does not say
 * which particles go; each particle is kept independently with probability
 * 1/factor, decided by its own counter-based draw (stream 5 of the particle's
 * id at the current step), so the kept set does not depend on storage order
 * and total charge, density profile and velocity distribution are preserved
 * in expectation.  The kept particles are unchanged and keep their order. */
int64_t orc_reweight(orc_sim* s, int factor) {
  if (factor < 1) return -1;
  int64_t kept = 0;
  for (int sp = 0; sp < 2; ++sp) {
    pstore* p = &s->sp[sp];
    int64_t out = 0;
    for (int64_t k = 0; k < p->n; ++k) {
      uint64_t ctr[4] = {(uint64_t)p->id[k], (uint64_t)s->step, 5, 0};
      uint64_t key[2] = {s->c.seed, (uint64_t)sp};
      uint64_t w[4];
      orc_philox4x64(ctr, key, w);
      if (w[0] % (uint64_t)factor != 0) continue;
      p->r[out] = p->r[k]; p->z[out] = p->z[k];
      p->vr[out] = p->vr[k]; p->vt[out] = p->vt[k]; p->vz[out] = p->vz[k];
      p->id[out] = p->id[k];
      ++out;
    }
    p->n = out;
    kept += out;
  }
  s->c.weight *= (double)factor;
  return kept;
}

double orc_get_weight(const orc_sim* s) { return s->c.weight; }
void orc_get_diag(const orc_sim* s, orc_diag* d) { *d = s->d; }

/* B at a particle: bilinear interpolation of the node table. */
static void b_at(const orc_sim* s, double r, double z, double* Br, double* Bz) {
  const orc_config* c = &s->c;
  int m, n;
  double fr, fz;
  locate(r, dr_of(c), c->nr, &m, &fr);
  locate(z, dz_of(c), c->nz, &n, &fz);
  double w00 = (1 - fr) * (1 - fz), w10 = fr * (1 - fz), w01 = (1 - fr) * fz, w11 = fr * fz;
  *Br = w00 * s->Bnr[nidx(c, m, n)] + w10 * s->Bnr[nidx(c, m + 1, n)] +
        w01 * s->Bnr[nidx(c, m, n + 1)] + w11 * s->Bnr[nidx(c, m + 1, n + 1)];
  *Bz = w00 * s->Bnz[nidx(c, m, n)] + w10 * s->Bnz[nidx(c, m + 1, n)] +
        w01 * s->Bnz[nidx(c, m, n + 1)] + w11 * s->Bnz[nidx(c, m + 1, n + 1)];
}

/* An ionizing collision of electron k (reactions (1c) and (1d)): the electron
 * loses the threshold I and shares E - I uniformly with a new electron
 * (isotropic); the ion is born with a Maxwellian at the gas temperature.
 * Returns the primary's new energy. */
static double ionize(orc_sim* s, int64_t k, double E, double I, const double e[3], blist* be,
                     blist* bi) {
  const orc_config* c = &s->c;
  pstore* p = &s->sp[0];
  double u2[4], g[4];
  draws(c, 0, p->id[k], s->step, 1, u2);
  double Ex = E - I;
  double Enew = u2[0] * Ex;
  double E2 = Ex - Enew;
  double d2[3];
  scatter_dir(e, 1.0 - 2.0 * u2[1], 2.0 * PI * u2[2], d2);
  double v2 = sqrt(2.0 * E2 * QE / ME);
  uint64_t key = ((uint64_t)p->id[k] << 2) | 0u;
  bl_push(be, key, p->r[k], p->z[k], v2 * d2[0], v2 * d2[1], v2 * d2[2]);
  /* ion: Maxwellian at T_gas by Box-Muller */
  draws(c, 0, p->id[k], s->step, 4, g);
  double sig = sqrt(KBOLTZ * c->T_gas / c->m_ion);
  double rho1 = sqrt(-2.0 * log(1.0 - g[0])), th1 = 2.0 * PI * g[1];
  double rho2 = sqrt(-2.0 * log(1.0 - g[2])), th2 = 2.0 * PI * g[3];
  bl_push(bi, key, p->r[k], p->z[k], sig * rho1 * cos(th1), sig * rho1 * sin(th1),
          sig * rho2 * cos(th2));
  return Enew;
}

/* MCC for one electron (Section 3: MCC [14], reactions (1a)-(1d)); null
 * collision with probability 1 - exp(-nu_max dt) of a candidate, the process
 * chosen by U nu_max against the cumulative frequencies n_g sigma_k v (1a-1c)
 * and n_meta sigma_1d v (1d).  Reading: isotropic scattering; elastic loss
 * E' = E (1 - 2 m/M (1 - cos chi)); excitation loses 11.55 eV; ionization
 * loses 15.76 eV (1c) or 4.20 eV (1d) and shares the rest uniformly; the ion
 * is born at rest-frame gas temperature. */
static void mcc_electron(orc_sim* s, int64_t k, blist* be, blist* bi) {
  const orc_config* c = &s->c;
  pstore* p = &s->sp[0];
  if (!(candidate_draw(c, p->id[k], s->step) < s->p_null)) return;
  double u[4];
  draws(c, 0, p->id[k], s->step, 0, u);   /* u[1..3]: process and angles */
  double v[3] = {p->vr[k], p->vt[k], p->vz[k]};
  double vmag = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  double E = 0.5 * ME * vmag * vmag / QE;
  double sg[3];
  orc_sigma(c, E, sg);
  double nu_el = c->n_gas * sg[0] * vmag, nu_ex = c->n_gas * sg[1] * vmag;
  double nu_io = c->n_gas * sg[2] * vmag;
  double nu_md = c->n_meta * orc_sigma_meta(c, E) * vmag;
  double R = u[1] * s->nu_max;
  double e[3] = {v[0] / (vmag > 0 ? vmag : 1), v[1] / (vmag > 0 ? vmag : 1),
                 v[2] / (vmag > 0 ? vmag : 1)};
  double cos_chi = 1.0 - 2.0 * u[2], phi = 2.0 * PI * u[3];
  double d[3], Enew;
  if (R < nu_el) {
    Enew = E * (1.0 - 2.0 * ME / c->m_ion * (1.0 - cos_chi));
    s->d.n_elastic++;
  } else if (R < nu_el + nu_ex) {
    Enew = E - c->exc_E;
    s->d.n_excite++;
  } else if (R < nu_el + nu_ex + nu_io) {
    Enew = ionize(s, k, E, c->ion_I, e, be, bi);
    s->d.n_ionize++;
  } else if (R < nu_el + nu_ex + nu_io + nu_md) {
    Enew = ionize(s, k, E, c->meta_I, e, be, bi);
    s->d.n_ionize_meta++;
  } else {
    return; /* null collision */
  }
  scatter_dir(e, cos_chi, phi, d);
  double vn = sqrt(2.0 * Enew * QE / ME);
  p->vr[k] = vn * d[0];
  p->vt[k] = vn * d[1];
  p->vz[k] = vn * d[2];
}

/* Largest number of macroparticles of a species in one cell (the quantity
 * Section 6 watches before re-weighting). */
static int64_t max_per_cell(const orc_sim* s, int sp) {
  const orc_config* c = &s->c;
  int64_t* cnt = (int64_t*)calloc((size_t)c->nr * c->nz, sizeof(int64_t));
  const pstore* p = &s->sp[sp];
  int64_t best = 0;
  for (int64_t k = 0; k < p->n; ++k) {
    int m, n;
    double f;
    locate(p->r[k], dr_of(c), c->nr, &m, &f);
    locate(p->z[k], dz_of(c), c->nz, &n, &f);
    int64_t v = ++cnt[(size_t)m * c->nz + n];
    if (v > best) best = v;
  }
  free(cnt);
  return best;
}

int orc_step(orc_sim* s, int64_t nsteps) {
  const orc_config* c = &s->c;
  for (int64_t it = 0; it < nsteps; ++it) {
    blist be = {0, 0, NULL}, bi = {0, 0, NULL};
    int64_t n_ion_cath = 0, n_e_cath = 0, n_sey = 0;
    memset(&s->d, 0, sizeof(s->d));
    s->d.W_field = orc_field_energy(c, s->phi);
    for (int sp = 0; sp < 2; ++sp) {
      pstore* p = &s->sp[sp];
      double q = sp == 0 ? -QE : QE, mass = sp == 0 ? ME : c->m_ion;
      double K = 0.0;
      int64_t out = 0;
      for (int64_t k = 0; k < p->n; ++k) {
        double r = p->r[k], z = p->z[k], vr = p->vr[k], vt = p->vt[k], vz = p->vz[k];
        double r0 = r, z0 = z, x1 = r, y1 = 0.0;
        double v2old = vr * vr + vt * vt + vz * vz;
        if (c->push_on) {
          double Er = 0.0, Ez = 0.0, Br, Bz, v[3];
          if (c->field_on) orc_efield_at(c, s->phi, r, z, &Er, &Ez);
          b_at(s, r, z, &Br, &Bz);
          boris_velocity(q / mass, c->dt, Er, Ez, Br, Bz, vr, vt, vz, v);
          move_rotate(c->dt, v, &r, &z, &vr, &vt, &vz, &x1, &y1);
        }
        double v2new = vr * vr + vt * vt + vz * vz;
        K += 0.5 * mass * c->weight * 0.5 * (v2old + v2new);
        /* particle walls (Section 3): absorb at z = 0, z = L, r = R; the axis
         * reflects by construction (r >= 0).  Reading: z < 0, z >= L, r >= R. */
        int absorbed = 0;
        if (c->walls_reflect) {
          if (z < 0.0) { z = -z; vz = -vz; }
          if (z >= c->L) { z = 2.0 * c->L - z; vz = -vz; if (z >= c->L) z = nextafter(c->L, 0.0); }
          if (r >= c->R) { r = 2.0 * c->R - r; vr = -vr; if (r >= c->R) r = nextafter(c->R, 0.0); }
        } else if (z < 0.0 || z >= c->L || r >= c->R) {
          absorbed = 1;
          if (z < 0.0) {
            /* the point where the straight path crossed z = 0 */
            double tc = z0 / (z0 - z);
            double xh = r0 + tc * (x1 - r0), yh = tc * y1;
            double rhit = sqrt(xh * xh + yh * yh);
            if (rhit <= c->Rc) {
              /* cathode impact: tally, and secondary emission with yield
               * gamma at zero velocity (Section 3) */
              double u[4];
              draws(c, sp, p->id[k], s->step, 2, u);
              double gam = sp == 0 ? c->gamma_e : c->gamma_i;
              if (sp == 1) n_ion_cath++; else n_e_cath++;
              /* cathode ion energy distribution (Section 7): impacts in the
               * radial band, energy of the velocity the ion arrives with */
              if (sp == 1 && c->ied_bins > 0 && rhit >= c->band_r_lo && rhit <= c->band_r_hi) {
                double E = 0.5 * mass * (vr * vr + vt * vt + vz * vz) / QE;
                double fb = floor(E / (c->ied_emax / c->ied_bins));
                if (fb < (double)c->ied_bins) s->ied[(int)fb]++; else s->ied_over++;
              }
              if (u[0] < gam) {
                uint64_t key = ((uint64_t)p->id[k] << 2) | (sp == 1 ? 1u : 2u);
                bl_push(&be, key, rhit, 0.0, 0.0, 0.0, 0.0);
                n_sey++;
              }
            }
          }
        }
        if (absorbed) continue;
        p->r[out] = r; p->z[out] = z; p->vr[out] = vr; p->vt[out] = vt; p->vz[out] = vz;
        p->id[out] = p->id[k];
        if (sp == 0 && c->mcc_on) mcc_electron(s, out, &be, &bi);
        ++out;
      }
      p->n = out;
      if (sp == 0) s->d.K_e = K; else s->d.K_i = K;
    }
    /* births: ids in order of (parent id, kind), electrons first, then ions */
    qsort(be.b, (size_t)be.n, sizeof(birth), cmp_birth);
    qsort(bi.b, (size_t)bi.n, sizeof(birth), cmp_birth);
    for (int sp = 0; sp < 2; ++sp) {
      blist* l = sp == 0 ? &be : &bi;
      pstore* p = &s->sp[sp];
      ps_reserve(p, p->n + l->n);
      for (int64_t k = 0; k < l->n; ++k) {
        int64_t j = p->n++;
        p->r[j] = l->b[k].r; p->z[j] = l->b[k].z;
        p->vr[j] = l->b[k].vr; p->vt[j] = l->b[k].vt; p->vz[j] = l->b[k].vz;
        p->id[j] = s->next_id++;
      }
      free(l->b);
    }
    /* deposit at the new positions */
    deposit_all(s);
    /* external circuit (Section 3/4): cathode charge this step, mean current
     * over the last n_avg steps, V_c = -V_s + I R_ext clamped to [-V_s, 0] */
    double qcath = QE * c->weight * (double)(n_ion_cath + n_sey - n_e_cath);
    int na = c->n_avg > 0 ? c->n_avg : 1;
    s->qhist[s->step % na] = qcath;
    int64_t cnt = s->step + 1 < na ? s->step + 1 : na;
    double qs = 0.0;
    for (int64_t k = 0; k < cnt; ++k) qs += s->qhist[k];
    double I = qs / ((double)cnt * c->dt);
    if (c->circuit_mode == 1) {
      double V = -c->Vs + I * c->Rext;
      if (V < -c->Vs) V = -c->Vs;
      if (V > 0.0) V = 0.0;
      s->Vc = V;
    } else {
      s->Vc = c->Vc_fixed;
    }
    solve_phi(s);
    /* diagnostics */
    double pk[2] = {0.0, 0.0};
    for (int m = 0; m <= c->nr; ++m)
      for (int n = 0; n <= c->nz; ++n)
        for (int sp = 0; sp < 2; ++sp) {
          double dens = fabs(s->Qs[sp][nidx(c, m, n)]) / (QE * orc_node_volume(c, m, n));
          if (dens > pk[sp]) pk[sp] = dens;
        }
    s->d.t = s->step * c->dt;
    s->d.I_cath = I;
    s->d.V_cath = s->Vc;
    s->d.n_e_peak = pk[0];
    s->d.n_i_peak = pk[1];
    s->d.N_e = s->sp[0].n;
    s->d.N_i = s->sp[1].n;
    s->d.n_ion_cath = n_ion_cath;
    s->d.n_e_cath = n_e_cath;
    s->d.n_sey = n_sey;
    s->d.ppc_max_e = max_per_cell(s, 0);
    s->d.ppc_max_i = max_per_cell(s, 1);
    s->step++;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Region diagnostics (Sections 4, 5 and 7).  Section 4 puts the sheath     */
/* edge where the electron density is half the ion density and the bulk    */
/* where E_z = d phi / dz vanishes; Section 5 averages the electron         */
/* temperature, from the second moment of the particle velocities, over    */
/* each region within 1.0 cm < r < 1.5 cm; Section 7 bins the energies of   */
/* the ions hitting the cathode in the same radial band.  Readings: the     */
/* state is accumulated over samples (the paper's steady-state averages);   */
/* per cell column m (r_m .. r_{m+1}), walking up from the cathode, the     */
/* sheath ends at the first cell with n_e >= n_i / 2 (2 N_e >= N_i in       */
/* accumulated counts: same cell volume and weight) and the bulk starts at  */
/* the first cell from there on whose axial field E_z = -d phi / dz, from   */
/* the cell's four corner potentials, is >= 0; a cell's temperature is      */
/* m_e (<|v|^2> - |<v>|^2) / (3 e) over its electron samples (cells with    */
/* at least two), and a region's temperature the plain mean over its cells  */
/* whose column centre lies in the band.                                   */
/* ------------------------------------------------------------------------ */
void orc_region_sample(orc_sim* s) {
  const orc_config* c = &s->c;
  for (int sp = 0; sp < 2; ++sp) {
    const pstore* p = &s->sp[sp];
    for (int64_t k = 0; k < p->n; ++k) {
      int m, n;
      double f;
      locate(p->r[k], dr_of(c), c->nr, &m, &f);
      locate(p->z[k], dz_of(c), c->nz, &n, &f);
      size_t cell = (size_t)m * c->nz + n;
      s->rc_n[sp][cell]++;
      if (sp == 0) {
        double vr = p->vr[k], vt = p->vt[k], vz = p->vz[k];
        s->rc_mom[cell * 4 + 0] += vr;
        s->rc_mom[cell * 4 + 1] += vt;
        s->rc_mom[cell * 4 + 2] += vz;
        s->rc_mom[cell * 4 + 3] += vr * vr + vt * vt + vz * vz;
      }
    }
  }
  size_t nn = (size_t)(c->nr + 1) * (c->nz + 1);
  for (size_t i = 0; i < nn; ++i) s->rc_phi[i] += s->phi[i];
  s->rc_samples++;
}

int orc_region_result(const orc_sim* s, orc_regions* out, double* zs, double* zb) {
  const orc_config* c = &s->c;
  memset(out, 0, sizeof(*out));
  out->samples = s->rc_samples;
  double dz = dz_of(c), dr = dr_of(c);
  double tsum[3] = {0.0, 0.0, 0.0};
  double zs_sum = 0.0, zb_sum = 0.0;
  int ncol = 0;
  for (int m = 0; m < c->nr; ++m) {
    int ns = c->nz, nb = c->nz;
    for (int n = 0; n < c->nz; ++n) {
      size_t cell = (size_t)m * c->nz + n;
      if (2 * s->rc_n[0][cell] >= s->rc_n[1][cell]) { ns = n; break; }
    }
    for (int n = ns; n < c->nz; ++n) {
      /* -dphi/dz >= 0  <=>  upper-face potential sum <= lower-face sum */
      double up = s->rc_phi[nidx(c, m, n + 1)] + s->rc_phi[nidx(c, m + 1, n + 1)];
      double lo = s->rc_phi[nidx(c, m, n)] + s->rc_phi[nidx(c, m + 1, n)];
      if (up - lo <= 0.0) { nb = n; break; }
    }
    if (zs) zs[m] = ns * dz;
    if (zb) zb[m] = nb * dz;
    double rcen = (m + 0.5) * dr;
    if (rcen < c->band_r_lo || rcen > c->band_r_hi) continue;
    ++ncol;
    zs_sum += ns * dz;
    zb_sum += nb * dz;
    for (int n = 0; n < c->nz; ++n) {
      size_t cell = (size_t)m * c->nz + n;
      int64_t N = s->rc_n[0][cell];
      if (N < 2) continue;
      const double* mo = &s->rc_mom[cell * 4];
      double mr = mo[0] / N, mt = mo[1] / N, mz = mo[2] / N;
      double T = ME * (mo[3] / N - (mr * mr + mt * mt + mz * mz)) / (3.0 * QE);
      int reg = n < ns ? 0 : (n < nb ? 1 : 2);
      tsum[reg] += T;
      out->ncell[reg]++;
    }
  }
  for (int k = 0; k < 3; ++k) out->Te[k] = out->ncell[k] > 0 ? tsum[k] / out->ncell[k] : 0.0;
  out->z_sheath = ncol > 0 ? zs_sum / ncol : 0.0;
  out->z_bulk = ncol > 0 ? zb_sum / ncol : 0.0;
  int64_t imp = s->ied_over;
  for (int b = 0; b < c->ied_bins; ++b) imp += s->ied[b];
  out->ion_impacts = imp;
  return 0;
}

void orc_ied_get(const orc_sim* s, int64_t* hist, int64_t* overflow) {
  for (int b = 0; b < s->c.ied_bins; ++b) hist[b] = s->ied[b];
  if (overflow) *overflow = s->ied_over;
}

void orc_region_reset(orc_sim* s) {
  const orc_config* c = &s->c;
  size_t ncell = (size_t)c->nr * c->nz, nn = (size_t)(c->nr + 1) * (c->nz + 1);
  memset(s->rc_n[0], 0, ncell * sizeof(int64_t));
  memset(s->rc_n[1], 0, ncell * sizeof(int64_t));
  memset(s->rc_mom, 0, ncell * 4 * sizeof(double));
  memset(s->rc_phi, 0, nn * sizeof(double));
  if (c->ied_bins > 0) memset(s->ied, 0, (size_t)c->ied_bins * sizeof(int64_t));
  s->ied_over = 0;
  s->rc_samples = 0;
}
