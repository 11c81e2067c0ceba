// step.cu -- the per-step particle kernels of the RZ PIC-MCC method.
//
// Order inside one step (arXiv:2507.10727, Sections 2-4):
//   k_field_tables    E from phi (edge-centred for EC-PIC, nodal for MC-PIC)
//                     folded into per-cell gather tables; field energy
//   k_push<e>, <i>    gather + Boris push + walls + secondary emission + MCC,
//                     new cell key, histogram, charge deposit of the new
//                     position into a shared-memory patch (no per-particle
//                     global atomics), births appended to a birth buffer
//   k_births          births sorted by (parent id, kind), ids assigned
//   k_scan            exclusive scan of the cell histogram -> cursors
//   k_scatter         counting-sort scatter into the other buffer
//   k_charge          node charge Q from the fixed-point sums
//   k_circuit         cathode current, V_c, cathode Dirichlet values
//   (Poisson solve, poisson.cu)
//   k_step_end        diagnostics record, counters, step index
#include <cstdio>

#include <cooperative_groups.h>

#include "common.cuh"
#include "device_util.cuh"
#include "launch.h"

namespace pic {

namespace cg = cooperative_groups;

constexpr int kPushThreads = 256;
constexpr int kScanCta = 8;                      // CTAs of one species' scan (a cluster)
constexpr int kHalo = 3;                         // cells a particle may move and still hit the patch
// The deposit patch: (tile extent in r + 2 halo + 1) x (two tiles along z + 2
// halo + 1) nodes; the arrays hold the largest of the tile shapes.
__device__ __forceinline__ int patch_pr(const Inst& I) { return (1 << I.tsr) + 2 * kHalo + 1; }
__device__ __forceinline__ int patch_pz(const Inst& I) { return (2 << I.tsz) + 2 * kHalo + 1; }
constexpr int patch_nodes(int lr, int lz) { return ((1 << lr) + 2 * kHalo + 1) * ((2 << lz) + 2 * kHalo + 1); }
constexpr int patch_cells(int lr, int lz) { return ((1 << lr) + 2 * kHalo) * ((2 << lz) + 2 * kHalo); }
constexpr int cmax(int a, int b) { return a > b ? a : b; }
constexpr int kPatchNodes = cmax(patch_nodes(3, 3), cmax(patch_nodes(4, 3), patch_nodes(3, 4)));
constexpr int kPatchCells = cmax(patch_cells(3, 3), cmax(patch_cells(4, 3), patch_cells(3, 4)));
constexpr int kCollQ = 512;                      // deferred collision candidates per chunk

// ---------------------------------------------------------------------------
// Field gather tables (Section 2).
//  EC-PIC: E_r stored on edges [r_{m+1/2}, z_n], interpolated NGP in r
//  (the cell's own edge) and linear in z; E_z on [r_m, z_{n+1/2}], linear in
//  r and NGP in z.  Table per cell: {E_r(lower z edge), E_r(upper) -
//  E_r(lower), E_z(inner r edge), E_z(outer) - E_z(inner)}; with volume
//  weighting the E_r entries are divided by r_{m+1/2} (dS/dr = 2r / (r_{m+1}^2
//  - r_m^2) gives E_r a factor r / r_{m+1/2}).
//  MC-PIC: nodal E (mean of the adjacent edges, one-sided on conducting
//  walls, no normal component on insulating ones, E_r = 0 on the axis) in
//  bilinear coefficient form in the deposit's weights.
// Field energy (diagnostic): 1/2 sum over edges of a_e (delta phi)^2.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void k_field_tables_body(const Inst& I) {
  const Scalars* S = I.S;
  if (S->status & ST_FATAL) return;
  const int ncell = I.nr * I.nz;
  const bool diag = S->diag_on != 0;
  double wloc = 0.0;
  const int nz1 = I.nz + 1;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) {
    const int m = c / I.nz, n = c - m * I.nz;
    const double* ph = I.phi;
    const double p00 = ph[m * nz1 + n], p01 = ph[m * nz1 + n + 1];
    const double p10 = ph[(m + 1) * nz1 + n], p11 = ph[(m + 1) * nz1 + n + 1];
    const int key = cell_key(I, m, n);
    if (I.gather == 0) {
      double4_32a t = make_d4(0.0, 0.0, 0.0, 0.0);
      if (I.field_on) {
        double er_lo = -(p10 - p00) * I.inv_dr, er_hi = -(p11 - p01) * I.inv_dr;
        double ez_lo = -(p01 - p00) * I.inv_dz, ez_hi = -(p11 - p10) * I.inv_dz;
        if (I.rweight == 1) {
          double s = 1.0 / ((m + 0.5) * I.dr);
          er_lo *= s;
          er_hi *= s;
        }
        t = make_d4(er_lo, er_hi - er_lo, ez_lo, ez_hi - ez_lo);
      }
      if (I.prec32) {
        I.etab32[key] = make_float4((float)t.x, (float)t.y, (float)t.z, (float)t.w);
      } else {
        for (int sp = 0; sp < 2; ++sp) {
          // volume weighting: the push multiplies by r in cell units, r / dr
          const double hs = 0.5 * I.qm[sp] * I.dt, hr = I.rweight == 1 ? hs * I.dr : hs;
          I.etab[sp][key] = make_d4(hr * t.x, hr * t.y, hs * t.z, hs * t.w);
        }
      }
    } else {
      double er[2][2], ez[2][2];
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
          const int mm = m + a, nn = n + b;
          double e;
          if (mm == 0) e = 0.0;
          else if (mm == I.nr)
            e = I.bc_wall ? 0.0 : -(ph[mm * nz1 + nn] - ph[(mm - 1) * nz1 + nn]) * I.inv_dr;
          else e = -(ph[(mm + 1) * nz1 + nn] - ph[(mm - 1) * nz1 + nn]) * (0.5 * I.inv_dr);
          er[a][b] = e;
          if (nn == 0)
            e = field_free(mm, 0, I.nr, I.nz, I.bc_g, I.bc_wall)
                    ? 0.0
                    : -(ph[mm * nz1 + 1] - ph[mm * nz1]) * I.inv_dz;
          else if (nn == I.nz) e = -(ph[mm * nz1 + nn] - ph[mm * nz1 + nn - 1]) * I.inv_dz;
          else e = -(ph[mm * nz1 + nn + 1] - ph[mm * nz1 + nn - 1]) * (0.5 * I.inv_dz);
          ez[a][b] = e;
        }
      double4_32a tr = make_d4(0.0, 0.0, 0.0, 0.0), tz = tr;
      if (I.field_on) {
        tr = make_d4(er[0][0], er[1][0] - er[0][0], er[0][1] - er[0][0],
                          er[1][1] - er[1][0] - er[0][1] + er[0][0]);
        tz = make_d4(ez[0][0], ez[1][0] - ez[0][0], ez[0][1] - ez[0][0],
                          ez[1][1] - ez[1][0] - ez[0][1] + ez[0][0]);
      }
      if (I.prec32) {
        I.etab32[2 * key] = make_float4((float)tr.x, (float)tr.y, (float)tr.z, (float)tr.w);
        I.etab32[2 * key + 1] = make_float4((float)tz.x, (float)tz.y, (float)tz.z, (float)tz.w);
      } else {
        for (int sp = 0; sp < 2; ++sp) {
          const double hs = 0.5 * I.qm[sp] * I.dt;
          I.etab[sp][2 * key] = make_d4(hs * tr.x, hs * tr.y, hs * tr.z, hs * tr.w);
          I.etab[sp][2 * key + 1] = make_d4(hs * tz.x, hs * tz.y, hs * tz.z, hs * tz.w);
        }
      }
    }
    if (diag) {
      // edges owned by this cell: r-edge (m,n), z-edge (m,n); the last row /
      // column also own r-edge (m,nz) and z-edge (nr,n)
      const double c0 = 2.0 * kPi * kEps0;
      const double ar = c0 * (m + 0.5) * I.dz;
      const double az = kEps0 * node_area(I, m) / I.dz;
      double d = p10 - p00;
      wloc += 0.5 * ar * (n == 0 ? 0.5 : 1.0) * d * d;
      d = p01 - p00;
      wloc += 0.5 * az * d * d;
      if (n == I.nz - 1) {
        d = p11 - p01;
        wloc += 0.5 * ar * 0.5 * d * d;
      }
      if (m == I.nr - 1) {
        d = p11 - p10;
        wloc += 0.5 * (kEps0 * node_area(I, I.nr) / I.dz) * d * d;
      }
    }
  }
  if (diag) block_add(wloc, &I.S->W);
}
__global__ void k_field_tables(Inst I) { k_field_tables_body(I); }
__global__ void k_field_tables_b(const Inst* insts) {
  __shared__ Inst sI;
  stage_inst(insts + blockIdx.z, &sI);
  k_field_tables_body(sI);
}

// ---------------------------------------------------------------------------
// births
// ---------------------------------------------------------------------------
// A particle born this step at (r, z) in cell units with velocity (m/s): the
// births buffer of its species, its cell's count and its charge.
__device__ void add_birth(const Inst& I, int sp, unsigned long long pkey, double r, double z,
                          double vr, double vt, double vz) {
  Scalars* S = I.S;
  unsigned long long b = atomicAdd((unsigned long long*)&S->nbirth[sp], 1ULL);
  if ((long long)b >= I.birth_cap) {
    atomicOr(&S->status, ST_CAPACITY);
    return;
  }
  const BirthsDev& B = I.births[sp];
  B.r[b] = r; B.z[b] = z; B.vr[b] = vr; B.vt[b] = vt; B.vz[b] = vz;
  B.pkey[b] = pkey;
  int m, n;
  double fr, fz;
  split_cell(r, I.nr, m, fr);
  split_cell(z, I.nz, n, fz);
  const int key = cell_key(I, m, n);
  B.cell[b] = key;
  atomicAdd(&I.counts[sp][key], 1);
  const FixW f = fix_weights(rweight_upper(I, r, m, fr), fz);
  unsigned long long* q = I.qacc[sp];
  atomicAdd(q + node_index(I, m, n), f.w00);
  atomicAdd(q + node_index(I, m + 1, n), f.w10);
  atomicAdd(q + node_index(I, m, n + 1), f.w01);
  atomicAdd(q + node_index(I, m + 1, n + 1), f.w11);
}

// Null-collision MCC for one electron (Section 3, reactions (1a)-(1d), [14]).
// Returns true when the velocity changed.
// An ionizing collision ((1c) or (1d), threshold Ith): the electron keeps a
// uniform share of E - Ith, a new electron (isotropic) the rest; the ion is born
// with a Maxwellian at the gas temperature.  Returns the primary's new energy.
__device__ double ionize64(const Inst& I, long long id, long long step, double r, double z,
                           double E, double Ith, const double e[3]) {
  double u2[4], g[4];
  draws(I, 0, id, step, 1, u2);
  const double Ex = E - Ith;
  const double Enew = u2[0] * Ex;
  const double E2 = Ex - Enew;
  double d2[3];
  scatter_dir(e, 1.0 - 2.0 * u2[1], 2.0 * kPi * u2[2], d2);
  const double v2 = sqrt(2.0 * E2 * kQe / kMe);
  const unsigned long long key = ((unsigned long long)id << 2) | 0ULL;
  add_birth(I, 0, key, r, z, v2 * d2[0], v2 * d2[1], v2 * d2[2]);
  draws(I, 0, id, step, 4, g);
  const double sig = sqrt(kBoltz * I.T_gas / I.m_ion);
  const double rho1 = sqrt(-2.0 * log(1.0 - g[0])), th1 = 2.0 * kPi * g[1];
  const double rho2 = sqrt(-2.0 * log(1.0 - g[2])), th2 = 2.0 * kPi * g[3];
  double s1, c1, s2, c2;
  sincos(th1, &s1, &c1);
  sincos(th2, &s2, &c2);
  add_birth(I, 1, key, r, z, sig * rho1 * c1, sig * rho1 * s1, sig * rho2 * c2);
  return Enew;
}

__device__ bool mcc_electron(const Inst& I, long long id, long long step, double r, double z,
                             double& vr, double& vt, double& vz) {
  // a candidate (mcc_candidate): process and angles from words 1..3 of stream 0
  unsigned long long w[4];
  philox4x64((unsigned long long)id, (unsigned long long)step, 0ULL, 0ULL, I.seed, 0ULL, w);
  double u[4];
  u[1] = u01(w[1]); u[2] = u01(w[2]); u[3] = u01(w[3]);
  const double v[3] = {vr, vt, vz};
  const double vmag = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  const double E = 0.5 * kMe * vmag * vmag / kQe;
  const double s_el = E > 0.0 ? I.sigma_el : 0.0;
  const double s_ex = E > I.exc_E ? I.exc_C * log(E / I.exc_E) / (E * I.exc_E) : 0.0;
  const double s_io = E > I.ion_I ? I.ion_a * log(E / I.ion_I) / (E * I.ion_I) : 0.0;
  const double s_md = E > I.meta_I ? I.meta_a * log(E / I.meta_I) / (E * I.meta_I) : 0.0;
  const double nu_el = I.n_gas * s_el * vmag, nu_ex = I.n_gas * s_ex * vmag;
  const double nu_io = I.n_gas * s_io * vmag;
  const double nu_md = I.n_meta * s_md * vmag;
  const double R = u[1] * I.nu_max;
  const double inv = vmag > 0.0 ? 1.0 / vmag : 1.0;
  const double e[3] = {v[0] * inv, v[1] * inv, v[2] * inv};
  const double cos_chi = 1.0 - 2.0 * u[2], phi = 2.0 * kPi * u[3];
  double Enew;
  Scalars* S = I.S;
  if (R < nu_el) {
    Enew = E * (1.0 - 2.0 * kMe / I.m_ion * (1.0 - cos_chi));
    atomicAdd(&S->cnt_elastic, 1ULL);
  } else if (R < nu_el + nu_ex) {
    Enew = E - I.exc_E;
    atomicAdd(&S->cnt_excite, 1ULL);
  } else if (R < nu_el + nu_ex + nu_io) {
    Enew = ionize64(I, id, step, r, z, E, I.ion_I, e);
    atomicAdd(&S->cnt_ionize, 1ULL);
  } else if (R < nu_el + nu_ex + nu_io + nu_md) {
    Enew = ionize64(I, id, step, r, z, E, I.meta_I, e);
    atomicAdd(&S->cnt_ionize_meta, 1ULL);
  } else {
    return false;
  }
  double d[3];
  scatter_dir(e, cos_chi, phi, d);
  const double vn = sqrt(2.0 * Enew * kQe / kMe);
  vr = vn * d[0];
  vt = vn * d[1];
  vz = vn * d[2];
  return true;
}

// The collision of a queued candidate i, on its state after the move.
__device__ __noinline__ void collide_at(const Inst& I, const ParticlesDev& P, long long i,
                                           long long step) {
  double vr = P.vr[i], vt = P.vt[i], vz = P.vz[i];
  if (mcc_electron(I, P.id[i], step, P.r[i], P.z[i], vr, vt, vz)) {
    P.vr[i] = vr;
    P.vt[i] = vt;
    P.vz[i] = vz;
  }
}

// ---------------------------------------------------------------------------
// The push.  One CTA processes chunks of ppt x kPushThreads consecutive
// (cell-sorted) particles, warp w the contiguous run of 32 ppt of them from
// c0 + 32 ppt w, 32 consecutive particles per iteration.  A lane therefore
// meets the same new cell over many iterations: it sums its fixed-point
// deposit weights and its cell count in registers (integers: exact, order
// free) and adds them, when its cell changes, to the CTA's shared patches of
// pr x pz nodes (charge) and pr-1 x pz-1 cells (counts) anchored at the
// tile of the chunk's first particle, flushed with one atomic per touched
// node or cell.  Cells whose nodes fall outside the patch (fast movers, chunk
// tails in sparse regions) add to global memory.
// ---------------------------------------------------------------------------
template <int SP>
__device__ __forceinline__ void deposit_run64(const Inst& I, int key, int m, int n,
                                              unsigned long long a00, unsigned long long a10,
                                              unsigned long long a01, unsigned long long a11,
                                              int cnt, int pm0, int pn0, int pr, int pz,
                                              unsigned long long* patch, int* cpatch) {
  const int lm = m - pm0, ln = n - pn0;
  if (lm >= 0 && lm + 1 < pr && ln >= 0 && ln + 1 < pz) {
    unsigned long long* p = patch + lm * pz + ln;
    atomicAdd(p, a00);
    atomicAdd(p + pz, a10);
    atomicAdd(p + 1, a01);
    atomicAdd(p + pz + 1, a11);
    atomicAdd(cpatch + lm * (pz - 1) + ln, cnt);
  } else {
    unsigned long long* q = I.qacc[SP];
    atomicAdd(q + node_index(I, m, n), a00);
    atomicAdd(q + node_index(I, m + 1, n), a10);
    atomicAdd(q + node_index(I, m, n + 1), a01);
    atomicAdd(q + node_index(I, m + 1, n + 1), a11);
    atomicAdd(&I.counts[SP][key], cnt);
  }
}

// The flush of the lanes whose cell changed this iteration (flag fl), by the
// whole warp: lanes of one cell form runs of adjacent lanes (they hold
// consecutive particles); a segmented suffix sum by shuffles leaves each run's
// sums in its first lane, which alone adds the cell's four node weights to the
// patch (lanes of one cell would conflict on the same shared words).  The open
// sums are sr = sum round(w_r 2^44), sz = sum round(w_z 2^44), srz = sum of the
// rounded products and the count c; integer sums, so the result is exact and
// independent of the grouping.  All 32 lanes must take part.
template <int SP>
__device__ __forceinline__ void warp_flush64(const Inst& I, bool fl, int key, int m, int n,
                                             unsigned long long sr, unsigned long long sz,
                                             unsigned long long srz, int cnt, int pm0, int pn0,
                                             int pr, int pz, unsigned long long* patch, int* cpatch,
                                             int lane) {
  const unsigned full = 0xffffffffu;
  const int k = fl ? key : -1;
  const int kprev = __shfl_up_sync(full, k, 1);
  const bool head = fl && (lane == 0 || kprev != k);
  const unsigned starts = __ballot_sync(full, head || !fl);
  const unsigned above = lane == 31 ? 0u : (starts & (full << (lane + 1)));
  const int end = above ? __ffs(above) - 1 : 32;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned long long br = __shfl_down_sync(full, sr, off);
    const unsigned long long bz = __shfl_down_sync(full, sz, off);
    const unsigned long long brz = __shfl_down_sync(full, srz, off);
    const int bc = __shfl_down_sync(full, cnt, off);
    if (lane + off < end) {
      sr += br;
      sz += bz;
      srz += brz;
      cnt += bc;
    }
  }
  if (head)
    deposit_run64<SP>(I, key, m, n, ((unsigned long long)cnt << kFixBits) - sr - sz + srz,
                      sr - srz, sz - srz, srz, cnt, pm0, pn0, pr, pz, patch, cpatch);
}

// Push the chunk of `ppt * blockDim.x` particles of species SP starting at c0
// (the whole CTA takes part).  `patch` is the CTA's zeroed shared deposit
// patch; it is flushed and zeroed again before return.  `anchor` holds the
// patch origin and the candidate count, `cq` the chunk's collision candidates:
// the collision itself changes only the velocity, so it runs after the chunk
// with the candidates packed onto consecutive lanes (a warp that met one
// candidate inside the loop would run the whole collision for one lane).
// Returns this thread's share of the kinetic energy (diagnostic steps only).
template <int SP, int GATHER, bool PLAIN>
__device__ __forceinline__ double push_chunk64(const Inst& I, long long c0, int ppt,
                                               unsigned long long* patch, int* cpatch, int* anchor,
                                               int* cq) {
  Scalars* S = I.S;
  const long long n = S->n[SP];
  const long long step = S->step;
  const bool diag = S->diag_on != 0;
  const ParticlesDev P = I.buf[SP][S->flip[SP]];
  const double4_32a* etab = I.etab[SP];   // h E, h B of this species (h = q dt / 2m)
  const double4_32a* btab = I.btab[SP];
  const int lane = threadIdx.x & 31;
  double Kloc = 0.0;
  {
    if (threadIdx.x == 0) {
      int m, nn;
      double f;
      split_cell(P.r[c0], I.nr, m, f);
      split_cell(P.z[c0], I.nz, nn, f);
      anchor[0] = (m & ~((1 << I.tsr) - 1)) - kHalo;
      anchor[1] = (nn & ~((1 << I.tsz) - 1)) - kHalo;
      anchor[2] = 0;
    }
    __syncthreads();
    const int pm0 = anchor[0], pn0 = anchor[1];
    const int pr = patch_pr(I), pz = patch_pz(I);
    const long long run0 = c0 + (long long)(threadIdx.x >> 5) * 32 * ppt + lane;
    // this lane's open deposit: cell, its fixed-point weight sums and count
    int acc_key = -1, acc_m = 0, acc_n = 0, acc_cnt = 0;
    unsigned long long sr = 0ULL, sz = 0ULL, srz = 0ULL;
    unsigned over = 0u;   // candidates that found the queue full, bit j (ppt <= 32)
#pragma unroll 1
    for (int j = 0; j < ppt; ++j) {
      const long long i = run0 + (long long)j * 32;
      int newkey = -1;
      bool add = false, fl = false;   // this particle's deposit; flush of the open sums
      int nm = 0, nn1 = 0;
      unsigned long long ir = 0ULL, iz = 0ULL, i11 = 0ULL;
      // between full sorts the arrays hold dead slots, marked by r = -1
      const bool live = i < n && (long long)bits_of(P.r[i]) >= 0;
      if (!live) {
        if (i < n) I.key[SP][i] = -1;
      } else {
        double r = P.r[i], z = P.z[i], vr = P.vr[i], vt = P.vt[i], vz = P.vz[i];
        const double v2old = vr * vr + vt * vt + vz * vz;
        double x1 = r, y1 = 0.0, r1 = r, z1 = z;
        if (PLAIN || I.push_on) {
          int m, nn;
          double fr, fz;
          split_cell(r, I.nr, m, fr);
          split_cell(z, I.nz, nn, fz);
          const int ck = cell_key(I, m, nn);
          // gather h E
          double hEr, hEz;
          if (GATHER == 0) {
            const double4_32a t = etab[ck];
            const double wr = PLAIN ? fr : rweight_upper(I, r, m, fr);
            hEr = t.x + t.y * fz;
            if (!PLAIN && I.rweight == 1) hEr *= r;
            hEz = t.z + t.w * wr;
          } else {
            const double wr = PLAIN ? fr : rweight_upper(I, r, m, fr);
            const double4_32a a = etab[2 * ck];
            const double4_32a b = etab[2 * ck + 1];
            hEr = a.x + wr * (a.y + fz * a.w) + fz * a.z;
            hEz = b.x + wr * (b.y + fz * b.w) + fz * b.z;
          }
          // gather t = h B (bilinear node table)
          const double4_32a br = btab[2 * ck];
          const double4_32a bz = btab[2 * ck + 1];
          const double tx = br.x + fr * (br.y + fz * br.w) + fz * br.z;
          const double tz = bz.x + fr * (bz.y + fz * bz.w) + fz * bz.z;
          // Boris: half kick, rotation about B, half kick
          const double ax = vr + hEr, ay = vt, az = vz + hEz;
          const double f2 = recip2(1.0 + tx * tx + tz * tz);   // 2 / (1 + t^2), 1 + t^2 >= 1
          const double sx = f2 * tx, sz = f2 * tz;
          const double px = ax + ay * tz;
          const double py = fma(az, tx, fma(-ax, tz, ay));   // ay + (az tx - ax tz), two FMAs
          const double pz = az - ay * tx;
          const double vx = ax + py * sz + hEr;
          const double vy = fma(pz, sx, fma(-px, sz, ay));   // ay + (pz sx - px sz)
          const double vzn = az - py * sx + hEz;
          // straight move (in cell units), then rotate the frame onto the new radius
          x1 = r + vx * I.kr64;
          y1 = vy * I.kr64;
          z1 = z + vzn * I.kz64;
          const double s2 = x1 * x1 + y1 * y1;
          if (nonzero_sq(s2)) {   // s2 > 0 (a NaN goes on and is flagged below)
            const double inv = rsqrt(s2);
            r1 = s2 * inv;
            vr = (x1 * vx + y1 * vy) * inv;
            vt = (x1 * vy - y1 * vx) * inv;
          } else {
            r1 = 0.0;
            vr = vx;
            vt = vy;
          }
          vz = vzn;
        }
        if (diag) Kloc += 0.5 * I.mass[SP] * I.weight * 0.5 * (v2old + vr * vr + vt * vt + vz * vz);
        bool alive = true;
        const double Lc = (double)I.nz, Rw = (double)I.nr;   // z = L, r = R in cell units
        if (!PLAIN && I.walls_reflect) {
          if (z1 < 0.0) { z1 = -z1; vz = -vz; }
          if (z1 >= Lc) { z1 = 2.0 * Lc - z1; vz = -vz; if (z1 >= Lc) z1 = nextafter(Lc, 0.0); }
          if (r1 >= Rw) { r1 = 2.0 * Rw - r1; vr = -vr; if (r1 >= Rw) r1 = nextafter(Rw, 0.0); }
        } else if (lt_zero(z1) || ge_pos(z1, Lc) || ge_pos(r1, Rw)) {   // integer-pipe compares
          alive = false;
          if (lt_zero(z1)) {
            const double tc = z / (z - z1);
            const double xh = r + tc * (x1 - r), yh = tc * y1;
            const double rhit = sqrt(xh * xh + yh * yh);   // cell units
            if (rhit <= I.Rc * I.inv_dr) {
              // cathode impact (Section 3): tally; secondary electron with
              // probability gamma, born at the impact point at rest
              atomicAdd(SP == 1 ? &S->cnt_ion_cath : &S->cnt_e_cath, 1ULL);
              // ion energy distribution on the cathode band (Section 7)
              if (SP == 1 && I.ied_bins > 0 && rhit * I.dr >= I.band_lo && rhit * I.dr <= I.band_hi) {
                const double E = 0.5 * I.mass[1] * (vr * vr + vt * vt + vz * vz) / kQe;
                const double fb = floor(E / I.ied_de);
                atomicAdd(&I.reg.ied[fb < (double)I.ied_bins ? (int)fb : I.ied_bins], 1ULL);
              }
              if (I.gamma[SP] > 0.0) {
                const long long id = P.id[i];
                double u[4];
                draws(I, SP, id, step, 2, u);
                if (u[0] < I.gamma[SP]) {
                  atomicAdd(&S->cnt_sey, 1ULL);
                  add_birth(I, 0, ((unsigned long long)id << 2) | (SP == 1 ? 1ULL : 2ULL), rhit,
                            0.0, 0.0, 0.0, 0.0);
                }
              }
            }
          }
        }
        if (alive) {
          // a non-finite velocity component makes the new position non-finite
          if (!(finite64(r1) && finite64(z1))) {
            atomicOr(&S->status, ST_NAN);
            alive = false;
          }
        }
        if (alive) {
          if (SP == 0 && I.mcc_on) {
            const long long id = P.id[i];
            if (mcc_candidate(I, id, step)) {
              const int slot = atomicAdd(&anchor[2], 1);
              if (slot < kCollQ) cq[slot] = (int)(i - c0);
              else over |= 1u << j;   // queue full: this thread runs it after the queue
            }
          }
          int m1, n1;
          double fr1, fz1;
          split_cell(r1, I.nr, m1, fr1);
          split_cell(z1, I.nz, n1, fz1);
          newkey = cell_key(I, m1, n1);
          P.r[i] = r1; P.z[i] = z1; P.vr[i] = vr; P.vt[i] = vt; P.vz[i] = vz;
          // deposit weights of x^{n+1} (Section 2: tent functions), summed per
          // cell; a lane whose cell changes flushes its open sums below
          fix_parts(PLAIN ? fr1 : rweight_upper(I, r1, m1, fr1), fz1, ir, iz, i11);
          add = true;
          nm = m1;
          nn1 = n1;
          fl = newkey != acc_key && acc_key >= 0;
        } else {
          P.r[i] = -1.0;   // dead slot until the next full sort
        }
        I.key[SP][i] = newkey;
      }
      if (__any_sync(0xffffffffu, fl))
        warp_flush64<SP>(I, fl, acc_key, acc_m, acc_n, sr, sz, srz, acc_cnt, pm0, pn0, pr, pz,
                         patch, cpatch, lane);
      if (add) {
        if (newkey != acc_key) {
          acc_key = newkey;
          acc_m = nm;
          acc_n = nn1;
          acc_cnt = 0;
          sr = sz = srz = 0ULL;
        }
        sr += ir;
        sz += iz;
        srz += i11;
        ++acc_cnt;
      }
    }
    warp_flush64<SP>(I, acc_key >= 0, acc_key, acc_m, acc_n, sr, sz, srz, acc_cnt, pm0, pn0, pr,
                     pz, patch, cpatch, lane);
    __syncthreads();
    if (SP == 0) {
      // the queued collisions (Section 3), on the state written above
      const int nq = min(anchor[2], kCollQ);
      for (int k = threadIdx.x; k < nq; k += blockDim.x) collide_at(I, P, c0 + cq[k], step);
      while (over) {
        const int j = __ffs(over) - 1;
        over &= over - 1;
        collide_at(I, P, run0 + (long long)j * 32, step);
      }
    }
    // flush the patches
    for (int k = threadIdx.x; k < pr * pz; k += blockDim.x) {
      const unsigned long long v = patch[k];
      if (v != 0ULL) {
        const int gm = pm0 + k / pz, gn = pn0 + k % pz;
        atomicAdd(I.qacc[SP] + node_index(I, gm, gn), v);
        patch[k] = 0ULL;
      }
    }
    for (int k = threadIdx.x; k < (pr - 1) * (pz - 1); k += blockDim.x) {
      const int c = cpatch[k];
      if (c != 0) {
        const int gm = pm0 + k / (pz - 1), gn = pn0 + k % (pz - 1);
        atomicAdd(&I.counts[SP][cell_key(I, gm, gn)], c);
        cpatch[k] = 0;
      }
    }
    __syncthreads();
  }
  return diag ? Kloc : 0.0;
}

// The push of both species of every instance: persistent CTAs take (instance,
// species, chunk) items from the work queue; an instance's parameters are
// staged in shared memory when a CTA moves to it.
template <int GATHER, bool PLAIN>
__global__ void __launch_bounds__(kPushThreads, 2) k_push_all(const Inst* insts, WorkQueue* q,
                                                               int ppt) {
  __shared__ unsigned long long patch[kPatchNodes];
  __shared__ int cpatch[kPatchCells];
  __shared__ int anchor[3];
  __shared__ int cq[kCollQ];
  __shared__ Inst sI;
  __shared__ int s_inst, s_sp, s_skip;
  __shared__ long long s_c0;
  for (int k = threadIdx.x; k < kPatchNodes; k += blockDim.x) patch[k] = 0ULL;
  for (int k = threadIdx.x; k < kPatchCells; k += blockDim.x) cpatch[k] = 0;
  int cur = -1;
  double K0 = 0.0, K1 = 0.0;
  const long long chunk = (long long)ppt * blockDim.x;
  for (;;) {
    if (threadIdx.x == 0) {
      const int item = (int)atomicAdd(&q->next, 1u);
      int inst = -1, sp = 0, c = 0;
      if (!queue_item(q, item, inst, sp, c)) inst = -1;
      s_inst = inst;
      s_sp = sp;
      s_c0 = (long long)c * chunk;
      // one reading of the status word for the whole CTA (it may change
      // while the kernel runs; the chunk's barriers need a uniform decision)
      s_skip = inst >= 0 ? (*(volatile int*)&insts[inst].S->status & ST_FATAL) : 0;
    }
    __syncthreads();
    const int inst = s_inst;
    // a CTA may find the queue empty on its first fetch (cur == -1 == inst)
    if (inst != cur || inst < 0) {
      if (cur >= 0 && sI.S->diag_on) {
        block_add(K0, &sI.S->K[0]);
        block_add(K1, &sI.S->K[1]);
      }
      K0 = K1 = 0.0;
      if (inst < 0) break;
      const unsigned* src = reinterpret_cast<const unsigned*>(insts + inst);
      unsigned* dst = reinterpret_cast<unsigned*>(&sI);
      for (int k = threadIdx.x; k < (int)(sizeof(Inst) / 4); k += blockDim.x) dst[k] = src[k];
      __syncthreads();
      cur = inst;
    }
    if (!s_skip) {
      if (s_sp == 0) K0 += push_chunk64<0, GATHER, PLAIN>(sI, s_c0, ppt, patch, cpatch, anchor, cq);
      else K1 += push_chunk64<1, GATHER, PLAIN>(sI, s_c0, ppt, patch, cpatch, anchor, cq);
    }
    __syncthreads();
  }
}

// The FP64 push of a single-instance handle: the instance's parameters are a
// kernel argument (constant-bank operands in the particle loop instead of
// shared-memory loads); otherwise k_push_all.
template <int GATHER, bool PLAIN>
__global__ void __launch_bounds__(kPushThreads, 2) k_push_one(const Inst I, WorkQueue* q,
                                                               int ppt) {
  __shared__ unsigned long long patch[kPatchNodes];
  __shared__ int cpatch[kPatchCells];
  __shared__ int anchor[3];
  __shared__ int cq[kCollQ];
  __shared__ int s_sp, s_done, s_skip;
  __shared__ long long s_c0;
  for (int k = threadIdx.x; k < kPatchNodes; k += blockDim.x) patch[k] = 0ULL;
  for (int k = threadIdx.x; k < kPatchCells; k += blockDim.x) cpatch[k] = 0;
  double K0 = 0.0, K1 = 0.0;
  const long long chunk = (long long)ppt * blockDim.x;
  for (;;) {
    if (threadIdx.x == 0) {
      const int item = (int)atomicAdd(&q->next, 1u);
      int inst = -1, sp = 0, c = 0;
      if (!queue_item(q, item, inst, sp, c)) inst = -1;
      s_done = inst < 0;
      s_sp = sp;
      s_c0 = (long long)c * chunk;
      s_skip = *(volatile int*)&I.S->status & ST_FATAL;
    }
    __syncthreads();
    if (s_done) break;
    if (!s_skip) {
      if (s_sp == 0) K0 += push_chunk64<0, GATHER, PLAIN>(I, s_c0, ppt, patch, cpatch, anchor, cq);
      else K1 += push_chunk64<1, GATHER, PLAIN>(I, s_c0, ppt, patch, cpatch, anchor, cq);
    }
    __syncthreads();
  }
  if (I.S->diag_on) {
    block_add(K0, &I.S->K[0]);
    block_add(K1, &I.S->K[1]);
  }
}

// ---------------------------------------------------------------------------
// Births: the births of a step get ids next_id, next_id + 1, ... in order of
// (parent id, kind), electrons first, then ions.  Only each birth's rank is
// needed: chunks of kBirthChunk keys are sorted in shared memory, one CTA per
// chunk (k_births_sort); a birth's rank is its place in its own sorted chunk
// plus, for every other chunk, the number of keys there below it (binary
// search; the keys are distinct) (k_births_rank); next_id advances last
// (k_births_commit).
// ---------------------------------------------------------------------------
constexpr int kBirthChunk = 8192;
constexpr int kBirthSmem = kBirthChunk * (8 + 4);

__device__ __forceinline__ long long births_of(const Inst& I, int sp) {
  const long long nb = I.S->nbirth[sp];
  return nb < I.birth_cap ? nb : I.birth_cap;
}

__device__ __forceinline__ void k_births_sort_body(const Inst& I) {
  if (I.S->status & ST_FATAL) return;
  extern __shared__ __align__(16) unsigned char bsm[];
  unsigned long long* key = reinterpret_cast<unsigned long long*>(bsm);
  unsigned int* idx = reinterpret_cast<unsigned int*>(key + kBirthChunk);
  const long long c0 = (long long)blockIdx.x * kBirthChunk;
  {
    const int sp = blockIdx.y;                       // the species' chunks sort side by side
    const long long nb = births_of(I, sp);
    if (c0 >= nb) return;                            // uniform over the block
    const int len = (int)(nb - c0 < kBirthChunk ? nb - c0 : kBirthChunk);
    int P = 1;
    while (P < len) P <<= 1;
    const BirthsDev B = I.births[sp];
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
      key[i] = i < len ? B.pkey[c0 + i] : ~0ULL;
      idx[i] = (unsigned int)(c0 + i);
    }
    __syncthreads();
    bitonic(key, idx, P);
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
      B.skey[c0 + i] = key[i];
      B.sidx[c0 + i] = idx[i];
    }
    __syncthreads();
  }
}
__global__ void __launch_bounds__(1024) k_births_sort(Inst I) { k_births_sort_body(I); }
__global__ void __launch_bounds__(1024) k_births_sort_b(const Inst* insts) {
  __shared__ Inst sI;
  stage_inst(insts + blockIdx.z, &sI);
  k_births_sort_body(sI);
}

template <bool F32>
__device__ __forceinline__ void k_births_rank_body(const Inst& I) {
  const Scalars* S = I.S;
  if (S->status & ST_FATAL) return;
  const long long nb0 = births_of(I, 0), nb1 = births_of(I, 1);
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nb0 + nb1;
       e += (long long)gridDim.x * blockDim.x) {
    const int sp = e < nb0 ? 0 : 1;
    const long long nb = sp == 0 ? nb0 : nb1, q = sp == 0 ? e : e - nb0;
    const BirthsDev B = I.births[sp];
    const unsigned long long k = B.skey[q];
    const long long c = q / kBirthChunk;
    long long rank = q - c * kBirthChunk;
    for (long long o = 0; o < nb; o += kBirthChunk) {
      if (o == c * kBirthChunk) continue;
      long long lo = 0, hi = nb - o < kBirthChunk ? nb - o : kBirthChunk;   // keys below k
      while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (B.skey[o + mid] < k) lo = mid + 1;
        else hi = mid;
      }
      rank += lo;
    }
    const unsigned long long id =
        (unsigned long long)(S->next_id + (sp == 0 ? 0 : nb0) + rank);
    const unsigned int b = B.sidx[q];
    if (F32) {
      unsigned int* rec = reinterpret_cast<unsigned int*>(B.b32 + b);
      rec[2] = (unsigned int)(id & 0xffffffffULL);
      rec[3] = (unsigned int)(id >> 32);
    } else {
      B.id[b] = (long long)id;
    }
  }
}
template <bool F32>
__global__ void k_births_rank(Inst I) { k_births_rank_body<F32>(I); }
template <bool F32>
__global__ void k_births_rank_b(const Inst* insts) {
  __shared__ Inst sI;
  stage_inst(insts + blockIdx.z, &sI);
  k_births_rank_body<F32>(sI);
}

__device__ __forceinline__ void k_births_commit_body(const Inst& I) {
  Scalars* S = I.S;
  if (threadIdx.x == 0 && !(S->status & ST_FATAL))
    S->next_id += births_of(I, 0) + births_of(I, 1);
}
__global__ void k_births_commit(Inst I) { k_births_commit_body(I); }
__global__ void k_births_commit_b(const Inst* insts) {
  __shared__ Inst sI;
  stage_inst(insts + blockIdx.z, &sI);
  k_births_commit_body(sI);
}

cudaError_t launch_births(const Inst& I, int num_sms, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_births_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, kBirthSmem);
    attr = true;
  }
  const int chunks = (int)((I.birth_cap + kBirthChunk - 1) / kBirthChunk);
  k_births_sort<<<dim3(chunks > 0 ? chunks : 1, 2), 1024, kBirthSmem, st>>>(I);
  const long long work = 2 * I.birth_cap;
  const int blocks = (int)((work + 255) / 256 < (long long)num_sms * 4 ? (work + 255) / 256
                                                                       : (long long)num_sms * 4);
  if (I.prec32) k_births_rank<true><<<blocks > 0 ? blocks : 1, 256, 0, st>>>(I);
  else k_births_rank<false><<<blocks > 0 ? blocks : 1, 256, 0, st>>>(I);
  k_births_commit<<<1, 32, 0, st>>>(I);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Exclusive scan of the cell histogram of one species -> cursors; clears the
// histogram; n_next = total (checked against the capacity).
// ---------------------------------------------------------------------------
// One species' scan runs on a cluster of kScanCta CTAs (distributed shared
// memory): CTA c owns a contiguous kScanCta-th of the keys and thread t of it
// `per` consecutive keys (per a multiple of 4).  One pass sums them, a
// block-wide scan of the thread sums gives the CTA's total, the CTAs read
// the totals of the lower ranks after a cluster barrier, and a second pass
// (from L1/L2) writes the bin starts and clears the counts.  A CTA stays
// until every CTA has read its totals (second cluster barrier).
__device__ __forceinline__ void k_scan_body(const Inst& I, int sp0) {
  cg::cluster_group cl = cg::this_cluster();
  Scalars* S = I.S;
  // every CTA takes part in the cluster barriers, so a fatal status skips
  // the work instead of returning (it is read before any CTA writes it)
  const bool fatal = (S->status & ST_FATAL) != 0;
  const int rank = (int)cl.block_rank();
  const int sp = sp0 + (int)(blockIdx.x / kScanCta);
  int* counts = I.counts[sp];
  int* cursor = I.cursor[sp];
  __shared__ int wsum[32], wmax[32];
  __shared__ int ctot, cmaxv;            // this CTA's total and largest count
  __shared__ int sbase, stotal, smax;    // lower ranks' total; the cluster's
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (int)blockDim.x >> 5;
  const int nkey = fatal ? 0 : I.nkey;
  const int span = kScanCta * (int)blockDim.x;
  const int per = ((nkey + span - 1) / span + 3) & ~3;
  const int i0 = (rank * (int)blockDim.x + (int)threadIdx.x) * per;
  int vmax = 0;   // most particles in one cell
  int s = 0;
  for (int k = 0; k < per; k += 4) {
    const int i = i0 + k;
    if (i + 3 < nkey) {
      const int4 v = *reinterpret_cast<const int4*>(counts + i);
      s += v.x + v.y + v.z + v.w;
      vmax = max(vmax, max(max(v.x, v.y), max(v.z, v.w)));
    } else {
      for (int q = i; q < nkey && q < i + 4; ++q) {
        const int v = counts[q];
        s += v;
        vmax = max(vmax, v);
      }
    }
  }
  int incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) vmax = max(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
  if (lane == 31) wsum[w] = incl;
  if (lane == 0) wmax[w] = vmax;
  __syncthreads();
  if (w == 0) {
    int x = lane < nw ? wsum[lane] : 0;
    int m = lane < nw ? wmax[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += t;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    wsum[lane] = x;  // inclusive over warps
    if (lane == 31) {
      ctot = x;
      cmaxv = m;
    }
  }
  cl.sync();   // every CTA's total and maximum are written
  if (w == 0) {
    int t = 0, m = 0;
    if (lane < kScanCta) {
      t = *cl.map_shared_rank(&ctot, (unsigned)lane);
      m = *cl.map_shared_rank(&cmaxv, (unsigned)lane);
    }
    const int below = lane < rank ? t : 0;
    int tb = below, tt = t;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      tb += __shfl_xor_sync(0xffffffffu, tb, o);
      tt += __shfl_xor_sync(0xffffffffu, tt, o);
      m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    if (lane == 0) {
      sbase = tb;
      stotal = tt;
      smax = m;
    }
  }
  cl.sync();   // the remote reads are done; sbase, stotal, smax visible to the CTA
  int off = sbase + (w > 0 ? wsum[w - 1] : 0) + (incl - s);
  for (int k = 0; k < per; k += 4) {
    const int i = i0 + k;
    if (i + 3 < nkey) {
      const int4 v = *reinterpret_cast<const int4*>(counts + i);
      int4 c;
      c.x = off;
      c.y = c.x + v.x;
      c.z = c.y + v.y;
      c.w = c.z + v.z;
      off = c.w + v.w;
      *reinterpret_cast<int4*>(cursor + i) = c;
      *reinterpret_cast<int4*>(counts + i) = make_int4(0, 0, 0, 0);
    } else {
      for (int q = i; q < nkey && q < i + 4; ++q) {
        const int v = counts[q];
        cursor[q] = off;
        counts[q] = 0;
        off += v;
      }
    }
  }
  if (rank == 0 && threadIdx.x == 0 && !fatal) {
    S->ppc_max[sp] = smax;
    S->n_next[sp] = stotal;
    if (stotal > I.cap[sp]) atomicOr(&S->status, ST_CAPACITY);
    // FP64 deposit: a node's u64 sum of 2^44-scaled weights holds fewer than
    // 2^20 macroparticles, and a node gathers from at most 4 cells
    if (!I.prec32 && 4LL * smax >= (1LL << (64 - kFixBits))) atomicOr(&S->status, ST_CAPACITY);
  }
}
__global__ void __cluster_dims__(kScanCta, 1, 1) __launch_bounds__(1024)
    k_scan(Inst I, int sp0) { k_scan_body(I, sp0); }
__global__ void __cluster_dims__(kScanCta, 1, 1) __launch_bounds__(1024)
    k_scan_b(const Inst* insts, int sp0) {
  __shared__ Inst sI;
  stage_inst(insts + blockIdx.z, &sI);
  k_scan_body(sI, sp0);
}

// ---------------------------------------------------------------------------
// Counting-sort scatter cur -> nxt of the surviving particles and the
// births (blockIdx.y = species).  per_step: on a step without the full sort
// (sort_this_step) the births are appended to the current arrays instead.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void k_scatter_body(const Inst& I, int sp0, int per_step) {
  Scalars* S = I.S;
  if (S->status & ST_FATAL) return;
  const int sp = sp0 + blockIdx.y;
  const long long n_old = S->n[sp];
  const long long nb = S->nbirth[sp] < I.birth_cap ? S->nbirth[sp] : I.birth_cap;
  const long long total = n_old + nb;
  const int fl = S->flip[sp];
  const ParticlesDev src = I.buf[sp][fl], dst = I.buf[sp][fl ^ 1];
  const BirthsDev B = I.births[sp];
  if (per_step && !sort_this_step(I, S)) return;   // k_append does this step
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarp = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long base = warp * 32; base < total; base += nwarp * 32) {
    const long long i = base + lane;
    int key = -1;
    if (i < n_old) key = I.key[sp][i];
    else if (i < total) key = B.cell[i - n_old];
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int leader = __ffs(peers) - 1;
    int pos0 = 0;
    if (lane == leader && key >= 0) pos0 = atomicAdd(&I.cursor[sp][key], __popc(peers));
    pos0 = __shfl_sync(0xffffffffu, pos0, leader);
    if (key >= 0) {
      const int pos = pos0 + __popc(peers & ((1u << lane) - 1u));
      if (i < n_old) {
        dst.r[pos] = src.r[i]; dst.z[pos] = src.z[i];
        dst.vr[pos] = src.vr[i]; dst.vt[pos] = src.vt[i]; dst.vz[pos] = src.vz[i];
        dst.id[pos] = src.id[i];
      } else {
        const long long b = i - n_old;
        dst.r[pos] = B.r[b]; dst.z[pos] = B.z[b];
        dst.vr[pos] = B.vr[b]; dst.vt[pos] = B.vt[b]; dst.vz[pos] = B.vz[b];
        dst.id[pos] = B.id[b];
      }
    }
  }
}
__global__ void k_scatter(Inst I, int sp0, int per_step) { k_scatter_body(I, sp0, per_step); }
__global__ void k_scatter_b(const Inst* insts, int sp0, int per_step) {
  __shared__ Inst sI;
  stage_inst(insts + blockIdx.z, &sI);
  k_scatter_body(sI, sp0, per_step);
}

// On a step without the full sort the births go to the end of the current
// arrays (blockIdx.y = species); sort_this_step checked that they fit.
__device__ __forceinline__ void k_append_body(const Inst& I) {
  const Scalars* S = I.S;
  if ((S->status & ST_FATAL) || sort_this_step(I, S)) return;
  const int sp = blockIdx.y;
  const long long n_old = S->n[sp];
  const long long nb = S->nbirth[sp] < I.birth_cap ? S->nbirth[sp] : I.birth_cap;
  const ParticlesDev P = I.buf[sp][S->flip[sp]];
  const BirthsDev B = I.births[sp];
  for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < nb;
       b += (long long)gridDim.x * blockDim.x) {
    const long long j = n_old + b;
    P.r[j] = B.r[b]; P.z[j] = B.z[b];
    P.vr[j] = B.vr[b]; P.vt[j] = B.vt[b]; P.vz[j] = B.vz[b];
    P.id[j] = B.id[b];
  }
}
__global__ void k_append(Inst I) { k_append_body(I); }
__global__ void k_append_b(const Inst* insts) {
  __shared__ Inst sI;
  stage_inst(insts + blockIdx.z, &sI);
  k_append_body(sI);
}

// keys + histogram of particles loaded by pic_set_particles; range check.
// Histogram increments are aggregated over the lanes of a warp that share a
// cell, and the id maximum over the warp, to keep atomics off hot addresses.
__global__ void k_keys(Inst I, int sp) {
  Scalars* S = I.S;
  const long long n = S->n[sp];
  const ParticlesDev P = I.buf[sp][S->flip[sp]];
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarp = ((long long)gridDim.x * blockDim.x) >> 5;
  long long idmax = -1;
  bool bad = false;
  for (long long base = warp * 32; base < n; base += nwarp * 32) {
    const long long i = base + lane;
    int key = -1;
    if (i < n) {
      const double r = P.r[i], z = P.z[i];   // cell units
      if (r >= 0.0 && r < (double)I.nr && z >= 0.0 && z < (double)I.nz && finite64(P.vr[i]) &&
          finite64(P.vt[i]) &&
          finite64(P.vz[i]) && P.id[i] >= 0) {
        int m, nn;
        double f;
        split_cell(r, I.nr, m, f);
        split_cell(z, I.nz, nn, f);
        key = cell_key(I, m, nn);
        idmax = P.id[i] > idmax ? P.id[i] : idmax;
      } else {
        bad = true;
      }
      I.key[sp][i] = key;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    if (key >= 0 && lane == __ffs(peers) - 1) atomicAdd(&I.counts[sp][key], __popc(peers));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long other = __shfl_xor_sync(0xffffffffu, idmax, o);
    idmax = other > idmax ? other : idmax;
  }
  if (lane == 0 && idmax >= 0) atomicMax(&S->next_id, idmax + 1);
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&S->status, ST_NAN);
}

// Re-weighting (Section 6): particle `id` of species sp stays iff word 0 of
// its stream-5 draw at the current step is divisible by `factor`; kept
// particles get their cell key and are counted, the others key -1 (the
// scatter drops them).
__device__ __forceinline__ bool thin_keep(const Inst& I, int sp, long long id, long long s,
                                          int factor) {
  unsigned long long w[4];
  philox4x64((unsigned long long)id, (unsigned long long)s, 5ULL, 0ULL, I.seed,
             (unsigned long long)sp, w);
  return w[0] % (unsigned long long)factor == 0ULL;
}

__global__ void k_thin(Inst I, int sp, int factor) {
  Scalars* S = I.S;
  if (S->status & ST_FATAL) return;
  const long long n = S->n[sp], s = S->step;
  const ParticlesDev P = I.buf[sp][S->flip[sp]];
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarp = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long base = warp * 32; base < n; base += nwarp * 32) {
    const long long i = base + lane;
    int key = -1;
    if (i < n) {
      // dead slots (r = -1) go; factor 1 keeps every live particle (compaction)
      const bool dead = (long long)bits_of(P.r[i]) < 0;
      if (!dead && (factor == 1 || thin_keep(I, sp, P.id[i], s, factor))) {
        int m, nn;
        double f;
        split_cell(P.r[i], I.nr, m, f);
        split_cell(P.z[i], I.nz, nn, f);
        key = cell_key(I, m, nn);
      }
      I.key[sp][i] = key;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    if (key >= 0 && lane == __ffs(peers) - 1) atomicAdd(&I.counts[sp][key], __popc(peers));
  }
}

// ---------------------------------------------------------------------------
// Region diagnostics (Sections 4, 5): one sample of the state is added to the
// per-cell sums (particle counts of both species, electron velocity moments)
// and phi to the node sums.  The particle arrays are sorted by cell: after the
// scatter, cursor[k] is the end of cell bin k (its start the end of bin k - 1),
// so one warp sums one cell's particles (strided per-lane sums, one warp
// reduction per cell) and is the only writer of that cell's accumulators.
// ---------------------------------------------------------------------------
template <bool F32>
__global__ void k_region_sample(Inst I, int sp) {
  const Scalars* S = I.S;
  if (S->status & ST_FATAL) return;
  const long long n = S->n[sp];
  const int* ends = I.cursor[sp];
  const int lane = threadIdx.x & 31;
  const int warp = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nwarp = (int)(((long long)gridDim.x * blockDim.x) >> 5);
  const unsigned full = 0xffffffffu;
  for (int k = warp; k < I.nkey; k += nwarp) {
    long long b0 = k > 0 ? ends[k - 1] : 0, b1 = ends[k];
    if (b1 > n) b1 = n;
    if (b1 <= b0) continue;
    int m, nn;
    key_cell(I, k, m, nn);
    if (m >= I.nr || nn >= I.nz) continue;   // padding keys hold no particles
    const int cell = m * I.nz + nn;
    if (sp == 0) {
      double s[4] = {0.0, 0.0, 0.0, 0.0};
      for (long long i = b0 + lane; i < b1; i += 32) {
        double vr, vt, vz;
        if (F32) {
          const float4 a = I.buf32[0][S->flip[0]].a[i];
          const uint4 b = I.buf32[0][S->flip[0]].b[i];
          vr = (double)a.z;
          vt = (double)a.w;
          vz = (double)__uint_as_float(b.x);
        } else {
          const ParticlesDev P = I.buf[0][S->flip[0]];
          vr = P.vr[i];
          vt = P.vt[i];
          vz = P.vz[i];
        }
        s[0] += vr;
        s[1] += vt;
        s[2] += vz;
        s[3] += vr * vr + vt * vt + vz * vz;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s[q] += __shfl_xor_sync(full, s[q], o);
      if (lane == 0)
        for (int q = 0; q < 4; ++q) I.reg.mom[(size_t)cell * 4 + q] += s[q];
    }
    if (lane == 0) I.reg.n[sp][cell] += (unsigned long long)(b1 - b0);
  }
}

__global__ void k_region_phi(Inst I) {
  if (I.S->status & ST_FATAL) return;
  const long long nn = (long long)(I.nr + 1) * (I.nz + 1);
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < nn;
       k += (long long)gridDim.x * blockDim.x)
    I.reg.phi[k] += I.phi[k];
  if (blockIdx.x == 0 && threadIdx.x == 0) *I.reg.samples += 1ULL;
}

// Evaluation of the accumulated samples (Section 4: the sheath ends where
// n_e >= n_i / 2 -- 2 N_e >= N_i in counts, same volume and weight; the bulk
// starts at the first cell from there on with E_z = -d phi/dz >= 0 from the
// cell's corner potentials; Section 5: a cell's electron temperature is
// m_e (<|v|^2> - |<v>|^2) / (3 e) over its samples (at least two), a
// region's the plain mean over its cells in the radial band).  One warp per
// cell column (ballots find the edges, warp sums per region), then the sums
// over columns in column order (k_region_total).
__global__ void k_region_cols(Inst I) {
  const RegionDev R = I.reg;
  const int nr = I.nr, nz = I.nz, nz1 = nz + 1;
  const int lane = threadIdx.x & 31;
  const unsigned full = 0xffffffffu;
  const int warp = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nwarp = (int)(((long long)gridDim.x * blockDim.x) >> 5);
  for (int m = warp; m < nr; m += nwarp) {
    int ns = nz, nb = nz;
    for (int n0 = 0; n0 < nz; n0 += 32) {
      const int n = n0 + lane;
      const size_t c = (size_t)m * nz + n;
      const unsigned hit = __ballot_sync(full, n < nz && 2ULL * R.n[0][c] >= R.n[1][c]);
      if (hit) {
        ns = n0 + __ffs(hit) - 1;
        break;
      }
    }
    for (int n0 = ns; n0 < nz; n0 += 32) {
      const int n = n0 + lane;
      bool ok = false;
      if (n < nz) {
        const double up = R.phi[m * nz1 + n + 1] + R.phi[(m + 1) * nz1 + n + 1];
        const double lo = R.phi[m * nz1 + n] + R.phi[(m + 1) * nz1 + n];
        ok = up - lo <= 0.0;
      }
      const unsigned hit = __ballot_sync(full, ok);
      if (hit) {
        nb = n0 + __ffs(hit) - 1;
        break;
      }
    }
    double t[3] = {0.0, 0.0, 0.0}, cnt[3] = {0.0, 0.0, 0.0};
    const double rcen = (m + 0.5) * I.dr;
    const bool band = !(rcen < I.band_lo || rcen > I.band_hi);
    if (band) {
      for (int n = lane; n < nz; n += 32) {
        const size_t c = (size_t)m * nz + n;
        const unsigned long long N = R.n[0][c];
        if (N < 2ULL) continue;
        const double Nd = (double)N;
        const double* mo = R.mom + c * 4;
        const double mr = mo[0] / Nd, mt = mo[1] / Nd, mz = mo[2] / Nd;
        const double T = kMe * (mo[3] / Nd - (mr * mr + mt * mt + mz * mz)) / (3.0 * kQe);
        const int reg = n < ns ? 0 : (n < nb ? 1 : 2);
        t[reg] += T;
        cnt[reg] += 1.0;
      }
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          t[k] += __shfl_xor_sync(full, t[k], o);
          cnt[k] += __shfl_xor_sync(full, cnt[k], o);
        }
    }
    if (lane == 0) {
      R.zs[m] = ns * I.dz;
      R.zb[m] = nb * I.dz;
      double* col = R.col + (size_t)m * 8;
      for (int k = 0; k < 3; ++k) {
        col[k] = t[k];
        col[3 + k] = cnt[k];
      }
      col[6] = band ? 1.0 : 0.0;
    }
  }
}

__global__ void k_region_total(Inst I) {
  if (threadIdx.x != 0) return;
  const RegionDev R = I.reg;
  double t[3] = {0.0, 0.0, 0.0}, c[3] = {0.0, 0.0, 0.0}, zs = 0.0, zb = 0.0, ncol = 0.0;
  for (int m = 0; m < I.nr; ++m) {
    const double* col = R.col + (size_t)m * 8;
    if (col[6] == 0.0) continue;
    for (int k = 0; k < 3; ++k) {
      t[k] += col[k];
      c[k] += col[3 + k];
    }
    zs += R.zs[m];
    zb += R.zb[m];
    ncol += 1.0;
  }
  for (int k = 0; k < 3; ++k) {
    R.out[k] = c[k] > 0.0 ? t[k] / c[k] : 0.0;
    R.out[3 + k] = c[k];
  }
  R.out[6] = ncol > 0.0 ? zs / ncol : 0.0;
  R.out[7] = ncol > 0.0 ? zb / ncol : 0.0;
}

// n = n_next after a set-up sort (no births); the arrays are compact
__global__ void k_commit_n(Inst I, int sp) {
  if (threadIdx.x == 0 && !(I.S->status & ST_FATAL)) {
    I.S->n[sp] = I.S->n_next[sp];
    I.S->n_live[sp] = I.S->n_next[sp];
    I.S->flip[sp] ^= 1;
    if (sp == 1) I.S->unsorted = 0;   // sorts of both species run species 0 first
  }
}

__global__ void k_set_n(Inst I, int sp, long long n) {
  if (threadIdx.x == 0) {
    I.S->n[sp] = n;
    I.S->n_live[sp] = n;
    I.S->nbirth[sp] = 0;
  }
}

// deposit every particle of the current arrays (global atomics; set-up only)
__global__ void k_deposit_all(Inst I, int sp) {
  const long long n = I.S->n[sp];
  const ParticlesDev P = I.buf[sp][I.S->flip[sp]];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    int m, nn;
    double fr, fz;
    split_cell(P.r[i], I.nr, m, fr);
    split_cell(P.z[i], I.nz, nn, fz);
    const FixW f = fix_weights(rweight_upper(I, P.r[i], m, fr), fz);
    unsigned long long* q = I.qacc[sp];
    atomicAdd(q + node_index(I, m, nn), f.w00);
    atomicAdd(q + node_index(I, m + 1, nn), f.w10);
    atomicAdd(q + node_index(I, m, nn + 1), f.w01);
    atomicAdd(q + node_index(I, m + 1, nn + 1), f.w11);
  }
}

// ---------------------------------------------------------------------------
// Node charge Q = e w (sum_i - sum_e) 2^-44; peak densities on diagnostic steps
// ---------------------------------------------------------------------------
// Node charges Q from the deposit sums (zeroed for the next step); with `step`
// and phi_extrap the unknown nodes of phi also move to the start of this
// step's solve, 2 phi^{n-1} - phi^{n-2}, and phi_old to phi^{n-1}.
__device__ __forceinline__ void k_charge_body(const Inst& I, bool step) {
  Scalars* S = I.S;
  const int nn = (I.nr + 1) * (I.nz + 1);
  const bool extrap = step && I.phi_extrap;
  const bool diag = S->diag_on != 0;
  const double scale = kQe * I.weight * kFixInv;
  double pe = 0.0, pi = 0.0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nn; k += gridDim.x * blockDim.x) {
    double se, si;   // deposited macroparticles of each species at the node
    if (I.prec32) {
      se = I.qacc64[0][k];
      si = I.qacc64[1][k];
      I.qacc64[0][k] = 0.0;
      I.qacc64[1][k] = 0.0;
      I.Q[k] = (si - se) * (kQe * I.weight);
    } else {
      const unsigned long long ue = I.qacc[0][k], ui = I.qacc[1][k];
      I.qacc[0][k] = 0ULL;
      I.qacc[1][k] = 0ULL;
      I.Q[k] = (double)(long long)(ui - ue) * scale;
      se = (double)ue * kFixInv;
      si = (double)ui * kFixInv;
    }
    I.qs[0][k] = -se * (kQe * I.weight);
    I.qs[1][k] = si * (kQe * I.weight);
    if (extrap) {
      const int m = k / (I.nz + 1), n = k - m * (I.nz + 1);
      const double p1 = I.phi[k];
      if (field_free(m, n, I.nr, I.nz, I.bc_g, I.bc_wall)) I.phi[k] = 2.0 * p1 - I.phi_old[k];
      I.phi_old[k] = p1;
    }
    if (diag) {
      const int m = k / (I.nz + 1), n = k - m * (I.nz + 1);
      const double sv = I.weight / node_volume(I, m, n);
      pe = fmax(pe, se * sv);
      pi = fmax(pi, si * sv);
    }
  }
  if (diag) {
    // block maximum, then one atomic per block (positive doubles order like
    // their bit patterns)
    __shared__ double red[2][32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      pe = fmax(pe, __shfl_xor_sync(0xffffffffu, pe, o));
      pi = fmax(pi, __shfl_xor_sync(0xffffffffu, pi, o));
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
      red[0][w] = pe;
      red[1][w] = pi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0, b = 0.0;
      for (int j = 0; j < (int)(blockDim.x >> 5); ++j) {
        a = fmax(a, red[0][j]);
        b = fmax(b, red[1][j]);
      }
      if (a > 0.0) atomicMax(&S->peak_bits[0], (unsigned long long)__double_as_longlong(a));
      if (b > 0.0) atomicMax(&S->peak_bits[1], (unsigned long long)__double_as_longlong(b));
    }
  }
}
__global__ void k_charge(Inst I, bool step) { k_charge_body(I, step); }
__global__ void k_charge_b(const Inst* insts, bool step) {
  __shared__ Inst sI;
  stage_inst(insts + blockIdx.z, &sI);
  k_charge_body(sI, step);
}

// ---------------------------------------------------------------------------
// External circuit (Sections 3, 4, 6): cathode charge of the step, running
// mean current over n_avg steps, V_c = -V_s + I R_ext clamped to [-V_s, 0];
// writes the cathode nodes' Dirichlet value into phi.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void k_circuit_body(const Inst& I) {
  Scalars* S = I.S;
  if (S->status & ST_FATAL) return;
  if (threadIdx.x == 0) {
    const long long cnt_q = (long long)S->cnt_ion_cath + (long long)S->cnt_sey - (long long)S->cnt_e_cath;
    const double qc = kQe * I.weight * (double)cnt_q;
    const int na = I.n_avg > 0 ? I.n_avg : 1;
    const long long st = S->step;
    I.qhist[st % na] = qc;
    const long long cnt = st + 1 < na ? st + 1 : na;
    double qs = 0.0;
    for (long long k = 0; k < cnt; ++k) qs += I.qhist[k];
    const double cur = qs / ((double)cnt * I.dt);
    double V = I.Vc_fixed;
    if (I.circuit_mode == 1) {
      V = -I.Vs + cur * I.Rext;
      if (V < -I.Vs) V = -I.Vs;
      if (V > 0.0) V = 0.0;
    }
    S->I = cur;
    S->Vc = V;
  }
  __syncthreads();
  const double V = S->Vc;
  for (int m = threadIdx.x; m <= I.m_cath; m += blockDim.x) I.phi[m * (I.nz + 1)] = V;
}
__global__ void k_circuit(Inst I) { k_circuit_body(I); }
__global__ void k_circuit_b(const Inst* insts) {
  __shared__ Inst sI;
  stage_inst(insts + blockIdx.z, &sI);
  k_circuit_body(sI);
}

__global__ void k_set_cathode(Inst I) {
  const double V = I.S->Vc;
  for (int m = threadIdx.x; m <= I.m_cath; m += blockDim.x) I.phi[m * (I.nz + 1)] = V;
}

// diagnostics record, counters for the next step, step index
__device__ __forceinline__ void k_step_end_body(const Inst& I) {
  Scalars* S = I.S;
  if (threadIdx.x != 0) return;
  const long long nb0 = S->nbirth[0] < I.birth_cap ? S->nbirth[0] : I.birth_cap;
  const long long nb1 = S->nbirth[1] < I.birth_cap ? S->nbirth[1] : I.birth_cap;
  const bool ok = !(S->status & ST_FATAL);
  if (S->diag_on) {
    DiagDev* d = I.diag;
    d->t = S->step * I.dt;
    d->I_cath = S->I;
    d->V_cath = S->Vc;
    d->n_e_peak = __longlong_as_double((long long)S->peak_bits[0]);
    d->n_i_peak = __longlong_as_double((long long)S->peak_bits[1]);
    d->W_field = S->W;
    d->K_e = S->K[0];
    d->K_i = S->K[1];
    d->N_e = ok ? S->n_next[0] : S->n[0];
    d->N_i = ok ? S->n_next[1] : S->n[1];
    d->n_ion_cath = (long long)S->cnt_ion_cath;
    d->n_e_cath = (long long)S->cnt_e_cath;
    d->n_sey = (long long)S->cnt_sey;
    d->n_ionize = (long long)S->cnt_ionize;
    d->n_excite = (long long)S->cnt_excite;
    d->n_elastic = (long long)S->cnt_elastic;
    d->n_ionize_meta = (long long)S->cnt_ionize_meta;
    d->ppc_max[0] = S->ppc_max[0];
    d->ppc_max[1] = S->ppc_max[1];
    d->step = S->step;
    d->poisson_iters = S->poisson_iters;
    d->poisson_resid = S->poisson_resid;
    d->status = S->status;
  }
  I.diag->particle_steps = S->pushed + (ok ? S->n_live[0] + S->n_live[1] : 0);  // every step
  if (ok) {
    S->pushed += S->n_live[0] + S->n_live[1];   // the live particles this step pushed
    if (sort_this_step(I, S)) {
      S->flip[0] ^= 1;   // the scatter wrote the other buffer
      S->flip[1] ^= 1;
      S->n[0] = S->n_next[0];
      S->n[1] = S->n_next[1];
      S->unsorted = 0;
    } else {             // births appended in place, dead slots kept
      S->n[0] += nb0;
      S->n[1] += nb1;
      S->unsorted = 1;
    }
    S->n_live[0] = S->n_next[0];
    S->n_live[1] = S->n_next[1];
    S->step = S->step + 1;
  }
  S->nbirth[0] = S->nbirth[1] = 0;
  S->cnt_ion_cath = S->cnt_e_cath = S->cnt_sey = 0ULL;
  S->cnt_ionize = S->cnt_excite = S->cnt_elastic = 0ULL;
  S->cnt_ionize_meta = 0ULL;
  S->K[0] = S->K[1] = 0.0;
  S->W = 0.0;
  S->peak_bits[0] = S->peak_bits[1] = 0ULL;
  S->diag_on = (S->step % (I.diag_every > 0 ? I.diag_every : 1)) == 0;
}
__global__ void k_step_end(Inst I) { k_step_end_body(I); }
__global__ void k_step_end_b(const Inst* insts) {
  __shared__ Inst sI;
  stage_inst(insts + blockIdx.z, &sI);
  k_step_end_body(sI);
}

// live particles of all instances (the autotuner's view of the work)
__global__ void k_live_total(const Inst* insts, int n_inst, long long* out) {
  if (threadIdx.x != 0) return;
  long long t = 0;
  for (int k = 0; k < n_inst; ++k) t += insts[k].S->n_live[0] + insts[k].S->n_live[1];
  *out = t;
}

cudaError_t launch_live_total(const Inst* d_insts, int n_inst, long long* out, cudaStream_t st) {
  k_live_total<<<1, 32, 0, st>>>(d_insts, n_inst, out);
  return cudaGetLastError();
}

// Fill the push queue: chunks of `chunk` particles per instance and species
// (none for an instance whose status is latched).
__global__ void k_queue_setup(const Inst* insts, WorkQueue* q, int n_inst, long long chunk) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  q->n_inst = n_inst;
  int acc = 0;
  q->prefix[0] = 0;
  for (int k = 0; k < n_inst; ++k) {
    const Scalars* S = insts[k].S;
    const bool dead = (S->status & ST_FATAL) != 0;
    for (int sp = 0; sp < 2; ++sp) {
      const long long n = dead ? 0 : S->n[sp];
      q->nch[k][sp] = (int)((n + chunk - 1) / chunk);
      acc += q->nch[k][sp];
    }
    q->prefix[k + 1] = acc;
  }
  q->next = 0u;
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
// one wave of a persistent kernel: resident blocks per SM x SMs (cached per
// kernel function)
int resident_blocks(const void* fn, int threads, int num_sms) {
  static const void* keys[16];
  static int vals[16];
  static int used = 0;
  for (int k = 0; k < used; ++k)
    if (keys[k] == fn) return vals[k] * num_sms;
  int p = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p, fn, threads, 0) != cudaSuccess || p < 1) p = 1;
  if (used < 16) {
    keys[used] = fn;
    vals[used] = p;
    ++used;
  }
  return p * num_sms;
}

static int grid_for(long long work, int threads, int num_sms, int per_sm) {
  long long g = (work + threads - 1) / threads;
  long long cap = (long long)num_sms * per_sm;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

cudaError_t launch_queue_setup(const Inst* d_insts, WorkQueue* q, int n_inst, long long chunk,
                               cudaStream_t st) {
  k_queue_setup<<<1, 32, 0, st>>>(d_insts, q, n_inst, chunk);
  return cudaGetLastError();
}

template <int GATHER, bool PLAIN>
static void push_one(const Inst& I, WorkQueue* q, int ppt, int num_sms, cudaStream_t st) {
  k_push_one<GATHER, PLAIN><<<resident_blocks((const void*)k_push_one<GATHER, PLAIN>,
                                              kPushThreads, num_sms),
                              kPushThreads, 0, st>>>(I, q, ppt);
}

template <int GATHER, bool PLAIN>
static void push_all(const Inst* d_insts, WorkQueue* q, int ppt, int num_sms, cudaStream_t st) {
  k_push_all<GATHER, PLAIN><<<resident_blocks((const void*)k_push_all<GATHER, PLAIN>,
                                              kPushThreads, num_sms),
                              kPushThreads, 0, st>>>(d_insts, q, ppt);
}

cudaError_t launch_push_one(const Inst& I, WorkQueue* q, int ppt, int num_sms, cudaStream_t st) {
  if (I.prec32) return launch_push32_one(I, q, ppt, num_sms, st);
  // plain: the model's own switches (push on, tent weights in r, absorbing walls)
  const bool plain = I.push_on && I.rweight == 0 && !I.walls_reflect;
  if (I.gather == 0) {
    if (plain) push_one<0, true>(I, q, ppt, num_sms, st);
    else push_one<0, false>(I, q, ppt, num_sms, st);
  } else {
    if (plain) push_one<1, true>(I, q, ppt, num_sms, st);
    else push_one<1, false>(I, q, ppt, num_sms, st);
  }
  return cudaGetLastError();
}

cudaError_t launch_push_all(const Inst* d_insts, WorkQueue* q, int prec32, int gather, bool plain,
                            int ppt, int num_sms, cudaStream_t st) {
  // a thread's queue-overflow candidates are a 32-bit mask over its chunk slots
  if (ppt < 1 || ppt > 32) return cudaErrorInvalidValue;
  if (prec32) return launch_push32_all(d_insts, q, gather, plain, ppt, num_sms, st);
  if (gather == 0) {
    if (plain) push_all<0, true>(d_insts, q, ppt, num_sms, st);
    else push_all<0, false>(d_insts, q, ppt, num_sms, st);
  } else {
    if (plain) push_all<1, true>(d_insts, q, ppt, num_sms, st);
    else push_all<1, false>(d_insts, q, ppt, num_sms, st);
  }
  return cudaGetLastError();
}

cudaError_t launch_charge(const Inst& I, bool step, cudaStream_t st) {
  const int nn = (I.nr + 1) * (I.nz + 1);
  k_charge<<<grid_for(nn, 256, 1024, 1), 256, 0, st>>>(I, step);
  return cudaGetLastError();
}

cudaError_t launch_set_n(const Inst& I, int sp, long long n, cudaStream_t st) {
  k_set_n<<<1, 32, 0, st>>>(I, sp, n);
  return cudaGetLastError();
}

cudaError_t launch_sort_species(const Inst& I, int sp, int num_sms, cudaStream_t st) {
  // n is already in S->n[sp]; births are none
  long long cap = I.cap[sp];
  k_keys<<<grid_for(cap, 256, num_sms, 8), 256, 0, st>>>(I, sp);
  k_scan<<<kScanCta, 1024, 0, st>>>(I, sp);
  k_scatter<<<dim3(grid_for(cap, 256, num_sms, 8), 1), 256, 0, st>>>(I, sp, 0);
  k_commit_n<<<1, 32, 0, st>>>(I, sp);
  return cudaGetLastError();
}

cudaError_t launch_thin(const Inst& I, int factor, int num_sms, cudaStream_t st) {
  for (int sp = 0; sp < 2; ++sp) {
    if (I.prec32) {
      launch_thin32(I, sp, factor, num_sms, st);
      launch_sort_species32(I, sp, num_sms, st);
    } else {
      const long long cap = I.cap[sp];
      k_thin<<<grid_for(cap, 256, num_sms, 8), 256, 0, st>>>(I, sp, factor);
      k_scan<<<kScanCta, 1024, 0, st>>>(I, sp);
      k_scatter<<<dim3(grid_for(cap, 256, num_sms, 8), 1), 256, 0, st>>>(I, sp, 0);
      k_commit_n<<<1, 32, 0, st>>>(I, sp);
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_region_sample(const Inst& I, int num_sms, cudaStream_t st) {
  // one warp per cell bin, eight warps per block
  const int blocks = grid_for((long long)I.nkey * 32, 256, num_sms, 8);
  for (int sp = 0; sp < 2; ++sp) {
    if (I.prec32) k_region_sample<true><<<blocks, 256, 0, st>>>(I, sp);
    else k_region_sample<false><<<blocks, 256, 0, st>>>(I, sp);
  }
  const long long nn = (long long)(I.nr + 1) * (I.nz + 1);
  k_region_phi<<<grid_for(nn, 256, num_sms, 2), 256, 0, st>>>(I);
  return cudaGetLastError();
}

cudaError_t launch_region_eval(const Inst& I, cudaStream_t st) {
  k_region_cols<<<(I.nr + 7) / 8, 256, 0, st>>>(I);   // one warp per cell column
  k_region_total<<<1, 32, 0, st>>>(I);
  return cudaGetLastError();
}

// Particle arrays read in place from host memory that the device addresses
// directly (pinned memory under unified addressing, over the CPU-GPU link):
// six arrays of n 8-byte words, one pass by the SMs.
struct Copy6 {
  const unsigned long long* src[6];
  unsigned long long* dst[6];
};

// r, z, v_r, v_theta, v_z, id in, positions converted from SI to cell units;
// with src == dst for the velocities and ids (already in place) only the
// positions are rewritten
__global__ void k_copy_in(Copy6 c, long long n, Inst I) {
  const bool all = c.src[2] != c.dst[2];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double r = double_of(c.src[0][i]), z = double_of(c.src[1][i]);
    if (all) {
      unsigned long long v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = c.src[k + 2][i];
#pragma unroll
      for (int k = 0; k < 4; ++k) c.dst[k + 2][i] = v[k];
    }
    c.dst[0][i] = bits_of(to_cells(r, I.inv_dr, I.nr, I.R));
    c.dst[1][i] = bits_of(to_cells(z, I.inv_dz, I.nz, I.L));
  }
}

cudaError_t launch_copy_in(const void* const src[6], void* const dst[6], long long n,
                           const Inst& I, int num_sms, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  Copy6 c;
  for (int k = 0; k < 6; ++k) {
    c.src[k] = (const unsigned long long*)src[k];
    c.dst[k] = (unsigned long long*)dst[k];
  }
  k_copy_in<<<grid_for(n, 256, num_sms, 8), 256, 0, st>>>(c, n, I);
  return cudaGetLastError();
}

// positions out in SI (either output may be null)
__global__ void k_positions_out(const double* rc, const double* zc, double* r, double* z,
                                long long n, Inst I) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    if (r) r[i] = from_cells(rc[i], I.dr, I.R);
    if (z) z[i] = from_cells(zc[i], I.dz, I.L);
  }
}

cudaError_t launch_positions_out(const Inst& I, const double* rc, const double* zc, double* r,
                                 double* z, long long n, int num_sms, cudaStream_t st) {
  if (n <= 0 || (!r && !z)) return cudaSuccess;
  k_positions_out<<<grid_for(n, 256, num_sms, 8), 256, 0, st>>>(rc, zc, r, z, n, I);
  return cudaGetLastError();
}

cudaError_t launch_scan(const Inst& I, int sp0, int nsp, cudaStream_t st) {
  k_scan<<<nsp * kScanCta, 1024, 0, st>>>(I, sp0);
  return cudaGetLastError();
}

cudaError_t launch_commit_n(const Inst& I, int sp, cudaStream_t st) {
  k_commit_n<<<1, 32, 0, st>>>(I, sp);
  return cudaGetLastError();
}

cudaError_t launch_solve_fields(const Inst& I, PoissonWork* pw, int num_sms, cudaStream_t st) {
  if (I.prec32) {
    cudaError_t e0 = launch_deposit_all32(I, num_sms, st);
    if (e0 != cudaSuccess) return e0;
  } else {
    for (int sp = 0; sp < 2; ++sp)
      k_deposit_all<<<grid_for(I.cap[sp], 256, num_sms, 8), 256, 0, st>>>(I, sp);
  }
  cudaError_t e = launch_charge(I, false, st);
  if (e != cudaSuccess) return e;
  k_set_cathode<<<1, 256, 0, st>>>(I);
  e = launch_poisson(pw, I.Q, I.phi, I.poisson_tol, I.poisson_max_iter, &I.S->status,
                     &I.S->poisson_iters, &I.S->poisson_resid, st);
  if (e != cudaSuccess) return e;
  // no earlier solution: the next step's extrapolation starts from this one
  return cudaMemcpyAsync(I.phi_old, I.phi, (size_t)(I.nr + 1) * (I.nz + 1) * 8,
                         cudaMemcpyDeviceToDevice, st);
}

cudaError_t launch_field_tables(const Inst& I, int num_sms, cudaStream_t st) {
  k_field_tables<<<grid_for(I.nr * I.nz, 256, num_sms, 8), 256, 0, st>>>(I);
  return cudaGetLastError();
}

// births, scan, scatter, charge and circuit of one instance (after its push)
cudaError_t launch_post_push(const Inst& I, int num_sms, cudaStream_t st) {
  launch_births(I, num_sms, st);
  k_scan<<<2 * kScanCta, 1024, 0, st>>>(I, 0);
  if (I.prec32) launch_scatter32(I, num_sms, st);
  else k_scatter<<<dim3(num_sms * 8, 2), 256, 0, st>>>(I, 0, 1);
  if (I.sort_every > 1) {
    if (I.prec32) launch_append32(I, num_sms, st);
    else k_append<<<dim3(num_sms, 2), 256, 0, st>>>(I);
  }
  cudaError_t e = launch_charge(I, true, st);
  if (e != cudaSuccess) return e;
  k_circuit<<<1, 256, 0, st>>>(I);
  return cudaGetLastError();
}

// ---- batched launches of the per-instance kernels of an ensemble ----------
// gridDim.z = instances (the kernels take the instance from blockIdx.z); the
// x extent covers the largest instance, and the grid-stride loops of the
// per-instance kernels make any extent correct.
cudaError_t launch_field_tables_batch(const Inst* d_insts, int n_inst, const BatchDims& bd,
                                      int num_sms, cudaStream_t st) {
  const int g = grid_for(bd.cells_max, 256, num_sms, 8 / n_inst > 0 ? 8 / n_inst : 1);
  k_field_tables_b<<<dim3(g, 1, n_inst), 256, 0, st>>>(d_insts);
  return cudaGetLastError();
}

cudaError_t launch_post_push_batch(const Inst* d_insts, int n_inst, const BatchDims& bd,
                                   int num_sms, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_births_sort_b, cudaFuncAttributeMaxDynamicSharedMemorySize, kBirthSmem);
    attr = true;
  }
  const int per = num_sms / n_inst > 0 ? num_sms / n_inst : 1;   // blocks of one instance per SM-share
  const int chunks = (int)((bd.birth_cap_max + kBirthChunk - 1) / kBirthChunk);
  k_births_sort_b<<<dim3(chunks > 0 ? chunks : 1, 2, n_inst), 1024, kBirthSmem, st>>>(d_insts);
  const int rank_blocks = grid_for(2 * bd.birth_cap_max, 256, per, 4);
  if (bd.prec32) k_births_rank_b<true><<<dim3(rank_blocks, 1, n_inst), 256, 0, st>>>(d_insts);
  else k_births_rank_b<false><<<dim3(rank_blocks, 1, n_inst), 256, 0, st>>>(d_insts);
  k_births_commit_b<<<dim3(1, 1, n_inst), 32, 0, st>>>(d_insts);
  k_scan_b<<<dim3(2 * kScanCta, 1, n_inst), 1024, 0, st>>>(d_insts, 0);
  if (bd.prec32) launch_scatter32_batch(d_insts, n_inst, per * 8, st);
  else k_scatter_b<<<dim3(per * 8, 2, n_inst), 256, 0, st>>>(d_insts, 0, 1);
  if (bd.any_append) {
    if (bd.prec32) launch_append32_batch(d_insts, n_inst, per, st);
    else k_append_b<<<dim3(per, 2, n_inst), 256, 0, st>>>(d_insts);
  }
  k_charge_b<<<dim3(grid_for(bd.nodes_max, 256, 1024, 1), 1, n_inst), 256, 0, st>>>(d_insts, true);
  k_circuit_b<<<dim3(1, 1, n_inst), 256, 0, st>>>(d_insts);
  return cudaGetLastError();
}

cudaError_t launch_step_end_batch(const Inst* d_insts, int n_inst, cudaStream_t st) {
  k_step_end_b<<<dim3(1, 1, n_inst), 32, 0, st>>>(d_insts);
  return cudaGetLastError();
}

cudaError_t launch_step_end(const Inst& I, cudaStream_t st) {
  k_step_end<<<1, 32, 0, st>>>(I);
  return cudaGetLastError();
}

cudaError_t launch_step(const Inst& I, PoissonWork* pw, int num_sms, cudaStream_t st,
                        const StepMarks* marks, const StepHooks* hooks, const Inst* d_inst,
                        WorkQueue* q, int ppt) {
  auto mk = [&](int g, bool b) {
    if (marks) marks->mark(marks->ctx, g, b, st);
  };
  const int ncell = I.nr * I.nz;
  mk(G_FIELD, true);
  k_field_tables<<<grid_for(ncell, 256, num_sms, 8), 256, 0, st>>>(I);
  mk(G_FIELD, false);
  mk(G_PUSH, true);
  cudaError_t e0 = launch_queue_setup(d_inst, q, 1, (long long)ppt * kPushThreads, st);
  if (e0 == cudaSuccess) e0 = launch_push_one(I, q, ppt, num_sms, st);
  mk(G_PUSH, false);
  if (e0 != cudaSuccess) return e0;
  mk(G_BIRTHS, true);
  launch_births(I, num_sms, st);
  mk(G_BIRTHS, false);
  mk(G_SCAN, true);
  k_scan<<<2 * kScanCta, 1024, 0, st>>>(I, 0);
  mk(G_SCAN, false);
  mk(G_SCATTER, true);
  if (I.prec32) launch_scatter32(I, num_sms, st);
  else k_scatter<<<dim3(num_sms * 8, 2), 256, 0, st>>>(I, 0, 1);
  if (I.sort_every > 1) {
    if (I.prec32) launch_append32(I, num_sms, st);
    else k_append<<<dim3(num_sms, 2), 256, 0, st>>>(I);
  }
  mk(G_SCATTER, false);
  mk(G_CHARGE, true);
  cudaError_t e = launch_charge(I, true, st);
  mk(G_CHARGE, false);
  if (e != cudaSuccess) return e;
  mk(G_CIRCUIT, true);
  k_circuit<<<1, 256, 0, st>>>(I);
  mk(G_CIRCUIT, false);
  if (hooks && hooks->pre_poisson) {
    mk(G_WARM, true);
    e = hooks->pre_poisson(hooks->ctx, I, pw, st);
    mk(G_WARM, false);
    if (e != cudaSuccess) return e;
  }
  mk(G_POISSON, true);
  e = launch_poisson(pw, I.Q, I.phi, I.poisson_tol, I.poisson_max_iter, &I.S->status,
                     &I.S->poisson_iters, &I.S->poisson_resid, st);
  mk(G_POISSON, false);
  if (e != cudaSuccess) return e;
  if (hooks && hooks->post_poisson) {
    e = hooks->post_poisson(hooks->ctx, I, st);
    if (e != cudaSuccess) return e;
  }
  mk(G_STEP_END, true);
  k_step_end<<<1, 32, 0, st>>>(I);
  mk(G_STEP_END, false);
  return cudaGetLastError();
}

}  // namespace pic
