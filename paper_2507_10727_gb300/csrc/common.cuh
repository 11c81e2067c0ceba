// common.cuh -- device-side types and helpers of the GB300 PIC-MCC library.
//
// Layout decisions (all memory is HBM-resident for the whole run):
//  * particles: structure of arrays per species, double buffered, sorted by a
//    tile-major cell key (tiles of 8 x 8, 16 x 8 or 8 x 16 cells in r x z, the
//    shape chosen by the autotuner) so that a CTA's chunk of consecutive
//    particles covers a compact patch of the grid;
//  * node arrays (phi, Q): (nr+1) x (nz+1), z fastest;
//  * per-cell gather tables: the field and the magnetic field around a cell
//    folded into polynomial coefficients in the in-cell offsets, so one cell
//    lookup (contiguous 16-byte loads through L1) feeds the push;
//  * charge: per-species node sums in 44-bit fixed point (u64), so that the
//    deposit is exact, order independent and deterministic; weights are
//    rounded to 2^-44 of a macroparticle and sum to exactly one.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "bits.cuh"

namespace pic {

// CODATA 2018
constexpr double kQe = 1.602176634e-19;
constexpr double kMe = 9.1093837015e-31;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kBoltz = 1.380649e-23;
constexpr double kPi = 3.14159265358979323846;

// cell tiles: 2^tsr x 2^tsz cells (r x z); the shapes 8 x 8, 16 x 8, 8 x 16
constexpr int kTileShapes = 3;
constexpr int kTileLog[kTileShapes][2] = {{3, 3}, {4, 3}, {3, 4}};
constexpr int kFixBits = 44;             // fixed-point fraction bits of the deposit
constexpr double kFixOne = 17592186044416.0;          // 2^44
constexpr double kFixInv = 1.0 / 17592186044416.0;    // 2^-44

// latched status bits (device side); translated to pic_status by the host
enum : int {
  ST_CAPACITY = 1,
  ST_NONCONV = 2,
  ST_NAN = 4,
  ST_TIMEOUT = 8,
};
constexpr int ST_FATAL = ST_CAPACITY | ST_NONCONV | ST_NAN | ST_TIMEOUT;

// FP64 particle arrays.  Positions are stored in cell units, r / dr in
// [0, nr) and z / dz in [0, nz) (r = -1 marks a removed particle), so that a
// cell split needs no scaling; velocities are in m/s.
struct ParticlesDev {
  double *r, *z, *vr, *vt, *vz;
  long long* id;
};

// FP32 particle mode: 32 bytes per particle in two 16-byte records,
// a = {dr, dz, v_r, v_theta} (dr, dz: FP32 offsets in [0,1) inside the cell),
// b = {v_z (bits), cell (m << 16 | n), id low word, id high word}; a cell
// word of all ones marks a removed particle.
struct Particles32 {
  float4* a;
  uint4* b;
};

struct BirthsDev {
  float4* a32;                // FP32 mode records (cell key in b32.y, id in b32.z/w)
  uint4* b32;
  double *r, *z, *vr, *vt, *vz;   // FP64 mode: positions in cell units, as ParticlesDev
  unsigned long long* pkey;   // (parent id << 2) | kind
  int* cell;                  // cell key of the birth position
  long long* id;              // id assigned by the births kernel
  unsigned long long* skey;   // sort scratch: keys (power-of-two length)
  unsigned int* sidx;         // sort scratch: indices
  long long sort_len;         // length of the scratch arrays
};

// Device-resident scalars of one instance.
struct Scalars {
  long long n[2];          // particles in the sorted arrays
  long long n_next[2];     // after the current step's scatter
  long long nbirth[2];     // births of the current step
  long long step;          // index of the step being taken
  long long next_id;
  unsigned long long cnt_ion_cath, cnt_e_cath, cnt_sey;
  unsigned long long cnt_ionize, cnt_excite, cnt_elastic;
  double Vc;               // cathode potential used by the current field
  double I;                // cathode current (running mean)
  double K[2];             // kinetic energy accumulators of the step
  double W;                // field energy of the step's phi
  unsigned long long peak_bits[2];  // max density (bits of a positive double)
  int status;
  int diag_on;
  int poisson_iters;
  int pad0;
  double poisson_resid;
  long long pushed;        // cumulative particle-steps
  int flip[2];             // which of the two particle buffers of a species is current
  int pad1[2];
  unsigned long long cnt_ionize_meta;   // stepwise ionizations from Ar* (1d) this step
  long long ppc_max[2];    // most particles in one cell, from the last sort's histogram
  long long n_live[2];     // live particles (n also counts the dead slots between sorts)
  int unsorted;            // 1: the arrays hold dead slots and appended births (no sort yet)
  int sort_force;          // 1: every step ends with a full sort (while the push is tuned)
};

struct DiagDev {           // mirrors pic_diag
  double t, I_cath, V_cath, n_e_peak, n_i_peak, W_field, K_e, K_i;
  long long N_e, N_i;
  long long n_ion_cath, n_e_cath, n_sey, n_ionize, n_excite, n_elastic;
  long long step;
  long long particle_steps;
  int poisson_iters;
  int status;
  double poisson_resid;
  long long n_ionize_meta;
  long long ppc_max[2];
};

// Work queue of the push: items are (instance, species, chunk) triples.  Per
// instance the electron and ion chunks alternate while both species have
// some left (the electron push is bound by its random-number arithmetic, the
// ion push by memory traffic; interleaving runs both at once on every SM),
// then the rest of the larger species follows.
constexpr int kMaxInstances = 64;
struct WorkQueue {
  unsigned int next;                 // next item to hand out
  int n_inst;
  int prefix[kMaxInstances + 1];     // first item of instance k
  int nch[kMaxInstances][2];         // chunks per species of instance k
};

// item -> (instance, species, chunk index); false past the last item
__device__ __forceinline__ bool queue_item(const WorkQueue* q, int item, int& inst, int& sp,
                                           int& chunk) {
  int k = -1;
  for (int j = 0; j < q->n_inst; ++j)
    if (item >= q->prefix[j] && item < q->prefix[j + 1]) k = j;
  if (k < 0) return false;
  const int local = item - q->prefix[k];
  const int ce = q->nch[k][0], ci = q->nch[k][1];
  const int m = ce < ci ? ce : ci;
  if (local < 2 * m) {
    sp = local & 1;
    chunk = local >> 1;
  } else {
    sp = ce > ci ? 0 : 1;
    chunk = m + (local - 2 * m);
  }
  inst = k;
  return true;
}

// Everything a kernel needs about one instance; passed by value.
// Region diagnostics (Sections 4, 5, 7): accumulated state and the cathode
// ion energy histogram of one instance.
struct RegionDev {
  unsigned long long* ied;      // ied_bins + 1 counts; the last: above the top edge
  unsigned long long* n[2];     // per cell particle counts, summed over samples
  double* mom;                  // per cell electron sums: v_r, v_theta, v_z, |v|^2
  double* phi;                  // per node potential, summed over samples
  unsigned long long* samples;  // states accumulated
  double* col;                  // evaluation: per cell column 8 values
  double* zs;                   // evaluation: per column sheath and bulk edges (m)
  double* zb;
  double* out;                  // evaluation: Te[3], ncell[3], z_sheath, z_bulk
};

struct Inst {
  // geometry
  int nr, nz, ntz, nkey;   // ntz: tiles along z; nkey: number of cell keys (this shape)
  int tsr, tsz;            // log2 of the tile's extent in r and in z (cells)
  int m_cath;              // last radial node index of the cathode (r_m <= Rc)
  double R, L, Rc, dr, dz, inv_dr, inv_dz;
  double dt;
  double kr64, kz64;       // dt / dr, dt / dz: FP64 moves in cell units
  // species
  double weight;
  double qm[2], mass[2], gamma[2];
  // collisions
  double n_gas, T_gas, m_ion, sigma_el, ion_a, ion_I, exc_C, exc_E, nu_max, p_null;
  double n_meta, meta_a, meta_I;   // reaction (1d) off a constant Ar* background
  unsigned long long pnull32;   // ceil(p_null 2^32): word 2^-32 < p_null  <=>  word < pnull32
  unsigned long long seed;
  // switches
  int gather, rweight, mcc_on, push_on, field_on, walls_reflect, circuit_mode, n_avg;
  int sort_every;          // full cell sort every this many steps (others append in place)
  int bc_g;                // first insulating node of row z = 0 (nr + 1: none)
  int bc_wall;             // 1: the wall r = R is insulating
  // region diagnostics: radial band (m), ion energy histogram bins of width ied_de (eV)
  double band_lo, band_hi, ied_de;
  int ied_bins;
  RegionDev reg;
  int diag_every;
  double Vc_fixed, Vs, Rext;
  int phi_extrap;          // per-step solves start from 2 phi - phi_old on the unknown nodes
  double* phi_old;         // the solution before phi (the previous step's)
  double poisson_tol;
  int poisson_max_iter;
  long long cap[2], birth_cap;
  // FP32 particle mode
  int prec32;
  float hq32[2];           // q dt / 2m per species
  float kr32, kz32;        // dt / dr, dt / dz
  Particles32 buf32[2][2];  // [species][buffer]; current = buf32[sp][S->flip[sp]]
  double* qacc64[2];       // FP32 mode: FP64 node sums of deposited macro-charges
  float4* etab32;          // FP32 gather tables (layout as etab / btab)
  float4* btab32;
  double* stage;           // FP64 staging of pic_set/get_particles in FP32 mode
  long long stage_len;     // particles per staging chunk
  // device arrays
  ParticlesDev buf[2][2];   // [species][buffer]; current = buf[sp][S->flip[sp]]
  int* key[2];
  int* counts[2];
  int* cursor[2];
  BirthsDev births[2];
  double* phi;
  double* Q;
  double* qs[2];           // node charge (C) of each species from the last deposit
  unsigned long long* qacc[2];
  // FP64 gather tables per species, scaled by that species' h = q dt / (2 m):
  // the push reads h E and h B directly
  double4_32a* etab[2];        // EC: 1 per cell {Er0, dEr/dfz, Ez0, dEz/dwr}; MC: 2 per cell
  double4_32a* btab[2];        // 2 per cell: {Br c0..c3}, {Bz c0..c3}
  double* qhist;
  Scalars* S;
  DiagDev* diag;
};

// Copy an instance's parameters into shared memory (whole block; ends with a
// barrier): the batched launches of an ensemble's per-instance kernels take
// the instance from blockIdx.z and the array of the instances' parameters.
__device__ __forceinline__ void stage_inst(const Inst* src, Inst* dst) {
  const unsigned* s4 = reinterpret_cast<const unsigned*>(src);
  unsigned* d4 = reinterpret_cast<unsigned*>(dst);
  for (int k = threadIdx.x; k < (int)(sizeof(Inst) / 4); k += blockDim.x) d4[k] = s4[k];
  __syncthreads();
}

// Whether this step ends with the full cell sort: every sort_every-th step,
// and whenever appending the births in place would overflow a buffer.  The
// scatter and the step-end kernel take the same decision from the same state.
__device__ __forceinline__ bool sort_this_step(const Inst& I, const Scalars* S) {
  if (I.sort_every <= 1 || S->sort_force || (S->step + 1) % I.sort_every == 0) return true;
  for (int sp = 0; sp < 2; ++sp) {
    const long long nb = S->nbirth[sp] < I.birth_cap ? S->nbirth[sp] : I.birth_cap;
    if (S->n[sp] + nb > I.cap[sp]) return true;
  }
  return false;
}

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox4x64(unsigned long long c0, unsigned long long c1,
                                           unsigned long long c2, unsigned long long c3,
                                           unsigned long long k0, unsigned long long k1,
                                           unsigned long long out[4]) {
  const unsigned long long M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const unsigned long long W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += W0; k1 += W1; }
    unsigned long long hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
    unsigned long long hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
    unsigned long long y0 = hi1 ^ c1 ^ k0, y2 = hi0 ^ c3 ^ k1;
    c0 = y0; c1 = lo1; c2 = y2; c3 = lo0;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

__device__ __forceinline__ double u01(unsigned long long x) {
  return (double)(x >> 11) * (1.0 / 9007199254740992.0);
}

// four uniforms of stream k for particle id at step s of a species
__device__ __forceinline__ void draws(const Inst& I, int sp, long long id, long long s, int k,
                                      double u[4]) {
  unsigned long long w[4];
  philox4x64((unsigned long long)id, (unsigned long long)s, (unsigned long long)k, 0ULL, I.seed,
             (unsigned long long)sp, w);
  u[0] = u01(w[0]); u[1] = u01(w[1]); u[2] = u01(w[2]); u[3] = u01(w[3]);
}

// The first word of Philox4x32-10 (same paper): multipliers 0xD2511F53 and
// 0xCD9E8D57, Weyl key increments 0x9E3779B9 and 0xBB67AE85; the 32 x 32 ->
// 64-bit products are single integer multiply-adds on the GPU, against the
// several a 64 x 64 -> 128-bit product of the 64-bit form takes.
__device__ __forceinline__ unsigned philox4x32_w0(unsigned c0, unsigned c1, unsigned c2,
                                                  unsigned c3, unsigned k0, unsigned k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const unsigned hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const unsigned hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const unsigned y0 = hi1 ^ c1 ^ k0, y2 = hi0 ^ c3 ^ k1;
    c0 = y0; c1 = lo1; c2 = y2; c3 = lo0;
  }
  return c0;
}

// The null-collision candidate test of an electron (Section 3: U < p_null):
// U is the first word of Philox4x32-10 with counter (id, step) as 32-bit
// halves, low half first, and key (seed low, seed high), times 2^-32; the
// test is done exactly on the integer word.  The collision of a candidate
// draws its process and angles from stream 0 of Philox4x64-10.
__device__ __forceinline__ bool mcc_candidate(const Inst& I, long long id, long long step) {
  const unsigned long long uid = (unsigned long long)id, ust = (unsigned long long)step;
  const unsigned w = philox4x32_w0((unsigned)uid, (unsigned)(uid >> 32), (unsigned)ust,
                                   (unsigned)(ust >> 32), (unsigned)I.seed,
                                   (unsigned)(I.seed >> 32));
  return (unsigned long long)w < I.pnull32;
}

// ---------------------------------------------------------------------------
// grid helpers
// ---------------------------------------------------------------------------
// cell k = (int)(x / d) (clamped to ncell - 1) and offset f = x / d - k of an
// SI coordinate, with x / d taken as x * inv_d; the split runs on the integer
// pipes (bits.cuh).  FP64 particle positions are stored in cell units and
// split directly (split_cell).
__device__ __forceinline__ void locate(double x, double inv_d, int ncell, int& k, double& f) {
  split_cell(x * inv_d, ncell, k, f);
}


__host__ __device__ __forceinline__ int cell_key(const Inst& I, int m, int n) {
  const int tile = (m >> I.tsr) * I.ntz + (n >> I.tsz);
  return (tile << (I.tsr + I.tsz)) + ((m & ((1 << I.tsr) - 1)) << I.tsz) + (n & ((1 << I.tsz) - 1));
}

// the cell (m, n) of key k (cells of padding keys lie outside the grid)
__device__ __forceinline__ void key_cell(const Inst& I, int k, int& m, int& n) {
  const int tile = k >> (I.tsr + I.tsz), within = k & ((1 << (I.tsr + I.tsz)) - 1);
  const int tm = tile / I.ntz, tn = tile - tm * I.ntz;
  m = (tm << I.tsr) + (within >> I.tsz);
  n = (tn << I.tsz) + (within & ((1 << I.tsz) - 1));
}

// tile shape `shape` (index into kTileLog) on an nr x nz grid: its extents,
// tiles along z and number of keys (host)
inline void set_tile_shape(Inst& I, int shape) {
  I.tsr = kTileLog[shape][0];
  I.tsz = kTileLog[shape][1];
  const int ntr = (I.nr + (1 << I.tsr) - 1) >> I.tsr;
  I.ntz = (I.nz + (1 << I.tsz) - 1) >> I.tsz;
  I.nkey = (ntr * I.ntz) << (I.tsr + I.tsz);
}

__device__ __forceinline__ int node_index(const Inst& I, int m, int n) { return m * (I.nz + 1) + n; }

// radial weight of node m+1 (tent in r, or in r^2 for volume weighting)
__device__ __forceinline__ double rweight_upper(const Inst& I, double r, int m, double fr) {
  if (I.rweight == 0) return fr;
  // (r^2 - r_m^2) / (r_{m+1}^2 - r_m^2) = fr (2m + fr) / (2m + 1)
  return fr * (2.0 * m + fr) / (2.0 * m + 1.0);
}

// Fixed-point corner weights of a unit charge at in-cell weights (wr, wz):
// exact integers summing to 2^44.  w11 = round(ir iz / 2^44) from the 88-bit
// integer product; ir, iz come from the weights' bit patterns (no FP64 work).
// the three fixed-point quantities of the tent weights: round(wr 2^44),
// round(wz 2^44) and their product rounded to 2^-44 (the weights of the four
// nodes are 2^44 - ir - iz + i11, ir - i11, iz - i11 and i11)
__device__ __forceinline__ void fix_parts(double wr, double wz, unsigned long long& ir,
                                          unsigned long long& iz, unsigned long long& i11) {
  ir = fix44(wr);   // round(wr 2^44), integer pipes
  iz = fix44(wz);
  const unsigned long long lo = ir * iz, hi = __umul64hi(ir, iz);
  i11 = ((hi << (64 - kFixBits)) | (lo >> kFixBits)) + ((lo >> (kFixBits - 1)) & 1ULL);
}

struct FixW { unsigned long long w00, w10, w01, w11; };
__device__ __forceinline__ FixW fix_weights(double wr, double wz) {
  const unsigned long long ir = fix44(wr);   // round(wr 2^44), integer pipes
  const unsigned long long iz = fix44(wz);
  const unsigned long long lo = ir * iz, hi = __umul64hi(ir, iz);
  const unsigned long long i11 = ((hi << (64 - kFixBits)) | (lo >> kFixBits)) + ((lo >> (kFixBits - 1)) & 1ULL);
  FixW f;
  f.w11 = i11;
  f.w10 = ir - i11;
  f.w01 = iz - i11;
  f.w00 = (1ULL << kFixBits) - ir - iz + i11;   // modular arithmetic keeps the sum exact
  return f;
}

// 2 / x for x >= 1 below the FP32 overflow: the FP32 approximate reciprocal
// (PTX rcp.approx.ftz.f32, within one FP32 ulp) refined in FP64, the doubling
// on the exponent bits (bits.cuh)
__device__ __forceinline__ double recip2(double x) {
  float yf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"((float)x));
  return recip2_refine(x, (double)yf);
}

// finite test on the exponent bits (integer pipe)
__device__ __forceinline__ bool finite64(double x) {
  return ((__double_as_longlong(x) >> 52) & 0x7ff) != 0x7ff;
}

// Field boundary (Section 3).  Conductors (Dirichlet nodes): the anode row
// n = nz, the cathode nodes of row 0, and -- unless insulating -- the rest of
// row 0 and the wall m = nr.  Insulating parts (the Neumann block) are
// unknowns: row 0 from node g on (g = nr + 1: none), the wall when `wall`.
__host__ __device__ __forceinline__ bool field_free(int m, int n, int nr, int nz, int g, int wall) {
  if (n < 0 || n >= nz || m < 0 || m > nr) return false;
  if (n == 0) return m >= g && (m < nr || wall != 0);
  return m < nr || wall != 0;
}

__device__ __forceinline__ double node_area(const Inst& I, int m) {
  if (m == 0) return kPi * 0.25 * I.dr * I.dr;
  if (m == I.nr) return kPi * (I.R * I.R - (I.R - 0.5 * I.dr) * (I.R - 0.5 * I.dr));
  return 2.0 * kPi * (m * I.dr) * I.dr;
}

__device__ __forceinline__ double node_volume(const Inst& I, int m, int n) {
  double h = (n == 0 || n == I.nz) ? 0.5 : 1.0;
  return node_area(I, m) * I.dz * h;
}

__host__ __device__ __forceinline__ double4_32a make_d4(double x, double y, double z, double w) {
  double4_32a v;
  v.x = x; v.y = y; v.z = z; v.w = w;
  return v;
}

__device__ __forceinline__ double global_time_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return (double)t;
}

}  // namespace pic
