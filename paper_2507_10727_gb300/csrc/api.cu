// api.cu -- the C ABI (include/pic.h): handle life cycle, host<->device
// transfers, the per-step launch loop, checkpoints and the standalone Poisson
// solve.  No compute happens here beyond set-up tables (the magnetron field
// table, the null-collision frequency) evaluated once on the host in FP64.
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/pic.h"
#include "common.cuh"
#include "launch.h"
#include "unet.h"

using namespace pic;

namespace {

struct InstHost {
  pic_config cfg;
  Inst I;
  PoissonWork* pw = nullptr;
  int swapped = 0;
  int nkey_max = 0;                  // cell keys of the tile shape with the most
  std::vector<double4_32a> bcell;    // B-table entries of cell m nz + n (2 per cell)
};

}  // namespace

struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  struct Rec { int group; cudaEvent_t b, e; };
  std::vector<Rec> recs;
  cudaEvent_t open[G_COUNT] = {};
};

struct pic_handle {
  std::vector<InstHost> inst;
  Profiler prof;
  cudaGraphExec_t graph = nullptr;   // one step of every instance, captured once
  bool graph_failed = false;
  // ensemble (n_instances > 1): batched push over a work queue, grouped Poisson
  Inst* d_insts = nullptr;
  WorkQueue* d_queue = nullptr;
  void* d_pargs = nullptr;
  std::vector<PoissonWork*> pws;
  int ppt = 8;                       // particles per thread per work item (autotuned)
  int tune_next = 0;                 // next autotuner candidate; -1 = done
  float tune_ms[4] = {0, 0, 0, 0};
  int tile = 0;                      // cell tile shape of every instance (index of kTileLog)
  int tile0 = 0;                     // shape during the chunk-size candidates of a tuning
  bool tile_tune = true;             // off after pic_set_tile with a fixed shape
  float tile_ms[kTileShapes] = {0, 0, 0};
  // re-tuning when the particle count has changed by kRetuneFactor since the
  // last tuning: the live count of all instances is copied to page-locked
  // host memory after each pic_step call and read at the next one
  bool retune = true;                // off after pic_set_chunk with a fixed size
  int tunings = 0;                   // tunings completed
  long long tuned_at = 0;            // live particles (all instances) at the last tuning
  long long* d_live = nullptr;       // device: live particles after the last step
  long long* h_live = nullptr;       // page-locked copy
  cudaEvent_t live_ev = nullptr;     // recorded after the copy
  UNet* unet = nullptr;              // learned warm start (all instances)
  pic_alloc alloc;
  bool own_alloc = true;
  cudaStream_t stream = nullptr;
  int num_sms = 1;
  std::vector<void*> blocks;
  std::string err;
};

namespace {

int fail(pic_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

int cuda_fail(pic_handle* h, cudaError_t e, const char* what) {
  return fail(h, PIC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void* dev_alloc(pic_handle* h, size_t bytes) {
  if (bytes == 0) bytes = 256;
  bytes = (bytes + 255) & ~(size_t)255;
  void* p = nullptr;
  if (h->own_alloc) {
    if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
  } else {
    p = h->alloc.alloc(h->alloc.ctx, bytes);
  }
  if (p) h->blocks.push_back(p);
  return p;
}

int status_code(int st) {
  if (st & ST_NAN) return PIC_ERR_NAN;
  if (st & ST_CAPACITY) return PIC_ERR_CAPACITY;
  if (st & ST_TIMEOUT) return PIC_ERR_TIMEOUT;
  if (st & ST_NONCONV) return PIC_ERR_NONCONVERGED;
  return PIC_OK;
}

const char* status_text(int code) {
  switch (code) {
    case PIC_ERR_NAN: return "non-finite or out-of-domain particle";
    case PIC_ERR_CAPACITY: return "particle or birth capacity exceeded";
    case PIC_ERR_TIMEOUT: return "device wait reached its limit";
    case PIC_ERR_NONCONVERGED: return "Poisson solve did not converge";
    default: return "ok";
  }
}

// null-collision frequency: 1.001 max over a log grid of 100001 energies of
// (n_g sigma_T + n_meta sigma_1d) v
double nu_max_of(const pic_config& c) {
  double best = 0.0;
  for (int k = 0; k <= 100000; ++k) {
    double E = 1e-4 * std::pow(c.E_cap / 1e-4, k / 100000.0);
    if (k == 100000) E = c.E_cap;
    const double s_el = E > 0.0 ? c.sigma_el : 0.0;
    const double s_ex = E > c.exc_E ? c.exc_C * std::log(E / c.exc_E) / (E * c.exc_E) : 0.0;
    const double s_io = E > c.ion_I ? c.ion_a * std::log(E / c.ion_I) / (E * c.ion_I) : 0.0;
    const double s_md =
        E > c.meta_I ? c.meta_a * std::log(E / c.meta_I) / (E * c.meta_I) : 0.0;
    const double v = std::sqrt(2.0 * E * kQe / kMe);
    const double nu = (c.n_gas * (s_el + s_ex + s_io) + c.n_meta * s_md) * v;
    if (nu > best) best = nu;
  }
  return 1.001 * best;
}

std::string validate(const pic_config& c) {
  if (c.struct_size != sizeof(pic_config)) return "pic_config.struct_size mismatch";
  if (c.nr < 2 || c.nz < 2 || (c.nr & 1) || (c.nz & 1)) return "nr, nz must be even and >= 2";
  if ((long long)c.nr * c.nz > (1LL << 26)) return "grid too large";
  if (!(c.R > 0) || !(c.L > 0) || !(c.dt > 0) || !(c.weight > 0) || !(c.m_ion > 0))
    return "R, L, dt, weight, m_ion must be positive";
  if (c.Rc < 0) return "Rc must be >= 0";
  if (c.cap_e <= 0 || c.cap_i <= 0 || c.birth_cap <= 0) return "capacities must be positive";
  if (c.cap_e >= (1LL << 31) || c.cap_i >= (1LL << 31) || c.birth_cap >= (1LL << 30))
    return "capacities must stay below 2^31 (2^30 births)";
  if (c.precision != 0 && c.precision != 1) return "precision must be 0 (FP64) or 1 (FP32 particles)";
  if (c.sort_every < 1 || c.sort_every > 64) return "sort_every must be in [1, 64]";
  if (c.gather < 0 || c.gather > 1 || c.rweight < 0 || c.rweight > 1) return "gather/rweight";
  if (c.circuit_mode < 0 || c.circuit_mode > 1 || c.b_mode < 0 || c.b_mode > 1) return "modes";
  if (!(c.poisson_tol > 0) || c.poisson_max_iter < 1) return "poisson_tol/max_iter";
  if (c.n_avg < 1) return "n_avg must be >= 1";
  if (!(c.E_cap > 0)) return "E_cap must be positive";
  if (!(c.n_meta >= 0.0)) return "n_meta must be >= 0";
  if (c.n_meta > 0.0 && !(c.meta_I > 0.0 && c.meta_a >= 0.0)) return "meta_I > 0, meta_a >= 0";
  if ((c.gap_neumann != 0 && c.gap_neumann != 1) || (c.wall_neumann != 0 && c.wall_neumann != 1))
    return "gap_neumann, wall_neumann must be 0 or 1";
  if (c.ied_bins < 0 || c.ied_bins > 65536) return "ied_bins must be in [0, 65536]";
  if (c.phi_extrapolate != 0 && c.phi_extrapolate != 1) return "phi_extrapolate must be 0 or 1";
  if (c.poisson_precond != 0 && c.poisson_precond != 1) return "poisson_precond must be 0 or 1";
  if (c.ied_bins > 0 && !(c.ied_emax > 0.0)) return "ied_emax must be positive";
  if (!(c.band_r_lo <= c.band_r_hi)) return "band_r_lo must not exceed band_r_hi";
  return "";
}

// zero the region accumulators and the ion energy histogram of one instance
cudaError_t region_clear(const Inst& I, cudaStream_t st) {
  const RegionDev& R = I.reg;
  const size_t ncell = (size_t)I.nr * I.nz, nn = (size_t)(I.nr + 1) * (I.nz + 1);
  cudaError_t e = cudaMemsetAsync(R.ied, 0, (size_t)(I.ied_bins + 1) * 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(R.n[0], 0, ncell * 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(R.n[1], 0, ncell * 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(R.mom, 0, ncell * 32, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(R.phi, 0, nn * 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(R.samples, 0, 8, st);
  return e;
}

// The magnetic-field table in the order of the cell keys of the instance's
// tile shape (FP32 coefficients, or per species FP64 scaled by h = q dt / 2m:
// the push reads t = h B); synchronous.
cudaError_t upload_btab(const InstHost& ih, cudaStream_t st) {
  const Inst& I = ih.I;
  const int nr = I.nr, nz = I.nz;
  cudaError_t e = cudaSuccess;
  if (I.prec32) {
    std::vector<float4> bt((size_t)I.nkey * 2, make_float4(0.f, 0.f, 0.f, 0.f));
    for (int m = 0; m < nr; ++m)
      for (int n = 0; n < nz; ++n)
        for (int comp = 0; comp < 2; ++comp) {
          const double4_32a& v = ih.bcell[((size_t)m * nz + n) * 2 + comp];
          bt[(size_t)2 * cell_key(I, m, n) + comp] =
              make_float4((float)v.x, (float)v.y, (float)v.z, (float)v.w);
        }
    e = cudaMemcpyAsync(I.btab32, bt.data(), bt.size() * sizeof(float4), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  } else {
    for (int sp = 0; sp < 2 && e == cudaSuccess; ++sp) {
      const double hs = 0.5 * I.qm[sp] * I.dt;
      std::vector<double4_32a> bs((size_t)I.nkey * 2, make_d4(0, 0, 0, 0));
      for (int m = 0; m < nr; ++m)
        for (int n = 0; n < nz; ++n)
          for (int comp = 0; comp < 2; ++comp) {
            const double4_32a& v = ih.bcell[((size_t)m * nz + n) * 2 + comp];
            bs[(size_t)2 * cell_key(I, m, n) + comp] = make_d4(hs * v.x, hs * v.y, hs * v.z, hs * v.w);
          }
      e = cudaMemcpyAsync(I.btab[sp], bs.data(), bs.size() * sizeof(double4_32a),
                          cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // bs is freed at the loop end
    }
  }
  return e;
}

int build_instance(pic_handle* h, const pic_config& c, InstHost& ih) {
  ih.cfg = c;
  Inst& I = ih.I;
  std::memset(&I, 0, sizeof(I));
  I.nr = c.nr;
  I.nz = c.nz;
  ih.nkey_max = 0;
  for (int shape = 0; shape < kTileShapes; ++shape) {
    set_tile_shape(I, shape);
    ih.nkey_max = I.nkey > ih.nkey_max ? I.nkey : ih.nkey_max;
  }
  set_tile_shape(I, h->tile);
  I.R = c.R;
  I.L = c.L;
  I.Rc = c.Rc;
  I.dr = c.R / c.nr;
  I.dz = c.L / c.nz;
  I.inv_dr = 1.0 / I.dr;
  I.inv_dz = 1.0 / I.dz;
  I.m_cath = -1;
  for (int m = 0; m <= c.nr; ++m)
    if (m * I.dr <= c.Rc && m < c.nr) I.m_cath = m;
  I.sort_every = c.sort_every;
  I.bc_g = c.gap_neumann ? I.m_cath + 1 : c.nr + 1;
  I.bc_wall = c.wall_neumann ? 1 : 0;
  I.band_lo = c.band_r_lo;
  I.band_hi = c.band_r_hi;
  I.ied_bins = c.ied_bins;
  I.ied_de = c.ied_bins > 0 ? c.ied_emax / c.ied_bins : 1.0;
  I.dt = c.dt;
  I.weight = c.weight;
  I.qm[0] = -kQe / kMe;
  I.qm[1] = kQe / c.m_ion;
  I.mass[0] = kMe;
  I.mass[1] = c.m_ion;
  I.gamma[0] = c.gamma_e;
  I.gamma[1] = c.gamma_i;
  I.n_gas = c.n_gas;
  I.T_gas = c.T_gas;
  I.m_ion = c.m_ion;
  I.sigma_el = c.sigma_el;
  I.ion_a = c.ion_a;
  I.ion_I = c.ion_I;
  I.n_meta = c.n_meta;
  I.meta_a = c.meta_a;
  I.meta_I = c.meta_I;
  I.exc_C = c.exc_C;
  I.exc_E = c.exc_E;
  I.nu_max = nu_max_of(c);
  I.p_null = -std::expm1(-I.nu_max * c.dt);
  I.pnull32 = (unsigned long long)std::ceil(std::ldexp(I.p_null, 32));
  I.seed = c.seed;
  I.gather = c.gather;
  I.rweight = c.rweight;
  I.mcc_on = c.mcc_on;
  I.push_on = c.push_on;
  I.field_on = c.field_on;
  I.walls_reflect = c.walls_reflect;
  I.circuit_mode = c.circuit_mode;
  I.n_avg = c.n_avg;
  I.diag_every = c.diag_every > 0 ? c.diag_every : 1;
  I.Vc_fixed = c.Vc_fixed;
  I.Vs = c.Vs;
  I.Rext = c.Rext;
  I.poisson_tol = c.poisson_tol;
  I.phi_extrap = c.phi_extrapolate;
  I.poisson_max_iter = c.poisson_max_iter;
  I.cap[0] = c.cap_e;
  I.cap[1] = c.cap_i;
  I.birth_cap = c.birth_cap;

  const size_t nn = (size_t)(c.nr + 1) * (c.nz + 1);
  auto A = [&](size_t b) { return dev_alloc(h, b); };
  bool ok = true;
  auto chk = [&](void* p) { ok = ok && p != nullptr; return p; };
  const bool p32 = c.precision == 1;
  I.prec32 = p32 ? 1 : 0;
  I.hq32[0] = (float)(0.5 * I.qm[0] * c.dt);
  I.hq32[1] = (float)(0.5 * I.qm[1] * c.dt);
  I.kr32 = (float)(c.dt * I.inv_dr);
  I.kz32 = (float)(c.dt * I.inv_dz);
  I.kr64 = c.dt * I.inv_dr;
  I.kz64 = c.dt * I.inv_dz;
  for (int sp = 0; sp < 2; ++sp) {
    const size_t cap = (size_t)I.cap[sp];
    if (p32) {
      for (Particles32* P : {&I.buf32[sp][0], &I.buf32[sp][1]}) {
        P->a = (float4*)chk(A(cap * 16));
        P->b = (uint4*)chk(A(cap * 16));
      }
      I.qacc64[sp] = (double*)chk(A(nn * 8));
    } else {
      for (ParticlesDev* P : {&I.buf[sp][0], &I.buf[sp][1]}) {
        P->r = (double*)chk(A(cap * 8));
        P->z = (double*)chk(A(cap * 8));
        P->vr = (double*)chk(A(cap * 8));
        P->vt = (double*)chk(A(cap * 8));
        P->vz = (double*)chk(A(cap * 8));
        P->id = (long long*)chk(A(cap * 8));
      }
      I.key[sp] = (int*)chk(A(cap * 4));
      I.qacc[sp] = (unsigned long long*)chk(A(nn * 8));
    }
    I.counts[sp] = (int*)chk(A((size_t)ih.nkey_max * 4));
    I.cursor[sp] = (int*)chk(A((size_t)ih.nkey_max * 4));
    BirthsDev& B = I.births[sp];
    const size_t bc = (size_t)c.birth_cap;
    if (p32) {
      B.a32 = (float4*)chk(A(bc * 16));
      B.b32 = (uint4*)chk(A(bc * 16));
    } else {
      B.r = (double*)chk(A(bc * 8));
      B.z = (double*)chk(A(bc * 8));
      B.vr = (double*)chk(A(bc * 8));
      B.vt = (double*)chk(A(bc * 8));
      B.vz = (double*)chk(A(bc * 8));
      B.cell = (int*)chk(A(bc * 4));
      B.id = (long long*)chk(A(bc * 8));
    }
    B.pkey = (unsigned long long*)chk(A(bc * 8));
    long long P2 = 1;
    while (P2 < (long long)bc) P2 <<= 1;
    B.sort_len = P2;
    B.skey = (unsigned long long*)chk(A((size_t)P2 * 8));
    B.sidx = (unsigned int*)chk(A((size_t)P2 * 4));
  }
  I.phi = (double*)chk(A(nn * 8));
  I.phi_old = (double*)chk(A(nn * 8));
  I.Q = (double*)chk(A(nn * 8));
  I.qs[0] = (double*)chk(A(nn * 8));
  I.qs[1] = (double*)chk(A(nn * 8));
  if (p32) {
    I.etab32 = (float4*)chk(A((size_t)ih.nkey_max * (c.gather == 0 ? 1 : 2) * sizeof(float4)));
    I.btab32 = (float4*)chk(A((size_t)ih.nkey_max * 2 * sizeof(float4)));
    long long cmax = I.cap[0] > I.cap[1] ? I.cap[0] : I.cap[1];
    I.stage_len = cmax < (1LL << 22) ? cmax : (1LL << 22);
    I.stage = (double*)chk(A((size_t)I.stage_len * 6 * 8));
  } else {
    for (int sp = 0; sp < 2; ++sp) {
      I.etab[sp] = (double4_32a*)chk(A((size_t)ih.nkey_max * (c.gather == 0 ? 1 : 2) * sizeof(double4_32a)));
      I.btab[sp] = (double4_32a*)chk(A((size_t)ih.nkey_max * 2 * sizeof(double4_32a)));
    }
  }
  I.qhist = (double*)chk(A((size_t)c.n_avg * 8));
  const size_t ncell = (size_t)c.nr * c.nz;
  RegionDev& RG = I.reg;
  RG.ied = (unsigned long long*)chk(A((size_t)(c.ied_bins + 1) * 8));
  RG.n[0] = (unsigned long long*)chk(A(ncell * 8));
  RG.n[1] = (unsigned long long*)chk(A(ncell * 8));
  RG.mom = (double*)chk(A(ncell * 32));
  RG.phi = (double*)chk(A(nn * 8));
  RG.samples = (unsigned long long*)chk(A(8));
  RG.col = (double*)chk(A((size_t)c.nr * 64));
  RG.zs = (double*)chk(A((size_t)c.nr * 8));
  RG.zb = (double*)chk(A((size_t)c.nr * 8));
  RG.out = (double*)chk(A(64));
  I.S = (Scalars*)chk(A(sizeof(Scalars)));
  I.diag = (DiagDev*)chk(A(sizeof(DiagDev)));
  const size_t pwb = poisson_work_bytes(c.nr, c.nz);
  void* pwbase = chk(A(pwb));
  if (!ok) return fail(h, PIC_ERR_OOM, "device allocation failed");
  cudaStream_t st = h->stream;
  cudaError_t e = cudaSuccess;
  for (int sp = 0; sp < 2 && e == cudaSuccess; ++sp) {
    e = cudaMemsetAsync(I.counts[sp], 0, (size_t)ih.nkey_max * 4, st);
    // cell bin ends of the sorted arrays (all empty until particles are set)
    if (e == cudaSuccess) e = cudaMemsetAsync(I.cursor[sp], 0, (size_t)ih.nkey_max * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(p32 ? (void*)I.qacc64[sp] : (void*)I.qacc[sp], 0, nn * 8, st);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(I.phi, 0, nn * 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(I.phi_old, 0, nn * 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(I.Q, 0, nn * 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(I.qs[0], 0, nn * 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(I.qs[1], 0, nn * 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(I.qhist, 0, (size_t)c.n_avg * 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(I.diag, 0, sizeof(DiagDev), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(pwbase, 0, pwb, st);
  if (e == cudaSuccess) e = region_clear(I, st);
  if (e != cudaSuccess) return cuda_fail(h, e, "memset");
  ih.pw = poisson_work_init(pwbase, c.nr, c.nz, c.R, c.L, I.bc_g, I.bc_wall, h->num_sms);
  if (c.poisson_precond == 0 && poisson_sep_possible(ih.pw)) {
    void* sb = dev_alloc(h, poisson_sep_bytes(c.nr, c.nz));
    if (!sb) return fail(h, PIC_ERR_OOM, "device allocation failed");
    e = poisson_sep_attach(ih.pw, sb, h->num_sms, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "Poisson tables");
  }

  // static magnetic field: node values in FP64, folded per cell into
  // bilinear coefficients (B table keyed like the cells)
  std::vector<double> br(nn), bz(nn);
  for (int m = 0; m <= c.nr; ++m)
    for (int n = 0; n <= c.nz; ++n) {
      const double r = m * I.dr, z = n * I.dz;
      double vr = c.B0r, vz = c.B0z;
      if (c.b_mode == 0) {
        const double ex = std::exp(-c.B_k * z);
        vr = c.B_kA0 * ::j1(c.B_k * r) * ex;
        vz = c.B_kA0 * ::j0(c.B_k * r) * ex;
      }
      br[(size_t)m * (c.nz + 1) + n] = vr;
      bz[(size_t)m * (c.nz + 1) + n] = vz;
    }
  ih.bcell.assign((size_t)c.nr * c.nz * 2, make_d4(0, 0, 0, 0));
  for (int m = 0; m < c.nr; ++m)
    for (int n = 0; n < c.nz; ++n) {
      auto at = [&](const std::vector<double>& v, int a, int b) {
        return v[(size_t)(m + a) * (c.nz + 1) + (n + b)];
      };
      for (int comp = 0; comp < 2; ++comp) {
        const std::vector<double>& v = comp == 0 ? br : bz;
        const double b00 = at(v, 0, 0), b10 = at(v, 1, 0), b01 = at(v, 0, 1), b11 = at(v, 1, 1);
        ih.bcell[((size_t)m * c.nz + n) * 2 + comp] =
            make_d4(b00, b10 - b00, b01 - b00, b11 - b10 - b01 + b00);
      }
    }
  e = upload_btab(ih, st);
  if (e != cudaSuccess) return cuda_fail(h, e, "upload B table");
  Scalars s0;
  std::memset(&s0, 0, sizeof(s0));
  s0.Vc = c.circuit_mode == 1 ? -c.Vs : c.Vc_fixed;
  s0.diag_on = 1;
  e = cudaMemcpyAsync(I.S, &s0, sizeof(s0), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(h, e, "upload scalars");
  e = cudaStreamSynchronize(st);  // host vectors go out of scope
  if (e != cudaSuccess) return cuda_fail(h, e, "create sync");
  return PIC_OK;
}

int read_status(pic_handle* h, int instance, Scalars* out) {
  Scalars s;
  cudaError_t e = cudaMemcpyAsync(&s, h->inst[instance].I.S, sizeof(s), cudaMemcpyDeviceToHost,
                                  h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "read status");
  if (out) *out = s;
  const int code = status_code(s.status);
  if (code != PIC_OK) return fail(h, code, status_text(code));
  return PIC_OK;
}

bool bad_instance(pic_handle* h, int instance) {
  return !h || instance < 0 || instance >= (int)h->inst.size();
}

const char* kGroupNames[G_COUNT] = {"field_tables", "push", "births", "scan", "scatter",
                                   "charge", "circuit", "poisson", "step_end", "warm_start"};

void prof_mark(void* ctx, int group, bool begin, cudaStream_t st) {
  Profiler& P = *(Profiler*)ctx;
  if (P.used == P.pool.size()) {
    cudaEvent_t ev;
    if (cudaEventCreate(&ev) != cudaSuccess) return;
    P.pool.push_back(ev);
  }
  cudaEvent_t ev = P.pool[P.used++];
  cudaEventRecord(ev, st);
  if (begin) P.open[group] = ev;
  else P.recs.push_back({group, P.open[group], ev});
}

// index of the current particle buffer of a species (device-side parity)
int current_buffer(pic_handle* h, int instance, int sp) {
  Scalars s;
  read_status(h, instance, &s);
  return s.flip[sp] & 1;
}

}  // namespace

extern "C" {

int pic_create(const pic_config* cfgs, int n_instances, const pic_alloc* alloc, void* cuda_stream,
               pic_handle** out) {
  if (!out) return PIC_ERR_INVALID;
  *out = nullptr;
  if (!cfgs || n_instances < 1) return PIC_ERR_INVALID;
  for (int k = 0; k < n_instances; ++k)
    if (!validate(cfgs[k]).empty()) return PIC_ERR_INVALID;
  pic_handle* h = new pic_handle();
  if (alloc && alloc->alloc && alloc->free) {
    h->alloc = *alloc;
    h->own_alloc = false;
  }
  h->stream = (cudaStream_t)cuda_stream;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    delete h;
    return PIC_ERR_CUDA;
  }
  if (n_instances > kMaxInstances) {
    delete h;
    return PIC_ERR_INVALID;
  }
  for (int k = 1; k < n_instances; ++k)
    if (cfgs[k].gather != cfgs[0].gather || cfgs[k].precision != cfgs[0].precision) {
      delete h;
      return PIC_ERR_INVALID;   // one kernel variant serves all instances of a handle
    }
  h->inst.resize(n_instances);
  for (int k = 0; k < n_instances; ++k) {
    const int rc = build_instance(h, cfgs[k], h->inst[k]);
    if (rc != PIC_OK) {
      pic_destroy(h);
      return rc;
    }
  }
  {
    h->d_insts = (Inst*)dev_alloc(h, sizeof(Inst) * n_instances);
    h->d_queue = (WorkQueue*)dev_alloc(h, sizeof(WorkQueue));
    h->d_pargs = dev_alloc(h, poisson_args_bytes() * n_instances);
    h->d_live = (long long*)dev_alloc(h, sizeof(long long));
    if (!h->d_insts || !h->d_queue || !h->d_pargs || !h->d_live ||
        cudaHostAlloc((void**)&h->h_live, sizeof(long long), cudaHostAllocDefault) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->live_ev, cudaEventDisableTiming) != cudaSuccess) {
      pic_destroy(h);
      return PIC_ERR_OOM;
    }
    *h->h_live = -1;
    std::vector<Inst> hi(n_instances);
    for (int k = 0; k < n_instances; ++k) {
      hi[k] = h->inst[k].I;
      h->pws.push_back(h->inst[k].pw);
    }
    cudaError_t e = cudaMemcpyAsync(h->d_insts, hi.data(), sizeof(Inst) * n_instances,
                                    cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_queue, 0, sizeof(WorkQueue), h->stream);
    if (e == cudaSuccess)
      e = poisson_group_upload(h->pws.data(), hi.data(), n_instances, h->d_pargs, h->num_sms,
                               h->stream);
    if (e != cudaSuccess) {
      pic_destroy(h);
      return PIC_ERR_CUDA;
    }
  }
  *out = h;
  return PIC_OK;
}

void pic_destroy(pic_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  if (h->graph) cudaGraphExecDestroy(h->graph);
  for (cudaEvent_t ev : h->prof.pool) cudaEventDestroy(ev);
  if (h->live_ev) cudaEventDestroy(h->live_ev);
  if (h->h_live) cudaFreeHost(h->h_live);
  for (InstHost& ih : h->inst)
    if (ih.pw) poisson_work_free(ih.pw);
  if (h->unet) unet_destroy(h->unet);
  for (void* p : h->blocks) {
    if (h->own_alloc) cudaFree(p);
    else h->alloc.free(h->alloc.ctx, p);
  }
  delete h;
}

const char* pic_last_error(const pic_handle* h) { return h ? h->err.c_str() : "null handle"; }

// Between full sorts (sort_every > 1) the particle arrays hold dead slots and
// appended births; calls that read or replace particles first compact and
// sort them (the thinning kernels with factor 1 keep every live particle).
static int ensure_sorted(pic_handle* h, int instance) {
  Scalars s{};
  const int rc = read_status(h, instance, &s);
  if (rc != PIC_OK && rc != PIC_ERR_NONCONVERGED) return rc;
  if (!s.unsorted) return PIC_OK;
  cudaError_t e = launch_thin(h->inst[instance].I, 1, h->num_sms, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "compaction");
  return read_status(h, instance, nullptr);
}

// Device addresses of host arrays that the device can read in place (pinned
// memory under unified addressing); false when any of them is not such memory.
static bool device_views(const void* const* host, int k, const void** dev) {
  for (int i = 0; i < k; ++i) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, host[i]) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return false;
    dev[i] = a.devicePointer;
  }
  return true;
}

// pic_set_particles; `cells`: FP64 positions given in cell units already (a
// checkpoint's arrays, host memory), copied without conversion
static int set_particles(pic_handle* h, int instance, int species, int64_t n, const double* r,
                         const double* z, const double* vr, const double* vt, const double* vz,
                         const int64_t* id, int on_device, bool cells) {
  if (bad_instance(h, instance) || species < 0 || species > 1 || n < 0)
    return fail(h, PIC_ERR_INVALID, "bad instance/species/count");
  InstHost& ih = h->inst[instance];
  if (n > ih.I.cap[species]) return fail(h, PIC_ERR_CAPACITY, "n exceeds the species capacity");
  if (n > 0 && (!r || !z || !vr || !vt || !vz || !id))
    return fail(h, PIC_ERR_INVALID, "null array");
  {
    const int rc = ensure_sorted(h, instance);   // the other species must be compact too
    if (rc != PIC_OK && rc != PIC_ERR_NONCONVERGED) return rc;
  }
  cudaStream_t st = h->stream;
  cudaError_t e = cudaSuccess;
  // pinned host arrays are read in place by the kernels (faster than a copy engine)
  const void* hv[6] = {r, z, vr, vt, vz, id};
  const void* dv[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  const bool direct = !on_device && !cells && n > 0 && device_views(hv, 6, dv);
  if (ih.I.prec32) {
    e = launch_set_n(ih.I, species, n, st);
    if (direct) {
      if (e == cudaSuccess)
        e = launch_pack32(ih.I, species, 0, n, (const double*)dv[0], (const double*)dv[1],
                          (const double*)dv[2], (const double*)dv[3], (const double*)dv[4],
                          (const long long*)dv[5], h->num_sms, st);
    } else if (on_device) {
      if (e == cudaSuccess && n > 0)
        e = launch_pack32(ih.I, species, 0, n, r, z, vr, vt, vz, (const long long*)id, h->num_sms, st);
    } else {
      // host arrays: through the FP64 staging chunk
      const long long L = ih.I.stage_len;
      double* sg = ih.I.stage;
      for (long long off = 0; off < n && e == cudaSuccess; off += L) {
        const long long cnt = n - off < L ? n - off : L;
        const size_t b = (size_t)cnt * 8;
        const double* srcs[5] = {r + off, z + off, vr + off, vt + off, vz + off};
        for (int k = 0; k < 5 && e == cudaSuccess; ++k)
          e = cudaMemcpyAsync(sg + (size_t)k * L, srcs[k], b, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(sg + (size_t)5 * L, id + off, b, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
          e = launch_pack32(ih.I, species, off, cnt, sg, sg + L, sg + 2 * L, sg + 3 * L, sg + 4 * L,
                            (const long long*)(sg + 5 * L), h->num_sms, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // staging reused
      }
    }
    if (e == cudaSuccess) e = launch_sort_species32(ih.I, species, h->num_sms, st);
  } else {
    // positions go to cell units on the way in (launch_copy_in)
    const ParticlesDev& P = ih.I.buf[species][current_buffer(h, instance, species)];
    const size_t b = (size_t)n * 8;
    void* const dst[6] = {P.r, P.z, P.vr, P.vt, P.vz, P.id};
    if (direct) {
      e = launch_copy_in(dv, dst, n, ih.I, h->num_sms, st);
    } else if (on_device) {
      e = launch_copy_in(hv, dst, n, ih.I, h->num_sms, st);
    } else if (n > 0) {
      // pageable host arrays: copy, then convert the positions in place
      e = cudaMemcpyAsync(P.r, r, b, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(P.z, z, b, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(P.vr, vr, b, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(P.vt, vt, b, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(P.vz, vz, b, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(P.id, id, b, cudaMemcpyHostToDevice, st);
      const void* const in_place[6] = {P.r, P.z, P.vr, P.vt, P.vz, P.id};
      if (e == cudaSuccess && !cells) e = launch_copy_in(in_place, dst, n, ih.I, h->num_sms, st);
    }
    if (e == cudaSuccess) e = launch_set_n(ih.I, species, n, st);
    if (e == cudaSuccess) e = launch_sort_species(ih.I, species, h->num_sms, st);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "set_particles");
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(h, e, "set_particles sync");
  return read_status(h, instance, nullptr);
}

int pic_set_particles(pic_handle* h, int instance, int species, int64_t n, const double* r,
                      const double* z, const double* vr, const double* vt, const double* vz,
                      const int64_t* id, int on_device) {
  return set_particles(h, instance, species, n, r, z, vr, vt, vz, id, on_device, false);
}

int pic_count(pic_handle* h, int instance, int species, int64_t* n_out) {
  if (bad_instance(h, instance) || species < 0 || species > 1 || !n_out)
    return fail(h, PIC_ERR_INVALID, "bad argument");
  {
    const int rc = ensure_sorted(h, instance);
    if (rc != PIC_OK && rc != PIC_ERR_NONCONVERGED) return rc;
  }
  Scalars s;
  const int rc = read_status(h, instance, &s);
  *n_out = s.n[species];
  return rc;
}

int pic_get_particles(pic_handle* h, int instance, int species, double* r, double* z, double* vr,
                      double* vt, double* vz, int64_t* id, int on_device) {
  int64_t n = 0;
  int rc = pic_count(h, instance, species, &n);
  if (rc != PIC_OK && rc != PIC_ERR_NONCONVERGED) return rc;
  const Inst& I = h->inst[instance].I;
  cudaStream_t st = h->stream;
  cudaError_t e = cudaSuccess;
  bool host_convert = false;   // FP64 positions copied to pageable memory
  if (I.prec32) {
    if (on_device) {
      if (n > 0)
        e = launch_unpack32(I, species, 0, n, r, z, vr, vt, vz, (long long*)id, h->num_sms, st);
    } else {
      const long long L = I.stage_len;
      double* sg = I.stage;
      for (long long off = 0; off < n && e == cudaSuccess; off += L) {
        const long long cnt = n - off < L ? n - off : L;
        const size_t b = (size_t)cnt * 8;
        e = launch_unpack32(I, species, off, cnt, sg, sg + L, sg + 2 * L, sg + 3 * L, sg + 4 * L,
                            (long long*)(sg + 5 * L), h->num_sms, st);
        double* dsts[5] = {r, z, vr, vt, vz};
        for (int k = 0; k < 5 && e == cudaSuccess; ++k)
          if (dsts[k])
            e = cudaMemcpyAsync(dsts[k] + off, sg + (size_t)k * L, b, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && id)
          e = cudaMemcpyAsync(id + off, sg + (size_t)5 * L, b, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      }
    }
  } else {
    const ParticlesDev& P = I.buf[species][current_buffer(h, instance, species)];
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const size_t b = (size_t)n * 8;
    // positions leave cell units: by a kernel into device or page-locked
    // host memory, else copied and converted on the host (the same product
    // and clamp, from_cells)
    if (n > 0 && (r || z)) {
      const void* hv[2] = {r ? (const void*)r : (const void*)z, z ? (const void*)z : (const void*)r};
      const void* dvw[2] = {nullptr, nullptr};
      if (on_device) {
        e = launch_positions_out(I, P.r, P.z, r, z, n, h->num_sms, st);
      } else if (device_views(hv, 2, dvw)) {
        e = launch_positions_out(I, P.r, P.z, r ? (double*)dvw[0] : nullptr,
                                 z ? (double*)dvw[1] : nullptr, n, h->num_sms, st);
      } else {
        if (r) e = cudaMemcpyAsync(r, P.r, b, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && z) e = cudaMemcpyAsync(z, P.z, b, cudaMemcpyDeviceToHost, st);
        host_convert = true;
      }
    }
    if (n > 0) {
      if (e == cudaSuccess && vr) e = cudaMemcpyAsync(vr, P.vr, b, kind, st);
      if (e == cudaSuccess && vt) e = cudaMemcpyAsync(vt, P.vt, b, kind, st);
      if (e == cudaSuccess && vz) e = cudaMemcpyAsync(vz, P.vz, b, kind, st);
      if (e == cudaSuccess && id) e = cudaMemcpyAsync(id, P.id, b, kind, st);
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(h, e, "get_particles");
  if (host_convert) {
    for (int64_t i = 0; i < n; ++i) {
      if (r) r[i] = from_cells(r[i], I.dr, I.R);
      if (z) z[i] = from_cells(z[i], I.dz, I.L);
    }
  }
  return rc;
}

int pic_solve_fields(pic_handle* h, int instance) {
  if (bad_instance(h, instance)) return fail(h, PIC_ERR_INVALID, "bad instance");
  {
    const int rc = ensure_sorted(h, instance);
    if (rc != PIC_OK && rc != PIC_ERR_NONCONVERGED) return rc;
  }
  InstHost& ih = h->inst[instance];
  cudaError_t e = launch_solve_fields(ih.I, ih.pw, h->num_sms, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "solve_fields");
  return PIC_OK;
}

int pic_set_phi(pic_handle* h, int instance, const double* phi, int on_device) {
  if (bad_instance(h, instance) || !phi) return fail(h, PIC_ERR_INVALID, "bad argument");
  InstHost& ih = h->inst[instance];
  const size_t nn = (size_t)(ih.cfg.nr + 1) * (ih.cfg.nz + 1);
  cudaError_t e = cudaMemcpyAsync(ih.I.phi, phi, nn * 8,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  h->stream);
  // no earlier solution: the next step's extrapolation starts from this phi
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ih.I.phi_old, ih.I.phi, nn * 8, cudaMemcpyDeviceToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "set_phi");
  return PIC_OK;
}

int pic_get_fields(pic_handle* h, int instance, double* phi, double* rho, double* Q, int on_device) {
  if (bad_instance(h, instance)) return fail(h, PIC_ERR_INVALID, "bad instance");
  InstHost& ih = h->inst[instance];
  const pic_config& c = ih.cfg;
  const size_t nn = (size_t)(c.nr + 1) * (c.nz + 1);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  cudaError_t e = cudaSuccess;
  if (phi) e = cudaMemcpyAsync(phi, ih.I.phi, nn * 8, kind, h->stream);
  if (e == cudaSuccess && Q) e = cudaMemcpyAsync(Q, ih.I.Q, nn * 8, kind, h->stream);
  std::vector<double> qh;
  if (e == cudaSuccess && rho) {
    qh.resize(nn);
    e = cudaMemcpyAsync(qh.data(), ih.I.Q, nn * 8, cudaMemcpyDeviceToHost, h->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "get_fields");
  if (rho) {
    // rho = Q / V with the node control volumes (half volume on z walls)
    std::vector<double> rh(nn);
    const double dr = c.R / c.nr, dz = c.L / c.nz;
    for (int m = 0; m <= c.nr; ++m) {
      double area;
      if (m == 0) area = kPi * 0.25 * dr * dr;
      else if (m == c.nr) area = kPi * (c.R * c.R - (c.R - 0.5 * dr) * (c.R - 0.5 * dr));
      else area = 2.0 * kPi * (m * dr) * dr;
      for (int n = 0; n <= c.nz; ++n) {
        const double hz = (n == 0 || n == c.nz) ? 0.5 : 1.0;
        rh[(size_t)m * (c.nz + 1) + n] = qh[(size_t)m * (c.nz + 1) + n] / (area * dz * hz);
      }
    }
    if (on_device) e = cudaMemcpy(rho, rh.data(), nn * 8, cudaMemcpyHostToDevice);
    else std::memcpy(rho, rh.data(), nn * 8);
    if (e != cudaSuccess) return cuda_fail(h, e, "get_fields rho");
  }
  return PIC_OK;
}

int pic_get_species_charge(pic_handle* h, int instance, int species, double* Q, int on_device) {
  if (bad_instance(h, instance) || species < 0 || species > 1 || !Q)
    return fail(h, PIC_ERR_INVALID, "bad argument");
  InstHost& ih = h->inst[instance];
  const size_t nn = (size_t)(ih.cfg.nr + 1) * (ih.cfg.nz + 1);
  cudaError_t e = cudaMemcpyAsync(Q, ih.I.qs[species], nn * 8,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                  h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "get_species_charge");
  return PIC_OK;
}

int pic_set_circuit(pic_handle* h, int instance, double Vc, int64_t step, const double* qhist,
                    int n) {
  if (bad_instance(h, instance) || step < 0 || n < 0 || (n > 0 && !qhist))
    return fail(h, PIC_ERR_INVALID, "bad argument");
  InstHost& ih = h->inst[instance];
  Scalars s;
  int rc = read_status(h, instance, &s);
  (void)rc;
  s.Vc = Vc;
  s.step = step;
  s.diag_on = (step % ih.I.diag_every) == 0;
  std::vector<double> q((size_t)ih.cfg.n_avg, 0.0);
  for (int k = 0; k < n && k < ih.cfg.n_avg; ++k) q[k] = qhist[k];
  cudaError_t e = cudaMemcpyAsync(ih.I.S, &s, sizeof(s), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ih.I.qhist, q.data(), q.size() * 8, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "set_circuit");
  return PIC_OK;
}

int pic_set_next_id(pic_handle* h, int instance, int64_t next_id) {
  if (bad_instance(h, instance) || next_id < 0) return fail(h, PIC_ERR_INVALID, "bad argument");
  Scalars s;
  read_status(h, instance, &s);
  s.next_id = next_id;
  cudaError_t e = cudaMemcpyAsync(h->inst[instance].I.S, &s, sizeof(s), cudaMemcpyHostToDevice,
                                  h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "set_next_id");
  return PIC_OK;
}

int pic_get_next_id(pic_handle* h, int instance, int64_t* next_id) {
  if (bad_instance(h, instance) || !next_id) return fail(h, PIC_ERR_INVALID, "bad argument");
  Scalars s;
  const int rc = read_status(h, instance, &s);
  *next_id = s.next_id;
  return rc;
}

// One step of an ensemble: field tables per instance, both species pushed by
// persistent CTAs over a queue of (instance, chunk) items, the rest of the
// particle step per instance, all Poisson solves in one grouped launch.
static const int kTuneCandidates[4] = {4, 8, 16, 32};

static cudaError_t launch_ensemble_step(pic_handle* h, const StepMarks* marks) {
  auto mk = [&](int g, bool b) {
    if (marks) marks->mark(marks->ctx, g, b, h->stream);
  };
  const int n = (int)h->inst.size();
  const Inst& I0 = h->inst[0].I;
  cudaStream_t st = h->stream;
  cudaError_t e = cudaSuccess;
  BatchDims bd{};
  for (const InstHost& ih : h->inst) {
    const long long cells = (long long)ih.I.nr * ih.I.nz;
    const long long nodes = (long long)(ih.I.nr + 1) * (ih.I.nz + 1);
    bd.cells_max = cells > bd.cells_max ? cells : bd.cells_max;
    bd.nodes_max = nodes > bd.nodes_max ? nodes : bd.nodes_max;
    bd.birth_cap_max = ih.I.birth_cap > bd.birth_cap_max ? ih.I.birth_cap : bd.birth_cap_max;
    bd.any_append = bd.any_append || ih.I.sort_every > 1;
  }
  bd.prec32 = I0.prec32;
  bool plain = true;   // the model's own switches in every instance (fixed at creation)
  for (const InstHost& ih : h->inst)
    plain = plain && ih.I.push_on && ih.I.rweight == 0 && !ih.I.walls_reflect;
  mk(G_FIELD, true);
  if (e == cudaSuccess) e = launch_field_tables_batch(h->d_insts, n, bd, h->num_sms, st);
  mk(G_FIELD, false);
  const int threads = 256;
  mk(G_PUSH, true);
  if (e == cudaSuccess) e = launch_queue_setup(h->d_insts, h->d_queue, n, (long long)h->ppt * threads, st);
  if (e == cudaSuccess)
    e = launch_push_all(h->d_insts, h->d_queue, I0.prec32, I0.gather, plain, h->ppt, h->num_sms,
                        st);
  mk(G_PUSH, false);
  mk(G_SCATTER, true);
  if (e == cudaSuccess) e = launch_post_push_batch(h->d_insts, n, bd, h->num_sms, st);
  mk(G_SCATTER, false);
  if (e == cudaSuccess && h->unet && unet_pre_solve_needed(h->unet)) {
    mk(G_WARM, true);
    e = launch_pre_solve(h->unet, h->d_insts, h->d_pargs, n, st);
    mk(G_WARM, false);
  }
  mk(G_POISSON, true);
  if (e == cudaSuccess) e = launch_poisson_group(h->pws.data(), nullptr, n, h->d_pargs, h->num_sms, st);
  mk(G_POISSON, false);
  if (e == cudaSuccess && h->unet) e = launch_after_solve(h->unet, h->d_insts, n, st);
  mk(G_STEP_END, true);
  if (e == cudaSuccess) e = launch_step_end_batch(h->d_insts, n, st);
  mk(G_STEP_END, false);
  return e;
}

// launches around the Poisson solve of a single-instance step: the learned
// warm start before it, snapshot recording and iteration counts after it
static cudaError_t hook_pre_poisson(void* ctx, const Inst& I, PoissonWork* pw, cudaStream_t st) {
  (void)I;
  (void)pw;
  const pic_handle* h = (const pic_handle*)ctx;
  return launch_pre_solve(h->unet, h->d_insts, h->d_pargs, 1, st);
}
static cudaError_t hook_post_poisson(void* ctx, const Inst& I, cudaStream_t st) {
  (void)I;
  const pic_handle* h = (const pic_handle*)ctx;
  return launch_after_solve(h->unet, h->d_insts, 1, st);
}

static cudaError_t launch_all(pic_handle* h, const StepMarks* marks) {
  if (h->inst.size() > 1) return launch_ensemble_step(h, marks);
  StepHooks hooks{nullptr, nullptr, h};
  if (h->unet) {
    hooks.post_poisson = hook_post_poisson;
    if (unet_pre_solve_needed(h->unet)) hooks.pre_poisson = hook_pre_poisson;
  }
  cudaError_t e = cudaSuccess;
  for (InstHost& ih : h->inst)
    if (e == cudaSuccess)
      e = launch_step(ih.I, ih.pw, h->num_sms, h->stream, marks, h->unet ? &hooks : nullptr,
                      h->d_insts, h->d_queue, h->ppt);
  return e;
}

// Online autotuner of the push: the first steps of a handle run one
// candidate chunk size each (timed with events around the push); the fastest
// is kept for the rest of the run.
// The push gets slower as the arrays lose their cell order between full
// sorts, so every tuning step ends with a full sort: each candidate is timed
// on freshly sorted arrays (set_particles and pic_load leave them sorted).
static cudaError_t force_sorts(pic_handle* h, int on) {
  cudaError_t e = cudaSuccess;
  for (InstHost& ih : h->inst)
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&ih.I.S->sort_force, &on, sizeof(int), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return e;
}

// live particles of all instances: `out` after a synchronous read (tuning),
// or copied to h_live behind the step's work (read at the next pic_step)
static cudaError_t enqueue_live_count(pic_handle* h) {
  cudaError_t e = launch_live_total(h->d_insts, (int)h->inst.size(), h->d_live, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->h_live, h->d_live, sizeof(long long), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaEventRecord(h->live_ev, h->stream);
  return e;
}

static cudaError_t live_count(pic_handle* h, long long* out) {
  cudaError_t e = enqueue_live_count(h);
  if (e == cudaSuccess) e = cudaEventSynchronize(h->live_ev);
  if (e == cudaSuccess) *out = *h->h_live;
  return e;
}

static void drop_graph(pic_handle* h);

// Switch every instance to cell tile shape `shape`: the keys, the B table in
// the new key order and the particles re-sorted by the new keys (compacted,
// as after a full sort); the captured step is dropped.
static int apply_tile(pic_handle* h, int shape) {
  if (shape == h->tile) return PIC_OK;
  drop_graph(h);
  cudaError_t e = cudaSuccess;
  for (InstHost& ih : h->inst) {
    set_tile_shape(ih.I, shape);
    if (e == cudaSuccess) e = upload_btab(ih, h->stream);
  }
  std::vector<Inst> hi;
  for (const InstHost& ih : h->inst) hi.push_back(ih.I);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->d_insts, hi.data(), sizeof(Inst) * hi.size(), cudaMemcpyHostToDevice,
                        h->stream);
  for (InstHost& ih : h->inst)
    if (e == cudaSuccess) e = launch_thin(ih.I, 1, h->num_sms, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "tile shape");
  h->tile = shape;
  for (int k = 0; k < (int)h->inst.size(); ++k) {
    const int rc = read_status(h, k, nullptr);
    if (rc != PIC_OK && rc != PIC_ERR_NONCONVERGED) return rc;
  }
  return PIC_OK;
}

// Tuning sequence: steps 0..3 time the chunk sizes on the current tile shape;
// then (unless the shape is fixed) steps 4 and 5 time the other two shapes
// with the chosen chunk size, each after re-sorting the particles by its keys,
// and the fastest shape is kept.
static int autotune_step(pic_handle* h) {
  const int c = h->tune_next;
  if (c < 4) h->ppt = kTuneCandidates[c];
  if (c == 0) {
    h->tile0 = h->tile;
    const cudaError_t e0 = force_sorts(h, 1);
    if (e0 != cudaSuccess) return cuda_fail(h, e0, "tune");
  }
  int shape = h->tile;
  if (c >= 4) {
    shape = (h->tile0 + (c - 3)) % kTileShapes;
    const int rc = apply_tile(h, shape);
    if (rc != PIC_OK) return rc;
  }
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  struct Ctx { cudaEvent_t a, b; } ctx{a, b};
  StepMarks marks{[](void* p, int g, bool begin, cudaStream_t st) {
                    Ctx* x = (Ctx*)p;
                    if (g == G_PUSH && begin) cudaEventRecord(x->a, st);
                    if (g == G_PUSH && !begin) cudaEventRecord(x->b, st);
                  },
                  &ctx};
  const cudaError_t e = launch_all(h, &marks);
  float ms = 0.0f;
  if (e == cudaSuccess && cudaEventSynchronize(b) == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return cuda_fail(h, e, "step");
  if (c < 4) h->tune_ms[c] = ms;
  else h->tile_ms[shape] = ms;
  ++h->tune_next;
  if (h->tune_next == 4) {
    int best = 0;
    for (int k = 1; k < 4; ++k)
      if (h->tune_ms[k] < h->tune_ms[best]) best = k;
    h->ppt = kTuneCandidates[best];
    h->tile_ms[h->tile0] = h->tune_ms[best];
  }
  if ((h->tune_next == 4 && !h->tile_tune) || h->tune_next == 4 + kTileShapes - 1) {
    if (h->tune_next > 4) {
      int best = 0;
      for (int k = 1; k < kTileShapes; ++k)
        if (h->tile_ms[k] < h->tile_ms[best]) best = k;
      const int rc = apply_tile(h, best);
      if (rc != PIC_OK) return rc;
    }
    h->tune_next = -1;
    ++h->tunings;
    long long live = 0;
    const cudaError_t e2 = live_count(h, &live);
    if (e2 != cudaSuccess) return cuda_fail(h, e2, "tune");
    h->tuned_at = live;
    const cudaError_t e1 = force_sorts(h, 0);
    if (e1 != cudaSuccess) return cuda_fail(h, e1, "tune");
  }
  return PIC_OK;
}

// the step's launch sequence changed: capture a new graph at the next step
static void drop_graph(pic_handle* h) {
  if (h->graph) {
    cudaStreamSynchronize(h->stream);
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  h->graph_failed = false;
}

// Capture one time step of every instance into a CUDA graph.  Every step
// launches the same kernels with the same arguments (buffer parity, counts and
// the step index live on the device), so the graph is replayed as is.
static void build_graph(pic_handle* h) {
  cudaStreamCaptureStatus cs;
  if (cudaStreamIsCapturing(h->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    h->graph_failed = true;
    return;
  }
  if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    h->graph_failed = true;
    return;
  }
  bool ok = launch_all(h, nullptr) == cudaSuccess;
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(h->stream, &g);
  ok = ok && e == cudaSuccess && g != nullptr;
  cudaGraphExec_t ex = nullptr;
  if (ok) ok = cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();
  if (ok) h->graph = ex;
  else h->graph_failed = true;
}

static int step_calls(pic_handle* h, int64_t nsteps);
static const double kRetuneFactor = 4.0;

// Re-tune the push when the live particle count seen after the previous call
// differs from the count at the last tuning by kRetuneFactor or more (the
// best chunk size depends on the work per instance); the captured graph is
// rebuilt after the tuning steps.
static void check_retune(pic_handle* h) {
  if (!h->retune || h->tune_next >= 0 || h->tunings == 0) return;
  if (cudaEventQuery(h->live_ev) != cudaSuccess) {
    cudaGetLastError();   // not done yet: look again at the next call
    return;
  }
  const long long live = *h->h_live;
  if (live < 0 || h->tuned_at <= 0) return;
  const double ratio = (double)live / (double)h->tuned_at;
  if (ratio >= kRetuneFactor || ratio <= 1.0 / kRetuneFactor) {
    drop_graph(h);
    h->tune_next = 0;
  }
}

int pic_step(pic_handle* h, int64_t nsteps) {
  if (!h || nsteps < 0) return fail(h, PIC_ERR_INVALID, "bad argument");
  if (nsteps == 0) return PIC_OK;
  check_retune(h);
  const int rc = step_calls(h, nsteps);
  if (rc != PIC_OK) return rc;
  const cudaError_t e = enqueue_live_count(h);
  if (e != cudaSuccess) return cuda_fail(h, e, "live count");
  return PIC_OK;
}

static int step_calls(pic_handle* h, int64_t nsteps) {
  // the first steps of a handle tune the push's chunk size
  while (h->tune_next >= 0 && nsteps > 0) {
    const int rc = autotune_step(h);
    if (rc != PIC_OK) return rc;
    --nsteps;
  }
  if (nsteps == 0) return PIC_OK;
  // graphs need a capturable stream; profiling needs the per-kernel events
  const bool use_graph = !h->prof.on && h->stream != nullptr && !h->graph_failed;
  if (use_graph && !h->graph) build_graph(h);
  if (use_graph && h->graph) {
    for (int64_t s = 0; s < nsteps; ++s) {
      const cudaError_t e = cudaGraphLaunch(h->graph, h->stream);
      if (e != cudaSuccess) return cuda_fail(h, e, "graph launch");
    }
    return PIC_OK;
  }
  StepMarks marks{prof_mark, &h->prof};
  for (int64_t s = 0; s < nsteps; ++s) {
    const cudaError_t e = launch_all(h, h->prof.on ? &marks : nullptr);
    if (e != cudaSuccess) return cuda_fail(h, e, "step launch");
  }
  return PIC_OK;
}

int pic_set_chunk(pic_handle* h, int particles_per_thread) {
  if (!h) return PIC_ERR_INVALID;
  int k = -1;
  for (int j = 0; j < 4; ++j)
    if (kTuneCandidates[j] == particles_per_thread) k = j;
  if (particles_per_thread != 0 && k < 0)
    return fail(h, PIC_ERR_INVALID, "particles_per_thread must be 0, 4, 8, 16 or 32");
  drop_graph(h);
  if (h->tune_next > 0) {   // tuning was under way: its forced sorts end here
    const cudaError_t e = force_sorts(h, 0);
    if (e != cudaSuccess) return cuda_fail(h, e, "set_chunk");
  }
  if (k >= 0) {
    h->ppt = particles_per_thread;
    h->tune_next = -1;
    h->retune = false;      // fixed by the caller
  } else {
    h->tune_next = 0;       // tune again over the next steps
    h->retune = true;
  }
  return PIC_OK;
}

int pic_set_tile(pic_handle* h, int shape) {
  if (!h) return PIC_ERR_INVALID;
  if (shape < 0 || shape > kTileShapes) return fail(h, PIC_ERR_INVALID, "shape must be 0, 1, 2 or 3");
  if (shape == 0) {
    h->tile_tune = true;
    drop_graph(h);
    if (h->tune_next > 0) {
      const cudaError_t e = force_sorts(h, 0);
      if (e != cudaSuccess) return cuda_fail(h, e, "set_tile");
    }
    h->tune_next = 0;       // tune chunk size and tile shape over the next steps
    h->retune = true;
    return PIC_OK;
  }
  h->tile_tune = false;
  if (h->tune_next >= 4) {  // the shape trials of a tuning end here (its chunk size is chosen)
    h->tune_next = -1;
    ++h->tunings;
    const cudaError_t e = force_sorts(h, 0);
    if (e != cudaSuccess) return cuda_fail(h, e, "set_tile");
  }
  return apply_tile(h, shape - 1);
}

int pic_tuned_tile(pic_handle* h, int* shape) {
  if (!h || !shape) return PIC_ERR_INVALID;
  *shape = h->tile + 1;
  return PIC_OK;
}

int pic_autotune_info(pic_handle* h, int* tunings, int* particles_per_thread,
                      int64_t* particles_at_tuning) {
  if (!h) return PIC_ERR_INVALID;
  if (tunings) *tunings = h->tunings;
  if (particles_per_thread) *particles_per_thread = h->tune_next < 0 ? h->ppt : 0;
  if (particles_at_tuning) *particles_at_tuning = h->tuned_at;
  return PIC_OK;
}

int pic_tuned_chunk(pic_handle* h, int* particles_per_thread) {
  if (!h || !particles_per_thread) return PIC_ERR_INVALID;
  *particles_per_thread = h->tune_next < 0 ? h->ppt : 0;
  return PIC_OK;
}

int pic_uses_graph(pic_handle* h) { return h && h->graph ? 1 : 0; }

int pic_sync(pic_handle* h) {
  if (!h) return PIC_ERR_INVALID;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "sync");
  for (int k = 0; k < (int)h->inst.size(); ++k) {
    const int rc = read_status(h, k, nullptr);
    if (rc != PIC_OK) return rc;
  }
  return PIC_OK;
}

int pic_diagnostics(pic_handle* h, int instance, pic_diag* out) {
  if (bad_instance(h, instance) || !out) return fail(h, PIC_ERR_INVALID, "bad argument");
  DiagDev d;
  cudaError_t e = cudaMemcpyAsync(&d, h->inst[instance].I.diag, sizeof(d), cudaMemcpyDeviceToHost,
                                  h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "diagnostics");
  out->t = d.t;
  out->I_cath = d.I_cath;
  out->V_cath = d.V_cath;
  out->n_e_peak = d.n_e_peak;
  out->n_i_peak = d.n_i_peak;
  out->W_field = d.W_field;
  out->K_e = d.K_e;
  out->K_i = d.K_i;
  out->N_e = d.N_e;
  out->N_i = d.N_i;
  out->n_ion_cath = d.n_ion_cath;
  out->n_e_cath = d.n_e_cath;
  out->n_sey = d.n_sey;
  out->n_ionize = d.n_ionize;
  out->n_excite = d.n_excite;
  out->n_elastic = d.n_elastic;
  out->n_ionize_meta = d.n_ionize_meta;
  out->ppc_max_e = d.ppc_max[0];
  out->ppc_max_i = d.ppc_max[1];
  out->weight = h->inst[instance].I.weight;
  out->step = d.step;
  out->particle_steps = d.particle_steps;
  out->poisson_iters = d.poisson_iters;
  out->poisson_resid = d.poisson_resid;
  Scalars s;
  const int rc = read_status(h, instance, &s);
  out->status = rc;
  return rc;
}

// New macroparticle weight of one instance: host copies, the device copy
// read by the push, and the captured step (its kernels hold the weight by
// value).
static int set_weight(pic_handle* h, int instance, double w) {
  InstHost& ih = h->inst[instance];
  ih.cfg.weight = w;
  ih.I.weight = w;
  drop_graph(h);
  cudaError_t e = cudaMemcpyAsync(h->d_insts + instance, &ih.I, sizeof(Inst), cudaMemcpyHostToDevice,
                                  h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "weight upload");
  return PIC_OK;
}

int pic_reweight(pic_handle* h, int instance, int factor) {
  if (bad_instance(h, instance) || factor < 1) return fail(h, PIC_ERR_INVALID, "bad argument");
  if (factor == 1) return read_status(h, instance, nullptr);
  InstHost& ih = h->inst[instance];
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "reweight sync");
  int rc = read_status(h, instance, nullptr);
  if (rc != PIC_OK && rc != PIC_ERR_NONCONVERGED) return rc;
  e = launch_thin(ih.I, factor, h->num_sms, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "reweight");
  rc = set_weight(h, instance, ih.I.weight * (double)factor);
  if (rc != PIC_OK) return rc;
  return read_status(h, instance, nullptr);
}

// ---------------------------------------------------------------------------
// region diagnostics
// ---------------------------------------------------------------------------
int pic_region_sample(pic_handle* h, int instance) {
  if (bad_instance(h, instance)) return fail(h, PIC_ERR_INVALID, "bad instance");
  {
    const int rc = ensure_sorted(h, instance);   // the sampler walks the cell bins
    if (rc != PIC_OK && rc != PIC_ERR_NONCONVERGED) return rc;
  }
  const cudaError_t e = launch_region_sample(h->inst[instance].I, h->num_sms, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "region sample");
  return PIC_OK;
}

int pic_region_read(pic_handle* h, int instance, pic_regions* out, double* zs, double* zb,
                    int64_t* ied, int64_t* ied_overflow) {
  if (bad_instance(h, instance) || !out) return fail(h, PIC_ERR_INVALID, "bad argument");
  const Inst& I = h->inst[instance].I;
  cudaStream_t st = h->stream;
  cudaError_t e = launch_region_eval(I, st);
  double o[8];
  unsigned long long samples = 0;
  std::vector<unsigned long long> hist((size_t)I.ied_bins + 1);
  if (e == cudaSuccess) e = cudaMemcpyAsync(o, I.reg.out, sizeof(o), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&samples, I.reg.samples, 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hist.data(), I.reg.ied, hist.size() * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && zs)
    e = cudaMemcpyAsync(zs, I.reg.zs, (size_t)I.nr * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && zb)
    e = cudaMemcpyAsync(zb, I.reg.zb, (size_t)I.nr * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(h, e, "region read");
  out->samples = (int64_t)samples;
  long long impacts = 0;
  for (int k = 0; k < 3; ++k) {
    out->Te[k] = o[k];
    out->ncell[k] = (int64_t)o[3 + k];
  }
  out->z_sheath = o[6];
  out->z_bulk = o[7];
  for (int b = 0; b <= I.ied_bins; ++b) {
    impacts += (long long)hist[b];
    if (ied && b < I.ied_bins) ied[b] = (int64_t)hist[b];
  }
  if (ied_overflow) *ied_overflow = (int64_t)hist[I.ied_bins];
  out->ion_impacts = impacts;
  return read_status(h, instance, nullptr);
}

int pic_region_reset(pic_handle* h, int instance) {
  if (bad_instance(h, instance)) return fail(h, PIC_ERR_INVALID, "bad instance");
  const cudaError_t e = region_clear(h->inst[instance].I, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "region reset");
  return PIC_OK;
}

// ---------------------------------------------------------------------------
// checkpoints: a flat little-endian file
//   "PICCKPT4", pic_config, Scalars, qhist[n_avg], phi[nodes], phi_old[nodes],
//   then per species: n, r[n], z[n], vr[n], vt[n], vz[n], id[n] (the device
//   arrays as they are: positions in cell units) or, in FP32 mode, the raw
//   records
// ---------------------------------------------------------------------------
int pic_save(pic_handle* h, int instance, const char* path) {
  if (bad_instance(h, instance) || !path) return fail(h, PIC_ERR_INVALID, "bad argument");
  InstHost& ih = h->inst[instance];
  Scalars s;
  int rc = ensure_sorted(h, instance);
  if (rc != PIC_OK) return rc;
  rc = read_status(h, instance, &s);
  if (rc != PIC_OK) return rc;
  const pic_config& c = ih.cfg;
  const size_t nn = (size_t)(c.nr + 1) * (c.nz + 1);
  std::vector<double> qh((size_t)c.n_avg), phi(nn), phi_old(nn);
  cudaError_t e = cudaMemcpy(qh.data(), ih.I.qhist, qh.size() * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(phi.data(), ih.I.phi, nn * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(phi_old.data(), ih.I.phi_old, nn * 8, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "save copy");
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(h, PIC_ERR_IO, std::string("cannot open ") + path);
  bool ok = std::fwrite("PICCKPT4", 1, 8, f) == 8;
  ok = ok && std::fwrite(&c, sizeof(c), 1, f) == 1;
  ok = ok && std::fwrite(&s, sizeof(s), 1, f) == 1;
  ok = ok && std::fwrite(qh.data(), 8, qh.size(), f) == qh.size();
  ok = ok && std::fwrite(phi.data(), 8, nn, f) == nn;
  ok = ok && std::fwrite(phi_old.data(), 8, nn, f) == nn;
  for (int sp = 0; sp < 2 && ok; ++sp) {
    const long long n = s.n[sp];
    ok = std::fwrite(&n, 8, 1, f) == 1;
    if (ih.I.prec32) {
      // raw FP32 records: the checkpoint restores the state bit for bit
      std::vector<float4> ra((size_t)n);
      std::vector<uint4> rb((size_t)n);
      if (ok && n > 0 &&
          (cudaMemcpy(ra.data(), ih.I.buf32[sp][s.flip[sp] & 1].a, (size_t)n * 16, cudaMemcpyDeviceToHost) != cudaSuccess ||
           cudaMemcpy(rb.data(), ih.I.buf32[sp][s.flip[sp] & 1].b, (size_t)n * 16, cudaMemcpyDeviceToHost) != cudaSuccess))
        ok = false;
      ok = ok && std::fwrite(ra.data(), 16, (size_t)n, f) == (size_t)n;
      ok = ok && std::fwrite(rb.data(), 16, (size_t)n, f) == (size_t)n;
      continue;
    }
    std::vector<double> buf((size_t)n);
    std::vector<long long> ids((size_t)n);
    const ParticlesDev& P = ih.I.buf[sp][s.flip[sp] & 1];
    for (double* src : {P.r, P.z, P.vr, P.vt, P.vz}) {
      if (!ok) break;
      if (n > 0 && cudaMemcpy(buf.data(), src, (size_t)n * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
        ok = false;
      ok = ok && std::fwrite(buf.data(), 8, (size_t)n, f) == (size_t)n;
    }
    if (ok && n > 0 && cudaMemcpy(ids.data(), P.id, (size_t)n * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
      ok = false;
    ok = ok && std::fwrite(ids.data(), 8, (size_t)n, f) == (size_t)n;
  }
  ok = (std::fclose(f) == 0) && ok;
  return ok ? PIC_OK : fail(h, PIC_ERR_IO, "checkpoint write failed");
}

int pic_load(pic_handle* h, int instance, const char* path) {
  if (bad_instance(h, instance) || !path) return fail(h, PIC_ERR_INVALID, "bad argument");
  InstHost& ih = h->inst[instance];
  const pic_config& c = ih.cfg;
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(h, PIC_ERR_IO, std::string("cannot open ") + path);
  char magic[8];
  pic_config fc;
  Scalars s;
  const size_t nn = (size_t)(c.nr + 1) * (c.nz + 1);
  std::vector<double> qh((size_t)c.n_avg), phi(nn), phi_old(nn);
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "PICCKPT4", 8) == 0;
  ok = ok && std::fread(&fc, sizeof(fc), 1, f) == 1;
  ok = ok && fc.nr == c.nr && fc.nz == c.nz && fc.n_avg == c.n_avg && fc.precision == c.precision;
  ok = ok && std::fread(&s, sizeof(s), 1, f) == 1;
  ok = ok && std::fread(qh.data(), 8, qh.size(), f) == qh.size();
  ok = ok && std::fread(phi.data(), 8, nn, f) == nn;
  ok = ok && std::fread(phi_old.data(), 8, nn, f) == nn;
  std::vector<double> arr[2][5];
  std::vector<long long> ids[2];
  std::vector<float4> ra[2];
  std::vector<uint4> rb[2];
  long long n[2] = {0, 0};
  for (int sp = 0; sp < 2 && ok; ++sp) {
    ok = std::fread(&n[sp], 8, 1, f) == 1 && n[sp] >= 0 && n[sp] <= ih.I.cap[sp];
    if (ok && ih.I.prec32) {
      ra[sp].resize((size_t)n[sp]);
      rb[sp].resize((size_t)n[sp]);
      ok = std::fread(ra[sp].data(), 16, (size_t)n[sp], f) == (size_t)n[sp];
      ok = ok && std::fread(rb[sp].data(), 16, (size_t)n[sp], f) == (size_t)n[sp];
      continue;
    }
    for (int k = 0; k < 5 && ok; ++k) {
      arr[sp][k].resize((size_t)n[sp]);
      ok = std::fread(arr[sp][k].data(), 8, (size_t)n[sp], f) == (size_t)n[sp];
    }
    if (ok) {
      ids[sp].resize((size_t)n[sp]);
      ok = std::fread(ids[sp].data(), 8, (size_t)n[sp], f) == (size_t)n[sp];
    }
  }
  std::fclose(f);
  if (!ok) return fail(h, PIC_ERR_IO, "checkpoint read failed or does not match the handle");
  for (int sp = 0; sp < 2; ++sp) {
    if (ih.I.prec32) {
      cudaError_t e0 = cudaSuccess;
      const int fl = current_buffer(h, instance, sp);
      if (n[sp] > 0) {
        e0 = cudaMemcpy(ih.I.buf32[sp][fl].a, ra[sp].data(), (size_t)n[sp] * 16, cudaMemcpyHostToDevice);
        if (e0 == cudaSuccess)
          e0 = cudaMemcpy(ih.I.buf32[sp][fl].b, rb[sp].data(), (size_t)n[sp] * 16, cudaMemcpyHostToDevice);
      }
      if (e0 != cudaSuccess) return cuda_fail(h, e0, "load copy");
      continue;
    }
    const int rc = set_particles(h, instance, sp, n[sp], arr[sp][0].data(), arr[sp][1].data(),
                                 arr[sp][2].data(), arr[sp][3].data(), arr[sp][4].data(),
                                 (const int64_t*)ids[sp].data(), 0, true);
    if (rc != PIC_OK) return rc;
  }
  Scalars cur;
  read_status(h, instance, &cur);
  s.n[0] = ih.I.prec32 ? n[0] : cur.n[0];
  s.n[1] = ih.I.prec32 ? n[1] : cur.n[1];
  s.flip[0] = cur.flip[0];   // the particles were placed in this handle's current buffers
  s.flip[1] = cur.flip[1];
  s.n_live[0] = s.n[0];      // checkpoints hold compact arrays
  s.n_live[1] = s.n[1];
  s.unsorted = 0;
  s.sort_force = h->tune_next > 0 ? 1 : 0;   // this handle's tuner, not the saved one's
  cudaError_t e = cudaMemcpy(ih.I.S, &s, sizeof(s), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(ih.I.qhist, qh.data(), qh.size() * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(ih.I.phi, phi.data(), nn * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(ih.I.phi_old, phi_old.data(), nn * 8, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(h, e, "load copy");
  // FP32 records were copied as saved: sort them once here so that this
  // handle's cell bins describe them (factor 1 keeps every particle)
  if (ih.I.prec32) {
    e = launch_thin(ih.I, 1, h->num_sms, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "load sort");
  }
  // the checkpoint's weight (it differs from the handle's after re-weighting)
  if (fc.weight != ih.I.weight) return set_weight(h, instance, fc.weight);
  return PIC_OK;
}

// ---------------------------------------------------------------------------
// learned warm start
// ---------------------------------------------------------------------------
static void* unet_alloc_cb(void* ctx, size_t bytes) { return dev_alloc((pic_handle*)ctx, bytes); }

static int need_unet(pic_handle* h) {
  if (!h) return PIC_ERR_INVALID;
  if (!h->unet) return fail(h, PIC_ERR_INVALID, "no network on this handle (pic_unet_create)");
  return PIC_OK;
}

int pic_unet_param_count(int64_t* n) {
  if (!n) return PIC_ERR_INVALID;
  *n = unet_param_count();
  return PIC_OK;
}

int pic_unet_create(pic_handle* h, uint64_t seed, int max_batch, int mode) {
  if (!h) return PIC_ERR_INVALID;
  if (h->unet) return fail(h, PIC_ERR_INVALID, "the handle already has a network");
  const pic_config& c = h->inst[0].cfg;
  for (const InstHost& ih : h->inst)
    if (ih.cfg.nr != c.nr || ih.cfg.nz != c.nz || ih.I.bc_g != h->inst[0].I.bc_g ||
        ih.I.bc_wall != h->inst[0].I.bc_wall)
      return fail(h, PIC_ERR_INVALID, "the instances must share the grid and its boundary kinds");
  if (c.nr % 8 || c.nz % 8 || max_batch < 1 || mode < 0 || mode > 1)
    return fail(h, PIC_ERR_INVALID, "nr and nz must be multiples of 8, max_batch >= 1, mode 0 or 1");
  const double vref = c.circuit_mode == 1 ? std::fabs(c.Vs) : std::fabs(c.Vc_fixed);
  UNet* u = unet_create(c.nr, c.nz, max_batch, (int)h->inst.size(), mode, seed,
                        vref > 0.0 ? vref : 1.0, unet_alloc_cb, h, h->stream);
  if (!u) return fail(h, PIC_ERR_OOM, "network allocation or set-up failed");
  unet_set_boundary(u, h->inst[0].I.bc_g, h->inst[0].I.bc_wall);
  h->unet = u;
  drop_graph(h);
  return PIC_OK;
}

int pic_unet_set_params(pic_handle* h, const float* params, int64_t n) {
  const int rc = need_unet(h);
  if (rc != PIC_OK) return rc;
  if (!params || n != unet_param_count()) return fail(h, PIC_ERR_INVALID, "parameter count");
  const cudaError_t e = unet_set_params(h->unet, params, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "unet_set_params");
  return PIC_OK;
}

int pic_unet_get_params(pic_handle* h, float* params, int64_t n) {
  const int rc = need_unet(h);
  if (rc != PIC_OK) return rc;
  if (!params || n != unet_param_count()) return fail(h, PIC_ERR_INVALID, "parameter count");
  const cudaError_t e = unet_get_params(h->unet, params, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "unet_get_params");
  return PIC_OK;
}

int pic_unet_loss_grad(pic_handle* h, int batch, const float* x, const float* y, float* out,
                       float* grad, double* loss) {
  const int rc = need_unet(h);
  if (rc != PIC_OK) return rc;
  if (!x || batch < 1 || batch > unet_bmax(h->unet)) return fail(h, PIC_ERR_INVALID, "batch or x");
  const cudaError_t e = unet_loss_grad(h->unet, batch, x, y, out, grad, loss, h->stream);
  if (e == cudaErrorTimeout) return fail(h, PIC_ERR_TIMEOUT, "tensor-core wait reached its limit");
  if (e != cudaSuccess) return cuda_fail(h, e, "unet_loss_grad");
  return PIC_OK;
}

int pic_unet_snapshots(pic_handle* h, int64_t capacity, int every) {
  const int rc = need_unet(h);
  if (rc != PIC_OK) return rc;
  if (capacity < 1 || every < 1) return fail(h, PIC_ERR_INVALID, "capacity, every >= 1");
  if (unet_recording(h->unet)) return fail(h, PIC_ERR_INVALID, "snapshot ring already set");
  const cudaError_t e = unet_snapshots(h->unet, capacity, every, unet_alloc_cb, h);
  if (e != cudaSuccess) return fail(h, PIC_ERR_OOM, "snapshot ring allocation failed");
  drop_graph(h);
  return PIC_OK;
}

int pic_unet_train(pic_handle* h, int iters, int batch, float lr, uint64_t seed,
                   double* loss_first, double* loss_last) {
  const int rc = need_unet(h);
  if (rc != PIC_OK) return rc;
  if (iters < 1 || batch < 1 || batch > unet_bmax(h->unet) || !(lr > 0.0f))
    return fail(h, PIC_ERR_INVALID, "iters, batch or lr");
  if (!unet_recording(h->unet)) return fail(h, PIC_ERR_INVALID, "no snapshots (pic_unet_snapshots)");
  const cudaError_t e = unet_train(h->unet, iters, batch, lr, seed, loss_first, loss_last, h->stream);
  if (e == cudaErrorInvalidValue) return fail(h, PIC_ERR_INVALID, "no snapshot recorded yet");
  if (e == cudaErrorTimeout) return fail(h, PIC_ERR_TIMEOUT, "tensor-core wait reached its limit");
  if (e != cudaSuccess) return cuda_fail(h, e, "unet_train");
  return PIC_OK;
}

int pic_unet_record(pic_handle* h, int on) {
  const int rc = need_unet(h);
  if (rc != PIC_OK) return rc;
  if (!unet_recording(h->unet)) return fail(h, PIC_ERR_INVALID, "no snapshot ring (pic_unet_snapshots)");
  unet_set_record(h->unet, on != 0);
  drop_graph(h);
  return PIC_OK;
}

int pic_unet_set_norms(pic_handle* h, double in_norm, double out_norm) {
  const int rc = need_unet(h);
  if (rc != PIC_OK) return rc;
  if (!(in_norm > 0.0) || !(out_norm > 0.0) || !std::isfinite(in_norm) || !std::isfinite(out_norm))
    return fail(h, PIC_ERR_INVALID, "scales must be positive and finite");
  const double v[2] = {in_norm, out_norm};
  static_assert(offsetof(UDev, out_norm) == offsetof(UDev, in_norm) + sizeof(double),
                "in_norm and out_norm adjacent");
  cudaError_t e = cudaMemcpyAsync((char*)unet_dev(h->unet) + offsetof(UDev, in_norm), v, sizeof(v),
                                  cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "unet_set_norms");
  return PIC_OK;
}

int pic_unet_warm_start(pic_handle* h, int on) {
  const int rc = need_unet(h);
  if (rc != PIC_OK) return rc;
  if (unet_warm(h->unet) != (on != 0)) {
    unet_set_warm(h->unet, on != 0);
    drop_graph(h);
  }
  return PIC_OK;
}

int pic_unet_stats_read(pic_handle* h, pic_unet_stats* out) {
  const int rc = need_unet(h);
  if (rc != PIC_OK) return rc;
  if (!out) return fail(h, PIC_ERR_INVALID, "null out");
  UDev d;
  cudaError_t e = cudaMemcpyAsync(&d, unet_dev(h->unet), sizeof(UDev), cudaMemcpyDeviceToHost,
                                  h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "unet stats");
  out->snapshots = d.snap_count;
  out->starts_previous = d.n_choice[0];
  out->starts_network = d.n_choice[1];
  out->starts_zero = d.n_choice[2];
  out->poisson_iters = d.iters_total;
  out->in_norm = d.in_norm;
  out->out_norm = d.out_norm;
  out->last_start = d.choice;
  out->pad = 0;
  return PIC_OK;
}

int pic_profile(pic_handle* h, int enable) {
  if (!h) return PIC_ERR_INVALID;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "profile");
  h->prof.on = enable != 0;
  if (enable) {
    h->prof.used = 0;
    h->prof.recs.clear();
  }
  return PIC_OK;
}

int pic_profile_read(pic_handle* h, pic_kernel_time* out, int max, int* n_out) {
  if (!h || !out || max < 0) return PIC_ERR_INVALID;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "profile read");
  double tot[G_COUNT] = {};
  long long cnt[G_COUNT] = {};
  for (const Profiler::Rec& r : h->prof.recs) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, r.b, r.e) == cudaSuccess) {
      tot[r.group] += ms;
      cnt[r.group] += 1;
    }
  }
  for (int g = 0; g < G_COUNT && g < max; ++g) {
    out[g].name = kGroupNames[g];
    out[g].launches = cnt[g];
    out[g].total_ms = tot[g];
  }
  if (n_out) *n_out = G_COUNT;
  return PIC_OK;
}

size_t pic_poisson_workspace_bytes(int nr, int nz) {
  if (nr < 2 || nz < 2) return 0;
  return poisson_work_bytes(nr, nz) + 256;
}

int pic_poisson_solve(int nr, int nz, double R, double L, double tol, int max_iter,
                      const double* Q_dev, double* phi_dev, void* work_dev, void* cuda_stream,
                      int* iters, double* resid) {
  return pic_poisson_solve_mixed(nr, nz, R, L, nr + 1, 0, tol, max_iter, Q_dev, phi_dev, work_dev,
                                 cuda_stream, iters, resid);
}

int pic_poisson_solve_mixed(int nr, int nz, double R, double L, int first_insulating_z0,
                            int wall_insulating, double tol, int max_iter, const double* Q_dev,
                            double* phi_dev, void* work_dev, void* cuda_stream, int* iters,
                            double* resid) {
  if (nr < 2 || nz < 2 || (nr & 1) || (nz & 1) || !(R > 0) || !(L > 0) || !(tol > 0) ||
      max_iter < 1 || !Q_dev || !phi_dev || !work_dev || ((uintptr_t)work_dev & 255) ||
      first_insulating_z0 < 0 || first_insulating_z0 > nr + 1 ||
      (wall_insulating != 0 && wall_insulating != 1))
    return PIC_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t wb = poisson_work_bytes(nr, nz);
  cudaError_t e = cudaMemsetAsync(work_dev, 0, wb + 256, st);
  if (e != cudaSuccess) return PIC_ERR_CUDA;
  PoissonWork* pw = poisson_work_init(work_dev, nr, nz, R, L, first_insulating_z0, wall_insulating,
                                      sms);
  char* tailp = (char*)work_dev + wb;
  int* status = (int*)tailp;
  int* it_dev = (int*)(tailp + 16);
  double* res_dev = (double*)(tailp + 32);
  e = launch_poisson(pw, Q_dev, phi_dev, tol, max_iter, status, it_dev, res_dev, st);
  poisson_work_free(pw);
  if (e != cudaSuccess) return PIC_ERR_CUDA;
  int hs[2] = {0, 0};
  double hr = 0.0;
  e = cudaMemcpyAsync(hs, status, 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs[1], it_dev, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hr, res_dev, 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return PIC_ERR_CUDA;
  if (iters) *iters = hs[1];
  if (resid) *resid = hr;
  return status_code(hs[0]);
}

}  // extern "C"
