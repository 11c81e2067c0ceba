// step32.cu -- FP32 particle path (precision mode 1) of the RZ PIC-MCC step.
//
// Same method and step order as the FP64 path (step.cu); what changes is the
// arithmetic of the particle loop:
//  * a particle is 32 bytes: {dr, dz, v_r, v_theta} + {v_z, cell key, id}; the
//    position is the cell index plus FP32 offsets in [0,1) of the cell, so its
//    resolution is 2^-24 of a cell everywhere in the domain;
//  * gather, Boris, move and MCC run in FP32; the move is done in local cell
//    units, and the new radius relative to the old cell uses the cancellation-
//    free form  r' - m = (x' - m) + y'^2 / (r' + x')  (x' > 0);
//  * the deposit accumulates FP32 weights in a shared-memory patch and flushes
//    it into FP64 node sums; the Poisson residuals, the circuit and the
//    energy / charge reductions stay FP64 (the shared kernels of step.cu and
//    poisson.cu).
#include "common.cuh"
#include "device_util.cuh"
#include "launch.h"

namespace pic {

constexpr int kPush32Threads = 256;
constexpr int kCollQ32 = 256;   // deferred collision candidates per chunk
constexpr int kHalo32 = 3;
// the deposit patch: (tile extent in r + 2 halo + 1) x (two tiles along z + 2
// halo + 1) nodes; the arrays hold the largest of the tile shapes
__device__ __forceinline__ int patch32_pr(const Inst& I) { return (1 << I.tsr) + 2 * kHalo32 + 1; }
__device__ __forceinline__ int patch32_pz(const Inst& I) { return (2 << I.tsz) + 2 * kHalo32 + 1; }
constexpr int patch32_nodes(int lr, int lz) {
  return ((1 << lr) + 2 * kHalo32 + 1) * ((2 << lz) + 2 * kHalo32 + 1);
}
constexpr int patch32_cells(int lr, int lz) { return ((1 << lr) + 2 * kHalo32) * ((2 << lz) + 2 * kHalo32); }
constexpr int cmax32(int a, int b) { return a > b ? a : b; }
constexpr int kPatch32Nodes = cmax32(patch32_nodes(3, 3), cmax32(patch32_nodes(4, 3), patch32_nodes(3, 4)));
constexpr int kPatch32Cells = cmax32(patch32_cells(3, 3), cmax32(patch32_cells(4, 3), patch32_cells(3, 4)));
constexpr float kHalfMeOverE = (float)(0.5 * kMe / kQe);   // E[eV] = kHalfMeOverE v^2
constexpr float kTwoEOverMe = (float)(2.0 * kQe / kMe);    // v^2 = kTwoEOverMe E[eV]

// The record's cell word holds (m << 16) | n; all ones marks a removed
// particle.  The sort key (8 x 8 tile-major) is derived from it.
constexpr unsigned kDead = 0xffffffffu;
__device__ __forceinline__ void cell_mn(unsigned c, int& m, int& n) {
  m = (int)(c >> 16);
  n = (int)(c & 0xffffu);
}
__device__ __forceinline__ unsigned pack_mn(int m, int n) { return ((unsigned)m << 16) | (unsigned)n; }

__device__ __forceinline__ float rweight_upper32(const Inst& I, float dr, int m) {
  if (I.rweight == 0) return dr;
  return dr * (2.0f * (float)m + dr) / (2.0f * (float)m + 1.0f);
}

__device__ __forceinline__ float u01f(unsigned long long x) {
  return (float)(x >> 40) * (1.0f / 16777216.0f);
}

__device__ __forceinline__ long long id_of(const uint4& b) {
  return (long long)(((unsigned long long)b.w << 32) | (unsigned long long)b.z);
}

// global deposit of one macroparticle (FP32 weights into FP64 node sums)
__device__ __forceinline__ void deposit_global32(const Inst& I, int sp, int m, int n, float wr,
                                                 float wz) {
  double* q = I.qacc64[sp];
  const int i = node_index(I, m, n), nz1 = I.nz + 1;
  atomicAdd(q + i, (double)((1.0f - wr) * (1.0f - wz)));
  atomicAdd(q + i + nz1, (double)(wr * (1.0f - wz)));
  atomicAdd(q + i + 1, (double)((1.0f - wr) * wz));
  atomicAdd(q + i + nz1 + 1, (double)(wr * wz));
}

__device__ void add_birth32(const Inst& I, int sp, unsigned long long pkey, int m, float dr, int n,
                            float dz, float vr, float vt, float vz) {
  Scalars* S = I.S;
  const unsigned long long b = atomicAdd((unsigned long long*)&S->nbirth[sp], 1ULL);
  if ((long long)b >= I.birth_cap) {
    atomicOr(&S->status, ST_CAPACITY);
    return;
  }
  const int key = cell_key(I, m, n);
  const BirthsDev& B = I.births[sp];
  B.a32[b] = make_float4(dr, dz, vr, vt);
  B.b32[b] = make_uint4(__float_as_uint(vz), pack_mn(m, n), 0u, 0u);
  B.pkey[b] = pkey;
  atomicAdd(&I.counts[sp][key], 1);
  deposit_global32(I, sp, m, n, rweight_upper32(I, dr, m), dz);
}

__device__ __forceinline__ void scatter_dir32(const float e[3], float cos_chi, float phi,
                                              float out[3]) {
  int a = 0;
  if (fabsf(e[1]) < fabsf(e[a])) a = 1;
  if (fabsf(e[2]) < fabsf(e[a])) a = 2;
  float ax[3] = {0.0f, 0.0f, 0.0f};
  ax[a] = 1.0f;
  float u[3] = {ax[1] * e[2] - ax[2] * e[1], ax[2] * e[0] - ax[0] * e[2],
                ax[0] * e[1] - ax[1] * e[0]};
  const float un = rsqrtf(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  u[0] *= un; u[1] *= un; u[2] *= un;
  const float w[3] = {e[1] * u[2] - e[2] * u[1], e[2] * u[0] - e[0] * u[2],
                      e[0] * u[1] - e[1] * u[0]};
  const float sin_chi = sqrtf(fmaxf(0.0f, 1.0f - cos_chi * cos_chi));
  float sp, cp;
  sincosf(phi, &sp, &cp);
  for (int j = 0; j < 3; ++j) out[j] = cos_chi * e[j] + sin_chi * (cp * u[j] + sp * w[j]);
}

// null-collision MCC of one electron in FP32 (candidate test exact on the
// 64-bit Philox word, as in FP64 mode)
// FP32 ionizing collision ((1c) or (1d), threshold Ith): see ionize64
__device__ float ionize32(const Inst& I, long long id, long long step, int m, float dr, int n,
                          float dz, float E, float Ith, const float e[3]) {
  unsigned long long w2[4], g[4];
  philox4x64((unsigned long long)id, (unsigned long long)step, 1ULL, 0ULL, I.seed, 0ULL, w2);
  const float Ex = E - Ith;
  const float Enew = u01f(w2[0]) * Ex;
  const float E2 = Ex - Enew;
  float d2[3];
  scatter_dir32(e, 1.0f - 2.0f * u01f(w2[1]), 2.0f * (float)kPi * u01f(w2[2]), d2);
  const float v2n = sqrtf(kTwoEOverMe * E2);
  const unsigned long long key = ((unsigned long long)id << 2) | 0ULL;
  add_birth32(I, 0, key, m, dr, n, dz, v2n * d2[0], v2n * d2[1], v2n * d2[2]);
  philox4x64((unsigned long long)id, (unsigned long long)step, 4ULL, 0ULL, I.seed, 0ULL, g);
  const float sig = (float)sqrt(kBoltz * I.T_gas / I.m_ion);
  const float rho1 = sqrtf(-2.0f * logf(1.0f - u01f(g[0]))), th1 = 2.0f * (float)kPi * u01f(g[1]);
  const float rho2 = sqrtf(-2.0f * logf(1.0f - u01f(g[2]))), th2 = 2.0f * (float)kPi * u01f(g[3]);
  float s1, c1, s2, c2;
  sincosf(th1, &s1, &c1);
  sincosf(th2, &s2, &c2);
  add_birth32(I, 1, key, m, dr, n, dz, sig * rho1 * c1, sig * rho1 * s1, sig * rho2 * c2);
  return Enew;
}

__device__ void mcc_electron32(const Inst& I, long long id, long long step, int m, float dr, int n,
                               float dz, float& vr, float& vt, float& vz) {
  // a candidate (mcc_candidate): process and angles from words 1..3 of stream 0
  unsigned long long w[4];
  philox4x64((unsigned long long)id, (unsigned long long)step, 0ULL, 0ULL, I.seed, 0ULL, w);
  const float v2 = vr * vr + vt * vt + vz * vz;
  const float vmag = sqrtf(v2);
  const float E = kHalfMeOverE * v2;
  const float exE = (float)I.exc_E, ioI = (float)I.ion_I, mdI = (float)I.meta_I;
  const float s_el = E > 0.0f ? (float)I.sigma_el : 0.0f;
  const float s_ex = E > exE ? (float)I.exc_C * logf(E / exE) / (E * exE) : 0.0f;
  const float s_io = E > ioI ? (float)I.ion_a * logf(E / ioI) / (E * ioI) : 0.0f;
  const float s_md = E > mdI ? (float)I.meta_a * logf(E / mdI) / (E * mdI) : 0.0f;
  const float ng = (float)I.n_gas;
  const float nu_el = ng * s_el * vmag, nu_ex = ng * s_ex * vmag, nu_io = ng * s_io * vmag;
  const float nu_md = (float)I.n_meta * s_md * vmag;
  const float R = u01f(w[1]) * (float)I.nu_max;
  const float inv = vmag > 0.0f ? 1.0f / vmag : 1.0f;
  const float e[3] = {vr * inv, vt * inv, vz * inv};
  const float cos_chi = 1.0f - 2.0f * u01f(w[2]);
  const float phi = 2.0f * (float)kPi * u01f(w[3]);
  float Enew;
  Scalars* S = I.S;
  if (R < nu_el) {
    Enew = E * (1.0f - 2.0f * (float)(kMe / I.m_ion) * (1.0f - cos_chi));
    atomicAdd(&S->cnt_elastic, 1ULL);
  } else if (R < nu_el + nu_ex) {
    Enew = E - exE;
    atomicAdd(&S->cnt_excite, 1ULL);
  } else if (R < nu_el + nu_ex + nu_io) {
    Enew = ionize32(I, id, step, m, dr, n, dz, E, ioI, e);
    atomicAdd(&S->cnt_ionize, 1ULL);
  } else if (R < nu_el + nu_ex + nu_io + nu_md) {
    Enew = ionize32(I, id, step, m, dr, n, dz, E, mdI, e);
    atomicAdd(&S->cnt_ionize_meta, 1ULL);
  } else {
    return;
  }
  float d[3];
  scatter_dir32(e, cos_chi, phi, d);
  const float vn = sqrtf(kTwoEOverMe * fmaxf(Enew, 0.0f));
  vr = vn * d[0];
  vt = vn * d[1];
  vz = vn * d[2];
}

// ---------------------------------------------------------------------------
// The collision of a queued candidate i, on its state after the move.
__device__ __noinline__ void collide_at32(const Inst& I, const Particles32& P, long long i,
                                          long long step) {
  const float4 a = P.a[i];
  const uint4 b = P.b[i];
  int m, n;
  cell_mn(b.y, m, n);
  float vr = a.z, vt = a.w, vz = __uint_as_float(b.x);
  mcc_electron32(I, id_of(b), step, m, a.x, n, a.y, vr, vt, vz);
  P.a[i] = make_float4(a.x, a.y, vr, vt);
  reinterpret_cast<unsigned int*>(P.b + i)[0] = __float_as_uint(vz);
}

// A particle that crossed z = 0 during the move (in cell units: from radius Xo at
// height zo to (X, y) at height zn), on a cold path kept out of the push loop:
// the cathode impact tally, the ion energy histogram of the cathode band and
// secondary emission (Section 3).
template <int SP>
__device__ __noinline__ void cathode_hit32(const Inst& I, float Xo, float X, float y, float zo,
                                           float zn, float vr, float vt, float vz, uint4 b,
                                           long long step) {
  Scalars* S = I.S;
  const float tc = zo / (zo - zn);
  const float xh = Xo + tc * (X - Xo), yh = tc * y;
  const float rhit = sqrtf(xh * xh + yh * yh);   // cells
  if (!(rhit <= (float)(I.Rc * I.inv_dr))) return;
  atomicAdd(SP == 1 ? &S->cnt_ion_cath : &S->cnt_e_cath, 1ULL);
  if (SP == 1 && I.ied_bins > 0) {
    const double rh = (double)rhit * I.dr;
    if (rh >= I.band_lo && rh <= I.band_hi) {
      const double E =
          0.5 * I.mass[1] * ((double)vr * vr + (double)vt * vt + (double)vz * vz) / kQe;
      const double fb = floor(E / I.ied_de);
      atomicAdd(&I.reg.ied[fb < (double)I.ied_bins ? (int)fb : I.ied_bins], 1ULL);
    }
  }
  if (I.gamma[SP] > 0.0) {
    const long long id = id_of(b);
    double u[4];
    draws(I, SP, id, step, 2, u);
    if (u[0] < I.gamma[SP]) {
      atomicAdd(&S->cnt_sey, 1ULL);
      int mh = (int)floorf(rhit);
      float drh = rhit - (float)mh;
      if (mh > I.nr - 1) { mh = I.nr - 1; drh = 1.0f; }
      add_birth32(I, 0, ((unsigned long long)id << 2) | (SP == 1 ? 1ULL : 2ULL), mh, drh, 0,
                  0.0f, 0.0f, 0.0f, 0.0f);
    }
  }
}

// The FP32 push: gather + Boris + move + walls + SEY + MCC + deposit, state
// rewritten in place with the new cell key (read by the scatter).
// ---------------------------------------------------------------------------
// Push the chunk of `ppt * blockDim.x` particles starting at c0 (whole CTA).
// Warp w takes the contiguous run [c0 + 32 ppt w, c0 + 32 ppt (w + 1)), 32
// consecutive particles per iteration, so that a lane meets the same new cell
// over many iterations in a cell-sorted array: it sums its deposit weights
// and its cell count in registers and adds them to the CTA's shared patches
// (node charge `patch`, cell counts `cpatch`; global memory outside them)
// only when its cell changes.  The patches are flushed and zeroed on return.
// `anchor` holds the patch origin and the candidate count, `cq` the chunk's
// collision candidates, run after the chunk as in push_chunk64 (step.cu).
template <int SP>
__device__ __forceinline__ void deposit_run32(const Inst& I, int key, int m, int n, float a00,
                                              float a10, float a01, float a11, int cnt, int pm0,
                                              int pn0, int pr, int pz, float* patch, int* cpatch) {
  const int lm = m - pm0, ln = n - pn0;
  if (lm >= 0 && lm + 1 < pr && ln >= 0 && ln + 1 < pz) {
    float* p = patch + lm * pz + ln;
    atomicAdd(p, a00);
    atomicAdd(p + pz, a10);
    atomicAdd(p + 1, a01);
    atomicAdd(p + pz + 1, a11);
    atomicAdd(cpatch + lm * (pz - 1) + ln, cnt);
  } else {
    double* q = I.qacc64[SP];
    const int gi = node_index(I, m, n), nz1 = I.nz + 1;
    atomicAdd(q + gi, (double)a00);
    atomicAdd(q + gi + nz1, (double)a10);
    atomicAdd(q + gi + 1, (double)a01);
    atomicAdd(q + gi + nz1 + 1, (double)a11);
    atomicAdd(&I.counts[SP][key], cnt);
  }
}

// The flush of the lanes whose cell changed this iteration (flag fl), by the
// whole warp: the flushing lanes hold consecutive particles, so lanes of one
// cell form runs of adjacent lanes; a segmented suffix sum by shuffles (runs
// of adjacent flushing lanes with the same key) leaves each run's sums in its
// first lane, which alone adds them to the patch (one set of shared atomics
// per cell instead of one per lane: lanes of one cell would conflict on the
// same words).  All 32 lanes must take part.
// The open sums of a lane are sr = sum w_r, sz = sum w_z, srz = sum w_r w_z
// and the count c: the four tent weights of the cell's nodes are
// c - sr - sz + srz, sr - srz, sz - srz and srz.
template <int SP>
__device__ __forceinline__ void warp_flush32(const Inst& I, bool fl, int key, int m, int n,
                                             float sr, float sz, float srz, int cnt,
                                             int pm0, int pn0, int pr, int pz, float* patch,
                                             int* cpatch, int lane) {
  const unsigned full = 0xffffffffu;
  const int k = fl ? key : -1;
  const int kprev = __shfl_up_sync(full, k, 1);
  const bool head = fl && (lane == 0 || kprev != k);
  // a run ends below the next lane that starts a run or does not flush
  const unsigned starts = __ballot_sync(full, head || !fl);
  const unsigned above = lane == 31 ? 0u : (starts & (full << (lane + 1)));
  const int end = above ? __ffs(above) - 1 : 32;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const float br = __shfl_down_sync(full, sr, off), bz = __shfl_down_sync(full, sz, off);
    const float brz = __shfl_down_sync(full, srz, off);
    const int bc = __shfl_down_sync(full, cnt, off);
    if (lane + off < end) {
      sr += br;
      sz += bz;
      srz += brz;
      cnt += bc;
    }
  }
  if (head)
    deposit_run32<SP>(I, key, m, n, ((float)cnt - sr) - (sz - srz), sr - srz, sz - srz, srz, cnt,
                      pm0, pn0, pr, pz, patch, cpatch);
}

template <int SP, int GATHER, bool PLAIN>
__device__ __forceinline__ double push_chunk32(const Inst& I, int c0, int ppt, float* patch,
                                               int* cpatch, int* anchor, int* cq) {
  Scalars* S = I.S;
  const int n = (int)S->n[SP];   // counts stay below 2^31 (capacities are checked)
  const long long step = S->step;
  const bool diag = S->diag_on != 0;
  const Particles32 P = I.buf32[SP][S->flip[SP]];
  const float h = I.hq32[SP], kr = I.kr32, kz = I.kz32;
  const int lane = threadIdx.x & 31;
  const int run0 = c0 + (threadIdx.x >> 5) * 32 * ppt;
  double Kloc = 0.0;
  {
    if (threadIdx.x == 0) {
      int m, nn;
      cell_mn(P.b[c0].y, m, nn);
      anchor[0] = (m & ~((1 << I.tsr) - 1)) - kHalo32;
      anchor[1] = (nn & ~((1 << I.tsz) - 1)) - kHalo32;
      anchor[2] = 0;
    }
    __syncthreads();
    const int pm0 = anchor[0], pn0 = anchor[1];
    const int pr = patch32_pr(I), pz = patch32_pz(I);
    // the next particle's two records are loaded while this one is pushed
    int i = run0 + lane;
    float4 a_nx = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    uint4 b_nx = make_uint4(0u, 0u, 0u, 0u);
    if (i < n) {
      a_nx = P.a[i];
      b_nx = P.b[i];
    }
    // this lane's open deposit: cell, its weight sums and particle count
    int acc_key = -1, acc_m = 0, acc_n = 0, acc_cnt = 0;
    float sr = 0.0f, sz = 0.0f, srz = 0.0f;
    unsigned over = 0u;   // candidates that found the queue full, bit j (ppt <= 32)
    float k2 = 0.0f;
#pragma unroll 1
    for (int j = 0; j < ppt; ++j, i += 32) {
      const float4 a = a_nx;
      const uint4 b = b_nx;
      bool add = false, fl = false;   // this particle's deposit; flush of the open sums
      int nkey = 0, nm = 0, nn1 = 0;
      float wr1 = 0.0f, wz1 = 0.0f;
      {
        const int i2 = i + 32;
        if (j + 1 < ppt && i2 < n) {
          a_nx = P.a[i2];
          b_nx = P.b[i2];
        }
      }
      if (i < n && b.y != kDead) {   // dead slots stay until the next full sort
        int m, nn;
        cell_mn(b.y, m, nn);
        const float dr = a.x, dz = a.y;
        float vr = a.z, vt = a.w, vz = __uint_as_float(b.x);
        const float v2old = vr * vr + vt * vt + vz * vz;
        float rho = dr, zeta = dz, X = (float)m + dr, y = 0.0f;
        if (PLAIN || I.push_on) {
          const int ck = cell_key(I, m, nn);
          const float wr = PLAIN ? dr : rweight_upper32(I, dr, m);
          float Er, Ez;
          if (GATHER == 0) {
            const float4 t = I.etab32[ck];
            Er = t.x + t.y * dz;
            if (!PLAIN && I.rweight == 1) Er *= ((float)m + dr) * (float)I.dr;
            Ez = t.z + t.w * wr;
          } else {
            const float4 ta = I.etab32[2 * ck];
            const float4 tb = I.etab32[2 * ck + 1];
            Er = ta.x + wr * (ta.y + dz * ta.w) + dz * ta.z;
            Ez = tb.x + wr * (tb.y + dz * tb.w) + dz * tb.z;
          }
          const float4 br = I.btab32[2 * ck];
          const float4 bz = I.btab32[2 * ck + 1];
          const float Br = br.x + dr * (br.y + dz * br.w) + dz * br.z;
          const float Bz = bz.x + dr * (bz.y + dz * bz.w) + dz * bz.z;
          const float ax = vr + h * Er, ay = vt, az = vz + h * Ez;
          const float tx = h * Br, tz = h * Bz;
          // FP32 mode: the fast division / reciprocal square root intrinsics
          // (error of a few ulp, far inside the mode's 1e-5 bar)
          const float f2 = __fdividef(2.0f, 1.0f + tx * tx + tz * tz);
          const float sx = f2 * tx, sz = f2 * tz;
          const float px = ax + ay * tz;
          const float py = ay + (az * tx - ax * tz);
          const float pz = az - ay * tx;
          const float vx = ax + py * sz + h * Er;
          const float vy = ay + (pz * sx - px * sz);
          const float vzn = az - py * sx + h * Ez;
          // move in cell units relative to the old cell
          const float xl = dr + vx * kr;
          y = vy * kr;
          X = (float)m + xl;
          const float R2 = X * X + y * y;
          const float inv = R2 > 0.0f ? rsqrtf(R2) : 0.0f;
          const float Rn = R2 * inv;
          rho = X > 0.0f ? xl + __fdividef(y * y, Rn + X) : Rn - (float)m;
          if (R2 > 0.0f) {
            vr = (X * vx + y * vy) * inv;
            vt = (X * vy - y * vx) * inv;
          } else {
            vr = vx;
            vt = vy;
          }
          vz = vzn;
          zeta = dz + vzn * kz;
        }
        // kinetic energy: |v|^2 before and after summed in FP32 over this
        // thread's particles of the chunk (at most 32), the FP64 sum is the
        // block's and the step's
        if (diag) k2 += v2old + (vr * vr + vt * vt + vz * vz);
        bool alive = true;
        int m1, n1;
        float dr1, dz1;
        if (!PLAIN && I.walls_reflect) {
          float rc = (float)m + rho, zc = (float)nn + zeta;
          if (zc < 0.0f) { zc = -zc; vz = -vz; }
          if (zc >= (float)I.nz) { zc = 2.0f * I.nz - zc; vz = -vz; if (zc >= (float)I.nz) zc = nextafterf((float)I.nz, 0.0f); }
          if (rc >= (float)I.nr) { rc = 2.0f * I.nr - rc; vr = -vr; if (rc >= (float)I.nr) rc = nextafterf((float)I.nr, 0.0f); }
          m1 = (int)floorf(rc);
          n1 = (int)floorf(zc);
          dr1 = rc - (float)m1;
          dz1 = zc - (float)n1;
        } else {
          const float fm = floorf(rho), fn = floorf(zeta);
          m1 = m + (int)fm;
          n1 = nn + (int)fn;
          dr1 = rho - fm;
          dz1 = zeta - fn;
        }
        if (dr1 >= 1.0f) { dr1 = 0.0f; ++m1; }
        if (dz1 >= 1.0f) { dz1 = 0.0f; ++n1; }
        if (m1 < 0) { m1 = 0; dr1 = 0.0f; }
        if (!(isfinite(rho) && isfinite(zeta))) {
          atomicOr(&S->status, ST_NAN);
          alive = false;
        } else if ((PLAIN || !I.walls_reflect) && (n1 < 0 || n1 >= I.nz || m1 >= I.nr)) {
          alive = false;
          if (n1 < 0)
            cathode_hit32<SP>(I, (float)m + dr, X, y, (float)nn + dz, (float)nn + zeta, vr, vt,
                              vz, b, step);
        }
        if (alive) {
          if (SP == 0 && I.mcc_on && mcc_candidate(I, id_of(b), step)) {
            const int slot = atomicAdd(&anchor[2], 1);
            if (slot < kCollQ32) cq[slot] = (int)(i - c0);
            else over |= 1u << j;   // queue full: this thread runs it after the queue
          }
          const int newkey = cell_key(I, m1, n1);
          P.a[i] = make_float4(dr1, dz1, vr, vt);
          P.b[i] = make_uint4(__float_as_uint(vz), pack_mn(m1, n1), b.z, b.w);
          // deposit of x^{n+1} (Section 2: tent functions), summed per cell;
          // a lane whose cell changes flushes its open sums below (whole warp)
          add = true;
          nkey = newkey;
          nm = m1;
          nn1 = n1;
          wr1 = PLAIN ? dr1 : rweight_upper32(I, dr1, m1);
          wz1 = dz1;
          fl = newkey != acc_key && acc_key >= 0;
        } else {
          reinterpret_cast<unsigned int*>(P.b + i)[1] = kDead;
        }
      }
      if (__any_sync(0xffffffffu, fl))
        warp_flush32<SP>(I, fl, acc_key, acc_m, acc_n, sr, sz, srz, acc_cnt, pm0, pn0, pr, pz,
                         patch, cpatch, lane);
      if (add) {
        if (nkey != acc_key) {
          acc_key = nkey;
          acc_m = nm;
          acc_n = nn1;
          acc_cnt = 0;
          sr = sz = srz = 0.0f;
        }
        sr += wr1;
        sz += wz1;
        srz = fmaf(wr1, wz1, srz);
        ++acc_cnt;
      }
    }
    warp_flush32<SP>(I, acc_key >= 0, acc_key, acc_m, acc_n, sr, sz, srz, acc_cnt, pm0, pn0, pr,
                     pz, patch, cpatch, lane);
    if (diag) Kloc = 0.25 * I.mass[SP] * I.weight * (double)k2;
    __syncthreads();
    if (SP == 0) {
      // the queued collisions (Section 3), on the state written above
      const int nq = min(anchor[2], kCollQ32);
      for (int k = threadIdx.x; k < nq; k += blockDim.x) collide_at32(I, P, c0 + cq[k], step);
      while (over) {
        const int j = __ffs(over) - 1;
        over &= over - 1;
        collide_at32(I, P, run0 + j * 32 + lane, step);
      }
    }
    for (int k = threadIdx.x; k < pr * pz; k += blockDim.x) {
      const float v = patch[k];
      if (v != 0.0f) {
        const int gm = pm0 + k / pz, gn = pn0 + k % pz;
        atomicAdd(I.qacc64[SP] + node_index(I, gm, gn), (double)v);
        patch[k] = 0.0f;
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

// one wave of the persistent push: resident blocks per SM x SMs (cached per kernel)
int resident_blocks(const void* fn, int threads, int num_sms);   // step.cu

// The FP32 push of both species of every instance over the work queue (see
// k_push_all in step.cu).  PLAIN: every instance runs the model's own switches
// (push on, tent weights in r, absorbing walls; see k_push32_one).
template <int GATHER, bool PLAIN>
__global__ void __launch_bounds__(kPush32Threads, 4) k_push32_all(const Inst* insts, WorkQueue* q,
                                                                   int ppt) {
  __shared__ float patch[kPatch32Nodes];
  __shared__ int cpatch[kPatch32Cells];
  __shared__ int anchor[3];
  __shared__ int cq[kCollQ32];
  __shared__ Inst sI;
  __shared__ int s_inst, s_sp, s_skip;
  __shared__ long long s_c0;
  for (int k = threadIdx.x; k < kPatch32Nodes; k += blockDim.x) patch[k] = 0.0f;
  for (int k = threadIdx.x; k < kPatch32Cells; k += blockDim.x) cpatch[k] = 0;
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
      s_skip = inst >= 0 ? (*(volatile int*)&insts[inst].S->status & ST_FATAL) : 0;
    }
    __syncthreads();
    const int inst = s_inst;
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
      if (s_sp == 0) K0 += push_chunk32<0, GATHER, PLAIN>(sI, (int)s_c0, ppt, patch, cpatch, anchor, cq);
      else K1 += push_chunk32<1, GATHER, PLAIN>(sI, (int)s_c0, ppt, patch, cpatch, anchor, cq);
    }
    __syncthreads();
  }
}

// The FP32 push of a single-instance handle: the same chunks over the same
// queue, with the instance's parameters a kernel argument, so that the push
// reads them as constant-bank operands instead of loads from shared memory
// (fewer instructions and registers in the particle loop).
// PLAIN: the model's own switches (push on, tent weights in r, absorbing
// walls) fixed at compile time; the other settings take the general variant.
template <int GATHER, bool PLAIN>
__global__ void __launch_bounds__(kPush32Threads, 4) k_push32_one(const Inst I, WorkQueue* q,
                                                                   int ppt) {
  __shared__ float patch[kPatch32Nodes];
  __shared__ int cpatch[kPatch32Cells];
  __shared__ int anchor[3];
  __shared__ int cq[kCollQ32];
  __shared__ int s_sp, s_done, s_skip;
  __shared__ long long s_c0;
  for (int k = threadIdx.x; k < kPatch32Nodes; k += blockDim.x) patch[k] = 0.0f;
  for (int k = threadIdx.x; k < kPatch32Cells; k += blockDim.x) cpatch[k] = 0;
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
      // one reading of the status word for the whole CTA (see k_push_all)
      s_skip = *(volatile int*)&I.S->status & ST_FATAL;
    }
    __syncthreads();
    if (s_done) break;
    if (!s_skip) {
      if (s_sp == 0) K0 += push_chunk32<0, GATHER, PLAIN>(I, (int)s_c0, ppt, patch, cpatch, anchor, cq);
      else K1 += push_chunk32<1, GATHER, PLAIN>(I, (int)s_c0, ppt, patch, cpatch, anchor, cq);
    }
    __syncthreads();
  }
  if (I.S->diag_on) {
    block_add(K0, &I.S->K[0]);
    block_add(K1, &I.S->K[1]);
  }
}

template <int GATHER, bool PLAIN>
static void push32_one(const Inst& I, WorkQueue* q, int ppt, int num_sms, cudaStream_t st) {
  k_push32_one<GATHER, PLAIN><<<resident_blocks((const void*)k_push32_one<GATHER, PLAIN>,
                                                kPush32Threads, num_sms),
                                kPush32Threads, 0, st>>>(I, q, ppt);
}

cudaError_t launch_push32_one(const Inst& I, WorkQueue* q, int ppt, int num_sms,
                              cudaStream_t st) {
  const bool plain = I.push_on && I.rweight == 0 && !I.walls_reflect;
  if (I.gather == 0) {
    if (plain) push32_one<0, true>(I, q, ppt, num_sms, st);
    else push32_one<0, false>(I, q, ppt, num_sms, st);
  } else {
    if (plain) push32_one<1, true>(I, q, ppt, num_sms, st);
    else push32_one<1, false>(I, q, ppt, num_sms, st);
  }
  return cudaGetLastError();
}

__device__ __forceinline__ void k_scatter32_body(const Inst& I, int sp0, int per_step) {
  Scalars* S = I.S;
  if (S->status & ST_FATAL) return;
  const int sp = sp0 + blockIdx.y;
  const long long n_old = S->n[sp];
  const long long nb = S->nbirth[sp] < I.birth_cap ? S->nbirth[sp] : I.birth_cap;
  const long long total = n_old + nb;
  const int fl = S->flip[sp];
  const Particles32 src = I.buf32[sp][fl], dst = I.buf32[sp][fl ^ 1];
  const BirthsDev B = I.births[sp];
  if (per_step && !sort_this_step(I, S)) return;   // k_append32 does this step
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarp = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long base = warp * 32; base < total; base += nwarp * 32) {
    const long long i = base + lane;
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
    uint4 b = make_uint4(0u, kDead, 0u, 0u);
    if (i < n_old) {
      a = src.a[i];
      b = src.b[i];
    } else if (i < total) {
      a = B.a32[i - n_old];
      b = B.b32[i - n_old];
    }
    int key = -1;
    if (b.y != kDead) {
      int m, nn;
      cell_mn(b.y, m, nn);
      key = cell_key(I, m, nn);
    }
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int leader = __ffs(peers) - 1;
    int pos0 = 0;
    if (lane == leader && key >= 0) pos0 = atomicAdd(&I.cursor[sp][key], __popc(peers));
    pos0 = __shfl_sync(0xffffffffu, pos0, leader);
    if (key >= 0) {
      const int pos = pos0 + __popc(peers & ((1u << lane) - 1u));
      dst.a[pos] = a;
      dst.b[pos] = b;
    }
  }
}
__global__ void k_scatter32(Inst I, int sp0, int per_step) { k_scatter32_body(I, sp0, per_step); }
__global__ void k_scatter32_b(const Inst* insts, int sp0, int per_step) {
  __shared__ Inst sI;
  stage_inst(insts + blockIdx.z, &sI);
  k_scatter32_body(sI, sp0, per_step);
}

// FP64 SoA (r, z, v, id) -> FP32 records at [offset, offset + count) of cur32,
// keys counted; out-of-domain input removed and flagged
__global__ void k_pack32(Inst I, int sp, long long offset, long long count, const double* r,
                         const double* z, const double* vr, const double* vt, const double* vz,
                         const long long* id) {
  Scalars* S = I.S;
  const Particles32 P = I.buf32[sp][S->flip[sp]];
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarp = ((long long)gridDim.x * blockDim.x) >> 5;
  long long idmax = -1;
  bool bad = false;
  for (long long base = warp * 32; base < count; base += nwarp * 32) {
    const long long k = base + lane;
    int key = -1;
    if (k < count) {
      const double rr = r[k], zz = z[k];
      const long long pid = id[k];
      float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
      uint4 b = make_uint4(0u, kDead, 0u, 0u);
      if (rr >= 0.0 && rr < I.R && zz >= 0.0 && zz < I.L && finite64(vr[k]) && finite64(vt[k]) &&
          finite64(vz[k]) && pid >= 0) {
        int m, nn;
        double fr, fz;
        locate(rr, I.inv_dr, I.nr, m, fr);
        locate(zz, I.inv_dz, I.nz, nn, fz);
        float dr = (float)fr, dz = (float)fz;
        if (dr >= 1.0f) dr = nextafterf(1.0f, 0.0f);
        if (dz >= 1.0f) dz = nextafterf(1.0f, 0.0f);
        key = cell_key(I, m, nn);
        a = make_float4(dr, dz, (float)vr[k], (float)vt[k]);
        b = make_uint4(__float_as_uint((float)vz[k]), pack_mn(m, nn),
                       (unsigned)((unsigned long long)pid & 0xffffffffULL),
                       (unsigned)((unsigned long long)pid >> 32));
        idmax = pid > idmax ? pid : idmax;
      } else {
        bad = true;
      }
      P.a[offset + k] = a;
      P.b[offset + k] = b;
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

// Re-weighting in FP32 mode: the same per-id draw as the FP64 path; dropped
// records are marked dead in place, kept ones counted for the sort.
__global__ void k_thin32(Inst I, int sp, int factor) {
  Scalars* S = I.S;
  if (S->status & ST_FATAL) return;
  const long long n = S->n[sp], s = S->step;
  const Particles32 P = I.buf32[sp][S->flip[sp]];
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarp = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long base = warp * 32; base < n; base += nwarp * 32) {
    const long long i = base + lane;
    int key = -1;
    if (i < n) {
      uint4 b = P.b[i];
      bool keep = b.y != kDead;   // dead slots go; factor 1 keeps every live particle
      if (keep && factor > 1) {
        unsigned long long w[4];
        philox4x64((unsigned long long)id_of(b), (unsigned long long)s, 5ULL, 0ULL, I.seed,
                   (unsigned long long)sp, w);
        keep = w[0] % (unsigned long long)factor == 0ULL;
      }
      if (keep) {
        int m, nn;
        cell_mn(b.y, m, nn);
        key = cell_key(I, m, nn);
      } else {
        b.y = kDead;
        P.b[i] = b;
      }
    }
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    if (key >= 0 && lane == __ffs(peers) - 1) atomicAdd(&I.counts[sp][key], __popc(peers));
  }
}

// FP32 records [offset, offset + count) of cur32 -> FP64 SoA
__global__ void k_unpack32(Inst I, int sp, long long offset, long long count, double* r, double* z,
                           double* vr, double* vt, double* vz, long long* id) {
  const Particles32 P = I.buf32[sp][I.S->flip[sp]];
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < count;
       k += (long long)gridDim.x * blockDim.x) {
    const float4 a = P.a[offset + k];
    const uint4 b = P.b[offset + k];
    int m, nn;
    cell_mn(b.y, m, nn);
    if (r) r[k] = ((double)m + (double)a.x) * I.dr;
    if (z) z[k] = ((double)nn + (double)a.y) * I.dz;
    if (vr) vr[k] = (double)a.z;
    if (vt) vt[k] = (double)a.w;
    if (vz) vz[k] = (double)__uint_as_float(b.x);
    if (id) id[k] = id_of(b);
  }
}

__global__ void k_deposit_all32(Inst I, int sp) {
  const long long n = I.S->n[sp];
  const Particles32 P = I.buf32[sp][I.S->flip[sp]];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float4 a = P.a[i];
    int m, nn;
    cell_mn(P.b[i].y, m, nn);
    deposit_global32(I, sp, m, nn, rweight_upper32(I, a.x, m), a.y);
  }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
static int grid32(long long work, int threads, int num_sms, int per_sm) {
  long long g = (work + threads - 1) / threads;
  const long long cap = (long long)num_sms * per_sm;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

cudaError_t launch_pack32(const Inst& I, int sp, long long offset, long long count, const double* r,
                          const double* z, const double* vr, const double* vt, const double* vz,
                          const long long* id, int num_sms, cudaStream_t st) {
  k_pack32<<<grid32(count, 256, num_sms, 8), 256, 0, st>>>(I, sp, offset, count, r, z, vr, vt, vz,
                                                             id);
  return cudaGetLastError();
}

cudaError_t launch_unpack32(const Inst& I, int sp, long long offset, long long count, double* r,
                            double* z, double* vr, double* vt, double* vz, long long* id,
                            int num_sms, cudaStream_t st) {
  k_unpack32<<<grid32(count, 256, num_sms, 8), 256, 0, st>>>(I, sp, offset, count, r, z, vr, vt, vz,
                                                               id);
  return cudaGetLastError();
}

cudaError_t launch_sort_species32(const Inst& I, int sp, int num_sms, cudaStream_t st) {
  launch_scan(I, sp, 1, st);
  k_scatter32<<<dim3(grid32(I.cap[sp], 256, num_sms, 8), 1), 256, 0, st>>>(I, sp, 0);
  return launch_commit_n(I, sp, st);
}

cudaError_t launch_thin32(const Inst& I, int sp, int factor, int num_sms, cudaStream_t st) {
  k_thin32<<<grid32(I.cap[sp], 256, num_sms, 8), 256, 0, st>>>(I, sp, factor);
  return cudaGetLastError();
}

cudaError_t launch_deposit_all32(const Inst& I, int num_sms, cudaStream_t st) {
  for (int sp = 0; sp < 2; ++sp)
    k_deposit_all32<<<grid32(I.cap[sp], 256, num_sms, 8), 256, 0, st>>>(I, sp);
  return cudaGetLastError();
}


template <int GATHER, bool PLAIN>
static void push32_all(const Inst* d_insts, WorkQueue* q, int ppt, int num_sms, cudaStream_t st) {
  k_push32_all<GATHER, PLAIN><<<resident_blocks((const void*)k_push32_all<GATHER, PLAIN>,
                                                kPush32Threads, num_sms),
                                kPush32Threads, 0, st>>>(d_insts, q, ppt);
}

cudaError_t launch_push32_all(const Inst* d_insts, WorkQueue* q, int gather, bool plain, int ppt,
                              int num_sms, cudaStream_t st) {
  if (gather == 0) {
    if (plain) push32_all<0, true>(d_insts, q, ppt, num_sms, st);
    else push32_all<0, false>(d_insts, q, ppt, num_sms, st);
  } else {
    if (plain) push32_all<1, true>(d_insts, q, ppt, num_sms, st);
    else push32_all<1, false>(d_insts, q, ppt, num_sms, st);
  }
  return cudaGetLastError();
}

// births appended to the current records on a step without the full sort
__device__ __forceinline__ void k_append32_body(const Inst& I) {
  const Scalars* S = I.S;
  if ((S->status & ST_FATAL) || sort_this_step(I, S)) return;
  const int sp = blockIdx.y;
  const long long n_old = S->n[sp];
  const long long nb = S->nbirth[sp] < I.birth_cap ? S->nbirth[sp] : I.birth_cap;
  const Particles32 P = I.buf32[sp][S->flip[sp]];
  const BirthsDev B = I.births[sp];
  for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < nb;
       b += (long long)gridDim.x * blockDim.x) {
    P.a[n_old + b] = B.a32[b];
    P.b[n_old + b] = B.b32[b];
  }
}
__global__ void k_append32(Inst I) { k_append32_body(I); }
__global__ void k_append32_b(const Inst* insts) {
  __shared__ Inst sI;
  stage_inst(insts + blockIdx.z, &sI);
  k_append32_body(sI);
}

cudaError_t launch_append32(const Inst& I, int num_sms, cudaStream_t st) {
  k_append32<<<dim3(num_sms, 2), 256, 0, st>>>(I);
  return cudaGetLastError();
}

cudaError_t launch_scatter32_batch(const Inst* d_insts, int n_inst, int blocks, cudaStream_t st) {
  k_scatter32_b<<<dim3(blocks, 2, n_inst), 256, 0, st>>>(d_insts, 0, 1);
  return cudaGetLastError();
}

cudaError_t launch_append32_batch(const Inst* d_insts, int n_inst, int blocks, cudaStream_t st) {
  k_append32_b<<<dim3(blocks, 2, n_inst), 256, 0, st>>>(d_insts);
  return cudaGetLastError();
}

cudaError_t launch_scatter32(const Inst& I, int num_sms, cudaStream_t st) {
  k_scatter32<<<dim3(num_sms * 8, 2), 256, 0, st>>>(I, 0, 1);
  return cudaGetLastError();
}

}  // namespace pic
