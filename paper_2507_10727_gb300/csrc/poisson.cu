// poisson.cu -- RZ Poisson solve (arXiv:2507.10727, Section 3: anode and
// walls grounded, cathode at the circuit voltage, Gauss's law on the axis).
//
// Discretisation (the paper gives none; finite-volume reading): for a free
// node (m, n), m = 0..nr-1, n = 1..nz-1, the equation times the node's
// control volume reads  sum_j a_kj (phi_k - phi_j) = Q_k  with
//   a_r(m) = 2 pi eps0 (m + 1/2) dz           between (m,n) and (m+1,n)
//   a_z(m) = eps0 area(m) / dz                between (m,n) and (m,n+1)
//   area(m) = 2 pi m dr^2 (m >= 1), pi dr^2 / 4 (axis: Gauss on the disk dr/2)
// which is symmetric positive definite on the free nodes.
//
// Solver: one cooperative persistent kernel.  Flexible preconditioned
// conjugate gradients with iterates, residuals and dot products in FP64
// (deterministic block-ordered reductions); the preconditioner is one
// geometric-multigrid V-cycle in FP32 on the same operator rediscretised at
// 2x, 4x ... coarser spacing (red-black Gauss-Seidel, residual restriction by
// the transpose of bilinear prolongation).  Because the outer iteration and
// its stopping test (relative residual ||b - A phi||_2 <= tol ||b||_2) are
// FP64, the converged phi does not depend on the preconditioner's precision.
// Coarse levels (<= kTailNodes nodes) run inside one CTA; finer levels use
// the whole grid with a time-bounded grid barrier.
#include <cstdio>
#include <cstring>

#include "common.cuh"
#include "launch.h"

namespace pic {

constexpr int kMaxLev = 16;
constexpr int kPoisThreads = 512;
constexpr int kTailNodes = 4225;        // 65 x 65
constexpr double kBarrierLimitNs = 2.0e9;

struct PoissonWork {
  int nr, nz, nlev, tail;
  double dr, dz;
  int nblocks;
  int lnr[kMaxLev], lnz[kMaxLev];
  float* u[kMaxLev];
  float* f[kMaxLev];
  double *r, *p, *q, *z;
  double* partial;
  unsigned int* bar;
};

struct PoissonArgs {
  PoissonWork W;
  const double* Q;
  double* phi;
  double tol;
  int max_iter;
  int* status;
  int* iters;
  double* resid;
};

size_t poisson_work_bytes(int nr, int nz) {
  size_t bytes = 0;
  auto add = [&](size_t b) { bytes += (b + 255) & ~(size_t)255; };
  const size_t nn = (size_t)(nr + 1) * (nz + 1);
  for (int k = 0; k < 4; ++k) add(nn * sizeof(double));
  int lr = nr, lz = nz;
  for (int l = 0; l < kMaxLev; ++l) {
    const size_t ln = (size_t)(lr + 1) * (lz + 1);
    add(ln * sizeof(float));
    add(ln * sizeof(float));
    if (!(lr % 2 == 0 && lz % 2 == 0 && lr >= 4 && lz >= 4)) break;
    lr /= 2;
    lz /= 2;
  }
  add(8 * 2048 * sizeof(double));  // partial sums: 2 parities x 4 slots x blocks
  add(256);                        // barrier words
  return bytes;
}

// ----------------------------------------------------------------------------
// device pieces
// ----------------------------------------------------------------------------
// Grid barrier with a time limit.  The arrival counter and the generation word
// sit in different 128-byte lines so that the waiting blocks' polling does not
// contend with the arrivals.
constexpr int kBarGen = 32;   // bar[0]: arrivals, bar[kBarGen]: generation

__device__ __forceinline__ bool barrier_grid(unsigned int* bar, int* status) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = bar + kBarGen;
    const unsigned int g = *vgen;
    __threadfence();
    const unsigned int arrived = atomicAdd(bar, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + kBarGen, 1u);
    } else {
      const double t0 = global_time_ns();
      unsigned int spins = 0;
      while (*vgen == g) {
        if ((++spins & 255u) == 0u && global_time_ns() - t0 > kBarrierLimitNs) {
          atomicOr(status, ST_TIMEOUT);
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return (*(volatile int*)status & ST_TIMEOUT) == 0;
}

// physical couplings (FP64) at the finest level
__device__ __forceinline__ double ar64(const PoissonWork& W, int m) {
  return 2.0 * kPi * kEps0 * (m + 0.5) * W.dz;
}
__device__ __forceinline__ double az64(const PoissonWork& W, int m) {
  const double area = m == 0 ? kPi * 0.25 * W.dr * W.dr : 2.0 * kPi * (m * W.dr) * W.dr;
  return kEps0 * area / W.dz;
}
// scaled couplings (operator / (2 pi eps0)) of level l, FP32
__device__ __forceinline__ float ar32(float dzl, int m) { return dzl * ((float)m + 0.5f); }
__device__ __forceinline__ float az32(float drl, float dzl, int m) {
  return m == 0 ? drl * drl / (8.0f * dzl) : (float)m * drl * drl / dzl;
}

struct Lev {
  int nr, nz;
  float dr, dz;
  float* u;
  float* f;
};

__device__ __forceinline__ Lev lev(const PoissonWork& W, int l) {
  Lev L;
  L.nr = W.lnr[l];
  L.nz = W.lnz[l];
  L.dr = (float)(W.dr * (double)(1 << l));
  L.dz = (float)(W.dz * (double)(1 << l));
  L.u = W.u[l];
  L.f = W.f[l];
  return L;
}

// red-black Gauss-Seidel half sweep over free nodes of `color`
__device__ void smooth(const Lev& L, int color, int tid, int nthr) {
  const int nzf = L.nz - 1;          // free nodes per radial line
  const int nfree = L.nr * nzf;
  const int nz1 = L.nz + 1;
  for (int k = tid; k < nfree; k += nthr) {
    const int m = k / nzf, n = 1 + (k - m * nzf);
    if (((m + n) & 1) != color) continue;
    const int i = m * nz1 + n;
    const float az = az32(L.dr, L.dz, m);
    const float arp = ar32(L.dz, m);
    const float arm = m > 0 ? ar32(L.dz, m - 1) : 0.0f;
    float s = L.f[i] + az * (L.u[i - 1] + L.u[i + 1]) + arp * L.u[i + nz1];
    if (m > 0) s += arm * L.u[i - nz1];
    L.u[i] = s / (2.0f * az + arp + arm);
  }
}

__device__ __forceinline__ float resid_at(const Lev& L, int m, int n) {
  // residual of a free node (zero outside the free set)
  if (m < 0 || m >= L.nr || n < 1 || n >= L.nz) return 0.0f;
  const int nz1 = L.nz + 1;
  const int i = m * nz1 + n;
  const float az = az32(L.dr, L.dz, m);
  const float arp = ar32(L.dz, m);
  const float arm = m > 0 ? ar32(L.dz, m - 1) : 0.0f;
  float a = (2.0f * az + arp + arm) * L.u[i] - az * (L.u[i - 1] + L.u[i + 1]) - arp * L.u[i + nz1];
  if (m > 0) a -= arm * L.u[i - nz1];
  return L.f[i] - a;
}

// coarse f = P^T (fine residual), coarse u = 0
__device__ void restrict_to(const Lev& F, const Lev& C, int tid, int nthr) {
  const int nzf = C.nz - 1;
  const int nfree = C.nr * nzf;
  const int nz1 = C.nz + 1;
  for (int k = tid; k < nfree; k += nthr) {
    const int M = k / nzf, N = 1 + (k - M * nzf);
    float s = 0.0f;
#pragma unroll
    for (int di = -1; di <= 1; ++di) {
      const float wi = di == 0 ? 1.0f : 0.5f;
#pragma unroll
      for (int dj = -1; dj <= 1; ++dj) {
        const float wj = dj == 0 ? 1.0f : 0.5f;
        s += wi * wj * resid_at(F, 2 * M + di, 2 * N + dj);
      }
    }
    C.f[M * nz1 + N] = s;
    C.u[M * nz1 + N] = 0.0f;
  }
}

// fine u += bilinear interpolation of coarse u (zero on coarse Dirichlet nodes)
__device__ void prolong_from(const Lev& F, const Lev& C, int tid, int nthr) {
  const int nzf = F.nz - 1;
  const int nfree = F.nr * nzf;
  const int fz1 = F.nz + 1, cz1 = C.nz + 1;
  for (int k = tid; k < nfree; k += nthr) {
    const int m = k / nzf, n = 1 + (k - m * nzf);
    const int cm = m >> 1, cn = n >> 1;
    float v;
    const float* u = C.u;
    if ((m & 1) == 0 && (n & 1) == 0) v = u[cm * cz1 + cn];
    else if ((n & 1) == 0) v = 0.5f * (u[cm * cz1 + cn] + u[(cm + 1) * cz1 + cn]);
    else if ((m & 1) == 0) v = 0.5f * (u[cm * cz1 + cn] + u[cm * cz1 + cn + 1]);
    else
      v = 0.25f * (u[cm * cz1 + cn] + u[(cm + 1) * cz1 + cn] + u[cm * cz1 + cn + 1] +
                   u[(cm + 1) * cz1 + cn + 1]);
    F.u[m * fz1 + n] += v;
  }
}

// Levels >= l0 inside one CTA (block-level synchronisation only).
constexpr int kTailSmemFloats = 2 * 5800;   // u and f of levels with <= kTailNodes nodes

__device__ void vcycle_levels(Lev* T, int l0, int nlev) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int l = l0; l < nlev - 1; ++l) {
    smooth(T[l], 0, tid, nthr);
    __syncthreads();
    smooth(T[l], 1, tid, nthr);
    __syncthreads();
    restrict_to(T[l], T[l + 1], tid, nthr);
    __syncthreads();
  }
  {
    const Lev& C = T[nlev - 1];
    for (int s = 0; s < 8; ++s) {
      smooth(C, 0, tid, nthr);
      __syncthreads();
      smooth(C, 1, tid, nthr);
      __syncthreads();
    }
    for (int s = 0; s < 8; ++s) {
      smooth(C, 1, tid, nthr);
      __syncthreads();
      smooth(C, 0, tid, nthr);
      __syncthreads();
    }
  }
  for (int l = nlev - 2; l >= l0; --l) {
    prolong_from(T[l], T[l + 1], tid, nthr);
    __syncthreads();
    smooth(T[l], 1, tid, nthr);
    __syncthreads();
    smooth(T[l], 0, tid, nthr);
    __syncthreads();
  }
}

// The tail in shared memory when it fits in `buf` (f of level l0 loaded, u
// of level l0 written back), else in the global level arrays.
__device__ void vcycle_tail(const PoissonWork& W, int l0, float* buf) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  Lev T[kMaxLev];
  int total = 0;
  for (int l = l0; l < W.nlev; ++l) {
    T[l] = lev(W, l);
    total += 2 * (T[l].nr + 1) * (T[l].nz + 1);
  }
  if (total > kTailSmemFloats) {
    vcycle_levels(T, l0, W.nlev);
    return;
  }
  float* p = buf;
  for (int l = l0; l < W.nlev; ++l) {
    const int nn = (T[l].nr + 1) * (T[l].nz + 1);
    T[l].u = p;
    T[l].f = p + nn;
    p += 2 * nn;
  }
  for (int k = tid; k < total; k += nthr) buf[k] = 0.0f;
  __syncthreads();
  const int nn0 = (T[l0].nr + 1) * (T[l0].nz + 1);
  const float* fg = W.f[l0];
  for (int k = tid; k < nn0; k += nthr) T[l0].f[k] = fg[k];
  __syncthreads();
  vcycle_levels(T, l0, W.nlev);
  float* ug = W.u[l0];
  for (int k = tid; k < nn0; k += nthr) ug[k] = T[l0].u[k];
}

__device__ __forceinline__ double warp_sum64(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block partial sums of up to 3 values written to partial[slot][block]; after
// a grid barrier every block reads them back in block order (deterministic).
__device__ void block_partials(double* partial, int parity, int nvals, const double* v) {
  __shared__ double red[3][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int j = 0; j < nvals; ++j) {
    const double s = warp_sum64(v[j]);
    if (lane == 0) red[j][w] = s;
  }
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    for (int j = 0; j < nvals; ++j) {
      double s = lane < nw ? red[j][lane] : 0.0;
      s = warp_sum64(s);
      if (lane == 0) partial[(parity * 4 + j) * gridDim.x + blockIdx.x] = s;
    }
  }
  __syncthreads();
}

__device__ void read_partials(const double* partial, int parity, int nvals, double* out) {
  __shared__ double res[3];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (w == 0) {
    for (int j = 0; j < nvals; ++j) {
      double s = 0.0;
      const volatile double* p = partial + (parity * 4 + j) * gridDim.x;
      for (int b = lane; b < (int)gridDim.x; b += 32) s += p[b];
      s = warp_sum64(s);
      if (lane == 0) res[j] = s;
    }
  }
  __syncthreads();
  for (int j = 0; j < nvals; ++j) out[j] = res[j];
  __syncthreads();
}

__global__ void __launch_bounds__(kPoisThreads) k_poisson(PoissonArgs A) {
  const PoissonWork& W = A.W;
  if (*(volatile int*)A.status & (ST_FATAL)) return;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int gthr = gridDim.x * blockDim.x;
  const int nr = W.nr, nz = W.nz, nz1 = nz + 1;
  const int nzf = nz - 1, nfree = nr * nzf;
  double* phi = A.phi;
  int parity = 0;
  double vals[3];
  __shared__ float tail_buf[kTailSmemFloats];

  // residual r = Q - A phi (Dirichlet values in phi), ||b||^2, ||r||^2
  double bb = 0.0, rr = 0.0;
  for (int k = gtid; k < nfree; k += gthr) {
    const int m = k / nzf, n = 1 + (k - m * nzf);
    const int i = m * nz1 + n;
    const double az = az64(W, m), arp = ar64(W, m), arm = m > 0 ? ar64(W, m - 1) : 0.0;
    double a = az * (2.0 * phi[i] - phi[i - 1] - phi[i + 1]) + arp * (phi[i] - phi[i + nz1]);
    if (m > 0) a += arm * (phi[i] - phi[i - nz1]);
    double b = A.Q[i];
    if (n == 1) b += az * phi[i - 1];
    if (n == nz - 1) b += az * phi[i + 1];
    if (m == nr - 1) b += arp * phi[i + nz1];
    const double r = A.Q[i] - a;
    W.r[i] = r;
    bb += b * b;
    rr += r * r;
  }
  vals[0] = bb;
  vals[1] = rr;
  block_partials(W.partial, parity, 2, vals);
  if (!barrier_grid(W.bar, A.status)) return;
  read_partials(W.partial, parity, 2, vals);
  parity ^= 1;
  bb = vals[0];
  rr = vals[1];
  const double tol2bb = A.tol * A.tol * bb;
  int it = 0;
  bool converged = rr <= tol2bb;
  double rz = 0.0, alpha = 0.0;
  bool first = true;
  int restarts = 0;

  while (!converged && it < A.max_iter) {
    // ---- z = M^{-1} r : scale, V-cycle in FP32, unscale -------------------
    const double scale = rr > 0.0 ? 1.0 / sqrt(rr / (double)nfree) : 1.0;
    {
      const Lev L0 = lev(W, 0);
      for (int k = gtid; k < nfree; k += gthr) {
        const int m = k / nzf, n = 1 + (k - m * nzf);
        const int i = m * nz1 + n;
        L0.f[i] = (float)(W.r[i] * scale);
        L0.u[i] = 0.0f;
      }
      if (!barrier_grid(W.bar, A.status)) return;
    }
    for (int l = 0; l < W.tail; ++l) {
      const Lev F = lev(W, l), C = lev(W, l + 1);
      smooth(F, 0, gtid, gthr);
      if (!barrier_grid(W.bar, A.status)) return;
      smooth(F, 1, gtid, gthr);
      if (!barrier_grid(W.bar, A.status)) return;
      restrict_to(F, C, gtid, gthr);
      if (!barrier_grid(W.bar, A.status)) return;
    }
    if (blockIdx.x == 0) vcycle_tail(W, W.tail, tail_buf);
    if (!barrier_grid(W.bar, A.status)) return;
    for (int l = W.tail - 1; l >= 0; --l) {
      const Lev F = lev(W, l), C = lev(W, l + 1);
      prolong_from(F, C, gtid, gthr);
      if (!barrier_grid(W.bar, A.status)) return;
      smooth(F, 1, gtid, gthr);
      if (!barrier_grid(W.bar, A.status)) return;
      smooth(F, 0, gtid, gthr);
      if (!barrier_grid(W.bar, A.status)) return;
    }
    {
      const Lev L0 = lev(W, 0);
      const double unscale = 1.0 / (2.0 * kPi * kEps0 * scale);
      double rz_loc = 0.0, zq_loc = 0.0;
      for (int k = gtid; k < nfree; k += gthr) {
        const int m = k / nzf, n = 1 + (k - m * nzf);
        const int i = m * nz1 + n;
        const double zi = (double)L0.u[i] * unscale;
        W.z[i] = zi;
        rz_loc += W.r[i] * zi;
        if (!first) zq_loc += zi * W.q[i];
      }
      vals[0] = rz_loc;
      vals[1] = zq_loc;
      block_partials(W.partial, parity, 2, vals);
      if (!barrier_grid(W.bar, A.status)) return;
      read_partials(W.partial, parity, 2, vals);
      parity ^= 1;
    }
    // ---- direction: p = z + beta p (flexible Polak-Ribiere beta) ----------
    const double beta = first ? 0.0 : -alpha * vals[1] / rz;
    rz = vals[0];
    first = false;
    for (int k = gtid; k < nfree; k += gthr) {
      const int m = k / nzf, n = 1 + (k - m * nzf);
      const int i = m * nz1 + n;
      W.p[i] = W.z[i] + beta * W.p[i];
    }
    if (!barrier_grid(W.bar, A.status)) return;
    // ---- q = A p, alpha = rz / (p.q) --------------------------------------
    double pq = 0.0;
    for (int k = gtid; k < nfree; k += gthr) {
      const int m = k / nzf, n = 1 + (k - m * nzf);
      const int i = m * nz1 + n;
      const double az = az64(W, m), arp = ar64(W, m), arm = m > 0 ? ar64(W, m - 1) : 0.0;
      const double pi = W.p[i];
      const double pl = n > 1 ? W.p[i - 1] : 0.0, pu = n < nz - 1 ? W.p[i + 1] : 0.0;
      const double po = m < nr - 1 ? W.p[i + nz1] : 0.0, pn = m > 0 ? W.p[i - nz1] : 0.0;
      double a = az * (2.0 * pi - pl - pu) + arp * (pi - po);
      if (m > 0) a += arm * (pi - pn);
      W.q[i] = a;
      pq += pi * a;
    }
    vals[0] = pq;
    block_partials(W.partial, parity, 1, vals);
    if (!barrier_grid(W.bar, A.status)) return;
    read_partials(W.partial, parity, 1, vals);
    parity ^= 1;
    alpha = vals[0] != 0.0 ? rz / vals[0] : 0.0;
    // ---- phi += alpha p, r -= alpha q --------------------------------------
    double rl = 0.0;
    for (int k = gtid; k < nfree; k += gthr) {
      const int m = k / nzf, n = 1 + (k - m * nzf);
      const int i = m * nz1 + n;
      phi[i] += alpha * W.p[i];
      const double r = W.r[i] - alpha * W.q[i];
      W.r[i] = r;
      rl += r * r;
    }
    vals[0] = rl;
    block_partials(W.partial, parity, 1, vals);
    if (!barrier_grid(W.bar, A.status)) return;
    read_partials(W.partial, parity, 1, vals);
    parity ^= 1;
    rr = vals[0];
    ++it;
    if (rr <= tol2bb) {
      // confirm with the true residual b - A phi
      double rt = 0.0;
      for (int k = gtid; k < nfree; k += gthr) {
        const int m = k / nzf, n = 1 + (k - m * nzf);
        const int i = m * nz1 + n;
        const double az = az64(W, m), arp = ar64(W, m), arm = m > 0 ? ar64(W, m - 1) : 0.0;
        double a = az * (2.0 * phi[i] - phi[i - 1] - phi[i + 1]) + arp * (phi[i] - phi[i + nz1]);
        if (m > 0) a += arm * (phi[i] - phi[i - nz1]);
        const double r = A.Q[i] - a;
        W.r[i] = r;
        rt += r * r;
      }
      vals[0] = rt;
      block_partials(W.partial, parity, 1, vals);
      if (!barrier_grid(W.bar, A.status)) return;
      read_partials(W.partial, parity, 1, vals);
      parity ^= 1;
      rr = vals[0];
      if (rr <= tol2bb || restarts >= 3) {
        converged = rr <= tol2bb;
        break;
      }
      ++restarts;
      first = true;  // restart the Krylov space from the true residual
    }
  }
  if (gtid == 0) {
    *A.iters = it;
    *A.resid = bb > 0.0 ? sqrt(rr / bb) : sqrt(rr);
    if (!converged) atomicOr(A.status, ST_NONCONV);
  }
}

// ----------------------------------------------------------------------------
// host side
// ----------------------------------------------------------------------------
struct PoissonWorkHost {
  PoissonWork w;
  double tol;
  int max_iter;
};

PoissonWork* poisson_work_init(void* base, int nr, int nz, double R, double L, int num_sms) {
  PoissonWork* pw = new PoissonWork();
  std::memset(pw, 0, sizeof(*pw));
  pw->nr = nr;
  pw->nz = nz;
  pw->dr = R / nr;
  pw->dz = L / nz;
  char* p = (char*)base;
  auto take = [&](size_t b) {
    char* q = p;
    p += (b + 255) & ~(size_t)255;
    return (void*)q;
  };
  const size_t nn = (size_t)(nr + 1) * (nz + 1);
  pw->r = (double*)take(nn * sizeof(double));
  pw->p = (double*)take(nn * sizeof(double));
  pw->q = (double*)take(nn * sizeof(double));
  pw->z = (double*)take(nn * sizeof(double));
  int lr = nr, lz = nz, l = 0;
  pw->tail = -1;
  for (; l < kMaxLev; ++l) {
    const size_t ln = (size_t)(lr + 1) * (lz + 1);
    pw->lnr[l] = lr;
    pw->lnz[l] = lz;
    pw->u[l] = (float*)take(ln * sizeof(float));
    pw->f[l] = (float*)take(ln * sizeof(float));
    if (pw->tail < 0 && ln <= (size_t)kTailNodes) pw->tail = l;
    if (!(lr % 2 == 0 && lz % 2 == 0 && lr >= 4 && lz >= 4)) break;
    lr /= 2;
    lz /= 2;
  }
  pw->nlev = l + 1;
  if (pw->tail < 0) pw->tail = pw->nlev - 1;
  pw->partial = (double*)take(8 * 2048 * sizeof(double));
  pw->bar = (unsigned int*)take(256);
  // blocks: enough for the free nodes at ~1 per thread, at most one wave
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_poisson, kPoisThreads, 0);
  if (per_sm < 1) per_sm = 1;
  long long want = ((long long)nr * (nz - 1) + kPoisThreads - 1) / kPoisThreads;
  long long cap = (long long)num_sms * per_sm;
  if (cap > 2048) cap = 2048;
  if (want > cap) want = cap;
  if (want < 1) want = 1;
  pw->nblocks = (int)want;
  return pw;
}

void poisson_work_free(PoissonWork* pw) { delete pw; }

cudaError_t launch_poisson(PoissonWork* pw, const double* Q, double* phi, double tol, int max_iter,
                           int* status_dev, int* iters_dev, double* resid_dev, cudaStream_t st) {
  PoissonArgs a;
  a.W = *pw;
  a.Q = Q;
  a.phi = phi;
  a.tol = tol;
  a.max_iter = max_iter;
  a.status = status_dev;
  a.iters = iters_dev;
  a.resid = resid_dev;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel((const void*)k_poisson, dim3(pw->nblocks), dim3(kPoisThreads),
                                     args, 0, st);
}

}  // namespace pic

// ----------------------------------------------------------------------------
// Variant for pic_poisson_solve_static: the workspace layout is built in a
// struct on the host stack (no host or device allocation), over the caller's
// scratch at `base`.  The layout is the one poisson_work_bytes() sizes.
// ----------------------------------------------------------------------------
namespace pic {

cudaError_t launch_poisson_in_place(void* base, int nr, int nz, double R, double L, int num_sms,
                                    const double* Q, double* phi, double tol, int max_iter,
                                    int* status_dev, int* iters_dev, double* resid_dev,
                                    cudaStream_t st) {
  PoissonArgs a;
  std::memset(&a, 0, sizeof(a));
  PoissonWork& w = a.W;
  w.nr = nr;
  w.nz = nz;
  w.dr = R / nr;
  w.dz = L / nz;
  char* p = (char*)base;
  auto take = [&](size_t b) {
    char* q = p;
    p += (b + 255) & ~(size_t)255;
    return (void*)q;
  };
  const size_t nn = (size_t)(nr + 1) * (nz + 1);
  w.r = (double*)take(nn * sizeof(double));
  w.p = (double*)take(nn * sizeof(double));
  w.q = (double*)take(nn * sizeof(double));
  w.z = (double*)take(nn * sizeof(double));
  int lr = nr, lz = nz, l = 0;
  w.tail = -1;
  for (; l < kMaxLev; ++l) {
    const size_t ln = (size_t)(lr + 1) * (lz + 1);
    w.lnr[l] = lr;
    w.lnz[l] = lz;
    w.u[l] = (float*)take(ln * sizeof(float));
    w.f[l] = (float*)take(ln * sizeof(float));
    if (w.tail < 0 && ln <= (size_t)kTailNodes) w.tail = l;
    if (!(lr % 2 == 0 && lz % 2 == 0 && lr >= 4 && lz >= 4)) break;
    lr /= 2;
    lz /= 2;
  }
  w.nlev = l + 1;
  if (w.tail < 0) w.tail = w.nlev - 1;
  w.partial = (double*)take(8 * 2048 * sizeof(double));
  w.bar = (unsigned int*)take(256);
  if ((size_t)(p - (char*)base) != poisson_work_bytes(nr, nz)) return cudaErrorInvalidValue;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_poisson, kPoisThreads, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  long long want = ((long long)nr * (nz - 1) + kPoisThreads - 1) / kPoisThreads;
  long long cap = (long long)num_sms * per_sm;
  if (cap > 2048) cap = 2048;
  if (want > cap) want = cap;
  if (want < 1) want = 1;
  w.nblocks = (int)want;
  a.Q = Q;
  a.phi = phi;
  a.tol = tol;
  a.max_iter = max_iter;
  a.status = status_dev;
  a.iters = iters_dev;
  a.resid = resid_dev;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel((const void*)k_poisson, dim3(w.nblocks), dim3(kPoisThreads),
                                     args, 0, st);
}

}  // namespace pic
