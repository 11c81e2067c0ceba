// poisson.cu -- RZ Poisson solve (arXiv:2507.10727, Section 3: anode
// grounded, cathode at the circuit voltage, the insulating block a Neumann
// boundary, Gauss's law on the axis).
//
// Discretisation (the paper gives none; finite-volume reading): for a free
// node (m, n) the equation times the node's control volume (its part of the
// box r_m -+ dr/2, z_n -+ dz/2 inside the domain) reads
// sum_j a_kj (phi_k - phi_j) = Q_k  with
//   a_r(m) h(n) = 2 pi eps0 (m + 1/2) dz h(n)  between (m,n) and (m+1,n),
//                 h = 1/2 on z = 0 (half-height faces), else 1
//   a_z(m) = eps0 area(m) / dz                between (m,n) and (m,n+1)
//   area(m) = 2 pi m dr^2 (0 < m < nr), pi dr^2 / 4 (axis: Gauss on the disk
//   dr/2), pi (nr - 1/4) dr^2 (half annulus at r = R)
// and no flux through the domain's surface, which is symmetric positive
// definite on the free nodes.  Free nodes: the interior m = 0..nr-1,
// n = 1..nz-1, plus the insulating boundary "line" (row 0 from node g on,
// then the wall column m = nr when it is insulating); the rest of the
// boundary holds Dirichlet values.
//
// Solver: one cooperative persistent kernel.  Flexible preconditioned
// conjugate gradients with iterates, residuals and dot products in FP64
// (deterministic block-ordered reductions); the preconditioner is one
// geometric-multigrid V-cycle in FP32 on the same operator rediscretised at
// 2x, 4x ... coarser spacing (red-black Gauss-Seidel, residual restriction by
// the transpose of bilinear prolongation).  Because the outer iteration and
// its stopping test (relative residual ||b - A phi||_2 <= tol ||b||_2) are
// FP64, the converged phi does not depend on the preconditioner's precision.
//
// Layout of the work: the couplings of every level are tabulated per radial
// index in shared memory at the start of the launch; the coarse levels that
// fit in shared memory run inside one CTA ("tail"); the finer levels use the
// whole grid with a time-bounded grid barrier.  Nodes are visited as (row,
// 32-wide segment) items per warp, so no per-node integer division is needed.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "launch.h"
#include "unet.h"

namespace pic {

constexpr int kMaxLev = 16;
constexpr int kPoisThreads = 512;
constexpr double kBarrierLimitNs = 2.0e9;
constexpr size_t kSmemBudget = 200 * 1024;   // dynamic shared memory per block
constexpr int kTailMaxNodes = 65 * 65;       // finest level handled inside one CTA
constexpr int kCoarseSweeps = 4;             // symmetric sweep pairs on the coarsest level

struct PoissonWork {
  int nr, nz, nlev, tail;
  double dr, dz;
  int nblocks;
  int smem_bytes;          // dynamic shared memory per block
  int lnr[kMaxLev], lnz[kMaxLev];
  int bc_g[kMaxLev];       // first free node of row 0 per level (lnr + 1: none)
  int bc_wall;             // 1: the wall column m = nr is free (insulating)
  int coef_off[kMaxLev];   // offset of level l in the per-level coupling tables
  int ncoef;               // entries of each coupling table
  int tail_floats;         // shared-memory floats of the tail levels (u and f)
  float* u[kMaxLev];
  float* f[kMaxLev];
  double *r, *p, *q, *z;
  double* partial;
  unsigned int* bar;
  // Sine-transform preconditioner (every boundary node a conductor): the
  // operator is D (x) T + L (x) I on the free nodes (m = 0..nr-1, n = 1..nz-1;
  // T the 1D second difference along z, D = a_z(m), L the radial part), so
  // the discrete sine transform along z splits it into nz-1 tridiagonal
  // systems in m.  Null when the multigrid preconditioner is used.
  int nk;                  // modes: nz - 1
  int rows_per_block;      // rows of one block in the row-wise phases
  int sep_blocks;          // blocks of one solve
  int ldS;                 // row stride of sMat: nk rounded up to a multiple of 4
  float* sMat;             // nk x ldS: the orthonormal DST-I matrix S[n][k] =
                           // sqrt(2/nz) sin(pi (n+1)(k+1) / nz) (symmetric), zero for k >= nk
  float* sW;               // nr x nk: 1 / pivot of the Thomas elimination of mode k at row m
  float* sC;               // nr x nk: its upper factor
  float* sE;               // nr: coupling a_r(m) / (2 pi eps0) between rows m and m + 1
  float* sHat;             // nr x nk: transformed residual, then the mode solutions
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

static size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

static int level_count(int nr, int nz, int* lnr, int* lnz) {
  int lr = nr, lz = nz, l = 0;
  for (; l < kMaxLev; ++l) {
    lnr[l] = lr;
    lnz[l] = lz;
    if (!(lr % 2 == 0 && lz % 2 == 0 && lr >= 4 && lz >= 4)) break;
    lr /= 2;
    lz /= 2;
  }
  return l + 1;
}

size_t poisson_work_bytes(int nr, int nz) {
  size_t bytes = 0;
  const size_t nn = (size_t)(nr + 1) * (nz + 1);
  for (int k = 0; k < 4; ++k) bytes += round256(nn * sizeof(double));
  int lnr[kMaxLev], lnz[kMaxLev];
  const int nlev = level_count(nr, nz, lnr, lnz);
  for (int l = 0; l < nlev; ++l) {
    const size_t ln = (size_t)(lnr[l] + 1) * (lnz[l] + 1);
    bytes += 2 * round256(ln * sizeof(float));
  }
  bytes += round256(8 * 2048 * sizeof(double));  // partial sums: 2 parities x 4 slots x blocks
  bytes += 256;                                  // barrier words
  return bytes;
}

// Layout of the workspace at `base` (poisson_work_bytes bytes) and of the
// shared memory: FP64 level-0 tables, three FP32 tables, then the tail levels.
static void layout(PoissonWork& w, void* base, int nr, int nz, double R, double L, int g,
                   int wall) {
  std::memset(&w, 0, sizeof(w));
  w.nr = nr;
  w.nz = nz;
  w.bc_wall = wall ? 1 : 0;
  w.dr = R / nr;
  w.dz = L / nz;
  char* p = (char*)base;
  auto take = [&](size_t b) {
    char* q = p;
    p += round256(b);
    return (void*)q;
  };
  const size_t nn = (size_t)(nr + 1) * (nz + 1);
  w.r = (double*)take(nn * sizeof(double));
  w.p = (double*)take(nn * sizeof(double));
  w.q = (double*)take(nn * sizeof(double));
  w.z = (double*)take(nn * sizeof(double));
  w.nlev = level_count(nr, nz, w.lnr, w.lnz);
  // a coarse row-0 node is free when the fine node at the same place is
  w.bc_g[0] = g < 0 ? 0 : (g > nr + 1 ? nr + 1 : g);
  for (int l = 1; l < w.nlev; ++l) w.bc_g[l] = (w.bc_g[l - 1] + 1) / 2;
  int off = 0;
  for (int l = 0; l < w.nlev; ++l) {
    const size_t ln = (size_t)(w.lnr[l] + 1) * (w.lnz[l] + 1);
    w.u[l] = (float*)take(ln * sizeof(float));
    w.f[l] = (float*)take(ln * sizeof(float));
    w.coef_off[l] = off;
    off += w.lnr[l] + 1;
  }
  w.ncoef = off;
  w.partial = (double*)take(8 * 2048 * sizeof(double));
  w.bar = (unsigned int*)take(256);
  const size_t tables = 2 * (size_t)(nr + 1) * sizeof(double) + 3 * (size_t)w.ncoef * sizeof(float);
  w.tail = w.nlev - 1;
  w.tail_floats = 2 * (w.lnr[w.nlev - 1] + 1) * (w.lnz[w.nlev - 1] + 1);
  for (int l = w.nlev - 1; l >= 0; --l) {
    size_t fl = 0;
    for (int k = l; k < w.nlev; ++k) fl += 2 * (size_t)(w.lnr[k] + 1) * (w.lnz[k] + 1);
    if (tables + fl * sizeof(float) > kSmemBudget) break;
    if (l < w.nlev - 1 && (size_t)(w.lnr[l] + 1) * (w.lnz[l] + 1) > (size_t)kTailMaxNodes) break;
    w.tail = l;
    w.tail_floats = (int)fl;
  }
  w.smem_bytes = (int)(tables + (size_t)w.tail_floats * sizeof(float));
}

// ----------------------------------------------------------------------------
// device pieces
// ----------------------------------------------------------------------------
// Grid barrier with a time limit.  The arrival counter and the generation word
// sit in different 128-byte lines so that the waiting blocks' polling does not
// contend with the arrivals.
constexpr int kBarGen = 32;   // bar[0]: arrivals, bar[kBarGen]: generation

// The block's writes are ordered before its arrival by the CTA barrier and
// the arrival's release; the last arrival's release of the generation word,
// read with acquire by the waiting blocks, orders every block's writes before
// what the waiters do after the barrier (acquire/release at GPU scope instead
// of sequentially consistent fences).
__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ bool barrier_grid(unsigned int* bar, int* status, int nb) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int g = ld_acquire_gpu(bar + kBarGen);
    unsigned int arrived;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(arrived) : "l"(bar) : "memory");
    if (arrived == (unsigned)nb - 1u) {
      // every block has arrived, none arrives again before the generation moves
      asm volatile("st.relaxed.gpu.global.u32 [%0], 0;" ::"l"(bar) : "memory");
      asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar + kBarGen) : "memory");
    } else {
      const double t0 = global_time_ns();
      unsigned int spins = 0;
      while (ld_acquire_gpu(bar + kBarGen) == g) {
        if ((++spins & 255u) == 0u && global_time_ns() - t0 > kBarrierLimitNs) {
          atomicOr(status, ST_TIMEOUT);
          break;
        }
      }
    }
  }
  __syncthreads();
  return (*(volatile int*)status & ST_TIMEOUT) == 0;
}

// One level: node arrays and its coupling tables per radial index m, scaled
// by 1/(2 pi eps0): az = a_z(m), ar = a_r(m) (between m and m+1), idg = 1 /
// diagonal.
struct Lev {
  int nr, nz;
  int g, wall;   // insulating boundary nodes (row 0 from g on, the wall column)
  float* u;
  float* f;
  const float* az;
  const float* ar;
  const float* idg;
};

struct Tables {
  const double* az0;   // level 0, FP64, physical units
  const double* ar0;
  const float* az;
  const float* ar;
  const float* idg;
};

__device__ __forceinline__ Lev lev(const PoissonWork& W, const Tables& T, int l, float* u, float* f) {
  Lev L;
  L.nr = W.lnr[l];
  L.nz = W.lnz[l];
  L.g = W.bc_g[l];
  L.wall = W.bc_wall;
  L.u = u;
  L.f = f;
  L.az = T.az + W.coef_off[l];
  L.ar = T.ar + W.coef_off[l];
  L.idg = T.idg + W.coef_off[l];
  return L;
}

// Fine-level couplings of the volume-scaled RZ operator at radial index m:
// az (along z, between n and n +- 1) and ar (between m and m + 1).
__device__ __forceinline__ void fine_coef(const PoissonWork& W, int m, double& az, double& ar) {
  const double c = 2.0 * kPi * kEps0;
  az = m == 0       ? c * W.dr * W.dr / (8.0 * W.dz)
       : m == W.nr ? c * (m - 0.25) * W.dr * W.dr / (2.0 * W.dz)
                   : c * m * W.dr * W.dr / W.dz;
  ar = c * (m + 0.5) * W.dz;
}

// Insulating boundary nodes of a level, numbered j = 0, 1, ...: row 0 from
// node g to nr - 1 (to nr when the wall is insulating too), then the wall
// column m = nr, n = 1 .. nz - 1.
__host__ __device__ __forceinline__ int line_gap(int nr, int g, int wall) {
  const int last = wall ? nr : nr - 1;
  return last >= g ? last - g + 1 : 0;
}
__host__ __device__ __forceinline__ int line_count(int nr, int nz, int g, int wall) {
  return line_gap(nr, g, wall) + (wall ? nz - 1 : 0);
}
__device__ __forceinline__ void line_node(int j, int nr, int g, int ngap, int& m, int& n) {
  if (j < ngap) {
    m = g + j;
    n = 0;
  } else {
    m = nr;
    n = 1 + (j - ngap);
  }
}

// Gauss-Seidel pieces at an insulating boundary node: s = sum of couplings
// times neighbour values (neighbours inside the grid; r-couplings halved on
// row 0), diag = sum of couplings.  Values on Dirichlet nodes are zero in the
// multigrid arrays (corrections).
__device__ __forceinline__ float line_sum(const Lev& L, int m, int n, float& diag) {
  const int nz1 = L.nz + 1, i = m * nz1 + n;
  const float h = n == 0 ? 0.5f : 1.0f;
  const float az = L.az[m];
  float s = az * L.u[i + 1];
  diag = az;
  if (n > 0) {
    s += az * L.u[i - 1];
    diag += az;
  }
  if (m < L.nr) {
    const float c = h * L.ar[m];
    s += c * L.u[i + nz1];
    diag += c;
  }
  if (m > 0) {
    const float c = h * L.ar[m - 1];
    s += c * L.u[i - nz1];
    diag += c;
  }
  return s;
}

// Nodes are visited as warp items (row m, 32-wide segment of n):
//   full sweep:    n = 1 + 32 seg + lane
//   colour sweep:  the nodes of row m with (m + n) % 2 == colour,
//                  n = 2 (32 seg + lane) + 1 (odd n) or + 2 (even n)
__device__ __forceinline__ int segs_full(int nz) { return (nz - 1 + 31) >> 5; }
__device__ __forceinline__ int segs_color(int nz) { return (nz / 2 + 32) >> 5; }

// LINES: the problem has insulating boundary nodes (else the interior loops
// alone, the all-conductor case)
template <bool LINES>
__device__ void smooth(const Lev L, int color, int wid, int nw, int lane) {
  const int ns = segs_color(L.nz), nz1 = L.nz + 1;
  const int items = L.nr * ns;
  const int ngap = LINES ? line_gap(L.nr, L.g, L.wall) : 0;
  const int nline = LINES ? ngap + (L.wall ? L.nz - 1 : 0) : 0;
  const int total = LINES ? items + ((nline + 31) >> 5) : items;
  for (int it = wid; it < total; it += nw) {
    if (it < items) {
      const int m = it / ns, s = it - m * ns;
      const int odd = (color + m) & 1;
      const int n = 2 * (s * 32 + lane) + (odd ? 1 : 2);
      if (n > L.nz - 1) continue;
      const int i = m * nz1 + n;
      float sum = L.f[i] + L.az[m] * (L.u[i - 1] + L.u[i + 1]) + L.ar[m] * L.u[i + nz1];
      if (m > 0) sum += L.ar[m - 1] * L.u[i - nz1];
      L.u[i] = sum * L.idg[m];
    } else if constexpr (LINES) {
      const int j = (it - items) * 32 + lane;
      if (j >= nline) continue;
      int m, n;
      line_node(j, L.nr, L.g, ngap, m, n);
      if (((m + n) & 1) != color) continue;
      float diag;
      const float sum = line_sum(L, m, n, diag);
      const int i = m * nz1 + n;
      L.u[i] = (L.f[i] + sum) / diag;
    }
  }
}

template <bool LINES>
__device__ __forceinline__ float resid_at(const Lev L, int m, int n) {
  if (m < 0 || m >= L.nr || n < 1 || n >= L.nz) {
    if constexpr (LINES) {
      if (!field_free(m, n, L.nr, L.nz, L.g, L.wall)) return 0.0f;
      float diag;
      const float s = line_sum(L, m, n, diag);
      const int i = m * (L.nz + 1) + n;
      return L.f[i] - (diag * L.u[i] - s);
    } else {
      return 0.0f;
    }
  }
  const int nz1 = L.nz + 1, i = m * nz1 + n;
  const float arm = m > 0 ? L.ar[m - 1] : 0.0f;
  const float diag = 2.0f * L.az[m] + L.ar[m] + arm;
  float a = diag * L.u[i] - L.az[m] * (L.u[i - 1] + L.u[i + 1]) - L.ar[m] * L.u[i + nz1];
  if (m > 0) a -= arm * L.u[i - nz1];
  return L.f[i] - a;
}

// coarse f = P^T (fine residual), coarse u = 0
template <bool LINES>
__device__ void restrict_to(const Lev F, const Lev C, int wid, int nw, int lane) {
  const int ns = segs_full(C.nz), nz1 = C.nz + 1;
  const int items = C.nr * ns;
  const int ngap = LINES ? line_gap(C.nr, C.g, C.wall) : 0;
  const int nline = LINES ? ngap + (C.wall ? C.nz - 1 : 0) : 0;
  const int total = LINES ? items + ((nline + 31) >> 5) : items;
  for (int it = wid; it < total; it += nw) {
    int M, N;
    if (!LINES || it < items) {
      M = it / ns;
      N = 1 + (it - M * ns) * 32 + lane;
      if (N > C.nz - 1) continue;
    } else {
      const int j = (it - items) * 32 + lane;
      if (j >= nline) continue;
      line_node(j, C.nr, C.g, ngap, M, N);
    }
    float acc = 0.0f;
#pragma unroll
    for (int di = -1; di <= 1; ++di) {
      const float wi = di == 0 ? 1.0f : 0.5f;
#pragma unroll
      for (int dj = -1; dj <= 1; ++dj) {
        const float wj = dj == 0 ? 1.0f : 0.5f;
        acc += wi * wj * resid_at<LINES>(F, 2 * M + di, 2 * N + dj);
      }
    }
    C.f[M * nz1 + N] = acc;
    C.u[M * nz1 + N] = 0.0f;
  }
}

// fine u += bilinear interpolation of coarse u (zero on coarse Dirichlet nodes)
template <bool LINES>
__device__ void prolong_from(const Lev F, const Lev C, int wid, int nw, int lane) {
  const int ns = segs_full(F.nz), fz1 = F.nz + 1, cz1 = C.nz + 1;
  const int items = F.nr * ns;
  const int ngap = LINES ? line_gap(F.nr, F.g, F.wall) : 0;
  const int nline = LINES ? ngap + (F.wall ? F.nz - 1 : 0) : 0;
  const int total = LINES ? items + ((nline + 31) >> 5) : items;
  for (int it = wid; it < total; it += nw) {
    int m, n;
    if (!LINES || it < items) {
      m = it / ns;
      n = 1 + (it - m * ns) * 32 + lane;
      if (n > F.nz - 1) continue;
    } else {
      const int j = (it - items) * 32 + lane;
      if (j >= nline) continue;
      line_node(j, F.nr, F.g, ngap, m, n);
    }
    const int cm = m >> 1, cn = n >> 1;
    const float* u = C.u;
    float v;
    if ((m & 1) == 0 && (n & 1) == 0) v = u[cm * cz1 + cn];
    else if ((n & 1) == 0) v = 0.5f * (u[cm * cz1 + cn] + u[(cm + 1) * cz1 + cn]);
    else if ((m & 1) == 0) v = 0.5f * (u[cm * cz1 + cn] + u[cm * cz1 + cn + 1]);
    else
      v = 0.25f * (u[cm * cz1 + cn] + u[(cm + 1) * cz1 + cn] + u[cm * cz1 + cn + 1] +
                   u[(cm + 1) * cz1 + cn + 1]);
    F.u[m * fz1 + n] += v;
  }
}

// Levels >= l0 inside this CTA, in shared memory: f of level l0 is loaded
// from global memory (u starts at zero), u of level l0 is written back.  Level
// descriptors are rebuilt from the shared buffer's offsets where they are
// used, so the sweeps address shared memory directly.
__device__ __forceinline__ Lev tail_lev(const PoissonWork& W, const Tables& T, int l0, int l,
                                        float* buf) {
  int off = 0;
  for (int k = l0; k < l; ++k) off += 2 * (W.lnr[k] + 1) * (W.lnz[k] + 1);
  const int nn = (W.lnr[l] + 1) * (W.lnz[l] + 1);
  return lev(W, T, l, buf + off, buf + off + nn);
}

template <bool LINES>
__device__ void vcycle_tail(const PoissonWork& W, const Tables& T, int l0, float* buf) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int k = threadIdx.x; k < W.tail_floats; k += blockDim.x) buf[k] = 0.0f;
  __syncthreads();
  const int nn0 = (W.lnr[l0] + 1) * (W.lnz[l0] + 1);
  {
    const Lev L0 = tail_lev(W, T, l0, l0, buf);
    const float* fg = W.f[l0];
    // eight independent loads in flight per thread
    int k = threadIdx.x;
    for (; k + 7 * (int)blockDim.x < nn0; k += 8 * blockDim.x) {
      float v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = fg[k + j * blockDim.x];
#pragma unroll
      for (int j = 0; j < 8; ++j) L0.f[k + j * blockDim.x] = v[j];
    }
    for (; k < nn0; k += blockDim.x) L0.f[k] = fg[k];
  }
  __syncthreads();
  for (int l = l0; l < W.nlev - 1; ++l) {
    const Lev F = tail_lev(W, T, l0, l, buf), C = tail_lev(W, T, l0, l + 1, buf);
    smooth<LINES>(F, 0, wid, nw, lane);
    __syncthreads();
    smooth<LINES>(F, 1, wid, nw, lane);
    __syncthreads();
    restrict_to<LINES>(F, C, wid, nw, lane);
    __syncthreads();
  }
  if (wid == 0) {
    // coarsest level: one warp, symmetric Gauss-Seidel sweeps
    const Lev C = tail_lev(W, T, l0, W.nlev - 1, buf);
    for (int s = 0; s < kCoarseSweeps; ++s) {
      smooth<LINES>(C, 0, 0, 1, lane);
      __syncwarp();
      smooth<LINES>(C, 1, 0, 1, lane);
      __syncwarp();
    }
    for (int s = 0; s < kCoarseSweeps; ++s) {
      smooth<LINES>(C, 1, 0, 1, lane);
      __syncwarp();
      smooth<LINES>(C, 0, 0, 1, lane);
      __syncwarp();
    }
  }
  __syncthreads();
  for (int l = W.nlev - 2; l >= l0; --l) {
    const Lev F = tail_lev(W, T, l0, l, buf), C = tail_lev(W, T, l0, l + 1, buf);
    prolong_from<LINES>(F, C, wid, nw, lane);
    __syncthreads();
    smooth<LINES>(F, 1, wid, nw, lane);
    __syncthreads();
    smooth<LINES>(F, 0, wid, nw, lane);
    __syncthreads();
  }
  {
    const Lev L0 = tail_lev(W, T, l0, l0, buf);
    float* ug = W.u[l0];
    int k = threadIdx.x;
    for (; k + 7 * (int)blockDim.x < nn0; k += 8 * blockDim.x) {
      float v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = L0.u[k + j * blockDim.x];
#pragma unroll
      for (int j = 0; j < 8; ++j) ug[k + j * blockDim.x] = v[j];
    }
    for (; k < nn0; k += blockDim.x) ug[k] = L0.u[k];
  }
}

__device__ __forceinline__ double warp_sum64(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block partial sums of up to 3 values written to partial[slot][block]; after
// a grid barrier every block reads them back in block order (deterministic).
__device__ void block_partials(double* partial, int parity, int nvals, const double* v, int lb,
                               int nb) {
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
      if (lane == 0) partial[(parity * 4 + j) * nb + lb] = s;
    }
  }
  __syncthreads();
}

__device__ void read_partials(const double* partial, int parity, int nvals, double* out, int nb) {
  __shared__ double res[3];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (w == 0) {
    for (int j = 0; j < nvals; ++j) {
      double s = 0.0;
      const volatile double* p = partial + (parity * 4 + j) * nb;
      for (int b = lane; b < nb; b += 32) s += p[b];
      s = warp_sum64(s);
      if (lane == 0) res[j] = s;
    }
  }
  __syncthreads();
  for (int j = 0; j < nvals; ++j) out[j] = res[j];
  __syncthreads();
}

// (A x) at a free fine node, x holding the Dirichlet values on the boundary
__device__ __forceinline__ double apply64(const Tables& T, const double* x, int m, int i, int nz1) {
  double a = T.az0[m] * (2.0 * x[i] - x[i - 1] - x[i + 1]) + T.ar0[m] * (x[i] - x[i + nz1]);
  if (m > 0) a += T.ar0[m - 1] * (x[i] - x[i - nz1]);
  return a;
}

// (A x) at an insulating boundary node of the fine level; with `masked`
// the neighbours that are Dirichlet nodes count as zero (x a correction),
// else x holds their values.  Optionally adds the Dirichlet couplings
// (a_kj x_j over Dirichlet neighbours j) to *bd.
__device__ __forceinline__ double line_apply64(const Tables& T, const double* x, int m, int n,
                                               int nr, int nz, int g, int wall, bool masked,
                                               double* bd) {
  const int nz1 = nz + 1, i = m * nz1 + n;
  const double h = n == 0 ? 0.5 : 1.0, xi = x[i];
  double a = 0.0;
  auto nb = [&](int mm, int nn, int j, double c) {
    const bool fr = field_free(mm, nn, nr, nz, g, wall);
    const double xj = (masked && !fr) ? 0.0 : x[j];
    a += c * (xi - xj);
    if (bd && !fr) *bd += c * x[j];
  };
  nb(m, n + 1, i + 1, T.az0[m]);
  if (n > 0) nb(m, n - 1, i - 1, T.az0[m]);
  if (m < nr) nb(m + 1, n, i + nz1, h * T.ar0[m]);
  if (m > 0) nb(m - 1, n, i - nz1, h * T.ar0[m - 1]);
  return a;
}

// diagonal of the FP32 operator at an insulating boundary node
__device__ __forceinline__ float line_diag(const Lev& L, int m, int n) {
  const float h = n == 0 ? 0.5f : 1.0f;
  float d = L.az[m] * (n > 0 ? 2.0f : 1.0f);
  if (m < L.nr) d += h * L.ar[m];
  if (m > 0) d += h * L.ar[m - 1];
  return d;
}

// One solve per block group: `group` == nullptr -> the whole grid solves A0;
// otherwise block b works on group[b / bpi] with bpi blocks per solve (the
// ensemble's discharges solved side by side in one launch).
template <bool LINES>
__global__ void __launch_bounds__(kPoisThreads) k_poisson(PoissonArgs A0, const PoissonArgs* group,
                                                          int bpi) {
  __shared__ PoissonArgs sA;
  int lb, nb;
  {
    const PoissonArgs* src = &A0;
    if (group) {
      const int inst = blockIdx.x / bpi;
      lb = blockIdx.x - inst * bpi;
      nb = bpi;
      src = group + inst;
    } else {
      lb = blockIdx.x;
      nb = gridDim.x;
    }
    const unsigned* s4 = reinterpret_cast<const unsigned*>(src);
    unsigned* d4 = reinterpret_cast<unsigned*>(&sA);
    for (int k = threadIdx.x; k < (int)(sizeof(PoissonArgs) / 4); k += blockDim.x) d4[k] = s4[k];
    __syncthreads();
  }
  const PoissonArgs& A = sA;
  const PoissonWork& W = A.W;
  if (*(volatile int*)A.status & (ST_FATAL)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int nr = W.nr, nz = W.nz, nz1 = nz + 1;
  const int lane = threadIdx.x & 31;
  const int gw = (lb * blockDim.x + threadIdx.x) >> 5;
  const int ngw = (nb * blockDim.x) >> 5;
  const int nsf = (nz - 1 + 31) >> 5;            // segments of a fine row
  const int items0 = nr * nsf;
  // insulating boundary nodes follow the interior rows as extra warp items
  const int g0 = W.bc_g[0], wall = W.bc_wall;
  const int ngap0 = LINES ? line_gap(nr, g0, wall) : 0;
  const int nline0 = LINES ? ngap0 + (wall ? nz - 1 : 0) : 0;
  const int itemsT = LINES ? items0 + ((nline0 + 31) >> 5) : items0;
  auto interior = [&](int it) -> bool { return !LINES || it < items0; };
  const long long nfree = (long long)nr * (nz - 1) + nline0;
  double* phi = A.phi;
  // node of warp item `it` for this lane; false when the lane has none
  auto node_of = [&](int it, int& m, int& n) -> bool {
    if (interior(it)) {
      m = it / nsf;
      n = 1 + (it - m * nsf) * 32 + lane;
      return n <= nz - 1;
    }
    const int j = (it - items0) * 32 + lane;
    if (j >= nline0) return false;
    line_node(j, nr, g0, ngap0, m, n);
    return true;
  };

  // ---- coupling tables of every level in shared memory ----------------------
  double* az0 = (double*)smem;
  double* ar0 = az0 + (nr + 1);
  float* taz = (float*)(ar0 + (nr + 1));
  float* tar = taz + W.ncoef;
  float* tidg = tar + W.ncoef;
  float* tailbuf = tidg + W.ncoef;
  for (int m = threadIdx.x; m <= nr; m += blockDim.x) fine_coef(W, m, az0[m], ar0[m]);
  for (int l = 0; l < W.nlev; ++l) {
    const float drl = (float)(W.dr * (double)(1 << l)), dzl = (float)(W.dz * (double)(1 << l));
    const int o = W.coef_off[l], lr = W.lnr[l];
    for (int m = threadIdx.x; m <= lr; m += blockDim.x) {
      const float az = m == 0    ? drl * drl / (8.0f * dzl)
                       : m == lr ? ((float)m - 0.25f) * drl * drl / (2.0f * dzl)
                                 : (float)m * drl * drl / dzl;
      const float arp = dzl * ((float)m + 0.5f);
      const float arm = m > 0 ? dzl * ((float)m - 0.5f) : 0.0f;
      taz[o + m] = az;
      tar[o + m] = arp;
      tidg[o + m] = 1.0f / (2.0f * az + arp + arm);
    }
  }
  __syncthreads();
  const Tables T{az0, ar0, taz, tar, tidg};

  int parity = 0;
  double vals[3];
  // ---- r = Q - A phi (Dirichlet values in phi), ||b||^2, ||r||^2 ------------
  double bb = 0.0, rr = 0.0;
  for (int it = gw; it < itemsT; it += ngw) {
    int m, n;
    if (!node_of(it, m, n)) continue;
    const int i = m * nz1 + n;
    double b = A.Q[i], a;
    if (interior(it)) {
      if (n == 1 && (!LINES || !field_free(m, 0, nr, nz, g0, wall))) b += az0[m] * phi[i - 1];
      if (n == nz - 1) b += az0[m] * phi[i + 1];
      if (m == nr - 1 && (!LINES || !wall)) b += ar0[m] * phi[i + nz1];
      a = apply64(T, phi, m, i, nz1);
    } else {
      a = line_apply64(T, phi, m, n, nr, nz, g0, wall, false, &b);
    }
    const double r = A.Q[i] - a;
    W.r[i] = r;
    bb += b * b;
    rr += r * r;
  }
  vals[0] = bb;
  vals[1] = rr;
  block_partials(W.partial, parity, 2, vals, lb, nb);
  if (!barrier_grid(W.bar, A.status, nb)) return;
  read_partials(W.partial, parity, 2, vals, nb);
  parity ^= 1;
  bb = vals[0];
  rr = vals[1];
  const double tol2bb = A.tol * A.tol * bb;
  // the preconditioner works on r scaled to O(1) (FP32 range), unscaled after
  const double ref = bb > 0.0 ? bb : rr;
  const double scale = ref > 0.0 ? 1.0 / sqrt(ref / (double)nfree) : 1.0;
  const double unscale = 1.0 / (2.0 * kPi * kEps0 * scale);
  const Lev L0 = lev(W, T, 0, W.u[0], W.f[0]);

  int it = 0;
  bool converged = rr <= tol2bb;
  double rz = 0.0, alpha = 0.0;
  bool first = true;
  int restarts = 0;
  if (!converged) {
    // f0 = scale r; the first red half sweep from u0 = 0 is u0 = f0 / diag
    for (int itm = gw; itm < itemsT; itm += ngw) {
      int m, n;
      if (!node_of(itm, m, n)) continue;
      const int i = m * nz1 + n;
      const float f = (float)(W.r[i] * scale);
      L0.f[i] = f;
      const float idg = interior(itm) ? L0.idg[m] : 1.0f / line_diag(L0, m, n);
      L0.u[i] = ((m + n) & 1) == 0 ? f * idg : 0.0f;
    }
    if (!barrier_grid(W.bar, A.status, nb)) return;
  }
  while (!converged && it < A.max_iter) {
    // ---- V-cycle, grid levels down (red of level 0 already done) -----------
    for (int l = 0; l < W.tail; ++l) {
      const Lev F = lev(W, T, l, W.u[l], W.f[l]);
      const Lev C = lev(W, T, l + 1, W.u[l + 1], W.f[l + 1]);
      if (l > 0) {
        smooth<LINES>(F, 0, gw, ngw, lane);
        if (!barrier_grid(W.bar, A.status, nb)) return;
      }
      smooth<LINES>(F, 1, gw, ngw, lane);
      if (!barrier_grid(W.bar, A.status, nb)) return;
      restrict_to<LINES>(F, C, gw, ngw, lane);
      if (!barrier_grid(W.bar, A.status, nb)) return;
    }
    if (lb == 0) vcycle_tail<LINES>(W, T, W.tail, tailbuf);
    if (!barrier_grid(W.bar, A.status, nb)) return;
    for (int l = W.tail - 1; l >= 0; --l) {
      const Lev F = lev(W, T, l, W.u[l], W.f[l]);
      const Lev C = lev(W, T, l + 1, W.u[l + 1], W.f[l + 1]);
      prolong_from<LINES>(F, C, gw, ngw, lane);
      if (!barrier_grid(W.bar, A.status, nb)) return;
      smooth<LINES>(F, 1, gw, ngw, lane);
      if (!barrier_grid(W.bar, A.status, nb)) return;
      smooth<LINES>(F, 0, gw, ngw, lane);
      if (!barrier_grid(W.bar, A.status, nb)) return;
    }
    // ---- z = M^{-1} r, r.z and z.q_old ------------------------------------
    double rz_loc = 0.0, zq_loc = 0.0;
    for (int itm = gw; itm < itemsT; itm += ngw) {
      int m, n;
      if (!node_of(itm, m, n)) continue;
      const int i = m * nz1 + n;
      const double zi = (double)L0.u[i] * unscale;
      W.z[i] = zi;
      rz_loc += W.r[i] * zi;
      if (!first) zq_loc += zi * W.q[i];
    }
    vals[0] = rz_loc;
    vals[1] = zq_loc;
    block_partials(W.partial, parity, 2, vals, lb, nb);
    if (!barrier_grid(W.bar, A.status, nb)) return;
    read_partials(W.partial, parity, 2, vals, nb);
    parity ^= 1;
    // ---- p = z + beta p, q = A z + beta q (flexible Polak-Ribiere beta) ---
    const double beta = first ? 0.0 : -alpha * vals[1] / rz;
    rz = vals[0];
    first = false;
    double pq = 0.0;
    for (int itm = gw; itm < itemsT; itm += ngw) {
      int m, n;
      if (!node_of(itm, m, n)) continue;
      const int i = m * nz1 + n;
      const double zi = W.z[i];
      double a;
      if (interior(itm)) {
        const double zl = (n > 1 || (LINES && m >= g0)) ? W.z[i - 1] : 0.0;
        const double zu = n < nz - 1 ? W.z[i + 1] : 0.0;
        const double zo = (m < nr - 1 || (LINES && wall)) ? W.z[i + nz1] : 0.0;
        a = az0[m] * (2.0 * zi - zl - zu) + ar0[m] * (zi - zo);
        if (m > 0) a += ar0[m - 1] * (zi - W.z[i - nz1]);
      } else {
        a = line_apply64(T, W.z, m, n, nr, nz, g0, wall, true, nullptr);
      }
      const double pi = zi + beta * W.p[i];
      const double qi = a + beta * W.q[i];
      W.p[i] = pi;
      W.q[i] = qi;
      pq += pi * qi;
    }
    vals[0] = pq;
    block_partials(W.partial, parity, 1, vals, lb, nb);
    if (!barrier_grid(W.bar, A.status, nb)) return;
    read_partials(W.partial, parity, 1, vals, nb);
    parity ^= 1;
    alpha = vals[0] != 0.0 ? rz / vals[0] : 0.0;
    // ---- phi += alpha p, r -= alpha q, next V-cycle's f0 and red sweep ----
    double rl = 0.0;
    for (int itm = gw; itm < itemsT; itm += ngw) {
      int m, n;
      if (!node_of(itm, m, n)) continue;
      const int i = m * nz1 + n;
      phi[i] += alpha * W.p[i];
      const double r = W.r[i] - alpha * W.q[i];
      W.r[i] = r;
      rl += r * r;
      const float f = (float)(r * scale);
      L0.f[i] = f;
      const float idg = interior(itm) ? L0.idg[m] : 1.0f / line_diag(L0, m, n);
      L0.u[i] = ((m + n) & 1) == 0 ? f * idg : 0.0f;
    }
    vals[0] = rl;
    block_partials(W.partial, parity, 1, vals, lb, nb);
    if (!barrier_grid(W.bar, A.status, nb)) return;
    read_partials(W.partial, parity, 1, vals, nb);
    parity ^= 1;
    rr = vals[0];
    ++it;
    if (rr <= tol2bb) {
      // confirm with the true residual b - A phi (also the restart's input)
      double rt = 0.0;
      for (int itm = gw; itm < itemsT; itm += ngw) {
        int m, n;
        if (!node_of(itm, m, n)) continue;
        const int i = m * nz1 + n;
        const double a = interior(itm)
                             ? apply64(T, phi, m, i, nz1)
                             : line_apply64(T, phi, m, n, nr, nz, g0, wall, false, nullptr);
        const double r = A.Q[i] - a;
        W.r[i] = r;
        rt += r * r;
        const float f = (float)(r * scale);
        L0.f[i] = f;
        const float idg = interior(itm) ? L0.idg[m] : 1.0f / line_diag(L0, m, n);
        L0.u[i] = ((m + n) & 1) == 0 ? f * idg : 0.0f;
      }
      vals[0] = rt;
      block_partials(W.partial, parity, 1, vals, lb, nb);
      if (!barrier_grid(W.bar, A.status, nb)) return;
      read_partials(W.partial, parity, 1, vals, nb);
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
  if (lb == 0 && threadIdx.x == 0) {
    *A.iters = it;
    *A.resid = bb > 0.0 ? sqrt(rr / bb) : sqrt(rr);
    if (!converged) atomicOr(A.status, ST_NONCONV);
  }
}

// ----------------------------------------------------------------------------
// Flexible PCG with the sine-transform preconditioner (all boundary nodes
// conductors).  z = M^{-1} r:
//   rows:    f_hat[m][k] = sum_n S[k][n] r[m][n]  (FP32)
//   columns: (lambda_k D + L) u_hat[:, k] = f_hat[:, k], Thomas in m
//   rows:    u[m][n] = sum_k S[n][k] u_hat[m][k];  z = u / (2 pi eps0) (FP64)
// lambda_k = 4 sin^2(pi (k+1) / (2 nz)).  The FP32 transform makes M^{-1} A
// the identity to about 1e-6, so the outer FP64 iteration ends after two or
// three iterations.
//
// Block b of a solve owns rows [b R, (b + 1) R) (R = rows_per_block) for
// everything but the column phase, so an iteration needs three grid barriers:
//   1. columns: the Thomas eliminations, 32 modes per block at a time, staged
//      in shared memory;
//   2. rows: u_hat -> z of the own rows and the two neighbour rows, A z, and
//      the row sums of r.z, z.q_old, z.Az;
//   3. rows: the coefficients from the row sums, p = z + beta p,
//      q = A z + beta q, phi += alpha p, r -= alpha q, the row sums of r.r,
//      and the next f_hat of the own rows.
// The first f_hat is computed with the initial residual, before the first
// barrier; the true-residual check at convergence transforms again only when
// the iteration restarts.
// p.q comes from the identity (z + beta p).A(z + beta p) = z.Az + 2 beta z.q +
// beta^2 p.q (A symmetric, q = A p).  Every dot product is summed per row by
// one warp (lanes over n, then a fixed shuffle tree) and over the rows in
// row order by every block, so phi does not depend on the number of blocks.
// ----------------------------------------------------------------------------
constexpr int kSepModes = 32;   // most modes per block in the column phase
enum { kRzSlot = 0, kZqSlot, kZazSlot, kRrSlot, kBbSlot, kRtSlot, kSepSlots };

// row sums of `nv` values, summed over rows in order (every thread gets the
// totals); the last slot's row r is at rows[slot * nr + r]
__device__ __forceinline__ void sum_rows(const double* rows, int nr, int slot0, int nv,
                                         double* out) {
  __shared__ double tot[4];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (w < nv) {
    const volatile double* p = rows + (size_t)(slot0 + w) * nr;
    double s = 0.0;
    for (int r = lane; r < nr; r += 32) s += p[r];
    s = warp_sum64(s);
    if (lane == 0) tot[w] = s;
  }
  __syncthreads();
  for (int j = 0; j < nv; ++j) out[j] = tot[j];
  __syncthreads();
}

// out(j, k, sum_n S[n][k] in[j][n]) for the block's rows j < nrow (in: FP32
// rows of nk values in shared memory), S read from global memory (L2
// resident, shared by every block) as float4 rows.  Thread t takes the four
// modes 4g..4g+3 (g = t mod ldS/4) of up to four rows over the part t div
// (ldS/4) of the n range; the parts' sums meet in `part` (shared memory,
// 16 blockDim.x floats), summed over the parts in a fixed order.
template <typename Out>
__device__ __forceinline__ void sep_transform(const PoissonWork& W, const float* in, int nrow,
                                              float* part, Out out) {
  const int nk = W.nk, ld = W.ldS, kg = ld >> 2;
  const int T = (int)blockDim.x;
  const int ns = T / kg;                              // parts of the n range (>= 1)
  const int g = (int)threadIdx.x % kg, pt = (int)threadIdx.x / kg;
  const int per = (nk + ns - 1) / ns;
  const int n0 = pt * per, n1 = min(nk, n0 + per);
  const float4* S4 = reinterpret_cast<const float4*>(W.sMat);
  for (int r0 = 0; r0 < nrow; r0 += 4) {
    const int nr4 = min(4, nrow - r0);
    if (pt < ns) {
      float acc[4][4];
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[j][c] = 0.0f;
      const float* row = in + (size_t)r0 * nk;
#pragma unroll 4
      for (int n = n0; n < n1; ++n) {
        const float4 sv = __ldg(S4 + (size_t)n * kg + g);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (j < nr4) {
            const float a = row[j * nk + n];
            acc[j][0] = fmaf(a, sv.x, acc[j][0]);
            acc[j][1] = fmaf(a, sv.y, acc[j][1]);
            acc[j][2] = fmaf(a, sv.z, acc[j][2]);
            acc[j][3] = fmaf(a, sv.w, acc[j][3]);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j)
        *reinterpret_cast<float4*>(part + (size_t)(pt * 4 + j) * ld + 4 * g) =
            make_float4(acc[j][0], acc[j][1], acc[j][2], acc[j][3]);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nr4 * ld; t += T) {
      const int j = t / ld, k = t - j * ld;
      if (k < nk) {
        float v = 0.0f;
        for (int q = 0; q < ns; ++q) v += part[(size_t)(q * 4 + j) * ld + k];
        out(r0 + j, k, v);
      }
    }
    __syncthreads();
  }
}

// Thomas eliminations of the block's modes in shared memory: the nk modes
// are spread evenly over the nb blocks (mpb = ceil(nk / nb) <= kSepModes per
// block, so every block works), h, w, c staged column-wise (mpb per row); one
// thread per mode runs the forward sweep and the back substitution, then the
// block writes u_hat back.
__device__ void sep_columns(const PoissonWork& W, int lb, int nb, float* sm) {
  const int nk = W.nk, nr = W.nr;
  int mpb = (nk + nb - 1) / nb;
  if (mpb > kSepModes) mpb = kSepModes;
  float* h = sm;
  float* w = h + (size_t)nr * mpb;
  float* c = w + (size_t)nr * mpb;
  float* e = c + (size_t)nr * mpb;   // e[m] = a_r(m - 1) (e[0] = 0)
  for (int m = threadIdx.x; m < nr; m += blockDim.x) e[m] = m > 0 ? W.sE[m - 1] : 0.0f;
  for (int k0 = lb * mpb; k0 < nk; k0 += nb * mpb) {
    const int nm = nk - k0 < mpb ? nk - k0 : mpb;
    for (int t = threadIdx.x; t < nr * mpb; t += blockDim.x) {
      const int m = t / mpb, j = t - m * mpb;
      if (j < nm) {
        const size_t g = (size_t)m * nk + k0 + j;
        h[t] = W.sHat[g];
        w[t] = W.sW[g];
        c[t] = W.sC[g];
      }
    }
    __syncthreads();
    if ((int)threadIdx.x < nm) {
      const int j = threadIdx.x;
      // y_m = (f_m + e_m y_{m-1}) / pivot_m  (off-diagonals -e), eight rows of
      // operands loaded ahead of the recurrence
      float y = 0.0f;
      int m = 0;
      for (; m + 7 < nr; m += 8) {
        float hv[8], wv[8], ev[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          hv[u] = h[(m + u) * mpb + j];
          wv[u] = w[(m + u) * mpb + j];
          ev[u] = e[m + u];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          y = (hv[u] + ev[u] * y) * wv[u];
          h[(m + u) * mpb + j] = y;
        }
      }
      for (; m < nr; ++m) {
        y = (h[m * mpb + j] + e[m] * y) * w[m * mpb + j];
        h[m * mpb + j] = y;
      }
      // x_m = y_m + c_m x_{m+1}
      float x = 0.0f;
      m = nr - 1;
      for (; m - 7 >= 0; m -= 8) {
        float hv[8], cv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          hv[u] = h[(m - u) * mpb + j];
          cv[u] = c[(m - u) * mpb + j];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          x = fmaf(cv[u], x, hv[u]);
          h[(m - u) * mpb + j] = x;
        }
      }
      for (; m >= 0; --m) {
        x = fmaf(c[m * mpb + j], x, h[m * mpb + j]);
        h[m * mpb + j] = x;
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nr * mpb; t += blockDim.x) {
      const int m = t / mpb, j = t - m * mpb;
      if (j < nm) W.sHat[(size_t)m * nk + k0 + j] = h[t];
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kPoisThreads) k_poisson_sep(PoissonArgs A0,
                                                              const PoissonArgs* group, int bpi) {
  __shared__ PoissonArgs sA;
  int lb, nb;
  {
    const PoissonArgs* src = &A0;
    if (group) {
      const int inst = blockIdx.x / bpi;
      lb = blockIdx.x - inst * bpi;
      nb = bpi;
      src = group + inst;
    } else {
      lb = blockIdx.x;
      nb = gridDim.x;
    }
    const unsigned* s4 = reinterpret_cast<const unsigned*>(src);
    unsigned* d4 = reinterpret_cast<unsigned*>(&sA);
    for (int k = threadIdx.x; k < (int)(sizeof(PoissonArgs) / 4); k += blockDim.x) d4[k] = s4[k];
    __syncthreads();
  }
  const PoissonArgs& A = sA;
  const PoissonWork& W = A.W;
  if (*(volatile int*)A.status & (ST_FATAL)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int nr = W.nr, nz = W.nz, nz1 = nz + 1, nk = W.nk;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const long long nfree = (long long)nr * (nz - 1);
  double* phi = A.phi;
  double* rows = W.partial;     // kSepSlots x nr row sums
  double* az0 = (double*)smem;
  double* ar0 = az0 + (nr + 1);
  unsigned char* work = (unsigned char*)(ar0 + (nr + 1));
  for (int m = threadIdx.x; m <= nr; m += blockDim.x) fine_coef(W, m, az0[m], ar0[m]);
  __syncthreads();
  const Tables T{az0, ar0, nullptr, nullptr, nullptr};
  const int R = W.rows_per_block;
  const int m0 = lb * R;
  const int nrow = m0 >= nr ? 0 : (m0 + R <= nr ? R : nr - m0);
  // shared layout of the row phases: z of rows m0 - 1 .. m0 + R (FP64), A z
  // of the own rows (FP64), f or u_hat rows (FP32), the transform's partial
  // sums (16 blockDim.x floats); the column phase reuses the same memory
  double* zs = (double*)work;
  double* azs = zs + (size_t)(R + 2) * nk;
  float* fs = (float*)(azs + (size_t)R * nk);
  float* tpart = (float*)(((uintptr_t)(fs + (size_t)(R + 2) * nk) + 15) & ~(uintptr_t)15);

  // f_hat of the own rows from W.r.  The transform solve is linear and its
  // values (charges of 1e-20 .. 1e-8 C over couplings of ~1e-4 m) sit many
  // decades inside FP32's normal range, so r enters unscaled
  const double unscale = 1.0 / (2.0 * kPi * kEps0);
  auto forward_own = [&]() {
    for (int t = threadIdx.x; t < nrow * nk; t += blockDim.x) {
      const int j = t / nk, n = t - j * nk;
      fs[t] = (float)W.r[(m0 + j) * nz1 + 1 + n];
    }
    __syncthreads();
    if (nrow > 0) {
      float* hat = W.sHat + (size_t)m0 * nk;
      sep_transform(W, fs, nrow, tpart, [&](int j, int k, float v) { hat[(size_t)j * nk + k] = v; });
    }
  };

  // ---- r = Q - A phi (Dirichlet values in phi), row sums of b.b and r.r,
  //      and the first f_hat ------------------------------------------------
  for (int j = wid; j < nrow; j += nw) {
    const int m = m0 + j;
    double bb = 0.0, rr = 0.0;
    for (int n = 1 + lane; n <= nz - 1; n += 32) {
      const int i = m * nz1 + n;
      double b = A.Q[i];
      if (n == 1) b += az0[m] * phi[i - 1];
      if (n == nz - 1) b += az0[m] * phi[i + 1];
      if (m == nr - 1) b += ar0[m] * phi[i + nz1];
      const double r = A.Q[i] - apply64(T, phi, m, i, nz1);
      W.r[i] = r;
      bb += b * b;
      rr += r * r;
    }
    bb = warp_sum64(bb);
    rr = warp_sum64(rr);
    if (lane == 0) {
      rows[kBbSlot * nr + m] = bb;
      rows[kRrSlot * nr + m] = rr;
    }
  }
  __syncthreads();
  forward_own();
  if (!barrier_grid(W.bar, A.status, nb)) return;
  double tot[4];
  sum_rows(rows, nr, kRrSlot, 2, tot);   // slots kRrSlot, kBbSlot
  double rr = tot[0];
  const double bb = tot[1];
  const double tol2bb = A.tol * A.tol * bb;

  int it = 0;
  bool converged = rr <= tol2bb;
  double rz_old = 0.0, alpha = 0.0, pq_old = 0.0;
  bool first = true;
  int restarts = 0;
  while (!converged && it < A.max_iter) {
    // ---- 1. columns ---------------------------------------------------------
    sep_columns(W, lb, nb, (float*)work);
    if (!barrier_grid(W.bar, A.status, nb)) return;
    // ---- 2. rows: z (own rows and neighbours), A z, row sums ---------------
    if (nrow > 0) {
      const int ja = m0 > 0 ? 0 : 1;                          // first staged row (m0 - 1)
      const int jb = m0 + nrow < nr ? nrow + 2 : nrow + 1;    // past the last (m0 + nrow)
      for (int t = threadIdx.x; t < (jb - ja) * nk; t += blockDim.x) {
        const int j = ja + t / nk, k = t - (t / nk) * nk;
        fs[j * nk + k] = W.sHat[(size_t)(m0 - 1 + j) * nk + k];
      }
      __syncthreads();
      // u rows: zs[j][n] = unscale sum_k S[n][k] u_hat[j][k] (S symmetric)
      sep_transform(W, fs + ja * nk, jb - ja, tpart, [&](int j, int n, float v) {
        zs[(size_t)(ja + j) * nk + n] = (double)v * unscale;
      });
      __syncthreads();
      for (int j = wid; j < nrow; j += nw) {
        const int m = m0 + j;
        const double* zr = zs + (size_t)(j + 1) * nk;
        double rz = 0.0, zq = 0.0, zaz = 0.0;
        for (int n = lane; n < nk; n += 32) {
          const int i = m * nz1 + 1 + n;
          const double zi = zr[n];
          const double zl = n > 0 ? zr[n - 1] : 0.0;
          const double zu = n < nk - 1 ? zr[n + 1] : 0.0;
          const double zo = m < nr - 1 ? zr[n + nk] : 0.0;
          double a = az0[m] * (2.0 * zi - zl - zu) + ar0[m] * (zi - zo);
          if (m > 0) a += ar0[m - 1] * (zi - zr[n - nk]);
          azs[(size_t)j * nk + n] = a;
          rz += W.r[i] * zi;
          if (!first) zq += zi * W.q[i];
          zaz += zi * a;
        }
        rz = warp_sum64(rz);
        zq = warp_sum64(zq);
        zaz = warp_sum64(zaz);
        if (lane == 0) {
          rows[kRzSlot * nr + m] = rz;
          rows[kZqSlot * nr + m] = zq;
          rows[kZazSlot * nr + m] = zaz;
        }
      }
    }
    if (!barrier_grid(W.bar, A.status, nb)) return;
    // ---- 3. rows: coefficients, p, q, phi, r, next f_hat -------------------
    sum_rows(rows, nr, kRzSlot, 3, tot);
    const double rz = tot[0], zq = tot[1], zaz = tot[2];
    // flexible (Polak-Ribiere) beta = -alpha z.q_old / r.z_old
    const double beta = first ? 0.0 : -alpha * zq / rz_old;
    const double pq = first ? zaz : zaz + 2.0 * beta * zq + beta * beta * pq_old;
    alpha = pq != 0.0 ? rz / pq : 0.0;
    rz_old = rz;
    pq_old = pq;
    for (int j = wid; j < nrow; j += nw) {
      const int m = m0 + j;
      double rl = 0.0;
      for (int n = lane; n < nk; n += 32) {
        const int i = m * nz1 + 1 + n;
        const double pi = zs[(size_t)(j + 1) * nk + n] + (first ? 0.0 : beta * W.p[i]);
        const double qi = azs[(size_t)j * nk + n] + (first ? 0.0 : beta * W.q[i]);
        W.p[i] = pi;
        W.q[i] = qi;
        phi[i] += alpha * pi;
        const double r = W.r[i] - alpha * qi;
        W.r[i] = r;
        rl += r * r;
      }
      rl = warp_sum64(rl);
      if (lane == 0) rows[kRrSlot * nr + m] = rl;
    }
    first = false;
    __syncthreads();
    forward_own();
    if (!barrier_grid(W.bar, A.status, nb)) return;
    sum_rows(rows, nr, kRrSlot, 1, tot);
    rr = tot[0];
    ++it;
    if (rr <= tol2bb) {
      // confirm with the true residual b - A phi (also the restart's input)
      for (int j = wid; j < nrow; j += nw) {
        const int m = m0 + j;
        double rt = 0.0;
        for (int n = 1 + lane; n <= nz - 1; n += 32) {
          const int i = m * nz1 + n;
          const double r = A.Q[i] - apply64(T, phi, m, i, nz1);
          W.r[i] = r;
          rt += r * r;
        }
        rt = warp_sum64(rt);
        if (lane == 0) rows[kRtSlot * nr + m] = rt;
      }
      if (!barrier_grid(W.bar, A.status, nb)) return;
      sum_rows(rows, nr, kRtSlot, 1, tot);
      rr = tot[0];
      if (rr <= tol2bb || restarts >= 3) {
        converged = rr <= tol2bb;
        break;
      }
      ++restarts;
      first = true;  // restart the Krylov space from the true residual
      forward_own();
      if (!barrier_grid(W.bar, A.status, nb)) return;
    }
  }
  if (lb == 0 && threadIdx.x == 0) {
    *A.iters = it;
    *A.resid = bb > 0.0 ? sqrt(rr / bb) : sqrt(rr);
    if (!converged) atomicOr(A.status, ST_NONCONV);
  }
}

// ----------------------------------------------------------------------------
// Pieces of the learned warm start, on the fine FP64 operator of the solve.
// Start selection among three starting points -- x = phi as it stands (the
// previous solution with this step's Dirichlet values), x = the candidate from
// the network, x = 0 -- all with the Dirichlet values of phi on the boundary:
// the smallest score (below) wins, ties keep the earlier candidate, and the
// winner is copied into phi's free nodes.
// ----------------------------------------------------------------------------
__device__ __forceinline__ bool free_node(const PoissonWork& W, int m, int n) {
  return field_free(m, n, W.nr, W.nz, W.bc_g[0], W.bc_wall);
}

// couplings of fine node (m, n) to (m-1, n), (m+1, n), (m, n-1), (m, n+1);
// 0 for neighbours outside the grid, r-couplings halved on row 0
__device__ __forceinline__ void node_coup(const PoissonWork& W, int m, int n, double c[4]) {
  double az, ar, azm, arm = 0.0;
  fine_coef(W, m, az, ar);
  if (m > 0) fine_coef(W, m - 1, azm, arm);
  const double h = n == 0 ? 0.5 : 1.0;
  c[0] = m > 0 ? h * arm : 0.0;
  c[1] = m < W.nr ? h * ar : 0.0;
  c[2] = n > 0 ? az : 0.0;
  c[3] = n < W.nz ? az : 0.0;
}

__device__ __forceinline__ double start_value(int k, const double* phi, const double* cand,
                                              bool fr, int i) {
  if (k == 0 || !fr) return phi[i];
  return k == 1 ? cand[i] : 0.0;
}

// The warm-start pieces run over all instances of a handle at once:
// blockIdx.y = instance k, its operator, Q and phi from A[k] (the device
// PoissonArgs of the grouped solve), its node fields at offset k * stride of
// the per-instance buffers.

// Score of a start: ||Q - A x||_2^2 over the free nodes; partial[k][j][b]
// for start j of instance k from block b.
__global__ void __launch_bounds__(256) k_guess_norms(const PoissonArgs* A, const double* cand_all,
                                                     long long stride, double* partial) {
  __shared__ double red[3][8];
  const int k = blockIdx.y;
  const PoissonWork& W = A[k].W;
  const double* Q = A[k].Q;
  const double* phi = A[k].phi;
  const double* cand = cand_all + k * stride;
  const int nr = W.nr, nz = W.nz, nz1 = nz + 1;
  const long long nn = (long long)(nr + 1) * nz1;
  const int dm[4] = {-1, 1, 0, 0}, dn[4] = {0, 0, -1, 1};
  double loc[3] = {0.0, 0.0, 0.0};
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nn;
       e += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(e / nz1), n = (int)(e - (long long)m * nz1);
    if (!free_node(W, m, n)) continue;
    const int i = (int)e;
    double c[4];
    node_coup(W, m, n, c);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const double xi = start_value(j, phi, cand, true, i);
      double a = 0.0;
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        if (c[d] == 0.0) continue;
        const int mm = m + dm[d], nn2 = n + dn[d];
        a += c[d] * (xi - start_value(j, phi, cand, free_node(W, mm, nn2), mm * nz1 + nn2));
      }
      const double r = Q[i] - a;
      loc[j] += r * r;
    }
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const double s = warp_sum64(loc[j]);
    if (lane == 0) red[j][w] = s;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double s = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[threadIdx.x][q];
    partial[((long long)k * 3 + threadIdx.x) * gridDim.x + blockIdx.x] = s;
  }
}

// one block per instance: the start with the smallest score (block-ordered
// sums); counts summed over the instances, ud->choice = the last instance's
__global__ void k_guess_pick(const PoissonArgs* A, const double* partial, int nblk, UDev* ud,
                             int* choice) {
  __shared__ double tot[3];
  const int k = blockIdx.x;
  if (threadIdx.x < 3) {
    double s = 0.0;
    const double* p = partial + ((long long)k * 3 + threadIdx.x) * nblk;
    for (int b = 0; b < nblk; ++b) s += p[b];
    tot[threadIdx.x] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int best = 0;
    if (!(*A[k].status & ST_FATAL)) {
      for (int j = 1; j < 3; ++j)
        if (tot[j] < tot[best]) best = j;   // NaN norms never win
      atomicAdd((unsigned long long*)&ud->n_choice[best], 1ULL);
    }
    choice[k] = best;
    if (k == (int)gridDim.x - 1) ud->choice = best;
  }
}

__global__ void k_guess_apply(const PoissonArgs* A, const double* cand_all, long long stride,
                              const int* choice) {
  const int k = blockIdx.y;
  const int c = choice[k];
  if (c == 0) return;
  const PoissonWork& W = A[k].W;
  double* phi = A[k].phi;
  const double* cand = cand_all + k * stride;
  const int nz1 = W.nz + 1;
  const long long nn = (long long)(W.nr + 1) * nz1;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nn;
       e += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(e / nz1), n = (int)(e - (long long)m * nz1);
    if (free_node(W, m, n)) phi[e] = c == 1 ? cand[e] : 0.0;
  }
}

// res = Q - A phi on free nodes, 0 on Dirichlet nodes
__global__ void k_residual32(const PoissonArgs* A, float* res_all, long long stride) {
  const int k = blockIdx.y;
  const PoissonWork& W = A[k].W;
  const double* Q = A[k].Q;
  const double* phi = A[k].phi;
  float* res = res_all + k * stride;
  const int nr = W.nr, nz = W.nz, nz1 = nz + 1;
  const long long nn = (long long)(nr + 1) * nz1;
  const int off[4] = {-nz1, nz1, -1, 1};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nn;
       i += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(i / nz1), n = (int)(i - (long long)m * nz1);
    if (!free_node(W, m, n)) {
      res[i] = 0.0f;
      continue;
    }
    double c[4];
    node_coup(W, m, n, c);
    double a = 0.0;
#pragma unroll
    for (int d = 0; d < 4; ++d)
      if (c[d] != 0.0) a += c[d] * (phi[i] - phi[i + off[d]]);
    res[i] = (float)(Q[i] - a);
  }
}

// one colour of a red-black Gauss-Seidel sweep on A x = Q
__global__ void k_gs_color(const PoissonArgs* A, double* x_all, long long stride, int color) {
  const int k = blockIdx.y;
  const PoissonWork& W = A[k].W;
  const double* Q = A[k].Q;
  double* x = x_all + k * stride;
  const int nr = W.nr, nz = W.nz, nz1 = nz + 1;
  const long long nn = (long long)(nr + 1) * nz1;
  const int off[4] = {-nz1, nz1, -1, 1};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nn;
       i += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(i / nz1), n = (int)(i - (long long)m * nz1);
    if (((m + n) & 1) != color || !free_node(W, m, n)) continue;
    double c[4];
    node_coup(W, m, n, c);
    double s = Q[i], d = 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (c[q] != 0.0) {
        s += c[q] * x[i + off[q]];
        d += c[q];
      }
    x[i] = s / d;
  }
}

int guess_blocks(int nr, int nz) {
  const long long nn = (long long)(nr + 1) * (nz + 1);
  long long b = (nn + 255) / 256;
  if (b > 592) b = 592;
  if (b < 1) b = 1;
  return (int)b;
}

cudaError_t launch_residual32(const void* pargs, int n, int nr, int nz, float* res,
                              cudaStream_t st) {
  const long long nn = (long long)(nr + 1) * (nz + 1);
  k_residual32<<<dim3(guess_blocks(nr, nz), n), 256, 0, st>>>((const PoissonArgs*)pargs, res, nn);
  return cudaGetLastError();
}

cudaError_t launch_gs_sweeps(const void* pargs, int n, int nr, int nz, double* x, int sweeps,
                             cudaStream_t st) {
  const long long nn = (long long)(nr + 1) * (nz + 1);
  const dim3 grid(guess_blocks(nr, nz), n);
  for (int s = 0; s < sweeps; ++s) {
    k_gs_color<<<grid, 256, 0, st>>>((const PoissonArgs*)pargs, x, nn, 0);
    k_gs_color<<<grid, 256, 0, st>>>((const PoissonArgs*)pargs, x, nn, 1);
  }
  return cudaGetLastError();
}

cudaError_t launch_guess_select(const void* pargs, int n, int nr, int nz, const double* cand,
                                double* partial, UDev* ud, int* choice, cudaStream_t st) {
  const long long nn = (long long)(nr + 1) * (nz + 1);
  const int nblk = guess_blocks(nr, nz);
  const PoissonArgs* A = (const PoissonArgs*)pargs;
  k_guess_norms<<<dim3(nblk, n), 256, 0, st>>>(A, cand, nn, partial);
  k_guess_pick<<<n, 32, 0, st>>>(A, partial, nblk, ud, choice);
  k_guess_apply<<<dim3(nblk, n), 256, 0, st>>>(A, cand, nn, choice);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// host side
// ----------------------------------------------------------------------------
// the kernel variant of a problem: with insulating boundary nodes or without
static bool has_lines(const PoissonWork& w) {
  return line_count(w.nr, w.nz, w.bc_g[0], w.bc_wall) > 0;
}

static const void* poisson_kernel(bool lines) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_poisson<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kSmemBudget);
    cudaFuncSetAttribute(k_poisson<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kSmemBudget);
    attr_set = true;
  }
  return lines ? (const void*)k_poisson<true> : (const void*)k_poisson<false>;
}

static int poisson_blocks(const PoissonWork& w, int num_sms) {
  const void* kern = poisson_kernel(has_lines(w));
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPoisThreads, w.smem_bytes);
  if (per_sm < 1) per_sm = 1;
  // about one row segment per warp, at most one wave
  const long long items = (long long)w.nr * ((w.nz - 1 + 31) / 32);
  long long want = (items + kPoisThreads / 32 - 1) / (kPoisThreads / 32);
  long long cap = (long long)num_sms * per_sm;
  if (cap > 2048) cap = 2048;
  if (want > cap) want = cap;
  if (want < 1) want = 1;
  return (int)want;
}

PoissonWork* poisson_work_init(void* base, int nr, int nz, double R, double L, int g, int wall,
                               int num_sms) {
  PoissonWork* pw = new PoissonWork();
  layout(*pw, base, nr, nz, R, L, g, wall);
  pw->nblocks = poisson_blocks(*pw, num_sms);
  return pw;
}

// ---- sine-transform preconditioner ------------------------------------------
constexpr int kSepMaxBlocks = 256;

static int sep_smem(const PoissonWork& w);

// row stride of the transform matrix (float4 rows)
static int sep_ld(int nk) { return (nk + 3) & ~3; }

// every boundary node a conductor, the column phase's staging of
// kSepModes columns fits in shared memory, and a block's threads cover the
// transform's float4 columns
bool poisson_sep_possible(const PoissonWork* pw) {
  if (has_lines(*pw) || pw->nz < 3) return false;
  PoissonWork w = *pw;
  w.nk = w.nz - 1;
  w.ldS = sep_ld(w.nk);
  if (w.ldS / 4 > kPoisThreads) return false;
  w.rows_per_block = 1;
  return sep_smem(w) <= (int)kSmemBudget;
}

size_t poisson_sep_bytes(int nr, int nz) {
  const size_t nk = (size_t)(nz - 1);
  return round256(nk * (size_t)sep_ld((int)nk) * 4) + 3 * round256((size_t)nr * nk * 4) +
         round256((size_t)nr * 4);
}

static void sep_rows_per_block(PoissonWork& w, int blocks) {
  if (blocks < 1) blocks = 1;
  w.rows_per_block = (w.nr + blocks - 1) / blocks;
}

static int sep_smem(const PoissonWork& w) {
  const size_t R = (size_t)w.rows_per_block, nk = (size_t)w.nk;
  const size_t rows = (R + 2) * nk * 8 + R * nk * 8 + (R + 2) * nk * 4 + 16 +
                      (size_t)16 * kPoisThreads * 4;
  const size_t cols = (3 * (size_t)w.nr * kSepModes + (size_t)w.nr) * 4;
  return (int)(2 * (size_t)(w.nr + 1) * sizeof(double) + (rows > cols ? rows : cols));
}

cudaError_t poisson_sep_attach(PoissonWork* pw, void* base, int num_sms, cudaStream_t st) {
  PoissonWork& w = *pw;
  const int nr = w.nr, nk = w.nz - 1;
  w.nk = nk;
  char* p = (char*)base;
  auto take = [&](size_t b) {
    char* q = p;
    p += round256(b);
    return (float*)q;
  };
  w.ldS = sep_ld(nk);
  w.sMat = take((size_t)nk * w.ldS * 4);
  w.sW = take((size_t)nr * nk * 4);
  w.sC = take((size_t)nr * nk * 4);
  w.sHat = take((size_t)nr * nk * 4);
  w.sE = take((size_t)nr * 4);
  // tables in FP64 on the host, stored in FP32; couplings scaled by
  // 1 / (2 pi eps0) like the multigrid tables
  std::vector<float> S((size_t)nk * w.ldS, 0.0f), Wt((size_t)nr * nk), Ct((size_t)nr * nk), E(nr);
  const double norm = std::sqrt(2.0 / w.nz);
  for (int n = 0; n < nk; ++n)
    for (int k = 0; k < nk; ++k) {
      const long long a = (long long)(n + 1) * (k + 1) % (2LL * w.nz);   // exact argument
      S[(size_t)n * w.ldS + k] = (float)(norm * std::sin(kPi * (double)a / w.nz));
    }
  std::vector<double> az(nr), ar(nr);
  for (int m = 0; m < nr; ++m) {
    az[m] = m == 0 ? w.dr * w.dr / (8.0 * w.dz) : m * w.dr * w.dr / w.dz;
    ar[m] = w.dz * (m + 0.5);
    E[m] = (float)ar[m];
  }
  for (int k = 0; k < nk; ++k) {
    const double sk = std::sin(kPi * (k + 1) / (2.0 * w.nz));
    const double lam = 4.0 * sk * sk;
    double cprev = 0.0;   // c'_{m-1} = -ar(m-1) / pivot_{m-1}
    for (int m = 0; m < nr; ++m) {
      const double d = lam * az[m] + ar[m] + (m > 0 ? ar[m - 1] : 0.0);
      const double piv = d - (m > 0 ? -ar[m - 1] * cprev : 0.0);
      const double cm = m < nr - 1 ? -ar[m] / piv : 0.0;
      Wt[(size_t)m * nk + k] = (float)(1.0 / piv);
      Ct[(size_t)m * nk + k] = (float)(-cm);
      cprev = cm;
    }
  }
  cudaError_t e = cudaMemcpyAsync(w.sMat, S.data(), S.size() * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(w.sW, Wt.data(), Wt.size() * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(w.sC, Ct.data(), Ct.size() * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(w.sE, E.data(), E.size() * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // host tables go out of scope
  if (e != cudaSuccess) return e;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_poisson_sep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kSmemBudget);
    attr = true;
  }
  int blocks = nr / 2 < kSepMaxBlocks ? nr / 2 : kSepMaxBlocks;
  if (blocks > num_sms) blocks = num_sms;
  sep_rows_per_block(w, blocks);
  w.sep_blocks = (nr + w.rows_per_block - 1) / w.rows_per_block;
  return cudaSuccess;
}

void poisson_work_free(PoissonWork* pw) { delete pw; }

cudaError_t launch_poisson(PoissonWork* pw, const double* Q, double* phi, double tol, int max_iter,
                           int* status_dev, int* iters_dev, double* resid_dev, cudaStream_t st) {
  if (pw->sMat) {
    PoissonArgs a;
    a.W = *pw;
    a.Q = Q;
    a.phi = phi;
    a.tol = tol;
    a.max_iter = max_iter;
    a.status = status_dev;
    a.iters = iters_dev;
    a.resid = resid_dev;
    const PoissonArgs* none = nullptr;
    int one = 1;
    void* args[] = {&a, &none, &one};
    return cudaLaunchCooperativeKernel((const void*)k_poisson_sep, dim3(pw->sep_blocks),
                                       dim3(kPoisThreads), args, (size_t)sep_smem(*pw), st);
  }
  PoissonArgs a;
  a.W = *pw;
  a.Q = Q;
  a.phi = phi;
  a.tol = tol;
  a.max_iter = max_iter;
  a.status = status_dev;
  a.iters = iters_dev;
  a.resid = resid_dev;
  const PoissonArgs* none = nullptr;
  int one = 1;
  void* args[] = {&a, &none, &one};
  return cudaLaunchCooperativeKernel(poisson_kernel(has_lines(*pw)), dim3(pw->nblocks),
                                     dim3(kPoisThreads), args, (size_t)pw->smem_bytes, st);
}

size_t poisson_args_bytes() { return sizeof(PoissonArgs); }

// Argument records of the grouped launch, written once (the pointers they hold
// do not change over a handle's life) to d_args: n_inst * poisson_args_bytes().
static bool group_sep(PoissonWork* const* pws, int n_inst) {
  for (int k = 0; k < n_inst; ++k)
    if (!pws[k]->sMat) return false;
  return true;
}

// dynamic shared memory of the grouped sine-transform solve with bpi blocks
// per instance
static int group_sep_smem(PoissonWork* const* pws, int n_inst, int bpi) {
  int smem = 0;
  for (int k = 0; k < n_inst; ++k) {
    PoissonWork w = *pws[k];
    sep_rows_per_block(w, bpi);
    smem = sep_smem(w) > smem ? sep_smem(w) : smem;
  }
  return smem;
}

// blocks per instance of the grouped sine-transform solve: the most (up to
// each instance's own count) for which every block of the launch is resident
static int group_sep_bpi(PoissonWork* const* pws, int n_inst, int num_sms) {
  int want = 1;
  for (int k = 0; k < n_inst; ++k) want = pws[k]->sep_blocks > want ? pws[k]->sep_blocks : want;
  for (int bpi = want; bpi >= 1; --bpi) {
    const int smem = group_sep_smem(pws, n_inst, bpi);
    if (smem > (int)kSmemBudget) return 0;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k_poisson_sep,
                                                  kPoisThreads, smem);
    if ((long long)bpi * n_inst <= (long long)num_sms * per_sm) return bpi;
  }
  return 0;
}

cudaError_t poisson_group_upload(PoissonWork* const* pws, const Inst* insts, int n_inst,
                                 void* d_args, int num_sms, cudaStream_t st) {
  std::vector<PoissonArgs> host((size_t)n_inst);
  const int bpi = group_sep(pws, n_inst) ? group_sep_bpi(pws, n_inst, num_sms) : 0;
  const bool sep = bpi > 0;   // else the multigrid kernel serves the group
  for (int k = 0; k < n_inst; ++k) {
    PoissonArgs& a = host[k];
    std::memset(&a, 0, sizeof(a));
    a.W = *pws[k];
    if (sep) sep_rows_per_block(a.W, bpi);
    a.Q = insts[k].Q;
    a.phi = insts[k].phi;
    a.tol = insts[k].poisson_tol;
    a.max_iter = insts[k].poisson_max_iter;
    a.status = &insts[k].S->status;
    a.iters = &insts[k].S->poisson_iters;
    a.resid = &insts[k].S->poisson_resid;
  }
  cudaError_t e = cudaMemcpyAsync(d_args, host.data(), host.size() * sizeof(PoissonArgs),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

// All instances' solves in one cooperative launch, bpi blocks per instance.
cudaError_t launch_poisson_group(PoissonWork* const* pws, const Inst* insts, int n_inst,
                                 void* d_args, int num_sms, cudaStream_t st) {
  (void)insts;
  int bpi = group_sep(pws, n_inst) ? group_sep_bpi(pws, n_inst, num_sms) : 0;
  if (bpi > 0) {
    const int smem = group_sep_smem(pws, n_inst, bpi);
    PoissonArgs a0;
    std::memset(&a0, 0, sizeof(a0));
    const PoissonArgs* g = (const PoissonArgs*)d_args;
    void* args[] = {&a0, &g, &bpi};
    return cudaLaunchCooperativeKernel((const void*)k_poisson_sep, dim3(n_inst * bpi),
                                       dim3(kPoisThreads), args, (size_t)smem, st);
  }
  int smem = 0, want = 1;
  bool lines = false;
  for (int k = 0; k < n_inst; ++k) {
    smem = pws[k]->smem_bytes > smem ? pws[k]->smem_bytes : smem;
    want = pws[k]->nblocks > want ? pws[k]->nblocks : want;
    lines = lines || has_lines(*pws[k]);
  }
  const void* kern = poisson_kernel(lines);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPoisThreads, smem);
  if (per_sm < 1) per_sm = 1;
  bpi = (num_sms * per_sm) / n_inst;
  if (bpi > want) bpi = want;
  if (bpi < 1) return cudaErrorInvalidConfiguration;
  PoissonArgs a0;
  std::memset(&a0, 0, sizeof(a0));
  const PoissonArgs* g = (const PoissonArgs*)d_args;
  void* args[] = {&a0, &g, &bpi};
  return cudaLaunchCooperativeKernel(kern, dim3(n_inst * bpi), dim3(kPoisThreads),
                                     args, (size_t)smem, st);
}

// ----------------------------------------------------------------------------
// Variant for pic_poisson_solve_static: the workspace layout is built in a
// struct on the host stack (no host or device allocation), over the caller's
// scratch at `base`.  The layout is the one poisson_work_bytes() sizes.
// ----------------------------------------------------------------------------
cudaError_t launch_poisson_in_place(void* base, int nr, int nz, double R, double L, int g, int wall,
                                    int num_sms, const double* Q, double* phi, double tol,
                                    int max_iter, int* status_dev, int* iters_dev,
                                    double* resid_dev, cudaStream_t st) {
  PoissonWork w;
  layout(w, base, nr, nz, R, L, g, wall);
  w.nblocks = poisson_blocks(w, num_sms);
  return launch_poisson(&w, Q, phi, tol, max_iter, status_dev, iters_dev, resid_dev, st);
}

}  // namespace pic
