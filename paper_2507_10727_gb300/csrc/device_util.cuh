// device_util.cuh -- small device helpers shared by the FP64 and FP32 step kernels.
#pragma once

#include "common.cuh"

namespace pic {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum of v added atomically to *dst (used for diagnostics only)
static __device__ void block_add(double v, double* dst) {
  __shared__ double red[32];
  v = warp_sum(v);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    int nw = (blockDim.x + 31) >> 5;
    double s = lane < nw ? red[lane] : 0.0;
    s = warp_sum(s);
    if (lane == 0 && s != 0.0) atomicAdd(dst, s);
  }
  __syncthreads();
}

// new direction: e rotated by polar angle chi (cos given) and azimuth phi,
// in the frame (u, w) built from the coordinate axis of e's smallest component
static __device__ __forceinline__ void scatter_dir(const double e[3], double cos_chi, double phi,
                                            double out[3]) {
  int a = 0;
  if (fabs(e[1]) < fabs(e[a])) a = 1;
  if (fabs(e[2]) < fabs(e[a])) a = 2;
  double ax[3] = {0.0, 0.0, 0.0};
  ax[a] = 1.0;
  double u[3] = {ax[1] * e[2] - ax[2] * e[1], ax[2] * e[0] - ax[0] * e[2],
                 ax[0] * e[1] - ax[1] * e[0]};
  const double un = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  u[0] /= un; u[1] /= un; u[2] /= un;
  const double w[3] = {e[1] * u[2] - e[2] * u[1], e[2] * u[0] - e[0] * u[2],
                       e[0] * u[1] - e[1] * u[0]};
  const double sin_chi = sqrt(fmax(0.0, 1.0 - cos_chi * cos_chi));
  double sp, cp;
  sincos(phi, &sp, &cp);
  for (int j = 0; j < 3; ++j) out[j] = cos_chi * e[j] + sin_chi * (cp * u[j] + sp * w[j]);
}

// Contiguous-run reduction over the lanes of a warp: lanes with equal `key`
// next to each other form a run; on return the last lane of every run holds
// the run's sums of the four values (fixed order, so deterministic) and the
// function returns true there.  All 32 lanes must call it.
template <typename T>
__device__ __forceinline__ bool run_sum4(int key, T& a, T& b, T& c, T& d) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int prev = __shfl_up_sync(full, key, 1);
  const int next = __shfl_down_sync(full, key, 1);
  const bool head = lane == 0 || prev != key;
  const bool tail = lane == 31 || next != key;
  if (__all_sync(full, head)) return tail;          // no two neighbours share a key
  int start = head ? lane : 0;                        // first lane of this lane's run
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(full, start, o);
    if (lane >= o && t > start) start = t;
  }
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T ta = __shfl_up_sync(full, a, o), tb = __shfl_up_sync(full, b, o);
    const T tc = __shfl_up_sync(full, c, o), td = __shfl_up_sync(full, d, o);
    if (lane - o >= start) {
      a += ta;
      b += tb;
      c += tc;
      d += td;
    }
  }
  return tail;
}

// Bitonic sort of P (a power of two) keys with their indices, one CTA.
static __device__ void bitonic(unsigned long long* key, unsigned int* idx, int P) {
  const int half = P >> 1;   // compare-exchange pairs per stage, one per thread and pass
  for (int k = 2; k <= P; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int q = threadIdx.x; q < half; q += blockDim.x) {
        const int i = ((q & ~(j - 1)) << 1) | (q & (j - 1));   // pair q: (i, i + j), bit j of i clear
        const int l = i + j;
        const bool up = (i & k) == 0;
        const unsigned long long a = key[i], b = key[l];
        if ((a > b) == up) {
          key[i] = b;
          key[l] = a;
          const unsigned int t = idx[i];
          idx[i] = idx[l];
          idx[l] = t;
        }
      }
      __syncthreads();
    }
}

}  // namespace pic
