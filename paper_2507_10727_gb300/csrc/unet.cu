// unet.cu -- the learned Poisson warm start: a BF16 U-Net on the node grid,
// its forward and backward passes, Adam training on snapshots the simulation
// records, and the per-step guess of the Poisson start (the solver still
// runs to its tolerance: the guess only changes where the solve starts, never
// where it ends).
//
// All convolutions run on the 5th-generation tensor cores (tcgen05.mma, BF16
// operands, FP32 accumulator in tensor memory) over output tiles of 8 x 16
// nodes, their operands staged by TMA tiled loads (4-D tensor maps over
// channels, columns, rows and batch of the node-major activations; zero fill
// outside the grid).  The forward convolution (and the data gradient, the same
// kernel on flipped, transposed weights) is persistent: a tap (dr, dc) is a
// box of column shift dc read from row dr on, a descriptor offset, and the
// next chunk loads while this one's MMAs run.  The weight gradient contracts
// over nodes: its operands are transposed into K-major tiles by ldmatrix.trans
// and each output row takes three MMAs (one per row shift); split-K over tiles
// with a deterministic reduction.
#include <cmath>
#include <cstring>
#include <random>
#include <vector>

#include <cuda.h>
#include <cuda_bf16.h>

#include "launch.h"
#include "unet.h"

namespace pic {

typedef __nv_bfloat16 bf16;

namespace {

constexpr int kLev = 4;
constexpr int kCh[kLev] = {16, 32, 64, 64};
constexpr int kInReal = 3;
constexpr int kInPad = 16;
constexpr int kNumConv = 14;
constexpr int kHead = 14;
constexpr int kNumLayers = 15;

constexpr int kWgThreads = 256;               // weight gradient: 8 warps stage, 2 read TMEM
constexpr int kMaxSplit = 608;                // bound of splits x input chunks (partials)
constexpr int kHeadVals = 18;                 // loss, d bias, d w[16]

// ---------------------------------------------------------------------------
// PTX helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
// 16-byte async copy global -> shared; bytes < 16 zero-fills the rest
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ void ldsm_x4_t(unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3,
                                          const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
  // splitmix64 finaliser (Steele, Lea, Flood 2014)
  x += 0x9E3779B97F4A7C15ULL;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
  return x ^ (x >> 31);
}

// ---------------------------------------------------------------------------
// 3x3 convolution (forward; also the data gradient on flipped weights)
// ---------------------------------------------------------------------------
struct ConvArgs {
  const bf16* x;      // input buffer; logical node (i, j) at buffer node (i, j) * x_step
  long long x_bs;     // batch stride (elements)
  int x_cs, x_c0, x_step, x_w;   // channel stride, channel offset, node step, buffer row length
  const bf16* w;      // packed weights [cin / 16][9][cout][16]
  const float* bias;  // cout entries or null
  int cin, cout;      // cin multiple of 16
  bf16* y;
  long long y_bs;
  int y_cs, y_c0, y_step, y_w;
  int H, W, B;        // logical node grid of the convolution, batch
  int relu, accumulate;
  int* err;           // set to 1 if a tensor-core wait reached its time limit
};

__device__ __forceinline__ void load8(const bf16* p, float* v) {
  const uint4 u = *reinterpret_cast<const uint4*>(p);
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float2 f = __bfloat1622float2(h[q]);
    v[2 * q] = f.x;
    v[2 * q + 1] = f.y;
  }
}
__device__ __forceinline__ void store8(bf16* p, const float* v) {
  uint4 u;
  __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
  for (int q = 0; q < 4; ++q) h[q] = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
  *reinterpret_cast<uint4*>(p) = u;
}

// ---- tcgen05 helpers --------------------------------------------------------
constexpr int kTcThreads = 128;          // 4 warps = the 4 TMEM lane quarters
constexpr int kTcM = 128;                // output nodes per tile (MMA M)
constexpr double kWaitLimitNs = 1.0e9;   // tensor-core completion wait limit

// forward convolution: output tiles of 8 x 16 nodes; per 16-channel input
// chunk six input boxes (3 column shifts x 2 groups of 8 channels) of 10 rows
// x 16 columns x 8 channels, then the chunk's 9 x 2 x COB weight rows
constexpr int kFwTH = 8, kFwTW = 16;
constexpr int kFwBox = (kFwTH + 2) * kFwTW * 16;          // 2,560 bytes
constexpr int kFwA = 6 * kFwBox;
__host__ __device__ constexpr int tc_b_stage(int cob) { return 9 * 2 * cob * 16; }
__host__ __device__ constexpr int tc_stage(int cob) { return kFwA + tc_b_stage(cob); }
__host__ __device__ constexpr int tc_smem(int cob) { return 2 * tc_stage(cob) + 64; }
__host__ __device__ constexpr int tc_tcols(int cob) { return cob <= 32 ? 32 : 64; }

// shared-memory matrix descriptor: canonical K-major layout without swizzle;
// lbo = byte step between core matrices along K, sbo = along M (or N)
__device__ __forceinline__ unsigned long long smem_desc(unsigned addr, unsigned lbo, unsigned sbo) {
  unsigned long long d = (unsigned long long)((addr >> 4) & 0x3FFFu);
  d |= (unsigned long long)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (unsigned long long)((sbo >> 4) & 0x3FFFu) << 32;
  d |= 1ULL << 46;   // descriptor version of the 5th-generation tensor cores
  return d;
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// wait for the phase of the given parity; false after the time limit
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
  const unsigned a = smem_u32(bar);
  double t0 = -1.0;
  for (unsigned it = 0;; ++it) {
    unsigned done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 1023u) == 0u) {
      unsigned long long t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (t0 < 0.0) t0 = (double)t;
      else if ((double)t - t0 > kWaitLimitNs) return false;
    }
  }
}

template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// 16 consecutive FP32 accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float* v) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

// TMA: a 4-D tiled load into shared memory, completion counted on an mbarrier
__device__ __forceinline__ void tma_load4(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                          int c3, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
      "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// bulk copy of `bytes` (a multiple of 16) from global to shared memory
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes,
                                          unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Persistent: a CTA takes work items (output tile of 8 x 16 nodes, block of
// COB output channels), item = blockIdx.x, + gridDim.x, ...; its chunks of 16
// input channels run through two stages: thread 0 loads a chunk's six input
// boxes by TMA (tensor map tmx over channels, columns, rows, batch of the
// input; zero fill outside the grid) and its weight rows by bulk copies
// (packed [cin / 16][9][2][cout][8]), one mbarrier per stage counting the
// bytes; the next chunk (of this item, or the next item's first) loads while
// this one's MMAs run.  A tap (dr, dc) is the box of column shift dc read
// from row dr on: 8 output rows x 16 columns are M = 128 consecutive 16-byte
// rows of the K-major layout, so its A descriptor starts dr x 16 nodes into
// the box.  The accumulator (COB FP32 columns of TMEM) is read after the
// item's last chunk, bias, ReLU and the accumulate option applied, stored as
// BF16 (output node step y_step).
template <int COB>
__global__ void __launch_bounds__(kTcThreads) k_conv3_tc(ConvArgs a,
                                                         const __grid_constant__ CUtensorMap tmx) {
  extern __shared__ __align__(1024) unsigned char sm[];
  constexpr int BST = tc_b_stage(COB);
  constexpr int STG = tc_stage(COB);
  constexpr unsigned TCOLS = tc_tcols(COB);
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(sm + 2 * STG);   // [s] loads, [2 + s] MMAs
  unsigned* taddr_s = reinterpret_cast<unsigned*>(bar + 4);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tw = (a.W + kFwTW - 1) / kFwTW, th = (a.H + kFwTH - 1) / kFwTH;
  const int ncob = a.cout / COB;
  const long long items = (long long)a.B * tw * th * ncob;
  const int nkc = a.cin >> 4;
  auto decode = [&](long long item, int& b, int& i0, int& j0, int& co0) {
    const long long tile = item / ncob;
    co0 = (int)(item - tile * ncob) * COB;
    b = (int)(tile / ((long long)tw * th));
    const int r = (int)(tile - (long long)b * tw * th);
    i0 = (r / tw) * kFwTH;
    j0 = (r % tw) * kFwTW;
  };
  // thread 0: the loads of chunk kc of `item` into stage st
  auto stage = [&](long long item, int kc, int st) {
    int b, i0, j0, co0;
    decode(item, b, i0, j0, co0);
    unsigned char* base = sm + st * STG;
    mbar_expect_tx(&bar[st], (unsigned)STG);
#pragma unroll
    for (int dc = 0; dc < 3; ++dc)
#pragma unroll
      for (int g = 0; g < 2; ++g)
        tma_load4(base + (dc * 2 + g) * kFwBox, &tmx, a.x_c0 + kc * 16 + g * 8, j0 + dc - 1, i0 - 1,
                  b, &bar[st]);
    for (int q = 0; q < 18; ++q)   // q = 2 tap + g
      bulk_load(base + kFwA + q * COB * 16, a.w + (((long long)kc * 18 + q) * a.cout + co0) * 8,
                COB * 16, &bar[st]);
  };
  if (tid == 0) {
    for (int q = 0; q < 4; ++q) mbar_init(&bar[q], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (blockIdx.x < items) stage(blockIdx.x, 0, 0);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(taddr_s)),
                 "r"(TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned taddr = *taddr_s;
  // D f32, A and B bf16, both K-major, N = COB, M = 128
  const unsigned idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(COB >> 3) << 17) |
                         ((unsigned)(kTcM >> 4) << 24);
  long long g = 0;                                  // chunk being computed (thread 0)
  long long issued = blockIdx.x < items ? 1 : 0;    // chunks whose loads were issued (thread 0)
  bool bad = false;
  for (long long item = blockIdx.x; item < items; item += gridDim.x) {
    bool f = false;
    if (tid == 0) {
      for (int kc = 0; kc < nkc && !f; ++kc, ++g) {
        const int st = (int)(g & 1);
        // the next chunk into the other stage, once the MMAs of chunk g - 1
        // (which read that stage) are done
        const bool more = kc + 1 < nkc || item + gridDim.x < items;
        if (more) {
          if (g >= 1) f = !mbar_wait(&bar[2 + (st ^ 1)], (unsigned)((g - 1) >> 1) & 1u);
          if (f) break;
          if (kc + 1 < nkc) stage(item, kc + 1, st ^ 1);
          else stage(item + gridDim.x, 0, st ^ 1);
          ++issued;
        }
        f = !mbar_wait(&bar[st], (unsigned)(g >> 1) & 1u);
        if (f) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const unsigned aA = smem_u32(sm + st * STG), aB = aA + kFwA;
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
          const int dr = tap / 3, dc = tap - dr * 3;
          const unsigned long long ad =
              smem_desc(aA + (unsigned)(dc * 2 * kFwBox + dr * kFwTW * 16), kFwBox, 128);
          const unsigned long long bd = smem_desc(aB + (unsigned)(tap * 2 * COB * 16), COB * 16, 128);
          const unsigned acc = (kc > 0 || tap > 0) ? 1u : 0u;
          asm volatile(
              "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(taddr),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&bar[2 + st]))
                     : "memory");
      }
      // the item's accumulator is complete once its last chunk's MMAs are
      if (!f) f = !mbar_wait(&bar[2 + (int)((g - 1) & 1)], (unsigned)((g - 1) >> 1) & 1u);
    }
    if (__syncthreads_or(f)) {
      bad = true;
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    int b, i0, j0, co0;
    decode(item, b, i0, j0, co0);
    const int r = 32 * warp + lane;
    const int gi = i0 + (r >> 4), gj = j0 + (r & 15);
    const bool mine = gi < a.H && gj < a.W;
    bf16* dst = a.y + (long long)b * a.y_bs +
                ((long long)gi * a.y_step * a.y_w + (long long)gj * a.y_step) * a.y_cs + a.y_c0 + co0;
#pragma unroll
    for (int c = 0; c < COB; c += 16) {
      float v[16];
      tmem_ld16(taddr + ((unsigned)(32 * warp) << 16) + (unsigned)c, v);   // all lanes take part
      if (!mine) continue;
#pragma unroll
      for (int k = 0; k < 16; ++k) v[k] += a.bias ? a.bias[co0 + c + k] : 0.0f;
      if (a.accumulate) {
        float o[16];
        load8(dst + c, o);
        load8(dst + c + 8, o + 8);
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] += o[k];
      }
      if (a.relu) {
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = fmaxf(v[k], 0.0f);
      }
      store8(dst + c, v);
      store8(dst + c + 8, v + 8);
    }
    // the next item's MMAs overwrite the accumulator after every lane read it
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  if (bad) {
    if (tid == 0) {
      atomicExch(a.err, 1);
      // loads still in flight must land before the CTA goes: wait
      // (time-limited) for every issued chunk not yet consumed
      for (long long c = g; c < issued; ++c) mbar_wait(&bar[c & 1], (unsigned)(c >> 1) & 1u);
    }
    __syncthreads();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TCOLS));
}

// ---------------------------------------------------------------------------
// Weight gradient on the tensor cores: dW[co][ci][tap] = sum over nodes of
// dZ[node][co] X[node + (dr - 1, dc - 1)][ci], tap = 3 dr + dc.  A CTA (input
// channel chunk kc, split s) runs over output tiles of 8 x 16 nodes, t = s,
// s + S, ...  Per tile the input patch (10 x 18 nodes x 16 channels) and the
// dZ tile (128 nodes x COUT) are staged node-major by two TMA tiled loads
// (4-D tensor maps over channels, columns, rows, batch; zero fill outside
// the grid; two buffers: the next tile loads while this one is transposed),
// then transposed by ldmatrix.trans into K-major operand tiles with the nodes
// as K:
//   A[(dc, ci)][patch node (pr, c)] = X at patch (pr, c + dc): 48 rows, 10
//     patch rows x 16 columns of K, so a row shift dr is a shift of K by 16
//     (two core matrices: a descriptor offset);
//   B[co][output node (i, c)] = dZ: COUT rows.
// Per output row i three MMAs (M = 128, N = COUT, K = 16), one per dr, A from
// patch row i + dr, each into its own TMEM accumulator of COUT columns; A rows
// 48..127 read neighbouring operand memory and their accumulator lanes are
// discarded.  The accumulator stays in TMEM over the CTA's tiles; the splits'
// partials are summed in split order afterwards (deterministic).
// ---------------------------------------------------------------------------
struct WgArgs {
  const bf16* x;
  long long x_bs;
  int x_cs, x_c0, x_step, x_w;
  const bf16* dz;     // output gradient (after the ReLU mask), node step 1, row length W
  long long dz_bs;
  int dz_cs, dz_c0;
  int cin, H, W, B;   // cin: padded (multiple of 16)
  float* pw;          // [S][cin / 16][9][COUT][16]
  float* pb;          // [S][COUT]
  int* err;           // set to 1 if a tensor-core wait reached its time limit
};

constexpr int kWgTH = 8, kWgTW = 16;                     // output tile: rows x columns
constexpr int kWgPH = kWgTH + 2, kWgPW = kWgTW + 2;      // input patch
constexpr int kWgPatch = kWgPH * kWgPW * 32;             // patch bytes (16 channels)
constexpr int kWgLboA = 48 * 16;                         // A: bytes per core-matrix column
constexpr int kWgA = kWgPH * 2 * kWgLboA;                // A tile bytes (20 core-matrix columns)
constexpr int kWgAOver = 128 * 16 - 48 * 16;             // A rows 48..127 past a core-matrix column
__host__ __device__ constexpr int wg_b(int cout) { return kWgTH * kWgTW * cout * 2; }
__host__ __device__ constexpr int wg_raw(int cout) { return kWgPatch + wg_b(cout); }
__host__ __device__ constexpr int wg_smem(int cout) {
  return 2 * wg_raw(cout) + kWgA + wg_b(cout) + 64;
}
__host__ __device__ constexpr unsigned wg_tcols(int cout) {
  return 3 * cout <= 32 ? 32u : 3 * cout <= 64 ? 64u : 3 * cout <= 128 ? 128u : 256u;
}
static_assert(kWgAOver <= wg_b(16), "A rows read past the A tile stay inside the B tile");

// tmx: the layer input (channels, columns, rows, batch; the column and row
// steps of a strided input in its byte strides); tmd: dZ (channels, columns,
// rows, batch)
template <int COUT>
__global__ void __launch_bounds__(kWgThreads) k_conv3_wgrad(WgArgs a,
                                                            const __grid_constant__ CUtensorMap tmx,
                                                            const __grid_constant__ CUtensorMap tmd) {
  extern __shared__ __align__(1024) unsigned char sm[];
  constexpr int BB = wg_b(COUT);
  constexpr int RAW = wg_raw(COUT);
  constexpr unsigned TCOLS = wg_tcols(COUT);
  // raw buffer r at sm + r RAW: patch [10][18][16 channels], then dZ [8][16][COUT]
  unsigned char* At = sm + 2 * RAW;        // A operand tile (its last MMAs read into Bt)
  unsigned char* Bt = At + kWgA;           // B operand tile
  unsigned long long* mbar = reinterpret_cast<unsigned long long*>(Bt + BB);   // [0] MMA, [1..2] raw
  unsigned* taddr_s = reinterpret_cast<unsigned*>(mbar + 3);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int kc = blockIdx.x, nkc = gridDim.x, s = blockIdx.y, S = gridDim.y;
  const int tw = (a.W + kWgTW - 1) / kWgTW, th = (a.H + kWgTH - 1) / kWgTH;
  const int T = a.B * tw * th;

  // one thread: the TMA loads of tile t into raw buffer r
  auto stage_raw = [&](int t, int r) {
    unsigned char* Xp = sm + r * RAW;
    const int b = t / (tw * th), rr = t - b * tw * th;
    const int i0 = (rr / tw) * kWgTH, j0 = (rr % tw) * kWgTW;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // after the generic reads
    mbar_expect_tx(&mbar[1 + r], (unsigned)(kWgPatch + BB));
    tma_load4(Xp, &tmx, a.x_c0 + kc * 16, j0 - 1, i0 - 1, b, &mbar[1 + r]);
    tma_load4(Xp + kWgPatch, &tmd, a.dz_c0, j0, i0, b, &mbar[1 + r]);
  };

  float bpart[COUT / 16];
#pragma unroll
  for (int m = 0; m < COUT / 16; ++m) bpart[m] = 0.0f;

  // node-major raw tiles of buffer r -> K-major operand tiles (four 8 x 8
  // blocks per ldmatrix.x4.trans; a lane then holds one channel at two
  // consecutive nodes, one 32-bit word of the K-major layout); the bias
  // gradient's per-lane partial sums come from the dZ words
  auto transpose = [&](int r) {
    const unsigned char* Xp = sm + r * RAW;
    const unsigned char* Ds = Xp + kWgPatch;
    // A: 6 row blocks (dc, channel half) x 20 node blocks (patch row, column half)
    for (int job = warp; job < 6 * 20 / 4; job += kWgThreads / 32) {
      const int blk = job * 4 + (lane >> 3);
      const int rb = blk / 20, kb = blk - rb * 20;
      const int dc = rb >> 1, g = rb & 1;
      const int pr = kb >> 1, c = (kb & 1) * 8 + (lane & 7) + dc;
      unsigned v[4];
      ldsm_x4_t(v[0], v[1], v[2], v[3], Xp + (pr * kWgPW + c) * 32 + g * 16);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int bj = job * 4 + j;
        const int rbj = bj / 20, kbj = bj - rbj * 20;
        const int row = rbj * 8 + (lane >> 2);
        *reinterpret_cast<unsigned*>(At + kbj * kWgLboA + row * 16 + (lane & 3) * 4) = v[j];
      }
    }
    // B: COUT / 8 row blocks x 16 node blocks; job m of this warp holds
    // channel block (warp + 8 m) / 4
#pragma unroll
    for (int m = 0; m < COUT / 16; ++m) {
      const int job = warp + 8 * m;
      const int blk = job * 4 + (lane >> 3);
      const int cb = blk >> 4, kb = blk & 15;
      unsigned v[4];
      ldsm_x4_t(v[0], v[1], v[2], v[3], Ds + (kb * 8 + (lane & 7)) * (COUT * 2) + cb * 16);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int bj = job * 4 + j;
        const int row = (bj >> 4) * 8 + (lane >> 2);
        *reinterpret_cast<unsigned*>(Bt + (bj & 15) * (COUT * 16) + row * 16 + (lane & 3) * 4) = v[j];
        const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&v[j]));
        bpart[m] += f.x + f.y;
      }
    }
  };

  if (tid == 0) {
    for (int q = 0; q < 3; ++q) mbar_init(&mbar[q], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    stage_raw(s, 0);   // s < T: the host launches at most T splits
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(taddr_s)),
                 "r"(TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned taddr = *taddr_s;
  // D f32, A and B bf16, both K-major, N = COUT, M = 128
  const unsigned idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(COUT >> 3) << 17) |
                         ((unsigned)(128 >> 4) << 24);
  bool bad = false;
  int i = 0;
  for (int t = s; t < T; t += S, ++i) {
    const int rb = i & 1;
    // the next tile loads while this one is transposed (raw buffer rb ^ 1 was
    // read by the transposition of tile i - 1, finished at that iteration's
    // last barrier)
    if (tid == 0 && t + S < T) stage_raw(t + S, rb ^ 1);
    // tile i in raw buffer rb (its (i / 2)-th load), and the MMAs of tile
    // i - 1 done with the operand tiles
    bool f = !mbar_wait(&mbar[1 + rb], (unsigned)(i >> 1) & 1u);
    if (i >= 1) f = f || !mbar_wait(&mbar[0], (unsigned)(i - 1) & 1u);
    if (__syncthreads_or(f)) {
      bad = true;
      break;
    }
    transpose(rb);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned aA = smem_u32(At), aB = smem_u32(Bt);
#pragma unroll
      for (int kk = 0; kk < kWgTH; ++kk) {
        const unsigned long long bd = smem_desc(aB + (unsigned)(kk * 2 * COUT * 16), COUT * 16, 128);
#pragma unroll
        for (int dr = 0; dr < 3; ++dr) {
          const unsigned long long ad = smem_desc(aA + (unsigned)((kk + dr) * 2 * kWgLboA), kWgLboA, 128);
          const unsigned acc = (i > 0 || kk > 0) ? 1u : 0u;
          asm volatile(
              "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(taddr + (unsigned)(dr * COUT)),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&mbar[0]))
                   : "memory");
    }
  }
  if (!bad && i > 0) {
    const bool f = !mbar_wait(&mbar[0], (unsigned)(i - 1) & 1u);
    bad = __syncthreads_or(f);
  }
  if (bad) {
    if (tid == 0) atomicExch(a.err, 1);
    // a load still in flight must not land after the CTA has gone: wait
    // (time-limited) for tile i's load and, if it was issued, tile i + 1's
    if (tid == 0) {
      mbar_wait(&mbar[1 + (i & 1)], (unsigned)(i >> 1) & 1u);
      if (s + (long long)(i + 1) * S < T) mbar_wait(&mbar[1 + ((i + 1) & 1)], (unsigned)((i + 1) >> 1) & 1u);
    }
    __syncthreads();
  } else {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp < 2) {
      // TMEM lane 32 warp + lane = A row (dc, ci); lanes 48.. discarded
      const int r = 32 * warp + lane;
      float* pw = a.pw + ((long long)s * nkc + kc) * 9 * COUT * 16 + (r & 15);
#pragma unroll
      for (int dr = 0; dr < 3; ++dr) {
        const int tap = dr * 3 + (r >> 4);
#pragma unroll
        for (int c = 0; c < COUT; c += 16) {
          float v[16];
          tmem_ld16(taddr + ((unsigned)(32 * warp) << 16) + (unsigned)(dr * COUT + c), v);
          if (r < 48) {
#pragma unroll
            for (int k = 0; k < 16; ++k) pw[((long long)tap * COUT + c + k) * 16] = v[k];
          }
        }
      }
    }
    if (kc == 0) {
      // bias gradient: the four lanes of a channel, then the warps, in order
      float* red = reinterpret_cast<float*>(At);   // the operand tiles are free now
      for (int q = tid; q < 8 * COUT; q += kWgThreads) red[q] = 0.0f;
      __syncthreads();
#pragma unroll
      for (int m = 0; m < COUT / 16; ++m) {
        float v = bpart[m];
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        const int cb = (warp + 8 * m) >> 2;
        if ((lane & 3) == 0) red[warp * COUT + cb * 8 + (lane >> 2)] = v;
      }
      __syncthreads();
      if (tid < COUT) {
        float v = 0.0f;
        for (int w = 0; w < 8; ++w) v += red[w * COUT + tid];
        a.pb[(long long)s * COUT + tid] = v;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TCOLS));
}

// sum the split partials into the layer's weight/bias gradient.  A block
// (256 threads) owns 16 consecutive partial words e (the partials' own layout
// (kc, tap, co, k), so neighbouring threads read neighbouring words); its 16
// split groups g sum splits g, g + 16, ... in order, then the 16 group sums
// are added in group order (deterministic).
constexpr int kRedE = 16, kRedG = 16;
__global__ void __launch_bounds__(kRedE * kRedG) k_wgrad_reduce(const float* pw, const float* pb,
                                                                  int S, int cin, int cin_pad,
                                                                  int cout, float* gw, float* gb) {
  __shared__ float part[kRedG][kRedE];
  const long long per = (long long)(cin_pad >> 4) * 9 * cout * 16;   // one split's partials
  const int tx = threadIdx.x % kRedE, g = threadIdx.x / kRedE;
  const long long e = (long long)blockIdx.x * kRedE + tx;
  float s = 0.0f;
  if (e < per) {
#pragma unroll 4
    for (int sp = g; sp < S; sp += kRedG) s += pw[(long long)sp * per + e];
  } else if (e < per + cout) {
    const int co = (int)(e - per);
#pragma unroll 4
    for (int sp = g; sp < S; sp += kRedG) s += pb[(long long)sp * cout + co];
  }
  part[g][tx] = s;
  __syncthreads();
  if (g != 0 || e >= per + cout) return;
  float t = 0.0f;
  for (int q = 0; q < kRedG; ++q) t += part[q][tx];
  if (e < per) {
    const int k = (int)(e & 15);
    long long r = e >> 4;
    const int co = (int)(r % cout);
    r /= cout;
    const int tap = (int)(r % 9);
    const int kc = (int)(r / 9);
    const int ci = kc * 16 + k;
    if (ci < cin) gw[((long long)co * cin + ci) * 9 + tap] = t;
  } else {
    gb[e - per] = t;
  }
}

// ---------------------------------------------------------------------------
// element-wise pieces
// ---------------------------------------------------------------------------
// g <- g * (y > 0) on a channel slice (ReLU backward), 8 channels per item
__global__ void k_relu_mask(bf16* g, int g_cs, int g_c0, const bf16* y, int y_cs, int y_c0, int C,
                            long long npx) {
  const int c8n = C >> 3;
  const long long total = npx * c8n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long p = e / c8n;
    const int c8 = (int)(e - p * c8n);
    uint4* gp = reinterpret_cast<uint4*>(g + p * g_cs + g_c0 + c8 * 8);
    const uint4 yv = *reinterpret_cast<const uint4*>(y + p * y_cs + y_c0 + c8 * 8);
    uint4 gv = *gp;
    unsigned* gw = &gv.x;
    const unsigned* yw = &yv.x;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const unsigned lo = yw[q] & 0xFFFFu, hi = yw[q] >> 16;
      const bool plo = (lo & 0x8000u) == 0 && (lo & 0x7FFFu) != 0;
      const bool phi = (hi & 0x8000u) == 0 && (hi & 0x7FFFu) != 0;
      gw[q] &= (plo ? 0x0000FFFFu : 0u) | (phi ? 0xFFFF0000u : 0u);
    }
    *gp = gv;
  }
}

// bilinear node up-sampling: coarse node (I, J) sits on fine node (2I, 2J)
__global__ void k_up(const bf16* src, int s_cs, int s_c0, int Hc, int Wc, bf16* dst, int d_cs,
                     int d_c0, int Hf, int Wf, int C, int B) {
  const int c8n = C >> 3;
  const long long total = (long long)B * Hf * Wf * c8n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int c8 = (int)(e % c8n);
    const long long p = e / c8n;
    const int b = (int)(p / ((long long)Hf * Wf));
    const int q = (int)(p - (long long)b * Hf * Wf);
    const int i = q / Wf, j = q - i * Wf;
    const int I = i >> 1, J = j >> 1, oi = i & 1, oj = j & 1;
    const bf16* cb = src + (long long)b * Hc * Wc * s_cs + s_c0 + c8 * 8;
    float v[8], t[8];
    load8(cb + ((long long)I * Wc + J) * s_cs, v);
    if (oi) {
      load8(cb + ((long long)(I + 1) * Wc + J) * s_cs, t);
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] += t[k];
    }
    if (oj) {
      load8(cb + ((long long)I * Wc + J + 1) * s_cs, t);
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] += t[k];
    }
    if (oi && oj) {
      load8(cb + ((long long)(I + 1) * Wc + J + 1) * s_cs, t);
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] += t[k];
    }
    const float sc = (oi && oj) ? 0.25f : (oi || oj) ? 0.5f : 1.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] *= sc;
    store8(dst + (p * d_cs) + d_c0 + c8 * 8, v);
  }
}

// transpose of k_up: coarse gradient = sum over the fine nodes it feeds
__global__ void k_up_t(const bf16* gf, int f_cs, int f_c0, int Hf, int Wf, bf16* gc, int c_cs,
                       int c_c0, int Hc, int Wc, int C, int B) {
  const int c8n = C >> 3;
  const long long total = (long long)B * Hc * Wc * c8n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int c8 = (int)(e % c8n);
    const long long p = e / c8n;
    const int b = (int)(p / ((long long)Hc * Wc));
    const int q = (int)(p - (long long)b * Hc * Wc);
    const int I = q / Wc, J = q - I * Wc;
    const bf16* fb = gf + (long long)b * Hf * Wf * f_cs + f_c0 + c8 * 8;
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0}, t[8];
    for (int di = -1; di <= 1; ++di) {
      const int i = 2 * I + di;
      if (i < 0 || i >= Hf) continue;
      const float wi = di == 0 ? 1.0f : 0.5f;
      for (int dj = -1; dj <= 1; ++dj) {
        const int j = 2 * J + dj;
        if (j < 0 || j >= Wf) continue;
        const float w = wi * (dj == 0 ? 1.0f : 0.5f);
        load8(fb + ((long long)i * Wf + j) * f_cs, t);
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] += w * t[k];
      }
    }
    store8(gc + p * c_cs + c_c0 + c8 * 8, acc);
  }
}

// 1x1 head (16 -> 1), FP32
__global__ void k_head_fwd(const bf16* h, const float* w, const float* bias, float* out, long long npx) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npx;
       p += (long long)gridDim.x * blockDim.x) {
    float v[16];
    load8(h + p * 16, v);
    load8(h + p * 16 + 8, v + 8);
    float s = bias[0];
#pragma unroll
    for (int c = 0; c < 16; ++c) s += w[c] * v[c];
    out[p] = s;
  }
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// MSE loss and the head's backward: d out = 2 (out - y) / N, d h = w d out;
// block partial sums of (sum d^2, d bias, d w[16]) in FP64
__global__ void __launch_bounds__(256) k_head_bwd(const bf16* h, const float* w, const float* out,
                                                  const float* y, bf16* gh, long long npx,
                                                  double inv_n, double* partial) {
  __shared__ double red[kHeadVals][8];
  // a thread's partial sums in FP32 (a few tens of nodes each; the FP64
  // pipes of this part are a small fraction of its FP32 rate), FP64 from the
  // warp sums on
  float loc[kHeadVals];
#pragma unroll
  for (int k = 0; k < kHeadVals; ++k) loc[k] = 0.0f;
  const float ginv = (float)(2.0 * inv_n);
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npx;
       p += (long long)gridDim.x * blockDim.x) {
    const float d = out[p] - y[p];
    const float g = ginv * d;
    loc[0] = fmaf(d, d, loc[0]);
    loc[1] += g;
    float v[16], o[16];
    load8(h + p * 16, v);
    load8(h + p * 16 + 8, v + 8);
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      loc[2 + c] = fmaf(g, v[c], loc[2 + c]);
      o[c] = w[c] * g;
    }
    store8(gh + p * 16, o);
    store8(gh + p * 16 + 8, o + 8);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kHeadVals; ++k) {
    const double s = warp_sum_d((double)loc[k]);
    if (lane == 0) red[k][wid] = s;
  }
  __syncthreads();
  if (threadIdx.x < kHeadVals) {
    double s = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[threadIdx.x][q];
    partial[(long long)blockIdx.x * kHeadVals + threadIdx.x] = s;
  }
}

__global__ void k_head_final(const double* partial, int nblk, double inv_n, double* loss,
                             float* gw, float* gb) {
  const int k = threadIdx.x;
  if (k >= kHeadVals) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += partial[(long long)b * kHeadVals + k];
  if (k == 0) *loss = s * inv_n;
  else if (k == 1) gb[0] = (float)s;
  else gw[k - 2] = (float)s;
}

// network input from host arrays in the (B, 3, H, W) layout
__global__ void k_pack_input(const float* xs, int B, int H, int W, bf16* x_in) {
  const long long npx = (long long)H * W, total = (long long)B * npx;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long b = e / npx, q = e - b * npx;
    float v[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = c < kInReal ? xs[(b * kInReal + c) * npx + q] : 0.0f;
    store8(x_in + e * 16, v);
    store8(x_in + e * 16 + 8, v + 8);
  }
}

// conductor nodes (Dirichlet values) of the field boundary; g, wall as in
// field_free
__device__ __forceinline__ bool dirichlet_node(int m, int n, int nr, int nz, int g, int wall) {
  return !field_free(m, n, nr, nz, g, wall);
}

// training batch: B snapshots drawn by hash of (seed, iteration, b).
// Slot fields: mode 0 (rho, phi), mode 1 (res, phi - phi_prev).
__global__ void k_train_input(const float* f0, const float* f1, const float* slot_scale,
                              long long avail, int B, unsigned long long seed, long long iter,
                              int nr, int nz, int g, int wall, int mode, const UDev* ud,
                              bf16* x_in, float* y) {
  const int W = nz + 1;
  const long long npx = (long long)(nr + 1) * W, total = (long long)B * npx;
  const double K = ud->out_norm / ud->in_norm;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long b = e / npx, q = e - b * npx;
    const unsigned long long hsh =
        mix64(seed ^ mix64((unsigned long long)iter * 0x100000001B3ULL + (unsigned long long)b));
    const long long slot = (long long)(hsh % (unsigned long long)avail);
    const int m = (int)(q / W), n = (int)(q - (long long)m * W);
    const float a = f0[slot * npx + q], t = f1[slot * npx + q];
    const bool dir = dirichlet_node(m, n, nr, nz, g, wall);
    // mode 0: global scales; mode 1: the snapshot's own residual RMS
    const double sc = mode == 0 ? 1.0 : (double)slot_scale[slot];
    const float inv_in = (float)(1.0 / (mode == 0 ? ud->in_norm : sc));
    const float inv_out = (float)(1.0 / (mode == 0 ? ud->out_norm : sc * K));
    float v[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = 0.0f;
    v[0] = a * inv_in;
    v[1] = (float)m / (float)nr;
    v[2] = mode == 0 ? (dir ? t * inv_out : 0.0f) : (dir ? 1.0f : 0.0f);
    store8(x_in + e * 16, v);
    store8(x_in + e * 16 + 8, v + 8);
    y[e] = t * inv_out;
  }
}

// The per-step kernels run over all instances of a handle at once:
// blockIdx.y (grid-stride kernels) or blockIdx.x (one-CTA kernels) = instance
// k, read from the device array insts; instance k's node fields sit at
// offset k * npx of the per-instance buffers.

// network input of each instance from its live state (sample k of the
// batch): mode 0 from rho = Q / V and phi's Dirichlet values, mode 1 from the
// residual of the previous solution scaled by its RMS scale[k]
__global__ void k_step_input(const Inst* insts, const UDev* ud, int mode, const float* res_all,
                             const double* scale, bf16* x_all) {
  const int k = blockIdx.y;
  const Inst& I = insts[k];
  const int W = I.nz + 1;
  const long long npx = (long long)(I.nr + 1) * W;
  if (I.S->status & ST_FATAL) return;
  const float* res = res_all + k * npx;
  bf16* x_in = x_all + k * npx * kInPad;
  const double inv_in = 1.0 / (mode == 0 ? ud->in_norm : scale[k]);
  const double inv_out = 1.0 / ud->out_norm;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < npx;
       q += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(q / W), n = (int)(q - (long long)m * W);
    const bool dir = dirichlet_node(m, n, I.nr, I.nz, I.bc_g, I.bc_wall);
    float v[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = 0.0f;
    if (mode == 0) {
      v[0] = (float)(I.Q[q] / node_volume(I, m, n) * inv_in);
      v[2] = dir ? (float)(I.phi[q] * inv_out) : 0.0f;
    } else {
      v[0] = (float)(res[q] * inv_in);
      v[2] = dir ? 1.0f : 0.0f;
    }
    v[1] = (float)m / (float)I.nr;
    store8(x_in + q * 16, v);
    store8(x_in + q * 16 + 8, v + 8);
  }
}

// candidate start of each instance from its network output (Dirichlet
// values of phi)
__global__ void k_make_cand(const Inst* insts, const float* net_all, const UDev* ud,
                            const double* scale, int mode, double* cand_all) {
  const int k = blockIdx.y;
  const Inst& I = insts[k];
  const int W = I.nz + 1;
  const long long npx = (long long)(I.nr + 1) * W;
  const float* net = net_all + k * npx;
  double* cand = cand_all + k * npx;
  const double* phi = I.phi;
  const double s = mode == 0 ? ud->out_norm : scale[k] * (ud->out_norm / ud->in_norm);
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < npx;
       q += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(q / W), n = (int)(q - (long long)m * W);
    if (dirichlet_node(m, n, I.nr, I.nz, I.bc_g, I.bc_wall)) cand[q] = phi[q];
    else cand[q] = (mode == 0 ? 0.0 : phi[q]) + s * (double)net[q];
  }
}

// Recording: instance k of a recording step (instance 0's step a multiple of
// `every`) writes slot (snap_count + k) mod cap.
__device__ __forceinline__ bool records(const Inst* insts, const Inst& I, int every) {
  return !(I.S->status & ST_FATAL) && (insts[0].S->step % every) == 0;
}

// mode 0 recording (after the solve): rho and phi
__global__ void k_snap_record(const Inst* insts, const UDev* ud, float* f0, float* f1,
                              long long cap, int every) {
  const int k = blockIdx.y;
  const Inst& I = insts[k];
  if (!records(insts, I, every)) return;
  const int W = I.nz + 1;
  const long long npx = (long long)(I.nr + 1) * W;
  const long long slot = (ud->snap_count + k) % cap;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < npx;
       q += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(q / W), n = (int)(q - (long long)m * W);
    f0[slot * npx + q] = (float)(I.Q[q] / node_volume(I, m, n));
    f1[slot * npx + q] = (float)I.phi[q];
  }
}

// mode 1 recording, before the solve: the residual of the previous solution
// into the slot, the previous solution kept in FP64
__global__ void k_snap_pre(const Inst* insts, const UDev* ud, const float* res_all, float* f0,
                           double* phi_prev_all, long long cap, int every) {
  const int k = blockIdx.y;
  const Inst& I = insts[k];
  if (!records(insts, I, every)) return;
  const long long npx = (long long)(I.nr + 1) * (I.nz + 1);
  const long long slot = (ud->snap_count + k) % cap;
  const float* res = res_all + k * npx;
  double* phi_prev = phi_prev_all + k * npx;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < npx;
       q += (long long)gridDim.x * blockDim.x) {
    f0[slot * npx + q] = res[q];
    phi_prev[q] = I.phi[q];
  }
}

// mode 1 recording, after the solve: the change of phi
__global__ void k_snap_post(const Inst* insts, const UDev* ud, float* f1,
                            const double* phi_prev_all, long long cap, int every) {
  const int k = blockIdx.y;
  const Inst& I = insts[k];
  if (!records(insts, I, every)) return;
  const long long npx = (long long)(I.nr + 1) * (I.nz + 1);
  const long long slot = (ud->snap_count + k) % cap;
  const double* phi_prev = phi_prev_all + k * npx;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < npx;
       q += (long long)gridDim.x * blockDim.x)
    f1[slot * npx + q] = (float)(I.phi[q] - phi_prev[q]);
}

// RMS of n floats by one CTA (1024 threads), FP64 accumulation, fixed order;
// zero RMS is stored as 1 (an all-zero input stays zero after scaling)
__device__ void cta_rms(const float* f, long long n, double* out_d, float* out_f) {
  __shared__ double red[32];
  double s = 0.0;
  for (long long k = threadIdx.x; k < n; k += blockDim.x) {
    const double v = f[k];
    s += v * v;
  }
  s = warp_sum_d(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
    double r = n > 0 ? sqrt(t / (double)n) : 0.0;
    if (!(r > 0.0)) r = 1.0;
    if (out_d) *out_d = r;
    if (out_f) *out_f = (float)r;
  }
}

// mode-1 recording: RMS of the residual just stored in instance k's slot
// (one CTA per instance)
__global__ void __launch_bounds__(1024) k_slot_rms(const Inst* insts, const UDev* ud,
                                                   const float* f0, float* slot_scale,
                                                   long long cap, int every) {
  const int k = blockIdx.x;
  const Inst& I = insts[k];
  if (!records(insts, I, every)) return;
  const long long npx = (long long)(I.nr + 1) * (I.nz + 1);
  const long long slot = (ud->snap_count + k) % cap;
  cta_rms(f0 + slot * npx, npx, nullptr, slot_scale + slot);
}

// mode-1 warm start: RMS of each instance's live residual (one CTA each)
__global__ void __launch_bounds__(1024) k_live_rms(const float* res_all, long long npx,
                                                   double* scale) {
  cta_rms(res_all + blockIdx.x * npx, npx, scale + blockIdx.x, nullptr);
}

// after the solves: each instance's iterations; a recording step advances
// the ring by n (one thread, instances in order)
__global__ void k_after_solve(const Inst* insts, int n, UDev* ud, int every, int record) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int k = 0; k < n; ++k) {
    Scalars* S = insts[k].S;
    if (ud->err) atomicOr(&S->status, ST_TIMEOUT);
    if (!(S->status & ST_FATAL)) ud->iters_total += S->poisson_iters;
  }
  if (record && (insts[0].S->step % every) == 0) ud->snap_count += n;
}

// mean square of a recorded field over the stored snapshots (input and
// output scales, set by the first training call)
__global__ void k_ms_partial(const float* f, long long n, double* partial) {
  __shared__ double red[8];
  double s = 0.0;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const double v = f[k];
    s += v * v;
  }
  s = warp_sum_d(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
    partial[blockIdx.x] = t;
  }
}

__global__ void k_norm_set(const double* partial, int nblk, long long n, double* target) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += partial[b];
  const double rms = n > 0 ? sqrt(s / (double)n) : 0.0;
  *target = rms > 0.0 ? rms : 1.0;
}

__global__ void k_adam(float* p, const float* g, float* m, float* v, long long n, float lr_t,
                       float b1, float b2, float eps) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr_t * mi / (sqrtf(vi) + eps);
  }
}

// packed BF16 weights of every conv layer: forward [cin_pad/16][9][cout][16]
// and data-gradient (flipped taps, in/out swapped) [cout/16][9][cin_pad][16]
struct PackTable {
  int cin[kNumConv], cin_pad[kNumConv], cout[kNumConv];
  long long w_off[kNumConv], wf_off[kNumConv], wd_off[kNumConv];
};

// packed layout [K / 16][9][2][N][8]: element e holds input channel
// 16 kc + 8 g + k8 of output channel n for tap `tap` (the forward weights:
// K = cin_pad, N = cout; the data gradient's: K = cout, N = cin_pad, taps
// flipped), so that a chunk's rows of 8 channels for a block of N are one
// contiguous run
__global__ void k_pack_all(PackTable t, const float* p, bf16* wf, bf16* wd) {
  const int L = blockIdx.y;
  const int cin = t.cin[L], cinp = t.cin_pad[L], cout = t.cout[L];
  const float* W = p + t.w_off[L];
  const long long nf = (long long)cinp * 9 * cout;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nf;
       e += (long long)gridDim.x * blockDim.x) {
    const int k8 = (int)(e & 7);
    long long r = e >> 3;
    const int co = (int)(r % cout);
    r /= cout;
    const int g = (int)(r & 1);
    r >>= 1;
    const int tap = (int)(r % 9);
    const int kc = (int)(r / 9);
    const int ci = kc * 16 + g * 8 + k8;
    wf[t.wf_off[L] + e] = __float2bfloat16_rn(ci < cin ? W[((long long)co * cin + ci) * 9 + tap] : 0.0f);
  }
  if (t.wd_off[L] < 0) return;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nf;
       e += (long long)gridDim.x * blockDim.x) {
    const int k8 = (int)(e & 7);
    long long r = e >> 3;
    const int ci = (int)(r % cinp);
    r /= cinp;
    const int g = (int)(r & 1);
    r >>= 1;
    const int tapd = (int)(r % 9);
    const int kc = (int)(r / 9);
    const int co = kc * 16 + g * 8 + k8;
    wd[t.wd_off[L] + e] =
        __float2bfloat16_rn(ci < cin ? W[((long long)co * cin + ci) * 9 + (8 - tapd)] : 0.0f);
  }
}

int grid1(long long n, int threads) {
  long long g = (n + threads - 1) / threads;
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct ULayerInfo {
  int cin, cin_pad, cout;
  long long w_off, b_off, wf_off, wd_off;
};

struct UNet {
  int nr, nz, bmax;
  int n_inst = 1;              // instances served (forward batch of a step)
  int H[kLev], W[kLev];
  double v_ref;
  ULayerInfo L[kNumLayers];
  PackTable pack;
  long long np = 0, nwf = 0, nwd = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  bf16 *wf = nullptr, *wd = nullptr;
  bf16* x_in = nullptr;
  bf16 *ea[kLev] = {}, *cat[kLev - 1] = {}, *h3 = nullptr, *da[kLev - 1] = {}, *db[kLev - 1] = {};
  bf16 *g_ea[kLev] = {}, *g_cat[kLev - 1] = {}, *g_h3 = nullptr, *g_da[kLev - 1] = {},
       *g_db[kLev - 1] = {};
  float *out = nullptr, *y = nullptr, *xs = nullptr;
  float* part = nullptr;       // weight-gradient partials
  double* red = nullptr;       // head partials
  int red_blocks = 0;
  double* d_loss = nullptr;    // per-iteration losses of a training call
  long long d_loss_len = 0;
  UDev* ud = nullptr;
  double* gpart = nullptr;     // guess-selection partials
  int gblk = 0;
  int mode = 0;
  // per instance k at offset k * npx(0) (gpart: k * gblk * 3, scale: k)
  double* cand = nullptr;      // candidate start (FP64 node array)
  float* res = nullptr;        // residual of the previous solution (mode 1)
  double* phi_prev = nullptr;  // previous solution (mode-1 recording)
  double* scale = nullptr;     // mode 1: RMS of the live residual of this step
  int* choice = nullptr;       // start chosen for each instance's solve
  float *snap_f0 = nullptr, *snap_f1 = nullptr;
  float* slot_scale = nullptr;  // mode 1: residual RMS of each snapshot
  long long snap_cap = 0;
  int snap_every = 1;
  bool rec_on = true;          // recording into the ring (paused by unet_set_record)
  int bc_g = 0, bc_wall = 0;   // insulating boundary nodes (field_free), set at creation
  bool warm = false;
  long long adam_t = 0;
  int wg_ctas[3] = {0, 0, 0};  // resident weight-gradient CTAs (COUT 16, 32, 64), at most kMaxSplit
  long long tc_ctas[4] = {1, 1, 1, 1};   // resident forward-convolution CTAs (COB 16, 32, 48, 64)
  UAllocFn alloc = nullptr;
  void* actx = nullptr;
  long long npx(int l) const { return (long long)H[l] * W[l]; }
};

namespace {

void* ua(UNet* u, size_t bytes) { return u->alloc(u->actx, bytes); }

int cob_for(int cout) {
  if (cout % 64 == 0) return 64;
  if (cout % 48 == 0) return 48;
  if (cout % 32 == 0) return 32;
  return 16;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// A 4-D BF16 tensor map (channels, columns, rows, batch) over node-major
// activations: `cs` channels per node, nodes `step` apart along a row of
// `row` buffer nodes, rows `step` apart, images `bs` elements apart; box of
// bc channels x bw columns x bh rows x 1 image, zero fill outside.  Every
// stride is a multiple of 16 bytes because cs is a multiple of 8.
bool tensor_map4(CUtensorMap* m, const bf16* base, int cs, int W, int H, int B, int step, int row,
                 long long bs, int bc, int bw, int bh) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn || cs % 8 || bc % 8) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)cs, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
  const cuuint64_t strides[3] = {(cuuint64_t)step * cs * 2, (cuuint64_t)step * row * cs * 2,
                                 (cuuint64_t)bs * 2};
  const cuuint32_t box[4] = {(cuuint32_t)bc, (cuuint32_t)bw, (cuuint32_t)bh, 1u};
  const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void*)base, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t run_conv(UNet* u, const ConvArgs& a, cudaStream_t st) {
  const int cob = cob_for(a.cout);
  // the TMA boxes start at channel x_c0 + 16 kc + 8 g: a multiple of 8 (16
  // bytes), as a tiled load's innermost coordinate must be
  if (a.x_c0 % 8) return cudaErrorInvalidValue;
  alignas(64) CUtensorMap tmx;
  if (!tensor_map4(&tmx, a.x, a.x_cs, a.W, a.H, a.B, a.x_step, a.x_w, a.x_bs, 8, kFwTW, kFwTH + 2))
    return cudaErrorInvalidValue;
  const long long items = (long long)a.B * ((a.W + kFwTW - 1) / kFwTW) *
                          ((a.H + kFwTH - 1) / kFwTH) * (a.cout / cob);
  const int q = cob == 64 ? 3 : cob == 48 ? 2 : cob == 32 ? 1 : 0;
  const long long grid = items < u->tc_ctas[q] ? items : u->tc_ctas[q];
  switch (cob) {
    case 64: k_conv3_tc<64><<<(unsigned)grid, kTcThreads, tc_smem(64), st>>>(a, tmx); break;
    case 48: k_conv3_tc<48><<<(unsigned)grid, kTcThreads, tc_smem(48), st>>>(a, tmx); break;
    case 32: k_conv3_tc<32><<<(unsigned)grid, kTcThreads, tc_smem(32), st>>>(a, tmx); break;
    default: k_conv3_tc<16><<<(unsigned)grid, kTcThreads, tc_smem(16), st>>>(a, tmx); break;
  }
  return cudaGetLastError();
}

// forward conv of layer L
cudaError_t conv_fwd(UNet* u, int Lx, const bf16* x, long long x_bs, int x_cs, int x_c0, int x_step,
                     int x_w, bf16* y, long long y_bs, int y_cs, int y_c0, int H, int W, int B,
                     cudaStream_t st) {
  const ULayerInfo& L = u->L[Lx];
  ConvArgs a;
  a.x = x; a.x_bs = x_bs; a.x_cs = x_cs; a.x_c0 = x_c0; a.x_step = x_step; a.x_w = x_w;
  a.w = u->wf + L.wf_off; a.bias = u->p + L.b_off; a.cin = L.cin_pad; a.cout = L.cout;
  a.y = y; a.y_bs = y_bs; a.y_cs = y_cs; a.y_c0 = y_c0; a.y_step = 1; a.y_w = W;
  a.H = H; a.W = W; a.B = B; a.relu = 1; a.accumulate = 0; a.err = &u->ud->err;
  return run_conv(u, a, st);
}

// data gradient of layer L: dz (node step 1) -> dx (node step dx_step)
cudaError_t conv_dgrad(UNet* u, int Lx, const bf16* dz, long long dz_bs, int dz_cs, int dz_c0,
                       bf16* dx, long long dx_bs, int dx_cs, int dx_c0, int dx_step, int dx_w,
                       int H, int W, int B, bool accumulate, cudaStream_t st) {
  const ULayerInfo& L = u->L[Lx];
  ConvArgs a;
  a.x = dz; a.x_bs = dz_bs; a.x_cs = dz_cs; a.x_c0 = dz_c0; a.x_step = 1; a.x_w = W;
  a.w = u->wd + L.wd_off; a.bias = nullptr; a.cin = L.cout; a.cout = L.cin_pad;
  a.y = dx; a.y_bs = dx_bs; a.y_cs = dx_cs; a.y_c0 = dx_c0; a.y_step = dx_step; a.y_w = dx_w;
  a.H = H; a.W = W; a.B = B; a.relu = 0; a.accumulate = accumulate ? 1 : 0; a.err = &u->ud->err;
  return run_conv(u, a, st);
}

cudaError_t conv_wgrad(UNet* u, int Lx, const bf16* x, long long x_bs, int x_cs, int x_c0,
                       int x_step, int x_w, const bf16* dz, long long dz_bs, int dz_cs, int dz_c0,
                       int H, int W, int B, cudaStream_t st) {
  const ULayerInfo& L = u->L[Lx];
  WgArgs a;
  a.x = x; a.x_bs = x_bs; a.x_cs = x_cs; a.x_c0 = x_c0; a.x_step = x_step; a.x_w = x_w;
  a.dz = dz; a.dz_bs = dz_bs; a.dz_cs = dz_cs; a.dz_c0 = dz_c0;
  a.cin = L.cin_pad; a.H = H; a.W = W; a.B = B;
  a.pw = u->part;
  a.pb = u->part + (long long)kMaxSplit * 9 * 16 * 64;
  a.err = &u->ud->err;
  const int nkc = L.cin_pad >> 4;
  const long long T = (long long)B * ((H + kWgTH - 1) / kWgTH) * ((W + kWgTW - 1) / kWgTW);
  const int ctas = L.cout == 64 ? u->wg_ctas[2] : L.cout == 32 ? u->wg_ctas[1] : u->wg_ctas[0];
  long long S = ctas / nkc;
  if (S > T) S = T;
  if (S < 1) S = 1;
  const dim3 grid(nkc, (unsigned)S);
  // the TMA boxes start at channels x_c0 + 16 kc and dz_c0: multiples of 8
  // (16 bytes), as a tiled load's innermost coordinate must be
  if (x_c0 % 8 || dz_c0 % 8) return cudaErrorInvalidValue;
  alignas(64) CUtensorMap tmx, tmd;
  if (!tensor_map4(&tmx, x, x_cs, W, H, B, x_step, x_w, x_bs, 16, kWgPW, kWgPH) ||
      !tensor_map4(&tmd, dz, dz_cs, W, H, B, 1, W, dz_bs, L.cout, kWgTW, kWgTH))
    return cudaErrorInvalidValue;
  switch (L.cout) {
    case 64: k_conv3_wgrad<64><<<grid, kWgThreads, wg_smem(64), st>>>(a, tmx, tmd); break;
    case 32: k_conv3_wgrad<32><<<grid, kWgThreads, wg_smem(32), st>>>(a, tmx, tmd); break;
    default: k_conv3_wgrad<16><<<grid, kWgThreads, wg_smem(16), st>>>(a, tmx, tmd); break;
  }
  const long long n = (long long)(L.cin_pad >> 4) * 9 * L.cout * 16 + L.cout;
  k_wgrad_reduce<<<(unsigned)((n + kRedE - 1) / kRedE), kRedE * kRedG, 0, st>>>(
      a.pw, a.pb, (int)S, L.cin, L.cin_pad, L.cout, u->g + L.w_off, u->g + L.b_off);
  return cudaGetLastError();
}

cudaError_t relu_mask(bf16* g, int g_cs, int g_c0, const bf16* y, int y_cs, int y_c0, int C,
                      long long npx, cudaStream_t st) {
  k_relu_mask<<<grid1(npx * (C / 8), 256), 256, 0, st>>>(g, g_cs, g_c0, y, y_cs, y_c0, C, npx);
  return cudaGetLastError();
}

// channel counts of the level buffers
int cat_cs(int l) { return kCh[l + 1] + kCh[l]; }

cudaError_t forward(UNet* u, int B, cudaStream_t st) {
  const int* H = u->H;
  const int* W = u->W;
  cudaError_t e;
  // encoder
  e = conv_fwd(u, 0, u->x_in, u->npx(0) * kInPad, kInPad, 0, 1, W[0], u->ea[0], u->npx(0) * kCh[0],
               kCh[0], 0, H[0], W[0], B, st);
  if (e) return e;
  e = conv_fwd(u, 1, u->ea[0], u->npx(0) * kCh[0], kCh[0], 0, 1, W[0], u->cat[0],
               u->npx(0) * cat_cs(0), cat_cs(0), kCh[1], H[0], W[0], B, st);
  if (e) return e;
  for (int l = 1; l < kLev; ++l) {
    e = conv_fwd(u, 2 * l, u->cat[l - 1], u->npx(l - 1) * cat_cs(l - 1), cat_cs(l - 1), kCh[l], 2,
                 W[l - 1], u->ea[l], u->npx(l) * kCh[l], kCh[l], 0, H[l], W[l], B, st);
    if (e) return e;
    if (l < kLev - 1)
      e = conv_fwd(u, 2 * l + 1, u->ea[l], u->npx(l) * kCh[l], kCh[l], 0, 1, W[l], u->cat[l],
                   u->npx(l) * cat_cs(l), cat_cs(l), kCh[l + 1], H[l], W[l], B, st);
    else
      e = conv_fwd(u, 2 * l + 1, u->ea[l], u->npx(l) * kCh[l], kCh[l], 0, 1, W[l], u->h3,
                   u->npx(l) * kCh[l], kCh[l], 0, H[l], W[l], B, st);
    if (e) return e;
  }
  // decoder
  const bf16* src = u->h3;
  int src_c = kCh[kLev - 1];
  for (int l = kLev - 2; l >= 0; --l) {
    const long long n = (long long)B * u->npx(l) * (src_c / 8);
    k_up<<<grid1(n, 256), 256, 0, st>>>(src, src_c, 0, H[l + 1], W[l + 1], u->cat[l], cat_cs(l), 0,
                                        H[l], W[l], src_c, B);
    const int la = 8 + 2 * (kLev - 2 - l), lb = la + 1;
    e = conv_fwd(u, la, u->cat[l], u->npx(l) * cat_cs(l), cat_cs(l), 0, 1, W[l], u->da[l],
                 u->npx(l) * kCh[l], kCh[l], 0, H[l], W[l], B, st);
    if (e) return e;
    e = conv_fwd(u, lb, u->da[l], u->npx(l) * kCh[l], kCh[l], 0, 1, W[l], u->db[l],
                 u->npx(l) * kCh[l], kCh[l], 0, H[l], W[l], B, st);
    if (e) return e;
    src = u->db[l];
    src_c = kCh[l];
  }
  const ULayerInfo& Lh = u->L[kHead];
  const long long n0 = (long long)B * u->npx(0);
  k_head_fwd<<<grid1(n0, 256), 256, 0, st>>>(u->db[0], u->p + Lh.w_off, u->p + Lh.b_off, u->out, n0);
  return cudaGetLastError();
}

// backward from the MSE loss against u->y; the loss lands in *d_loss
cudaError_t backward(UNet* u, int B, double* d_loss, cudaStream_t st) {
  const int* H = u->H;
  const int* W = u->W;
  cudaError_t e;
  const ULayerInfo& Lh = u->L[kHead];
  const long long n0 = (long long)B * u->npx(0);
  const double inv_n = 1.0 / (double)n0;
  k_head_bwd<<<u->red_blocks, 256, 0, st>>>(u->db[0], u->p + Lh.w_off, u->out, u->y, u->g_db[0],
                                            n0, inv_n, u->red);
  k_head_final<<<1, 32, 0, st>>>(u->red, u->red_blocks, inv_n, d_loss, u->g + Lh.w_off,
                                 u->g + Lh.b_off);
  // decoder, level 0 first
  for (int l = 0; l < kLev - 1; ++l) {
    const int la = 8 + 2 * (kLev - 2 - l), lb = la + 1;
    const long long np = (long long)B * u->npx(l);
    const long long bs = u->npx(l) * kCh[l];
    e = relu_mask(u->g_db[l], kCh[l], 0, u->db[l], kCh[l], 0, kCh[l], np, st);
    if (e) return e;
    e = conv_wgrad(u, lb, u->da[l], bs, kCh[l], 0, 1, W[l], u->g_db[l], bs, kCh[l], 0, H[l], W[l], B, st);
    if (e) return e;
    e = conv_dgrad(u, lb, u->g_db[l], bs, kCh[l], 0, u->g_da[l], bs, kCh[l], 0, 1, W[l], H[l], W[l],
                   B, false, st);
    if (e) return e;
    e = relu_mask(u->g_da[l], kCh[l], 0, u->da[l], kCh[l], 0, kCh[l], np, st);
    if (e) return e;
    const long long cbs = u->npx(l) * cat_cs(l);
    e = conv_wgrad(u, la, u->cat[l], cbs, cat_cs(l), 0, 1, W[l], u->g_da[l], bs, kCh[l], 0, H[l],
                   W[l], B, st);
    if (e) return e;
    e = conv_dgrad(u, la, u->g_da[l], bs, kCh[l], 0, u->g_cat[l], cbs, cat_cs(l), 0, 1, W[l], H[l],
                   W[l], B, false, st);
    if (e) return e;
    // up-sampling transpose into the coarse source's gradient
    bf16* gsrc = l + 1 < kLev - 1 ? u->g_db[l + 1] : u->g_h3;
    const int C = kCh[l + 1];
    const long long n = (long long)B * u->npx(l + 1) * (C / 8);
    k_up_t<<<grid1(n, 256), 256, 0, st>>>(u->g_cat[l], cat_cs(l), 0, H[l], W[l], gsrc, C, 0,
                                          H[l + 1], W[l + 1], C, B);
  }
  // encoder, bottom level first
  for (int l = kLev - 1; l >= 0; --l) {
    const long long np = (long long)B * u->npx(l);
    const long long bs = u->npx(l) * kCh[l];
    bf16 *yo, *go;
    int o_cs, o_c0;
    if (l == kLev - 1) {
      yo = u->h3; go = u->g_h3; o_cs = kCh[l]; o_c0 = 0;
    } else {
      yo = u->cat[l]; go = u->g_cat[l]; o_cs = cat_cs(l); o_c0 = kCh[l + 1];
    }
    const long long obs = u->npx(l) * o_cs;
    e = relu_mask(go, o_cs, o_c0, yo, o_cs, o_c0, kCh[l], np, st);
    if (e) return e;
    e = conv_wgrad(u, 2 * l + 1, u->ea[l], bs, kCh[l], 0, 1, W[l], go, obs, o_cs, o_c0, H[l], W[l],
                   B, st);
    if (e) return e;
    e = conv_dgrad(u, 2 * l + 1, go, obs, o_cs, o_c0, u->g_ea[l], bs, kCh[l], 0, 1, W[l], H[l], W[l],
                   B, false, st);
    if (e) return e;
    e = relu_mask(u->g_ea[l], kCh[l], 0, u->ea[l], kCh[l], 0, kCh[l], np, st);
    if (e) return e;
    if (l == 0) {
      e = conv_wgrad(u, 0, u->x_in, u->npx(0) * kInPad, kInPad, 0, 1, W[0], u->g_ea[0], bs, kCh[0], 0,
                     H[0], W[0], B, st);
      if (e) return e;
    } else {
      const long long pbs = u->npx(l - 1) * cat_cs(l - 1);
      e = conv_wgrad(u, 2 * l, u->cat[l - 1], pbs, cat_cs(l - 1), kCh[l], 2, W[l - 1], u->g_ea[l], bs,
                     kCh[l], 0, H[l], W[l], B, st);
      if (e) return e;
      e = conv_dgrad(u, 2 * l, u->g_ea[l], bs, kCh[l], 0, u->g_cat[l - 1], pbs, cat_cs(l - 1), kCh[l],
                     2, W[l - 1], H[l], W[l], B, true, st);
      if (e) return e;
    }
  }
  return cudaGetLastError();
}

cudaError_t pack_weights(UNet* u, cudaStream_t st) {
  k_pack_all<<<dim3(64, kNumConv), 256, 0, st>>>(u->pack, u->p, u->wf, u->wd);
  return cudaGetLastError();
}

}  // namespace

long long unet_param_count() {
  long long n = 0;
  int ci[kNumConv], co[kNumConv];
  for (int l = 0; l < kLev; ++l) {
    ci[2 * l] = l == 0 ? kInReal : kCh[l - 1];
    co[2 * l] = kCh[l];
    ci[2 * l + 1] = kCh[l];
    co[2 * l + 1] = kCh[l];
  }
  for (int l = kLev - 2, k = 8; l >= 0; --l, k += 2) {
    ci[k] = kCh[l + 1] + kCh[l];
    co[k] = kCh[l];
    ci[k + 1] = kCh[l];
    co[k + 1] = kCh[l];
  }
  for (int k = 0; k < kNumConv; ++k) n += (long long)co[k] * ci[k] * 9 + co[k];
  return n + kCh[0] + 1;
}

UNet* unet_create(int nr, int nz, int bmax, int n_inst, int mode, unsigned long long seed,
                  double v_ref, UAllocFn alloc, void* ctx, cudaStream_t st) {
  if (nr % 8 || nz % 8 || nr < 8 || nz < 8 || bmax < 1 || n_inst < 1 || !alloc || mode < 0 ||
      mode > 1)
    return nullptr;
  UNet* u = new UNet();
  u->mode = mode;
  u->nr = nr;
  u->nz = nz;
  u->bmax = bmax;
  u->n_inst = n_inst;
  u->v_ref = v_ref > 0.0 ? v_ref : 1.0;
  u->bc_g = nr + 1;
  u->alloc = alloc;
  u->actx = ctx;
  for (int l = 0; l < kLev; ++l) {
    u->H[l] = (nr >> l) + 1;
    u->W[l] = (nz >> l) + 1;
  }
  // layer table in the reference order
  int ci[kNumLayers], co[kNumLayers];
  for (int l = 0; l < kLev; ++l) {
    ci[2 * l] = l == 0 ? kInReal : kCh[l - 1];
    co[2 * l] = kCh[l];
    ci[2 * l + 1] = kCh[l];
    co[2 * l + 1] = kCh[l];
  }
  for (int l = kLev - 2, k = 8; l >= 0; --l, k += 2) {
    ci[k] = kCh[l + 1] + kCh[l];
    co[k] = kCh[l];
    ci[k + 1] = kCh[l];
    co[k + 1] = kCh[l];
  }
  ci[kHead] = kCh[0];
  co[kHead] = 1;
  long long off = 0, of = 0, od = 0;
  for (int k = 0; k < kNumLayers; ++k) {
    ULayerInfo& L = u->L[k];
    L.cin = ci[k];
    L.cin_pad = (ci[k] + 15) / 16 * 16;
    L.cout = co[k];
    L.w_off = off;
    off += (long long)co[k] * ci[k] * (k == kHead ? 1 : 9);
    L.b_off = off;
    off += co[k];
    L.wf_off = L.wd_off = -1;
    if (k < kNumConv) {
      L.wf_off = of;
      of += (long long)L.cin_pad * 9 * L.cout;
      if (k != 0) {
        L.wd_off = od;
        od += (long long)L.cin_pad * 9 * L.cout;
      }
      u->pack.cin[k] = L.cin;
      u->pack.cin_pad[k] = L.cin_pad;
      u->pack.cout[k] = L.cout;
      u->pack.w_off[k] = L.w_off;
      u->pack.wf_off[k] = L.wf_off;
      u->pack.wd_off[k] = L.wd_off;
    }
  }
  u->np = off;
  u->nwf = of;
  u->nwd = od;
  bool ok = true;
  auto A = [&](size_t b) {
    void* p = ua(u, b);
    ok = ok && p;
    return p;
  };
  u->p = (float*)A(u->np * 4);
  u->g = (float*)A(u->np * 4);
  u->m = (float*)A(u->np * 4);
  u->v = (float*)A(u->np * 4);
  u->wf = (bf16*)A(u->nwf * 2);
  u->wd = (bf16*)A(u->nwd * 2);
  const long long B = bmax > n_inst ? bmax : n_inst;   // activations of the larger batch
  u->x_in = (bf16*)A(B * u->npx(0) * kInPad * 2);
  for (int l = 0; l < kLev; ++l) {
    u->ea[l] = (bf16*)A(B * u->npx(l) * kCh[l] * 2);
    u->g_ea[l] = (bf16*)A(B * u->npx(l) * kCh[l] * 2);
  }
  for (int l = 0; l < kLev - 1; ++l) {
    u->cat[l] = (bf16*)A(B * u->npx(l) * cat_cs(l) * 2);
    u->g_cat[l] = (bf16*)A(B * u->npx(l) * cat_cs(l) * 2);
    u->da[l] = (bf16*)A(B * u->npx(l) * kCh[l] * 2);
    u->g_da[l] = (bf16*)A(B * u->npx(l) * kCh[l] * 2);
    u->db[l] = (bf16*)A(B * u->npx(l) * kCh[l] * 2);
    u->g_db[l] = (bf16*)A(B * u->npx(l) * kCh[l] * 2);
  }
  u->h3 = (bf16*)A(B * u->npx(kLev - 1) * kCh[kLev - 1] * 2);
  u->g_h3 = (bf16*)A(B * u->npx(kLev - 1) * kCh[kLev - 1] * 2);
  u->out = (float*)A(B * u->npx(0) * 4);
  u->y = (float*)A(B * u->npx(0) * 4);
  u->xs = (float*)A(B * u->npx(0) * kInReal * 4);
  u->part = (float*)A(((size_t)kMaxSplit * 9 * 16 * 64 + (size_t)kMaxSplit * 64) * 4);
  u->red_blocks = 296;
  u->red = (double*)A((size_t)u->red_blocks * kHeadVals * 8);
  u->d_loss_len = 1;
  u->d_loss = (double*)A(8);
  u->ud = (UDev*)A(sizeof(UDev));
  u->gblk = guess_blocks(nr, nz);
  u->gpart = (double*)A((size_t)n_inst * u->gblk * 3 * 8);
  u->cand = (double*)A((size_t)n_inst * u->npx(0) * 8);
  u->res = (float*)A((size_t)n_inst * u->npx(0) * 4);
  u->phi_prev = (double*)A((size_t)n_inst * u->npx(0) * 8);
  u->scale = (double*)A((size_t)n_inst * 8);
  u->choice = (int*)A((size_t)n_inst * 4);
  if (!ok) {
    delete u;
    return nullptr;
  }
  // He-normal weights, zero biases (std::mt19937_64 + normal_distribution)
  std::vector<float> hp((size_t)u->np, 0.0f);
  std::mt19937_64 rng(seed);
  for (int k = 0; k < kNumLayers; ++k) {
    const ULayerInfo& L = u->L[k];
    const int taps = k == kHead ? 1 : 9;
    std::normal_distribution<double> nd(0.0, std::sqrt(2.0 / (double)(L.cin * taps)));
    for (long long q = 0; q < (long long)L.cout * L.cin * taps; ++q) hp[L.w_off + q] = (float)nd(rng);
  }
  UDev ud0;
  std::memset(&ud0, 0, sizeof(ud0));
  ud0.out_norm = mode == 0 ? u->v_ref : 0.0;
  cudaError_t e = cudaMemcpyAsync(u->p, hp.data(), u->np * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(u->m, 0, u->np * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(u->v, 0, u->np * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(u->g, 0, u->np * 4, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(u->ud, &ud0, sizeof(UDev), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = pack_weights(u, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_conv3_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem(64));
    cudaFuncSetAttribute(k_conv3_tc<48>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem(48));
    cudaFuncSetAttribute(k_conv3_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem(32));
    cudaFuncSetAttribute(k_conv3_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem(16));
    cudaFuncSetAttribute(k_conv3_wgrad<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, wg_smem(64));
    cudaFuncSetAttribute(k_conv3_wgrad<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, wg_smem(32));
    cudaFuncSetAttribute(k_conv3_wgrad<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, wg_smem(16));
    // all of the unified L1 as shared memory, so that the occupancy below is
    // what the launches get
    const void* kerns[7] = {(const void*)k_conv3_tc<64>, (const void*)k_conv3_tc<48>,
                            (const void*)k_conv3_tc<32>, (const void*)k_conv3_tc<16>,
                            (const void*)k_conv3_wgrad<64>, (const void*)k_conv3_wgrad<32>,
                            (const void*)k_conv3_wgrad<16>};
    for (const void* k : kerns)
      cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared);
    attr = true;
  }
  {
    // resident weight-gradient CTAs per SM: by threads, registers, shared
    // memory and the 512 TMEM columns of an SM
    int dev = 0, sms = 1, smem_sm = 0, smem_rsv = 0, regs_sm = 65536;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    const void* wk[3] = {(const void*)k_conv3_wgrad<16>, (const void*)k_conv3_wgrad<32>,
                         (const void*)k_conv3_wgrad<64>};
    const int wsm[3] = {wg_smem(16), wg_smem(32), wg_smem(64)};
    const int tcols[3] = {(int)wg_tcols(16), (int)wg_tcols(32), (int)wg_tcols(64)};
    const void* tk[4] = {(const void*)k_conv3_tc<16>, (const void*)k_conv3_tc<32>,
                         (const void*)k_conv3_tc<48>, (const void*)k_conv3_tc<64>};
    const int tsm[4] = {tc_smem(16), tc_smem(32), tc_smem(48), tc_smem(64)};
    const int tcc[4] = {tc_tcols(16), tc_tcols(32), tc_tcols(48), tc_tcols(64)};
    for (int q = 0; q < 4; ++q) {
      cudaFuncAttributes fa;
      int regs = 64;
      if (cudaFuncGetAttributes(&fa, tk[q]) == cudaSuccess && fa.numRegs > 0) regs = fa.numRegs;
      int per_sm = 2048 / kTcThreads;
      const int by_regs = regs_sm / (((regs + 7) / 8 * 8) * kTcThreads);
      const int by_smem = smem_sm > 0 ? smem_sm / (tsm[q] + smem_rsv) : 1;
      per_sm = by_regs < per_sm ? by_regs : per_sm;
      per_sm = by_smem < per_sm ? by_smem : per_sm;
      per_sm = 512 / tcc[q] < per_sm ? 512 / tcc[q] : per_sm;
      if (per_sm < 1) per_sm = 1;
      u->tc_ctas[q] = (long long)per_sm * (sms > 0 ? sms : 1);
    }
    for (int q = 0; q < 3; ++q) {
      cudaFuncAttributes fa;
      int regs = 64;
      if (cudaFuncGetAttributes(&fa, wk[q]) == cudaSuccess && fa.numRegs > 0) regs = fa.numRegs;
      int per_sm = 2048 / kWgThreads;
      const int by_regs = regs_sm / (((regs + 7) / 8 * 8) * kWgThreads);
      const int by_smem = smem_sm > 0 ? smem_sm / (wsm[q] + smem_rsv) : 1;
      per_sm = by_regs < per_sm ? by_regs : per_sm;
      per_sm = by_smem < per_sm ? by_smem : per_sm;
      per_sm = 512 / tcols[q] < per_sm ? 512 / tcols[q] : per_sm;
      if (per_sm < 1) per_sm = 1;
      const int c = per_sm * (sms > 0 ? sms : 1);
      u->wg_ctas[q] = c < kMaxSplit ? c : kMaxSplit;
    }
  }
  if (e != cudaSuccess) {
    delete u;
    return nullptr;
  }
  return u;
}

void unet_destroy(UNet* u) { delete u; }
void unet_set_boundary(UNet* u, int g, int wall) {
  u->bc_g = g;
  u->bc_wall = wall ? 1 : 0;
}

int unet_mode(const UNet* u) { return u->mode; }
int unet_bmax(const UNet* u) { return u->bmax; }
UDev* unet_dev(UNet* u) { return u->ud; }

// the tensor-core kernels' error word (a completion wait reached its limit)
cudaError_t unet_check_err(UNet* u, cudaStream_t st) {
  int err = 0;
  cudaError_t e = cudaMemcpyAsync(&err, &u->ud->err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && err) e = cudaErrorTimeout;
  return e;
}

cudaError_t unet_set_params(UNet* u, const float* host, cudaStream_t st) {
  cudaError_t e = cudaMemcpyAsync(u->p, host, u->np * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = pack_weights(u, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

cudaError_t unet_get_params(UNet* u, float* host, cudaStream_t st) {
  cudaError_t e = cudaMemcpyAsync(host, u->p, u->np * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

cudaError_t unet_loss_grad(UNet* u, int B, const float* x, const float* y, float* out, float* grad,
                           double* loss, cudaStream_t st) {
  if (B < 1 || B > u->bmax) return cudaErrorInvalidValue;
  const long long n0 = (long long)B * u->npx(0);
  cudaError_t e = cudaMemcpyAsync(u->xs, x, n0 * kInReal * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && y) e = cudaMemcpyAsync(u->y, y, n0 * 4, cudaMemcpyHostToDevice, st);
  if (e) return e;
  k_pack_input<<<grid1(n0, 256), 256, 0, st>>>(u->xs, B, u->H[0], u->W[0], u->x_in);
  e = forward(u, B, st);
  if (e == cudaSuccess && y) e = backward(u, B, u->d_loss, st);
  if (e == cudaSuccess && out) e = cudaMemcpyAsync(out, u->out, n0 * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && y && grad) e = cudaMemcpyAsync(grad, u->g, u->np * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && y && loss) e = cudaMemcpyAsync(loss, u->d_loss, 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = unet_check_err(u, st);
  return e;
}

cudaError_t unet_snapshots(UNet* u, long long cap, int every, UAllocFn alloc, void* ctx) {
  if (cap < 1 || every < 1) return cudaErrorInvalidValue;
  const size_t bytes = (size_t)cap * u->npx(0) * 4;
  float* a = (float*)alloc(ctx, bytes);
  float* b = (float*)alloc(ctx, bytes);
  float* c = (float*)alloc(ctx, (size_t)cap * 4);
  if (!a || !b || !c) return cudaErrorMemoryAllocation;
  u->snap_f0 = a;
  u->snap_f1 = b;
  u->slot_scale = c;
  u->snap_cap = cap;
  u->snap_every = every;
  return cudaSuccess;
}

bool unet_recording(const UNet* u) { return u->snap_cap > 0; }

static bool rec_live(const UNet* u) { return u->snap_cap > 0 && u->rec_on; }
void unet_set_record(UNet* u, bool on) { u->rec_on = on; }
bool unet_pre_solve_needed(const UNet* u) { return u->warm || (u->mode == 1 && rec_live(u)); }

cudaError_t launch_pre_solve(UNet* u, const Inst* d_insts, const void* d_pargs, int n,
                             cudaStream_t st) {
  if (n < 1 || n > u->n_inst) return cudaErrorInvalidValue;
  const long long npx = u->npx(0);
  const dim3 g0(grid1(npx, 256), n);
  cudaError_t e = cudaSuccess;
  if (u->mode == 1) {
    e = launch_residual32(d_pargs, n, u->nr, u->nz, u->res, st);
    if (e) return e;
    if (rec_live(u)) {
      k_snap_pre<<<g0, 256, 0, st>>>(d_insts, u->ud, u->res, u->snap_f0, u->phi_prev, u->snap_cap,
                                     u->snap_every);
      k_slot_rms<<<n, 1024, 0, st>>>(d_insts, u->ud, u->snap_f0, u->slot_scale, u->snap_cap,
                                     u->snap_every);
    }
    if (u->warm) k_live_rms<<<n, 1024, 0, st>>>(u->res, npx, u->scale);
  }
  if (!u->warm) return cudaGetLastError();
  // the inputs of all instances as one batch of the forward pass
  k_step_input<<<g0, 256, 0, st>>>(d_insts, u->ud, u->mode, u->res, u->scale, u->x_in);
  e = forward(u, n, st);
  if (e) return e;
  k_make_cand<<<g0, 256, 0, st>>>(d_insts, u->out, u->ud, u->scale, u->mode, u->cand);
  e = launch_gs_sweeps(d_pargs, n, u->nr, u->nz, u->cand, 2, st);
  if (e) return e;
  return launch_guess_select(d_pargs, n, u->nr, u->nz, u->cand, u->gpart, u->ud, u->choice, st);
}

cudaError_t launch_after_solve(UNet* u, const Inst* d_insts, int n, cudaStream_t st) {
  if (n < 1 || n > u->n_inst) return cudaErrorInvalidValue;
  const dim3 g0(grid1(u->npx(0), 256), n);
  if (rec_live(u)) {
    if (u->mode == 0)
      k_snap_record<<<g0, 256, 0, st>>>(d_insts, u->ud, u->snap_f0, u->snap_f1, u->snap_cap,
                                        u->snap_every);
    else
      k_snap_post<<<g0, 256, 0, st>>>(d_insts, u->ud, u->snap_f1, u->phi_prev, u->snap_cap,
                                      u->snap_every);
  }
  k_after_solve<<<1, 32, 0, st>>>(d_insts, n, u->ud, u->snap_every, rec_live(u) ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t unet_train(UNet* u, int iters, int batch, float lr, unsigned long long seed,
                       double* loss_first, double* loss_last, cudaStream_t st) {
  if (iters < 1 || batch < 1 || batch > u->bmax || u->snap_cap <= 0) return cudaErrorInvalidValue;
  UDev ud;
  cudaError_t e = cudaMemcpyAsync(&ud, u->ud, sizeof(UDev), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e) return e;
  const long long avail = ud.snap_count < u->snap_cap ? ud.snap_count : u->snap_cap;
  if (avail < 1) return cudaErrorInvalidValue;
  if (ud.in_norm <= 0.0) {
    const long long n = avail * u->npx(0);
    const int nb = 592;
    k_ms_partial<<<nb, 256, 0, st>>>(u->snap_f0, n, u->red);
    k_norm_set<<<1, 32, 0, st>>>(u->red, nb, n, &u->ud->in_norm);
    if (u->mode == 1) {
      k_ms_partial<<<nb, 256, 0, st>>>(u->snap_f1, n, u->red);
      k_norm_set<<<1, 32, 0, st>>>(u->red, nb, n, &u->ud->out_norm);
    }
  }
  if (u->d_loss_len < iters) {
    double* d = (double*)ua(u, (size_t)iters * 8);
    if (!d) return cudaErrorMemoryAllocation;
    u->d_loss = d;
    u->d_loss_len = iters;
  }
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const long long n0 = (long long)batch * u->npx(0);
  for (int it = 0; it < iters && e == cudaSuccess; ++it) {
    k_train_input<<<grid1(n0, 256), 256, 0, st>>>(u->snap_f0, u->snap_f1, u->slot_scale, avail,
                                                  batch, seed, it, u->nr, u->nz, u->bc_g,
                                                  u->bc_wall, u->mode, u->ud, u->x_in, u->y);
    e = forward(u, batch, st);
    if (e == cudaSuccess) e = backward(u, batch, u->d_loss + it, st);
    if (e != cudaSuccess) break;
    ++u->adam_t;
    const double t = (double)u->adam_t;
    const float lr_t = (float)(lr * std::sqrt(1.0 - std::pow((double)b2, t)) / (1.0 - std::pow((double)b1, t)));
    k_adam<<<grid1(u->np, 256), 256, 0, st>>>(u->p, u->g, u->m, u->v, u->np, lr_t, b1, b2, eps);
    e = pack_weights(u, st);
  }
  double l0 = 0.0, l1 = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&l0, u->d_loss, 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&l1, u->d_loss + (iters - 1), 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (loss_first) *loss_first = l0;
  if (loss_last) *loss_last = l1;
  if (e == cudaSuccess) e = unet_check_err(u, st);
  return e;
}

void unet_set_warm(UNet* u, bool on) { u->warm = on; }
bool unet_warm(const UNet* u) { return u->warm; }

}  // namespace pic
