// unet.h -- host interface of the learned Poisson warm start (internal).
//
// A 4-level U-Net on the node grid ((nr >> l) + 1) x ((nz >> l) + 1),
// channels 16, 32, 64, 64, 3x3 convolutions with zero padding, ReLU, even-node
// down-sampling, bilinear node up-sampling, [up, skip] concatenation and a
// 1x1 head.  Activations are BF16 (NHWC, channels innermost), accumulation
// FP32, master parameters FP32 in the layer order enc0a, enc0b, ..., enc3b,
// dec2a, dec2b, dec1a, dec1b, dec0a, dec0b, head (weights (cout, cin, 3, 3)
// then biases for each layer).  Two input/output readings:
//   mode 0 (potential):  x = (rho / in_norm, r / R, Dirichlet value / V_ref)
//                        -> phi / V_ref
//   mode 1 (correction): x = (res / s, r / R, Dirichlet mask)
//                        -> (phi - phi_prev) / (s K),
//                        res = Q - A phi_prev (this step's charge and
//                        electrode values against the previous solution),
//                        s = RMS of res of the same step (the change of phi
//                        is linear in res, so every snapshot is scaled to
//                        unit size), K = out_norm / in_norm (RMS over the
//                        recorded snapshots)
// The guess (mode 0: V_ref * y; mode 1: phi_prev + s K y on the free
// nodes) is smoothed by two red-black Gauss-Seidel sweeps of the FP64 fine
// operator, then competes with phi_prev and zero by residual norm.
//
// One network serves every instance of a handle whose instances share the
// grid and its boundary kinds: the inputs of all instances form one batch of
// the forward pass, each instance keeps its own residual scale, candidate and
// start choice, and every instance records into the one snapshot ring
// (instance k of a recording step into slot count + k).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace pic {

struct PoissonWork;
struct UNet;

// device counters of the warm start (one per handle; counts summed over the
// instances)
struct UDev {
  long long snap_count;     // snapshots recorded so far
  long long n_choice[3];    // solves started from: previous phi, network, zero
  long long iters_total;    // Poisson iterations summed over steps
  double in_norm;           // input scale of channel 0 (set by the first training)
  double out_norm;          // output scale (mode 0: V_ref; mode 1: set by the first training)
  int choice;               // guess used by the last solve
  int err;                  // 1 once a tensor-core wait reached its time limit
};

typedef void* (*UAllocFn)(void* ctx, size_t bytes);

long long unet_param_count();
// nr, nz divisible by 8; bmax = largest training/gradient batch; n_inst =
// instances served (the forward batch of a step); mode 0 / 1
UNet* unet_create(int nr, int nz, int bmax, int n_inst, int mode, unsigned long long seed,
                  double v_ref, UAllocFn alloc, void* ctx, cudaStream_t st);
int unet_mode(const UNet* u);
// insulating boundary nodes of the field (field_free's g and wall): they are
// unknowns of the solve, not Dirichlet inputs of the network
void unet_set_boundary(UNet* u, int g, int wall);
void unet_destroy(UNet* u);
int unet_bmax(const UNet* u);
UDev* unet_dev(UNet* u);

cudaError_t unet_set_params(UNet* u, const float* host, cudaStream_t st);
cudaError_t unet_get_params(UNet* u, float* host, cudaStream_t st);
// forward (and backward when grad != nullptr) on B inputs given in the
// oracle's layout: x (B, 3, H0, W0), y (B, H0, W0), host FP32 arrays
cudaError_t unet_loss_grad(UNet* u, int B, const float* x, const float* y, float* out,
                           float* grad, double* loss, cudaStream_t st);

// snapshot ring of every `every`-th step, `cap` slots of two node fields:
// mode 0 (rho, phi), mode 1 (res, phi - phi_prev)
cudaError_t unet_snapshots(UNet* u, long long cap, int every, UAllocFn alloc, void* ctx);
bool unet_recording(const UNet* u);
// pause (false) / resume (true) the recording into the ring
void unet_set_record(UNet* u, bool on);

// Adam training on the snapshot ring
cudaError_t unet_train(UNet* u, int iters, int batch, float lr, unsigned long long seed,
                       double* loss_first, double* loss_last, cudaStream_t st);

// before the solve: mode-1 recording (residual, previous phi) and, with the
// warm start on, the network guess and the choice of the start
void unet_set_warm(UNet* u, bool on);
bool unet_warm(const UNet* u);
bool unet_pre_solve_needed(const UNet* u);
// before the solves of the n instances of a handle (n at most the network's
// n_inst): d_insts and d_pargs are the handle's device copies of the
// instances and of their solve arguments (only fields fixed at creation are
// read: grid, boundary kinds, Q, phi, the scalars); instance 0's step counter
// is the recording clock of all
cudaError_t launch_pre_solve(UNet* u, const Inst* d_insts, const void* d_pargs, int n,
                             cudaStream_t st);
// after the solves: recording and iteration count bookkeeping
cudaError_t launch_after_solve(UNet* u, const Inst* d_insts, int n, cudaStream_t st);

// operator pieces (poisson.cu), all on the fine FP64 operator of the solve,
// over the n instances of the device PoissonArgs array pargs at once
// (instance k's node fields at offset k (nr+1)(nz+1) of res, x, cand)
// res = Q - A phi on free nodes (0 on Dirichlet nodes), FP32 output
cudaError_t launch_residual32(const void* pargs, int n, int nr, int nz, float* res,
                              cudaStream_t st);
// `sweeps` red-black Gauss-Seidel sweeps on A x = Q (Dirichlet values in x)
cudaError_t launch_gs_sweeps(const void* pargs, int n, int nr, int nz, double* x, int sweeps,
                             cudaStream_t st);
// start of each solve: of x in {phi, cand, 0} (Dirichlet values of phi) the
// one with the smallest residual norm is copied into phi; choice[k] = the
// start of instance k, counts in *ud; partial: n * 3 * guess_blocks doubles
cudaError_t launch_guess_select(const void* pargs, int n, int nr, int nz, const double* cand,
                                double* partial, UDev* ud, int* choice, cudaStream_t st);
int guess_blocks(int nr, int nz);

}  // namespace pic
