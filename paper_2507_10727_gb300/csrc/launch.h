// launch.h -- host-side launchers of the kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace pic {

struct PoissonWork;  // defined in poisson.cu

// optional per-kernel-group event marks around the launches of a step
enum StepGroup {
  G_FIELD = 0, G_PUSH, G_BIRTHS, G_SCAN, G_SCATTER, G_CHARGE, G_CIRCUIT, G_POISSON,
  G_STEP_END, G_WARM, G_COUNT
};
struct StepMarks {
  void (*mark)(void* ctx, int group, bool begin, cudaStream_t st);
  void* ctx;
};

// optional launches around the Poisson solve of a step (the learned warm
// start before it, snapshot recording after it)
struct StepHooks {
  cudaError_t (*pre_poisson)(void* ctx, const Inst& I, PoissonWork* pw, cudaStream_t st);
  cudaError_t (*post_poisson)(void* ctx, const Inst& I, cudaStream_t st);
  void* ctx;
};

// one time step of one instance (all kernels of the step, in order); the push
// runs over the work queue q with the device copy d_inst of I
cudaError_t launch_step(const Inst& I, PoissonWork* pw, int num_sms, cudaStream_t st,
                        const StepMarks* marks, const StepHooks* hooks, const Inst* d_inst,
                        WorkQueue* q, int ppt);

// sort the particles of species `sp` currently in cur[sp] into nxt[sp]
// (keys, histogram, scan, scatter); the caller swaps cur/nxt afterwards
cudaError_t launch_sort_species(const Inst& I, int sp, int num_sms, cudaStream_t st);

// re-weighting between steps: keep each particle with probability 1/factor
// (per-id draw, stream 5 of the current step), both species, re-sorted; the
// caller multiplies the weight
cudaError_t launch_thin(const Inst& I, int factor, int num_sms, cudaStream_t st);
cudaError_t launch_thin32(const Inst& I, int sp, int factor, int num_sms, cudaStream_t st);

// region diagnostics: add one sample of the current state (both species and
// phi) to the accumulators; evaluate the accumulated samples into reg.out,
// reg.zs, reg.zb
cudaError_t launch_region_sample(const Inst& I, int num_sms, cudaStream_t st);
cudaError_t launch_region_eval(const Inst& I, cudaStream_t st);

// ids of the step's births (both species, both precisions)
cudaError_t launch_births(const Inst& I, int num_sms, cudaStream_t st);

// load FP64 particles: r, z, v_r, v_theta, v_z, id from device-addressable
// memory (device or page-locked host) into the particle arrays, positions
// converted to cell units; with src == dst for the last four (already copied)
// only the positions are converted in place
cudaError_t launch_copy_in(const void* const src[6], void* const dst[6], long long n,
                           const Inst& I, int num_sms, cudaStream_t st);
// FP64 positions in cell units -> SI into device-addressable r, z (either null)
cudaError_t launch_positions_out(const Inst& I, const double* rc, const double* zc, double* r,
                                 double* z, long long n, int num_sms, cudaStream_t st);

// set the particle count of species sp (set-up)
cudaError_t launch_set_n(const Inst& I, int sp, long long n, cudaStream_t st);

// deposit the current particles, set the cathode values and solve phi
cudaError_t launch_solve_fields(const Inst& I, PoissonWork* pw, int num_sms, cudaStream_t st);

// ensemble pieces: field tables, batched pushes over a work queue, the
// per-instance rest of the step
cudaError_t launch_field_tables(const Inst& I, int num_sms, cudaStream_t st);
cudaError_t launch_queue_setup(const Inst* d_insts, WorkQueue* q, int n_inst, long long chunk,
                               cudaStream_t st);
// the push of both species of every instance over the work queue (plain:
// every instance has the push on, tent weights in r and absorbing walls)
cudaError_t launch_push_all(const Inst* d_insts, WorkQueue* q, int prec32, int gather, bool plain,
                            int ppt, int num_sms, cudaStream_t st);
cudaError_t launch_push32_all(const Inst* d_insts, WorkQueue* q, int gather, bool plain, int ppt,
                              int num_sms, cudaStream_t st);
// the push of a single-instance handle (the instance a kernel argument)
cudaError_t launch_push_one(const Inst& I, WorkQueue* q, int ppt, int num_sms, cudaStream_t st);
cudaError_t launch_push32_one(const Inst& I, WorkQueue* q, int ppt, int num_sms, cudaStream_t st);
cudaError_t launch_post_push(const Inst& I, int num_sms, cudaStream_t st);
// the per-instance kernels of an ensemble step as one launch each over all
// instances (gridDim.z = instances); extents from the largest instance
struct BatchDims {
  long long cells_max, nodes_max, birth_cap_max;
  int prec32;
  int any_append;   // some instance appends births between full sorts
};
cudaError_t launch_field_tables_batch(const Inst* d_insts, int n_inst, const BatchDims& bd,
                                      int num_sms, cudaStream_t st);
cudaError_t launch_post_push_batch(const Inst* d_insts, int n_inst, const BatchDims& bd,
                                   int num_sms, cudaStream_t st);
cudaError_t launch_step_end_batch(const Inst* d_insts, int n_inst, cudaStream_t st);
cudaError_t launch_scatter32_batch(const Inst* d_insts, int n_inst, int blocks, cudaStream_t st);
cudaError_t launch_append32_batch(const Inst* d_insts, int n_inst, int blocks, cudaStream_t st);
// live particles summed over the instances into *out (device)
cudaError_t launch_live_total(const Inst* d_insts, int n_inst, long long* out, cudaStream_t st);
cudaError_t launch_step_end(const Inst& I, cudaStream_t st);
// all instances' Poisson solves in one cooperative launch (block groups)
cudaError_t launch_poisson_group(PoissonWork* const* pws, const Inst* insts, int n_inst,
                                 void* d_args, int num_sms, cudaStream_t st);
size_t poisson_args_bytes();
cudaError_t poisson_group_upload(PoissonWork* const* pws, const Inst* insts, int n_inst,
                                 void* d_args, int num_sms, cudaStream_t st);

// pieces shared with the FP32 path
cudaError_t launch_scan(const Inst& I, int sp0, int nsp, cudaStream_t st);
cudaError_t launch_commit_n(const Inst& I, int sp, cudaStream_t st);

// FP32 particle path (step32.cu)
cudaError_t launch_pack32(const Inst& I, int sp, long long offset, long long count, const double* r,
                          const double* z, const double* vr, const double* vt, const double* vz,
                          const long long* id, int num_sms, cudaStream_t st);
cudaError_t launch_unpack32(const Inst& I, int sp, long long offset, long long count, double* r,
                            double* z, double* vr, double* vt, double* vz, long long* id,
                            int num_sms, cudaStream_t st);
cudaError_t launch_sort_species32(const Inst& I, int sp, int num_sms, cudaStream_t st);
cudaError_t launch_deposit_all32(const Inst& I, int num_sms, cudaStream_t st);
cudaError_t launch_scatter32(const Inst& I, int num_sms, cudaStream_t st);
cudaError_t launch_append32(const Inst& I, int num_sms, cudaStream_t st);

// compute node charge Q from the fixed-point sums (and clear them)
// node charges from the deposit; `step`: a step's (phi extrapolation when on)
cudaError_t launch_charge(const Inst& I, bool step, cudaStream_t st);

// Poisson workspace
size_t poisson_work_bytes(int nr, int nz);
// g: first free (insulating) node of row z = 0 (nr + 1: none); wall: 1 when
// the wall r = R is insulating
PoissonWork* poisson_work_init(void* base, int nr, int nz, double R, double L, int g, int wall,
                               int num_sms);
void poisson_work_free(PoissonWork* pw);
// sine-transform preconditioner: possible when every boundary node is a
// conductor; its extra workspace; attach it (tables filled, synchronous) --
// later solves of pw use it instead of the multigrid V-cycle
bool poisson_sep_possible(const PoissonWork* pw);
size_t poisson_sep_bytes(int nr, int nz);
cudaError_t poisson_sep_attach(PoissonWork* pw, void* base, int num_sms, cudaStream_t st);
// solve A phi = Q (+ Dirichlet values held in phi's boundary nodes)
cudaError_t launch_poisson(PoissonWork* pw, const double* Q, double* phi, double tol, int max_iter,
                           int* status_dev, int* iters_dev, double* resid_dev, cudaStream_t st);

}  // namespace pic

namespace pic {
// Poisson solve over a caller-provided workspace of poisson_work_bytes(nr, nz)
// bytes at `base` (already cleared); allocates nothing.
cudaError_t launch_poisson_in_place(void* base, int nr, int nz, double R, double L, int g, int wall,
                                    int num_sms, const double* Q, double* phi, double tol,
                                    int max_iter, int* status_dev, int* iters_dev,
                                    double* resid_dev, cudaStream_t st);
}  // namespace pic
