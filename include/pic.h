/*
 * pic.h -- C ABI of the GB300 (sm_103a) library for the explicit
 * electrostatic PIC-MCC model of a dc magnetron discharge in 2D (r,z)
 * geometry of arXiv:2507.10727 ("Modeling the Role of Secondary Electron
 * Emission in Direct Current Magnetron Sputtering using Explicit
 * Energy-Conserving Particle-in-Cell Methods").
 *
 * One call of pic_step advances every particle and the field by one or more
 * time steps entirely on the GPU:
 *   E from phi (Section 2: edge-centred E for EC-PIC, nodal E for MC-PIC)
 *   -> gather + Boris push in the static magnetron field (Sections 2, 3)
 *   -> absorbing walls, reflecting axis, ion-induced secondary electrons
 *      with yield gamma at zero velocity (Section 3)
 *   -> null-collision Monte Carlo e-Ar collisions, reactions (1a)-(1c)
 *      (Section 3)
 *   -> births with deterministic ids -> charge deposit with tent functions
 *      (Section 2) divided by the annular node volume
 *   -> external circuit V_c = -V_s + I R_ext (Sections 3, 4, 6)
 *   -> RZ Poisson solve with electrode Dirichlet values and Gauss's law on
 *      the axis (Section 3) by multigrid-preconditioned conjugate gradients.
 *
 * Conventions for every function:
 *   - Return value: PIC_OK (0) or one of the negative PIC_ERR_* codes; the
 *     text of the last error of a handle is pic_last_error().  Nothing throws
 *     or aborts across this boundary.
 *   - Device work runs on the CUDA stream given to pic_create (a cudaStream_t
 *     passed as void*; NULL = legacy default stream).  Calls marked "async"
 *     only enqueue work; device-side failures (capacity, non-convergence,
 *     non-finite values, wait timeouts) are latched in a status word that the
 *     next synchronising call (pic_sync, pic_diagnostics, pic_get_*) returns.
 *     Once a status is latched, later steps do no work.
 *   - Units are SI (m, s, V, kg, C); energies in eV where named so.
 *   - Node arrays are (nr+1) x (nz+1) doubles, row-major with z fastest:
 *     element (m, n) at m*(nz+1) + n, node m at r = m*R/nr, n at z = n*L/nz.
 *   - A handle may hold several independent discharges ("instances") that
 *     advance together; per-instance calls take the instance index.
 *   - A handle is used by one host thread at a time.
 */
#ifndef PIC_GB300_H
#define PIC_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PIC_ABI_VERSION 1

enum pic_status {
  PIC_OK = 0,
  PIC_ERR_INVALID = -1,      /* bad argument or configuration */
  PIC_ERR_OOM = -2,          /* device allocation failed */
  PIC_ERR_CAPACITY = -3,     /* particle or birth capacity exceeded, or (FP64 particles) a
                                cell holding 2^18 or more macroparticles of one species, where
                                a node's 44-bit fixed-point charge sum could wrap */
  PIC_ERR_NONCONVERGED = -4, /* Poisson solve reached poisson_max_iter */
  PIC_ERR_NAN = -5,          /* non-finite particle coordinate */
  PIC_ERR_TIMEOUT = -6,      /* a device-side wait reached its iteration limit */
  PIC_ERR_CUDA = -7,         /* CUDA runtime error */
  PIC_ERR_IO = -8           /* checkpoint file error */
};

enum pic_species { PIC_ELECTRON = 0, PIC_ION = 1 };

/* Run parameters of one discharge.  Plain data; fill every field. */
typedef struct pic_config {
  uint32_t struct_size;      /* must be sizeof(pic_config) */
  int32_t nr, nz;            /* cells in r and z; both >= 2 and even */
  double R, L, Rc;           /* domain radius, length; cathode disk radius at z = 0 (m) */
  double dt;                 /* time step (s) */
  double weight;             /* real particles per macroparticle, both species (Section 5: constant) */
  double m_ion;              /* ion mass (kg) */
  double n_gas, T_gas;       /* background Ar density (m^-3) and temperature (K) (Section 3) */
  int32_t b_mode;            /* 0: magnetron stand-in B = -grad(A0 J0(kr) e^{-kz}); 1: uniform B0 */
  double B_kA0, B_k;         /* k*A0 (T) and k (1/m) */
  double B0r, B0z;           /* uniform field (T) when b_mode = 1 */
  double gamma_i, gamma_e;   /* ion- and electron-induced secondary electron yields (Section 3) */
  int32_t circuit_mode;      /* 0: cathode fixed at Vc_fixed; 1: V_c = -V_s + I R_ext in [-V_s, 0] */
  double Vc_fixed, Vs, Rext; /* V, V, Ohm */
  int32_t n_avg;             /* steps in the running mean of the cathode current */
  int32_t gather;            /* 0: EC-PIC, 1: MC-PIC (Section 2) */
  int32_t rweight;           /* 0: tent in r; 1: tent in r^2 (volume weighting) */
  int32_t precision;         /* 0: FP64 particles; 1: FP32 particles (cell index + FP32 offsets,
                                FP32 push/deposit, FP64 field solve, circuit and reductions) */
  int32_t mcc_on, push_on, field_on, walls_reflect; /* 1,1,1,0 for the physical model */
  uint64_t seed;             /* random-number key: word 0 of the Philox4x64-10 key of the
                                collision, emission and re-weighting draws (key word 1 the
                                species); the two 32-bit halves of the Philox4x32-10 key of
                                the null-collision candidate draw (counter: id and step as
                                32-bit halves, low first) */
  double sigma_el;           /* elastic cross section (m^2) */
  double ion_a, ion_I;       /* ionization: sigma = ion_a ln(E/I)/(E I) (m^2 eV^2, eV) */
  double exc_C, exc_E;       /* excitation: sigma = exc_C ln(E/E_x)/(E E_x) (m^2 eV^2, eV) */
  double E_cap;              /* energy bound of the null-collision frequency (eV) */
  double poisson_tol;        /* relative residual ||b - A phi||_2 / ||b||_2 to reach */
  int32_t poisson_max_iter;  /* PCG iterations before PIC_ERR_NONCONVERGED */
  int64_t cap_e, cap_i;      /* particle capacities per species */
  int64_t birth_cap;         /* births per species per step */
  int32_t diag_every;        /* diagnostics are accumulated on steps that are multiples */
  int32_t sort_every;        /* full cell sort every this many steps (1..64); on the steps
                                between, absorbed particles stay as dead slots and births
                                are appended in place (a full sort also runs whenever the
                                appended births would not fit).  Results do not depend on
                                it (FP64 bit for bit); calls that read or replace particles
                                (pic_count, pic_get_particles, pic_set_particles, pic_save,
                                pic_solve_fields, pic_region_sample) compact first. */
  double n_meta;             /* metastable Ar* density (m^-3), a constant background; 0 = off */
  double meta_a, meta_I;     /* stepwise ionization (1d) from Ar*: sigma = meta_a ln(E/meta_I)/(E meta_I)
                                (m^2 eV^2, eV; Section 3: threshold 4.20 eV) */
  int32_t gap_neumann;       /* 1: the plane z = 0 outside the cathode is the insulating block
                                (Section 3: Neumann boundary, no normal field; its nodes are
                                unknowns of the Poisson solve); 0: grounded conductor */
  int32_t wall_neumann;      /* 1: the wall r = R is insulating as well; 0: grounded */
  double band_r_lo, band_r_hi; /* radial band of the region diagnostics (m); the paper's
                                discharge region is 1.0 cm < r < 1.5 cm (Sections 5, 7) */
  int32_t ied_bins;          /* cathode ion energy histogram: bins (0: off, at most 65536) */
  double ied_emax;           /* its upper edge (eV); bins of width ied_emax / ied_bins */
  int32_t phi_extrapolate;   /* 1: each step's Poisson solve starts, on the unknown nodes,
                                from the linear extrapolation 2 phi^{n-1} - phi^{n-2} of the
                                last two solutions instead of phi^{n-1} (fewer iterations;
                                phi is still solved to poisson_tol); 0: from phi^{n-1} */
  int32_t poisson_precond;   /* preconditioner of the flexible PCG Poisson solve:
                                0: a sine transform along z with one tridiagonal solve in r
                                per mode (FP32), exact for the operator when every boundary
                                node is a conductor (gap_neumann = wall_neumann = 0), so two
                                or three PCG iterations reach poisson_tol; with insulating
                                boundary parts the multigrid V-cycle instead;
                                1: always the FP32 geometric-multigrid V-cycle */
} pic_config;

/* Device-memory provider.  alloc returns a device pointer aligned to at least
 * 256 bytes or NULL; free releases it.  All device memory of a handle comes
 * from here (when the pointer to this struct is NULL, cudaMalloc/cudaFree). */
typedef struct pic_alloc {
  void* ctx;
  void* (*alloc)(void* ctx, size_t bytes);
  void (*free)(void* ctx, void* ptr);
} pic_alloc;

/* Diagnostics of the last diagnostic step of one instance (Sections 4-6:
 * cathode current and voltage, densities, energies). */
typedef struct pic_diag {
  double t;             /* time of the step whose energies are reported (s) */
  double I_cath;        /* cathode current after the step (A), running mean */
  double V_cath;        /* cathode potential after the step (V) */
  double n_e_peak;      /* max over nodes of the electron density after the step (m^-3) */
  double n_i_peak;      /* same for ions */
  double W_field;       /* field energy 1/2 sum_edges eps0 E^2 V_edge at the step (J) */
  double K_e, K_i;      /* kinetic energies, mean of |v|^2 before and after the push (J) */
  int64_t N_e, N_i;     /* macroparticles after the step */
  int64_t n_ion_cath, n_e_cath, n_sey; /* cathode impacts and secondary electrons this step */
  int64_t n_ionize, n_excite, n_elastic; /* collisions this step */
  int64_t step;         /* index of the step the record belongs to */
  int64_t particle_steps; /* particles pushed, summed over all steps so far (updated every step) */
  int32_t poisson_iters;
  int32_t status;       /* latched device status (pic_status) */
  double poisson_resid; /* final relative residual */
  int64_t n_ionize_meta; /* stepwise ionizations from Ar* (1d) this step */
  int64_t ppc_max_e, ppc_max_i; /* most macroparticles in one cell after the step */
  double weight;        /* current macroparticle weight (changed by pic_reweight) */
} pic_diag;

typedef struct pic_handle pic_handle;

/* Create a handle for n_instances discharges (cfgs[0..n_instances-1]; at most
 * 64, all with the same gather and precision).
 * Allocates all device state, builds the static B table on the host in FP64
 * and uploads it.  Particles start empty (pic_set_particles); phi starts at
 * zero.  cuda_stream: cudaStream_t of all later work.  Returns PIC_OK and
 * *out, or an error with *out = NULL. */
int pic_create(const pic_config* cfgs, int n_instances, const pic_alloc* alloc,
               void* cuda_stream, pic_handle** out);

/* Release all device memory of the handle (after synchronising its stream). */
void pic_destroy(pic_handle* h);

/* Text of the last error on this handle (static storage of the handle). */
const char* pic_last_error(const pic_handle* h);

/* Replace the particles of one species of one instance.  Arrays of length n
 * (r in [0,R), z in [0,L), velocities (v_r, v_theta, v_z) in m/s, ids unique
 * and >= 0); host memory when on_device = 0, device memory otherwise.  Page-
 * locked host arrays (all six) are read in place by the kernels; pageable ones
 * go through staging copies.  The particles are sorted by cell on the device.  next_id becomes max(id)+1 over
 * both species if that is larger.  Synchronous. */
int pic_set_particles(pic_handle* h, int instance, int species, int64_t n, const double* r,
                      const double* z, const double* vr, const double* vt, const double* vz,
                      const int64_t* id, int on_device);

/* Number of macroparticles of a species (synchronous). */
int pic_count(pic_handle* h, int instance, int species, int64_t* n_out);

/* Copy out the particles (any order; compare by id).  Arrays must hold the
 * count returned by pic_count.  Host or device memory per on_device. */
int pic_get_particles(pic_handle* h, int instance, int species, double* r, double* z,
                      double* vr, double* vt, double* vz, int64_t* id, int on_device);

/* Deposit the current particles and solve for phi with the current cathode
 * voltage (used after pic_set_particles to obtain phi at step 0).  Async. */
int pic_solve_fields(pic_handle* h, int instance);

/* Overwrite phi (node array, host or device).  Synchronous. */
int pic_set_phi(pic_handle* h, int instance, const double* phi, int on_device);

/* Copy out phi, rho = Q/V and Q (node arrays; any may be NULL).  Synchronous. */
int pic_get_fields(pic_handle* h, int instance, double* phi, double* rho, double* Q,
                   int on_device);

/* Copy out the node charge (C) that one species deposited in the last step
 * (or by pic_solve_fields): q_s w sum_p S_mn(x_p) over that species' particles
 * (Section 2: tent functions; the same weights as the deposit into Q, whose
 * sum over both species it is).  Node array as above, host or device memory
 * per on_device.  Dividing by the node control volume gives the species'
 * density, e.g. for time averages of the density profile.  Synchronous. */
int pic_get_species_charge(pic_handle* h, int instance, int species, double* Q, int on_device);

/* Set the circuit state: cathode voltage, step index and the last n_avg
 * cathode charges (C; ring buffer indexed by step % n_avg).  Synchronous. */
int pic_set_circuit(pic_handle* h, int instance, double Vc, int64_t step, const double* qhist,
                    int n);

/* Set / get the next particle id handed to a birth.  Synchronous. */
int pic_set_next_id(pic_handle* h, int instance, int64_t next_id);
int pic_get_next_id(pic_handle* h, int instance, int64_t* next_id);

/* Advance all instances by nsteps time steps.  Async (see conventions), except
 * for the first four steps of a handle, which tune the push (see
 * pic_tuned_chunk) and wait for their own completion.  After them, on a stream
 * other than the legacy default stream, one step of all instances is captured
 * into a CUDA graph and replayed (eager launches while pic_profile is on, or
 * if capture is unavailable). */
int pic_step(pic_handle* h, int64_t nsteps);

/* 1 when pic_step replays a captured CUDA graph on this handle, else 0. */
int pic_uses_graph(pic_handle* h);

/* The push of both species of every instance is one persistent kernel over a
 * device queue of (instance, species, chunk) work items, electron and ion
 * chunks interleaved; ensembles (n_instances > 1) also solve all Poisson
 * problems in one grouped launch.  The first four steps of a handle each try
 * one chunk size (4, 8, 16, 32 particles per thread) with eager launches and
 * the fastest is kept (then two more steps try the other tile shapes, see
 * pic_set_tile): *particles_per_thread receives it, or 0 while tuning is
 * unfinished. */
int pic_tuned_chunk(pic_handle* h, int* particles_per_thread);

/* Fix the push's chunk size (particles_per_thread 4, 8, 16 or 32) for the
 * rest of the run, ending any tuning under way (the tile shape then stays);
 * 0 restarts the tuning, so the next steps time the four sizes (and the tile
 * shapes) again (e.g. after the particle counts have grown).  Results do not depend on the chunk size (FP64 bit for bit).
 * Drops the captured step graph.  PIC_ERR_INVALID for any other value. */
int pic_set_chunk(pic_handle* h, int particles_per_thread);

/* Cell tile shape of the particle sort key and of the push's shared deposit
 * patch, for every instance of the handle: 1 = 8 x 8, 2 = 16 x 8, 3 = 8 x 16
 * cells (r x z) fixed from now on, the particles re-sorted by the new keys at
 * once (results do not depend on the shape: FP64 exactly, FP32 up to the
 * order of the FP32 patch sums); 0 = chosen by the autotuner, which (after the
 * chunk size) times one step on each shape and keeps the fastest, here and at
 * every re-tuning (this restarts the tuning).  Default 0, starting on 8 x 8.
 * Synchronous.  PIC_ERR_INVALID for another shape. */
int pic_set_tile(pic_handle* h, int shape);

/* The current tile shape (1, 2 or 3 as in pic_set_tile). */
int pic_tuned_tile(pic_handle* h, int* shape);

/* The push's online tuning.  The first four steps of a handle time the four
 * chunk sizes and the next two the other two tile shapes (pic_set_tile);
 * later, when at the start of a pic_step call the live particle count of all
 * instances (as copied after the previous call) differs from the count at the
 * last tuning by a factor of 4 or more, the next steps tune again and the step
 * graph is captured anew (unless the size was fixed with pic_set_chunk).  *tunings: tunings completed; *particles_per_thread: the
 * size in use (0 while tuning); *particles_at_tuning: live particles when the
 * last tuning ended.  Any pointer may be NULL. */
int pic_autotune_info(pic_handle* h, int* tunings, int* particles_per_thread,
                      int64_t* particles_at_tuning);

/* Wait for the handle's stream; return the latched status of all instances. */
int pic_sync(pic_handle* h);

/* Synchronise and copy the diagnostics record of one instance into *out
 * (caller-owned).  Returns the latched status of that instance. */
int pic_diagnostics(pic_handle* h, int instance, pic_diag* out);

/* Particle re-weighting of one instance between steps (Section 6: at high
 * density, two thirds of the particles removed and the weight of the rest
 * tripled).  Each particle of both species is kept with probability
 * 1/factor: particle `id` of species s stays iff word 0 of Philox4x64-10 with
 * counter (id, step, 5, 0) and key (seed, s) is divisible by factor, `step`
 * being the index of the next step.  The kept particles are unchanged; the
 * macroparticle weight (charge, current, energies and densities from the
 * next step on) is multiplied by factor; phi stays until the next solve.
 * Synchronous; drops the captured step graph.  factor 1 is a no-op;
 * factor < 1 returns PIC_ERR_INVALID. */
int pic_reweight(pic_handle* h, int instance, int factor);

/* Region diagnostics (Sections 4, 5 and 7).
 *   pic_region_sample  adds the current state to per-cell accumulators:
 *                      particle counts of both species, electron velocity
 *                      sums (v_r, v_theta, v_z, |v|^2), node potentials.
 *                      Async (a few kernels on the handle's stream).
 *   pic_region_read    evaluates the accumulated samples (synchronous).  Per
 *                      cell column m (r_m .. r_{m+1}), walking up from the
 *                      cathode, the sheath ends at the first cell whose
 *                      accumulated counts give n_e >= n_i / 2, the bulk
 *                      starts at the first cell from there on whose axial
 *                      field from the accumulated corner potentials is
 *                      E_z >= 0; zs[m], zb[m] (m, nr values each, may be
 *                      NULL) are those edges.  A cell's electron temperature
 *                      is m_e (<|v|^2> - |<v>|^2) / (3 e) over its samples
 *                      (cells with >= 2); Te[k] is the plain mean over the
 *                      cells of region k (sheath, pre-sheath, bulk) whose
 *                      column centre lies in [band_r_lo, band_r_hi].
 *                      z_sheath, z_bulk: the edges averaged over those
 *                      columns.  ied (ied_bins values, may be NULL) and
 *                      *ied_overflow (may be NULL): ions that hit the cathode
 *                      at band_r_lo <= r <= band_r_hi since the last reset,
 *                      binned by 1/2 M |v|^2 of the arriving ion, the
 *                      overflow counting energies at or above ied_emax; the
 *                      histogram is filled by every step's push.
 *   pic_region_reset   clears the accumulators and the histogram (async). */
typedef struct pic_regions {
  int64_t samples;         /* states accumulated */
  double Te[3];            /* sheath, pre-sheath, bulk electron temperature (eV) */
  int64_t ncell[3];        /* cells averaged in each region */
  double z_sheath, z_bulk; /* mean region edges over the band's columns (m) */
  int64_t ion_impacts;     /* ions in the histogram, overflow included */
} pic_regions;
int pic_region_sample(pic_handle* h, int instance);
int pic_region_read(pic_handle* h, int instance, pic_regions* out, double* zs, double* zb,
                    int64_t* ied, int64_t* ied_overflow);
int pic_region_reset(pic_handle* h, int instance);

/* Checkpoint of one instance to / from a file (particles as stored on the
 * device, FP64 positions in cell units; phi and the solution before it, the
 * start of an extrapolated solve; circuit state, step and id counters,
 * weight).  A resumed run continues bit for bit up to the order of particles
 * inside a cell.  The file is for a handle of the same grid, n_avg and
 * precision (PIC_ERR_IO otherwise).  Synchronous. */
int pic_save(pic_handle* h, int instance, const char* path);
int pic_load(pic_handle* h, int instance, const char* path);

/* Per-kernel timing of pic_step (CUDA events on the handle's stream around
 * each kernel group).  pic_profile(h, 1) clears the counters and starts
 * recording, pic_profile(h, 0) stops.  pic_profile_read synchronises and
 * fills up to `max` records (names are static strings: "field_tables",
 * "push", "births", "scan", "scatter", "charge", "circuit", "poisson",
 * "step_end", "warm_start"); *n_out is the number of kernel groups. */
typedef struct pic_kernel_time {
  const char* name;
  int64_t launches;
  double total_ms;
} pic_kernel_time;
int pic_profile(pic_handle* h, int enable);
int pic_profile_read(pic_handle* h, pic_kernel_time* out, int max, int* n_out);

/* ---------------------------------------------------------------------------
 * Learned warm start of the Poisson solve (single-instance handles).
 *
 * A small U-Net, trained on the GPU on snapshots the simulation records,
 * proposes where each Poisson solve starts.  Network: 4 levels of
 * ((nr >> l) + 1) x ((nz >> l) + 1) nodes, channels 16, 32, 64, 64; two 3x3
 * convolutions (zero padding, ReLU) per level and stage; even nodes down,
 * bilinear node interpolation up, [up, skip] concatenation; 1x1 head.
 * 302,849 parameters, FP32 master copy, BF16 tensor-core arithmetic with FP32
 * accumulation.  Parameter vector order: for each layer enc0a, enc0b, enc1a,
 * enc1b, enc2a, enc2b, enc3a, enc3b, dec2a, dec2b, dec1a, dec1b, dec0a, dec0b,
 * head: weights (cout, cin, kh, kw) row-major, then biases.
 *
 * Two readings of what the network maps (chosen at pic_unet_create):
 *   mode 0 (potential):  x0 = rho / in_norm (rho = Q / V), x1 = r / R,
 *                        x2 = Dirichlet value / V_ref on z = 0, z = L, r = R
 *                        (0 elsewhere)  ->  phi / V_ref;
 *                        V_ref = |V_s| (circuit_mode 1) or |Vc_fixed|.
 *   mode 1 (correction): x0 = res / s with res = Q - A phi_prev (this
 *                        step's charge and electrode values against the
 *                        previous solution) and s the RMS of res over the
 *                        nodes of that step, x1 = r / R, x2 = 1 on Dirichlet
 *                        nodes  ->  (phi - phi_prev) / (s K), K = out_norm /
 *                        in_norm (the change of phi is linear in res, so each
 *                        snapshot is scaled to unit size).
 * in_norm (and out_norm in mode 1) are the RMS of the recorded fields, fixed
 * by the first pic_unet_train call.
 *
 * With the warm start on, the network's candidate (mode 0: V_ref y; mode 1:
 * phi_prev + s K y, on the free nodes) is smoothed by two red-black
 * Gauss-Seidel sweeps of the FP64 operator, and the solve starts from
 * whichever of {phi_prev, candidate, zero} has the smallest residual
 * ||Q - A x||_2.  The solve still runs to poisson_tol: only the iteration
 * count (and time) changes, never the tolerance phi is solved to.
 * ------------------------------------------------------------------------- */

/* Number of network parameters (302849). */
int pic_unet_param_count(int64_t* n);

/* Attach a network to a handle (nr, nz divisible by 8).  On an ensemble the
 * instances must share nr, nz and the boundary kinds (insulating z = 0 nodes
 * and wall); the one network then serves all of them: each step's inputs of
 * all instances form one forward batch, each instance's solve picks its own
 * start, and every instance records into the one snapshot ring (instance k
 * of a recording step into slot count + k, the step counter of instance 0
 * deciding which steps record).  V_ref is instance 0's.  He-normal weights
 * from `seed`, zero biases; max_batch = largest batch of pic_unet_loss_grad /
 * pic_unet_train; mode 0 or 1 (see above).  Allocates through the handle's
 * allocator.  Synchronous.  PIC_ERR_INVALID for instances of different grids
 * or boundary kinds, other grid sizes, another mode or a second call. */
int pic_unet_create(pic_handle* h, uint64_t seed, int max_batch, int mode);

/* Set / get the FP32 parameter vector (host, n = pic_unet_param_count). */
int pic_unet_set_params(pic_handle* h, const float* params, int64_t n);
int pic_unet_get_params(pic_handle* h, float* params, int64_t n);

/* Forward pass on `batch` inputs and, when y != NULL, the mean squared error
 * against y and its gradient with respect to every parameter.  Host arrays:
 *   x    (batch, 3, nr+1, nz+1) network inputs (already normalised)
 *   y    (batch, nr+1, nz+1) targets, or NULL (forward only)
 *   out  (batch, nr+1, nz+1) network output, or NULL
 *   grad parameter-vector gradient, or NULL; loss: mean squared error, or NULL.
 * Parameters are not changed.  Synchronous. */
int pic_unet_loss_grad(pic_handle* h, int batch, const float* x, const float* y, float* out,
                       float* grad, double* loss);

/* Record the training pairs of every `every`-th step into a device ring of
 * `capacity` snapshots of two FP32 node fields (8 (nr+1)(nz+1) bytes per
 * snapshot): mode 0 (rho, phi) after the solve; mode 1 (res, phi - phi_prev)
 * around it.  Recording continues in later pic_step calls.  Synchronous. */
int pic_unet_snapshots(pic_handle* h, int64_t capacity, int every);

/* Pause (on = 0) or resume (on = 1) the recording into the ring set by
 * pic_unet_snapshots; the ring and its snapshots are kept (training still
 * draws from them).  PIC_ERR_INVALID without a ring. */
int pic_unet_record(pic_handle* h, int on);

/* `iters` Adam steps (beta 0.9, 0.999) of learning rate lr on batches of
 * `batch` snapshots drawn from the ring by a hash of (seed, iteration,
 * index); targets as the mode defines.  *loss_first and *loss_last (may be NULL)
 * receive the training loss of the first and the last batch.  Synchronous. */
int pic_unet_train(pic_handle* h, int iters, int batch, float lr, uint64_t seed,
                   double* loss_first, double* loss_last);

/* Set the network's input and output scales (in_norm, out_norm as in the
 * stats below; both > 0), which the first pic_unet_train call otherwise fixes
 * from the recorded snapshots: with pic_unet_set_params this moves a trained
 * network to another handle.  Synchronous.  PIC_ERR_INVALID for a scale that
 * is not positive and finite. */
int pic_unet_set_norms(pic_handle* h, double in_norm, double out_norm);

/* Turn the warm start of later pic_step solves on (1) or off (0). */
int pic_unet_warm_start(pic_handle* h, int on);

/* Counters since pic_unet_create, summed over the instances of the handle
 * (synchronous); last_start is that of the last instance solved. */
typedef struct pic_unet_stats {
  int64_t snapshots;           /* snapshots recorded */
  int64_t starts_previous;     /* solves started from the previous phi */
  int64_t starts_network;      /* solves started from the network's guess */
  int64_t starts_zero;         /* solves started from zero */
  int64_t poisson_iters;       /* PCG iterations summed over steps */
  double in_norm;              /* input scale of channel 0 (0 until trained) */
  double out_norm;             /* output scale (mode 0: V_ref; mode 1: 0 until trained) */
  int32_t last_start;          /* 0 previous, 1 network, 2 zero */
  int32_t pad;
} pic_unet_stats;
int pic_unet_stats_read(pic_handle* h, pic_unet_stats* out);

/* Bytes of device scratch that pic_poisson_solve needs for an nr x nz grid. */
size_t pic_poisson_workspace_bytes(int nr, int nz);

/* pic_poisson_solve with insulating (Neumann) boundary parts: the nodes of
 * row z = 0 from radial index first_insulating_z0 on (nr + 1: none) and,
 * when wall_insulating is 1, the wall r = R (n = 1 .. nz - 1, and the corner
 * r = R, z = 0 when row 0 is insulating there too) are unknowns with zero
 * normal flux; every other boundary node holds its Dirichlet value from
 * phi_dev.  Other arguments, ownership and errors as pic_poisson_solve;
 * PIC_ERR_INVALID also for first_insulating_z0 outside [0, nr + 1] or
 * wall_insulating not 0/1. */
int pic_poisson_solve_mixed(int nr, int nz, double R, double L, int first_insulating_z0,
                            int wall_insulating, double tol, int max_iter, const double* Q_dev,
                            double* phi_dev, void* work_dev, void* cuda_stream, int* iters,
                            double* resid);

/* Standalone RZ Poisson solve (Section 3: Dirichlet electrodes, Gauss's law
 * on the axis) on the stream `cuda_stream`.
 *   Q_dev    node charges (C), device, (nr+1)(nz+1) doubles (input)
 *   phi_dev  device node array: on input the boundary nodes (z = 0, z = L,
 *            r = R) hold the Dirichlet values and the others the initial
 *            guess; on output the solution.
 *   work_dev device scratch of pic_poisson_workspace_bytes(nr, nz) bytes,
 *            256-byte aligned, owned by the caller; contents not preserved.
 *   iters, resid (host, may be NULL): PCG iterations and final relative
 *            residual.
 * Synchronous.  Returns PIC_ERR_NONCONVERGED when tol is not met in max_iter
 * iterations (phi then holds the last iterate). */
int pic_poisson_solve(int nr, int nz, double R, double L, double tol, int max_iter,
                      const double* Q_dev, double* phi_dev, void* work_dev, void* cuda_stream,
                      int* iters, double* resid);

/* Measured FP64 FMA throughput of the current device (TFLOP/s, an FMA = 2
 * flop): independent FMA chains on every SM, the fastest of three timed
 * launches on `cuda_stream` (NULL: the default stream).  The denominator of
 * the roofline of an FP64-pipe-bound kernel.  Allocates and frees a small
 * output buffer on the stream; synchronous. */
int pic_fp64_fma_rate(void* cuda_stream, double* tflops);

/* Size in bytes of the device array that pic_poisson_solve_static uses as
 * its scratch; it holds the workspace of grids up to 256 x 512 cells. */
#define PIC_POISSON_STATIC_BYTES (6u * 1024u * 1024u)

/* pic_poisson_solve for callers that cannot allocate device memory while
 * they run -- e.g. an application whose memory pool already owns the GPU, or a
 * loop that cannot afford the device-wide synchronisation of cudaMalloc.
 * The paper has no counterpart: this is an allocation policy of this library.
 * Same arguments and results as pic_poisson_solve, minus work_dev: the
 * scratch is a file-scope device array of PIC_POISSON_STATIC_BYTES that every
 * GPU which loads the library holds until the process exits.  Nothing is
 * allocated: no cudaMalloc/cudaFree, no allocator of any framework.
 *   - Grids whose pic_poisson_workspace_bytes(nr, nz) exceeds
 *     PIC_POISSON_STATIC_BYTES - 256 are rejected with PIC_ERR_CAPACITY.
 *   - Each call looks up the array's device address on the current device
 *     (cudaGetSymbolAddress), so a device reset between calls is harmless;
 *     the first call on a device also loads the library's device code there.
 *   - All calls on a device share the one array, which keeps the previous
 *     call's contents (each call clears what must start at zero).  Calls that
 *     overlap on the GPU race on it: serialise them (one stream, one thread).
 * Synchronous. */
int pic_poisson_solve_static(int nr, int nz, double R, double L, double tol, int max_iter,
                             const double* Q_dev, double* phi_dev, void* cuda_stream, int* iters,
                             double* resid);

#ifdef __cplusplus
}
#endif
#endif /* PIC_GB300_H */
