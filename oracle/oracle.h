/*
 * oracle.h -- plain FP64 CPU reference ("oracle") of the RZ electrostatic
 * PIC-MCC step of the dc magnetron model (arXiv:2507.10727).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA library
 * against an independent, slow, obviously correct implementation.  Only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg may load
 * it.  It shares no code, header, table or constant with the CUDA library.
 *
 * Everything is double precision, single threaded, in the order the method
 * states: gather -> Boris push -> walls / secondary emission -> MCC -> births
 * -> deposit -> circuit -> Poisson.  Citations name the paper's sections,
 * equations and Table 1; where the paper is silent the comment says which
 * reading is taken (the readings are listed with the design notes).
 *
 * Parity status per function (what pins it, in tests/test_oracle_*.py):
 *   orc_philox4x64         known-answer test against numpy's Philox
 *   orc_philox4x32         the published Philox4x32-10 known-answer vectors
 *   orc_boris_move         Larmor polygon radius, rotation angle, E x B drift,
 *                          |v| conservation (closed forms)
 *   orc_bfield             div B = 0, curl B = 0 (finite differences), B_r zero
 *                          near the J1 root at the cathode edge
 *   orc_deposit            total charge, single-particle split, r^2 moment
 *   orc_poisson            exact quadratic solution, 2nd-order convergence,
 *                          Gauss law; insulating boundaries: exact quadratic
 *                          solutions with zero normal derivative, mirror image
 *                          of the all-insulating z = 0 plane
 *   orc_efield_at          MC zero axial self-force, EC force = -dW/dx
 *   MCC inside orc_step    collision counts vs nu_k dt, exact energy losses
 *   circuit inside orc_step  prescribed-charge drive; Table 1 cases 1-2
 *   region diagnostics     hand-built states with known sheath and bulk edges
 *                          and temperatures; IED of mono-energetic beams
 *   orc_reweight           kept fraction within binomial bounds, kept records
 *                          unchanged, independent of particle order, charge
 *                          and density profile conserved in expectation
 */
#ifndef PIC_ORACLE_H
#define PIC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_config {
  int32_t nr, nz;          /* cells in r and z */
  double R, L, Rc;         /* domain radius, length, cathode radius (m) */
  double dt;               /* time step (s) */
  double weight;           /* real particles per macroparticle */
  double m_ion;            /* ion mass (kg) */
  double n_gas, T_gas;     /* background argon density (m^-3), temperature (K) */
  int32_t b_mode;          /* 0: magnetron node table, 1: uniform (B0r, B0z) */
  double B_kA0, B_k;       /* k*A0 (T), k (1/m) */
  double B0r, B0z;         /* uniform field (T), b_mode 1 */
  double gamma_i, gamma_e; /* ion- and electron-induced secondary yields */
  int32_t circuit_mode;    /* 0: cathode fixed at Vc_fixed, 1: external circuit */
  double Vc_fixed, Vs, Rext;
  int32_t n_avg;           /* steps in the cathode-current average */
  int32_t gather;          /* 0: EC-PIC, 1: MC-PIC */
  int32_t rweight;         /* 0: linear tent in r, 1: volume (r^2) weighting */
  int32_t mcc_on, push_on, field_on, walls_reflect;
  uint64_t seed;
  double sigma_el, ion_a, ion_I, exc_C, exc_E, E_cap;
  double n_meta;           /* metastable Ar* density (m^-3), constant background */
  double meta_a, meta_I;   /* reaction (1d): sigma = meta_a ln(E/meta_I)/(E meta_I) */
  int32_t gap_neumann;     /* 1: z = 0 outside the cathode is the insulating block */
  int32_t wall_neumann;    /* 1: the wall r = R is insulating too */
  double band_r_lo, band_r_hi; /* radial band of the region diagnostics (m) */
  int32_t ied_bins;        /* cathode ion energy histogram bins (0: off) */
  double ied_emax;         /* its upper edge (eV); bins of width ied_emax / ied_bins */
} orc_config;

typedef struct orc_diag {
  double t, I_cath, V_cath, n_e_peak, n_i_peak, W_field, K_e, K_i;
  int64_t N_e, N_i;
  int64_t n_ion_cath, n_e_cath, n_sey, n_ionize, n_excite, n_elastic;
  int64_t n_ionize_meta;   /* reaction (1d) events */
  int64_t ppc_max_e, ppc_max_i;  /* most macroparticles in one cell after the step */
} orc_diag;

/* Region diagnostics (Sections 4 and 5): the sheath (n_e < n_i / 2), the
 * pre-sheath and the bulk (from the first E_z >= 0 on) along z in each cell
 * column, electron temperatures by region in the radial band. */
typedef struct orc_regions {
  int64_t samples;         /* states accumulated */
  double Te[3];            /* sheath, pre-sheath, bulk: mean cell temperature (eV) */
  int64_t ncell[3];        /* band cells with >= 2 electron samples in each region */
  double z_sheath, z_bulk; /* region edges averaged over the band's columns (m) */
  int64_t ion_impacts;     /* ion cathode impacts in the band (IED incl. overflow) */
} orc_regions;

typedef struct orc_sim orc_sim;

/* ---- pure pieces (used by the pins) ---- */
void orc_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);
void orc_philox4x32(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void orc_boris_move(double q_over_m, double dt, double Er, double Ez, double Br, double Bz,
                    double* r, double* z, double* vr, double* vt, double* vz);
void orc_bfield(const orc_config* c, double r, double z, double* Br, double* Bz);
double orc_node_volume(const orc_config* c, int m, int n);
void orc_deposit(const orc_config* c, int64_t np, const double* r, const double* z,
                 double qw, double* Q /* (nr+1)*(nz+1), accumulated into */);
int orc_poisson(const orc_config* c, const double* rho, const double* phi_bc, double* phi);
void orc_efield_at(const orc_config* c, const double* phi, double r, double z,
                   double* Er, double* Ez);
void orc_sigma(const orc_config* c, double E_eV, double out[3]);
double orc_sigma_meta(const orc_config* c, double E_eV);
double orc_nu_max(const orc_config* c);
double orc_field_energy(const orc_config* c, const double* phi);

/* ---- the time stepper ---- */
orc_sim* orc_create(const orc_config* c);
int orc_set_particles(orc_sim* s, int species, int64_t n, const double* r, const double* z,
                      const double* vr, const double* vt, const double* vz, const int64_t* id);
int64_t orc_count(const orc_sim* s, int species);
int orc_get_particles(const orc_sim* s, int species, double* r, double* z, double* vr,
                      double* vt, double* vz, int64_t* id);
int orc_solve_fields(orc_sim* s);              /* phi from current particles and V_c */
void orc_set_phi(orc_sim* s, const double* phi);
void orc_get_fields(const orc_sim* s, double* phi, double* rho, double* Q);
/* node charge (C) deposited by one species in the last step (Q = sum of both) */
void orc_get_species_charge(const orc_sim* s, int species, double* Q);
void orc_set_circuit(orc_sim* s, double Vc, int64_t step, const double* qhist, int n);
int orc_step(orc_sim* s, int64_t nsteps);
void orc_get_diag(const orc_sim* s, orc_diag* d);
void orc_set_next_id(orc_sim* s, int64_t next_id);
int64_t orc_get_next_id(const orc_sim* s);
int64_t orc_get_step(const orc_sim* s);
/* Particle re-weighting (Section 6): keep each particle with probability
 * 1/factor and multiply the macroparticle weight by factor.  Returns the
 * particles kept (both species), or -1 for factor < 1. */
int64_t orc_reweight(orc_sim* s, int factor);
double orc_get_weight(const orc_sim* s);
/* Region diagnostics: accumulate the current state (per cell particle counts
 * and electron velocity moments, node potential); evaluate the regions (the
 * per-column edges zs, zb may be NULL, else nr values); read the cathode ion
 * energy histogram (ied_bins values and the overflow count); clear both. */
void orc_region_sample(orc_sim* s);
int orc_region_result(const orc_sim* s, orc_regions* out, double* zs, double* zb);
void orc_ied_get(const orc_sim* s, int64_t* hist, int64_t* overflow);
void orc_region_reset(orc_sim* s);
void orc_destroy(orc_sim* s);

#ifdef __cplusplus
}
#endif
#endif
