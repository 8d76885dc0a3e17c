/*
 * emt_oracle.h -- plain FP64 CPU oracle for the electromagnetic shower
 * transport loop of arXiv:2203.09467 (Celeritas roadmap).
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the GPU library; it is
 * called from the test suite, from the smoke check and from the CPU-baseline
 * leg of the benchmark, and compiled by oracle/census.cpp (a count of the
 * step's FP64 operations), and from nothing else.  It shares no code with
 * the CUDA path.
 *
 * The paper names the physics models (Sec. 2.2, Table 1) and capabilities
 * (material properties, continuous slowing down, competing discrete
 * processes, secondaries, energy cutoffs) but prints no formula.  Every
 * formula below is a textbook closed form, cited at its definition in
 * emt_oracle.c; the step order is the reading documented there.
 *
 * Units: MeV, cm, g/cm^3, tesla.
 */
#ifndef EMT_ORACLE_H
#define EMT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* process bits (same meaning as the library's, defined independently) */
#define ORC_PHOTO 1u
#define ORC_COMPTON 2u
#define ORC_PAIR 4u
#define ORC_IONI 8u
#define ORC_BREMS 16u
#define ORC_ANNIH 32u
#define ORC_MSC 64u     /* multiple scattering of e+- (Highland width) */
#define ORC_ANGULAR 128u /* angular distributions: dipole for brems and pair, Sauter for the photoelectron */
#define ORC_RAYLEIGH 256u /* Rayleigh scattering (screened-atom form factor) */

typedef struct orc_handle orc_handle;

/* ---- Philox4x32-10 (Salmon et al., SC'11) ---- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* draw j of step `step` of track `uid` in event `event_id` */
double orc_track_uniform(uint32_t seed, uint64_t event_id, uint64_t uid, uint32_t step, uint32_t j);
uint64_t orc_child_uid(uint32_t seed, uint64_t event_id, uint64_t uid, uint32_t step, uint32_t k);

/* ---- closed forms ---- */
double orc_x0_gcm2(double Z, double A);
double orc_sigma_kn(double k);                  /* per electron, cm^2 */
double orc_dsigma_kn_deps(double k, double eps); /* per electron, cm^2 per unit eps=k'/k */
double orc_sigma_pair_atom(double Z, double A, double k);  /* cm^2 per atom */
double orc_dsigma_pair_dx(double Z, double A, double k, double x);
double orc_sigma_photo_atom(double Z, double k, double bk);
double orc_sigma_moller(double T, double cut);   /* per electron, cm^2 */
double orc_dsigma_moller_deps(double T, double eps);
double orc_sigma_bhabha(double T, double cut);
double orc_dsigma_bhabha_deps(double T, double eps);
double orc_sigma_heitler(double T);              /* per electron, cm^2 */
double orc_sigma_rayleigh_atom(double Z, double k); /* cm^2 per atom */
double orc_dsigma_rayleigh_dx(double Z, double k, double x); /* per unit x = 1 - cos */
double orc_dsigma_heitler_deps(double T, double eps);
double orc_sigma_brems_macro(double x0_cm, double T, double kc); /* 1/cm */
double orc_dsigma_brems_macro_dk(double x0_cm, double T, double k);
double orc_dedx_rad(double x0_cm, double T, double kc);          /* MeV/cm */
/* restricted collision stopping power; charge -1 (e-) or +1 (e+); cut MeV */
double orc_dedx_coll(double Z, double A, double rho, double I_eV, int charge,
                     double T, double cut);

/* ---- Gauss-Legendre 16 ---- */
void orc_gauss_legendre(int n, double* x, double* w);

/* ---- samplers (single interaction, from a track's draw stream) ---- */
/* out layout per sampler documented in emt_oracle.c; process 7, 8 and 10
 * are bremsstrahlung, pair production and the photoelectric effect with the
 * angular option; 9 is Rayleigh scattering (cut_e carries Z) */
int orc_sample(int process, double E, double cut_e, double cut_g, uint32_t seed,
               uint64_t event_id, uint64_t uid, uint32_t step, double* out);
/* multiple scattering: Highland width, and the deflection of dir (in
 * place) after a step of length s at pre-step kinetic energy T */
double orc_highland(double T, double s, double x0_cm);
int orc_msc(double T, double s, double x0_cm, uint32_t seed, uint64_t event_id,
            uint64_t uid, uint32_t step, double* dir);

/* ---- set-up ---- */
/* materials: n x {Z, A, rho, I_eV, bk_MeV}; rho == 0 -> vacuum
 * physics  : {cut_g, cut_em, cut_ep, e_lo, e_hi, bins_per_decade, step_frac,
 *             final_range, process_mask}
 * layers   : n_layers x {material, thickness_cm, score_bin}
 * world    : {z0, half_x, half_y, wlo[3], whi[3], B[3], rk_delta_cm,
 *             max_steps, n_bins, max_field_step_cm, geometry, half_z_cm,
 *             score_z, score_z_lo_cm, score_z_hi_cm}
 *   geometry 0: layers are slabs stacked along +z from z0 inside
 *               |x| <= half_x, |y| <= half_y, in the world box wlo..whi;
 *   geometry 1: layers are concentric cylindrical shells about the z axis,
 *               radii accumulated from z0 (must be 0), |z| <= half_z; the
 *               outermost shell and the end planes bound the world.
 *   score_z 0 : histogram bin = the score bin of the deposit's volume;
 *   score_z 1 : n_bins equal bins of z over [score_z_lo, score_z_hi).
 * Returns NULL for an invalid configuration.                                */
orc_handle* orc_create(const double* materials, int n_mat, const double* physics,
                       const double* layers, int n_layers, const double* world,
                       uint32_t seed);
void orc_destroy(orc_handle*);
int orc_grid_size(const orc_handle*);
/* table of material m, particle p (0 gamma, 1 e-, 2 e+), quantity q:
 *  gamma: 0 photo, 1 compton, 2 pair
 *  e-   : 0 ioni, 1 brems, 2 (zero), 3 range, 4 dedx
 *  e+   : 0 ioni, 1 brems, 2 annih, 3 range, 4 dedx
 * q == 5 returns the energy grid.  Writes grid_size values. */
int orc_get_table(const orc_handle*, int m, int p, int q, double* out);
double orc_range(const orc_handle*, int m, int charge_index, double T);
double orc_inv_range(const orc_handle*, int m, int charge_index, double r);

/* ---- transport ----
 * primaries (SoA): ev[n] (index of the event in [0,n_events)), type[n],
 * T[n], pos[3n], dir[3n]; event_ids[n_events].
 * outputs: hist[n_events*n_bins]; summary[n_events*6] =
 *   {edep, escaped, killed, e_in, n_steps, n_tracks}
 * n_threads <= 0 : all available cores.
 * step_hist (optional, NULL = off): adds the number of steps of every
 * transported track, by particle type, into step_hist[3][step_bins]
 * (counts of step_bins - 1 or more steps in the last bin).                  */
int orc_run(orc_handle*, int n_prim, const int32_t* ev, const int32_t* type,
            const double* T, const double* pos, const double* dir,
            int n_events, const uint64_t* event_ids, double* hist,
            double* summary, int n_threads, uint64_t* step_hist, int step_bins);

/* geometry pins: exit parameter along d from p in volume vol (returns the
 * next volume, writes t), and the volume of a starting point */
int orc_nav_exit(const orc_handle*, int vol, const double* p, const double* d, double* t);
int orc_locate(const orc_handle*, const double* p);

/* one step of one track (diagnostics and single-step pins).
 * track in/out: {type, T, x, y, z, ux, uy, uz, vol, step}, uid, event_id.
 * returns number of secondaries written to sec (each 8 doubles:
 * {type, T, x, y, z, ux, uy, uz}) and sec_uid; info[8] = {s, edep,
 * boundary, interacted, process, alive, escaped, killed}.                  */
int orc_step_one(orc_handle*, double* track, uint64_t uid, uint64_t event_id,
                 double* sec, uint64_t* sec_uid, double* info);

#ifdef __cplusplus
}
#endif
#endif
