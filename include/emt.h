/*
 * emt.h -- C ABI of the GB300 electromagnetic shower transport library.
 *
 * The library runs the per-step Monte Carlo transport loop for photons,
 * electrons and positrons described in arXiv:2203.09467 (Celeritas):
 * cross sections from tabulated log-spaced grids (Sec. 2.2: the
 * discrete cross sections of every particle type come from tables and are
 * evaluated together in one kernel), continuous slowing down and energy
 * cutoffs (Sec. 2.2 list of capabilities), the six electromagnetic models
 * of Table 1 (Klein-Nishina, Bethe-Heitler, photoelectric, bremsstrahlung,
 * Moller-Bhabha, two-photon annihilation), straight-line and uniform-field
 * propagation through layered-box or concentric-cylinder geometry (Sec. 2.3;
 * the cylinders are Sec. 3.2's CMS-like test problem), secondary
 * allocation with a capacity-bounded device stack (Sec. 2.1:
 * secondaries are reserved from a stack by an atomic add, and running out
 * of room must not break reproducibility), and scoring in device kernels instead of host
 * callbacks (Sec. 2.4).  The call sequence follows the paper's statement of
 * the problem: load materials and physics tables, load geometry, submit
 * primaries for many concurrent events, step until done, read the scores.
 *
 * Conventions
 *  - Units: MeV, cm, g/cm^3, tesla.
 *  - Every call returns an emt_status; no exception or abort crosses the
 *    ABI.  emt_last_error() gives a message for the last failed call on the
 *    context (valid until the next call).
 *  - Pointers marked "host" are read (or written) during the call only; the
 *    caller keeps ownership.  Pointers marked "where" follow the `where`
 *    argument: EMT_HOST (pageable or pinned host memory) or EMT_DEVICE
 *    (device memory of the context's GPU; read on the context's stream).
 *  - One context per host thread at a time.  All device work is ordered on
 *    the context's stream (the caller's, if one is given in emt_options).
 *  - Results are bitwise independent of how events are batched, of the
 *    track-slot capacity and of scheduling, except for the summation order
 *    of floating-point deposits (each track draws from its own
 *    counter-based random stream keyed on event, track id and step).
 */
#ifndef EMT_H
#define EMT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t emt_status;
#define EMT_OK 0
#define EMT_ERR_INVALID_ARG (-1) /* bad argument; nothing changed */
#define EMT_ERR_CAPACITY (-2)    /* does not fit; nothing admitted, state unchanged */
#define EMT_ERR_CUDA (-3)        /* CUDA error; the context is unusable */
#define EMT_ERR_BAD_STATE (-4)   /* call out of order (e.g. run before load) */
#define EMT_ERR_TIMEOUT (-5)     /* a bounded device wait gave up */
#define EMT_ERR_NOT_READY (-6)   /* the event has not finished */
#define EMT_ERR_HOST_OOM (-7)

#define EMT_PRECISION_FP64 0  /* FP64 everywhere: matches the FP64 oracle */
#define EMT_PRECISION_MIXED 1 /* FP32 tables and sampling; FP64 positions, distances, tallies */

#define EMT_HOST 0
#define EMT_DEVICE 1

/* process bits of emt_physics.process_mask */
#define EMT_PHOTO 1u
#define EMT_COMPTON 2u
#define EMT_PAIR 4u
#define EMT_IONI 8u
#define EMT_BREMS 16u
#define EMT_ANNIH 32u
#define EMT_ALL_PROCESSES 63u /* the six discrete processes */
/* options of the physics list (Table 1's multiple scattering is listed as
 * "in progress"; the Urban/WentzelVI and Livermore data are not available,
 * so each option is a published closed form):
 * MSC: after every e+- step in matter the direction turns by a polar angle
 *   whose projections are Gaussians of Highland's width (PDG review, Eq.
 *   34.15) for the pre-step momentum and the step length; no lateral
 *   displacement.
 * ANGULAR: bremsstrahlung photons and pair leptons leave at angles of the
 *   dipole distribution dN/dcos ~ (1 - beta cos)^-2, photoelectrons at
 *   angles of Sauter's K-shell distribution, instead of along the parent.
 * RAYLEIGH: coherent photon scattering, Thomson scattering off the atom
 *   with the form factor of an exponentially screened charge
 *   (Thomas-Fermi radius); a fourth photon process. */
#define EMT_MSC 64u
#define EMT_ANGULAR 128u
#define EMT_RAYLEIGH 256u

/* step-loop driver of emt_run */
#define EMT_LOOP_PLAIN 0 /* host loop: one kernel launch and one counter read per step */
#define EMT_LOOP_GRAPH 1 /* CUDA graph of several steps; one counter read per graph */
/* one persistent kernel (cooperative launch, fused step) runs up to
 * graph_steps steps per launch with a grid barrier between steps and ends
 * early when no track is left; one counter read per launch.  Removes the
 * launch gaps between steps (the paper's many synchronization points per
 * step, Sec. 3.2) where steps are short: one event at a time, the tail of
 * a run, a served stream at a low rate.  Every barrier wait is bounded
 * (10 s): a wait that gives up ends the launch and emt_run returns
 * EMT_ERR_TIMEOUT (the context is then unusable). */
#define EMT_LOOP_PERSISTENT 2

/* how one step is laid out on the GPU (same results either way):
 * FUSED: one kernel; interacting tracks are regrouped by model inside each
 *   block.  SPLIT: a transport kernel queues the interacting tracks in
 *   device memory and an interaction kernel samples them in full chunks
 *   sorted by model (needs one more buffer of slot_capacity records). */
#define EMT_SCHEDULE_FUSED 0
#define EMT_SCHEDULE_SPLIT 1
/* PIPELINED: one kernel per step: its blocks first sample the interactions
 * queued in the previous step (chunks sorted by model), then transport this
 * step's tracks, so transport and sampling work overlap on the GPU; an
 * interacting track's step completes one iteration later (no result
 * changes; two queue buffers of slot_capacity records; no track selection
 * or host spill). */
#define EMT_SCHEDULE_PIPELINED 2

typedef struct emt_ctx emt_ctx;

typedef struct emt_options {
    int32_t device;        /* CUDA device ordinal */
    int32_t precision;     /* EMT_PRECISION_* */
    int64_t slot_capacity; /* tracks in flight per step (each of two ping-pong buffers) */
    int32_t max_events;    /* events that can be in flight (score slots) */
    int32_t max_bins;      /* histogram width capacity (>= emt_world.n_bins) */
    int32_t block_size;    /* threads per block of the step kernel: 128 or 256; 0 = 256 */
    int32_t loop_mode;     /* EMT_LOOP_* */
    int32_t graph_steps;   /* steps per graph launch (EMT_LOOP_GRAPH; multiple of 6) or per
                              persistent launch (EMT_LOOP_PERSISTENT) */
    int32_t schedule;      /* EMT_SCHEDULE_*: how a step's interactions are grouped */
    uint32_t seed;         /* random stream seed */
    void* cuda_stream;     /* cudaStream_t to use, or NULL for a context-owned stream */
    void* device_pool;     /* caller-owned device memory, or NULL: see emt_pool_bytes */
    size_t pool_bytes;
    int32_t step_hist_bins; /* > 0: keep the steps-per-track histogram (Sec. 3.2 diagnostics),
                               emt_read_step_hist; 0: off (no cost) */
    int32_t select_policy;  /* EMT_SELECT_*: which tracks step when more than max_active are in flight */
    int64_t max_active;     /* > 0: at most this many tracks step per iteration, the others are
                               held unchanged (split schedule only); 0: every track steps */
    int64_t spill_above;    /* > 0 (with LOW_ENERGY selection, >= max_active): held tracks beyond
                               the spill_above lowest-energy ones move to host memory and come
                               back when fewer than spill_above/2 remain on the device (the
                               paper's buffering of secondaries in CPU memory; plain driver);
                               0: off */
} emt_options;

/* Track selection (Sec. 3.2: stepping the low-energy tracks first may lower
 * the number of track slots a problem needs).  Held
 * tracks keep their step counter, so they draw the same random numbers
 * when they step later: results do not depend on the policy or the budget
 * (up to the summation order of deposits).
 * ORDER: the first max_active tracks of the input (photons, then charged).
 * LOW_ENERGY: the max_active tracks of lowest kinetic energy, by quarter-
 *   octave energy classes counted as each step writes its outputs (ties in
 *   the last class admitted are broken arbitrarily). */
#define EMT_SELECT_ORDER 0
#define EMT_SELECT_LOW_ENERGY 1

/* Fill `opt` with defaults (device 0, FP64, 2^22 slots, 10,000 events,
 * 128 bins, plain loop, seed 1). */
void emt_default_options(emt_options* opt);

/* Bytes of device memory a context with these options needs.  A caller
 * that passes device_pool must pass at least this many bytes, aligned to
 * 256 bytes; the context then allocates no device memory of its own. */
size_t emt_pool_bytes(const emt_options* opt);

/* Create a context on opt->device.  Host: opt.  out receives the context. */
emt_status emt_create(const emt_options* opt, emt_ctx** out);
void emt_destroy(emt_ctx* ctx);
const char* emt_last_error(const emt_ctx* ctx);

/* Materials (Sec. 2.2: material-dependent properties; single element per
 * material, as in the paper's demonstration, Sec. 3.2 caveats).
 * rho_g_cm3 == 0 marks vacuum.  bk_MeV is the K-shell binding energy used by
 * the photoelectric model. */
typedef struct emt_material {
    double Z, A_g_mol, rho_g_cm3, I_eV, bk_MeV;
} emt_material;

/* Physics options (Sec. 2.2: processes, models and energy cutoffs).
 * cut_MeV: production and tracking cuts for gamma, e-, e+.
 * Tables are built on the device on the grid
 * E_n = grid_lo * 10^(n / bins_per_decade), n = 0..bpd*log10(hi/lo). */
typedef struct emt_physics {
    double cut_MeV[3];
    double grid_lo_MeV, grid_hi_MeV;
    int32_t bins_per_decade;
    uint32_t process_mask;
    double step_frac;      /* e+- step limit: max(step_frac R, min(R, final_range)) */
    double final_range_cm;
} emt_physics;

/* Load materials and build every cross-section and range table on the
 * device (host: mats[n], phys).  Replaces earlier tables.  n in [1, 16]. */
emt_status emt_load_materials(emt_ctx* ctx, const emt_material* mats, int32_t n, const emt_physics* phys);

/* Layered-box geometry (Sec. 2.3): layers stacked along +z from z0, each
 * |x| <= half_x, |y| <= half_y, inside the world box [lo, hi]; the world
 * outside the stack is vacuum.  material -1 means vacuum.  score_bin is
 * the histogram column of the layer (-1: not scored in the histogram). */
typedef struct emt_layer {
    int32_t material;
    int32_t score_bin;
    double thickness_cm;
} emt_layer;

/* Geometry kinds (Sec. 2.3; the paper's navigators are VecGeom and ORANGE,
 * a CSG of quadric surfaces, which this library replaces by two volume
 * kinds with exact logical volume indices):
 * LAYERS: layer i is the slab zb[i] <= z < zb[i+1] (zb[0] = z0, zb[i+1] =
 *   zb[i] + thickness) within |x| <= half_x, |y| <= half_y, inside the world
 *   box lo..hi of vacuum; leaving the box leaves the world.
 * CYLINDERS: layer i is the shell zb[i] <= rho < zb[i+1] about the z axis
 *   (radii accumulated from z0, which must be 0; the first layer is a solid
 *   cylinder) for |z| <= half_z; leaving the outermost shell or the end
 *   planes leaves the world (the envelope is the world).  half_x, half_y,
 *   lo and hi are ignored.  This is the geometry of Sec. 3.2's test problem
 *   (six single-element shells out to 375 cm). */
#define EMT_GEOM_LAYERS 0
#define EMT_GEOM_CYLINDERS 1

typedef struct emt_world {
    double z0_cm, half_x_cm, half_y_cm;
    double lo_cm[3], hi_cm[3];
    double B_tesla[3];        /* uniform field; zero = straight lines */
    double rk_delta_cm;       /* RK4 miss distance (chord sagitta bound) */
    double max_field_step_cm; /* longest path of one step in a field */
    int32_t max_steps;        /* per-track step limit; then the track is killed */
    int32_t n_bins;           /* histogram width (<= options.max_bins) */
    int32_t geometry;         /* EMT_GEOM_* */
    int32_t score_z;          /* 0: bin = the layer's score_bin; 1: n_bins equal bins of z
                                 over [score_z_lo, score_z_hi) (Sec. 3.2 tallies the
                                 deposition along z) */
    double half_z_cm;         /* CYLINDERS: half-length */
    double score_z_lo_cm, score_z_hi_cm;
} emt_world;

/* host: layers[n], world.  n in [1, 4096].  Every deposit of a step is
 * made at the step's end point, in the volume the step started in. */
emt_status emt_load_geometry(emt_ctx* ctx, const emt_layer* layers, int32_t n, const emt_world* world);

/* Primaries of a batch of events, structure of arrays, n entries:
 * event[i] indexes event_ids[] of the same submit call; type 0 gamma,
 * 1 e-, 2 e+; pos and dir are [n][3]; dir must be unit vectors.  Within an
 * event, primaries get track ids 1, 2, ... in submission order. */
typedef struct emt_primaries {
    int32_t n;
    const int32_t* event;
    const int32_t* type;
    const double* T_MeV;
    const double* pos_cm;
    const double* dir;
} emt_primaries;

/* Submit n_events new events (ids distinct from every event in flight)
 * with their primaries.  event_ids is host memory; the primary arrays
 * follow `where`.  Returns EMT_ERR_CAPACITY, admitting nothing, when the
 * free score slots or track slots do not suffice. */
emt_status emt_submit(emt_ctx* ctx, int32_t n_events, const uint64_t* event_ids, const emt_primaries* prim,
                      int32_t where);

typedef struct emt_run_stats {
    int64_t iterations;   /* step-loop iterations executed by this call */
    int64_t track_steps;  /* tracks advanced by one step, summed over iterations */
    int64_t peak_tracks;  /* largest number of tracks in flight seen by the host */
    int64_t deferred;     /* track-steps postponed for lack of output capacity */
    int64_t live_tracks;  /* tracks still in flight when the call returned */
    int64_t state_bytes;  /* track-state bytes read plus written by the step kernel */
    double kernel_ms;     /* device time of the step-kernel launches (CUDA events
                             around each launch, or each graph launch) */
    int32_t kernel_launches;
    int64_t held;         /* track copies held back by the track selection */
    int64_t spilled;      /* tracks moved to host memory by the host spill */
    int64_t peak_spilled; /* most tracks in host memory at once */
    int64_t rk4_substeps; /* RK4 substeps of charged tracks in a field (each evaluation of the
                             integrator, the repeat of a substep cut at a boundary included) */
} emt_run_stats;

/* Step every track in flight until none is left or max_iterations
 * (<= 0: no limit) iterations have run.  stats may be NULL.  When the track
 * slots cannot hold the next step (every track's step needs a second slot
 * and none is free), half of the stored tracks move to host memory with
 * their state and step counters and come back once fewer than a quarter of
 * the slots are in use (the paper's buffering of tracks in CPU memory,
 * Sec. 3.2); results do not change (stats.spilled counts those moves).
 * EMT_ERR_CAPACITY remains only for a pipelined interaction queue that
 * fills the slots by itself. */
emt_status emt_run(emt_ctx* ctx, int32_t max_iterations, emt_run_stats* stats);

/* Per-step diagnostics (Sec. 3.2, tracks in flight and time per step): as
 * emt_run with the plain driver, recording for each iteration the photons
 * and charged tracks in flight at its start, the tracks queued for an
 * interaction (split schedule; -1 under the fused one), the track-steps
 * deferred for lack of output capacity, the tracks held back by the track
 * selection (emt_options.max_active), and the device time of the step's
 * launches.  host rec[cap]; *n_rec = records written (iterations beyond
 * cap are run but not recorded). */
typedef struct emt_step_record {
    int64_t photons;
    int64_t charged;
    int64_t interacting;
    int64_t deferred;
    int64_t held;  /* held back by the track selection */
    double ms;
} emt_step_record;

emt_status emt_run_traced(emt_ctx* ctx, int32_t max_iterations, emt_run_stats* stats, emt_step_record* rec,
                          int32_t cap, int32_t* n_rec);

/* Steps-per-track histogram (Sec. 3.2: steps per track by particle type),
 * kept when emt_options.step_hist_bins > 0: host out[3][step_hist_bins],
 * counts of finished tracks by type (0 gamma, 1 e-, 2 e+) and number of
 * steps, tracks of step_hist_bins - 1 or more steps in the last bin,
 * accumulated over every run since the context was created or the last
 * reset (reset != 0 clears it after reading).  EMT_ERR_BAD_STATE if the
 * histogram is off. */
emt_status emt_read_step_hist(emt_ctx* ctx, uint64_t* out, int32_t bins, int32_t reset);

/* Per-event results: summary = {edep, escaped, killed, e_in, n_steps,
 * n_tracks} (MeV, MeV, MeV, MeV, count, count); edep includes deposits in
 * layers without a score bin. */
#define EMT_SUMMARY_LEN 6

/* Events finished since the last poll (host: done_ids[cap]). */
emt_status emt_poll(emt_ctx* ctx, uint64_t* done_ids, int32_t cap, int32_t* n_done);

/* Read and release one finished event.  host: hist[n_bins], summary[6]
 * (either may be NULL).  EMT_ERR_NOT_READY if it has not finished. */
emt_status emt_read_event(emt_ctx* ctx, uint64_t event_id, double* hist, double* summary);

/* Read and release every event in flight, in submission order, after an
 * emt_run that left no track (EMT_ERR_NOT_READY otherwise).
 * hist[n_events][n_bins] and summary[n_events][6] follow `where`;
 * ids (host, may be NULL) receives the event ids. */
emt_status emt_read_all(emt_ctx* ctx, double* hist, double* summary, uint64_t* ids, int32_t where);
int32_t emt_events_in_flight(const emt_ctx* ctx);
/* Tracks waiting for their next step (as of the last call), including
 * tracks spilled to host memory. */
int64_t emt_tracks_in_flight(const emt_ctx* ctx);

/* ---------------------------------------------------------------------
 * Serving (Sec. 2.4: many concurrent events keep the device busy; Sec. 3.2:
 * workflows must batch events).  emt_serve replays a stream of event
 * requests against one context in real time (arrival times divided by
 * time_scale) and returns when every request has been answered.
 *   EMT_SERVE_CONTINUOUS: requests are admitted as soon as event slots and
 *     track slots allow, while earlier events are still in flight; the step
 *     loop advances steps_per_poll iterations between admissions and
 *     finished events are read back immediately (continuous batching).
 *   EMT_SERVE_BATCH: one batch at a time: whenever no event is in flight,
 *     every request that has arrived is admitted and run to completion.
 * host arrays, n_events entries in arrival order: event_ids (distinct, none
 * in flight), arrival_s (non-decreasing), first/count (the request's
 * primaries are prim[first .. first+count), requests contiguous and in
 * order); prim: host primaries as in emt_submit (its `event` field is
 * ignored).  Outputs (host): admit_s, done_s (seconds since the call
 * started; admit_s may be NULL), hist[n_events][n_bins] and
 * summary[n_events][6] (either may be NULL).  The loop uses only the entry
 * points above and leaves the context empty.
 * --------------------------------------------------------------------- */
#define EMT_SERVE_CONTINUOUS 0
#define EMT_SERVE_BATCH 1

typedef struct emt_serve_options {
    int32_t mode;           /* EMT_SERVE_* */
    int32_t steps_per_poll; /* iterations between admissions (continuous) */
    int32_t n_bins;         /* histogram width of hist (the geometry's n_bins) */
    double time_scale;      /* 1 = real time; > 1 replays faster */
    int64_t admit_below;    /* admit new requests only while fewer tracks are in
                               flight (room for showers to grow); <= 0: no limit */
} emt_serve_options;

emt_status emt_serve(emt_ctx* ctx, int32_t n_events, const uint64_t* event_ids, const double* arrival_s,
                     const int32_t* first, const int32_t* count, const emt_primaries* prim,
                     const emt_serve_options* opt, double* admit_s, double* done_s, double* hist, double* summary);

/* Measurement support (the paper has no counterpart): the FP64 fused
 * multiply-add rate of device `device`, measured with independent DFMA
 * chains over four full-occupancy waves of every SM, best of `repeats`
 * launches of `iters` iterations (CUDA events); the denominator of the
 * step kernels' FP64 roofline.  Allocates and frees a small buffer of its
 * own.  host fma_per_s receives DFMA operations (one per thread) per
 * second.  EMT_ERR_INVALID_ARG for non-positive counts, EMT_ERR_CUDA if
 * the device cannot run it. */
emt_status emt_measure_dfma_rate(int32_t device, int32_t iters, int32_t repeats, double* fma_per_s);

/* Measurement support (the paper has no counterpart): throughput of FP64
 * division and natural logarithm on device `device`, native and as the step
 * kernels compute them on the integer pipe (bit-identical division;
 * logarithm correctly rounded but for rare arguments), each with
 * independent chains per thread over eight blocks of 256 threads per SM,
 * best of `repeats` launches of `iters` iterations (CUDA events); every
 * operation carries one FP64 addition.  host rates[4] receives operations
 * per second: native division, integer-pipe division, native log,
 * integer-pipe log.  Allocates and frees a small buffer of its own.
 * EMT_ERR_INVALID_ARG for non-positive counts or a null pointer,
 * EMT_ERR_CUDA if the device cannot run it. */
emt_status emt_measure_fp64_op_rates(int32_t device, int32_t iters, int32_t repeats, double* rates);

/* Diagnostics of the bounded device wait of EMT_LOOP_PERSISTENT (the
 * paper has no counterpart): launches the same grid barrier on a device
 * with one participant missing, so that its wait can only run out after
 * timeout_ms (1..60000).  Returns EMT_ERR_TIMEOUT when the wait gave up,
 * ended the kernel and reported it in the status word, as it must;
 * EMT_OK would mean the barrier did not wait; EMT_ERR_INVALID_ARG for a
 * bad timeout; EMT_ERR_CUDA on a CUDA failure.  Allocates and frees a few
 * bytes of device memory of its own; the device stays usable. */
emt_status emt_debug_wait_timeout(int32_t device, int32_t timeout_ms);

/* Diagnostics: copy table (material m, particle p, quantity q) to host
 * out[n] (n = grid size).  gamma q: 0 photo, 1 compton, 2 pair;
 * e-: 0 ioni, 1 brems, 3 range; e+: 0 ioni, 1 brems, 2 annih, 3 range;
 * q = 4: restricted stopping power; q = 5: energy grid.  Returns the grid
 * size in *n_out.  Values are FP64 regardless of precision.  gamma q = 3 is
 * the Rayleigh cross section (zero unless EMT_RAYLEIGH is on). */
emt_status emt_get_table(emt_ctx* ctx, int32_t m, int32_t p, int32_t q, double* out, int32_t cap, int32_t* n_out);

/* Diagnostics: replace the tracks in flight by explicit track states and
 * read them back, to check single steps (fused or split schedule;
 * EMT_ERR_BAD_STATE with the pipelined one).  rec[n][10] = {type, T, x, y, z,
 * ux, uy, uz, volume (-1 world vacuum), step}; uid[n]; event_slot[n]
 * indexes the events of the last submit.  host memory. */
emt_status emt_debug_set_tracks(emt_ctx* ctx, int32_t n, const double* rec, const uint64_t* uid,
                                const int32_t* event_slot);
/* Returns every track in flight (photons first) in rec/uid/event_slot
 * (host, capacity cap); *n_out = number of tracks. */
emt_status emt_debug_get_tracks(emt_ctx* ctx, int32_t cap, double* rec, uint64_t* uid, int32_t* event_slot,
                                int32_t* n_out);

/* ---------------------------------------------------------------------
 * Allocation-free transport.  The paper has no counterpart to this call.
 *
 * For callers that must not allocate device memory: code running inside a
 * framework whose caching allocator already owns the GPU's memory, a host
 * plugin whose sandbox forbids new device allocations, or a latency-bound
 * serving loop that cannot afford the device-wide synchronisation a
 * cudaMalloc/cudaFree may cause.  This one call transports a small batch
 * of events from start to finish (FP64, plain step loop) using only a
 * fixed device array compiled into the library (64 MiB, held by every GPU
 * that loads the library until the process exits).  It calls no
 * cudaMalloc, cudaFree or other allocating routine.
 *
 * Limits (larger inputs return EMT_ERR_CAPACITY, nothing is run):
 * n_events <= EMT_STATIC_MAX_EVENTS, prim->n <= EMT_STATIC_MAX_PRIMARIES,
 * world->n_bins <= EMT_STATIC_MAX_BINS, and the tracks in flight at any
 * step <= EMT_STATIC_MAX_TRACKS (a step that would exceed it is deferred;
 * if no track can advance the call returns EMT_ERR_CAPACITY).
 *
 * Arguments: device ordinal; seed; host arrays mats[n_mat], phys,
 * layers[n_layers], world, event_ids[n_events] (as emt_load_materials,
 * emt_load_geometry and emt_submit); prim: device arrays grouped by event
 * as in emt_submit; hist[n_events][n_bins] and summary[n_events][6]:
 * caller-owned device buffers written in event order; cuda_stream: the
 * stream to run on (NULL: the legacy default stream).  Returns when the
 * results are complete.  A primary whose type is not 0, 1 or 2 returns
 * EMT_ERR_INVALID_ARG before any step runs (hist and summary unwritten).
 *
 * The first call on a device looks up the device address of the fixed
 * array (cudaGetSymbolAddress); make that first call before any stream
 * capture.  Every call reuses the same array and clears what must start
 * at zero, so calls that overlap on the GPU (from two threads or on two
 * streams) race with each other: serialize them.
 * --------------------------------------------------------------------- */
#define EMT_STATIC_MAX_EVENTS 256
#define EMT_STATIC_MAX_PRIMARIES 65536
#define EMT_STATIC_MAX_BINS 128
#define EMT_STATIC_MAX_TRACKS (1 << 18)

emt_status emt_transport_static(int32_t device, uint32_t seed, const emt_material* mats, int32_t n_mat,
                                const emt_physics* phys, const emt_layer* layers, int32_t n_layers,
                                const emt_world* world, int32_t n_events, const uint64_t* event_ids,
                                const emt_primaries* prim, double* hist, double* summary, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* EMT_H */
