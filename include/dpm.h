/*
 * dpm.h -- C ABI of the GB300 coupled electron-photon Monte Carlo dose library.
 *
 * Method: Jia et al., "Development of a GPU-based Monte Carlo dose calculation
 * code for coupled electron-photon transport" (arXiv:0910.0329):
 *   Sec. 2.1  DPM transport scheme (condensed-history electrons with CSDA below
 *             the cuts and detailed Moller/bremsstrahlung above them, random
 *             hinge elastic deflections, Woodcock photon tracking);
 *   Sec. 2.2  the run: load data, transport N histories (each source particle
 *             with all its secondaries), read the dose back;
 *   Sec. 2.3  single-precision transport arithmetic;
 *   Sec. 2.4  per-voxel dose accumulation with atomic adds; per-thread RNG;
 *   Sec. 3    point source, field at SAD, absorption energies, sigma_D.
 *
 * Conventions for every call:
 *   - returns a dpm_status code (0 = success); no exceptions cross the ABI;
 *     dpm_last_error() gives a message for the last failing call on a context;
 *   - host pointers are owned by the caller and only read (or written, for
 *     outputs) during the call; the context owns every device allocation it
 *     makes and frees it in dpm_destroy();
 *   - work is queued on the context's stream (dpm_set_stream, default: a
 *     stream the context creates); dpm_run() is asynchronous, dpm_read_dose()
 *     and dpm_sync() synchronise and report device-side errors;
 *   - a context is used by one host thread at a time (contexts on different
 *     threads, or different devices, are independent);
 *   - phantom layout: voxel v = i + nx*(j + ny*k); the phantom occupies
 *     [0,nx*dx] x [0,ny*dy] x [0,nz*dz] cm; mat[v] indexes the material list
 *     given to dpm_build_tables(); rho[v] is the mass density in g/cm^3.
 * Units: MeV, cm, g/cm^3.
 */
#ifndef DPM_H
#define DPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dpm_ctx dpm_ctx;

typedef enum {
    DPM_OK = 0,
    DPM_EINVAL = -1,          /* bad argument (null pointer, size, range) */
    DPM_ENOMEM = -2,          /* device allocation failed */
    DPM_ECUDA = -3,           /* a CUDA runtime call failed (message has the CUDA error) */
    DPM_EQUEUE_OVERFLOW = -4, /* a particle queue or stack overflowed: rerun with larger capacity */
    DPM_ETIMEOUT = -5,        /* a bounded device wait gave up */
    DPM_ESTATE = -6,          /* call out of order (e.g. run before tables) */
    DPM_ESTEPCAP = -7         /* a particle exceeded its step or flight limit (far above any
                                 real track); its remaining energy was deposited where it stopped */
} dpm_status;

#define DPM_MAX_ELEM 8
#define DPM_MAX_MAT 16

/* A material: elements (atomic number Z, molar mass A in g/mol, mass fraction
   w) and mean excitation energy I in eV. */
typedef struct {
    int n_elem;
    double Z[DPM_MAX_ELEM], A[DPM_MAX_ELEM], w[DPM_MAX_ELEM];
    double i_ev;
    double rho_de;  /* g/cm^3 at which the Sternheimer-Peierls density-effect
                       correction of the collision stopping power is evaluated
                       (the material's nominal density); 0 = no density effect */
} dpm_material;

/* Transport and table parameters (Sec. 3 absorption energies; the cuts and
   step parameter of the condensed-history scheme of Sec. 2.1). */
typedef struct {
    double eabs_e;  /* electron absorption energy (MeV) */
    double eabs_g;  /* photon absorption energy (MeV) */
    double wcc;     /* Moller hard-collision cut (MeV) */
    double wcr;     /* bremsstrahlung hard-emission cut (MeV) */
    double f_e;     /* maximum fractional CSDA energy loss per electron step */
    double c_pe;    /* photoelectric strength: mu_pe/rho = c_pe sum(w Z^4/A) / E^3 */
    double e_max;   /* highest particle energy the tables must cover (MeV) */
    int n_e;        /* energy nodes of the per-material tables (>= 64) */
} dpm_table_params;

/* Beam (Sec. 3): point source at distance `sad` from the isocentre `iso`;
   the fx x fy field lies in the isocentre plane normal to the beam axis;
   gantry_deg rotates the beam about the y axis through the isocentre
   (0 = travelling along +z). */
typedef struct {
    int particle;   /* 0 photon, 1 electron */
    int spectrum;   /* 0 monoenergetic at `energy`, 1 synthetic 6 MV (1-E/6)E^-1/2 on [0.25,6] MeV */
    double energy;
    double iso[3];
    double sad, fx, fy, gantry_deg;
} dpm_source;

/* Kernel selection and launch shape.  Zero fields take defaults. */
enum {
    DPM_KERNEL_QUEUE = 0,
    DPM_KERNEL_HISTORY = 1,
    DPM_KERNEL_PAPER_F32 = 2,
    DPM_KERNEL_PAPER_CAS = 3,
    DPM_KERNEL_HISTORY_F64 = 4
};
typedef struct {
    int kernel;        /* DPM_KERNEL_QUEUE (persistent, particle queues);
                          DPM_KERNEL_HISTORY (one history per thread, private stack);
                          DPM_KERNEL_PAPER_F32 / _CAS: DPM_KERNEL_HISTORY with the paper's
                          tally (Sec. 2.4) instead of the exact one, as an ablation: a
                          sparse per-thread (voxel, energy) counter emptied at the end of
                          each history into float slabs by atomic float adds (native, or
                          a compare-and-swap loop), then rounded to the fixed-point tally.
                          Same trajectories as the other kernels; the tally differs from
                          theirs by float rounding and is not reproducible bit for bit.
                          DPM_KERNEL_HISTORY_F64: DPM_KERNEL_HISTORY with every transport
                          operation in FP64 and the tables in FP64 (Sec. 2.3 runs the
                          transport in single precision; this measures what that costs).
                          Same random numbers; trajectories part from the FP32 ones where
                          a rounding flips a decision, so its tally agrees statistically.
                          The kernels other than DPM_KERNEL_QUEUE are dpm_run only
                          (DPM_EINVAL elsewhere or for other values). */
    int n_batches;     /* history batches for the sigma estimate (default 50, max 1024) */
    int block_size;    /* per-history kernel: threads per block (multiple of 32; 0 = 128).
                          The queue kernel always runs blocks of 128 threads (it schedules
                          per warp); its size is set by blocks_per_sm */
    int blocks_per_sm; /* queue kernel: resident blocks per SM (0 = as many as fit, 8) */
    int queue_log2;    /* queue kernel: log2 of each queue shard's capacity (7..20; 0 = 15 for
                          an electron-beam dpm_run, 14 otherwise) */
    int refill_min;    /* queue kernel: idle lanes before a warp refills (1..32; 0 = 24 for
                          photon warps, 12 for electron warps) */
    double timeout_s;  /* bound on any device wait (default 20 s) */
    int physics_flags; /* DPM_NO_HARD: no Moller/bremsstrahlung events; DPM_NO_MSC: no
                          elastic deflections (test and ablation switches; 0 = full physics);
                          DPM_SAUTER: photoelectrons leave at Sauter's K-shell polar angle
                          about the photon direction (default: along it); dpm_run only
                          (dpm_run_batch returns DPM_EINVAL) */
    int queue_limit;   /* fault injection: largest occupancy of a queue shard (0 = capacity);
                          a push that finds no shard below it is an overflow */
    int use_graph;     /* dpm_run_batch only: capture zero -> transport -> fold in a CUDA
                          graph and replay it while the batch keeps its shape */
    int count_events;  /* queue kernel: 1 = also count electron steps, photon flights and
                          interactions, tally atomics and secondaries for dpm_run_stats
                          (about 10 % slower); 0 = those counts read 0.  The energy
                          counters and the tally are the same either way.  The per-history
                          kernels always count. */
    int refill_pause;  /* queue kernel: a warp with particles whose refill found nothing
                          waits 128 steps before it tries again (1), or tries on every
                          step (-1); 0 = automatic: the pause for launches of at most
                          1.6e7 photon-beam histories or 2e6 electron-beam histories
                          (a batch launch: its jobs' histories, an electron history
                          counting 8), where it shortens the end of the launch, and none
                          above, where it costs about 1.5 %; none either with queue
                          shards below 2^13 slots (queue_log2 < 13, or
                          dpm_run_noalloc's), which need every refill to keep from
                          overflowing.  Scheduling only: the tally is the same either
                          way, unless a queue overflows. */
} dpm_run_opts;
enum { DPM_NO_HARD = 1, DPM_NO_MSC = 2, DPM_SAUTER = 4 };

/* Run summary returned by dpm_read_dose(). Energies in MeV. */
typedef struct {
    uint64_t n_histories;
    int32_t n_batches;
    int32_t error_flags;          /* bit 0 stack/queue overflow, bit 1 step cap, bit 2 timeout */
    double emitted, deposited, escaped, missed;
    uint64_t n_e_steps, n_g_flights, n_g_interactions;
    uint64_t n_tally_atomics;     /* 64-bit atomic adds issued to the tally */
    uint64_t n_pushed;            /* secondaries created */
    double transport_ms;          /* device time of the transport kernels of the runs read
                                     (CUDA events recorded around each launch on its stream; a
                                     phantom keeps the events of at most 1024 unread runs, the
                                     times of older ones are summed early, waiting for them) */
    double fold_ms;               /* device time of the batch folds of those runs */
    uint64_t n_transport_launches;/* transport kernel launches since the previous read */
    uint64_t n_phase_switches;    /* queue kernel: grid-wide switches between the source phase and
                                     the secondary phase (0 for the per-history kernel) */
} dpm_run_stats;

/* A context on CUDA device `cuda_device`.  hbm_budget_bytes (0 = no limit)
   bounds the device memory the context keeps: tables, phantoms, tallies,
   particle queues, batch and server buffers, and the diagnostics' temporary
   buffers while they live.  An allocation that would exceed it fails with
   DPM_ENOMEM before calling cudaMalloc, and the call that needed it fails
   with that status (a run's admission control; the request server applies
   its own budget to its slots on top).  DPM_ECUDA if the device is absent.
   The call also loads, on that device, the library's kernels and the fixed
   scratch of dpm_run_noalloc() (see there). */
int dpm_create(dpm_ctx **out, int cuda_device, uint64_t hbm_budget_bytes);
void dpm_destroy(dpm_ctx *ctx);
const char *dpm_last_error(const dpm_ctx *ctx);
/* Device bytes the context holds now and its budget (either may be NULL). */
int dpm_device_bytes(const dpm_ctx *ctx, uint64_t *in_use, uint64_t *budget);

/* Use an external CUDA stream (cudaStream_t passed as void*); NULL restores
   the context's own stream.  Waits for the work queued on the previous stream
   first, so that no run of the context overlaps another. */
int dpm_set_stream(dpm_ctx *ctx, void *cuda_stream);

/* Copy a voxel phantom (host arrays, nx*ny*nz entries) to the device.  Sizes
   up to 2047 x 2047 x 1023 voxels.  Returns its id in *phantom_id. */
int dpm_load_phantom(dpm_ctx *ctx, int nx, int ny, int nz, double dx, double dy, double dz,
                     const uint8_t *mat, const float *rho, int *phantom_id);
int dpm_free_phantom(dpm_ctx *ctx, int phantom_id);

/* A new phantom with the geometry, materials, densities and photon majorant
   of phantom src_id and an empty tally, copied on the device (no host
   arrays, no wait: the copies are queued on the context's stream).  For
   several tallies of one geometry, e.g. concurrent dose requests. */
int dpm_clone_phantom(dpm_ctx *ctx, int src_phantom_id, int *phantom_id);

/* Replace the contents (materials and densities, host arrays of nx*ny*nz
   entries with the phantom's dimensions) of a loaded phantom without
   reallocating: waits for earlier work on the context's stream, copies the
   arrays (page-locked host memory makes the copies faster), recomputes the
   photon majorant and resets the tally as dpm_reset_tally() does.  Same
   validation as dpm_load_phantom(). */
int dpm_update_phantom(dpm_ctx *ctx, int phantom_id, const uint8_t *mat, const float *rho);

/* Build the FP32 device tables (per-material attenuation, range, stopping
   power, hard cross sections, transport mean free path; inverse-CDF sampling
   tables) from FP64 closed forms of the model.  The per-material tables have
   n_e nodes uniformly spaced in ln E from 0.99*min(eabs_e, eabs_g) to
   1.01*e_max and are interpolated linearly.  Must precede dpm_run(). */
int dpm_build_tables(dpm_ctx *ctx, const dpm_material *mats, int n_mat, const dpm_table_params *p);

/* Transport histories [first_history, first_history + n_histories) from
   `src` into the phantom's tally (Sec. 2.2).  Random numbers are keyed by
   (seed, history id, particle id), so the tally does not depend on launch
   shape, and splitting a history range over several calls adds up to the
   same integer tally.  Asynchronous on the context stream. */
int dpm_run(dpm_ctx *ctx, int phantom_id, const dpm_source *src, uint64_t first_history,
            uint64_t n_histories, uint64_t seed, const dpm_run_opts *opts);

/* One entry of a batch: a loaded phantom, a beam, a history range and a seed. */
typedef struct {
    int phantom_id;
    dpm_source src;
    uint64_t first_history, n_histories, seed;
} dpm_job;

/* Transport several jobs in ONE persistent queue launch (up to 1024 jobs on
   distinct phantoms).  New histories are drawn job after job while the
   particles of earlier jobs are still in flight, so the GPU stays full across
   job boundaries.  Each job accumulates into its phantom's tally exactly as
   dpm_run() with the same arguments would: the random numbers are keyed by
   (seed, history, particle), so the integer tally is the same.  With
   opts->use_graph the device work (zero slabs -> transport -> folds) is
   captured in a CUDA graph on the first call and replayed on later calls whose
   jobs have the same phantoms, history counts and options; the history ranges,
   seeds and beams may change between replays.  Asynchronous like dpm_run(). */
int dpm_run_batch(dpm_ctx *ctx, const dpm_job *jobs, int n_jobs, const dpm_run_opts *opts);

/* Counters (summed over jobs) and transport time of the batches run since
   the previous call; synchronises and reports device-side errors. */
int dpm_batch_stats(dpm_ctx *ctx, dpm_run_stats *stats);

/* Zero the phantom's accumulated tally and statistics. */
int dpm_reset_tally(dpm_ctx *ctx, int phantom_id);

/* Synchronise and read the accumulated result.  dose_gy and sigma_gy (Gy per
   history, sigma of the mean by the batch method) and s1_raw (integer tally,
   units of 2^-32 MeV) are caller-allocated host arrays of nx*ny*nz entries;
   any of them may be NULL.  stats may be NULL. */
int dpm_read_dose(dpm_ctx *ctx, int phantom_id, double *dose_gy, double *sigma_gy, int64_t *s1_raw,
                  dpm_run_stats *stats);

/* Same, writing dose and sigma into caller-allocated *device* arrays. */
int dpm_read_dose_device(dpm_ctx *ctx, int phantom_id, double *d_dose_gy, double *d_sigma_gy,
                         dpm_run_stats *stats);

/* The stop rule of a dose request (Sec. 3 reports sigma_D/D; here at D_max):
   for each of n phantoms, find on the device the voxel of largest accumulated
   dose and return its dose (Gy per history), its sigma (batch method) and its
   index in out[3*i .. 3*i+2] (index -1 when nothing was deposited).
   Synchronises.  ids and out are host arrays. */
int dpm_dmax_sigma(dpm_ctx *ctx, const int *phantom_ids, int n, double *out);

/* Wait for queued work; reports device-side errors of earlier runs. */
int dpm_sync(dpm_ctx *ctx);

/* ---- serving: dose requests with continuous batching --------------------
   Not a step of the paper's method (it runs one problem per program,
   Sec. 2.2).  A server works on one context.  A request is a beam on a
   geometry: a phantom loaded in the context.  An admitted request gets a
   tally slot, a device copy of its geometry (dpm_clone_phantom), while the
   slots' device memory stays within hbm_budget_bytes.  Each call of
   dpm_server_round():
   - admits pending requests in submission order;
   - takes the active requests oldest first while their next chunks fit
     round_budget histories (the oldest always);
   - transports them in one dpm_run_batch();
   - measures each one's D_max and sigma on the device (dpm_dmax_sigma);
   - marks done the requests whose relative sigma at D_max reached
     target_rel_sigma.
   A request's first round has first_chunk histories.  With `adaptive`, later
   rounds run about n (r/target)^2 * overshoot - n histories (r the relative
   sigma after n histories), within [first_chunk, max_chunk].  Round sizes,
   history ranges (consecutive, with the request's seed) and the stop
   decision depend only on the request's own tally, so its result is the
   same alone or with any other requests.  A done request keeps its slot,
   whose tally dpm_read_dose(ctx, status.slot, ...) reads, until
   dpm_server_release() returns the slot to its geometry's pool.  A slot
   that does not fit the budget frees released slots of other geometries
   first (dpm_free_phantom).  The server keeps its slots as phantoms of the
   context; they are freed with the context, not with the server.  Errors of
   a round (queue overflow, timed-out wait, device allocation) are returned
   by dpm_server_round(), with the message in dpm_last_error(ctx); the
   server's calls are not thread-safe (one caller per context). */
typedef struct dpm_server dpm_server;
typedef struct {
    double target_rel_sigma;   /* stop at sigma/D at D_max <= this, in (0, 1) */
    uint64_t first_chunk;      /* histories of a request's first round (0 = 200000) */
    uint64_t max_chunk;        /* cap of a later round (0 = 32 * first_chunk; <= 2^31-1) */
    double overshoot;          /* factor on the histories a later round aims at (0 = 1.15) */
    uint64_t round_budget;     /* histories per round (0 = 40 * first_chunk) */
    int n_batches;             /* history batches per round for sigma (0 = 10) */
    int max_active;            /* admitted requests at most (0 or > 1024 = 1024) */
    int adaptive;              /* 1: size later rounds from sigma; 0: every round first_chunk */
    uint64_t hbm_budget_bytes; /* device memory of all slots (0 = no limit) */
} dpm_serve_opts;
enum { DPM_REQ_PENDING = 0, DPM_REQ_ACTIVE = 1, DPM_REQ_DONE = 2, DPM_REQ_RELEASED = 3 };
typedef struct {
    int state;                 /* DPM_REQ_* */
    int slot;                  /* phantom id of the request's tally slot (-1 before admission / after release) */
    uint64_t histories;        /* transported so far */
    int rounds;
    double rel_sigma;          /* relative sigma at D_max after the last round (inf before) */
    double dose_max;           /* D_max, Gy per history */
    int dmax_voxel;
} dpm_request_status;
/* A server on ctx (opts may be NULL: all defaults; target_rel_sigma must then
   be set, so NULL gives DPM_EINVAL).  DPM_EINVAL for invalid options. */
int dpm_server_create(dpm_ctx *ctx, const dpm_serve_opts *opts, dpm_server **server);
/* Frees the server's host state; its slots stay phantoms of the context. */
void dpm_server_destroy(dpm_server *server);
/* Queue a request on geometry_id (a loaded phantom, not a slot); *request_id
   numbers requests from 0 in submission order.  The source is copied.
   DPM_EINVAL for a bad geometry id or a null pointer. */
int dpm_server_submit(dpm_server *server, int geometry_id, const dpm_source *src, uint64_t seed, int *request_id);
/* One round (synchronous); *n_completed receives the requests it finished.
   Does nothing when no request is active or admissible.  If it returns an
   error the round's requests keep their state from before the round, but
   their tallies may hold part of the failed round: destroy the server and
   resubmit the requests to a new one (the old slots stay phantoms of the
   context until dpm_free_phantom or dpm_destroy). */
int dpm_server_round(dpm_server *server, int *n_completed);
/* A request's state and statistics; DPM_EINVAL for a bad id. */
int dpm_server_status(dpm_server *server, int request_id, dpm_request_status *status);
typedef struct {
    int n_pending;             /* submitted, not yet admitted */
    int n_active;              /* admitted, not done */
    int n_done;                /* done, not yet released */
    int max_active;            /* most requests active in one round */
    uint64_t n_rounds;         /* rounds that ran a batch */
    uint64_t n_completed;      /* requests that reached the target */
    uint64_t histories;        /* histories transported by all rounds */
    uint64_t slot_bytes;       /* device bytes the slots hold now (counted as dpm_server_slot_bytes) */
    uint64_t peak_slot_bytes;  /* most slot bytes held at once */
    double gpu_ms;             /* device time of the rounds' batches (CUDA events) */
} dpm_server_info;
/* The server's counters; DPM_EINVAL for a null pointer. */
int dpm_server_info_get(dpm_server *server, dpm_server_info *info);
/* Device bytes one slot of geometry_id counts against hbm_budget_bytes:
   material, density, S1, Q, n_batches batch slabs per voxel and the fixed
   per-phantom buffers.  DPM_EINVAL for a bad geometry id. */
int dpm_server_slot_bytes(dpm_server *server, int geometry_id, uint64_t *bytes);
/* Return a done request's slot (tally reset) to its geometry's pool;
   DPM_ESTATE unless the request is done. */
int dpm_server_release(dpm_server *server, int request_id);
/* The server's policies as pure host functions (no context, no GPU):
   the histories of a request's next round after `histories` at relative
   sigma `rel_sigma` (0 for invalid options), and the round selection over
   requests oldest first (next_n[i] histories each; fills chosen with the
   indexes taken; returns their count, -1 for bad arguments). */
uint64_t dpm_serve_next_chunk(const dpm_serve_opts *opts, uint64_t histories, double rel_sigma);
int dpm_serve_select(const uint64_t *next_n, int n, uint64_t budget, int *chosen);

/* ---- diagnostics used by the parity tests ------------------------------ */

/* Evaluate the device tables at n energies (host arrays).  which: 0 mu/rho
   total (cm^2/g), 1 Compton fraction, 2 photoelectric fraction, 3 range
   R(T) from the lowest table energy (g/cm^2), 4 stopping power (MeV cm^2/g),
   5 hard cross section (cm^2/g), 6 inverse transport mfp (cm^2/g), 7 Moller
   fraction of the hard cross section, 8 CSDA energy after mass path
   aux[i] starting from energy[i], 9 majorant mu_max of phantom `mat`
   (1/cm, `mat` is then the phantom id). */
int dpm_diag_table(dpm_ctx *ctx, int which, int mat, int n, const double *energy, const double *aux, double *out);

/* Run the device samplers on n uniforms u[i] (host) at energy e (MeV):
   which 0 KN eps, 1 Moller eps = W/T, 2 brems k (MeV), 3 pair eps,
   4 MSC 1-mu for q = aux (mean of 1-mu), 5 6 MV spectrum energy,
   6 exponential path -ln(u) in mean free paths, 7 direction rotation: the
   unit vector (0.36, -0.48, 0.8) (aux 0..2) or +z (aux 3..5) turned by polar
   cosine e and azimuth 2 pi u, its component int(aux) % 3, 8 path from
   x = u cm to the far face of a 1 cm voxel [0, 1) along direction cosine e,
   9 Sauter's 1 - cos(theta) of a photoelectron of kinetic energy e. */
int dpm_diag_sample(dpm_ctx *ctx, int which, double e, double aux, int n, const double *u, double *out);

/* n Philox4x32-10 blocks for counters ctr[4*i..] and keys key[2*i..] (host). */
int dpm_diag_philox(dpm_ctx *ctx, int n, const uint32_t *ctr, const uint32_t *key, uint32_t *out);

/* L2 ceilings of this GPU for the roofline of the transport kernel (not a
   step of the paper's method).  Over a device buffer of ws_bytes (a power of
   two in [1 MiB, 64 MiB], small enough to stay in L2; the call allocates and
   frees it) it times, after a warm-up launch of each:
     out[0]  scattered 64-bit atomic adds per second (xorshift32 addresses,
             the access pattern of the voxel tally);
     out[1]  bytes per second of 16-byte loads that bypass L1, swept 16 times
             over the buffer.
   Synchronous.  DPM_EINVAL for a bad size or a null out (host, 2 doubles). */
int dpm_diag_l2_peaks(dpm_ctx *ctx, uint64_t ws_bytes, double *out);

/* The atomic ceiling of the voxel tally for a given deposit address stream
   (not a step of the paper's method): ids[0..n) (host; voxel indices below
   n_vox, n <= 2^28) are issued as 64-bit atomic adds into a zeroed slab of
   n_vox counters by a grid of 8 blocks of 256 threads per SM, once to warm
   L2 and once timed.  *rate receives adds per second.  The call allocates
   and frees its device buffers and is synchronous.  DPM_EINVAL for bad
   sizes or an id out of range. */
int dpm_diag_atomic_replay(dpm_ctx *ctx, const uint32_t *ids, uint64_t n, uint64_t n_vox, double *rate);

/* ---- transport without device allocation -------------------------------
   Not a step of the paper's method (the paper has no counterpart): an entry
   point for callers that cannot allocate device memory once they are running,
   e.g. a program whose device memory is owned by a pool or arena that forbids
   further cudaMalloc, or one held to a fixed device-memory budget set at
   start-up.  It runs the persistent queue transport of dpm_run() with the same
   physics and random numbers for histories [first_history, first_history +
   n_histories) and ADDS the integer tally (units of 2^-32 MeV, nx*ny*nz
   int64, voxel layout as above) to the caller-allocated device array d_tally;
   no batch statistics are kept.
   Memory: its scratch (particle queues, counters, error word) is a fixed
   device array of DPM_NOALLOC_SCRATCH_BYTES.  The driver places that array in
   a device's memory when it loads the library's module holding it there;
   dpm_create() forces that load (and the load of the queue kernels) on its
   device, so that after dpm_create() this call allocates nothing, and the
   array then stays on the device until the process exits.  The call looks
   the array's device address up each time (cudaGetSymbolAddress, no
   allocation once loaded); it never calls cudaMalloc, cudaFree or an
   allocating library routine.
   Sharing: every call in the process shares the one array, which keeps the
   last call's contents (each call clears the counters it uses): calls that
   overlap on the GPU (e.g. from two contexts or streams at once) race and must
   be serialised by the caller.
   Result: the call waits for the transport and returns its status.  On
   success d_tally holds its previous contents plus this run's tally.  On
   DPM_EQUEUE_OVERFLOW (the fixed queues overflowed), DPM_ETIMEOUT (a bounded
   wait gave up) or DPM_ESTEPCAP (a particle hit the step limit), part of the
   run has already been added to d_tally and the amount is unknown: discard
   d_tally or restore it from a copy.  DPM_ESTATE before dpm_build_tables(),
   DPM_EINVAL for bad arguments or more than 2^31-1 histories (d_tally
   untouched).  stats (host, may be NULL) receives the run's counters
   (emitted, escaped and missed energy, steps, flights, atomics, pushes, error
   flags) with `deposited` set to NaN: the deposited energy is the increase of
   the caller's d_tally times 2^-32 MeV.  With stats given the kernel also
   counts events (dpm_run_opts.count_events), about 10 % slower; the tally is
   the same either way. */
#define DPM_NOALLOC_SCRATCH_BYTES (48u << 20)
int dpm_run_noalloc(dpm_ctx *ctx, int phantom_id, const dpm_source *src, uint64_t first_history,
                    uint64_t n_histories, uint64_t seed, int64_t *d_tally, dpm_run_stats *stats);

#ifdef __cplusplus
}
#endif
#endif
