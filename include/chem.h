/*
 * chem.h - C ABI of the GB300 step-by-step (SBS) radiolysis chemistry library.
 *
 * The library advances radiolytic species (e_aq, OH, H, H3O+, OH-, H2, H2O2, or any
 * table of up to 8 types and 16 reactions) through the non-homogeneous chemical stage
 * of arxiv 2509.03313 Sec. 2.1: Brownian diffusion in a periodic cubic box (Eq. 1),
 * pair search under the minimum-image convention (Eq. 2), diffusion-controlled
 * reactions whose radii follow from the tabulated rate constants (Table 1, Table S2,
 * Eq. kdiff1/kdiff2), and species injected pulse by pulse and carried across the
 * intervals between pulses.
 *
 * Every step of that path runs in the library's own sm_103a kernels; the host only
 * queues work on a CUDA stream and copies results back. There is no CPU fallback: on a
 * machine without a usable GPU every call that needs one returns CHEM_ECUDA.
 *
 * Conventions shared by every entry point:
 *  - Pointer arguments are HOST pointers owned by the caller unless stated otherwise;
 *    the library copies what it needs before returning and keeps no reference.
 *  - A context owns all the device memory it allocates (through the caller's allocator
 *    callbacks when given, cudaMalloc otherwise) and releases it in chem_destroy.
 *  - No exception crosses the ABI. A non-OK status is sticky: every later call on the
 *    context returns it again, and chem_last_error() explains it. The context can then
 *    only be destroyed (chem_tally and chem_get_* still read the last completed step).
 *  - One context is used by one host thread at a time.
 *
 * Units: lengths nm, times s, diffusion coefficients nm^2/s, rate constants
 * L mol^-1 s^-1, energies eV.
 */
#ifndef CHEM_H
#define CHEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct chem_ctx chem_ctx; /* opaque */

typedef enum chem_status {
  CHEM_OK = 0,
  CHEM_EINVAL = 1,    /* bad argument or configuration                              */
  CHEM_ENOMEM = 2,    /* device or host allocation failed                           */
  CHEM_ECAPACITY = 3, /* a capacity given in chem_config was exceeded on the device  */
  CHEM_ECUDA = 4,     /* a CUDA runtime call failed (message in chem_last_error)     */
  CHEM_ETIMEOUT = 5,  /* a bounded device-side wait ran out (sort look-back, grid
                         barrier); the kernels returned instead of waiting further   */
  CHEM_ESTATE = 6     /* call not valid in the context's current state               */
} chem_status;

enum { CHEM_FP64 = 0, CHEM_FP32_LOCAL = 1 };
enum { CHEM_LAUNCH_AUTO = 0, CHEM_LAUNCH_PHASES = 1, CHEM_LAUNCH_PERSISTENT = 2 };
enum { CHEM_MAX_TYPES = 8, CHEM_MAX_RXN = 16, CHEM_MAX_PRODUCTS = 3 };

/* One diffusion-controlled reaction A + B -> products (Table 1). */
typedef struct chem_reaction {
  int32_t a, b;       /* reactant species types; a == b is a self reaction            */
  double k_tab;       /* rate constant as tabulated (L mol^-1 s^-1). For a self
                         reaction this is the printed "2k" value: the library uses it
                         directly in R = k_tab / (4 pi D_AB N_A), Eq. kdiff2.          */
  int32_t n_prod;     /* 0..3                                                          */
  int32_t prod[3];    /* product species types; all placed at the encounter point     */
  int32_t water_delta;/* water molecules created (+) or consumed (-) per event        */
} chem_reaction;

/* Device allocator callbacks (optional). alloc returns device memory of at least
 * `bytes` bytes aligned to 256 B, or NULL; free releases it. `user` is passed back. */
typedef void* (*chem_alloc_fn)(size_t bytes, void* user);
typedef void (*chem_free_fn)(void* ptr, size_t bytes, void* user);

/* Configuration of one pulse train. */
typedef struct chem_config {
  int32_t n_types;             /* 1..8 species types                                   */
  const double* D_nm2_s;       /* [n_types] diffusion coefficients (Table S2)          */
  int32_t n_rxn;               /* 0..16 reactions; at most one per unordered type pair */
  const chem_reaction* rxn;    /* [n_rxn]                                              */
  double L_nm;                 /* side of the periodic box [-L/2, L/2)^3 (Eq. 1)       */
  uint64_t seed;               /* Philox4x32-10 key = (seed lo, seed hi ^ train_id)    */
  uint32_t train_id;
  int32_t precision;           /* CHEM_FP64: positions, distances and random normals in
                                  FP64, reproducing the FP64 reference step for step.
                                  CHEM_FP32_LOCAL: positions held as FP32 offsets from
                                  their hash cell's origin, FP32 normals and distances;
                                  clock, schedule, reaction probabilities and tallies
                                  stay FP64.                                           */
  double dt_min_s;             /* first step and the step after every release         */
  double dt_max_s;             /* largest step                                         */
  double dt_growth;            /* per-step growth factor (1 = fixed step)              */
  int32_t dt_reset_on_release; /* nonzero: restart at dt_min when species are released */
  double cutoff_c;             /* pair cutoff R + c sqrt(2 D_AB dt); typically 3       */
  double sbs_horizon_s;        /* >0: after this long without a release, jump by free
                                  diffusion (no reactions) to the next arrival or end  */
  int64_t capacity_species;    /* max species alive at once (incl. one step's products)*/
  int64_t capacity_pending;    /* max species queued by inject and not yet released    */
  int64_t capacity_candidates; /* max accepted reactive pairs in one step              */
  int64_t capacity_event_log;  /* >0: keep up to this many events for chem_get_events  */
  int64_t capacity_step_log;   /* >0: keep up to this many per-step records            */
  int32_t cells_per_axis_max;  /* spatial-hash resolution limit; 0 = automatic         */
  int32_t steps_per_launch;    /* steps per captured graph replay; 0 = automatic       */
  int32_t launch_mode;         /* CHEM_LAUNCH_AUTO: persistent for batches, one kernel
                                  per phase otherwise; CHEM_LAUNCH_PHASES;
                                  CHEM_LAUNCH_PERSISTENT (cooperative, grid barriers)  */
  void* cuda_stream;           /* cudaStream_t to run on; NULL = library-owned stream  */
  chem_alloc_fn dev_alloc;     /* NULL = cudaMalloc / cudaFree                         */
  chem_free_fn dev_free;
  void* alloc_user;
} chem_config;

/* One reaction event (recorded when capacity_event_log > 0). */
typedef struct chem_event {
  uint32_t step;     /* step index of the train                                      */
  int32_t rxn;       /* reaction index into chem_config.rxn                          */
  uint32_t id_lo;    /* reactant ids, id_lo < id_hi                                   */
  uint32_t id_hi;
  uint32_t prod_id0; /* id of the first product; the others follow consecutively     */
  int32_t n_prod;
  uint32_t train;    /* train index within the context                               */
  uint32_t reserved;
} chem_event;

/* Per-step record (recorded when capacity_step_log > 0). */
typedef struct chem_step_record {
  uint32_t step, train;
  double t_start_s, dt_s;
  int64_t n_live;     /* species that took this step (after the release)             */
  int64_t n_events;   /* reactions committed in this step                            */
  int64_t counts[8];  /* species per type after the step                              */
} chem_step_record;

/* ---- single pulse train ------------------------------------------------------------ */

/* Validate cfg (EINVAL), compute every reaction radius R = k_tab / (4 pi D_AB N_A)
 * (Eq. kdiff1; D_AB = D_a + D_b), check 2 R_cut <= 2L/3 at dt_min, and allocate all
 * device buffers for the capacities given. On success *out is a new context at t = 0
 * with no species. */
chem_status chem_init(const chem_config* cfg, chem_ctx** out);

/* Queue n species for release (Sec. 2.1: the products of each radiation event enter
 * the SBS at their sampled arrival time). type[n] in [0, n_types), xyz[3n] absolute
 * positions in [-L/2, L/2)^3 (host, row-major x,y,z), t_arrival[n] >= the current
 * time (host, s). A species is released at the first step boundary at or after its
 * arrival; ids are assigned at release in (arrival, call order, index) order.
 * energy_eV is added to the deposited energy used for G-values at call time.
 * Blocks until the copy to the device has completed. */
chem_status chem_inject_pulse(chem_ctx* ctx, int64_t n, const int32_t* type, const double* xyz,
                              const double* t_arrival, double energy_eV);

/* Advance to t_end_s (the last step is trimmed to land on it). Each step: release
 * arrived species, diffuse with periodic wrap (Eq. 1), rebuild the spatial hash, find
 * reactive pairs within the cutoff under the minimum image (Eq. 2) and accept them with
 * the probability that their relative path touched the reaction sphere during the step
 * given both separations (the absorbing-sphere kinetics of Eq. kdiff1 in expectation at
 * any dt), keep one reaction per species (closest pair first,
 * lower ids break ties), write products and tallies, advance the FP64 clock.
 * Blocks until the device has finished. */
chem_status chem_run_until(chem_ctx* ctx, double t_end_s);

/* Tallies of train 0 after the last completed step (or homogeneous stage). Any output
 * pointer may be NULL. counts[n_types]: live species, including survivors of a
 * homogeneous stage not yet re-created; G_per_100eV[n_types]: the G-values of Sec. 1
 * (species per 100 eV of deposited energy), counts * 100 / E_dep with E_dep in eV the
 * sum of the energies passed to chem_inject_pulse (multiply by 1.0364e-7 for mol/J);
 * events[n_rxn]: reactions so far, the whole events of homogeneous stages included;
 * t_now: clock; species_steps: sum over steps of the species that took the step. */
chem_status chem_tally(chem_ctx* ctx, int64_t* counts, double* G_per_100eV, int64_t* events,
                       double* t_now, int64_t* species_steps);

/* Live species of train 0 in device order: type[cap], id[cap], xyz[3*cap] (FP64
 * absolute positions). *n receives the live count; EINVAL if it exceeds cap. */
chem_status chem_get_state(chem_ctx* ctx, int64_t cap, int32_t* type, uint32_t* id, double* xyz,
                           int64_t* n);

/* Recorded events of the step-by-step stage (all trains, in step order, within a step in
 * (train, id_lo) order) and per-step records; homogeneous stages add to the event tallies
 * but not to these logs. *n receives the number copied; ECAPACITY (sticky) if the log
 * overflowed on the device. */
chem_status chem_get_events(chem_ctx* ctx, int64_t cap, chem_event* ev, int64_t* n);
chem_status chem_get_step_log(chem_ctx* ctx, int64_t cap, chem_step_record* rec, int64_t* n);

/* Return every train to t = 0 with no species, empty logs and zero tallies, keeping
 * the allocations and captured graphs; seed replaces the seeds of all trains (train b
 * gets seed + b for b > 0 unless chem_batch_reset is used). */
chem_status chem_reset(chem_ctx* ctx, uint64_t seed);

/* Human-readable description of the last error on ctx (never NULL). */
const char* chem_last_error(const chem_ctx* ctx);

/* Release everything ctx owns. NULL is ignored. */
void chem_destroy(chem_ctx* ctx);

/* ---- many independent pulse trains advanced together ------------------------------ */

/* Like chem_init for n_trains trains. All trains share n_types, D, the reaction table
 * and precision; each has its own box, seed, train_id, time-step policy, capacities
 * and clock. Species of all trains live in one hash sorted by (train, cell); every
 * step of every train runs in the same persistent launches. */
chem_status chem_batch_init(const chem_config* cfgs, int32_t n_trains, chem_ctx** out);
chem_status chem_batch_inject(chem_ctx* ctx, int32_t train, int64_t n, const int32_t* type,
                              const double* xyz, const double* t_arrival, double energy_eV);
/* t_end_s[n_trains]: each train advances to its own end time. */
chem_status chem_batch_run_until(chem_ctx* ctx, const double* t_end_s);
chem_status chem_batch_tally(chem_ctx* ctx, int32_t train, int64_t* counts, double* G_per_100eV,
                             int64_t* events, double* t_now, int64_t* species_steps);
chem_status chem_batch_get_state(chem_ctx* ctx, int32_t train, int64_t cap, int32_t* type,
                                 uint32_t* id, double* xyz, int64_t* n);
/* seeds[n_trains] */
chem_status chem_batch_reset(chem_ctx* ctx, const uint64_t* seeds);
int32_t chem_batch_size(const chem_ctx* ctx);

/* ---- homogeneous (beam-off) stage ------------------------------------------------
 * Sec. 2.3 (and the workflow of Sec. 2.1): during the beam-off time between pulses, and
 * for 10 s after the last pulse, the paper follows the species as a well-mixed system
 * with the rate equations of Table 1 (Eq. 3, Eq. 4) instead of step by step. For every train whose clock is below
 * t_end_s[b] (trains at or past it are left alone):
 *  - its species counts, plus pending species already due (arrival <= clock), become
 *    molecule numbers in the box volume L^3; its particles are removed;
 *  - the rate equations are integrated for the reaction extents e_r (events): de_r/dt =
 *    kappa_r n_a n_b, kappa_r = k_tab / (N_A V), (k_tab / 2) / (N_A V) for a self
 *    reaction, n = n0 + nu e; stiff-stable extrapolated linearly implicit Euler on the
 *    device (per step 1e-12 relative + 1e-8 events);
 *  - the extents are rounded to whole events without bias (floor(e_r) plus one with
 *    probability frac(e_r), uniform from Philox4x32-10 at counter (stage, r, 0, 4));
 *    while a count would be negative, the lowest-index reaction consuming the lowest
 *    negative species gives back one event; counts, event tallies and the water balance
 *    take the whole events, so charge and atoms stay exactly conserved;
 *  - the clock moves to t_end_s[b]. chem_tally reports the survivors at once; they are
 *    re-created as particles when the train takes its next step: ids from the next id
 *    in ascending type order, ahead of the species released in that step, uniform
 *    positions -L/2 + L u from counters (id, 0, 0, 3) (x from words 0-1, y from words
 *    2-3) and (id, 1, 0, 3) (z), then released like injected species (the step time
 *    resets to dt_min when dt_reset_on_release is set). chem_get_state lists them only
 *    from that step on.
 * A pending species arriving strictly between the clock and t_end_s[b] is an error:
 * CHEM_EINVAL, nothing changed. CHEM_ECAPACITY (sticky) if the integrator exceeds its
 * step limit. Blocks until the device has finished. */
chem_status chem_run_homogeneous(chem_ctx* ctx, double t_end_s);
chem_status chem_batch_run_homogeneous(chem_ctx* ctx, const double* t_end_s);
/* The last homogeneous stage of a train: extents[n_rxn] real extents (events) before
 * rounding, events[n_rxn] the whole events applied, *integrator_steps the accepted
 * steps. Any output pointer may be NULL. */
chem_status chem_batch_homogeneous_report(chem_ctx* ctx, int32_t train, double* extents, int64_t* events,
                                          int64_t* integrator_steps);

/* Choose, by timing short runs from the current state, the launch form (one kernel per
 * phase in a graph, or the persistent cooperative kernel), the steps per graph replay
 * and the hash resolution limit (cells per axis at small cutoffs, i.e. the cell size).
 * The pair-search mapping is kept (set it with chem_set_tuning): 0 = one thread per
 * home species; 1..32 = cell tiles, the number of home species one warp takes per work
 * item of a cell; -1 = chosen per step (cell tiles when the last step found more than 3
 * pairs inside the cutoffs per live species; the default). The device state is saved
 * before and restored after every trial; trials run past the end time. FP64 results do not depend on the choice; FP32-local results
 * depend on the hash resolution only through rounding. budget_ms bounds the time spent
 * (at least one trial runs). chosen[4] = {steps_per_launch, cells_per_axis_limit,
 * species_per_item, launch_mode} when chosen is not NULL. */
chem_status chem_autotune(chem_ctx* ctx, double budget_ms, int32_t* chosen);

/* Apply tuning parameters directly, in the layout chem_autotune reports: tuning[4] =
 * {steps_per_launch (1..1024), cells_per_axis_limit (>= 3; clamped to the allocated hash),
 * species_per_item (-1..32: -1 per step, 0 one thread per home species), launch_mode
 * (CHEM_LAUNCH_PHASES or CHEM_LAUNCH_PERSISTENT)}.
 * Allowed between runs; the device state is kept. Results depend on the parameters as
 * described for chem_autotune. Out-of-range values: CHEM_EINVAL, nothing changed. No
 * counterpart in the paper (a performance setting). */
chem_status chem_set_tuning(chem_ctx* ctx, const int32_t* tuning);

/* Counters of a context since chem_init (host side, exact). Phase indices:
 * 0 step begin, 1 release (runs inside the diffusion kernel, so 0), 2 release +
 * diffusion + hash keys, 3 radix sort (all passes),
 * 4 gather + cell ranges, 5 pair search, 6 matching + products + tallies,
 * 7 persistent step kernel (batched contexts). phase_ms and phase_launches are only
 * accumulated while profiling is on (chem_set_profiling), from CUDA events recorded
 * inside the captured graph around each kernel, over the steps that advanced a train. */
typedef struct chem_stats {
  int64_t graph_replays;    /* graph launches                                         */
  int64_t kernel_launches;  /* library kernels launched (graph nodes counted per replay)*/
  int64_t steps_launched;   /* SBS steps launched, including no-op steps past the end  */
  int64_t bytes_h2d;        /* bytes copied host -> device                             */
  int64_t bytes_d2h;        /* bytes copied device -> host                             */
  double phase_ms[8];       /* summed device time per phase                            */
  int64_t phase_launches[8];/* kernel launches per phase behind phase_ms               */
  /* Which branches reaction resolution took (device counters, summed over resets). The
   * conflict rounds run in shared memory for up to 1,536 conflicting accepted pairs and
   * in global memory beyond (always in the persistent kernel); the events of a step are
   * ordered in shared memory for up to 8,192 events (bucket sort, or a block radix sort
   * when the keys cluster) and in global memory beyond. The results do not depend on the
   * branch; these counters let tests show that each branch ran. */
  int64_t react_rounds_global;  /* steps whose conflict rounds ran in global memory     */
  int64_t react_order_global;   /* steps whose event order ran in global memory         */
  int64_t react_order_radix;    /* steps whose shared-memory event order used the radix
                                   sort because a bucket held more than 64 keys          */
  int64_t max_conflict_pairs;   /* most conflicting accepted pairs in one step          */
  int64_t max_step_events;      /* most events in one step                              */
  /* Pair-search work (device counters, summed over resets): pairs of reacting types in
   * the cells the search visits for each species (the box-gap test against the largest
   * cutoff of the species' type; the same set for both search mappings), those inside
   * their cutoff (each costs one acceptance test: a Philox block and the touch
   * probability), and the accepted ones. */
  int64_t pairs_tested;
  int64_t pairs_in_cutoff;
  int64_t pairs_accepted;
  int64_t steps_advanced;       /* SBS steps in which at least one train advanced       */
  int64_t steps_cell_tiles;     /* of them, steps whose pair search ran the cell tiles  */
} chem_stats;
chem_status chem_get_stats(const chem_ctx* ctx, chem_stats* out);
/* on != 0: re-capture the step graph with CUDA events around every phase kernel (adds
 * one event-record node per kernel boundary). on == 0 removes them. Resets phase_ms. */
chem_status chem_set_profiling(chem_ctx* ctx, int32_t on);

/* ---- allocation-free single step ---------------------------------------------------
 * The paper has no counterpart to this entry point. It serves callers that cannot let a
 * library allocate device memory: code running under another framework's memory pool
 * that owns the whole device, real-time loops that must never allocate, and hosts whose
 * allocator must not be re-entered from inside a library call. It advances ONE FP64 SBS
 * step (diffusion, hash and radix sort, pair search, matching, products) of one small
 * train whose species the caller keeps in its own device buffers, exactly as a context
 * created by chem_init with dt_min = dt_max = dt_s would take that step.
 *
 * Memory: it calls no cudaMalloc, cudaFree or allocator callback. All working memory is
 * one file-scope __device__ array of about 4.2 MB sized for CHEM_NOALLOC_MAX_SPECIES
 * species; every GPU that loads this library holds that array until the process exits.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before any
 * stream capture. Every call on a device shares the array and finds the previous call's
 * contents there (the call clears what must start empty), so calls that overlap on the
 * GPU race: issue one at a time per device.
 *
 * Arguments: cfg gives the chemistry, box, seed/train_id, cutoff_c and the stream
 * (cfg->cuda_stream, NULL = legacy default stream); precision must be CHEM_FP64 and the
 * capacity, allocator and dt-policy fields are ignored. step, t_s, dt_s: the step index
 * (Philox counter), its start time and length (dt_s must not exceed the L/3 cutoff cap);
 * next_id: first id for products. Inputs (DEVICE): id[n], type[n], xyz[3n]. Outputs
 * (DEVICE): id_out/type_out/xyz_out with room for CHEM_NOALLOC_MAX_SPECIES species,
 * *n_out species after the step, *next_id_out, events_out[CHEM_NOALLOC_MAX_SPECIES/2]
 * and *n_events_out. Blocks until the step has finished on the stream.
 * Returns CHEM_ECAPACITY when n exceeds CHEM_NOALLOC_MAX_SPECIES or the step would need
 * more room than the fixed array has (candidates, products), CHEM_EINVAL for bad
 * arguments, CHEM_ECUDA when a CUDA call fails. The device inputs are checked on the
 * device: a type outside [0, n_types), an id >= 2^29 - 1, or a position that is not
 * finite and inside [-L/2, L/2)^3 gives CHEM_EINVAL with *n_out = *n_events_out = 0,
 * *next_id_out = next_id and no species or event written. */
enum { CHEM_NOALLOC_MAX_SPECIES = 16384 };
chem_status chem_step_noalloc(const chem_config* cfg, uint32_t step, double t_s, double dt_s,
                              uint32_t next_id, int32_t n, const uint32_t* id, const int32_t* type,
                              const double* xyz, uint32_t* id_out, int32_t* type_out,
                              double* xyz_out, int32_t* n_out, uint32_t* next_id_out,
                              chem_event* events_out, int32_t* n_events_out);

/* Diagnostic with no counterpart in the paper: one device thread waits for a word that
 * nothing writes, bounded by limit_s seconds (0 < limit_s <= 10), the way every device-side
 * wait of the library is bounded (sort look-back, grid barrier). Returns CHEM_ETIMEOUT,
 * sticky on ctx like any device error, with the CUDA context left usable: the error
 * path a caller sees when a bounded wait runs out, produced without a GPU fault.
 * CHEM_EINVAL (nothing launched) for a limit outside that range. */
chem_status chem_check_bounded_wait(chem_ctx* ctx, double limit_s);

/* Diagnostic with no counterpart in the paper: the pair search's acceptance test alone.
 * For each i, the pair (id_lo[i], id_hi[i]) of reaction rxn[i] with squared start and end
 * separations d0sq[i], d1sq[i] (nm^2) in a step `step` of length dt_s (s) of train 0 is
 * accepted when its uniform u (Philox4x32-10 of train 0's key at counter (id_lo, step,
 * id_hi, 2), 53 bits) is below the touch probability p of chem_run_until. The search
 * decides most pairs on an FP32 estimate of p with a rigorous error band and forms p in
 * FP64 only when u falls inside the band; this call lets a test check, with u placed
 * within a few ulp of p, that the tiered decision always equals the FP64 one.
 * precision: CHEM_FP64 runs the FP64 mode's test on the squared separations as given;
 * CHEM_FP32_LOCAL runs the FP32-local mode's test on their FP32 roundings. Output
 * (host, n bytes): accept[i] bit 0 = the tiered decision, bit 1 = u < p evaluated in
 * FP64 on the same inputs. All array arguments are host arrays of n elements. Returns
 * CHEM_EINVAL for a reaction index out of range, a negative or non-finite input, or
 * n > 2^24; uses a temporary device block (through the allocator callbacks when given). */
chem_status chem_check_acceptance(chem_ctx* ctx, int32_t precision, uint32_t step, double dt_s, int64_t n,
                                  const double* d0sq, const double* d1sq, const int32_t* rxn,
                                  const uint32_t* id_lo, const uint32_t* id_hi, uint8_t* accept);

/* Library version string. */
const char* chem_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CHEM_H */
