/*
 * hande.h -- C ABI of the GPU FCIQMC engine (libhande.so, one NVIDIA GB300, sm_103a).
 *
 * The engine advances the walker population dynamics of full configuration
 * interaction quantum Monte Carlo as described in the HANDE-QMC paper
 * (arXiv:1811.11679):
 *   Sec. 2.1, Eq. (fciqmc)   c_i(t+dt) = c_i(t) - dt sum_j H_ij c_j(t), applied
 *                            stochastically with signed (real-weight) particles,
 *                            shift S as a diagonal energy offset, initiator
 *                            approximation, semi-stochastic propagation;
 *   Sec. 2.4                 one iteration = spawning, death, annihilation;
 *   App. A.1                 projected energy E = E_HF + sum_{i!=0} C_i H_0i / C_0,
 *                            numerator and denominator reported separately;
 *   App. A.2                 deterministic space "high" of size `semi_stoch_size`
 *                            chosen at iteration `semi_stoch_start`;
 *   App. B                   sorted main list + spawned array, annihilation by
 *                            sorting the spawns and merging them into the list.
 * The run parameters mirror the paper's `qmc` / `semi_stoch` input tables
 * (Supplementary tutorial: tau, rng_seed, init_pop, target_population,
 * initiator, real_amplitudes, spawn_cutoff, state_size, spawned_state_size).
 *
 * Conventions
 *   - Determinants are bit strings over spin orbitals p = 2*spatial + spin
 *     (alpha = 0), stored as `key_words` 64-bit words; bit p is in word p/64.
 *     Keys order as unsigned big integers with word key_words-1 most significant.
 *   - Populations are int64 fixed point: one walker = 2^32 (HANDE_ONE_WALKER).
 *   - All pointers in this header are HOST pointers unless stated otherwise;
 *     inputs are copied, the library never keeps a caller pointer.  The
 *     library owns all device memory of a context (allocated through the
 *     optional allocator, else cudaMalloc) and frees it in hande_destroy.
 *   - Every call returns a hande_status; nothing aborts or prints.  Device-side
 *     errors (capacity, overflow, bounded-wait timeout) are latched on the
 *     device and reported by the next synchronising call (hande_estimators,
 *     hande_get_walkers, hande_synchronize); afterwards the context only
 *     accepts hande_destroy / hande_last_error.
 *   - hande_iterate is asynchronous and stream-ordered on the context's stream.
 */
#ifndef HANDE_H
#define HANDE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HANDE_ONE_WALKER ((int64_t)1 << 32)

typedef enum {
  HANDE_OK = 0,
  HANDE_ERR_INVALID = -1,   /* bad argument or system/run parameter */
  HANDE_ERR_NOMEM = -2,     /* device allocation failed */
  HANDE_ERR_CAPACITY = -3,  /* walker, spawn or annihilation-tile capacity exceeded */
  HANDE_ERR_OVERFLOW = -4,  /* a population reached 2^62 in fixed point */
  HANDE_ERR_CUDA = -5,      /* a CUDA runtime call failed */
  HANDE_ERR_TIMEOUT = -6,   /* a bounded device-side wait gave up */
  HANDE_ERR_STATE = -7      /* context unusable after an earlier error */
} hande_status;

typedef enum { HANDE_HUBBARD = 0, HANDE_UEG = 1, HANDE_MOLECULE = 2 } hande_system_kind;

/* The Hamiltonian (the paper's `sys` table).
 *   HUBBARD   real-space Hubbard model, hopping -t between neighbours, on-site
 *             U.  ndim = 0: a 1D chain of `norb` sites (periodic needs norb >= 3).
 *             ndim = d in 1..3: the periodic lattice whose cell is spanned by
 *             the integer vectors lattice[3k .. 3k+d) (the paper's `lattice`
 *             input; e.g. {3, 3}, {3, -3} is the tilted 18-site square
 *             cluster); its sites are the integer points r with fractional
 *             coordinates r A^-1 in [0, 1)^d, in lexicographic order of r
 *             (when every lattice vector has an even coordinate sum the cell is
 *             bipartite: its even- and odd-parity sites then alternate, each
 *             half lexicographic, so that the reference below is the Neel
 *             state), and norb must be |det A|; hops go to r +- e_k (reduced into the cell),
 *             which must reach 2d distinct other sites.  Reference determinant:
 *             alpha on even sites, beta on odd sites.
 *   UEG       3D uniform electron gas in the `norb` plane waves of lowest
 *             |n|^2 (ties by (nx, ny, nz)), box from the Wigner-Seitz radius
 *             rs, Coulomb kernel 4 pi / (Omega |q|^2), q = 0 and Madelung terms
 *             omitted.  Reference: aufbau.
 *   MOLECULE  one- and two-electron integrals h1[norb*norb] (row-major,
 *             symmetric) and eri[norb^4] (chemist order (pq|rs), exactly
 *             8-fold symmetric), core energy ecore.  Reference: aufbau.
 *             Host pointers, copied at init. */
typedef struct {
  int kind;          /* hande_system_kind */
  int key_words;     /* 1, 2 or 8; 2*norb must fit in 64*key_words bits */
  int norb;          /* spatial orbitals (Hubbard: sites) */
  int nalpha, nbeta; /* electrons per spin */
  int periodic;      /* Hubbard only */
  double t, U;       /* Hubbard only */
  double rs;         /* UEG only */
  const double* h1;  /* MOLECULE only */
  const double* eri; /* MOLECULE only */
  double ecore;      /* MOLECULE only */
  int ndim;          /* HUBBARD: 0 = chain of norb sites, else lattice dimension */
  int lattice[9];    /* HUBBARD: row k (lattice[3k .. 3k+ndim)) = lattice vector k */
} hande_system;

/* Run parameters (the paper's `qmc` and `semi_stoch` tables). */
typedef struct {
  double tau;                 /* time step */
  double target_population;   /* walkers at which the shift starts to vary */
  double shift_damping;       /* zeta in S <- S - zeta/(A tau) ln(N_w(t)/N_w(t-A)) */
  double spawn_cutoff;        /* real weights: smaller spawns are rounded stochastically */
  double init_pop;            /* walkers placed on the reference at start */
  double initiator_threshold; /* n_a: a parent is an initiator if |N| > n_a */
  double p_single;            /* MOLECULE: probability of a single excitation */
  int shift_period;           /* A: iterations between shift updates (>= 1) */
  int initiator;              /* 1 = initiator approximation */
  int real_amplitudes;        /* 1 = real weights, 0 = integer walkers */
  int semi_stoch_size;        /* deterministic space size, 0 = off (needs real weights) */
  int semi_stoch_start;       /* iteration at whose end the space is chosen; 0 = at start */
  uint64_t seed;              /* rng_seed: Philox4x64-10 key word 0 */
  uint64_t replica;           /* Philox key word 1 (independent replicas) */
  int64_t state_capacity;     /* max determinants in the main list (0 = default) */
  int64_t spawn_capacity;     /* max spawns per iteration (0 = default) */
  int record_capacity;        /* estimator records kept on the device (0 = default) */
  int tile_capacity;          /* distinct new spawned keys one annihilation tile holds on
                                 chip: 0 = default (128 per warp on the warp path, 64 for
                                 512-bit keys; 512 for
                                 64/128-bit and 256 for 512-bit keys on the block path),
                                 else a power of two in [64, default]; smaller values only
                                 send more buckets through the slower paths */
  int annihilation;           /* annihilation kernel: 0 = default (one warp per
                                 bucket), 1 = block tiles, 2 = one warp per bucket (large
                                 or overflowing buckets go to block tiles on that path);
                                 every choice gives the same walker list */
  int excit_gen;              /* excitation generator (the paper's `excit_gen`): 0 = the
                                 system's own (HUBBARD and UEG uniform, MOLECULE heat-bath);
                                 1 = UEG proposal table (the learned proposal's table, see
                                 hande_set_proposal / hande_learn_proposal), which starts
                                 with weight 1 on every drawable particle orbital */
  int tau_search;             /* the paper's `tau_search`: 1 = until the population first
                                 exceeds target_population, after each iteration
                                 tau <- min(tau, 1 / R), R the largest |H_ij| / p_gen =
                                 (|H_ij| inv_a) inv_b of any spawning attempt so far, so
                                 that no attempt spawns more than one walker; tau is
                                 fixed afterwards.  Synchronises once per iteration while
                                 searching */
} hande_qmc;

/* Optional device allocator (e.g. a framework's caching allocator).  `alloc`
 * returns a device pointer aligned to 256 bytes or NULL; `free` releases it. */
typedef struct {
  void* (*alloc)(size_t bytes, void* user);
  void (*free)(void* ptr, size_t bytes, void* user);
  void* user;
} hande_allocator;

/* One iteration's estimators (App. A.1), evaluated on the list at the start
 * of the iteration, plus population and throughput counters.  The projected
 * energy itself is the caller's ratio: over the iterations of an averaging
 * window, E_proj = E_ref + <num> / <n0> (numerator and denominator averaged
 * separately, App. A.1; both carry the same 2^32 population scale, so it
 * cancels, and num carries an extra 2^16 in num_hi/num_lo only), with E_ref
 * from hande_reference.  The library reports no ratio because a per-iteration
 * ratio of two noisy sums is biased and has no finite variance when n0 can
 * approach zero. */
typedef struct {
  int64_t iter;        /* iteration number t >= 1 */
  double shift;        /* S after the update at the end of iteration t */
  int64_t nw_pre;      /* sum |N_i| at the start of t (fixed point) */
  int64_t n0;          /* N on the reference determinant (fixed point) */
  int64_t num_hi;      /* numerator sum_{j!=0} N_j H_0j * 2^16, exact 128-bit (hi word) */
  uint64_t num_lo;     /*   ... (lo word) */
  double num;          /* the same numerator as a double, in fixed-point population units */
  int64_t nw_post;     /* sum |N_i| after annihilation */
  int64_t ndet;        /* occupied determinants after annihilation */
  int64_t natt;        /* spawning attempts */
  int64_t nspawn;      /* nonzero spawns */
  double tau;          /* the time step iteration t used */
} hande_estimate;

typedef struct hande_ctx hande_ctx;

/* Build the system tables, the reference determinant with `init_pop` walkers
 * and the device buffers on `cuda_stream` (a cudaStream_t; NULL = legacy
 * default stream).  `allocator` may be NULL.  On success *out owns the context. */
hande_status hande_init_system(const hande_system* sys, const hande_qmc* qmc, const hande_allocator* allocator,
                               void* cuda_stream, hande_ctx** out);

/* Advance n >= 0 iterations (asynchronous; one CUDA-graph launch per iteration).
 * Errors of an iteration surface at the next synchronising call.  Annihilation
 * buckets are sized from the previous iteration's spawn and new-key counts; a
 * bucket that still receives more spawns than one warp takes is split into at
 * most 256 key sub-ranges of about a quarter tile each (splitters sampled from
 * its spawns), so one list entry whose spawns in a single iteration exceed
 * about 256 x tile_capacity / 4 mostly distinct new keys (16 384 at the 512-bit
 * default tile, 32 768 otherwise) can end the run with HANDE_ERR_CAPACITY
 * (annihilation tile); start such runs from a smaller init_pop. */
hande_status hande_iterate(hande_ctx* ctx, int n);

/* Number of phases reported by hande_iterate_timed, in order: determinant pass
 * (estimators, initiator flags, attempt counts, death), attempt-count scan,
 * bucket splitters, deterministic-space projection, spawning attempts,
 * bucket-count scan, bucket scatter, merge (annihilation), diagonal elements
 * of new determinants, shift/record. */
#define HANDE_NPHASES 10

/* Advance n iterations like hande_iterate, but launched kernel by kernel
 * (no graph) with CUDA events between the phases; phase_ms[0..HANDE_NPHASES)
 * receives the device time of each phase summed over the n iterations.
 * Synchronises after every iteration.  For profiling only. */
hande_status hande_iterate_timed(hande_ctx* ctx, int n, float* phase_ms, int nphases);

/* Wait for the stream and report latched device errors. */
hande_status hande_synchronize(hande_ctx* ctx);

/* Copy the records not yet fetched (oldest first, at most `max`) to `out`;
 * *n_out = records written.  Synchronises.  HANDE_ERR_CAPACITY if records
 * were overwritten before being fetched (record_capacity too small). */
hande_status hande_estimators(hande_ctx* ctx, hande_estimate* out, int max, int* n_out);

/* Copy the current walker list, sorted by key: keys[n*key_words] (word 0
 * first per walker), pops[n], hdiag[n] (H_ii - E_ref, may be NULL), flags[n]
 * (bit0 = in the deterministic space, may be NULL).  HANDE_ERR_CAPACITY with
 * *n set if cap is too small.  Synchronises. */
hande_status hande_get_walkers(hande_ctx* ctx, uint64_t* keys, int64_t* pops, double* hdiag, uint8_t* flags,
                               int64_t cap, int64_t* n);

/* Replace the walker list with n entries (keys strictly ascending, each with
 * nalpha + nbeta electrons, the reference determinant present).  hdiag may be
 * NULL, in which case H_ii - E_ref is evaluated on the device.  Before the
 * first iteration with semi_stoch_start == 0 the deterministic space is chosen
 * from this list; an active deterministic space is kept (its matrix is not
 * rebuilt) and must lie in the new list (else HANDE_ERR_INVALID and the space
 * is off; hande_set_state installs a different one).  The iteration counter is
 * kept.  In a context that has not iterated yet, the first iteration sizes
 * its annihilation buckets as if every one of the list's attempts (sum of
 * ceil |N_i|) spawned a new determinant; later lists keep the sizing from the
 * previous iteration's counts.  Synchronises. */
hande_status hande_set_walkers(hande_ctx* ctx, const uint64_t* keys, const int64_t* pops, const double* hdiag,
                               int64_t n);

/* Launch and bucket geometry chosen by hande_autotune. */
typedef struct {
  int bucket_spawns;      /* expected spawns per annihilation bucket */
  int bucket_new;         /* expected distinct new determinants per bucket (warp path) */
  int attempt_blocks;     /* blocks of the spawning kernel */
  double ms_per_iteration;
} hande_tuning;

/* Autotune the annihilation bucket size (expected spawns and new determinants
 * per bucket, 0.5 to 1.25 times the defaults) and the spawning kernel's grid
 * (one or two blocks per SM): time `iterations` iterations of each candidate
 * and keep the fastest.  The iterations are real (the run advances by
 * 16 x (iterations + 1)); the walker lists do not depend on the choice.  *out
 * (may be NULL) receives it.  Synchronises. */
hande_status hande_autotune(hande_ctx* ctx, int iterations, hande_tuning* out);

/* Diagnostics of the last iteration (synchronises; usable after an error). */
typedef struct {
  uint32_t error_bits;        /* device error latch: 1 spawn capacity, 2 walker capacity,
                                 4 population overflow, 8 wait timeout, 16 tile capacity,
                                 32 bucket capacity */
  int64_t ndet;               /* current list length */
  int64_t natt, nspawn;       /* attempts and spawns of the last iteration */
  int64_t nbuckets;           /* annihilation buckets of the last iteration */
  int64_t bucket_main;        /* main-list entries per bucket */
  int64_t max_bucket_spawns;  /* largest number of spawns that fell in one bucket */
  int64_t tile_capacity;      /* distinct spawned keys one bucket can hold on chip */
  int64_t ncore;              /* deterministic-space size */
  int64_t launches_per_iteration; /* kernels one iteration launches (current settings) */
  int64_t deferred_buckets;   /* buckets the warp annihilation left to block tiles */
} hande_diag;
hande_status hande_diagnostics(hande_ctx* ctx, hande_diag* out);

/* No-allocation projected-energy sums.  The paper has no counterpart: this
 * entry point exists for callers that may not allocate device memory when they
 * need the estimator -- applications that reserve their whole device-memory
 * budget up front and give plug-in code none of it, code whose memory pool
 * owns every free byte of the device, and latency-critical loops that must not
 * call cudaMalloc/cudaFree because those calls can synchronise the device.
 * It computes, for the walker list given in caller-owned DEVICE arrays,
 *   d_out[0] = sum |N_i|, d_out[1] = N on the reference determinant,
 *   d_out[2], d_out[3] = lo, hi words of the exact 128-bit numerator
 *                         sum_{j != ref} N_j H_0j * 2^16 (as in hande_estimate),
 * with d_keys[n*key_words] (row-major, word 0 first per walker, any order) and
 * d_pops[n] (fixed point), asynchronously on the context's stream; the arrays
 * must live on the device the context was created on (made current for the
 * call, the caller's current device restored afterwards).  n = 0 writes zeros.
 * It calls no allocation routine: its per-block partial sums use one fixed
 * device array of 4096 slots (128 KiB, held by every device that loads the
 * library until the process exits), so n may be at most 16,777,216
 * (4096 x 4096); larger n returns HANDE_ERR_CAPACITY.  Every call shares that
 * array and overwrites the slots it uses, so calls in flight at the same time
 * (on different streams) race.  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture. */
hande_status hande_estimate_noalloc(hande_ctx* ctx, const uint64_t* d_keys, const int64_t* d_pops, int64_t n,
                                    int64_t* d_out);

/* Run state beyond the walker list, for restarting a calculation (Sec. 3.1:
 * restart files carry everything -- the random-number state included -- that
 * a restarted calculation needs to follow the same Markov chain as one that
 * ran uninterrupted).  The random numbers here are counter-based (Philox keyed
 * by seed and replica, counter = iteration, attempt, determinant), so their
 * whole state is the iteration number. */
typedef struct {
  int64_t iter;       /* completed iterations t */
  double shift;       /* S after iteration t */
  int64_t nw_ref;     /* sum |N| at the last shift update (or when the target was
                         first exceeded), fixed point; 0 before that */
  int vary;           /* 1 once the population exceeded target_population */
  int core_active;    /* 1 once the deterministic space was chosen */
  int64_t ncore;      /* its size (0 when not active) */
  double tau;         /* the time step of the next iteration */
  double rmax;        /* time-step search: largest |H_ij| / p_gen seen (0 = none) */
} hande_state;

/* Copy the run state to *out and, if core_keys is not NULL and the
 * deterministic space is active, its keys to core_keys[ncore*key_words]
 * (ascending, word 0 first per key); HANDE_ERR_CAPACITY if ncore > core_cap.
 * Synchronises.  Together with hande_get_walkers this is a restart snapshot. */
hande_status hande_get_state(hande_ctx* ctx, hande_state* out, uint64_t* core_keys, int64_t core_cap);

/* Restore a snapshot into a context made with the same system and run
 * parameters: call hande_set_walkers(list) first, then this.  It sets the
 * iteration counter, the shift, its latch and reference population, and (with
 * core_active) installs the given deterministic space (every key must be in
 * the list, the reference among them, at most semi_stoch_size keys) in place
 * of any space set_walkers chose; without core_active the context has no
 * deterministic space until semi_stoch_start (if still ahead).  Records start
 * after the restored iteration.  The continued run equals the uninterrupted one
 * bit for bit.  HANDE_ERR_INVALID (context unchanged except its deterministic
 * space, which is then off) on inconsistent input.  Synchronises. */
hande_status hande_set_state(hande_ctx* ctx, const hande_state* state, const uint64_t* core_keys);

/* E_ref = H_00 of the reference determinant, and its key (key_words words). */
hande_status hande_reference(hande_ctx* ctx, double* e_ref, uint64_t* key);

/* Completed iterations. */
int64_t hande_iterations(const hande_ctx* ctx);

/* Free all device memory and the context (safe on NULL). */
void hande_destroy(hande_ctx* ctx);

/* Last error message of the context ("" if none); static text for NULL. */
const char* hande_last_error(const hande_ctx* ctx);

/* ---------------------------------------------------------------- batches
 * Independent replicas advanced together.  The paper has no batched form: a
 * calculation is one run whose error bar comes from reblocking its own
 * autocorrelated series (Sec. 3.1); only DMQMC averages over independent
 * calculations.  A batch advances many independent runs on one GPU.  Replica r
 * is exactly the run hande_init_system(&sys[r], &qmc[r], ...) would make: its
 * walker lists and estimator records are bit-identical, so distinct seeds (or
 * distinct qmc.replica words) give independent Markov chains.
 *
 * Replicas sharing a key width, system kind and annihilation tile form a group.
 * A batch iteration is one CUDA graph on `cuda_stream` (a cudaStream_t, NULL =
 * legacy default stream): each phase of a group's iteration is one kernel
 * launch over all its replicas, whose blocks a planner kernel divides among
 * the replicas in proportion to their work (list length, last attempt count),
 * every replica reading its own parameter block; groups (at most 8 replicas
 * each unless hande_batch_autotune chose otherwise) run on parallel graph
 * branches.  Each replica also
 * owns a non-blocking stream used by single-replica calls on it (walkers,
 * estimators, hande_iterate of that replica alone), which is ordered with
 * `cuda_stream` at the start and end of every batch call.  While a replica
 * needs per-iteration host work (learned proposal, running time-step search)
 * or has been advanced alone, the batch instead launches one captured graph
 * per replica on the replica streams. */
typedef struct hande_batch hande_batch;

/* Build n >= 1 replicas from the caller-owned arrays sys[n] and qmc[n]
 * (copied).  `allocator` may be NULL and serves every replica.  On failure
 * nothing is left allocated and, if err_replica is not NULL, *err_replica is
 * the index of the replica that failed (-1 for a failure of the batch itself). */
hande_status hande_batch_init(const hande_system* sys, const hande_qmc* qmc, int n, const hande_allocator* allocator,
                              void* cuda_stream, hande_batch** out, int* err_replica);

/* Advance every replica by n_iterations >= 0 iterations (asynchronous, iteration
 * by iteration across the replicas).  On a replica error the remaining launches
 * are skipped, `cuda_stream` still waits for what was launched, and the error of
 * the first failing replica is returned (its context holds the message;
 * hande_batch_failed_replica names it).  Replicas may then differ by one
 * iteration in their iteration counts. */
hande_status hande_batch_iterate(hande_batch* b, int n_iterations);

/* Index of the replica whose error the last hande_batch_iterate or
 * hande_batch_synchronize returned (-1 if none). */
int hande_batch_failed_replica(const hande_batch* b);

/* Autotune the batched launch shape: for each candidate (replicas per group
 * at most 4, 8, 16 or unlimited; block budget = the single run's grid of each
 * phase times 1, 2, 4 or 8), time `iterations` batched iterations and keep
 * the fastest.  The iterations are
 * real (the replicas advance by 16 x (iterations + 1)); the walker
 * lists do not depend on the shape.  *best_scale and *best_ms (ms per batched
 * iteration) receive the choice (either may be NULL).  HANDE_ERR_STATE if a
 * replica needs per-iteration host work.  Synchronises. */
hande_status hande_batch_autotune(hande_batch* b, int iterations, double* best_scale, double* best_ms);

/* Number of replicas (0 for NULL). */
int hande_batch_size(const hande_batch* b);

/* Launch layout in use: *groups (may be NULL) receives the number of launch
 * groups of a batched iteration (0 before the first batched iteration) and
 * *group_cap (may be NULL) the most replicas a group takes (0 = no limit).
 * HANDE_ERR_INVALID for NULL b. */
hande_status hande_batch_layout(const hande_batch* b, int* groups, int* group_cap);

/* Context of replica r, owned by the batch (NULL when r is out of range).  All
 * single-context calls apply to it; hande_iterate on it advances that replica
 * alone, on its own stream. */
hande_ctx* hande_batch_replica(hande_batch* b, int r);

/* Synchronise every replica and report the first latched device error. */
hande_status hande_batch_synchronize(hande_batch* b);

/* Free all replicas, their streams and the batch (safe on NULL). */
void hande_batch_destroy(hande_batch* b);

/* ---------------------------------------------------------------- learned proposal
 * Not in the paper, whose generators are uniform or heat-bath (Sec. 2.1,
 * Sec. 4).  With excit_gen = 1 (UEG only) a double excitation draws its
 * occupied pair (i < j) uniformly and its particle orbital A (the spin of i)
 * from a table row r = (I M + J) 2 + [spin i == spin j] (I, J spatial, M =
 * norb) of integer weights q_r[A]; b follows from momentum conservation and
 *   p_gen = [1 / C(N,2)] (q_r[A] + [same spin] q_r[B]) / sum_A' q_r[A'],
 * exact in the integers, enters the spawn weight tau |H| / p_gen, so the
 * estimators stay unbiased for any table.  A weight must be in [1, 2^24]
 * exactly on the drawable orbitals (B in the basis and, for a same-spin pair,
 * B != A) and 0 elsewhere; drawable orbitals with weight >= 1 keep every
 * nonzero H_ij reachable. */

/* Replace the table with q[2 M^2][M] (host; synchronises).  HANDE_ERR_INVALID
 * for a context without the table generator or a table breaking the rule above. */
hande_status hande_set_proposal(hande_ctx* ctx, const uint32_t* q);
/* Copy the current table to q[2 M^2][M] (host; synchronises). */
hande_status hande_get_proposal(hande_ctx* ctx, uint32_t* q);

/* The learned proposal: an MLP (features x(r) = [one-hot I, one-hot J, same
 * spin], two ReLU hidden layers of `width`, M logits; BF16 weights and
 * activations on the tensor cores, FP32 accumulation) whose masked softmax p
 * gives the table q_r[A] = max(1, floor(p(A | r) 2^24)).  It is trained online
 * on the spawning attempts of the run: the spawning kernel records (row, A,
 * |H| / p_draw) for `batch` attempts spread over each iteration, and every
 * `period` iterations (after hande_iterate's iteration) one Adam step lowers
 *   L = - sum_n c_n log p(A_n | r_n),  c_n = (|H_n| / p_n) / sum_m (|H_m| / p_m),
 * the sampled cross-entropy to the distribution proportional to |H|, and the
 * table is recomputed from the network. */
typedef struct {
  int width;             /* hidden width, a multiple of 64 up to 512 (0 = 256) */
  int batch;             /* training samples per step, a multiple of 128 (0 = 4096) */
  int period;            /* iterations between training steps (0 = no online training) */
  double learning_rate;  /* Adam step size (0 = 1e-3) */
  uint64_t seed;         /* initial weights: uniform in +-sqrt(6 / fan-in), zero biases */
} hande_learning;

/* Attach the learned proposal to a UEG context made with excit_gen = 1 (at
 * most 256 orbitals) and recompute the table from its initial network.
 * Synchronises. */
hande_status hande_learn_proposal(hande_ctx* ctx, const hande_learning* learning);

/* Network parameters as one FP32 vector, in this order: W1 [width][2M+1], b1
 * [width], W2 [width][width], b2 [width], W3 [M][width], b3 [M] (row-major).
 * Copies them to `get` and/or replaces them with `set` (host, n entries each,
 * either may be NULL; setting resets the Adam moments).  n must be the
 * parameter count, which *n_out receives when get and set are NULL.
 * Synchronises. */
hande_status hande_learn_params(hande_ctx* ctx, float* get, const float* set, int64_t n, int64_t* n_out);

/* Loss L and its gradient (grads[n_params], host) for a batch of n <= batch
 * samples: rows[n], drawn orbitals targets[n] (drawable), weights[n] >= 0 (the
 * |H| / p of each sample).  The same BF16 forward and backward kernels the
 * online training runs.  Synchronises. */
hande_status hande_learn_gradients(hande_ctx* ctx, const int32_t* rows, const int32_t* targets, const float* weights,
                                   int n, float* grads, double* loss);

/* Masked softmax probabilities p(A | rows[i]) into probs[n][M] (host), n <= batch. */
hande_status hande_learn_probabilities(hande_ctx* ctx, const int32_t* rows, int n, float* probs);

/* Recompute the table from the current network now (normally done after every
 * training step).  Synchronises. */
hande_status hande_learn_refresh(hande_ctx* ctx);

/* ---------------------------------------------------------------- tensor cores
 * The paper has no learned part: its excitation generators are uniform or
 * heat-bath tables (Sec. 2.1, Sec. 4).  The learned excitation proposal of this
 * library (a small MLP whose output becomes the generator's selection table)
 * runs its dense layers on the tensor cores through this GEMM.
 *
 * D[m][n] = sum_k A[m][k] B[n][k] for DEVICE arrays: A (m x k) and B (n x k)
 * row-major BF16 (raw 16-bit patterns) with leading dimensions lda, ldb >= k
 * that are multiples of 8 and rows starting on 16-byte boundaries; D (m x n)
 * row-major FP32 with leading dimension ldd >= n.  Products of BF16 values are
 * exact and are accumulated in FP32 by tcgen05 MMAs (128 x 128 output tiles).
 * Runs on `cuda_stream` (a cudaStream_t).  With d_status NULL the call
 * synchronises the stream and returns HANDE_ERR_TIMEOUT if a bounded device
 * wait gave up; with a caller-owned DEVICE word d_status it returns at once and
 * the kernel ORs 1 into *d_status on such a failure.  HANDE_ERR_INVALID on bad
 * sizes or alignment, HANDE_ERR_CUDA on a failed CUDA call. */
hande_status hande_gemm_bf16(const uint16_t* d_a, int64_t lda, const uint16_t* d_b, int64_t ldb, float* d_d,
                             int64_t ldd, int m, int n, int k, unsigned* d_status, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* HANDE_H */
