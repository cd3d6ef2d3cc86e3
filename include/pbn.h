/*
 * pbn.h -- C ABI of the GB300 (sm_103a) engine for approximate steady-state
 * analysis of probabilistic Boolean networks (PBNs) by many parallel Markov
 * chains, after Mizera, Pang & Yuan, "Parallel Approximate Steady-state
 * Analysis of Large Probabilistic Boolean Networks".
 *
 * Conventions for every entry point:
 *   - The return value is a pbn_status.  No C++ exception crosses this ABI.
 *     On failure pbn_last_error() returns a thread-local message.
 *   - Pointers documented as "device" must point to CUDA device memory of the
 *     current device; "host" pointers to ordinary host memory.  The caller
 *     owns every buffer it passes in; the library never frees or keeps them.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Device work
 *     is stream-ordered on it.  Entry points that return results in host
 *     memory synchronise the stream before returning; the others do not.
 *   - The library owns pbn_net handles (device copies of the network tables).
 *
 * Chain layout (bit-sliced, 32 chains per 32-bit word):
 *   chain c belongs to group g = c / 32 and lane c % 32.
 *   state[g * n + i]: bit (c % 32) is the value of node i of chain c.
 *   bits[g * bits_cap + j]: bit (c % 32) is the indicator of the state of
 *   interest (meta state 1, Sec. 3.1) of chain c at trajectory position
 *   bits_base + j.  Trajectory position q holds the state after transition q
 *   (state q+1); the initial state is not a sample.
 *   Bits of lanes >= omega in the last group are unspecified.
 *
 * Random numbers (the paper does not fix them): Philox4x32-10 keyed by the
 * 64-bit seed; node i, transition t and chain group g address counters
 * (i, t lo32, (t hi32 & 0xFFFFFF) | b << 24, g), b = 0..7; chain c's uniform
 * u takes bit c % 32 of the 32 output words as its digits, most significant
 * first.  Perturbation iff u < P32 = round(p 2^32); otherwise function j of
 * node i is selected when T_{j-1} <= u < T_j, T the quantised cumulative
 * selection probabilities.  Every trajectory is a pure function of
 * (seed, chain, transition, node), so runs are replayable and resumable.
 */
#ifndef PBN_H
#define PBN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pbn_status {
    PBN_OK = 0,
    PBN_ERR_INVALID = 1,        /* malformed argument or network */
    PBN_ERR_OOM = 2,            /* device or host allocation refused */
    PBN_ERR_CUDA = 3,           /* a CUDA runtime call failed */
    PBN_ERR_TIMEOUT = 4,        /* a bounded device-side wait gave up */
    PBN_ERR_NOT_CONVERGED = 5,  /* a stopping rule was not met within the length cap */
    PBN_ERR_INSUFFICIENT = 6,   /* the window cannot give alpha and beta (no 0->1 or 1->0) */
    PBN_ERR_UNSUPPORTED = 7,    /* valid input beyond the library's limits */
    PBN_ERR_CANCELLED = 8       /* an engine query withdrawn by pbn_engine_cancel */
} pbn_status;

enum { PBN_PERTURB_PER_NODE = 0, PBN_PERTURB_GLOBAL = 1 };

/* Limits of this library. */
#define PBN_MAX_NODES 4096          /* node ids are 12-bit in the device tables */
#define PBN_MAX_PARENTS 15          /* truth tables up to 32768 bits (1024 words) */
#define PBN_MAX_FUNCTIONS_PER_NODE 16
#define PBN_MAX_SOI 32               /* state-of-interest entries of one run, over all its properties */
#define PBN_MAX_PROPERTIES 8         /* properties abstracted from one set of trajectories (Sec. 4.2) */

/*
 * A PBN G(V,F) (Sec. 2.2) with perturbation probability p, in CSR form.  All
 * arrays are host memory and are copied by pbn_load.
 *   fn_offset   [n+1]  functions of node i are fn_offset[i] .. fn_offset[i+1]-1
 *   par_offset  [F+1]  parents of function f are parents[par_offset[f] ..]
 *   parents     [par_offset[F]]  node ids; parent m is bit m of the index
 *   truth_table [F]    f(x) = bit (sum_m x_m 2^m) of truth_table[f]
 *   select_prob [F]    c_j^(i); per node they sum to 1 (within 1e-9)
 */
typedef struct pbn_network_desc {
    int32_t n;
    int32_t n_functions;
    const int32_t *fn_offset;
    const int32_t *par_offset;
    const int32_t *parents;
    const uint32_t *truth_table;   /* one word per function (used when tt_offset is NULL; then k <= 5) */
    const double *select_prob;
    double p;
    /* Truth tables of any size up to PBN_MAX_PARENTS inputs (may be NULL):
     * function f's table is tt_words[tt_offset[f] .. tt_offset[f+1]-1],
     * max(1, 2^k / 32) words; bit j of the table is bit j % 32 of word j / 32. */
    const int32_t *tt_offset;
    const uint32_t *tt_words;
} pbn_network_desc;

typedef struct pbn_net pbn_net;

typedef struct pbn_net_info {
    int32_t n;
    int32_t n_functions;
    uint32_t perturb_threshold;   /* P32 */
    int64_t table_bytes;          /* device bytes of the staged tables */
} pbn_net_info;

/* State of interest: meta state 1 = every listed node holds its value
 * (Sec. 3.1).  Host arrays, 1 <= size <= PBN_MAX_SOI. */
typedef struct pbn_soi {
    int32_t size;
    const int32_t *nodes;
    const uint8_t *values;
} pbn_soi;

/* Caller-owned chain buffers (device memory) and their position bookkeeping. */
typedef struct pbn_chains {
    int64_t omega;          /* number of chains (>= 1) */
    uint32_t *state;        /* device [ceil(omega/32) * n] */
    uint32_t *bits;         /* device [ceil(omega/32) * bits_cap], may be NULL if bits_cap == 0 */
    int64_t bits_cap;       /* positions per group held by `bits` */
    int64_t bits_base;      /* trajectory position of column 0 */
    int64_t length;         /* trajectory length L: `state` holds state L */
} pbn_chains;

typedef struct pbn_run_cfg {
    uint64_t seed;
    int32_t perturb_mode;   /* PBN_PERTURB_PER_NODE or PBN_PERTURB_GLOBAL */
    pbn_soi soi;
    int32_t groups_per_block;   /* 0 = automatic */
    int32_t threads_per_block;  /* 0 = automatic */
    int32_t threads_per_item;   /* threads sharing one (node, chain group) update: 1, 2, 4; 0 = automatic */
    int32_t blocks_per_round;   /* Philox blocks per thread per round when threads_per_item = 1: 1, 2; 0 = auto */
    int32_t staging;            /* function records: 0 = automatic (shared memory if they fit, else read
                                   from global memory through L1), 1 = whole tables in shared memory,
                                   2 = TMA tiles streamed through shared memory, 3 = global */
    int32_t schedule;           /* PBN_SCHEDULE_*: how the steps are laid on the GPU (same chains either way) */
    /* Several properties recorded in one pass (Sec. 4.2, last part): when
     * n_props > 0, props[0 .. n_props-1] replace `soi` (each non-empty; at most
     * PBN_MAX_PROPERTIES, PBN_MAX_SOI entries in total) and chains->bits holds
     * n_props bitstreams one after the other, property m at
     * bits + m * ceil(omega/32) * bits_cap. */
    int32_t n_props;
    const pbn_soi *props;
} pbn_run_cfg;

/* Schedules of pbn_run_chains.  FUSED: one kernel draws each item's category
 * and updates it, step by step.  SELECT_AHEAD: a first kernel draws the
 * categories of a chunk of steps for all chains at once (they do not depend
 * on the state), a second applies them step by step; for few chain groups,
 * where the fused step waits on its Philox rounds with most SMs idle.  A run
 * longer than one chunk draws chunk i+1 on a library-owned side stream while
 * chunk i is applied on the caller's stream; events order the two, so the
 * call stays stream-ordered on the caller's stream (and can be captured in a
 * CUDA graph like any fork and join).  SELECT_AHEAD takes staging 0, 1 or 3
 * and needs device scratch of up to two 32 MiB buffers per stream (kept by
 * the library, grown on demand).  AUTO: select-ahead when the chain groups
 * (ceil(omega / 32)) number at most the SMs, the network has at most 1000
 * nodes or the groups at most half the SMs, and its shared memory fits; else
 * fused.  FUSED with more groups than SMs, not a whole multiple of them, an
 * automatic groups_per_block and at least 64 steps: two launches, the first
 * running the SMs that carry one group more for fewer steps, the second
 * finishing those groups spread over all SMs (same chains). */
enum { PBN_SCHEDULE_AUTO = 0, PBN_SCHEDULE_FUSED = 1, PBN_SCHEDULE_SELECT_AHEAD = 2 };

/* ---------------------------------------------------------------- network */

/* Validate and stage a PBN (Sec. 2.2) on the current device: quantises p and
 * the selection probabilities (see above) and builds the device tables.
 * Errors: PBN_ERR_INVALID (structure, probabilities), PBN_ERR_UNSUPPORTED
 * (n, parents or functions per node beyond the limits), PBN_ERR_OOM. */
int pbn_load(const pbn_network_desc *desc, pbn_net **out);
void pbn_free(pbn_net *net);
int pbn_net_get_info(const pbn_net *net, pbn_net_info *out);

/* ----------------------------------------------------------------- chains */

/* Initial states (state 0): any initial state is allowed (Sec. 2.2); node i of
 * chain c is bit c % 32 of word 0 of Philox(i, 0xFFFFFFFF, 0xFFFFFFFF, g).
 * Sets chains->length = 0.  Errors: PBN_ERR_INVALID, PBN_ERR_CUDA. */
int pbn_init_chains(const pbn_net *net, const pbn_run_cfg *cfg, pbn_chains *chains, void *stream);

/* Extend every chain by `steps` transitions (Sec. 2.2: synchronous update of
 * all nodes, each node perturbed with probability p or updated by a predictor
 * function drawn by its selection probabilities; "Extend all trajectories",
 * Alg. GR / Alg. 3 / Alg. 4).  Writes the indicator bits of positions
 * length .. length+steps-1 that fall at or after bits_base; the caller must
 * have made bits_cap cover them.  chains->length += steps.
 * Errors: PBN_ERR_INVALID (SOI, capacity, launch shape), PBN_ERR_UNSUPPORTED
 * (a requested schedule or staging that does not fit shared memory),
 * PBN_ERR_OOM (select-ahead scratch), PBN_ERR_CUDA. */
int pbn_run_chains(const pbn_net *net, const pbn_run_cfg *cfg, pbn_chains *chains, int64_t steps,
                   void *stream);

/* The balanced split of one FUSED call into two launches (host arithmetic
 * only, no device work; pbn_run_chains applies it with R = the device's SM
 * count and its own launch shape).  Inputs: G chain groups, R SMs, CTAs of at
 * most gpb groups with T threads per item and `threads` threads, an n-node
 * network, k steps.  On *split = 1, launch[20] holds for launch 1 then
 * launch 2, for segment 0 then 1, {CTAs, first group, groups, steps, step
 * offset}; a segment's CTAs split its groups evenly (CTA b of nb takes groups
 * first + b*groups/nb up to first + (b+1)*groups/nb - 1) and advance them
 * `steps` transitions from transition length + offset.  *split = 0: one
 * launch (launch untouched).  pbn_run_chains splits a call into launches of
 * at most 2^30 steps first, so k is at most 2^30 here.  Errors:
 * PBN_ERR_INVALID (NULL pointer, a size below 1, T not 1, 2 or 4, k outside
 * 0 .. 2^30). */
int pbn_balance_phases(int32_t G, int32_t R, int32_t gpb, int32_t T, int32_t threads, int32_t n, int64_t k,
                       int32_t launch[20], int32_t *split);

/* Simulation launches record a failed bounded device-side wait (a TMA tile
 * that did not arrive within 1 s) in a per-device status word instead of
 * waiting forever; the drivers check it after every query.  This call
 * synchronises the device, returns the word in *status (0 or
 * PBN_ERR_TIMEOUT) and clears it.  (Test hook: with the environment
 * variable PBN_TEST_STALL_FIRST_TILE=1 at load time, tiled launches never
 * issue their first tile, so the wait must run out.) */
int pbn_take_device_status(int *status);

/* ------------------------------------------------------------- statistics */

typedef struct pbn_gr_result {
    double rhat;            /* +inf when W = 0 */
    double W, B, sigma2;
    uint64_t S1;            /* sum over chains of ones in the window */
    uint64_t S2_lo, S2_hi;  /* sum of squares, 128-bit */
} pbn_gr_result;

/* Gelman & Rubin (Sec. 4.1, Alg. GR) on the window of positions
 * [start, start+psi) of every chain's indicator: per-chain mean and sample
 * variance (denominator psi-1), B, W, sigma^2 = (1-1/psi) W + B/psi,
 * R-hat = sqrt(sigma^2 / W).  Computed on the device from exact integer sums.
 * out: device pointer, written asynchronously.  Needs omega >= 2, psi >= 2. */
int pbn_gelman_rubin(const pbn_chains *chains, int64_t start, int64_t psi, pbn_gr_result *out,
                     void *stream);

typedef struct pbn_two_state_result {
    int64_t n00, n01, n10, n11;  /* transitions within chains, both ends in the window */
    int64_t ones;                /* ones in the window */
    double alpha, beta;          /* alpha = n01/(n00+n01), beta = n10/(n10+n11) */
    double prob;                 /* ones / (omega * len) */
    int64_t M, N;                /* Alg. 1 line 8 */
    int32_t status;              /* PBN_OK, PBN_ERR_INSUFFICIENT or PBN_ERR_NOT_CONVERGED (alpha = beta = 1) */
    int32_t pad;
} pbn_two_state_result;

/* Two-state Markov chain statistics (Sec. 3.1, Alg. 1 line 8, Alg. 3) of the
 * merged window [start, start+len) of all chains: transition counts, alpha,
 * beta, burn-in M = ceil(log(eps (a+b)/max(a,b)) / log|1-a-b|), sample size
 * N = ceil(a b (2-a-b)/(a+b)^3 (Phi^-1((1+s)/2))^2 / r^2), estimate.  On the
 * device; out is a device pointer written asynchronously. */
int pbn_two_state(const pbn_chains *chains, int64_t start, int64_t len, double eps, double r, double s,
                  pbn_two_state_result *out, void *stream);

typedef struct pbn_skart_result {
    double mean, var, skew, phi, A, H, ci_lo, ci_hi;
    double vn_stat;          /* von Neumann statistic of the spaced batch means */
    int32_t vn_pass;         /* randomness test passed */
    int32_t pad;
    int64_t batches;         /* omega * batches_per_chain */
} pbn_skart_result;

/* Skart batch statistics (Sec. 3.2, Alg. 2; parallel layout Fig. 2b, Alg. 4):
 * every chain contributes batches_per_chain consecutive batches of kappa
 * positions from `start`; computes the von Neumann randomness test on the
 * spaced batch means (spacer `spacer`, size alpha_ran) and the skewness- and
 * autoregression-adjusted CI of the nonspaced batch means at level
 * 1 - alpha_ci.  out: device pointer, written asynchronously.  Errors:
 * PBN_ERR_INVALID (window outside the recorded positions, kappa or
 * batches_per_chain below 1, spacer below 0, fewer than 2 batches),
 * PBN_ERR_UNSUPPORTED (kappa above 2^30, batches_per_chain above 2^32). */
int pbn_skart(const pbn_chains *chains, int64_t start, int64_t kappa, int64_t batches_per_chain,
              int64_t spacer, double alpha_ci, double alpha_ran, pbn_skart_result *out, void *stream);

/* Maximum omega * batches_per_chain of pbn_skart_static. */
#define PBN_SKART_STATIC_MAX_BATCHES (1 << 18)

/* pbn_skart without any device allocation.  The paper has no counterpart;
 * this is for callers that cannot let a library call cudaMalloc, such as a
 * host program that owns all device memory through its own allocator, or a
 * latency-critical loop in which an allocation would stall the device.
 * Computes exactly what pbn_skart computes, but keeps the per-batch sums in
 * a fixed array of PBN_SKART_STATIC_MAX_BATCHES entries (1 MiB) inside the
 * library's device image, which every GPU that loads the library holds until
 * the process exits.  The caller still passes the chains and the result slot.
 * The first call on a device looks up the array's device address (make that
 * first call before any stream capture); CUDA loads the library's device
 * code lazily, so that first call also loads it and reserves the 1 MiB array
 * on the device, and can fail with PBN_ERR_CUDA when device memory is short.
 * Later calls on that device allocate nothing.  All calls share the one array:
 * calls whose work overlaps on the GPU (different streams, or other host
 * threads) race and must be serialised by the caller.  Each call overwrites
 * every batch sum it reads, so nothing needs clearing between calls.
 * Errors: PBN_ERR_UNSUPPORTED when omega * batches_per_chain exceeds
 * PBN_SKART_STATIC_MAX_BATCHES or kappa exceeds 2^30, PBN_ERR_INVALID as
 * pbn_skart, PBN_ERR_CUDA. */
int pbn_skart_static(const pbn_chains *chains, int64_t start, int64_t kappa, int64_t batches_per_chain,
                     int64_t spacer, double alpha_ci, double alpha_ran, pbn_skart_result *out, void *stream);

/* -------------------------------------------------------------- drivers */

typedef struct pbn_two_state_query {
    int64_t omega;           /* chains, >= 2 */
    int64_t psi0;            /* initial G&R burn-in */
    double rhat_threshold;   /* converged when R-hat < threshold */
    double eps, r, s;        /* Alg. 1 parameters */
    int64_t max_length;      /* cap on the chain length */
    uint64_t seed;
    int32_t perturb_mode;
    pbn_soi soi;
} pbn_two_state_query;

typedef struct pbn_two_state_report {
    double prob, rhat, alpha, beta;
    int64_t psi, gr_psi, length, sample_size, M, N, ones;
    int64_t n4[4];
    int32_t gr_rounds, ts_rounds;
    int64_t chain_node_updates;   /* omega * length * n */
    double device_ms;             /* device time of the whole query */
    double sim_ms;                /* CUDA-event time of the simulation launches (same stream) */
    int64_t sim_launches;         /* simulation kernel launches */
    int64_t kernel_launches;      /* all kernel launches of the query */
    int64_t sim_items;            /* (node, chain group, transition) items simulated */
    int64_t d2h_bytes;            /* device -> host bytes read for the stopping decisions */
    double apply_ms;              /* select-ahead schedule: CUDA-event time of the apply launches alone */
    int64_t apply_launches;       /* select-ahead schedule: apply launches (0 under the fused schedule) */
} pbn_two_state_report;

/* Alg. GR then Alg. 3 (Sec. 4.2) end to end on the device: chains are
 * extended, checked and extended again until the two-state rule and the
 * burn-in check hold; only the stopping decisions cross to the host.
 * Allocates its own device buffers.  Synchronises `stream`.
 * Errors: PBN_ERR_NOT_CONVERGED (max_length), PBN_ERR_INVALID, PBN_ERR_OOM, PBN_ERR_CUDA. */
int pbn_estimate_two_state(const pbn_net *net, const pbn_two_state_query *q, pbn_two_state_report *out,
                           void *stream);

/* Sequential two-state Markov chain approach on one chain (Sec. 3.1,
 * Alg. 1): the control of the parallel method (Sec. 5.1 compares the two). */
typedef struct pbn_two_state_seq_query {
    int64_t m0, n0;          /* initial burn-in (>= 0) and sample size (>= 2) */
    double eps, r, s;
    int64_t max_length;
    uint64_t seed;           /* chain 0 of this seed's family is simulated */
    int32_t perturb_mode;
    pbn_soi soi;
} pbn_two_state_seq_query;

typedef struct pbn_two_state_seq_report {
    double prob, alpha, beta;
    int64_t M, N, length, ones;
    int64_t n4[4];           /* transitions of the last alpha, beta window */
    int64_t ab_window;       /* its length */
    int32_t rounds;
    int64_t chain_node_updates;   /* length * n */
    double device_ms, sim_ms;
    int64_t sim_launches, kernel_launches, d2h_bytes;
} pbn_two_state_seq_report;

/* Alg. 1: start from length l = m0 + n0; each round extends the chain to
 * M + N (none in the first), estimates alpha and beta from the last N
 * positions and recomputes M and N (Alg. 1 line 8), until M + N <= l; the
 * estimate is the fraction of ones in the last N positions.  A window without
 * a 0->1 or 1->0 transition doubles N.  Synchronises `stream`.
 * Errors: PBN_ERR_NOT_CONVERGED (max_length, or alpha = beta = 1),
 * PBN_ERR_INVALID, PBN_ERR_OOM, PBN_ERR_CUDA. */
int pbn_estimate_two_state_seq(const pbn_net *net, const pbn_two_state_seq_query *q,
                               pbn_two_state_seq_report *out, void *stream);

/* One property's part of a multi-property query (Sec. 4.2, last part). */
typedef struct pbn_property_result {
    double prob, alpha, beta;
    double rhat;            /* its R-hat at the accepted Gelman-Rubin psi */
    int64_t M, N, ones;
    int64_t n4[4];
} pbn_property_result;

/* Several properties (sets of states of interest) from the same trajectories
 * (Sec. 4.2, last part): one set of chains, each property abstracted from it
 * in the same simulation pass.  Alg. GR doubles psi until every property's
 * R-hat is below the threshold; each round estimates alpha, beta, M, N per
 * property; the chains grow by the smallest deficit among the properties
 * whose N exceeds the merged sample, until none does; the burn-in check
 * takes the largest M.  One property gives exactly pbn_estimate_two_state.
 * q->soi is ignored; props[0 .. n_props-1] (1 <= n_props <= PBN_MAX_PROPERTIES,
 * at most PBN_MAX_SOI entries in total) name the properties; each[m] receives
 * property m's result and `out` the common fields (its per-property fields
 * repeat property 0).  Synchronises `stream`.  Errors as pbn_estimate_two_state. */
int pbn_estimate_two_state_multi(const pbn_net *net, const pbn_two_state_query *q, int32_t n_props,
                                 const pbn_soi *props, pbn_two_state_report *out, pbn_property_result *each,
                                 void *stream);

typedef struct pbn_skart_query {
    int64_t omega;
    int64_t psi0;
    double rhat_threshold;
    double H_star;           /* precision requirement */
    int32_t relative;        /* 1: the requirement is H_star * |mean| */
    double alpha;            /* CI level 1 - alpha */
    int64_t max_length;
    uint64_t seed;
    int32_t perturb_mode;
    pbn_soi soi;
} pbn_skart_query;

typedef struct pbn_skart_report {
    double mean, ci_lo, ci_hi, H, var, skew, phi, rhat;
    int64_t psi, length, kappa, batches, spacer, sample_size;
    int32_t gr_rounds, rand_rounds, ci_rounds;
    int64_t chain_node_updates;
    double device_ms;
    double sim_ms;
    int64_t sim_launches, kernel_launches, sim_items, d2h_bytes;
    double apply_ms;
    int64_t apply_launches;
} pbn_skart_report;

/* Alg. GR then Alg. 4 (Sec. 4.3) end to end on the device.  Synchronises
 * `stream`.  Errors as pbn_estimate_two_state. */
int pbn_estimate_skart(const pbn_net *net, const pbn_skart_query *q, pbn_skart_report *out, void *stream);

/* Alg. 2 (Sec. 3.2), the sequential Skart method on chain 0 of the seed's
 * family (the control of Alg. 4), with Alg. 4's constants: skewness of the
 * last 1024 of 1280 samples, the randomness test on the whole trajectory with
 * spacer d, then the CI on the batches after the d skipped ones.  q->omega,
 * q->psi0 and q->rhat_threshold are ignored; out->psi is the skipped d kappa,
 * out->batches the batches after it.  Synchronises `stream`.
 * Errors as pbn_estimate_skart. */
int pbn_estimate_skart_seq(const pbn_net *net, const pbn_skart_query *q, pbn_skart_report *out, void *stream);

/* ------------------------------------------------- batched / served queries
 *
 * The engine advances many independent queries (each: a network, a state of
 * interest, Alg. GR then Alg. 3 or Alg. 4 with its own seed and chain count)
 * together.  Each epoch is one persistent simulation launch that extends
 * every active query towards its next check, then one batched launch of the
 * Gelman & Rubin / two-state statistics of the queries at a check (Skart
 * checks run as their own launches after it).  The host then applies each
 * query's stopping rule.  Chain states and bitstreams stay resident on the
 * device from admission to completion.  Queries are admitted while a slot
 * is free and the device-memory budget allows; a query's result is the same
 * alone (pbn_estimate_two_state / pbn_estimate_skart) and in any mix,
 * because its trajectory is a function of its own seed and its checks
 * happen at the same lengths.  An autotuner picks transitions per epoch,
 * threads per CTA and chain groups per CTA by timing live epochs.  The
 * paper has no counterpart: this is the batching and serving layer. */

enum { PBN_METHOD_TWO_STATE = 0, PBN_METHOD_SKART = 1 };
#define PBN_ENGINE_MAX_ACTIVE 128

typedef struct pbn_engine pbn_engine;

typedef struct pbn_engine_cfg {
    int64_t hbm_budget_bytes;   /* device bytes for chain states and bitstreams; 0 = 8 GiB */
    int32_t max_active;         /* query slots, 1..PBN_ENGINE_MAX_ACTIVE; 0 = the maximum */
    int32_t steps_per_epoch;    /* most transitions a query advances per epoch; 0 = autotuned */
    int32_t threads_per_block;  /* 256 or 512; 0 = autotuned */
    int32_t items_per_thread;   /* (node, chain group) items per thread when sizing CTAs; 0 = autotuned */
    int32_t use_graph;          /* 1: each epoch is a captured CUDA graph, replayed */
    /* Latency bound for serving: when > 0, a query's extension in one epoch is
     * capped at about this many milliseconds of device time (estimated from the
     * rates of earlier epochs, at least 64 transitions), so that queries that
     * arrive wait at most about that long for the next epoch to admit them.
     * 0: epochs end only at steps_per_epoch or a query's next check (more work
     * per launch, the better setting for a batch submitted at once). */
    double epoch_target_ms;
} pbn_engine_cfg;

typedef struct pbn_engine_query {
    const pbn_net *net;                /* must outlive the query */
    int32_t method;                    /* PBN_METHOD_TWO_STATE or PBN_METHOD_SKART */
    pbn_two_state_query two_state;     /* used for PBN_METHOD_TWO_STATE */
    pbn_skart_query skart;             /* used for PBN_METHOD_SKART */
    uint64_t tag;                      /* returned with the result */
} pbn_engine_query;

typedef struct pbn_engine_result {
    int64_t id;
    uint64_t tag;
    int32_t method;
    int32_t status;                    /* PBN_OK or the error that ended the query */
    pbn_two_state_report two_state;
    pbn_skart_report skart;
    int64_t submit_epoch, admit_epoch, finish_epoch;
} pbn_engine_result;

typedef struct pbn_engine_stats {
    int64_t epoch;
    int32_t active, pending;
    int64_t finished;                  /* results waiting to be polled */
    int64_t updates;                   /* chain-node updates of this epoch */
    double epoch_ms;                   /* device time of this epoch's launches */
    int64_t hbm_in_use;
    int32_t steps_per_epoch, threads_per_block, items_per_thread;
    int32_t kernel_launches;           /* kernels this epoch launched */
    double sim_ms;                     /* CUDA-event time of this epoch's batch_sim_kernel launch (0: none) */
    int64_t sim_items;                 /* its (node, chain group, transition) items */
    int64_t d2h_bytes;                 /* device -> host bytes this epoch read (results, status) */
    int32_t tuning;                    /* 1 while the autotuner is still timing candidates */
    int32_t pad;
} pbn_engine_stats;

/* Create an engine on the current device.  It runs on a stream of its own,
 * ordered after the work already queued on `stream`, and allocates its fixed
 * epoch buffers.  Errors: PBN_ERR_INVALID, PBN_ERR_OOM, PBN_ERR_CUDA. */
int pbn_engine_create(const pbn_engine_cfg *cfg, void *stream, pbn_engine **out);
void pbn_engine_destroy(pbn_engine *engine);
/* Queue a query (host arguments copied).  *id identifies its result.
 * Errors: PBN_ERR_INVALID (as the single-query drivers). */
int pbn_engine_submit(pbn_engine *engine, const pbn_engine_query *query, int64_t *id);
/* One epoch: admit, simulate, check, retire.  Synchronises the stream.
 * A query that fails ends with its status in the result; the call itself
 * fails only for engine-wide errors (PBN_ERR_CUDA, PBN_ERR_OOM). */
int pbn_engine_step(pbn_engine *engine, pbn_engine_stats *stats);
/* Move up to max_results finished results into out (host memory).  In a
 * result, two_state.sim_items / skart.sim_items count the query's items
 * simulated by the batched kernel (not those of epochs in which a lone query
 * ran on the single-query schedule). */
int pbn_engine_poll(pbn_engine *engine, pbn_engine_result *out, int32_t max_results, int32_t *count);
/* Withdraw query `id` (waiting or active) between epochs, for a client that
 * no longer wants its answer (a stopping rule that may never fire short of
 * max_length, a deadline passed).  Its chain buffers are freed and its
 * result is queued for pbn_engine_poll with status PBN_ERR_CANCELLED; the
 * other queries are not affected (their results stay the same).
 * Errors: PBN_ERR_INVALID (NULL engine, or no waiting or active query with
 * that id: unknown, finished or already cancelled). */
int pbn_engine_cancel(pbn_engine *engine, int64_t id);

/* ---------------------------------------------------------------- errors */

const char *pbn_last_error(void);
const char *pbn_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* PBN_H */
