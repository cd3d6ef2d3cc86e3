// Internal declarations of the GB300 PBN engine (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pbn.h"

namespace pbn {

// Functions per node (= category bounds per node, P32 included): the draw keeps
// up to kMaxL bounds in registers; nodes with kMaxL+1 .. kMaxLAll functions
// (the dense class of the paper's sweep) take an out-of-line variant.
constexpr int kMaxL = 8;
constexpr int kMaxLAll = PBN_MAX_FUNCTIONS_PER_NODE;
// Inputs of one function: the common kernels gather up to kWideK parents per
// looked-up chain; networks with more (up to PBN_MAX_PARENTS) take the same
// out-of-line variant as those with more than kMaxL functions per node.
constexpr int kWideK = 12;
static_assert(PBN_MAX_PARENTS <= 15, "a function record keeps its input count in 4 bits");
constexpr int kMaxSoi = PBN_MAX_SOI;
constexpr int kMaxProps = PBN_MAX_PROPERTIES;

// Device tables of one network (built by pbn_load).
//  node record (processing order r):  bits 0-11 node id, 12-15 l-1, 16-31 first function
//  function record (uint4), k <= 5 inputs:
//    x = truth table
//    y = upper category bound T_j (unused for the last function of a node)
//    z = p0 | p1 << 12 | (p4 & 0xFF) << 24
//    w = p2 | p3 << 12 | (p4 >> 8) << 24 | k << 28
//  k = 6 .. 15 inputs ("wide"): x = first of its 2^(k-5) table words in
//    d_wide_tt, z = first of its k parents in d_wide_par, w = k << 28
struct NetDev {
  int n = 0, F = 0;
  uint32_t P32 = 0;
  int max_l = 0;
  int max_k = 0;                  // most inputs of one function
  uint32_t *d_node = nullptr;
  uint4 *d_fn = nullptr;          // function records in processing order
  int32_t *d_tiles = nullptr;     // [ntiles+1] first processing position of each tile
  int ntiles = 0;
  int tile_bytes = 0;             // largest tile
  int64_t table_bytes = 0;
  int has_wide = 0;               // some function has more than 5 inputs
  uint32_t *d_wide_tt = nullptr;  // their truth tables (record x = first word)
  uint16_t *d_wide_par = nullptr; // their parents (record z = first entry)
};

// Records per TMA tile (24 KB of function records).
constexpr int kTileRecords = 1536;

// Where a CTA reads the function records from.
enum Staging { STAGE_GLOBAL = 0, STAGE_SMEM = 1, STAGE_TILES = 2 };

__host__ __device__ __forceinline__ int node_id(uint32_t rec) { return (int)(rec & 0xFFFu); }
__host__ __device__ __forceinline__ int node_l(uint32_t rec) { return (int)((rec >> 12) & 0xFu) + 1; }
__host__ __device__ __forceinline__ int node_f0(uint32_t rec) { return (int)(rec >> 16); }
__host__ __device__ __forceinline__ int fn_k(uint4 r) { return (int)(r.w >> 28); }

// Philox4x32-10 round constants (Salmon et al., SC'11).
constexpr uint32_t kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u, kPhiloxW1 = 0xBB67AE85u;

// Round keys k_r = key + r * W, r = 0..9, precomputed on the host.
struct RoundKeys {
  uint32_t k0[10];
  uint32_t k1[10];
};

inline RoundKeys make_round_keys(uint64_t seed) {
  RoundKeys rk;
  uint32_t a = (uint32_t)seed, b = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; r++) {
    rk.k0[r] = a;
    rk.k1[r] = b;
    a += kPhiloxW0;
    b += kPhiloxW1;
  }
  return rk;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const RoundKeys &rk) {
#pragma unroll
  for (int r = 0; r < 10; r++) {
    uint64_t p0 = (uint64_t)kPhiloxM0 * c.x;
    uint64_t p1 = (uint64_t)kPhiloxM1 * c.z;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c = make_uint4(hi1 ^ c.y ^ rk.k0[r], lo1, hi0 ^ c.w ^ rk.k1[r], lo0);
  }
  return c;
}

// Simulation launch arguments (passed by value, lives in the parameter bank).
struct SimArgs {
  RoundKeys rk;
  const uint32_t *node;
  const uint4 *fn;
  uint32_t *state;
  uint32_t *bits;
  int64_t bits_cap;
  int64_t col0;          // bits column of the first simulated position (may be < 0)
  int64_t omega;
  uint64_t t0;           // first transition index
  int n, F, G;
  int steps;
  int gpb;               // chain groups per block
  uint32_t P32;
  int staging;           // Staging: global, whole tables in shared memory, or TMA tiles
  const int32_t *tiles;  // tile starts (processing positions), for STAGE_TILES
  int ntiles;
  int tile_bytes;
  int *status;           // device status word: PBN_ERR_TIMEOUT after a bounded wait gave up
  int test_stall;        // test hook: never issue tile 0 (fused kernel) or step 0's category words
                         // (register-resident apply), so the wait for it must time out
  int soi_size;
  uint16_t soi_node[kMaxSoi];
  uint32_t soi_val;      // bit m = required value of soi_node[m]
  int mode;              // perturbation reading (batched kernel only)
  const uint32_t *wide_tt;   // tables and parents of functions with more than 5 inputs (NetDev)
  const uint16_t *wide_par;
  int has_wide;
  int many;              // some node has more than kMaxL functions or some function more than kWideK
                         // inputs (the fused kernel's kMaxLAll / PBN_MAX_PARENTS variant)
  int W;                 // select-ahead: category words per (step, group): F (+1 under global
                         // perturbation: word F is the OR of the perturbed lanes), rounded up to 4
  uint32_t *planes;      // select-ahead: category words [steps][G][W] of the chunk
  int ring_log2;         // select-ahead, register-resident apply: log2 of the ring slots
  int n_props;           // properties recorded (entries soi_node[m] belong to property soi_prop[m])
  int64_t prop_stride;   // words between two properties' bitstreams (G * bits_cap)
  // Fused kernel, balanced launch: CTAs 0 .. seg_blocks[0]-1 split groups
  // seg_g0[0] .. seg_g0[0]+seg_ng[0]-1 evenly and advance them seg_steps[0]
  // steps from transition t0 + seg_soff[0]; the next seg_blocks[1] CTAs do the
  // same with segment 1.  seg_blocks[0] = 0: CTA b takes groups b*gpb ..
  // b*gpb+gpb-1 for all `steps`.  gpb bounds the groups of any CTA.
  int seg_blocks[2];
  int seg_g0[2], seg_ng[2];
  int seg_steps[2], seg_soff[2];
  uint8_t soi_prop[kMaxSoi];
};
static_assert(sizeof(SimArgs) % 4 == 0, "SimArgs is copied word by word");

// One extension of a chain set by the schedule pbn_run_chains picks, its
// bounded waits reporting to `status` (pbn_api.cu; the engine's epochs with a
// single small query).  Advances ch.length; adds its launches to *launches.
int run_chains_alone(const NetDev &net, const pbn_run_cfg &cfg, pbn_chains &ch, int64_t steps, cudaStream_t s,
                     int *status, int64_t *launches);

// Sets the thread-local message returned by pbn_last_error (pbn_api.cu).
void set_last_error(const char *msg);

// Host-side launchers (defined in pbn_sim.cu / pbn_stats.cu).
cudaError_t launch_init(const NetDev &net, uint64_t seed, uint32_t *state, int64_t omega, cudaStream_t s);
// T = threads per (node, group) item (1, 2 or 4); BPR = Philox blocks per
// thread per round (T = 1: 1 or 2; T = 2 uses 2; T = 4 uses 1).
cudaError_t launch_sim(const SimArgs &a, int mode, int T, int BPR, int threads, size_t smem, cudaStream_t s);
size_t sim_smem_bytes(int n, int F, int gpb, int mode, int staging, int tile_bytes);
// Dynamic shared memory a simulation or apply launch may use: the device's
// per-block opt-in limit less kStaticSmemReserve, which covers the kernels'
// static shared memory (the CTA body's 256-byte nibble table).
constexpr int kStaticSmemReserve = 1024;
// Select-ahead schedule (pbn_split.cu): the category words of a.steps steps
// of all groups, then their application (a.staging: STAGE_SMEM or STAGE_GLOBAL).
// pad: unused dynamic shared memory per block (placement only; 0 = none).
cudaError_t launch_select(const SimArgs &a, int mode, int BPR, cudaStream_t s, size_t pad = 0);
// T = threads per (node, group) item: 1, 2 or 4 (each a share of the depth-5 tree).
cudaError_t launch_apply(const SimArgs &a, int mode, int ring, int T, int threads, size_t smem, cudaStream_t s);
size_t apply_smem_bytes(int n, int F, int gpb, int W, int staging, int ring, int n_props);
// Register-resident apply (two threads per item, at most kResidentItems items
// per CTA, no function with more than 5 inputs; function records beyond a
// node's second are read from global memory): threads = 2 x items rounded up
// to a warp, plus one producer warp; ring = 4, 8 or 16 slots.
constexpr int kResidentItems = 480;
// rest: some node has more than two functions (compiles that path in).
cudaError_t launch_apply_resident(const SimArgs &a, int mode, bool rest, int threads, size_t smem, cudaStream_t s);
size_t apply_resident_smem_bytes(int gpb, int W, int ring, int n_props);
int apply_threads_limit(int T);  // largest CTA of the apply variant for T
// Device status word of the simulation kernels on the current device (0 = ok).
int *device_status();
int sim_max_smem();

struct StatsScratch {
  // device scratch for the reductions: block partials + a ticket counter
  unsigned long long *partials = nullptr;  // [kMaxStatBlocks * 8]
  unsigned int *ticket = nullptr;
  int32_t *batch = nullptr;               // Skart batch sums
  int64_t batch_cap = 0;
};
constexpr int kMaxStatBlocks = 512;

cudaError_t scratch_init(StatsScratch &sc, cudaStream_t s);
void scratch_free(StatsScratch &sc);
cudaError_t scratch_reserve_batches(StatsScratch &sc, int64_t count, cudaStream_t s);

cudaError_t launch_gelman_rubin(const pbn_chains &ch, int64_t col, int64_t psi, pbn_gr_result *out,
                                StatsScratch &sc, cudaStream_t s);
cudaError_t launch_two_state(const pbn_chains &ch, int64_t col, int64_t len, double eps, double r, double sconf,
                             pbn_two_state_result *out, StatsScratch &sc, cudaStream_t s);
cudaError_t launch_skart(const pbn_chains &ch, int64_t col, int64_t kappa, int64_t bpc, int64_t spacer,
                         double alpha_ci, double alpha_ran, pbn_skart_result *out, StatsScratch &sc,
                         cudaStream_t s);
// Same kernels with a caller-provided batch-sum buffer of at least omega * bpc entries.
cudaError_t launch_skart_into(const pbn_chains &ch, int64_t col, int64_t kappa, int64_t bpc, int64_t spacer,
                              double alpha_ci, double alpha_ran, pbn_skart_result *out, int32_t *batch,
                              cudaStream_t s);

}  // namespace pbn

// The library-owned network handle of the C ABI.
struct pbn_net {
  pbn::NetDev dev;
  int device = 0;
  void *d_base = nullptr;  // the one device allocation holding every table of dev
};
