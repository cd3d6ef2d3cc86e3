// Chain initialisation and the synchronous PBN step (Sec. 2.2) on sm_103a.
//
// Layout: bit-sliced chains.  One 32-bit word holds one node of 32 chains (a
// chain group).  A CTA owns up to `gpb` groups and all n nodes of them: their
// current and next states sit in shared memory as [node][group] words, next
// to the network tables.  An item is one (node, group) pair of one step:
// 32 chain-node updates.  T threads share an item (T = 1, 2 or 4).  A
// balanced launch gives CTAs different group counts and step ranges (two
// segments of SimArgs), so that two launches spread a group count that is not
// a multiple of the SM count evenly over the SMs.
//
// Per item and transition t:
//  1. Category of every lane's uniform u against the node's sorted bounds
//     (P32, T_0 .. T_{l-2}).  u's binary digits are bit `lane` of Philox output
//     words, most significant first; every Philox block gives 4 digits.  The
//     comparison walks the digits and stops once no lane is tied with any
//     bound (2-3 blocks instead of the 8 a full 32-bit u per lane needs).  The
//     T threads of an item take consecutive blocks in parallel and merge their
//     partial comparisons in digit order with an associative butterfly:
//     (undecided, less) o (undecided', less') = (u & u', l | (u & l')).
//  2. Value of each selected predictor function on the 32 chains by a
//     multiplexer tree over the parents' state words (truth-table bits as
//     leaves); each lane takes its own category's function.  Tree depth and
//     function count are made warp-uniform (__reduce_max_sync): a shallower
//     truth table is replicated to the common depth (extra parents then select
//     between equal halves) and missing functions get an unreachable bound, so
//     no lane of a warp branches away from the others.
//  3. Per-node perturbation: perturbed lanes flip.  Global perturbation: lanes
//     with any perturbed node take s XOR gamma (second pass after a barrier).
// After each step every group's indicator word of the state of interest
// (Sec. 3.1) is an AND-reduction across one warp's lanes, stored to the
// bitstream.
#include <mutex>

#include "pbn_step.cuh"

namespace pbn {

// WIDE: the variant for networks with functions of more than 5 inputs (one
// thread per item, one Philox block per round only).  LMAX: functions per node
// (kMaxLAll in the variant for networks with nodes of more than kMaxL).
template <int MODE, int T, int BPR, bool WIDE, int LMAX = kMaxL>
__global__ void __launch_bounds__(max_threads<T>()) sim_kernel(const __grid_constant__ SimArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  int g0 = (int)blockIdx.x * a.gpb, ngl = min(a.gpb, a.G - g0), nsteps = a.steps, soff = 0;
  if (a.seg_blocks[0] != 0) {
    // balanced launch: this CTA's share of its segment's groups
    int b = (int)blockIdx.x, q = 0;
    if (b >= a.seg_blocks[0]) {
      b -= a.seg_blocks[0];
      q = 1;
    }
    const int nb = a.seg_blocks[q];
    const int lo = (int)((int64_t)b * a.seg_ng[q] / nb), hi = (int)((int64_t)(b + 1) * a.seg_ng[q] / nb);
    g0 = a.seg_g0[q] + lo;
    ngl = hi - lo;
    nsteps = a.seg_steps[q];
    soff = a.seg_soff[q];
  }
  // layout stride ngl: a CTA with fewer groups than a.gpb runs fewer item rounds
  cta_simulate<MODE, T, BPR, WIDE, LMAX>(a, a.rk, (uint32_t)g0, ngl, ngl, smem, nsteps, soff);
}

__global__ void init_kernel(const __grid_constant__ RoundKeys rk, uint32_t *state, int n, int G, int64_t omega) {
  const int64_t total = (int64_t)G * n;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t g = (uint32_t)(idx / n);
    const uint32_t i = (uint32_t)(idx - (int64_t)g * n);
    uint4 R = philox4x32_10(make_uint4(i, 0xFFFFFFFFu, 0xFFFFFFFFu, g), rk);
    state[idx] = R.x & lane_mask(omega, g);
  }
}

size_t sim_smem_bytes(int n, int F, int gpb, int mode, int staging, int tile_bytes) {
  size_t b = 0;
  const size_t node_bytes = ((size_t)n * 4 + 15) & ~(size_t)15;
  if (staging == STAGE_SMEM) b += (size_t)F * 16 + node_bytes;
  if (staging == STAGE_TILES) b += 2 * (((size_t)tile_bytes + 127) & ~(size_t)127) + node_bytes + 16;
  size_t items = (size_t)n * gpb;
  b += 2 * items * 4;
  if (mode == PBN_PERTURB_GLOBAL) b += items * 4 + 2 * (size_t)gpb * 4;
  return b;
}

int *device_status() {
  static std::mutex mu;
  static int *ptr[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!ptr[dev]) {
    if (cudaMalloc(&ptr[dev], sizeof(int)) != cudaSuccess) return nullptr;
    cudaMemset(ptr[dev], 0, sizeof(int));
  }
  return ptr[dev];
}

int sim_max_smem() {
  static int v = -1;
  if (v < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) v = 48 * 1024;
    v -= kStaticSmemReserve;
  }
  return v;
}

template <int MODE, int T, int BPR, bool WIDE = false, int LMAX = kMaxL>
static cudaError_t launch_variant(const SimArgs &a, int blocks, int threads, size_t smem, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(sim_kernel<MODE, T, BPR, WIDE, LMAX>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, sim_max_smem());
    if (e != cudaSuccess) return e;
    attr = true;
  }
  sim_kernel<MODE, T, BPR, WIDE, LMAX><<<blocks, threads, smem, s>>>(a);
  return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_mode(const SimArgs &a, int T, int BPR, int blocks, int threads, size_t smem,
                               cudaStream_t s) {
  if (a.many) {
    if (T != 1 || BPR != 1) return cudaErrorInvalidValue;  // the planner gives such networks T = 1, BPR = 1
    return launch_variant<MODE, 1, 1, true, kMaxLAll>(a, blocks, threads, smem, s);
  }
  if (a.has_wide) {
    if (T != 1 || BPR != 1) return cudaErrorInvalidValue;  // the planner gives wide networks T = 1, BPR = 1
    return launch_variant<MODE, 1, 1, true>(a, blocks, threads, smem, s);
  }
  if (T == 4) return launch_variant<MODE, 4, 1>(a, blocks, threads, smem, s);
  if (T == 2) return launch_variant<MODE, 2, 2>(a, blocks, threads, smem, s);
  if (BPR == 1) return launch_variant<MODE, 1, 1>(a, blocks, threads, smem, s);
  return launch_variant<MODE, 1, 2>(a, blocks, threads, smem, s);
}

cudaError_t launch_sim(const SimArgs &a, int mode, int T, int BPR, int threads, size_t smem, cudaStream_t s) {
  const int blocks = a.seg_blocks[0] ? a.seg_blocks[0] + a.seg_blocks[1] : (a.G + a.gpb - 1) / a.gpb;
  if (blocks == 0 || a.steps == 0) return cudaSuccess;
  if (mode == PBN_PERTURB_PER_NODE) return launch_mode<PBN_PERTURB_PER_NODE>(a, T, BPR, blocks, threads, smem, s);
  return launch_mode<PBN_PERTURB_GLOBAL>(a, T, BPR, blocks, threads, smem, s);
}

cudaError_t launch_init(const NetDev &net, uint64_t seed, uint32_t *state, int64_t omega, cudaStream_t s) {
  const int G = (int)((omega + 31) / 32);
  const int64_t total = (int64_t)G * net.n;
  if (total == 0) return cudaSuccess;
  int threads = 256;
  int64_t blocks = (total + threads - 1) / threads;
  if (blocks > 4096) blocks = 4096;
  init_kernel<<<(unsigned)blocks, threads, 0, s>>>(make_round_keys(seed), state, net.n, G, omega);
  return cudaGetLastError();
}

}  // namespace pbn
