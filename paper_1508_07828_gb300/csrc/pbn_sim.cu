// Chain initialisation and the synchronous PBN step (Sec. 2.2) on sm_103a.
//
// Layout: bit-sliced chains.  One 32-bit word holds one node of 32 chains (a
// chain group).  A CTA owns `gpb` groups and all n nodes of them: their
// current and next states sit in shared memory as [node][group] words, next
// to the network tables.  An item is one (node, group) pair of one step:
// 32 chain-node updates.  T threads share an item (T = 1, 2 or 4).
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
#include "pbn_internal.cuh"

namespace pbn {

constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t sext_bit(uint32_t w, int b) {
  return (uint32_t)((int32_t)(w << (31 - b)) >> 31);
}

// Multiplexer-tree evaluation of a K-input truth table on bit-sliced inputs:
// leaf j = truth-table bit j (as 0 or ~0); level m selects on x[m].
template <int K>
__device__ __forceinline__ uint32_t eval_tt(uint32_t tt, const uint32_t *x) {
  if constexpr (K == 0) {
    return sext_bit(tt, 0);
  } else {
    constexpr int NL = 1 << K;
    uint32_t v[NL / 2];
#pragma unroll
    for (int q = 0; q < NL / 2; q++) {
      const uint32_t lo = sext_bit(tt, 2 * q), hi = sext_bit(tt, 2 * q + 1);
      v[q] = (x[0] & hi) | (~x[0] & lo);
    }
#pragma unroll
    for (int m = 1; m < K; m++) {
#pragma unroll
      for (int q = 0; q < (NL >> (m + 1)); q++) v[q] = (x[m] & v[2 * q + 1]) | (~x[m] & v[2 * q]);
    }
    return v[0];
  }
}

// Function record evaluated at tree depth K >= its own k: the truth table is
// replicated to 2^K leaves; parents m >= k are node 0 (their value then does
// not matter).
template <int K>
__device__ __forceinline__ uint32_t eval_at_depth(uint4 rec, int k, const uint32_t *cur, int gpb, int gl) {
  uint32_t tt = rec.x;
#pragma unroll
  for (int e = 0; e < K; e++)
    if (e >= k) tt |= tt << (1 << e);
  int p[5];
  p[0] = rec.z & 0xFFF;
  p[1] = (rec.z >> 12) & 0xFFF;
  p[2] = rec.w & 0xFFF;
  p[3] = (rec.w >> 12) & 0xFFF;
  p[4] = (int)((rec.z >> 24) | (((rec.w >> 24) & 0xFu) << 8));
  uint32_t x[5];
#pragma unroll
  for (int m = 0; m < K; m++) x[m] = cur[p[m] * gpb + gl];
  return eval_tt<K>(tt, x);
}

// K is warp-uniform, so the switch does not diverge.
__device__ __forceinline__ uint32_t eval_uniform(int K, uint4 rec, int k, const uint32_t *cur, int gpb, int gl) {
  switch (K) {
    case 0: return eval_at_depth<0>(rec, k, cur, gpb, gl);
    case 1: return eval_at_depth<1>(rec, k, cur, gpb, gl);
    case 2: return eval_at_depth<2>(rec, k, cur, gpb, gl);
    case 3: return eval_at_depth<3>(rec, k, cur, gpb, gl);
    case 4: return eval_at_depth<4>(rec, k, cur, gpb, gl);
    default: return eval_at_depth<5>(rec, k, cur, gpb, gl);
  }
}

struct ItemCtx {
  const uint4 *fn_s;
  const uint32_t *cur;
  uint32_t *nxt;
  uint32_t *pbuf;
  unsigned int *anyP;
  bool active;
  int i, L, f0;
  uint32_t g;
  int gl, gpb;
  uint32_t vmask;
  uint64_t t;
  int sub;
};

// One item of one transition with LW (warp-uniform) category bounds; bound 0
// is P32, bound m is T_{m-1}; bounds m >= L are unreachable (all lanes below).
template <int LW, int MODE, int T, int BPR>
__device__ __forceinline__ void step_item(const SimArgs &a, const ItemCtx &c) {
  uint32_t ts[LW], und[LW], lt[LW];
#pragma unroll
  for (int m = 0; m < LW; m++) {
    const bool real = m < c.L;
    ts[m] = (m == 0) ? a.P32 : (real ? c.fn_s[c.f0 + m - 1].y : 0u);
    und[m] = real ? c.vmask : 0u;
    lt[m] = real ? 0u : kFull;
  }
  const uint32_t cy = (uint32_t)c.t, cz = (uint32_t)(c.t >> 32) & 0xFFFFFFu;
#pragma unroll 1
  for (int round = 0; round * T * BPR < 8; round++) {
    uint32_t pend = 0u;
#pragma unroll
    for (int m = 0; m < LW; m++) pend |= und[m];
    if (!__any_sync(kFull, pend != 0u)) break;
    uint32_t u[LW], l[LW];
#pragma unroll
    for (int m = 0; m < LW; m++) {
      u[m] = kFull;
      l[m] = 0u;
    }
#pragma unroll
    for (int cblk = 0; cblk < BPR; cblk++) {
      const uint32_t b = (uint32_t)((round * T + c.sub) * BPR + cblk);
      const uint4 R = philox4x32_10(make_uint4((uint32_t)c.i, cy, cz | (b << 24), c.g), a.rk);
      const uint32_t Rq[4] = {R.x, R.y, R.z, R.w};
#pragma unroll
      for (int m = 0; m < LW; m++) {
        const uint32_t tsb = ts[m] << (4u * b);
#pragma unroll
        for (int q = 0; q < 4; q++) {
          // bound digit as 0 / ~0; lanes whose digit differs are decided
          const uint32_t tm = (uint32_t)((int32_t)(tsb << q) >> 31);
          const uint32_t dec = u[m] & (Rq[q] ^ tm);
          l[m] |= dec & tm;  // bound digit 1, lane digit 0: u < bound
          u[m] &= ~dec;
        }
      }
    }
    // merge the T threads' consecutive digit blocks in order
#pragma unroll
    for (int k = 1; k < T; k <<= 1) {
#pragma unroll
      for (int m = 0; m < LW; m++) {
        const uint32_t pu = __shfl_xor_sync(kFull, u[m], k);
        const uint32_t pl = __shfl_xor_sync(kFull, l[m], k);
        if (c.sub & k) {
          l[m] = pl | (pu & l[m]);
        } else {
          l[m] = l[m] | (u[m] & pl);
        }
        u[m] &= pu;
      }
    }
#pragma unroll
    for (int m = 0; m < LW; m++) {
      lt[m] |= und[m] & l[m];
      und[m] &= u[m];
    }
  }
  // lanes of function j: below bound j+1 and not below bound j
  uint32_t sel[LW];
  {
    uint32_t prev = lt[0];
#pragma unroll
    for (int j = 0; j < LW; j++) {
      const uint32_t upto = (j + 1 < LW) ? lt[j + 1] : kFull;
      sel[j] = upto & ~prev & c.vmask;
      prev = upto;
    }
  }
  uint32_t fword = 0u;
#pragma unroll
  for (int p0 = 0; p0 < LW; p0 += T) {
    uint32_t my_sel = 0u;
#pragma unroll
    for (int s = 0; s < T; s++)
      if (s == c.sub && p0 + s < LW) my_sel = sel[p0 + s];
    const int j = p0 + c.sub;
    const bool has = (j < c.L) && my_sel != 0u;
    const uint4 rec = has ? c.fn_s[c.f0 + j] : make_uint4(0u, 0u, 0u, 0u);
    const int k = has ? fn_k(rec) : 0;
    const int K = __reduce_max_sync(kFull, (unsigned)k);
    if (__any_sync(kFull, has)) fword |= my_sel & eval_uniform(K, rec, k, c.cur, c.gpb, c.gl);
  }
#pragma unroll
  for (int k = 1; k < T; k <<= 1) fword |= __shfl_xor_sync(kFull, fword, k);
  if (c.active && c.sub == 0) {
    const int idx = c.i * c.gpb + c.gl;
    if (MODE == PBN_PERTURB_PER_NODE) {
      c.nxt[idx] = (lt[0] & ~c.cur[idx]) | fword;
    } else {
      c.nxt[idx] = fword;
      c.pbuf[idx] = lt[0];
      if (lt[0]) atomicOr(&c.anyP[c.gl], lt[0]);
    }
  }
}

__device__ __forceinline__ uint32_t lane_mask(int64_t omega, uint32_t g) {
  int64_t rem = omega - (int64_t)g * 32;
  return rem >= 32 ? 0xFFFFFFFFu : ((1u << rem) - 1u);
}

// Nodes with more than 4 functions are rare; their variant is kept out of
// line so its register demand does not raise the common path's.
template <int MODE, int T, int BPR>
__device__ __noinline__ void step_item_wide(const SimArgs &a, const ItemCtx &c) {
  step_item<kMaxL, MODE, T, BPR>(a, c);
}

template <int MODE, int T, int BPR>
__device__ __forceinline__ void dispatch_item(int LW, const SimArgs &a, const ItemCtx &c) {
  switch (LW) {
    case 0: break;
    case 1: step_item<1, MODE, T, BPR>(a, c); break;
    case 2: step_item<2, MODE, T, BPR>(a, c); break;
    case 3: step_item<3, MODE, T, BPR>(a, c); break;
    case 4: step_item<4, MODE, T, BPR>(a, c); break;
    default: step_item_wide<MODE, T, BPR>(a, c); break;
  }
}

// Threads per CTA a variant is compiled for: one thread per item may fill
// 1024 threads (64 registers each); shared items run at most 512 threads.
template <int T>
constexpr int max_threads() { return T == 1 ? 1024 : 512; }

template <int MODE, int T, int BPR>
__global__ void __launch_bounds__(max_threads<T>()) sim_kernel(const __grid_constant__ SimArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int gpb = a.gpb;
  const int n = a.n;
  const uint32_t g0 = blockIdx.x * (uint32_t)gpb;
  const int ngl = min(gpb, a.G - (int)g0);
  const uint4 *fn_s = a.fn;
  const uint32_t *node_s = a.node;
  size_t off = 0;
  if (a.tables_in_smem) {
    uint4 *f = reinterpret_cast<uint4 *>(smem);
    for (int j = threadIdx.x; j < a.F; j += blockDim.x) f[j] = a.fn[j];
    off = (size_t)a.F * 16;
    uint32_t *nd = reinterpret_cast<uint32_t *>(smem + off);
    for (int j = threadIdx.x; j < n; j += blockDim.x) nd[j] = a.node[j];
    off += ((size_t)n * 4 + 15) & ~(size_t)15;
    fn_s = f;
    node_s = nd;
  }
  const int items = n * gpb;
  uint32_t *bufA = reinterpret_cast<uint32_t *>(smem + off);
  uint32_t *bufB = bufA + items;
  uint32_t *pbuf = bufB + items;
  unsigned int *anyP = reinterpret_cast<unsigned int *>(pbuf + items);  // [2][gpb]
  for (int idx = threadIdx.x; idx < items; idx += blockDim.x) {
    int i = idx / gpb, gl = idx - i * gpb;
    bufA[idx] = gl < ngl ? a.state[(size_t)(g0 + gl) * n + i] : 0u;
  }
  if (MODE == PBN_PERTURB_GLOBAL)
    for (int j = threadIdx.x; j < 2 * gpb; j += blockDim.x) anyP[j] = 0u;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int sub = lane & (T - 1);
  const int slot = threadIdx.x / T;
  const int nslots = blockDim.x / T;
  uint32_t *cur = bufA, *nxt = bufB;
  for (int s = 0; s < a.steps; s++) {
    ItemCtx c;
    c.fn_s = fn_s;
    c.cur = cur;
    c.nxt = nxt;
    c.pbuf = pbuf;
    c.anyP = anyP + (s & 1) * gpb;
    c.gpb = gpb;
    c.t = a.t0 + (uint64_t)s;
    c.sub = sub;
    for (int base = 0; base < items; base += nslots) {  // uniform trip count
      const int q = base + slot;
      const int r = q / gpb;
      c.gl = q - r * gpb;
      c.active = (q < items) && (c.gl < ngl);
      const uint32_t rec = c.active ? node_s[r] : 0u;
      c.L = c.active ? node_l(rec) : 0;
      c.i = node_id(rec);
      c.f0 = node_f0(rec);
      c.g = g0 + (uint32_t)c.gl;
      c.vmask = c.active ? lane_mask(a.omega, c.g) : 0u;
      const int LW = (int)__reduce_max_sync(kFull, (unsigned)c.L);
      dispatch_item<MODE, T, BPR>(LW, a, c);
    }
    __syncthreads();
    if (MODE == PBN_PERTURB_GLOBAL) {
      for (int idx = threadIdx.x; idx < items; idx += blockDim.x) {
        const uint32_t any = c.anyP[idx % gpb];
        nxt[idx] = (any & (cur[idx] ^ pbuf[idx])) | (~any & nxt[idx]);
      }
      unsigned int *anyN = anyP + ((s + 1) & 1) * gpb;
      for (int j = threadIdx.x; j < gpb; j += blockDim.x) anyN[j] = 0u;
      __syncthreads();
    }
    if (a.soi_size > 0) {
      const int64_t col = a.col0 + s;
      for (int gl = warp; gl < ngl; gl += nwarps) {
        uint32_t v = kFull;
        if (lane < a.soi_size) {
          const uint32_t w = nxt[a.soi_node[lane] * gpb + gl];
          v = ((a.soi_val >> lane) & 1u) ? w : ~w;
        }
        v = __reduce_and_sync(kFull, v);
        if (lane == 0 && col >= 0) a.bits[(size_t)(g0 + gl) * a.bits_cap + col] = v & lane_mask(a.omega, g0 + gl);
      }
    }
    uint32_t *tmp = cur;
    cur = nxt;
    nxt = tmp;
  }
  for (int idx = threadIdx.x; idx < items; idx += blockDim.x) {
    int i = idx / gpb, gl = idx - i * gpb;
    if (gl < ngl) a.state[(size_t)(g0 + gl) * n + i] = cur[idx];
  }
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

size_t sim_smem_bytes(int n, int F, int gpb, int mode, bool tables_in_smem) {
  size_t b = 0;
  if (tables_in_smem) b += (size_t)F * 16 + (((size_t)n * 4 + 15) & ~(size_t)15);
  size_t items = (size_t)n * gpb;
  b += 2 * items * 4;
  if (mode == PBN_PERTURB_GLOBAL) b += items * 4 + 2 * (size_t)gpb * 4;
  return b;
}

int sim_max_smem() {
  static int v = -1;
  if (v < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) v = 48 * 1024;
  }
  return v;
}

template <int MODE, int T, int BPR>
static cudaError_t launch_variant(const SimArgs &a, int blocks, int threads, size_t smem, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(sim_kernel<MODE, T, BPR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         sim_max_smem());
    if (e != cudaSuccess) return e;
    attr = true;
  }
  sim_kernel<MODE, T, BPR><<<blocks, threads, smem, s>>>(a);
  return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_mode(const SimArgs &a, int T, int BPR, int blocks, int threads, size_t smem,
                               cudaStream_t s) {
  if (T == 4) return launch_variant<MODE, 4, 1>(a, blocks, threads, smem, s);
  if (T == 2) return launch_variant<MODE, 2, 2>(a, blocks, threads, smem, s);
  if (BPR == 1) return launch_variant<MODE, 1, 1>(a, blocks, threads, smem, s);
  return launch_variant<MODE, 1, 2>(a, blocks, threads, smem, s);
}

cudaError_t launch_sim(const SimArgs &a, int mode, int T, int BPR, int threads, size_t smem, cudaStream_t s) {
  const int blocks = (a.G + a.gpb - 1) / a.gpb;
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
