// Chain initialisation and the synchronous PBN step (Sec. 2.2) on sm_103a.
//
// Layout: bit-sliced chains.  One 32-bit word holds one node of 32 chains (a
// chain group); a CTA owns `gpb` groups and all n nodes of them, with the
// groups' current and next states in shared memory ([node][group] words) and
// the network tables staged in shared memory.  One thread computes one
// (node, group) item per step: 32 chain-node updates at once.
//
// Per item and transition t:
//  1. Category of every lane's uniform u against the node's sorted bounds
//     (P32, T_0 .. T_{l-2}): u's digits are bit (lane) of Philox output words,
//     most significant first, so the comparison walks digits and stops as soon
//     as no lane is still tied with any bound (usually after 2-3 Philox blocks
//     instead of the 8 that a full 32-bit u per lane would need).
//  2. Function value of each selected predictor function on the 32 chains by
//     a multiplexer tree over the parents' state words (truth-table bits as
//     leaves); lanes take the value of their own category's function.
//  3. Per-node perturbation: perturbed lanes flip.  Global perturbation: lanes
//     with any perturbed node take s XOR gamma (a second pass after a barrier).
// After each step one thread per group forms the indicator word of the state
// of interest (Sec. 3.1) and stores it to the bitstream.
#include "pbn_internal.cuh"

namespace pbn {

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
      uint32_t lo = sext_bit(tt, 2 * q), hi = sext_bit(tt, 2 * q + 1);
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

template <int K>
__device__ __forceinline__ uint32_t eval_fn_k(uint4 rec, const uint32_t *cur, int gpb, int gl) {
  uint32_t x[5];
  int p[5];
  p[0] = rec.z & 0xFFF;
  p[1] = (rec.z >> 12) & 0xFFF;
  p[2] = rec.w & 0xFFF;
  p[3] = (rec.w >> 12) & 0xFFF;
  p[4] = (int)((rec.z >> 24) | (((rec.w >> 24) & 0xFu) << 8));
#pragma unroll
  for (int m = 0; m < K; m++) x[m] = cur[p[m] * gpb + gl];
  return eval_tt<K>(rec.x, x);
}

__device__ __forceinline__ uint32_t eval_fn(uint4 rec, const uint32_t *cur, int gpb, int gl) {
  switch (fn_k(rec)) {
    case 0: return eval_fn_k<0>(rec, cur, gpb, gl);
    case 1: return eval_fn_k<1>(rec, cur, gpb, gl);
    case 2: return eval_fn_k<2>(rec, cur, gpb, gl);
    case 3: return eval_fn_k<3>(rec, cur, gpb, gl);
    case 4: return eval_fn_k<4>(rec, cur, gpb, gl);
    default: return eval_fn_k<5>(rec, cur, gpb, gl);
  }
}

// One (node, group) item of one transition.  L = number of category bounds =
// functions of the node (bound 0 is P32, bound m is T_{m-1}).
template <int L, int MODE>
__device__ __forceinline__ void step_item(const SimArgs &a, const uint4 *fn_s, const uint32_t *cur,
                                          uint32_t *nxt, uint32_t *pbuf, unsigned int *anyP, int i, int f0,
                                          uint32_t g, int gl, int gpb, uint32_t vmask, uint64_t t) {
  uint32_t ts[L], und[L], lt[L];
  ts[0] = a.P32;
#pragma unroll
  for (int m = 1; m < L; m++) ts[m] = fn_s[f0 + m - 1].y;
#pragma unroll
  for (int m = 0; m < L; m++) {
    und[m] = vmask;
    lt[m] = 0u;
  }
  const uint32_t cy = (uint32_t)t, cz = (uint32_t)(t >> 32) & 0xFFFFFFu;
#pragma unroll 1
  for (uint32_t b = 0; b < 8; b++) {
    uint32_t pend = 0;
#pragma unroll
    for (int m = 0; m < L; m++) pend |= und[m];
    if (pend == 0u) break;
    uint4 R = philox4x32_10(make_uint4((uint32_t)i, cy, cz | (b << 24), g), a.rk);
    const uint32_t Rq[4] = {R.x, R.y, R.z, R.w};
#pragma unroll
    for (int q = 0; q < 4; q++) {
#pragma unroll
      for (int m = 0; m < L; m++) {
        // threshold digit as 0 / ~0; decided lanes are those whose digit differs
        uint32_t tm = (uint32_t)((int32_t)(ts[m] << q) >> 31);
        uint32_t dec = und[m] & (Rq[q] ^ tm);
        lt[m] |= dec & tm;   // threshold digit 1, lane digit 0: u < bound
        und[m] &= ~dec;
      }
    }
#pragma unroll
    for (int m = 0; m < L; m++) ts[m] <<= 4;
  }
  uint32_t fword = 0u, prev = lt[0];
#pragma unroll
  for (int j = 0; j < L; j++) {
    uint32_t upto = (j + 1 < L) ? lt[j + 1] : 0xFFFFFFFFu;
    uint32_t sel = upto & ~prev & vmask;
    prev = upto;
    if (sel) fword |= sel & eval_fn(fn_s[f0 + j], cur, gpb, gl);
  }
  const int idx = i * gpb + gl;
  if (MODE == PBN_PERTURB_PER_NODE) {
    nxt[idx] = (lt[0] & ~cur[idx]) | fword;
  } else {
    nxt[idx] = fword;
    pbuf[idx] = lt[0];
    if (lt[0]) atomicOr(&anyP[gl], lt[0]);
  }
}

template <int MODE>
__device__ __forceinline__ void dispatch_item(int l, const SimArgs &a, const uint4 *fn_s, const uint32_t *cur,
                                              uint32_t *nxt, uint32_t *pbuf, unsigned int *anyP, int i,
                                              int f0, uint32_t g, int gl, int gpb, uint32_t vmask,
                                              uint64_t t) {
  switch (l) {
    case 1: step_item<1, MODE>(a, fn_s, cur, nxt, pbuf, anyP, i, f0, g, gl, gpb, vmask, t); break;
    case 2: step_item<2, MODE>(a, fn_s, cur, nxt, pbuf, anyP, i, f0, g, gl, gpb, vmask, t); break;
    case 3: step_item<3, MODE>(a, fn_s, cur, nxt, pbuf, anyP, i, f0, g, gl, gpb, vmask, t); break;
    case 4: step_item<4, MODE>(a, fn_s, cur, nxt, pbuf, anyP, i, f0, g, gl, gpb, vmask, t); break;
    case 5: step_item<5, MODE>(a, fn_s, cur, nxt, pbuf, anyP, i, f0, g, gl, gpb, vmask, t); break;
    case 6: step_item<6, MODE>(a, fn_s, cur, nxt, pbuf, anyP, i, f0, g, gl, gpb, vmask, t); break;
    case 7: step_item<7, MODE>(a, fn_s, cur, nxt, pbuf, anyP, i, f0, g, gl, gpb, vmask, t); break;
    default: step_item<8, MODE>(a, fn_s, cur, nxt, pbuf, anyP, i, f0, g, gl, gpb, vmask, t); break;
  }
}

__device__ __forceinline__ uint32_t lane_mask(int64_t omega, uint32_t g) {
  int64_t rem = omega - (int64_t)g * 32;
  return rem >= 32 ? 0xFFFFFFFFu : ((1u << rem) - 1u);
}

template <int MODE>
__global__ void __launch_bounds__(1024) sim_kernel(const __grid_constant__ SimArgs a) {
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
  uint32_t *cur = bufA, *nxt = bufB;
  for (int s = 0; s < a.steps; s++) {
    const uint64_t t = a.t0 + (uint64_t)s;
    unsigned int *anyS = anyP + (s & 1) * gpb;
    for (int q = threadIdx.x; q < items; q += blockDim.x) {
      const int r = q / gpb, gl = q - r * gpb;
      if (gl >= ngl) continue;
      const uint32_t rec = node_s[r];
      const uint32_t g = g0 + gl;
      dispatch_item<MODE>(node_l(rec), a, fn_s, cur, nxt, pbuf, anyS, node_id(rec), node_f0(rec), g, gl, gpb,
                          lane_mask(a.omega, g), t);
    }
    __syncthreads();
    if (MODE == PBN_PERTURB_GLOBAL) {
      for (int idx = threadIdx.x; idx < items; idx += blockDim.x) {
        const int gl = idx % gpb;
        const uint32_t any = anyS[gl];
        nxt[idx] = (any & (cur[idx] ^ pbuf[idx])) | (~any & nxt[idx]);
      }
      unsigned int *anyN = anyP + ((s + 1) & 1) * gpb;
      for (int j = threadIdx.x; j < gpb; j += blockDim.x) anyN[j] = 0u;
      __syncthreads();
    }
    if ((int)threadIdx.x < ngl && a.soi_size > 0) {
      const int gl = threadIdx.x;
      const uint32_t g = g0 + gl;
      uint32_t ind = lane_mask(a.omega, g);
      for (int m = 0; m < a.soi_size; m++) {
        const uint32_t w = nxt[a.soi_node[m] * gpb + gl];
        ind &= ((a.soi_val >> m) & 1u) ? w : ~w;
      }
      const int64_t col = a.col0 + s;
      if (col >= 0) a.bits[(size_t)g * a.bits_cap + col] = ind;
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

cudaError_t launch_sim(const SimArgs &a, int mode, int threads, size_t smem, cudaStream_t s) {
  const int blocks = (a.G + a.gpb - 1) / a.gpb;
  if (blocks == 0 || a.steps == 0) return cudaSuccess;
  if (mode == PBN_PERTURB_PER_NODE) {
    static bool attr = false;
    if (!attr) {
      cudaError_t e = cudaFuncSetAttribute(sim_kernel<PBN_PERTURB_PER_NODE>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, sim_max_smem());
      if (e != cudaSuccess) return e;
      attr = true;
    }
    sim_kernel<PBN_PERTURB_PER_NODE><<<blocks, threads, smem, s>>>(a);
  } else {
    static bool attr = false;
    if (!attr) {
      cudaError_t e = cudaFuncSetAttribute(sim_kernel<PBN_PERTURB_GLOBAL>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, sim_max_smem());
      if (e != cudaSuccess) return e;
      attr = true;
    }
    sim_kernel<PBN_PERTURB_GLOBAL><<<blocks, threads, smem, s>>>(a);
  }
  return cudaGetLastError();
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
