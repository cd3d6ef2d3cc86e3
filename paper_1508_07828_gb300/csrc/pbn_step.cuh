// Device code of the synchronous PBN step shared by the single-task and the
// batched simulation kernels (see pbn_sim.cu for the method).
#pragma once

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

// The same tree with its leaves taken four at a time from the nibble table
// (nib[v] = bits 3, 2, 1, 0 of v as 0 / ~0 masks): one shared load per four
// leaves instead of two shifts per leaf.  The apply kernels of the
// select-ahead schedule keep eval_tt.
template <int K>
__device__ __forceinline__ uint32_t eval_tt_nib(uint32_t tt, const uint32_t *x, const uint4 *nib) {
  if constexpr (K < 2) {
    return eval_tt<K>(tt, x);
  } else {
    constexpr int NL = 1 << K;
    uint32_t v[NL / 2];
#pragma unroll
    for (int j = 0; j < NL / 4; j++) {
      const uint4 nm = nib[(tt >> (4 * j)) & 0xFu];
      v[2 * j] = (x[0] & nm.z) | (~x[0] & nm.w);
      v[2 * j + 1] = (x[0] & nm.x) | (~x[0] & nm.y);
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
__device__ __forceinline__ uint32_t eval_at_depth(uint4 rec, int k, const uint32_t *cur, int gpb, int gl,
                                                 const uint4 *nib) {
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
  return eval_tt_nib<K>(tt, x, nib);
}

// K is warp-uniform, so the switch does not diverge.
__device__ __forceinline__ uint32_t eval_uniform(int K, uint4 rec, int k, const uint32_t *cur, int gpb, int gl,
                                                const uint4 *nib) {
  switch (K) {
    case 0: return eval_at_depth<0>(rec, k, cur, gpb, gl, nib);
    case 1: return eval_at_depth<1>(rec, k, cur, gpb, gl, nib);
    case 2: return eval_at_depth<2>(rec, k, cur, gpb, gl, nib);
    case 3: return eval_at_depth<3>(rec, k, cur, gpb, gl, nib);
    case 4: return eval_at_depth<4>(rec, k, cur, gpb, gl, nib);
    default: return eval_at_depth<5>(rec, k, cur, gpb, gl, nib);
  }
}

// Functions with more than 5 inputs ("wide"): a multiplexer tree would have
// 2^k leaves, so the thread looks the value up chain by chain instead, and
// only for the chains that selected the function (`lanes`): chain q's table
// index gathers bit q of the k parents' state words, and bit q of the result
// is that entry of the table.  Over an item's functions every chain is looked
// up once.
// KMAX: most inputs the variant takes (kWideK, or PBN_MAX_PARENTS in the
// kernels for the sweep's dense class).
template <int KMAX = kWideK>
static __device__ __noinline__ uint32_t eval_wide_lanes(uint4 rec, uint32_t lanes, const uint32_t *cur, int gpb,
                                                        int gl, const uint32_t *wide_tt, const uint16_t *wide_par) {
  const int k = fn_k(rec);
  uint32_t w[KMAX];
#pragma unroll
  for (int m = 0; m < KMAX; m++) w[m] = m < k ? cur[(int)wide_par[rec.z + m] * gpb + gl] : 0u;
  uint32_t out = 0u;
  while (lanes) {
    const int q = __ffs(lanes) - 1;
    lanes &= lanes - 1;
    uint32_t idx = 0u;
#pragma unroll
    for (int m = 0; m < KMAX; m++) idx |= ((w[m] >> q) & 1u) << m;
    out |= ((wide_tt[rec.x + (idx >> 5)] >> (idx & 31u)) & 1u) << q;
  }
  return out;
}

struct ItemCtx {
  const uint4 *fn_s;
  const uint32_t *wide_tt;
  const uint16_t *wide_par;
  int has_wide;
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
  const uint4 *nib;  // nibble v -> its four bits, most significant first, as 0 / ~0 masks (shared memory)
};

// The table ItemCtx::nib points to: one CTA's 16 entries, thread v < 16 fills
// entry v.
__device__ __forceinline__ void fill_nibble_masks(uint4 *nib) {
  if (threadIdx.x < 16) {
    const uint32_t v = threadIdx.x;
    nib[v] = make_uint4(0u - ((v >> 3) & 1u), 0u - ((v >> 2) & 1u), 0u - ((v >> 1) & 1u), 0u - (v & 1u));
  }
}

// Category draw of one item of one transition with LW (warp-uniform)
// category bounds; bound 0 is P32, bound m is T_{m-1}; bounds m >= L are
// unreachable (all lanes below).  On return lt[m] holds the lanes whose
// uniform lies below bound m (complete in every one of the T threads).
// NIB: the bound's four digits of a block come as 0 / ~0 masks from the
// nibble table c.nib (one shared load) instead of being spread bit by bit.
template <int LW, int T, int BPR, bool NIB = false>
__device__ __forceinline__ void draw_below(const RoundKeys &rk, uint32_t P32, const ItemCtx &c, uint32_t (&lt)[LW]) {
  uint32_t ts[LW], und[LW];
#pragma unroll
  for (int m = 0; m < LW; m++) {
    const bool real = m < c.L;
    ts[m] = (m == 0) ? P32 : (real ? c.fn_s[c.f0 + m - 1].y : 0u);
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
      const uint4 R = philox4x32_10(make_uint4((uint32_t)c.i, cy, cz | (b << 24), c.g), rk);
      const uint32_t Rq[4] = {R.x, R.y, R.z, R.w};
#pragma unroll
      for (int m = 0; m < LW; m++) {
        // the bound's digits 4b .. 4b+3 as 0 / ~0
        uint32_t tmq[4];
        if (NIB) {
          const uint4 nm = c.nib[(ts[m] >> (28u - 4u * b)) & 0xFu];
          tmq[0] = nm.x;
          tmq[1] = nm.y;
          tmq[2] = nm.z;
          tmq[3] = nm.w;
        } else {
          const uint32_t tsb = ts[m] << (4u * b);
#pragma unroll
          for (int q = 0; q < 4; q++) tmq[q] = (uint32_t)((int32_t)(tsb << q) >> 31);
        }
#pragma unroll
        for (int q = 0; q < 4; q++) {
          // lanes whose digit differs from the bound's are decided
          const uint32_t tm = tmq[q];
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
}

// Lanes of function j: below bound j+1 and not below bound j.
template <int LW>
__device__ __forceinline__ void select_masks(const uint32_t (&lt)[LW], uint32_t vmask, uint32_t (&sel)[LW]) {
  uint32_t prev = lt[0];
#pragma unroll
  for (int j = 0; j < LW; j++) {
    const uint32_t upto = (j + 1 < LW) ? lt[j + 1] : kFull;
    sel[j] = upto & ~prev & vmask;
    prev = upto;
  }
}

// One item of one transition: category draw, then the selected functions.
// WIDE: compiled with the lookup of functions with more than 5 inputs (used
// when c.has_wide); without it the code is the common path alone.
template <int LW, int MODE, int T, int BPR, bool WIDE, int KMAX = kWideK>
__device__ __forceinline__ void step_item(const RoundKeys &rk, uint32_t P32, const ItemCtx &c) {
  uint32_t lt[LW];
  draw_below<LW, T, BPR, true>(rk, P32, c, lt);
  uint32_t sel[LW];
  select_masks<LW>(lt, c.vmask, sel);
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
    if (WIDE && c.has_wide) {  // kernel-uniform
      const bool wide = k > 5;
      const uint4 tr = wide ? make_uint4(0u, 0u, 0u, 0u) : rec;
      const int kt = wide ? 0 : k;
      const int K = __reduce_max_sync(kFull, (unsigned)kt);
      if (__any_sync(kFull, has && !wide)) fword |= (wide ? 0u : my_sel) & eval_uniform(K, tr, kt, c.cur, c.gpb, c.gl, c.nib);
      if (wide) fword |= eval_wide_lanes<KMAX>(rec, my_sel, c.cur, c.gpb, c.gl, c.wide_tt, c.wide_par);
    } else {
      const int K = __reduce_max_sync(kFull, (unsigned)k);
      if (__any_sync(kFull, has)) fword |= my_sel & eval_uniform(K, rec, k, c.cur, c.gpb, c.gl, c.nib);
    }
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
// line so its register demand does not raise the common path's.  LMAX bounds
// the functions per node: kMaxL in the common kernels, kMaxLAll in the
// variant for networks of the sweep's dense class (a separate kernel, so the
// common kernels' register allocation does not see the wider arrays).
// The variant with more functions per node also takes functions of up to
// PBN_MAX_PARENTS inputs (the common kernels: kWideK).
template <int LMAX>
__host__ __device__ constexpr int kmax_of() { return LMAX > kMaxL ? PBN_MAX_PARENTS : kWideK; }

template <int MODE, int T, int BPR, bool WIDE, int LMAX>
__device__ __noinline__ void step_item_wide(const RoundKeys &rk, uint32_t P32, const ItemCtx &c) {
  step_item<LMAX, MODE, T, BPR, WIDE, kmax_of<LMAX>()>(rk, P32, c);
}

template <int MODE, int T, int BPR, bool WIDE, int LMAX>
__device__ __forceinline__ void dispatch_item(int LW, const RoundKeys &rk, uint32_t P32, const ItemCtx &c) {
  constexpr int K = kmax_of<LMAX>();
  switch (LW) {
    case 0: break;
    case 1: step_item<1, MODE, T, BPR, WIDE, K>(rk, P32, c); break;
    case 2: step_item<2, MODE, T, BPR, WIDE, K>(rk, P32, c); break;
    case 3: step_item<3, MODE, T, BPR, WIDE, K>(rk, P32, c); break;
    case 4: step_item<4, MODE, T, BPR, WIDE, K>(rk, P32, c); break;
    default: step_item_wide<MODE, T, BPR, WIDE, LMAX>(rk, P32, c); break;
  }
}

// Threads per CTA a variant is compiled for: one thread per item may fill
// 1024 threads (64 registers each); shared items run at most 512 threads.
template <int T>
constexpr int max_threads() { return T == 1 ? 1024 : 512; }

// ---- TMA tile staging (bulk copies completing on an mbarrier)

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}

// One bulk copy of `bytes` (a multiple of 16, both addresses 16-byte
// aligned) into shared memory, completing the barrier's current phase.
__device__ __forceinline__ void tile_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for a barrier phase for at most limit_ns nanoseconds.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
  const uint64_t t0 = global_ns();
  while (!mbar_test(bar, parity))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}

constexpr uint64_t kWaitLimitNs = 1000000000ull;  // 1 s: a 24 KB tile arrives in microseconds

// One CTA's work: advance chain groups g0 .. g0+ngl-1 of task `a` by nsteps
// transitions, from transition a.t0 + soff (bitstream column a.col0 + soff).
// `rk` are the task's Philox round keys (kernel parameters in the
// single-task kernel, registers in the batched one).  The groups' words are
// laid out [node][gpb] in shared memory, ngl <= gpb <= a.gpb.
// Function records come from shared memory (whole tables), from TMA tiles
// streamed through two shared buffers (tile u of the launch's sequence
// s*ntiles + t goes to buffer u & 1), or straight from global memory.
template <int MODE, int T, int BPR, bool WIDE, int LMAX = kMaxL>
__device__ __forceinline__ void cta_simulate(const SimArgs &a, const RoundKeys &rk, uint32_t g0, int ngl, int gpb,
                                             unsigned char *smem, int nsteps, int64_t soff) {
  if (ngl <= 0) return;  // CTA-uniform
  const int n = a.n;
  const uint32_t P32 = a.P32;
  const int staging = a.staging;
  const uint4 *fn_s = a.fn;
  const uint32_t *node_s = a.node;
  uint4 *tilebuf[2] = {nullptr, nullptr};
  uint64_t *bar = nullptr;
  size_t off = 0;
  const size_t node_bytes = ((size_t)n * 4 + 15) & ~(size_t)15;
  if (staging == STAGE_SMEM) {
    uint4 *f = reinterpret_cast<uint4 *>(smem);
    for (int j = threadIdx.x; j < a.F; j += blockDim.x) f[j] = a.fn[j];
    off = (size_t)a.F * 16;
    fn_s = f;
  } else if (staging == STAGE_TILES) {
    const size_t tb = ((size_t)a.tile_bytes + 127) & ~(size_t)127;
    tilebuf[0] = reinterpret_cast<uint4 *>(smem);
    tilebuf[1] = reinterpret_cast<uint4 *>(smem + tb);
    off = 2 * tb;
  }
  if (staging != STAGE_GLOBAL) {
    uint32_t *nd = reinterpret_cast<uint32_t *>(smem + off);
    for (int j = threadIdx.x; j < n; j += blockDim.x) nd[j] = a.node[j];
    off += node_bytes;
    node_s = nd;
  }
  if (staging == STAGE_TILES) {
    bar = reinterpret_cast<uint64_t *>(smem + off);
    off += 16;
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
  __shared__ uint4 s_nib[16];
  fill_nibble_masks(s_nib);
  const int ntiles = staging == STAGE_TILES ? a.ntiles : 1;
  const int64_t total_tiles = (int64_t)nsteps * ntiles;
  if (staging == STAGE_TILES && threadIdx.x == 0) {
    mbar_init(&bar[0]);
    mbar_init(&bar[1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // tile u of the sequence into buffer u & 1 (thread 0 only)
  auto issue = [&](int64_t u) {
    const int t = (int)(u % ntiles);
    const int r0 = a.tiles[t], r1 = a.tiles[t + 1];
    const int rec0 = node_f0(node_s[r0]);
    const int rec1 = r1 < n ? node_f0(node_s[r1]) : a.F;
    if (a.test_stall && u == 0) return;  // test hook: this tile never arrives
    tile_load(tilebuf[u & 1], a.fn + rec0, (uint32_t)(rec1 - rec0) * 16u, &bar[u & 1]);
  };
  if (staging == STAGE_TILES && threadIdx.x == 0) {
    issue(0);
    if (total_tiles > 1) issue(1);
  }
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  // lane m's state-of-interest node, read once (a per-lane index into the
  // parameter bank would serialise every step)
  const int my_soi = lane < a.soi_size ? (int)a.soi_node[lane] : 0;
  const bool my_val = (a.soi_val >> lane) & 1u;
  const int my_prop = lane < a.soi_size ? (int)a.soi_prop[lane] : -1;
  const int sub = lane & (T - 1);
  const int slot = threadIdx.x / T;
  const int nslots = blockDim.x / T;
  const int dr = nslots / gpb, dgl = nslots - dr * gpb;
  // valid lanes: every group but the last is full
  const uint32_t last_g = (uint32_t)((a.omega - 1) / 32), last_mask = lane_mask(a.omega, last_g);
  uint32_t *cur = bufA, *nxt = bufB;
  for (int s = 0; s < nsteps; s++) {
    ItemCtx c;
    c.wide_tt = a.wide_tt;
    c.wide_par = a.wide_par;
    c.has_wide = a.has_wide;
    c.cur = cur;
    c.nxt = nxt;
    c.pbuf = pbuf;
    c.anyP = anyP + (s & 1) * gpb;
    c.gpb = gpb;
    c.t = a.t0 + (uint64_t)(soff + s);
    c.sub = sub;
    c.nib = s_nib;
    for (int t = 0; t < ntiles; t++) {
      int p0 = 0, p1 = n;
      c.fn_s = fn_s;
      if (staging == STAGE_TILES) {
        const int64_t u = (int64_t)s * ntiles + t;
        const bool ok = mbar_wait_bounded(&bar[u & 1], (uint32_t)((u >> 1) & 1), kWaitLimitNs);
        if (!__syncthreads_and(ok)) {
          // a tile never arrived: report, let the other buffer's copy land, leave
          if (threadIdx.x == 0) {
            atomicExch(a.status, PBN_ERR_TIMEOUT);
            if (u + 1 < total_tiles) mbar_wait_bounded(&bar[(u + 1) & 1], (uint32_t)(((u + 1) >> 1) & 1), kWaitLimitNs);
          }
          __syncthreads();
          return;
        }
        p0 = a.tiles[t];
        p1 = a.tiles[t + 1];
        c.fn_s = tilebuf[u & 1] - node_f0(node_s[p0]);
      }
      // item q = base + slot is (node position r, group gl) with q = r gpb + gl;
      // (r, gl) advance by (nslots / gpb, nslots % gpb) per round, so no
      // division runs per item
      int r = (p0 * gpb + slot) / gpb;
      int gl = (p0 * gpb + slot) - r * gpb;
      for (int base = p0 * gpb; base < p1 * gpb; base += nslots) {  // uniform trip count
        const int q = base + slot;
        c.gl = gl;
        c.active = (q < p1 * gpb) && (c.gl < ngl);
        const uint32_t rec = c.active ? node_s[r] : 0u;
        c.L = c.active ? node_l(rec) : 0;
        c.i = node_id(rec);
        c.f0 = node_f0(rec);
        c.g = g0 + (uint32_t)c.gl;
        c.vmask = c.active ? (c.g == last_g ? last_mask : kFull) : 0u;
        const int LW = (int)__reduce_max_sync(kFull, (unsigned)c.L);
        dispatch_item<MODE, T, BPR, WIDE, LMAX>(LW, rk, P32, c);
        r += dr;
        gl += dgl;
        if (gl >= gpb) {
          gl -= gpb;
          r++;
        }
      }
      __syncthreads();
      if (staging == STAGE_TILES && threadIdx.x == 0) {
        const int64_t u = (int64_t)s * ntiles + t;
        if (u + 2 < total_tiles) issue(u + 2);
      }
    }
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
      const int64_t col = a.col0 + soff + s;
      for (int gl = warp; gl < ngl; gl += nwarps) {
        uint32_t v = kFull;
        if (lane < a.soi_size) {
          const uint32_t w = nxt[my_soi * gpb + gl];
          v = my_val ? w : ~w;
        }
        // one AND-reduction per property over the lanes of its entries
        for (int m = 0; m < a.n_props; m++) {
          const uint32_t vm = __reduce_and_sync(kFull, my_prop == m ? v : kFull);
          if (lane == 0 && col >= 0)
            a.bits[m * a.prop_stride + (int64_t)(g0 + gl) * a.bits_cap + col] = vm & lane_mask(a.omega, g0 + gl);
        }
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

}  // namespace pbn
