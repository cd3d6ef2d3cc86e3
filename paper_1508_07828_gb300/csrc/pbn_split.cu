// Select-ahead schedule of the synchronous PBN step (Sec. 2.2): the category
// draws of a whole chunk of steps first, the state updates after.
//
// The uniform that picks a node's category at transition t (perturbed, or
// predictor function j) depends on (seed, node, t, chain) only, never on the
// state.  So the draws of every (step, chain group, node) of a chunk of steps
// are independent work: select_kernel spreads them over the whole GPU.  What
// stays sequential is the state update proper, which apply_resident_kernel
// (or apply_kernel for the shapes it does not take) runs with one CTA per
// chain group(s): per step a thread reads its item's category words,
// evaluates the selected truth tables on the parents' words and writes the
// next state; one barrier per step.  When few chain groups exist (a query
// of about a thousand chains) the fused kernel leaves most SMs idle and waits
// on a chain of Philox rounds every step; here the Philox work runs at full
// width and the sequential part is short.
//
// Category words of item (step s, group g, processing position r) at
// planes[(g * S + s) * W + f0_r + w], w < l_r (S = the chunk's steps, f0_r =
// the node's first function record in processing order, W = F rounded up to
// 4 words):
//   w = 0:          lanes perturbed at this node (category 0)
//   w = 1 .. l-1:   lanes that selected function w-1
// The last function's lanes are the valid lanes in none of those words.
// Global perturbation also stores, per (s, g), the OR of all nodes' w = 0
// words in word F of the same run (W = F + 1 rounded up to 4): the chains
// that take s XOR gamma.  A group's words of consecutive steps are one
// contiguous, 16-byte aligned run, so one bulk copy moves several steps of a
// group.
//
// Both kernels compare the same digits against the same bounds as the fused
// kernel (draw_below), so the chains are bit-identical under either schedule.
#include <algorithm>
#include <type_traits>

#include "pbn_step.cuh"

namespace pbn {

namespace {

template <int LW, int MODE, int BPR>
__device__ __forceinline__ void select_item(const RoundKeys &rk, uint32_t P32, const ItemCtx &c, uint32_t *out,
                                            uint32_t *anyw) {
  uint32_t lt[LW];
  draw_below<LW, 1, BPR>(rk, P32, c, lt);
  uint32_t sel[LW];
  select_masks<LW>(lt, c.vmask, sel);
  if (c.L > 0) {
    out[0] = lt[0];
#pragma unroll
    for (int j = 0; j + 1 < LW; j++)
      if (j + 1 < c.L) out[1 + j] = sel[j];
    if (MODE == PBN_PERTURB_GLOBAL && lt[0]) atomicOr(anyw, lt[0]);
  }
}

template <int MODE, int BPR>
__device__ __noinline__ void select_item_wide(const RoundKeys &rk, uint32_t P32, const ItemCtx &c, uint32_t *out,
                                              uint32_t *anyw) {
  select_item<kMaxL, MODE, BPR>(rk, P32, c, out, anyw);
}

}  // namespace

// One thread per (step, group, processing position) of a chunk of a.steps
// steps starting at transition a.t0; position fastest, so a warp's lanes
// mostly share one node shape (processing order groups shapes).
template <int MODE, int BPR>
__global__ void __launch_bounds__(256) select_kernel(const __grid_constant__ SimArgs a) {
  // 32-bit index arithmetic: the launcher keeps steps x G x n below 2^32
  const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t total = (uint32_t)a.steps * (uint32_t)a.G * (uint32_t)a.n;
  const bool active = q < total;
  const uint32_t sg = active ? q / (uint32_t)a.n : 0u;
  const int r = active ? (int)(q - sg * (uint32_t)a.n) : 0;
  const uint32_t su = sg / (uint32_t)a.G;
  const int s = (int)su;
  ItemCtx c;
  c.fn_s = a.fn;
  c.g = sg - su * (uint32_t)a.G;
  const uint32_t rec = active ? a.node[r] : 0u;
  c.L = active ? node_l(rec) : 0;
  c.i = node_id(rec);
  c.f0 = node_f0(rec);
  c.vmask = active ? lane_mask(a.omega, c.g) : 0u;
  c.t = a.t0 + (uint64_t)s;
  c.sub = 0;
  const int64_t run = (int64_t)c.g * a.steps + s;  // group-major: a group's steps are contiguous
  uint32_t *out = a.planes + run * a.W + c.f0;
  uint32_t *anyw = a.planes + run * a.W + a.F;
  switch ((int)__reduce_max_sync(kFull, (unsigned)c.L)) {
    case 0: break;
    case 1: select_item<1, MODE, BPR>(a.rk, a.P32, c, out, anyw); break;
    case 2: select_item<2, MODE, BPR>(a.rk, a.P32, c, out, anyw); break;
    case 3: select_item<3, MODE, BPR>(a.rk, a.P32, c, out, anyw); break;
    case 4: select_item<4, MODE, BPR>(a.rk, a.P32, c, out, anyw); break;
    default: select_item_wide<MODE, BPR>(a.rk, a.P32, c, out, anyw); break;
  }
}

namespace {

__device__ __forceinline__ void copy16_async(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(__cvta_generic_to_global(src))
               : "memory");
}

__device__ __forceinline__ void async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

}  // namespace

// Indicator words of the last kIndRing steps per group (register-resident
// path): the threads of the state-of-interest nodes AND their part into the
// word of their step; the producer warp stores them 32 steps at a time.
constexpr int kIndRing = 64;

// Ring slots of category words: RING - 1 steps are in flight ahead of the
// step being applied (8, or 3 when 8 slots do not fit shared memory).
size_t apply_smem_bytes(int n, int F, int gpb, int W, int staging, int ring, int n_props) {
  size_t b = (size_t)ring * gpb * W * 4;  // category words ring
  if (staging == STAGE_SMEM) b += (size_t)F * 16;
  b += ((size_t)n * 4 + 15) & ~(size_t)15;                 // node records
  b += 2 * (size_t)n * gpb * 4;                            // current and next state
  b += (size_t)std::max(n_props, 1) * gpb * kIndRing * 4;  // indicator words of recent steps
  return b;
}

// Truth table of a k-input function as a 5-input one: its 2^k bits repeated
// up to 32 leaves, so inputs k..4 (node 0 in the record) select between equal
// halves.  Every function is then evaluated at depth 5: no per-warp depth.
__device__ __forceinline__ uint32_t replicate5(uint32_t tt, int k) {
#pragma unroll
  for (int e = 0; e < 5; e++)
    if (e >= k) tt |= tt << (1 << e);
  return tt;
}

// T threads share one depth-5 multiplexer tree: thread `sub` evaluates the
// subtree of leaves [sub * 32/T, (sub+1) * 32/T) over inputs x0 .. x(D-1),
// D = 5 - log2 T; then log2 T exchange levels, level m selecting on input
// x(D+m) between the halves held by threads that differ in bit m of sub.
template <int T>
struct TreeSplit {
  static constexpr int LT = T == 4 ? 2 : (T == 2 ? 1 : 0);  // exchange levels
  static constexpr int D = 5 - LT;                          // depth of a thread's subtree
};

template <int T>
__device__ __forceinline__ uint32_t merge_shared(uint32_t v, const uint32_t (&x)[5], int sub) {
  constexpr int D = TreeSplit<T>::D;
#pragma unroll
  for (int m = 0; m < TreeSplit<T>::LT; m++) {
    const uint32_t o = __shfl_xor_sync(kFull, v, 1 << m);
    const bool upper = (sub >> m) & 1;
    const uint32_t lo = upper ? o : v, hi = upper ? v : o;
    v = (x[D + m] & hi) | (~x[D + m] & lo);
  }
  return v;
}

template <int T>
__device__ __forceinline__ uint32_t eval5_shared(uint32_t tt5, const uint32_t (&x)[5], int sub) {
  constexpr int D = TreeSplit<T>::D;
  return merge_shared<T>(eval_tt<D>(tt5 >> (sub << D), x), x, sub);
}

// The first kResident functions of a thread's item, decoded once per launch:
// the thread's leaves as pairs (leaf 2q as 0 / ~0, and its XOR with leaf
// 2q+1, so the first tree level is one operation per pair) and the parents'
// offsets in the state buffers.  A step then reads five words and runs the
// remaining tree levels and exchanges.
constexpr int kResident = 2;

template <int T>
struct ResidentItem {
  static constexpr int NP = 16 / T;  // leaf pairs per thread
  uint32_t lo[kResident][NP], dx[kResident][NP];
  int off[kResident][5];

  __device__ __forceinline__ void load(int c, const uint4 &fr, bool replicated, int gpb, int gl, int sub) {
    const uint32_t tt5 = replicated ? fr.x : replicate5(fr.x, fn_k(fr));
    const uint32_t chunk = tt5 >> (sub * (32 / T));
#pragma unroll
    for (int q = 0; q < NP; q++) {
      lo[c][q] = sext_bit(chunk, 2 * q);
      dx[c][q] = lo[c][q] ^ sext_bit(chunk, 2 * q + 1);
    }
    const int pr[5] = {(int)(fr.z & 0xFFF), (int)((fr.z >> 12) & 0xFFF), (int)(fr.w & 0xFFF),
                       (int)((fr.w >> 12) & 0xFFF), (int)((fr.z >> 24) | (((fr.w >> 24) & 0xFu) << 8))};
#pragma unroll
    for (int m = 0; m < 5; m++) off[c][m] = pr[m] * gpb + gl;
  }

  __device__ __forceinline__ void clear(int c) {
#pragma unroll
    for (int q = 0; q < NP; q++) lo[c][q] = dx[c][q] = 0u;
#pragma unroll
    for (int m = 0; m < 5; m++) off[c][m] = 0;
  }

  __device__ __forceinline__ uint32_t eval(int c, const uint32_t *cur, int sub) const {
    uint32_t x[5];
#pragma unroll
    for (int m = 0; m < 5; m++) x[m] = cur[off[c][m]];
    uint32_t v[NP];
#pragma unroll
    for (int q = 0; q < NP; q++) v[q] = lo[c][q] ^ (x[0] & dx[c][q]);
#pragma unroll
    for (int m = 1; m < TreeSplit<T>::D; m++) {
#pragma unroll
      for (int q = 0; q < (NP >> m); q++) v[q] = (x[m] & v[2 * q + 1]) | (~x[m] & v[2 * q]);
    }
    return merge_shared<T>(v[0], x, sub);
  }
};

// Threads per CTA an apply variant is compiled for: with one or two threads
// per item a thread keeps 32 or 16 leaves per function in registers, so those
// variants get 128 registers per thread (512 threads); four threads, 64.
template <int T>
constexpr int apply_max_threads() { return T == 4 ? 1024 : 512; }

int apply_threads_limit(int T) { return T == 4 ? apply_max_threads<4>() : apply_max_threads<1>(); }

// One CTA per `gpb` chain groups applies a.steps steps of category words;
// T threads per (node, group) item.
template <int MODE, int kRing, int T, bool WIDE>
__global__ void __launch_bounds__(apply_max_threads<T>(), 1) apply_kernel(const __grid_constant__ SimArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int gpb = a.gpb, n = a.n, W = a.W;
  const uint32_t g0 = blockIdx.x * (uint32_t)gpb;
  const int ngl = min(gpb, a.G - (int)g0);
  uint32_t *ring = reinterpret_cast<uint32_t *>(smem);
  unsigned char *p = reinterpret_cast<unsigned char *>(ring + (size_t)kRing * gpb * W);
  const uint4 *fn_s = a.fn;
  const bool tt_replicated = a.staging == STAGE_SMEM;
  if (tt_replicated) {
    // the shared copy carries every truth table already replicated to 32
    // leaves (wide records keep their table offset)
    uint4 *f = reinterpret_cast<uint4 *>(p);
    for (int j = threadIdx.x; j < a.F; j += blockDim.x) {
      uint4 r = a.fn[j];
      if (fn_k(r) <= 5) r.x = replicate5(r.x, fn_k(r));
      f[j] = r;
    }
    fn_s = f;
    p += (size_t)a.F * 16;
  }
  uint32_t *node_s = reinterpret_cast<uint32_t *>(p);
  for (int j = threadIdx.x; j < n; j += blockDim.x) node_s[j] = a.node[j];
  p += ((size_t)n * 4 + 15) & ~(size_t)15;
  const int items = n * gpb;
  uint32_t *cur = reinterpret_cast<uint32_t *>(p);
  uint32_t *nxt = cur + items;
  uint32_t *ind = nxt + items;  // [n_props][gpb][kIndRing]
  for (int idx = threadIdx.x; idx < items; idx += blockDim.x) {
    const int i = idx / gpb, gl = idx - i * gpb;
    cur[idx] = gl < ngl ? a.state[(size_t)(g0 + gl) * n + i] : 0u;
  }
  for (int j = threadIdx.x; j < max(a.n_props, 1) * gpb * kIndRing; j += blockDim.x) ind[j] = kFull;
  __syncthreads();  // tables and state staged before any thread reads another's records
  // step s's words of this CTA's groups: ngl runs of W words (group-major
  // layout), copied 16 bytes at a time into slot s % kRing
  const int w16 = W / 4, chunks16 = ngl * w16;
  auto chunk_src = [&](int s, int j) {
    const int gl = j / w16;
    return a.planes + ((size_t)(g0 + gl) * a.steps + s) * W + 4 * (j - gl * w16);
  };
  auto issue = [&](int s) {
    if (s < a.steps) {
      uint32_t *dst = ring + (size_t)(s % kRing) * gpb * W;
      for (int j = threadIdx.x; j < chunks16; j += blockDim.x) copy16_async(dst + 4 * j, chunk_src(s, j));
    }
    async_commit();  // one group per step, empty past the end, so the wait count stays uniform
  };
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  // lane m's state-of-interest node, read once (a per-lane index into the
  // parameter bank would serialise every step)
  const int my_soi = lane < a.soi_size ? (int)a.soi_node[lane] : 0;
  const bool my_val = (a.soi_val >> lane) & 1u;
  const int my_prop = lane < a.soi_size ? (int)a.soi_prop[lane] : -1;
  // indicators of the properties after step s (state in `st`)
  auto indicator = [&](const uint32_t *st, int s) {
    if (a.soi_size == 0) return;
    const int64_t col = a.col0 + s;
    for (int gl = nwarps - 1 - warp; gl < ngl; gl += nwarps) {
      uint32_t v = kFull;
      if (lane < a.soi_size) {
        const uint32_t w = st[my_soi * gpb + gl];
        v = my_val ? w : ~w;
      }
      for (int m = 0; m < a.n_props; m++) {
        const uint32_t vm = __reduce_and_sync(kFull, my_prop == m ? v : kFull);
        if (lane == 0 && col >= 0)
          a.bits[m * a.prop_stride + (int64_t)(g0 + gl) * a.bits_cap + col] = vm & lane_mask(a.omega, g0 + gl);
      }
    }
  };
  // start of step s: its words landed and visible, the state after step s-1
  // complete; its indicator written, and the words of step s + kRing - 1
  // requested into the slot step s-1 used
  auto step_top = [&](int s) {
    async_wait<kRing - 2>();
    __syncthreads();
    if (s > 0) indicator(cur, s - 1);
    issue(s + kRing - 1);
  };
  // functions j >= first of an item, decoded from the records every step
  auto eval_rest = [&](int first, int LW, int L, int f0, int gl, int sub, const uint32_t *w, uint32_t &rest,
                       uint32_t &fword) {
#pragma unroll 1
    for (int j = first; j < LW; j++) {
      uint32_t sel = 0u;
      if (j + 1 < L) sel = w[1 + j];
      else if (j + 1 == L) sel = rest;
      rest &= ~sel;
      const bool has = sel != 0u;  // the same in the T threads of an item
      if (__any_sync(kFull, has)) {
        uint4 fr = has ? fn_s[f0 + j] : make_uint4(0u, 0u, 0u, 0u);
        bool wide = false;
        if (WIDE && a.has_wide) {  // kernel-uniform (wide networks run T = 1)
          wide = fn_k(fr) > 5;
          if (wide) {
            fword |= eval_wide_lanes(fr, sel, cur, gpb, gl, a.wide_tt, a.wide_par);
            fr = make_uint4(0u, 0u, 0u, 0u);
          }
        }
        const int pr[5] = {(int)(fr.z & 0xFFF), (int)((fr.z >> 12) & 0xFFF), (int)(fr.w & 0xFFF),
                           (int)((fr.w >> 12) & 0xFFF), (int)((fr.z >> 24) | (((fr.w >> 24) & 0xFu) << 8))};
        uint32_t x[5];
#pragma unroll
        for (int m = 0; m < 5; m++) x[m] = cur[pr[m] * gpb + gl];
        const uint32_t tt5 = tt_replicated ? fr.x : replicate5(fr.x, fn_k(fr));
        const uint32_t v = eval5_shared<T>(tt5, x, sub);
        if (!wide) fword |= sel & v;
      }
    }
  };
  // slot: the step's words of this CTA's groups (word F of a group's run is
  // the OR of its perturbed lanes under global perturbation)
  auto finish = [&](int idx, int gl, uint32_t P, uint32_t fword, const uint32_t *slot) -> uint32_t {
    uint32_t v;
    if (MODE == PBN_PERTURB_PER_NODE) {
      v = (P & ~cur[idx]) | fword;
    } else {
      const uint32_t any = slot[gl * W + a.F];
      v = (any & (cur[idx] ^ P)) | (~any & fword);
    }
    nxt[idx] = v;
    return v;
  };
  if (T > 1 && !WIDE && items * T <= (int)blockDim.x - 32) {
    // One item per T (2 or 4) threads for the whole launch (one thread per
    // item runs in apply_resident_kernel), everything that does not change
    // from step to step in registers; the last warp is the producer:
    // it waits for the category words, writes the indicator and requests the
    // words of later steps, so the item warps only compute between barriers.
    const bool producer = warp == nwarps - 1;
    const int it = threadIdx.x / T, sub = threadIdx.x & (T - 1);
    const int r = it / gpb, gl = it - r * gpb;
    const bool active = !producer && it < items && gl < ngl;
    const uint32_t rec = active ? node_s[r] : 0u;
    const int L = active ? node_l(rec) : 0;
    const int f0 = node_f0(rec);
    const int idx = node_id(rec) * gpb + gl;
    const uint32_t vmask = active ? lane_mask(a.omega, g0 + gl) : 0u;
    const int LW = (int)__reduce_max_sync(kFull, (unsigned)L);
    const int woff = active ? gl * W + f0 : 0;
    const int slot_words = gpb * W;
    ResidentItem<T> R;
#pragma unroll
    for (int c = 0; c < kResident; c++) {
      if (c < L) R.load(c, fn_s[f0 + c], tt_replicated, gpb, gl, sub);
      else R.clear(c);
    }
    auto issue_warp = [&](int s) {
      if (s < a.steps) {
        uint32_t *dst = ring + (size_t)(s % kRing) * slot_words;
        for (int j = lane; j < chunks16; j += 32) copy16_async(dst + 4 * j, chunk_src(s, j));
      }
      async_commit();
    };
    // this item's part of the state of interest: the node must be 1 (need1)
    // and/or 0 (need0; both when the state of interest names it twice)
    // bit m: property m needs the node at 1 (need1) and/or at 0 (need0; both
    // when a property names it twice)
    uint32_t need1 = 0u, need0 = 0u;
    if (active && sub == 0)
      for (int e = 0; e < a.soi_size; e++)
        if ((int)a.soi_node[e] == node_id(rec)) {
          const uint32_t bit = 1u << a.soi_prop[e];
          if ((a.soi_val >> e) & 1u) need1 |= bit;
          else need0 |= bit;
        }
    const uint32_t in_props = need1 | need0;
    // store the indicator words of steps s0 .. s0+cnt-1 (complete) and make
    // their ring words ready for reuse
    auto flush = [&](int s0, int cnt) {
      if (a.soi_size == 0) return;
      for (int m = 0; m < a.n_props; m++)
        for (int g = 0; g < ngl; g++) {
          const int st = s0 + lane;
          if (lane < cnt) {
            uint32_t *word = ind + (m * gpb + g) * kIndRing + (st & (kIndRing - 1));
            const int64_t col = a.col0 + st;
            if (col >= 0)
              a.bits[m * a.prop_stride + (int64_t)(g0 + g) * a.bits_cap + col] = *word & lane_mask(a.omega, g0 + g);
            *word = kFull;
          }
        }
    };
    if (producer)
      for (int s = 0; s < kRing - 1; s++) issue_warp(s);
    int ring_slot = 0;
    for (int s = 0; s < a.steps; s++) {
      if (producer) async_wait<kRing - 2>();
      __syncthreads();
      if (producer) {
        if (s > 0 && (s & 31) == 0) flush(s - 32, 32);  // steps s-32 .. s-1 are complete
        issue_warp(s + kRing - 1);
      } else {
        const uint32_t *w = ring + ring_slot * slot_words + woff;
        const uint32_t P = active ? w[0] : 0u;
        uint32_t rest = vmask & ~P;
        uint32_t sel = L > 1 ? w[1] : (L == 1 ? rest : 0u);
        rest &= ~sel;
        uint32_t fword = sel & R.eval(0, cur, sub);
        if (LW > 1) {
          sel = L > 2 ? w[2] : (L == 2 ? rest : 0u);
          rest &= ~sel;
          fword |= sel & R.eval(1, cur, sub);
          if (LW > kResident) eval_rest(kResident, LW, L, f0, gl, sub, w, rest, fword);
        }
        if (active && sub == 0) {
          const uint32_t v = finish(idx, gl, P, fword, ring + ring_slot * slot_words);
          for (uint32_t props = in_props; props; props &= props - 1) {
            const int m = __ffs(props) - 1;
            const uint32_t term = ((need1 >> m) & 1u ? v : kFull) & ((need0 >> m) & 1u ? ~v : kFull);
            atomicAnd(ind + (m * gpb + gl) * kIndRing + (s & (kIndRing - 1)), term);
          }
        }
      }
      ring_slot = ring_slot + 1 == kRing ? 0 : ring_slot + 1;
      uint32_t *tmp = cur;
      cur = nxt;
      nxt = tmp;
    }
    if (producer) async_wait<0>();
    __syncthreads();
    if (producer) {
      const int done = ((a.steps - 1) >> 5) << 5;  // steps already stored
      flush(done, a.steps - done);
    }
  } else {
    const int dit = (int)blockDim.x / T, dr = dit / gpb, dgl = dit - dr * gpb;
    for (int s = 0; s < kRing - 1; s++) issue(s);
    for (int s = 0; s < a.steps; s++) {
      step_top(s);
      const uint32_t *slot = ring + (size_t)(s % kRing) * gpb * W;
      // item it = r gpb + gl of thread q = it T + sub; (r, gl) advance by the
      // CTA's items per round without a division per item
      int r = (int)(threadIdx.x / T) / gpb, gl = (int)(threadIdx.x / T) - r * gpb;
      for (int base = 0; base < items * T; base += blockDim.x) {  // uniform trip count
        const int q = base + threadIdx.x;
        const int it = q / T, sub = q & (T - 1);
        const bool active = it < items && gl < ngl;
        const uint32_t rec = active ? node_s[r] : 0u;
        const int L = active ? node_l(rec) : 0;
        const int f0 = node_f0(rec);
        const uint32_t *w = slot + gl * W + f0;
        const uint32_t P = active ? w[0] : 0u;
        uint32_t rest = (active ? lane_mask(a.omega, g0 + gl) : 0u) & ~P;
        const int LW = (int)__reduce_max_sync(kFull, (unsigned)L);
        uint32_t fword = 0u;
        eval_rest(0, LW, L, f0, gl, sub, w, rest, fword);
        if (active && sub == 0) finish(node_id(rec) * gpb + gl, gl, P, fword, slot);
        r += dr;
        gl += dgl;
        if (gl >= gpb) {
          gl -= gpb;
          r++;
        }
      }
      uint32_t *tmp = cur;
      cur = nxt;
      nxt = tmp;
    }
    async_wait<0>();
    __syncthreads();
    indicator(cur, a.steps - 1);
  }
  for (int idx = threadIdx.x; idx < items; idx += blockDim.x) {
    const int i = idx / gpb, gl = idx - i * gpb;
    if (gl < ngl) a.state[(size_t)(g0 + gl) * n + i] = cur[idx];
  }
}

// ---------------------------------------------------------------------------
// Register-resident apply: two threads per (node, group) item, one per
// function slot.
//
// Thread 2i+f holds function f (f = 0, 1) of item i, decoded once per launch:
// its truth table as leaf pairs in registers (leaf 2q as 0 / ~0 and its XOR
// with leaf 2q+1) and the shared-memory addresses of its parents' state
// words.  A step then reads five parent words and runs one depth-5
// multiplexer tree (tables are replicated to 32 leaves, so inputs k..4 select
// between equal halves); each thread masks its value with the lanes that
// selected its function(s) and one shuffle ORs the pair.  Every tree has
// depth 5: warps of equal work keep the per-step barrier short (measured on
// GB300: a loop per warp-uniform depth runs fewer instructions but the
// deepest warps then set every step, and the step got longer).  Functions j >= 2
// (nodes with more than two) are decoded from their records every step,
// thread f taking those with j = f mod 2.  Two threads per item give every
// scheduler two or more warps of equal work, so the dependent levels of one
// warp's trees overlap with another's.
//
// Feeding: a group's category words of kCopySteps consecutive steps are one
// contiguous run (group-major layout), so one thread of the last warp (the
// producer) moves a chunk of kCopySteps = 8 steps with one bulk copy
// (cp.async.bulk) per group of the CTA into a ring slot, completing the slot's
// mbarrier.  At the first step of chunk c it refills the slot chunk c-1 used;
// at the last step of chunk c it waits for chunk c+1's words, so the barrier
// that ends that step also publishes them.  Copy and wait, whose latency the
// barrier of that step pays, come once per 8 steps; the item threads never
// wait on an mbarrier.
// The wait is bounded (1 s): if it gives up, the producer records
// PBN_ERR_TIMEOUT in the device status word, issues nothing more and lets the
// launch run to its end (the results are then invalid and the status says
// so); before the CTA leaves it waits (bounded) for every copy it issued.
//
// The two state buffers sit at fixed shared offsets (kResStride words apart)
// so a step's loads and store are register + immediate addresses, with the
// step loop unrolled by two.

namespace {

constexpr int kResStride = 512;  // words between the two state buffers
constexpr int kCopyLog = 3;                 // log2 of the steps of category words per bulk copy
constexpr int kCopySteps = 1 << kCopyLog;
constexpr int kRingLogMax = 4;              // at most 16 steps in flight

__device__ __forceinline__ uint32_t lds_u32(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
  return v;
}

template <int OFF>
__device__ __forceinline__ uint32_t lds_u32_at(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1 + %2];" : "=r"(v) : "r"(addr), "n"(OFF));
  return v;
}

template <int OFF>
__device__ __forceinline__ void sts_u32_at(uint32_t addr, uint32_t v) {
  asm volatile("st.shared.u32 [%0 + %1], %2;" ::"r"(addr), "n"(OFF), "r"(v) : "memory");
}

__device__ __forceinline__ void atom_and_shared(uint32_t addr, uint32_t v) {
  asm volatile("atom.shared.and.b32 _, [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// Three-input bitwise function with truth table LUT over (a, b, c) = (0xF0,
// 0xCC, 0xAA): one instruction for a multiplexer level.
template <int LUT>
__device__ __forceinline__ uint32_t lop3(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(LUT));
  return d;
}

// CTA-wide barrier in its non-aligned form: the producer warp and the item
// warps reach it from different loops.
__device__ __forceinline__ void cta_barrier() { asm volatile("barrier.sync 0;" ::: "memory"); }

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for a phase of an mbarrier for at most kWaitLimitNs.
__device__ __noinline__ bool mbar_wait_slow(uint32_t bar, uint32_t parity) {
  const uint64_t t0 = global_ns();
  while (!mbar_try(bar, parity))
    if (global_ns() - t0 > kWaitLimitNs) return false;
  return true;
}

__device__ __forceinline__ bool mbar_wait_fast(uint32_t bar, uint32_t parity) {
  return mbar_try(bar, parity) || mbar_wait_slow(bar, parity);
}

// The slot's mbarrier expects `bytes` from the copies that follow (this
// arrival completes the phase once they have landed).
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// One bulk copy global -> shared (16-byte aligned, size a multiple of 16)
// completing its bytes on the mbarrier.
__device__ __forceinline__ void bulk_copy_to(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// One function of an item, decoded once per launch.
struct ResidentFn {
  uint32_t lo[16], dx[16];
  uint32_t par[5];  // shared addresses of the parents' words in state buffer 0

  __device__ __forceinline__ void load(uint4 fr, uint32_t st0, int gpb, int gl) {
    const uint32_t tt5 = replicate5(fr.x, fn_k(fr));
#pragma unroll
    for (int q = 0; q < 16; q++) {
      lo[q] = sext_bit(tt5, 2 * q);
      dx[q] = lo[q] ^ sext_bit(tt5, 2 * q + 1);
    }
    const int pr[5] = {(int)(fr.z & 0xFFF), (int)((fr.z >> 12) & 0xFFF), (int)(fr.w & 0xFFF),
                       (int)((fr.w >> 12) & 0xFFF), (int)((fr.z >> 24) | (((fr.w >> 24) & 0xFu) << 8))};
#pragma unroll
    for (int m = 0; m < 5; m++) par[m] = st0 + 4u * (uint32_t)(pr[m] * gpb + gl);
  }

  __device__ __forceinline__ void clear(uint32_t st0) {
#pragma unroll
    for (int q = 0; q < 16; q++) lo[q] = dx[q] = 0u;
#pragma unroll
    for (int m = 0; m < 5; m++) par[m] = st0;
  }

  // subtree of level M over leaf pairs [Q, Q + 2^(M-1)), depth first so few
  // partial results are live at once
  template <int M, int Q>
  __device__ __forceinline__ uint32_t sub(const uint32_t (&x)[5]) const {
    if constexpr (M == 1) {
      return lop3<0x6A>(x[0], dx[Q], lo[Q]);  // lo ^ (x0 & dx)
    } else {
      const uint32_t a = sub<M - 1, Q>(x), b = sub<M - 1, Q + (1 << (M - 2))>(x);
      return lop3<0xCA>(x[M - 1], b, a);  // x ? b : a, bitwise
    }
  }

  // the function on state buffer OFF (byte offset of the buffer)
  template <int OFF>
  __device__ __forceinline__ uint32_t eval() const {
    uint32_t x[5];
#pragma unroll
    for (int m = 0; m < 5; m++) x[m] = lds_u32_at<OFF>(par[m]);
    return sub<5, 0>(x);
  }
};

// Depth-first multiplexer tree of a truth table replicated to 32 leaves:
// subtree of level M over leaves [Q, Q + 2^M).
template <int M, int Q>
__device__ __forceinline__ uint32_t tt_subtree(uint32_t tt5, const uint32_t (&x)[5]) {
  if constexpr (M == 0) {
    return sext_bit(tt5, Q);
  } else {
    const uint32_t a = tt_subtree<M - 1, Q>(tt5, x), b = tt_subtree<M - 1, Q + (1 << (M - 1))>(tt5, x);
    return (x[M - 1] & b) | (~x[M - 1] & a);
  }
}

// An item of a node with more than two functions (LW > 2, warp-uniform):
// this thread's functions j = f, f+2, ... < LW, the resident one (value v)
// first, further ones decoded from their records; the lanes of function
// j < L-1 are category word 1+j, the last function's are the lanes in none of
// them.
__device__ __forceinline__ uint32_t rest_part(uint32_t w, int L, int LW, int f, uint32_t rest, uint32_t v,
                                              uint32_t cur, const uint4 *fn, int f0, int gpb, int gl) {
  uint32_t taken = 0u;
  for (int j = 0; j + 1 < L; j++) taken |= lds_u32(w + 4u * (uint32_t)(1 + j));
  auto lanes_of = [&](int j) -> uint32_t {
    if (j + 1 < L) return lds_u32(w + 4u * (uint32_t)(1 + j));
    return j + 1 == L ? rest & ~taken : 0u;
  };
  uint32_t part = lanes_of(f) & v;
  // the same trip count in every lane (the warp votes in each round)
#pragma unroll 1
  for (int jb = 2; jb < LW; jb += 2) {
    const int j = jb + f;
    const uint32_t sel = j < L ? lanes_of(j) : 0u;
    const bool has = sel != 0u;
    if (__any_sync(kFull, has)) {
      const uint4 fr = has ? fn[f0 + j] : make_uint4(0u, 0u, 0u, 0u);
      const int pr[5] = {(int)(fr.z & 0xFFF), (int)((fr.z >> 12) & 0xFFF), (int)(fr.w & 0xFFF),
                         (int)((fr.w >> 12) & 0xFFF), (int)((fr.z >> 24) | (((fr.w >> 24) & 0xFu) << 8))};
      uint32_t x[5];
#pragma unroll
      for (int m = 0; m < 5; m++) x[m] = lds_u32(cur + 4u * (uint32_t)(pr[m] * gpb + gl));
      part |= sel & tt_subtree<5, 0>(replicate5(fr.x, fn_k(fr)), x);
    }
  }
  return part;
}

}  // namespace

// ring: steps in flight (16), in slots of kCopySteps steps each
size_t apply_resident_smem_bytes(int gpb, int W, int ring, int n_props) {
  size_t b = (size_t)2 * kResStride * 4;                     // state buffers
  b += (size_t)ring * gpb * W * 4;                           // category words ring (16-byte slots)
  b += (size_t)(ring / kCopySteps) * 8;                      // one mbarrier per slot
  b += (size_t)std::max(n_props, 1) * gpb * kIndRing * 4;    // indicator words of recent steps
  return b;
}

// REST: compiled with the path of nodes with more than two functions (a
// network whose nodes have at most two runs the variant without it).
template <int MODE, bool REST>
__global__ void __launch_bounds__(2 * kResidentItems + 32, 1) apply_resident_kernel(const __grid_constant__ SimArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int gpb = a.gpb, n = a.n, W = a.W;
  const uint32_t g0 = blockIdx.x * (uint32_t)gpb;
  const int ngl = min(gpb, a.G - (int)g0);
  constexpr int K = kCopySteps;
  const int nslot = (1 << a.ring_log2) / K, smask = nslot - 1, slog = a.ring_log2 - kCopyLog;
  const int slot_words = gpb * K * W;                          // [gl][K steps][W]
  uint32_t *st = reinterpret_cast<uint32_t *>(smem);          // [2][kResStride]
  uint32_t *ringp = st + 2 * kResStride;                      // [nslot][slot_words]
  uint64_t *full = reinterpret_cast<uint64_t *>(ringp + (size_t)nslot * slot_words);
  uint32_t *ind = reinterpret_cast<uint32_t *>(full + nslot);  // [n_props][gpb][kIndRing]
  const int n_ind = max(a.n_props, 1) * gpb * kIndRing;
  const int items = n * gpb;
  for (int idx = threadIdx.x; idx < items; idx += blockDim.x) {
    const int i = idx / gpb, gl = idx - i * gpb;
    st[idx] = gl < ngl ? a.state[(size_t)(g0 + gl) * n + i] : 0u;
  }
  for (int j = threadIdx.x; j < n_ind; j += blockDim.x) ind[j] = kFull;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool producer = warp == (int)(blockDim.x >> 5) - 1;
  const uint32_t full0 = smem_u32(full), ring0 = smem_u32(ringp);
  const uint32_t slot_bytes = (uint32_t)slot_words * 4u;
  const int nchunks = (a.steps + K - 1) / K;  // copies of K steps (the last may be shorter)
  if (threadIdx.x == 0) {
    for (int j = 0; j < nslot; j++) mbar_init(full + j);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  cta_barrier();  // tables, state and barriers ready
  if (producer) {
    // thread 0 of the warp: chunks of K steps issued (0 .. issued-1) and
    // confirmed (0 .. waited-1); `dead` once a wait gave up.  Chunk c is one
    // bulk copy per group of the CTA into slot c % nslot, all completing the
    // slot's mbarrier.
    int issued = 0, waited = 0;
    bool dead = false;
    auto issue = [&](int c) {
      const int slot = c & smask;
      const int kc = min(K, a.steps - c * K);
      const uint32_t bar = full0 + 8u * slot, bytes = (uint32_t)(kc * W) * 4u;
      mbar_expect_tx(bar, bytes * (uint32_t)ngl);
      for (int gl = 0; gl < ngl; gl++)
        bulk_copy_to(ring0 + (uint32_t)slot * slot_bytes + (uint32_t)(gl * K * W) * 4u,
                     a.planes + ((size_t)(g0 + gl) * a.steps + (size_t)c * K) * W, bytes, bar);
      issued = c + 1;
    };
    auto wait_chunk = [&](int c) {
      if (dead) return;
      if (!mbar_wait_fast(full0 + 8u * (c & smask), (uint32_t)((c >> slog) & 1))) {
        atomicExch(a.status, PBN_ERR_TIMEOUT);
        dead = true;
        return;
      }
      waited = c + 1;
    };
    // the warp stores the indicator words of steps s0 .. s0+cnt-1 (complete)
    // and makes their ring words ready for reuse
    auto flush = [&](int s0, int cnt) {
      if (a.soi_size == 0) return;
      for (int m = 0; m < a.n_props; m++)
        for (int g = 0; g < ngl; g++) {
          const int sl = s0 + lane;
          if (lane < cnt) {
            uint32_t *word = ind + (m * gpb + g) * kIndRing + (sl & (kIndRing - 1));
            const int64_t col = a.col0 + sl;
            if (col >= 0)
              a.bits[m * a.prop_stride + (int64_t)(g0 + g) * a.bits_cap + col] = *word & lane_mask(a.omega, g0 + g);
            *word = kFull;
          }
        }
    };
    if (lane == 0) {
      for (int c = 0; c < min(nslot, nchunks); c++)
        if (!(a.test_stall && c == 0)) issue(c);  // test hook: the first chunk never arrives
      wait_chunk(0);
    }
    cta_barrier();  // the words of chunk 0 landed
    for (int s = 0; s < a.steps; s++) {
      if (lane == 0) {
        const int c = s / K;
        // first step of chunk c: refill the slot chunk c-1 used (its steps are done)
        if (s % K == 0 && c >= 1 && !dead && c - 1 + nslot < nchunks) issue(c - 1 + nslot);
        // last step of chunk c: the words of chunk c+1 must land before this step's barrier
        if (s % K == K - 1 && c + 1 < nchunks) wait_chunk(c + 1);
      }
      __syncwarp();
      if (s > 0 && (s & 31) == 0) flush(s - 32, 32);  // steps s-32 .. s-1 are complete
      cta_barrier();  // state after step s complete; the words of step s+1 landed
    }
    const int done = ((a.steps - 1) >> 5) << 5;  // steps already stored
    flush(done, a.steps - done);
    // every issued copy has landed before the CTA's shared memory goes away
    if (lane == 0)
      for (int c = waited; c < issued; c++)
        if (!mbar_wait_fast(full0 + 8u * (c & smask), (uint32_t)((c >> slog) & 1))) {
          atomicExch(a.status, PBN_ERR_TIMEOUT);
          break;
        }
    return;
  }
  // this thread: function slot f of item it
  const int it = threadIdx.x >> 1, f = threadIdx.x & 1;
  const int r = it / gpb, gl = it - r * gpb;
  const bool active = it < items && gl < ngl;
  const uint32_t rec = active ? a.node[r] : 0u;
  const int L = active ? node_l(rec) : 0;
  const int f0 = node_f0(rec);
  const int idx = node_id(rec) * gpb + gl;
  const uint32_t vmask = active ? lane_mask(a.omega, g0 + gl) : 0u;
  const uint32_t st0 = smem_u32(st);
  const uint32_t own = st0 + 4u * (uint32_t)(active ? idx : 0);
  // the item's words of step s: ring0 + (s/K % nslot) slot_bytes + (s % K) W + woff (bytes: x 4)
  const uint32_t woff = active ? 4u * (uint32_t)(gl * K * W + f0) : 0u;
  const uint32_t aoff = active ? 4u * (uint32_t)(gl * K * W + a.F) : 0u;  // the group's OR of perturbed lanes
  const uint32_t step_bytes = 4u * (uint32_t)W;
  const bool writer = active && f == 0;
  ResidentFn R;
  if (f < L) R.load(a.fn[f0 + f], st0, gpb, gl);
  else R.clear(st0);
  const int LW = (int)__reduce_max_sync(kFull, (unsigned)L);
  // bit m: property m needs this node at 1 (need1) and/or at 0 (need0; both
  // when a property names it twice)
  uint32_t need1 = 0u, need0 = 0u;
  if (writer)
    for (int e = 0; e < a.soi_size; e++)
      if ((int)a.soi_node[e] == node_id(rec)) {
        const uint32_t bit = 1u << a.soi_prop[e];
        if ((a.soi_val >> e) & 1u) need1 |= bit;
        else need0 |= bit;
      }
  const uint32_t in_props = need1 | need0;
  // this item's indicator words: property m, step s at ind_me + 4 (m gpb kIndRing + s % kIndRing)
  const uint32_t ind_me = smem_u32(ind) + 4u * (uint32_t)(gl * kIndRing);
  cta_barrier();  // the words of step 0 landed
  // one transition: state buffer CUR (0 or 1) to the other
  auto step = [&](int s, auto cur_tag) {
    constexpr int CUR = decltype(cur_tag)::value;
    constexpr int OFF_CUR = CUR * kResStride * 4, OFF_NXT = (1 - CUR) * kResStride * 4;
    {
      const uint32_t sb = ring0 + (uint32_t)((s / K) & smask) * slot_bytes + (uint32_t)(s % K) * step_bytes;
      const uint32_t w = sb + woff;
      const uint32_t P = lds_u32(w);
      const uint32_t S1 = L > 1 ? lds_u32(w + 4u) : 0u;  // lanes of function 0 (L > 1)
      const uint32_t old = writer ? lds_u32_at<OFF_CUR>(own) : 0u;
      const uint32_t v = R.eval<OFF_CUR>();
      const uint32_t rest = vmask & ~P;  // lanes that take one of the functions
      uint32_t part;
      if (!REST || LW <= 2) {
        // f = 0: function 0's lanes (all of `rest` when L = 1); f = 1: the others
        const uint32_t sel = f == 0 ? (L > 1 ? S1 : rest) : (L == 2 ? rest & ~S1 : 0u);
        part = sel & v;
      } else {
        part = rest_part(w, L, LW, f, rest, v, st0 + (uint32_t)OFF_CUR, a.fn, f0, a.gpb, gl);
      }
      const uint32_t fword = part | __shfl_xor_sync(kFull, part, 1);
      uint32_t nv;
      if (MODE == PBN_PERTURB_PER_NODE) {
        nv = (P & ~old) | fword;
      } else {
        const uint32_t any = lds_u32(sb + aoff);
        nv = (any & (old ^ P)) | (~any & fword);
      }
      if (writer) sts_u32_at<OFF_NXT>(own, nv);
      for (uint32_t props = in_props; props; props &= props - 1) {
        const int m = __ffs(props) - 1;
        const uint32_t term = ((need1 >> m) & 1u ? nv : kFull) & ((need0 >> m) & 1u ? ~nv : kFull);
        atom_and_shared(ind_me + 4u * (uint32_t)(m * gpb * kIndRing + (s & (kIndRing - 1))), term);
      }
    }
    cta_barrier();  // state after step s complete; the words of step s+1 landed
  };
  for (int s = 0; s < a.steps; s += 2) {
    step(s, std::integral_constant<int, 0>());
    if (s + 1 < a.steps) step(s + 1, std::integral_constant<int, 1>());
  }
  // the state after the last step (complete since its barrier)
  if (writer) a.state[(size_t)(g0 + gl) * n + node_id(rec)] = st[(a.steps & 1) * kResStride + idx];
}

template <int MODE, bool REST>
static cudaError_t launch_resident_mode(const SimArgs &a, int blocks, int threads, size_t smem, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(apply_resident_kernel<MODE, REST>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, sim_max_smem());
    if (e != cudaSuccess) return e;
    attr = true;
  }
  apply_resident_kernel<MODE, REST><<<blocks, threads, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_apply_resident(const SimArgs &a, int mode, bool rest, int threads, size_t smem, cudaStream_t s) {
  const int blocks = (a.G + a.gpb - 1) / a.gpb;
  if (blocks == 0 || a.steps == 0) return cudaSuccess;
  if (threads % 32 || threads < 64 || threads > 2 * kResidentItems + 32 || 2 * a.n * a.gpb > threads - 32 ||
      a.ring_log2 < kCopyLog + 1 || a.ring_log2 > kRingLogMax || a.has_wide)
    return cudaErrorInvalidValue;
  if (mode == PBN_PERTURB_PER_NODE)
    return rest ? launch_resident_mode<PBN_PERTURB_PER_NODE, true>(a, blocks, threads, smem, s)
                : launch_resident_mode<PBN_PERTURB_PER_NODE, false>(a, blocks, threads, smem, s);
  return rest ? launch_resident_mode<PBN_PERTURB_GLOBAL, true>(a, blocks, threads, smem, s)
              : launch_resident_mode<PBN_PERTURB_GLOBAL, false>(a, blocks, threads, smem, s);
}

// pad: dynamic shared memory the kernel does not use, requested only to
// limit where its blocks may run (see run_select_ahead).
template <int MODE, int BPR>
static cudaError_t launch_select_variant(const SimArgs &a, size_t pad, cudaStream_t s) {
  const int64_t total = (int64_t)a.steps * a.G * a.n;
  const int threads = 256;
  const int64_t blocks = (total + threads - 1) / threads;
  if (total >= (int64_t)1 << 32) return cudaErrorInvalidValue;  // the kernel indexes items in 32 bits
  static bool attr = false;
  if (pad > 0 && !attr) {
    cudaError_t e = cudaFuncSetAttribute(select_kernel<MODE, BPR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         sim_max_smem());
    if (e != cudaSuccess) return e;
    attr = true;
  }
  select_kernel<MODE, BPR><<<(unsigned)blocks, threads, pad, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_select(const SimArgs &a, int mode, int BPR, cudaStream_t s, size_t pad) {
  if (a.steps == 0 || a.G == 0) return cudaSuccess;
  if ((int64_t)pad > sim_max_smem()) return cudaErrorInvalidValue;
  if (mode == PBN_PERTURB_PER_NODE)
    return BPR == 2 ? launch_select_variant<PBN_PERTURB_PER_NODE, 2>(a, pad, s)
                    : launch_select_variant<PBN_PERTURB_PER_NODE, 1>(a, pad, s);
  return BPR == 2 ? launch_select_variant<PBN_PERTURB_GLOBAL, 2>(a, pad, s)
                  : launch_select_variant<PBN_PERTURB_GLOBAL, 1>(a, pad, s);
}

template <int MODE, int RING, int T, bool WIDE = false>
static cudaError_t launch_apply_variant(const SimArgs &a, int blocks, int threads, size_t smem, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(apply_kernel<MODE, RING, T, WIDE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, sim_max_smem());
    if (e != cudaSuccess) return e;
    attr = true;
  }
  apply_kernel<MODE, RING, T, WIDE><<<blocks, threads, smem, s>>>(a);
  return cudaGetLastError();
}

// Networks with functions of more than 5 inputs run the generic loop with one
// thread per item (the planner gives them T = 1).
template <int MODE, int RING>
static cudaError_t launch_apply_ring(const SimArgs &a, int T, int blocks, int threads, size_t smem, cudaStream_t s) {
  if (a.has_wide) return T == 1 ? launch_apply_variant<MODE, RING, 1, true>(a, blocks, threads, smem, s)
                                : cudaErrorInvalidValue;
  if (T == 4) return launch_apply_variant<MODE, RING, 4>(a, blocks, threads, smem, s);
  if (T == 2) return launch_apply_variant<MODE, RING, 2>(a, blocks, threads, smem, s);
  return launch_apply_variant<MODE, RING, 1>(a, blocks, threads, smem, s);
}

template <int MODE>
static cudaError_t launch_apply_mode(const SimArgs &a, int ring, int T, int blocks, int threads, size_t smem,
                                     cudaStream_t s) {
  return ring == 8 ? launch_apply_ring<MODE, 8>(a, T, blocks, threads, smem, s)
                   : launch_apply_ring<MODE, 3>(a, T, blocks, threads, smem, s);
}

cudaError_t launch_apply(const SimArgs &a, int mode, int ring, int T, int threads, size_t smem, cudaStream_t s) {
  const int blocks = (a.G + a.gpb - 1) / a.gpb;
  if (blocks == 0 || a.steps == 0) return cudaSuccess;
  if ((ring != 8 && ring != 3) || (T != 1 && T != 2 && T != 4) || threads % 32 || threads > apply_threads_limit(T))
    return cudaErrorInvalidValue;
  if (mode == PBN_PERTURB_PER_NODE) return launch_apply_mode<PBN_PERTURB_PER_NODE>(a, ring, T, blocks, threads, smem, s);
  return launch_apply_mode<PBN_PERTURB_GLOBAL>(a, ring, T, blocks, threads, smem, s);
}

}  // namespace pbn
