// Select-ahead schedule of the synchronous PBN step (Sec. 2.2): the category
// draws of a whole chunk of steps first, the state updates after.
//
// The uniform that picks a node's category at transition t (perturbed, or
// predictor function j) depends on (seed, node, t, chain) only, never on the
// state.  So the draws of every (step, chain group, node) of a chunk of steps
// are independent work: select_kernel spreads them over the whole GPU.  What
// stays sequential is the state update proper, which apply_kernel runs with
// one CTA per chain group(s): per step a thread reads its item's category
// words, evaluates the selected truth tables on the parents' words and writes
// the next state; one barrier per step.  When few chain groups exist (a query
// of about a thousand chains) the fused kernel leaves most SMs idle and waits
// on a chain of Philox rounds every step; here the Philox work runs at full
// width and the sequential part is short.
//
// Category words of item (step s, group g, processing position r) at
// planes[(s * G + g) * W + f0_r + w], w < l_r (f0_r = the node's first
// function record in processing order, W = F rounded up to 4 words):
//   w = 0:          lanes perturbed at this node (category 0)
//   w = 1 .. l-1:   lanes that selected function w-1
// The last function's lanes are the valid lanes in none of those words.
// Global perturbation also stores, per (s, g), the OR of all nodes' w = 0
// words (anyw[s * G + g]): the chains that take s XOR gamma.
//
// Both kernels compare the same digits against the same bounds as the fused
// kernel (draw_below), so the chains are bit-identical under either schedule.
#include <algorithm>

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
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t total = (int64_t)a.steps * a.G * a.n;
  const bool active = q < total;
  const int64_t sg = active ? q / a.n : 0;
  const int r = active ? (int)(q - sg * a.n) : 0;
  const int s = (int)(sg / a.G);
  ItemCtx c;
  c.fn_s = a.fn;
  c.g = (uint32_t)(sg - (int64_t)s * a.G);
  const uint32_t rec = active ? a.node[r] : 0u;
  c.L = active ? node_l(rec) : 0;
  c.i = node_id(rec);
  c.f0 = node_f0(rec);
  c.vmask = active ? lane_mask(a.omega, c.g) : 0u;
  c.t = a.t0 + (uint64_t)s;
  c.sub = 0;
  uint32_t *out = a.planes + sg * a.W + c.f0;
  uint32_t *anyw = a.anyw + sg;
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

__device__ __forceinline__ void copy4_async(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(__cvta_generic_to_global(src))
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
  size_t b = (size_t)ring * gpb * W * 4;                      // category words ring
  b += (size_t)ring * (((size_t)gpb + 3) & ~(size_t)3) * 4;   // OR-of-perturbations ring
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
  const int gpbA = (gpb + 3) & ~3;
  uint32_t *ring = reinterpret_cast<uint32_t *>(smem);
  uint32_t *ring_any = ring + (size_t)kRing * gpb * W;
  unsigned char *p = reinterpret_cast<unsigned char *>(ring_any + (size_t)kRing * gpbA);
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
  // step s's words of this CTA's groups: one contiguous run of ngl * W words
  const int chunks16 = ngl * W / 4;
  auto issue = [&](int s) {
    if (s < a.steps) {
      const uint32_t *src = a.planes + ((size_t)s * a.G + g0) * W;
      uint32_t *dst = ring + (size_t)(s % kRing) * gpb * W;
      for (int j = threadIdx.x; j < chunks16; j += blockDim.x) copy16_async(dst + 4 * j, src + 4 * j);
      if (MODE == PBN_PERTURB_GLOBAL)
        for (int gl = threadIdx.x; gl < ngl; gl += blockDim.x)
          copy4_async(ring_any + (s % kRing) * gpbA + gl, a.anyw + (size_t)s * a.G + g0 + gl);
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
  auto finish = [&](int idx, int gl, uint32_t P, uint32_t fword, const uint32_t *slot_any) -> uint32_t {
    uint32_t v;
    if (MODE == PBN_PERTURB_PER_NODE) {
      v = (P & ~cur[idx]) | fword;
    } else {
      const uint32_t any = slot_any[gl];
      v = (any & (cur[idx] ^ P)) | (~any & fword);
    }
    nxt[idx] = v;
    return v;
  };
  if (!WIDE && items * T <= (int)blockDim.x - 32) {
    // One item per T threads for the whole launch, everything that does not
    // change from step to step in registers; the last warp is the producer:
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
        const uint32_t *src = a.planes + ((size_t)s * a.G + g0) * W;
        uint32_t *dst = ring + (size_t)(s % kRing) * slot_words;
        for (int j = lane; j < chunks16; j += 32) copy16_async(dst + 4 * j, src + 4 * j);
        if (MODE == PBN_PERTURB_GLOBAL)
          for (int g = lane; g < ngl; g += 32)
            copy4_async(ring_any + (s % kRing) * gpbA + g, a.anyw + (size_t)s * a.G + g0 + g);
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
          const uint32_t v = finish(idx, gl, P, fword, ring_any + ring_slot * gpbA);
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
    for (int s = 0; s < kRing - 1; s++) issue(s);
    for (int s = 0; s < a.steps; s++) {
      step_top(s);
      const uint32_t *slot = ring + (size_t)(s % kRing) * gpb * W;
      for (int base = 0; base < items * T; base += blockDim.x) {  // uniform trip count
        const int q = base + threadIdx.x;
        const int it = q / T, sub = q & (T - 1);
        const int r = it / gpb, gl = it - r * gpb;
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
        if (active && sub == 0) finish(node_id(rec) * gpb + gl, gl, P, fword, ring_any + (s % kRing) * gpbA);
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

template <int MODE, int BPR>
static cudaError_t launch_select_variant(const SimArgs &a, cudaStream_t s) {
  const int64_t total = (int64_t)a.steps * a.G * a.n;
  const int threads = 256;
  const int64_t blocks = (total + threads - 1) / threads;
  if (blocks > 0x7FFFFFFF) return cudaErrorInvalidValue;
  select_kernel<MODE, BPR><<<(unsigned)blocks, threads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_select(const SimArgs &a, int mode, int BPR, cudaStream_t s) {
  if (a.steps == 0 || a.G == 0) return cudaSuccess;
  if (mode == PBN_PERTURB_PER_NODE)
    return BPR == 2 ? launch_select_variant<PBN_PERTURB_PER_NODE, 2>(a, s)
                    : launch_select_variant<PBN_PERTURB_PER_NODE, 1>(a, s);
  return BPR == 2 ? launch_select_variant<PBN_PERTURB_GLOBAL, 2>(a, s)
                  : launch_select_variant<PBN_PERTURB_GLOBAL, 1>(a, s);
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
