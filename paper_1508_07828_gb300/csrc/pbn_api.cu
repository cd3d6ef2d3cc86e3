// C ABI of the GB300 PBN engine: network staging, chain runs, statistics and
// the end-to-end drivers (Alg. GR followed by Alg. 3 or Alg. 4).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "pbn_internal.cuh"


namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char *what) {
  return fail(e == cudaErrorMemoryAllocation ? PBN_ERR_OOM : PBN_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CUDA_TRY(expr, what)                      \
  do {                                            \
    cudaError_t _e = (expr);                      \
    if (_e != cudaSuccess) return cuda_fail(_e, what); \
  } while (0)

// Quantisation of the perturbation probability: P32 = round(p 2^32), at most 2^32-1.
uint32_t quantise_p(double p) {
  long long q = llround(p * 4294967296.0);
  if (q < 0) q = 0;
  if (q > 4294967295LL) q = 4294967295LL;
  return (uint32_t)q;
}

int sm_count() {
  static int v = 0;
  if (!v) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 1;
  }
  return v;
}

// Scratch of the primitive statistics entry points, one per stream.
std::mutex g_scratch_mu;
std::map<std::pair<int, cudaStream_t>, pbn::StatsScratch> g_scratch;

int scratch_for(cudaStream_t s, pbn::StatsScratch **out) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  auto key = std::make_pair(dev, s);
  auto it = g_scratch.find(key);
  if (it == g_scratch.end()) {
    pbn::StatsScratch sc;
    cudaError_t e = pbn::scratch_init(sc, s);
    if (e != cudaSuccess) {
      pbn::scratch_free(sc);
      return cuda_fail(e, "statistics scratch");
    }
    it = g_scratch.emplace(key, sc).first;
  }
  *out = &it->second;
  return PBN_OK;
}

int check_soi(const pbn_soi &soi, int n, bool allow_empty) {
  if (soi.size == 0 && allow_empty) return PBN_OK;
  if (soi.size < 1 || soi.size > PBN_MAX_SOI) return fail(PBN_ERR_INVALID, "state of interest size %d", soi.size);
  if (!soi.nodes || !soi.values) return fail(PBN_ERR_INVALID, "state of interest arrays are NULL");
  for (int m = 0; m < soi.size; m++) {
    if (soi.nodes[m] < 0 || soi.nodes[m] >= n) return fail(PBN_ERR_INVALID, "SOI node %d out of range", soi.nodes[m]);
    if (soi.values[m] > 1) return fail(PBN_ERR_INVALID, "SOI value must be 0 or 1");
  }
  return PBN_OK;
}

struct LaunchPlan {
  int gpb, threads, T, BPR;
  size_t smem;
  int staging;
};

// Launch shape: chain groups per CTA from the group count and the SM count
// (shared memory permitting); with fewer groups than SMs the step is
// latency-bound, so 2 threads share an item (each runs 2 Philox blocks, in
// parallel); otherwise one thread per item, one block per round.
int plan_launch(const pbn::NetDev &net, int64_t omega, int mode, int gpb_req, int threads_req, int T_req,
                int BPR_req, int staging_req, LaunchPlan *p) {
  const int G = (int)((omega + 31) / 32);
  const int maxs = pbn::sim_max_smem();
  int gpb = gpb_req > 0 ? gpb_req : std::max(1, (G + sm_count() - 1) / sm_count());
  gpb = std::min(gpb, std::max(G, 1));
  // staging preference: whole tables in shared memory, else global reads
  // (the records a warp touches stay in L1; measured faster than TMA tiles,
  // whose buffers cost chain groups per CTA and whose per-tile barriers cost
  // time); TMA tiles only when requested
  const int prefs[3] = {pbn::STAGE_SMEM, pbn::STAGE_GLOBAL, pbn::STAGE_TILES};
  // public values: 1 = whole tables in shared memory, 2 = TMA tiles, 3 = global
  const int wanted = staging_req == 1 ? pbn::STAGE_SMEM
                     : staging_req == 2 ? pbn::STAGE_TILES
                     : staging_req == 3 ? pbn::STAGE_GLOBAL
                                        : -1;
  for (;;) {
    bool found = false;
    for (int st : prefs) {
      if (wanted >= 0 && st != wanted) continue;
      const size_t b = pbn::sim_smem_bytes(net.n, net.F, gpb, mode, st, net.tile_bytes);
      if ((int64_t)b <= maxs) {
        p->staging = st;
        p->smem = b;
        found = true;
        break;
      }
    }
    if (found) break;
    if (gpb == 1) return fail(PBN_ERR_UNSUPPORTED, "chain state of one group does not fit shared memory");
    gpb = std::max(1, gpb / 2);
  }
  int T = T_req;
  const bool many = net.max_l > pbn::kMaxL || net.max_k > pbn::kWideK;
  if (T == 0) T = (G < sm_count() && net.n * gpb * 2 <= 512 && !net.has_wide && !many) ? 2 : 1;
  if (T != 1 && T != 2 && T != 4) return fail(PBN_ERR_INVALID, "threads_per_item %d (1, 2 or 4)", T);
  if (net.has_wide && (T != 1 || (BPR_req && BPR_req != 1)))
    return fail(PBN_ERR_UNSUPPORTED, "functions with more than 5 inputs run one thread per item, one block per round");
  if (many && (T != 1 || (BPR_req && BPR_req != 1)))
    return fail(PBN_ERR_UNSUPPORTED,
                "nodes with more than %d functions or functions of more than %d inputs run one thread per item, "
                "one block per round", pbn::kMaxL, pbn::kWideK);
  int BPR = BPR_req ? BPR_req : 1;
  if (T == 2) BPR = 2;
  if (T == 4) BPR = 1;
  if (BPR != 1 && BPR != 2) return fail(PBN_ERR_INVALID, "blocks_per_round %d (1 or 2)", BPR);
  const int items = net.n * gpb;
  const int tmax = T == 1 ? 1024 : 512;
  int threads = threads_req > 0 ? threads_req : std::min(tmax, std::max(32, (items * T + 31) / 32 * 32));
  if (threads % 32 || threads > tmax || threads < 32)
    return fail(PBN_ERR_INVALID, "threads_per_block %d (a multiple of 32, at most %d here)", threads, tmax);
  p->gpb = gpb;
  p->threads = threads;
  p->T = T;
  p->BPR = BPR;
  return PBN_OK;
}

// status: the device status word the kernels' bounded waits report to (the
// device's own word unless a caller such as the engine keeps one)
pbn::SimArgs make_args(const pbn::NetDev &net, const pbn_run_cfg &cfg, const pbn_chains &ch, int64_t steps,
                       const LaunchPlan &plan, int *status = nullptr) {
  pbn::SimArgs a;
  memset(&a, 0, sizeof a);
  a.rk = pbn::make_round_keys(cfg.seed);
  a.node = net.d_node;
  a.fn = net.d_fn;
  a.state = ch.state;
  a.bits = ch.bits;
  a.bits_cap = ch.bits_cap;
  a.col0 = ch.length - ch.bits_base;
  a.omega = ch.omega;
  a.t0 = (uint64_t)ch.length;
  a.n = net.n;
  a.F = net.F;
  a.G = (int)((ch.omega + 31) / 32);
  a.steps = (int)steps;
  a.gpb = plan.gpb;
  a.P32 = net.P32;
  a.staging = plan.staging;
  a.tiles = net.d_tiles;
  a.ntiles = net.ntiles;
  a.tile_bytes = net.tile_bytes;
  a.wide_tt = net.d_wide_tt;
  a.wide_par = net.d_wide_par;
  a.has_wide = net.has_wide;
  a.many = (net.max_l > pbn::kMaxL || net.max_k > pbn::kWideK) ? 1 : 0;
  a.status = status ? status : pbn::device_status();
  {
    static const int stall = getenv("PBN_TEST_STALL_FIRST_TILE") ? atoi(getenv("PBN_TEST_STALL_FIRST_TILE")) : 0;
    a.test_stall = stall;
  }
  // state-of-interest entries of every recorded property, flattened
  const bool bits = ch.bits && ch.bits_cap > 0;
  const int np = cfg.n_props > 0 ? cfg.n_props : (cfg.soi.size > 0 ? 1 : 0);
  a.soi_val = 0;
  a.soi_size = 0;
  a.n_props = bits ? np : 0;
  a.prop_stride = (int64_t)a.G * ch.bits_cap;
  for (int m = 0; m < np && bits; m++) {
    const pbn_soi &p = cfg.n_props > 0 ? cfg.props[m] : cfg.soi;
    for (int e = 0; e < p.size && a.soi_size < PBN_MAX_SOI; e++, a.soi_size++) {
      a.soi_node[a.soi_size] = (uint16_t)p.nodes[e];
      a.soi_prop[a.soi_size] = (uint8_t)m;
      if (p.values[e]) a.soi_val |= 1u << a.soi_size;
    }
  }
  return a;
}

// Properties of a run configuration (pbn_run_cfg.n_props / props, else soi).
int check_props(const pbn_run_cfg &cfg, int n) {
  if (cfg.n_props < 0 || cfg.n_props > PBN_MAX_PROPERTIES)
    return fail(PBN_ERR_INVALID, "n_props %d (0 .. %d)", cfg.n_props, PBN_MAX_PROPERTIES);
  if (cfg.n_props == 0) return check_soi(cfg.soi, n, true);
  if (!cfg.props) return fail(PBN_ERR_INVALID, "props is NULL");
  int total = 0;
  for (int m = 0; m < cfg.n_props; m++) {
    int rc = check_soi(cfg.props[m], n, false);
    if (rc) return rc;
    total += cfg.props[m].size;
  }
  if (total > PBN_MAX_SOI) return fail(PBN_ERR_INVALID, "%d state-of-interest entries over all properties (at most %d)",
                                       total, PBN_MAX_SOI);
  return PBN_OK;
}

int n_recorded_props(const pbn_run_cfg &cfg) { return cfg.n_props > 0 ? cfg.n_props : (cfg.soi.size > 0 ? 1 : 0); }

// Select-ahead scratch per (device, stream): the category words of a chunk
// of steps (for global perturbation with their per-group OR in word F of each
// run), two buffers when chunks are pipelined.  Grown on the stream, so
// launches already queued keep the old buffer until they finish.  A
// pipelined run draws chunk i+1 on the side stream while chunk i is applied
// on the caller's stream; events order the two (start; selected[b],
// applied[b] per buffer).
struct SelectScratch {
  uint32_t *planes[2] = {nullptr, nullptr};
  size_t planes_words[2] = {0, 0};
  cudaStream_t side = nullptr;
  cudaEvent_t start = nullptr, selected[2] = {nullptr, nullptr}, applied[2] = {nullptr, nullptr};
};
std::mutex g_sel_mu;
std::map<std::pair<int, cudaStream_t>, SelectScratch> g_sel;

int grow(uint32_t *&buf, size_t &have, size_t words, cudaStream_t s) {
  if (words <= have) return PBN_OK;
  if (buf) cudaFreeAsync(buf, s);
  buf = nullptr;
  have = 0;
  cudaError_t e = cudaMallocAsync(&buf, words * 4, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? PBN_ERR_OOM : PBN_ERR_CUDA, "select-ahead scratch: %s",
                cudaGetErrorString(e));
  }
  have = words;
  return PBN_OK;
}

// Largest chunk of the select-ahead schedule: 2048 steps, or fewer when the
// category words of all groups would exceed 32 MiB per buffer (both buffers
// of a pipelined run stay in L2 between the kernels at the chain counts this
// schedule is for).  A run longer than one chunk starts with kSelectFirst
// steps and doubles the chunk up to the largest, so the first apply starts
// early and every later chunk is drawn while the previous one is applied.
constexpr int64_t kSelectMaxSteps = 2048;
constexpr int64_t kSelectBudgetBytes = 32ll << 20;
constexpr int64_t kSelectFirst = 128;

int ensure_side(SelectScratch *sc) {
  if (sc->side) return PBN_OK;
  cudaError_t e = cudaStreamCreateWithFlags(&sc->side, cudaStreamNonBlocking);
  cudaEvent_t *evs[5] = {&sc->start, &sc->selected[0], &sc->selected[1], &sc->applied[0], &sc->applied[1]};
  for (int i = 0; i < 5 && e == cudaSuccess; i++) e = cudaEventCreateWithFlags(evs[i], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(PBN_ERR_CUDA, "select-ahead side stream: %s", cudaGetErrorString(e));
  }
  return PBN_OK;
}

struct SelectPlan {
  int gpb, threads, staging, W, T;
  int ring;       // one-thread apply: ring slots; resident apply: log2 of the ring's steps
  bool resident;  // apply_resident_kernel (two threads per item, bulk-copied steps)
  size_t smem;
};

// Launch shape of the select-ahead schedule, or PBN_ERR_UNSUPPORTED when its
// shared memory does not fit (staging_req: public values 0, 1, 3; 2 = tiles
// is not supported).
int plan_select(const pbn::NetDev &net, int64_t omega, int mode, int gpb_req, int threads_req, int T_req,
                int staging_req, int n_props, SelectPlan *p) {
  const int G = (int)((omega + 31) / 32);
  const int maxs = pbn::sim_max_smem();
  if (staging_req == 2) return fail(PBN_ERR_UNSUPPORTED, "select-ahead schedule with TMA tiles");
  if (net.max_l > pbn::kMaxL || net.max_k > pbn::kWideK)
    return fail(PBN_ERR_UNSUPPORTED, "select-ahead schedule with nodes of more than %d functions or functions of "
                "more than %d inputs", pbn::kMaxL, pbn::kWideK);
  int gpb = gpb_req > 0 ? gpb_req : std::max(1, (G + sm_count() - 1) / sm_count());
  gpb = std::min(gpb, std::max(G, 1));
  const int W = (net.F + (mode == PBN_PERTURB_GLOBAL ? 1 : 0) + 3) & ~3;
  // a deep ring (latency of the category words hidden 7 steps ahead) before
  // tables in shared memory; the records a warp reads stay in L1 otherwise
  const int opts[4][2] = {{8, pbn::STAGE_SMEM}, {8, pbn::STAGE_GLOBAL}, {3, pbn::STAGE_SMEM}, {3, pbn::STAGE_GLOBAL}};
  for (;;) {
    bool found = false;
    for (const auto &o : opts) {
      const int st = o[1];
      if (staging_req == 1 && st != pbn::STAGE_SMEM) continue;
      if (staging_req == 3 && st != pbn::STAGE_GLOBAL) continue;
      const size_t b = pbn::apply_smem_bytes(net.n, net.F, gpb, W, st, o[0], n_props);
      if ((int64_t)b <= maxs) {
        p->staging = st;
        p->ring = o[0];
        p->smem = b;
        found = true;
        break;
      }
    }
    if (found) break;
    if (gpb == 1 || gpb_req > 0)
      return fail(PBN_ERR_UNSUPPORTED, "select-ahead shared memory does not fit (n %d, F %d)", net.n, net.F);
    gpb = std::max(1, gpb / 2);
  }
  // Threads per item unless asked (measured on GB300 over n = 100 .. 3000 with
  // 256 .. 4096 chains): 1 when every function of an item stays in registers
  // (at most two per node) or when the CTA holds more than 240 items (two
  // threads per item would no longer fit the register-resident path); else 2,
  // which splits the per-step decoding of a node's further functions.
  const bool two = net.max_l > 2 && net.n * gpb <= 240 && !net.has_wide;
  const int T = T_req > 0 ? T_req : (two ? 2 : 1);
  if (T != 1 && T != 2 && T != 4) return fail(PBN_ERR_INVALID, "threads_per_item %d (1, 2 or 4)", T);
  if (net.has_wide && T != 1)
    return fail(PBN_ERR_UNSUPPORTED, "functions with more than 5 inputs run one thread per item");
  const int items = net.n * gpb;
  const int tmax = pbn::apply_threads_limit(T);
  // with one item per T threads for the whole launch, one more warp feeds the others
  const int item_threads = (items * T + 31) / 32 * 32;
  int threads = threads_req > 0                                  ? threads_req
                : (!net.has_wide && item_threads + 32 <= tmax)    ? item_threads + 32
                                                                 : std::min(tmax, std::max(32, item_threads));
  if (threads % 32 || threads > tmax || threads < 32)
    return fail(PBN_ERR_INVALID, "threads_per_block %d (a multiple of 32, at most %d here)", threads, tmax);
  p->T = T;
  p->gpb = gpb;
  p->threads = threads;
  p->W = W;
  p->resident = false;
  // One thread per item asked for, every item resident for the whole launch:
  // the register-resident kernel (two threads per item, one per function
  // slot) with a ring of 16 bulk-copied steps (two copies of 8 in flight;
  // measured: 32 steps gain nothing).  When the ring does not fit in shared
  // memory the one-thread apply runs instead.  Staging requests other than
  // tiles read the records beyond a node's second from global memory there.
  const int pair_threads = (2 * items + 31) / 32 * 32;
  if (T == 1 && !net.has_wide && items <= pbn::kResidentItems &&
      (threads_req == 0 || threads_req == pair_threads + 32)) {
    const int lg = 4;
    const size_t b = pbn::apply_resident_smem_bytes(gpb, W, 1 << lg, n_props);
    if ((int64_t)b <= maxs) {
      p->resident = true;
      p->ring = lg;
      p->staging = pbn::STAGE_GLOBAL;
      p->smem = b;
      p->threads = pair_threads + 32;
    }
  }
  return PBN_OK;
}

// Optional CUDA-event timing of the apply launches (the dominant kernel of the
// select-ahead schedule): `next` hands out events from the caller's pool.
struct ApplyTiming {
  cudaEvent_t (*next)(void *ctx) = nullptr;
  void *ctx = nullptr;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pairs;
};

int run_select_ahead(const pbn::NetDev &net, const pbn_run_cfg &cfg, pbn_chains &ch, int64_t steps, bool record,
                     const SelectPlan &sp, cudaStream_t s, int64_t *launches, ApplyTiming *timing,
                     int *status = nullptr) {
  const int G = (int)((ch.omega + 31) / 32);
  const int64_t per_step = (int64_t)G * sp.W * 4;
  const int64_t C = std::max<int64_t>(1, std::min(kSelectMaxSteps, kSelectBudgetBytes / per_step));
  const bool pipe = steps > C;
  SelectScratch *sc;
  {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_sel_mu);
    sc = &g_sel[std::make_pair(dev, s)];
  }
  const size_t words = (size_t)std::min(C, steps) * G * sp.W;
  int rc = grow(sc->planes[0], sc->planes_words[0], words, s);
  if (rc) return rc;
  if (pipe) {
    if ((rc = grow(sc->planes[1], sc->planes_words[1], words, s)) || (rc = ensure_side(sc))) return rc;
    // the side stream starts after everything queued on the caller's stream
    CUDA_TRY(cudaEventRecord(sc->start, s), "event");
    CUDA_TRY(cudaStreamWaitEvent(sc->side, sc->start, 0), "stream wait");
  }
  // While chunk i is applied, chunk i+1 is drawn on the SMs the apply CTAs
  // leave free: an apply CTA and a select block together ask for more shared
  // memory than an SM has, so select blocks (four per SM) never share an SM
  // with the latency-bound apply, which keeps its issue slots.
  size_t select_pad = 0, apply_smem = sp.smem;
  if (pipe && (G + sp.gpb - 1) / sp.gpb < sm_count()) {
    static int per_sm = -1, reserved = -1;  // device attributes, read once
    if (per_sm < 0) {
      int dev = 0;
      cudaGetDevice(&dev);
      if (cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
          cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess) {
        cudaGetLastError();
        per_sm = reserved = 0;
      }
    }
    if (per_sm > 0) {
      const int64_t pad = per_sm / 4 - reserved;
      const int64_t need = (int64_t)per_sm - pad - 2 * reserved + 16;
      if (pad > 0 && need <= pbn::sim_max_smem()) {
        select_pad = (size_t)pad;
        apply_smem = std::max(apply_smem, (size_t)need);
      }
    }
  }
  LaunchPlan lp;
  lp.gpb = sp.gpb;
  lp.threads = sp.threads;
  lp.T = 1;
  lp.BPR = 1;
  lp.smem = apply_smem;
  lp.staging = sp.staging;
  int64_t k = 0;
  for (int64_t done = 0, i = 0; done < steps; done += k, i++) {
    // ramp 128, 256, 512, then chunks of C; from the fourth on, a rest that
    // fits one chunk is taken whole (it is drawn while 512 or more steps apply)
    k = pipe ? std::min(std::min(C, kSelectFirst << std::min<int64_t>(i, 20)), steps - done) : steps - done;
    if (pipe && i >= 3 && steps - done <= C) k = steps - done;
    const int b = pipe ? (int)(i & 1) : 0;
    cudaStream_t ss = pipe ? sc->side : s;
    pbn::SimArgs a = make_args(net, cfg, ch, k, lp, status);
    if (!record) a.soi_size = 0;
    a.W = sp.W;
    a.planes = sc->planes[b];
    a.ring_log2 = sp.resident ? sp.ring : 0;
    // buffer b was last read by the apply of chunk i-2
    if (pipe && i >= 2) CUDA_TRY(cudaStreamWaitEvent(ss, sc->applied[b], 0), "stream wait");
    if (cfg.perturb_mode == PBN_PERTURB_GLOBAL)  // word F of every (step, group) run: OR-ed into by select
      CUDA_TRY(cudaMemset2DAsync(a.planes + net.F, (size_t)sp.W * 4, 0, 4, (size_t)k * G, ss),
               "select-ahead clear");
    CUDA_TRY(pbn::launch_select(a, cfg.perturb_mode, 1, ss, select_pad), "select launch");
    if (pipe) {
      CUDA_TRY(cudaEventRecord(sc->selected[b], ss), "event");
      CUDA_TRY(cudaStreamWaitEvent(s, sc->selected[b], 0), "stream wait");
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (timing) {
      e0 = timing->next(timing->ctx);
      e1 = timing->next(timing->ctx);
      if (!e0 || !e1) return fail(PBN_ERR_CUDA, "event creation failed");
      CUDA_TRY(cudaEventRecord(e0, s), "event");
    }
    if (sp.resident)
      CUDA_TRY(pbn::launch_apply_resident(a, cfg.perturb_mode, net.max_l > 2, sp.threads, apply_smem, s),
               "apply launch");
    else
      CUDA_TRY(pbn::launch_apply(a, cfg.perturb_mode, sp.ring, sp.T, sp.threads, apply_smem, s), "apply launch");
    if (timing) {
      CUDA_TRY(cudaEventRecord(e1, s), "event");
      timing->pairs.emplace_back(e0, e1);
    }
    if (pipe) CUDA_TRY(cudaEventRecord(sc->applied[b], s), "event");
    ch.length += k;
    if (launches) *launches += 2;
  }
  return PBN_OK;
}

// Balanced fused launches for G chain groups over R CTAs (one per SM), when
// G / R is not whole: with q = G / R and rem = G % R, one launch makes every SM
// carry q + 1 groups for all k steps.  Instead, phase 1 gives R - rem CTAs q
// groups for k steps and rem CTAs q + 1 groups for x < k steps, x chosen so
// that both finish together; phase 2 spreads the rem (q+1) lagging groups
// over the R CTAs for their last k - x steps.  Every group still takes its
// own transitions in order, so the chains are the same.  Step cost of a CTA
// with g groups: its item rounds ceil(n g T / threads) plus about 1.5 rounds
// that do not scale with g (barrier, indicator, the last partial round);
// measured on n = 2000, 1024 threads: 3 and 2 groups take 0.80 and 0.575 of
// a 4-group step (the model: 0.79 and 0.58).  Returns false (one launch) when
// the model saves nothing.
bool balance_phases(int G, int R, const LaunchPlan &plan, int n, int64_t k, pbn::SimArgs *ph1,
                    pbn::SimArgs *ph2) {
  if (R <= 0 || G <= R || k < 64) return false;
  const int q = G / R, rem = G % R;
  if (rem == 0 || plan.gpb < q + 1) return false;
  auto cost = [&](int g) {
    return (double)(((int64_t)n * g * plan.T + plan.threads - 1) / plan.threads) + 1.5;
  };
  const int lag = rem * (q + 1);
  const int b2 = std::min(R, lag);
  const int per2 = (lag + b2 - 1) / b2;
  const int64_t x = std::min(k - 1, std::max<int64_t>(1, (int64_t)((double)k * cost(q) / cost(q + 1))));
  if (cost(q) * (double)k + cost(per2) * (double)(k - x) >= cost(q + 1) * (double)k) return false;
  ph1->seg_blocks[0] = R - rem;
  ph1->seg_g0[0] = 0;
  ph1->seg_ng[0] = (R - rem) * q;
  ph1->seg_steps[0] = (int)k;
  ph1->seg_soff[0] = 0;
  ph1->seg_blocks[1] = rem;
  ph1->seg_g0[1] = (R - rem) * q;
  ph1->seg_ng[1] = lag;
  ph1->seg_steps[1] = (int)x;
  ph1->seg_soff[1] = 0;
  ph2->seg_blocks[0] = b2;
  ph2->seg_g0[0] = (R - rem) * q;
  ph2->seg_ng[0] = lag;
  ph2->seg_steps[0] = (int)(k - x);
  ph2->seg_soff[0] = (int)x;
  ph2->seg_blocks[1] = 0;
  ph2->seg_g0[1] = ph2->seg_ng[1] = ph2->seg_steps[1] = ph2->seg_soff[1] = 0;
  return true;
}

int run_steps(const pbn::NetDev &net, const pbn_run_cfg &cfg, pbn_chains &ch, int64_t steps, cudaStream_t s,
              int64_t *launches = nullptr, ApplyTiming *timing = nullptr, int *status = nullptr) {
  if (steps < 0) return fail(PBN_ERR_INVALID, "negative step count");
  if (steps == 0) return PBN_OK;
  const bool record = ch.bits && ch.bits_cap > 0 && n_recorded_props(cfg) > 0;
  if (record) {
    const int64_t last = ch.length + steps - 1 - ch.bits_base;
    if (last >= ch.bits_cap) return fail(PBN_ERR_INVALID, "bitstream capacity %lld too small for position %lld",
                                         (long long)ch.bits_cap, (long long)(ch.length + steps - 1));
  }
  LaunchPlan plan;
  if (cfg.staging < 0 || cfg.staging > 3) return fail(PBN_ERR_INVALID, "staging %d", cfg.staging);
  if (cfg.schedule < PBN_SCHEDULE_AUTO || cfg.schedule > PBN_SCHEDULE_SELECT_AHEAD)
    return fail(PBN_ERR_INVALID, "schedule %d", cfg.schedule);
  if (!pbn::device_status()) return fail(PBN_ERR_CUDA, "device status word unavailable");
  const int G = (int)((ch.omega + 31) / 32);
  // automatic: select-ahead while one CTA per chain group leaves SMs idle,
  // except for large networks with groups for more than half the SMs, where
  // the fused kernel's per-step work is already spread well (measured)
  const bool want_select = cfg.schedule == PBN_SCHEDULE_SELECT_AHEAD ||
                           (cfg.schedule == PBN_SCHEDULE_AUTO && G <= sm_count() &&
                            (net.n <= 1000 || 2 * G <= sm_count()) && cfg.staging != 2 &&
                            cfg.threads_per_item == 0 && cfg.blocks_per_round == 0);
  if (want_select) {
    SelectPlan sp;
    const std::string saved = g_err;
    int rc = plan_select(net, ch.omega, cfg.perturb_mode, cfg.groups_per_block, cfg.threads_per_block,
                         cfg.threads_per_item, cfg.staging, n_recorded_props(cfg), &sp);
    if (rc == PBN_OK) return run_select_ahead(net, cfg, ch, steps, record, sp, s, launches, timing, status);
    if (cfg.schedule == PBN_SCHEDULE_SELECT_AHEAD) return rc;
    g_err = saved;  // automatic choice: fall back to the fused schedule
  }
  int rc = plan_launch(net, ch.omega, cfg.perturb_mode, cfg.groups_per_block, cfg.threads_per_block,
                       cfg.threads_per_item, cfg.blocks_per_round, cfg.staging, &plan);
  if (rc) return rc;
  // one launch covers at most 2^30 steps; the step counter itself is 64-bit
  const int64_t chunk = 1 << 30;
  for (int64_t done = 0; done < steps; done += chunk) {
    const int64_t k = std::min(chunk, steps - done);
    pbn::SimArgs a = make_args(net, cfg, ch, k, plan, status);
    if (!record) a.soi_size = 0;
    pbn::SimArgs a2 = a;
    // automatic shape only: a requested groups_per_block keeps its one launch
    if (cfg.groups_per_block == 0 && balance_phases(a.G, sm_count(), plan, net.n, k, &a, &a2)) {
      CUDA_TRY(pbn::launch_sim(a, cfg.perturb_mode, plan.T, plan.BPR, plan.threads, plan.smem, s),
               "simulation launch");
      CUDA_TRY(pbn::launch_sim(a2, cfg.perturb_mode, plan.T, plan.BPR, plan.threads, plan.smem, s),
               "simulation launch");
      if (launches) *launches += 2;
    } else {
      CUDA_TRY(pbn::launch_sim(a, cfg.perturb_mode, plan.T, plan.BPR, plan.threads, plan.smem, s),
               "simulation launch");
      if (launches) *launches += 1;
    }
    ch.length += k;
  }
  return PBN_OK;
}

}  // namespace

void pbn::set_last_error(const char *msg) { g_err = msg; }

// One query's extension outside the batched kernel (the engine's epochs with
// a single small query): the schedule pbn_run_chains would pick, the bounded
// waits reporting to `status`.
int pbn::run_chains_alone(const NetDev &net, const pbn_run_cfg &cfg, pbn_chains &ch, int64_t steps, cudaStream_t s,
                          int *status, int64_t *launches) {
  return run_steps(net, cfg, ch, steps, s, launches, nullptr, status);
}

namespace {
// Reads and clears the device status word (synchronous).
int take_status(int *out) {
  int *d = pbn::device_status();
  if (!d) return fail(PBN_ERR_CUDA, "device status word unavailable");
  int v = 0;
  CUDA_TRY(cudaMemcpy(&v, d, sizeof v, cudaMemcpyDeviceToHost), "status read");
  if (v) CUDA_TRY(cudaMemset(d, 0, sizeof v), "status clear");
  *out = v;
  return PBN_OK;
}
}  // namespace

extern "C" int pbn_balance_phases(int32_t G, int32_t R, int32_t gpb, int32_t T, int32_t threads, int32_t n,
                                  int64_t k, int32_t launch[20], int32_t *split) {
  if (!launch || !split) return fail(PBN_ERR_INVALID, "NULL argument");
  if (G < 1 || R < 1 || gpb < 1 || threads < 1 || n < 1 || k < 0 || k > (int64_t)1 << 30)
    return fail(PBN_ERR_INVALID, "sizes must be positive, k at most 2^30 (G %d, R %d, gpb %d, threads %d, n %d, "
                "k %lld)", G, R, gpb, threads, n, (long long)k);
  if (T != 1 && T != 2 && T != 4) return fail(PBN_ERR_INVALID, "threads_per_item %d (1, 2 or 4)", T);
  LaunchPlan plan{};
  plan.gpb = gpb;
  plan.threads = threads;
  plan.T = T;
  plan.BPR = 1;
  pbn::SimArgs a1, a2;
  memset(&a1, 0, sizeof a1);
  memset(&a2, 0, sizeof a2);
  *split = 0;
  if (!balance_phases(G, R, plan, n, k, &a1, &a2)) return PBN_OK;
  const pbn::SimArgs *ph[2] = {&a1, &a2};
  for (int l = 0; l < 2; l++)
    for (int q = 0; q < 2; q++) {
      int32_t *o = launch + 10 * l + 5 * q;
      o[0] = ph[l]->seg_blocks[q];
      o[1] = ph[l]->seg_g0[q];
      o[2] = ph[l]->seg_ng[q];
      o[3] = ph[l]->seg_steps[q];
      o[4] = ph[l]->seg_soff[q];
    }
  *split = 1;
  return PBN_OK;
}

extern "C" int pbn_take_device_status(int *status) {
  if (!status) return fail(PBN_ERR_INVALID, "NULL argument");
  return take_status(status);
}

extern "C" {

const char *pbn_last_error(void) { return g_err.c_str(); }

const char *pbn_status_string(int status) {
  switch (status) {
    case PBN_OK: return "ok";
    case PBN_ERR_INVALID: return "invalid argument";
    case PBN_ERR_OOM: return "out of memory";
    case PBN_ERR_CUDA: return "CUDA error";
    case PBN_ERR_TIMEOUT: return "device wait timed out";
    case PBN_ERR_NOT_CONVERGED: return "not converged within the length cap";
    case PBN_ERR_INSUFFICIENT: return "window cannot give alpha and beta";
    case PBN_ERR_UNSUPPORTED: return "unsupported by this library";
    case PBN_ERR_CANCELLED: return "cancelled";
    default: return "unknown status";
  }
}

int pbn_load(const pbn_network_desc *d, pbn_net **out) {
  if (!d || !out) return fail(PBN_ERR_INVALID, "NULL argument");
  *out = nullptr;
  const int n = d->n;
  if (n < 1) return fail(PBN_ERR_INVALID, "n = %d", n);
  if (n > PBN_MAX_NODES) return fail(PBN_ERR_UNSUPPORTED, "n = %d exceeds %d", n, PBN_MAX_NODES);
  if (!d->fn_offset || !d->par_offset || !d->truth_table || !d->select_prob)
    return fail(PBN_ERR_INVALID, "NULL network array");
  if (!(d->p >= 0.0 && d->p < 1.0)) return fail(PBN_ERR_INVALID, "perturbation probability %g", d->p);
  const int F = d->n_functions;
  if (F < n) return fail(PBN_ERR_INVALID, "n_functions = %d for %d nodes", F, n);
  if (F > 65535) return fail(PBN_ERR_UNSUPPORTED, "F = %d exceeds 65535", F);
  // offsets first, so that every read below stays inside the arrays' stated
  // lengths: fn_offset [n+1], par_offset and tt_offset [F+1], the rest [F]
  // or par_offset[F] / tt_offset[F]
  if (d->fn_offset[0] != 0 || d->fn_offset[n] != F) return fail(PBN_ERR_INVALID, "fn_offset does not span F");
  for (int i = 0; i < n; i++) {
    const int l = d->fn_offset[i + 1] - d->fn_offset[i];
    if (l < 1) return fail(PBN_ERR_INVALID, "node %d has no predictor function", i);
    if (l > PBN_MAX_FUNCTIONS_PER_NODE)
      return fail(PBN_ERR_UNSUPPORTED, "node %d has %d functions (max %d)", i, l, PBN_MAX_FUNCTIONS_PER_NODE);
  }
  if (d->par_offset[0] != 0) return fail(PBN_ERR_INVALID, "par_offset[0] != 0");
  for (int f = 0; f < F; f++) {
    const int k = d->par_offset[f + 1] - d->par_offset[f];
    if (k < 0) return fail(PBN_ERR_INVALID, "par_offset decreasing at %d", f);
    if (k > PBN_MAX_PARENTS) return fail(PBN_ERR_UNSUPPORTED, "function %d has %d parents", f, k);
  }
  if (d->par_offset[F] > 0 && !d->parents) return fail(PBN_ERR_INVALID, "parents is NULL");
  if (d->tt_offset) {
    if (!d->tt_words) return fail(PBN_ERR_INVALID, "tt_words is NULL");
    if (d->tt_offset[0] < 0) return fail(PBN_ERR_INVALID, "tt_offset[0] < 0");
    for (int f = 0; f < F; f++)
      if (d->tt_offset[f + 1] < d->tt_offset[f]) return fail(PBN_ERR_INVALID, "tt_offset decreasing at %d", f);
  }
  const uint32_t P32 = quantise_p(d->p);
  const uint64_t span = 4294967296ull - P32;
  std::vector<uint4> fn(F);
  std::vector<uint32_t> node(n);
  std::vector<std::pair<uint64_t, int>> order(n);
  // tables of functions with more than 5 inputs, and their parents
  std::vector<uint32_t> wide_tt;
  std::vector<uint16_t> wide_par;
  int max_l = 0, max_k = 0;
  for (int i = 0; i < n; i++) {
    const int f0 = d->fn_offset[i], f1 = d->fn_offset[i + 1];
    const int l = f1 - f0;
    if (l < 1) return fail(PBN_ERR_INVALID, "node %d has no predictor function", i);
    if (l > PBN_MAX_FUNCTIONS_PER_NODE)
      return fail(PBN_ERR_UNSUPPORTED, "node %d has %d functions (max %d)", i, l, PBN_MAX_FUNCTIONS_PER_NODE);
    max_l = std::max(max_l, l);
    for (int f = f0; f < f1; f++) max_k = std::max(max_k, d->par_offset[f + 1] - d->par_offset[f]);
    double sum = 0.0, S = 0.0;
    uint64_t shape = (uint64_t)l;
    for (int f = f0; f < f1; f++) {
      const double c = d->select_prob[f];
      if (!(c >= 0.0 && c <= 1.0)) return fail(PBN_ERR_INVALID, "selection probability %g", c);
      sum += c;
      const int k = d->par_offset[f + 1] - d->par_offset[f];
      if (k < 0) return fail(PBN_ERR_INVALID, "par_offset decreasing at %d", f);
      if (k > PBN_MAX_PARENTS) return fail(PBN_ERR_UNSUPPORTED, "function %d has %d parents", f, k);
      shape = shape * 16 + (uint64_t)k;
      for (int m = 0; m < k; m++) {
        const int v = d->parents[d->par_offset[f] + m];
        if (v < 0 || v >= n) return fail(PBN_ERR_INVALID, "parent %d out of range", v);
      }
      const int words = k > 5 ? 1 << (k - 5) : 1;
      const uint32_t *tt;
      if (d->tt_offset) {
        if (!d->tt_words) return fail(PBN_ERR_INVALID, "tt_words is NULL");
        if (d->tt_offset[f + 1] - d->tt_offset[f] != words)
          return fail(PBN_ERR_INVALID, "function %d: %d table words for %d inputs (need %d)", f,
                      d->tt_offset[f + 1] - d->tt_offset[f], k, words);
        tt = d->tt_words + d->tt_offset[f];
      } else {
        if (k > 5) return fail(PBN_ERR_INVALID, "function %d has %d inputs: its table needs tt_offset/tt_words", f, k);
        tt = d->truth_table + f;
      }
      // upper category bound of function f (the last one of a node is 2^32, never compared)
      uint32_t T = 0xFFFFFFFFu;
      S += c;
      if (f < f1 - 1) {
        long long q = llround((double)span * S);
        if (q < 0) q = 0;
        if ((uint64_t)q > span) q = (long long)span;
        uint64_t t = (uint64_t)P32 + (uint64_t)q;
        T = t > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)t;
      }
      uint4 r;
      r.y = T;
      if (k <= 5) {
        int par[5] = {0, 0, 0, 0, 0};
        for (int m = 0; m < k; m++) par[m] = d->parents[d->par_offset[f] + m];
        // bits at or above 2^k are not part of the function; the kernels rely on them being 0
        r.x = k == 5 ? tt[0] : (tt[0] & ((1u << (1u << k)) - 1u));
        r.z = (uint32_t)par[0] | ((uint32_t)par[1] << 12) | (((uint32_t)par[4] & 0xFFu) << 24);
        r.w = (uint32_t)par[2] | ((uint32_t)par[3] << 12) | (((uint32_t)par[4] >> 8) << 24) | ((uint32_t)k << 28);
      } else {
        // wide function: x = first table word in wide_tt, z = first parent in wide_par
        r.x = (uint32_t)wide_tt.size();
        r.z = (uint32_t)wide_par.size();
        r.w = (uint32_t)k << 28;
        wide_tt.insert(wide_tt.end(), tt, tt + words);
        for (int m = 0; m < k; m++) wide_par.push_back((uint16_t)d->parents[d->par_offset[f] + m]);
      }
      fn[f] = r;
    }
    if (fabs(sum - 1.0) > 1e-9) return fail(PBN_ERR_INVALID, "selection probabilities of node %d sum to %.17g", i, sum);
    node[i] = (uint32_t)i | ((uint32_t)(l - 1) << 12) | ((uint32_t)f0 << 16);
    order[i] = std::make_pair(shape, i);
  }
  // processing order: nodes of the same shape (l, k of each function) next to
  // each other so a warp's threads take the same branches; the synchronous
  // update makes the order immaterial to the result.
  std::stable_sort(order.begin(), order.end(),
                   [](const std::pair<uint64_t, int> &a, const std::pair<uint64_t, int> &b) { return a.first < b.first; });
  // function records in processing order, so that a range of processing
  // positions is one contiguous range of records (a tile for TMA staging)
  std::vector<uint32_t> node_sorted(n);
  std::vector<uint4> fn_sorted((size_t)F);
  std::vector<int32_t> tiles(1, 0);
  int max_tile = 0;
  {
    int next = 0, tile_recs = 0;
    for (int r = 0; r < n; r++) {
      const int i = order[r].second;
      const int f0 = d->fn_offset[i], l = d->fn_offset[i + 1] - f0;
      if (tile_recs + l > pbn::kTileRecords) {
        tiles.push_back(r);
        max_tile = std::max(max_tile, tile_recs);
        tile_recs = 0;
      }
      for (int j = 0; j < l; j++) fn_sorted[(size_t)next + j] = fn[(size_t)f0 + j];
      node_sorted[r] = (uint32_t)i | ((uint32_t)(l - 1) << 12) | ((uint32_t)next << 16);
      next += l;
      tile_recs += l;
    }
    tiles.push_back(n);
    max_tile = std::max(max_tile, tile_recs);
  }
  pbn_net *net = new pbn_net();
  cudaGetDevice(&net->device);
  net->dev.n = n;
  net->dev.F = F;
  net->dev.P32 = P32;
  net->dev.max_l = max_l;
  net->dev.max_k = max_k;
  net->dev.ntiles = (int)tiles.size() - 1;
  net->dev.tile_bytes = max_tile * 16;
  // every table in one device allocation, filled by one copy: function
  // records, node records, tile starts, wide tables, wide parents (each
  // 16-byte aligned)
  auto up16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
  const size_t o_node = up16(sizeof(uint4) * (size_t)F);
  const size_t o_tiles = o_node + up16(sizeof(uint32_t) * (size_t)n);
  const size_t o_wtt = o_tiles + up16(sizeof(int32_t) * tiles.size());
  const size_t o_wpar = o_wtt + up16(sizeof(uint32_t) * wide_tt.size());
  const size_t total = o_wpar + up16(sizeof(uint16_t) * wide_par.size());
  std::vector<unsigned char> pack(total, 0);
  memcpy(pack.data(), fn_sorted.data(), sizeof(uint4) * (size_t)F);
  memcpy(pack.data() + o_node, node_sorted.data(), sizeof(uint32_t) * (size_t)n);
  memcpy(pack.data() + o_tiles, tiles.data(), sizeof(int32_t) * tiles.size());
  if (!wide_tt.empty()) {
    memcpy(pack.data() + o_wtt, wide_tt.data(), sizeof(uint32_t) * wide_tt.size());
    memcpy(pack.data() + o_wpar, wide_par.data(), sizeof(uint16_t) * wide_par.size());
  }
  cudaError_t e = cudaMalloc(&net->d_base, total);
  if (e == cudaSuccess) e = cudaMemcpy(net->d_base, pack.data(), total, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    pbn_free(net);
    return cuda_fail(e, "staging network tables");
  }
  unsigned char *base = static_cast<unsigned char *>(net->d_base);
  net->dev.d_fn = reinterpret_cast<uint4 *>(base);
  net->dev.d_node = reinterpret_cast<uint32_t *>(base + o_node);
  net->dev.d_tiles = reinterpret_cast<int32_t *>(base + o_tiles);
  if (!wide_tt.empty()) {
    net->dev.has_wide = 1;
    net->dev.d_wide_tt = reinterpret_cast<uint32_t *>(base + o_wtt);
    net->dev.d_wide_par = reinterpret_cast<uint16_t *>(base + o_wpar);
  }
  net->dev.table_bytes = (int64_t)F * 16 + (int64_t)n * 4 + (int64_t)wide_tt.size() * 4 + (int64_t)wide_par.size() * 2;
  *out = net;
  return PBN_OK;
}

void pbn_free(pbn_net *net) {
  if (!net) return;
  if (net->d_base) cudaFree(net->d_base);
  delete net;
}

int pbn_net_get_info(const pbn_net *net, pbn_net_info *out) {
  if (!net || !out) return fail(PBN_ERR_INVALID, "NULL argument");
  out->n = net->dev.n;
  out->n_functions = net->dev.F;
  out->perturb_threshold = net->dev.P32;
  out->table_bytes = net->dev.table_bytes;
  return PBN_OK;
}

int pbn_init_chains(const pbn_net *net, const pbn_run_cfg *cfg, pbn_chains *ch, void *stream) {
  if (!net || !cfg || !ch) return fail(PBN_ERR_INVALID, "NULL argument");
  if (ch->omega < 1 || !ch->state) return fail(PBN_ERR_INVALID, "chains: omega %lld, state %p", (long long)ch->omega, (void *)ch->state);
  CUDA_TRY(pbn::launch_init(net->dev, cfg->seed, ch->state, ch->omega, (cudaStream_t)stream), "init launch");
  ch->length = 0;
  return PBN_OK;
}

int pbn_run_chains(const pbn_net *net, const pbn_run_cfg *cfg, pbn_chains *ch, int64_t steps, void *stream) {
  if (!net || !cfg || !ch) return fail(PBN_ERR_INVALID, "NULL argument");
  if (ch->omega < 1 || !ch->state) return fail(PBN_ERR_INVALID, "chains not initialised");
  if (cfg->perturb_mode != PBN_PERTURB_PER_NODE && cfg->perturb_mode != PBN_PERTURB_GLOBAL)
    return fail(PBN_ERR_INVALID, "perturb_mode %d", cfg->perturb_mode);
  int rc = check_props(*cfg, net->dev.n);
  if (rc) return rc;
  return run_steps(net->dev, *cfg, *ch, steps, (cudaStream_t)stream);
}

static int check_window(const pbn_chains *ch, int64_t start, int64_t len) {
  if (!ch || !ch->bits) return fail(PBN_ERR_INVALID, "chains without bitstream");
  if (len < 1 || start < ch->bits_base || start + len - ch->bits_base > ch->bits_cap || start + len > ch->length)
    return fail(PBN_ERR_INVALID, "window [%lld, %lld) outside the recorded positions", (long long)start,
                (long long)(start + len));
  return PBN_OK;
}

int pbn_gelman_rubin(const pbn_chains *ch, int64_t start, int64_t psi, pbn_gr_result *out, void *stream) {
  int rc = check_window(ch, start, psi);
  if (rc) return rc;
  if (ch->omega < 2 || psi < 2) return fail(PBN_ERR_INVALID, "Gelman-Rubin needs omega >= 2 and psi >= 2");
  pbn::StatsScratch *sc;
  if ((rc = scratch_for((cudaStream_t)stream, &sc))) return rc;
  CUDA_TRY(pbn::launch_gelman_rubin(*ch, start - ch->bits_base, psi, out, *sc, (cudaStream_t)stream), "G&R launch");
  return PBN_OK;
}

int pbn_two_state(const pbn_chains *ch, int64_t start, int64_t len, double eps, double r, double s,
                  pbn_two_state_result *out, void *stream) {
  int rc = check_window(ch, start, len);
  if (rc) return rc;
  if (!(eps > 0 && r > 0 && s > 0 && s < 1)) return fail(PBN_ERR_INVALID, "eps, r, s out of range");
  pbn::StatsScratch *sc;
  if ((rc = scratch_for((cudaStream_t)stream, &sc))) return rc;
  CUDA_TRY(pbn::launch_two_state(*ch, start - ch->bits_base, len, eps, r, s, out, *sc, (cudaStream_t)stream),
           "two-state launch");
  return PBN_OK;
}

int pbn_skart(const pbn_chains *ch, int64_t start, int64_t kappa, int64_t bpc, int64_t spacer, double alpha_ci,
              double alpha_ran, pbn_skart_result *out, void *stream) {
  if (kappa < 1 || bpc < 1 || spacer < 0) return fail(PBN_ERR_INVALID, "kappa, batches, spacer");
  if (kappa > (1ll << 30)) return fail(PBN_ERR_UNSUPPORTED, "batch size above 2^30");
  if (bpc > (1ll << 32)) return fail(PBN_ERR_UNSUPPORTED, "batches per chain above 2^32");  // kappa * bpc < 2^63
  int rc = check_window(ch, start, kappa * bpc);
  if (rc) return rc;
  if (ch->omega * bpc < 2) return fail(PBN_ERR_INVALID, "Skart needs at least 2 batches");
  pbn::StatsScratch *sc;
  if ((rc = scratch_for((cudaStream_t)stream, &sc))) return rc;
  CUDA_TRY(pbn::launch_skart(*ch, start - ch->bits_base, kappa, bpc, spacer, alpha_ci, alpha_ran, out, *sc,
                             (cudaStream_t)stream),
           "Skart launch");
  return PBN_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ drivers

namespace {

// Device result slot of a driver query: one statistics result per property,
// the two-state results launched together with a Gelman & Rubin check at
// kAheadOffset, then the device status word.
constexpr size_t kResultBytes = 4096;
constexpr size_t kAheadOffset = 2048;
constexpr size_t kStatusOffset = kResultBytes - 64;
static_assert(sizeof(pbn_gr_result) * PBN_MAX_PROPERTIES <= kAheadOffset, "result slot");
static_assert(kAheadOffset + sizeof(pbn_two_state_result) * PBN_MAX_PROPERTIES <= kStatusOffset, "result slot");

// Per-(device, stream) driver workspace, kept across queries so that a query
// makes no allocation once the buffers have grown to its size: statistics
// scratch, a device result slot with its pinned host copy, chain state, two
// bitstream buffers (one is the copy target when the window must grow) and
// a pool of timing events.  One driver query at a time per workspace.
struct Workspace {
  std::mutex mu;
  pbn::StatsScratch sc;
  void *d_res = nullptr;
  void *h_res = nullptr;
  uint32_t *state = nullptr;
  size_t state_words = 0;
  uint32_t *bits[2] = {nullptr, nullptr};
  size_t bits_words[2] = {0, 0};
  int cur_bits = 0;
  std::vector<cudaEvent_t> events;
  bool ready = false;

  int setup(cudaStream_t s) {
    if (ready) return PBN_OK;
    CUDA_TRY(pbn::scratch_init(sc, s), "scratch");
    CUDA_TRY(cudaMalloc(&d_res, kResultBytes), "result alloc");
    CUDA_TRY(cudaMallocHost(&h_res, kResultBytes), "pinned alloc");
    ready = true;
    return PBN_OK;
  }

  int ensure(uint32_t *&buf, size_t &have, size_t words, cudaStream_t s, const char *what) {
    if (words <= have) return PBN_OK;
    if (buf) cudaFreeAsync(buf, s);
    buf = nullptr;
    have = 0;
    size_t w = std::max<size_t>(words, 1024);
    CUDA_TRY(cudaMallocAsync(&buf, w * sizeof(uint32_t), s), what);
    have = w;
    return PBN_OK;
  }

  cudaEvent_t event(size_t k) {
    while (events.size() <= k) {
      cudaEvent_t e = nullptr;
      if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
      events.push_back(e);
    }
    return events[k];
  }
};

std::mutex g_ws_mu;
std::map<std::pair<int, cudaStream_t>, std::unique_ptr<Workspace>> g_ws;

Workspace &workspace_for(cudaStream_t s) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_ws_mu);
  auto &slot = g_ws[std::make_pair(dev, s)];
  if (!slot) slot.reset(new Workspace());
  return *slot;
}

// Chains of one driver call on a borrowed workspace: state, a growing
// bitstream window and the statistics scratch.
struct Query {
  const pbn::NetDev &net;
  pbn_run_cfg cfg;
  cudaStream_t s;
  Workspace &ws;
  std::lock_guard<std::mutex> hold;
  pbn_chains ch;
  pbn::StatsScratch &sc;
  void *d_res = nullptr;
  size_t n_events = 0;   // events 0, 1: whole query; then start/stop pairs of simulation launches
  int64_t sim_launches = 0, kernel_launches = 0, sim_items = 0, d2h_bytes = 0;
  ApplyTiming apply_timing;
  bool unchecked = false;  // simulation launched since the status word was last read

  Query(const pbn::NetDev &n, cudaStream_t st)
      : net(n), s(st), ws(workspace_for(st)), hold(ws.mu), sc(ws.sc) {
    memset(&cfg, 0, sizeof cfg);
    memset(&ch, 0, sizeof ch);
  }

  int open(int64_t omega) {
    int rc = ws.setup(s);
    if (rc) return rc;
    d_res = ws.d_res;
    ch.omega = omega;
    const int G = (int)((omega + 31) / 32);
    if ((rc = ws.ensure(ws.state, ws.state_words, (size_t)G * net.n, s, "state alloc"))) return rc;
    ch.state = ws.state;
    cudaEvent_t e0 = ws.event(0), e1 = ws.event(1);
    if (!e0 || !e1) return fail(PBN_ERR_CUDA, "event creation failed");
    n_events = 2;
    CUDA_TRY(cudaEventRecord(e0, s), "event");
    CUDA_TRY(pbn::launch_init(net, cfg.seed, ch.state, omega, s), "init");
    kernel_launches++;
    ch.length = 0;
    return PBN_OK;
  }

  // Make the bitstream hold positions [base, upto): re-base in place when
  // nothing recorded at or after `base` must be kept, otherwise copy the kept
  // columns into the other buffer.
  int reserve(int64_t base, int64_t upto) {
    const int G = (int)((ch.omega + 31) / 32);
    const int rows = G * std::max(1, n_recorded_props(cfg));  // one bitstream per property, one after the other
    if (ch.bits && base >= ch.bits_base && upto - ch.bits_base <= ch.bits_cap) return PBN_OK;
    const int64_t keep_from = std::max(base, ch.bits_base);
    const int64_t kept =
        ch.bits ? std::max<int64_t>(0, std::min(ch.length, ch.bits_base + ch.bits_cap) - keep_from) : 0;
    int64_t cap = std::max<int64_t>(upto - base, 64);
    cap = std::max<int64_t>(cap, 2 * (ch.bits ? (ch.length - base) : 0));
    cap = (cap + 3) & ~int64_t(3);
    int target = ws.cur_bits;
    if (ch.bits && kept > 0) target ^= 1;   // copy source stays intact
    int rc = ws.ensure(ws.bits[target], ws.bits_words[target], (size_t)rows * cap, s, "bitstream alloc");
    if (rc) return rc;
    uint32_t *nb = ws.bits[target];
    if (ch.bits && kept > 0) {
      CUDA_TRY(cudaMemcpy2DAsync(nb + (keep_from - base), cap * 4, ch.bits + (keep_from - ch.bits_base),
                                 ch.bits_cap * 4, kept * 4, rows, cudaMemcpyDeviceToDevice, s),
               "bitstream copy");
    }
    ws.cur_bits = target;
    ch.bits = nb;
    ch.bits_cap = cap;
    ch.bits_base = base;
    return PBN_OK;
  }

  int extend_to(int64_t len, int64_t keep_from) {
    if (len <= ch.length) return PBN_OK;
    int rc = reserve(keep_from, len);
    if (rc) return rc;
    const int64_t steps = len - ch.length;
    cudaEvent_t a = ws.event(n_events), b = ws.event(n_events + 1);
    if (!a || !b) return fail(PBN_ERR_CUDA, "event creation failed");
    n_events += 2;
    sim_pairs.emplace_back(a, b);
    apply_timing.next = &Query::next_event;
    apply_timing.ctx = this;
    CUDA_TRY(cudaEventRecord(a, s), "event");
    int64_t launches = 0;
    rc = run_steps(net, cfg, ch, steps, s, &launches, &apply_timing);
    if (rc) return rc;
    CUDA_TRY(cudaEventRecord(b, s), "event");
    sim_launches += launches;
    kernel_launches += launches;
    unchecked = true;
    sim_items += steps * (int64_t)net.n * ((ch.omega + 31) / 32);
    return PBN_OK;
  }

  int stat_launched(int k) {
    kernel_launches += k;
    return PBN_OK;
  }

  // Result of the last statistics launch, read together with the device
  // status word (one synchronisation): a bounded wait that gave up during
  // the query fails it here.  ahead: also the two-state results at
  // kAheadOffset (count of them), in the same copy.
  template <typename T>
  int fetch(T *h, int count = 1, pbn_two_state_result *ahead = nullptr) {
    static_assert(sizeof(T) * PBN_MAX_PROPERTIES <= kStatusOffset, "result slot");
    int *status = pbn::device_status();
    if (!status) return fail(PBN_ERR_CUDA, "device status word unavailable");
    const size_t bytes = ahead ? kAheadOffset + sizeof(pbn_two_state_result) * count : sizeof(T) * count;
    CUDA_TRY(cudaEventRecord(ws.events[1], s), "event");  // the query's device time so far
    CUDA_TRY(cudaMemcpyAsync(ws.h_res, d_res, bytes, cudaMemcpyDeviceToHost, s), "result copy");
    CUDA_TRY(cudaMemcpyAsync((char *)ws.h_res + kStatusOffset, status, sizeof(int), cudaMemcpyDeviceToHost, s),
             "status copy");
    CUDA_TRY(cudaStreamSynchronize(s), "stream sync");
    memcpy(h, ws.h_res, sizeof(T) * count);
    if (ahead) memcpy(ahead, (char *)ws.h_res + kAheadOffset, sizeof(pbn_two_state_result) * count);
    d2h_bytes += bytes + sizeof(int);
    int st = 0;
    memcpy(&st, (char *)ws.h_res + kStatusOffset, sizeof st);
    unchecked = false;
    if (st) {
      CUDA_TRY(cudaMemset(status, 0, sizeof st), "status clear");
      return fail(st, "a bounded device wait gave up during the query");
    }
    return PBN_OK;
  }

  // End of a query: a bounded wait that gave up in a launch after the last
  // result read fails the query (the reads check the status word themselves).
  int final_status() {
    if (!unchecked) return PBN_OK;
    int st = 0;
    int rc = take_status(&st);
    if (rc) return rc;
    if (st) return fail(st, "a bounded device wait gave up during the query");
    unchecked = false;
    return PBN_OK;
  }

  // Property m's bitstream as a chain set of its own.
  pbn_chains view(int m) const {
    pbn_chains v = ch;
    v.bits = ch.bits + (size_t)m * ((ch.omega + 31) / 32) * ch.bits_cap;
    return v;
  }

  // Two-state statistics (Alg. 3's first check) launched with every Gelman &
  // Rubin check on the same window [psi, 2 psi) and read in the same
  // synchronisation: when R-hat converges, Alg. 3 starts on exactly that
  // window, so its first round needs no launch or read of its own.
  struct TwoStateAhead {
    double eps = 0, r = 0, s = 0;
    bool valid = false;  // results of the window [psi, 2 psi) of the returned psi
    pbn_two_state_result res[PBN_MAX_PROPERTIES];
  };

  // Alg. GR; with several properties psi doubles until every property's
  // R-hat is below the threshold (*rhat: the largest, rhat_each[m]: each).
  int gelman_rubin(int64_t psi0, double thr, int64_t max_length, int64_t *psi_out, double *rhat, int32_t *rounds,
                   double *rhat_each = nullptr, TwoStateAhead *ahead = nullptr) {
    const int q = std::max(1, n_recorded_props(cfg));
    int64_t psi = psi0;
    *rounds = 0;
    for (;;) {
      if (2 * psi > max_length) return fail(PBN_ERR_NOT_CONVERGED, "Gelman-Rubin not converged below length %lld", (long long)max_length);
      int rc = extend_to(2 * psi, psi);
      if (rc) return rc;
      for (int m = 0; m < q; m++)
        CUDA_TRY(pbn::launch_gelman_rubin(view(m), psi - ch.bits_base, psi, (pbn_gr_result *)d_res + m, sc, s),
                 "G&R");
      stat_launched(q);
      if (ahead) {
        for (int m = 0; m < q; m++)
          CUDA_TRY(pbn::launch_two_state(view(m), psi - ch.bits_base, psi, ahead->eps, ahead->r, ahead->s,
                                         (pbn_two_state_result *)((char *)d_res + kAheadOffset) + m, sc, s),
                   "two-state");
        stat_launched(q);
      }
      pbn_gr_result r[PBN_MAX_PROPERTIES];
      if ((rc = fetch(r, q, ahead ? ahead->res : nullptr))) return rc;
      if (ahead) ahead->valid = true;
      (*rounds)++;
      bool all = true;
      double worst = -INFINITY;
      for (int m = 0; m < q; m++) {
        if (rhat_each) rhat_each[m] = r[m].rhat;
        if (!(r[m].rhat < thr)) all = false;
        if (!(r[m].rhat <= worst)) worst = r[m].rhat;
      }
      *rhat = worst;
      if (all) { *psi_out = psi; return PBN_OK; }
      psi *= 2;
    }
  }

  // Device time of the query: from its first launch to the last result read
  // (event 1 is recorded with every read, which synchronises after it), or
  // to now when launches followed the last read.
  double elapsed_ms() {
    float ms = 0.f;
    if (unchecked) {
      cudaEventRecord(ws.events[1], s);
      cudaEventSynchronize(ws.events[1]);
    }
    cudaEventElapsedTime(&ms, ws.events[0], ws.events[1]);
    return ms;
  }

  // events 2.. hold (start, stop) pairs around each run of steps; the apply
  // launches' pairs are drawn from the same pool, so the two sets are kept apart
  double sim_ms() {
    double total = 0.0;
    for (const auto &pr : sim_pairs) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) total += ms;
    }
    return total;
  }

  double apply_ms() {
    double total = 0.0;
    for (const auto &pr : apply_timing.pairs) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) total += ms;
    }
    return total;
  }

  static cudaEvent_t next_event(void *ctx) {
    Query *q = static_cast<Query *>(ctx);
    return q->ws.event(q->n_events++);
  }
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> sim_pairs;
};

int check_query_common(const pbn_net *net, int64_t omega, int64_t psi0, double thr, int64_t max_length,
                       int mode, const pbn_soi &soi) {
  if (!net) return fail(PBN_ERR_INVALID, "NULL network");
  if (omega < 2) return fail(PBN_ERR_INVALID, "omega must be >= 2");
  if (psi0 < 2) return fail(PBN_ERR_INVALID, "psi0 must be >= 2");
  if (!(thr > 0)) return fail(PBN_ERR_INVALID, "R-hat threshold");
  if (max_length < 2 * psi0) return fail(PBN_ERR_INVALID, "max_length below 2 psi0");
  if (mode != PBN_PERTURB_PER_NODE && mode != PBN_PERTURB_GLOBAL) return fail(PBN_ERR_INVALID, "perturb_mode");
  if ((int64_t)((omega + 31) / 32) > (1ll << 31) - 1) return fail(PBN_ERR_UNSUPPORTED, "omega too large");
  return check_soi(soi, net->dev.n, false);
}

}  // namespace

namespace {

// Alg. GR then Alg. 3 for one property, or for several properties from the
// same trajectories (Sec. 4.2, last part): psi doubles until every
// property's R-hat is below the threshold; every round counts every
// property; the chains grow by the smallest deficit among the properties
// whose N exceeds the merged sample until none does; the burn-in check takes
// the largest M.  With one property every step is Alg. 3's.  `out` carries
// the common fields and property 0's estimate; each[m] (if given) every
// property's.
int two_state_driver(const pbn_net *net, const pbn_two_state_query *q, int n_props, const pbn_soi *props,
                     pbn_two_state_report *out, pbn_property_result *each, void *stream) {
  if (!q || !out) return fail(PBN_ERR_INVALID, "NULL argument");
  int rc = check_query_common(net, q->omega, q->psi0, q->rhat_threshold, q->max_length, q->perturb_mode,
                              n_props > 0 ? props[0] : q->soi);
  if (rc) return rc;
  if (!(q->eps > 0 && q->r > 0 && q->s > 0 && q->s < 1)) return fail(PBN_ERR_INVALID, "eps, r, s out of range");
  memset(out, 0, sizeof *out);
  Query Q(net->dev, (cudaStream_t)stream);
  Q.cfg.seed = q->seed;
  Q.cfg.perturb_mode = q->perturb_mode;
  if (n_props > 0) {
    Q.cfg.n_props = n_props;
    Q.cfg.props = props;
  } else {
    Q.cfg.soi = q->soi;
  }
  if ((rc = check_props(Q.cfg, net->dev.n))) return rc;
  const int np = std::max(1, n_props);
  if ((rc = Q.open(q->omega))) return rc;
  int64_t psi;
  double rhat_each[PBN_MAX_PROPERTIES];
  Query::TwoStateAhead ahead;
  ahead.eps = q->eps;
  ahead.r = q->r;
  ahead.s = q->s;
  if ((rc = Q.gelman_rubin(q->psi0, q->rhat_threshold, q->max_length, &psi, &out->rhat, &out->gr_rounds,
                           rhat_each, &ahead)))
    return rc;
  out->gr_psi = psi;
  const int64_t omega = q->omega;
  pbn_two_state_result r[PBN_MAX_PROPERTIES];
  memset(r, 0, sizeof r);
  for (;;) {      // burn-in check (Alg. 3: M against psi)
    for (;;) {    // sample-size check (Alg. 3: N against the merged sample)
      int64_t n = Q.ch.length - psi;
      if (n < 2) {
        if (psi + 2 > q->max_length) return fail(PBN_ERR_NOT_CONVERGED, "two-state: length cap");
        if ((rc = Q.extend_to(psi + 2, psi))) return rc;
        continue;
      }
      pbn_two_state_result got[PBN_MAX_PROPERTIES];
      if (ahead.valid && n == psi) {
        // the window of the converged Gelman & Rubin check: read with it
        memcpy(got, ahead.res, sizeof(pbn_two_state_result) * np);
      } else {
        for (int m = 0; m < np; m++)
          CUDA_TRY(pbn::launch_two_state(Q.view(m), psi - Q.ch.bits_base, n, q->eps, q->r, q->s,
                                         (pbn_two_state_result *)Q.d_res + m, Q.sc, Q.s),
                   "two-state");
        Q.stat_launched(np);
        if ((rc = Q.fetch(got, np))) return rc;
      }
      ahead.valid = false;
      out->ts_rounds++;
      bool insufficient = false;
      for (int m = 0; m < np; m++) insufficient |= got[m].status == PBN_ERR_INSUFFICIENT;
      if (insufficient) {
        if (Q.ch.length + n > q->max_length) return fail(PBN_ERR_NOT_CONVERGED, "two-state: no transitions below the length cap");
        if ((rc = Q.extend_to(Q.ch.length + n, psi))) return rc;
        continue;
      }
      int64_t smallest = -1;
      for (int m = 0; m < np; m++) {
        if (got[m].status != PBN_OK) return fail(got[m].status, "two-state chain is periodic (alpha = beta = 1)");
        r[m] = got[m];
        const int64_t deficit = r[m].N - omega * n;
        if (deficit > 0 && (smallest < 0 || deficit < smallest)) smallest = deficit;
      }
      if (smallest < 0) break;
      const int64_t extend_by = (smallest + omega - 1) / omega;
      if (Q.ch.length + extend_by > q->max_length) return fail(PBN_ERR_NOT_CONVERGED, "two-state: length cap");
      if ((rc = Q.extend_to(Q.ch.length + extend_by, psi))) return rc;
    }
    int64_t Mmax = r[0].M;
    for (int m = 1; m < np; m++) Mmax = std::max(Mmax, r[m].M);
    if (Mmax > psi) { psi = Mmax; continue; }
    break;
  }
  out->prob = r[0].prob;
  out->alpha = r[0].alpha;
  out->beta = r[0].beta;
  out->M = r[0].M;
  out->N = r[0].N;
  out->ones = r[0].ones;
  out->n4[0] = r[0].n00; out->n4[1] = r[0].n01; out->n4[2] = r[0].n10; out->n4[3] = r[0].n11;
  for (int m = 0; each && m < np; m++) {
    pbn_property_result &e = each[m];
    e.prob = r[m].prob;
    e.alpha = r[m].alpha;
    e.beta = r[m].beta;
    e.rhat = rhat_each[m];
    e.M = r[m].M;
    e.N = r[m].N;
    e.ones = r[m].ones;
    e.n4[0] = r[m].n00; e.n4[1] = r[m].n01; e.n4[2] = r[m].n10; e.n4[3] = r[m].n11;
  }
  if ((rc = Q.final_status())) return rc;
  out->psi = psi;
  out->length = Q.ch.length;
  out->sample_size = omega * (Q.ch.length - psi);
  out->chain_node_updates = omega * Q.ch.length * (int64_t)net->dev.n;
  out->device_ms = Q.elapsed_ms();
  out->sim_ms = Q.sim_ms();
  out->sim_launches = Q.sim_launches;
  out->apply_ms = Q.apply_ms();
  out->apply_launches = (int64_t)Q.apply_timing.pairs.size();
  out->kernel_launches = Q.kernel_launches;
  out->sim_items = Q.sim_items;
  out->d2h_bytes = Q.d2h_bytes;
  return PBN_OK;
}

}  // namespace

extern "C" int pbn_estimate_two_state(const pbn_net *net, const pbn_two_state_query *q, pbn_two_state_report *out,
                                      void *stream) {
  return two_state_driver(net, q, 0, nullptr, out, nullptr, stream);
}

extern "C" int pbn_estimate_two_state_seq(const pbn_net *net, const pbn_two_state_seq_query *q,
                                          pbn_two_state_seq_report *out, void *stream) {
  if (!net || !q || !out) return fail(PBN_ERR_INVALID, "NULL argument");
  if (q->m0 < 0 || q->n0 < 2) return fail(PBN_ERR_INVALID, "m0 %lld (>= 0), n0 %lld (>= 2)", (long long)q->m0,
                                          (long long)q->n0);
  if (q->perturb_mode != PBN_PERTURB_PER_NODE && q->perturb_mode != PBN_PERTURB_GLOBAL)
    return fail(PBN_ERR_INVALID, "perturb_mode %d", q->perturb_mode);
  if (!(q->eps > 0 && q->r > 0 && q->s > 0 && q->s < 1)) return fail(PBN_ERR_INVALID, "eps, r, s out of range");
  int rc = check_soi(q->soi, net->dev.n, false);
  if (rc) return rc;
  memset(out, 0, sizeof *out);
  Query Q(net->dev, (cudaStream_t)stream);
  Q.cfg.seed = q->seed;
  Q.cfg.perturb_mode = q->perturb_mode;
  Q.cfg.soi = q->soi;
  if ((rc = Q.open(1))) return rc;
  // The whole trajectory stays recorded: the final window (last N) may start
  // before the last alpha, beta window when N grows while M shrinks.
  int64_t M = q->m0, N = q->n0, l = M + N;
  if (l > q->max_length) return fail(PBN_ERR_NOT_CONVERGED, "sequential two-state: length cap");
  if ((rc = Q.extend_to(l, 0))) return rc;
  pbn_two_state_result r;
  for (;;) {
    if (M + N > l) {
      if (M + N > q->max_length) return fail(PBN_ERR_NOT_CONVERGED, "sequential two-state: length cap");
      if ((rc = Q.extend_to(M + N, 0))) return rc;
      l = M + N;
    }
    out->rounds++;
    CUDA_TRY(pbn::launch_two_state(Q.ch, l - N - Q.ch.bits_base, N, q->eps, q->r, q->s,
                                   (pbn_two_state_result *)Q.d_res, Q.sc, Q.s),
             "two-state");
    Q.stat_launched(1);
    if ((rc = Q.fetch(&r))) return rc;
    out->n4[0] = r.n00; out->n4[1] = r.n01; out->n4[2] = r.n10; out->n4[3] = r.n11;
    out->ab_window = N;
    if (r.status == PBN_ERR_INSUFFICIENT) {
      N = 2 * N;
      continue;
    }
    if (r.status != PBN_OK) return fail(r.status, "two-state chain is periodic (alpha = beta = 1)");
    out->alpha = r.alpha;
    out->beta = r.beta;
    M = r.M;
    N = r.N;
    if (M + N <= l) break;
  }
  // the estimate over the last N positions (the kernel's ones count; its
  // two-state status does not matter here)
  CUDA_TRY(pbn::launch_two_state(Q.ch, l - N - Q.ch.bits_base, N, q->eps, q->r, q->s,
                                 (pbn_two_state_result *)Q.d_res, Q.sc, Q.s),
           "two-state");
  Q.stat_launched(1);
  if ((rc = Q.fetch(&r))) return rc;
  if ((rc = Q.final_status())) return rc;
  out->ones = r.ones;
  out->prob = (double)r.ones / (double)N;
  out->M = M;
  out->N = N;
  out->length = l;
  out->chain_node_updates = l * (int64_t)net->dev.n;
  out->device_ms = Q.elapsed_ms();
  out->sim_ms = Q.sim_ms();
  out->sim_launches = Q.sim_launches;
  out->kernel_launches = Q.kernel_launches;
  out->d2h_bytes = Q.d2h_bytes;
  return PBN_OK;
}

extern "C" int pbn_estimate_two_state_multi(const pbn_net *net, const pbn_two_state_query *q, int32_t n_props,
                                            const pbn_soi *props, pbn_two_state_report *out,
                                            pbn_property_result *each, void *stream) {
  if (n_props < 1 || n_props > PBN_MAX_PROPERTIES || !props)
    return fail(PBN_ERR_INVALID, "n_props %d (1 .. %d) or props NULL", n_props, PBN_MAX_PROPERTIES);
  return two_state_driver(net, q, n_props, props, out, each, stream);
}

// Alg. 2 (Sec. 3.2) on chain 0 of the seed's family, with the same constants
// as the parallel driver below (placeholders for the Skart reference):
// skewness of the last 1024 of 1280 samples; the randomness test on the whole
// trajectory's batch means with spacer d; then the CI on the p' = p - d
// nonspaced batches after the skipped d kappa samples, eta := kappa (p' + d).
extern "C" int pbn_estimate_skart_seq(const pbn_net *net, const pbn_skart_query *q, pbn_skart_report *out,
                                      void *stream) {
  if (!net || !q || !out) return fail(PBN_ERR_INVALID, "NULL argument");
  if (q->perturb_mode != PBN_PERTURB_PER_NODE && q->perturb_mode != PBN_PERTURB_GLOBAL)
    return fail(PBN_ERR_INVALID, "perturb_mode %d", q->perturb_mode);
  if (!(q->H_star > 0 && q->alpha > 0 && q->alpha < 1)) return fail(PBN_ERR_INVALID, "H_star, alpha");
  int rc = check_soi(q->soi, net->dev.n, false);
  if (rc) return rc;
  memset(out, 0, sizeof *out);
  Query Q(net->dev, (cudaStream_t)stream);
  Q.cfg.seed = q->seed;
  Q.cfg.perturb_mode = q->perturb_mode;
  Q.cfg.soi = q->soi;
  if ((rc = Q.open(1))) return rc;
  int64_t eta = 1280;
  const int64_t l = 1024;
  if (eta > q->max_length) return fail(PBN_ERR_NOT_CONVERGED, "sequential Skart: length cap");
  if ((rc = Q.extend_to(eta, 0))) return rc;
  pbn_skart_result sk;
  // skewness of the last l samples: batch size 1, one batch per sample
  CUDA_TRY(pbn::launch_skart(Q.ch, eta - l - Q.ch.bits_base, 1, l, 0, q->alpha, 0.20, (pbn_skart_result *)Q.d_res,
                             Q.sc, Q.s),
           "Skart");
  Q.stat_launched(2);
  if ((rc = Q.fetch(&sk))) return rc;
  int64_t kappa = fabs(sk.skew) > 4.0 ? 16 : 1;
  int64_t p = eta;
  eta = kappa * p;
  int64_t d = 0;
  const double alpha_ran = 0.20;
  for (;;) {  // randomness test on the whole trajectory
    if (eta > q->max_length) return fail(PBN_ERR_NOT_CONVERGED, "sequential Skart: length cap");
    if ((rc = Q.extend_to(eta, 0))) return rc;
    CUDA_TRY(pbn::launch_skart(Q.ch, 0 - Q.ch.bits_base, kappa, p, d, q->alpha, alpha_ran,
                               (pbn_skart_result *)Q.d_res, Q.sc, Q.s),
             "Skart");
    Q.stat_launched(2);
    if ((rc = Q.fetch(&sk))) return rc;
    out->rand_rounds++;
    if (sk.vn_pass) break;
    d += 1;
    if (d > 10) {
      d = 0;
      kappa = (int64_t)ceil(sqrt(2.0) * (double)kappa);
      p = (int64_t)ceil(0.9 * (double)p);
    }
    eta = kappa * p;
  }
  out->spacer = d;
  int64_t pp = p - d;  // batches after the d skipped ones
  if (pp < 2) return fail(PBN_ERR_NOT_CONVERGED, "sequential Skart: fewer than 2 batches after the spacer");
  for (;;) {  // CI loop
    eta = kappa * (pp + d);
    if (eta > q->max_length) return fail(PBN_ERR_NOT_CONVERGED, "sequential Skart: length cap");
    if (kappa > (1ll << 30)) return fail(PBN_ERR_UNSUPPORTED, "Skart batch size above 2^30");
    if ((rc = Q.extend_to(eta, 0))) return rc;
    CUDA_TRY(pbn::launch_skart(Q.ch, d * kappa - Q.ch.bits_base, kappa, pp, 0, q->alpha, alpha_ran,
                               (pbn_skart_result *)Q.d_res, Q.sc, Q.s),
             "Skart");
    Q.stat_launched(2);
    if ((rc = Q.fetch(&sk))) return rc;
    out->ci_rounds++;
    out->mean = sk.mean; out->ci_lo = sk.ci_lo; out->ci_hi = sk.ci_hi; out->H = sk.H;
    out->var = sk.var; out->skew = sk.skew; out->phi = sk.phi;
    const double Hs = q->relative ? q->H_star * fabs(sk.mean) : q->H_star;
    if (!(sk.H > Hs)) break;
    const double f = (sk.H / Hs) * (sk.H / Hs);
    const int64_t pmax = pp > 1024 ? pp : 1024;
    const double pf = ceil(f * (double)pp);
    const int64_t p1 = pf > (double)pmax ? pmax : (int64_t)pf;
    int64_t k1 = (int64_t)ceil((double)kappa * f * (double)pp / (double)p1);
    if (k1 < kappa) k1 = kappa;
    kappa = k1;
    pp = p1;
  }
  if ((rc = Q.final_status())) return rc;
  out->psi = d * kappa;
  out->length = Q.ch.length;
  out->kappa = kappa;
  out->batches = pp;
  out->sample_size = kappa * pp;
  out->chain_node_updates = Q.ch.length * (int64_t)net->dev.n;
  out->device_ms = Q.elapsed_ms();
  out->sim_ms = Q.sim_ms();
  out->sim_launches = Q.sim_launches;
  out->apply_ms = Q.apply_ms();
  out->apply_launches = (int64_t)Q.apply_timing.pairs.size();
  out->kernel_launches = Q.kernel_launches;
  out->sim_items = Q.sim_items;
  out->d2h_bytes = Q.d2h_bytes;
  return PBN_OK;
}

extern "C" int pbn_estimate_skart(const pbn_net *net, const pbn_skart_query *q, pbn_skart_report *out, void *stream) {
  if (!q || !out) return fail(PBN_ERR_INVALID, "NULL argument");
  int rc = check_query_common(net, q->omega, q->psi0, q->rhat_threshold, q->max_length, q->perturb_mode, q->soi);
  if (rc) return rc;
  if (!(q->H_star > 0 && q->alpha > 0 && q->alpha < 1)) return fail(PBN_ERR_INVALID, "H_star, alpha");
  memset(out, 0, sizeof *out);
  Query Q(net->dev, (cudaStream_t)stream);
  Q.cfg.seed = q->seed;
  Q.cfg.perturb_mode = q->perturb_mode;
  Q.cfg.soi = q->soi;
  if ((rc = Q.open(q->omega))) return rc;
  int64_t psi;
  if ((rc = Q.gelman_rubin(q->psi0, q->rhat_threshold, q->max_length, &psi, &out->rhat, &out->gr_rounds))) return rc;
  const int64_t omega = q->omega;
  const int64_t start = psi;  // the first psi samples of every chain are skipped
  auto cdiv = [](int64_t a, int64_t b) { return (a + b - 1) / b; };
  int64_t eta = cdiv(1280, omega) * omega;
  // initial skewness of all eta samples: batch size 1, one batch per sample
  if ((rc = Q.extend_to(start + eta / omega, start))) return rc;
  pbn_skart_result sk;
  CUDA_TRY(pbn::launch_skart(Q.ch, start - Q.ch.bits_base, 1, eta / omega, 0, q->alpha, 0.20,
                             (pbn_skart_result *)Q.d_res, Q.sc, Q.s),
           "Skart");
  Q.stat_launched(2);
  if ((rc = Q.fetch(&sk))) return rc;
  int64_t kappa = fabs(sk.skew) > 4.0 ? 16 : 1;
  int64_t p = cdiv(eta, omega) * omega;
  eta = kappa * p;
  int64_t d = 0;
  const double alpha_ran = 0.20;
  for (;;) {  // randomness test loop
    if (start + eta / omega > q->max_length) return fail(PBN_ERR_NOT_CONVERGED, "Skart: length cap");
    if ((rc = Q.extend_to(start + eta / omega, start))) return rc;
    CUDA_TRY(pbn::launch_skart(Q.ch, start - Q.ch.bits_base, kappa, p / omega, d, q->alpha, alpha_ran,
                               (pbn_skart_result *)Q.d_res, Q.sc, Q.s),
             "Skart");
    Q.stat_launched(2);
    if ((rc = Q.fetch(&sk))) return rc;
    out->rand_rounds++;
    if (sk.vn_pass) break;
    d += 1;
    if (d > 10) {
      d = 0;
      kappa = (int64_t)ceil(sqrt(2.0) * (double)kappa);
      p = (int64_t)ceil(0.9 * (double)p);
    }
    p = cdiv(p, omega) * omega;
    eta = kappa * p;
  }
  out->spacer = d;
  for (;;) {  // CI loop
    if (start + eta / omega > q->max_length) return fail(PBN_ERR_NOT_CONVERGED, "Skart: length cap");
    if (kappa > (1ll << 30)) return fail(PBN_ERR_UNSUPPORTED, "Skart batch size above 2^30");
    if ((rc = Q.extend_to(start + eta / omega, start))) return rc;
    CUDA_TRY(pbn::launch_skart(Q.ch, start - Q.ch.bits_base, kappa, p / omega, 0, q->alpha, alpha_ran,
                               (pbn_skart_result *)Q.d_res, Q.sc, Q.s),
             "Skart");
    Q.stat_launched(2);
    if ((rc = Q.fetch(&sk))) return rc;
    out->ci_rounds++;
    out->mean = sk.mean; out->ci_lo = sk.ci_lo; out->ci_hi = sk.ci_hi; out->H = sk.H;
    out->var = sk.var; out->skew = sk.skew; out->phi = sk.phi;
    const double Hs = q->relative ? q->H_star * fabs(sk.mean) : q->H_star;
    if (!(sk.H > Hs)) break;
    const double f = (sk.H / Hs) * (sk.H / Hs);
    const int64_t pmax = p > 1024 ? p : 1024;
    const double pf = ceil(f * (double)p);
    const int64_t p1 = pf > (double)pmax ? pmax : (int64_t)pf;
    int64_t k1 = (int64_t)ceil((double)kappa * f * (double)p / (double)p1);
    if (k1 < kappa) k1 = kappa;
    kappa = k1;
    p = cdiv(p1, omega) * omega;
    eta = kappa * p;
  }
  if ((rc = Q.final_status())) return rc;
  out->psi = psi;
  out->length = Q.ch.length;
  out->kappa = kappa;
  out->batches = p;
  out->sample_size = kappa * p;
  out->chain_node_updates = omega * Q.ch.length * (int64_t)net->dev.n;
  out->device_ms = Q.elapsed_ms();
  out->sim_ms = Q.sim_ms();
  out->sim_launches = Q.sim_launches;
  out->apply_ms = Q.apply_ms();
  out->apply_launches = (int64_t)Q.apply_timing.pairs.size();
  out->kernel_launches = Q.kernel_launches;
  out->sim_items = Q.sim_items;
  out->d2h_bytes = Q.d2h_bytes;
  return PBN_OK;
}
