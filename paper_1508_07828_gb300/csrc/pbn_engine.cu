// Batched and served queries (the engine of include/pbn.h).
//
// Many independent queries share the GPU.  Each query is one run of Alg. GR
// followed by Alg. 3 (two-state) or Alg. 4 (Skart) on its own network, state
// of interest, chain count and seed.  Its chain state and indicator
// bitstream stay resident in device memory from admission to completion.
// Work proceeds in epochs:
//   1. the host plans, for every active query, how far to extend its chains
//      this epoch (up to its next check, at most S transitions) and which
//      queries are at a check;
//   2. one persistent simulation launch (batch_sim_kernel) pulls
//      (query, chain-group range) work items from an atomic counter, each CTA
//      staging that query's tables and states in shared memory and running
//      the same step code as the single-query kernel;
//   3. one persistent statistics launch (batch_stats_kernel) computes the
//      Gelman & Rubin or two-state statistics of every query at a check, each
//      request split into virtual blocks whose exact partial sums the last
//      one folds; Skart checks run as their own launches afterwards;
//   4. the host applies each query's stopping rule (the same decisions, in
//      the same order, as pbn_estimate_two_state / pbn_estimate_skart),
//      retires finished queries and admits waiting ones as slots and the
//      device-memory budget allow.
// Steps 2 and 3, with the copies of the epoch's plan in and the results out,
// form a CUDA graph captured once and replayed every epoch.  The autotuner
// times live epochs under candidate (transitions per epoch, threads per CTA,
// items per thread) settings and keeps the fastest; results do not depend
// on the setting.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <deque>
#include <memory>
#include <mutex>
#include <vector>

#include "pbn_stats.cuh"
#include "pbn_step.cuh"

namespace pbn {

struct BatchItem {
  int32_t task, g0, ngl, pad;
};

enum { REQ_GR = 0, REQ_TS = 1 };

struct StatReq {
  int32_t kind, nblocks, block0, G;
  const uint32_t *bits;
  int64_t cap, col, len, omega;
  double eps, r, s;
};

union ReqOut {
  pbn_gr_result gr;
  pbn_two_state_result ts;
};

constexpr int kReqBlocks = 64;   // most virtual blocks of one statistics request
// Statistics requests per query and epoch: a two-state query at its Gelman &
// Rubin check also asks for the first two-state counts of the same window.
constexpr int kReqPerQuery = 2;
// With a latency bound (pbn_engine_cfg.epoch_target_ms) an epoch's extension
// of a query is never below kMinEpochSteps transitions.
constexpr int64_t kMinEpochSteps = 64;
// At most this many queries to extend in an epoch for the light-load path.
constexpr int kAloneMax = 4;
constexpr int kCounters = 8;     // items, next item, virtual blocks, next virtual block, requests

// ------------------------------------------------------------------ kernels

// At most 80 registers (a few bytes spill), so that three 256-thread CTAs
// share an SM: 24 warps to hide the dependent Philox rounds, against 16 when
// the compiler takes 108.
__global__ void __maxnreg__(80) batch_sim_kernel(const SimArgs *__restrict__ tasks,
                                                        const BatchItem *__restrict__ items, int *counters) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(16) SimArgs s_task;
  __shared__ int s_it;
  const int count = counters[0];
  for (;;) {
    if (threadIdx.x == 0) s_it = atomicAdd(&counters[1], 1);
    __syncthreads();
    const int it = s_it;
    if (it >= count) break;
    const BatchItem w = items[it];
    const uint32_t *src = reinterpret_cast<const uint32_t *>(tasks + w.task);
    for (int k = threadIdx.x; k < (int)(sizeof(SimArgs) / 4); k += blockDim.x)
      reinterpret_cast<uint32_t *>(&s_task)[k] = src[k];
    __syncthreads();
    const RoundKeys rk = s_task.rk;
    if (s_task.mode == PBN_PERTURB_PER_NODE)
      cta_simulate<PBN_PERTURB_PER_NODE, 1, 1, true>(s_task, rk, (uint32_t)w.g0, w.ngl, s_task.gpb, smem, s_task.steps, 0);
    else
      cta_simulate<PBN_PERTURB_GLOBAL, 1, 1, true>(s_task, rk, (uint32_t)w.g0, w.ngl, s_task.gpb, smem, s_task.steps, 0);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) batch_stats_kernel(const StatReq *__restrict__ reqs, int *counters,
                                                          unsigned long long *partials, unsigned int *tickets,
                                                          ReqOut *out) {
  __shared__ int s_vb;
  __shared__ bool s_last;
  __shared__ unsigned long long red[32][3];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int total = counters[2], nreq = counters[4];
  for (;;) {
    if (threadIdx.x == 0) s_vb = atomicAdd(&counters[3], 1);
    __syncthreads();
    const int vb = s_vb;
    if (vb >= total) break;
    int lo = 0, hi = nreq - 1;   // the request whose blocks contain vb
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (reqs[mid].block0 <= vb) lo = mid; else hi = mid - 1;
    }
    const StatReq q = reqs[lo];
    const int lb = vb - q.block0;
    uint64_t v[4] = {0, 0, 0, 0};
    if (q.kind == REQ_GR) {
      uint64_t s1 = 0;
      u128 s2 = 0;
      for (int64_t g = (int64_t)lb * wpb + w; g < q.G; g += (int64_t)q.nblocks * wpb) {
        const uint32_t *row = q.bits + (size_t)g * q.cap + q.col;
        uint32_t cnt = 0;
        for (int64_t j = 0; j < q.len; j += 32) {
          const uint32_t x = (j + lane < q.len) ? row[j + lane] : 0u;
          cnt += __popc(warp_transpose32(x, lane));
        }
        if (!((group_lanes(q.omega, g) >> lane) & 1u)) cnt = 0;
        s1 += warp_sum<uint64_t>(cnt);
        s2 += warp_sum_u128((u128)((uint64_t)cnt * cnt));
      }
      if (lane == 0) {
        red[w][0] = s1;
        red[w][1] = (uint64_t)s2;
        red[w][2] = (uint64_t)(s2 >> 64);
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        uint64_t a = 0;
        u128 b = 0;
        for (int k = 0; k < wpb; k++) {
          a += red[k][0];
          b += ((u128)red[k][2] << 64) | red[k][1];
        }
        v[0] = a;
        v[1] = (uint64_t)b;
        v[2] = (uint64_t)(b >> 64);
      }
    } else {
      const int64_t chunks = (q.len + 31) / 32;
      const int64_t nitems = (int64_t)q.G * chunks;
      for (int64_t it = (int64_t)lb * wpb + w; it < nitems; it += (int64_t)q.nblocks * wpb) {
        const int64_t g = it / chunks, ch = it - g * chunks;
        const uint32_t vm = group_lanes(q.omega, g);
        const uint32_t *row = q.bits + (size_t)g * q.cap + q.col;
        const int64_t j = ch * 32 + lane;
        const uint32_t x = j < q.len ? (row[j] & vm) : 0u;
        uint32_t nx = __shfl_down_sync(0xFFFFFFFFu, x, 1);
        if (lane == 31) nx = (j + 1 < q.len) ? (row[j + 1] & vm) : 0u;
        v[3] += __popc(x);
        if (j + 1 < q.len) {
          v[0] += __popc(x & nx);
          v[1] += __popc(x);
          v[2] += __popc(nx);
        }
      }
      block_sum64<4>(v);
    }
    if (threadIdx.x == 0) {
      unsigned long long *slot = partials + ((size_t)lo * kReqBlocks + lb) * 4;
      for (int k = 0; k < 4; k++) slot[k] = v[k];
      __threadfence();
      const unsigned int t = atomicAdd(&tickets[lo], 1u);
      s_last = (t == (unsigned)q.nblocks - 1u);
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
      __threadfence();
      const unsigned long long *base = partials + (size_t)lo * kReqBlocks * 4;
      tickets[lo] = 0u;
      if (q.kind == REQ_GR) {
        uint64_t S1 = 0;
        u128 S2 = 0;
        for (int b = 0; b < q.nblocks; b++) {
          S1 += base[b * 4];
          S2 += ((u128)base[b * 4 + 2] << 64) | base[b * 4 + 1];
        }
        pbn_gr_result r;
        gr_formulas(r, S1, S2, q.len, q.omega);
        out[lo].gr = r;
      } else {
        uint64_t t[4] = {0, 0, 0, 0};
        for (int b = 0; b < q.nblocks; b++)
          for (int k = 0; k < 4; k++) t[k] += base[b * 4 + k];
        pbn_two_state_result r;
        r.n11 = (int64_t)t[0];
        r.n10 = (int64_t)t[1] - r.n11;
        r.n01 = (int64_t)t[2] - r.n11;
        r.n00 = (q.len >= 1 ? q.omega * (q.len - 1) : 0) - r.n11 - r.n10 - r.n01;
        r.ones = (int64_t)t[3];
        r.pad = 0;
        two_state_formulas(r, q.omega, q.len, q.eps, q.r, q.s);
        out[lo].ts = r;
      }
    }
    __syncthreads();
  }
}

}  // namespace pbn

// ------------------------------------------------------------------ host

namespace {

using namespace pbn;

int efail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return code;
}

#define ECUDA(expr, what)                                                                          \
  do {                                                                                              \
    cudaError_t _e = (expr);                                                                        \
    if (_e != cudaSuccess)                                                                          \
      return efail(_e == cudaErrorMemoryAllocation ? PBN_ERR_OOM : PBN_ERR_CUDA, "%s: %s", what,     \
                   cudaGetErrorString(_e));                                                         \
  } while (0)

enum Phase { PH_GR, PH_TS, PH_SK_SKEW, PH_SK_RAND, PH_SK_CI, PH_DONE };

struct EQuery {
  int64_t id = 0;
  uint64_t tag = 0;
  int method = 0;
  int status = PBN_OK;
  const pbn_net *net = nullptr;
  pbn_two_state_query tsq;
  pbn_skart_query skq;
  std::vector<int32_t> soi_nodes;
  std::vector<uint8_t> soi_vals;
  int64_t omega = 0, max_length = 0, psi0 = 0;
  double thr = 0;
  uint64_t seed = 0;
  int mode = 0, G = 0;
  pbn_chains ch;
  int64_t state_bytes = 0, bits_bytes = 0;
  int phase = PH_GR;
  int64_t psi = 0, target = 0, keep_from = 0;
  int64_t sim_D = 0;
  int req = -1, req2 = -1;
  // Skart
  int64_t start = 0, eta = 0, kappa = 1, p = 0, d = 0;
  pbn_two_state_report tr;
  pbn_skart_report sr;
  int64_t submit_epoch = 0, admit_epoch = -1, finish_epoch = -1;
  int64_t updates = 0;
  int64_t batch_items = 0;   // (node, group, transition) items of batch_sim_kernel launches
  int64_t batch_items_epoch = 0;

  EQuery() {
    memset(&tsq, 0, sizeof tsq);
    memset(&skq, 0, sizeof skq);
    memset(&ch, 0, sizeof ch);
    memset(&tr, 0, sizeof tr);
    memset(&sr, 0, sizeof sr);
  }
  const NetDev &dev() const { return net->dev; }
};

struct Candidate {
  int S, threads, ipt, big;
  double ms = 0;
  int64_t updates = 0;
  int trials = 0;
};

}  // namespace

struct pbn_engine {
  int dev = 0;
  cudaStream_t s = nullptr;
  pbn_engine_cfg cfg;
  int sms = 1;
  int64_t next_id = 0, epoch = 0, mem = 0;
  std::deque<std::unique_ptr<EQuery>> pending;
  std::vector<std::unique_ptr<EQuery>> active;
  std::vector<pbn_engine_result> done;
  int max_items = 1 << 15;
  SimArgs *d_tasks = nullptr, *h_tasks = nullptr;
  BatchItem *d_items = nullptr, *h_items = nullptr;
  int *d_cnt = nullptr, *h_cnt = nullptr;
  StatReq *d_reqs = nullptr, *h_reqs = nullptr;
  ReqOut *d_out = nullptr, *h_out = nullptr;
  unsigned long long *d_partials = nullptr;
  unsigned int *d_tickets = nullptr;
  StatsScratch sk;
  pbn_skart_result *d_sk = nullptr, *h_sk = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEvent_t es0 = nullptr, es1 = nullptr;  // around batch_sim_kernel (graph: external event nodes)
  cudaGraphExec_t exec = nullptr;
  int *status = nullptr;                 // device status word of the batched launches
  std::vector<EQuery *> epoch_queries;   // queries simulated in the current epoch
  size_t graph_smem = 0;
  int graph_threads = 0;
  std::vector<Candidate> cands;
  int best = -1;
  int round_robin = 0;
  double items_per_ms = 0;   // batch_sim_kernel rate (moving average over epochs)
  int sim_ctas = 0;          // CTAs of its last persistent grid
};

namespace {

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// The autotuner's last choice in this process: later engines without fixed
// settings start from it instead of tuning again.
std::mutex g_tuned_mu;
bool g_tuned = false;
Candidate g_tuned_cand;

// Dynamic shared memory one batched-simulation CTA may use: the opt-in
// maximum less the kernel's own static shared memory.
int smem_limit() {
  static int v = -1;
  if (v < 0) {
    cudaFuncAttributes fa;
    size_t stat = 0;
    if (cudaFuncGetAttributes(&fa, batch_sim_kernel) == cudaSuccess) stat = fa.sharedSizeBytes;
    v = sim_max_smem() - (int)stat;
  }
  return v;
}

// Dynamic shared memory per CTA for a CTA size: 256-thread CTAs are sized so
// that three share an SM (the kernel is held to 80 registers, which three
// 256-thread CTAs fit), 512-thread CTAs take one SM each.
int smem_cap_for(int threads) {
  static int per_sm = -1;
  if (per_sm < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess) per_sm = 0;
  }
  if (threads > 256 || per_sm <= 0) return smem_limit();
  cudaFuncAttributes fa;
  size_t stat = 0;
  if (cudaFuncGetAttributes(&fa, batch_sim_kernel) == cudaSuccess) stat = fa.sharedSizeBytes;
  // each CTA also takes 1 KB of shared memory that the system reserves
  return std::min(smem_limit(), per_sm / 3 - 1024 - (int)stat);
}

// Chain groups per CTA for one query: about threads * ipt items, at most
// gpb_cap (so that a light epoch still spreads over the SMs), within the
// shared memory one CTA may use.
// Tables that do not fit shared memory are staged as TMA tiles or read from
// global memory (`big` chooses).
void size_task(const EQuery &q, int threads, int ipt, int gpb_cap, size_t smem_cap, int big, int *gpb_out,
               int *staging_out) {
  const NetDev &d = q.dev();
  int gpb = std::max(1, threads * ipt / std::max(1, d.n));
  gpb = std::min(gpb, std::max(1, gpb_cap));
  gpb = std::min(gpb, q.G);
  for (;;) {
    if (sim_smem_bytes(d.n, d.F, gpb, q.mode, STAGE_SMEM, d.tile_bytes) <= smem_cap) { *staging_out = STAGE_SMEM; break; }
    if (sim_smem_bytes(d.n, d.F, gpb, q.mode, big, d.tile_bytes) <= smem_cap) { *staging_out = big; break; }
    if (gpb == 1) { *staging_out = STAGE_GLOBAL; break; }
    gpb = std::max(1, gpb / 2);
  }
  *gpb_out = gpb;
}

int reserve_bits(pbn_engine *e, EQuery &q, int64_t base, int64_t upto) {
  pbn_chains &ch = q.ch;
  if (ch.bits && base >= ch.bits_base && upto - ch.bits_base <= ch.bits_cap) return PBN_OK;
  const int64_t keep_from = std::max(base, ch.bits_base);
  const int64_t kept =
      ch.bits ? std::max<int64_t>(0, std::min(ch.length, ch.bits_base + ch.bits_cap) - keep_from) : 0;
  int64_t cap = std::max<int64_t>(upto - base, 64);
  cap = std::max<int64_t>(cap, 2 * (ch.bits ? (ch.length - base) : 0));
  cap = (cap + 3) & ~int64_t(3);
  uint32_t *nb = nullptr;
  const size_t bytes = sizeof(uint32_t) * (size_t)q.G * cap;
  ECUDA(cudaMallocAsync(&nb, bytes, e->s), "engine bitstream alloc");
  if (ch.bits && kept > 0) {
    ECUDA(cudaMemcpy2DAsync(nb + (keep_from - base), cap * 4, ch.bits + (keep_from - ch.bits_base), ch.bits_cap * 4,
                            kept * 4, q.G, cudaMemcpyDeviceToDevice, e->s),
          "engine bitstream copy");
  }
  if (ch.bits) cudaFreeAsync(ch.bits, e->s);
  e->mem += (int64_t)bytes - q.bits_bytes;
  q.bits_bytes = (int64_t)bytes;
  ch.bits = nb;
  ch.bits_cap = cap;
  ch.bits_base = base;
  return PBN_OK;
}

void finish(pbn_engine *e, EQuery &q, int status) {
  q.status = status;
  q.phase = PH_DONE;
  q.finish_epoch = e->epoch;
}

// -------- two-state machine (mirrors pbn_estimate_two_state)

void ts_after_gr(pbn_engine *e, EQuery &q, const pbn_gr_result &r) {
  q.tr.gr_rounds++;
  q.tr.rhat = r.rhat;
  q.sr.gr_rounds++;
  q.sr.rhat = r.rhat;
  if (r.rhat < q.thr) {
    q.tr.gr_psi = q.psi;
    if (q.method == PBN_METHOD_TWO_STATE) {
      q.phase = PH_TS;
      q.keep_from = q.psi;
      q.target = q.ch.length;           // n = psi >= 2: count at once
    } else {
      q.start = q.psi;
      q.eta = cdiv(1280, q.omega) * q.omega;
      q.phase = PH_SK_SKEW;
      q.keep_from = q.start;
      q.target = std::max(q.ch.length, q.start + q.eta / q.omega);
    }
    return;
  }
  q.psi *= 2;
  if (2 * q.psi > q.max_length) { finish(e, q, PBN_ERR_NOT_CONVERGED); return; }
  q.target = 2 * q.psi;
  q.keep_from = q.psi;
}

void ts_after_counts(pbn_engine *e, EQuery &q, const pbn_two_state_result &r) {
  q.tr.ts_rounds++;
  const int64_t n = q.ch.length - q.psi;
  if (r.status == PBN_ERR_INSUFFICIENT) {
    if (q.ch.length + n > q.max_length) { finish(e, q, PBN_ERR_NOT_CONVERGED); return; }
    q.target = q.ch.length + n;
    return;
  }
  if (r.status != PBN_OK) { finish(e, q, r.status); return; }
  q.tr.prob = r.prob;
  q.tr.alpha = r.alpha;
  q.tr.beta = r.beta;
  q.tr.M = r.M;
  q.tr.N = r.N;
  q.tr.ones = r.ones;
  q.tr.n4[0] = r.n00; q.tr.n4[1] = r.n01; q.tr.n4[2] = r.n10; q.tr.n4[3] = r.n11;
  const int64_t deficit = r.N - q.omega * n;
  if (deficit > 0) {
    const int64_t eb = cdiv(deficit, q.omega);
    if (q.ch.length + eb > q.max_length) { finish(e, q, PBN_ERR_NOT_CONVERGED); return; }
    q.target = q.ch.length + eb;
    return;
  }
  if (r.M > q.psi) {
    q.psi = r.M;
    q.keep_from = q.psi;
    if (q.ch.length - q.psi < 2) {
      if (q.psi + 2 > q.max_length) { finish(e, q, PBN_ERR_NOT_CONVERGED); return; }
      q.target = q.psi + 2;
    } else {
      q.target = q.ch.length;
    }
    return;
  }
  q.tr.psi = q.psi;
  q.tr.length = q.ch.length;
  q.tr.sample_size = q.omega * (q.ch.length - q.psi);
  finish(e, q, PBN_OK);
}

// -------- Skart machine (mirrors pbn_estimate_skart)

int skart_check(pbn_engine *e, EQuery &q) {
  pbn_skart_result r;
  const int64_t bpc = (q.phase == PH_SK_SKEW) ? q.eta / q.omega : q.p / q.omega;
  const int64_t kap = (q.phase == PH_SK_SKEW) ? 1 : q.kappa;
  const int64_t sp = (q.phase == PH_SK_RAND) ? q.d : 0;
  if (q.phase == PH_SK_CI && q.kappa > (1ll << 30)) { finish(e, q, PBN_ERR_UNSUPPORTED); return PBN_OK; }
  ECUDA(launch_skart(q.ch, q.start - q.ch.bits_base, kap, bpc, sp, q.skq.alpha, 0.20, e->d_sk, e->sk, e->s), "Skart");
  ECUDA(cudaMemcpyAsync(e->h_sk, e->d_sk, sizeof(r), cudaMemcpyDeviceToHost, e->s), "Skart copy");
  ECUDA(cudaStreamSynchronize(e->s), "Skart sync");
  r = *e->h_sk;
  if (q.phase == PH_SK_SKEW) {
    q.kappa = fabs(r.skew) > 4.0 ? 16 : 1;
    q.p = cdiv(q.eta, q.omega) * q.omega;
    q.eta = q.kappa * q.p;
    q.d = 0;
    q.phase = PH_SK_RAND;
  } else if (q.phase == PH_SK_RAND) {
    q.sr.rand_rounds++;
    if (r.vn_pass) {
      q.sr.spacer = q.d;
      q.phase = PH_SK_CI;
      q.target = q.ch.length;
      return PBN_OK;
    }
    q.d += 1;
    if (q.d > 10) {
      q.d = 0;
      q.kappa = (int64_t)ceil(sqrt(2.0) * (double)q.kappa);
      q.p = (int64_t)ceil(0.9 * (double)q.p);
    }
    q.p = cdiv(q.p, q.omega) * q.omega;
    q.eta = q.kappa * q.p;
  } else {
    q.sr.ci_rounds++;
    q.sr.mean = r.mean; q.sr.ci_lo = r.ci_lo; q.sr.ci_hi = r.ci_hi; q.sr.H = r.H;
    q.sr.var = r.var; q.sr.skew = r.skew; q.sr.phi = r.phi;
    const double Hs = q.skq.relative ? q.skq.H_star * fabs(r.mean) : q.skq.H_star;
    if (!(r.H > Hs)) {
      q.sr.psi = q.psi;
      q.sr.length = q.ch.length;
      q.sr.kappa = q.kappa;
      q.sr.batches = q.p;
      q.sr.sample_size = q.kappa * q.p;
      finish(e, q, PBN_OK);
      return PBN_OK;
    }
    const double f = (r.H / Hs) * (r.H / Hs);
    const int64_t pmax = q.p > 1024 ? q.p : 1024;
    const double pf = ceil(f * (double)q.p);
    const int64_t p1 = pf > (double)pmax ? pmax : (int64_t)pf;
    int64_t k1 = (int64_t)ceil((double)q.kappa * f * (double)q.p / (double)p1);
    if (k1 < q.kappa) k1 = q.kappa;
    q.kappa = k1;
    q.p = cdiv(p1, q.omega) * q.omega;
    q.eta = q.kappa * q.p;
  }
  if (q.start + q.eta / q.omega > q.max_length) { finish(e, q, PBN_ERR_NOT_CONVERGED); return PBN_OK; }
  q.target = q.start + q.eta / q.omega;
  return PBN_OK;
}

int admit(pbn_engine *e) {
  while (!e->pending.empty() && (int)e->active.size() < e->cfg.max_active) {
    EQuery &q = *e->pending.front();
    const NetDev &d = q.dev();
    const int64_t state_bytes = (int64_t)q.G * d.n * 4;
    const int64_t est = state_bytes + (int64_t)q.G * 4 * std::max<int64_t>(64, 2 * q.psi0);
    if (e->mem + est > e->cfg.hbm_budget_bytes && !e->active.empty()) break;
    ECUDA(cudaMallocAsync(&q.ch.state, (size_t)state_bytes, e->s), "engine state alloc");
    q.state_bytes = state_bytes;
    e->mem += state_bytes;
    q.ch.omega = q.omega;
    q.ch.length = 0;
    ECUDA(launch_init(d, q.seed, q.ch.state, q.omega, e->s), "engine init");
    q.phase = PH_GR;
    q.psi = q.psi0;
    q.target = 2 * q.psi0;
    q.keep_from = q.psi0;
    q.admit_epoch = e->epoch;
    e->active.push_back(std::move(e->pending.front()));
    e->pending.pop_front();
  }
  return PBN_OK;
}

void retire(pbn_engine *e) {
  std::vector<std::unique_ptr<EQuery>> keep;
  for (auto &qp : e->active) {
    EQuery &q = *qp;
    if (q.phase != PH_DONE) { keep.push_back(std::move(qp)); continue; }
    pbn_engine_result r;
    memset(&r, 0, sizeof r);
    r.id = q.id;
    r.tag = q.tag;
    r.method = q.method;
    r.status = q.status;
    q.tr.chain_node_updates = q.updates;
    q.sr.chain_node_updates = q.updates;
    q.tr.sim_items = q.batch_items;
    q.sr.sim_items = q.batch_items;
    r.two_state = q.tr;
    r.skart = q.sr;
    r.submit_epoch = q.submit_epoch;
    r.admit_epoch = q.admit_epoch;
    r.finish_epoch = q.finish_epoch;
    e->done.push_back(r);
    if (q.ch.state) cudaFreeAsync(q.ch.state, e->s);
    if (q.ch.bits) cudaFreeAsync(q.ch.bits, e->s);
    e->mem -= q.state_bytes + q.bits_bytes;
  }
  e->active.swap(keep);
}

int capture_graph(pbn_engine *e, int threads, size_t smem) {
  if (e->exec && e->graph_threads == threads && e->graph_smem >= smem) return PBN_OK;
  // the same CTA size keeps the largest shared-memory size seen (epochs of
  // other mixes then reuse the graph); another CTA size starts afresh, since
  // its CTAs per SM depend on it
  const size_t gsmem = e->exec && e->graph_threads == threads ? std::max(smem, e->graph_smem) : smem;
  if (e->exec) { cudaGraphExecDestroy(e->exec); e->exec = nullptr; }
  int per_sm = 0;
  ECUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_sim_kernel, threads, gsmem), "occupancy");
  const int sim_blocks = std::max(1, per_sm) * e->sms;
  e->sim_ctas = sim_blocks;
  cudaGraph_t g;
  ECUDA(cudaStreamBeginCapture(e->s, cudaStreamCaptureModeThreadLocal), "begin capture");
  cudaMemcpyAsync(e->d_tasks, e->h_tasks, sizeof(SimArgs) * e->cfg.max_active, cudaMemcpyHostToDevice, e->s);
  cudaMemcpyAsync(e->d_items, e->h_items, sizeof(BatchItem) * e->max_items, cudaMemcpyHostToDevice, e->s);
  cudaMemcpyAsync(e->d_reqs, e->h_reqs, sizeof(StatReq) * kReqPerQuery * e->cfg.max_active, cudaMemcpyHostToDevice,
                  e->s);
  cudaMemcpyAsync(e->d_cnt, e->h_cnt, sizeof(int) * kCounters, cudaMemcpyHostToDevice, e->s);
  // timing events of the simulation launch, kept in the graph as event nodes
  cudaEventRecordWithFlags(e->es0, e->s, cudaEventRecordExternal);
  batch_sim_kernel<<<sim_blocks, threads, gsmem, e->s>>>(e->d_tasks, e->d_items, e->d_cnt);
  cudaEventRecordWithFlags(e->es1, e->s, cudaEventRecordExternal);
  batch_stats_kernel<<<e->sms, 256, 0, e->s>>>(e->d_reqs, e->d_cnt, e->d_partials, e->d_tickets, e->d_out);
  cudaMemcpyAsync(e->h_out, e->d_out, sizeof(ReqOut) * kReqPerQuery * e->cfg.max_active, cudaMemcpyDeviceToHost,
                  e->s);
  ECUDA(cudaStreamEndCapture(e->s, &g), "end capture");
  cudaError_t err = cudaGraphInstantiate(&e->exec, g, 0);
  cudaGraphDestroy(g);
  ECUDA(err, "graph instantiate");
  e->graph_threads = threads;
  e->graph_smem = gsmem;
  return PBN_OK;
}

int launch_direct(pbn_engine *e, int threads, size_t smem, int ntask, int nitems, int nreq) {
  int per_sm = 0;
  ECUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_sim_kernel, threads, smem), "occupancy");
  const int sim_blocks = std::max(1, std::min(std::max(1, per_sm) * e->sms, nitems));
  e->sim_ctas = std::max(1, per_sm) * e->sms;
  if (ntask) ECUDA(cudaMemcpyAsync(e->d_tasks, e->h_tasks, sizeof(SimArgs) * ntask, cudaMemcpyHostToDevice, e->s), "tasks");
  if (nitems) ECUDA(cudaMemcpyAsync(e->d_items, e->h_items, sizeof(BatchItem) * nitems, cudaMemcpyHostToDevice, e->s), "items");
  if (nreq) ECUDA(cudaMemcpyAsync(e->d_reqs, e->h_reqs, sizeof(StatReq) * nreq, cudaMemcpyHostToDevice, e->s), "reqs");
  ECUDA(cudaMemcpyAsync(e->d_cnt, e->h_cnt, sizeof(int) * kCounters, cudaMemcpyHostToDevice, e->s), "counters");
  if (nitems) {
    ECUDA(cudaEventRecord(e->es0, e->s), "event");
    batch_sim_kernel<<<sim_blocks, threads, smem, e->s>>>(e->d_tasks, e->d_items, e->d_cnt);
    ECUDA(cudaGetLastError(), "batch simulation launch");
    ECUDA(cudaEventRecord(e->es1, e->s), "event");
  }
  if (nreq) {
    batch_stats_kernel<<<e->sms, 256, 0, e->s>>>(e->d_reqs, e->d_cnt, e->d_partials, e->d_tickets, e->d_out);
    ECUDA(cudaGetLastError(), "batch statistics launch");
    ECUDA(cudaMemcpyAsync(e->h_out, e->d_out, sizeof(ReqOut) * nreq, cudaMemcpyDeviceToHost, e->s), "results");
  }
  return PBN_OK;
}

}  // namespace

extern "C" int pbn_engine_create(const pbn_engine_cfg *cfg, void *stream, pbn_engine **out) {
  if (!out) return efail(PBN_ERR_INVALID, "NULL output");
  *out = nullptr;
  pbn_engine_cfg c;
  memset(&c, 0, sizeof c);
  if (cfg) c = *cfg;
  if (c.hbm_budget_bytes <= 0) c.hbm_budget_bytes = 8ll << 30;
  if (c.max_active <= 0) c.max_active = PBN_ENGINE_MAX_ACTIVE;
  if (c.max_active > PBN_ENGINE_MAX_ACTIVE) return efail(PBN_ERR_INVALID, "max_active above %d", PBN_ENGINE_MAX_ACTIVE);
  if (c.steps_per_epoch < 0 || c.items_per_thread < 0) return efail(PBN_ERR_INVALID, "negative tuning value");
  if (!(c.epoch_target_ms >= 0.0)) return efail(PBN_ERR_INVALID, "epoch_target_ms %g", c.epoch_target_ms);
  if (c.threads_per_block && c.threads_per_block != 256 && c.threads_per_block != 512)
    return efail(PBN_ERR_INVALID, "threads_per_block must be 256 or 512");
  std::unique_ptr<pbn_engine> e(new pbn_engine());
  e->cfg = c;
  ECUDA(cudaGetDevice(&e->dev), "device");
  // the engine runs on a stream of its own (graph capture needs one that is
  // not the legacy default stream), after the work already queued on `stream`
  ECUDA(cudaStreamCreateWithFlags(&e->s, cudaStreamNonBlocking), "engine stream");
  {
    cudaEvent_t ready;
    ECUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming), "event");
    ECUDA(cudaEventRecord(ready, (cudaStream_t)stream), "event");
    ECUDA(cudaStreamWaitEvent(e->s, ready, 0), "stream wait");
    cudaEventDestroy(ready);
  }
  ECUDA(cudaDeviceGetAttribute(&e->sms, cudaDevAttrMultiProcessorCount, e->dev), "SM count");
  const int A = c.max_active;
  ECUDA(cudaMalloc(&e->d_tasks, sizeof(SimArgs) * A), "engine alloc");
  ECUDA(cudaMallocHost(&e->h_tasks, sizeof(SimArgs) * A), "engine alloc");
  ECUDA(cudaMalloc(&e->d_items, sizeof(BatchItem) * e->max_items), "engine alloc");
  ECUDA(cudaMallocHost(&e->h_items, sizeof(BatchItem) * e->max_items), "engine alloc");
  ECUDA(cudaMalloc(&e->d_cnt, sizeof(int) * kCounters), "engine alloc");
  ECUDA(cudaMallocHost(&e->h_cnt, sizeof(int) * kCounters), "engine alloc");
  const int AR = kReqPerQuery * A;  // statistics requests of one epoch
  ECUDA(cudaMalloc(&e->d_reqs, sizeof(StatReq) * AR), "engine alloc");
  ECUDA(cudaMallocHost(&e->h_reqs, sizeof(StatReq) * AR), "engine alloc");
  ECUDA(cudaMalloc(&e->d_out, sizeof(ReqOut) * AR), "engine alloc");
  ECUDA(cudaMallocHost(&e->h_out, sizeof(ReqOut) * AR), "engine alloc");
  ECUDA(cudaMalloc(&e->d_partials, sizeof(unsigned long long) * AR * kReqBlocks * 4), "engine alloc");
  ECUDA(cudaMalloc(&e->d_tickets, sizeof(unsigned int) * AR), "engine alloc");
  ECUDA(cudaMemsetAsync(e->d_tickets, 0, sizeof(unsigned int) * AR, e->s), "engine memset");
  ECUDA(scratch_init(e->sk, e->s), "engine scratch");
  ECUDA(cudaMalloc(&e->d_sk, sizeof(pbn_skart_result)), "engine alloc");
  ECUDA(cudaMallocHost(&e->h_sk, sizeof(pbn_skart_result)), "engine alloc");
  ECUDA(cudaEventCreate(&e->e0), "event");
  ECUDA(cudaEventCreate(&e->e1), "event");
  ECUDA(cudaEventCreate(&e->es0), "event");
  ECUDA(cudaEventCreate(&e->es1), "event");
  ECUDA(cudaMalloc(&e->status, sizeof(int)), "engine alloc");
  ECUDA(cudaMemsetAsync(e->status, 0, sizeof(int), e->s), "engine memset");
  memset(e->h_tasks, 0, sizeof(SimArgs) * A);
  memset(e->h_items, 0, sizeof(BatchItem) * e->max_items);
  memset(e->h_reqs, 0, sizeof(StatReq) * AR);
  memset(e->h_cnt, 0, sizeof(int) * kCounters);
  ECUDA(cudaFuncSetAttribute(batch_sim_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_limit()), "smem attr");
  // candidates of the autotuner (a fixed setting leaves one candidate)
  // 512-thread CTAs (one per SM at 80 registers) measured slower than three
  // 256-thread CTAs per SM on every setting tried, so the tuner keeps 256
  const int Ss[] = {1024, 4096};
  const int Ts[] = {256};
  const int Is[] = {2, 8};
  const int Bs[] = {STAGE_TILES, STAGE_GLOBAL};
  for (int S : Ss)
    for (int T : Ts)
      for (int I : Is)
        for (int B : Bs) {
          if (c.steps_per_epoch && S != Ss[0]) continue;
          if (c.threads_per_block && T != Ts[0]) continue;
          if (c.items_per_thread && I != Is[0]) continue;
          if (B != Bs[0] && (c.steps_per_epoch || c.threads_per_block || c.items_per_thread)) continue;
          Candidate cd;
          cd.S = c.steps_per_epoch ? c.steps_per_epoch : S;
          cd.threads = c.threads_per_block ? c.threads_per_block : T;
          cd.ipt = c.items_per_thread ? c.items_per_thread : I;
          cd.big = B;
          e->cands.push_back(cd);
        }
  if (e->cands.size() == 1) e->best = 0;
  if (e->best < 0) {
    std::lock_guard<std::mutex> lk(g_tuned_mu);
    if (g_tuned) {
      e->cands.assign(1, g_tuned_cand);
      e->best = 0;
    }
  }
  *out = e.release();
  return PBN_OK;
}

extern "C" void pbn_engine_destroy(pbn_engine *e) {
  if (!e) return;
  cudaStreamSynchronize(e->s);
  for (auto &q : e->active) {
    if (q->ch.state) cudaFree(q->ch.state);
    if (q->ch.bits) cudaFree(q->ch.bits);
  }
  if (e->exec) cudaGraphExecDestroy(e->exec);
  cudaFree(e->d_tasks); cudaFreeHost(e->h_tasks);
  cudaFree(e->d_items); cudaFreeHost(e->h_items);
  cudaFree(e->d_cnt); cudaFreeHost(e->h_cnt);
  cudaFree(e->d_reqs); cudaFreeHost(e->h_reqs);
  cudaFree(e->d_out); cudaFreeHost(e->h_out);
  cudaFree(e->d_partials); cudaFree(e->d_tickets);
  scratch_free(e->sk);
  cudaFree(e->d_sk); cudaFreeHost(e->h_sk);
  cudaEventDestroy(e->e0); cudaEventDestroy(e->e1);
  cudaEventDestroy(e->es0); cudaEventDestroy(e->es1);
  cudaFree(e->status);
  cudaStreamDestroy(e->s);
  delete e;
}

extern "C" int pbn_engine_submit(pbn_engine *e, const pbn_engine_query *qin, int64_t *id) {
  if (!e || !qin || !qin->net) return efail(PBN_ERR_INVALID, "NULL engine, query or network");
  std::unique_ptr<EQuery> q(new EQuery());
  q->method = qin->method;
  q->net = qin->net;
  q->tag = qin->tag;
  const pbn_soi *soi;
  if (qin->method == PBN_METHOD_TWO_STATE) {
    const pbn_two_state_query &t = qin->two_state;
    if (!(t.eps > 0 && t.r > 0 && t.s > 0 && t.s < 1)) return efail(PBN_ERR_INVALID, "eps, r, s out of range");
    q->tsq = t;
    q->omega = t.omega; q->psi0 = t.psi0; q->thr = t.rhat_threshold; q->max_length = t.max_length;
    q->seed = t.seed; q->mode = t.perturb_mode;
    soi = &t.soi;
  } else if (qin->method == PBN_METHOD_SKART) {
    const pbn_skart_query &k = qin->skart;
    if (!(k.H_star > 0 && k.alpha > 0 && k.alpha < 1)) return efail(PBN_ERR_INVALID, "H_star, alpha");
    q->skq = k;
    q->omega = k.omega; q->psi0 = k.psi0; q->thr = k.rhat_threshold; q->max_length = k.max_length;
    q->seed = k.seed; q->mode = k.perturb_mode;
    soi = &k.soi;
  } else {
    return efail(PBN_ERR_INVALID, "method %d", qin->method);
  }
  if (q->omega < 2 || q->psi0 < 2 || !(q->thr > 0) || q->max_length < 2 * q->psi0)
    return efail(PBN_ERR_INVALID, "omega, psi0, R-hat threshold or max_length");
  if (q->mode != PBN_PERTURB_PER_NODE && q->mode != PBN_PERTURB_GLOBAL) return efail(PBN_ERR_INVALID, "perturb_mode");
  if (soi->size < 1 || soi->size > PBN_MAX_SOI || !soi->nodes || !soi->values)
    return efail(PBN_ERR_INVALID, "state of interest");
  for (int m = 0; m < soi->size; m++) {
    if (soi->nodes[m] < 0 || soi->nodes[m] >= qin->net->dev.n || soi->values[m] > 1)
      return efail(PBN_ERR_INVALID, "state of interest entry %d", m);
    q->soi_nodes.push_back(soi->nodes[m]);
    q->soi_vals.push_back(soi->values[m]);
  }
  if (qin->net->dev.max_l > kMaxL || qin->net->dev.max_k > kWideK)
    return efail(PBN_ERR_UNSUPPORTED,
                 "the engine's batched kernel takes nodes of at most %d functions of at most %d inputs", kMaxL, kWideK);
  q->G = (int)((q->omega + 31) / 32);
  if ((int64_t)q->G * 1 > (1ll << 30)) return efail(PBN_ERR_UNSUPPORTED, "omega too large");
  q->id = e->next_id++;
  q->submit_epoch = e->epoch;
  if (id) *id = q->id;
  e->pending.push_back(std::move(q));
  return PBN_OK;
}

extern "C" int pbn_engine_step(pbn_engine *e, pbn_engine_stats *st) {
  if (!e) return efail(PBN_ERR_INVALID, "NULL engine");
  int rc = admit(e);
  if (rc) return rc;
  // tuning candidate of this epoch
  int ci = e->best;
  if (ci < 0) ci = e->round_robin++ % (int)e->cands.size();
  const Candidate &cand = e->cands[ci];
  size_t smem_cap = (size_t)smem_cap_for(cand.threads);
  e->epoch_queries.clear();
  // spread light epochs: at least about two CTAs per SM when the active
  // chain groups allow it
  int64_t total_groups = 0;
  int nsim = 0;
  for (auto &qp : e->active)
    if (qp->phase != PH_DONE && qp->ch.length < qp->target) {
      total_groups += qp->G;
      nsim++;
    }
  const int gpb_cap = (int)std::max<int64_t>(1, total_groups / (2 * (int64_t)e->sms));
  // light load (a few queries to extend, none waiting for admission): queries
  // with few chain groups are extended outside the batched kernel, one after
  // another, by the schedule pbn_run_chains picks (select-ahead for them: the
  // batched fused kernel would leave most SMs idle and wait on its Philox
  // rounds every step); the same chains, bit for bit
  const bool few = nsim <= kAloneMax && e->pending.empty();
  int ntask = 0, nitems = 0, nreq = 0, vblocks = 0;
  size_t smem = 0;
  int64_t updates = 0;
  int launches = 0;
  std::vector<std::pair<int64_t, int>> order;  // (cost, task) for longest-first items
  std::vector<std::pair<int, int>> task_groups;  // (task, gpb)
  for (auto &qp : e->active) {
    EQuery &q = *qp;
    q.sim_D = 0;
    q.req = -1;
    q.req2 = -1;
    q.batch_items_epoch = 0;
    if (q.phase == PH_DONE) continue;
    if (q.ch.length < q.target) {
      if (ntask >= e->cfg.max_active) continue;
      int gpb, staging;
      size_task(q, cand.threads, cand.ipt, gpb_cap, smem_cap, cand.big, &gpb, &staging);
      int64_t D = std::min<int64_t>(cand.S, q.target - q.ch.length);
      const bool alone_ok = few && 2 * q.G <= e->sms;
      if (e->cfg.epoch_target_ms > 0 && !alone_ok && e->items_per_ms > 0 && e->sim_ctas > 0) {
        // each work item (gpb groups of this query on one CTA) takes at most
        // about epoch_target_ms, so that queries arriving meanwhile wait at most
        // that long for the next epoch: a CTA's step costs one round of its
        // threads per `threads` items, at the rate the last epochs measured
        const double round_ms = (double)cand.threads * e->sim_ctas / e->items_per_ms;
        const double rounds = std::max(1.0, std::ceil((double)q.dev().n * gpb / cand.threads));
        const int64_t cap =
            std::max<int64_t>(kMinEpochSteps, (int64_t)(e->cfg.epoch_target_ms / (rounds * round_ms)));
        D = std::min(D, cap);
      }
      if ((rc = reserve_bits(e, q, q.keep_from, q.ch.length + D))) { finish(e, q, rc); continue; }
      const int64_t groups_items = cdiv(q.G, gpb);
      if (nitems + groups_items > e->max_items) continue;   // next epoch
      SimArgs &a = e->h_tasks[ntask];
      memset(&a, 0, sizeof a);
      const NetDev &d = q.dev();
      a.rk = make_round_keys(q.seed);
      a.node = d.d_node;
      a.fn = d.d_fn;
      a.state = q.ch.state;
      a.bits = q.ch.bits;
      a.bits_cap = q.ch.bits_cap;
      a.col0 = q.ch.length - q.ch.bits_base;
      a.omega = q.omega;
      a.t0 = (uint64_t)q.ch.length;
      a.n = d.n;
      a.F = d.F;
      a.G = q.G;
      a.steps = (int)D;
      a.gpb = gpb;
      a.P32 = d.P32;
      a.staging = staging;
      a.tiles = d.d_tiles;
      a.ntiles = d.ntiles;
      a.tile_bytes = d.tile_bytes;
      a.wide_tt = d.d_wide_tt;
      a.wide_par = d.d_wide_par;
      a.has_wide = d.has_wide;
      a.status = e->status;
      a.soi_size = (int)q.soi_nodes.size();
      a.n_props = 1;  // one property per engine query (soi_prop all 0)
      a.prop_stride = 0;
      for (size_t m = 0; m < q.soi_nodes.size(); m++) {
        a.soi_node[m] = (uint16_t)q.soi_nodes[m];
        if (q.soi_vals[m]) a.soi_val |= 1u << m;
      }
      a.mode = q.mode;
      smem = std::max(smem, sim_smem_bytes(d.n, d.F, gpb, q.mode, staging, d.tile_bytes));
      e->epoch_queries.push_back(&q);
      order.push_back(std::make_pair(-(int64_t)d.n * gpb * D, ntask));
      task_groups.push_back(std::make_pair(ntask, gpb));
      nitems += (int)groups_items;
      q.sim_D = D;
      q.batch_items_epoch = (int64_t)d.n * q.G * D;
      updates += q.omega * D * d.n;
      q.updates += q.omega * D * d.n;
      ntask++;
    }
    if (q.ch.length + q.sim_D == q.target && (q.phase == PH_GR || q.phase == PH_TS)) {
      StatReq &r = e->h_reqs[nreq];
      memset(&r, 0, sizeof r);
      r.kind = q.phase == PH_GR ? REQ_GR : REQ_TS;
      r.bits = q.ch.bits;
      r.cap = q.ch.bits_cap;
      r.col = q.psi - q.ch.bits_base;
      r.len = q.phase == PH_GR ? q.psi : q.target - q.psi;
      r.omega = q.omega;
      r.G = q.G;
      r.eps = q.tsq.eps;
      r.r = q.tsq.r;
      r.s = q.tsq.s;
      const int64_t work = (int64_t)q.G * cdiv(r.len, 32);
      r.nblocks = (int)std::max<int64_t>(1, std::min<int64_t>(kReqBlocks, cdiv(work, 64)));
      r.block0 = vblocks;
      vblocks += r.nblocks;
      q.req = nreq++;
      if (q.phase == PH_GR && q.method == PBN_METHOD_TWO_STATE) {
        // Alg. 3's first check counts the same window [psi, 2 psi) the
        // Gelman & Rubin check reads: asked for now, used if R-hat converges
        // (as pbn_estimate_two_state does), so the query needs no epoch of its own for it
        StatReq &t = e->h_reqs[nreq];
        t = r;
        t.kind = REQ_TS;
        t.block0 = vblocks;
        vblocks += t.nblocks;
        q.req2 = nreq++;
      }
    }
  }
  ECUDA(cudaEventRecord(e->e0, e->s), "event");
  // the light-load path (see `few`); a task it cannot take stays batched.
  // Not a tuning sample.
  std::vector<char> alone_task(ntask, 0);
  int nalone = 0;
  for (int t = 0; t < ntask && few; t++) {
    EQuery &q = *e->epoch_queries[t];
    if (!(2 * q.G <= e->sms && q.sim_D > 0)) continue;
    pbn_run_cfg rc_cfg;
    memset(&rc_cfg, 0, sizeof rc_cfg);
    rc_cfg.seed = q.seed;
    rc_cfg.perturb_mode = q.mode;
    rc_cfg.soi.size = (int32_t)q.soi_nodes.size();
    rc_cfg.soi.nodes = q.soi_nodes.data();
    rc_cfg.soi.values = q.soi_vals.data();
    pbn_chains c = q.ch;  // q.ch.length advances when the epoch is applied
    int64_t l = 0;
    if (run_chains_alone(q.dev(), rc_cfg, c, q.sim_D, e->s, e->status, &l) == PBN_OK) {
      alone_task[t] = 1;
      nalone++;
      nitems -= (int)cdiv(q.G, e->h_tasks[t].gpb);
      q.batch_items_epoch = 0;
      launches += (int)l;
    } else {
      set_last_error("");  // fall back to the batched kernel
    }
  }
  const bool alone = nalone > 0;
  // items, longest tasks first
  std::sort(order.begin(), order.end());
  {
    int k = 0;
    for (auto &o : order) {
      const int t = o.second;
      if (alone_task[t]) continue;
      const int gpb = task_groups[t].second;
      const int G = e->h_tasks[t].G;
      for (int g0 = 0; g0 < G; g0 += gpb) {
        BatchItem &it = e->h_items[k++];
        it.task = t;
        it.g0 = g0;
        it.ngl = std::min(gpb, G - g0);
        it.pad = 0;
      }
    }
  }
  e->h_cnt[0] = nitems;
  e->h_cnt[1] = 0;
  e->h_cnt[2] = vblocks;
  e->h_cnt[3] = 0;
  e->h_cnt[4] = nreq;
  int64_t d2h = sizeof(int);  // the status word
  if (nitems || nreq) {
    if (e->cfg.use_graph) {
      if ((rc = capture_graph(e, cand.threads, smem))) return rc;
      ECUDA(cudaGraphLaunch(e->exec, e->s), "graph launch");
      launches += 2;
      d2h += (int64_t)sizeof(ReqOut) * kReqPerQuery * e->cfg.max_active;
    } else {
      if ((rc = launch_direct(e, cand.threads, smem, ntask, nitems, nreq))) return rc;
      launches += (nitems ? 1 : 0) + (nreq ? 1 : 0);
      if (nreq) d2h += (int64_t)sizeof(ReqOut) * nreq;
    }
  }
  ECUDA(cudaEventRecord(e->e1, e->s), "event");
  ECUDA(cudaStreamSynchronize(e->s), "epoch sync");
  float ms = 0.f, sim_ms = 0.f;
  cudaEventElapsedTime(&ms, e->e0, e->e1);
  int64_t sim_items = 0;
  if (nitems) {
    cudaEventElapsedTime(&sim_ms, e->es0, e->es1);
    for (EQuery *q : e->epoch_queries) {
      q->batch_items += q->batch_items_epoch;
      sim_items += q->batch_items_epoch;
    }
    // the rate of epochs that keep every CTA busy (at least a few items per CTA)
    if (sim_ms > 0.f && nitems >= 2 * e->sim_ctas) {
      const double r = (double)sim_items / sim_ms;
      e->items_per_ms = e->items_per_ms > 0 ? 0.7 * e->items_per_ms + 0.3 * r : r;
    }
  }
  {
    // a bounded device wait that gave up fails every query of this epoch
    int stv = 0;
    ECUDA(cudaMemcpy(&stv, e->status, sizeof stv, cudaMemcpyDeviceToHost), "status read");
    if (stv) {
      ECUDA(cudaMemset(e->status, 0, sizeof stv), "status clear");
      for (EQuery *q : e->epoch_queries) {
        q->sim_D = 0;
        q->req = -1;
        finish(e, *q, stv);
      }
    }
  }
  // apply the epoch
  for (auto &qp : e->active) {
    EQuery &q = *qp;
    if (q.phase == PH_DONE) continue;
    q.ch.length += q.sim_D;
    if (q.req >= 0) {
      if (q.phase == PH_GR) {
        ts_after_gr(e, q, e->h_out[q.req].gr);
        // converged: the first two-state check's window is the one counted
        if (q.req2 >= 0 && q.phase == PH_TS && q.target == q.ch.length) ts_after_counts(e, q, e->h_out[q.req2].ts);
      } else {
        ts_after_counts(e, q, e->h_out[q.req].ts);
      }
    }
  }
  for (auto &qp : e->active) {
    EQuery &q = *qp;
    // a Skart window may end before the chains' current length (the chains
    // are already long enough): check as soon as length >= target
    if ((q.phase == PH_SK_SKEW || q.phase == PH_SK_RAND || q.phase == PH_SK_CI) && q.ch.length >= q.target) {
      if ((rc = skart_check(e, q))) return rc;
      launches += 2;
      d2h += sizeof(pbn_skart_result);
    }
  }
  if (e->best < 0 && updates > 0 && !alone) {
    Candidate &c = e->cands[ci];
    c.ms += ms;
    c.updates += updates;
    c.trials++;
    bool all = true;
    for (auto &x : e->cands) all = all && x.trials >= 1;
    if (all) {
      double bestv = -1;
      for (size_t k = 0; k < e->cands.size(); k++) {
        const double v = e->cands[k].updates / std::max(1e-9, e->cands[k].ms);
        if (v > bestv) { bestv = v; e->best = (int)k; }
      }
      std::lock_guard<std::mutex> lk(g_tuned_mu);
      g_tuned = true;
      g_tuned_cand = e->cands[e->best];
    }
  }
  retire(e);
  e->epoch++;
  if (st) {
    memset(st, 0, sizeof *st);
    st->epoch = e->epoch;
    st->active = (int)e->active.size();
    st->pending = (int)e->pending.size();
    st->finished = (int64_t)e->done.size();
    st->updates = updates;
    st->epoch_ms = ms;
    st->hbm_in_use = e->mem;
    st->steps_per_epoch = cand.S;
    st->threads_per_block = cand.threads;
    st->items_per_thread = cand.ipt;
    st->kernel_launches = launches;
    st->sim_ms = sim_ms;
    st->sim_items = sim_items;
    st->d2h_bytes = d2h;
    st->tuning = e->best < 0 ? 1 : 0;
  }
  return PBN_OK;
}

extern "C" int pbn_engine_cancel(pbn_engine *e, int64_t id) {
  if (!e) return efail(PBN_ERR_INVALID, "NULL engine");
  // no work is in flight between calls (pbn_engine_step synchronises), so a
  // cancelled query's buffers can be released at once
  for (auto it = e->pending.begin(); it != e->pending.end(); ++it) {
    if ((*it)->id != id) continue;
    EQuery &q = **it;
    q.status = PBN_ERR_CANCELLED;
    q.phase = PH_DONE;
    q.finish_epoch = e->epoch;
    e->active.push_back(std::move(*it));
    e->pending.erase(it);
    retire(e);
    return PBN_OK;
  }
  for (auto &qp : e->active) {
    if (qp->id != id || qp->phase == PH_DONE) continue;
    finish(e, *qp, PBN_ERR_CANCELLED);
    retire(e);
    return PBN_OK;
  }
  return efail(PBN_ERR_INVALID, "no waiting or active query %lld", (long long)id);
}

extern "C" int pbn_engine_poll(pbn_engine *e, pbn_engine_result *out, int32_t max_results, int32_t *count) {
  if (!e || !count || (max_results > 0 && !out)) return efail(PBN_ERR_INVALID, "NULL argument");
  int32_t k = 0;
  while (k < max_results && !e->done.empty()) {
    out[k++] = e->done.front();
    e->done.erase(e->done.begin());
  }
  *count = k;
  return PBN_OK;
}
