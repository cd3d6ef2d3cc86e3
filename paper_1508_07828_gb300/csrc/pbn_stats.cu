// Statistics of the indicator bitstream on sm_103a: Gelman & Rubin
// (Sec. 4.1), the two-state Markov chain quantities (Sec. 3.1, Alg. 1 line 8)
// and the Skart batch statistics (Sec. 3.2, Alg. 4).
//
// Every reduction is exact: integer counts (popc of bitstream words, warp
// bit-transposes to per-chain words, warp shuffles, 64/128-bit block sums),
// written as per-block partials; the last block to finish (ticket counter)
// folds the partials in a fixed order and does the few FP64 operations of
// the statistic on one thread.  This translation unit is compiled without
// FMA contraction so the FP64 formulas round the same way as plain C.
#include "pbn_stats.cuh"

namespace pbn {

// ------------------------------------------------------------ Gelman-Rubin

// One block per chain group (blocks loop over groups when there are more):
// its 8 warps split the window's columns, each warp counting the ones of its
// columns per chain (bit-transpose + popc, lane = chain); the per-chain
// counts c_i are summed over the warps in shared memory, then S1 = sum c_i and
// S2 = sum c_i^2 (128-bit) over the group's valid chains.
__global__ void __launch_bounds__(256) gr_kernel(const uint32_t *bits, int64_t cap, int64_t col, int64_t psi,
                                                 int64_t omega, int G, unsigned long long *partials,
                                                 unsigned int *ticket, pbn_gr_result *out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  __shared__ uint32_t cnt_s[8][32];
  // columns of the window per warp: a multiple of 32
  const int64_t per_warp = ((psi + wpb - 1) / wpb + 31) / 32 * 32;
  uint64_t acc1 = 0;
  u128 acc2 = 0;
  for (int64_t g = blockIdx.x; g < G; g += gridDim.x) {
    const uint32_t *row = bits + (size_t)g * cap + col;
    uint32_t cnt = 0;
    const int64_t j0 = (int64_t)w * per_warp, j1 = min(psi, j0 + per_warp);
    for (int64_t j = j0; j < j1; j += 32) {
      const uint32_t v = (j + lane < j1) ? row[j + lane] : 0u;
      cnt += __popc(warp_transpose32(v, lane));
    }
    cnt_s[w][lane] = cnt;
    __syncthreads();
    if (w == 0) {
      uint32_t c = 0;
      for (int k = 0; k < wpb; k++) c += cnt_s[k][lane];
      if (!((group_lanes(omega, g) >> lane) & 1u)) c = 0;
      const uint64_t s1 = warp_sum<uint64_t>(c);
      const u128 s2 = warp_sum_u128((u128)((uint64_t)c * c));
      if (lane == 0) {
        acc1 += s1;
        acc2 += s2;
      }
    }
    __syncthreads();  // cnt_s reused by the next group
  }
  uint64_t part[3] = {0, 0, 0};
  if (threadIdx.x == 0) {
    part[0] = acc1;
    part[1] = (uint64_t)acc2;
    part[2] = (uint64_t)(acc2 >> 64);
  }
  if (!publish_partials<3>(part, partials, ticket)) return;
  // the last block folds the partials, every thread a strided share
  uint64_t S1 = 0;
  u128 S2 = 0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
    S1 += partials[(size_t)b * 3];
    S2 += ((u128)partials[(size_t)b * 3 + 2] << 64) | partials[(size_t)b * 3 + 1];
  }
  S1 = warp_sum<uint64_t>(S1);
  S2 = warp_sum_u128(S2);
  __shared__ uint64_t f1[8];
  __shared__ u128 f2[8];
  if (lane == 0) {
    f1[w] = S1;
    f2[w] = S2;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  S1 = 0;
  S2 = 0;
  for (int k = 0; k < wpb; k++) {
    S1 += f1[k];
    S2 += f2[k];
  }
  *ticket = 0u;
  pbn_gr_result r;
  gr_formulas(r, S1, S2, psi, omega);
  *out = r;
}

__global__ void __launch_bounds__(256) two_state_kernel(const uint32_t *bits, int64_t cap, int64_t col,
                                                        int64_t len, int64_t omega, int G, double eps, double rr,
                                                        double s, unsigned long long *partials,
                                                        unsigned int *ticket, pbn_two_state_result *out) {
  const int lane = threadIdx.x & 31;
  const int64_t chunks = (len + 31) / 32;
  const int64_t items = (int64_t)G * chunks;
  uint64_t v[4] = {0, 0, 0, 0};  // n11, from-ones, to-ones, ones
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t it = wid; it < items; it += nwarps) {
    const int64_t g = it / chunks, ch = it - g * chunks;
    const uint32_t vm = group_lanes(omega, g);
    const uint32_t *row = bits + (size_t)g * cap + col;
    const int64_t j = ch * 32 + lane;  // window position of this lane's word
    const uint32_t w = j < len ? (row[j] & vm) : 0u;
    uint32_t nx = __shfl_down_sync(0xFFFFFFFFu, w, 1);
    if (lane == 31) nx = (j + 1 < len) ? (row[j + 1] & vm) : 0u;
    const bool pair = (j + 1 < len);
    v[3] += __popc(w);
    if (pair) {
      v[0] += __popc(w & nx);
      v[1] += __popc(w);
      v[2] += __popc(nx);
    }
  }
  block_sum64<4>(v);
  if (!publish_partials<4>(v, partials, ticket)) return;
  // the last block folds the partials, every thread a strided share
  uint64_t t[4] = {0, 0, 0, 0};
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
    for (int k = 0; k < 4; k++) t[k] += partials[(size_t)b * 4 + k];
  block_sum64<4>(t);
  if (threadIdx.x != 0) return;
  *ticket = 0u;
  pbn_two_state_result r;
  r.n11 = (int64_t)t[0];
  r.n10 = (int64_t)t[1] - r.n11;
  r.n01 = (int64_t)t[2] - r.n11;
  r.n00 = (len >= 1 ? omega * (len - 1) : 0) - r.n11 - r.n10 - r.n01;
  r.ones = (int64_t)t[3];
  r.pad = 0;
  two_state_formulas(r, omega, len, eps, rr, s);
  *out = r;
}

// ------------------------------------------------------------------- Skart

// Batch sums: chain c, batch j (j < bpc) covers window columns
// [j*kappa, (j+1)*kappa); out[c * bpc + j].
__global__ void __launch_bounds__(256) skart_batch_kernel(const uint32_t *bits, int64_t cap, int64_t col,
                                                          int64_t kappa, int64_t bpc, int64_t omega, int G,
                                                          int32_t *out) {
  const int lane = threadIdx.x & 31;
  const int64_t items = (int64_t)G * bpc;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t it = wid; it < items; it += nwarps) {
    const int64_t g = it / bpc, j = it - g * bpc;
    const uint32_t *row = bits + (size_t)g * cap + col + j * kappa;
    uint32_t cnt = 0;
    for (int64_t q = 0; q < kappa; q += 32) {
      const uint32_t w = (q + lane < kappa) ? row[q + lane] : 0u;
      cnt += __popc(warp_transpose32(w, lane));
    }
    const int64_t c = g * 32 + lane;
    if (c < omega) out[c * bpc + j] = (int32_t)cnt;
  }
}

// Moments of the batch sums and the Skart statistics, one block.
__global__ void __launch_bounds__(1024) skart_stats_kernel(const int32_t *bs, int64_t omega, int64_t bpc,
                                                           int64_t kappa, int64_t spacer, double alpha_ci,
                                                           double alpha_ran, pbn_skart_result *out) {
  const int64_t K = omega * bpc;
  __shared__ long long s_c0;
  // pass 1: total -> integer shift c0 = round(mean batch sum)
  {
    uint64_t v[1] = {0};
    for (int64_t k = threadIdx.x; k < K; k += blockDim.x) v[0] += (uint64_t)bs[k];
    block_sum64<1>(v);
    if (threadIdx.x == 0) s_c0 = (long long)((v[0] + (uint64_t)K / 2) / (uint64_t)K);
    __syncthreads();
  }
  const long long c0 = s_c0;
  const int64_t per = bpc / (spacer + 1);  // retained (spaced) batches per chain
  // pass 2: shifted moments (exact, 128-bit)
  i128 S1 = 0, S2 = 0, S3 = 0, Q = 0, Fst = 0, Lst = 0, T1 = 0, T2 = 0, D2 = 0;
  for (int64_t k = threadIdx.x; k < K; k += blockDim.x) {
    const int64_t c = k / bpc, j = k - c * bpc;
    const i128 d = (i128)((long long)bs[k] - c0);
    S1 += d; S2 += d * d; S3 += d * d * d;
    if (j + 1 < bpc) Q += d * (i128)((long long)bs[k + 1] - c0);
    if (j == 0) Fst += d;
    if (j == bpc - 1) Lst += d;
    if (j % (spacer + 1) == spacer && j / (spacer + 1) < per) {
      T1 += d; T2 += d * d;
      const int64_t jn = j + spacer + 1;
      if (jn / (spacer + 1) < per) {
        const i128 e = (i128)((long long)bs[c * bpc + jn] - c0) - d;
        D2 += e * e;
      }
    }
  }
  __shared__ i128 red[32][9];
  i128 vals[9] = {S1, S2, S3, Q, Fst, Lst, T1, T2, D2};
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 9; q++) {
    i128 x = vals[q];
    for (int o = 16; o > 0; o >>= 1) {
      uint64_t lo = (uint64_t)x, hi = (uint64_t)((u128)x >> 64);
      lo = __shfl_xor_sync(0xFFFFFFFFu, lo, o);
      hi = __shfl_xor_sync(0xFFFFFFFFu, hi, o);
      x += (i128)(((u128)hi << 64) | lo);
    }
    if (lane == 0) red[w][q] = x;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const int nw = (blockDim.x + 31) >> 5;
  for (int q = 0; q < 9; q++) {
    i128 x = 0;
    for (int k = 0; k < nw; k++) x += red[k][q];
    vals[q] = x;
  }
  const double Kd = (double)K, kap = (double)kappa;
  const double m1 = (double)vals[0] / Kd;            // mean shifted batch sum
  const double r2 = (double)vals[1] / Kd, r3 = (double)vals[2] / Kd;
  const double m2 = r2 - m1 * m1;                    // population variance (batch-sum units)
  const double m3 = r3 - 3.0 * m1 * r2 + 2.0 * m1 * m1 * m1;
  pbn_skart_result res;
  res.batches = K;
  res.mean = ((double)c0 + m1) / kap;
  res.var = (K > 1) ? m2 * Kd / (Kd - 1.0) / (kap * kap) : 0.0;
  res.skew = m2 > 0.0 ? m3 / pow(m2, 1.5) : 0.0;
  // pooled within-chain lag-1 autocorrelation
  const int64_t P = omega * (bpc - 1);
  double phi = 0.0;
  if (P > 0 && m2 > 0.0) {
    const double lsum = (double)(vals[0] - vals[5]), rsum = (double)(vals[0] - vals[4]);
    const double cov = ((double)vals[3] - m1 * (lsum + rsum) + (double)P * m1 * m1) / (double)P;
    phi = cov / m2;
  }
  if (phi > 0.999) phi = 0.999;
  if (phi < -0.999) phi = -0.999;
  res.phi = phi;
  res.A = (1.0 + phi) / (1.0 - phi);
  const double beta = res.skew / (6.0 * sqrt(Kd));
  const double tu = student_quantile(1.0 - alpha_ci / 2.0, Kd - 1.0);
  const double tl = -tu;
  const double au = cbrt(1.0 + 6.0 * beta * (tu - beta));
  const double al = cbrt(1.0 + 6.0 * beta * (tl - beta));
  const double Gu = 3.0 * (tu - beta) / (au * au + au + 1.0);
  const double Gl = 3.0 * (tl - beta) / (al * al + al + 1.0);
  const double se = sqrt(res.A * res.var / Kd);
  res.ci_lo = res.mean - Gu * se;
  res.ci_hi = res.mean - Gl * se;
  res.H = fmax(res.mean - res.ci_lo, res.ci_hi - res.mean);
  // von Neumann randomness test on the spaced batch means
  const int64_t Kp = per * omega, Pp = per > 1 ? (per - 1) * omega : 0;
  res.vn_stat = 0.0;
  res.vn_pass = 1;
  if (Pp > 0 && Kp >= 3) {
    const double t1 = (double)vals[6], t2 = (double)vals[7];
    const double ss = t2 - t1 * t1 / (double)Kp;
    if (ss > 0.0) {
      const double C = 1.0 - ((double)(Kp - 1) / (double)Pp) * (double)vals[8] / (2.0 * ss);
      const double mm = (double)(Pp + 1);
      const double crit = normal_quantile(1.0 - alpha_ran) * sqrt((mm - 2.0) / (mm * mm - 1.0));
      res.vn_stat = C;
      res.vn_pass = C <= crit;
    }
  }
  res.pad = 0;
  *out = res;
}

// ---------------------------------------------------------------- launchers

static int stat_blocks(int64_t work_warps, int wpb) {
  int64_t b = (work_warps + wpb - 1) / wpb;
  if (b < 1) b = 1;
  if (b > kMaxStatBlocks) b = kMaxStatBlocks;
  return (int)b;
}

cudaError_t scratch_init(StatsScratch &sc, cudaStream_t s) {
  cudaError_t e = cudaMalloc(&sc.partials, sizeof(unsigned long long) * kMaxStatBlocks * 8);
  if (e != cudaSuccess) return e;
  e = cudaMalloc(&sc.ticket, sizeof(unsigned int));
  if (e != cudaSuccess) return e;
  return cudaMemsetAsync(sc.ticket, 0, sizeof(unsigned int), s);
}

void scratch_free(StatsScratch &sc) {
  if (sc.partials) cudaFree(sc.partials);
  if (sc.ticket) cudaFree(sc.ticket);
  if (sc.batch) cudaFree(sc.batch);
  sc = StatsScratch();
}

cudaError_t scratch_reserve_batches(StatsScratch &sc, int64_t count, cudaStream_t s) {
  if (count <= sc.batch_cap) return cudaSuccess;
  if (sc.batch) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    cudaFree(sc.batch);
    sc.batch = nullptr;
  }
  int64_t cap = sc.batch_cap ? sc.batch_cap : 4096;
  while (cap < count) cap *= 2;
  cudaError_t e = cudaMalloc(&sc.batch, sizeof(int32_t) * cap);
  if (e != cudaSuccess) { sc.batch_cap = 0; return e; }
  sc.batch_cap = cap;
  return cudaSuccess;
}

cudaError_t launch_gelman_rubin(const pbn_chains &ch, int64_t col, int64_t psi, pbn_gr_result *out,
                                StatsScratch &sc, cudaStream_t s) {
  const int G = (int)((ch.omega + 31) / 32);
  const int blocks = (int)std::min<int64_t>(std::max(G, 1), kMaxStatBlocks);  // one block per group
  gr_kernel<<<blocks, 256, 0, s>>>(ch.bits, ch.bits_cap, col, psi, ch.omega, G, sc.partials, sc.ticket, out);
  return cudaGetLastError();
}

cudaError_t launch_two_state(const pbn_chains &ch, int64_t col, int64_t len, double eps, double r, double sconf,
                             pbn_two_state_result *out, StatsScratch &sc, cudaStream_t s) {
  const int G = (int)((ch.omega + 31) / 32);
  const int threads = 256;
  const int64_t warps = (int64_t)G * ((len + 31) / 32);
  const int blocks = stat_blocks(warps, threads / 32);
  two_state_kernel<<<blocks, threads, 0, s>>>(ch.bits, ch.bits_cap, col, len, ch.omega, G, eps, r, sconf,
                                              sc.partials, sc.ticket, out);
  return cudaGetLastError();
}

cudaError_t launch_skart(const pbn_chains &ch, int64_t col, int64_t kappa, int64_t bpc, int64_t spacer,
                         double alpha_ci, double alpha_ran, pbn_skart_result *out, StatsScratch &sc,
                         cudaStream_t s) {
  const int G = (int)((ch.omega + 31) / 32);
  cudaError_t e = scratch_reserve_batches(sc, ch.omega * bpc, s);
  if (e != cudaSuccess) return e;
  const int threads = 256;
  int64_t blocks = ((int64_t)G * bpc + 7) / 8;
  if (blocks > 65535) blocks = 65535;
  if (blocks < 1) blocks = 1;
  skart_batch_kernel<<<(unsigned)blocks, threads, 0, s>>>(ch.bits, ch.bits_cap, col, kappa, bpc, ch.omega, G,
                                                          sc.batch);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  skart_stats_kernel<<<1, 1024, 0, s>>>(sc.batch, ch.omega, bpc, kappa, spacer, alpha_ci, alpha_ran, out);
  return cudaGetLastError();
}

cudaError_t launch_skart_into(const pbn_chains &ch, int64_t col, int64_t kappa, int64_t bpc, int64_t spacer,
                              double alpha_ci, double alpha_ran, pbn_skart_result *out, int32_t *batch,
                              cudaStream_t s) {
  const int G = (int)((ch.omega + 31) / 32);
  int64_t blocks = ((int64_t)G * bpc + 7) / 8;
  if (blocks > 65535) blocks = 65535;
  if (blocks < 1) blocks = 1;
  skart_batch_kernel<<<(unsigned)blocks, 256, 0, s>>>(ch.bits, ch.bits_cap, col, kappa, bpc, ch.omega, G, batch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  skart_stats_kernel<<<1, 1024, 0, s>>>(batch, ch.omega, bpc, kappa, spacer, alpha_ci, alpha_ran, out);
  return cudaGetLastError();
}

}  // namespace pbn
