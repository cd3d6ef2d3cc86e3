// Device helpers of the bitstream statistics (exact integer reductions and
// the FP64 formulas), shared by the single-query and batched kernels.
#pragma once

#include <math.h>

#include "pbn_internal.cuh"

namespace pbn {

typedef unsigned __int128 u128;
typedef __int128 i128;

// ------------------------------------------------------------------ helpers

// 32x32 bit transpose across a warp: lane j holds row j on entry; on exit
// lane c holds column c (bit j = bit c of row j).  Each stage swaps the
// off-diagonal s x s blocks between lanes j and j^s.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, int lane) {
  const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int k = 0; k < 5; k++) {
    const int s = 16 >> k;
    const uint32_t m = masks[k];
    const uint32_t y = __shfl_xor_sync(0xFFFFFFFFu, x, s);
    x = (lane & s) ? ((x & ~m) | ((y & ~m) >> s)) : ((x & m) | ((y & m) << s));
  }
  return x;
}

__device__ __forceinline__ uint32_t group_lanes(int64_t omega, int64_t g) {
  int64_t rem = omega - g * 32;
  return rem >= 32 ? 0xFFFFFFFFu : (rem <= 0 ? 0u : ((1u << rem) - 1u));
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

__device__ __forceinline__ u128 warp_sum_u128(u128 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    uint64_t lo = (uint64_t)v, hi = (uint64_t)(v >> 64);
    lo = __shfl_xor_sync(0xFFFFFFFFu, lo, o);
    hi = __shfl_xor_sync(0xFFFFFFFFu, hi, o);
    v += ((u128)hi << 64) | lo;
  }
  return v;
}

// Block partials: NV 64-bit values per block.  Returns true in the last
// block to finish, after which partials[0..gridDim.x) are all visible.
template <int NV>
__device__ inline bool publish_partials(const uint64_t (&vals)[NV], unsigned long long *partials, unsigned int *ticket) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    for (int k = 0; k < NV; k++) partials[(size_t)blockIdx.x * NV + k] = vals[k];
    __threadfence();
    unsigned int t = atomicAdd(ticket, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// Block-wide sum of NV 64-bit values (wrapping; callers split 128-bit values).
template <int NV>
__device__ inline void block_sum64(uint64_t (&v)[NV]) {
  __shared__ uint64_t red[32][NV];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; k++) v[k] = warp_sum<uint64_t>(v[k]);
  if (lane == 0)
    for (int k = 0; k < NV; k++) red[w][k] = v[k];
  __syncthreads();
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++) v[k] = lane < nw ? red[lane][k] : 0ull;
#pragma unroll
    for (int k = 0; k < NV; k++) v[k] = warp_sum<uint64_t>(v[k]);
  }
  __syncthreads();
}

// -------------------------------------------------------- FP64 math pieces

// Phi(-x) for x >= 0 through erfc, accurate in the tail.
__device__ inline double upper_normal_tail(double x) { return 0.5 * erfc(x * 0.70710678118654752440); }

// x >= 0 with Phi(-x) = tail (0 < tail <= 1/2): start from the rational
// approximation of Abramowitz & Stegun 26.2.23 (|error| < 4.5e-4) and refine
// with Newton steps on Phi(-x), whose derivative is -pdf(x).
__device__ inline double normal_tail_quantile(double tail) {
  double x = sqrt(-2.0 * log(tail));
  x = x - (2.515517 + 0.802853 * x + 0.010328 * x * x) /
              (1.0 + 1.432788 * x + 0.189269 * x * x + 0.001308 * x * x * x);
  if (x < 0.0) x = 0.0;
  for (int it = 0; it < 60; it++) {
    const double q = upper_normal_tail(x);
    const double pdf = 0.39894228040143267794 * exp(-0.5 * x * x);
    const double step = (q - tail) / pdf;
    x += step;
    if (fabs(step) <= 4e-16 * fmax(1.0, x)) break;
  }
  return x;
}

__device__ inline double normal_quantile(double q) {
  if (q == 0.5) return 0.0;
  return q < 0.5 ? -normal_tail_quantile(q) : normal_tail_quantile(1.0 - q);
}

// ln Gamma(a+b) - ln Gamma(a); for large a by differencing Stirling's series.
__device__ inline double ln_gamma_ratio(double a, double b) {
  if (a < 25.0) return lgamma(a + b) - lgamma(a);
  auto tail = [](double z) {
    const double iz = 1.0 / z, iz2 = iz * iz;
    return iz * (1.0 / 12.0 - iz2 * (1.0 / 360.0 - iz2 * (1.0 / 1260.0 - iz2 * (1.0 / 1680.0))));
  };
  return (a - 0.5) * log1p(b / a) + b * log(a + b) - b + (tail(a + b) - tail(a));
}

// Regularised incomplete beta function I_x(a, b) from its continued fraction
// (DLMF 8.17.22): I_x(a,b) = x^a (1-x)^b / (a B(a,b)) K, where
// K = 1/(1 + d_1/(1 + d_2/(1 + ...))) with
//   d_{2m}   =  m (b - m) x / ((a + 2m - 1)(a + 2m)),
//   d_{2m+1} = -(a + m)(a + b + m) x / ((a + 2m)(a + 2m + 1)).
// K is the limit of the convergents P_j / Q_j, P_j = P_{j-1} + d_{j-1} P_{j-2}
// and Q_j likewise (P_0 = 0, P_1 = 1, Q_0 = Q_1 = 1).  Each pass of the loop
// below advances two convergents (one even and one odd coefficient) and then
// divides the kept pairs by the newest Q, so the newest P is the convergent.
__device__ inline double ibeta_fraction(double a, double b, double x) {
  double p2 = 0.0, p1 = 1.0;  // P_{j-2}, P_{j-1}; Q_{j-1} = 1 after scaling
  double q2 = 1.0;            // Q_{j-2}
  double last = 1.0;
  for (int m = 1; m < 100000; ++m) {
    const double fm = (double)m;
    const double c_odd = -(a + fm - 1.0) * (a + b + fm - 1.0) * x / ((a + 2.0 * fm - 2.0) * (a + 2.0 * fm - 1.0));
    const double c_even = fm * (b - fm) * x / ((a + 2.0 * fm - 1.0) * (a + 2.0 * fm));
    // d_{2m-1} (for m = 1: d_1 = -(a+b) x / (a+1), the odd formula at index 0)
    double pn = p1 + c_odd * p2, qn = 1.0 + c_odd * q2;
    if (qn == 0.0) qn = 1e-300;
    p2 = p1 / qn; q2 = 1.0 / qn; p1 = pn / qn;
    // d_{2m}
    pn = p1 + c_even * p2; qn = 1.0 + c_even * q2;
    if (qn == 0.0) qn = 1e-300;
    p2 = p1 / qn; q2 = 1.0 / qn; p1 = pn / qn;
    if (fabs(p1 - last) <= 1e-16 * fabs(p1)) break;
    last = p1;
  }
  return p1;
}

// I_x(a, b) with y = 1 - x given exactly.  The fraction is used where it
// converges fast, x < (a+1)/(a+b+2); elsewhere I_x(a,b) = 1 - I_y(b,a).
__device__ inline double reg_incomplete_beta(double a, double b, double x, double y) {
  if (x <= 0.0) return 0.0;
  if (y <= 0.0) return 1.0;
  const bool flip = !(x < (a + 1.0) / (a + b + 2.0));
  const double ea = flip ? b : a, eb = flip ? a : b;
  const double ex = flip ? y : x, ey = flip ? x : y;
  // logs of ex and ey; the one near 1 from log1p of the other, exact to rounding
  const double lx = ex > 0.5 ? log1p(-ey) : log(ex);
  const double ly = ey > 0.5 ? log1p(-ex) : log(ey);
  // ln B(ea, eb) through the larger argument, so no two large ln Gamma cancel
  const double big = fmax(ea, eb), small = fmin(ea, eb);
  const double lnB = lgamma(small) - ln_gamma_ratio(big, small);
  const double I = exp(ea * lx + eb * ly - log(ea) - lnB) * ibeta_fraction(ea, eb, ex);
  return flip ? 1.0 - I : I;
}

// P(T > t) for Student t with nu degrees of freedom (t >= 0):
// I_x(nu/2, 1/2) / 2 with x = nu/(nu + t^2), 1 - x = t^2/(nu + t^2).
__device__ inline double student_upper_tail(double t, double nu) {
  const double x = nu / (nu + t * t), y = (t * t) / (nu + t * t);
  if (y <= 0.0) return 0.5;
  return 0.5 * reg_incomplete_beta(0.5 * nu, 0.5, x, y);
}

// Student t quantile: Newton on the upper tail from the normal quantile.
__device__ inline double student_quantile(double q, double nu) {
  if (q == 0.5) return 0.0;
  const double tail = q < 0.5 ? q : 1.0 - q;
  double t = normal_tail_quantile(tail);
  // first term of the Cornish-Fisher expansion of t in z for a closer start
  t = t + (t * t * t + t) / (4.0 * nu);
  const double lc = ln_gamma_ratio(0.5 * nu, 0.5) - 0.5 * log(nu * 3.14159265358979323846);
  for (int it = 0; it < 100; it++) {
    const double pdf = exp(lc - 0.5 * (nu + 1.0) * log1p(t * t / nu));
    const double step = (student_upper_tail(t, nu) - tail) / pdf;
    t += step;
    if (t < 0.0) t = 0.0;
    if (fabs(step) <= 4e-16 * fmax(1.0, t)) break;
  }
  return q < 0.5 ? -t : t;
}

// --------------------------------------------------------------- two-state

__device__ inline void two_state_formulas(pbn_two_state_result &r, int64_t omega, int64_t len, double eps, double rr,
                                   double s) {
  r.status = PBN_OK;
  r.alpha = r.beta = 0.0;
  r.M = r.N = 0;
  r.prob = (double)r.ones / ((double)omega * (double)len);
  if (len < 2 || r.n01 == 0 || r.n10 == 0) { r.status = PBN_ERR_INSUFFICIENT; return; }
  const double a = (double)r.n01 / (double)(r.n00 + r.n01);
  const double b = (double)r.n10 / (double)(r.n10 + r.n11);
  r.alpha = a;
  r.beta = b;
  const double z = normal_quantile(0.5 * (1.0 + s));
  const double apb = a + b;
  const double Nreal = a * b * (2.0 - a - b) / (apb * apb * apb) * (z * z) / (rr * rr);
  r.N = (int64_t)ceil(Nreal);
  const double lam = fabs(1.0 - a - b);
  if (lam == 0.0) { r.M = 0; return; }
  if (lam >= 1.0) { r.status = PBN_ERR_NOT_CONVERGED; return; }
  double Mreal = log(eps * apb / (a > b ? a : b)) / log(lam);
  if (Mreal < 0.0) Mreal = 0.0;
  r.M = (int64_t)ceil(Mreal);
}


// R-hat from the exact sums S1 = sum c_i, S2 = sum c_i^2 of ones counts over
// windows of psi positions of omega chains (Alg. GR with s_i^2 over psi-1):
// W = (psi S1 - S2) / (omega psi (psi-1)),  B = (omega S2 - S1^2) / (omega (omega-1) psi).
__device__ inline void gr_formulas(pbn_gr_result &r, uint64_t S1, u128 S2, int64_t psi, int64_t omega) {
  const double p = (double)psi, w_ = (double)omega;
  const i128 wnum = (i128)((u128)psi * S1) - (i128)S2;
  const i128 bnum = (i128)((u128)omega * S2) - (i128)((u128)S1 * S1);
  const double W = (double)wnum / (w_ * p * (p - 1.0));
  const double B = (double)bnum / (w_ * (w_ - 1.0) * p);
  const double sigma2 = (1.0 - 1.0 / p) * W + B / p;
  r.W = W;
  r.B = B;
  r.sigma2 = sigma2;
  r.rhat = (W > 0.0) ? sqrt(sigma2 / W) : (double)INFINITY;
  r.S1 = S1;
  r.S2_lo = (uint64_t)S2;
  r.S2_hi = (uint64_t)(S2 >> 64);
}

}  // namespace pbn
