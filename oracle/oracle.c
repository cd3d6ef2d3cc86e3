/*
 * oracle.c -- plain, single-threaded CPU reference of the parallel PBN
 * steady-state method (Mizera, Pang & Yuan, "Parallel Approximate Steady-state
 * Analysis of Large Probabilistic Boolean Networks").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA path; it is written for clarity, not
 * speed: one chain at a time, one node at a time, one byte per node value.
 *
 * Conventions fixed here where the paper is silent (the CUDA path implements
 * the same conventions independently):
 *   - Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
 *     key = (seed lo32, seed hi32).  Chain c belongs to group g = c / 32 and
 *     lane c % 32.  For node i and transition t (state t -> state t+1) the
 *     digit words R_0..R_31 come from blocks b = 0..7:
 *        (R_4b .. R_4b+3) = Philox(ctr = (i, t lo32, (t hi32 & 0xFFFFFF) | b<<24, g))
 *     and chain c's uniform is u = sum_d bit_{c%32}(R_d) * 2^(31-d)
 *     (bit c%32 of R_0 is the most significant digit).
 *   - Initial state (state 0): node i of chain c is bit c%32 of word 0 of
 *     Philox(ctr = (i, 0xFFFFFFFF, 0xFFFFFFFF, g)).
 *   - Quantisation: P32 = min(round(p 2^32), 2^32-1).  For node i with
 *     functions j = 0..l-1 and running sums S_j = c_0 + .. + c_j (fp64, left to
 *     right): T_j = P32 + min(round((2^32-P32) S_j), 2^32-P32), clamped to
 *     2^32-1, for j < l-1; T_{l-1} = 2^32.  The category of u is the number of
 *     values in (P32, T_0, .., T_{l-2}) that are <= u: category 0 means the
 *     node is perturbed (gamma_i = 1), category j+1 selects function j.
 *   - Truth table: value = bit j = (sum_m s[parent_m] << m) of the function's
 *     table, stored as words: bit j % 32 of word j / 32 (k <= 16 parents).
 *   - Perturbation reading PER_NODE (mode 0): a perturbed node flips, every
 *     other node takes its selected function's value.  Reading GLOBAL (mode 1):
 *     if any node is perturbed the next state is s XOR gamma, else every node
 *     takes its selected function's value (Sec. 2.2).
 *   - Trajectory of length L = states 1..L (the initial state is not a sample);
 *     position j (0-based) holds state j+1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_INVALID 1
#define ORC_ERR_OOM 2
#define ORC_ERR_NOT_CONVERGED 5
#define ORC_MAX_PARENTS 16

/* ------------------------------------------------------------------------- */
/* Philox4x32-10, from the round function and key schedule published in       */
/* Salmon et al., SC'11: two 32x32->64 multiplies per round, Weyl key bumps.  */
/* ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    const uint64_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        uint64_t prod0 = M0 * (uint64_t)x0;
        uint64_t prod1 = M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += W0; k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ------------------------------------------------------------------------- */
/* PBN G(V,F) (Sec. 2.2), CSR arrays as supplied by the caller.               */
/* ------------------------------------------------------------------------- */
typedef struct {
    int32_t n;
    int32_t F;
    const int32_t *fn_offset;   /* [n+1] */
    const int32_t *par_offset;  /* [F+1] */
    const int32_t *parents;     /* [par_offset[F]] */
    const int32_t *tt_offset;   /* [F+1] truth-table words of function f: tt_offset[f] .. tt_offset[f+1]-1 */
    const uint32_t *tt_words;   /* bit j of a table is bit j % 32 of its word j / 32 */
    const double *select_prob;  /* [F] */
    double p;
} orc_net;

int orc_validate(const orc_net *net) {
    if (net->n < 1 || net->F < net->n) return ORC_ERR_INVALID;
    if (!(net->p >= 0.0 && net->p < 1.0)) return ORC_ERR_INVALID;
    if (net->fn_offset[0] != 0 || net->fn_offset[net->n] != net->F) return ORC_ERR_INVALID;
    for (int i = 0; i < net->n; i++) {
        int l = net->fn_offset[i + 1] - net->fn_offset[i];
        if (l < 1) return ORC_ERR_INVALID;
        double sum = 0.0;
        for (int f = net->fn_offset[i]; f < net->fn_offset[i + 1]; f++) {
            double c = net->select_prob[f];
            if (!(c >= 0.0 && c <= 1.0)) return ORC_ERR_INVALID;
            sum += c;
        }
        if (fabs(sum - 1.0) > 1e-9) return ORC_ERR_INVALID;
    }
    if (net->par_offset[0] != 0) return ORC_ERR_INVALID;
    for (int f = 0; f < net->F; f++) {
        int k = net->par_offset[f + 1] - net->par_offset[f];
        if (k < 0 || k > ORC_MAX_PARENTS) return ORC_ERR_INVALID;
        int words = (1 << k) / 32 > 1 ? (1 << k) / 32 : 1;
        if (net->tt_offset[f + 1] - net->tt_offset[f] != words) return ORC_ERR_INVALID;
        for (int m = 0; m < k; m++) {
            int v = net->parents[net->par_offset[f] + m];
            if (v < 0 || v >= net->n) return ORC_ERR_INVALID;
        }
    }
    return ORC_OK;
}

/* Perturbation threshold: gamma_i = 1 iff u < P32 (probability P32 / 2^32). */
uint32_t orc_perturb_threshold(double p) {
    double v = p * 4294967296.0;
    long long q = llround(v);
    if (q < 0) q = 0;
    if (q > 4294967295LL) q = 4294967295LL;
    return (uint32_t)q;
}

/* Upper category bounds T_j for every function (as 64-bit so 2^32 fits). */
void orc_select_thresholds(const orc_net *net, uint64_t *thr) {
    uint32_t P32 = orc_perturb_threshold(net->p);
    uint64_t span = 4294967296ULL - P32;
    for (int i = 0; i < net->n; i++) {
        int f0 = net->fn_offset[i], f1 = net->fn_offset[i + 1];
        double S = 0.0;
        for (int f = f0; f < f1; f++) {
            S += net->select_prob[f];
            if (f == f1 - 1) { thr[f] = 4294967296ULL; break; }
            long long q = llround((double)span * S);
            if (q < 0) q = 0;
            if ((uint64_t)q > span) q = (long long)span;
            uint64_t T = (uint64_t)P32 + (uint64_t)q;
            if (T > 4294967295ULL) T = 4294967295ULL;
            thr[f] = T;
        }
    }
}

/* Philox counter of digit block b for (node, transition t, group). */
static void digit_block(uint64_t seed, int32_t node, uint64_t t, uint64_t group, int b, uint32_t out[4]) {
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)node, (uint32_t)t,
                       ((uint32_t)(t >> 32) & 0xFFFFFFu) | ((uint32_t)b << 24),
                       (uint32_t)group};
    orc_philox4x32_10(ctr, key, out);
}

/* All 32 digit words of the chain group (node, t, group). */
static void digit_words(uint64_t seed, int32_t node, uint64_t t, uint64_t group, uint32_t R[32]) {
    for (int b = 0; b < 8; b++) digit_block(seed, node, t, group, b, R + 4 * b);
}

static uint32_t uniform_from_words(const uint32_t R[32], int lane) {
    uint32_t u = 0;
    for (int d = 0; d < 32; d++) u |= ((R[d] >> lane) & 1u) << (31 - d);
    return u;
}

/* u of chain `chain` at (node, t). */
uint32_t orc_uniform(uint64_t seed, int32_t node, uint64_t t, int64_t chain) {
    uint32_t R[32];
    digit_words(seed, node, t, (uint64_t)chain >> 5, R);
    return uniform_from_words(R, (int)(chain & 31));
}

/* Initial states (any initial state is allowed, Sec. 2.2; here fair coins). */
void orc_init_states_from(const orc_net *net, uint64_t seed, int64_t chain0, int64_t omega, uint8_t *states) {
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t row = 0; row < omega; row++) {
        int64_t c = chain0 + row;
        for (int i = 0; i < net->n; i++) {
            uint32_t ctr[4] = {(uint32_t)i, 0xFFFFFFFFu, 0xFFFFFFFFu, (uint32_t)((uint64_t)c >> 5)};
            uint32_t out[4];
            orc_philox4x32_10(ctr, key, out);
            states[row * net->n + i] = (uint8_t)((out[0] >> (c & 31)) & 1u);
        }
    }
}

void orc_init_states(const orc_net *net, uint64_t seed, int64_t omega, uint8_t *states) {
    orc_init_states_from(net, seed, 0, omega, states);
}

/* Category of u at node i (0 = perturbed, j+1 = function j). */
static int category(const orc_net *net, const uint64_t *thr, uint32_t P32, int i, uint32_t u) {
    if (u < P32) return 0;
    int f0 = net->fn_offset[i], f1 = net->fn_offset[i + 1];
    for (int f = f0; f < f1; f++)
        if ((uint64_t)u < thr[f]) return f - f0 + 1;
    return f1 - f0; /* unreachable: the last bound is 2^32 */
}

/* Boolean function value f(s) by truth-table lookup on the parents. */
static int eval_fn(const orc_net *net, int f, const uint8_t *s) {
    uint32_t idx = 0;
    int k = net->par_offset[f + 1] - net->par_offset[f];
    for (int m = 0; m < k; m++) idx |= (uint32_t)s[net->parents[net->par_offset[f] + m]] << m;
    return (int)((net->tt_words[net->tt_offset[f] + (idx >> 5)] >> (idx & 31u)) & 1u);
}

static int indicator(const uint8_t *s, const int32_t *soi_nodes, const uint8_t *soi_values, int soi_size) {
    for (int m = 0; m < soi_size; m++)
        if (s[soi_nodes[m]] != soi_values[m]) return 0;
    return 1;
}

/*
 * Advance omega chains by `steps` transitions, transitions t0 .. t0+steps-1
 * (Sec. 2.2: synchronous update of all nodes from the old state, with
 * perturbations).  ind (may be NULL) receives ind[c*ind_stride + s] = indicator
 * of the meta state (Sec. 3.1) of chain c's state after transition t0+s.
 */
int orc_simulate_from(const orc_net *net, int mode, uint64_t seed, int64_t chain0, int64_t omega, uint64_t t0,
                      int64_t steps, uint8_t *states, const int32_t *soi_nodes, const uint8_t *soi_values,
                      int32_t soi_size, uint8_t *ind, int64_t ind_stride) {
    int n = net->n;
    uint64_t *thr = (uint64_t *)malloc(sizeof(uint64_t) * net->F);
    uint8_t *next = (uint8_t *)malloc((size_t)n);
    uint8_t *cat = (uint8_t *)malloc((size_t)n);
    uint32_t *R = (uint32_t *)malloc(sizeof(uint32_t) * 32 * (size_t)n);
    if (!thr || !next || !cat || !R) { free(thr); free(next); free(cat); free(R); return ORC_ERR_OOM; }
    orc_select_thresholds(net, thr);
    uint32_t P32 = orc_perturb_threshold(net->p);
    for (int64_t s = 0; s < steps; s++) {
        uint64_t t = t0 + (uint64_t)s;
        int64_t cached_group = -1;
        for (int64_t row = 0; row < omega; row++) {
            int64_t c = chain0 + row;            /* global chain index */
            int64_t g = c >> 5;
            int lane = (int)(c & 31);
            if (g != cached_group) {
                /* the group's digit words for every node at transition t */
                for (int i = 0; i < n; i++) digit_words(seed, i, t, (uint64_t)g, R + 32 * (size_t)i);
                cached_group = g;
            }
            {
                uint8_t *st = states + row * n;
                int any_perturbed = 0;
                for (int i = 0; i < n; i++) {
                    uint32_t u = uniform_from_words(R + 32 * (size_t)i, lane);
                    cat[i] = (uint8_t)category(net, thr, P32, i, u);
                    if (cat[i] == 0) any_perturbed = 1;
                }
                for (int i = 0; i < n; i++) {
                    if (mode == 0) {
                        if (cat[i] == 0) next[i] = (uint8_t)(st[i] ^ 1u);
                        else next[i] = (uint8_t)eval_fn(net, net->fn_offset[i] + cat[i] - 1, st);
                    } else {
                        if (any_perturbed) next[i] = (uint8_t)(st[i] ^ (cat[i] == 0 ? 1u : 0u));
                        else next[i] = (uint8_t)eval_fn(net, net->fn_offset[i] + cat[i] - 1, st);
                    }
                }
                memcpy(st, next, (size_t)n);
                if (ind) ind[row * ind_stride + s] = (uint8_t)indicator(st, soi_nodes, soi_values, soi_size);
            }
        }
    }
    free(thr); free(next); free(cat); free(R);
    return ORC_OK;
}

/* Chains 0 .. omega-1 (see orc_simulate_from). */
int orc_simulate(const orc_net *net, int mode, uint64_t seed, int64_t omega, uint64_t t0, int64_t steps,
                 uint8_t *states, const int32_t *soi_nodes, const uint8_t *soi_values, int32_t soi_size,
                 uint8_t *ind, int64_t ind_stride) {
    return orc_simulate_from(net, mode, seed, 0, omega, t0, steps, states, soi_nodes, soi_values, soi_size, ind,
                             ind_stride);
}

/* ------------------------------------------------------------------------- */
/* Gelman & Rubin (Sec. 4.1, Alg. GR): mean and standard deviation of the last */
/* psi values of each chain, between (B) and within (W) variances, sigma^2,   */
/* R-hat.  Sample variance with denominator psi-1; W = 0 gives R-hat = +inf.  */
/* x[c*stride + start + j], j < psi.                                          */
/* ------------------------------------------------------------------------- */
double orc_gelman_rubin(const uint8_t *x, int64_t omega, int64_t stride, int64_t start, int64_t psi) {
    double *mu = (double *)malloc(sizeof(double) * omega);
    double *s2 = (double *)malloc(sizeof(double) * omega);
    for (int64_t c = 0; c < omega; c++) {
        const uint8_t *xc = x + c * stride + start;
        double m = 0.0;
        for (int64_t j = 0; j < psi; j++) m += xc[j];
        m /= (double)psi;
        double v = 0.0;
        for (int64_t j = 0; j < psi; j++) { double d = xc[j] - m; v += d * d; }
        mu[c] = m;
        s2[c] = v / (double)(psi - 1);
    }
    double mu_all = 0.0;
    for (int64_t c = 0; c < omega; c++) mu_all += mu[c];
    mu_all /= (double)omega;
    double B = 0.0, W = 0.0;
    for (int64_t c = 0; c < omega; c++) { double d = mu[c] - mu_all; B += d * d; W += s2[c]; }
    B *= (double)psi / (double)(omega - 1);
    W /= (double)omega;
    free(mu); free(s2);
    double sigma2 = (1.0 - 1.0 / (double)psi) * W + B / (double)psi;
    if (!(W > 0.0)) return INFINITY;
    return sqrt(sigma2 / W);
}

/* ------------------------------------------------------------------------- */
/* Standard normal quantile Phi^-1(q): Newton's method on                     */
/* Phi(x) = erfc(-x/sqrt 2)/2 from a bisection-bracketed start.               */
/* ------------------------------------------------------------------------- */
/* Lower tail Phi(-x) = erfc(x/sqrt 2)/2 for x >= 0, accurate in the tail. */
static double norm_upper_tail(double x) { return 0.5 * erfc(x / sqrt(2.0)); }

/* Solve Phi(-x) = tail for x >= 0 (tail <= 1/2): bisection to a bracket,
 * then Newton steps on the tail function. */
static double norm_tail_inverse(double tail) {
    double lo = 0.0, hi = 40.0;
    for (int it = 0; it < 200 && hi - lo > 1e-3; it++) {
        double mid = 0.5 * (lo + hi);
        if (norm_upper_tail(mid) > tail) lo = mid; else hi = mid;
    }
    double x = 0.5 * (lo + hi);
    for (int it = 0; it < 100; it++) {
        double pdf = exp(-0.5 * x * x) / sqrt(2.0 * M_PI);
        double step = (tail - norm_upper_tail(x)) / pdf;   /* d/dx Phi(-x) = -pdf */
        x -= step;
        if (fabs(step) <= 1e-16 * (1.0 + fabs(x))) break;
    }
    return x;
}

double orc_norm_ppf(double q) {
    if (!(q > 0.0 && q < 1.0)) return NAN;
    if (q == 0.5) return 0.0;
    if (q < 0.5) return -norm_tail_inverse(q);
    return norm_tail_inverse(1.0 - q);   /* 1 - q is exact for q in [1/2, 1) */
}

/* ------------------------------------------------------------------------- */
/* Two-state Markov chain (Sec. 3.1, Alg. 1 line 8): burn-in M and sample     */
/* size N from alpha, beta, eps, r, s.                                        */
/*   M = ceil( log(eps (a+b) / max(a,b)) / log|1-a-b| )                       */
/*   N = ceil( a b (2-a-b) / (a+b)^3 * (Phi^-1((1+s)/2))^2 / r^2 )            */
/* |1-a-b| = 0 gives M = 0.  Returns ORC_ERR_INVALID when a or b is 0 (the    */
/* formulas are then undefined for this purpose) and ORC_ERR_NOT_CONVERGED    */
/* when a = b = 1 (a periodic two-state chain never forgets its start).       */
/* ------------------------------------------------------------------------- */
int orc_two_state_MN(double a, double b, double eps, double r, double s, int64_t *M, int64_t *N) {
    if (!(a > 0.0) || !(b > 0.0)) return ORC_ERR_INVALID;
    double z = orc_norm_ppf(0.5 * (1.0 + s));
    double apb = a + b;
    double Nreal = a * b * (2.0 - a - b) / (apb * apb * apb) * (z * z) / (r * r);
    *N = (int64_t)ceil(Nreal);
    double lam = fabs(1.0 - a - b);
    if (lam == 0.0) { *M = 0; return ORC_OK; }
    if (lam >= 1.0) return ORC_ERR_NOT_CONVERGED;
    double num = log(eps * apb / (a > b ? a : b));
    double Mreal = num / log(lam);
    if (Mreal < 0.0) Mreal = 0.0;
    *M = (int64_t)ceil(Mreal);
    return ORC_OK;
}

/* Transition counts n[0]=n00, n[1]=n01, n[2]=n10, n[3]=n11 within each chain
 * between consecutive positions start..start+len-1 (len-1 pairs per chain). */
void orc_transition_counts(const uint8_t *x, int64_t omega, int64_t stride, int64_t start, int64_t len,
                           int64_t n4[4]) {
    n4[0] = n4[1] = n4[2] = n4[3] = 0;
    for (int64_t c = 0; c < omega; c++) {
        const uint8_t *xc = x + c * stride + start;
        for (int64_t j = 0; j + 1 < len; j++) n4[(xc[j] << 1) | xc[j + 1]]++;
    }
}

/* ------------------------------------------------------------------------- */
/* Drivers: Alg. GR followed by Alg. 3 (two-state) or Alg. 4 (Skart).          */
/* The chains' indicator history is kept in one byte per chain and position.  */
/* ------------------------------------------------------------------------- */
typedef struct {
    const orc_net *net;
    int mode;
    uint64_t seed;
    int64_t omega;
    const int32_t *soi_nodes;
    const uint8_t *soi_values;
    int32_t soi_size;
    uint8_t *states;     /* omega * n */
    uint8_t *x;          /* omega * cap indicator history, position j = state j+1 */
    int64_t cap;
    int64_t L;           /* current chain length */
    int64_t chain0;      /* global index of the first chain (0 unless set) */
} chains_t;

static int chains_reserve(chains_t *ch, int64_t len) {
    if (len <= ch->cap) return ORC_OK;
    int64_t ncap = ch->cap ? ch->cap : 1024;
    while (ncap < len) ncap *= 2;
    uint8_t *nx = (uint8_t *)calloc((size_t)(ch->omega * ncap), 1);
    if (!nx) return ORC_ERR_OOM;
    for (int64_t c = 0; c < ch->omega; c++) memcpy(nx + c * ncap, ch->x + c * ch->cap, (size_t)ch->L);
    free(ch->x);
    ch->x = nx;
    ch->cap = ncap;
    return ORC_OK;
}

/* Extend all chains to length `len` (no-op if already that long). */
static int chains_extend_to(chains_t *ch, int64_t len) {
    if (len <= ch->L) return ORC_OK;
    int rc = chains_reserve(ch, len);
    if (rc) return rc;
    int64_t steps = len - ch->L;
    uint8_t *tmp = (uint8_t *)malloc((size_t)(ch->omega * steps));
    if (!tmp) return ORC_ERR_OOM;
    rc = orc_simulate_from(ch->net, ch->mode, ch->seed, ch->chain0, ch->omega, (uint64_t)ch->L, steps, ch->states,
                           ch->soi_nodes, ch->soi_values, ch->soi_size, tmp, steps);
    for (int64_t c = 0; c < ch->omega; c++) memcpy(ch->x + c * ch->cap + ch->L, tmp + c * steps, (size_t)steps);
    free(tmp);
    ch->L = len;
    return rc;
}

typedef struct {
    /* inputs */
    int64_t omega;
    int64_t psi0;
    double rhat_threshold;
    int64_t max_length;      /* cap on the chain length; exceeding it is NOT_CONVERGED */
    int32_t mode;
    uint64_t seed;
    double eps, r, s;
    /* outputs */
    double prob;
    double rhat;
    double alpha, beta;
    int64_t psi;             /* final burn-in (G&R psi, raised to M if needed) */
    int64_t gr_psi;          /* psi returned by Alg. GR */
    int64_t length;          /* final chain length */
    int64_t sample_size;     /* omega * (length - psi) */
    int64_t M, N;
    int64_t n4[4];
    int64_t ones;
    int32_t gr_rounds;
    int32_t ts_rounds;
    int32_t status;
} orc_two_state_run;

static int chains_open(chains_t *ch, const orc_net *net, int mode, uint64_t seed, int64_t omega,
                       const int32_t *soi_nodes, const uint8_t *soi_values, int32_t soi_size) {
    memset(ch, 0, sizeof(*ch));
    ch->net = net; ch->mode = mode; ch->seed = seed; ch->omega = omega;
    ch->soi_nodes = soi_nodes; ch->soi_values = soi_values; ch->soi_size = soi_size;
    ch->states = (uint8_t *)malloc((size_t)(omega * net->n));
    if (!ch->states) return ORC_ERR_OOM;
    orc_init_states(net, seed, omega, ch->states);
    return ORC_OK;
}

static void chains_close(chains_t *ch) { free(ch->states); free(ch->x); }

/* Alg. GR: start from length 2*psi0; compute R-hat on the last psi values;
 * double psi until R-hat < threshold.  Returns the last checked psi. */
static int run_gelman_rubin(chains_t *ch, int64_t psi0, double thr, int64_t max_length,
                            int64_t *psi_out, double *rhat_out, int32_t *rounds) {
    int64_t psi = psi0;
    *rounds = 0;
    for (;;) {
        if (2 * psi > max_length) return ORC_ERR_NOT_CONVERGED;
        int rc = chains_extend_to(ch, 2 * psi);
        if (rc) return rc;
        double R = orc_gelman_rubin(ch->x, ch->omega, ch->cap, psi, psi);
        (*rounds)++;
        *rhat_out = R;
        if (R < thr) { *psi_out = psi; return ORC_OK; }
        psi *= 2;
    }
}

/*
 * Alg. 3 (Sec. 4.2), read as follows where the printed steps are garbled:
 *  - the merged sample is every chain's positions [psi, L) (the second halves
 *    after Alg. GR: no further burn-in);
 *  - alpha = n01/(n00+n01), beta = n10/(n10+n11) from transitions within
 *    chains; N by Alg. 1 line 8;
 *  - extend_by = ceil((N - omega*n)/omega) with n = L - psi; stop extending
 *    when N <= omega*n (the text: N not bigger than the merged sample);
 *  - then M by Alg. 1 line 8; if M > psi, drop the first M - psi values of
 *    every chain (psi := M) and repeat, else stop;
 *  - the estimate is the fraction of ones in the final merged sample.
 *  A window with n01 = 0 or n10 = 0 (or fewer than 2 positions) cannot give
 *  alpha, beta: the chains are extended by max(n, 2) positions and counted again.
 */
int orc_estimate_two_state(const orc_net *net, const int32_t *soi_nodes, const uint8_t *soi_values,
                           int32_t soi_size, orc_two_state_run *run) {
    chains_t ch;
    int rc = chains_open(&ch, net, run->mode, run->seed, run->omega, soi_nodes, soi_values, soi_size);
    if (rc) return rc;
    run->status = ORC_OK;
    int64_t psi;
    rc = run_gelman_rubin(&ch, run->psi0, run->rhat_threshold, run->max_length, &psi, &run->rhat, &run->gr_rounds);
    if (rc) { run->status = rc; chains_close(&ch); return rc; }
    run->gr_psi = psi;
    run->ts_rounds = 0;
    int64_t omega = run->omega;
    for (;;) {                       /* outer: burn-in check */
        for (;;) {                   /* inner: sample-size check */
            int64_t n = ch.L - psi;
            if (n < 2) {
                if (psi + 2 > run->max_length) { rc = ORC_ERR_NOT_CONVERGED; goto done; }
                rc = chains_extend_to(&ch, psi + 2);
                if (rc) goto done;
                continue;
            }
            int64_t n4[4];
            orc_transition_counts(ch.x, omega, ch.cap, psi, n, n4);
            run->ts_rounds++;
            memcpy(run->n4, n4, sizeof(n4));
            if (n4[1] == 0 || n4[2] == 0 || (n4[0] + n4[1]) == 0 || (n4[2] + n4[3]) == 0) {
                if (ch.L + n > run->max_length) { rc = ORC_ERR_NOT_CONVERGED; goto done; }
                rc = chains_extend_to(&ch, ch.L + n);
                if (rc) goto done;
                continue;
            }
            double a = (double)n4[1] / (double)(n4[0] + n4[1]);
            double b = (double)n4[2] / (double)(n4[2] + n4[3]);
            int64_t M, N;
            rc = orc_two_state_MN(a, b, run->eps, run->r, run->s, &M, &N);
            if (rc) goto done;
            run->alpha = a; run->beta = b; run->M = M; run->N = N;
            int64_t deficit = N - omega * n;
            if (deficit <= 0) break;
            int64_t extend_by = (deficit + omega - 1) / omega;
            if (ch.L + extend_by > run->max_length) { rc = ORC_ERR_NOT_CONVERGED; goto done; }
            rc = chains_extend_to(&ch, ch.L + extend_by);
            if (rc) goto done;
        }
        if (run->M > psi) { psi = run->M; continue; }
        break;
    }
    {
        int64_t n = ch.L - psi, ones = 0;
        for (int64_t c = 0; c < omega; c++)
            for (int64_t j = 0; j < n; j++) ones += ch.x[c * ch.cap + psi + j];
        run->ones = ones;
        run->psi = psi;
        run->length = ch.L;
        run->sample_size = omega * n;
        run->prob = (double)ones / (double)(omega * n);
    }
done:
    run->status = rc;
    chains_close(&ch);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Sequential two-state Markov chain approach (Sec. 3.1, Alg. 1).               */
/* ------------------------------------------------------------------------- */

typedef struct {
    /* inputs */
    int64_t m0, n0;          /* initial burn-in and sample size */
    int64_t max_length;
    int32_t mode;
    uint64_t seed;
    int64_t chain;           /* which chain of the seed's family is simulated */
    double eps, r, s;
    /* outputs */
    double prob, alpha, beta;
    int64_t M, N, length, ones;
    int64_t n4[4];           /* transitions of the last alpha, beta window */
    int64_t ab_window;       /* its length (the N of the round before the last) */
    int32_t rounds;
    int32_t status;
} orc_two_state_seq_run;

/*
 * Alg. 1 on one chain: start from length l = m0 + n0; in each round extend
 * the trajectory to M + N (no-op in the first round), l := M + N, estimate
 * alpha and beta from transitions within the last N positions, recompute M
 * and N by Alg. 1 line 8; stop when M + N <= l; the estimate is the fraction
 * of ones in the last N positions.  Read where the text is silent: a window
 * without a 0->1 or a 1->0 transition (or shorter than 2) cannot give alpha
 * and beta, so N doubles and the round repeats; alpha = beta = 1 (a periodic
 * two-state chain) is not converged.
 */
int orc_estimate_two_state_seq(const orc_net *net, const int32_t *soi_nodes, const uint8_t *soi_values,
                               int32_t soi_size, orc_two_state_seq_run *run) {
    if (run->m0 < 0 || run->n0 < 2) return ORC_ERR_INVALID;
    chains_t ch;
    int rc = chains_open(&ch, net, run->mode, run->seed, 1, soi_nodes, soi_values, soi_size);
    if (rc) return rc;
    /* chain `chain` of the seed's family: its own initial state and draws */
    orc_init_states_from(net, run->seed, run->chain, 1, ch.states);
    ch.chain0 = run->chain;
    int64_t M = run->m0, N = run->n0, l = M + N;
    run->rounds = 0;
    if (l > run->max_length) { rc = ORC_ERR_NOT_CONVERGED; goto done; }
    if ((rc = chains_extend_to(&ch, l))) goto done;
    for (;;) {
        if (M + N > l) {
            if (M + N > run->max_length) { rc = ORC_ERR_NOT_CONVERGED; goto done; }
            if ((rc = chains_extend_to(&ch, M + N))) goto done;
            l = M + N;
        }
        run->rounds++;
        int64_t c[4];
        const int64_t start = l - N;
        orc_transition_counts(ch.x, 1, ch.cap, start, N, c);
        memcpy(run->n4, c, sizeof(c));
        run->ab_window = N;
        if (N < 2 || c[1] == 0 || c[2] == 0 || (c[0] + c[1]) == 0 || (c[2] + c[3]) == 0) {
            N = 2 * (N < 2 ? 2 : N);
            continue;
        }
        double a = (double)c[1] / (double)(c[0] + c[1]);
        double b = (double)c[2] / (double)(c[2] + c[3]);
        int64_t M1, N1;
        if ((rc = orc_two_state_MN(a, b, run->eps, run->r, run->s, &M1, &N1))) goto done;
        run->alpha = a; run->beta = b;
        M = M1; N = N1;
        if (M + N <= l) break;
    }
    {
        int64_t ones = 0;
        for (int64_t j = l - N; j < l; j++) ones += ch.x[j];
        run->ones = ones;
        run->prob = (double)ones / (double)N;
        run->M = M; run->N = N; run->length = l;
    }
done:
    run->status = rc;
    chains_close(&ch);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Several properties from the same trajectories (Sec. 4.2, last part).        */
/* ------------------------------------------------------------------------- */

#define ORC_MAX_PROPERTIES 8

typedef struct {
    double prob, alpha, beta, rhat;
    int64_t M, N, ones;
    int64_t n4[4];
} orc_property;

/*
 * q properties (sets of states of interest) share one set of chains; every
 * property abstracts the same trajectories into its own meta-state sequence.
 * Here the sharing is literal: q chain sets opened with the same seed follow
 * the same trajectories (counter-based randomness) and differ only in the
 * property they record.  Read as follows where the text is silent:
 *  - Alg. GR holds for every property: psi doubles until each property's
 *    R-hat is below the threshold (run->rhat: the largest);
 *  - in each round alpha, beta, M, N are computed per property; the chains
 *    are extended by the smallest deficit among the properties whose N is
 *    larger than the merged sample (the text: the next extension follows the
 *    smallest N), until no N is larger than the sample;
 *  - the burn-in check takes the largest M: if it exceeds psi, psi := that M
 *    and the rounds repeat for every property;
 *  - each property's estimate is its fraction of ones in the common final
 *    window.
 * With q = 1 every step is Alg. 3's.  run's per-property fields (prob, alpha,
 * beta, M, N, n4, ones) repeat property 0.
 */
int orc_estimate_two_state_multi(const orc_net *net, int32_t q, const int32_t *soi_nodes,
                                 const uint8_t *soi_values, const int32_t *soi_sizes, orc_two_state_run *run,
                                 orc_property *props) {
    if (q < 1 || q > ORC_MAX_PROPERTIES) return ORC_ERR_INVALID;
    chains_t ch[ORC_MAX_PROPERTIES];
    int rc = ORC_OK, opened = 0;
    int64_t off = 0;
    for (int m = 0; m < q; m++) {
        rc = chains_open(&ch[m], net, run->mode, run->seed, run->omega, soi_nodes + off, soi_values + off,
                         soi_sizes[m]);
        if (rc) goto done;
        opened++;
        off += soi_sizes[m];
    }
    int64_t omega = run->omega;
    /* Alg. GR over every property */
    int64_t psi = run->psi0;
    run->gr_rounds = 0;
    for (;;) {
        if (2 * psi > run->max_length) { rc = ORC_ERR_NOT_CONVERGED; goto done; }
        for (int m = 0; m < q; m++)
            if ((rc = chains_extend_to(&ch[m], 2 * psi))) goto done;
        run->gr_rounds++;
        int all = 1;
        double worst = -INFINITY;
        for (int m = 0; m < q; m++) {
            double R = orc_gelman_rubin(ch[m].x, omega, ch[m].cap, psi, psi);
            props[m].rhat = R;
            if (!(R < run->rhat_threshold)) all = 0;
            if (!(R <= worst)) worst = R;   /* NaN or larger */
        }
        run->rhat = worst;
        if (all) break;
        psi *= 2;
    }
    run->gr_psi = psi;
    run->ts_rounds = 0;
    for (;;) {                        /* burn-in check */
        for (;;) {                    /* sample-size check */
            int64_t L = ch[0].L, n = L - psi;
            if (n < 2) {
                if (psi + 2 > run->max_length) { rc = ORC_ERR_NOT_CONVERGED; goto done; }
                for (int m = 0; m < q; m++)
                    if ((rc = chains_extend_to(&ch[m], psi + 2))) goto done;
                continue;
            }
            run->ts_rounds++;
            int insufficient = 0;
            for (int m = 0; m < q; m++) {
                int64_t *c = props[m].n4;
                orc_transition_counts(ch[m].x, omega, ch[m].cap, psi, n, c);
                if (c[1] == 0 || c[2] == 0 || (c[0] + c[1]) == 0 || (c[2] + c[3]) == 0) insufficient = 1;
            }
            if (insufficient) {
                if (L + n > run->max_length) { rc = ORC_ERR_NOT_CONVERGED; goto done; }
                for (int m = 0; m < q; m++)
                    if ((rc = chains_extend_to(&ch[m], L + n))) goto done;
                continue;
            }
            int64_t smallest = -1;
            for (int m = 0; m < q; m++) {
                const int64_t *c = props[m].n4;
                double a = (double)c[1] / (double)(c[0] + c[1]);
                double b = (double)c[2] / (double)(c[2] + c[3]);
                int64_t M, N;
                if ((rc = orc_two_state_MN(a, b, run->eps, run->r, run->s, &M, &N))) goto done;
                props[m].alpha = a; props[m].beta = b; props[m].M = M; props[m].N = N;
                int64_t deficit = N - omega * n;
                if (deficit > 0 && (smallest < 0 || deficit < smallest)) smallest = deficit;
            }
            if (smallest < 0) break;
            int64_t extend_by = (smallest + omega - 1) / omega;
            if (L + extend_by > run->max_length) { rc = ORC_ERR_NOT_CONVERGED; goto done; }
            for (int m = 0; m < q; m++)
                if ((rc = chains_extend_to(&ch[m], L + extend_by))) goto done;
        }
        int64_t Mmax = props[0].M;
        for (int m = 1; m < q; m++)
            if (props[m].M > Mmax) Mmax = props[m].M;
        if (Mmax > psi) { psi = Mmax; continue; }
        break;
    }
    {
        int64_t L = ch[0].L, n = L - psi;
        for (int m = 0; m < q; m++) {
            int64_t ones = 0;
            for (int64_t c = 0; c < omega; c++)
                for (int64_t j = 0; j < n; j++) ones += ch[m].x[c * ch[m].cap + psi + j];
            props[m].ones = ones;
            props[m].prob = (double)ones / (double)(omega * n);
        }
        run->psi = psi;
        run->length = L;
        run->sample_size = omega * n;
        run->prob = props[0].prob; run->alpha = props[0].alpha; run->beta = props[0].beta;
        run->M = props[0].M; run->N = props[0].N; run->ones = props[0].ones;
        memcpy(run->n4, props[0].n4, sizeof(run->n4));
    }
done:
    run->status = rc;
    for (int m = 0; m < opened; m++) chains_close(&ch[m]);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Skart pieces (Sec. 3.2, Alg. 2; parallel Alg. 4).                           */
/* ------------------------------------------------------------------------- */

/* Sample skewness m3 / m2^(3/2) with population moments (0 when m2 = 0). */
double orc_skewness(const double *v, int64_t K) {
    double m = 0.0;
    for (int64_t j = 0; j < K; j++) m += v[j];
    m /= (double)K;
    double m2 = 0.0, m3 = 0.0;
    for (int64_t j = 0; j < K; j++) { double d = v[j] - m; m2 += d * d; m3 += d * d * d; }
    m2 /= (double)K; m3 /= (double)K;
    if (!(m2 > 0.0)) return 0.0;
    return m3 / pow(m2, 1.5);
}

/* The continued fraction of the regularised incomplete beta function
 * (DLMF 8.17.22):
 *   I_x(a,b) = x^a (1-x)^b / (a B(a,b)) * 1/(1 + d_1/(1 + d_2/(1 + ...))),
 *   d_{2m}   =  m (b - m) x / ((a + 2m - 1)(a + 2m)),
 *   d_{2m+1} = -(a + m)(a + b + m) x / ((a + 2m)(a + 2m + 1)).
 * cf_term(j) is d_j. */
static double cf_term(double a, double b, double x, long j) {
    double m = (double)(j / 2);
    if (j % 2 == 0) return m * (b - m) * x / ((a + 2.0 * m - 1.0) * (a + 2.0 * m));
    return -(a + m) * (a + b + m) * x / ((a + 2.0 * m) * (a + 2.0 * m + 1.0));
}

/* Value of 1/(1 + d_1/(1 + d_2/(1 + ...))) as the limit of its convergents
 * A_j / B_j, which obey the fundamental (Wallis) recurrences
 * A_j = A_{j-1} + d_{j-1} A_{j-2}, B_j = B_{j-1} + d_{j-1} B_{j-2} from
 * A_0 = 0, A_1 = 1, B_0 = 1, B_1 = 1.  Each step divides the last two pairs
 * by the new B_j, so B_j stays 1 and A_j is the convergent itself. */
static double cf_value(double a, double b, double x) {
    double A_older = 0.0, A_old = 1.0, B_older = 1.0;
    double value = 1.0;
    for (long j = 2; j < 400000; j++) {
        double d = cf_term(a, b, x, j - 1);
        double A = A_old + d * A_older;
        double B = 1.0 + d * B_older;          /* B_{j-1} is 1 after rescaling */
        if (B == 0.0) B = 1e-300;
        A_older = A_old / B;
        B_older = 1.0 / B;
        A_old = A / B;
        double change = fabs(A_old - value);
        value = A_old;
        if (change <= 1e-16 * fabs(value)) break;
    }
    return value;
}

/* log Gamma(a+b) - log Gamma(a) without cancellation for large a: the
 * Stirling series ln Gamma(z) = (z-1/2) ln z - z + ln(2 pi)/2 + 1/(12z)
 * - 1/(360z^3) + 1/(1260z^5) - 1/(1680z^7) + ... differenced term by term. */
static double stirling_tail(double z) {
    double z2 = z * z;
    return 1.0 / (12.0 * z) - 1.0 / (360.0 * z * z2) + 1.0 / (1260.0 * z * z2 * z2)
           - 1.0 / (1680.0 * z * z2 * z2 * z2);
}

static double lgamma_ratio(double a, double b) {
    if (a < 20.0) return lgamma(a + b) - lgamma(a);
    return (a - 0.5) * log1p(b / a) + b * log(a + b) - b + (stirling_tail(a + b) - stirling_tail(a));
}

/* ln B(p,q) = ln Gamma(s) - [ln Gamma(g+s) - ln Gamma(g)], g the larger and s
 * the smaller argument, so that the difference of two large ln Gamma values is
 * formed by lgamma_ratio without cancellation. */
static double log_beta(double p, double q) {
    double g = p > q ? p : q, sm = p > q ? q : p;
    return lgamma(sm) - lgamma_ratio(g, sm);
}

/* Regularised incomplete beta I_x(a,b), y = 1 - x given exactly.  The
 * fraction converges fast for x < (a+1)/(a+b+2) (DLMF 8.17(v)); otherwise the
 * reflection I_x(a,b) = 1 - I_y(b,a) (DLMF 8.17.4) moves x below that point. */
static double inc_beta(double a, double b, double x, double y) {
    if (x <= 0.0) return 0.0;
    if (y <= 0.0) return 1.0;
    int reflect = !(x < (a + 1.0) / (a + b + 2.0));
    double p = reflect ? b : a, q = reflect ? a : b;
    double u = reflect ? y : x, w = reflect ? x : y;      /* w = 1 - u */
    /* ln(u^p w^q / (p B(p,q))); the log of whichever of u, w is near 1 is
     * taken as log1p of minus the other, which is exact to rounding */
    double ln_u = u > 0.5 ? log1p(-w) : log(u);
    double ln_w = w > 0.5 ? log1p(-u) : log(w);
    double ln_front = p * ln_u + q * ln_w - log(p) - log_beta(p, q);
    double I = exp(ln_front) * cf_value(p, q, u);
    return reflect ? 1.0 - I : I;
}

/* Student t CDF with dof degrees of freedom:
 * P(T <= t) = 1 - I_x(dof/2, 1/2)/2 for t > 0, x = dof/(dof+t^2). */
static double t_cdf(double t, double dof) {
    double x = dof / (dof + t * t);
    double y = (t * t) / (dof + t * t);
    double tail = 0.5 * inc_beta(0.5 * dof, 0.5, x, y);
    return t > 0.0 ? 1.0 - tail : tail;
}

/* Student t quantile by bisection on the CDF (to a relative 1e-15). */
double orc_t_ppf(double q, double dof) {
    if (!(q > 0.0 && q < 1.0) || !(dof > 0.0)) return NAN;
    if (q == 0.5) return 0.0;
    double lo = -1.0, hi = 1.0;
    while (t_cdf(lo, dof) > q) lo *= 2.0;
    while (t_cdf(hi, dof) < q) hi *= 2.0;
    for (int it = 0; it < 400; it++) {
        double mid = 0.5 * (lo + hi);
        if (t_cdf(mid, dof) < q) lo = mid; else hi = mid;
        if (hi - lo <= 1e-15 * fabs(mid)) break;
    }
    return 0.5 * (lo + hi);
}

/* Batch means of the parallel layout (Fig. 2b): chain c contributes bpc
 * consecutive batches of kappa values starting at position `start`.
 * means[c*bpc + j] = mean of chain c's positions start + j*kappa .. +kappa-1. */
static void batch_means(const chains_t *ch, int64_t start, int64_t kappa, int64_t bpc, double *means) {
    for (int64_t c = 0; c < ch->omega; c++)
        for (int64_t j = 0; j < bpc; j++) {
            const uint8_t *xc = ch->x + c * ch->cap + start + j * kappa;
            int64_t s = 0;
            for (int64_t q = 0; q < kappa; q++) s += xc[q];
            means[c * bpc + j] = (double)s / (double)kappa;
        }
}

/* von Neumann randomness test on the spaced batch means: of every chain's
 * bpc batches keep those preceded by d skipped batches (j = d, 2d+1, ...).
 * C = 1 - (K-1)/P * sum_pairs (x_{j+1}-x_j)^2 / (2 sum (x - mean)^2) over the
 * P within-chain adjacent pairs of retained means (K of them).  Passes if
 * P = 0, if all means are equal, or if C <= z_{1-alpha_ran} sqrt((m-2)/(m^2-1))
 * with m = P + 1. */
int orc_vonneumann_pass(const double *means, int64_t omega, int64_t bpc, int64_t d, double alpha_ran,
                        double *stat_out) {
    int64_t per = bpc / (d + 1);
    int64_t K = per * omega;
    int64_t P = (per > 1) ? (per - 1) * omega : 0;
    *stat_out = 0.0;
    if (P == 0 || K < 3) return 1;
    double m = 0.0;
    for (int64_t c = 0; c < omega; c++)
        for (int64_t q = 0; q < per; q++) m += means[c * bpc + q * (d + 1) + d];
    m /= (double)K;
    double ss = 0.0, sd = 0.0;
    for (int64_t c = 0; c < omega; c++)
        for (int64_t q = 0; q < per; q++) {
            double v = means[c * bpc + q * (d + 1) + d];
            ss += (v - m) * (v - m);
            if (q + 1 < per) {
                double w = means[c * bpc + (q + 1) * (d + 1) + d];
                sd += (w - v) * (w - v);
            }
        }
    if (!(ss > 0.0)) return 1;
    double C = 1.0 - ((double)(K - 1) / (double)P) * sd / (2.0 * ss);
    *stat_out = C;
    double mm = (double)(P + 1);
    double crit = orc_norm_ppf(1.0 - alpha_ran) * sqrt((mm - 2.0) / (mm * mm - 1.0));
    return C <= crit;
}

typedef struct {
    double mean, var, skew, phi, A, H, ci_lo, ci_hi;
} orc_skart_ci;

/* Skewness- and autoregression-adjusted CI of the nonspaced batch means
 * (Alg. 2 / Alg. 4 "Compute skewness and autoregression adjusted CI"):
 * X = grand mean, S^2 = sample variance, phi = pooled within-chain lag-1
 * autocorrelation, A = (1+phi)/(1-phi), beta = skew/(6 sqrt K),
 * G(z) = ((1 + 6 beta (z - beta))^(1/3) - 1)/(2 beta),
 * CI = [X - G(t_{1-a/2}) sqrt(A S^2/K), X - G(t_{a/2}) sqrt(A S^2/K)]. */
void orc_skart_ci_from_means(const double *means, int64_t omega, int64_t bpc, double alpha, orc_skart_ci *o) {
    int64_t K = omega * bpc;
    double m = 0.0;
    for (int64_t j = 0; j < K; j++) m += means[j];
    m /= (double)K;
    double ss = 0.0, sp = 0.0;
    int64_t P = 0;
    for (int64_t c = 0; c < omega; c++)
        for (int64_t q = 0; q < bpc; q++) {
            double v = means[c * bpc + q] - m;
            ss += v * v;
            if (q + 1 < bpc) { sp += v * (means[c * bpc + q + 1] - m); P++; }
        }
    o->mean = m;
    o->var = ss / (double)(K - 1);
    o->skew = orc_skewness(means, K);
    double phi = 0.0;
    if (P > 0 && ss > 0.0) phi = (sp / (double)P) / (ss / (double)K);
    if (phi > 0.999) phi = 0.999;
    if (phi < -0.999) phi = -0.999;
    o->phi = phi;
    o->A = (1.0 + phi) / (1.0 - phi);
    double beta = o->skew / (6.0 * sqrt((double)K));
    double tu = orc_t_ppf(1.0 - alpha / 2.0, (double)(K - 1));
    double tl = orc_t_ppf(alpha / 2.0, (double)(K - 1));
    /* G(z) = ((1 + 6 beta (z - beta))^(1/3) - 1) / (2 beta), written with
     * a^3 - 1 = (a - 1)(a^2 + a + 1) as 3 (z - beta) / (a^2 + a + 1) so that
     * it stays exact as beta -> 0 (where G(z) = z). */
    double au = cbrt(1.0 + 6.0 * beta * (tu - beta));
    double al = cbrt(1.0 + 6.0 * beta * (tl - beta));
    double Gu = 3.0 * (tu - beta) / (au * au + au + 1.0);
    double Gl = 3.0 * (tl - beta) / (al * al + al + 1.0);
    double se = sqrt(o->A * o->var / (double)K);
    o->ci_lo = m - Gu * se;
    o->ci_hi = m - Gl * se;
    double h1 = m - o->ci_lo, h2 = o->ci_hi - m;
    o->H = h1 > h2 ? h1 : h2;
}

typedef struct {
    /* inputs */
    int64_t omega;
    int64_t psi0;
    double rhat_threshold;
    int64_t max_length;
    int32_t mode;
    uint64_t seed;
    double H_star;           /* precision requirement */
    int32_t relative;        /* 1: H* = H_star * |mean| */
    double alpha;            /* CI confidence 1 - alpha */
    /* outputs */
    double mean, ci_lo, ci_hi, H, var, skew, phi;
    double rhat;
    int64_t psi, length, kappa, batches, spacer;
    int64_t sample_size;     /* batches * kappa */
    int32_t gr_rounds, rand_rounds, ci_rounds;
    int32_t status;
} orc_skart_run;

static int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

/*
 * Alg. 4 (Sec. 4.3).  Constants that the paper leaves to its Skart reference
 * (skewness threshold 4 giving batch size 16, randomness-test size 0.20,
 * largest spacer 10, batch-size factor sqrt 2 with a 10% batch-count cut when
 * the largest spacer fails, at most max(1024, current) batches when the CI is
 * too wide) are placeholders of this implementation, not verified against that
 * reference: parity between the two implementations holds, agreement with the
 * reference's Skart does not.
 */
int orc_estimate_skart(const orc_net *net, const int32_t *soi_nodes, const uint8_t *soi_values,
                       int32_t soi_size, orc_skart_run *run) {
    chains_t ch;
    int rc = chains_open(&ch, net, run->mode, run->seed, run->omega, soi_nodes, soi_values, soi_size);
    if (rc) return rc;
    int64_t psi;
    rc = run_gelman_rubin(&ch, run->psi0, run->rhat_threshold, run->max_length, &psi, &run->rhat, &run->gr_rounds);
    if (rc) { run->status = rc; chains_close(&ch); return rc; }
    int64_t omega = run->omega;
    const int64_t start = psi;                      /* skip the first psi samples */
    int64_t eta = ceil_div(1280, omega) * omega;
    double *buf = NULL;
    rc = chains_extend_to(&ch, start + eta / omega);
    if (rc) goto done;
    /* skewness of all eta samples */
    {
        int64_t per = eta / omega, K = eta;
        buf = (double *)malloc(sizeof(double) * (size_t)K);
        for (int64_t c = 0; c < omega; c++)
            for (int64_t j = 0; j < per; j++) buf[c * per + j] = ch.x[c * ch.cap + start + j];
        double B = orc_skewness(buf, K);
        free(buf); buf = NULL;
        run->kappa = fabs(B) > 4.0 ? 16 : 1;
    }
    int64_t kappa = run->kappa;
    int64_t p = ceil_div(eta, omega) * omega;
    eta = kappa * p;
    int64_t d = 0;
    const double alpha_ran = 0.20;
    run->rand_rounds = 0;
    for (;;) {
        if (start + eta / omega > run->max_length) { rc = ORC_ERR_NOT_CONVERGED; goto done; }
        rc = chains_extend_to(&ch, start + eta / omega);
        if (rc) goto done;
        int64_t bpc = p / omega;
        buf = (double *)malloc(sizeof(double) * (size_t)p);
        batch_means(&ch, start, kappa, bpc, buf);
        double C;
        int pass = orc_vonneumann_pass(buf, omega, bpc, d, alpha_ran, &C);
        free(buf); buf = NULL;
        run->rand_rounds++;
        if (pass) break;
        d += 1;
        if (d > 10) {
            d = 0;
            kappa = (int64_t)ceil(sqrt(2.0) * (double)kappa);
            p = (int64_t)ceil(0.9 * (double)p);
        }
        p = ceil_div(p, omega) * omega;
        eta = kappa * p;
    }
    run->spacer = d;
    run->ci_rounds = 0;
    for (;;) {
        if (start + eta / omega > run->max_length) { rc = ORC_ERR_NOT_CONVERGED; goto done; }
        rc = chains_extend_to(&ch, start + eta / omega);
        if (rc) goto done;
        int64_t bpc = p / omega;
        buf = (double *)malloc(sizeof(double) * (size_t)p);
        batch_means(&ch, start, kappa, bpc, buf);
        orc_skart_ci ci;
        orc_skart_ci_from_means(buf, omega, bpc, run->alpha, &ci);
        free(buf); buf = NULL;
        run->ci_rounds++;
        run->mean = ci.mean; run->ci_lo = ci.ci_lo; run->ci_hi = ci.ci_hi; run->H = ci.H;
        run->var = ci.var; run->skew = ci.skew; run->phi = ci.phi;
        double Hs = run->relative ? run->H_star * fabs(ci.mean) : run->H_star;
        if (!(ci.H > Hs)) break;
        double f = (ci.H / Hs) * (ci.H / Hs);
        int64_t pmax = p > 1024 ? p : 1024;
        double pf = ceil(f * (double)p);
        int64_t p1 = pf > (double)pmax ? pmax : (int64_t)pf;
        int64_t k1 = (int64_t)ceil((double)kappa * f * (double)p / (double)p1);
        if (k1 < kappa) k1 = kappa;
        kappa = k1;
        p = ceil_div(p1, omega) * omega;
        eta = kappa * p;
    }
    run->psi = psi;
    run->length = ch.L;
    run->kappa = kappa;
    run->batches = p;
    run->sample_size = kappa * p;
done:
    free(buf);
    run->status = rc;
    chains_close(&ch);
    return rc;
}

/*
 * Alg. 2 (Sec. 3.2), the sequential Skart method on chain 0 of the seed's
 * family, with the constants of this oracle's Alg. 4 (placeholders for the
 * Skart reference, see orc_estimate_skart):
 *  - eta = 1280 samples; skewness of the last 1024 gives the batch size
 *    (16 when |skewness| > 4, else 1); p := eta batches, eta := kappa p;
 *  - the randomness test runs on the batch means of the whole trajectory
 *    with spacer d, adjusting (d, kappa, p) as Alg. 4 does until it passes;
 *  - then zeta = d kappa samples are skipped and the CI uses the p' = p - d
 *    nonspaced batches after them; when H > H* the batch size and count are
 *    adjusted as in Alg. 4 and eta := kappa (p' + d), the skipped part being
 *    d batches of the current size.
 * run->psi reports the skipped zeta; run->batches the final p'.
 */
int orc_estimate_skart_seq(const orc_net *net, const int32_t *soi_nodes, const uint8_t *soi_values,
                           int32_t soi_size, orc_skart_run *run) {
    chains_t ch;
    int rc = chains_open(&ch, net, run->mode, run->seed, 1, soi_nodes, soi_values, soi_size);
    if (rc) return rc;
    double *buf = NULL;
    run->gr_rounds = 0;
    run->rhat = 0.0;
    int64_t eta = 1280;
    const int64_t l = 1024;
    if (eta > run->max_length) { rc = ORC_ERR_NOT_CONVERGED; goto done; }
    if ((rc = chains_extend_to(&ch, eta))) goto done;
    {
        buf = (double *)malloc(sizeof(double) * (size_t)l);
        if (!buf) { rc = ORC_ERR_OOM; goto done; }
        for (int64_t j = 0; j < l; j++) buf[j] = ch.x[eta - l + j];
        double B = orc_skewness(buf, l);
        free(buf); buf = NULL;
        run->kappa = fabs(B) > 4.0 ? 16 : 1;
    }
    int64_t kappa = run->kappa;
    int64_t p = eta;
    eta = kappa * p;
    int64_t d = 0;
    const double alpha_ran = 0.20;
    run->rand_rounds = 0;
    for (;;) {
        if (eta > run->max_length) { rc = ORC_ERR_NOT_CONVERGED; goto done; }
        if ((rc = chains_extend_to(&ch, eta))) goto done;
        buf = (double *)malloc(sizeof(double) * (size_t)p);
        if (!buf) { rc = ORC_ERR_OOM; goto done; }
        batch_means(&ch, 0, kappa, p, buf);
        double C;
        int pass = orc_vonneumann_pass(buf, 1, p, d, alpha_ran, &C);
        free(buf); buf = NULL;
        run->rand_rounds++;
        if (pass) break;
        d += 1;
        if (d > 10) {
            d = 0;
            kappa = (int64_t)ceil(sqrt(2.0) * (double)kappa);
            p = (int64_t)ceil(0.9 * (double)p);
        }
        eta = kappa * p;
    }
    run->spacer = d;
    int64_t pp = p - d;           /* batches after the skipped d */
    if (pp < 2) { rc = ORC_ERR_NOT_CONVERGED; goto done; }
    run->ci_rounds = 0;
    for (;;) {
        eta = kappa * (pp + d);
        if (eta > run->max_length) { rc = ORC_ERR_NOT_CONVERGED; goto done; }
        if ((rc = chains_extend_to(&ch, eta))) goto done;
        buf = (double *)malloc(sizeof(double) * (size_t)pp);
        if (!buf) { rc = ORC_ERR_OOM; goto done; }
        batch_means(&ch, d * kappa, kappa, pp, buf);
        orc_skart_ci ci;
        orc_skart_ci_from_means(buf, 1, pp, run->alpha, &ci);
        free(buf); buf = NULL;
        run->ci_rounds++;
        run->mean = ci.mean; run->ci_lo = ci.ci_lo; run->ci_hi = ci.ci_hi; run->H = ci.H;
        run->var = ci.var; run->skew = ci.skew; run->phi = ci.phi;
        double Hs = run->relative ? run->H_star * fabs(ci.mean) : run->H_star;
        if (!(ci.H > Hs)) break;
        double f = (ci.H / Hs) * (ci.H / Hs);
        int64_t pmax = pp > 1024 ? pp : 1024;
        double pf = ceil(f * (double)pp);
        int64_t p1 = pf > (double)pmax ? pmax : (int64_t)pf;
        int64_t k1 = (int64_t)ceil((double)kappa * f * (double)pp / (double)p1);
        if (k1 < kappa) k1 = kappa;
        kappa = k1;
        pp = p1;
    }
    run->psi = d * kappa;
    run->length = ch.L;
    run->kappa = kappa;
    run->batches = pp;
    run->sample_size = kappa * pp;
done:
    free(buf);
    run->status = rc;
    chains_close(&ch);
    return rc;
}
