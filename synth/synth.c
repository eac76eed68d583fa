/*
 * synth.c -- seeded synthetic matching-LP instances.
 *
 * This module only draws random numbers and lays them out; it holds none of
 * the solver's arithmetic.  Both the CUDA solver (through the Python wrapper
 * and the benchmark) and the FP64 oracle (through the tests) are fed from it.
 *
 * Randomness is counter-based: every value is a pure function of
 * (seed, user id, purpose, draw index), produced by Philox4x32-10 as defined
 * by Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy as
 * 1, 2, 3" (SC'11).  So any user's row can be regenerated on its own (used for
 * sampled checks of large instances) and results do not depend on the number
 * of threads.
 *
 * Instance shapes follow the matching workloads of the paper (Sec. 3.3 and
 * App. A): users i with a set of eligible items j, per-edge cost c_ij and
 * capacity coefficient a_ij, and item capacities b_j.  The storage is
 * user-major CSR: row_ptr (int64, I+1), col (int32, nnz), c and a (float32).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x32-10                                                             */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

static inline void philox_round(uint32_t c[4], uint32_t k0, uint32_t k1) {
  uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c[0];
  uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c[2];
  uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  uint32_t n0 = hi1 ^ c[1] ^ k0;
  uint32_t n2 = hi0 ^ c[3] ^ k1;
  c[0] = n0;
  c[1] = lo1;
  c[2] = n2;
  c[3] = lo0;
}

static inline void philox10(const uint32_t ctr[4], uint32_t k0, uint32_t k1, uint32_t out[4]) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    philox_round(c, k0, k1);
  }
  out[0] = c[0];
  out[1] = c[1];
  out[2] = c[2];
  out[3] = c[3];
}

/* Exported for known-answer tests of the generator itself. */
void synth_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  philox10(ctr, key[0], key[1], out);
}

/* One random stream: key = seed, counter = (id lo, id hi, purpose, block). */
typedef struct {
  uint32_t k0, k1;
  uint32_t ctr[4];
  uint32_t buf[4];
  int pos;
} rng_t;

static void rng_init(rng_t* r, uint64_t seed, uint64_t id, uint32_t purpose) {
  r->k0 = (uint32_t)seed;
  r->k1 = (uint32_t)(seed >> 32);
  r->ctr[0] = (uint32_t)id;
  r->ctr[1] = (uint32_t)(id >> 32);
  r->ctr[2] = purpose;
  r->ctr[3] = 0;
  r->pos = 4;
}

static inline uint32_t rng_u32(rng_t* r) {
  if (r->pos == 4) {
    philox10(r->ctr, r->k0, r->k1, r->buf);
    r->ctr[3]++;
    r->pos = 0;
  }
  return r->buf[r->pos++];
}

/* Uniform on [0, 1) with 53 random bits. */
static inline double rng_uniform(rng_t* r) {
  uint32_t a = rng_u32(r) >> 5, b = rng_u32(r) >> 6;
  return ((double)a * 67108864.0 + (double)b) * (1.0 / 9007199254740992.0);
}

/* Standard normal by the Box-Muller transform (one output per call). */
static inline double rng_normal(rng_t* r) {
  double u1 = 1.0 - rng_uniform(r); /* (0, 1] */
  double u2 = rng_uniform(r);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

/* Poisson(mu) by sequential inversion of the CDF (mu is small here). */
static int rng_poisson(rng_t* r, double mu) {
  double u = rng_uniform(r);
  double p = exp(-mu), F = p;
  int k = 0;
  while (u > F && k < 100000) {
    ++k;
    p *= mu / (double)k;
    F += p;
  }
  return k;
}

/* ------------------------------------------------------------------------ */
/* Parameters                                                                */
/* ------------------------------------------------------------------------ */
enum { DEG_POISSON = 0, DEG_LOGNORMAL = 1 };
enum { ITEMS_UNIFORM = 0, ITEMS_ZIPF = 1 };
enum { C_NEG_UNIFORM = 0, C_NEG_LOGNORMAL = 1 };
enum { A_ONE = 0, A_UNIFORM = 1 };
enum { B_ITEM_DEGREE = 0, B_SUM_A = 1 };

typedef struct {
  int64_t I;        /* users */
  int32_t J;        /* items */
  int32_t _pad0;
  uint64_t seed;
  int32_t deg_model; /* DEG_POISSON: 1 + Poisson(deg_mean - 1); DEG_LOGNORMAL: truncated lognormal */
  int32_t deg_max;   /* lognormal: resample above this */
  double deg_mean;   /* mean degree */
  double deg_sigma;  /* lognormal sigma */
  int32_t item_model;
  int32_t c_model;
  double zipf_s;     /* popularity of item with rank r (= id + 1) is r^-zipf_s */
  double c_mu, c_sigma;
  int32_t a_model;
  int32_t b_model;
  double a_lo, a_hi;
  double b_frac;
} synth_params;

enum { PURPOSE_DEGREE = 1, PURPOSE_ITEMS = 2, PURPOSE_VALUES = 3, PURPOSE_NOISE = 4, PURPOSE_CHURN = 5 };

static int32_t draw_degree(const synth_params* p, uint64_t uid) {
  rng_t r;
  rng_init(&r, p->seed, uid, PURPOSE_DEGREE);
  int64_t d;
  if (p->deg_model == DEG_POISSON) {
    d = 1 + rng_poisson(&r, p->deg_mean - 1.0);
  } else {
    double s = p->deg_sigma;
    double mu = log(p->deg_mean) - 0.5 * s * s;
    d = -1;
    for (int tries = 0; tries < 1000; ++tries) {
      double v = exp(mu + s * rng_normal(&r));
      if (v > (double)p->deg_max + 0.5) continue;
      d = (int64_t)llround(v);
      break;
    }
    if (d < 0) d = p->deg_max;
    if (d < 1) d = 1;
  }
  if (d > p->J) d = p->J;
  return (int32_t)d;
}

/* Per-degree-table used by both item samplers. */
typedef struct {
  double* cdf;  /* Zipf cumulative weights, size J */
  double total; /* cdf[J-1] */
} item_table;

static int cmp_i32(const void* x, const void* y) {
  int32_t a = *(const int32_t*)x, b = *(const int32_t*)y;
  return (a > b) - (a < b);
}

typedef struct {
  uint64_t* bits; /* J-bit set */
  int32_t* idx;   /* J indices */
} scratch_t;

static void scratch_alloc(scratch_t* s, int32_t J) {
  s->bits = (uint64_t*)calloc((size_t)(J + 63) / 64, sizeof(uint64_t));
  s->idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)J);
}
static void scratch_free(scratch_t* s) {
  free(s->bits);
  free(s->idx);
}

/* Comparator for Efraimidis-Spirakis keys: larger key first, ties by index. */
typedef struct {
  double key;
  int32_t j;
} keyed_t;
static int cmp_keyed_desc(const void* x, const void* y) {
  const keyed_t *a = (const keyed_t*)x, *b = (const keyed_t*)y;
  if (a->key > b->key) return -1;
  if (a->key < b->key) return 1;
  return (a->j > b->j) - (a->j < b->j);
}

/* Draw d distinct items for user uid.  Uniform items: rejection (or partial
 * Fisher-Yates when d is a large share of J).  Zipf items: successive
 * weighted draws without replacement, by rejection of repeats (or by the
 * Efraimidis-Spirakis keys u^(1/w) when d is a large share of J); both are
 * exact samplers of the same distribution.  Output sorted ascending. */
static void draw_items(const synth_params* p, const item_table* t, uint64_t uid, int32_t d, int32_t* out,
                       scratch_t* s) {
  const int32_t J = p->J;
  rng_t r;
  rng_init(&r, p->seed, uid, PURPOSE_ITEMS);
  if (d >= J) {
    for (int32_t j = 0; j < J; ++j) out[j] = j;
    return;
  }
  int large = (int64_t)d * 4 > (int64_t)J;
  if (p->item_model == ITEMS_UNIFORM) {
    if (large) {
      for (int32_t j = 0; j < J; ++j) s->idx[j] = j;
      for (int32_t k = 0; k < d; ++k) {
        int32_t m = k + (int32_t)(rng_uniform(&r) * (double)(J - k));
        if (m >= J) m = J - 1;
        int32_t tmp = s->idx[k];
        s->idx[k] = s->idx[m];
        s->idx[m] = tmp;
        out[k] = s->idx[k];
      }
    } else {
      int32_t k = 0;
      while (k < d) {
        int32_t j = (int32_t)(rng_uniform(&r) * (double)J);
        if (j >= J) j = J - 1;
        uint64_t m = 1ull << (j & 63);
        if (s->bits[j >> 6] & m) continue;
        s->bits[j >> 6] |= m;
        out[k++] = j;
      }
      for (int32_t q = 0; q < d; ++q) s->bits[out[q] >> 6] = 0;
    }
  } else {
    if (large) {
      keyed_t* kk = (keyed_t*)malloc(sizeof(keyed_t) * (size_t)J);
      for (int32_t j = 0; j < J; ++j) {
        double w = pow((double)(j + 1), -p->zipf_s);
        double u = 1.0 - rng_uniform(&r);
        kk[j].key = log(u) / w; /* monotone in u^(1/w) */
        kk[j].j = j;
      }
      qsort(kk, (size_t)J, sizeof(keyed_t), cmp_keyed_desc);
      for (int32_t k = 0; k < d; ++k) out[k] = kk[k].j;
      free(kk);
    } else {
      int32_t k = 0;
      while (k < d) {
        double u = rng_uniform(&r) * t->total;
        int32_t lo = 0, hi = J - 1;
        while (lo < hi) {
          int32_t mid = lo + (hi - lo) / 2;
          if (t->cdf[mid] > u)
            hi = mid;
          else
            lo = mid + 1;
        }
        int32_t j = lo;
        uint64_t m = 1ull << (j & 63);
        if (s->bits[j >> 6] & m) continue;
        s->bits[j >> 6] |= m;
        out[k++] = j;
      }
      for (int32_t q = 0; q < d; ++q) s->bits[out[q] >> 6] = 0;
    }
  }
  qsort(out, (size_t)d, sizeof(int32_t), cmp_i32);
}

static void draw_values(const synth_params* p, uint64_t uid, int32_t d, float* c, float* a) {
  rng_t r;
  rng_init(&r, p->seed, uid, PURPOSE_VALUES);
  for (int32_t k = 0; k < d; ++k) {
    double cv, av;
    if (p->c_model == C_NEG_UNIFORM)
      cv = -rng_uniform(&r);
    else
      cv = -exp(p->c_mu + p->c_sigma * rng_normal(&r));
    if (p->a_model == A_ONE)
      av = 1.0;
    else
      av = p->a_lo + (p->a_hi - p->a_lo) * rng_uniform(&r);
    c[k] = (float)cv;
    a[k] = (float)av;
  }
}

static void table_build(const synth_params* p, item_table* t) {
  t->cdf = NULL;
  t->total = 0;
  if (p->item_model != ITEMS_ZIPF) return;
  t->cdf = (double*)malloc(sizeof(double) * (size_t)p->J);
  double acc = 0;
  for (int32_t j = 0; j < p->J; ++j) {
    acc += pow((double)(j + 1), -p->zipf_s);
    t->cdf[j] = acc;
  }
  t->total = acc;
}

static inline uint64_t uid_of(const int64_t* ids, int64_t i) { return ids ? (uint64_t)ids[i] : (uint64_t)i; }

static int threads_or_default(int nthreads) {
#ifdef _OPENMP
  return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
  (void)nthreads;
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Exported entry points                                                     */
/* ------------------------------------------------------------------------ */

/* Degrees of n users (ids[i], or i when ids is NULL). */
int synth_degrees(const synth_params* p, const int64_t* ids, int64_t n, int32_t* deg, int nthreads) {
  int nt = threads_or_default(nthreads);
#pragma omp parallel for schedule(static) num_threads(nt)
  for (int64_t i = 0; i < n; ++i) deg[i] = draw_degree(p, uid_of(ids, i));
  return 0;
}

/* Items and values of n users whose rows start at row_ptr[i]. */
int synth_fill(const synth_params* p, const int64_t* ids, int64_t n, const int64_t* row_ptr, int32_t* col, float* c,
               float* a, int nthreads) {
  item_table t;
  table_build(p, &t);
  int nt = threads_or_default(nthreads);
#pragma omp parallel num_threads(nt)
  {
    scratch_t s;
    scratch_alloc(&s, p->J);
#pragma omp for schedule(dynamic, 4096)
    for (int64_t i = 0; i < n; ++i) {
      int64_t b = row_ptr[i];
      int32_t d = (int32_t)(row_ptr[i + 1] - b);
      if (d <= 0) continue;
      uint64_t uid = uid_of(ids, i);
      draw_items(p, &t, uid, d, col + b, &s);
      draw_values(p, uid, d, c + b, a + b);
    }
    scratch_free(&s);
  }
  free(t.cdf);
  return 0;
}

/* Item capacities: b_j = frac * deg_j (B_ITEM_DEGREE) or frac * sum_i a_ij
 * (B_SUM_A).  Sums run over fixed user chunks in chunk order, so the result
 * does not depend on the thread count. */
int synth_capacity(const synth_params* p, int64_t n, const int64_t* row_ptr, const int32_t* col, const float* a,
                   double* b, int nthreads) {
  const int32_t J = p->J;
  int64_t nchunks = n / 65536;
  if (nchunks < 1) nchunks = 1;
  if (nchunks > 256) nchunks = 256;
  double* part = (double*)calloc((size_t)nchunks * (size_t)J, sizeof(double));
  if (!part) return -1;
  int nt = threads_or_default(nthreads);
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
  for (int64_t ch = 0; ch < nchunks; ++ch) {
    int64_t u0 = n * ch / nchunks, u1 = n * (ch + 1) / nchunks;
    double* row = part + (size_t)ch * (size_t)J;
    for (int64_t e = row_ptr[u0]; e < row_ptr[u1]; ++e)
      row[col[e]] += (p->b_model == B_ITEM_DEGREE) ? 1.0 : (double)a[e];
  }
  for (int32_t j = 0; j < J; ++j) {
    double s = 0;
    for (int64_t ch = 0; ch < nchunks; ++ch) s += part[(size_t)ch * (size_t)J + j];
    b[j] = p->b_frac * s;
  }
  free(part);
  return 0;
}

/* Round-to-nearest-even float32 -> bfloat16 bit patterns (finite inputs). */
void synth_round_bf16(const float* in, uint16_t* out, int64_t n, int nthreads) {
  int nt = threads_or_default(nthreads);
#pragma omp parallel for schedule(static) num_threads(nt)
  for (int64_t i = 0; i < n; ++i) {
    uint32_t u;
    memcpy(&u, &in[i], 4);
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7FFFu + lsb;
    out[i] = (uint16_t)(u >> 16);
  }
}

/* Day-to-day drift of a recurring instance.
 *   churn:  each user slot is replaced with probability churn_p by a new user
 *           (new id from new_id_base + slot); its row is regenerated.
 *   noise:  on the surviving rows, each edge gets c += noise_sd * N(0,1) with
 *           probability noise_p.
 * Pass 1 (out_row_ptr == NULL): write new ids and degrees (new_deg).
 * Pass 2: fill out arrays from the previous day's arrays. */
int synth_next_day_ids(uint64_t day_seed, int64_t n, const int64_t* prev_ids, double churn_p, int64_t new_id_base,
                       int64_t* new_ids, int nthreads) {
  int nt = threads_or_default(nthreads);
#pragma omp parallel for schedule(static) num_threads(nt)
  for (int64_t i = 0; i < n; ++i) {
    rng_t r;
    rng_init(&r, day_seed, (uint64_t)i, PURPOSE_CHURN);
    new_ids[i] = (rng_uniform(&r) < churn_p) ? new_id_base + i : prev_ids[i];
  }
  return 0;
}

int synth_next_day_fill(const synth_params* p, uint64_t day_seed, int64_t n, const int64_t* prev_ids,
                        const int64_t* prev_row_ptr, const int32_t* prev_col, const float* prev_c,
                        const float* prev_a, const int64_t* new_ids, const int64_t* new_row_ptr, int32_t* col,
                        float* c, float* a, double noise_p, double noise_sd, int nthreads) {
  item_table t;
  table_build(p, &t);
  int nt = threads_or_default(nthreads);
#pragma omp parallel num_threads(nt)
  {
    scratch_t s;
    scratch_alloc(&s, p->J);
#pragma omp for schedule(dynamic, 4096)
    for (int64_t i = 0; i < n; ++i) {
      int64_t b = new_row_ptr[i];
      int32_t d = (int32_t)(new_row_ptr[i + 1] - b);
      if (new_ids[i] != prev_ids[i]) {
        draw_items(p, &t, (uint64_t)new_ids[i], d, col + b, &s);
        draw_values(p, (uint64_t)new_ids[i], d, c + b, a + b);
        continue;
      }
      int64_t pb = prev_row_ptr[i];
      rng_t r;
      rng_init(&r, day_seed, (uint64_t)new_ids[i], PURPOSE_NOISE);
      for (int32_t k = 0; k < d; ++k) {
        col[b + k] = prev_col[pb + k];
        a[b + k] = prev_a[pb + k];
        double u = rng_uniform(&r);
        double z = rng_normal(&r);
        double cv = prev_c[pb + k];
        if (u < noise_p) cv += noise_sd * z;
        c[b + k] = (float)cv;
      }
    }
    scratch_free(&s);
  }
  free(t.cdf);
  return 0;
}

/* b_j <- b_j * max(0, 1 + sd * N(0,1)), keyed by (day_seed, item). */
int synth_scale_capacity(uint64_t day_seed, int32_t J, double sd, double* b) {
  for (int32_t j = 0; j < J; ++j) {
    rng_t r;
    rng_init(&r, day_seed, (uint64_t)j, PURPOSE_NOISE + 16);
    double f = 1.0 + sd * rng_normal(&r);
    if (f < 0) f = 0;
    b[j] *= f;
  }
  return 0;
}

/* Uniform draws keyed by (seed, id, purpose): used for seeded samples. */
void synth_uniforms(uint64_t seed, uint64_t id, uint32_t purpose, int64_t n, double* out) {
  rng_t r;
  rng_init(&r, seed, id, purpose);
  for (int64_t i = 0; i < n; ++i) out[i] = rng_uniform(&r);
}

/* ------------------------------------------------------------------------ */
/* The appendix generator (App. A)                                           */
/* ------------------------------------------------------------------------ */
/* Item-major construction: resource j draws a lognormal breadth w_j, gets
 * p_j = w_j / sum_k w_k and K_j ~ Poisson(p_j I nu) requests (truncated at I),
 * chosen as K_j distinct requests uniformly at random.  Edge values are
 * v_j u_i eps_ij capped at c_max (v, u, eps lognormal); the stored cost is
 * its negation (minimisation); a_ij = s_j * value with lognormal s_j.
 * Capacities come from the greedy load: every request sends its largest a_ij
 * (first such item on ties) to that item, l_j is the sum, and
 * b_j = rho_j (l_j + eps_b) with rho_j ~ U[rho_lo, rho_hi].
 * Distribution parameters are inputs; the paper leaves them open. */
typedef struct {
  int64_t I;
  int32_t J;
  int32_t _pad0;
  uint64_t seed;
  double nu;            /* mean edges per request */
  double breadth_sigma; /* w_j ~ LogNormal(0, breadth_sigma) */
  double v_sigma;       /* v_j ~ LogNormal(0, v_sigma) */
  double u_sigma;       /* u_i ~ LogNormal(0, u_sigma) */
  double eps_sigma;     /* eps_ij ~ LogNormal(0, eps_sigma) */
  double c_max;
  double s_mu, s_sigma; /* s_j ~ LogNormal(s_mu, s_sigma) */
  double rho_lo, rho_hi;
  double b_eps;
} synth_app_params;

enum {
  PURPOSE_APP_BREADTH = 32,
  PURPOSE_APP_COUNT = 33,
  PURPOSE_APP_PICK = 34,
  PURPOSE_APP_V = 35,
  PURPOSE_APP_U = 36,
  PURPOSE_APP_EPS = 37,
  PURPOSE_APP_S = 38,
  PURPOSE_APP_RHO = 39
};

/* Poisson(mu) for any mu >= 0: the sum of independent Poisson draws over
 * pieces of mu of at most 200 (Poisson laws add), each by inversion. */
static int64_t rng_poisson_big(rng_t* r, double mu) {
  int64_t k = 0;
  while (mu > 200.0) {
    k += rng_poisson(r, 200.0);
    mu -= 200.0;
  }
  if (mu > 0) k += rng_poisson(r, mu);
  return k;
}

static double keyed_lognormal(uint64_t seed, uint64_t id, uint32_t purpose, double mu, double sigma) {
  rng_t r;
  rng_init(&r, seed, id, purpose);
  return exp(mu + sigma * rng_normal(&r));
}

/* Draw 1: K_j for every resource (sequential over j; O(J + I nu)). */
int synth_app_counts(const synth_app_params* p, int64_t* K) {
  const int32_t J = p->J;
  double* w = (double*)malloc(sizeof(double) * (size_t)(J > 0 ? J : 1));
  if (!w) return -1;
  double tot = 0;
  for (int32_t j = 0; j < J; ++j) {
    w[j] = keyed_lognormal(p->seed, (uint64_t)j, PURPOSE_APP_BREADTH, 0.0, p->breadth_sigma);
    tot += w[j];
  }
  for (int32_t j = 0; j < J; ++j) {
    rng_t r;
    rng_init(&r, p->seed, (uint64_t)j, PURPOSE_APP_COUNT);
    int64_t k = rng_poisson_big(&r, w[j] / tot * (double)p->I * p->nu);
    K[j] = k > p->I ? p->I : k;
  }
  free(w);
  return 0;
}

static int cmp_i64(const void* x, const void* y) {
  int64_t a = *(const int64_t*)x, b = *(const int64_t*)y;
  return (a > b) - (a < b);
}

/* Draw 2: the K_j distinct requests of every resource, ascending, written to
 * users[col_ptr[j] ..].  Rejection against a bitmap of taken requests; above
 * I / 2 the I - K_j requests left out are drawn instead. */
int synth_app_pick(const synth_app_params* p, const int64_t* col_ptr, int64_t* users, int nthreads) {
  const int64_t I = p->I;
  const size_t words = (size_t)((I + 63) / 64);
  int nt = threads_or_default(nthreads);
  int fail = 0;
#pragma omp parallel num_threads(nt)
  {
    uint64_t* bm = (uint64_t*)calloc(words ? words : 1, sizeof(uint64_t));
    int64_t* tmp = NULL;
    int64_t cap = 0;
    if (!bm) {
#pragma omp atomic write
      fail = 1;
    }
#pragma omp for schedule(dynamic, 1)
    for (int32_t j = 0; j < p->J; ++j) {
      if (!bm) continue;
      const int64_t K = col_ptr[j + 1] - col_ptr[j];
      int64_t* out = users + col_ptr[j];
      const int complement = K > I / 2;
      const int64_t n = complement ? I - K : K;
      if (n > cap) {
        free(tmp);
        cap = n;
        tmp = (int64_t*)malloc(sizeof(int64_t) * (size_t)cap);
      }
      rng_t r;
      rng_init(&r, p->seed, (uint64_t)j, PURPOSE_APP_PICK);
      for (int64_t t = 0; t < n; ++t) {
        int64_t i;
        do {
          i = (int64_t)(rng_uniform(&r) * (double)I);
          if (i >= I) i = I - 1;
        } while (bm[i >> 6] >> (i & 63) & 1u);
        bm[i >> 6] |= (uint64_t)1 << (i & 63);
        tmp[t] = i;
      }
      if (complement) {
        int64_t o = 0;
        for (int64_t i = 0; i < I; ++i)
          if (!(bm[i >> 6] >> (i & 63) & 1u)) out[o++] = i;
      } else {
        memcpy(out, tmp, sizeof(int64_t) * (size_t)n);
        qsort(out, (size_t)n, sizeof(int64_t), cmp_i64);
      }
      for (int64_t t = 0; t < n; ++t) bm[tmp[t] >> 6] = 0;
    }
    free(tmp);
    free(bm);
  }
  return fail ? -1 : 0;
}

/* Item-major (col_ptr, users) -> user-major columns: row i lists its
 * resources ascending at row_ptr[i] ..  Threads own request ranges and find
 * their part of every resource list by binary search. */
int synth_app_transpose(int64_t I, int32_t J, const int64_t* col_ptr, const int64_t* users, const int64_t* row_ptr,
                        int32_t* col, int nthreads) {
  int nt = threads_or_default(nthreads);
  int64_t nranges = (int64_t)nt * 16;
  if (nranges > I) nranges = I > 0 ? I : 1;
  int fail = 0;
#pragma omp parallel num_threads(nt)
  {
    int64_t* fill = NULL;
    int64_t fcap = 0;
#pragma omp for schedule(dynamic, 1)
    for (int64_t g = 0; g < nranges; ++g) {
      const int64_t u0 = I * g / nranges, u1 = I * (g + 1) / nranges;
      if (u1 - u0 > fcap) {
        free(fill);
        fcap = u1 - u0;
        fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)fcap);
        if (!fill) {
#pragma omp atomic write
          fail = 1;
          fcap = 0;
          continue;
        }
      }
      for (int64_t u = u0; u < u1; ++u) fill[u - u0] = row_ptr[u];
      for (int32_t j = 0; j < J; ++j) {
        int64_t lo = col_ptr[j], hi = col_ptr[j + 1];
        while (lo < hi) { /* first entry >= u0 */
          int64_t mid = lo + (hi - lo) / 2;
          if (users[mid] < u0) lo = mid + 1; else hi = mid;
        }
        for (int64_t e = lo; e < col_ptr[j + 1] && users[e] < u1; ++e) col[fill[users[e] - u0]++] = j;
      }
    }
    free(fill);
  }
  return fail ? -1 : 0;
}

/* Edge values of n requests (user-major rows from synth_app_transpose). */
int synth_app_values(const synth_app_params* p, int64_t n, const int64_t* row_ptr, const int32_t* col, float* c,
                     float* a, int nthreads) {
  const int32_t J = p->J;
  double* v = (double*)malloc(sizeof(double) * (size_t)(J > 0 ? J : 1));
  double* s = (double*)malloc(sizeof(double) * (size_t)(J > 0 ? J : 1));
  if (!v || !s) {
    free(v);
    free(s);
    return -1;
  }
  for (int32_t j = 0; j < J; ++j) {
    v[j] = keyed_lognormal(p->seed, (uint64_t)j, PURPOSE_APP_V, 0.0, p->v_sigma);
    s[j] = keyed_lognormal(p->seed, (uint64_t)j, PURPOSE_APP_S, p->s_mu, p->s_sigma);
  }
  int nt = threads_or_default(nthreads);
#pragma omp parallel for schedule(dynamic, 4096) num_threads(nt)
  for (int64_t i = 0; i < n; ++i) {
    if (row_ptr[i + 1] == row_ptr[i]) continue;
    const double u = keyed_lognormal(p->seed, (uint64_t)i, PURPOSE_APP_U, 0.0, p->u_sigma);
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
      const int32_t j = col[e];
      const double eps =
          keyed_lognormal(p->seed, (uint64_t)i * (uint64_t)J + (uint64_t)j, PURPOSE_APP_EPS, 0.0, p->eps_sigma);
      double val = v[j] * u * eps;
      if (val > p->c_max) val = p->c_max;
      c[e] = (float)(-val);
      a[e] = (float)(s[j] * val);
    }
  }
  free(v);
  free(s);
  return 0;
}

/* Greedy loads l_j (sums of the float a in fixed request chunks, chunk
 * order) and b_j = rho_j (l_j + eps_b).  load may be NULL. */
int synth_app_capacity(const synth_app_params* p, int64_t n, const int64_t* row_ptr, const int32_t* col,
                       const float* a, double* load, double* b, int nthreads) {
  const int32_t J = p->J;
  int64_t nchunks = n / 65536;
  if (nchunks < 1) nchunks = 1;
  if (nchunks > 256) nchunks = 256;
  double* part = (double*)calloc((size_t)nchunks * (size_t)J, sizeof(double));
  if (!part) return -1;
  int nt = threads_or_default(nthreads);
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
  for (int64_t ch = 0; ch < nchunks; ++ch) {
    int64_t u0 = n * ch / nchunks, u1 = n * (ch + 1) / nchunks;
    double* row = part + (size_t)ch * (size_t)J;
    for (int64_t i = u0; i < u1; ++i) {
      int64_t best = -1;
      for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
        if (best < 0 || a[e] > a[best]) best = e;
      if (best >= 0) row[col[best]] += (double)a[best];
    }
  }
  for (int32_t j = 0; j < J; ++j) {
    double l = 0;
    for (int64_t ch = 0; ch < nchunks; ++ch) l += part[(size_t)ch * (size_t)J + j];
    rng_t r;
    rng_init(&r, p->seed, (uint64_t)j, PURPOSE_APP_RHO);
    const double rho = p->rho_lo + (p->rho_hi - p->rho_lo) * rng_uniform(&r);
    if (load) load[j] = l;
    b[j] = rho * (l + p->b_eps);
  }
  free(part);
  return 0;
}

/* n draws of Poisson(mu) from the stream (seed, id, purpose): exposes the
 * sampler behind K_j for distribution tests. */
void synth_poisson(uint64_t seed, uint64_t id, uint32_t purpose, double mu, int64_t n, int64_t* out) {
  rng_t r;
  rng_init(&r, seed, id, purpose);
  for (int64_t i = 0; i < n; ++i) out[i] = rng_poisson_big(&r, mu);
}
