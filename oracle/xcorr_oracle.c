/*
 * CPU ORACLE for the 4-bit X-engine -- test infrastructure, not product code.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * call this file. It shares no code with the GPU library, and the GPU
 * library never calls it.
 *
 * It is the plain definition of what the correlator computes, written out
 * with int64 accumulators and explicit loops:
 *
 *   Eq. 1 (Sec. II.A): the correlation of two complex samples X, Y at one
 *     instant is X * conj(Y) = (XrYr + XiYi, XiYr - XrYi).
 *   Sec. II.A: the products are accumulated over many time samples, and the
 *     matrix A of all (X, Y) pairs is Hermitian, so only the upper triangle
 *     (autocorrelations included) is needed (Eq. 2 counts N(N+1)/2 entries).
 *   Sec. III: each part is an excess-8 4-bit integer, value = nibble - 8 in
 *     [-8, 7]; real and imaginary parts share one byte. Reading taken where
 *     the paper is silent: the high nibble is the real part.
 *   Fig. 2: samples are ordered [time][band][element].
 *
 * So, for band f and elements i <= j (X = element i, Y = element j):
 *   Re V[f,i,j] = sum_t xr[t,f,i]*xr[t,f,j] + xi[t,f,i]*xi[t,f,j]
 *   Im V[f,i,j] = sum_t xi[t,f,i]*xr[t,f,j] - xr[t,f,i]*xi[t,f,j]
 * stored packed, row-major over the upper triangle:
 *   p(i,j) = i*N - i*(i-1)/2 + (j - i), V[(f*B + p)*2 + {0: Re, 1: Im}],
 *   B = N(N+1)/2.
 *
 * Also here: single entries on demand (sampled checks at full size), the
 * full square for small N, the Freivalds right-hand side sum_t x_i *
 * sum_j conj(x_j) w_j (= row i of V w for the full Hermitian V), and the
 * Eq. 3 offset terms for offset-encoded (unsigned) products.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline int8_t re_of(uint8_t b) { return (int8_t)((int)(b >> 4) - 8); }
static inline int8_t im_of(uint8_t b) { return (int8_t)((int)(b & 15) - 8); }

/* ------------------------------------------------------------------------ */
/* Decoded planes xr[f][n][t], xi[f][n][t]: a plain transposition of the input. */
typedef struct {
  int8_t* xr;
  int8_t* xi;
} planes_t;

static int decode_planes(const uint8_t* x, int64_t N, int64_t F, int64_t T, planes_t* p) {
  const size_t n = (size_t)F * (size_t)N * (size_t)T;
  p->xr = (int8_t*)malloc(n ? n : 1);
  p->xi = (int8_t*)malloc(n ? n : 1);
  if (!p->xr || !p->xi) {
    free(p->xr);
    free(p->xi);
    return -2;
  }
  for (int64_t t = 0; t < T; ++t)
    for (int64_t f = 0; f < F; ++f)
      for (int64_t e = 0; e < N; ++e) {
        const uint8_t b = x[(t * F + f) * N + e];
        const size_t o = ((size_t)f * N + e) * T + t;
        p->xr[o] = re_of(b);
        p->xi[o] = im_of(b);
      }
  return 0;
}

/* One visibility from decoded planes: Eq. 1 accumulated over t. */
static inline void corr_pair(const planes_t* p, int64_t N, int64_t T, int64_t f, int64_t i, int64_t j,
                             int64_t* re_out, int64_t* im_out) {
  const int8_t* ri = p->xr + ((size_t)f * N + i) * T;
  const int8_t* ii = p->xi + ((size_t)f * N + i) * T;
  const int8_t* rj = p->xr + ((size_t)f * N + j) * T;
  const int8_t* ij = p->xi + ((size_t)f * N + j) * T;
  int64_t re = 0, im = 0;
  for (int64_t t = 0; t < T; ++t) {
    re += (int64_t)ri[t] * rj[t] + (int64_t)ii[t] * ij[t];
    im += (int64_t)ii[t] * rj[t] - (int64_t)ri[t] * ij[t];
  }
  *re_out = re;
  *im_out = im;
}

/* ------------------------------------------------------------------------ */
typedef struct {
  const planes_t* p;
  int64_t N, F, T;
  int64_t* V;
  int full;      /* 0: packed upper triangle, 1: full square [F][N][N][2] */
  int tid, nthreads;
} vis_job_t;

static void* vis_worker(void* arg) {
  const vis_job_t* j = (const vis_job_t*)arg;
  const int64_t N = j->N, B = N * (N + 1) / 2;
  /* rows (f, i) dealt round-robin: row lengths fall linearly, so this balances */
  for (int64_t r = j->tid; r < j->F * N; r += j->nthreads) {
    const int64_t f = r / N, i = r % N;
    if (j->full) {
      for (int64_t c = 0; c < N; ++c) {
        int64_t re, im;
        corr_pair(j->p, N, j->T, f, i, c, &re, &im);
        int64_t* o = j->V + (((size_t)f * N + i) * N + c) * 2;
        o[0] = re;
        o[1] = im;
      }
    } else {
      const int64_t row0 = i * N - i * (i - 1) / 2; /* p(i, i) */
      for (int64_t c = i; c < N; ++c) {
        int64_t re, im;
        corr_pair(j->p, N, j->T, f, i, c, &re, &im);
        int64_t* o = j->V + ((size_t)f * B + row0 + (c - i)) * 2;
        o[0] = re;
        o[1] = im;
      }
    }
  }
  return NULL;
}

static int run_vis(const uint8_t* x, int64_t N, int64_t F, int64_t T, int64_t* V, int full, int nthreads) {
  if (!x || !V || N < 1 || F < 1 || T < 0) return -1;
  planes_t p;
  int rc = decode_planes(x, N, F, T, &p);
  if (rc) return rc;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 512) nthreads = 512;
  pthread_t th[512];
  int ok[512];
  vis_job_t jobs[512];
  for (int k = 0; k < nthreads; ++k) {
    vis_job_t jj = {&p, N, F, T, V, full, k, nthreads};
    jobs[k] = jj;
    ok[k] = pthread_create(&th[k], NULL, vis_worker, &jobs[k]) == 0;
    if (!ok[k]) vis_worker(&jobs[k]);
  }
  for (int k = 0; k < nthreads; ++k)
    if (ok[k]) pthread_join(th[k], NULL);
  free(p.xr);
  free(p.xi);
  return 0;
}

/* Packed upper triangle V[F][N(N+1)/2][2], int64. */
int oracle_visibilities(const uint8_t* x, int64_t N, int64_t F, int64_t T, int64_t* V, int nthreads) {
  return run_vis(x, N, F, T, V, 0, nthreads);
}

/* Every ordered pair (i, j): V[F][N][N][2], int64 (small N only). */
int oracle_visibilities_full(const uint8_t* x, int64_t N, int64_t F, int64_t T, int64_t* V, int nthreads) {
  return run_vis(x, N, F, T, V, 1, nthreads);
}

/* ------------------------------------------------------------------------ */
/* Single entries straight from the bytes: out[k] = (Re, Im) of V[f_k, i_k, j_k]. */
typedef struct {
  const uint8_t* x;
  int64_t N, F, T;
  const int64_t* fij;
  int64_t count;
  int64_t* out;
  int tid, nthreads;
} ent_job_t;

static void* ent_worker(void* arg) {
  const ent_job_t* j = (const ent_job_t*)arg;
  for (int64_t k = j->tid; k < j->count; k += j->nthreads) {
    const int64_t f = j->fij[3 * k], a = j->fij[3 * k + 1], b = j->fij[3 * k + 2];
    int64_t re = 0, im = 0;
    for (int64_t t = 0; t < j->T; ++t) {
      const uint8_t xa = j->x[(t * j->F + f) * j->N + a];
      const uint8_t xb = j->x[(t * j->F + f) * j->N + b];
      re += (int64_t)re_of(xa) * re_of(xb) + (int64_t)im_of(xa) * im_of(xb);
      im += (int64_t)im_of(xa) * re_of(xb) - (int64_t)re_of(xa) * im_of(xb);
    }
    j->out[2 * k] = re;
    j->out[2 * k + 1] = im;
  }
  return NULL;
}

int oracle_entries(const uint8_t* x, int64_t N, int64_t F, int64_t T, const int64_t* fij, int64_t count,
                   int64_t* out, int nthreads) {
  if (!x || !fij || !out || N < 1 || F < 1 || T < 0 || count < 0) return -1;
  for (int64_t k = 0; k < count; ++k) {
    const int64_t f = fij[3 * k], a = fij[3 * k + 1], b = fij[3 * k + 2];
    if (f < 0 || f >= F || a < 0 || a >= N || b < 0 || b >= N) return -1;
  }
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 512) nthreads = 512;
  pthread_t th[512];
  int ok[512];
  ent_job_t jobs[512];
  for (int k = 0; k < nthreads; ++k) {
    ent_job_t jj = {x, N, F, T, fij, count, out, k, nthreads};
    jobs[k] = jj;
    ok[k] = pthread_create(&th[k], NULL, ent_worker, &jobs[k]) == 0;
    if (!ok[k]) ent_worker(&jobs[k]);
  }
  for (int k = 0; k < nthreads; ++k)
    if (ok[k]) pthread_join(th[k], NULL);
  return 0;
}

/* ------------------------------------------------------------------------ */
/*
 * Freivalds right-hand side. For weights w[f][n] (complex int, (Re, Im)):
 *   r[f][i] = sum_t x[t,f,i] * s_t,   s_t = sum_j conj(x[t,f,j]) * w[f][j]
 * which equals sum_j V[f,i,j] * w[f][j] over the full Hermitian matrix.
 * O(F*N*T) work; the caller forms sum_j V_ij w_j from a packed result and
 * compares.
 */
int oracle_freivalds_rhs(const uint8_t* x, int64_t N, int64_t F, int64_t T, const int64_t* w, int64_t* r) {
  if (!x || !w || !r || N < 1 || F < 1 || T < 0) return -1;
  memset(r, 0, sizeof(int64_t) * 2 * (size_t)F * (size_t)N);
  for (int64_t t = 0; t < T; ++t)
    for (int64_t f = 0; f < F; ++f) {
      const uint8_t* row = x + (t * F + f) * N;
      const int64_t* wf = w + 2 * f * N;
      int64_t sr = 0, si = 0; /* s_t = sum_j conj(x_j) w_j */
      for (int64_t j = 0; j < N; ++j) {
        const int64_t a = re_of(row[j]), b = im_of(row[j]);
        /* (a - ib)(wr + i wi) = (a wr + b wi) + i (a wi - b wr) */
        sr += a * wf[2 * j] + b * wf[2 * j + 1];
        si += a * wf[2 * j + 1] - b * wf[2 * j];
      }
      int64_t* rf = r + 2 * f * N;
      for (int64_t i = 0; i < N; ++i) {
        const int64_t a = re_of(row[i]), b = im_of(row[i]);
        /* (a + ib)(sr + i si) */
        rf[2 * i] += a * sr - b * si;
        rf[2 * i + 1] += a * si + b * sr;
      }
    }
  return 0;
}

/* ------------------------------------------------------------------------ */
/*
 * Eq. 3 (Sec. III): offset terms for products of offset-ENCODED values
 * u = x + 8, accumulated over the T samples (the sum's upper limit is read
 * as T terms, t = 0..T-1). For elements X = i, Y = j:
 *   Re B = sum_t -8((uXr + uXi) + (uYr + uYi)) + 128
 *   Im B = sum_t  8((uXr - uXi) - (uYr - uYi))
 * Adding B to the encoded-value correlation sum_t (uXr uYr + uXi uYi,
 * uXi uYr - uXr uYi) gives the signed correlation. Output packed like V.
 */
int oracle_offset_terms(const uint8_t* x, int64_t N, int64_t F, int64_t T, int64_t* Bout) {
  if (!x || !Bout || N < 1 || F < 1 || T < 0) return -1;
  const int64_t B = N * (N + 1) / 2;
  int64_t* sp = (int64_t*)calloc((size_t)F * N, sizeof(int64_t)); /* sum_t (uRe + uIm) */
  int64_t* sm = (int64_t*)calloc((size_t)F * N, sizeof(int64_t)); /* sum_t (uRe - uIm) */
  if (!sp || !sm) {
    free(sp);
    free(sm);
    return -2;
  }
  for (int64_t t = 0; t < T; ++t)
    for (int64_t f = 0; f < F; ++f)
      for (int64_t e = 0; e < N; ++e) {
        const uint8_t b = x[(t * F + f) * N + e];
        const int64_t ur = b >> 4, ui = b & 15;
        sp[f * N + e] += ur + ui;
        sm[f * N + e] += ur - ui;
      }
  for (int64_t f = 0; f < F; ++f)
    for (int64_t i = 0; i < N; ++i)
      for (int64_t j = i; j < N; ++j) {
        int64_t* o = Bout + ((size_t)f * B + i * N - i * (i - 1) / 2 + (j - i)) * 2;
        o[0] = -8 * (sp[f * N + i] + sp[f * N + j]) + 128 * T;
        o[1] = 8 * (sm[f * N + i] - sm[f * N + j]);
      }
  free(sp);
  free(sm);
  return 0;
}

/* ------------------------------------------------------------------------ */
/*
 * Per-element integer time shift before correlation (Sec. IV: a kernel that
 * shifts individual elements by integer time steps, to create or compensate
 * lags). out[t,f,i] = in[t - lag_i, f, i] when 0 <= t - lag_i < T, else the
 * code of 0 + 0i (0x88): samples shifted in from outside the frame are zero.
 */
int oracle_shift_lags(const uint8_t* in, int64_t N, int64_t F, int64_t T, const int32_t* lags, uint8_t* out) {
  if (!in || !out || !lags || N < 1 || F < 1 || T < 0) return -1;
  for (int64_t t = 0; t < T; ++t)
    for (int64_t f = 0; f < F; ++f)
      for (int64_t i = 0; i < N; ++i) {
        const int64_t src = t - (int64_t)lags[i];
        out[(t * F + f) * N + i] = (src >= 0 && src < T) ? in[(src * F + f) * N + i] : (uint8_t)0x88;
      }
  return 0;
}

/* ------------------------------------------------------------------------ */
/*
 * Gated correlation (Sec. IV: the products are binned by time into several
 * gates, for periodic signals such as pulsars or calibration sources).
 * Reading: gate(t) = floor(((t + phase) mod period) * G / period), i.e. G
 * equal phase bins of a repeating period. V[g][f][p][2] accumulates Eq. 1's
 * products of the samples with gate(t) = g; packed like oracle_visibilities.
 */
int oracle_gated(const uint8_t* x, int64_t N, int64_t F, int64_t T, int64_t G, int64_t period, int64_t phase,
                 int64_t* V) {
  if (!x || !V || N < 1 || F < 1 || T < 0 || G < 1 || period < 1 || phase < 0) return -1;
  const int64_t B = N * (N + 1) / 2;
  int64_t* gate = (int64_t*)malloc(sizeof(int64_t) * (size_t)(T ? T : 1));
  if (!gate) return -2;
  for (int64_t t = 0; t < T; ++t) gate[t] = ((t + phase) % period) * G / period;
  memset(V, 0, sizeof(int64_t) * 2 * (size_t)(G * F * B));
  for (int64_t t = 0; t < T; ++t)
    for (int64_t f = 0; f < F; ++f) {
      const uint8_t* row = x + (t * F + f) * N;
      int64_t* Vg = V + 2 * (gate[t] * F + f) * B;
      for (int64_t i = 0; i < N; ++i)
        for (int64_t j = i; j < N; ++j) {
          const int64_t xr = re_of(row[i]), xi = im_of(row[i]), yr = re_of(row[j]), yi = im_of(row[j]);
          int64_t* o = Vg + 2 * (i * N - i * (i - 1) / 2 + (j - i));
          o[0] += xr * yr + xi * yi;
          o[1] += xi * yr - xr * yi;
        }
    }
  free(gate);
  return 0;
}
