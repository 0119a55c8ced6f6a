/*
 * Seeded synthetic X-engine input: 4+4-bit offset-encoded complex samples.
 *
 * This module only MAKES input bytes. It holds none of the correlator's
 * arithmetic; both the CPU oracle and the GPU library consume its output.
 *
 * Data format (Sec. III, Fig. 2 of the paper): one byte per complex sample,
 * ordered [time][band][element]; each part is an excess-8 integer, value
 * in [-8, 7] stored as value + 8 in [0, 15]; high nibble = real part,
 * low nibble = imaginary part (the paper only says both parts share a byte).
 *
 * Random numbers come from SplitMix64 (G. Steele, D. Lea, C. Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014) used as a
 * counter-based generator: draw c of stream `seed` is mix(seed + (c+1)*gamma),
 * which equals the c-th output of a SplitMix64 generator seeded with `seed`.
 * Gaussian draws use the Box-Muller transform (Box & Muller, 1958).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SYNTH_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t synth_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Draw number c (0-based) of the SplitMix64 stream seeded with `seed`. */
uint64_t synth_draw(uint64_t seed, uint64_t c) { return synth_mix(seed + (c + 1) * SYNTH_GAMMA); }

static inline int clip_level(double v) {
  double r = nearbyint(v); /* round half to even under the default rounding mode */
  if (r < -8.0) r = -8.0;
  if (r > 7.0) r = 7.0;
  return (int)r;
}

static inline uint8_t encode(int re, int im) { return (uint8_t)(((re + 8) << 4) | (im + 8)); }

typedef struct {
  uint8_t* out;
  int64_t N, F, T;
  double sigma, tone_amp, tone_k;
  uint64_t seed;
  int mode; /* 0 uniform nibbles, 1 gaussian (+tone) */
  int64_t t0, t1;
} job_t;

static void* worker(void* arg) {
  const job_t* j = (const job_t*)arg;
  const int64_t FN = j->F * j->N;
  const double two_pi = 6.283185307179586476925286766559;
  for (int64_t t = j->t0; t < j->t1; ++t) {
    double tr = 0.0, ti = 0.0;
    if (j->mode == 1 && j->tone_amp != 0.0) {
      double th = two_pi * j->tone_k * (double)t / (double)j->T;
      tr = j->tone_amp * cos(th);
      ti = j->tone_amp * sin(th);
    }
    uint8_t* row = j->out + t * FN;
    for (int64_t k = 0; k < FN; ++k) {
      const uint64_t c = (uint64_t)(t * FN + k);
      if (j->mode == 0) {
        row[k] = (uint8_t)(synth_draw(j->seed, c) >> 56);
      } else {
        const uint64_t r1 = synth_draw(j->seed, 2 * c), r2 = synth_draw(j->seed, 2 * c + 1);
        const double u1 = (double)((r1 >> 11) + 1) * 0x1.0p-53; /* (0, 1] */
        const double u2 = (double)(r2 >> 11) * 0x1.0p-53;       /* [0, 1) */
        const double rad = sqrt(-2.0 * log(u1));
        const double zr = rad * cos(two_pi * u2), zi = rad * sin(two_pi * u2);
        row[k] = encode(clip_level(j->sigma * zr + tr), clip_level(j->sigma * zi + ti));
      }
    }
  }
  return NULL;
}

static int run_jobs(job_t proto, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if (proto.T < (int64_t)nthreads) nthreads = proto.T > 0 ? (int)proto.T : 1;
  pthread_t th[256];
  int ok[256];
  job_t jobs[256];
  for (int i = 0; i < nthreads; ++i) {
    jobs[i] = proto;
    jobs[i].t0 = proto.T * i / nthreads;
    jobs[i].t1 = proto.T * (i + 1) / nthreads;
    ok[i] = pthread_create(&th[i], NULL, worker, &jobs[i]) == 0;
    if (!ok[i]) worker(&jobs[i]); /* run inline if a thread cannot be started */
  }
  for (int i = 0; i < nthreads; ++i)
    if (ok[i]) pthread_join(th[i], NULL);
  return 0;
}

/* Uniform nibbles: byte (t, f, n) = top 8 bits of draw number ((t*F+f)*N+n). */
int synth_uniform(uint8_t* out, int64_t N, int64_t F, int64_t T, uint64_t seed, int nthreads) {
  if (!out || N < 0 || F < 0 || T < 0) return -1;
  job_t p;
  memset(&p, 0, sizeof p);
  p.out = out; p.N = N; p.F = F; p.T = T; p.seed = seed; p.mode = 0;
  return run_jobs(p, nthreads);
}

/*
 * Gaussian levels: for sample c = (t*F+f)*N+n, draws 2c and 2c+1 give one
 * Box-Muller pair (zr, zi); part = clip(rint(sigma*z + tone), -8, 7), where
 * the common tone is tone_amp * exp(2*pi*i*tone_k*t/T), the same for every
 * element and band (tone_amp = 0 disables it).
 */
int synth_gauss(uint8_t* out, int64_t N, int64_t F, int64_t T, double sigma, double tone_amp, double tone_k,
                uint64_t seed, int nthreads) {
  if (!out || N < 0 || F < 0 || T < 0) return -1;
  job_t p;
  memset(&p, 0, sizeof p);
  p.out = out; p.N = N; p.F = F; p.T = T; p.seed = seed; p.mode = 1;
  p.sigma = sigma; p.tone_amp = tone_amp; p.tone_k = tone_k;
  return run_jobs(p, nthreads);
}
