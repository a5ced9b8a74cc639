/* Seeded synthetic inputs, native and threaded: the same streams as
 * sbbf_inputs.py, for sizes (billions of hashes) that numpy produces too
 * slowly.  Test infrastructure: input generation only, none of the filter's
 * arithmetic.
 *
 * splitmix64 in counter form (Steele, Lea, Flood 2014; Vigna's public-domain
 * generator): output i of seed s is mix(s + (i + 1) * 0x9E3779B97F4A7C15).
 *
 * Query recipe (threshold thr = round(member fraction * 2^32)): query k is a
 * member when (r_k >> 32) < thr, r = the member-selector stream; a member is
 * inserted hash base + (((r_k & 0xffffffff) * n) >> 32) of the insert
 * stream, n the number inserted, otherwise the fresh stream's output k.
 */
#include <pthread.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>

static uint64_t mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

uint64_t sin_splitmix64_at(uint64_t seed, uint64_t i) {
  return mix(seed + (i + 1) * 0x9E3779B97F4A7C15ull);
}

/* One query of a filter of the multi-filter recipe: k indexes the
 * member-selector and fresh streams, members are drawn from inserted hashes
 * [base, base + n); a filter with no inserted hashes gets fresh ones only. */
static uint64_t query_at(uint64_t seed_ins, uint64_t seed_fresh, uint64_t seed_member,
                         uint64_t thr, uint64_t base, uint64_t n, uint64_t k) {
  const uint64_t r = sin_splitmix64_at(seed_member, k);
  if (n > 0 && (r >> 32) < thr)
    return sin_splitmix64_at(seed_ins, base + (((r & 0xFFFFFFFFull) * n) >> 32));
  return sin_splitmix64_at(seed_fresh, k);
}

enum { KIND_FILL, KIND_WORKLOAD, KIND_SEGMENT };

typedef struct {
  int kind;
  uint64_t seed_ins, seed_fresh, seed_member, thr;
  uint64_t n_inserted, prefix;          /* workload queries */
  const int64_t *ins_off, *q_off;       /* segment queries */
  uint32_t t0, t1;
  uint64_t start;                       /* index of out[0] */
  size_t lo, hi;                        /* this thread's part of out */
  uint64_t *out;
} job_t;

static void *run_job(void *arg) {
  job_t *j = (job_t *)arg;
  if (j->kind == KIND_FILL) {
    for (size_t x = j->lo; x < j->hi; ++x) j->out[x] = sin_splitmix64_at(j->seed_ins, j->start + x);
  } else if (j->kind == KIND_WORKLOAD) {
    for (size_t x = j->lo; x < j->hi; ++x) {
      const uint64_t q = j->start + x;
      if (q < j->prefix) {
        j->out[x] = sin_splitmix64_at(j->seed_ins, q);
      } else {  /* members index the insert stream from 0 (n_inserted > 0 here) */
        const uint64_t k = q - j->prefix, r = sin_splitmix64_at(j->seed_member, k);
        j->out[x] = (r >> 32) < j->thr
                        ? sin_splitmix64_at(j->seed_ins, ((r & 0xFFFFFFFFull) * j->n_inserted) >> 32)
                        : sin_splitmix64_at(j->seed_fresh, k);
      }
    }
  } else {
    /* global query index k = start + x; filter t holds [q_off[t], q_off[t+1]) */
    uint32_t t = j->t0;
    for (size_t x = j->lo; x < j->hi; ++x) {
      const uint64_t k = j->start + x;
      while (t + 1 < j->t1 && (uint64_t)j->q_off[t + 1] <= k) ++t;
      const uint64_t base = (uint64_t)j->ins_off[t];
      const uint64_t n = (uint64_t)(j->ins_off[t + 1] - j->ins_off[t]);
      j->out[x] = query_at(j->seed_ins, j->seed_fresh, j->seed_member, j->thr, base, n, k);
    }
  }
  return NULL;
}

/* Runs `proto` over out[0..n) split between `threads` threads. */
static int run_split(const job_t *proto, size_t n, int threads) {
  if (threads < 1) threads = 1;
  if ((size_t)threads > n / 65536 + 1) threads = (int)(n / 65536 + 1);
  pthread_t *tid = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
  job_t *jobs = (job_t *)calloc((size_t)threads, sizeof(job_t));
  if (!tid || !jobs) {
    free(tid);
    free(jobs);
    return -1;
  }
  for (int t = 0; t < threads; ++t) {
    jobs[t] = *proto;
    jobs[t].lo = n * (size_t)t / (size_t)threads;
    jobs[t].hi = n * (size_t)(t + 1) / (size_t)threads;
  }
  /* the segment walk starts each thread at the filter holding its first index */
  if (proto->kind == KIND_SEGMENT) {
    for (int t = 0; t < threads; ++t) {
      const uint64_t k = proto->start + jobs[t].lo;
      uint32_t a = proto->t0, b = proto->t1;  /* last f in [t0, t1) with q_off[f] <= k */
      while (b - a > 1) {
        const uint32_t m = a + (b - a) / 2;
        if ((uint64_t)proto->q_off[m] <= k) a = m; else b = m;
      }
      jobs[t].t0 = a;
    }
  }
  int started = 0;
  for (int t = 0; t < threads; ++t) {
    if (pthread_create(&tid[t], NULL, run_job, &jobs[t]) != 0) {
      run_job(&jobs[t]);
      tid[t] = 0;
    } else {
      ++started;
    }
  }
  for (int t = 0; t < threads; ++t)
    if (tid[t]) pthread_join(tid[t], NULL);
  free(tid);
  free(jobs);
  return started;
}

/* out[x] = splitmix64 output start + x of seed, x < n. */
int sin_fill(uint64_t seed, uint64_t start, size_t n, uint64_t *out, int threads) {
  job_t j = {0};
  j.kind = KIND_FILL;
  j.seed_ins = seed;
  j.start = start;
  j.out = out;
  return run_split(&j, n, threads);
}

/* Lookups start..start+n-1 of a single-filter workload: indices below
 * `prefix` are inserted hashes in order; the rest follow the recipe indexed
 * from prefix, members drawn from inserted hashes [0, n_inserted). */
int sin_workload_queries(uint64_t seed_ins, uint64_t seed_fresh, uint64_t seed_member,
                         uint64_t thr, uint64_t n_inserted, uint64_t prefix, uint64_t start,
                         size_t n, uint64_t *out, int threads) {
  job_t j = {0};
  j.kind = KIND_WORKLOAD;
  j.seed_ins = seed_ins;
  j.seed_fresh = seed_fresh;
  j.seed_member = seed_member;
  j.thr = thr;
  j.n_inserted = n_inserted;
  j.prefix = prefix;
  j.start = start;
  j.out = out;
  return run_split(&j, n, threads);
}

/* Lookups of filters t0..t1-1 of a multi-filter workload in the segment
 * layout, written to out[0 .. q_off[t1] - q_off[t0]): query k of filter t
 * draws its members from that filter's inserted hashes
 * [ins_off[t], ins_off[t+1]). */
int sin_segment_queries(uint64_t seed_ins, uint64_t seed_fresh, uint64_t seed_member,
                        uint64_t thr, const int64_t *ins_off, const int64_t *q_off, uint32_t t0,
                        uint32_t t1, uint64_t *out, int threads) {
  if (t1 <= t0) return 0;
  job_t j = {0};
  j.kind = KIND_SEGMENT;
  j.seed_ins = seed_ins;
  j.seed_fresh = seed_fresh;
  j.seed_member = seed_member;
  j.thr = thr;
  j.ins_off = ins_off;
  j.q_off = q_off;
  j.t0 = t0;
  j.t1 = t1;
  j.start = (uint64_t)q_off[t0];
  j.out = out;
  return run_split(&j, (size_t)(q_off[t1] - q_off[t0]), threads);
}
