/*
 * Seeded synthetic signed bipartite graphs (COO: int32 u, int32 v, int8 sign).
 *
 * This module only draws inputs. It holds none of the counting arithmetic and
 * is used by both the CPU oracle tests and the GPU path, so that both see the
 * same edges for the same seed.
 *
 * Random numbers: SplitMix64 (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), used as a counter-based
 * generator: the k-th draw of stream s under seed x is mix(key(x, s) + k*phi),
 * so every draw can be computed independently and in any order.
 *
 * Models:
 *   - uniform:  endpoints uniform on each side.
 *   - Chung-Lu: endpoint i of a side is drawn with probability proportional to
 *     its expected degree d_i = min(cap, c * (i+1)^(-1/(gamma-1))), c chosen so
 *     that the expected degrees sum to m (Vose alias tables).
 * Edges are made distinct by rejection: candidate k is kept iff it is the
 * first occurrence of its (u, v) pair, and the graph is the first m distinct
 * candidates in candidate order. A concurrent hash set records, per pair, the
 * smallest candidate index that produced it, so the result does not depend on
 * the number of threads. Vertex ids are then permuted at random on each side
 * so that id order carries no degree information.
 *
 * Signs (per output edge i):
 *   - iid:  +1 with probability p_plus, else -1.
 *   - camp: each vertex gets a camp bit; +1 w.p. p_camp if the endpoints share
 *           a camp, else -1 w.p. p_camp.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define PHI 0x9E3779B97F4A7C15ULL

static inline uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
/* Stream key: a distinct SplitMix64 state per (seed, stream). */
static inline uint64_t sm64_key(uint64_t seed, uint64_t stream) {
  return sm64_mix(seed * PHI + sm64_mix(stream + 0x5851F42D4C957F2DULL));
}
/* k-th output of the stream (k >= 0). */
static inline uint64_t sm64_at(uint64_t key, uint64_t k) { return sm64_mix(key + (k + 1) * PHI); }
static inline double u01(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }
static inline uint64_t below(uint64_t x, uint64_t n) {
  return (uint64_t)(((unsigned __int128)x * (unsigned __int128)n) >> 64);
}

enum { ST_U_IDX = 1, ST_U_COIN, ST_V_IDX, ST_V_COIN, ST_PERM_U, ST_PERM_V, ST_SIGN, ST_CAMP_U, ST_CAMP_V };

/* Exported for tests: the k-th output of a SplitMix64 sequence started at
 * state x (identical to calling the sequential generator k+1 times). */
uint64_t synth_splitmix_raw(uint64_t x, uint64_t k) { return sm64_at(x, k); }

/* Exported for tests: the raw generator. */
uint64_t synth_splitmix_at(uint64_t seed, uint64_t stream, uint64_t k) {
  return sm64_at(sm64_key(seed, stream), k);
}

/* ------------------------------------------------------------------ */
/* Expected degrees and alias tables                                    */
/* ------------------------------------------------------------------ */
/* Expected degrees of a Chung-Lu side, sorted descending, capped at cap and
 * summing to m (when feasible). */
int synth_chung_lu_weights(int64_t n, double gamma, double m, double cap, double* d) {
  if (n <= 0) return -1;
  double ex = -1.0 / (gamma - 1.0);
  for (int64_t i = 0; i < n; i++) d[i] = pow((double)(i + 1), ex);
  /* suffix sums of raw weights */
  double* suf = (double*)malloc(sizeof(double) * (size_t)(n + 1));
  if (!suf) return -2;
  suf[n] = 0.0;
  for (int64_t i = n - 1; i >= 0; i--) suf[i] = suf[i + 1] + d[i];
  /* smallest k (number of capped vertices) such that the rest, scaled to
   * carry m - k*cap, stays below cap at vertex k. */
  int64_t k = 0;
  double s = m / suf[0];
  while (k < n && s * d[k] > cap) {
    k++;
    if (k == n) break;
    double rest = m - (double)k * cap;
    s = rest > 0 ? rest / suf[k] : 0.0;
  }
  for (int64_t i = 0; i < n; i++) d[i] = (i < k) ? cap : s * d[i];
  free(suf);
  return 0;
}

typedef struct {
  int64_t n;
  double* prob;
  int32_t* alias;
} alias_t;

static int alias_build(alias_t* a, const double* w, int64_t n) {
  a->n = n;
  a->prob = (double*)malloc(sizeof(double) * (size_t)n);
  a->alias = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* small = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* large = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!a->prob || !a->alias || !small || !large) return -2;
  double tot = 0;
  for (int64_t i = 0; i < n; i++) tot += w[i];
  int64_t ns = 0, nl = 0;
  for (int64_t i = 0; i < n; i++) {
    a->prob[i] = w[i] * (double)n / tot;
    a->alias[i] = (int32_t)i;
    if (a->prob[i] < 1.0) small[ns++] = (int32_t)i; else large[nl++] = (int32_t)i;
  }
  while (ns > 0 && nl > 0) {
    int32_t s = small[--ns], l = large[--nl];
    a->alias[s] = l;
    a->prob[l] = (a->prob[l] + a->prob[s]) - 1.0;
    if (a->prob[l] < 1.0) small[ns++] = l; else large[nl++] = l;
  }
  while (nl > 0) a->prob[large[--nl]] = 1.0;
  while (ns > 0) a->prob[small[--ns]] = 1.0;
  free(small);
  free(large);
  return 0;
}
static void alias_free(alias_t* a) { free(a->prob); free(a->alias); }
static inline int32_t alias_draw(const alias_t* a, uint64_t r_idx, uint64_t r_coin) {
  int64_t i = (int64_t)below(r_idx, (uint64_t)a->n);
  return (u01(r_coin) < a->prob[i]) ? (int32_t)i : a->alias[i];
}

/* ------------------------------------------------------------------ */
/* Candidate edges and the concurrent first-occurrence set              */
/* ------------------------------------------------------------------ */
typedef struct {
  int model; /* 0 uniform, 1 Chung-Lu */
  int32_t n_u, n_v;
  uint64_t k_uidx, k_ucoin, k_vidx, k_vcoin;
  alias_t au, av;
} cand_t;

static inline uint64_t cand_key(const cand_t* c, uint64_t k) {
  uint32_t u, v;
  if (c->model == 0) {
    u = (uint32_t)below(sm64_at(c->k_uidx, k), (uint64_t)c->n_u);
    v = (uint32_t)below(sm64_at(c->k_vidx, k), (uint64_t)c->n_v);
  } else {
    u = (uint32_t)alias_draw(&c->au, sm64_at(c->k_uidx, k), sm64_at(c->k_ucoin, k));
    v = (uint32_t)alias_draw(&c->av, sm64_at(c->k_vidx, k), sm64_at(c->k_vcoin, k));
  }
  return ((uint64_t)u << 32) | v;
}

#define EMPTY_KEY 0xFFFFFFFFFFFFFFFFULL
typedef struct {
  uint64_t mask;
  uint64_t* keys;
  uint64_t* first; /* smallest candidate index per key */
} hset_t;

/* Insert key seen at candidate k; returns 1 if the key is new, 0 if it was
 * present, -1 if the table is full (callers keep it at most half full). */
static inline int hset_insert(hset_t* h, uint64_t key, uint64_t k) {
  uint64_t i = sm64_mix(key) & h->mask;
  for (uint64_t probe = 0; probe <= h->mask; probe++) {
    uint64_t cur = __atomic_load_n(&h->keys[i], __ATOMIC_RELAXED);
    if (cur == EMPTY_KEY) {
      uint64_t exp = EMPTY_KEY;
      if (__atomic_compare_exchange_n(&h->keys[i], &exp, key, 0, __ATOMIC_ACQ_REL, __ATOMIC_RELAXED)) {
        /* slot claimed: lower the recorded first index to k */
        uint64_t f = __atomic_load_n(&h->first[i], __ATOMIC_RELAXED);
        while (k < f && !__atomic_compare_exchange_n(&h->first[i], &f, k, 1, __ATOMIC_ACQ_REL, __ATOMIC_RELAXED)) {}
        return 1;
      }
      cur = exp;
    }
    if (cur == key) {
      uint64_t f = __atomic_load_n(&h->first[i], __ATOMIC_RELAXED);
      while (k < f && !__atomic_compare_exchange_n(&h->first[i], &f, k, 1, __ATOMIC_ACQ_REL, __ATOMIC_RELAXED)) {}
      return 0;
    }
    i = (i + 1) & h->mask;
  }
  return -1;
}

typedef struct {
  const cand_t* c;
  hset_t* h;
  uint64_t k0, k1;
  int64_t fresh;
} ins_job_t;

static void* ins_worker(void* p) {
  ins_job_t* j = (ins_job_t*)p;
  int64_t fresh = 0;
  for (uint64_t k = j->k0; k < j->k1; k++) {
    const int r = hset_insert(j->h, cand_key(j->c, k), k);
    if (r < 0) {
      j->fresh = -1;
      return NULL;
    }
    fresh += r;
  }
  j->fresh = fresh;
  return NULL;
}

typedef struct {
  const hset_t* h;
  uint8_t* flag;
  uint64_t s0, s1;
} flag_job_t;
static void* flag_worker(void* p) {
  flag_job_t* j = (flag_job_t*)p;
  for (uint64_t i = j->s0; i < j->s1; i++)
    if (j->h->keys[i] != EMPTY_KEY) j->flag[j->h->first[i]] = 1;
  return NULL;
}

typedef struct {
  const cand_t* c;
  const uint8_t* flag;
  uint64_t k0, k1;
  int64_t out0; /* first output position of this range */
  int64_t cnt;
  const int32_t* perm_u;
  const int32_t* perm_v;
  int32_t* u;
  int32_t* v;
} emit_job_t;
static void* count_worker(void* p) {
  emit_job_t* j = (emit_job_t*)p;
  int64_t c = 0;
  for (uint64_t k = j->k0; k < j->k1; k++) c += j->flag[k];
  j->cnt = c;
  return NULL;
}
static void* emit_worker(void* p) {
  emit_job_t* j = (emit_job_t*)p;
  int64_t o = j->out0;
  for (uint64_t k = j->k0; k < j->k1; k++) {
    if (!j->flag[k]) continue;
    uint64_t key = cand_key(j->c, k);
    j->u[o] = j->perm_u[(uint32_t)(key >> 32)];
    j->v[o] = j->perm_v[(uint32_t)(key & 0xFFFFFFFFu)];
    o++;
  }
  return NULL;
}

static void run_jobs(void* (*fn)(void*), void* jobs, size_t job_size, int nt) {
  pthread_t th[256];
  if (nt == 1) { fn(jobs); return; }
  for (int t = 0; t < nt; t++) pthread_create(&th[t], NULL, fn, (char*)jobs + (size_t)t * job_size);
  for (int t = 0; t < nt; t++) pthread_join(th[t], NULL);
}

static void fisher_yates(int32_t* p, int32_t n, uint64_t key) {
  for (int32_t i = 0; i < n; i++) p[i] = i;
  for (int32_t i = n - 1; i > 0; i--) {
    int32_t j = (int32_t)below(sm64_at(key, (uint64_t)i), (uint64_t)i + 1);
    int32_t t = p[i]; p[i] = p[j]; p[j] = t;
  }
}

/*
 * Generate one graph. Returns 0 on success, negative on error:
 *   -1 bad arguments (including m > n_u*n_v), -2 out of memory,
 *   -3 the candidate stream did not reach m distinct edges, -4 the
 *   first-occurrence set filled up (an internal sizing error).
 * sign_model: 0 = iid (p_plus), 1 = camp (p_camp).
 */
int synth_graph(uint64_t seed, int model, int32_t n_u, int32_t n_v, int64_t m, double gamma_u, double gamma_v,
                double cap_u, double cap_v, int sign_model, double p_plus, double p_camp, int threads,
                int32_t* u_out, int32_t* v_out, int8_t* s_out) {
  if (n_u <= 0 || n_v <= 0 || m < 0 || (double)m > (double)n_u * (double)n_v) return -1;
  if (m == 0) return 0;
  if (threads < 1) threads = 1;
  if (threads > 256) threads = 256;
  cand_t c;
  memset(&c, 0, sizeof(c));
  c.model = model;
  c.n_u = n_u;
  c.n_v = n_v;
  c.k_uidx = sm64_key(seed, ST_U_IDX);
  c.k_ucoin = sm64_key(seed, ST_U_COIN);
  c.k_vidx = sm64_key(seed, ST_V_IDX);
  c.k_vcoin = sm64_key(seed, ST_V_COIN);
  if (model == 1) {
    double* w = (double*)malloc(sizeof(double) * (size_t)(n_u > n_v ? n_u : n_v));
    if (!w) return -2;
    synth_chung_lu_weights(n_u, gamma_u, (double)m, cap_u, w);
    if (alias_build(&c.au, w, n_u)) { free(w); return -2; }
    synth_chung_lu_weights(n_v, gamma_v, (double)m, cap_v, w);
    if (alias_build(&c.av, w, n_v)) { free(w); return -2; }
    free(w);
  }
  int rc = 0;
  /* hash set sized for ~50% load at m keys */
  uint64_t cap = 1024;
  while (cap < (uint64_t)(2 * m + 16)) cap <<= 1;
  hset_t h;
  h.mask = cap - 1;
  h.keys = (uint64_t*)malloc(sizeof(uint64_t) * cap);
  h.first = (uint64_t*)malloc(sizeof(uint64_t) * cap);
  uint8_t* flag = NULL;
  int32_t* perm_u = NULL;
  int32_t* perm_v = NULL;
  if (!h.keys || !h.first) { rc = -2; goto done; }
  memset(h.keys, 0xFF, sizeof(uint64_t) * cap);
  memset(h.first, 0xFF, sizeof(uint64_t) * cap);

  /* Insert candidates in growing windows until m distinct pairs exist. */
  int64_t distinct = 0;
  uint64_t kdone = 0;
  uint64_t kmax = (uint64_t)m * 64 + 4096;
  while (distinct < m) {
    uint64_t need = (uint64_t)(m - distinct);
    uint64_t win = need + need / 8 + 1024;
    /* a window adds at most `win` keys: keep the set at most half full */
    const uint64_t room = (h.mask + 1) / 2 - (uint64_t)distinct;
    if (win > room) win = room;
    if (kdone + win > kmax) win = kmax - kdone;
    if (win == 0) { rc = -3; goto done; }
    ins_job_t jobs[256];
    for (int t = 0; t < threads; t++) {
      jobs[t].c = &c;
      jobs[t].h = &h;
      jobs[t].k0 = kdone + win * (uint64_t)t / (uint64_t)threads;
      jobs[t].k1 = kdone + win * (uint64_t)(t + 1) / (uint64_t)threads;
      jobs[t].fresh = 0;
    }
    run_jobs(ins_worker, jobs, sizeof(ins_job_t), threads);
    for (int t = 0; t < threads; t++) {
      if (jobs[t].fresh < 0) { rc = -4; goto done; }
      distinct += jobs[t].fresh;
    }
    kdone += win;
  }
  /* flag[k] = 1 iff candidate k is the first occurrence of its pair */
  flag = (uint8_t*)calloc((size_t)kdone, 1);
  if (!flag) { rc = -2; goto done; }
  {
    flag_job_t fj[256];
    for (int t = 0; t < threads; t++) {
      fj[t].h = &h;
      fj[t].flag = flag;
      fj[t].s0 = cap * (uint64_t)t / (uint64_t)threads;
      fj[t].s1 = cap * (uint64_t)(t + 1) / (uint64_t)threads;
    }
    run_jobs(flag_worker, fj, sizeof(flag_job_t), threads);
  }
  /* keep the first m flagged candidates: find the cut-off index */
  {
    int64_t seen = 0;
    uint64_t kcut = kdone;
    for (uint64_t k = 0; k < kdone; k++) {
      seen += flag[k];
      if (seen == m) { kcut = k + 1; break; }
    }
    if (m == 0) kcut = 0;
    perm_u = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_u);
    perm_v = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_v);
    if (!perm_u || !perm_v) { rc = -2; goto done; }
    fisher_yates(perm_u, n_u, sm64_key(seed, ST_PERM_U));
    fisher_yates(perm_v, n_v, sm64_key(seed, ST_PERM_V));
    emit_job_t ej[256];
    for (int t = 0; t < threads; t++) {
      ej[t].c = &c;
      ej[t].flag = flag;
      ej[t].k0 = kcut * (uint64_t)t / (uint64_t)threads;
      ej[t].k1 = kcut * (uint64_t)(t + 1) / (uint64_t)threads;
      ej[t].perm_u = perm_u;
      ej[t].perm_v = perm_v;
      ej[t].u = u_out;
      ej[t].v = v_out;
    }
    run_jobs(count_worker, ej, sizeof(emit_job_t), threads);
    int64_t off = 0;
    for (int t = 0; t < threads; t++) { ej[t].out0 = off; off += ej[t].cnt; }
    run_jobs(emit_worker, ej, sizeof(emit_job_t), threads);
  }
  /* signs */
  {
    uint64_t ks = sm64_key(seed, ST_SIGN);
    if (sign_model == 0) {
      for (int64_t i = 0; i < m; i++) s_out[i] = (u01(sm64_at(ks, (uint64_t)i)) < p_plus) ? 1 : -1;
    } else {
      uint64_t kcu = sm64_key(seed, ST_CAMP_U), kcv = sm64_key(seed, ST_CAMP_V);
      for (int64_t i = 0; i < m; i++) {
        int cu = (int)(sm64_at(kcu, (uint64_t)u_out[i]) >> 63);
        int cv = (int)(sm64_at(kcv, (uint64_t)v_out[i]) >> 63);
        int agree = u01(sm64_at(ks, (uint64_t)i)) < p_camp;
        int pos = (cu == cv) ? agree : !agree;
        s_out[i] = pos ? 1 : -1;
      }
    }
  }
done:
  if (model == 1) { alias_free(&c.au); alias_free(&c.av); }
  free(h.keys);
  free(h.first);
  free(flag);
  free(perm_u);
  free(perm_v);
  return rc;
}

/* Batch-form sizes for graph g: |U|, |V| log-uniform in [lo_n, hi_n],
 * m log-uniform in [lo_m, hi_m] capped at |U||V|/2. */
void synth_batch_sizes(uint64_t seed, int64_t g, int32_t lo_n, int32_t hi_n, int64_t lo_m, int64_t hi_m,
                       int32_t* n_u, int32_t* n_v, int64_t* m) {
  uint64_t key = sm64_key(seed, 0x1000 + (uint64_t)g);
  double a = log((double)lo_n), b = log((double)hi_n);
  double x = exp(a + (b - a) * u01(sm64_at(key, 0)));
  double y = exp(a + (b - a) * u01(sm64_at(key, 1)));
  double c = log((double)lo_m), d = log((double)hi_m);
  double z = exp(c + (d - c) * u01(sm64_at(key, 2)));
  int32_t nu = (int32_t)llround(x), nv = (int32_t)llround(y);
  int64_t mm = (int64_t)llround(z);
  int64_t mcap = ((int64_t)nu * (int64_t)nv) / 2;
  if (mm > mcap) mm = mcap;
  *n_u = nu;
  *n_v = nv;
  *m = mm;
}
