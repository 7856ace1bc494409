/*
 * ORACLE - test infrastructure only.
 *
 * A plain, slow CPU statement of what exact range search by adaptive group
 * testing computes (Shah, Mittal, Rajwade, "Group Testing for Accurate and
 * Efficient Range-Based Near Neighbor Search for Plagiarism Detection").
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load this library.  It shares no code with the GPU library.
 *
 * Two independent answers to the same question:
 *
 *  orc_brute_force  - the definition (Sec. 1 and Sec. 2): the neighbours of q
 *                     are { i : q.f_i >= rho }.  Every product of two FP32
 *                     values is exact in FP64 and the FP64 sum of d of them is
 *                     off by at most d * 2^-53 * q.f_i, so with the input
 *                     margin of 1e-5 the decision is exact.
 *
 *  orc_alg1         - Algorithm 1 (iterative binary splitting) in the paper's
 *                     order: FP64 cumulative sums (Eq. 1), a stack of
 *                     {si, ei, sim} triples, the right half tested, the left
 *                     half's score taken as sim - rsim, floor-left split,
 *                     ">= rho" everywhere, 1-based indices as printed.  It also
 *                     counts dot products per query in the paper's convention
 *                     (the root test, then one per split), which is what
 *                     Table 3 reports.
 *
 * orc_alg1 additionally carries a rigorous bound on the FP64 rounding error
 * of every score it derives (prefix sums of up to N terms, the difference of
 * two of them, the dot product, and the subtractions of Algorithm 1; the
 * prefix sums' errors enter a score only through its pool's two ends, see
 * pool_dot).  A
 * neighbour flag raised or withheld with |sim - rho| inside that bound, or a
 * pool pruned while its exact score could still reach rho + margin (the
 * least score a neighbour can have under the input margin), is counted as
 * "ambiguous"; tests require zero.
 *
 * orc_alg1_scores runs the same traversal on scalar scores (each pool scores
 * the sum of its members' scores), the model behind Sec. 5's count analysis.
 *
 * orc_maxpool is binary splitting with pools formed by element-wise maximum
 * (Sec. 2, pooling by maximum): Algorithm 1's splitting tree, both halves of
 * every kept pool tested, the same exact sets.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAX_ROUNDS 64

typedef struct {
  int64_t B;
  int64_t *count;      /* neighbours per query */
  int32_t **ids;       /* per query, ascending 0-based database ids */
  int64_t *tests;      /* dot products per query (paper convention) */
  int64_t *ambiguous;  /* decisions inside the rounding bound */
  int64_t rounds[MAX_ROUNDS]; /* tests per tree depth, summed over queries */
  double seconds;
} orc_result;

static double now_s(void) {
  struct timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

static orc_result *new_result(int64_t B) {
  orc_result *r = (orc_result *)calloc(1, sizeof(orc_result));
  r->B = B;
  r->count = (int64_t *)calloc((size_t)B + 1, sizeof(int64_t));
  r->ids = (int32_t **)calloc((size_t)B + 1, sizeof(int32_t *));
  r->tests = (int64_t *)calloc((size_t)B + 1, sizeof(int64_t));
  r->ambiguous = (int64_t *)calloc((size_t)B + 1, sizeof(int64_t));
  return r;
}

typedef struct {
  int32_t *v;
  int64_t n, cap;
} ivec;

static void ivec_push(ivec *a, int32_t x) {
  if (a->n == a->cap) {
    a->cap = a->cap ? 2 * a->cap : 64;
    a->v = (int32_t *)realloc(a->v, sizeof(int32_t) * (size_t)a->cap);
  }
  a->v[a->n++] = x;
}

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

static void set_threads(int threads) {
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#else
  (void)threads;
#endif
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ---------------------------------------------------------------------- */
/* The definition: sim(q, f_i) = q^t f_i >= rho (Sec. 1, Sec. 2).         */
/* ---------------------------------------------------------------------- */
orc_result *orc_brute_force(const float *F, int64_t N, int d, const float *Q,
                            int64_t B, const float *rho, double margin,
                            int threads) {
  orc_result *res = new_result(B);
  double t0 = now_s();
  set_threads(threads);
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t q = 0; q < B; ++q) {
    const float *qv = Q + (size_t)q * (size_t)d;
    const double r = (double)rho[q];
    ivec out = {0, 0, 0};
    int64_t amb = 0;
    for (int64_t i = 0; i < N; ++i) {
      const float *f = F + (size_t)i * (size_t)d;
      double s = 0.0;
      for (int j = 0; j < d; ++j) s += (double)qv[j] * (double)f[j];
      if (s >= r) ivec_push(&out, (int32_t)i);
      if (fabs(s - r) < margin) ++amb;
    }
    res->count[q] = out.n;
    res->ids[q] = out.v;
    res->tests[q] = N;
    res->ambiguous[q] = amb;
  }
  res->seconds = now_s() - t0;
  return res;
}

/* ---------------------------------------------------------------------- */
/* Algorithm 1 over FP64 cumulative sums (Eq. 1).                          */
/* ---------------------------------------------------------------------- */
typedef struct {
  int64_t si, ei; /* 1-based, inclusive */
  double sim;     /* q^t (pool) */
  double ta, tb;  /* error terms of the running sums at the pool's ends si - 1 and ei */
  double rr;      /* accumulated rounding of the differences, dots and subtractions */
  int depth;      /* round of binary splitting the pool belongs to */
} triple;

/* The rounding bound.  Let E_k be the exact sum of the first k FP32 rows and
 * Fs_k the FP64 running sum.  All terms are >= 0, so elementwise
 * |Fs_k - E_k| <= gamma_k E_k and, with q >= 0,
 *   |q^t (Fs_k - E_k)| <= T_k = 1.01 (k + 1) 2^-53 q^t Fs_k.
 * A direct score q^t (Fs_b - Fs_a) (pool_dot) differs from the exact
 * q^t (E_b - E_a) by the two ends' terms, T_b + T_a, plus the rounding of the
 * element differences and of the d-term dot product, at most
 * 1.01 (d + 3) 2^-53 sum_j q_j |Fs_b[j] - Fs_a[j]|.
 * A left half scored by subtraction, sim(parent) - sim(right half), shares
 * the parent's end ei with the right half: the terms q^t (Fs_ei - E_ei) of
 * the two cancel exactly, so its error is again the running-sum terms of its
 * own two ends (si - 1 and the split point) plus the roundings accumulated
 * down the run of subtractions (the parent's, the right half's, and
 * 2^-53 |lsim| for the subtraction itself).  The running sums' own errors,
 * the large part at N = 10^6, therefore do not grow along a run of left
 * halves. */
static double pool_dot(const double *Fs, int d, const float *q, int64_t b,
                       int64_t a, double *tb, double *ta, double *rr) {
  const double *hb = Fs + (size_t)b * (size_t)d;
  const double *ha = Fs + (size_t)a * (size_t)d;
  double dot = 0.0, adot = 0.0, qb = 0.0, qa = 0.0;
  for (int j = 0; j < d; ++j) {
    double diff = hb[j] - ha[j];
    dot += (double)q[j] * diff;
    adot += (double)q[j] * fabs(diff);
    qb += (double)q[j] * hb[j];
    qa += (double)q[j] * ha[j];
  }
  const double u = ldexp(1.0, -53);
  *tb = 1.01 * u * (double)(b + 1) * qb;
  *ta = 1.01 * u * (double)(a + 1) * qa;
  *rr = 1.01 * u * (double)(d + 3) * adot;
  return dot;
}

/* The offline index of Eq. 1: Fs[k] = f_1 + ... + f_k in FP64, Fs[0] = 0. */
typedef struct {
  int64_t N;
  int d;
  double *Fs;
} orc_index;

orc_index *orc_index_new(const float *F, int64_t N, int d, int threads) {
  set_threads(threads);
  orc_index *ix = (orc_index *)calloc(1, sizeof(orc_index));
  ix->N = N;
  ix->d = d;
  ix->Fs = (double *)malloc(sizeof(double) * (size_t)(N + 1) * (size_t)d);
  if (!ix->Fs) {
    free(ix);
    return NULL;
  }
  double *Fs = ix->Fs;
  memset(Fs, 0, sizeof(double) * (size_t)d);
  /* columns are independent running sums: parallel over columns */
#pragma omp parallel for schedule(static)
  for (int j = 0; j < d; ++j) {
    double acc = 0.0;
    for (int64_t k = 1; k <= N; ++k) {
      acc += (double)F[(size_t)(k - 1) * (size_t)d + (size_t)j];
      Fs[(size_t)k * (size_t)d + (size_t)j] = acc;
    }
  }
  return ix;
}

void orc_index_free(orc_index *ix) {
  if (!ix) return;
  free(ix->Fs);
  free(ix);
}

orc_result *orc_index_query(const orc_index *ix, const float *Q, int64_t B,
                            const float *rho, double margin, int threads) {
  orc_result *res = new_result(B);
  set_threads(threads);
  const int64_t N = ix->N;
  const int d = ix->d;
  const double *Fs = ix->Fs;
  int64_t rounds[MAX_ROUNDS];
  memset(rounds, 0, sizeof(rounds));
  double t0 = now_s();
  #pragma omp parallel
  {
    int64_t my_rounds[MAX_ROUNDS];
    memset(my_rounds, 0, sizeof(my_rounds));
    triple *S = (triple *)malloc(sizeof(triple) * 4 * MAX_ROUNDS);
#pragma omp for schedule(dynamic, 1)
    for (int64_t qi = 0; qi < B; ++qi) {
      const float *q = Q + (size_t)qi * (size_t)d;
      const double r = (double)rho[qi];
      const double u = ldexp(1.0, -53);
      ivec out = {0, 0, 0};
      int64_t tests = 0, amb = 0;
      int top = 0;
      double e;
      /* push {1, N, q^t Fs_N} */
      double tb, ta, rr;
      double s0 = pool_dot(Fs, d, q, N, 0, &tb, &ta, &rr);
      ++tests;
      ++my_rounds[0];
      S[top++] = (triple){1, N, s0, ta, tb, rr, 0};
      while (top > 0) {
        triple t = S[--top];
        const double terr = t.ta + t.tb + t.rr; /* bound on |t.sim - exact| */
        if (t.sim >= r) {
          int64_t n = t.ei - t.si + 1;
          if (n > 2) {
            int64_t h = n / 2;
            /* right half [si + h, ei]: q^t (Fs_ei - Fs_{si+h-1}) */
            double rtb, rta, rrr;
            double rsim = pool_dot(Fs, d, q, t.ei, t.si + h - 1, &rtb, &rta, &rrr);
            ++tests;
            if (t.depth + 1 < MAX_ROUNDS) ++my_rounds[t.depth + 1];
            double lsim = t.sim - rsim;
            S[top++] = (triple){t.si + h, t.ei, rsim, rta, rtb, rrr, t.depth + 1};
            S[top++] = (triple){t.si, t.si + h - 1, lsim, t.ta, rta,
                                t.rr + rrr + u * fabs(lsim), t.depth + 1};
          } else if (n == 2) {
            double rtb, rta, rrr;
            double rsim = pool_dot(Fs, d, q, t.ei, t.si, &rtb, &rta, &rrr);
            ++tests;
            if (t.depth + 1 < MAX_ROUNDS) ++my_rounds[t.depth + 1];
            double lsim = t.sim - rsim;
            double er = rta + rtb + rrr;
            double el = t.ta + rta + t.rr + rrr + u * fabs(lsim);
            if (rsim >= r) ivec_push(&out, (int32_t)(t.ei - 1));
            if (fabs(rsim - r) <= er) ++amb;
            if (lsim >= r) ivec_push(&out, (int32_t)(t.si - 1));
            if (fabs(lsim - r) <= el) ++amb;
          } else {
            /* a single item whose (derived) score passed */
            ivec_push(&out, (int32_t)(t.si - 1));
            if (fabs(t.sim - r) <= terr) ++amb;
          }
        } else if (t.ei == t.si) {
          if (fabs(t.sim - r) <= terr) ++amb; /* an item withheld inside the bound */
        } else if (t.sim + terr >= r + margin) {
          /* a pruned pool could hold a neighbour only if its exact score
           * reached rho + margin (all member scores are >= 0) */
          ++amb;
        }
      }
      if (out.n > 1) qsort(out.v, (size_t)out.n, sizeof(int32_t), cmp_i32);
      res->count[qi] = out.n;
      res->ids[qi] = out.v;
      res->tests[qi] = tests;
      res->ambiguous[qi] = amb;
    }
#pragma omp critical
    for (int k = 0; k < MAX_ROUNDS; ++k) rounds[k] += my_rounds[k];
    free(S);
  }
  res->seconds = now_s() - t0;
  memcpy(res->rounds, rounds, sizeof(rounds));
  return res;
}

orc_result *orc_alg1(const float *F, int64_t N, int d, const float *Q,
                     int64_t B, const float *rho, double margin, int threads) {
  orc_index *ix = orc_index_new(F, N, d, threads);
  if (!ix) return new_result(B);
  orc_result *res = orc_index_query(ix, Q, B, rho, margin, threads);
  orc_index_free(ix);
  return res;
}


/* Algorithm 1 on scalar scores x_1..x_N (pool score = sum of members'):
 * returns the number of dot products the traversal would compute. */
int64_t orc_alg1_scores(const double *x, int64_t N, double rho,
                        int64_t *rounds_out) {
  double *cs = (double *)malloc(sizeof(double) * (size_t)(N + 1));
  cs[0] = 0.0;
  for (int64_t k = 1; k <= N; ++k) cs[k] = cs[k - 1] + x[k - 1];
  triple *S = (triple *)malloc(sizeof(triple) * 4 * MAX_ROUNDS);
  int top = 0;
  int64_t tests = 1;
  if (rounds_out) rounds_out[0] += 1;
  S[top++] = (triple){1, N, cs[N], 0.0, 0};
  while (top > 0) {
    triple t = S[--top];
    if (t.sim < rho) continue;
    int64_t n = t.ei - t.si + 1;
    if (n > 2) {
      int64_t h = n / 2;
      double rsim = cs[t.ei] - cs[t.si + h - 1];
      ++tests;
      if (rounds_out && t.depth + 1 < MAX_ROUNDS) rounds_out[t.depth + 1] += 1;
      S[top++] = (triple){t.si + h, t.ei, rsim, 0.0, t.depth + 1};
      S[top++] = (triple){t.si, t.si + h - 1, t.sim - rsim, 0.0, t.depth + 1};
    } else if (n == 2) {
      ++tests;
      if (rounds_out && t.depth + 1 < MAX_ROUNDS) rounds_out[t.depth + 1] += 1;
    }
  }
  free(S);
  free(cs);
  return tests;
}

/* ---------------------------------------------------------------------- */
/* Binary splitting with pools formed by element-wise maximum (Sec. 2,      */
/* pooling by maximum).                                                     */
/* ---------------------------------------------------------------------- */
/* The splitting tree is Algorithm 1's (a pool of n items splits into a left
 * half of floor(n/2) items and a right half of the rest).  A pool's vector
 * is the element-wise maximum of its members' FP32 rows, which is exact, and
 * for non-negative q its score q.y is at least every member's score, so a
 * pool scoring below rho holds no neighbour.  A parent's score says nothing
 * exact about its children's, so both halves of a kept pool are tested:
 * the count is the root test plus two per split. */
typedef struct {
  int64_t N;
  int d;
  int64_t n_nodes;
  float *vec;             /* n_nodes x d pool vectors */
  int64_t *left, *right;  /* child node ids (-1 at an item) */
  int64_t *first;         /* first item of the node, 0-based */
} orc_maxindex;

static int64_t maxnode(orc_maxindex *ix, const float *F, int64_t si, int64_t ei, int64_t *next) {
  const int d = ix->d;
  const int64_t id = (*next)++;
  float *v = ix->vec + (size_t)id * (size_t)d;
  ix->first[id] = si;
  if (si == ei) {
    memcpy(v, F + (size_t)si * (size_t)d, sizeof(float) * (size_t)d);
    ix->left[id] = ix->right[id] = -1;
    return id;
  }
  const int64_t h = (ei - si + 1) / 2;
  const int64_t l = maxnode(ix, F, si, si + h - 1, next);
  const int64_t r = maxnode(ix, F, si + h, ei, next);
  ix->left[id] = l;
  ix->right[id] = r;
  const float *a = ix->vec + (size_t)l * (size_t)d, *b = ix->vec + (size_t)r * (size_t)d;
  for (int j = 0; j < d; ++j) v[j] = a[j] > b[j] ? a[j] : b[j];
  return id;
}

orc_maxindex *orc_maxindex_new(const float *F, int64_t N, int d) {
  orc_maxindex *ix = (orc_maxindex *)calloc(1, sizeof(orc_maxindex));
  ix->N = N;
  ix->d = d;
  const int64_t nodes = 2 * N - 1;
  ix->vec = (float *)malloc(sizeof(float) * (size_t)nodes * (size_t)d);
  ix->left = (int64_t *)malloc(sizeof(int64_t) * (size_t)nodes);
  ix->right = (int64_t *)malloc(sizeof(int64_t) * (size_t)nodes);
  ix->first = (int64_t *)malloc(sizeof(int64_t) * (size_t)nodes);
  if (!ix->vec || !ix->left || !ix->right || !ix->first) {
    free(ix->vec); free(ix->left); free(ix->right); free(ix->first); free(ix);
    return NULL;
  }
  int64_t next = 0;
  maxnode(ix, F, 0, N - 1, &next);
  ix->n_nodes = next;
  return ix;
}

void orc_maxindex_free(orc_maxindex *ix) {
  if (!ix) return;
  free(ix->vec); free(ix->left); free(ix->right); free(ix->first);
  free(ix);
}

/* FP64 dot of q with node vector v and a bound on its rounding error (each
 * product of FP32 values is exact; d additions). */
static double node_dot(const float *v, const float *q, int d, double *err) {
  double s = 0.0;
  for (int j = 0; j < d; ++j) s += (double)q[j] * (double)v[j];
  *err = 1.01 * (double)(d + 1) * ldexp(1.0, -53) * s;
  return s;
}

orc_result *orc_maxindex_query(const orc_maxindex *ix, const float *Q, int64_t B,
                               const float *rho, double margin, int threads) {
  orc_result *res = new_result(B);
  set_threads(threads);
  const int d = ix->d;
  int64_t rounds[MAX_ROUNDS];
  memset(rounds, 0, sizeof(rounds));
  double t0 = now_s();
  #pragma omp parallel
  {
    int64_t my_rounds[MAX_ROUNDS];
    memset(my_rounds, 0, sizeof(my_rounds));
    int64_t *S = (int64_t *)malloc(sizeof(int64_t) * 2 * 4 * MAX_ROUNDS);
#pragma omp for schedule(dynamic, 1)
    for (int64_t qi = 0; qi < B; ++qi) {
      const float *q = Q + (size_t)qi * (size_t)d;
      const double r = (double)rho[qi];
      ivec out = {0, 0, 0};
      int64_t tests = 0, amb = 0;
      int top = 0;
      /* stack of (node, depth); a node is tested when it is popped */
      S[top++] = 0;
      S[top++] = 0;
      while (top > 0) {
        const int depth = (int)S[--top];
        const int64_t node = S[--top];
        double e;
        const double s = node_dot(ix->vec + (size_t)node * (size_t)d, q, d, &e);
        ++tests;
        if (depth < MAX_ROUNDS) ++my_rounds[depth];
        const int is_item = ix->left[node] < 0;
        if (s >= r) {
          if (is_item) {
            ivec_push(&out, (int32_t)ix->first[node]);
            if (s - r <= e) ++amb;
          } else {
            S[top++] = ix->right[node];
            S[top++] = depth + 1;
            S[top++] = ix->left[node];
            S[top++] = depth + 1;
          }
        } else if (is_item ? (r - s <= e) : (s + e >= r)) {
          ++amb; /* a decision inside the rounding bound */
        }
      }
      if (out.n > 1) qsort(out.v, (size_t)out.n, sizeof(int32_t), cmp_i32);
      res->count[qi] = out.n;
      res->ids[qi] = out.v;
      res->tests[qi] = tests;
      res->ambiguous[qi] = amb;
    }
#pragma omp critical
    for (int k = 0; k < MAX_ROUNDS; ++k) rounds[k] += my_rounds[k];
    free(S);
  }
  res->seconds = now_s() - t0;
  memcpy(res->rounds, rounds, sizeof(rounds));
  (void)margin;
  return res;
}

orc_result *orc_maxpool(const float *F, int64_t N, int d, const float *Q, int64_t B,
                        const float *rho, double margin, int threads) {
  orc_maxindex *ix = orc_maxindex_new(F, N, d);
  if (!ix) return new_result(B);
  orc_result *res = orc_maxindex_query(ix, Q, B, rho, margin, threads);
  orc_maxindex_free(ix);
  return res;
}

/* Pool vector of the node covering items [first, first + n) in the max
 * splitting tree, written to out (d floats); 0 if no node covers exactly
 * that range.  Lets the tests compare GPU rows with the oracle's. */
int orc_maxindex_vec(const orc_maxindex *ix, int64_t first, int64_t n, float *out) {
  int64_t node = 0, si = 0, ei = ix->N - 1;
  while (1) {
    if (si == first && ei - si + 1 == n) {
      memcpy(out, ix->vec + (size_t)node * (size_t)ix->d, sizeof(float) * (size_t)ix->d);
      return 1;
    }
    if (ix->left[node] < 0) return 0;
    const int64_t h = (ei - si + 1) / 2;
    if (first < si + h) {
      node = ix->left[node];
      ei = si + h - 1;
    } else {
      node = ix->right[node];
      si = si + h;
    }
  }
}

/* ---------------------------------------------------------------------- */
int64_t orc_total(const orc_result *r) {
  int64_t t = 0;
  for (int64_t q = 0; q < r->B; ++q) t += r->count[q];
  return t;
}

double orc_seconds(const orc_result *r) { return r->seconds; }

void orc_copy(const orc_result *r, int64_t *offsets, int32_t *ids,
              int64_t *tests, int64_t *ambiguous, int64_t *rounds) {
  int64_t o = 0;
  for (int64_t q = 0; q < r->B; ++q) {
    offsets[q] = o;
    if (r->count[q]) memcpy(ids + o, r->ids[q], sizeof(int32_t) * (size_t)r->count[q]);
    o += r->count[q];
    if (tests) tests[q] = r->tests[q];
    if (ambiguous) ambiguous[q] = r->ambiguous[q];
  }
  offsets[r->B] = o;
  if (rounds) memcpy(rounds, r->rounds, sizeof(r->rounds));
}

void orc_free(orc_result *r) {
  if (!r) return;
  for (int64_t q = 0; q < r->B; ++q) free(r->ids[q]);
  free(r->ids);
  free(r->count);
  free(r->tests);
  free(r->ambiguous);
  free(r);
}
